/*
 * sp2_oracle.c -- plain, slow, FP64 reference of the direct-summation gravity
 * pass (predictor + softened acceleration / jerk / snap / potential / nearest
 * neighbour).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file; the GPU library never does, and
 * the two share no code.
 *
 * The paper (Sec. 3, "Results") names the quantities -- acceleration, jerk (the
 * first time derivative of the acceleration, needed by 4th-order Hermite),
 * snap for the 6th-order scheme (Sec. 3.5), potential, nearest neighbour id and
 * distance -- and states (Sec. 1) that prediction of the sources happens on the
 * device before the force sum.  It prints no formulas.  The definitions below
 * are the standard ones of the literature the paper relies on (Makino & Aarseth
 * 1992 for 4th order, Nitadori & Makino 2008 for 6th order):
 *
 *   r = x_j - x_i,  v = v_j - v_i,  a = a_j - a_i   (predicted values)
 *   s = (r.r + eps^2)^(-1/2)                         (Plummer softening)
 *   A_ij = m_j s^3 r
 *   alpha = (r.v) s^2
 *   J_ij = m_j s^3 v - 3 alpha A_ij                  (= dA_ij/dt)
 *   beta = (v.v + r.a) s^2 + alpha^2
 *   S_ij = m_j s^3 a - 6 alpha J_ij - 3 beta A_ij    (= dJ_ij/dt)
 *   phi_ij = -m_j s
 *
 * summed in natural j order over every j whose id differs from the sink's id.
 * The nearest neighbour is the j (id differing) with the smallest unsoftened
 * r.r, ties going to the smaller id; with no other particle it is id -1 at
 * distance +infinity.  The scale sums returned with the results are the sums of
 * the absolute values of each term (see sp2o_forces).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared.  No FMA contraction
 * and no fast-math, so every operation rounds exactly as written.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int sp2o_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void sp2o_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * Taylor predictor of the sources to time t (Sec. 2.2, "predict the particles
 * to the new time-step"; the polynomial is the Hermite predictor of Makino &
 * Aarseth 1992 and, for 6th order, of Nitadori & Makino 2008).
 *
 *   dt = t - t_j
 *   order 4:  x_p = x + v dt + a dt^2/2 + j dt^3/6
 *             v_p = v + a dt + j dt^2/2
 *   order 6:  x_p = x + v dt + a dt^2/2 + j dt^3/6 + s dt^4/24
 *             v_p = v + a dt + j dt^2/2 + s dt^3/6
 *             a_p = a + j dt + s dt^2/2
 *
 * The coefficients dt^k / k! are formed as (dt^k) * c_k with c_k the double
 * nearest 1/k!, and every sum is evaluated left to right.  Arrays are n x 3
 * row-major; snap and a_p are used only for order 6.
 */
void sp2o_predict(int64_t n, int order, double t, const double *tj,
                  const double *x, const double *v, const double *a,
                  const double *jk, const double *sn,
                  double *xp, double *vp, double *ap)
{
    const double c2 = 0.5, c3 = 1.0 / 6.0, c4 = 1.0 / 24.0;
    for (int64_t j = 0; j < n; ++j) {
        const double dt = t - tj[j];
        const double dt2 = dt * dt;
        const double dt3 = dt2 * dt;
        const double dt4 = dt3 * dt;
        for (int k = 0; k < 3; ++k) {
            const int64_t q = 3 * j + k;
            if (order == 6) {
                xp[q] = x[q] + v[q] * dt + a[q] * (dt2 * c2) + jk[q] * (dt3 * c3) + sn[q] * (dt4 * c4);
                vp[q] = v[q] + a[q] * dt + jk[q] * (dt2 * c2) + sn[q] * (dt3 * c3);
                ap[q] = a[q] + jk[q] * dt + sn[q] * (dt2 * c2);
            } else {
                xp[q] = x[q] + v[q] * dt + a[q] * (dt2 * c2) + jk[q] * (dt3 * c3);
                vp[q] = v[q] + a[q] * dt + jk[q] * (dt2 * c2);
            }
        }
    }
}

/*
 * Direct sum of the softened interactions of n_j sources on n_i sinks.
 *
 * Sinks:   id_i[n_i], xi/vi/ai [n_i x 3]   (ai only for order 6)
 * Sources: id_j[n_j], mj[n_j], xj/vj/aj [n_j x 3]
 * Outputs: acc, jerk, snap [n_i x 3] (snap only for order 6), pot[n_i],
 *          nn_id[n_i], nn_r2[n_i], and the scale sums
 *            sc_acc  = sum |A_ij|            = sum m s^3 |r|
 *            sc_jerk = sum m s^3 (|v| + 3|alpha||r|)        >= sum |J_ij|
 *            sc_snap = sum m s^3 (|a| + 6|alpha|(|v| + 3|alpha||r|)
 *                                 + 3|beta||r|)            >= sum |S_ij|
 *          against which summation-order and precision differences are judged.
 * Any output pointer may be NULL.
 */
void sp2o_forces(int64_t n_i, const int32_t *id_i, const double *xi, const double *vi,
                 const double *ai,
                 int64_t n_j, const int32_t *id_j, const double *mj, const double *xj,
                 const double *vj, const double *aj,
                 double eps2, int order,
                 double *acc, double *jerk, double *snap, double *pot,
                 int32_t *nn_id, double *nn_r2,
                 double *sc_acc, double *sc_jerk, double *sc_snap)
{
    const int six = (order == 6);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n_i; ++i) {
        double A[3] = {0.0, 0.0, 0.0}, J[3] = {0.0, 0.0, 0.0}, S[3] = {0.0, 0.0, 0.0};
        double P = 0.0, Ah = 0.0, Jh = 0.0, Sh = 0.0;
        double best = INFINITY;
        int32_t best_id = -1;
        const int32_t me = id_i[i];
        for (int64_t j = 0; j < n_j; ++j) {
            if (id_j[j] == me) continue;
            double r[3], v[3], a[3] = {0.0, 0.0, 0.0};
            for (int k = 0; k < 3; ++k) {
                r[k] = xj[3 * j + k] - xi[3 * i + k];
                v[k] = vj[3 * j + k] - vi[3 * i + k];
                if (six) a[k] = aj[3 * j + k] - ai[3 * i + k];
            }
            const double d2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            const double s = 1.0 / sqrt(d2 + eps2);
            const double s2 = s * s;
            const double ms3 = mj[j] * s * s2;
            const double rv = r[0] * v[0] + r[1] * v[1] + r[2] * v[2];
            const double alpha = rv * s2;
            double Aij[3], Jij[3];
            for (int k = 0; k < 3; ++k) {
                Aij[k] = ms3 * r[k];
                Jij[k] = ms3 * v[k] - 3.0 * alpha * Aij[k];
                A[k] += Aij[k];
                J[k] += Jij[k];
            }
            P -= mj[j] * s;
            const double rn = sqrt(d2);
            const double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            Ah += ms3 * rn;
            Jh += ms3 * (vn + 3.0 * fabs(alpha) * rn);
            if (six) {
                const double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
                const double ra = r[0] * a[0] + r[1] * a[1] + r[2] * a[2];
                const double beta = (vv + ra) * s2 + alpha * alpha;
                for (int k = 0; k < 3; ++k)
                    S[k] += ms3 * a[k] - 6.0 * alpha * Jij[k] - 3.0 * beta * Aij[k];
                const double an = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
                Sh += ms3 * (an + 6.0 * fabs(alpha) * (vn + 3.0 * fabs(alpha) * rn)
                             + 3.0 * fabs(beta) * rn);
            }
            if (d2 < best || (d2 == best && id_j[j] < best_id)) {
                best = d2;
                best_id = id_j[j];
            }
        }
        for (int k = 0; k < 3; ++k) {
            if (acc) acc[3 * i + k] = A[k];
            if (jerk) jerk[3 * i + k] = J[k];
            if (snap && six) snap[3 * i + k] = S[k];
        }
        if (pot) pot[i] = P;
        if (nn_id) nn_id[i] = best_id;
        if (nn_r2) nn_r2[i] = best;
        if (sc_acc) sc_acc[i] = Ah;
        if (sc_jerk) sc_jerk[i] = Jh;
        if (sc_snap) sc_snap[i] = Sh;
    }
}

/*
 * Neighbour lists.  The paper (Sec. 1) states that the library can return, for
 * each particle, the list of all particles within a given radius, and Sec. 3
 * uses them as the perturber lists of NBODY4-style integrators.  For sink i
 * (position i of the sink arrays) the neighbours are the sources j whose id
 * differs from the sink's and whose unsoftened r.r is below h2[i] (strictly),
 * r.r formed exactly as in sp2o_forces (left to right, no FMA).
 *   count[i]                 number of neighbours;
 *   ids[i * nb_max + k]      k < min(count[i], nb_max): the neighbour ids in
 *                            ascending order (the nb_max smallest when the
 *                            list overflows).
 */
void sp2o_neighbours(int64_t n_i, const int32_t *id_i, const double *xi, const double *h2,
                     int64_t n_j, const int32_t *id_j, const double *xj,
                     int32_t nb_max, int32_t *count, int32_t *ids)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n_i; ++i) {
        int32_t c = 0;
        int32_t *row = ids + i * (int64_t)nb_max;
        for (int64_t j = 0; j < n_j; ++j) {
            if (id_j[j] == id_i[i]) continue;
            double r[3];
            for (int k = 0; k < 3; ++k) r[k] = xj[3 * j + k] - xi[3 * i + k];
            const double d2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            if (!(d2 < h2[i])) continue;
            /* insert id_j[j] into the sorted row, keeping the nb_max smallest */
            const int32_t v = id_j[j];
            int32_t n = c < nb_max ? c : nb_max;
            if (n == nb_max && v >= row[n - 1]) { ++c; continue; }
            int32_t q = (n == nb_max) ? n - 1 : n;
            while (q > 0 && row[q - 1] > v) { row[q] = row[q - 1]; --q; }
            row[q] = v;
            ++c;
        }
        count[i] = c;
    }
}
