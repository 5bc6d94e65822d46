"""The C-ABI library builds, loads and exports every symbol include/*.h declares;
argument validation and allocation failure are reported without a GPU."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    from paper_1510_04068_gb300 import build, sp2
    build.build()
    return sp2.load()


def _declared():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        src = h.read_text()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        for m in re.finditer(r"\b(sp2_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    from paper_1510_04068_gb300 import sp2
    declared = _declared()
    assert len(declared) >= 25
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(sp2.EXPORTED), declared ^ set(sp2.EXPORTED)


def test_config_validation_without_gpu(lib):
    from paper_1510_04068_gb300 import sp2
    cfg = sp2.sp2_config()
    lib.sp2_config_default(ctypes.byref(cfg))
    assert (cfg.order, cfg.precision, cfg.with_nn) == (4, sp2.SP2_MIXED, 1)
    ctx = ctypes.c_void_p()
    for field, bad in (("order", 5), ("precision", 7), ("n_max", 0), ("n_max", -3),
                       ("eps2", -1.0), ("eps2", float("nan")), ("with_nn", 2)):
        c = sp2.sp2_config()
        lib.sp2_config_default(ctypes.byref(c))
        c.n_max = 16
        setattr(c, field, bad)
        assert lib.sp2_open(ctypes.byref(ctx), ctypes.byref(c)) == -1, field
        assert not ctx.value
    assert lib.sp2_open(None, ctypes.byref(cfg)) == -1
    assert lib.sp2_close(None) == 0


def test_allocation_failure_is_reported(lib):
    """An allocator that fails (host-side fault injection) gives SP2_ERR_NOMEM,
    and every successful allocation is released again."""
    from paper_1510_04068_gb300 import sp2
    live = []

    @sp2.ALLOC_FN
    def alloc(nbytes, user):
        if len(live) >= 3:
            return None
        buf = ctypes.create_string_buffer(int(nbytes))
        live.append(buf)
        return ctypes.addressof(buf)

    freed = []

    @sp2.FREE_FN
    def free(ptr, user):
        freed.append(ptr)

    cfg = sp2.sp2_config()
    lib.sp2_config_default(ctypes.byref(cfg))
    cfg.n_max = 64
    cfg.alloc, cfg.free = alloc, free
    ctx = ctypes.c_void_p()
    assert lib.sp2_open(ctypes.byref(ctx), ctypes.byref(cfg)) == -3
    assert len(freed) == 3 and not ctx.value
    # an allocator without a matching free is an argument error
    cfg.free = sp2.FREE_FN()
    assert lib.sp2_open(ctypes.byref(ctx), ctypes.byref(cfg)) == -1


def test_status_strings(lib):
    for s in range(0, -9, -1):
        assert lib.sp2_strerror(s)
    assert lib.sp2_kernel_launches(None) == -1


def test_binding_refuses_mixed_host_and_device(lib):
    import numpy as np
    from paper_1510_04068_gb300 import sp2
    with pytest.raises(TypeError):
        sp2._marshal([np.zeros(3), np.zeros(3, np.float32)], [np.float64, np.float64])


C_CLIENT = r"""
#include <stdio.h>
#include "sapporo_gb.h"

/* A plain C99 caller of the ABI: config defaults and argument validation,
   which need no GPU. */
int main(void) {
    sp2_config cfg;
    sp2_ctx *ctx = NULL;
    sp2_config_default(&cfg);
    cfg.n_max = 16;
    cfg.order = 3;
    if (sp2_open(&ctx, &cfg) != SP2_ERR_ARG || ctx != NULL) return 1;
    if (sp2_close(NULL) != SP2_OK) return 2;
    {
        sp2_block_stats st;
        if (sp2_block_run(NULL, 1.0, 0.01, 0.0625, &st) != SP2_ERR_ARG) return 3;
        if (sp2_block_run_h6(NULL, 1.0, 0.01, 0.1, 0.0625, &st) != SP2_ERR_ARG) return 4;
        if (sp2_measure_pipe_peaks(NULL) != SP2_ERR_ARG) return 5;
    }
    printf("%s\n", sp2_strerror(SP2_ERR_RANGE));
    return 0;
}
"""


def test_header_compiles_and_links_as_c(lib, tmp_path):
    """include/sapporo_gb.h is a C header: a C99 client compiles with warnings
    as errors, links against the library and runs the GPU-free calls."""
    import shutil
    import subprocess
    from paper_1510_04068_gb300 import build
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = str(build.LIB.parent)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", f"-I{ROOT / 'include'}",
                        str(src), "-o", str(exe), f"-L{libdir}", "-lsapporo_gb", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert r.stdout.strip()
