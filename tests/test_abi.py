"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
symbol declared in include/lbcuboid.h, and rejects invalid parameters before any
device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "lbcuboid.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2107_14774_gb300 import _lib
    from paper_2107_14774_gb300.build import LIB
    if not os.path.exists(LIB):
        from paper_2107_14774_gb300.build import build
        build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2107_14774_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _declared_functions()


def test_config_struct_layout_matches_header(lib):
    from paper_2107_14774_gb300._lib import lb_config
    cfg = lb_config()
    lib.lb_config_default(ctypes.byref(cfg), 7, 8, 9, 0.5, 2.0, 0.01)
    assert (cfg.nx, cfg.ny, cfg.nz) == (7, 8, 9)
    assert (cfg.r_y, cfg.r_z, cfg.nu) == (0.5, 2.0, 0.01)
    assert cfg.storage == 1 and cfg.corr == 2 and cfg.wall_mask == 0 and cfg.lid_u == 0.0


@pytest.mark.parametrize("kw,msg", [
    (dict(nx=0), "dimensions"),
    (dict(r_y=-1.0), "aspect"),
    (dict(nu=0.0), "nu"),
    (dict(cs2=0.3), "cs2"),          # >= min(1, r^2, s^2) = 0.25
    (dict(nu=1e-9, cs2=0.0), None),  # valid: omega_nu -> 2 from below
    (dict(storage=9), "storage"),
    (dict(corr=7), "corr"),
    (dict(wall_mask=8), "wall_mask"),
    (dict(lid_u=0.1), "lid"),
])
def test_invalid_parameters_are_rejected_without_a_gpu(lib, kw, msg):
    from paper_2107_14774_gb300._lib import LB_EINVAL, lb_config
    if msg is None:
        pytest.skip("valid configuration: would allocate device memory")
    cfg = lb_config()
    lib.lb_config_default(ctypes.byref(cfg), 8, 8, 8, 1.0, 0.5, 0.01)
    for k, v in kw.items():
        setattr(cfg, k, v)
    ctx = ctypes.c_void_p()
    assert lib.lb_create_ex(ctypes.byref(cfg), ctypes.byref(ctx)) == LB_EINVAL
    assert not ctx.value
    assert msg in lib.lb_last_error().decode()


def test_rates_outside_stability_interval_rejected(lib):
    from paper_2107_14774_gb300._lib import LB_EINVAL
    ctx = ctypes.c_void_p()
    # zeta < 0 selects omega_xi = 1, fine; a negative nu is rejected
    assert lib.lb_create(4, 4, 4, 1.0, 1.0, -0.1, 0.0, ctypes.byref(ctx)) == LB_EINVAL


def test_header_compiles_as_c_and_a_c_caller_links(lib, tmp_path):
    """The boundary is plain C: a C99 program that includes the header, fills a
    configuration, gets LB_EINVAL for a zero-sized lattice and reads the message,
    compiles with -Wall -Werror, links against the library and runs (no GPU needed)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2107_14774_gb300.build import LIB
    src = tmp_path / "caller.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "lbcuboid.h"
int main(void)
{
    lb_config cfg;
    lb_ctx *ctx = NULL;
    lb_config_default(&cfg, 0, 8, 8, 0.5, 1.0, 0.01);
    lb_status st = lb_create_ex(&cfg, &ctx);
    if (st != LB_EINVAL || ctx != NULL) return 1;
    const char *msg = lb_last_error();
    if (!msg || !strstr(msg, "dimensions")) return 2;
    printf("%d %s\n", (int)st, msg);
    return 0;
}
''')
    exe = tmp_path / "caller"
    libdir = os.path.dirname(LIB)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-llbcuboid", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("1 ")
