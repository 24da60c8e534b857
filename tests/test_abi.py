"""The C-ABI library without a GPU: it loads, exports every symbol that
include/lb.h declares, and its host-only entry points (FP64 thermodynamics,
initial pool, validation, workspace layout) agree with the oracle and the
input generator."""

import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1501_03857_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lb():
    from paper_1501_03857_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_1501_03857_gb300 import lb as lbmod
    return lbmod


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(lb):
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lb.lib, n), n


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++17")])
def test_header_is_plain_c_and_cxx(lang, std, tmp_path):
    """include/lb.h compiles on its own as strict C99 and as C++17, and a C
    translation unit can take the address of every declared entry point
    (the signatures use plain pointers and sizes only)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / ("use." + ("c" if lang == "c" else "cpp"))
    refs = "\n".join(f"    (void)&{n};" for n in declared_symbols())
    src.write_text('#include "lb.h"\nvoid touch(void) {\n' + refs + "\n}\n")
    r = subprocess.run([cc, "-fsyntax-only", std, "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_plain_c_program_links_and_calls_host_entry_points(lb, tmp_path):
    """A C program (no Python, no PyTorch) links liblbboil.so and calls the
    host-only entry points: T_c, the coexistence densities and the
    workspace size agree with the oracle and the layout rule; a bad grid
    returns LB_E_INVAL with a message."""
    import shutil
    import subprocess
    from paper_1501_03857_gb300 import build
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / "host.c"
    src.write_text(r"""
#include <stdio.h>
#include "lb.h"
int main(void) {
    lb_eos e = {3.0 / 49.0, 2.0 / 21.0, 1.0, 0.344, -1.0, 1.2};
    double Tc, rv, rl;
    size_t n;
    lb_grid g = {100, 100, LB_BC_WALLS, 0, 0, 0};
    lb_grid bad = {0, 100, LB_BC_WALLS, 0, 0, 0};
    if (lb_critical_temperature(&e, &Tc) != LB_OK) return 1;
    if (lb_coexistence(&e, 0.86 * Tc, &rv, &rl) != LB_OK) return 2;
    if (lb_workspace_bytes(&g, &n) != LB_OK) return 3;
    if (lb_workspace_bytes(&bad, &n) != LB_E_INVAL || lb_last_error()[0] == 0) return 4;
    lb_workspace_bytes(&g, &n);
    printf("%.17g %.17g %.17g %zu\n", Tc, rv, rl, n);
    return 0;
}
""")
    exe = tmp_path / "host"
    libdir = os.path.dirname(build.LIB)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe), "-L", libdir, "-llbboil", "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    Tc, rv, rl, nbytes = r.stdout.split()
    Tc_o = O.critical_temperature(3 / 49, 2 / 21, 1.0)
    rv_o, rl_o = O.maxwell_coexistence(3 / 49, 2 / 21, 1.0, 0.344, 0.86 * Tc_o)
    assert abs(float(Tc) - Tc_o) < 1e-14 * Tc_o
    assert abs(float(rv) - rv_o) < 1e-9 * rv_o and abs(float(rl) - rl_o) < 1e-9 * rl_o
    assert int(nbytes) == lb.workspace_bytes(lb.Config(Lx=100, Ly=100))


def test_checked_build_exports_every_declared_symbol(lb):
    """The bounds-checked build (-DLB_CHECKED) exposes the same C ABI."""
    import ctypes
    from paper_1501_03857_gb300 import build
    assert os.path.exists(build.LIB_CHECKED), "build() makes liblbboil_checked.so beside liblbboil.so"
    lib = ctypes.CDLL(build.LIB_CHECKED)
    for n in declared_symbols():
        assert hasattr(lib, n), n


def test_critical_temperature_matches_oracle(lb):
    for a in (3 / 49, 2 / 49):
        cfg = lb.Config(a=a)
        assert abs(lb.critical_temperature(cfg) - O.critical_temperature(a, cfg.b, cfg.R)) < 1e-15


@pytest.mark.parametrize("a,tr", [(3 / 49, 0.86), (2 / 49, 0.86), (3 / 49, 0.7), (3 / 49, 0.95)])
def test_coexistence_matches_oracle(lb, a, tr):
    cfg = lb.Config(a=a, Ts_over_Tc=tr)
    T = tr * lb.critical_temperature(cfg)
    rv, rl = lb.coexistence(cfg)
    orv, orl = O.maxwell_coexistence(a, cfg.b, cfg.R, cfg.omega, T)
    assert abs(rv / orv - 1) < 1e-10 and abs(rl / orl - 1) < 1e-10


def test_initial_density_matches_input_generator(lb):
    cfg = lb.Config(Lx=37, Ly=23, pool_height=9.5, noise_amp=1e-4, seed=7)
    got = lb.initial_density(cfg)
    rv, rl = lb.coexistence(cfg)
    want = inputs.pool_density(37, 23, rl, rv, 9.5, noise_amp=1e-4, seed=7)
    assert got.shape == want.shape
    ulp = np.abs(got.view(np.int32).astype(np.int64) - want.view(np.int32).astype(np.int64))
    assert ulp.max() <= 1


def test_workspace_layout_grows_with_grid(lb):
    small = lb.workspace_bytes(lb.Config(Lx=10, Ly=10))
    big = lb.workspace_bytes(lb.Config(Lx=4096, Ly=4096))
    assert big >= 2 * 10 * 4096 * 4096 * 4  # two copies of 9 populations + theta
    assert small % 256 == 0 and big % 256 == 0


@pytest.mark.parametrize("kw", [dict(Lx=0), dict(Ly=2), dict(bc_y=7), dict(G=1.0), dict(s_e=2.0),
                                dict(Ts_over_Tc=1.2), dict(nu_l=0.0)])
def test_invalid_parameters_rejected_before_any_device_call(lb, kw):
    cfg = lb.Config(Lx=16, Ly=16)
    for k, v in kw.items():
        setattr(cfg, k, v)
    g, e, t = cfg.structs()
    import ctypes as C
    h = C.c_void_p()
    rc = lb.lib.lb_init(C.byref(h), C.byref(g), C.byref(e), C.byref(t), None, 0.0, 0.0, None, None, 0, None)
    assert rc == -1
    assert lb.lib.lb_last_error().decode()


def test_workspace_too_small_rejected(lb):
    import ctypes as C
    cfg = lb.Config(Lx=16, Ly=16)
    g, e, t = cfg.structs()
    h = C.c_void_p()
    rc = lb.lib.lb_init(C.byref(h), C.byref(g), C.byref(e), C.byref(t), None, 0.0, 0.0, None,
                        C.c_void_p(256), 10, None)
    assert rc == -1 and "workspace" in lb.lib.lb_last_error().decode()


def test_null_handle_calls_fail_cleanly(lb):
    assert lb.lib.lb_step(None, 1) == -1
    assert lb.lib.lb_sync(None) == -1
    assert lb.lib.lb_destroy(None) == -1


def test_largest_grid_accepted_one_row_more_rejected(lb):
    """Population offsets are 32-bit: 9 * pitch * Ly < 2^31. At Lx = 16384
    (pitch 16384) the largest Ly is 14563; one row more is rejected with a
    message, before any device call."""
    ok = lb.workspace_bytes(lb.Config(Lx=16384, Ly=14563))
    assert ok >= 2 * 10 * 16384 * 14563 * 4
    with pytest.raises(lb.LBError, match="too large"):
        lb.workspace_bytes(lb.Config(Lx=16384, Ly=14564))


def test_empty_batch_rejected_before_any_device_call(lb):
    """A batch of no instances (n = 0) or a null descriptor array is rejected
    by the host before anything touches the device."""
    import ctypes as C
    desc = lb.lb_batch_desc()
    n = C.c_size_t()
    assert lb.lib.lb_batch_workspace_bytes(C.byref(desc), 0, C.byref(n)) == -1
    assert "n >= 1" in lb.lib.lb_last_error().decode()
    assert lb.lib.lb_batch_workspace_bytes(None, 1, C.byref(n)) == -1
    b = C.c_void_p()
    assert lb.lib.lb_batch_init(C.byref(b), C.byref(desc), 0, None, 0, None) == -1
    assert not b.value


HANDLE_CALLS = ["lb_step", "lb_set_wall_temperature", "lb_set_wettability", "lb_heat_flux", "lb_fields",
                "lb_get_state", "lb_set_state", "lb_mass", "lb_sync", "lb_info", "lb_set_launch", "lb_save_bytes",
                "lb_save", "lb_load", "lb_destroy", "lb_adjoint_scratch_bytes", "lb_adjoint_pick_ckpt", "lb_adjoint",
                "lb_set_probes", "lb_probe_read", "lb_batch_step", "lb_batch_set_launch", "lb_batch_set_persistent",
                "lb_batch_heat_flux", "lb_batch_get_state", "lb_batch_set_state", "lb_batch_fields",
                "lb_batch_set_wall_temperature", "lb_batch_set_wettability", "lb_batch_info", "lb_batch_sync",
                "lb_batch_destroy"]


@pytest.mark.parametrize("name", HANDLE_CALLS)
def test_null_handle_rejected_before_any_device_call(lb, name):
    """Every entry point that takes a simulation or batch handle rejects a
    null one with LB_E_INVAL and a message, whatever its other arguments
    (zeros and null pointers here), before it touches the device."""
    import ctypes as C
    fn = getattr(lb.lib, name)
    args = []
    for t in fn.argtypes:
        if t in (C.c_double, C.c_float):
            args.append(0.0)
        elif t in (C.c_int, C.c_int32, C.c_int64, C.c_longlong, C.c_size_t, C.c_uint64):
            args.append(0)
        else:
            args.append(None)
    assert fn(*args) == -1, name
    msg = lb.lib.lb_last_error().decode()
    assert "null" in msg or "bad batch" in msg, msg
