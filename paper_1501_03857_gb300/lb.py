"""Thin ctypes binding of the C ABI in include/lb.h (argument marshalling only).

Every step of the boiling model runs in the CUDA kernels of liblbboil.so;
PyTorch supplies the device workspace and the stream. If the library is
missing the import of this module fails loudly: there is no fallback.
"""

from __future__ import annotations

import ctypes as C
import dataclasses
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# LBBOIL_LIB selects another build of the library, e.g. _lib/liblbboil_checked.so
LIB_PATH = os.environ.get("LBBOIL_LIB") or os.path.join(_PKG, "_lib", "liblbboil.so")

LB_OK = 0
ERRORS = {-1: "LB_E_INVAL", -2: "LB_E_CUDA", -3: "LB_E_EOS_DOMAIN", -4: "LB_E_NONFINITE", -5: "LB_E_TIMEOUT",
          -6: "LB_E_BOUNDS"}
BC_WALLS, BC_TOP_OUTFLOW, BC_PERIODIC = 0, 1, 2


class LBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class lb_grid(C.Structure):
    _fields_ = [("Lx", C.c_int32), ("Ly", C.c_int32), ("bc_y", C.c_int32), ("ghost_layer", C.c_int32),
                ("isothermal", C.c_int32), ("reserved", C.c_int32)]


class lb_eos(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("a", "b", "R", "omega", "G", "sigma")]


class lb_thermal(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("Ts_over_Tc", "cv", "cv_chi", "g", "nu_l", "nu_v", "s_e", "s_zeta",
                                          "s_q", "pool_height", "noise_amp")] + [("seed", C.c_uint64)]


class lb_batch_desc(C.Structure):
    _fields_ = [("grid", lb_grid), ("eos", lb_eos), ("th", lb_thermal), ("superheat", C.c_double),
                ("Gw", C.c_double), ("Tb_profile", C.c_void_p), ("rho0", C.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with python -m paper_1501_03857_gb300.build")
    lib = C.CDLL(LIB_PATH)
    P, I, D, SZ = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    DP, FP, I64P = C.POINTER(C.c_double), C.c_void_p, C.POINTER(C.c_int64)
    sig = {
        "lb_critical_temperature": [C.POINTER(lb_eos), DP],
        "lb_coexistence": [C.POINTER(lb_eos), D, DP, DP],
        "lb_initial_density": [C.POINTER(lb_grid), C.POINTER(lb_eos), C.POINTER(lb_thermal), FP],
        "lb_workspace_bytes": [C.POINTER(lb_grid), C.POINTER(C.c_size_t)],
        "lb_init": [C.POINTER(P), C.POINTER(lb_grid), C.POINTER(lb_eos), C.POINTER(lb_thermal), P, D, D, P, P, SZ, P],
        "lb_step": [P, I],
        "lb_set_wall_temperature": [P, P, D],
        "lb_set_wettability": [P, D],
        "lb_heat_flux": [P, DP, DP, DP, I64P, I],
        "lb_fields": [P, FP, FP, FP, FP, I],
        "lb_get_state": [P, FP, FP, I],
        "lb_set_state": [P, FP, FP, I],
        "lb_mass": [P, DP],
        "lb_sync": [P],
        "lb_info": [P, I64P, C.POINTER(I), C.POINTER(I), C.POINTER(I)],
        "lb_set_launch": [P, I, I],
        "lb_save_bytes": [P, C.POINTER(C.c_size_t)],
        "lb_save": [P, P, SZ],
        "lb_load": [P, P, SZ],
        "lb_destroy": [P],
        "lb_batch_workspace_bytes": [C.POINTER(lb_batch_desc), I, C.POINTER(C.c_size_t)],
        "lb_batch_init": [C.POINTER(P), C.POINTER(lb_batch_desc), I, P, SZ, P],
        "lb_batch_step": [P, I],
        "lb_batch_set_launch": [P, I, I],
        "lb_batch_set_persistent": [P, I, C.c_longlong],
        "lb_batch_heat_flux": [P, P, P, P, P, I],
        "lb_batch_get_state": [P, I, FP, FP, I],
        "lb_batch_set_state": [P, I, FP, FP, I],
        "lb_batch_fields": [P, I, FP, FP, FP, FP, I],
        "lb_batch_set_wall_temperature": [P, I, P, D],
        "lb_batch_set_wettability": [P, I, D],
        "lb_batch_info": [P, I64P, C.POINTER(I), C.POINTER(I)],
        "lb_batch_sync": [P],
        "lb_batch_destroy": [P],
        "lb_adjoint_scratch_bytes": [P, I, I, C.POINTER(C.c_size_t)],
        "lb_adjoint_pick_ckpt": [P, I, SZ, C.POINTER(I), C.POINTER(C.c_size_t)],
        "lb_adjoint": [P, I, I, P, SZ, DP, P, DP],
        "lb_fields_noalloc": [C.POINTER(lb_grid), C.POINTER(lb_eos), C.POINTER(lb_thermal), D, D, P, P, P, P, P,
                              P, P],
        "lb_probe_ring_bytes": [I, I, C.POINTER(C.c_size_t)],
        "lb_set_probes": [P, I, P, P, P, SZ, I],
        "lb_probe_read": [P, I, FP, I64P, C.POINTER(I)],
        "lb_eos_pressure": [C.POINTER(lb_eos), C.c_int64, FP, FP, FP],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.lb_last_error.argtypes = []
    lib.lb_last_error.restype = C.c_char_p
    return lib


lib = _load()


def check(rc: int):
    if rc != LB_OK:
        raise LBError(rc, lib.lb_last_error().decode())
    return rc


@dataclasses.dataclass
class Config:
    """Grid, EOS and thermal parameters; defaults are the paper's (Sec. 3.1,
    after Eq. 21) on a 600 x 150 domain with the pool up to y = 90."""
    Lx: int = 600
    Ly: int = 150
    bc_y: int = BC_WALLS
    ghost_layer: bool = False
    isothermal: bool = False
    a: float = 3.0 / 49.0
    b: float = 2.0 / 21.0
    R: float = 1.0
    omega: float = 0.344
    G: float = -1.0
    sigma: float = 1.2
    Ts_over_Tc: float = 0.86
    cv: float = 6.0
    cv_chi: float = 0.028
    g: float = 3e-5
    nu_l: float = 0.1
    nu_v: float = 0.5 / 3.0
    s_e: float = 0.8
    s_zeta: float = 0.8
    s_q: float = 1.1
    pool_height: float = 90.0
    noise_amp: float = 1e-4
    seed: int = 1

    def structs(self):
        g = lb_grid(self.Lx, self.Ly, self.bc_y, int(self.ghost_layer), int(self.isothermal), 0)
        e = lb_eos(self.a, self.b, self.R, self.omega, self.G, self.sigma)
        t = lb_thermal(self.Ts_over_Tc, self.cv, self.cv_chi, self.g, self.nu_l, self.nu_v, self.s_e, self.s_zeta,
                       self.s_q, self.pool_height, self.noise_amp, self.seed)
        return g, e, t


def critical_temperature(cfg: Config) -> float:
    _, e, _ = cfg.structs()
    out = C.c_double()
    check(lib.lb_critical_temperature(C.byref(e), C.byref(out)))
    return out.value


def coexistence(cfg: Config, T: Optional[float] = None):
    _, e, _ = cfg.structs()
    if T is None:
        T = cfg.Ts_over_Tc * critical_temperature(cfg)
    rv, rl = C.c_double(), C.c_double()
    check(lib.lb_coexistence(C.byref(e), T, C.byref(rv), C.byref(rl)))
    return rv.value, rl.value


def initial_density(cfg: Config) -> np.ndarray:
    g, e, t = cfg.structs()
    out = np.empty((cfg.Ly, cfg.Lx), dtype=np.float32)
    check(lib.lb_initial_density(C.byref(g), C.byref(e), C.byref(t), out.ctypes.data))
    return out


def workspace_bytes(cfg: Config) -> int:
    g, _, _ = cfg.structs()
    n = C.c_size_t()
    check(lib.lb_workspace_bytes(C.byref(g), C.byref(n)))
    return n.value


NOALLOC_MAX_CELLS = 262144
PROBE_MAX = 8


def eos_pressure(cfg: Config, rho, T) -> np.ndarray:
    """p_EOS(rho, T) of Eq. 21 (FP64, host; lb_eos_pressure) for arrays of
    equal shape."""
    _, e, _ = cfg.structs()
    r = np.ascontiguousarray(rho, dtype=np.float32)
    t = np.ascontiguousarray(np.broadcast_to(T, r.shape), dtype=np.float32)
    out = np.empty(r.shape, dtype=np.float64)
    check(lib.lb_eos_pressure(C.byref(e), int(r.size), r.ctypes.data, t.ctypes.data, out.ctypes.data))
    return out


def fields_noalloc(cfg: Config, Gw: float, rho_ave: float, fpost, theta, rho=None, ux=None, uy=None, T=None,
                   stream=None):
    """Macroscopic fields of a device-resident state without a handle or any
    device allocation (lb_fields_noalloc). fpost [9, Ly, Lx] and theta
    [Ly, Lx] are contiguous float32 CUDA tensors; outputs are preallocated
    contiguous float32 CUDA tensors [Ly, Lx] or None. Grids above
    NOALLOC_MAX_CELLS cells are rejected. Raises ValueError before any call
    into the library when a tensor has the wrong dtype, device, layout or
    shape (the kernels would read or write past a smaller buffer)."""
    import torch
    shapes = {"fpost": (9, cfg.Ly, cfg.Lx), "theta": (cfg.Ly, cfg.Lx)}
    for name, x in (("fpost", fpost), ("theta", theta), ("rho", rho), ("ux", ux), ("uy", uy), ("T", T)):
        if x is None:
            if name in shapes:
                raise ValueError(f"{name} is required")
            continue
        want = shapes.get(name, (cfg.Ly, cfg.Lx))
        if not isinstance(x, torch.Tensor) or x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous() \
                or tuple(x.shape) != want:
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of shape {want}")
    g, e, t = cfg.structs()
    st = stream if stream is not None else torch.cuda.current_stream()
    ptr = lambda x: None if x is None else x.data_ptr()
    check(lib.lb_fields_noalloc(C.byref(g), C.byref(e), C.byref(t), float(Gw), float(rho_ave), ptr(fpost),
                                ptr(theta), ptr(rho), ptr(ux), ptr(uy), ptr(T), st.cuda_stream))


def _host_ptr(a: Optional[np.ndarray], dtype):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data


class Simulation:
    """One boiling domain on the current CUDA device.

    cfg: Config; superheat: T_b - T_s on the bottom wall (plus an optional
    per-x profile); Gw: Eq. 22's wettability strength; rho0: optional initial
    density [Ly, Lx] (host array). Device memory is a torch uint8 tensor owned
    by this object; work runs on `stream` (default: torch's current stream)."""

    def __init__(self, cfg: Config, superheat: float = 0.0, Gw: float = 0.0, profile=None, rho0=None,
                 stream=None):
        import torch
        self.cfg = cfg
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        nbytes = workspace_bytes(cfg)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        self._ws = base + ((-base) % 256)
        g, e, t = cfg.structs()
        prof, pp = _host_ptr(profile, np.float64)
        r0, rp = _host_ptr(rho0, np.float32)
        h = C.c_void_p()
        check(lib.lb_init(C.byref(h), C.byref(g), C.byref(e), C.byref(t), pp, float(superheat), float(Gw), rp,
                          self._ws, nbytes, self.stream.cuda_stream))
        self.h = h
        self.Lx, self.Ly = cfg.Lx, cfg.Ly

    # -- stepping -----------------------------------------------------------
    def step(self, n: int = 1):
        check(lib.lb_step(self.h, int(n)))

    def set_wall_temperature(self, superheat: float, profile=None):
        prof, pp = _host_ptr(profile, np.float64)
        check(lib.lb_set_wall_temperature(self.h, pp, float(superheat)))

    def set_wettability(self, Gw: float):
        check(lib.lb_set_wettability(self.h, float(Gw)))

    def set_launch(self, block_x: int = 0, seg_rows: int = 0):
        check(lib.lb_set_launch(self.h, int(block_x), int(seg_rows)))

    def info(self):
        st, bx, sr, nb = C.c_int64(), C.c_int(), C.c_int(), C.c_int()
        check(lib.lb_info(self.h, C.byref(st), C.byref(bx), C.byref(sr), C.byref(nb)))
        return {"steps": st.value, "block_x": bx.value, "seg_rows": sr.value, "blocks": nb.value}

    # -- pressure probes (Fig. 3) --------------------------------------------
    def set_probes(self, points, capacity: int = 65536):
        """Record (rho^t, T^t, p_EOS) after every step at the cells
        points = [(x, y), ...] (at most PROBE_MAX) in a device ring keeping the
        last `capacity` steps (lb_set_probes); [] removes the probes."""
        torch = self.torch
        n = len(points)
        if n == 0:
            check(lib.lb_set_probes(self.h, 0, None, None, None, 0, 0))
            self._ring = None
            return
        nb = C.c_size_t()
        check(lib.lb_probe_ring_bytes(n, int(capacity), C.byref(nb)))
        ring = torch.empty(nb.value + 256, dtype=torch.uint8, device="cuda")
        base = ring.data_ptr()
        xs = np.array([int(p[0]) for p in points], dtype=np.int32)
        ys = np.array([int(p[1]) for p in points], dtype=np.int32)
        check(lib.lb_set_probes(self.h, n, xs.ctypes.data, ys.ctypes.data, base + ((-base) % 256), nb.value,
                                int(capacity)))
        self._ring, self._probe_n, self._probe_cap = ring, n, int(capacity)

    def probe_read(self, max_records: Optional[int] = None):
        """The newest records of every probe, oldest first: {"count": steps
        probed since set_probes, "rho", "T", "p": arrays [n_probes, m]}."""
        mmax = self._probe_cap if max_records is None else int(max_records)
        out = np.empty(self._probe_n * max(mmax, 1) * 3, dtype=np.float32)
        cnt, m = C.c_int64(), C.c_int()
        check(lib.lb_probe_read(self.h, mmax, out.ctypes.data, C.byref(cnt), C.byref(m)))
        rec = out[: self._probe_n * m.value * 3].reshape(self._probe_n, m.value, 3)
        return {"count": cnt.value, "rho": rec[..., 0].copy(), "T": rec[..., 1].copy(), "p": rec[..., 2].copy()}

    # -- read-back ----------------------------------------------------------
    def heat_flux(self, reset: bool = False):
        qi, qm, qs, n = C.c_double(), C.c_double(), C.c_double(), C.c_int64()
        check(lib.lb_heat_flux(self.h, C.byref(qi), C.byref(qm), C.byref(qs), C.byref(n), int(reset)))
        return {"q_inst": qi.value, "q_mean": qm.value, "q_std": qs.value, "n": n.value}

    def fields(self):
        out = [np.empty((self.Ly, self.Lx), dtype=np.float32) for _ in range(4)]
        check(lib.lb_fields(self.h, *[o.ctypes.data for o in out], 0))
        return dict(zip(("rho", "ux", "uy", "T"), out))

    def fields_device(self, rho, ux, uy, T):
        ptr = lambda t: None if t is None else t.data_ptr()
        check(lib.lb_fields(self.h, ptr(rho), ptr(ux), ptr(uy), ptr(T), 1))

    def get_state(self):
        f = np.empty((9, self.Ly, self.Lx), dtype=np.float32)
        th = np.empty((self.Ly, self.Lx), dtype=np.float32)
        check(lib.lb_get_state(self.h, f.ctypes.data, th.ctypes.data, 0))
        return f, th

    def get_state_device(self, fpost=None, theta=None):
        """Copy the state into preallocated contiguous float32 CUDA tensors
        fpost [9, Ly, Lx] and theta [Ly, Lx] (either may be None)."""
        ptr = lambda t: None if t is None else t.data_ptr()
        check(lib.lb_get_state(self.h, ptr(fpost), ptr(theta), 1))

    def set_state(self, fpost=None, theta=None):
        f, fp = _host_ptr(fpost, np.float32)
        t, tp = _host_ptr(theta, np.float32)
        check(lib.lb_set_state(self.h, fp, tp, 0))

    def mass(self) -> float:
        m = C.c_double()
        check(lib.lb_mass(self.h, C.byref(m)))
        return m.value

    def sync(self):
        check(lib.lb_sync(self.h))

    def adjoint_scratch_bytes(self, nsteps: int, ckpt_every: int = 100) -> int:
        """Device scratch adjoint(nsteps, ckpt_every) allocates (lb_adjoint_scratch_bytes)."""
        n = C.c_size_t()
        check(lib.lb_adjoint_scratch_bytes(self.h, int(nsteps), int(ckpt_every), C.byref(n)))
        return n.value

    def adjoint_ckpt(self, nsteps: int, budget_bytes=None) -> int:
        """Checkpoint interval for adjoint(nsteps) within budget_bytes of
        scratch (lb_adjoint_pick_ckpt): 1, every step stored, when that fits,
        else the interval with the smallest scratch. The default budget is
        half the device memory free now."""
        if budget_bytes is None:
            budget_bytes = self.torch.cuda.mem_get_info()[0] // 2
        c, n = C.c_int(), C.c_size_t()
        check(lib.lb_adjoint_pick_ckpt(self.h, int(nsteps), int(budget_bytes), C.byref(c), C.byref(n)))
        return c.value

    def adjoint(self, nsteps: int, ckpt_every=None):
        """J = mean wall heat flux over the next nsteps steps and its gradients
        dJ/d(T_b(x) - T_s) [Lx] and dJ/dG_w by the discrete adjoint
        (lb_adjoint), with a checkpoint every ckpt_every steps; ckpt_every = 1
        stores every step and replays none (faster, about 20 planes of
        scratch per step); None picks it with adjoint_ckpt (every step stored
        whenever that takes at most half the free device memory). Advances
        the simulation by nsteps."""
        torch = self.torch
        if ckpt_every is None:
            ckpt_every = self.adjoint_ckpt(nsteps)
        n = C.c_size_t(self.adjoint_scratch_bytes(nsteps, ckpt_every))
        scratch = torch.empty(n.value + 256, dtype=torch.uint8, device="cuda")
        base = scratch.data_ptr()
        J, dGw = C.c_double(), C.c_double()
        dTb = np.zeros(self.Lx, dtype=np.float64)
        check(lib.lb_adjoint(self.h, int(nsteps), int(ckpt_every), base + ((-base) % 256), n.value, C.byref(J),
                             dTb.ctypes.data, C.byref(dGw)))
        return J.value, dTb, dGw.value

    def save(self) -> bytes:
        n = C.c_size_t()
        check(lib.lb_save_bytes(self.h, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        check(lib.lb_save(self.h, buf, n.value))
        return buf.raw

    def load(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        check(lib.lb_load(self.h, buf, len(blob)))

    def close(self):
        if getattr(self, "h", None):
            lib.lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent boiling domains advanced by one launch per step
    (lb_batch_*). instances: a list of dicts with keys cfg (Config) and
    optionally superheat, Gw, profile, rho0."""

    def __init__(self, instances, stream=None):
        import torch
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        n = len(instances)
        self.n = n
        self.cfgs = [d["cfg"] for d in instances]
        self._keep = []
        descs = (lb_batch_desc * n)()
        for i, d in enumerate(instances):
            g, e, t = d["cfg"].structs()
            descs[i].grid, descs[i].eos, descs[i].th = g, e, t
            descs[i].superheat = float(d.get("superheat", 0.0))
            descs[i].Gw = float(d.get("Gw", 0.0))
            prof, pp = _host_ptr(d.get("profile"), np.float64)
            r0, rp = _host_ptr(d.get("rho0"), np.float32)
            self._keep += [prof, r0]
            descs[i].Tb_profile = pp
            descs[i].rho0 = rp
        nb = C.c_size_t()
        check(lib.lb_batch_workspace_bytes(descs, n, C.byref(nb)))
        self.workspace = torch.empty(nb.value + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        ws = base + ((-base) % 256)
        h = C.c_void_p()
        check(lib.lb_batch_init(C.byref(h), descs, n, ws, nb.value, self.stream.cuda_stream))
        self._keep = []
        self.h = h

    def step(self, n: int = 1):
        check(lib.lb_batch_step(self.h, int(n)))

    def set_launch(self, block_x: int = 128, seg_rows: int = 0):
        check(lib.lb_batch_set_launch(self.h, int(block_x), int(seg_rows)))

    def set_persistent(self, tiles_per_block: int = 2, wait_limit: int = 0):
        """tiles_per_block >= 1: one cooperative launch per run of 32 steps
        (lb_batch_set_persistent); 0: one launch per step."""
        check(lib.lb_batch_set_persistent(self.h, int(tiles_per_block), int(wait_limit)))

    def info(self):
        st, bx, nb = C.c_int64(), C.c_int(), C.c_int()
        check(lib.lb_batch_info(self.h, C.byref(st), C.byref(bx), C.byref(nb)))
        return {"steps": st.value, "block_x": bx.value, "blocks": nb.value}

    def heat_flux(self, reset: bool = False):
        out = {k: np.zeros(self.n) for k in ("q_inst", "q_mean", "q_std")}
        ns = np.zeros(self.n, dtype=np.int64)
        check(lib.lb_batch_heat_flux(self.h, out["q_inst"].ctypes.data, out["q_mean"].ctypes.data,
                                     out["q_std"].ctypes.data, ns.ctypes.data, int(reset)))
        out["n"] = ns
        return out

    def get_state(self, i: int):
        c = self.cfgs[i]
        f = np.empty((9, c.Ly, c.Lx), dtype=np.float32)
        th = np.empty((c.Ly, c.Lx), dtype=np.float32)
        check(lib.lb_batch_get_state(self.h, int(i), f.ctypes.data, th.ctypes.data, 0))
        return f, th

    def set_state(self, i: int, fpost=None, theta=None):
        f, fp = _host_ptr(fpost, np.float32)
        t, tp = _host_ptr(theta, np.float32)
        check(lib.lb_batch_set_state(self.h, int(i), fp, tp, 0))

    def fields(self, i: int, which=("rho", "ux", "uy", "T")):
        """Macroscopic fields of instance i (lb_batch_fields) as host arrays
        [Ly, Lx]; only the names in `which` are computed and copied."""
        c = self.cfgs[i]
        out = {k: np.empty((c.Ly, c.Lx), dtype=np.float32) for k in which}
        ptr = lambda k: out[k].ctypes.data if k in out else None
        check(lib.lb_batch_fields(self.h, int(i), ptr("rho"), ptr("ux"), ptr("uy"), ptr("T"), 0))
        return out

    def set_wall_temperature(self, i: int, superheat: float, profile=None):
        prof, pp = _host_ptr(profile, np.float64)
        check(lib.lb_batch_set_wall_temperature(self.h, int(i), pp, float(superheat)))

    def set_wettability(self, i: int, Gw: float):
        check(lib.lb_batch_set_wettability(self.h, int(i), float(Gw)))

    def sync(self):
        check(lib.lb_batch_sync(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib.lb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_fn():
    import torch

    class HeatFluxWindow(torch.autograd.Function):
        """J = mean bottom-wall heat flux over a window of `nsteps` steps as a
        differentiable function of the wall superheat profile Tb (tensor [Lx],
        T_b(x) - T_s) and the wettability Gw (0-d tensor); the window starts
        from the state saved in `blob`. Gradients come from the hand-written
        discrete adjoint (lb_adjoint)."""

        @staticmethod
        def forward(ctx, Tb, Gw, sim, blob, nsteps, ckpt_every):
            sim.load(blob)
            sim.set_wall_temperature(0.0, Tb.detach().double().cpu().numpy())
            sim.set_wettability(float(Gw))
            J, dTb, dGw = sim.adjoint(int(nsteps), None if ckpt_every is None else int(ckpt_every))
            ctx.save_for_backward(torch.as_tensor(dTb, dtype=Tb.dtype, device=Tb.device),
                                  torch.as_tensor(dGw, dtype=Gw.dtype, device=Gw.device))
            return torch.as_tensor(J, dtype=torch.float64, device=Tb.device)

        @staticmethod
        def backward(ctx, gJ):
            dTb, dGw = ctx.saved_tensors
            return gJ.to(dTb.dtype) * dTb, gJ.to(dGw.dtype) * dGw, None, None, None, None

    return HeatFluxWindow


def heat_flux_window(Tb, Gw, sim, blob, nsteps, ckpt_every=None):
    """Differentiable J(Tb, Gw); see HeatFluxWindow."""
    return _autograd_fn().apply(Tb, Gw, sim, blob, nsteps, ckpt_every)
