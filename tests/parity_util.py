"""Shared helpers of the parity tests: oracle parameters from a library
Config, and normalised field errors."""

import numpy as np
import torch

import oracle as O

F64 = torch.float64


def oracle_params(cfg, rho0, superheat=0.0, Gw=0.0, profile=None, rho_ave=None):
    P = O.Params(Lx=cfg.Lx, Ly=cfg.Ly, bc_y=cfg.bc_y, ghost=bool(cfg.ghost_layer), isothermal=bool(cfg.isothermal),
                 a=cfg.a, b=cfg.b, R=cfg.R, omega=cfg.omega, G=cfg.G, sigma=cfg.sigma, Ts_over_Tc=cfg.Ts_over_Tc,
                 cv=cfg.cv, cv_chi=cfg.cv_chi, g=cfg.g, nu_l=cfg.nu_l, nu_v=cfg.nu_v, s_e=cfg.s_e, s_z=cfg.s_zeta,
                 s_q=cfg.s_q, Gw=Gw)
    P.finalize(rho0=None if rho0 is None else torch.tensor(np.asarray(rho0, dtype=np.float32), dtype=F64),
               superheat=superheat, profile=profile)
    if rho_ave is not None:
        P.rho_ave = rho_ave
    return P


def norm_err(got, ref, scale=None):
    """max |got - ref| / max |ref| (normalised max-norm error); `scale`
    replaces max |ref| where the field's natural scale is known."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if scale is None:
        scale = np.abs(ref).max()
    return float(np.abs(got - ref).max() / (scale if scale > 0 else 1.0))


def rel_err(got, ref):
    """max over elements of |got - ref| / |ref| (for strictly positive fields)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float((np.abs(got - ref) / np.abs(ref)).max())


def theta_err(got, ref, superheat):
    """Temperature error relative to the temperature scale of the problem,
    max(max |theta_ref|, wall superheat): where theta is still ~0 (only the
    div v source has acted) its own maximum is not a meaningful scale."""
    return norm_err(got, ref, max(float(np.abs(np.asarray(ref)).max()), abs(superheat)))


def oracle_initial_fp32(rho0, P):
    """The oracle's initial state, rounded to FP32 (the state both sides start from)."""
    f, th = O.initial_state(torch.tensor(np.asarray(rho0, dtype=np.float32), dtype=F64), P)
    return f.numpy().astype(np.float32), th.numpy().astype(np.float32)


def run_oracle(f32, th32, P, nsteps):
    f = torch.tensor(f32, dtype=F64)
    th = torch.tensor(th32, dtype=F64)
    qs = []
    info = None
    for _ in range(nsteps):
        f, th, info = O.step(f, th, P)
        if info.q is not None:
            qs.append(float(info.q))
    return f, th, qs


def oracle_fields(f, th, P):
    ff = O.flow_fields(f, th, P)
    return ff.rho.numpy(), ff.vx.numpy(), ff.vy.numpy(), (P.Ts + th).numpy()
