"""FP64 CPU oracle: one time step of the hybrid thermal pseudopotential lattice
Boltzmann boiling model of Li, Kang, Francois, He and Luo (arXiv 1501.03857).

Test infrastructure only. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this module; the
CUDA product path shares no code with it and never imports it.

Everything here is plain PyTorch CPU arithmetic in float64 on whole arrays
(``torch.roll`` for neighbour access, one einsum per moment transform), in the
order the paper states the method, so it can be checked against the paper by
eye. Autograd through :func:`step` gives the exact discrete adjoint of this
oracle (used to pin gradient parity).

Array conventions: a field is indexed ``[y, x]``; populations are ``[alpha, y,
x]``. Row ``y = 0`` is the heated bottom wall and row ``Ly - 1`` the top wall
(Sec. 3.1). The stored state between steps is the post-collision population
``f*`` (Eq. 3) and ``theta = T - T_s``.

Readings of points the paper leaves open (each is also listed in the design
notes):

* G = -1 so that ``p_EOS - rho c_s^2 < 0`` makes the square root real (Sec. 2,
  psi definition). Where the argument has the wrong sign psi is set to 0 and
  the EOS-domain flag is raised.
* Unstated relaxation rates: s_rho = s_j = 1, s_e = s_zeta = 0.8, s_q = 1.1
  (Eq. 4 names them but gives no values); s_nu = 1/tau_nu with tau_nu linear in
  rho between the Maxwell vapour (nu_V = 0.5/3) and liquid (nu_L = 0.1)
  densities, clamped (Sec. 3.1 gives only the two viscosities).
* Force weights w = 1/3 (axis) and 1/12 (diagonal): the coefficients of the
  pressure tensor, Eq. 12, fix them.
* Wall rows are Zou-He wet nodes with u = 0 (Sec. 3.1). The total force is 0
  on wall rows ("the interaction force is not applied at the solid walls",
  Sec. 3.2); with the ghost-layer option F_m is applied on wall rows with a
  ghost row that copies the wall row's psi.
* F_ads (Eq. 22) uses s = 1 on the bottom wall row only and acts on fluid
  rows; |F_m|^2 in the sigma term of Eq. 8 uses F_m alone.
* rho_ave of Eq. 9 is the mean density at t = 0, held fixed.
* div(lambda grad T) of Eq. 18 is expanded as lambda lap T + grad lambda . grad T
  with lambda = c_v chi rho (Sec. 3.1) and the isotropic stencils of Sec. 2.
* rho and v in all four RK stages are the level-t values of this step
  (Sec. 2, after Eq. 20); the temperature in psi is T^t.
* Wall heat flux q_w = -lambda dT/dy at y = 0 with the second-order one-sided
  difference (-3 T0 + 4 T1 - T2)/2 (Sec. 3.2 defines q_w, not its stencil),
  evaluated from (theta^t, rho^t) inside step t.

Every term of the step is pinned (tests/test_oracle_pins.py), including the
sigma term of Eq. 8 in both rows it enters: the e row through the relaxed
flat interface's coexistence densities, and the zeta row through its fixed
relation to the e row (its share of m*_zeta is -s_zeta/s_e times the e row's
share, for any rates). tests/test_oracle_mutations.py plants a slip in each
part and checks that a pin fails.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import torch

F64 = torch.float64

BC_WALLS = 0          # no-slip walls at y = 0 and y = Ly - 1 (Sec. 3.1)
BC_TOP_OUTFLOW = 1    # bottom wall, zero-gradient top (optional variant)
BC_PERIODIC = 2       # periodic in y as well (invariant tests only)

# D2Q9 discrete velocities (Sec. 2, D2Q9 lattice), order: rest, +x, +y, -x, -y,
# (+,+), (-,+), (-,-), (+,-).
EX = (0, 1, 0, -1, 0, 1, -1, -1, 1)
EY = (0, 0, 1, 0, -1, 1, 1, -1, -1)
OPP = (0, 3, 4, 1, 2, 7, 8, 5, 6)

# Lallemand-Luo transformation matrix (Eq. 2; its row order is fixed by the
# order of the equilibrium moments in Eq. 5: rho, e, zeta, jx, qx, jy, qy,
# pxx, pxy).
M_ROWS = (
    (1, 1, 1, 1, 1, 1, 1, 1, 1),
    (-4, -1, -1, -1, -1, 2, 2, 2, 2),
    (4, -2, -2, -2, -2, 1, 1, 1, 1),
    (0, 1, 0, -1, 0, 1, -1, -1, 1),
    (0, -2, 0, 2, 0, 1, -1, -1, 1),
    (0, 0, 1, 0, -1, 1, 1, -1, -1),
    (0, 0, -2, 0, 2, 1, 1, -1, -1),
    (0, 1, -1, 1, -1, 0, 0, 0, 0),
    (0, 0, 0, 0, 0, 1, -1, 1, -1),
)


def transform_matrix() -> torch.Tensor:
    """M of Eq. 2 as a float64 9x9 tensor."""
    return torch.tensor(M_ROWS, dtype=F64)


def inverse_transform_matrix() -> torch.Tensor:
    """M^-1 of Eq. 3 (f* = M^-1 m*), computed by a general matrix inverse."""
    return torch.linalg.inv(transform_matrix())


# Weights of the interaction force, Eq. 7 (w(1) = 1/3, w(2) = 1/12).
FORCE_W = (0.0,) + (1.0 / 3.0,) * 4 + (1.0 / 12.0,) * 4

# Weights of the isotropic central differences (Lee and Lin, cited in Sec. 2
# after Eq. 20): the D2Q9 equilibrium weights 4/9, 1/9, 1/36.
STENCIL_W = (4.0 / 9.0,) + (1.0 / 9.0,) * 4 + (1.0 / 36.0,) * 4


CS2 = 1.0 / 3.0  # lattice sound speed squared (c = 1)


# ---------------------------------------------------------------------------
# Thermodynamics: Peng-Robinson EOS, Eq. 21
# ---------------------------------------------------------------------------

def critical_temperature(a: float, b: float, R: float) -> float:
    """T_c from the two relations after Eq. 21: a = 0.45724 R^2 Tc^2 / pc and
    b = 0.0778 R Tc / pc; dividing them eliminates pc."""
    return 0.0778 * a / (0.45724 * b * R)


def pr_kappa(omega: float) -> float:
    """The acentric-factor polynomial inside phi(T), Eq. 21."""
    return 0.37464 + 1.54226 * omega - 0.26992 * omega * omega


def pr_phi(T, Tc: float, omega: float):
    """phi(T) = [1 + kappa (1 - sqrt(T/Tc))]^2, Eq. 21."""
    k = pr_kappa(omega)
    sq = torch.sqrt(T / Tc) if torch.is_tensor(T) else math.sqrt(T / Tc)
    return (1.0 + k * (1.0 - sq)) ** 2


def pr_dphi_dT(T, Tc: float, omega: float):
    """d phi / dT of the phi(T) in Eq. 21."""
    k = pr_kappa(omega)
    if torch.is_tensor(T):
        return -k * (1.0 + k * (1.0 - torch.sqrt(T / Tc))) / torch.sqrt(T * Tc)
    return -k * (1.0 + k * (1.0 - math.sqrt(T / Tc))) / math.sqrt(T * Tc)


def pr_pressure(rho, T, a: float, b: float, R: float, omega: float, Tc: float):
    """p_EOS(rho, T), Eq. 21."""
    return rho * R * T / (1.0 - b * rho) - a * pr_phi(T, Tc, omega) * rho * rho / (
        1.0 + 2.0 * b * rho - b * b * rho * rho)


def pr_dp_dT(rho, T, a: float, b: float, R: float, omega: float, Tc: float):
    """(d p_EOS / d T) at constant rho, the coefficient in Eq. 18."""
    return rho * R / (1.0 - b * rho) - a * pr_dphi_dT(T, Tc, omega) * rho * rho / (
        1.0 + 2.0 * b * rho - b * b * rho * rho)


def _pr_area(v1: float, v2: float, T: float, a, b, R, omega, Tc) -> float:
    """Integral of p dv from v1 to v2 for the PR EOS written in v = 1/rho:
    p = R T/(v - b) - a phi /((v + b)^2 - 2 b^2)."""
    ph = pr_phi(T, Tc, omega)
    s2 = math.sqrt(2.0)

    def prim(v):
        return R * T * math.log(v - b) - a * ph / (2.0 * s2 * b) * math.log(
            (v + b - s2 * b) / (v + b + s2 * b))

    return prim(v2) - prim(v1)


def maxwell_coexistence(a: float, b: float, R: float, omega: float, T: float):
    """Liquid-vapour coexistence densities (rho_V, rho_L) of the PR EOS at T by
    the Maxwell equal-area construction (Sec. 1 and Sec. 3.1: the densities a
    thermodynamically consistent model must reproduce, rho_L ~ 6.5 and
    rho_V ~ 0.38 at 0.86 Tc for the parameters after Eq. 21).

    Solved by nested bracketing: for a trial pressure P between the spinodal
    pressures (bracketed on a grid) the outer roots of p(rho) = P are found
    by brentq, and P is bisected until the area between the isotherm and P
    vanishes."""
    from scipy.optimize import brentq

    Tc = critical_temperature(a, b, R)
    if not (0.0 < T < Tc):
        raise ValueError("coexistence needs 0 < T < Tc")
    p = lambda r: float(pr_pressure(r, T, a, b, R, omega, Tc))
    rmax = (1.0 / b) * (1.0 - 1e-9)
    # bracket the spinodal extrema of the isotherm on a fine grid
    grid = np.linspace(1e-6, rmax * 0.999, 20001)
    pg = pr_pressure(grid, T, a, b, R, omega, Tc)
    dp = np.diff(pg)
    idx = np.where(np.sign(dp[:-1]) != np.sign(dp[1:]))[0]
    if len(idx) < 2:
        raise ValueError("isotherm has no van der Waals loop")
    i_hi, i_lo = idx[0] + 1, idx[1] + 1       # grid local max, local min
    r_hi, r_lo = grid[i_hi], grid[i_lo]
    p_hi, p_lo = pg[i_hi], max(pg[i_lo], 1e-8 * pg[i_hi])

    def roots(P):
        rv = brentq(lambda r: p(r) - P, 1e-18, r_hi, xtol=1e-15, rtol=1e-15)
        rl = brentq(lambda r: p(r) - P, r_lo, rmax, xtol=1e-15, rtol=1e-15)
        return rv, rl

    def area_mismatch(P):
        rv, rl = roots(P)
        vv, vl = 1.0 / rv, 1.0 / rl
        return _pr_area(vl, vv, T, a, b, R, omega, Tc) - P * (vv - vl)

    Psat = brentq(area_mismatch, p_lo * (1 + 1e-12), p_hi * (1 - 1e-12), xtol=1e-18, rtol=1e-15)
    return roots(Psat)


# ---------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Params:
    """Every constant of one simulation (Sec. 2, Sec. 3.1)."""
    Lx: int
    Ly: int
    bc_y: int = BC_WALLS
    ghost: bool = False
    isothermal: bool = False
    # EOS, Eq. 21 (paper: a = 3/49, b = 2/21, R = 1, omega = 0.344)
    a: float = 3.0 / 49.0
    b: float = 2.0 / 21.0
    R: float = 1.0
    omega: float = 0.344
    G: float = -1.0
    sigma: float = 1.2           # Eq. 8, value after Eq. 21
    Ts_over_Tc: float = 0.86     # Sec. 3.1
    # transport, Sec. 3.1
    cv: float = 6.0
    cv_chi: float = 0.028
    g: float = 3e-5
    nu_l: float = 0.1
    nu_v: float = 0.5 / 3.0
    s_e: float = 0.8
    s_z: float = 0.8
    s_q: float = 1.1
    Gw: float = 0.0              # Eq. 22
    # derived (filled by finalize)
    Tc: float = 0.0
    Ts: float = 0.0
    rho_v: float = 0.0
    rho_l: float = 0.0
    rho_ave: float = 0.0
    theta_b: Optional[torch.Tensor] = None   # bottom-wall T_b(x) - T_s, length Lx

    def finalize(self, rho0=None, superheat: float = 0.0, profile=None,
                 rho_v: Optional[float] = None, rho_l: Optional[float] = None):
        self.Tc = critical_temperature(self.a, self.b, self.R)
        self.Ts = self.Ts_over_Tc * self.Tc
        if rho_v is None or rho_l is None:
            rho_v, rho_l = maxwell_coexistence(self.a, self.b, self.R, self.omega, self.Ts)
        self.rho_v, self.rho_l = float(rho_v), float(rho_l)
        if rho0 is not None:
            self.rho_ave = float(torch.as_tensor(rho0, dtype=F64).mean())
        tb = torch.full((self.Lx,), float(superheat), dtype=F64)
        if profile is not None:
            tb = tb + torch.as_tensor(profile, dtype=F64)
        self.theta_b = tb
        return self


# ---------------------------------------------------------------------------
# Flow part (Eqs. 1-9, Eq. 22)
# ---------------------------------------------------------------------------

def _row_masks(P: Params):
    """Boolean [Ly, 1] masks of the bottom and top boundary rows."""
    y = torch.arange(P.Ly).unsqueeze(1)
    if P.bc_y == BC_PERIODIC:
        z = torch.zeros_like(y, dtype=torch.bool)
        return z, z
    return (y == 0), (y == P.Ly - 1)


def stream_pull(fpost: torch.Tensor, P: Params) -> torch.Tensor:
    """Streaming, Eq. 3, as a pull: f_a(x, t+1) = f*_a(x - e_a, t), periodic in
    x (Sec. 3.1). Populations that would come from outside a wall row are
    filled afterwards by :func:`wall_fill`."""
    return torch.stack([torch.roll(fpost[a], shifts=(EY[a], EX[a]), dims=(0, 1))
                        for a in range(9)])


def wall_fill(f: torch.Tensor, fpost: torch.Tensor, P: Params) -> torch.Tensor:
    """Zou-He no-slip (u = 0) at the wall rows (Sec. 3.1): the unknown
    populations follow from zero momentum and bounce-back of the normal
    non-equilibrium part. Bottom row unknowns are 2, 5, 6; top row 4, 7, 8.
    With the top-outflow variant the top unknowns are pulled from the top row
    itself (zero normal gradient)."""
    if P.bc_y == BC_PERIODIC:
        return f
    bot, top = _row_masks(P)
    f = list(f.unbind(0))
    # bottom wall, u = 0
    d = 0.5 * (f[1] - f[3])
    f[2] = torch.where(bot, f[4], f[2])
    f[5] = torch.where(bot, f[7] - d, f[5])
    f[6] = torch.where(bot, f[8] + d, f[6])
    if P.bc_y == BC_WALLS:
        d = 0.5 * (f[1] - f[3])
        f[4] = torch.where(top, f[2], f[4])
        f[7] = torch.where(top, f[5] + d, f[7])
        f[8] = torch.where(top, f[6] - d, f[8])
    else:  # zero-gradient top: source row clamped to the top row
        for a in (4, 7, 8):
            own = torch.roll(fpost[a], shifts=(0, EX[a]), dims=(0, 1))
            f[a] = torch.where(top, own, f[a])
    return torch.stack(f)


def pseudopotential(rho, T, P: Params):
    """psi = sqrt(2 (p_EOS - rho c_s^2) / (G c^2)) with c = 1 (Sec. 2, after
    Eq. 7, and after Eq. 20). Returns (psi, bad) where bad marks cells whose
    square-root argument is negative (psi set to 0 there)."""
    p = pr_pressure(rho, T, P.a, P.b, P.R, P.omega, P.Tc)
    arg = 2.0 * (p - rho * CS2) / P.G
    bad = arg < 0
    psi = torch.sqrt(torch.clamp(arg, min=0.0))
    return psi, bad


def _neighbour(field, a, P: Params, ghost_rows: bool):
    """field(x + e_a): periodic in x; in y periodic for BC_PERIODIC, otherwise
    rows beyond the domain are a ghost copy of the boundary row (only used by
    the ghost-layer option; other uses are masked by the caller)."""
    if P.bc_y == BC_PERIODIC or not ghost_rows:
        return torch.roll(field, shifts=(-EY[a], -EX[a]), dims=(0, 1))
    ext = torch.cat([field[:1], field, field[-1:]], dim=0)
    ext = torch.roll(ext, shifts=(-EY[a], -EX[a]), dims=(0, 1))
    return ext[1:-1]


def interaction_force(psi, P: Params):
    """F_m = -G psi(x) sum_a w_a psi(x + e_a) e_a, Eq. 7."""
    w = FORCE_W
    fx = torch.zeros_like(psi)
    fy = torch.zeros_like(psi)
    for a in range(1, 9):
        nb = _neighbour(psi, a, P, ghost_rows=P.ghost)
        fx = fx + w[a] * nb * EX[a]
        fy = fy + w[a] * nb * EY[a]
    return -P.G * psi * fx, -P.G * psi * fy


def solid_switch(P: Params):
    """s(x) of Eq. 22 on an extended grid: 1 on the bottom wall row (the
    heating surface, the only wall given a wettability in Sec. 3.3)."""
    s = torch.zeros(P.Ly, P.Lx, dtype=F64)
    if P.bc_y != BC_PERIODIC:
        s[0] = 1.0
    return s


def adhesion_force(psi, P: Params):
    """F_ads = -G_w psi(x) sum_a omega_a S(x + e_a) e_a with
    S(x + e_a) = phi(x) s(x + e_a), phi = psi, omega_a = w_a / 3 (Eq. 22)."""
    w = [wa / 3.0 for wa in FORCE_W]
    s = solid_switch(P)
    sx = torch.zeros_like(psi)
    sy = torch.zeros_like(psi)
    for a in range(1, 9):
        nb = torch.roll(s, shifts=(-EY[a], -EX[a]), dims=(0, 1))
        if P.bc_y != BC_PERIODIC:
            # no solid beyond the top row (the roll would wrap row 0 there)
            nb = torch.where(torch.arange(P.Ly).unsqueeze(1) + EY[a] >= P.Ly,
                             torch.zeros_like(nb), nb)
        sx = sx + w[a] * nb * EX[a]
        sy = sy + w[a] * nb * EY[a]
    return -P.Gw * psi * psi * sx, -P.Gw * psi * psi * sy


def buoyancy(rho, P: Params):
    """F_b = (rho - rho_ave) g with g = (0, -g), Eq. 9."""
    return torch.zeros_like(rho), -(rho - P.rho_ave) * P.g


@dataclasses.dataclass
class FlowFields:
    f: torch.Tensor      # post-streaming, wall-filled populations
    rho: torch.Tensor
    psi: torch.Tensor
    Fmx: torch.Tensor
    Fmy: torch.Tensor
    Fx: torch.Tensor
    Fy: torch.Tensor
    vx: torch.Tensor
    vy: torch.Tensor
    eos_bad: torch.Tensor


def flow_fields(fpost, theta, P: Params) -> FlowFields:
    """Stream (Eq. 3), wall fill, density and velocity with the half-force
    correction (Eq. 6), pseudopotential (Eq. 21) and forces (Eqs. 7, 9, 22)
    at time level t. T^t enters psi."""
    f = wall_fill(stream_pull(fpost, P), fpost, P)
    rho = f.sum(0)
    T = P.Ts + theta
    psi, bad = pseudopotential(rho, T, P)
    Fmx, Fmy = interaction_force(psi, P)
    Fax, Fay = adhesion_force(psi, P)
    Fbx, Fby = buoyancy(rho, P)
    Fx = Fmx + Fax + Fbx
    Fy = Fmy + Fay + Fby
    bot, top = _row_masks(P)
    wall = bot | top
    if P.ghost:
        # Sec. 3.2 variant: F_m acts on the wall rows too (ghost layer), the
        # other forces do not.
        Fx = torch.where(wall, Fmx, Fx)
        Fy = torch.where(wall, Fmy, Fy)
    else:
        Fx = torch.where(wall, torch.zeros_like(Fx), Fx)
        Fy = torch.where(wall, torch.zeros_like(Fy), Fy)
        Fmx = torch.where(wall, torch.zeros_like(Fmx), Fmx)
        Fmy = torch.where(wall, torch.zeros_like(Fmy), Fmy)
    ex = torch.tensor(EX, dtype=F64).view(9, 1, 1)
    ey = torch.tensor(EY, dtype=F64).view(9, 1, 1)
    vx = ((ex * f).sum(0) + 0.5 * Fx) / rho
    vy = ((ey * f).sum(0) + 0.5 * Fy) / rho
    return FlowFields(f, rho, psi, Fmx, Fmy, Fx, Fy, vx, vy, bad)


def equilibrium_moments(rho, vx, vy):
    """m^eq, Eq. 5."""
    v2 = vx * vx + vy * vy
    return torch.stack([rho, rho * (-2.0 + 3.0 * v2), rho * (1.0 - 3.0 * v2),
                        rho * vx, -rho * vx, rho * vy, -rho * vy,
                        rho * (vx * vx - vy * vy), rho * vx * vy])


def tau_nu(rho, P: Params):
    """Shear relaxation time tau_nu(rho): nu = (tau - 0.5) c_s^2 with
    nu_L = 0.1 and nu_V = 0.5/3 (Sec. 3.1), linear in rho between the Maxwell
    vapour and liquid densities and clamped outside them."""
    tl = P.nu_l / CS2 + 0.5
    tv = P.nu_v / CS2 + 0.5
    s = torch.clamp((rho - P.rho_v) / (P.rho_l - P.rho_v), 0.0, 1.0)
    return tv + (tl - tv) * s


def relaxation_rates(rho, P: Params):
    """Diagonal of Lambda, Eq. 4: (1/tau_rho, 1/tau_e, 1/tau_zeta, 1/tau_j,
    1/tau_q, 1/tau_j, 1/tau_q, 1/tau_nu, 1/tau_nu)."""
    one = torch.ones_like(rho)
    snu = 1.0 / tau_nu(rho, P)
    return torch.stack([one, P.s_e * one, P.s_z * one, one, P.s_q * one, one,
                        P.s_q * one, snu, snu])


def forcing_moments(vx, vy, Fx, Fy, Fmx, Fmy, psi, P: Params):
    """S of Eq. 8, the improved forcing term in moment space (delta_t = 1)."""
    vF = vx * Fx + vy * Fy
    Fm2 = Fmx * Fmx + Fmy * Fmy
    psi2 = psi * psi
    safe = torch.where(psi2 > 0, psi2, torch.ones_like(psi2))
    ratio = torch.where(psi2 > 0, Fm2 / safe, torch.zeros_like(psi2))
    tau_e = 1.0 / P.s_e
    tau_z = 1.0 / P.s_z
    zero = torch.zeros_like(vx)
    return torch.stack([zero,
                        6.0 * vF + P.sigma * ratio / (tau_e - 0.5),
                        -6.0 * vF - P.sigma * ratio / (tau_z - 0.5),
                        Fx, -Fx, Fy, -Fy,
                        2.0 * (vx * Fx - vy * Fy),
                        vx * Fy + vy * Fx])


def collide(ff: FlowFields, P: Params):
    """MRT collision in moment space, Eq. 2: m* = m - Lambda (m - m^eq)
    + (I - Lambda/2) S, then f* = M^-1 m* (Eq. 3)."""
    M = transform_matrix()
    Minv = inverse_transform_matrix()
    m = torch.einsum('ab,byx->ayx', M, ff.f)
    meq = equilibrium_moments(ff.rho, ff.vx, ff.vy)
    S = forcing_moments(ff.vx, ff.vy, ff.Fx, ff.Fy, ff.Fmx, ff.Fmy, ff.psi, P)
    lam = relaxation_rates(ff.rho, P)
    mstar = m - lam * (m - meq) + (1.0 - 0.5 * lam) * S
    return torch.einsum('ab,byx->ayx', Minv, mstar)


# ---------------------------------------------------------------------------
# Temperature part (Eqs. 18-20)
# ---------------------------------------------------------------------------

def neighbours(phi):
    """phi(x + e_a) for a = 0..8, the neighbourhood the isotropic stencils of
    Sec. 2 (after Eq. 20) read; periodic wrap in both directions. Rows that
    wrap through a wall are only read by stencils centred on wall rows, whose
    results are discarded (wall rows are Dirichlet)."""
    return torch.stack([torch.roll(phi, shifts=(-EY[a], -EX[a]), dims=(0, 1))
                        for a in range(9)])


def grad_iso(phi, nb=None):
    """Isotropic central first derivative (Lee and Lin, Sec. 2 after Eq. 20):
    d_i phi = sum_a w_a e_ai [phi(x + e_a) - phi(x - e_a)] / (2 c_s^2)."""
    nb = neighbours(phi) if nb is None else nb
    w = STENCIL_W
    gx = torch.zeros_like(phi)
    gy = torch.zeros_like(phi)
    for a in range(1, 9):
        diff = nb[a] - nb[OPP[a]]
        gx = gx + w[a] * EX[a] * diff
        gy = gy + w[a] * EY[a] * diff
    return gx / (2.0 * CS2), gy / (2.0 * CS2)


def lap_iso(phi, nb=None):
    """Isotropic central Laplacian (Lee and Lin, Sec. 2 after Eq. 20):
    lap phi = sum_a w_a [phi(x + e_a) - 2 phi(x) + phi(x - e_a)] / c_s^2."""
    nb = neighbours(phi) if nb is None else nb
    w = STENCIL_W
    acc = torch.zeros_like(phi)
    for a in range(1, 9):
        acc = acc + w[a] * (nb[a] - 2.0 * phi + nb[OPP[a]])
    return acc / CS2


@dataclasses.dataclass
class FrozenFlow:
    """rho, v and their derivatives at level t; Eq. 18 is integrated with
    these held fixed through the four RK stages (Sec. 2, after Eq. 20)."""
    rho: torch.Tensor
    vx: torch.Tensor
    vy: torch.Tensor
    drx: torch.Tensor
    dry: torch.Tensor
    div_v: torch.Tensor


def frozen_flow(rho, vx, vy) -> FrozenFlow:
    """The parts of K(T) (Eq. 18) that depend on rho and v only: grad rho and
    div v with the isotropic stencils, computed once per step because rho
    and v stay at level t through the four RK stages (Sec. 2, after Eq. 20)."""
    drx, dry = grad_iso(rho)
    dvx, _ = grad_iso(vx)
    _, dvy = grad_iso(vy)
    return FrozenFlow(rho, vx, vy, drx, dry, dvx + dvy)


def temperature_rhs(T, fl: FrozenFlow, P: Params):
    """K(T), the right-hand side of Eq. 18:
    -v.grad T + div(lambda grad T)/(rho c_v) - T/(rho c_v) (dp/dT)_rho div v,
    lambda = c_v chi rho (Sec. 3.1)."""
    nb = neighbours(T)
    dTx, dTy = grad_iso(T, nb)
    lapT = lap_iso(T, nb)
    lam = P.cv_chi * fl.rho
    div_lam_gradT = lam * lapT + P.cv_chi * (fl.drx * dTx + fl.dry * dTy)
    dpdT = pr_dp_dT(fl.rho, T, P.a, P.b, P.R, P.omega, P.Tc)
    return (-(fl.vx * dTx + fl.vy * dTy) + div_lam_gradT / (fl.rho * P.cv)
            - T / (fl.rho * P.cv) * dpdT * fl.div_v)


def rk4_temperature(theta, rho, vx, vy, P: Params):
    """Classical RK4, Eqs. 19-20, with rho and v frozen at level t. Wall rows
    keep their level-t value through the stages; the new wall rows are the
    Dirichlet values T_b(x) (bottom) and T_s (top)."""
    if P.isothermal:
        return theta.clone()
    bot, top = _row_masks(P)
    fluid = (~(bot | top)).to(F64)
    fl = frozen_flow(rho, vx, vy)
    T = P.Ts + theta
    h1 = fluid * temperature_rhs(T, fl, P)
    h2 = fluid * temperature_rhs(T + 0.5 * h1, fl, P)
    h3 = fluid * temperature_rhs(T + 0.5 * h2, fl, P)
    h4 = fluid * temperature_rhs(T + h3, fl, P)
    theta_new = theta + (h1 + 2.0 * h2 + 2.0 * h3 + h4) / 6.0
    if P.bc_y != BC_PERIODIC:
        tb = P.theta_b.view(1, -1).expand(P.Ly, P.Lx)
        theta_new = torch.where(bot, tb, theta_new)
        theta_new = torch.where(top, torch.zeros_like(theta_new), theta_new)
    return theta_new


def wall_heat_flux(theta, rho, P: Params):
    """Local and mean bottom-wall heat flux (Sec. 3.2): q_w(x) =
    -lambda dT/dy at y = 0, lambda = c_v chi rho, one-sided second-order
    difference; q = (1/L_x) sum_x q_w(x)."""
    dTdy = (-3.0 * theta[0] + 4.0 * theta[1] - theta[2]) / 2.0
    qw = -P.cv_chi * rho[0] * dTdy
    return qw, qw.mean()


# ---------------------------------------------------------------------------
# One step, initial state, diagnostics
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class StepInfo:
    q: Optional[torch.Tensor]
    eos_bad: int
    fields: FlowFields


def step(fpost, theta, P: Params):
    """One time step of the hybrid model (Sec. 2 summary after Eq. 20):
    stream + wall fill, rho, psi, forces, v, MRT collision with the improved
    forcing term; RK4 of the temperature with rho^t, v^t; the bottom-wall heat
    flux of level t. Returns (f*_{t+1}, theta_{t+1}, StepInfo)."""
    ff = flow_fields(fpost, theta, P)
    fnew = collide(ff, P)
    q = None
    if P.bc_y != BC_PERIODIC:
        q = wall_heat_flux(theta, ff.rho, P)[1]
    theta_new = rk4_temperature(theta, ff.rho, ff.vx, ff.vy, P)
    return fnew, theta_new, StepInfo(q, int(ff.eos_bad.sum()), ff)


def initial_state(rho0, P: Params, vx0=None, vy0=None):
    """f* = f^eq(rho0, v0) = M^-1 m^eq (Eq. 5), theta = 0 in the fluid and
    the Dirichlet values on the wall rows (Sec. 3.1: the domain starts at T_s,
    the bottom wall is held at T_b)."""
    rho0 = torch.as_tensor(rho0, dtype=F64)
    vx0 = torch.zeros_like(rho0) if vx0 is None else torch.as_tensor(vx0, dtype=F64)
    vy0 = torch.zeros_like(rho0) if vy0 is None else torch.as_tensor(vy0, dtype=F64)
    f = torch.einsum('ab,byx->ayx', inverse_transform_matrix(),
                     equilibrium_moments(rho0, vx0, vy0))
    theta = torch.zeros_like(rho0)
    if P.bc_y != BC_PERIODIC:
        theta[0] = P.theta_b
    return f, theta


def total_mass(fpost):
    """sum over cells of rho = sum_a f*_a (collision conserves mass); the
    mean over cells at t = 0 is rho_ave of Eq. 9."""
    return float(fpost.sum())


def run(fpost, theta, P: Params, nsteps: int):
    """nsteps steps of the step above; returns the final state and the
    per-step q(t) series (Sec. 3.2)."""
    qs = []
    for _ in range(nsteps):
        fpost, theta, info = step(fpost, theta, P)
        if info.q is not None:
            qs.append(float(info.q))
    return fpost, theta, qs
