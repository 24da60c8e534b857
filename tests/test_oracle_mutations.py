"""Planted mistakes: each plausible slip in the FP64 oracle must make at
least one of its pins fail.

Every case replaces one oracle function (or constant) by a copy with a single
deliberate error, on the CPU, and runs the pins that should notice it. A
pin that still passes under a mutation would not be pinning that part of the
oracle. The pins are the functions of test_oracle_pins.py, called directly.
"""

import math

import pytest
import torch

import oracle as O
import oracle.lbm as L
import test_oracle_pins as pins

F64 = torch.float64


@pytest.fixture(scope="module")
def coex():
    Tc = O.critical_temperature(pins.A_PAPER, pins.B_PAPER, 1.0)
    rv, rl = O.maxwell_coexistence(pins.A_PAPER, pins.B_PAPER, 1.0, 0.344, 0.86 * Tc)
    return Tc, rv, rl


def _patch(monkeypatch, name, value):
    """Replace `name` in the oracle module (seen by the oracle's own calls)
    and in the package namespace (seen by the pins)."""
    monkeypatch.setattr(L, name, value)
    if hasattr(O, name):
        monkeypatch.setattr(O, name, value)


# ---- the mutations ---------------------------------------------------------

_rhs = L.temperature_rhs
_eq = L.equilibrium_moments
_fm = L.forcing_moments
_ads = L.adhesion_force
_fill = L.wall_fill


def rhs_advection_sign(T, fl, P):
    """+v.grad T instead of -v.grad T in Eq. 18."""
    dTx, dTy = L.grad_iso(T)
    return _rhs(T, fl, P) + 2.0 * (fl.vx * dTx + fl.vy * dTy)


def rhs_no_conductivity_gradient(T, fl, P):
    """div(lambda grad T) without the grad lambda . grad T part."""
    dTx, dTy = L.grad_iso(T)
    return _rhs(T, fl, P) - P.cv_chi * (fl.drx * dTx + fl.dry * dTy) / (fl.rho * P.cv)


def rhs_source_sign(T, fl, P):
    """+T/(rho c_v) (dp/dT) div v instead of minus."""
    dpdT = L.pr_dp_dT(fl.rho, T, P.a, P.b, P.R, P.omega, P.Tc)
    return _rhs(T, fl, P) + 2.0 * T / (fl.rho * P.cv) * dpdT * fl.div_v


def eq_energy_row(rho, vx, vy):
    """e^eq = rho (-2 + 2 v^2) instead of rho (-2 + 3 v^2) (Eq. 5)."""
    m = _eq(rho, vx, vy).clone()
    m[1] = m[1] - rho * (vx * vx + vy * vy)
    return m


def forcing_pxy_row(vx, vy, Fx, Fy, Fmx, Fmy, psi, P):
    """The p_xy row of S (Eq. 8) doubled."""
    S = _fm(vx, vy, Fx, Fy, Fmx, Fmy, psi, P).clone()
    S[8] = 2.0 * S[8]
    return S


def collide_forcing_factor(ff, P):
    """(I - Lambda) S instead of (I - Lambda/2) S in Eq. 2."""
    M, Minv = L.transform_matrix(), L.inverse_transform_matrix()
    m = torch.einsum('ab,byx->ayx', M, ff.f)
    meq = L.equilibrium_moments(ff.rho, ff.vx, ff.vy)
    S = L.forcing_moments(ff.vx, ff.vy, ff.Fx, ff.Fy, ff.Fmx, ff.Fmy, ff.psi, P)
    lam = L.relaxation_rates(ff.rho, P)
    return torch.einsum('ab,byx->ayx', Minv, m - lam * (m - meq) + (1.0 - lam) * S)


def rk4_stage3(theta, rho, vx, vy, P):
    """The third RK stage taken from T + h2 instead of T + h2/2 (Eq. 19)."""
    bot, top = L._row_masks(P)
    fluid = (~(bot | top)).to(F64)
    fl = L.frozen_flow(rho, vx, vy)
    T = P.Ts + theta
    h1 = fluid * L.temperature_rhs(T, fl, P)
    h2 = fluid * L.temperature_rhs(T + 0.5 * h1, fl, P)
    h3 = fluid * L.temperature_rhs(T + h2, fl, P)
    h4 = fluid * L.temperature_rhs(T + h3, fl, P)
    return theta + (h1 + 2.0 * h2 + 2.0 * h3 + h4) / 6.0


def wall_fill_sign(f, fpost, P):
    """Zou-He at the bottom wall with f5 = f7 + (f1 - f3)/2 (sign slip)."""
    out = _fill(f, fpost, P).clone()
    bot, _ = L._row_masks(P)
    d = 0.5 * (out[1] - out[3])
    out[5] = torch.where(bot, out[7] + d, out[5])
    return out


def wall_fill_top_sign(f, fpost, P):
    """Zou-He at the top wall with f7 = f5 - (f1 - f3)/2 (sign slip)."""
    out = _fill(f, fpost, P).clone()
    _, top = L._row_masks(P)
    d = 0.5 * (out[1] - out[3])
    out[7] = torch.where(top, out[5] - d, out[7]) if P.bc_y == L.BC_WALLS else out[7]
    return out


_wflux = L.wall_heat_flux
_rk4 = L.rk4_temperature


def flux_sign(theta, rho, P):
    """q_w = +lambda dT/dy instead of -lambda dT/dy (Sec. 3.2)."""
    qw, q = _wflux(theta, rho, P)
    return -qw, -q


def top_wall_zero_gradient(theta, rho, vx, vy, P):
    """The new top wall row copies the row below (zero gradient) instead of
    the Dirichlet T_s."""
    th = _rk4(theta, rho, vx, vy, P)
    if P.bc_y != L.BC_PERIODIC and not P.isothermal:
        th = th.clone()
        th[-1] = th[-2]
    return th


_fmf = L.interaction_force


def interaction_sign(psi, P):
    """F_m = +G psi sum_a w_a psi(x + e_a) e_a (Eq. 7 with the sign lost)."""
    fx, fy = _fmf(psi, P)
    return -fx, -fy


def kappa_sign(omega):
    """The acentric-factor polynomial of Eq. 21 with + on the omega^2 term."""
    return 0.37464 + 1.54226 * omega + 0.26992 * omega * omega


def solid_both_walls(P):
    """s = 1 on the top wall row too (R7 gives the wettability to the
    heating surface only)."""
    s_ = torch.zeros(P.Ly, P.Lx, dtype=F64)
    if P.bc_y != L.BC_PERIODIC:
        s_[0] = 1.0
        s_[-1] = 1.0
    return s_


def adhesion_sign(psi, P):
    """F_ads with the opposite sign (Eq. 22)."""
    fx, fy = _ads(psi, P)
    return -fx, -fy


def stream_push(fpost, P):
    """Streaming with e_a reversed (a push read as a pull, Eq. 3)."""
    return torch.stack([torch.roll(fpost[a], shifts=(-L.EY[a], -L.EX[a]), dims=(0, 1)) for a in range(9)])


def psi_half(rho, T, P):
    """psi without the factor 2 under the square root."""
    p = L.pr_pressure(rho, T, P.a, P.b, P.R, P.omega, P.Tc)
    arg = (p - rho * L.CS2) / P.G
    return torch.sqrt(torch.clamp(arg, min=0.0)), arg < 0


def tau_nu_no_half(rho, P):
    """tau = nu / c_s^2 without the + 1/2."""
    tl, tv = P.nu_l / L.CS2, P.nu_v / L.CS2
    s = torch.clamp((rho - P.rho_v) / (P.rho_l - P.rho_v), 0.0, 1.0)
    return tv + (tl - tv) * s


def flux_first_order(theta, rho, P):
    """q_w with the first-order wall difference T_1 - T_0."""
    qw = -P.cv_chi * rho[0] * (theta[1] - theta[0])
    return qw, qw.mean()


_dphi = L.pr_dphi_dT


def dphi_sign(T, Tc, omega):
    """d phi / dT with the opposite sign."""
    return -_dphi(T, Tc, omega)


def buoyancy_sign(rho, P):
    """F_b = -(rho - rho_ave) g: light fluid pushed down."""
    return torch.zeros_like(rho), (rho - P.rho_ave) * P.g


def area_half_log(v1, v2, T, a, b, R, omega, Tc):
    """The attractive part of the isotherm's primitive with 1/sqrt(2) b in
    place of 1/(2 sqrt(2) b)."""
    ph = L.pr_phi(T, Tc, omega)
    s2 = math.sqrt(2.0)

    def prim(v):
        return R * T * math.log(v - b) - a * ph / (s2 * b) * math.log((v + b - s2 * b) / (v + b + s2 * b))

    return prim(v2) - prim(v1)


def forcing_sigma_tau(vx, vy, Fx, Fy, Fmx, Fmy, psi, P):
    """The sigma term of Eq. 8 over tau_e, tau_zeta instead of tau - 1/2."""
    S = _fm(vx, vy, Fx, Fy, Fmx, Fmy, psi, P).clone()
    psi2 = psi * psi
    ratio = torch.where(psi2 > 0, (Fmx * Fmx + Fmy * Fmy) / torch.where(psi2 > 0, psi2, torch.ones_like(psi2)),
                        torch.zeros_like(psi2))
    te, tz = 1.0 / P.s_e, 1.0 / P.s_z
    S[1] = S[1] + P.sigma * ratio * (1.0 / te - 1.0 / (te - 0.5))
    S[2] = S[2] - P.sigma * ratio * (1.0 / tz - 1.0 / (tz - 0.5))
    return S


def _sigma_ratio(Fmx, Fmy, psi):
    psi2 = psi * psi
    return torch.where(psi2 > 0, (Fmx * Fmx + Fmy * Fmy) / torch.where(psi2 > 0, psi2, torch.ones_like(psi2)),
                       torch.zeros_like(psi2))


def forcing_zeta_sigma_dropped(vx, vy, Fx, Fy, Fmx, Fmy, psi, P):
    """The zeta row of S (Eq. 8) without its sigma term."""
    S = _fm(vx, vy, Fx, Fy, Fmx, Fmy, psi, P).clone()
    S[2] = S[2] + P.sigma * _sigma_ratio(Fmx, Fmy, psi) / (1.0 / P.s_z - 0.5)
    return S


def forcing_zeta_sigma_sign(vx, vy, Fx, Fy, Fmx, Fmy, psi, P):
    """The sigma term of the zeta row of S (Eq. 8) with a plus sign."""
    S = _fm(vx, vy, Fx, Fy, Fmx, Fmy, psi, P).clone()
    S[2] = S[2] + 2.0 * P.sigma * _sigma_ratio(Fmx, Fmy, psi) / (1.0 / P.s_z - 0.5)
    return S


def forcing_zeta_sigma_tau_e(vx, vy, Fx, Fy, Fmx, Fmy, psi, P):
    """The sigma term of the zeta row of S (Eq. 8) over tau_e - 1/2 instead of
    tau_zeta - 1/2."""
    S = _fm(vx, vy, Fx, Fy, Fmx, Fmy, psi, P).clone()
    r = P.sigma * _sigma_ratio(Fmx, Fmy, psi)
    S[2] = S[2] + r / (1.0 / P.s_z - 0.5) - r / (1.0 / P.s_e - 0.5)
    return S


_nb = L._neighbour


def ghost_mirrored(field, a, P, ghost_rows):
    """The ghost row beyond each wall mirrors the first fluid row
    (psi(-1) = psi(1)) instead of copying the wall row."""
    if P.bc_y == L.BC_PERIODIC or not ghost_rows:
        return _nb(field, a, P, ghost_rows)
    ext = torch.cat([field[1:2], field, field[-2:-1]], dim=0)
    ext = torch.roll(ext, shifts=(-L.EY[a], -L.EX[a]), dims=(0, 1))
    return ext[1:-1]


def ghost_wrapped(field, a, P, ghost_rows):
    """Rows beyond the walls taken periodically (the ghost layer ignored)."""
    return _nb(field, a, P, False)


FORCE_W_WRONG = (0.0,) + (1.0 / 3.0,) * 4 + (1.0 / 6.0,) * 4  # diagonal 1/6 instead of 1/12
STENCIL_W_WRONG = (4.0 / 9.0,) + (1.0 / 9.0,) * 4 + (1.0 / 18.0,) * 4  # diagonal 1/18 instead of 1/36

# name -> (what is replaced, replacement, pins expected to fail, changes a step)
MUTATIONS = {
    "advection sign": ("temperature_rhs", rhs_advection_sign, ["manufactured"], True),
    "dropped conductivity gradient": ("temperature_rhs", rhs_no_conductivity_gradient, ["manufactured"], True),
    "source-term sign": ("temperature_rhs", rhs_source_sign, ["manufactured"], True),
    "equilibrium energy row": ("equilibrium_moments", eq_energy_row, ["equilibrium"], True),
    "forcing p_xy row": ("forcing_moments", forcing_pxy_row, ["guo"], True),
    "forcing factor": ("collide", collide_forcing_factor, ["guo"], True),
    "RK4 stage": ("rk4_temperature", rk4_stage3, ["rk4"], True),
    "Zou-He sign": ("wall_fill", wall_fill_sign, ["zou_he"], True),
    "Zou-He top sign": ("wall_fill", wall_fill_top_sign, ["zou_he"], True),
    "adhesion sign": ("adhesion_force", adhesion_sign, ["adhesion"], True),
    "adhesion on both walls": ("solid_switch", solid_both_walls, ["adhesion"], True),
    "force weight": ("FORCE_W", FORCE_W_WRONG, ["taylor"], True),
    "interaction-force sign": ("interaction_force", interaction_sign, ["taylor"], True),
    "kappa polynomial": ("pr_kappa", kappa_sign, ["maxwell"], True),
    "streaming direction": ("stream_pull", stream_push, ["stream"], True),
    "stencil weight": ("STENCIL_W", STENCIL_W_WRONG, ["quadratics", "symbol"], True),
    "psi factor": ("pseudopotential", psi_half, ["bulk_pressure"], True),
    "relaxation time": ("tau_nu", tau_nu_no_half, ["tau_nu"], True),
    "wall derivative order": ("wall_heat_flux", flux_first_order, ["wall_flux"], True),
    "wall flux sign": ("wall_heat_flux", flux_sign, ["wall_flux", "conduction"], True),
    "top wall temperature": ("rk4_temperature", top_wall_zero_gradient, ["conduction"], True),
    "d phi / dT sign": ("pr_dphi_dT", dphi_sign, ["dp_dT"], True),
    "buoyancy sign": ("buoyancy", buoyancy_sign, ["buoyancy"], True),
    "equal-area primitive": ("_pr_area", area_half_log, ["maxwell"], False),
    "sigma-term denominator": ("forcing_moments", forcing_sigma_tau, ["coexistence"], True),
    "zeta sigma term dropped": ("forcing_moments", forcing_zeta_sigma_dropped, ["sigma_rows"], True),
    "zeta sigma term sign": ("forcing_moments", forcing_zeta_sigma_sign, ["sigma_rows"], True),
    # the ghost layer is an option the default step does not use
    "ghost row mirrored": ("_neighbour", ghost_mirrored, ["ghost"], False),
    "ghost row wrapped": ("_neighbour", ghost_wrapped, ["ghost"], False),
    # identical to the oracle at the default s_e = s_zeta, so not a change of
    # the default step; the pin runs it at unequal rates
    "zeta sigma term rate": ("forcing_moments", forcing_zeta_sigma_tau_e, ["sigma_rows"], False),
}


def _sigma_rows(_):
    """The e/zeta sigma-term pin at unequal and at equal rates."""
    pins.test_sigma_term_of_e_and_zeta_rows(0.8, 1.25)
    pins.test_sigma_term_of_e_and_zeta_rows(0.8, 0.8)


def _maxwell_pins(_):
    """The coexistence pins on densities recomputed under the mutation."""
    Tc = O.critical_temperature(pins.A_PAPER, pins.B_PAPER, 1.0)
    c = (Tc,) + tuple(O.maxwell_coexistence(pins.A_PAPER, pins.B_PAPER, 1.0, 0.344, 0.86 * Tc))
    pins.test_maxwell_equal_area_by_quadrature(c)
    pins.test_maxwell_matches_paper_printed_values(c)


PINS = {
    "manufactured": lambda c: pins.test_temperature_rhs_manufactured_solution(c),
    "equilibrium": lambda c: pins.test_equilibrium_moments_are_moments_of_textbook_equilibrium(),
    "guo": lambda c: pins.test_collision_reduces_to_bgk_with_guo_forcing(1.3),
    "rk4": lambda c: pins.test_rk4_fourier_mode_closed_form(c),
    "zou_he": lambda c: pins.test_zou_he_wall_fill_solves_its_conditions(),
    "adhesion": lambda c: pins.test_adhesion_force_bruteforce(),
    "taylor": lambda c: pins.test_interaction_force_taylor_limit(),
    "stream": lambda c: pins.test_stream_pull_bruteforce(),
    "quadratics": lambda c: pins.test_stencils_exact_on_quadratics(),
    "symbol": lambda c: pins.test_laplacian_fourier_symbol(),
    "bulk_pressure": lambda c: pins.test_pseudopotential_bulk_pressure(c),
    "tau_nu": lambda c: pins.test_tau_nu_endpoints(c),
    "wall_flux": lambda c: pins.test_wall_flux_exact_on_quadratic(c),
    "dp_dT": lambda c: pins.test_dp_dT_against_central_difference(c),
    "buoyancy": lambda c: pins.test_buoyancy_direction(),
    "maxwell": _maxwell_pins,
    "coexistence": lambda c: pins.test_flat_interface_coexistence_matches_maxwell(c),
    "sigma_rows": _sigma_rows,
    "ghost": lambda c: pins.test_ghost_layer_wall_rows_on_linear_psi(),
    "conduction": lambda c: pins.test_linear_conduction_profile_is_steady(c),
}


@pytest.mark.parametrize("pin", sorted(PINS))
def test_pin_passes_on_the_oracle(coex, pin):
    PINS[pin](coex)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(coex, monkeypatch, name):
    target, replacement, expected, _ = MUTATIONS[name]
    _patch(monkeypatch, target, replacement)
    for pin in expected:
        with pytest.raises(AssertionError):
            PINS[pin](coex)


def test_mutations_change_a_whole_step(coex, monkeypatch):
    """Every mutation of the step's arithmetic also changes what one full
    oracle step computes (populations, temperature or the wall flux) on a
    heated pool with an interface, so none of them is a no-op."""
    Tc, rv, rl = coex
    from paper_1501_03857_gb300 import inputs
    Lx, Ly = 10, 12
    rho0 = inputs.pool_density(Lx, Ly, rl, rv, 6, noise_amp=1e-2, seed=5)
    P = pins.make(Lx, Ly, rho0, coex, Gw=0.05, superheat=0.02)
    f0, th0 = O.initial_state(torch.tensor(rho0, dtype=F64), P)
    f0, th0, _ = O.step(f0, th0, P)
    ref_f, ref_t, ref = O.step(f0, th0, P)
    for name, (target, replacement, _, in_step) in MUTATIONS.items():
        if not in_step:
            continue
        with monkeypatch.context() as m:
            m.setattr(L, target, replacement)
            f, t, info = L.step(f0, th0, P)
        diff = max(float((f - ref_f).abs().max()), float((t - ref_t).abs().max()), abs(float(info.q - ref.q)))
        assert diff > 1e-12, name
    assert math.isfinite(float(ref_f.sum()))
