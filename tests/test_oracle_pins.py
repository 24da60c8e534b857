"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a value the
paper prints, a closed form, an invariant, a textbook special case, or a brute
force on a tiny input.
"""

import math
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_1501_03857_gb300 import inputs

torch.set_num_threads(min(4, os.cpu_count() or 1))
F64 = torch.float64
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

A_PAPER, B_PAPER = 3.0 / 49.0, 2.0 / 21.0


def paper_values():
    out = {}
    for line in open(os.path.join(GOLDEN, "paper_values.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v, tol = line.split()
            out[k] = (float(v), float(tol))
    return out


@pytest.fixture(scope="module")
def coex():
    Tc = O.critical_temperature(A_PAPER, B_PAPER, 1.0)
    rv, rl = O.maxwell_coexistence(A_PAPER, B_PAPER, 1.0, 0.344, 0.86 * Tc)
    return Tc, rv, rl


def make(Lx, Ly, rho0, coex, **kw):
    Tc, rv, rl = coex
    superheat = kw.pop("superheat", 0.0)
    P = O.Params(Lx=Lx, Ly=Ly, **kw)
    return P.finalize(rho0=rho0, superheat=superheat, rho_v=rv, rho_l=rl)


# --------------------------------------------------------------------------
# Equation of state (Eq. 21) and coexistence
# --------------------------------------------------------------------------

def test_critical_point_of_eos():
    """T_c from the two relations after Eq. 21 is the temperature where the
    isotherm gets an inflection point with zero slope."""
    a, b, R, om = A_PAPER, B_PAPER, 1.0, 0.344
    Tc = O.critical_temperature(a, b, R)
    rho = np.linspace(0.05, 0.95 / b, 400001)

    def slope(T):
        p = O.pr_pressure(rho, T, a, b, R, om, Tc)
        return np.diff(p) / np.diff(rho)

    s_c = slope(Tc)
    assert s_c.min() > -1e-6 and abs(s_c.min()) < 1e-4
    assert slope(0.99 * Tc).min() < -1e-4      # loop below Tc
    assert slope(1.01 * Tc).min() > 0.0        # no loop above Tc


def test_maxwell_matches_paper_printed_values(coex):
    Tc, rv, rl = coex
    pv = paper_values()
    assert abs(rl - pv["rho_l"][0]) < pv["rho_l"][1]
    assert abs(rv - pv["rho_v"][0]) < pv["rho_v"][1]
    mu = (rl * 0.1) / (rv * 0.5 / 3.0)
    assert abs(mu - pv["mu_ratio"][0]) < pv["mu_ratio"][1]
    assert abs(rl / rv - pv["lambda_ratio"][0]) < pv["lambda_ratio"][1]


def test_maxwell_equal_area_by_quadrature(coex):
    """Equal pressures and equal areas, checked by numerical quadrature of
    p(v) rather than the closed-form primitive the solver uses."""
    from scipy.integrate import quad
    Tc, rv, rl = coex
    a, b, R, om, T = A_PAPER, B_PAPER, 1.0, 0.344, 0.86 * Tc
    pv_ = O.pr_pressure(rv, T, a, b, R, om, Tc)
    pl_ = O.pr_pressure(rl, T, a, b, R, om, Tc)
    assert abs(pv_ - pl_) < 1e-12 * abs(pv_)
    area, _ = quad(lambda v: O.pr_pressure(1.0 / v, T, a, b, R, om, Tc), 1.0 / rl, 1.0 / rv,
                   epsabs=1e-14, epsrel=1e-13, limit=200)
    assert abs(area - pv_ * (1.0 / rv - 1.0 / rl)) < 1e-9 * abs(area)


def test_maxwell_independent_of_a():
    """The reduced PR isotherm depends on T/Tc only, so a = 2/49 and a = 3/49
    give the same coexistence densities at 0.86 Tc."""
    r1 = O.maxwell_coexistence(3 / 49, B_PAPER, 1.0, 0.344, 0.86 * O.critical_temperature(3 / 49, B_PAPER, 1.0))
    r2 = O.maxwell_coexistence(2 / 49, B_PAPER, 1.0, 0.344, 0.86 * O.critical_temperature(2 / 49, B_PAPER, 1.0))
    assert np.allclose(r1, r2, rtol=1e-10)


def test_dp_dT_against_central_difference(coex):
    Tc, rv, rl = coex
    rho = torch.linspace(0.2, 7.5, 50, dtype=F64)
    T = torch.full_like(rho, 0.86 * Tc)
    h = 1e-6 * Tc
    fd = (O.pr_pressure(rho, T + h, A_PAPER, B_PAPER, 1.0, 0.344, Tc)
          - O.pr_pressure(rho, T - h, A_PAPER, B_PAPER, 1.0, 0.344, Tc)) / (2 * h)
    an = O.pr_dp_dT(rho, T, A_PAPER, B_PAPER, 1.0, 0.344, Tc)
    assert torch.allclose(an, fd, rtol=1e-8, atol=0)


def test_pseudopotential_bulk_pressure(coex):
    """With the psi of Sec. 2 the bulk pressure of the pseudopotential fluid,
    rho c_s^2 + G c^2 psi^2 / 2, is the EOS pressure."""
    Tc, rv, rl = coex
    P = O.Params(Lx=1, Ly=1)
    P.finalize(rho_v=rv, rho_l=rl)
    rho = torch.linspace(0.3, 7.0, 40, dtype=F64)
    T = torch.full_like(rho, P.Ts)
    psi, bad = O.pseudopotential(rho, T, P)
    assert not bad.any()
    p = O.pr_pressure(rho, T, P.a, P.b, P.R, P.omega, P.Tc)
    assert torch.allclose(rho / 3.0 + P.G * psi * psi / 2.0, p, rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------------------
# Lattice, MRT and forcing (Eqs. 1-9)
# --------------------------------------------------------------------------

def test_transform_matrix_structure():
    M = O.transform_matrix()
    Minv = O.inverse_transform_matrix()
    assert torch.allclose(M @ Minv, torch.eye(9, dtype=F64), atol=1e-14)
    G = M @ M.T
    assert torch.allclose(G, torch.diag(torch.tensor([9., 36, 36, 6, 12, 6, 12, 4, 4], dtype=F64)))
    assert torch.equal(M[0], torch.ones(9, dtype=F64))
    assert torch.equal(M[3], torch.tensor(O.EX, dtype=F64))
    assert torch.equal(M[5], torch.tensor(O.EY, dtype=F64))
    for a in range(9):
        assert O.EX[O.OPP[a]] == -O.EX[a] and O.EY[O.OPP[a]] == -O.EY[a]


def textbook_feq(rho, vx, vy):
    """Second-order D2Q9 equilibrium written in velocity space."""
    w = torch.tensor(inputs.D2Q9_WEIGHTS, dtype=F64).view(9, 1, 1)
    ex = torch.tensor(O.EX, dtype=F64).view(9, 1, 1)
    ey = torch.tensor(O.EY, dtype=F64).view(9, 1, 1)
    eu = ex * vx + ey * vy
    return w * rho * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * (vx * vx + vy * vy))


def test_equilibrium_moments_are_moments_of_textbook_equilibrium():
    g = torch.Generator().manual_seed(0)
    rho = 0.3 + 6 * torch.rand(4, 5, generator=g, dtype=F64)
    vx = 0.1 * (torch.rand(4, 5, generator=g, dtype=F64) - 0.5)
    vy = 0.1 * (torch.rand(4, 5, generator=g, dtype=F64) - 0.5)
    m = torch.einsum('ab,byx->ayx', O.transform_matrix(), textbook_feq(rho, vx, vy))
    assert torch.allclose(m, O.equilibrium_moments(rho, vx, vy), atol=1e-13)


@pytest.mark.parametrize("tau", [0.8, 1.0, 1.3])
def test_collision_reduces_to_bgk_with_guo_forcing(tau):
    """With one relaxation time for every non-conserved moment and sigma = 0,
    Eq. 2 with the forcing of Eq. 8 is the BGK collision with Guo's forcing
    term F'_a = (1 - 1/(2 tau)) w_a [3 (e_a - v) + 9 (e_a . v) e_a] . F."""
    g = torch.Generator().manual_seed(1)
    Ly, Lx = 3, 4
    nu = (tau - 0.5) / 3.0
    P = O.Params(Lx=Lx, Ly=Ly, s_e=1 / tau, s_z=1 / tau, s_q=1 / tau, nu_l=nu, nu_v=nu, sigma=0.0)
    P.finalize(rho_v=0.38, rho_l=6.5)
    rho = 1 + torch.rand(Ly, Lx, generator=g, dtype=F64)
    f = textbook_feq(rho, 0.05 * torch.ones_like(rho), -0.02 * torch.ones_like(rho))
    f = f * (1 + 0.05 * (torch.rand(9, Ly, Lx, generator=g, dtype=F64) - 0.5))
    rho = f.sum(0)
    Fx = 1e-3 * (torch.rand(Ly, Lx, generator=g, dtype=F64) - 0.5)
    Fy = 1e-3 * (torch.rand(Ly, Lx, generator=g, dtype=F64) - 0.5)
    ex = torch.tensor(O.EX, dtype=F64).view(9, 1, 1)
    ey = torch.tensor(O.EY, dtype=F64).view(9, 1, 1)
    vx = ((ex * f).sum(0) + 0.5 * Fx) / rho
    vy = ((ey * f).sum(0) + 0.5 * Fy) / rho
    z = torch.zeros_like(rho)
    ff = O.FlowFields(f, rho, torch.ones_like(rho), z, z, Fx, Fy, vx, vy, z.bool())
    got = O.collide(ff, P)
    w = torch.tensor(inputs.D2Q9_WEIGHTS, dtype=F64).view(9, 1, 1)
    eu = ex * vx + ey * vy
    guo = (1 - 0.5 / tau) * w * (3 * ((ex - vx) * Fx + (ey - vy) * Fy) + 9 * eu * (ex * Fx + ey * Fy))
    want = f - (f - textbook_feq(rho, vx, vy)) / tau + guo
    assert torch.allclose(got, want, atol=1e-14, rtol=1e-12)


def sigma_term_split(s_e, s_z, sigmas=(0.0, 1.2, 2.5)):
    """Post-collision moments m* = M f* of one oracle collision on a heated
    pool with an interface (F_m, psi non-zero), for each sigma of Eq. 8."""
    Lx, Ly = 12, 10
    Tc = O.critical_temperature(A_PAPER, B_PAPER, 1.0)
    rv, rl = O.maxwell_coexistence(A_PAPER, B_PAPER, 1.0, 0.344, 0.86 * Tc)
    rho0, fpost, th0 = inputs.random_state(Lx, Ly, rl, rv, 5, seed=21)
    out = {}
    for sigma in sigmas:
        P = O.Params(Lx=Lx, Ly=Ly, bc_y=O.BC_PERIODIC, s_e=s_e, s_z=s_z, sigma=sigma)
        P.finalize(rho0=rho0, rho_v=rv, rho_l=rl)
        ff = O.flow_fields(torch.tensor(fpost, dtype=F64), torch.tensor(th0, dtype=F64), P)
        out[sigma] = torch.einsum('ab,byx->ayx', O.transform_matrix(), O.collide(ff, P))
    return out


@pytest.mark.parametrize("s_e,s_z", [(0.8, 0.8), (0.8, 1.25), (1.4, 0.7)])
def test_sigma_term_of_e_and_zeta_rows(s_e, s_z):
    """The sigma term of Eq. 8 enters the e row as +sigma X/(tau_e - 1/2) and
    the zeta row as -sigma X/(tau_zeta - 1/2) (X = |F_m|^2/psi^2); Eq. 2 then
    scales each by (1 - s/2), and (1 - s/2)/(1/s - 1/2) = s. So the sigma
    part of m*_e is sigma X s_e and that of m*_zeta is -sigma X s_zeta:
    dm*_e/s_e + dm*_zeta/s_zeta = 0 for any rates, which with tau_e =
    tau_zeta says m*_e + m*_zeta is independent of sigma. Both parts are
    linear in sigma, they are not zero where F_m is not, and sigma touches
    no other moment (it only changes the bulk and fourth-order energy
    moments, not mass or momentum)."""
    m = sigma_term_split(s_e, s_z)
    d1 = {s: m[s] - m[0.0] for s in (1.2, 2.5)}
    de, dz = d1[1.2][1], d1[1.2][2]
    assert float(de.abs().max()) > 1e-3 * float(m[0.0][1].abs().max())
    assert torch.allclose(de / s_e + dz / s_z, torch.zeros_like(de), atol=1e-13)
    assert torch.allclose(d1[2.5][1:3], d1[1.2][1:3] * (2.5 / 1.2), atol=1e-13, rtol=1e-11)
    others = [k for k in range(9) if k not in (1, 2)]
    assert torch.allclose(d1[1.2][others], torch.zeros_like(d1[1.2][others]), atol=1e-13)
    if s_e == s_z:
        assert torch.allclose(m[1.2][1] + m[1.2][2], m[0.0][1] + m[0.0][2], atol=1e-13)


def test_stream_pull_bruteforce():
    Ly, Lx = 4, 5
    fpost = torch.arange(9 * Ly * Lx, dtype=F64).view(9, Ly, Lx)
    P = O.Params(Lx=Lx, Ly=Ly, bc_y=O.BC_PERIODIC)
    f = O.stream_pull(fpost, P)
    for a in range(9):
        for y in range(Ly):
            for x in range(Lx):
                assert f[a, y, x] == fpost[a, (y - O.EY[a]) % Ly, (x - O.EX[a]) % Lx]


def test_zou_he_wall_fill_solves_its_conditions():
    """At a wall row the three unknowns solve: zero x and y momentum and
    bounce-back of the normal non-equilibrium parts (u = 0). Solved here as a
    linear system per cell."""
    g = torch.Generator().manual_seed(2)
    Ly, Lx = 5, 6
    fpost = 0.1 + torch.rand(9, Ly, Lx, generator=g, dtype=F64)
    P = O.Params(Lx=Lx, Ly=Ly, bc_y=O.BC_WALLS)
    f = O.wall_fill(O.stream_pull(fpost, P), fpost, P)
    for row, unk, nrm in ((0, (2, 5, 6), (2, 4)), (Ly - 1, (4, 7, 8), (4, 2))):
        for x in range(Lx):
            fk = f[:, row, x].numpy().copy()
            A = np.zeros((3, 3))
            rhs = np.zeros(3)
            for j, a in enumerate(unk):
                A[0, j] = O.EX[a]
                A[1, j] = O.EY[a]
            known = [a for a in range(9) if a not in unk]
            rhs[0] = -sum(O.EX[a] * fk[a] for a in known)
            rhs[1] = -sum(O.EY[a] * fk[a] for a in known)
            A[2, unk.index(nrm[0])] = 1.0
            rhs[2] = fk[nrm[1]]
            sol = np.linalg.solve(A, rhs)
            assert np.allclose(sol, fk[list(unk)], atol=1e-14)


def test_top_outflow_copies_top_row_pull():
    g = torch.Generator().manual_seed(3)
    Ly, Lx = 5, 6
    fpost = torch.rand(9, Ly, Lx, generator=g, dtype=F64)
    P = O.Params(Lx=Lx, Ly=Ly, bc_y=O.BC_TOP_OUTFLOW)
    f = O.wall_fill(O.stream_pull(fpost, P), fpost, P)
    for a in (4, 7, 8):
        for x in range(Lx):
            assert f[a, Ly - 1, x] == fpost[a, Ly - 1, (x - O.EX[a]) % Lx]


def test_interaction_force_taylor_limit():
    """For smooth psi, F_m = -G psi grad psi + O(k^2) (the weights satisfy
    sum_a w_a e_a e_a = I); the error falls 4x when the wavelength doubles."""
    errs = []
    for L in (48, 96):
        P = O.Params(Lx=L, Ly=L, bc_y=O.BC_PERIODIC)
        k = 2 * math.pi / L
        y, x = torch.meshgrid(torch.arange(L, dtype=F64), torch.arange(L, dtype=F64), indexing="ij")
        psi = 1.0 + 0.2 * torch.sin(k * x) * torch.cos(k * y + 0.3)
        dpx = 0.2 * k * torch.cos(k * x) * torch.cos(k * y + 0.3)
        dpy = -0.2 * k * torch.sin(k * x) * torch.sin(k * y + 0.3)
        fx, fy = O.interaction_force(psi, P)
        ex_, ey_ = -P.G * psi * dpx, -P.G * psi * dpy
        scale = float(torch.hypot(ex_, ey_).max())
        errs.append(float(torch.hypot(fx - ex_, fy - ey_).max()) / scale)
    assert errs[0] < 0.01
    assert 3.6 < errs[0] / errs[1] < 4.4


def test_ghost_layer_wall_rows_on_linear_psi():
    """The ghost-layer variant (Sec. 3.2; reading: the ghost row beyond each
    wall copies the wall row's psi). On psi = c + b y, uniform in x, the
    stencil of Eq. 7 gives the exact -G psi b in the interior (it is exact on
    linear fields), and on each wall row, where the ghost row equals the wall
    row, half of it: -G psi (1/3 + 2/12)(psi(1) - psi(0)) = -G psi b / 2.
    F_x vanishes everywhere. A mirrored ghost row (psi(-1) = psi(1)) would
    give 0 on the wall rows and a periodic wrap -G psi (1/2)(psi(1) -
    psi(Ly - 1)); neither matches."""
    for bc in (O.BC_WALLS, O.BC_TOP_OUTFLOW):
        Ly, Lx, c, b = 9, 5, 0.7, 0.05
        P = O.Params(Lx=Lx, Ly=Ly, bc_y=bc, ghost=True)
        psi = (c + b * torch.arange(Ly, dtype=F64)).unsqueeze(1).expand(Ly, Lx).clone()
        fx, fy = O.interaction_force(psi, P)
        want = -P.G * psi * b
        want[0] *= 0.5
        want[-1] *= 0.5
        assert torch.allclose(fy, want, rtol=1e-13, atol=1e-15)
        assert float(fx.abs().max()) < 1e-15


def test_interaction_force_sums_to_zero_periodic():
    g = torch.Generator().manual_seed(4)
    P = O.Params(Lx=7, Ly=9, bc_y=O.BC_PERIODIC)
    psi = torch.rand(9, 7, generator=g, dtype=F64)
    fx, fy = O.interaction_force(psi, P)
    assert abs(float(fx.sum())) < 1e-13 and abs(float(fy.sum())) < 1e-13


def test_adhesion_force_bruteforce():
    """Eq. 22 evaluated cell by cell with an explicit solid mask."""
    g = torch.Generator().manual_seed(5)
    Ly, Lx = 5, 4
    P = O.Params(Lx=Lx, Ly=Ly, bc_y=O.BC_WALLS, Gw=0.1)
    psi = 0.5 + torch.rand(Ly, Lx, generator=g, dtype=F64)
    fx, fy = O.adhesion_force(psi, P)
    for y in range(Ly):
        for x in range(Lx):
            sx = sy = 0.0
            for a in range(1, 9):
                yy = y + O.EY[a]
                solid = 1.0 if yy == 0 else 0.0   # the heating wall row
                omega = (1 / 3 if a < 5 else 1 / 12) / 3.0
                S = float(psi[y, x]) * solid
                sx += omega * S * O.EX[a]
                sy += omega * S * O.EY[a]
            assert abs(float(fx[y, x]) - (-P.Gw * float(psi[y, x]) * sx)) < 1e-15
            assert abs(float(fy[y, x]) - (-P.Gw * float(psi[y, x]) * sy)) < 1e-15
    # on the first fluid row the force points away from the wall for G_w > 0
    assert torch.all(fy[1] > 0)


def test_buoyancy_direction():
    P = O.Params(Lx=1, Ly=2)
    P.rho_ave = 3.0
    _, fy = O.buoyancy(torch.tensor([[0.4], [6.5]], dtype=F64), P)
    assert fy[0, 0] > 0 and fy[1, 0] < 0


def test_tau_nu_endpoints(coex):
    Tc, rv, rl = coex
    P = make(1, 1, None, coex)
    t = O.tau_nu(torch.tensor([0.0, rv, 0.5 * (rv + rl), rl, 9.0], dtype=F64), P)
    assert torch.allclose(t, torch.tensor([1.0, 1.0, 0.9, 0.8, 0.8], dtype=F64), atol=1e-14)


@pytest.mark.parametrize("which", ["liquid", "vapour"])
def test_shear_wave_decay_gives_viscosity(coex, which):
    """A transverse shear wave in uniform fluid decays as exp(-nu k^2 t) with
    nu_L = 0.1 or nu_V = 0.5/3 (Sec. 3.1)."""
    Tc, rv, rl = coex
    rho_val = rl if which == "liquid" else rv
    nu = 0.1 if which == "liquid" else 0.5 / 3
    Ly = 64
    rho0 = np.full((Ly, 1), rho_val, dtype=np.float32)
    P = make(1, Ly, rho0, coex, bc_y=O.BC_PERIODIC, isothermal=True, g=0.0)
    k = 2 * math.pi / Ly
    y = torch.arange(Ly, dtype=F64).view(Ly, 1)
    U = 1e-3
    f, th = O.initial_state(torch.tensor(rho0, dtype=F64), P, vx0=U * torch.sin(k * y))
    n = 600
    for _ in range(n):
        f, th, info = O.step(f, th, P)
    vx = info.fields.vx[:, 0]
    amp = float((vx * torch.sin(k * y[:, 0])).sum() * 2 / Ly)
    expect = U * math.exp(-nu * k * k * (n - 0.5))
    assert abs(amp / expect - 1) < 5e-3


def test_mass_and_momentum_conservation_periodic(coex):
    """Fully periodic domain: total mass is exact, and total post-collision
    momentum changes by the total force, which is zero (F_m in pairs, F_b
    with rho_ave = mean)."""
    Tc, rv, rl = coex
    Lx, Ly = 24, 20
    rho0, fpost, th0 = inputs.random_state(Lx, Ly, rl, rv, 10, seed=11)
    P = make(Lx, Ly, rho0, coex, bc_y=O.BC_PERIODIC)
    f = torch.tensor(fpost, dtype=F64)
    P.rho_ave = float(f.sum(0).mean())
    th = torch.tensor(th0, dtype=F64)
    ex = torch.tensor(O.EX, dtype=F64).view(9, 1, 1)
    ey = torch.tensor(O.EY, dtype=F64).view(9, 1, 1)
    m0 = float(f.sum())
    for _ in range(60):
        px0, py0 = float((ex * f).sum()), float((ey * f).sum())
        f, th, info = O.step(f, th, P)
        ff = info.fields
        assert abs(float(ff.Fx.sum())) < 1e-11 and abs(float(ff.Fy.sum())) < 1e-11
        assert abs(float((ex * f).sum()) - px0) < 1e-11
        assert abs(float((ey * f).sum()) - py0) < 1e-11
    assert abs(float(f.sum()) - m0) < 1e-12 * m0


def test_rest_state_is_fixed_point(coex):
    """Uniform fluid at rest with no force stays exactly at rest."""
    Tc, rv, rl = coex
    rho0 = np.full((6, 5), rl, dtype=np.float32)
    P = make(5, 6, rho0, coex, bc_y=O.BC_PERIODIC, g=3e-5)
    f0, th = O.initial_state(torch.tensor(rho0, dtype=F64), P)
    f1, th1, _ = O.step(f0, th, P)
    assert torch.allclose(f1, f0, atol=1e-14)
    assert torch.allclose(th1, th, atol=1e-16)


def test_flat_interface_coexistence_matches_maxwell(coex):
    """A flat liquid slab relaxes to the Maxwell densities when sigma = 1.2
    with a = 3/49 (the pairing stated after Eq. 21); sigma = 0 does not."""
    Tc, rv, rl = coex
    Ly = 64
    res = {}
    for sigma in (1.2, 0.0):
        rho0 = inputs.slab_density(1, Ly, rl, rv, 16, 48)
        P = make(1, Ly, rho0, coex, bc_y=O.BC_PERIODIC, isothermal=True, g=0.0, sigma=sigma)
        f, th = O.initial_state(torch.tensor(rho0, dtype=F64), P)
        for _ in range(2500):
            f, th, info = O.step(f, th, P)
        r = info.fields.rho[:, 0]
        res[sigma] = (float(r[32]), float(r[0]))
    rl1, rv1 = res[1.2]
    assert abs(rl1 / rl - 1) < 0.005
    assert abs(rv1 / rv - 1) < 0.04
    rl0, rv0 = res[0.0]
    assert abs(rv0 / rv - 1) > 0.3


@pytest.mark.slow
def test_laplace_law_static_droplets(coex):
    """Young-Laplace (Sec. 3.2): the pressure jump across a static droplet,
    p_EOS(rho_in) - p_EOS(rho_out), is linear in 1/R through the origin."""
    Tc, rv, rl = coex
    L = 40
    inv_r, dp = [], []
    for R0 in (7.0, 9.0, 11.0, 13.0):
        rho0 = inputs.droplet_density(L, L, rl, rv, R0)
        P = make(L, L, rho0, coex, bc_y=O.BC_PERIODIC, isothermal=True, g=0.0)
        f, th = O.initial_state(torch.tensor(rho0, dtype=F64), P)
        for _ in range(1500):
            f, th, info = O.step(f, th, P)
        rho = info.fields.rho
        r_in, r_out = float(rho[L // 2, L // 2]), float(rho[0, 0])
        T = torch.tensor(P.Ts, dtype=F64)
        p = lambda r: float(O.pr_pressure(torch.tensor(r, dtype=F64), T, P.a, P.b, P.R, P.omega, P.Tc))
        Req = math.sqrt(float((rho - r_out).sum()) / (math.pi * (r_in - r_out)))
        inv_r.append(1.0 / Req)
        dp.append(p(r_in) - p(r_out))
    slope, icpt = np.polyfit(inv_r, dp, 1)
    pred = slope * np.array(inv_r) + icpt
    r2 = 1 - np.sum((np.array(dp) - pred) ** 2) / np.sum((np.array(dp) - np.mean(dp)) ** 2)
    assert slope > 0
    assert r2 > 0.99
    assert abs(icpt) < 0.1 * max(dp)


# --------------------------------------------------------------------------
# Temperature equation (Eqs. 18-20)
# --------------------------------------------------------------------------

def test_stencils_exact_on_quadratics():
    P = O.Params(Lx=9, Ly=8, bc_y=O.BC_PERIODIC)
    y, x = torch.meshgrid(torch.arange(8, dtype=F64), torch.arange(9, dtype=F64), indexing="ij")
    phi = 0.3 + 1.7 * x - 0.9 * y + 0.25 * x * x - 0.4 * x * y + 0.6 * y * y
    gx, gy = O.grad_iso(phi)
    lap = O.lap_iso(phi)
    inner = (slice(1, -1), slice(1, -1))
    assert torch.allclose(gx[inner], (1.7 + 0.5 * x - 0.4 * y)[inner], atol=1e-12)
    assert torch.allclose(gy[inner], (-0.9 - 0.4 * x + 1.2 * y)[inner], atol=1e-12)
    assert torch.allclose(lap[inner], torch.full_like(lap[inner], 0.5 + 1.2), atol=1e-12)


def test_laplacian_fourier_symbol():
    """lap_iso cos(kx) = 2 (cos k - 1) cos(kx) exactly for the isotropic
    9-point Laplacian."""
    L = 16
    k = 2 * math.pi * 3 / L
    x = torch.arange(L, dtype=F64).view(1, L).expand(5, L)
    phi = torch.cos(k * x)
    assert torch.allclose(O.lap_iso(phi), 2 * (math.cos(k) - 1) * phi, atol=1e-13)


def test_rk4_fourier_mode_closed_form(coex):
    """Pure conduction (v = 0, uniform rho): a Fourier mode is multiplied per
    step by the RK4 stability polynomial R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24,
    z = (c_v chi / c_v) * 2 (cos k - 1)."""
    Tc, rv, rl = coex
    L = 12
    rho0 = np.full((4, L), rl, dtype=np.float32)
    P = make(L, 4, rho0, coex, bc_y=O.BC_PERIODIC)
    rho = torch.tensor(rho0, dtype=F64)
    z0 = torch.zeros_like(rho)
    k = 2 * math.pi / L
    x = torch.arange(L, dtype=F64).view(1, L).expand(4, L)
    th = 1e-3 * torch.cos(k * x)
    z = (P.cv_chi / P.cv) * 2 * (math.cos(k) - 1)
    Rz = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    for n in range(1, 41):
        th = O.rk4_temperature(th, rho, z0, z0, P)
    assert torch.allclose(th, 1e-3 * Rz ** 40 * torch.cos(k * x), atol=1e-17, rtol=1e-12)


def test_linear_conduction_profile_is_steady(coex):
    """Before boiling onset (v = 0, uniform liquid) the linear profile between
    T_b and T_s is an exact fixed point of the discrete temperature update,
    and the wall flux equals lambda * dT/dy exactly."""
    Tc, rv, rl = coex
    Lx, Ly = 6, 11
    rho0 = np.full((Ly, Lx), rl, dtype=np.float32)
    P = make(Lx, Ly, rho0, coex, superheat=0.02)
    rho = torch.tensor(rho0, dtype=F64)
    z0 = torch.zeros_like(rho)
    y = torch.arange(Ly, dtype=F64).view(Ly, 1).expand(Ly, Lx)
    th = 0.02 * (1 - y / (Ly - 1))
    th1 = O.rk4_temperature(th, rho, z0, z0, P)
    assert torch.allclose(th1, th, atol=1e-17)
    qw, q = O.wall_heat_flux(th, rho, P)
    assert abs(float(q) - P.cv_chi * float(rho[0, 0]) * 0.02 / (Ly - 1)) < 1e-16


def test_wall_flux_exact_on_quadratic(coex):
    Tc, rv, rl = coex
    P = make(3, 5, None, coex)
    y = torch.arange(5, dtype=F64).view(5, 1).expand(5, 3)
    th = 0.01 - 0.003 * y + 0.0004 * y * y
    rho = torch.full((5, 3), 2.0, dtype=F64)
    qw, q = O.wall_heat_flux(th, rho, P)
    assert torch.allclose(qw, torch.full((3,), P.cv_chi * 2.0 * 0.003, dtype=F64), atol=1e-17)


def test_isothermal_interface_has_no_spurious_source(coex):
    """Uniform T with a sharp density interface and v = 0: every term of
    Eq. 18 vanishes exactly (the property the hybrid scheme is built for,
    Sec. 1 and Sec. 2)."""
    Tc, rv, rl = coex
    Lx, Ly = 8, 32
    rho0 = inputs.pool_density(Lx, Ly, rl, rv, 16, noise_amp=0.0)
    P = make(Lx, Ly, rho0, coex, bc_y=O.BC_PERIODIC)
    rho = torch.tensor(rho0, dtype=F64)
    z0 = torch.zeros_like(rho)
    th = torch.zeros_like(rho)
    assert torch.equal(O.rk4_temperature(th, rho, z0, z0, P), th)


def test_temperature_rhs_manufactured_solution(coex):
    """Eq. 18 on smooth periodic fields against the continuous right-hand side
    from symbolic differentiation: second-order convergence."""
    import sympy as sp
    Tc, rv, rl = coex
    X, Y = sp.symbols("x y")
    P0 = O.Params(Lx=1, Ly=1)
    P0.finalize(rho_v=rv, rho_l=rl)
    errs = []
    for L in (32, 64):
        k = 2 * sp.pi / L
        rho_s = 3 + 2 * sp.sin(k * X) * sp.cos(k * Y)
        vx_s = 0.01 * sp.cos(k * Y)
        vy_s = 0.02 * sp.sin(k * X + k * Y)
        T_s = P0.Ts * (1 + 0.1 * sp.cos(k * X) * sp.sin(2 * k * Y))
        lam = P0.cv_chi * rho_s
        b, a, R, om = P0.b, P0.a, P0.R, P0.omega
        kap = O.pr_kappa(om)
        Tv = sp.Symbol("Tv", positive=True)
        phi = (1 + kap * (1 - sp.sqrt(Tv / P0.Tc))) ** 2
        p = rho_s * R * Tv / (1 - b * rho_s) - a * phi * rho_s ** 2 / (1 + 2 * b * rho_s - b * b * rho_s ** 2)
        p_T = sp.diff(p, Tv).subs(Tv, T_s)
        K = (-(vx_s * sp.diff(T_s, X) + vy_s * sp.diff(T_s, Y))
             + (sp.diff(lam * sp.diff(T_s, X), X) + sp.diff(lam * sp.diff(T_s, Y), Y)) / (rho_s * P0.cv)
             - T_s / (rho_s * P0.cv) * p_T * (sp.diff(vx_s, X) + sp.diff(vy_s, Y)))
        f = sp.lambdify((X, Y), [rho_s, vx_s, vy_s, T_s, K], "numpy")
        yy, xx = np.mgrid[0:L, 0:L].astype(np.float64)
        rho, vx, vy, T, Kex = [torch.tensor(np.broadcast_to(v, (L, L)).copy(), dtype=F64) for v in f(xx, yy)]
        P = O.Params(Lx=L, Ly=L, bc_y=O.BC_PERIODIC)
        P.finalize(rho_v=rv, rho_l=rl)
        got = O.temperature_rhs(T, O.frozen_flow(rho, vx, vy), P)
        errs.append(float((got - Kex).abs().max() / Kex.abs().max()))
    assert errs[0] < 0.02
    assert 3.5 < errs[0] / errs[1] < 4.5


# --------------------------------------------------------------------------
# Whole step: adjoint by autograd against central differences
# --------------------------------------------------------------------------

def test_autograd_adjoint_matches_central_differences(coex):
    """d(mean q over n steps)/d(theta_b(x)) and d/d(G_w) by autograd through
    the oracle's step agree with central differences of the oracle."""
    Tc, rv, rl = coex
    Lx, Ly, n = 12, 10, 6
    rho0 = inputs.pool_density(Lx, Ly, rl, rv, 5, noise_amp=1e-2, seed=3)

    def J(tb, gw):
        P = make(Lx, Ly, rho0, coex, Gw=0.0)
        P.theta_b = tb
        P.Gw = gw
        f, th = O.initial_state(torch.tensor(rho0, dtype=F64), P)
        qs = []
        for _ in range(n):
            f, th, info = O.step(f, th, P)
            qs.append(info.q)
        return torch.stack(qs).mean()

    tb = torch.full((Lx,), 0.01, dtype=F64, requires_grad=True)
    gw = torch.tensor(0.05, dtype=F64, requires_grad=True)
    val = J(tb, gw)
    gtb, ggw = torch.autograd.grad(val, (tb, gw))
    h = 1e-5
    for x in (0, 5, 11):
        e = torch.zeros(Lx, dtype=F64)
        e[x] = h
        fd = (J(tb.detach() + e, gw.detach()) - J(tb.detach() - e, gw.detach())) / (2 * h)
        assert abs(float(fd) - float(gtb[x])) < 1e-6 * abs(float(gtb[x])) + 1e-12
    fd = (J(tb.detach(), gw.detach() + h) - J(tb.detach(), gw.detach() - h)) / (2 * h)
    assert abs(float(fd) - float(ggw)) < 1e-5 * abs(float(ggw)) + 1e-12


@pytest.mark.filterwarnings("ignore::DeprecationWarning")  # torch scripts a forward-mode helper internally
def test_adjoint_is_transpose_of_tangent_linear_model(coex):
    """Dot-product test of the whole-state adjoint: for the map Phi taking
    (f*, theta) through n steps, <w, J u> from the tangent-linear model
    (forward-mode derivatives) equals <J^T w, u> from the reverse sweep, for
    random u and w, on a heated pool with interface, adhesion and gravity."""
    import torch.autograd.forward_ad as fwAD
    Tc, rv, rl = coex
    Lx, Ly, n = 12, 10, 3
    rho0 = inputs.pool_density(Lx, Ly, rl, rv, 5, noise_amp=1e-2, seed=3)
    P = make(Lx, Ly, rho0, coex, Gw=0.05, superheat=0.02)
    f0, th0 = O.initial_state(torch.tensor(rho0, dtype=F64), P)
    for _ in range(5):
        f0, th0, _ = O.step(f0, th0, P)

    def phi(f, th):
        for _ in range(n):
            f, th, _ = O.step(f, th, P)
        return f, th

    g = torch.Generator().manual_seed(7)
    uf, ut, wf, wt = (torch.randn(t.shape, generator=g, dtype=F64) for t in (f0, th0, f0, th0))
    with fwAD.dual_level():
        fo, to = phi(fwAD.make_dual(f0, uf), fwAD.make_dual(th0, ut))
        jf, jt = fwAD.unpack_dual(fo).tangent, fwAD.unpack_dual(to).tangent
    lhs = float((wf * jf).sum() + (wt * jt).sum())
    fr, tr = f0.clone().requires_grad_(), th0.clone().requires_grad_()
    fo, to = phi(fr, tr)
    gf, gt = torch.autograd.grad((wf * fo).sum() + (wt * to).sum(), (fr, tr))
    rhs = float((gf * uf).sum() + (gt * ut).sum())
    assert abs(lhs) > 1e-3
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
    # the tangent itself against a central difference of Phi along u
    h = 1e-6
    fp, tp = phi(f0 + h * uf, th0 + h * ut)
    fm, tm = phi(f0 - h * uf, th0 - h * ut)
    fd = float((wf * (fp - fm)).sum() + (wt * (tp - tm)).sum()) / (2 * h)
    assert abs(fd - lhs) <= 1e-6 * abs(lhs)


# --------------------------------------------------------------------------
# Seeded input generator
# --------------------------------------------------------------------------

def test_splitmix64_reference_sequence():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.startswith("0x")]
    got = [int(v) for v in inputs.splitmix64(0, np.arange(4))]
    assert got == want
