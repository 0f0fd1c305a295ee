"""Pins of the HMC trajectory oracle (gauge force, link exponential,
leapfrog, the Omelyan integrator, the leapfrog on two time scales) against what the mathematics fixes: central
finite differences of the plaquette action (with scipy's expm, not the
oracle's exponential), closed forms of the exponential, the O(dt^2) energy
error of both integrators and their time reversibility, the Omelyan
integrator at lam = 1/2 and the two-scale leapfrog at one substep reducing
to the leapfrog, and their smaller energy errors (the minimum-norm lam at
the same force count; gauge substeps on a field whose gauge action
dominates the error).  A
wrong sign, a dropped staple or a wrong boundary rule in the gauge force
breaks the finite differences; a wrong kick order or sign breaks the dt^2
scaling and reversibility; a misplaced lam breaks the lam = 1/2 reduction or
the comparison with the leapfrog."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import hmc
from paper_1009_5169_gb300 import inputs


def _rotate(U, C, omega):
    """U_mu(x) -> exp(i omega C^a T^a) U_mu(x) where C != 0 (scipy expm)."""
    lam = hmc.gell_mann()
    out = U.copy()
    for x, mu in zip(*np.nonzero(np.any(C != 0, axis=-1))):
        out[x, mu] = scipy.linalg.expm(1j * omega * np.einsum("a,aij->ij", C[x, mu], lam / 2)) @ U[x, mu]
    return out


@pytest.fixture(scope="module")
def gcase():
    L, T, beta = 4, 5, 4.52
    U = inputs.links(L, T, 0.4, 91)
    return dict(L=L, T=T, beta=beta, U=U, F=oracle.gauge_force(U, L, T, beta))


def _fd(c, C, h):
    sp = oracle.plaquette_action(_rotate(c["U"], C, +h), c["L"], c["T"], c["beta"])
    sm = oracle.plaquette_action(_rotate(c["U"], C, -h), c["L"], c["T"], c["beta"])
    return (sp - sm) / (2 * h)


@pytest.mark.parametrize("site,mu", [((0, 1, 2, 3), 0), ((1, 0, 3, 2), 1), ((4, 2, 2, 0), 0),
                                     ((4, 3, 1, 1), 3), ((2, 2, 0, 1), 2)])
def test_gauge_force_single_link_matches_finite_differences(gcase, site, mu):
    c = gcase
    L, T = c["L"], c["T"]
    gi = ((site[0] * L + site[1]) * L + site[2]) * L + site[3]
    C = np.zeros(((T + 1) * L ** 3, 4, 8))
    C[gi, mu] = inputs.su3_directions((), 95 + gi * 4 + mu)
    exact = float(np.sum(C * c["F"]))
    d1, d2 = _fd(c, C, 2e-3), _fd(c, C, 1e-3)
    rich = (4 * d2 - d1) / 3
    assert abs(exact) > 1e-4
    assert abs(rich - exact) <= 1e-8 * abs(exact) + 1e-11


def test_gauge_force_all_links_matches_finite_differences(gcase):
    c = gcase
    L, T = c["L"], c["T"]
    C = inputs.su3_directions(((T + 1) * L ** 3, 4), 96) * hmc.dynamic_mask(L, T)[..., None]
    exact = float(np.sum(C * c["F"]))
    d1, d2 = _fd(c, C, 2e-3), _fd(c, C, 1e-3)
    assert abs((4 * d2 - d1) / 3 - exact) <= 1e-8 * abs(exact)


def test_gauge_force_fixed_links_and_identity_field(gcase):
    """Zero on the fixed boundary links; zero everywhere on the identity field
    (S_g at its minimum)."""
    c = gcase
    L, T = c["L"], c["T"]
    m = hmc.dynamic_mask(L, T)
    assert np.all(c["F"][~m] == 0.0)
    assert np.max(np.abs(c["F"][m])) > 0.1
    U1 = np.zeros_like(c["U"])
    U1[:] = np.eye(3)
    assert np.max(np.abs(oracle.gauge_force(U1, L, T, c["beta"]))) < 1e-14


def test_expi_closed_forms():
    """exp(i dt c lambda^3 / 2) = diag(e^{i dt c/2}, e^{-i dt c/2}, 1); for a
    random Hermitian traceless H the result is unitary with unit determinant
    and matches scipy's expm."""
    c, dt = 0.7, 0.3
    H = c * hmc.gell_mann()[2] / 2
    E = hmc.expi(H, dt)
    assert np.allclose(E, np.diag([np.exp(0.5j * dt * c), np.exp(-0.5j * dt * c), 1.0]), atol=1e-15)
    P = inputs.su3_directions((16,), 97)
    Hs = hmc.algebra(P)
    E = hmc.expi(Hs, dt)
    assert np.allclose(np.einsum("nab,ncb->nac", E, E.conj()), np.eye(3), atol=1e-14)
    assert np.allclose(np.linalg.det(E), 1.0, atol=1e-14)
    for k in range(4):
        assert np.allclose(E[k], scipy.linalg.expm(1j * dt * Hs[k]), atol=1e-14)


@pytest.fixture(scope="module")
def mdcase():
    L, T, theta, kappa, beta = 4, 5, 0.5, 0.12, 4.52
    U = inputs.links(L, T, 0.25, 101)
    P = inputs.su3_directions(((T + 1) * L ** 3, 4), 102)
    eta = inputs.sources(L, T, 2, 103)
    phi = oracle.apply_dhat(U, eta, L, T, theta, kappa)
    return dict(L=L, T=T, theta=theta, kappa=kappa, beta=beta, U=U, P=P, phi=phi, eta=eta)


def _traj(c, nsteps, dt, U=None, P=None):
    return hmc.leapfrog(c["U"] if U is None else U, c["P"] if P is None else P, c["phi"], c["L"], c["T"],
                        c["theta"], c["kappa"], c["beta"], nsteps, dt)


def test_leapfrog_energy_error_is_second_order(mdcase):
    """dH(dt) / dH(dt/2) -> 4 at fixed trajectory length; S_f at the start is
    |eta|^2 (phi = Dhat eta)."""
    c = mdcase
    _, _, h0, h1 = _traj(c, 4, 0.05)
    _, _, g0, g1 = _traj(c, 8, 0.025)
    assert abs(h0[2] - float(np.sum(np.abs(c["eta"]) ** 2))) <= 1e-9 * h0[2]
    dh1 = sum(h1) - sum(h0)
    dh2 = sum(g1) - sum(g0)
    assert abs(dh1) > 1e-6
    assert 3.2 < dh1 / dh2 < 4.8, (dh1, dh2)


def test_leapfrog_is_reversible(mdcase):
    """Integrating back with the momenta negated returns to the start."""
    c = mdcase
    U1, P1, _, _ = _traj(c, 3, 0.05)
    U2, P2, _, _ = _traj(c, 3, 0.05, U=U1, P=-P1)
    m = hmc.dynamic_mask(c["L"], c["T"])
    assert np.max(np.abs(U2 - c["U"])) < 1e-10
    assert np.max(np.abs(-P2[m] - c["P"][m])) < 1e-9


def _om(c, nsteps, dt, U=None, P=None, lam=hmc.OMELYAN_LAMBDA):
    return hmc.omelyan(c["U"] if U is None else U, c["P"] if P is None else P, c["phi"], c["L"], c["T"],
                       c["theta"], c["kappa"], c["beta"], nsteps, dt, lam=lam)


def test_omelyan_with_half_is_leapfrog(mdcase):
    """lam = 1/2: the middle kick vanishes and the two half drifts make one, so
    the trajectory is the leapfrog's of the same step (to rounding)."""
    c = mdcase
    Ua, Pa, a0, a1 = _om(c, 3, 0.05, lam=0.5)
    Ub, Pb, b0, b1 = _traj(c, 3, 0.05)
    m = hmc.dynamic_mask(c["L"], c["T"])
    assert np.max(np.abs(Ua - Ub)) < 1e-13
    assert np.max(np.abs(Pa[m] - Pb[m])) < 1e-12
    assert abs((sum(a1) - sum(a0)) - (sum(b1) - sum(b0))) < 1e-10


def test_omelyan_energy_error_is_second_order(mdcase):
    c = mdcase
    _, _, h0, h1 = _om(c, 4, 0.05)
    _, _, g0, g1 = _om(c, 8, 0.025)
    dh1 = sum(h1) - sum(h0)
    dh2 = sum(g1) - sum(g0)
    assert abs(dh1) > 1e-6
    assert 3.2 < dh1 / dh2 < 4.8, (dh1, dh2)


def test_omelyan_is_reversible(mdcase):
    c = mdcase
    U1, P1, _, _ = _om(c, 3, 0.05)
    U2, P2, _, _ = _om(c, 3, 0.05, U=U1, P=-P1)
    m = hmc.dynamic_mask(c["L"], c["T"])
    assert np.max(np.abs(U2 - c["U"])) < 1e-10
    assert np.max(np.abs(-P2[m] - c["P"][m])) < 1e-9


def test_omelyan_beats_leapfrog_at_equal_force_count(mdcase):
    """The minimum-norm parameter makes the leading error small: with the
    same number of force evaluations (Omelyan, 4 steps of dt: 9; leapfrog, 8
    steps of dt / 2: 9) the energy error is several times smaller."""
    c = mdcase
    _, _, h0, h1 = _om(c, 4, 0.05)
    _, _, g0, g1 = _traj(c, 8, 0.025)
    assert abs(sum(h1) - sum(h0)) < 0.5 * abs(sum(g1) - sum(g0))


def _ts(c, nsteps, dt, m, U=None, P=None):
    return hmc.leapfrog_two_scales(c["U"] if U is None else U, c["P"] if P is None else P, c["phi"], c["L"],
                                   c["T"], c["theta"], c["kappa"], c["beta"], nsteps, dt, m)


def test_two_scales_with_one_substep_is_leapfrog(mdcase):
    c = mdcase
    Ua, Pa, a0, a1 = _ts(c, 3, 0.05, 1)
    Ub, Pb, b0, b1 = _traj(c, 3, 0.05)
    m = hmc.dynamic_mask(c["L"], c["T"])
    assert np.max(np.abs(Ua - Ub)) < 1e-13
    assert np.max(np.abs(Pa[m] - Pb[m])) < 1e-12


def test_two_scales_second_order_and_reversible(mdcase):
    c = mdcase
    _, _, h0, h1 = _ts(c, 4, 0.05, 4)
    _, _, g0, g1 = _ts(c, 8, 0.025, 4)
    dh1, dh2 = sum(h1) - sum(h0), sum(g1) - sum(g0)
    assert abs(dh1) > 1e-6
    assert 3.2 < dh1 / dh2 < 4.8, (dh1, dh2)
    U1, P1, _, _ = _ts(c, 3, 0.05, 3)
    U2, P2, _, _ = _ts(c, 3, 0.05, 3, U=U1, P=-P1)
    m = hmc.dynamic_mask(c["L"], c["T"])
    assert np.max(np.abs(U2 - c["U"])) < 1e-10
    assert np.max(np.abs(-P2[m] - c["P"][m])) < 1e-9


def test_two_scales_shrink_the_gauge_error(mdcase):
    """On this field the gauge force dominates the leapfrog's energy error
    (the plaquette action moves by about 170 over the trajectory, the fermion
    action by 2): four gauge substeps per fermion step cut |dH| several-fold
    at the same number of fermion force evaluations."""
    c = mdcase
    _, _, a0, a1 = _ts(c, 4, 0.05, 1)
    _, _, b0, b1 = _ts(c, 4, 0.05, 4)
    assert abs(sum(b1) - sum(b0)) < 0.25 * abs(sum(a1) - sum(a0))
