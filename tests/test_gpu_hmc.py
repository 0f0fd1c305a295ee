"""GPU parity of the HMC trajectory pieces (gauge force, link update, the
leapfrog, two-time-scale and Omelyan trajectories around Alg. 2) against the
FP64 oracle, through the C ABI.

Tolerances: the gauge force and the link exponential are single FP64
evaluations (1e-12 / 1e-13 relative); the trajectory composes solves to
1e-12, so links, momenta and the Hamiltonian parts agree to about 1e-9.
"""
import numpy as np
import pytest

import oracle
from oracle import hmc
from paper_1009_5169_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sf():
    from paper_1009_5169_gb300 import binding, build
    build.build()
    return binding


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _lat(sf, U, L, T, theta=0.5, kappa=0.12, beta=4.52):
    return sf.Lattice(L, T, theta, kappa, beta, torch.from_numpy(U).cuda())


def test_gauge_force_matches_oracle(sf):
    L, T, beta = 6, 7, 4.52
    U = inputs.links(L, T, 0.4, 111)
    lat = _lat(sf, U, L, T, beta=beta)
    F = torch.full(((T + 1) * L ** 3, 4, 8), 7.0, dtype=torch.float64, device="cuda")
    mom = torch.ones_like(F)
    sf.gauge_force(lat, F, mom, eps=0.3)
    Fo = oracle.gauge_force(U, L, T, beta)
    assert relerr(F.cpu().numpy(), Fo) <= 1e-12
    assert relerr(mom.cpu().numpy(), 1.0 - 0.3 * Fo) <= 1e-14
    assert np.all(F.cpu().numpy()[~hmc.dynamic_mask(L, T)] == 0.0)
    lat.close()


def test_link_update_matches_oracle(sf):
    """U <- exp(i dt P) U on the dynamic links; the fixed links do not move;
    the updated field stays in SU(3) and the prepared copies follow it (Dhat
    with the new links matches the oracle's)."""
    L, T, dt = 4, 6, 0.37
    U = inputs.links(L, T, 0.3, 112)
    P = inputs.su3_directions(((T + 1) * L ** 3, 4), 113) * 2.0  # some links need scaling and squaring
    lat = _lat(sf, U, L, T)
    sf.update_links(lat, torch.from_numpy(P).cuda(), dt)
    out = torch.empty(((T + 1) * L ** 3, 4, 3, 3), dtype=torch.complex128, device="cuda")
    sf.get_links(lat, out)
    Ug = out.cpu().numpy()
    Uo = hmc.update_links(U, P, dt, L, T)
    assert relerr(Ug, Uo) <= 1e-13
    m = hmc.dynamic_mask(L, T)
    assert np.array_equal(Ug[~m], U[~m])
    x = inputs.sources(L, T, 2, 114)
    y = torch.empty((2, (T - 1) * L ** 3 // 2, 4, 3), dtype=torch.complex128, device="cuda")
    sf.wilson_apply_block(lat, "dhat", "fp64", torch.from_numpy(x).cuda(), y)
    assert relerr(y.cpu().numpy(), oracle.apply_dhat(Uo, x, L, T, 0.5, 0.12)) <= 1e-12
    lat.close()


@pytest.fixture(scope="module")
def mdcase():
    L, T, theta, kappa, beta = 4, 5, 0.5, 0.12, 4.52
    U = inputs.links(L, T, 0.25, 101)
    P = inputs.su3_directions(((T + 1) * L ** 3, 4), 102)
    eta = inputs.sources(L, T, 2, 103)
    phi = oracle.apply_dhat(U, eta, L, T, theta, kappa)
    return dict(L=L, T=T, theta=theta, kappa=kappa, beta=beta, U=U, P=P, phi=phi)


@pytest.mark.parametrize("algo", ["mixed_dc", "cg_normal"])
def test_md_trajectory_matches_oracle_leapfrog(sf, mdcase, algo):
    """The whole trajectory (gauge + fermion forces, link updates, the
    Hamiltonian at both ends) against the oracle's leapfrog on the same
    inputs."""
    c = mdcase
    L, T = c["L"], c["T"]
    Uo, Po, h0, h1 = hmc.leapfrog(c["U"], c["P"], c["phi"], L, T, c["theta"], c["kappa"], c["beta"], 3, 0.05)
    lat = _lat(sf, c["U"], L, T, c["theta"], c["kappa"], c["beta"])
    mom = torch.from_numpy(c["P"].copy()).cuda()
    info = sf.md_trajectory(lat, algo, torch.from_numpy(c["phi"]).cuda(), mom, 3, 0.05, tol=1e-12)
    assert info["force_evals"] == 4
    out = torch.empty(((T + 1) * L ** 3, 4, 3, 3), dtype=torch.complex128, device="cuda")
    sf.get_links(lat, out)
    assert relerr(out.cpu().numpy(), Uo) <= 1e-9
    assert relerr(mom.cpu().numpy(), Po) <= 1e-8
    for k in range(3):
        assert abs(info["kinetic"][0] - h0[0]) <= 1e-12 * h0[0]
        assert abs([info["kinetic"], info["s_gauge"], info["s_fermion"]][k][1] - h1[k]) <= 1e-9 * abs(h1[k])
    assert abs(info["dH"] - (sum(h1) - sum(h0))) <= 1e-7
    lat.close()


@pytest.mark.parametrize("algo", ["mixed_dc", "cg_normal"])
def test_md_trajectory_matches_oracle_omelyan(sf, mdcase, algo):
    """The Omelyan (second-order minimum-norm) trajectory against the oracle's
    on the same inputs: two force evaluations per step."""
    c = mdcase
    L, T = c["L"], c["T"]
    Uo, Po, h0, h1 = hmc.omelyan(c["U"], c["P"], c["phi"], L, T, c["theta"], c["kappa"], c["beta"], 3, 0.05)
    lat = _lat(sf, c["U"], L, T, c["theta"], c["kappa"], c["beta"])
    mom = torch.from_numpy(c["P"].copy()).cuda()
    info = sf.md_trajectory(lat, algo, torch.from_numpy(c["phi"]).cuda(), mom, 3, 0.05, tol=1e-12,
                            integrator="omelyan")
    assert info["force_evals"] == 7
    out = torch.empty(((T + 1) * L ** 3, 4, 3, 3), dtype=torch.complex128, device="cuda")
    sf.get_links(lat, out)
    assert relerr(out.cpu().numpy(), Uo) <= 1e-9
    assert relerr(mom.cpu().numpy(), Po) <= 1e-8
    for k in range(3):
        assert abs([info["kinetic"], info["s_gauge"], info["s_fermion"]][k][1] - h1[k]) <= 1e-9 * abs(h1[k])
    assert abs(info["dH"] - (sum(h1) - sum(h0))) <= 1e-7
    lat.close()


@pytest.mark.parametrize("algo", ["mixed_dc", "cg_normal"])
def test_md_trajectory_matches_oracle_two_scales(sf, mdcase, algo):
    """The leapfrog with the gauge force on 3 substeps of each step against
    the oracle's nested leapfrog; the fermion force is evaluated nsteps + 1
    times."""
    c = mdcase
    L, T = c["L"], c["T"]
    Uo, Po, h0, h1 = hmc.leapfrog_two_scales(c["U"], c["P"], c["phi"], L, T, c["theta"], c["kappa"], c["beta"],
                                             3, 0.05, 3)
    lat = _lat(sf, c["U"], L, T, c["theta"], c["kappa"], c["beta"])
    mom = torch.from_numpy(c["P"].copy()).cuda()
    info = sf.md_trajectory(lat, algo, torch.from_numpy(c["phi"]).cuda(), mom, 3, 0.05, tol=1e-12,
                            gauge_substeps=3)
    assert info["force_evals"] == 4
    out = torch.empty(((T + 1) * L ** 3, 4, 3, 3), dtype=torch.complex128, device="cuda")
    sf.get_links(lat, out)
    assert relerr(out.cpu().numpy(), Uo) <= 1e-9
    assert relerr(mom.cpu().numpy(), Po) <= 1e-8
    for k in range(3):
        assert abs([info["kinetic"], info["s_gauge"], info["s_fermion"]][k][1] - h1[k]) <= 1e-9 * abs(h1[k])
    assert abs(info["dH"] - (sum(h1) - sum(h0))) <= 1e-7
    lat.close()


def test_two_scales_with_one_substep_is_the_leapfrog(sf, mdcase):
    """gauge_substeps = 1 runs the same kicks and drifts in the same order as
    sf_md_trajectory: bitwise the same links and momenta."""
    c = mdcase
    L, T = c["L"], c["T"]
    outs = []
    for fn in ("leapfrog", "two_scales"):
        lat = _lat(sf, c["U"], L, T, c["theta"], c["kappa"], c["beta"])
        mom = torch.from_numpy(c["P"].copy()).cuda()
        phi = torch.from_numpy(c["phi"]).cuda()
        if fn == "leapfrog":
            sf.md_trajectory(lat, "cg_normal", phi, mom, 2, 0.05, tol=1e-12)
        else:
            n = sf.lib().sf_md_trajectory_two_scales(lat.handle, sf.ALGOS["cg_normal"], 2, sf._ptr(phi),
                                                     sf._ptr(mom), 2, 0.05, 1, 1e-12, 10000, None)
            assert n == 0
        out = torch.empty(((T + 1) * L ** 3, 4, 3, 3), dtype=torch.complex128, device="cuda")
        sf.get_links(lat, out)
        outs.append((out.cpu().numpy(), mom.cpu().numpy()))
        lat.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_integrators_reject_bad_parameters(sf, mdcase):
    c = mdcase
    lat = _lat(sf, c["U"], c["L"], c["T"], c["theta"], c["kappa"], c["beta"])
    mom = torch.from_numpy(c["P"].copy()).cuda()
    for lam in (0.0, 0.5, -0.1, 0.7):
        with pytest.raises(sf.SFError):
            sf.md_trajectory(lat, "cg_normal", torch.from_numpy(c["phi"]).cuda(), mom, 1, 0.05,
                             integrator="omelyan", lam=lam)
    for m in (0, -2, 1001):
        with pytest.raises(sf.SFError):
            sf.md_trajectory(lat, "cg_normal", torch.from_numpy(c["phi"]).cuda(), mom, 1, 0.05, gauge_substeps=m)
    assert np.array_equal(mom.cpu().numpy(), c["P"])
    lat.close()


def test_md_trajectory_reversible_and_second_order(sf):
    """On 6^3 x 6 with 3 pseudo-fermions: integrating back with the momenta
    negated returns to the start (to the solver tolerance), and dH shrinks
    by about 4 when dt halves at fixed trajectory length."""
    L, T, theta, kappa, beta = 6, 6, 0.5, 0.13, 4.52
    U = inputs.links(L, T, 0.25, 121)
    P = inputs.su3_directions(((T + 1) * L ** 3, 4), 122)
    lat = _lat(sf, U, L, T, theta, kappa, beta)
    eta = torch.from_numpy(inputs.sources(L, T, 3, 123)).cuda()
    phi = torch.empty_like(eta)
    sf.wilson_apply_block(lat, "dhat", "fp64", eta, phi)
    mom = torch.from_numpy(P.copy()).cuda()
    d1 = sf.md_trajectory(lat, "cg_normal", phi, mom, 4, 0.04, tol=1e-12)
    assert abs(d1["s_fermion"][0] - float((eta.abs() ** 2).sum())) <= 1e-9 * d1["s_fermion"][0]
    mom.neg_()
    sf.md_trajectory(lat, "cg_normal", phi, mom, 4, 0.04, tol=1e-12)
    out = torch.empty(((T + 1) * L ** 3, 4, 3, 3), dtype=torch.complex128, device="cuda")
    sf.get_links(lat, out)
    assert np.max(np.abs(out.cpu().numpy() - U)) < 1e-9
    m = hmc.dynamic_mask(L, T)
    assert np.max(np.abs(-mom.cpu().numpy()[m] - P[m])) < 1e-8
    lat.set_links(torch.from_numpy(U).cuda())
    mom = torch.from_numpy(P.copy()).cuda()
    d2 = sf.md_trajectory(lat, "cg_normal", phi, mom, 8, 0.02, tol=1e-12)
    assert 3.2 < d1["dH"] / d2["dH"] < 4.8, (d1["dH"], d2["dH"])
    lat.close()


def test_hmc_trajectory_metropolis(sf):
    """sf_hmc_trajectory (phi = Dhat eta, MD, Metropolis in the library).
    Accepted: the links moved; rejected (uniform above exp(-dH)): the links
    are restored exactly, for the leapfrog and the Omelyan integrator."""
    L, T = 4, 5
    U = inputs.links(L, T, 0.25, 131)
    P = inputs.su3_directions(((T + 1) * L ** 3, 4), 132)
    eta = torch.from_numpy(inputs.sources(L, T, 2, 133)).cuda()
    lat = _lat(sf, U, L, T)
    out = torch.empty(((T + 1) * L ** 3, 4, 3, 3), dtype=torch.complex128, device="cuda")
    d = sf.hmc_trajectory(lat, "mixed_dc", eta, torch.from_numpy(P.copy()).cuda(), 0.0, 3, 0.05)
    assert d["accepted"]
    sf.get_links(lat, out)
    assert np.max(np.abs(out.cpu().numpy() - U)) > 1e-3
    lat.set_links(torch.from_numpy(U).cuda())
    d = sf.hmc_trajectory(lat, "mixed_dc", eta, torch.from_numpy(P.copy()).cuda(), 1.0 + 1e-9, 3, 0.05)
    assert not d["accepted"]
    sf.get_links(lat, out)
    assert np.array_equal(out.cpu().numpy(), U)
    # the Omelyan integrator through the same call; rejected: the links are restored exactly
    d = sf.hmc_trajectory(lat, "cg_normal", eta, torch.from_numpy(P.copy()).cuda(), 1.0 + 1e-9, 2, 0.05,
                          integrator="omelyan")
    assert not d["accepted"] and d["force_evals"] == 5
    sf.get_links(lat, out)
    assert np.array_equal(out.cpu().numpy(), U)
    with pytest.raises(sf.SFError):
        sf.hmc_trajectory(lat, "cg_normal", eta, torch.from_numpy(P.copy()).cuda(), 0.5, 2, 0.05,
                          integrator="omelyan", lam=0.6)
    lat.close()
