"""Pins of the FP64 oracle against what the physics and mathematics fix.

None of these re-types an oracle formula: each compares the oracle with an
independent statement (momentum-space closed form, a symmetry, a dense LU
solve of the operator's own matrix, central finite differences of the action,
closed forms of the plaquette action), so a dropped term, a sign, a transposed
link or a wrong boundary rule in the oracle fails at least one of them.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_1009_5169_gb300 import inputs

# the documented basis (Euclidean, Hermitian, chiral), written independently
I = 1j
GAMMA = {
    0: np.array([[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]], complex),
    1: np.array([[0, 0, 0, I], [0, 0, I, 0], [0, -I, 0, 0], [-I, 0, 0, 0]], complex),
    2: np.array([[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]], complex),
    3: np.array([[0, 0, I, 0], [0, 0, 0, -I], [-I, 0, 0, 0], [0, I, 0, 0]], complex),
}


def _identity_links(L, T):
    U = np.zeros(((T + 1) * L ** 3, 4, 3, 3), complex)
    U[:] = np.eye(3)
    return U


def _inner(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


# ------------------------------------------------------------------ gammas

def test_gamma_clifford_and_basis():
    g = [oracle.gamma(m) for m in range(4)]
    for m in range(4):
        assert np.allclose(g[m], GAMMA[m], atol=0)
        assert np.allclose(g[m], g[m].conj().T, atol=0)
        for n in range(4):
            anti = g[m] @ g[n] + g[n] @ g[m]
            assert np.allclose(anti, 2 * (m == n) * np.eye(4), atol=0)
    g5 = oracle.gamma(4)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]), atol=0)
    for m in range(4):
        assert np.allclose(g5 @ g[m] + g[m] @ g5, 0)


# ------------------------------------------------------- free field (U = 1)

def _free_D_momentum(psi, L, T, theta, kappa):
    """D psi for U = 1 from its momentum-space form: a spatial FFT reduces D
    to a block-tridiagonal operator in x0 with diagonal
    B(p) = 1 - 2 kappa sum_k (cos pt_k - i gamma_k sin pt_k), pt_k = p_k + theta/L,
    and off-diagonals -kappa (1 -+ gamma_0) to x0 +- 1; psi(0) = psi(T) = 0."""
    f = psi.reshape(T - 1, L, L, L, 4, 3)
    ft = np.fft.fftn(f, axes=(1, 2, 3))
    p = 2 * np.pi * np.fft.fftfreq(L) * 1.0  # 2 pi n / L, n in FFT order
    p = 2 * np.pi * np.arange(L) / L
    out = np.zeros_like(ft)
    one = np.eye(4)
    for n1 in range(L):
        for n2 in range(L):
            for n3 in range(L):
                B = one.astype(complex).copy()
                for k, pk in zip((1, 2, 3), (p[n1], p[n2], p[n3])):
                    pt = pk + theta / L
                    B = B - 2 * kappa * (np.cos(pt) * one - 1j * np.sin(pt) * GAMMA[k])
                for t in range(T - 1):
                    v = B @ ft[t, n1, n2, n3]
                    if t + 1 <= T - 2:
                        v = v - kappa * (one - GAMMA[0]) @ ft[t + 1, n1, n2, n3]
                    if t - 1 >= 0:
                        v = v - kappa * (one + GAMMA[0]) @ ft[t - 1, n1, n2, n3]
                    out[t, n1, n2, n3] = v
    return np.fft.ifftn(out, axes=(1, 2, 3)).reshape(psi.shape)


@pytest.mark.parametrize("L,T,theta", [(4, 5, 0.5), (4, 4, 0.0), (6, 4, 1.3)])
def test_free_field_matches_momentum_space(L, T, theta):
    kappa = 0.13
    U = _identity_links(L, T)
    psi = inputs.full_sources(L, T, 1, 11)[0]
    got = oracle.apply_D(U, psi, L, T, theta, kappa)[0]
    ref = _free_D_momentum(psi, L, T, theta, kappa)
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref)) * 10


# ------------------------------------------------------ gamma5-hermiticity

def test_gamma5_hermiticity_D_and_Dhat():
    L, T, theta, kappa = 4, 6, 0.5, 0.13
    U = inputs.links(L, T, 0.4, 21)
    a = inputs.full_sources(L, T, 1, 22)[0]
    b = inputs.full_sources(L, T, 1, 23)[0]
    Db = oracle.apply_D(U, b, L, T, theta, kappa)[0]
    g5Dg5a = oracle.gamma5(oracle.apply_D(U, oracle.gamma5(a), L, T, theta, kappa)[0])
    lhs, rhs = _inner(a, Db), _inner(g5Dg5a, b)
    assert abs(lhs - rhs) <= 1e-14 * abs(lhs) * 10
    ae = inputs.sources(L, T, 1, 24)[0]
    be = inputs.sources(L, T, 1, 25)[0]
    Dhb = oracle.apply_dhat(U, be, L, T, theta, kappa)[0]
    Dhda = oracle.apply_dhat(U, ae, L, T, theta, kappa, dagger=True)[0]
    lhs, rhs = _inner(ae, Dhb), _inner(Dhda, be)
    assert abs(lhs - rhs) <= 1e-14 * abs(lhs) * 10


# ------------------------------------------------------ gauge covariance

def _gauge_transform(U, G, L, T):
    """U'_mu(x) = G(x) U_mu(x) G(x+mu)^dag on the whole gauge lattice
    (time links at x0 = T are not links and are left as they are)."""
    Ug = U.reshape(T + 1, L, L, L, 4, 3, 3)
    Gg = G.reshape(T + 1, L, L, L, 3, 3)
    out = Ug.copy()
    for mu in range(4):
        if mu == 0:
            Gn = np.concatenate([Gg[1:], Gg[:1]], axis=0)  # x0 + 1 (last row unused)
        else:
            Gn = np.roll(Gg, -1, axis=mu)
        out[..., mu, :, :] = Gg @ Ug[..., mu, :, :] @ np.swapaxes(Gn.conj(), -1, -2)
    out[T, :, :, :, 0] = Ug[T, :, :, :, 0]
    return out.reshape(U.shape)


def _apply_G_fermion(G, psi, L, T):
    Gf = G.reshape(T + 1, L ** 3, 3, 3)[1:T].reshape(-1, 3, 3)
    return np.einsum("xab,...xsb->...xsa", Gf, psi)


def test_gauge_covariance_D():
    L, T, theta, kappa = 4, 5, 0.5, 0.13
    U = inputs.links(L, T, 0.5, 31)
    G = inputs.random_su3((T + 1) * L ** 3, 32)
    Up = _gauge_transform(U, G, L, T)
    psi = inputs.full_sources(L, T, 2, 33)
    lhs = oracle.apply_D(Up, _apply_G_fermion(G, psi, L, T), L, T, theta, kappa)
    rhs = _apply_G_fermion(G, oracle.apply_D(U, psi, L, T, theta, kappa), L, T)
    assert np.max(np.abs(lhs - rhs)) <= 1e-13 * np.max(np.abs(rhs))


def _eo_transform(G, x_e, L, T):
    par = oracle.parity_of_full_sites(L, T)
    Gf = G.reshape(T + 1, L ** 3, 3, 3)[1:T].reshape(-1, 3, 3)[par == 0]
    return np.einsum("xab,...xsb->...xsa", Gf, x_e)


def test_gauge_covariance_Dhat_plaquette_and_force():
    L, T, theta, kappa = 4, 5, 0.5, 0.13
    U = inputs.links(L, T, 0.5, 41)
    # make the boundary spatial links non-trivial too, the plaquette sees them
    G = inputs.random_su3((T + 1) * L ** 3, 42)
    Up = _gauge_transform(U, G, L, T)
    x = inputs.sources(L, T, 2, 43)
    y = inputs.sources(L, T, 2, 44)
    lhs = oracle.apply_dhat(Up, _eo_transform(G, x, L, T), L, T, theta, kappa)
    rhs = _eo_transform(G, oracle.apply_dhat(U, x, L, T, theta, kappa), L, T)
    assert np.max(np.abs(lhs - rhs)) <= 1e-13 * np.max(np.abs(rhs))
    # plaquette action is gauge invariant
    s0 = oracle.plaquette_action(U, L, T, 4.52)
    s1 = oracle.plaquette_action(Up, L, T, 4.52)
    assert abs(s0 - s1) <= 1e-12 * abs(s0)
    # force matrix transforms as G(x) F G(x)^dag
    F = oracle.force(U, x, y, L, T, theta, kappa)
    Fp = oracle.force(Up, _eo_transform(G, x, L, T), _eo_transform(G, y, L, T), L, T, theta, kappa)
    lam = _gell_mann()
    Fm = np.einsum("xma,aij->xmij", F, lam / 2)
    Fpm = np.einsum("xma,aij->xmij", Fp, lam / 2)
    Gx = G.reshape(-1, 1, 3, 3)
    rot = Gx @ Fm @ np.swapaxes(Gx.conj(), -1, -2)
    assert np.max(np.abs(Fpm - rot)) <= 1e-13 * np.max(np.abs(Fm))
    assert np.max(np.abs(F)) > 0


# ------------------------------------------------------------ theta twist

def test_uniform_phase_equals_wrap_phase():
    """Uniform e^{i theta/L} per hop equals e^{i theta} on wrapping hops up to
    psi_w(x) = e^{i theta (x1+x2+x3)/L} psi_u(x)."""
    L, T, theta, kappa = 4, 5, 0.7, 0.13
    U = inputs.links(L, T, 0.3, 51)
    chi = inputs.full_sources(L, T, 1, 52)[0]
    c = np.arange(L)
    s = (c[:, None, None] + c[None, :, None] + c[None, None, :]).reshape(-1)
    R = np.tile(np.exp(1j * theta * s / L), T - 1)[:, None, None]
    lhs = oracle.apply_D(U, R * chi, L, T, theta, kappa, theta_mode=1)[0]
    rhs = R * oracle.apply_D(U, chi, L, T, theta, kappa, theta_mode=0)[0]
    assert np.max(np.abs(lhs - rhs)) <= 1e-13 * np.max(np.abs(rhs))
    # and theta does matter
    other = oracle.apply_D(U, chi, L, T, 0.0, kappa)[0]
    assert np.max(np.abs(other - oracle.apply_D(U, chi, L, T, theta, kappa)[0])) > 1e-3


# ------------------------------------------- Schur complement / dense LU

def _dense(op, n):
    eye = np.eye(n, dtype=complex)
    cols = op(eye)  # op maps [n_vec, n] -> [n_vec, n]
    return cols.T


@pytest.fixture(scope="module")
def small():
    L, T, theta, kappa = 4, 4, 0.5, 0.125
    U = inputs.links(L, T, 0.3, 61)
    V = (T - 1) * L ** 3
    Vh = V // 2

    def opD(E):
        return oracle.apply_D(U, E.reshape(-1, V, 4, 3), L, T, theta, kappa).reshape(E.shape[0], -1)

    def opDh(E, dag=False):
        return oracle.apply_dhat(U, E.reshape(-1, Vh, 4, 3), L, T, theta, kappa,
                                 dagger=dag).reshape(E.shape[0], -1)

    D = _dense(opD, V * 12)
    Dh = _dense(opDh, Vh * 12)
    return dict(L=L, T=T, theta=theta, kappa=kappa, U=U, V=V, Vh=Vh, D=D, Dh=Dh)


def test_schur_complement_matches_dense_D(small):
    s = small
    par = oracle.parity_of_full_sites(s["L"], s["T"])
    idx = np.arange(s["V"] * 12).reshape(s["V"], 12)
    e = idx[par == 0].reshape(-1)
    o = idx[par == 1].reshape(-1)
    D = s["D"]
    assert np.allclose(D[np.ix_(o, o)], np.eye(o.size), atol=0)
    schur = D[np.ix_(e, e)] - D[np.ix_(e, o)] @ np.linalg.solve(D[np.ix_(o, o)], D[np.ix_(o, e)])
    assert np.max(np.abs(schur - s["Dh"])) <= 1e-14
    # det D = det Dhat (D_oo = 1)
    sd, ld = np.linalg.slogdet(D)
    sh, lh = np.linalg.slogdet(s["Dh"])
    assert abs(ld - lh) <= 1e-10 * abs(ld) + 1e-10
    assert abs(sd - sh) <= 1e-9


def test_bicgstab_matches_dense_lu(small):
    s = small
    b = inputs.sources(s["L"], s["T"], 2, 62)
    x, it, res = oracle.bicgstab(s["U"], b, s["L"], s["T"], s["theta"], s["kappa"], tol=1e-13)
    assert np.all(res <= 1e-13) and np.all(it > 0)
    for i in range(2):
        ref = scipy.linalg.lu_solve(scipy.linalg.lu_factor(s["Dh"]), b[i].reshape(-1))
        err = np.linalg.norm(x[i].reshape(-1) - ref) / np.linalg.norm(ref)
        assert err <= 1e-11
    y, it, res = oracle.bicgstab(s["U"], x, s["L"], s["T"], s["theta"], s["kappa"], tol=1e-13,
                                 dagger=True)
    for i in range(2):
        ref = np.linalg.solve(s["Dh"].conj().T, x[i].reshape(-1))
        err = np.linalg.norm(y[i].reshape(-1) - ref) / np.linalg.norm(ref)
        assert err <= 1e-11


def test_full_solve_via_even_odd(small):
    """x = D^-1 phi from the even/odd route: Dhat x_e = phi_e + kappa H_eo phi_o,
    x_o = phi_o + kappa H_oe x_e, against the dense full solve."""
    s = small
    L, T, kp = s["L"], s["T"], s["kappa"]
    phi = inputs.full_sources(L, T, 1, 63)
    ref = np.linalg.solve(s["D"], phi[0].reshape(-1)).reshape(s["V"], 4, 3)
    pe, po = oracle.split_eo(phi, L, T)
    Hpo = oracle.hop(s["U"], oracle.join_eo(np.zeros_like(pe), po, L, T), L, T, s["theta"])
    rhs = pe + kp * oracle.split_eo(Hpo, L, T)[0]
    xe, _, _ = oracle.bicgstab(s["U"], rhs, L, T, s["theta"], kp, tol=1e-13)
    Hxe = oracle.hop(s["U"], oracle.join_eo(xe, np.zeros_like(po), L, T), L, T, s["theta"])
    xo = po + kp * oracle.split_eo(Hxe, L, T)[1]
    x = oracle.join_eo(xe, xo, L, T)[0]
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-11


# ------------------------------------------------------ force vs FD of S

def _gell_mann():
    lam = np.zeros((8, 3, 3), complex)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return lam


def _action_dense(U, phi, L, T, theta, kappa):
    """S = sum_i |Dhat^-1 phi_i|^2 via a dense LU of Dhat (Eq. 2)."""
    Vh = (T - 1) * L ** 3 // 2
    eye = np.eye(Vh * 12, dtype=complex)
    Dh = oracle.apply_dhat(U, eye.reshape(-1, Vh, 4, 3), L, T, theta, kappa).reshape(Vh * 12, -1).T
    x = np.linalg.solve(Dh, phi.reshape(phi.shape[0], -1).T)
    return float(np.sum(np.abs(x) ** 2)), x.T.reshape(phi.shape), Dh


def _rotate(U, C, omega):
    """U_mu(x) -> exp(i omega C^a T^a) U_mu(x) for every link with C != 0."""
    lam = _gell_mann()
    out = U.copy()
    nz = np.nonzero(np.any(C != 0, axis=-1))
    for x, mu in zip(*nz):
        A = np.einsum("a,aij->ij", C[x, mu], lam / 2)
        out[x, mu] = scipy.linalg.expm(1j * omega * A) @ U[x, mu]
    return out


@pytest.fixture(scope="module")
def force_case():
    L, T, theta, kappa = 4, 5, 0.5, 0.12
    U = inputs.links(L, T, 0.35, 71)
    phi = inputs.sources(L, T, 2, 72)
    S, X, Dh = _action_dense(U, phi, L, T, theta, kappa)
    Y = np.linalg.solve(Dh.conj().T, X.reshape(2, -1).T).T.reshape(X.shape)
    F = oracle.force(U, X, Y, L, T, theta, kappa)
    return dict(L=L, T=T, theta=theta, kappa=kappa, U=U, phi=phi, F=F)


def _fd(case, C, h):
    L, T, th, kp = case["L"], case["T"], case["theta"], case["kappa"]
    sp = _action_dense(_rotate(case["U"], C, +h), case["phi"], L, T, th, kp)[0]
    sm = _action_dense(_rotate(case["U"], C, -h), case["phi"], L, T, th, kp)[0]
    return (sp - sm) / (2 * h)


def _fd_richardson(case, C, h=2e-3):
    d1 = _fd(case, C, h)
    d2 = _fd(case, C, h / 2)
    return (4 * d2 - d1) / 3, d1, d2


@pytest.mark.parametrize("site,mu", [((2, 1, 3, 0), 0), ((3, 2, 0, 3), 2), ((1, 0, 0, 1), 1),
                                     ((4, 3, 3, 3), 3), ((1, 1, 2, 3), 0)])
def test_force_single_link_matches_finite_differences(force_case, site, mu):
    c = force_case
    L, T = c["L"], c["T"]
    gi = ((site[0] * L + site[1]) * L + site[2]) * L + site[3]
    C = np.zeros(((T + 1) * L ** 3, 4, 8))
    C[gi, mu] = inputs.su3_directions((), 73 + gi * 4 + mu)
    exact = float(np.sum(C * c["F"]))
    rich, d1, d2 = _fd_richardson(c, C)
    assert abs(exact) > 1e-6
    assert abs(rich - exact) <= 1e-8 * abs(exact) + 1e-11
    # the plain central difference converges at O(h^2)
    assert abs(d2 - exact) < abs(d1 - exact) / 3


def test_force_all_links_matches_finite_differences(force_case):
    c = force_case
    L, T = c["L"], c["T"]
    C = inputs.su3_directions(((T + 1) * L ** 3, 4), 74)
    exact = float(np.sum(C * c["F"]))
    rich, d1, d2 = _fd_richardson(c, C)
    assert abs(rich - exact) <= 1e-8 * abs(exact)


def test_force_zero_on_links_without_fermion_support(force_case):
    c = force_case
    L, T = c["L"], c["T"]
    F = c["F"].reshape(T + 1, L ** 3, 4, 8)
    assert np.all(F[0] == 0) and np.all(F[T] == 0)          # boundary slices
    assert np.all(F[T - 1, :, 0] == 0)                        # time link into x0 = T
    assert np.max(np.abs(F[1:T - 1, :, 0])) > 0
    assert np.max(np.abs(F[T - 1, :, 1:])) > 0


# ------------------------------------------------------ plaquette action

def test_plaquette_closed_forms():
    L, T, beta = 4, 5, 4.52
    U = _identity_links(L, T)
    assert oracle.plaquette_action(U, L, T, beta) == 0.0
    A = inputs.gaussian_traceless_hermitian(inputs.rng(81, 0), ())
    E = scipy.linalg.expm(0.7j * A)
    one = 1 - np.real(np.trace(E)) / 3

    def with_link(x0, mu):
        V = U.copy()
        gi = ((x0 * L + 1) * L + 2) * L + 3
        V[gi, mu] = E
        return oracle.plaquette_action(V, L, T, beta)

    # bulk spatial link: 6 plaquettes of weight 1
    assert abs(with_link(2, 1) - 6 * beta * one) <= 1e-13
    # bulk time link: 6 plaquettes of weight 1
    assert abs(with_link(2, 0) - 6 * beta * one) <= 1e-13
    # boundary spatial link at x0 = 0: 4 spatial plaquettes of weight 1/2 and 1 time-like
    assert abs(with_link(0, 2) - 3 * beta * one) <= 1e-13
    # boundary spatial link at x0 = T: same
    assert abs(with_link(T, 3) - 3 * beta * one) <= 1e-13
    # time link at x0 = 0: 6 time-like plaquettes
    assert abs(with_link(0, 0) - 6 * beta * one) <= 1e-13
    # the non-link U_0 at x0 = T is never used
    assert with_link(T, 0) == 0.0


def test_links_are_su3():
    U = inputs.links(4, 4, 0.3, 91)
    M = U.reshape(-1, 3, 3)
    err = np.max(np.abs(M.conj().transpose(0, 2, 1) @ M - np.eye(3)))
    assert err < 1e-14
    assert np.max(np.abs(np.linalg.det(M) - 1)) < 1e-14
