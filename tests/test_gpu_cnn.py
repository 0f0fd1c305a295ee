"""The learned preconditioner on the GPU, through the C ABI, against the
network oracle (oracle/cnn.py): forward output and parameter gradients
(BF16 storage, FP32 accumulation: relative 2e-2 / 5e-2 in the Frobenius
norm), training reduces the loss, and flexible GCR with the trained network
reaches the FP64 true residual (judged by the FP64 oracle) in fewer
iterations than the same FGCR without it."""
import numpy as np
import pytest

import oracle
from oracle import cnn as ocnn
from paper_1009_5169_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sf():
    from paper_1009_5169_gb300 import binding, build
    build.build()
    return binding


def frob(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _oracle_forward(params, U, r, L, T):
    return np.stack([ocnn.precondition(params, U, r[i], L, T, bf16_acts=True) for i in range(r.shape[0])])


@pytest.mark.parametrize("hidden", [16, 32])
def test_forward_matches_oracle(sf, hidden):
    L, T = 4, 6
    U = inputs.links(L, T, 0.3, 301)
    r = inputs.sources(L, T, 3, 302)
    p = inputs.cnn_init_params(hidden, 303)
    p[-24:] = 0.05 * np.arange(24) / 24          # a non-zero last bias
    net = sf.Cnn(hidden, p)
    lat = sf.Lattice(L, T, 0.5, 0.13, 4.52, U)
    out = np.empty_like(r)
    net.forward(lat, r, out)
    ref = _oracle_forward(inputs.cnn_unflatten(p, hidden), U, r, L, T)
    assert frob(out, ref) <= 2e-2
    assert np.max(np.abs(out - ref)) <= 5e-2 * np.max(np.abs(ref))
    lat.close()
    net.close()


def _even_channels(f, par, V):
    out = np.zeros((V, 24))
    g = f.reshape(-1, 12)
    out[par == 0, 0:24:2] = g.real
    out[par == 0, 1:24:2] = g.imag
    return out


def _oracle_grad(params, U, r, e, L, T):
    """Gradient of mean_b |rh_b + (out(rh_b) - out(-rh_b))/2 - t_b|^2 / |t_b|^2
    over the even sites, rh_b = r_b/s_b, t_b = e_b/s_b, s_b the RMS scale."""
    V = (T - 1) * L ** 3
    par = oracle.parity_of_full_sites(L, T)
    pb = [(ocnn.bf16(W), b) for W, b in params]
    nb = r.shape[0]
    grads_tot = None
    loss = 0.0

    def add(g):
        nonlocal grads_tot
        grads_tot = g if grads_tot is None else [(a[0] + b[0], a[1] + b[1]) for a, b in zip(grads_tot, g)]

    for i in range(nb):
        s = ocnn.rms_scale(r[i])
        op, hp = ocnn.forward(pb, ocnn.features(U, r[i] / s, L, T), L, T, bf16_acts=True, keep=True)
        om, hm = ocnn.forward(pb, ocnn.features(U, -r[i] / s, L, T), L, T, bf16_acts=True, keep=True)
        t = _even_channels(e[i] / s, par, V)
        rh = _even_channels(r[i] / s, par, V)
        diff = (rh + 0.5 * (op - om) - t) * (par == 0)[:, None]
        t2 = np.sum(t ** 2)
        loss += np.sum(diff ** 2) / t2 / nb
        d = 2.0 * diff / (nb * t2)
        add(ocnn.backward(pb, hp, 0.5 * d, L, T)[0])
        add(ocnn.backward(pb, hm, -0.5 * d, L, T)[0])
    return grads_tot, loss


def test_gradients_match_oracle(sf):
    L, T, hidden = 4, 6, 16
    U = inputs.links(L, T, 0.3, 311)
    r = inputs.sources(L, T, 2, 312)
    e = inputs.sources(L, T, 2, 313)
    p = inputs.cnn_init_params(hidden, 314)
    net = sf.Cnn(hidden, p)
    lat = sf.Lattice(L, T, 0.5, 0.13, 4.52, U)
    g, loss = net.gradients(lat, r, e)
    ref, ref_loss = _oracle_grad(inputs.cnn_unflatten(p, hidden), U, r, e, L, T)
    assert abs(loss - ref_loss) <= 1e-2 * ref_loss
    gl = inputs.cnn_unflatten(g, hidden)
    for l, ((dW, db), (rW, rb)) in enumerate(zip(gl, ref)):
        assert frob(dW, rW) <= 5e-2, l
        if np.any(rb != 0):
            assert frob(db, rb) <= 5e-2, l
        else:   # the last bias cancels in the symmetrised output
            assert np.max(np.abs(db)) <= 1e-6 * np.max(np.abs(rW)), l
    lat.close()
    net.close()


def test_residual_gradients_match_oracle(sf):
    """Residual-norm training mode: L = mean_b |r_b - Dhat M(r_b)|^2 / |r_b|^2,
    d L / d M(r_b) = -2 Dhat^dag (r_b - Dhat M(r_b)) / (n |r_b|^2), through the
    network's symmetrised output (oracle Dhat, oracle network)."""
    L, T, hidden, theta, kappa = 4, 6, 16, 0.5, 0.13
    U = inputs.links(L, T, 0.3, 331)
    r = inputs.sources(L, T, 2, 332)
    p = inputs.cnn_init_params(hidden, 333, last_scale=1.0)
    net = sf.Cnn(hidden, p)
    lat = sf.Lattice(L, T, theta, kappa, 4.52, U)
    g, loss = net.gradients(lat, r, None)
    params = inputs.cnn_unflatten(p, hidden)
    pb = [(ocnn.bf16(W), b) for W, b in params]
    V = (T - 1) * L ** 3
    par = oracle.parity_of_full_sites(L, T)
    nb = r.shape[0]
    ref, ref_loss = None, 0.0
    for i in range(nb):
        s = ocnn.rms_scale(r[i])
        op, hp = ocnn.forward(pb, ocnn.features(U, r[i] / s, L, T), L, T, bf16_acts=True, keep=True)
        om, hm = ocnn.forward(pb, ocnn.features(U, -r[i] / s, L, T), L, T, bf16_acts=True, keep=True)
        z = r[i] + s * 0.5 * (ocnn.output_to_even(op, L, T) - ocnn.output_to_even(om, L, T))
        res = r[i] - oracle.apply_dhat(U, z, L, T, theta, kappa)[0]
        r2 = np.sum(np.abs(r[i]) ** 2)
        ref_loss += np.sum(np.abs(res) ** 2) / r2 / nb
        G = -2.0 * oracle.apply_dhat(U, res, L, T, theta, kappa, dagger=True)[0] / (nb * r2)
        dout = _even_channels(G, par, V) * (0.5 * s)
        for hs, sign in ((hp, 1.0), (hm, -1.0)):
            gl = ocnn.backward(pb, hs, sign * dout, L, T)[0]
            ref = gl if ref is None else [(a[0] + b[0], a[1] + b[1]) for a, b in zip(ref, gl)]
    assert abs(loss - ref_loss) <= 2e-2 * ref_loss
    for l, ((dW, db), (rW, rb)) in enumerate(zip(inputs.cnn_unflatten(g, hidden), ref)):
        assert frob(dW, rW) <= 5e-2, l
    lat.close()
    net.close()


def _pairs(sf, lat, L, T, seeds, tol=1e-8):
    """(r, e = Dhat^-1 r) pairs from this library's own solves: X = Dhat^-1 phi
    gives (phi, X); Dhat^dag Y = X gives Dhat (g5 Y) = g5 X, i.e. the pair
    (g5 X, g5 Y) whose residual is smooth, like those a Krylov solver leaves."""
    out = []
    for s in seeds:
        r = inputs.sources(L, T, 5, s)
        x, y = np.empty_like(r), np.empty_like(r)
        sf.solve_block(lat, "mixed_dc", r, x, y, tol=tol, maxiter=4000)
        out.append((r, x))
        out.append((np.ascontiguousarray(oracle.gamma5(x)), np.ascontiguousarray(oracle.gamma5(y))))
    return out


def test_training_and_fgcr_gain(sf):
    L, T, hidden = 8, 8, 16
    lt = inputs.Lattice(L, T, 0.2, 0.13, 321)
    U = lt.make_links()
    lat = sf.Lattice(L, T, lt.theta, lt.kappa, lt.beta, U)
    train = _pairs(sf, lat, L, T, range(400, 412))
    net = sf.Cnn(hidden, inputs.cnn_init_params(hidden, 322))
    losses = []
    for epoch in range(20):
        for r, e in train:
            losses.append(net.train_step(lat, r, None, 1e-3))   # residual-norm loss
    first, last = np.mean(losses[:24]), np.mean(losses[-24:])
    print(f"training loss |r - Dhat M(r)|^2/|r|^2: {first:.4f} -> {last:.4f}")
    assert last < 0.8 * first, (first, last)
    # held-out right-hand sides: FGCR with and without the network
    sf.set_preconditioner(lat, net)
    phi = inputs.sources(L, T, 5, 499)
    X1, Y1 = np.empty_like(phi), np.empty_like(phi)
    i_cnn = sf.solve_block(lat, "fgcr_cnn", phi, X1, Y1, tol=1e-10, maxiter=400)
    X0, Y0 = np.empty_like(phi), np.empty_like(phi)
    i_id = sf.solve_block(lat, "fgcr", phi, X0, Y0, tol=1e-10, maxiter=400)
    for X, Y in ((X1, Y1), (X0, Y0)):
        rx = oracle.true_residual(U, phi, X, L, T, lt.theta, lt.kappa)
        ry = oracle.true_residual(U, X, Y, L, T, lt.theta, lt.kappa, dagger=True)
        assert np.all(rx <= 1.05e-10) and np.all(ry <= 1.05e-10)
    print(f"FGCR iterations X/Y: learned {i_cnn['iters_inner']}/{i_cnn['iters_inner_y']}, "
          f"identity {i_id['iters_inner']}/{i_id['iters_inner_y']}")
    assert i_cnn["iters_inner"] < i_id["iters_inner"], (i_cnn, i_id)
    # the mixed-precision form: FP32 flexible GCR under FP64 defect correction
    res = {}
    for algo in ("fgcr_cnn_mixed", "fgcr_mixed"):
        X, Y = np.empty_like(phi), np.empty_like(phi)
        res[algo] = sf.solve_block(lat, algo, phi, X, Y, tol=1e-10, maxiter=2000)
        rx = oracle.true_residual(U, phi, X, L, T, lt.theta, lt.kappa)
        ry = oracle.true_residual(U, X, Y, L, T, lt.theta, lt.kappa, dagger=True)
        assert np.all(rx <= 1.05e-10) and np.all(ry <= 1.05e-10), (algo, rx, ry)
        assert np.max(np.abs(X - X1)) <= 1e-7 * np.max(np.abs(X1)), algo   # the same solution as the FP64 FGCR
    print(f"mixed FGCR iterations X/Y: learned {res['fgcr_cnn_mixed']['iters_inner']}/"
          f"{res['fgcr_cnn_mixed']['iters_inner_y']}, identity {res['fgcr_mixed']['iters_inner']}/"
          f"{res['fgcr_mixed']['iters_inner_y']}")
    assert res["fgcr_cnn_mixed"]["iters_inner"] < res["fgcr_mixed"]["iters_inner"], res
    lat.close()
    net.close()


@pytest.mark.parametrize("L,T", [(4, 6), (6, 5), (8, 8), (12, 4), (16, 3)])
def test_tcgen05_convolutions_match_mma_sync(sf, L, T):
    """The tcgen05 convolutions (tiles of 16 x2-lines by 8 x3-sites, padded
    and wrapped at L = 4, 6, 12) against the mma.sync kernel on the same
    network: forward output and the parameter gradients (whose backward-data
    convolutions also run on tcgen05).  Both accumulate the same BF16
    products in FP32 in different orders, so the difference is at BF16
    rounding of the intermediate activations."""
    U = inputs.links(L, T, 0.3, 401 + L)
    r = inputs.sources(L, T, 3, 402 + L)
    e = inputs.sources(L, T, 3, 403 + L)
    p = inputs.cnn_init_params(16, 404, last_scale=1.0)
    p[-24:] = 0.05 * np.arange(24) / 24
    lat = sf.Lattice(L, T, 0.5, 0.13, 4.52, U)
    outs, grads = {}, {}
    for impl in ("mma_sync", "tcgen05"):
        net = sf.Cnn(16, p)
        net.set_conv_impl(impl)
        out = np.empty_like(r)
        net.forward(lat, r, out)
        outs[impl] = out
        grads[impl] = net.gradients(lat, r, e)[0]
        net.close()
    lat.close()
    assert frob(outs["tcgen05"], outs["mma_sync"]) <= 5e-3, frob(outs["tcgen05"], outs["mma_sync"])
    assert frob(grads["tcgen05"], grads["mma_sync"]) <= 2e-2, frob(grads["tcgen05"], grads["mma_sync"])


def test_trained_network_checkpoint_round_trip(sf, tmp_path):
    """A network trained a few steps, written to a checkpoint with the links
    and sources and read back into a new network: bitwise the same
    parameters and forward output."""
    from paper_1009_5169_gb300 import checkpoint
    L, T, hidden = 4, 6, 16
    U = inputs.links(L, T, 0.3, 311)
    r = inputs.sources(L, T, 2, 312)
    net = sf.Cnn(hidden, inputs.cnn_init_params(hidden, 313))
    lat = sf.Lattice(L, T, 0.5, 0.13, 4.52, U)
    for _ in range(3):
        net.train_step(lat, r, None, 1e-3)
    path = str(tmp_path / "net.npz")
    checkpoint.save_cnn(path, net, meta={"steps": 3, "seed": 313}, links=U, sources=r)
    net2 = checkpoint.load_cnn(path)
    c = checkpoint.load(path)
    assert c["meta"]["steps"] == 3 and np.array_equal(c["links"], U)
    assert np.array_equal(net2.params(), net.params())
    o1, o2 = np.empty_like(r), np.empty_like(r)
    net.forward(lat, r, o1)
    net2.forward(lat, r, o2)
    assert np.array_equal(o1, o2)
    lat.close()
    net.close()
    net2.close()
