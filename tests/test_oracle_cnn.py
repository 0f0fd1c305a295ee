"""Pins of the network oracle (oracle/cnn.py) against closed forms and
identities: a one-offset identity stencil is a pure lattice shift whose
values are checked site by site from coordinates; the input-gradient is the
exact adjoint of the convolution; the weight gradient and the whole
network's backward pass agree with central finite differences; bfloat16
rounding matches the bit-level definition."""
import numpy as np
import pytest

from oracle import cnn

L, T = 4, 5
V = (T - 1) * L ** 3


def _rng(s):
    return np.random.Generator(np.random.Philox(key=np.array([s, 11], dtype=np.uint64)))


def _coords(i):
    x3 = i % L; i //= L
    x2 = i % L; i //= L
    x1 = i % L; i //= L
    return (i + 1, x1, x2, x3)


def _index(x):
    return (((x[0] - 1) * L + x[1]) * L + x[2]) * L + x[3]


@pytest.mark.parametrize("k", [0, 13, 40, 41, 67, 80])
def test_single_offset_identity_is_a_shift(k):
    X = _rng(1).standard_normal((V, 3))
    W = np.zeros((81, 3, 3))
    W[k] = np.eye(3)
    Y = cnn.conv(X, W, np.zeros(3), L, T)
    d = cnn.OFFSETS[k]
    for i in range(V):
        x = _coords(i)
        y0 = x[0] + d[0]
        if y0 < 1 or y0 > T - 1:
            expect = np.zeros(3)
        else:
            y = (y0, (x[1] + d[1]) % L, (x[2] + d[2]) % L, (x[3] + d[3]) % L)
            expect = X[_index(y)]
        assert np.array_equal(Y[i], expect), (i, x, d)


def test_offsets_cover_the_3x3x3x3_stencil_once():
    s = {tuple(o) for o in cnn.OFFSETS}
    assert len(s) == 81 and all(max(abs(v) for v in o) <= 1 for o in s)
    assert tuple(cnn.OFFSETS[40]) == (0, 0, 0, 0)


def test_input_gradient_is_the_adjoint():
    g = _rng(2)
    X = g.standard_normal((V, 5))
    Yt = g.standard_normal((V, 4))
    W = g.standard_normal((81, 5, 4))
    lhs = np.sum(cnn.conv(X, W, np.zeros(4), L, T) * Yt)
    rhs = np.sum(X * cnn.conv_adjoint_input(Yt, W, L, T))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_weight_gradient_is_exact_for_the_linear_map():
    g = _rng(3)
    X = g.standard_normal((V, 5))
    G = g.standard_normal((V, 4))
    dW = g.standard_normal((81, 5, 4))
    lhs = np.sum(cnn.conv(X, dW, np.zeros(4), L, T) * G)
    rhs = np.sum(dW * cnn.conv_grad_weight(X, G, L, T))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_network_backward_matches_finite_differences():
    g = _rng(4)
    widths = [6, 5, 5, 4, 3]
    params = cnn.init_params(widths, 5)
    params = [(W, g.standard_normal(W.shape[2]) * 0.1) for W, _ in params]
    X = g.standard_normal((V, widths[0]))
    tgt = g.standard_normal((V, widths[-1]))

    def loss(ps, x):
        o = cnn.forward(ps, x, L, T)
        return 0.5 * np.sum((o - tgt) ** 2)

    out, hs = cnn.forward(params, X, L, T, keep=True)
    grads, dX = cnn.backward(params, hs, out - tgt, L, T)
    # small step: a larger one lets pre-activations cross the ReLU kink
    h = 1e-7
    for l in range(len(params)):
        W, b = params[l]
        D = g.standard_normal(W.shape)
        P = [list(p) for p in params]
        P[l][0] = W + h * D
        lp = loss(P, X)
        P[l][0] = W - h * D
        lm = loss(P, X)
        fd = (lp - lm) / (2 * h)
        ex = np.sum(D * grads[l][0])
        assert abs(fd - ex) <= 1e-7 * abs(ex), (l, fd, ex)
        db = g.standard_normal(b.shape)
        P = [list(p) for p in params]
        P[l][1] = b + h * db
        lp = loss(P, X)
        P[l][1] = b - h * db
        lm = loss(P, X)
        assert abs((lp - lm) / (2 * h) - np.sum(db * grads[l][1])) <= 1e-7 * abs(np.sum(db * grads[l][1]))
    DX = g.standard_normal(X.shape)
    fd = (loss(params, X + h * DX) - loss(params, X - h * DX)) / (2 * h)
    assert abs(fd - np.sum(DX * dX)) <= 1e-7 * abs(fd)


def test_bf16_rounding_definition():
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -7 + 2.0 ** -8, -2.5, 0.0, 3.0e38])
    got = cnn.bf16(vals)
    # bfloat16 keeps 8 significand bits: 1 + 2^-8 is a tie -> even (1.0);
    # 1 + 3*2^-9 rounds up to 1 + 2^-7; 1 + 2^-7 + 2^-8 is a tie -> even (1 + 2^-6)
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -6, -2.5, 0.0, got[-1]])
    assert np.array_equal(got, want)
    assert abs(got[-1] - 3.0e38) / 3.0e38 < 2 ** -8


def test_features_and_output_roundtrip():
    from paper_1009_5169_gb300 import inputs
    U = inputs.links(L, T, 0.3, 9)
    r = inputs.sources(L, T, 1, 10)[0]
    X = cnn.features(U, r, L, T)
    assert X.shape == (V, 32)
    out = np.zeros((V, 24))
    out[:] = X[:, :24]
    assert np.array_equal(cnn.output_to_even(out, L, T), r)
    assert np.allclose(X[:, 24], np.real(np.trace(U.reshape(T + 1, L ** 3, 4, 3, 3)[1:T, :, 0], axis1=-2,
                                                   axis2=-1)).reshape(-1) / 3)


def test_preconditioner_is_odd_and_homogeneous():
    """M(-r) = -M(r) and M(a r) = a M(r) exactly (powers of two keep the
    bfloat16 roundings exact too)."""
    from paper_1009_5169_gb300 import inputs
    U = inputs.links(L, T, 0.3, 21)
    r = inputs.sources(L, T, 1, 22)[0]
    params = cnn.init_params([32, 8, 8, 8, 24], 23)
    params = [(W, np.full(W.shape[2], 0.1)) for W, _ in params]   # biases break oddness of the bare net
    for bf in (False, True):
        m = cnn.precondition(params, U, r, L, T, bf16_acts=bf)
        assert np.array_equal(cnn.precondition(params, U, -r, L, T, bf16_acts=bf), -m)
        assert np.allclose(cnn.precondition(params, U, 4.0 * r, L, T, bf16_acts=bf), 4.0 * m, rtol=0, atol=1e-12)
    # unit mean square per real component: mean |z|^2 over complex entries is 2
    assert abs(np.mean(np.abs(r / cnn.rms_scale(r)) ** 2) - 2.0) < 1e-12
