"""FP64 numpy oracle of the learned preconditioner's network (TEST INFRASTRUCTURE).

Only tests/, __graft_entry__.smoke() and bench.py's baseline legs may use it;
it shares no code with the CUDA kernels.

The network maps a residual on the even sites of the SF fermion lattice to an
approximate correction (a learned stand-in for Dhat^{-1} r inside flexible
GCR; the paper's preconditioners are the single-precision solves of Sec. 3.2,
this learned one is an addition).  Plain definitions:

* a feature map lives on the full fermion lattice x0 = 1..T-1, x1..x3 =
  0..L-1 (lexicographic, x3 fastest), channels last: X[site, c];
* the 3^4-stencil convolution with weights W[k, ci, co] (k runs over the 81
  offsets d in {-1,0,1}^4, d0 slowest) and bias b[co]:
      Y(x)[co] = b[co] + sum_k sum_ci X(x + d_k)[ci] W[k, ci, co],
  with X(x + d) = 0 when x0 + d0 leaves 1..T-1 and spatial offsets periodic;
* the network: h0 = X, h_{l+1} = relu(conv_l(h_l)) for l < 3, out = conv_3(h_3);
* input channels: 24 residual components (spin, colour, re/im) on the even
  sites (zero on odd sites) then 8 link features (Re, Im of tr U_mu(x) / 3 for
  mu = 0..3), the residual divided by its RMS scale s = |r| / sqrt(24 V/2);
  the preconditioner returns r + s (out(r/s) - out(-r/s)) / 2 on the even
  sites (the network learns the correction to the identity; the
  symmetrisation makes M odd and positively homogeneous).

The GPU stores activations and weights in bfloat16 and accumulates in FP32;
``forward(..., bf16=True)`` rounds the same tensors to bfloat16 (round to
nearest even) and computes everything else in FP64.
"""
from __future__ import annotations

import numpy as np

OFFSETS = np.array([(a, b, c, d) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)
                    for d in (-1, 0, 1)], dtype=np.int64)
N_LINK_FEATURES = 8
N_RESIDUAL = 24


def bf16(x: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def shift(X: np.ndarray, L: int, T: int, d) -> np.ndarray:
    """X(x + d) on the fermion lattice: zero across the time boundaries,
    periodic in space.  X: [(T-1) L^3, C]."""
    C = X.shape[-1]
    A = X.reshape(T - 1, L, L, L, C)
    out = np.zeros_like(A)
    d0 = int(d[0])
    B = A
    for ax, dk in ((1, d[1]), (2, d[2]), (3, d[3])):
        if dk:
            B = np.roll(B, -int(dk), axis=ax)
    if d0 == 0:
        out[:] = B
    elif d0 == 1:
        out[:-1] = B[1:]
    else:
        out[1:] = B[:-1]
    return out.reshape(X.shape)


def conv(X, W, b, L, T):
    """Y(x) = b + sum_k X(x + d_k) W[k]."""
    Y = np.zeros((X.shape[0], W.shape[2]))
    for k in range(81):
        Y += shift(X, L, T, OFFSETS[k]) @ W[k]
    return Y + b


def conv_adjoint_input(dY, W, L, T):
    """dX(z) = sum_k dY(z - d_k) W[k]^T, the adjoint of conv in its input."""
    dX = np.zeros((dY.shape[0], W.shape[1]))
    for k in range(81):
        dX += shift(dY @ W[k].T, L, T, -OFFSETS[k])
    return dX


def conv_grad_weight(X, dY, L, T):
    """dW[k] = sum_x X(x + d_k)^T dY(x)."""
    return np.stack([shift(X, L, T, OFFSETS[k]).T @ dY for k in range(81)])


def init_params(widths, seed: int):
    """He-style Gaussian weights (scaled for the 81-point stencil), zero biases."""
    g = np.random.Generator(np.random.Philox(key=np.array([seed, 7], dtype=np.uint64)))
    params = []
    for ci, co in zip(widths[:-1], widths[1:]):
        W = g.standard_normal((81, ci, co)) * np.sqrt(2.0 / (81 * ci))
        params.append((W, np.zeros(co)))
    return params


def forward(params, X, L, T, bf16_acts: bool = False, keep=False):
    """Network output and (optionally) the activations of every layer."""
    hs = [bf16(X) if bf16_acts else X]
    h = hs[0]
    n = len(params)
    for l, (W, b) in enumerate(params):
        Wl = bf16(W) if bf16_acts else W
        z = conv(h, Wl, b, L, T)
        if l < n - 1:
            h = np.maximum(z, 0.0)
            if bf16_acts:
                h = bf16(h)
        else:
            h = z
        hs.append(h)
    return (h, hs) if keep else h


def backward(params, hs, dout, L, T):
    """Gradients (dW, db) per layer and dX for the network, given the
    activations from forward(keep=True) and d loss / d out."""
    grads = [None] * len(params)
    g = dout
    for l in range(len(params) - 1, -1, -1):
        W, b = params[l]
        if l < len(params) - 1:
            g = g * (hs[l + 1] > 0)
        grads[l] = (conv_grad_weight(hs[l], g, L, T), g.sum(axis=0))
        g = conv_adjoint_input(g, W, L, T)
    return grads, g


def features(U, r_even, L, T):
    """Network input for one even-site residual (already normalised):
    [(T-1) L^3, 32] with the residual on even sites and the link features."""
    V = (T - 1) * L ** 3
    x0 = np.arange(1, T)[:, None, None, None]
    x1 = np.arange(L)[None, :, None, None]
    x2 = np.arange(L)[None, None, :, None]
    x3 = np.arange(L)[None, None, None, :]
    par = ((x0 + x1 + x2 + x3) % 2).reshape(-1)
    X = np.zeros((V, N_RESIDUAL + N_LINK_FEATURES))
    r = np.asarray(r_even).reshape(-1, 12)
    X[par == 0, 0:24:2] = r.real
    X[par == 0, 1:24:2] = r.imag
    Uf = np.asarray(U).reshape(T + 1, L ** 3, 4, 3, 3)[1:T].reshape(V, 4, 3, 3)
    tr = np.trace(Uf, axis1=-2, axis2=-1) / 3.0
    X[:, 24:32:2] = tr.real
    X[:, 25:32:2] = tr.imag
    return X


def output_to_even(out, L, T):
    """Even-site complex field [V/2, 4, 3] from the network output [V, 24]."""
    x0 = np.arange(1, T)[:, None, None, None]
    x1 = np.arange(L)[None, :, None, None]
    x2 = np.arange(L)[None, None, :, None]
    x3 = np.arange(L)[None, None, None, :]
    par = ((x0 + x1 + x2 + x3) % 2).reshape(-1)
    o = out[par == 0]
    return (o[:, 0:24:2] + 1j * o[:, 1:24:2]).reshape(-1, 4, 3)


def rms_scale(r_even) -> float:
    """s = |r| / sqrt(number of real components): r / s has unit RMS."""
    r = np.asarray(r_even)
    return float(np.linalg.norm(r) / np.sqrt(2 * r.size))


def precondition(params, U, r_even, L, T, bf16_acts: bool = True):
    """M(r) = r + s (out(r/s) - out(-r/s)) / 2 on the even sites, s the RMS
    scale of r: the network learns the correction to the identity, and the
    symmetrisation makes M odd and positively homogeneous, M(a r) = a M(r)."""
    s = rms_scale(r_even)
    if s == 0:
        return np.zeros_like(r_even)
    op = output_to_even(forward(params, features(U, r_even / s, L, T), L, T, bf16_acts), L, T)
    om = output_to_even(forward(params, features(U, -r_even / s, L, T), L, T, bf16_acts), L, T)
    return r_even + s * 0.5 * (op - om)
