"""FP64 CPU oracle for the SF Wilson fermion MD step (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference legs may import this package.  It wraps ``sf_oracle.c`` (plain C,
FP64, optional OpenMP) through ctypes and shares no code with the CUDA
library.  Each wrapper states the passage of arXiv:1009.5169 it follows; the
readings of the paper the oracle takes are listed in ``sf_oracle.c``.

Array conventions (numpy complex128):
  U      [(T+1) L^3, 4, 3, 3]
  full   [nrhs, (T-1) L^3, 4, 3]
  even   [nrhs, (T-1) L^3 / 2, 4, 3]
  force  [(T+1) L^3, 4, 8]  (float64, components along T^a = lambda^a / 2)

Parity pins: every function here is pinned by a ``-m "not gpu"`` test
(free-field closed form, gamma_5-hermiticity, gauge covariance, theta-twist
equivalence, Schur complement vs. dense LU, BiCGStab vs. dense LU, force and
gauge force vs. central finite differences, plaquette closed forms).
``oracle.hmc`` adds the HMC trajectory around the MD step (momenta, link
exponential, leapfrog), pinned by closed forms, the O(dt^2) energy error and
reversibility.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsf_oracle.so")
_lock = threading.Lock()
_lib = None


def compile_oracle(force: bool = False) -> str:
    """Compile sf_oracle.c into oracle/_build/libsf_oracle.so with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            compile_oracle()
            L = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i, d = ctypes.c_int, ctypes.c_double
            L.sfo_gamma.argtypes = [i, dp]
            L.sfo_hop_full.argtypes = [i, i, d, i, dp, i, dp, dp]
            L.sfo_apply_D.argtypes = [i, i, d, i, d, dp, i, dp, dp]
            L.sfo_apply_dhat.argtypes = [i, i, d, d, dp, i, i, dp, dp]
            L.sfo_bicgstab.argtypes = [i, i, d, d, dp, i, i, dp, dp, d, i, ip, dp]
            L.sfo_force.argtypes = [i, i, d, d, dp, i, dp, dp, dp]
            L.sfo_plaquette_action.argtypes = [i, i, d, dp]
            L.sfo_gauge_force.argtypes = [i, i, d, dp, dp]
            L.sfo_plaquette_action.restype = d
            L.sfo_num_threads.restype = i
            L.sfo_set_num_threads.argtypes = [i]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _block(a, L, T, half):
    a = _c(a)
    V = (T - 1) * L ** 3 // (2 if half else 1)
    if a.ndim == 3:
        a = a[None]
    assert a.shape[1:] == (V, 4, 3), a.shape
    return np.ascontiguousarray(a)


def num_threads() -> int:
    return lib().sfo_num_threads()


def set_num_threads(n: int) -> None:
    lib().sfo_set_num_threads(int(n))


def gamma(mu: int) -> np.ndarray:
    """The oracle's gamma matrix: mu = 0..3 (0 = time) or 4 (gamma_5)."""
    out = np.zeros((4, 4), np.complex128)
    lib().sfo_gamma(mu, _p(out))
    return out


def hop(U, psi, L, T, theta, theta_mode=0):
    """H psi on the full SF fermion lattice (Wilson hopping term, Sec. 3.1).

    theta_mode 0 puts the uniform phase e^{i theta/L} on every forward spatial
    hop; theta_mode 1 puts e^{+-i theta} only on the hops that wrap around."""
    psi = _block(psi, L, T, False)
    out = np.empty_like(psi)
    rc = lib().sfo_hop_full(L, T, theta, theta_mode, _p(_c(U)), psi.shape[0], _p(psi), _p(out))
    assert rc == 0
    return out


def apply_D(U, psi, L, T, theta, kappa, theta_mode=0):
    """D psi, D = 1 - kappa H on the full SF fermion lattice."""
    psi = _block(psi, L, T, False)
    out = np.empty_like(psi)
    rc = lib().sfo_apply_D(L, T, theta, theta_mode, kappa, _p(_c(U)), psi.shape[0], _p(psi), _p(out))
    assert rc == 0
    return out


def apply_dhat(U, x_e, L, T, theta, kappa, dagger=False):
    """Dhat x_e with Dhat = 1 - kappa^2 H_eo H_oe (site even/odd
    preconditioning, Sec. 3.1), or Dhat^dag = gamma_5 Dhat gamma_5."""
    x_e = _block(x_e, L, T, True)
    out = np.empty_like(x_e)
    rc = lib().sfo_apply_dhat(L, T, theta, kappa, _p(_c(U)), int(dagger), x_e.shape[0], _p(x_e), _p(out))
    assert rc == 0
    return out


def bicgstab(U, b_e, L, T, theta, kappa, tol=1e-12, maxiter=10000, dagger=False):
    """Solve Dhat x_i = b_i (or Dhat^dag x_i = b_i) for every right-hand side
    in turn with textbook BiCGStab (Alg. 1; case A of Table 1).

    Returns (x, iters, true_rel_resid)."""
    b_e = _block(b_e, L, T, True)
    n = b_e.shape[0]
    x = np.zeros_like(b_e)
    iters = np.zeros(n, np.int32)
    res = np.zeros(n, np.float64)
    lib().sfo_bicgstab(L, T, theta, kappa, _p(_c(U)), int(dagger), n, _p(b_e), _p(x), tol,
                       int(maxiter), iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(res))
    return x, iters, res


def force(U, X_e, Y_e, L, T, theta, kappa):
    """MD force F_mu(n) = sum_i f[x_i, y_i] of Eq. (3) (the force steps of Alg. 2),
    the gradient of S = sum_i |Dhat^-1 phi_i|^2 with respect to
    U_mu(x) -> exp(i omega^a T^a) U_mu(x).  Shape [(T+1)L^3, 4, 8]."""
    X_e = _block(X_e, L, T, True)
    Y_e = _block(Y_e, L, T, True)
    F = np.zeros(((T + 1) * L ** 3, 4, 8), np.float64)
    rc = lib().sfo_force(L, T, theta, kappa, _p(_c(U)), X_e.shape[0], _p(X_e), _p(Y_e), _p(F))
    assert rc == 0
    return F


def plaquette_action(U, L, T, beta):
    """SF Wilson plaquette action S_g = beta sum_p w(p) (1 - Re tr U_p / 3)."""
    return float(lib().sfo_plaquette_action(L, T, beta, _p(_c(U))))


def gauge_force(U, L, T, beta):
    """Force of the SF plaquette action, F^a_mu(x) = dS_g/d omega^a for
    U_mu(x) -> exp(i omega^a T^a) U_mu(x); zero on the fixed boundary links.
    Shape [(T+1)L^3, 4, 8]."""
    F = np.zeros(((T + 1) * L ** 3, 4, 8), np.float64)
    rc = lib().sfo_gauge_force(L, T, beta, _p(_c(U)), _p(F))
    assert rc == 0
    return F


# ---------------------------------------------------------------- helpers

def parity_of_full_sites(L, T):
    """Parity (x0+x1+x2+x3) mod 2 of every full fermion site, lexicographic."""
    x0 = np.arange(1, T)[:, None, None, None]
    x1 = np.arange(L)[None, :, None, None]
    x2 = np.arange(L)[None, None, :, None]
    x3 = np.arange(L)[None, None, None, :]
    return ((x0 + x1 + x2 + x3) % 2).reshape(-1)


def split_eo(full, L, T):
    """Full fermion block -> (even block, odd block) in the library's order."""
    full = _block(full, L, T, False)
    par = parity_of_full_sites(L, T)
    return full[:, par == 0], full[:, par == 1]


def join_eo(even, odd, L, T):
    even = _block(even, L, T, True)
    odd = _block(odd, L, T, True)
    par = parity_of_full_sites(L, T)
    out = np.zeros((even.shape[0], par.size, 4, 3), np.complex128)
    out[:, par == 0] = even
    out[:, par == 1] = odd
    return out


def gamma5(psi):
    g5 = np.array([1, 1, -1, -1], np.float64)
    return psi * g5[:, None]


def solve_pair(U, phi_e, L, T, theta, kappa, tol=1e-12, maxiter=10000):
    """The two solves of Alg. 2 by the sequential solver: X = Dhat^-1 Phi,
    Y = Dhat^-dag X.  Returns (X, Y, info dict)."""
    X, itx, rx = bicgstab(U, phi_e, L, T, theta, kappa, tol, maxiter, dagger=False)
    Y, ity, ry = bicgstab(U, X, L, T, theta, kappa, tol, maxiter, dagger=True)
    return X, Y, dict(iters_x=itx, iters_y=ity, resid_x=rx, resid_y=ry)


def true_residual(U, b_e, x_e, L, T, theta, kappa, dagger=False):
    """Per-RHS |b - Dhat x| / |b| (or with Dhat^dag), computed by the oracle."""
    Ax = apply_dhat(U, x_e, L, T, theta, kappa, dagger)
    b_e = _block(b_e, L, T, True)
    num = np.linalg.norm((b_e - Ax).reshape(b_e.shape[0], -1), axis=1)
    den = np.linalg.norm(b_e.reshape(b_e.shape[0], -1), axis=1)
    return num / np.where(den == 0, 1, den)
