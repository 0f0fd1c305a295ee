"""Seeded synthetic inputs for the Schroedinger-functional Wilson workloads.

This module is the only code shared by the CUDA path's tests/benchmarks and the
FP64 oracle: it draws gauge links and pseudo-fermion sources and holds none of
the method's arithmetic (no hopping term, no solver, no force).

Layouts (the library's canonical host layout, see include/sf_lattice.h):

* gauge links: complex128 array ``[(T+1)*L^3, 4, 3, 3]``.  The site index is
  lexicographic over ``x0 = 0..T`` and ``x1, x2, x3 = 0..L-1`` with x3 fastest;
  direction 0 is time.  ``U[x, mu, a, b]`` is the colour matrix element (row a,
  column b) of ``U_mu(x)``.  The time link at ``x0 = T`` does not exist on the
  SF lattice and is set to the identity; the spatial links on the boundary
  slices ``x0 = 0`` and ``x0 = T`` are the SF boundary fields, taken as the
  identity (zero background field, C = C' = 0).
* even-site fermion block: complex128 ``[nrhs, V/2, 4, 3]`` (spin, colour).  The
  fermion lives on ``x0 = 1..T-1``; V = L^3 (T-1).  Sites of one parity
  ``(x0+x1+x2+x3) mod 2`` are numbered in lexicographic order of the fermion
  lattice (x0 slowest, x3 fastest), which for even L is ``lex_index // 2``.

Synthetic ensembles follow the workloads the paper measures (Sec. 4: SF, SU(3)
plaquette action, Wilson quarks, 5 pseudo-fermion fields) with links
``U = exp(i eps H)``, H a Gaussian traceless Hermitian 3x3 matrix with
``A_ab ~ N(0,1) + i N(0,1)``, ``H = (A + A^dag)/2 - tr/3``.
Random numbers come from numpy's counter-based Philox generator keyed by
``(seed, field)``.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np

SEED_BASE = 0x5F1009

# field ids under one seed
FIELD_LINKS = 0
FIELD_SOURCES = 1
FIELD_GAUGE_TRANSFORM = 2
FIELD_AUX = 3


def rng(seed: int, field_id: int) -> np.random.Generator:
    """Counter-based Philox generator keyed by (seed, field id)."""
    key = np.array([seed & 0xFFFFFFFFFFFFFFFF, field_id & 0xFFFFFFFFFFFFFFFF],
                   dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


def gauge_sites(L: int, T: int) -> int:
    return (T + 1) * L ** 3


def fermion_volume(L: int, T: int) -> int:
    return (T - 1) * L ** 3


def half_volume(L: int, T: int) -> int:
    V = fermion_volume(L, T)
    if L % 2 != 0:
        raise ValueError("spatial extent L must be even")
    return V // 2


def _expi_chunk(H: np.ndarray, eps: float) -> np.ndarray:
    w, V = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    return (V * ph[..., None, :]) @ np.swapaxes(V.conj(), -1, -2)


def _expi_hermitian(H: np.ndarray, eps: float, device=None) -> np.ndarray:
    """exp(i eps H) for a batch of Hermitian matrices via eigendecomposition.
    (``device`` is accepted for API compatibility and ignored.)"""
    return _expi_chunk(H, eps)


def gaussian_traceless_hermitian(g: np.random.Generator, shape) -> np.ndarray:
    A = g.standard_normal(tuple(shape) + (3, 3)) + 1j * g.standard_normal(tuple(shape) + (3, 3))
    H = 0.5 * (A + np.swapaxes(A.conj(), -1, -2))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    H = H - tr[..., None, None] * np.eye(3)
    return H


def links(L: int, T: int, eps: float, seed: int, field_id: int = FIELD_LINKS, device=None) -> np.ndarray:
    """SF gauge field U = exp(i eps H), shape [(T+1) L^3, 4, 3, 3] complex128."""
    if L % 2 or L < 2 or T < 2:
        raise ValueError("need even L >= 2 and T >= 2")
    g = rng(seed, field_id)
    n = gauge_sites(L, T)
    H = gaussian_traceless_hermitian(g, (n, 4))
    U = _expi_hermitian(H, eps, device)
    U = U.reshape(T + 1, L ** 3, 4, 3, 3)
    eye = np.eye(3, dtype=np.complex128)
    U[0, :, 1:] = eye          # boundary spatial links at x0 = 0
    U[T, :, 1:] = eye          # boundary spatial links at x0 = T
    U[T, :, 0] = eye           # no time link leaves x0 = T
    return np.ascontiguousarray(U.reshape(n, 4, 3, 3))


def random_su3(n: int, seed: int, field_id: int = FIELD_GAUGE_TRANSFORM,
               eps: float = 2.0) -> np.ndarray:
    """n random SU(3) matrices exp(i eps H) (for gauge transformations)."""
    g = rng(seed, field_id)
    H = gaussian_traceless_hermitian(g, (n,))
    return _expi_hermitian(H, eps)


def sources(L: int, T: int, nrhs: int, seed: int, field_id: int = FIELD_SOURCES) -> np.ndarray:
    """Even-site Gaussian pseudo-fermion block, [nrhs, V/2, 4, 3] complex128.

    Each real and imaginary part is N(0, 1/2)."""
    g = rng(seed, field_id)
    Vh = half_volume(L, T)
    s = np.sqrt(0.5)
    re = g.standard_normal((nrhs, Vh, 4, 3)) * s
    im = g.standard_normal((nrhs, Vh, 4, 3)) * s
    return re + 1j * im


def full_sources(L: int, T: int, nrhs: int, seed: int, field_id: int = FIELD_AUX) -> np.ndarray:
    """Full fermion-lattice Gaussian block, [nrhs, V, 4, 3] complex128."""
    g = rng(seed, field_id)
    V = fermion_volume(L, T)
    s = np.sqrt(0.5)
    return (g.standard_normal((nrhs, V, 4, 3)) + 1j * g.standard_normal((nrhs, V, 4, 3))) * s


def su3_directions(shape, seed: int, field_id: int = FIELD_AUX) -> np.ndarray:
    """Random real su(3) component vectors c^a, shape ``shape + (8,)``."""
    return rng(seed, field_id).standard_normal(tuple(shape) + (8,))


def cnn_widths(hidden: int):
    """Channel widths of the learned preconditioner's four layers."""
    return [32, hidden, hidden, hidden, 24]


def cnn_init_params(hidden: int, seed: int, last_scale: float = 0.05) -> np.ndarray:
    """Seeded initial parameters (flat FP32: per layer W[81][ci][co], then the
    bias), Gaussian with variance 2 / (81 ci), zero biases; the last layer is
    scaled by ``last_scale`` so the preconditioner starts close to the identity."""
    g = rng(seed, 7)
    w = cnn_widths(hidden)
    parts = []
    for l, (ci, co) in enumerate(zip(w[:-1], w[1:])):
        sc = np.sqrt(2.0 / (81 * ci)) * (last_scale if l == len(w) - 2 else 1.0)
        parts.append((g.standard_normal((81, ci, co)) * sc).reshape(-1))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def cnn_unflatten(params: np.ndarray, hidden: int):
    """[(W [81, ci, co], b [co]), ...] views of a flat parameter array."""
    w = cnn_widths(hidden)
    out, off = [], 0
    for ci, co in zip(w[:-1], w[1:]):
        n = 81 * ci * co
        out.append((np.asarray(params[off:off + n], dtype=np.float64).reshape(81, ci, co),
                    np.asarray(params[off + n:off + n + co], dtype=np.float64)))
        off += n + co
    return out


# --------------------------------------------------------------------------
# Workloads: synthetic stand-ins for the paper's 16^4 SF N_f=10 ensemble.
# --------------------------------------------------------------------------
@dataclass
class Lattice:
    L: int
    T: int
    eps: float
    kappa: float
    seed: int
    theta: float = 0.5
    beta: float = 4.52

    @property
    def V(self) -> int:
        return fermion_volume(self.L, self.T)

    @property
    def Vh(self) -> int:
        return half_volume(self.L, self.T)

    def make_links(self) -> np.ndarray:
        return links(self.L, self.T, self.eps, self.seed)

    def make_sources(self, nrhs: int) -> np.ndarray:
        return sources(self.L, self.T, nrhs, self.seed)


@dataclass
class Workload:
    name: str
    lattices: List[Lattice]
    nrhs: int
    tol: float
    note: str = ""


def workload(name: str) -> Workload:
    """The five synthetic workloads (sizes, kappa, eps) the build measures."""
    if name == "sf8_plain_1rhs":
        return Workload(name, [Lattice(8, 8, 0.3, 0.125, SEED_BASE + 0)], 1, 1e-12,
                        "8^3x8 SF, FP64, 1 RHS, solve to 1e-12 then force")
    if name == "sf12_nf10":
        return Workload(name, [Lattice(12, 12, 0.25, 0.13, SEED_BASE + 1)], 5, 1e-10,
                        "12^4 SF, 5 pseudo-fermions (N_f=10), FP32 inner / FP64 outer, 1e-10")
    if name == "sf16_mixed":
        return Workload(name, [Lattice(16, 16, 0.2, 0.134, SEED_BASE + 2)], 5, 1e-10,
                        "16^4 SF, kappa=0.134, FP16/FP32 inner under FP64 defect correction")
    if name == "batched_uneven":
        lats = []
        epss = (0.15, 0.25, 0.35)
        k = 0
        for L in (8, 12, 16):
            for j in range(8):
                lats.append(Lattice(L, L, epss[k % 3], 0.13, SEED_BASE + 3 + 1000 * (k + 1)))
                k += 1
        return Workload(name, lats, 5, 1e-10,
                        "24 SF fields (8 each of 8^4, 12^4, 16^4), eps cycling 0.15/0.25/0.35")
    if name == "sf24_cnn":
        return Workload(name, [Lattice(24, 24, 0.2, 0.134, SEED_BASE + 4)], 5, 1e-10,
                        "24^4 SF, kappa=0.134, learned preconditioner in FGCR")
    raise KeyError(name)


WORKLOADS = ("sf8_plain_1rhs", "sf12_nf10", "sf16_mixed", "batched_uneven", "sf24_cnn")
