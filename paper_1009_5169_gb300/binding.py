"""ctypes binding of include/sf_lattice.h (argument marshalling only).

Every step of the path runs in the CUDA library ``_build/libsfgb300.so``;
this module only converts arguments.  There is no fallback: if the library
is missing the calls raise.  Arrays may be numpy arrays (host) or torch
tensors (host or CUDA), complex128 in the canonical layouts of the header:

  links  [(T+1) L^3, 4, 3, 3]      even/odd  [nrhs, V/2, 4, 3]
  full   [2, nrhs, V/2, 4, 3]      force     [(T+1) L^3, 4, 8] float64
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsfgb300.so")
MAX_RHS = 16

SF_OK, SF_EINVAL, SF_ENOMEM, SF_ECUDA, SF_ENOCONV, SF_ETIMEOUT, SF_ENOTSU3 = range(7)
STATUS = {0: "SF_OK", 1: "SF_EINVAL", 2: "SF_ENOMEM", 3: "SF_ECUDA", 4: "SF_ENOCONV", 5: "SF_ETIMEOUT",
          6: "SF_ENOTSU3"}
OPS = {"dhat": 0, "dhat_dag": 1, "dhatdag_dhat": 2, "d_full": 3, "hop_eo": 4, "hop_oe": 5}
PRECS = {"fp64": 0, "fp32": 1, "fp16": 2}
ALGOS = {"bicgstab": 0, "mixed_dc": 1, "mixed_dc_half": 2, "fgcr_cnn": 3, "fgcr": 4, "cg_normal": 5,
         "gl_bicgstab": 6, "bl_bicgstab": 7, "fgcr_cnn_mixed": 8, "fgcr_mixed": 9}


class SFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class SolveInfo(ctypes.Structure):
    _fields_ = [
        ("iters_outer", ctypes.c_int), ("iters_inner", ctypes.c_int),
        ("iters_outer_y", ctypes.c_int), ("iters_inner_y", ctypes.c_int),
        ("iters_inner_rhs", ctypes.c_int * MAX_RHS),
        ("true_resid", ctypes.c_double * MAX_RHS),
        ("true_resid_y", ctypes.c_double * MAX_RHS),
        ("seconds", ctypes.c_double),
        ("kernel_launches", ctypes.c_longlong),
    ]

    def as_dict(self, nrhs: int) -> dict:
        return dict(iters_outer=self.iters_outer, iters_inner=self.iters_inner,
                    iters_outer_y=self.iters_outer_y, iters_inner_y=self.iters_inner_y,
                    iters_inner_rhs=list(self.iters_inner_rhs[:nrhs]),
                    true_resid=list(self.true_resid[:nrhs]), true_resid_y=list(self.true_resid_y[:nrhs]),
                    seconds=self.seconds, kernel_launches=self.kernel_launches)


class MdInfo(ctypes.Structure):
    _fields_ = [
        ("kinetic", ctypes.c_double * 2), ("s_gauge", ctypes.c_double * 2),
        ("s_fermion", ctypes.c_double * 2), ("dH", ctypes.c_double),
        ("force_evals", ctypes.c_int), ("inner_iters", ctypes.c_int),
        ("seconds", ctypes.c_double), ("kernel_launches", ctypes.c_longlong),
    ]

    def as_dict(self) -> dict:
        return dict(kinetic=list(self.kinetic), s_gauge=list(self.s_gauge), s_fermion=list(self.s_fermion),
                    dH=self.dH, force_evals=self.force_evals, inner_iters=self.inner_iters,
                    seconds=self.seconds, kernel_launches=self.kernel_launches)


_lib = None


def lib() -> ctypes.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library missing: {LIB_PATH} (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.sf_lattice_create.argtypes = [ctypes.POINTER(vp), i, i, d, d, d, vp, i, vp]
        L.sf_lattice_set_links.argtypes = [vp, vp]
        L.sf_lattice_set_tuning.argtypes = [vp, i, i, i, i]
        L.sf_lattice_get_tuning.argtypes = [vp, i, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
        L.sf_lattice_destroy.argtypes = [vp]
        L.sf_lattice_destroy.restype = None
        L.wilson_apply_block.argtypes = [vp, i, i, i, vp, vp]
        L.wilson_hop_resident.argtypes = [vp, i, i, i]
        L.solve_block.argtypes = [vp, i, i, vp, vp, vp, d, i, ctypes.POINTER(SolveInfo)]
        L.fermion_force.argtypes = [vp, i, vp, vp, vp, vp, d]
        L.fermion_force_resident.argtypes = [vp, i, vp]
        L.md_force_step.argtypes = [vp, i, i, vp, vp, vp, vp, vp, d, d, i, ctypes.POINTER(SolveInfo)]
        L.plaquette_action.argtypes = [vp, ctypes.POINTER(d)]
        L.gauge_force.argtypes = [vp, vp, vp, d]
        L.sf_lattice_update_links.argtypes = [vp, vp, d]
        L.sf_lattice_get_links.argtypes = [vp, vp]
        L.sf_md_trajectory.argtypes = [vp, i, i, vp, vp, i, d, d, i, ctypes.POINTER(MdInfo)]
        L.sf_md_trajectory_omelyan.argtypes = [vp, i, i, vp, vp, i, d, d, d, i, ctypes.POINTER(MdInfo)]
        L.sf_md_trajectory_two_scales.argtypes = [vp, i, i, vp, vp, i, d, i, d, i, ctypes.POINTER(MdInfo)]
        L.sf_hmc_trajectory.argtypes = [vp, i, i, vp, vp, d, i, i, d, i, d, d, i, ctypes.POINTER(MdInfo),
                                        ctypes.POINTER(ctypes.c_int)]
        L.plaquette_action_noalloc.argtypes = [i, i, d, vp, vp, i, vp]
        L.plaquette_action_noalloc.restype = ctypes.c_int
        L.sf_cnn_num_params.argtypes = [i]
        L.sf_cnn_num_params.restype = ctypes.c_longlong
        L.sf_cnn_create.argtypes = [ctypes.POINTER(vp), i, vp, i, vp]
        L.sf_cnn_get_params.argtypes = [vp, vp]
        L.sf_cnn_destroy.argtypes = [vp]
        L.sf_cnn_destroy.restype = None
        L.sf_cnn_forward.argtypes = [vp, vp, i, vp, vp]
        L.sf_cnn_train_step.argtypes = [vp, vp, i, vp, vp, ctypes.c_float, ctypes.POINTER(d)]
        L.sf_cnn_gradients.argtypes = [vp, vp, i, vp, vp, vp, ctypes.POINTER(d)]
        L.sf_lattice_set_preconditioner.argtypes = [vp, vp]
        L.sf_cnn_set_conv_impl.argtypes = [vp, i]
        for fn in ("sf_cnn_create", "sf_cnn_get_params", "sf_cnn_forward", "sf_cnn_train_step", "sf_cnn_gradients",
                   "sf_lattice_set_preconditioner", "sf_cnn_set_conv_impl"):
            getattr(L, fn).restype = ctypes.c_int
        L.sf_last_error.restype = ctypes.c_char_p
        L.sf_batch_create.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp), i]
        L.sf_batch_solve.argtypes = [vp, i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), d, i,
                                     ctypes.POINTER(SolveInfo)]
        L.sf_batch_destroy.argtypes = [vp]
        L.sf_batch_destroy.restype = None
        L.sf_batch_num_groups.argtypes = [vp]
        L.sf_batch_num_groups.restype = i
        for fn in ("sf_lattice_create", "sf_lattice_set_links", "sf_lattice_set_tuning", "sf_lattice_get_tuning",
                   "wilson_apply_block", "wilson_hop_resident", "solve_block", "fermion_force", "fermion_force_resident",
                   "md_force_step",
                   "plaquette_action", "sf_batch_create",
                   "sf_batch_solve"):
            getattr(L, fn).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int, allow_noconv: bool = False) -> int:
    if rc == SF_OK or (allow_noconv and rc == SF_ENOCONV):
        return rc
    raise SFError(rc, lib().sf_last_error().decode())


def _ptr(a) -> int:
    """Address of a contiguous numpy array or torch tensor."""
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _nbytes(a) -> int:
    if isinstance(a, np.ndarray):
        return a.nbytes
    return a.numel() * a.element_size()


def _current_stream(device: int) -> int:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream(device).cuda_stream
    except Exception:
        pass
    return 0


class Lattice:
    """Owner of one ``sf_lattice`` (device copies of the links, workspaces)."""

    def __init__(self, L: int, T: int, theta: float, kappa: float, beta: float, links, device: int = 0,
                 stream: Optional[int] = None):
        self.L, self.T, self.theta, self.kappa, self.beta = L, T, theta, kappa, beta
        self.V = (T - 1) * L ** 3
        self.Vh = self.V // 2
        self.device = device
        self._h = ctypes.c_void_p()
        self._links_keep = links
        _check_size(links, (T + 1) * L ** 3 * 4 * 18 * 8, "links")
        s = _current_stream(device) if stream is None else stream
        _check(lib().sf_lattice_create(ctypes.byref(self._h), L, T, theta, kappa, beta, _ptr(links), device, s))

    @property
    def handle(self):
        return self._h

    def set_links(self, links) -> None:
        _check_size(links, (self.T + 1) * self.L ** 3 * 4 * 18 * 8, "links")
        _check(lib().sf_lattice_set_links(self._h, _ptr(links)))

    def set_tuning(self, prec: str, TS: int, NR: int, pipe: int = 0) -> None:
        """Fix (TS sites per tile, NR rhs per thread, pipelined hop 0/1); TS = 0 autotunes."""
        _check(lib().sf_lattice_set_tuning(self._h, PRECS[prec], TS, NR, pipe))

    def get_tuning(self, prec: str, nrhs: int):
        """(TS, NR, pipe) in use for nrhs right-hand sides (autotunes on first use)."""
        ts, nr, pp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().sf_lattice_get_tuning(self._h, PRECS[prec], nrhs, ctypes.byref(ts), ctypes.byref(nr),
                                           ctypes.byref(pp)))
        return ts.value, nr.value, pp.value

    def close(self) -> None:
        if self._h:
            lib().sf_lattice_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _check_size(a, nbytes: int, name: str) -> None:
    if _nbytes(a) != nbytes:
        raise ValueError(f"{name}: expected {nbytes} bytes, got {_nbytes(a)}")


def _nrhs_of(a, per_rhs_bytes: int) -> int:
    n = _nbytes(a)
    if n % per_rhs_bytes:
        raise ValueError("array size is not a whole number of fields")
    return n // per_rhs_bytes


def wilson_apply_block(lat: Lattice, op: str, prec: str, inp, out) -> None:
    """out = op(inp) (see sf_op); in/out complex128, FP64 values."""
    half = lat.Vh * 24 * 8
    per = 2 * half if op == "d_full" else half
    nrhs = _nrhs_of(inp, per)
    _check_size(out, nrhs * per, "out")
    _check(lib().wilson_apply_block(lat.handle, OPS[op], PRECS[prec], nrhs, _ptr(inp), _ptr(out)))


def wilson_hop_resident(lat: Lattice, prec: str, nrhs: int, out_parity: int = 1) -> None:
    """One hopping-term kernel launch on the lattice's resident buffers."""
    _check(lib().wilson_hop_resident(lat.handle, PRECS[prec], nrhs, out_parity))


def solve_block(lat: Lattice, algo: str, phi, X, Y=None, tol: float = 1e-10, maxiter: int = 10000,
                allow_noconv: bool = False) -> dict:
    """The two solves of Alg. 2: X = Dhat^-1 phi, Y = Dhat^-dag X.  Returns the info dict."""
    nrhs = _nrhs_of(phi, lat.Vh * 24 * 8)
    _check_size(X, nrhs * lat.Vh * 24 * 8, "X")
    if Y is not None:
        _check_size(Y, nrhs * lat.Vh * 24 * 8, "Y")
    info = SolveInfo()
    rc = lib().solve_block(lat.handle, ALGOS[algo], nrhs, _ptr(phi), _ptr(X), _ptr(Y), tol, maxiter,
                           ctypes.byref(info))
    _check(rc, allow_noconv)
    d = info.as_dict(nrhs)
    d["status"] = STATUS[rc]
    return d


def fermion_force(lat: Lattice, X, Y, F=None, mom=None, eps: float = 0.0) -> None:
    """Eq. (3): F = sum_i f[x_i, y_i]; optionally mom -= eps F."""
    nrhs = _nrhs_of(X, lat.Vh * 24 * 8)
    _check_size(Y, nrhs * lat.Vh * 24 * 8, "Y")
    fb = (lat.T + 1) * lat.L ** 3 * 4 * 8 * 8
    if F is not None:
        _check_size(F, fb, "F")
    if mom is not None:
        _check_size(mom, fb, "mom")
    _check(lib().fermion_force(lat.handle, nrhs, _ptr(X), _ptr(Y), _ptr(F), _ptr(mom), eps))


def fermion_force_resident(lat: Lattice, nrhs: int, F) -> None:
    """One force-kernel launch on the resident X, Y of the last force call
    (profiling aid); F a device tensor of the force layout, not cleared."""
    _check_size(F, (lat.T + 1) * lat.L ** 3 * 4 * 8 * 8, "F")
    _check(lib().fermion_force_resident(lat.handle, nrhs, _ptr(F)))


def md_force_step(lat: Lattice, algo: str, phi, X, Y, F=None, mom=None, eps: float = 0.0, tol: float = 1e-10,
                  maxiter: int = 10000, allow_noconv: bool = False) -> dict:
    """Alg. 2 in one call: X = Dhat^-1 phi, Y = Dhat^-dag X and the force of Eq. (3)
    (F and / or mom -= eps F), reusing the odd-site hops of the final residuals."""
    nrhs = _nrhs_of(phi, lat.Vh * 24 * 8)
    _check_size(X, nrhs * lat.Vh * 24 * 8, "X")
    _check_size(Y, nrhs * lat.Vh * 24 * 8, "Y")
    fb = (lat.T + 1) * lat.L ** 3 * 4 * 8 * 8
    if F is not None:
        _check_size(F, fb, "F")
    if mom is not None:
        _check_size(mom, fb, "mom")
    info = SolveInfo()
    rc = lib().md_force_step(lat.handle, ALGOS[algo], nrhs, _ptr(phi), _ptr(X), _ptr(Y), _ptr(F), _ptr(mom), eps,
                             tol, maxiter, ctypes.byref(info))
    _check(rc, allow_noconv)
    d = info.as_dict(nrhs)
    d["status"] = STATUS[rc]
    return d


def plaquette_action(lat: Lattice) -> float:
    S = ctypes.c_double()
    _check(lib().plaquette_action(lat.handle, ctypes.byref(S)))
    return S.value


# ---------------------------------------------------------------- HMC trajectory

def _mom_bytes(lat: Lattice) -> int:
    return (lat.T + 1) * lat.L ** 3 * 4 * 8 * 8


def gauge_force(lat: Lattice, F=None, mom=None, eps: float = 0.0) -> None:
    """Force of the plaquette action (F and / or mom -= eps F), zero on the
    fixed boundary links."""
    if F is not None:
        _check_size(F, _mom_bytes(lat), "F")
    if mom is not None:
        _check_size(mom, _mom_bytes(lat), "mom")
    _check(lib().gauge_force(lat.handle, _ptr(F), _ptr(mom), eps))


def update_links(lat: Lattice, mom, dt: float) -> None:
    """U <- exp(i dt P) U on the dynamic links (P = P^a T^a from mom)."""
    _check_size(mom, _mom_bytes(lat), "mom")
    _check(lib().sf_lattice_update_links(lat.handle, _ptr(mom), dt))


def get_links(lat: Lattice, out) -> None:
    """Copy the lattice's current FP64 links into out (canonical layout)."""
    _check_size(out, (lat.T + 1) * lat.L ** 3 * 4 * 18 * 8, "links")
    _check(lib().sf_lattice_get_links(lat.handle, _ptr(out)))


OMELYAN_LAMBDA = 0.1931833275037836


def md_trajectory(lat: Lattice, algo: str, phi, mom, nsteps: int, dt: float, tol: float = 1e-10,
                  maxiter: int = 10000, allow_noconv: bool = False, integrator: str = "leapfrog",
                  lam: float = OMELYAN_LAMBDA, gauge_substeps: int = 1) -> dict:
    """One MD trajectory (gauge + fermion force for the pseudo-fermions phi)
    by the leapfrog (with the gauge force on gauge_substeps substeps of each
    step: two time scales) or the Omelyan integrator (parameter lam); moves
    the lattice's links and mom in place; returns the Hamiltonian parts at
    both ends and dH."""
    nrhs = _nrhs_of(phi, lat.Vh * 24 * 8)
    _check_size(mom, _mom_bytes(lat), "mom")
    info = MdInfo()
    if integrator == "leapfrog" and gauge_substeps == 1:
        rc = lib().sf_md_trajectory(lat.handle, ALGOS[algo], nrhs, _ptr(phi), _ptr(mom), nsteps, dt, tol, maxiter,
                                    ctypes.byref(info))
    elif integrator == "leapfrog":
        rc = lib().sf_md_trajectory_two_scales(lat.handle, ALGOS[algo], nrhs, _ptr(phi), _ptr(mom), nsteps, dt,
                                               gauge_substeps, tol, maxiter, ctypes.byref(info))
    elif integrator == "omelyan":
        rc = lib().sf_md_trajectory_omelyan(lat.handle, ALGOS[algo], nrhs, _ptr(phi), _ptr(mom), nsteps, dt, lam,
                                            tol, maxiter, ctypes.byref(info))
    else:
        raise ValueError(f"integrator must be leapfrog or omelyan, got {integrator!r}")
    _check(rc, allow_noconv)
    d = info.as_dict()
    d["status"] = STATUS[rc]
    return d


INTEGRATORS = {"leapfrog": 0, "omelyan": 1}


def hmc_trajectory(lat: Lattice, algo: str, eta, mom, uniform: float, nsteps: int, dt: float,
                   tol: float = 1e-10, maxiter: int = 10000, integrator: str = "leapfrog",
                   gauge_substeps: int = 1, lam: float = OMELYAN_LAMBDA, allow_noconv: bool = False) -> dict:
    """One HMC trajectory with the caller's random numbers (sf_hmc_trajectory):
    pseudo-fermions phi = Dhat eta, an MD trajectory from the momenta mom and
    the Metropolis test with the uniform number.  Returns the md_trajectory
    dict with "accepted"."""
    nrhs = _nrhs_of(eta, lat.Vh * 24 * 8)
    _check_size(mom, _mom_bytes(lat), "mom")
    if integrator not in INTEGRATORS:
        raise ValueError(f"integrator must be leapfrog or omelyan, got {integrator!r}")
    info = MdInfo()
    acc = ctypes.c_int()
    rc = lib().sf_hmc_trajectory(lat.handle, ALGOS[algo], nrhs, _ptr(eta), _ptr(mom), uniform,
                                 INTEGRATORS[integrator], nsteps, dt, gauge_substeps, lam, tol, maxiter,
                                 ctypes.byref(info), ctypes.byref(acc))
    _check(rc, allow_noconv)
    d = info.as_dict()
    d["status"] = STATUS[rc]
    d["accepted"] = bool(acc.value)
    return d


class Batch:
    """Several lattices (any sizes) solved with one launch per kernel and
    group of lattices whose working set fits in L2 (see sf_batch_create)."""

    def __init__(self, lattices: Sequence[Lattice], nrhs: int):
        self.lattices = list(lattices)
        self.nrhs = nrhs
        self._h = ctypes.c_void_p()
        arr = (ctypes.c_void_p * len(self.lattices))(*[l.handle.value for l in self.lattices])
        _check(lib().sf_batch_create(ctypes.byref(self._h), len(self.lattices), arr, nrhs))

    def solve(self, algo: str, phis, Xs, Ys=None, tol: float = 1e-10, maxiter: int = 10000,
              allow_noconv: bool = False) -> List[dict]:
        n = len(self.lattices)
        for l, lat in enumerate(self.lattices):
            _check_size(phis[l], self.nrhs * lat.Vh * 24 * 8, "phi")
            _check_size(Xs[l], self.nrhs * lat.Vh * 24 * 8, "X")
        P = (ctypes.c_void_p * n)(*[_ptr(a) for a in phis])
        Xp = (ctypes.c_void_p * n)(*[_ptr(a) for a in Xs])
        Yp = (ctypes.c_void_p * n)(*[_ptr(a) for a in Ys]) if Ys is not None else None
        infos = (SolveInfo * n)()
        rc = lib().sf_batch_solve(self._h, ALGOS[algo], P, Xp, Yp, tol, maxiter, infos)
        _check(rc, allow_noconv)
        out = [infos[l].as_dict(self.nrhs) for l in range(n)]
        for d in out:
            d["status"] = STATUS[rc]
        return out

    @property
    def num_groups(self) -> int:
        return int(lib().sf_batch_num_groups(self._h))

    def close(self) -> None:
        if self._h:
            lib().sf_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Cnn:
    """The learned preconditioner's network (see sf_cnn_* in the header)."""

    def __init__(self, hidden: int, params: np.ndarray, device: int = 0, stream: Optional[int] = None):
        self.hidden = hidden
        self.nparams = int(lib().sf_cnn_num_params(hidden))
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.nparams:
            raise ValueError(f"expected {self.nparams} parameters, got {p.size}")
        self._h = ctypes.c_void_p()
        s = _current_stream(device) if stream is None else stream
        _check(lib().sf_cnn_create(ctypes.byref(self._h), hidden, _ptr(p), device, s))

    @property
    def handle(self):
        return self._h

    def params(self) -> np.ndarray:
        out = np.empty(self.nparams, np.float32)
        _check(lib().sf_cnn_get_params(self._h, _ptr(out)))
        return out

    def forward(self, lat: Lattice, r, out) -> None:
        nrhs = _nrhs_of(r, lat.Vh * 24 * 8)
        _check_size(out, nrhs * lat.Vh * 24 * 8, "out")
        _check(lib().sf_cnn_forward(self._h, lat.handle, nrhs, _ptr(r), _ptr(out)))

    def train_step(self, lat: Lattice, r, e, lr: float) -> float:
        """e = None trains on the residual norm |r - Dhat M(r)|^2 / |r|^2."""
        nrhs = _nrhs_of(r, lat.Vh * 24 * 8)
        if e is not None:
            _check_size(e, nrhs * lat.Vh * 24 * 8, "e")
        loss = ctypes.c_double()
        _check(lib().sf_cnn_train_step(self._h, lat.handle, nrhs, _ptr(r), _ptr(e), lr, ctypes.byref(loss)))
        return loss.value

    def gradients(self, lat: Lattice, r, e):
        nrhs = _nrhs_of(r, lat.Vh * 24 * 8)
        g = np.empty(self.nparams, np.float32)
        loss = ctypes.c_double()
        _check(lib().sf_cnn_gradients(self._h, lat.handle, nrhs, _ptr(r), _ptr(e), _ptr(g), ctypes.byref(loss)))
        return g, loss.value

    def set_conv_impl(self, impl: str) -> None:
        """"tcgen05" (the default: the tensor-core convolution where the layer
        shape fits) or "mma_sync" (the mma.sync kernel everywhere)."""
        _check(lib().sf_cnn_set_conv_impl(self._h, {"tcgen05": 0, "mma_sync": 1}[impl]))

    def close(self) -> None:
        if self._h:
            lib().sf_cnn_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_preconditioner(lat: Lattice, cnn: Optional[Cnn]) -> None:
    _check(lib().sf_lattice_set_preconditioner(lat.handle, cnn.handle if cnn is not None else None))
