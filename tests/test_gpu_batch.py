"""Batched solves of several SF lattices of uneven sizes in one launch per
kernel (the batched workload: 8 each of 8^4, 12^4 and 16^4, 5 RHS), judged
by the oracle's FP64 true residual, lattice by lattice."""
import numpy as np
import pytest

import oracle
from paper_1009_5169_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sf():
    from paper_1009_5169_gb300 import binding, build
    build.build()
    return binding


def _solve_batch(sf, lts, nrhs, algo, tol, check, groups=None):
    Us = [lt.make_links() for lt in lts]
    phis = [lt.make_sources(nrhs) for lt in lts]
    lats = [sf.Lattice(lt.L, lt.T, lt.theta, lt.kappa, lt.beta, torch.from_numpy(U).cuda())
            for lt, U in zip(lts, Us)]
    b = sf.Batch(lats, nrhs)
    if groups is not None:
        assert b.num_groups == groups
    P = [torch.from_numpy(p).cuda() for p in phis]
    X = [torch.empty_like(p) for p in P]
    Y = [torch.empty_like(p) for p in P]
    infos = b.solve(algo, P, X, Y, tol=tol, maxiter=5000)
    for l in check:
        lt = lts[l]
        Xn, Yn = X[l].cpu().numpy(), Y[l].cpu().numpy()
        rx = oracle.true_residual(Us[l], phis[l], Xn, lt.L, lt.T, lt.theta, lt.kappa)
        ry = oracle.true_residual(Us[l], Xn, Yn, lt.L, lt.T, lt.theta, lt.kappa, dagger=True)
        assert np.all(rx <= tol * 1.05), (l, rx, infos[l])
        assert np.all(ry <= tol * 1.05), (l, ry, infos[l])
    for inf in infos:
        assert max(inf["true_resid"]) <= tol and max(inf["true_resid_y"]) <= tol
    b.close()
    for lat in lats:
        lat.close()
    return infos, X, Y


@pytest.mark.parametrize("algo", ["mixed_dc", "bicgstab", "mixed_dc_half", "cg_normal"])
def test_small_uneven_batch(sf, algo):
    lts = [inputs.Lattice(4, 4, 0.3, 0.125, 101), inputs.Lattice(6, 5, 0.35, 0.13, 102),
           inputs.Lattice(8, 8, 0.25, 0.13, 103), inputs.Lattice(4, 7, 0.2, 0.12, 104)]
    _solve_batch(sf, lts, 3, algo, 1e-10, check=range(len(lts)))


@pytest.mark.parametrize("algo", ["mixed_dc", "cg_normal"])
def test_batch_split_into_groups(sf, algo, monkeypatch):
    """A batch whose lattices do not fit the grouping budget together is
    solved as several groups (first-fit, largest first), each with its own
    workspace and tiling; every lattice still meets the oracle's residual.
    The budget here admits the 8^4 lattice alone and the three smaller ones
    together."""
    lts = [inputs.Lattice(4, 4, 0.3, 0.125, 101), inputs.Lattice(6, 5, 0.35, 0.13, 102),
           inputs.Lattice(8, 8, 0.25, 0.13, 103), inputs.Lattice(4, 7, 0.2, 0.12, 104)]
    nrhs = 3
    ws = [lt.L ** 3 * (lt.T - 1) // 2 for lt in lts]
    vpad = [(v + 63) // 64 * 64 for v in ws]
    per = [v * (4 * 2 * 3 * 16 + nrhs * 6 * 96) for v in vpad]
    budget = max(per[0] + per[1] + per[3], per[2])
    assert per[2] + min(per[0], per[1], per[3]) > budget
    monkeypatch.setenv("SF_BATCH_BUDGET_BYTES", str(budget))
    _solve_batch(sf, lts, nrhs, algo, 1e-10, check=range(len(lts)), groups=2)


def test_batch_matches_single_lattice_solves(sf):
    lts = [inputs.Lattice(6, 6, 0.3, 0.13, 111), inputs.Lattice(8, 6, 0.3, 0.13, 112)]
    infos, Xb, Yb = _solve_batch(sf, lts, 2, "mixed_dc", 1e-11, check=[])
    for l, lt in enumerate(lts):
        U = lt.make_links()
        phi = torch.from_numpy(lt.make_sources(2)).cuda()
        lat = sf.Lattice(lt.L, lt.T, lt.theta, lt.kappa, lt.beta, U)
        X = torch.empty_like(phi)
        sf.solve_block(lat, "mixed_dc", phi, X, None, tol=1e-11)
        # both are within 1e-11 of the same solution; cond(Dhat) is O(10) here
        d = (X - Xb[l]).abs().max().item() / X.abs().max().item()
        assert d <= 1e-8
        lat.close()


@pytest.mark.parametrize("algo", ["mixed_dc", "cg_normal"])
def test_batched_uneven_workload(sf, algo):
    """The full batched workload: 24 fields, 8 each of 8^4, 12^4, 16^4, eps
    cycling 0.15/0.25/0.35, kappa 0.13, 5 RHS, FP32 inner / FP64 outer, by
    the defect-correction BiCGStab and by the normal-equation CG route (the
    one the bench times); X and Y of every RHS of all 24 lattices judged by
    the oracle's true residual."""
    w = inputs.workload("batched_uneven")
    _solve_batch(sf, w.lattices, w.nrhs, algo, w.tol, check=range(len(w.lattices)))
