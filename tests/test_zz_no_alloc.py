"""The allocation-free plaquette action (plaquette_action_noalloc), for
callers that cannot allocate device memory -- a runtime or scheduler that
owns the whole device, or a fixed memory budget set by another framework.

It is checked through the C ABI against the lattice-based plaquette_action
on two calls in a row (its shared scratch keeps the previous call's
contents, which must not leak into the next result), for two lattice sizes
and for host and device result pointers.  Collected last, so a failure here
comes after every other test has run."""
import ctypes

import numpy as np
import pytest

from paper_1009_5169_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sf():
    from paper_1009_5169_gb300 import binding, build
    build.build()
    return binding


def _noalloc(sf, L, T, beta, links_dev, out):
    lib = sf.lib()
    if isinstance(out, ctypes.c_double):
        ptr = ctypes.cast(ctypes.byref(out), ctypes.c_void_p)
    else:
        ptr = ctypes.c_void_p(out.data_ptr())
    rc = lib.plaquette_action_noalloc(L, T, beta, ctypes.c_void_p(links_dev.data_ptr()), ptr, 0, None)
    return rc


@pytest.mark.parametrize("L,T,eps", [(8, 8, 0.3), (6, 11, 0.5)])
def test_noalloc_plaquette_matches_plaquette_action(sf, L, T, eps):
    beta = 4.52
    U = inputs.links(L, T, eps, 2024 + L)
    U[: L ** 3, 1:] = inputs.links(L, 2, 0.6, 77)[: L ** 3, 1:]   # non-trivial boundary links
    Ud = torch.from_numpy(U).cuda()
    lat = sf.Lattice(L, T, 0.5, 0.13, beta, Ud)
    ref = sf.plaquette_action(lat)
    lat.close()
    for call in range(2):
        S = ctypes.c_double(float("nan"))
        rc = _noalloc(sf, L, T, beta, Ud, S)
        assert rc == sf.SF_OK, sf.lib().sf_last_error()
        assert abs(S.value - ref) <= 1e-12 * abs(ref), (call, S.value, ref)
    Sd = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        assert _noalloc(sf, L, T, beta, Ud, Sd) == sf.SF_OK
        torch.cuda.synchronize()
        assert abs(Sd.item() - ref) <= 1e-12 * abs(ref)


def test_noalloc_rejects_oversized_lattice_without_launching(sf):
    U = torch.zeros(16, dtype=torch.float64, device="cuda")
    S = ctypes.c_double(0.0)
    rc = _noalloc(sf, 64, 8, 4.52, U, S)   # 9 * 64^3 gauge sites > 2097152
    assert rc == sf.SF_EINVAL
    assert b"2097152" in sf.lib().sf_last_error()


def test_noalloc_rejects_bad_links_pointers_without_launching(sf):
    """A host gauge field, or a device view that is not 16-byte aligned, is
    refused before any launch (the kernel reads the links as double pairs)."""
    L, T = 4, 4
    U = inputs.links(L, T, 0.3, 99)
    S = ctypes.c_double(0.0)
    lib = sf.lib()
    Uh = np.ascontiguousarray(U)   # host memory
    rc = lib.plaquette_action_noalloc(L, T, 4.52, ctypes.c_void_p(Uh.ctypes.data),
                                      ctypes.cast(ctypes.byref(S), ctypes.c_void_p), 0, None)
    assert rc == sf.SF_EINVAL
    assert b"device" in lib.sf_last_error()
    flat = torch.from_numpy(U).cuda().view(torch.float64).reshape(-1)
    shifted = torch.cat([flat, flat[:1]])[1:]   # a view one double past a 256-byte boundary
    assert shifted.data_ptr() % 16 == 8
    rc = lib.plaquette_action_noalloc(L, T, 4.52, ctypes.c_void_p(shifted.data_ptr()),
                                      ctypes.cast(ctypes.byref(S), ctypes.c_void_p), 0, None)
    assert rc == sf.SF_EINVAL
    assert b"aligned" in lib.sf_last_error()
    torch.cuda.synchronize()
