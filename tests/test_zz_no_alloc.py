"""The allocation-free eigensolve entry point (chase_heevj_noalloc) against chase_heevj.

Callers whose device memory is reserved by someone else (a framework's caching
allocator, an application arena) cannot call cudaMalloc; chase_heevj_noalloc
serves them from a fixed scratch array in the library.  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2205_02491_gb300 as P
    from paper_2205_02491_gb300 import _lib
    return torch, P, _lib.load(), _lib


def _herm(k, cplx, seed):
    g = np.random.default_rng(seed)
    X = g.standard_normal((k, k)) + (1j * g.standard_normal((k, k)) if cplx else 0)
    return 0.5 * (X + np.conj(X.T))


@pytest.mark.parametrize("cplx,k", [(True, 200), (False, 256), (True, 1)])
def test_noalloc_matches_heevj_on_two_calls(env, cplx, k):
    torch, P, lib, L = env
    dt = torch.complex128 if cplx else torch.float64
    ref_ctx = P.Chase(max(k, 2), k, complex_=cplx)
    for call in range(2):
        H = _herm(k, cplx, 100 * call + k)
        Gt = torch.from_numpy(np.ascontiguousarray(H.T)).cuda()
        w_ref, Zref_t = ref_ctx.heevj(Gt)
        Zt = torch.empty((k, k), dtype=dt, device="cuda")
        w = np.zeros(k)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = lib.chase_heevj_noalloc(C.c_void_p(Gt.data_ptr()), k, k, L.CHASE_C128 if cplx else L.CHASE_R64,
                                     w.ctypes.data_as(C.c_void_p), C.c_void_p(Zt.data_ptr()), k, None)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert st == 0
        if call == 1:
            assert free1 == free0  # no device allocation by the call
        nrm = max(1.0, np.linalg.norm(H, 2))
        assert np.max(np.abs(w - w_ref)) <= 1e-13 * nrm
        Z = Zt.cpu().numpy().T
        Zr = Zref_t.cpu().numpy().T
        # same eigenvectors up to a unit phase per column
        ov = np.abs(np.sum(np.conj(Zr) * Z, axis=0))
        assert np.max(np.abs(ov - 1.0)) <= 1e-12
        assert np.max(np.abs(H @ Z - Z * w)) <= 1e-13 * nrm * max(1, np.sqrt(k) / 4)
    ref_ctx.close()


def test_noalloc_rejects_oversize(env):
    torch, P, lib, L = env
    k = 257
    Gt = torch.zeros((k, k), dtype=torch.complex128, device="cuda")
    Zt = torch.zeros_like(Gt)
    w = np.zeros(k)
    st = lib.chase_heevj_noalloc(C.c_void_p(Gt.data_ptr()), k, k, L.CHASE_C128, w.ctypes.data_as(C.c_void_p),
                                 C.c_void_p(Zt.data_ptr()), k, None)
    assert st == 1  # CHASE_ERR_ARG
