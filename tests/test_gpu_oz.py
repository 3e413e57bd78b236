"""Split-BF16 tensor-core products (tcgen05) against exact products and the oracle."""
import numpy as np
import pytest

from gen import problems as G
from oracle import chase_oracle as O
from tests.helpers import dev, host, subspace_sin

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2205_02491_gb300 as P
    return P


def _rel_err(C, ref, A, B):
    # error relative to the per-row / per-column scales the split uses, per K term
    ra = np.max(np.maximum(np.abs(A.real), np.abs(A.imag)), axis=1)
    cb = np.max(np.maximum(np.abs(B.real), np.abs(B.imag)), axis=0)
    return np.max(np.abs(C - ref) / (ra[:, None] * cb[None, :])) / A.shape[1]


def _exact(A, B):
    # A B in extended precision (complex via longdouble real parts)
    Ar = np.real(A).astype(np.longdouble)
    Ai = np.imag(A).astype(np.longdouble)
    Br = np.real(B).astype(np.longdouble)
    Bi = np.imag(B).astype(np.longdouble)
    return (Ar @ Br - Ai @ Bi).astype(np.float64) + 1j * (Ar @ Bi + Ai @ Br).astype(np.float64)


@pytest.mark.parametrize("n,k", [(300, 70), (129, 1), (1000, 130)])
def test_hemm_fp64_split_complex(pkg, n, k):
    p = G.problem_small(n, 2, 2, complex_=True, seed_pid=n + 1)
    A = p.dense()
    B = G.gaussian(np.random.default_rng(n), (n, k), True)
    s = pkg.Chase(n, k, complex_=True)
    C = host(s.hemm(dev(A), dev(B), "fp64"))
    ref = _exact(A, B)
    assert _rel_err(C, ref, A, B) <= 2.0 ** -53


@pytest.mark.parametrize("cplx,n,k", [(True, 4096, 16), (True, 5000, 6), (False, 3000, 8), (False, 2500, 70)])
def test_hemm_split_along_k(pkg, cplx, n, k):
    """Products with few output tiles are split along K (FP64 partial sums per slice, then one reduction);
    the narrow Lanczos-width case (up to 8 complex / 16 real columns) takes the 16-column tile.  Same
    per-term bound as the unsplit products."""
    p = G.problem_small(n, 2, 2, complex_=cplx, seed_pid=n + 3)
    A = p.dense()
    B = G.gaussian(np.random.default_rng(n + 1), (n, k), cplx)
    s = pkg.Chase(n, max(k, 4), complex_=cplx)
    C = host(s.hemm(dev(A), dev(B), "fp64"))
    if cplx:
        ref = _exact(A, B)
        assert _rel_err(C, ref, A, B) <= 2.0 ** -53
    else:
        ref = (A.astype(np.longdouble) @ B.astype(np.longdouble)).astype(np.float64)
        ra = np.max(np.abs(A), axis=1)
        cb = np.max(np.abs(B), axis=0)
        assert np.max(np.abs(C - ref) / (ra[:, None] * cb[None, :])) / n <= 2.0 ** -53


@pytest.mark.parametrize("n,k", [(257, 200), (64, 3)])
def test_hemm_fp64_split_real(pkg, n, k):
    p = G.problem_small(n, 2, 2, complex_=False, seed_pid=n + 2)
    A = p.dense()
    B = np.random.default_rng(n).standard_normal((n, k))
    s = pkg.Chase(n, k, complex_=False)
    C = host(s.hemm(dev(A), dev(B), "fp64"))
    ref = (A.astype(np.longdouble) @ B.astype(np.longdouble)).astype(np.float64)
    ra = np.max(np.abs(A), axis=1)
    cb = np.max(np.abs(B), axis=0)
    assert np.max(np.abs(C - ref) / (ra[:, None] * cb[None, :])) / n <= 2.0 ** -53


def test_exact_levels_at_worst_case_sums(pkg):
    # all-positive operands near the row/column maxima make every level sum as large as the
    # exactness bound allows; an inexact FP32 level sum would show up as ~2^-24 relative error
    n, k = 1024, 64
    g = np.random.default_rng(3)
    X = g.uniform(0.995, 1.0, (n, n)) + 1j * g.uniform(0.995, 1.0, (n, n))
    A = 0.5 * (X + np.conj(X.T))
    B = g.uniform(0.995, 1.0, (n, k)) - 1j * g.uniform(0.995, 1.0, (n, k))
    s = pkg.Chase(n, k, complex_=True)
    C = host(s.hemm(dev(A), dev(B), "fp64"))
    ref = _exact(A, B)
    assert np.max(np.abs(C - ref) / np.abs(ref)) <= 1e-14


@pytest.mark.parametrize("mode,bound", [("bf16x3", 2.0 ** -13), ("bf16x6", 2.0 ** -20)])
def test_hemm_mixed_modes(pkg, mode, bound):
    n, k = 512, 96
    p = G.problem_small(n, 2, 2, complex_=True, seed_pid=5)
    A = p.dense()
    B = G.gaussian(np.random.default_rng(9), (n, k), True)
    s = pkg.Chase(n, k, complex_=True)
    C = host(s.hemm(dev(A), dev(B), mode))
    ref = _exact(A, B)
    assert _rel_err(C, ref, A, B) <= bound


def test_filter_fp64_split_vs_oracle(pkg):
    n, k = 400, 33
    p = G.problem_small(n, 10, 23, complex_=True, seed_pid=12)
    A = p.dense()
    V = p.V0[:, :k]
    m = np.sort(np.random.default_rng(2).integers(1, 37, size=k))
    ref, _ = O.chebyshev_filter(A, V, m, 1.05, -1.0, -0.7)
    s = pkg.Chase(n, k, complex_=True)
    Vt = dev(V)
    s.filter(dev(A), Vt, m, 1.05, -1.0, -0.7, "fp64")
    out = host(Vt)
    scale = np.max(np.abs(ref), axis=0)
    assert np.max(np.abs(out - ref) / scale[None, :]) <= 1e-11


def _solve(pkg, p, mode, A):
    s = pkg.Chase(p.n, p.ne, complex_=p.complex_)
    w, Vt = s.solve(dev(A), p.nev, p.nex, p.tol, p.deg, mode, dev(p.V0), dev(p.L0))
    return w.cpu().numpy(), host(Vt), s.stats()


@pytest.mark.parametrize("cplx,n,nev,nex", [(True, 96, 8, 4), (False, 300, 12, 6), (True, 700, 20, 10)])
def test_solve_fp64_split_vs_oracle(pkg, cplx, n, nev, nex):
    p = G.problem_small(n, nev, nex, complex_=cplx, seed_pid=n + 7)
    A = p.dense()
    ref = O.chase_solve(A, nev, nex, p.tol, p.deg, p.maxdeg, p.V0, p.L0, p.lanczos_steps)
    w, V, st = _solve(pkg, p, "fp64", A)
    nrm = p.norm2()
    assert np.max(np.abs(w - ref.eigvals)) <= 1e-10 * nrm
    R = A @ V - V * w[None, :]
    assert np.max(np.linalg.norm(R, axis=0)) <= 1e-10 * nrm * 1.01
    assert abs(st["iterations"] - ref.iterations) <= 1


def test_solve_with_library_start_vectors(pkg):
    """chase_solve with V0 and L0 left to the library (null): it draws them with the header's seeded
    generator, reaches the prescribed spectrum, and takes the iterations of the oracle run from the host
    restatement of the same vectors (within one)."""
    p = G.problem_c1()
    A = p.dense()
    s = pkg.Chase(p.n, p.ne, complex_=True)
    w, Vt = s.solve(dev(A), p.nev, p.nex, p.tol, p.deg, "fp64")
    w = w.cpu().numpy()
    V = host(Vt)
    nrm = p.norm2()
    assert np.max(np.abs(w - p.lam[:p.nev])) <= 1e-10 * nrm
    R = G.implicit_matvec(p.lam, p.U, V) - V * w[None, :]
    assert np.max(np.linalg.norm(R, axis=0)) <= 1e-10 * nrm * 1.01
    V0 = G.library_start_vectors(p.n, p.ne, G.LIBRARY_SEED_V0, True)
    L0 = G.library_start_vectors(p.n, 4, G.LIBRARY_SEED_L0, True)
    ref = O.chase_solve(A, p.nev, p.nex, p.tol, p.deg, p.maxdeg, V0, L0, p.lanczos_steps)
    assert abs(s.stats()["iterations"] - ref.iterations) <= 1


@pytest.mark.parametrize("mode", ["fp64", "bf16x3", "bf16x6"])
def test_solve_c1_modes(pkg, mode):
    p = G.problem_c1()
    A = p.dense()
    ref = O.chase_solve(A, p.nev, p.nex, p.tol, p.deg, p.maxdeg, p.V0, p.L0, p.lanczos_steps)
    w, V, st = _solve(pkg, p, mode, A)
    nrm = p.norm2()
    assert np.max(np.abs(w - ref.eigvals)) <= 1e-10 * nrm
    assert np.max(np.abs(w - p.lam[:p.nev])) <= 1e-10 * nrm
    R = G.implicit_matvec(p.lam, p.U, V) - V * w[None, :]
    assert np.max(np.linalg.norm(R, axis=0)) <= 1e-10 * nrm * 1.01
    E = G.exact_eigvecs(p.U, np.arange(p.nev))
    gap = p.lam[p.nev] - p.lam[p.nev - 1]
    assert subspace_sin(E, V) <= max(1e-8, 1.01 * np.linalg.norm(R) / gap)
    if mode != "fp64":
        assert st["lowp_iterations"] >= 1


SPLIT_ALL = {"native_below_mflop": 0}


def test_qr_split_products(pkg):
    n, k, l = 700, 48, 9
    g = np.random.default_rng(19)
    Y, _ = np.linalg.qr(g.standard_normal((n, l)) + 1j * g.standard_normal((n, l)))
    X = g.standard_normal((n, k - l)) + 1j * g.standard_normal((n, k - l))
    X[:, 5] = X[:, 4] + 1e-6 * X[:, 5]
    s = pkg.Chase(n, k, complex_=True, opts=SPLIT_ALL)
    Xt = dev(np.concatenate([Y, X], axis=1))
    s.qr(Xt, nlocked=l)
    Q = host(Xt)
    assert np.array_equal(Q[:, :l], Y)
    assert np.max(np.abs(np.conj(Q.T) @ Q - np.eye(k))) <= 1e-12
    assert subspace_sin(Q, O.qr_step(Y, X)) <= 1e-6


@pytest.mark.parametrize("cplx", [True, False])
def test_rayleigh_ritz_split_products(pkg, cplx):
    n, k = 600, 40
    p = G.problem_small(n, 20, 20, complex_=cplx, seed_pid=21)
    A = p.dense()
    Q, _ = np.linalg.qr(p.V0[:, :k])
    wo, Vo = O.rayleigh_ritz(A, Q)
    ro = O.residuals(A, Vo, wo)
    s = pkg.Chase(n, k, complex_=cplx, opts=SPLIT_ALL)
    Qt = dev(Q)
    w, r = s.rayleigh_ritz(dev(A), Qt)
    V = host(Qt)
    assert np.max(np.abs(w - wo)) <= 1e-12
    assert np.max(np.abs(r - ro)) <= 1e-11
    assert np.max(np.abs(np.conj(V.T) @ V - np.eye(k))) <= 1e-12


@pytest.mark.parametrize("mode", ["fp64", "bf16x6"])
def test_solve_c1_all_split_products(pkg, mode):
    p = G.problem_c1()
    A = p.dense()
    s = pkg.Chase(p.n, p.ne, complex_=True, opts=SPLIT_ALL)
    w, Vt = s.solve(dev(A), p.nev, p.nex, p.tol, p.deg, mode, dev(p.V0), dev(p.L0))
    w = w.cpu().numpy()
    V = host(Vt)
    nrm = p.norm2()
    assert np.max(np.abs(w - p.lam[:p.nev])) <= 1e-10 * nrm
    R = G.implicit_matvec(p.lam, p.U, V) - V * w[None, :]
    assert np.max(np.linalg.norm(R, axis=0)) <= 1e-10 * nrm * 1.01


@pytest.mark.parametrize("cplx,k,fine", [(True, 160, False), (False, 160, False), (True, 97, False),
                                         (True, 300, False), (False, 300, False), (False, 300, True)])
def test_rayleigh_ritz_mixed_eigensolve(pkg, cplx, k, fine):
    # k >= 64 takes the FP32 Jacobi + FP64-class refinement path (k >= 128: block Jacobi, blocks of 32 paired
    # in a round-robin tournament; below: the scalar cooperative sweep); include exact eigenvalue clusters;
    # odd k exercises the dummy index of the scalar round-robin order, k = 160 an odd block count (a padding
    # block), k = 300 a partial last block
    n = 900
    g = np.random.default_rng(31)
    lam = np.sort(g.uniform(-1, 1, n))
    lam[10:13] = lam[10]          # a triple eigenvalue inside the projected window
    lam[40] = lam[41] + 1e-9       # a near-degenerate pair
    if fine:
        # a dense stretch: 250 eigenvalues 2e-4 apart (relative gaps like the Table 2 Geometric spectrum's),
        # where the FP32 pass must stop well below the gaps for the FP64 corrections to converge
        lam[50:300] = lam[50] + 2e-4 * np.arange(250)
    lam = np.sort(lam)
    p = G.problem_small(n, 100, max(60, k - 100), complex_=cplx, lam=lam, seed_pid=31)
    A = p.dense()
    # a basis of (nearly) the lowest eigenvectors, mixed by a random unitary so that the quotient is
    # full; the 1e-7 perturbation moves Ritz values by ~1e-14, so the clusters survive in G
    E = G.exact_eigvecs(p.U, np.arange(k))
    R, _ = np.linalg.qr(p.V0[:k, :k])
    Q, _ = np.linalg.qr(E @ R + 1e-7 * p.V0[:, :k])
    wo, Vo = O.rayleigh_ritz(A, Q)
    s = pkg.Chase(n, k, complex_=cplx)
    Qt = dev(Q)
    w, r = s.rayleigh_ritz(dev(A), Qt)
    V = host(Qt)
    assert np.max(np.abs(w - wo)) <= 1e-12
    Rt = A @ V - V * w[None, :]
    assert np.max(np.linalg.norm(Rt, axis=0) - r) <= 1e-11
    assert np.max(np.abs(np.conj(V.T) @ V - np.eye(k))) <= 1e-12
    st = s.stats()
    assert st["rr_fallbacks"] == 0
    assert st["rr_clusters"] >= 1


@pytest.mark.parametrize("pinned", [True, False])
def test_solve_host_buffers_match_device(pkg, pinned):
    """chase_solve given host A, V0, L0 (pinned or pageable) copies them itself and returns the same
    eigenpairs as the device-pointer call."""
    import torch
    p = G.problem_c1()
    A = p.dense()
    s = pkg.Chase(p.n, p.ne, complex_=True)
    w_d, V_d = s.solve(dev(A), p.nev, p.nex, p.tol, p.deg, "fp64", dev(p.V0), dev(p.L0))
    hostT = lambda x: torch.from_numpy(np.ascontiguousarray(np.asarray(x).T))
    Ah, V0h, L0h = hostT(A), hostT(p.V0), hostT(p.L0)
    if pinned:
        Ah, V0h, L0h = Ah.pin_memory(), V0h.pin_memory(), L0h.pin_memory()
    w_h, V_h = s.solve(Ah, p.nev, p.nex, p.tol, p.deg, "fp64", V0h, L0h)
    assert not w_h.is_cuda and not V_h.is_cuda
    assert np.array_equal(w_h.numpy(), w_d.cpu().numpy())
    assert np.array_equal(V_h.numpy(), V_d.cpu().numpy())
    assert np.max(np.abs(w_h.numpy() - p.lam[:p.nev])) <= 1e-10 * p.norm2()
    # caller-owned result buffers (out=): the same pairs, written in place
    w_o = torch.empty(p.nev, dtype=torch.float64, pin_memory=pinned)
    V_o = torch.empty((p.nev, p.n), dtype=torch.complex128, pin_memory=pinned)
    r = s.solve(Ah, p.nev, p.nex, p.tol, p.deg, "fp64", V0h, L0h, out=(w_o, V_o))
    assert r[0] is w_o and r[1] is V_o
    assert np.array_equal(w_o.numpy(), w_d.cpu().numpy())
    assert np.array_equal(V_o.numpy(), V_d.cpu().numpy())
