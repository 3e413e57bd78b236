"""GPU parity of each step of Algorithm 1 against the CPU oracle (FP64 DFMA kernels)."""
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


@pytest.mark.parametrize("cplx", [True, False])
@pytest.mark.parametrize("n,k", [(200, 37), (129, 1), (64, 64)])
def test_hemm_native(pkg, cplx, n, k):
    p = G.problem_small(n, 2, 2, complex_=cplx, seed_pid=n)
    A = p.dense()
    B = G.gaussian(np.random.default_rng(1), (n, k), cplx)
    s = pkg.Chase(n, max(k, 4), complex_=cplx)
    C = host(s.hemm(dev(A), dev(B), "fp64_native"))
    ref = A @ B
    assert np.max(np.abs(C - ref)) <= 1e-13 * np.max(np.abs(ref)) * np.sqrt(n)


@pytest.mark.parametrize("cplx", [True, False])
def test_filter_native_vs_oracle(pkg, cplx):
    n, k = 300, 21
    p = G.problem_small(n, 8, 13, complex_=cplx, seed_pid=3)
    A = p.dense()
    V = p.V0[:, :k]
    m = np.sort(np.random.default_rng(5).integers(1, 37, size=k))
    b_sup, mu_1, mu_ne = 1.05, -1.0, -0.7
    ref, mv = O.chebyshev_filter(A, V, m, b_sup, mu_1, mu_ne)
    s = pkg.Chase(n, k, complex_=cplx)
    Vt = dev(V)
    s.filter(dev(A), Vt, m, b_sup, mu_1, mu_ne, "fp64_native")
    out = host(Vt)
    scale = np.max(np.abs(ref), axis=0)
    assert np.max(np.abs(out - ref) / scale[None, :]) <= 1e-11


def test_qr_native(pkg):
    n, k, l = 257, 30, 7
    g = np.random.default_rng(9)
    Y, _ = np.linalg.qr(g.standard_normal((n, l)) + 1j * g.standard_normal((n, l)))
    X = g.standard_normal((n, k - l)) + 1j * g.standard_normal((n, k - l))
    X[:, 3] = X[:, 2] * 1e-3 + X[:, 3] * 1e-9  # ill-conditioned pair
    s = pkg.Chase(n, k, complex_=True)
    Xt = dev(np.concatenate([Y, X], axis=1))
    s.qr(Xt, nlocked=l)
    Q = host(Xt)
    assert np.array_equal(Q[:, :l], Y)
    assert np.max(np.abs(np.conj(Q.T) @ Q - np.eye(k))) <= 1e-12
    Qo = O.qr_step(Y, X)
    assert subspace_sin(Q, Qo) <= 1e-7  # span of [Y X]; the ill-conditioned pair limits it


@pytest.mark.parametrize("cplx", [True, False])
@pytest.mark.parametrize("k", [1, 2, 17, 64, 101])
def test_heevj_vs_lapack(pkg, cplx, k):
    g = np.random.default_rng(k)
    X = g.standard_normal((k, k)) + (1j * g.standard_normal((k, k)) if cplx else 0)
    H = 0.5 * (X + np.conj(X.T))
    s = pkg.Chase(max(k, 2), k, complex_=cplx)
    w, Zt = s.heevj(dev(H))
    Z = host(Zt)
    nrm = np.linalg.norm(H, 2)
    assert np.max(np.abs(w - np.linalg.eigvalsh(H))) <= 1e-13 * nrm * max(1, np.sqrt(k) / 4)
    assert np.max(np.abs(H @ Z - Z * w)) <= 1e-13 * nrm * max(1, np.sqrt(k) / 4)
    assert np.max(np.abs(np.conj(Z.T) @ Z - np.eye(k))) <= 1e-13 * max(1, np.sqrt(k) / 4)


def test_heevj_oracle_cross_check(pkg):
    g = np.random.default_rng(77)
    k = 40
    X = g.standard_normal((k, k)) + 1j * g.standard_normal((k, k))
    H = 0.5 * (X + np.conj(X.T))
    wo, _ = O.jacobi_eigh(H)
    s = pkg.Chase(k, k, complex_=True)
    w, _ = s.heevj(dev(H))
    assert np.max(np.abs(w - wo)) <= 1e-13 * np.linalg.norm(H, 2)


@pytest.mark.parametrize("cplx", [True, False])
def test_rayleigh_ritz_vs_oracle(pkg, cplx):
    n, k = 180, 24
    p = G.problem_small(n, 10, 14, complex_=cplx, seed_pid=4)
    A = p.dense()
    Q, _ = np.linalg.qr(p.V0[:, :k])
    wo, Vo = O.rayleigh_ritz(A, Q)
    ro = O.residuals(A, Vo, wo)
    s = pkg.Chase(n, k, complex_=cplx)
    Qt = dev(Q)
    w, r = s.rayleigh_ritz(dev(A), Qt)
    V = host(Qt)
    assert np.max(np.abs(w - wo)) <= 1e-13
    assert np.max(np.abs(r - ro)) <= 1e-12
    Rt = A @ V - V * w[None, :]
    assert np.max(np.abs(np.linalg.norm(Rt, axis=0) - r)) <= 1e-12


@pytest.mark.parametrize("cplx", [True, False])
def test_lanczos_vs_oracle(pkg, cplx):
    n = 400
    p = G.problem_small(n, 20, 10, complex_=cplx, seed_pid=8)
    A = p.dense()
    ref = O.lanczos_bounds(A, p.L0, 25, p.ne)
    s = pkg.Chase(n, p.ne, complex_=cplx)
    out = s.lanczos(dev(A), p.ne, dev(p.L0), 4, 25)
    for key, val in (("b_sup", ref.b_sup), ("mu_1", ref.mu_1), ("mu_ne", ref.mu_ne), ("theta_max", ref.theta_max)):
        assert abs(out[key] - val) <= 1e-10 * max(1.0, abs(val)), key


def test_generator_matches_host(pkg):
    import torch
    n = 300
    p = G.problem_small(n, 4, 4, complex_=True, k_reflect=6, seed_pid=11)
    B, D = G.wy_factors(p.lam, p.U)
    s = pkg.Chase(n, 8, complex_=True)
    At = torch.empty((n, n), dtype=torch.complex128, device="cuda:0")
    s.generate(At, torch.from_numpy(p.lam).cuda(), dev(p.U), dev(B), dev(D))
    Ad = host(At)
    assert np.array_equal(Ad, np.conj(Ad.T))
    assert np.max(np.abs(Ad - p.dense())) <= 1e-14 * np.sqrt(n)


def _solve(pkg, p, mode, A=None):
    A = p.dense() if A is None else A
    s = pkg.Chase(p.n, p.ne, complex_=p.complex_)
    w, Vt = s.solve(dev(A), p.nev, p.nex, p.tol, p.deg, mode, dev(p.V0), dev(p.L0))
    return w.cpu().numpy(), host(Vt), s.stats()


@pytest.mark.parametrize("cplx,n,nev,nex", [(True, 40, 4, 4), (False, 64, 6, 6), (True, 96, 8, 4), (True, 300, 12, 6)])
def test_solve_native_small_vs_oracle(pkg, cplx, n, nev, nex):
    p = G.problem_small(n, nev, nex, complex_=cplx, seed_pid=n)
    A = p.dense()
    ref = O.chase_solve(A, nev, nex, p.tol, p.deg, p.maxdeg, p.V0, p.L0, p.lanczos_steps)
    w, V, st = _solve(pkg, p, "fp64_native", A)
    nrm = p.norm2()
    assert np.max(np.abs(w - ref.eigvals)) <= 1e-10 * nrm
    assert np.max(np.abs(w - p.lam[:nev])) <= 1e-10 * nrm
    R = A @ V - V * w[None, :]
    assert np.max(np.linalg.norm(R, axis=0)) <= 1e-10 * nrm * 1.01
    assert np.max(np.abs(np.conj(V.T) @ V - np.eye(nev))) <= 1e-12
    assert abs(st["iterations"] - ref.iterations) <= 1


def test_solve_native_c1_vs_oracle(pkg):
    p = G.problem_c1()
    A = p.dense()
    ref = O.chase_solve(A, p.nev, p.nex, p.tol, p.deg, p.maxdeg, p.V0, p.L0, p.lanczos_steps)
    w, V, st = _solve(pkg, p, "fp64_native", A)
    nrm = p.norm2()
    assert np.max(np.abs(w - ref.eigvals)) <= 1e-10 * nrm
    R = G.implicit_matvec(p.lam, p.U, V) - V * w[None, :]
    assert np.max(np.linalg.norm(R, axis=0)) <= 1e-10 * nrm * 1.01
    # Davis-Kahan: sin angle(span V, exact) <= ||R||_F / gap, gap = lambda_{nev+1} - lambda_nev
    E = G.exact_eigvecs(p.U, np.arange(p.nev))
    gap = p.lam[p.nev] - p.lam[p.nev - 1]
    rf = np.linalg.norm(R)
    Ro = G.implicit_matvec(p.lam, p.U, ref.eigvecs) - ref.eigvecs * ref.eigvals[None, :]
    assert subspace_sin(E, V) <= max(1e-8, 1.01 * rf / gap)
    assert subspace_sin(ref.eigvecs, V) <= max(1e-8, 1.01 * (rf + np.linalg.norm(Ro)) / gap)
    assert abs(st["iterations"] - ref.iterations) <= 1
    assert abs(st["matvecs"] - ref.matvecs) <= 0.1 * ref.matvecs


def test_solve_121_closed_form_gpu(pkg):
    n = 200
    A = G.matrix_121(n)
    p = G.from_dense("121", A, 8, 6)
    w, V, st = _solve(pkg, p, "fp64_native", A)
    assert np.max(np.abs(w - G.spectrum_121(n)[:8])) <= 1e-10 * 4


def test_errors_are_statuses(pkg):
    import torch
    p = G.problem_small(50, 4, 4, complex_=True)
    A = p.dense()
    A[3, 7] = np.nan
    s = pkg.Chase(p.n, p.ne, complex_=True)
    with pytest.raises(pkg.ChaseError) as ei:
        s.solve(dev(A), p.nev, p.nex, p.tol, p.deg, "fp64_native", dev(p.V0), dev(p.L0))
    assert ei.value.status == 5
    with pytest.raises(pkg.ChaseError) as ei:
        big = torch.zeros((60, 60), dtype=torch.complex128, device="cuda:0")
        s.solve(big, 4, 4, 1e-10, 20, "fp64_native", dev(np.zeros((60, 8), complex)), dev(np.zeros((60, 4), complex)))
    assert ei.value.status == 1
    s2 = pkg.Chase(p.n, p.ne, complex_=True)
    import ctypes as C
    w = torch.empty(4, dtype=torch.float64, device="cuda:0")
    assert s2.lib.chase_eigvals(s2.ctx, C.c_void_p(w.data_ptr()), 1) == 7
