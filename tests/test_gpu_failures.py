"""Failure paths of the library, each made on the host or by a bounded device wait (nothing faults or
hangs the GPU): out-of-memory at context creation, a numerically rank-deficient block that needs the
shifted Cholesky-QR fallback, the outer-iteration cap, and a grid-barrier wait that reaches its limit."""
import numpy as np
import pytest

from gen import problems as G
from oracle import chase_oracle as O
from tests.helpers import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2205_02491_gb300 as P
    return P


def test_create_oom_is_a_status(pkg):
    """A workspace far beyond device memory is refused before any allocation (Eq. GPU_mem check)."""
    import torch
    free0, _ = torch.cuda.mem_get_info()
    with pytest.raises(pkg.ChaseError) as e:
        pkg.Chase(2_000_000, 64, complex_=True)
    assert e.value.status == 2
    # nothing was left allocated, and a normal context still works
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (64 << 20)
    s = pkg.Chase(64, 8, complex_=True)
    s.close()


def test_maxiter_cap_returns_noconv(pkg):
    p = G.problem_small(200, 8, 6, complex_=True, seed_pid=4)
    s = pkg.Chase(p.n, p.ne, complex_=True, opts={"maxiter": 1})
    with pytest.raises(pkg.ChaseError) as e:
        s.solve(dev(p.dense()), p.nev, p.nex, p.tol, p.deg, "fp64", dev(p.V0), dev(p.L0))
    assert e.value.status == 3
    st = s.stats()
    assert st["iterations"] == 1 and st["locked"] < p.nev
    s.close()


def test_qr_householder_for_numerically_dependent_column(pkg):
    """Two columns equal to 1e-13 relative: Cholesky-QR's first pass sees a pivot at rounding level, so
    the block goes to the Householder QR and still gets an orthonormal basis whose span contains every
    column of X to rounding."""
    n, k = 400, 24
    g = np.random.default_rng(21)
    X = g.standard_normal((n, k)) + 1j * g.standard_normal((n, k))
    X[:, 9] = X[:, 4] + 1e-13 * (g.standard_normal(n) + 1j * g.standard_normal(n))
    s = pkg.Chase(n, k, complex_=True)
    before = s.stats()["qr_householder"]
    Xt = dev(X)
    s.qr(Xt)
    assert s.stats()["qr_householder"] >= before + 1
    Q = host(Xt)
    assert np.max(np.abs(np.conj(Q.T) @ Q - np.eye(k))) <= 1e-12
    # every column of X lies in span(Q)
    R = X - Q @ (np.conj(Q.T) @ X)
    assert np.max(np.linalg.norm(R, axis=0) / np.linalg.norm(X, axis=0)) <= 1e-10
    s.close()


def test_solve_with_near_duplicate_start_columns(pkg):
    """A start block with two nearly equal columns: the first QR goes to the Householder QR and the solve
    still converges to the oracle's eigenvalues (or reports CHASE_ERR_QR_BREAKDOWN, never a wrong
    result)."""
    p = G.problem_small(300, 10, 6, complex_=True, seed_pid=6)
    A = p.dense()
    V0 = p.V0.copy()
    g = np.random.default_rng(3)
    V0[:, 5] = V0[:, 2] + 1e-12 * (g.standard_normal(p.n) + 1j * g.standard_normal(p.n))
    ref = O.chase_solve(A, p.nev, p.nex, p.tol, p.deg, p.maxdeg, p.V0, p.L0, p.lanczos_steps)
    s = pkg.Chase(p.n, p.ne, complex_=True)
    try:
        w, Vt = s.solve(dev(A), p.nev, p.nex, p.tol, p.deg, "fp64", dev(V0), dev(p.L0))
    except pkg.ChaseError as e:
        assert e.status == 4
        return
    assert s.stats()["qr_householder"] >= 1
    assert np.max(np.abs(w.cpu().numpy() - ref.eigvals)) <= 1e-10 * p.norm2()
    V = host(Vt)
    R = A @ V - V * w.cpu().numpy()[None, :]
    assert np.max(np.linalg.norm(R, axis=0)) <= 1e-10 * p.norm2() * 1.01
    s.close()


def test_grid_barrier_wait_limit_returns_timeout_and_context_recovers(pkg):
    """With the wait limit shortened to 1 ns, the first grid barrier of the persistent Jacobi sweep
    (Rayleigh-Ritz eigensolve of the 96 active columns) gives up: every block returns and the solve
    reports CHASE_ERR_TIMEOUT.  With the default limit restored the same context solves normally."""
    p = G.problem_small(400, 64, 32, complex_=True, seed_pid=8)
    A = p.dense()
    s = pkg.Chase(p.n, p.ne, complex_=True)
    At, V0t, L0t = dev(A), dev(p.V0), dev(p.L0)
    pkg.set_wait_limit_ns(1)
    try:
        with pytest.raises(pkg.ChaseError) as e:
            s.solve(At, p.nev, p.nex, p.tol, p.deg, "fp64", V0t, L0t)
        assert e.value.status == 8
    finally:
        pkg.set_wait_limit_ns(0)
    w, _ = s.solve(At, p.nev, p.nex, p.tol, p.deg, "fp64", V0t, L0t)
    assert np.max(np.abs(w.cpu().numpy() - p.lam[:p.nev])) <= 1e-10 * p.norm2()
    s.close()
