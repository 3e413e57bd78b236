"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Every test here runs without a GPU.  Each pin checks the oracle against something
other than itself: a library routine, a closed form, an invariant, brute force or
a value the paper prints (tests/golden/).
"""
import json
import os

import numpy as np
import pytest

from gen import problems as G
from oracle import chase_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Jacobi eig

@pytest.mark.parametrize("k", [1, 2, 3, 7, 16, 33])
@pytest.mark.parametrize("cplx", [False, True])
def test_jacobi_matches_lapack(k, cplx):
    g = np.random.default_rng(k + 100 * cplx)
    X = g.standard_normal((k, k)) + (1j * g.standard_normal((k, k)) if cplx else 0)
    H = 0.5 * (X + np.conj(X.T))
    w, Z = O.jacobi_eigh(H)
    wl = np.linalg.eigvalsh(H)
    nrm = np.linalg.norm(H, 2)
    assert np.max(np.abs(w - wl)) <= 1e-13 * nrm
    assert np.max(np.abs(np.conj(Z.T) @ Z - np.eye(k))) <= 1e-13
    assert np.max(np.abs(H @ Z - Z * w)) <= 1e-13 * nrm
    assert np.all(np.diff(w) >= 0)


def test_jacobi_closed_form_121():
    n = 40
    w, _ = O.jacobi_eigh(G.matrix_121(n))
    assert np.max(np.abs(w - G.spectrum_121(n))) <= 1e-14 * 4


def test_jacobi_wilkinson_vs_sturm():
    for n in (21, 20):
        W = G.matrix_wilkinson(n)
        w, _ = O.jacobi_eigh(W)
        ws = O.tridiag_bisection(np.diag(W).copy(), np.ones(n - 1))
        assert np.max(np.abs(w - ws)) <= 1e-12 * np.max(np.abs(ws))
        assert np.sum(w < 0) == 1  # Table 1: all positive but one


def test_jacobi_degenerate_cluster():
    # exactly repeated eigenvalues: any orthonormal basis of the eigenspace is valid
    g = np.random.default_rng(7)
    Qm, _ = np.linalg.qr(g.standard_normal((12, 12)) + 1j * g.standard_normal((12, 12)))
    lam = np.array([-1.0] * 4 + [0.5] * 5 + [2.0] * 3)
    H = Qm @ np.diag(lam) @ np.conj(Qm.T)
    H = 0.5 * (H + np.conj(H.T))
    w, Z = O.jacobi_eigh(H)
    assert np.max(np.abs(w - lam)) <= 1e-13 * 2
    assert np.max(np.abs(H @ Z - Z * w)) <= 1e-13 * 2


# ---------------------------------------------------------------- paper-printed condition numbers

def _sturm_kth(d, e, j):
    r = np.max(np.abs(d)) + 2.0
    lo, hi = -r, r
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if O.sturm_count(d, e, mid) > j:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def test_condition_numbers_printed_in_paper():
    gold = json.load(open(os.path.join(GOLDEN, "condition_numbers_20k.json")))
    n = gold["n"]
    sig = gold["significant_digits"]

    def same(x, y):
        return float(f"{x:.{sig - 1}e}") == float(f"{y:.{sig - 1}e}")

    lam = G.spectrum_121(n)
    assert same(lam[-1] / lam[0], gold["kappa"]["1-2-1"])
    for name, fn in (("Uniform", G.spectrum_uniform_table1), ("Geometric", G.spectrum_geometric_table1)):
        lam = fn(n)
        assert same(np.max(np.abs(lam)) / np.min(np.abs(lam)), gold["kappa"][name])
    d = G.wilkinson_diagonal(n)
    e = np.ones(n - 1)
    neg = O.sturm_count(d, e, 0.0)
    assert neg == gold["wilkinson_negative_eigenvalues"]
    lmax = _sturm_kth(d, e, n - 1)
    small = min(abs(_sturm_kth(d, e, neg - 1)), abs(_sturm_kth(d, e, neg)))
    assert same(lmax / small, gold["kappa"]["Wilkinson"])


# ---------------------------------------------------------------- generators

def test_dense_generator_matches_prescribed_spectrum_and_wy():
    p = G.problem_small(48, 4, 4, complex_=True, k_reflect=5)
    A = p.dense()
    assert np.allclose(A, np.conj(A.T), atol=0)
    assert np.max(np.abs(np.linalg.eigvalsh(A) - p.lam)) <= 1e-13
    E = G.exact_eigvecs(p.U, np.arange(48))
    assert np.max(np.abs(np.conj(E.T) @ E - np.eye(48))) <= 1e-13
    assert np.max(np.abs(A @ E - E * p.lam)) <= 1e-13
    x = p.V0[:, :3]
    assert np.max(np.abs(G.implicit_matvec(p.lam, p.U, x) - A @ x)) <= 1e-13
    B, D = G.wy_factors(p.lam, p.U)
    n = p.n
    Aw = np.diag(p.lam).astype(complex) - (B @ np.conj(p.U.T)) * p.lam[None, :] \
        - p.lam[:, None] * (p.U @ np.conj(B.T)) + D @ np.conj(B.T)
    assert np.max(np.abs(Aw - A)) <= 1e-13


# ---------------------------------------------------------------- QR

@pytest.mark.parametrize("cplx", [False, True])
def test_householder_qr_invariants(cplx):
    g = np.random.default_rng(3)
    X = g.standard_normal((80, 12)) + (1j * g.standard_normal((80, 12)) if cplx else 0)
    Q, R = O.householder_qr(X)
    assert np.max(np.abs(np.conj(Q.T) @ Q - np.eye(12))) <= 1e-14 * 12
    assert np.linalg.norm(Q @ R - X) <= 1e-14 * np.linalg.norm(X)
    Ql, _ = np.linalg.qr(X)
    # same span as LAPACK's QR
    s = np.linalg.svd(np.conj(Ql.T) @ Q, compute_uv=False)
    assert np.min(s) >= 1 - 1e-13


def test_qr_step_restores_locked():
    g = np.random.default_rng(4)
    Y, _ = np.linalg.qr(g.standard_normal((50, 3)) + 1j * g.standard_normal((50, 3)))
    V = g.standard_normal((50, 5)) + 1j * g.standard_normal((50, 5))
    Q = O.qr_step(Y, V)
    assert np.array_equal(Q[:, :3], Y)
    assert np.max(np.abs(np.conj(Q.T) @ Q - np.eye(8))) <= 1e-13


# ---------------------------------------------------------------- filter

def test_filter_coefficients_reproduce_scaled_chebyshev():
    b_sup, mu_1, mu_ne = 3.0, -2.0, 0.5
    c, e, al, be = O.filter_coefficients(b_sup, mu_1, mu_ne, 30)
    x = np.linspace(-2.5, 3.0, 41)
    y_prev = np.ones_like(x)
    y = al[1] * (x - c) * y_prev
    for s in range(2, 31):
        y, y_prev = al[s] * (x - c) * y + be[s] * y_prev, y
        ref = O.chebyshev_scalar(x, s, b_sup, mu_1, mu_ne)
        assert np.max(np.abs(y - ref) / np.maximum(1, np.abs(ref))) <= 1e-12
    # normalisation: p_m(mu_1) = 1
    assert abs(O.chebyshev_scalar(np.array([mu_1]), 17, b_sup, mu_1, mu_ne)[0] - 1.0) <= 1e-14


def test_filter_on_exact_eigenvectors():
    p = G.problem_small(60, 4, 4, complex_=True)
    A = p.dense()
    idx = np.array([0, 3, 7, 20, 45, 59])
    E = G.exact_eigvecs(p.U, idx)
    m = np.array([1, 2, 5, 9, 13, 20])
    b_sup, mu_1, mu_ne = 1.1, -0.95, -0.6
    out, mv = O.chebyshev_filter(A, E, m, b_sup, mu_1, mu_ne)
    assert mv == m.sum()
    for a in range(idx.size):
        pm = O.chebyshev_scalar(np.array([p.lam[idx[a]]]), int(m[a]), b_sup, mu_1, mu_ne)[0]
        assert np.linalg.norm(out[:, a] - pm * E[:, a]) <= 1e-12 * max(1.0, abs(pm))


def test_filter_degree_zero_columns_independent():
    # a column's result depends only on its own degree, not on the others
    p = G.problem_small(40, 4, 4, complex_=False)
    A = p.dense()
    V = p.V0[:, :4]
    m = np.array([3, 3, 8, 11])
    out, _ = O.chebyshev_filter(A, V, m, 1.2, -1.0, -0.3)
    for a in range(4):
        single, _ = O.chebyshev_filter(A, V[:, a:a + 1], m[a:a + 1], 1.2, -1.0, -0.3)
        assert np.allclose(single[:, 0], out[:, a], rtol=0, atol=1e-13)


# ---------------------------------------------------------------- Lanczos

@pytest.mark.parametrize("cplx", [False, True])
def test_lanczos_bounds_bracket_spectrum(cplx):
    p = G.problem_small(300, 10, 6, complex_=cplx, seed_pid=2)
    A = p.dense()
    lz = O.lanczos_bounds(A, p.L0, 25, p.ne)
    assert lz.b_sup >= p.lam[-1]
    assert lz.mu_1 >= p.lam[0] - 1e-12
    assert lz.mu_1 <= p.lam[0] + 0.05 * (p.lam[-1] - p.lam[0])
    assert lz.mu_1 < lz.mu_ne < lz.b_sup
    # DoS estimate of the ne-th eigenvalue lies in the lower part of the spectrum
    assert lz.mu_ne <= p.lam[0] + 0.5 * (p.lam[-1] - p.lam[0])
    # tau^2 of each run sums to one (spectral measure of a unit start vector)
    for t2 in lz.tau2:
        assert abs(np.sum(t2) - 1.0) <= 1e-12


def test_lanczos_tridiagonal_exact_on_small_matrix():
    # n steps of Lanczos on an n x n matrix reproduce its full spectrum
    p = G.problem_small(12, 2, 2, complex_=True)
    A = p.dense()
    lz = O.lanczos_bounds(A, p.L0[:, :1], 12, 4)
    assert np.max(np.abs(lz.thetas[0] - p.lam)) <= 1e-12



def _dos_quantile_from_eigh(A, starts, ne):
    """The density-of-states quantile written from a full eigendecomposition (LAPACK eigh).

    The spectral measure of a unit start vector v puts weight |q_j^H v|^2 on eigenvalue lambda_j; the
    quantile is the smallest lambda_j at which the run-averaged measure reaches ne/n.
    """
    lam, Q = np.linalg.eigh(A)
    n = A.shape[0]
    wts = np.zeros(n)
    for r in range(starts.shape[1]):
        v = starts[:, r] / np.linalg.norm(starts[:, r])
        wts += np.abs(np.conj(Q.T) @ v) ** 2 / starts.shape[1]
    cdf = np.cumsum(wts)
    j = int(np.argmax(cdf >= ne / n))
    return lam, cdf, j


@pytest.mark.parametrize("cplx", [False, True])
def test_lanczos_dos_quantile_exact_with_full_steps(cplx):
    """With n Lanczos steps each run's Ritz values are the eigenvalues of A and tau_j^2 = |q_j^H v|^2
    (Gauss quadrature of the spectral measure is then exact), so the DoS estimate of mu_ne must equal
    the quantile computed from eigh alone.  A wrong weighting (last instead of first components, no
    1/runs) or an off-by-one in the quantile picks another eigenvalue and fails."""
    n = 40
    lam_p = np.linspace(-1.0, 1.0, n) + 0.3 * np.sin(np.arange(n))  # distinct, irregular gaps
    lam_p = np.sort(lam_p)
    p = G.problem_small(n, 4, 3, complex_=cplx, lam=lam_p, seed_pid=11)
    A = p.dense()
    for ne in (3, 7, 11):
        lz = O.lanczos_bounds(A, p.L0, n, ne)
        lam, cdf, j = _dos_quantile_from_eigh(A, p.L0, ne)
        # the crossing is not at a rounding-level tie
        assert cdf[j] - ne / n > 1e-6 and (j == 0 or ne / n - cdf[j - 1] > 1e-6)
        span = lz.b_sup - lz.mu_1
        assert abs(lz.b_sup - lam[-1]) <= 1e-10 and abs(lz.mu_1 - lam[0]) <= 1e-10
        expect = min(max(lam[j], lz.mu_1 + 1e-3 * span), lz.b_sup - 1e-3 * span)
        assert abs(lz.mu_ne - expect) <= 1e-10 * span, (ne, lz.mu_ne, expect)


@pytest.mark.parametrize("cplx", [False, True])
def test_lanczos_dos_quantile_statistical(cplx):
    """With the reading's 4 runs of 25 steps the DoS estimate is a quadrature of the spectral measure, so
    the index of mu_ne in the spectrum lies within about one Ritz spacing (n/steps eigenvalues) of ne in
    every seeded case and is unbiased on average."""
    n, steps = 300, 25
    for ne in (16, 30, 60):
        idx = []
        for pid in range(8):
            p = G.problem_small(n, ne // 2, ne - ne // 2, complex_=cplx, seed_pid=pid)
            lz = O.lanczos_bounds(p.dense(), p.L0, steps, ne)
            idx.append(int(np.sum(p.lam <= lz.mu_ne)))
        assert max(abs(i - ne) for i in idx) <= n // steps, (ne, idx)
        assert abs(np.mean(idx) - ne) <= 0.15 * ne + 1, (ne, idx)


def test_chebyshev_step_rows_matches_filter():
    """The row-block step (the CPU sample the benchmark times) equals the same rows of the full filter."""
    p = G.problem_small(90, 6, 4, complex_=True, seed_pid=5)
    A = p.dense()
    V = p.V0
    b_sup, mu_1, mu_ne = 1.05, -1.0, -0.4
    c, e, al, be = O.filter_coefficients(b_sup, mu_1, mu_ne, 6)
    rows = np.arange(17, 53)
    for s in (1, 2, 5, 6):
        Ys = O.chebyshev_filter(A, V, np.full(V.shape[1], s), b_sup, mu_1, mu_ne)[0]
        Y1 = O.chebyshev_filter(A, V, np.full(V.shape[1], s - 1), b_sup, mu_1, mu_ne)[0] if s > 1 else V
        Y2 = O.chebyshev_filter(A, V, np.full(V.shape[1], s - 2), b_sup, mu_1, mu_ne)[0] if s > 2 else V
        out = O.chebyshev_step_rows(A[rows], rows, Y1, Y2[rows], s, c, al, be)
        assert np.max(np.abs(out - Ys[rows])) <= 1e-12 * max(1.0, np.max(np.abs(Ys))), s


# ---------------------------------------------------------------- Table 2 Geometric reading

def _cheb_growth(t, m):
    return np.cosh(m * np.arccosh(abs(t)))


def test_table2_geometric_positive_dmax_contradicts_paper_counts():
    """Table 2 solves the Geometric matrix (n = 20k, nev 1500, nex 500) in 8 iterations with 285192
    Matvecs.  With Table 1's formula and dmax = +1 the 2000 lowest eigenvalues fall in [1e-4, 2.5e-4]
    of a spectrum of norm 1.  A polynomial of degree m bounded by 1 on the unwanted interval
    [lambda_{ne+1}, lambda_n] is at most C_m(|t|) at lambda_nev (Chebyshev's minimax property); with
    degrees <= 36, 8 iterations apply at most degree 20 + 7 * 36 = 272, which separates lambda_nev from
    the unwanted part by a factor below 100, while a residual of 1e-10 needs about 1e9.  The degree
    formula also returns the cap for every wanted vector there, whereas the paper's Matvecs average
    17.8 per vector and iteration.  With dmax = -1 (the reading used for Table 2) the lowest
    eigenvalues are the sparse end and one degree-20 filter already separates them by more than 1e6."""
    n, nev, ne = 20000, 1500, 2000
    for lam, converges in ((G.spectrum_geometric_table1(n), False), (G.spectrum_geometric_table2(n), True)):
        a, b = lam[ne], lam[-1]                 # unwanted interval [lambda_{ne+1}, lambda_n]
        c, e = 0.5 * (a + b), 0.5 * (b - a)
        t = (lam[nev - 1] - c) / e
        assert abs(t) > 1
        if converges:
            assert _cheb_growth(t, 20) > 1e6
        else:
            assert _cheb_growth(t, 20 + 7 * 36) < 100
            rho = abs(t) + np.sqrt(t * t - 1)
            assert np.log(10.0) / np.log(rho) > 36   # one decade of residual needs more than the cap
    # both readings have the condition number the paper prints
    for lam in (G.spectrum_geometric_table1(n), G.spectrum_geometric_table2(n)):
        assert abs(np.max(np.abs(lam)) / np.min(np.abs(lam)) - 1e4) <= 1e-6 * 1e4
    assert 285192 / (ne * 8) < 18


def test_solve_table2_geometric_scaled():
    """The Table 2 Geometric type at a tenth of the size (n = 2000, nev 150, nex 50, the same
    spectral shape) converges in the oracle to the prescribed eigenvalues."""
    n, nev, nex = 2000, 150, 50
    lam = G.spectrum_geometric_table2(n)
    p = G.problem_small(n, nev, nex, complex_=False, k_reflect=8, lam=lam, seed_pid=7)
    A = p.dense()
    r = O.chase_solve(A, nev, nex, 1e-10, 20, 36, p.V0, p.L0, 25)
    assert r.converged and r.iterations <= 8
    assert np.max(np.abs(r.eigvals - lam[:nev])) <= 1e-10
    R = A @ r.eigvecs - r.eigvecs * r.eigvals[None, :]
    assert np.max(np.linalg.norm(R, axis=0)) <= 1e-10 * 1.0000001


# ---------------------------------------------------------------- residuals, degrees, locking

def test_residuals_and_lock():
    p = G.problem_small(30, 3, 3, complex_=True)
    A = p.dense()
    E = G.exact_eigvecs(p.U, [0, 1, 2])
    r = O.residuals(A, E, p.lam[:3])
    assert np.max(r) <= 1e-13
    assert O.lock_prefix(np.array([1e-12, 1e-11, 1.0, 1e-15]), 1e-10) == 2
    assert O.lock_prefix(np.array([1.0, 1e-15]), 1e-10) == 0


def test_degrees_properties():
    c, e = 10.0, 9.0        # damped interval [1, 19]
    w = np.array([-5.0, -5.0, -1.0, 0.999, 1.0])
    res = np.array([1e-2, 1e-6, 1e-2, 1e-2, 1e-2])
    m = O.degrees(res, w, 1e-10, c, e, 36)
    assert m[0] > m[1]                  # smaller residual -> lower degree
    assert m[2] >= m[0]                 # closer to the interval -> higher degree
    assert m[4] == 36                   # on the interval edge
    assert np.all((m >= 1) & (m <= 36))
    # converged residual -> minimum degree range
    assert O.degrees(np.array([1e-12]), np.array([-5.0]), 1e-10, c, e, 36)[0] <= 2
    # explicit value: rho = |t| + sqrt(t^2 - 1)
    t = (-5.0 - c) / e
    rho = abs(t) + np.sqrt(t * t - 1)
    assert m[0] == int(np.ceil(np.log(1e-2 / 1e-10) / np.log(rho))) + 2


def test_sort_by_degree_stable():
    m = np.array([5, 3, 5, 3, 7])
    w = np.array([0.1, 0.5, -0.2, 0.4, 0.0])
    order = O.sort_by_degree(m, w)
    assert list(order) == [3, 1, 2, 0, 4]


# ---------------------------------------------------------------- full solve

@pytest.mark.parametrize("cplx,n,nev,nex", [(True, 40, 4, 4), (False, 64, 6, 6), (True, 96, 8, 4)])
def test_solve_brute_force_small(cplx, n, nev, nex):
    p = G.problem_small(n, nev, nex, complex_=cplx, seed_pid=n)
    A = p.dense()
    r = O.chase_solve(A, nev, nex, 1e-10, 20, 36, p.V0, p.L0, 25)
    assert r.converged
    wl = np.linalg.eigvalsh(A)[:nev]
    nrm = np.max(np.abs(p.lam))
    assert np.max(np.abs(r.eigvals - wl)) <= 1e-10 * nrm
    res = O.residuals(A, r.eigvecs, r.eigvals)
    assert np.max(res) <= 1e-10 * nrm * 1.0000001
    assert np.max(np.abs(np.conj(r.eigvecs.T) @ r.eigvecs - np.eye(nev))) <= 1e-12


def test_solve_c1_prescribed_spectrum():
    p = G.problem_c1()
    A = p.dense()
    r = O.chase_solve(A, p.nev, p.nex, p.tol, p.deg, p.maxdeg, p.V0, p.L0, p.lanczos_steps)
    assert r.converged
    nrm = p.norm2()
    assert np.max(np.abs(r.eigvals - p.lam[:p.nev])) <= 1e-10 * nrm
    # exact residuals through the implicit operator Q diag(lam) Q^H
    R = G.implicit_matvec(p.lam, p.U, r.eigvecs) - r.eigvecs * r.eigvals[None, :]
    assert np.max(np.linalg.norm(R, axis=0)) <= 1e-10 * nrm * 1.0000001
    # subspace angle vs exact Q e_i within the Davis-Kahan bound tol*||A|| / gap
    E = G.exact_eigvecs(p.U, np.arange(p.nev))
    s = np.linalg.svd(np.conj(E.T) @ r.eigvecs, compute_uv=False)
    angle = np.sqrt(max(0.0, 1 - np.min(s) ** 2))
    gap = p.lam[p.nev] - p.lam[p.nev - 1]
    assert angle <= 2.0 * p.tol * nrm / gap
    assert r.matvecs > 0 and r.iterations >= 2


def test_solve_121_closed_form():
    n = 200
    A = G.matrix_121(n)
    p = G.from_dense("121", A, 8, 6)
    r = O.chase_solve(A, 8, 6, 1e-10, 20, 36, p.V0, p.L0, 25)
    assert r.converged
    assert np.max(np.abs(r.eigvals - G.spectrum_121(n)[:8])) <= 1e-10 * 4


def test_warm_start_from_previous_eigenvectors_needs_fewer_matvecs():
    """Correlated sequence (the premise of the batched form): after A -> A + 1e-3 H, restarting from the
    previous eigenvectors (padded with the rest of the previous search block) converges to the new
    spectrum with fewer filter products than a cold start from the random block."""
    n, nev, nex = 300, 12, 8
    p = G.problem_c4(3, n)
    p = G.from_dense("seq", p.dense(), nev, nex)
    A0 = p.dense()
    r0 = O.chase_solve(A0, nev, nex, 1e-10, 20, 36, p.V0, p.L0, 25)
    assert r0.converged
    A1 = A0 + 1e-3 * G.perturbation(n, G.sequence_seed(3, 0), True)
    # warm block: the locked eigenvectors, then the remaining random columns re-orthogonalised against them
    rest = p.V0[:, nev:] - r0.eigvecs @ (np.conj(r0.eigvecs.T) @ p.V0[:, nev:])
    V_warm = np.concatenate([r0.eigvecs, rest], axis=1)
    cold = O.chase_solve(A1, nev, nex, 1e-10, 20, 36, p.V0, p.L0, 25)
    warm = O.chase_solve(A1, nev, nex, 1e-10, 20, 36, V_warm, p.L0, 25)
    ref = np.linalg.eigvalsh(A1)[:nev]
    nrm = np.max(np.abs(np.linalg.eigvalsh(A1)))
    for r in (cold, warm):
        assert r.converged
        assert np.max(np.abs(r.eigvals - ref)) <= 1e-10 * nrm
    assert warm.matvecs < cold.matvecs


def test_planted_sign_error_in_filter_is_caught(monkeypatch):
    # a plausible mistake (wrong sign of the three-term beta) must fail the closed-form pin
    orig = O.filter_coefficients

    def wrong(b_sup, mu_1, mu_ne, mmax):
        c, e, al, be = orig(b_sup, mu_1, mu_ne, mmax)
        return c, e, al, -be

    monkeypatch.setattr(O, "filter_coefficients", wrong)
    p = G.problem_small(60, 4, 4, complex_=True)
    A = p.dense()
    E = G.exact_eigvecs(p.U, [0])
    out, _ = O.chebyshev_filter(A, E, np.array([6]), 1.1, -0.95, -0.6)
    pm = O.chebyshev_scalar(np.array([p.lam[0]]), 6, 1.1, -0.95, -0.6)[0]
    assert np.linalg.norm(out[:, 0] - pm * E[:, 0]) > 1e-6


# ---------------------------------------------------------------- backward

def _loss_parts(A, nev, w, B):
    lam, V = np.linalg.eigh(A)
    lam, V = lam[:nev], V[:, :nev]
    M = V.T @ B @ V
    L = float(w @ lam + np.sum(M * M))
    gV = 4.0 * B @ V @ M
    return L, lam, V, gV


def test_backward_dense_vs_finite_differences():
    n, nev = 30, 4
    g = np.random.default_rng(11)
    lam = G.spectrum_gapped(g, n, nlow=nev + 2, gap=5e-2)
    U = g.standard_normal((n, 4))
    A = G.dense_A(lam, U)
    w = g.standard_normal(nev)
    Bm = g.standard_normal((n, n))
    Bm = 0.5 * (Bm + Bm.T)
    L, lam_c, V, gV = _loss_parts(A, nev, w, Bm)
    Ab = O.eig_backward_dense(A, w, gV, nev)
    h = 1e-6
    for t in range(4):
        D = g.standard_normal((n, n))
        D = 0.5 * (D + D.T)
        Lp = _loss_parts(A + h * D, nev, w, Bm)[0]
        Lm = _loss_parts(A - h * D, nev, w, Bm)[0]
        fd = (Lp - Lm) / (2 * h)
        an = float(np.sum(Ab * D))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_backward_minres_matches_dense():
    n, nev = 50, 5
    g = np.random.default_rng(12)
    lam = G.spectrum_gapped(g, n, nlow=nev + 2, gap=2e-2)
    A = G.dense_A(lam, g.standard_normal((n, 3)))
    w = g.standard_normal(nev)
    Bm = g.standard_normal((n, n))
    Bm = 0.5 * (Bm + Bm.T)
    _, lam_c, V, gV = _loss_parts(A, nev, w, Bm)
    Ab_alg = O.eig_backward(A, lam_c, V, w, gV, minres_tol=1e-13)
    Ab_ref = O.eig_backward_dense(A, w, gV, nev)
    assert np.max(np.abs(Ab_alg - Ab_ref)) <= 1e-9 * np.max(np.abs(Ab_ref))


def test_backward_eigenvalue_only_is_v_diag_vt():
    n, nev = 25, 3
    g = np.random.default_rng(13)
    lam = G.spectrum_gapped(g, n, nlow=nev + 1, gap=5e-2)
    A = G.dense_A(lam, g.standard_normal((n, 3)))
    lam_c, V = np.linalg.eigh(A)
    lam_c, V = lam_c[:nev], V[:, :nev]
    w = g.standard_normal(nev)
    Ab = O.eig_backward(A, lam_c, V, w, np.zeros((n, nev)))
    assert np.max(np.abs(Ab - V @ np.diag(w) @ V.T)) <= 1e-14


def test_solve_with_lapack_small_eigensolver_matches_jacobi():
    """The Rayleigh-Ritz step accepts LAPACK's eigh as its dense solver (used by large GPU parity tests);
    it reaches the same eigenpairs, iterations and final search block span as the textbook Jacobi."""
    p = G.problem_small(120, 8, 6, complex_=True, seed_pid=17)
    A = p.dense()
    r1 = O.chase_solve(A, p.nev, p.nex, 1e-10, 20, 36, p.V0, p.L0, 25)
    r2 = O.chase_solve(A, p.nev, p.nex, 1e-10, 20, 36, p.V0, p.L0, 25, small_eigh=np.linalg.eigh)
    assert r1.converged and r2.converged
    assert np.max(np.abs(r1.eigvals - r2.eigvals)) <= 1e-12
    assert abs(r1.iterations - r2.iterations) <= 1
    assert r1.block.shape == (120, p.ne) and r2.block.shape == (120, p.ne)
    # the block starts with the eigenvectors, ascending
    assert np.allclose(r1.block[:, :p.nev], r1.eigvecs, atol=0)
