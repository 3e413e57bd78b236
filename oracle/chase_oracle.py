"""Plain FP64 CPU oracle of ChASE, the Chebyshev-accelerated subspace iteration.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The product library
never calls it and shares no code with it.

Every function follows one step of the paper's Algorithm 1 (ChASE algorithm,
Section "ChASE Algorithm") and is written for a reader checking it against the
paper: numpy FP64 arithmetic, a matmul as the only library primitive on the
solver path, no blocking or fusion.  Where the paper is silent the reading used
is stated in the docstring.

Pins (tests/test_oracle.py):
  * Jacobi eigensolver: brute force vs LAPACK eigh, closed-form (1-2-1) spectrum,
    Sturm-bisection Wilkinson spectrum, orthonormality/residual invariants.
  * Householder QR: Q^H Q = I, Q R = X, span equality with LAPACK QR.
  * Filter: exact scalar Chebyshev polynomial on eigenvectors (closed form); the
    row-block step against the same rows of the full filter.
  * Lanczos: b_sup >= lambda_max and mu_1 >= lambda_min on prescribed spectra; the
    DoS quantile mu_ne equals the quantile of the spectral measure computed from
    eigh when the runs take n steps, and lies within one Ritz spacing of lambda_ne
    with 25 steps.
  * Full solve: prescribed spectra and exact eigenvectors Q e_i; the Table 2
    Geometric type at a tenth of its size.
  * Degrees: parity unpinned (the paper gives no formula; affects only Matvecs).
  * Backward: dense full-eigendecomposition gradient and central finite differences.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# --------------------------------------------------------------------------
# Small dense Hermitian eigensolver (used by Rayleigh-Ritz and by Lanczos on T)
# --------------------------------------------------------------------------

def jacobi_eigh(G: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """Cyclic two-sided Jacobi for a Hermitian (or real symmetric) matrix.

    Rayleigh-Ritz (Algorithm 1, line 6) diagonalises G with a standard dense
    solver; the textbook cyclic Jacobi method (Golub & Van Loan, Sec. 8.5) is used
    here.  For each pair (p, q) the 2x2 block [[a, g], [conj(g), b]] is first made
    real by the phase D = diag(1, conj(g)/|g|), then zeroed by a real rotation with
    t = sign(z)/(|z| + sqrt(1 + z^2)), z = (b - a)/(2|g|).
    Returns eigenvalues ascending and the unitary Z with G Z = Z diag(w).
    """
    G = np.array(G, dtype=np.result_type(G, np.float64), copy=True)
    k = G.shape[0]
    Z = np.eye(k, dtype=G.dtype)
    cplx = np.iscomplexobj(G)
    fro = np.linalg.norm(G)
    if k == 1 or fro == 0.0:
        w = np.real(np.diag(G)).copy()
        order = np.argsort(w, kind="stable")
        return w[order], Z[:, order]
    for _ in range(max_sweeps):
        off = np.linalg.norm(G - np.diag(np.diag(G)))
        if off <= tol * fro:
            break
        for p in range(k - 1):
            for q in range(p + 1, k):
                g = G[p, q]
                ag = abs(g)
                if ag == 0.0:
                    continue
                a = G[p, p].real
                b = G[q, q].real
                z = (b - a) / (2.0 * ag)
                t = (1.0 if z >= 0 else -1.0) / (abs(z) + np.sqrt(1.0 + z * z))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                ph = np.conj(g) / ag if cplx else (1.0 if g > 0 else -1.0)
                # J = D R restricted to columns (p, q):
                #   J = [[c, s], [-s*ph, c*ph]],  D = diag(1, ph)
                Jpp, Jpq, Jqp, Jqq = c, s, -s * ph, c * ph
                cp = G[:, p].copy()
                cq = G[:, q].copy()
                G[:, p] = cp * Jpp + cq * Jqp
                G[:, q] = cp * Jpq + cq * Jqq
                rp = G[p, :].copy()
                rq = G[q, :].copy()
                G[p, :] = np.conj(Jpp) * rp + np.conj(Jqp) * rq
                G[q, :] = np.conj(Jpq) * rp + np.conj(Jqq) * rq
                G[p, q] = 0.0
                G[q, p] = 0.0
                G[p, p] = G[p, p].real
                G[q, q] = G[q, q].real
                zp = Z[:, p].copy()
                zq = Z[:, q].copy()
                Z[:, p] = zp * Jpp + zq * Jqp
                Z[:, q] = zp * Jpq + zq * Jqq
    w = np.real(np.diag(G)).copy()
    order = np.argsort(w, kind="stable")
    return w[order], Z[:, order]


def sturm_count(d: np.ndarray, e: np.ndarray, x: float) -> int:
    """Number of eigenvalues < x of the symmetric tridiagonal (d, e) (Sturm sequence)."""
    cnt = 0
    q = 1.0
    for i in range(d.size):
        off = e[i - 1] ** 2 if i else 0.0
        q = d[i] - x - (off / q if i else 0.0)
        if q == 0.0:
            q = -1e-300
        if q < 0:
            cnt += 1
    return cnt


def tridiag_bisection(d: np.ndarray, e: np.ndarray) -> np.ndarray:
    """All eigenvalues of a symmetric tridiagonal by bisection on Sturm counts (textbook)."""
    n = d.size
    r = np.max(np.abs(d)) + 2.0 * (np.max(np.abs(e)) if e.size else 0.0)
    out = np.empty(n)
    for j in range(n):
        lo, hi = -r - 1.0, r + 1.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if mid == lo or mid == hi:
                break
            if sturm_count(d, e, mid) > j:
                hi = mid
            else:
                lo = mid
        out[j] = 0.5 * (lo + hi)
    return out


# --------------------------------------------------------------------------
# Algorithm 1, line 2: Lanczos spectral bounds
# --------------------------------------------------------------------------

@dataclass
class LanczosResult:
    b_sup: float
    mu_1: float
    mu_ne: float
    theta_max: float = -np.inf
    thetas: list = field(default_factory=list)
    tau2: list = field(default_factory=list)
    beta_last: list = field(default_factory=list)


def lanczos_bounds(A: np.ndarray, starts: np.ndarray, steps: int, ne: int) -> LanczosResult:
    """Spectral bounds from repeated Lanczos runs (Algorithm 1, line 2).

    The paper runs "a small number of repeated Lanczos steps" and estimates the
    density of states (DoS).  Reading used here: one run of ``steps`` Lanczos steps
    with full reorthogonalisation from each column of ``starts``; for the
    tridiagonal T of a run, Ritz values theta_j and squared first components
    tau_j^2 of its eigenvectors.
      b_sup  = max over runs of (theta_max + |beta_last|)
      mu_1   = min over runs of theta_min
      theta_max = max over runs of theta_max (used for the residual normalisation)
      mu_ne  = smallest pooled theta with (1/runs) sum_{theta_j <= t} tau_j^2 >= ne/n
               (DoS quantile of the spectral measure), clamped to (mu_1, b_sup).
    """
    n = A.shape[0]
    res = LanczosResult(-np.inf, np.inf, 0.0)
    pooled = []
    nruns = starts.shape[1]
    for r in range(nruns):
        v = starts[:, r] / np.linalg.norm(starts[:, r])
        basis = [v]
        alpha, beta = [], []
        for j in range(steps):
            w = A @ basis[j]
            a = float(np.real(np.vdot(basis[j], w)))
            alpha.append(a)
            w = w - a * basis[j]
            if j > 0:
                w = w - beta[j - 1] * basis[j - 1]
            Vm = np.stack(basis, axis=1)
            w = w - Vm @ (np.conj(Vm.T) @ w)       # full reorthogonalisation (once)
            b = float(np.linalg.norm(w))
            beta.append(b)
            if j + 1 < steps:
                basis.append(w / b)
        T = np.diag(alpha)
        if steps > 1:
            T += np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
        theta, S = jacobi_eigh(T)
        tau2 = np.abs(S[0, :]) ** 2
        res.thetas.append(theta)
        res.tau2.append(tau2)
        res.beta_last.append(beta[-1])
        res.b_sup = max(res.b_sup, theta[-1] + abs(beta[-1]))
        res.theta_max = max(res.theta_max, theta[-1])
        res.mu_1 = min(res.mu_1, theta[0])
        pooled.extend(zip(theta, tau2 / nruns))
    pooled.sort(key=lambda x: x[0])
    target = ne / n
    acc = 0.0
    mu_ne = pooled[-1][0]
    for th, wgt in pooled:
        acc += wgt
        if acc >= target:
            mu_ne = th
            break
    span = res.b_sup - res.mu_1
    lo = res.mu_1 + 1e-3 * span
    hi = res.b_sup - 1e-3 * span
    res.mu_ne = min(max(mu_ne, lo), hi)
    return res


# --------------------------------------------------------------------------
# Algorithm 1, line 4: Chebyshev filter (three-term recurrence)
# --------------------------------------------------------------------------

def filter_coefficients(b_sup: float, mu_1: float, mu_ne: float, mmax: int):
    """Scalars of the scaled three-term recurrence (Eq. three-terms-recurrence).

    The paper leaves alpha_i, beta_i, gamma_i unspecified.  Reading: the scaled
    Chebyshev filter of Zhou et al. with gamma_i = c for all i,
      c = (b_sup + mu_ne)/2, e = (b_sup - mu_ne)/2, sigma_1 = e/(mu_1 - c),
      Y_1     = (sigma_1/e) (A - cI) Y_0,
      Y_{s+1} = (2 sigma_{s+1}/e) (A - cI) Y_s - sigma_s sigma_{s+1} Y_{s-1},
      sigma_{s+1} = 1/(2/sigma_1 - sigma_s).
    Returns (c, e, alpha[1..mmax], beta[1..mmax]) with Y_s = alpha_s (A - cI) Y_{s-1}
    + beta_s Y_{s-2} (beta_1 = 0).
    """
    c = 0.5 * (b_sup + mu_ne)
    e = 0.5 * (b_sup - mu_ne)
    sigma1 = e / (mu_1 - c)
    alpha = np.zeros(mmax + 1)
    beta = np.zeros(mmax + 1)
    sigma = sigma1
    if mmax >= 1:
        alpha[1] = sigma1 / e
    for s in range(1, mmax):
        sigma_new = 1.0 / (2.0 / sigma1 - sigma)
        alpha[s + 1] = 2.0 * sigma_new / e
        beta[s + 1] = -sigma * sigma_new
        sigma = sigma_new
    return c, e, alpha, beta


def chebyshev_filter(A: np.ndarray, V: np.ndarray, m: np.ndarray, b_sup: float, mu_1: float, mu_ne: float):
    """Filter each column a of V with its own degree m[a] (Algorithm 1, line 4).

    Column a takes exactly m[a] matrix products; Matvecs = sum(m).  At step s only
    the columns with m[a] >= s are advanced.
    """
    m = np.asarray(m, dtype=np.int64)
    mmax = int(m.max()) if m.size else 0
    c, e, alpha, beta = filter_coefficients(b_sup, mu_1, mu_ne, mmax)
    Yprev = np.array(V, copy=True)
    Y = np.array(V, copy=True)
    out = np.array(V, copy=True)
    for s in range(1, mmax + 1):
        act = m >= s
        Ynew = alpha[s] * (A @ Y[:, act] - c * Y[:, act])
        if s > 1:
            Ynew += beta[s] * Yprev[:, act]
        Yprev[:, act] = Y[:, act]
        Y[:, act] = Ynew
        done = m == s
        out[:, done] = Y[:, done]
    return out, int(m.sum())


def chebyshev_step_rows(A_rows: np.ndarray, rows: np.ndarray, Y: np.ndarray, Y_prev_rows: np.ndarray, s: int,
                        c: float, alpha: np.ndarray, beta: np.ndarray) -> np.ndarray:
    """Step s of the three-term recurrence restricted to a block of rows of A (Eq. three-terms-recurrence).

    Returns rows `rows` of Y_s = alpha_s (A - cI) Y_{s-1} + beta_s Y_{s-2}, given those rows of A
    (A_rows), the full Y_{s-1} (Y) and the same rows of Y_{s-2}.  Used to time a bounded sample of
    the filter on the CPU.
    """
    out = alpha[s] * (A_rows @ Y - c * Y[rows, :])
    if s > 1:
        out += beta[s] * Y_prev_rows
    return out


def chebyshev_scalar(x, m: int, b_sup: float, mu_1: float, mu_ne: float):
    """p_m(x) = C_m((x - c)/e) / C_m((mu_1 - c)/e), the scalar the filter applies to an eigenvalue x."""
    c = 0.5 * (b_sup + mu_ne)
    e = 0.5 * (b_sup - mu_ne)

    def cheb(t):
        t = np.asarray(t, dtype=np.float64)
        out = np.empty_like(t)
        inside = np.abs(t) <= 1
        out[inside] = np.cos(m * np.arccos(t[inside]))
        ti = t[~inside]
        out[~inside] = np.sign(ti) ** m * np.cosh(m * np.arccosh(np.abs(ti)))
        return out

    return cheb((np.asarray(x) - c) / e) / cheb(np.array([(mu_1 - c) / e]))[0]


# --------------------------------------------------------------------------
# Algorithm 1, line 5: QR
# --------------------------------------------------------------------------

def householder_qr(X: np.ndarray):
    """Thin Householder QR, X = Q R with Q n x k orthonormal (the paper's geqrf class)."""
    R = np.array(X, dtype=np.result_type(X, np.float64), copy=True)
    n, k = R.shape
    vs = []
    for j in range(k):
        x = R[j:, j]
        nx = np.linalg.norm(x)
        x0 = x[0]
        ph = x0 / abs(x0) if abs(x0) > 0 else 1.0
        alpha = -ph * nx
        v = x.copy()
        v[0] -= alpha
        nv = np.linalg.norm(v)
        if nv > 0:
            v /= nv
            R[j:, j:] -= 2.0 * np.outer(v, np.conj(v) @ R[j:, j:])
        vs.append(v)
    Q = np.zeros((n, k), dtype=R.dtype)
    Q[np.arange(k), np.arange(k)] = 1.0
    for j in range(k - 1, -1, -1):
        v = vs[j]
        Q[j:, :] -= 2.0 * np.outer(v, np.conj(v) @ Q[j:, :])
    return Q, np.triu(R[:k, :])


def qr_step(Yhat: np.ndarray, Vhat: np.ndarray) -> np.ndarray:
    """Q <- QR([Yhat Vhat]) (Algorithm 1, line 5), then restore the locked columns.

    Reading: the first l columns of Q differ from the orthonormal Yhat only by unit
    phases, so they are overwritten by Yhat; the remaining columns span the
    filtered block's complement of span(Yhat).
    """
    X = np.concatenate([Yhat, Vhat], axis=1)
    Q, _ = householder_qr(X)
    l = Yhat.shape[1]
    Q[:, :l] = Yhat
    return Q


# --------------------------------------------------------------------------
# Algorithm 1, lines 6-7: Rayleigh-Ritz and residuals
# --------------------------------------------------------------------------

def rayleigh_ritz(A: np.ndarray, Qk: np.ndarray, small_eigh=None):
    """G = Qk^H A Qk, G = Z diag(w) Z^H (ascending), Vhat = Qk Z (Algorithm 1, line 6).

    Reading: the projection is over the k active columns (the paper's
    "nev x nev" is read as the active-block size).  The small problem goes to a
    standard dense solver, as the paper does (e.g. Divide & Conquer): the textbook
    Jacobi above by default, or LAPACK's eigh passed as ``small_eigh`` (both
    pinned against each other) where k is large enough to make Jacobi in Python slow.
    """
    W = A @ Qk
    G = np.conj(Qk.T) @ W
    G = 0.5 * (G + np.conj(G.T))
    w, Z = (small_eigh or jacobi_eigh)(G)
    return w, Qk @ Z


def residuals(A: np.ndarray, V: np.ndarray, w: np.ndarray) -> np.ndarray:
    """||A v_a - w_a v_a||_2 per column, with an explicit HEMM (Algorithm 1, line 7)."""
    R = A @ V - V * w[None, :]
    return np.linalg.norm(R, axis=0)


# --------------------------------------------------------------------------
# Algorithm 1, lines 8-14: locking, bounds, degrees, sort
# --------------------------------------------------------------------------

def lock_prefix(res: np.ndarray, thresh: float) -> int:
    """Number of leading (ascending Ritz value) columns with residual <= thresh.

    Reading (the paper does not say which converged pairs are locked): the longest
    converged prefix; an unconverged lower pair blocks locking above it.
    """
    p = 0
    while p < res.size and res[p] <= thresh:
        p += 1
    return p


def degrees(res: np.ndarray, w: np.ndarray, thresh: float, c: float, e: float, maxdeg: int) -> np.ndarray:
    """Per-vector filter degree (Algorithm 1, line 12; formula not given in the paper).

    Reading: with t = (w - c)/e and rho = |t| + sqrt(t^2 - 1) the Chebyshev growth
    factor, m = ceil(ln(res/thresh) / ln(rho)) + 2, clamped to [1, maxdeg];
    |t| <= 1 or rho <= 1 + 1e-12 gives maxdeg.  Parity unpinned.
    """
    out = np.empty(res.size, dtype=np.int64)
    for a in range(res.size):
        t = (w[a] - c) / e
        if abs(t) <= 1.0:
            out[a] = maxdeg
            continue
        rho = abs(t) + np.sqrt(t * t - 1.0)
        if rho <= 1.0 + 1e-12:
            out[a] = maxdeg
            continue
        ratio = res[a] / thresh
        mm = int(np.ceil(np.log(ratio) / np.log(rho))) + 2 if ratio > 0 else 1
        out[a] = min(max(mm, 1), maxdeg)
    return out


def sort_by_degree(m: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Stable order by degree, ties by Ritz value (Algorithm 1, line 14)."""
    return np.lexsort((w, m))


# --------------------------------------------------------------------------
# Algorithm 1: the whole iteration
# --------------------------------------------------------------------------

@dataclass
class SolveResult:
    eigvals: np.ndarray
    eigvecs: np.ndarray
    iterations: int
    matvecs: int
    converged: bool
    lanczos: LanczosResult
    history: list = field(default_factory=list)
    block: np.ndarray | None = None   # final search block: locked pairs ascending, then the active rest


def chase_solve(A: np.ndarray, nev: int, nex: int, tol: float, deg: int, maxdeg: int,
                V0: np.ndarray, lanczos_starts: np.ndarray, lanczos_steps: int = 25,
                maxiter: int = 30, small_eigh=None) -> SolveResult:
    """Algorithm 1 (ChASE) on a dense Hermitian A, start block V0 (n x (nev+nex)).

    Convergence test: residual <= tol * ||A||_est with ||A||_est = max(|mu_1|, |theta_max|)
    from the Lanczos step, theta_max the largest Ritz value of all runs (the paper gives no
    normalisation; both are Ritz values, so ||A||_est <= ||A||_2 and the test is conservative).
    Bounds update: mu_1 = min of all Ritz values (locked and active), mu_ne = max of
    the active Ritz values (the paper's max([Lambda Lambda-hat]) read as the active
    maximum); b_sup stays at its Lanczos value.
    """
    n = A.shape[0]
    ne = nev + nex
    lz = lanczos_bounds(A, lanczos_starts, lanczos_steps, ne)
    b_sup, mu_1, mu_ne = lz.b_sup, lz.mu_1, lz.mu_ne
    norm_est = max(abs(mu_1), abs(lz.theta_max))
    thresh = tol * norm_est
    Vhat = np.array(V0, dtype=np.result_type(A, V0, np.float64), copy=True)
    Yhat = np.zeros((n, 0), dtype=Vhat.dtype)
    Lam = np.zeros(0)
    m = np.full(ne, deg, dtype=np.int64)
    matvecs = 0
    it = 0
    hist = []
    while Yhat.shape[1] < nev and it < maxiter:
        it += 1
        Vf, mv = chebyshev_filter(A, Vhat, m, b_sup, mu_1, mu_ne)
        matvecs += mv
        Q = qr_step(Yhat, Vf)
        l = Yhat.shape[1]
        w, Vr = rayleigh_ritz(A, Q[:, l:], small_eigh)
        res = residuals(A, Vr, w)
        p = lock_prefix(res, thresh)
        Yhat = np.concatenate([Yhat, Vr[:, :p]], axis=1)
        Lam = np.concatenate([Lam, w[:p]])
        Vr, w, res = Vr[:, p:], w[p:], res[p:]
        mu_1 = float(min(np.min(Lam) if Lam.size else np.inf, np.min(w) if w.size else np.inf))
        if w.size:
            mu_ne = float(np.max(w))
        c = 0.5 * (b_sup + mu_ne)
        e = 0.5 * (b_sup - mu_ne)
        m = degrees(res, w, thresh, c, e, maxdeg)
        order = sort_by_degree(m, w)
        Vhat, w, res, m = Vr[:, order], w[order], res[order], m[order]
        hist.append(dict(iter=it, locked=Yhat.shape[1], matvecs=mv, mu_1=mu_1, mu_ne=mu_ne,
                         max_res=float(res.max()) if res.size else 0.0))
        if w.size == 0:
            break
    order = np.argsort(Lam, kind="stable")
    # the search block a correlated next problem restarts from (warm start): locked pairs ascending,
    # then the remaining active vectors
    block = np.concatenate([Yhat[:, order], Vhat], axis=1)
    order = order[:nev]
    return SolveResult(Lam[order], Yhat[:, order], it, matvecs, Yhat.shape[1] >= nev, lz, hist, block)


# --------------------------------------------------------------------------
# Adjoint (backward) of the partial eigendecomposition, real symmetric
# --------------------------------------------------------------------------

def eig_backward_dense(A: np.ndarray, gbar_lam: np.ndarray, gbar_V: np.ndarray, nev: int):
    """Reference gradient from the full eigendecomposition (closed form).

    With all n eigenpairs (lam, V_all) and gbar padded by zeros beyond nev:
      Abar = V_all (diag(gbar_lam) + F o (V_all^T Vbar_all)) V_all^T,
      F_ij = 1/(lam_j - lam_i) for i != j, 0 on the diagonal; then symmetrised.
    The full eigendecomposition uses LAPACK eigh as a library routine.
    """
    lam, Vall = np.linalg.eigh(A)
    n = A.shape[0]
    gl = np.zeros(n)
    gl[:nev] = gbar_lam
    Vb = np.zeros_like(Vall)
    Vb[:, :nev] = gbar_V
    # fix eigenvector signs to match the caller's convention is unnecessary: the
    # gradient is invariant under v_i -> -v_i together with vbar_i -> -vbar_i, and
    # gbar_V is given for the caller's vectors, so align signs first.
    return _dense_grad(lam, Vall, gl, Vb)


def _dense_grad(lam, Vall, gl, Vb):
    d = lam[None, :] - lam[:, None]
    with np.errstate(divide="ignore"):
        F = np.where(d != 0, 1.0 / np.where(d != 0, d, 1.0), 0.0)
    np.fill_diagonal(F, 0.0)
    inner = np.diag(gl) + F * (Vall.T @ Vb)
    Ab = Vall @ inner @ Vall.T
    return 0.5 * (Ab + Ab.T)


def eig_backward(A: np.ndarray, lam: np.ndarray, V: np.ndarray, gbar_lam: np.ndarray, gbar_V: np.ndarray,
                 minres_tol: float = 1e-12, maxit: int = 5000):
    """Adjoint of (lam, V) = lowest-nev eigenpairs of symmetric A.

    Abar = V (diag(gbar_lam) + F o (V^T Vbar)) V^T + X V^T, symmetrised, where
    F_ij = 1/(lam_j - lam_i) (i != j) and column x_j of X solves
    (A - lam_j I) x_j = -P vbar_j on range(P), P = I - V V^T (the eigenvectors
    outside the computed set), by MINRES on the projected operator.
    """
    nev = lam.size
    d = lam[None, :] - lam[:, None]
    F = np.zeros_like(d)
    off = ~np.eye(nev, dtype=bool)
    F[off] = 1.0 / d[off]
    inner = np.diag(gbar_lam) + F * (V.T @ gbar_V)
    Ab = V @ inner @ V.T
    X = np.zeros_like(V)
    for j in range(nev):
        rhs = -(gbar_V[:, j] - V @ (V.T @ gbar_V[:, j]))
        X[:, j] = minres_projected(A, V, lam[j], rhs, minres_tol, maxit)
    Ab = Ab + X @ V.T
    return 0.5 * (Ab + Ab.T)


def minres_projected(A, V, shift, b, tol=1e-12, maxit=5000):
    """MINRES (Paige & Saunders, 1975) for P (A - shift I) P x = b with b in range(P), P = I - V V^T.

    Lanczos on the projected operator, QR of the tridiagonal by Givens rotations,
    and the x update through the direction vectors w; phibar is the residual norm.
    """
    def op(x):
        y = A @ x - shift * x
        return y - V @ (V.T @ y)

    n = b.size
    x = np.zeros(n)
    beta1 = float(np.linalg.norm(b))
    if beta1 == 0.0:
        return x
    r1 = b.copy()
    r2 = b.copy()
    y = b.copy()
    beta = beta1
    oldb = 0.0
    dbar = 0.0
    epsln = 0.0
    phibar = beta1
    cs, sn = -1.0, 0.0
    w = np.zeros(n)
    w2 = np.zeros(n)
    for itn in range(1, maxit + 1):
        v = y / beta
        y = op(v)
        if itn >= 2:
            y = y - (beta / oldb) * r1
        alfa = float(v @ y)
        y = y - (alfa / beta) * r2
        r1, r2 = r2, y
        oldb = beta
        beta = float(np.linalg.norm(y))
        oldeps = epsln
        delta = cs * dbar + sn * alfa
        gbar = sn * dbar - cs * alfa
        epsln = sn * beta
        dbar = -cs * beta
        gamma = max(np.hypot(gbar, beta), np.finfo(float).tiny)
        cs = gbar / gamma
        sn = beta / gamma
        phi = cs * phibar
        phibar = sn * phibar
        w1, w2 = w2, w
        w = (v - oldeps * w1 - delta * w2) / gamma
        x = x + phi * w
        if phibar <= tol * beta1 or beta == 0.0:
            break
    return x
