"""Seeded synthetic inputs for the Chebyshev-filtered subspace iteration.

This module builds inputs only: prescribed spectra, Householder reflector
vectors, the dense matrix ``A = Q diag(lam) Q^H`` they define, start blocks and
Lanczos start vectors.  It contains none of the eigensolver's arithmetic, so the
CPU oracle and the CUDA path can both draw their inputs from here without
sharing any solver code.

Test-matrix families follow the paper's test suite (Section "Test matrix
suite", Table 1): Uniform, Geometric, (1-2-1) and Wilkinson, plus dense
prescribed-spectrum matrices ``A = Q D Q^H``.  The paper builds Q from a QR of
a Gaussian matrix; here Q is a product of k dense Householder reflectors, which
keeps the exact eigenvectors ``Q e_i`` and an O(k n) implicit matvec available
at any n.

Random numbers come from numpy's PCG64 with the seed
``2205024910 + config_id * 1000 + problem_id`` and a per-purpose stream index,
so every input is reproducible on any machine.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2205024910

# stream indices: one independent PCG64 stream per purpose
_S_LAMBDA, _S_REFLECT, _S_V0, _S_LANCZOS, _S_SIZES, _S_PERTURB, _S_LOSS = range(7)


def rng(config_id: int, problem_id: int = 0, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([SEED_BASE + config_id * 1000 + problem_id, stream]))


def gaussian(g: np.random.Generator, shape, complex_: bool) -> np.ndarray:
    """Standard (complex) Gaussian: complex entries have re, im ~ N(0, 1/2)."""
    if complex_:
        s = np.sqrt(0.5)
        return (g.standard_normal(shape) * s + 1j * (g.standard_normal(shape) * s)).astype(np.complex128)
    return g.standard_normal(shape).astype(np.float64)


# --------------------------------------------------------------------------
# Spectra (Table 1 and the prescribed-spectrum workloads)
# --------------------------------------------------------------------------

def spectrum_uniform_table1(n: int, dmax: float = 1.0, eps: float = 1e-4) -> np.ndarray:
    """Table 1, Uniform: lambda_k = dmax (eps + (k-1)(1-eps)/(n-1)), k = 1..n."""
    k = np.arange(1, n + 1, dtype=np.float64)
    return dmax * (eps + (k - 1) * (1 - eps) / (n - 1))


def spectrum_geometric_table1(n: int, dmax: float = 1.0, eps: float = 1e-4) -> np.ndarray:
    """Table 1, Geometric: lambda_k = dmax eps^((n-k)/(n-1)), k = 1..n."""
    k = np.arange(1, n + 1, dtype=np.float64)
    return dmax * eps ** ((n - k) / (n - 1))


def spectrum_geometric_table2(n: int, eps: float = 1e-4) -> np.ndarray:
    """Geometric matrix of the eigen-type suite (Table 2), ascending: Table 1's formula with dmax = -1.

    The eigenvalues lie in [-1, -eps] (condition number 1/eps = 1e4, as the paper prints) and follow a
    geometric law, clustered toward zero and sparse at the lower end the solver computes.  With dmax = +1
    the lowest eigenvalues are the clustered ones; the filter bound that rules that reading out is checked
    in the tests.
    """
    return np.sort(spectrum_geometric_table1(n, dmax=-1.0, eps=eps))


def spectrum_121(n: int) -> np.ndarray:
    """Table 1, (1-2-1): lambda_k = 2 - 2 cos(pi k / (n+1)), ascending."""
    k = np.arange(1, n + 1, dtype=np.float64)
    return 2.0 - 2.0 * np.cos(np.pi * k / (n + 1))


def matrix_121(n: int) -> np.ndarray:
    """(1-2-1) tridiagonal: diagonal 2, first sub- and super-diagonal 1."""
    return np.diag(np.full(n, 2.0)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)


def matrix_wilkinson(n: int) -> np.ndarray:
    """Wilkinson tridiagonal: off-diagonals 1, diagonal |i - m| for i = 0..n-1, m = (n-1)/2.

    For odd n this is the classical W+ (diagonal m, ..., 1, 0, 1, ..., m).  For even n,
    m = (n-1)/2 is a half-integer and the diagonal runs m, ..., 1/2, 1/2, ..., m; this
    reading reproduces the condition number 4.7e4 the paper reports at n = 20k.
    """
    m = 0.5 * (n - 1)
    d = np.abs(np.arange(n, dtype=np.float64) - m)
    return np.diag(d) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)


def wilkinson_diagonal(n: int) -> np.ndarray:
    return np.abs(np.arange(n, dtype=np.float64) - 0.5 * (n - 1))


def spectrum_sorted_uniform(g, n, lo, hi) -> np.ndarray:
    return np.sort(g.uniform(lo, hi, size=n))


# --------------------------------------------------------------------------
# Householder-product Q and A = Q diag(lam) Q^H
# --------------------------------------------------------------------------

def _tau(U: np.ndarray) -> np.ndarray:
    return 2.0 / np.real(np.sum(np.conj(U) * U, axis=0))


def apply_Q(U: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Q X with Q = H_1 H_2 ... H_k, H_j = I - tau_j u_j u_j^H (applied H_k first)."""
    X = np.array(X, dtype=np.result_type(U, X, np.float64), copy=True)
    tau = _tau(U)
    for j in range(U.shape[1] - 1, -1, -1):
        u = U[:, j]
        X -= tau[j] * np.outer(u, np.conj(u) @ X) if X.ndim == 2 else tau[j] * u * (np.conj(u) @ X)
    return X


def apply_QH(U: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Q^H X = H_k ... H_1 X (applied H_1 first)."""
    X = np.array(X, dtype=np.result_type(U, X, np.float64), copy=True)
    tau = _tau(U)
    for j in range(U.shape[1]):
        u = U[:, j]
        X -= tau[j] * np.outer(u, np.conj(u) @ X) if X.ndim == 2 else tau[j] * u * (np.conj(u) @ X)
    return X


def dense_A(lam: np.ndarray, U: np.ndarray) -> np.ndarray:
    """Dense A = Q diag(lam) Q^H by two-sided reflector application, made exactly Hermitian."""
    M = np.diag(lam.astype(np.result_type(U, np.float64)))
    tau = _tau(U)
    for j in range(U.shape[1] - 1, -1, -1):
        u = U[:, j]
        # M <- H_j M H_j
        M -= tau[j] * np.outer(u, np.conj(u) @ M)
        M -= tau[j] * np.outer(M @ u, np.conj(u))
    return 0.5 * (M + np.conj(M.T))


def implicit_matvec(lam: np.ndarray, U: np.ndarray, X: np.ndarray) -> np.ndarray:
    """A X = Q diag(lam) Q^H X in O(k n) per column, without forming A."""
    Y = apply_QH(U, X)
    Y = (lam[:, None] * Y) if Y.ndim == 2 else lam * Y
    return apply_Q(U, Y)


def exact_eigvecs(U: np.ndarray, idx) -> np.ndarray:
    """Columns Q e_i for the given indices (eigenvectors of A for lam[idx])."""
    n = U.shape[0]
    idx = np.atleast_1d(np.asarray(idx))
    E = np.zeros((n, idx.size), dtype=np.result_type(U, np.float64))
    E[idx, np.arange(idx.size)] = 1.0
    return apply_Q(U, E)


def wy_factors(lam: np.ndarray, U: np.ndarray):
    """Low-rank factors of A = Q diag(lam) Q^H for an elementwise device generator.

    Q = I - U T U^H (compact WY form of H_1...H_k), B = U T, C = U^H diag(lam) U,
    D = B C.  Then
        A_ij = lam_i d_ij - lam_j sum_a B_ia conj(U_ja) - lam_i sum_a U_ia conj(B_ja)
               + sum_a D_ia conj(B_ja).
    """
    n, k = U.shape
    tau = _tau(U)
    T = np.zeros((k, k), dtype=np.result_type(U, np.float64))
    for j in range(k):
        T[j, j] = tau[j]
        if j:
            T[:j, j] = -tau[j] * (T[:j, :j] @ (np.conj(U[:, :j].T) @ U[:, j]))
    B = U @ T
    C = np.conj(U.T) @ (lam[:, None] * U)
    D = B @ C
    return B, D


# --------------------------------------------------------------------------
# Problems
# --------------------------------------------------------------------------

@dataclass
class Problem:
    name: str
    n: int
    nev: int
    nex: int
    tol: float
    deg: int
    maxdeg: int
    complex_: bool
    lam: np.ndarray            # prescribed spectrum, ascending
    U: np.ndarray              # reflector vectors (n x k)
    V0: np.ndarray             # start block (n x ne)
    L0: np.ndarray             # Lanczos start vectors (n x nruns)
    lanczos_steps: int = 25
    extra: dict = field(default_factory=dict)

    @property
    def ne(self) -> int:
        return self.nev + self.nex

    def dense(self) -> np.ndarray:
        if "A" in self.extra:
            return self.extra["A"]
        return dense_A(self.lam, self.U)

    def norm2(self) -> float:
        return float(np.max(np.abs(self.lam)))


def _make(name, cfg, pid, n, nev, nex, lam, k_reflect, complex_, tol=1e-10, deg=20, maxdeg=36,
          nruns=4, lanczos_steps=25, extra=None) -> Problem:
    U = gaussian(rng(cfg, pid, _S_REFLECT), (n, k_reflect), complex_)
    V0 = gaussian(rng(cfg, pid, _S_V0), (n, nev + nex), complex_)
    L0 = gaussian(rng(cfg, pid, _S_LANCZOS), (n, nruns), complex_)
    return Problem(name, n, nev, nex, tol, deg, maxdeg, complex_, np.asarray(lam, np.float64), U, V0, L0,
                   lanczos_steps, extra or {})


def problem_c1(n: int = 512, nev: int = 16, nex: int = 8) -> Problem:
    """Complex Hermitian, 8 reflectors, lam sorted i.i.d. U[-1,1]; nev 16, nex 8, deg 20..36."""
    lam = spectrum_sorted_uniform(rng(1, 0, _S_LAMBDA), n, -1.0, 1.0)
    return _make("c1", 1, 0, n, nev, nex, lam, 8, True)


def spectrum_c2(n: int = 30000, n_low: int = 2000) -> np.ndarray:
    g = rng(2, 0, _S_LAMBDA)
    low = spectrum_sorted_uniform(g, n_low, -2.0, 0.0)
    high = spectrum_sorted_uniform(g, n - n_low, 0.0, 50.0)
    return np.concatenate([low, high])


def problem_c2(n: int = 30000, nev: int = 1200, nex: int = 400, n_low: int = 2000) -> Problem:
    """Complex Hermitian, 16 reflectors; lowest n_low i.i.d. U[-2,0], rest U[0,50]."""
    return _make("c2", 2, 0, n, nev, nex, spectrum_c2(n, n_low), 16, True)


def spectrum_c3(n: int = 60000, n_low: int = 3000) -> np.ndarray:
    g = rng(3, 0, _S_LAMBDA)
    low = spectrum_sorted_uniform(g, n_low, -2.0, 0.0)
    N = n - n_low
    j = np.arange(1, N + 1, dtype=np.float64)
    high = 0.01 * (1e4) ** ((j - 1) / (N - 1))
    return np.concatenate([low, high])


def problem_c3(n: int = 60000, nev: int = 2000, nex: int = 500, n_low: int = 3000) -> Problem:
    """Complex Hermitian, 16 reflectors; lowest n_low U[-2,0], rest geometric on [0.01, 100]."""
    return _make("c3", 3, 0, n, nev, nex, spectrum_c3(n, n_low), 16, True)


def batched_sizes(nprob: int = 64, lo: int = 512, hi: int = 8192) -> np.ndarray:
    return rng(4, 0, _S_SIZES).integers(lo, hi + 1, size=nprob)


def problem_c4(pid: int, n: int | None = None) -> Problem:
    """One problem of the batched set: lam U[-1,1], 8 reflectors, nev = round(0.05 n), nex = nev // 2."""
    if n is None:
        n = int(batched_sizes()[pid])
    nev = max(1, int(round(0.05 * n)))
    nex = max(1, nev // 2)
    lam = spectrum_sorted_uniform(rng(4, pid + 1, _S_LAMBDA), n, -1.0, 1.0)
    return _make(f"c4.{pid}", 4, pid + 1, n, nev, nex, lam, 8, True)


_M64 = (1 << 64) - 1


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea & Flood 2014) on uint64 arrays (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)).astype(np.uint64)
        return z ^ (z >> np.uint64(31))


def counter_normal_pairs(seed: int, ctr: np.ndarray):
    """Counter-based standard normal pairs: SplitMix64 hash of (seed, 2c) and (seed, 2c+1), Box-Muller."""
    s = np.uint64(seed & _M64)
    c = ctr.astype(np.uint64)
    a = _splitmix64(s ^ _splitmix64(np.uint64(2) * c))
    b = _splitmix64(s ^ _splitmix64(np.uint64(2) * c + np.uint64(1)))
    u1 = ((a >> np.uint64(11)).astype(np.float64) + 1.0) * 1.1102230246251565e-16
    u2 = (b >> np.uint64(11)).astype(np.float64) * 1.1102230246251565e-16
    r = np.sqrt(-2.0 * np.log(u1))
    t = 6.283185307179586 * u2
    return r * np.cos(t), r * np.sin(t)


def perturbation(n: int, seed: int, complex_: bool = True) -> np.ndarray:
    """H = s (G + G^H)/2 with G_ij from counter_normal_pairs(seed, i + j n), s = 1/sqrt(2n).

    Complex: G_ij = (x + i y)/sqrt(2); real: G_ij = x.  s is the semicircle-edge estimate of
    1/||(G+G^H)/2||_2 (the spectral normalisation of the correlated-sequence workload).
    """
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    x, y = counter_normal_pairs(seed, (i + j * n).reshape(-1))
    x = x.reshape(n, n)
    y = y.reshape(n, n)
    s = 1.0 / np.sqrt(2.0 * n)
    if complex_:
        Gm = (x + 1j * y) * np.sqrt(0.5)
        H = 0.5 * (Gm + np.conj(Gm.T))
        H[np.arange(n), np.arange(n)] = np.real(np.diag(H))
    else:
        H = 0.5 * (x + x.T)
    return s * H


# Seeds of the start vectors the library draws when the caller passes none (CHASE_SEED_V0 / CHASE_SEED_L0 of
# include/chase_gb300.h; a CPU test checks that the two agree).
LIBRARY_SEED_V0 = 0x2205024910000001
LIBRARY_SEED_L0 = 0x2205024910000002


def library_start_vectors(n: int, m: int, seed: int, complex_: bool = True) -> np.ndarray:
    """The n x m block the library draws for a null V0 (seed LIBRARY_SEED_V0, m = nev + nex) or a null L0
    (seed LIBRARY_SEED_L0, m = Lanczos runs): element (i, j) is the counter-based normal of counter i + j n,
    (x + i y)/sqrt(2) complex, x real."""
    i = np.arange(n)[:, None]
    j = np.arange(m)[None, :]
    x, y = counter_normal_pairs(seed, (i + j * n).astype(np.uint64))
    return (x + 1j * y) * np.sqrt(0.5) if complex_ else x


def sequence_seed(pid: int, step: int) -> int:
    return (SEED_BASE + 4 * 1000 + pid) * 16 + step


def spectrum_gapped(g, n: int, nlow: int = 80, gap: float = 1e-3, lo=-1.0, hi=1.0) -> np.ndarray:
    """U[lo,hi] spectrum whose lowest nlow+1 values have gaps >= gap.

    A sorted uniform sample x is spread as x_i + min(i, nlow+1) g' (g' = gap (hi-lo)/((hi-lo) - (nlow+1) gap))
    and mapped affinely back onto [lo, hi]: the lowest nlow+1 gaps become >= gap, everything stays sorted.
    """
    x = np.sort(g.uniform(lo, hi, size=n))
    span = hi - lo
    gp = gap * span / (span - (nlow + 1) * gap)
    y = x + np.minimum(np.arange(n), nlow + 1) * gp
    return lo + (y - lo) * span / (span + (nlow + 1) * gp)


def problem_c5(n: int = 4096, nev: int = 64, nex: int = 32) -> Problem:
    """Real symmetric, 8 reflectors, gapped U[-1,1] spectrum; loss weights w and symmetric B."""
    cfg = 5
    pid = 0 if n == 4096 else 1
    lam = spectrum_gapped(rng(cfg, pid, _S_LAMBDA), n)
    p = _make(f"c5.{n}", cfg, pid, n, nev, nex, lam, 8, False)
    gl = rng(cfg, pid, _S_LOSS)
    p.extra["w"] = gl.standard_normal(nev)
    G = gl.standard_normal((n, n))
    p.extra["B"] = 0.5 * (G + G.T)
    return p


def problem_small(n: int, nev: int, nex: int, complex_: bool = True, k_reflect: int = 4,
                  lo=-1.0, hi=1.0, seed_pid: int = 0, lam: np.ndarray | None = None, cfg: int = 9) -> Problem:
    """Small prescribed-spectrum problem for unit tests (config id 9 by default)."""
    if lam is None:
        lam = spectrum_sorted_uniform(rng(cfg, seed_pid, _S_LAMBDA), n, lo, hi)
    return _make(f"small.{n}.{seed_pid}", cfg, seed_pid, n, nev, nex, lam, k_reflect, complex_)


def from_dense(name: str, A: np.ndarray, nev: int, nex: int, cfg: int = 8, pid: int = 0,
               lam: np.ndarray | None = None) -> Problem:
    """Wrap an explicit matrix (e.g. 1-2-1, Wilkinson) with seeded start blocks; U is empty."""
    n = A.shape[0]
    complex_ = np.iscomplexobj(A)
    V0 = gaussian(rng(cfg, pid, _S_V0), (n, nev + nex), complex_)
    L0 = gaussian(rng(cfg, pid, _S_LANCZOS), (n, 4), complex_)
    p = Problem(name, n, nev, nex, 1e-10, 20, 36, complex_,
                np.asarray(lam if lam is not None else np.full(n, np.nan)),
                np.zeros((n, 0), dtype=A.dtype), V0, L0)
    p.extra["A"] = A
    return p
