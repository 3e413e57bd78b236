"""CPU checks of the arithmetic the FP64-class split-BF16 products rely on (no GPU).

Each operand row or column is scaled by a power of two to max |x| <= 1 and written as S signed digits,
x = sum_t d_t 2^(-7-8t), by the recurrence r_0 = 128 x, d_t = rint(r_t), r_{t+1} = 256 (r_t - d_t).
The claims checked here:
- every digit is an integer with |d_t| <= 128, so d_t 2^(-8t) is exact in bf16 (8-bit significand);
- the digits reconstruct x to within 2^(-8S) (S = 7: 2^-56, below FP64's 2^-53 unit roundoff);
- a level L = t + u collects at most L + 1 digit pairs (2 (L + 1) for complex operands), so its sum over a
  chunk of 96 K values stays below 2^24 for L <= 4 and is exact in FP32;
- the exact levels 0..4 of one product add up to at most 2^14 (1 + 2^-29) in level-0 units, so their int64
  accumulation in units of 2^-32 cannot overflow for K <= 65472 (and that limit is tight);
- the level-by-level product equals the FP64 product to 2^-53 per K term (FP64's unit roundoff, the parity
  tests' bound) when levels 0..4 are exact and the rest are rounded, and one slice fewer (S = 6) misses it;
- the mixed modes (2 or 3 slices, one rounded accumulator) meet the per-term bounds 2^-13 and 2^-20.
"""
import numpy as np
import pytest

S_FP64 = 7
NEX = 5
CHUNK = 96


def split_digits(x: np.ndarray, S: int) -> np.ndarray:
    """Digits d_t (float64 integers), shape (S,) + x.shape, of x with |x| <= 1."""
    r = np.asarray(x, dtype=np.float64) * 128.0
    out = []
    for _ in range(S):
        d = np.rint(r)
        out.append(d)
        r = (r - d) * 256.0
    return np.stack(out)


def bf16_exact(v: np.ndarray) -> bool:
    """True where v is exactly representable in bf16 (8 significant bits, no exponent limit issue here)."""
    v = np.asarray(v, dtype=np.float64)
    m, _ = np.frexp(np.abs(v))          # v = m 2^e, m in [0.5, 1)
    return bool(np.all(np.ldexp(m, 8) == np.rint(np.ldexp(m, 8))))


def test_digits_are_small_integers_exact_in_bf16():
    g = np.random.default_rng(0)
    x = np.concatenate([g.uniform(-1, 1, 20000), [1.0, -1.0, 0.0, 2.0 ** -60, -(1 - 2.0 ** -53), 0.5 + 2.0 ** -40]])
    d = split_digits(x, S_FP64)
    assert np.all(d == np.rint(d))
    assert np.max(np.abs(d)) <= 128
    for t in range(S_FP64):
        assert bf16_exact(d[t] * 2.0 ** (-8 * t))


@pytest.mark.parametrize("S", [2, 3, 6, 7])
def test_digits_reconstruct_within_truncation_bound(S):
    g = np.random.default_rng(S)
    x = g.uniform(-1, 1, 50000)
    d = split_digits(x, S)
    w = 2.0 ** (-7 - 8 * np.arange(S, dtype=np.float64))
    # sum in an order that is exact: the partial sums are multiples of 2^(-7-8(S-1)) below 1
    rec = np.zeros_like(x)
    for t in range(S):
        rec = rec + d[t] * w[t]
    assert np.max(np.abs(rec - x)) <= 2.0 ** (-8 * S)


def test_level_sums_fit_fp32_exactly():
    # worst case: every digit at its bound, all products of one level adding up over a chunk
    for L in range(NEX):
        pairs = L + 1
        for cplx_factor in (1, 2):
            worst = CHUNK * cplx_factor * pairs * 128 * 128
            assert worst < 2 ** 24, (L, worst)
    # the first inexact level would not fit: it is why levels >= 5 share the rounded accumulator
    assert CHUNK * 2 * (NEX + 1) * 128 * 128 >= 2 ** 24


def _exact_level_value(x, y, S=S_FP64, nex=NEX):
    """sum over digit pairs with t + u < nex of d_t(x) d_u(y) 2^(-8 (t + u)), in units of level 0."""
    dx, dy = split_digits(x, S), split_digits(y, S)
    v = np.zeros(np.broadcast(x, y).shape)
    for t in range(S):
        for u in range(S):
            if t + u < nex:
                v = v + dx[t] * dy[u] * 2.0 ** (-8 * (t + u))
    return v


def test_int64_exact_accumulator_cannot_overflow():
    # The exact levels of one product add up to (nearly) the product of the digit expansions,
    # 128 x * 128 y, so |value| <= 2^14 (1 + 2^-29) in level-0 units (the digits after the first
    # nex - 1 levels and the pairs t + u >= nex, t, u < nex, change it by far less than 2^-29).
    g = np.random.default_rng(5)
    x = np.concatenate([g.uniform(-1, 1, 200000), [1.0, -1.0, 1 - 2.0 ** -9, 1 - 2.0 ** -30]])
    y = np.concatenate([g.uniform(-1, 1, 200000), [1.0, 1.0, 1 - 2.0 ** -9, 1 - 2.0 ** -30]])
    per_product = 2.0 ** 14 * (1 + 2.0 ** -29)
    assert np.max(np.abs(_exact_level_value(x, y))) <= per_product
    # accumulated as int64 in units of 2^(-8 (nex - 1)): per chunk of 96 K values (two products per K
    # for complex operands) and over ceil(K / 96) chunks with K <= 65472; the level-by-level additions
    # inside a chunk overshoot its total by at most the levels 1..nex-1 (below 2^47)
    kmax = 65472
    chunks = -(-kmax // CHUNK)
    unit = 2 ** (8 * (NEX - 1))
    per_chunk = CHUNK * 2 * per_product * unit
    transient = sum(CHUNK * 2 * (L + 1) * 2 ** 14 * 2 ** (8 * (NEX - 1 - L)) for L in range(1, NEX))
    assert transient < 2 ** 47
    assert chunks * per_chunk + transient < 2 ** 63
    # one more chunk (K = 65568) would not be safe: the limit is tight
    assert (chunks + 1) * per_chunk >= 2 ** 63


def _split_product(A, B, S, nex, chunk=CHUNK):
    """C = A B from digit planes: levels < nex summed exactly per chunk (integers, accumulated without
    rounding), the levels from nex on added to one FP32 accumulator once per chunk and level (a coarse
    model of the shared rounded accumulator)."""
    ra = np.max(np.abs(A), axis=1)
    cb = np.max(np.abs(B), axis=0)
    sa = 2.0 ** np.ceil(np.log2(ra))
    sb = 2.0 ** np.ceil(np.log2(cb))
    da = split_digits(A / sa[:, None], S)          # (S, M, K)
    db = split_digits(B / sb[None, :], S)          # (S, K, N)
    M, K = A.shape
    N = B.shape[1]
    exact = np.zeros((M, N), dtype=object)         # python ints in units of 2^(-8 (nex - 1))
    inexact = np.zeros((M, N), dtype=np.float32)
    for k0 in range(0, K, chunk):
        ks = slice(k0, min(K, k0 + chunk))
        for L in range(2 * S - 1):
            lev = np.zeros((M, N))
            for t in range(S):
                u = L - t
                if 0 <= u < S and t + u <= S - 1:
                    lev += da[t][:, ks] @ db[u][ks, :]  # integer-valued, < 2^24 for exact levels
            if L >= S:
                continue
            if L < nex:
                assert np.max(np.abs(lev)) < 2 ** 24
                exact += (lev.astype(np.int64).astype(object) * (1 << (8 * (nex - 1 - L))))
            else:
                inexact = (inexact + np.float32(lev * 2.0 ** (-8 * L))).astype(np.float32)
    v = np.array(exact, dtype=np.float64) * 2.0 ** (-8 * (nex - 1)) + inexact.astype(np.float64)
    return v * (sa[:, None] * sb[None, :]) * 2.0 ** -14


def test_level_product_meets_the_fp64_parity_bound():
    g = np.random.default_rng(11)
    M, K, N = 24, 300, 16
    A = g.standard_normal((M, K))
    B = g.standard_normal((K, N))
    C = _split_product(A, B, S_FP64, NEX)
    ref = (A.astype(np.longdouble) @ B.astype(np.longdouble)).astype(np.float64)
    ra = np.max(np.abs(A), axis=1)
    cb = np.max(np.abs(B), axis=0)
    assert np.max(np.abs(C - ref) / (ra[:, None] * cb[None, :])) / K <= 2.0 ** -53
    # the bound is tight enough to catch a precision regression: six slices (truncation 2^-48) miss it
    C6 = _split_product(A, B, S_FP64 - 1, NEX)
    assert np.max(np.abs(C6 - ref) / (ra[:, None] * cb[None, :])) / K > 2.0 ** -53


@pytest.mark.parametrize("S,bound", [(2, 2.0 ** -13), (3, 2.0 ** -20)])
def test_mixed_mode_products_meet_their_bounds(S, bound):
    """The mixed modes (2 or 3 slices, 3 or 6 digit pairs, one rounded FP32 accumulator) stay within the
    per-term bounds the GPU tests use for them."""
    g = np.random.default_rng(20 + S)
    M, K, N = 16, 512, 12
    A = g.standard_normal((M, K))
    B = g.standard_normal((K, N))
    C = _split_product(A, B, S, 0)
    ref = (A.astype(np.longdouble) @ B.astype(np.longdouble)).astype(np.float64)
    ra = np.max(np.abs(A), axis=1)
    cb = np.max(np.abs(B), axis=0)
    err = np.max(np.abs(C - ref) / (ra[:, None] * cb[None, :])) / K
    assert err <= bound
    # and the truncation is what limits them: one slice fewer would not meet the bound
    C1 = _split_product(A, B, S - 1, 0) if S > 2 else None
    if C1 is not None:
        assert np.max(np.abs(C1 - ref) / (ra[:, None] * cb[None, :])) / K > bound
