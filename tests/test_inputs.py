"""Seeded inputs (CPU): the start vectors the library draws when the caller passes none.

`chase_solve` with a null V0 or L0 fills the block on the device with the counter-based normal generator
documented in include/chase_gb300.h (SplitMix64 + Box-Muller, CHASE_SEED_V0 / CHASE_SEED_L0);
`gen.problems.library_start_vectors` is its host restatement, so that the oracle can be run from the same
start vectors.  These checks pin the host side: its seeds are the header's, its layout is the documented
counter order, its draws have the moments of a standard (complex) normal, and Algorithm 1 started from them
reaches the prescribed spectrum.
"""
import os
import re

import numpy as np

from gen import problems as G
from oracle import chase_oracle as O

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "chase_gb300.h")


def test_seeds_match_the_header():
    text = open(HEADER).read()
    seeds = {m.group(1): int(m.group(2), 16) for m in re.finditer(r"#define (CHASE_SEED_\w+) 0x([0-9a-fA-F]+)ull", text)}
    assert seeds["CHASE_SEED_V0"] == G.LIBRARY_SEED_V0
    assert seeds["CHASE_SEED_L0"] == G.LIBRARY_SEED_L0
    assert G.LIBRARY_SEED_V0 != G.LIBRARY_SEED_L0


def test_layout_is_the_documented_counter_order():
    n, m = 37, 5
    V = G.library_start_vectors(n, m, G.LIBRARY_SEED_V0, True)
    for j in (0, 3):
        x, y = G.counter_normal_pairs(G.LIBRARY_SEED_V0, np.arange(j * n, (j + 1) * n, dtype=np.uint64))
        assert np.array_equal(V[:, j], (x + 1j * y) * np.sqrt(0.5))
    R = G.library_start_vectors(n, m, G.LIBRARY_SEED_L0, False)
    x, _ = G.counter_normal_pairs(G.LIBRARY_SEED_L0, np.arange(n * m, dtype=np.uint64))
    assert np.array_equal(R, x.reshape(m, n).T)
    # deterministic, and the two seeds give unrelated blocks
    assert np.array_equal(V, G.library_start_vectors(n, m, G.LIBRARY_SEED_V0, True))
    W = G.library_start_vectors(n, m, G.LIBRARY_SEED_L0, True)
    assert abs(np.vdot(V.ravel(), W.ravel())) / (np.linalg.norm(V) * np.linalg.norm(W)) < 0.1


def test_moments_of_a_standard_normal():
    N = 200000
    V = G.library_start_vectors(N, 1, G.LIBRARY_SEED_V0, True)[:, 0]
    # complex standard normal: E z = 0, E |z|^2 = 1, E z^2 = 0 (4-sigma bounds)
    assert abs(np.mean(V)) < 4 * np.sqrt(1.0 / N)
    assert abs(np.mean(np.abs(V) ** 2) - 1.0) < 4 * np.sqrt(1.0 / N)
    assert abs(np.mean(V ** 2)) < 4 * np.sqrt(2.0 / N)
    x = G.library_start_vectors(N, 1, G.LIBRARY_SEED_L0, False)[:, 0]
    assert abs(np.mean(x)) < 4 * np.sqrt(1.0 / N)
    assert abs(np.var(x) - 1.0) < 4 * np.sqrt(2.0 / N)
    # Gaussian tails: P(|x| > 2) = 0.0455
    assert abs(np.mean(np.abs(x) > 2.0) - 0.0455) < 4 * np.sqrt(0.0455 / N)


def test_algorithm_1_from_the_library_start_vectors():
    p = G.problem_c1()
    A = p.dense()
    V0 = G.library_start_vectors(p.n, p.ne, G.LIBRARY_SEED_V0, True)
    L0 = G.library_start_vectors(p.n, 4, G.LIBRARY_SEED_L0, True)
    r = O.chase_solve(A, p.nev, p.nex, p.tol, p.deg, p.maxdeg, V0, L0, p.lanczos_steps)
    assert r.converged
    assert np.max(np.abs(r.eigvals - p.lam[:p.nev])) <= 1e-10 * p.norm2()
