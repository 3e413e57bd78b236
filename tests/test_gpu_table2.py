"""The eigen-type suite of Table 2 (matrices of Table 1) at n = 1000 on the GPU against the CPU oracle:
Wilkinson, Uniform and Geometric (and 1-2-1), real symmetric, nev 75, nex 25 (the paper's 7.5% + 2.5%
of n), tol 1e-10, every product on the split tensor-core path."""
import numpy as np
import pytest

from gen import problems as G
from oracle import chase_oracle as O
from tests.helpers import dev, host

pytestmark = pytest.mark.gpu

N, NEV, NEX = 1000, 75, 25


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2205_02491_gb300 as P
    return P


def _matrix(name):
    if name == "Wilkinson":
        return G.matrix_wilkinson(N)
    if name == "1-2-1":
        return G.matrix_121(N)
    lam = G.spectrum_uniform_table1(N) if name == "Uniform" else G.spectrum_geometric_table2(N)
    return G.problem_small(N, NEV, NEX, complex_=False, k_reflect=8, lam=lam, seed_pid=31).dense()


@pytest.mark.parametrize("name", ["Wilkinson", "Uniform", "Geometric", "1-2-1"])
def test_table2_type_vs_oracle(pkg, name):
    A = _matrix(name)
    p = G.from_dense(name, A, NEV, NEX, cfg=6, pid=3)
    ref = O.chase_solve(A, NEV, NEX, 1e-10, 20, 36, p.V0, p.L0, 25)
    assert ref.converged
    nrm = float(np.max(np.abs(np.linalg.eigvalsh(A))))
    s = pkg.Chase(N, NEV + NEX, complex_=False, opts={"native_below_mflop": 0})
    w, Vt = s.solve(dev(A), NEV, NEX, 1e-10, 20, "fp64", dev(p.V0), dev(p.L0))
    w = w.cpu().numpy()
    st = s.stats()
    assert np.max(np.abs(w - ref.eigvals)) <= 1e-10 * nrm
    V = host(Vt)
    R = A @ V - V * w[None, :]
    assert np.max(np.linalg.norm(R, axis=0)) <= 1e-10 * nrm * 1.01
    assert np.max(np.abs(V.T @ V - np.eye(NEV))) <= 1e-12
    assert abs(st["iterations"] - ref.iterations) <= 1
    s.close()
