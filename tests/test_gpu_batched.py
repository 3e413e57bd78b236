"""Batched solves of correlated sequences A_{k+1} = A_k + 1e-3 H_k with warm starts (GPU)."""
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


def test_device_perturbation_matches_host(pkg):
    for cplx in (True, False):
        n = 257
        A = G.problem_small(n, 2, 2, complex_=cplx).dense()
        s = pkg.Chase(n, 4, complex_=cplx)
        At = dev(A)
        s.perturb(At, 1e-3, 99)
        ref = A + 1e-3 * G.perturbation(n, 99, cplx)
        got = host(At)
        assert np.max(np.abs(got - ref)) <= 1e-15
        assert np.array_equal(got, np.conj(got.T))


def test_batched_warm_start_sequence(pkg):
    ns = [300, 420, 515]
    probs = [G.problem_c4(pid, n) for pid, n in enumerate(ns)]
    nevs = [p.nev for p in probs]
    nexs = [p.nex for p in probs]
    ctx = pkg.Chase(max(ns), max(p.ne for p in probs), complex_=True)
    A_host = [p.dense() for p in probs]
    A_dev = [dev(a) for a in A_host]
    V = [dev(p.V0) for p in probs]
    L0 = [dev(p.L0) for p in probs]
    mv = []
    for step in range(3):
        ws, stats = ctx.solve_batched(A_dev, nevs, nexs, 1e-10, 20, "fp64", V, L0)
        mv.append([st["matvecs"] for st in stats])
        for q, p in enumerate(probs):
            ref = np.linalg.eigvalsh(A_host[q])[: p.nev]
            nrm = np.max(np.abs(np.linalg.eigvalsh(A_host[q])))
            w = ws[q].cpu().numpy()
            assert np.max(np.abs(w - ref)) <= 1e-10 * nrm
            Vq = host(V[q])[:, : p.nev]
            R = A_host[q] @ Vq - Vq * w[None, :]
            assert np.max(np.linalg.norm(R, axis=0)) <= 1e-10 * nrm * 1.01
            seed = G.sequence_seed(q, step)
            ctx.perturb(A_dev[q], 1e-3, seed)
            A_host[q] = A_host[q] + 1e-3 * G.perturbation(p.n, seed, True)
    # warm starts from the previous eigenvectors need fewer filter products than the cold start
    for q in range(len(probs)):
        assert max(mv[1][q], mv[2][q]) < mv[0][q]


@pytest.mark.parametrize("workers,grouped", [(1, 0), (3, 0), (1, 1), (3, 1)])
def test_batched_workers_uneven_sizes(pkg, workers, grouped):
    """A batch of uneven sizes, in the worker-pool mode (concurrent workers, one stream and workspace
    each) and in the grouped mode (lockstep problems, one grouped filter launch per degree step, the
    other stages on `workers` host threads): every problem meets the eigenvalue and residual tolerance
    against a dense eigendecomposition, and the returned start blocks warm-start a second, perturbed
    step."""
    ns = [160, 613, 96, 401, 257, 520, 333]
    probs = [G.problem_c4(pid, n) for pid, n in enumerate(ns)]
    ctx = pkg.Chase(max(ns), max(p.ne for p in probs), complex_=True,
                    opts={"batch_workers": workers, "batch_grouped": grouped})
    A_host = [p.dense() for p in probs]
    A_dev = [dev(a) for a in A_host]
    V = [dev(p.V0) for p in probs]
    L0 = [dev(p.L0) for p in probs]
    for step in range(2):
        ws, stats = ctx.solve_batched(A_dev, [p.nev for p in probs], [p.nex for p in probs], 1e-10, 20, "fp64", V, L0)
        for q, p in enumerate(probs):
            lam_all = np.linalg.eigvalsh(A_host[q])
            nrm = np.max(np.abs(lam_all))
            w = ws[q].cpu().numpy()
            assert np.max(np.abs(w - lam_all[: p.nev])) <= 1e-10 * nrm
            Vq = host(V[q])[:, : p.nev]
            R = A_host[q] @ Vq - Vq * w[None, :]
            assert np.max(np.linalg.norm(R, axis=0)) <= 1e-10 * nrm * 1.01
            assert stats[q]["locked"] >= p.nev and 0.0 < stats[q]["max_resid"] <= 1e-10
        for q, p in enumerate(probs):
            seed = G.sequence_seed(q, step)
            ctx.perturb(A_dev[q], 1e-3, seed)
            A_host[q] = A_host[q] + 1e-3 * G.perturbation(p.n, seed, True)
    ctx.close()


def test_batched_rejects_oversize_problem(pkg):
    """A problem larger than the context is an argument error, reported as a status (no device work)."""
    ctx = pkg.Chase(128, 12, complex_=True, opts={"batch_workers": 2})
    p = G.problem_c4(0, 200)
    with pytest.raises(pkg.ChaseError) as e:
        ctx.solve_batched([dev(p.dense())], [p.nev], [p.nex], 1e-10, 20, "fp64", [dev(p.V0)], [dev(p.L0)])
    assert e.value.status == 1
    ctx.close()


def test_batched_c4_subset_vs_oracle(pkg):
    """Problems of the 64-problem batched workload at their own sizes (n = 4155 and n = 568, nev 5% of n,
    nex nev/2), two steps of the correlated sequence: the cold step from the seeded block, then
    A += 1e-3 H and a warm start from each side's own previous search block.  Eigenvalues, residuals and
    iteration counts against the CPU oracle run the same way (its small eigensolves by LAPACK)."""
    pids = [41, 19]
    probs = [G.problem_c4(pid) for pid in pids]
    assert probs[0].n >= 4096 and probs[1].n <= 600
    ctx = pkg.Chase(max(p.n for p in probs), max(p.ne for p in probs), complex_=True,
                    opts={"batch_workers": 2})
    A_host = [p.dense() for p in probs]
    A_dev = [dev(a) for a in A_host]
    V = [dev(p.V0) for p in probs]
    L0 = [dev(p.L0) for p in probs]
    blocks = [p.V0 for p in probs]
    for step in range(2):
        ws, stats = ctx.solve_batched(A_dev, [p.nev for p in probs], [p.nex for p in probs], 1e-10, 20, "fp64",
                                      V, L0)
        for q, p in enumerate(probs):
            ref = O.chase_solve(A_host[q], p.nev, p.nex, 1e-10, 20, 36, blocks[q], p.L0, 25,
                                small_eigh=np.linalg.eigh)
            assert ref.converged
            nrm = p.norm2() * (1 + 2e-3)      # |lam| <= 1, plus the perturbations
            w = ws[q].cpu().numpy()
            assert np.max(np.abs(w - ref.eigvals)) <= 1e-10 * nrm
            if step == 0:
                assert np.max(np.abs(w - p.lam[: p.nev])) <= 1e-10 * nrm
            Vq = host(V[q])[:, : p.nev]
            R = A_host[q] @ Vq - Vq * w[None, :]
            assert np.max(np.linalg.norm(R, axis=0)) <= 1e-10 * nrm * 1.01
            assert abs(stats[q]["iterations"] - ref.iterations) <= 1
            blocks[q] = ref.block
        for q, p in enumerate(probs):
            seed = G.sequence_seed(pids[q], step)
            ctx.perturb(A_dev[q], 1e-3, seed)
            A_host[q] = A_host[q] + 1e-3 * G.perturbation(p.n, seed, True)
    ctx.close()
