"""Torch-facing wrapper of the C ABI: device memory and streams from PyTorch,
every step of the eigensolver in the library's CUDA kernels.

Layout convention: the library works on column-major matrices.  A torch tensor
``Xt`` of shape (cols, rows), contiguous, *is* the column-major storage of the
rows x cols matrix ``Xt.mT``; ``colmajor(X)`` builds it and ``Xt.mT`` reads it.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L


def colmajor(X: torch.Tensor) -> torch.Tensor:
    """(rows x cols) tensor -> contiguous (cols x rows) tensor holding its column-major storage."""
    return X.mT.contiguous()


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


def _cuda_stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    return stream.cuda_stream


class Chase:
    """One solver context (workspace preallocated for n <= n_max, nev+nex <= ne_max)."""

    def __init__(self, n_max: int, ne_max: int, complex_: bool = True, opts: dict | None = None,
                 stream: torch.cuda.Stream | None = None):
        self.lib = L.load()
        self.complex_ = complex_
        self.dtype = torch.complex128 if complex_ else torch.float64
        o = L.Opts()
        self.lib.chase_default_opts(C.byref(o))
        for k, v in (opts or {}).items():
            setattr(o, k, int(v))
        self.opts = o
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ctx = C.c_void_p()
        st = self.lib.chase_create(C.byref(ctx), int(n_max), int(ne_max), L.CHASE_C128 if complex_ else L.CHASE_R64,
                                   C.byref(o), _cuda_stream_ptr(self.stream))
        if st != 0:
            raise L.ChaseError(st, "chase_create failed (workspace does not fit or bad arguments)")
        self.ctx = ctx
        self.n_max, self.ne_max = n_max, ne_max

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.chase_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        L.check(self.ctx, st)

    # ------------------------------------------------------------------ full solve
    def solve(self, At: torch.Tensor, nev: int, nex: int, tol: float, deg: int, mode="fp64",
              V0t: torch.Tensor | None = None, L0t: torch.Tensor | None = None, out=None):
        """At: column-major storage (n x n) of A; V0t: (ne x n) storage of V0; L0t: (runs x n).

        The inputs may be CUDA tensors or CPU tensors (pinned for DMA speed): the library copies host inputs
        to the device itself.  Returns (eigvals[nev] float64, eigvecs storage (nev x n), i.e. eigvecs =
        result.mT), on At's device, written into out = (w, Vt) when given (for host results, pinned buffers
        the caller keeps avoid a pageable copy and a fresh allocation per call).
        """
        n = At.shape[-1]
        mode = L.MODES[mode] if isinstance(mode, str) else int(mode)
        self._chk(self.lib.chase_solve(self.ctx, _ptr(At), n, n, nev, nex, float(tol), int(deg), mode, _ptr(V0t),
                                       _ptr(L0t)))
        on_dev = 1 if At.is_cuda else 0
        if out is not None:
            w, Vt = out
            if (w.shape != (nev,) or w.dtype != torch.float64 or Vt.shape != (nev, n) or Vt.dtype != self.dtype
                    or w.is_cuda != At.is_cuda or Vt.is_cuda != At.is_cuda or not Vt.is_contiguous()):
                raise ValueError("out must be (float64 [nev], contiguous [nev, n] of the solver dtype) on At's device")
        else:
            w = torch.empty(nev, dtype=torch.float64, device=At.device)
            Vt = torch.empty((nev, n), dtype=self.dtype, device=At.device)
        self._chk(self.lib.chase_eigvals(self.ctx, _ptr(w), on_dev))
        self._chk(self.lib.chase_eigvecs(self.ctx, _ptr(Vt), n, on_dev))
        return w, Vt

    def stats(self) -> dict:
        s = L.Stats()
        self._chk(self.lib.chase_stats(self.ctx, C.byref(s)))
        return s.as_dict()

    def solve_batched(self, Ats, nevs, nexs, tol, deg, mode, Vts, L0ts):
        nprob = len(Ats)
        P = C.c_void_p * nprob
        Ap = P(*[_ptr(a) for a in Ats])
        ns = (C.c_int64 * nprob)(*[a.shape[-1] for a in Ats])
        nv = (C.c_int * nprob)(*nevs)
        nx = (C.c_int * nprob)(*nexs)
        Vp = P(*[_ptr(v) for v in Vts])
        Lp = P(*[_ptr(x) for x in L0ts])
        ws = [torch.empty(nevs[p], dtype=torch.float64, device=Ats[p].device) for p in range(nprob)]
        Wp = P(*[_ptr(w) for w in ws])
        stats = (L.Stats * nprob)()
        mode = L.MODES[mode] if isinstance(mode, str) else int(mode)
        self._chk(self.lib.chase_solve_batched(self.ctx, nprob, Ap, ns, nv, nx, float(tol), int(deg), mode, Vp, Lp, Wp,
                                               stats))
        return ws, [s.as_dict() for s in stats]

    def backward(self, At, gbar_lambda, gbar_Vt, minres_tol=1e-12, maxit=5000):
        """Real symmetric only.  gbar_Vt: (nev x n) storage of Vbar; returns Abar storage (n x n)."""
        n = At.shape[-1]
        out = torch.empty((n, n), dtype=torch.float64, device=At.device)
        self._chk(self.lib.chase_backward(self.ctx, _ptr(At), n, _ptr(gbar_lambda), _ptr(gbar_Vt), n, _ptr(out), n,
                                          float(minres_tol), int(maxit)))
        return out

    # ------------------------------------------------------------------ steps
    def lanczos(self, At, ne: int, L0t, runs: int, steps: int):
        out = (C.c_double * 4)()
        n = At.shape[-1]
        self._chk(self.lib.chase_lanczos(self.ctx, _ptr(At), n, n, ne, _ptr(L0t), runs, steps, out))
        return dict(b_sup=out[0], mu_1=out[1], mu_ne=out[2], theta_max=out[3])

    def filter(self, At, Vt, degrees, b_sup, mu_1, mu_ne, mode="fp64_native"):
        n = At.shape[-1]
        k = Vt.shape[0]
        d = (C.c_int * k)(*[int(x) for x in degrees])
        mode = L.MODES[mode] if isinstance(mode, str) else int(mode)
        self._chk(self.lib.chase_filter(self.ctx, _ptr(At), n, n, _ptr(Vt), n, k, d, float(b_sup), float(mu_1),
                                        float(mu_ne), mode))
        return Vt

    def qr(self, Xt, nlocked: int = 0):
        n = Xt.shape[-1]
        self._chk(self.lib.chase_qr(self.ctx, _ptr(Xt), n, n, Xt.shape[0], nlocked))
        return Xt

    def rayleigh_ritz(self, At, Qt):
        n = At.shape[-1]
        k = Qt.shape[0]
        w = np.zeros(k)
        r = np.zeros(k)
        self._chk(self.lib.chase_rayleigh_ritz(self.ctx, _ptr(At), n, n, _ptr(Qt), n, k,
                                               w.ctypes.data_as(C.c_void_p), r.ctypes.data_as(C.c_void_p)))
        return w, r

    def heevj(self, Gt):
        k = Gt.shape[0]
        w = np.zeros(k)
        Zt = torch.empty_like(Gt)
        self._chk(self.lib.chase_heevj(self.ctx, _ptr(Gt), k, k, w.ctypes.data_as(C.c_void_p), _ptr(Zt), k))
        return w, Zt

    def hemm(self, At, Bt, mode="fp64"):
        n = At.shape[-1]
        k = Bt.shape[0]
        Ct = torch.empty_like(Bt)
        mode = L.MODES[mode] if isinstance(mode, str) else int(mode)
        self._chk(self.lib.chase_hemm(self.ctx, _ptr(At), n, n, _ptr(Bt), n, k, _ptr(Ct), n, mode))
        return Ct

    def perturb(self, At, eps: float, seed: int):
        """A += eps * H(seed) in place (seeded Hermitian Gaussian of spectral norm about 1)."""
        n = At.shape[-1]
        self._chk(self.lib.chase_perturb(self.ctx, _ptr(At), n, n, float(eps), int(seed) & ((1 << 64) - 1)))
        return At

    def generate(self, At, lam, Ut, Bt, Dt):
        n = At.shape[-1]
        k = Ut.shape[0]
        self._chk(self.lib.chase_generate(self.ctx, _ptr(At), n, n, _ptr(lam), _ptr(Ut), _ptr(Bt), _ptr(Dt), k))
        return At


class ChaseEigh(torch.autograd.Function):
    """Lowest nev eigenpairs of a real symmetric A with a hand-written adjoint (chase_backward).

    forward(A, solver, nev, nex, tol, deg, mode, V0t, L0t, minres_tol, minres_maxit) -> (lam, V), V: n x nev.
    A is a float64 CUDA tensor (symmetric, so its row-major storage is its column-major storage).
    The backward uses the solver's last result: run backward before the next solve on the same solver.
    Gradient: Abar = V (diag(gbar_lam) + F o (V^T Vbar)) V^T + X V^T, X from projected MINRES.
    """

    @staticmethod
    def forward(ctx, A, solver, nev, nex, tol, deg, mode, V0t, L0t, minres_tol=1e-12, minres_maxit=5000):
        At = A.detach().contiguous()
        w, Vt = solver.solve(At, nev, nex, tol, deg, mode, V0t, L0t)
        ctx.solver = solver
        ctx.minres = (minres_tol, minres_maxit)
        ctx.save_for_backward(At)
        return w, Vt.mT

    @staticmethod
    def backward(ctx, gw, gV):
        (At,) = ctx.saved_tensors
        gw = gw.contiguous() if gw is not None else None
        gVt = colmajor(gV) if gV is not None else None
        gA = ctx.solver.backward(At, gw, gVt, *ctx.minres)
        return (gA,) + (None,) * 10


def measure_fp64_peak(which: str = "dfma") -> float:
    """Measured FP64 rate of this device in TFLOP/s: "dfma" (CUDA cores) or "dmma" (tensor cores)."""
    lib = L.load()
    out, ms = C.c_double(), C.c_double()
    L.check(None, lib.chase_measure_fp64_peak(0 if which == "dfma" else 1, C.byref(out), C.byref(ms)))
    return float(out.value)


def measure_mma_issue(n_cols: int = 80, variant: int = 0) -> float:
    """Cycles per tcgen05.mma of the split-product kernel's issue pattern (see chase_measure_mma_issue)."""
    lib = L.load()
    out = C.c_double()
    L.check(None, lib.chase_measure_mma_issue(int(n_cols), int(variant), C.byref(out)))
    return float(out.value)


def set_wait_limit_ns(ns: int) -> None:
    """Testing hook: wall-clock limit of the Jacobi sweep kernel's grid-barrier waits (0: default 2 s)."""
    L.load().chase_set_wait_limit_ns(int(ns))


def kernel_launch_count() -> int:
    """Kernel launches made by the library in this process so far."""
    return int(L.load().chase_kernel_launch_count())


def workspace_bytes(n_max: int, ne_max: int, complex_: bool = True, opts: dict | None = None) -> int:
    lib = L.load()
    o = L.Opts()
    lib.chase_default_opts(C.byref(o))
    for k, v in (opts or {}).items():
        setattr(o, k, int(v))
    return int(lib.chase_workspace_bytes(int(n_max), int(ne_max), L.CHASE_C128 if complex_ else L.CHASE_R64,
                                         C.byref(o)))
