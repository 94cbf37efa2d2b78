"""Learned warm start for sequences of related problems (binding and driver).

Section 3 of the paper motivates sequences of related eigenproblems (each
self-consistency cycle of a DFT code solves dozens).  Here a small MLP
(two hidden layers of 256), trained on the GPU by the library's own forward
and backward kernels (``gsyeig_mlp_*``: bf16 tcgen05 products, fp32
parameters and Adam), reads the previous two problems' eigenvalues and the
overlaps of their eigenvectors and predicts, per wanted pair, how far to
extrapolate each eigenvector along the sequence.  The extrapolated block is
the start block of the solver's FP64 block refinement
(``gsyeig_opts.block_start``).  The solver's residual test alone decides
acceptance; a start block whose refinement does not converge falls back to
the FP64 Lanczos stage inside the library.

This module only sequences library calls: features, alignment, training
targets and the extrapolation run in the library's kernels
(``gsyeig_ws_features / _align / _coef_targets / _extrapolate``), and torch
supplies device memory.
"""
from __future__ import annotations

import ctypes

import torch

from . import GsyeigError, Solver, colmajor_empty, load


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(dev):
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


class Mlp:
    """The n_in -> hidden -> hidden -> n_out network, its Adam state and a workspace."""

    def __init__(self, n_in: int, n_out: int, hidden: int = 256, seed: int = 0, batch_max: int = 256,
                 device="cuda"):
        self.lib = load()
        self.dims = (n_in, hidden, n_out)
        self.device = torch.device(device)
        P = self.lib.gsyeig_mlp_param_count(*self.dims)
        if P < 0:
            raise ValueError(f"unsupported network sizes {self.dims}")
        self.P = P
        f32 = dict(device=self.device, dtype=torch.float32)
        self.params = torch.empty(P, **f32)
        self.m = torch.zeros(P, **f32)
        self.v = torch.zeros(P, **f32)
        self.grad = torch.empty(P, **f32)
        self.loss = torch.zeros(1, **f32)
        self.batch_max = batch_max
        self.ws = torch.empty(self.lib.gsyeig_mlp_workspace_floats(*self.dims, batch_max), **f32)
        self.step = 0
        self._chk(self.lib.gsyeig_mlp_init(_p(self.params), *self.dims, seed, _stream(self.device)), "init")

    def _chk(self, st, what):
        if st != 0:
            raise GsyeigError(st, f"mlp {what}: " + self.lib.gsyeig_strerror(st).decode())

    def forward(self, X: torch.Tensor) -> torch.Tensor:
        X = X.contiguous()
        b = X.shape[0]
        if b > self.batch_max:
            raise ValueError("batch larger than the workspace")
        Y = torch.empty(b, self.dims[2], device=self.device, dtype=torch.float32)
        self._chk(self.lib.gsyeig_mlp_forward(_p(self.params), *self.dims, _p(X), b, _p(Y), _p(self.ws),
                                              _stream(self.device)), "forward")
        return Y

    def gradient(self, X, T, out_weights=None):
        """(loss, gradient) of the weighted mean squared error on (X, T)."""
        X, T = X.contiguous(), T.contiguous()
        self._chk(self.lib.gsyeig_mlp_grad(_p(self.params), *self.dims, _p(X), _p(T), _p(out_weights), X.shape[0],
                                           _p(self.grad), _p(self.loss), _p(self.ws), _stream(self.device)), "grad")
        return float(self.loss.item()), self.grad

    def adam_step(self, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step += 1
        self._chk(self.lib.gsyeig_mlp_adam(_p(self.params), _p(self.m), _p(self.v), _p(self.grad), self.P, self.step,
                                           lr, beta1, beta2, eps, _stream(self.device)), "adam")

    def train(self, X, T, iters: int, lr: float = 1e-3, out_weights=None):
        """Full-batch Adam; returns the loss history (one value per iteration)."""
        hist = []
        for _ in range(iters):
            loss, _ = self.gradient(X, T, out_weights)
            self.adam_step(lr)
            hist.append(loss)
        return hist


class SequenceSolver:
    """Solves a sequence of pencils (A_t, B) for the s smallest eigenpairs,
    each solve started from the previous solutions in one of three ways:

    * ``"random"``: the counter-based random start vector of the plain solver;
    * ``"reuse"``: the start vector F sum_j x_j(t-1) built from the previous
      problem's eigenvectors, unchanged (the unlearned control);
    * ``"learned"``: the same construction from the block the network
      proposes: every previous eigenvector extrapolated along the sequence,
      x_j(t-1) + c_j (x_j(t-1) - x_j(t-2)) (aligned by their overlaps), with
      the coefficients c_j predicted from the previous two problems'
      eigenvalues and overlaps.

    The two warm methods also set the shift of the next solve
    (``gsyeig_opts.shift``): half a mean spacing of the wanted eigenvalues
    below the previous smallest one (reuse), or below its extrapolation by a
    coefficient the network predicts as its last output (learned).  With
    A - shift B positive definite the solve takes the inverse route of
    Section 3.1 even when A itself is indefinite (as the sequence's A(t)
    become once an eigenvalue crosses zero); otherwise it falls back to the
    direct route.  Every method runs the same Lanczos iteration with Ritz
    tests every ``check_every`` steps, so a start vector rich in the wanted
    eigenvectors stops early.  The solver's residual test decides acceptance
    in every case."""

    C_LO, C_HI = 0.0, 1.5  # range of the extrapolation coefficients
    SHIFT_FRAC = 0.5       # margin of the shift below the smallest eigenvalue, in mean spacings

    def __init__(self, s: int, method: str, B: torch.Tensor, mlp: Mlp | None = None, device=0, check_every: int = 16,
                 **opts):
        assert method in ("random", "reuse", "learned")
        self.s, self.method, self.mlp, self.B = s, method, mlp, B
        # the inverse route (largest mu = 1/lambda of L^-T B L^-1) by default;
        # a pencil whose A is not definite falls back to the direct route
        # inside the library
        self.solver = Solver(device, **{"inverse": 1, "check_every": check_every, **opts})
        self.lib = self.solver.lib
        self.prev = []  # (w, X) of the last two solves
        dev = torch.device("cuda", device)
        self.dev = dev
        n = B.shape[0]
        self.D = colmajor_empty(n, s, device=dev)
        self.start = colmajor_empty(n, s, device=dev)
        self.weights = torch.ones(s, device=dev, dtype=torch.float64)
        self.sigma = torch.zeros(1, device=dev, dtype=torch.float64)

    def _st(self):
        return _stream(self.dev)

    def overlaps(self, X, Y):
        """P = X^T B Y (s x s) on the library's GEMM engine (B symmetric: its
        transpose is the same matrix, in column-major storage)."""
        return self.solver.gemm(X, self.solver.gemm(self.B.t(), Y), transA=True)

    def align(self, X, Y, out, match=None):
        """out_j = sgn_j Y[:, pi_j] - X[:, j] (gsyeig_ws_align)."""
        P = self.overlaps(X, Y)
        n, s = X.shape
        st = self.lib.gsyeig_ws_align(n, s, _p(X), X.stride(1), _p(Y), Y.stride(1), _p(P), P.stride(1), _p(out),
                                      out.stride(1), _p(match), self._st())
        if st != 0:
            raise GsyeigError(st, "ws_align")
        return out

    def features(self, w, w_prev, X, X_prev):
        """Network input for the problem after (w, X): the eigenvalue features
        of gsyeig_ws_features (2s + 1) and the best overlaps of the eigenvectors
        with the previous ones (s); also leaves the aligned difference in self.D."""
        s = self.s
        f = torch.empty(3 * s + 1, device=self.dev, dtype=torch.float32)
        scal = torch.empty(2, device=self.dev, dtype=torch.float64)
        st = self.lib.gsyeig_ws_features(s, _p(w), _p(w_prev), 1.0, _p(f), _p(scal), self._st())
        if st != 0:
            raise GsyeigError(st, "ws_features")
        self.align(X, X_prev, self.D, match=f[2 * s + 1:])
        return f

    def shift_target(self, w_prev, w, w_next, out):
        """The extrapolation coefficient of the smallest eigenvalue (gsyeig_ws_shift_target)."""
        st = self.lib.gsyeig_ws_shift_target(_p(w_prev), _p(w), _p(w_next), self.C_LO, self.C_HI, _p(out), self._st())
        if st != 0:
            raise GsyeigError(st, "ws_shift_target")
        return out

    def targets(self, X_prev, X, X_next, out):
        """B-optimal extrapolation coefficients of x_j(t) (gsyeig_ws_coef_targets)."""
        n, s = X.shape
        D = self.align(X, X_prev, colmajor_empty(n, s, device=self.dev))
        E = self.align(X, X_next, colmajor_empty(n, s, device=self.dev))
        BD = self.solver.gemm(self.B.t(), D)
        BE = self.solver.gemm(self.B.t(), E)
        st = self.lib.gsyeig_ws_coef_targets(n, s, _p(D), D.stride(1), _p(BD), BD.stride(1), _p(BE), BE.stride(1),
                                             self.C_LO, self.C_HI, _p(out), self._st())
        if st != 0:
            raise GsyeigError(st, "ws_coef_targets")
        return out

    def solve(self, A: torch.Tensor, B: torch.Tensor):
        """One solve of the sequence (A, B not modified): (w, X, info, ms)."""
        s, sol = self.s, self.solver
        opts = dict(start_block=None, start_weights=None, shift=0.0)
        coef = None
        if self.method != "random" and self.prev:
            opts.update(start_block=self.prev[-1][1], start_weights=self.weights)
        if self.method == "learned" and len(self.prev) >= 2:
            (w1, X1), (w0, X0) = self.prev[-1], self.prev[-2]
            f = self.features(w1, w0, X1, X0)
            c = self.mlp.forward(f.unsqueeze(0))
            n = X1.shape[0]
            st = self.lib.gsyeig_ws_extrapolate(n, s, _p(X1), X1.stride(1), _p(self.D), self.D.stride(1), _p(c),
                                                self.C_LO, self.C_HI, _p(self.start), self.start.stride(1), self._st())
            if st != 0:
                raise GsyeigError(st, "ws_extrapolate")
            opts.update(start_block=self.start, start_weights=self.weights)
            coef = c[0, s:]
        if self.method != "random" and self.prev:
            w1 = self.prev[-1][0]
            w0 = self.prev[-2][0] if len(self.prev) >= 2 else None
            st = self.lib.gsyeig_ws_shift(s, _p(w0 if coef is not None else None), _p(w1), _p(coef), self.C_LO,
                                          self.C_HI, self.SHIFT_FRAC, _p(self.sigma), self._st())
            if st != 0:
                raise GsyeigError(st, "ws_shift")
            opts.update(shift=float(self.sigma.item()))
        sol.set_options(**opts)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        w, X, info = sol.solve(A, B, s)
        e1.record()
        torch.cuda.synchronize()
        self.prev = (self.prev + [(w, X)])[-2:]
        return w, X, info, e0.elapsed_time(e1)


def evaluate_sequence(pencil, B, n: int, s: int, T: int, T_train: int, iters: int = 2000, lr: float = 1e-3,
                      check=None, device=0, seed: int = 0):
    """The warm-start experiment on a sequence: ``pencil(k)`` returns
    (A_k, B, lam_k).  Problems 0..T_train-1 are solved with the plain random
    start; the network is trained on them (features of t; targets from t-1,
    t, t+1: the B-optimal extrapolation coefficients of the eigenvectors and
    the one of the smallest eigenvalue); problems T_train..T-1 are then
    solved by the three methods, each from its own previous solutions.
    ``check(A, B, w, X, lam)`` (optional; lam the whole constructed spectrum,
    ascending) is called on every solution.
    Returns (totals {method: [operator applications, ms, restarts]},
    training loss history, ms of the training)."""
    runs = {m: SequenceSolver(s, m, B, device=device) for m in ("random", "reuse", "learned")}
    collect = runs["random"]
    dev = collect.dev
    sols = []
    for k in range(T_train):
        A, Bk, lam = pencil(k)
        w, X, info, _ = collect.solve(A, Bk)
        if check:
            check(A, Bk, w, X, lam)
        sols.append((w, X))
    feats, targs = [], []
    for k in range(1, T_train - 1):
        feats.append(collect.features(sols[k][0], sols[k - 1][0], sols[k][1], sols[k - 1][1]).clone())
        tk = torch.empty(s + 1, device=dev, dtype=torch.float32)
        collect.targets(sols[k - 1][1], sols[k][1], sols[k + 1][1], tk[:s])
        collect.shift_target(sols[k - 1][0], sols[k][0], sols[k + 1][0], tk[s:])
        targs.append(tk)
    Xf, Tf = torch.stack(feats), torch.stack(targs)
    net = Mlp(3 * s + 1, s + 1, seed=seed, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    hist = net.train(Xf, Tf, iters, lr=lr)
    e1.record()
    torch.cuda.synchronize()
    runs["learned"].mlp = net
    # one untimed solve per method (problem T_train - 1 again) so that no
    # method's first-call set-up falls into its times
    A, Bk, _ = pencil(T_train - 1)
    for m in ("reuse", "learned"):
        runs[m].prev = [sols[-3], sols[-2]]
        runs[m].solve(A, Bk)
        runs[m].prev = [sols[-2], sols[-1]]
    stats = {m: [0, 0.0, 0] for m in runs}
    for k in range(T_train, T):
        A, Bk, lam = pencil(k)
        for m, r in runs.items():
            w, X, info, ms = r.solve(A, Bk)
            if check:
                check(A, Bk, w, X, lam)
            stats[m][0] += info["matvecs"]
            stats[m][1] += ms
            stats[m][2] += info["restarts"]
    return stats, hist, e0.elapsed_time(e1)
