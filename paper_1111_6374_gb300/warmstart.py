"""Learned warm start for sequences of related problems (binding and driver).

The paper's Section 3 motivates sequences of related eigenproblems (each
self-consistency cycle of a DFT code solves dozens).  Here a small MLP,
trained on the GPU by the library's own forward and backward kernels
(``gsyeig_mlp_*``: bf16 tcgen05 products, fp32 parameters and Adam), reads
a solved problem's Ritz values and the parameter step and proposes, for the
next problem, the weights of a start block built from the previous
eigenvectors and the cut of a Chebyshev filter applied to it
(``gsyeig_opts.start_block / start_weights / filter_*``).  The solver's
residual test alone decides acceptance; a random start is the fallback
when a proposal does not converge.

This module only sequences library calls: features, targets and the
decoding of the network's outputs run in the library's kernels
(``gsyeig_ws_features / _targets / _decode``), and torch supplies device
memory.
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
    """Solves a sequence of pencils (A_k, B) for the s smallest eigenpairs,
    starting each solve from the previous solution in one of three ways:

    * ``"random"``: the counter-based random start (no reuse);
    * ``"reuse"``: the start vector U (sum_j x_j) from the previous
      eigenvectors, no filter (the unlearned control);
    * ``"learned"``: weights and a filter cut proposed by the network from
      the previous two problems' Ritz values.

    Every method tests convergence every ``check_every`` steps."""

    def __init__(self, s: int, method: str, mlp: Mlp | None = None, check_every: int = 16, filter_degree: int = 8,
                 margin: float = 2.0, wmin: float = 0.05, dt_rel: float = 1.0, device=0, **opts):
        assert method in ("random", "reuse", "learned")
        self.s, self.method, self.mlp = s, method, mlp
        self.check_every, self.degree, self.margin, self.wmin, self.dt_rel = (check_every, filter_degree, margin,
                                                                              wmin, dt_rel)
        self.solver = Solver(device, check_every=check_every, **opts)
        self.lib = self.solver.lib
        self.prev = []  # (w, X, info) of the last two solves
        dev = torch.device("cuda", device)
        self.dev = dev
        self.feat = torch.empty(2 * s + 1, device=dev, dtype=torch.float32)
        self.scal = torch.empty(2, device=dev, dtype=torch.float64)
        self.weights = torch.empty(s, device=dev, dtype=torch.float64)
        self.cut = torch.empty(1, device=dev, dtype=torch.float64)

    def features(self, w, w_prev, out=None, scal=None):
        out = self.feat if out is None else out
        scal = self.scal if scal is None else scal
        st = self.lib.gsyeig_ws_features(self.s, _p(w), _p(w_prev), self.dt_rel, _p(out), _p(scal), _stream(self.dev))
        if st != 0:
            raise GsyeigError(st, "ws_features")
        return out, scal

    def solve(self, A: torch.Tensor, B: torch.Tensor):
        """One solve of the sequence (A and B are not modified).  Returns
        (w, X, info, ms); info["fallback"] is 1 when a proposal did not
        converge and the random start took over."""
        s, sol = self.s, self.solver
        opts = dict(start_block=None, start_weights=None, filter_degree=0, filter_cut=0.0, filter_edge=0.0)
        if self.method != "random" and self.prev:
            opts["start_block"] = self.prev[-1][1]
        if self.method == "learned" and len(self.prev) >= 2:
            feat, scal = self.features(self.prev[-1][0], self.prev[-2][0])
            out = self.mlp.forward(feat.unsqueeze(0))
            st = self.lib.gsyeig_ws_decode(s, _p(out), _p(scal), self.margin, self.wmin, _p(self.weights),
                                           _p(self.cut), _stream(self.dev))
            if st != 0:
                raise GsyeigError(st, "ws_decode")
            opts.update(start_weights=self.weights, filter_degree=self.degree, filter_cut=float(self.cut.item()),
                        filter_edge=float(self.prev[-1][2]["tnorm"]))
        sol.set_options(**opts)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        w, X, info = sol.solve(A, B, s, allow_unconverged=True)
        fallback = 0
        if info["status"] != 0 and opts["start_block"] is not None:
            # the proposal did not converge: random start (the residual test decides)
            sol.set_options(start_block=None, start_weights=None, filter_degree=0)
            m0 = info["matvecs"]
            w, X, info = sol.solve(A, B, s)
            info["matvecs"] += m0
            fallback = 1
        e1.record()
        torch.cuda.synchronize()
        info["fallback"] = fallback
        self.prev = (self.prev + [(w, X, info)])[-2:]
        return w, X, info, e0.elapsed_time(e1)

    def overlaps(self, X_next, X, B):
        """P = X_next^T B X (s x s) on the library's GEMM engine (B symmetric:
        its transpose is the same matrix, in column-major storage)."""
        BX = self.solver.gemm(B.t(), X)
        return self.solver.gemm(X_next, BX, transA=True)

    def targets(self, w_next, scal, P, out):
        st = self.lib.gsyeig_ws_targets(self.s, _p(w_next), _p(scal), _p(P), P.stride(1), _p(out), _stream(self.dev))
        if st != 0:
            raise GsyeigError(st, "ws_targets")
        return out
