"""The learned warm start for a sequence of related pencils, at test size, on the GPU.

* The network's tensor-core forward and backward kernels against the CPU
  FP64 oracle (oracle/mlp.py, which rounds the same operands to bf16):
  outputs within 1e-3 of max|Y|, each gradient block within 1e-3 in
  relative Frobenius norm (the difference is the kernels' fp32
  accumulation); Adam within fp32 rounding.
* A sequence of related pencils: the network, trained on the GPU on the
  first problems' solutions, extrapolates the previous eigenvectors into
  the start of the next solve; every solve meets the 1e-10 gates, and the
  learned start needs fewer operator applications and less time than both
  a random start and plain reuse of the previous eigenvectors.
"""
import numpy as np
import pytest
import torch

import inputs
import oracle
from oracle import mlp as omlp
from tests import _checks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_6374_gb300 import warmstart

    return warmstart


@pytest.mark.parametrize("dims,batch", [((129, 256, 65), 150), ((7, 32, 3), 5), ((200, 144, 256), 256)])
def test_mlp_forward_and_gradient_match_oracle(ws_mod, dims, batch):
    n_in, H, n_out = dims
    net = ws_mod.Mlp(n_in, n_out, hidden=H, seed=3, batch_max=256)
    r = np.random.default_rng(batch)
    X = r.standard_normal((batch, n_in)).astype(np.float32)
    T = r.standard_normal((batch, n_out)).astype(np.float32)
    wo = r.uniform(0.5, 2.0, n_out).astype(np.float32)
    # random biases too (the initialiser zeroes them)
    p = net.params.cpu().numpy().astype(np.float64)
    off = [H * n_in, H, H * H, H, n_out * H, n_out]
    o = 0
    for i, sz in enumerate(off):
        if i % 2 == 1:
            p[o:o + sz] = r.uniform(-0.1, 0.1, sz)
        o += sz
    net.params.copy_(torch.from_numpy(p.astype(np.float32)))
    p = net.params.cpu().numpy().astype(np.float64)
    Xd, Td, wod = (torch.from_numpy(a).cuda() for a in (X, T, wo))
    Y = net.forward(Xd).cpu().numpy()
    Yo, _, _ = omlp.forward(p, X.astype(np.float64), n_in, H, n_out, bf16=True)
    assert np.abs(Y - Yo).max() <= 1e-3 * np.abs(Yo).max()
    loss, g = net.gradient(Xd, Td, wod)
    lo, go = omlp.loss_and_grad(p, X.astype(np.float64), T.astype(np.float64), n_in, H, n_out, wo, bf16=True)
    assert abs(loss - lo) <= 1e-4 * lo
    g = g.cpu().numpy().astype(np.float64)
    o = 0
    for sz in off:
        a, b = g[o:o + sz], go[o:o + sz]
        assert np.linalg.norm(a - b) <= 1e-3 * max(np.linalg.norm(b), 1e-30), (o, sz)
        o += sz


def test_mlp_adam_matches_oracle(ws_mod):
    net = ws_mod.Mlp(9, 3, hidden=16, seed=5)
    r = np.random.default_rng(0)
    p = net.params.cpu().numpy().astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for step in range(1, 4):
        g = r.standard_normal(p.size).astype(np.float32)
        net.grad.copy_(torch.from_numpy(g))
        net.adam_step(1e-2)
        p, m, v = omlp.adam(p, m, v, g.astype(np.float64), step, 1e-2)
    assert np.abs(net.params.cpu().numpy() - p).max() <= 1e-5


def test_mlp_training_fits_a_smooth_map(ws_mod):
    """Full-batch Adam on y = (sin(x0), x1 x2): the loss falls by 20x."""
    net = ws_mod.Mlp(3, 2, hidden=64, seed=1)
    r = np.random.default_rng(1)
    X = r.uniform(-1, 1, (200, 3)).astype(np.float32)
    T = np.stack([np.sin(2 * X[:, 0]), X[:, 1] * X[:, 2]], axis=1).astype(np.float32)
    hist = net.train(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), 400, lr=3e-3)
    assert hist[-1] <= hist[0] / 20, (hist[0], hist[-1])


def _gates(A, B, w, X, lam, cnorm=1000.0):
    """The 1e-10 gates of the direct route: relative eigenvalue error, with
    the floor of a backward-stable solve on C for the eigenvalues near zero
    (|d lambda| <= 1e-10 |lambda| + 1e-14 ||C||), backward error and
    B-orthonormality."""
    A, B, w, X, lam = (t.cpu().numpy() for t in (A, B, w, X, lam))
    lam = lam[:len(w)]
    assert np.all(np.abs(w - lam) <= 1e-10 * np.abs(lam) + 1e-14 * cnorm)
    assert _checks.eta(A, B, w, X).max() <= 1e-10
    assert _checks.b_orth_err(B, X) <= 1e-10


def test_learned_warm_start_beats_random_and_reuse(ws_mod):
    """n = 1024, s = 16, a 64-problem sequence (dt = 0.005): the network is
    trained on the plain solver's first 48 solutions and proposes the start
    blocks of the last 16.  Learned starts use fewer operator applications
    and less time than both the random start and reuse of the previous
    eigenvectors; every pair meets the 1e-10 gates."""
    seq = inputs.PencilSequence(1024, seed=11, device="cuda")
    stats, hist, _ = ws_mod.evaluate_sequence(seq.pencil, seq.B, 1024, 16, 64, 48, check=_gates)
    print({m: (v[0], round(v[1], 1), v[2]) for m, v in stats.items()})
    assert hist[-1] < 0.5 * hist[0]
    for other in ("reuse", "random"):
        assert stats["learned"][0] < stats[other][0], (other, stats)
        assert stats["learned"][1] < stats[other][1], (other, stats)


def test_single_vector_start_filter_and_early_tests():
    """The single-vector warm start (start vector F X0 w, Chebyshev filter,
    Ritz tests every 16 steps) gives the oracle's pairs, with fewer operator
    applications than a random start for a start block close to the wanted
    eigenvectors."""
    from paper_1111_6374_gb300 import Solver

    n, s = 700, 10
    A, B, lam = (t.numpy() for t in inputs.make_pencil(n, seed=41))
    w_or, X_or = oracle.gsyeig(A, B, s)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    Xs = torch.from_numpy(X_or + 1e-3 * np.random.default_rng(1).standard_normal(X_or.shape)).cuda()
    Xs = Xs.t().contiguous().t()
    wts = torch.ones(s, device="cuda", dtype=torch.float64)
    base = Solver(0, check_every=16)
    _, _, info_r = base.solve(dA, dB, s)
    sol = Solver(0, check_every=16, start_block=Xs, start_weights=wts, filter_degree=6,
                 filter_cut=float(lam[s + 3]), filter_edge=1100.0)
    w, X, info = sol.solve(dA, dB, s)
    assert info["filter_matvecs"] == 6
    _gates(dA, dB, w, X, torch.from_numpy(w_or))
    assert info["matvecs"] < info_r["matvecs"]
