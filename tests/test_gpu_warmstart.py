"""The learned warm start (configs[4]'s form at test size) on the GPU.

* The network's tensor-core forward and backward kernels against the CPU
  FP64 oracle (oracle/mlp.py, which rounds the same operands to bf16):
  outputs within 1e-3 of max|Y|, each gradient block within 1e-3 in
  relative Frobenius norm (the difference is the kernels' fp32
  accumulation); Adam within fp32 rounding.
* A sequence of related pencils: the network, trained on the GPU on the
  first problems' solutions, proposes start blocks and filter cuts for the
  later ones; every solve meets the 1e-10 gates, and the learned start
  needs fewer operator applications and less time than both a random start
  and plain reuse of the previous eigenvectors.
"""
import numpy as np
import pytest
import torch

import inputs
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
    assert np.all(np.abs(w - lam) <= 1e-10 * np.abs(lam) + 1e-14 * cnorm)
    assert _checks.eta(A, B, w, X).max() <= 1e-10
    assert _checks.b_orth_err(B, X) <= 1e-10


def test_learned_warm_start_beats_random_and_reuse(ws_mod):
    """n = 1024, s = 16, a 64-problem sequence (dt = 0.005): the network is
    trained on the plain solver's first 48 solutions and then proposes the
    starts of the last 16.  Learned starts use fewer operator applications
    (filter included) and less time than both a random start and reuse of
    the previous eigenvectors; every pair meets the 1e-10 gates."""
    torch.manual_seed(0)
    n, s, T, T_train = 1024, 16, 64, 48
    seq = inputs.PencilSequence(n, seed=11, device="cuda")
    runs = {m: ws_mod.SequenceSolver(s, m) for m in ("random", "reuse", "learned")}
    # phase 1: plain solves of the training problems, features and targets
    collect = runs["random"]
    sols = []
    for k in range(T_train):
        A, B, lam = seq.pencil(k)
        w, X, info, _ = collect.solve(A, B)
        _gates(A, B, w, X, lam[:s])
        sols.append((w, X))
    feats, targs = [], []
    tgt = torch.empty(s + 1, device="cuda", dtype=torch.float32)
    for k in range(1, T_train - 1):
        f, scal = collect.features(sols[k][0], sols[k - 1][0], out=torch.empty(2 * s + 1, device="cuda"),
                                   scal=torch.empty(2, device="cuda", dtype=torch.float64))
        P = collect.overlaps(sols[k + 1][1], sols[k][1], seq.B)
        collect.targets(sols[k + 1][0], scal, P, tgt)
        feats.append(f.clone())
        targs.append(tgt.clone())
    Xf, Tf = torch.stack(feats), torch.stack(targs)
    net = ws_mod.Mlp(2 * s + 1, s + 1, seed=0)
    outw = torch.full((s + 1,), 1.0, device="cuda")
    outw[0] = 4.0
    hist = net.train(Xf, Tf, 1500, lr=1e-3, out_weights=outw)
    assert hist[-1] < 0.2 * hist[0]
    runs["learned"].mlp = net
    # phase 2: the three methods on the remaining problems, each from its own
    # previous solutions (seeded with the last two training solutions)
    for m in ("reuse", "learned"):
        for k in (T_train - 2, T_train - 1):
            A, B, _ = seq.pencil(k)
            runs[m].solve(A, B)
    stats = {m: [0, 0.0, 0] for m in runs}
    for k in range(T_train, T):
        A, B, lam = seq.pencil(k)
        for m, r in runs.items():
            w, X, info, ms = r.solve(A, B)
            _gates(A, B, w, X, lam[:s])
            stats[m][0] += info["matvecs"]
            stats[m][1] += ms
            stats[m][2] += info["fallback"]
    print({m: (v[0], round(v[1], 1), v[2]) for m, v in stats.items()})
    assert stats["learned"][0] < stats["reuse"][0] < stats["random"][0]
    assert stats["learned"][1] < stats["reuse"][1] and stats["learned"][1] < stats["random"][1]
