"""Batches of independent problems of uneven order (a smaller form of the 64-problem benchmark):
gsyeig_solve_batched against the oracle and against one-by-one solves.

Every problem of a batch of uneven orders meets the 1e-10 gates against
the CPU oracle; the batched results agree with the sequential gsyeig_solve
results; the autotuner's panel width is one of its candidates."""
import numpy as np
import pytest
import torch

import inputs
import oracle
from tests import _checks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_6374_gb300 import Solver

    return Solver(0)


def test_batched_problems_match_oracle_and_sequential(solver):
    rng = np.random.default_rng(7)
    ns = [int(x) for x in rng.choice(np.arange(512, 1537, 64), 10)] + [512, 1536]
    s = 8
    host = [inputs.make_pencil(n, seed=1000 + i) for i, n in enumerate(ns)]
    pencils = [(A.cuda(), B.cuda()) for A, B, _ in host]
    res = solver.solve_batched(pencils, s, streams=4)
    assert all(r[2]["status"] == 0 for r in res)
    for i, ((A, B, lam), (w, X, info), n) in enumerate(zip(host, res, ns)):
        An, Bn = A.numpy(), B.numpy()
        w, X = w.cpu().numpy(), X.cpu().numpy()
        w_or, X_or = oracle.gsyeig(An, Bn, s)
        assert np.all(np.abs(w - w_or) <= 1e-10 * np.abs(w_or) + 1e-14 * lam.max().item()), n
        assert _checks.eta(An, Bn, w, X).max() <= 1e-10
        assert _checks.b_orth_err(Bn, X) <= 1e-10
        w1, X1, _ = solver.solve(pencils[i][0], pencils[i][1], s)
        assert np.abs(w - w1.cpu().numpy()).max() <= 1e-10 * np.abs(w_or).max()
    for n in (512, 1536):
        assert solver.autotuned_block(n) in (64, 128)


def test_batched_graph_replay_matches_plain_cycles(solver):
    """opts.graph: the Lanczos cycles replayed from CUDA graphs give the same
    pairs as the plain launches, over restarts (the restart cycle is a
    second graph) and over repeated solves (cache hits)."""
    from paper_1111_6374_gb300 import Solver

    A, B, lam = inputs.make_pencil(700, seed=12)
    g = Solver(0, graph=1)
    p = Solver(0)
    for _ in range(2):
        wg, Xg, ig = g.solve(A.cuda(), B.cuda(), 20)
        wp, Xp, ip = p.solve(A.cuda(), B.cuda(), 20)
        assert ig["restarts"] == ip["restarts"] > 0
        assert torch.equal(wg, wp) and torch.equal(Xg, Xp)
