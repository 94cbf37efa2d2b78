"""Time the CPU oracle once on the benchmark workload and on its bounded
sample, and record both in profiles/cpu_oracle.json.

The benchmark's CPU baseline (and its reference arm) times the oracle on the
leading n_sample x n_sample sub-pencil only, so that a run stays within a few
minutes, and scales that time to the full order with an exponent p.  This
script measures the full-size run once on the same host cores, so that p is
fitted rather than assumed:  p = log(t_full / t_sample) / log(n_full / n_sample).

    python oracle/time_full.py [--n 16384] [--s 100] [--sample-n 4096] [--reps 3]

Test infrastructure only, like the rest of oracle/.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pencil(n: int):
    """The benchmark pencil (seed 0) as numpy arrays; built on the GPU when
    there is one (input generation only), else on the host."""
    import torch

    import inputs

    dev = "cuda" if torch.cuda.is_available() else "cpu"
    A, B, lam = inputs.make_pencil(n, seed=0, device=dev)
    out = A.cpu().numpy(), B.cpu().numpy(), lam.cpu().numpy()
    del A, B
    if dev == "cuda":
        torch.cuda.empty_cache()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--s", type=int, default=100)
    ap.add_argument("--sample-n", type=int, default=4096)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=os.path.join(ROOT, "profiles", "cpu_oracle.json"))
    args = ap.parse_args(argv)
    import numpy as np

    import oracle

    # the sample exactly as the benchmark takes it: the leading sub-pencil of
    # an n_sample pencil, s scaled in proportion
    s_sample = max(1, round(args.s * args.sample_n / args.n))
    import inputs

    As, Bs, _ = (t.numpy() for t in inputs.make_pencil(args.sample_n, seed=0))
    ts = []
    for _ in range(args.reps):
        t0 = time.perf_counter()
        oracle.gsyeig(As, Bs, s_sample, vectors="invit")
        ts.append(time.perf_counter() - t0)
    t_sample = statistics.mean(ts)
    A, B, lam = pencil(args.n)
    t0 = time.perf_counter()
    w, X = oracle.gsyeig(A, B, args.s, vectors="invit")
    t_full = time.perf_counter() - t0
    rel = float(np.max(np.abs(w - lam[: args.s]) / np.abs(lam[: args.s])))
    p = math.log(t_full / t_sample) / math.log(args.n / args.sample_n)
    rec = {"n_full": args.n, "s_full": args.s, "seconds_full": t_full, "n_sample": args.sample_n,
           "s_sample": s_sample, "seconds_sample": t_sample, "seconds_sample_reps": ts, "exponent": p,
           "cores": oracle.num_threads(), "machine": platform.machine(),
           "max_rel_eig_err_vs_constructed": rel,
           "command": "python oracle/time_full.py " + " ".join(argv if argv is not None else sys.argv[1:])}
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    with open(args.out, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))
    return 0


if __name__ == "__main__":
    sys.exit(main())
