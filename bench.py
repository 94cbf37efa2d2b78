"""Benchmark: time-to-solution of s generalized eigenpairs (A X = B X Lambda)
through the KE route on one GB300, plus roofline and CPU-oracle baseline.

Workload (default): n = 16384, s = 100 smallest, float64, synthetic pencil
A = U^T Q diag(lambda) Q^T U, B = G G^T / n + I, lambda ~ U(0, 1000) (the
stand-in for the paper's n ~ 10^4 molecular-dynamics / DFT pencils).

One step = one full gsyeig_solve (potrf, sygst, Lanczos with restarts, Ritz
vectors, back-transform) on inputs already resident in HBM; A and B are
restored from pristine device copies between steps, outside the timed
interval.  Inputs (2 x 2.1 GB) are far larger than the 129 MB L2.

Route (--route): by default the solve takes the paper's own route for the
smallest eigenpairs of a pencil whose A is positive definite too (Section
3.1): the largest eigenpairs of the inverse problem B X = A X Lambda^-1.  The
direct route (smallest eigenvalues of C = U^-T A U^-1) is timed on the same
pencil afterwards and reported under "other_route".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun) runs independent replicas, one problem per GPU, no
collective on the data path; the reported time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-solution for s gen. eigenpairs @rel. residual ≤1e-10"
HBM_GBS = 6797.9
BF16_TFLOPS = 1906.4
FP64_OVER_BF16_NOMINAL = 1.25 / 2250.0  # GB300 nominal dense FP64 / bf16
ROUTES = {"inverse": "KE on the inverse problem B X = A X Lambda^-1 (A = L^T L, largest mu = 1/lambda of "
                     "L^-T B L^-1), as the paper does for its smallest-eigenpair workload (Section 3.1)",
          "direct": "KE on C = U^-T A U^-1 (B = U^T U), smallest eigenvalues"}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, backend):
    import torch.distributed as dist

    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29511")
        dist.init_process_group(backend=backend)
    return dist


def max_over_ranks(value: float, ws: int, device=None) -> float:
    """Max of a float over ranks (identity when ws == 1)."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(os.environ.get("GSYEIG_CLOCKS_DIR", tempfile.gettempdir()), f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def kernel_traffic(kernel: str, n: int):
    """DRAM bytes per launch of `kernel` at order n, from the committed ncu
    summary (profiles/traffic.json), if it was taken on the current source of
    that kernel; a smaller captured case is scaled by the units it processes
    (n^2 for the operator tiles)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except OSError:
        return None
    e = d.get(kernel)
    if not e:
        return None
    src = os.path.join(ROOT, e["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if h != e.get("source_sha256_16"):
        return None
    scale = (n / e["n"]) ** 2 if e.get("scales_with") == "n^2" else 1.0
    return {"dram_bytes": e["dram_bytes_per_launch"] * scale,
            "note": f"ncu capture at n={e['n']} ({e['dram_bytes_per_launch']:.4g} B), scaled by {e.get('scales_with', '1')}"}


def oracle_exponent(n_full: int, n_sample: int):
    """Growth exponent p of the oracle's time, t(n_full) = t(n_sample)
    (n_full / n_sample)^p, fitted from the committed full-size timing
    (profiles/cpu_oracle.json: one run at n_full and runs at n_sample on the
    same host cores); p = 3 (every oracle stage is O(n^3)) if that record is
    absent or for other sizes."""
    try:
        with open(os.path.join(ROOT, "profiles", "cpu_oracle.json")) as f:
            d = json.load(f)
        if d["n_full"] == n_full and d["n_sample"] == n_sample:
            import math

            p = math.log(d["seconds_full"] / d["seconds_sample"]) / math.log(n_full / n_sample)
            return p, (f"fitted from one oracle run at n={n_full} ({d['seconds_full']:.0f} s) and n={n_sample} "
                       f"({d['seconds_sample']:.2f} s) on {d['cores']} cores (profiles/cpu_oracle.json)")
    except (OSError, KeyError, ValueError, ZeroDivisionError):
        pass
    return 3.0, "assumed (every oracle stage is O(n^3)); no committed full-size timing for this size"


def cpu_oracle_sample(n_full: int, s_full: int, n_sample: int):
    """Time the oracle on the leading n_sample x n_sample sub-pencil and
    scale by (n_full / n_sample)^p, p from oracle_exponent (the value is an
    extrapolation and says so)."""
    import inputs
    import oracle

    s = max(1, round(s_full * n_sample / n_full))
    A, B, _ = (t.numpy() for t in inputs.make_pencil(n_sample, seed=0))
    t0 = time.perf_counter()
    oracle.gsyeig(A, B, s, vectors="invit")
    dt = time.perf_counter() - t0
    p, how = oracle_exponent(n_full, n_sample)
    scale = (n_full / n_sample) ** p
    return {"value": dt * scale, "unit": "s", "cores": oracle.num_threads(), "kind": "oracle",
            "extrapolated": n_sample != n_full, "exponent": p, "exponent_source": how, "sample_seconds": dt,
            "sample": f"oracle on the leading {n_sample}x{n_sample} sub-pencil (s={s}), {dt:.2f} s measured, "
                      f"scaled by (n/{n_sample})^{p:.3f} = {scale:.1f}"}


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    n_sample = args.cpu_sample_n
    vals = []
    for _ in range(args.warmup):
        cpu_oracle_sample(args.n, args.s, n_sample)
    for _ in range(args.steps):
        vals.append(cpu_oracle_sample(args.n, args.s, n_sample))
    v = statistics.mean(x["value"] for x in vals)
    sample_ms = statistics.mean(x["sample_seconds"] for x in vals) * 1e3
    # each timed step is one oracle run on the bounded sample: ms_per_step is
    # that measured time; value is the time-to-solution at the configured n,
    # extrapolated from it with the exponent stated
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sample_ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "extrapolated": vals[0]["extrapolated"],
            "config": {"workload": args.workload, "n": args.n, "s": args.s, "which": "smallest",
                       "sample_n": n_sample},
            "cpu_baseline": {"value": v, "unit": "s", "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"], "extrapolated": vals[0]["extrapolated"],
                             "exponent": vals[0]["exponent"], "exponent_source": vals[0]["exponent_source"]},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, ws, rank, local):
    import torch

    if not torch.cuda.is_available():
        print(json.dumps({"error": "bench.py needs a CUDA GPU"}), flush=True)
        return 2
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    init_dist(ws, "nccl")
    import inputs
    from paper_1111_6374_gb300 import Solver, kernel_launches

    n, s = args.n, args.s
    if args.gen_device == "cpu":  # e.g. under a profiler that cannot load torch's CUDA linear algebra
        A0, B0, lam = (t.to(dev) for t in inputs.make_pencil(n, seed=args.seed + rank))
    else:
        A0, B0, lam = inputs.make_pencil(n, seed=args.seed + rank, device=dev)
    A = torch.empty_like(A0)
    B = torch.empty_like(B0)
    solver = Solver(local, inverse=1 if args.route == "inverse" else 0, block=args.block, graph=args.graph,
                    check_every=args.check_every)
    stream = torch.cuda.current_stream(dev)

    def restore():
        A.copy_(A0)
        B.copy_(B0)

    def timed(sol, steps, warmup, profile=False):
        """Time `steps` solves; profile=True also records CUDA events around
        every kernel class (for the breakdown; the events cost time)."""
        for _ in range(warmup):
            restore()
            sol.solve(A, B, s, overwrite=True)
        torch.cuda.synchronize()
        sol.set_options(profile=1 if profile else 0)
        times, infos = [], []
        for _ in range(steps):
            restore()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            w, X, info = sol.solve(A, B, s, overwrite=True)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(info)
        sol.set_options(profile=0)
        return w, X, times, infos

    for _ in range(args.warmup):
        restore()
        w, X, info = solver.solve(A, B, s, overwrite=True)
    torch.cuda.synchronize()
    l_before = kernel_launches()
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        w, X, times, _ = timed(solver, args.steps, 0)
    torch.cuda.synchronize()
    barrier(ws)
    launches = (kernel_launches() - l_before) // max(1, args.steps)
    ms = statistics.mean(times)
    ms_all = max_over_ranks(ms, ws, dev)
    # one more step with CUDA events around every kernel class: the breakdown
    # and the roofline of the dominant kernel (event times of that step)
    _, _, ptimes, infos = timed(solver, 1, 0, profile=True)
    ms_prof = ptimes[0]

    # accuracy of the last timed solve against the constructed spectrum and (A, B)
    rel = float(((w - lam[:s]).abs() / lam[:s].abs()).max())
    R = A0 @ X - (B0 @ X) * w
    nA = _power(A0)
    nB = _power(B0)
    eta = float((R.norm(dim=0) / ((nA + w.abs() * nB) * X.norm(dim=0))).max())
    orth = float((X.T @ (B0 @ X) - torch.eye(s, device=dev, dtype=X.dtype)).abs().max())

    # end to end: host buffers through the same C-ABI call, copies inside the timed interval
    e2e = None
    if not args.no_e2e:
        Ah = A0.cpu().pin_memory()
        Bh = B0.cpu().pin_memory()
        solver.solve(Ah, Bh, s)  # warm the staging buffers
        e2e_times = []
        for _ in range(max(1, min(args.steps, args.e2e_steps))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            wh, Xh, _ = solver.solve(Ah, Bh, s)
            e2e_times.append(time.perf_counter() - t0)
        e2e = statistics.mean(e2e_times)
        e2e = max_over_ranks(e2e, ws, dev)

    # the other route on the same pencil, for comparison (fewer steps)
    other = None
    if not args.no_other_route:
        osol = Solver(local, inverse=0 if args.route == "inverse" else 1)
        _, _, ot, oi = timed(osol, max(1, min(args.steps, 2)), 1, profile=True)
        oi = oi[-1]
        other = {"route": "direct" if args.route == "inverse" else "inverse", "inverse_used": oi["inverse"],
                 "ms_per_step": max_over_ranks(statistics.mean(ot), ws, dev), "steps": len(ot),
                 "stages_ms": {k: oi[k] for k in ("ms_gs1", "ms_gs2", "ms_ke", "ms_ke3", "ms_bt1", "ms_total")},
                 "matvecs": oi["matvecs"], "restarts": oi["restarts"], "ms_symv": oi["symv_ms"],
                 "ms_orth": oi["orth_ms"]}
        osol.close()

    def one_solve(**opts):
        """One profiled solve of the benchmark pencil with other options (no warm-up)."""
        sol = Solver(local, **opts)
        _, _, t, i = timed(sol, 1, 0, profile=True)
        i = i[-1]
        sol.close()
        return {"ms_per_step": max_over_ranks(t[0], ws, dev), "steps": 1, "options": opts,
                "inverse_used": i["inverse"], "matvecs": i["matvecs"], "restarts": i["restarts"],
                "stages_ms": {k: i[k] for k in ("ms_gs1", "ms_gs2", "ms_ke", "ms_ke3", "ms_bt1", "ms_total")}}

    # variant KI (C never formed, U^-1 applied by triangular products)
    ki = None if args.no_extra else one_solve(inverse=1 if args.route == "inverse" else 0, implicit=1)
    # the same route in plain FP64 arithmetic (FP64 FMA GEMMs and symv)
    plain = None if args.no_extra else one_solve(inverse=1 if args.route == "inverse" else 0, fp64_gemm=1,
                                                  fp64_symv=1)
    # library comparison on the same GPU: cuSOLVER through torch.linalg
    # (Cholesky, two triangular solves, a full symmetric eigensolver)
    library = None if args.no_extra else _library_point(A0, B0, s, lam)

    if rank != 0:
        return 0
    peaks, src = load_peaks()
    hbm = peaks.get("hbm_gbs", HBM_GBS)
    bf16 = peaks.get("bf16_tflops", BF16_TFLOPS)
    nst = len(infos)
    g_ms = sum(i["gemm_ms"] for i in infos) / nst
    g_fl = sum(i["gemm_flops"] for i in infos) / nst
    g_n = sum(i["gemm_launches"] for i in infos) / nst
    c_ms = sum(i["gemm_core_ms"] for i in infos) / nst
    c_fl = sum(i["gemm_core_flops"] for i in infos) / nst
    c_n = sum(i["gemm_core_launches"] for i in infos) / nst
    s_ms = sum(i["symv_ms"] for i in infos) / nst
    s_fl = sum(i["symv_flops"] for i in infos) / nst
    s_by = sum(i["symv_bytes"] for i in infos) / nst
    s_n = sum(i["symv_launches"] for i in infos) / nst
    sliced = solver.opts.fp64_gemm != 1
    # GEMM engine of gs1/gs2/bt1: FP64-equivalent rate; on the tensor path the
    # algorithmic tensor work is 28 bf16 digit-pair products per FP64 product
    g_fp64eq = g_fl / (g_ms * 1e-3) / 1e12 if g_ms > 0 else 0.0
    core = None
    if sliced:
        gemm = {"kernel": "GEMM engine calls (k_sliced_umma + the kernels slicing FP64 operands into bf16 digits)",
                "bound": "tensor", "achieved": 28 * g_fp64eq, "peak": bf16, "unit": "TFLOP/s",
                "frac": 28 * g_fp64eq / bf16, "fp64_equivalent_tflops": g_fp64eq,
                "peak_source": f"{src} bf16 (MEASURED_PEAKS.json)"}
        if c_ms > 0 and solver.opts.fp64_gemm == 0:
            c_eq = c_fl / (c_ms * 1e-3) / 1e12
            core = {"kernel": "k_sliced_umma: the tcgen05 kernel alone (28 bf16 digit products per FP64 product)",
                    "bound": "tensor", "achieved": 28 * c_eq, "peak": bf16, "unit": "TFLOP/s",
                    "frac": 28 * c_eq / bf16, "fp64_equivalent_tflops": c_eq,
                    "peak_source": f"{src} bf16 burst (MEASURED_PEAKS.json)",
                    "launches_per_step": c_n, "ms_per_step": c_ms, "share_of_step": c_ms / ms_prof,
                    "ms_per_launch": c_ms / max(1.0, c_n),
                    "algorithmic_flops_per_launch": 28 * c_fl / max(1.0, c_n),
                    "slicing_ms_per_step": g_ms - c_ms}
    else:
        fp64_peak = bf16 * FP64_OVER_BF16_NOMINAL
        gemm = {"kernel": "k_dgemm: FP64 FMA GEMM of gs1/gs2/bt1", "bound": "alu", "achieved": g_fp64eq,
                "peak": fp64_peak, "unit": "TFLOP/s", "frac": g_fp64eq / fp64_peak,
                "peak_source": f"{src} bf16 x nominal FP64/bf16 1.25/2250"}
    gemm.update({"launches_per_step": g_n, "ms_per_step": g_ms, "share_of_step": g_ms / ms_prof})
    df = solver.opts.fp64_symv == 0
    sym_gbs = s_by / (s_ms * 1e-3) / 1e9 if s_ms > 0 else 0.0
    symv = {"kernel": "k_symv_df (+ split, reduce): ke1 on fp32 hi/lo triangle tiles" if df else
            "k_symv_cols_v2: ke1 in FP64", "bound": "hbm", "achieved": sym_gbs, "peak": hbm, "unit": "GB/s",
            "frac": sym_gbs / hbm, "peak_source": f"{src} HBM copy (MEASURED_PEAKS.json)",
            "algorithmic_bytes_per_launch": s_by / max(1, s_n), "launches_per_step": s_n,
            "ms_per_launch": s_ms / max(1, s_n), "fp64_equivalent_tflops": s_fl / (s_ms * 1e-3) / 1e12 if s_ms else 0.0,
            "share_of_step": s_ms / ms_prof}
    for k, name in ((core, "k_sliced_umma"), (symv, "k_symv_df" if df else "k_symv_cols_v2")):
        if k is None:
            continue
        tr = kernel_traffic(name, n)
        k["traffic"] = tr["dram_bytes"] if tr else None
        k["traffic_note"] = tr["note"] if tr else "no ncu capture of the current source"
    dominant = core if core is not None else gemm
    roof = symv if symv["share_of_step"] >= dominant["share_of_step"] else dominant
    last = infos[-1]
    acc_ok = bool(rel <= 1e-10 and eta <= 1e-10 and orth <= 1e-10)
    line = {
        "metric": METRIC, "value": ms_all / 1e3, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "s": s, "which": "smallest", "route": ROUTES[args.route],
                   "inverse_used": last["inverse"], "krylov_dim": last["krylov_dim"], "graph": args.graph,
                   "check_every": args.check_every,
                   "keep": last["keep"], "tol": 1e-12, "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (2 x %.1f GB vs 129 MB)" % (n * n * 8 / 1e9)},
        "stages_ms": {k: last[k] for k in ("ms_gs1", "ms_gs2", "ms_ke", "ms_ke3", "ms_bt1", "ms_total")},
        "lanczos": {"matvecs": last["matvecs"], "restarts": last["restarts"], "nconv": last["nconv"],
                    "ms_symv": last["symv_ms"], "ms_orth": last["orth_ms"], "ms_restart": last["restart_ms"],
                    "ms_ritz": last["ritz_ms"]},
        # live per-class CUDA-event times of one step (the library stream, profile = 1)
        "profiled_step_ms": ms_prof,
        "classes_ms_per_step": {"gemm_core (k_sliced_umma)": c_ms,
                                "gemm_slicing_kernels": sum(i["slice_ms"] for i in infos) / nst,
                                "gemm_calls_other (launch gaps, copies)": g_ms - c_ms - sum(i["slice_ms"] for i in infos) / nst,
                                "diag_blocks (k_chol_sub, k_chol_panel, k_chol_update, k_trtri_cols)": sum(i["diag_ms"] for i in infos) / nst,
                                "symv (ke1)": s_ms, "orth (CGS2 + normalise)": sum(i["orth_ms"] for i in infos) / nst,
                                "ritz": sum(i["ritz_ms"] for i in infos) / nst,
                                "restart": sum(i["restart_ms"] for i in infos) / nst},
        "accuracy": {"max_rel_eig_err_vs_constructed": rel, "max_eta": eta, "orth_err": orth},
        "accuracy_ok": acc_ok,
        "roofline": roof, "kernels": {"gemm_core": core, "gemm_engine": gemm, "symv": symv},
        "e2e": ({"value": e2e, "unit": "s", "h2d_bytes_per_step": 2 * n * n * 8, "d2h_bytes_per_step": (n * s + s) * 8}
                if e2e is not None else None),
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "other_route": other,
        "variant_ki": ki,
        "plain_fp64": plain,
        "library_cusolver": library,
    }
    if args.gpus == 1 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample(n, s, args.cpu_sample_n)
    print(json.dumps(line), flush=True)
    # a time that does not meet the accuracy the metric is quoted at is not a result
    return 0 if acc_ok else 3



# ---- the three extensions of the route, each against the plain path ----------
#
# `--next mixed|batched|warm` runs one of them instead of the headline and
# prints one JSON line with its own metric; the timed region of each is
# stated in the line.


def _accuracy(A, B, w, X, lam, lam_max):
    """Relative eigenvalue error against the constructed spectrum, backward
    error eta and B-orthonormality (device tensors).  The eigenvalue gate
    is |d lambda| <= 1e-10 |lambda| + 1e-14 max|lambda|: the pencil itself is
    formed in FP64, so an eigenvalue near zero is known only to about
    eps ||A|| (the floor of any backward-stable solve)."""
    import torch

    d = (w - lam).abs()
    rel = float((d / lam.abs()).max())
    gate = float((d / (1e-10 * lam.abs() + 1e-14 * lam_max)).max())
    R = A @ X - (B @ X) * w
    eta = float((R.norm(dim=0) / ((_power(A) + w.abs() * _power(B)) * X.norm(dim=0))).max())
    orth = float((X.T @ (B @ X) - torch.eye(X.shape[1], device=X.device, dtype=X.dtype)).abs().max())
    return {"max_rel_eig_err_vs_constructed": rel, "eig_gate_ratio": gate, "max_eta": eta, "orth_err": orth,
            "ok": bool(gate <= 1.0 and eta <= 1e-10 and orth <= 1e-10)}


def _event_time(fn, stream):
    import torch

    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def next_mixed(args, dev):
    """Mixed precision against plain FP64 on one structured pencil (order
    args.n, default 65536, s = 256 smallest, inverse route): warm-up solves,
    then one timed solve each, inputs restored between solves outside the
    timed interval.  The operator's inputs (2 x 34 GB at n = 65536) are far
    larger than L2."""
    import torch

    import inputs
    from paper_1111_6374_gb300 import Solver

    n, s = args.n, args.s
    t0 = time.perf_counter()
    A0, B0, lam = inputs.make_pencil_structured(n, seed=args.seed, device=dev)
    gen_s = time.perf_counter() - t0
    A, B = torch.empty_like(A0), torch.empty_like(B0)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for name, opts in (("mixed", dict(mixed=1)), ("mixed_block_refinement", dict(mixed=2)),
                       ("plain_fp64_route", dict(mixed=0))):
        sol = Solver(dev.index, inverse=1, **opts)
        for _ in range(args.warmup):
            A.copy_(A0)
            B.copy_(B0)
            sol.solve(A, B, s, overwrite=True)
        ts, info = [], None
        for _ in range(args.steps):
            A.copy_(A0)
            B.copy_(B0)
            ms, (w, X, info) = _event_time(lambda: sol.solve(A, B, s, overwrite=True), stream)
            ts.append(ms)
        acc = _accuracy(A0, B0, w, X, lam[:s], float(lam.abs().max()))
        out[name] = {"ms_per_step": statistics.mean(ts), "steps": len(ts), "accuracy": acc,
                     "stages_ms": {k: info[k] for k in ("ms_gs1", "ms_gs2", "ms_ke", "ms_ke3", "ms_bt1", "ms_total")},
                     "matvecs": info["matvecs"], "restarts": info["restarts"]}
        if name.startswith("mixed"):
            out[name].update({k: info[k] for k in ("block_steps", "refine_iters", "ms_block_lanczos", "ms_refine",
                                                    "refine_fallback", "breakdowns")})
        if name == "mixed":
            # one more solve with CUDA events around every kernel class
            A.copy_(A0)
            B.copy_(B0)
            sol.set_options(profile=1)
            _, _, pi = sol.solve(A, B, s, overwrite=True)
            sol.set_options(profile=0)
            out[name]["profiled_classes_ms"] = {
                "symm32 (fp32 block operator)": pi["symm32_ms"], "symv (double-float operator)": pi["symv_ms"],
                "orth (FP64 CGS2 of both stages)": pi["orth_ms"], "gemm engine": pi["gemm_ms"],
                "ritz": pi["ritz_ms"], "restart": pi["restart_ms"], "symm32_launches": pi["symm32_launches"]}
        if name == "mixed":
            w_mixed = w
        else:
            out[name]["eig_diff_vs_mixed"] = float(((w - w_mixed).abs() / w.abs()).max())
        del w, X
        sol.close()
        torch.cuda.empty_cache()
    m, p = out["mixed"], out["plain_fp64_route"]
    return {"leg": "mixed", "metric": METRIC, "value": m["ms_per_step"] / 1e3, "unit": "s",
            "higher_is_better": False, "dtype": "f32 operator, f64 elsewhere", "data": "synthetic",
            "config": {"workload": f"gsyeig n={n} s={s} smallest, structured known-spectrum pencil "
                                   f"(16 reflectors, banded U), mixed precision vs plain FP64 route",
                       "n": n, "s": s, "route": ROUTES["inverse"], "generate_s": gen_s,
                       "l2": "inputs larger than L2"},
            "speedup_vs_plain": p["ms_per_step"] / m["ms_per_step"], "mixed": m, "plain": p,
            "mixed_block_refinement": out["mixed_block_refinement"],
            "accuracy_ok": all(out[k]["accuracy"]["ok"] for k in out)}


def next_batched(args, dev):
    """64 independent problems, n uniform over the multiples of 64 in
    [512, 4096], s = 16 smallest, seeds 1000 + i: one gsyeig_solve_batched
    call (graph-captured Lanczos cycles, autotuned panel width, 8 streams)
    against the same 64 problems solved one after another by the plain
    solver, both on the inverse route.  Each timed region covers all 64 solves; inputs are restored
    outside it."""
    import numpy as np
    import torch

    import inputs
    from paper_1111_6374_gb300 import Solver

    count, s = args.batch, 16
    rng = np.random.default_rng(args.seed)
    ns = [int(x) for x in rng.choice(np.arange(512, 4097, 64), count)]
    pristine = [inputs.make_pencil(n, seed=1000 + i, device=dev) for i, n in enumerate(ns)]
    work = [(torch.empty_like(A), torch.empty_like(B)) for A, B, _ in pristine]
    stream = torch.cuda.current_stream(dev)

    def restore():
        for (A0, B0, _), (A, B) in zip(pristine, work):
            A.copy_(A0)
            B.copy_(B0)

    # the inverse route for both (every pencil here has A positive definite):
    # its smallest lambda = 1/mu are resolved to 1e-10 relative
    bsol = Solver(dev.index, graph=1, inverse=1)
    psol = Solver(dev.index, inverse=1)
    t0 = time.perf_counter()
    tuned = {n: bsol.autotuned_block(n) for n in sorted(set(ns))}
    tune_s = time.perf_counter() - t0
    bt, pt = [], []
    for it in range(args.warmup + args.steps):
        restore()
        ms, res = _event_time(lambda: bsol.solve_batched(work, s, streams=8, overwrite=True), stream)
        if it >= args.warmup:
            bt.append(ms)
    acc = [_accuracy(A0, B0, w, X, lam[:s], float(lam.abs().max())) for (A0, B0, lam), (w, X, _) in zip(pristine, res)]
    wb = [w.clone() for w, _, _ in res]
    del res
    for it in range(args.warmup + args.steps):
        restore()
        ms, res = _event_time(lambda: [psol.solve(A, B, s, overwrite=True) for A, B in work], stream)
        if it >= args.warmup:
            pt.append(ms)
    diff = max(float(((w - r[0]).abs() / r[0].abs()).max()) for w, r in zip(wb, res))
    mb, mp = statistics.mean(bt), statistics.mean(pt)
    return {"leg": "batched", "metric": "time-to-solution of the whole batch", "value": mb / 1e3, "unit": "s",
            "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{count} problems, n uniform on multiples of 64 in [512, 4096], s={s} smallest, "
                                   "known-spectrum pencils, seeds 1000+i", "orders": ns,
                       "streams": 8, "graph": True, "panel_width_by_n": tuned, "autotune_s": tune_s},
            "steps": len(bt), "warmup": args.warmup, "ms_batched": mb, "ms_sequential": mp, "speedup": mp / mb,
            "max_rel_diff_batched_vs_sequential": diff,
            "accuracy": {"max_rel_eig_err": max(a["max_rel_eig_err_vs_constructed"] for a in acc),
                         "max_eig_gate_ratio": max(a["eig_gate_ratio"] for a in acc),
                         "max_eta": max(a["max_eta"] for a in acc), "max_orth_err": max(a["orth_err"] for a in acc)},
            "accuracy_ok": all(a["ok"] for a in acc)}


def next_warm(args, dev):
    """The learned warm start over a sequence of related pencils (n =
    args.n, default 8192, s = 64, 200 problems, dt = 0.005): the first 150
    solved from random starts give the training data; the network (two
    hidden layers of 256) trains on the GPU; the last 50 are solved from a
    random start, from the previous eigenvectors, and from the learned
    extrapolation.  Times are CUDA-event times of each solve (the pencil of
    each step is built outside them)."""
    import torch

    import inputs
    from paper_1111_6374_gb300 import warmstart

    n, s, T, T_train = args.n, args.s, args.seq_len, args.seq_train
    seq = inputs.PencilSequence(n, seed=args.seed, device=dev)
    worst = {"rel": 0.0, "gate": 0.0, "eta": 0.0, "orth": 0.0, "ok": True}

    def check(A, B, w, X, lam):
        a = _accuracy(A, B, w, X, lam[:s], float(lam.abs().max()))
        worst["rel"] = max(worst["rel"], a["max_rel_eig_err_vs_constructed"])
        worst["gate"] = max(worst["gate"], a["eig_gate_ratio"])
        worst["eta"] = max(worst["eta"], a["max_eta"])
        worst["orth"] = max(worst["orth"], a["orth_err"])
        worst["ok"] &= a["ok"]

    stats, hist, train_ms = warmstart.evaluate_sequence(seq.pencil, seq.B, n, s, T, T_train, iters=args.train_iters,
                                                        check=check, device=dev.index)
    per = {m: {"matvecs": v[0], "ms": v[1], "restarts": v[2], "ms_per_solve": v[1] / (T - T_train),
               "matvecs_per_solve": v[0] / (T - T_train)} for m, v in stats.items()}
    return {"leg": "warm", "metric": "solve time over the sequence's last problems", "value": per["learned"]["ms"] / 1e3,
            "unit": "s", "higher_is_better": False, "dtype": "f64 solve, bf16 network", "data": "synthetic",
            "config": {"workload": f"sequence of {T} related pencils n={n} s={s} (8 moving reflectors, "
                                   f"lambda(t) = lambda0 + t d, dt = 0.005), trained on the first {T_train}",
                       "n": n, "s": s, "T": T, "T_train": T_train, "train_iters": args.train_iters},
            "methods": per, "train_ms": train_ms, "loss_first_last": [hist[0], hist[-1]],
            "speedup_vs_random": per["random"]["ms"] / per["learned"]["ms"],
            "speedup_vs_reuse": per["reuse"]["ms"] / per["learned"]["ms"],
            "accuracy": {"max_rel_eig_err": worst["rel"], "max_eig_gate_ratio": worst["gate"], "max_eta": worst["eta"],
                         "max_orth_err": worst["orth"]},
            "accuracy_ok": worst["ok"]}


def run_next(args, ws, rank, local):
    import torch

    if not torch.cuda.is_available():
        print(json.dumps({"error": "bench.py needs a CUDA GPU"}), flush=True)
        return 2
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    leg = {"mixed": next_mixed, "batched": next_batched, "warm": next_warm}[args.next]
    with ClockSampler(local) as clk:
        line = leg(args, dev)
    line["clocks"] = clk.summary()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0 if line.get("accuracy_ok") else 3

def _library_point(A0, B0, s, lam):
    """cuSOLVER (torch.linalg) on the same pencil and GPU, for comparison
    only: B = U^T U, C = U^-T A U^-1 by two triangular solves, all
    eigenpairs of C (syevd), the s smallest back-transformed.  One timed run
    after a small warm-up call."""
    import torch

    def run(A, B):
        U = torch.linalg.cholesky(B, upper=True)
        W = torch.linalg.solve_triangular(U.T, A, upper=False)
        C = torch.linalg.solve_triangular(U.T, W.T, upper=False).T
        del W
        C = 0.5 * (C + C.T)
        w, Y = torch.linalg.eigh(C)
        X = torch.linalg.solve_triangular(U, Y[:, :s].contiguous(), upper=True)
        return w[:s], X

    try:
        run(A0[:256, :256].clone(), B0[:256, :256].clone())  # library handles and workspaces
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        w, X = run(A0, B0)
        e1.record()
        torch.cuda.synchronize()
        rel = float(((w - lam[:s]).abs() / lam[:s].abs()).max())
        out = {"ms": e0.elapsed_time(e1), "what": "torch.linalg cholesky + 2 x solve_triangular + eigh (cuSOLVER "
               "syevd, all n pairs) + solve_triangular, FP64", "max_rel_eig_err_vs_constructed": rel}
        del w, X
        torch.cuda.empty_cache()
        return out
    except RuntimeError as e:  # e.g. out of memory
        return {"error": str(e).splitlines()[0][:200]}


def _power(M, iters=30):
    import torch

    g = torch.Generator(device=M.device).manual_seed(0)
    v = torch.randn(M.shape[0], device=M.device, dtype=M.dtype, generator=g)
    v /= v.norm()
    lam = 0.0
    for _ in range(iters):
        w = M @ v
        lam = float(w.norm())
        v = w / lam
    return lam


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=None, help="order (default 16384; --next: 65536 mixed, 8192 warm)")
    ap.add_argument("--s", type=int, default=None, help="wanted pairs (default 100; --next: 256 mixed, 64 warm)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-sample-n", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg (profiling runs)")
    ap.add_argument("--route", choices=["inverse", "direct"], default="inverse",
                    help="inverse: largest eigenpairs of B X = A X Lambda^-1 (A is positive definite here); "
                         "direct: smallest of C = U^-T A U^-1")
    ap.add_argument("--no-other-route", action="store_true", help="skip the comparison run of the other route")
    ap.add_argument("--gen-device", choices=["cuda", "cpu"], default="cuda",
                    help="where the synthetic pencil is built (input generation only, outside any timing)")
    ap.add_argument("--block", type=int, default=0, help="panel width nb of the blocked factorisations (0 = default)")
    ap.add_argument("--check-every", type=int, default=50,
                    help="Ritz tests every this many Lanczos steps inside a cycle (gsyeig_opts.check_every; 0: only at "
                         "its end); at 50 the headline solve stops after 250 of its 300 steps")
    ap.add_argument("--graph", type=int, choices=[0, 1], default=0,
                    help="1: replay the Lanczos cycles from CUDA graphs (gsyeig_opts.graph)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the comparison solves (variant KI, plain FP64, cuSOLVER)")
    ap.add_argument("--next", choices=["mixed", "batched", "warm"], default=None,
                    help="run one extension of the route (mixed precision, a batch, the learned warm start) "
                         "against the plain path instead of the headline")
    ap.add_argument("--batch", type=int, default=64, help="--next batched: number of problems")
    ap.add_argument("--seq-len", type=int, default=200, help="--next warm: problems in the sequence")
    ap.add_argument("--seq-train", type=int, default=150, help="--next warm: problems used for training")
    ap.add_argument("--train-iters", type=int, default=2000, help="--next warm: Adam iterations")
    args = ap.parse_args(argv)
    n_def, s_def = {None: (16384, 100), "mixed": (65536, 256), "batched": (0, 16), "warm": (8192, 64)}[args.next]
    args.n = n_def if args.n is None else args.n
    args.s = s_def if args.s is None else args.s
    args.workload = f"gsyeig n={args.n} s={args.s} smallest, FP64, known-spectrum synthetic pencil"
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.next:
        return run_next(args, ws, rank, local)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
