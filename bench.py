#!/usr/bin/env python
"""Benchmark of the SNMPBB solve on one GB300 (or N replicas under torchrun).

Metric: time to reach relative projected gradient 1e-4 (seconds, lower is better) on
the dense planted n = 8192, r = 64 workload: by default BF16 A, the learned step
controller and 8 random restarts in one solve, against the plain FP32 path solving the
same 8 restarts one at a time (the "compare" block), with the achieved A*W product
bandwidth of the dominant kernel beside it.  A "step" is one full solve of all restarts
from their seeded starts to the tolerance (penalty form, Sec. 2.1).

  python bench.py [--gpus N --steps K --warmup W] [--r 64 --batch 1 --precision f32]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time to proj-grad 1e-4 (s) & AW GB/s: BF16+learned+batched vs plain FP32"
L2_BYTES = 129 * 1024 * 1024
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_NOMINAL = 2070.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=8192)
    p.add_argument("--r", type=int, default=64)
    p.add_argument("--batch", type=int, default=8, help="random restarts sharing A in one solve")
    p.add_argument("--precision", default="bf16", choices=["f64", "f32", "bf16", "fp8"])
    p.add_argument("--formulation", default="penalty", choices=["penalty", "direct"])
    p.add_argument("--max-iter", type=int, default=500)
    p.add_argument("--tol", type=float, default=1e-4)
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--workload", default="dense8192", choices=["dense8192", "uneven", "graph", "lai"],
                   help="dense8192: one n=8192 problem (restarts); uneven: 256 planted problems of "
                        "uneven size in one batched solve; graph: Graph-SNMPBB on a 20000-point GMM kNN "
                        "graph with 32 restarts; lai: LAI-SNMPBB on a 2e6-node Chung-Lu graph")
    p.add_argument("--nprob", type=int, default=256)
    p.add_argument("--controller", default="auto", choices=["auto", "off", "on"],
                   help="learned step controller (auto: on when trained weights are present)")
    p.add_argument("--no-compare", action="store_true", help="skip the plain FP32 comparison runs")
    p.add_argument("--autotune", type=int, default=1, help="dense workload: tune the product at create")
    p.add_argument("--tune-cache", default=None, help="JSON cache of tuned configurations")
    p.add_argument("--cpu-iters", type=int, default=10, help="oracle outer iterations timed for cpu_baseline")
    p.add_argument("--x-parts", type=int, default=2, choices=[1, 2],
                   help="BF16 product: X as hi + lo BF16 parts (2) or rounded to BF16 (1)")
    p.add_argument("--sym-half", type=int, default=1, choices=[0, 1],
                   help="BF16 dense: keep only the 128 x 128 tiles of A on and above the diagonal "
                        "(default; the products are bitwise those of full storage)")
    return p.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        for ln in open(self.tmp.name):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=reasons, samples=len(rows),
                   power_w_max=max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                   if any(r[3].replace(".", "").isdigit() for r in rows) else None)
        return out


def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads", 0) for i in threadpool_info()), default=0)
        if n:
            return n
    except Exception:
        pass
    return os.cpu_count()


def oracle_seconds_per_iter(A, W0, r, iters, formulation):
    """FP64 CPU oracle, as it stands, timed over `iters` outer iterations."""
    import oracle as O

    opts = O.Options(formulation=formulation, memory=10, max_iter=iters, tol=0.0, objective="closed")
    t = time.perf_counter()
    if formulation == "penalty":
        O.snmpbb_penalty(A, W0, W0, opts)
    else:
        O.snmpbb_direct(A, W0, opts)
    return (time.perf_counter() - t) / iters


def oracle_golden(args):
    """The FP64 oracle's solve of restart 0 of the dense workload (iterations, residual), as
    written by tests/golden/make_oracle_iters.py; None for other shapes."""
    gold = os.path.join(ROOT, "tests", "golden", "oracle_iters_dense8192.json")
    if args.n != 8192 or args.formulation != "penalty" or not os.path.exists(gold):
        return None
    return json.load(open(gold)).get(str(args.r))


def residuals_true_A(A_np, W, H, r, b, dev):
    """||A - W_j H_j^T||_F / ||A||_F per restart against the true (FP64) A, evaluated with
    torch on the device after the timed region."""
    import torch
    Ad = torch.tensor(A_np, dtype=torch.float64, device=dev)
    nA = float(torch.linalg.norm(Ad))
    out = []
    for j in range(b):
        Wj = W[:, j * r:(j + 1) * r].double()
        Hj = H[:, j * r:(j + 1) * r].double()
        out.append(float(torch.linalg.norm(Ad - Wj @ Hj.T)) / nA)
    del Ad
    return out


def workload_name(args):
    return (f"dense planted n={args.n} r={args.r} (W0~U[0,1], A=W0W0^T+|N(0,0.05^2)| sym noise), "
            f"{args.batch} restart(s), {args.formulation} form, tol {args.tol:g} relative proj-grad")


def run_reference(args):
    """The FP64 CPU oracle timed on the host cores: each step one outer iteration on the
    same workload, extrapolated by the oracle's own iteration count to the tolerance."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from workloads.configs import dense_planted_8192

    A, starts = dense_planted_8192(args.r, 1, n=args.n)
    gold = os.path.join(ROOT, "tests", "golden", "oracle_iters_dense8192.json")
    data = json.load(open(gold)) if os.path.exists(gold) else {}
    rec = data.get(str(args.r))
    iters_to_tol = rec["iters"] if rec else args.max_iter
    for _ in range(args.warmup):
        oracle_seconds_per_iter(A, starts[0], args.r, 1, args.formulation)
    per = [oracle_seconds_per_iter(A, starts[0], args.r, 1, args.formulation) for _ in range(args.steps)]
    spi = statistics.mean(per)
    value = spi * iters_to_tol * args.batch
    sample = (f"{args.steps} single outer iterations of the oracle (closed-form objective mode) on the "
              f"n={args.n} r={args.r} workload, x {iters_to_tol} iterations to tolerance "
              f"({'oracle count, tests/golden' if rec else 'max_iter'}) x {args.batch} restart(s)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args), "n": args.n, "r": args.r, "batch": args.batch,
                       "formulation": args.formulation, "tol": args.tol},
            "cpu_baseline": {"value": value, "unit": "s", "cores": cpu_cores(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# dram__bytes_read.sum + dram__bytes_write.sum per launch, from the ncu captures summarised
# in profiles/ (k_gemm_tc_dense8192_N512.md, k_rowfuse_dstep_dense8192_N512.md,
# k_rowtc_dense8192_N512.md, k_rowtma_dense8192_N512.md, k_bgemm_tc_uneven256.md); keys:
# (workload, precision, r, batch, kernel, row-kernel body or X parts; "dense8192-sym": A held
# as its upper tiles), values: (bytes, the tuned tile shapes of the capture, which the run must
# share).  Other configurations, and runs tuned to other tiles, report null.
PROFILED_TRAFFIC = {
    ("uneven", "bf16", None, None, "product"): (875.5e6, {}),
    ("dense8192", "bf16", 64, 8, "dstep", 2): (51.4e6, {"row_bm": 128}),
    ("dense8192", "bf16", 64, 8, "product", 2): (274.31e6, {"splits": 4, "bn": 128}),
    ("dense8192-sym", "bf16", 64, 8, "product", 2): (213.78e6, {"splits": 4, "bn": 128}),
    ("dense8192", "bf16", 64, 8, "dstep", 3): (51.03e6, {}),
    ("dense8192", "bf16", 64, 8, "update", 3): (68.16e6, {}),
    ("dense8192", "bf16", 64, 8, "dstep", 4): (51.10e6, {}),
    ("dense8192", "bf16", 64, 8, "update", 4): (68.78e6, {}),
}


def profiled_traffic(key, tuning):
    """Captured DRAM traffic of one launch, or None when the run's tiles differ from the capture's."""
    got = PROFILED_TRAFFIC.get(key)
    if got is None:
        return None
    traffic, tiles = got
    if tiles and not all((tuning or {}).get(k) == v for k, v in tiles.items()):
        return None
    return traffic


def rank_restarts(batch, rank):
    """Restart indices of this rank: each rank solves its own `batch` restarts (weak scaling,
    no data exchange between ranks)."""
    return list(range(rank * batch, (rank + 1) * batch))


def uneven_seed(rank):
    """Problem-set seed of a rank: rank 0 uses the bench's set, others disjoint sets."""
    return 5000 + 100000 * rank


def max_over_ranks(value, world, device=None):
    """Whole-job time: the maximum over ranks (all_reduce MAX; any backend)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def controller_weights(args):
    """Trained controller weights shipped with the package (None when absent or disabled)."""
    if args.controller == "off":
        return None
    from paper_2606_02887_gb300.train_controller import WEIGHTS_PATH, load_weights
    if os.path.exists(WEIGHTS_PATH):
        return load_weights()
    if args.controller == "on":
        raise SystemExit("controller weights not found: " + WEIGHTS_PATH)
    return None


def uneven_problems(count, seed=5000):
    """256 planted problems, n ~ U{64..2048}, r ~ U{4..32}, 1% relative noise (problem seeds
    seed + 1 ..); starts U[0, sqrt(mean(A_p)/r_p)] with seed 6000 + p."""
    from workloads import uneven_batch, uniform_init
    out = []
    for p, (A, _, r) in enumerate(uneven_batch(count, seed=seed)):
        out.append((A, uniform_init(A.shape[0], r, math.sqrt(A.mean() / r), seed=6000 + p), r))
    return out


def uneven_name(args):
    return (f"uneven batch: {args.nprob} dense planted problems, n~U{{64..2048}}, r~U{{4..32}}, "
            f"1% relative noise, penalty form, tol {args.tol:g} relative proj-grad per problem")


def run_uneven(args):
    """Many uneven problems in one batched solve (grouped launches + CUDA graph), against the
    plain FP32 path solving the same problems one at a time."""
    import numpy as np
    import torch

    import paper_2606_02887_gb300.snmf as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    S.load_library()
    probs = uneven_problems(args.nprob, uneven_seed(rank))  # weak scaling: own problems per rank
    ns = [A.shape[0] for A, _, _ in probs]
    rs = [r for _, _, r in probs]
    vals = torch.tensor(np.concatenate([A.ravel() for A, _, _ in probs]), dtype=torch.float32, device=dev)
    W0 = torch.tensor(np.concatenate([W.ravel() for _, W, _ in probs]), dtype=torch.float32, device=dev)
    W = torch.empty_like(W0)
    H = torch.empty_like(W0)
    prec = {"f64": S.SNMF_F64, "f32": S.SNMF_F32, "bf16": S.SNMF_BF16, "fp8": S.SNMF_FP8}[args.precision]
    weights = controller_weights(args)
    ctl = 3 if weights is not None else 0  # lean learned step
    stream = torch.cuda.current_stream(dev)

    def handle(pr, c):
        o = S.snmf_default_options(precision=pr, max_iter=args.max_iter, tol=args.tol, nonmonotone_M=10,
                                   step_controller=c)
        return S.snmf_create(S.dense_batch_matrix(vals, ns, rs), 0, o, stream=stream,
                             mlp_weights=weights if c else None)

    def solve(h):
        W.copy_(W0)
        H.copy_(W0)
        return S.snmf_solve(h, W, H)

    h = handle(prec, ctl)
    for _ in range(args.warmup):
        solve(h)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches, last = 0, None
    for k in range(args.steps):
        ev[k][0].record(stream)
        st, stats = solve(h)
        ev[k][1].record(stream)
        launches += stats["kernel_launches"]
        last = (st, stats)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    times = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(statistics.mean(times), world, dev)
    st, stats = last
    per = S.snmf_restart_stats(h, len(probs))
    ms_prod, _ = S.snmf_profile_ax(h, 10)
    esz_a = {"f64": 8, "f32": 4, "bf16": 2}[args.precision]
    esz = 8 if args.precision == "f64" else 4
    alg_bytes = sum(n * n * esz_a + 2 * n * r * esz for n, r in zip(ns, rs))
    flops = sum(2.0 * n * n * r for n, r in zip(ns, rs))
    S.snmf_destroy(h)
    peaks, peak_kind = measured_peaks()
    gbs = alg_bytes / (ms_prod * 1e-3) / 1e9
    kname = ("k_bsplit_x + k_bgemm_tc (grouped tcgen05 A_p (X_hi + X_lo), BF16 A)" if args.precision == "bf16"
             else "k_bgemm (grouped A_p X_p, CUDA cores, %s A)" % args.precision)
    traffic = profiled_traffic(("uneven", args.precision, None, None, "product"), None) if args.nprob == 256 else None
    roof = {"bound": "hbm", "kernel": kname, "traffic_bytes": traffic,
            "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
            "traffic": traffic, "peak_source": peak_kind, "alg_bytes_per_launch": alg_bytes,
            "flops_per_launch": flops, "tflops": flops / (ms_prod * 1e-3) / 1e12, "ms_per_launch": ms_prod}

    compare = None
    if not args.no_compare and rank == 0:
        compare = {}
        for name, pr, c in (("batched_bf16_plain", S.SNMF_BF16, 0), ("batched_f32_plain", S.SNMF_F32, 0)):
            if pr == prec and c == ctl:
                continue
            hc = handle(pr, c)
            solve(hc)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stc, sc = solve(hc)
            e1.record(stream)
            torch.cuda.synchronize()
            pc = S.snmf_restart_stats(hc, len(probs))
            S.snmf_destroy(hc)
            compare[name] = {"s": e0.elapsed_time(e1) / 1e3, "status": stc, "outer_iters_total": int(pc["iters"].sum()),
                             "max_pg_rel": float(pc["pg_rel"].max())}
        # plain FP32: one problem per snmf_solve, FP32 A, no controller (device time of the solves)
        tot, it_plain, res_plain = 0.0, [], []
        o = S.snmf_default_options(precision=S.SNMF_F32, max_iter=args.max_iter, tol=args.tol, nonmonotone_M=10)
        for A, W0p, r in probs:
            At = torch.tensor(A, dtype=torch.float32, device=dev)
            hp_ = S.snmf_create(S.dense_matrix(At), r, o, stream=stream)
            Wp = torch.tensor(W0p, dtype=torch.float32, device=dev)
            stp, sp = S.snmf_solve(hp_, Wp, Wp.clone())
            S.snmf_destroy(hp_)
            tot += sp["seconds"]
            it_plain.append(sp["iters"])
            res_plain.append(sp["residual"])
        res_plain = np.array(res_plain)
        dres = np.abs(per["residual"] - res_plain)
        compare["plain_f32_one_problem_per_solve"] = {
            "s": tot, "outer_iters_total": int(np.sum(it_plain)),
            "speedup_of_value": tot / (ms / 1e3),
            "residual_max_abs_diff": float(dres.max()), "problems_within_1e-3": int(np.sum(dres <= 1e-3))}

    cpu = None
    if not args.no_cpu and rank == 0:
        import oracle as O
        sample = [0, 1, 2]
        t0 = time.perf_counter()
        for p in sample:
            A, W0p, r = probs[p]
            O.snmpbb_penalty(A, W0p, W0p, O.Options(max_iter=2, tol=0.0, memory=10, objective="closed"))
        spi = (time.perf_counter() - t0) / (2.0 * sum(float(ns[p]) ** 2 * rs[p] for p in sample))
        est = spi * sum(float(n) * n * r * int(it) for n, r, it in zip(ns, rs, per["iters"]))
        cpu = {"value": est, "unit": "s", "cores": cpu_cores(), "kind": "oracle",
               "sample": "2 outer iterations of the FP64 oracle on problems 0-2, scaled by n_p^2 r_p x the "
                         "iterations each problem took on the GPU"}

    e2e = None
    if not args.no_e2e:
        vals_h = vals.cpu()
        W_h = torch.empty_like(W0, device="cpu").pin_memory()
        H_h = torch.empty_like(W0, device="cpu").pin_memory()
        W0_h = W0.cpu()
        o = S.snmf_default_options(precision=prec, max_iter=args.max_iter, tol=args.tol, nonmonotone_M=10,
                                   step_controller=ctl)
        et = []
        for k in range(2):
            W_h.copy_(W0_h)
            H_h.copy_(W0_h)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            he = S.snmf_create(S.dense_batch_matrix(vals_h, ns, rs), 0, o, stream=stream,
                               mlp_weights=weights if ctl else None)
            S.snmf_solve_host(he, W_h, H_h)
            S.snmf_destroy(he)
            torch.cuda.synchronize()
            if k:
                et.append(time.perf_counter() - t0)
        fb = W0.numel() * 4
        e2e = {"value": statistics.mean(et), "unit": "s", "h2d_bytes_per_step": vals.numel() * 4 + 2 * fb,
               "d2h_bytes_per_step": 2 * fb,
               "path": "snmf_create(host A, batch) + snmf_solve_host + snmf_destroy, wall clock"}

    if rank == 0:
        line = {"metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
                "config": {"workload": uneven_name(args), "nprob": args.nprob, "precision": args.precision,
                           "controller": "learned" if ctl else "plain BB", "tol": args.tol,
                           "max_iter": args.max_iter,
                           "l2": "inputs larger than L2 (sum of A_p %.0f MB)" % (alg_bytes / 2**20),
                           "parallelism": "single GPU"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
                "solve": {"status": st, "max_iters": stats["iters"], "outer_iters_total": int(per["iters"].sum()),
                          "max_pg_rel": float(per["pg_rel"].max()), "max_residual": float(per["residual"].max()),
                          "ctl_proposals": stats["ctl_proposals"], "ctl_accepted": stats["ctl_accepted"],
                          "ms_per_step_all": times},
                "compare": compare}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _sparse_common(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    return world, rank, torch.device("cuda", local)


def _cluster_accuracy(labels, pred, k):
    """Fraction of points in the best one-to-one matching of clusters to planted labels."""
    import numpy as np
    from scipy.optimize import linear_sum_assignment
    C = np.zeros((k, k))
    np.add.at(C, (pred, labels), 1)
    row, col = linear_sum_assignment(-C)
    return float(C[row, col].sum() / len(labels))


def run_sparse(args):
    """Graph-SNMPBB on the GMM kNN graph (CSR A_hat, CSR L, gamma 0.1, r 20, 32 restarts in one
    solve) or LAI-SNMPBB on the Chung-Lu graph (k 64 + 10, 2 power iterations, r 32)."""
    import numpy as np
    import torch

    import paper_2606_02887_gb300.snmf as S
    from workloads import chung_lu_csr, gmm_knn_graph, uniform_init

    world, rank, dev = _sparse_common(args)
    S.load_library()
    t_gen = time.perf_counter()
    if args.workload == "graph":
        A_hat, L, labels, _ = gmm_knn_graph(n=20000, d=64, comps=20, k=10, seed=3000 + 7 * rank)
        r, b, gamma = 20, 32, 0.1
    else:
        A_hat = chung_lu_csr(n=2_000_000, exponent=2.1, mean_degree=16.0, seed=4000 + 7 * rank)
        L, labels = None, None
        r, b, gamma = 32, 1, 0.0
    t_gen = time.perf_counter() - t_gen
    n = A_hat.n
    nnz = int(len(A_hat.values))
    tens = lambda x, dt: torch.tensor(np.ascontiguousarray(x), dtype=dt, device=dev)
    Am = (tens(A_hat.rowptr, torch.int32), tens(A_hat.colidx, torch.int32), tens(A_hat.values, torch.float32))
    mean = float(A_hat.values.sum()) / (float(n) * n)
    W0 = np.concatenate([uniform_init(n, r, math.sqrt(mean / r), seed=3100 + j) for j in range(b)], 1)
    W0t = torch.tensor(W0, dtype=torch.float32, device=dev)
    W, H = torch.empty_like(W0t), torch.empty_like(W0t)
    opts = S.snmf_default_options(precision=S.SNMF_F32, batch=b, max_iter=args.max_iter, tol=args.tol,
                                  nonmonotone_M=10)
    stream = torch.cuda.current_stream(dev)
    h = S.snmf_create(S.csr_matrix(n, *Am), r, opts, stream=stream)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sketch_ms = None
    if args.workload == "graph":
        Lm = (tens(L.rowptr, torch.int32), tens(L.colidx, torch.int32), tens(L.values, torch.float32))
        S.snmf_set_graph_reg(h, S.csr_matrix(n, *Lm), gamma)
    else:
        ev0.record(stream)
        S.snmf_lai_sketch(h, 64, 10, 2, 4242)
        ev1.record(stream)
        torch.cuda.synchronize()
        sketch_ms = ev0.elapsed_time(ev1)

    def solve():
        W.copy_(W0t)
        H.copy_(W0t)
        return S.snmf_solve(h, W, H)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    times, launches, last = [], 0, None
    for _ in range(args.steps):
        ev0.record(stream)
        st, stats = solve()
        ev1.record(stream)
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1))
        launches += stats["kernel_launches"]
        last = (st, stats)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(statistics.mean(times), world, dev)
    st, stats = last
    per = S.snmf_restart_stats(h, b)
    ms_prod, ms_kern = S.snmf_profile_ax(h, 10)
    peaks, peak_kind = measured_peaks()
    N = r * b
    if args.workload == "graph":
        alg = nnz * 8 + (n + 1) * 4 + 2 * n * N * 4  # CSR (col index + value), row pointers, X, Y
        kname = "k_spmm_csr (+ k_ax_finish)"
    else:
        ell = 64
        alg = 2 * n * ell * 4 + 2 * n * N * 4  # U read by U^T X and by U (Lambda X^), X, Y
        kname = "k_utx + k_rowmul (LAI product U (Lambda (U^T X)))"
    gbs = alg / (ms_prod * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": kname, "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": gbs / peaks["hbm_gbs"], "traffic": None, "peak_source": peak_kind,
            "alg_bytes_per_launch": alg, "ms_per_launch": ms_prod}
    extra = {}
    if labels is not None:
        Wn = W.cpu().numpy()
        best = int(np.argmin(per["f"]))
        pred = np.argmax(Wn[:, best * r:(best + 1) * r], axis=1)
        extra["accuracy_best_restart"] = _cluster_accuracy(np.asarray(labels), pred, r)
    S.snmf_destroy(h)
    if rank == 0:
        line = {"metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": ("Graph-SNMPBB, GMM kNN graph n=20000 (20 components, d=64, k=10), "
                                        "gamma 0.1, r=20, 32 restarts" if args.workload == "graph" else
                                        "LAI-SNMPBB, Chung-Lu n=2e6 (exponent 2.1, mean degree 16), "
                                        "sketch k=64+10, q=2, r=32"),
                           "n": n, "nnz": nnz, "r": r, "batch": b, "tol": args.tol, "max_iter": args.max_iter,
                           "generation_s": t_gen, "sketch_ms": sketch_ms,
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "roofline": roof, "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clk,
                "solve": {"status": st, "iters": stats["iters"], "residual_best": stats["residual"],
                          "pg_rel": stats["pg_rel"], "ms_per_step_all": times, **extra}}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "uneven":
        return run_uneven(args)
    if args.workload in ("graph", "lai"):
        return run_sparse(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2606_02887_gb300.snmf as S
    from workloads.configs import dense_planted_8192

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    S.load_library()

    prec = {"f64": S.SNMF_F64, "f32": S.SNMF_F32, "bf16": S.SNMF_BF16, "fp8": S.SNMF_FP8}[args.precision]
    tdt = torch.float64 if args.precision == "f64" else torch.float32
    mine = rank_restarts(args.batch, rank)  # replicas: own restarts per rank
    A_np, starts = dense_planted_8192(args.r, mine[-1] + 1, n=args.n)
    starts = [starts[j] for j in mine]
    W0_np = np.concatenate(starts, axis=1)
    A = torch.tensor(A_np, dtype=tdt, device=dev)
    W0 = torch.tensor(W0_np, dtype=tdt, device=dev)
    W = torch.empty_like(W0)
    H = torch.empty_like(W0)
    form = S.SNMF_PENALTY if args.formulation == "penalty" else S.SNMF_DIRECT
    weights = controller_weights(args) if form == S.SNMF_PENALTY and args.r <= 64 else None
    ctl = 3 if weights is not None else 0  # lean learned step
    opts = S.snmf_default_options(precision=prec, formulation=form, batch=args.batch, max_iter=args.max_iter,
                                  tol=args.tol, nonmonotone_M=10, autotune=args.autotune,
                                  tune_cache=args.tune_cache, step_controller=ctl, x_parts=args.x_parts,
                                  sym_half=args.sym_half if args.precision == "bf16" else 0)
    stream = torch.cuda.current_stream(dev)
    h = S.snmf_create(S.dense_matrix(A), args.r, opts, stream=stream, mlp_weights=weights)
    tuning = None
    if args.autotune:
        try:
            tuning = S.snmf_tuned_config(h)
        except S.SnmfError:  # no candidate fitted this shape: built-in configuration
            tuning = {"tuned": False}
    a_bytes = A.numel() * {"bf16": 2, "fp8": 1}.get(args.precision, A.element_size())
    if args.sym_half and args.precision == "bf16":
        a_bytes = args.n * (args.n + 1) // 2 * 2  # the triangle on and above the diagonal
    flush = None if a_bytes > 2 * L2_BYTES else torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step():
        W.copy_(W0)
        H.copy_(W0)
        return S.snmf_solve(h, W, H if form == S.SNMF_PENALTY else None)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    launches = 0
    stats_list = []
    for k in range(args.steps):
        if flush is not None:
            flush.zero_()
        ev[k][0].record(stream)
        st, stats = step()
        ev[k][1].record(stream)
        launches += stats["kernel_launches"]
        stats_list.append((st, stats))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    times = [a.elapsed_time(b) for a, b in ev]
    ms = statistics.mean(times)
    ms_max = max_over_ranks(ms, world, dev)
    st, stats = stats_list[-1]

    # dominant kernel: the A*X product, timed alone on the library's stream (CUDA events)
    ms_prod, ms_kern = S.snmf_profile_ax(h, 20)
    n, N = args.n, args.r * args.batch
    esz = 8 if args.precision == "f64" else 4
    a_esz = {"bf16": 2, "fp8": 1}.get(args.precision, esz)
    sym = bool(args.sym_half and args.precision == "bf16")
    # symmetric-half storage: A's algorithmic bytes are the triangle on and above the diagonal
    alg_bytes = (n * (n + 1) // 2 if sym else n * n) * a_esz + 2 * n * N * esz
    flops = 2.0 * n * n * N
    peaks, peak_kind = measured_peaks()
    sm_mhz = clk.get("sm_mhz") or SM_MAX_MHZ_NOMINAL
    alu_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12  # TFLOP/s at max clock
    achieved_tflops = flops / (ms_kern * 1e-3) / 1e12 if ms_kern > 0 else None
    aw_gbs = alg_bytes / (ms_kern * 1e-3) / 1e9 if ms_kern > 0 else None
    if args.precision == "f32":
        kn = "k_gemm_dense<float> (CUDA-core FFMA)"
        roof = {"bound": "alu", "kernel": kn, "achieved": achieved_tflops,
                "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved_tflops / alu_peak if achieved_tflops else None,
                "traffic": None, "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                "aw_gbs": aw_gbs, "aw_hbm_frac": aw_gbs / peaks["hbm_gbs"] if aw_gbs else None,
                "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_peak_source": peak_kind,
                "alg_bytes_per_launch": alg_bytes, "flops_per_launch": flops,
                "ms_per_launch": ms_kern, "ms_per_product_with_epilogue": ms_prod}
    elif args.precision in ("bf16", "fp8"):
        # E4M3 A: the same tcgen05 kernel with the code tiles decoded to BF16 in shared memory
        workload_key = "dense8192" + ("-sym" if sym else "") if args.n == 8192 and args.precision == "bf16" else None
        # the method's flops 2 n^2 N; the tensor pipes execute x_parts times that (X as hi + lo
        # BF16 parts takes two MMA passes)
        tflops = flops / (ms_kern * 1e-3) / 1e12
        ridge = peaks["bf16_tflops"] * 1e12 / (peaks["hbm_gbs"] * 1e9)
        intensity = args.x_parts * flops / alg_bytes
        tensor_bound = intensity > ridge
        roof = {"bound": "tensor" if tensor_bound else "hbm",
                "kernel": "k_split_x + %s (tcgen05 BF16, X as %s, split-K reduced and epilogue fused "
                          "in the kernel%s)" % ("k_gemm_tc" if args.precision == "bf16" else
                                               "k_gemm_tc<true> (E4M3 code tiles decoded to BF16 in shared memory)",
                                               "hi+lo BF16 parts" if args.x_parts == 2 else "one BF16 part",
                                               "; A as its upper 128 x 128 tiles" if sym else ""),
                "achieved": tflops if tensor_bound else aw_gbs,
                "peak": peaks["bf16_tflops"] if tensor_bound else peaks["hbm_gbs"],
                "unit": "TFLOP/s" if tensor_bound else "GB/s",
                "frac": (tflops / peaks["bf16_tflops"]) if tensor_bound else (aw_gbs / peaks["hbm_gbs"]),
                "traffic": profiled_traffic((workload_key, args.precision, args.r, args.batch, "product",
                                             args.x_parts), tuning),
                "peak_source": peak_kind + (" bf16_tflops (burst cuBLAS)" if tensor_bound else " hbm_gbs (burst copy)"),
                "intensity_flop_per_byte": intensity, "ridge_flop_per_byte": ridge,
                "tensor_pipe_tflops": args.x_parts * tflops,
                "aw_gbs": aw_gbs, "aw_hbm_frac": aw_gbs / peaks["hbm_gbs"],
                "alg_bytes_per_launch": alg_bytes, "flops_per_launch": flops,
                "flops_note": "method flops 2 n^2 N; the tensor pipes execute x_parts x that",
                "ms_per_launch": ms_kern, "ms_per_product_with_epilogue": ms_prod}
    else:
        roof = {"bound": "alu", "kernel": "k_gemm_dense<double>", "achieved": achieved_tflops, "peak": None,
                "unit": "TFLOP/s", "frac": None, "traffic": None, "aw_gbs": aw_gbs,
                "ms_per_launch": ms_kern}

    # the row kernels of an inner step, timed alone (CUDA events on the library's stream);
    # per outer iteration: 2 products, 2 K D-step launches, 2 K update launches (K = 5)
    kernels = {"product": roof}
    if form == S.SNMF_PENALTY and args.r <= 64:
        ms_d, ms_u = S.snmf_profile_steps(h, 20)
        K = opts.inner_iters
        # the library reports which row-kernel body runs and the arrays each launch moves
        sc = S.snmf_step_config(h)
        body = {0: "k_rowgemm (general)", 1: "k_rowtile (shared-memory tile body)",
                2: "k_rowfuse (Z and D recomputed, not stored; row products on CUDA cores)",
                3: "k_rowtc (Z and D recomputed, not stored; row products on tcgen05, TF32 hi + lo)",
                4: "k_rowtma (as k_rowtc, persistent: one CTA per SM, inputs streamed by TMA)"}[sc["body"]]
        prefix = {2: "k_rowfuse", 3: "k_rowtc"}.get(sc["body"])
        names = {"dstep": (prefix + "_dstep" if prefix else "k_rowgemm<OP_ZSTEP, EPI_DIR>"),
                 "update": (prefix + "_update" if prefix else "k_rowgemm<OP_UPD, EPI_GRAD>")}
        if sc["body"] == 4:
            names = {"dstep": "k_rowtma<0> (D step)", "update": "k_rowtma<1> (update)"}
        for name, ms_k, nbytes in (("dstep", ms_d, sc["dstep_bytes"]), ("update", ms_u, sc["update_bytes"])):
            gb = nbytes / (ms_k * 1e-3) / 1e9
            kernels[name] = {"bound": "hbm", "kernel": names[name], "body": body,
                             "rows_per_cta": sc["rows_per_cta"],
                             "achieved": gb, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                             "frac": gb / peaks["hbm_gbs"], "peak_source": peak_kind,
                             "traffic": profiled_traffic(("dense8192" if args.n == 8192 else None, args.precision,
                                                          args.r, args.batch, name, sc["body"]), tuning),
                             "alg_bytes_per_launch": nbytes, "arrays_per_launch": nbytes // (n * N * esz),
                             "ms_per_launch": ms_k, "launches_per_outer_iteration": 2 * K,
                             "note": "working set of one launch fits in L2, as inside the iteration"}
        per_iter = {"product": 2 * ms_kern, "dstep": 2 * K * ms_d, "update": 2 * K * ms_u}
        dominant = max(per_iter, key=per_iter.get)
        roof = dict(kernels[dominant])
        roof["dominant_by"] = {k: round(v, 4) for k, v in per_iter.items()}
        roof["dominant_unit"] = "ms of kernel time per outer iteration"

    # end to end through the C ABI with host buffers (inputs and result cross PCIe/C2C)
    e2e = None
    if not args.no_e2e:
        A_host = A.cpu().pin_memory()
        W_host = torch.empty_like(W0, device="cpu").pin_memory()
        H_host = torch.empty_like(W0, device="cpu").pin_memory()
        W0_host = W0.cpu()
        e_times = []
        for k in range(args.e2e_steps + 1):
            W_host.copy_(W0_host)
            H_host.copy_(W0_host)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            he = S.snmf_create(S.dense_matrix(A_host), args.r, opts, stream=stream, mlp_weights=weights)
            S.snmf_solve_host(he, W_host, H_host if form == S.SNMF_PENALTY else None)
            S.snmf_destroy(he)
            torch.cuda.synchronize()
            if k > 0:
                e_times.append(time.perf_counter() - t0)
        fb = W0.numel() * W0.element_size()
        nf = 2 if form == S.SNMF_PENALTY else 1
        a_host_bytes = A_host.numel() * A_host.element_size()  # A crosses in its host dtype
        e2e = {"value": statistics.mean(e_times), "unit": "s", "h2d_bytes_per_step": a_host_bytes + nf * fb,
               "d2h_bytes_per_step": nf * fb,
               "path": "snmf_create(host A, %s) + snmf_solve_host + snmf_destroy, wall clock; the library "
                       "converts A to its storage precision on the device" % str(A_host.dtype).replace("torch.", "")}
    per = S.snmf_restart_stats(h, args.batch)
    S.snmf_destroy(h)
    res_true = residuals_true_A(A_np, W, H if form == S.SNMF_PENALTY else W, args.r, len(mine), dev)
    error_vs_oracle = None
    gold = oracle_golden(args)
    if gold is not None and mine[0] == 0:
        error_vs_oracle = {
            "restart": 0, "residual_true_A": res_true[0], "oracle_residual": gold["residual"],
            "abs_diff": abs(res_true[0] - gold["residual"]), "bar": 1e-3,
            "within_bar": bool(abs(res_true[0] - gold["residual"]) <= 1e-3),
            "iters": int(per["iters"][0]), "oracle_iters": gold["iters"],
            "pg_rel": float(per["pg_rel"][0]), "oracle_pg_rel": gold["pg_rel"],
            "source": "tests/golden/oracle_iters_dense8192.json (FP64 oracle, same start, penalty form, M=10)"}

    # the same restarts solved by the plain FP32 path: one restart per snmf_solve, FP32 A,
    # no controller (device time of each solve, CUDA events inside the library)
    compare = None
    if rank == 0 and not args.no_compare:
        A32 = A.float() if A.dtype != torch.float32 else A
        o32 = S.snmf_default_options(precision=S.SNMF_F32, formulation=form, max_iter=args.max_iter, tol=args.tol,
                                     nonmonotone_M=10)
        hp = S.snmf_create(S.dense_matrix(A32), args.r, o32, stream=stream)
        tot, its, res = 0.0, [], []
        for j in range(args.batch):
            Wj = W0[:, j * args.r:(j + 1) * args.r].float().contiguous()
            Hj = Wj.clone()
            stp, sp = S.snmf_solve(hp, Wj, Hj if form == S.SNMF_PENALTY else None)
            tot += sp["seconds"]
            its.append(sp["iters"])
            res.append(sp["residual"])
        S.snmf_destroy(hp)
        dres = np.abs(np.asarray(per["residual"]) - np.asarray(res))
        compare = {"plain_f32_one_restart_per_solve": {
            "s": tot, "iters": its, "residual": res, "speedup_of_value": tot / (ms_max / 1e3),
            "residual_max_abs_diff": float(dres.max()), "restarts_within_1e-3": int(np.sum(dres <= 1e-3))},
            "this_run": {"iters": [int(x) for x in per["iters"]], "residual": [float(x) for x in per["residual"]],
                         "residual_true_A": res_true, "pg_rel_max": float(np.max(per["pg_rel"]))}}
        if ctl:
            # the same batched solve with the plain BB step (separates the controller's share of
            # the gain from batching and storage precision), and with the learned step in mode 1
            # (every rejected proposal falls back to the plain BB step; two directions per step)
            for name, mode in (("batched_plain_bb_same_precision", 0), ("learned_with_bb_fallback_mode1", 1)):
                ob = S.snmf_default_options(precision=prec, formulation=form, batch=args.batch,
                                            max_iter=args.max_iter, tol=args.tol, nonmonotone_M=10,
                                            autotune=args.autotune, tune_cache=args.tune_cache, step_controller=mode,
                                            x_parts=args.x_parts,
                                            sym_half=args.sym_half if args.precision == "bf16" else 0)
                hb = S.snmf_create(S.dense_matrix(A), args.r, ob, stream=stream,
                                   mlp_weights=weights if mode else None)
                bt = []
                for k in range(2):
                    W.copy_(W0)
                    H.copy_(W0)
                    stb, sb = S.snmf_solve(hb, W, H if form == S.SNMF_PENALTY else None)
                    bt.append(sb["seconds"])
                pb = S.snmf_restart_stats(hb, args.batch)
                S.snmf_destroy(hb)
                compare[name] = {
                    "s": bt[-1], "status": int(stb), "iters": [int(x) for x in pb["iters"]],
                    "residual": [float(x) for x in pb["residual"]], "pg_rel_max": float(np.max(pb["pg_rel"])),
                    "value_over_this": bt[-1] / (ms_max / 1e3),
                    "note": "device time of one solve (CUDA events in the library), second of two runs"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        iters_s = args.cpu_iters
        spi = oracle_seconds_per_iter(A_np, starts[0], args.r, iters_s, args.formulation)
        iters_to_tol = gold["iters"] if gold is not None else stats["iters"]
        est = spi * iters_to_tol * args.batch
        cpu = {"value": est, "unit": "s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"{iters_s} outer iterations of the FP64 oracle (closed-form objective) on restart 0 of "
                         f"this workload ({spi:.3f} s/iteration), x {iters_to_tol} iterations to tolerance "
                         f"({'the oracle own count, tests/golden' if gold is not None else 'this run count'}) "
                         f"x {args.batch} restart(s)"}

    if rank == 0:
        line = {"metric": METRIC, "value": ms_max / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
                "config": {"workload": workload_name(args), "n": args.n, "r": args.r, "batch": args.batch,
                           "precision": args.precision, "formulation": args.formulation, "tol": args.tol,
                           "max_iter": args.max_iter, "controller": "learned" if ctl else "plain BB",
                           "a_storage": "upper 128 x 128 tiles (symmetric half)" if args.sym_half and
                           args.precision == "bf16" else "full",
                           "l2": ("inputs larger than L2 (A = %.0f MB)" % (a_bytes / 2**20)) if flush is None
                           else "L2 flushed between timed steps (256 MB write)",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "roofline": roof, "roofline_kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
                "error_vs_oracle": error_vs_oracle,
                "gpu_launches": launches, "clocks": clk, "tuning": tuning,
                "solve": {"status": st, "iters": stats["iters"], "residual": stats["residual"],
                          "pg_rel": stats["pg_rel"], "ls_fail": stats["ls_fail"],
                          "ax_products": stats["ax_products"], "graph_replays": stats["graph_replays"],
                          "ctl_proposals": stats["ctl_proposals"], "ctl_accepted": stats["ctl_accepted"],
                          "ms_per_step_all": times},
                "compare": compare}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
