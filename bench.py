#!/usr/bin/env python
"""MC-PDIPM benchmark: seconds per solve (relative gap 1e-7, FP64) on the chordal block-arrow
SDP with n = 2020 (40 blocks of 50 + a 20-wide border), m = 2000.

One step = one full MC-PDIPM solve from the fixed start (X̄ = I on E, z = y0), i.e. every stage
of the hot path (Y = N N^T, Algorithm 1, SCM assembly, SCM Cholesky, P-MATRIX, step lengths,
update) once per iteration until the stopping criterion.  With --gpus N (torchrun) each rank
solves its own replica (the path is not sharded: replicas only) and value = total time / total
solves (max over ranks).

--impl reference times the oracle (oracle/pdipm.py, dense FP64 HKM PDIPM) on the host cores:
each step is one oracle iteration on the same instance with the SCM evaluated on a 1/32 row
sample (scaled by 32), and value = per-iteration time x the oracle's iteration count.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MC-PDIPM s/solve & SCM-assembly GB/s at rel gap 1e-7, mixed vs FP64 on GB300"
WORKLOAD = "block_arrow_2020"
WORKLOAD_DESC = ("block-arrow SDP: 40 diagonal blocks of 50 + 20-wide border (n=2020), m=2000, "
                 "8 N(0,1) upper positions per A_p inside one block+border clique, b=A(I), "
                 "A_0=I+sum y0_p A_p, seed 20131103")
FP64_PEAK_GFLOPS = 1250.0   # GB300 nominal dense FP64 (152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz)
# DRAM bytes (read + write) per launch of the dominant kernel from an ncu capture of its current
# source; None until one is taken (the k_chol_dag capture in profiles/ predates the move of its
# ticket decode into a host+device function)
CHOL_TRAFFIC = None
KCLASS_DESC = {"ychol": "k_ychol (Y = N N^T)", "alg1": "k_alg1 (Algorithm 1)",
               "scm_panel": "k_lfwd2/k_lbwd2 (SCM panel solves)",
               "scm_tile": "k_scm_tiles (SCM tile contraction)",
               "scm_chol": "k_chol_dag (SCM Cholesky, one persistent task-queue launch)",
               "sce_backsolve": "k_backsolve_cluster (SCE back substitution)",
               "pmatrix": "k_lfwd2/k_lbwd2/k_dY_times (P-MATRIX)", "primal_step": "k_primal_step",
               "pmatrix_side": "k_lfwd2/k_lbwd2 (P-MATRIX Y^-1 columns, side stream)",
               "scm_panel_side": "k_lfwd2/k_lbwd2 (SCM N solves, side stream)",
               "dual_step": "k_ychol candidates (dual step)", "other": "scatter/scalars/update"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, device):
    """The largest value of a per-rank number over all ranks (a MAX all-reduce; identity when
    the run is not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(total_ms_max, steps, world_size):
    """Seconds per solve of the whole job: every rank solved `steps` problems in at most
    total_ms_max milliseconds (replicas, weak scaling)."""
    return total_ms_max * 1e-3 / (steps * world_size)


def golden_iters():
    try:
        with open(os.path.join(ROOT, "tests", "golden", WORKLOAD + ".json")) as f:
            return int(json.load(f)["iters"])
    except Exception:
        return None


def oracle_sample_step(inst, A, rows_frac=32):
    """One dense-oracle PDIPM iteration at the start point; SCM on every rows_frac-th row."""
    import scipy.linalg as sla
    from oracle.sdp import dual_slack
    from oracle.scm import scm_sparse_rows, hkm_rhs
    from oracle.pdipm import max_step
    n, m = inst.n, inst.m
    t0 = time.perf_counter()
    X = np.eye(n)
    z = inst.z0.copy()
    Y = dual_slack(A, z)
    mu = float(np.sum(X * Y)) / n
    Yinv = np.linalg.inv(Y)
    Yinv = 0.5 * (Yinv + Yinv.T)
    t1 = time.perf_counter()
    rows = list(range(0, m, rows_frac))
    Bs = scm_sparse_rows(A, X, Yinv, rows)
    t2 = time.perf_counter()
    # the rest of the iteration in full, on an SPD stand-in for the unsampled B rows
    B = np.eye(m) * float(np.mean(np.diag(Bs[:, rows]))) if len(rows) else np.eye(m)
    g = hkm_rhs(A, inst.b, X, Yinv, None, 0.1, mu)
    dz = sla.cho_solve(sla.cho_factor(B, lower=True), g)
    dY = -A.adjoint(dz)
    dXh = 0.1 * mu * Yinv - X - X @ dY @ Yinv
    dX = 0.5 * (dXh + dXh.T)
    max_step(X, dX)
    max_step(Y, dY)
    t3 = time.perf_counter()
    return (t1 - t0) + (t2 - t1) * rows_frac + (t3 - t2)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from instances import workload
    from oracle.sdp import SparseSym
    inst = workload(WORKLOAD)
    A = SparseSym.from_instance(inst)
    iters = golden_iters() or 30
    for _ in range(args.warmup):
        oracle_sample_step(inst, A)
    ts = [oracle_sample_step(inst, A) for _ in range(args.steps)]
    per_iter = float(np.mean(ts))
    value = per_iter * iters
    cores = os.cpu_count()
    sample = (f"one dense-oracle PDIPM iteration per step on {WORKLOAD} (SCM on 1/32 of the rows, "
              f"scaled x32), times the oracle's {iters} iterations to gap 1e-7")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s/solve",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_iter * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "desc": WORKLOAD_DESC, "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": "s/solve", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "s/solve", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200",
                                       "-i", str(gpu_index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def run_gb300(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = local if ws > 1 else 0
    torch.cuda.set_device(dev)
    from paper_1310_6919_gb300 import Problem, build_library
    if rank == 0 or ws == 1:
        build_library()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    from instances import workload
    inst = workload(WORKLOAD)
    P = Problem(inst.n, inst.m, inst.b, inst.mat, inst.row, inst.col, inst.val, form=1,
                device=dev, profile=1)
    X0 = P.identity_layout()
    z0 = torch.tensor(inst.z0, dtype=torch.float64, device=f"cuda:{dev}")
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream(dev)

    def one_solve():
        P.set_iterate(X0, z0)
        return P.solve()

    for _ in range(max(args.warmup, 0)):
        r = one_solve()
    torch.cuda.synchronize(dev)
    P.stats_reset()
    clocks = Clocks(dev)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    step_ms, results = [], []
    for _ in range(args.steps):
        flush.fill_(1)        # L2 flush (512 MiB > 129 MB L2), outside the timed events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = one_solve()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        results.append(r)
    torch.cuda.synchronize(dev)
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    stats = P.stats()
    total_ms = max_over_ranks(float(np.sum(step_ms)), f"cuda:{dev}")
    n_solves = args.steps * ws
    value = job_throughput(total_ms, args.steps, ws)
    r = results[-1]
    iters = int(r["iters"])
    ok = all(x["status"] == 0 for x in results)

    # roofline of the dominant kernel class (FP64 ALU bound)
    work = P.work_model()
    ms = stats["ms"]
    # the dominant class among those on the main stream (alg1, primal_step, pmatrix_side and
    # scm_panel_side run on side streams beside other phases, so their times overlap)
    dom = max((k for k in ms if k not in ("other", "alg1", "primal_step", "pmatrix_side",
                                          "scm_panel_side")), key=lambda k: ms[k])
    tot_iters = sum(int(x["iters"]) for x in results)
    launches_dom = stats["count"][dom]
    flops_dom = work["flops"][dom] * tot_iters
    if dom == "dual_step":
        flops_dom = work["flops"][dom] * stats["count"][dom] / max(1, P.info["tree_height"])
    avg_ms = ms[dom] / max(1, launches_dom)
    achieved = flops_dom / (ms[dom] * 1e-3) / 1e12 if ms[dom] > 0 else 0.0
    roof = {"bound": "alu", "kernel": KCLASS_DESC.get(dom, dom), "achieved": achieved,
            "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
            "frac": achieved / (FP64_PEAK_GFLOPS / 1e3),
            "traffic": CHOL_TRAFFIC if dom == "scm_chol" else None,
            "traffic_scope": ("DRAM bytes of one k_chol_dag launch (one factorisation) from an "
                              "ncu capture of this kernel" if dom == "scm_chol" and CHOL_TRAFFIC
                              else "no ncu capture of the current kernel source"),
            "avg_launch_ms": avg_ms, "launches": launches_dom,
            "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (recipe table); probe measured 1.19"}
    scm_ms = (ms["scm_panel"] + ms["scm_tile"]) / max(1, tot_iters)
    scm_bytes = work["bytes"]["scm_panel"] + work["bytes"]["scm_tile"]
    scm = {"ms_per_iter": scm_ms, "bytes_min_per_iter": scm_bytes,
           "gbs_min_bytes": scm_bytes / (scm_ms * 1e-3) / 1e9 if scm_ms > 0 else None,
           "tflops_fp64": (work["flops"]["scm_panel"] + work["flops"]["scm_tile"]) /
           (scm_ms * 1e-3) / 1e12 if scm_ms > 0 else None}
    phases = {k: ms[k] / args.steps for k in ms}

    mixed = batched = e2e = None
    if args.legs == "all":
        mixed, e2e, batched = other_legs(args, inst, dev, stream, flush, X0, z0, r, value, n_solves)

    line = None
    if rank == 0:
        # oracle timed on the host cores, bounded sample (rank 0, N = 1 only)
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            from oracle.sdp import SparseSym
            A = SparseSym.from_instance(inst)
            oi = golden_iters() or iters
            tcpu = oracle_sample_step(inst, A)
            cpu = {"value": tcpu * oi, "unit": "s/solve", "cores": os.cpu_count(),
                   "kind": "oracle",
                   "sample": (f"one dense-oracle PDIPM iteration on {WORKLOAD} (SCM on 1/32 of the "
                              f"rows, scaled x32) = {tcpu:.2f} s, times the oracle's {oi} "
                              "iterations; numpy/BLAS default threading")}
        line = {"metric": METRIC, "value": value, "unit": "s/solve", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "desc": WORKLOAD_DESC, "precision": "fp64",
                           "iterations": iters, "pobj": r["pobj"], "gap": r["gap"],
                           "all_optimal": ok, "l2": "flushed between solves (512 MiB write)",
                           "parallelism": f"replicas x{ws}"},
                "roofline": roof, "scm_assembly": scm, "phases_ms_per_solve": phases,
                "mixed": mixed, "batched": batched,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(stats["launches"]),
                "gpu_launches_per_solve": stats["launches"] / args.steps, "clocks": clk}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def other_legs(args, inst, dev, stream, flush, X0, z0, r, value, n_solves):
    """The mixed-form leg, the end-to-end leg and the batched leg of the JSON line."""
    import torch
    from paper_1310_6919_gb300 import Problem
    # the mixed form on the same workload: FP32 factor of the SCM + FP64 refinement, promoted to
    # the FP64 factor when the refinement stalls (same L2 flush, same event timing)
    Pm = Problem(inst.n, inst.m, inst.b, inst.mat, inst.row, inst.col, inst.val, form=1,
                 device=dev, profile=1, precision=1)

    def one_mixed():
        Pm.set_iterate(X0, z0)
        return Pm.solve()

    for _ in range(max(args.warmup, 0)):
        one_mixed()
    torch.cuda.synchronize(dev)
    Pm.stats_reset()
    mixed_ms, mixed_res = [], []
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rm = one_mixed()
        e1.record(stream)
        e1.synchronize()
        mixed_ms.append(e0.elapsed_time(e1))
        mixed_res.append(rm)
    mstats = Pm.stats()
    mixed_total = max_over_ranks(float(np.sum(mixed_ms)), f"cuda:{dev}")
    rm = mixed_res[-1]
    mixed = {"value": mixed_total * 1e-3 / n_solves, "unit": "s/solve",
             "speedup_vs_fp64": value / (mixed_total * 1e-3 / n_solves),
             "iterations": int(rm["iters"]), "pobj": rm["pobj"], "gap": rm["gap"],
             "pobj_diff_vs_fp64": abs(rm["pobj"] - r["pobj"]),
             "promoted_iter": int(rm["promoted_iter"]), "refine_steps": int(rm["refine_steps"]),
             "all_optimal": all(x["status"] == 0 for x in mixed_res),
             "phases_ms_per_solve": {k: mstats["ms"][k] / args.steps for k in mstats["ms"]},
             "desc": ("SCM solves and tile contraction in FP32 from FP32 copies of the factors "
                      "(B entries are FP64 numbers of FP32 sums); SCE by an FP32 Cholesky factor "
                      "of B and FP64 iterative refinement against the stored B (backward error "
                      "1e-10); FP64 throughout once the relative gap is below 1e-5 or the "
                      "refinement stalls; everything else FP64")}

    # end to end through the public API with host buffers: create (symbolic analysis + upload),
    # solve, copy the solution (X̄ on E, z) back to pinned host memory
    e2e_ms = []
    h2d = d2h = 0
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        Q = Problem(inst.n, inst.m, inst.b, inst.mat, inst.row, inst.col, inst.val, form=1,
                    device=dev)
        zh = torch.tensor(inst.z0, dtype=torch.float64).pin_memory()
        zd = zh.to(f"cuda:{dev}", non_blocking=True)
        Q.set_iterate(None, zd)
        rq = Q.solve()
        X, z, _ = Q.get_iterate()
        Xh = torch.empty(X.shape, dtype=X.dtype, pin_memory=True)
        zo = torch.empty(z.shape, dtype=z.dtype, pin_memory=True)
        Xh.copy_(X, non_blocking=True)
        zo.copy_(z, non_blocking=True)
        torch.cuda.synchronize(dev)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        h2d = Q.info.get("table_bytes", 0) + zh.numel() * 8
        d2h = Xh.numel() * 8 + zo.numel() * 8
        del Q
    e2e = {"value": float(np.median(e2e_ms)) * 1e-3, "unit": "s/solve",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # the batched form on a mix of small SDPs (48 max-cut with n ~ U{50..400}, 16 block-arrow
    # with n ~ U{100..600}): one at a time on one stream vs mcsdp_solve_batch (16 host threads,
    # a stream per problem); problems the library rejects (cliques beyond its shared-memory
    # kernels) are counted and left out of both
    from instances import batch_mix
    from paper_1310_6919_gb300 import solve_batch, MCSDPError
    mix = batch_mix(48, 16)

    def make(inst, stream):
        Q = Problem(inst.n, inst.m, inst.b, inst.mat, inst.row, inst.col, inst.val, form=1,
                    device=dev, stream=stream)
        if inst.meta.get("kind") != "maxcut":
            Q.set_iterate(None, torch.tensor(inst.z0, dtype=torch.float64, device=f"cuda:{dev}"))
        return Q

    seq_probs, bat_probs, skipped = [], [], 0
    for inst in mix:
        try:
            seq_probs.append(make(inst, None))
            bat_probs.append(make(inst, torch.cuda.Stream(dev)))
        except MCSDPError:
            skipped += 1
    make(mix[0], None).solve()  # warm-up: first-use setup of the kernels, outside the timing
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    seq_res = [Q.solve() for Q in seq_probs]
    torch.cuda.synchronize(dev)
    t_seq = time.perf_counter() - t0
    t0 = time.perf_counter()
    bat_res = solve_batch(bat_probs, nthreads=16)
    torch.cuda.synchronize(dev)
    t_bat = time.perf_counter() - t0
    batched = {"problems": len(bat_probs), "skipped": skipped,
               "sequential_problems_per_s": len(seq_probs) / t_seq,
               "batched_problems_per_s": len(bat_probs) / t_bat,
               "speedup": t_seq / t_bat,
               "all_optimal": all(r["status"] == 0 for r in bat_res),
               "same_as_sequential": all(a["pobj"] == b["pobj"] for a, b in zip(seq_res, bat_res)),
               "desc": ("48 max-cut G(n, 5n/2), n ~ U{50..400}, w ~ U[0,1) and 16 block-arrow "
                        "SDPs, n ~ U{100..600}, border 20, m = n (seeded); host wall time, "
                        "inputs resident")}
    return mixed, e2e, batched


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--legs", default="all", choices=["all", "fp64"],
                    help="fp64: only the headline FP64 leg (for profiling runs)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
