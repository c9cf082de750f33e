#!/usr/bin/env python
"""MC-PDIPM benchmark: seconds per solve (relative gap 1e-7), mixed vs FP64, on the max-cut SDP of
a random sparse graph with n = m = 20000 (a Hamiltonian ring over a seeded permutation plus 2n
distinct random edges, average degree 6, weights U[0, 1)).

One step = one full MC-PDIPM solve of that workload from the fixed start (X̄ = I on E, the
dual-feasible z0), every stage of the hot path (Y = N N^T, Algorithm 1, SCM assembly, SCM
Cholesky, P-MATRIX, step lengths, update) once per iteration until the stopping criterion.  The
headline value is the mixed form (FP32 tensor-core products and factor, FP64 refinement, staged
promotion to FP64); the line's `fp64` object is the same workload solved in FP64, timed the same
way.  With --gpus N (torchrun) each rank solves its own replica (the path is not sharded:
replicas only) and value = total time / total solves (max over ranks).

--impl reference times the oracle (oracle/pdipm.py, the dense FP64 HKM PDIPM) on the host cores.
A full oracle iteration at n = 20000 runs for many minutes (dense inverses, eigenvalue problems
and products of order n), so each step times one of its operations on the real sizes, the dense
Cholesky factorisation of the 20000 x 20000 Schur complement matrix (sla.cho_factor, as the oracle
calls it), and scales it by the oracle iteration's dense flop count (13 n^3 against n^3 / 3) and
by the iteration count: an extrapolation, labelled as such.
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
WORKLOAD = "ring_maxcut_20000"
WORKLOAD_DESC = ("max-cut SDP of a random sparse graph: Hamiltonian ring over a seeded permutation "
                 "+ 2n distinct random edges (average degree 6), w ~ U[0,1), C = -L/4, "
                 "A_k = e_k e_k^T, b = 1, n = m = 20000, seed 20131104")
CONTEXT_WORKLOAD = "block_arrow_2020"
BLOCKS_WORKLOAD = "maxcut_sum_64"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12  # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_SOURCE = ("derived: 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz = 1.26 TFLOP/s "
                    "(nominal 1.25; no measured FP64 peak on this pool)")
TF32_BF16_RATIO = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor rates (recipe table)
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch, from ncu captures on
# ring_maxcut_8000 (nR = 3158, m = 8000; the current kernel sources), per unit of work, scaled to
# a full launch by the work it does (nR^3 for the root GEMM, m^3 for the SCM Cholesky: both tile
# their operands through L2 the same way at either size)
TRAFFIC_PER_UNIT = {"root_gemm": (1.238365e9 + 77.669888e6) / 3158 ** 3,
                    "scm_chol": (13.867930e9 + 18.936653e9) / 8000 ** 3}
ORACLE_ITER_OVER_CHOL = 13.0 / (1.0 / 3.0)  # dense oracle iteration flops / SCM Cholesky flops
KCLASS_DESC = {"ychol": "k_ychol + k_root_gather + k_chol_dag (Y = N N^T, root FP64 Cholesky)",
               "alg1": "k_alg1 + k_chol_dag + k_gemm_tn<double> (Algorithm 1; root Cholesky and "
                       "triangular inverse of X̄_RR)",
               "scm_panel": "level solves + triangular inverse + X^T X (X̂, Y^-1 formed whole)",
               "scm_tile": "k_scm_hadamard (SCM assembly, B = X̂ o Y^-1 streamed)",
               "scm_chol": "k_chol_dag<double> (SCM Cholesky, FP64 task queue)",
               "scm_chol32": "k_gemm_3xtf32 + 32-column kernels (FP32 SCM Cholesky, tensor cores)",
               "sce_backsolve": "SCE substitutions / refinement",
               "pmatrix": "k_forest_M + forest solve + k_root_pull (+ k_gemm_3xtf32 in FP32) (P-MATRIX)",
               "root_gemm": "k_gemm_tn<double> (P-MATRIX root block M_RR = X̂_RR T, FP64)",
               "primal_step": "k_primal_step + Lanczos (primal step)",
               "dual_step": "Lanczos with Y^-1 (dual step)", "other": "scatter/scalars/update",
               "pmatrix_side": "side-stream P-MATRIX columns",
               "scm_panel_side": "side-stream SCM N solves"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


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


def oracle_chol_sample(m, seed=0):
    """The dense oracle's SCM factorisation at the workload's size: sla.cho_factor of an m x m
    symmetric positive definite matrix (its timing does not depend on the values).  Seconds."""
    import scipy.linalg as sla
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((m, 8))
    B = B @ B.T
    B[np.diag_indices(m)] += m
    t0 = time.perf_counter()
    sla.cho_factor(B, lower=True, overwrite_a=True, check_finite=False)
    return time.perf_counter() - t0


def cpu_sample(m, iters):
    t = oracle_chol_sample(m)
    per_iter = t * ORACLE_ITER_OVER_CHOL
    sample = (f"extrapolated: the oracle's dense SCM Cholesky (sla.cho_factor, {m} x {m}) timed "
              f"once = {t:.2f} s on the host cores, scaled by the dense oracle iteration's flops "
              f"(13 n^3: inverse of Y, two n x n products, two dense step-length eigenproblems, "
              f"the Cholesky) over the Cholesky's (n^3 / 3) and by {iters} iterations (the GPU "
              f"solve's count; the dense oracle's own count at this size is not measured)")
    return t, per_iter * iters, sample


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    m = 20000
    iters = 47
    for _ in range(args.warmup):
        oracle_chol_sample(m)
    ts = [oracle_chol_sample(m) for _ in range(args.steps)]
    t = float(np.mean(ts))
    value = t * ORACLE_ITER_OVER_CHOL * iters
    sample = (f"extrapolated: the oracle's dense SCM Cholesky (sla.cho_factor, {m} x {m}) per step, "
              f"mean {t:.2f} s, scaled by the dense oracle iteration's flops over the Cholesky's (39) "
              f"and by {iters} iterations (the GPU solve's count)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s/solve",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "desc": WORKLOAD_DESC, "precision": "fp64",
                       "step": "one dense SCM Cholesky of the oracle at m = 20000"},
            "cpu_baseline": {"value": value, "unit": "s/solve", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
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


def timed_solves(P, X0, zh, zd, stream, dev, steps):
    """`steps` solves from the fixed start.  Each: the start vector copied from pinned host memory,
    the solve, the solution (X̄ on E, z) copied back to pinned host memory.  Device time of the
    solve alone (CUDA events on the solve's stream) and host wall time of the whole step."""
    import torch
    dev_ms, e2e_ms, res = [], [], []
    Xh = torch.empty(X0.shape, dtype=X0.dtype, pin_memory=True)
    zo = torch.empty(zd.shape, dtype=zd.dtype, pin_memory=True)
    for _ in range(steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        zd.copy_(zh, non_blocking=True)
        P.set_iterate(X0, zd)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = P.solve()
        e1.record(stream)
        X, z, _ = P.get_iterate()
        Xh.copy_(X, non_blocking=True)
        zo.copy_(z, non_blocking=True)
        torch.cuda.synchronize(dev)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        dev_ms.append(e0.elapsed_time(e1))
        res.append(r)
    h2d = zh.numel() * 8
    d2h = Xh.numel() * 8 + zo.numel() * 8
    return dev_ms, e2e_ms, res, h2d, d2h


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
    hbm_peak, bf16_peak, bf16_sus, peak_src = measured_peaks()
    inst = workload(args.workload)
    stream = torch.cuda.current_stream(dev)
    zh = torch.tensor(inst.z0, dtype=torch.float64).pin_memory()
    zd = torch.empty(inst.m, dtype=torch.float64, device=f"cuda:{dev}")

    # ---- headline: the mixed form ----
    t0 = time.perf_counter()
    Pm = Problem(inst.n, inst.m, inst.b, inst.mat, inst.row, inst.col, inst.val, form=1,
                 device=dev, profile=1, precision=1)
    torch.cuda.synchronize(dev)
    create_s = time.perf_counter() - t0
    X0 = Pm.identity_layout()
    timed_solves(Pm, X0, zh, zd, stream, dev, max(args.warmup, 0))
    Pm.stats_reset()
    clocks = Clocks(dev)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    dev_ms, e2e_ms, results, h2d, d2h = timed_solves(Pm, X0, zh, zd, stream, dev, args.steps)
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    mstats = Pm.stats()
    mwork = Pm.work_model()
    total_ms = max_over_ranks(float(np.sum(dev_ms)), f"cuda:{dev}")
    value = job_throughput(total_ms, args.steps, ws)
    e2e_val = job_throughput(max_over_ranks(float(np.sum(e2e_ms)), f"cuda:{dev}"), args.steps, ws)
    rm = results[-1]
    mms = mstats["ms"]
    iters_m = sum(int(x["iters"]) for x in results)
    ok = all(x["status"] == 0 for x in results)
    m = inst.m

    # the FP32 SCM Cholesky on the tensor cores (graded against the TF32 tensor peak): per
    # factorisation, the trailing products run three TF32 products per FP32 product
    tf32_peak = bf16_peak * TF32_BF16_RATIO
    chol32_ms = mms["scm_chol32"]
    # FP32 factorisations: one per iteration up to and including the one that promoted
    nfac = sum((x["promoted_iter"] + 1 if x["promoted_iter"] >= 0 else x["iters"]) for x in results)
    chol_useful = m ** 3 / 3.0
    chol_avg_ms = chol32_ms / max(1, nfac)
    chol_tc = {"kernel": KCLASS_DESC["scm_chol32"], "factorisations": nfac,
               "avg_ms": chol_avg_ms,
               "useful_tflops": chol_useful / (chol_avg_ms * 1e-3) / 1e12 if chol_avg_ms > 0 else None,
               "tensor_tflops": 3 * chol_useful / (chol_avg_ms * 1e-3) / 1e12 if chol_avg_ms > 0 else None,
               "tf32_peak_tflops": tf32_peak,
               "tensor_frac": (3 * chol_useful / (chol_avg_ms * 1e-3) / 1e12) / tf32_peak
               if chol_avg_ms > 0 else None,
               "peak_source": f"{peak_src} bf16 {bf16_peak} TFLOP/s x nominal TF32/BF16 ratio "
                              f"{TF32_BF16_RATIO:.3f}; three TF32 products per FP32 product"}

    # SCM assembly: the streamed Hadamard stage B = X̂ o Y^-1 (reads both matrices' lower
    # triangles, writes lower(B)) and the whole assembly (forming X̂ and Y^-1 included)
    nt = max(1, mstats["count"]["scm_tile"])
    tile_ms = mms["scm_tile"] / nt
    n = inst.n
    asm_iters_fp32 = sum((x["assembly_iter"] if x["assembly_iter"] >= 0 else x["iters"]) for x in results)
    es_mix = (4.0 * asm_iters_fp32 + 8.0 * (iters_m - asm_iters_fp32)) / max(1, iters_m)
    tile_bytes = 2 * es_mix * n * (n + 1) / 2 + 8.0 * m * (m + 1) / 2
    scm = {"stage": "k_scm_hadamard: B = X̂ o Y^-1, lower triangle",
           "bytes_per_launch": tile_bytes, "avg_launch_ms": tile_ms,
           "gbs": tile_bytes / (tile_ms * 1e-3) / 1e9 if tile_ms > 0 else None,
           "hbm_peak_gbs": hbm_peak, "frac": (tile_bytes / (tile_ms * 1e-3) / 1e9) / hbm_peak
           if tile_ms > 0 else None,
           "assembly_ms_per_iter": (mms["scm_panel"] + mms["scm_tile"]) / max(1, iters_m),
           "assembly_bytes_per_iter": mwork["bytes"]["scm_panel"] + mwork["bytes"]["scm_tile"]}

    # roofline of the dominant kernel of the headline solve, among the three single-kernel
    # classes that carry its bulk: the FP64 SCM Cholesky (k_chol_dag, after promotion), the dense
    # root's FP64 P-MATRIX GEMM (k_gemm_tn<double>, X̂_RR T: 2 nR^3 flops) and the FP32 SCM
    # Cholesky on the tensor cores
    nR = int(Pm.info["max_nrow"])
    nfac64 = sum((x["iters"] - x["promoted_iter"] if x["promoted_iter"] >= 0 else 0) for x in results)
    kern = {}
    if mms["scm_chol"] > 0 and nfac64 > 0:
        avg = mms["scm_chol"] / nfac64
        ach = (m ** 3 / 3.0) / (avg * 1e-3) / 1e12
        kern["scm_chol"] = {"bound": "alu", "kernel": KCLASS_DESC["scm_chol"], "achieved": ach,
                            "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                            "traffic": TRAFFIC_PER_UNIT["scm_chol"] * m ** 3,
                            "traffic_note": "ncu on ring_maxcut_8000 scaled by m^3",
                            "avg_launch_ms": avg, "launches": nfac64,
                            "total_ms": mms["scm_chol"], "peak_source": FP64_PEAK_SOURCE}
    if mms["root_gemm"] > 0:
        cnt = max(1, mstats["count"]["root_gemm"])
        avg = mms["root_gemm"] / cnt
        ach = (2.0 * nR ** 3) / (avg * 1e-3) / 1e12
        kern["root_gemm"] = {"bound": "alu", "kernel": KCLASS_DESC["root_gemm"], "achieved": ach,
                             "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                             "traffic": TRAFFIC_PER_UNIT["root_gemm"] * nR ** 3,
                             "traffic_note": "ncu on ring_maxcut_8000 scaled by nR^3",
                             "avg_launch_ms": avg, "launches": cnt,
                             "total_ms": mms["root_gemm"], "peak_source": FP64_PEAK_SOURCE}
    if chol32_ms > 0:
        kern["scm_chol32"] = {"bound": "tensor", "kernel": KCLASS_DESC["scm_chol32"],
                              "achieved": chol_tc["tensor_tflops"], "peak": tf32_peak,
                              "unit": "TFLOP/s", "frac": chol_tc["tensor_frac"], "traffic": None,
                              "avg_launch_ms": chol_avg_ms, "launches": nfac,
                              "total_ms": chol32_ms, "peak_source": chol_tc["peak_source"]}
    dom = max(kern, key=lambda k: kern[k]["total_ms"]) if kern else None
    roof = dict(kern[dom]) if dom else None
    if roof is not None:
        roof["others"] = {k: {"frac": v["frac"], "total_ms": v["total_ms"]} for k, v in kern.items()
                          if k != dom}

    # ---- the FP64 form of the same workload ----
    fp64 = None
    if not args.no_fp64:
        P64 = Problem(inst.n, inst.m, inst.b, inst.mat, inst.row, inst.col, inst.val, form=1,
                      device=dev, profile=1, precision=0)
        d64, e64, r64s, _, _ = timed_solves(P64, X0, zh, zd, stream, dev, 1)
        s64 = P64.stats()
        r64 = r64s[-1]
        fp64 = {"value": d64[-1] * 1e-3, "unit": "s/solve", "iterations": int(r64["iters"]),
                "pobj": r64["pobj"], "dobj": r64["dobj"], "gap": r64["gap"], "pinf": r64["pinf"],
                "status": int(r64["status"]), "e2e_s": e64[-1] * 1e-3,
                "phases_ms_per_solve": {k: v for k, v in s64["ms"].items()},
                "scm_chol_tflops_fp64": (m ** 3 / 3.0) / (s64["ms"]["scm_chol"] / max(1, s64["count"]["scm_chol"]) * 1e-3) / 1e12
                if s64["ms"]["scm_chol"] > 0 else None,
                "root_gemm_tflops_fp64": (2.0 * nR ** 3) / (s64["ms"]["root_gemm"] / max(1, s64["count"]["root_gemm"]) * 1e-3) / 1e12
                if s64["ms"]["root_gemm"] > 0 else None,
                "timing": "one solve after the mixed leg's warm-ups (same kernels warmed)"}
        del P64
        torch.cuda.empty_cache()

    batched = context = None
    if args.legs == "all":
        context, batched = other_legs(args, dev, stream)

    line = None
    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            t, v, sample = cpu_sample(m, int(rm["iters"]))
            cpu = {"value": v, "unit": "s/solve", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": sample}
        mixed = {"value": value, "unit": "s/solve", "iterations": int(rm["iters"]),
                 "pobj": rm["pobj"], "dobj": rm["dobj"], "gap": rm["gap"], "pinf": rm["pinf"],
                 "assembly_iter": int(rm["assembly_iter"]), "promoted_iter": int(rm["promoted_iter"]),
                 "refine_steps": int(rm["refine_steps"]),
                 "speedup_vs_fp64": (fp64["value"] / value) if fp64 else None,
                 "pobj_diff_vs_fp64": abs(rm["pobj"] - fp64["pobj"]) if fp64 else None,
                 "phases_ms_per_solve": {k: v / args.steps for k, v in mms.items()},
                 "desc": ("FP32 stage (relative gap above 1e-2): X̂ and Y^-1 formed in FP32, the "
                          "root blocks of Y and X̄ factored (X̄_RR's factor inverted) in FP32, the "
                          "root's products and the SCM Cholesky's trailing updates on the tensor "
                          "cores (three TF32 products), the SCE corrected in FP64 by GMRES "
                          "preconditioned by the equilibrated FP32 factor, the direction "
                          "projected onto the primal affine set in FP64; then FP64 assembly with "
                          "the FP32 tensor-core factor and GMRES; FP64 factorisations of B once "
                          "GMRES stalls or the FP32 factor breaks down; the forest's factors, "
                          "step-length bounds and update FP64")}
        line = {"metric": METRIC, "value": value, "unit": "s/solve", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic",
                "config": {"workload": args.workload,
                           "desc": WORKLOAD_DESC if args.workload == WORKLOAD else args.workload,
                           "precision": "mixed",
                           "iterations": int(rm["iters"]), "pobj": rm["pobj"], "gap": rm["gap"],
                           "all_optimal": ok, "create_s": create_s,
                           "l2": "inputs larger than L2 (X̂, Y^-1 and B are 1.6-3.2 GB each)",
                           "parallelism": f"replicas x{ws}"},
                "roofline": roof, "scm_assembly": scm, "scm_cholesky_tc": chol_tc,
                "mixed": mixed, "fp64": fp64, "context": context, "batched": batched,
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_val, "unit": "s/solve", "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "gpu_launches": int(mstats["launches"]),
                "gpu_launches_per_solve": mstats["launches"] / args.steps, "clocks": clk}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def other_legs(args, dev, stream):
    """Context: the n = 2020 block-arrow SDP (FP64 and mixed, small cliques, no dense root) and
    the batched form on a mix of small SDPs."""
    import torch
    from instances import workload, batch_mix
    from paper_1310_6919_gb300 import Problem, solve_batch, MCSDPError, tune, tune_cache_clear
    inst = workload(CONTEXT_WORKLOAD)
    z0 = torch.tensor(inst.z0, dtype=torch.float64, device=f"cuda:{dev}")
    out = {"workload": CONTEXT_WORKLOAD}
    for name, prec in (("fp64", 0), ("mixed", 1)):
        P = Problem(inst.n, inst.m, inst.b, inst.mat, inst.row, inst.col, inst.val, form=1,
                    device=dev, precision=prec)
        X0 = P.identity_layout()
        for _ in range(3):
            P.set_iterate(X0, z0)
            P.solve()
        ts = []
        for _ in range(3):
            P.set_iterate(X0, z0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = P.solve()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        out[name] = {"s_per_solve": float(np.median(ts)) * 1e-3, "iterations": int(r["iters"]),
                     "pobj": r["pobj"], "status": int(r["status"])}
        del P
    # config 4: 512 max-cut + 128 block-arrow SDPs, each form through mcsdp_solve_batch (host
    # threads, one stream per problem); one at a time on a 64-problem subset for comparison
    mix = batch_mix(512, 128)
    subset = set(range(48)) | set(range(512, 528))

    def make(inst, st, prec, graph=0, **opts):
        Q = Problem(inst.n, inst.m, inst.b, inst.mat, inst.row, inst.col, inst.val, form=1,
                    device=dev, stream=st, precision=prec, graph=graph, **opts)
        if inst.meta.get("kind") != "maxcut":
            Q.set_iterate(None, torch.tensor(inst.z0, dtype=torch.float64, device=f"cuda:{dev}"))
        return Q

    batched = {"problems": len(mix),
               "desc": ("512 max-cut G(n, 5n/2), n ~ U{50..400}, w ~ U[0,1) and 128 block-arrow "
                        "SDPs, n ~ U{100..600}, border 20, m = n (seeded); host wall time, inputs "
                        "resident; one-at-a-time on the 64-problem subset (first 48 max-cut, first "
                        "16 block-arrow)")}
    make(mix[0], None, 0).solve()
    # fp64: iterations replayed as captured CUDA graphs (options.graph); fp64_host_loop: the
    # host-driven loop (about a hundred launches and eight synchronisations per iteration);
    # fp64_tuned: the graph form with each problem's SCM grouping from the tile-shape tuner
    # (mcsdp_tune, cached per (n, m, largest clique) bucket; tuning time reported apart)
    tuned, keys, t_tune = {}, set(), 0.0
    tune_cache_clear()
    t0 = time.perf_counter()
    for i, q in enumerate(mix):
        try:
            o, info = tune(q, z0=None if q.meta.get("kind") == "maxcut" else q.z0, iters=3,
                           device=dev, graph=1)
            tuned[i] = {"group_max": o["group_max"], "panel_max": o["panel_max"]}
            keys.add(tuple(info["key"]))
        except MCSDPError:
            pass
    torch.cuda.synchronize(dev)
    t_tune = time.perf_counter() - t0
    for name, prec, graph in (("fp64", 0, 1), ("fp64_host_loop", 0, 0), ("mixed", 1, 0),
                              ("fp64_tuned", 0, 1)):
        probs, idx, skipped = [], [], 0
        for i, q in enumerate(mix):
            try:
                extra = tuned.get(i, {}) if name == "fp64_tuned" else {}
                probs.append(make(q, torch.cuda.Stream(dev), prec, graph, **extra))
                idx.append(i)
            except MCSDPError:
                skipped += 1
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        res = solve_batch(probs, nthreads=16)
        torch.cuda.synchronize(dev)
        t_bat = time.perf_counter() - t0
        leg = {"problems_per_s": len(probs) / t_bat, "seconds": t_bat, "skipped": skipped,
               "all_optimal": all(r["status"] == 0 for r in res)}
        if name == "fp64":
            seq = [make(mix[i], None, 0) for i in sorted(subset)]
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            seq_res = [Q.solve() for Q in seq]
            torch.cuda.synchronize(dev)
            t_seq = time.perf_counter() - t0
            bat_sub = {i: r for i, r in zip(idx, res)}
            leg["sequential_problems_per_s_subset"] = len(seq) / t_seq
            leg["speedup_vs_sequential"] = leg["problems_per_s"] / (len(seq) / t_seq)
            leg["same_as_sequential_subset"] = all(
                bat_sub[i]["pobj"] == r["pobj"] for i, r in zip(sorted(subset), seq_res) if i in bat_sub)
            del seq
        if name == "fp64_tuned":
            leg["tuning_seconds"] = t_tune
            leg["tuned_keys"] = len(keys)
            choice = {}
            for v in tuned.values():
                k = f"{v['group_max']}x{v['panel_max']}"
                choice[k] = choice.get(k, 0) + 1
            leg["choices"] = choice
            leg["speedup_vs_fp64"] = leg["problems_per_s"] / batched["fp64"]["problems_per_s"]
        batched[name] = leg
        del probs
        torch.cuda.empty_cache()
    try:
        out["scm_blocks"] = blocks_leg(dev, stream)
    except Exception as e:  # a failed side leg is reported, not allowed to drop the line
        out["scm_blocks"] = {"error": f"{type(e).__name__}: {e}"}
    return out, batched


def blocks_leg(dev, stream):
    """The block-diagonal SCM (the sparse-SCM case): 64 random max-cut SDPs as one SDP, solved
    with B assembled and factored block by block, and the whole-matrix factorisation of the same
    B for three iterations (its per-iteration time; a whole solve would take minutes)."""
    import torch
    from instances import workload
    from paper_1310_6919_gb300 import Problem
    inst = workload(BLOCKS_WORKLOAD)
    z0 = torch.tensor(inst.z0, dtype=torch.float64, device=f"cuda:{dev}")

    def run(max_iter, **o):
        P = Problem.from_instance(inst, device=dev, profile=1, max_iter=max_iter, **o)
        P.set_iterate(None, z0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = P.solve()
        e1.record(stream)
        e1.synchronize()
        st = P.stats()
        it = max(1, int(r["iters"]))
        chol = (st["ms"]["scm_chol"] + st["ms"]["sce_backsolve"]) / it
        return r, e0.elapsed_time(e1), chol, P.info

    run(100)  # warm-up (kernel attributes, first-use paths)
    r, ms, chol, info = run(100)
    it = max(1, int(r["iters"]))
    out = {"workload": BLOCKS_WORKLOAD, "n": inst.n, "m": inst.m, "components": info["ncomp"],
           "scm_density": float(sum(p[2] ** 2 for p in inst.meta["parts"])) / inst.m ** 2,
           "blocks": {"s_per_solve": ms * 1e-3, "iterations": it, "status": int(r["status"]),
                      "pobj": r["pobj"], "gap": r["gap"], "ms_per_iter": ms / it,
                      "scm_factor_solve_ms_per_iter": chol}}
    r1, ms1, chol1, _ = run(3, scm_blocks=1)
    it1 = max(1, int(r1["iters"]))
    out["whole"] = {"iterations": it1, "ms_per_iter": ms1 / it1, "scm_factor_solve_ms_per_iter": chol1}
    out["factor_solve_speedup"] = chol1 / chol if chol > 0 else None
    out["timing"] = ("CUDA events around mcsdp_solve with per-class profiling on (profile = 1); "
                     "the factor+solve figures are the scm_chol + sce_backsolve classes")
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="leave out the FP64 leg")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="named workload of the timed legs (default: the headline's)")
    ap.add_argument("--legs", default="all", choices=["all", "main"],
                    help="main: only the config-3 legs (mixed headline and FP64)")
    ap.add_argument("--newton-steps", type=int, default=0,
                    help="profiling entry, not a bench run: this many Newton steps of the "
                         "workload at its start point (--precision), per-class device times "
                         "printed; no JSON line")
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1],
                    help="form of the --newton-steps run")
    args = ap.parse_args()
    if args.newton_steps > 0:
        return newton_steps(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gb300(args)


def newton_steps(args):
    """K Newton steps (mcsdp_newton_step) at (X̄ = I, z0) of the named workload: the command the
    per-kernel profiles are captured with (one step runs every kernel of one iteration)."""
    import torch
    from paper_1310_6919_gb300 import Problem, build_library
    from instances import workload
    build_library()
    inst = workload(args.workload)
    P = Problem.from_instance(inst, device=0, precision=args.precision, profile=1)
    X0 = P.identity_layout()
    z0 = torch.tensor(inst.z0, dtype=torch.float64, device="cuda:0")
    for k in range(args.newton_steps):
        st = P.newton_step(X0, z0)
        print(f"step {k}: alpha_p {st['alpha_p']:.4f} alpha_d {st['alpha_d']:.4f}", flush=True)
    s = P.stats()
    print("ms per class", json.dumps({k: round(v, 3) for k, v in s["ms"].items() if v > 0}),
          "launches", s["launches"], "root rows", P.info["max_nrow"], flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
