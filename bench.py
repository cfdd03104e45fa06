#!/usr/bin/env python3
"""Benchmark of the FMM-preconditioned 3D Helmholtz solve on GB300.

One step = one right-preconditioned GMRES solve to a relative residual of
1e-6 of the 7-point FDM system -Lap u - k^2 u = f on 64^3 interior nodes
(k = 16, p = 6, leaf 64, theta = 0.4, GMRES(50), f = 8 Gaussian sources on a
uniform[-1,1] background), preconditioned by the BEM-coupled FMM with its FMM
stages in FP32 (complex64), the inner boundary solve in complex64 and the
outer GMRES in FP64.  The tree and operators are built before the timed
region (reported as build_s).

Printed JSON line (rank 0):
  value        seconds per solve (time-to-1e-6, device time, inputs resident),
               K solves with no instrumentation
  e2e          the same through host buffers (H2D of f, D2H of u inside)
  roofline     the near-field kernel (largest share of device time): live
               CUDA-event timers around its launches over a second pass of the
               K solves, 23 flop-equivalents per pair against the FP32 FMA
               rate measured by hfmm_pipe_peaks; per pass beside it
  pipe_peaks   the measured pipe rates (FP32, FP64, XU, shared memory, TF32)
  cpu_baseline the FP64 CPU oracle on a bounded sample, scaled to one solve
  fp64         the plain FP64 form of the same solve (time, iterations)
  n128         one FP32 solve of the 128^3, k = 32, p = 8 workload
  bicgstab     BiCGSTAB with the same preconditioner (time, iterations, applies)
  fmm_apply_mpts_s  (N_vol + N_bnd) / time of one full FMM apply (FP32 form)

--impl reference times the oracle alone on the host (bounded sample).
Multi-GPU (torchrun): every rank solves its own replica (replicas only).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GMRES time-to-1e-6 and FMM apply Mpts/s: FP32/batched vs plain FP64, same GB300"
WORKLOAD = "helmholtz_n64_k16_p6"

# Algorithmic work of one near-field pair, as a direct evaluation counts it:
# 3 subtractions, 5 for r^2, 1 rsqrt, 1 for r, 1 for kr, sin + cos, 2 for G,
# 6 for the complex product with q, 2 for the accumulation: about 23
# flop-equivalents (3 of them XU ops).  The roofline divides 23 x pairs/s by
# the measured FP32 (FP64) FMA rate, the busiest pipe of that evaluation.
P2P_FLOP_EQ_PER_PAIR = 23
P2P_XU_OPS_PER_PAIR = 3
# The FP32 lattice kernel replaces that evaluation by a table: per pair one
# 8-byte table entry and a quarter of a 16-byte staged source record come
# from shared memory, so shared-memory loads bound it (secondary figure).
P2P_SMEM_BYTES_PER_PAIR = 12
# dram__bytes_read.sum + dram__bytes_write.sum of one k_p2p_lat launch (ncu,
# 64^3 k=16 p=6 FP32 workload) for the three passes of the preconditioner:
# volume -> boundary, boundary -> boundary, all -> volume
P2P_DRAM_BYTES = {"A": 2617088, "B": 520704, "C": 5694976}
# The boundary operator's kernel (k_bnd_op, one launch = one inner GMRES
# cycle): dram__bytes_read.sum + dram__bytes_write.sum of one such launch in
# the benchmark solve (ncu, 64^3 k=16 p=6 FP32, 20 steps), and its steps
BND_DRAM_BYTES = 264148224
# pass C's volume near field runs on the tensor cores in the FP32 form
# (several launches), so the per-launch near-field counters above do not apply
NEAR_TC_IN_STAGE = True
BND_DRAM_STEPS = 20
L2_FLUSH_BYTES = 512 << 20  # larger than the 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--inner-rtol", type=float, default=1e-2)
    ap.add_argument("--inner-maxit", type=int, default=20)
    ap.add_argument("--inner-p", type=int, default=0,
                    help="expansion order of the inner solve's boundary -> boundary applies "
                         "(0: the workload's p)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 48-solve batched measurement")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default kernel variants and tile shapes (no fmm_autotune before timing)")
    ap.add_argument("--no-big", action="store_true", help="skip the 128^3 solve")
    ap.add_argument("--no-bicgstab", action="store_true", help="skip the BiCGSTAB solve of the same system")
    ap.add_argument("--dirichlet", action="store_true",
                    help="also time the solve with Dirichlet data (plane-wave boundary values): "
                         "the FDM system with the boundary lift, from zero and from the BEM "
                         "solution with the data, and the double-layer FMM apply")
    ap.add_argument("--batched-maxit", type=int, default=200)
    ap.add_argument("--sweep", choices=("kh", "p"),
                    help="print one JSON line per point of a sweep (fixed kh = 0.3125 over n, or the "
                         "expansion order p at n = 31, k = 10) instead of the benchmark line")
    ap.add_argument("--apply-only", nargs=2, type=int, metavar=("SRC", "TGT"),
                    help="profiling case: build the tree and run two FMM applies with these "
                         "source/target set masks (1 volume, 2 boundary, 3 both), print nothing else")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, enabled, gpu_index):
        self.proc = None
        self.path = None
        self.gpu_index = gpu_index
        if not enabled:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(r[0] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier_max(value, world, device):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ oracle timing

def oracle_sample(w, inner_per_apply, outer_iters, leaf_fraction=1.0 / 16):
    """Time the FP64 CPU oracle on a bounded sample of one solve and scale it to
    seconds per solve.  The far field (P2M, M2M, M2L, L2L) of the three FMM
    passes of a preconditioner application runs in full; the near field (P2P)
    runs for the targets in a random subset of leaves and is scaled by the
    fraction of target points sampled.  Returns (seconds_per_solve, text)."""
    from oracle import bem, fdm
    t0 = time.perf_counter()
    pr = bem.Problem(w["n"], w["k"], w["p"], w["leaf"], w["theta"])
    f = pr.fmm
    rng = np.random.default_rng(0)
    q = rng.standard_normal(pr.NO + pr.NG) + 1j * rng.standard_normal(pr.NO + pr.NG)

    def far(src, tgt):
        L = f.L
        M = {L: f.p2m(q, src)}
        for l in range(L - 1, 1, -1):
            M[l] = f.m2m(M[l + 1], l)
        Lc = {l: f.m2l(M[l], l) for l in range(2, L + 1)}
        for l in range(2, L):
            Lc[l + 1] = f.l2l(Lc[l], Lc[l + 1], l)
        return f.l2p(Lc[L], tgt)

    def timed(fn):
        a = time.perf_counter()
        fn()
        return time.perf_counter() - a

    far(pr.vol, pr.bnd)          # translation operators are built on first use: not timed
    leaves = np.unique(f.tree.leaf)
    pick = rng.choice(leaves, size=max(1, int(leaf_fraction * len(leaves))), replace=False)
    sel = np.isin(f.tree.leaf, pick)
    tv = pr.vol & sel
    tb = pr.bnd & sel
    sv = pr.NO / max(1, tv.sum())
    sb = pr.NG / max(1, tb.sum())
    t_a = timed(lambda: far(pr.vol, pr.bnd)) + sb * timed(lambda: f.p2p(q, pr.vol, tb))
    t_b = timed(lambda: far(pr.bnd, pr.bnd)) + sb * timed(lambda: f.p2p(q, pr.bnd, tb))
    t_c = timed(lambda: far(pr.vol | pr.bnd, pr.vol)) + sv * timed(lambda: f.p2p(q, pr.vol | pr.bnd, tv))
    t_fdm = timed(lambda: fdm.fdm_apply(q[:pr.NO], w["n"], w["k"]))
    per_apply = t_a + inner_per_apply * t_b + t_c
    per_solve = outer_iters * (per_apply + t_fdm)
    desc = (f"oracle FMM passes at {w['n']}^3 (A: vol->bnd, B: bnd->bnd, C: all->vol): far field in "
            f"full, P2P for targets in {len(pick)}/{len(leaves)} random leaves scaled by point "
            f"fraction; per solve = {outer_iters} x (A + {inner_per_apply:.1f} B + C + FDM); "
            f"sample wall {time.perf_counter() - t0:.1f} s")
    return per_solve, desc


def torch_threads():
    try:
        import torch
        return torch.get_num_threads()
    except Exception:
        return os.cpu_count()


# ------------------------------------------------------------------ arms

def run_reference(args, world, rank):
    """The oracle alone on the host: each step times a bounded sample of the
    same workload scaled to one solve.  The iteration counts come from the
    oracle's own recorded solve when present, else from the paper-free default
    (one outer iteration per step)."""
    if rank != 0:
        return
    from paper_1608_02461_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    golden = os.path.join(ROOT, "tests", "golden", f"oracle_{args.workload}.json")
    if os.path.exists(golden):
        g = json.load(open(golden))
        outer, inner = g["iters"], g["inner_iters_total"] / max(1, g["iters"])
        basis = "iteration counts of the oracle's recorded FP64 solve"
    else:
        outer, inner = 1, 10.0
        basis = "one outer iteration with 10 inner iterations (no recorded oracle solve)"
    times = []
    desc = ""
    for i in range(args.warmup + args.steps):
        v, desc = oracle_sample(w, inner, outer)
        if i >= args.warmup:
            times.append(v)
    val = float(np.mean(times))
    cores = torch_threads()
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": val * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, **{k: w[k] for k in ("n", "k", "p", "leaf", "theta")}},
            "cpu_baseline": {"value": val, "unit": "s", "cores": cores, "kind": "oracle",
                             "sample": desc + "; " + basis},
            "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def p2p_roofline(live, pk, lattice, info, bench_workload, passb_kernel, steps):
    """Roofline object of the near-field stage from its stage timers: (ms,
    launches, point pairs) over the timed solves.  The stage is the lattice
    kernel k_p2p_lat, and in passes with volume targets on a regular lattice
    the volume sources' part on the tensor cores (k_tc_near_split, k_m2l_tc,
    k_tc_reduce, k_tc_near_add) with k_p2p_lat for the boundary sources.
    passb_kernel: the boundary -> boundary applies ran in the one-kernel
    boundary operator (no near-field stage there).  Per apply: the solves'
    preconditioner applications x passes A and C."""
    sm_, nl_, work_ = live
    pairs_s = work_ / (sm_ * 1e-3) if sm_ > 0 else 0.0
    achieved = P2P_FLOP_EQ_PER_PAIR * pairs_s / 1e12
    peak = pk["fp32_tflops"] if lattice else pk["fp64_tflops"]
    # DRAM counters exist for the single-kernel near field only (pass C's
    # volume part now runs as several tensor-core launches)
    traffic = None
    if lattice and bench_workload and not passb_kernel and not NEAR_TC_IN_STAGE:
        na, nb_, nc = info.iters, info.inner_iters_total, info.iters
        traffic = (na * P2P_DRAM_BYTES["A"] + nb_ * P2P_DRAM_BYTES["B"] + nc * P2P_DRAM_BYTES["C"]) / (na + nb_ + nc)
    napply = max(1, 2 * info.iters * steps)
    roof = {"bound": "alu", "kernel": "near-field stage (k_p2p_lat; pass C's volume sources on the tensor cores)",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "peak_kind": "measured",
            "peak_source": ("FP32" if lattice else "FP64") + " FMA rate measured by hfmm_pipe_peaks",
            "per_apply_ms": sm_ / napply, "work_per_apply": work_ / napply, "launches": nl_,
            "work_unit": f"point pairs, {P2P_FLOP_EQ_PER_PAIR} flop-equivalents each",
            "gpair_s": pairs_s / 1e9,
            "frac_of_xu": P2P_XU_OPS_PER_PAIR * pairs_s / (pk["xu_gops"] * 1e9),
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, weighted by the "
                               "solve's pass mix") if traffic is not None else None,
            "source": "CUDA events around every launch of the kernel (on its own stream) over a second pass "
                      "of the K timed solves; the headline pass runs without them"}
    if lattice:
        roof["smem"] = {"bytes_per_pair": P2P_SMEM_BYTES_PER_PAIR,
                        "achieved_gbs": P2P_SMEM_BYTES_PER_PAIR * pairs_s / 1e9, "peak_gbs": pk["smem_gbs"],
                        "frac": P2P_SMEM_BYTES_PER_PAIR * pairs_s / (pk["smem_gbs"] * 1e9)}
    return roof


def bnd_roofline(live, pk, lattice, info, w, hfmm, dev):
    """Roofline object of the boundary operator's kernel (one launch = one
    inner GMRES cycle of Pass B applies): algorithmic work per step = the
    boundary -> boundary M2L (8 P^2 flop per cell pair) + the near field (23
    flop-equivalents per point pair), counted by the library's stage counters
    on a stage-chain apply of the same tree geometry; steps per launch = inner
    steps of the timed solves / launches; time = CUDA events around every
    launch (live, over the second pass of the K solves)."""
    import torch
    sm_, nl_, _ = live
    old = os.environ.get("HFMM_BND_OP")
    os.environ["HFMM_BND_OP"] = "0"  # the stage chain counts the work of each stage
    try:
        tc = hfmm.Tree(w["n"], w["k"], w["p"], w["theta"], w["leaf"], "fp32" if lattice else "fp64")
    finally:
        if old is None:
            os.environ.pop("HFMM_BND_OP", None)
        else:
            os.environ["HFMM_BND_OP"] = old
    qb = torch.zeros(tc.n_bnd, dtype=torch.complex128, device=dev)
    tc.set_timing(True)
    tc.apply(None, qb, src=hfmm.SET_BND, tgt=hfmm.SET_BND)
    torch.cuda.synchronize()
    st = tc.stage_times()
    tc.set_timing(False)
    tc.close()
    m2l_flop, p2p_pairs = st["m2l"][2], st["p2p"][2]
    per_step = m2l_flop + P2P_FLOP_EQ_PER_PAIR * p2p_pairs
    steps = info.inner_iters_total / max(1, info.iters)  # one cycle launch per outer iteration
    per_launch_ms = sm_ / max(1, nl_)
    work = per_step * steps
    achieved = work / (per_launch_ms * 1e-3) / 1e12 if per_launch_ms > 0 else 0.0
    peak = pk["fp32_tflops"] if lattice else pk["fp64_tflops"]
    traffic = None
    if BND_DRAM_BYTES is not None and lattice:
        traffic = BND_DRAM_BYTES * steps / BND_DRAM_STEPS
    return {"bound": "alu", "kernel": "k_bnd_op", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "peak_kind": "measured",
            "peak_source": ("FP32" if lattice else "FP64") + " FMA rate measured by hfmm_pipe_peaks",
            "per_launch_ms": per_launch_ms, "work_per_launch": work, "steps_per_launch": steps,
            "work_unit": f"flop-equivalents: 8 P^2 per M2L cell pair + {P2P_FLOP_EQ_PER_PAIR} per near-field "
                         "point pair, boundary -> boundary, per inner step",
            "m2l_flop_per_step": m2l_flop, "p2p_pairs_per_step": p2p_pairs,
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one cycle launch of the "
                               "benchmark solve, scaled by steps") if traffic is not None else None,
            "source": "CUDA events around every launch of the kernel over a second pass of the K timed "
                      "solves; the headline pass runs without them"}


def p2p_per_pass(tree, hfmm, inputs, n, dev, pk, lattice, reps=10):
    """Near-field rate of each pass of the preconditioner (A: volume ->
    boundary, B: boundary -> boundary, C: all -> volume) from standalone
    applies with the near-field stage timed."""
    import torch
    peak = pk["fp32_tflops"] if lattice else pk["fp64_tflops"]
    qv = torch.from_numpy(inputs.complex_normal(n ** 3, 53)).to(dev)
    qb = torch.from_numpy(inputs.complex_normal(6 * n * n, 54)).to(dev)
    out = {}
    for name, src, tgt in (("A", hfmm.SET_VOL, hfmm.SET_BND), ("B", hfmm.SET_BND, hfmm.SET_BND),
                           ("C", hfmm.SET_VOL | hfmm.SET_BND, hfmm.SET_VOL)):
        pv, pb = tree.apply(qv, qb, src=src, tgt=tgt)
        tree.set_timing(True, stages=["p2p"])
        for _ in range(reps):
            tree.apply(qv, qb, src=src, tgt=tgt, phi_vol=pv, phi_bnd=pb)
        torch.cuda.synchronize()
        ms, nl, work = tree.stage_times()["p2p"]
        tree.set_timing(False)
        if nl == 0 or ms <= 0:  # the pass ran as the one-kernel boundary operator
            out[name] = {"per_apply_ms": None, "note": "near field inside the boundary-operator kernel"}
            continue
        pairs_s = work / (ms * 1e-3)
        out[name] = {"per_apply_ms": ms / reps, "launches_per_apply": nl / reps, "gpair_s": pairs_s / 1e9,
                     "achieved": P2P_FLOP_EQ_PER_PAIR * pairs_s / 1e12,
                     "frac": P2P_FLOP_EQ_PER_PAIR * pairs_s / 1e12 / peak}
    return out


def run_ours(args, world, rank, local):
    import torch
    from __graft_entry__ import build
    build()
    from paper_1608_02461_gb300 import hfmm, inputs

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    w = inputs.WORKLOADS[args.workload]
    n = w["n"]
    gm = dict(restart=w["restart"], rtol=1e-6, inner_rtol=args.inner_rtol, inner_maxit=args.inner_maxit,
              inner_m=args.inner_maxit)

    t0 = time.perf_counter()
    tree = hfmm.Tree(n, w["k"], w["p"], w["theta"], w["leaf"], args.precision)
    if args.inner_p:
        tree.set_inner_order(args.inner_p)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    # kernel variants and tile shapes picked by timing (outside the timed
    # region, like the tree build)
    t0 = time.perf_counter()
    if not args.no_autotune:
        tree.autotune()
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    b_host = inputs.workload_rhs(args.workload)
    b = torch.from_numpy(b_host).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def solve():
        x, info = tree.gmres(b, **gm)
        return x, info

    for _ in range(args.warmup):
        x, info = solve()
    assert info.status == 0, f"warm-up solve did not converge: {info}"

    # per-stage times of one solve with every stage timed (reported, not the value)
    tree.set_timing(True)
    solve()
    torch.cuda.synchronize()
    stages = tree.stage_times()
    tree.set_timing(False)
    # the kernel with the largest share of device time in the launch list: the
    # boundary operator's (the inner solves) when it serves Pass B, else the
    # near field
    dom = "bnd" if stages["bnd"][1] > 0 else "p2p"
    pk = hfmm.pipe_peaks()

    # the headline: K solves with no instrumentation
    clocks = ClockSampler(not args.no_clocks and rank == 0, local)
    launches0 = tree.stats().launches
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    evs = []
    infos = []
    for _ in range(args.steps):
        flush.fill_(1.0)                      # evict L2 between steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, info = solve()
        e1.record(stream)
        evs.append((e0, e1))
        infos.append(info)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    st = tree.stats()
    launches = st.launches - launches0
    ms = sum(a.elapsed_time(c) for a, c in evs) / args.steps
    ms = barrier_max(ms, world, dev)
    info = infos[-1]
    relres = info.relres_true

    # the roofline pass: the same K solves again, with CUDA events around
    # every launch of the near-field kernel (on the stream each launch uses)
    tree.set_timing(True, stages=sorted({dom, "p2p"}))
    for _ in range(args.steps):
        flush.fill_(1.0)
        solve()
    torch.cuda.synchronize()
    live = tree.stage_times()
    tree.set_timing(False)
    lattice = args.precision == "fp32"
    roof_p2p = p2p_roofline(live["p2p"], pk, lattice, info, args.workload == WORKLOAD, stages["bnd"][1] > 0,
                            args.steps)
    roof_p2p["per_pass"] = p2p_per_pass(tree, hfmm, inputs, n, dev, pk, lattice)
    roof = bnd_roofline(live["bnd"], pk, lattice, info, w, hfmm, dev) if dom == "bnd" else roof_p2p
    stage_summary = {k: {"ms": v[0], "launches": v[1]} for k, v in stages.items()}
    # the far field's M2L stage over one fully timed solve (outside the timed
    # region): algorithmic 8 P^2 flop per cell pair over all its launches
    # (tensor-core kernel at levels >= 4 of the volume-target pass, CUDA-core
    # pipelines and pair lists elsewhere)
    m2l_ms, m2l_nl, m2l_flop = stages["m2l"]
    roof_m2l = None
    if m2l_ms > 0 and m2l_flop > 0 and pk is not None:
        a2 = m2l_flop / (m2l_ms * 1e-3) / 1e12
        p2 = pk["fp32_tflops"] if lattice else pk["fp64_tflops"]
        roof_m2l = {"bound": "alu", "kernel": "M2L stage (k_m2l_tc, k_m2l_ws, k_m2l_pairs)", "achieved": a2,
                    "peak": p2, "unit": "TFLOP/s", "frac": a2 / p2, "launches": m2l_nl,
                    "ms_per_solve": m2l_ms, "work_unit": "8 P^2 flop per cell pair",
                    "peak_kind": "measured",
                    "peak_source": ("FP32 FMA rate measured by hfmm_pipe_peaks" if lattice
                                    else "FP64 FMA rate measured by hfmm_pipe_peaks"),
                    # tensor-core M2L in FP32 accuracy: three TF32 products per
                    # algorithmic one, against the measured tcgen05 TF32 rate
                    "frac_of_tf32_tensor": (a2 / (pk["tf32_tflops"] / 3)) if lattice else None,
                    "source": "stage timers of one fully timed solve (outside the timed region)"}

    # FMM apply throughput (full apply, all points sources and targets)
    qv = torch.from_numpy(inputs.complex_normal(n ** 3, 51)).to(dev)
    qb = torch.from_numpy(inputs.complex_normal(6 * n * n, 52)).to(dev)
    pv, pb = tree.apply(qv, qb)
    torch.cuda.synchronize()
    reps = 5
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    app_ms = 0.0
    for _ in range(reps):
        flush.fill_(1.0)
        e0.record(stream)
        tree.apply(qv, qb, phi_vol=pv, phi_bnd=pb)
        e1.record(stream)
        torch.cuda.synchronize()
        app_ms += e0.elapsed_time(e1)
    app_ms /= reps
    mpts = (n ** 3 + 6 * n * n) / (app_ms * 1e-3) / 1e6

    # end to end through host buffers
    b_pin = torch.from_numpy(b_host).pin_memory()
    x_pin = torch.empty_like(b_pin).pin_memory()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0.record(stream)
        bd = b_pin.to(dev, non_blocking=True)
        xd, _ = tree.gmres(bd, **gm)
        x_pin.copy_(xd, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_ms /= args.steps
    e2e_ms = barrier_max(e2e_ms, world, dev)
    nbytes = b_pin.numel() * b_pin.element_size()

    # plain FP64 form of the same solve
    fp64 = None
    if not args.no_fp64 and args.precision == "fp32":
        t64 = hfmm.Tree(n, w["k"], w["p"], w["theta"], w["leaf"], "fp64")
        if not args.no_autotune:
            t64.autotune()
        t64.gmres(b, **gm)          # warm-up
        flush.fill_(1.0)
        e0.record(stream)
        _, i64 = t64.gmres(b, **gm)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64 = {"time_to_solution_s": e0.elapsed_time(e1) * 1e-3, "gmres_iters": i64.iters,
                "inner_iters_total": i64.inner_iters_total, "relres_true": i64.relres_true,
                "iters_ratio_fp32_over_fp64": info.iters / max(1, i64.iters)}
        t64.close()

    # the FP32 form at scale: one solve of the 128^3 workload (k = 32, p = 8,
    # theta = 0.35), timed like a step (L2 flushed, device time)
    big = None
    if not args.no_big and args.workload == WORKLOAD and args.precision == "fp32":
        name_b = "helmholtz_n128_k32_p8"
        wb = inputs.WORKLOADS[name_b]
        tb0 = time.perf_counter()
        t128 = hfmm.Tree(wb["n"], wb["k"], wb["p"], wb["theta"], wb["leaf"], "fp32")
        torch.cuda.synchronize()
        build_b = time.perf_counter() - tb0
        if not args.no_autotune:
            t128.autotune()
        bb = torch.from_numpy(inputs.workload_rhs(name_b)).to(dev)
        gmb = dict(gm, restart=wb["restart"])
        t128.gmres(bb, **gmb)          # warm-up
        flush.fill_(1.0)
        e0.record(stream)
        _, ib128 = t128.gmres(bb, **gmb)
        e1.record(stream)
        torch.cuda.synchronize()
        big = {"workload": name_b, "time_to_solution_s": e0.elapsed_time(e1) * 1e-3,
               "gmres_iters": ib128.iters, "inner_iters_total": ib128.inner_iters_total,
               "relres_true": ib128.relres_true, "converged": ib128.status == 0, "build_s": build_b}
        t128.close()
        del bb

    # BiCGSTAB with the same preconditioner (the paper's GMRES / BiCGSTAB
    # comparison).  BiCGSTAB needs a nearly fixed preconditioner: with the
    # benchmark's loose inner solve it stagnates, so both methods are run here
    # with the inner boundary solve to 1e-4 (at most 120 steps)
    bicg = None
    if not args.no_bicgstab:
        ikw = dict(inner_rtol=1e-4, inner_maxit=120, inner_m=120)
        tree.bicgstab(b, rtol=1e-6, maxit=200, **ikw)   # warm-up
        flush.fill_(1.0)
        e0.record(stream)
        _, ib = tree.bicgstab(b, rtol=1e-6, maxit=200, **ikw)
        e1.record(stream)
        torch.cuda.synchronize()
        tb_ = e0.elapsed_time(e1) * 1e-3
        flush.fill_(1.0)
        e0.record(stream)
        _, ig = tree.gmres(b, restart=w["restart"], rtol=1e-6, **ikw)
        e1.record(stream)
        torch.cuda.synchronize()
        bicg = {"inner_rtol": 1e-4, "inner_maxit": 120,
                "time_to_solution_s": tb_, "iters": ib.iters, "precond_applies": ib.restarts,
                "inner_iters_total": ib.inner_iters_total, "relres_true": ib.relres_true,
                "converged": ib.status == 0,
                "gmres_same_inner": {"time_to_solution_s": e0.elapsed_time(e1) * 1e-3, "iters": ig.iters,
                                     "inner_iters_total": ig.inner_iters_total, "relres_true": ig.relres_true}}

    # inhomogeneous Dirichlet data: u = plane wave on the boundary, volume data
    # b; A u = b + lift(u_Gamma) solved from zero and from the BEM solution
    # with the data (double layer included), and the double-layer apply alone
    dirich = None
    if args.dirichlet:
        ub = torch.from_numpy(inputs.plane_wave_boundary(n, w["k"])).to(dev)
        ikw = dict(inner_rtol=args.inner_rtol, inner_maxit=args.inner_maxit, inner_m=args.inner_maxit)
        bd = tree.dirichlet_rhs(b, ub)
        tree.gmres(bd, **gm)                                   # warm-up
        x0, _ = tree.bem_solve_dirichlet(b, ub, **ikw)
        flush.fill_(1.0)
        e0.record(stream)
        tree.dirichlet_rhs(b, ub, b=bd)
        _, iz = tree.gmres(bd, **gm)
        e1.record(stream)
        torch.cuda.synchronize()
        t_zero = e0.elapsed_time(e1) * 1e-3
        flush.fill_(1.0)
        e0.record(stream)
        tree.dirichlet_rhs(b, ub, b=bd)
        _, its_bem = tree.bem_solve_dirichlet(b, ub, u=x0, **ikw)
        _, ibm = tree.gmres(bd, x=x0, **gm)
        e1.record(stream)
        torch.cuda.synchronize()
        t_bem = e0.elapsed_time(e1) * 1e-3
        tgt_all = hfmm.SET_VOL | hfmm.SET_BND
        pv_d, pb_d = tree.apply(None, ub, src=hfmm.SET_BND, tgt=tgt_all, mode=hfmm.DLP)
        e0.record(stream)
        for _ in range(5):
            tree.apply(None, ub, src=hfmm.SET_BND, tgt=tgt_all, phi_vol=pv_d, phi_bnd=pb_d, mode=hfmm.DLP)
        e1.record(stream)
        torch.cuda.synchronize()
        dl_ms = e0.elapsed_time(e1) / 5
        dirich = {"boundary_data": "plane wave exp(i k d.x), d = (1, 2, 2)/3",
                  "from_zero": {"time_to_solution_s": t_zero, "gmres_iters": iz.iters,
                                "inner_iters_total": iz.inner_iters_total, "relres_true": iz.relres_true,
                                "converged": iz.status == 0},
                  "from_bem_solution": {"time_to_solution_s": t_bem, "gmres_iters": ibm.iters,
                                        "inner_iters_total": ibm.inner_iters_total + its_bem,
                                        "relres_true": ibm.relres_true, "converged": ibm.status == 0},
                  "double_layer_apply_ms": dl_ms,
                  "double_layer_apply_mpts_s": (n ** 3 + 6 * n * n) / (dl_ms * 1e-3) / 1e6}

    # batched form: 48 independent solves of uneven size and wavenumber
    batched = None
    if not args.no_batched:
        probs = inputs.batched_problems()
        orders = [hfmm.order_for_k(q["k"], q["p"]) for q in probs]
        tb0 = time.perf_counter()
        trees = [hfmm.Tree(q["n"], q["k"], p_, q["theta"], q["leaf"], "fp32") for q, p_ in zip(probs, orders)]
        for tr in trees:
            tr.autotune()
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - tb0
        bs = [torch.from_numpy(inputs.rhs(q["rhs"], q["n"], q["seed"])).to(dev) for q in probs]
        gmb = dict(gm, restart=50, maxit=args.batched_maxit)
        hfmm.gmres_solve_batched(trees, bs, **gmb)  # warm-up
        torch.cuda.synchronize()
        e0.record(stream)
        _, binfos = hfmm.gmres_solve_batched(trees, bs, **gmb)
        e1.record(stream)
        torch.cuda.synchronize()
        tbat = e0.elapsed_time(e1) * 1e-3
        e0.record(stream)
        for tr, b_ in zip(trees, bs):
            try:
                tr.gmres(b_, **gmb)
            except hfmm.HfmmError as err:  # a solve that stopped on a non-finite value
                if err.status != hfmm.HFMM_ERR_NONFINITE:
                    raise
        e1.record(stream)
        torch.cuda.synchronize()
        tseq = e0.elapsed_time(e1) * 1e-3
        conv = [i.status == 0 for i in binfos]
        batched = {"solves": len(probs), "converged": int(sum(conv)), "maxit": args.batched_maxit,
                   "batched_s": tbat, "sequential_s": tseq, "speedup": tseq / tbat,
                   "setup_s": setup_s, "gmres_iters": [i.iters for i in binfos],
                   "order_rule": "hfmm_order_for_k(k, p requested)",
                   "orders_raised": sum(1 for q, p_ in zip(probs, orders) if p_ != q["p"]),
                   "unconverged": [dict(n=q["n"], k=round(q["k"], 3), p=p_)
                                   for q, p_, c in zip(probs, orders, conv) if not c]}
        for tr in trees:
            tr.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        inner = info.inner_iters_total / max(1, info.iters)
        v, desc = oracle_sample(w, inner, info.iters)
        cpu = {"value": v, "unit": "s", "cores": torch_threads(), "kind": "oracle",
               "sample": desc + "; iteration counts of this run's solve"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": ms * 1e-3, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "k": w["k"], "p": w["p"], "leaf": w["leaf"],
                       "theta": w["theta"], "restart": w["restart"], "inner_rtol": args.inner_rtol,
                       "inner_maxit": args.inner_maxit, "inner_p": args.inner_p or w["p"],
                       "fmm_precision": args.precision,
                       "krylov_precision": ("outer fp64, inner fp32" if args.precision == "fp32" else "fp64"),
                       "l2": "flushed (512 MB write) before every timed step",
                       "autotuned": not args.no_autotune,
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "gmres_iters": info.iters, "inner_iters_total": info.inner_iters_total,
            "relres_true": relres, "build_s": build_s, "autotune_s": tune_s,
            "solves_per_s": world / (ms * 1e-3),
            "fmm_apply_ms": app_ms, "fmm_apply_mpts_s": mpts,
            "gpu_launches": int(launches),
            "roofline": roof, "roofline_p2p": roof_p2p if roof is not roof_p2p else None,
            "roofline_m2l": roof_m2l, "stages_per_solve": stage_summary,
            "e2e": {"value": e2e_ms * 1e-3, "unit": "s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes},
            "fp64": fp64, "n128": big, "bicgstab": bicg, "batched": batched, "cpu_baseline": cpu, "clocks": clk,
            "pipe_peaks": pk,
        }
        if dirich is not None:
            line["dirichlet"] = dirich
        print(json.dumps(line), flush=True)
    tree.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_apply_only(args):
    import torch
    from __graft_entry__ import build
    build()
    from paper_1608_02461_gb300 import hfmm, inputs
    w = inputs.WORKLOADS[args.workload]
    n = w["n"]
    dev = torch.device("cuda:0")
    tree = hfmm.Tree(n, w["k"], w["p"], w["theta"], w["leaf"], args.precision)
    qv = torch.from_numpy(inputs.complex_normal(n ** 3, 1)).to(dev)
    qb = torch.from_numpy(inputs.complex_normal(6 * n * n, 2)).to(dev)
    src, tgt = args.apply_only
    for _ in range(2):
        tree.apply(qv, qb, src=src, tgt=tgt)
    torch.cuda.synchronize()
    tree.close()


def run_sweep(args):
    """GMRES iterations and time of the preconditioned solve along one sweep;
    inner boundary solve to 1e-4 (at most 200 steps) so that the FMM
    accuracy, not the inner solve, sets the outer iteration count."""
    import torch
    from __graft_entry__ import build
    build()
    from paper_1608_02461_gb300 import hfmm, inputs
    dev = torch.device("cuda:0")
    if args.sweep == "kh":
        points = [dict(q, p=inputs.SWEEP_KH_P, prec="fp32") for q in inputs.SWEEP_KH]
    else:
        sp = inputs.SWEEP_P
        points = [dict(n=sp["n"], k=sp["k"], p=p, prec="fp64") for p in sp["ps"]]
    for q in points:
        n = q["n"]
        t = hfmm.Tree(n, q["k"], q["p"], 0.4, 32 if n < 32 else 64, q["prec"])
        b = torch.from_numpy(inputs.rhs("uniform_real", n, 6)).to(dev)
        kw = dict(restart=30, rtol=1e-6, inner_rtol=1e-4, inner_maxit=200, inner_m=200)
        t.gmres(b, **kw)  # warm-up (builds the preconditioner graph)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        _, info = t.gmres(b, **kw)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"sweep": args.sweep, "n": n, "k": q["k"], "kh": q["k"] / (n + 1), "p": q["p"],
                          "precision": q["prec"], "gmres_iters": info.iters,
                          "inner_iters_total": info.inner_iters_total, "relres_true": info.relres_true,
                          "time_s": e0.elapsed_time(e1) * 1e-3, "converged": info.status == 0}), flush=True)
        t.close()


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.apply_only:
        run_apply_only(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
