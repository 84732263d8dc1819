"""Benchmark: Torontonian subset-terms/s at N = 24 on one GB300 (FP64 per-term arithmetic).

Workload (one step): the click probability of one 24-click pattern of the
200-mode pure state with uniform squeezing r = 0.8 behind a Haar-random
interferometer (seed 1), i.e. 2^24 subset determinants of up to 48 x 48
matrices, their alternating sum and p = Tor / sqrt(det Sigma).  The state is
resident on the device when the timed region starts; the 24 click modes come
from the host each step.

Output: one JSON line (rank 0).  `value` is device time (CUDA events around
each step on the library's stream); `e2e` runs the same step through the public
API from pinned host buffers (state build from U, r included) with wall-clock
timing; `roofline` is the dominant kernel (the register depth-first leaf
kernel) against the FP64 rate measured in the same run; `cpu_baseline` is the
oracle timed on this host's cores on a bounded sample.

`--impl reference` times the oracle itself (the only reference there is: the
paper's code is not available and ran on Titan CPUs) on a bounded sample.
Multi-GPU (torchrun): independent replicas, no collective in the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Tor subset-terms/s (FP64, N=24)"
UNIT = "subset-terms/s"


def sym(d):
    return d * (d + 1) // 2


def leading_flops(q: int, complex_basis: bool = False) -> float:
    """Algorithmic flops of the subtree below a node with q undecided modes, the
    leading-order count of the method: the include child of a node with t + 1
    undecided modes does a rank-2 update of 2t rows, 4 t^2 real multiply-adds
    (8 t^2 flops) in the real basis (complex: 4 t^2 complex multiply-adds, 32 t^2
    flops), plus one inverse square root and one addition per subset term."""
    per = 32.0 if complex_basis else 8.0
    return per * sum(2.0 ** (q - k) * (k - 1) ** 2 for k in range(1, q + 1)) + 2.0 * 2.0 ** q


def executed_flops(q: int, Q: int, complex_basis: bool = False) -> float:
    """FP64 flops the kernels execute below a node with q undecided modes when the
    last Q levels run in registers (FMA = 2, any other FP64 operation = 1; the
    inverse square roots run on the integer pipes and count 0).  Levels above the
    register subtree (shared memory) factor the pivot by its adjugate: det (3),
    1/det (1), the scaled inverse (3), s g (1), L = u P^-1 (3 flops per entry of 2t
    rows) and the update (two FMAs per lower-triangle entry).  The real-basis
    register levels factor it by Cholesky (w, d1, g, the row coefficient, s g: 6;
    rows w = u R^-T at 4 flops per row); one-mode nodes form det (3) and add their
    two leaf terms (one FMA, one add: 3).  Complex entries count 4x the real flops."""
    def node(k, reg):
        t = k - 1
        if k == 1:
            return 6.0
        sym2t = t * (2 * t + 1)
        if reg and not complex_basis:
            return 6.0 + 8.0 * t + 4.0 * sym2t
        return 8.0 + 12.0 * t + 4.0 * sym2t
    total = 0.0
    for k in range(1, q + 1):
        total += 2.0 ** (q - k) * node(k, k <= Q)
    return total * (4.0 if complex_basis else 1.0)


def fx_products(n: int) -> float:
    """Fixed-point products of a whole tree of n modes, in units of one product of two
    FX entries (six 32-bit limbs: 26 partial products of 32 x 32 bits).  Every node
    with m >= 2 undecided modes forms its include child: pivot determinant (2),
    inverse square root (89 partial products of short operands: 3.42), 1/det (1),
    the scaled inverse (3), s g (a 7-limb scale: 39 partial products, 1.5),
    L = u P^-1 (4 per row of 2(m-1) rows) and the update (2 per lower-triangle entry);
    a one-mode node forms det, its inverse square root and s g for its leaf term."""
    R, SG = 89.0 / 26.0, 39.0 / 26.0
    total = 0.0
    for d in range(n - 1):
        t = n - d - 1
        total += 2.0 ** d * (2.0 + R + 1.0 + 3.0 + SG + 8.0 * t + 2.0 * t * (2 * t + 1))
    return total + 2.0 ** (n - 1) * (2.0 + R + SG)


class ClockSampler:
    """nvidia-smi samples (every 20 ms) around the timed region; the samples read between
    begin() and end() (plus one sampling period) are the ones reported."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.t_begin = self.t_end = None

    def start(self):
        """Start sampling and wait (up to 3 s) for the first sample, so that the timed
        region that follows is covered from its start."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", str(self.PERIOD_MS)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 3.0:
                time.sleep(0.005)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def begin(self):
        self.t_begin = time.perf_counter()

    def end(self):
        self.t_end = time.perf_counter()

    def stop(self):
        if not self.proc:
            return None
        if self.t_end is None:
            self.end()
        time.sleep(2 * self.PERIOD_MS / 1e3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        t_b = self.t_begin if self.t_begin is not None else -1e300
        inside = [ln for t, ln in self.lines if t_b <= t <= self.t_end + self.PERIOD_MS / 1e3]
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in inside:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = max(smax, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "period_ms": self.PERIOD_MS}


def dist_setup():
    """One process per GPU (torchrun environment).  The replicas share nothing on the
    data path; the process group only carries the barrier and the max-over-ranks time
    (NCCL on GPUs, gloo where there is none)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(ws, x: float, local: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda:%d" % local if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def other_accountings(n: int, step_s: float):
    """Flops per step under the per-subset Cholesky accountings, as context for the Schur tree's
    count: complex (2k)^3/3 multiply-adds per subset of k modes without prefix reuse, and with
    the shared prefix reused (only the trailing rows per subset, 4 (k-1)^2), 8 real flops each;
    'equivalent' = those flops over the measured step time."""
    from math import comb
    ek3 = sum(comb(n, k) * k ** 3 for k in range(n + 1))
    ekm12 = sum(comb(n, k) * max(k - 1, 0) ** 2 for k in range(n + 1))
    no_reuse = 8.0 * (8.0 / 3.0) * ek3
    prefix = 8.0 * 4.0 * ekm12
    return {"cholesky_no_reuse_flops": no_reuse, "cholesky_prefix_reuse_flops": prefix,
            "equivalent_tflops_no_reuse": no_reuse / step_s / 1e12,
            "equivalent_tflops_prefix_reuse": prefix / step_s / 1e12}


def captured_traffic(args, tuning):
    """DRAM bytes (read + write) per launch of the dominant kernel, from an ncu capture of the same
    kernel code and launch shape (FP64 real basis, N = 24, the shared-memory levels and register
    depth given here); None for any other shape, or once the kernel changed since the capture."""
    return CAPTURED_TRAFFIC.get((args.prec, args.basis, args.N, tuning["sub_e"], tuning["q_drop"],
                                 tuning["grid_per_sm"]))


# (prec, basis, N, sub_e, q_drop, grid_per_sm) -> bytes per launch of the subtree kernel,
# dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of the current kernel code
CAPTURED_TRAFFIC = {
    # 2^15 depth-15 roots of 171 entries (44.8 MB of input) into one-warp CTAs of two roots each;
    # one CTA per pair of roots (16,384 partials, which stay in L2) or 8 persistent CTAs per SM
    ("fp64", "real", 24, 4, 0, 0): 45235456 + 39424,
    ("fp64", "real", 24, 4, 0, 8): 45235456 + 4096000,
}


def whole_job_rate(ws: int, units_per_rank: float, seconds_max: float) -> float:
    """Units all replicas processed divided by the slowest replica's time (weak scaling)."""
    return ws * units_per_rank / seconds_max


def cpu_oracle_rate(n_sample: int, threads: int = 0):
    """Oracle subset-terms/s on this host: the decision-tree oracle (~212-bit) on
    the first n_sample modes of the N = 24 pattern (threads <= 0: every core)."""
    import gbs_inputs as gi
    import oracle
    st, modes = gi.single_large_torontonian_workload()
    Sig = oracle.sigma(oracle.covariance(st.U, st.r, st.eta))
    H = oracle.sigma_inv_block(Sig, modes[:n_sample])
    threads = threads if threads > 0 else (os.cpu_count() or 1)
    t0 = time.perf_counter()
    oracle.torontonian(H, "tree", nthreads=threads)
    dt = time.perf_counter() - t0
    return (2 ** n_sample) / dt, dt, threads


def cpu_fp64_block(ctx, gbs, st, modes, gpu_terms_per_s):
    """The same Torontonian in plain FP64 on the host cores: the decision tree in C++ with OpenMP
    over subtrees (cpu_baseline/), on the very click block the GPU tree starts from (read back
    from the library), single-core and on every core; median of three runs each."""
    import cpu_baseline
    cpu_baseline.build()
    G = gbs.sigma_inv_block(ctx, st, modes, "real")
    n = len(modes)
    cores = cpu_baseline.max_threads()
    out = {}
    for name, th in (("single_core", 1), ("all_cores", cores)):
        runs = [cpu_baseline.torontonian_fp64(G, th, 10) for _ in range(3)]
        sec = float(np.median([r[2] for r in runs]))
        out[name] = {"value": 2.0 ** n / sec, "seconds": sec, "threads": th, "tor": runs[-1][0]}
    return {"metric": "Tor subset-terms/s (FP64, N=%d), host cores" % n, "unit": UNIT, "cores": cores,
            "kind": "plain FP64 decision tree (same algorithm and precision), OpenMP over 2^10 subtrees",
            "single_core": out["single_core"], "all_cores": out["all_cores"],
            "gpu_over_all_cores": gpu_terms_per_s / out["all_cores"]["value"],
            "gpu_over_single_core": gpu_terms_per_s / out["single_core"]["value"]}


def _haar_job(job):
    import gbs_inputs as gi
    return gi.haar_unitary(*job)


def haar_unitaries(jobs):
    """Haar unitaries for (M, seed) jobs, built by a pool of fresh (spawned) host processes."""
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")
    workers = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_haar_job, jobs, chunksize=8)


def sampler_block(ctx, gbs, gi, n_traj, ws, local, autotune=True):
    """M = 800, r ~ U[0.3, 0.9], Haar seed 2, n_traj forced trajectories of 20 uniformly placed clicks
    (the paper's forced-outcome benchmark); p0 is evaluated at all 800 steps of every trajectory.
    Without autotuning the fixed-point shapes are the ones the autotuner usually picks here."""
    stp, clicks = gi.chain_sampling_workload(800, 20, n_traj, seed=2)
    st = gbs.build_state(ctx, stp.U, stp.r, stp.eta)
    for prec in ("fxn", "fx", "fxw"):
        if autotune:
            # the late steps batch 64 trees of ~13..21 modes: tune on such a batch
            ctx.autotune(prec, "real", 21, n_trees=9)
        else:
            ctx.set_tuning(prec, "real", sub_e=0, d_top=6, grid_per_sm=0, level_threads=1 << 17, q_drop=1, mid_e=0)
    # the library draws the forced positions from the seed (the same as the workload's `clicks`)
    gbs.sample_forced_random(ctx, st, 2, seed=2, n_clicks=20)  # warm-up
    l0 = ctx.launch_count  # also locates the timed run in a launch list of the whole process
    barrier(ws)
    t0 = time.perf_counter()
    pats, p0, stats = gbs.sample_forced_random(ctx, st, n_traj, seed=2, n_clicks=20, want_p0=True)
    dt = allreduce_max(ws, time.perf_counter() - t0, local)
    status = 0 if all(np.nonzero(p)[0].tolist() == list(c) for p, c in zip(pats, clicks)) else -1
    st.free()
    return {"metric": "M=800,N=20 samples/s", "value": whole_job_rate(ws, n_traj, dt), "unit": "samples/s",
            "seconds": dt, "trajectories": n_traj, "steps_evaluated": stats["steps"],
            "escalations": stats["escalations"], "uncertified_steps": stats["uncertified"],
            "gpu_launches": ctx.launch_count - l0, "library_launches_before": l0,
            "trees_fp64_dd_td_fx_fxw_fxn": stats["trees"], "tree_seconds_fp64_dd_td_fx_fxw_fxn": stats["tree_seconds"],
            "other_seconds": stats["cond_seconds"], "fx_tuning": ctx.tuning("fx", "real"),
            "fxw_tuning": ctx.tuning("fxw", "real"), "fxn_tuning": ctx.tuning("fxn", "real"),
            "p0_range": [float(p0.min()), float(p0.max())], "status": status,
            "workload": "M=800 modes, r~U[0.3,0.9], Haar seed 2, eta=1; %d forced trajectories with 20 uniform "
                        "click positions; no-click probability at every one of the 800 steps" % n_traj}


def certified_block(ctx, gbs, st, modes, steps, stream):
    """The same N = 24 Torontonian evaluated to the 1e-10 relative tolerance (AUTO precision),
    device time per evaluation, next to the FP64 throughput figure of the headline."""
    ctx.autotune("fx", "real", 24)
    gbs.torontonian(ctx, st, modes, "auto", "real")
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    res = []
    for i in range(steps):
        ev[i][0].record(stream)
        res.append(gbs.torontonian(ctx, st, modes, "auto", "real"))
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    out = {"metric": "certified Tor subset-terms/s (N=24, rel. error bound <= 1e-10)",
           "value": 2.0 ** 24 / (ms * 1e-3), "ms_per_evaluation": ms, "prec": res[-1].prec,
           "rel_err_bound": res[-1].err_bound / abs(res[-1].p), "kappa": res[-1].kappa, "p": res[-1].p,
           "fx_tuning": ctx.tuning("fx", "real")}
    if res[-1].prec == "fx":
        peak = ctx.measure_fx_peak()
        products = fx_products(24)
        out["roofline"] = {
            "bound": "alu", "unit": "G products/s", "achieved": products / (ms * 1e-3) / 1e9,
            "peak": peak / 1e9, "frac": products / (ms * 1e-3) / peak,
            "scope": "the whole certified evaluation (click block, tree, reduction, readback)",
            "products_per_term": products / 2.0 ** 24,
            "model": "fx_products: 192-bit fixed-point products of the tree's Schur steps, "
                     "inverse square roots and scale updates",
            "peak_source": "independent chains of FX products, 16 warps per SM, measured in this run "
                           "(gbs_measure_fx_peak)"}
    return out


def paired_block(ctx, gbs, st, modes, steps, stream, cert, fp64_result):
    """The same N = 24 Torontonian in FP64 with the last two tree levels summed cancellation-free:
    device time per evaluation, its error bound, how much smaller its sum of group magnitudes is
    than the plain sum of |terms| (and the effective cancellation ratio that leaves, against the
    certified Torontonian), and the observed relative error against the certified (fixed-point)
    value next to the plain FP64 one."""
    import torch
    ctx.autotune("fp64p", "real", 22)
    for _ in range(2):
        gbs.torontonian(ctx, st, modes, "fp64p", "real")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    res = []
    for i in range(steps):
        ev[i][0].record(stream)
        res.append(gbs.torontonian(ctx, st, modes, "fp64p", "real"))
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    pr = res[-1]
    ref = cert["p"]
    return {"metric": "Tor subset-terms/s (FP64, last two levels cancellation-free, N=24)",
            "value": 2.0 ** 24 / (ms * 1e-3), "ms_per_evaluation": ms, "tuning": ctx.tuning("fp64p", "real"),
            "rel_err_bound": pr.err_bound / abs(pr.p),
            "magnitude_sum_reduction": fp64_result.abs_sum / pr.abs_sum,
            "kappa_groups": cert["kappa"] * pr.abs_sum / fp64_result.abs_sum,
            "observed_rel_err_vs_certified": abs(pr.p - ref) / abs(ref),
            "plain_fp64": {"rel_err_bound": fp64_result.err_bound / abs(fp64_result.p), "kappa": fp64_result.kappa,
                           "observed_rel_err_vs_certified": abs(fp64_result.p - ref) / abs(ref)}}


def complex_basis_block(ctx, gbs, st, modes, steps, stream, peak):
    """The same N = 24 FP64 Torontonian with the click block in the complex (a, a^+) basis, the form
    the determinants are usually written in (Hermitian 48 x 48); equal determinants, 4x the flops."""
    import torch
    ctx.autotune("fp64", "complex", 22)
    for _ in range(2):
        gbs.torontonian(ctx, st, modes, "fp64", "complex")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    ctx.kernel_time()
    ctx.enable_timing(True)
    for i in range(steps):
        ev[i][0].record(stream)
        gbs.torontonian(ctx, st, modes, "fp64", "complex")
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ctx.enable_timing(False)
    leaf_ms, leaf_n = ctx.kernel_time()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    t = ctx.tuning("fp64", "complex")
    Q = max(1, min(4 - t["q_drop"], 24))
    q_root = min(24, Q + t["sub_e"])
    leaf_flops = (2 ** (24 - q_root)) * leading_flops(q_root, True)
    achieved = leaf_flops / (leaf_ms / max(leaf_n, 1) * 1e-3) / 1e12
    return {"metric": "Tor subset-terms/s (FP64, N=24, complex basis)", "value": 2.0 ** 24 / (ms * 1e-3),
            "ms_per_evaluation": ms, "tuning": t, "leading_flops_per_term": leading_flops(24, True) / 2.0 ** 24,
            "dominant_kernel_tflops": achieved, "frac_of_fp64_peak": achieved / peak}


def walltime_block(ctx, gbs, gi, ms):
    """One worst-case sample per click count m at the paper's Table II sizes (l modes,
    8 dB, all m clicks first), AUTO precision; the paper's Titan walltimes beside it as
    context (hours on the quoted node counts, quad precision; none past its m = 20); and eight
    samples with the m clicks at uniformly random positions, run together (the paper's typical
    case)."""
    paper = {10: (0.11, 1), 12: (0.68, 4), 14: (0.97, 32), 16: (1.98, 128), 18: (1.90, 1024), 20: (1.83, 8192)}
    # one trajectory: each step is a single tree of up to m + 1 modes
    tune_n = min(max(ms) + 1, 21)
    ctx.autotune("fxn", "real", tune_n)
    ctx.autotune("fx", "real", tune_n)
    ctx.autotune("fxw", "real", tune_n)
    rows = []
    for m in ms:
        stp, clicks = gi.walltime_workload(m)
        st = gbs.build_state(ctx, stp.U, stp.r, stp.eta)
        forced = np.asarray(clicks, dtype=np.int32)[None, :]
        t0 = time.perf_counter()
        pats, p0, stats, status = gbs.sample(ctx, st, 1, seed=m, N_post=m, forced_clicks=forced, want_p0=True)
        dt = time.perf_counter() - t0
        st.free()
        st = gbs.build_state(ctx, stp.U, stp.r, stp.eta)
        rnd = gi.walltime_random_positions(m, 8).astype(np.int32)
        t0 = time.perf_counter()
        _, _, _, status_r = gbs.sample(ctx, st, len(rnd), seed=m, N_post=m, forced_clicks=rnd)
        dt_r = (time.perf_counter() - t0) / len(rnd)
        st.free()
        rows.append({"m": m, "modes": int(stp.U.shape[0]), "seconds_per_sample": dt, "status": status,
                     "random_positions_seconds_per_sample": dt_r, "random_positions_status": status_r,
                     "trees_fp64_dd_td_fx_fxw_fxn": stats["trees"], "tree_seconds_fp64_dd_td_fx_fxw_fxn": stats["tree_seconds"],
                     "escalations": stats["escalations"], "uncertified_steps": stats["uncertified"],
                     "p0_min": float(p0.min()),
                     "paper_titan_hours": paper.get(m, (None, None))[0],
                     "paper_titan_nodes": paper.get(m, (None, None))[1]})
    return {"metric": "seconds per worst-case sample (paper Table II sizes)", "rows": rows,
            "workload": "l in {200,288,392,512,624,800} modes for m in {10..20} clicks (the paper's Table II), "
                        "then l = 2 m^2 beyond; 8 dB squeezing, Haar, no loss; the m clicks forced on the "
                        "first m measured modes (one sample), or at uniformly random positions (8 samples "
                        "run together, time per sample)"}


def batched_block(ctx, gbs, gi, n_req, n_err, autotune=True):
    """Uneven probability requests (N ~ U{8..22}, M ~ U{100, 200, 400}, r ~ U[0.4, 1.0],
    eta ~ U[0.25, 1.0], Haar unitary seeded per request) evaluated as one batch in FP64 and
    one at a time; plus the FP32 / FP64 / paired-FP64 error study on a subsample against certified
    values."""
    reqs = gi.batched_requests(4096)[:n_req]
    if autotune:
        # launch shapes for a batch of uneven trees like this one (22 .. 8 modes), not the single
        # 24-mode tree of the headline
        ctx.autotune("fp64", "real", 22, n_trees=15)
    t0 = time.perf_counter()
    Us = haar_unitaries([(q.M, q.seed) for q in reqs])
    states = [gbs.build_state(ctx, U, np.full(q.M, q.r), q.eta) for U, q in zip(Us, reqs)]
    del Us
    t_inputs = time.perf_counter() - t0
    pats = [q.modes for q in reqs]
    terms = float(sum(2 ** q.N for q in reqs))
    gbs.torontonian_batch(ctx, states[:64], pats[:64], "fp64", "real", check=False)
    l0 = ctx.launch_count
    t0 = time.perf_counter()
    batch = gbs.torontonian_batch(ctx, states, pats, "fp64", "real", check=False)
    t_batch = time.perf_counter() - t0
    launches = ctx.launch_count - l0
    t0 = time.perf_counter()
    for st, pat in zip(states, pats):
        gbs.torontonian(ctx, st, pat, "fp64", "real")
    t_single = time.perf_counter() - t0
    # the same batch certified to 1e-10 relative (AUTO: FP64, then fixed point, then triple-double)
    t0 = time.perf_counter()
    cert, cert_status = gbs.torontonian_batch(ctx, states, pats, "auto", "real", check=False, return_status=True)
    t_cert = time.perf_counter() - t0
    if cert_status not in (0, 4):  # GBS_OK, or GBS_EPRECISION with every value filled in
        raise RuntimeError("certified batch failed with status %d: %s"
                           % (cert_status, ctx.L.gbs_ctx_last_error(ctx.h).decode()))
    prec_counts = {}
    for c in cert:
        prec_counts[c.prec] = prec_counts.get(c.prec, 0) + 1
    worst_bound = max(c.err_bound / abs(c.p) for c in cert if c.p)
    # FP32 error study: relative error of FP32 and FP64 terms against the certified (AUTO) value
    idx = list(range(0, n_req, max(1, n_req // n_err)))[:n_err]
    sub_s, sub_p = [states[i] for i in idx], [pats[i] for i in idx]
    ref = gbs.torontonian_batch(ctx, sub_s, sub_p, "auto", "real", check=False)
    f32 = gbs.torontonian_batch(ctx, sub_s, sub_p, "fp32", "real", check=False)
    f64p = gbs.torontonian_batch(ctx, sub_s, sub_p, "fp64p", "real", check=False)
    by_n = {}
    for i, r_, a, b, c in zip(idx, ref, f32, [batch[i] for i in idx], f64p):
        rel = (lambda x: abs(x.p - r_.p) / abs(r_.p) if r_.p else float("inf"))
        by_n.setdefault(reqs[i].N, []).append((rel(a), rel(b), r_.kappa, rel(c), r_.kappa * c.abs_sum / r_.abs_sum))
    err = {int(n): {"fp32_median_rel_err": float(np.median([x[0] for x in v])),
                    "fp64_median_rel_err": float(np.median([x[1] for x in v])),
                    "fp64p_median_rel_err": float(np.median([x[3] for x in v])),
                    "kappa_median": float(np.median([x[2] for x in v])),
                    "kappa_groups_median": float(np.median([x[4] for x in v])), "count": len(v)}
           for n, v in sorted(by_n.items())}
    for st in states:
        st.free()
    return {"metric": "batched Torontonians (FP64, uneven N)", "requests": n_req, "subset_terms": terms,
            "batch_seconds": t_batch, "batch_requests_per_s": n_req / t_batch, "batch_terms_per_s": terms / t_batch,
            "one_at_a_time_seconds": t_single, "one_at_a_time_requests_per_s": n_req / t_single,
            "speedup_vs_one_at_a_time": t_single / t_batch, "batch_gpu_launches": launches,
            "fp64_tuning": ctx.tuning("fp64", "real"),
            "certified": {"seconds": t_cert, "requests_per_s": n_req / t_cert, "precisions": prec_counts,
                          "max_rel_err_bound": worst_bound, "status": cert_status,
                          "above_1e-10": sum(1 for c in cert if c.p and c.err_bound > 1e-10 * abs(c.p))},
            "input_seconds": t_inputs, "fp32_error_study": err,
            "workload": "%d of the 4096 requests: N~U{8..22}, M~U{100,200,400}, r~U[0.4,1.0], "
                        "eta~U[0.25,1.0], Haar seeded per request; inputs built outside the timed "
                        "region" % n_req}


def _pct(x, q):
    return float(np.percentile(x, q)) if len(x) else None


def served_block(ctx, gbs, gi, plan, max_attempts, width, n_one):
    """The served dense-subgraph stream: Poisson arrivals of postselected sampling jobs on
    graph-encoded states (graph, loss, N per request), at several arrival rates -- below the loop's
    capacity (steady-state latency) and at the stated 200 per second (a burst the loop drains at its
    capacity).  Latency percentiles are over accepted samples; requests that exhaust their
    postselection attempts (GBS_EREJECT) are counted and timed apart.  Beside it, the first n_one
    requests served one at a time through the same loop (one active request, the same attempt
    width): their measured service times replayed as a single FIFO queue at each rate give the
    latency without batching across requests; their results must equal the loop's."""
    n_max = max(n for _, n in plan)
    _, reqs, graphs = gi.served_stream_workload(n_max)
    cache, sts = {}, []
    for g, eta, N in reqs:
        if (g, eta, N) not in cache:
            sp = gi.graph_state(graphs[g], 2.0 * N, eta)
            cache[(g, eta, N)] = gbs.build_state(ctx, sp.U, sp.r, sp.eta)
        sts.append(cache[(g, eta, N)])
    rows, first_results = [], None
    for rate, n_req in plan:
        arrivals, _, _ = gi.served_stream_workload(n_req, rate_hz=rate)
        srv = gbs.Server(ctx, arena_bytes=8 << 30, max_active=64, attempt_width=width)
        ctx.host_gaps()
        t0 = time.perf_counter()
        tickets = []
        for i, a in enumerate(arrivals):
            dt = t0 + a - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit_sample(sts[i], seed=1000 + i, sample_index=0, N_post=reqs[i][2],
                                             max_attempts=max_attempts))
        res = [srv.poll(t, timeout_s=1800) for t in tickets]
        wall = time.perf_counter() - t0
        stats = srv.stats()
        gap_s, waits = ctx.host_gaps()
        srv.stop()
        acc = np.array([r["latency_s"] for r in res if r["status"] == 0])
        rej = np.array([r["latency_s"] for r in res if r["status"] != 0])
        rows.append({"rate_hz": rate, "requests": n_req, "accepted": int(acc.size), "rejected": int(rej.size),
                     "samples_per_s": acc.size / wall, "wall_seconds": wall,
                     "p50_s": _pct(acc, 50), "p99_s": _pct(acc, 99), "mean_s": float(acc.mean()) if acc.size else None,
                     "rejected_p50_s": _pct(rej, 50), "rejected_p99_s": _pct(rej, 99),
                     "loop_busy_fraction": stats["busy_s"] / max(stats["wall_s"], 1e-9),
                     "host_gap_seconds": gap_s, "host_waits": waits,
                     "host_gap_fraction_of_busy": gap_s / max(stats["busy_s"], 1e-9)})
        if first_results is None or len(res) > len(first_results):
            first_results = res
    # one at a time: the first n_one requests, each alone in the loop (same attempt width)
    n_one = min(n_one, len(first_results))
    srv = gbs.Server(ctx, arena_bytes=8 << 30, max_active=1, attempt_width=width)
    svc, same = [], True
    for i in range(n_one):
        t1 = time.perf_counter()
        r = srv.poll(srv.submit_sample(sts[i], seed=1000 + i, sample_index=0, N_post=reqs[i][2],
                                       max_attempts=max_attempts), timeout_s=1800)
        svc.append(time.perf_counter() - t1)
        same &= r["status"] == first_results[i]["status"] and r.get("clicks") == first_results[i].get("clicks")
    srv.stop()
    one = []
    for rate, _ in plan:
        arrivals, _, _ = gi.served_stream_workload(n_one, rate_hz=rate)
        free_at, lat_acc = 0.0, []
        for i, (a, sv) in enumerate(zip(arrivals, svc)):
            free_at = max(a, free_at) + sv
            if first_results[i]["status"] == 0:
                lat_acc.append(free_at - a)
        one.append({"rate_hz": rate, "requests": n_one, "accepted": len(lat_acc), "p50_s": _pct(lat_acc, 50),
                    "p99_s": _pct(lat_acc, 99), "samples_per_s": len(lat_acc) / max(free_at, 1e-9)})
    for st in cache.values():
        st.free()
    return {"metric": "served p50/p99", "rates": rows, "attempt_width": width, "max_attempts": max_attempts,
            "one_at_a_time": one, "one_at_a_time_service_seconds": float(sum(svc)),
            "one_at_a_time_summary": {"requests": n_one, "samples_per_s": one[-1]["samples_per_s"] if one else None,
                                      "service_p50_s": _pct(svc, 50), "service_p99_s": _pct(svc, 99)},
            "results_identical_to_one_at_a_time": bool(same),
            "workload": "Poisson arrivals; ER graphs n in [100,200] p=0.1 with a planted 20-vertex p=0.9 part; "
                        "c for mean photon number 2N; eta in {1,0.5,0.25}; one sample postselected on N in "
                        "[8,20] per request, up to %d attempts, %d at once" % (max_attempts, width)}


def subgraph_density(A, nodes):
    """Edges inside the vertex set over the number of vertex pairs."""
    nodes = np.asarray(nodes)
    k = len(nodes)
    return float(A[np.ix_(nodes, nodes)].sum() / 2.0) / (k * (k - 1) / 2.0) if k > 1 else 0.0


def dense_subgraph_block(ctx, gbs, gi, n_samples):
    """The paper's application (Sec. IV): random search for a dense subgraph with GBS samples of the
    graph-encoded state against uniformly random vertex sets of the same size, on a 100-vertex
    Erdos-Renyi graph (p = 0.1) with a planted 20-vertex part (p = 0.9)."""
    A = gi.planted_graph(100, 11)
    planted = set(gi.planted_vertices(100, 11).tolist())
    rows = []
    for N in (8, 12, 16):
        sp = gi.graph_state(A, 2.0 * N, 1.0)
        st = gbs.build_state(ctx, sp.U, sp.r, sp.eta)
        t0 = time.perf_counter()
        pats, _, stats, status = gbs.sample(ctx, st, n_samples, seed=N, N_post=N, max_attempts=256, check=False)
        dt = time.perf_counter() - t0
        st.free()
        ok = [np.nonzero(p)[0] for p in pats if p[0] != 0xFF]
        uni = gi.uniform_subsets(100, N, n_samples, seed=N)
        d_gbs = [subgraph_density(A, s) for s in ok]
        d_uni = [subgraph_density(A, s) for s in uni]
        rows.append({"N": N, "samples": len(ok), "seconds": dt, "samples_per_s": len(ok) / dt,
                     "attempts_rejected": stats["rejections"],
                     "mean_density_gbs": float(np.mean(d_gbs)) if d_gbs else None,
                     "mean_density_uniform": float(np.mean(d_uni)),
                     "max_density_gbs": float(np.max(d_gbs)) if d_gbs else None,
                     "max_density_uniform": float(np.max(d_uni)),
                     "mean_planted_fraction_gbs": float(np.mean([len(planted & set(s.tolist())) / N for s in ok]))
                     if ok else None,
                     "mean_planted_fraction_uniform": float(np.mean([len(planted & set(s.tolist())) / N
                                                                     for s in uni]))})
    return {"metric": "dense-subgraph random search: GBS samples vs uniform subsets", "rows": rows,
            "workload": "ER(100, 0.1) with a planted 20-vertex part at 0.9 (seed 11); state with mean photon "
                        "number 2N, no loss; %d samples postselected on N clicks per row, the same number of "
                        "uniform N-subsets" % n_samples}


def summary_of(line):
    """The headline figures of every block in one short object, printed last on the line."""
    def get(*path):
        x = line
        for k in path:
            if not isinstance(x, dict) or k not in x:
                return None
            x = x[k]
        return x
    sm = {"fp64_terms_per_s": line.get("value"), "roofline_frac": get("roofline", "frac"),
          "roofline_frac_executed": get("roofline", "executed", "frac"),
          "certified_ms": get("certified", "ms_per_evaluation"),
          "certified_rel_err_bound": get("certified", "rel_err_bound"),
          "certified_fx_roofline_frac": get("certified", "roofline", "frac"),
          "sampler_samples_per_s": get("sampler", "value"),
          "batched_fp64_requests_per_s": get("batched", "batch_requests_per_s"),
          "batched_certified_requests_per_s": get("batched", "certified", "requests_per_s"),
          "batched_requests": get("batched", "requests"),
          "cpu_fp64_all_cores_terms_per_s": get("cpu_fp64", "all_cores", "value"),
          "cpu_fp64_single_core_terms_per_s": get("cpu_fp64", "single_core", "value")}
    served = line.get("served")
    if isinstance(served, dict):
        for row in served.get("rates", []):
            key = "served_%g_per_s" % row["rate_hz"]
            sm[key] = {k: row.get(k) for k in ("requests", "accepted", "rejected", "p50_s", "p99_s",
                                               "samples_per_s")}
        sm["served_one_at_a_time"] = served.get("one_at_a_time_summary")
    return sm


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    n_sample = args.ref_sample
    for _ in range(args.warmup):
        cpu_oracle_rate(min(n_sample, 12))
    rates, total = [], 0.0
    for _ in range(args.steps):
        r, dt, threads = cpu_oracle_rate(n_sample)
        rates.append(r)
        total += dt
    value = (2 ** n_sample) * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "qd (~212-bit)",
        "data": "synthetic",
        "config": {"workload": "Torontonian of the 200-mode r=0.8 Haar state (seed 1), first %d of its 24 click "
                               "modes (bounded sample of the N=24 workload)" % n_sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "N=%d sub-pattern, 2^%d terms per step" % (n_sample, n_sample)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbs", choices=["gbs", "reference"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp64p", "dd", "td", "fp32", "fxn", "fx", "fxw"])
    ap.add_argument("--basis", default="real", choices=["real", "complex"])
    ap.add_argument("--N", type=int, default=24)
    ap.add_argument("--cpu-sample", type=int, default=19, help="click count of the oracle's CPU sample")
    ap.add_argument("--ref-sample", type=int, default=16, help="click count per step of --impl reference")
    ap.add_argument("--cpu-sample-single", type=int, default=14, help="click count of the oracle's one-core sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the certified, paired-FP64 and complex-basis evaluations of the headline tree")
    ap.add_argument("--tuning", default="",
                    help="sub_e,d_top,grid_per_sm,level_threads[,q_drop[,mid_e]] (skips the autotuner)")
    ap.add_argument("--sampler-traj", type=int, default=64, help="forced trajectories of the M=800 sampler run (0: skip)")
    ap.add_argument("--batched-req", type=int, default=4096, help="requests of the uneven batch (of 4096; 0: skip)")
    ap.add_argument("--served", default="4:150,8:250,200:500",
                    help="rate_hz:requests pairs of the served stream runs (empty: skip)")
    ap.add_argument("--served-one", type=int, default=100,
                    help="requests served one at a time for the comparison")
    ap.add_argument("--served-attempts", type=int, default=24, help="postselection attempts per served request")
    ap.add_argument("--served-width", type=int, default=8,
                    help="postselection attempts a served request runs at once (1: one after another)")
    ap.add_argument("--dense-samples", type=int, default=128,
                    help="GBS samples per row of the dense-subgraph search (0: skip)")
    ap.add_argument("--walltime-m", default="10,12,14,16,18,20,22",
                    help="click counts of the worst-case walltime rows (paper Table II sizes; empty: skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import torch

    import gbs_inputs as gi
    from paper_1810_00900_gb300 import build as gbs_build

    if local == 0:
        gbs_build.build()
    barrier(ws)
    import paper_1810_00900_gb300 as gbs

    dev = local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    ctx = gbs.Context(dev)
    ctx.set_stream(stream.cuda_stream)
    peak_gflops = ctx.measure_fp64_peak()

    st_p, modes24 = gi.single_large_torontonian_workload(args.N)
    modes = np.ascontiguousarray(modes24, dtype=np.int32)
    st = gbs.build_state(ctx, st_p.U, st_p.r, st_p.eta)
    complex_basis = args.basis == "complex"
    if args.tuning:
        ctx.set_tuning(args.prec, args.basis, *(int(x) for x in args.tuning.split(",")))
        tune_report = []
    else:
        tune_report = ctx.autotune(args.prec, args.basis, min(args.N, 22)) if not args.no_autotune else []
    tuning = ctx.tuning(args.prec, args.basis)
    Q = {("fp64", False): 5, ("fp64", True): 4, ("dd", False): 4, ("dd", True): 3, ("td", False): 3,
         ("td", True): 2, ("fp32", False): 5, ("fp32", True): 4, ("fx", False): 3,
         ("fxw", False): 3, ("fp64p", False): 5, ("fxn", False): 3}[(args.prec, complex_basis)]
    Q = max(1, min(Q - tuning["q_drop"], args.N))
    q_root = min(args.N, Q + tuning["sub_e"])
    depth = args.N - q_root
    leaf_flops = (2 ** depth) * leading_flops(q_root, complex_basis)
    leaf_exec = (2 ** depth) * executed_flops(q_root, Q, complex_basis)
    total_flops = leading_flops(args.N, complex_basis)
    kernel_name = ("batch_subtree_kernel (%d levels expanded in shared memory, then register depth-first %d levels)"
                   % (q_root - Q, Q)) if tuning["sub_e"] else "batch_leaf_kernel (register depth-first, %d levels)" % Q

    # L2 flush buffer (larger than the 129 MB L2), written between timed steps.
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device="cuda:%d" % dev)

    def step():
        return gbs.torontonian(ctx, st, modes, args.prec, args.basis)

    clocks = ClockSampler(dev)
    clocks.start()  # running before the warm-up, so it samples the whole timed region
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.kernel_time()  # reset
    ctx.enable_timing(True)
    launches0 = ctx.launch_count
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    clocks.begin()
    results = []
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
            ev[i][0].record(stream)
        results.append(step())
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks.end()
    barrier(ws)
    clk = clocks.stop()
    launches = ctx.launch_count - launches0
    ctx.enable_timing(False)
    leaf_ms, leaf_n = ctx.kernel_time()
    dev_ms = sum(a.elapsed_time(b) for a, b in ev)
    dev_ms = allreduce_max(ws, dev_ms, local)
    terms = float(2 ** args.N)
    value = whole_job_rate(ws, args.steps * terms, dev_ms * 1e-3)
    leaf_avg_s = leaf_ms / max(leaf_n, 1) * 1e-3
    achieved = leaf_flops / leaf_avg_s / 1e12
    achieved_exec = leaf_exec / leaf_avg_s / 1e12
    peak = peak_gflops / 1e3

    # e2e: the same step through the public API from pinned host buffers, state build included.
    U_pin = torch.empty((st_p.M, st_p.M), dtype=torch.complex128, pin_memory=True)
    U_pin.numpy()[:] = st_p.U
    r_pin = torch.empty(st_p.M, dtype=torch.float64, pin_memory=True)
    r_pin.numpy()[:] = st_p.r
    for _ in range(2):
        s2 = gbs.build_state(ctx, U_pin.numpy(), r_pin.numpy(), st_p.eta)
        gbs.torontonian(ctx, s2, modes, args.prec, args.basis)
        s2.free()
    barrier(ws)
    t0 = time.perf_counter()
    for i in range(args.steps):
        s2 = gbs.build_state(ctx, U_pin.numpy(), r_pin.numpy(), st_p.eta)
        pr = gbs.torontonian(ctx, s2, modes, args.prec, args.basis)
        s2.free()
    e2e_s = allreduce_max(ws, time.perf_counter() - t0, local)
    e2e_value = whole_job_rate(ws, args.steps * terms, e2e_s)
    h2d = st_p.M * st_p.M * 16 + st_p.M * 8 + modes.nbytes
    d2h = 8 * 16  # the probability record

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dev_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.prec == "fp64" else args.prec, "data": "synthetic",
        "config": {
            "workload": "single Torontonian, N=%d clicks of the M=200 pure state (r=0.8, Haar seed 1): "
                        "2^%d subset determinants per step" % (args.N, args.N),
            "M": 200, "N": args.N, "basis": args.basis, "per_term_arithmetic": args.prec,
            "sum": {"fp64": "double-double", "fp64p": "double-double", "dd": "double-double",
                    "fp32": "double-double", "td": "triple-double", "fxn": "exact fixed point",
                    "fx": "exact fixed point", "fxw": "exact fixed point"}[args.prec],
            "l2": "flushed between steps (256 MB write); tree level buffers also exceed L2",
            "parallelism": "replicas" if ws > 1 else "single GPU",
            "tuning": tuning, "autotune_candidates": len(tune_report),
            "autotune_fastest": sorted(tune_report, key=lambda c: c["ms"])[:5] if tune_report else [],
        },
        "roofline": {
            "bound": "alu", "kernel": kernel_name,
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": "FP64 DFMA-chain kernel measured in this run (gbs_measure_fp64_peak)",
            "traffic": captured_traffic(args, tuning), "traffic_unit": "bytes per launch",
            "traffic_source": "stored ncu capture of this kernel code and launch shape (not measured in this run)",
            "flop_model": "8 t^2 flops per rank-2 update of 2t rows (real basis) + rsqrt and add per subset term",
            "flops_per_launch": leaf_flops, "leaf_ms_avg": leaf_avg_s * 1e3,
            "executed": {"flops_per_launch": leaf_exec, "achieved": achieved_exec, "frac": achieved_exec / peak,
                         "model": "every FP64 operation the kernel executes (FMA = 2, other = 1; the inverse "
                                  "square roots run on the integer pipes)"},
            "step_flops": total_flops,
            "step_tflops": total_flops * args.steps / (dev_ms * 1e-3) / 1e12,
            "other_accountings": other_accountings(args.N, dev_ms * 1e-3 / args.steps),
        },
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "result": {"p": results[-1].p, "kappa": results[-1].kappa, "prec": results[-1].prec},
    }
    if args.prec == "fp64" and args.N == 24 and not args.no_extras:
        line["certified"] = certified_block(ctx, gbs, st, modes, max(3, args.steps // 2), stream)
        line["paired_fp64"] = paired_block(ctx, gbs, st, modes, max(3, args.steps // 2), stream, line["certified"],
                                           results[-1])
        line["complex_basis"] = complex_basis_block(ctx, gbs, st, modes, max(3, args.steps // 2), stream, peak)
    if args.sampler_traj > 0:
        line["sampler"] = sampler_block(ctx, gbs, gi, args.sampler_traj, ws, local, autotune=not args.no_autotune)
    if args.batched_req > 0:
        line["batched"] = batched_block(ctx, gbs, gi, args.batched_req, 48, autotune=not args.no_autotune)
    if args.served:
        plan = [(float(x.split(":")[0]), int(x.split(":")[1])) for x in args.served.split(",")]
        line["served"] = served_block(ctx, gbs, gi, plan, args.served_attempts, args.served_width, args.served_one)
    if args.walltime_m:
        line["walltime"] = walltime_block(ctx, gbs, gi, [int(x) for x in args.walltime_m.split(",")])
    if args.dense_samples > 0:
        line["dense_subgraph"] = dense_subgraph_block(ctx, gbs, gi, args.dense_samples)
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        rate, dt, threads = cpu_oracle_rate(args.cpu_sample)
        rate1, dt1, _ = cpu_oracle_rate(args.cpu_sample_single, threads=1)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": "N=%d sub-pattern of the same state (2^%d terms, %.1f s, ~212-bit "
                                          "decision-tree oracle)" % (args.cpu_sample, args.cpu_sample, dt),
                                "single_core": {"value": rate1, "sample": "N=%d sub-pattern, %.1f s, one thread"
                                                % (args.cpu_sample_single, dt1)}}
        if args.prec == "fp64" and args.basis == "real":
            line["cpu_fp64"] = cpu_fp64_block(ctx, gbs, st, modes, value)
    line["summary"] = summary_of(line)
    if rank == 0:
        print(json.dumps(line), flush=True)
    st.free()
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
