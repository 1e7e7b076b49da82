#!/usr/bin/env python3
"""Throughput of the fused EM-Step on one GB300: particle-steps per second.

Workload (per GPU): the 16-edge Langevin star -- lengths U[0.5, 2],
quadratic potentials V_e = a_e (x - c_e)^2 with a_e ~ U[0.5, 4], c_e ~ U[0,
L_e], sigma = sqrt(2), equal jump weights, reflecting leaves -- with
N = 2^24 particles, dt = 1e-3, M = 16 splits per step at most, FP32-mixed,
and a fused 32-bin-per-edge snapshot histogram.  One benchmark step is one
mg_simulate call of 10^4 EM-Steps over all particles (one kernel launch) on
device-resident state.  The state (N x 24 bytes = 403 MB) is larger than L2
(129 MB), so no explicit flush is needed between steps.

Printed: one JSON line (rank 0).  ``value`` is device-timed (CUDA events on
the launch stream); ``e2e`` times the same work through the C ABI with host
buffers: positions uploaded from pinned host memory (mg_particles_reset),
mg_simulate, the histogram and the counters read back to the host.
``--impl reference`` times the plain CPU oracle on the host cores instead.
Under torchrun each rank simulates its own N particles (ids rank*N ..), so
the scaling is weak; there is no collective on the data path.
``--workload`` runs the other configurations instead (the 3-edge Brownian
star, the vascular network, the 512-instance batch, the served trace).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2512_02175_gb300 import workloads as W  # noqa: E402

DT, EM_STEPS, M, BINS, SEED = 1e-3, 10_000, 16, 32, 0
# Algorithmic thread-instructions of one particle-step on the fast path (the
# floor without vertex hits): Philox-4x32-10 per 4 steps = 10 rounds x (2 wide
# multiplies + 2 three-input XORs) / 4 = 10; Box-Muller per normal = 7; EM
# update 2 FMA, interior test 2 compares + 1 branch = 5; loop control 1.
I_ALG = 23
# Thread-instructions per particle-step of the fast path plus the vertex
# splits' share (the estimate 35-45; its middle)
I_MIN = 40
METRIC = "particle-steps/sec"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp32", "fp64"], default=None,
                    help="default: mixed (star3_brownian: fp64; vascular and batch512: fp32 -- "
                         "each as its configuration is given)")
    ap.add_argument("--split-batch", type=int, default=0)
    ap.add_argument("--n", type=int, default=1 << 24)
    ap.add_argument("--em-steps", type=int, default=EM_STEPS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-hist", action="store_true",
                    help="time the EM-Steps without the fused histogram tail")
    ap.add_argument("--no-extras", action="store_true",
                    help="star16_langevin: skip the FP32, FP64 and served sub-measurements "
                         "the default line carries")
    ap.add_argument("--full", action="store_true",
                    help="served: the configured request sizes (n = 2^U[14,24]) over a 10-s "
                         "Poisson window instead of the reduced trace")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="batch512: scale every instance's particle count by this factor")
    ap.add_argument("--cpu-sample", type=int, default=16_384)
    ap.add_argument("--workload", default="star16_langevin",
                    choices=["star16_langevin", "star3_brownian", "vascular", "batch512",
                             "served"],
                    help="star16_langevin is the headline; the others report the "
                         "vascular, batched and served configurations")
    args = ap.parse_args()
    args.precision_given = args.precision is not None
    if args.precision is None:
        args.precision = "mixed"
    return args


def config(args, world):
    return {"workload": "star16_langevin", "graph": "star, 16 edges, L~U[0.5,2], quadratic "
            "potentials, sigma=sqrt(2), equal b, reflecting leaves",
            "n_particles_per_gpu": args.n, "global_particles": args.n * world,
            "dt": DT, "em_steps_per_step": args.em_steps, "M": M,
            "hist_bins_per_edge": 0 if args.no_hist else BINS,
            "precision": {"mixed": "fp32 positions, increments and normals; the split's "
                                   "hitting fraction (root to binary64 accuracy, alpha = s^2) "
                                   "and time left in fp64",
                          "fp32": "fp32 throughout", "fp64": "fp64 throughout"}[args.precision],
            "parallelism": f"particle shards x{world}",
            "l2": f"state {28 if args.precision == 'fp64' else 24} B/particle x N > L2 (129 MB): "
                  "no flush needed"}


# ------------------------------------------------------------------ clocks

class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms",
               "200"]
        if gpu_id is not None:
            cmd += ["-i", str(gpu_id)]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 6]
        os.unlink(self.f.name)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm = [float(r[0]) for r in rows if r[0].strip().replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[3 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------ cpu oracle

def _oracle_chunk(args):
    desc, edge, x, pid, steps = args
    from oracle import oracle as O
    g = O.Graph.from_desc(desc)
    st = O.State(edge, x, pid)
    cnt = O.Counters(g)
    O.simulate(g, st, cnt, seed=SEED, instance=0, dt=DT, steps=steps, M=M)
    return int(cnt.particle_steps[0])


def cpu_oracle(desc, e0, x0, sample, steps, pool, cores):
    """Times the plain oracle on `sample` particles x `steps` EM-Steps."""
    d = {k: desc[k] for k in ("n_vertices", "src", "dst", "length", "c0", "c1", "sigma",
                              "w_init", "w_term")}
    b = np.linspace(0, sample, cores + 1).astype(int)
    jobs = [(d, e0[i:j], x0[i:j], np.arange(i, j, dtype=np.uint32), steps)
            for i, j in zip(b[:-1], b[1:]) if j > i]
    t = time.perf_counter()
    ps = sum(pool.map(_oracle_chunk, jobs))
    return ps, time.perf_counter() - t


def make_pool():
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    return mp.get_context("spawn").Pool(cores), cores


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    desc = W.star_langevin(16)
    e0, x0 = W.uniform_on_edges(desc, args.cpu_sample, 11)
    pool, cores = make_pool()
    sample = args.cpu_sample
    for _ in range(args.warmup):
        cpu_oracle(desc, e0, x0, sample, args.em_steps, pool, cores)
    total_ps, total_t = 0, 0.0
    for _ in range(args.steps):
        ps, t = cpu_oracle(desc, e0, x0, sample, args.em_steps, pool, cores)
        total_ps += ps
        total_t += t
    pool.close()
    v = total_ps / total_t
    desc_sample = (f"{sample} particles x {args.em_steps} EM-Steps per step of the "
                   f"star16_langevin workload (pids 0..{sample - 1}), FP64 oracle, "
                   f"{cores} processes")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "particle-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(args, 1),
        "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": cores,
                         "kind": "oracle", "sample": desc_sample},
        "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))
    return 0


# --------------------------------------------------------------- our path

PROFILE_KEYS = ("kernel-sha256", "dram-bytes-per-launch-full-size", "issue-active-pct",
                "warp-inst-per-warp-step", "fp64-pipe-active-pct")
PROFILE_N = 1 << 24  # particles of the launch the summaries' traffic is scaled to


def _profile(kernel_hash, name="em_step_star16_langevin.md"):
    """Figures of a committed ncu summary of the fused kernel (the FP32-mixed
    one by default), if it was taken on the current kernel source (else an
    empty dict)."""
    path = os.path.join(ROOT, "profiles", name)
    rec = {}
    try:
        with open(path) as f:
            for line in f:
                if ":" in line and line.split(":", 1)[0] in PROFILE_KEYS:
                    k, v = line.split(":", 1)
                    rec[k] = v.strip()
    except OSError:
        return {}
    return rec if rec.get("kernel-sha256") == kernel_hash else {}


def _traffic(prof, n):
    """DRAM bytes per launch of n particles from an ncu summary (state
    traffic is per particle per launch), or null."""
    v = prof.get("dram-bytes-per-launch-full-size")
    return int(int(v) * n / PROFILE_N) if v else None


def kernel_hash():
    """sha256 of the sources that define the fused EM-Step kernel (its body,
    its table layouts and the logarithm table of the binary64 mode): a
    committed ncu figure counts only while these are unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2512_02175_gb300", "csrc")
    for f in ("mg_em_step.cuh", "mg_types.h", "mg_log_table.h"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def time_precision(B, torch, g, e0, x0, precision, em_steps, steps, warmup, stream):
    """Particle-steps/s of `steps` launches of `em_steps` EM-Steps of the
    benchmark's workload (fused histogram) in another precision mode, timed
    like the headline (CUDA events on the launch stream, resident state)."""
    p = B.Particles(g, e0, x0, seed=SEED, precision=_mode(B, precision), stream=stream)
    hist = torch.zeros(g.n_edges * BINS, dtype=torch.int32, device="cuda")

    def step():
        hist.zero_()
        p.simulate(DT, em_steps, M, BINS, hist, stream)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step()
    torch.cuda.synchronize()
    c0 = p.counts(stream)["particle_steps"]
    ev = _events(torch, steps)
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(steps):
            step()
            ev[k + 1].record(stream)
    torch.cuda.synchronize()
    ps = p.counts(stream)["particle_steps"] - c0
    ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    p.close()
    return {"value": ps / (sum(ms) / 1e3), "unit": "particle-steps/s",
            "ms_per_launch": statistics.mean(ms), "em_steps_per_launch": em_steps,
            "launches": steps, "warmup": warmup, "n_particles": len(e0)}


def sub_measurements(args, B, torch, g, e0, x0, stream):
    """The metric's other parts, measured in the same run: the FP32 and FP64
    modes on the same workload (FP64 at 10^3 EM-Steps per launch), and the
    served trace (continuous batching, FP32-mixed and FP64, against the plain
    one-launch-per-request FP64 path)."""
    out = {}
    fp32 = time_precision(B, torch, g, e0, x0, "fp32", args.em_steps, 3, 2, stream)
    out["fp32"] = fp32
    fp64 = time_precision(B, torch, g, e0, x0, "fp64", 1000, 2, 1, stream)
    prof = _profile(kernel_hash(), "em_step_star16_fp64.md")
    fp64["roofline"] = {"bound": "fp64", "unit": "FP64-pipe busy fraction",
                        "frac": float(prof["fp64-pipe-active-pct"]) / 100.0 if prof else None,
                        "source": "ncu capture of the binary64 kernel "
                                  "(profiles/em_step_star16_fp64.md), while its source hash "
                                  "matches"}
    out["fp64"] = fp64
    torch.cuda.synchronize()
    out["served"] = served_trace(B, torch, full=False)
    return out


def run_ours(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    desc = W.star_langevin(16)
    n = args.n
    # the rank's shard: particles rank*n .. rank*n + n - 1 of the global workload
    e0, x0 = W.uniform_on_edges(desc, n, 11 + rank)
    pool = cores = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool, cores = make_pool()  # spawn, before the first CUDA call
        ce, cx = W.uniform_on_edges(desc, args.cpu_sample, 11)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2512_02175_gb300 import binding as B
    B.load()
    B.use_torch_allocator()
    prec = {"mixed": B.MG_FP32_MIXED, "fp32": B.MG_FP32, "fp64": B.MG_FP64}[args.precision]
    stream = torch.cuda.Stream()
    g = B.Graph(desc)
    p = B.Particles(g, e0, x0, pid_base=rank * n, seed=SEED, precision=prec, stream=stream)
    if args.split_batch:
        p.set_tuning(split_batch=args.split_batch)
    hist = torch.zeros(g.n_edges * BINS, dtype=torch.int32, device="cuda")

    def step():
        if args.no_hist:
            p.simulate(DT, args.em_steps, M, 0, None, stream)
        else:
            hist.zero_()
            p.simulate(DT, args.em_steps, M, BINS, hist, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    c0 = p.counts(stream)["particle_steps"]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local if "CUDA_VISIBLE_DEVICES" not in os.environ else None)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(args.steps):
            step()
            ev[k + 1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launch_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    elapsed = sum(launch_ms) / 1e3
    ps = p.counts(stream)["particle_steps"] - c0
    if dist:
        t = torch.tensor([elapsed], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
        s = torch.tensor([ps], device="cuda", dtype=torch.float64)
        dist.all_reduce(s)
        ps = int(s.item())
    value = ps / elapsed
    per_launch = ps / (world * args.steps)
    achieved = I_ALG * per_launch / (statistics.mean(launch_ms) / 1e3) / 1e12  # Tinst/s
    props = torch.cuda.get_device_properties(local)
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * 128 * sm_max * 1e6 / 1e12
    if args.precision == "fp64":
        # bound by the binary64 pipe: its busy fraction in the committed ncu
        # capture of the binary64 kernel (while that matches the source)
        prof = _profile(kernel_hash(), "em_step_star16_fp64.md")
        phi = float(prof["fp64-pipe-active-pct"]) / 100.0 if prof else None
        roofline = {"bound": "fp64", "achieved": phi, "peak": 1.0 if prof else None,
                    "unit": "FP64-pipe busy fraction", "frac": phi,
                    "traffic": _traffic(prof, n),
                    "note": "binary64 pipe cycles active / peak (ncu, "
                            "profiles/em_step_star16_fp64.md); the binary64 mode is "
                            "bound by GB300's binary64 rate"}
    else:
        # the summary's figures describe the FP32-mixed kernel
        prof = _profile(kernel_hash()) if args.precision == "mixed" else {}
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinst/s",
                    "frac": achieved / peak, "traffic": _traffic(prof, n),
                    "note": f"{I_ALG} algorithmic thread-instructions per particle-step (fast "
                            f"path) x particle-steps per launch / mean launch time; peak = "
                            f"{props.multi_processor_count} SMs x 128 lanes x {sm_max:.0f} MHz",
                    # the same against the estimate of 35-45 instructions per
                    # particle-step that counts the splits' share (40 taken)
                    "frac_at_i_min_40": achieved * I_MIN / I_ALG / peak}
        if prof:  # the issue-rate view, from the committed ncu capture of this kernel
            roofline["issue_active_frac"] = float(prof["issue-active-pct"]) / 100.0
            roofline["warp_inst_per_warp_step"] = float(prof["warp-inst-per-warp-step"])

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        he = torch.from_numpy(e0).pin_memory()
        hx = torch.from_numpy(x0).pin_memory()
        hh = np.zeros(g.n_edges * BINS, np.uint32)
        e2e_steps = max(1, min(args.steps, 3))
        times, eps = [], 0
        for k in range(e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p.reset(he.numpy(), hx.numpy(), stream)
            p.simulate(DT, args.em_steps, M, 0, None, stream)
            p.histogram(BINS, hh, stream)
            cnt = p.counts(stream)
            dt_ = time.perf_counter() - t0
            if k > 0:  # first round warms the allocator and the host pages
                times.append(dt_)
                eps += cnt["particle_steps"]
        h2d = int(he.numel() * 4 + hx.numel() * 8)
        d2h = int(hh.nbytes + 8 * (g.n_slots + g.n_vertices + 2))
        e2e = {"value": eps / sum(times) * world, "unit": "particle-steps/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    cpu = None
    if pool is not None:
        ps_c, t_c = cpu_oracle(desc, ce, cx, args.cpu_sample, args.em_steps, pool, cores)
        pool.close()
        cpu = {"value": ps_c / t_c, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_sample} particles x {args.em_steps} EM-Steps of the same "
                         f"workload (pids 0..{args.cpu_sample - 1}), FP64 oracle, one process "
                         f"per core"}
    counts = p.counts(stream)
    p.close()
    extras = {}
    if world == 1 and not args.no_extras:
        extras = sub_measurements(args, B, torch, g, e0, x0, stream)
    g.close()
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
            "config": config(args, world), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": args.steps, "clocks": clk,
            "nominal_particle_steps_per_s": n * world * args.em_steps * args.steps / elapsed,
            "launch_ms": launch_ms,
            "truncations": counts["truncations"],
        }
        out.update(extras)
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------- other configurations

def _mode(B, precision):
    return {"mixed": B.MG_FP32_MIXED, "fp32": B.MG_FP32, "fp64": B.MG_FP64}[precision]


def _events(torch, k):
    return [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]


def run_vascular(args):
    """The synthetic vascular network: 2^26 tracers injected at the inlets,
    2000 EM-Steps (dt = 10x the explicit one-cell finite-volume limit), M = 32,
    16-bin histograms, FP32 as that configuration is given (--precision
    overrides); each benchmark step restarts from the injected state
    (device-resident) so every step does the same work."""
    import torch
    from paper_2512_02175_gb300 import binding as B
    d = W.vascular()
    n = 1 << 26 if args.n == (1 << 24) else args.n
    steps = 2000 if args.em_steps == EM_STEPS else args.em_steps
    Mv, bins = 32, 16
    prec = args.precision if args.precision_given else "fp32"
    e0, x0 = W.inject_at_inlets(d, n, 11)
    B.load()
    B.use_torch_allocator()
    stream = torch.cuda.Stream()
    g = B.Graph(d)
    de, dx = torch.from_numpy(e0).cuda(), torch.from_numpy(x0).cuda()
    p = B.Particles(g, de, dx, seed=SEED, precision=_mode(B, prec), stream=stream)
    if args.split_batch:
        p.set_tuning(split_batch=args.split_batch)
    hist = torch.zeros(g.n_edges * bins, dtype=torch.int32, device="cuda")

    def step():
        p.reset(de, dx, stream)
        hist.zero_()
        p.simulate(d["dt"], steps, Mv, bins, hist, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    ev = _events(torch, args.steps)
    ps = 0
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(args.steps):
            step()
            ev[k + 1].record(stream)
    torch.cuda.synchronize()
    c = p.counts(stream)
    ps = c["particle_steps"] * args.steps  # counters restart with every reset
    ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    out = {"metric": METRIC, "value": ps / (sum(ms) / 1e3), "unit": "particle-steps/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": statistics.mean(ms), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32",
           "data": "synthetic",
           "config": {"workload": "vascular", "vertices": int(d["n_vertices"]),
                      "edges": int(len(d["src"])), "n_particles": n, "dt_s": d["dt"],
                      "em_steps_per_step": steps, "M": Mv, "hist_bins_per_edge": bins,
                      "precision": prec},
           "absorbed_fraction": float(sum(c["absorbed"]) / n),
           "truncations_per_step": c["truncations"] / steps, "launch_ms": ms}
    p.close()
    g.close()
    print(json.dumps(out))
    return 0


def run_star3(args):
    """The small star: 3 edges of length 1, standard Brownian motion, 10^4
    particles round-robin on the edges, dt = 1e-3, 1000 EM-Steps, M = 8,
    32-bin histograms and the exit counts; FP64 unless --precision says
    otherwise.  Each benchmark step restarts from the device-resident start.
    The library spreads so small a set over the GPU's resident blocks (313
    blocks of 32 particles on 152 SMs), which still leaves most lanes idle:
    the number shows what a single small launch costs, not the kernel's
    throughput."""
    import torch
    from paper_2512_02175_gb300 import binding as B
    d = W.star_brownian(3)
    n = 10_000 if args.n == (1 << 24) else args.n
    steps = 1000 if args.em_steps == EM_STEPS else args.em_steps
    M3, bins = 8, 32
    prec = args.precision if args.precision_given else "fp64"
    e0, x0 = W.round_robin_uniform(d, n, 0)
    B.load()
    B.use_torch_allocator()
    stream = torch.cuda.Stream()
    g = B.Graph(d)
    de, dx = torch.from_numpy(e0).cuda(), torch.from_numpy(x0).cuda()
    p = B.Particles(g, de, dx, seed=0, precision=_mode(B, prec), stream=stream)
    if args.split_batch:
        p.set_tuning(split_batch=args.split_batch)
    hist = torch.zeros(g.n_edges * bins, dtype=torch.int32, device="cuda")

    def step():
        p.reset(de, dx, stream)
        hist.zero_()
        p.simulate(1e-3, steps, M3, bins, hist, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    ev = _events(torch, args.steps)
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(args.steps):
            step()
            ev[k + 1].record(stream)
    torch.cuda.synchronize()
    c = p.counts(stream)
    ps = c["particle_steps"] * args.steps  # counters restart with every reset
    ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    out = {"metric": METRIC, "value": ps / (sum(ms) / 1e3), "unit": "particle-steps/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": statistics.mean(ms), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32",
           "data": "synthetic",
           "config": {"workload": "star3_brownian", "edges": 3, "n_particles": n, "dt": 1e-3,
                      "em_steps_per_step": steps, "M": M3, "hist_bins_per_edge": bins,
                      "precision": prec,
                      "l2": "state below L2; each step restarts from the same start"},
           "centre_exits": [int(v) for v in c["exits"][:3]], "launch_ms": ms}
    p.close()
    g.close()
    print(json.dumps(out))
    return 0


def run_batch512(args):
    """512 uneven instances (stars with 3..64 edges, random trees with
    100..10^4 edges, N ~ 2^U[12,22], 100..5000 steps) in one persistent launch,
    replayed from a captured CUDA graph, with autotuned launch tuning; FP32 as
    that configuration is given (--precision fp64 for its FP64 variant)."""
    import torch
    from paper_2512_02175_gb300 import autotune as A
    from paper_2512_02175_gb300 import binding as B
    B.load()
    B.use_torch_allocator()
    insts = W.batch_instances(512, n_scale=args.scale)
    prec_name = args.precision if args.precision_given else "fp32"
    prec = _mode(B, prec_name)
    graphs, parts = [], []
    for k, it in enumerate(insts):
        g = B.Graph(it["graph"])
        e, x = W.uniform_on_edges(it["graph"], it["n"], 100 + k)
        parts.append(B.Particles(g, e, x, seed=SEED, instance=k, precision=prec))
        graphs.append(g)
    stream = torch.cuda.Stream()

    def make(steps_of):
        b = B.Batch()
        for p, it in zip(parts, insts):
            b.add(p, it["dt"], steps_of(it), it["M"])
        return b

    def trial(t):
        b = make(lambda it: max(1, it["steps"] // 50))
        b.set_tuning(**t.as_dict())
        b.run(False, stream)  # build
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.run(False, stream)
        torch.cuda.synchronize()
        dt_ = time.perf_counter() - t0
        b.close()
        return dt_

    key = f"{torch.cuda.get_device_name()}-prec{prec}-batch512"
    tun = A.tune(key, trial)
    b = make(lambda it: it["steps"])
    b.set_tuning(**tun.as_dict())
    for _ in range(args.warmup):
        b.run(True, stream)
    torch.cuda.synchronize()
    c0 = sum(p.counts(stream)["particle_steps"] for p in parts)
    ev = _events(torch, args.steps)
    ev[0].record(stream)
    for k in range(args.steps):
        b.run(True, stream)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    ps = sum(p.counts(stream)["particle_steps"] for p in parts) - c0
    ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    n_members, n_items, blocks = b.info()
    out = {"metric": METRIC, "value": ps / (sum(ms) / 1e3), "unit": "particle-steps/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": statistics.mean(ms), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if prec_name == "fp64" else "f32",
           "data": "synthetic",
           "config": {"workload": "batch512", "instances": n_members, "work_items": n_items,
                      "persistent_blocks": blocks, "particles": int(sum(i["n"] for i in insts)),
                      "particle_steps_per_step": int(sum(i["n"] * i["steps"] for i in insts)),
                      "cuda_graph": True, "tuning": tun.as_dict(), "precision": prec_name,
                      "particle_scale": args.scale},
           "launch_ms": ms}
    b.close()
    for p in parts:
        p.close()
    for g in graphs:
        g.close()
    print(json.dumps(out))
    return 0


SERVED_GRAPHS = None


def served_trace(B, torch, full=False, precisions=None):
    """A Poisson request stream (200 requests/s) over the 3-edge Brownian
    star, the 16-edge Langevin star and the vascular network; steps
    log-U[100, 5000], dt log-U[1e-4, 1e-2]; n = 2^U[12,18] over 3 s (the
    reduced trace), or with ``full`` the configured n = 2^U[14,24] over 10 s
    (about 6e11 particle-steps offered per second, more than one GPU
    serves).  The continuous-batching server (2 streams, rounds of max(500
    steps, 2^27 particle-steps) per member, 32 GB admission budget) in each
    of ``precisions`` (default: FP32-mixed and FP64 on the reduced trace;
    FP32-mixed alone on the full one, which offers some 70 times what the
    FP64 path can do, so the equal-accuracy comparison is the reduced
    trace's), then the plain path -- each request alone as one FP64
    mg_simulate, in arrival order -- on the same trace.  A run is cut off
    after 120 s (full) or 600 s: unanswered requests count as latencies
    beyond the cut (their percentiles are then reported as lower bounds).
    The trace -- its requests' starting positions included -- is generated
    once, before any timing, and replayed by every run."""
    import copy

    from paper_2512_02175_gb300 import serve
    if precisions is None:
        precisions = ("mixed",) if full else ("mixed", "fp64")
    graphs = {"star3": W.star_brownian(3), "star16": W.star_langevin(16),
              "vascular": W.vascular()}
    rate, window, n_range, limit = (200.0, 10.0, (14, 24), 120.0) if full else \
        (200.0, 3.0, (12, 18), 600.0)
    reqs = serve.poisson_trace(rate, window, 17, graphs, n_range=n_range,
                               init=serve.default_init)
    trace = lambda: [copy.copy(r) for r in reqs]  # run_trace rebases the arrivals
    offered = sum(r.n * r.steps for r in reqs)
    out = {"trace": {"rate_per_s": rate, "window_s": window, "requests": len(reqs),
                     "n_range_log2": list(n_range), "steps_range": [100, 5000],
                     "dt_range": [1e-4, 1e-2], "offered_particle_steps_per_s": offered / window,
                     "cut_off_s": limit, "lanes": 2, "chunk_steps": 500,
                     "round_work": 1 << 27}}

    def summary(results, t_run):
        s = serve.latency_summary(results)
        ok = [r for r in results if r.error is None]
        s["answered"] = len(ok)
        s["wall_s"] = t_run
        if len(ok) < len(reqs):  # open requests waited at least until the cut
            lat = np.sort([r.latency for r in ok] + [np.inf] * (len(reqs) - len(ok)))
            for q, key in ((50, "p50_s"), (99, "p99_s")):
                v = float(lat[max(0, math.ceil(q / 100 * len(lat)) - 1)])  # nearest rank
                s[key] = v if np.isfinite(v) else None
                if not np.isfinite(v):
                    s[key + "_at_least"] = limit - window
        return s

    for prec in precisions:
        be = serve.GpuBackend(graphs, _mode(B, prec), seed=SEED, n_lanes=2)
        srv = serve.Server(be, mem_budget=32 << 30, n_lanes=2, chunk_steps=500,
                           round_work=1 << 27)
        warm = serve.poisson_trace(200.0, 0.2, 99, graphs, n_range=(10, 12),
                                   init=serve.default_init)
        srv.run_trace(warm)
        srv.results = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = srv.run_trace(trace(), time_limit=limit, partial=True)
        out[f"served_{prec}"] = summary(res, time.perf_counter() - t0)
        be.close()
        torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = serve.serve_plain(trace(), graphs, B.MG_FP64, seed=SEED, time_limit=limit)
    out["plain_fp64"] = summary(plain, time.perf_counter() - t0)
    return out


def run_served(args):
    """The served configuration alone (see served_trace): its line reports the
    FP32-mixed served throughput as ``value``, every served and plain
    summary beside it."""
    import torch
    from paper_2512_02175_gb300 import binding as B
    B.load()
    B.use_torch_allocator()
    res = served_trace(B, torch, full=args.full)
    out = {"metric": METRIC, "value": res["served_mixed"]["served_particle_steps_per_s"],
           "unit": "particle-steps/s", "n_gpus": 1, "steps": 1, "warmup": 1,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": "served_full" if args.full else "served", **res["trace"]},
           **{k: v for k, v in res.items() if k != "trace"}}
    print(json.dumps(out))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "vascular":
        return run_vascular(args)
    if args.workload == "star3_brownian":
        return run_star3(args)
    if args.workload == "batch512":
        return run_batch512(args)
    if args.workload == "served":
        return run_served(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
