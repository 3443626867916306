#!/usr/bin/env python
"""Throughput of the dipolar Barnes-Hut ferrofluid step on GB300.

Metric: particle-steps/s of the full step (root cube, Morton keys, radix
sort, tree build, aggregation, traversal with near-field pairs, integration
with Philox noise, FP64 observables) on N = 1,048,576 dipoles at volume
fraction 0.05, FP32, theta = 0.5, next to the GPU all-pairs kernel and the
FP64 path.  One JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--gpus N > 1 runs under torch.distributed.run: every rank advances its own
replica of the workload (the single-system method does not shard), timing
is the maximum over ranks, and value counts all ranks' particle-steps.
--workload batched steps 256 independent dilute systems of uneven sizes
together (one forest, one CUDA graph per step); on several GPUs each rank
takes its own batch (weak scaling) or, with --split, a particle-balanced
share of one batch (strong scaling).  Systems never interact, so no rank
exchanges data while stepping.
--impl reference times the CPU oracle on this host's cores instead.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s at 1M particles theta=0.5 (FP32 BH vs GPU all-pairs vs FP64)"
UNIT = "particle-steps/s"
# algorithmic FP32 operations of one dipole interaction (field + force, FMA = 2):
# separation 3, r^2 5, rsqrt 1, powers of 1/r 4, three dot products 15,
# field 14, force 26
FLOPS_PER_INTERACTION = 68


def simt_peaks(dev):
    """FP32 and FP64 fused multiply-add rates of this GPU, measured by the library's FMA-chain
    microbenchmark (libffpeak.so: every thread runs independent FMA chains; CUDA events; the
    SM clock read from the SMs' own counters during the run).  The FP32 peak is the larger of
    the scalar and the paired (two floats per instruction) forms."""
    import ctypes

    from paper_1212_2934_gb300 import _build

    L = ctypes.CDLL(_build.PEAK_LIB)
    L.ffp_simt_peak.restype = ctypes.c_int
    out = {}
    for kind, name in ((0, "fp32_fma"), (1, "fp32_fma2"), (2, "fp64_fma")):
        tf, ms, mhz = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        rc = L.ffp_simt_peak(kind, int(dev), ctypes.byref(tf), ctypes.byref(ms),
                             ctypes.byref(mhz))
        if rc != 0:
            raise RuntimeError("SIMT peak microbenchmark failed (%s): %d" % (name, rc))
        out[name] = {"tflops": tf.value, "launch_ms": ms.value, "sm_mhz": mhz.value}
    out["fp32_tflops"] = max(out["fp32_fma"]["tflops"], out["fp32_fma2"]["tflops"])
    out["fp64_tflops"] = out["fp64_fma"]["tflops"]
    return out


def peak_note(pk, key):
    parts = ["%s %.2f TFLOP/s at %.0f MHz" % (k, pk[k]["tflops"], pk[k]["sm_mhz"])
             for k in (("fp32_fma", "fp32_fma2") if key == "fp32" else ("fp64_fma",))]
    return ("measured by the FMA-chain microbenchmark (csrc/peak/simt_peak.cu) in this run: "
            + "; ".join(parts))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1048576)
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--leaf-max", type=int, default=1)
    ap.add_argument("--group", type=int, default=0,
                    help="lanes walking the cell list together (0: picked by the library's "
                         "autotuner on the workload before warm-up)")
    ap.add_argument("--schedule", type=int, default=0,
                    help="traversal launch schedule (ff_schedule_info index); 0: tuned on the "
                         "workload before warm-up unless --group is given")
    ap.add_argument("--workload", default="phi05", choices=["phi05", "batched", "chains", "grad"],
                    help="phi05: one system of --n particles (default); batched: 256 independent "
                         "dilute systems of log-uniform sizes 1,024..65,536 at fields 0..5; "
                         "chains: 65,536 straight chains of 64 touching dipoles (4,194,304 "
                         "particles) at volume fraction 0.01, FP32 with the mixed and FP64 paths "
                         "timed beside it; grad: gradient of the dipolar energy with respect to "
                         "all positions and moments at N = 262,144, volume fraction 0.05")
    ap.add_argument("--split", action="store_true",
                    help="batched workload on several GPUs: share one 256-system batch among "
                         "the ranks (strong scaling) instead of one batch per rank (weak)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the all-pairs, FP64, e2e and CPU-baseline legs")
    return ap.parse_args()


def workload(n, seed=1):
    """Synthetic ensemble (generated once per host and cached under the temp dir)."""
    from paper_1212_2934_gb300 import synth

    path = os.path.join(tempfile.gettempdir(), "ff_phi05_n%d_s%d.npz" % (n, seed))
    if os.path.exists(path):
        d = np.load(path)
        pos, u, side = d["pos"], d["u"], float(d["side"])
    else:
        e = synth.make_ensemble("phi05", seed=seed, n=n)
        pos, u, side = e["pos"], e["u"], e["side"]
        tmp = path + ".%d.npz" % os.getpid()
        np.savez(tmp, pos=pos, u=u, side=side)
        os.replace(tmp, path)
    return pos, u, side


def batched_workload(seed=1):
    """256 dilute systems (phi 0.02), sizes log-uniform in [1024, 65536], fields 0..5 along z
    (generated once per host and cached under the temp dir)."""
    from paper_1212_2934_gb300 import synth

    path = os.path.join(tempfile.gettempdir(), "ff_batched256_s%d.npz" % seed)
    if os.path.exists(path):
        d = np.load(path)
        return {k: d[k] for k in d.files}
    b = synth.batched_ensembles(256, 0.02, 5.0, seed)
    tmp = path + ".%d.npz" % os.getpid()
    np.savez(tmp, **b)
    os.replace(tmp, path)
    return b


BATCHED_METRIC = ("particle-steps/s, 256 batched ensembles (N 1,024..65,536 log-uniform, "
                  "phi 0.02, fields 0..5, theta=0.5)")


def batched_config(args, n, world):
    return {"workload": "256 independent systems, sizes round(1024 64^((i+1/2)/256)) "
                        "(3,970,997 particles), phi = 0.02 hard-core gases, isotropic moments, "
                        "applied fields 0..5 along z on a linear grid (seeded permutation), "
                        "dip_scale 1/8, kT = 1, Gamma_t = Gamma_r = 1, dt = 1e-3, LJ, walls",
            "n": n, "systems": 256, "theta": args.theta, "leaf_max": args.leaf_max,
            "precision": "fp32", "algo": "barnes-hut",
            "l2": "flushed between timed steps (256 MB write outside the timed events)",
            "parallelism": ("single-gpu" if world == 1 else
                            "one 256-system batch shared among the ranks (particle-balanced "
                            "split), no data-path exchange; per-system moments gathered after "
                            "timing" if args.split else
                            "one independent 256-system batch per rank (seed 1 + rank), no "
                            "data-path exchange; per-system moments gathered after timing")}


CHAINS_METRIC = ("particle-steps/s, 4,194,304 dipoles in 65,536 chains of 64, phi 0.01, "
                 "theta=0.5 (FP32 BH; mixed and FP64 beside)")
CHAINS, CHAIN_LEN = 65536, 64


def chains_workload(seed=1):
    """65,536 straight chains of 64 touching dipoles, isotropic axes, head-to-tail moments with a
    random sign per chain, at volume fraction 0.01 (generated once per host and cached)."""
    from paper_1212_2934_gb300 import synth

    path = os.path.join(tempfile.gettempdir(), "ff_chains%dx%d_s%d.npz" % (CHAINS, CHAIN_LEN, seed))
    if os.path.exists(path):
        d = np.load(path)
        return d["pos"], d["u"], float(d["side"])
    side = synth.box_side_for_fraction(CHAINS * CHAIN_LEN, 0.01)
    pos, u = synth.chains_cube(CHAINS, CHAIN_LEN, side, seed)
    pos, u = pos.astype(np.float32), u.astype(np.float32)
    tmp = path + ".%d.npz" % os.getpid()
    np.savez(tmp, pos=pos, u=u, side=side)
    os.replace(tmp, path)
    return pos, u, side


def chains_config(args, n, side, world):
    return {"workload": "65,536 straight chains of 64 touching dipoles (spacing 1), isotropic "
                        "axes, moments along the axis head-to-tail with a random sign per chain, "
                        "random sequential addition of rods at volume fraction 0.01, h_ext=(0,0,1), "
                        "kT=1, Gamma_t=Gamma_r=0.1, dt=1e-3, LJ eps=1 sigma=1 rcut=2.5, walls",
            "n": n, "box_side": round(side, 4), "theta": args.theta, "leaf_max": args.leaf_max,
            "precision": "fp32 (mixed and fp64 in paths)", "algo": "barnes-hut",
            "l2": "flushed between timed steps (256 MB write outside the timed events)",
            "parallelism": "replicas" if world > 1 else "single-gpu"}


def config_dict(args, side):
    return {
        "workload": "dipoles at volume fraction 0.05 (hard core 1.0, RSA), isotropic moments, "
                    "h_ext=(0,0,1), kT=1, Gamma_t=Gamma_r=0.1, dt=1e-3, LJ eps=1 sigma=1 "
                    "rcut=2.5, LJ walls",
        "n": args.n, "box_side": round(side, 4), "theta": args.theta, "leaf_max": args.leaf_max,
        "traverse_group": args.group or "default",
        "precision": "fp32", "algo": "barnes-hut",
        "l2": "flushed between timed steps (256 MB write outside the timed events); "
              "per-step working set ~0.3 GB",
        "parallelism": "replicas" if args.gpus > 1 else "single-gpu",
    }


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons; only samples whose timestamps fall
    inside the marked timed window are reported."""

    FIELDS = ["timestamp", "clocks.sm", "clocks.max.sm", "power.draw",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.out = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # wait (bounded) for the first sample so the window is covered from its start
        for _ in range(50):
            time.sleep(0.1)
            if os.path.getsize(self.out.name) > 0:
                break

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().strip().splitlines() if r.strip()]
        os.unlink(self.out.name)
        import datetime

        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < len(self.FIELDS):
                continue
            try:
                ts = datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                c, m = float(r[1]), float(r[2])
            except ValueError:
                continue
            # a sample describes the interval that ends at its timestamp
            if self.t0 is not None and not (self.t0 - 0.05 <= ts <= self.t1 + 0.1):
                continue
            sm.append(c)
            mx.append(m)
            try:
                power.append(float(r[3]))
            except ValueError:
                pass
            for name, val in zip(names, r[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": float(np.median(power)) if power else None}


def traffic_for(kernel_src, n, workload, theta, leaf_max, schedule, kernel="k_bh"):
    """DRAM bytes per launch from the committed ncu summaries (one record per launch
    schedule), if one was taken on this source, this workload and this schedule."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        recs = json.load(open(path))
        sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()
        for d in recs if isinstance(recs, list) else [recs]:
            same = (d.get("kernel", "k_bh") == kernel and
                    d.get("source_sha256") == sha and d.get("n") == n and
                    d.get("workload_name") == workload and d.get("theta") == theta and
                    d.get("leaf_max") == leaf_max and d.get("schedule") == schedule)
            if same:
                return d.get("dram_bytes_per_launch")
    except (OSError, ValueError, AttributeError):
        pass
    return None


def max_over_ranks(x, device="cpu"):
    """Maximum of a float over the ranks of the default process group (the value itself
    when no group is initialised); the tensor lives on `device` (cuda for NCCL)."""
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(n_per_rank, steps, world, max_seconds):
    """Units all ranks processed divided by the slowest rank's time (replicas: weak scaling)."""
    return world * n_per_rank * steps / max_seconds


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_step_sample(pos, u, theta, leaf_max, side, sample, threads=None):
    """One CPU-oracle step on a bounded sample: tree + integration of all n, traversal of `sample`.

    Returns (particle-steps/s, seconds of CPU work, threads)."""
    import oracle

    if threads:
        oracle.set_threads(threads)
    n = pos.shape[0]
    p64 = pos.astype(np.float32).astype(np.float64)
    u = np.asarray(u, dtype=np.float64)
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(n, size=min(sample, n), replace=False))
    t0 = time.perf_counter()
    oracle.bh(p64, u, theta, leaf_max, "f32", 1.0, 1.0, 1.0, 2.5, True, only=idx[:1])
    t1 = time.perf_counter()
    r = oracle.bh(p64, u, theta, leaf_max, "f32", 1.0, 1.0, 1.0, 2.5, True, only=idx)
    t2 = time.perf_counter()
    st = dict(pos=p64.copy(), vel=np.zeros_like(p64), u=u.copy(), om=np.zeros_like(p64),
              id=np.arange(n, dtype=np.int64))
    dyn = oracle.make_dyn(h_ext=(0, 0, 1.0), box_lo=(0, 0, 0), box_hi=(side, side, side),
                          walls=True)
    t3 = time.perf_counter()
    oracle.em_step(st, r["h"], r["f"], dyn, 0)
    t4 = time.perf_counter()
    t_build = t1 - t0
    t_trav = max((t2 - t1) - t_build, 1e-9)
    t_int = t4 - t3
    per_step = t_build + t_int + t_trav * n / len(idx)
    return n / per_step, (t4 - t0), oracle.get_threads(), len(idx)


def cpu_allpairs_sample(pos, u, targets, threads=None):
    """The oracle's FP64 all-pairs field and force (Sec. 3.1) on `targets` sampled target
    particles against all n sources; returns (particle-steps/s extrapolated to all n targets,
    seconds, threads)."""
    import oracle

    if threads:
        oracle.set_threads(threads)
    n = pos.shape[0]
    p64 = pos.astype(np.float32).astype(np.float64)
    idx = np.sort(np.random.default_rng(6).choice(n, size=min(targets, n), replace=False))
    t0 = time.perf_counter()
    oracle.allpairs(p64, np.asarray(u, dtype=np.float64), lj_eps=1.0, only=idx)
    secs = time.perf_counter() - t0
    return n / (secs * n / len(idx)), secs, oracle.get_threads()


def cpu_baselines(pos, u, theta, leaf_max, side, sample):
    """The oracle on this host: Barnes-Hut on all cores (the headline CPU figure), Barnes-Hut
    on one core (the paper's Table 1 convention) and all-pairs on all cores and on one core,
    each on a bounded sample scaled to one full step."""
    import oracle

    cores = oracle.get_threads()
    rate, cpu_s, threads, s = cpu_step_sample(pos, u, theta, leaf_max, side, sample)
    n = pos.shape[0]
    out = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": "tree build, aggregation and integration of all %d particles plus "
                     "traversal of %d sampled particles (%.1f s of CPU work), scaled to one "
                     "full step" % (n, s, cpu_s)}
    try:
        r1, s1, t1, m1 = cpu_step_sample(pos, u, theta, leaf_max, side, max(sample // 32, 1024),
                                         threads=1)
        out["single_core"] = {"value": r1, "unit": UNIT, "cores": t1,
                              "sample": "as above on one core, traversal of %d sampled "
                                        "particles (%.1f s), scaled to one full step" % (m1, s1)}
        ra, sa, ta = cpu_allpairs_sample(pos, u, 2048, threads=cores)
        out["allpairs"] = {"value": ra, "unit": UNIT, "cores": ta,
                           "sample": "FP64 all-pairs field and force of 2048 sampled targets "
                                     "against all %d sources (%.1f s), extrapolated to all "
                                     "targets" % (n, sa)}
        ra1, sa1, ta1 = cpu_allpairs_sample(pos, u, 128, threads=1)
        out["allpairs_single_core"] = {
            "value": ra1, "unit": UNIT, "cores": ta1,
            "sample": "the same for 128 sampled targets on one core (%.1f s), extrapolated to "
                      "all targets" % sa1}
    finally:
        oracle.set_threads(cores)
    return out


def cpu_batched_sample(batch, theta, leaf_max, stride=8):
    """One CPU-oracle step of every stride-th system of a batch: tree, traversal and
    integration of all of its particles, with the system's own field and box.

    Returns (particle-steps/s, seconds of CPU work, threads, systems, particles)."""
    import oracle

    sizes = np.asarray(batch["sizes"], dtype=np.int64)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    pos = batch["pos"].astype(np.float32).astype(np.float64)
    u = batch["u"].astype(np.float64)
    picked = list(range(0, len(sizes), stride))
    secs, m = 0.0, 0
    for s in picked:
        a, b = int(starts[s]), int(starts[s + 1])
        p, us = pos[a:b], u[a:b]
        t0 = time.perf_counter()
        r = oracle.bh(p, us, theta, leaf_max, "f32", 0.125, 1.0, 1.0, 2.5, True)
        st = dict(pos=p.copy(), vel=np.zeros_like(p), u=us.copy(), om=np.zeros_like(p),
                  id=np.arange(a, b, dtype=np.int64))
        dyn = oracle.make_dyn(kT=1.0, gamma_t=1.0, gamma_r=1.0, h_ext=batch["fields"][s],
                              box_lo=batch["box_lo"][s], box_hi=batch["box_hi"][s], walls=True)
        oracle.em_step(st, r["h"], r["f"], dyn, 0)
        secs += time.perf_counter() - t0
        m += b - a
    return m / secs, secs, oracle.get_threads(), len(picked), m


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    if args.workload == "batched":
        return run_reference_batched(args)
    if args.workload == "grad":
        return run_reference_grad(args)
    if args.workload == "chains":
        pos, u, side = chains_workload(seed=1)
        args.n = pos.shape[0]
    else:
        pos, u, side = workload(args.n)
    sample = 65536
    for _ in range(args.warmup):
        cpu_step_sample(pos, u, args.theta, args.leaf_max, side, sample)
    rates = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r, _, threads, s = cpu_step_sample(pos, u, args.theta, args.leaf_max, side, sample)
        rates.append(r)
    wall = time.perf_counter() - t0
    value = float(np.mean(rates))
    cfg = config_dict(args, side) if args.workload != "chains" else chains_config(args, args.n,
                                                                                     side, 1)
    cfg["precision"] = "fp64 sums, fp32 tree"
    line = {
        "impl": "reference", "metric": METRIC if args.workload != "chains" else CHAINS_METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        # the bounded steps this run timed; a whole step of all particles would take
        # full_step_ms_extrapolated
        "ms_per_step": 1e3 * wall / args.steps, "full_step_ms_extrapolated": 1e3 * args.n / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "per step: tree build, aggregation and integration of all %d "
                                   "particles, traversal of %d sampled particles, scaled to all"
                                   % (args.n, s)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line))
    return 0


def run_reference_grad(args):
    """The oracle's energy gradient (all particles) per step on the gradient workload."""
    import oracle

    pos, u, side = workload(GRAD_N)
    p64 = pos.astype(np.float32).astype(np.float64)
    u64 = u.astype(np.float64)

    def once():
        oracle.bh_energy_grad(p64, u64, args.theta, args.leaf_max, "f32", lj_eps=1.0,
                              tree_centres=True)

    for _ in range(args.warmup):
        once()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        once()
    wall = time.perf_counter() - t0
    value = GRAD_N * args.steps / wall
    line = {
        "impl": "reference", "metric": GRAD_METRIC, "value": value,
        "unit": "particle-gradients/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "gradient of E_dip (Barnes-Hut, decisions frozen), volume "
                               "fraction 0.05", "n": GRAD_N, "theta": args.theta,
                   "leaf_max": args.leaf_max, "precision": "fp64 sums, fp32 tree"},
        "cpu_baseline": {"value": value, "unit": "particle-gradients/s",
                         "cores": oracle.get_threads(), "kind": "oracle",
                         "sample": "every step: the full gradient of all %d particles" % GRAD_N},
        "e2e": {"value": value, "unit": "particle-gradients/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line))
    return 0


def run_reference_batched(args):
    """The oracle on the batched workload: each step one full step of every 16th system."""
    batch = batched_workload()
    for _ in range(args.warmup):
        cpu_batched_sample(batch, args.theta, args.leaf_max, stride=16)
    rates = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r, _, threads, nsys_s, m = cpu_batched_sample(batch, args.theta, args.leaf_max, stride=16)
        rates.append(r)
    wall = time.perf_counter() - t0
    value = float(np.mean(rates))
    n = int(np.sum(batch["sizes"]))
    line = {
        "impl": "reference", "metric": BATCHED_METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * wall / args.steps, "full_step_ms_extrapolated": 1e3 * n / value,
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": batched_config(args, n, 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "per step: one full step of every 16th system (%d systems, "
                                   "%d particles), rate scaled by particle count" % (nsys_s, m)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    line["config"]["precision"] = "fp64 sums, fp32 tree"
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch

    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    import __graft_entry__

    __graft_entry__.build()
    from paper_1212_2934_gb300 import ff

    K, W = args.steps, args.warmup
    batch = None
    if args.workload == "batched":
        # every rank advances its own batch of 256 systems (seed 1 + rank): the systems are
        # independent, so ranks exchange nothing on the data path
        if args.split:
            # one batch shared among the ranks: each takes a particle-balanced share
            from paper_1212_2934_gb300 import shard

            full = batched_workload(seed=1)
            n_job = int(np.sum(full["sizes"]))
            mine = shard.partition_systems(full["sizes"], world)[rank]
            batch = shard.rank_slice(full, mine)
        else:
            batch = batched_workload(seed=1 + rank)
        pos, u = batch["pos"], batch["u"]
        side = float(batch["sides"].max())
        n = pos.shape[0]
    elif args.workload == "chains":
        pos, u, side = chains_workload(seed=1 + rank)
        n = pos.shape[0]
    else:
        n = args.n
        pos, u, side = workload(n)
    # a dedicated stream: the library launches on it, and the CUDA events, the L2
    # flush and every torch op of the timed region are issued on the same stream
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    def params(**kw):
        base = dict(n=n, precision="f32", theta=args.theta, leaf_max=args.leaf_max,
                    h_ext=(0, 0, 1.0), box_lo=(0, 0, 0), box_hi=(side, side, side), walls=1,
                    count_interactions=1, seed=1, device=dev, stream=stream.cuda_stream,
                    traverse_group=args.group)
        if batch is not None:
            # dilute, weakly coupled members (lambda = 0.25), near-critical damping
            base.update(dip_scale=0.125, gamma_t=1.0, gamma_r=1.0)
        base.update(kw)
        return ff.ff_params_default(**base)

    def create(p):
        c = ff.ff_create(p)
        if batch is not None:
            ff.ff_set_systems(c, batch["sizes"], batch["fields"], batch["box_lo"], batch["box_hi"])
        return c

    pos_d = torch.tensor(pos, dtype=torch.float32, device="cuda")
    u_d = torch.tensor(u, dtype=torch.float32, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- main leg: FP32 Barnes-Hut steps (interaction counting off while timed)
    ctx = create(params(count_interactions=0))
    ff.ff_set_particles(ctx, pos_d, u_d)
    tuning = None
    if args.schedule > 0:
        ff.ff_set_schedule(ctx, args.schedule)
        args.group = ff.ff_schedules()[args.schedule][0]
        tuning = {"chosen": "group %d, %d threads x %d blocks/SM (fixed by --schedule)"
                            % ff.ff_schedules()[args.schedule]}
    elif args.group == 0:
        # the traversal's launch schedule (lane group, block shape, blocks per SM) is picked by
        # the library's autotuner on this very workload; every choice gives the same bits, only
        # the speed differs
        scheds = ff.ff_schedules()
        best, tms = ff.ff_tune_schedule(ctx, reps=3)
        name = lambda i: "group %d, %d threads x %d blocks/SM" % scheds[i]
        tuning = {"chosen": name(best),
                  "ms_per_candidate": {name(i): round(m, 4) for i, m in tms.items()}}
        args.group = scheds[best][0]
        args.schedule = best
    clocks = Clocks(dev)
    clocks.start()
    for _ in range(W):
        ff.ff_step(ctx, 1)
        flush.zero_()
    ff.ff_synchronize(ctx)
    barrier()
    launches0 = ff.ff_profile_read(ctx)["launches"]
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    clocks.mark_start()
    for k in range(K):
        evs[k][0].record(stream)
        ff.ff_step(ctx, 1)  # one CUDA-graph launch per step
        evs[k][1].record(stream)
        flush.zero_()
    ff.ff_synchronize(ctx)
    clocks.mark_end()
    barrier()
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    launches = ff.ff_profile_read(ctx)["launches"] - launches0
    # stage breakdown and the traversal's own launch time: a separate pass with
    # CUDA events between the stages (eager launches on the same stream)
    kprof = min(K, 20)
    ff.ff_profile(ctx, True)
    for k in range(kprof):
        ff.ff_step(ctx, 1)
        flush.zero_()
    prof = ff.ff_profile_read(ctx)
    ff.ff_profile(ctx, False)
    max_ms = max_over_ranks(total_ms, "cuda")
    split = batch is not None and args.split

    def job_rate(max_seconds):
        # a shared batch counts its particles once; replicas and per-rank batches count every rank
        return n_job * K / max_seconds if split else whole_job_rate(n, K, world, max_seconds)

    value = job_rate(max_ms / 1e3)
    energy = ff.ff_energy(ctx)
    systems_done = None
    if batch is not None:
        # the only exchange of a batched job: per-system moment sums (4 doubles a system)
        # gathered once, after the timed region
        sums, _ = ff.ff_system_moments(ctx)
        if world > 1 and split:
            systems_done = len(shard.gather_system_values(sums, mine, len(full["sizes"])))
        elif world > 1:
            every = [None] * world
            torch.distributed.all_gather_object(every, sums.tolist())
            systems_done = sum(len(a) for a in every)
        else:
            systems_done = len(sums)
    # interaction counts of the final state, from one counted evaluation (the timed steps
    # move particles by ~1e-4 diameters, so the per-launch work is the same to < 0.1 %)
    xs = ff.ff_get_particles(ctx, dtype=np.float32, device_like=pos_d)
    ctxc = create(params(count_interactions=1))
    ff.ff_set_particles(ctxc, xs[0], xs[1], xs[2], xs[3])
    hc = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    ff.ff_dipolar_field(ctxc, ff.FF_ALGO_BH, args.theta, True, hc, torch.empty_like(hc))
    info = ff.ff_tree_info(ctxc)
    del ctxc, xs, hc

    # roofline of the dominant kernel (the traversal), from this run's events, against the
    # FP32 peak measured on this GPU right after the timed region
    field_ms = prof["ms"]["field"] / max(prof["calls"]["field"], 1)
    flops = info["interactions"] * FLOPS_PER_INTERACTION
    peaks = simt_peaks(dev)
    peak = peaks["fp32_tflops"]
    achieved = flops / (field_ms / 1e3) / 1e12
    traffic = traffic_for(os.path.join(ROOT, "paper_1212_2934_gb300", "csrc", "k_field.cu"), n,
                          args.workload, args.theta, args.leaf_max, args.schedule)
    stages = {k: v / max(prof["calls"][k], 1) for k, v in prof["ms"].items() if prof["calls"][k]}

    extras = {}
    e2e = None
    if not args.no_extras and args.workload == "chains":
        # ---- the same chains stepped with FP64 cell sums (mixed) and entirely in FP64
        for prec, kk in (("mixed", K), ("f64", max(3, K // 10))):
            c = ff.ff_create(params(precision=prec, count_interactions=0))
            ff.ff_set_particles(c, pos_d.double() if prec == "f64" else pos_d,
                                u_d.double() if prec == "f64" else u_d)
            for _ in range(W):
                ff.ff_step(c, 1)
                flush.zero_()
            barrier()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(kk)]
            for a, b in ev:
                a.record(stream)
                ff.ff_step(c, 1)
                b.record(stream)
                flush.zero_()
            barrier()
            ms = sum(a.elapsed_time(b) for a, b in ev) / kk
            extras["bh_" + ("fp64" if prec == "f64" else prec)] = {
                "particle_steps_per_s": n / (ms / 1e3), "ms_per_step": ms, "steps": kk}
            del c
        extras["bh_fp32"] = {"particle_steps_per_s": value / world, "ms_per_step": max_ms / K,
                             "interactions_per_particle": info["interactions"] / n,
                             "cells": info["ncells"]}
        extras["error_note"] = ("errors of each path against the FP64 all-pairs oracle on a "
                                "16,384-particle subsample are measured by the chain precision "
                                "test, not here")
    if not args.no_extras and args.workload == "phi05":
        # ---- FP64 Barnes-Hut path
        ctx64 = ff.ff_create(params(precision="f64", count_interactions=0))
        ff.ff_set_particles(ctx64, pos_d.double(), u_d.double())
        ff.ff_step(ctx64, 1)
        flush.zero_()
        barrier()
        k64 = 3
        e64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(k64)]
        for k in range(k64):
            e64[k][0].record(stream)
            ff.ff_step(ctx64, 1)
            e64[k][1].record(stream)
            flush.zero_()
        barrier()
        ms64 = sum(a.elapsed_time(b) for a, b in e64) / k64
        # the FP64 traversal's own launch time and interaction count, for its roofline
        ff.ff_profile(ctx64, True)
        for _ in range(2):
            ff.ff_step(ctx64, 1)
            flush.zero_()
        prof64 = ff.ff_profile_read(ctx64)
        del ctx64
        field64_ms = prof64["ms"]["field"] / max(prof64["calls"]["field"], 1)
        ctxc64 = ff.ff_create(params(precision="f64", count_interactions=1))
        ff.ff_set_particles(ctxc64, pos_d.double(), u_d.double())
        h64 = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        ff.ff_dipolar_field(ctxc64, ff.FF_ALGO_BH, args.theta, True, h64, torch.empty_like(h64))
        info64 = ff.ff_tree_info(ctxc64)
        del ctxc64, h64
        ach64 = info64["interactions"] * FLOPS_PER_INTERACTION / (field64_ms / 1e3) / 1e12
        # ---- FP32 Barnes-Hut with up to 8 particles per leaf (same theta; near field exact
        # inside leaves) -- a tuning comparison, not the paper's one-particle leaves
        ctx8 = ff.ff_create(params(leaf_max=8, count_interactions=0))
        ff.ff_set_particles(ctx8, pos_d, u_d)
        ff.ff_step(ctx8, 2)
        barrier()
        e8 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(10)]
        for a, b in e8:
            a.record(stream)
            ff.ff_step(ctx8, 1)
            b.record(stream)
            flush.zero_()
        barrier()
        ms8 = sum(a.elapsed_time(b) for a, b in e8) / len(e8)
        del ctx8
        # ---- GPU all-pairs step (FP32)
        ctxap = ff.ff_create(params(algo="ap", count_interactions=0))
        ff.ff_set_particles(ctxap, pos_d, u_d)
        ff.ff_profile(ctxap, True)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        ff.ff_step(ctxap, 1)
        a1.record(stream)
        barrier()
        ms_ap = a0.elapsed_time(a1)
        prof_ap = ff.ff_profile_read(ctxap)
        del ctxap
        ap_field_ms = prof_ap["ms"]["field"]
        # ---- accuracy against the all-pairs field (same GPU, FP32) at theta 0.5 and 0.7,
        # with the paper's pseudo-particles and with the dipole-position (quadrupole) terms
        hap = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        fap = torch.empty_like(hap)
        ctxr = ff.ff_create(params(count_interactions=0))
        ff.ff_set_particles(ctxr, pos_d, u_d)
        ff.ff_dipolar_field(ctxr, ff.FF_ALGO_AP, 0.0, False, hap, fap)
        del ctxr
        href = hap.double()
        hn2 = (href ** 2).sum(dim=1).mean()
        hb = torch.empty_like(hap)
        fb = torch.empty_like(hap)
        accuracy = {}
        for q in (0, 1):
            ctxq = ff.ff_create(params(count_interactions=0, quadrupole=q))
            ff.ff_set_particles(ctxq, pos_d, u_d)
            for th in (0.3, 0.5, 0.7):
                ff.ff_dipolar_field(ctxq, ff.FF_ALGO_BH, th, False, hb, fb)
                q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                q0.record(stream)
                ff.ff_dipolar_field(ctxq, ff.FF_ALGO_BH, th, False, hb, fb)
                q1.record(stream)
                barrier()
                err = float(torch.sqrt(((hb.double() - href) ** 2).sum(dim=1).mean() / hn2))
                accuracy["%s_theta%.1f" % ("quad" if q else "mono", th)] = {
                    "field_eval_ms": q0.elapsed_time(q1), "h_rms_rel_err_vs_allpairs": err}
            del ctxq
        extras_accuracy = accuracy
        extras = {
            "bh_fp32": {"particle_steps_per_s": value / world, "ms_per_step": max_ms / K,
                        "interactions_per_s": info["interactions"] / (field_ms / 1e3),
                        "interactions_per_particle": info["interactions"] / n,
                        "accepted_cells_per_particle": info["accepted"] / n,
                        "exact_pairs_per_particle": info["pairs"] / n,
                        "opened_cells_per_particle": info["opened"] / n,
                        "cells": info["ncells"]},
            "ap_fp32": {"particle_steps_per_s": n / (ms_ap / 1e3), "ms_per_step": ms_ap,
                        "pair_interactions_per_s": n * (n - 1) / (ap_field_ms / 1e3),
                        "field_tflops": n * (n - 1) * FLOPS_PER_INTERACTION / (ap_field_ms / 1e3) / 1e12},
            "bh_fp64": {"particle_steps_per_s": n / (ms64 / 1e3), "ms_per_step": ms64,
                        "roofline": {"bound": "alu", "kernel": "k_bh<double> (FP64 traversal)",
                                     "achieved": ach64, "peak": peaks["fp64_tflops"],
                                     "unit": "TFLOP/s", "frac": ach64 / peaks["fp64_tflops"],
                                     "avg_launch_ms": field64_ms,
                                     "algorithmic_flops_per_launch":
                                         info64["interactions"] * FLOPS_PER_INTERACTION,
                                     "peak_note": peak_note(peaks, "fp64")}},
            "bh_fp32_leaf8": {"particle_steps_per_s": n / (ms8 / 1e3), "ms_per_step": ms8,
                              "note": "leaf_max = 8 (the paper's leaves hold one particle)"},
            "accuracy_vs_allpairs": dict(extras_accuracy, note=(
                "field evaluation (keys, sort, build, aggregation, traversal) and RMS relative "
                "error of h against the GPU all-pairs field; quad = with each accepted cell's "
                "dipole-position term (an option beyond the paper's pseudo-particles)")),
            "speedup_bh_fp32_over_ap": ms_ap / (max_ms / K),
            "speedup_bh_fp32_over_fp64": ms64 / (max_ms / K),
        }
    if not args.no_extras:
        # ---- end to end through the C interface with pinned host buffers
        host = [torch.empty((n, 3), dtype=torch.float32, pin_memory=True) for _ in range(4)]
        host[0].copy_(torch.from_numpy(pos.astype(np.float32)))
        host[1].copy_(torch.from_numpy(u.astype(np.float32)))
        host[2].zero_()
        host[3].zero_()
        hn = [h.numpy() for h in host]
        outs = [torch.empty((n, 3), dtype=torch.float32, pin_memory=True).numpy() for _ in range(4)]
        ctxe = create(params(count_interactions=0))
        lib = ff.lib()
        import ctypes

        ptr = lambda a: ctypes.c_void_p(a.ctypes.data)

        bufs = [hn, outs]

        def e2e_step():
            src, dst = bufs
            ff._check(ctxe.handle, lib.ff_set_particles(ctxe.handle, *[ptr(h) for h in src],
                                                        ff.FF_DTYPE_F32, ff.FF_HOST))
            ff._check(ctxe.handle, lib.ff_step(ctxe.handle, 1))
            ff._check(ctxe.handle, lib.ff_get_particles(ctxe.handle, *[ptr(o) for o in dst],
                                                        ff.FF_DTYPE_F32, ff.FF_HOST))
            bufs.reverse()  # the next step starts from the state just read back

        for _ in range(max(W, 1)):
            e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(K):
            e2e_step()
        barrier()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": job_rate(max_over_ranks(e2e_s, "cuda")), "unit": UNIT,
               "h2d_bytes_per_step": 4 * n * 3 * 4, "d2h_bytes_per_step": 4 * n * 3 * 4,
               "note": "ff_set_particles + ff_step + ff_get_particles on pinned host float32 "
                       "arrays (positions, moments, velocities, angular velocities), wall clock"}
        del ctxe

    cfg = config_dict(args, side)
    cfg["traverse_tuning"] = tuning
    metric = METRIC
    if args.workload == "chains":
        metric = CHAINS_METRIC
        cfg = chains_config(args, n, side, world)
        cfg["traverse_group"] = args.group
        cfg["traverse_tuning"] = tuning
    if batch is not None:
        metric = BATCHED_METRIC
        cfg = batched_config(args, n_job if args.split else n, world)
        cfg["systems_all_ranks"] = systems_done
        cfg["traverse_group"] = args.group
        cfg["traverse_tuning"] = tuning
    line = {
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": max_ms / K, "higher_is_better": True,
        "scaling": "strong" if split else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_bh (Barnes-Hut traversal)",
                     "peak_note": peak_note(peaks, "fp32"),
                     "peaks_measured": peaks,
                     "algorithmic_flops_per_launch": flops,
                     "avg_launch_ms": field_ms,
                     "timing": "CUDA events around the traversal launch on the library's stream, "
                               "%d steps of a separate eager pass right after the timed region"
                               % kprof},
        "stage_ms_per_step": stages,
        "gpu_launches": int(launches),
        "gpu_launch_note": "kernels of this library launched in the timed region (each step is "
                           "one CUDA graph of %d kernels)" % (launches // max(K, 1)),
        "clocks": clk,
        "paths": extras,
        "observables_last": {"m_z": float(energy["m"][2]), "e_dip_per_particle": energy["e_dip"] / n},
    }
    if e2e is not None:
        line["e2e"] = e2e
    if rank == 0 and world == 1 and not args.no_extras and batch is None:
        line["cpu_baseline"] = cpu_baselines(pos, u, args.theta, args.leaf_max, side,
                                             262144 if args.workload == "phi05" else 131072)
    elif rank == 0 and world == 1 and not args.no_extras:
        rate, cpu_s, threads, nsys_s, m = cpu_batched_sample(batch, args.theta, args.leaf_max)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": "one full step (tree, traversal, integration) of every "
                                          "8th system: %d systems, %d particles (%.1f s of CPU "
                                          "work)" % (nsys_s, m, cpu_s)}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


GRAD_METRIC = ("particle-gradients/s: dE_dip/dpos and dE_dip/du of the Barnes-Hut energy "
               "(decisions frozen) at N=262,144, phi 0.05, theta=0.5, FP32")
GRAD_N = 262144


def run_grad(args):
    """Times ff_energy_grad (energy and its gradient w.r.t. every position and moment) on one
    GPU; each repetition re-sorts, rebuilds and traverses the current state."""
    import torch

    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    import __graft_entry__

    __graft_entry__.build()
    from paper_1212_2934_gb300 import ff

    K, W = args.steps, args.warmup
    pos, u, side = workload(GRAD_N)
    n = GRAD_N
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    p = ff.ff_params_default(n=n, precision="f32", theta=args.theta, leaf_max=args.leaf_max,
                             device=dev, stream=stream.cuda_stream)
    ctx = ff.ff_create(p)
    pos_d = torch.tensor(pos, dtype=torch.float32, device="cuda")
    u_d = torch.tensor(u, dtype=torch.float32, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ff.ff_set_particles(ctx, pos_d, u_d)
    gp = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    gu = torch.empty_like(gp)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def grad_once():
        e = ff.C.c_double()
        ff._check(ctx.handle, ff.lib().ff_energy_grad(
            ctx.handle, ff.FF_ALGO_BH, float(args.theta), ff.C.byref(e),
            ff.C.c_void_p(gp.data_ptr()), ff.C.c_void_p(gu.data_ptr()), ff.FF_DTYPE_F32,
            ff.FF_DEVICE))
        return e.value

    for _ in range(W):
        grad_once()
        flush.zero_()
    barrier()
    clocks = Clocks(dev)
    clocks.start()
    launches0 = ff.ff_profile_read(ctx)["launches"]
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    clocks.mark_start()
    for a, b in evs:
        a.record(stream)
        e = grad_once()
        b.record(stream)
        flush.zero_()
    barrier()
    clocks.mark_end()
    clk = clocks.stop()
    launches = ff.ff_profile_read(ctx)["launches"] - launches0
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    max_ms = max_over_ranks(total_ms, "cuda")
    value = whole_job_rate(n, K, world, max_ms / 1e3)
    # the forward field alone on the same state, for the cost ratio
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hb = torch.empty_like(gp)
    fb = torch.empty_like(gp)
    f0.record(stream)
    for _ in range(K):
        ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, args.theta, False, hb, fb)
    f1.record(stream)
    barrier()
    field_ms = f0.elapsed_time(f1) / K
    # roofline of the largest kernel, the counting walk that also writes the source lists
    # (k_bh_rec): its launch time from the library's stage events over K more gradients,
    # its work from the interaction counts of the same walk
    ff.ff_profile(ctx, True)
    for _ in range(K):
        grad_once()
        flush.zero_()
    barrier()
    prof = ff.ff_profile_read(ctx)
    ff.ff_profile(ctx, False)
    rec_ms = prof["ms"]["field"] / max(prof["calls"]["field"], 1)
    nacc, npair, _ = ff.ff_get_counts(ctx)
    inter = float(np.sum(nacc, dtype=np.int64) + np.sum(npair, dtype=np.int64))
    peaks = simt_peaks(dev)
    rec_flops = inter * FLOPS_PER_INTERACTION
    achieved = rec_flops / (rec_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peaks["fp32_tflops"],
                "unit": "TFLOP/s", "frac": achieved / peaks["fp32_tflops"],
                "traffic": traffic_for(os.path.join(ROOT, "paper_1212_2934_gb300", "csrc",
                                                    "k_field.cu"), n, "grad", args.theta,
                                       args.leaf_max, 0, kernel="k_bh_rec"),
                "kernel": "k_bh_rec (counting walk writing every particle's source list)",
                "peak_note": peak_note(peaks, "fp32"), "peaks_measured": peaks,
                "algorithmic_flops_per_launch": rec_flops,
                "list_bytes_per_launch": 4.0 * inter,
                "avg_launch_ms": rec_ms,
                "timing": "CUDA events around the walk's launch on the library's stream, %d "
                          "gradients right after the timed region" % K}
    # end to end: host state in, gradients out to pinned host memory
    host_p = torch.from_numpy(pos.astype(np.float32)).pin_memory().numpy()
    host_u = torch.from_numpy(u.astype(np.float32)).pin_memory().numpy()
    out_p = torch.empty((n, 3), dtype=torch.float32).pin_memory().numpy()
    out_u = torch.empty((n, 3), dtype=torch.float32).pin_memory().numpy()
    ptr = lambda a: ff.C.c_void_p(a.ctypes.data)

    def e2e_once():
        ff._check(ctx.handle, ff.lib().ff_set_particles(ctx.handle, ptr(host_p), ptr(host_u), None,
                                                        None, ff.FF_DTYPE_F32, ff.FF_HOST))
        e = ff.C.c_double()
        ff._check(ctx.handle, ff.lib().ff_energy_grad(ctx.handle, ff.FF_ALGO_BH, float(args.theta),
                                                      ff.C.byref(e), ptr(out_p), ptr(out_u),
                                                      ff.FF_DTYPE_F32, ff.FF_HOST))

    e2e_once()
    barrier()
    t0 = time.perf_counter()
    for _ in range(K):
        e2e_once()
    barrier()
    e2e_s = time.perf_counter() - t0
    # d<M_z>/dh_ext through a 200-step unroll saved every 20 steps, next to the same 200
    # steps without the derivative (a fresh context each, from the same state)
    sens = None
    if not args.no_extras:
        def fresh():
            c2 = ff.ff_create(ff.ff_params_default(n=n, precision="f32", theta=args.theta,
                                                   leaf_max=args.leaf_max, device=dev,
                                                   stream=stream.cuda_stream, h_ext=(0, 0, 1.0)))
            ff.ff_set_particles(c2, pos_d, u_d)
            return c2

        c2 = fresh()
        ff.ff_step(c2, 3)
        barrier()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c2 = fresh()
        s0.record(stream)
        ff.ff_step(c2, 200)
        s1.record(stream)
        barrier()
        fwd_ms = s0.elapsed_time(s1)
        c2 = fresh()
        barrier()
        t0 = time.perf_counter()
        mzv, gv = ff.ff_mz_sensitivity(c2, 200, 20)
        barrier()
        sens_ms = 1e3 * (time.perf_counter() - t0)
        sens = {"steps": 200, "checkpoint_every": 20, "ms": sens_ms, "forward_200_steps_ms": fwd_ms,
                "ratio_to_forward": sens_ms / fwd_ms, "mz": mzv, "dmz_dh": list(gv),
                "note": "wall clock of ff_mz_sensitivity (forward with checkpoints, segment "
                        "recomputation, adjoint of every step) vs CUDA-event time of 200 plain steps"}
        del c2
    line = {
        "metric": GRAD_METRIC, "value": value, "unit": "particle-gradients/s", "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": max_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "gradient of E_dip = -1/2 sum u.h (Barnes-Hut, decisions frozen) "
                               "w.r.t. all positions and moments; dipoles at volume fraction "
                               "0.05 (hard core 1.0, RSA), isotropic moments",
                   "n": n, "box_side": round(side, 4), "theta": args.theta,
                   "leaf_max": args.leaf_max, "precision": "fp32",
                   "l2": "flushed between timed evaluations (256 MB write outside the events)",
                   "parallelism": "replicas" if world > 1 else "single-gpu"},
        "roofline": roofline,
        "gpu_launches": int(launches),
        "clocks": clk,
        "paths": {"field_only_ms": field_ms, "gradient_over_field": (max_ms / K) / field_ms,
                  "energy": e, "mz_sensitivity": sens},
        "e2e": {"value": whole_job_rate(n, K, world, max_over_ranks(e2e_s, "cuda")),
                "unit": "particle-gradients/s", "h2d_bytes_per_step": 2 * n * 3 * 4,
                "d2h_bytes_per_step": 2 * n * 3 * 4,
                "note": "ff_set_particles + ff_energy_grad on pinned host float32 arrays, "
                        "wall clock"},
    }
    if rank == 0 and world == 1 and not args.no_extras:
        import oracle

        p64 = pos.astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        oracle.bh_energy_grad(p64, u.astype(np.float64), args.theta, args.leaf_max, "f32",
                              lj_eps=1.0, tree_centres=True)
        cpu_s = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": n / cpu_s, "unit": "particle-gradients/s",
                                "cores": oracle.get_threads(), "kind": "oracle",
                                "sample": "one full gradient of all %d particles (%.1f s)"
                                          % (n, cpu_s)}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "grad":
        return run_grad(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
