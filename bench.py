#!/usr/bin/env python3
"""Benchmark: FP+BP voxel-samples/s on the 512^3 clinical cone-beam workload.

Workload (synthetic, seeded): 512^3 FP32 volume at 0.5 mm holding a
40-ellipsoid phantom, 720 angles over 2 pi, 768 x 1024 detector at 0.4 mm,
DSO 1000 mm, DSD 1536 mm, measured data = Siddon projection of the phantom
with Poisson noise at I0 = 1e5.

One step = one pass over every operation of the hot path, each through the
C ABI:
  * tg_cgls, one iteration from x0 = 0 (two interpolated forward
    projections, two matched backprojections, fused FP64 inner products and
    vector updates),
  * tg_ossart, one iteration from x0 = 0 with blocks of 20 angles (the SIRT
    weights W = 1/(A 1) and V_s = 1/(A_s^T 1), then one sweep over the 36
    blocks: a projection and a backprojection each),
  * tg_forward with the Siddon projector,
  * tg_fdk (cosine weight + Ram-Lak filter + FDK backprojection).
Units: forward samples (trilinear samples taken, or Siddon voxel segments)
plus backprojected voxel-angle pairs; value = units per step / step time.

Timing: W untimed warm-up steps, then K steps between a barrier and
torch.cuda.synchronize(), on CUDA events of the launching stream; max over
ranks.  Inputs (0.5 GB volume, 2.3 GB projections) exceed the 129 MB L2, so
no flush is needed between steps.  Multi-GPU runs are independent replicas
(the operators shard, but one GPU holds the whole problem; no collective).
``--impl reference`` times the CPU FP64 oracle on a bounded sample of the
same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "FP+BP voxel-samples/s at 512^3 (% roofline); s to PSNR: learned vs CGLS"
UNIT = "voxel-samples/s"
WORKLOAD = "512^3 FP32 volume (0.5 mm), 720 angles over 2pi, 768x1024 detector (0.4 mm), 40-ellipsoid phantom"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


CASES = {
    # name: (workload text, geometry factory, ellipsoids)
    "clinical": (WORKLOAD, "config_clinical", 40),
    # the same scan at half the resolution (profiling captures: inputs still
    # exceed L2, one launch runs well under a second)
    "medium": ("256^3 FP32 volume (1 mm), 360 angles over 2pi, 384x512 detector (0.8 mm), 20-ellipsoid phantom",
               None, 20),
}


def bench_config(case, world):
    """The `config` object both arms print for a workload."""
    return {"workload": CASES[case][0], "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs (2.8 GB) exceed L2 (129 MB); no flush" if case == "clinical"
            else "inputs (0.35 GB) exceed L2 (129 MB); no flush",
            "step": "tg_cgls 1 iteration + tg_ossart 1 iteration (blocks of 20) + tg_forward(siddon) + tg_fdk"}


def make_inputs(case="clinical", seed=1):
    from paper_2412_10129_gb300 import inputs
    if case == "medium":
        g = inputs.circular_geometry((256, 256, 256), (1.0,) * 3, (512, 384), (0.8, 0.8), 360, 1000.0, 1536.0)
    else:
        g = inputs.config_clinical()
    x = inputs.ellipsoid_phantom(g, CASES[case][2], seed=seed)
    return g, x


def dist_setup(n_gpus, backend=None):
    """Rank, world size and local rank from the launcher's environment; for
    N > 1 one process per GPU joins a process group (NCCL on GPUs, gloo for
    host-only runs).  The replicas exchange only the barrier and the maximum
    of their timings: the work itself has no collective."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank, steps, secs_max, world):
    """Whole-job throughput of `world` replicas: every rank does
    `units_per_rank` per step; the job takes the slowest rank's time."""
    return world * units_per_rank * steps / secs_max


# ---------------------------------------------------------------------------
# CPU FP64 oracle on a bounded sample of the workload.
# ---------------------------------------------------------------------------

# The bounded oracle sample both CPU legs time: the interpolated FP of every
# pixel of REF_FP_ANGLES angles and the matched BP (gather form) of
# REF_BP_VOXELS random voxels over all angles.
REF_FP_ANGLES = 1
REF_BP_VOXELS = 32


def oracle_sample(g, x, y, n_fp_angles=REF_FP_ANGLES, n_bp_voxels=REF_BP_VOXELS, seed=0):
    """Time the oracle: interpolated FP of every pixel of `n_fp_angles`
    angles, matched BP (gather form) of `n_bp_voxels` voxels over all angles.
    Units are counted on the host in FP64 (no GPU library is loaded).
    Returns (units, seconds, description)."""
    import oracle
    rng = np.random.default_rng(seed)
    sub = g.subset(np.linspace(0, g.nAngles - 1, n_fp_angles).astype(int))
    rays = np.stack(np.meshgrid(np.arange(sub.nAngles), np.arange(g.nDetector[1]), np.arange(g.nDetector[0]),
                                indexing="ij"), -1).reshape(-1, 3)
    vox = np.stack([rng.integers(0, n, n_bp_voxels) for n in g.nVoxel], 1)
    t0 = time.perf_counter()
    oracle.forward_rays(sub, x, rays, "interp")
    t1 = time.perf_counter()
    oracle.backproject_voxels(g, y, vox, "matched")
    t2 = time.perf_counter()
    fp_units = _count_samples_host(sub)
    units = fp_units + n_bp_voxels * g.nAngles
    desc = (f"oracle interpolated FP of all {len(rays)} rays of {n_fp_angles} angle(s) ({fp_units} samples) + "
            f"matched BP of {n_bp_voxels} random voxels x {g.nAngles} angles")
    return units, t2 - t0, desc


def cpu_baseline_line(g, x, y, min_seconds=10.0):
    """cpu_baseline: the oracle sample repeated until at least `min_seconds`
    of host time have been spent."""
    units = 0
    secs = 0.0
    reps = 0
    desc = ""
    while secs < min_seconds or reps == 0:
        u, t, desc = oracle_sample(g, x, y)
        units += u
        secs += t
        reps += 1
    return {"value": units / secs, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{reps} x ({desc})"}


def _gpu_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except ImportError:
        return False


def _count_samples_host(g):
    """Samples of the interpolated projector, counted in FP64 on the host."""
    import oracle
    f = oracle.frames(g)
    delta = g.accuracy * min(g.dVoxel)
    h = 0.5 * np.asarray(g.nVoxel) * np.asarray(g.dVoxel)
    total = 0
    for a in range(g.nAngles):
        P = oracle.pixel_centres(g, a).reshape(-1, 3)
        S = f["S"][a]
        d = P - S
        L = np.linalg.norm(d, axis=1)
        dh = d / L[:, None]
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = (-h[None] - S[None]) / dh
            tb = (h[None] - S[None]) / dh
        lo = np.nanmax(np.minimum(ta, tb), axis=1).clip(min=0)
        hi = np.minimum(np.nanmin(np.maximum(ta, tb), axis=1), L)
        n = np.floor(hi / delta) - np.ceil(lo / delta) + 1
        total += int(np.sum(np.where(hi >= lo, np.maximum(n, 0), 0)))
    return total


def cpu_cores():
    try:
        import oracle
        return oracle.num_threads()
    except Exception:
        return os.cpu_count()


# ---------------------------------------------------------------------------
# Reference arm: the oracle, timed on the host cores.
# ---------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), 0
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    from paper_2412_10129_gb300 import inputs
    g, x = make_inputs()
    y = inputs.random_projections(g.subset(np.arange(g.nAngles)), seed=3)
    for _ in range(args.warmup):
        oracle_sample(g, x, y)
    units = 0
    secs = 0.0
    desc = ""
    for _ in range(args.steps):
        u, s, desc = oracle_sample(g, x, y)
        units += u
        secs += s
    value = units / secs
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": bench_config("clinical", world), "sample_per_step": desc,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm.
# ---------------------------------------------------------------------------

def run_gpu(args):
    import torch

    from paper_2412_10129_gb300 import build, inputs, tg
    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    build.build()
    tg.load()
    dev = torch.device("cuda", local)
    g, x_np = make_inputs(args.case)
    b_np = inputs.poisson_noise(_siddon_gpu(g, x_np, dev), 1e5, seed=2)
    vol_elems = int(np.prod(g.vol_shape))
    proj_elems = int(np.prod(g.proj_shape))
    b = torch.from_numpy(b_np).to(dev)
    x = torch.from_numpy(x_np).to(dev)
    xw = torch.zeros(g.vol_shape, device=dev)
    p_sid = torch.empty(g.proj_shape, device=dev)
    v_fdk = torch.empty(g.vol_shape, device=dev)
    stream = torch.cuda.current_stream(dev)

    s_interp = tg.count_samples(g, "interp")
    s_siddon = tg.count_samples(g, "siddon")
    bp_pairs = vol_elems * g.nAngles
    units_cgls = 2 * s_interp + 2 * bp_pairs      # initial s = A^T r, then q = A p and s = A^T r
    units_ossart = 2 * s_interp + 2 * bp_pairs    # W = 1/(A 1), V_s = 1/(A_s^T 1), one sweep
    units_step = units_cgls + units_ossart + s_siddon + bp_pairs
    xo = torch.zeros(g.vol_shape, device=dev)

    def step():
        xw.zero_()
        tg.cgls(g, b, 1, x0=xw)
        xo.zero_()
        tg.ossart(g, b, 1, blocksize=20, x0=xo)
        tg.forward(g, x, "siddon", out=p_sid)
        tg.fdk(g, b, out=v_fdk)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    # per-kernel times (outside the headline): one launch each
    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    p_tmp = torch.empty(g.proj_shape, device=dev)
    v_tmp = torch.empty(g.vol_shape, device=dev)
    t_fp = timed(lambda: tg.forward(g, x, "interp", out=p_tmp))
    t_bp = timed(lambda: tg.backproject(g, b, "matched", out=v_tmp))
    t_sid = timed(lambda: tg.forward(g, x, "siddon", out=p_tmp))
    t_bpf = timed(lambda: tg.backproject(g, b, "fdk", out=v_tmp))
    t_fdk = timed(lambda: tg.fdk(g, b, out=v_tmp))
    del p_tmp, v_tmp
    torch.cuda.empty_cache()

    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)
    n0 = tg.launch_count()
    tg.kernel_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    e1.synchronize()
    launches = tg.launch_count() - n0
    kt = tg.kernel_timing_read()
    tg.kernel_timing(False)
    barrier(world)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    secs = max_over_ranks(e0.elapsed_time(e1) * 1e-3, world)
    value = replica_value(units_step, args.steps, secs, world)

    # end to end: the same step through the C ABI with pinned host buffers,
    # host<->device copies inside the timed region
    bh = torch.from_numpy(b_np).pin_memory()
    xh = torch.from_numpy(x_np).pin_memory()
    xwh = torch.zeros(g.vol_shape).pin_memory()
    xoh = torch.zeros(g.vol_shape).pin_memory()
    sidh = torch.empty(g.proj_shape).pin_memory()
    fdkh = torch.empty(g.vol_shape).pin_memory()
    # cgls (b, x0), ossart (b, x0), siddon (x), fdk (b)
    h2d = 2 * 4 * (proj_elems + vol_elems) + 4 * vol_elems + 4 * proj_elems
    d2h = 2 * 4 * vol_elems + 4 * proj_elems + 4 * vol_elems                # cgls x, ossart x, siddon proj, fdk vol

    def step_host():
        xwh.zero_()
        tg.cgls(g, bh, 1, x0=xwh)
        xoh.zero_()
        tg.ossart(g, bh, 1, blocksize=20, x0=xoh)
        tg.forward(g, xh, "siddon", out=sidh)
        tg.fdk(g, bh, out=fdkh)

    step_host()
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_host()
    torch.cuda.synchronize(dev)
    secs_e2e = max_over_ranks(time.perf_counter() - t0, world)
    e2e = replica_value(units_step, args.steps, secs_e2e, world)
    del bh, xh, xwh, xoh, sidh, fdkh

    # device time of each kernel class inside the timed region (tg_kernel_timing)
    # and the units those launches processed: per step, the interpolated
    # projector runs 4 full projections (CGLS: r0 and q; OS-SART: W and one
    # sweep), the fixed-point transpose 2 (CGLS) and the split transpose 2
    # (OS-SART: V_s and one sweep)
    rates = _probe_rates()
    per_step_samples = {"fp_interp": 4 * s_interp, "bp_matched": 2 * s_interp, "bp_matched_split": 2 * s_interp}
    roofs = {}
    for name, fn in (("fp_interp", roofline_fp), ("bp_matched", roofline_bp), ("bp_matched_split", roofline_bp_split)):
        ms, n = kt[name]
        if n:
            roofs[name] = fn(per_step_samples[name] * args.steps, ms * 1e-3, rates)
            roofs[name]["launches_in_timed_region"] = n
            # DRAM bytes per launch (ncu per-sample figure x this launch's samples)
            roofs[name]["traffic"] = DRAM_BYTES_PER_SAMPLE[name] * per_step_samples[name] * args.steps / n
            roofs[name]["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum per sample on the "
                                             "256^3 / 360-view case, scaled by the samples per launch")
    dominant = max(roofs, key=lambda k: kt[k][0])
    roof = dict(roofs[dominant])
    t_fp_live = kt["fp_interp"][0] * 1e-3 / (4 * args.steps)
    t_bp_live = kt["bp_matched"][0] * 1e-3 / (2 * args.steps)
    both = (s_interp / roofs["fp_interp"]["peak_samples_per_s"] + s_interp / roofs["bp_matched"]["peak_samples_per_s"])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": bench_config(args.case, world), "units_per_step": units_step,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
            "roofline": roof,
            "rooflines": roofs,
            "roofline_fp_bp": {"kernels": "k_fp_interp_tex + k_bp_mx fixed point (one A and one A^T)",
                               "achieved_s": t_fp_live + t_bp_live, "roofline_s": both,
                               "frac": both / (t_fp_live + t_bp_live)},
            "kernels_in_timed_region": {k: {"launches": n, "total_ms": ms, "share_of_step": ms * 1e-3 / secs,
                                            "avg_ms": (ms / n if n else None)} for k, (ms, n) in kt.items()},
            "kernels_s": {"fp_interp": t_fp, "bp_matched": t_bp, "fp_siddon": t_sid, "bp_fdk": t_bpf,
                          "fdk": t_fdk},
            "rates": {"fp_interp_samples_per_s": s_interp / t_fp_live, "bp_matched_samples_per_s": s_interp / t_bp_live,
                      "bp_matched_pairs_per_s": bp_pairs / t_bp_live,
                      "fp_siddon_segments_per_s": s_siddon / t_sid, "bp_fdk_pairs_per_s": bp_pairs / t_bpf,
                      "fp_plus_bp_matched": (s_interp + bp_pairs) / (t_fp_live + t_bp_live)},
            "probe": rates}
    if rank == 0 and world == 1 and args.learned_pretrain + args.learned_finetune > 0:
        # the second half of the metric: seconds to PSNR, learned vs CGLS, after
        # a shortened training pass (its budget is stated in the object)
        del x, xw, xo, p_sid, v_fdk, b
        torch.cuda.empty_cache()
        line["learned"] = learned_measure(args.learned_pretrain, args.learned_finetune, 1, ragged=False)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_line(g, x_np, b_np)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def _probe_rates():
    """Gather and scatter ceilings measured on this device now (libtgprobe)."""
    from paper_2412_10129_gb300 import probe
    return {"smem_atomic_conflict_free": probe.smem_atomic(False)["atomics_per_s"],
            "smem_atomic_random": probe.smem_atomic(True)["atomics_per_s"],
            "tex_gather_coherent_l1": probe.tex_gather(64, 64, 4, True)["gathers_per_s"],
            "tex_gather_coherent_l2": probe.tex_gather(512, 512, 64, True)["gathers_per_s"],
            "l2_sector_gather_gbs": probe.sector_gather(64 << 20)["gbs"]}


# DRAM bytes (read + write) per interpolated sample, from one ncu capture of
# each kernel as built now on the 256^3 / 360-view case (3.348e10 samples;
# profiles/k_fp_interp_tex_medium_256.md, k_bp_mx_medium_256.md,
# k_bp_mx_split_medium_256.md), scaled to a launch by its samples.  The
# projector's traffic is the volume and the projections once; the
# transposes' is dominated by the rays' set-up table, read by every brick a
# ray passes near, which grows with the samples (rays x bricks per ray).
DRAM_BYTES_PER_SAMPLE = {"fp_interp": (68.581e6 + 236.597e6) / 3.348e10,
                         "bp_matched": (20.517e9 + 1.146e9) / 3.348e10,
                         "bp_matched_split": (20.865e9 + 1.185e9) / 3.348e10}


def roofline_bp(samples, t, rates):
    """k_bp_matched: every sample of the interpolated projector scatters eight
    32-bit fixed-point contributions into shared memory with integer atomic
    adds, so its ceiling is the SM's shared-memory atomic rate / 8, measured
    with conflict-free addresses (one 32-lane wavefront per clock)."""
    peak = rates["smem_atomic_conflict_free"] / 8.0
    achieved = samples / t
    return {"bound": "smem_atomic", "kernel": "k_bp_mx (fixed point)", "achieved": achieved / 1e9, "peak": peak / 1e9,
            "unit": "Gsamples/s", "frac": achieved / peak, "traffic": None,
            "peak_samples_per_s": peak,
            "peak_source": "measured conflict-free shared-memory 32-bit atomic adds (libtgprobe tgp_smem_atomic) / "
                           "8 atomics per sample",
            "random_scatter_peak": rates["smem_atomic_random"] / 8.0 / 1e9,
            "unit_of_work": "one trilinear sample of the interpolated projector (8 contributions)"}


def roofline_bp_split(samples, t, rates):
    """k_bp_mx with split accumulation (SIRT / OS-SART / EM epilogues): every
    product goes to two fixed-point words, 16 atomics per sample."""
    peak = rates["smem_atomic_conflict_free"] / 16.0
    achieved = samples / t
    return {"bound": "smem_atomic", "kernel": "k_bp_mx (split words)", "achieved": achieved / 1e9, "peak": peak / 1e9,
            "unit": "Gsamples/s", "frac": achieved / peak, "traffic": None, "peak_samples_per_s": peak,
            "peak_source": "measured conflict-free shared-memory 32-bit atomic adds (libtgprobe tgp_smem_atomic) / "
                           "16 atomics per sample",
            "random_scatter_peak": rates["smem_atomic_random"] / 16.0 / 1e9,
            "unit_of_work": "one trilinear sample of the interpolated projector (8 contributions, two words each)"}


def roofline_fp(samples, t, rates):
    """k_fp_interp_tex: every sample gathers its 2x2x2 corners with two
    2x2 texture gathers; ceiling = the measured warp-coherent tld4 rate (L1-
    resident array) / 2.  The random-sector L2 ceiling (32 B per sample) is
    reported beside it: the projector exceeds it because neighbouring
    samples of a ray reuse L1-resident lines."""
    peak = rates["tex_gather_coherent_l1"] / 2.0
    achieved = samples / t
    return {"bound": "tex_gather", "kernel": "k_fp_interp_tex", "achieved": achieved / 1e9, "peak": peak / 1e9,
            "unit": "Gsamples/s", "frac": achieved / peak, "traffic": None, "peak_samples_per_s": peak,
            "peak_source": "measured warp-coherent 2x2 FP32 texture gathers, L1-resident array (libtgprobe "
                           "tgp_tex_gather) / 2 gathers per sample",
            "l2_random_gather_peak": rates["l2_sector_gather_gbs"] * 1e9 / 32.0 / 1e9}


def learned_measure(pretrain, finetune, n_eval, ragged=True, log=None):
    """Seconds to PSNR, learned-gradient scheme vs plain CGLS, on the 256^3
    sparse-view workload (60 angles, 512^2 detector at 0.8 mm, 20-ellipsoid
    phantoms, Poisson noise at I0 = 1e4).  The network is trained here first:
    `pretrain` batches of 2 phantoms on the same scan at 64^3 (4 mm voxels),
    then `finetune` phantoms at 256^3; `n_eval` held-out phantoms (seeds
    5000+) are then reconstructed both ways.  The CGLS target is its best
    PSNR over its iteration count (CGLS semi-converges on noisy data); the
    learned time is FDK plus the learned steps needed to reach that PSNR.
    Timed with synchronisation on both sides (host wall clock over
    device-resident inputs).  Data residuals ||A x - b|| are FP32 projections
    with FP64 sums."""
    import torch

    from paper_2412_10129_gb300 import inputs, learned as L, tg
    dev = torch.device("cuda", torch.cuda.current_device())
    t_start = time.perf_counter()
    net = L.LearnedGradient(seed=0).to(dev)
    g64, g256 = inputs.config_learned(64), inputs.config_learned(256)
    l_pre = L.train(net, g64, range(1000, 1000 + 2 * pretrain), steps=10, batch=2, lr=3e-4) if pretrain else []
    torch.cuda.synchronize()
    t_ft0 = time.perf_counter()
    l_ft = L.train(net, g256, range(3000, 3000 + finetune), steps=10, batch=1, lr=1e-4) if finetune else []
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t_start
    s_per_phantom = (time.perf_counter() - t_ft0) / finetune if finetune else None
    eta = 1.0 / L.operator_norm_sq(g256, device=dev)
    rows = []
    for k in range(n_eval):
        b, x0, gt = L.make_sample(g256, 5000 + k, device=dev)
        cand = {}
        for it in (4, 8, 12, 16, 20, 25, 30, 40):
            cand[it] = L.psnr(tg.cgls(g256, b, it), gt)
        k0 = max(cand, key=cand.get)
        for it in range(max(1, k0 - 3), k0 + 4):
            if it not in cand:
                cand[it] = L.psnr(tg.cgls(g256, b, it), gt)
        k_best = max(cand, key=cand.get)
        p_cgls = cand[k_best]
        t_cgls = L.timed(lambda: tg.cgls(g256, b, k_best))
        with torch.no_grad():
            x = tg.fdk(g256, b)
            curve = []
            for _ in range(10):
                x = net.step(x[None], b[None], g256, eta)[0]
                curve.append(L.psnr(x, gt))
        reach = next((i + 1 for i, p in enumerate(curve) if p >= p_cgls), None)

        def recon(steps):
            with torch.no_grad():
                xx = tg.fdk(g256, b)
                for _ in range(steps):
                    xx = net.step(xx[None], b[None], g256, eta)[0]
            return xx

        t_full = L.timed(lambda: recon(10))
        t_reach = L.timed(lambda: recon(reach)) if reach else None
        x_l = recon(10)
        x_c = tg.cgls(g256, b, k_best)
        res = {name: float(torch.linalg.vector_norm((tg.forward(g256, v) - b).double()))
               for name, v in (("learned", x_l), ("cgls", x_c), ("fdk", x0))}
        rows.append({"seed": 5000 + k, "cgls_psnr": p_cgls, "cgls_iters": k_best, "cgls_s": t_cgls,
                     "learned_psnr_10": curve[-1], "learned_psnr_curve": curve, "learned_steps_to_cgls_psnr": reach,
                     "learned_s_to_cgls_psnr": t_reach, "learned_s_10": t_full, "fdk_psnr": L.psnr(x0, gt),
                     "residual_fp64_sum": res})
    out = {"workload": "256^3 at 1 mm, 60 angles over 2pi, 512x512 detector at 0.8 mm, 20-ellipsoid phantoms, "
                       "Poisson noise I0=1e4; learned gradient 10 steps, 5x conv3d 3^3 32 ch (BF16, FP32 acc)",
           "training": {"pretrain_64_batches_of_2": pretrain, "finetune_256_phantoms": finetune,
                        "seconds": t_train, "seconds_per_256_phantom": s_per_phantom,
                        "projected_seconds_2000_phantoms_256": 2000 * s_per_phantom if s_per_phantom else None,
                        "loss_first": l_pre[:3], "loss_last": (l_ft or l_pre)[-3:]},
           "per_phantom": rows}
    reached = [r["learned_s_to_cgls_psnr"] for r in rows if r["learned_s_to_cgls_psnr"] is not None]
    out["learned_s_to_cgls_psnr"] = float(np.mean(reached)) if rows and len(reached) == len(rows) else None
    out["cgls_s_to_best_psnr"] = float(np.mean([r["cgls_s"] for r in rows])) if rows else None
    if ragged:
        sizes = (192, 208, 224, 240, 256, 272, 288, 320)
        geos = [inputs.circular_geometry((n,) * 3, (1.0,) * 3, (2 * n, 2 * n), (0.8, 0.8), 60, 1000.0, 1536.0)
                for n in sizes]
        data = [L.make_sample(gg, 7000 + i, device=dev) for i, gg in enumerate(geos)]
        etas = [1.0 / L.operator_norm_sq(gg, device=dev) for gg in geos]
        bs, x0s = [d[0] for d in data], [d[1] for d in data]
        t_rag = L.timed(lambda: L.infer_ragged(net, geos, bs, x0s, steps=10, etas=etas), reps=2)

        def one_by_one():
            with torch.no_grad():
                for gg, bb, xx, ee in zip(geos, bs, x0s, etas):
                    net(xx, bb, gg, steps=10, eta=ee)

        t_seq = L.timed(one_by_one, reps=2)
        xs = L.infer_ragged(net, geos, bs, x0s, steps=10, etas=etas)
        out["ragged_inference"] = {"sizes": list(sizes), "voxels": int(sum(n ** 3 for n in sizes)), "steps": 10,
                                   "seconds_batched": t_rag, "seconds_one_by_one": t_seq,
                                   "voxel_steps_per_s": 10 * sum(n ** 3 for n in sizes) / t_rag,
                                   "psnr": [L.psnr(x, d[2]) for x, d in zip(xs, data)],
                                   "fdk_psnr": [L.psnr(d[1], d[2]) for d in data]}
        del data, bs, x0s, xs
    torch.cuda.empty_cache()
    return out


def run_learned(args):
    """The learned-vs-CGLS measurement on its own (one JSON line)."""
    import torch

    from paper_2412_10129_gb300 import build, tg
    torch.cuda.set_device(0)
    build.build()
    tg.load()
    n0 = tg.launch_count()
    res = learned_measure(args.pretrain, args.finetune, args.eval, ragged=True)
    line = {"metric": "seconds to PSNR: learned vs CGLS", "value": res["learned_s_to_cgls_psnr"], "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "dtype": "bf16/f32", "data": "synthetic",
            "cgls_value": res["cgls_s_to_best_psnr"], "config": {"workload": res["workload"]},
            "gpu_launches": tg.launch_count() - n0, "learned": res}
    print(json.dumps(line), flush=True)
    return 0


def run_solvers(args):
    """Per-iteration times of the solvers and the extra operators on the
    512^3 / 720-angle workload (one JSON line): each iterative method runs 1
    and 2 iterations from x0 (CUDA events); an iteration costs the
    difference, its set-up (weights, sensitivities, the first projections)
    the rest."""
    import math

    import torch

    from paper_2412_10129_gb300 import build, inputs, tg
    torch.cuda.set_device(0)
    build.build()
    tg.load()
    dev = torch.device("cuda", 0)
    g, x_np = make_inputs(args.case)
    b = torch.from_numpy(inputs.poisson_noise(_siddon_gpu(g, x_np, dev), 1e5, seed=2)).to(dev)
    stream = torch.cuda.current_stream(dev)
    s_interp = tg.count_samples(g, "interp")
    s_siddon = tg.count_samples(g, "siddon")
    pairs = int(np.prod(g.vol_shape)) * g.nAngles

    def timed(fn):
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    def iters(name, call, units):
        t1 = timed(lambda: call(1))
        t2 = timed(lambda: call(2))
        it = t2 - t1
        return {"s_per_iteration": it, "setup_s": t1 - it, "voxel_samples_per_s": units / it if it > 0 else None}

    out = {}
    v = torch.empty(g.vol_shape, device=dev)
    ones = lambda: torch.ones(g.vol_shape, device=dev)  # noqa: E731
    zeros = lambda: torch.zeros(g.vol_shape, device=dev)  # noqa: E731
    fp_bp = s_interp + pairs
    out["mlem"] = iters("mlem", lambda n: tg.mlem(g, b, n, x0=ones()), fp_bp)
    out["osem_20"] = iters("osem", lambda n: tg.osem(g, b, n, blocksize=20, x0=ones()), fp_bp)
    out["mlem_siddon"] = iters("mlem_siddon", lambda n: tg.mlem(g, b, n, x0=ones(), method="siddon"),
                               s_siddon + s_siddon)
    out["os_asd_pocs_20"] = iters("asd", lambda n: tg.asd_pocs(g, b, n, blocksize=20, x0=zeros()), fp_bp)
    out["lsqr"] = iters("lsqr", lambda n: tg.lsqr(g, b, n, x0=zeros()), fp_bp)
    out["lsmr"] = iters("lsmr", lambda n: tg.lsmr(g, b, n, x0=zeros()), fp_bp)
    out["cgls"] = iters("cgls", lambda n: tg.cgls(g, b, n, x0=zeros()), fp_bp)
    tg.backproject(g, b, "siddon", out=v)
    t = timed(lambda: tg.backproject(g, b, "siddon", out=v))
    out["bp_siddon"] = {"s": t, "segments_per_s": s_siddon / t}
    tv = torch.rand(g.vol_shape, device=dev)
    tg.tv_descent(tv, 2, 1e-3)
    out["tv_descent_20_steps"] = {"s": timed(lambda: tg.tv_descent(tv, 20, 1e-3))}
    filt = torch.empty_like(b)
    for name in ("ram-lak", "hamming"):
        tg.fdk_filter(g, b, name, out=filt)
        out[f"fdk_filter_{name}"] = {"s": timed(lambda: tg.fdk_filter(g, b, name, out=filt))}
        out[f"fdk_{name}"] = {"s": timed(lambda: tg.fdk(g, b, name, out=v))}
    # a 200-degree short scan (Parker) and a detector displaced by a quarter
    # of its width (Wang), 720 views each, same volume and detector
    n = g.nAngles
    short = inputs.circular_geometry(g.nVoxel, g.dVoxel, g.nDetector, g.dDetector, n, 1000.0, 1536.0,
                                     arc=math.radians(200.0) * n / (n - 1))
    out["fdk_parker_200deg"] = {"s": timed(lambda: tg.fdk(short, b, parker=True, out=v))}
    off = inputs.circular_geometry(g.nVoxel, g.dVoxel, g.nDetector, g.dDetector, n, 1000.0, 1536.0)
    off.offDetector[:, 0] = 0.25 * g.nDetector[0] * g.dDetector[0]
    out["fdk_wang_quarter_offset"] = {"s": timed(lambda: tg.fdk(off, b, wang=True, out=v))}
    line = {"metric": "solver seconds per iteration at 512^3", "unit": "s", "higher_is_better": False,
            "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": CASES[args.case][0], "units": "voxel_samples = interpolated samples (or Siddon "
                                                                   "segments) + voxel-angle pairs per iteration"},
            "solvers": out}
    print(json.dumps(line), flush=True)
    return 0


def run_micro(args):
    """The micro-CT workload on its own (one JSON line): 1024^3 at 0.125 mm,
    1600 angles over 2 pi, 1024^2 detector at 0.2 mm, every angle with its
    own seeded detector offset, in-plane tilt and source jitter; phantom =
    200 ellipsoids + a porous cylinder, data = its Siddon projection with
    Poisson noise at I0 = 1e5.  Forward and back projection throughput (one
    launch each after a warm-up one, CUDA events) and 10 CGLS iterations."""
    import torch

    from paper_2412_10129_gb300 import build, inputs, tg
    torch.cuda.set_device(0)
    build.build()
    tg.load()
    dev = torch.device("cuda", 0)
    g = inputs.config_micro()
    x_np = inputs.micro_phantom(g, seed=1)
    x = torch.from_numpy(x_np).to(dev)
    b = inputs.poisson_noise_device(tg.forward(g, x, "siddon"), 1e5, seed=2)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, warm=True):
        if warm:
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    s_interp = tg.count_samples(g, "interp")
    s_siddon = tg.count_samples(g, "siddon")
    pairs = int(np.prod(g.vol_shape)) * g.nAngles
    p_tmp = torch.empty(g.proj_shape, device=dev)
    v_tmp = torch.empty(g.vol_shape, device=dev)
    clocks = ClockSampler(0)
    clocks.start()
    t = {"fp_interp": timed(lambda: tg.forward(g, x, "interp", out=p_tmp)),
         "fp_siddon": timed(lambda: tg.forward(g, x, "siddon", out=p_tmp)),
         "bp_matched": timed(lambda: tg.backproject(g, b, "matched", out=v_tmp)),
         "bp_fdk": timed(lambda: tg.backproject(g, b, "fdk", out=v_tmp))}
    del p_tmp, v_tmp
    torch.cuda.empty_cache()
    hist = []
    t["cgls_10"] = timed(lambda: hist.append(tg.cgls(g, b, 10, resid=True)[1]), warm=False)
    clk = clocks.stop()
    rates = _probe_rates()
    value = (s_interp + pairs) / (t["fp_interp"] + t["bp_matched"])
    line = {"metric": "FP+BP voxel-samples/s at 1024^3 micro-CT (per-angle jitter)", "value": value, "unit": UNIT,
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "1024^3 FP32 volume (0.125 mm), 1600 angles over 2pi, 1024x1024 detector (0.2 mm), "
                                   "per-angle detector offset +-2 px, tilt +-0.5 deg, source jitter +-0.5 mm; "
                                   "200 ellipsoids + porous cylinder; Poisson noise I0=1e5"},
            "seconds": t, "clocks": clk,
            "units": {"interp_samples": s_interp, "siddon_segments": s_siddon, "voxel_angle_pairs": pairs},
            "rates": {"fp_interp_samples_per_s": s_interp / t["fp_interp"],
                      "fp_siddon_segments_per_s": s_siddon / t["fp_siddon"],
                      "bp_matched_samples_per_s": s_interp / t["bp_matched"],
                      "bp_fdk_pairs_per_s": pairs / t["bp_fdk"],
                      "cgls_s_per_iteration": t["cgls_10"] / 10},
            "cgls_residual_history": [float(v) for v in np.asarray(hist[-1]).ravel()],
            "roofline": roofline_bp(s_interp, t["bp_matched"], rates),
            "roofline_fp": roofline_fp(s_interp, t["fp_interp"], rates)}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_line(g, x_np, b.cpu().numpy())
    print(json.dumps(line), flush=True)
    return 0


KERNEL_CASES = ("fp_interp", "fp_siddon", "bp_matched", "bp_fdk", "bp_siddon", "fdk_rows_hamming", "tv_march",
                "sirt")


def run_kernel(args):
    """The capture workload of one kernel for a profiler (no JSON line):
    the half-resolution scan (256^3 at 1 mm, 360 views, 384 x 512 detector:
    inputs above the 129 MB L2, a few GB on the device), one warm-up and one
    further launch of the named operator; tv_march runs on a 512^3 volume;
    sirt is one SIRT iteration (its backprojections use the split-word
    accumulation)."""
    import torch

    from paper_2412_10129_gb300 import build, inputs, tg
    torch.cuda.set_device(0)
    build.build()
    tg.load()
    g = inputs.circular_geometry((256, 256, 256), (1.0,) * 3, (512, 384), (0.8, 0.8), 360, 1000.0, 1536.0)
    gen = torch.Generator(device="cuda").manual_seed(3)
    b = torch.rand(g.proj_shape, generator=gen, device="cuda")
    x = torch.rand(g.vol_shape, generator=gen, device="cuda")
    v = torch.empty(g.vol_shape, device="cuda")
    p = torch.empty(g.proj_shape, device="cuda")
    ops = {"fp_interp": lambda: tg.forward(g, x, "interp", out=p),
           "fp_siddon": lambda: tg.forward(g, x, "siddon", out=p),
           "bp_matched": lambda: tg.backproject(g, b, "matched", out=v),
           "bp_fdk": lambda: tg.backproject(g, b, "fdk", out=v),
           "bp_siddon": lambda: tg.backproject(g, b, "siddon", out=v),
           "fdk_rows_hamming": lambda: tg.fdk_filter(g, b, "hamming", out=p),
           # one SIRT iteration: column weights (split-word BP of ones) and one update
           "sirt": lambda: tg.sirt(g, b, 1)}
    if args.kernel == "tv_march":
        xt = torch.rand((512, 512, 512), generator=gen, device="cuda")
        fn = lambda: tg.tv_descent(xt, 1, 1e-3)  # noqa: E731
    else:
        fn = ops[args.kernel]
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    return 0


def _siddon_gpu(g, x_np, dev):
    import torch

    from paper_2412_10129_gb300 import tg
    return tg.forward(g, torch.from_numpy(x_np).to(dev), "siddon").cpu().numpy()


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tg", choices=["tg", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", default="bp_matched", choices=KERNEL_CASES,
                    help="--case kernel: the operator whose capture workload runs")
    ap.add_argument("--case", default="clinical", choices=sorted(CASES) + ["learned", "solvers", "micro", "kernel"],
                    help="workload; 'medium' is the half-resolution scan used for profiler captures; 'learned' "
                         "trains the learned-gradient scheme and times it against CGLS; 'solvers' times one "
                         "iteration of every solver and the extra operators at 512^3")
    ap.add_argument("--pretrain", type=int, default=300, help="learned: 64^3 training batches (2 phantoms each)")
    ap.add_argument("--finetune", type=int, default=40, help="learned: 256^3 training phantoms")
    ap.add_argument("--eval", type=int, default=2, help="learned: held-out phantoms")
    ap.add_argument("--learned-pretrain", type=int, default=150,
                    help="default case: 64^3 training batches of the learned-vs-CGLS object (0 = leave it out)")
    ap.add_argument("--learned-finetune", type=int, default=20,
                    help="default case: 256^3 training phantoms of the learned-vs-CGLS object")
    args = ap.parse_args()
    if args.case == "learned":
        return run_learned(args) if args.impl != "reference" else 0
    if args.case == "micro":
        return run_micro(args) if args.impl != "reference" else 0
    if args.case == "kernel":
        return run_kernel(args) if args.impl != "reference" else 0
    if args.case == "solvers":
        args.case = "clinical"
        return run_solvers(args) if args.impl != "reference" else 0
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
