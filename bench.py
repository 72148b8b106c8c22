"""Benchmark: HEALPix analysis throughput (Gpix/s) of the HP2SPH path on GB300.

Workload: 32 FP32 maps at Nside 1024 (12,582,912 pixels each), lmax 2048,
seeded power-law skies (C_l = l^-alpha, alpha ~ U[1.5, 2.5] per map) plus
N(0, 1e-3) white noise.  One step = hpx_analyze + hpx_cl over the whole batch.
The maps (1.61 GB) are larger than L2, so every step streams them from HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun each rank analyses its own batch of 32 maps (weak scaling, no
collective on the data path); rank 0 prints one JSON line.  `--impl reference`
times the FP64 CPU oracle on the host cores on a bounded sample of the same
workload.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HEALPix analysis Gpix/s at Nside=1024 (batched FP32 vs plain FP64, err<=1e-5)"
NSIDE, LMAX, BATCH = 1024, 2048, 32
WORKLOAD = "bench_nside1024x32"
MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
# measured DRAM traffic (read + written, GB) / algorithmic bytes of each stage at Nside 512, 32 maps
# (ncu --set full captures of the stage's launches; the summaries are in profiles/).  Dirty lines
# still in L2 when a kernel ends are not counted, so a ratio can fall below 1.
TRAFFIC_OVER_ALGORITHMIC = {
    "fused_fsht": (1.4479 + 0.1249) / 1.4828,                      # fused_tc_ws_kernel, packed b
    "ring_fft": (0.11342 + 0.08983 + 0.31140 + 0.34239) / 0.94031,  # ring_ct_kernel + ring_fft_kernel
    "lat_fft": (0.53804 + 0.24894) / 0.80688,                      # lat_fft_pair_ct_kernel, packed b
    "spread": (0.54846 + 0.49414) / 1.07532,                       # spread_rb_kernel
}
# forms of the FP32 run-time sweep kernel (hpx_plan_tuning)
SWEEP_FORMS = ["complex lanes, 32 stages per pass", "complex lanes, 16 stages per pass",
               "real lanes, 32 stages per pass"]
# FP32 SIMT peak: 152 SMs x 128 FP32 lanes x 2 flop/FMA x 2.070 GHz (maximum SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def config_dict():
    return {"workload": "%s: %d FP32 maps, Nside %d, lmax %d, power-law skies + 1e-3 noise"
                        % (WORKLOAD, BATCH, NSIDE, LMAX),
            "nside": NSIDE, "lmax": LMAX, "batch_per_gpu": BATCH,
            "l2": "inputs larger than L2 (1.61 GB of maps per step)"}


# ------------------------------------------------------------------ ranks (weak scaling, no collective on the data path)
def first_map(rank, batch):
    """Index of the first map of `rank`'s batch: every rank analyses its own maps."""
    return rank * batch


def max_over_ranks(seconds, world, device):
    """The slowest rank's time (the job's time); one all-reduce outside the timed region."""
    if world == 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gpix(world, pixels_per_rank, seconds):
    """Whole-job throughput: the pixels of all ranks over the slowest rank's time."""
    return world * pixels_per_rank / seconds / 1e9


# ------------------------------------------------------------------ accounting
def chain_len(mp, c, L):
    return (L - mp - c) // 2 + 1 if L >= mp + c else 0


def rotation_count(L):
    n = 0
    for m in range(L + 1):
        m0 = m & 1
        for c in (0, 1):
            for s in range((m - m0) // 2):
                n += chain_len(m0 + 2 + 2 * s, c, L)
    return n


def stage_work(ns, L, B, es=8):
    """Algorithmic HBM bytes or flops of one launch of each stage (FP32)."""
    p = 2 * ns
    Q = 4 * ns + 1
    P2 = p // 2 + 1
    npix = 12 * ns * ns
    dense = 0
    for mpar in (0, 1):
        nm = (L - mpar) // 2 + 1
        for par in (0, 1):
            nl = len([l for l in range(mpar, L + 1) if l % 2 == par])
            nj = len([j for j in range(mpar, p + 1) if j % 2 == par])
            dense += nm * nl * nj * 4          # real matrix x complex vector: 2 FMA
    nalm = (L + 1) * (L + 2) // 2
    return {
        "ring_fft": ("hbm", B * (npix * es // 2 + Q * (p + 1) * es)),
        "poles": ("hbm", B * 2 * 36 * 4),
        # half-grid spreading: read the L+1 used columns of Y, write U (M/2 + 1 per column)
        "spread": ("hbm", B * (L + 1) * (Q * es + (4 * ns + 1) * es)),
        # grid FFT: read U, write the right-hand sides
        "lat_fft": ("hbm", B * (L + 1) * ((4 * ns + 1) * es + 2 * P2 * es)),
        "lat_solve": ("alu", B * dense),
        "rot_sweep": ("alu", B * rotation_count(L) * 12),
        # per-order operators on the tensor cores: read M (n_alm x P2 entries of 4 bytes, an FP16
        # pair each, once per launch for up to 32 maps) and the right-hand sides, write the
        # coefficients
        "fused_fsht": ("hbm", ((B + 31) // 32) * nalm * P2 * 4 + B * (L + 1) * 2 * P2 * es + B * nalm * es),
        "unused": ("alu", 0),
    }


def fused_compute_view(work, ms, peaks):
    """The per-order operator stage under the survey's accounting of steps a-4 + a-5: its algorithmic
    work is the flops of the latitude operator D and of the Givens sweeps it replaces (exact counts),
    a compute-bound stage; the kernel runs on the tensor cores (FP16 pairs, three MMAs per product),
    so the peak is the measured dense FP16/BF16 rate.  The operator stream and the MMA flops the kernel
    executes are reported beside it."""
    flops = work["lat_solve"][1] + work["rot_sweep"][1]
    peak = peaks.get("bf16_tflops", 1900.0)
    t = ms / 1e3
    return {"bound": "tensor", "achieved": flops / t / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac": flops / t / 1e12 / peak,
            "peak_source": "measured bf16 dense (FP16 MMAs run at the same rate)" if "bf16_tflops" in peaks
            else "fallback",
            "algorithmic_flops": flops, "what": "D application + Givens sweeps (steps a-4, a-5), exact counts"}


def stage_roofline(kind, amount, ms, peaks):
    """Roofline entry of one stage: algorithmic bytes (or flops) of one launch over its time."""
    t = ms / 1e3
    if kind == "hbm":
        peak = peaks.get("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "achieved": amount / t / 1e9, "peak": peak, "unit": "GB/s",
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    else:
        roof = {"bound": "alu", "achieved": amount / t / 1e12, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "peak_source": "FP32 FMA pipes: 152 SMs x 128 lanes x 2 flop x 2.070 GHz"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    return roof


def roofline_report(work, per_launch, peaks):
    """The roofline object of the dominant stage (longest time per call) and a short entry per stage.

    work: stage -> (bound, algorithmic bytes or flops per launch); per_launch: stage -> ms per launch.
    DRAM bytes per launch come from an ncu capture (dram__bytes_read + write) over the algorithmic bytes of
    the same kernel at Nside 512 x 32 maps, scaled to this launch (traffic grows with the operator size like
    the algorithmic bytes: tile rows padded to 8, K to a multiple of 32); null for stages without a capture.
    """
    names = [n for n in per_launch if n in work and work[n][1] > 0]
    dom = max(names, key=lambda n: per_launch[n])
    kind, amount = work[dom]
    ratio = TRAFFIC_OVER_ALGORITHMIC.get(dom)
    if dom == "fused_fsht" and "lat_solve" in work:
        roof = fused_compute_view(work, per_launch[dom], peaks)
        stream = stage_roofline(kind, amount, per_launch[dom], peaks)
        roof["operator_stream"] = {"bytes": amount, "achieved_gbs": stream["achieved"], "frac_hbm": stream["frac"]}
        roof["traffic"] = amount * ratio if ratio else None
    else:
        roof = stage_roofline(kind, amount, per_launch[dom], peaks)
        roof["traffic"] = amount * ratio if (ratio and kind == "hbm") else None
    roof["traffic_source"] = ("ncu at Nside 512, 32 maps: %.4f x the stage's algorithmic bytes, scaled" % ratio
                              if roof.get("traffic") else None)
    roof["kernel"] = dom
    roof["per_launch_ms"] = per_launch[dom]
    per_stage = {}
    for n in names:
        r = stage_roofline(work[n][0], work[n][1], per_launch[n], peaks)
        per_stage[n] = {"bound": r["bound"], "ms": per_launch[n], "achieved": r["achieved"], "unit": r["unit"],
                        "frac": r["frac"]}
        if n in TRAFFIC_OVER_ALGORITHMIC and work[n][0] == "hbm":
            per_stage[n]["traffic"] = work[n][1] * TRAFFIC_OVER_ALGORITHMIC[n]
    return roof, per_stage


# ------------------------------------------------------------------ clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(maps0, ms):
    """Time the FP64 oracle on orders `ms` of one map; returns (seconds, columns)."""
    from oracle import hp2sph
    t0 = time.perf_counter()
    cols = hp2sph.analyze_columns(maps0.astype(np.float64), NSIDE, LMAX, ms)
    return time.perf_counter() - t0, cols


def fit_cost_model(n_small, t_small, n_large, t_large):
    """The oracle's time for n orders of one map is fixed + n * per_order: the fixed part
    (the least-squares factorisation in latitude, the per-ring Python loop, the Fourier
    basis at the quadrature nodes) does not grow with the number of orders.  Two sample
    sizes give both terms."""
    per = max((t_large - t_small) / (n_large - n_small), 1e-9)
    fixed = max(t_small - n_small * per, 0.0)
    return fixed, per


def full_map_seconds(fixed, per):
    return fixed + (LMAX + 1) * per


def cpu_gpix(seconds_full_map):
    return 12 * NSIDE * NSIDE / seconds_full_map / 1e9


SMALL_ORDERS, LARGE_ORDERS = [0, 1], list(range(8))


def run_reference(args, rank):
    if rank != 0:
        return
    import skies
    maps0 = skies.workload_maps(WORKLOAD, nmaps=1, dtype=np.float32)[0]
    # warm-up steps alternate two sample sizes to fit the fixed and per-order costs
    ts_s, ts_l = [], []
    for k in range(args.warmup):
        if k % 2 == 0:
            ts_l.append(oracle_sample(maps0, LARGE_ORDERS)[0])
        else:
            ts_s.append(oracle_sample(maps0, SMALL_ORDERS)[0])
    if not ts_s:
        ts_s.append(oracle_sample(maps0, SMALL_ORDERS)[0])
    fixed, _ = fit_cost_model(len(SMALL_ORDERS), float(np.median(ts_s)), len(LARGE_ORDERS), float(np.median(ts_l)))
    # every timed step: orders 0..7 of map 0; its full-map time = fixed + 2049 x its per-order time
    ts = [oracle_sample(maps0, LARGE_ORDERS)[0] for _ in range(args.steps)]
    fulls = [full_map_seconds(fixed, max(t - fixed, 1e-9) / len(LARGE_ORDERS)) for t in ts]
    t = float(np.mean(ts))
    v = cpu_gpix(float(np.mean(fulls)))
    sample = ("orders m=0..7 of map 0 (8 of 2049 columns) per step; full-map time = fixed + 2049 x per-order "
              "(fixed part %.2f s fitted from the warm-up steps' 2- and 8-order samples); FP64 oracle (direct "
              "ring DFTs, dense least squares, Gauss-Legendre projection)" % fixed)
    line = {"metric": METRIC, "value": v, "unit": "Gpix/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(),
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "Gpix/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample, "model": {"fixed_s": fixed,
                                                         "full_map_s": float(np.mean(fulls))}},
            "e2e": {"value": v, "unit": "Gpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ other workloads
def uneven_leg(hp, torch, stream, args):
    """200 FP32 maps with Nside drawn from {64, 128, 256, 512, 1024} (probabilities .40/.30/.15/.10/.05,
    skies.uneven_nsides), lmax = 2 Nside: one group plan replayed as one CUDA graph, and the same maps
    as one uniform plan per Nside run one after the other (the sum of their times).  Timing inputs:
    seeded white-noise maps of those sizes (the throughput does not depend on the sky)."""
    import skies
    nsides = [int(v) for v in skies.uneven_nsides(200)]
    rng = np.random.default_rng(4000)
    npix = [12 * n * n for n in nsides]
    x = torch.as_tensor(rng.standard_normal(sum(npix)).astype(np.float32), device="cuda")
    plan = hp.Plan(nsides=nsides, precision="fp32", graph=True)
    alm = torch.empty(plan.nalm, dtype=torch.complex64, device="cuda")
    cl = torch.empty(plan.ncl, dtype=torch.float64, device="cuda")
    for _ in range(3):
        plan.analyze(x, out=alm)
        plan.cl(alm, out=cl)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = max(3, min(args.steps, 10))
    e0.record(stream)
    for _ in range(n):
        plan.analyze(x, out=alm)
        plan.cl(alm, out=cl)
    e1.record(stream)
    torch.cuda.synchronize()
    t_group = e0.elapsed_time(e1) / n / 1e3
    launches = hp.lib().hpx_plan_launches(plan.handle)
    plan.close()
    # one uniform plan per Nside, maps gathered by Nside
    t_sum = 0.0
    counts = {}
    for ns in sorted(set(nsides)):
        cnt = nsides.count(ns)
        counts[ns] = cnt
        p1 = hp.Plan(ns, 2 * ns, cnt, "fp32")
        xs = torch.as_tensor(rng.standard_normal((cnt, 12 * ns * ns)).astype(np.float32), device="cuda")
        a1 = p1.analyze(xs)
        c1 = p1.cl(a1)
        for _ in range(2):
            p1.analyze(xs, out=a1)
            p1.cl(a1, out=c1)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n):
            p1.analyze(xs, out=a1)
            p1.cl(a1, out=c1)
        e1.record(stream)
        torch.cuda.synchronize()
        t_sum += e0.elapsed_time(e1) / n / 1e3
        p1.close()
    pix = float(sum(npix))
    return {"value": pix / t_group / 1e9, "unit": "Gpix/s", "ms_per_step": t_group * 1e3,
            "maps_per_nside": counts, "pixels": int(pix), "graph_nodes_kernels": launches,
            "separate_uniform_plans": {"value": pix / t_sum / 1e9, "unit": "Gpix/s", "ms_per_step": t_sum * 1e3},
            "inputs": "seeded white-noise maps of the workload's sizes"}


def gradient_leg(hp, torch, stream, args):
    """8 FP32 maps at Nside 2048, lmax 4096: loss = sum_l w_l (C_l - C*_l)^2 (w_l = 1/l, l >= 2) and its
    gradient with respect to the maps (analysis, C_l, then the C_l and analysis vector-Jacobian products
    in the library).  Timing inputs: seeded white-noise maps."""
    ns, L, B = 2048, 4096, 8
    rng = np.random.default_rng(2048)
    x = torch.as_tensor(rng.standard_normal((B, 12 * ns * ns)).astype(np.float32), device="cuda")
    plan = hp.Plan(ns, L, B, "fp32", autotune=True)   # the sweeps: stages per pass and FFT launch shapes
    w = torch.zeros(L + 1, dtype=torch.float64, device="cuda")
    w[2:] = 1.0 / torch.arange(2, L + 1, dtype=torch.float64, device="cuda")
    cstar = torch.as_tensor(np.r_[0.0, 0.0, np.arange(2, L + 1, dtype=np.float64) ** -2.0], device="cuda")

    def step():
        xg = x.detach().requires_grad_(True)
        c = hp.cl(hp.analyze(xg, plan), plan)
        loss = torch.sum(w * (c - cstar) ** 2)
        loss.backward()
        return xg.grad

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 3
    e0.record(stream)
    for _ in range(n):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / n / 1e3
    path = "sweeps" if plan.flags & hp.HPX_FLAG_SWEEPS else "per-order operators"
    form = SWEEP_FORMS[plan.tuning[2]]
    plan.close()
    return {"value": B * 12 * ns * ns / t / 1e9, "unit": "Gpix/s (loss + map gradient)", "ms_per_step": t * 1e3,
            "path": path, "sweep_form": form, "inputs": "seeded white-noise maps"}


# ------------------------------------------------------------------ GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes (e.g. under a profiler, whose serialised timings "
                         "would steer the tuning)")
    ap.add_argument("--kernels-only", action="store_true",
                    help="time only the device-resident step (for profiler runs): no e2e, FP64 or CPU legs")
    ap.add_argument("--nside", type=int, default=NSIDE, help="smaller cases for profiler captures")
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--sweeps", action="store_true",
                    help="with --kernels-only: the run-time Givens sweeps instead of the per-order operators")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist

    import paper_1904_10514_gb300 as hp
    import skies

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    ns, nb = args.nside, args.batch
    if ns == NSIDE:
        maps_np = skies.workload_maps(WORKLOAD, nmaps=nb, first=first_map(rank, nb), dtype=np.float32)
    else:
        maps_np = skies.small_powerlaw_maps(ns, nb, seed=6000 + rank, alpha=2.0, noise=1e-3)[0].astype(np.float32)
    t_plan0 = time.perf_counter()
    # autotune: launch shapes of the FFT stages, and the operators against the sweeps
    plan = hp.Plan(ns, 2 * ns, nb, "fp32", sweeps=args.sweeps and args.kernels_only, autotune=not args.no_autotune)
    torch.cuda.synchronize()
    plan_build_s = time.perf_counter() - t_plan0
    maps = torch.from_numpy(maps_np).cuda()
    alm = torch.empty((nb, plan.nalm), dtype=torch.complex64, device="cuda")
    cl = torch.empty((nb, plan.lmax + 1), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        plan.analyze(maps, out=alm)
        plan.cl(alm, out=cl)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = Clocks(local)
    hp.hpx_set_profiling(plan.handle, 1)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    stage_ms, ncalls = hp.hpx_stage_times(plan.handle)
    hp.hpx_set_profiling(plan.handle, 0)
    t_step = e0.elapsed_time(e1) / args.steps / 1e3
    t_step = max_over_ranks(t_step, world, "cuda")
    npix_step = nb * plan.npix
    value = job_gpix(world, npix_step, t_step)
    if args.kernels_only:
        if rank == 0:
            per_launch = {n: stage_ms[k] / max(ncalls, 1) for k, n in enumerate(plan.stages)}
            print(json.dumps({"nside": ns, "batch": nb, "value": value, "unit": "Gpix/s",
                              "ms_per_step": t_step * 1e3, "stages_ms_per_launch": per_launch,
                              "plan_build_s": plan_build_s, "plan_gb": plan.nbytes / 1e9,
                              "launch_shapes": list(plan.tuning)}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    # end to end through the public API from pinned host memory: every step copies its
    # maps host -> device and its alm and C_l device -> host.  The steps are pipelined as
    # a user would run a stream of batches: the upload of step k+1 and the download of
    # step k-1 run on their own streams while step k is analysed (double buffers, events).
    host_maps = torch.from_numpy(maps_np).pin_memory()
    host_alm = [torch.empty((nb, plan.nalm), dtype=torch.complex64).pin_memory() for _ in range(2)]
    host_cl = [torch.empty((nb, plan.lmax + 1), dtype=torch.float64).pin_memory() for _ in range(2)]
    dmaps = [maps, torch.empty_like(maps)]
    dalm = [alm, torch.empty_like(alm)]
    dcl = [cl, torch.empty_like(cl)]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_comp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def e2e_run(K):
        s_in.wait_stream(stream)
        s_out.wait_stream(stream)
        for k in range(K):
            i = k % 2
            with torch.cuda.stream(s_in):
                if k >= 2:
                    s_in.wait_event(ev_comp[i])          # step k-2 has read dmaps[i]
                dmaps[i].copy_(host_maps, non_blocking=True)
                ev_in[i].record(s_in)
            stream.wait_event(ev_in[i])
            if k >= 2:
                stream.wait_event(ev_out[i])             # step k-2's results are on the host
            plan.analyze(dmaps[i], out=dalm[i])
            plan.cl(dalm[i], out=dcl[i])
            ev_comp[i].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_comp[i])
                host_alm[i].copy_(dalm[i], non_blocking=True)
                host_cl[i].copy_(dcl[i], non_blocking=True)
                ev_out[i].record(s_out)
        stream.wait_stream(s_out)

    # the copies alone, to show what bounds the pipelined steps
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s_in):
        dmaps[1].copy_(host_maps, non_blocking=True)
        c0.record(s_in)
        for _ in range(3):
            dmaps[1].copy_(host_maps, non_blocking=True)
        c1.record(s_in)
    torch.cuda.synchronize()
    h2d_gbs = 3 * host_maps.numel() * 4 / (c0.elapsed_time(c1) / 1e3) / 1e9
    with torch.cuda.stream(s_out):
        c0.record(s_out)
        for _ in range(3):
            host_alm[1].copy_(dalm[0], non_blocking=True)
        c1.record(s_out)
    torch.cuda.synchronize()
    d2h_gbs = 3 * host_alm[1].numel() * 8 / (c0.elapsed_time(c1) / 1e3) / 1e9

    e2e_run(2)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    t_e2e = e0.elapsed_time(e1) / args.steps / 1e3
    t_e2e = max_over_ranks(t_e2e, world, "cuda")
    e2e = {"value": job_gpix(world, npix_step, t_e2e), "unit": "Gpix/s",
           "h2d_bytes_per_step": int(host_maps.numel() * 4),
           "d2h_bytes_per_step": int(host_alm[0].numel() * 8 + host_cl[0].numel() * 8),
           "pipelined": "upload of step k+1 and download of step k-1 overlap the analysis of step k",
           "h2d_gbs_alone": h2d_gbs, "d2h_gbs_alone": d2h_gbs,
           "host_result_matches_device": bool(torch.equal(host_alm[(args.steps - 1) % 2],
                                                          dalm[(args.steps - 1) % 2].cpu()))}

    # spherical-harmonic synthesis of the same batch (the inverse direction): alm -> maps
    t_syn0 = time.perf_counter()
    plan_syn = hp.Plan(NSIDE, LMAX, nb, "fp32", jacobi=True)   # synthesis + the Jacobi workspace
    torch.cuda.synchronize()
    syn_build_s = time.perf_counter() - t_syn0
    maps_syn = torch.empty_like(maps)
    for _ in range(2):
        plan_syn.sh_synthesis(alm, out=maps_syn)
    torch.cuda.synchronize()
    nsyn = max(2, min(args.steps, 5))
    hp.hpx_set_profiling(plan_syn.handle, 1)
    e0.record(stream)
    for _ in range(nsyn):
        plan_syn.sh_synthesis(alm, out=maps_syn)
    e1.record(stream)
    torch.cuda.synchronize()
    syn_ms, syn_calls = hp.hpx_stage_times(plan_syn.handle)
    hp.hpx_set_profiling(plan_syn.handle, 0)
    t_syn = e0.elapsed_time(e1) / nsyn / 1e3
    synthesis = {"value": npix_step / t_syn / 1e9, "unit": "Gpix/s", "ms_per_step": t_syn * 1e3,
                 "stages_ms_per_launch": {n: syn_ms[k] / max(syn_calls, 1)
                                          for k, n in enumerate(hp.STAGES_SYNTH) if n != "unused"},
                 "plan_build_s": syn_build_s,
                 "path": "per-order synthesis operators" if plan_syn.flags & hp.HPX_FLAG_SWEEPS == 0 else "sweeps"}
    # the HEALPix software's analysis (Sec. 2.2), the paper's comparison method: equal-weight
    # quadrature (niter = 0) and with the default 3 Jacobi iterations, same batch
    healpix_sw = {}
    alm_hs = torch.empty_like(alm)
    for niter in (0, 3):
        plan_syn.healpix_analysis(maps, niter=niter, out=alm_hs)
        torch.cuda.synchronize()
        nh = 3
        e0.record(stream)
        for _ in range(nh):
            plan_syn.healpix_analysis(maps, niter=niter, out=alm_hs)
        e1.record(stream)
        torch.cuda.synchronize()
        th = e0.elapsed_time(e1) / nh / 1e3
        healpix_sw["niter_%d" % niter] = {"value": npix_step / th / 1e9, "unit": "Gpix/s", "ms_per_step": th * 1e3}
    plan_syn.close()
    del maps_syn, alm_hs

    # ablation: the paper's form of the latitude solve (CG on the normal equations per
    # column) with the run-time sweeps, same batch
    plan_cg = hp.Plan(NSIDE, LMAX, nb, "fp32", cg=True)
    alm_cg = torch.empty_like(alm)
    plan_cg.analyze(maps, out=alm_cg)
    torch.cuda.synchronize()
    ncg = 2
    e0.record(stream)
    for _ in range(ncg):
        plan_cg.analyze(maps, out=alm_cg)
    e1.record(stream)
    torch.cuda.synchronize()
    t_cg = e0.elapsed_time(e1) / ncg / 1e3
    cg = {"value": npix_step / t_cg / 1e9, "unit": "Gpix/s", "ms_per_step": t_cg * 1e3,
          "max_abs_diff_vs_default": float((alm_cg - alm).abs().max() / alm.abs().max())}
    plan_cg.close()
    del alm_cg

    # the run-time Givens sweeps (HPX_FLAG_SWEEPS): D applied alone and the rotation kernel,
    # stage by stage, same batch
    plan_sw = hp.Plan(NSIDE, LMAX, nb, "fp32", sweeps=True, autotune=True)
    alm_sw = torch.empty_like(alm)
    for _ in range(2):
        plan_sw.analyze(maps, out=alm_sw)
    torch.cuda.synchronize()
    nsw = 3
    hp.hpx_set_profiling(plan_sw.handle, 1)
    e0.record(stream)
    for _ in range(nsw):
        plan_sw.analyze(maps, out=alm_sw)
    e1.record(stream)
    torch.cuda.synchronize()
    t_sw = e0.elapsed_time(e1) / nsw / 1e3
    sw_ms, sw_calls = hp.hpx_stage_times(plan_sw.handle)
    hp.hpx_set_profiling(plan_sw.handle, 0)
    sw_stage = {n: sw_ms[k] / max(sw_calls, 1) for k, n in enumerate(plan_sw.stages)}
    sw_work = stage_work(NSIDE, LMAX, nb)
    rot_flops = sw_work["rot_sweep"][1]
    sweeps = {"value": npix_step / t_sw / 1e9, "unit": "Gpix/s", "ms_per_step": t_sw * 1e3,
              "stages_ms_per_launch": sw_stage,
              "rot_sweep": {"flops": rot_flops, "tflops": rot_flops / (sw_stage["rot_sweep"] / 1e3) / 1e12,
                            "fp32_pipe_frac": rot_flops / (sw_stage["rot_sweep"] / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
                            "peak": "FP32 FMA pipes: 152 SMs x 128 lanes x 2 flop x 2.070 GHz"},
              "lat_solve": {"flops": sw_work["lat_solve"][1],
                            "tflops": sw_work["lat_solve"][1] / (sw_stage["lat_solve"] / 1e3) / 1e12},
              "max_abs_diff_vs_default": float((alm_sw - alm).abs().max() / alm.abs().max()),
              "sweep_form": SWEEP_FORMS[plan_sw.tuning[2]]}
    plan_sw.close()
    del alm_sw

    # uneven batch (200 maps, Nside drawn from {64, ..., 1024}, lmax = 2 Nside) in one plan replayed
    # as one CUDA graph, against the same maps as separate uniform plans (one per Nside)
    uneven = uneven_leg(hp, torch, stream, args)
    # differentiation workload: 8 maps at Nside 2048, C_l loss, gradient through the library's
    # vector-Jacobian products (hpx_cl_vjp, hpx_analyze_vjp)
    diffw = gradient_leg(hp, torch, stream, args)

    # the plain FP64 single-map form on the same GPU
    plan64 = hp.Plan(NSIDE, LMAX, 1, "fp64")
    m64 = maps[:1].double().contiguous()
    a64 = torch.empty((1, plan64.nalm), dtype=torch.complex128, device="cuda")
    c64 = torch.empty((1, LMAX + 1), dtype=torch.float64, device="cuda")
    for _ in range(2):
        plan64.analyze(m64, out=a64)
        plan64.cl(a64, out=c64)
    torch.cuda.synchronize()
    n64 = max(2, min(args.steps, 5))
    e0.record(stream)
    for _ in range(n64):
        plan64.analyze(m64, out=a64)
        plan64.cl(a64, out=c64)
    e1.record(stream)
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1) / n64 / 1e3
    fp64 = {"value": plan64.npix / t64 / 1e9, "unit": "Gpix/s", "ms_per_map": t64 * 1e3}
    plan64.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel (and of every stage)
    work = stage_work(NSIDE, LMAX, BATCH)
    per_launch = {n: stage_ms[k] / max(ncalls, 1) for k, n in enumerate(plan.stages) if n != "unused"}
    peaks = json.load(open(MEASURED)) if os.path.exists(MEASURED) else {}
    roof, per_stage = roofline_report(work, per_launch, peaks)

    cpu = None
    if not args.no_cpu:
        t_small, _ = oracle_sample(maps_np[0], SMALL_ORDERS)
        ms = list(range(16))
        secs, cols = oracle_sample(maps_np[0], ms)
        fixed, per = fit_cost_model(len(SMALL_ORDERS), t_small, len(ms), secs)
        got = alm[0].cpu().numpy()
        worst = 0.0
        for m in ms:
            i0 = m * (2 * LMAX + 1 - m) // 2 + m
            g = got[i0:i0 + LMAX - m + 1]
            r = cols[m][0]
            worst = max(worst, float(np.max(np.abs(g - r)) / np.max(np.abs(r))))
        # a directly measured point: one whole Nside-256 map (lmax 512), no extrapolation
        from oracle import hp2sph
        m256 = skies.small_powerlaw_maps(256, 1, seed=6256, alpha=2.0, noise=1e-3)[0][0]
        t0 = time.perf_counter()
        hp2sph.analyze(m256, 256, 512)
        t256 = time.perf_counter() - t0
        cpu = {"value": cpu_gpix(full_map_seconds(fixed, per)), "unit": "Gpix/s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": "orders m=0..1 (%.1f s) and m=0..15 (%.1f s) of map 0, FP64 oracle; full-map time = "
                         "fixed + 2049 x per-order = %.1f + 2049 x %.3f s" % (t_small, secs, fixed, per),
               "model": {"fixed_s": fixed, "per_order_s": per, "full_map_s": full_map_seconds(fixed, per)},
               "direct_nside256": {"value": 12 * 256 * 256 / t256 / 1e9, "unit": "Gpix/s", "seconds": t256,
                                   "what": "one whole Nside-256 map, lmax 512, measured end to end"},
               "sample_max_rel_err_vs_gpu": worst}

    line = {"metric": METRIC, "value": value, "unit": "Gpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (operator contraction: f16 hi/lo pairs on tcgen05, f32 accumulation)",
            "data": "synthetic",
            "config": config_dict(), "roofline": roof, "roofline_stages": per_stage, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": (hp.lib().hpx_plan_launches(plan.handle) + 1) * args.steps, "clocks": clk, "fp64_single_map": fp64, "sh_synthesis_fp32": synthesis, "ablation_cg_latitude_solve": cg,
            "sweeps_path": sweeps, "uneven_batch_200": uneven, "differentiation_nside2048x8": diffw,
            "healpix_software_analysis": healpix_sw,
            "fp32_batched_over_fp64_single": value / world / fp64["value"],
            "stages_ms_per_launch": per_launch, "plan_build_s": plan_build_s, "plan_gb": plan.nbytes / 1e9,
            "plan_path": "sweeps" if plan.flags & hp.HPX_FLAG_SWEEPS else "per-order operators",
            "launch_shapes": {"ring_fft_elems_per_thread": plan.tuning[0], "grid_fft_elems_per_thread": plan.tuning[1],
                              "b_packing": "own pass" if plan.tuning[3] else "in the grid-FFT kernel",
                              "bluestein_rings": "four quarter-length transforms" if plan.tuning[4] else "whole ring"}}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
