"""Benchmark of the BST filtered-backprojection path on GB300.

One step = BST FBP of the whole workload volume (default: 2048 slices x 2048
angles x 2048 rays FP32 -> 2048^3 FP32 volume, pad factor 2), with inputs
resident in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): by default every rank reconstructs
its own volume of the same size (weak scaling: slices are independent, so the
path shards with no collective on the data path).  --scaling strong instead
splits ONE volume of --slices slices into contiguous whole-pair ranges, one
per rank (the distribution of blocks of slices over GPUs of Sec. 3), again
with no data-path collective.  Either way the timed region is bracketed by
barriers and the slowest rank's time is used.

CPU baseline (`cpu_baseline`, rank 0 at one GPU) and --impl reference: the
FP64 CPU oracle (the plain restatement of the method used by the tests), as
it stands, on all host cores: one spawned single-threaded worker process per
core (capped by the host memory, about 1.5 GB per worker at 2048 rays), each
reconstructing one slice of the same workload, all started together; the
throughput is the slices done divided by the wall time from the common start
to the last finish.  The worker count is reported as `cores`.
"""
from __future__ import annotations

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

METRIC = "BST FBP voxels/s and % HBM roofline at 2048³ FP32 on 1 GB300 vs brute-force BP"
UNIT = "voxels/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


# FP32 ALU peak of GB300: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x max SM clock
def fp32_peak_tflops(sm_mhz: float) -> float:
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def fft_flops(M: int) -> float:
    return 5.0 * M * np.log2(M)


def disk_points(M: int) -> int:
    k = np.arange(M) - M // 2
    return int(np.count_nonzero(k[None, :] ** 2 + k[:, None] ** 2 < (M // 2) ** 2))


def stage_bytes(N: int, V: int, M: int) -> dict:
    """Compulsory DRAM bytes per launch (one slice pair) of each forward
    kernel: its own input read once and its output written once.  The ray
    kernel reads two slices' sinograms and writes Z (V x M complex64); the
    gridding kernel reads Z and writes T (4 ceil(N/4) x M complex64); the row
    kernel reads T and writes two slices' images."""
    z = V * M * 8
    t = 4 * ((N + 3) // 4) * M * 8
    return {0: 2 * V * N * 4 + z, 1: z + t, 2: t + 2 * N * N * 4}


def stage_flops(N: int, V: int, M: int, kb_width: int = 0) -> dict:
    """Algorithmic flops per launch (one slice pair) of each kernel of the
    forward path: conventional 5 M log2 M per complex FFT line, 6 flops per
    weighted spectrum sample, 12 per bilinear gather (three complex lerps),
    2 per kept output sample.  With Kaiser-Bessel gridding of width W the
    gridding stage counts 6 flops per (sample, grid point) pair of the W x W
    footprints (a real weight product and a complex multiply-add) for the
    V (M - 1) polar samples."""
    grid = 12.0 * disk_points(M) if kb_width <= 0 else 6.0 * kb_width * kb_width * V * (M - 1)
    return {
        0: V * (fft_flops(M) + 6.0 * M),
        1: M * fft_flops(M) + grid,
        2: N * fft_flops(M) + 2.0 * N * N * 2,
    }


STAGE_NAMES = {0: "k_ray_fft", 1: "k_grid_col", 2: "k_row_ifft", 3: "k_ss_filter", 4: "k_ss_bp"}

# DRAM bytes (read + write) per launch of each forward kernel from one ncu
# capture of the dram__bytes_read.sum and dram__bytes_write.sum counters on
# the volume-2048 geometry (16 slices: one launch of 8 pairs each, cold cache), keyed by
# a SHA-256 over the kernels' device-code headers (the host launcher lives in
# another file, so host-only edits keep the record) and by the launch shape
# that the capture ran.  A record applies only while the device code hashes
# to its `sha` and the benchmark runs the same shape; otherwise the roofline
# reports traffic null.
KERNEL_SOURCES = ["paper_1704_08364_gb300/csrc/bst_forward.cuh", "paper_1704_08364_gb300/csrc/bst_stages.cuh",
                  "paper_1704_08364_gb300/csrc/bst_fft.cuh", "paper_1704_08364_gb300/csrc/bst_geo.cuh"]
CAPTURED_TRAFFIC = [
    {"sha": "5182a6ef3146a9c4f464342e17da68624378eacd4d1d37d661da52193c60e7df",
     "rays": 2048, "pad": 2,
     "shape": {"layout": "paired", "chunk_pairs": 8, "pair_fast": 1, "max_radix": 16, "grid_xchg": 1},
     "bytes": {"k_ray_fft": 271184896 + 476406272, "k_grid_col": 629041664 + 486836480,
               "k_row_ifft": 536912640 + 237447424}},
]


def device_code_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def captured_traffic(kernel: str, rays: int, pad: int, shape: dict):
    """Stored DRAM bytes per launch of `kernel` for this geometry and launch
    shape, or None when no capture of the current device code matches."""
    sha = device_code_sha()
    keys = ("layout", "chunk_pairs", "pair_fast", "max_radix", "grid_xchg")
    for c in CAPTURED_TRAFFIC:
        if (c["sha"] == sha and c["rays"] == rays and c["pad"] == pad
                and all(c["shape"][k] == shape[k] for k in keys)):
            return c["bytes"].get(kernel)
    return None


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if len(s) > 3 + i and s[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def _oracle_worker(idx, N, V, alpha, kb_width, barrier, out):
    """One spawned worker: generate its slice, wait for the common start,
    reconstruct it with the FP64 oracle, report the finish time."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    import synth
    from oracle import bst as ob
    from oracle import kb as okb
    theta, sino, _ = synth.workload_slices("volume-2048", [idx], rays=N, angles=V)
    y = sino[0].astype(np.float64)
    barrier.wait()
    if kb_width:
        okb.kb_fbp(y, theta, alpha, width=kb_width)
    else:
        ob.fbp(y, theta, alpha)
    out.put(time.time())


def oracle_workers(N: int) -> int:
    """Worker processes for the oracle timing: every host core, capped so that
    the workers (about 1.5 GB each at 2048 rays, scaling with N^2) fit in half
    of the available host memory."""
    cores = os.cpu_count() or 1
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError, AttributeError):
        return cores
    per = max(1.6e9 * (N / 2048.0) ** 2, 5e7)
    return max(1, min(cores, int(0.5 * avail / per)))


class OraclePool:
    """Times the FP64 oracle on `workers` slices reconstructed concurrently by
    as many spawned single-threaded processes (spawned, never forked, so that
    a CUDA context of the parent is not inherited)."""

    def __init__(self, N: int, V: int, alpha: int = 2, kb_width: int = 0, workers: int | None = None):
        self.N, self.V, self.alpha, self.kb_width = N, V, alpha, kb_width
        self.workers = workers or oracle_workers(N)

    def run(self) -> float:
        """Wall seconds from the common start to the last worker's finish."""
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        barrier = ctx.Barrier(self.workers + 1)
        out = ctx.Queue()
        procs = [ctx.Process(target=_oracle_worker, args=(i, self.N, self.V, self.alpha, self.kb_width,
                                                          barrier, out)) for i in range(self.workers)]
        for p in procs:
            p.start()
        barrier.wait()
        t0 = time.time()
        finish = [out.get() for _ in procs]
        for p in procs:
            p.join()
        if any(p.exitcode != 0 for p in procs):
            raise RuntimeError("an oracle worker failed")
        return max(finish) - t0

    def sample(self) -> str:
        g = f"kaiser-bessel W={self.kb_width}" if self.kb_width else "bilinear"
        return (f"{self.workers} slices of {self.N}x{self.N} ({self.V} angles, pad {self.alpha}, {g}) of the same "
                f"workload, one per worker process, reconstructed concurrently by the FP64 numpy oracle")


L2_BYTES = 126 << 20   # GB300 L2 (about 129 MB)


def rank_slices(args, rank: int, world: int) -> tuple[int, int]:
    """[start, stop) of the workload's slices that this rank reconstructs per
    step: the whole volume (weak scaling) or its contiguous whole-pair share of
    one volume (strong scaling)."""
    if args.scaling == "strong" and world > 1:
        from paper_1704_08364_gb300.shard import slice_range
        return slice_range(rank, world, args.slices)
    return 0, args.slices


def workload_config(args, world: int) -> dict:
    """The `config` of the JSON line, the same for both arms."""
    N = V = args.rays
    S, alpha = args.slices, args.pad
    kbw = args.kb_width if args.gridding == "kb" else 0
    strong = args.scaling == "strong" and world > 1
    per_gpu = (S + world - 1) // world if strong else S
    return {"workload": f"volume-{N} ({S} slices x {V} angles x {N} rays FP32, pad {alpha}, M={alpha * N})",
            "gridding": f"kaiser-bessel W={kbw}" if kbw else "bilinear",
            "slices_per_gpu": per_gpu,
            "l2": ("inputs (%.1f GiB) larger than L2" if per_gpu * V * N * 4 > L2_BYTES else
                   "inputs (%.3f GiB) fit in L2: no flush between steps") % (per_gpu * V * N * 4 / 2**30),
            "parallelism": (f"slices, {world} GPU(s), one volume split in whole-pair ranges" if strong else
                            f"slices, {world} GPU(s), one volume per GPU")}


def link_probe(h_a, h_b, dev, nbytes: int = 1 << 30) -> dict:
    """Host-link rates (GB/s) with pinned buffers: upload alone, download
    alone, and both at once on two streams (per direction), best of three."""
    import torch
    n = min(nbytes // 4, h_a.numel(), h_b.numel())
    ha, hb = h_a.view(-1)[:n], h_b.view(-1)[:n]
    da = torch.empty(n, dtype=torch.float32, device=dev)
    db = torch.empty(n, dtype=torch.float32, device=dev)
    s1, s2 = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def best(fn):
        ts = []
        for _ in range(3):
            torch.cuda.synchronize()
            t = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t)
        return 4 * n / min(ts) / 1e9

    def both():
        with torch.cuda.stream(s1):
            da.copy_(ha, non_blocking=True)
        with torch.cuda.stream(s2):
            hb.copy_(db, non_blocking=True)

    out = {"h2d_gbs": best(lambda: da.copy_(ha, non_blocking=True)),
           "d2h_gbs": best(lambda: hb.copy_(db, non_blocking=True)), "both_gbs": best(both)}
    del da, db
    return out


def _event_ms(fn, steps, warmup=2):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def bench_ragged(bst, synth, sdev, dev, steps):
    """64 sinograms, rays drawn from {256 ... 2048}, angles = rays, pad 2."""
    import torch
    sizes = synth.ragged_sizes()
    groups = {}
    for i, N in enumerate(sizes):
        groups.setdefault(N, []).append(i)
    plans, sino_g, vol_g = {}, {}, {}
    for N, idx in groups.items():
        plans[N] = bst.Plan(N, synth.uniform_angles(N), 2)
        plans[N].autotune()
        sino_g[N] = sdev.ellipse_volume(synth.WORKLOADS["ragged-64"].index * 10 + N, len(idx), N, N,
                                        noise_frac=0.01, device=dev)
        vol_g[N] = torch.empty((len(idx), N, N), dtype=torch.float32, device=dev)
    pos = {}
    for N, idx in groups.items():
        for k, i in enumerate(idx):
            pos[i] = (N, k)
    sinos = [sino_g[pos[i][0]][pos[i][1]] for i in range(len(sizes))]
    vols = [vol_g[pos[i][0]][pos[i][1]] for i in range(len(sizes))]
    rb = bst.RaggedBatch([plans[N] for N in sizes]).bind(sinos, vols)
    voxels = float(sum(N * N for N in sizes))

    def per_size():
        for N in groups:
            plans[N].fbp(sino_g[N], out=vol_g[N])

    ms_per_size = _event_ms(per_size, steps)
    ms_direct = _event_ms(lambda: rb.run(False), steps)
    ms_graph = _event_ms(lambda: rb.run(True), steps)
    ok = rb.status() == 0
    rb.bind(sinos, vols, flags=2)
    ms_overlap = _event_ms(lambda: rb.run(True), steps)
    ok = ok and rb.status() == 0
    return {"items": len(sizes), "pair_items": rb.pair_items, "voxels": voxels,
            "tuned": {str(N): plans[N].forward_config for N in sorted(plans)},
            "per_size_ms": ms_per_size, "persistent_ms": ms_direct, "persistent_graph_ms": ms_graph,
            "persistent_overlapped_order_graph_ms": ms_overlap,
            "persistent_graph_voxels_per_s": voxels / (ms_graph / 1e3), "status_ok": ok}


def bench_autograd(bst, synth, dev, steps):
    """Loss ||FBP(p; g) - f||^2 over 16 slices x 1024 angles x 1024 rays with a
    learnable 1024-tap filter (init ramp): forward + backward per step."""
    import torch
    N = V = 1024
    theta, p, imgs = synth.workload_slices("autograd-1024", list(range(16)), with_images=True, supersample=1)
    plan = bst.Plan(N, theta, 2)
    sino = torch.from_numpy(p).to(dev)
    f = torch.from_numpy(imgs.astype(np.float32)).to(dev)
    g = torch.ones(N, device=dev, requires_grad=True)
    sino.requires_grad_(True)

    def step():
        g.grad = None
        sino.grad = None
        x = bst.fbp_autograd(sino, g, plan)
        loss = ((x - f) ** 2).sum()
        loss.backward()

    ms = _event_ms(step, steps)
    return {"workload": "autograd-1024 (16 x 1024 x 1024, 1024 taps)", "fwd_bwd_ms": ms,
            "voxels_per_s": 16 * N * N / (ms / 1e3)}


def bench_pad1(bst, theta, sino, vol, steps, hbm_peak):
    """The same volume at pad factor 1 (M = N): a quarter of the gridded points
    and half the FFT length, at lower accuracy near the field-of-view edge."""
    S, V, N = sino.shape
    plan = bst.Plan(N, theta, 1)
    tuned = plan.autotune()
    plan.fbp(sino, out=vol)
    ms = _event_ms(lambda: plan.fbp(sino, out=vol), steps)
    alg = 4.0 * (V * N + N * N) * S
    return {"pad": 1, "M": plan.M, "tuned_forward_config": tuned, "ms_per_step": ms,
            "voxels_per_s": S * N * N / (ms / 1e3),
            "path_hbm_frac": alg / (ms / 1e3) / 1e9 / hbm_peak}


def stage_avg_us(plan, fn, steps, names=("k_ray_fft", "k_grid_col", "k_row_ifft")):
    """Average device time per launch of the three forward kernels (the
    library's per-launch events, single stream)."""
    import ctypes
    from paper_1704_08364_gb300 import _lib
    L = _lib.load()
    L.bst_plan_set_timing(plan._h, 1)
    for _ in range(steps):
        fn()
    sms = (ctypes.c_double * 8)()
    sl = (ctypes.c_longlong * 8)()
    L.bst_plan_timing(plan._h, sms, sl, 8)
    L.bst_plan_set_timing(plan._h, 0)
    return {names[i]: 1e3 * sms[i] / max(sl[i], 1) for i in range(3)}


def bench_kb(bst, theta, sino, vol, steps):
    """The same volume with Kaiser-Bessel gridding in P5 (W = 6) at pad factors
    2 and 1: the spread + column FFT kernel replaces the bilinear gather."""
    S, V, N = sino.shape
    out = {}
    for pad in (2, 1):
        plan = bst.Plan(N, theta, pad)
        plan.set_gridding("kaiser-bessel", 6)
        run = lambda: plan.fbp(sino, out=vol)
        run()
        ms = _event_ms(run, steps)
        out[f"pad{pad}"] = {"M": plan.M, "width": 6, "ms_per_step": ms, "voxels_per_s": S * N * N / (ms / 1e3),
                            "stage_avg_us": stage_avg_us(plan, run, 2, ("k_ray_fft", "k_kb_col", "k_row_ifft"))}
        del plan
    return out


def run_reference(args, rank, world):
    N = V = args.rays
    if rank != 0:
        return
    kbw = args.kb_width if args.gridding == "kb" else 0
    pool = OraclePool(N, V, args.pad, kbw, min(oracle_workers(N), max(1, args.slices)))
    for _ in range(args.warmup):
        pool.run()
    times = [pool.run() for _ in range(args.steps)]
    per_step = float(np.mean(times))
    value = pool.workers * N * N / per_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": args.scaling, "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.workers, "host_cores": os.cpu_count(),
                         "kind": "oracle", "sample": pool.sample() + " (one such batch per step)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world):
    import torch
    import torch.distributed as dist

    import paper_1704_08364_gb300 as bst
    from paper_1704_08364_gb300 import _lib
    import synth
    from synth import device as sdev

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    N = V = args.rays
    s0, s1 = rank_slices(args, rank, world)
    S = s1 - s0                       # slices this rank reconstructs per step
    total_slices = args.slices if args.scaling == "strong" else world * S
    alpha = args.pad
    theta = synth.uniform_angles(V)
    plan = bst.Plan(N, theta, alpha)
    kbw = args.kb_width if args.gridding == "kb" else 0
    if kbw:
        plan.set_gridding("kaiser-bessel", kbw)
    M = plan.M
    # the launch shape (radix schedule, spectrum layout, chunk, block order)
    # picked by the library's autotuner on a 256 MiB batch of this geometry
    tuned = plan.autotune() if not args.no_tune else plan.forward_config
    # this rank's slices of the workload (the generator seeds each slice by its
    # index; the strong-scaling ranges are regenerated from the same seeds)
    sino = sdev.ellipse_volume(synth.WORKLOADS["volume-2048"].index, S, V, N, noise_frac=0.01, device=dev,
                               first_slice=s0)
    vol = torch.empty((S, N, N), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        plan.fbp(sino, out=vol)
    plan.status()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(dev.index) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(st)
        marks[0].record(st)
        for k in range(args.steps):
            plan.fbp(sino, out=vol)
            marks[k + 1].record(st)
        e1.record(st)
        torch.cuda.synchronize()
        barrier()
    ms = e0.elapsed_time(e1) / args.steps
    step_ms = [marks[k].elapsed_time(marks[k + 1]) for k in range(args.steps)]
    plan.status()
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = total_slices * N * N / (ms / 1e3)

    # end to end through the C-ABI host entry point: the step's input in pinned
    # host memory, uploads / kernels / downloads overlapped in chunks, the
    # volume back in pinned host memory, all inside the timed region.  The
    # host<->device link of this machine is shared with other jobs, so the
    # fastest and slowest step are reported beside the mean.
    e2e = None
    # one 2048-slice volume of pinned host memory per node: with N ranks each
    # rank streams its 1/N share of it
    es = min(args.e2e_slices, S, max(2, (2048 // world) & ~1))
    try:
        h_in = torch.empty((es, V, N), dtype=torch.float32, pin_memory=True)
        h_in.copy_(sino[:es])
        h_out = torch.empty((es, N, N), dtype=torch.float32, pin_memory=True)
        plan.fbp_host(h_in, out=h_out)
        torch.cuda.synchronize()
        barrier()
        per_step = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            t1 = time.perf_counter()
            plan.fbp_host(h_in, out=h_out)
            per_step.append(time.perf_counter() - t1)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        if world > 1:
            t = torch.tensor([dt], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": world * es * N * N / dt, "unit": UNIT, "h2d_bytes_per_step": world * es * V * N * 4,
               "d2h_bytes_per_step": world * es * N * N * 4, "slices": world * es, "ms_per_step": dt * 1e3,
               "best_ms": 1e3 * min(per_step), "worst_ms": 1e3 * max(per_step),
               "api": "bst_fbp_host (pinned host buffers, chunked copy/compute overlap)"}
        # the host link right after: its rates bound e2e from below (the
        # link is shared with other jobs on the node, so it varies by run)
        link = link_probe(h_in, h_out, dev)
        link["floor_ms"] = 1e3 * max(es * V * N * 4, es * N * N * 4) / (link["both_gbs"] * 1e9)
        e2e["link"] = link
        del h_in, h_out
    except Exception as ex:  # pragma: no cover - host memory limits
        e2e = {"value": None, "unit": UNIT, "error": str(ex)[:200]}

    # per-kernel device times over K more steps (events after every launch)
    L = _lib.load()
    import ctypes
    L.bst_plan_set_timing(plan.handle, 1)
    for _ in range(args.steps):
        plan.fbp(sino, out=vol)
    sms = (ctypes.c_double * 8)()
    sl = (ctypes.c_longlong * 8)()
    L.bst_plan_timing(plan.handle, sms, sl, 8)
    L.bst_plan_set_timing(plan.handle, 0)
    stage_ms = {s: sms[s] for s in range(3)}
    stage_n = {s: sl[s] for s in range(3)}
    flops = stage_flops(N, V, M, kbw)
    names = dict(STAGE_NAMES)
    if kbw:
        names[1] = "k_kb_col"
    dom = max(stage_ms, key=lambda s: stage_ms[s])
    # slice pairs per launch: the tuned chunk (the last chunk of a step may be
    # shorter; the average below counts launches, so use whole-step pairs)
    pairs_per_launch = ((S + 1) // 2) / max(stage_n[dom] / max(args.steps, 1), 1)
    avg_ms = stage_ms[dom] / max(stage_n[dom], 1)
    hbm_peak, sm_max, src = _peaks()
    peak_tf = fp32_peak_tflops(sm_max)
    flops = {k: v * pairs_per_launch for k, v in flops.items()}
    achieved_tf = flops[dom] / (avg_ms / 1e3) / 1e12
    traffic = None if kbw else captured_traffic(names[dom], N, alpha, tuned)
    # the bound is whichever floor is higher for this kernel: its algorithmic
    # flops at the FP32 peak, or its compulsory bytes (its own inputs and
    # outputs read or written once) at the HBM peak
    cbytes = stage_bytes(N, V, M)[dom] * pairs_per_launch
    alu_floor_us = flops[dom] / (peak_tf * 1e12) * 1e6
    hbm_floor_us = cbytes / (hbm_peak * 1e9) * 1e6
    if alu_floor_us >= hbm_floor_us:
        roofline = {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                    "frac": achieved_tf / peak_tf}
    else:
        gbs = cbytes / (avg_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak}
    roofline.update({
        "kernel": names[dom], "traffic": traffic, "pairs_per_launch": pairs_per_launch,
        "stage_avg_us_per_pair": {names[s]: 1e3 * stage_ms[s] / max(stage_n[s], 1) / pairs_per_launch
                                  for s in stage_ms},
        "alu_floor_us": alu_floor_us, "hbm_floor_us": hbm_floor_us, "avg_us": avg_ms * 1e3,
        "alu": {"achieved_tflops": achieved_tf, "peak_tflops": peak_tf, "frac": achieved_tf / peak_tf,
                "algorithmic_flops_per_launch": flops[dom],
                "peak_source": "FP32 152 SM x 128 lanes x 2 x %.0f MHz (derived)" % sm_max},
        "hbm": {"compulsory_bytes_per_launch": cbytes, "achieved_gbs": cbytes / (avg_ms / 1e3) / 1e9,
                "peak_gbs": hbm_peak, "frac": cbytes / (avg_ms / 1e3) / 1e9 / hbm_peak,
                "peak_source": f"MEASURED_PEAKS hbm_gbs ({src})"},
        "dram_gbs": None if traffic is None else traffic / (avg_ms / 1e3) / 1e9,
        "dram_frac_of_hbm_peak": None if traffic is None else traffic / (avg_ms / 1e3) / 1e9 / hbm_peak,
        "traffic_note": "DRAM bytes per launch from one cold-cache ncu capture of the current device code "
                        "(null if it changed since)",
        "stage_share": {names[s]: stage_ms[s] / max(sum(stage_ms.values()), 1e-9) for s in stage_ms},
        "stage_avg_us": {names[s]: 1e3 * stage_ms[s] / max(stage_n[s], 1) for s in stage_ms}})
    alg_bytes = 4.0 * (V * N + N * N) * S
    path_hbm = {"algorithmic_bytes_per_step": alg_bytes, "achieved_gbs": alg_bytes / (ms / 1e3) / 1e9,
                "peak_gbs": hbm_peak, "frac": alg_bytes / (ms / 1e3) / 1e9 / hbm_peak, "peak_source": src}

    # brute-force slant stack on a slice subset, extrapolated per slice
    bs = min(args.brute_slices, S)
    out_b = torch.empty((bs, N, N), dtype=torch.float32, device=dev)
    plan.brute_backproject(sino[:bs], out=out_b)
    torch.cuda.synchronize()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(st)
    plan.brute_backproject(sino[:bs], out=out_b)
    b1.record(st)
    torch.cuda.synchronize()
    brute_ms_per_slice = b0.elapsed_time(b1) / bs
    bst_ms_per_slice = ms / S

    # the ragged batch: 64 sinograms of mixed sizes, one persistent launch
    # (direct and replayed from a CUDA graph) vs plain per-size launches
    ragged = autograd = pad1 = kbg = None
    if not args.no_extras and world == 1:
        pad1 = bench_pad1(bst, theta, sino, vol, args.steps, hbm_peak)
        kbg = bench_kb(bst, theta, sino, vol, args.steps)
        ragged = bench_ragged(bst, synth, sdev, dev, args.steps)
        autograd = bench_autograd(bst, synth, dev, args.steps)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        pool = OraclePool(N, V, alpha, kbw)
        t = pool.run()
        cpu = {"value": pool.workers * N * N / t, "unit": UNIT, "cores": pool.workers,
               "host_cores": os.cpu_count(), "kind": "oracle", "seconds": t, "sample": pool.sample()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "median_step_ms": statistics.median(step_ms),
            "higher_is_better": True, "scaling": args.scaling,
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args, world),
            "slices_per_s": total_slices / (ms / 1e3),
            "roofline": roofline, "path_hbm": path_hbm,
            "vs_brute": {"brute_ms_per_slice": brute_ms_per_slice, "bst_ms_per_slice": bst_ms_per_slice,
                         "speedup": brute_ms_per_slice / bst_ms_per_slice, "brute_slices_timed": bs},
            "clocks": clk.summary(), "e2e": e2e,
            "gpu_launches": 3 * (((S + 1) // 2 + tuned["chunk_pairs"] - 1) // tuned["chunk_pairs"]) * args.steps,
            "tuned_forward_config": tuned,
            "pad1": pad1, "kb_gridding": kbg, "ragged": ragged, "autograd": autograd,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rays", type=int, default=2048)
    ap.add_argument("--slices", type=int, default=2048)
    ap.add_argument("--pad", type=int, default=2)
    ap.add_argument("--brute-slices", type=int, default=64)
    ap.add_argument("--e2e-slices", type=int, default=2048)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the ragged-batch and autograd lines")
    ap.add_argument("--gridding", default="bilinear", choices=["bilinear", "kb"],
                    help="interpolation kernel of stage P5 for the main step (kb: Kaiser-Bessel)")
    ap.add_argument("--kb-width", type=int, default=6)
    ap.add_argument("--no-tune", action="store_true", help="keep the plan's default launch shape")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="with several GPUs: one volume per GPU (weak) or one volume split over the GPUs (strong)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
