#!/usr/bin/env python
"""Benchmark of the extended-correlation hot path on GB300.

Workload (one step = one image through the whole path): rotation-independent
pattern matching on a 2048 x 2048 float32 image (Gaussian noise sigma 0.1 plus
20 planted 65 x 65 templates), filter = the template's angular band-limit
|k| <= 16, sweep over 64 uniformly spaced angles, output = per-pixel maximum
score (float32) and argmax angle index (int32).

Metric: Mpx/s of the whole path (R2C FFT, 17 component correlations through
inverse FFTs, angular sweep with max/argmax).  Filter spectra are built once
per plan (warm-up) and reused, like any fixed-template matcher.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With --gpus N > 1 (launched by torch.distributed.run) every rank processes its
own image per step (independent problems, no collective on the data path) and
rank 0 prints the whole-job throughput over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "extended-correlation Mpx/s at K=16 vs plain FP32 path; HBM/TC % of peak"
WORKLOAD = "so2 pattern matching: 2048x2048 f32, 20 planted 65x65 templates, K=16, 64 angles, max+argmax"


def headline_config(n):
    """The workload keys shared by the GPU line and the reference line."""
    return {"workload": WORKLOAD, "parallelism": f"replicas{n}",
            "l2": "inputs cold each step: the GPU arm writes a 256 MB buffer (> 129 MB L2) between timed steps"}
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=2048)
    ap.add_argument("--cpu-sample", type=int, default=65536, help="pixels in the oracle's timed sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-timed", action="store_true",
                    help="plan, warm-up and timed steps only (for ncu launch lists)")
    ap.add_argument("--so3-size", type=int, default=128,
                    help="so3 / so3p: volume side (128 is the workload; smaller only for profiling captures)")
    ap.add_argument("--so3-L", type=int, default=6,
                    help="so3conv: filter degree (6 is the workload; lower only for profiling captures)")
    ap.add_argument("--train-steps", type=int, default=6000,
                    help="so3p: Adam steps of the proposal network (setup, not timed)")
    ap.add_argument("--workload", default="so2",
                    choices=["so2", "conv", "conv_batched", "scale", "batched", "so3", "so3p", "ght", "lic", "defocus", "budget",
                             "so3conv", "similarity"],
                    help="so2: the pattern-matching sweep, 2048x2048, K=16, 64 angles (default, the headline metric); "
                         "conv: SO(2) extended convolution of a 256x256 image, K=4; "
                         "conv_batched: 512 such images (own angle fields) per step in one captured graph; "
                         "scale: scale-adaptive smoothing of a 4096x4096x3 image, 24 Mellin harmonics; "
                         "defocus: depth-defocus blur of a 2048x2048x3 image, 64 Mellin harmonics; "
                         "lic: normalised convolution (line integral convolution) of a 2048x2048 image; "
                         "ght: pattern detection (gradient field, consensus filter, convolution), 2048x2048; "
                         "budget: sweeps over 5 and 9 of the 17 components, chosen by energy or lowest order; "
                         "batched: 512 uneven images in one captured graph; "
                         "so3: 128^3 volume, L=6, 4608-rotation sweep; "
                         "so3p: the same with the learned proposal; "
                         "so3conv: SO(3) extended convolution of a 128^3 volume, L=6, smooth rotation field; "
                         "similarity: smoothing of a 2048x2048x3 image under joint rotation and scale fields")
    ap.add_argument("--n-images", type=int, default=512)
    ap.add_argument("--simil-shape", default="2048x2048",
                    help="similarity: image rows x columns (2048x2048 is the workload; smaller only for profiling)")
    ap.add_argument("--scale-shape", default="4096x4096",
                    help="scale: image rows x columns (4096x4096 is the workload; smaller only for profiling captures)")
    return ap.parse_args()


# ------------------------------------------------------------------ peaks ---
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def committed_traffic():
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu
    summary (profiles/traffic.txt: '<kernel> <workload> <bytes>' lines)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    out = {}
    try:
        for line in open(path):
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, wl, b = line.split()[:3]
            out[(k, wl)] = float(b)
    except OSError:
        pass
    return out


# ----------------------------------------------------------------- clocks ---
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.file.flush()
        rows = []
        try:
            with open(self.file.name) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        finally:
            os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------- distributed ---
def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"   # gloo: the host-side tests on CPU
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_throughput(world, steps, units_per_rank_step, max_ms):
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (in millions of units per second)."""
    return world * steps * units_per_rank_step / (max_ms * 1e-3) / 1e6


def reduce_max(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------- oracle timings ---
def cpu_model():
    """The host CPU's model name (x86 'model name', else the Arm part code)."""
    import platform
    try:
        text = open("/proc/cpuinfo").read()
    except OSError:
        text = ""
    for key in ("model name", "Model name", "Hardware"):
        for line in text.splitlines():
            if line.startswith(key) and ":" in line:
                return line.split(":", 1)[1].strip()
    parts = {line.split(":", 1)[1].strip() for line in text.splitlines() if line.startswith("CPU part")}
    impl = {line.split(":", 1)[1].strip() for line in text.splitlines() if line.startswith("CPU implementer")}
    if parts:
        return f"{platform.machine()} (CPU implementer {','.join(sorted(impl))}, part {','.join(sorted(parts))})"
    return platform.machine() or "unknown"


_ORACLE_STATE = {}


def _oracle_worker_init(H, tab, radius, J, bank):
    _ORACLE_STATE.update(H=H, tab=tab, radius=radius, J=J, bank=bank)


def _oracle_worker_sweep(pix):
    from oracle.so2 import sweep_so2_at
    st = _ORACLE_STATE
    S = sweep_so2_at(st["H"], st["tab"], st["radius"], st["J"], pix, bank=st["bank"]).real
    return len(pix), float(S.max())


class OraclePool:
    """The FP64 brute-force sweep (the oracle as it stands) over all host
    cores: one spawned worker per core, each single-threaded, each holding the
    image, the decomposed filter and the bank of J rotated filters (built once,
    the filter setup; the per-pixel sums are what is timed)."""

    def __init__(self, prob, cores=None):
        import multiprocessing as mp
        from oracle.filters_so2 import decompose_sampled
        from oracle.so2 import rotated_filter_bank
        self.prob = prob
        self.cores = cores or os.cpu_count() or 1
        tab = decompose_sampled(prob["template"], prob["K"], prob["dr"], prob["n_theta"])
        bank = rotated_filter_bank(tab, prob["radius"], prob["J"])
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(
                self.cores, initializer=_oracle_worker_init,
                initargs=(prob["H"].astype("float64"), tab, prob["radius"], prob["J"], bank))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.pool.map(_oracle_worker_sweep, [self._pixels(16, s) for s in range(self.cores)])   # warm every worker

    def _pixels(self, n, seed):
        import numpy as np
        h, w = self.prob["H"].shape
        rng = np.random.default_rng(seed)
        return np.stack([rng.integers(0, h, n), rng.integers(0, w, n)], 1)

    def time(self, n_pix, seed=0):
        """Wall seconds for the sweep at n_pix random pixels, split over the workers."""
        import numpy as np
        pix = self._pixels(n_pix, seed)
        chunks = np.array_split(pix, self.cores * 4)
        t0 = time.perf_counter()
        self.pool.map(_oracle_worker_sweep, chunks)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def time_fft_steered(prob):
    """The labelled second CPU number: the whole image by the paper's own FFT
    route in FP64 (K + 1 component correlations through SciPy's FFT on all
    cores, linear combination at every angle, max/argmax)."""
    from oracle.filters_so2 import decompose_sampled
    from oracle.so2 import sweep_so2_steered
    tab = decompose_sampled(prob["template"], prob["K"], prob["dr"], prob["n_theta"])
    t0 = time.perf_counter()
    sweep_so2_steered(prob["H"], tab, prob["K"], prob["radius"], prob["J"], workers=-1)
    return time.perf_counter() - t0


def time_oracle(prob, n_pix, seed=0):
    """FP64 brute-force sweep (the oracle as it stands) at n_pix random pixels."""
    import numpy as np
    from oracle.filters_so2 import decompose_sampled
    from oracle.so2 import sweep_so2_at
    tab = decompose_sampled(prob["template"], prob["K"], prob["dr"], prob["n_theta"])
    h, w = prob["H"].shape
    rng = np.random.default_rng(seed)
    pix = np.stack([rng.integers(0, h, n_pix), rng.integers(0, w, n_pix)], 1)
    t0 = time.perf_counter()
    for c in range(0, n_pix, 4096):
        sweep_so2_at(prob["H"], tab, prob["radius"], prob["J"], pix[c:c + 4096])
    return time.perf_counter() - t0


# ----------------------------------------------------------- algorithmic ---
def algorithmic_bytes(kernel, h, w, K, kc):
    """Compulsory DRAM bytes of one launch of each kernel (inputs read once,
    outputs written once), for the launch shapes the sweep path uses."""
    P = h * w
    wh = w // 2 + 1
    half = h * wh * 8
    if kernel == "rows_r2c":
        return 4 * P + half
    if kernel == "cols_fwd_half":   # half spectrum in place, plus the full spectrum for the TMA column pass
        return 2 * half + 8 * P
    if kernel in ("cols_inv_corr", "cols_inv_corr_pipe", "cols_inv_corr_tma"):   # H once, kc spectra in, kc products out
        return half + kc * (8 * P) + kc * (8 * P)
    if kernel in ("rows_inv_components", "rows_inv_components_pipe"):   # kc products in, 2 planes out each
        return kc * 8 * P + kc * 8 * P
    if kernel in ("sweep_fp32", "sweep_bf16x3"):
        return (2 * K + 1) * 4 * P + 8 * P
    return None


# --------------------------------------------------------- conv workload ---
CONV_WORKLOAD = ("SO(2) extended convolution: 256^2 f32 image (blurred uniform noise), analytic filter K=4 "
                 "(a_k r^|k| exp(-r^2/72)), 31x31 box, per-pixel angle field; one image per call")


def bench_conv(args, world, rank, local):
    import numpy as np
    import torch
    import paper_2006_13188_gb300 as ec
    import synth
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    prob = synth.so2_conv_problem(seed=synth.seed_for(1) + rank)
    n = prob["H"].shape[0]
    P = n * n
    plan = ec.Plan(local)
    F = ec.FilterSO2.analytic(prob["a"], prob["sigma"], prob["radius"])
    H = torch.from_numpy(prob["H"]).to(device)
    al = torch.from_numpy(prob["alpha"]).to(device)
    out = torch.empty_like(H)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)

    def call():
        ec.ext_conv_so2(plan, H, n, n, F, al, out)
    call()
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    barrier(world)
    total = 0.0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
    total = reduce_max(total, world, device)
    plan.profile_read()
    plan.profile(True)
    call()
    torch.cuda.synchronize()
    prof = {k: v for k, v in plan.profile_read().items() if v[1] > 0}
    plan.profile(False)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle.filters_so2 import AnalyticGaussPow
        from oracle.so2 import ext_conv_so2_at
        rng = np.random.default_rng(0)
        pix = rng.integers(0, n, (2048, 2))
        t0 = time.perf_counter()
        ext_conv_so2_at(prob["H"].astype(np.float64), AnalyticGaussPow(prob["a"], prob["sigma"]),
                        prob["alpha"].astype(np.float64), prob["radius"], pix)
        t = time.perf_counter() - t0
        cpu = {"value": len(pix) / t / 1e6, "unit": "Mpx/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"FP64 brute-force scatter-form convolution at {len(pix)} random pixels ({t:.1f} s)"}
    if rank == 0:
        print(json.dumps({
            "metric": "SO(2) extended-convolution Mpx/s", "value": world * args.steps * P / (total * 1e-3) / 1e6,
            "unit": "Mpx/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": CONV_WORKLOAD, "l2": "256 MB written between steps",
                       "note": "a single 256^2 image is launch- and latency-bound"},
            "clocks": clk.summary(), "gpu_launches": int(sum(v[1] for v in prof.values())),
            "kernels": {k: {"ms_per_call": v[0], "launches": v[1]} for k, v in prof.items()},
            "cpu_baseline": cpu}))
    plan.close()
    return 0


CONV_BATCH_WORKLOAD = ("SO(2) extended convolution, batched: 512 images of 256^2 f32 (blurred uniform noise), each with "
                       "its own angle field, one analytic filter K=4 (31x31 box); all images per step in one captured "
                       "CUDA graph, calls spread over 8 streams (one plan each)")


def bench_conv_batched(args, world, rank, local):
    import numpy as np
    import torch
    import paper_2006_13188_gb300 as ec
    import synth
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    nimg, nb = args.n_images, 8
    base = synth.seed_for(1) + 1000 * rank
    probs = [synth.so2_conv_problem(seed=base + i) for i in range(nimg)]
    n = probs[0]["H"].shape[0]
    P = n * n
    F = ec.FilterSO2.analytic(probs[0]["a"], probs[0]["sigma"], probs[0]["radius"])   # one filter for the batch
    H = torch.from_numpy(np.stack([p["H"] for p in probs])).to(device)
    al = torch.from_numpy(np.stack([p["alpha"] for p in probs])).to(device)
    out = torch.empty_like(H)
    plans = [ec.Plan(local) for _ in range(nb)]       # one plan (workspace) per stream
    streams = [torch.cuda.Stream(device) for _ in range(nb)]
    for b in range(nb):                                # spectra and workspace built before capture
        ec.ext_conv_so2(plans[b], H[b], n, n, F, al[b], out[b], streams[b])
    torch.cuda.synchronize()

    def body():
        cap = torch.cuda.current_stream()              # the capturing stream inside the graph context
        for b in range(nb):
            streams[b].wait_stream(cap)
        for i in range(nimg):
            b = i % nb
            ec.ext_conv_so2(plans[b], H[i], n, n, F, al[i], out[i], streams[b])
        for b in range(nb):
            cap.wait_stream(streams[b])
    for p in plans:
        p.profile_read()                               # launches recorded into the graph are counted below
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        body()
    torch.cuda.synchronize()
    launches = sum(c for p in plans for _, c in p.profile_read().values())
    main = torch.cuda.current_stream()
    out.zero_()
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    barrier(world)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    total = 0.0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(main)
            g.replay()
            e1.record(main)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
    total = reduce_max(total, world, device)
    errs = cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle.filters_so2 import AnalyticGaussPow
        from oracle.so2 import ext_conv_so2_at
        rng = np.random.default_rng(0)
        got = out.cpu().numpy()
        worst, t_or, n_or = 0.0, 0.0, 0
        for i in range(0, nimg, max(1, nimg // 32)):
            pix = rng.integers(0, n, (16, 2))
            t1 = time.perf_counter()
            ref = ext_conv_so2_at(probs[i]["H"].astype(np.float64), AnalyticGaussPow(probs[0]["a"], probs[0]["sigma"]),
                                  probs[i]["alpha"].astype(np.float64), probs[0]["radius"], pix).real
            t_or += time.perf_counter() - t1
            n_or += len(pix)
            worst = max(worst, float(np.max(np.abs(got[i][pix[:, 0], pix[:, 1]] - ref)) / np.abs(got[i]).max()))
        errs = {"images_checked": len(range(0, nimg, max(1, nimg // 32))), "pixels_per_image": 16,
                "max_error_of_scale": worst}
        cpu = {"value": n_or / t_or / 1e6, "unit": "Mpx/s", "cores": 1, "cpu": cpu_model(), "kind": "oracle",
               "sample": f"FP64 brute-force scatter-form convolution at {n_or} pixels of sampled images"}
    if rank == 0:
        print(json.dumps({
            "metric": "SO(2) extended-convolution Mpx/s (batched)",
            "value": world * args.steps * nimg * P / (total * 1e-3) / 1e6, "unit": "Mpx/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": CONV_BATCH_WORKLOAD, "images": nimg, "l2": "256 MB written between steps"},
            "clocks": clk.summary(), "gpu_launches": launches,
            "errors_vs_oracle": errs, "cpu_baseline": cpu}))
    for p in plans:
        p.close()
    return 0


# --------------------------------------------------------- GHT workload ---
GHT_WORKLOAD = ("pattern detection (Sec. 5 generalised Hough transform): 2048x2048 f32 image (noise 0.05 blurred "
                "sigma 1 + 12 planted 49x49 patterns at random angles); consensus filter eps=22 (47x47 box), K=16; "
                "per step: gradient signal and field, extended convolution")


def bench_ght(args, world, rank, local):
    import numpy as np
    import torch
    import paper_2006_13188_gb300 as ec
    from paper_2006_13188_gb300 import ght
    import synth
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    prob = synth.ght_problem(seed=synth.seed_for(6) + rank)
    h, w = prob["I"].shape
    P = h * w
    K, eps = 16, 22.0
    r = prob["radius"]
    plan = ec.Plan(local)
    t0 = time.perf_counter()
    filt, _ = ght.consensus_filter(plan, prob["pattern"], (r, r), eps, K)
    I = torch.from_numpy(prob["I"]).to(device)
    out = torch.empty_like(I)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)

    def call():
        ght.detect(plan, I, h, w, filt, out)
    call()
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    barrier(world)
    total = 0.0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
    total = reduce_max(total, world, device)
    plan.profile_read()
    plan.profile(True)
    prof_steps = 5
    for _ in range(prof_steps):
        call()
    torch.cuda.synchronize()
    prof = {k: v for k, v in plan.profile_read().items() if v[1] > 0}
    plan.profile(False)
    # detection check: planted centres whose 7x7 neighbourhood beats every pixel away from all centres
    resp = out.cpu().numpy()
    away = np.ones(resp.shape, bool)
    for cy, cx in prob["centres"]:
        away[max(cy - 3, 0):cy + 4, max(cx - 3, 0):cx + 4] = False
    background = float(resp[away].max())
    peaks = [float(resp[max(cy - 3, 0):cy + 4, max(cx - 3, 0):cx + 4].max()) for cy, cx in prob["centres"]]
    found = sum(p > background for p in peaks)
    # end to end through the C ABI with pinned host buffers (image in, response written in place)
    Ih = torch.from_numpy(prob["I"]).pin_memory()
    oh = torch.empty((h, w), dtype=torch.float32).pin_memory()
    e2e_steps = max(5, min(args.steps, 50))
    ght.detect(plan, Ih, h, w, filt, oh)
    barrier(world)
    t1 = time.perf_counter()
    for _ in range(e2e_steps):
        ght.detect(plan, Ih, h, w, filt, oh)
    e2e_s = reduce_max(time.perf_counter() - t1, world, device)
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_n) = dom
    avg_ms = dom_ms / dom_n
    kc = K + 1
    alg = {"cols_conv": kc * 8 * P * 2 + 8 * P, "cols_conv_tma": kc * 8 * P * 2 + 8 * P,
           "rows_fwd_phase": 8 * P + kc * 8 * P}.get(dom_name)
    peak, peak_kind = measured_peaks()
    achieved = alg / (avg_ms * 1e-3) / 1e9 if alg else None
    roofline = {"kernel": dom_name, "bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                "traffic": committed_traffic().get((dom_name, f"{h}x{w}K{K}")),
                "algorithmic_bytes": alg, "avg_launch_ms": avg_ms,
                "kernels": {k: {"ms_per_step": v[0] / prof_steps, "launches_per_step": v[1] / prof_steps}
                            for k, v in prof.items()}}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle.filters_so2 import decompose_sampled
        from oracle.ght import consensus_filter as cf_ref, consensus_radius, gradient_field
        from oracle.so2 import ext_conv_so2_at
        rng = np.random.default_rng(0)
        pix = rng.integers(0, h, (256, 2))
        t2 = time.perf_counter()
        Hr, Tr = gradient_field(prob["I"])
        fr = decompose_sampled(cf_ref(prob["pattern"], (r, r), eps), K, 0.25, 128)
        ext_conv_so2_at(Hr, fr, Tr, consensus_radius(eps), pix)
        t = time.perf_counter() - t2
        cpu = {"value": len(pix) / t / 1e6, "unit": "Mpx/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"FP64 gradient field of the whole image, consensus filter, brute-force extended "
                         f"convolution at {len(pix)} random pixels ({t:.1f} s)"}
    if rank == 0:
        print(json.dumps({
            "metric": "GHT pattern detection Mpx/s", "value": world * args.steps * P / (total * 1e-3) / 1e6,
            "unit": "Mpx/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (filter FP64)", "data": "synthetic",
            "config": {"workload": GHT_WORKLOAD, "l2": "256 MB written between steps", "plan_ms": plan_ms,
                       "planted_found": f"{found}/{len(prob['centres'])}",
                       "weakest_peak_over_background": min(peaks) / background},
            "clocks": clk.summary(),
            "e2e": {"value": world * e2e_steps * P / e2e_s / 1e6, "unit": "Mpx/s", "h2d_bytes_per_step": 4 * P,
                    "d2h_bytes_per_step": 4 * P, "steps": e2e_steps},
            "gpu_launches": int(sum(v[1] for v in prof.values()) // prof_steps),
            "roofline": roofline, "cpu_baseline": cpu}))
    plan.close()
    return 0


# --------------------------------------------------------- LIC workload ---
LIC_WORKLOAD = ("normalised extended convolution (Sec. 8, Line Integral Convolution): 2048x2048 f32 U[0,1] noise, "
                "low-frequency angle field, anisotropic Gaussian sigma 8 x 1 px sampled on the 49x49 box and "
                "decomposed by the library (K=16, dr 0.25, 128 angles), numerator and denominator")


def bench_lic(args, world, rank, local):
    import numpy as np
    import torch
    import paper_2006_13188_gb300 as ec
    import synth
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    n = 2048
    P = n * n
    rng = np.random.default_rng(synth.seed_for(7) + rank)
    Hn = rng.uniform(0, 1, (n, n)).astype(np.float32)
    an = synth.random_angle_field(synth.seed_for(7) + rank, n, n).astype(np.float32)
    K, R, su, sv = 16, 24, 8.0, 1.0
    tpl = synth.aniso_gauss_template(su, sv, R)   # sampled on the box; decomposed on the GPU
    F = ec.FilterSO2.sampled(tpl, K, 0.25, 128)
    plan = ec.Plan(local)
    H = torch.from_numpy(Hn).to(device)
    al = torch.from_numpy(an).to(device)
    out = torch.empty_like(H)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)

    def call():
        ec.ext_conv_so2_normalized(plan, H, 1, n, n, F, al, out)
    t0 = time.perf_counter()
    call()
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    barrier(world)
    total = 0.0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
    total = reduce_max(total, world, device)
    plan.profile_read()
    plan.profile(True)
    prof_steps = 5
    for _ in range(prof_steps):
        call()
    torch.cuda.synchronize()
    prof = {k: v for k, v in plan.profile_read().items() if v[1] > 0}
    plan.profile(False)
    Hh = torch.from_numpy(Hn).pin_memory()
    ah = torch.from_numpy(an).pin_memory()
    oh = torch.empty((n, n), dtype=torch.float32).pin_memory()
    e2e_steps = max(5, min(args.steps, 50))
    ec.ext_conv_so2_normalized(plan, Hh, 1, n, n, F, ah, oh)
    barrier(world)
    t1 = time.perf_counter()
    for _ in range(e2e_steps):
        ec.ext_conv_so2_normalized(plan, Hh, 1, n, n, F, ah, oh)
    e2e_s = reduce_max(time.perf_counter() - t1, world, device)
    dom_name, (dom_ms, dom_n) = max(prof.items(), key=lambda kv: kv[1][0])
    avg_ms = dom_ms / dom_n
    kc = K + 1
    col = conv_column_bytes(kc, P, 2, dom_n / prof_steps)   # the channel and the denominator
    alg = {"cols_conv_tma": col, "cols_conv": col, "rows_fwd_phase": 8 * P + kc * 8 * P}.get(dom_name)
    peak, peak_kind = measured_peaks()
    achieved = alg / (avg_ms * 1e-3) / 1e9 if alg else None
    roofline = {"kernel": dom_name, "bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                "traffic": committed_traffic().get((dom_name, f"{n}x{n}K{K}")),
                "algorithmic_bytes": alg, "avg_launch_ms": avg_ms,
                "kernels": {k: {"ms_per_step": v[0] / prof_steps, "launches_per_step": v[1] / prof_steps}
                            for k, v in prof.items()}}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle.filters_so2 import decompose_sampled
        from oracle.normalized import normalized_conv_so2_at
        pix = np.random.default_rng(0).integers(0, n, (128, 2))
        t2 = time.perf_counter()
        normalized_conv_so2_at(Hn, decompose_sampled(tpl, K, 0.25, 128), an, R, pix)
        t = time.perf_counter() - t2
        cpu = {"value": len(pix) / t / 1e6, "unit": "Mpx/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"FP64 brute-force numerator and denominator at {len(pix)} random pixels ({t:.1f} s)"}
    if rank == 0:
        print(json.dumps({
            "metric": "normalised extended convolution (LIC) Mpx/s",
            "value": world * args.steps * P / (total * 1e-3) / 1e6, "unit": "Mpx/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": LIC_WORKLOAD, "l2": "256 MB written between steps", "plan_ms": plan_ms},
            "clocks": clk.summary(),
            "e2e": {"value": world * e2e_steps * P / e2e_s / 1e6, "unit": "Mpx/s", "h2d_bytes_per_step": 8 * P,
                    "d2h_bytes_per_step": 4 * P, "steps": e2e_steps},
            "gpu_launches": int(sum(v[1] for v in prof.values()) // prof_steps),
            "roofline": roofline, "cpu_baseline": cpu}))
    plan.close()
    return 0


# ------------------------------------------------------ budget workload ---
BUDGET_WORKLOAD = ("fixed-budget component selection (Sec. 5 Band-Limiting Revisited): the 2048x2048 sweep workload "
                   "(20 planted 65x65 templates, K=16, 64 angles, BF16x3), budgets of 5 and 9 components chosen by "
                   "lattice energy or as the lowest orders, against the full 17-component sweep")


def bench_budget(args, world, rank, local):
    import numpy as np
    import torch
    import paper_2006_13188_gb300 as ec
    from paper_2006_13188_gb300 import selection
    import synth
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    prob = synth.so2_match_problem(seed=synth.seed_for(2) + rank)
    K, J = prob["K"], prob["J"]
    h, w = prob["H"].shape
    P = h * w
    plan = ec.Plan(local)
    F = ec.FilterSO2.sampled(prob["template"], K, prob["dr"], prob["n_theta"])
    H = torch.from_numpy(prob["H"]).to(device)
    E = ec.ext_filter_so2_energy(plan, F)
    total_e = E[0] + 2 * E[1:].sum()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    full_m = torch.empty((h, w), dtype=torch.float32, device=device)
    full_a = torch.empty((h, w), dtype=torch.int32, device=device)
    ec.ext_corr_so2(plan, H, h, w, F, None, J, full_m, full_a, ec.EXT_PREC_BF16X3)
    torch.cuda.synchronize()
    ref_a = full_a.cpu().numpy()
    pix = [(cy + dy, cx + dx) for cy, cx in prob["centres"] for dy in range(-2, 3) for dx in range(-2, 3)]
    pix = np.array(pix) % np.array([h, w])
    rows = []
    with ClockSampler(local) as clk:
        for budget in (5, 9, K + 1):
            for rule in (("energy", "lowest") if budget <= K else ("all",)):
                ks = selection.select(plan, F, budget) if rule == "energy" else selection.lowest(F, budget)
                mx = torch.empty((h, w), dtype=torch.float32, device=device)
                am = torch.empty((h, w), dtype=torch.int32, device=device)

                def call():
                    ec.ext_corr_so2_subset(plan, H, h, w, F, ks, J, mx, am, ec.EXT_PREC_BF16X3)
                call()
                torch.cuda.synchronize()
                for _ in range(args.warmup):
                    call()
                torch.cuda.synchronize()
                barrier(world)
                t = 0.0
                for _ in range(args.steps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    call()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    t += e0.elapsed_time(e1)
                t = reduce_max(t, world, device)
                a = am.cpu().numpy()
                dropped = sum(2 * E[k] for k in range(1, K + 1) if k not in ks)
                rows.append({"budget": budget, "rule": rule, "components": ks,
                             "mpx_s": world * args.steps * P / (t * 1e-3) / 1e6, "ms_per_step": t / args.steps,
                             "rel_steering_error": float(np.sqrt(dropped / total_e)),
                             "argmax_agreement_image": float((a == ref_a).mean()),
                             "argmax_agreement_templates": float((a[pix[:, 0], pix[:, 1]] == ref_a[pix[:, 0], pix[:, 1]]).mean())})
    if rank == 0:
        head = next(r for r in rows if r["budget"] == 9 and r["rule"] == "energy")
        print(json.dumps({
            "metric": "component-budget sweep Mpx/s (9 of 17 components, chosen by energy)",
            "value": head["mpx_s"], "unit": "Mpx/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 FFT + bf16x3 sweep (f32 accumulate)", "data": "synthetic",
            "config": {"workload": BUDGET_WORKLOAD, "l2": "256 MB written between steps"},
            "clocks": clk.summary(), "budgets": rows, "cpu_baseline": None}))
    plan.close()
    return 0


# ------------------------------------------------------- scale workload ---
DEFOCUS_WORKLOAD = ("depth-defocus smoothing (Sec. 8): 2048x2048x3 f32 wire-frame-like image (600 one-pixel line "
                    "segments), scale field 1 + 7 |Z - Z(p0)| / max from a smooth depth map, radially smoothed disk "
                    "(logistic edge 0.1 in log-radius) with 64 Mellin frequencies, radii 1-16, normalised mode")
SCALE_WORKLOAD = ("scale-adaptive smoothing: 4096x4096x3 f32 Voronoi image, scale field in [1,8] px, "
                  "24 Mellin harmonics, radii 1-64, normalised (unit-integral) mode")


def conv_column_bytes(n_comp, P, n_sig, launches):
    """Algorithmic bytes of one launch of the convolution column pass: the
    steered row transforms (n_comp complex planes of P pixels) of the launch's
    signals, the n_comp filter spectra once, and one complex sum per signal."""
    per = n_sig / max(launches, 1)
    return per * (n_comp * 8 * P + 8 * P) + n_comp * 8 * P


def bench_scale(args, world, rank, local):
    import numpy as np
    import torch
    import paper_2006_13188_gb300 as ec
    import synth
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if args.workload == "defocus":   # Sec. 8 depth defocus: smoothed disk, 64 Mellin frequencies
        d = synth.depth_defocus_problem(seed=synth.seed_for(8) + rank)
        prob = dict(img=d["img"], s=d["s"], c=synth.mellin_disk_coeffs(), log_period=8.0, r_min=1.0, r_max=16.0,
                    centre_tap=1.0)
    else:
        hs, ws_ = (int(v) for v in args.scale_shape.lower().split("x"))
        prob = synth.scale_smoothing_problem(seed=synth.seed_for(3) + rank, size=(hs, ws_))
    img, s, c = prob["img"], prob["s"], prob["c"]
    h, w = s.shape
    P = h * w
    plan = ec.Plan(local)
    H = torch.from_numpy(img).to(device)
    S = torch.from_numpy(s).to(device)
    out = torch.empty_like(H)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream()

    def call():
        ec.ext_conv_scale(plan, H, 3, h, w, c, prob["log_period"], prob["r_min"], prob["r_max"], prob["centre_tap"],
                          S, 2, out)
    t0 = time.perf_counter()
    call()
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    barrier(world)
    plan.profile_read()
    total = 0.0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
    launches = sum(v[1] for v in plan.profile_read().values())
    total = reduce_max(total, world, device)
    value = world * args.steps * P / (total * 1e-3) / 1e6
    plan.profile(True)
    call()
    torch.cuda.synchronize()
    prof = {k: v for k, v in plan.profile_read().items() if v[1] > 0}
    plan.profile(False)
    dom, (dms, dn) = max(prof.items(), key=lambda kv: kv[1][0])
    n_h = len(c)
    # per launch: the column pass reads the n_h steered row transforms of each of its signals and
    # the n_h spectra (once per launch) and writes each signal's sum; the row pass reads H and the
    # (t, wgt) table and writes n_h planes
    col = conv_column_bytes(n_h, P, 4, dn)
    alg = {"cols_conv": col, "cols_conv_tma": col, "rows_fwd_scale": 12 * P + n_h * 8 * P}.get(dom)
    peak, kind = measured_peaks()
    ach = alg / (dms / dn * 1e-3) / 1e9 if alg else None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle.scale import MellinFilter, smooth
        filt = MellinFilter(c, prob["log_period"], prob["r_min"], prob["r_max"], prob["centre_tap"])
        rng = np.random.default_rng(0)
        pix = rng.integers(0, h, (16, 2))
        t0 = time.perf_counter()
        smooth(img, s, filt, mode=2, pixels=pix)
        t = time.perf_counter() - t0
        cpu = {"value": len(pix) / t / 1e6, "unit": "Mpx/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"FP64 gather-form smoothing at {len(pix)} random pixels ({t:.1f} s)"}
    if rank == 0:
        print(json.dumps({
            "metric": ("depth-defocus smoothing Mpx/s" if args.workload == "defocus" else
                       "scale-adaptive smoothing Mpx/s"), "value": value, "unit": "Mpx/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": DEFOCUS_WORKLOAD if args.workload == "defocus" else SCALE_WORKLOAD,
                       "plan_ms": plan_ms, "l2": "256 MB written between steps"},
            "clocks": clk.summary(), "gpu_launches": launches,
            "roofline": {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peak, "peak_kind": kind,
                         "unit": "GB/s", "frac": ach / peak if ach else None, "traffic": None,
                         "kernels": {k: {"ms_per_call": v[0], "launches": v[1]} for k, v in prof.items()}},
            "cpu_baseline": cpu}))
    plan.close()
    return 0


# ----------------------------------------------------- batched workload ---
BATCH_WORKLOAD = ("batched uneven SO(2) correlation sweep: 512 f32 images, sides 128..1024 step 64 (non-square), "
                  "one planted 33..97 px template each, K in {4,8,16}, 32..128 angles, BF16x3 sweep; the templates' "
                  "spectra are built once per plan (plan_ms, setup graph), each step replays one captured graph of "
                  "every image's forward FFT, correlation passes and sweep")


def _batched_oracle_image(task):
    """Oracle scores of one batched image at its sampled pixels (spawned worker)."""
    from oracle.filters_so2 import decompose_sampled
    from oracle.so2 import sweep_so2_at
    H, template, K, dr, n_theta, radius, J, pix = task
    tab = decompose_sampled(template, K, dr, n_theta)
    return sweep_so2_at(H, tab, radius, J, pix).real


def bench_batched(args, world, rank, local):
    import numpy as np
    import torch
    import paper_2006_13188_gb300 as ec
    import synth
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    descs = synth.batched_descriptors(seed=synth.seed_for(4) + rank, n_images=args.n_images)
    items, probs = [], []
    for d in descs:
        prob = synth.batched_image(d)
        F = ec.FilterSO2.sampled(prob["template"], d["K"], prob["dr"], prob["n_theta"])
        H = torch.from_numpy(prob["H"]).to(device)
        mx = torch.empty((d["h"], d["w"]), dtype=torch.float32, device=device)
        am = torch.empty((d["h"], d["w"]), dtype=torch.int32, device=device)
        items.append((H, d["h"], d["w"], F, d["J"], mx, am))
        probs.append(prob)
    P = sum(d["h"] * d["w"] for d in descs)
    plan = ec.Plan(local)
    batch = ec.BatchDescriptors(items)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    t0 = time.perf_counter()
    ec.ext_batch_corr_so2(plan, batch)
    plan.sync()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    for _ in range(args.warmup):
        ec.ext_batch_corr_so2(plan, batch)
    plan.sync()
    barrier(world)
    total = 0.0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ec.ext_batch_corr_so2(plan, batch)
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
    plan.sync()
    total = reduce_max(total, world, device)
    value = world * args.steps * P / (total * 1e-3) / 1e6
    # per-image error against the FP64 oracle: every image, 32 random pixels each, on all host cores
    errs, cpu = None, None
    if rank == 0 and not args.no_cpu_baseline:   # the oracle leg: timed, and compared on the side
        import multiprocessing as mp
        rng = np.random.default_rng(0)
        tasks = []
        for (H, h, w, F, J, mx, am), prob in zip(items, probs):
            pix = np.stack([rng.integers(0, h, 32), rng.integers(0, w, 32)], 1)
            tasks.append((prob["H"], prob["template"], prob["K"], prob["dr"], prob["n_theta"], prob["radius"], J, pix))
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        cores = os.cpu_count() or 1
        try:
            with mp.get_context("spawn").Pool(cores) as pool:
                t1 = time.perf_counter()
                results = pool.map(_batched_oracle_image, tasks, chunksize=4)
                t_or = time.perf_counter() - t1
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        worst, agree, clear_agree, n_clear, n = 0.0, 0, 0, 0, 0
        per_image = []
        for (H, h, w, F, J, mx, am), task, S in zip(items, tasks, results):
            pix = task[-1]
            got = mx.cpu().numpy()[pix[:, 0], pix[:, 1]]
            arg = am.cpu().numpy()[pix[:, 0], pix[:, 1]]
            scale = np.abs(S).max()
            e = float(np.max(np.abs(got - S.max(1))) / scale)
            srt = np.sort(S, axis=1)
            clear = (srt[:, -1] - srt[:, -2]) > 2e-4 * scale
            ok = arg == S.argmax(1)
            per_image.append(e)
            worst = max(worst, e)
            agree += int(ok.sum())
            clear_agree += int(ok[clear].sum())
            n_clear += int(clear.sum())
            n += len(pix)
        errs = {"images_checked": len(items), "pixels_per_image": 32, "max_rel_score_error": worst,
                "median_rel_score_error": float(np.median(per_image)), "argmax_agreement": agree / n,
                "argmax_agreement_outside_2e-4_window": clear_agree / max(1, n_clear)}
        cpu = {"value": n / t_or / 1e6, "unit": "Mpx/s", "cores": cores, "cpu": cpu_model(), "kind": "oracle",
               "sample": f"FP64 brute-force sweep at 32 pixels of every image ({n} pixels, filter decomposition "
                         f"and rotated-filter bank per image included)"}
    if rank == 0:
        print(json.dumps({
            "metric": "batched extended-correlation Mpx/s", "value": value, "unit": "Mpx/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 FFT + bf16x3 sweep", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "images": len(items), "total_px": P, "plan_ms": plan_ms,
                       "l2": "256 MB written between steps"},
            "clocks": clk.summary(), "gpu_launches": "one CUDA graph per step", "errors_vs_oracle": errs,
            "cpu_baseline": cpu}))
    plan.close()
    return 0


# --------------------------------------------------------- SO(3) workload ---
SO3_WORKLOAD = ("SO(3) matching: 128^3 f32 volume (noise 0.1 + 16 planted 17^3 templates), SH degree L=6 "
                "(455 real channels, 231 complex correlations), 4608-rotation grid sweep with max/argmax")


def measured_bf16():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "measured"
    except Exception:
        return 1900.0, 1700.0, "fallback"


def bench_so3(args, world, rank, local):
    import numpy as np
    import torch
    import paper_2006_13188_gb300 as ec
    import synth
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    prob = synth.so3_match_problem(seed=synth.seed_for(5) + rank, size=args.so3_size,
                                     n_plant=16 if args.so3_size >= 128 else 4)
    grid = synth.so3_rotation_grid()
    n = prob["V"].shape[0]
    P = n ** 3
    L = prob["L"]
    plan = ec.Plan(local)
    V = torch.from_numpy(prob["V"]).to(device)
    mx = torch.empty((n, n, n), dtype=torch.float32, device=device)
    am = torch.empty((n, n, n), dtype=torch.int32, device=device)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)

    dirs, n_psi = synth.so3_rotation_grid_factors()

    def call(prec, factored=True):
        # the 4608-rotation grid is 192 directions x 24 in-plane angles: the factored sweep steers the
        # in-plane angle in the GEMM's epilogue; the plain one sweeps the expanded list
        if factored:
            ec.ext_corr_so3_grid(plan, V, n, n, n, prob["tables"], prob["dr"], prob["radius"], dirs, n_psi, mx, am,
                                 prec)
        else:
            ec.ext_corr_so3(plan, V, n, n, n, prob["tables"], prob["dr"], prob["radius"], grid, mx, am, prec)
    t0 = time.perf_counter()
    call(ec.EXT_PREC_BF16X3)
    plan.sync()
    plan_ms = 1e3 * (time.perf_counter() - t0)

    def timed(prec, steps, factored=True):
        for _ in range(args.warmup):
            call(prec, factored)
        plan.sync()
        barrier(world)
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call(prec, factored)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return reduce_max(tot, world, device)
    with ClockSampler(local) as clk:
        total = timed(ec.EXT_PREC_BF16X3, args.steps)
    list_steps = max(1, min(args.steps, 5))
    list_total = timed(ec.EXT_PREC_BF16X3, list_steps, factored=False)
    plain = timed(ec.EXT_PREC_FP32, max(1, min(args.steps, 3)))
    plain_steps = max(1, min(args.steps, 3))
    value = world * args.steps * P / (total * 1e-3) / 1e6
    nch = ec.ext_so3_channels(L)
    burst, sustained, kind = measured_bf16()

    def profile(factored):
        plan.profile_read()
        plan.profile(True)
        call(ec.EXT_PREC_BF16X3, factored)
        plan.sync()
        out = {k: v for k, v in plan.profile_read().items() if v[1] > 0}
        plan.profile(False)
        return out
    prof_list = profile(False)
    prof = profile(True)
    sweep_name = "so3_sweep_ws" if "so3_sweep_ws" in prof_list else "so3_sweep_bf16x3"
    sweep_ms = prof_list.get(sweep_name, (None, 1))[0]
    flops = 3 * 2.0 * P * nch * len(grid)          # three split-BF16 products over the expanded list
    ach = flops / (sweep_ms * 1e-3) / 1e12 if sweep_ms else None
    gms = prof.get("so3_sweep_grid", (None, 1))[0]
    gflops = 3 * 2.0 * P * nch * 16 * len(dirs)    # the factored GEMM: 16 rows per direction
    gach = gflops / (gms * 1e-3) / 1e12 if gms else None
    if rank == 0:
        print(json.dumps({
            "metric": "SO(3) extended-correlation Mvox/s (4608-rotation sweep)", "value": value, "unit": "Mvox/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 FFT + bf16x3 sweep (f32 accumulate)", "data": "synthetic",
            "config": {"workload": SO3_WORKLOAD, "volume_side": n, "plan_ms": plan_ms,
                       "l2": "256 MB written between steps"},
            "clocks": clk.summary(),
            "plain_fp32": {"value": world * plain_steps * P / (plain * 1e-3) / 1e6, "unit": "Mvox/s",
                           "ms_per_step": plain / plain_steps},
            "list_sweep": {"value": world * list_steps * P / (list_total * 1e-3) / 1e6, "unit": "Mvox/s",
                           "ms_per_step": list_total / list_steps,
                           "note": "the same grid swept as the expanded list of 4608 rotations"},
            "roofline": {"kernel": "so3_sweep_grid", "bound": "tensor", "achieved": gach, "peak": burst,
                         "peak_kind": kind + " bf16 burst (one launch of a few ms at full clocks)", "unit": "TFLOP/s",
                         "frac": gach / burst if gach else None,
                         "frac_of_sustained": gach / sustained if gach else None, "traffic": None,
                         "algorithmic_flops": gflops,
                         "note": "the factored GEMM's own work: 3 split products x 2 x 455 channels x 16 rows per "
                                 "direction x 192 directions per voxel; equivalent_tflops counts the expanded "
                                 "4608-rotation GEMM's work in the same time",
                         "equivalent_tflops": flops / (gms * 1e-3) / 1e12 if gms else None,
                         "kernels": {k: {"ms_per_call": v[0], "launches": v[1]} for k, v in prof.items()}},
            "list_sweep_roofline": {"kernel": sweep_name, "bound": "tensor", "achieved": ach, "peak": burst,
                                    "unit": "TFLOP/s", "frac": ach / burst if ach else None,
                                    "frac_of_sustained": ach / sustained if ach else None,
                                    "traffic": (520.055e6 + 4.978e6) * 8 if sweep_name == "so3_sweep_ws" else None,
                                    "traffic_note": "ncu dram read+write of the 64^3 launch (525 MB) scaled by the 8x "
                                                    "voxel tiles of 128^3; A' and B' read once from DRAM",
                                    "algorithmic_flops": flops,
                                    "kernels": {k: {"ms_per_call": v[0], "launches": v[1]}
                                                for k, v in prof_list.items()}}}))
    plan.close()
    return 0


# ---------------------------------------------- SO(3) with the learned proposal ---
SO3P_WORKLOAD = ("SO(3) matching with the learned proposal: 128^3 f32 volume (noise 0.1 + 16 planted 17^3 "
                 "templates), L=6; score bound, refined nuclear-norm bound, MLP 455-256-256-4 (BF16 tensor cores), "
                 "5 FP32 ascent steps, BF16x3 fallback sweep over the 4608-rotation grid")


def bench_so3p(args, world, rank, local):
    import numpy as np
    import torch
    import paper_2006_13188_gb300 as ec
    from paper_2006_13188_gb300 import proposal
    import synth
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    prob = synth.so3_match_problem(seed=synth.seed_for(5) + rank, size=args.so3_size,
                                     n_plant=16 if args.so3_size >= 128 else 4)
    tables, grid = prob["tables"], synth.so3_rotation_grid()
    n = prob["V"].shape[0]
    P = n ** 3
    L = prob["L"]
    C = ec.ext_so3_channels(L)
    plan = ec.Plan(local)
    # training on 64 method-generated volumes with the same filter (setup, not timed)
    t0 = time.perf_counter()
    X, qt, peaks = proposal.training_set(
        plan, synth.so3_training_volumes(synth.seed_for(5) + 1000 + 64 * rank, tables, 64), grid)
    torch.cuda.synchronize()
    label_ms = 1e3 * (time.perf_counter() - t0)
    net = ec.MLP(plan, C, 256)
    net.set_params(synth.mlp_init(11, C, 256))
    steps, batch = max(1, args.train_steps), 512
    r, Q = synth.training_draws(12, X.shape[0], steps, batch)
    t1 = time.perf_counter()
    losses = proposal.train(net, X, qt, L, torch.from_numpy(r).to(device), torch.from_numpy(Q).to(device), steps,
                            batch)
    torch.cuda.synchronize()
    train_ms = 1e3 * (time.perf_counter() - t1)
    bound = 0.5 * float(np.median(peaks))
    V = torch.from_numpy(prob["V"]).to(device)
    sc = torch.empty(P, dtype=torch.float32, device=device)
    qq = torch.empty((P, 4), dtype=torch.float32, device=device)
    gi = torch.empty(P, dtype=torch.int32, device=device)
    mx = torch.empty(P, dtype=torch.float32, device=device)
    am = torch.empty(P, dtype=torch.int32, device=device)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    counts = {}

    def call():
        counts["c"] = ec.ext_corr_so3_propose(plan, V, n, n, n, tables, prob["dr"], prob["radius"], net, grid, bound,
                                              sc, qq, gi, ec.EXT_PREC_BF16X3)

    dirs, n_psi = synth.so3_rotation_grid_factors()

    def exhaustive():   # the same 4608-rotation grid, factored as 192 directions x 24 in-plane angles
        ec.ext_corr_so3_grid(plan, V, n, n, n, tables, prob["dr"], prob["radius"], dirs, n_psi, mx, am,
                             ec.EXT_PREC_BF16X3)
    t0 = time.perf_counter()
    call()
    plan.sync()
    plan_ms = 1e3 * (time.perf_counter() - t0)

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        plan.sync()
        barrier(world)
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return reduce_max(tot, world, device)
    with ClockSampler(local) as clk:
        total = timed(call, args.steps)
    ex_steps = max(1, min(args.steps, 3))
    ex_total = timed(exhaustive, ex_steps)
    value = world * args.steps * P / (total * 1e-3) / 1e6
    # the same call through the public API with host buffers (copies inside the timed region)
    Vh = torch.from_numpy(prob["V"]).pin_memory()
    sch = torch.empty(P, dtype=torch.float32).pin_memory()
    qqh = torch.empty((P, 4), dtype=torch.float32).pin_memory()
    gih = torch.empty(P, dtype=torch.int32).pin_memory()

    def call_host():
        ec.ext_corr_so3_propose(plan, Vh, n, n, n, tables, prob["dr"], prob["radius"], net, grid, bound, sch, qqh, gih,
                                ec.EXT_PREC_BF16X3)
    e2e_total = timed(call_host, max(1, min(args.steps, 5)))
    e2e_steps = max(1, min(args.steps, 5))
    # ablation: the same call without the network (every candidate swept)
    sc0 = torch.empty(P, dtype=torch.float32, device=device)
    gi0 = torch.empty(P, dtype=torch.int32, device=device)
    abl = {}

    def call_plain():
        abl["c"] = ec.ext_corr_so3_propose(plan, V, n, n, n, tables, prob["dr"], prob["radius"], None, grid, bound,
                                           sc0, None, gi0, ec.EXT_PREC_BF16X3)
    abl_steps = max(1, min(args.steps, 3))
    abl_total = timed(call_plain, abl_steps)
    # held-out agreement with the exhaustive judge over the candidate voxels
    exhaustive()
    call()
    plan.sync()
    mxn, scn = mx.cpu().numpy(), sc.cpu().numpy()
    cand = np.isfinite(scn)
    scale = float(np.abs(mxn).max())
    dev_err = (mxn[cand] - scn[cand]) / scale
    agreement = {"candidates": int(cand.sum()), "score_err_le_1e-4": float(np.mean(dev_err <= 1e-4)),
                 "worst_one_sided_err": float(dev_err.max()) if dev_err.size else 0.0,
                 "grid_max_ge_B_kept": bool(np.all(scn[mxn >= bound] >= bound))}
    plan.profile_read()
    plan.profile(True)
    call()
    plan.sync()
    prof = {k: v for k, v in plan.profile_read().items() if v[1] > 0}
    plan.profile(False)
    # dominant kernel of the step and its roofline: the 3D FFT passes and the bound are HBM-bound
    top = max(prof.items(), key=lambda kv: kv[1][0])
    top_name, (top_ms, top_n) = top[0], top[1]
    nub, nc, nf = counts["c"]
    if rank == 0:
        print(json.dumps({
            "metric": "SO(3) matching Mvox/s with the learned proposal", "value": value, "unit": "Mvox/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 FFT + bf16 MLP + f32 refinement + bf16x3 sweep", "data": "synthetic",
            "config": {"workload": SO3P_WORKLOAD, "volume_side": n, "l2": "256 MB written between steps"},
            "plan_ms": plan_ms, "training": {
                "volumes": 64, "rows": int(X.shape[0]), "label_ms": label_ms, "train_ms": train_ms, "steps": steps,
                "loss_per_500_steps": [float(losses[i:i + 500].mean()) for i in range(0, steps, 500)]},
            "bound": bound, "voxels_ub_ge_B": nub, "candidates": nc, "swept": nf,
            "held_out_agreement": agreement,
            "ablation_without_network": {"swept": int(abl["c"][2]), "ms_per_step": abl_total / abl_steps,
                                         "value": world * abl_steps * P / (abl_total * 1e-3) / 1e6,
                                         "unit": "Mvox/s"},
            "clocks": clk.summary(),
            "exhaustive": {"value": world * ex_steps * P / (ex_total * 1e-3) / 1e6, "unit": "Mvox/s",
                           "ms_per_step": ex_total / ex_steps},
            "e2e": {"value": world * e2e_steps * P / (e2e_total * 1e-3) / 1e6, "unit": "Mvox/s",
                    "h2d_bytes_per_step": 4 * P, "d2h_bytes_per_step": 4 * P + 16 * P + 4 * P},
            "gpu_launches": int(sum(v[1] for v in prof.values())),
            "kernels": {k: {"ms_per_call": v[0], "launches": v[1]} for k, v in prof.items()},
            "top_kernel": {"name": top_name, "ms": top_ms, "launches": top_n}}))
    plan.close()
    return 0


# ----------------------------------------------------- SO(3) convolution ---
SO3CONV_WORKLOAD = ("SO(3) extended convolution (Eq. Def-EConv, scatter, component form of Sec. 9): 128^3 f32 volume "
                    "(periodic Gaussian-blurred noise, sigma 1.5), random band-limited filter of SH degree L=6 "
                    "(231 unique (l,a,b) components), box radius 8, smooth per-voxel rotation field (blurred "
                    "4-vector noise, sigma 4, normalised)")


def bench_so3conv(args, world, rank, local):
    import numpy as np
    import torch
    import paper_2006_13188_gb300 as ec
    import synth
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    n = args.so3_size
    P = n ** 3
    prob = synth.so3_conv_problem(seed=synth.seed_for(9) + rank, shape=(n, n, n), L=args.so3_L)
    tables, dr, R = prob["tables"], prob["dr"], prob["radius"]
    plan = ec.Plan(local)
    V = torch.from_numpy(prob["V"]).to(device)
    Q = torch.from_numpy(prob["Q"]).to(device)
    out = torch.empty_like(V)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)

    def call():
        ec.ext_conv_so3(plan, V, n, n, n, tables, dr, R, Q, out)
    t0 = time.perf_counter()
    call()
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    barrier(world)
    total = 0.0
    steps = args.steps
    with ClockSampler(local) as clk:
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
    total = reduce_max(total, world, device)
    if args.only_timed:
        plan.close()
        return 0
    plan.profile_read()
    plan.profile(True)
    prof_steps = 3
    for _ in range(prof_steps):
        call()
    torch.cuda.synchronize()
    prof = {k: v for k, v in plan.profile_read().items() if v[1] > 0}
    plan.profile(False)
    Vh = torch.from_numpy(prob["V"]).pin_memory()
    Qh = torch.from_numpy(prob["Q"]).pin_memory()
    oh = torch.empty((n, n, n), dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(steps, 20))
    ec.ext_conv_so3(plan, Vh, n, n, n, tables, dr, R, Qh, oh)
    barrier(world)
    t1 = time.perf_counter()
    for _ in range(e2e_steps):
        ec.ext_conv_so3(plan, Vh, n, n, n, tables, dr, R, Qh, oh)
    e2e_s = reduce_max(time.perf_counter() - t1, world, device)
    dom_name, (dom_ms, dom_n) = max(prof.items(), key=lambda kv: kv[1][0])
    avg_ms = dom_ms / dom_n
    nc = sum(2 * l * (l + 1) + 1 for l in range(len(tables)))   # unique (l, a, b)
    alg = {"so3c_cols_z_conv_tma": nc * 16 * P + 8 * P, "so3c_cols_z_conv": nc * 16 * P + 8 * P,
           "so3c_rows_x": nc * 16 * P, "so3c_cols_y": nc * 16 * P, "so3c_planes_yx_fwd": nc * 16 * P,
           "so3c_modulate": 20 * P + nc * 8 * P}.get(dom_name)
    peak, peak_kind = measured_peaks()
    achieved = alg / (avg_ms * 1e-3) / 1e9 if alg else None
    roofline = {"kernel": dom_name, "bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                "traffic": committed_traffic().get((dom_name, f"{n}^3L{len(tables) - 1}")),
                "algorithmic_bytes": alg, "avg_launch_ms": avg_ms,
                "kernels": {k: {"ms_per_step": v[0] / prof_steps, "launches_per_step": v[1] / prof_steps}
                            for k, v in prof.items()}}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle.so3 import SHFilter, conv_so3_at
        vox = np.random.default_rng(0).integers(0, n, (120, 3))
        t2 = time.perf_counter()
        conv_so3_at(prob["V"], SHFilter(tables, dr), R, prob["Q"], vox)
        t = time.perf_counter() - t2
        cpu = {"value": len(vox) / t / 1e6, "unit": "Mvox/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"FP64 brute-force scatter sum (filter rotated per input voxel) at {len(vox)} random "
                         f"voxels ({t:.1f} s)"}
    if rank == 0:
        print(json.dumps({
            "metric": "SO(3) extended convolution Mvox/s",
            "value": world * steps * P / (total * 1e-3) / 1e6, "unit": "Mvox/s", "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": total / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": SO3CONV_WORKLOAD, "volume_side": n, "components": nc,
                       "l2": "256 MB written between steps; working set > L2", "plan_ms": plan_ms},
            "clocks": clk.summary(),
            "e2e": {"value": world * e2e_steps * P / e2e_s / 1e6, "unit": "Mvox/s", "h2d_bytes_per_step": 20 * P,
                    "d2h_bytes_per_step": 4 * P, "steps": e2e_steps},
            "gpu_launches": int(sum(v[1] for v in prof.values()) // prof_steps),
            "roofline": roofline, "cpu_baseline": cpu}))
    plan.close()
    return 0


# ------------------------------------------- rotation x scale smoothing ---
SIMIL_WORKLOAD = ("smoothing under joint rotation and scale fields (rotations and isotropic scales, log-polar "
                  "harmonics; Eq. Def-EConv, Sec. 4.1 x Sec. 8): 2048x2048x3 f32 Voronoi image (300 cells), "
                  "low-frequency angle field, smooth scale field in [1, 3], oriented brush A(phi) B(ln r) with "
                  "|k| <= 4 and 8 log-radial harmonics (68 unique harmonics), radii 1-16, normalised with H/s^2 "
                  "(mode 2: 3 channels + denominator)")


def bench_similarity(args, world, rank, local):
    import numpy as np
    import torch
    import paper_2006_13188_gb300 as ec
    import synth
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    hs, ws_ = (int(v) for v in args.simil_shape.lower().split("x"))
    p = synth.similarity_problem(seed=synth.seed_for(10) + rank, size=(hs, ws_))
    C, h, w = p["img"].shape
    P = h * w
    K, nj = p["c"].shape[0] - 1, p["c"].shape[1]
    n_h = (nj + 1) // 2
    nc = n_h + K * nj
    plan = ec.Plan(local)
    img = torch.from_numpy(p["img"]).to(device)
    al = torch.from_numpy(p["alpha"]).to(device)
    sf = torch.from_numpy(p["s"]).to(device)
    out = torch.empty_like(img)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    fargs = (p["c"], p["log_period"], p["r_min"], p["r_max"], p["centre_tap"])

    def call():
        ec.ext_conv_similarity(plan, img, C, h, w, *fargs, al, sf, 2, out)
    t0 = time.perf_counter()
    call()
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - t0)
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    barrier(world)
    total = 0.0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
    total = reduce_max(total, world, device)
    if args.only_timed:
        plan.close()
        return 0
    plan.profile_read()
    plan.profile(True)
    prof_steps = 3
    for _ in range(prof_steps):
        call()
    torch.cuda.synchronize()
    prof = {k: v for k, v in plan.profile_read().items() if v[1] > 0}
    plan.profile(False)
    ih = torch.from_numpy(p["img"]).pin_memory()
    ah = torch.from_numpy(p["alpha"]).pin_memory()
    sh = torch.from_numpy(p["s"]).pin_memory()
    oh = torch.empty((C, h, w), dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))
    ec.ext_conv_similarity(plan, ih, C, h, w, *fargs, ah, sh, 2, oh)
    barrier(world)
    t1 = time.perf_counter()
    for _ in range(e2e_steps):
        ec.ext_conv_similarity(plan, ih, C, h, w, *fargs, ah, sh, 2, oh)
    e2e_s = reduce_max(time.perf_counter() - t1, world, device)
    dom_name, (dom_ms, dom_n) = max(prof.items(), key=lambda kv: kv[1][0])
    avg_ms = dom_ms / dom_n
    col = conv_column_bytes(nc, P, C + 1, dom_n / prof_steps)
    alg = {"cols_conv_tma": col, "cols_conv": col, "rows_fwd_simil": 12 * P + nc * 8 * P}.get(dom_name)
    peak, peak_kind = measured_peaks()
    achieved = alg / (avg_ms * 1e-3) / 1e9 if alg else None
    roofline = {"kernel": dom_name, "bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                "traffic": committed_traffic().get((dom_name, f"{h}x{w}simil{nc}")),
                "algorithmic_bytes": alg, "avg_launch_ms": avg_ms,
                "kernels": {k: {"ms_per_step": v[0] / prof_steps, "launches_per_step": v[1] / prof_steps}
                            for k, v in prof.items()}}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle.similarity import SimilarityFilter, smooth
        pix = np.random.default_rng(0).integers(0, h, (300, 2))
        t2 = time.perf_counter()
        smooth(p["img"], p["alpha"], p["s"], SimilarityFilter(*fargs), 2, pixels=pix)
        t = time.perf_counter() - t2
        cpu = {"value": len(pix) / t / 1e6, "unit": "Mpx/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"FP64 brute-force gather (3 channels and the denominator) at {len(pix)} random pixels "
                         f"({t:.1f} s)"}
    if rank == 0:
        print(json.dumps({
            "metric": "rotation x scale smoothing Mpx/s",
            "value": world * args.steps * P / (total * 1e-3) / 1e6, "unit": "Mpx/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": SIMIL_WORKLOAD, "harmonics": nc, "l2": "256 MB written between steps",
                       "plan_ms": plan_ms},
            "clocks": clk.summary(),
            "e2e": {"value": world * e2e_steps * P / e2e_s / 1e6, "unit": "Mpx/s",
                    "h2d_bytes_per_step": (4 * C + 8) * P, "d2h_bytes_per_step": 4 * C * P, "steps": e2e_steps},
            "gpu_launches": int(sum(v[1] for v in prof.values()) // prof_steps),
            "roofline": roofline, "cpu_baseline": cpu}))
    plan.close()
    return 0


# ------------------------------------------------------------------ main ---
def main():
    args = parse_args()
    world, rank, local = dist_setup(args.gpus)
    if args.workload == "conv" and args.impl == "ours":
        return bench_conv(args, world, rank, local)
    if args.workload == "conv_batched" and args.impl == "ours":
        return bench_conv_batched(args, world, rank, local)
    if args.workload == "ght" and args.impl == "ours":
        return bench_ght(args, world, rank, local)
    if args.workload == "lic" and args.impl == "ours":
        return bench_lic(args, world, rank, local)
    if args.workload == "budget" and args.impl == "ours":
        return bench_budget(args, world, rank, local)
    if args.workload in ("scale", "defocus") and args.impl == "ours":
        return bench_scale(args, world, rank, local)
    if args.workload == "batched" and args.impl == "ours":
        return bench_batched(args, world, rank, local)
    if args.workload == "so3" and args.impl == "ours":
        return bench_so3(args, world, rank, local)
    if args.workload == "so3p" and args.impl == "ours":
        return bench_so3p(args, world, rank, local)
    if args.workload == "so3conv" and args.impl == "ours":
        return bench_so3conv(args, world, rank, local)
    if args.workload == "similarity" and args.impl == "ours":
        return bench_similarity(args, world, rank, local)

    import numpy as np
    import synth

    if args.impl == "reference":
        if rank != 0:
            return 0
        prob = synth.so2_match_problem(size=args.size)
        n_pix = max(256, args.cpu_sample // 4)
        pool = OraclePool(prob)
        for _ in range(args.warmup):
            pool.time(256, seed=1)
        total = 0.0
        for s in range(args.steps):
            total += pool.time(n_pix, seed=100 + s)
        pool.close()
        value = args.steps * n_pix / total / 1e6
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpx/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": headline_config(args.gpus),
            "cpu_baseline": {"value": value, "unit": "Mpx/s", "cores": pool.cores, "cpu": cpu_model(),
                             "kind": "oracle",
                             "sample": f"FP64 brute-force sweep at {n_pix} random pixels of the image per step, "
                                       f"{pool.cores} single-threaded worker processes"},
            "e2e": {"value": value, "unit": "Mpx/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line))
        return 0

    import torch
    import paper_2006_13188_gb300 as ec

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    prob = synth.so2_match_problem(seed=synth.seed_for(2) + rank, size=args.size)
    h = w = args.size
    P = h * w
    K, J = prob["K"], prob["J"]
    plan = ec.Plan(local)
    F = ec.FilterSO2.sampled(prob["template"], K, prob["dr"], prob["n_theta"])
    H = torch.from_numpy(prob["H"]).to(device)
    mx = torch.empty((h, w), dtype=torch.float32, device=device)
    am = torch.empty((h, w), dtype=torch.int32, device=device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)   # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    precision = ec.EXT_PREC_BF16X3
    plan_t0 = time.perf_counter()
    ec.ext_corr_so2(plan, H, h, w, F, None, J, mx, am, precision)
    torch.cuda.synchronize()
    plan_ms = 1e3 * (time.perf_counter() - plan_t0)

    def run_loop(prec, steps, warm):
        for _ in range(warm):
            ec.ext_corr_so2(plan, H, h, w, F, None, J, mx, am, prec)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            ec.ext_corr_so2(plan, H, h, w, F, None, J, mx, am, prec)
            e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        return sum(e0.elapsed_time(e1) for e0, e1 in evs)

    plan.profile_read()   # clear launch counters
    with ClockSampler(local) as clk:
        total_ms = run_loop(precision, args.steps, args.warmup)
    launches = sum(c for _, c in plan.profile_read().values())
    clocks = clk.summary()
    total_ms = reduce_max(total_ms, world, device)
    value = job_throughput(world, args.steps, P, total_ms)
    if args.only_timed:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "Mpx/s", "steps": args.steps,
                              "ms_per_step": total_ms / args.steps, "gpu_launches": launches}))
        plan.close()
        return 0

    # plain FP32 path: the same FFT passes with the CUDA-core FP32 sweep
    plain_ms = reduce_max(run_loop(ec.EXT_PREC_FP32, args.steps, args.warmup), world, device)
    plain = {"value": world * args.steps * P / (plain_ms * 1e-3) / 1e6, "unit": "Mpx/s",
             "ms_per_step": plain_ms / args.steps, "precision": "fp32",
             "speedup_of_value": plain_ms / total_ms}

    # per-kernel times (events around every launch, on the launch stream)
    prof_steps = max(10, min(args.steps, 50))
    plan.profile_read()   # drop the launch counts of the loops above
    plan.profile(True)
    for _ in range(prof_steps):
        flush.zero_()
        ec.ext_corr_so2(plan, H, h, w, F, None, J, mx, am, precision)
    torch.cuda.synchronize()
    prof = {k: v for k, v in plan.profile_read().items() if v[1] > 0 and v[0] > 0}
    plan.profile(False)
    kc = K + 1
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_n) = dom
    avg_ms = dom_ms / dom_n
    alg = algorithmic_bytes(dom_name, h, w, K, kc)
    peak, peak_kind = measured_peaks()
    achieved = alg / (avg_ms * 1e-3) / 1e9 if alg else None
    traffic = committed_traffic().get((dom_name, f"{h}x{w}K{K}"))
    roofline = {"kernel": dom_name, "bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                "unit": "GB/s", "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "algorithmic_bytes": alg, "avg_launch_ms": avg_ms,
                "kernels": {k: {"ms_per_step": v[0] / prof_steps, "launches_per_step": v[1] / prof_steps,
                                "share": v[0] / sum(x[0] for x in prof.values())} for k, v in prof.items()}}

    # end to end through the C ABI with pinned host buffers
    Hh = torch.from_numpy(prob["H"]).pin_memory()
    mxh = torch.empty((h, w), dtype=torch.float32).pin_memory()
    amh = torch.empty((h, w), dtype=torch.int32).pin_memory()
    e2e_steps = max(5, min(args.steps, 50))
    ec.ext_corr_so2(plan, Hh, h, w, F, None, J, mxh, amh, precision)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ec.ext_corr_so2(plan, Hh, h, w, F, None, J, mxh, amh, precision)
    e2e_s = reduce_max(time.perf_counter() - t0, world, device)
    e2e = {"value": world * e2e_steps * P / e2e_s / 1e6, "unit": "Mpx/s", "h2d_bytes_per_step": 4 * P,
           "d2h_bytes_per_step": 8 * P, "steps": e2e_steps}

    cpu = cpu_fft = None
    if rank == 0 and not args.no_cpu_baseline:
        pool = OraclePool(prob)
        t = pool.time(args.cpu_sample)
        pool.close()
        cpu = {"value": args.cpu_sample / t / 1e6, "unit": "Mpx/s", "cores": pool.cores, "cpu": cpu_model(),
               "kind": "oracle",
               "sample": f"FP64 brute-force sweep at {args.cpu_sample} random pixels of the same image ({t:.1f} s, "
                         f"{pool.cores} single-threaded worker processes)"}
        tf = time_fft_steered(prob)
        cpu_fft = {"value": P / tf / 1e6, "unit": "Mpx/s", "cores": os.cpu_count(), "cpu": cpu_model(),
                   "kind": "oracle FFT-steered route (labelled second CPU number)",
                   "sample": f"the whole {h}x{w} image in FP64: 17 SciPy FFT correlations (workers = all cores), "
                             f"linear combination at 64 angles, max/argmax ({tf:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Mpx/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 FFT + bf16x3 sweep (f32 accumulate)",
            "data": "synthetic",
            "config": headline_config(world), "precision": "bf16x3 sweep", "plan_ms": plan_ms,
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
            "cpu_baseline": cpu, "cpu_fft_steered": cpu_fft, "plain_fp32": plain,
        }
        print(json.dumps(line))
    plan.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
