"""Benchmark: 512^3 complex-to-complex 3D FFT on one GB300.

One step is the paper's timing protocol (Section 5: a forward and an inverse
transform back to back, reported per transform) on a 512^3 complex64 array
already resident in HBM.  The line also carries the FP16/BF16-storage form of
the same step (speedup and round-trip error), the roofline of the dominant
kernel, the same metric end to end through the host-buffer entry point, and
the FP64 CPU oracle timed on this host's cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl wsfft|reference]

Under torchrun (N > 1) every rank runs its own independent transforms
(replicas: the single-GPU path has no exchange step); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

N_AXIS = 512
DIMS = (N_AXIS, N_AXIS, N_AXIS)
ELEMS = N_AXIS ** 3
FLOPS = 5.0 * ELEMS * math.log2(ELEMS)  # 5 N log2 N (Section 1)
WORKLOAD = "3D C2C FFT 512x512x512 complex64, forward+inverse per step"
METRIC = "512^3 C2C 3D FFT us per transform (FFT+IFFT)/2"
PAPER_CS2_US = 959.3  # Table 1, 512^3 FP32 on a CS-2 (other hardware: context)
REF_PASSES = 2        # minimum-bytes roofline: 2 passes over the array for 3D


# The sources that define, instantiate and select the superstep kernels of
# the benchmark's complex64 512^3 plan: recorded DRAM counters describe
# those kernels only while these files are unchanged.
KERNEL_SOURCES = ("fft_core.cuh", "pass_kernels.cuh", "pass_launch.cuh", "pass_desc.h", "pass_c32.cu",
                  "wsfft_api.cu", "plan_internal.h")


def source_sha256() -> str:
    """Fingerprint of the kernel sources of the benchmark's plan, to tell
    whether recorded counters still describe the kernels being run."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        f = os.path.join(ROOT, "paper_2209_15040_gb300", "csrc", name)
        h.update(name.encode())
        if os.path.exists(f):
            with open(f, "rb") as fh:
                h.update(b"\1" + fh.read())
        else:
            h.update(b"\0")
    return h.hexdigest()


def kernel_traffic(pass_index: int):
    """DRAM bytes (read + write) of one launch of the given pass, from the
    ncu capture recorded in profiles/traffic.json; None once the kernels
    have changed since that capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    if rec.get("source_sha256") != source_sha256():
        return None
    return rec.get("c32_512_pass%d" % pass_index)


def device_info(dev):
    """GPU name and SM count of the device the bench ran on (None if unknown)."""
    try:
        p = torch.cuda.get_device_properties(dev)
        return {"name": p.name, "sms": p.multi_processor_count}
    except Exception:
        return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, v: float) -> float:
    if world <= 1:
        return v
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.path = os.path.join("/tmp", f"wsfft_clocks_{os.getpid()}.csv")
        try:
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            ident = uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
        except Exception:
            ident = str(device_index)
        self.ident = ident

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.ident, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "10"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    @staticmethod
    def parse(lines, window=None):
        """Median SM clock, max clock and throttle reasons of the samples
        whose timestamp lies in `window` (host seconds since the epoch,
        start and end), or of all samples when none does."""
        from datetime import datetime
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                ts = datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[1]), float(parts[2]),
                             [nm for nm, v in zip(names, parts[4:8]) if v.lower() == "active"]))
            except ValueError:
                continue
        inside = [r for r in rows if window and window[0] - 0.01 <= r[0] <= window[1] + 0.01]
        use = inside or rows
        reasons = sorted({nm for r in use for nm in r[3]})
        return {"sm_mhz": statistics.median(r[1] for r in use) if use else None,
                "sm_max_mhz": max(r[2] for r in use) if use else None,
                "reasons": reasons, "samples": len(use), "samples_in_timed_region": len(inside)}

    def stop(self, window=None):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            out = self.parse(f.readlines(), window)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return out


def oracle_pair(x):
    """One FP64 forward + inverse pair of the oracle on x; seconds."""
    import oracle
    t0 = time.perf_counter()
    y = oracle.fftn(x, sign=-1)
    oracle.fftn(y, sign=+1)
    return time.perf_counter() - t0


def oracle_input(n=N_AXIS):
    from paper_2209_15040_gb300 import inputs
    return inputs.complex_input((n, n, n), 1, "normal", "c32").astype(np.complex128)


def cpu_sample_oracle(reps: int = 3):
    """FP64 CPU oracle at the benchmark size: `reps` forward+inverse pairs of
    the 512^3 transform (about 1-2 s each on 16 cores), median per transform.
    Also returns the oracle's input and its forward transform, for the
    element-by-element check of the GPU path at the same size."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    x = oracle_input()
    times, y_ref = [], None
    for _ in range(reps):
        t0 = time.perf_counter()
        y = oracle.fftn(x, sign=-1)
        oracle.fftn(y, sign=+1)
        times.append(time.perf_counter() - t0)
        if y_ref is None:
            y_ref = y
    us = statistics.median(times) / 2 * 1e6
    rec = {"value": round(us, 1), "unit": "us per 512^3 transform", "cores": oracle.get_threads(),
           "kind": "oracle",
           "sample": f"median of {reps} FP64 forward+inverse pairs at 512^3 (the benchmark size), /2"}
    return rec, x, y_ref


def _errs(got, ref):
    """rel-L2 over all elements (re and im as reals), max-abs, max-abs over the
    largest reference magnitude."""
    d = got - ref
    num = float(np.sqrt(np.sum(d.real ** 2 + d.imag ** 2)))
    den = float(np.sqrt(np.sum(ref.real ** 2 + ref.imag ** 2)))
    mabs = float(np.max(np.abs(d)))
    return {"rel_l2": num / den, "max_abs": mabs, "max_abs_rel": mabs / float(np.max(np.abs(ref)))}


def oracle_per_config(W, dev, stream, reps=3):
    """Part of the CPU-baseline leg: the other configurations of the workload
    family -- 32^3 (uniform[-1,1), seed 0), 128^3, 256^3, 2D 4096^2 and 1D 2^20
    (N(0,1), seed 1; the 1D one on a batch of 2, the same kernels as batch 512)
    -- each run once forward on the GPU and compared element by element with
    the FP64 oracle's forward of the same bytes; the oracle's time per
    transform (best of `reps`) on the host cores beside it."""
    import oracle
    from paper_2209_15040_gb300 import inputs
    oracle.set_threads(len(os.sched_getaffinity(0)))
    cases = [((32, 32, 32), 1, 0, "uniform"), ((128, 128, 128), 1, 1, "normal"),
             ((256, 256, 256), 1, 1, "normal"), ((4096, 4096), 1, 1, "normal"),
             ((1 << 20,), 2, 1, "normal")]
    parity, times = [], []
    for dims, batch, seed, dist in cases:
        xs = inputs.complex_input((batch,) + dims, seed, dist, "c32")
        xc = xs.astype(np.complex128)
        xd = torch.from_numpy(np.ascontiguousarray(xs)).to(dev)
        yd = torch.empty_like(xd)
        p = W.Plan(dims, W.C32, W.FORWARD, batch)
        p.execute(xd.data_ptr(), yd.data_ptr(), stream)
        torch.cuda.synchronize()
        p.close()
        got = yd.cpu().numpy().astype(np.complex128)
        best, ref = None, None
        for _ in range(reps):
            t0 = time.perf_counter()
            ref = oracle.fftn(xc, rank=len(dims), sign=-1)
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        e = _errs(got, ref)
        parity.append({"dims": list(dims), "batch": batch, "rel_l2": e["rel_l2"], "max_abs": e["max_abs"],
                       "max_abs_rel": e["max_abs_rel"]})
        times.append({"dims": list(dims), "oracle_us_per_transform": round(best / batch * 1e6, 1),
                      "sample": f"best of {reps} FP64 forwards of batch {batch}"})
        del xd, yd
    return parity, times


def parity_512(W, x_c128, y_ref, dev, stream):
    """The GPU forward transform of the oracle's own 512^3 input, element by
    element against the FP64 oracle's forward: complex64 (paper
    normalisation), and FP16 / BF16 storage against the oracle run on the
    16-bit-rounded input with the orthonormal scaling."""
    import oracle
    from paper_2209_15040_gb300 import inputs
    errs = _errs

    out = {}
    xd = torch.from_numpy(x_c128.astype(np.complex64)).to(dev)
    yd = torch.empty_like(xd)
    p = W.Plan(DIMS, W.C32, W.FORWARD, 1)
    p.execute(xd.data_ptr(), yd.data_ptr(), stream)
    torch.cuda.synchronize()
    p.close()
    out["c32"] = errs(yd.cpu().numpy().astype(np.complex128), y_ref)
    del xd, yd
    for name, code, tdt in (("c16f", W.C16F, torch.float16), ("c16bf", W.C16BF, torch.bfloat16)):
        xs = inputs.to_storage(np.stack([x_c128.real, x_c128.imag], axis=-1), name)
        ref = oracle.fftn(inputs.storage_to_c128(xs, name), norm=oracle.NORM_ORTHO)
        if name == "c16f":
            xh = torch.from_numpy(np.ascontiguousarray(xs)).to(dev)
        else:
            xh = torch.from_numpy(np.ascontiguousarray(xs).view(np.int16)).view(torch.bfloat16).to(dev)
        yh = torch.empty_like(xh)
        p = W.Plan(DIMS, code, W.FORWARD, 1)
        p.execute(xh.data_ptr(), yh.data_ptr(), stream)
        torch.cuda.synchronize()
        p.close()
        got = yh.cpu()
        got = got.numpy() if name == "c16f" else got.view(torch.int16).numpy().view(np.uint16)
        out[name] = errs(inputs.storage_to_c128(got, name), ref)
        del xh, yh, ref
    out["note"] = "forward at 512^3 on the oracle's seeded N(0,1) input, every element against the FP64 oracle"
    return out


def run_reference(args, world, rank):
    """The oracle as it stands, on host cores: the reference arm.  Each step
    is one FP64 forward + inverse pair at 512^3, the benchmark's own
    workload (no scaling)."""
    if rank != 0:
        return
    import oracle
    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    n = args.ref_n
    x = oracle_input(n)
    for _ in range(args.warmup):
        oracle_pair(x)
    dt = sum(oracle_pair(x) for _ in range(args.steps))
    us = dt / args.steps / 2 * 1e6
    line = {"metric": METRIC, "value": round(us, 1), "unit": "us", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "dims": [n, n, n], "l2": "input larger than L2"},
            "cpu_baseline": {"value": round(us, 1), "unit": "us", "cores": oracle.get_threads(),
                             "kind": "oracle",
                             "sample": f"each step one FP64 forward+inverse pair at {n}^3, /2"},
            "e2e": {"value": round(us, 1), "unit": "us", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def sizes_leg(W, dev, stream, hbm_peak, steps=20, warmup=3):
    """The other transform sizes of the workload family, each timed like the
    main step ((FFT + IFFT)/2 per execute of the whole batch, data resident,
    CUDA events on the stream): cubes 32^3 (the small configuration:
    latency-bound, three launches), 128^3, 256^3 and 1024^3 (complex64 and
    float16 storage), 2D
    4096 x 4096 and 1D 2^20 x batch 512 (complex64).  GB/s counts one read and
    one write of the array per launch; the minimum-bytes fraction uses 2
    passes for 2D and 3D and 1 for 1D.  Arrays of 16 MiB (128^3) sit in L2:
    no roofline claim there; those sizes are also timed replayed from a
    captured CUDA graph."""
    cases = [((32, 32, 32), 1, W.C32, 8), ((128, 128, 128), 1, W.C32, 8), ((256, 256, 256), 1, W.C32, 8),
             ((1024, 1024, 1024), 1, W.C32, 8), ((1024, 1024, 1024), 1, W.C16F, 4),
             ((4096, 4096), 1, W.C32, 8), ((1 << 20,), 512, W.C32, 8)]
    out = []
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    for dims, batch, code, eb in cases:
        elems = batch * int(np.prod(dims))
        if code == W.C32:
            xs = torch.view_as_complex(torch.randn((elems, 2), generator=g, device=dev)).contiguous()
        else:
            xs = (torch.rand((elems, 2), generator=g, device=dev) * 2 - 1).to(torch.float16)
        ys = torch.empty_like(xs)
        norm = W.NORM_PAPER if code == W.C32 else W.NORM_ORTHO
        f = W.Plan(dims, code, W.FORWARD, batch, norm)
        i = W.Plan(dims, code, W.INVERSE, batch, norm)
        npass = f.passes()[0]
        ms = timed_pairs(f, i, xs, ys, steps, warmup, 1, stream)
        us = ms / steps * 1e3 / 2
        nbytes = elems * eb
        min_passes = 1 if len(dims) == 1 else 2
        rec = {"dims": list(dims), "batch": batch, "dtype": "complex64" if code == W.C32 else "float16 storage",
               "us_per_execute": round(us, 2), "us_per_transform": round(us / batch, 3), "passes_used": npass,
               "gb_per_s": round(npass * 2 * nbytes / (us * 1e-6) / 1e9, 1),
               "gflops": round(5 * elems * np.log2(elems / batch) / (us * 1e-6) / 1e9, 1)}
        if nbytes > 256 * 2 ** 20:
            rec["min_bytes_roofline_frac"] = round(min_passes * 2 * nbytes / (hbm_peak * 1e9) / (us * 1e-6), 4)
        else:
            rec["note"] = "array fits in L2: no roofline claim"
        if nbytes <= 16 * 2 ** 20:
            # launch-bound sizes: the same pair replayed from a captured CUDA graph
            gms = graph_pairs(f, i, xs, ys, steps, warmup)
            rec["graph_us_per_transform"] = round(gms / steps * 1e3 / 2 / batch, 3)
        out.append(rec)
        f.close()
        i.close()
        del xs, ys
        torch.cuda.empty_cache()
    return out


def layouts_leg(W, x, y, stream, us_natural, steps=20, warmup=3):
    """The same 512^3 complex64 step (forward + inverse per transform pair)
    with the spectral side in the other layouts: swapped (the last two axes
    swapped) and the wafer's [n2][n0][n1]; three trips each, like natural
    order."""
    out = {"natural_us": round(us_natural, 2)}
    for name, code in (("swapped", W.LAYOUT_SWAPPED), ("wafer", W.LAYOUT_WAFER)):
        f = W.Plan(DIMS, W.C32, W.FORWARD, 1)
        i = W.Plan(DIMS, W.C32, W.INVERSE, 1)
        f.set_layout(code)
        i.set_layout(code)
        ms = timed_pairs(f, i, x, y, steps, warmup, 1, stream)
        out[name + "_us"] = round(ms / steps * 1e3 / 2, 2)
        f.close()
        i.close()
    return out


def autograd_leg(W, dev, stream, steps=20, warmup=3):
    """The differentiable configuration: batch 8 x 128^3 complex64 (N(0,1)),
    loss = sum |W * FFT3(x)|^2 with W real uniform[0,1) of the same shape;
    one step = forward (transform + loss) and backward (the hand-written
    adjoint transform + torch's elementwise gradient of the loss), timed
    with CUDA events.  Beside it: the forward and adjoint transforms alone."""
    g = torch.Generator(device=dev)
    g.manual_seed(4)
    shape = (8, 128, 128, 128)
    x = torch.view_as_complex(torch.randn(shape + (2,), generator=g, device=dev)).contiguous()
    x.requires_grad_(True)
    w = torch.rand(shape, generator=g, device=dev)

    def step():
        x.grad = None
        y = W.fftn(x, rank=3)
        loss = (w * y).abs().square().sum()
        loss.backward()
        return loss

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    t_step = e0.elapsed_time(e1) / steps * 1e3
    fwd = W.Plan((128, 128, 128), W.C32, W.FORWARD, 8)
    adj = W.Plan((128, 128, 128), W.C32, W.INVERSE, 8, W.NORM_NONE)
    y = torch.empty_like(x.detach())
    xd = x.detach()
    for _ in range(warmup):
        fwd.execute(xd.data_ptr(), y.data_ptr(), stream)
        adj.execute(y.data_ptr(), y.data_ptr(), stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fwd.execute(xd.data_ptr(), y.data_ptr(), stream)
        adj.execute(y.data_ptr(), y.data_ptr(), stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_pair = e0.elapsed_time(e1) / steps * 1e3
    fwd.close()
    adj.close()
    nbytes = 8 * 128 ** 3 * 8
    return {"shape": list(shape), "dtype": "complex64", "us_per_step_fwd_bwd": round(t_step, 2),
            "us_forward_plus_adjoint_transforms": round(t_pair, 2),
            "transforms_gb_per_s_3pass": round(2 * 3 * 2 * nbytes / (t_pair * 1e-6) / 1e9, 1),
            "note": "step includes torch's elementwise loss and its gradient; the 128 MiB batch sits in L2"}


def _ragged_graph_time(plan, ins, outs, dev, stream, reps):
    """Microseconds per replay of the ragged plan's launch captured in a
    CUDA graph (CUDA events on the stream, after warm-up replays)."""
    side = torch.cuda.Stream(dev)
    with torch.cuda.stream(side):
        plan.execute(ins, outs, side)
        side.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            plan.execute(ins, outs, torch.cuda.current_stream())
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps * 1e3


def ragged_leg(W, dev, stream, reps=5):
    """The ragged configuration (256 uneven 3D shapes from seed 4, N(0,1)):
    one persistent launch replayed from a captured CUDA graph, with the
    default tile shapes and after wsfft_autotune, vs one plan execute per
    instance (3 launches each)."""
    from paper_2209_15040_gb300 import inputs
    shapes = inputs.ragged_shapes(256, 4)
    g = torch.Generator(device=dev)
    xs, ys = [], []
    for i, s in enumerate(shapes):
        g.manual_seed(1000 + i)
        xs.append(torch.view_as_complex(torch.randn(tuple(int(v) for v in s) + (2,), generator=g,
                                                    device=dev)).contiguous())
        ys.append(torch.empty_like(xs[-1]))
    elems = int(sum(int(np.prod(s)) for s in shapes))
    ins, outs = [x.data_ptr() for x in xs], [y.data_ptr() for y in ys]
    plan = W.RaggedPlan(shapes, W.C32, W.FORWARD)
    # the default tile shapes and lag, then the autotuned choice (tile shape
    # per axis length, queue lag), each replayed from a captured graph
    t_default = _ragged_graph_time(plan, ins, outs, dev, stream, reps)
    import tempfile
    tune = {}
    with tempfile.TemporaryDirectory() as td:
        prev = os.environ.get("WSFFT_TUNE_CACHE")
        os.environ["WSFFT_TUNE_CACHE"] = os.path.join(td, "tune.jsonl")
        try:
            plan.autotune()
            with open(os.environ["WSFFT_TUNE_CACHE"]) as fh:
                rec = json.loads(fh.read().strip().splitlines()[-1])
            tune = {"shape_select": rec["variants"][0][1], "lag": rec["mode"]}
        finally:
            if prev is None:
                del os.environ["WSFFT_TUNE_CACHE"]
            else:
                os.environ["WSFFT_TUNE_CACHE"] = prev
    t_graph = _ragged_graph_time(plan, ins, outs, dev, stream, reps)
    plans = [W.Plan(tuple(int(v) for v in s), W.C32, W.FORWARD, 1) for s in shapes]
    launches = sum(p.passes()[0] for p in plans)
    def per_instance():
        for p, i, o in zip(plans, ins, outs):
            p.execute(i, o, stream)
    for _ in range(2):
        per_instance()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        per_instance()
    e1.record(stream)
    torch.cuda.synchronize()
    t_inst = e0.elapsed_time(e1) / reps * 1e3
    for p in plans:
        p.close()
    plan.close()
    return {"instances": len(shapes), "elements": elems, "bytes": elems * 8,
            "persistent_graph_us": round(t_graph, 1), "persistent_graph_default_us": round(t_default, 1),
            "autotuned": tune, "per_instance_us": round(t_inst, 1),
            "speedup": round(t_inst / t_graph, 3), "launches_persistent": 1,
            "launches_per_instance": launches,
            "hbm_gbs_3pass_equiv": round(3 * 2 * elems * 8 / (t_graph * 1e-6) / 1e9, 1)}


def run_sweep(args):
    """Batched 1D transforms of length n (the analogue of the paper's
    single-processor pencil experiment, Section 5.1) over 2^27 elements."""
    from paper_2209_15040_gb300 import build as _build
    from paper_2209_15040_gb300 import wsfft as W
    _build.build_library()
    hbm, kind = peaks()
    total = 1 << 27
    for dtype, code, tdt, eb in (("c32", W.C32, None, 8), ("c16f", W.C16F, torch.float16, 4)):
        if tdt is None:
            x = torch.view_as_complex(torch.randn(total, 2, device="cuda")).contiguous()
        else:
            x = torch.randn(total, 2, device="cuda", dtype=tdt)
        y = torch.empty_like(x)
        for lg in range(4, 13):
            n = 1 << lg
            plan = W.Plan((n,), code, W.FORWARD, total // n)
            for _ in range(3):
                plan.execute(x.data_ptr(), y.data_ptr())
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                plan.execute(x.data_ptr(), y.data_ptr())
            e1.record()
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) / args.steps * 1e3
            flops = 5.0 * n * lg * (total // n)
            gbs = 2 * total * eb / (us * 1e-6) / 1e9
            print(json.dumps({"sweep": "batched 1D", "n": n, "batch": total // n, "dtype": dtype,
                              "us": round(us, 1), "gflops": round(flops / (us * 1e-6) / 1e9, 1),
                              "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 3),
                              "peak_kind": kind}), flush=True)
            plan.close()
        del x, y


def run_case(args):
    """A small case for ncu captures: the default plan of one shape, a few
    executes, nothing timed."""
    from paper_2209_15040_gb300 import build as _build
    from paper_2209_15040_gb300 import wsfft as W
    _build.build_library()
    dims = tuple(int(v) for v in args.case.split(","))
    code = {"c32": W.C32, "c16f": W.C16F, "c16bf": W.C16BF}[args.case_dtype]
    if code == W.C32:
        x = torch.view_as_complex(torch.randn(dims + (2,), device="cuda")).contiguous()
    else:
        x = torch.randn(dims + (2,), device="cuda").to(torch.float16 if code == W.C16F else torch.bfloat16)
    y = torch.empty_like(x)
    plan = W.Plan(dims, code, W.FORWARD, 1)
    if args.case_layout != "natural":
        plan.set_layout({"swapped": W.LAYOUT_SWAPPED, "wafer": W.LAYOUT_WAFER}[args.case_layout])
    if args.case_engine is not None:
        plan.set_engine(args.case_engine)
    if args.case_variant:
        plan.set_pass_variant(*(int(v) for v in args.case_variant.split(",")))
    for _ in range(args.case_reps):
        plan.execute(x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    print(json.dumps({"case": list(dims), "dtype": args.case_dtype, "variant": args.case_variant,
                      "engine": args.case_engine, "layout": args.case_layout,
                      "passes": plan.passes()[0], "reps": args.case_reps, "status": plan.sync_status()}))
    plan.close()


def timed_pairs(fwd, inv, x, y, steps, warmup, world, stream):
    for _ in range(warmup):
        fwd.execute(x.data_ptr(), y.data_ptr(), stream)
        inv.execute(y.data_ptr(), y.data_ptr(), stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fwd.execute(x.data_ptr(), y.data_ptr(), stream)
        inv.execute(y.data_ptr(), y.data_ptr(), stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def graph_pairs(fwd, inv, x, y, steps, warmup):
    """The pair of timed_pairs captured once into a CUDA graph and replayed
    `steps` times (CUDA events on the replaying stream): what a caller that
    replays a captured transform pays, without the per-launch host cost."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fwd.execute(x.data_ptr(), y.data_ptr(), s)
        inv.execute(y.data_ptr(), y.data_ptr(), s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        fwd.execute(x.data_ptr(), y.data_ptr())
        inv.execute(y.data_ptr(), y.data_ptr())
    with torch.cuda.stream(s):
        for _ in range(warmup):
            graph.replay()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            graph.replay()
        e1.record(s)
    torch.cuda.synchronize()
    del graph
    return e0.elapsed_time(e1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wsfft", choices=["wsfft", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--ref-n", type=int, default=N_AXIS,
                    help="reference arm: cube edge of its transforms (default: the benchmark's 512; "
                         "smaller only for tests of the launch path)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    ap.add_argument("--no-ragged", action="store_true", help="skip the ragged-batch leg")
    ap.add_argument("--no-sizes", action="store_true", help="skip the other-sizes leg")
    ap.add_argument("--no-autograd", action="store_true", help="skip the differentiable leg")
    ap.add_argument("--case", default=None,
                    help="profiling helper: run the default plan of shape D0,D1,D2 "
                         "--case-reps times (forward, N(0,1) input, storage --case-dtype) and exit")
    ap.add_argument("--case-reps", type=int, default=3)
    ap.add_argument("--case-dtype", default="c32", choices=["c32", "c16f", "c16bf"])
    ap.add_argument("--case-engine", type=int, default=None,
                    help="schedule of the case's plan (wsfft_plan_set_engine: 0..4)")
    ap.add_argument("--case-layout", default="natural", choices=["natural", "swapped", "wafer"],
                    help="spectral layout of the case's plan (wsfft_plan_set_layout)")
    ap.add_argument("--case-variant", default=None,
                    help="PASS,E,TILE: kernel shape of one pass (wsfft_plan_set_pass_variant)")
    ap.add_argument("--sweep", action="store_true",
                    help="batched 1D pencil sweep n = 16..4096 over 2^27 complex elements "
                         "(FP32 and FP16 storage); one JSON line per point, then exit")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.steps < 1:
        ap.error("--steps must be >= 1")
    world, rank, local = dist_init()

    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.case:
        run_case(args)
        return
    if args.sweep:
        run_sweep(args)
        return

    from paper_2209_15040_gb300 import build as _build
    from paper_2209_15040_gb300 import wsfft as W
    _build.build_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    hbm_peak, peak_kind = peaks()

    # inputs: N(0,1) re/im, generated on the device (seeded), 1 GiB > L2
    g = torch.Generator(device=dev)
    g.manual_seed(1 + rank)
    x = torch.randn(DIMS + (2,), generator=g, device=dev, dtype=torch.float32)
    x = torch.view_as_complex(x).contiguous()
    y = torch.empty_like(x)

    fwd = W.Plan(DIMS, W.C32, W.FORWARD, 1)
    inv = W.Plan(DIMS, W.C32, W.INVERSE, 1)
    npass, bytes_exec = fwd.passes()
    launches_per_step = 2 * npass

    # --- timed region: FP32 pairs as a user runs them (CUDA events around the
    # K steps only).  Clock samples: the sampler starts before the warm-up
    # (nvidia-smi takes a while to start) and only the samples stamped inside
    # the timed region count.
    clocks = Clocks(local)
    clocks.start()
    timed_pairs(fwd, inv, x, y, 0, args.warmup, world, stream)  # warm-up, not recorded
    t_region = [time.time(), 0.0]
    ms = timed_pairs(fwd, inv, x, y, args.steps, 0, world, stream)
    t_region[1] = time.time()
    clk = clocks.stop(t_region)
    ms = allmax(world, ms)
    # --- the same K steps again with a pair of CUDA events around every
    # launch on the launching stream: the per-kernel durations of the
    # roofline (the events stop consecutive launches from overlapping under
    # programmatic dependent launch, so this region runs ~2% slower)
    fwd.profile(args.steps * npass)
    inv.profile(args.steps * npass)
    ms_instr = allmax(world, timed_pairs(fwd, inv, x, y, args.steps, 0, world, stream))
    per_launch = fwd.launch_times(args.steps * npass) + inv.launch_times(args.steps * npass)
    fwd.profile(0)
    inv.profile(0)
    ms_per_step = ms / args.steps
    us_per_transform = ms_per_step * 1e3 / 2 / world  # whole job: world ranks in parallel

    # round-trip error of the FP32 path (paper normalisation: inverse of forward)
    fwd.execute(x.data_ptr(), y.data_ptr(), stream)
    inv.execute(y.data_ptr(), y.data_ptr(), stream)
    torch.cuda.synchronize()
    rt32 = float(torch.linalg.vector_norm(y - x) / torch.linalg.vector_norm(x))
    try:
        rt32_max_abs = float((y - x).abs().max())
    except Exception:  # reporting only: never fail the bench over it
        rt32_max_abs = None

    # dominant kernel: pass index with the largest mean time
    pass_ms = [[] for _ in range(npass)]
    for i, t in enumerate(per_launch):
        pass_ms[i % npass].append(t)
    mean_ms = [statistics.mean(v) if v else 0.0 for v in pass_ms]
    dom = int(np.argmax(mean_ms))
    # algorithmic bytes of one launch: its share of the minimum-bytes
    # roofline of a transform (2 passes x read + write of the 1 GiB array,
    # whatever the schedule), i.e. 4 GiB / launches per transform
    min_bytes = REF_PASSES * 2 * ELEMS * 8
    bytes_launch = min_bytes / npass
    achieved = bytes_launch / (mean_ms[dom] * 1e-3) / 1e9
    # the launch's own read + write of the whole array (what it moves)
    io_launch = 2 * ELEMS * 8
    traffic = kernel_traffic(dom)

    # --- FP16 / BF16 storage, same step
    half = {}
    for name, code, tdt in (("c16f", W.C16F, torch.float16), ("c16bf", W.C16BF, torch.bfloat16)):
        xh = torch.view_as_real(x).to(tdt).contiguous()
        yh = torch.empty_like(xh)
        f16 = W.Plan(DIMS, code, W.FORWARD, 1)
        i16 = W.Plan(DIMS, code, W.INVERSE, 1)
        ms16 = allmax(world, timed_pairs(f16, i16, xh, yh, args.steps, args.warmup, world, stream))
        # forward result vs the FP32 path (orthonormal scaling on both)
        f16.execute(xh.data_ptr(), yh.data_ptr(), stream)
        f32o = W.Plan(DIMS, W.C32, W.FORWARD, 1, W.NORM_ORTHO)
        f32o.execute(x.data_ptr(), y.data_ptr(), stream)
        torch.cuda.synchronize()
        yv = torch.view_as_complex(yh.float().contiguous())
        err_fwd = float(torch.linalg.vector_norm(yv - y) / torch.linalg.vector_norm(y))
        i16.execute(yh.data_ptr(), yh.data_ptr(), stream)
        torch.cuda.synchronize()
        xr = torch.view_as_complex(xh.float().contiguous())
        yr = torch.view_as_complex(yh.float().contiguous())
        err_rt = float(torch.linalg.vector_norm(yr - xr) / torch.linalg.vector_norm(xr))
        us16 = ms16 / args.steps * 1e3 / 2 / world
        half[name] = {"us_per_transform": round(us16, 2),
                      "speedup_vs_c32": round(us_per_transform / us16, 3),
                      "rel_l2_fwd_vs_c32_path": err_fwd, "rel_l2_roundtrip": err_rt}
        for p in (f16, i16, f32o):
            p.close()
        del xh, yh

    # --- end to end through the C ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        hx = torch.empty(DIMS, dtype=torch.complex64).pin_memory()
        hx.copy_(x.cpu())
        hy = torch.empty_like(hx).pin_memory()
        for _ in range(2):
            fwd.execute_host(hx.data_ptr(), hy.data_ptr(), stream)
            inv.execute_host(hy.data_ptr(), hy.data_ptr(), stream)
        esteps = max(2, min(args.steps, 10))
        torch.cuda.synchronize()
        barrier(world)
        # each step timed on its own (host clock, synchronised: the copies of
        # one step cannot overlap the next, whose input waits on them anyway);
        # the median is the value, the mean and the extremes go beside it (the
        # host link is shared with the machine's other work)
        step_s = []
        t0 = time.perf_counter()
        for _ in range(esteps):
            ts = time.perf_counter()
            fwd.execute_host(hx.data_ptr(), hy.data_ptr(), stream)
            inv.execute_host(hy.data_ptr(), hy.data_ptr(), stream)
            torch.cuda.synchronize()
            step_s.append(time.perf_counter() - ts)
        barrier(world)
        dt = allmax(world, time.perf_counter() - t0)
        med = allmax(world, statistics.median(step_s))
        lo, hi = allmax(world, min(step_s)), allmax(world, max(step_s))
        # the host link as it ran during this leg (one 1 GiB copy each way,
        # the same pinned buffers): the floor the end-to-end number sits on
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        with torch.cuda.stream(stream):
            x.copy_(hx, non_blocking=True)
            ev[1].record(stream)
            hy.copy_(x, non_blocking=True)
            ev[2].record(stream)
        torch.cuda.synchronize()
        nbytes = ELEMS * 8
        h2d = nbytes / (ev[0].elapsed_time(ev[1]) * 1e-3) / 1e9
        d2h = nbytes / (ev[1].elapsed_time(ev[2]) * 1e-3) / 1e9
        e2e = {"value": round(med * 1e6 / 2 / world, 2), "unit": "us",
               "h2d_bytes_per_step": 2 * ELEMS * 8, "d2h_bytes_per_step": 2 * ELEMS * 8,
               "steps": esteps, "statistic": "median of the per-step times",
               "mean_us": round(dt / esteps * 1e6 / 2 / world, 2),
               "min_us": round(lo * 1e6 / 2 / world, 2), "max_us": round(hi * 1e6 / 2 / world, 2),
               "entry": "wsfft_execute_host (pinned host buffers)",
               "link_h2d_gbs": round(h2d, 1), "link_d2h_gbs": round(d2h, 1),
               "copy_floor_us": round((nbytes / h2d + nbytes / d2h) / 1e3, 1)}
        del hx, hy
        # beside it: one forward call on a batch of 4 arrays in pinned host
        # memory, where the next array's copies in overlap the previous one's
        # copies out (the two directions of the link)
        if world == 1:
            nb = 4
            bx = torch.empty((nb,) + DIMS, dtype=torch.complex64).pin_memory()
            for b in range(nb):
                bx[b].copy_(x.cpu())
            by = torch.empty_like(bx).pin_memory()
            fb = W.Plan(DIMS, W.C32, W.FORWARD, nb)
            fb.execute_host(bx.data_ptr(), by.data_ptr(), stream)
            calls = []
            for _ in range(3):
                ts = time.perf_counter()
                fb.execute_host(bx.data_ptr(), by.data_ptr(), stream)
                calls.append(time.perf_counter() - ts)
            fb.close()
            e2e["batched"] = {"batch": nb, "direction": "forward",
                              "us_per_transform": round(statistics.median(calls) / nb * 1e6, 2),
                              "calls": len(calls), "statistic": "median of the calls, per transform"}
            del bx, by

    sizes = None
    if not args.no_sizes and world == 1:
        sizes = sizes_leg(W, dev, stream, hbm_peak)

    layouts = None
    if not args.no_sizes and world == 1:
        layouts = layouts_leg(W, x, y, stream, us_per_transform)

    grad = None
    if not args.no_autograd and world == 1:
        grad = autograd_leg(W, dev, stream)

    ragged = None
    if not args.no_ragged:
        ragged = ragged_leg(W, dev, stream)

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, x_or, y_or = cpu_sample_oracle()
        parity = parity_512(W, x_or, y_or, dev, stream)
        del x_or, y_or
        cfg_parity, cfg_times = oracle_per_config(W, dev, stream)
        parity["per_config"] = cfg_parity
        cpu["per_config"] = cfg_times

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(us_per_transform, 2), "unit": "us",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_per_step, 4),
            "ms_per_step_with_launch_events": round(ms_instr / args.steps, 4),
            "higher_is_better": False,
            "scaling": "weak", "vs_baseline": round(us_per_transform / PAPER_CS2_US, 4),
            "vs_baseline_note": "value / 959.3 us, the paper's 512^3 FP32 time on a CS-2 (Table 1): context on other hardware",
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "dims": list(DIMS), "dtype": "complex64",
                       "input": "N(0,1) re/im, seeded, device-generated",
                       "l2": "inputs larger than L2 (1 GiB array vs 126 MB L2)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "gflops": round(FLOPS / (us_per_transform * 1e-6) / 1e9 * 1.0, 1),
            "hbm_min_bytes_roofline": {
                "passes": REF_PASSES, "bytes": min_bytes,
                "time_us_at_peak": round(min_bytes / (hbm_peak * 1e9) * 1e6, 1),
                "frac": round(min_bytes / (hbm_peak * 1e9) / (us_per_transform * 1e-6), 4),
                "peak_gbs": hbm_peak, "peak_kind": peak_kind},
            "passes_used": npass,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak,
                         "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                         "traffic": traffic, "kernel": f"pass {dom} of {npass}",
                         "per_pass_ms": [round(v, 4) for v in mean_ms],
                         "timing": "mean CUDA-event time per launch over a second timed region of the same K steps with events around every launch",
                         "bytes_per_launch": int(bytes_launch),
                         "bytes_per_launch_note": "2-pass minimum bytes of a transform / launches per transform",
                         "io_bytes_per_launch": io_launch,
                         "io_gbs": round(io_launch / (mean_ms[dom] * 1e-3) / 1e9, 1),
                         "io_frac": round(io_launch / (mean_ms[dom] * 1e-3) / 1e9 / hbm_peak, 4),
                         "peak_kind": peak_kind},
            "rel_l2_roundtrip_c32": rt32,
            "max_abs_roundtrip_c32": rt32_max_abs,
            "device": device_info(dev),
            "half_storage": half,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
            "paper_cs2_us": PAPER_CS2_US,
        }
        if e2e:
            line["e2e"] = e2e
        if ragged:
            line["ragged_batch"] = ragged
        if sizes:
            line["other_sizes"] = sizes
        if layouts:
            line["spectral_layouts"] = layouts
        if grad:
            line["autograd"] = grad
        if cpu:
            line["cpu_baseline"] = cpu
        if parity:
            line["parity_vs_fp64_oracle"] = parity
        print(json.dumps(line), flush=True)
    for p in (fwd, inv):
        p.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
