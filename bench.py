#!/usr/bin/env python3
"""Kron-STAP throughput benchmark on B300.

One step = the whole per-cell hot path (kstap_fit_project + kstap_detect:
frame scale, exact lag-sum moments, Alg. 2 flip-flop, B / U_B fit, Eq.
KronSTAP projection and velocity bank) over one synthetic 1024 x 1024-cell
frame (p = 3, q = 16, r_b = 3, n = 120, V = 64, 40 dB CNR, 200 targets).

value  : test cells/s with the frame resident in HBM (sum of per-step CUDA
         event times; a 256 MiB L2 flush runs between steps, outside the events)
e2e    : the same metric through the C ABI with the frame in pinned host memory:
         H2D copy + fit + detect + D2H of Tmax / vidx / map inside the events
N > 1  : one rank per GPU, each on its own frame (independent problems, no
         collective on the data path): weak scaling, value = all cells / max time.
--impl reference : the FP64 CPU oracle timed on a bounded sample of the same
         workload's cells (host cores), same metric and unit.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Kron-STAP test cells/s and p50/p99 frame latency on 1 B300, batched vs plain"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kstap", choices=["kstap", "reference"])
    ap.add_argument("--peaks", metavar="PATH",
                    help="measure the arithmetic pipes (FP32 and packed f32x2 FMA, 64-bit "
                         "integer multiply-add, FP64 FMA) with kstap_alu_probe, write their "
                         "peaks to PATH (JSON) and exit")
    ap.add_argument("--workload", default="frame1024")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16x3", "bf16x3"],
                    help="arithmetic of the velocity-bank contraction (fp32: CUDA cores; "
                         "fp16x3 / bf16x3: tensor cores, hi + lo splits)")
    ap.add_argument("--cpu-sample", type=int, default=1024,
                    help="cells of the oracle CPU baseline sample")
    ap.add_argument("--lag-store", type=int, default=1, choices=[0, 1],
                    help="1: the moments pass writes the exact lag sums to a workspace store "
                         "the B pass reads; 0: the B pass recomputes them (no store)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer e2e leg")
    ap.add_argument("--no-robustness", action="store_true",
                    help="skip the SIRV / corrupted-training detection study")
    ap.add_argument("--no-multipass", action="store_true",
                    help="skip the two-pass (p = 6) stacked frame and change map")
    ap.add_argument("--no-paper-timing", action="store_true",
                    help="skip the single large-covariance LR-Kron timing grid")
    ap.add_argument("--no-precision-leg", action="store_true",
                    help="skip the 2048^2 q = 32 frame (FP32 and FP16X3 banks)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-vs-plain leg on the 256-tile workload")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-domain", action="store_true",
                    help="skip the q = 12 / 24 and r_b > 4 frames")
    ap.add_argument("--serve-requests", type=int, default=300,
                    help="requests in the Poisson serving stream")
    ap.add_argument("--cells", type=int, nargs=2, metavar=("H", "W"),
                    help="run the workload's model on an H x W cell grid (profiling cases)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(seed: int, rank: int, s: int) -> int:
    """Seed of frame s of a rank: every rank works on its own frames."""
    return seed + 7919 * rank + s


def max_over_ranks(x: float, ws: int, device=None) -> float:
    """Max of a per-rank time over all ranks (the job is as slow as its
    slowest rank); a barrier-like host collective, not on the data path."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(cells_per_frame: int, steps: int, ws: int, total_ms: float) -> float:
    """Whole-job throughput under weak scaling: each of the ws ranks processed
    `steps` frames of `cells_per_frame` cells in at most total_ms."""
    return cells_per_frame * steps * ws / (total_ms / 1e3)


# ----------------------------------------------------------- reference arm --
def run_reference(args):
    import gen
    import oracle
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    wl = gen.WORKLOADS[args.workload]
    f = gen.make_frame(wl)
    nthr = oracle.num_threads()
    sample = max(64, args.cpu_sample // 4)
    times = []
    for s in range(args.warmup + args.steps):
        cells = gen.random_cells(wl, sample, seed=1000 + s)
        t0 = time.perf_counter()
        oracle.run_workload(f, cells=cells, want_T_all=False, want_proj=False)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = sample * len(times) / total
    line = dict(metric=METRIC, value=value, unit="cells/s", n_gpus=ws, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * total / len(times),
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", impl="reference",
                config=dict(workload=wl.name, cells_per_frame=wl.H * wl.W, q=wl.q, r_b=wl.r_b,
                            n=wl.n, V=wl.V, p=wl.p, sample_cells_per_step=sample),
                cpu_baseline=dict(value=value, unit="cells/s", cores=nthr, kind="oracle",
                                  sample=f"{sample} seeded random cells per step of the "
                                         f"{wl.H}x{wl.W} frame"),
                e2e=dict(value=value, unit="cells/s", h2d_bytes_per_step=0,
                         d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, enabled: bool = True):
        self.index = index
        self.proc = None
        self.path = None
        if enabled:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            try:
                self.fh = open(self.path, "w")
                self.proc = subprocess.Popen(
                    ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                     "-i", str(index), "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
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
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(parts)
            except Exception:
                pass
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return dict(sm_mhz=statistics.median(sm) if sm else None,
                    sm_max_mhz=max(mx) if mx else None, reasons=reasons, samples=len(rows))


# ------------------------------------------------------------- ALU peaks ---
PEAKS_FILE = os.path.join(ROOT, "peaks.json")


def measure_peaks(path: str, seconds: float = 3.0):
    """Throughput of each arithmetic pipe on cuda:0 (kstap_alu_probe), about
    `seconds` of launches per pipe with the SM clock sampled meanwhile; the
    result (ops/s, flop rates, median MHz) is written to `path`."""
    import torch
    import paper_1604_03622_b300 as K
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    out = dict(device=torch.cuda.get_device_name(0), sms=torch.cuda.get_device_properties(0)
               .multi_processor_count, when=time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
               how="kstap_alu_probe: SMs x 8 CTAs x 256 threads, 8 independent chains per "
                   "thread, CUDA events over ~%.0f s of launches per pipe" % seconds)
    for op, iters in (("ffma", 1 << 16), ("ffma2", 1 << 16), ("imad64", 1 << 13),
                      ("dfma", 1 << 10)):
        rate = K.kstap_alu_probe(op, iters, 4, stream)          # warm-up and calibration
        per_launch = (out["sms"] * 8 * 256 * iters * 8 * (2 if op == "ffma2" else 1)) / rate
        reps = max(4, int(seconds / per_launch))
        clk = ClockSampler(0, True)
        rate = K.kstap_alu_probe(op, iters, reps, stream)
        c = clk.stop() or {}
        out[op] = dict(ops_per_s=rate, iters=iters, reps=reps, sm_mhz=c.get("sm_mhz"),
                       sm_max_mhz=c.get("sm_max_mhz"), reasons=c.get("reasons"))
    out["fp32_fma_tflops"] = 2 * max(out["ffma"]["ops_per_s"], out["ffma2"]["ops_per_s"]) / 1e12
    out["fp32_fma_mhz"] = (out["ffma2"] if out["ffma2"]["ops_per_s"] >= out["ffma"]["ops_per_s"]
                           else out["ffma"])["sm_mhz"]
    out["imad64_tops"] = out["imad64"]["ops_per_s"] / 1e12
    out["fp64_fma_tflops"] = 2 * out["dfma"]["ops_per_s"] / 1e12
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out), flush=True)


def alu_peak():
    """(FP32 FMA peak TFLOP/s, the median SM MHz it was measured at, note) from
    peaks.json, else the unit-count figure at the maximum clock."""
    try:
        with open(PEAKS_FILE) as fh:
            pk = json.load(fh)
        mhz = pk.get("fp32_fma_mhz") or 2032.0
        return (float(pk["fp32_fma_tflops"]), float(mhz),
                "measured: FP32 FMA peak of kstap_alu_probe (bench.py --peaks, peaks.json) at "
                "%.0f MHz median SM clock (%s)" % (mhz, pk.get("when", "")))
    except (OSError, KeyError, ValueError):
        return (148 * 128 * 2 * 2032e6 / 1e12, 2032.0,
                "derived: 148 SMs x 128 FP32 lanes x 2 x 2032 MHz (no peaks.json)")


# ------------------------------------------------------------ work model ---
def work_per_cell(wl):
    """Algorithmic arithmetic per cell of each kernel.

    Units: single-precision flops (FMA = 2) for floating point, and integer
    multiply-adds (one 32x32->64 product-accumulate = 2 ops) for the exact
    lag sums; a float-float product-accumulate counts as 2 flops (the flops
    of the exact-arithmetic formula, not of its emulation).
    """
    p, q, rb, V = wl.p, wl.q, wl.r_b, wl.V
    PP = p * p
    NE = PP * (PP + 1) // 2
    NR = 2 * wl.ring_r + 1
    tc = 32 if q < 32 else 16
    # lag sums for one tile of tc cells, all lags g in [0, q): vertical box
    # (NR products per plane and column) + horizontal ring (2Ra+1 + 2Ga+1 adds)
    lag = 0
    for g in range(q):
        nu = tc + q - 1 - g
        kw = nu + 2 * wl.ring_a
        lag += PP * kw * NR * 8 + PP * nu * (2 * wl.ring_a + 1 + 2 * wl.guard_a + 1) * 2
    lag_per_cell = lag / tc
    m_flops = sum(q - g for g in range(q)) * NE * 8
    b_flops = sum(q - g for g in range(q)) * PP * 8
    # eigen phase: one FP32 and one float-float subspace product B V (q^2 r_b
    # complex MACs each; >99.9 % of cells converge after one float-float
    # step) plus the Gram and H products (2 q r_b^2 complex MACs)
    eig_flops = 2 * (q * q * rb * 8) + 2 * (q * rb * rb * 8)
    det_flops = V * (p * q + q * rb + p) * 8 + 2 * p * q * rb * 8
    # the B pass streams the lag sums the moments pass stored: no lag work
    return dict(frame_scale=6.0, moments=lag_per_cell + m_flops, flipflop=6 * (PP * PP * 8),
                bfit=b_flops + eig_flops, detect=det_flops)


# DRAM bytes per launch of a kernel on a workload, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), valid only for the kernel
# sources it was taken on: the bench reports null once either file changes.
KERNEL_SRC = [os.path.join(ROOT, "paper_1604_03622_b300", "csrc", f)
              for f in ("kstap_kernels.cuh", "kstap_ff.cuh")]


def kernel_src_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for path in KERNEL_SRC:
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


TRAFFIC = {
    # 512 x 1024-cell capture (1.262 GB read + 0.389 GB write) x 2 for the 1024^2
    # frame: bfit's traffic is the lag store read once per position plus the
    # per-cell a and U_B hi/lo, so it grows with the cell count
    ("frame1024", "fp32", "bfit"): dict(
        bytes=2 * (1.262305e9 + 0.389270e9),
        # issue slots used (smsp__issue_active) and FMA-pipe activity of the
        # same capture: the kernel's float-float arithmetic costs ~10
        # instructions per algorithmic flop (packed f32x2 pairs issue two
        # lanes at once but hold the FMA pipe for two cycles)
        issue_active=0.607, fma_pipe_active=0.504,
        sha256="32e5dc5619861b04ef509804d53d9da2bf75981946f4ed3531902e00d6f40d5b",
        source="profiles/bfit_frame1024_512x1024.md"),
}


def measured_peak(key: str):
    """A figure of MEASURED_PEAKS.json (measured on this machine), or None."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key])
    except (OSError, KeyError, ValueError):
        return None


def measured_traffic(workload: str, precision: str, kernel: str, key: str = "bytes"):
    t = TRAFFIC.get((workload, precision, kernel))
    if t is None or key not in t:
        return None, None
    if kernel_src_sha256() != t["sha256"]:
        return None, "kernel source changed since the capture"
    return t[key], t["source"]


# ------------------------------------------------------- batched vs plain ---
def class_precision(precision: str, q: int) -> str:
    """Bank arithmetic of one (q, r_b) class: "mixed" takes the tensor-core
    FP16X3 bank at q = 32, where it is faster (32.7 against 49.1 ms on a 2048^2
    frame), and the FP32 bank below, where the packed CUDA-core bank wins."""
    if precision == "mixed":
        return "fp16x3" if q >= 32 else "fp32"
    return precision


MIXED = "mixed (FP16X3 bank at q = 32, FP32 below)"


def batched_leg(dev, steps: int, warmup: int, precision: str = "mixed"):
    """256 uneven tiles (q in {8,16,32}, r_b in {2,3,4}): plain = one tile at a
    time through kstap_fit_project + kstap_detect (5 launches per tile, no
    overlap, FP32 bank); batched = one CUDA graph holding one autotuned batch
    per (q, r_b) class on parallel branches, with the FP32 bank (batching
    alone) and with `precision` (default: the tensor-core bank at q = 32, FP32
    below).  The fits are bit-identical; T agrees to the 16-bit route's bar
    (tested)."""
    import torch
    import gen
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    tiles = gen.tile_batch()
    frames = [gen.make_frame(w) for w in tiles]
    classes = {}
    for i, w in enumerate(tiles):
        classes.setdefault((w.q, w.r_b), []).append(i)
    keys = sorted(classes)
    Ys = [torch.from_numpy(f.Y).to(dev) for f in frames]
    ctxs = {}
    for key in keys:
        w0, f0 = tiles[classes[key][0]], frames[classes[key][0]]
        ctxs[key] = KStap.from_workload(w0, f0.bank_a, f0.bank_b, device=str(dev))
    stream = torch.cuda.current_stream(dev)

    def make_graph(prec):
        """Per-class contexts, output buffers, autotuned tuning and the graph."""
        bctxs, bufs, descs, tuning = {}, {}, {}, {}
        for key in keys:
            idx = classes[key]
            w0, f0 = tiles[idx[0]], frames[idx[0]]
            ks = KStap.from_workload(w0, f0.bank_a, f0.bank_b, device=str(dev),
                                     precision=class_precision(prec, key[0]))
            bctxs[key] = ks
            # the descriptors hold raw device pointers: keep the tensors alive
            bufs[key] = [ks.alloc_outputs(Ys[i].shape[1], Ys[i].shape[2]) for i in idx]
            descs[key] = [ks.frame_desc(Ys[i], b) for i, b in zip(idx, bufs[key])]
            t = K.kstap_autotune(ks.ctx, descs[key], reps=2)
            tuning[f"q{key[0]}_r{key[1]}"] = dict(waves=t.waves, tc=t.tc,
                                                  ms=round(t.ms_per_batch, 3))
        graph = K.kstap_graph_create([bctxs[k].ctx for k in keys], [descs[k] for k in keys])
        return bctxs, bufs, graph, tuning

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ncells = sum(w.cells for w in tiles)

    def timed(fn):
        out = []
        for s in range(warmup + steps):
            flush.fill_(s & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            if s >= warmup:
                out.append(a.elapsed_time(b))
        return out

    def plain():
        for key in keys:
            ks = ctxs[key]
            for i in classes[key]:
                ks.run(Ys[i])

    plain_ms = timed(plain)
    arms, tunings = {}, {}
    for tag, prec in (("batched_fp32", "fp32"), ("batched", precision)):
        bctxs, bufs, graph, tuning = make_graph(prec)
        ms = timed(lambda: K.kstap_graph_launch(graph, stream.cuda_stream))
        K.kstap_graph_destroy(graph)
        for ks in bctxs.values():
            ks.close()
        m = sum(ms) / len(ms)
        arms[tag] = dict(cells_per_s=ncells / (m / 1e3), ms_per_batch=m, p99_ms=sorted(ms)[-1],
                         graph_launches=1, kernel_launches=5 * len(keys),
                         precision=MIXED if prec == "mixed" else prec)
        tunings[tag] = tuning
    for ks in ctxs.values():
        ks.close()
    pm = sum(plain_ms) / len(plain_ms)
    return dict(workload="tiles256", tiles=len(tiles), cells=ncells, classes=len(keys),
                plain=dict(cells_per_s=ncells / (pm / 1e3), ms_per_batch=pm,
                           p99_ms=sorted(plain_ms)[-1], kernel_launches=5 * len(tiles),
                           precision="fp32"),
                **arms, speedup=pm / arms["batched"]["ms_per_batch"],
                speedup_fp32=pm / arms["batched_fp32"]["ms_per_batch"], tuning=tunings)


# --------------------------------------------------------- q = 32 frame ---
def precision_leg(dev, steps: int, warmup: int, err_cells: int = 256, cpu: bool = True):
    """The 2048 x 2048-cell q = 32 frame (p = 3, r_b = 4, n = 192, V = 128,
    40 dB CNR): plain path, per-step CUDA events with an L2 flush between
    steps, with the FP32 bank and with the FP16X3 and BF16X3 tensor-core banks;
    per-kernel times from the library's events; the error of the statistic
    against the FP64 oracle on `err_cells` seeded cells (all V velocities):
    max |T - T_ref| / max(T_ref, sigma^2)."""
    import torch
    import gen
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    wl = gen.WORKLOADS["precision2048"]
    f = gen.make_frame(wl)
    Y = torch.from_numpy(f.Y).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = dict(workload=wl.name, cells_per_frame=wl.cells, q=wl.q, r_b=wl.r_b, n=wl.n, V=wl.V)
    ref = None
    if cpu and err_cells > 0:
        import oracle
        cells = gen.random_cells(wl, err_cells, seed=77)
        ref = oracle.run_workload(f, cells=cells, want_proj=False)
        out["error_sample"] = f"{len(cells)} seeded random cells x {wl.V} velocities (FP64 oracle)"
    for prec in ("fp32", "fp16x3", "bf16x3"):
        ks = KStap.from_workload(wl, f.bank_a, f.bank_b, device=str(dev), stream=stream,
                                 precision=prec)
        for _ in range(warmup):
            ks.run(Y)
        torch.cuda.synchronize(dev)
        K.kstap_set_profiling(ks.ctx, True)
        ms = []
        for s in range(steps):
            flush.fill_(s & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ks.run(Y)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        kt = K.kstap_kernel_times(ks.ctx)
        K.kstap_set_profiling(ks.ctx, False)
        err = None
        if ref is not None:
            T = ks.run(Y, T_all=True)["T_all"][torch.from_numpy(ref["cells"]).to(dev)]
            T = T.double().cpu().numpy()
            err = float((np.abs(T - ref["T_all"]) / np.maximum(ref["T_all"], wl.sigma2)).max())
        ks.close()
        out[prec] = dict(cells_per_s=wl.cells * len(ms) / (sum(ms) / 1e3),
                         ms_per_frame=sum(ms) / len(ms), p99_ms=sorted(ms)[-1],
                         max_rel_err_T=err,
                         kernel_ms_per_launch={k: v[0] / max(v[1], 1) for k, v in kt.items()})
        if prec != "fp32":
            # tensor-pipe roofline of the bank contraction: per cell the GEMM
            # rows are 2 (p + r_b) real operand rows (Re|Im, Im|-Re), K = 2q,
            # V velocities, three 16-bit products (hi hi, hi lo, lo hi)
            det_ms = kt["detect"][0] / max(kt["detect"][1], 1)
            flops = 3 * 2 * wl.V * 2 * (wl.p + wl.r_b) * 2 * wl.q * wl.cells
            peak = measured_peak("bf16_tflops")
            achieved = flops / (det_ms / 1e3) / 1e12
            out[prec]["detect_roofline"] = dict(
                bound="tensor", achieved=achieved, peak=peak, unit="TFLOP/s",
                frac=achieved / peak if peak else None, kernel="detect",
                note="MMA flops of the bank contraction over the whole detect kernel time "
                     "(the projection and epilogue on the CUDA cores dominate it); peak = "
                     "measured dense bf16 burst (fp16 has the same dense rate)")
    del Y, flush
    torch.cuda.empty_cache()
    return out


# ------------------------------------------- the rest of the (q, r_b) domain ---
def domain_leg(dev, steps: int, warmup: int, err_cells: int = 256, cpu: bool = True):
    """Frames of 1024 x 1024 cells at the window lengths and ranks between and
    above the configurations': q = 12 (r_b = 3, n = 72) and q = 24 (r_b = 4,
    n = 144) on the FP32 and FP16X3 banks, and r_b = 8 at q = 16 and r_b = 6 at
    q = 32 (block Rayleigh-Ritz path, FP32 bank); plain path, CUDA events per
    frame with an L2 flush between frames, per-kernel times, and the error of
    T against the FP64 oracle on `err_cells` seeded cells (all velocities)."""
    import dataclasses
    import torch
    import gen
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    cases = [("frame_q12", 3, "fp32"), ("frame_q12", 3, "fp16x3"), ("frame_q24", 4, "fp32"),
             ("frame_q24", 4, "fp16x3"), ("frame1024", 8, "fp32"), ("precision2048", 6, "fp32")]
    rows = []
    for name, r_b, prec in cases:
        wl = dataclasses.replace(gen.WORKLOADS[name], r_b=r_b).with_size(1024, 1024)
        f = gen.make_frame(wl)
        Y = torch.from_numpy(f.Y).to(dev)
        ks = KStap.from_workload(wl, f.bank_a, f.bank_b, device=str(dev), stream=stream,
                                 precision=prec)
        for _ in range(warmup):
            ks.run(Y)
        torch.cuda.synchronize(dev)
        K.kstap_set_profiling(ks.ctx, True)
        ms = []
        for s_ in range(steps):
            flush.fill_(s_ & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ks.run(Y)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        kt = K.kstap_kernel_times(ks.ctx)
        K.kstap_set_profiling(ks.ctx, False)
        err = None
        if cpu and err_cells > 0:
            import oracle
            cells = gen.random_cells(wl, err_cells, seed=78)
            ref = oracle.run_workload(f, cells=cells, want_proj=False)
            T = ks.run(Y, T_all=True)["T_all"][torch.from_numpy(ref["cells"]).to(dev)]
            T = T.double().cpu().numpy()
            ok = ref["gapB"] >= 1e-6
            e = np.abs(T - ref["T_all"]) / np.maximum(ref["T_all"], wl.sigma2)
            err = dict(max_rel_err_T=float(e[ok].max()) if ok.any() else None,
                       cells=int(len(cells)), cells_gap_below_1e_6=int((~ok).sum()))
        ks.close()
        rows.append(dict(workload=wl.name, q=wl.q, r_b=wl.r_b, n=wl.n, V=wl.V, precision=prec,
                         cells_per_s=wl.cells * len(ms) / (sum(ms) / 1e3),
                         ms_per_frame=sum(ms) / len(ms), error=err,
                         kernel_ms_per_launch={k: v[0] / max(v[1], 1) for k, v in kt.items()}))
        del Y
    del flush
    torch.cuda.empty_cache()
    return dict(rows=rows, note="error: max |T - T_ref| / max(T_ref, sigma^2) over the sampled "
                               "cells whose oracle eigengap of B is >= 1e-6")


# --------------------------------------------------- robustness (Sec. 5) ---
def robustness_leg(dev):
    """Detection on synthetic data under the SIRV texture and corrupted
    training (Sec. 2, Sec. 5): a 512 x 512-cell cut of the 1024^2 frame model
    with 400 targets (SNR U(0, 15) dB per element), clean / K-distributed
    texture (nu = 0.5) / two copies of every target in its training ring /
    both, with the Kron-STAP and the classical projector.  Pd = targets with
    Tmax > tau at their cell; Pfa and mean Tmax over cells whose window holds
    no target sample, planted copies included (sigma^2 = 1 is perfect
    cancellation)."""
    import dataclasses
    import torch
    import gen
    from paper_1604_03622_b300.runner import KStap
    wl = dataclasses.replace(gen.WORKLOADS["frame1024"].with_size(512, 512), n_targets=400)
    out = dict(workload=f"{wl.name}, 400 targets", tau=wl.tau, rows=[])
    for name, kw in (("clean", {}), ("sirv_nu0.5", dict(texture_nu=0.5)),
                     ("training_targets_2", dict(training_targets=2)),
                     ("both", dict(texture_nu=0.5, training_targets=2))):
        f = gen.make_frame(wl, **kw)
        busy = np.zeros((wl.H, wl.W), bool)      # cells whose window holds a target sample
        for (r0, c0, v, beta) in f.targets + f.ring_targets:
            if 0 <= r0 < wl.H:
                busy[r0, max(0, c0 - wl.q + 1):max(0, c0 + wl.q)] = True
        Y = torch.from_numpy(f.Y).to(dev)
        for filt in ("kron", "classical"):
            ks = KStap.from_workload(wl, f.bank_a, f.bank_b, device=str(dev), filter=filt)
            o = ks.run(Y)
            Tmax = o["Tmax"].cpu().numpy().reshape(wl.H, wl.W)
            ks.close()
            det = [Tmax[r0, c0] > wl.tau for (r0, c0, v, b) in f.targets]
            free = Tmax[~busy]
            out["rows"].append(dict(scenario=name, filter=filt, pd=float(np.mean(det)),
                                    pfa=float(np.mean(free > wl.tau)),
                                    mean_T_free=float(np.mean(free))))
        del Y
    return out


# ------------------------------------------------ stacked passes (Sec. 8) ---
def multipass_leg(dev, steps: int, warmup: int, H: int = 1024, W: int = 1024):
    """Two registered passes of the 1024^2 frame model (q = 16, r_b = 3,
    n = 120, V = 64 per pass, 40 dB CNR, pass-to-pass clutter coherence 0.9)
    stacked as p = 6 channels with r_a = 2: fit + detect over the 2V-entry
    bank per step (CUDA events, L2 flushed between steps), then the change
    map.  Change Pd: targets (each present in one pass) whose cell has
    |change| > tau with the sign of their pass; change Pfa: cells whose
    window holds no target sample with |change| > tau."""
    import torch
    import gen
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    wl = gen.WORKLOADS["frame1024"].with_size(H, W)
    f = gen.make_multipass_frame(wl, K=2)
    Y = torch.from_numpy(f.Y).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ks = KStap(2 * wl.p, wl.q, 2, wl.r_b, wl.ring_r, wl.ring_a, wl.guard_r, wl.guard_a, wl.tau,
               f.bank_a, f.bank_b, device=str(dev), stream=stream)
    for _ in range(warmup):
        ks.run(Y, T_all=True)
    torch.cuda.synchronize(dev)
    K.kstap_set_profiling(ks.ctx, True)
    ms, cms = [], []
    for s in range(steps):
        flush.fill_(s & 0xff)
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        o = ks.run(Y, T_all=True)
        b.record(stream)
        Tk, ch = K.kstap_change_map(o["T_all"], wl.V, 2, stream=stream.cuda_stream)
        c.record(stream)
        c.synchronize()
        ms.append(a.elapsed_time(b))
        cms.append(b.elapsed_time(c))
    kt = K.kstap_kernel_times(ks.ctx)
    ch = ch.cpu().numpy().reshape(wl.H, wl.W)
    ks.close()
    busy = np.zeros((wl.H, wl.W), bool)
    for (kk, r0, c0, v, beta) in f.targets:
        busy[r0, max(0, c0 - wl.q + 1):c0 + wl.q] = True
    hits = [abs(ch[r0, c0]) > wl.tau and np.sign(ch[r0, c0]) == (1 if kk == 1 else -1)
            for (kk, r0, c0, v, beta) in f.targets]
    del Y, flush
    torch.cuda.empty_cache()
    return dict(workload=f"{wl.name} x 2 passes", cells_per_frame=wl.cells, p=6, q=wl.q, r_a=2,
                r_b=wl.r_b, V_bank=2 * wl.V, cells_per_s=wl.cells * len(ms) / (sum(ms) / 1e3),
                ms_per_frame=sum(ms) / len(ms), change_map_ms=sum(cms) / len(cms),
                kernel_ms_per_launch={k: v[0] / max(v[1], 1) for k, v in kt.items() if v[1]},
                change_pd=float(np.mean(hits)), change_pfa=float(np.mean(np.abs(ch[~busy]) > wl.tau)),
                targets=len(f.targets), tau=wl.tau)


# ------------------------------------------- paper's LR-Kron timing workload ---
def paper_timing_leg(dev, reps: int = 5, cpu: bool = True):
    """One large-covariance LR-Kron fit (Sec. 7.1: rank-one A, B = I, n = 5) for
    p = 3, q in {50, 250, 1000, 2500} and p = 6, q in {25, 125, 500, 1250}, at
    eps = 1e-4 and 1e-6: kstap_lrkron_fit timed with CUDA events (median of
    `reps` after a warm-up, snapshots resident on the device), and the FP64
    oracle (dense S, literal Alg. 1 and Alg. 2) on the host cores for the two
    smallest q of each p."""
    import torch
    import gen
    import oracle
    import paper_1604_03622_b300 as K
    stream = torch.cuda.current_stream(dev)
    rows = []
    for p, qs in ((3, (50, 250, 1000, 2500)), (6, (25, 125, 500, 1250))):
        for q in qs:
            X = gen.lrkron_timing_case(p, q)
            Xd = torch.from_numpy(X).to(dev)
            A = torch.empty(p, p, dtype=torch.complex64, device=dev)
            B = torch.empty(q, q, dtype=torch.complex64, device=dev)
            for eps in (1e-4, 1e-6):
                K.kstap_lrkron_fit(Xd, 1, eps, 100, A, B, stream.cuda_stream)
                ms = []
                for _ in range(reps):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    _, _, it, eta = K.kstap_lrkron_fit(Xd, 1, eps, 100, A, B, stream.cuda_stream)
                    b.record(stream)
                    b.synchronize()
                    ms.append(a.elapsed_time(b))
                row = dict(p=p, q=q, n=X.shape[0], eps=eps, iters=it, eta=eta,
                           gpu_ms=statistics.median(ms))
                if cpu and q <= (250 if p == 3 else 125):
                    x = np.stack([X[m].reshape(-1) for m in range(X.shape[0])]).astype(np.complex128)
                    t0 = time.perf_counter()
                    S = (x.T @ x.conj()) / X.shape[0]
                    oracle.lrkron(S, p, q, 1, q, eps=eps, max_iter=100)
                    row["cpu_oracle_ms"] = 1e3 * (time.perf_counter() - t0)
                rows.append(row)
            del Xd, A, B
    return dict(workload="single large-covariance LR-Kron (Sec. 7.1)", rows=rows,
                cpu_cores=__import__("oracle").num_threads())


# ----------------------------------------------------------------- serving ---
def serving_leg(dev, n_requests: int, precision: str = "mixed",
                batched_cfg=(16, 4, 1 << 20), loads=(0.8, 1.5)):
    """Poisson streams of frames (sides U{256..4096}, q in {16, 32}, r_b = 3,
    V = 64) through kstap_submit / kstap_poll with a 120 GB HBM budget (60 GB
    per q class), at each load in `loads` x the measured plain capacity (0.8:
    latency below saturation; 1.5: arrivals outpace service, so cells/s is the
    service rate).  Arms on the same arrivals: plain (one frame at a time:
    batch 1, one stream, FP32 bank), batched FP32 (continuous batching: batch
    <= 16 frames and <= 1 M cells, 4 streams) and batched with `precision`
    (default: the tensor-core bank at q = 32, FP32 below), which separates
    batching from precision.
    Latency = completion - arrival."""
    import threading
    import torch
    import gen
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    pool = gen.serving_pool()
    frames = [gen.make_frame(w) for w in pool]
    Ys = [torch.from_numpy(f.Y).to(dev) for f in frames]
    qs = sorted({w.q for w in pool})
    budget = 120 << 30
    # plain capacity: mean per-frame time of the plain path over the pool
    per_frame_s = []
    for q in qs:
        idx = [i for i, w in enumerate(pool) if w.q == q]
        ks = KStap.from_workload(pool[idx[0]], frames[idx[0]].bank_a, frames[idx[0]].bank_b,
                                 device=str(dev))
        for i in idx:
            ks.run(Ys[i])
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ks.run(Ys[i])
            b.record()
            b.synchronize()
            per_frame_s.append(a.elapsed_time(b) / 1e3)
        ks.close()
    capacity = 1.0 / float(np.mean(per_frame_s))

    def run(t_arr, pick, max_batch, max_inflight, prec, cap=None):
        ctxs = {}
        for q in qs:
            i0 = [i for i, w in enumerate(pool) if w.q == q][0]
            ks = KStap.from_workload(pool[i0], frames[i0].bank_a, frames[i0].bank_b,
                                     device=str(dev), hbm_budget_bytes=budget // len(qs),
                                     precision=class_precision(prec, q))
            K.kstap_serve_config(ks.ctx, max_batch, max_inflight)
            if cap is not None:
                K.kstap_serve_batch_cells(ks.ctx, cap)
            ctxs[q] = ks
        tickets = [None] * n_requests
        t0 = time.perf_counter()

        def submitter():
            for k in range(n_requests):
                dt = t_arr[k] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                i = int(pick[k])
                ks = ctxs[pool[i].q]
                tickets[k] = (ks, K.kstap_submit(ks.ctx, Ys[i], Ys[i].shape[1], Ys[i].shape[2]))

        th = threading.Thread(target=submitter)
        th.start()
        lat, cells = [], 0
        for k in range(n_requests):
            while tickets[k] is None:
                time.sleep(1e-4)
            ks, tk = tickets[k]
            r = K.kstap_poll(ks.ctx, tk, timeout_us=-1)
            lat.append((r.t_done_us - r.t_submit_us) / 1e3)
            cells += r.H * r.W
            K.kstap_release(ks.ctx, tk)
        t_end = time.perf_counter() - t0
        th.join()
        for ks in ctxs.values():
            ks.close()
        lat = sorted(lat)
        return dict(cells_per_s=cells / t_end, p50_ms=lat[len(lat) // 2],
                    p99_ms=lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
                    mean_ms=float(np.mean(lat)), wall_s=t_end, max_batch=max_batch,
                    streams=max_inflight, precision=MIXED if prec == "mixed" else prec,
                    batch_cells=cap)

    out = dict(workload="serving_stream", requests=n_requests, pool_frames=len(pool),
               q=qs, r_b=3, V=64, budget_gb=120, plain_capacity_frames_per_s=capacity)
    for load in loads:
        t_arr, pick = gen.poisson_arrivals(n_requests, load * capacity, len(pool))
        out[f"load_{load:g}"] = dict(
            arrival_rate_hz=load * capacity,
            mean_cells_per_frame=float(np.mean([pool[int(i)].cells for i in pick])),
            plain=run(t_arr, pick, 1, 1, "fp32"),
            batched_fp32=run(t_arr, pick, batched_cfg[0], batched_cfg[1], "fp32",
                             batched_cfg[2]),
            batched=run(t_arr, pick, batched_cfg[0], batched_cfg[1], precision,
                        batched_cfg[2]))
    return out


# ------------------------------------------------------------------ main ----
def main():
    args = parse()
    if args.peaks:
        measure_peaks(args.peaks)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import gen
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = gen.WORKLOADS[args.workload]
    if args.cells:
        wl = wl.with_size(*args.cells)
    frames = [gen.make_frame(wl, seed=rank_seed(wl.seed, rank, s)) for s in range(2)]
    Ys = [torch.from_numpy(f.Y).to(dev) for f in frames]
    stream = torch.cuda.current_stream(dev)
    ks = KStap.from_workload(wl, frames[0].bank_a, frames[0].bank_b, device=str(dev),
                             precision=args.precision,
                             stream=stream)
    K.kstap_set_tuning(ks.ctx, 64, 0, lag_store=args.lag_store)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ncell = wl.H * wl.W

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for s in range(args.warmup):
        ks.run(Ys[s % 2])
    barrier()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    K.kstap_set_profiling(ks.ctx, True)
    clk = ClockSampler(local, enabled=not args.no_clocks)
    barrier()
    t_wall = time.perf_counter()
    for s in range(args.steps):
        flush.fill_(s & 0xff)
        ev[s][0].record(stream)
        ks.run(Ys[s % 2])
        ev[s][1].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clocks = clk.stop()
    kt = K.kstap_kernel_times(ks.ctx)
    K.kstap_set_profiling(ks.ctx, False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    iters_mean = float(ks.buffers(wl.H_in, wl.W_in)["iters"].float().mean().item())
    total_ms = max_over_ranks(sum(step_ms), ws, dev)
    value = job_value(ncell, args.steps, ws, total_ms)

    # ---- e2e: pinned host frame in, Tmax / vidx / map out, through the C ABI.
    # Every step copies its frame host -> device and its results back inside
    # the timed region; the copy of frame s + 1 runs on a second stream while
    # frame s is processed (two device frame buffers), as a streaming user of
    # the library would run it.  The timed region spans the first copy to the
    # last result read.
    Yh = [torch.from_numpy(f.Y).pin_memory() for f in frames]
    Ydb = [torch.empty_like(Ys[0]) for _ in range(2)]
    outh = dict(Tmax=torch.empty(ncell, dtype=torch.float32).pin_memory(),
                vidx=torch.empty(ncell, dtype=torch.int32).pin_memory(),
                map=torch.empty(ncell, dtype=torch.uint8).pin_memory())
    cstream = torch.cuda.Stream(dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]

    def copy_in(k):
        with torch.cuda.stream(cstream):
            cstream.wait_event(freed[k % 2])      # buffer k % 2 no longer read
            Ydb[k % 2].copy_(Yh[k % 2], non_blocking=True)
            copied[k % 2].record(cstream)

    def e2e_steps(n, timed):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        cstream.wait_event(ev0)
        copy_in(0)
        for k in range(n):
            if k + 1 < n:
                copy_in(k + 1)
            stream.wait_event(copied[k % 2])
            flush.fill_(k & 0xff)
            o = ks.run(Ydb[k % 2])
            freed[k % 2].record(stream)
            for key in outh:
                outh[key].copy_(o[key], non_blocking=True)
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1)

    e2e_ms = []
    if not args.no_e2e:
        e2e_steps(args.warmup, False)
        e2e_ms = [e2e_steps(args.steps, True)]
    e2e_total = max_over_ranks(sum(e2e_ms) if e2e_ms else float("nan"), ws, dev)
    e2e_value = job_value(ncell, args.steps, ws, e2e_total)
    h2d = frames[0].Y.nbytes
    d2h = ncell * (4 + 4 + 1)

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (bound by ALU issue: per cell it moves
    # ~1 KB and executes 1e4-1e6 instructions)
    work = work_per_cell(wl)
    dom = max(kt, key=lambda k: kt[k][0])
    dom_ms, dom_n = kt[dom]
    per_launch_ms = dom_ms / max(dom_n, 1)
    achieved = work[dom] * ncell / (per_launch_ms / 1e3) / 1e12
    traffic_bytes, traffic_src = measured_traffic(wl.name, args.precision, dom)
    sm_mhz = (clocks or {}).get("sm_mhz") or 2032.0
    peak, peak_mhz, peak_note = alu_peak()
    peak_clock = peak * sm_mhz / peak_mhz                  # the same pipe at this run's clock
    roof = dict(bound="alu", kernel=dom, achieved=achieved, peak=peak, unit="TFLOP/s",
                frac=achieved / peak, frac_at_measured_clock=achieved / peak_clock,
                traffic=traffic_bytes, traffic_source=traffic_src,
                issue_active_ncu=measured_traffic(wl.name, args.precision, dom, "issue_active")[0],
                fma_pipe_active_ncu=measured_traffic(wl.name, args.precision, dom,
                                                     "fma_pipe_active")[0],
                peak_note=peak_note,
                kernel_ms_per_launch={k: v[0] / max(v[1], 1) for k, v in kt.items()},
                kernel_share={k: v[0] / max(sum(x[0] for x in kt.values()), 1e-9)
                              for k, v in kt.items()})

    batched = None if args.no_batched else batched_leg(dev, max(3, min(args.steps, 10)),
                                                         max(2, args.warmup))

    serving = None if args.no_serving else serving_leg(dev, args.serve_requests)

    precision = None if args.no_precision_leg else precision_leg(
        dev, 3, 3, cpu=not args.no_cpu_baseline)

    robustness = None if args.no_robustness else robustness_leg(dev)

    domain = None if args.no_domain else domain_leg(dev, 3, 2, cpu=not args.no_cpu_baseline)

    multipass = None if args.no_multipass else multipass_leg(dev, 3, 2)

    paper_timing = None if args.no_paper_timing else paper_timing_leg(
        dev, cpu=not args.no_cpu_baseline)

    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        cells = gen.random_cells(wl, args.cpu_sample, seed=99)
        t0 = time.perf_counter()
        oracle.run_workload(frames[0], cells=cells, want_T_all=False, want_proj=False)
        dt = time.perf_counter() - t0
        cpu = dict(value=len(cells) / dt, unit="cells/s", cores=oracle.num_threads(),
                   kind="oracle", sample=f"{len(cells)} seeded random cells of the "
                                         f"{wl.H}x{wl.W} frame (FP64, OpenMP)")

    # the metric's comparison, batched vs plain, from the batched and serving legs
    bvp = {}
    if batched:
        bvp["tiles256_cells_per_s"] = dict(plain=batched["plain"]["cells_per_s"],
                                           batched_fp32=batched["batched_fp32"]["cells_per_s"],
                                           batched=batched["batched"]["cells_per_s"])
    if serving:
        for load, tag in (("load_1.5", "serving_saturated"), ("load_0.8", "serving_0.8_load")):
            if load in serving:
                arms = serving[load]
                bvp[tag] = {a: dict(cells_per_s=arms[a]["cells_per_s"], p50_ms=arms[a]["p50_ms"],
                                    p99_ms=arms[a]["p99_ms"])
                            for a in ("plain", "batched_fp32", "batched")}

    lat = sorted(step_ms)
    line = dict(
        metric=METRIC, value=value, unit="cells/s", n_gpus=ws, steps=args.steps,
        warmup=args.warmup, ms_per_step=total_ms / args.steps, higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="f32+ff/i64" + ("" if args.precision == "fp32" else "+" + args.precision),
        data="synthetic",
        config=dict(workload=wl.name, path="plain", precision=args.precision, cells_per_frame=ncell,
                    lag_store=args.lag_store,
                    p=wl.p, q=wl.q,
                    r_a=wl.r_a, r_b=wl.r_b, n=wl.n, V=wl.V, cnr_db=wl.cnr_db,
                    l2="256 MiB flush between timed steps, outside the events",
                    flipflop_iters_mean=iters_mean,
                    parallelism=f"replicas x{ws}"),
        latency_ms=dict(p50=lat[len(lat) // 2], p99=lat[min(len(lat) - 1,
                                                            math.ceil(0.99 * len(lat)) - 1)]),
        e2e=None if args.no_e2e else dict(value=e2e_value, unit="cells/s", h2d_bytes_per_step=h2d,
                                          d2h_bytes_per_step=d2h,
                                          ms_per_step=e2e_total / args.steps,
                                          overlap="the copy of frame s+1 runs on a second "
                                                  "stream during frame s"),
        gpu_launches=sum(v[1] for v in kt.values()),
        roofline=roof, cpu_baseline=cpu, clocks=clocks, wall_s_timed_loop=t_wall,
        batched_vs_plain=bvp or None,
        batched=batched, serving=serving, precision_q32=precision, paper_timing=paper_timing,
        robustness=robustness, multipass=multipass, domain=domain)
    print(json.dumps(line), flush=True)
    ks.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
