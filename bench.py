"""Benchmark of the hybrid-dealiased convolution path on GB300.

Workloads (``--workload``; the default, ``all``, prints the 1D batch as the
headline line and every other workload under ``workloads``, in one run):
  batch1d   4096 independent 1D complex convolutions, A = 2, B = 1,
            L = 4096, complex64, once with the centered 2/3 padding
            M = ceil(3L/2) = 6144 and once with the 1/2 padding M = 2L-1 = 8191:
            two hd_convolve_batched calls, 8192 convolutions per step.
  single64  one 1D convolution, L = 1024, M = 2047, complex128, FP64, integer
            inputs in -8..8, (m, p, q) by exhaustive timed search; K launches
            per step replayed from a CUDA graph.
  2d        2048 x 2048 complex, M = 4095 per axis, complex64, amplitude
            (1+|k|)^-1: FP32 hybrid vs FP64 hybrid vs cuFFT explicit padding.
  ragged    10,000 1D convolutions, L log-uniform on [64, 65536], L/M uniform
            on [0.3, 0.67], A in {2, 3}: one persistent launch from a CUDA
            graph, parameters from the learned selector (headline), the cost
            model and, with --exhaustive, the per-instance timed search.
  3d        256^3 centered Hermitian (128 stored in the last axis), M = 384
            per axis, amplitude |k|^-5/3.
  ns2d      the nonlinear term of 2D incompressible Navier-Stokes in
            Basdevant's form: velocity spectra u, v of 2048^2 (centered x,
            Hermitian y, 1024 stored), M = 3072 per axis (2/3 rule), A = B = 2
            outputs u v and u^2 - v^2, amplitude |k|^-5/3.
Inputs are seeded synthetic data resident in HBM.

One JSON line per run (rank 0).  Keys beyond the base contract: `roofline`
(dominant kernel's algorithmic bytes (A+B) * L * sizeof(element) per
convolution / CUDA-event launch time vs the measured HBM copy bandwidth of
MEASURED_PEAKS.json), `alu` (FFT flop rate, 5 S log2 S per transform, vs the
FP32 CUDA-core peak at the sampled clock), `cpu_baseline` (the FP64 oracle on
this host's cores, bounded sample), `e2e` (the same metric through the C ABI
from pinned host buffers), `baselines` (cuFFT explicit zero padding, the FP64
paths; for the 1D batch also the FP64 explicit FFT convolution on one host
thread), `accuracy` (rel-L2 / max-abs against the FP64 oracle).

``--impl reference`` runs the oracle arm of the selected workload on the
host cores (bounded samples), same metric and unit.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import inputs  # noqa: E402

L1D = 4096
SUBS = (("centered", (3 * L1D + 1) // 2), ("complex", 2 * L1D - 1))   # (kind, M)
SM_COUNT = 152
FP32_LANES = 128          # FP32 FMA lanes per SM
RAGGED_SEED = 4


def rank_seed(rank, base, a=0):
    """Seed of input array `a` of a rank's shard: every (rank, base, a) with
    a < 10 and base < 1000 gets its own stream, so ranks convolve different
    data."""
    return 1000 * (rank + 1) + 10 * base + a


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sms)) if sms else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


def fft_flops(S):
    """Radix-2 flop convention for one complex FFT of size S: 5 S log2 S."""
    return 5.0 * S * math.log2(max(S, 2))


def conv_flops(S, n, A=2, B=1):
    """FFT flops of one 1D convolution with n residues of size S (twists and
    mult not counted)."""
    return n * (A + B) * fft_flops(S)


def conv_flops_nd(axes, stored, A, B, hermitian):
    """FFT flops of one N-D convolution by the decomposition of Section 5, in
    the convention of conv_flops: on outer axis k, (A + B) n_k transforms of
    size S_k per column for every transformed instance of the axes before it;
    on the innermost axis, (A + B) transforms per residue (Hermitian residues
    in pairs, one FFT per pair) for every row the outer axes produce."""
    fl, inst = 0.0, 1
    for k, ax in enumerate(axes[:-1]):
        cols = int(np.prod(stored[k + 1:]))
        fl += inst * cols * (A + B) * ax["n"] * fft_flops(ax["S"])
        inst *= ax["n"] * ax["S"]
    ax = axes[-1]
    groups = (ax["n"] + 1) // 2 if hermitian else ax["n"]
    return fl + inst * (A + B) * groups * fft_flops(ax["S"])


# ----------------------------------------------------------------------------- CPU oracle rates

def oracle_rate_1d(budget_s, L, kinds, integer=False):
    """Convolutions/s of the FP64 direct-sum oracle (plain C, threads over the batch)."""
    from oracle import cdirect
    cdirect.build()
    nt = os.cpu_count() or 1
    done, t_total, i = 0, 0.0, 0
    per = max(nt, 8)
    gen = inputs.integer_complex if integer else inputs.uniform_complex
    while t_total < budget_s:
        kind = kinds[i % len(kinds)]
        fs = [gen((per, L), 500 + 2 * i + a) for a in range(2)]
        t0 = time.perf_counter()
        cdirect.conv1d_batch(fs, L, kind, "product", nthreads=nt)
        t_total += time.perf_counter() - t0
        done += per
        i += 1
    return done / t_total, nt, f"{done} convolutions of L={L} ({'/'.join(kinds)}), FP64 direct sum, {nt} threads"


def oracle_rate_explicit_1d(budget_s, L, subs):
    """Convolutions/s of the FP64 explicit zero-padded FFT convolution (numpy,
    the paper's comparison method) on one host thread, over the sub-configs
    (kind, M) in turn; the padded length is M (centered) or the next power of
    two (complex), as in the cuFFT baseline."""
    from oracle import explicit
    done, t_total, i = 0, 0.0, 0
    while t_total < budget_s:
        kind, M = subs[i % len(subs)]
        N = M if kind != "complex" else 1 << (M - 1).bit_length()
        fs = [inputs.uniform_complex(L, 700 + 2 * i + a) for a in range(2)]
        t0 = time.perf_counter()
        explicit.convnd_explicit(fs, (kind,), [N])
        t_total += time.perf_counter() - t0
        done += 1
        i += 1
    return done / t_total, (f"{done} convolutions of L={L} ({'/'.join(k for k, _ in subs)}), "
                            "FP64 explicit zero-padded FFT (numpy), one thread")


def oracle_rate_ragged(budget_s, descs, bins=8):
    """Convolutions/s of the FP64 direct-sum oracle over the ragged set,
    estimated from a stratified sample: the instances are split into `bins`
    equal-count bins by L, instances are drawn from every bin in turn until
    the budget is spent, and the set's total time is the sum over bins of
    (instances in the bin) x (mean sampled time in the bin).  Instances are
    independent, so the host's cores run one each."""
    from oracle import cdirect
    cdirect.build()
    nt = os.cpu_count() or 1
    g = np.random.default_rng(7)
    order = np.argsort([d["L"] for d in descs], kind="stable")
    groups = np.array_split(order, bins)
    times = [[] for _ in groups]
    done, t_total, b = 0, 0.0, 0
    while t_total < budget_s or min(len(t) for t in times) == 0:
        grp = groups[b % bins]
        d = descs[int(grp[int(g.integers(len(grp)))])]
        fs = [inputs.uniform_complex((1, d["L"]), 900 + 3 * done + a) for a in range(d["A"])]
        t0 = time.perf_counter()
        cdirect.conv1d_batch(fs, d["L"], d["kind"], "product" if d["A"] == 2 else "sum_pairs3", nthreads=1)
        dt = time.perf_counter() - t0
        times[b % bins].append(dt)
        t_total += dt
        done += 1
        b += 1
    total = sum(len(grp) * float(np.mean(t)) for grp, t in zip(groups, times))
    return len(descs) / total * nt, nt, (f"{done} instances, stratified over {bins} L-bins of the ragged set, "
                                         f"FP64 direct sum, one instance per core, rate x{nt} cores")


def oracle_rate_nd(workload):
    """Convolutions/s of the FP64 explicit zero-padded FFT oracle (numpy) on one full field."""
    from oracle import explicit
    mult = "product"
    if workload == "2d":
        f = [inputs.spectral_2d(2048, 2048, 3 + a, dtype=np.complex128) for a in range(2)]
        kinds, Ns = ("complex", "complex"), [4096, 4096]
    elif workload == "ns2d":
        f = [inputs.hermitian_2d(2048, NS2D_SEED + a, dtype=np.complex128) for a in range(2)]
        kinds, Ns, mult = ("centered", "hermitian"), [3072, 3072], "basdevant2"
    else:
        f = [inputs.hermitian_3d(256, 5 + a, dtype=np.complex128) for a in range(2)]
        kinds, Ns = ("centered", "centered", "hermitian"), [384, 384, 384]
    t0 = time.perf_counter()
    explicit.convnd_explicit(f, kinds, Ns, mult)
    dt = time.perf_counter() - t0
    return 1.0 / dt, 1, f"one full {workload} field, FP64 explicit zero-padded FFT (numpy), {dt:.1f} s"


WORKLOAD_NAMES = {
    "batch1d": "1d_batch_L4096_x4096_centered_M6144_and_standard_M8191",
    "single64": "1d_single_L1024_M2047_f64",
    "2d": "2d_2048x2048_M4095",
    "ragged": "1d_ragged_10000_L64_65536",
    "3d": "3d_centered_hermitian_256_M384",
    "ns2d": "2d_navier_stokes_basdevant_hermitian_2048_M3072_A2_B2",
}
NS2D_SEED = 7


def run_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    budget = max(3.0, min(20.0, 2.0 * args.steps))
    wl = args.workload
    if wl == "batch1d":
        rate, nt, sample = oracle_rate_1d(budget, L1D, [k for k, _ in SUBS])
    elif wl == "single64":
        rate, nt, sample = oracle_rate_1d(budget, 1024, ["complex"], integer=True)
    elif wl == "ragged":
        from oracle import params
        rate, nt, sample = oracle_rate_ragged(budget, inputs.ragged_instances(args.ragged_n, RAGGED_SEED,
                                                                              params.dealias_bound))
    else:
        rate, nt, sample = oracle_rate_nd(wl)
    cfg = {"workload": WORKLOAD_NAMES[wl]}
    out = {"impl": "reference", "metric": "convolutions/s", "value": rate, "unit": "conv/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / rate, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)", "config": cfg,
           "cpu_baseline": {"value": rate, "unit": "conv/s", "cores": nt, "kind": "oracle", "sample": sample},
           "e2e": {"value": rate, "unit": "conv/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- GPU helpers

class Ctx:
    """Rank context: one process per GPU (RANK / LOCAL_RANK / WORLD_SIZE from
    the launcher).  Ranks share nothing on the data path; the process group
    carries only the barrier around the timed region and the max-over-ranks
    of the timings.  `device="cpu"` with the gloo backend exercises the same
    host logic without a GPU."""

    def __init__(self, device=None, backend=None):
        import torch
        self.torch = torch
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.cuda = device is None
        if self.cuda:
            torch.cuda.set_device(self.local)
            self.dev = torch.device("cuda", self.local)
            self.stream = torch.cuda.current_stream()
        else:
            self.dev = torch.device(device)
            self.stream = None
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend or ("nccl" if self.cuda else "gloo"))
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()
        if self.cuda:
            self.torch.cuda.synchronize()

    def max_over_ranks(self, x):
        if self.dist is None:
            return x
        t = self.torch.tensor([x], device=self.dev, dtype=self.torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def job_rate(self, units_per_rank, ms_max):
        """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
        return units_per_rank * self.world / (ms_max * 1e-3)

    def event(self):
        return self.torch.cuda.Event(enable_timing=True)

    def time_it(self, fn, reps, warm=2, label=None):
        """Mean ms per call of fn over reps calls, CUDA events on the launching
        stream; `label` names an NVTX range around the timed calls."""
        for _ in range(warm):
            fn()
        self.barrier()
        e0, e1 = self.event(), self.event()
        if label:
            self.torch.cuda.nvtx.range_push(label)
        e0.record(self.stream)
        for _ in range(reps):
            fn()
        e1.record(self.stream)
        if label:
            self.torch.cuda.nvtx.range_pop()
        self.barrier()
        return e0.elapsed_time(e1) / reps


def base_line(args, ctx, value, ms_step, dtype, data, config):
    return {"metric": "convolutions/s", "value": value, "unit": "conv/s", "n_gpus": ctx.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": data, "config": config}


def roofline(bytes_launch, ms_launch, traffic=None, kernel=""):
    hbm, kind = peaks()
    ach = bytes_launch / (ms_launch * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": traffic,
            "peak_source": f"{kind} (MEASURED_PEAKS.json hbm_gbs)" if kind == "measured" else "fallback",
            "bytes_per_launch": bytes_launch, "ms_per_launch": ms_launch, "kernel": kernel}


ALU_PEAKS = {}


def measure_alu_peaks(hd):
    """FP32 and FP64 FMA peaks of this GPU, measured by the library's own
    microbenchmark (hd_alu_peak): the best of scalar and packed FP32 FMAs, and
    FP64 FMAs.  Taken once per run, before the workloads."""
    if not ALU_PEAKS:
        f32, f32x2 = hd.alu_peak("f32"), hd.alu_peak("f32x2")
        ALU_PEAKS.update({"f32_tflops": max(f32, f32x2), "f32_scalar_fma_tflops": f32, "f32x2_fma_tflops": f32x2,
                          "f64_tflops": hd.alu_peak("f64"),
                          "how": "hd_alu_peak: 8 chains of dependent FMAs per thread, 8 CTAs x 256 threads per SM, "
                                 "CUDA events over 5 launches"})
    return ALU_PEAKS


def alu(flops_launch, ms_launch, clocks, dtype="f32"):
    """FFT flop rate of the dominant kernel against the measured FMA peak of its
    precision (nominal spec figure for context)."""
    mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    nominal = SM_COUNT * FP32_LANES * 2 * mhz * 1e6 / 1e12
    peak = ALU_PEAKS.get(f"{dtype}_tflops")
    ach = flops_launch / (ms_launch * 1e-3) / 1e12
    out = {"achieved_tflops": ach, "peak_tflops": peak, "frac": ach / peak if peak else None,
           "flops_per_launch": flops_launch, "peak_source": "measured (hd_alu_peak, this run)" if peak else None,
           "convention": "5 S log2 S per complex FFT of size S, (A+B) n transforms per convolution"}
    if dtype == "f32":
        out["nominal_peak_tflops"] = nominal
        out["nominal_basis"] = f"{SM_COUNT} SMs x {FP32_LANES} FP32 lanes x 2 (FMA) x {mhz:.0f} MHz (sampled)"
    return out


_CODE_TOKENS = re.compile(r'("(?:\\.|[^"\\\n])*")|//[^\n]*|/\*.*?\*/', re.S)


def code_only(text):
    """C/C++/CUDA source without its comments, trailing blanks and empty
    lines (string literals kept)."""
    text = _CODE_TOKENS.sub(lambda m: m.group(1) or "", text)
    return "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip())


def source_digest(d=None):
    """SHA-256 over the code of the CUDA sources (csrc/*, comments left out),
    so that DRAM counters taken from an older build of a kernel are not
    reported for a newer one."""
    import hashlib
    d = d or os.path.join(ROOT, "paper_2303_17510_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h")):
            h.update(name.encode())
            h.update(code_only(open(os.path.join(d, name), encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


def read_traffic(key):
    """DRAM read+write bytes per launch of the dominant kernel from the
    committed ncu summary (profiles/traffic.json), or None when there is none
    for this kernel or it was taken from other kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        tj = json.load(open(p))
        if tj.get("source_digest") != source_digest():
            return None
        e = tj.get("launches", {}).get(key)
        return None if e is None else e["bytes_per_launch"]
    except Exception:
        return None


def emit(ctx, out):
    if ctx.rank == 0:
        print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- batch1d (default)

def run_batch1d(args, ctx, hd):
    from oracle import cdirect
    torch = ctx.torch
    COUNT = args.count
    tuned = {}
    ms_over = [0, 0] if args.m == "auto" else [int(x) for x in args.m.split(",")]
    if args.m == "auto":
        for kind, M in SUBS:
            best, allc = hd.autotune(COUNT, reps=5, L=L1D, M=M, kind=kind, dtype="f32")
            tuned[kind] = {"best": {k: best[k] for k in ("m", "p", "q", "S", "n", "E", "minb", "comp", "ms")},
                           "candidates": [{k: c[k] for k in ("m", "p", "q", "S", "n", "E", "minb", "comp", "ms")}
                                          for c in allc]}
    plans, fin, hout = [], [], []
    for si, (kind, M) in enumerate(SUBS):
        fs = [inputs.uniform_complex((COUNT, L1D), rank_seed(ctx.rank, si, a), dtype=np.complex64)
              for a in range(2)]
        fin.append([torch.from_numpy(x).to(ctx.dev) for x in fs])
        hout.append(torch.empty((COUNT, L1D), dtype=torch.complex64, device=ctx.dev))
        plans.append(hd.Plan(L1D, M, m=ms_over[si], kind=kind, dtype="f32"))
    ax = [p.axis_params(0) for p in plans]

    def launch(si):
        plans[si].convolve_batched(fin[si], hout[si], COUNT, L1D, stream=ctx.stream)

    for _ in range(args.warmup):
        for si in range(len(SUBS)):
            launch(si)
    ev = [[(ctx.event(), ctx.event()) for _ in SUBS] for _ in range(args.steps)]
    clk = ClockSampler(ctx.local).start()
    ctx.barrier()
    t0, t1 = ctx.event(), ctx.event()
    torch.cuda.nvtx.range_push("timed")
    t0.record(ctx.stream)
    for k in range(args.steps):
        for si in range(len(SUBS)):
            ev[k][si][0].record(ctx.stream)
            launch(si)
            ev[k][si][1].record(ctx.stream)
    t1.record(ctx.stream)
    torch.cuda.nvtx.range_pop()
    ctx.barrier()
    clocks = clk.stop()
    ms_step = ctx.max_over_ranks(t0.elapsed_time(t1)) / args.steps
    per_kernel = [float(np.mean([ev[k][si][0].elapsed_time(ev[k][si][1]) for k in range(args.steps)]))
                  for si in range(len(SUBS))]
    convs_step = COUNT * len(SUBS) * ctx.world
    value = ctx.job_rate(COUNT * len(SUBS), ms_step)

    acc = {}
    samp = [0, 1, COUNT // 2, COUNT - 1]
    for si, (kind, M) in enumerate(SUBS):
        fs = [fin[si][a][samp].cpu().numpy().astype(np.complex128) for a in range(2)]
        ref = cdirect.conv1d_batch(fs, L1D, kind)
        got = hout[si][samp].cpu().numpy().astype(np.complex128)
        acc[kind] = {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                     "max_abs": float(np.max(np.abs(got - ref))), "instances": len(samp)}

    # end to end through the C ABI: pinned host inputs -> device -> convolve -> pinned host outputs.
    # The batch is cut into chunks that rotate over NS streams (one plan per stream and sub-config), so
    # the host->device copy of one chunk, the convolutions of another and the device->host copy of a
    # third overlap; the timed region waits for every stream.
    NS, NCH = args.e2e_streams, args.e2e_chunks
    csz = (COUNT + NCH - 1) // NCH
    h_in = [[fin[si][a].cpu().pin_memory() for a in range(2)] for si in range(len(SUBS))]
    h_out = [torch.empty((COUNT, L1D), dtype=torch.complex64).pin_memory() for _ in SUBS]
    d_in = [[torch.empty_like(fin[si][a]) for a in range(2)] for si in range(len(SUBS))]
    d_out = [torch.empty_like(hout[si]) for si in range(len(SUBS))]
    streams = [torch.cuda.Stream() for _ in range(NS)]
    # built like the timed plans (m = 0 takes the autotuned candidate from the tuning cache)
    splans = [[hd.Plan(L1D, SUBS[si][1], m=ms_over[si], kind=SUBS[si][0], dtype="f32") for si in range(len(SUBS))]
              for _ in range(NS)]

    def e2e_step():
        start = torch.cuda.Event()
        start.record(ctx.stream)
        i = 0
        for si in range(len(SUBS)):
            for c0 in range(0, COUNT, csz):
                n = min(csz, COUNT - c0)
                s_ = streams[i % NS]
                s_.wait_event(start)
                with torch.cuda.stream(s_):
                    for a in range(2):
                        d_in[si][a][c0:c0 + n].copy_(h_in[si][a][c0:c0 + n], non_blocking=True)
                    splans[i % NS][si].convolve_batched([d_in[si][a][c0:c0 + n] for a in range(2)],
                                                        d_out[si][c0:c0 + n], n, L1D, stream=s_)
                    h_out[si][c0:c0 + n].copy_(d_out[si][c0:c0 + n], non_blocking=True)
                i += 1
        for s_ in streams:
            ctx.stream.wait_stream(s_)

    e2e_ms = ctx.max_over_ranks(ctx.time_it(e2e_step, max(3, min(args.steps, 10))))
    e2e_ok = all(torch.equal(h_out[si], hout[si].cpu()) for si in range(len(SUBS)))
    link = host_link(ctx, [x for row in h_in for x in row], [x for row in d_in for x in row], h_out, d_out)
    for row in splans:
        for p_ in row:
            p_.close()

    # baselines on the same GPU and inputs: cuFFT explicit zero padding (FP32), FP64 explicit, FP64 hybrid
    def cufft_step():
        for si, (kind, M) in enumerate(SUBS):
            f, g = fin[si]
            if kind == "complex":
                N = 8192
                torch.fft.ifft(torch.fft.fft(f, n=N, dim=-1) * torch.fft.fft(g, n=N, dim=-1), dim=-1)[:, :L1D]
            else:
                N, H = 6144, L1D // 2
                fp = torch.zeros((COUNT, N), dtype=f.dtype, device=ctx.dev)
                gp = torch.zeros_like(fp)
                fp[:, :L1D - H], fp[:, N - H:] = f[:, H:], f[:, :H]
                gp[:, :L1D - H], gp[:, N - H:] = g[:, H:], g[:, :H]
                y = torch.fft.ifft(torch.fft.fft(fp, dim=-1) * torch.fft.fft(gp, dim=-1), dim=-1)
                torch.cat([y[:, N - H:], y[:, :L1D - H]], dim=-1)
    cufft_ms = ctx.time_it(cufft_step, 5)
    baselines = {"cufft_f32_explicit": {"value": COUNT * len(SUBS) / (cufft_ms * 1e-3), "unit": "conv/s",
                                        "ms_per_step": cufft_ms, "padded_lengths": {"centered": 6144, "complex": 8192}}}
    if not args.no_fp64:
        f64in = [[x.to(torch.complex128) for x in fin[si]] for si in range(len(SUBS))]
        f64out = [torch.empty((COUNT, L1D), dtype=torch.complex128, device=ctx.dev) for _ in SUBS]
        for name in ("fp64_explicit", "fp64_hybrid"):
            p64 = []
            for si, (kind, M) in enumerate(SUBS):
                if name == "fp64_explicit":
                    p64.append(hd.Plan(L1D, M, m=1 << (M - 1).bit_length(), p=1, q=1, kind=kind, dtype="f64"))
                else:
                    best, _ = hd.autotune(COUNT, reps=3, L=L1D, M=M, kind=kind, dtype="f64")
                    p64.append(hd.Plan(L1D, M, kind=kind, dtype="f64", candidate=best))

            def step64():
                for si in range(len(SUBS)):
                    p64[si].convolve_batched(f64in[si], f64out[si], COUNT, L1D, stream=ctx.stream)
            t64 = ctx.time_it(step64, 3, warm=1)
            err = {}
            for si, (kind, M) in enumerate(SUBS):
                fs = [fin[si][a][samp].cpu().numpy().astype(np.complex128) for a in range(2)]
                ref = cdirect.conv1d_batch(fs, L1D, kind)
                got = f64out[si][samp].cpu().numpy()
                err[kind] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
            f64_flops = sum(COUNT * conv_flops(p64[i].axis_params(0)["S"], p64[i].axis_params(0)["n"])
                            for i in range(len(SUBS)))
            baselines[name] = {"value": COUNT * len(SUBS) / (t64 * 1e-3), "unit": "conv/s", "ms_per_step": t64,
                               "alu": alu(f64_flops, t64, {}, "f64"), "rel_l2": err,
                               "params": {SUBS[i][0]: p64[i].axis_params(0) for i in range(len(SUBS))}}
            for p in p64:
                p.close()
        del f64in, f64out

    dom = int(np.argmax(per_kernel))
    bytes_launch = 3 * L1D * 8 * COUNT
    tkey = f"{SUBS[dom][0]}:S{ax[dom]['S']}:n{ax[dom]['n']}"
    flops = COUNT * conv_flops(ax[dom]["S"], ax[dom]["n"])
    out = base_line(args, ctx, value, ms_step, "f32", "synthetic (seeded uniform[-1,1] complex64)",
                    dict({"workload": WORKLOAD_NAMES["batch1d"], "L": L1D, "batch_per_sub_config": COUNT, "A": 2,
                          "B": 1, "parallelism": f"independent batches x{ctx.world}",
                          "l2": "working set 768 MiB > L2 (inputs larger than L2, no flush)",
                          "params": {SUBS[i][0]: dict(plans[i].params(), **ax[i]) for i in range(len(SUBS))},
                          "autotune": tuned}))
    out.update({
        "roofline": dict(roofline(bytes_launch, per_kernel[dom], read_traffic(tkey), f"conv1d_kernel {tkey}"),
                         per_kernel_ms={SUBS[i][0]: per_kernel[i] for i in range(len(SUBS))}),
        "alu": alu(flops, per_kernel[dom], clocks),
        "e2e": {"value": convs_step / (e2e_ms * 1e-3), "unit": "conv/s",
                "h2d_bytes_per_step": len(SUBS) * 2 * COUNT * L1D * 8,
                "d2h_bytes_per_step": len(SUBS) * COUNT * L1D * 8, "ms_per_step": e2e_ms,
                "pipelining": f"{NCH} chunks per sub-config over {NS} streams", "outputs_match_device_run": e2e_ok,
                "host_link": link},
        "gpu_launches": args.steps * len(SUBS),
        "clocks": clocks,
        "accuracy": acc,
        "baselines": baselines,
    })
    if ctx.rank == 0 and not args.no_cpu_baseline:
        rate, nt, sample = oracle_rate_1d(10.0, L1D, [k for k, _ in SUBS])
        out["cpu_baseline"] = {"value": rate, "unit": "conv/s", "cores": nt, "kind": "oracle", "sample": sample}
        rate_x, sample_x = oracle_rate_explicit_1d(3.0, L1D, SUBS)
        out["baselines"]["cpu_fp64_explicit_fft"] = {"value": rate_x, "unit": "conv/s", "cores": 1,
                                                     "sample": sample_x}
    for p in plans:
        p.close()
    return out


# ----------------------------------------------------------------------------- single64

def run_single64(args, ctx, hd):
    from oracle import cdirect
    torch = ctx.torch
    L, M, K = 1024, 2047, 100
    best, allc = hd.autotune(1, reps=20, L=L, M=M, dtype="f64")
    plan = hd.Plan(L, M, dtype="f64", candidate=best)
    fs = inputs.integer_complex((2, L), rank_seed(ctx.rank, 2))
    f = [torch.from_numpy(np.ascontiguousarray(fs[a])).to(ctx.dev) for a in range(2)]
    h = torch.empty(L, dtype=torch.complex128, device=ctx.dev)
    s = torch.cuda.Stream()
    s.wait_stream(ctx.stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        plan.convolve(f, h, stream=s)
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            for _ in range(K):
                plan.convolve(f, h, stream=s)
    torch.cuda.synchronize()
    clk = ClockSampler(ctx.local).start()
    reps = max(3, args.steps)
    ms_step = ctx.max_over_ranks(ctx.time_it(g.replay, reps, warm=args.warmup, label="timed"))
    clocks = clk.stop()
    got = h.cpu().numpy()
    ref = cdirect.conv1d_batch([fs[0][None], fs[1][None]], L, "complex")[0]
    r = np.rint(got.real) + 1j * np.rint(got.imag)
    ms1 = ms_step / K
    out = base_line(args, ctx, ctx.job_rate(K, ms_step), ms_step, "f64", "synthetic (seeded integers in -8..8)",
                    {"workload": WORKLOAD_NAMES["single64"], "launches_per_step": K, "graph": True,
                     "params": {k: best[k] for k in ("m", "p", "q", "S", "n", "E", "minb", "ms")},
                     "candidates": [{k: c[k] for k in ("m", "p", "q", "S", "n", "ms")} for c in allc]})
    out.update({"roofline": roofline(3 * L * 16, ms1, None, "conv1d_kernel f64 (latency-bound single convolution)"),
                "alu": alu(conv_flops(best["S"], best["n"]), ms1, clocks, "f64"),
                "accuracy": {"exact_after_rint": bool(np.array_equal(r, ref)),
                             "max_dev_from_integer": float(np.max(np.abs(got - r)))},
                "gpu_launches": K * reps, "clocks": clocks,
                "e2e": e2e_single(ctx, plan, fs, L)})
    if ctx.rank == 0 and not args.no_cpu_baseline:
        rate, nt, sample = oracle_rate_1d(10.0, L, ["complex"], integer=True)
        out["cpu_baseline"] = {"value": rate, "unit": "conv/s", "cores": nt, "kind": "oracle", "sample": sample}
    plan.close()
    return out


def host_link(ctx, h_src, d_dst, h_dst, d_src, reps=5):
    """Plain copies between pinned host memory and the device with the byte
    counts of one end-to-end step: host->device alone, device->host alone, and
    both at once on two streams (GB/s).  The ceiling of the e2e figure."""
    torch = ctx.torch
    up = sum(x.numel() * x.element_size() for x in h_src)
    down = sum(x.numel() * x.element_size() for x in h_dst)

    def h2d():
        for a, b in zip(d_dst, h_src):
            a.copy_(b, non_blocking=True)

    def d2h():
        for a, b in zip(h_dst, d_src):
            a.copy_(b, non_blocking=True)
    s2 = torch.cuda.Stream()

    def both():
        s2.wait_stream(ctx.stream)
        h2d()
        with torch.cuda.stream(s2):
            d2h()
        ctx.stream.wait_stream(s2)
    t_up = ctx.time_it(h2d, reps)
    t_down = ctx.time_it(d2h, reps)
    t_both = ctx.time_it(both, reps)
    return {"h2d_gbs": up / (t_up * 1e-3) / 1e9, "d2h_gbs": down / (t_down * 1e-3) / 1e9,
            "both_gbs": (up + down) / (t_both * 1e-3) / 1e9, "h2d_bytes": up, "d2h_bytes": down,
            "ms_h2d": t_up, "ms_d2h": t_down, "ms_both": t_both}


def e2e_single(ctx, plan, fs, L):
    torch = ctx.torch
    h_in = [torch.from_numpy(np.ascontiguousarray(fs[a])).pin_memory() for a in range(2)]
    h_out = torch.empty(L, dtype=torch.complex128).pin_memory()
    d_in = [torch.empty(L, dtype=torch.complex128, device=ctx.dev) for _ in range(2)]
    d_out = torch.empty(L, dtype=torch.complex128, device=ctx.dev)

    def step():
        for a in range(2):
            d_in[a].copy_(h_in[a], non_blocking=True)
        plan.convolve(d_in, d_out, stream=ctx.stream)
        h_out.copy_(d_out, non_blocking=True)
    ms = ctx.time_it(step, 50, warm=5)
    return {"value": 1e3 / ms, "unit": "conv/s", "h2d_bytes_per_step": 2 * L * 16, "d2h_bytes_per_step": L * 16,
            "ms_per_step": ms}


# ----------------------------------------------------------------------------- 2d

def run_2d(args, ctx, hd):
    from oracle import direct
    torch = ctx.torch
    L = 2048
    fs = [inputs.spectral_2d(L, L, rank_seed(ctx.rank, 3, a), dtype=np.complex64) for a in range(2)]
    f = [torch.from_numpy(x).to(ctx.dev) for x in fs]
    g = np.random.default_rng(0)
    pts = np.stack([g.integers(0, L, 48), g.integers(0, L, 48)], 1)
    want = direct.convnd_points([x.astype(np.complex128) for x in fs], ("complex", "complex"), pts)
    res = {}
    # the inner axis is a batch of 1D convolutions (outer residues x slots = 4 x 1024 rows of L = 2048):
    # tune it on that batch; the plans then take its candidate from the tuning cache
    hd.tune_cache_clear()
    inner_tuned = {}
    for dtype in ("f32", "f64"):
        b_, allc = hd.autotune(4096, reps=3, L=L, M=2 * L - 1, dtype=dtype)
        inner_tuned[dtype] = {"best": {k: b_[k] for k in ("m", "p", "q", "S", "n", "E", "minb", "ms")},
                              "candidates": len(allc)}
    for dtype in ("f32", "f64"):
        ff = f if dtype == "f32" else [x.to(torch.complex128) for x in f]
        hh = torch.empty_like(ff[0])
        plan = hd.Plan([L, L], [2 * L - 1, 2 * L - 1], dtype=dtype)
        reps = max(3, args.steps) if dtype == "f32" else 3
        clk = ClockSampler(ctx.local).start()
        ms = ctx.max_over_ranks(ctx.time_it(lambda: plan.convolve(ff, hh, stream=ctx.stream), reps,
                                            warm=args.warmup, label="timed" if dtype == "f32" else None))
        clocks = clk.stop()
        got = hh.cpu().numpy()[tuple(pts.T)]
        res[dtype] = {"ms": ms, "clocks": clocks, "axes": [plan.axis_params(0), plan.axis_params(1)],
                      "scratch_bytes": plan.params()["scratch_bytes"],
                      "rel_l2_sampled": float(np.linalg.norm(got - want) / np.linalg.norm(want))}
        if dtype == "f32":
            e2e = e2e_nd(ctx, plan, f, hh)
        plan.close()

    def cufft():
        F = torch.fft.fft2(f[0], s=(2 * L, 2 * L))
        G = torch.fft.fft2(f[1], s=(2 * L, 2 * L))
        return torch.fft.ifft2(F * G)[:L, :L]
    cu = ctx.time_it(cufft, 5)
    ms = res["f32"]["ms"]
    out = base_line(args, ctx, ctx.job_rate(1, ms), ms, "f32", "synthetic (seeded, amplitude (1+|k|)^-1)",
                    {"workload": WORKLOAD_NAMES["2d"], "l2": "inputs+outputs 96 MiB; work buffer larger than L2",
                     "inner_axis_autotune": inner_tuned,
                     "f32": {k: v for k, v in res["f32"].items() if k != "clocks"},
                     "f64": {k: v for k, v in res["f64"].items() if k != "clocks"}})
    out.update({"roofline": roofline(3 * L * L * 8, ms, read_traffic("2d"), "2d plan (all kernels of one convolution)"),
                "alu": alu(conv_flops_nd(res["f32"]["axes"], [L, L], 2, 1, False), ms, res["f32"]["clocks"]),
                "accuracy": {"rel_l2_sampled": res["f32"]["rel_l2_sampled"], "points": len(pts)},
                "baselines": {"fp64_hybrid": {"value": 1e3 / res["f64"]["ms"], "unit": "conv/s",
                                              "rel_l2_sampled": res["f64"]["rel_l2_sampled"]},
                              "cufft_f32_explicit_4096x4096": {"value": 1e3 / cu, "unit": "conv/s", "ms": cu}},
                # one convolution: outer-axis forward, the inner batch of rows, outer-axis backward
                "gpu_launches": 3 * max(3, args.steps),
                "e2e": e2e, "clocks": res["f32"]["clocks"]})
    if ctx.rank == 0 and not args.no_cpu_baseline:
        rate, nt, sample = oracle_rate_nd("2d")
        out["cpu_baseline"] = {"value": rate, "unit": "conv/s", "cores": nt, "kind": "oracle", "sample": sample}
    return out


def e2e_nd(ctx, plan, f, hh):
    """One convolution per step from pinned host inputs to pinned host
    outputs (hh: the device output, or the list of B outputs)."""
    torch = ctx.torch
    hh = list(hh) if isinstance(hh, (list, tuple)) else [hh]
    h_in = [x.cpu().pin_memory() for x in f]
    h_out = [torch.empty(x.shape, dtype=x.dtype).pin_memory() for x in hh]
    d_in = [torch.empty_like(x) for x in f]
    d_out = [torch.empty_like(x) for x in hh]

    def step():
        for a in range(len(f)):
            d_in[a].copy_(h_in[a], non_blocking=True)
        plan.convolve(d_in, d_out if len(d_out) > 1 else d_out[0], stream=ctx.stream)
        for b in range(len(d_out)):
            h_out[b].copy_(d_out[b], non_blocking=True)
    ms = ctx.time_it(step, 5)
    nb = f[0].numel() * f[0].element_size()
    return {"value": 1e3 / ms, "unit": "conv/s", "h2d_bytes_per_step": len(f) * nb,
            "d2h_bytes_per_step": len(d_out) * nb, "ms_per_step": ms}


# ----------------------------------------------------------------------------- ns2d

def run_ns2d(args, ctx, hd):
    """Nonlinear term of 2D incompressible Navier-Stokes (Basdevant form):
    velocity spectra u, v in, the spectra of u v and u^2 - v^2 out."""
    from oracle import direct
    torch = ctx.torch
    L, M = 2048, 3072
    H = L // 2
    # four input/output sets (4 x 64 MiB, more than L2) rotated over the timed calls
    sets = []
    for k in range(4):
        xs = [inputs.hermitian_2d(L, rank_seed(ctx.rank, NS2D_SEED, a) + 100 * k, dtype=np.complex64)
              for a in range(2)]
        fk = [torch.from_numpy(x).to(ctx.dev) for x in xs]
        sets.append((xs, fk, [torch.empty_like(fk[0]) for _ in range(2)]))
    fs, f, hh = sets[0]
    g = np.random.default_rng(2)
    pts = np.stack([g.integers(0, L, 32), g.integers(0, H, 32)], 1)
    want = direct.convnd_points([x.astype(np.complex128) for x in fs], ("centered", "hermitian"), pts,
                                "basdevant2")
    # the inner (Hermitian) axis is a batch of 1D convolutions: tune it on a batch of its rows
    hd.tune_cache_clear()
    b_, allc = hd.autotune(4096, reps=3, L=L, M=M, A=2, B=2, kind="hermitian")
    inner = {"best": {k: b_[k] for k in ("m", "p", "q", "S", "n", "E", "minb", "ms")}, "candidates": len(allc)}
    plan = hd.Plan([L, L], [M, M], A=2, B=2, kind="hermitian")
    reps = max(4, args.steps)
    it = [0]

    def step():
        _, fk, hk = sets[it[0] % len(sets)]
        it[0] += 1
        plan.convolve(fk, hk, stream=ctx.stream)
    clk = ClockSampler(ctx.local).start()
    ms = ctx.max_over_ranks(ctx.time_it(step, reps, warm=args.warmup, label="timed"))
    clocks = clk.stop()
    plan.convolve(f, hh, stream=ctx.stream)
    torch.cuda.synchronize()
    acc = [float(np.linalg.norm(hh[b].cpu().numpy()[tuple(pts.T)] - want[b]) / np.linalg.norm(want[b]))
           for b in range(2)]
    e2e = e2e_nd(ctx, plan, f, hh)
    axes = [plan.axis_params(0), plan.axis_params(1)]
    scratch = plan.params()["scratch_bytes"]
    plan.close()
    hd.tune_cache_clear()

    def cufft():
        # explicit dealiasing: the velocity fields on the 3072^2 real grid, the two products, back to spectra
        full = torch.zeros((2, M, M // 2 + 1), dtype=torch.complex64, device=ctx.dev)
        for a in range(2):
            c = torch.fft.ifftshift(f[a], dim=0)          # centered x -> FFT order
            full[a, :H, :H] = c[:H]
            full[a, -H:, :H] = c[H:]
        u, v = torch.fft.irfft2(full, s=(M, M))
        return torch.fft.rfft2(u * v), torch.fft.rfft2((u + v) * (u - v))
    cu = ctx.time_it(cufft, 5)
    out = base_line(args, ctx, ctx.job_rate(1, ms), ms, "f32",
                    "synthetic (seeded real fields, amplitude |k|^-5/3, exact Hermitian symmetry)",
                    {"workload": WORKLOAD_NAMES["ns2d"], "axes": axes, "inner_axis_autotune": inner,
                     "scratch_bytes": scratch,
                     "l2": "4 input/output sets of 64 MiB rotated over the timed calls (256 MiB > L2)"})
    out.update({"roofline": roofline(4 * L * H * 8, ms, read_traffic("ns2d"), "ns2d plan (all kernels)"),
                "alu": alu(conv_flops_nd(axes, [L, H], 2, 2, True), ms, clocks),
                "accuracy": {"rel_l2_sampled": acc, "points": len(pts)},
                "baselines": {"cufft_f32_explicit_3072^2_real": {"value": 1e3 / cu, "unit": "conv/s", "ms": cu}},
                # one convolution: outer-axis forward, the inner batch of rows, outer-axis backward
                "gpu_launches": 3 * reps,
                "e2e": e2e, "clocks": clocks})
    if ctx.rank == 0 and not args.no_cpu_baseline:
        rate, nt, sample = oracle_rate_nd("ns2d")
        out["cpu_baseline"] = {"value": rate, "unit": "conv/s", "cores": nt, "kind": "oracle", "sample": sample}
    return out


# ----------------------------------------------------------------------------- 3d

def run_3d(args, ctx, hd):
    from oracle import direct
    torch = ctx.torch
    L = 256
    fs = [inputs.hermitian_3d(L, rank_seed(ctx.rank, 4, a), dtype=np.complex64) for a in range(2)]
    f = [torch.from_numpy(x).to(ctx.dev) for x in fs]
    h = torch.empty_like(f[0])
    g = np.random.default_rng(1)
    pts = np.stack([g.integers(0, L, 16), g.integers(0, L, 16), g.integers(0, L // 2, 16)], 1)
    want = direct.convnd_points([x.astype(np.complex128) for x in fs], ("centered", "centered", "hermitian"), pts)

    def rel(hh):
        got = hh.cpu().numpy()[tuple(pts.T)]
        return float(np.linalg.norm(got - want) / np.linalg.norm(want))

    def time_plan(p_, label=None):
        return ctx.max_over_ranks(ctx.time_it(lambda: p_.convolve(f, h, stream=ctx.stream), max(3, args.steps),
                                              warm=args.warmup, label=label))

    # parameters of the innermost (Hermitian) axis: cost model, then the learned selector (with the timed
    # search as its fallback when the ensemble is unsure); outer axes: cost model
    from paper_2303_17510_gb300 import selector
    hd.tune_cache_clear()
    hd.selector_clear()
    with hd.Plan([L, L, L], [384, 384, 384], kind="hermitian") as pcm:
        ms_cm = time_plan(pcm)
        axes_cm = [pcm.axis_params(i) for i in range(3)]
    models, _ = selector.train(selector.load_data(), k=4, steps=args.train_steps)
    hd.selector_install(models, tau=0.05, sigma=0.25, fallback=True)
    t0 = time.perf_counter()
    plan = hd.Plan([L, L, L], [384, 384, 384], kind="hermitian")
    plan_s = time.perf_counter() - t0
    hd.selector_clear()
    clk = ClockSampler(ctx.local).start()
    ms = time_plan(plan, "timed")
    clocks = clk.stop()
    acc = rel(h)
    e2e = e2e_nd(ctx, plan, f, h)
    axes = [plan.axis_params(i) for i in range(3)]
    # the same parameters with compensated (TwoSum) residue sums in the inner convolutions
    os.environ["HD_COMP"] = "1"
    try:
        pc = hd.Plan([L, L, L], [384, 384, 384], kind="hermitian", m=[a["m"] for a in axes],
                     p=[a["p"] for a in axes], q=[a["q"] for a in axes])
    finally:
        del os.environ["HD_COMP"]
    with pc:
        ms_comp = time_plan(pc)
        acc_comp = rel(h)

    def cufft():
        # explicit dealiasing of the same field: 384^3 real grid, inverse real FFTs, product, forward real FFT
        N = 384
        full = torch.zeros((2, N, N, N // 2 + 1), dtype=torch.complex64, device=ctx.dev)
        for a in range(2):
            c = torch.fft.ifftshift(f[a], dim=(0, 1))
            full[a, :128, :128, :128] = c[:128, :128]
            full[a, -128:, :128, :128] = c[128:, :128]
            full[a, :128, -128:, :128] = c[:128, 128:]
            full[a, -128:, -128:, :128] = c[128:, 128:]
        r = torch.fft.irfftn(full, s=(N, N, N), dim=(1, 2, 3))
        return torch.fft.rfftn(r[0] * r[1])
    cu = ctx.time_it(cufft, 3)
    out = base_line(args, ctx, ctx.job_rate(1, ms), ms, "f32",
                    "synthetic (seeded real field, amplitude |k|^-5/3, exact Hermitian symmetry)",
                    {"workload": WORKLOAD_NAMES["3d"], "axes": axes, "planning_s": plan_s,
                     "parameters": "innermost axis: learned selector (timed search when unsure); outer: cost model",
                     "scratch_bytes": plan.params()["scratch_bytes"],
                     "l2": "inputs+outputs 96 MiB; work buffers larger than L2"})
    out.update({"roofline": roofline(3 * L * L * (L // 2) * 8, ms, read_traffic("3d"), "3d plan (all kernels)"),
                "alu": alu(conv_flops_nd(axes, [L, L, L // 2], 2, 1, True), ms, clocks),
                "accuracy": {"rel_l2_sampled": acc, "points": len(pts)},
                "variants": {"cost_model_params": {"ms": ms_cm, "axes": axes_cm},
                             "compensated_sums": {"ms": ms_comp, "rel_l2_sampled": acc_comp}},
                "baselines": {"cufft_f32_explicit_384^3_real": {"value": 1e3 / cu, "unit": "conv/s", "ms": cu}},
                # one convolution: two outer-axis forward kernels, the inner batch, two outer-axis backward
                "gpu_launches": 5 * max(3, args.steps),
                "e2e": e2e, "clocks": clocks})
    if ctx.rank == 0 and not args.no_cpu_baseline:
        rate, nt, sample = oracle_rate_nd("3d")
        out["cpu_baseline"] = {"value": rate, "unit": "conv/s", "cores": nt, "kind": "oracle", "sample": sample}
    plan.close()
    return out


# ----------------------------------------------------------------------------- ragged

def run_ragged(args, ctx, hd):
    from oracle import cdirect
    from paper_2303_17510_gb300 import selector
    torch = ctx.torch
    descs = inputs.ragged_instances(args.ragged_n, RAGGED_SEED, hd.dealias_bound)
    tot = sum(d["L"] for d in descs)
    base = [torch.from_numpy(inputs.uniform_complex(tot, rank_seed(ctx.rank, 5, a), dtype=np.complex64)).to(ctx.dev)
            for a in range(3)]
    outb = torch.empty(tot, dtype=torch.complex64, device=ctx.dev)
    fs, hs, off = [], [], 0
    for d in descs:
        fs.append([base[a][off:off + d["L"]] for a in range(d["A"])])
        hs.append(outb[off:off + d["L"]])
        off += d["L"]
    bytes_ = sum((d["A"] + 1) * d["L"] * 8 for d in descs)
    reps = max(3, args.steps)

    def timed(plan, label=None):
        plan.bind(fs, hs)
        ms = ctx.max_over_ranks(ctx.time_it(plan.run, reps, warm=args.warmup, label=label))
        st = plan.status()
        if st != "HD_OK":
            raise RuntimeError(f"ragged run: {st}")
        return ms

    res, setup = {}, {}
    hd.tune_cache_clear()
    hd.selector_clear()
    t0 = time.perf_counter()
    with hd.RaggedPlan(descs) as p:
        setup["cost_model"] = time.perf_counter() - t0
        res["cost_model"] = timed(p)
    # learned selector: ensemble trained on the committed autotuner timings by the library's GPU kernels
    t0 = time.perf_counter()
    models, losses = selector.train(selector.load_data(), k=4, steps=args.train_steps)
    train_s = time.perf_counter() - t0
    hd.selector_install(models, tau=0.05, sigma=0.25, fallback=False)
    t0 = time.perf_counter()
    clk = ClockSampler(ctx.local).start()
    with hd.RaggedPlan(descs) as p:
        setup["selector"] = time.perf_counter() - t0
        res["selector"] = timed(p, "timed")
        sel = [p.params(i) for i in range(len(descs))]
        clocks = clk.stop()
        # end to end through the C ABI: pinned host inputs -> device buffers the plan is bound to
        # -> one ragged launch -> pinned host outputs
        h_in = [x.cpu().pin_memory() for x in base]
        h_out = torch.empty(tot, dtype=torch.complex64).pin_memory()

        def e2e_step():
            for a in range(3):
                base[a].copy_(h_in[a], non_blocking=True)
            p.run(ctx.stream)
            h_out.copy_(outb, non_blocking=True)
        e2e_ms = ctx.max_over_ranks(ctx.time_it(e2e_step, max(3, min(args.steps, 10))))
        e2e = {"value": ctx.job_rate(len(descs), e2e_ms), "unit": "conv/s", "h2d_bytes_per_step": 3 * tot * 8,
               "d2h_bytes_per_step": tot * 8, "ms_per_step": e2e_ms}
    hd.selector_clear()
    out_sel = outb.clone()
    matched = None
    if args.exhaustive:
        t0 = time.perf_counter()
        best = []
        for d in descs:
            b_, _ = hd.autotune(selector.batch_count(d["L"]), reps=3, L=d["L"], M=d["M"], A=d["A"], kind=d["kind"],
                                dtype="f32")
            best.append(b_)
        setup["exhaustive"] = time.perf_counter() - t0
        with hd.RaggedPlan(descs) as p:       # picks each instance's tuned (S, n) where the kernel supports it
            res["exhaustive"] = timed(p)
            got = [p.params(i) for i in range(len(descs))]
        matched = sum(1 for a, b_ in zip(got, best) if a["S"] == b_["S"] and a["n"] == b_["n"])
        hd.tune_cache_clear()
    # accuracy of the selector plan's output on sampled instances (6 of them, 32 points each)
    order = np.argsort([d["L"] for d in descs])
    pick = list(order[:2]) + list(order[len(order) // 2:len(order) // 2 + 2]) + list(order[-2:])
    errs = []
    for i in pick:
        d = descs[i]
        idx = np.unique(np.linspace(0, d["L"] - 1, 32).astype(np.int64))
        xs = [x.cpu().numpy().astype(np.complex128) for x in fs[i]]
        off = int(sum(descs[j]["L"] for j in range(i)))
        want = cdirect.conv1d_points(xs, d["L"], idx, d["kind"], "product" if d["A"] == 2 else "sum_pairs3")
        got_i = out_sel[off:off + d["L"]].cpu().numpy()[idx]
        errs.append(float(np.linalg.norm(got_i - want) / np.linalg.norm(want)))
    ms = res["selector"]
    out = base_line(args, ctx, ctx.job_rate(len(descs), ms), ms, "f32", "synthetic (seeded uniform[-1,1])",
                    {"workload": WORKLOAD_NAMES["ragged"] if args.ragged_n == 10000 else
                     f"1d_ragged_{args.ragged_n}_L64_65536",
                     "instances": len(descs), "algorithmic_bytes": bytes_, "launch": "one persistent kernel, CUDA graph",
                     "selector_train_s": train_s, "selector_train_mse": losses, "setup_s": setup,
                     "split_instances": sum(1 for c in sel if c["S"] > 4096),
                     "exhaustive_matched_instances": matched,
                     "l2": f"inputs+outputs {bytes_ / 2**20:.0f} MiB > L2"})
    out.update({"ragged_ms": res,
                "selector_vs_exhaustive": (res["selector"] / res["exhaustive"]) if "exhaustive" in res else None,
                "selector_vs_cost_model": res["selector"] / res["cost_model"],
                "roofline": roofline(bytes_, ms, read_traffic("ragged"), "ragged_kernel"),
                "alu": alu(sum(conv_flops(c["S"], c["n"], d["A"], 1) for c, d in zip(sel, descs)), ms, clocks),
                "accuracy": {"rel_l2_sampled_max": max(errs), "instances": len(pick)},
                "e2e": e2e, "gpu_launches": reps, "clocks": clocks})
    if ctx.rank == 0 and not args.no_cpu_baseline:
        rate, nt, sample = oracle_rate_ragged(10.0, descs)
        out["cpu_baseline"] = {"value": rate, "unit": "conv/s", "cores": nt, "kind": "oracle", "sample": sample}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hd", choices=["hd", "reference"])
    ap.add_argument("--workload", default="all", choices=["all"] + list(WORKLOAD_NAMES),
                    help="all (default): the 1D batch as the headline line, every other workload under `workloads`")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="batch1d: skip the FP64 baselines")
    ap.add_argument("--m", type=str, default="auto", help="batch1d: m per sub-config, e.g. 2048,4096")
    ap.add_argument("--count", type=int, default=4096, help="batch1d: batch size per sub-config")
    ap.add_argument("--ragged-n", type=int, default=10000)
    ap.add_argument("--e2e-streams", type=int, default=3, help="batch1d e2e: streams the chunks rotate over")
    ap.add_argument("--e2e-chunks", type=int, default=8, help="batch1d e2e: chunks per sub-config")
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--exhaustive", action="store_true", help="ragged: also time the per-instance exhaustive search")
    ap.add_argument("--no-exhaustive", action="store_true",
                    help="all: skip the ragged per-instance exhaustive search (on by default there)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        if args.workload == "all":
            args.workload = "batch1d"
        run_reference(args)
        return
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_17510_gb300 as hd
    ctx = Ctx()
    runs = {"batch1d": run_batch1d, "single64": run_single64, "2d": run_2d, "ragged": run_ragged,
            "3d": run_3d, "ns2d": run_ns2d}
    peaks_ = measure_alu_peaks(hd)
    if args.workload != "all":
        out = runs[args.workload](args, ctx, hd)
        out["alu_peaks"] = peaks_
        emit(ctx, out)
    else:
        # the 1D batch is the headline line; every other workload runs after it in the same
        # process, under one clock record (`clocks_all`), and is reported under `workloads`
        clk_all = ClockSampler(ctx.local).start()
        t_all = time.perf_counter()
        out = run_batch1d(args, ctx, hd)
        args.exhaustive = not args.no_exhaustive
        wl = {}
        for name in ("single64", "2d", "3d", "ragged", "ns2d"):
            t0 = time.perf_counter()
            o = runs[name](args, ctx, hd)
            for k in ("metric", "n_gpus", "steps", "warmup", "higher_is_better", "scaling", "vs_baseline"):
                o.pop(k, None)
            o["wall_s"] = time.perf_counter() - t0
            wl[name] = o
        out["workloads"] = wl
        out["alu_peaks"] = peaks_
        out["clocks_all"] = dict(clk_all.stop(), wall_s=time.perf_counter() - t_all)
        emit(ctx, out)
    if ctx.dist is not None:
        ctx.dist.destroy_process_group()


if __name__ == "__main__":
    main()
