"""Benchmark of the hybrid-dealiased convolution path on GB300.

Default workload (one step): the batch of 4096 independent 1D complex
convolutions, A = 2, B = 1, L = 4096, complex64, once with the centered 2/3
padding M = ceil(3L/2) = 6144 and once with the 1/2 padding M = 2L-1 = 8191
(two hd_convolve_batched calls, 8192 convolutions per step).  Inputs are
seeded uniform[-1, 1] and resident in HBM; the working set (768 MiB) is
larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  Keys beyond the base contract:
  roofline      dominant kernel's algorithmic bytes / CUDA-event launch time
                vs the measured HBM copy bandwidth (MEASURED_PEAKS.json)
  cpu_baseline  the FP64 direct-sum oracle timed on this host's cores on a
                bounded sample of the same workload
  e2e           the same metric through the C ABI with pinned host buffers
                (host->device inputs and device->host outputs inside the timed
                region)
  baselines     cuFFT explicit zero padding (FP32, via torch.fft) on the same GPU
  accuracy      rel-L2 and max-abs error vs the FP64 oracle on sampled instances

--impl reference runs the oracle arm: the FP64 direct sum on the host cores,
bounded samples of the same workload, same metric and unit.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import inputs  # noqa: E402

L = 4096
COUNT = 4096
SUBS = (("centered", (3 * L + 1) // 2), ("complex", 2 * L - 1))   # (kind, M)
BYTES_PER_CONV = 3 * L * 8                                         # (A+B) L sizeof(complex64)


def _peaks():
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
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

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


def cpu_oracle_rate(budget_s=10.0, kinds=SUBS, L_=L, nthreads=None):
    """Convolutions/s of the FP64 direct-sum oracle on this host (bounded sample)."""
    from oracle import cdirect
    cdirect.build()
    nt = nthreads or os.cpu_count() or 1
    done, t_total = 0, 0.0
    per = max(nt, 8)
    i = 0
    while t_total < budget_s:
        kind, _ = kinds[i % len(kinds)]
        fs = [inputs.uniform_complex((per, L_), 500 + i + a) for a in range(2)]
        t0 = time.perf_counter()
        cdirect.conv1d_batch(fs, L_, kind, "product", nthreads=nt)
        t_total += time.perf_counter() - t0
        done += per
        i += 1
    return done / t_total, nt, f"{done} convolutions of L={L_} (both paddings alternating), FP64 direct sum"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    budget = max(3.0, min(20.0, 2.0 * args.steps))
    rate, nt, sample = cpu_oracle_rate(budget)
    out = {"impl": "reference", "metric": "convolutions/s", "value": rate, "unit": "conv/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 2 * COUNT / rate * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded uniform[-1,1] complex)",
           "config": {"workload": "1d_batch_L4096_x4096_centered_M6144_and_standard_M8191", "A": 2, "B": 1},
           "cpu_baseline": {"value": rate, "unit": "conv/s", "cores": nt, "kind": "oracle", "sample": sample},
           "e2e": {"value": rate, "unit": "conv/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hd", choices=["hd", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--m", type=str, default="auto", help="override m per sub-config, e.g. 2048,4096")
    ap.add_argument("--count", type=int, default=4096, help="batch size per sub-config (profiling cases)")
    args = ap.parse_args()
    global COUNT
    COUNT = args.count
    if args.impl == "reference":
        run_reference(args)
        return
    args.warmup = max(3, args.warmup)

    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_17510_gb300 as hd
    from oracle import cdirect

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    # device-timed autotuning of (m, p, q, D, kernel variant), outside the timed region
    tuned = {}
    ms = [0, 0] if args.m == "auto" else [int(x) for x in args.m.split(",")]
    if args.m == "auto":
        for kind, M in SUBS:
            best, allc = hd.autotune(COUNT, reps=5, L=L, M=M, kind=kind, dtype="f32")
            tuned[kind] = {"best": best, "candidates": [{k: c[k] for k in ("m", "p", "q", "S", "n", "E", "minb", "ms")}
                                                        for c in allc]}

    # inputs (seeded per rank) and plans
    plans, fin, hout = [], [], []
    for si, (kind, M) in enumerate(SUBS):
        fs = [inputs.uniform_complex((COUNT, L), 1000 * rank + 10 * si + a, dtype=np.complex64) for a in range(2)]
        fin.append([torch.from_numpy(x).to(dev) for x in fs])
        hout.append(torch.empty((COUNT, L), dtype=torch.complex64, device=dev))
        plans.append(hd.Plan(L, M, m=ms[si], kind=kind, dtype="f32"))

    def launch(si):
        plans[si].convolve_batched(fin[si], hout[si], COUNT, L, stream=stream)

    def step():
        for si in range(len(SUBS)):
            launch(si)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()

    # per-launch CUDA events on the launching stream
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in SUBS]
          for _ in range(args.steps)]
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        for si in range(len(SUBS)):
            ev[k][si][0].record(stream)
            launch(si)
            ev[k][si][1].record(stream)
    t_end.record(stream)
    barrier()
    clocks = clk.stop()
    ms_total = t_start.elapsed_time(t_end)
    if dist is not None:
        t = torch.tensor([ms_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    per_kernel = [float(np.mean([ev[k][si][0].elapsed_time(ev[k][si][1]) for k in range(args.steps)]))
                  for si in range(len(SUBS))]
    ms_step = ms_total / args.steps
    convs_step = COUNT * len(SUBS) * world
    value = convs_step / (ms_step * 1e-3)

    # accuracy on sampled instances (FP64 oracle)
    acc = {}
    samp = [0, 1, COUNT // 2, COUNT - 1]
    for si, (kind, M) in enumerate(SUBS):
        fs = [fin[si][a][samp].cpu().numpy().astype(np.complex128) for a in range(2)]
        ref = cdirect.conv1d_batch(fs, L, kind)
        got = hout[si][samp].cpu().numpy().astype(np.complex128)
        acc[kind] = {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                     "max_abs": float(np.max(np.abs(got - ref))), "instances": len(samp),
                     "params": plans[si].params()}

    # end to end through the C ABI with pinned host buffers
    h_in = [[torch.empty((COUNT, L), dtype=torch.complex64).pin_memory() for _ in range(2)] for _ in SUBS]
    h_out = [torch.empty((COUNT, L), dtype=torch.complex64).pin_memory() for _ in SUBS]
    for si in range(len(SUBS)):
        for a in range(2):
            h_in[si][a].copy_(fin[si][a].cpu())
    d_in = [[torch.empty_like(fin[si][a]) for a in range(2)] for si in range(len(SUBS))]
    d_out = [torch.empty_like(hout[si]) for si in range(len(SUBS))]

    def e2e_step():
        for si in range(len(SUBS)):
            for a in range(2):
                d_in[si][a].copy_(h_in[si][a], non_blocking=True)
            plans[si].convolve_batched(d_in[si], d_out[si], COUNT, L, stream=stream)
            h_out[si].copy_(d_out[si], non_blocking=True)

    e2e_steps = max(3, min(args.steps, 10))
    for _ in range(2):
        e2e_step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    h2d = sum(2 * COUNT * L * 8 for _ in SUBS)
    d2h = sum(COUNT * L * 8 for _ in SUBS)

    # cuFFT explicit zero padding (FP32) on the same inputs
    def cufft_step():
        outs = []
        for si, (kind, M) in enumerate(SUBS):
            N = 8192 if kind == "complex" else 6144
            f, g = fin[si]
            if kind == "complex":
                F = torch.fft.fft(f, n=N, dim=-1)
                G = torch.fft.fft(g, n=N, dim=-1)
                outs.append(torch.fft.ifft(F * G, dim=-1)[:, :L])
            else:
                H = L // 2
                fp = torch.zeros((COUNT, N), dtype=f.dtype, device=dev)
                gp = torch.zeros_like(fp)
                fp[:, :L - H] = f[:, H:]
                fp[:, N - H:] = f[:, :H]
                gp[:, :L - H] = g[:, H:]
                gp[:, N - H:] = g[:, :H]
                y = torch.fft.ifft(torch.fft.fft(fp, dim=-1) * torch.fft.fft(gp, dim=-1), dim=-1)
                outs.append(torch.cat([y[:, N - H:], y[:, :L - H]], dim=-1))
        return outs

    for _ in range(2):
        cufft_step()
    barrier()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    nrep = 5
    for _ in range(nrep):
        cufft_step()
    c1.record(stream)
    barrier()
    cufft_ms = c0.elapsed_time(c1) / nrep

    hbm_peak, peak_kind = _peaks()
    dom = int(np.argmax(per_kernel))
    achieved = BYTES_PER_CONV * COUNT / (per_kernel[dom] * 1e-3) / 1e9
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path):
        try:
            traffic = json.load(open(tr_path)).get(SUBS[dom][0])
        except Exception:
            traffic = None

    out = {
        "metric": "convolutions/s", "value": value, "unit": "conv/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded uniform[-1,1] complex64)",
        "config": {"workload": "1d_batch_L4096_x4096_centered_M6144_and_standard_M8191", "L": L,
                   "batch_per_sub_config": COUNT, "A": 2, "B": 1, "parallelism": f"independent batches x{world}",
                   "l2": "working set 768 MiB > L2 (inputs larger than L2, no flush)",
                   "params": {SUBS[i][0]: plans[i].params() for i in range(len(SUBS))},
                   "autotune": tuned},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic, "peak_source": peak_kind,
                     "kernel": f"conv1d_kernel ({SUBS[dom][0]})",
                     "per_kernel_ms": {SUBS[i][0]: per_kernel[i] for i in range(len(SUBS))},
                     "bytes_per_launch": BYTES_PER_CONV * COUNT},
        "e2e": {"value": convs_step / world / (e2e_ms * 1e-3) * world, "unit": "conv/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": args.steps * len(SUBS),
        "clocks": clocks,
        "accuracy": acc,
        "baselines": {"cufft_f32_explicit": {"value": COUNT * len(SUBS) / (cufft_ms * 1e-3), "unit": "conv/s",
                                             "ms_per_step": cufft_ms}},
    }
    if rank == 0 and not args.no_cpu_baseline:
        rate, nt, sample = cpu_oracle_rate(10.0)
        out["cpu_baseline"] = {"value": rate, "unit": "conv/s", "cores": nt, "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(out), flush=True)
    for p in plans:
        p.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
