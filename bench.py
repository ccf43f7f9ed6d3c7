#!/usr/bin/env python
"""Throughput of the feedforward decentralized precoding path on GB300.

Headline workload (one rank): the batched uneven form.  512 precoding
instances, each with U in {8, 16, 24, 32, 48, 64} users, B in {64, ..., 1024}
antennas, C clusters dividing B, 72..3300 subcarriers, K = 14 OFDM symbols,
64-QAM, 10 dB, i.i.d. or Kronecker-correlated channel and PD-WF or FD-WF
(tau = 0.125), drawn with a fixed seed.  They are precoded by the
reduced-precision path (FP16 Gram and split-FP16 apply on the tensor cores,
FP32 solve) in persistent bucket launches replayed from a CUDA graph, after
the autotuner picked each bucket's CTAs per SM.  One step is one batched pass
over all instances (826,516 subcarriers; about 114 GB of algorithmic traffic,
so every step streams from HBM: the 129 MB L2 holds a thousandth of it).
Metric: precoded subcarriers per second.

Beside the headline: the plain FP32 path instance by instance on the same
instances (the metric's denominator), the roofline of the dominant bucket from
per-bucket CUDA events, the FP64 CPU oracle on a bounded sample of the timed
inputs (also the parity check of the timed outputs), an end-to-end figure
through host buffers, and secondary records: single plans on the U = 16,
B = 256 slot and on the U = 32, B = 512 precision workload, and the serving
sweep.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torchrun, one rank per GPU, each rank precoding its own draw of the batch
(replicas: instances are independent, no collective on the data path).
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

C2 = dict(name="c2", U=16, B=256, C=8, n_sc=1200, K=14, qam=16, snr_db=10.0)
C3 = dict(name="c3", U=32, B=512, C=16, n_sc=3300, K=14, qam=64, snr_db=10.0)
C4_INSTANCES = 512
K_SYM = 14
DTYPE_TC = ("fp16 Gram and split-fp16 apply on the tensor cores (tcgen05, f32 accumulate), "
            "f32 solve")
_CS = "paper_1804_10987_gb300/csrc/"
KERNEL_SOURCES = {
    "fp32": [_CS + f for f in ("dp_fp32_impl.cuh", "dp_blocks.cuh", "dp_common.cuh")],
    "pipe": [_CS + f for f in ("dp_tcpipe.cu", "dp_tc.cuh", "dp_blocks.cuh", "dp_common.cuh")],
    "tc": [_CS + f for f in ("dp_tc_impl.cuh", "dp_quad.cuh", "dp_tc.cuh", "dp_blocks.cuh",
                             "dp_common.cuh")],
    "fdsmall": [_CS + f for f in ("dp_fdsmall.cu", "dp_blocks.cuh", "dp_common.cuh")],
    "rows": [_CS + f for f in ("dp_rowsolve.cu", "dp_blocks.cuh", "dp_common.cuh")],
    # the split form's three launches (tensor-core Gram, row solve, apply)
    "split": [_CS + f for f in ("dp_tc_impl.cuh", "dp_quad.cuh", "dp_tc.cuh", "dp_rowsolve.cu",
                                "dp_blocks.cuh", "dp_common.cuh")],
}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
PAPER_CONTEXT = ("PD-WF U=16 B=256 C=8 on 8 V100 (one per cluster), K=7: 0.607 ms per "
                 "1200-subcarrier slot = 1.98 M subcarriers/s (FD-WF 0.472 ms = 2.54 M)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["c4", "c2"], default="c4",
                    help="headline workload: the batched uneven form (c4) or the single "
                         "U=16 B=256 slot (c2, as a plain line for profiling)")
    ap.add_argument("--prec", choices=["bf16", "fp16"], default="fp16",
                    help="arithmetic of the reduced-precision headline path")
    ap.add_argument("--instances", type=int, default=C4_INSTANCES,
                    help="instances of the batched workload (the first N of the 512-draw)")
    ap.add_argument("--mode", choices=["wf", "zf", "fdwf"], default="wf",
                    help="mode of the c2 record")
    ap.add_argument("--slots", type=int, default=8, help="slots of 1200 subcarriers per c2 step")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip timing the plain FP32 path beside the headline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-c2", action="store_true", help="skip the c2 single-plan record")
    ap.add_argument("--no-c3", action="store_true", help="skip the c3 precision record")
    ap.add_argument("--no-library", action="store_true",
                    help="skip the paper-style library pipeline (context baseline)")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving sweep (Poisson arrivals)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="bound of the CPU oracle sample")
    ap.add_argument("--serve-requests", type=int, default=1500,
                    help="requests per arrival rate in the serving sweep")
    ap.add_argument("--serving-knee", type=int, default=0, metavar="N",
                    help="only this: the steady-state serving sweep with N and N/4 requests "
                         "per rate (e.g. 20000); reports each server's knee rate; one JSON line")
    ap.add_argument("--serving-burst", type=int, default=0, metavar="N",
                    help="only this: N requests submitted at once to the solve-cached FP32 "
                         "server over the serving cells (i.i.d. channels); one JSON line")
    return ap.parse_args()


# ------------------------------------------------------------ ranks ----------
def job_time_ms(ms, world, device):
    """The job's time for N ranks: the slowest rank's (max over ranks)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput: the units all ranks processed per second of the
    job's time (each rank processes its own units: weak scaling)."""
    return units_per_rank * world / (ms / 1e3)


def rank_seed(synth, rank):
    """Seed of a rank's c2 input shard: every rank precodes its own slots."""
    return synth.seed_for(2, 500 + rank)


def c4_rank_seed(synth, rank):
    """Seed of a rank's draw of the batched workload's channels and symbols."""
    return synth.seed_for(4, 1 + 1000 * rank)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------- clocks ----
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.bus_id = bus_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]),
                                 power=float(parts[3]) if parts[3] not in ("[N/A]", "N/A") else 0.0,
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        loaded = [r for r in rows if r["power"] > 0.25 * max(x["power"] for x in rows)] or rows
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in loaded),
                "sm_max_mhz": max(r["smax"] for r in rows), "samples": len(rows),
                "reasons": sorted(reasons)}


def start_clocks(torch, local):
    try:
        bus = torch.cuda.get_device_properties(local).pci_bus_id
    except Exception:
        bus = None
    s = ClockSampler(bus)
    s.start()
    return s


# -------------------------------------------------------------- helpers ------
def sources_hash(kind):
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def kernel_kind(kernel):
    if "k_solve_rows" in kernel and kernel.startswith("k_batch_tc"):
        return "split"
    if kernel.startswith("k_pipe_tc"):
        return "pipe"
    if kernel.startswith(("k_batch_tc", "k_fused_tc")):
        return "tc"
    if kernel.startswith(("k_batch_fd_small", "k_fd_small")):
        return "fdsmall"
    if kernel.startswith("k_solve_rows"):
        return "rows"
    return "fp32"


def traffic_per_launch(kernel, units):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (bytes per unit of its capture, scaled to this launch's units); None if
    missing or taken on other code."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)[kernel]
    except Exception:
        return None
    if t.get("sources_hash") != sources_hash(kernel_kind(kernel)):
        return None
    return t["dram_bytes_per_unit"] * units


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def rel_err_rows(Xg, Xr):
    """Per-subcarrier ||X_gpu - X_ref||_F / ||X_ref||_F (arrays [n][K][B])."""
    import numpy as np
    n = Xr.shape[0]
    d = np.linalg.norm((Xg.astype(np.complex128) - Xr).reshape(n, -1), axis=1)
    r = np.linalg.norm(Xr.reshape(n, -1), axis=1)
    return d / np.where(r > 0, r, 1.0)


def entry_err(Xg, Xr):
    """Largest entry error relative to the largest entry of the subcarrier."""
    import numpy as np
    n = Xr.shape[0]
    d = np.abs(Xg.astype(np.complex128) - Xr).reshape(n, -1).max(axis=1)
    r = np.abs(Xr).reshape(n, -1).max(axis=1)
    return d / np.where(r > 0, r, 1.0)


# --------------------------------------------------- the batched workload ----
def c4_shapes(synth, n):
    return synth.c4_instance_shapes(C4_INSTANCES, synth.seed_for(4))[:n]


def c4_inputs(torch, synth, shapes, seed):
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    Hs, Ss, Xs = [], [], []
    for sh in shapes:
        Hs.append(synth.torch_channel(sh["n_sc"], sh["B"], sh["U"], sh["channel"], gen, "cuda"))
        Ss.append(synth.torch_symbols(64, (sh["n_sc"], K_SYM, sh["U"]), gen, "cuda"))
        Xs.append(torch.empty((sh["n_sc"], K_SYM, sh["B"]), dtype=torch.complex64,
                              device="cuda"))
    return Hs, Ss, Xs


def c4_descs(synth, shapes, prec):
    N0 = synth.n0_from_snr(10.0)
    return [dict(U=sh["U"], B=sh["B"], C=sh["C"], n_sc=sh["n_sc"], K=K_SYM, mode=sh["mode"],
                 prec=prec, N0=N0, tau=0.125) for sh in shapes]


def alg_bytes_of(shapes):
    """H once, S and X per subcarrier (8UB + 8KU + 8KB), summed."""
    return sum(sh["n_sc"] * 8 * (sh["U"] * sh["B"] + K_SYM * sh["U"] + K_SYM * sh["B"])
               for sh in shapes)


def c4_sample(shapes, per_inst=8, stride=8):
    """The bounded sample the CPU oracle runs: every stride-th instance, per_inst
    consecutive subcarriers from a fixed offset inside it."""
    out = []
    for i in range(0, len(shapes), stride):
        n = shapes[i]["n_sc"]
        m = min(per_inst, n)
        lo = (i * 7919) % (n - m + 1)
        out.append((i, lo, lo + m))
    return out


def c4_workload_name(n):
    return (f"c4: {n} uneven instances, U {{8..64}}, B {{64..1024}}, C | B, n_sc U[72,3300], "
            f"K=14, 64-QAM, 10 dB, iid/Kronecker, PD-WF/FD-WF (tau 0.125)")


def measure_c4(args, dp, synth, torch, rank, world, local):
    """The headline: batched passes over the instances, graph-replayed, with
    per-bucket CUDA events inside the graph."""
    shapes = c4_shapes(synth, args.instances)
    Hs, Ss, Xs = c4_inputs(torch, synth, shapes, c4_rank_seed(synth, rank))
    stream = torch.cuda.current_stream()
    b = dp.Batch(c4_descs(synth, shapes, args.prec), stream=stream)
    b.tune(Hs, Ss, Xs, trials=3)
    timing = 1
    try:  # per-bucket events recorded from the graph; eager launches otherwise
        b.set_timing(1)
        b.precode(Hs, Ss, Xs)
        b.bucket_ms()
    except dp.DPError:
        timing = 2
        b.set_timing(2)
    for _ in range(args.warmup):
        b.precode(Hs, Ss, Xs)
    bad = [i for i, st in enumerate(b.status_get()) if not (st == 0).all()]
    assert not bad, f"batched pass reported failures in instances {bad[:8]}"
    info = b.describe()
    nb = len(info["buckets"])
    sampler = start_clocks(torch, local)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per_bucket = [[] for _ in range(nb)]
    t0.record(stream)
    for _ in range(args.steps):
        b.precode(Hs, Ss, Xs)
        for k, ms in enumerate(b.bucket_ms()):  # waits for the step
            per_bucket[k].append(ms)
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms_total = job_time_ms(t0.elapsed_time(t1), world, "cuda")
    n_sc = sum(sh["n_sc"] for sh in shapes)
    peak, peak_src = load_peaks()
    buckets = []
    for k, bk in enumerate(info["buckets"]):
        if not bk["items"]:
            continue
        mean = statistics.mean(per_bucket[k])
        fam, upad = bk["family"], bk["users_padded"]
        kern = (f"k_pipe_tc<{upad},{args.prec}>" if fam.startswith("tc_pipe")
                else f"k_batch_tc<{upad},{args.prec}> Gram + k_solve_rows<{upad}> + "
                     f"k_batch_tc<{upad},{args.prec}> apply"
                if fam.startswith("tc_split")
                else f"k_batch_tc<{upad},{args.prec}>" if fam.startswith("tc")
                else f"k_batch_fd_small<{upad}>" if fam == "fd_small_clusters"
                else f"k_batch_fused<{upad}>")
        buckets.append({"kernel": kern, "family": bk["family"], "systems": bk["systems"],
                        "items": bk["items"], "ctas_per_sm": bk["ctas_per_sm"],
                        "max_ctas_per_sm": bk["max_ctas_per_sm"], "tuned_ms": bk["tuned_ms"],
                        "launch_ms_mean": mean, "alg_bytes": bk["alg_bytes"],
                        "achieved_gbs": bk["alg_bytes"] / (mean / 1e3) / 1e9,
                        "frac": bk["alg_bytes"] / (mean / 1e3) / 1e9 / peak})
    dom = max(buckets, key=lambda x: x["launch_ms_mean"])
    roofline = {"bound": "hbm", "kernel": dom["kernel"], "achieved": dom["achieved_gbs"],
                "peak": peak, "peak_source": peak_src, "unit": "GB/s", "frac": dom["frac"],
                "traffic": traffic_per_launch(dom["kernel"], dom["systems"]),
                "algorithmic_bytes": dom["alg_bytes"], "launch_ms_mean": dom["launch_ms_mean"],
                "timing": "CUDA events around every bucket launch inside the replayed graph"
                          if timing == 1 else "CUDA events around eager bucket launches",
                "whole_pass": {"algorithmic_bytes": alg_bytes_of(shapes),
                               "achieved": alg_bytes_of(shapes) / (ms_total / args.steps / 1e3) / 1e9,
                               "frac": alg_bytes_of(shapes) / (ms_total / args.steps / 1e3) / 1e9
                               / peak}}
    out = {"value": job_rate(n_sc * args.steps, world, ms_total), "ms_per_step": ms_total / args.steps,
           "subcarriers": n_sc, "roofline": roofline, "buckets": buckets, "clocks": clocks,
           "gpu_launches": args.steps * sum(bk.get("launches", 1) for bk in info["buckets"]),
           "streaming_instances": info["streaming_instances"], "shapes": shapes}
    b.close()
    return out, Hs, Ss, Xs


def measure_c4_plain(args, dp, synth, torch, shapes, Hs, Ss):
    """The metric's denominator: the plain FP32 path, one plan per instance,
    instance after instance (every step of the path in FP32 on the SIMT cores)."""
    stream = torch.cuda.current_stream()
    N0 = synth.n0_from_snr(10.0)
    plans = [dp.Plan(sh["U"], sh["B"], sh["C"], sh["n_sc"], K_SYM, mode=sh["mode"], prec="fp32",
                     N0=N0, tau=0.125, stream=stream) for sh in shapes]
    Xp = [torch.empty((sh["n_sc"], K_SYM, sh["B"]), dtype=torch.complex64, device="cuda")
          for sh in shapes]
    for pl, H, S, X in zip(plans, Hs, Ss, Xp):
        pl.precode(H, S, X)
    reps = 2
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        for pl, H, S, X in zip(plans, Hs, Ss, Xp):
            pl.precode(H, S, X)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    for pl in plans:
        pl.close()
    n_sc = sum(sh["n_sc"] for sh in shapes)
    peak, _ = load_peaks()
    alg = alg_bytes_of(shapes)
    return {"value": n_sc / (ms / 1e3), "unit": "subcarriers/s", "ms_per_pass": ms,
            "dtype": "f32", "passes": reps,
            "roofline": {"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": alg / (ms / 1e3) / 1e9 / peak,
                         "note": "whole pass: algorithmic bytes over the pass's time"}}, Xp


def c4_cpu_baseline(args, synth, shapes, Hs, Ss, Xs, Xplain=None):
    """The FP64 oracle, as it stands, on a bounded sample of the timed inputs
    (the same subcarriers the GPU precoded); its outputs also give the error
    of the timed GPU outputs on that sample."""
    import numpy as np

    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    N0 = synth.n0_from_snr(10.0)
    sample = c4_sample(shapes)
    probs = []
    for i, lo, hi in sample:
        sh = shapes[i]
        H = Hs[i][lo:hi].cpu().numpy()
        S = Ss[i][lo:hi].cpu().numpy()
        probs.append((i, lo, hi, H, S, synth.equal_clusters(sh["B"], sh["C"]), sh["mode"]))

    def run_all():
        outs = []
        for i, lo, hi, H, S, cs, mode in probs:
            outs.append(oracle.precode(H, S, cs, mode, rho2=1.0, N0=N0, Es=1.0, tau=0.125,
                                       nthreads=cores, outputs=("X",))["X"])
        return outs

    per, outs = [], None
    t_end = time.perf_counter() + args.cpu_seconds
    while not per or time.perf_counter() < t_end:
        t0 = time.perf_counter()
        outs = run_all()
        per.append(time.perf_counter() - t0)
    nsub = sum(hi - lo for _, lo, hi, *_ in probs)
    err, eerr, errp = [], [], []
    for (i, lo, hi, *_), Xr in zip(probs, outs):
        Xg = Xs[i][lo:hi].cpu().numpy()
        err.append(rel_err_rows(Xg, Xr).max())
        eerr.append(entry_err(Xg, Xr).max())
        if Xplain is not None:
            errp.append(rel_err_rows(Xplain[i][lo:hi].cpu().numpy(), Xr).max())
    out = {"value": nsub * len(per) / sum(per), "unit": "subcarriers/s", "cores": cores,
           "kind": "oracle",
           "sample": f"{len(per)} x {nsub} subcarriers: {len(probs)} of the {len(shapes)} "
                     f"instances (every 8th), 8 consecutive subcarriers each, {cores} threads",
           "value_median": nsub / statistics.median(per),
           "rel_err_max": float(max(err)), "entry_err_max": float(max(eerr))}
    if errp:
        out["rel_err_max_plain_fp32"] = float(max(errp))
    return out


def c4_e2e(args, dp, synth, torch, shapes, Hs, Ss, world):
    """End to end through the public host-memory call (dp_precode_host): each
    instance's H and S are uploaded from pinned host memory, precoded and X
    read back inside the timed region, on a bounded set of the instances."""
    n = min(len(shapes), 48)
    sub = shapes[:n]
    stream = torch.cuda.current_stream()
    N0 = synth.n0_from_snr(10.0)
    plans = [dp.Plan(sh["U"], sh["B"], sh["C"], sh["n_sc"], K_SYM, mode=sh["mode"],
                     prec=args.prec, N0=N0, tau=0.125, stream=stream) for sh in sub]
    Hh = [Hs[i].cpu().pin_memory() for i in range(n)]
    Sh = [Ss[i].cpu().pin_memory() for i in range(n)]
    Xh = [torch.empty((sh["n_sc"], K_SYM, sh["B"]), dtype=torch.complex64).pin_memory()
          for sh in sub]

    def one():
        for pl, H, S, X, sh in zip(plans, Hh, Sh, Xh, sub):
            pl.precode_host(H, S, X, max(1, sh["n_sc"] // 4))

    one()
    torch.cuda.synchronize()
    steps = 3
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        one()
    b.record(stream)
    torch.cuda.synchronize()
    ms = job_time_ms(a.elapsed_time(b), world, "cuda") / steps
    for pl in plans:
        pl.close()
    n_sc = sum(sh["n_sc"] for sh in sub)
    return {"value": job_rate(n_sc, world, ms), "unit": "subcarriers/s",
            "h2d_bytes_per_step": sum(h.numel() * 8 + s.numel() * 8 for h, s in zip(Hh, Sh)),
            "d2h_bytes_per_step": sum(x.numel() * 8 for x in Xh), "steps": steps,
            "sample": f"the first {n} of the instances ({n_sc} subcarriers) per step, "
                      f"dp_precode_host with pinned buffers, 4 chunks per instance"}


# --------------------------------------------------- single-plan records ----
def measure_plan(dp, torch, stream, U, B, C, n_sc, K, mode, prec, N0, H, S, X, steps, warmup,
                 tau=0.125):
    plan = dp.Plan(U, B, C, n_sc, K, mode=mode, prec=prec, N0=N0, tau=tau, stream=stream)
    for _ in range(warmup):
        plan.precode(H, S, X)
    st = plan.status_get()
    assert (st == 0).all(), f"{prec}: precoding reported failures"
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(steps):
        ev[i][0].record(stream)
        plan.precode(H, S, X)
        ev[i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    return plan, t0.elapsed_time(t1), [a.elapsed_time(b) for a, b in ev]


def c2_kernel_name(prec):
    """The one kernel of a single-plan launch on the c2 workload (U = 16,
    K = 14): the FP32 fused kernel, or the warp-specialized tensor-core kernel."""
    return "k_fused<16>" if prec == "fp32" else f"k_pipe_tc<16,{prec}>"


def measure_c2(args, dp, synth, torch, rank, world, local, headline=False):
    """PD-WF (or ZF / FD-WF) on the U = 16, B = 256 slot: one dp_precode per
    step over `slots` slots of 1200 subcarriers."""
    import numpy as np
    w = C2
    slots = args.slots
    n_sc = w["n_sc"] * slots
    U, B, C, K = w["U"], w["B"], w["C"], w["K"]
    N0 = synth.n0_from_snr(w["snr_db"])
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(rank_seed(synth, rank))
    H = synth.torch_channel(n_sc, B, U, "iid", gen, "cuda")
    S = synth.torch_symbols(w["qam"], (n_sc, K, U), gen, "cuda")
    X = torch.empty((n_sc, K, B), dtype=torch.complex64, device="cuda")
    alg = n_sc * (B * U * 8 + K * U * 8 + K * B * 8)
    peak, peak_src = load_peaks()
    steps = args.steps if headline else min(args.steps, 20)

    def roof(prec, launch_ms):
        kern_s = statistics.mean(launch_ms) / 1e3
        return {"bound": "hbm", "kernel": c2_kernel_name(prec), "achieved": alg / kern_s / 1e9,
                "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                "frac": alg / kern_s / 1e9 / peak,
                "traffic": traffic_per_launch(c2_kernel_name(prec), n_sc),
                "algorithmic_bytes": alg, "launch_ms_mean": kern_s * 1e3}

    plain = None
    if not args.no_plain:
        Xp = torch.empty_like(X)
        pl, p_ms, p_launch = measure_plan(dp, torch, stream, U, B, C, n_sc, K, args.mode, "fp32",
                                          N0, H, S, Xp, steps, args.warmup)
        pl.close()
        plain = {"value": job_rate(n_sc * steps, world, p_ms), "unit": "subcarriers/s",
                 "ms_per_step": p_ms / steps, "dtype": "f32", "roofline": roof("fp32", p_launch)}
        del Xp
    sampler = start_clocks(torch, local) if headline else None
    if world > 1:
        torch.distributed.barrier()
    plan, ms, launch = measure_plan(dp, torch, stream, U, B, C, n_sc, K, args.mode, args.prec, N0,
                                    H, S, X, steps, args.warmup)
    clocks = sampler.stop() if sampler else None
    ms = job_time_ms(ms, world, "cuda")
    out = {"workload": f"c2: U={U} B={B} C={C}x32 n_sc={w['n_sc']}/slot x {slots} slots K={K} "
                       f"{w['qam']}-QAM SNR {w['snr_db']:g} dB iid Rayleigh, {args.mode}",
           "value": job_rate(n_sc * steps, world, ms), "unit": "subcarriers/s",
           "ms_per_step": ms / steps, "steps": steps, "prec": args.prec,
           "roofline": roof(args.prec, launch), "plain_fp32": plain, "clocks": clocks,
           "l2": f"inputs larger than L2 ({n_sc * (8 * U * B + 8 * K * U) / 1e6:.0f} MB per "
                 f"step vs 129 MB L2)"}
    if plain:
        out["speedup_vs_plain_fp32"] = out["value"] / plain["value"]
    if not args.no_library and rank == 0:
        out["library_pipeline"] = measure_library_pipeline(torch, H, S, N0, args.mode, steps,
                                                           args.warmup, X)
    e2e = None
    if not args.no_e2e and headline:
        Hh, Sh = H.cpu().pin_memory(), S.cpu().pin_memory()
        Xh = torch.empty(X.shape, dtype=X.dtype).pin_memory()
        for _ in range(2):
            plan.precode_host(Hh, Sh, Xh, w["n_sc"])
        torch.cuda.synchronize()
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_steps = max(3, min(steps, 10))
        a.record(stream)
        for _ in range(e_steps):
            plan.precode_host(Hh, Sh, Xh, w["n_sc"])
        b2.record(stream)
        torch.cuda.synchronize()
        e_ms = job_time_ms(a.elapsed_time(b2), world, "cuda")
        e2e = {"value": job_rate(n_sc * e_steps, world, e_ms), "unit": "subcarriers/s",
               "h2d_bytes_per_step": H.numel() * 8 + S.numel() * 8,
               "d2h_bytes_per_step": X.numel() * 8, "steps": e_steps}
        assert np.isfinite(Xh[:2].numpy()).all()
    out["e2e"] = e2e
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        sub = 240
        Hs, Ss = H[:sub].cpu().numpy(), S[:sub].cpu().numpy()
        cores = os.cpu_count() or 1
        per = []
        t_end = time.perf_counter() + (args.cpu_seconds if headline else 3.0)
        while not per or time.perf_counter() < t_end:
            t0 = time.perf_counter()
            Xr = oracle.precode(Hs, Ss, [B // C] * C, args.mode, rho2=1.0, N0=N0, Es=1.0,
                                tau=0.125, nthreads=cores, outputs=("X",))["X"]
            per.append(time.perf_counter() - t0)
        out["cpu_baseline"] = {"value": sub * len(per) / sum(per), "unit": "subcarriers/s",
                               "cores": cores, "kind": "oracle",
                               "sample": f"{len(per)} x the first {sub} subcarriers of the "
                                         f"timed input, {cores} threads",
                               "rel_err_max": float(rel_err_rows(X[:sub].cpu().numpy(), Xr).max()),
                               "entry_err_max": float(entry_err(X[:sub].cpu().numpy(), Xr).max())}
    plan.close()
    return out


def measure_c3(args, dp, synth, torch):
    """The precision workload: U = 32, B = 512, C = 16 clusters of 32, 3300
    subcarriers, K = 14, 64-QAM, 10 dB, PD-WF; BF16 and FP16 Gram on i.i.d. and
    Kronecker channels; throughput of one dp_precode and its error against the
    FP64 oracle on sampled subcarriers."""
    import oracle
    oracle.build()
    w = C3
    U, B, C, n_sc, K = w["U"], w["B"], w["C"], w["n_sc"], w["K"]
    N0 = synth.n0_from_snr(w["snr_db"])
    stream = torch.cuda.current_stream()
    peak, _ = load_peaks()
    alg = n_sc * (B * U * 8 + K * U * 8 + K * B * 8)
    recs = []
    for chan in ("iid", "kron"):
        gen = torch.Generator(device="cuda")
        gen.manual_seed(synth.seed_for(3, 10 if chan == "iid" else 11))
        H = synth.torch_channel(n_sc, B, U, chan, gen, "cuda")
        S = synth.torch_symbols(w["qam"], (n_sc, K, U), gen, "cuda")
        X = torch.empty((n_sc, K, B), dtype=torch.complex64, device="cuda")
        idx = list(range(0, n_sc, n_sc // 64))[:64]
        Hc, Sc = H[idx].cpu().numpy(), S[idx].cpu().numpy()
        Xr = oracle.precode(Hc, Sc, [B // C] * C, "wf", rho2=1.0, N0=N0, Es=1.0,
                            nthreads=os.cpu_count() or 1, outputs=("X",))["X"]
        for prec in ("bf16", "fp16", "fp32"):
            pl, ms, launch = measure_plan(dp, torch, stream, U, B, C, n_sc, K, "wf", prec, N0,
                                          H, S, X, 10, 3)
            pl.close()
            Xg = X[idx].cpu().numpy()
            kern_s = statistics.mean(launch) / 1e3
            recs.append({"channel": chan, "prec": prec, "value": n_sc * 10 / (ms / 1e3),
                         "unit": "subcarriers/s", "ms_per_step": ms / 10,
                         "hbm_frac_of_measured": alg / kern_s / 1e9 / peak,
                         "rel_err_max": float(rel_err_rows(Xg, Xr).max()),
                         "entry_err_max": float(entry_err(Xg, Xr).max()),
                         "error_sample": f"{len(idx)} subcarriers (every {n_sc // 64}th)"})
        del H, S, X
    return {"workload": f"c3: U={U} B={B} C={C}x32 n_sc={n_sc} K={K} 64-QAM 10 dB PD-WF",
            "records": recs}


def measure_library_pipeline(torch, H, S, N0, mode, steps, warmup, Xours):
    """The paper's own GPU design on the same workload, from vendor libraries
    through torch (Sec. IV-B): batched complex GEMM for the Grams
    (G = H H^H; the cluster sum is the full-array Gram, Sec. III-B), batched
    inverse of A = G + kappa I, t by Lemma 1, batched GEMMs for z = A^{-1} s
    and x = scale H^H z.  A context baseline beside the fused kernel, not a
    path of this library; WF/ZF only (the FD-WF per-cluster form is not
    timed here)."""
    if mode == "fdwf":
        return None
    n_sc, Bn, Un = H.shape
    kappa = 0.0 if mode == "zf" else Un * N0 / 1.0
    eye = torch.eye(Un, dtype=torch.complex64, device=H.device)

    def step():
        Hm = H.transpose(1, 2)                      # [n][U][B]: the paper's U x B H
        G = torch.matmul(Hm, Hm.conj().transpose(1, 2))
        T = torch.linalg.inv(G + kappa * eye)
        tr = torch.diagonal(T, dim1=1, dim2=2).real.sum(-1)
        fro = (T.abs() ** 2).sum((1, 2))
        scale = torch.rsqrt(tr - kappa * fro)       # rho = Es = 1
        Z = torch.matmul(T, S.transpose(1, 2))      # [n][U][K]
        Xm = torch.matmul(Hm.conj().transpose(1, 2), Z) * scale[:, None, None]
        return Xm.transpose(1, 2)                   # [n][K][B]

    for _ in range(warmup):
        X = step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        X = step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    diff = (X - Xours).abs().pow(2).sum((1, 2)).sqrt() / Xours.abs().pow(2).sum((1, 2)).sqrt()
    return {"value": n_sc / (ms / 1e3), "unit": "subcarriers/s", "ms_per_step": ms,
            "ops": "torch.matmul (cuBLAS batched CGEMM) x3, torch.linalg.inv (batched LU "
                   "inverse), elementwise t and scale",
            "rel_err_vs_ours_max": float(diff.max())}


# ---------------------------------------------------------------- serving ----
def serving_cells(synth, torch):
    """The serving cells: 32 cells whose sizes follow the batched
    configuration, two channel estimates and two symbol slots each."""
    shapes = synth.c4_instance_shapes(32, synth.seed_for(5))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(synth.seed_for(5, 1))
    cells = []
    for sh in shapes:
        Ha = synth.torch_channel(sh["n_sc"], sh["B"], sh["U"], sh["channel"], gen, "cuda")
        Hb = synth.torch_channel(sh["n_sc"], sh["B"], sh["U"], sh["channel"], gen, "cuda")
        Sp = [synth.torch_symbols(64, (sh["n_sc"], 14, sh["U"]), gen, "cuda") for _ in range(2)]
        cells.append((sh, Ha, Hb, Sp))
    return cells


def serve_run(dp, synth, cells, prec, rate, n, max_inflight=64, cache=False):
    """n Poisson arrivals at `rate` requests/s over the cells (each cell's
    channel switched every 5 of its slots); the server's statistics."""
    import numpy as np
    N0 = synth.n0_from_snr(10.0)
    srv = dp.Server(streams=16, max_inflight=max_inflight, arena_bytes=16 << 30,
                    auto_release=True, cache_solve=cache)
    ids = [srv.add_cell(dict(U=sh["U"], B=sh["B"], C=sh["C"], n_sc=sh["n_sc"], K=14,
                             mode=sh["mode"], prec=prec, N0=N0, tau=0.125), Ha)
           for sh, Ha, _, _ in cells]
    g = np.random.default_rng(int(rate))
    cell_of = g.integers(0, len(cells), n)
    t = np.cumsum(g.exponential(1.0 / rate, n)) if rate > 0 else np.zeros(n)
    count = np.zeros(len(cells), int)
    S_list, H_sw = [], []
    for c in cell_of:
        sh, Ha, Hb, Sp = cells[c]
        S_list.append(Sp[count[c] % 2])
        H_sw.append((Hb if (count[c] // 5) % 2 else Ha) if count[c] % 5 == 0 else None)
        count[c] += 1
    # warm-up pass (kernel attributes, first launches)
    srv.replay([ids[c] for c in cell_of[:64]], S_list[:64], np.zeros(min(64, n)))
    srv.reset_stats()
    srv.replay([ids[c] for c in cell_of], S_list, t, H_sw)
    st = srv.stats()
    srv.close()
    st["offered_subcarriers_per_s"] = (
        rate * float(np.mean([cells[c][0]["n_sc"] for c in cell_of])) if rate > 0 else None)
    return st


def measure_serving(dp, synth, torch, n_req):
    """Serving: Poisson arrivals of per-slot requests over 32 cells whose sizes
    follow the batched configuration, 14 symbols per slot, each cell's channel
    switched to a fresh device-resident estimate every 5 of its slots,
    admission by free arena memory; p50 / p99 latency and throughput per
    arrival rate, FP16 Gram cells, and the plain FP32 path one request at a
    time for comparison."""
    cells = serving_cells(synth, torch)
    out = {"workload": "32 cells sized as the batched configuration, K=14, channel switched "
                       "every 5 slots", "rates": []}

    def run(prec, rate, n, max_inflight=64, cache=False):
        return serve_run(dp, synth, cells, prec, rate, n, max_inflight, cache)

    for rate in (2000, 5000, 10000, 20000, 40000):
        st = run("fp16", rate, n_req)
        out["rates"].append({"req_per_s": rate, "requests": st["completed"],
                             "failed": st["failed"], "p50_ms": st["p50_ms"],
                             "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
                             "subcarriers_per_s": st["subcarriers"] / max(st["wall_s"], 1e-9),
                             "inflight_peak": st["inflight_peak"]})
    # the per-channel solve cache (FP32 Gram, inverse and scale once per
    # channel; every request only whitens and applies, in FP32)
    out["cached_fp32"] = []
    for rate in (2000, 10000, 40000):
        st = run("fp32", rate, n_req, cache=True)
        out["cached_fp32"].append({"req_per_s": rate, "requests": st["completed"],
                                   "failed": st["failed"], "p50_ms": st["p50_ms"],
                                   "p99_ms": st["p99_ms"],
                                   "subcarriers_per_s": st["subcarriers"] / max(st["wall_s"], 1e-9),
                                   "inflight_peak": st["inflight_peak"]})
    # plain FP32 path, one request at a time (no overlap): its throughput bound
    st = run("fp32", 0, min(n_req, 600), max_inflight=1)
    out["plain_fp32_per_request"] = {"subcarriers_per_s": st["subcarriers"] / max(st["wall_s"], 1e-9),
                                     "note": "all requests submitted at t=0, one in flight",
                                     "p50_ms": st["p50_ms"]}
    return out


def serving_burst(n):
    """N requests submitted at t = 0 to the solve-cached FP32 server over the
    32 serving cells (shapes of the batched configuration, K = 14, i.i.d.
    channels, one channel per cell): throughput and latency of a burst."""
    import numpy as np
    import torch

    from paper_1804_10987_gb300 import dp, synth
    shapes = synth.c4_instance_shapes(32, synth.seed_for(5))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(synth.seed_for(5, 1))
    N0 = synth.n0_from_snr(10.0)
    cells = []
    for sh in shapes:
        H = synth.torch_channel(sh["n_sc"], sh["B"], sh["U"], "iid", gen, "cuda")
        S = synth.torch_symbols(64, (sh["n_sc"], 14, sh["U"]), gen, "cuda")
        cells.append((sh, H, S))
    srv = dp.Server(streams=16, max_inflight=64, arena_bytes=16 << 30, auto_release=True,
                    cache_solve=True)
    ids = [srv.add_cell(dict(U=sh["U"], B=sh["B"], C=sh["C"], n_sc=sh["n_sc"], K=14,
                             mode=sh["mode"], prec="fp32", N0=N0, tau=0.125), H)
           for sh, H, _ in cells]
    cell_of = np.random.default_rng(1).integers(0, len(cells), n)
    srv.replay([ids[c] for c in cell_of], [cells[c][2] for c in cell_of], np.zeros(n))
    st = srv.stats()
    srv.close()
    print(json.dumps({"serving_burst": n, "cache_solve": True, "prec": "fp32",
                      "subcarriers_per_s": st["subcarriers"] / max(st["wall_s"], 1e-9),
                      "wall_ms": st["wall_s"] * 1e3, "p50_ms": st["p50_ms"],
                      "p99_ms": st["p99_ms"], "failed": st["failed"]}))


# ------------------------------------------------------- reference arm ------
def reference_arm(args):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of
    the headline workload per step (every 8th instance's shape, 8 subcarriers
    each, drawn on the host with the same recipe)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle

    from paper_1804_10987_gb300 import synth
    oracle.build()
    cores = os.cpu_count() or 1
    N0 = synth.n0_from_snr(10.0)
    if args.workload == "c2":
        w = C2
        probs = [synth.make_problem(w["U"], w["B"], w["C"], 240, w["K"], w["qam"], w["snr_db"],
                                    seed=synth.seed_for(2, 100), mode=args.mode)]
        workload = f"c2 sample: 240 subcarriers of the U=16 B=256 slot, {args.mode}"
    else:
        shapes = c4_shapes(synth, args.instances)
        probs = []
        for i, lo, hi in c4_sample(shapes):
            sh = shapes[i]
            probs.append(synth.make_problem(sh["U"], sh["B"], sh["C"], hi - lo, K_SYM, 64, 10.0,
                                            seed=synth.seed_for(4, 5000 + i), mode=sh["mode"],
                                            channel=sh["channel"]))
        workload = c4_workload_name(len(shapes))
    nsub = sum(p.n_sc for p in probs)

    def step():
        for p in probs:
            oracle.precode(p.H, p.S, p.cluster_sizes, p.mode, rho2=1.0, N0=N0, Es=1.0, tau=0.125,
                           nthreads=cores, outputs=("X",))

    for _ in range(max(1, args.warmup)):
        step()
    per = []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        step()
        per.append(time.perf_counter() - t0)
    rate = nsub * len(per) / sum(per)
    sample = (f"per step {nsub} subcarriers: every 8th instance's shape, 8 subcarriers each, "
              f"drawn on the host; {cores} threads") if args.workload == "c4" else \
        f"per step 240 subcarriers, {cores} threads"
    line = {"impl": "reference", "metric": metric_name(args), "value": rate,
            "unit": "subcarriers/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(per) / len(per),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload, "prec": "f64 oracle",
                       "l2": "host run of the CPU oracle (no GPU caches involved)",
                       "subcarriers_per_step": nsub, "parallelism": "host threads"},
            "cpu_baseline": {"value": rate, "unit": "subcarriers/s", "cores": cores,
                             "kind": "oracle", "sample": sample,
                             "value_median": nsub / statistics.median(per)},
            "e2e": {"value": rate, "unit": "subcarriers/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def metric_name(args):
    if args.workload == "c2":
        return (f"precoded subcarriers/s ({args.mode.upper()}, U=16 B=256 C=8 K=14, "
                f"complex64 I/O)")
    return ("precoded subcarriers/s of the batched uneven workload (reduced precision, "
            "<= 1e-3 rel err) vs the plain FP32 per-instance path")


# --------------------------------------------------------------- our arm ----
def our_arm(args):
    import torch
    import torch.distributed as dist

    from paper_1804_10987_gb300 import dp, synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    if args.workload == "c2":
        rec = measure_c2(args, dp, synth, torch, rank, world, local, headline=True)
        if rank == 0:
            line = {"metric": metric_name(args), "value": rec["value"], "unit": "subcarriers/s",
                    "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                    "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
                    "scaling": "weak", "vs_baseline": None,
                    "dtype": DTYPE_TC.replace("fp16", args.prec, 1), "data": "synthetic",
                    "config": {"workload": rec["workload"], "prec": args.prec,
                               "slots_per_step": args.slots,
                               "subcarriers_per_step": C2["n_sc"] * args.slots,
                               "l2": rec["l2"], "parallelism": f"replicas x{world}"},
                    "roofline": rec["roofline"], "cpu_baseline": rec.get("cpu_baseline"),
                    "e2e": rec["e2e"], "clocks": rec["clocks"],
                    # per step: the warp-specialized kernel and the escalation
                    # fix-up launch (automatic escalation is the default)
                    "gpu_launches": 2 * args.steps,
                    "plain_fp32": rec["plain_fp32"],
                    "library_pipeline": rec.get("library_pipeline"),
                    "paper_context": PAPER_CONTEXT}
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    head, Hs, Ss, Xs = measure_c4(args, dp, synth, torch, rank, world, local)
    shapes = head["shapes"]
    plain = Xplain = None
    if not args.no_plain:
        plain, Xplain = measure_c4_plain(args, dp, synth, torch, shapes, Hs, Ss)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = c4_cpu_baseline(args, synth, shapes, Hs, Ss, Xs, Xplain)
    del Xplain
    torch.cuda.empty_cache()
    e2e = None
    if not args.no_e2e:
        e2e = c4_e2e(args, dp, synth, torch, shapes, Hs, Ss, world)
    del Hs, Ss, Xs
    torch.cuda.empty_cache()
    c2 = c3 = serving = None
    if rank == 0 and world == 1:
        if not args.no_c2:
            c2 = measure_c2(args, dp, synth, torch, rank, world, local)
            torch.cuda.empty_cache()
        if not args.no_c3:
            c3 = measure_c3(args, dp, synth, torch)
            torch.cuda.empty_cache()
        if not args.no_serving:
            serving = measure_serving(dp, synth, torch, args.serve_requests)
    if rank == 0:
        n = len(shapes)
        line = {"metric": metric_name(args), "value": head["value"], "unit": "subcarriers/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": head["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE_TC.replace("fp16", args.prec, 1), "data": "synthetic",
                "config": {"workload": c4_workload_name(n), "instances": n,
                           "subcarriers_per_step": head["subcarriers"], "prec": args.prec,
                           "launch": "persistent bucket launches replayed from a CUDA graph, "
                                     "CTAs per SM from the autotuner",
                           "l2": f"inputs larger than L2 ({alg_bytes_of(shapes) / 1e9:.0f} GB "
                                 f"algorithmic per step vs 129 MB L2)",
                           "parallelism": f"replicas x{world}"},
                "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": e2e,
                "clocks": head["clocks"], "gpu_launches": head["gpu_launches"],
                "plain_fp32": plain,
                "speedup_vs_plain_fp32": head["value"] / plain["value"] if plain else None,
                "rel_err_max": cpu["rel_err_max"] if cpu else None,
                "buckets": head["buckets"],
                "streaming_instances": head["streaming_instances"],
                "vectors_per_s": head["value"] * K_SYM,
                "c2": c2, "c3": c3, "serving": serving, "paper_context": PAPER_CONTEXT}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def serving_knee(n_long, n_short):
    """Steady-state serving: for each arrival rate, n_short and n_long Poisson
    requests to the uncached reduced-precision (FP16 Gram) server and to the
    solve-cached FP32 server. A rate is sustained when the server delivers at
    least 95 % of the offered subcarriers/s and its p99 stays flat as the run
    grows (p99 of n_long requests within 1.5x that of n_short); the knee is
    the highest sustained rate. One JSON line."""
    import torch

    from paper_1804_10987_gb300 import dp, synth
    cells = serving_cells(synth, torch)
    rates = (1000, 1500, 2000, 2500, 3000, 3500)
    out = {"serving_knee": True, "requests": [n_short, n_long],
           "workload": "32 cells sized as the batched configuration, K=14, channel switched "
                       "every 5 slots", "target_p99_ms": 0.5}
    for name, prec, cache in (("uncached_fp16", "fp16", False), ("cached_fp32", "fp32", True)):
        recs, knee = [], None
        for rate in rates:
            r = {"req_per_s": rate}
            for n in (n_short, n_long):
                st = serve_run(dp, synth, cells, prec, rate, n, cache=cache)
                served = st["subcarriers"] / max(st["wall_s"], 1e-9)
                r[str(n)] = {"p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
                             "failed": st["failed"], "subcarriers_per_s": served,
                             "offered_subcarriers_per_s": st["offered_subcarriers_per_s"],
                             "inflight_peak": st["inflight_peak"]}
            lo, hi = r[str(n_short)], r[str(n_long)]
            r["sustained"] = bool(hi["subcarriers_per_s"] >= 0.95 * hi["offered_subcarriers_per_s"]
                                  and hi["p99_ms"] <= 1.5 * lo["p99_ms"] and hi["failed"] == 0)
            recs.append(r)
            if r["sustained"]:
                knee = rate
            elif knee is not None:
                break  # past the knee: the queue grows with the run
        out[name] = {"rates": recs, "knee_req_per_s": knee}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    elif args.serving_burst > 0:
        serving_burst(args.serving_burst)
    elif args.serving_knee > 0:
        serving_knee(args.serving_knee, max(1, args.serving_knee // 4))
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
