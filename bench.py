#!/usr/bin/env python
"""Throughput of the feedforward decentralized precoding path on GB300.

Workload (one rank): PD-WF precoding of the 20 MHz LTE-like slot with U = 16
users, B = 256 antennas in C = 8 clusters of 32, 1200 subcarriers x K = 14
OFDM symbols, 16-QAM, SNR 10 dB, i.i.d. Rayleigh channel, complex64.  One
step is one dp_precode call over `--slots` such slots (default 8, so that a
step's inputs, 331 MB, exceed the 129 MB L2 and every step streams from HBM).
Metric: precoded subcarriers per second (each subcarrier carries K vectors).

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torchrun, one rank per GPU, each rank precoding its own slots (replicas:
subcarriers are independent, no collective on the data path).
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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="c2", U=16, B=256, C=8, n_sc=1200, K=14, qam=16, snr_db=10.0)
KERNEL_SOURCES = {
    "fp32": ["paper_1804_10987_gb300/csrc/dp_fp32.cu", "paper_1804_10987_gb300/csrc/dp_blocks.cuh",
             "paper_1804_10987_gb300/csrc/dp_common.cuh"],
    "tc": ["paper_1804_10987_gb300/csrc/dp_tcpipe.cu", "paper_1804_10987_gb300/csrc/dp_tc.cuh",
           "paper_1804_10987_gb300/csrc/dp_blocks.cuh", "paper_1804_10987_gb300/csrc/dp_common.cuh"],
}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["wf", "zf", "fdwf"], default="wf")
    ap.add_argument("--prec", choices=["fp32", "bf16", "fp16"], default="fp16",
                    help="Gram arithmetic of the headline path")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip timing the plain FP32 path beside the headline path")
    ap.add_argument("--slots", type=int, default=8, help="slots of 1200 subcarriers per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-library", action="store_true",
                    help="skip the paper-style library pipeline (context baseline)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="bound of the CPU oracle sample")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched uneven workload (512 instances)")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving sweep (Poisson arrivals)")
    ap.add_argument("--serve-requests", type=int, default=1500,
                    help="requests per arrival rate in the serving sweep")
    ap.add_argument("--serving-burst", type=int, default=0, metavar="N",
                    help="only this: N requests submitted at once to the solve-cached FP32 "
                         "server over the serving cells (i.i.d. channels); one JSON line")
    return ap.parse_args()


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
    """Seed of a rank's input shard: every rank precodes its own slots."""
    return synth.seed_for(2, 500 + rank)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def metric_name(mode):
    return f"precoded subcarriers/s ({mode.upper()}, U=16 B=256 C=8 K=14, complex64 I/O)"


def kernel_name(prec):
    """The one kernel of a single-plan launch on this workload (U = 16, K = 14):
    the FP32 fused kernel, or the warp-specialized tensor-core kernel."""
    return "k_fused<16>" if prec == "fp32" else f"k_pipe_tc<16,{'bf16' if prec == 'bf16' else 'fp16'}>"


def config_dict(args, world, slots):
    w = WORKLOAD
    return {"workload": f"c2: U={w['U']} B={w['B']} C={w['C']}x32 n_sc={w['n_sc']}/slot "
                        f"K={w['K']} {w['qam']}-QAM SNR {w['snr_db']:g} dB iid Rayleigh",
            "mode": args.mode, "prec": args.prec, "slots_per_step": slots,
            "subcarriers_per_step": w["n_sc"] * slots,
            "l2": l2_note(slots),
            "parallelism": f"replicas x{world}"}


def l2_note(slots):
    """Whether one step's inputs (H and S of every slot) exceed the 129 MB L2,
    so that timed steps read HBM without an L2 flush."""
    w = WORKLOAD
    mb = slots * w["n_sc"] * (8 * w["U"] * w["B"] + 8 * w["K"] * w["U"]) / 1e6
    rel = "larger than" if mb > 129 else "not larger than"
    return f"inputs {rel} L2 ({mb:.0f} MB per step of {slots} slots vs 129 MB L2)"


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


# ------------------------------------------------------------ CPU oracle -----
def make_slot_host(slot_index: int, mode: str):
    from paper_1804_10987_gb300 import synth
    w = WORKLOAD
    return synth.make_problem(w["U"], w["B"], w["C"], w["n_sc"], w["K"], w["qam"], w["snr_db"],
                              seed=synth.seed_for(2, 100 + slot_index), mode=mode)


def rel_err_max(Xg, Xr):
    import numpy as np
    n = Xr.shape[0]
    d = np.linalg.norm((Xg.astype(np.complex128) - Xr).reshape(n, -1), axis=1)
    r = np.linalg.norm(Xr.reshape(n, -1), axis=1)
    return float((d / np.where(r > 0, r, 1.0)).max())


def cpu_oracle_rate(mode: str, seconds: float, steps=None, problem=None):
    """Time the FP64 oracle, as it stands, on the host cores: slots of 1200
    subcarriers until `seconds` elapse (or `steps` slots).  Returns
    (subcarriers/s, cores, sample description, per-step seconds, X of the slot)."""
    import oracle
    p = problem if problem is not None else make_slot_host(0, mode)
    cores = os.cpu_count() or 1
    oracle.build()
    per = []
    t_end = time.perf_counter() + seconds
    while True:
        t0 = time.perf_counter()
        out = oracle.precode(p.H, p.S, p.cluster_sizes, mode, rho2=p.rho2, N0=p.N0, Es=p.Es,
                             tau=p.tau, nthreads=cores, outputs=("X",))
        per.append(time.perf_counter() - t0)
        if steps is not None and len(per) >= steps:
            break
        if steps is None and time.perf_counter() >= t_end:
            break
    rate = p.n_sc * len(per) / sum(per)
    sample = (f"{len(per)} x one slot of {p.n_sc} subcarriers (U=16, B=256, K=14, {mode}), "
              f"{cores} threads")
    return rate, cores, sample, per, out["X"]


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cpu_oracle_rate(args.mode, 0.0, steps=max(1, args.warmup))
    rate, cores, sample, per, _ = cpu_oracle_rate(args.mode, 0.0, steps=max(1, args.steps))
    ms = 1e3 * sum(per) / len(per)
    line = {"impl": "reference", "metric": metric_name(args.mode), "value": rate,
            "unit": "subcarriers/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(config_dict(args, 1, 1), slots_per_step=1, prec="f64 oracle",
                           l2="host run of the CPU oracle (no GPU caches involved)",
                           subcarriers_per_step=WORKLOAD["n_sc"]),
            "cpu_baseline": {"value": rate, "unit": "subcarriers/s", "cores": cores,
                             "kind": "oracle", "sample": sample,
                             "value_median": WORKLOAD["n_sc"] / statistics.median(per)},
            "e2e": {"value": rate, "unit": "subcarriers/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------- our arm ---------
def sources_hash(kind):
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_per_launch(kernel, subcarriers_per_launch):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled
    by subcarriers; None if missing or taken on other code."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)[kernel]
    except Exception:
        return None
    kind = "fp32" if kernel.startswith("k_fused<") else "tc"
    if t.get("sources_hash") != sources_hash(kind):
        return None
    return t["dram_bytes_per_subcarrier"] * subcarriers_per_launch


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


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


def measure_batched(dp, synth, torch):
    """Batched uneven workload: 512 instances (U, B, C, n_sc drawn from the
    batched configuration's sets, K = 14, 64-QAM, mixed i.i.d. / Kronecker,
    WF / FD-WF, 10 dB), FP16 Gram, persistent bucket launches in a CUDA graph,
    tuned; against the plain FP32 path run instance by instance."""
    shapes = synth.c4_instance_shapes(512, synth.seed_for(4))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(synth.seed_for(4, 1))
    N0 = synth.n0_from_snr(10.0)
    descs, Hs, Ss, Xs = [], [], [], []
    for sh in shapes:
        Hs.append(synth.torch_channel(sh["n_sc"], sh["B"], sh["U"], sh["channel"], gen, "cuda"))
        Ss.append(synth.torch_symbols(64, (sh["n_sc"], 14, sh["U"]), gen, "cuda"))
        Xs.append(torch.empty((sh["n_sc"], 14, sh["B"]), dtype=torch.complex64, device="cuda"))
        descs.append(dict(U=sh["U"], B=sh["B"], C=sh["C"], n_sc=sh["n_sc"], K=14,
                          mode=sh["mode"], prec="fp16", N0=N0, tau=0.125))
    n_sc = sum(sh["n_sc"] for sh in shapes)
    alg = sum(sh["n_sc"] * (sh["B"] * sh["U"] * 8 + 14 * sh["U"] * 8 + 14 * sh["B"] * 8)
              for sh in shapes)
    stream = torch.cuda.current_stream()
    b = dp.Batch(descs, stream=stream)
    b.tune(Hs, Ss, Xs, trials=1)
    for _ in range(2):
        b.precode(Hs, Ss, Xs)
    assert all((st == 0).all() for st in b.status_get())
    reps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        b.precode(Hs, Ss, Xs)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    info = b.describe()
    b.close()
    # plain FP32 path, one instance (one plan) at a time
    plans = [dp.Plan(d["U"], d["B"], d["C"], d["n_sc"], 14, mode=d["mode"], prec="fp32", N0=N0,
                     tau=0.125, stream=stream) for d in descs]
    for pl, H, S, X in zip(plans, Hs, Ss, Xs):
        pl.precode(H, S, X)
    e0.record(stream)
    for pl, H, S, X in zip(plans, Hs, Ss, Xs):
        pl.precode(H, S, X)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    for pl in plans:
        pl.close()
    del Hs, Ss, Xs
    torch.cuda.empty_cache()
    return {"workload": "512 uneven instances: U {8..64}, B {64..1024}, C | B, n_sc U[72,3300], "
                        "K=14, 64-QAM, iid/Kronecker, WF/FD-WF, 10 dB",
            "subcarriers": n_sc, "prec": "fp16 Gram", "ms_per_pass": ms,
            "value": n_sc / (ms / 1e3), "unit": "subcarriers/s",
            "hbm_frac_of_measured": alg / (ms / 1e3) / 1e9 / load_peaks()[0],
            "plain_fp32_per_instance": {"ms_per_pass": ms_plain,
                                        "value": n_sc / (ms_plain / 1e3)},
            "speedup_vs_plain_fp32": ms_plain / ms, "buckets": info["buckets"],
            "streaming_instances": info["streaming_instances"]}


def measure_serving(dp, synth, torch, n_req):
    """Serving: Poisson arrivals of per-slot requests over 32 cells whose sizes
    follow the batched configuration, 14 symbols per slot, each cell's channel
    switched to a fresh device-resident estimate every 5 of its slots,
    admission by free arena memory; p50 / p99 latency and throughput per
    arrival rate, FP16 Gram cells, and the plain FP32 path one request at a
    time for comparison."""
    import numpy as np
    shapes = synth.c4_instance_shapes(32, synth.seed_for(5))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(synth.seed_for(5, 1))
    N0 = synth.n0_from_snr(10.0)
    cells = []
    for sh in shapes:
        Ha = synth.torch_channel(sh["n_sc"], sh["B"], sh["U"], sh["channel"], gen, "cuda")
        Hb = synth.torch_channel(sh["n_sc"], sh["B"], sh["U"], sh["channel"], gen, "cuda")
        Sp = [synth.torch_symbols(64, (sh["n_sc"], 14, sh["U"]), gen, "cuda") for _ in range(2)]
        cells.append((sh, Ha, Hb, Sp))
    out = {"workload": "32 cells sized as the batched configuration, K=14, channel switched "
                       "every 5 slots", "rates": []}

    def run(prec, rate, n, max_inflight=64, cache=False):
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
        return st

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


def our_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1804_10987_gb300 import dp, synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = WORKLOAD
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

    def barrier():
        if world > 1:
            dist.barrier()

    def time_path(prec, Xout, sample_clocks):
        plan = dp.Plan(U, B, C, n_sc, K, mode=args.mode, prec=prec, N0=N0, tau=0.125,
                       stream=stream)
        for _ in range(args.warmup):
            plan.precode(H, S, Xout)
        st = plan.status_get()
        assert (st == 0).all(), f"{prec}: precoding reported failures"
        sampler = None
        if sample_clocks:
            bus = None
            try:
                bus = torch.cuda.get_device_properties(local).pci_bus_id
            except Exception:
                bus = None
            sampler = ClockSampler(bus)
            sampler.start()
        torch.cuda.synchronize()
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            plan.precode(H, S, Xout)
            ev[i][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clocks = sampler.stop() if sampler else None
        ms_total = job_time_ms(t0.elapsed_time(t1), world, "cuda")
        launch_ms = [a.elapsed_time(b) for a, b in ev]
        return plan, ms_total, launch_ms, clocks

    # algorithmic bytes of one launch: H once + S + X
    alg_bytes = n_sc * (B * U * 8 + K * U * 8 + K * B * 8)
    peak, peak_src = load_peaks()

    def roofline_of(prec, launch_ms):
        kern_s = statistics.mean(launch_ms) / 1e3
        achieved = alg_bytes / kern_s / 1e9
        return {"bound": "hbm", "kernel": kernel_name(prec), "achieved": achieved, "peak": peak,
                "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_per_launch(kernel_name(prec), n_sc),
                "algorithmic_bytes": alg_bytes, "launch_ms_mean": kern_s * 1e3}

    plain = None
    X_plain = None
    if args.prec != "fp32" and not args.no_plain:
        X_plain = torch.empty_like(X)
        pplan, p_ms, p_launch, _ = time_path("fp32", X_plain, False)
        pplan.close()
        plain = {"value": job_rate(n_sc * args.steps, world, p_ms), "unit": "subcarriers/s",
                 "ms_per_step": p_ms / args.steps, "dtype": "f32",
                 "roofline": roofline_of("fp32", p_launch)}
    plan, ms_total, launch_ms, clocks = time_path(args.prec, X, True)
    ms_step = ms_total / args.steps
    value = job_rate(n_sc * args.steps, world, ms_total)
    roofline = roofline_of(args.prec, launch_ms)
    library = None
    if not args.no_library:
        library = measure_library_pipeline(torch, H, S, N0, args.mode, args.steps, args.warmup, X)

    # end to end through the public call with host buffers
    e2e = None
    if not args.no_e2e:
        Hh = H.cpu().pin_memory()
        Sh = S.cpu().pin_memory()
        Xh = torch.empty(X.shape, dtype=X.dtype).pin_memory()
        e_steps = max(3, min(args.steps, 10))
        # dp_precode_host: chunked uploads of H and S, kernels and downloads
        # of X overlap on the plan's staging ring (one slot per chunk)
        for _ in range(2):
            plan.precode_host(Hh, Sh, Xh, WORKLOAD["n_sc"])
        torch.cuda.synchronize()
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(e_steps):
            plan.precode_host(Hh, Sh, Xh, WORKLOAD["n_sc"])
        b.record(stream)
        torch.cuda.synchronize()
        e_ms = job_time_ms(a.elapsed_time(b), world, "cuda")
        e2e = {"value": job_rate(n_sc * e_steps, world, e_ms), "unit": "subcarriers/s",
               "h2d_bytes_per_step": H.numel() * 8 + S.numel() * 8,
               "d2h_bytes_per_step": X.numel() * 8, "steps": e_steps}
        assert np.isfinite(Xh[:2].numpy()).all()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on the first slot of the timed input; its outputs also give
        # the relative error of the timed GPU outputs on that slot
        Hs = H[: w["n_sc"]].cpu().numpy()
        Ss = S[: w["n_sc"]].cpu().numpy()
        slot = synth.Problem(U, B, [B // C] * C, w["n_sc"], K, Hs, Ss, 1.0, N0, 1.0, 0.125,
                             args.mode)
        rate, cores, sample, per, Xref = cpu_oracle_rate(args.mode, args.cpu_seconds, problem=slot)
        cpu = {"value": rate, "unit": "subcarriers/s", "cores": cores, "kind": "oracle",
               "sample": sample, "value_median": w["n_sc"] / statistics.median(per),
               "rel_err_max": rel_err_max(X[: w["n_sc"]].cpu().numpy(), Xref)}
        if X_plain is not None:
            cpu["rel_err_max_plain_fp32"] = rel_err_max(X_plain[: w["n_sc"]].cpu().numpy(), Xref)
        # the same oracle on one host thread, over the slot's first 120 subcarriers
        import oracle
        sub, per1 = 120, []
        t_end = time.perf_counter() + min(3.0, args.cpu_seconds)
        while not per1 or time.perf_counter() < t_end:
            t0 = time.perf_counter()
            oracle.precode(Hs[:sub], Ss[:sub], slot.cluster_sizes, args.mode, rho2=1.0, N0=N0,
                           Es=1.0, tau=0.125, nthreads=1, outputs=("X",))
            per1.append(time.perf_counter() - t0)
        cpu["value_1_thread"] = sub * len(per1) / sum(per1)
        cpu["sample_1_thread"] = f"{len(per1)} x the slot's first {sub} subcarriers, 1 thread"

    plan.close()
    del H, S, X, X_plain
    torch.cuda.empty_cache()
    batched = serving = None
    if rank == 0 and world == 1 and not args.no_batched:
        batched = measure_batched(dp, synth, torch)
    if rank == 0 and world == 1 and not args.no_serving:
        serving = measure_serving(dp, synth, torch, args.serve_requests)
    if rank == 0:
        line = {"metric": metric_name(args.mode), "value": value, "unit": "subcarriers/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None,
                "dtype": "f32" if args.prec == "fp32" else f"{args.prec} Gram (tensor cores, f32 "
                                                          "accumulate) + f32 solve/apply",
                "data": "synthetic",
                "config": config_dict(args, world, slots), "roofline": roofline,
                "plain_fp32": plain,
                "speedup_vs_plain_fp32": (value / plain["value"]) if plain else None,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
                "library_pipeline": library,
                "clocks": clocks, "batched": batched, "serving": serving,
                "vectors_per_s": value * K,
                "paper_context": "PD-WF U=16 B=256 C=8 on 8 V100 (one per cluster), K=7: "
                                 "0.607 ms per 1200-subcarrier slot = 1.98 M subcarriers/s"}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    elif args.serving_burst > 0:
        serving_burst(args.serving_burst)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
