"""Thin Python binding of the C ABI in include/dprecode.h (argument marshalling
only: every step of the precoding path runs in the CUDA library).

Tensors are torch CUDA tensors, complex64 (or float32 for ``scale``), C-
contiguous, in the layouts the header states:
  H [n_sc][B][U], S [n_sc][K][U], X [n_sc][K][B], G [n_sc][U][U],
  Gloc [C][n_sc][U][U], Z [n_sc][K][U] (FD: [n_sc][C][K][U]),
  scale [n_sc] (FD: [n_sc][C]).
Calls enqueue on the plan's stream (by default torch's current stream at plan
creation) and return immediately.  There is no fallback: if the library is
missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

OK, INVALID_ARG, PARTITION, UNSUPPORTED, OOM, CUDA, NOT_PD, NONFINITE, TIMEOUT = range(9)
MODES = {"zf": 0, "wf": 1, "fdwf": 2, "mrt": 3}
PRECISIONS = {"fp32": 0, "bf16": 1, "fp16": 2}

_lock = threading.Lock()
_lib = None


class DPError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {status_string(code)} ({code})")
        self.code = code


class PlanDesc(ctypes.Structure):
    _fields_ = [("U", ctypes.c_int), ("B", ctypes.c_int), ("C", ctypes.c_int),
                ("cluster_sizes", ctypes.POINTER(ctypes.c_int)),
                ("n_sc", ctypes.c_int), ("K", ctypes.c_int),
                ("mode", ctypes.c_int), ("prec", ctypes.c_int),
                ("rho2", ctypes.c_float), ("N0", ctypes.c_float), ("Es", ctypes.c_float),
                ("tau", ctypes.c_float), ("refine", ctypes.c_int),
                ("cluster_power", ctypes.POINTER(ctypes.c_float))]


class ServerConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("streams", ctypes.c_int), ("max_inflight", ctypes.c_int),
                ("arena_bytes", ctypes.c_size_t), ("auto_release", ctypes.c_int),
                ("cache_solve", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("subcarriers", ctypes.c_longlong), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("wall_s", ctypes.c_double),
                ("inflight_peak", ctypes.c_int), ("arena_high_water", ctypes.c_longlong)]


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load libdprecode.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; run paper_1804_10987_gb300.build")
        L = ctypes.CDLL(path)
        P, I, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        L.dp_plan_create.argtypes = [ctypes.POINTER(PlanDesc), P, ctypes.POINTER(P)]
        L.dp_plan_destroy.argtypes = [P]
        L.dp_plan_set_stream.argtypes = [P, P]
        L.dp_gram_local.argtypes = [P, P, P]
        L.dp_gram_reduce.argtypes = [P, P, P]
        L.dp_solve.argtypes = [P, P, P, P, P]
        L.dp_precode_apply.argtypes = [P, P, P, P, P]
        L.dp_precode.argtypes = [P, P, P, P]
        L.dp_precode_host.argtypes = [P, P, P, P, I]
        L.dp_status_get.argtypes = [P, P]
        L.dp_debug_stall.argtypes = [P, I]
        L.dp_status_string.argtypes = [I]
        L.dp_status_string.restype = ctypes.c_char_p
        L.dp_version.restype = ctypes.c_char_p
        L.dp_batch_create.argtypes = [ctypes.POINTER(PlanDesc), I, P, ctypes.POINTER(P)]
        L.dp_batch_destroy.argtypes = [P]
        L.dp_batch_precode.argtypes = [P, P, P, P]
        L.dp_batch_tune.argtypes = [P, P, P, P, I]
        L.dp_batch_status_get.argtypes = [P, P]
        L.dp_batch_describe.argtypes = [P]
        L.dp_batch_describe.restype = ctypes.c_char_p
        L.dp_batch_set_timing.argtypes = [P, I]
        L.dp_batch_bucket_ms.argtypes = [P, P, I]
        for name in ("dp_batch_create", "dp_batch_destroy", "dp_batch_precode", "dp_batch_tune",
                     "dp_batch_status_get", "dp_batch_set_timing", "dp_batch_bucket_ms"):
            getattr(L, name).restype = I
        U64 = ctypes.c_ulonglong
        L.dp_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(P)]
        L.dp_server_destroy.argtypes = [P]
        L.dp_server_add_cell.argtypes = [P, ctypes.POINTER(PlanDesc), P, ctypes.POINTER(I)]
        L.dp_server_set_channel.argtypes = [P, I, P]
        L.dp_server_submit.argtypes = [P, I, P, ctypes.POINTER(U64)]
        L.dp_server_drain.argtypes = [P]
        L.dp_server_result.argtypes = [P, U64, ctypes.POINTER(P), ctypes.POINTER(I)]
        L.dp_server_copy_result.argtypes = [P, U64, P, I]
        L.dp_server_release.argtypes = [P, U64]
        L.dp_server_replay.argtypes = [P, I, P, P, P, P]
        L.dp_server_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
        L.dp_server_reset_stats.argtypes = [P]
        for name in ("dp_server_create", "dp_server_destroy", "dp_server_add_cell",
                     "dp_server_set_channel", "dp_server_submit", "dp_server_drain",
                     "dp_server_result", "dp_server_copy_result", "dp_server_release",
                     "dp_server_replay", "dp_server_stats", "dp_server_reset_stats"):
            getattr(L, name).restype = I
        for name in ("dp_plan_create", "dp_plan_destroy", "dp_plan_set_stream", "dp_gram_local",
                     "dp_gram_reduce", "dp_solve", "dp_precode_apply", "dp_precode",
                     "dp_status_get", "dp_debug_stall"):
            getattr(L, name).restype = I
        _ = (F,)
        _lib = L
        return L


def status_string(code: int) -> str:
    return load().dp_status_string(int(code)).decode()


def _check(code: int, what: str):
    if code != OK:
        raise DPError(code, what)


def _ptr(t, dtype, shape, name):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must live on a CUDA device")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(t, dtype, shape, name):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.device.type != "cpu":
        raise ValueError(f"{name} must live in host memory")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A precoding plan (dp_plan_t): problem sizes, cluster partition, mode,
    precision and power / noise parameters; owns the device workspace."""

    def __init__(self, U: int, B: int, C: int, n_sc: int, K: int, mode: str = "wf",
                 prec: str = "fp32", rho2: float = 1.0, N0: float = 0.1, Es: float = 1.0,
                 tau: float = 0.125, refine: int = 0, cluster_sizes=None, stream=None,
                 cluster_power=None):
        import torch
        self.U, self.B, self.C, self.n_sc, self.K = int(U), int(B), int(C), int(n_sc), int(K)
        self.mode, self.prec = mode, prec
        self.rho2, self.N0, self.Es, self.tau, self.refine = rho2, N0, Es, tau, refine
        self.cluster_sizes = None if cluster_sizes is None else [int(c) for c in cluster_sizes]
        self.cluster_power = None if cluster_power is None else [float(w) for w in cluster_power]
        self._lib = load()
        d, self._keep = _desc(dict(U=self.U, B=self.B, C=self.C, n_sc=self.n_sc, K=self.K,
                                   mode=mode, prec=prec, rho2=rho2, N0=N0, Es=Es, tau=tau,
                                   refine=refine, cluster_sizes=self.cluster_sizes,
                                   cluster_power=self.cluster_power))
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        handle = ctypes.c_void_p()
        _check(self._lib.dp_plan_create(ctypes.byref(d), ctypes.c_void_p(stream.cuda_stream),
                                        ctypes.byref(handle)), "dp_plan_create")
        self._h = handle

    @property
    def nsys(self) -> int:
        return self.C if self.mode == "fdwf" else 1

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dp_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def debug_stall(self, microseconds: int):
        """Failure injection for tests: the warp-specialized kernel's bounded
        wait on a flag that nothing sets (dp_debug_stall); 0 turns it off."""
        _check(self._lib.dp_debug_stall(self._h, int(microseconds)), "dp_debug_stall")

    def set_stream(self, stream):
        self._stream = stream
        _check(self._lib.dp_plan_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)),
               "dp_plan_set_stream")

    # -- shapes -------------------------------------------------------------------
    def shapes(self) -> dict:
        n, U, B, C, K = self.n_sc, self.U, self.B, self.C, self.K
        fd = self.mode == "fdwf"
        return dict(H=(n, B, U), S=(n, K, U), X=(n, K, B), G=(n, U, U), Gloc=(C, n, U, U),
                    Z=(n, C, K, U) if fd else (n, K, U), scale=(n, C) if fd else (n,))

    # -- the C entry points ----------------------------------------------------------
    def gram_local(self, H, Gloc):
        import torch
        s = self.shapes()
        _check(self._lib.dp_gram_local(self._h, _ptr(H, torch.complex64, s["H"], "H"),
                                       _ptr(Gloc, torch.complex64, s["Gloc"], "Gloc")),
               "dp_gram_local")

    def gram_reduce(self, Gloc, G):
        import torch
        s = self.shapes()
        _check(self._lib.dp_gram_reduce(self._h, _ptr(Gloc, torch.complex64, s["Gloc"], "Gloc"),
                                        _ptr(G, torch.complex64, s["G"], "G")), "dp_gram_reduce")

    def solve(self, G_or_Gloc, S, Z, scale):
        import torch
        s = self.shapes()
        gshape = s["Gloc"] if self.mode == "fdwf" else s["G"]
        _check(self._lib.dp_solve(self._h, _ptr(G_or_Gloc, torch.complex64, gshape, "G"),
                                  _ptr(S, torch.complex64, s["S"], "S"),
                                  _ptr(Z, torch.complex64, s["Z"], "Z"),
                                  _ptr(scale, torch.float32, s["scale"], "scale")), "dp_solve")

    def precode_apply(self, H, Z, scale, X):
        import torch
        s = self.shapes()
        _check(self._lib.dp_precode_apply(self._h, _ptr(H, torch.complex64, s["H"], "H"),
                                          _ptr(Z, torch.complex64, s["Z"], "Z"),
                                          _ptr(scale, torch.float32, s["scale"], "scale"),
                                          _ptr(X, torch.complex64, s["X"], "X")),
               "dp_precode_apply")

    def precode(self, H, S, X):
        import torch
        s = self.shapes()
        _check(self._lib.dp_precode(self._h, _ptr(H, torch.complex64, s["H"], "H"),
                                    _ptr(S, torch.complex64, s["S"], "S"),
                                    _ptr(X, torch.complex64, s["X"], "X")), "dp_precode")

    def precode_host(self, H, S, X, chunk: int = 0):
        """dp_precode_host: H, S, X are host (CPU) tensors -- page-locked ones
        (``pin_memory()``) let the chunked uploads, kernels and downloads
        overlap.  Completes on the plan's stream."""
        import torch
        s = self.shapes()
        _check(self._lib.dp_precode_host(self._h, _host_ptr(H, torch.complex64, s["H"], "H"),
                                         _host_ptr(S, torch.complex64, s["S"], "S"),
                                         _host_ptr(X, torch.complex64, s["X"], "X"), int(chunk)),
               "dp_precode_host")

    def status_get(self) -> np.ndarray:
        out = np.zeros(max(self.n_sc, 1), np.int32)
        self._lib.dp_status_get(self._h, out.ctypes.data_as(ctypes.c_void_p))
        return out[: self.n_sc]

    # -- conveniences -------------------------------------------------------------
    def empty(self, name: str):
        import torch
        dt = torch.float32 if name == "scale" else torch.complex64
        return torch.empty(self.shapes()[name], dtype=dt, device="cuda")


class Batch:
    """Batched uneven precoding (dp_batch_t): n instances, each described by a
    dict with the Plan keyword arguments (U, B, C, n_sc, K, mode, prec, rho2,
    N0, Es, tau, refine, cluster_sizes, cluster_power).  precode() takes per-instance lists of device
    tensors in the single-plan layouts."""

    def __init__(self, descs, stream=None):
        import torch
        self._lib = load()
        self.descs = [dict(d) for d in descs]
        n = len(self.descs)
        arr = (PlanDesc * n)()
        self._keep = []
        for i, d in enumerate(self.descs):
            arr[i], keep = _desc(d)
            self._keep.extend(keep)
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        h = ctypes.c_void_p()
        _check(self._lib.dp_batch_create(arr, n, ctypes.c_void_p(stream.cuda_stream),
                                         ctypes.byref(h)), "dp_batch_create")
        self._h = h

    def __len__(self):
        return len(self.descs)

    def _ptrs(self, tensors):
        n = len(self.descs)
        if len(tensors) != n:
            raise ValueError(f"expected {n} tensors")
        arr = (ctypes.c_void_p * n)()
        for i, t in enumerate(tensors):
            if not (t.is_cuda and t.is_contiguous()):
                raise ValueError("batch arrays must be contiguous CUDA tensors")
            arr[i] = t.data_ptr()
        return arr

    def precode(self, Hs, Ss, Xs):
        _check(self._lib.dp_batch_precode(self._h, self._ptrs(Hs), self._ptrs(Ss),
                                          self._ptrs(Xs)), "dp_batch_precode")

    def tune(self, Hs, Ss, Xs, trials: int = 3):
        _check(self._lib.dp_batch_tune(self._h, self._ptrs(Hs), self._ptrs(Ss), self._ptrs(Xs),
                                       int(trials)), "dp_batch_tune")

    def status_get(self):
        total = sum(int(d["n_sc"]) for d in self.descs)
        out = np.zeros(max(total, 1), np.int32)
        self._lib.dp_batch_status_get(self._h, out.ctypes.data_as(ctypes.c_void_p))
        res, o = [], 0
        for d in self.descs:
            res.append(out[o:o + int(d["n_sc"])].copy())
            o += int(d["n_sc"])
        return res

    def describe(self) -> dict:
        import json
        return json.loads(self._lib.dp_batch_describe(self._h).decode())

    def set_timing(self, mode: int):
        """Per-bucket CUDA events: 1 inside the graph, 2 with eager launches,
        0 off (dp_batch_set_timing)."""
        _check(self._lib.dp_batch_set_timing(self._h, int(mode)), "dp_batch_set_timing")

    def bucket_ms(self):
        """Device time of each bucket of the last call (waits for the stream)."""
        n = len(self.describe()["buckets"])
        out = np.zeros(max(n, 1), np.float32)
        _check(self._lib.dp_batch_bucket_ms(self._h, out.ctypes.data_as(ctypes.c_void_p), n),
               "dp_batch_bucket_ms")
        return [float(x) for x in out[:n]]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _desc(d: dict):
    """A PlanDesc from the Plan keyword arguments as a dict, and the ctypes
    arrays it points to (kept alive by the caller)."""
    keep = []
    cs_ptr = cp_ptr = None
    cs = d.get("cluster_sizes")
    if cs is not None:
        a = (ctypes.c_int * len(cs))(*[int(x) for x in cs])
        keep.append(a)
        cs_ptr = ctypes.cast(a, ctypes.POINTER(ctypes.c_int))
    cp = d.get("cluster_power")
    if cp is not None:
        a = (ctypes.c_float * len(cp))(*[float(x) for x in cp])
        keep.append(a)
        cp_ptr = ctypes.cast(a, ctypes.POINTER(ctypes.c_float))
    mode, prec = d.get("mode", "wf"), d.get("prec", "fp32")
    if mode not in MODES or prec not in PRECISIONS:
        raise ValueError(f"mode {mode!r} / precision {prec!r} unknown")
    pd = PlanDesc(int(d["U"]), int(d["B"]), int(d["C"]), cs_ptr, int(d["n_sc"]), int(d["K"]),
                  MODES[mode], PRECISIONS[prec], float(d.get("rho2", 1.0)),
                  float(d.get("N0", 0.1)), float(d.get("Es", 1.0)), float(d.get("tau", 0.125)),
                  int(d.get("refine", 0)), cp_ptr)
    return pd, keep


class Server:
    """Continuous-batching server (dp_server_t).  Cells hold device-resident
    channels; requests precode one slot from device symbols into the
    server's arena."""

    def __init__(self, streams: int = 8, max_inflight: int = 32, arena_bytes: int = 1 << 30,
                 auto_release: bool = False, device: int = 0, cache_solve: bool = False):
        self._lib = load()
        cfg = ServerConfig(int(device), int(streams), int(max_inflight), int(arena_bytes),
                           int(bool(auto_release)), int(bool(cache_solve)))
        h = ctypes.c_void_p()
        _check(self._lib.dp_server_create(ctypes.byref(cfg), ctypes.byref(h)), "dp_server_create")
        self._h = h
        self.cells = []
        self._hold = []

    def add_cell(self, desc: dict, H) -> int:
        pd, keep = _desc(desc)
        cid = ctypes.c_int()
        _check(self._lib.dp_server_add_cell(self._h, ctypes.byref(pd), ctypes.c_void_p(H.data_ptr()),
                                            ctypes.byref(cid)), "dp_server_add_cell")
        self.cells.append(dict(desc))
        self._hold.append(H)
        return cid.value

    def set_channel(self, cell: int, H):
        self._hold.append(H)
        _check(self._lib.dp_server_set_channel(self._h, int(cell), ctypes.c_void_p(H.data_ptr())),
               "dp_server_set_channel")

    def submit(self, cell: int, S) -> int:
        rid = ctypes.c_ulonglong()
        _check(self._lib.dp_server_submit(self._h, int(cell), ctypes.c_void_p(S.data_ptr()),
                                          ctypes.byref(rid)), "dp_server_submit")
        return rid.value

    def drain(self):
        _check(self._lib.dp_server_drain(self._h), "dp_server_drain")

    def result(self, rid: int):
        """The request's worst status code (0 when every subcarrier succeeded);
        copy_result copies its X out of the arena."""
        x = ctypes.c_void_p()
        st = ctypes.c_int()
        _check(self._lib.dp_server_result(self._h, ctypes.c_ulonglong(rid), ctypes.byref(x),
                                          ctypes.byref(st)), "dp_server_result")
        return st.value

    def copy_result(self, rid: int, out):
        _check(self._lib.dp_server_copy_result(self._h, ctypes.c_ulonglong(rid),
                                               ctypes.c_void_p(out.data_ptr()), int(not out.is_cuda)),
               "dp_server_copy_result")

    def release(self, rid: int):
        _check(self._lib.dp_server_release(self._h, ctypes.c_ulonglong(rid)), "dp_server_release")

    def replay(self, cells, S_list, arrival_s, H_switch=None):
        n = len(cells)
        c = (ctypes.c_int * n)(*[int(x) for x in cells])
        sp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in S_list])
        at = (ctypes.c_double * n)(*[float(t) for t in arrival_s])
        hs = None
        if H_switch is not None:
            hs = (ctypes.c_void_p * n)(*[(t.data_ptr() if t is not None else None) for t in H_switch])
        _check(self._lib.dp_server_replay(self._h, n, c, sp, at, hs), "dp_server_replay")

    def stats(self) -> dict:
        s = ServerStats()
        _check(self._lib.dp_server_stats(self._h, ctypes.byref(s)), "dp_server_stats")
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def reset_stats(self):
        _check(self._lib.dp_server_reset_stats(self._h), "dp_server_reset_stats")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dp_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
