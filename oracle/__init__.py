"""FP64 CPU oracle for feedforward decentralized WF / ZF precoding
(arXiv:1804.10987): Python loader for ``dp_oracle.c``.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it, and it shares no code with the CUDA library.

Every function takes and returns numpy arrays; complex arrays are complex128
(the complex64 inputs the GPU sees are promoted exactly).  Layouts are the
ones the C header states: H [n_sc][B][U], S [n_sc][K][U], X [n_sc][K][B].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dp_oracle.c")
_HDR = os.path.join(_HERE, "dp_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

ZF, WF, FDWF, MRT = 0, 1, 2, 3
MODES = {"zf": ZF, "wf": WF, "fdwf": FDWF, "mrt": MRT}
FORM_PAPER, FORM_UXU, FORM_BCXBC = 0, 1, 2
OK, NOT_PD, NONFINITE, BAD_ARG = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile dp_oracle.c into oracle/_build/liboracle.so (gcc, FP64, no FMA
    contraction so x86 and Arm hosts round identically)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fcx-limited-range", "-fPIC", "-shared",
           "-pthread", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Desc(ctypes.Structure):
    _fields_ = [("U", ctypes.c_int), ("B", ctypes.c_int), ("C", ctypes.c_int),
                ("cluster_sizes", ctypes.POINTER(ctypes.c_int)),
                ("n_sc", ctypes.c_int), ("K", ctypes.c_int), ("mode", ctypes.c_int),
                ("rho2", ctypes.c_double), ("N0", ctypes.c_double),
                ("Es", ctypes.c_double), ("tau", ctypes.c_double),
                ("fd_form", ctypes.c_int),
                ("cluster_power", ctypes.POINTER(ctypes.c_double))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_gram.argtypes = [ctypes.c_int, P, ctypes.c_int, ctypes.c_int, P]
            lib.orc_gram_antenna.argtypes = [ctypes.c_int, P, ctypes.c_int, ctypes.c_int, P]
            lib.orc_cholesky.argtypes = [ctypes.c_int, P, P]
            lib.orc_cholesky.restype = ctypes.c_int
            lib.orc_inverse_from_cholesky.argtypes = [ctypes.c_int, P, P]
            lib.orc_t_lemma.argtypes = [ctypes.c_int, P, ctypes.c_double]
            lib.orc_t_lemma.restype = ctypes.c_double
            lib.orc_t_direct.argtypes = [ctypes.c_int, P, P]
            lib.orc_t_direct.restype = ctypes.c_double
            lib.orc_precode.argtypes = [ctypes.POINTER(_Desc), P, P, P, P, P, P, P, P, P, P,
                                        ctypes.c_int]
            lib.orc_precode.restype = ctypes.c_int
            _lib = lib
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.complex128)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --- single steps (one subcarrier) ------------------------------------------------

def gram(H: np.ndarray, lo: int = 0, hi: int | None = None) -> np.ndarray:
    """G_c = H_c H_c^H for one subcarrier, H given as [B][U]."""
    H = _c128(H)
    B, U = H.shape
    hi = B if hi is None else hi
    G = np.zeros((U, U), np.complex128)
    _load().orc_gram(U, _ptr(H), lo, hi, _ptr(G))
    return G


def gram_antenna(H: np.ndarray, lo: int, hi: int) -> np.ndarray:
    H = _c128(H)
    B, U = H.shape
    n = hi - lo
    G = np.zeros((n, n), np.complex128)
    _load().orc_gram_antenna(U, _ptr(H), lo, hi, _ptr(G))
    return G


def cholesky(A: np.ndarray):
    A = _c128(A)
    n = A.shape[0]
    L = np.zeros_like(A)
    st = _load().orc_cholesky(n, _ptr(A), _ptr(L))
    return st, L


def inverse_from_cholesky(L: np.ndarray) -> np.ndarray:
    L = _c128(L)
    T = np.zeros_like(L)
    _load().orc_inverse_from_cholesky(L.shape[0], _ptr(L), _ptr(T))
    return T


def t_lemma(T: np.ndarray, kappa: float) -> float:
    T = _c128(T)
    return float(_load().orc_t_lemma(T.shape[0], _ptr(T), float(kappa)))


def t_direct(T: np.ndarray, G: np.ndarray) -> float:
    T, G = _c128(T), _c128(G)
    return float(_load().orc_t_direct(T.shape[0], _ptr(T), _ptr(G)))


# --- whole precoder --------------------------------------------------------------

def kappa_of(mode: str, U: int, N0: float, rho2: float, C: int = 1, tau: float = 0.125) -> float:
    """The regularizer each mode uses: Thm. 1 (WF), 0 (ZF), Eq. (16) (FD-WF)."""
    if mode == "wf":
        return U * N0 / rho2
    if mode == "zf":
        return 0.0
    return tau * U * N0 / (rho2 / C)


def precode(H, S, cluster_sizes, mode: str = "wf", rho2: float = 1.0, N0: float = 0.1,
            Es: float = 1.0, tau: float = 0.125, fd_form: int = FORM_PAPER,
            nthreads: int = 1, outputs=("X", "scale", "t", "t_alt", "Z", "G", "Gloc", "status"),
            cluster_power=None):
    """Run the oracle over all subcarriers.  H [n_sc][B][U], S [n_sc][K][U].

    Returns a dict with X [n_sc][K][B], scale/t/t_alt ([n_sc] or FD [n_sc][C]),
    Z ([n_sc][K][U] or FD [n_sc][C][K][U]), G [n_sc][U][U], Gloc [C][n_sc][U][U],
    status [n_sc] (0 ok, 1 not positive definite, 2 non-finite input).
    cluster_power: FD-WF per-cluster weights (rho_c^2 = rho2 w_c / sum w),
    None for the paper's equal split (Sec. III-D)."""
    H, S = _c128(H), _c128(S)
    n_sc, B, U = H.shape
    K = S.shape[1]
    assert S.shape == (n_sc, K, U), S.shape
    cs = np.ascontiguousarray(cluster_sizes, dtype=np.int32)
    C = int(cs.size)
    m = MODES[mode]
    nsys = C if m == FDWF else 1
    out = {}
    want = set(outputs)

    def arr(name, shape, dt):
        if name in want:
            out[name] = np.zeros(shape, dt)
            return _ptr(out[name])
        return None

    pX = arr("X", (n_sc, K, B), np.complex128)
    pscale = arr("scale", (n_sc, nsys) if nsys > 1 else (n_sc,), np.float64)
    pt = arr("t", (n_sc, nsys) if nsys > 1 else (n_sc,), np.float64)
    pta = arr("t_alt", (n_sc, nsys) if nsys > 1 else (n_sc,), np.float64)
    pZ = arr("Z", (n_sc, C, K, U) if m == FDWF else (n_sc, K, U), np.complex128)
    pG = arr("G", (n_sc, U, U), np.complex128)
    pGl = arr("Gloc", (C, n_sc, U, U), np.complex128)
    pst = arr("status", (n_sc,), np.int32)
    cp = None if cluster_power is None else np.ascontiguousarray(cluster_power, dtype=np.float64)
    d = _Desc(U, B, C, cs.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), n_sc, K, m,
              float(rho2), float(N0), float(Es), float(tau), int(fd_form),
              None if cp is None else cp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    rc = _load().orc_precode(ctypes.byref(d), _ptr(H), _ptr(S), pX, pscale, pt, pta, pZ, pG,
                             pGl, pst, int(nthreads))
    if rc != OK:
        raise ValueError(f"oracle rejected the problem (code {rc})")
    return out
