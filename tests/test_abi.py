"""The C-ABI library builds, loads and exports every function the public
header declares; host-side argument validation (no device work).  CPU only."""
import ctypes
import os
import re

import pytest

from paper_1804_10987_gb300 import dp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        for m in re.finditer(r"\b(dp_\w+)\s*\(", txt):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dp_plan_create", "dp_plan_destroy", "dp_gram_local", "dp_gram_reduce",
                     "dp_solve", "dp_precode_apply", "dp_precode", "dp_status_get",
                     "dp_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = dp.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings():
    assert dp.status_string(dp.OK) == "ok"
    assert "positive definite" in dp.status_string(dp.NOT_PD)
    assert dp.load().dp_version().decode().startswith("dprecode")


def _create(**kw):
    lib = dp.load()
    base = dict(U=8, B=64, C=2, cs=None, n_sc=4, K=2, mode=1, prec=0, rho2=1.0, N0=0.1, Es=1.0,
                tau=0.125, refine=0)
    base.update(kw)
    cs = base.pop("cs")
    cp = base.pop("cp", None)
    arr = parr = None
    if cs is not None:
        arr = (ctypes.c_int * len(cs))(*cs)
    if cp is not None:
        parr = (ctypes.c_float * len(cp))(*cp)
    d = dp.PlanDesc(base["U"], base["B"], base["C"],
                    ctypes.cast(arr, ctypes.POINTER(ctypes.c_int)) if arr else None,
                    base["n_sc"], base["K"], base["mode"], base["prec"], base["rho2"],
                    base["N0"], base["Es"], base["tau"], base["refine"],
                    ctypes.cast(parr, ctypes.POINTER(ctypes.c_float)) if parr else None)
    h = ctypes.c_void_p()
    rc = lib.dp_plan_create(ctypes.byref(d), None, ctypes.byref(h))
    if rc == dp.OK:
        lib.dp_plan_destroy(h)
    return rc


@pytest.mark.parametrize("kw,code", [
    (dict(U=0), dp.INVALID_ARG), (dict(U=65), dp.INVALID_ARG), (dict(B=0), dp.INVALID_ARG),
    (dict(C=0), dp.INVALID_ARG), (dict(C=65, B=64), dp.INVALID_ARG),
    (dict(n_sc=-1), dp.INVALID_ARG), (dict(K=65), dp.INVALID_ARG), (dict(mode=7), dp.INVALID_ARG),
    (dict(prec=9), dp.INVALID_ARG), (dict(rho2=0.0), dp.INVALID_ARG),
    (dict(N0=-1.0), dp.INVALID_ARG), (dict(Es=float("nan")), dp.INVALID_ARG),
    (dict(refine=2), dp.INVALID_ARG),
    (dict(C=3), dp.PARTITION), (dict(C=2, cs=[30, 30]), dp.PARTITION),
    (dict(C=2, cs=[64, 0]), dp.PARTITION),
    (dict(mode=0, U=8, B=6, C=1), dp.UNSUPPORTED),
    (dict(mode=2, N0=0.0, U=8, B=12, C=2), dp.UNSUPPORTED),
    # per-cluster power: FD-WF only, positive finite weights
    (dict(mode=1, cp=[1.0, 2.0]), dp.INVALID_ARG),
    (dict(mode=2, cp=[1.0, 0.0]), dp.INVALID_ARG),
    (dict(mode=2, cp=[1.0, -2.0]), dp.INVALID_ARG),
    (dict(mode=2, cp=[1.0, float("inf")]), dp.INVALID_ARG),
    (dict(mode=2, cp=[float("nan"), 1.0]), dp.INVALID_ARG),
])
def test_plan_validation_on_host(kw, code):
    assert _create(**kw) == code


def test_null_arguments():
    lib = dp.load()
    assert lib.dp_plan_create(None, None, None) == dp.INVALID_ARG
    assert lib.dp_precode(None, None, None, None) == dp.INVALID_ARG
    assert lib.dp_status_get(None, None) == dp.INVALID_ARG


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's ctypes structures have the header's field offsets and
    sizes (a C program built against include/dprecode.h prints them)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {"dp_plan_desc": dp.PlanDesc, "dp_server_config": dp.ServerConfig,
               "dp_server_stats_t": dp.ServerStats}
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "dprecode.h"', "int main(void) {"]
    for cname, cls in structs.items():
        src.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            src.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    src.append("  return 0;\n}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)],
                   check=True, capture_output=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                        text=True).stdout.splitlines())
    for cname, cls in structs.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)


@pytest.mark.parametrize("kw", [
    dict(max_inflight=0), dict(max_inflight=1025), dict(streams=0), dict(streams=65),
    dict(arena_bytes=4095), dict(auto_release=2), dict(auto_release=-1), dict(cache_solve=2),
    dict(cache_solve=-1),
])
def test_server_config_validation_on_host(kw):
    lib = dp.load()
    base = dict(device=0, streams=4, max_inflight=8, arena_bytes=1 << 20, auto_release=0,
                cache_solve=0)
    base.update(kw)
    cfg = dp.ServerConfig(*[base[f] for f, _ in dp.ServerConfig._fields_])
    h = ctypes.c_void_p()
    assert lib.dp_server_create(ctypes.byref(cfg), ctypes.byref(h)) == dp.INVALID_ARG
    assert not h.value


def test_server_null_handles():
    lib = dp.load()
    rid = ctypes.c_ulonglong()
    st = dp.ServerStats()
    assert lib.dp_server_create(None, None) == dp.INVALID_ARG
    assert lib.dp_server_destroy(None) == dp.INVALID_ARG
    assert lib.dp_server_add_cell(None, None, None, None) == dp.INVALID_ARG
    assert lib.dp_server_set_channel(None, 0, None) == dp.INVALID_ARG
    assert lib.dp_server_submit(None, 0, None, ctypes.byref(rid)) == dp.INVALID_ARG
    assert lib.dp_server_drain(None) == dp.INVALID_ARG
    assert lib.dp_server_result(None, ctypes.c_ulonglong(1), None, None) == dp.INVALID_ARG
    assert lib.dp_server_copy_result(None, ctypes.c_ulonglong(1), None, 0) == dp.INVALID_ARG
    assert lib.dp_server_release(None, ctypes.c_ulonglong(1)) == dp.INVALID_ARG
    assert lib.dp_server_replay(None, 0, None, None, None, None) == dp.INVALID_ARG
    assert lib.dp_server_stats(None, ctypes.byref(st)) == dp.INVALID_ARG
    assert lib.dp_server_reset_stats(None) == dp.INVALID_ARG


_KEEP = []


def _desc(**kw):
    base = dict(U=8, B=64, C=2, n_sc=4, K=2, mode=1, prec=0, rho2=1.0, N0=0.1, Es=1.0,
                tau=0.125, refine=0, cp=None)
    base.update(kw)
    cp = None
    if base["cp"] is not None:
        arr = (ctypes.c_float * len(base["cp"]))(*base["cp"])
        _KEEP.append(arr)
        cp = ctypes.cast(arr, ctypes.POINTER(ctypes.c_float))
    return dp.PlanDesc(base["U"], base["B"], base["C"], None, base["n_sc"], base["K"],
                       base["mode"], base["prec"], base["rho2"], base["N0"], base["Es"],
                       base["tau"], base["refine"], cp)


def test_batch_validation_on_host():
    lib = dp.load()
    h = ctypes.c_void_p()
    arr = (dp.PlanDesc * 2)(_desc(), _desc())
    assert lib.dp_batch_create(None, 1, None, ctypes.byref(h)) == dp.INVALID_ARG
    assert lib.dp_batch_create(arr, 0, None, ctypes.byref(h)) == dp.INVALID_ARG
    assert lib.dp_batch_create(arr, 2, None, None) == dp.INVALID_ARG
    for bad, code in ((dict(U=0), dp.INVALID_ARG), (dict(C=3), dp.PARTITION),
                      (dict(mode=0, U=8, B=6, C=1), dp.UNSUPPORTED)):
        arr = (dp.PlanDesc * 2)(_desc(), _desc(**bad))  # the second instance is invalid
        assert lib.dp_batch_create(arr, 2, None, ctypes.byref(h)) == code, bad
        assert not h.value
    assert lib.dp_batch_destroy(None) == dp.INVALID_ARG


@pytest.mark.parametrize("kw,code", [
    (dict(U=0), dp.INVALID_ARG), (dict(K=65), dp.INVALID_ARG), (dict(mode=9), dp.INVALID_ARG),
    (dict(prec=2), dp.UNSUPPORTED), (dict(refine=1), dp.UNSUPPORTED), (dict(C=3), dp.PARTITION),
    (dict(mode=0, U=8, B=6, C=1), dp.UNSUPPORTED),
    # workspace beyond the static array: 4000 subcarriers of U = 64 need 131 MB of G
    (dict(U=64, B=128, C=1, n_sc=4000), dp.UNSUPPORTED),
    (dict(mode=2, cp=[1.0, 3.0]), dp.UNSUPPORTED),  # per-cluster power needs a plan
    (dict(mode=1, cp=[1.0, 3.0]), dp.INVALID_ARG),
    (dict(n_sc=0), dp.OK),  # nothing to do, nothing enqueued
    (dict(), dp.INVALID_ARG),  # a valid description with null device arrays
])
def test_noalloc_validation_on_host(kw, code):
    lib = dp.load()
    d = _desc(**kw)
    assert lib.dp_precode_noalloc(ctypes.byref(d), None, None, None, None, None) == code
