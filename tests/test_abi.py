"""The C-ABI libraries load and export every function their headers declare
(no GPU needed: nothing here launches work on a device)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2401_10068_gb300 import _build, vbh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# header -> the library that exports it
HEADERS = {os.path.join(ROOT, "include", "vbh.h"): "vbh",
           os.path.join(ROOT, "include", "vbh_ws.h"): "vbh",
           os.path.join(ROOT, "include", "vbh_synth.h"): "vbh_synth"}


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build_all()


def _declared(header):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(vbh_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.mark.parametrize("header", sorted(HEADERS))
def test_library_exports_every_declared_symbol(header):
    lib = HEADERS[header]
    names = _declared(header)
    assert names, "no declarations parsed"
    so = ctypes.CDLL(_build.lib_path(lib))
    for n in names:
        assert hasattr(so, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", _build.lib_path(lib)], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (vbh_\w+)", out))
    assert set(names) <= exported


def test_every_include_header_is_covered():
    hs = sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    assert hs == sorted(os.path.basename(p) for p in HEADERS)


def test_host_only_entry_points():
    lib = vbh._lib()
    assert lib.vbh_strerror(0) == b"ok"
    assert lib.vbh_strerror(-1) == b"invalid argument"
    assert lib.vbh_strerror(-12345) == b"unknown status"
    p = vbh.Prior()
    lib.vbh_prior_default(3, ctypes.byref(p))
    assert (p.S, p.q0, p.n0, p.a0, p.b0) == (3, 1e-3, 1.0, 0.5, 0.5)
    assert not p.K0 and not p.Lambda0_inv
    o = vbh.Opts()
    lib.vbh_opts_default(ctypes.byref(o))
    assert (o.tol, o.max_iter, o.precision, o.init, o.refine_iters, o.method) == (1e-8, 200, vbh.FP32,
                                                                                 vbh.INIT_PAPER, 10, vbh.CAVI)
    assert o.grouped == 0 and o.stats == vbh.STATS_AUTO and o.loop == vbh.LOOP_AUTO


def test_result_struct_layout_matches_header():
    # offsets of the ctypes mirror against the C layout rules of the header
    assert ctypes.sizeof(vbh.Result) == 4 * 5 + 4 + 8 * (31 + 32 + 31 * 31) + 8 * 7
    assert vbh.Opts.refine_iters.offset == 20
    assert vbh.Opts.init_state.offset == 24 and vbh.Opts.elbo_trace.offset == 32
    assert vbh.Opts.method.offset == 40 and vbh.Opts.grouped.offset == 44 and vbh.Opts.stats.offset == 48
    assert vbh.Opts.loop.offset == 52
    assert ctypes.sizeof(vbh.Opts) == 56
    assert ctypes.sizeof(vbh.BatchPlan) == 24 and vbh.BatchPlan.pass_ms.offset == 20


def test_batched_plan_refuses_null_arguments():
    lib = vbh._lib()
    n = ctypes.c_int(-1)
    assert lib.vbh_batched_plan(None, None, 0, ctypes.byref(n)) == -1 and n.value == -1


def test_create_fails_loudly_without_a_gpu():
    """No CPU fallback: on a host without a GPU the library's first device
    call fails and the binding raises with the library's status."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(vbh.VBHError) as e:
        vbh.Handle(0, None)
    assert e.value.status == -3 and "vbh_create" in str(e.value)
    assert "cudaGetDeviceCount" in vbh._lib().vbh_last_error_detail().decode()


def test_binding_refuses_short_or_non_float32_inputs():
    """Plain pointers carry no size: the binding refuses, with VBH_EINVAL
    before any library call, an input that holds fewer values than the call
    reads or is not float32 (host arrays and tensors alike)."""
    import numpy as np
    import torch
    V, S = 10, 3
    r, d = np.zeros(V, np.float32), np.zeros((V, S), np.float32)
    vbh._check_inputs(r, d, V, S, "vbh_fit")                           # exact sizes pass
    vbh._check_inputs(None, None, 5, S, "vbh_fit")                     # null inputs: the library decides
    vbh._check_inputs(r, d[:, :2], V, 33, "vbh_fit")                   # S out of range: the library decides
    cases = [(r[:9], d, "r holds 9"), (r, d[:9], "d holds 27"), (r.astype(np.float64), d, "float64"),
             (torch.zeros(V), torch.zeros(V * S - 1), "d holds 29"),
             (torch.zeros(V, dtype=torch.float64), torch.zeros(V * S), "torch.float64")]
    for rr, dd, msg in cases:
        with pytest.raises(vbh.VBHError) as e:
            vbh._check_inputs(rr, dd, V, S, "vbh_fit")
        assert e.value.status == -1 and msg in str(e.value), (msg, str(e.value))
