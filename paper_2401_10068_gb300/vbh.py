"""Thin ctypes binding of ``libvbh.so`` (C ABI in ``include/vbh.h``).

Argument marshalling only: every step of the CAVI sweep runs in the CUDA
kernels of the library.  Inputs may be torch tensors (device or pinned host
memory) or numpy arrays (host memory); PyTorch is used only for device memory
and streams.  The library must have been built (``__graft_entry__.build()``);
there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

SMAX = 32
MMAX = 31
FP32 = 0
BF16 = 1
CAVI = 0
EM = 1
INIT_PAPER = 0
INIT_GIVEN = 1
STATS_AUTO = 0          # compensated statistics when tol > 0 (vbh_opts.stats)
STATS_COMPENSATED = 1
STATS_PLAIN = 2
LOOP_AUTO = 0           # resident sweep loop when the data set fits in shared memory (vbh_opts.loop)
LOOP_STREAM = 1
LOOP_RESIDENT = 2

STATUS = {0: "VBH_OK", -1: "VBH_EINVAL", -2: "VBH_ENOMEM", -3: "VBH_ECUDA", -4: "VBH_ENONFINITE",
          -5: "VBH_ETIMEOUT", -6: "VBH_ESTATE", -7: "VBH_EUNSUPPORTED"}


def selftest_wait(budget_ns: int, device: int = 0, stream=None):
    """``vbh_selftest_wait``: statuses of the bounded waits (expired, expired,
    completed, bytes) and the nanoseconds the first wait took."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    st = (ctypes.c_int * 4)()
    waited = ctypes.c_uint64()
    rc = _lib().vbh_selftest_wait(int(device), ctypes.c_void_p(stream) if stream else None, int(budget_ns), st,
                                  ctypes.byref(waited))
    if rc != 0:
        raise VBHError(rc, "vbh_selftest_wait")
    return list(st), int(waited.value)


class VBHError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = f"{what}: {STATUS.get(status, status)} ({_lib().vbh_strerror(status).decode()})"
        if status in (-2, -3):
            detail = _lib().vbh_last_error_detail().decode()
            if detail:
                msg += f" [{detail}]"
        super().__init__(msg)


_dp = ctypes.POINTER(ctypes.c_double)


class Prior(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int), ("K0", _dp), ("q0", ctypes.c_double), ("n0", ctypes.c_double),
                ("a0", ctypes.c_double), ("b0", ctypes.c_double), ("Lambda0_inv", _dp)]


class Result(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int), ("iters", ctypes.c_int), ("converged", ctypes.c_int), ("status", ctypes.c_int),
                ("elbo_const_dropped", ctypes.c_int), ("kappa", ctypes.c_double * MMAX),
                ("weights", ctypes.c_double * SMAX), ("W_inv", ctypes.c_double * (MMAX * MMAX)),
                ("nu", ctypes.c_double), ("lam", ctypes.c_double), ("a_rho", ctypes.c_double),
                ("b_rho", ctypes.c_double), ("rho_mean", ctypes.c_double), ("rho_mode", ctypes.c_double),
                ("elbo", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("init", ctypes.c_int), ("refine_iters", ctypes.c_int), ("init_state", ctypes.POINTER(Result)),
                ("elbo_trace", _dp), ("method", ctypes.c_int), ("grouped", ctypes.c_int), ("stats", ctypes.c_int),
                ("loop", ctypes.c_int)]


class BatchPlan(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int), ("tile", ctypes.c_int), ("chunk_tiles", ctypes.c_int), ("stages", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("pass_ms", ctypes.c_float)]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.lib_path("vbh")
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build the CUDA library first (__graft_entry__.build())")
        lib = ctypes.CDLL(path)
        vp, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        P, R, O = ctypes.POINTER(Prior), ctypes.POINTER(Result), ctypes.POINTER(Opts)
        sigs = {
            "vbh_prior_default": (None, [ci, P]),
            "vbh_opts_default": (None, [O]),
            "vbh_create": (ci, [ctypes.POINTER(vp), ci, vp]),
            "vbh_destroy": (None, [vp]),
            "vbh_strerror": (ctypes.c_char_p, [ci]),
            "vbh_state_bytes": (ctypes.c_size_t, []),
            "vbh_last_error_detail": (ctypes.c_char_p, []),
            "vbh_selftest_wait": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64,
                                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_uint64)]),
            "vbh_selftest_math": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, _dp, _dp, ctypes.c_int]),
            "vbh_fit": (ci, [vp, vp, vp, i64, ci, P, O, R]),
            "vbh_fit_begin": (ci, [vp, vp, vp, i64, ci, P, O]),
            "vbh_fit_step": (ci, [vp, ci, ctypes.POINTER(ci)]),
            "vbh_fit_result": (ci, [vp, R]),
            "vbh_elbo": (ci, [vp, vp, vp, i64, ci, P, R, _dp]),
            "vbh_fit_static": (ci, [vp, vp, i64, ci, P, O, R, ci, vp]),
            "vbh_fit_batched": (ci, [vp, ci, ctypes.POINTER(i64), ctypes.POINTER(ci), ctypes.POINTER(vp),
                                     ctypes.POINTER(vp), P, O, R]),
            "vbh_batched_plan": (ci, [vp, ctypes.POINTER(BatchPlan), ci, ctypes.POINTER(ci)]),
            "vbh_ws_create": (ci, [ctypes.POINTER(vp), ctypes.c_uint64, ci, vp]),
            "vbh_ws_destroy": (None, [vp]),
            "vbh_ws_num_params": (ctypes.c_size_t, [vp]),
            "vbh_ws_get_params": (ci, [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t]),
            "vbh_ws_set_params": (ci, [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t]),
            "vbh_ws_set_norm": (ci, [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
            "vbh_ws_features": (ci, [vp, vp, vp, i64, ci, i64, vp]),
            "vbh_ws_forward": (ci, [vp, ci, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i64),
                                    ctypes.POINTER(ci), ctypes.POINTER(i64), vp]),
            "vbh_ws_loss_grad": (ci, [vp, ci, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i64),
                                      ctypes.POINTER(ci), ctypes.POINTER(i64), vp, vp, _dp,
                                      ctypes.POINTER(ctypes.c_float)]),
            "vbh_ws_train_step": (ci, [vp, ci, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i64),
                                       ctypes.POINTER(ci), ctypes.POINTER(i64), vp, vp, ctypes.c_float, _dp]),
            "vbh_ws_predict": (ci, [vp, ci, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i64),
                                    ctypes.POINTER(ci), P, R]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def state_bytes() -> int:
    return int(_lib().vbh_state_bytes())


def library_path() -> str:
    return _build.lib_path("vbh")


def _ptr(x):
    """Address of a torch tensor or numpy array (contiguous float32)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("inputs must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if x.dtype != np.float32 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy inputs must be C-contiguous float32")
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError("expected a torch tensor or a numpy array")


def _check_inputs(r, d, V: int, S: int, call: str):
    """The library reads V float32 values of r and V*S of d through plain
    pointers, which carry no size: refuse a tensor or array that is not
    float32 or holds fewer values, with VBH_EINVAL, before the call.  Null
    inputs and S outside 1..32 are left to the library's own checks."""
    if not (1 <= int(S) <= 32) or int(V) < 0:
        return
    for x, n, what in ((r, int(V), "r"), (d, int(V) * int(S), "d")):
        if x is None:
            continue
        if hasattr(x, "data_ptr"):
            if str(x.dtype) != "torch.float32":
                raise VBHError(-1, f"{call} ({what} is {x.dtype}, float32 is read)")
            cnt = x.numel()
        elif isinstance(x, np.ndarray):
            if x.dtype != np.float32:
                raise VBHError(-1, f"{call} ({what} is {x.dtype}, float32 is read)")
            cnt = x.size
        else:
            continue
        if cnt < n:
            raise VBHError(-1, f"{call} ({what} holds {cnt} values, {n} are read)")


class _PriorArgs:
    """Keeps the numpy buffers of a Prior alive."""

    def __init__(self, prior: dict | None, S: int):
        self.c = Prior()
        _lib().vbh_prior_default(S, ctypes.byref(self.c))
        self._k = self._l = None
        if prior:
            M = S - 1
            for key in ("q0", "n0", "a0", "b0"):
                if key in prior:
                    setattr(self.c, key, float(prior[key]))
            if prior.get("K0") is not None:
                self._k = np.ascontiguousarray(np.asarray(prior["K0"], dtype=np.float64).reshape(M))
                self.c.K0 = self._k.ctypes.data_as(_dp)
            if prior.get("L0inv") is not None:
                self._l = np.ascontiguousarray(np.asarray(prior["L0inv"], dtype=np.float64).reshape(M, M))
                self.c.Lambda0_inv = self._l.ctypes.data_as(_dp)


def result_to_dict(res: Result) -> dict:
    S = max(int(res.S), 0)
    M = max(S - 1, 0)
    return {"S": S, "iters": res.iters, "converged": bool(res.converged), "status": res.status,
            "const_dropped": bool(res.elbo_const_dropped), "kappa": np.array(res.kappa[:M]),
            "weights": np.array(res.weights[:S]), "Winv": np.array(res.W_inv[:M * M]).reshape(M, M),
            "nu": res.nu, "lam": res.lam, "a_rho": res.a_rho, "b_rho": res.b_rho, "rho_mean": res.rho_mean,
            "rho_mode": res.rho_mode, "elbo": res.elbo}


def dict_to_result(g: dict, S: int) -> Result:
    M = S - 1
    res = Result()
    res.S = S
    k = np.asarray(g["kappa"], dtype=np.float64).reshape(M)
    W = np.asarray(g["Winv"], dtype=np.float64).reshape(M * M)
    for j in range(M):
        res.kappa[j] = k[j]
    for j in range(M * M):
        res.W_inv[j] = W[j]
    res.nu, res.lam, res.a_rho, res.b_rho = float(g["nu"]), float(g["lam"]), float(g["a_rho"]), float(g["b_rho"])
    return res


class Handle:
    """One ``vbh_handle``: a device and a borrowed stream (a torch stream, a
    raw cudaStream_t integer, or None for the legacy default stream)."""

    def __init__(self, device: int = 0, stream=None):
        lib = _lib()
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self._stream = stream
        self._h = ctypes.c_void_p()
        rc = lib.vbh_create(ctypes.byref(self._h), int(device), ctypes.c_void_p(stream) if stream else None)
        if rc != 0:
            raise VBHError(rc, "vbh_create")
        self._keep = None
        self._trace = None

    def close(self):
        if self._h:
            _lib().vbh_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def _opts(tol, max_iter, init_state, S, trace, precision=FP32, refine_iters=10, method=CAVI, grouped=False,
              stats=STATS_AUTO, loop=LOOP_AUTO):
        o = Opts()
        _lib().vbh_opts_default(ctypes.byref(o))
        o.tol = float(tol)
        o.max_iter = int(max_iter)
        o.precision = int(precision)
        o.refine_iters = int(refine_iters)
        o.method = int(method)
        o.grouped = 1 if grouped else 0
        o.stats = int(stats)
        o.loop = int(loop)
        keep = []
        if init_state is not None:
            st = dict_to_result(init_state, S) if isinstance(init_state, dict) else init_state
            keep.append(st)
            o.init = INIT_GIVEN
            o.init_state = ctypes.pointer(st)
        buf = None
        if trace:
            buf = np.zeros(int(max_iter) + 1)
            o.elbo_trace = buf.ctypes.data_as(_dp)
        return o, keep, buf

    def fit(self, r, d, S: int, prior: dict | None = None, tol: float = 1e-8, max_iter: int = 200,
            init_state=None, trace: bool = False, V: int | None = None, precision: int = FP32,
            refine_iters: int = 10, method: int = CAVI, grouped: bool = False, stats: int = STATS_AUTO,
            loop: int = LOOP_AUTO) -> dict:
        V = int(V if V is not None else (r.shape[0] if r is not None else 0))
        _check_inputs(r, d, V, S, "vbh_fit")
        pa = _PriorArgs(prior, S)
        o, keep, buf = self._opts(tol, max_iter, init_state, S, trace, precision, refine_iters, method, grouped,
                                  stats, loop)
        res = Result()
        rc = _lib().vbh_fit(self._h, _ptr(r), _ptr(d), V, int(S), ctypes.byref(pa.c), ctypes.byref(o),
                            ctypes.byref(res))
        if rc != 0:
            raise VBHError(rc, "vbh_fit")
        out = result_to_dict(res)
        if buf is not None:
            out["trace"] = buf[:res.iters + 1].copy()
        return out

    def fit_begin(self, r, d, S: int, prior: dict | None = None, tol: float = 1e-8, max_iter: int = 200,
                  init_state=None, trace: bool = False, V: int | None = None, precision: int = FP32,
                  refine_iters: int = 10, method: int = CAVI, grouped: bool = False, stats: int = STATS_AUTO,
                  loop: int = LOOP_AUTO):
        V = int(V if V is not None else (r.shape[0] if r is not None else 0))
        _check_inputs(r, d, V, S, "vbh_fit_begin")
        pa = _PriorArgs(prior, S)
        o, keep, buf = self._opts(tol, max_iter, init_state, S, trace, precision, refine_iters, method, grouped,
                                  stats, loop)
        rc = _lib().vbh_fit_begin(self._h, _ptr(r), _ptr(d), V, int(S), ctypes.byref(pa.c), ctypes.byref(o))
        if rc != 0:
            raise VBHError(rc, "vbh_fit_begin")
        self._keep = (r, d, keep)
        self._trace = buf

    def fit_step(self, nsweeps: int) -> bool:
        conv = ctypes.c_int()
        rc = _lib().vbh_fit_step(self._h, int(nsweeps), ctypes.byref(conv))
        if rc != 0:
            raise VBHError(rc, "vbh_fit_step")
        return bool(conv.value)

    def fit_result(self) -> dict:
        res = Result()
        rc = _lib().vbh_fit_result(self._h, ctypes.byref(res))
        if rc != 0:
            raise VBHError(rc, "vbh_fit_result")
        out = result_to_dict(res)
        if self._trace is not None:
            out["trace"] = self._trace[:res.iters + 1].copy()
        return out

    def fit_batched(self, rs, ds, Ss, priors=None, tol: float = 1e-8, max_iter: int = 200, init_states=None,
                    trace: bool = False, stats: int = STATS_AUTO) -> list:
        """``vbh_fit_batched``: B independent fits (lists of inputs, one S per
        data set; priors and init_states are lists of dicts or None)."""
        B = len(rs)
        if not (len(ds) == len(Ss) == B):
            raise ValueError("rs, ds and Ss must have the same length")
        Vs = (ctypes.c_int64 * B)(*[int(r.shape[0]) if r is not None else 0 for r in rs])
        Sa = (ctypes.c_int * B)(*[int(x) for x in Ss])
        for b in range(B):
            _check_inputs(rs[b], ds[b], Vs[b], Sa[b], f"vbh_fit_batched (data set {b})")
        rp = (ctypes.c_void_p * B)(*[(_ptr(r).value if r is not None else None) for r in rs])
        dp = (ctypes.c_void_p * B)(*[(_ptr(d).value if d is not None else None) for d in ds])
        keep = []
        pa = None
        if priors is not None:
            pa = (Prior * B)()
            for b in range(B):
                pb = _PriorArgs(priors[b], int(Ss[b]))
                keep.append(pb)
                pa[b] = pb.c
        o = Opts()
        _lib().vbh_opts_default(ctypes.byref(o))
        o.tol = float(tol)
        o.max_iter = int(max_iter)
        o.stats = int(stats)
        if init_states is not None:
            ia = (Result * B)()
            for b in range(B):
                ia[b] = dict_to_result(init_states[b], int(Ss[b])) if isinstance(init_states[b], dict) else init_states[b]
            keep.append(ia)
            o.init = INIT_GIVEN
            o.init_state = ctypes.cast(ia, ctypes.POINTER(Result))
        buf = None
        if trace:
            buf = np.zeros((B, int(max_iter) + 1))
            o.elbo_trace = buf.ctypes.data_as(_dp)
        out = (Result * B)()
        rc = _lib().vbh_fit_batched(self._h, B, Vs, Sa, rp, dp,
                                    ctypes.cast(pa, ctypes.POINTER(Prior)) if pa is not None else None,
                                    ctypes.byref(o), out)
        res = [result_to_dict(out[b]) for b in range(B)]
        if buf is not None:
            for b in range(B):
                res[b]["trace"] = buf[b, :res[b]["iters"] + 1].copy()
        if rc != 0:
            err = VBHError(rc, "vbh_fit_batched")
            err.results = res
            raise err
        return res

    def batched_plan(self) -> list:
        """``vbh_batched_plan``: per class of the last ``fit_batched`` call, the
        data-pass shape (tile, tiles per chunk, stages, blocks per SM) and the
        autotuner's pass time."""
        n = ctypes.c_int(0)
        _check(_lib().vbh_batched_plan(self._h, None, 0, ctypes.byref(n)), "vbh_batched_plan")
        buf = (BatchPlan * max(n.value, 1))()
        _check(_lib().vbh_batched_plan(self._h, buf, n.value, ctypes.byref(n)), "vbh_batched_plan")
        return [{f: getattr(buf[i], f) for f, _ in BatchPlan._fields_} for i in range(n.value)]

    def elbo(self, r, d, S: int, state: dict, prior: dict | None = None, V: int | None = None) -> float:
        V = int(V if V is not None else (r.shape[0] if r is not None else 0))
        _check_inputs(r, d, V, S, "vbh_elbo")
        pa = _PriorArgs(prior, S)
        q = dict_to_result(state, S)
        out = ctypes.c_double()
        rc = _lib().vbh_elbo(self._h, _ptr(r), _ptr(d), V, int(S), ctypes.byref(pa.c), ctypes.byref(q),
                             ctypes.byref(out))
        if rc != 0:
            raise VBHError(rc, "vbh_elbo")
        return out.value


STATIC_TRACE_MAX = 4097


def fit_static(r, d, S: int, prior: dict | None = None, tol: float = 1e-8, max_iter: int = 200,
               init_state=None, trace: bool = False, device: int = 0, stream=None, V: int | None = None,
               stats: int = STATS_AUTO) -> dict:
    """``vbh_fit_static``: the fit of ``Handle.fit`` for callers that cannot
    allocate device memory (no handle; the scratch is a static device array of
    the library).  r and d must be device tensors."""
    V = int(V if V is not None else (r.shape[0] if r is not None else 0))
    _check_inputs(r, d, V, S, "vbh_fit_static")
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    pa = _PriorArgs(prior, S)
    o, keep, buf = Handle._opts(tol, max_iter, init_state, S, trace, stats=stats)
    res = Result()
    rc = _lib().vbh_fit_static(_ptr(r), _ptr(d), V, int(S), ctypes.byref(pa.c), ctypes.byref(o), ctypes.byref(res),
                               int(device), ctypes.c_void_p(stream) if stream else None)
    if rc != 0:
        raise VBHError(rc, "vbh_fit_static")
    out = result_to_dict(res)
    if buf is not None:
        out["trace"] = buf[:res.iters + 1].copy()
    return out


WS_SMAX = 10
WS_F = 64
WS_P = 64


def ws_slots(S: int) -> np.ndarray:
    """Output slots a data set with S subpopulations uses (vbh_ws.h): kappa,
    ln E[rho], the packed Cholesky factor of Sigma0."""
    M = S - 1
    used = np.zeros(WS_P, dtype=bool)
    used[:M] = True
    used[9] = True
    for j in range(M):
        for k in range(j + 1):
            used[10 + j * (j + 1) // 2 + k] = True
    return used


class WarmStart:
    """The learned warm start (``include/vbh_ws.h``): one set encoder for
    every S in 2..10.  Data sets are given as lists of device tensors."""

    def __init__(self, seed: int = 1, device: int = 0, stream=None):
        lib = _lib()
        self._m = ctypes.c_void_p()
        st = getattr(stream, "cuda_stream", stream)
        rc = lib.vbh_ws_create(ctypes.byref(self._m), ctypes.c_uint64(seed), int(device),
                               ctypes.c_void_p(st) if st else None)
        if rc != 0:
            raise VBHError(rc, "vbh_ws_create")
        self.nparams = int(lib.vbh_ws_num_params(self._m))
        self.mean = np.zeros((WS_SMAX + 1, WS_P), dtype=np.float32)
        self.std = np.ones((WS_SMAX + 1, WS_P), dtype=np.float32)

    def close(self):
        if self._m:
            _lib().vbh_ws_destroy(self._m)
            self._m = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.empty(self.nparams, dtype=np.float32)
        _check(_lib().vbh_ws_get_params(self._m, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size),
               "vbh_ws_get_params")
        return out

    def set_params(self, theta) -> None:
        t = np.ascontiguousarray(theta, dtype=np.float32)
        _check(_lib().vbh_ws_set_params(self._m, t.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), t.size),
               "vbh_ws_set_params")

    def set_norm(self, mean, std) -> None:
        mu = np.ascontiguousarray(mean, dtype=np.float32).reshape(WS_SMAX + 1, WS_P)
        sd = np.ascontiguousarray(std, dtype=np.float32).reshape(WS_SMAX + 1, WS_P)
        fp = ctypes.POINTER(ctypes.c_float)
        _check(_lib().vbh_ws_set_norm(self._m, mu.ctypes.data_as(fp), sd.ctypes.data_as(fp)), "vbh_ws_set_norm")
        self.mean, self.std = mu.copy(), sd.copy()

    @staticmethod
    def _batch(rs, ds, Ss, ns=None):
        B = len(rs)
        for b in range(B):
            _check_inputs(rs[b], ds[b], int(rs[b].shape[0]), int(Ss[b]), f"set encoder (data set {b})")
        rp = (ctypes.c_void_p * B)(*[_ptr(x).value for x in rs])
        dp = (ctypes.c_void_p * B)(*[_ptr(x).value for x in ds])
        Vs = (ctypes.c_int64 * B)(*[int(x.shape[0]) for x in rs])
        Sa = (ctypes.c_int * B)(*[int(x) for x in Ss])
        na = (ctypes.c_int64 * B)(*([0] * B if ns is None else [int(x) for x in ns]))
        return B, rp, dp, Vs, Sa, na

    def features(self, r, d, S: int, n: int = 0):
        """The encoder's input for one data set (pooled observations x 64), FP32."""
        import torch
        V = int(r.shape[0])
        cnt = V if (n <= 0 or n >= V) else int(n)
        x = torch.empty((cnt, WS_F), dtype=torch.float32, device=r.device)
        _check(_lib().vbh_ws_features(self._m, _ptr(r), _ptr(d), V, int(S), int(n), _ptr(x)), "vbh_ws_features")
        return x

    def forward(self, rs, ds, Ss, ns=None):
        import torch
        B, rp, dp, Vs, Sa, na = self._batch(rs, ds, Ss, ns)
        out = torch.empty((B, WS_P), dtype=torch.float32, device=rs[0].device)
        _check(_lib().vbh_ws_forward(self._m, B, rp, dp, Vs, Sa, na, _ptr(out)), "vbh_ws_forward")
        return out

    def loss_grad(self, rs, ds, Ss, ns, target, weight):
        B, rp, dp, Vs, Sa, na = self._batch(rs, ds, Ss, ns)
        loss = ctypes.c_double()
        g = np.empty(self.nparams, dtype=np.float32)
        _check(_lib().vbh_ws_loss_grad(self._m, B, rp, dp, Vs, Sa, na, _ptr(target), _ptr(weight), ctypes.byref(loss),
                                       g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "vbh_ws_loss_grad")
        return loss.value, g

    def train_step(self, rs, ds, Ss, ns, target, weight, lr: float) -> float:
        B, rp, dp, Vs, Sa, na = self._batch(rs, ds, Ss, ns)
        loss = ctypes.c_double()
        _check(_lib().vbh_ws_train_step(self._m, B, rp, dp, Vs, Sa, na, _ptr(target), _ptr(weight), float(lr),
                                        ctypes.byref(loss)), "vbh_ws_train_step")
        return loss.value

    def predict(self, rs, ds, Ss, priors=None) -> list:
        """Starting points (result dicts) for fits with init_state, from all observations."""
        B, rp, dp, Vs, Sa, na = self._batch(rs, ds, Ss)
        keep = []
        pa = None
        if priors is not None:
            pa = (Prior * B)()
            for b in range(B):
                pb = _PriorArgs(priors[b], int(Ss[b]))
                keep.append(pb)
                pa[b] = pb.c
        res = (Result * B)()
        rc = _lib().vbh_ws_predict(self._m, B, rp, dp, Vs, Sa, ctypes.cast(pa, ctypes.POINTER(Prior)) if pa is not None
                                   else None, res)
        out = [result_to_dict(res[b]) for b in range(B)]
        if rc != 0:
            err = VBHError(rc, "vbh_ws_predict")
            err.results = out
            raise err
        return out


def _check(rc: int, what: str):
    if rc != 0:
        raise VBHError(rc, what)
