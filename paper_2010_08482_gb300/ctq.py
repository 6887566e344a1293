"""Python binding of libctq (include/ctq.h): argument marshalling only.

Every step of the local-trace evaluation runs in the library's CUDA kernels.
PyTorch supplies device memory and the current stream; nothing here computes
a trace.  If libctq.so is missing the import fails loudly (build it with
``python -c "import __graft_entry__ as g; g.build()"``); there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t, c_void_p
from typing import Optional

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libctq.so")

CTQ_OK = 0
CTQ_ERR_ARG, CTQ_ERR_NOMEM, CTQ_ERR_CUDA, CTQ_ERR_TIMEOUT = -1, -2, -3, -4
CTQ_ERR_UNSUPPORTED, CTQ_ERR_NUMERIC, CTQ_ERR_WORKSPACE = -5, -6, -7

CHAIN_OK, CHAIN_ZERO, CHAIN_REJECTED_EARLY, CHAIN_ACCEPTED, CHAIN_REJECTED = 0, 1, 2, 3, 4
CHAIN_ERR_ARG, CHAIN_ERR_TIMEOUT = -1, -4
DEBUG_STALL_WAIT = 1

KANAMORI, SLATER = 0, 1
MU_GIVEN, MU_PH_SYMMETRIC = 0, 1
SECTORS_N_SZ, SECTORS_N = 0, 1
FP64, TF32, BF16X3, TF32X3, F32X2 = 0, 1, 2, 3, 4


class CtqError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.ctq_strerror(code).decode()
        detail = _lib.ctq_last_error_message().decode()
        super().__init__(f"{where}: {msg} ({code}){': ' + detail if detail else ''}")
        self.code = code


class ModelParamsC(ctypes.Structure):
    _fields_ = [("n_orb", c_int), ("l", c_int), ("interaction", c_int), ("U", c_double), ("J", c_double),
                ("mu_mode", c_int), ("mu", c_double), ("n0", c_int), ("soc_xi", c_double),
                ("cf_re", POINTER(c_double)), ("cf_im", POINTER(c_double)), ("sector_mode", c_int),
                ("n_min", c_int), ("n_max", c_int), ("device", c_int)]


class InfoC(ctypes.Structure):
    _fields_ = [("n_flav", c_int), ("n_sec", c_int), ("max_dim", c_int), ("is_complex", c_int),
                ("mu", c_double), ("E_gs", c_double), ("n_block_elems", c_int64), ("n_alpha", c_int)]


class BatchC(ctypes.Structure):
    _fields_ = [("n_chains", c_int), ("beta", c_double), ("offsets", c_void_p), ("tau", c_void_p),
                ("op", c_void_p), ("log_threshold", c_void_p)]


class EvalOptsC(ctypes.Structure):
    _fields_ = [("precision", c_int), ("lazy", c_int), ("segment", c_int), ("max_ops", c_int),
                ("timeout_ns", c_int64), ("timing_events", c_void_p), ("debug_flags", c_int32),
                ("threads_per_cta", c_int32), ("ctas_per_sm", c_int32), ("stages", c_int32), ("tile_order", c_int32)]


class ResultC(ctypes.Structure):
    _fields_ = [("log_abs", c_void_p), ("phase", c_void_p), ("status", c_void_p), ("bounds", c_void_p)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libctq.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    P = c_void_p
    sig = {
        "ctq_build_impurity": (c_int, [POINTER(ModelParamsC), POINTER(P)]),
        "ctq_load_impurity": (c_int, [c_int, c_int, P, P, P, P, P, P, P, c_double, c_int, POINTER(P)]),
        "ctq_impurity_info": (c_int, [P, POINTER(InfoC)]),
        "ctq_get_sectors": (c_int, [P, P, P, P, P]),
        "ctq_get_energies": (c_int, [P, c_int, P]),
        "ctq_get_block": (c_int, [P, c_int, c_int, P, P]),
        "ctq_workspace_size": (c_size_t, [P, c_int, POINTER(EvalOptsC)]),
        "ctq_eval_traces": (c_int, [P, POINTER(BatchC), POINTER(EvalOptsC), POINTER(ResultC), P, c_size_t, P]),
        "ctq_launches_per_eval": (c_int, [P, POINTER(EvalOptsC)]),
        "ctq_free_impurity": (None, [P]),
        "ctq_strerror": (c_char_p, [c_int]),
        "ctq_last_error_message": (c_char_p, []),
        "ctq_probe_fma_rate": (c_int, [c_int, c_int, c_int, POINTER(c_double)]),
        "ctq_probe_exp": (c_int, [c_int, c_int, P, P, P]),
        "ctq_tc_gemm_check": (c_int, [c_int, P, P, P, c_int, c_int, c_int]),
        "ctq_big_gemm_check": (c_int, [c_int, P, P, P, c_int, c_int, c_int]),
        "ctq_trace_kernel": (c_int, [P, c_int]),
        "ctq_density_size": (c_size_t, [P]),
        "ctq_density_workspace_size": (c_size_t, [P, c_int, POINTER(EvalOptsC)]),
        "ctq_eval_density_matrices": (c_int, [P, POINTER(BatchC), POINTER(EvalOptsC), POINTER(ResultC), P, P,
                                              c_size_t, P]),
        "ctq_eval_traces_static": (c_int, [P, POINTER(BatchC), POINTER(EvalOptsC), POINTER(ResultC), P]),
        "ctq_add_bulla_operators": (c_int, [P, P, P]),
        "ctq_static_ratios": (c_int, [c_int, P, c_int, P, P, P, P, P, P]),
        "ctq_static_ratio_workspace_size": (c_size_t, [P, c_int, POINTER(EvalOptsC)]),
        "ctq_eval_static_ratios": (c_int, [P, POINTER(BatchC), POINTER(EvalOptsC), POINTER(ResultC), P, c_int, P,
                                           c_size_t, P]),
        "ctq_skiplist_create": (c_int, [P, c_double, ctypes.c_uint64, P, POINTER(P)]),
        "ctq_skiplist_set": (c_int, [P, c_int, P, P]),
        "ctq_skiplist_insert": (c_int, [P, c_int, P, P]),
        "ctq_skiplist_remove": (c_int, [P, c_int, P]),
        "ctq_skiplist_evaluate": (c_int, [P, POINTER(c_double), P, P]),
        "ctq_skiplist_set_precision": (c_int, [P, c_int]),
        "ctq_skiplist_free": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
EXPORTED = ("ctq_build_impurity", "ctq_load_impurity", "ctq_impurity_info", "ctq_get_sectors",
            "ctq_get_energies", "ctq_get_block", "ctq_workspace_size", "ctq_eval_traces",
            "ctq_launches_per_eval", "ctq_free_impurity", "ctq_strerror", "ctq_last_error_message",
            "ctq_probe_fma_rate", "ctq_probe_exp", "ctq_tc_gemm_check", "ctq_big_gemm_check", "ctq_eval_traces_static",
            "ctq_trace_kernel", "ctq_density_size", "ctq_density_workspace_size", "ctq_eval_density_matrices",
            "ctq_add_bulla_operators", "ctq_static_ratios", "ctq_static_ratio_workspace_size",
            "ctq_eval_static_ratios", "ctq_skiplist_create", "ctq_skiplist_set", "ctq_skiplist_insert",
            "ctq_skiplist_remove", "ctq_skiplist_evaluate", "ctq_skiplist_set_precision", "ctq_skiplist_free")

# Size of the library-owned scratch used by eval_traces_static (ctq.h).
STATIC_SCRATCH_BYTES = 32 << 20


def tc_gemm_check(A: np.ndarray, Bm: np.ndarray, split: int = 3, device: int = 0) -> np.ndarray:
    """D = A B^T through one tcgen05 MMA sequence (diagnostic, see ctq.h)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    Bm = np.ascontiguousarray(Bm, dtype=np.float32)
    N, K = Bm.shape
    D = np.zeros((128, N), np.float32)
    _check(_lib.ctq_tc_gemm_check(device, _ptr(A), _ptr(Bm), _ptr(D), N, K, split), "ctq_tc_gemm_check")
    return D


def big_gemm_check(A: np.ndarray, Bm: np.ndarray, precision: int = TF32X3, device: int = 0) -> np.ndarray:
    """D = A B^T with the large-block kernel's operand conventions (diagnostic, see ctq.h)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    Bm = np.ascontiguousarray(Bm, dtype=np.float32)
    N, K = Bm.shape
    D = np.zeros((128, N), np.float32)
    _check(_lib.ctq_big_gemm_check(device, _ptr(A), _ptr(Bm), _ptr(D), N, K, precision), "ctq_big_gemm_check")
    return D


def probe_fma_rate(device: int = 0, kind: int = 0, iters: int = 20000) -> float:
    """Measured multiply-add throughput (flop/s): FP64 FMA (kind 0), FP32 FMA
    (kind 1) or the FP64 warp-level MMA mma.sync.m8n8k4 (kind 2)."""
    out = c_double()
    _check(_lib.ctq_probe_fma_rate(device, kind, iters, ctypes.byref(out)), "ctq_probe_fma_rate")
    return out.value


def probe_exp(x, device: int = 0):
    """(table exponential of the float64 trace kernel, CUDA exp) of the host
    values x <= 0, both computed on the device."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    yt, yl = np.empty_like(x), np.empty_like(x)
    _check(_lib.ctq_probe_exp(device, x.size, _ptr(x), _ptr(yt), _ptr(yl)), "ctq_probe_exp")
    return yt, yl


def lib_path() -> str:
    return _LIB_PATH


def strerror(code: int) -> str:
    return _lib.ctq_strerror(code).decode()


def _check(code: int, where: str):
    if code != CTQ_OK:
        raise CtqError(code, where)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(c_void_p) if a is not None else None


class Impurity:
    """Owner of a ctq_impurity handle (freed with ctq_free_impurity)."""

    def __init__(self, handle: c_void_p):
        self.handle = handle
        info = InfoC()
        _check(_lib.ctq_impurity_info(handle, ctypes.byref(info)), "ctq_impurity_info")
        self.n_flav = info.n_flav
        self.n_sec = info.n_sec
        self.max_dim = info.max_dim
        self.is_complex = bool(info.is_complex)
        self.mu = info.mu
        self.E_gs = info.E_gs
        self.n_block_elems = info.n_block_elems
        self.n_alpha = info.n_alpha

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.ctq_free_impurity(h)
            self.handle = None

    def sectors(self):
        dims = np.zeros(self.n_sec, np.int32)
        N = np.zeros(self.n_sec, np.int32)
        Emin = np.zeros(self.n_sec)
        s = np.zeros((2 * self.n_flav, self.n_sec), np.int32)
        _check(_lib.ctq_get_sectors(self.handle, _ptr(dims), _ptr(N), _ptr(Emin), _ptr(s)), "ctq_get_sectors")
        return dims, N, Emin, s

    def energies(self, q: int) -> np.ndarray:
        dims = self.sectors()[0]
        E = np.zeros(int(dims[q]))
        _check(_lib.ctq_get_energies(self.handle, q, _ptr(E)), "ctq_get_energies")
        return E

    def add_bulla_operators(self, h: Optional[np.ndarray] = None):
        """ctq_add_bulla_operators: operator codes 2 n_flav + f become the
        Bulla operators [c_f, U]; h: the one-body matrix t - mu (n_flav x
        n_flav, flavour basis), or None for the one the library built."""
        h_re = h_im = None
        if h is not None:
            h = np.asarray(h, dtype=np.complex128).reshape(self.n_flav, self.n_flav)
            h_re = np.ascontiguousarray(h.real)
            h_im = np.ascontiguousarray(h.imag) if np.any(h.imag != 0) else None
        _check(_lib.ctq_add_bulla_operators(self.handle, _ptr(h_re), _ptr(h_im)), "ctq_add_bulla_operators")
        info = InfoC()
        _check(_lib.ctq_impurity_info(self.handle, ctypes.byref(info)), "ctq_impurity_info")
        self.n_alpha = info.n_alpha
        self.n_block_elems = info.n_block_elems

    def block(self, alpha: int, q: int) -> np.ndarray:
        dims, _, _, s = self.sectors()
        # a Bulla operator 2 n_flav + f maps sectors as c_f (code 2 f)
        row = alpha if alpha < 2 * self.n_flav else 2 * (alpha - 2 * self.n_flav)
        qp = int(s[row, q])
        if qp < 0:
            raise CtqError(CTQ_ERR_ARG, "zero block")
        re = np.zeros((int(dims[qp]), int(dims[q])))
        im = np.zeros_like(re)
        _check(_lib.ctq_get_block(self.handle, alpha, q, _ptr(re), _ptr(im)), "ctq_get_block")
        return re + 1j * im if self.is_complex else re


def build_impurity(p, device: int = 0) -> Impurity:
    """ctq_build_impurity from a workloads.ModelParams-like object."""
    nf = 2 * p.n_orb
    cf_re = cf_im = None
    if p.cf is not None:
        cf = np.asarray(p.cf, dtype=np.complex128).reshape(nf, nf)
        cf_re = np.ascontiguousarray(cf.real)
        cf_im = np.ascontiguousarray(cf.imag)
    c = ModelParamsC()
    c.n_orb = p.n_orb
    c.l = p.l
    c.interaction = KANAMORI if p.interaction == "kanamori" else SLATER
    c.U, c.J = p.U, p.J
    c.mu_mode = MU_PH_SYMMETRIC if p.mu is None else MU_GIVEN
    c.mu = 0.0 if p.mu is None else float(p.mu)
    c.n0 = p.n0
    c.soc_xi = p.soc_xi
    c.cf_re = cf_re.ctypes.data_as(POINTER(c_double)) if cf_re is not None else None
    c.cf_im = cf_im.ctypes.data_as(POINTER(c_double)) if cf_im is not None else None
    c.sector_mode = SECTORS_N_SZ if p.sector_mode == "n_sz" else SECTORS_N
    c.n_min, c.n_max = p.n_min, p.n_max
    c.device = device
    h = c_void_p()
    _check(_lib.ctq_build_impurity(ctypes.byref(c), ctypes.byref(h)), "ctq_build_impurity")
    return Impurity(h)


def load_impurity(n_flav: int, dims, N, energies, s_table, blocks, mu: float = 0.0,
                  opnorm=None, device: int = 0) -> Impurity:
    """ctq_load_impurity: blocks is a dict {(alpha, q): matrix} (every nonzero block)."""
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    n_sec = len(dims)
    N = np.ascontiguousarray(N, dtype=np.int32)
    E = np.ascontiguousarray(np.concatenate([np.asarray(e, np.float64) for e in energies]))
    s = np.ascontiguousarray(s_table, dtype=np.int32).reshape(2 * n_flav, n_sec)
    parts, norms = [], []
    is_c = any(np.iscomplexobj(b) for b in blocks.values())
    for a in range(2 * n_flav):
        for q in range(n_sec):
            if s[a, q] < 0:
                continue
            parts.append(np.asarray(blocks[(a, q)]).reshape(-1))
            if opnorm is not None:
                norms.append(opnorm[(a, q)])
    flat = np.concatenate(parts) if parts else np.zeros(0)
    re = np.ascontiguousarray(flat.real, dtype=np.float64)
    im = np.ascontiguousarray(flat.imag, dtype=np.float64) if is_c else None
    nrm = np.ascontiguousarray(norms, dtype=np.float64) if opnorm is not None else None
    h = c_void_p()
    _check(_lib.ctq_load_impurity(n_flav, n_sec, _ptr(dims), _ptr(N), _ptr(E), _ptr(s), _ptr(re), _ptr(im),
                                  _ptr(nrm), float(mu), device, ctypes.byref(h)), "ctq_load_impurity")
    return Impurity(h)


# Launch-tuning keys of ctq_eval_opts (0 = library default); see ctq.h.
TUNE_KEYS = ("threads_per_cta", "ctas_per_sm", "stages", "tile_order")


def _opts(precision=FP64, lazy=False, segment=8, max_ops=0, timeout_ns=0, events=None, debug_flags=0,
          tune=None) -> EvalOptsC:
    o = EvalOptsC()
    o.precision, o.lazy, o.segment, o.max_ops, o.timeout_ns = precision, int(lazy), segment, max_ops, timeout_ns
    o.timing_events = events
    o.debug_flags = debug_flags
    for k, v in (tune or {}).items():
        if k not in TUNE_KEYS:
            raise ValueError(f"unknown launch-tuning key {k!r}")
        setattr(o, k, int(v))
    return o


def workspace_size(imp: Impurity, n_chains: int, precision=FP64, lazy=False, segment=8, max_ops=0) -> int:
    o = _opts(precision, lazy, segment, max_ops)
    return int(_lib.ctq_workspace_size(imp.handle, n_chains, ctypes.byref(o)))


# ctq_trace_kernel results
KERNEL_FP64_SHARED, KERNEL_FP64_LARGE, KERNEL_TC_SMALL, KERNEL_TC_LARGE = 0, 1, 2, 3


def trace_kernel(imp: Impurity, precision: int) -> int:
    """Which trace kernel evaluates this impurity at this precision (KERNEL_*)."""
    k = int(_lib.ctq_trace_kernel(imp.handle, precision))
    _check(min(k, 0), "ctq_trace_kernel")
    return k


def launches_per_eval(imp: Impurity, precision=FP64) -> int:
    o = _opts(precision)
    return int(_lib.ctq_launches_per_eval(imp.handle, ctypes.byref(o)))


def eval_traces(imp: Impurity, n_chains: int, beta: float, offsets, tau, op, log_threshold,
                log_abs, phase, status, bounds, workspace, workspace_bytes: int, stream,
                precision=FP64, lazy=False, segment=8, max_ops=0, timeout_ns=0, events=None, debug_flags=0,
                tune=None):
    """ctq_eval_traces with raw device pointers (ints) and a cudaStream_t (int);
    events: optional address of an array of cudaEvent_t handles (see ctq.h);
    tune: optional launch-tuning dict (TUNE_KEYS)."""
    b = BatchC()
    b.n_chains, b.beta = n_chains, beta
    b.offsets, b.tau, b.op, b.log_threshold = offsets, tau, op, log_threshold
    r = ResultC()
    r.log_abs, r.phase, r.status, r.bounds = log_abs, phase, status, bounds
    o = _opts(precision, lazy, segment, max_ops, timeout_ns, events, debug_flags, tune)
    _check(_lib.ctq_eval_traces(imp.handle, ctypes.byref(b), ctypes.byref(o), ctypes.byref(r),
                                workspace, workspace_bytes, stream), "ctq_eval_traces")


def eval_traces_static(imp: Impurity, n_chains: int, beta: float, offsets, tau, op, log_threshold,
                       log_abs, phase, status, bounds, stream, precision=FP64, lazy=False, segment=8,
                       max_ops=0, timeout_ns=0):
    """ctq_eval_traces_static: as eval_traces, with the scratch in the library's
    fixed device array instead of a caller workspace (for callers that cannot
    allocate device memory; see ctq.h for the size limit and the sharing rule)."""
    b = BatchC()
    b.n_chains, b.beta = n_chains, beta
    b.offsets, b.tau, b.op, b.log_threshold = offsets, tau, op, log_threshold
    r = ResultC()
    r.log_abs, r.phase, r.status, r.bounds = log_abs, phase, status, bounds
    o = _opts(precision, lazy, segment, max_ops, timeout_ns, None)
    _check(_lib.ctq_eval_traces_static(imp.handle, ctypes.byref(b), ctypes.byref(o), ctypes.byref(r), stream),
           "ctq_eval_traces_static")


free_impurity = Impurity.__del__


# --------------------------------------------------------------------------- torch helpers

class DeviceBatch:
    """A workloads.Batch copied to device tensors (int32 offsets/op, float64 tau)."""

    def __init__(self, batch, device="cuda", log_threshold: Optional[np.ndarray] = None):
        import torch
        self.n_chains = batch.n_chains
        self.n_ops = len(batch.tau)
        self.beta = float(batch.beta)
        self.max_ops = int(np.max(np.diff(batch.offsets))) if batch.n_chains else 0
        self.offsets = torch.as_tensor(np.asarray(batch.offsets, np.int32), device=device)
        n = max(1, len(batch.tau))
        self.tau = torch.zeros(n, dtype=torch.float64, device=device)
        self.op = torch.zeros(n, dtype=torch.int32, device=device)
        if len(batch.tau):
            self.tau[: len(batch.tau)] = torch.as_tensor(np.asarray(batch.tau, np.float64), device=device)
            self.op[: len(batch.op)] = torch.as_tensor(np.asarray(batch.op, np.int32), device=device)
        self.log_threshold = None
        if log_threshold is not None:
            self.log_threshold = torch.as_tensor(np.asarray(log_threshold, np.float64), device=device)


class TraceEvaluator:
    """Pre-allocates the workspace and result tensors for batches of up to
    n_chains chains with at most max_ops operators, then evaluates batches on
    the current torch stream (no allocation per call)."""

    def __init__(self, imp: Impurity, n_chains: int, max_ops: int, precision=FP64, segment=8,
                 with_bounds=True, device="cuda", tune=None):
        import torch
        self.imp = imp
        self.n_chains = n_chains
        self.max_ops = max_ops
        self.precision = precision
        self.tune = dict(tune or {})  # launch tuning (TUNE_KEYS), e.g. from autotune.tune()
        self.segment = segment
        self.n_seg = (max_ops + segment - 1) // segment
        self.ws_bytes = workspace_size(imp, n_chains, precision, False, segment, max_ops)
        # 256-byte aligned workspace
        self._ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=device)
        base = self._ws.data_ptr()
        self.ws_ptr = (base + 255) // 256 * 256
        self.log_abs = torch.empty(n_chains, dtype=torch.float64, device=device)
        self.phase = torch.empty(2 * n_chains, dtype=torch.float64, device=device)
        self.status = torch.empty(n_chains, dtype=torch.int32, device=device)
        self.bounds = (torch.empty(n_chains * (self.n_seg + 1), dtype=torch.float64, device=device)
                       if with_bounds else None)

    def __call__(self, db: DeviceBatch, lazy=False, stream=None, events=None, timeout_ns=0, debug_flags=0):
        import torch
        if db.n_chains > self.n_chains or db.max_ops > self.max_ops:
            raise ValueError("batch larger than the evaluator was sized for")
        s = torch.cuda.current_stream() if stream is None else stream
        thr = db.log_threshold.data_ptr() if db.log_threshold is not None else None
        eval_traces(self.imp, db.n_chains, db.beta, db.offsets.data_ptr(), db.tau.data_ptr(), db.op.data_ptr(),
                    thr, self.log_abs.data_ptr(), self.phase.data_ptr(), self.status.data_ptr(),
                    self.bounds.data_ptr() if self.bounds is not None else None,
                    self.ws_ptr, self.ws_bytes, s.cuda_stream, self.precision, lazy, self.segment, self.max_ops,
                    timeout_ns, events, debug_flags, self.tune)

    def results(self, n_chains: Optional[int] = None):
        n = self.n_chains if n_chains is None else n_chains
        out = {
            "log_abs": self.log_abs[:n].cpu().numpy(),
            "phase": self.phase[: 2 * n].cpu().numpy().reshape(n, 2),
            "status": self.status[:n].cpu().numpy(),
        }
        if self.bounds is not None:
            out["bounds"] = self.bounds[: n * (self.n_seg + 1)].cpu().numpy().reshape(n, self.n_seg + 1)
        return out


def bulla_code(n_flav: int, f: int) -> int:
    """Operator code of the Bulla operator [c_f, U] (after ctq_add_bulla_operators)."""
    return 2 * n_flav + f


def static_ratios(chain, n_chains: int, log_abs, phase, log_abs_u, phase_u, out, stream=None):
    """ctq_static_ratios on device tensors: chain int32 [m] (configuration of
    each replaced sequence), log_abs / phase of the configurations, log_abs_u /
    phase_u of the replaced sequences, out float64 [2 m] (h^st as re, im)."""
    import torch
    m = int(chain.numel())
    if out.numel() < 2 * m or log_abs_u.numel() < m or phase_u.numel() < 2 * m:
        raise ValueError("ratio buffers smaller than the sequence count")
    s = torch.cuda.current_stream() if stream is None else stream
    _check(_lib.ctq_static_ratios(m, chain.data_ptr(), int(n_chains), log_abs.data_ptr(), phase.data_ptr(),
                                  log_abs_u.data_ptr(), phase_u.data_ptr(), out.data_ptr(), s.cuda_stream),
           "ctq_static_ratios")


class StaticImprovedEvaluator:
    """Static part of the improved estimator for the self-energy (Eq.
    PImprovedEstimatorStatic) for every annihilator of every configuration:
    evaluates the configurations and the replaced sequences
    (workloads.bulla_sequences) with the library's trace kernels, then
    h^st = w^U / w with ctq_static_ratios.  The impurity must hold the Bulla
    operators (Impurity.add_bulla_operators)."""

    def __init__(self, imp: Impurity, n_chains: int, n_seq: int, max_ops: int, precision=FP64, device="cuda",
                 tune=None):
        import torch
        if imp.n_alpha < 3 * imp.n_flav:
            raise ValueError("the impurity has no Bulla operators (Impurity.add_bulla_operators)")
        self.base = TraceEvaluator(imp, n_chains, max_ops, precision=precision, with_bounds=False, device=device,
                                   tune=tune)
        self.repl = TraceEvaluator(imp, n_seq, max_ops, precision=precision, with_bounds=False, device=device,
                                   tune=tune)
        self.h = torch.empty(2 * max(n_seq, 1), dtype=torch.float64, device=device)

    def __call__(self, db: "DeviceBatch", db_u: "DeviceBatch", chain, stream=None):
        self.base(db, stream=stream)
        self.repl(db_u, stream=stream)
        static_ratios(chain, db.n_chains, self.base.log_abs, self.base.phase, self.repl.log_abs, self.repl.phase,
                      self.h, stream)

    def ratios(self, n_seq: int) -> np.ndarray:
        v = self.h[: 2 * n_seq].cpu().numpy()
        return v[0::2] + 1j * v[1::2]


class FusedStaticEvaluator:
    """ctq_eval_static_ratios: the static improved-estimator ratio of every
    annihilator of every configuration in one pass over the configurations
    (forward and backward products, one extra product per annihilator),
    float64.  The impurity must hold the Bulla operators."""

    def __init__(self, imp: Impurity, n_chains: int, max_ops: int, n_ops: int, device="cuda"):
        import torch
        if imp.n_alpha < 3 * imp.n_flav:
            raise ValueError("the impurity has no Bulla operators (Impurity.add_bulla_operators)")
        self.imp = imp
        self.n_chains, self.max_ops, self.n_ops = n_chains, max_ops, n_ops
        o = _opts(FP64, False, 8, max_ops)
        self.ws_bytes = int(_lib.ctq_static_ratio_workspace_size(imp.handle, n_chains, ctypes.byref(o)))
        self._ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=device)
        self.ws_ptr = (self._ws.data_ptr() + 255) // 256 * 256
        self.log_abs = torch.empty(n_chains, dtype=torch.float64, device=device)
        self.phase = torch.empty(2 * n_chains, dtype=torch.float64, device=device)
        self.status = torch.empty(n_chains, dtype=torch.int32, device=device)
        self.h = torch.empty(2 * max(n_ops, 1), dtype=torch.float64, device=device)

    def __call__(self, db: "DeviceBatch", stream=None):
        import torch
        if db.n_chains > self.n_chains or db.max_ops > self.max_ops or db.n_ops > self.n_ops:
            raise ValueError("batch larger than the evaluator was sized for")
        s = torch.cuda.current_stream() if stream is None else stream
        b = BatchC()
        b.n_chains, b.beta = db.n_chains, db.beta
        b.offsets, b.tau, b.op, b.log_threshold = db.offsets.data_ptr(), db.tau.data_ptr(), db.op.data_ptr(), None
        r = ResultC()
        r.log_abs, r.phase, r.status, r.bounds = (self.log_abs.data_ptr(), self.phase.data_ptr(),
                                                  self.status.data_ptr(), None)
        o = _opts(FP64, False, 8, self.max_ops)
        _check(_lib.ctq_eval_static_ratios(self.imp.handle, ctypes.byref(b), ctypes.byref(o), ctypes.byref(r),
                                           self.h.data_ptr(), db.n_ops, self.ws_ptr, self.ws_bytes, s.cuda_stream),
               "ctq_eval_static_ratios")

    def ratios(self, n_ops: int) -> np.ndarray:
        """h^st by global operator index (0 where the operator is not an annihilator)."""
        v = self.h[: 2 * n_ops].cpu().numpy()
        return v[0::2] + 1j * v[1::2]


def log_value(log_abs: float, phase) -> complex:
    """w as a complex number (may overflow for large log|w|)."""
    if log_abs == -math.inf:
        return 0j
    return complex(phase[0], phase[1]) * math.exp(log_abs)


class DensityEvaluator:
    """The reduced-density-matrix estimator of every chain (ctq.h,
    ctq_eval_density_matrices): pre-allocated workspace, traces and per-chain
    estimators; evaluates on the current torch stream."""

    def __init__(self, imp: Impurity, n_chains: int, max_ops: int, device="cuda"):
        import torch
        self.imp = imp
        self.n_chains = n_chains
        self.max_ops = max_ops
        self.size = int(_lib.ctq_density_size(imp.handle))
        o = _opts(FP64, False, 8, max_ops)
        self.ws_bytes = int(_lib.ctq_density_workspace_size(imp.handle, n_chains, ctypes.byref(o)))
        self._ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=device)
        self.ws_ptr = (self._ws.data_ptr() + 255) // 256 * 256
        self.log_abs = torch.empty(n_chains, dtype=torch.float64, device=device)
        self.phase = torch.empty(2 * n_chains, dtype=torch.float64, device=device)
        self.status = torch.empty(n_chains, dtype=torch.int32, device=device)
        self.rho = torch.empty(n_chains * self.size, dtype=torch.float64, device=device)

    def __call__(self, db: "DeviceBatch", stream=None):
        import torch
        if db.n_chains > self.n_chains or db.max_ops > self.max_ops:
            raise ValueError("batch larger than the evaluator was sized for")
        s = torch.cuda.current_stream() if stream is None else stream
        b = BatchC()
        b.n_chains, b.beta = db.n_chains, db.beta
        b.offsets, b.tau, b.op, b.log_threshold = db.offsets.data_ptr(), db.tau.data_ptr(), db.op.data_ptr(), None
        r = ResultC()
        r.log_abs, r.phase, r.status, r.bounds = (self.log_abs.data_ptr(), self.phase.data_ptr(),
                                                  self.status.data_ptr(), None)
        o = _opts(FP64, False, 8, self.max_ops)
        _check(_lib.ctq_eval_density_matrices(self.imp.handle, ctypes.byref(b), ctypes.byref(o), ctypes.byref(r),
                                              self.rho.data_ptr(), self.ws_ptr, self.ws_bytes, s.cuda_stream),
               "ctq_eval_density_matrices")

    def blocks(self, chain: int):
        """The estimator of one chain as {sector q: d_q x d_q matrix}."""
        dims = self.imp.sectors()[0]
        flat = self.rho[chain * self.size:(chain + 1) * self.size].cpu().numpy()
        if self.imp.is_complex:
            flat = flat[0::2] + 1j * flat[1::2]
        out, o = {}, 0
        for q, d in enumerate(dims):
            d = int(d)
            out[q] = flat[o:o + d * d].reshape(d, d)
            o += d * d
        return out


class SkipListStatsC(ctypes.Structure):
    _fields_ = [("products", c_int64), ("leaves", c_int64), ("reused", c_int64), ("cached", c_int64),
                ("flops", c_double), ("n_ops", c_int), ("n_strings", c_int), ("device_bytes", c_int64),
                ("launches", c_int64), ("rounds", c_int)]


class SkipListTrace:
    """ctq_skiplist: the local trace of one configuration kept as a skip
    list of cached segment products, updated by inserting and removing
    operators (see ctq.h).  Host arrays in, host results out."""

    def __init__(self, imp: Impurity, beta: float, seed: int = 0, stream=None, precision=FP64):
        import torch
        self.imp = imp
        s = torch.cuda.current_stream() if stream is None else stream
        self._stream = s
        h = c_void_p()
        _check(_lib.ctq_skiplist_create(imp.handle, float(beta), ctypes.c_uint64(seed), s.cuda_stream,
                                        ctypes.byref(h)), "ctq_skiplist_create")
        self.handle = h
        if precision != FP64:
            self.set_precision(precision)

    def set_precision(self, precision):
        """FP64 (float64 SIMT products) or BF16X3 (tensor-core products)."""
        _check(_lib.ctq_skiplist_set_precision(self.handle, precision), "ctq_skiplist_set_precision")

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.ctq_skiplist_free(h)
            self.handle = None

    def set(self, tau, op):
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        op = np.ascontiguousarray(op, dtype=np.int32)
        _check(_lib.ctq_skiplist_set(self.handle, len(tau), _ptr(tau), _ptr(op)), "ctq_skiplist_set")

    def insert(self, tau, op):
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        op = np.ascontiguousarray(op, dtype=np.int32)
        _check(_lib.ctq_skiplist_insert(self.handle, len(tau), _ptr(tau), _ptr(op)), "ctq_skiplist_insert")

    def remove(self, tau):
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        _check(_lib.ctq_skiplist_remove(self.handle, len(tau), _ptr(tau)), "ctq_skiplist_remove")

    def evaluate(self):
        """(log|w|, phase as complex, stats dict) of the current configuration."""
        la = c_double()
        ph = np.zeros(2)
        st = SkipListStatsC()
        _check(_lib.ctq_skiplist_evaluate(self.handle, ctypes.byref(la), _ptr(ph), ctypes.byref(st)),
               "ctq_skiplist_evaluate")
        stats = {k: getattr(st, k) for k, _ in SkipListStatsC._fields_}
        return la.value, complex(ph[0], ph[1]), stats
