"""Thin Python binding of the LEAD C ABI (include/lead.h): argument marshalling only.

Every computation runs in liblead.so; this module loads it with ctypes, passes torch tensors'
device pointers and the current CUDA stream, and raises on any non-zero status. There is no
fallback: if the library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# LEAD_CHECKED=1 selects the checked build (kernels test their table indices; failures come back
# as LEAD_ECHECK); build it with `python -m paper_2605_17796_gb300.build --checked`.
CHECKED = os.environ.get("LEAD_CHECKED", "0") not in ("", "0")
LIB_PATH = os.path.join(HERE, "liblead_checked.so" if CHECKED else "liblead.so")

NOISE_X, NOISE_Z, NOISE_DEPOL = 0, 1, 2
ST_CONVERGED, ST_MAX_ITER, ST_OSD = 1, 2, 4
ECHECK = -10                      # checked build: a kernel index failed its bounds check
BUILD_CHECKED = 1                 # lead_build_flags() bit of the checked build
PREC_FP32, PREC_BF16, PREC_FP16 = 0, 1, 2
EST_EXACT, EST_MINSUM = 0, 1
NOALLOC_TABLE_BYTES = 444928      # LEAD_NOALLOC_TABLE_BYTES: the fixed tables of lead_decode_noalloc

_c_int32_p = ctypes.POINTER(ctypes.c_int32)
_c_uint8_p = ctypes.POINTER(ctypes.c_uint8)


class LeadGroup(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("mul", _c_int32_p)]


class LeadCodeInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("order", ctypes.c_int32), ("delta", ctypes.c_int32),
                ("k_A", ctypes.c_int32), ("k_B", ctypes.c_int32),
                ("m_l", ctypes.c_int32 * 2), ("m", ctypes.c_int32 * 2), ("rank", ctypes.c_int32 * 2),
                ("k", ctypes.c_int32), ("words_n", ctypes.c_int32), ("words_m", ctypes.c_int32 * 2),
                ("max_row_weight", ctypes.c_int32 * 2), ("prepared_device", ctypes.c_int32)]


class LeadDecodeOpts(ctypes.Structure):
    _fields_ = [("side", ctypes.c_int32), ("use_lead", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("alpha", ctypes.c_float), ("p", ctypes.c_double),
                ("estimator", ctypes.c_int32)]


class LeadServerConfig(ctypes.Structure):
    _fields_ = [("ncodes", ctypes.c_int32), ("codes", ctypes.POINTER(ctypes.c_void_p)),
                ("p_side", ctypes.POINTER(ctypes.c_double)), ("sides_mask", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("streams", ctypes.c_int32), ("budget_bytes", ctypes.c_size_t),
                ("max_iter", ctypes.c_int32), ("alpha", ctypes.c_float), ("precision", ctypes.c_int32)]


class LeadServerResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("code", ctypes.c_int32), ("status", ctypes.c_uint8 * 2),
                ("arrival_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64)]


EXPORTS = {
    "lead_build_code": (ctypes.c_int, [ctypes.POINTER(LeadGroup), _c_int32_p, _c_int32_p, ctypes.c_int32,
                                       _c_uint8_p, ctypes.c_int32, _c_uint8_p, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "lead_code_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(LeadCodeInfo)]),
    "lead_code_get_views": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _c_int32_p]),
    "lead_code_get_check_matrix": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _c_uint8_p]),
    "lead_code_compile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]),
    "lead_code_prepare": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "lead_code_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                          ctypes.c_int64, ctypes.c_char_p, ctypes.c_size_t]),
    "lead_code_get_enumerators": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _c_int32_p, _c_int32_p,
                                                 ctypes.POINTER(ctypes.c_uint64)]),
    "lead_free_code": (None, [ctypes.c_void_p]),
    "lead_sample": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_int64,
                                   ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lead_prior_llr": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "lead_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.POINTER(LeadDecodeOpts), ctypes.c_int64]),
    "lead_local_table": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "lead_local_table_est": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lead_local_estimate": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(LeadDecodeOpts), ctypes.c_void_p,
                                           ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                           ctypes.c_void_p]),
    "lead_decode": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(LeadDecodeOpts), ctypes.c_void_p,
                                   ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "lead_decode_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(LeadDecodeOpts), ctypes.c_void_p,
                                           ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "lead_priors_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.POINTER(LeadDecodeOpts),
                                                      ctypes.c_int64]),
    "lead_local_estimate_priors": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(LeadDecodeOpts), ctypes.c_void_p,
                                                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                                  ctypes.c_void_p]),
    "lead_decode_priors": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(LeadDecodeOpts), ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_void_p]),
    "lead_iterated_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.POINTER(LeadDecodeOpts),
                                                        ctypes.c_int64]),
    "lead_decode_iterated": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(LeadDecodeOpts), ctypes.c_int32,
                                            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                            ctypes.c_void_p]),
    "lead_osd_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.POINTER(LeadDecodeOpts), ctypes.c_int64]),
    "lead_osd": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(LeadDecodeOpts), ctypes.c_int32, ctypes.c_void_p,
                                ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "lead_check": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "lead_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lead_build_flags": (ctypes.c_int, []),
    "lead_code_check_record": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "lead_code_device_errors": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int32]),
    "lead_server_create": (ctypes.c_int, [ctypes.POINTER(LeadServerConfig), ctypes.POINTER(ctypes.c_void_p)]),
    "lead_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "lead_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(LeadServerResult), ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "lead_server_pending": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "lead_server_clock_ns": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "lead_server_destroy": (None, [ctypes.c_void_p]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        flag = " --checked" if CHECKED else ""
        raise ImportError(f"{os.path.basename(LIB_PATH)} is not built ({LIB_PATH}); run "
                          f"`python -m paper_2605_17796_gb300.build{flag}`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


class LeadError(RuntimeError):
    def __init__(self, call: str, rc: int):
        super().__init__(f"{call} failed: {rc} ({LIB.lead_status_string(rc).decode()})")
        self.rc = rc


def _check(call: str, rc: int):
    if rc != 0:
        raise LeadError(call, rc)


def _ptr(t) -> int | None:
    """Device pointer of a CUDA tensor (None for None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(stream=None) -> int | None:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def prior_llr(p, llr, stream=None):
    """llr[i] = lambda(p[i]) = ln((1 - p[i])/p[i]) in binary32 (lead_prior_llr); p, llr float32 CUDA
    tensors of the same size."""
    if p.numel() != llr.numel():
        raise ValueError("p and llr must have the same number of elements")
    _check("lead_prior_llr", LIB.lead_prior_llr(_ptr(p), _ptr(llr), p.numel(), _stream(stream)))


@dataclass
class CodeInfo:
    n: int
    order: int
    delta: int
    k_A: int
    k_B: int
    m_l: tuple
    m: tuple
    rank: tuple
    k: int
    words_n: int
    words_m: tuple
    max_row_weight: tuple
    prepared_device: int


class Code:
    """A quantum Tanner code built by the library from (G, A, B, C_A[, C_B])."""

    def __init__(self, mul: np.ndarray, A, B, GA: np.ndarray, GB: np.ndarray | None = None):
        mul = np.ascontiguousarray(mul, dtype=np.int32)
        A = np.ascontiguousarray(A, dtype=np.int32)
        B = np.ascontiguousarray(B, dtype=np.int32)
        GA = np.ascontiguousarray(GA, dtype=np.uint8)
        grp = LeadGroup(order=mul.shape[0], mul=mul.ctypes.data_as(_c_int32_p))
        out = ctypes.c_void_p()
        gb_p = None
        kB = 0
        if GB is not None:
            GB = np.ascontiguousarray(GB, dtype=np.uint8)
            gb_p = GB.ctypes.data_as(_c_uint8_p)
            kB = GB.shape[0]
        rc = LIB.lead_build_code(ctypes.byref(grp), A.ctypes.data_as(_c_int32_p), B.ctypes.data_as(_c_int32_p),
                                 len(A), GA.ctypes.data_as(_c_uint8_p), GA.shape[0], gb_p, kB, ctypes.byref(out))
        _check("lead_build_code", rc)
        self._h = out
        self.info = self._info()

    @classmethod
    def from_instance(cls, inst) -> "Code":
        G = inst.G
        return cls(G.mul, inst.A, inst.B, inst.GA, inst.GB)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            LIB.lead_free_code(h)
            self._h = None

    def _info(self) -> CodeInfo:
        ci = LeadCodeInfo()
        _check("lead_code_get_info", LIB.lead_code_get_info(self._h, ctypes.byref(ci)))
        return CodeInfo(ci.n, ci.order, ci.delta, ci.k_A, ci.k_B, tuple(ci.m_l), tuple(ci.m), tuple(ci.rank),
                        ci.k, ci.words_n, tuple(ci.words_m), tuple(ci.max_row_weight), ci.prepared_device)

    def views(self, side: int) -> np.ndarray:
        out = np.zeros((self.info.order, self.info.delta ** 2), dtype=np.int32)
        _check("lead_code_get_views", LIB.lead_code_get_views(self._h, side, out.ctypes.data_as(_c_int32_p)))
        return out

    def check_matrix(self, side: int) -> np.ndarray:
        out = np.zeros((self.info.m[side], self.info.n), dtype=np.uint8)
        _check("lead_code_get_check_matrix",
               LIB.lead_code_get_check_matrix(self._h, side, out.ctypes.data_as(_c_uint8_p)))
        return out

    def compile(self) -> str:
        """Specialise the min-sum kernel to this code (host only); returns the compiler log."""
        buf = ctypes.create_string_buffer(1 << 16)
        rc = LIB.lead_code_compile(self._h, buf, len(buf))
        if rc != 0:
            raise LeadError("lead_code_compile", rc) from RuntimeError(buf.value.decode(errors="replace"))
        return buf.value.decode(errors="replace")

    def prepare(self, device: int = 0) -> "Code":
        _check("lead_code_prepare", LIB.lead_code_prepare(self._h, device))
        self.info = self._info()
        return self

    def autotune(self, side: int, precision: int = 0, p: float = 0.05, shots: int = 4096) -> str:
        """Time the min-sum kernel of (side, precision) at several register caps on `shots`
        sampled shots at p and keep the fastest (outputs are unchanged); returns the timings."""
        buf = ctypes.create_string_buffer(1 << 12)
        _check("lead_code_autotune", LIB.lead_code_autotune(self._h, side, precision, p, shots, buf, len(buf)))
        return buf.value.decode(errors="replace")

    def enumerators(self, side: int):
        i = self.info
        nl = i.delta ** 2
        S = 1 << i.m_l[side]
        N = np.zeros((S, nl + 1), dtype=np.int32)
        N1 = np.zeros((S, nl, nl + 1), dtype=np.int32)
        ml = np.zeros(S, dtype=np.uint64)
        _check("lead_code_get_enumerators", LIB.lead_code_get_enumerators(
            self._h, side, N.ctypes.data_as(_c_int32_p), N1.ctypes.data_as(_c_int32_p),
            ml.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        return N, N1, ml

    # ---- device calls (torch tensors in, enqueued on the current stream) --------------------

    def sample(self, noise: int, p: float, shots: int, seed: int, shot_offset: int = 0,
               err_x=None, err_z=None, syn_z=None, syn_x=None, stream=None):
        _check("lead_sample", LIB.lead_sample(self._h, noise, p, shots, seed, shot_offset, _ptr(err_x),
                                              _ptr(err_z), _ptr(syn_z), _ptr(syn_x), _stream(stream)))

    def workspace_bytes(self, opts: LeadDecodeOpts, shots: int = 0) -> int:
        return int(LIB.lead_workspace_bytes(self._h, ctypes.byref(opts), shots))

    def local_table(self, side: int, p: float, table, stream=None):
        _check("lead_local_table", LIB.lead_local_table(self._h, side, p, _ptr(table), _stream(stream)))

    def local_table_est(self, side: int, p: float, estimator: int, table, iters=None, stream=None):
        _check("lead_local_table_est", LIB.lead_local_table_est(self._h, side, p, estimator, _ptr(table),
                                                                _ptr(iters), _stream(stream)))

    def local_estimate(self, opts: LeadDecodeOpts, syn, shots: int, llr, workspace, stream=None):
        ws = _ptr(workspace)
        nb = workspace.numel() * workspace.element_size() if workspace is not None else 0
        _check("lead_local_estimate", LIB.lead_local_estimate(self._h, ctypes.byref(opts), _ptr(syn), shots,
                                                              _ptr(llr), ws, nb, _stream(stream)))

    def decode(self, opts: LeadDecodeOpts, syn, shots: int, corr, status, iters=None, llr=None,
               workspace=None, stream=None):
        ws = _ptr(workspace)
        nb = workspace.numel() * workspace.element_size() if workspace is not None else 0
        _check("lead_decode", LIB.lead_decode(self._h, ctypes.byref(opts), _ptr(syn), shots, _ptr(corr),
                                              _ptr(status), _ptr(iters), _ptr(llr), ws, nb, _stream(stream)))

    def decode_noalloc(self, opts: LeadDecodeOpts, syn, shots: int, corr, status, iters=None, llr=None,
                       stream=None):
        """lead_decode_noalloc: like decode, with the library's fixed device scratch instead of a
        caller workspace (for callers that cannot allocate device memory)."""
        _check("lead_decode_noalloc", LIB.lead_decode_noalloc(self._h, ctypes.byref(opts), _ptr(syn), shots,
                                                              _ptr(corr), _ptr(status), _ptr(iters), _ptr(llr),
                                                              _stream(stream)))

    def priors_workspace_bytes(self, opts: LeadDecodeOpts, shots: int) -> int:
        return int(LIB.lead_priors_workspace_bytes(self._h, ctypes.byref(opts), shots))

    def local_estimate_priors(self, opts: LeadDecodeOpts, syn, shots: int, prior, llr, q=None, ml=None,
                              workspace=None, stream=None):
        """lead_local_estimate_priors: Phases 1-2 with one prior probability per shot and qubit."""
        ws = _ptr(workspace)
        nb = workspace.numel() * workspace.element_size() if workspace is not None else 0
        _check("lead_local_estimate_priors", LIB.lead_local_estimate_priors(
            self._h, ctypes.byref(opts), _ptr(syn), shots, _ptr(prior), _ptr(llr), _ptr(q), _ptr(ml), ws, nb,
            _stream(stream)))

    def decode_priors(self, opts: LeadDecodeOpts, syn, shots: int, prior, corr, status, iters=None, llr=None,
                      workspace=None, stream=None):
        """lead_decode_priors: Algorithm 1 with one prior probability per shot and qubit."""
        ws = _ptr(workspace)
        nb = workspace.numel() * workspace.element_size() if workspace is not None else 0
        _check("lead_decode_priors", LIB.lead_decode_priors(
            self._h, ctypes.byref(opts), _ptr(syn), shots, _ptr(prior), _ptr(corr), _ptr(status), _ptr(iters),
            _ptr(llr), ws, nb, _stream(stream)))

    def iterated_workspace_bytes(self, opts: LeadDecodeOpts, shots: int) -> int:
        return int(LIB.lead_iterated_workspace_bytes(self._h, ctypes.byref(opts), shots))

    def decode_iterated(self, opts: LeadDecodeOpts, rounds: int, syn, shots: int, corr, status, iters=None,
                        llr=None, workspace=None, stream=None):
        """lead_decode_iterated: Algorithm 1, then up to rounds - 1 more rounds on the unconverged
        shots with the last posterior as per-qubit prior (an extension of the paper)."""
        ws = _ptr(workspace)
        nb = workspace.numel() * workspace.element_size() if workspace is not None else 0
        _check("lead_decode_iterated", LIB.lead_decode_iterated(
            self._h, ctypes.byref(opts), rounds, _ptr(syn), shots, _ptr(corr), _ptr(status), _ptr(iters),
            _ptr(llr), ws, nb, _stream(stream)))

    def osd_workspace_bytes(self, opts: LeadDecodeOpts, shots: int) -> int:
        return int(LIB.lead_osd_workspace_bytes(self._h, ctypes.byref(opts), shots))

    def osd(self, opts: LeadDecodeOpts, order: int, syn, shots: int, post, status, corr, prior=None,
            workspace=None, stream=None):
        """lead_osd: OSD-CS of the given order on the shots whose min-sum did not converge."""
        ws = _ptr(workspace)
        nb = workspace.numel() * workspace.element_size() if workspace is not None else 0
        _check("lead_osd", LIB.lead_osd(self._h, ctypes.byref(opts), order, _ptr(syn), shots, _ptr(prior), _ptr(post),
                                        _ptr(status), _ptr(corr), ws, nb, _stream(stream)))

    def check_record(self):
        """The last failed bounds check of a checked build: (failures, site, index, bound)."""
        rec = (ctypes.c_uint64 * 4)()
        _check("lead_code_check_record", LIB.lead_code_check_record(self._h, rec))
        return tuple(int(x) for x in rec)

    def device_errors(self, clear: bool = False) -> int:
        """Device error flags of the code's kernels (lead_code_device_errors; waits for the device)."""
        f = ctypes.c_uint32()
        _check("lead_code_device_errors", LIB.lead_code_device_errors(self._h, ctypes.byref(f), 1 if clear else 0))
        return int(f.value)

    def check(self, side: int, err, corr, shots: int, fail, stream=None):
        _check("lead_check", LIB.lead_check(self._h, side, _ptr(err), _ptr(corr), shots, _ptr(fail),
                                            _stream(stream)))


def opts(side: int = 0, p: float = 0.05, alpha: float = 1.0, max_iter: int = 32, use_lead: bool = True,
         precision: int = PREC_FP32, estimator: int = EST_EXACT) -> LeadDecodeOpts:
    return LeadDecodeOpts(side=side, use_lead=1 if use_lead else 0, max_iter=max_iter, precision=precision,
                          alpha=alpha, p=p, estimator=estimator)


class Server:
    """Continuous-batching decode server (lead_server_*): submit single-shot requests with arrival
    times, poll results. Codes must be prepared on the same device."""

    def __init__(self, codes, p_side, sides_mask: int = 3, max_batch: int = 256, streams: int = 4,
                 budget_bytes: int = 1 << 30, max_iter: int = 32, alpha: float = 1.0, precision: int = 0):
        self.codes = list(codes)
        self._handles = (ctypes.c_void_p * len(self.codes))(*[c._h.value for c in self.codes])
        self._p = (ctypes.c_double * len(self.codes))(*p_side)
        cfg = LeadServerConfig(ncodes=len(self.codes), codes=self._handles, p_side=self._p, sides_mask=sides_mask,
                               max_batch=max_batch, streams=streams, budget_bytes=budget_bytes, max_iter=max_iter,
                               alpha=alpha, precision=precision)
        out = ctypes.c_void_p()
        _check("lead_server_create", LIB.lead_server_create(ctypes.byref(cfg), ctypes.byref(out)))
        self._h = out
        self.W = max(c.info.words_n for c in self.codes)

    def close(self):
        if getattr(self, "_h", None):
            LIB.lead_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def clock_ns(self) -> int:
        t = ctypes.c_int64()
        _check("lead_server_clock_ns", LIB.lead_server_clock_ns(self._h, ctypes.byref(t)))
        return t.value

    def submit(self, code: int, syn: np.ndarray, ids: np.ndarray, arrival_ns: np.ndarray | None = None):
        """syn: (n, words_m[0] + words_m[1]) uint32 host rows (side 0 then side 1)."""
        syn = np.ascontiguousarray(syn, dtype=np.uint32)
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        arr = None if arrival_ns is None else np.ascontiguousarray(arrival_ns, dtype=np.int64)
        _check("lead_server_submit", LIB.lead_server_submit(self._h, code, len(ids), syn.ctypes.data, ids.ctypes.data,
                                                            None if arr is None else arr.ctypes.data))

    def poll(self, max_results: int = 65536):
        """Returns (results structured array, corrections (k, 2, W) uint32)."""
        out = (LeadServerResult * max_results)()
        corr = np.zeros((max_results, 2, self.W), dtype=np.uint32)
        got = ctypes.c_int64()
        _check("lead_server_poll", LIB.lead_server_poll(self._h, out, corr.ctypes.data, max_results, ctypes.byref(got)))
        k = got.value
        res = np.zeros(k, dtype=[("id", np.uint64), ("code", np.int32), ("status", np.uint8, 2),
                                 ("arrival_ns", np.int64), ("done_ns", np.int64)])
        for i in range(k):
            r = out[i]
            res[i] = (r.id, r.code, tuple(r.status), r.arrival_ns, r.done_ns)
        return res, corr[:k]

    def pending(self) -> int:
        p = ctypes.c_int64()
        _check("lead_server_pending", LIB.lead_server_pending(self._h, ctypes.byref(p)))
        return p.value
