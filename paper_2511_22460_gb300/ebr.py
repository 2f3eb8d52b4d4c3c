"""Thin ctypes binding of ``libebr.so`` (C ABI in ``include/ebr.h``).

Argument marshalling only: every step of the retrieval path runs in the CUDA
library.  Arrays are passed as torch CUDA tensors (device pointers) or numpy
arrays / pinned torch CPU tensors (host pointers), exactly as the C function
documents.  Importing this module fails if the library is missing: there is
no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libebr.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libebr.so is not built: run __graft_entry__.build() "
                      "(or python -m paper_2511_22460_gb300._build)")
_lib = C.CDLL(LIB_PATH)

EBR_OK, EBR_EINVAL, EBR_ENOMEM, EBR_ECUDA, EBR_EAGAIN, EBR_ETIMEDOUT, EBR_EDATA = \
    0, -1, -2, -3, -4, -5, -6
F32, BF16, FP8E4M3 = 0, 1, 2
W_DENSE, W_HASHED = 0, 1
IO_DEVICE, IO_HOST = 0, 1
QF_KEY_MAJOR = 1
QF_WINDOW_MAJOR = 2
_DTYPES = {"f32": F32, "bf16": BF16, "fp8e4m3": FP8E4M3}

vp, u32, u64, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int


class IndexDesc(C.Structure):
    _fields_ = [("n_ads", u32), ("n_keys", u32), ("nnz", u64), ("post_key", vp),
                ("post_ad", vp), ("d", u32), ("emb_dtype", i32), ("emb_f32", vp),
                ("rescore_mult", u32), ("device", i32), ("stream", vp)]


class IndexInfo(C.Structure):
    _fields_ = [("n_ads", u32), ("n_keys", u32), ("d", u32), ("emb_dtype", i32),
                ("rescore_mult", u32), ("nnz_unique", u64), ("n_blocks", u64 * 9),
                ("index_bytes", u64), ("emb_bytes", u64), ("build_ms", C.c_float),
                ("window_view_ms", C.c_float), ("window_view_bytes", u64),
                ("n_windows", u32), ("max_keys_per_ad", u32), ("max_window_slots", u32),
                ("max_window_chunks", u32)]


class CrossDesc(C.Structure):
    _fields_ = [("f_u", u32), ("f_a", u32), ("vocab_u", vp), ("vocab_a", vp),
                ("n_pairs", u32), ("pairs", vp), ("kind", i32), ("w_table", vp),
                ("w_len", u64), ("w_off", vp), ("hash_bits", u32), ("device", i32),
                ("stream", vp)]


class QueryC(C.Structure):
    _fields_ = [("h_u", vp), ("user_vals", vp), ("n_q", u32), ("q_key", vp), ("q_w", vp),
                ("filter", vp), ("k", u32), ("flags", u32), ("user_ptr", vp),
                ("n_user_vals", u32)]


class ServerCfg(C.Structure):
    _fields_ = [("hbm_budget", u64), ("max_batch", u32), ("max_slots", u32), ("k_max", u32),
                ("queue_timeout_ms", u32), ("max_user_vals", u32), ("host_driven", u32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", u64), ("admitted", u64), ("rejected", u64), ("completed", u64),
                ("failed", u64), ("batches", u64), ("batched_requests", u64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("max_batch", u32), ("max_slots", u32), ("device_bytes", u64),
                ("slot_bytes", u64), ("launch_ms", C.c_double), ("finish_ms", C.c_double),
                ("index_swaps", u64), ("loop_launches", u64)]


class Profile(C.Structure):
    _fields_ = [("calls", u64), ("launches", u64), ("lib_launches", u64),
                ("ms_expand", C.c_double), ("ms_wide", C.c_double), ("ms_scan", C.c_double),
                ("ms_final", C.c_double), ("batched", u64), ("recomputed", u64),
                ("batch_calls", u64), ("ms_batch_stage", C.c_double),
                ("ms_batch_scan", C.c_double), ("ms_batch_merge", C.c_double),
                ("auto_routed", u64), ("window_routed", u64)]


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


ebr_last_error = _sig("ebr_last_error", C.c_char_p, [])
ebr_version = _sig("ebr_version", i32, [])
ebr_build_index = _sig("ebr_build_index", i32, [C.POINTER(IndexDesc), C.POINTER(vp)])
ebr_index_free = _sig("ebr_index_free", None, [vp])
ebr_index_get_info = _sig("ebr_index_get_info", i32, [vp, C.POINTER(IndexInfo)])
ebr_index_export = _sig("ebr_index_export", i32, [vp, u32, vp, vp, vp])
ebr_index_export_emb = _sig("ebr_index_export_emb", i32, [vp, vp, vp])
ebr_cross_create = _sig("ebr_cross_create", i32, [C.POINTER(CrossDesc), C.POINTER(vp)])
ebr_cross_free = _sig("ebr_cross_free", None, [vp])
ebr_cross_n_keys = _sig("ebr_cross_n_keys", u32, [vp])
ebr_expand_query = _sig("ebr_expand_query", i32, [vp, vp, u32, vp, vp])
ebr_expand_query_seq = _sig("ebr_expand_query_seq", i32, [vp, vp, vp, u32, vp, vp])
ebr_score_topk = _sig("ebr_score_topk", i32, [vp, vp, C.POINTER(QueryC), u32, vp, vp, i32, vp])
ebr_score_all = _sig("ebr_score_all", i32, [vp, vp, C.POINTER(QueryC), vp, vp])
ebr_wide_scores = _sig("ebr_wide_scores", i32, [vp, vp, C.POINTER(QueryC), vp, vp])
ebr_quantize = _sig("ebr_quantize", i32, [vp, u64, i32, vp, vp])
ebr_scan_topk_noalloc = _sig("ebr_scan_topk_noalloc", i32,
                             [vp, u32, u32, vp, vp, vp, u32, vp, vp, i32, vp])
ebr_debug_gemm_bf16 = _sig("ebr_debug_gemm_bf16", i32, [vp, u32, vp, u32, u32, vp, vp])
ebr_debug_gemm_e4m3 = _sig("ebr_debug_gemm_e4m3", i32, [vp, u32, vp, u32, u32, vp, vp])
ebr_debug_wait_timeout = _sig("ebr_debug_wait_timeout", i32, [u32, vp])
ebr_profile_enable = _sig("ebr_profile_enable", i32, [vp, i32])
ebr_profile_read = _sig("ebr_profile_read", i32, [vp, C.POINTER(Profile)])
ebr_server_create = _sig("ebr_server_create", i32, [vp, vp, vp, C.POINTER(vp)])
ebr_submit = _sig("ebr_submit", i32, [vp, C.POINTER(QueryC), C.POINTER(u64)])
ebr_poll = _sig("ebr_poll", i32, [vp, u64, vp, vp])
ebr_server_get_stats = _sig("ebr_server_get_stats", i32, [vp, vp])
ebr_server_destroy = _sig("ebr_server_destroy", i32, [vp])
ebr_server_swap_index = _sig("ebr_server_swap_index", i32, [vp, vp])
ebr_server_reset_stats = _sig("ebr_server_reset_stats", i32, [vp])
ebr_server_completed = _sig("ebr_server_completed", i32, [vp, vp, u32, C.POINTER(u32)])


class EbrError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = ebr_last_error().decode(errors="replace")
        super().__init__("%s failed (%d): %s" % (where, code, msg))


def _check(rc, where):
    if rc != EBR_OK:
        raise EbrError(rc, where)


def ptr(x):
    """Raw address of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous, "array must be contiguous"
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "tensor must be contiguous"
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(type(x))


def stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Index:
    """Owning handle of an ``ebr_index``."""

    def __init__(self, handle):
        self.h = handle

    def close(self):
        if self.h:
            ebr_index_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> IndexInfo:
        out = IndexInfo()
        _check(ebr_index_get_info(self.h, C.byref(out)), "ebr_index_get_info")
        return out

    def export(self, g: int):
        inf = self.info()
        nb = int(inf.n_blocks[g])
        keys = np.empty(inf.n_keys + 1, np.uint32)
        hdr = np.empty(max(nb, 1), np.uint32)
        vals = np.empty(max(nb << g, 1), np.uint8)
        _check(ebr_index_export(self.h, g, ptr(keys), ptr(hdr), ptr(vals)), "ebr_index_export")
        return keys, hdr[:nb], vals[:nb << g]

    def profile_enable(self, on=True):
        _check(ebr_profile_enable(self.h, 1 if on else 0), "ebr_profile_enable")

    def profile_read(self) -> Profile:
        out = Profile()
        _check(ebr_profile_read(self.h, C.byref(out)), "ebr_profile_read")
        return out

    def export_emb(self):
        inf = self.info()
        n = inf.n_ads * inf.d
        dt = {F32: np.float32, BF16: np.uint16, FP8E4M3: np.uint8}[inf.emb_dtype]
        codes = np.empty(n, dt)
        scale = np.empty(inf.n_ads, np.float32) if inf.emb_dtype == FP8E4M3 else None
        _check(ebr_index_export_emb(self.h, ptr(codes), ptr(scale)), "ebr_index_export_emb")
        return codes.reshape(inf.n_ads, inf.d), scale


def build_index(n_ads, n_keys, post_key, post_ad, emb, dtype="f32", rescore_mult=0, device=0,
                stream=None) -> Index:
    emb_dtype = _DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    d = IndexDesc(n_ads, n_keys, int(post_key.numel() if hasattr(post_key, "numel") else
                                      post_key.size),
                  ptr(post_key), ptr(post_ad), int(emb.shape[1]), emb_dtype, ptr(emb),
                  rescore_mult, device, stream_ptr(stream))
    h = vp()
    _check(ebr_build_index(C.byref(d), C.byref(h)), "ebr_build_index")
    return Index(h)


class Cross:
    """Owning handle of an ``ebr_cross`` (cross pairs + weight table on device)."""

    def __init__(self, handle, f_u, n_keys):
        self.h = handle
        self.f_u = f_u
        self.n_keys = n_keys

    def close(self):
        if self.h:
            ebr_cross_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cross_create(vocab_u, vocab_a, pairs, w_table, w_off=None, hashed=True, hash_bits=24,
                 device=0, stream=None) -> Cross:
    vocab_u = np.ascontiguousarray(vocab_u, np.uint32)
    vocab_a = np.ascontiguousarray(vocab_a, np.uint32)
    pairs = np.ascontiguousarray(np.asarray(pairs).reshape(-1, 2), np.uint32)
    if isinstance(w_table, np.ndarray):
        w_table = np.ascontiguousarray(w_table, np.float32)
        w_len = w_table.size
    else:
        w_len = w_table.numel()
    w_off_a = None if w_off is None else np.ascontiguousarray(w_off, np.uint64)
    d = CrossDesc(len(vocab_u), len(vocab_a), ptr(vocab_u), ptr(vocab_a), len(pairs),
                  ptr(pairs), W_HASHED if hashed else W_DENSE, ptr(w_table), w_len,
                  ptr(w_off_a), hash_bits, device, stream_ptr(stream))
    h = vp()
    _check(ebr_cross_create(C.byref(d), C.byref(h)), "ebr_cross_create")
    return Cross(h, len(vocab_u), int(np.sum(vocab_a.astype(np.uint64))))


def cross_from_workload(w, device=0) -> Cross:
    return cross_create(w.vocab_u, w.vocab_a, w.pairs, w.w_table, w.w_off,
                        hashed=(w.recipe.weights == "hashed"), device=device)


def expand_query(cross: Cross, user_vals, w_hat, stream=None):
    batch = int(user_vals.shape[0]) if user_vals.dim() == 2 else 1
    _check(ebr_expand_query(cross.h, ptr(user_vals), batch, ptr(w_hat), stream_ptr(stream)),
           "ebr_expand_query")


def expand_query_seq(cross: Cross, user_ptr, user_vals, w_hat, stream=None):
    """One user's expansion with multi-valued fields (device arrays)."""
    n = int(user_vals.numel())
    _check(ebr_expand_query_seq(cross.h, ptr(user_ptr), ptr(user_vals), n, ptr(w_hat),
                                stream_ptr(stream)), "ebr_expand_query_seq")


def _numel(x) -> int:
    return int(x.numel() if hasattr(x, "numel") else x.size)


@dataclass
class Query:
    h_u: object
    k: int
    user_vals: object = None
    q_key: object = None
    q_w: object = None
    n_q: int = 0
    filter: object = None
    flags: int = 0
    user_ptr: object = None  # multi-valued user fields: offsets [f_u + 1] into user_vals

    def c(self) -> QueryC:
        n_q = self.n_q
        if self.q_key is not None and not n_q:
            n_q = _numel(self.q_key)
        n_uv = _numel(self.user_vals) if self.user_ptr is not None else 0
        return QueryC(ptr(self.h_u), ptr(self.user_vals), n_q, ptr(self.q_key), ptr(self.q_w),
                      ptr(self.filter), int(self.k), int(self.flags), ptr(self.user_ptr), n_uv)


def _queries(qs: Sequence[Query]):
    arr = (QueryC * len(qs))()
    for i, q in enumerate(qs):
        arr[i] = q.c()
    return arr


def score_topk(index: Index, cross: Optional[Cross], queries: Sequence[Query], out_ids, out_scores,
               io=IO_DEVICE, stream=None):
    arr = _queries(queries)
    _check(ebr_score_topk(index.h, cross.h if cross else None, arr, len(queries), ptr(out_ids),
                          ptr(out_scores), io, stream_ptr(stream)), "ebr_score_topk")


def score_all(index: Index, cross: Optional[Cross], query: Query, out_scores, stream=None):
    arr = _queries([query])
    _check(ebr_score_all(index.h, cross.h if cross else None, arr, ptr(out_scores),
                         stream_ptr(stream)), "ebr_score_all")


def wide_scores(index: Index, cross: Optional[Cross], query: Query, out_wide, stream=None):
    arr = _queries([query])
    _check(ebr_wide_scores(index.h, cross.h if cross else None, arr, ptr(out_wide),
                           stream_ptr(stream)), "ebr_wide_scores")


def quantize(x, dtype, out, stream=None):
    dt = _DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    _check(ebr_quantize(ptr(x), int(x.numel()), dt, ptr(out), stream_ptr(stream)), "ebr_quantize")


NOALLOC_DIMS = (4, 8, 16, 32, 64, 128)
NOALLOC_MAX_K = 1024


def scan_topk_noalloc(emb, h_u, wide, filt, k, out_ids, out_scores, stream=None):
    """Allocation-free scan + top-K over caller-owned device buffers.

    Every tensor must be a contiguous CUDA tensor on emb's device: emb
    float32 [n_ads][d] with d in NOALLOC_DIMS, h_u float32 [d], wide float32
    [n_ads] or None, filt int64/uint64 words [>= ceil(n_ads / 64)] or None,
    out_ids int32/uint32 [>= k], out_scores float32 [>= k]; 1 <= k <= 1024.
    The shapes are checked here, before anything reaches the device, because
    the kernel trusts them (a short buffer would be read or written out of
    bounds rather than rejected)."""
    import torch

    def need(cond, msg):
        if not cond:
            raise ValueError("scan_topk_noalloc: " + msg)

    k = int(k)
    need(isinstance(emb, torch.Tensor) and emb.dim() == 2, "emb must be a 2-D tensor")
    need(emb.dtype == torch.float32, "emb must be float32")
    need(emb.is_contiguous(), "emb must be contiguous")
    n_ads, d = int(emb.shape[0]), int(emb.shape[1])
    need(n_ads > 0 and d in NOALLOC_DIMS, "need n_ads > 0 and d in %s" % (NOALLOC_DIMS,))
    need(1 <= k <= NOALLOC_MAX_K, "k must be in 1..%d" % NOALLOC_MAX_K)

    def vec(t, name, dtypes, min_len):
        need(isinstance(t, torch.Tensor), "%s must be a tensor" % name)
        need(t.dtype in dtypes, "%s must have dtype in %s" % (name, dtypes))
        need(t.is_contiguous(), "%s must be contiguous" % name)
        need(t.numel() >= min_len, "%s needs at least %d elements" % (name, min_len))

    vec(h_u, "h_u", (torch.float32,), d)
    if wide is not None:
        vec(wide, "wide", (torch.float32,), n_ads)
    if filt is not None:
        vec(filt, "filter", (torch.int64, torch.uint64), (n_ads + 63) // 64)
    vec(out_ids, "out_ids", (torch.int32, torch.uint32), k)
    vec(out_scores, "out_scores", (torch.float32,), k)
    need(emb.is_cuda, "emb must be a CUDA tensor")
    device = emb.device.index if emb.device.index is not None else torch.cuda.current_device()
    for name, t in (("h_u", h_u), ("wide", wide), ("filter", filt), ("out_ids", out_ids),
                    ("out_scores", out_scores)):
        need(t is None or (t.is_cuda and t.device.index == device),
             "%s must be on emb's device (cuda:%d)" % (name, device))
    _check(ebr_scan_topk_noalloc(ptr(emb), n_ads, d, ptr(h_u), ptr(wide), ptr(filt), k,
                                 ptr(out_ids), ptr(out_scores), device, stream_ptr(stream)),
           "ebr_scan_topk_noalloc")


def debug_wait_timeout(timeout_us, stream=None):
    """Status of a device wait that nothing ends (EBR_ETIMEDOUT expected)."""
    return ebr_debug_wait_timeout(int(timeout_us), stream_ptr(stream))


def debug_gemm_e4m3(A, U, out, stream=None):
    """out[n][B] = e4m3(A[n][d]) @ e4m3(U[B][d])^T on the tensor cores (FP8 codes in, FP32 out)."""
    _check(ebr_debug_gemm_e4m3(ptr(A), int(A.shape[0]), ptr(U), int(U.shape[0]), int(A.shape[1]),
                               ptr(out), stream_ptr(stream)), "ebr_debug_gemm_e4m3")


def debug_gemm_bf16(A, U, out, stream=None):
    """out[n][B] = A[n][d] @ U[B][d]^T on the tensor cores (BF16 in, FP32 out)."""
    _check(ebr_debug_gemm_bf16(ptr(A), int(A.shape[0]), ptr(U), int(U.shape[0]), int(A.shape[1]),
                               ptr(out), stream_ptr(stream)), "ebr_debug_gemm_bf16")


class Server:
    """Continuous-batching request loop (ebr_server_create / ebr_submit / ebr_poll).

    Requests are host arrays; results come back as host arrays."""

    def __init__(self, index: Index, cross: Cross, hbm_budget=0, max_batch=0, max_slots=0,
                 k_max=0, queue_timeout_ms=0, max_user_vals=0, host_driven=False):
        cfg = ServerCfg(int(hbm_budget), int(max_batch), int(max_slots), int(k_max),
                        int(queue_timeout_ms), int(max_user_vals), int(bool(host_driven)))
        h = vp()
        _check(ebr_server_create(index.h, cross.h, C.byref(cfg), C.byref(h)), "ebr_server_create")
        self.h = h.value
        self._keep = (index, cross)

    def submit(self, h_u, user_vals, k, filter=None, user_ptr=None):
        """Ticket of the admitted request, or None when admission is refused.
        user_ptr (uint32 [f_u + 1]) makes user_vals a history per field."""
        n_uv = 0 if user_ptr is None else int(len(user_vals))
        q = QueryC(ptr(h_u), ptr(user_vals), 0, None, None, ptr(filter), int(k), 0,
                   ptr(user_ptr), n_uv)
        t = u64()
        rc = ebr_submit(self.h, C.byref(q), C.byref(t))
        if rc == EBR_ENOMEM:
            return None
        _check(rc, "ebr_submit")
        return t.value

    def poll(self, ticket, k):
        """(ids, scores) once done, None while pending; raises on a failed request."""
        ids = np.empty(k, np.uint32)
        sc = np.empty(k, np.float32)
        rc = ebr_poll(self.h, int(ticket), ids.ctypes.data, sc.ctypes.data)
        if rc == EBR_EAGAIN:
            return None
        _check(rc, "ebr_poll")
        return ids, sc

    def wait(self, ticket, k, timeout_s=60.0):
        import time
        t0 = time.monotonic()
        while True:
            r = self.poll(ticket, k)
            if r is not None:
                return r
            if time.monotonic() - t0 > timeout_s:
                raise TimeoutError("request %d not done after %.0f s" % (ticket, timeout_s))
            time.sleep(0.0002)

    def stats(self) -> ServerStats:
        st = ServerStats()
        _check(ebr_server_get_stats(self.h, C.byref(st)), "ebr_server_get_stats")
        return st

    def reset_stats(self):
        _check(ebr_server_reset_stats(self.h), "ebr_server_reset_stats")

    def swap_index(self, index: Index) -> Index:
        """Serve requests not yet launched from `index`; returns the index it
        replaced, which the server no longer uses (ebr_server_swap_index)."""
        _check(ebr_server_swap_index(self.h, index.h), "ebr_server_swap_index")
        old = self._keep[0]
        self._keep = (index, self._keep[1])
        return old

    def completed(self, cap=4096):
        """Tickets finished since the previous call (done or failed)."""
        buf = np.empty(cap, np.uint64)
        n = u32()
        _check(ebr_server_completed(self.h, buf.ctypes.data, cap, C.byref(n)),
               "ebr_server_completed")
        return buf[:n.value]

    def close(self):
        if self.h:
            ebr_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
