"""CPU FP64 oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use this package.  It wraps ``ebr_oracle.c`` (plain C, compiled with gcc,
no fast-math, no FMA contraction) through ctypes and shares no code with the
CUDA library.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(brute force on tiny inputs, a hand-worked example, closed-form layout rules,
invariants, library special cases, published test vectors); none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ebr_oracle.c")
_LIB = os.path.join(_HERE, "_ebr_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, -O2, IEEE semantics)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Cross(C.Structure):
    _fields_ = [("f_u", C.c_uint32), ("f_a", C.c_uint32),
                ("vocab_u", C.c_void_p), ("vocab_a", C.c_void_p),
                ("n_pairs", C.c_uint32), ("pairs", C.c_void_p),
                ("hashed", C.c_int), ("w_table", C.c_void_p), ("w_off", C.c_void_p),
                ("hash_bits", C.c_uint32)]


class _Index(C.Structure):
    _fields_ = [("n_keys", C.c_uint32), ("n_blocks", C.c_uint64 * 9),
                ("keys", C.c_void_p * 9), ("header", C.c_void_p * 9),
                ("values", C.c_void_p * 9)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            vp, u32, u64, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
            lib.orc_splitmix64.restype = u64
            lib.orc_splitmix64.argtypes = [u64]
            lib.orc_scores_brute.restype = i32
            lib.orc_scores_brute.argtypes = [u32, u32, vp, vp, vp, vp, vp, vp, vp]
            lib.orc_expand.restype = i32
            lib.orc_expand.argtypes = [vp, vp, vp, vp]
            lib.orc_scores_brute_seq.restype = i32
            lib.orc_scores_brute_seq.argtypes = [u32, u32, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.orc_expand_seq.restype = i32
            lib.orc_expand_seq.argtypes = [vp, vp, vp, vp, vp]
            lib.orc_scores_postings.restype = i32
            lib.orc_scores_postings.argtypes = [u32, u32, vp, vp, u32, u64, vp, vp, u32, vp,
                                                vp, vp]
            lib.orc_unique_pairs.restype = C.c_int64
            lib.orc_unique_pairs.argtypes = [u64, vp, vp, vp, vp]
            lib.orc_build_index.restype = i32
            lib.orc_build_index.argtypes = [u32, u32, u64, vp, vp, vp]
            lib.orc_free_index.restype = None
            lib.orc_free_index.argtypes = [vp]
            lib.orc_decode_index.restype = C.c_int64
            lib.orc_decode_index.argtypes = [vp, vp, vp, u32, vp, vp, u64]
            lib.orc_topk.restype = C.c_int64
            lib.orc_topk.argtypes = [u32, vp, vp, u32, vp, vp]
            lib.orc_bf16_rne.restype = C.c_uint16
            lib.orc_bf16_rne.argtypes = [C.c_float]
            lib.orc_bf16_value.restype = C.c_float
            lib.orc_bf16_value.argtypes = [C.c_uint16]
            lib.orc_fp8_e4m3_value.restype = C.c_double
            lib.orc_fp8_e4m3_value.argtypes = [C.c_uint8]
            lib.orc_fp8_e4m3_rne_sat.restype = C.c_uint8
            lib.orc_fp8_e4m3_rne_sat.argtypes = [C.c_float]
            lib.orc_quantize_fp8_rows.restype = None
            lib.orc_quantize_fp8_rows.argtypes = [u64, u32, vp, vp, vp]
            lib.orc_quantize_bf16.restype = None
            lib.orc_quantize_bf16.argtypes = [u64, vp, vp]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Cross:
    """Cross-feature model: user/ad vocabularies, cross pairs, weight table."""

    def __init__(self, vocab_u, vocab_a, pairs, w_table, w_off=None, hashed=True,
                 hash_bits=24):
        self.vocab_u = _c(vocab_u, np.uint32)
        self.vocab_a = _c(vocab_a, np.uint32)
        self.pairs = _c(np.asarray(pairs).reshape(-1, 2), np.uint32)
        self.w_table = _c(w_table, np.float32)
        self.w_off = _c(w_off if w_off is not None else np.zeros(len(self.pairs)), np.uint64)
        self.hashed = bool(hashed)
        self.hash_bits = int(hash_bits)
        self.key_off = np.zeros(len(self.vocab_a) + 1, dtype=np.uint32)
        self.key_off[1:] = np.cumsum(self.vocab_a.astype(np.uint64)).astype(np.uint32)
        self._s = _Cross(len(self.vocab_u), len(self.vocab_a), _p(self.vocab_u),
                         _p(self.vocab_a), len(self.pairs), _p(self.pairs), int(self.hashed),
                         _p(self.w_table), _p(self.w_off), self.hash_bits)

    @classmethod
    def from_workload(cls, w):
        return cls(w.vocab_u, w.vocab_a, w.pairs, w.w_table, w.w_off,
                   hashed=(w.recipe.weights == "hashed"))

    @property
    def n_keys(self):
        return int(self.key_off[-1])


def splitmix64(x: int) -> int:
    return int(_load().orc_splitmix64(C.c_uint64(x)))


def scores_brute(cross: Cross, h_u, emb, ad_vals, user, with_cond=False):
    """O1: FP64 scores of every ad from raw per-ad values (and condition scale)."""
    lib = _load()
    emb = _c(emb, np.float32)
    n, d = emb.shape
    h_u = _c(h_u, np.float32)
    ad_vals = _c(ad_vals, np.uint32)
    user = _c(user, np.uint32)
    assert ad_vals.shape == (n, len(cross.vocab_a)) and h_u.shape == (d,)
    out = np.empty(n, dtype=np.float64)
    cond = np.empty(n, dtype=np.float64) if with_cond else None
    rc = lib.orc_scores_brute(n, d, _p(h_u), _p(emb), C.addressof(cross._s), _p(ad_vals),
                              _p(user), _p(out), _p(cond))
    if rc != 0:
        raise ValueError("orc_scores_brute failed: %d" % rc)
    return (out, cond) if with_cond else out


def expand(cross: Cross, user):
    """Query expansion: dense FP64 w_hat over the ad-field key space."""
    lib = _load()
    user = _c(user, np.uint32)
    out = np.empty(cross.n_keys, dtype=np.float64)
    rc = lib.orc_expand(C.addressof(cross._s), _p(cross.key_off), _p(user), _p(out))
    if rc != 0:
        raise ValueError("orc_expand failed: %d" % rc)
    return out


EMPTY = 0xFFFFFFFF  # an ad field without a value


def _seq(cross: Cross, user_ptr, user_vals):
    user_ptr = _c(user_ptr, np.uint32)
    user_vals = _c(user_vals, np.uint32)
    assert user_ptr.shape == (len(cross.vocab_u) + 1,)
    if user_vals.size == 0:
        user_vals = np.zeros(1, np.uint32)
    return user_ptr, user_vals


def scores_brute_seq(cross: Cross, h_u, emb, ad_vals, user_ptr, user_vals, with_cond=False):
    """O1 for multi-valued user fields: field i holds user_vals[user_ptr[i]:user_ptr[i+1]]."""
    lib = _load()
    emb = _c(emb, np.float32)
    n, d = emb.shape
    h_u = _c(h_u, np.float32)
    ad_vals = _c(ad_vals, np.uint32)
    user_ptr, user_vals = _seq(cross, user_ptr, user_vals)
    assert ad_vals.shape == (n, len(cross.vocab_a)) and h_u.shape == (d,)
    out = np.empty(n, dtype=np.float64)
    cond = np.empty(n, dtype=np.float64) if with_cond else None
    rc = lib.orc_scores_brute_seq(n, d, _p(h_u), _p(emb), C.addressof(cross._s), _p(ad_vals),
                                  _p(user_ptr), _p(user_vals), _p(out), _p(cond))
    if rc != 0:
        raise ValueError("orc_scores_brute_seq failed: %d" % rc)
    return (out, cond) if with_cond else out


def expand_seq(cross: Cross, user_ptr, user_vals):
    """Query expansion for multi-valued user fields: dense FP64 w_hat."""
    lib = _load()
    user_ptr, user_vals = _seq(cross, user_ptr, user_vals)
    out = np.empty(cross.n_keys, dtype=np.float64)
    rc = lib.orc_expand_seq(C.addressof(cross._s), _p(cross.key_off), _p(user_ptr),
                            _p(user_vals), _p(out))
    if rc != 0:
        raise ValueError("orc_expand_seq failed: %d" % rc)
    return out


def unique_pairs(post_key, post_ad):
    """Distinct (key, ad) pairs: L is a 0/1 matrix, a repeated pair is one non-zero."""
    lib = _load()
    post_key, post_ad = _c(post_key, np.uint32), _c(post_ad, np.uint32)
    ok = np.empty(max(post_key.size, 1), np.uint32)
    oa = np.empty(max(post_key.size, 1), np.uint32)
    m = lib.orc_unique_pairs(post_key.size, _p(post_key), _p(post_ad), _p(ok), _p(oa))
    if m < 0:
        raise MemoryError
    return ok[:m].copy(), oa[:m].copy()


def scores_postings(h_u, emb, n_keys, post_key, post_ad, q_key, q_w, assume_unique=False):
    """O2: FP64 scores from uncompressed postings and the query's (key, w_hat) list.

    Repeated (key, ad) pairs are collapsed first unless the caller guarantees
    there are none (workload postings are distinct by construction)."""
    lib = _load()
    emb = _c(emb, np.float32)
    n, d = emb.shape
    h_u = _c(h_u, np.float32)
    post_key, post_ad = _c(post_key, np.uint32), _c(post_ad, np.uint32)
    if not assume_unique:
        post_key, post_ad = unique_pairs(post_key, post_ad)
    q_key, q_w = _c(q_key, np.uint32), _c(q_w, np.float64)
    out = np.empty(n, dtype=np.float64)
    rc = lib.orc_scores_postings(n, d, _p(h_u), _p(emb), n_keys, post_key.size, _p(post_key),
                                 _p(post_ad), q_key.size, _p(q_key), _p(q_w), _p(out))
    if rc != 0:
        raise ValueError("orc_scores_postings failed: %d" % rc)
    return out


def build_index(n_keys, n_ads, post_key, post_ad):
    """O3: Algorithm 1.  Returns dict with per-group lists keys/header/values."""
    lib = _load()
    post_key, post_ad = _c(post_key, np.uint32), _c(post_ad, np.uint32)
    ix = _Index()
    rc = lib.orc_build_index(n_keys, n_ads, post_key.size, _p(post_key), _p(post_ad),
                             C.addressof(ix))
    if rc != 0:
        lib.orc_free_index(C.addressof(ix))
        raise ValueError("orc_build_index failed: %d" % rc)
    out = {"keys": [], "header": [], "values": [], "n_keys": n_keys}
    for g in range(9):
        nb = int(ix.n_blocks[g])
        out["keys"].append(np.ctypeslib.as_array(C.cast(ix.keys[g], C.POINTER(C.c_uint32)),
                                                 (n_keys + 1,)).copy())
        hdr = np.ctypeslib.as_array(C.cast(ix.header[g], C.POINTER(C.c_uint32)), (max(nb, 1),))
        out["header"].append(hdr[:nb].copy())
        vals = np.ctypeslib.as_array(C.cast(ix.values[g], C.POINTER(C.c_uint8)),
                                     (max(nb << g, 1),))
        out["values"].append(vals[:nb << g].copy())
    lib.orc_free_index(C.addressof(ix))
    return out


def decode_index(index):
    """Decode an index (dict of per-group arrays) back to (key, ad) pairs."""
    lib = _load()
    n_keys = int(index["n_keys"])
    keys = [_c(a, np.uint32) for a in index["keys"]]
    hdr = [_c(a, np.uint32) if a.size else np.zeros(1, np.uint32) for a in index["header"]]
    vals = [_c(a, np.uint8) if a.size else np.zeros(1, np.uint8) for a in index["values"]]
    kp = (C.c_void_p * 9)(*[_p(a) for a in keys])
    hp = (C.c_void_p * 9)(*[_p(a) for a in hdr])
    vp = (C.c_void_p * 9)(*[_p(a) for a in vals])
    cap = sum(int(v.size) for v in index["values"])
    ok = np.empty(max(cap, 1), np.uint32)
    oa = np.empty(max(cap, 1), np.uint32)
    n = lib.orc_decode_index(kp, hp, vp, n_keys, _p(ok), _p(oa), cap)
    if n < 0:
        raise ValueError("decode failed")
    return ok[:n].copy(), oa[:n].copy()


def topk(scores, k, filt=None):
    """O4: top-K (ids, scores) by score descending then id ascending."""
    lib = _load()
    scores = _c(scores, np.float64)
    ids = np.empty(max(k, 1), np.uint32)
    vals = np.empty(max(k, 1), np.float64)
    f = None if filt is None else _c(filt, np.uint64)
    r = lib.orc_topk(scores.size, _p(scores), _p(f), k, _p(ids), _p(vals))
    if r < 0:
        raise MemoryError
    return ids[:r].copy(), vals[:r].copy()


def bf16_rne(x):
    lib = _load()
    x = _c(x, np.float32)
    out = np.empty(x.shape, np.uint16)
    lib.orc_quantize_bf16(x.size, _p(x), _p(out))
    return out


def bf16_value(h):
    h = _c(h, np.uint16)
    return (h.astype(np.uint32) << 16).view(np.float32)


def fp8_e4m3_value(c):
    lib = _load()
    return np.array([lib.orc_fp8_e4m3_value(int(v)) for v in np.asarray(c).reshape(-1)],
                    dtype=np.float64).reshape(np.shape(c))


def fp8_e4m3_rne_sat(x):
    lib = _load()
    return np.array([lib.orc_fp8_e4m3_rne_sat(float(v)) for v in np.asarray(x).reshape(-1)],
                    dtype=np.uint8).reshape(np.shape(x))


def quantize_fp8_rows(x):
    """Per-row FP8-e4m3 quantisation: returns (codes uint8 [n,d], scale float32 [n])."""
    lib = _load()
    x = _c(x, np.float32)
    n, d = x.shape
    q = np.empty((n, d), np.uint8)
    s = np.empty(n, np.float32)
    lib.orc_quantize_fp8_rows(n, d, _p(x), _p(q), _p(s))
    return q, s


def score_query(w, b: int, cross: Cross = None, postings=None):
    """Full FP64 scores of request ``b`` of a workload via O2 (expansion + postings)."""
    cross = cross or Cross.from_workload(w)
    wh = expand(cross, w.users[b])
    keys = np.nonzero(wh)[0].astype(np.uint32)
    pk, pa = postings if postings is not None else w.postings()
    # one value per ad field and disjoint key ranges per field: pairs are distinct
    return scores_postings(w.h_u[b], w.emb, w.n_keys, pk, pa, keys, wh[keys], assume_unique=True)


def score_query_seq(w, h_u, user_ptr, user_vals, cross: Cross = None, postings=None):
    """Full FP64 scores of a request with multi-valued user fields via O2."""
    cross = cross or Cross.from_workload(w)
    wh = expand_seq(cross, user_ptr, user_vals)
    keys = np.nonzero(wh)[0].astype(np.uint32)
    pk, pa = postings if postings is not None else w.postings()
    return scores_postings(h_u, w.emb, w.n_keys, pk, pa, keys, wh[keys], assume_unique=True)


def tolerance(scores_ref, cond, rel=1e-5):
    """Per-ad absolute tolerance: rel * max(|s|, condition scale of the sum)."""
    return rel * np.maximum(np.abs(scores_ref), cond)
