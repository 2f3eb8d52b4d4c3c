"""Seeded synthetic inputs for the embedding-based ad retrieval hot path.

This module only draws random inputs: ad embeddings, per-ad field values, user
field values, cross pairs, cross-weight tables, targeting bitmaps and request
arrival times.  It holds none of the scoring arithmetic (no dot products, no
weight hashing, no index construction); the CUDA library and the CPU oracle
both consume the arrays it returns.

Shapes follow the paper's workload description: millions of ads (Sec. 4.4),
64-d tower outputs (Sec. 4.1), and heavy-tailed categorical ad features such as
categories and advertiser ids (Sec. 4.1, "Features").  The paper's own data is
private, so every array here is synthetic.

Random streams: ``numpy.random.PCG64`` seeded from ``SeedSequence(seed)``,
one spawned child stream per array, in the fixed order of ``_STREAMS``.

Distributions:
  * embeddings and user vectors: iid N(0, 1/d) float32 (the second parameter of
    N(.,.) is a variance);
  * vocabularies: fixed, or log-uniform integers in [10, 100000];
  * field values: finite Zipf, P(rank r) proportional to r^-s for r = 1..V,
    drawn by inverse CDF, rank mapped to a value id through a seeded
    permutation per field;
  * cross weights: iid N(0, var) float32, either one dense table per cross pair
    (shape V_user_i x V_ad_j, row-major [u][v]) or one shared table of 2^24
    entries addressed through a hash of (pair, u, v);
  * targeting bitmaps: bit a set iid with probability f, f ~ U[0.01, 1] per
    request, packed little-endian into uint64 words (bit a of word a >> 6).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

HASH_BITS = 24

_STREAMS = (
    "vocab_u", "vocab_a", "perm_u", "perm_a", "ad_vals", "user_vals", "pairs",
    "weights", "emb", "h_u", "filter", "shuffle", "k_choice", "arrivals",
)


@dataclass(frozen=True)
class Recipe:
    """Parameters of one synthetic workload."""
    name: str
    n_ads: int
    d: int
    f_u: int
    f_a: int
    vocab: object            # int (fixed) or "loguniform"
    zipf_ad: float
    zipf_user: float
    n_pairs: Optional[int]   # None = all F_u x F_a pairs
    weights: str             # "dense" | "hashed"
    w_var: float
    k: int
    batch: int = 1
    emb_dtype: str = "f32"   # "f32" | "bf16" | "fp8e4m3"
    rescore_mult: int = 0    # R: rescoring keeps R*K candidates (0 = no rescoring)
    k_choices: tuple = ()    # per-request K drawn uniformly from this set
    filter_frac: Optional[tuple] = None  # (lo, hi) for per-request filter density
    vocab_lo: int = 10
    vocab_hi: int = 100_000


RECIPES = {
    # Plain method, single request, small enough for the FP64 oracle.
    "single_fp32_10k": Recipe("single_fp32_10k", 10_000, 32, 4, 4, 50, 1.1, 1.1, None,
                              "dense", 0.1, 100),
    # Plain FP32 single request at inventory scale.
    "single_fp32_2m": Recipe("single_fp32_2m", 2_000_000, 64, 16, 16, "loguniform", 1.05,
                             1.05, 64, "hashed", 0.05, 500),
    # 256 users against 5M ads, BF16 embeddings, rescoring of the top 4K.
    "batch256_bf16_5m": Recipe("batch256_bf16_5m", 5_000_000, 128, 24, 24, "loguniform",
                               1.05, 1.05, 96, "hashed", 0.05, 1000, batch=256,
                               emb_dtype="bf16", rescore_mult=4),
    # FP8-e4m3 with per-row scale, 10M ads, posting lists Zipf(1.0) over V=15.
    "fp8_10m": Recipe("fp8_10m", 10_000_000, 64, 32, 32, 15, 1.0, 1.0, 128, "hashed",
                      0.05, 2000, batch=1, emb_dtype="fp8e4m3", rescore_mult=4),
    # Serving: 5M BF16 ads, per-request K and targeting bitmap.
    "serve_bf16_5m": Recipe("serve_bf16_5m", 5_000_000, 64, 32, 32, "loguniform", 1.05,
                            1.05, 128, "hashed", 0.05, 1000, batch=64, emb_dtype="bf16",
                            rescore_mult=4, k_choices=(100, 500, 1000),
                            filter_frac=(0.01, 1.0)),
}


# An ad field without a value in ``Workload.ad_vals`` (the ad lacks that
# feature); such a field contributes no (key, ad) pair.
EMPTY_VALUE = 0xFFFFFFFF


@dataclass
class Workload:
    """All synthetic arrays of one workload (host numpy arrays)."""
    recipe: Recipe
    vocab_u: np.ndarray          # uint32 [F_u]
    vocab_a: np.ndarray          # uint32 [F_a]
    key_off: np.ndarray          # uint32 [F_a + 1]: key(j, v) = key_off[j] + v
    ad_vals: np.ndarray          # uint32 [N, F_a]
    pairs: np.ndarray            # uint32 [P, 2]: (user field i, ad field j)
    w_table: np.ndarray          # float32: hashed table [2^24] or concatenated dense tables
    w_off: np.ndarray            # uint64 [P]: start of pair p's dense table (dense only)
    emb: np.ndarray              # float32 [N, d]
    users: np.ndarray            # uint32 [B, F_u]
    h_u: np.ndarray              # float32 [B, d]
    ks: np.ndarray               # uint32 [B]
    filters: Optional[np.ndarray] = None   # uint64 [B, ceil(N/64)] or None
    seed: int = 0
    _rngs: dict = field(default_factory=dict, repr=False)

    @property
    def n_ads(self) -> int:
        return self.recipe.n_ads

    @property
    def n_keys(self) -> int:
        return int(self.key_off[-1])

    @property
    def nnz(self) -> int:
        return int(np.count_nonzero(self.ad_vals != EMPTY_VALUE))

    def postings(self, shuffle: bool = False):
        """Uncompressed feature->ad map L as (key, ad) pairs, ad-major order.

        The pairs are the raw input of index construction: ad ``a`` is in the
        posting list of key(j, v) iff ad field j of ``a`` has value v (an
        EMPTY_VALUE field contributes no pair).
        """
        n, f_a = self.ad_vals.shape
        keys = (self.ad_vals + self.key_off[:f_a][None, :]).astype(np.uint32).reshape(-1)
        ads = np.repeat(np.arange(n, dtype=np.uint32), f_a)
        empty = self.ad_vals.reshape(-1) == EMPTY_VALUE
        if empty.any():
            keys, ads = keys[~empty], ads[~empty]
        if shuffle:
            perm = self._rngs["shuffle"].permutation(keys.size)
            keys, ads = keys[perm], ads[perm]
        return keys, ads


def _zipf_sample(rng, V: int, s: float, size: int, perm: np.ndarray) -> np.ndarray:
    w = np.arange(1, V + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(size)
    r = np.searchsorted(cdf, u, side="right")
    np.minimum(r, V - 1, out=r)
    return perm[r].astype(np.uint32)


def _vocab(rng, recipe: Recipe, n: int) -> np.ndarray:
    if recipe.vocab == "loguniform":
        lo, hi = np.log(recipe.vocab_lo), np.log(recipe.vocab_hi)
        return np.rint(np.exp(rng.uniform(lo, hi, size=n))).astype(np.uint32)
    return np.full(n, int(recipe.vocab), dtype=np.uint32)


def make_workload(name_or_recipe, seed: int = 0, **overrides) -> Workload:
    """Draw one workload.  ``overrides`` replace Recipe fields (e.g. n_ads, batch)."""
    recipe = RECIPES[name_or_recipe] if isinstance(name_or_recipe, str) else name_or_recipe
    if overrides:
        recipe = replace(recipe, **overrides)
    children = np.random.SeedSequence(seed).spawn(len(_STREAMS))
    rngs = {k: np.random.Generator(np.random.PCG64(c)) for k, c in zip(_STREAMS, children)}

    n, d, f_u, f_a, B = recipe.n_ads, recipe.d, recipe.f_u, recipe.f_a, recipe.batch
    vocab_u = _vocab(rngs["vocab_u"], recipe, f_u)
    vocab_a = _vocab(rngs["vocab_a"], recipe, f_a)
    key_off = np.zeros(f_a + 1, dtype=np.uint64)
    key_off[1:] = np.cumsum(vocab_a.astype(np.uint64))
    assert key_off[-1] < 2**32
    key_off = key_off.astype(np.uint32)

    perm_u = [rngs["perm_u"].permutation(int(v)) for v in vocab_u]
    perm_a = [rngs["perm_a"].permutation(int(v)) for v in vocab_a]

    ad_vals = np.empty((n, f_a), dtype=np.uint32)
    for j in range(f_a):
        ad_vals[:, j] = _zipf_sample(rngs["ad_vals"], int(vocab_a[j]), recipe.zipf_ad, n,
                                     perm_a[j])
    users = np.empty((B, f_u), dtype=np.uint32)
    for i in range(f_u):
        users[:, i] = _zipf_sample(rngs["user_vals"], int(vocab_u[i]), recipe.zipf_user, B,
                                   perm_u[i])

    all_pairs = np.array([(i, j) for i in range(f_u) for j in range(f_a)], dtype=np.uint32)
    if recipe.n_pairs is None or recipe.n_pairs >= len(all_pairs):
        pairs = all_pairs
    else:
        idx = np.sort(rngs["pairs"].choice(len(all_pairs), size=recipe.n_pairs, replace=False))
        pairs = all_pairs[idx]

    std = np.float32(np.sqrt(recipe.w_var))
    if recipe.weights == "dense":
        sizes = [int(vocab_u[i]) * int(vocab_a[j]) for i, j in pairs]
        w_off = np.zeros(len(pairs), dtype=np.uint64)
        w_off[1:] = np.cumsum(np.array(sizes[:-1], dtype=np.uint64))
        w_table = (rngs["weights"].standard_normal(sum(sizes), dtype=np.float32) * std)
    elif recipe.weights == "hashed":
        w_off = np.zeros(len(pairs), dtype=np.uint64)
        w_table = rngs["weights"].standard_normal(1 << HASH_BITS, dtype=np.float32) * std
    else:
        raise ValueError(recipe.weights)

    estd = np.float32(np.sqrt(1.0 / d))
    emb = rngs["emb"].standard_normal((n, d), dtype=np.float32)
    emb *= estd
    h_u = rngs["h_u"].standard_normal((B, d), dtype=np.float32) * estd

    if recipe.k_choices:
        ks = rngs["k_choice"].choice(np.array(recipe.k_choices, dtype=np.uint32), size=B)
    else:
        ks = np.full(B, recipe.k, dtype=np.uint32)
    ks = np.minimum(ks, n).astype(np.uint32)

    filters = None
    if recipe.filter_frac is not None:
        filters = make_filters(rngs["filter"], n, B, recipe.filter_frac)

    return Workload(recipe, vocab_u, vocab_a, key_off, ad_vals, pairs,
                    w_table.astype(np.float32), w_off, emb, users, h_u, ks, filters, seed,
                    rngs)


def make_filters(rng, n: int, B: int, frac) -> np.ndarray:
    """Per-request targeting bitmaps: bit a set iid with probability f ~ U[lo, hi]."""
    words = (n + 63) // 64
    out = np.zeros((B, words), dtype=np.uint64)
    for b in range(B):
        f = rng.uniform(frac[0], frac[1])
        bits = rng.random(n) < f
        padded = np.zeros(words * 64, dtype=bool)
        padded[:n] = bits
        out[b] = np.packbits(padded, bitorder="little").view(np.uint64)
    return out


def sparse_query(w: "Workload", n_q: int, seed: int = 0, var: float = 0.05):
    """A request whose cross term touches only a few hundred keys (the paper's
    own regime: the user's history values carry the non-zero weights): n_q
    distinct ad-field keys drawn with the frequency of their posting lists
    (popular values are the likely history matches), weights iid N(0, var).
    Returns (q_key uint32 [n], q_w float32 [n]), n <= n_q after de-duplication."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 11])))
    n, f_a = w.ad_vals.shape
    picks = rng.integers(0, n * f_a, size=4 * n_q)
    keys = (w.ad_vals.reshape(-1)[picks] + w.key_off[picks % f_a]).astype(np.uint32)
    _, first = np.unique(keys, return_index=True)
    q_key = keys[np.sort(first)][:n_q]
    q_w = (rng.standard_normal(q_key.size) * np.sqrt(var)).astype(np.float32)
    return q_key, q_w


def refreshed(w: "Workload", frac: float = 0.01, seed: int = 0) -> "Workload":
    """The same inventory after an update of the feature->ad map L: a fraction
    `frac` of the ads get new field values (uniform within each field's
    vocabulary) and a new embedding row; everything else is shared with `w`.
    Stands in for the periodic rebuild of the index from fresh logs."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 13])))
    n, f_a = w.ad_vals.shape
    ads = np.sort(rng.choice(n, size=max(1, int(frac * n)), replace=False))
    vals = w.ad_vals.copy()
    vals[ads] = (rng.random((ads.size, f_a)) * w.vocab_a[None, :]).astype(np.uint32)
    vals[ads] = np.minimum(vals[ads], w.vocab_a[None, :] - 1)
    emb = w.emb.copy()
    d = emb.shape[1]
    emb[ads] = (rng.standard_normal((ads.size, d)) / np.sqrt(d)).astype(np.float32)
    return replace(w, ad_vals=vals, emb=emb,
                   _rngs={"shuffle": np.random.Generator(np.random.PCG64(
                       np.random.SeedSequence([seed, 14])))})


def with_empty_ad_fields(w: "Workload", frac: float = 0.1, seed: int = 0) -> "Workload":
    """The same workload with a fraction `frac` of all (ad, field) entries
    emptied (set to EMPTY_VALUE): ads that lack some features."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 15])))
    vals = w.ad_vals.copy()
    vals[rng.random(vals.shape) < frac] = EMPTY_VALUE
    return replace(w, ad_vals=vals,
                   _rngs={"shuffle": np.random.Generator(np.random.PCG64(
                       np.random.SeedSequence([seed, 16])))})


def user_histories(w: "Workload", n_users: int, max_len: int = 8, seed: int = 0,
                   p_empty: float = 0.1):
    """Multi-valued user fields (a history of values per field): per user,
    (user_ptr uint32 [F_u + 1], user_vals uint32 [user_ptr[-1]]).  Each field
    holds 1..max_len values drawn uniformly (repeats allowed) from its
    vocabulary, or none with probability p_empty."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 17])))
    f_u = w.vocab_u.size
    out = []
    for _ in range(n_users):
        lens = rng.integers(1, max_len + 1, size=f_u)
        lens[rng.random(f_u) < p_empty] = 0
        ptr = np.zeros(f_u + 1, np.uint32)
        ptr[1:] = np.cumsum(lens)
        vals = np.concatenate([
            np.minimum((rng.random(int(n)) * int(w.vocab_u[i])).astype(np.uint32),
                       np.uint32(w.vocab_u[i] - 1)) for i, n in enumerate(lens)]
            + [np.zeros(0, np.uint32)]).astype(np.uint32)
        out.append((ptr, vals))
    return out


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int = 0) -> np.ndarray:
    """Open-loop request arrival times (seconds), exponential inter-arrivals."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 7])))
    n_est = int(rate_per_s * duration_s * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_est))
    while t[-1] < duration_s:
        t = np.concatenate([t, t[-1] + np.cumsum(rng.exponential(1.0 / rate_per_s,
                                                                 size=n_est))])
    return t[t < duration_s]
