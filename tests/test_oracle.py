"""Pins for the FP64 CPU oracle (no GPU).

Each test ties the oracle to something other than itself: a hand-worked example,
a published test vector, a library routine on a special case, brute force, or
an invariant of the method (Eq. 1, the HitMatch equation of Sec. 3.3,
Algorithm 1, Algorithm 2's output definition).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2511_22460_gb300.datagen import make_workload

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _expand_range(x):
    if isinstance(x, str) and ".." in x:
        a, b = x.split("..")
        return list(range(int(a), int(b) + 1))
    return x


# ---------------------------------------------------------------- hashing

def test_splitmix64_published_sequence():
    # SplitMix64 seeded with 0 yields e220a8397b1dcdaf, 6e789e6aa1b965f4,
    # 06c45d188009454f (the generator's published output).  The n-th output is
    # splitmix64((n - 1) * golden_gamma) in this oracle's one-shot form.
    g = 0x9E3779B97F4A7C15
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(g) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64((2 * g) % 2**64) == 0x06C45D188009454F


def test_hashed_weight_addressing():
    # Table entry i holds the float i, so w_hat reveals the address used.
    bits = 24
    table = np.arange(1 << bits, dtype=np.float32)
    vocab_u, vocab_a = [7, 3], [5, 4]
    pairs = [(1, 0), (0, 1)]
    cross = oracle.Cross(vocab_u, vocab_a, pairs, table, hashed=True, hash_bits=bits)
    user = np.array([6, 2], np.uint32)
    wh = oracle.expand(cross, user)
    mask = (1 << bits) - 1
    for p, (i, j) in enumerate(pairs):
        for v in range(vocab_a[j]):
            x = (p << 40) | (int(user[i]) << 20) | v
            assert wh[cross.key_off[j] + v] == float(oracle.splitmix64(x) & mask)


# ---------------------------------------------------------------- scores

def _tiny_cross(g):
    return oracle.Cross(g["vocab_u"], g["vocab_a"], g["pairs"],
                        np.array(g["w_table"], np.float32),
                        np.array(g["w_off"], np.uint64), hashed=False)


def test_brute_force_hand_example():
    g = _load("score_tiny.json")
    cross = _tiny_cross(g)
    s, cond = oracle.scores_brute(cross, g["h_u"], np.array(g["emb"], np.float32),
                                  g["ad_vals"], g["user"], with_cond=True)
    np.testing.assert_array_equal(s, g["expected_scores"])
    np.testing.assert_array_equal(cond, g["expected_cond"])
    wh = oracle.expand(cross, g["user"])
    np.testing.assert_array_equal(wh, g["expected_w_hat"])
    ids, vals = oracle.topk(s, 2)
    assert list(ids) == g["expected_top2_ids"]
    np.testing.assert_array_equal(vals, g["expected_top2_scores"])


def _small(name="single_fp32_10k", n_ads=2000, seed=0, **kw):
    return make_workload(name, seed=seed, n_ads=n_ads, **kw)


@pytest.mark.parametrize("name,kw", [
    ("single_fp32_10k", {}),
    ("single_fp32_2m", {"n_ads": 1500}),
    ("fp8_10m", {"n_ads": 1200, "f_u": 6, "f_a": 6, "n_pairs": 20}),
])
def test_postings_oracle_equals_brute_force(name, kw):
    kw = dict({"n_ads": 2000}, **kw)
    w = make_workload(name, seed=3, **kw)
    cross = oracle.Cross.from_workload(w)
    pk, pa = w.postings(shuffle=True)
    s1, cond = oracle.scores_brute(cross, w.h_u[0], w.emb, w.ad_vals, w.users[0],
                                   with_cond=True)
    s2 = oracle.score_query(w, 0, cross, (pk, pa))
    # Only the FP64 summation order differs.
    assert np.max(np.abs(s1 - s2) / np.maximum(cond, 1e-300)) < 1e-12


def test_zero_cross_weights_reduce_to_dual_tower():
    w = _small()
    cross = oracle.Cross(w.vocab_u, w.vocab_a, w.pairs, np.zeros_like(w.w_table), w.w_off,
                         hashed=False)
    s = oracle.scores_brute(cross, w.h_u[0], w.emb, w.ad_vals, w.users[0])
    ref = w.emb.astype(np.float64) @ w.h_u[0].astype(np.float64)
    np.testing.assert_allclose(s, ref, rtol=1e-13, atol=1e-15)


def test_zero_embeddings_equal_sparse_matvec():
    scipy_sparse = pytest.importorskip("scipy.sparse")
    w = _small()
    cross = oracle.Cross.from_workload(w)
    zero = np.zeros_like(w.emb)
    s = oracle.scores_brute(cross, w.h_u[0], zero, w.ad_vals, w.users[0])
    wh = oracle.expand(cross, w.users[0])
    pk, pa = w.postings()
    L = scipy_sparse.csr_matrix((np.ones(pk.size), (pa, pk)), shape=(w.n_ads, w.n_keys))
    np.testing.assert_allclose(s, L @ wh, rtol=1e-13, atol=1e-15)


def test_permutation_of_ad_ids_permutes_scores():
    w = _small()
    cross = oracle.Cross.from_workload(w)
    s = oracle.scores_brute(cross, w.h_u[0], w.emb, w.ad_vals, w.users[0])
    perm = np.random.default_rng(1).permutation(w.n_ads)  # new id of old ad a = perm[a]
    emb2 = np.empty_like(w.emb)
    vals2 = np.empty_like(w.ad_vals)
    emb2[perm] = w.emb
    vals2[perm] = w.ad_vals
    s2 = oracle.scores_brute(cross, w.h_u[0], emb2, vals2, w.users[0])
    np.testing.assert_array_equal(s2[perm], s)
    ids, _ = oracle.topk(s, 50)
    ids2, _ = oracle.topk(s2, 50)
    np.testing.assert_array_equal(ids2, perm[ids])


def test_linearity_duplicates_and_one_hot():
    w = _small()
    pk, pa = w.postings(shuffle=True)
    rng = np.random.default_rng(5)
    zero_u = np.zeros(w.recipe.d, np.float32)
    keys = np.arange(w.n_keys, dtype=np.uint32)
    w1 = rng.standard_normal(w.n_keys)
    w2 = rng.standard_normal(w.n_keys)
    s1 = oracle.scores_postings(w.h_u[0], w.emb, w.n_keys, pk, pa, keys, w1)
    s12 = oracle.scores_postings(w.h_u[0], w.emb, w.n_keys, pk, pa, keys, w1 + w2)
    wide2 = oracle.scores_postings(zero_u, w.emb, w.n_keys, pk, pa, keys, w2)
    np.testing.assert_allclose(s12 - s1, wide2, rtol=1e-12, atol=1e-12)
    # duplicate keys add: (k, a) and (k, b) == (k, a + b)
    dup = oracle.scores_postings(zero_u, w.emb, w.n_keys, pk, pa,
                                 np.concatenate([keys, keys]), np.concatenate([w1, w2]))
    one = oracle.scores_postings(zero_u, w.emb, w.n_keys, pk, pa, keys, w1 + w2)
    np.testing.assert_allclose(dup, one, rtol=1e-12, atol=1e-12)
    # one-hot: a single key adds exactly its weight to its posting list only
    k = int(pk[17])
    oh = oracle.scores_postings(zero_u, w.emb, w.n_keys, pk, pa, [k], [0.75])
    members = np.zeros(w.n_ads, bool)
    members[pa[pk == k]] = True
    np.testing.assert_array_equal(oh[members], 0.75)
    np.testing.assert_array_equal(oh[~members], 0.0)


# ------------------------------------ multi-valued user fields, empty ad fields

def test_multi_valued_hand_example():
    g = _load("score_seq_tiny.json")
    cross = _tiny_cross(g)
    emb = np.array(g["emb"], np.float32)
    s, cond = oracle.scores_brute_seq(cross, g["h_u"], emb, g["ad_vals"], g["user_ptr"],
                                      g["user_vals"], with_cond=True)
    np.testing.assert_array_equal(s, g["expected_scores"])
    np.testing.assert_array_equal(cond, g["expected_cond"])
    wh = oracle.expand_seq(cross, g["user_ptr"], g["user_vals"])
    np.testing.assert_array_equal(wh, g["expected_w_hat"])
    ids, _ = oracle.topk(s, 2)
    assert list(ids) == g["expected_top2_ids"]


def test_one_value_per_field_reduces_to_single_valued():
    w = _small(n_ads=800)
    cross = oracle.Cross.from_workload(w)
    ptr = np.arange(len(w.vocab_u) + 1, dtype=np.uint32)
    a, ca = oracle.scores_brute_seq(cross, w.h_u[0], w.emb, w.ad_vals, ptr, w.users[0],
                                    with_cond=True)
    b, cb = oracle.scores_brute(cross, w.h_u[0], w.emb, w.ad_vals, w.users[0], with_cond=True)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(ca, cb)
    np.testing.assert_array_equal(oracle.expand_seq(cross, ptr, w.users[0]),
                                  oracle.expand(cross, w.users[0]))


def test_history_is_additive_in_its_values():
    # each (user value, ad value) is its own hit feature: w_hat is linear in
    # the multiset of a field's values; an empty field adds nothing
    w = _small(n_ads=200)
    cross = oracle.Cross.from_workload(w)
    f_u = len(w.vocab_u)
    base = [int(x) for x in w.users[0]]
    a, b = 1, min(2, int(w.vocab_u[0]) - 1)

    def seq(first):
        vals = list(first) + base[1:]
        ptr = np.array([0, len(first)] + [len(first) + i for i in range(1, f_u)], np.uint32)
        return ptr, np.array(vals, np.uint32)

    e_ab = oracle.expand_seq(cross, *seq([a, b]))
    e_a = oracle.expand_seq(cross, *seq([a]))
    e_b = oracle.expand_seq(cross, *seq([b]))
    e_0 = oracle.expand_seq(cross, *seq([]))
    np.testing.assert_allclose(e_ab - e_a, e_b - e_0, rtol=1e-12, atol=1e-12)
    e_aa = oracle.expand_seq(cross, *seq([a, a]))
    np.testing.assert_allclose(e_aa - e_0, 2 * (e_a - e_0), rtol=1e-12, atol=1e-12)
    # with every field empty the score is the dual-tower term alone
    ptr0 = np.zeros(f_u + 1, np.uint32)
    s = oracle.scores_brute_seq(cross, w.h_u[0], w.emb, w.ad_vals, ptr0, np.zeros(0, np.uint32))
    np.testing.assert_allclose(s, w.emb.astype(np.float64) @ w.h_u[0].astype(np.float64),
                               rtol=1e-13, atol=1e-15)


def test_postings_oracle_equals_brute_force_with_histories_and_empty_fields():
    from paper_2511_22460_gb300.datagen import user_histories, with_empty_ad_fields
    w = with_empty_ad_fields(_small(n_ads=1500, seed=4), 0.15, seed=2)
    cross = oracle.Cross.from_workload(w)
    pk, pa = w.postings(shuffle=True)
    assert pk.size == w.nnz < w.ad_vals.size
    for ptr, vals in user_histories(w, 3, max_len=5, seed=7):
        s1, cond = oracle.scores_brute_seq(cross, w.h_u[0], w.emb, w.ad_vals, ptr, vals,
                                           with_cond=True)
        s2 = oracle.score_query_seq(w, w.h_u[0], ptr, vals, cross, (pk, pa))
        assert np.max(np.abs(s1 - s2) / np.maximum(cond, 1e-300)) < 1e-12


def test_history_rejects_bad_offsets_and_values():
    w = _small(n_ads=100)
    cross = oracle.Cross.from_workload(w)
    f_u = len(w.vocab_u)
    good = np.arange(f_u + 1, dtype=np.uint32)
    bad_ptr = good.copy()
    bad_ptr[2], bad_ptr[3] = 3, 2  # decreasing
    with pytest.raises(ValueError):
        oracle.expand_seq(cross, bad_ptr, w.users[0])
    vals = w.users[0].copy()
    vals[1] = w.vocab_u[1]
    with pytest.raises(ValueError):
        oracle.scores_brute_seq(cross, w.h_u[0], w.emb, w.ad_vals, good, vals)


def test_repeated_pairs_count_once():
    # L is binary (Sec. 3.3): listing a (key, ad) pair twice changes nothing.
    rng = np.random.default_rng(12)
    n_keys, n_ads = 40, 300
    pk = rng.integers(0, n_keys, 2000).astype(np.uint32)
    pa = rng.integers(0, n_ads, 2000).astype(np.uint32)
    pk2, pa2 = np.concatenate([pk, pk[:700]]), np.concatenate([pa, pa[:700]])
    w_k = rng.standard_normal(n_keys)
    keys = np.arange(n_keys, dtype=np.uint32)
    h = np.zeros(4, np.float32)
    emb = np.zeros((n_ads, 4), np.float32)
    dense = np.zeros((n_ads, n_keys))
    dense[pa, pk] = 1.0  # 0/1 matrix, repeats collapse
    got = oracle.scores_postings(h, emb, n_keys, pk2, pa2, keys, w_k)
    np.testing.assert_allclose(got, dense @ w_k, rtol=1e-13, atol=1e-13)
    uk, ua = oracle.unique_pairs(pk2, pa2)
    assert len(uk) == len(set(zip(pk.tolist(), pa.tolist())))


def test_postings_of_each_field_partition_the_ads():
    w = _small()
    pk, pa = w.postings()
    for j in range(w.recipe.f_a):
        lo, hi = int(w.key_off[j]), int(w.key_off[j + 1])
        m = (pk >= lo) & (pk < hi)
        ads = np.sort(pa[m])
        np.testing.assert_array_equal(ads, np.arange(w.n_ads))


# ---------------------------------------------------------------- top-K

def test_topk_matches_sorted_with_ties_and_filter():
    rng = np.random.default_rng(2)
    s = np.round(rng.standard_normal(3000), 1)  # many exact ties
    filt_bits = rng.random(3000) < 0.4
    words = np.zeros((3000 + 63) // 64, np.uint64)
    for a in np.nonzero(filt_bits)[0]:
        words[a >> 6] |= np.uint64(1) << np.uint64(a & 63)
    for k, f, mask in [(100, None, np.ones(3000, bool)), (77, words, filt_bits),
                       (5000, words, filt_bits)]:
        ids, vals = oracle.topk(s, k, f)
        ref = sorted((a for a in range(3000) if mask[a]), key=lambda a: (-s[a], a))[:k]
        assert list(ids) == ref
        np.testing.assert_array_equal(vals, s[ref])
    full = np.full(len(words), np.uint64(0xFFFFFFFFFFFFFFFF))
    a, _ = oracle.topk(s, 100, full)
    b, _ = oracle.topk(s, 100, None)
    np.testing.assert_array_equal(a, b)


# ---------------------------------------------------------------- Algorithm 1

def _gold_alg1():
    g = _load("alg1_tiny.json")
    pk, pa = [], []
    for k, a in g["postings"]:
        for ad in (_expand_range(a) if isinstance(a, str) else [a]):
            pk.append(k)
            pa.append(ad)
    return g, np.array(pk, np.uint32), np.array(pa, np.uint32)


def test_alg1_hand_example():
    g, pk, pa = _gold_alg1()
    ix = oracle.build_index(g["n_keys"], g["n_ads"], pk, pa)
    exp = g["expected"]
    for grp in range(9):
        assert list(ix["keys"][grp]) == exp["keys"][grp], grp
        assert list(ix["header"][grp]) == exp["header"][grp], grp
        assert list(ix["values"][grp]) == _expand_range(exp["values"][grp]), grp


def _check_layout_rules(ix, pk, pa):
    n_keys = ix["n_keys"]
    pairs = set(zip(pk.tolist(), pa.tolist()))
    dk, da = oracle.decode_index(ix)
    decoded = list(zip(dk.tolist(), da.tolist()))
    assert len(decoded) == len(set(decoded)) == len(pairs)
    assert set(decoded) == pairs
    total_real = 0
    for g in range(9):
        keys, hdr, vals = ix["keys"][g], ix["header"][g], ix["values"][g]
        assert keys[0] == 0 and keys[-1] == len(hdr) and np.all(np.diff(keys.astype(np.int64)) >= 0)
        assert vals.size == len(hdr) << g
        blocks = vals.reshape(-1, 1 << g) if len(hdr) else np.zeros((0, 1 << g), np.uint8)
        for k in range(n_keys):
            hs = hdr[keys[k]:keys[k + 1]]
            assert np.all(np.diff(hs.astype(np.int64)) > 0)  # (k, h) ascending, unique
        for b in range(len(hdr)):
            row = blocks[b]
            real = [row[0]] + [x for x in row[1:] if x != 0]
            n = len(real)
            assert (1 << g) >= n and (g == 0 or (1 << (g - 1)) < n)  # g = ceil(log2 n)
            assert all(real[i] < real[i + 1] for i in range(n - 1))
            assert all(x == 0 for x in row[n:])
            total_real += n
    assert total_real == len(pairs)


def test_alg1_layout_rules_on_random_postings():
    rng = np.random.default_rng(11)
    n_keys, n_ads = 60, 5000
    # skewed, with duplicates, empty keys, multi-valued and empty ads
    pk = (rng.zipf(1.6, 20000) % n_keys).astype(np.uint32)
    pk[pk == 7] = 8  # key 7 empty
    pa = rng.integers(0, n_ads, 20000).astype(np.uint32)
    pa[pa == 123] = 124  # ad 123 in no list
    ix = oracle.build_index(n_keys, n_ads, pk, pa)
    _check_layout_rules(ix, pk, pa)
    for g in range(9):
        assert ix["keys"][g][7] == ix["keys"][g][8]


def test_alg1_dense_window_and_workload_postings():
    w = _small(n_ads=3000)
    pk, pa = w.postings(shuffle=True)
    ix = oracle.build_index(w.n_keys, w.n_ads, pk, pa)
    _check_layout_rules(ix, pk, pa)
    # one key holding every ad: three full 256-slot blocks, then a tail of
    # 1000 - 768 = 232 ads, also group 8 (128 < 232 <= 256), padded with 24 zeros
    n = 1000
    ix2 = oracle.build_index(1, n, np.zeros(n, np.uint32), np.arange(n, dtype=np.uint32))
    assert list(ix2["header"][8]) == [0, 1, 2, 3]
    assert all(ix2["header"][g].size == 0 for g in range(8))
    v = ix2["values"][8].reshape(4, 256)
    np.testing.assert_array_equal(v[:3], np.tile(np.arange(256), (3, 1)))
    np.testing.assert_array_equal(v[3, :232], np.arange(232))
    assert np.all(v[3, 232:] == 0)


def test_alg1_rejects_out_of_range():
    with pytest.raises(ValueError):
        oracle.build_index(3, 10, np.array([3], np.uint32), np.array([0], np.uint32))
    with pytest.raises(ValueError):
        oracle.build_index(3, 10, np.array([0], np.uint32), np.array([10], np.uint32))


# ---------------------------------------------------------------- quantisers

def test_bf16_against_torch_and_round_trip():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10.0 ** rng.integers(
        -30, 30, 20000), np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, 3.3895314e38,
                                   3.4e38, 1e-40, -1e-42], np.float32)]).astype(np.float32)
    ours = oracle.bf16_rne(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(ours, ref)
    # halfway cases tie to even
    lo = np.uint32(0x3F800000)  # 1.0
    halfway = np.array([lo | 0x8000, (lo + 0x10000) | 0x8000], np.uint32).view(np.float32)
    assert list(oracle.bf16_rne(halfway)) == [0x3F80, 0x3F82]
    # every non-NaN encoding is a fixed point
    h = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    v = oracle.bf16_value(h)
    ok = ~np.isnan(v)
    np.testing.assert_array_equal(oracle.bf16_rne(v[ok]), h[ok])


def test_fp8_e4m3_spec_table():
    # OCP 8-bit FP, E4M3: bias 7, max 448 = 0x7E, min subnormal 2^-9 = 0x01,
    # 1.0 = 0x38, NaN = S.1111.111, no infinities.
    assert oracle.fp8_e4m3_value([0x7E]) == [448.0]
    assert oracle.fp8_e4m3_value([0x01]) == [2.0 ** -9]
    assert oracle.fp8_e4m3_value([0x08]) == [2.0 ** -6]
    assert oracle.fp8_e4m3_value([0x38]) == [1.0]
    assert oracle.fp8_e4m3_value([0xB8]) == [-1.0]
    assert np.isnan(oracle.fp8_e4m3_value([0x7F, 0xFF])).all()
    enc = oracle.fp8_e4m3_rne_sat
    assert list(enc([448.0, 500.0, 1e9, -1e9, 1.0, -1.0, 0.0, np.nan])) == \
        [0x7E, 0x7E, 0x7E, 0xFE, 0x38, 0xB8, 0x00, 0x7F]
    assert list(enc([2.0 ** -10, 3 * 2.0 ** -10, 1.0625, 1.1875])) == [0x00, 0x02, 0x38, 0x3A]
    # round trip of every finite code
    codes = [c for c in range(256) if (c & 0x7F) != 0x7F]
    vals = oracle.fp8_e4m3_value(codes)
    back = enc(vals.astype(np.float32))
    for c, b in zip(codes, back):
        assert b == c or (c == 0x80 and b == 0x80)


def test_fp8_e4m3_against_torch():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8")
    rng = np.random.default_rng(6)
    x = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-4, 2.6, 20000)).astype(np.float32)
    x = np.clip(x, -448, 448)
    ours = oracle.fp8_e4m3_rne_sat(x)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    np.testing.assert_array_equal(ours, ref)


def test_fp8_rows_scale_rule():
    rng = np.random.default_rng(8)
    x = rng.standard_normal((50, 16)).astype(np.float32)
    x[3] = 0.0
    q, s = oracle.quantize_fp8_rows(x)
    assert s[3] == 1.0 and np.all(q[3] == 0)
    mx = np.abs(x).max(axis=1)
    np.testing.assert_array_equal(s[mx > 0], (mx[mx > 0] / np.float32(448.0)).astype(np.float32))
    # the row maximum maps to +-448 exactly
    for r in range(50):
        if r == 3:
            continue
        t = int(np.argmax(np.abs(x[r])))
        assert q[r, t] & 0x7F == 0x7E
    deq = oracle.fp8_e4m3_value(q) * s[:, None]
    rel = np.abs(deq - x) / np.maximum(np.abs(x), 2.0 ** -6 * s[:, None])
    assert rel.max() <= 2.0 ** -4 + 1e-12  # half an ulp of a 3-bit mantissa
