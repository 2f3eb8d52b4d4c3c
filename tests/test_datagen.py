"""Host-side checks of the synthetic workload generator (no GPU)."""
import numpy as np

from paper_2511_22460_gb300.datagen import (RECIPES, make_filters, make_workload,
                                            poisson_arrivals)


def test_filter_bitmap_layout():
    rng = np.random.default_rng(0)
    n = 1000
    f = make_filters(rng, n, 2, (0.2, 0.6))
    assert f.shape == (2, (n + 63) // 64) and f.dtype == np.uint64
    for b in range(2):
        bits = [(int(f[b][a >> 6]) >> (a & 63)) & 1 for a in range(n)]
        ref = np.unpackbits(f[b].view(np.uint8), bitorder="little")[:n]
        assert bits == ref.tolist()
        assert all((int(f[b][-1]) >> s) & 1 == 0 for s in range(n % 64, 64))
        assert 0.15 < np.mean(bits) < 0.65


def test_workload_shapes_and_determinism():
    w1 = make_workload("single_fp32_2m", n_ads=5000, seed=3)
    w2 = make_workload("single_fp32_2m", n_ads=5000, seed=3)
    np.testing.assert_array_equal(w1.ad_vals, w2.ad_vals)
    np.testing.assert_array_equal(w1.emb, w2.emb)
    assert w1.emb.shape == (5000, 64) and w1.emb.dtype == np.float32
    assert len(w1.pairs) == 64 and len(set(map(tuple, w1.pairs.tolist()))) == 64
    assert np.all(w1.ad_vals < w1.vocab_a[None, :])
    assert np.all(w1.users < w1.vocab_u[None, :])
    assert np.all((w1.vocab_a >= 10) & (w1.vocab_a <= 100_000))
    assert abs(w1.emb.var() - 1 / 64) < 2e-3
    assert abs(w1.w_table.var() - 0.05) < 2e-3
    k, a = w1.postings(shuffle=True)
    assert k.size == a.size == 5000 * 16


def test_zipf_head_share_for_fp8_workload():
    w = make_workload("fp8_10m", n_ads=200_000, f_a=4, f_u=4, n_pairs=8, seed=1)
    for j in range(4):
        share = np.bincount(w.ad_vals[:, j]).max() / w.n_ads
        assert abs(share - 1 / sum(1 / r for r in range(1, 16))) < 0.01  # ~30%


def test_serving_recipe_draws_k_and_filters():
    w = make_workload("serve_bf16_5m", n_ads=3000, batch=50, seed=0)
    assert set(np.unique(w.ks)).issubset({100, 500, 1000})
    assert w.filters.shape == (50, (3000 + 63) // 64)
    t = poisson_arrivals(2000.0, 0.5, seed=1)
    assert np.all(np.diff(t) > 0) and 800 < t.size < 1200
    assert set(RECIPES) >= {"single_fp32_10k", "single_fp32_2m", "batch256_bf16_5m", "fp8_10m",
                            "serve_bf16_5m"}


def test_histories_empty_fields_and_refresh():
    from paper_2511_22460_gb300.datagen import (EMPTY_VALUE, refreshed, user_histories,
                                                with_empty_ad_fields)
    w = make_workload("single_fp32_10k", seed=0, n_ads=3000)
    hs = user_histories(w, 20, max_len=6, seed=1)
    f_u = w.vocab_u.size
    for ptr, vals in hs:
        assert ptr.shape == (f_u + 1,) and ptr[0] == 0 and np.all(np.diff(ptr.astype(int)) >= 0)
        assert vals.size == ptr[-1] and np.all(np.diff(ptr.astype(int)) <= 6)
        for i in range(f_u):
            assert np.all(vals[ptr[i]:ptr[i + 1]] < w.vocab_u[i])
    assert any(np.any(np.diff(p.astype(int)) == 0) for p, _ in hs)  # some empty field
    again = user_histories(w, 20, max_len=6, seed=1)
    assert all(np.array_equal(a[1], b[1]) for a, b in zip(hs, again))
    we = with_empty_ad_fields(w, 0.2, seed=3)
    frac = np.mean(we.ad_vals == EMPTY_VALUE)
    assert 0.17 < frac < 0.23 and we.nnz == int(np.sum(we.ad_vals != EMPTY_VALUE))
    pk, pa = we.postings()
    assert pk.size == we.nnz and np.all(pk < w.n_keys)
    w2 = refreshed(w, 0.05, seed=4)
    changed = np.any(w2.ad_vals != w.ad_vals, axis=1) | np.any(w2.emb != w.emb, axis=1)
    assert changed.sum() == 150 and w2.n_keys == w.n_keys
    assert np.all(w2.ad_vals < w.vocab_a[None, :])
