"""GPU parity when the query weights w^ span many orders of magnitude.

The window-major traversal accumulates each ad's wide term (the HitMatch sum of
Sec. 3.3) partly in fixed point with one quantum per request, chosen from the
request's largest |w^|.  The tolerance of the FP32 path is relative to each
ad's own condition scale (|s - s_ref| <= 1e-5 * max(|s|, sum |h_u h_a| +
sum |w|)), so an ad whose keys all carry weights far below the request's
largest must still get its small terms right.  These cases make exactly that
happen: one key boosted to 1e3 while every other weight is ~1e-6 (a range of
~1e9), ads that hold only tiny-weight keys, zero user vectors (no dot-product
term to hide an error behind), FP32 and BF16 tables, dense w^ and a heavy
sparse list that the device routes window-major.  Every comparison is against
the FP64 postings oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2511_22460_gb300 import ebr  # noqa: E402
from paper_2511_22460_gb300.datagen import make_workload, sparse_query  # noqa: E402

from gpu_util import check_scores, check_topk, recall  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _setup(n, seed, dtype="f32"):
    w = make_workload("single_fp32_2m", n_ads=n, seed=seed)
    pk, pa = w.postings()
    ix = ebr.build_index(w.n_ads, w.n_keys, pk, pa, w.emb, dtype=dtype)
    return w, pk, pa, ix


def _ref(w, pk, pa, h_u, q_key, q_w):
    """FP64 scores and the per-ad Z8 tolerance of an explicit (key, w) query."""
    q_w64 = q_w.astype(np.float64)
    ref = oracle.scores_postings(h_u, w.emb, w.n_keys, pk, pa, q_key, q_w64)
    wabs = np.zeros(w.n_keys)
    np.add.at(wabs, q_key, np.abs(q_w64))
    cond = np.abs(w.emb.astype(np.float64)) @ np.abs(h_u.astype(np.float64)) + np.bincount(
        pa, weights=wabs[pk], minlength=w.n_ads)
    return ref, 1e-5 * np.maximum(np.abs(ref), cond)


def _wide_range_weights(w, pk, pa, seed, quiet_ads=64):
    """Dense w^: the expansion of user 0, then every key of `quiet_ads` ads
    scaled by 1e-6, 5% of the other keys by 1e-4, and the most popular key
    held by none of the quiet ads set to 1e3."""
    rng = np.random.default_rng(seed)
    wh = oracle.expand(oracle.Cross.from_workload(w), w.users[0]).astype(np.float64)
    quiet = rng.choice(w.n_ads, quiet_ads, replace=False)
    qkeys = np.unique(pk[np.isin(pa, quiet)])
    wh[rng.random(w.n_keys) < 0.05] *= 1e-4
    wh[qkeys] *= 1e-6
    counts = np.bincount(pk, minlength=w.n_keys)
    counts[qkeys] = -1
    boost = int(np.argmax(counts))
    wh[boost] = 1e3
    return wh.astype(np.float32), quiet, boost


@pytest.mark.parametrize("zero_h", [True, False], ids=["h_zero", "h_user"])
def test_score_all_window_major_wide_range(zero_h):
    n = 150_011  # several windows per CTA, a ragged last window
    w, pk, pa, ix = _setup(n, seed=21)
    wh, quiet, boost = _wide_range_weights(w, pk, pa, seed=3)
    h_u = np.zeros(w.recipe.d, np.float32) if zero_h else w.h_u[0]
    keys = np.arange(w.n_keys, dtype=np.uint32)
    ref, tol = _ref(w, pk, pa, h_u, keys, wh)
    out = torch.empty(n, dtype=torch.float32, device=DEV)
    ebr.score_all(ix, None, ebr.Query(h_u=dev(h_u), k=1, q_w=dev(wh)), out)
    got = out.cpu().numpy()
    check_scores(got[quiet], ref[quiet], tol[quiet], "ads holding only tiny weights")
    check_scores(got, ref, tol, "every ad")
    # the key-major traversal (FP32 atomics, Algorithm 2) agrees as well
    ebr.score_all(ix, None, ebr.Query(h_u=dev(h_u), k=1, q_w=dev(wh),
                                      flags=ebr.QF_KEY_MAJOR), out)
    check_scores(out.cpu().numpy(), ref, tol, "key-major")


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_topk_ranked_by_tiny_weights(dtype):
    """Every weight ~1e-6 except one key at -1e3: with a zero user vector the
    ranking is decided by the tiny weights alone."""
    n, k = 120_007, 500
    w, pk, pa, ix = _setup(n, seed=22, dtype=dtype)
    rng = np.random.default_rng(4)
    wh = (rng.standard_normal(w.n_keys) * 1e-6).astype(np.float32)
    boost = int(np.argmax(np.bincount(pk, minlength=w.n_keys)))
    wh[boost] = -1e3
    h_u = np.zeros(w.recipe.d, np.float32)
    keys = np.arange(w.n_keys, dtype=np.uint32)
    ref, tol = _ref(w, pk, pa, h_u, keys, wh)
    ids = torch.empty(k, dtype=torch.int32, device=DEV)
    sc = torch.empty(k, dtype=torch.float32, device=DEV)
    ebr.score_topk(ix, None, [ebr.Query(h_u=dev(h_u), k=k, q_w=dev(wh))], ids, sc)
    got = ids.cpu().numpy().view(np.uint32)
    assert recall(got, ref, tol, k) == 1.0
    check_topk(got, sc.cpu().numpy(), ref, tol, k)


def test_heavy_sparse_list_wide_range_routed_window_major():
    """A heavy list (3000 keys drawn by list length, the device sends it
    window-major) whose weights span 1e-7 .. 1e3."""
    n, k = 200_003, 400
    w, pk, pa, ix = _setup(n, seed=23)
    qk, _ = sparse_query(w, 3000, seed=5)
    rng = np.random.default_rng(6)
    qw = (rng.standard_normal(qk.size) * 10.0 ** rng.uniform(-7, -3, qk.size)).astype(np.float32)
    qw[0] = 1e3
    qw[1] = -1e3
    h_u = w.h_u[0]
    ref, tol = _ref(w, pk, pa, h_u, qk, qw)
    ids = torch.empty(k, dtype=torch.int32, device=DEV)
    sc = torch.empty(k, dtype=torch.float32, device=DEV)
    ix.profile_enable(True)
    ebr.score_topk(ix, None, [ebr.Query(h_u=dev(h_u), k=k, q_key=dev(qk), q_w=dev(qw))], ids, sc)
    p = ix.profile_read()
    ix.profile_enable(False)
    assert (p.auto_routed, p.window_routed) == (1, 1), "the list should go window-major"
    check_topk(ids.cpu().numpy().view(np.uint32), sc.cpu().numpy(), ref, tol, k)
    # every score of the same list, summed into a dense w^ (the form the
    # window-major decode reads), against the oracle
    dense = np.zeros(w.n_keys)
    np.add.at(dense, qk, qw.astype(np.float64))
    out = torch.empty(n, dtype=torch.float32, device=DEV)
    ebr.score_all(ix, None, ebr.Query(h_u=dev(h_u), k=1, q_w=dev(dense.astype(np.float32))), out)
    check_scores(out.cpu().numpy(), ref, tol, "window-major sparse list")
