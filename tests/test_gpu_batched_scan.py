"""GPU parity of the batched tensor-core scan (many users per pass over the
inventory, BF16 deep term on tcgen05, FP32 rescoring) against the FP64 oracle.

The merge recomputes on the single-request scan any user whose per-CTA
candidate buffers cannot prove the top R*K exact; every test asserts that no
user was recomputed (so the results checked are the tensor-core path's own),
except the one built to make that proof fail."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import oracle  # noqa: E402
from gpu_util import bitmap_to_mask, check_topk, recall, ref_scores  # noqa: E402
from paper_2511_22460_gb300 import ebr  # noqa: E402
from paper_2511_22460_gb300.datagen import make_filters, make_workload  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _run(name, n, B, ks, seed, filt=None, io=ebr.IO_DEVICE, prep=None, dtype="bf16", **kw):
    w = make_workload(name, n_ads=n, seed=seed, batch=B, **kw)
    if prep is not None:
        prep(w)
    pk, pa = w.postings(shuffle=True)
    ix = ebr.build_index(w.n_ads, w.n_keys, pk, pa, w.emb, dtype=dtype)
    cross = ebr.cross_from_workload(w)
    kmax = max(ks)
    host = io == ebr.IO_HOST
    conv = (lambda a: np.ascontiguousarray(a)) if host else dev
    qs = [ebr.Query(h_u=conv(w.h_u[b]), k=ks[b], user_vals=conv(w.users[b]),
                    filter=None if filt is None or filt[b] is None else conv(filt[b]))
          for b in range(B)]
    if host:
        ids = np.empty((B, kmax), np.uint32)
        sc = np.empty((B, kmax), np.float32)
    else:
        ids = torch.empty((B, kmax), dtype=torch.int32, device=DEV)
        sc = torch.empty((B, kmax), dtype=torch.float32, device=DEV)
    before = ix.profile_read()
    b0, r0 = before.batched, before.recomputed
    ebr.score_topk(ix, cross, qs, ids, sc, io=io)
    after = ix.profile_read()
    if not host:
        ids = ids.cpu().numpy().view(np.uint32)
        sc = sc.cpu().numpy()
    return w, (pk, pa), ids, sc, after.batched - b0, after.recomputed - r0


def _check_all(w, post, ids, sc, ks, filt=None, users=None):
    for b in (range(len(ks)) if users is None else users):
        ref, tol = ref_scores(w, b, post)
        mask = None
        if filt is not None and filt[b] is not None:
            mask = bitmap_to_mask(filt[b], w.n_ads)
        assert recall(ids[b], ref, tol, ks[b], mask) == 1.0, "user %d" % b
        check_topk(ids[b], sc[b], ref, tol, ks[b], mask)


@pytest.mark.parametrize("name,n,B", [("serve_bf16_5m", 60_001, 64),
                                      ("batch256_bf16_5m", 40_000, 40),
                                      ("serve_bf16_5m", 20_000, 2),
                                      ("serve_bf16_5m", 30_000, 128),
                                      ("batch256_bf16_5m", 25_000, 200)])
def test_batched_topk_matches_oracle(name, n, B):
    ks = [100] * B
    w, post, ids, sc, nb, nr = _run(name, n, B, ks, seed=11)
    assert nb == B, "the batched path did not run"
    assert nr == 0, "%d users were recomputed on the single-request scan" % nr
    _check_all(w, post, ids, sc, ks)


def test_batched_mixed_k_filters_and_host_io():
    B, n = 33, 50_000
    rng = np.random.default_rng(5)
    ks = [int(x) for x in rng.choice([1, 100, 500, 1000], size=B)]
    fl = make_filters(rng, n, B, (0.001, 1.0))
    filt = [fl[b] if b % 3 else None for b in range(B)]
    filt[1] = np.zeros_like(fl[1])  # a filter that admits no ad
    w, post, ids, sc, nb, nr = _run("serve_bf16_5m", n, B, ks, seed=12, filt=filt, io=ebr.IO_HOST)
    assert nb == B and nr == 0
    _check_all(w, post, ids, sc, ks, filt, [b for b in range(B) if b != 1])
    assert np.all(ids[1] == 0xFFFFFFFF) and np.all(np.isneginf(sc[1]))


def test_batched_equals_single_request_path():
    """The same users through the batched scan and one at a time give the
    same ids (FP32 rescoring makes both exact up to score ties)."""
    B, n, k = 16, 30_000, 200
    w, post, ids, sc, nb, nr = _run("serve_bf16_5m", n, B, [k] * B, seed=13)
    assert nb == B and nr == 0
    pk, pa = post
    ix = ebr.build_index(w.n_ads, w.n_keys, pk, pa, w.emb, dtype="bf16")
    cross = ebr.cross_from_workload(w)
    for b in range(0, B, 5):
        i1 = torch.empty((1, k), dtype=torch.int32, device=DEV)
        s1 = torch.empty((1, k), dtype=torch.float32, device=DEV)
        ebr.score_topk(ix, cross, [ebr.Query(h_u=dev(w.h_u[b]), k=k, user_vals=dev(w.users[b]))],
                       i1, s1)
        ref, tol = ref_scores(w, b, post)
        a = set(ids[b].tolist())
        c = set(i1.cpu().numpy().view(np.uint32)[0].tolist())
        for x in a ^ c:  # any difference is a tie within tolerance at the K-th score
            kth = np.sort(ref)[::-1][k - 1]
            assert abs(ref[x] - kth) <= 2 * tol[x]


def test_batched_tiny_inventory_and_k_above_n():
    """Fewer ads than one window and K larger than the inventory."""
    B, n = 4, 200
    ks = [300, 50, 200, 1]
    w, post, ids, sc, nb, nr = _run("serve_bf16_5m", n, B, ks, seed=14)
    assert nb == B and nr == 0
    for b in range(B):
        ref, tol = ref_scores(w, b, post)
        take = check_topk(ids[b], sc[b], ref, tol, ks[b])
        assert take == min(ks[b], n)


def test_batched_proof_fails_for_a_crowded_window_and_is_recomputed():
    """200 ads of the first window are made the best of user 0 only (their
    rows point along the part of h_u[0] orthogonal to every other user):
    the first CTA keeps just its top m of them, so its threshold lies above
    user 0's R*K-th score and the merge cannot prove exactness for user 0
    alone; that user is recomputed on the single-request scan, and every
    result still matches the oracle."""
    B, n, k = 4, 20_000, 100

    def crowd(w):
        h = w.h_u.astype(np.float64)
        q, _ = np.linalg.qr(h[1:].T)  # basis of the other users' vectors
        v = h[0] - q @ (q.T @ h[0])
        v *= 40.0 / (v @ h[0])  # <v, h_u[0]> = 40: far above every wide term
        w.emb[:200] = (v[None, :] + 0.01 * w.emb[:200]).astype(np.float32)

    w, post, ids, sc, nb, nr = _run("serve_bf16_5m", n, B, [k] * B, seed=15, prep=crowd)
    assert nb == B
    assert nr == 1, "exactly the crowded user is recomputed (got %d)" % nr
    _check_all(w, post, ids, sc, [k] * B)
    assert np.all(ids[0].astype(np.int64) < 200), "user 0's top-K is the crowded window's"


@pytest.mark.parametrize("n,B,d,k", [(60_001, 64, 64, 500), (30_000, 40, 128, 300),
                                     (20_000, 2, 64, 100), (25_000, 200, 64, 200)])
def test_batched_fp8_topk_matches_oracle(n, B, d, k, capsys):
    """The FP8-e4m3 table with per-row scales on the tensor cores (kind::f8f6f4,
    users quantised per row the same way), FP32 rescoring of the top 4K: every
    user's top-K against the FP64 oracle, recall 1.0, nothing recomputed.  The
    recall of the quantised score before rescoring (FP8 x FP8 deep term plus
    the exact wide term, the order the tensor-core pass ranks by) is reported."""
    ks = [k] * B
    w, post, ids, sc, nb, nr = _run("fp8_10m", n, B, ks, seed=16, dtype="fp8e4m3", d=d)
    assert nb == B, "the batched path did not run"
    assert nr == 0, "%d users were recomputed on the single-request scan" % nr
    _check_all(w, post, ids, sc, ks)
    tab = oracle.fp8_e4m3_value(np.arange(256, dtype=np.uint8))
    qa, sa = oracle.quantize_fp8_rows(w.emb)
    qu, su = oracle.quantize_fp8_rows(w.h_u)
    approx_deep = (tab[qa] * sa[:, None].astype(np.float64)) @ (
        tab[qu] * su[:, None].astype(np.float64)).T
    pre = []
    for b in range(0, B, max(1, B // 8)):
        ref, tol = ref_scores(w, b, post)
        wide = ref - w.emb.astype(np.float64) @ w.h_u[b].astype(np.float64)
        approx = approx_deep[:, b] + wide
        pre.append(recall(np.lexsort((np.arange(n), -approx))[:k], ref, tol, k))
    with capsys.disabled():
        print("\n[recall] batched fp8 d=%d %d ads K=%d: before rescoring %.4f (min %.4f), after 1.0"
              % (d, n, k, float(np.mean(pre)), float(np.min(pre))))


def _history_refs(w, hs, post):
    cr = oracle.Cross.from_workload(w)
    refs = []
    for b, (p_b, v_b) in enumerate(hs):
        ref = oracle.score_query_seq(w, w.h_u[b], p_b, v_b, cr, post)
        _, cond = oracle.scores_brute_seq(cr, w.h_u[b], w.emb, w.ad_vals, p_b, v_b,
                                          with_cond=True)
        refs.append((ref, oracle.tolerance(ref, cond)))
    return refs


@pytest.mark.parametrize("dtype,io", [("bf16", ebr.IO_DEVICE), ("bf16", ebr.IO_HOST),
                                      ("fp8e4m3", ebr.IO_DEVICE)])
def test_batched_multi_valued_users(dtype, io):
    """Users whose fields hold histories (several values, some none; the
    HitMatch sum over every user value of a cross pair) mixed with
    single-valued users in one batch: all on the tensor-core scan, none
    recomputed, each against the FP64 oracle."""
    from paper_2511_22460_gb300.datagen import user_histories
    B, n, k = 24, 40_000, 200
    w = make_workload("serve_bf16_5m", n_ads=n, seed=21, batch=B)
    post = w.postings(shuffle=True)
    ix = ebr.build_index(w.n_ads, w.n_keys, *post, w.emb, dtype=dtype)
    cross = ebr.cross_from_workload(w)
    hs = user_histories(w, B, max_len=6, seed=5)
    # every third user keeps its single value per field
    hs = [(None, w.users[b]) if b % 3 == 0 else hs[b] for b in range(B)]
    host = io == ebr.IO_HOST
    conv = (lambda a: np.ascontiguousarray(a)) if host else dev
    qs = [ebr.Query(h_u=conv(w.h_u[b]), k=k, user_vals=conv(v),
                    user_ptr=None if p is None else conv(p)) for b, (p, v) in enumerate(hs)]
    if host:
        ids = np.empty((B, k), np.uint32)
        sc = np.empty((B, k), np.float32)
    else:
        ids = torch.empty((B, k), dtype=torch.int32, device=DEV)
        sc = torch.empty((B, k), dtype=torch.float32, device=DEV)
    before = ix.profile_read()
    ebr.score_topk(ix, cross, qs, ids, sc, io=io)
    after = ix.profile_read()
    assert after.batched - before.batched == B, "the batched path did not run"
    assert after.recomputed - before.recomputed == 0
    if not host:
        ids = ids.cpu().numpy().view(np.uint32)
        sc = sc.cpu().numpy()
    refs = _history_refs(w, [(p if p is not None else np.arange(w.vocab_u.size + 1,
                                                                  dtype=np.uint32), v)
                             for p, v in hs], post)
    for b, (p, v) in enumerate(hs):
        ref, tol = refs[b]
        assert recall(ids[b], ref, tol, k) == 1.0, "user %d" % b
        check_topk(ids[b], sc[b], ref, tol, k)


@pytest.mark.parametrize("io", [ebr.IO_DEVICE, ebr.IO_HOST])
def test_batched_multi_valued_bad_offsets(io):
    """Offsets that do not end at n_user_vals, or decrease, fail the batch
    with EBR_EDATA (host requests: found on the host; device requests: by
    the staging kernel), and the index stays usable."""
    from paper_2511_22460_gb300.datagen import user_histories
    B, n, k = 4, 20_000, 50
    w = make_workload("serve_bf16_5m", n_ads=n, seed=22, batch=B)
    post = w.postings()
    ix = ebr.build_index(w.n_ads, w.n_keys, *post, w.emb, dtype="bf16")
    cross = ebr.cross_from_workload(w)
    hs = user_histories(w, B, max_len=4, seed=6)
    host = io == ebr.IO_HOST
    conv = (lambda a: np.ascontiguousarray(a)) if host else dev
    ids = np.empty((B, k), np.uint32) if host else torch.empty((B, k), dtype=torch.int32,
                                                               device=DEV)
    sc = np.empty((B, k), np.float32) if host else torch.empty((B, k), dtype=torch.float32,
                                                               device=DEV)
    p2 = hs[2][0]
    bad_end = p2.copy()
    bad_end[-1] += 1
    bad_order = p2.copy()
    bad_order[1] = p2[-1] + 5
    for bad in (bad_end, bad_order):
        qs = [ebr.Query(h_u=conv(w.h_u[b]), k=k, user_vals=conv(hs[b][1]),
                        user_ptr=conv(bad if b == 2 else hs[b][0])) for b in range(B)]
        with pytest.raises(ebr.EbrError) as e:
            ebr.score_topk(ix, cross, qs, ids, sc, io=io)
        assert e.value.code == ebr.EBR_EDATA
    qs = [ebr.Query(h_u=conv(w.h_u[b]), k=k, user_vals=conv(hs[b][1]), user_ptr=conv(hs[b][0]))
          for b in range(B)]
    ebr.score_topk(ix, cross, qs, ids, sc, io=io)
    if not host:
        ids = ids.cpu().numpy().view(np.uint32)
        sc = sc.cpu().numpy()
    for b, (ref, tol) in enumerate(_history_refs(w, hs, post)):
        check_topk(ids[b], sc[b], ref, tol, k)
