"""Helpers shared by the GPU parity tests (comparison rules, device staging)."""
import numpy as np

import oracle

REL = 1e-5  # relative tolerance of the FP32 path against the FP64 oracle


def ref_scores(w, b=0, postings=None):
    """FP64 oracle scores of request b and the per-ad tolerance."""
    cross = oracle.Cross.from_workload(w)
    s = oracle.score_query(w, b, cross, postings)
    _, cond = oracle.scores_brute(cross, w.h_u[b], w.emb, w.ad_vals, w.users[b], with_cond=True)
    return s, oracle.tolerance(s, cond, REL)


def check_scores(got, ref, tol, what="scores"):
    err = np.abs(got.astype(np.float64) - ref)
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, "%s: %d of %d outside tolerance, worst at %d: got %r ref %r tol %r" % (
        what, bad.size, ref.size, bad[np.argmax(err[bad] / tol[bad])], got[bad[0]], ref[bad[0]],
        tol[bad[0]])


def check_topk(ids, scores, ref, tol, k, filt_mask=None):
    """Top-K ids equal the oracle's except for ties within tolerance."""
    ids = np.asarray(ids).astype(np.int64)
    elig = np.ones(ref.size, bool) if filt_mask is None else filt_mask
    n_elig = int(elig.sum())
    take = min(k, n_elig)
    valid = ids[:take]
    assert np.all(valid >= 0) and np.all(valid < ref.size), "invalid ids"
    assert len(set(valid.tolist())) == take, "duplicate ids"
    assert np.all(elig[valid]), "an id outside the filter"
    if take < k:
        assert np.all(ids[take:] == 0xFFFFFFFF) or np.all(ids[take:] == -1)
    r = np.where(elig, ref, -np.inf)
    order = np.lexsort((np.arange(ref.size), -r))
    kth = r[order[take - 1]]
    # every returned score is right, every clear winner is returned, no clear loser is
    check_scores(scores[:take], ref[valid], tol[valid], "top-K scores")
    must = order[:take][r[order[:take]] > kth + tol[order[:take]]]
    missing = set(must.tolist()) - set(valid.tolist())
    assert not missing, "missing clear winners: %s" % sorted(missing)[:10]
    assert np.all(ref[valid] >= kth - tol[valid]), "returned a clear loser"
    # sorted by score descending
    assert np.all(np.diff(scores[:take].astype(np.float64)) <= 0)
    return take


def recall(ids, ref, tol, k, filt_mask=None):
    """|S_gpu & S_oracle| / K, counting ties within tolerance as hits."""
    elig = np.ones(ref.size, bool) if filt_mask is None else filt_mask
    r = np.where(elig, ref, -np.inf)
    take = min(k, int(elig.sum()))
    order = np.lexsort((np.arange(ref.size), -r))
    kth = r[order[take - 1]]
    ids = np.asarray(ids[:take]).astype(np.int64)
    hit = sum(1 for a in ids if 0 <= a < ref.size and elig[a] and ref[a] >= kth - tol[a])
    return hit / take


def bitmap_to_mask(words, n):
    bits = np.unpackbits(words.view(np.uint8), bitorder="little")[:n]
    return bits.astype(bool)
