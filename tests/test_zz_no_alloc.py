"""The allocation-free scan + top-K entry point against the regular one.

ebr_scan_topk_noalloc serves callers that cannot call cudaMalloc (device
memory owned up front by another allocator, or threads that cannot take
cudaMalloc's implicit device synchronisation); its scratch is a static device
array shared by every call.  This file is collected last so that a run which
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2511_22460_gb300 import ebr  # noqa: E402
from paper_2511_22460_gb300.datagen import make_filters, make_workload  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
REL = 1e-5  # same relative tolerance as the oracle parity tests


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _compare(ids_a, sc_a, ids_b, sc_b, scale):
    """Same top-K up to ties within tolerance; matching ids have matching scores."""
    ids_a = ids_a.view(np.uint32)
    ids_b = ids_b.view(np.uint32)
    tol = REL * scale
    kth = min(sc_a[-1], sc_b[-1])
    common = {int(i): s for i, s in zip(ids_b, sc_b)}
    for i, s in zip(ids_a, sc_a):
        if int(i) in common:
            assert abs(float(s) - float(common[int(i)])) <= tol[i], (i, s, common[int(i)])
        else:
            assert float(s) <= kth + tol[i], "id %d only in one result, score %r" % (i, s)
    assert np.all(np.diff(sc_a.astype(np.float64)) <= 0)


def test_noalloc_matches_score_topk_on_two_calls_in_a_row():
    w = make_workload("single_fp32_2m", n_ads=300_000, batch=2, seed=11)
    pk, pa = w.postings()
    ix = ebr.build_index(w.n_ads, w.n_keys, pk, pa, w.emb)
    cross = ebr.cross_from_workload(w)
    emb = _dev(w.emb)
    filt = make_filters(np.random.default_rng(3), w.n_ads, 1, (0.2, 0.2))[0]
    oc = oracle.Cross.from_workload(w)
    for call, (b, k, f) in enumerate([(0, 500, None), (1, 300, filt)]):
        ref, cond = oracle.scores_brute(oc, w.h_u[b], w.emb, w.ad_vals, w.users[b], with_cond=True)
        scale = np.maximum(np.abs(ref), cond)
        h_u = _dev(w.h_u[b])
        user = _dev(w.users[b])
        q = ebr.Query(h_u=h_u, k=k, user_vals=user, filter=None if f is None else _dev(f))
        ids_ref = torch.empty(k, dtype=torch.int32, device=DEV)
        sc_ref = torch.empty(k, dtype=torch.float32, device=DEV)
        ebr.score_topk(ix, cross, [q], ids_ref, sc_ref)
        wide = torch.empty(w.n_ads, dtype=torch.float32, device=DEV)
        ebr.wide_scores(ix, cross, q, wide)
        ids = torch.full((k,), -7, dtype=torch.int32, device=DEV)
        sc = torch.full((k,), float("nan"), dtype=torch.float32, device=DEV)
        ebr.scan_topk_noalloc(emb, h_u, wide, q.filter, k, ids, sc)
        torch.cuda.synchronize()
        _compare(ids.cpu().numpy(), sc.cpu().numpy(), ids_ref.cpu().numpy(),
                 sc_ref.cpu().numpy(), scale)
        if f is not None:
            bits = np.unpackbits(f.view(np.uint8), bitorder="little")[:w.n_ads]
            assert np.all(bits[ids.cpu().numpy().view(np.uint32)] == 1)


def test_noalloc_rejects_k_beyond_its_scratch():
    emb = torch.zeros((1000, 16), dtype=torch.float32, device=DEV)
    h = torch.zeros(16, dtype=torch.float32, device=DEV)
    ids = torch.empty(2000, dtype=torch.int32, device=DEV)
    sc = torch.empty(2000, dtype=torch.float32, device=DEV)
    with pytest.raises(ValueError):  # the binding refuses it first
        ebr.scan_topk_noalloc(emb, h, None, None, 1025, ids, sc)
    # and so does the C ABI itself
    rc = ebr.ebr_scan_topk_noalloc(emb.data_ptr(), 1000, 16, h.data_ptr(), None, None, 1025,
                                   ids.data_ptr(), sc.data_ptr(), 0, None)
    assert rc == ebr.EBR_EINVAL


def test_noalloc_rejects_a_misaligned_table_on_the_host():
    """A view whose first row is not 16-byte aligned is refused before any
    launch (its rows are staged by bulk copies, which need that alignment)."""
    base = torch.zeros(1000 * 16 + 1, dtype=torch.float32, device=DEV)
    emb = base[1:].view(1000, 16)
    assert emb.data_ptr() % 16 != 0
    h = torch.zeros(16, dtype=torch.float32, device=DEV)
    ids = torch.empty(10, dtype=torch.int32, device=DEV)
    sc = torch.empty(10, dtype=torch.float32, device=DEV)
    with pytest.raises(ebr.EbrError) as e:
        ebr.scan_topk_noalloc(emb, h, None, None, 10, ids, sc)
    assert e.value.code == ebr.EBR_EINVAL
    # the context is untouched: an aligned call right after works
    ebr.scan_topk_noalloc(base[4:4 + 999 * 16].view(999, 16), h, None, None, 10, ids, sc)
    torch.cuda.synchronize()
    assert torch.all(ids >= 0)
