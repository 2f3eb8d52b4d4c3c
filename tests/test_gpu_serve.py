"""GPU tests of the continuous-batching request loop: each result is the same
alone and in a mix of concurrent requests (and matches the FP64 oracle),
admission by the HBM budget, ticket semantics and the per-request path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from gpu_util import bitmap_to_mask, check_topk, recall, ref_scores  # noqa: E402
from paper_2511_22460_gb300 import ebr  # noqa: E402
from paper_2511_22460_gb300.datagen import make_filters, make_workload, refreshed  # noqa: E402

pytestmark = pytest.mark.gpu


def _setup(n, B, dtype="bf16", seed=21):
    w = make_workload("serve_bf16_5m", n_ads=n, seed=seed, batch=B)
    pk, pa = w.postings(shuffle=True)
    ix = ebr.build_index(w.n_ads, w.n_keys, pk, pa, w.emb, dtype=dtype)
    cross = ebr.cross_from_workload(w)
    return w, (pk, pa), ix, cross


def _same_result(a, b, ref, tol, k, mask=None):
    """Two results of one request agree: equal id sets except for ties within
    tolerance at the K-th oracle score, scores within tolerance."""
    ids_a, sc_a = a
    ids_b, sc_b = b
    elig = np.ones(ref.size, bool) if mask is None else mask
    take = min(k, int(elig.sum()))
    r = np.where(elig, ref, -np.inf)
    kth = np.sort(r)[::-1][take - 1]
    diff = set(ids_a[:take].tolist()) ^ set(ids_b[:take].tolist())
    for x in diff:
        assert abs(ref[x] - kth) <= 2 * tol[x], "id %d differs and is not a tie" % x
    common = np.intersect1d(ids_a[:take], ids_b[:take])
    pa = {int(i): s for i, s in zip(ids_a[:take], sc_a[:take])}
    pb = {int(i): s for i, s in zip(ids_b[:take], sc_b[:take])}
    for i in common:
        assert abs(float(pa[int(i)]) - float(pb[int(i)])) <= 2 * tol[i]


@pytest.mark.parametrize("host_driven", [False, True])
def test_alone_and_in_a_mix_give_the_same_result(host_driven):
    """Default: the device-resident loop; host_driven: two pipelines."""
    n, B = 60_000, 40
    w, post, ix, cross = _setup(n, B)
    rng = np.random.default_rng(3)
    ks = [int(x) for x in rng.choice([100, 500, 1000], size=B)]
    fl = make_filters(rng, n, B, (0.01, 1.0))
    filt = [fl[b] if b % 2 else None for b in range(B)]
    srv = ebr.Server(ix, cross, max_batch=64, k_max=1000, host_driven=host_driven)
    try:
        probe = [0, 7, 13, 30]
        alone = {}
        for b in probe:  # one at a time: the single-request scan
            t = srv.submit(w.h_u[b], w.users[b], ks[b], filt[b])
            alone[b] = srv.wait(t, ks[b])
        # all at once: batched scans mixing users with different K and filters
        tickets = [srv.submit(w.h_u[b], w.users[b], ks[b], filt[b]) for b in range(B)]
        assert all(t is not None for t in tickets)
        mixed = {b: srv.wait(t, ks[b]) for b, t in enumerate(tickets)}
        st = srv.stats()
        assert st.completed == B + len(probe) and st.failed == 0
        assert st.batches < B + len(probe), "requests were never batched"
        assert (st.loop_launches > 0) == (not host_driven)
        prof = ix.profile_read()
        assert prof.batched > 0 and prof.recomputed == 0, "batched users were recomputed"
        for b in probe + [1, 2, 5, 39]:
            ref, tol = ref_scores(w, b, post)
            mask = None if filt[b] is None else bitmap_to_mask(filt[b], n)
            ids, sc = mixed[b]
            assert recall(ids, ref, tol, ks[b], mask) == 1.0
            check_topk(ids, sc, ref, tol, ks[b], mask)
            if b in alone:
                _same_result(alone[b], mixed[b], ref, tol, ks[b], mask)
    finally:
        srv.close()


def test_admission_by_hbm_budget_and_slot_reuse():
    n = 20_000
    w, post, ix, cross = _setup(n, 12)
    # the budget decides: far too small -> no server at all
    with pytest.raises(ebr.EbrError) as e:
        ebr.Server(ix, cross, hbm_budget=1 << 20, max_batch=8, k_max=100)
    assert e.value.code == ebr.EBR_ENOMEM
    # measure what 8-user pipelines and one slot cost, then allow 8 slots
    probe = ebr.Server(ix, cross, max_batch=8, max_slots=16, k_max=100)
    st = probe.stats()
    pipes = st.device_bytes - st.max_slots * st.slot_bytes
    probe.close()
    budget = pipes + 8 * st.slot_bytes + st.slot_bytes // 2
    srv = ebr.Server(ix, cross, hbm_budget=budget, max_batch=8, k_max=100)
    try:
        st = srv.stats()
        assert st.max_slots == 8 and st.max_batch == 8
        assert st.device_bytes <= budget
        tickets = [srv.submit(w.h_u[b], w.users[b], 50) for b in range(8)]
        assert all(t is not None for t in tickets)
        assert srv.submit(w.h_u[8], w.users[8], 50) is None  # refused: no free slot
        assert srv.stats().rejected == 1
        ids, sc = srv.wait(tickets[0], 50)
        t9 = srv.submit(w.h_u[8], w.users[8], 50)  # the retired slot is reused
        assert t9 is not None
        res9 = srv.wait(t9, 50)
        for t in tickets[1:]:
            srv.wait(t, 50)
        ref, tol = ref_scores(w, 8, post)
        check_topk(res9[0], res9[1], ref, tol, 50)
        # tickets are retired by the poll that returns them
        with pytest.raises(ebr.EbrError) as e:
            srv.poll(tickets[0], 50)
        assert e.value.code == ebr.EBR_EINVAL
    finally:
        srv.close()


def test_submit_rejects_bad_requests():
    w, post, ix, cross = _setup(5_000, 2)
    srv = ebr.Server(ix, cross, max_batch=4, k_max=100)
    try:
        for k in (0, 101):
            with pytest.raises(ebr.EbrError) as e:
                srv.submit(w.h_u[0], w.users[0], k)
            assert e.value.code == ebr.EBR_EINVAL
        bad = w.users[1].copy()
        bad[0] = 1 << 30  # a user value outside its vocabulary: refused at submit
        with pytest.raises(ebr.EbrError) as e:
            srv.submit(w.h_u[1], bad, 10)
        assert e.value.code == ebr.EBR_EINVAL
        t = srv.submit(w.h_u[0], w.users[0], 10)  # the server still serves
        ids, sc = srv.wait(t, 10)
        ref, tol = ref_scores(w, 0, post)
        check_topk(ids, sc, ref, tol, 10)
    finally:
        srv.close()


def test_fp32_index_server_matches_oracle():
    n, B = 30_000, 10
    w, post, ix, cross = _setup(n, B, dtype="f32")
    srv = ebr.Server(ix, cross, max_batch=16, k_max=500)
    try:
        tickets = [srv.submit(w.h_u[b], w.users[b], 200) for b in range(B)]
        res = [srv.wait(t, 200) for t in tickets]
        for b in (0, 4, 9):
            ref, tol = ref_scores(w, b, post)
            check_topk(res[b][0], res[b][1], ref, tol, 200)
        st = srv.stats()
        assert st.completed == B and st.p99_ms >= st.p50_ms > 0
    finally:
        srv.close()


def _check_either(res, refs, k):
    """The result matches the oracle of one of the indexes it may come from."""
    errs = []
    for ref, tol in refs:
        try:
            check_topk(res[0], res[1], ref, tol, k)
            return
        except AssertionError as e:
            errs.append(str(e))
    raise AssertionError("matches no index: %s" % errs)


def test_index_swap_under_serving():
    """The index is rebuilt from an updated feature->ad map and swapped in
    while requests flow: later requests are answered from the new index,
    requests in flight from one of the two, none fails, tickets survive;
    an index of another shape is refused; swapping back works."""
    n, k = 40_000, 200
    w, post, ix, cross = _setup(n, 24)
    w2 = refreshed(w, 0.05, seed=3)
    post2 = w2.postings(shuffle=True)
    srv = ebr.Server(ix, cross, max_batch=16, k_max=k)
    try:
        before = [srv.wait(srv.submit(w.h_u[b], w.users[b], k), k) for b in range(4)]
        mid = [srv.submit(w.h_u[b], w.users[b], k) for b in range(4, 16)]
        ix2 = ebr.build_index(w2.n_ads, w2.n_keys, post2[0], post2[1], w2.emb, dtype="bf16")
        assert srv.swap_index(ix2) is ix
        mid_res = [srv.wait(t, k) for t in mid]
        after = [srv.wait(srv.submit(w.h_u[b], w.users[b], k), k) for b in range(16, 24)]
        st = srv.stats()
        assert st.index_swaps == 1 and st.failed == 0 and st.completed == 24
        old = {b: ref_scores(w, b, post) for b in range(24)}
        new = {b: ref_scores(w2, b, post2) for b in range(24)}
        for b in (0, 3):
            check_topk(before[b][0], before[b][1], *old[b], k)
        for i, b in enumerate(range(4, 16)):
            if i % 3 == 0:
                _check_either(mid_res[i], (old[b], new[b]), k)
        for i, b in enumerate(range(16, 24)):
            check_topk(after[i][0], after[i][1], *new[b], k)
        # the update is visible: some request's top-K changed with the index
        assert any(set(after[i][0].tolist()) != set(
            np.argsort(-old[b][0], kind="stable")[:k].tolist()) for i, b in enumerate(range(16, 24)))
        wo = make_workload("serve_bf16_5m", n_ads=n // 2, seed=5, batch=1)
        pko, pao = wo.postings()
        ixo = ebr.build_index(wo.n_ads, wo.n_keys, pko, pao, wo.emb, dtype="bf16")
        with pytest.raises(ebr.EbrError) as e:
            srv.swap_index(ixo)
        assert e.value.code == ebr.EBR_EINVAL
        assert srv.swap_index(ix) is ix2  # and back
        res = srv.wait(srv.submit(w.h_u[5], w.users[5], k), k)
        check_topk(res[0], res[1], *old[5], k)
        assert srv.stats().index_swaps == 2
        print("\n[swap] rebuild of %d ads (%d postings) on the GPU: %.2f ms"
              % (n, post2[0].size, ix2.info().build_ms))
    finally:
        srv.close()


def test_destroy_while_swap_calls_wait():
    """ebr_server_destroy runs while one swap call is waiting for the worker to
    take the new index and a second waits for the first: destroy waits for
    both to return (each either swapped or reports that the server was
    destroyed) before it frees the server."""
    import threading
    import time
    n, k = 40_000, 100
    w, post, ix, cross = _setup(n, 48)
    w2 = refreshed(w, 0.05, seed=4)
    p2 = w2.postings()
    ix2 = ebr.build_index(w2.n_ads, w2.n_keys, p2[0], p2[1], w2.emb, dtype="bf16")
    for trial in range(3):
        srv = ebr.Server(ix, cross, max_batch=16, k_max=k)
        for b in range(48):  # keep the worker busy so that the swaps have to wait
            srv.submit(w.h_u[b], w.users[b], k)
        h = srv.h
        out, entered = [], threading.Semaphore(0)

        def swap(target):
            entered.release()
            out.append(ebr.ebr_server_swap_index(h, target.h))

        ts = [threading.Thread(target=swap, args=(x,)) for x in (ix2, ix)]
        for t in ts:
            t.start()
        for _ in ts:
            entered.acquire()
        time.sleep(0.05 + 0.02 * trial)  # both calls are inside the server by now
        assert ebr.ebr_server_destroy(h) == ebr.EBR_OK
        srv.h = None
        for t in ts:
            t.join(timeout=30)
        assert not any(t.is_alive() for t in ts)
        assert sorted(out) and all(rc in (ebr.EBR_OK, ebr.EBR_EINVAL) for rc in out), out


@pytest.mark.parametrize("dtype", ["bf16", "fp8e4m3"])
def test_multi_valued_requests_served_alone_and_in_a_mix(dtype):
    """Requests whose user fields hold histories are admitted as slots and
    served in the batched scan beside single-valued ones; each result equals
    the FP64 oracle's and the request served alone."""
    import oracle
    from paper_2511_22460_gb300.datagen import user_histories
    n, B, k = 40_000, 20, 300
    w, post, ix, cross = _setup(n, B, dtype=dtype, seed=23)
    f_u = w.vocab_u.size
    hs = user_histories(w, B, max_len=5, seed=8)
    hs = [(None, w.users[b]) if b % 4 == 0 else hs[b] for b in range(B)]
    srv = ebr.Server(ix, cross, max_batch=32, k_max=1000, max_user_vals=5 * f_u)
    try:
        def submit(b):
            p, v = hs[b]
            return srv.submit(w.h_u[b], np.ascontiguousarray(v), k, user_ptr=p)

        alone = {b: srv.wait(submit(b), k) for b in (1, 4)}
        tickets = [submit(b) for b in range(B)]
        assert all(t is not None for t in tickets)
        mixed = {b: srv.wait(t, k) for b, t in enumerate(tickets)}
        st = srv.stats()
        assert st.failed == 0 and st.batches < B + 2, "requests were never batched"
        prof = ix.profile_read()
        assert prof.batched > 0 and prof.recomputed == 0
        cr = oracle.Cross.from_workload(w)
        for b in range(B):
            p, v = hs[b]
            if p is None:
                p = np.arange(f_u + 1, dtype=np.uint32)
            ref = oracle.score_query_seq(w, w.h_u[b], p, v, cr, post)
            _, cond = oracle.scores_brute_seq(cr, w.h_u[b], w.emb, w.ad_vals, p, v,
                                              with_cond=True)
            tol = oracle.tolerance(ref, cond)
            ids, sc = mixed[b]
            assert recall(ids, ref, tol, k) == 1.0, "request %d" % b
            check_topk(ids, sc, ref, tol, k)
            if b in alone:
                _same_result(alone[b], mixed[b], ref, tol, k)
        # refused at submit: too many values, bad offsets, a value outside its vocabulary
        p1, v1 = hs[1]
        long_p = np.arange(f_u + 1, dtype=np.uint32) * 6
        long_v = np.zeros(int(long_p[-1]), np.uint32)
        bad_end = p1.copy()
        bad_end[-1] += 1
        bad_val = v1.copy()
        bad_val[0] = 1 << 30
        for p, v in ((long_p, long_v), (bad_end, v1), (p1, bad_val)):
            with pytest.raises(ebr.EbrError) as e:
                srv.submit(w.h_u[1], np.ascontiguousarray(v), k, user_ptr=p)
            assert e.value.code == ebr.EBR_EINVAL
    finally:
        srv.close()


def test_device_loop_leaves_when_idle_and_is_relaunched():
    """The device-resident loop leaves after a while without work (its polls
    are bounded) and the next request relaunches it; results stay exact."""
    import time
    n, k = 30_000, 100
    w, post, ix, cross = _setup(n, 6)
    srv = ebr.Server(ix, cross, max_batch=16, k_max=100)
    try:
        t = srv.submit(w.h_u[0], w.users[0], k)
        r0 = srv.wait(t, k)
        time.sleep(0.6)  # longer than the loop's idle exit
        tickets = [srv.submit(w.h_u[b], w.users[b], k) for b in range(1, 6)]
        res = [srv.wait(t, k) for t in tickets]
        st = srv.stats()
        assert st.failed == 0 and st.completed == 6
        assert st.loop_launches >= 2, "the loop was not relaunched after leaving"
        for b, (ids, sc) in enumerate([r0] + res):
            ref, tol = ref_scores(w, b, post)
            assert recall(ids, ref, tol, k) == 1.0
            check_topk(ids, sc, ref, tol, k)
    finally:
        srv.close()
