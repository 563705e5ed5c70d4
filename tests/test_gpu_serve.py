"""The request server: every result is the same alone and in the mix, memory
admission holds, and failures stay local (GPU).

Failures are made on the host (an oversized request, an invalid one, a client
that never releases its outputs); nothing here faults or stalls the GPU.
"""
import numpy as np
import pytest

import oracle as O
from paper_2309_16682_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vmt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_16682_gb300 as m
    from paper_2309_16682_gb300 import build
    build.build()
    m.lib()
    return m


def _alone(vmt, variant, lanes, dtype, seed, jump, n):
    g = vmt.VGenerator(variant, lanes, [seed], [jump])
    t = g.generate(n, dtype)
    if t.dtype == torch.uint32:
        return t.cpu().view(torch.int32).numpy().view(np.uint32)[0]
    if t.dtype == torch.uint64:
        return t.cpu().view(torch.int64).numpy().view(np.uint64)[0]
    return t.cpu().numpy()[0]


def test_mix_equals_alone(vmt):
    r = I.splitmix64(2024, 40 * 4).reshape(40, 4)
    kinds = [("mt32", "u32"), ("mt32", "f32"), ("mt64", "u64"), ("mt64", "f64"), ("sfmt", "u32"), ("sfmt", "f64")]
    sizes = [1, 2, 999, 10000, 123457, 624 * 16 + 3]
    srv = vmt.Server(state_budget=1 << 30, output_budget=1 << 30, max_batch=64)
    reqs = []
    for i in range(40):
        variant, dtype = kinds[int(r[i, 0] % np.uint64(len(kinds)))]
        lanes = [2, 4, 8, 16][int(r[i, 1] % np.uint64(4))]
        n = sizes[i % len(sizes)]
        seed, jump = int(r[i, 2]), int(r[i, 3])
        reqs.append((srv.submit(variant, lanes, dtype, seed, jump, n), variant, lanes, dtype, seed, jump, n))
    for rid, variant, lanes, dtype, seed, jump, n in reqs:
        srv.wait(rid)
        got = srv.copy(rid, dtype)
        ref = _alone(vmt, variant, lanes, dtype, seed, jump, n)
        assert np.array_equal(got, ref), (variant, lanes, dtype, n)
        st, ptr, nb, lat = srv.poll(rid)
        assert st == vmt.SERVER_DONE and lat >= 0
        srv.release(rid)
    s = srv.stats()
    assert s["completed"] == 40 and s["failed"] == 0 and s["output_bytes_in_use"] == 0
    srv.close()


def test_batched_calls_equal_alone(vmt):
    """submit_many / next_done_many / release_many: the same outputs as each
    request alone, every id completed once, and the latencies server-stamped."""
    r = I.splitmix64(77, 30 * 4).reshape(30, 4)
    kinds = [("mt32", "u32"), ("mt64", "u64"), ("sfmt", "u32"), ("mt32", "f64")]
    rows = []
    for i in range(30):
        variant, dtype = kinds[int(r[i, 0] % np.uint64(len(kinds)))]
        lanes = [2, 4, 8, 16][int(r[i, 1] % np.uint64(4))]
        rows.append((variant, lanes, dtype, int(r[i, 2]), int(r[i, 3]), [1, 777, 12345, 70000][i % 4]))
    srv = vmt.Server(state_budget=1 << 30, output_budget=1 << 30, max_batch=16)
    carr = vmt.Server.requests(rows)
    ids = np.concatenate([srv.submit_many(carr, 0, 11), srv.submit_many(carr, 11, 19)])
    assert len(set(ids.tolist())) == 30
    seen = {}
    while len(seen) < 30:
        got_ids, st, lat = srv.next_done_many(2_000_000, 7)
        assert len(got_ids) > 0
        for rid, s_, l_ in zip(got_ids.tolist(), st.tolist(), lat.tolist()):
            assert rid not in seen and s_ == vmt.SERVER_DONE and l_ >= 0
            seen[rid] = l_
    for rid, (variant, lanes, dtype, seed, jump, n) in zip(ids.tolist(), rows):
        assert np.array_equal(srv.copy(rid, dtype), _alone(vmt, variant, lanes, dtype, seed, jump, n))
    srv.release_many(ids)
    assert srv.stats()["output_bytes_in_use"] == 0
    bad = vmt.Server.requests([("mt64", 4, "u32", 1, 0, 10)])   # u32 from MT19937-64 is refused
    with pytest.raises(vmt.VMTError):
        srv.submit_many(bad, 0, 1)
    srv.close()


def test_mix_matches_oracle_for_a_few(vmt, oracle_polys):
    srv = vmt.Server(state_budget=1 << 28, output_budget=1 << 28, max_batch=8)
    cases = [("mt32", 4, "u32", 11, 1 << 40, 5000), ("sfmt", 4, "u32", 12, 3, 3000), ("mt64", 8, "u64", 13, 77, 4000)]
    ids = [srv.submit(*c) for c in cases]
    for rid, (variant, lanes, dtype, seed, jump, n) in zip(ids, cases):
        srv.wait(rid)
        got = srv.copy(rid, dtype)
        v = O.VARIANTS[variant]
        ref = O.vstream(v, lanes, seed, n, dtype, d=jump)
        assert np.array_equal(got, ref)
        srv.release(rid)
    srv.close()


def test_admission_never_exceeds_budgets(vmt):
    budget = 4 << 20
    srv = vmt.Server(state_budget=1 << 30, output_budget=budget, max_batch=16)
    ids = [srv.submit("mt32", 8, "u32", s, 0, 250_000) for s in range(12)]   # 1 MB each
    for rid in ids:
        srv.wait(rid)
        srv.release(rid)
    s = srv.stats()
    assert s["completed"] == 12 and s["peak_output_bytes"] <= budget and s["output_bytes_in_use"] == 0
    srv.close()


def test_oversized_and_invalid_requests_fail_alone(vmt):
    srv = vmt.Server(state_budget=1 << 30, output_budget=1 << 20, max_batch=16)
    big = srv.submit("mt32", 4, "u32", 1, 0, 1_000_000)          # 4 MB > budget
    ok = srv.submit("mt32", 4, "u32", 2, 0, 1000)
    with pytest.raises(vmt.VMTError) as ei:
        srv.wait(big)
    assert ei.value.code == vmt.VMT_ENOMEM
    srv.wait(ok)
    srv.release(ok)
    srv.release(big)
    with pytest.raises(vmt.VMTError) as ei:
        srv.submit("mt64", 4, "u32", 1, 0, 10)                     # u32 is not defined for MT19937-64
    assert ei.value.code == vmt.VMT_EINVAL
    srv.close()


def test_stalled_consumer_blocks_admission_then_recovers(vmt):
    srv = vmt.Server(state_budget=1 << 30, output_budget=(2 << 20) + 16, max_batch=16)
    a = srv.submit("sfmt", 4, "u32", 1, 0, 262_144)   # 1 MiB each
    b = srv.submit("sfmt", 4, "u32", 2, 0, 262_144)
    c = srv.submit("sfmt", 4, "u32", 3, 0, 262_144)
    srv.wait(a)
    srv.wait(b)
    with pytest.raises(vmt.VMTError) as ei:            # nobody released a or b yet
        srv.wait(c, timeout_ms=300)
    assert ei.value.code == vmt.VMT_ETIMEOUT
    assert srv.poll(c)[0] == vmt.SERVER_QUEUED
    srv.release(a)
    srv.wait(c)
    srv.release(b)
    srv.release(c)
    srv.close()


def test_long_requests_split_into_chunks_equal_alone(vmt):
    # requests longer than one chunk run as several generators, chunk c's
    # lanes jumped to the chunk's first word; the stream must not change
    srv = vmt.Server(state_budget=1 << 30, output_budget=1 << 30, max_batch=16)
    cases = [("mt32", 4, "u32", 31, 0, 3_000_000),        # 2 chunks
             ("mt32", 1, "f32", 32, 5, 5_000_000),        # 8 chunks, ragged tail
             ("mt64", 4, "f64", 33, 1 << 33, 3_000_000),  # 3 chunks
             ("sfmt", 2, "f64", 34, 9, 2_000_000),        # 4 chunks of 32-bit word pairs
             ("mt32", 2, "u32", 35, 0, 1000)]             # short one in the same batch
    ids = [srv.submit(*c) for c in cases]
    for rid, c in zip(ids, cases):
        srv.wait(rid)
        got = srv.copy(rid, c[2])
        assert np.array_equal(got, _alone(vmt, *c)), c
        srv.release(rid)
    srv.close()


def test_chunk_boundary_matches_oracle(vmt, oracle_polys):
    # the words on both sides of the first chunk boundary, against the oracle
    lanes = 4
    C = 1024 * lanes * 624
    srv = vmt.Server(state_budget=1 << 28, output_budget=1 << 28, max_batch=4)
    rid = srv.submit("mt32", lanes, "u32", 41, 3, C + 700)
    srv.wait(rid)
    got = srv.copy(rid, "u32")
    ref = O.vstream(O.VARIANTS["mt32"], lanes, 41, 1400, "u32", start_word=C - 700, d=3)
    assert np.array_equal(got[C - 700:], ref)
    srv.release(rid)
    srv.close()


def test_reserved_pool_and_counters(vmt):
    srv = vmt.Server(state_budget=1 << 26, output_budget=1 << 28, max_batch=8, reserve=True)
    ids = [srv.submit("mt32", 8, "u32", s, s, 300_000) for s in range(6)]
    for rid, s in zip(ids, range(6)):
        srv.wait(rid)
        assert np.array_equal(srv.copy(rid, "u32"), _alone(vmt, "mt32", 8, "u32", s, s, 300_000))
        srv.release(rid)
    st = srv.stats()
    assert st["completed"] == 6 and st["batches"] >= 1
    assert st["host_launch_s"] > 0 and 0 < st["init_gpu_s"] <= st["batch_gpu_s"]
    srv.close()
    free, _ = torch.cuda.mem_get_info()
    with pytest.raises(vmt.VMTError) as ei:   # budgets larger than the device: creation fails cleanly
        vmt.Server(state_budget=1 << 30, output_budget=4 * free, max_batch=8, reserve=True)
    assert ei.value.code == vmt.VMT_ENOMEM


def test_cancel_queued_request(vmt):
    # a small output budget keeps the later requests (too long for the express
    # slot) queued behind the first
    srv = vmt.Server(state_budget=1 << 30, output_budget=(4 << 20) + 64, max_batch=16)
    a = srv.submit("mt32", 4, "u32", 1, 0, 1 << 20)     # 4 MiB: the whole budget
    b = srv.submit("mt32", 4, "u32", 2, 0, 20000)
    c = srv.submit("mt32", 4, "u32", 3, 0, 20000)
    srv.wait(a)
    assert srv.poll(c)[0] == vmt.SERVER_QUEUED            # a is not released yet
    srv.cancel(c)
    with pytest.raises(vmt.VMTError) as ei:
        srv.wait(c)
    assert ei.value.code == vmt.VMT_ECANCELED
    with pytest.raises(vmt.VMTError) as ei:
        srv.cancel(a)                                     # finished: cannot be withdrawn
    assert ei.value.code == vmt.VMT_EBUSY
    srv.release(a)
    srv.wait(b)
    assert np.array_equal(srv.copy(b, "u32"), _alone(vmt, "mt32", 4, "u32", 2, 0, 20000))
    srv.release(b)
    srv.release(c)
    st = srv.stats()
    assert st["cancelled"] == 1 and st["completed"] == 2
    srv.close()


def test_injected_allocation_failures_fail_alone(vmt):
    srv = vmt.Server(state_budget=1 << 30, output_budget=1 << 30, max_batch=64)
    srv.inject_alloc_failures(2)
    cases = [("mt32", 4, "u32", 50 + i, i, 20000 + 7 * i) for i in range(6)]
    ids = [srv.submit(*c) for c in cases]
    failed = 0
    for rid, c in zip(ids, cases):
        try:
            srv.wait(rid)
        except vmt.VMTError as e:
            assert e.code == vmt.VMT_ENOMEM
            failed += 1
        else:
            assert np.array_equal(srv.copy(rid, "u32"), _alone(vmt, *c))
        srv.release(rid)
    assert failed == 2
    rid = srv.submit("mt32", 4, "u32", 99, 0, 5000)      # the server goes on
    srv.wait(rid)
    srv.release(rid)
    srv.close()


def test_device_wait_gives_up_with_status(vmt):
    # a bounded wait on a barrier nothing arrives at ends with a status, and
    # the context stays usable (no trap, no hang)
    rc, elapsed = vmt.selftest_wait(2_000_000)            # 2 ms limit
    assert rc == vmt.VMT_ETIMEOUT
    assert 2_000_000 <= elapsed < 1_000_000_000
    assert vmt.device_status() == 0                       # generation kernels untouched
    g = vmt.VGenerator("mt32", 4, [1])
    assert g.generate(100, "u32").numel() == 100


def test_completion_queue_reports_each_request_once(vmt):
    srv = vmt.Server(state_budget=1 << 30, output_budget=1 << 30, max_batch=8)
    assert srv.next_done(1000) is None                    # nothing submitted yet
    sizes = [50_000, 10, 3_000_000, 777, 120_000, 1, 64_000, 5]
    ids = [srv.submit("mt64", 4, "u64", 10 + i, 0, n) for i, n in enumerate(sizes)]
    bad = srv.submit("mt32", 4, "u32", 1, 0, 300_000_000)  # 1.2 GB > budget: fails at admission
    seen = []
    while len(seen) < len(ids) + 1:
        rid = srv.next_done(5_000_000)
        assert rid is not None
        seen.append(rid)
        st = srv.poll(rid)[0]
        assert st == vmt.SERVER_DONE or (rid == bad and st == vmt.VMT_ENOMEM)
        srv.release(rid)
    assert sorted(seen) == sorted(ids + [bad])
    assert srv.next_done(1000) is None
    srv.close()


def test_large_batch_uses_longer_chunks_and_stays_exact(vmt):
    # one batch writing several GB: chunks span several table steps (c * m)
    srv = vmt.Server(state_budget=1 << 30, output_budget=12 << 30, max_batch=64)
    cases = [("mt32", 2, "u32", 70 + i, i, 250_000_000 + 1237 * i) for i in range(8)]   # 1 GB each
    ids = [srv.submit(*c) for c in cases]
    for k, (rid, c) in enumerate(zip(ids, cases)):
        srv.wait(rid)
        if k in (0, 5):                                    # full comparison for two of them
            assert np.array_equal(srv.copy(rid, "u32"), _alone(vmt, *c)), c
        srv.release(rid)
    srv.close()


def test_small_requests_use_the_express_budget(vmt):
    # a (4 MiB) is done but not released; b (8 MiB) then waits for the output
    # budget (10 MiB).  Small requests go ahead of b on the express budget
    # (10 MiB / 16 = 640 KiB) without taking output memory b waits for; once
    # that budget is full the next small one queues like any other request.
    srv = vmt.Server(state_budget=1 << 30, output_budget=10 << 20, max_batch=16)
    a = srv.submit("mt32", 4, "u32", 1, 0, 1 << 20)
    srv.wait(a)
    b = srv.submit("mt32", 4, "u32", 2, 0, 2 << 20)
    small = [srv.submit("mt32", 4, "u32", 3 + i, 0, 16384) for i in range(10)]   # 64 KiB each
    for rid in small:
        srv.wait(rid)
    assert srv.poll(b)[0] == vmt.SERVER_QUEUED
    st = srv.stats()
    assert st["output_bytes_in_use"] == (4 << 20) + 10 * (64 << 10)
    extra = srv.submit("mt32", 4, "u32", 99, 0, 1000)      # express budget full, main budget held by b
    with pytest.raises(vmt.VMTError) as ei:
        srv.wait(extra, timeout_ms=300)
    assert ei.value.code == vmt.VMT_ETIMEOUT
    srv.release(small[0])                                 # frees express room: extra goes ahead of b
    srv.wait(extra)
    assert srv.poll(b)[0] == vmt.SERVER_QUEUED
    srv.release(a)
    srv.wait(b)
    assert np.array_equal(srv.copy(small[3], "u32"), _alone(vmt, "mt32", 4, "u32", 6, 0, 16384))
    assert np.array_equal(srv.copy(extra, "u32"), _alone(vmt, "mt32", 4, "u32", 99, 0, 1000))
    for rid in small[1:] + [b, extra]:
        srv.release(rid)
    assert srv.stats()["output_bytes_in_use"] == 0
    srv.close()


def test_small_request_goes_ahead_of_long_ones(vmt):
    # one request per batch: four long requests (4 GiB each) take the four
    # regular slots and a fifth waits for one of them; a small request
    # submitted after it runs in the express slot and finishes first
    srv = vmt.Server(state_budget=2 << 30, output_budget=32 << 30, max_batch=1)
    n = (1 << 30) - 1
    longs = [srv.submit("mt32", 16, "u32", 100 + i, 0, n) for i in range(5)]
    small = srv.submit("sfmt", 8, "u32", 7, 3, 5000)
    order = []
    while len(order) < 6:
        rid = srv.next_done(30_000_000)
        assert rid is not None
        assert srv.poll(rid)[0] == vmt.SERVER_DONE
        order.append(rid)
    assert order.index(small) < order.index(longs[4])
    assert np.array_equal(srv.copy(small, "u32"), _alone(vmt, "sfmt", 8, "u32", 7, 3, 5000))
    for rid in order:
        srv.release(rid)
    srv.close()


def test_small_requests_run_only_in_express_batches_one_variant_each(vmt):
    # Long requests keep the regular slots busy; small requests of all three
    # variants, submitted together, all run in express batches (never in a
    # regular batch), an express batch holds one variant only (so at least
    # three of them), and every output equals the request run alone.
    srv = vmt.Server(state_budget=2 << 30, output_budget=32 << 30, max_batch=64)
    st0 = srv.stats()
    n = (1 << 30) - 1
    longs = [srv.submit("mt32", 16, "u32", 200 + i, 0, n) for i in range(5)]
    cases = [("mt32", 8, "u32", 11, 5, 3000), ("mt64", 4, "u64", 12, 6, 2000), ("sfmt", 16, "f32", 13, 7, 16384),
             ("mt32", 16, "f32", 14, 0, 100), ("sfmt", 4, "u32", 15, 2**40 + 9, 4096), ("mt64", 16, "f64", 16, 3, 16384)]
    small = srv.submit_many(vmt.Server.requests(cases), 0, len(cases)).tolist()
    for rid in longs + small:
        srv.wait(rid, timeout_ms=60_000)
        assert srv.poll(rid)[0] == vmt.SERVER_DONE
    st1 = srv.stats()
    assert st1["express_completed"] - st0["express_completed"] == len(small)
    assert st1["express_batches"] - st0["express_batches"] >= 3
    for rid, c in zip(small, cases):
        assert np.array_equal(srv.copy(rid, c[2]), _alone(vmt, *c)), c
    for rid in longs + small:
        srv.release(rid)
    srv.close()
