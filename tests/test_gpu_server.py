"""Serving: queries over resident plans of different circuits arrive while
others run; each result equals the same query run alone (within the
complex64 tolerance) and admission respects the arena budget."""
import time

import numpy as np
import pytest

import tz_inputs as ti
from oracle import statevector as sv
from tests.gpu_util import grid_spec, make_plan, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tz():
    import torch
    import paper_1907_11217_gb300 as tz
    assert torch.cuda.is_available()
    return tz


def test_mix_equals_alone(tz):
    circuits = [(4, 4, 10, 1), (4, 5, 12, 3), (3, 5, 16, 8), (4, 4, 16, 5)]
    plans = []
    for i, (r, c, t, seed) in enumerate(circuits):
        spec = grid_spec(r, c, t, seed)
        # half the plans replay captured graphs on the server's slots (their
        # runs alone, without a stream of their own, launch directly)
        plan, *_ = make_plan(tz, spec, batch_log2=2, slice_bits=2, small_log2=5, max_bitstrings=256,
                             use_graph=(i % 2 == 0))
        plans.append((plan, spec, r * c))
    rng = np.random.default_rng(4)
    queries = []
    for i in range(24):
        j = int(rng.integers(len(plans)))
        plan, spec, n = plans[j]
        nb = int(rng.integers(1, 40))
        bits = ti.random_bitstrings(n, nb, 1000 + i)
        queries.append((j, bits))
    alone = [tz.tz_contract_amplitudes(plans[j][0], bits) for j, bits in queries]
    biggest = max(p[0].stats()["scratch_bytes"] for p in plans)
    srv = tz.tz_server_create(arena_bytes=3 * biggest + 4096, max_inflight=4)
    tickets = []
    for k, (j, bits) in enumerate(queries):      # arrivals spread over time
        tickets.append(srv.submit(plans[j][0], bits))
        if k % 5 == 4:
            time.sleep(0.002)
    results = [None] * len(tickets)
    t0 = time.time()
    while any(r is None for r in results) and time.time() - t0 < 120:
        for k, t in enumerate(tickets):
            if results[k] is None:
                results[k] = srv.poll(t)
    assert all(r is not None for r in results)
    for k, (j, bits) in enumerate(queries):
        n = plans[j][2]
        assert rel_err(results[k], alone[k], n) <= 1e-6
        assert rel_err(results[k], sv.amplitudes(plans[j][1], bits), n) <= 1e-5
    p50, p99, done = srv.latency()
    assert done == len(queries) and 0 < p50 <= p99
    srv.close()


def test_admission_budget(tz):
    spec = grid_spec(4, 4, 10, 1)
    plan, *_ = make_plan(tz, spec)
    need = plan.stats()["scratch_bytes"]
    small = tz.tz_server_create(arena_bytes=max(4096, need // 2), max_inflight=2)
    with pytest.raises(tz.TzError) as e:
        small.submit(plan, ti.random_bitstrings(16, 1, 1))
    assert e.value.code == -3   # TZ_EHBM_ADMIT
    small.close()
    one = tz.tz_server_create(arena_bytes=need + 4096, max_inflight=4, wait_admit=True)
    ts = [one.submit(plan, ti.random_bitstrings(16, 2, s)) for s in range(6)]   # queued, one at a time
    out = {}
    t0 = time.time()
    while len(out) < len(ts) and time.time() - t0 < 60:
        for t in ts:
            if t not in out:
                r = one.poll(t)
                if r is not None:
                    out[t] = r
    assert len(out) == len(ts)
    one.close()


def test_long_query_yields_its_slot(tz):
    """One slot, chunks of one slice: a query over 2^k slices submitted
    first yields the slot between chunks, so short queries submitted after
    it finish before it; every result equals the query run alone (the
    chunks' partial sums stay in the query's scratch part)."""
    big_spec = grid_spec(4, 5, 16, 4)
    big, *_ = make_plan(tz, big_spec, slice_bits=5, small_log2=5, k_max=6, use_graph=True, max_bitstrings=8)
    assert big.stats()["k"] >= 5
    small_spec = grid_spec(4, 4, 10, 1)
    small, *_ = make_plan(tz, small_spec, max_bitstrings=8)
    big_bits = ti.random_bitstrings(20, 3, 21)
    small_bits = [ti.random_bitstrings(16, 2, 30 + i) for i in range(4)]
    alone_big = tz.tz_contract_amplitudes(big, big_bits)
    alone_small = [tz.tz_contract_amplitudes(small, b) for b in small_bits]
    need = max(big.stats()["scratch_bytes"], small.stats()["scratch_bytes"])
    srv = tz.tz_server_create(arena_bytes=6 * need + 65536, max_inflight=1, chunk_ms=1e-6)
    t_big = srv.submit(big, big_bits)
    t_small = [srv.submit(small, b) for b in small_bits]
    order, res = [], {}
    t0 = time.time()
    while len(res) < 5 and time.time() - t0 < 120:
        for t in [t_big] + t_small:
            if t not in res:
                r = srv.poll(t)
                if r is not None:
                    res[t] = r
                    order.append(t)
    assert len(res) == 5
    assert order[-1] == t_big, order
    assert rel_err(res[t_big], alone_big, 20) <= 1e-6
    assert rel_err(res[t_big], sv.amplitudes(big_spec, big_bits), 20) <= 1e-5
    for t, a in zip(t_small, alone_small):
        assert rel_err(res[t], a, 16) <= 1e-6
    srv.close()
