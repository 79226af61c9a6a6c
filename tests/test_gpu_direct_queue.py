"""The direct-step queue launch on the GPU (C ABI; tz_plan_opts.direct_queue):
every run of small direct steps between two products is one persistent
launch whose blocks take work from a device ticket counter and wait,
bounded, for the steps they read. It must give bit-identical amplitudes to one launch per dependency
level (the per-element arithmetic is the same), match the FP64 oracle, leave
its counters ready for the next launch (many groups replayed from one
captured graph, several calls in a row), and report a wait that runs out as
TZ_ETIMEOUT without harm to the next call."""
import json

import numpy as np
import pytest

import tz_inputs as ti
from oracle import statevector as sv
from oracle import tn
from tests.gpu_util import grid_spec, make_plan, rel_err

pytestmark = pytest.mark.gpu
TOL = {"c64": 1e-5, "fp16x3": 1e-5, "tf32x3": 1e-5, "c128": 1e-12}
LIMIT_NS = 20_000_000   # 20 ms instead of 2 s, to keep the timeout test short


@pytest.fixture(scope="module")
def tz():
    import torch
    import paper_1907_11217_gb300 as tz
    assert torch.cuda.is_available()
    return tz


def _queue_items(plan):
    d = json.loads(plan.describe())
    return [it for it in d["var_items"] if it[0] == 1]


@pytest.mark.parametrize("prec", ["c64", "c128", "fp16x3"])
@pytest.mark.parametrize("rows,cols,t,seed,cut,g,small,graph", [
    (4, 5, 16, 4, 4, 2, 10, True),    # sliced, 4 bitstrings per group, replayed graph
    (4, 4, 20, 6, 3, 0, 20, False),   # everything direct: one queue per group
    (5, 5, 14, 2, 2, 3, 8, True),
])
def test_queue_matches_levels_and_statevector(tz, rows, cols, t, seed, cut, g, small, graph, prec):
    spec = grid_spec(rows, cols, t, seed)
    n = rows * cols
    bits = ti.random_bitstrings(n, 19, seed + 70)    # 19 rows: a ragged last chunk
    got = {}
    for levels in (False, True):
        plan, *_ = make_plan(tz, spec, batch_log2=g, slice_bits=cut, small_log2=small, precision=prec,
                             use_graph=graph, direct_queue=not levels, max_bitstrings=32)
        items = _queue_items(plan)
        assert items and all(it[6] == (0 if levels else 1) for it in items)
        # two calls in a row: the counters are left ready for the next launch
        a1 = tz.tz_contract_amplitudes(plan, bits)
        a2 = tz.tz_contract_amplitudes(plan, bits)
        assert np.array_equal(a1, a2)
        got[levels] = a1
        plan.close()
    assert np.array_equal(got[False], got[True])
    assert rel_err(got[False], sv.amplitudes(spec, bits), n) <= TOL[prec]


def test_queue_fewer_launches_same_result_7x7(tz):
    """7x7 depth 1+16+1, 64 bitstrings as one batch, split FP16 with the
    tensor-core products between the queues; checked against the oracle's
    contractor on 8 bitstrings."""
    spec = grid_spec(7, 7, 16, 5)
    bits = ti.random_bitstrings(49, 64, 91)
    res, launches = {}, {}
    for levels in (False, True):
        plan, *_ = make_plan(tz, spec, batch_log2=6, small_log2=12, precision="fp16x3", use_graph=True,
                             direct_queue=not levels, max_bitstrings=64, restarts=8)
        launches[levels] = plan.stats()["n_launches_per_group"]
        res[levels] = tz.tz_contract_amplitudes(plan, bits)
        plan.close()
    assert launches[False] < launches[True]
    assert np.array_equal(res[False], res[True])
    oc = tn.Contractor(spec, max_log2=24)
    ref = np.array([oc.amplitude(x) for x in bits[:8]])
    assert rel_err(res[False][:8], ref, 49) <= TOL["fp16x3"]


@pytest.mark.parametrize("graph", [False, True])
def test_queue_timeout_reports_then_recovers(tz, graph):
    from paper_1907_11217_gb300._lib import TZ_ETIMEOUT
    spec = grid_spec(4, 5, 16, 4)
    bits = ti.random_bitstrings(20, 8, 5)
    plan, *_ = make_plan(tz, spec, batch_log2=1, slice_bits=3, small_log2=10, use_graph=graph, max_bitstrings=8,
                         direct_queue=True)
    ref = sv.amplitudes(spec, bits)
    ok = tz.tz_contract_amplitudes(plan, bits)     # captures the graph before the stall
    assert rel_err(ok, ref, 20) <= TOL["c64"]
    tz.tz_debug_set_wait_limit(LIMIT_NS)
    tz.tz_debug_stall_direct_queue(True)
    try:
        with pytest.raises(tz.TzError) as e:
            tz.tz_contract_amplitudes(plan, bits)
        assert e.value.code == TZ_ETIMEOUT
    finally:
        tz.tz_debug_stall_direct_queue(False)
        tz.tz_debug_set_wait_limit(0)
    again = tz.tz_contract_amplitudes(plan, bits)
    tz.tz_plan_status(plan)
    assert np.array_equal(again, ok)
    plan.close()
