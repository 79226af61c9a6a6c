"""Bounded waits of the tensor-core product, exercised without any fault:
a test switch makes every product's MMA issuer first wait on an on-chip
barrier that nothing arrives at, so that wait runs out after the (shortened)
time limit. The product must stop, drain its copies in flight, free its
tensor memory and report TZ_ETIMEOUT through every path that runs it (the
operation's status, the plan's host and device entry points, the
allocation-free entry point, a server slot), and the next call, with the
switch off, must be correct."""
import ctypes

import numpy as np
import pytest

import tz_inputs as ti
from oracle import pathsum
from tests.gpu_util import grid_spec, make_plan, rel_err

pytestmark = pytest.mark.gpu
LIMIT_NS = 20_000_000   # 20 ms instead of 2 s, to keep the test short


@pytest.fixture(scope="module")
def tz():
    import torch
    import paper_1907_11217_gb300 as tz
    assert torch.cuda.is_available()
    return tz


@pytest.fixture
def stalled(tz):
    """Turn the stall on with a short wait limit; always restore both."""
    tz.tz_debug_set_wait_limit(LIMIT_NS)
    tz.tz_debug_stall_tensor_core(True)
    try:
        yield
    finally:
        tz.tz_debug_stall_tensor_core(False)
        tz.tz_debug_set_wait_limit(0)


def _operands(torch, batch, m, n, k, seed):
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal((batch, m, k)) + 1j * rng.standard_normal((batch, m, k))).astype(np.complex64)
    b = (rng.standard_normal((batch, n, k)) + 1j * rng.standard_normal((batch, n, k))).astype(np.complex64)
    dA = torch.from_numpy(a.view(np.float32).copy()).cuda()
    dB = torch.from_numpy(b.view(np.float32).copy()).cuda()
    ref = np.matmul(a.astype(np.complex128), np.swapaxes(b.astype(np.complex128), 1, 2))
    return dA, dB, ref


def _timeout_code():
    from paper_1907_11217_gb300._lib import TZ_ETIMEOUT
    return TZ_ETIMEOUT


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "fp16x3"])
def test_op_cgemm_reports_timeout_then_recovers(tz, prec):
    import torch
    batch, m, n, k = 2, 256, 48, 512
    dA, dB, ref = _operands(torch, batch, m, n, k, 3)
    C = torch.zeros(batch * m * n * 2, dtype=torch.float32, device="cuda")
    scratch = torch.empty(tz.tz_op_cgemm_scratch_bytes(prec, batch, m, n, k) // 4 + 64, dtype=torch.float32,
                          device="cuda")
    tz.tz_debug_set_wait_limit(LIMIT_NS)
    tz.tz_debug_stall_tensor_core(True)
    try:
        tz.tz_op_cgemm(prec, batch, m, n, k, dA, m * k, dB, n * k, C, m * n, scratch=scratch)
        with pytest.raises(tz.TzError) as e:
            tz.tz_op_cgemm_status(prec, scratch)
        assert e.value.code == _timeout_code()
    finally:
        tz.tz_debug_stall_tensor_core(False)
        tz.tz_debug_set_wait_limit(0)
    # the next call on the same scratch is correct and reports no timeout
    tz.tz_op_cgemm(prec, batch, m, n, k, dA, m * k, dB, n * k, C, m * n, scratch=scratch)
    tz.tz_op_cgemm_status(prec, scratch)
    got = C.cpu().numpy().view(np.complex64).reshape(batch, m, n)
    assert np.max(np.abs(got - ref)) <= 1e-3 * np.max(np.abs(ref))


def test_static_entry_point_reports_timeout_then_recovers(tz, stalled):
    import torch
    from paper_1907_11217_gb300._lib import PRECISIONS, check, lib
    L = lib()
    batch, m, n, k = 1, 256, 32, 256
    dA, dB, ref = _operands(torch, batch, m, n, k, 4)
    C = torch.zeros(batch * m * n * 2, dtype=torch.float32, device="cuda")
    args = (PRECISIONS["tf32x3"], batch, m, n, k, ctypes.c_void_p(dA.data_ptr()), m * k,
            ctypes.c_void_p(dB.data_ptr()), n * k, ctypes.c_void_p(C.data_ptr()), m * n, ctypes.c_void_p(0))
    check(L.tz_op_cgemm_static(*args))
    with pytest.raises(tz.TzError) as e:
        tz.tz_op_cgemm_static_status()
    assert e.value.code == _timeout_code()
    tz.tz_debug_stall_tensor_core(False)
    check(L.tz_op_cgemm_static(*args))
    tz.tz_op_cgemm_static_status()
    got = C.cpu().numpy().view(np.complex64).reshape(batch, m, n)
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))


_REF = {}


def _oracle(spec, bits):
    key = (spec, bits.tobytes())
    if key not in _REF:
        _REF[key] = pathsum.amplitudes(spec, bits)
    return _REF[key]


def _tc_plan(tz, use_graph, stream=None):
    """5x6 depth 1+20+1 with 64 bitstrings as one batch: its largest steps
    run on the tensor-core product (checked in test_gpu_amplitudes)."""
    spec = grid_spec(5, 6, 20, 7)
    bits = ti.random_bitstrings(30, 64, 77)
    plan, *_ = make_plan(tz, spec, batch_log2=6, precision="bf16x3", small_log2=8, restarts=8, seed=3,
                         max_bitstrings=64, use_graph=use_graph, stream=stream)
    return plan, spec, bits


def test_plan_host_entry_point_reports_timeout_then_recovers(tz):
    plan, spec, bits = _tc_plan(tz, use_graph=False)
    tz.tz_debug_set_wait_limit(LIMIT_NS)
    tz.tz_debug_stall_tensor_core(True)
    try:
        with pytest.raises(tz.TzError) as e:
            tz.tz_contract_amplitudes(plan, bits)
        assert e.value.code == _timeout_code()
    finally:
        tz.tz_debug_stall_tensor_core(False)
        tz.tz_debug_set_wait_limit(0)
    got = tz.tz_contract_amplitudes(plan, bits[:8])
    assert rel_err(got, _oracle(spec, bits[:8]), 30) <= 3e-5
    tz.tz_plan_status(plan)


def test_plan_device_entry_point_poisons_and_reports_then_recovers(tz, stalled):
    """Graph replay: the switch is read on the device, so a graph captured
    before the stall also stalls; the amplitudes come back NaN and the
    plan's status reports the timeout."""
    import torch
    stream = torch.cuda.Stream()
    plan, spec, bits = _tc_plan(tz, use_graph=True, stream=stream)
    d_bits = torch.from_numpy(bits).cuda()
    d_out = torch.zeros(2 * len(bits), dtype=torch.float64, device="cuda")
    tz.tz_debug_stall_tensor_core(False)
    tz.tz_contract_amplitudes_device(plan, d_bits, d_out)   # captures the graph
    tz.tz_plan_status(plan)
    tz.tz_debug_stall_tensor_core(True)
    tz.tz_contract_amplitudes_device(plan, d_bits, d_out)   # replays it, stalled
    with pytest.raises(tz.TzError) as e:
        tz.tz_plan_status(plan)
    assert e.value.code == _timeout_code()
    assert np.all(np.isnan(d_out.cpu().numpy()))
    tz.tz_debug_stall_tensor_core(False)
    tz.tz_contract_amplitudes_device(plan, d_bits, d_out)
    tz.tz_plan_status(plan)
    got = d_out.cpu().numpy().view(np.complex128)
    assert rel_err(got[:8], _oracle(spec, bits[:8]), 30) <= 3e-5


def test_server_slot_reports_timeout_then_recovers(tz, stalled):
    import time
    plan, spec, bits = _tc_plan(tz, use_graph=True)
    srv = tz.tz_server_create(arena_bytes=2 * plan.stats()["scratch_bytes"] + 4096, max_inflight=2)

    def wait(ticket):
        t0 = time.time()
        while time.time() - t0 < 60:
            r = srv.poll(ticket)
            if r is not None:
                return r
        raise AssertionError("query did not finish")

    t = srv.submit(plan, bits)
    with pytest.raises(tz.TzError) as e:
        wait(t)
    assert e.value.code == _timeout_code()
    tz.tz_debug_stall_tensor_core(False)
    got = wait(srv.submit(plan, bits[:8]))
    assert rel_err(got, _oracle(spec, bits[:8]), 30) <= 3e-5
    srv.close()
