"""Open output qubits on the GPU (Sec. 2, Table 1: more amplitudes per
contraction, less time each): a plan that leaves m output qubits open returns,
for every bitstring, the 2^m amplitudes of all assignments of those qubits.
Each is checked against the FP64 oracle's amplitude of the expanded
bitstring, computed one at a time."""
import numpy as np
import pytest

import tz_inputs as ti
from oracle import statevector as sv
from oracle import tn
from tests.gpu_util import expand_open, grid_spec, make_plan, rel_err

pytestmark = pytest.mark.gpu
TOL = {"c64": 1e-5, "tf32x3": 1e-5, "fp16x3": 1e-5, "bf16x3": 3e-5, "c128": 1e-12}


@pytest.fixture(scope="module")
def tz():
    import torch
    import paper_1907_11217_gb300 as tz
    assert torch.cuda.is_available()
    return tz


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("g,slice_bits,open_q", [(0, 0, (0, 7, 13, 19)), (2, 2, (3, 4)), (1, 3, (18,)),
                                                 (0, 2, (0, 1, 2, 5, 6, 9, 10, 11))])
def test_open_qubits_small_vs_statevector(tz, prec, g, slice_bits, open_q):
    """4x5 grid, depth 1+12+1: 6 bitstrings (a ragged last batch for g > 0),
    with and without slicing; every amplitude against the state vector."""
    spec = grid_spec(4, 5, 12, 3)
    bits = ti.random_bitstrings(20, 6, 31)
    plan, *_ = make_plan(tz, spec, batch_log2=g, slice_bits=slice_bits, small_log2=5, precision=prec,
                         open_qubits=open_q)
    got = tz.tz_contract_amplitudes(plan, bits)
    assert got.shape == (6, 1 << len(open_q))
    ref = sv.amplitudes(spec, expand_open(bits, open_q))
    assert rel_err(got.reshape(-1), ref, 20) <= TOL[prec]


def test_open_qubits_multi_block_accumulate(tz):
    """8 open qubits and batches of 32: 2^13 root values per group, so the
    FP64 sum runs over several blocks and the group state advances in a
    launch of its own; 40 bitstrings (a ragged second batch), 10240
    amplitudes against the state vector."""
    spec = grid_spec(4, 4, 10, 1)
    open_q = (1, 2, 4, 7, 8, 11, 13, 14)
    bits = ti.random_bitstrings(16, 40, 5)
    plan, *_ = make_plan(tz, spec, batch_log2=5, small_log2=4, slice_bits=1, open_qubits=open_q, max_bitstrings=64)
    got = tz.tz_contract_amplitudes(plan, bits)
    ref = sv.amplitudes(spec, expand_open(bits, open_q))
    assert rel_err(got.reshape(-1), ref, 16) <= TOL["c64"]


@pytest.fixture(scope="module")
def ref_5x6():
    spec = grid_spec(5, 6, 20, 7)
    open_q = (2, 11, 17, 26)
    bits = ti.random_bitstrings(30, 16, 78)
    c = tn.Contractor(spec, max_log2=24)
    ref = np.array([c.amplitude(x) for x in expand_open(bits, open_q)])
    return spec, open_q, bits, ref


@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3", "bf16x3", "c64"])
def test_open_qubits_tensor_core_5x6(tz, ref_5x6, prec):
    """5x6 grid, depth 1+20+1, 16 bitstrings in one batch, 4 open qubits:
    the open and batch indices make late products large enough for the
    split-precision tcgen05 path; 256 amplitudes against the oracle's
    contractor."""
    spec, open_q, bits, ref = ref_5x6
    plan, *_ = make_plan(tz, spec, batch_log2=4, precision=prec, small_log2=8, restarts=8, seed=3,
                         max_bitstrings=16, open_qubits=open_q)
    plan.profile_enable(True)
    got = tz.tz_contract_amplitudes(plan, bits)
    prof = plan.profile()
    err = rel_err(got.reshape(-1), ref, 30)
    print(f"5x6 d20 open 4 {prec}: max rel err {err:.3e}, tc launches {prof['gemm_tc']['launches']}")
    if prec != "c64":
        assert prof["gemm_tc"]["launches"] > 0
    assert err <= TOL[prec]


def test_open_qubits_device_entry_graph_and_server(tz):
    """The device entry point (graph replay) and a server slot return the
    same 2^m amplitudes per bitstring as the host entry point."""
    import torch
    spec = grid_spec(4, 4, 10, 1)
    open_q = (0, 15, 6)
    bits = ti.random_bitstrings(16, 12, 9)
    stream = torch.cuda.Stream()
    plan, *_ = make_plan(tz, spec, batch_log2=2, slice_bits=2, small_log2=4, use_graph=True, stream=stream,
                         open_qubits=open_q, max_bitstrings=16)
    ref = sv.amplitudes(spec, expand_open(bits, open_q))
    d_bits = torch.from_numpy(bits).cuda()
    d_out = torch.zeros(2 * len(bits) << len(open_q), dtype=torch.float64, device="cuda")
    for _ in range(2):
        d_out.zero_()
        tz.tz_contract_amplitudes_device(plan, d_bits, d_out)
        stream.synchronize()
        assert rel_err(d_out.cpu().numpy().view(np.complex128), ref, 16) <= TOL["c64"]
    host = tz.tz_contract_amplitudes(plan, bits)
    srv = tz.tz_server_create(arena_bytes=2 * plan.stats()["scratch_bytes"] + (1 << 20), max_inflight=2)
    t = srv.submit(plan, bits)
    got = None
    while got is None:
        got = srv.poll(t)
    assert got.shape == host.shape
    np.testing.assert_array_equal(got, host)
