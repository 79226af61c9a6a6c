"""Amplitude parity of the whole path on the GPU (C ABI) against the FP64
oracle (state vector and plain-wire contractor)."""
import os

import numpy as np
import pytest

import tz_inputs as ti
from oracle import statevector as sv
from oracle import tn
from tests.gpu_util import grid_spec, make_plan, rel_err

pytestmark = pytest.mark.gpu
TOL_C64 = 1e-5
TOL_C128 = 1e-12


@pytest.fixture(scope="module")
def tz():
    import torch
    import paper_1907_11217_gb300 as tz
    assert torch.cuda.is_available()
    return tz


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_config1_4x4_depth10_single_bitstring(tz, prec):
    """4x4 grid, depth 1+10+1, seed 1, one bitstring, no slicing."""
    spec = grid_spec(4, 4, 10, 1)
    bits = ti.random_bitstrings(16, 1, 101)
    plan, *_ = make_plan(tz, spec, precision=prec)
    got = tz.tz_contract_amplitudes(plan, bits)
    ref = sv.amplitudes(spec, bits)
    assert rel_err(got, ref, 16) <= (TOL_C64 if prec == "c64" else TOL_C128)


def test_golden_closed_forms(tz):
    path = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")
    for ln in open(path):
        if not ln.strip() or ln.startswith("#"):
            continue
        name, spec, bits, re, im = [f.strip() for f in ln.split("|")]
        spec = spec.replace(";", "\n") + "\n"
        x = np.array([[int(ch) for ch in bits]], dtype=np.uint8)
        plan, *_ = make_plan(tz, spec)
        got = tz.tz_contract_amplitudes(plan, x)[0]
        assert abs(got - complex(float(re), float(im))) <= 1e-6, name


@pytest.mark.parametrize("g", [0, 2, 4])
@pytest.mark.parametrize("small", [20, 4])
def test_batched_bitstrings_ragged(tz, g, small):
    spec = grid_spec(4, 4, 10, 1)
    bits = ti.random_bitstrings(16, 37, 7)   # 37 rows: a ragged last chunk
    plan, *_ = make_plan(tz, spec, batch_log2=g, small_log2=small)
    got = tz.tz_contract_amplitudes(plan, bits)
    assert rel_err(got, sv.amplitudes(spec, bits), 16) <= TOL_C64


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("rows,cols,t,seed,cut,g,small", [
    (4, 4, 10, 1, 2, 0, 3), (4, 5, 12, 3, 3, 1, 5), (4, 5, 16, 4, 4, 2, 6), (4, 4, 20, 6, 3, 0, 20)])
def test_sliced_against_statevector(tz, rows, cols, t, seed, cut, g, small, prec):
    spec = grid_spec(rows, cols, t, seed)
    n = rows * cols
    bits = ti.random_bitstrings(n, 6, seed + 50)
    plan, net, tree, sl = make_plan(tz, spec, batch_log2=g, slice_bits=cut, small_log2=small, precision=prec)
    assert cut <= len(sl) <= 8
    got = tz.tz_contract_amplitudes(plan, bits)
    assert rel_err(got, sv.amplitudes(spec, bits), n) <= (TOL_C64 if prec == "c64" else TOL_C128)


def test_slice_ranges_add_up_and_match_oracle_partials(tz):
    spec = grid_spec(4, 5, 12, 3)
    bits = ti.random_bitstrings(20, 3, 8)
    plan, net, tree, sl = make_plan(tz, spec, slice_bits=3, small_log2=5, k_max=4)
    k = len(sl)
    assert 3 <= k <= 4
    full = tz.tz_contract_amplitudes(plan, bits)
    parts = []
    for s in range(1 << k):
        plan.set_slice_range(s, s + 1)
        parts.append(tz.tz_contract_amplitudes(plan, bits))
    assert rel_err(np.sum(parts, axis=0), full, 20) <= 1e-6
    segs = plan.sliced_segments()
    c = tn.Contractor(spec, sliced=segs)
    for s in (0, (1 << k) - 1, (1 << k) // 3):
        ref = np.array([c.partial(x, s) for x in bits])
        assert rel_err(parts[s], ref, 20) <= TOL_C64


def test_device_entry_point_and_graph(tz):
    import torch
    spec = grid_spec(4, 4, 10, 1)
    bits = ti.random_bitstrings(16, 20, 9)
    stream = torch.cuda.Stream()
    plan, *_ = make_plan(tz, spec, batch_log2=2, slice_bits=2, small_log2=4, use_graph=True, stream=stream)
    d_bits = torch.from_numpy(bits).cuda()
    d_out = torch.zeros(40, dtype=torch.float64, device="cuda")
    for _ in range(2):   # second call replays the captured graph
        d_out.zero_()
        tz.tz_contract_amplitudes_device(plan, d_bits, d_out)
        stream.synchronize()
        got = d_out.cpu().numpy().view(np.complex128)
        assert rel_err(got, sv.amplitudes(spec, bits), 16) <= TOL_C64


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "fp16x3", "c64"])
def test_tensor_core_path_5x6(tz, prec):
    """5x6 grid, depth 1+20+1, a batch of 64 bitstrings contracted together:
    the batch indices make the late tensors large enough that GEMM steps
    with >= 128 rows and >= 8 columns run on the split-precision tcgen05
    product (checked through the per-kernel profile); compared with the
    oracle's plain-wire contractor, one bitstring at a time. TF32x3 and the
    scaled FP16x3 are held to the complex64 bar; the BF16x3 error is measured
    and only sanity-bounded."""
    spec = grid_spec(5, 6, 20, 7)
    bits = ti.random_bitstrings(30, 64, 77)
    plan, *_ = make_plan(tz, spec, batch_log2=6, precision=prec, small_log2=8, restarts=8, seed=3,
                         max_bitstrings=64)
    plan.profile_enable(True)
    got = tz.tz_contract_amplitudes(plan, bits)
    prof = plan.profile()
    c = tn.Contractor(spec, max_log2=24)
    ref = np.array([c.amplitude(x) for x in bits])
    err = rel_err(got, ref, 30)
    print(f"{prec}: max rel err {err:.3e}, tc launches {prof['gemm_tc']['launches']}")
    if prec == "c64":
        assert err <= TOL_C64
        assert prof["gemm_tc"]["launches"] == 0
        assert prof["gemm_simt"]["launches"] + prof["gemm_skinny"]["launches"] > 0
    else:
        assert prof["gemm_tc"]["launches"] > 0
        # bf16x3 measured 9.6e-6 on GB300
        assert err <= (3e-5 if prec == "bf16x3" else TOL_C64)


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("rows,cols,t,seed,g,small", [(5, 5, 20, 11, 4, 5), (6, 6, 16, 3, 0, 6)])
def test_in_place_skinny_steps(tz, rows, cols, t, seed, g, small, prec):
    """Plans whose skinny products read their operands in the producers'
    storage order (gather maps) and write through scatter maps, with the
    remaining operand permutes; against the plain-wire contractor."""
    import json
    spec = grid_spec(rows, cols, t, seed)
    n = rows * cols
    bits = ti.random_bitstrings(n, 1 << g, seed + 5)
    plan, *_ = make_plan(tz, spec, batch_log2=g, small_log2=small, restarts=8, seed=3, max_bitstrings=1 << g,
                         precision=prec)
    d = json.loads(plan.describe())
    assert sum(s["skinny"] for s in d["steps"]) >= 2
    got = tz.tz_contract_amplitudes(plan, bits)
    c = tn.Contractor(spec, max_log2=24)
    ref = np.array([c.amplitude(x) for x in bits])
    assert rel_err(got, ref, n) <= (TOL_C64 if prec == "c64" else TOL_C128)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "fp16x3"])
def test_tensor_core_scatter_epilogue_n_low(tz, prec):
    """7x7 grid, depth 1+16+1, 64 bitstrings as one batch: the plan has a
    tensor-core step whose output layout puts three column (n) bits lowest,
    written through the staged per-warp epilogue; all 64 amplitudes against
    the oracle's contractor."""
    import json
    spec = grid_spec(7, 7, 16, 2)
    bits = ti.random_bitstrings(49, 64, 77)
    c = tz.tz_circuit_from_spec(spec)
    net = tz.tz_network_from_circuit(c, 6)
    tree = tz.tz_path_greedy(net, restarts=16, seed=7, algorithm="elimination", precision="tf32x3")
    plan = tz.tz_plan_create(net, tree, [], precision=prec, max_bitstrings=64)
    steps = json.loads(plan.describe())["steps"]
    assert any(s.get("gemm") and s.get("tc") and not s["row_major"] and s["pn"][:3] == [0, 1, 2] for s in steps)
    plan.bind()
    got = tz.tz_contract_amplitudes(plan, bits)
    oc = tn.Contractor(spec, max_log2=24)
    ref = np.array([oc.amplitude(x) for x in bits])
    err = rel_err(got, ref, 49)
    print(f"grid7x7 d16 batch64 {prec}: max rel err {err:.3e}")
    assert err <= (3e-5 if prec == "bf16x3" else TOL_C64)   # bf16x3 measured 9.3e-6


def test_slice_farm_ledger_resume_on_gpu(tz, tmp_path):
    """The checkpointed slice farm on the GPU path: a run that stops after
    two ranges, then a resumed run, give the amplitudes of one whole run."""
    from paper_1907_11217_gb300 import ledger
    spec = grid_spec(4, 5, 12, 3)
    bits = ti.random_bitstrings(20, 3, 8)
    plan, net, tree, sl = make_plan(tz, spec, slice_bits=4, small_log2=5, k_max=6)
    n_slices = 1 << len(sl)
    assert n_slices >= 16
    key = ledger.job_key(spec=spec, tree=np.asarray(tree.pairs()), segs=[list(s) for s in plan.sliced_segments()],
                         bits=bits, precision="c64", chunk=3)
    f = ledger.plan_range_contractor(tz, plan, bits)
    d = str(tmp_path)
    assert ledger.run_ranges(f, d, key, n_slices, 3, 0, 1, stop_after=2) == 2
    assert ledger.total(d, key, n_slices, 3) is None
    ledger.run_ranges(f, d, key, n_slices, 3, 0, 1)
    got = ledger.total(d, key, n_slices, 3)
    plan.set_slice_range(0, n_slices)
    assert rel_err(got, tz.tz_contract_amplitudes(plan, bits), 20) <= 1e-6
    assert rel_err(got, sv.amplitudes(spec, bits), 20) <= TOL_C64


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
def test_autotuned_plan_matches_oracle(tz, prec):
    """A plan bound with autotune: every tensor-core step gets a timed
    launch choice (pairs of CTAs or single CTAs; K split or not; the
    CUDA-core kernel for small K), recorded in the plan description, and the
    amplitudes still match the oracle."""
    import json
    spec = grid_spec(7, 7, 16, 2)
    bits = ti.random_bitstrings(49, 64, 77)
    net = tz.tz_network_from_circuit(tz.tz_circuit_from_spec(spec), 6)
    tree = tz.tz_path_greedy(net, restarts=16, seed=7, algorithm="elimination", precision=prec)
    plan = tz.tz_plan_create(net, tree, [], precision=prec, max_bitstrings=64, autotune=True)
    plan.bind()
    st = plan.stats()
    steps = [s for s in json.loads(plan.describe())["steps"] if s.get("var") and s.get("gemm") and s.get("tc")]
    # small-K CUDA-core steps are tuned too (tiled or stream kernel)
    assert steps and st["n_tuned_steps"] >= len(steps)
    # each step: a tensor-core launch form, or (K <= 32) a CUDA-core kernel
    assert all((s["tc_simt"] == 0 and s["tc_pair"] in (0, 1) and s["tc_ksplit"] in (0, 1)) or
               (s["tc_simt"] in (1, 2) and s["K"] <= 32) for s in steps)
    print(f"{prec}: tuned {len(steps)} steps, pairs chosen for {sum(s['tc_pair'] == 1 for s in steps)}, "
          f"CUDA cores for {sum(s['tc_simt'] for s in steps)}")
    got = tz.tz_contract_amplitudes(plan, bits)
    ref = np.array([tn.Contractor(spec, max_log2=24).amplitude(x) for x in bits[:16]])
    assert rel_err(got[:16], ref, 49) <= (3e-5 if prec == "bf16x3" else TOL_C64)


def test_autotuned_small_k_steps_on_cuda_cores(tz):
    """The autotuner may run a small-K tensor-core step on the CUDA-core
    complex64 kernel, through the output layout chosen for the tensor-core
    product (the test hook forces that choice wherever it is allowed); the
    amplitudes still match the oracle."""
    import json
    spec = grid_spec(7, 7, 16, 2)
    bits = ti.random_bitstrings(49, 64, 77)
    net = tz.tz_network_from_circuit(tz.tz_circuit_from_spec(spec), 6)
    tree = tz.tz_path_greedy(net, restarts=16, seed=7, algorithm="elimination", precision="fp16x3")
    tz.tz_debug_tune_force_simt(True)
    try:
        plan = tz.tz_plan_create(net, tree, [], precision="fp16x3", max_bitstrings=64, autotune=True)
        plan.bind()
    finally:
        tz.tz_debug_tune_force_simt(False)
    steps = [s for s in json.loads(plan.describe())["steps"] if s.get("var") and s.get("gemm") and s.get("tc")]
    small = [s for s in steps if s["K"] <= 32]
    assert small and all(s["tc_simt"] == 1 for s in small)
    assert all(s["tc_simt"] == 0 for s in steps if s["K"] > 32)
    plan.profile_enable(True)
    got = tz.tz_contract_amplitudes(plan, bits)
    prof = plan.profile()
    assert prof["gemm_simt"]["launches"] >= len(small)
    ref = np.array([tn.Contractor(spec, max_log2=24).amplitude(x) for x in bits[:16]])
    assert rel_err(got[:16], ref, 49) <= TOL_C64


def test_autotuner_presets_reproduce_choices(tz):
    """Presets (tz_tune_preset) fill the autotuner's cache: a plan autotuned
    afterwards takes the preset choice for every step it covers, here the
    opposite of what a first plan measured, and its amplitudes match the
    first plan's within the split products' error."""
    import json
    spec = grid_spec(7, 7, 16, 2)
    bits = ti.random_bitstrings(49, 64, 77)
    net = tz.tz_network_from_circuit(tz.tz_circuit_from_spec(spec), 6)
    tree = tz.tz_path_greedy(net, restarts=16, seed=7, algorithm="elimination", precision="fp16x3")
    tz.tz_debug_tune_force_simt(False)   # also clears the cache of earlier tests
    p1 = tz.tz_plan_create(net, tree, [], precision="fp16x3", max_bitstrings=64, autotune=True)
    p1.bind()
    first = [s for s in json.loads(p1.describe())["steps"] if s["var"] and s["tc"]]
    a1 = tz.tz_contract_amplitudes(p1, bits)
    p1.close()
    want = []
    for s in first:
        if s["K"] <= 32:
            simt = 1 if s["tc_simt"] != 1 else 0
            pair = 0
        else:
            simt = 0
            pair = 1 - s["tc_pair"] if s["tc_pair"] in (0, 1) else 0
        want.append((s["batch"], s["M"], s["N"], s["K"], 0 if s["row_major"] else 1, pair, 0, simt))
        tz.tz_tune_preset("fp16x3", *want[-1])
    p2 = tz.tz_plan_create(net, tree, [], precision="fp16x3", max_bitstrings=64, autotune=True)
    p2.bind()
    second = [s for s in json.loads(p2.describe())["steps"] if s["var"] and s["tc"]]
    for s, w in zip(second, want):
        assert s["tc_simt"] == w[7] and (w[7] == 1 or (s["tc_pair"], s["tc_ksplit"]) == (w[5], w[6]))
    a2 = tz.tz_contract_amplitudes(p2, bits)
    p2.close()
    tz.tz_debug_tune_force_simt(False)   # leave no presets behind
    assert rel_err(a2, a1, 49) <= TOL_C64
    with pytest.raises(tz.TzError):
        tz.tz_tune_preset("fp16x3", 1, 128, 64, 64, 0, 0, 0, 1)   # the CUDA-core kernel only for k <= 32


@pytest.mark.parametrize("prec,rows,cols,t,seed,g", [("c64", 7, 7, 16, 2, 6), ("fp16x3", 7, 7, 16, 2, 6),
                                                     ("c64", 6, 6, 18, 9, 4), ("fp16x3", 6, 6, 18, 9, 4),
                                                     ("c64", 5, 5, 24, 3, 2)])
def test_stream_kernel_matches_tiled_kernel(tz, prec, rows, cols, t, seed, g, small=0):
    """The stream kernel for small-K products (K <= 32, outputs written in
    address order) sums in the same order and FP32 arithmetic as the tiled
    CUDA-core kernel: a plan autotuned with every small-K step forced onto it
    gives bit-identical amplitudes to the same plan with those steps forced
    onto the tiled kernel, and both match the oracle."""
    import json
    n = rows * cols
    spec = grid_spec(rows, cols, t, seed)
    bits = ti.random_bitstrings(n, 1 << g, 13)
    net = tz.tz_network_from_circuit(tz.tz_circuit_from_spec(spec), g)
    tree = tz.tz_path_greedy(net, restarts=16, seed=7, algorithm="elimination", precision=prec)
    got, n_stream = {}, 0
    try:
        for force in (1, 2):
            tz.tz_debug_tune_force_simt(force)
            plan = tz.tz_plan_create(net, tree, [], precision=prec, max_bitstrings=1 << g, autotune=True,
                                     small_log2=small)
            plan.bind()
            steps = [s for s in json.loads(plan.describe())["steps"] if s["var"] and s["gemm"]]
            if force == 2:
                n_stream = sum(s["tc_simt"] == 2 for s in steps)
            else:
                assert not any(s["tc_simt"] == 2 for s in steps)
            got[force] = tz.tz_contract_amplitudes(plan, bits)
            plan.close()
    finally:
        tz.tz_debug_tune_force_simt(0)
    assert n_stream > 0
    assert np.array_equal(got[1], got[2])
    ref = np.array([tn.Contractor(spec, max_log2=24).amplitude(x) for x in bits[:8]])
    assert rel_err(got[2][:8], ref, n) <= TOL_C64



@pytest.mark.parametrize("prec,rows,cols,t,seed,g,small", [("c64", 5, 5, 16, 3, 3, 4), ("c64", 6, 6, 14, 2, 2, 6),
                                                           ("fp16x3", 6, 6, 16, 4, 3, 6)])
def test_stream_kernel_short_sums(tz, prec, rows, cols, t, seed, g, small):
    """Plans cut with a low direct-step threshold hold many products with
    K = 1, 2 and 4 (outer products and short sums; K = 1 takes the kernel's
    element loads, since its rows are not 16-byte aligned): forced onto the
    stream kernel they match the tiled kernel bit for bit and the oracle."""
    test_stream_kernel_matches_tiled_kernel(tz, prec, rows, cols, t, seed, g, small)
