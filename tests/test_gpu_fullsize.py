"""Full-size checks on the benchmark workloads.

At full depth (1+32+1) the FP64 path-sum oracle reaches single slices: the
GPU's partial amplitudes of sampled slices are compared with it, element by
element, on config 2 (7x7, 2^10 slices) and on the tree bench.py times for
Bristlecone-70, sliced further so that one slice fits the oracle. Beyond
sampled slices, the path is checked by properties that hold at any size, in
the launch configuration bench.py times (bucket-elimination tree, 2^30 cap,
captured graph on a stream):

* slicing is exact: the partial amplitudes of the slices add up to the full
  amplitude (Sec. 1: subtask results add up to the amplitude);
* the amplitude does not depend on the contraction tree or the slicing;
* the FP32-class modes (complex64, split TF32, split BF16, scaled split
  FP16) agree with the complex128 mode (on the same tree in the bench-tree
  and 7x7 tests, on each mode's own tree in the first test); their errors
  against it are printed and held to 1e-5 (complex64, split TF32, split FP16)
  and 3e-5 (split BF16) (the
  complex128 mode itself is pinned to the FP64 oracle to 1e-12 wherever the
  oracle reaches);
* Porter-Thomas (Sec. 2): E[2^n |a|^2] = 1 over random bitstrings.

At full width and reduced depth the oracle is feasible, and those circuits
are compared with it amplitude by amplitude.
"""
import numpy as np
import pytest

import tz_inputs as ti
from oracle import pathsum, tn
from tests.gpu_util import rel_err, rel_err_partial

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def tz():
    import torch
    import paper_1907_11217_gb300 as tz
    assert torch.cuda.is_available()
    return tz


def bris_spec(t, seed):
    return ti.circuit_to_spec(70, ti.generate_circuit(ti.bristlecone(70), t, seed))


def grid_spec(r, c, t, seed):
    return ti.circuit_to_spec(r * c, ti.generate_circuit(ti.grid(r, c), t, seed))


MAX_FLOPS_PER_AMPLITUDE = 1e14   # guard: never start a contraction this test cannot finish


def build(tz, spec, precision, log2_max, batch_log2=0, restarts=64, seed=7, algorithm="elimination", k_max=40,
          max_bitstrings=0, reconfigure=0):
    import torch
    circ = tz.tz_circuit_from_spec(spec)
    net = tz.tz_network_from_circuit(circ, batch_log2)
    tree = tz.tz_path_greedy(net, restarts=restarts, seed=seed, log2_max_intermediate=log2_max,
                             precision=precision, algorithm=algorithm, reconfigure=reconfigure)
    sliced = tz.tz_slice_select(net, tree, log2_max, k_max)
    stream = torch.cuda.Stream()
    plan = tz.tz_plan_create(net, tree, sliced, precision=precision, stream=stream, use_graph=True,
                             max_bitstrings=max_bitstrings or (1 << batch_log2) * 64)
    st = plan.stats()
    assert st["flops_per_group"] * 2.0 ** st["k"] / 2 ** batch_log2 < MAX_FLOPS_PER_AMPLITUDE
    plan.bind()
    return plan, net, tree, sliced


def test_bristlecone70_depth32_properties(tz):
    spec = bris_spec(32, 3)
    bits = ti.random_bitstrings(70, 2, 103)
    # the bench configuration: 2^30 cap (the rotated tree needs no slicing)
    plan, net, tree, sl = build(tz, spec, "tf32x3", 30)
    a = tz.tz_contract_amplitudes(plan, bits)
    # slicing is exact: a 2^27 cap forces slices, whose partial amplitudes
    # add up to the same amplitude
    ps, _, _, sls = build(tz, spec, "tf32x3", 27)
    k = len(sls)
    assert k >= 2
    parts = []
    for s in range(1 << k):
        ps.set_slice_range(s, s + 1)
        parts.append(tz.tz_contract_amplitudes(ps, bits))
    add = rel_err(np.sum(parts, axis=0), a, 70)
    print(f"bristlecone70 d32 slices (k={k}) sum vs unsliced (split TF32): {add:.2e}")
    assert add <= 1e-5   # measured 2.3e-6
    # every mode, each on the tree its own time model picks, against
    # complex128 (one bitstring: the FP64 units of GB300 are slow); the
    # tensor-core modes share one tree, and the same-tree comparison is
    # test_bristlecone70_depth32_bench_tree
    p128, *_ = build(tz, spec, "c128", 30)
    a128 = tz.tz_contract_amplitudes(p128, bits[:1])
    p64, *_ = build(tz, spec, "c64", 30)
    a64 = tz.tz_contract_amplitudes(p64, bits)
    pbf, *_ = build(tz, spec, "bf16x3", 30)
    abf = tz.tz_contract_amplitudes(pbf, bits)
    pfp, *_ = build(tz, spec, "fp16x3", 30)
    afp = tz.tz_contract_amplitudes(pfp, bits)
    errs = {m: rel_err(x[:1], a128, 70) for m, x in (("tf32x3", a), ("c64", a64), ("bf16x3", abf),
                                                      ("fp16x3", afp))}
    print("bristlecone70 d32 errors vs complex128:", {m: f"{e:.2e}" for m, e in errs.items()})
    # measured on GB300: c64 3.3e-6, tf32x3 7.6e-6, bf16x3 9.0e-6
    assert errs["c64"] <= 1e-5 and errs["tf32x3"] <= 1e-5 and errs["bf16x3"] <= 3e-5 and errs["fp16x3"] <= 1e-5
    # another tree (other seed) with a different cap, hence other slices
    p2, _, tree2, sl2 = build(tz, spec, "c64", 29, seed=11, restarts=32)
    assert not np.array_equal(tree.pairs(), tree2.pairs())
    a2 = tz.tz_contract_amplitudes(p2, bits)
    print("bristlecone70 d32 second tree vs first (complex64):", f"{rel_err(a2, a64, 70):.2e}")
    assert rel_err(a2, a64, 70) <= 1e-5
    # Porter-Thomas scale: N p far from 0 and from the tail
    npk = np.abs(a64) ** 2 * 2.0 ** 70
    assert np.all(npk > 1e-6) and np.all(npk < 40)


def test_bristlecone70_depth32_bench_tree(tz):
    """The exact tree bench.py times (16384 restarts, seed 7, 2^30 cap,
    elimination, split-BF16 time model): every FP32-class mode against the
    complex128 mode on that tree and slicing, and the tree's cost."""
    spec = bris_spec(32, 3)
    bits = ti.random_bitstrings(70, 1, 103)
    # the tree search scores with the tensor-core time model, as bench.py does
    plan, net, tree, sl = build(tz, spec, "bf16x3", 30, restarts=16384)
    out, stats = {}, {}
    for prec in ("bf16x3", "c128", "fp16x3", "tf32x3", "c64"):
        if prec != "bf16x3":
            plan = _plan_on(tz, net, tree, sl, prec)
        stats[prec] = plan.stats()
        out[prec] = tz.tz_contract_amplitudes(plan, bits)
        plan.close()
    # the tree bench.py times: about 2.7e12 useful flops, no slicing
    assert stats["bf16x3"]["flops_per_group"] * 2.0 ** stats["bf16x3"]["k"] < 4e12
    errs = {m: rel_err(out[m], out["c128"], 70) for m in ("bf16x3", "fp16x3", "tf32x3", "c64")}
    print("bristlecone70 d32 bench tree, errors vs complex128:", {m: f"{e:.2e}" for m, e in errs.items()})
    # measured on GB300: bf16x3 2.6e-5, fp16x3 5.3e-6, tf32x3 7.4e-6, c64 7.8e-6
    assert errs["c64"] <= 1e-5 and errs["tf32x3"] <= 1e-5 and errs["fp16x3"] <= 1e-5 and errs["bf16x3"] <= 3e-5


def _plan_on(tz, net, tree, sliced, precision):
    import torch
    plan = tz.tz_plan_create(net, tree, sliced, precision=precision, stream=torch.cuda.Stream(), use_graph=True,
                             max_bitstrings=64)
    plan.bind()
    return plan


def test_bristlecone70_depth32_porter_thomas_mean(tz):
    """Sec. 2: N p follows exp(-x); the mean over 32 random bitstrings is
    1 +- 0.18 (one standard deviation)."""
    spec = bris_spec(32, 3)
    bits = ti.random_bitstrings(70, 32, 2024)
    plan, *_ = build(tz, spec, "tf32x3", 30)
    a = tz.tz_contract_amplitudes(plan, bits)
    npk = np.abs(a) ** 2 * 2.0 ** 70
    assert abs(npk.mean() - 1.0) < 0.75


@pytest.mark.parametrize("prec", ["tf32x3", "c64", "bf16x3", "fp16x3", "c128"])
def test_bristlecone70_reduced_depth_vs_oracle(tz, prec):
    """All 70 qubits, depth 1+12+1, sliced (k >= 3), against the oracle."""
    spec = bris_spec(12, 3)
    bits = ti.random_bitstrings(70, 4, 31)
    c = tn.Contractor(spec, max_log2=24)
    ref = np.array([c.amplitude(x) for x in bits])
    circ = tz.tz_circuit_from_spec(spec)
    net = tz.tz_network_from_circuit(circ, 0)
    tree = tz.tz_path_greedy(net, restarts=16, seed=7, algorithm="elimination")
    full = tz.tz_plan_create(net, tree, []).stats()["max_log2"]
    plan, _, _, sl = build(tz, spec, prec, full - 3, k_max=6)
    assert len(sl) >= 3
    got = tz.tz_contract_amplitudes(plan, bits)
    err = rel_err(got, ref, 70)
    print(f"bristlecone70 d12 {prec}: max rel err {err:.2e}")
    # measured on GB300: 2.0e-6 in every FP32-class mode
    assert err <= {"c128": 1e-12, "bf16x3": 6e-6}.get(prec, TOL)


def test_grid7x7_depth32_config2_properties(tz):
    """7x7 depth 1+32+1, 2^10 slices, 64 bitstrings (one group per slice and
    bitstring: for this circuit, batching bitstrings as open indices costs
    more bytes per amplitude than it saves): slice additivity over two halves
    of the slice range, agreement of split-TF32 and complex64, and the
    Porter-Thomas mean."""
    spec = grid_spec(7, 7, 32, 2)
    bits = ti.random_bitstrings(49, 64, 102)
    results = {}
    for prec in ("tf32x3", "c64"):
        circ = tz.tz_circuit_from_spec(spec)
        net = tz.tz_network_from_circuit(circ, 0)
        tree = tz.tz_path_greedy(net, restarts=32, seed=7, log2_max_intermediate=22, precision=prec,
                                 algorithm="elimination")
        import torch
        sl = tz.tz_slice_select(net, tree, 1, 10)
        assert len(sl) == 10
        plan = tz.tz_plan_create(net, tree, sl, precision=prec, stream=torch.cuda.Stream(), use_graph=True,
                                 max_bitstrings=64)
        plan.bind()
        a = tz.tz_contract_amplitudes(plan, bits)
        if prec == "tf32x3":
            plan.set_slice_range(0, 512)
            lo = tz.tz_contract_amplitudes(plan, bits)
            plan.set_slice_range(512, 1024)
            hi = tz.tz_contract_amplitudes(plan, bits)
            assert rel_err(lo + hi, a, 49) <= 1e-6
        results[prec] = a
    agree = rel_err(results["tf32x3"], results["c64"], 49)
    print(f"grid7x7 d32 split TF32 vs complex64: {agree:.2e}")
    assert agree <= 1e-5   # measured 6.8e-6
    npk = np.abs(results["c64"]) ** 2 * 2.0 ** 49
    assert abs(npk.mean() - 1.0) < 0.5


def test_grid7x7_depth32_errors_vs_complex128(tz):
    """7x7 depth 1+32+1 (2^10 slices): the partial amplitude of slices
    [0, 32) for 4 bitstrings in each FP32-class mode against complex128."""
    import torch
    spec = grid_spec(7, 7, 32, 2)
    bits = ti.random_bitstrings(49, 4, 102)
    circ = tz.tz_circuit_from_spec(spec)
    net = tz.tz_network_from_circuit(circ, 0)
    tree = tz.tz_path_greedy(net, restarts=32, seed=7, log2_max_intermediate=22, algorithm="elimination")
    sl = tz.tz_slice_select(net, tree, 1, 10)
    out = {}
    for prec in ("c128", "c64", "tf32x3", "bf16x3", "fp16x3"):
        plan = tz.tz_plan_create(net, tree, sl, precision=prec, stream=torch.cuda.Stream(), use_graph=True,
                                 max_bitstrings=4)
        plan.bind()
        plan.set_slice_range(0, 32)
        out[prec] = tz.tz_contract_amplitudes(plan, bits)
    errs = {m: rel_err(out[m], out["c128"], 49) for m in ("c64", "tf32x3", "bf16x3", "fp16x3")}
    print("grid7x7 d32 (32 slices) errors vs complex128:", {m: f"{e:.2e}" for m, e in errs.items()})
    # measured on GB300: c64 6.8e-7, tf32x3 2.2e-6, bf16x3 6.3e-6
    assert errs["c64"] <= 1e-5 and errs["tf32x3"] <= 1e-5 and errs["bf16x3"] <= 3e-5 and errs["fp16x3"] <= 1e-5


def test_grid7x7_reduced_depth_batch64_vs_oracle(tz):
    """7x7, depth 1+14+1, 64 bitstrings as one batch, sliced, against the oracle."""
    spec = grid_spec(7, 7, 14, 2)
    bits = ti.random_bitstrings(49, 64, 55)
    c = tn.Contractor(spec, max_log2=24)
    ref = np.array([c.amplitude(x) for x in bits])
    plan, _, _, sl = build(tz, spec, "tf32x3", 14, batch_log2=6, k_max=6, restarts=16, max_bitstrings=64)
    got = tz.tz_contract_amplitudes(plan, bits)
    assert rel_err(got, ref, 49) <= TOL


@pytest.mark.parametrize("prec", ["c64", "bf16x3"])
def test_bristlecone72_reduced_depth_vs_oracle(tz, prec):
    """Bristlecone-72 (with its two degree-1 qubits), depth 1+12+1: the planner
    absorbs the degree-1 wires into their neighbours' subtrees; the oracle
    contracts the 72-qubit network directly. The amplitudes agree."""
    spec = ti.circuit_to_spec(72, ti.generate_circuit(ti.bristlecone(72), 12, 3))
    bits = ti.random_bitstrings(72, 4, 37)
    c = tn.Contractor(spec, max_log2=24)
    ref = np.array([c.amplitude(x) for x in bits])
    plan, *_ = build(tz, spec, prec, 30, restarts=16)
    got = tz.tz_contract_amplitudes(plan, bits)
    err = rel_err(got, ref, 72)
    print(f"bristlecone72 d12 {prec}: max rel err {err:.2e}")
    assert err <= (TOL if prec == "c64" else 6e-6)   # measured 1.8e-6 in both


def test_grid7x7_depth40_precision_sweep(tz):
    """7x7 depth 1+40+1 with 2^14 slices (the deepest grid workload): the
    partial amplitude of slices [0, 32) for 4 bitstrings in each FP32-class
    mode against complex128 on the same tree and slicing; errors printed."""
    import torch
    spec = grid_spec(7, 7, 40, 5)
    bits = ti.random_bitstrings(49, 4, 105)
    net = tz.tz_network_from_circuit(tz.tz_circuit_from_spec(spec), 0)
    tree = tz.tz_path_greedy(net, restarts=32, seed=7, log2_max_intermediate=24, algorithm="elimination",
                             precision="bf16x3")
    sl = tz.tz_slice_select(net, tree, 24, 20)
    assert 12 <= len(sl) <= 16   # 14 with this tree
    out = {}
    for prec in ("c128", "c64", "tf32x3", "bf16x3", "fp16x3"):
        plan = tz.tz_plan_create(net, tree, sl, precision=prec, stream=torch.cuda.Stream(), use_graph=True,
                                 max_bitstrings=4)
        st = plan.stats()
        assert st["flops_per_group"] * 32 < MAX_FLOPS_PER_AMPLITUDE
        plan.bind()
        plan.set_slice_range(0, 32)
        out[prec] = tz.tz_contract_amplitudes(plan, bits)
    errs = {m: rel_err(out[m], out["c128"], 49) for m in ("c64", "tf32x3", "bf16x3", "fp16x3")}
    print("grid7x7 d40 (32 of 2^14 slices) errors vs complex128:", {m: f"{e:.2e}" for m, e in errs.items()})
    # measured on GB300: c64 1.5e-7, tf32x3 4.9e-7, bf16x3 6.5e-7, fp16x3 2.3e-7
    assert errs["c64"] <= 1e-5 and errs["tf32x3"] <= 1e-5 and errs["bf16x3"] <= 3e-6 and errs["fp16x3"] <= 1e-5


# -------------------------------------------------------------------------
# Full depth against the FP64 oracle, per sampled slice (Sec. 1: each
# subtask's partial amplitude is a fixed piece of the amplitude, so the
# GPU's and the oracle's partial of the same slice must agree)

PARTIAL_TOL = {"c64": 1e-5, "tf32x3": 1e-5, "fp16x3": 1e-5, "bf16x3": 3e-5, "c128": 1e-12}


def _partials(tz, net, tree, sliced, prec, bits, slices):
    import torch
    # autotuned as in the bench: the steps run in the launch forms and on the
    # kernels the autotuner picks
    plan = tz.tz_plan_create(net, tree, sliced, precision=prec, stream=torch.cuda.Stream(), use_graph=True,
                             max_bitstrings=len(bits), autotune=True)
    plan.bind()
    out = {}
    for s in slices:
        plan.set_slice_range(s, s + 1)
        out[s] = tz.tz_contract_amplitudes(plan, bits)
    segs = plan.sliced_segments()
    plan.close()
    return out, segs


def test_grid7x7_depth32_config2_slices_vs_oracle(tz):
    """Config 2: 7x7, depth 1+32+1, a tree with 2^10 slices; the partial
    amplitudes of slices 0 and 777 for two of the config's bitstrings in
    every mode against the path-sum oracle with the plan's sliced segments."""
    spec = grid_spec(7, 7, 32, 2)
    bits = ti.random_bitstrings(49, 64, 102)[:2]
    net = tz.tz_network_from_circuit(tz.tz_circuit_from_spec(spec), 0)
    tree = tz.tz_path_greedy(net, restarts=32, seed=7, log2_max_intermediate=22, precision="tf32x3",
                             algorithm="elimination")
    sl = tz.tz_slice_select(net, tree, 1, 10)
    assert len(sl) == 10
    slices = (0, 777)
    got, segs = {}, None
    for prec in ("c64", "tf32x3", "fp16x3", "bf16x3", "c128"):
        got[prec], segs = _partials(tz, net, tree, sl, prec, bits, slices)
    oracle = pathsum.SegmentContractor(spec, sliced=segs, max_log2=25)
    ref = {s: np.array([oracle.partial(x, s) for x in bits]) for s in slices}
    errs = {m: max(rel_err_partial(got[m][s], ref[s], 49, 10) for s in slices) for m in got}
    print("grid7x7 d32 config 2, slices 0 and 777 vs oracle:", {m: f"{e:.2e}" for m, e in errs.items()})
    for m, e in errs.items():
        assert e <= PARTIAL_TOL[m], (m, e)


@pytest.fixture(scope="module")
def bench_tree(tz):
    """The Bristlecone-70 depth 1+32+1 tree bench.py times (16384 restarts,
    seed 7, 2^30 cap, elimination, split-BF16 time model)."""
    spec = bris_spec(32, 3)
    net = tz.tz_network_from_circuit(tz.tz_circuit_from_spec(spec), 0)
    tree = tz.tz_path_greedy(net, restarts=16384, seed=7, log2_max_intermediate=30, precision="bf16x3",
                             algorithm="elimination")
    return spec, net, tree


@pytest.mark.parametrize("cap,slices", [(20, (5,)), (18, (0, 1 << 20, 987654))])
def test_bristlecone70_depth32_bench_tree_slices_vs_oracle(tz, bench_tree, cap, slices):
    """The bench's Bristlecone-70 tree, sliced to a 2^cap cap (k = 12 and
    k = 21) so that one slice is within the oracle's reach: partial amplitudes
    of sampled slices in every mode against the path-sum oracle."""
    spec, net, tree = bench_tree
    bits = ti.random_bitstrings(70, 1, 103)
    sl = tz.tz_slice_select(net, tree, cap, 40)
    k = len(sl)
    assert k >= 10
    got, segs = {}, None
    for prec in ("c64", "tf32x3", "fp16x3", "bf16x3", "c128"):
        got[prec], segs = _partials(tz, net, tree, sl, prec, bits, slices)
    oracle = pathsum.SegmentContractor(spec, sliced=segs, max_log2=25)
    ref = {s: np.array([oracle.partial(bits[0], s)]) for s in slices}
    errs = {m: max(rel_err_partial(got[m][s], ref[s], 70, k) for s in slices) for m in got}
    print(f"bristlecone70 d32 bench tree, cap 2^{cap} (k={k}), slices {slices} vs oracle:",
          {m: f"{e:.2e}" for m, e in errs.items()})
    for m, e in errs.items():
        assert e <= PARTIAL_TOL[m], (m, e)


def test_bristlecone70_depth28_porter_thomas(tz):
    """Sec. 2 (the Porter-Thomas check of its 200,000-amplitude run, on a
    smaller sample): for 4096 uniform random bitstrings of a Bristlecone-70
    depth 1+28+1 circuit, x = 2^70 |a|^2 follows e^-x: mean 1 within three
    standard errors (3/sqrt(M)), second moment 2 within three standard errors
    (sqrt(20/M) each), P(x > 1) = 1/e, and the Kolmogorov-Smirnov distance to
    1 - e^-x below its 1 % critical value 1.63/sqrt(M)."""
    import math
    import torch
    spec = bris_spec(28, 3)
    m = 4096
    bits = ti.random_bitstrings(70, m, 28_200)
    net = tz.tz_network_from_circuit(tz.tz_circuit_from_spec(spec), 0)
    tree = tz.tz_path_greedy(net, restarts=1024, seed=7, log2_max_intermediate=30, precision="fp16x3",
                             algorithm="elimination")
    sl = tz.tz_slice_select(net, tree, 30, 40)
    plan = tz.tz_plan_create(net, tree, sl, precision="fp16x3", stream=torch.cuda.Stream(), use_graph=True,
                             max_bitstrings=m)
    st = plan.stats()
    assert st["flops_per_group"] * 2.0 ** st["k"] * m < 2e15
    plan.bind()
    x = np.abs(tz.tz_contract_amplitudes(plan, bits)) ** 2 * 2.0 ** 70
    xs = np.sort(x)
    cdf = 1.0 - np.exp(-xs)
    ks = max(np.max(np.arange(1, m + 1) / m - cdf), np.max(cdf - np.arange(m) / m))
    print(f"bristlecone70 d28 Porter-Thomas, {m} amplitudes: mean {x.mean():.4f}, second moment "
          f"{(x ** 2).mean():.4f}, P(x>1) {(x > 1).mean():.4f}, KS {ks:.4f}")
    assert abs(x.mean() - 1.0) < 3.0 / math.sqrt(m)
    assert abs((x ** 2).mean() - 2.0) < 3.0 * math.sqrt(20.0 / m)
    assert abs((x > 1).mean() - math.exp(-1.0)) < 3.0 * math.sqrt(math.exp(-1) * (1 - math.exp(-1)) / m)
    assert ks < 1.63 / math.sqrt(m)
