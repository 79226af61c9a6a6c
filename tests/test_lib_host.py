"""Host-side checks of the library (no GPU): the C ABI loads and exports
every declared symbol, the C++ circuit generator matches the seeded input
generator, and the network/tree/slicing/plan logic keeps its invariants."""
import json
import os
import re

import numpy as np
import pytest

import tz_inputs as ti

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tz():
    import paper_1907_11217_gb300 as tz
    tz._lib.lib()
    return tz


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "tz.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tz_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(tz):
    import ctypes
    L = ctypes.CDLL(tz._lib.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 30
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(tz._lib.SIGNATURES), set(names) - set(tz._lib.SIGNATURES)


@pytest.mark.parametrize("lat,kind,args,t,seed", [
    (ti.grid(4, 4), 0, (4, 4, 0), 10, 1), (ti.grid(7, 7), 0, (7, 7, 0), 32, 2),
    (ti.bristlecone(70), 1, (0, 0, 70), 32, 3), (ti.bristlecone(72), 1, (0, 0, 72), 20, 9),
    (ti.grid(3, 5), 0, (3, 5, 0), 17, 12345678901234)])
def test_cpp_generator_matches_inputs(tz, lat, kind, args, t, seed):
    c = tz.tz_circuit_generate(kind, args[0], args[1], args[2], t, seed)
    assert c.to_spec() == ti.circuit_to_spec(lat.n_qubits, ti.generate_circuit(lat, t, seed))


def test_spec_roundtrip_and_errors(tz):
    spec = ti.circuit_to_spec(9, ti.generate_circuit(ti.grid(3, 3), 6, 4))
    assert tz.tz_circuit_from_spec(spec).to_spec() == spec
    for bad in ["", "2\n0 h 2\n", "2\n0 cz 0 0\n", "2\n0 foo 1\n", "x\n", "2\n0 h\n", "2\n0 cz 0\n"]:
        with pytest.raises(tz.TzError) as e:
            tz.tz_circuit_from_spec(bad)
        assert e.value.code == -1
    with pytest.raises(tz.TzError):
        tz.tz_circuit_generate(1, 0, 0, 71, 10, 1)


def test_network_structure(tz):
    c = tz.tz_circuit_generate_grid(4, 4, 10, 1)
    for g in (0, 3):
        net = tz.tz_network_from_circuit(c, g)
        seen_open = 0
        for i in range(net.n_indices):
            q, s = net.index_info(i)
            if q < 0:
                seen_open += 1
                assert 0 <= s < g
            else:
                assert 0 <= q < 16 and s >= 1
        assert seen_open == g
        # every wire index is held by at least two tensors; batch indices by the 16 outputs
        holders = {}
        for t in range(net.n_tensors):
            for i in net.tensor_indices(t):
                holders[i] = holders.get(i, 0) + 1
        for i, h in holders.items():
            q, _ = net.index_info(i)
            assert h >= 2 if q >= 0 else h == 16
    with pytest.raises(tz.TzError):
        tz.tz_network_from_circuit(c, 9)


def test_tree_validation(tz):
    c = tz.tz_circuit_generate_grid(3, 3, 8, 2)
    net = tz.tz_network_from_circuit(c, 0)
    tree = tz.tz_path_greedy(net)
    pairs = tree.pairs()
    assert len(pairs) == net.n_tensors - 1
    tz.tz_tree_from_pairs(net, pairs)
    with pytest.raises(tz.TzError):
        tz.tz_tree_from_pairs(net, pairs[:-1])
    bad = pairs.copy()
    bad[-1] = bad[0]
    with pytest.raises(tz.TzError):
        tz.tz_tree_from_pairs(net, bad)


def test_slicing_meets_target_and_equal_cost(tz):
    """Sec. 2: all subtasks have equal cost -- the same indices are sliced in
    every subtask, so every group runs the same steps."""
    c = tz.tz_circuit_generate_grid(5, 5, 16, 4)
    net = tz.tz_network_from_circuit(c, 0)
    tree = tz.tz_path_greedy(net, restarts=4, seed=3)
    full = tz.tz_plan_create(net, tree, []).stats()
    target = full["max_log2"] - 3
    sl = tz.tz_slice_select(net, tree, target, 40)
    assert len(sl) == len(set(sl)) >= 3
    st = tz.tz_plan_create(net, tree, sl).stats()
    assert st["max_log2"] <= target < full["max_log2"]
    assert st["k"] == len(sl)
    for e in sl:
        q, s = net.index_info(e)
        assert q >= 0
    with pytest.raises(tz.TzError):
        tz.tz_plan_create(net, tree, [sl[0], sl[0]])
    with pytest.raises(tz.TzError):
        tz.tz_plan_create(net, tree, [10 ** 6])


def test_plan_stats_and_workspace_sizes(tz):
    c = tz.tz_circuit_generate_grid(4, 4, 10, 1)
    net = tz.tz_network_from_circuit(c, 2)
    tree = tz.tz_path_greedy(net)
    for prec in ("c64", "tf32x3", "bf16x3", "fp16x3"):
        p = tz.tz_plan_create(net, tree, [], precision=prec, max_bitstrings=64)
        st = p.stats()
        assert st["workspace_bytes"] > 0 and st["n_steps"] == net.n_tensors - 1
        assert st["flops_per_group"] > 0
        assert '"steps"' in p.describe()


def test_fp16x3_scratch_and_launch_counts(tz):
    """The scaled split-FP16 product needs the split-BF16 product's scratch
    plus room for the partial maxima of |B| (304 words), and one
    more launch per tensor-core step (the maxima pass)."""
    import json
    for shape in [(1, 128, 8, 16), (4, 1024, 64, 256), (2, 128, 16, 4096)]:
        bf = tz.tz_op_cgemm_scratch_bytes("bf16x3", *shape)
        fp = tz.tz_op_cgemm_scratch_bytes("fp16x3", *shape)
        assert fp >= bf + 304 * 4
    with pytest.raises(tz.TzError):
        tz.tz_op_cgemm_scratch_bytes("fp16x3", 1, 128, 8, 6)   # K not a multiple of 4
    c = tz.tz_circuit_generate_grid(5, 6, 20, 7)
    net = tz.tz_network_from_circuit(c, 6)
    tree = tz.tz_path_greedy(net, restarts=4, seed=3, precision="bf16x3")
    st = {}
    for prec in ("bf16x3", "fp16x3"):
        p = tz.tz_plan_create(net, tree, [], precision=prec, small_log2=8, max_bitstrings=64)
        n_tc = sum(1 for x in json.loads(p.describe())["steps"] if x.get("tc"))
        st[prec] = (p.stats()["n_launches_per_group"], n_tc)
    assert st["fp16x3"][1] == st["bf16x3"][1] > 0
    assert st["fp16x3"][0] == st["bf16x3"][0] + st["fp16x3"][1]


def test_bind_rejects_bad_workspace(tz):
    import ctypes
    c = tz.tz_circuit_generate_grid(2, 2, 4, 1)
    net = tz.tz_network_from_circuit(c, 0)
    p = tz.tz_plan_create(net, tz.tz_path_greedy(net), [])
    L = tz._lib.lib()
    assert L.tz_plan_bind_workspace(p.handle, None, 1 << 20) == -1
    assert L.tz_plan_bind_workspace(p.handle, ctypes.c_void_p(256), 16) == -2
    assert L.tz_plan_bind_workspace(p.handle, ctypes.c_void_p(257), 1 << 30) == -1
    out = np.zeros(2)
    b = np.zeros(4, dtype=np.uint8)
    assert L.tz_contract_amplitudes(p.handle, b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), 1,
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == -1
    assert "workspace" in L.tz_last_error().decode()


@pytest.mark.parametrize("depth,seed", [(20, 3), (24, 5)])
def test_degree_one_qubits_cost_like_70(tz, depth, seed):
    """Sec. 1: the two qubits of Bristlecone-72 with one neighbour each add
    nothing of order to the contraction; the planner absorbs their wires, so
    a 72-qubit circuit costs about what a 70-qubit one of the same depth does
    (within a factor of 2 in flops per amplitude)."""
    import math
    flops = {}
    for n in (70, 72):
        spec = ti.circuit_to_spec(n, ti.generate_circuit(ti.bristlecone(n), depth, seed))
        net = tz.tz_network_from_circuit(tz.tz_circuit_from_spec(spec), 0)
        tree = tz.tz_path_greedy(net, restarts=32, seed=7, log2_max_intermediate=30, algorithm="elimination",
                                 precision="bf16x3")
        flops[n] = tz.tz_plan_create(net, tree, [], precision="bf16x3").stats()["flops_per_group"]
    assert abs(math.log2(flops[72]) - math.log2(flops[70])) <= 1.0, flops


def test_path_search_independent_of_thread_count(tz, monkeypatch):
    """Restarts run on host threads; the tree returned, and so every plan
    built on it, must not depend on how many (TZ_PATH_THREADS)."""
    c = tz.tz_circuit_generate_grid(5, 5, 16, 3)
    net = tz.tz_network_from_circuit(c, 0)
    trees = []
    for th in ("1", "3", "8"):
        monkeypatch.setenv("TZ_PATH_THREADS", th)
        for alg, rc in (("auto", 0), ("elimination", 0), ("elimination", 6)):
            t = tz.tz_path_greedy(net, restarts=24, seed=5, log2_max_intermediate=12, algorithm=alg, reconfigure=rc)
            trees.append((th, (alg, rc), t.pairs().tobytes()))
    for key in (("auto", 0), ("elimination", 0), ("elimination", 6)):
        got = {th: p for th, k, p in trees if k == key}
        assert got["1"] == got["3"] == got["8"]


def test_reconfigure_never_worse_and_valid(tz):
    """Exact window re-optimisation keeps a complete, valid tree (a plan
    builds on it, one step per pair), and the tree it returns is not much
    costlier in useful flops than the search without it (the time model,
    not the flop count, decides, so the check is loose); out-of-range
    window sizes are rejected."""
    c = tz.tz_circuit_generate_grid(5, 6, 16, 3)
    net = tz.tz_network_from_circuit(c, 0)
    base = tz.tz_path_greedy(net, restarts=8, seed=3, log2_max_intermediate=14, precision="bf16x3",
                             algorithm="elimination")
    for w in (4, 6, 8):
        t = tz.tz_path_greedy(net, restarts=8, seed=3, log2_max_intermediate=14, precision="bf16x3",
                              algorithm="elimination", reconfigure=w)
        p0 = tz.tz_plan_create(net, base, tz.tz_slice_select(net, base, 14, 40), precision="bf16x3")
        p1 = tz.tz_plan_create(net, t, tz.tz_slice_select(net, t, 14, 40), precision="bf16x3")
        s0, s1 = p0.stats(), p1.stats()
        assert s1["n_steps"] == net.n_tensors - 1
        assert s1["flops_per_group"] * 2.0 ** s1["k"] <= 1.5 * s0["flops_per_group"] * 2.0 ** s0["k"]
    with pytest.raises(tz.TzError):
        tz.tz_path_greedy(net, restarts=1, reconfigure=2)


def test_contract_empty_and_oversized_batches(tz):
    """Zero bitstrings is a valid, empty request (nothing is read or
    written, no device work); more than the plan's max_bitstrings is
    rejected before any device work."""
    c = tz.tz_circuit_generate_grid(4, 4, 10, 1)
    net = tz.tz_network_from_circuit(c, 0)
    tree = tz.tz_path_greedy(net, restarts=2, seed=1)
    plan = tz.tz_plan_create(net, tree, [], precision="c64", max_bitstrings=4)   # not bound
    out = tz.tz_contract_amplitudes(plan, np.zeros((0, 16), dtype=np.uint8))
    assert out.shape == (0,) and out.dtype == np.complex128
    with pytest.raises(tz.TzError) as e:
        tz.tz_contract_amplitudes(plan, np.zeros((5, 16), dtype=np.uint8))
    assert e.value.code == -1


def _contract_described(desc, bits, open_order):
    """Contract the network a plan describes, for one bitstring (batch of 1),
    by pairwise einsum in numpy, keeping the open indices; returns the
    tensor over the open indices in `open_order` (a test helper, no oracle)."""
    items = []
    for lf in desc["leaves"]:
        data = np.array([complex(re_, im_) for re_, im_ in lf["data"]])
        if lf["kind"] == 1:  # output tensor: row x of M[x * 2^rc + e]
            rc = lf["rc"]
            x = int(bits[lf["qubit"]])
            arr = data[x << rc:(x + 1) << rc]
            labels = lf["idx"][:rc]
        else:
            arr = data
            labels = lf["idx"]
        r = len(labels)
        items.append((arr.reshape((2,) * r) if r else arr.reshape(()), list(reversed(labels))))
    keep = set(open_order)
    while len(items) > 1:
        best = None
        for a in range(len(items)):
            for b in range(a + 1, len(items)):
                la, lb = items[a][1], items[b][1]
                if not set(la) & set(lb) and best is not None:
                    continue
                others = set()
                for c, (_, lc) in enumerate(items):
                    if c != a and c != b:
                        others |= set(lc)
                out = [e for e in dict.fromkeys(la + lb) if e in others or e in keep]
                if best is None or len(out) < best[0]:
                    best = (len(out), a, b, out)
        _, a, b, out = best
        (xa, la), (xb, lb) = items[a], items[b]
        names = {e: chr(97 + k) for k, e in enumerate(dict.fromkeys(la + lb))}
        sub = "".join(names[e] for e in la) + "," + "".join(names[e] for e in lb) + "->" + \
            "".join(names[e] for e in out)
        xc = np.einsum(sub, xa, xb)
        items = [it for c, it in enumerate(items) if c not in (a, b)] + [(xc, out)]
    x, labels = items[0]
    return np.transpose(x, [labels.index(e) for e in open_order]) * complex(*desc["scalar"])


@pytest.mark.parametrize("spec_kind, open_q", [("grid3x3", (0, 4, 8)), ("grid3x3", (2,)),
                                               ("idle", (1, 2)), ("idle", (0,))])
def test_open_output_qubits_network_matches_statevector(tz, spec_kind, open_q):
    """A network with open output qubits, contracted on the host from the
    plan's own description, gives the state-vector amplitudes of every
    assignment of the open qubits (Sec. 2: several amplitudes from one
    contraction). "idle": qubit 1 has only diagonal gates after |0>, qubit 2
    none at all, so their open index sits on the input tensor."""
    import json
    from oracle import statevector
    if spec_kind == "grid3x3":
        spec = ti.circuit_to_spec(9, ti.generate_circuit(ti.grid(3, 3), 8, 5))
        n = 9
    else:
        spec = "3\n0 h 0\n1 cz 0 1\n2 t 1\n3 x_1_2 0\n"
        n = 3
    net = tz.tz_network_from_circuit(tz.tz_circuit_from_spec(spec), 0, open_q)
    infos = [net.index_info(i) for i in range(net.n_indices)]
    open_idx = sorted((s, i) for i, (q, s) in enumerate(infos) if q == -2)
    assert [s for s, _ in open_idx] == list(range(len(open_q)))
    tree = tz.tz_path_greedy(net, restarts=4, seed=1, log2_max_intermediate=20, precision="c64")
    plan = tz.tz_plan_create(net, tree, [], precision="c64")
    assert plan.n_open == len(open_q)
    desc = json.loads(plan.describe())
    assert sorted(i for i, q, s in desc["open"] if q == -2) == sorted(i for _, i in open_idx)
    rng = np.random.default_rng(3)
    oq = sorted(open_q)
    for _ in range(3):
        bits = rng.integers(0, 2, n).astype(np.uint8)
        got = _contract_described(desc, bits, [i for _, i in open_idx]).reshape(-1, order="F")
        expanded = np.repeat(bits[None, :], 1 << len(oq), axis=0)
        for o in range(1 << len(oq)):
            for j, q in enumerate(oq):
                expanded[o, q] = (o >> j) & 1
        want = statevector.amplitudes(spec, expanded)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * max(1.0, np.abs(want).max()))


def test_open_output_qubits_rejected(tz):
    c = tz.tz_circuit_generate_grid(3, 3, 8, 1)
    for bad in [(9,), (-1,), (2, 2), tuple(range(9)), tuple(range(13))]:
        with pytest.raises(tz.TzError):
            tz.tz_network_from_circuit(c, 0, bad)


def _producers(desc):
    """Item index producing each tensor of a plan's group (None: exists
    before the group starts: constants and bind-time results)."""
    prod = {}
    for i, it in enumerate(desc["var_items"]):
        kind = it[0]
        if kind == 0:
            for t in desc["tensors"]:
                if t["var"] and t["leaf"] >= 0 and not t["full"]:
                    prod[t["id"]] = (i, -1)
        elif kind == 1:
            for d in range(it[3], it[3] + it[4]):
                prod[desc["dsteps"][d][2]] = (i, d)
        elif kind == 2:
            prod[it[2]] = (i, -1)
        elif kind == 3:
            st = desc["steps"][it[1]]
            prod[st["c_nat"] if st["c_nat"] >= 0 else st["c"]] = (i, -1)
    return prod


@pytest.mark.parametrize("rows,cols,t,seed,small,prec", [
    (4, 5, 16, 4, 10, "c64"), (5, 5, 14, 2, 8, "fp16x3"), (7, 7, 16, 5, 12, "fp16x3"), (4, 4, 20, 6, 20, "c64")])
def test_direct_queue_schedule(tz, rows, cols, t, seed, small, prec):
    """Queue launches (tz_plan_opts.direct_queue): every direct step runs after the items
    whose results it reads, or, inside its queue launch, after the steps it
    waits for (dep = their index in the launch); each product and permute
    still runs after its inputs; blocks add up; the launch count per group
    is at most that of one launch per dependency level, over the same steps."""
    spec = ti.circuit_to_spec(rows * cols, ti.generate_circuit(ti.grid(rows, cols), t, seed))
    net = tz.tz_network_from_circuit(tz.tz_circuit_from_spec(spec), 2)
    tree = tz.tz_path_greedy(net, restarts=4, seed=1, precision=prec)
    descs, stats = {}, {}
    for levels in (0, 1):
        plan = tz.tz_plan_create(net, tree, [], precision=prec, small_log2=small, direct_queue=not levels)
        descs[levels], stats[levels] = json.loads(plan.describe()), plan.stats()
    q, lv = descs[0], descs[1]
    assert stats[0]["n_launches_per_group"] <= stats[1]["n_launches_per_group"]
    directs = [it for it in q["var_items"] if it[0] == 1]
    assert directs and all(it[6] == 1 for it in directs)
    assert all(it[6] == 0 for it in lv["var_items"] if it[0] == 1)
    assert sorted(tuple(d[:3]) for d in q["dsteps"]) == sorted(tuple(d[:3]) for d in lv["dsteps"])
    prod = _producers(q)
    for i, it in enumerate(q["var_items"]):
        if it[0] == 1:
            assert it[5] == sum(q["dsteps"][d][3] for d in range(it[3], it[3] + it[4]))
            for d in range(it[3], it[3] + it[4]):
                a, b, c, nblk, dep0, dep1 = q["dsteps"][d]
                for x, dep in ((a, dep0), (b, dep1)):
                    pi, pd = prod.get(x, (None, -1))
                    if pi == i:          # made in this launch: wait for it
                        assert it[3] <= pd < d and dep == pd - it[3]
                    else:
                        assert dep == -1 and (pi is None or pi < i)
        elif it[0] in (2, 3):
            st = q["steps"][it[1]] if it[0] == 3 else None
            ins = [it[1]] if it[0] == 2 else [st["opX"], st["opY"]]
            for x in ins:
                pi, _ = prod.get(x, (None, -1))
                assert pi is None or pi < i



def _stream_cases():
    rng = np.random.default_rng(5)
    cases = [(1024, 4096, 8, 4, None), (512, 2048, 256, 8, None), (32, 512, 128, 32, None), (1, 256, 1, 1, None)]
    for _ in range(24):
        gz, gm, gn = rng.integers(0, 7), rng.integers(1, 12), rng.integers(0, 9)
        total = gz + gm + gn
        pos = rng.permutation(total)
        cases.append((1 << gz, 1 << gm, 1 << gn, int(rng.choice([1, 2, 4, 8, 16, 32])),
                      (pos[:gz], pos[gz:gz + gm], pos[gz + gm:])))
    return cases


@pytest.mark.parametrize("case", range(28))
def test_stream_tile_invariants(tz, case):
    """Host side of the stream kernel for small-K products: its tile covers
    the lowest output positions it can, ranks follow output positions, the
    lanes get a permutation of the warp's ranks, shared memory stays within
    40 KB, and (emulating the kernel's index arithmetic) every output of a
    tile is written once, each warp's 32 outputs forming one contiguous run
    when the 5 lowest positions are in the tile."""
    batch, m, n, k, maps = _stream_cases()[case]
    gz, gm, gn = (int(np.log2(x)) for x in (batch, m, n))
    total = gz + gm + gn
    if maps is None:
        pb, pm, pn = (list(range(gn + gm, total)), list(range(gn, gn + gm)), list(range(gn)))
        t = tz.tz_debug_stream_tile(batch, m, n, k)
    else:
        pb, pm, pn = (list(map(int, x)) for x in maps)
        t = tz.tz_debug_stream_tile(batch, m, n, k, pb, pm, pn)
    if batch * m * n < 256:
        assert t is None
        return
    assert t is not None
    pos_of = {0: pb, 1: pm, 2: pn}
    local = {0: t["bz"], 1: t["bm"], 2: t["bn"]}
    assert t["nl"] == sum(local.values()) == len(t["ranks"]) and t["smem"] <= 40 * 1024
    assert t["kmax"] >= k and t["kmax"] in (4, 8, 16, 32)
    # ranks: exactly the local bits, in increasing output position
    assert sorted((s, b) for s, b, _ in t["ranks"]) == sorted((s, b) for s in range(3) for b in range(local[s]))
    assert all(pos_of[s][b] == p for s, b, p in t["ranks"])
    assert [p for _, _, p in t["ranks"]] == sorted(p for _, _, p in t["ranks"])
    covered = 0
    while covered < total and any(p == covered for _, _, p in t["ranks"]):
        covered += 1
    # covering one more of the 6 lowest positions would not fit in 40 KB
    if covered < min(total, 6):
        owner = {}
        for s_, pos in pos_of.items():
            for b, p in enumerate(pos):
                owner[p] = (s_, b)
        need = [0, 0, 0]
        for p in range(covered + 1):
            s_, b = owner[p]
            need[s_] = max(need[s_], b + 1)
        rows = (1 << (need[0] + need[1])) + (1 << (need[0] + need[2]))
        assert rows * (t["kmax"] + 2) + (4 << need[0]) > 40 * 1024 // 8 or sum(need) > 16
    assert sorted(t["lane_rank"]) == list(range(32)) if t["nl"] >= 5 else t["lane_rank"] == list(range(32))
    # emulate one tile: thread rank, high rank bits, output offsets
    R = 1 << t["nl"]
    offs = []
    for rr in range(0, max(R, 256), 256):
        for w in range(8):
            warp = []
            for lane in range(32):
                rank = w * 32 + t["lane_rank"][lane] + rr
                if rank >= R:
                    continue
                o = sum(1 << p for r, (_, _, p) in enumerate(t["ranks"]) if (rank >> r) & 1)
                warp.append(o)
            offs += warp
            if len(warp) == 32 and covered >= 5:
                assert max(warp) - min(warp) == 31 and len(set(warp)) == 32
    want = set()
    for q in range(R):
        want.add(sum(1 << p for r, (_, _, p) in enumerate(t["ranks"]) if (q >> r) & 1))
    assert len(offs) == R and set(offs) == want
