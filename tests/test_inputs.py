"""Pins of the seeded input generators: the SplitMix64 stream and the circuit
prescription rules of Sec. 1."""
import itertools

import numpy as np
import pytest

import tz_inputs as ti


def test_splitmix64_published_vector():
    # first outputs of the published SplitMix64 reference implementation, seed 0
    r = ti.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_lattices():
    b72, b70 = ti.bristlecone(72), ti.bristlecone(70)
    assert b72.n_qubits == 72 and b70.n_qubits == 70
    rows = [sum(1 for (r, _) in b72.sites if r == i) for i in range(11)]
    assert rows == [2, 4, 6, 8, 10, 12, 10, 8, 6, 4, 2]
    deg = {s: 0 for s in b72.sites}
    for (a, b) in b72.couplers():
        deg[a] += 1
        deg[b] += 1
    assert sorted(s for s, d in deg.items() if d == 1) == [(5, 0), (5, 11)]
    assert ti.grid(7, 7).n_qubits == 49
    with pytest.raises(ValueError):
        ti.bristlecone(71)


@pytest.mark.parametrize("lat,t,seed", [(ti.grid(4, 4), 10, 1), (ti.grid(7, 7), 32, 2), (ti.bristlecone(70), 32, 3),
                                        (ti.grid(3, 5), 17, 9)])
def test_prescription_rules(lat, t, seed):
    gates = ti.generate_circuit(lat, t, seed)
    n = lat.n_qubits
    by_cycle = {}
    for (c, name, qs) in gates:
        by_cycle.setdefault(c, []).append((name, qs))
    # rule 1 and 4: H layers first and last
    assert sorted(q for (nm, (q,)) in by_cycle[0] if nm == "h") == list(range(n))
    assert [nm for nm, _ in by_cycle[t + 1]] == ["h"] * n
    prev = {q: "h" for q in range(n)}
    for c in range(1, t + 1):
        gs = by_cycle.get(c, [])
        used = list(itertools.chain.from_iterable(qs for _, qs in gs))
        assert len(used) == len(set(used)), "a qubit holds two gates in one cycle"
        cz = {q for nm, qs in gs if nm == "cz" for q in qs}
        assert sorted(tuple(qs) for nm, qs in gs if nm == "cz") == ti.cz_pattern_edges(lat, c)
        cur = {}
        for nm, qs in gs:
            for q in qs:
                cur[q] = nm
        for q in range(n):
            g = cur.get(q)
            if q in cz:
                continue
            if prev.get(q) == "cz":
                assert g in ("x_1_2", "y_1_2")           # rule 3a
            elif prev.get(q) in ("h", "x_1_2", "y_1_2"):
                assert g == "t"                           # rule 3b
            else:
                assert g is None
        prev = cur
    assert {nm for (_, nm, _) in gates} <= {"h", "cz", "t", "x_1_2", "y_1_2"}


@pytest.mark.parametrize("lat", [ti.grid(7, 7), ti.bristlecone(72), ti.grid(4, 5)])
def test_patterns_cover_every_coupler_once_per_8_cycles(lat):
    seen = []
    for c in range(1, 9):
        e = ti.cz_pattern_edges(lat, c)
        qs = [q for p in e for q in p]
        assert len(qs) == len(set(qs))
        seen += e
    want = sorted(tuple(sorted((lat.index[a], lat.index[b]))) for (a, b) in lat.couplers())
    assert sorted(seen) == want
    assert ti.cz_pattern_edges(lat, 3) == ti.cz_pattern_edges(lat, 11)


def test_sqrt_choice_is_seeded_and_balanced():
    g1 = ti.generate_circuit(ti.grid(7, 7), 32, 2)
    assert g1 == ti.generate_circuit(ti.grid(7, 7), 32, 2)
    assert g1 != ti.generate_circuit(ti.grid(7, 7), 32, 3)
    names = [nm for (_, nm, _) in g1]
    nx, ny = names.count("x_1_2"), names.count("y_1_2")
    assert abs(nx - ny) < 4 * np.sqrt(nx + ny)


def test_bitstrings():
    b = ti.random_bitstrings(49, 64, 102)
    assert b.shape == (64, 49) and b.dtype == np.uint8 and set(np.unique(b)) <= {0, 1}
    assert np.array_equal(b, ti.random_bitstrings(49, 64, 102))
    assert abs(b.mean() - 0.5) < 0.05


def test_spec_text_roundtrip():
    from oracle.spec import parse_spec
    lat = ti.grid(3, 3)
    gates = ti.generate_circuit(lat, 8, 4)
    n, parsed = parse_spec(ti.circuit_to_spec(9, gates))
    assert n == 9 and parsed == gates
