"""Pins of the FP64 oracle against facts outside itself: hand-derived closed
forms (tests/golden/closed_forms.txt), gate identities, a Kronecker-product
unitary, the norm, agreement of its two independent parts, the slicing
identity (Sec. 1: subtask results add up to the amplitude) and the
Porter-Thomas moments of Sec. 2."""
import os

import numpy as np
import pytest

import tz_inputs as ti
from oracle import gates as G
from oracle import statevector as sv
from oracle import tn
from oracle.spec import parse_spec, segments

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")


def load_golden():
    rows = []
    for ln in open(GOLDEN):
        if not ln.strip() or ln.startswith("#"):
            continue
        name, spec, bits, re, im = [f.strip() for f in ln.split("|")]
        rows.append((name, spec.replace(";", "\n") + "\n", [int(ch) for ch in bits], complex(float(re), float(im))))
    return rows


@pytest.mark.parametrize("row", load_golden(), ids=lambda r: r[0])
def test_closed_forms(row):
    name, spec, bits, want = row
    assert abs(sv.amplitudes(spec, [bits])[0] - want) < 1e-15
    assert abs(tn.amplitudes(spec, [bits])[0] - want) < 1e-15


def test_gate_identities():
    I2 = np.eye(2)
    assert np.allclose(G.H @ G.H, I2, atol=1e-15)
    assert np.allclose(G.SQRT_X @ G.SQRT_X, G.X, atol=1e-15)
    assert np.allclose(G.SQRT_Y @ G.SQRT_Y, G.Y, atol=1e-15)
    assert np.allclose(np.linalg.matrix_power(G.T, 2), np.diag([1, 1j]), atol=1e-15)
    assert np.allclose(np.linalg.matrix_power(G.T, 8), I2, atol=1e-15)
    for U in (G.H, G.T, G.SQRT_X, G.SQRT_Y, G.CZ):
        assert np.allclose(U @ U.conj().T, np.eye(U.shape[0]), atol=1e-15)
    # sqrt(Y) is not symmetric: a transposed operand would flip this sign
    assert G.SQRT_Y[1, 0] == 0.5 + 0.5j and G.SQRT_Y[0, 1] == -0.5 - 0.5j


def test_cz_split_identity():
    full = np.einsum("aik,bjk->abij", tn.CZ_HALF_COPY, tn.CZ_HALF_PHASE)
    assert np.array_equal(full, G.cz_tensor())


@pytest.mark.parametrize("rows,cols,t,seed", [(1, 3, 6, 1), (2, 2, 9, 2), (1, 5, 12, 3)])
def test_against_kronecker_unitary(rows, cols, t, seed):
    lat = ti.grid(rows, cols)
    spec = ti.circuit_to_spec(lat.n_qubits, ti.generate_circuit(lat, t, seed))
    n, gates = parse_spec(spec)
    U = sv.dense_unitary(n, gates)
    assert np.allclose(U @ U.conj().T, np.eye(1 << n), atol=1e-13)
    psi = sv.final_state(n, gates)
    assert np.allclose(U[:, 0], psi, atol=1e-14)
    allx = [[(i >> q) & 1 for q in range(n)] for i in range(1 << n)]
    assert np.allclose(tn.amplitudes(spec, allx), U[:, 0], atol=1e-14)


def test_norm_statevector_4x4():
    lat = ti.grid(4, 4)
    spec = ti.circuit_to_spec(16, ti.generate_circuit(lat, 10, 1))
    n, gates = parse_spec(spec)
    assert abs(np.sum(np.abs(sv.final_state(n, gates)) ** 2) - 1.0) < 1e-12


def test_norm_contractor_3x3():
    lat = ti.grid(3, 3)
    spec = ti.circuit_to_spec(9, ti.generate_circuit(lat, 12, 5))
    c = tn.Contractor(spec)
    allx = [[(i >> q) & 1 for q in range(9)] for i in range(512)]
    amps = np.array([c.amplitude(x) for x in allx])
    assert abs(np.sum(np.abs(amps) ** 2) - 1.0) < 1e-12


@pytest.mark.parametrize("rows,cols,t,seed,maxl", [(4, 4, 10, 1, 30), (4, 5, 12, 3, 30), (4, 4, 16, 6, 5)])
def test_statevector_vs_contractor(rows, cols, t, seed, maxl):
    lat = ti.grid(rows, cols)
    spec = ti.circuit_to_spec(lat.n_qubits, ti.generate_circuit(lat, t, seed))
    bs = ti.random_bitstrings(lat.n_qubits, 6, seed + 100)
    a = sv.amplitudes(spec, bs)
    c = tn.Contractor(spec, max_log2=maxl)
    b = np.array([c.amplitude(x) for x in bs])
    assert np.max(np.abs(a - b)) < 1e-13 * max(1.0, np.max(np.abs(a)) * 1e3)


@pytest.mark.parametrize("k", [1, 3, 6])
def test_sliced_sum_equals_unsliced(k):
    lat = ti.grid(4, 4)
    gates = ti.generate_circuit(lat, 10, 1)
    spec = ti.circuit_to_spec(16, gates)
    n, g = parse_spec(spec)
    _, nseg = segments(n, g)
    cand = [(q, j) for q in range(n) for j in range(1, nseg[q])]
    rng = np.random.default_rng(k)
    sliced = [cand[i] for i in rng.choice(len(cand), size=k, replace=False)]
    bits = ti.random_bitstrings(16, 1, 40 + k)[0]
    full = tn.Contractor(spec).amplitude(bits)
    c = tn.Contractor(spec, sliced=sliced)
    parts = [c.partial(bits, s) for s in range(1 << k)]
    assert abs(sum(parts) - full) < 1e-14
    # a partial amplitude is a genuine piece, not the whole
    assert max(abs(p - full) for p in parts) > 1e-6 * abs(full)
    assert abs(full - sv.amplitudes(spec, [bits])[0]) < 1e-14
    # each partial equals a state-vector run with the projector |v><v| put on
    # qubit q right after its j-th non-diagonal gate (the segment's value is
    # constant until the next one, since T and CZ are diagonal)
    for s_id in (0, (1 << k) - 1, (1 << k) // 3):
        fixed = {seg: (s_id >> i) & 1 for i, seg in enumerate(sliced)}
        assert abs(parts[s_id] - projected_amplitude(n, g, bits, fixed)) < 1e-14


def projected_amplitude(n, gates, bits, fixed):
    psi = np.zeros((2,) * n, dtype=np.complex128)
    psi[(0,) * n] = 1.0
    seg = [0] * n
    for (_, name, qs) in gates:
        if name == "cz":
            idx = [slice(None)] * n
            idx[n - 1 - qs[0]] = 1
            idx[n - 1 - qs[1]] = 1
            psi[tuple(idx)] *= -1.0
            continue
        q = qs[0]
        ax = n - 1 - q
        psi = np.moveaxis(np.tensordot(G.ONE_QUBIT[name], psi, axes=([1], [ax])), 0, ax)
        if name != "t":
            seg[q] += 1
            if (q, seg[q]) in fixed:
                idx = [slice(None)] * n
                idx[ax] = 1 - fixed[(q, seg[q])]
                psi[tuple(idx)] = 0.0
    return psi.reshape(-1)[sv.basis_index(bits)]


def test_porter_thomas_moments():
    """Sec. 2: for deep random circuits N*p follows exp(-x): E[Np] = 1,
    E[(Np)^2] = 2, P(Np > 1) = 1/e."""
    lat = ti.grid(4, 5)
    n, gates = parse_spec(ti.circuit_to_spec(20, ti.generate_circuit(lat, 24, 11)))
    p = np.abs(sv.final_state(n, gates)) ** 2 * (1 << n)
    assert abs(p.mean() - 1.0) < 1e-10
    assert abs((p ** 2).mean() - 2.0) < 0.1
    assert abs((p > 1).mean() - np.exp(-1)) < 0.01


def test_shallow_circuit_is_not_porter_thomas():
    # a depth-1 circuit is far from Porter-Thomas: the check above has power
    lat = ti.grid(4, 5)
    n, gates = parse_spec(ti.circuit_to_spec(20, ti.generate_circuit(lat, 1, 11)))
    p = np.abs(sv.final_state(n, gates)) ** 2 * (1 << n)
    assert abs((p ** 2).mean() - 2.0) > 0.5


# ----------------------------------------------------------------------------
# Pins of the per-step definitions (oracle/linalg.py): hand-worked values
# (tests/golden/linalg_ops.txt) and textbook formulations that share no code
# with them.

from oracle import linalg  # noqa: E402
from oracle import pathsum  # noqa: E402

LINALG_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "linalg_ops.txt")


def _golden_ops():
    ops = {}
    for ln in open(LINALG_GOLDEN):
        if not ln.strip() or ln.startswith("#"):
            continue
        op, inputs, want = [f.strip() for f in ln.split("|")]
        ops[op] = (inputs, want)
    return ops


def _cmat(text):
    return np.array([[complex(v) for v in row.split()] for row in text.split(";")], dtype=np.complex128)


def test_bit_permute_hand_example():
    inputs, want = _golden_ops()["permute"]
    x, perm = inputs.split(";")
    got = linalg.bit_permute(np.array([float(v) for v in x.split()]), [int(p) for p in perm.split()])
    assert got.tolist() == [float(v) for v in want.split()]


@pytest.mark.parametrize("r,seed", [(1, 0), (3, 1), (5, 2), (8, 3)])
def test_bit_permute_is_a_transpose(r, seed):
    """Bit p of a flat offset is axis r-1-p of the C-order (2,)*r view; output
    bit p = input bit perm[p] is the transpose that puts input axis
    r-1-perm[p] at output axis r-1-p."""
    rng = np.random.default_rng(seed)
    perm = [int(v) for v in rng.permutation(r)]
    x = rng.standard_normal(1 << r) + 1j * rng.standard_normal(1 << r)
    axes = [0] * r
    for p in range(r):
        axes[r - 1 - p] = r - 1 - perm[p]
    want = np.transpose(x.reshape((2,) * r), axes).reshape(-1)
    assert np.array_equal(linalg.bit_permute(x, perm), want)


def test_cgemm_hand_example():
    inputs, want = _golden_ops()["cgemm"]
    a, b = inputs.split("#")
    C = linalg.cgemm(_cmat(a)[None], _cmat(b)[None])
    assert np.array_equal(C[0], _cmat(want))


def test_cgemm_triple_loop():
    rng = np.random.default_rng(5)
    bt, m, n, k = 3, 4, 5, 6
    A = rng.standard_normal((bt, m, k)) + 1j * rng.standard_normal((bt, m, k))
    B = rng.standard_normal((bt, n, k)) + 1j * rng.standard_normal((bt, n, k))
    want = np.zeros((bt, m, n), dtype=np.complex128)
    for z in range(bt):
        for i in range(m):
            for j in range(n):
                for l in range(k):
                    want[z, i, j] += A[z, i, l] * B[z, j, l]
    assert np.allclose(linalg.cgemm(A, B), want, rtol=0, atol=1e-13)


def test_accumulate_hand_example():
    inputs, want = _golden_ops()["accumulate"]
    acc, part, scale = inputs.split("#")
    got = linalg.accumulate(_cmat(acc)[0], _cmat(part)[0], complex(scale.strip()))
    assert np.array_equal(got, _cmat(want)[0])


# ----------------------------------------------------------------------------
# Pins of the path-sum contractor (oracle/pathsum.py)

@pytest.mark.parametrize("row", load_golden(), ids=lambda r: r[0])
def test_pathsum_closed_forms(row):
    name, spec, bits, want = row
    assert abs(pathsum.amplitudes(spec, [bits])[0] - want) < 1e-15


@pytest.mark.parametrize("rows,cols,t,seed", [(1, 3, 6, 1), (2, 2, 9, 2), (1, 5, 12, 3)])
def test_pathsum_against_kronecker_unitary(rows, cols, t, seed):
    lat = ti.grid(rows, cols)
    spec = ti.circuit_to_spec(lat.n_qubits, ti.generate_circuit(lat, t, seed))
    n, gates = parse_spec(spec)
    U = sv.dense_unitary(n, gates)
    allx = [[(i >> q) & 1 for q in range(n)] for i in range(1 << n)]
    assert np.allclose(pathsum.amplitudes(spec, allx), U[:, 0], rtol=0, atol=1e-14)


def test_pathsum_norm_3x3():
    spec = ti.circuit_to_spec(9, ti.generate_circuit(ti.grid(3, 3), 12, 5))
    allx = [[(i >> q) & 1 for q in range(9)] for i in range(512)]
    assert abs(np.sum(np.abs(pathsum.amplitudes(spec, allx)) ** 2) - 1.0) < 1e-12


@pytest.mark.parametrize("rows,cols,t,seed,maxl", [(4, 4, 10, 1, 30), (4, 5, 12, 3, 30), (4, 5, 16, 4, 6)])
def test_pathsum_vs_statevector(rows, cols, t, seed, maxl):
    """The path sum against the state vector; a small cap forces the
    contractor to fix extra segments of its own and sum over them."""
    lat = ti.grid(rows, cols)
    spec = ti.circuit_to_spec(lat.n_qubits, ti.generate_circuit(lat, t, seed))
    bs = ti.random_bitstrings(lat.n_qubits, 6, seed + 200)
    c = pathsum.SegmentContractor(spec, max_log2=maxl)
    if maxl < 10:
        assert len(c.extra) > 0 and c.width - 1 <= maxl
    got = np.array([c.amplitude(x) for x in bs])
    ref = sv.amplitudes(spec, bs)
    assert np.max(np.abs(got - ref)) < 1e-13 * max(1.0, np.max(np.abs(ref)) * 1e3)


@pytest.mark.parametrize("k", [1, 4, 7])
def test_pathsum_partials_match_the_wire_contractor(k):
    """Per-slice partial amplitudes (Sec. 1 subtasks) of the path sum equal
    the plain-wire contractor's for the same sliced segments, and add up to
    the state-vector amplitude."""
    lat = ti.grid(4, 5)
    spec = ti.circuit_to_spec(20, ti.generate_circuit(lat, 12, 3))
    n, g = parse_spec(spec)
    _, nseg = segments(n, g)
    cand = [(q, j) for q in range(n) for j in range(1, nseg[q])]
    rng = np.random.default_rng(100 + k)
    sliced = [cand[i] for i in rng.choice(len(cand), size=k, replace=False)]
    bits = ti.random_bitstrings(20, 1, 60 + k)[0]
    ps = pathsum.SegmentContractor(spec, sliced=sliced)
    wc = tn.Contractor(spec, sliced=sliced)
    parts = [ps.partial(bits, s) for s in range(1 << k)]
    for s in sorted({0, (1 << k) - 1, (1 << k) // 3, (1 << k) // 2}):
        assert abs(parts[s] - wc.partial(bits, s)) < 1e-14
        fixed = {seg: (s >> i) & 1 for i, seg in enumerate(sliced)}
        assert abs(parts[s] - projected_amplitude(n, g, bits, fixed)) < 1e-14
    assert abs(sum(parts) - sv.amplitudes(spec, [bits])[0]) < 1e-14


def test_pathsum_rejects_unknown_segment():
    spec = ti.circuit_to_spec(4, ti.generate_circuit(ti.grid(2, 2), 4, 1))
    with pytest.raises(ValueError):
        pathsum.SegmentContractor(spec, sliced=[(0, 99)])
    with pytest.raises(ValueError):
        pathsum.SegmentContractor(spec, sliced=[(0, 1), (0, 1)])
