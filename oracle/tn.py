"""FP64 plain-wire tensor-network contractor (oracle part 2).

The network is built here from the spec with no hyperedges at all: every
gate, diagonal or not, is a tensor with one input and one output leg per
qubit it acts on (CZ is the rank-4 tensor [o0, o1, i0, i1]), the input is the
vector |0> and the output of qubit q is the vector <x_q|. Each wire edge
joins exactly two tensors, so a pairwise contraction is one tensordot over
the edges the two tensors share.

Slicing (Sec. 1: the contraction split into subtasks whose results add up to
the amplitude, done once as preprocessing): a wire *segment* (q, j) is the
stretch of qubit q's wire after its j-th non-diagonal gate (H, sqrt(X),
sqrt(Y)); diagonal gates (T, CZ) keep the value on the wire, so fixing a
segment to v fixes every wire edge of that stretch to v. The partial
amplitude of one slice is the contraction with the sliced segments fixed;
summing over all 2^k assignments gives the amplitude.

CZ is entered through the identity CZ = |0><0| (x) I + |1><1| (x) Z: two
rank-3 tensors, C0[o0, i0, k] = [o0 = i0 = k] on the first qubit and
C1[o1, i1, k] = (Z^k)[o1, i1] on the second, joined by a bond leg k of
dimension 2 (the rank-4 [o0, o1, i0, i1] tensor is their contraction over k;
a test checks this). The bond leg joins exactly two tensors like a wire edge.

Contraction order, the oracle's own: the better (smaller largest
intermediate) of
  * a greedy that repeatedly contracts the adjacent pair with the smallest
    growth 2^|out| - 2^|a| - 2^|b| (ties: fewer legs out, then lowest ids);
  * a sweep: fold each qubit's wire in time order into one tensor, then fold
    the qubit tensors in qubit-index order (a row sweep on row-major
    lattices);
and, to bound the largest intermediate, extra slicing of the segments that
occur most often in the largest intermediates of the chosen order.
"""
import heapq
import itertools

import numpy as np

from .gates import ONE_QUBIT, cz_tensor  # noqa: F401  (cz_tensor: rank-4 form, used by tests)
from .spec import parse_spec


# CZ = sum_k |k><k| (x) Z^k, split into its two halves (legs [out, in, k])
CZ_HALF_COPY = np.zeros((2, 2, 2), dtype=np.complex128)
CZ_HALF_COPY[0, 0, 0] = 1.0
CZ_HALF_COPY[1, 1, 1] = 1.0
CZ_HALF_PHASE = np.zeros((2, 2, 2), dtype=np.complex128)
CZ_HALF_PHASE[:, :, 0] = np.eye(2)
CZ_HALF_PHASE[:, :, 1] = np.diag([1.0, -1.0])


class WireNetwork:
    """Plain-wire network of a circuit, with output bitstring left symbolic."""

    def __init__(self, spec_text: str):
        n, gates = parse_spec(spec_text)
        self.n = n
        self.leaves = []        # list of (kind, payload, [edges]); kind: 'in','gate','out'
        self.edge_seg = []      # edge -> (q, segment)
        cur_edge = [None] * n
        seg = [0] * n
        for q in range(n):
            cur_edge[q] = self._new_edge(q, 0)
            self.leaves.append(("in", None, [cur_edge[q]]))
        for (_, name, qs) in gates:
            if name == "cz":
                a, b = qs
                ia, ib = cur_edge[a], cur_edge[b]
                oa, ob = self._new_edge(a, seg[a]), self._new_edge(b, seg[b])
                bond = self._new_edge(a, seg[a], bond=True)
                self.leaves.append(("gate", CZ_HALF_COPY, [oa, ia, bond]))
                self.leaves.append(("gate", CZ_HALF_PHASE, [ob, ib, bond]))
                cur_edge[a], cur_edge[b] = oa, ob
            else:
                q = qs[0]
                if name != "t":
                    seg[q] += 1
                o = self._new_edge(q, seg[q])
                self.leaves.append(("gate", ONE_QUBIT[name], [o, cur_edge[q]]))
                cur_edge[q] = o
        for q in range(n):
            self.leaves.append(("out", q, [cur_edge[q]]))
        self.n_segments = seg[:]   # last segment index per qubit

    def _new_edge(self, q, s, bond=False):
        # a bond leg carries the value of qubit q's wire at its CZ, so fixing
        # segment (q, s) fixes the bond too
        self.edge_seg.append((q, s))
        return len(self.edge_seg) - 1

    def edges_of_segments(self, segs):
        want = set(segs)
        return {e for e, qs in enumerate(self.edge_seg) if qs in want}

    # ---------------------------------------------------------------- values
    def leaf_values(self, bits, fixed):
        """Numeric leaves for output bitstring `bits`, with every edge in
        `fixed` (dict edge -> value) index-selected away. Returns a list of
        (array, [remaining edges])."""
        out = []
        for (kind, payload, edges) in self.leaves:
            if kind == "in":
                arr = np.array([1.0, 0.0], dtype=np.complex128)
            elif kind == "out":
                arr = np.zeros(2, dtype=np.complex128)
                arr[int(bits[payload])] = 1.0
            else:
                arr = payload
            idx = tuple(fixed[e] if e in fixed else slice(None) for e in edges)
            arr = arr[idx]
            rem = [e for e in edges if e not in fixed]
            out.append((np.array(arr, dtype=np.complex128), rem))
        return out


def greedy_path(leg_sets):
    """Oracle greedy order over a plain network given as a list of leg sets.
    Returns (pairs, max_legs); pairs use SSA ids (new id = next free id)."""
    sets = {i: frozenset(s) for i, s in enumerate(leg_sets)}
    owner = {}
    for i, s in sets.items():
        for e in s:
            owner.setdefault(e, set()).add(i)
    nxt = len(leg_sets)
    heap = []

    def push(a, b):
        sa, sb = sets[a], sets[b]
        out = len(sa ^ sb)
        growth = (1 << out) - (1 << len(sa)) - (1 << len(sb))
        heapq.heappush(heap, (growth, out, min(a, b), max(a, b)))

    for e, ts in owner.items():
        if len(ts) == 2:
            a, b = sorted(ts)
            push(a, b)
    pairs = []
    max_legs = max((len(s) for s in sets.values()), default=0)
    while heap:
        _, _, a, b = heapq.heappop(heap)
        if a not in sets or b not in sets:
            continue
        sa, sb = sets.pop(a), sets.pop(b)
        so = sa ^ sb
        c = nxt
        nxt += 1
        for e in sa | sb:
            owner[e].discard(a)
            owner[e].discard(b)
        for e in so:
            owner[e].add(c)
        sets[c] = so
        pairs.append((a, b))
        max_legs = max(max_legs, len(so))
        nbrs = set()
        for e in so:
            nbrs |= owner[e]
        nbrs.discard(c)
        for d in nbrs:
            push(c, d)
    # disconnected pieces (scalars after slicing): fold them in id order
    rest = sorted(sets)
    while len(rest) > 1:
        a, b = rest[0], rest[1]
        so = sets.pop(a) | sets.pop(b)
        c = nxt
        nxt += 1
        sets[c] = so
        pairs.append((a, b))
        rest = sorted(sets)
    return pairs, max_legs


def sweep_path(leaf_qubit, leg_sets):
    """Wire-then-sweep order: leaves of qubit q folded in list order, then
    the per-qubit tensors folded in qubit order. Returns (pairs, max_legs)."""
    sets = [frozenset(s) for s in leg_sets]
    pairs = []
    mx = max((len(s) for s in sets), default=0)
    by_q = {}
    for i, q in enumerate(leaf_qubit):
        by_q.setdefault(q, []).append(i)

    def fold(a, b):
        nonlocal mx
        so = sets[a] ^ sets[b]
        sets.append(so)
        pairs.append((a, b))
        mx = max(mx, len(so))
        return len(sets) - 1

    wires = []
    for q in sorted(by_q):
        ids = by_q[q]
        acc = ids[0]
        for i in ids[1:]:
            acc = fold(acc, i)
        wires.append(acc)
    acc = wires[0]
    for w in wires[1:]:
        acc = fold(acc, w)
    return pairs, mx


def contract_path(leaves, pairs):
    """Contract numeric leaves [(array, legs)] along SSA `pairs`."""
    items = {i: leaf for i, leaf in enumerate(leaves)}
    nxt = len(leaves)
    for (a, b) in pairs:
        (xa, la), (xb, lb) = items.pop(a), items.pop(b)
        shared = [e for e in la if e in lb]
        ax_a = [la.index(e) for e in shared]
        ax_b = [lb.index(e) for e in shared]
        xc = np.tensordot(xa, xb, axes=(ax_a, ax_b))
        lc = [e for e in la if e not in shared] + [e for e in lb if e not in shared]
        items[nxt] = (xc, lc)
        nxt += 1
    (x, legs), = items.values()
    assert not legs
    return complex(x)


class Contractor:
    """Amplitudes and per-slice partial amplitudes of one circuit.

    `sliced`: list of segments (q, j) fixed per slice (slice s sets the i-th
    listed segment to bit i of s). `max_log2`: largest intermediate (in legs)
    the oracle allows itself; it slices extra segments of its own choice to
    stay below it and sums over them.
    """

    def __init__(self, spec_text: str, sliced=(), max_log2: int = 26):
        self.net = WireNetwork(spec_text)
        self.sliced = [tuple(s) for s in sliced]
        net = self.net
        for (q, j) in self.sliced:
            if not (0 <= q < net.n and 0 <= j <= net.n_segments[q]):
                raise ValueError(f"no segment {(q, j)}")
        self.extra = []
        fixed_segs = list(self.sliced)
        leaf_qubit = [net.edge_seg[edges[0]][0] for (_, _, edges) in net.leaves]
        while True:
            legs = self._leg_sets(net.edges_of_segments(fixed_segs))
            pairs, mx = greedy_path(legs)
            p2, m2 = sweep_path(leaf_qubit, legs)
            if m2 < mx:
                pairs, mx = p2, m2
            if mx <= max_log2:
                break
            seg = self._busiest_segment(legs, pairs, mx, fixed_segs)
            if seg is None:
                break
            self.extra.append(seg)
            fixed_segs.append(seg)
        self.pairs = pairs
        self.max_log2 = mx
        self._fixed_segs = fixed_segs

    def _leg_sets(self, fixed_edges):
        return [[e for e in edges if e not in fixed_edges] for (_, _, edges) in self.net.leaves]

    def _busiest_segment(self, legs, pairs, mx, fixed_segs):
        """Extra segment to slice: among the segments in intermediates of >=
        mx-1 legs, the one whose fixing gives the smallest largest
        intermediate along the current order (ties: fewer intermediates at
        that size, then the most frequent segment)."""
        sets = [frozenset(s) for s in legs]
        inter = []
        count = {}
        for (a, b) in pairs:
            so = sets[a] ^ sets[b]
            sets.append(so)
            inter.append(so)
            if len(so) >= mx - 1:
                for seg in {self.net.edge_seg[e] for e in so}:
                    count[seg] = count.get(seg, 0) + (4 if len(so) == mx else 1)
        cands = sorted((c, seg) for seg, c in count.items() if seg not in fixed_segs)[-24:]
        if not cands:
            return None
        best = None
        for c, seg in cands:
            drop = self.net.edges_of_segments([seg])
            sizes = [len(x) - len(x & drop) for x in inter]
            m = max(sizes)
            key = (m, sizes.count(m), -c)
            if best is None or key < best[0]:
                best = (key, seg)
        return best[1]

    def _fixed_map(self, values):
        fixed = {}
        for seg, v in zip(self._fixed_segs, values):
            for e in self.net.edges_of_segments([seg]):
                fixed[e] = v
        return fixed

    def partial(self, bits, slice_id: int) -> complex:
        """Partial amplitude of slice `slice_id` for bitstring `bits`."""
        k = len(self.sliced)
        base = [(slice_id >> i) & 1 for i in range(k)]
        total = 0.0 + 0.0j
        for extra in itertools.product((0, 1), repeat=len(self.extra)):
            leaves = self.net.leaf_values(bits, self._fixed_map(base + list(extra)))
            total += contract_path(leaves, self.pairs)
        return total

    def amplitude(self, bits) -> complex:
        """Full amplitude: the sum of all 2^k partial amplitudes."""
        return sum(self.partial(bits, s) for s in range(1 << len(self.sliced)))


def amplitudes(spec_text: str, bitstrings, max_log2: int = 26) -> np.ndarray:
    c = Contractor(spec_text, (), max_log2)
    return np.array([c.amplitude(x) for x in np.asarray(bitstrings)], dtype=np.complex128)
