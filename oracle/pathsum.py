"""FP64 path-sum contractor over wire-segment variables (oracle part 3).

Test infrastructure: only the tests, the package's smoke check and the
benchmark's CPU-baseline leg use it; it imports nothing from the library.

The amplitude as a sum over paths. Write the circuit's state on each wire as
a basis value that changes only at a non-diagonal gate (H, sqrt(X),
sqrt(Y)); between two such gates the value is one variable, the wire
*segment* (q, j) (segment 0 is the input, segment j follows the qubit's j-th
non-diagonal gate; the same segments as the plain-wire contractor's). Then

    a(x) = <x| U_L ... U_1 |0^n>
         = sum over every segment value of  prod_gates (gate entry)
                                           * prod_q [segment (q, 0) = 0]
                                           * prod_q [last segment of q = x_q]

with one factor per gate: U[v_new, v_old] for a non-diagonal U on two
consecutive segments of its qubit, (1, exp(i pi/4))[v] for T on the current
segment, and (-1)^(v_a v_b) for CZ on the current segments of its qubits
(diagonal gates keep the basis value, so they only multiply). This is the
matrix product written out entry by entry; nothing else enters.

Slicing (Sec. 1: subtasks whose results add up to the amplitude): fixing the
variables of some segments to given values and summing over the rest gives
the partial amplitude of that slice; the 2^k slices add up to the amplitude.

Evaluation is textbook variable elimination: in an order of its own (greedy
minimum fill-in on the graph whose vertices are the free variables, adjacent
when they share a factor; ties by fewer neighbours, then the lowest
variable), each variable's factors are multiplied together and the variable
is summed out (numpy einsum in complex128 is the primitive). When the order's
largest factor exceeds 2^max_log2 entries, it fixes extra variables of its
own choice (the one in most of the largest factors) and sums over their
values too.
"""
import itertools

import numpy as np

from .gates import ONE_QUBIT
from .spec import parse_spec

CZ_PHASE = np.array([[1.0, 1.0], [1.0, -1.0]], dtype=np.complex128)   # (-1)^(v_a v_b)


class SegmentSum:
    """Factors of the path sum of one circuit, with the output bits left
    symbolic. Variables are (qubit, segment) pairs."""

    def __init__(self, spec_text: str):
        n, gates = parse_spec(spec_text)
        self.n = n
        cur = [0] * n
        # (array, variables); arrays are indexed in variable order
        self.gate_factors = []
        for (_, name, qs) in gates:
            if name == "cz":
                a, b = qs
                self.gate_factors.append((CZ_PHASE, ((a, cur[a]), (b, cur[b]))))
            elif name == "t":
                q = qs[0]
                self.gate_factors.append((np.diag(ONE_QUBIT["t"]).copy(), ((q, cur[q]),)))
            else:
                q = qs[0]
                self.gate_factors.append((ONE_QUBIT[name], ((q, cur[q] + 1), (q, cur[q]))))
                cur[q] += 1
        self.last = cur[:]   # last segment per qubit
        self.variables = [(q, j) for q in range(n) for j in range(cur[q] + 1)]

    def factors(self, bits):
        """All factors for output bitstring `bits`: the gates', the input
        projections [v = 0] and the output projections [v = x_q]."""
        fs = list(self.gate_factors)
        for q in range(self.n):
            fs.append((np.array([1.0, 0.0], dtype=np.complex128), ((q, 0),)))
            e = np.zeros(2, dtype=np.complex128)
            e[int(bits[q])] = 1.0
            fs.append((e, ((q, self.last[q]),)))
        return fs


def fix(factors, values):
    """Index-select every factor at the fixed variables (dict var -> 0/1)."""
    out = []
    for arr, vs in factors:
        idx = tuple(values[v] if v in values else slice(None) for v in vs)
        out.append((np.asarray(arr[idx]), tuple(v for v in vs if v not in values)))
    return out


def min_fill_order(var_sets):
    """Greedy minimum fill-in elimination order over the variables of the
    given factor scopes. Returns (order, width): width = the largest number
    of variables of a factor the elimination creates, the eliminated one
    included."""
    adj = {}
    for vs in var_sets:
        for v in vs:
            adj.setdefault(v, set()).update(w for w in vs if w != v)

    def fill(v):
        nb = list(adj[v])
        return sum(1 for i in range(len(nb)) for j in range(i + 1, len(nb)) if nb[j] not in adj[nb[i]])

    score = {v: (fill(v), len(adj[v]), v) for v in adj}
    order, width = [], 0
    while score:
        v = min(score.values())[2]
        nb = adj.pop(v)
        del score[v]
        order.append(v)
        width = max(width, len(nb) + 1)
        for a in nb:
            adj[a].discard(v)
            adj[a].update(w for w in nb if w != a)
        # fill-in changes only for the neighbours and their neighbours
        touched = set(nb)
        for a in nb:
            touched |= adj[a]
        for a in touched:
            score[a] = (fill(a), len(adj[a]), a)
    return order, width


def eliminate(factors, order):
    """Sum out the variables in `order`, each by multiplying its factors
    together (einsum) and summing over its value; the remaining scalars are
    multiplied. Returns the complex sum."""
    fs = [(np.asarray(a, dtype=np.complex128), tuple(vs)) for a, vs in factors]
    for v in order:
        bucket = [f for f in fs if v in f[1]]
        if not bucket:
            continue
        fs = [f for f in fs if v not in f[1]]
        keep = []
        for _, vs in bucket:
            for w in vs:
                if w != v and w not in keep:
                    keep.append(w)
        label = {w: i for i, w in enumerate(keep + [v])}   # einsum takes at most 52 labels
        ops = []
        for a, vs in bucket:
            ops += [a, [label[w] for w in vs]]
        res = np.einsum(*ops, [label[w] for w in keep], optimize="greedy")
        fs.append((res, tuple(keep)))
    total = 1.0 + 0.0j
    for a, vs in fs:
        assert not vs, "variable left after elimination"
        total *= complex(a)
    return total


class SegmentContractor:
    """Amplitudes and per-slice partial amplitudes by the path sum.

    `sliced`: segments (q, j) fixed per slice (slice s sets the i-th listed
    segment to bit i of s). `max_log2`: the largest factor (in variables) the
    elimination may create; extra segments of its own choice are fixed and
    summed over to stay within it.
    """

    def __init__(self, spec_text: str, sliced=(), max_log2: int = 25):
        self.ss = SegmentSum(spec_text)
        self.sliced = [tuple(s) for s in sliced]
        known = set(self.ss.variables)
        for s in self.sliced:
            if s not in known:
                raise ValueError(f"no segment {s}")
        if len(set(self.sliced)) != len(self.sliced):
            raise ValueError("repeated sliced segment")
        self.extra = []
        # the output and input projections fix their segments; the order is
        # taken over the gate factors with every fixed variable removed
        ends = {(q, 0) for q in range(self.ss.n)} | {(q, self.ss.last[q]) for q in range(self.ss.n)}
        while True:
            fixed = set(self.sliced) | set(self.extra)
            scopes = [tuple(v for v in vs if v not in fixed) for _, vs in self.ss.gate_factors]
            scopes += [(v,) for v in ends if v not in fixed]
            order, width = min_fill_order(scopes)
            if width - 1 <= max_log2:
                break
            self.extra.append(self._busiest(scopes, order, width))
        self.order = order
        self.width = width

    @staticmethod
    def _busiest(scopes, order, width):
        """The variable in the most factors of the largest size created along
        the order (ties: the lowest variable)."""
        adj = {}
        for vs in scopes:
            for v in vs:
                adj.setdefault(v, set()).update(w for w in vs if w != v)
        count = {}
        for v in order:
            nb = adj.pop(v)
            if len(nb) + 1 >= width - 1:
                for w in nb | {v}:
                    count[w] = count.get(w, 0) + 1
            for a in nb:
                adj[a].discard(v)
                adj[a].update(w for w in nb if w != a)
        return min(count, key=lambda w: (-count[w], w))

    def partial(self, bits, slice_id: int) -> complex:
        """Partial amplitude of slice `slice_id` for bitstring `bits`."""
        k = len(self.sliced)
        base = {seg: (slice_id >> i) & 1 for i, seg in enumerate(self.sliced)}
        fs = self.ss.factors(bits)
        total = 0.0 + 0.0j
        for vals in itertools.product((0, 1), repeat=len(self.extra)):
            fixed = dict(base)
            fixed.update(zip(self.extra, vals))
            total += eliminate(fix(fs, fixed), self.order)
        assert k == len(base)
        return total

    def amplitude(self, bits) -> complex:
        """Full amplitude: the sum of all 2^k partial amplitudes."""
        return sum(self.partial(bits, s) for s in range(1 << len(self.sliced)))


def amplitudes(spec_text: str, bitstrings, max_log2: int = 25) -> np.ndarray:
    c = SegmentContractor(spec_text, (), max_log2)
    return np.array([c.amplitude(x) for x in np.asarray(bitstrings)], dtype=np.complex128)
