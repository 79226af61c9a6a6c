"""Random benchmark circuits following the prescription of Sec. 1.

Readings where Sec. 1 leaves things open (fixed here, identically in the C++
generator of the library):

* The eight CZ configurations. Horizontal pattern H_a holds the couplers
  (r,c)-(r,c+1) with c = a + 2*(r mod 2) (mod 4); vertical pattern V_a holds
  (r,c)-(r+1,c) with r = a + 2*(c mod 2) (mod 4), a in 0..3. Within one
  pattern no qubit meets two couplers, and over eight cycles every coupler of
  the lattice is used once. Cycle t (1-based) uses pattern PATTERN_ORDER[(t-1)
  mod 8]. Couplers with an endpoint missing from the lattice are dropped.
* A qubit that is in a CZ in cycle t gets nothing else in cycle t. Otherwise,
  if it was in a CZ in cycle t-1 it gets sqrt(X) or sqrt(Y) at random; else if
  its gate in cycle t-1 was H, sqrt(X) or sqrt(Y) it gets T; else nothing.
  Cycle 0 is the initial H layer, so in cycle 1 every qubit outside a CZ gets T.
* The random choice: one SplitMix64 draw per qubit that needs it, in order of
  cycle then qubit index; the draw's top bit picks sqrt(Y) (1) or sqrt(X) (0).
* A depth "1+t+1" circuit is cycle 0 (H on all), cycles 1..t, and cycle t+1
  (H on all).

Gate names follow the GRCS text files: h, cz, t, x_1_2, y_1_2.
"""
from .splitmix64 import SplitMix64

PATTERN_ORDER = (("h", 0), ("v", 0), ("h", 2), ("v", 2), ("h", 1), ("v", 1), ("h", 3), ("v", 3))


def cz_pattern_edges(lattice, cycle: int):
    """Qubit pairs (q0 < q1) of the CZ layer of 1-based cycle `cycle`."""
    kind, a = PATTERN_ORDER[(cycle - 1) % 8]
    out = []
    for (r, c) in lattice.sites:
        if kind == "h":
            if (c - a - 2 * (r % 2)) % 4 == 0 and (r, c + 1) in lattice.index:
                out.append((lattice.index[(r, c)], lattice.index[(r, c + 1)]))
        else:
            if (r - a - 2 * (c % 2)) % 4 == 0 and (r + 1, c) in lattice.index:
                out.append((lattice.index[(r, c)], lattice.index[(r + 1, c)]))
    return sorted(tuple(sorted(e)) for e in out)


def generate_circuit(lattice, depth_t: int, seed: int):
    """Gate list [(cycle, name, (qubits...)), ...] of a depth 1+t+1 circuit."""
    if depth_t < 0:
        raise ValueError("depth must be >= 0")
    n = lattice.n_qubits
    rng = SplitMix64(seed)
    gates = [(0, "h", (q,)) for q in range(n)]
    prev = ["h"] * n            # gate name on each qubit in the previous cycle, or None
    for t in range(1, depth_t + 1):
        edges = cz_pattern_edges(lattice, t)
        in_cz = [False] * n
        for (a, b) in edges:
            in_cz[a] = in_cz[b] = True
            gates.append((t, "cz", (a, b)))
        cur = [None] * n
        for q in range(n):
            if in_cz[q]:
                cur[q] = "cz"
                continue
            if prev[q] == "cz":
                g = "y_1_2" if rng.next_bit() else "x_1_2"
            elif prev[q] in ("h", "x_1_2", "y_1_2"):
                g = "t"
            else:
                g = None
            if g is not None:
                gates.append((t, g, (q,)))
            cur[q] = g
        prev = cur
    gates.extend((depth_t + 1, "h", (q,)) for q in range(n))
    return gates


def circuit_to_spec(n_qubits: int, gates) -> str:
    """Plain-text spec: first line the qubit count, then one line per gate,
    `cycle name q0 [q1]`, in list order."""
    lines = [str(n_qubits)]
    for (cyc, name, qs) in gates:
        lines.append(" ".join([str(cyc), name] + [str(q) for q in qs]))
    return "\n".join(lines) + "\n"
