"""Parser of the plain-text circuit spec (oracle side).

Format: first non-empty line is the qubit count n; each further line is
`cycle name q0 [q1]` with name in {h, cz, t, x_1_2, y_1_2} (the GRCS gate
names of Sec. 1). Lines are applied in file order; gates of one cycle act on
distinct qubits.
"""

ONE_QUBIT = ("h", "t", "x_1_2", "y_1_2")


def parse_spec(text: str):
    lines = [ln.split() for ln in text.splitlines() if ln.strip() and not ln.lstrip().startswith("#")]
    if not lines:
        raise ValueError("empty spec")
    n = int(lines[0][0])
    gates = []
    for toks in lines[1:]:
        cyc, name = int(toks[0]), toks[1]
        qs = tuple(int(t) for t in toks[2:])
        if name in ONE_QUBIT:
            if len(qs) != 1:
                raise ValueError(f"{name} takes one qubit")
        elif name == "cz":
            if len(qs) != 2 or qs[0] == qs[1]:
                raise ValueError("cz takes two distinct qubits")
        else:
            raise ValueError(f"unknown gate {name}")
        if any(q < 0 or q >= n for q in qs):
            raise ValueError("qubit out of range")
        gates.append((cyc, name, qs))
    return n, gates


def segments(n, gates):
    """Wire segments per qubit: segment j of qubit q is the stretch of q's
    wire after its j-th non-diagonal gate (H, sqrt(X), sqrt(Y)); segment 0 is
    the input. Returns, for each gate in order, the segment index each of its
    qubits is on when the gate acts (for non-diagonal gates: the segment it
    ends), plus the final segment count per qubit."""
    cur = [0] * n
    at = []
    for (_, name, qs) in gates:
        at.append(tuple(cur[q] for q in qs))
        if name in ("h", "x_1_2", "y_1_2"):
            cur[qs[0]] += 1
    return at, cur
