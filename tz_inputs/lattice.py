"""Qubit lattices for the benchmark circuits of Sec. 1.

Qubits sit on sites (r, c) of the square lattice. Qubit indices are assigned
in row-major order of the sites (row ascending, then column ascending).
"""
from dataclasses import dataclass, field


@dataclass
class Lattice:
    name: str
    sites: list  # list of (r, c), row-major order; qubit q = sites[q]
    index: dict = field(default_factory=dict)

    def __post_init__(self):
        self.sites = sorted(self.sites)
        self.index = {s: q for q, s in enumerate(self.sites)}

    @property
    def n_qubits(self) -> int:
        return len(self.sites)

    def qubit(self, r: int, c: int):
        return self.index.get((r, c))

    def couplers(self):
        """Nearest-neighbour pairs present on the lattice."""
        out = []
        for (r, c) in self.sites:
            for (dr, dc) in ((0, 1), (1, 0)):
                if (r + dr, c + dc) in self.index:
                    out.append(((r, c), (r + dr, c + dc)))
        return out


def grid(rows: int, cols: int) -> Lattice:
    return Lattice(f"grid{rows}x{cols}", [(r, c) for r in range(rows) for c in range(cols)])


def bristlecone(n: int = 70) -> Lattice:
    """Bristlecone diamond (Sec. 1; circuits of 11 rows).

    Row r in 0..10 holds columns c in [5-m, 6+m] with m = min(r, 10-r):
    row lengths 2,4,6,8,10,12,10,8,6,4,2, i.e. 72 sites. The two sites of the
    widest row that have a single neighbour, (5,0) and (5,11), are the two
    qubits Sec. 1 says can be contracted into their only neighbour; n=70
    drops them.
    """
    if n not in (70, 72):
        raise ValueError("bristlecone lattice has 72 sites (or 70 without the two degree-1 sites)")
    sites = []
    for r in range(11):
        m = min(r, 10 - r)
        for c in range(5 - m, 7 + m):
            sites.append((r, c))
    if n == 70:
        sites = [s for s in sites if s not in ((5, 0), (5, 11))]
    return Lattice(f"bristlecone{n}", sites)
