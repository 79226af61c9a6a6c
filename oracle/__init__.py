"""CPU FP64 oracle for random-circuit output amplitudes (test infrastructure).

This package is test infrastructure only. Only the tests, the smoke check of
the package entry point and the CPU-baseline leg of the benchmark may import
it; the library itself never does, and this package imports nothing from the
library. It shares only the seeded input generators (`tz_inputs`) with it.

What it computes: the amplitude a(x) = <x| U_C |0^n> of a circuit C built by
the prescription of Sec. 1, in three independent ways:

* `statevector`  -- apply the gates one by one to the 2^n FP64 state.
* `tn`           -- a plain-wire tensor network (every gate, diagonal or not,
                    is a tensor with in/out legs; no hyperedges) contracted
                    pairwise in an order of its own, with optional slicing of
                    wire segments; it gives full amplitudes and the partial
                    amplitude of one slice (Sec. 1: the task split into
                    subtasks whose results add up to the amplitude).
* `pathsum`      -- the amplitude as a sum over the values of every wire
                    segment of the product of gate entries, evaluated by
                    variable elimination in a minimum-fill order of its own
                    (with extra slicing of its own to bound memory); it
                    reaches one slice of a depth 1+32+1 circuit on 49 qubits.
* `linalg`       -- the plain definitions of the per-step operations
                    (bit permutation of a tensor, batched complex matrix
                    product, FP64 sum of scaled partial results).

Pins (tests marked "not gpu"): hand-derived closed forms for one- and
two-qubit circuits, gate identities (H^2 = I, sqrt(X)^2 = X, sqrt(Y)^2 = Y,
unitarity), a dense 2^n x 2^n unitary built from Kronecker products at n <= 5,
the norm sum_x |a(x)|^2 = 1, state vector against both contractors, sliced
sum against unsliced contraction, per-slice partials of the two contractors
against each other and against projector-inserted state vectors, and the
Porter-Thomas moments of Sec. 2. The per-step definitions are pinned by
hand-worked values (tests/golden/linalg_ops.txt), an explicit triple loop and
numpy's axis transpose.
"""
