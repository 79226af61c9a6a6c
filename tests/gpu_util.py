"""Helpers shared by the GPU tests: plan construction through the C ABI and
the amplitude error measure.

Error measure: amplitudes of an n-qubit random circuit have the
Porter-Thomas scale 2^(-n/2); FP32 rounding errors of a contraction scale
with the magnitudes of the summed terms, i.e. with that scale, not with a
single (possibly tiny) amplitude. The relative error of amplitude j is
|a_gpu - a_ref| / max(|a_ref|, 2^(-n/2)).
"""
import numpy as np

import tz_inputs as ti


def rel_err(got, ref, n_qubits):
    got, ref = np.asarray(got), np.asarray(ref)
    floor = 2.0 ** (-n_qubits / 2)
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor)))


def make_plan(tz, spec, batch_log2=0, log2_max=0, precision="c64", small_log2=0, restarts=4, seed=1,
              use_graph=False, stream=None, k_max=8, max_bitstrings=0, slice_bits=0, open_qubits=(),
              direct_queue=False):
    """log2_max > 0: slice down to that size; slice_bits > 0: slice until the
    largest intermediate is slice_bits below the unsliced one."""
    c = tz.tz_circuit_from_spec(spec)
    net = tz.tz_network_from_circuit(c, batch_log2, open_qubits)
    tree = tz.tz_path_greedy(net, restarts=restarts, seed=seed, log2_max_intermediate=log2_max, precision=precision)
    if slice_bits > 0:
        full = tz.tz_plan_create(net, tree, []).stats()["max_log2"]
        log2_max = full - slice_bits
    sl = tz.tz_slice_select(net, tree, log2_max, k_max) if log2_max > 0 else []
    plan = tz.tz_plan_create(net, tree, sl, precision=precision, small_log2=small_log2, use_graph=use_graph,
                             stream=stream, max_bitstrings=max_bitstrings, direct_queue=direct_queue)
    plan.bind()
    return plan, net, tree, sl


def grid_spec(rows, cols, t, seed):
    return ti.circuit_to_spec(rows * cols, ti.generate_circuit(ti.grid(rows, cols), t, seed))


def rel_err_partial(got, ref, n_qubits, k):
    """rel_err for the partial amplitude of one of 2^k slices: the partials
    of random circuits sit near 2^(-(n+k)/2) (2^k terms of random phase add
    up to an amplitude of 2^(-n/2)), which is the floor here."""
    return rel_err(got, ref, n_qubits + k)


def expand_open(bits, open_qubits):
    """Every bitstring with each assignment of the open qubits: row
    r * 2^m + o has bit j of o on the j-th smallest open qubit (the order of
    the amplitudes a plan with open output qubits returns)."""
    oq = sorted(open_qubits)
    m = len(oq)
    out = np.repeat(np.asarray(bits, dtype=np.uint8), 1 << m, axis=0)
    o = np.tile(np.arange(1 << m), len(bits))
    for j, q in enumerate(oq):
        out[:, q] = (o >> j) & 1
    return out
