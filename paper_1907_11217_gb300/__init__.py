"""GB300 amplitude library for random quantum circuits (Python binding).

Thin wrappers over the C ABI of include/tz.h: every function marshals
arguments and calls the library; every step of the contraction runs in the
library's CUDA kernels. PyTorch is used only to own device memory (plan
workspaces) and to supply streams.

    import paper_1907_11217_gb300 as tz
    circ = tz.tz_circuit_generate_grid(4, 4, depth=10, seed=1)
    net = tz.tz_network_from_circuit(circ, batch_log2=0)
    tree = tz.tz_path_greedy(net, restarts=8, log2_max_intermediate=28)
    sliced = tz.tz_slice_select(net, tree, 28, 40)
    plan = tz.tz_plan_create(net, tree, sliced, precision="c64")
    plan.bind()                      # workspace from torch's allocator
    amps = tz.tz_contract_amplitudes(plan, bitstrings)   # complex128
"""
import ctypes

import numpy as np

from ._lib import (PROFILE_KINDS, tz_plan_profile, tz_server_opts, PRECISIONS, TZ_BF16X3, TZ_C64_SIMT, TZ_FP16X3, TZ_LATTICE_BRISTLECONE, TZ_LATTICE_GRID, TZ_TF32X3, TzError,
                   check, lib, tz_lattice, tz_network_opts, tz_path_opts, tz_plan_opts, tz_plan_stats)

__all__ = [
    "TzError", "Circuit", "Network", "Tree", "Plan", "tz_circuit_from_spec", "tz_circuit_generate",
    "tz_circuit_generate_grid", "tz_circuit_generate_bristlecone", "tz_network_from_circuit", "tz_path_greedy",
    "tz_tree_from_pairs", "tz_slice_select", "tz_plan_create", "tz_contract_amplitudes",
    "tz_contract_amplitudes_device", "tz_op_permute", "tz_op_cgemm", "tz_op_accumulate", "PRECISIONS",
    "tz_plan_status", "tz_op_cgemm_status", "tz_op_cgemm_static_status", "tz_debug_set_wait_limit",
    "tz_debug_stall_tensor_core", "tz_debug_stall_direct_queue", "tz_tune_tc_pairs", "tz_tune_tc_prefetch", "tz_debug_tune_force_simt", "tz_tune_preset", "tz_debug_stream_tile",
    "TZ_C64_SIMT", "TZ_TF32X3", "TZ_BF16X3", "TZ_FP16X3",
]


def _ptr(x):
    """Device pointer of a torch tensor (or an int)."""
    return ctypes.c_void_p(x if isinstance(x, int) else x.data_ptr())


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(0)
    return ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)


class _Handle:
    _destroy = None

    def __init__(self, h):
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            getattr(lib(), self._destroy)(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Circuit(_Handle):
    _destroy = "tz_circuit_destroy"

    @property
    def n_qubits(self):
        return check(lib().tz_circuit_n_qubits(self._h))

    @property
    def n_gates(self):
        return check(lib().tz_circuit_n_gates(self._h))

    def to_spec(self) -> str:
        n = ctypes.c_size_t()
        rc = lib().tz_circuit_to_spec(self._h, None, 0, ctypes.byref(n))
        buf = ctypes.create_string_buffer(n.value + 1)
        check(lib().tz_circuit_to_spec(self._h, buf, n.value + 1, ctypes.byref(n)))
        del rc
        return buf.value.decode()


def tz_circuit_from_spec(text: str) -> Circuit:
    b = text.encode()
    h = ctypes.c_void_p()
    check(lib().tz_circuit_from_spec(b, len(b), ctypes.byref(h)))
    return Circuit(h)


def tz_circuit_generate(kind: int, rows: int, cols: int, n_qubits: int, depth: int, seed: int) -> Circuit:
    lat = tz_lattice(kind, rows, cols, n_qubits)
    h = ctypes.c_void_p()
    check(lib().tz_circuit_generate(ctypes.byref(lat), depth, seed, ctypes.byref(h)))
    return Circuit(h)


def tz_circuit_generate_grid(rows, cols, depth, seed) -> Circuit:
    return tz_circuit_generate(TZ_LATTICE_GRID, rows, cols, 0, depth, seed)


def tz_circuit_generate_bristlecone(n_qubits, depth, seed) -> Circuit:
    return tz_circuit_generate(TZ_LATTICE_BRISTLECONE, 0, 0, n_qubits, depth, seed)


class Network(_Handle):
    _destroy = "tz_network_destroy"

    def __init__(self, h, n_qubits, batch_log2, open_qubits=()):
        super().__init__(h)
        self.n_qubits = n_qubits
        self.batch_log2 = batch_log2
        self.open_qubits = tuple(sorted(open_qubits))

    @property
    def n_tensors(self):
        return check(lib().tz_network_n_tensors(self._h))

    @property
    def n_indices(self):
        return check(lib().tz_network_n_indices(self._h))

    def index_info(self, i):
        q, s = ctypes.c_int(), ctypes.c_int()
        check(lib().tz_network_index_info(self._h, i, ctypes.byref(q), ctypes.byref(s)))
        return q.value, s.value

    def tensor_indices(self, t):
        buf = (ctypes.c_int32 * 64)()
        r = ctypes.c_int()
        check(lib().tz_network_tensor_indices(self._h, t, buf, 64, ctypes.byref(r)))
        return list(buf[: r.value])


def tz_network_from_circuit(circ: Circuit, batch_log2: int = 0, open_qubits=()) -> Network:
    """open_qubits: output qubits left open; each bitstring then yields the
    2^len(open_qubits) amplitudes of every assignment of their bits (bit j of
    the open value is the j-th smallest open qubit)."""
    arr = np.ascontiguousarray(np.asarray(list(open_qubits), dtype=np.int32))
    ptr = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if len(arr) else None
    o = tz_network_opts(batch_log2, len(arr), ptr)
    h = ctypes.c_void_p()
    check(lib().tz_network_from_circuit(circ.handle, ctypes.byref(o), ctypes.byref(h)))
    return Network(h, circ.n_qubits, batch_log2, arr.tolist())


class Tree(_Handle):
    _destroy = "tz_tree_destroy"

    def pairs(self) -> np.ndarray:
        n = ctypes.c_int()
        lib().tz_tree_pairs(self._h, None, 0, ctypes.byref(n))
        buf = np.zeros(2 * max(n.value, 1), dtype=np.int32)
        check(lib().tz_tree_pairs(self._h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n.value,
                                  ctypes.byref(n)))
        return buf[: 2 * n.value].reshape(-1, 2)


PATH_ALGORITHMS = {"auto": 0, "greedy": 1, "elimination": 2}


def tz_path_greedy(net: Network, restarts=1, seed=0, log2_max_intermediate=0, precision="c64",
                   algorithm="auto", reconfigure=0) -> Tree:
    o = tz_path_opts(restarts, seed, log2_max_intermediate, PRECISIONS.get(precision, precision),
                     PATH_ALGORITHMS.get(algorithm, algorithm), reconfigure)
    h = ctypes.c_void_p()
    check(lib().tz_path_greedy(net.handle, ctypes.byref(o), ctypes.byref(h)))
    return Tree(h)


def tz_tree_from_pairs(net: Network, pairs) -> Tree:
    arr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1))
    h = ctypes.c_void_p()
    check(lib().tz_tree_from_pairs(net.handle, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(arr) // 2,
                                   ctypes.byref(h)))
    return Tree(h)


def tz_slice_select(net: Network, tree: Tree, log2_max_intermediate: int, k_max: int = 40):
    buf = (ctypes.c_int32 * max(k_max, 1))()
    k = ctypes.c_int()
    check(lib().tz_slice_select(net.handle, tree.handle, log2_max_intermediate, k_max, buf, ctypes.byref(k)))
    return list(buf[: k.value])


class Plan(_Handle):
    _destroy = "tz_plan_destroy"

    def __init__(self, h, n_qubits, device):
        super().__init__(h)
        self.n_qubits = n_qubits
        self.device = device
        self.n_open = 0
        self._ws = None

    def stats(self) -> dict:
        s = tz_plan_stats()
        check(lib().tz_plan_stats_get(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in tz_plan_stats._fields_}

    def bind(self, workspace=None):
        """Bind device memory: a torch uint8 tensor, or None to allocate one
        with torch's caching allocator on the plan's device."""
        import torch
        need = self.stats()["workspace_bytes"]
        if workspace is None:
            workspace = torch.empty(need + 256, dtype=torch.uint8, device=f"cuda:{self.device}")
        base = workspace.data_ptr()
        aligned = (base + 255) & ~255
        check(lib().tz_plan_bind_workspace(self._h, ctypes.c_void_p(aligned), workspace.numel() - (aligned - base)))
        self._ws = workspace
        return self

    def set_slice_range(self, lo, hi):
        check(lib().tz_plan_set_slice_range(self._h, lo, hi))

    def sliced_segments(self):
        k = ctypes.c_int()
        lib().tz_plan_sliced_segments(self._h, None, 0, ctypes.byref(k))
        buf = (ctypes.c_int32 * max(2 * k.value, 2))()
        check(lib().tz_plan_sliced_segments(self._h, buf, k.value, ctypes.byref(k)))
        return [(buf[2 * j], buf[2 * j + 1]) for j in range(k.value)]

    def profile_enable(self, on=True):
        check(lib().tz_plan_profile_enable(self._h, int(on)))

    def profile(self) -> dict:
        """Per kernel kind: launches, ms, flops, bytes (synchronises)."""
        pr = tz_plan_profile()
        check(lib().tz_plan_profile_get(self._h, ctypes.byref(pr)))
        return {k: {"launches": pr.launches[i], "ms": pr.ms[i], "flops": pr.flops[i], "bytes": pr.bytes[i]}
                for i, k in enumerate(PROFILE_KINDS)}

    def profile_items(self):
        """Per launch item of a group: dicts with kind, ms, flops, bytes,
        step (GEMM items) and launches, summed over profiled groups."""
        n = ctypes.c_int()
        lib().tz_plan_profile_items(self._h, None, 0, ctypes.byref(n))
        buf = np.zeros(6 * max(n.value, 1))
        check(lib().tz_plan_profile_items(self._h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n.value,
                                          ctypes.byref(n)))
        out = []
        for i in range(n.value):
            k, ms, fl, by, st, cnt = buf[6 * i: 6 * i + 6]
            out.append({"kind": PROFILE_KINDS[int(k)], "ms": ms, "flops": fl, "bytes": by, "step": int(st),
                        "launches": int(cnt)})
        return out

    def describe(self) -> str:
        n = ctypes.c_size_t()
        lib().tz_plan_describe(self._h, None, 0, ctypes.byref(n))
        buf = ctypes.create_string_buffer(n.value + 1)
        check(lib().tz_plan_describe(self._h, buf, n.value + 1, ctypes.byref(n)))
        return buf.value.decode()


def tz_plan_create(net: Network, tree: Tree, sliced=(), precision="c64", device=0, stream=None, small_log2=0,
                   use_graph=False, max_bitstrings=0, autotune=False, direct_queue=False) -> Plan:
    arr = np.ascontiguousarray(np.asarray(list(sliced), dtype=np.int32))
    o = tz_plan_opts(PRECISIONS.get(precision, precision), device, _stream(stream), small_log2, int(use_graph),
                     max_bitstrings, int(autotune), int(direct_queue))
    h = ctypes.c_void_p()
    ptr = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if len(arr) else None
    check(lib().tz_plan_create(net.handle, tree.handle, ptr, len(arr), ctypes.byref(o), ctypes.byref(h)))
    plan = Plan(h, net.n_qubits, device)
    plan.n_open = plan.stats()["n_open"]
    return plan


def tz_contract_amplitudes(plan: Plan, bitstrings) -> np.ndarray:
    """Amplitudes of host bitstrings (n x n_qubits of 0/1) as complex128:
    shape (n,), or (n, 2^n_open) for a plan with open output qubits."""
    b = np.ascontiguousarray(np.asarray(bitstrings, dtype=np.uint8).reshape(-1, plan.n_qubits))
    m = plan.n_open
    out = np.zeros(2 * (len(b) << m), dtype=np.float64)
    check(lib().tz_contract_amplitudes(plan.handle, b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), len(b),
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    amps = out.view(np.complex128)
    return amps.reshape(len(b), 1 << m) if m else amps


def tz_contract_amplitudes_device(plan: Plan, d_bitstrings, d_out):
    """Device form: d_bitstrings (uint8, n x n_qubits) and d_out (float64,
    2n, or 2n * 2^n_open with open output qubits) are torch CUDA tensors;
    asynchronous on the plan's stream."""
    n = d_bitstrings.shape[0]
    check(lib().tz_contract_amplitudes_device(plan.handle, _ptr(d_bitstrings), n, _ptr(d_out)))


def tz_op_permute(d_in, d_out, perm, stream=None):
    arr = np.ascontiguousarray(np.asarray(perm, dtype=np.int32))
    check(lib().tz_op_permute(_ptr(d_in), _ptr(d_out), len(arr), arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                              _stream(stream)))


def tz_op_cgemm_scratch_bytes(precision, batch, m, n, k):
    b = ctypes.c_size_t()
    check(lib().tz_op_cgemm_scratch_bytes(PRECISIONS.get(precision, precision), batch, m, n, k, ctypes.byref(b)))
    return b.value


def tz_op_cgemm(precision, batch, m, n, k, A, sa, B, sb, C, sc, scratch=None, stream=None):
    p = PRECISIONS.get(precision, precision)
    sbytes = 0 if scratch is None else scratch.numel() * scratch.element_size()
    sptr = ctypes.c_void_p(0) if scratch is None else _ptr(scratch)
    check(lib().tz_op_cgemm(p, batch, m, n, k, _ptr(A), sa, _ptr(B), sb, _ptr(C), sc, sptr, sbytes, _stream(stream)))


def tz_op_cgemm_status(precision, scratch=None, stream=None):
    """Synchronise `stream`; raise TzError (TZ_ETIMEOUT) if the last
    tz_op_cgemm on `scratch` timed out in a bounded wait."""
    p = PRECISIONS.get(precision, precision)
    sptr = ctypes.c_void_p(0) if scratch is None else _ptr(scratch)
    check(lib().tz_op_cgemm_status(p, sptr, _stream(stream)))


def tz_op_cgemm_static_status(stream=None):
    check(lib().tz_op_cgemm_static_status(_stream(stream)))


def tz_plan_status(plan: "Plan"):
    """Synchronise the plan's stream; raise TzError (TZ_ETIMEOUT) if a
    tensor-core product of the plan's last call timed out."""
    check(lib().tz_plan_status(plan.handle))


def tz_debug_set_wait_limit(ns: int):
    """Test hook: limit of the products' bounded waits on the current device
    (0 restores the default, 2 s)."""
    check(lib().tz_debug_set_wait_limit(int(ns)))


def tz_debug_stall_tensor_core(on: bool):
    """Test hook: while on, every tensor-core product on the current device
    first waits on a barrier nothing arrives at, so its bounded wait runs out."""
    check(lib().tz_debug_stall_tensor_core(1 if on else 0))


def tz_debug_stall_direct_queue(on: bool):
    """Test hook: while on, the first block of every direct-step queue launch
    on the current device waits on a counter nothing increments, so its
    bounded wait runs out."""
    check(lib().tz_debug_stall_direct_queue(1 if on else 0))


def tz_tune_tc_pairs(mode: int):
    """Process default for the split BF16 / FP16 products: 1 pairs of CTAs
    (cta_group::2) where the shape allows, 0 single CTAs, -1 initial default."""
    check(lib().tz_tune_tc_pairs(int(mode)))


def tz_tune_preset(precision, batch, m, n, k, scatter, pair, ksplit, simt):
    """Preset one autotuner cache entry on the current device (see tz.h)."""
    check(lib().tz_tune_preset(PRECISIONS.get(precision, precision), int(batch), int(m), int(n), int(k),
                               int(scatter), int(pair), int(ksplit), int(simt)))


def tz_debug_stream_tile(batch, m, n, k, pb=None, pm=None, pn=None):
    """Test hook (host only): the stream kernel's tile for a product, as a
    dict, or None where the kernel does not apply. pb, pm, pn: output
    positions of the batch, row and column bits (None: C row-major)."""
    out = (ctypes.c_int32 * 86)()
    sup = ctypes.c_int()
    scatter = pb is not None
    arrs = [np.ascontiguousarray(np.asarray(x if x is not None else [0], dtype=np.int8)) for x in (pb, pm, pn)]
    ptrs = [a.ctypes.data_as(ctypes.c_void_p) for a in arrs]
    check(lib().tz_debug_stream_tile(int(batch), int(m), int(n), int(k), int(scatter), *ptrs,
                                     ctypes.cast(out, ctypes.c_void_p), ctypes.byref(sup)))
    if not sup.value:
        return None
    v = list(out)
    ranks = [(v[6 + 3 * r], v[7 + 3 * r], v[8 + 3 * r]) for r in range(16) if v[6 + 3 * r] >= 0]
    return {"bz": v[0], "bm": v[1], "bn": v[2], "nl": v[3], "kmax": v[4], "smem": v[5], "ranks": ranks,
            "lane_rank": v[54:86]}


def tz_debug_tune_force_simt(on):
    """Test hook: autotuned plans run every small-K tensor-core step on the
    tiled CUDA-core complex64 kernel (on = True or 1), or every small-K
    complex64 step the stream kernel supports on it (on = 2)."""
    check(lib().tz_debug_tune_force_simt(2 if on == 2 else int(bool(on))))


def tz_tune_tc_prefetch(kblocks: int):
    """Process default of the tensor-core products' L2 prefetch distance of
    A tiles, in k-blocks (0 off, -1 initial default)."""
    check(lib().tz_tune_tc_prefetch(int(kblocks)))


def tz_op_accumulate(d_part, d_acc, n, scale=1.0 + 0j, stream=None):
    check(lib().tz_op_accumulate(_ptr(d_part), ctypes.cast(ctypes.c_void_p(d_acc.data_ptr()),
                                                           ctypes.POINTER(ctypes.c_double)),
                                 n, float(np.real(scale)), float(np.imag(scale)), _stream(stream)))


class Server(_Handle):
    """Amplitude server over resident plans (continuous batching): queries
    are admitted while a slot and enough of the arena are free and run
    concurrently on separate streams."""
    _destroy = "tz_server_destroy"

    def __init__(self, h, arena):
        super().__init__(h)
        self._arena = arena

    def submit(self, plan: "Plan", bitstrings) -> int:
        b = np.ascontiguousarray(np.asarray(bitstrings, dtype=np.uint8).reshape(-1, plan.n_qubits))
        t = ctypes.c_uint64()
        check(lib().tz_server_submit(self._h, plan.handle, b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), len(b),
                                     ctypes.byref(t)))
        self._rows = getattr(self, "_rows", {})
        self._rows[t.value] = (len(b), plan.n_open)
        return t.value

    def poll(self, ticket: int):
        """complex128 amplitudes once the query is done, else None (shape
        (n,), or (n, 2^n_open) for a plan with open output qubits)."""
        n, m = self._rows[ticket]
        out = np.zeros(2 * (n << m), dtype=np.float64)
        done = ctypes.c_int()
        check(lib().tz_server_poll(self._h, ticket, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   ctypes.byref(done)))
        if done.value:
            del self._rows[ticket]
            amps = out.view(np.complex128)
            return amps.reshape(n, 1 << m) if m else amps
        return None

    def latency(self):
        p50, p99, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        check(lib().tz_server_latency(self._h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(n)))
        return p50.value, p99.value, n.value


def tz_server_create(arena_bytes, max_inflight=4, device=0, hbm_budget=0, wait_admit=True, arena=None,
                     chunk_ms=0.0) -> Server:
    """Server with a device arena of arena_bytes (a torch uint8 tensor is
    allocated when `arena` is None); queries run in chunks of about chunk_ms
    of estimated work (0: the default, 4 ms) and yield between chunks."""
    import torch
    if arena is None:
        arena = torch.empty(arena_bytes + 256, dtype=torch.uint8, device=f"cuda:{device}")
    base = arena.data_ptr()
    aligned = (base + 255) & ~255
    o = tz_server_opts(hbm_budget, max_inflight, device, ctypes.c_void_p(aligned), arena_bytes, int(wait_admit),
                       float(chunk_ms))
    h = ctypes.c_void_p()
    check(lib().tz_server_create(ctypes.byref(o), ctypes.byref(h)))
    return Server(h, arena)
