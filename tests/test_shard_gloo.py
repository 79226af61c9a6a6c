"""Multi-rank path on CPU: two gloo ranks each sum the partial amplitudes of
their own block of slices (oracle contractor, Sec. 1 subtasks), the FP64
partial sums are all-reduced, and the result equals the full amplitude."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1907_11217_gb300 import shard


def test_partition_covers_and_is_disjoint():
    for n in (1, 7, 8, 1024, 1000):
        for w in (1, 2, 3, 8):
            blocks = [shard.partition(n, w, r) for r in range(w)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            for (a, b), (c, d) in zip(blocks, blocks[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.partition(8, 2, 2)


def test_step_windows_of_ranks_are_disjoint_within_a_step():
    n, w, per = 64, 4, 4
    for step in range(5):
        seen = set()
        for r in range(w):
            lo, hi = shard.step_window(n, w, r, per, step)
            s = set(range(lo, hi))
            assert not (s & seen)
            seen |= s


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, spec, segs, bits, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import tn
    c = tn.Contractor(spec, sliced=segs)
    lo, hi = shard.partition(1 << len(segs), world, rank)
    part = np.zeros(len(bits), dtype=np.complex128)
    for s in range(lo, hi):
        part += np.array([c.partial(x, s) for x in bits])
    t = torch.from_numpy(part.view(np.float64).copy())
    shard.reduce_partials(t)
    if rank == 0:
        q.put(t.numpy().view(np.complex128).copy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_full_amplitude():
    import tz_inputs as ti
    from oracle import statevector as sv
    spec = ti.circuit_to_spec(12, ti.generate_circuit(ti.grid(3, 4), 12, 3))
    segs = [(1, 2), (5, 3), (7, 2), (10, 1)]
    bits = ti.random_bitstrings(12, 3, 9)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, spec, segs, bits, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref = sv.amplitudes(spec, bits)
    assert np.max(np.abs(got - ref)) < 1e-14
