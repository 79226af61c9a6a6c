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


@pytest.mark.parametrize("n,w,target", [(4096, 1, 1826), (4096, 1, 1977), (1024, 1, 1024), (1, 1, 3),
                                         (4096, 4, 700), (64, 8, 100), (2, 4, 1)])
def test_step_windows_are_whole(n, w, target):
    """Every timed step contracts the same number of slices: a window that
    ran past the end of the slice range would make the per-slice time look
    shorter than it is."""
    per = shard.window_size(n, w, target)
    assert per & (per - 1) == 0 and 1 <= per <= max(1, target)
    assert per * w <= n or per == 1
    for step in range(12):
        seen = set()
        for r in range(w):
            lo, hi = shard.step_window(n, w, r, per, step)
            assert hi - lo == min(per, n) and 0 <= lo and hi <= n
            if per * w <= n:
                assert not (set(range(lo, hi)) & seen)
                seen |= set(range(lo, hi))


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


# ---------------------------------------------------------------------------
# Checkpointed slice farm (ledger.py): a rank that leaves between ranges
# loses nothing it recorded, and a second run redoes only the rest.

from paper_1907_11217_gb300 import ledger  # noqa: E402


def _farm_worker(rank, world, port, spec, segs, bits, directory, key, chunk, stop_rank, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import tn
    c = tn.Contractor(spec, sliced=segs)
    calls = []

    def contract_range(lo, hi):
        calls.append((lo, hi))
        return np.sum([[c.partial(x, s) for x in bits] for s in range(lo, hi)], axis=0)

    n_slices = 1 << len(segs)
    stop = 1 if rank == stop_rank else None
    ledger.run_ranges(contract_range, directory, key, n_slices, chunk, rank, world, sync=dist.barrier,
                      stop_after=stop)
    # the others learn on the host that the job is incomplete; nothing is
    # left in flight when a rank leaves
    dist.barrier()
    q.put((rank, calls, None if rank else ledger.total(directory, key, n_slices, chunk)))
    dist.destroy_process_group()


def _farm_run(spec, segs, bits, directory, key, chunk, stop_rank):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_farm_worker, args=(r, 2, port, spec, segs, bits, directory, key, chunk,
                                                    stop_rank, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, calls, tot = q.get(timeout=180)
        out[rank] = (calls, tot)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return out


def test_slice_farm_resumes_from_ledgers(tmp_path):
    import tz_inputs as ti
    from oracle import statevector as sv
    spec = ti.circuit_to_spec(12, ti.generate_circuit(ti.grid(3, 4), 12, 3))
    segs = [(1, 2), (5, 3), (7, 2), (10, 1)]
    bits = ti.random_bitstrings(12, 3, 9)
    chunk = 2   # 16 slices in 8 ranges, 4 per rank
    key = ledger.job_key(spec=spec, segs=[list(s) for s in segs], bits=bits, chunk=chunk, precision="oracle")
    d = str(tmp_path / "farm")
    # run 1: rank 1 leaves after its first range
    out1 = _farm_run(spec, segs, bits, d, key, chunk, stop_rank=1)
    assert len(out1[0][0]) == 4 and len(out1[1][0]) == 1
    assert out1[0][1] is None          # incomplete: three ranges missing
    # run 2: only the three missing ranges are contracted, split over both ranks
    out2 = _farm_run(spec, segs, bits, d, key, chunk, stop_rank=-1)
    redone = sorted(out2[0][0] + out2[1][0])
    assert len(redone) == 3 and not set(redone) & set(out1[0][0] + out1[1][0])
    got = out2[0][1]
    ref = sv.amplitudes(spec, bits)
    assert np.max(np.abs(got - ref)) < 1e-14
    # the sum is in range order: the same bits as one run without a stop
    full = tmp_path / "one_run"
    out3 = _farm_run(spec, segs, bits, str(full), key, chunk, stop_rank=-1)
    assert np.array_equal(out3[0][1], got)


def test_ledger_refuses_another_job(tmp_path):
    d = str(tmp_path)
    k1 = ledger.job_key(spec="a", chunk=2)
    k2 = ledger.job_key(spec="b", chunk=2)
    assert k1 != k2
    led = ledger.SliceLedger(d, k1, 0)
    led.record(0, 2, np.array([1.0 + 2.0j]))
    assert ledger.pending(d, k1, 8, 2, 0, 1) == [(2, 4), (4, 6), (6, 8)]
    with pytest.raises(ValueError):
        ledger.recorded(d, k2)
    with pytest.raises(ValueError):
        ledger.SliceLedger(d, k2, 0)
    assert ledger.total(d, k1, 8, 2) is None
    for lo in (2, 4, 6):
        led.record(lo, lo + 2, np.array([1.0]))
    assert ledger.total(d, k1, 8, 2)[0] == 4.0 + 2.0j
