"""Checkpointed slice farm: resume a sliced amplitude computation.

Sec. 1 splits the contraction into subtasks (slices) and sums their results
until all of them add up to the amplitude; a node that fails loses only the
subtasks it had not reported. Here a job is the 2^k slices of one plan for
one batch of bitstrings, cut into fixed ranges of slices. Each rank records
the FP64 partial sum of every range it finishes in its own ledger file
(written to a temporary file, then renamed, so a file is always whole). A
rank that stops between ranges loses nothing it recorded; on the next run
every rank reads all ledgers, skips the ranges already recorded and shares
out the rest. The amplitude is the sum of the range partials in range order,
so it does not depend on which rank did which range, or when.

A ledger carries a key: the digest of everything that fixes the partial
sums (circuit, tree, sliced segments, precision, bitstrings, range size).
Ledgers with another key are refused, never mixed in.
"""
import hashlib
import json
import os

import numpy as np


def job_key(**parts) -> str:
    """Digest of the job's identity: keyword values that are str, int,
    float, lists of them, or numpy arrays (hashed by dtype, shape and bytes)."""
    h = hashlib.sha256()
    for name in sorted(parts):
        v = parts[name]
        h.update(name.encode())
        if isinstance(v, np.ndarray):
            h.update(str((v.dtype.str, v.shape)).encode())
            h.update(np.ascontiguousarray(v).tobytes())
        else:
            h.update(json.dumps(v, sort_keys=True, default=str).encode())
    return h.hexdigest()


def ranges(n_slices: int, chunk: int):
    """The fixed ranges [lo, hi) of the job."""
    if n_slices < 1 or chunk < 1:
        raise ValueError("n_slices and chunk must be >= 1")
    return [(lo, min(n_slices, lo + chunk)) for lo in range(0, n_slices, chunk)]


class SliceLedger:
    """The ranges one rank has finished, with their partial sums."""

    def __init__(self, directory: str, key: str, rank: int):
        self.dir = directory
        self.key = key
        self.rank = rank
        self.path = os.path.join(directory, f"ledger_rank{rank}.json")
        self.done = {}   # (lo, hi) -> complex128 array
        if os.path.exists(self.path):
            self.done = _read(self.path, key)

    def record(self, lo: int, hi: int, partial) -> None:
        """Record the FP64 partial sum of slices [lo, hi) and persist."""
        self.done[(int(lo), int(hi))] = np.asarray(partial, dtype=np.complex128).copy()
        body = {"key": self.key, "rank": self.rank,
                "ranges": [{"lo": lo, "hi": hi, "re": v.real.tolist(), "im": v.imag.tolist()}
                           for (lo, hi), v in sorted(self.done.items())]}
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(body, f)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, self.path)


def _read(path: str, key: str):
    with open(path) as f:
        body = json.load(f)
    if body.get("key") != key:
        raise ValueError(f"{path} belongs to another job (key mismatch); refusing to mix it in")
    return {(r["lo"], r["hi"]): np.array(r["re"]) + 1j * np.array(r["im"]) for r in body["ranges"]}


def recorded(directory: str, key: str):
    """Every range recorded by any rank's ledger in `directory`."""
    out = {}
    if not os.path.isdir(directory):
        return out
    for name in sorted(os.listdir(directory)):
        if name.startswith("ledger_rank") and name.endswith(".json"):
            out.update(_read(os.path.join(directory, name), key))
    return out


def pending(directory: str, key: str, n_slices: int, chunk: int, rank: int, world: int):
    """The ranges not yet recorded by anyone, dealt round-robin: this rank's
    share (the same deal on every rank, since all read the same ledgers)."""
    done = recorded(directory, key)
    todo = [r for r in ranges(n_slices, chunk) if r not in done]
    return todo[rank::world]


def run_ranges(contract_range, directory: str, key: str, n_slices: int, chunk: int, rank: int, world: int,
               sync=None, stop_after=None) -> int:
    """Contract this rank's pending ranges, recording each as it finishes.
    contract_range(lo, hi) returns the FP64 partial sum of slices [lo, hi).
    sync: a barrier over all ranks (e.g. torch.distributed.barrier), called
    once every rank has dealt the pending ranges and before any records one,
    so that all ranks deal from the same ledgers. stop_after: leave after
    that many ranges (a rank that stops between ranges). Returns the number
    of ranges done."""
    os.makedirs(directory, exist_ok=True)
    led = SliceLedger(directory, key, rank)
    mine = pending(directory, key, n_slices, chunk, rank, world)
    if sync is not None:
        sync()
    n = 0
    for (lo, hi) in mine:
        if stop_after is not None and n >= stop_after:
            break
        led.record(lo, hi, contract_range(lo, hi))
        n += 1
    return n


def total(directory: str, key: str, n_slices: int, chunk: int):
    """The amplitudes: the sum of all range partials in range order, or None
    while a range is missing."""
    done = recorded(directory, key)
    acc = None
    for r in ranges(n_slices, chunk):
        if r not in done:
            return None
        acc = done[r].copy() if acc is None else acc + done[r]
    return acc


def plan_range_contractor(tz, plan, bitstrings):
    """contract_range for a bound plan: the FP64 partial amplitudes of
    slices [lo, hi) of `bitstrings` (host arrays), through the C ABI."""
    def contract_range(lo, hi):
        plan.set_slice_range(lo, hi)
        return tz.tz_contract_amplitudes(plan, bitstrings)
    return contract_range
