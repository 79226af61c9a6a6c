"""Slice sharding across ranks (one process per GPU).

Slices are independent subtasks with no shared data (Sec. 2), so ranks
split the slice range and exchange nothing but their FP64 partial sums
(Sec. 1: subtask results add up to the amplitude): one all-reduce of 2n
doubles per call.
"""


def partition(n_slices: int, world: int, rank: int):
    """Contiguous block of slices [lo, hi) owned by `rank` (sizes differ by at
    most one slice)."""
    if world < 1 or not 0 <= rank < world or n_slices < 0:
        raise ValueError("bad partition request")
    base, extra = divmod(n_slices, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def window_size(n_slices: int, world: int, target: int):
    """Slices per rank and step: the largest power of two <= target (at
    least 1) that lets every rank take a whole window of its own. Slice
    counts are powers of two (2^k), so such windows tile the slice range and
    no step is ever cut short at its end."""
    per = max(1, min(int(target), max(1, n_slices // max(world, 1))))
    return 1 << (per.bit_length() - 1)


def step_window(n_slices: int, world: int, rank: int, per_rank: int, step: int):
    """Slices [lo, hi) a rank contracts in one timed step when every rank
    takes `per_rank` consecutive slices and successive steps move on through
    the range (wrapping). A window always holds min(per_rank, n_slices)
    slices: one that would run past the end of the range is moved back to
    end there (with window_size's windows that never happens)."""
    if per_rank < 1:
        raise ValueError("per_rank must be >= 1")
    n = max(n_slices, 1)
    per = min(per_rank, n)
    lo = ((step * world + rank) * per) % n
    lo = min(lo, n - per)
    return lo, lo + per


def reduce_partials(t):
    """Sum a tensor of FP64 partial amplitudes over all ranks in place (no-op
    without an initialised process group of more than one rank)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t
