"""One integration split in time across ranks (Sec. 2.3.2), and the host-staged visibility sum.

The paper's cluster hands consecutive time slices of every antenna's stream to different
nodes (with an overlap of the largest delay, so that each slice's delays can be applied in
full) and sums the partial visibilities of a split integration in a tree (Sec. 2.3.2).  Here a
rank correlates the frames ``frame_slice(n_int, world, rank)`` of an integration with its own
handle -- created for that many frames, fed the slice's samples plus the delay overlap, and
started at the global frame index of its first frame so that the Eq. 2 fringe phase runs on
-- and ``reduce_visibilities`` sums the ranks' visibilities on the host.

The sum goes through a key-value store (``torch.distributed`` TCPStore or FileStore):
every rank publishes its array under a key of the step and waits, with a bound, for the keys
of all the others, then adds them in rank order, so every rank holds the same bits.  A rank
that has left (or never arrives) is noticed on the host by that bounded wait, before any
further launch, and raises ``RankTimeout``; no collective is left half-entered.  The int8 form
is summed as int32 integer visibilities (exact: the same scales on every rank), the FP32 forms
as float32.
"""
from __future__ import annotations

import datetime

import numpy as np

CORR_E_TIMEOUT = -8                 # the C ABI's code for a wait that ran out


class RankTimeout(RuntimeError):
    """A rank's part of a split integration did not arrive within the timeout."""

    def __init__(self, missing, step):
        super().__init__(f"CORR_E_TIMEOUT: rank(s) {sorted(missing)} did not publish step {step}")
        self.code = CORR_E_TIMEOUT
        self.missing = sorted(missing)
        self.step = step


def frame_slice(n_int: int, world: int, rank: int):
    """(first frame, frame count) of rank's share of an n_int-frame integration: equal slices
    of a multiple of 16 frames (the handle's granularity), the remainder to the last ranks."""
    if world < 1 or not 0 <= rank < world or n_int % 16:
        raise ValueError("need 0 <= rank < world and n_int a multiple of 16")
    units = n_int // 16
    base, extra = divmod(units, world)
    if base == 0:
        raise ValueError("fewer 16-frame units than ranks")
    first = rank * base + max(0, rank - (world - extra))
    count = base + (1 if rank >= world - extra else 0)
    return 16 * first, 16 * count


def sample_slice(n_int: int, n_fft: int, world: int, rank: int, max_delay: int):
    """(first sample, sample count) a rank reads: its frames plus the delay overlap."""
    t0, nt = frame_slice(n_int, world, rank)
    return t0 * n_fft, nt * n_fft + max_delay


def reduce_visibilities(vis: np.ndarray, store, step: int, world: int, rank: int,
                        timeout_s: float = 30.0, prefix: str = "corr-vis") -> np.ndarray:
    """Sum of every rank's `vis` (the same shape and dtype on each: complex64 / float32, or int32
    integer visibilities), the same on every rank.  Raises RankTimeout when a rank's part does not
    arrive within timeout_s seconds."""
    arr = np.ascontiguousarray(vis)
    header = f"{arr.dtype.str}|{','.join(str(d) for d in arr.shape)}|".encode()
    store.set(f"{prefix}/{step}/{rank}", header + arr.tobytes())
    others = [r for r in range(world) if r != rank]
    keys = [f"{prefix}/{step}/{r}" for r in others]
    if keys:
        try:
            store.wait(keys, datetime.timedelta(seconds=timeout_s))
        except Exception as e:          # the store's own timeout error
            missing = [r for r, k in zip(others, keys) if not store.check([k])]
            raise RankTimeout(missing or others, step) from e
    total = None
    for r in range(world):                              # rank order: the same sum on every rank
        if r == rank:
            part = arr
        else:
            raw = store.get(f"{prefix}/{step}/{r}")
            dt, shape, body = raw.split(b"|", 2)
            if dt.decode() != arr.dtype.str or shape.decode() != ",".join(str(d) for d in arr.shape):
                raise ValueError(f"rank {r} published a {dt.decode()} array of shape ({shape.decode()})")
            part = np.frombuffer(body, dtype=arr.dtype).reshape(arr.shape)
        total = part.copy() if total is None else total + part
    return total
