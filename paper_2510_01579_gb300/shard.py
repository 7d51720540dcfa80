"""Split one slot's detection job across GPUs by contiguous PRB ranges.

The paper spreads a slot's subcarriers evenly over its GPUs, which then run
without any synchronisation (Sec. 3.2, processing flow; Sec. 5.3: execution
time falls as 1 / number of GPUs).  Here a shard is a contiguous range of
physical resource blocks (12 subcarriers each, with all of the slot's OFDM
symbols), so a channel held per subcarrier or per PRB never straddles two
shards, and each shard is an ordinary detection job:

* its problems are a contiguous slice [p0, p1) of the slot's (problem index
  p = subcarrier * n_sym + symbol);
* its channels are the contiguous slice [c0, c1) its problems use, and its
  chan_index is re-based to c0;
* its problem_offset is p0, so its Philox streams, and hence its results, are
  those of the same problems in the whole job.

Host-side index arithmetic only: no data moves and nothing is computed here.
Results are gathered by concatenating the shards' outputs in rank order.
"""
from __future__ import annotations

import numpy as np

SUBCARRIERS_PER_PRB = 12


def prb_ranges(n_prb: int, world: int):
    """[(prb0, prb1)] per rank: contiguous, sizes differing by at most one
    (the first n_prb % world ranks take one more); a rank may get none."""
    if n_prb < 0 or world < 1:
        raise ValueError("n_prb >= 0 and world >= 1 required")
    base, extra = divmod(n_prb, world)
    out, start = [], 0
    for r in range(world):
        size = base + (1 if r < extra else 0)
        out.append((start, start + size))
        start += size
    return out


def shard_problems(n_sub: int, n_sym: int, world: int, rank: int, sc_per_prb: int = SUBCARRIERS_PER_PRB):
    """Problem range [p0, p1) of `rank` for a slot of n_sub subcarriers x
    n_sym symbols; the last PRB may be ragged (n_sub not a multiple of 12)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    n_prb = -(-n_sub // sc_per_prb)
    b0, b1 = prb_ranges(n_prb, world)[rank]
    s0, s1 = min(b0 * sc_per_prb, n_sub), min(b1 * sc_per_prb, n_sub)
    return s0 * n_sym, s1 * n_sym


def shard_channels(chan_index, p0: int, p1: int):
    """(c0, c1, local_chan_index) of the problems [p0, p1): the channels they
    use are [c0, c1) and local_chan_index = chan_index[p0:p1] - c0.  Raises if
    a channel of the shard is also used by a problem outside it (the shard
    would straddle a channel group), or if the shard's channels are not one
    contiguous range."""
    ci = np.asarray(chan_index)
    if p1 <= p0:
        return 0, 0, ci[p0:p0].astype(np.int32)
    part = ci[p0:p1]
    c0, c1 = int(part.min()), int(part.max()) + 1
    rest = np.concatenate([ci[:p0], ci[p1:]])
    if np.any((rest >= c0) & (rest < c1)):
        raise ValueError("a channel of the shard is shared with problems outside it")
    if len(np.unique(part)) != c1 - c0:
        raise ValueError("the shard's channels are not a contiguous range")
    return c0, c1, (part - c0).astype(np.int32)


def shard_slot(chan_index, n_sub: int, n_sym: int, world: int, rank: int):
    """Everything a rank needs for its shard of a slot: dict(p0, p1, c0, c1,
    chan_index) with chan_index re-based to c0."""
    p0, p1 = shard_problems(n_sub, n_sym, world, rank)
    c0, c1, local = shard_channels(chan_index, p0, p1)
    return dict(p0=p0, p1=p1, c0=c0, c1=c1, chan_index=local)
