"""The task split of the paper's multi-process mode (arXiv:1705.04702
Sect. 5.2, task parallelization): every process launches its own share of
every wavelength's packets, and the absorbed, instrument and SED tables of
the processes are summed (one all-reduce) at the end of the phase.

On the device a share is a packet range of the run (skirt_trace_opts
first_packet / total_packets): the packets keep the random streams and the
luminosity they have in the run over all packets, so the summed tables equal
the tables of one call over every packet.  This module holds the host-side
arithmetic of that split only."""
from __future__ import annotations

import numpy as np


def packet_share(npackets, rank, world):
    """(first, count): the packet range of `rank` among `world` processes for
    every wavelength, contiguous ranges covering [0, npackets[j]) once, the
    counts differing by at most one."""
    n = np.asarray(npackets, dtype=np.uint64)
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    lo = (n * np.uint64(rank)) // np.uint64(world)
    hi = (n * np.uint64(rank + 1)) // np.uint64(world)
    return lo.astype(np.uint64), (hi - lo).astype(np.uint64)


def sum_tables(tables, dist=None):
    """Sums a list of tables (numpy FP64 arrays) over the processes of `dist`
    in place (all-reduce; no-op for one process) and returns them."""
    if dist is None or dist.get_world_size() == 1:
        return tables
    import torch
    for i, t in enumerate(tables):
        buf = torch.from_numpy(np.ascontiguousarray(t, dtype=np.float64))
        dist.all_reduce(buf, op=dist.ReduceOp.SUM)
        tables[i] = buf.numpy()
    return tables
