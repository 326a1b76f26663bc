"""The oracle on every host core, for full-size parity tests -- TEST
INFRASTRUCTURE ONLY.  Worker processes are spawned (never forked from a
process that has used CUDA); each builds the workload from its seeded
description, traces its own packet range with the unmodified FP64 oracle and
writes its tables to a temporary file; the tables are summed here."""
from __future__ import annotations

import multiprocessing as mp
import os
import tempfile

import numpy as np


def _work(spec, lo, hi, path):
    import oracle
    from paper_1705_04702_gb300 import workloads as W
    prob = getattr(W, spec["maker"])(**spec["kwargs"])
    r = oracle.trace(prob, lo, hi)
    np.savez(path, absorbed=r["absorbed"], images=r["images_flat"], sed=r["sed"], ledger=r["ledger"],
             status=np.array([r["status"]]))


def trace_all_cores(spec, npackets, cores=None):
    """Traces packets [0, npackets) of every wavelength of the problem
    workloads.<spec['maker']>(**spec['kwargs']) on `cores` processes
    (default: every host core); returns summed absorbed, images_flat, sed,
    ledger and the OR of the status bits."""
    import oracle
    oracle.build()
    cores = cores or os.cpu_count() or 1
    edges = np.linspace(0, npackets, cores + 1).round().astype(np.int64)
    ctx = mp.get_context("spawn")
    tmp = tempfile.mkdtemp(prefix="oracle_pool_")
    paths = [os.path.join(tmp, f"part{i}.npz") for i in range(cores)]
    procs = [ctx.Process(target=_work, args=(spec, int(edges[i]), int(edges[i + 1]), paths[i])) for i in range(cores)]
    for p in procs:
        p.start()
    for p in procs:
        p.join()
    if any(p.exitcode != 0 for p in procs):
        raise RuntimeError("an oracle worker failed")
    out = None
    status = 0
    for path in paths:
        with np.load(path) as z:
            if out is None:
                out = {k: z[k].copy() for k in ("absorbed", "images", "sed", "ledger")}
            else:
                for k in ("absorbed", "images", "sed", "ledger"):
                    out[k] += z[k]
            status |= int(z["status"][0])
        os.unlink(path)
    os.rmdir(tmp)
    out["status"] = status
    out["cores"] = cores
    return out
