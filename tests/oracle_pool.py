"""The oracle on every host core, for full-size parity tests -- TEST
INFRASTRUCTURE ONLY.  Worker processes are spawned (never forked from a
process that has used CUDA); each builds the workload from its seeded
description, traces its own packet range with the unmodified FP64 oracle and
writes its tables to a temporary file; the tables are summed here.  The
workers' packet ranges are also the batches of a batch-means estimate of the
Monte Carlo variance of every table entry."""
from __future__ import annotations

import multiprocessing as mp
import os
import tempfile

import numpy as np


def _work(spec, lo, hi, nrec, path):
    import oracle
    from paper_1705_04702_gb300 import workloads as W
    prob = getattr(W, spec["maker"])(**spec["kwargs"])
    r = oracle.trace(prob, lo, hi, nrec=nrec)
    np.savez(path, absorbed=r["absorbed"], images=r["images_flat"], sed=r["sed"], ledger=r["ledger"],
             records=r["records"], status=np.array([r["status"]]))


def trace_all_cores(spec, npackets, cores=None, nrec=0):
    """Traces packets [0, npackets) of every wavelength of the problem
    workloads.<spec['maker']>(**spec['kwargs']) on `cores` processes
    (default: every host core).  Returns the summed absorbed, images_flat,
    sed and ledger; absorbed_var, the batch-means variance of every absorbed
    entry over the workers' ranges; images_parts, each worker's images_flat;
    records of packets [0, nrec) (traced by the first worker, nrec <= its
    range); status (OR of the workers' bits); cores."""
    import oracle
    oracle.build()
    cores = cores or os.cpu_count() or 1
    edges = np.linspace(0, npackets, cores + 1).round().astype(np.int64)
    assert nrec <= edges[1]
    ctx = mp.get_context("spawn")
    tmp = tempfile.mkdtemp(prefix="oracle_pool_")
    paths = [os.path.join(tmp, f"part{i}.npz") for i in range(cores)]
    procs = [ctx.Process(target=_work, args=(spec, int(edges[i]), int(edges[i + 1]), nrec if i == 0 else 0, paths[i]))
             for i in range(cores)]
    for p in procs:
        p.start()
    for p in procs:
        p.join()
    if any(p.exitcode != 0 for p in procs):
        raise RuntimeError("an oracle worker failed")
    out = None
    sq = None
    parts = []
    status = 0
    for i, path in enumerate(paths):
        with np.load(path) as z:
            if out is None:
                out = {k: z[k].copy() for k in ("absorbed", "images", "sed", "ledger")}
                sq = z["absorbed"] ** 2
                out["records"] = z["records"].copy()
            else:
                for k in ("absorbed", "images", "sed", "ledger"):
                    out[k] += z[k]
                sq += z["absorbed"] ** 2
            parts.append(z["images"].copy())
            status |= int(z["status"][0])
        os.unlink(path)
    os.rmdir(tmp)
    B = float(cores)
    # variance of the sum of B batches: B/(B-1) sum_b (x_b - x/B)^2 = B/(B-1) (sum_b x_b^2 - x^2/B)
    out["absorbed_var"] = np.maximum(B / (B - 1.0) * (sq - out["absorbed"] ** 2 / B), 0.0) if cores > 1 else None
    out["images_parts"] = parts
    out["status"] = status
    out["cores"] = cores
    return out
