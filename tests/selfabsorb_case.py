"""A small self-absorption case shared by the oracle and GPU tests: the
clumpy torus on a 20^3 grid after a short stellar trace by the oracle, and a
dust wavelength table whose IR extinction is raised 20x so that the dust
re-absorbs about 30% of its own emission (seven cycles to converge at 1%)."""
import dataclasses

import numpy as np

from paper_1705_04702_gb300 import workloads as W

PACKETS_PER_LAMBDA = 300
SEED = 5


def stellar_case():
    import oracle
    from oracle import selfabsorb as OSA
    prob = W.torus_problem(n=20, nlambda=6, packet_scale=3e-5, npx=16)
    A = oracle.trace(prob)["absorbed"]
    g = prob.grid
    vol = np.prod([(g.bbox[2 * a + 1] - g.bbox[2 * a]) / n for a, n in enumerate((g.nx, g.ny, g.nz))])
    mass = (g.kr.ravel() * vol).astype(np.float32)
    wl = OSA.dust_wavelengths()
    wl = dataclasses.replace(wl, kscale=wl.kscale * 20.0)
    return prob, A, mass, wl
