"""Parity at full size: the 256^3 exponential-disk workload with 1e8 packets,
traced in the launch configuration the benchmark times (mixed form,
persistent launch replayed from a CUDA graph).  The oracle replays the first
packets of the same streams one by one; the tallies are checked through
properties that hold at any size."""
import math

import numpy as np
import pytest

from paper_1705_04702_gb300 import workloads as W

from parity import REL_MIXED_PACKET, compare_records

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1705_04702_gb300 import build
    build.build()
    from paper_1705_04702_gb300 import skirt
    return skirt


def test_disk_1e8_packets_sampled(S, oracle_lib):
    prob = W.disk_problem(100_000_000, n=256, nlambda=1, npx=512)
    nrec = 3000
    g = S.run_problem(prob, precision=S.PREC_MIXED, schedule=S.SCHED_PERSISTENT, nrec=nrec, use_graph=True)
    r = oracle_lib.trace(prob, 0, nrec, nrec=nrec)
    compare_records(g["records"].cpu().numpy(), r["records"], prob, REL_MIXED_PACKET, 0.999, same_n_min=0.999)

    led = g["ledger"]
    assert g["status"] == S.OK and led["status_bits"] == 0
    # every packet was launched with L0 = 1/N
    assert led["emitted"] == pytest.approx(1.0, rel=1e-6)
    closure = abs(led["emitted"] - led["absorbed"] - led["escaped"] - led["residual"]) / led["emitted"]
    assert closure < 1e-6
    # the absorbed table holds the deposits the ledger books
    assert float(g["absorbed"].sum()) == pytest.approx(led["absorbed"], rel=1e-6)
    assert float(g["absorbed"].min()) >= 0.0
    # the SED of every instrument is its image plus the out-of-frame peel-offs
    for q, img in enumerate(g["images"]):
        s_img = float(img.sum())
        assert s_img <= float(g["sed"][q, 0]) * (1 + 1e-12)
        assert s_img >= 0.9 * float(g["sed"][q, 0])
    # work counters match the oracle's per-packet averages on the sample
    c = r["counters"] / nrec
    assert led["scatterings"] / 1e8 == pytest.approx(c[0], rel=0.05)
    assert led["peel_steps"] / 1e8 == pytest.approx(c[3], rel=0.05)
    # the face-on SED is dominated by direct starlight: flux ~ L e^{-tau}/(4 pi d^2)
    F = 1.0 / (4 * math.pi * 100.0 ** 2)
    assert 0.3 * F < float(g["sed"][0, 0]) < 1.5 * F
