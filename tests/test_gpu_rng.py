"""The device random-number generator (the Philox4x32-10 function every trace
kernel samples with) against the generator's published known answers and
against the oracle's own, independently written Philox on random inputs."""
import os

import numpy as np
import pytest

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


def _kat():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([[int(w, 16) for w in part.split()] for part in line.split("|")])
    return rows


def test_device_philox_known_answers(S):
    kat = _kat()
    assert len(kat) == 3
    ctr = np.array([r[0] for r in kat], dtype=np.uint32)
    key = np.array([r[1] for r in kat], dtype=np.uint32)
    expect = np.array([r[2] for r in kat], dtype=np.uint32)
    np.testing.assert_array_equal(S.skirt_philox4x32_10(ctr, key), expect)


def test_device_philox_matches_the_oracle(S, oracle_lib):
    rng = np.random.default_rng(11)
    ctr = rng.integers(0, 2 ** 32, size=(2000, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(2000, 2), dtype=np.uint64).astype(np.uint32)
    out = S.skirt_philox4x32_10(ctr, key)
    ref = np.array([oracle_lib.philox4x32_10(c, k) for c, k in zip(ctr.tolist(), key.tolist())], dtype=np.uint32)
    np.testing.assert_array_equal(out, ref)
