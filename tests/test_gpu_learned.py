"""The learned form end to end on a small clumpy torus: stellar trace ->
band compression -> exact labels -> training -> surrogate emission with
fallback -> dust re-emission trace."""
import pytest

pytestmark = pytest.mark.gpu


def test_learned_pipeline_small():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1705_04702_gb300 import build
    build.build()
    from paper_1705_04702_gb300.learned import run_learned
    rep = run_learned(n=40, nlambda=40, packet_scale=2e-3, n_train=16000, n_test=3000, epochs=150, batch=512,
                      lr=3e-3, reemit_per_lambda=2000)
    assert rep["loss_first_last"][1] < rep["loss_first_last"][0]
    # held-out cells of this small, sparsely sampled torus (16k training cells,
    # a few packets per cell and wavelength): median within 3% of the exact
    # solver; the 2% bar applies to the full 256^3 run (1e6 training cells)
    assert rep["err_heldout"][50] < 0.03, rep["err_heldout"]
    # the surrogate's spectra carry exactly the absorbed power of their cells
    assert rep["energy_rel_err_surrogate"] < 1e-5
    # the dust source emits what the emission table holds, and the trace closes its ledger
    led = rep["reemission_ledger"]
    assert led["emitted"] == pytest.approx(rep["emitted_dust_luminosity"], rel=1e-6)
    closure = abs(led["emitted"] - led["absorbed"] - led["escaped"] - led["residual"]) / led["emitted"]
    assert closure < 1e-6
    sl = rep["stellar_ledger"]
    assert abs(sl["emitted"] - sl["absorbed"] - sl["escaped"] - sl["residual"]) / sl["emitted"] < 1e-6


def test_surrogate_gains_over_the_exact_solver():
    """What the trained network gains over the method without it: on 400k
    cells of 100 input wavelengths the surrogate emission step (band
    features, tensor-core MLP, exact fallback outside the hull) is faster
    than the exact equilibrium solve, keeps the energy exact and stays within
    2% (median) of it.  (Both read the absorbed table and write the same FP64
    emission rows, so with the exact solve's per-term work in double-float
    the margin is the exact solve's arithmetic: 2.6x measured here.)"""
    import numpy as np
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1705_04702_gb300 import build
    build.build()
    from paper_1705_04702_gb300 import skirt as S
    from paper_1705_04702_gb300 import workloads as W
    lam = np.geomspace(0.09, 10.0, 100)
    n, n_train = 400_000, 40_000
    a, m = W.absorbed_spectra(n, lam, seed=21)
    A = torch.as_tensor(a, dtype=torch.float64, device="cuda")
    M = torch.as_tensor(m, dtype=torch.float32, device="cuda")
    exact = torch.empty((n, 100), dtype=torch.float64, device="cuda")
    S.skirt_dust_emission(A, n, lam.size, lam, M, S.EMIT_EXACT, None, exact)  # warm-up and labels
    feat = torch.empty((n, 32), dtype=torch.float32, device="cuda")
    tot = torch.empty(n, dtype=torch.float64, device="cuda")
    S.skirt_band_features(A, n, lam.size, lam, M, feat, tot)
    net = S.MLP(seed=4)
    net.train(feat[:n_train].contiguous(), exact[:n_train].contiguous(), n_train, epochs=60, batch=1024)
    sur = torch.empty_like(exact)
    S.skirt_dust_emission(A, n, lam.size, lam, M, S.EMIT_SURROGATE, net, sur)  # warm-up

    def timed(mode, out):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record()
        st = S.skirt_dust_emission(A, n, lam.size, lam, M, mode, net if mode == S.EMIT_SURROGATE else None, out)
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]), st

    t_exact, _ = timed(S.EMIT_EXACT, exact)
    t_sur, st = timed(S.EMIT_SURROGATE, sur)
    net.close()
    assert t_sur * 1.5 < t_exact, (t_sur, t_exact, st)
    np.testing.assert_allclose(sur.sum(dim=1).cpu().numpy(), a.sum(axis=1), rtol=1e-5)
    err = (torch.linalg.vector_norm(sur - exact, dim=1) / torch.linalg.vector_norm(exact, dim=1)).cpu().numpy()
    assert np.median(err) < 0.02, np.median(err)
