"""GPU parity of the dust-emission step and of its MLP surrogate (band
compression, exact FP64 solver, training gradients, tensor-core inference,
hull fallback) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import emission as E
from paper_1705_04702_gb300 import workloads as W

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


def _dev(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.fixture(scope="module")
def fields():
    lam = np.geomspace(0.09, 10.0, 200)
    a, m = W.absorbed_spectra(3000, lam, seed=5)
    a[:3] = 0.0          # cells without absorbed power
    m[3:6] = 0.0         # dust-free cells
    return lam, a, m


def test_band_features_match_oracle(S, fields):
    import torch
    lam, a, m = fields
    n = a.shape[0]
    feat = torch.zeros((n, 32), dtype=torch.float32, device="cuda")
    tot = torch.zeros(n, dtype=torch.float64, device="cuda")
    S.skirt_band_features(_dev(a, torch.float64), n, lam.size, lam, _dev(m, torch.float32), feat, tot)
    B, x, total = E.band_features(a, lam, m.astype(np.float64))
    np.testing.assert_allclose(tot.cpu().numpy(), total, rtol=1e-13, atol=0)
    # FP32 log10 of the FP64 band power per unit mass, stored as FP32: a few ulp
    np.testing.assert_allclose(feat.cpu().numpy(), x, rtol=3e-7, atol=1e-6)


def test_band_features_into_an_unaligned_table(S, fields):
    """Features written through a pointer that is 4 bytes past a 16-byte
    boundary (a view one float into a buffer) equal the aligned result."""
    import torch
    lam, a, m = fields
    n = a.shape[0]
    ad, md = _dev(a, torch.float64), _dev(m, torch.float32)
    feat = torch.zeros((n, 32), dtype=torch.float32, device="cuda")
    tot = torch.zeros(n, dtype=torch.float64, device="cuda")
    S.skirt_band_features(ad, n, lam.size, lam, md, feat, tot)
    buf = torch.zeros(n * 32 + 1, dtype=torch.float32, device="cuda")
    tot2 = torch.zeros(n, dtype=torch.float64, device="cuda")
    S.skirt_band_features(ad, n, lam.size, lam, md, buf[1:], tot2)
    assert buf[1:].data_ptr() % 16 == 4
    assert torch.equal(buf[1:].view(n, 32), feat) and torch.equal(tot2, tot) and buf[0].item() == 0.0


def test_band_features_with_empty_cell_runs(S):
    """Runs of 32 empty cells (a warp's rows) skip the FP64 adds of their
    staged blocks; the band closures still run. Cases: whole empty tiles,
    a tile whose only power starts in its second column block, one whose
    power ends in its first block, one whose power sits in the ragged last
    block (200 = 6 x 32 + 8 columns), and an empty ragged tail of 13 cells."""
    import torch
    lam = np.geomspace(0.09, 10.0, 200)
    n = 32 * 8 + 13
    a, m = W.absorbed_spectra(n, lam, seed=23)
    a[0:160] = 0.0
    a[256:] = 0.0
    a2, _ = W.absorbed_spectra(3, lam, seed=29)
    a[70, 40:] = a2[0, 40:]
    a[100, :20] = a2[1, :20]
    a[159, 192:] = a2[2, 192:]
    feat = torch.zeros((n, 32), dtype=torch.float32, device="cuda")
    tot = torch.zeros(n, dtype=torch.float64, device="cuda")
    S.skirt_band_features(_dev(a, torch.float64), n, lam.size, lam, _dev(m, torch.float32), feat, tot)
    B, x, total = E.band_features(a, lam, m.astype(np.float64))
    np.testing.assert_allclose(tot.cpu().numpy(), total, rtol=1e-13, atol=0)
    np.testing.assert_allclose(feat.cpu().numpy(), x, rtol=3e-7, atol=1e-6)
    assert np.count_nonzero(total[:160]) == 3 and np.all(total[256:] == 0)


def test_exact_emission_matches_oracle(S, fields):
    import torch
    lam, a, m = fields
    n = a.shape[0]
    em = torch.zeros((n, 100), dtype=torch.float64, device="cuda")
    T = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    st = S.skirt_dust_emission(_dev(a, torch.float64), n, lam.size, lam, _dev(m, torch.float32), S.EMIT_EXACT,
                               None, em, T)
    assert st["n_cells"] == n and st["n_fallback"] == 0
    ref, Tref, P = E.exact_emission(a, lam, m.astype(np.float64))
    g = em.cpu().numpy()
    big = ref > 1e-9 * ref.sum(axis=1, keepdims=True)
    np.testing.assert_allclose(g[big], ref[big], rtol=1e-9)
    np.testing.assert_allclose(T.cpu().numpy(), Tref, rtol=1e-6)
    # energy: every row sums to the cell's absorbed power
    good = (m > 0) & (a.sum(axis=1) > 0)
    np.testing.assert_allclose(g[good].sum(axis=1), a[good].sum(axis=1), rtol=1e-12)
    assert np.all(g[~good] == 0)


def _small_params(seed):
    rng = np.random.default_rng(seed)
    return {"W1": rng.normal(size=(128, 32)) * 0.25, "b1": rng.normal(size=128) * 0.1,
            "W2": rng.normal(size=(128, 128)) * 0.09, "b2": rng.normal(size=128) * 0.1,
            "W3": rng.normal(size=(100, 128)) * 0.09, "b3": rng.normal(size=100) * 0.1}


def test_training_gradient_matches_oracle(S):
    import torch
    rng = np.random.default_rng(11)
    P = _small_params(3)
    net = S.MLP(seed=1)
    net.set_params(S.pack_params(P))
    P32 = S.unpack_params(S.pack_params(P))  # the FP32 values the device holds
    n = 257  # ragged: not a multiple of the GEMM tiles
    x = rng.normal(size=(n, 32)).astype(np.float32)
    t = rng.random((n, 100))
    t = (t / t.sum(axis=1, keepdims=True)).astype(np.float32)
    g, loss = net.grad(_dev(x, torch.float32), _dev(t, torch.float32), n)
    # the oracle with the kernel's BF16 rounding points; what remains is FP32
    # against FP64 accumulation, and the rare BF16 rounding that an FP32 value
    # on the other side of a rounding boundary takes (one BF16 unit, 2^-8, of
    # one element of one operand)
    ref, ref_loss = E.mlp_grad(P32, x.astype(np.float64), t.astype(np.float64), bf16=True)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    gd = S.unpack_params(g)
    for k in ref:
        scale = np.abs(ref[k]).max()
        np.testing.assert_allclose(gd[k], ref[k], rtol=0, atol=2e-3 * scale, err_msg=k)
    # and the exact gradient within the BF16 rounding bound of the oracle pin
    exact, _ = E.mlp_grad(P32, x.astype(np.float64), t.astype(np.float64))
    for k in exact:
        scale = np.abs(exact[k]).max()
        assert np.abs(gd[k] - exact[k]).max() <= 16 * 2.0 ** -9 * scale, k
    net.close()


def test_tensor_core_inference_matches_oracle(S):
    import torch
    rng = np.random.default_rng(12)
    P = _small_params(4)
    Pb = S.unpack_params(S.pack_params(P))
    Pb = {k: (E.bf16_round(v) if k.startswith("W") else v) for k, v in Pb.items()}
    mean = rng.normal(size=32).astype(np.float32)
    std = (0.5 + rng.random(32)).astype(np.float32)
    lo = (mean - 2 * std).astype(np.float32)
    hi = (mean + 2 * std).astype(np.float32)
    net = S.MLP(seed=1)
    net.set_params(S.pack_params(P), mean, std, lo, hi)
    n = 1000 + 37  # several 64-row tiles and a ragged tail
    x = (mean + std * rng.normal(size=(n, 32)) * 0.8).astype(np.float32)
    x[5, 7] = hi[7] + 1.0  # outside the hull
    x[9, 0] = lo[0] - 1.0
    tot = 10 ** rng.uniform(-3, 3, n)
    em = torch.zeros((n, 100), dtype=torch.float64, device="cuda")
    flags = torch.zeros(n, dtype=torch.uint8, device="cuda")
    net.forward(_dev(x, torch.float32), _dev(tot, torch.float64), n, em, flags)
    xs = (x.astype(np.float64) - mean) / std.astype(np.float64)
    p, _ = E.mlp_forward(Pb, xs, act_bf16=True)
    ref = p * tot[:, None]
    g = em.cpu().numpy()
    np.testing.assert_allclose(g.sum(axis=1), tot, rtol=1e-5)
    rel = np.abs(g - ref) / ref
    assert np.percentile(rel, 99) < 2e-3 and rel.max() < 3e-2
    f = flags.cpu().numpy()
    expect = np.any((x < lo) | (x > hi), axis=1)
    assert np.array_equal(f.astype(bool), expect) and f[5] == 1 and f[9] == 1
    # the guard on the dominant band's share: flags follow the oracle's share,
    # except within FP32 rounding of the threshold (the kernel sums 10^(f - max)
    # in FP32 in another order), where either decision is right
    share = E.dominant_share(x)
    thr = float(np.quantile(share, 0.8))
    net.set_guard(thr)
    assert net.get_guard() == pytest.approx(thr, rel=1e-7)
    flags.zero_()
    net.forward(_dev(x, torch.float32), _dev(tot, torch.float64), n, em, flags)
    f = flags.cpu().numpy().astype(bool)
    expect = np.any((x < lo) | (x > hi), axis=1) | (share > np.float32(thr))
    tie = np.abs(share / np.float32(thr) - 1.0) < 1e-5
    assert np.array_equal(f[~tie], expect[~tie]) and expect.sum() > 150
    # absorbed powers 8 bytes past a 16-byte boundary: the same rows and flags
    tbuf = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    tbuf[1:] = _dev(tot, torch.float64)
    assert tbuf[1:].data_ptr() % 16 == 8
    em2 = torch.zeros_like(em)
    flags2 = torch.zeros_like(flags)
    net.forward(_dev(x, torch.float32), tbuf[1:], n, em2, flags2)
    assert torch.equal(em2, em) and torch.equal(flags2, flags)
    net.close()


def test_inference_skips_tiles_without_absorbed_power(S):
    """Rows without absorbed power emit nothing; a 16-row tile of such rows
    skips the network and writes zero rows.  Whole empty tiles, a tile with
    one live row, and scattered zero rows: the zero rows are exactly zero and
    the others follow the oracle's BF16 forward pass as in the dense test."""
    import torch
    rng = np.random.default_rng(13)
    P = _small_params(7)
    Pb = S.unpack_params(S.pack_params(P))
    Pb = {k: (E.bf16_round(v) if k.startswith("W") else v) for k, v in Pb.items()}
    mean = rng.normal(size=32).astype(np.float32)
    std = (0.5 + rng.random(32)).astype(np.float32)
    net = S.MLP(seed=1)
    net.set_params(S.pack_params(P), mean, std, np.full(32, -1e30, np.float32), np.full(32, 1e30, np.float32))
    n = 200 + 7
    x = (mean + std * rng.normal(size=(n, 32)) * 0.8).astype(np.float32)
    tot = 10 ** rng.uniform(-3, 3, n)
    tot[0:48] = 0.0            # three whole tiles of empty cells
    tot[64:80] = 0.0
    tot[71] = 2.5              # ... one live row in the tile 64..79
    tot[100::7] = 0.0          # scattered zero rows in live tiles
    tot[200:] = 0.0            # an empty ragged tail
    em = torch.full((n, 100), -1.0, dtype=torch.float64, device="cuda")
    net.forward(_dev(x, torch.float32), _dev(tot, torch.float64), n, em)
    g = em.cpu().numpy()
    zero = tot == 0.0
    assert np.all(g[zero] == 0.0)
    xs = (x.astype(np.float64) - mean) / std.astype(np.float64)
    p, _ = E.mlp_forward(Pb, xs, act_bf16=True)
    ref = p[~zero] * tot[~zero][:, None]
    rel = np.abs(g[~zero] - ref) / ref
    assert np.percentile(rel, 99) < 2e-3 and rel.max() < 3e-2
    np.testing.assert_allclose(g[~zero].sum(axis=1), tot[~zero], rtol=1e-5)
    net.close()


def test_training_reaches_two_percent_and_fallback_is_exact(S):
    """Train on exact solutions of synthetic fields; held-out emission within
    2% (per-cell relative L2, median and 95th percentile); the surrogate mode
    sends out-of-hull cells to the exact solver."""
    import torch
    lam = np.geomspace(0.09, 10.0, 200)
    n_train, n_test = 60000, 4000
    a, m = W.absorbed_spectra(n_train + n_test, lam, seed=21)
    ad, md = _dev(a, torch.float64), _dev(m, torch.float32)
    N = a.shape[0]
    feat = torch.zeros((N, 32), dtype=torch.float32, device="cuda")
    tot = torch.zeros(N, dtype=torch.float64, device="cuda")
    S.skirt_band_features(ad, N, lam.size, lam, md, feat, tot)
    ex = torch.zeros((N, 100), dtype=torch.float64, device="cuda")
    S.skirt_dust_emission(ad, N, lam.size, lam, md, S.EMIT_EXACT, None, ex)
    net = S.MLP(seed=3)
    hist = net.train(feat[:n_train].contiguous(), ex[:n_train].contiguous(), n_train, epochs=40, batch=1024,
                     lr=3e-3, seed=5)
    assert hist[-1] < hist[0]
    # held-out cells through the surrogate mode of skirt_dust_emission
    em = torch.zeros((n_test, 100), dtype=torch.float64, device="cuda")
    st = S.skirt_dust_emission(ad[n_train:].contiguous(), n_test, lam.size, lam, md[n_train:].contiguous(),
                               S.EMIT_SURROGATE, net, em)
    ref = ex[n_train:].cpu().numpy()
    err = E.relative_l2(em.cpu().numpy(), ref)
    assert np.median(err) < 0.02 and np.percentile(err, 95) < 0.05, (np.median(err), np.percentile(err, 95))
    np.testing.assert_allclose(em.cpu().numpy().sum(axis=1), ref.sum(axis=1), rtol=1e-5)
    # cells pushed outside the hull (12 dex above every training cell's absorbed
    # power per unit mass) go to the exact solver and match it exactly
    a2 = a[n_train:n_train + 50].copy() * 1e12
    em2 = torch.zeros((50, 100), dtype=torch.float64, device="cuda")
    st2 = S.skirt_dust_emission(_dev(a2, torch.float64), 50, lam.size, lam, md[n_train:n_train + 50].contiguous(),
                                S.EMIT_SURROGATE, net, em2)
    assert st2["n_fallback"] == 50
    ref2, _, _ = E.exact_emission(a2, lam, m[n_train:n_train + 50].astype(np.float64))
    np.testing.assert_allclose(em2.cpu().numpy(), ref2, rtol=1e-9, atol=1e-12 * ref2.max())
    # the fallback rows go through the exact solver's own per-row arithmetic: bit-identical rows
    ex2 = torch.zeros((50, 100), dtype=torch.float64, device="cuda")
    S.skirt_dust_emission(_dev(a2, torch.float64), 50, lam.size, lam, md[n_train:n_train + 50].contiguous(),
                          S.EMIT_EXACT, None, ex2)
    assert torch.equal(em2, ex2)
    # the guard: the 99th percentile of the training rows' dominant-band share
    share_tr = E.dominant_share(feat[:n_train].cpu().numpy())
    k = int(0.99 * (n_train - 1))
    assert net.get_guard() == pytest.approx(np.partition(share_tr, k)[k], rel=1e-5)
    share_te = E.dominant_share(feat[n_train:].cpu().numpy())
    guarded = share_te > net.get_guard()
    assert abs(st["n_fallback"] - int(guarded.sum())) <= max(3, int(0.1 * guarded.sum()) + 3), st["n_fallback"]
    net.close()


@pytest.mark.parametrize("n_in", [1, 700], ids=["one_wavelength", "700_wavelengths"])
def test_band_features_and_exact_edges(S, n_in):
    """One input wavelength (all power in the first band, the other 31 at the
    floor) and 700 (22 staged column blocks per cell), on a cell count that
    is not a multiple of 32."""
    import torch
    lam = np.geomspace(0.09, 10.0, n_in) if n_in > 1 else np.array([0.55])
    n = 1001
    a, m = W.absorbed_spectra(n, lam, seed=11)
    a[5] = 0.0
    feat = torch.zeros((n, 32), dtype=torch.float32, device="cuda")
    tot = torch.zeros(n, dtype=torch.float64, device="cuda")
    S.skirt_band_features(_dev(a, torch.float64), n, lam.size, lam, _dev(m, torch.float32), feat, tot)
    B, x, total = E.band_features(a, lam, m.astype(np.float64))
    np.testing.assert_allclose(tot.cpu().numpy(), total, rtol=1e-13, atol=0)
    np.testing.assert_allclose(feat.cpu().numpy(), x, rtol=3e-7, atol=1e-6)
    em = torch.zeros((n, 100), dtype=torch.float64, device="cuda")
    S.skirt_dust_emission(_dev(a, torch.float64), n, lam.size, lam, _dev(m, torch.float32), S.EMIT_EXACT, None, em)
    ref, _, _ = E.exact_emission(a, lam, m.astype(np.float64))
    g = em.cpu().numpy()
    big = ref > 1e-9 * ref.sum(axis=1, keepdims=True)
    np.testing.assert_allclose(g[big], ref[big], rtol=1e-9)
    assert np.all(g[5] == 0)


@pytest.mark.parametrize("stride", [32, 64])
def test_exact_emission_from_a_coarse_start(S, fields, stride, monkeypatch):
    """The Newton solve started from every stride-th point of the temperature
    table (a start ~1e-8 from the root, so most populations take more Newton
    steps than the first evaluation) reaches the same rows: the oracle at
    1e-9, and the full table's rows to 1e-10 (both accept a point whose Newton
    step is below 1e-13 of ln T, and a term's relative change is x = a_l/T
    times the change of ln T, below ~50 for the terms above 1e-9 of the row)."""
    import torch
    lam, a, m = fields
    n = a.shape[0]
    rows = {}
    for st in (1, stride):
        monkeypatch.setenv("SKIRT_EXACT_TABLE_STRIDE", str(st))
        em = torch.zeros((n, 100), dtype=torch.float64, device="cuda")
        T = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
        S.skirt_dust_emission(_dev(a, torch.float64), n, lam.size, lam, _dev(m, torch.float32), S.EMIT_EXACT,
                              None, em, T)
        rows[st] = (em.cpu().numpy(), T.cpu().numpy())
    ref, Tref, _ = E.exact_emission(a, lam, m.astype(np.float64))
    g, T = rows[stride]
    big = ref > 1e-9 * ref.sum(axis=1, keepdims=True)
    np.testing.assert_allclose(g[big], ref[big], rtol=1e-9)
    np.testing.assert_allclose(T, Tref, rtol=1e-6)
    np.testing.assert_allclose(g[big], rows[1][0][big], rtol=1e-10)
    good = (m > 0) & (a.sum(axis=1) > 0)
    np.testing.assert_allclose(g[good].sum(axis=1), a[good].sum(axis=1), rtol=1e-12)


@pytest.mark.parametrize("scale", [1e-200, 1e-40, 1e40, 1e200])
def test_exact_emission_at_extreme_powers(S, scale):
    """Absorbed powers scaled far outside the temperature range: every
    population clamps at 3 K (small powers) or 2000 K (large ones), and the
    rows, whose powers the solve carries as a double-float times 2^E, still
    match the oracle and sum to the absorbed power, down to 1e-200 and up to
    1e200 of the cells' usual power (the synthetic spectra reach 1e-323, so
    a smaller scale would leave the rows' powers to subnormal arithmetic,
    which the host's matrix product may flush)."""
    import torch
    lam = np.geomspace(0.09, 10.0, 200)
    n = 257
    a, m = W.absorbed_spectra(n, lam, seed=13)
    a = a * scale
    em = torch.zeros((n, 100), dtype=torch.float64, device="cuda")
    T = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    S.skirt_dust_emission(_dev(a, torch.float64), n, lam.size, lam, _dev(m, torch.float32), S.EMIT_EXACT, None,
                          em, T)
    ref, Tref, _ = E.exact_emission(a, lam, m.astype(np.float64))
    np.testing.assert_allclose(Tref, 3.0 if scale < 1 else 2000.0, rtol=1e-14)  # the oracle clamps to exp(ln T)
    g = em.cpu().numpy()
    big = ref > 1e-9 * ref.sum(axis=1, keepdims=True)
    np.testing.assert_allclose(g[big], ref[big], rtol=1e-9)
    assert np.array_equal(T.cpu().numpy(), Tref.astype(np.float32))
    np.testing.assert_allclose(g.sum(axis=1), a.sum(axis=1), rtol=1e-12)
    # the band compression on the same rows: totals exact at every scale;
    # features where the band powers per unit mass stay inside the binary32
    # range they are formed in (at 1e-40 every band sits at the floor)
    feat = torch.zeros((n, 32), dtype=torch.float32, device="cuda")
    tot = torch.zeros(n, dtype=torch.float64, device="cuda")
    S.skirt_band_features(_dev(a, torch.float64), n, lam.size, lam, _dev(m, torch.float32), feat, tot)
    _, x, total = E.band_features(a, lam, m.astype(np.float64))
    np.testing.assert_allclose(tot.cpu().numpy(), total, rtol=1e-13, atol=0)
    if scale == 1e-40:
        np.testing.assert_allclose(feat.cpu().numpy(), x, rtol=3e-7, atol=1e-6)


def test_surrogate_calls_sharing_a_network(S):
    """Surrogate-mode calls keep their working tables in the network handle
    (grown on demand, one call at a time): calls of growing and shrinking
    size, then four threads calling at once on their own streams with the
    same network, give the rows of one call at a time."""
    import threading
    import torch
    lam = np.geomspace(0.09, 10.0, 200)
    sizes = (3000, 40000, 1000, 20000)
    data = []
    for k, n in enumerate(sizes):
        a, m = W.absorbed_spectra(n, lam, seed=40 + k)
        data.append((_dev(a, torch.float64), _dev(m, torch.float32), n))
    a0, m0, n0 = data[1]
    feat = torch.zeros((n0, 32), dtype=torch.float32, device="cuda")
    tot = torch.zeros(n0, dtype=torch.float64, device="cuda")
    S.skirt_band_features(a0, n0, lam.size, lam, m0, feat, tot)
    ex = torch.zeros((n0, 100), dtype=torch.float64, device="cuda")
    S.skirt_dust_emission(a0, n0, lam.size, lam, m0, S.EMIT_EXACT, None, ex)
    net = S.MLP(seed=2)
    net.train(feat, ex, n0, epochs=5, batch=1024)
    ref = []
    for a, m, n in data:  # one at a time: 3000, then a larger table, then smaller ones
        em = torch.zeros((n, 100), dtype=torch.float64, device="cuda")
        S.skirt_dust_emission(a, n, lam.size, lam, m, S.EMIT_SURROGATE, net, em)
        ref.append(em)
    outs = [torch.zeros_like(r) for r in ref]
    streams = [torch.cuda.Stream() for _ in data]
    errors = []

    def call(k):
        try:
            a, m, n = data[k]
            S.skirt_dust_emission(a, n, lam.size, lam, m, S.EMIT_SURROGATE, net, outs[k],
                                  stream=streams[k].cuda_stream)
        except Exception as e:  # reported below
            errors.append(e)

    threads = [threading.Thread(target=call, args=(k,)) for k in range(len(data))]
    torch.cuda.synchronize()  # inputs and zeroed outputs ready before other streams touch them
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    net.close()
    assert not errors, errors
    for r, o in zip(ref, outs):
        assert torch.equal(r, o)
