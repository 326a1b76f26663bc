"""Pins of the dust-emission oracle and of its surrogate network's reference
arithmetic against closed forms and finite differences."""
import math

import numpy as np
import pytest
from scipy.special import gamma, zeta

from oracle import emission as E


@pytest.mark.parametrize("i", [0, 1, 2])
@pytest.mark.parametrize("T", [15.0, 30.0, 80.0, 150.0])
def test_planck_sum_matches_closed_form(i, T):
    """sum_l W_l kappa_i B(lambda_l, T) approximates the integral
    100^beta (T/a)^(4+beta) Gamma(4+beta) zeta(4+beta) of the opacity-weighted
    Planck shape (substitution x = a/(lambda T))."""
    b = E.BETA[i]
    exact = 100.0 ** b * (T / E.A_HCK) ** (4 + b) * gamma(4 + b) * zeta(4 + b)
    assert E.G(i, T) == pytest.approx(exact, rel=1e-2)


def test_hck_constant():
    # h c / k_B from the exact SI values: 14387.768775... micron kelvin
    assert E.A_HCK == pytest.approx(14387.768775039337, rel=1e-14)


def test_wien_peak_of_the_emission_density():
    """The emission per unit wavelength of a beta population peaks where
    x = a/(lambda T) solves x = (5 + beta)(1 - e^-x)."""
    lam, W = E.emission_grid()
    for i, T in ((1, 30.0), (0, 60.0)):
        b = E.BETA[i]
        x = 5.0
        for _ in range(100):
            x = (5 + b) * (1 - math.exp(-x))
        lam_peak = E.A_HCK / (x * T)
        density = E.opacity(lam, b) * E.planck_shape(lam, T)
        k = int(np.argmax(density))
        assert lam[k - 1] < lam_peak < lam[k + 1]


def test_weights_and_normalisation():
    lam, W = E.emission_grid()
    assert lam[0] == pytest.approx(1.0) and lam[-1] == pytest.approx(1000.0)
    assert W.sum() == pytest.approx(999.0, rel=1e-14)  # trapezoid weights sum to the range
    for i in range(3):
        assert E.G(i, 30.0) * E.c_norm(i) == pytest.approx(1.0, rel=1e-15)
    w = E.absorption_shares(np.geomspace(0.09, 10, 200))
    np.testing.assert_allclose(w.sum(axis=0), 1.0, rtol=1e-15)
    assert np.all(np.diff(w[0]) < 0) and np.all(np.diff(w[2]) > 0)


@pytest.mark.parametrize("i", [0, 1, 2])
def test_temperature_solver(i):
    ratio = np.geomspace(1e-4, 1e5, 200)
    T = E.solve_temperature(i, ratio)
    assert np.all(np.diff(T) > 0)
    inside = (T > E.T_LO * (1 + 1e-9)) & (T < E.T_HI * (1 - 1e-9))
    np.testing.assert_allclose(E.G(i, T[inside]) / E.G(i, 30.0), ratio[inside], rtol=1e-11)
    assert E.solve_temperature(i, np.array([1.0]))[0] == pytest.approx(30.0, rel=1e-12)
    # outside the bracket the temperature clamps
    assert E.solve_temperature(i, np.array([1e-30]))[0] == pytest.approx(E.T_LO)
    assert E.solve_temperature(i, np.array([1e30]))[0] == pytest.approx(E.T_HI)


def test_exact_emission_conserves_energy():
    rng = np.random.default_rng(3)
    lam_in = np.geomspace(0.09, 10.0, 50)
    n = 300
    absorbed = np.exp(rng.normal(size=(n, 50))) * 10 ** rng.uniform(-3, 3, (n, 1))
    mass = 10 ** rng.uniform(-2, 2, n)
    mass[:5] = 0.0
    absorbed[5:10] = 0.0
    em, T, P = E.exact_emission(absorbed, lam_in, mass)
    np.testing.assert_allclose(P.sum(axis=1), absorbed.sum(axis=1), rtol=1e-13)
    good = (mass > 0) & (absorbed.sum(axis=1) > 0)
    np.testing.assert_allclose(em[good].sum(axis=1), absorbed[good].sum(axis=1), rtol=1e-12)
    assert np.all(em[~good] == 0) and np.all(T[~good] == 0)
    assert np.all(em >= 0)
    # hotter dust for more absorbed power per unit mass
    order = np.argsort(P[good, 1] / mass[good])
    assert np.all(np.diff(T[good, 1][order]) >= 0)


def test_band_features():
    lam_in = np.geomspace(0.09, 10.0, 200)
    idx = E.band_index(lam_in)
    assert idx[0] == 0 and idx[-1] == E.NBANDS - 1
    assert np.all(np.diff(idx) >= 0)
    assert np.bincount(idx, minlength=E.NBANDS).min() >= 1
    rng = np.random.default_rng(1)
    a = rng.random((20, 200))
    m = rng.random(20) + 0.1
    B, x, tot = E.band_features(a, lam_in, m)
    np.testing.assert_allclose(B.sum(axis=1), a.sum(axis=1), rtol=1e-14)
    np.testing.assert_allclose(x, np.log10(B / m[:, None]), rtol=1e-14)
    np.testing.assert_allclose(tot, a.sum(axis=1), rtol=1e-14)


def test_band_features_floor_of_empty_bands():
    """Cells with empty bands, computed by hand: an empty band sits at
    1e-6 of the cell's total absorbed power shared over the 32 bands, per unit
    mass; a dust-free or unheated cell sits at 1e-30 in every band.
    Cell 0: power 2 at the first wavelength only, mass 0.5:
      band 0 = log10(2 / 0.5) = log10(4); the rest log10(1e-6 * 2 / 32 / 0.5) = log10(1.25e-7).
    Cell 1: power 3 at the first and 1 at the last wavelength, mass 2:
      band 0 = log10(1.5), band 31 = log10(0.5), the rest log10(1e-6 * 4 / 32 / 2) = log10(6.25e-8).
    Cell 2: no dust; cell 3: no absorbed power."""
    lam_in = np.geomspace(0.1, 10.0, 50)
    a = np.zeros((4, 50))
    a[0, 0] = 2.0
    a[1, 0] = 3.0
    a[1, -1] = 1.0
    a[2, 5] = 1.0
    m = np.array([0.5, 2.0, 0.0, 1.0])
    B, x, tot = E.band_features(a, lam_in, m)
    exp = np.empty((4, E.NBANDS))
    exp[0] = math.log10(1.25e-7)
    exp[0, 0] = math.log10(4.0)
    exp[1] = math.log10(6.25e-8)
    exp[1, 0] = math.log10(1.5)
    exp[1, 31] = math.log10(0.5)
    exp[2:] = -30.0
    np.testing.assert_allclose(x, exp, rtol=1e-14, atol=1e-14)
    np.testing.assert_array_equal(tot, [2.0, 4.0, 1.0, 0.0])


def test_dominant_share_by_hand():
    """The guard's quantity on rows computed by hand: two equal bands and the
    rest empty (-30) -> 1/2; 32 equal bands -> 1/32; one band at 10x another
    (log10 difference 1), the rest empty -> 10/11."""
    x = np.full((3, 32), -30.0)
    x[0, :2] = 1.5
    x[1, :] = -2.0
    x[2, 4], x[2, 9] = 0.5, -0.5
    np.testing.assert_allclose(E.dominant_share(x), [0.5, 1.0 / 32, 10.0 / 11.0], rtol=1e-14)


def _params(rng, scale=0.3):
    return {"W1": rng.normal(size=(128, 32)) * scale, "b1": rng.normal(size=128) * 0.1,
            "W2": rng.normal(size=(128, 128)) * scale / 3, "b2": rng.normal(size=128) * 0.1,
            "W3": rng.normal(size=(100, 128)) * scale / 3, "b3": rng.normal(size=100) * 0.1}


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(7)
    P = _params(rng)
    x = rng.normal(size=(6, 32))
    t = rng.random((6, 100))
    t /= t.sum(axis=1, keepdims=True)
    g, loss = E.mlp_grad(P, x, t)
    assert loss == pytest.approx(E.mlp_loss(P, x, t), rel=1e-14)
    # central differences: truncation ~h^2, roundoff ~eps L / h ~ 1e-10 at h = 1e-5
    h = 1e-5
    for name, picks in (("W1", [(0, 0), (5, 31), (127, 7)]), ("b1", [(3,), (120,)]),
                        ("W2", [(0, 0), (64, 100)]), ("b2", [(9,)]), ("W3", [(0, 0), (99, 127)]),
                        ("b3", [(0,), (57,)])):
        for ij in picks:
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[name][ij] += h
            Pm[name][ij] -= h
            fd = (E.mlp_loss(Pp, x, t) - E.mlp_loss(Pm, x, t)) / (2 * h)
            assert g[name][ij] == pytest.approx(fd, rel=1e-5, abs=1e-9), (name, ij)


def test_mlp_gradient_with_bfloat16_operands():
    """The BF16-operand gradient (the tensor-core training arithmetic) stays
    within the rounding bound of the exact one, which the finite differences
    above pin: every product sees operands with relative errors <= 2^-9, and
    a gradient entry collects them from at most six rounding stages (input,
    two activations, three weights, three dz) along its path, so it moves by
    well under 16 x 2^-9 of its tensor's scale; and the rounding is applied
    (the two differ)."""
    rng = np.random.default_rng(8)
    P = _params(rng)
    x = rng.normal(size=(64, 32))
    t = rng.random((64, 100))
    t /= t.sum(axis=1, keepdims=True)
    g, _ = E.mlp_grad(P, x, t)
    gb, lb = E.mlp_grad(P, x, t, bf16=True)
    for k in g:
        scale = np.abs(g[k]).max()
        assert np.abs(gb[k] - g[k]).max() <= 16 * 2.0 ** -9 * scale, k
        assert np.abs(gb[k] - g[k]).max() > 0, k
    assert lb == pytest.approx(E.mlp_loss(P, x, t), rel=16 * 2.0 ** -9)


def test_surrogate_output_is_energy_exact():
    rng = np.random.default_rng(2)
    P = _params(rng)
    x = rng.normal(size=(10, 32))
    tot = 10 ** rng.uniform(-5, 5, 10)
    em = E.surrogate_emission(P, x, tot, np.zeros(32), np.ones(32))
    np.testing.assert_allclose(em.sum(axis=1), tot, rtol=1e-13)
    assert np.all(em > 0)


def test_bf16_rounding():
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, -2.5, 3.140625, 1e-20], dtype=np.float64)
    r = E.bf16_round(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # halfway: ties to even
    assert r[2] == 1 + 2 ** -7              # above halfway: rounds up
    assert r[3] == -2.5 and r[4] == 3.140625
    assert abs(r[5] - 1e-20) / 1e-20 < 2 ** -8


def test_mlp_forward_on_a_scalar_chain():
    """The network's wiring on weights with one path: input feature 7
    (standardised with its own mean and std) -> hidden unit 5 -> hidden unit
    11 -> output bin 42, every other weight and bias zero except b3[3].  The
    output is then a two-level softmax written out by hand: bin 42 takes
    e^{z}, bin 3 e^{b}, the other 98 bins 1 each, with
    z = g * s(b2 + w2 * s(w1 * x7)), s(v) = v / (1 + e^{-v})."""
    import math
    P = {"W1": np.zeros((128, 32)), "b1": np.zeros(128), "W2": np.zeros((128, 128)), "b2": np.zeros(128),
         "W3": np.zeros((100, 128)), "b3": np.zeros(100)}
    w1, w2, b2, g, b = 0.8, -1.3, 0.25, 2.0, -0.7
    P["W1"][5, 7] = w1
    P["W2"][11, 5] = w2
    P["b2"][11] = b2
    P["W3"][42, 11] = g
    P["b3"][3] = b
    x = np.zeros((3, 32))
    x[:, 7] = [0.5, -2.0, 3.0]
    x[:, 6] = 9.0  # a neighbouring feature with no path to the output
    mean, std = np.zeros(32), np.ones(32)
    mean[7], std[7] = 0.2, 2.0
    tot = np.array([1.0, 10.0, 0.5])
    em = E.surrogate_emission(P, x, tot, mean, std)

    def s(v):
        return v / (1.0 + math.exp(-v))
    for r in range(3):
        x7 = (x[r, 7] - 0.2) / 2.0
        z = g * s(b2 + w2 * s(w1 * x7))
        den = math.exp(z) + math.exp(b) + 98.0
        assert em[r, 42] == pytest.approx(tot[r] * math.exp(z) / den, rel=1e-13)
        assert em[r, 3] == pytest.approx(tot[r] * math.exp(b) / den, rel=1e-13)
        others = np.delete(em[r], [3, 42])
        np.testing.assert_allclose(others, tot[r] / den, rtol=1e-13)
