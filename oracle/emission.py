"""FP64 oracle of the dust-emission step and of its learned surrogate --
TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Method (arXiv:1705.04702, Sect. 3.2, dust self-absorption and dust emission
phases): the emission spectrum of every dust cell is computed from the
amount of absorbed (stellar) radiation in that cell, and the table of
emission spectra [cell, wavelength] is the source of the dust photon packets.
The paper names the step but not its model ("instantaneous dust emission",
Sect. 1).  Reading used here (equilibrium emission of three grain
populations):

* absorption shares w_i(lambda) ~ (lambda / 0.55 um)^delta_i, delta =
  (-0.5, 0, +0.5), normalised so that sum_i w_i(lambda) = 1; the power
  absorbed by population i in cell m is P_i = sum_j w_i(lambda_j) A(m, j);
* emission grid: 100 wavelengths log-spaced over 1-1000 um with trapezoid
  weights W_l; emission opacity kappa_i(lambda) = (lambda / 100 um)^-beta_i,
  beta = (1.5, 2, 2); Planck shape B(lambda, T) = lambda^-5 / (e^{a/(lambda T)} - 1)
  with a = h c / k_B;
* energy balance: M c_i G_i(T_i) = P_i with G_i(T) = sum_l W_l kappa_i B(lambda_l, T),
  M the cell's dust mass (extinction coefficient times volume) and
  c_i = 1 / G_i(30 K) (a population absorbing P_i = M sits at 30 K);
  T_i by bracketed Newton on ln T in [3 K, 2000 K] (clamped there);
* emission(m, l) = sum_i P_i W_l kappa_i B(lambda_l, T_i) / G_i(T_i), so
  sum_l emission(m, l) = sum_i P_i = sum_j A(m, j) exactly.

The surrogate: the absorbed spectrum is compressed to 32 log-spaced bands
(band sums per unit dust mass, log10), standardised, and mapped by an MLP
32 -> 128 -> 128 -> 100 (SiLU, SiLU, softmax) to the normalised emission
shape, which is multiplied by the cell's total absorbed power.
"""
from __future__ import annotations

import math

import numpy as np

# exact SI values: h c / k_B in micron kelvin
A_HCK = 6.62607015e-34 * 299792458.0 / 1.380649e-23 * 1e6
DELTA = np.array([-0.5, 0.0, 0.5])
BETA = np.array([1.5, 2.0, 2.0])
T_REF = 30.0
T_LO, T_HI = 3.0, 2000.0
NBANDS = 32
NOUT = 100
FEATURE_FLOOR = 1e-30


def emission_grid():
    """100 log-spaced wavelengths over 1-1000 micron and their trapezoid weights."""
    lam = np.geomspace(1.0, 1000.0, NOUT)
    W = np.empty(NOUT)
    W[0] = 0.5 * (lam[1] - lam[0])
    W[-1] = 0.5 * (lam[-1] - lam[-2])
    W[1:-1] = 0.5 * (lam[2:] - lam[:-2])
    return lam, W


def planck_shape(lam, T):
    """lambda^-5 / (exp(a / (lambda T)) - 1), broadcasting lam against T
    (zero where the exponential overflows)."""
    with np.errstate(over="ignore"):
        return lam ** -5.0 / np.expm1(A_HCK / (lam * T))


def opacity(lam, beta):
    return (lam / 100.0) ** (-beta)


def G(i, T, lam=None, W=None, beta=None):
    """sum_l W_l kappa_i(lambda_l) B(lambda_l, T); T scalar or array."""
    if lam is None:
        lam, W = emission_grid()
    b = BETA[i] if beta is None else beta
    T = np.asarray(T, dtype=np.float64)
    return np.sum(W * opacity(lam, b) * planck_shape(lam, T[..., None]), axis=-1)


def dlnG_dlnT(i, T):
    """d ln G / d ln T = sum W kappa B x/(1-e^-x) / G, x = a/(lambda T)."""
    lam, W = emission_grid()
    T = np.asarray(T, dtype=np.float64)
    x = A_HCK / (lam * T[..., None])
    terms = W * opacity(lam, BETA[i]) * planck_shape(lam, T[..., None])
    return np.sum(terms * x / (-np.expm1(-x)), axis=-1) / np.sum(terms, axis=-1)


def c_norm(i):
    return 1.0 / G(i, T_REF)


def absorption_shares(lam_in):
    """w_i(lambda) for the input wavelengths: [3, n]."""
    lam_in = np.asarray(lam_in, dtype=np.float64)
    raw = (lam_in[None, :] / 0.55) ** DELTA[:, None]
    return raw / raw.sum(axis=0, keepdims=True)


def solve_temperature(i, ratio, tol=1e-13, itmax=100):
    """T with G_i(T) / G_i(30 K) = ratio by Newton on y = ln T inside the
    bracket [ln 3, ln 2000], falling back to bisection when a step leaves
    it; ratio outside the bracket's range clamps T to the bracket end.
    Vectorised over ratio (> 0)."""
    ratio = np.asarray(ratio, dtype=np.float64)
    target = np.log(ratio / c_norm(i))  # ln G at the solution
    lo = np.full(ratio.shape, math.log(T_LO))
    hi = np.full(ratio.shape, math.log(T_HI))
    f_lo = np.log(G(i, np.exp(lo))) - target
    f_hi = np.log(G(i, np.exp(hi))) - target
    y = np.where(f_lo >= 0, lo, np.where(f_hi <= 0, hi, 0.5 * (lo + hi)))
    active = (f_lo < 0) & (f_hi > 0)
    for _ in range(itmax):
        if not active.any():
            break
        T = np.exp(y)
        f = np.log(G(i, T)) - target
        lo = np.where(active & (f < 0), y, lo)
        hi = np.where(active & (f > 0), y, hi)
        step = f / dlnG_dlnT(i, T)
        y_new = y - step
        outside = (y_new <= lo) | (y_new >= hi)
        y_new = np.where(outside, 0.5 * (lo + hi), y_new)
        done = np.abs(y_new - y) <= tol * np.abs(y)
        y = np.where(active, y_new, y)
        active = active & ~done
    return np.exp(y)


def exact_emission(absorbed, lam_in, mass):
    """absorbed [n_cell, n_in] (luminosity per cell and input wavelength),
    mass [n_cell] -> emission [n_cell, 100], T [n_cell, 3], P [n_cell, 3].
    Cells with no dust or no absorbed power emit nothing (T = 0)."""
    absorbed = np.asarray(absorbed, dtype=np.float64)
    P = absorbed @ absorption_shares(lam_in).T    # [n_cell, 3]
    return emission_from_power(P, mass)


def exact_emission_pair(absorbed_a, lam_a, absorbed_b, lam_b, mass):
    """Exact emission of cells heated by two absorbed fields on two
    wavelength grids, e.g. the stellar field and the dust's own emission
    (Sect. 3.2, dust self-absorption phase): the power each population
    absorbs adds, P = A w_a^T + B w_b^T."""
    P = (np.asarray(absorbed_a, dtype=np.float64) @ absorption_shares(lam_a).T +
         np.asarray(absorbed_b, dtype=np.float64) @ absorption_shares(lam_b).T)
    return emission_from_power(P, mass)


def emission_from_power(P, mass):
    """Equilibrium temperatures and emission rows from the power P [n_cell, 3]
    absorbed by each population and the dust mass [n_cell]."""
    P = np.asarray(P, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    lam, W = emission_grid()
    emission = np.zeros((P.shape[0], NOUT))
    T = np.zeros((P.shape[0], 3))
    for i in range(3):
        ok = (P[:, i] > 0) & (mass > 0)
        if not ok.any():
            continue
        Ti = solve_temperature(i, P[ok, i] / mass[ok])
        T[ok, i] = Ti
        shape = W * opacity(lam, BETA[i]) * planck_shape(lam, Ti[:, None])
        emission[ok] += P[ok, i][:, None] * shape / shape.sum(axis=1, keepdims=True)
    return emission, T, P


# --------------------------------------------------------------------------
# band compression and the surrogate network
# --------------------------------------------------------------------------
def band_index(lam_in, nbands=NBANDS):
    """Band of every input wavelength: nbands log-spaced bands over
    [min, max] of the input grid."""
    lam_in = np.asarray(lam_in, dtype=np.float64)
    lo, hi = lam_in.min(), lam_in.max()
    if hi <= lo:
        return np.zeros(lam_in.shape, dtype=np.int64)
    b = np.floor(nbands * np.log(lam_in / lo) / np.log(hi / lo)).astype(np.int64)
    return np.clip(b, 0, nbands - 1)


BAND_FLOOR_REL = 1e-6


def band_features(absorbed, lam_in, mass, nbands=NBANDS):
    """Band sums B [n, nbands], features and the total absorbed power T [n].
    Feature b is log10(max(B_b, 1e-6 T / nbands) / M): a band without
    absorbed power sits 6 dex (per band) below the cell's total instead of at
    an absolute floor; cells without dust or absorbed power get log10(1e-30)."""
    absorbed = np.asarray(absorbed, dtype=np.float64)
    idx = band_index(lam_in, nbands)
    B = np.zeros((absorbed.shape[0], nbands))
    for j, b in enumerate(idx):
        B[:, b] += absorbed[:, j]
    T = B.sum(axis=1)
    mass = np.asarray(mass, dtype=np.float64)
    ok = (mass > 0) & (T > 0)
    x = np.full(B.shape, math.log10(FEATURE_FLOOR))
    floor = BAND_FLOOR_REL * T[ok, None] / nbands
    x[ok] = np.log10(np.maximum(np.maximum(B[ok], floor) / mass[ok, None], FEATURE_FLOOR))
    return B, x, absorbed.sum(axis=1)


def dominant_share(x):
    """Share of a row's absorbed power held by its dominant band, from the
    band features x [n, 32] (log10 of band power per unit mass): the largest
    band power over their sum."""
    p = 10.0 ** (np.asarray(x, dtype=np.float64) - np.max(x, axis=1, keepdims=True))
    return 1.0 / p.sum(axis=1)


def bf16_round(a):
    """Round float values to bfloat16 (nearest, ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def mlp_forward(params, x_std, act_bf16=False):
    """params: dict W1 [128,32], b1, W2 [128,128], b2, W3 [100,128], b3.
    x_std: standardised inputs [n, 32].  With act_bf16 the inputs of every
    layer are rounded to bfloat16 first (the precision the tensor-core
    inference kernel feeds its multiplies).  Returns (probabilities [n,100],
    cache for the backward pass)."""
    q = bf16_round if act_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    a0 = q(x_std)
    z1 = a0 @ params["W1"].T + params["b1"]
    a1 = q(silu(z1))
    z2 = a1 @ params["W2"].T + params["b2"]
    a2 = q(silu(z2))
    z3 = a2 @ params["W3"].T + params["b3"]
    z3s = z3 - z3.max(axis=1, keepdims=True)
    e = np.exp(z3s)
    p = e / e.sum(axis=1, keepdims=True)
    return p, (a0, z1, a1, z2, a2, z3)


def mlp_loss(params, x_std, target):
    """Mean over the batch of the cross-entropy -sum_l t_l log p_l between
    target shapes (rows sum to 1) and the softmax output."""
    p, _ = mlp_forward(params, x_std)
    return float(-np.sum(target * np.log(np.maximum(p, 1e-300))) / x_std.shape[0])


def mlp_grad(params, x_std, target, bf16=False):
    """Gradients of mlp_loss by reverse-mode differentiation written out
    layer by layer (softmax + cross-entropy: dL/dz3 = (p - t) / n), and the
    loss.  With bf16, every operand of a matrix product is rounded to
    bfloat16 first, as the tensor-core training kernel feeds its products:
    the inputs, the weights, the activations and the back-propagated dz of
    each layer (the bias gradients sum the unrounded dz).  Returns (grads,
    mean loss)."""
    n = x_std.shape[0]
    q = bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    W = {k: q(params[k]) if k.startswith("W") else np.asarray(params[k], np.float64) for k in params}
    p, (a0, z1, a1, z2, a2, z3) = mlp_forward(W, x_std, act_bf16=bf16)
    loss = float(-np.sum(target * np.log(np.maximum(p, 1e-300))) / n)
    d3 = (p - target) / n
    g = {"b3": d3.sum(axis=0)}
    d3 = q(d3)
    g["W3"] = d3.T @ a2
    da2 = d3 @ W["W3"]
    s2 = 1.0 / (1.0 + np.exp(-z2))
    d2 = da2 * (s2 * (1.0 + z2 * (1.0 - s2)))
    g["b2"] = d2.sum(axis=0)
    d2 = q(d2)
    g["W2"] = d2.T @ a1
    da1 = d2 @ W["W2"]
    s1 = 1.0 / (1.0 + np.exp(-z1))
    d1 = da1 * (s1 * (1.0 + z1 * (1.0 - s1)))
    g["b1"] = d1.sum(axis=0)
    d1 = q(d1)
    g["W1"] = d1.T @ a0
    return g, loss


def surrogate_emission(params, x, total, mean, std, act_bf16=False):
    """Emission [n, 100] predicted from raw features x [n, 32]."""
    p, _ = mlp_forward(params, (x - mean) / std, act_bf16=act_bf16)
    return p * np.asarray(total, dtype=np.float64)[:, None]


def relative_l2(pred, ref):
    """Per-row relative L2 error over the 100 emission wavelengths."""
    num = np.sqrt(np.sum((pred - ref) ** 2, axis=1))
    den = np.sqrt(np.sum(ref ** 2, axis=1))
    return num / np.maximum(den, 1e-300)
