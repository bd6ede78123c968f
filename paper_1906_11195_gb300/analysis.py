"""Host-side analysis of measured correlations (SI, "Extrapolation to large sizes and large
times"): window averages, the extrapolation to infinite size in N^-nu, and the fits in time of
the inverse Frechet exponential, the polynomials in t^-gamma and the logarithmic decay on moving
windows of octaves.  Plain numpy (and scipy for the nonlinear polynomial fits); it consumes the
integer sums the library returns and never touches the GPU.

Readings of the text where it leaves a choice open:
  * Frechet fit: for a fixed gamma, A and B solve the linear least-squares problem for
    ln C = ln A + B t^-gamma; gamma is the value on a grid (refined by golden-section search)
    that minimises the sum of squared residuals C - G(t) in C itself.
  * Polynomial P_M = A + sum_{m=1..M} A B^m t^{-m gamma} (printed without factorials): for a
    fixed gamma, (A, B) minimise the squared residuals (linear for M = 1, nonlinear otherwise,
    started from the M = 1 solution); gamma as for the Frechet fit.
  * Logarithmic decay L = c (ln t)^-gamma: linear least squares for ln L = ln c - gamma ln ln t.
  * Moving windows: t in [2^(n-k), 2^n] (k = 8 for the exponential and polynomial fits, k = 4
    for the logarithmic one), n stepping by one octave.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "window_averages",
    "finite_size_extrapolation",
    "frechet_fit",
    "polynomial_fit",
    "log_fit",
    "moving_windows",
]


def window_averages(bounds, sums, counts):
    """Window averages of summed measurements: sums[..., m] / counts[m], with the mean time of
    the sweeps in each window (the lumps of the SI are treated as data at their mean time).
    Windows with no measurement give NaN."""
    bounds = np.asarray(bounds, dtype=np.int64)
    counts = np.asarray(counts, dtype=np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        avg = np.asarray(sums, dtype=np.float64) / counts
    t_mean = 0.5 * (bounds[:-1] + bounds[1:] - 1).astype(np.float64)
    return avg, t_mean


def finite_size_extrapolation(N, C, nu=2.0 / 3.0, order=2):
    """Least-squares fit C(N) = C_inf + sum_{k=1..order} a_k N^(-k nu) over the sizes N; returns
    (C_inf, [a_1 .. a_order], sum of squared residuals).  C may have extra trailing axes (one fit
    per column)."""
    N = np.asarray(N, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    x = N ** (-nu)
    X = np.stack([x ** k for k in range(order + 1)], axis=1)  # [n_sizes][order+1]
    Y = C.reshape(C.shape[0], -1)
    coef, _, _, _ = np.linalg.lstsq(X, Y, rcond=None)
    res = ((X @ coef - Y) ** 2).sum(axis=0)
    shape = C.shape[1:]
    return coef[0].reshape(shape), coef[1:].reshape((order,) + shape), res.reshape(shape)


def _golden(f, lo, hi, iters=60):
    g = (math.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(iters):
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = f(d)
    return (a + b) / 2.0


def _scan(ssr_of_gamma, gammas):
    gammas = np.asarray(gammas, dtype=np.float64)
    vals = np.array([ssr_of_gamma(g) for g in gammas])
    i = int(np.nanargmin(vals))
    lo = gammas[max(i - 1, 0)]
    hi = gammas[min(i + 1, len(gammas) - 1)]
    return _golden(ssr_of_gamma, lo, hi) if hi > lo else gammas[i]


def frechet_fit(t, C, gammas=np.linspace(0.01, 2.0, 200)):
    """Inverse Frechet exponential G(t) = A exp(B t^-gamma) (SI eq. frechet); returns
    (A, B, gamma, sum of squared residuals).  C must be positive."""
    t = np.asarray(t, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    lc = np.log(C)

    def solve(g):
        X = np.stack([np.ones_like(t), t ** (-g)], axis=1)
        (la, b), _, _, _ = np.linalg.lstsq(X, lc, rcond=None)
        return math.exp(la), b

    def ssr(g):
        a, b = solve(g)
        return float(((C - a * np.exp(b * t ** (-g))) ** 2).sum())

    g = _scan(ssr, gammas)
    a, b = solve(g)
    return a, b, g, ssr(g)


def polynomial_fit(t, C, M, gammas=np.linspace(0.01, 2.0, 200)):
    """P_M(t) = A + sum_{m=1..M} A B^m t^(-m gamma) (SI eq. pol); returns
    (A, B, gamma, sum of squared residuals)."""
    from scipy.optimize import least_squares

    t = np.asarray(t, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)

    def model(p, x):
        a, b = p
        return a * (1.0 + sum((b * x) ** m for m in range(1, M + 1)))

    def solve(g):
        x = t ** (-g)
        X = np.stack([np.ones_like(x), x], axis=1)
        (a, ab), _, _, _ = np.linalg.lstsq(X, C, rcond=None)
        p0 = np.array([a, ab / a if a != 0 else 0.0])
        if M == 1:
            return p0
        r = least_squares(lambda p: model(p, x) - C, p0, method="lm", xtol=1e-15, ftol=1e-15,
                          gtol=1e-15, max_nfev=2000)
        return r.x

    def ssr(g):
        p = solve(g)
        return float(((model(p, t ** (-g)) - C) ** 2).sum())

    g = _scan(ssr, gammas)
    a, b = solve(g)
    return a, b, g, ssr(g)


def log_fit(t, C):
    """Logarithmic decay L(t) = c (ln t)^-gamma; returns (c, gamma, sum of squared residuals in
    ln L).  Needs t > 1 and C > 0."""
    t = np.asarray(t, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    X = np.stack([np.ones_like(t), -np.log(np.log(t))], axis=1)
    (lc, g), _, _, _ = np.linalg.lstsq(X, np.log(C), rcond=None)
    res = float(((X @ np.array([lc, g]) - np.log(C)) ** 2).sum())
    return math.exp(lc), g, res


def moving_windows(t, C, k, fit, n_min=None, n_max=None):
    """Apply fit(t_w, C_w) on every window t in [2^(n-k), 2^n]; returns a list of
    (n, fit result) for the windows holding at least three points."""
    t = np.asarray(t, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    lo = int(math.floor(math.log2(t.min()))) + k if n_min is None else n_min
    hi = int(math.ceil(math.log2(t.max()))) if n_max is None else n_max
    out = []
    for n in range(lo, hi + 1):
        sel = (t >= 2.0 ** (n - k)) & (t <= 2.0 ** n)
        if sel.sum() >= 3:
            out.append((n, fit(t[sel], C[sel])))
    return out
