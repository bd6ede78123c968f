"""Host analysis (SI, extrapolations in size and time) pinned on data with known answers: every
fit must recover the parameters of data generated exactly from its own model."""
import numpy as np
import pytest

from paper_1906_11195_gb300 import analysis


def test_finite_size_extrapolation_recovers_the_limit():
    N = 2.0 ** np.arange(10, 23, 2)
    for nu in (1.0, 2.0 / 3.0):
        C = 0.137 + 0.8 * N ** (-nu) - 3.0 * N ** (-2 * nu)
        c_inf, a, res = analysis.finite_size_extrapolation(N, C, nu=nu, order=2)
        assert abs(c_inf - 0.137) < 1e-10 and abs(a[0] - 0.8) < 1e-6 and abs(a[1] + 3.0) < 1e-4
        assert res < 1e-20
    # several times at once; a linear fit of quadratic data leaves a residual
    C2 = np.stack([0.1 + 0.5 * N ** (-2 / 3), 0.2 + 0.7 * N ** (-2 / 3)], axis=1)
    c_inf, _, _ = analysis.finite_size_extrapolation(N, C2, order=1)
    assert np.allclose(c_inf, [0.1, 0.2], atol=1e-12)


def test_frechet_fit_recovers_parameters():
    t = 2.0 ** np.linspace(4, 20, 60)
    A, B, g = 0.09, 1.7, 0.35
    C = A * np.exp(B * t ** (-g))
    a, b, gg, ssr = analysis.frechet_fit(t, C)
    assert abs(a - A) < 1e-6 and abs(b - B) < 1e-4 and abs(gg - g) < 1e-5 and ssr < 1e-14


@pytest.mark.parametrize("M", [1, 2, 3])
def test_polynomial_fit_recovers_parameters(M):
    pytest.importorskip("scipy")
    t = 2.0 ** np.linspace(4, 20, 60)
    A, B, g = 0.12, 0.9, 0.4
    x = t ** (-g)
    C = A * (1.0 + sum((B * x) ** m for m in range(1, M + 1)))
    a, b, gg, ssr = analysis.polynomial_fit(t, C, M)
    assert abs(a - A) < 1e-6 and abs(b - B) < 1e-3 and abs(gg - g) < 1e-4 and ssr < 1e-14


def test_log_fit_recovers_parameters():
    t = 2.0 ** np.linspace(3, 25, 40)
    c, g = 0.8, 0.6
    C = c * np.log(t) ** (-g)
    cc, gg, res = analysis.log_fit(t, C)
    assert abs(cc - c) < 1e-10 and abs(gg - g) < 1e-10 and res < 1e-20


def test_moving_windows_cover_octaves():
    t = 2.0 ** np.arange(0, 17)
    C = 1.0 / np.log(t + 2.0)
    fits = analysis.moving_windows(t, C, 4, lambda tt, cc: (tt.min(), tt.max(), len(tt)))
    ns = [n for n, _ in fits]
    assert ns == list(range(4, 17))
    for n, (lo, hi, k) in fits:
        assert lo == 2.0 ** (n - 4) and hi == 2.0 ** n and k == 5


def test_window_averages_are_sums_over_counts():
    bounds = np.array([4, 6, 8, 12])
    sums = np.array([[10.0, 20.0, 0.0]])
    counts = np.array([2, 2, 0])
    avg, tm = analysis.window_averages(bounds, sums, counts)
    assert np.allclose(avg[0, :2], [5.0, 10.0]) and np.isnan(avg[0, 2])
    assert np.allclose(tm, [4.5, 6.5, 9.5])  # the first SK lump {4, 5} stands at 4.5
