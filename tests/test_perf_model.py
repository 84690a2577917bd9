"""The performance model of Sec. 3.5 (Eq. 2 and Eq. 3) as restated for the GPU, on the host:
the least-squares fit of perf(x, y) = a0 + a1 x + a2 y + a3 x^2 + a4 y^2 recovers a known
quadratic exactly, agrees with numpy's least squares on noisy samples, still answers for
samples on a line, and the argmax (Eq. 3) finds the known best candidate."""
import numpy as np
import pytest


def _features(x, y):
    return np.stack([np.ones_like(x), x, y, x * x, y * y], axis=1)


def test_fit_recovers_a_known_quadratic(loops_lib):
    lp = loops_lib
    a = np.array([120.0, 3.5e-7, -2.0e-7, -4.0e-16, 1.5e-16])
    gx, gy = np.meshgrid(np.linspace(0, 2e9, 4), np.linspace(0, 5e8, 3))
    x, y = gx.ravel(), gy.ravel()
    perf = _features(x, y) @ a
    coef = lp.perf_model_fit(x, y, perf)
    # predictions agree to rounding; the coefficients to the fit's conditioning
    assert np.allclose(_features(x, y) @ coef, perf, rtol=1e-9, atol=1e-9 * np.abs(perf).max())
    assert np.allclose(coef, a, rtol=1e-6, atol=0)


def test_fit_matches_numpy_least_squares_on_noisy_samples(loops_lib):
    lp = loops_lib
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1e9, 40)
    y = rng.uniform(0, 3e8, 40)
    perf = 900 + 1e-7 * x - 2e-6 * y - 1e-16 * x * x + 3e-15 * y * y + rng.normal(0, 5.0, 40)
    coef = lp.perf_model_fit(x, y, perf)
    # reference: numpy's SVD least squares on the scaled features, unscaled
    sx, sy = np.abs(x).max(), np.abs(y).max()
    ref, *_ = np.linalg.lstsq(_features(x / sx, y / sy), perf, rcond=None)
    ref = ref / np.array([1, sx, sy, sx * sx, sy * sy])
    assert np.allclose(_features(x, y) @ coef, _features(x, y) @ ref, rtol=1e-8)


def test_fit_with_samples_on_a_line_reproduces_them(loops_lib):
    # one matrix: the CSR work falls as the BCSR work grows, so the samples lie on a line
    lp = loops_lib
    t = np.array([0.0, 0.2, 0.5, 0.7, 1.0])
    x, y = 1e9 * (1 - t), 1.6e9 * t
    perf = 500 + 800 * t - 900 * t * t
    coef = lp.perf_model_fit(x, y, perf)
    assert np.allclose(_features(x, y) @ coef, perf, rtol=1e-6, atol=1e-6 * 500)
    # Eq. 3 on a finer grid of the same line: the vertex of the parabola, t = 800 / 1800
    tg = np.linspace(0, 1, 1801)
    best, pred = lp.perf_model_argmax(coef, 1e9 * (1 - tg), 1.6e9 * tg)
    assert abs(tg[best] - 800 / 1800) <= 1e-3
    assert pred == pytest.approx(500 + 800 ** 2 / (4 * 900), rel=1e-6)


def test_argmax_picks_the_highest_prediction(loops_lib):
    lp = loops_lib
    coef = np.array([10.0, 1.0, 2.0, -0.5, -0.25])
    x = np.array([0.0, 1.0, 2.0, 1.0, 3.0])
    y = np.array([0.0, 4.0, 1.0, 2.0, 4.0])
    pred = _features(x, y) @ coef
    best, bp = lp.perf_model_argmax(coef, x, y)
    assert best == int(np.argmax(pred)) and bp == pytest.approx(pred.max())


def test_fit_rejects_bad_arguments(loops_lib):
    lp = loops_lib
    with pytest.raises(lp.LoopsError):
        lp.perf_model_fit(np.zeros(0), np.zeros(0), np.zeros(0))
