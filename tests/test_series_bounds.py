"""Truncation bounds of the series the FP32 lattice kernels use in place of a
square root and a division (host mathematics, no GPU).

With x = num / |xi|^2 and r = sqrt(1 + x), the stencil kernels evaluate, to x^2:
  * the bond force coefficient's g(x) = 1 / (r (1 + r))        (Eqs. 4-5: num / D = num g / |xi|^3),
  * the state-based dilation term's 1 / (1 + r)                 (|xi| e~ = num / (1 + r)),
  * the state-based force factors |xi| / |y| = (1 + x)^(-1/2)
    and e~ / |y| = 1 - (1 + x)^(-1/2)                           (t / |y| of the linear solid),
and take the exact forms past |x| = 3e-3.  The claim checked here: within that
range every series is below a quarter of an FP32 ulp of its value, and past it
(|x| = 1e-2) the bond coefficient's series is not.
"""
import numpy as np

X_MAX = 3e-3                 # the series' range in the kernels
QUARTER_ULP = 2.0 ** -25     # a quarter of an FP32 ulp, relative to the value (at most)


def _g(x):
    r = np.sqrt(1.0 + x)
    return 1.0 / (r * (1.0 + r))


def _g_series(x):
    return 0.5 - 0.375 * x + 0.3125 * x * x


def _dil(x):
    return 1.0 / (1.0 + np.sqrt(1.0 + x))


def _dil_series(x):
    return 0.5 - 0.125 * x + 0.0625 * x * x


def _p(x):
    return np.exp(-0.5 * np.log1p(x))


def _p_series(x):
    return 1.0 - 0.5 * x + 0.375 * x * x


def _q(x):  # 1 - (1 + x)^(-1/2), without cancellation
    return -np.expm1(-0.5 * np.log1p(x))


def _q_series(x):
    return x * (0.5 - 0.375 * x + 0.3125 * x * x)


def _rel(a, b):
    return np.abs(a - b) / np.abs(b)


def _grid(xmax):
    x = np.concatenate([np.linspace(-xmax, xmax, 20001), -np.logspace(-9, np.log10(xmax), 200),
                        np.logspace(-9, np.log10(xmax), 200)])
    return x[x != 0.0]


def test_series_within_a_quarter_ulp_in_range():
    x = _grid(X_MAX)
    for exact, series in ((_g, _g_series), (_dil, _dil_series), (_p, _p_series),
                          (_q, _q_series)):
        err = _rel(series(x), exact(x)).max()
        assert err < QUARTER_ULP, (exact.__name__, err)


def test_next_terms_match_the_series_error():
    # the leading truncation terms: -35 x^3 / 128 for g, -5 x^3 / 128 for 1 / (1 + r),
    # -5 x^3 / 16 for (1 + x)^(-1/2), -35 x^4 / 128 for 1 - (1 + x)^(-1/2)
    x = np.array([-X_MAX, -1e-3, 1e-3, X_MAX])
    for exact, series, nxt in ((_g, _g_series, -35.0 / 128 * x ** 3),
                               (_dil, _dil_series, -5.0 / 128 * x ** 3),
                               (_p, _p_series, -5.0 / 16 * x ** 3),
                               (_q, _q_series, -35.0 / 128 * x ** 4)):
        d = exact(x) - series(x)
        assert np.allclose(d, nxt, rtol=0.02, atol=0.0), (exact.__name__, d, nxt)


def test_past_the_range_the_exact_form_is_needed():
    x = np.array([-1e-2, 1e-2])
    assert _rel(_g_series(x), _g(x)).max() > 10 * QUARTER_ULP
