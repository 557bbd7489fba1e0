"""The automatic series and order of the contour factor exp(beta_I s) (Eq. 22 and its
Chebyshev form) through cfft_contour_series_order, host only (no device).

The library bounds the remainders with its own power series for I_m; here the bounds are
evaluated independently with scipy's modified Bessel functions and the log-gamma function:
- Taylor: x^(N+1) / (N+1)! e^x;  Chebyshev: e^a 2 sum_{m>N} I_m(a), a = x / 2;
- the chosen order is the smallest whose bound is at most 1e-13 (FP64) or 2^-22 (FP32);
- the automatic choice takes the series with fewer transforms (Taylor on a tie);
- the full-size patch (height * rho_max = 1.2066) takes Chebyshev degree 6 in FP32 (8
  transforms), the strip of the series test (2.7) 16 Chebyshev transforms against 25 Taylor
  in FP64.
"""
import math

import pytest

from paper_1404_7357_gb300 import cfft

scipy_special = pytest.importorskip("scipy.special")

TOL = {cfft.CFFT_FP64: 1e-13, cfft.CFFT_FP32_MIXED: 2.0 ** -22}


def taylor_bound(x, n):
    return math.exp((n + 1) * math.log(x) - math.lgamma(n + 2) + x)


def chebyshev_bound(x, n):
    a = 0.5 * x
    return math.exp(a) * 2.0 * sum(scipy_special.iv(m, a) for m in range(n + 1, n + 120))


BOUND = {0: taylor_bound, 1: chebyshev_bound}


@pytest.mark.parametrize("precision", [cfft.CFFT_FP64, cfft.CFFT_FP32_MIXED])
@pytest.mark.parametrize("x", [0.05, 0.3, 1.2066, 2.7, 3.0, 5.0])
def test_order_is_the_smallest_within_the_bound(x, precision):
    tol = TOL[precision]
    for opt, series in ((1, 0), (2, 1)):
        s, n, f = cfft.contour_series_order(x, precision, opt)
        assert s == series
        assert f == n + (2 if series == 1 else 1)
        # the library's own tail sums stop early: allow 1 % on either side of the bound
        assert BOUND[series](x, n) <= 1.01 * tol, (x, series, n)
        assert n == 0 or BOUND[series](x, n - 1) > 0.99 * tol, (x, series, n)


@pytest.mark.parametrize("precision", [cfft.CFFT_FP64, cfft.CFFT_FP32_MIXED])
@pytest.mark.parametrize("x", [0.0, 0.05, 0.3, 1.2066, 2.7, 3.0, 5.0])
def test_automatic_choice_takes_fewer_transforms(x, precision):
    s, n, f = cfft.contour_series_order(x, precision, 0)
    ft = cfft.contour_series_order(x, precision, 1)[2]
    fc = cfft.contour_series_order(x, precision, 2)[2]
    assert f == min(ft, fc)
    assert s == (1 if fc < ft else 0)   # Taylor on a tie


def test_workload_orders():
    assert cfft.contour_series_order(1.2066, cfft.CFFT_FP32_MIXED) == (1, 6, 8)
    assert cfft.contour_series_order(0.0, cfft.CFFT_FP32_MIXED) == (0, 0, 1)
    assert cfft.contour_series_order(2.7, cfft.CFFT_FP64, 2)[2] == 16
    assert cfft.contour_series_order(2.7, cfft.CFFT_FP64, 1)[2] == 25


@pytest.mark.parametrize("x,precision", [(-1.0, cfft.CFFT_FP32_MIXED), (float("nan"), cfft.CFFT_FP64),
                                         (float("inf"), cfft.CFFT_FP64), (1.0, 7), (500.0, cfft.CFFT_FP64)])
def test_refused_arguments(x, precision):
    with pytest.raises(cfft.CfftError) as ei:
        cfft.contour_series_order(x, precision)
    assert ei.value.status == 1
