"""Pins of the oracle's Kerr-Schild 3+1 metric (App. A, Eqs. ks-coefficients,
gamma-inverse, ks-alpha-beta) against the textbook Boyer-Lindquist Kerr metric
moved to Kerr-Schild coordinates (tests/kerr_indep.py), and of its quadrature
rule against numpy's Gauss-Legendre routine."""
import math

import numpy as np
import pytest

import oracle as O
import kerr_indep as K

POINTS = [(0.9, 1.3, 0.4), (0.9, 3.0, 1.2), (0.99, 1.05, 2.9), (0.0, 5.0, 0.7), (0.5, 20.0, 1.5708),
          (0.998, 1.2, 0.05), (0.9, 48.0, 3.0)]


@pytest.mark.parametrize("a,r,th", POINTS)
def test_metric_matches_boyer_lindquist_transform(a, r, th):
    m = O.metric(a, r, th)
    alpha, beta, gam, gam_inv = K.three_plus_one(a, r, th)
    assert m["alpha"] == pytest.approx(alpha, rel=1e-13)
    assert m["beta"] == pytest.approx(beta[0], rel=1e-12)
    assert abs(beta[1]) < 1e-13 and abs(beta[2]) < 1e-12
    assert m["g_rr"] == pytest.approx(gam[0, 0], rel=1e-13)
    assert m["g_thth"] == pytest.approx(gam[1, 1], rel=1e-13)
    assert m["g_pp"] == pytest.approx(gam[2, 2], rel=1e-12)
    assert m["g_rp"] == pytest.approx(gam[0, 2], rel=1e-12, abs=1e-14)
    assert abs(gam[0, 1]) < 1e-14 and abs(gam[1, 2]) < 1e-14
    # closed-form inverse (Eq. gamma-inverse) against the numerical inverse
    assert m["gi_rr"] == pytest.approx(gam_inv[0, 0], rel=1e-11)
    assert m["gi_rp"] == pytest.approx(gam_inv[0, 2], rel=1e-11, abs=1e-14)
    assert m["gi_thth"] == pytest.approx(gam_inv[1, 1], rel=1e-12)
    assert m["gi_pp"] == pytest.approx(gam_inv[2, 2], rel=1e-10)
    # sqrt(-g) = rho^2 sin(theta) for Kerr (BL and KS alike), = alpha sqrt(gamma)
    rho2 = r * r + a * a * math.cos(th) ** 2
    assert m["alpha"] * m["sqrtg"] == pytest.approx(rho2 * math.sin(th), rel=1e-12)
    assert math.sqrt(-np.linalg.det(K.g_ks(a, r, th))) == pytest.approx(rho2 * math.sin(th), rel=1e-10)


DERIV = [("alpha", "da"), ("beta", "db"), ("gi_rr", "dgi_rr"), ("gi_rp", "dgi_rp"), ("gi_thth", "dgi_thth"),
         ("gi_pp", "dgi_pp")]


@pytest.mark.parametrize("a,r,th", POINTS)
def test_metric_derivatives_match_finite_differences(a, r, th):
    m = O.metric(a, r, th)
    h = 1e-4 * min(1.0, th, math.pi - th)
    for k, (name, dname) in enumerate(DERIV):
        for d, suffix in ((0, "_r"), (1, "_th")):
            def f(x):
                return O.metric(a, r + x, th)[name] if d == 0 else O.metric(a, r, th + x)[name]
            fd = (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)
            scale = max(abs(fd), abs(m[name]), 1e-12)
            assert abs(m[dname + suffix] - fd) <= 1e-7 * scale, (name, suffix, m[dname + suffix], fd)


def test_gauss_legendre_nodes_match_numpy():
    x, w = O.gauss_legendre()
    xr, wr = np.polynomial.legendre.leggauss(10)
    order = np.argsort(x)
    np.testing.assert_allclose(x[order], xr, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w[order], wr, rtol=0, atol=1e-14)
