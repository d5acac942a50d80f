"""Pins of the oracle's horizon Poynting flux, the objective of the
differentiable form: the radial component of S = E x H of the 3+1 fields
(Sec. 2.1, the Komissarov form E = alpha D + beta x B, H = alpha B - beta x D
with the auxiliary fields of App. B) summed over the ring of faces at r_iH.

Independent references:
  * the continuum integral of (E_theta H_phi - E_phi H_theta) over theta at
    r_iH, with E and H formed from analytic D, B by the textbook 3+1 metric
    (tests/kerr_indep.py) and the Levi-Civita tensor sqrt(gamma) [ijk], and
    scipy quadrature: the discrete ring sum converges to it at second order;
  * energy conservation: a stationary vacuum field (Wald) carries no net
    energy flux through any sphere, so the sum vanishes up to discretisation;
    with a = 0 the monopole has no electric field and the sum vanishes.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import kerr_indep as K
import oracle as O

A = 0.9
R_IN, R_OUT = 1.3, 20.0

# staggering (r, theta) of D^r, D^th, D^ph, B^r, B^th, B^ph (Yee lattice)
STAG = [(0.5, 0.0), (0.0, 0.5), (0.0, 0.0), (0.0, 0.5), (0.5, 0.0), (0.5, 0.5)]


def fields_analytic(r, th):
    """Smooth test fields (contravariant D^i, B^i), not a solution of anything."""
    s, c = math.sin(th), math.cos(th)
    D = np.array([0.5 * c / r**2 + 0.1, 0.3 * s * c / r**3, 0.2 / r**2 + 0.05 * c])
    B = np.array([c / r**2 + 0.2, 0.4 * s / r**3, 0.25 * c / r**2 - 0.1])
    return D, B


def levi(gamma_det_sqrt):
    e = np.zeros((3, 3, 3))
    for (i, j, k), sgn in {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1, (0, 2, 1): -1, (2, 1, 0): -1, (1, 0, 2): -1}.items():
        e[i, j, k] = sgn * gamma_det_sqrt
    return e


def EH(a, r, th):
    alpha, beta, gam, _ = K.three_plus_one(a, r, th)
    eps = levi(math.sqrt(np.linalg.det(gam)))
    D, B = fields_analytic(r, th)
    E = alpha * gam @ D + np.einsum("ijk,j,k->i", eps, beta, B)
    H = alpha * gam @ B - np.einsum("ijk,j,k->i", eps, beta, D)
    return E, H


def continuum_flux(a, r):
    def f(th):
        E, H = EH(a, r, th)
        return E[1] * H[2] - E[2] * H[1]
    v, _ = integrate.quad(f, 0.0, math.pi, epsabs=1e-14, epsrel=1e-12, limit=200)
    return v


def sampled(c, fn):
    shape = O.field_shape(c)
    D = [np.zeros(shape) for _ in range(3)]
    B = [np.zeros(shape) for _ in range(3)]
    for comp in range(6):
        sr, st = STAG[comp]
        arr = D[comp] if comp < 3 else B[comp - 3]
        for j in range(c.nth + 1):
            th = (j + st) * c.dth
            for col in range(c.ld):
                r = c.r_in * math.exp((col - c.ng + sr) * c.dx1)
                d, b = fn(r, th)
                arr[j, col] = (d if comp < 3 else b)[comp % 3]
    return D, B


def ring_case(n):
    """Grid whose column n/4 sits at the same radius for every n."""
    c = O.make_cfg(n, n, A, R_IN, R_OUT)
    iH = n // 4
    return c, iH, c.r_in * math.exp(iH * c.dx1)


def test_flux_converges_to_the_continuum_integral_at_second_order():
    errs = []
    for n in (32, 64, 128):
        c, iH, r = ring_case(n)
        D, B = sampled(c, fields_analytic)
        ref = continuum_flux(A, r)
        errs.append(abs(O.horizon_flux(c, D, B, iH) - ref) / abs(ref))
    assert errs[2] < 2e-3, errs
    assert 3.0 < errs[0] / errs[1] < 5.5 and 3.0 < errs[1] / errs[2] < 5.5, errs


def test_flux_is_a_quadratic_form():
    c, iH, _ = ring_case(32)
    D, B = sampled(c, fields_analytic)
    rng = np.random.default_rng(5)
    D2 = [rng.normal(size=x.shape) for x in D]
    B2 = [rng.normal(size=x.shape) for x in B]
    f = lambda s: O.horizon_flux(c, [x + s * y for x, y in zip(D, D2)], [x + s * y for x, y in zip(B, B2)], iH)
    f0, f1, fm = f(0.0), f(1.0), f(-1.0)
    f2 = f(2.0)
    # a quadratic in s has vanishing third difference
    assert abs(f2 - 3 * f1 + 3 * f0 - fm) < 1e-12 * max(abs(f2), abs(f1), 1.0)
    assert O.horizon_flux(c, [2 * x for x in D], [2 * x for x in B], iH) == pytest.approx(4 * f0, rel=1e-13)


def test_vacuum_wald_carries_no_net_flux():
    vals = []
    for n in (32, 64, 128):
        c = O.make_cfg(n, n, A, 0.9 * O.horizon(A), 20.0)
        D, B = O.init_fields(c, 0, 1.0)
        iH = O.horizon_index(c, A)
        vals.append(abs(O.horizon_flux(c, D, B, iH)))
    assert vals[2] < vals[1] < vals[0]
    assert vals[2] < 1e-3


def test_schwarzschild_monopole_has_no_flux():
    c = O.make_cfg(32, 32, 0.0, 0.9 * 2.0, 20.0)
    D, B = O.init_fields(c, 2, 1.0)
    assert np.all(D[0] == 0) and np.all(D[1] == 0) and np.all(D[2] == 0)
    # E = beta x B vanishes up to the rounding of the closed-form zeros of B^th, B^ph
    assert abs(O.horizon_flux(c, D, B, O.horizon_index(c, 0.0))) < 1e-28
