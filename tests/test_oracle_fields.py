"""Pins of the oracle's mesh geometry and field solver (Sec. 2.1, Eqs.
area-element, integral-form, fld-predictor/-corrector, App. B Eqs. D-update,
auxH, B-update, auxE; initial data of App. C).

Independent references: scipy quadrature of sqrt(gamma) (textbook Kerr,
tests/kerr_indep.py), exact closed forms of the a = 0 areas, the discrete
identity div(curl) = 0 behind div B = 0, the second-order convergence of the
discrete time derivative of stationary exact solutions, and the small-dt
limit of one predictor-corrector step."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
import kerr_indep as K


def rgrid(c, stag):
    i = np.arange(c.ld) - c.ng
    return c.r_in * np.exp((i + stag) * c.dx1)


def sqrtg_indep(a, r, th):
    alpha, _, _, _ = K.three_plus_one(a, r, th)
    return (r * r + a * a * math.cos(th) ** 2) * math.sin(th) / alpha


def test_areas_schwarzschild_closed_forms():
    """a = 0: sqrt(gamma) = r^2 sin(theta) sqrt(1 + 2/r); theta integrals are
    cosines, the r integral is a one-dimensional scipy quadrature."""
    c = O.make_cfg(16, 12, 0.0, 1.8, 30.0)
    AD, AB = O.areas(c)
    f = lambda r: r * r * math.sqrt(1 + 2 / r)
    Ir = lambda r0, r1: integrate.quad(f, r0, r1, epsabs=0, epsrel=1e-13)[0]
    rh = rgrid(c, 0.5)
    ri = rgrid(c, 0.0)
    for j in range(c.nth + 1):
        ta, tb = max(0.0, (j - 0.5) * c.dth), min(math.pi, (j + 0.5) * c.dth)
        for col in range(1, c.ld - 1):
            # D^r face: r = r_{i+1/2}, dual theta range (half width on the axis)
            assert AD[0][j, col] == pytest.approx(f(rh[col]) * (math.cos(ta) - math.cos(tb)), rel=1e-13)
            # D^phi: dual r and theta ranges
            assert AD[2][j, col] == pytest.approx(Ir(rh[col - 1], rh[col]) * (math.cos(ta) - math.cos(tb)), rel=1e-12)
            # B^theta face: theta_j, primal r range
            assert AB[1][j, col] == pytest.approx(Ir(ri[col], ri[col + 1]) * math.sin(j * c.dth), rel=1e-12, abs=1e-14)
            if j < c.nth:
                t0, t1 = j * c.dth, (j + 1) * c.dth
                assert AB[0][j, col] == pytest.approx(f(ri[col]) * (math.cos(t0) - math.cos(t1)), rel=1e-13)
                assert AB[2][j, col] == pytest.approx(Ir(ri[col], ri[col + 1]) * (math.cos(t0) - math.cos(t1)), rel=1e-12)
                assert AD[1][j, col] == pytest.approx(Ir(rh[col - 1], rh[col]) * math.sin((j + 0.5) * c.dth), rel=1e-12)


def test_areas_kerr_match_scipy_and_partition_the_shell():
    a = 0.9
    c = O.make_cfg(8, 8, a, 0.9 * O.horizon(a), 10.0)
    AD, AB = O.areas(c)
    rh = rgrid(c, 0.5)
    ri = rgrid(c, 0.0)
    col = c.ng + 3
    for j in (0, 3, 8):
        ta, tb = max(0.0, (j - 0.5) * c.dth), min(math.pi, (j + 0.5) * c.dth)
        ref = integrate.dblquad(lambda th, r: sqrtg_indep(a, r, th), rh[col - 1], rh[col], ta, tb,
                                epsabs=0, epsrel=1e-12)[0]
        assert AD[2][j, col] == pytest.approx(ref, rel=1e-10)
        ref = integrate.quad(lambda th: sqrtg_indep(a, rh[col], th), ta, tb, epsabs=0, epsrel=1e-13)[0]
        assert AD[0][j, col] == pytest.approx(ref, rel=1e-11)
    # dual volumes of one radial shell sum to the full shell volume
    shell = integrate.dblquad(lambda th, r: sqrtg_indep(a, r, th), rh[col - 1], rh[col], 0, math.pi,
                              epsabs=0, epsrel=1e-12)[0]
    assert AD[2][:, col].sum() == pytest.approx(shell, rel=1e-10)
    # primal B^phi faces of one row sum to the area of the whole theta range
    tot = integrate.dblquad(lambda th, r: sqrtg_indep(a, r, th), ri[col], ri[col + 1], 0, math.pi,
                            epsabs=0, epsrel=1e-12)[0]
    assert AB[2][:c.nth, col].sum() == pytest.approx(tot, rel=1e-10)


@pytest.mark.parametrize("kind", [O.WALD, O.WALD_A0, O.MONOPOLE, O.SPLIT_MONOPOLE])
@pytest.mark.parametrize("damp", [0.0, 0.1])
def test_initial_and_evolved_div_B_vanishes(kind, damp):
    """B^r, B^theta from Stokes' theorem on A_phi have zero discrete flux
    through every primal cell, and the curl update keeps it (Sec. 2.1).  The
    outer damping layer scales components independently, so with damping on
    the check covers the cells inside it."""
    a = 0.9
    c = O.make_cfg(24, 24, a, 0.9 * O.horizon(a), 20.0, damp_max=damp)
    D, B = O.init_fields(c, kind, 1.0)
    AD, AB = O.areas(c)
    scale = np.max(np.abs(B[0] * AB[0]))
    dB = O.divB(c, B)
    assert np.max(np.abs(dB[:, c.ng:c.ng + c.nr])) < 1e-13 * scale
    J = O.zeros_fields(c, 3)
    for _ in range(5):
        O.field_update(c, D, B, J)
    dB = O.divB(c, B)
    last = c.nr - (c.damp_cells + 1 if damp > 0 else 0)
    assert np.max(np.abs(dB[:, c.ng:c.ng + last])) < 1e-13 * scale


def _stationarity_errors(kind, n, a=0.9, T=0.5):
    c = O.make_cfg(n, n, a, 0.9 * O.horizon(a), 20.0, damp_max=0.0)
    ns = math.ceil(T / c.dt)
    c.dt = T / ns
    D, B = O.init_fields(c, kind, 1.0)
    X0 = [x.copy() for x in D + B]
    J = O.zeros_fields(c, 3)
    for _ in range(ns):
        O.field_update(c, D, B, J)
    rH = O.horizon(a)
    r = rgrid(c, 0.0)
    th = np.arange(c.nth + 1) * c.dth
    mask = (r[None, :] > 1.5 * rH) & (r[None, :] < 10) & (th[:, None] > 0.4) & (th[:, None] < math.pi - 0.4)
    errs = []
    for X, Y in zip(D + B, X0):
        sc = np.max(np.abs(Y[mask]))
        errs.append(np.max(np.abs(X - Y)[mask]) / sc)
    return np.array(errs)


@pytest.mark.parametrize("kind", [O.WALD, O.MONOPOLE])
def test_exact_solutions_are_discretely_stationary_to_second_order(kind):
    """The rotating Wald solution and the monopole are exact stationary vacuum
    solutions (Sec. 3.2, App. C); the solver's drift over a fixed time must fall
    by ~4x per doubling of resolution for all six components.  Any sign error,
    missing 1/2 or wrong edge length in Eqs. auxE/auxH/D-update/B-update gives
    an O(1) drift instead."""
    e1 = _stationarity_errors(kind, 48)
    e2 = _stationarity_errors(kind, 96)
    ratio = e1 / e2
    assert np.all(ratio > 3.5) and np.all(ratio < 4.5), ratio
    assert np.all(e2 < 2e-3), e2


def test_corrector_prefactor_small_dt_limit():
    """As dt -> 0 one predictor + N correctors step gives
    (D^{n+1} - D^n)/dt -> C_H(D^n, B^n) - J (and C_E for B): the prefactor in
    Eq. fld-corrector is dt (alpha + beta = 1), not dt/2."""
    a = 0.9
    c = O.make_cfg(16, 16, a, 0.9 * O.horizon(a), 20.0, damp_max=0.0)
    rng = np.random.default_rng(3)
    D, B = O.init_fields(c, O.WALD_A0, 1.0)   # not stationary in a spinning metric
    J = [rng.normal(size=O.field_shape(c)) * 1e-2 for _ in range(3)]
    CD, CB = O.circulations(c, D, B)
    c.dt = 1e-7
    D1 = [x.copy() for x in D]
    B1 = [x.copy() for x in B]
    O.field_update(c, D1, B1, J)
    sl = (slice(2, c.nth - 1), slice(c.ng + 1, c.ng + c.nr - 1))
    for k in range(3):
        rateD = (D1[k] - D[k]) / c.dt
        ref = CD[k] - J[k]
        assert np.max(np.abs(rateD - ref)[sl]) < 1e-5 * np.max(np.abs(ref[sl])), k
        rateB = (B1[k] - B[k]) / c.dt
        if np.max(np.abs(CB[k][sl])) > 0:
            assert np.max(np.abs(rateB - CB[k])[sl]) < 1e-5 * np.max(np.abs(CB[k][sl])), k


def test_boundary_conditions_after_update():
    a = 0.9
    c = O.make_cfg(16, 16, a, 0.9 * O.horizon(a), 20.0)
    D, B = O.init_fields(c, O.WALD, 1.0)
    O.field_update(c, D, B, O.zeros_fields(c, 3))
    # axis: D^phi = B^theta = 0 at theta = 0, pi (Sec. 2.1)
    for row in (0, c.nth):
        assert np.all(D[2][row] == 0) and np.all(B[1][row] == 0)
    # inner guard cells copy the first physical cell (zero derivative)
    for X in D + B:
        for g in range(c.ng):
            np.testing.assert_array_equal(X[:, g], X[:, c.ng])


def test_damping_layer_leaves_the_interior_and_only_scales_the_outer_columns():
    """The outer absorbing layer (a reading: the paper gives no profile) acts
    only on the last damp_cells columns, once per step, as a factor in
    [1 - d_max, 1] that does not increase outwards; elsewhere one update is
    bit-identical to the undamped one."""
    a = 0.9
    out = {}
    for damp in (0.0, 0.1):
        c = O.make_cfg(32, 24, a, 0.9 * O.horizon(a), 20.0, damp_max=damp)
        D, B = O.init_fields(c, O.WALD, 1.0)
        rng = np.random.default_rng(4)
        J = [rng.normal(size=O.field_shape(c)) * 0.01 for _ in range(3)]
        O.field_update(c, D, B, J)
        out[damp] = (c, D + B)
    c, und = out[0.0]
    _, dam = out[0.1]
    first = c.nr - c.damp_cells
    for k, (x, y) in enumerate(zip(dam, und)):
        cols_in = slice(0, c.ng + first - 1)
        assert np.array_equal(x[:, cols_in], y[:, cols_in]), k
        ratio = np.divide(x[:, c.ng + first:c.ng + c.nr], y[:, c.ng + first:c.ng + c.nr],
                          out=np.ones_like(x[:, c.ng + first:c.ng + c.nr]),
                          where=np.abs(y[:, c.ng + first:c.ng + c.nr]) > 1e-12)
        assert ratio.min() >= 1.0 - 0.1 - 1e-12 and ratio.max() <= 1.0 + 1e-12, k
        prof = np.median(ratio, axis=0)
        assert np.all(np.diff(prof) <= 1e-12), k
