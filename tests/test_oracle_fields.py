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


def _pulse_run(nr, damp, nsteps, nth=16, src_col=36, width=100.0, probe=(46, 54), layer=(56, 64)):
    """Vacuum Schwarzschild run (a = 0, r_in = 0.9 r_H) driven by a ring
    current J^phi ~ sin^2(theta) exp(-((n - 3w)/w)^2) at column src_col:
    a transient source whose wave leaves outwards (its ingoing half falls
    into the hole).  The grid has the cell size and time step of a 64-column
    grid on [r_in, 20]; nr > 64 extends it outwards with the same cells.
    Returns the fields of the probe columns at every step and the
    area-weighted field energy sum F^2 A of the layer columns."""
    a = 0.0
    rin = 0.9 * O.horizon(a)
    base = O.make_cfg(64, nth, a, rin, 20.0)
    c = O.make_cfg(nr, nth, a, rin, rin * math.exp(nr * base.dx1), dt=base.dt, damp_max=damp, damp_cells=8)
    D, B, J = O.zeros_fields(c, 3), O.zeros_fields(c, 3), O.zeros_fields(c, 3)
    AD, AB = O.areas(c)
    prof = np.sin(np.arange(nth + 1) * c.dth) ** 2
    cols = slice(probe[0] + c.ng, probe[1] + c.ng)
    lay = slice(layer[0] + c.ng, layer[1] + c.ng)
    hist, energy = [], []
    for n in range(nsteps):
        J[2][:, src_col + c.ng] = 1e-2 * math.exp(-((n - 3 * width) / width) ** 2) * prof
        O.field_update(c, D, B, J)
        hist.append(np.stack([x[:, cols] for x in D + B]))
        energy.append(sum(np.sum(x[:, lay] ** 2 * w[:, lay]) for x, w in zip(D + B, AD + AB)))
    return np.array(hist), np.array(energy)


def test_damping_layer_absorbs_an_outgoing_pulse():
    """The outer layer's job (Sec. 2.1: the fields are damped to zero at the
    outer boundary, so that outgoing waves leave the domain).  An outgoing
    pulse crosses a 64-column grid with the layer in its last 8 columns; the
    reference is the same run on a grid extended to 112 columns with no
    damping, whose outer boundary the pulse never reaches in the run.  The
    difference of the two in the probe columns between source and layer is
    the wave the layer sends back:
      * its peak is below 13 % of the pulse's peak there (measured 10 %;
        without the layer the zero-derivative boundary sends back 2.6 times
        the pulse, and a layer that damps the r-staggered components D^r,
        B^theta, B^phi at integer columns instead of their own half-integer
        ones sends back 18 %);
      * once the pulse has entered, the energy of the layer columns falls
        monotonically from its peak to below 20 % of it, while the undamped
        run still holds over half of its own peak in those columns;
      * the layer never holds more energy than the same columns of the
        undamped run (to 1e-6 relative: the mis-staggered layer exceeds it by
        5e-5)."""
    n = 1400
    h1, e1 = _pulse_run(64, 0.1, n)
    h2, e2 = _pulse_run(112, 0.0, n)
    norm = lambda x: np.sqrt(np.sum(x.reshape(len(x), -1) ** 2, axis=1))
    ref = norm(h2)
    refl = norm(h1 - h2)
    assert refl.max() < 0.13 * ref.max(), refl.max() / ref.max()
    pk = int(np.argmax(e1))
    end = pk + int(np.argmax(e1[pk:] < 0.2 * e1[pk]))
    assert end > pk and e1[end] < 0.2 * e1[pk]
    assert np.all(np.diff(e1[pk:end + 1]) <= 0.0)
    assert e2[end] > 0.5 * e2.max()
    assert np.all(e1[1:] <= e2[1:] * (1.0 + 1e-6))


def test_damping_profile_is_the_cubic_reading():
    """The profile the layer uses (reading: the paper names the damping, not
    its form) is f = 1 - d_max s^3 with s = (x - (n_r - N_d)) / N_d clipped
    to [0, 1] at each component's own r position x (i + 1/2 for D^r, B^theta,
    B^phi; i for D^theta, D^phi, B^r), applied once after the last corrector
    and followed by the boundary pass.  From one state, the damped update
    equals the undamped one times f entry by entry (to rounding), every
    column left of the layer is bit-identical, and the outer guard columns
    copy the damped last physical column."""
    a = 0.9
    out = {}
    for damp in (0.0, 0.1):
        c = O.make_cfg(48, 24, a, 0.9 * O.horizon(a), 20.0, damp_max=damp, damp_cells=12)
        D, B = O.init_fields(c, O.WALD, 1.0)
        rng = np.random.default_rng(4)
        J = [rng.normal(size=O.field_shape(c)) * 0.01 for _ in range(3)]
        O.field_update(c, D, B, J)
        out[damp] = (c, D + B)
    c, und = out[0.0]
    _, dam = out[0.1]
    x0 = c.nr - c.damp_cells
    for comp, (x, y) in enumerate(zip(dam, und)):
        half_r = comp in (0, 4, 5)
        half_t = comp in (1, 3, 5)
        rows = slice(0, c.nth if half_t else c.nth + 1)
        last = c.nr - 1 if half_r else c.nr
        i = np.arange(0, last + 1)
        s = np.clip((i + (0.5 if half_r else 0.0) - x0) / c.damp_cells, 0.0, 1.0)
        f = 1.0 - 0.1 * s ** 3
        cols = i + c.ng
        xv, yv = x[rows][:, cols], y[rows][:, cols]
        assert np.all(np.abs(xv - f * yv) <= 2e-16 * np.abs(yv) + 1e-300), comp
        inner = cols[s == 0.0]
        assert np.array_equal(xv[:, s == 0.0], yv[:, s == 0.0]), comp
        assert inner.size > 0 and np.any(s > 0.9)
        for g in range(last + 1 + c.ng, c.ld):
            assert np.array_equal(x[rows][:, g], x[rows][:, last + c.ng]), (comp, g)
