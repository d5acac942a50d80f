"""Pins of the oracle's charge-conserving deposit (Sec. 2.3, Eqs.
charge-continuity, J-integral-eqn, esirkepov-decomp, j-phi-deposit), its field
interpolation, its full time step (continuity of Sec. 3.4) and its sort.

Independent references: the discrete continuity equation written out with a
cloud-in-cell shape of the test's own, the total current moments of a moving
charge, exactness of bilinear interpolation on linear data, the stable
argsort of numpy; for the third-order (cubic B-) spline shape its moments and
knot smoothness, the same continuity with the test's own folded cubic
density, and linear reproduction."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2503_04558_gb300 import synth


def cfg(n=12, a=0.9, **kw):
    return O.make_cfg(n, n, a, 0.9 * O.horizon(a), 20.0, **kw)


def cic_density(c, x1, x2, q):
    """q * S_kl at every vertex (k, l), test's own cloud-in-cell."""
    out = np.zeros(O.field_shape(c))
    i, j = int(math.floor(x1)), min(int(math.floor(x2)), c.nth - 1)
    for k in (i, i + 1):
        for l in (j, j + 1):
            w = max(0.0, 1 - abs(x1 - k)) * max(0.0, 1 - abs(x2 - l))
            out[l, k + c.ng] += q * w
    return out


def divergence_of_flux(c, JrA, JtA):
    """(JrA_{k} - JrA_{k-1}) + (JtA_{l} - JtA_{l-1}) at every vertex (k, l)."""
    div = np.zeros_like(JrA)
    div[:, 1:] += JrA[:, 1:] - JrA[:, :-1]
    div[:, 0] += JrA[:, 0]
    div[:c.nth, :] += JtA[:c.nth, :]
    div[1:, :] -= JtA[:c.nth, :]
    return div


MOVES = [((3.2, 4.7), (3.9, 5.3)), ((3.95, 4.05), (4.05, 3.95)), ((5.5, 5.5), (4.6, 6.4)), ((2.0, 2.0), (2.9, 2.0)),
         ((6.3, 0.3), (6.1, 0.05)), ((7.5, 11.6), (7.2, 11.95)), ((0.2, 6.0), (-0.4, 6.3)), ((11.7, 3.0), (12.3, 3.1))]


@pytest.mark.parametrize("p0,p1", MOVES)
def test_single_particle_continuity_is_exact(p0, p1):
    """q (S^{n+1} - S^n) = -dt * div(J A) at every vertex (Eq. J-integral-eqn)."""
    c = cfg()
    qw = 0.37
    JrA, JtA, Jph = O.deposit_one(c, qw, p0[0], p0[1], p1[0], p1[1], 0.0)
    drho = cic_density(c, *p1, qw) - cic_density(c, *p0, qw)
    div = divergence_of_flux(c, JrA, JtA)
    np.testing.assert_allclose(drho, -c.dt * div, rtol=0, atol=1e-15)
    assert np.all(Jph == 0)


def test_static_particle_and_radial_motion():
    c = cfg()
    JrA, JtA, Jph = O.deposit_one(c, 1.0, 4.3, 5.6, 4.3, 5.6, 0.0)
    assert np.all(JrA == 0) and np.all(JtA == 0) and np.all(Jph == 0)
    JrA, JtA, Jph = O.deposit_one(c, 1.0, 4.3, 5.6, 4.9, 5.6, 0.0)
    assert np.all(JtA == 0)
    JrA, JtA, Jph = O.deposit_one(c, 1.0, 4.3, 5.6, 4.3, 5.1, 0.0)
    assert np.all(JrA == 0)


@pytest.mark.parametrize("q", [1.0, -2.0])
def test_current_moments_and_signs(q):
    """A charge moving by (dx1, dx2, dphi) in one step carries total
    sum JrA = q dx1/dt, sum JtA = q dx2/dt (logical units) and
    sum J^phi dV = q dphi/dt; each current has the sign of q times the
    velocity component (the 3-current is a vector)."""
    c = cfg()
    AD, AB = O.areas(c)
    x0, x1 = (4.3, 5.6), (4.8, 5.45)
    dphi = 0.013
    JrA, JtA, Jph = O.deposit_one(c, q, *x0, *x1, dphi)
    assert JrA.sum() == pytest.approx(q * (x1[0] - x0[0]) / c.dt, rel=1e-12)
    assert JtA.sum() == pytest.approx(q * (x1[1] - x0[1]) / c.dt, rel=1e-12)
    assert (Jph * AD[2]).sum() == pytest.approx(q * dphi / c.dt, rel=1e-12)
    for X, sgn in ((JrA, np.sign(q)), (JtA, -np.sign(q)), (Jph, np.sign(q))):
        big = np.abs(X) > 1e-12 * np.max(np.abs(X))
        assert np.all(np.sign(X[big]) == sgn)


def test_interpolation_reproduces_linear_fields_and_axis_parity():
    c = cfg()
    stag = [(0.5, 0.0), (0.0, 0.5), (0.0, 0.0), (0.0, 0.5), (0.5, 0.0), (0.5, 0.5)]
    coef = [(0.3, 1.1, -0.7), (-2.0, 0.4, 0.9), (1.5, -0.3, 0.2), (0.1, 0.2, 0.3), (-0.6, 0.8, -1.2), (2.2, 0.5, 0.5)]
    F = []
    for (sr, st), (a0, a1, a2) in zip(stag, coef):
        col = np.arange(c.ld) - c.ng + sr
        row = np.arange(c.nth + 1) + st
        F.append(a0 + a1 * col[None, :] + a2 * row[:, None])
    for x1, x2 in [(3.3, 4.6), (0.1, 7.2), (11.9, 1.3), (5.5, 5.5)]:
        v = O.interp(c, F[:3], F[3:], x1, x2)
        ref = [a0 + a1 * x1 + a2 * x2 for (a0, a1, a2) in coef]
        np.testing.assert_allclose(v, ref, rtol=0, atol=1e-13)
    # within half a cell of the axis the half-theta lattice mirrors across it:
    # theta components odd, r and phi components even
    G = [np.zeros(O.field_shape(c)) for _ in range(6)]
    for k in range(6):
        G[k][:, :] = 1.0
    v = O.interp(c, G[:3], G[3:], 4.2, 0.25)
    g = 0.75  # weight of row 0 (theta_{1/2}) for x2 - 1/2 = -0.25
    assert v[1] == pytest.approx(g * 1.0 + (1 - g) * (-1.0))   # D^theta
    assert v[3] == pytest.approx(1.0) and v[5] == pytest.approx(1.0)  # B^r, B^phi
    assert v[0] == pytest.approx(1.0) and v[2] == pytest.approx(1.0)


def _charge_residual(c, D0, P0, D1, P1):
    """max over interior vertices of |(div D - rho)^1 - (div D - rho)^0|.
    Interior: from column 1 (the cubic shape: 2, since a particle absorbed
    just inside r_in still covers vertex 1 with its cloud) to the damping
    layer."""
    r0 = O.divD(c, D0) - O.rho(c, P0)
    r1 = O.divD(c, D1) - O.rho(c, P1)
    last = c.nr - c.damp_cells - 1
    first = 2 if c.shape == 3 else 1
    sl = (slice(0, c.nth + 1), slice(c.ng + first, c.ng + last + 1))
    return np.max(np.abs(r1 - r0)[sl]), np.max(np.abs(O.rho(c, P1)[sl]))


def test_full_steps_conserve_charge_to_round_off():
    """Sec. 3.4: with the Esirkepov deposit div D - rho holds to round-off
    through push, deposit, field update and sort (interior vertices; the guard
    copy at r_in and the damping layer break it by design)."""
    c = cfg(n=24, qw=(-0.05, 0.05, 0.05, 0.0))
    D, B = O.init_fields(c, O.WALD, 1.0)
    arrs = synth.particles(c.nr, c.nth, c.r_in, c.r_out, 3000, seed=7, sigma=0.6)
    P = O.Particles(*arrs)
    # one particle heading through the axis and one through the inner boundary
    P.th[0], P.u2[0] = 0.3 * c.dth, -3.0 * P.r[0]
    P.r[2], P.u1[2] = c.r_in * math.exp(0.1 * c.dx1), -3.0
    D0 = [x.copy() for x in D]
    P0 = P.copy()
    worst = 0.0
    for _ in range(6):
        st, P, J = O.step(c, P, D, B)
        assert st == 0
        res, rmax = _charge_residual(c, D0, P0, D, P)
        worst = max(worst, res / rmax)
    assert worst < 1e-12, worst
    assert P.n < 3000   # the inner-boundary particle left the domain


# ---------------------------------------------------------------------------
# third-order spline shape (the configuration option of Sec. 2.3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("x", [0.0, 0.37, 0.5, 0.93, -1.2, 2.71])
def test_cubic_spline_weights_are_the_cubic_b_spline(x):
    """Partition of unity, first moment x and second moment x^2 + 1/3 (the
    variance of four unit boxes convolved) over the 4 nonzero weights, support
    |d| < 2, and C^2 joins at the knots 1 and 2."""
    ks = np.arange(math.floor(x) - 3, math.floor(x) + 5)
    w = np.array([O.w3(x - k) for k in ks])
    assert np.all(w >= 0) and np.count_nonzero(w) <= 4
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert (ks * w).sum() == pytest.approx(x, abs=1e-14)
    assert (ks * ks * w).sum() == pytest.approx(x * x + 1.0 / 3.0, abs=1e-13)
    for knot in (1.0, 2.0):
        h = 1e-5
        d1 = [(O.w3(knot + s * h + h) - O.w3(knot + s * h - h)) / (2 * h) for s in (-2, 2)]
        d2 = [(O.w3(knot + s * h + h) - 2 * O.w3(knot + s * h) + O.w3(knot + s * h - h)) / h ** 2 for s in (-2, 2)]
        # one-sided values 4h apart: the first derivatives differ by about
        # 4h times the second, the second derivatives by 4h times the third
        assert abs(d1[0] - d1[1]) < 10 * h and abs(d2[0] - d2[1]) < 1e-3
    assert O.w3(2.0) == 0.0 and O.w3(2.5) == 0.0


def cubic_density(c, x1, x2, q):
    """q * S_kl at every vertex with the cubic shape, rows past the polar axis
    added to their mirror rows (theta -> -theta, 2 pi - theta)."""
    out = np.zeros(O.field_shape(c))
    i, j = int(math.floor(x1)), int(math.floor(x2))
    for k in range(i - 1, i + 3):
        if k < -c.ng or k > c.nr + c.ng - 1:
            continue
        for l in range(j - 1, j + 3):
            m = -l if l < 0 else (2 * c.nth - l if l > c.nth else l)
            out[m, k + c.ng] += q * O.w3(x1 - k) * O.w3(x2 - l)
    return out


CUBIC_MOVES = MOVES[:6] + [((4.4, 0.6), (4.1, 0.1)), ((5.2, 1.4), (5.9, 0.6)), ((6.0, 11.3), (6.6, 11.98)),
                           ((3.1, 10.2), (3.7, 11.1)), ((2.5, 0.0), (2.5, 0.7))]


@pytest.mark.parametrize("p0,p1", CUBIC_MOVES)
def test_cubic_single_particle_continuity_is_exact(p0, p1):
    """With the cubic shape, near the polar axis included (ghost rows folded:
    J^r A even, J^theta A odd), q (S^{n+1} - S^n) = -dt div(J A) at every
    vertex."""
    c = cfg(shape=3)
    qw = 0.37
    JrA, JtA, Jph = O.deposit_one(c, qw, p0[0], p0[1], p1[0], p1[1], 0.0)
    drho = cubic_density(c, *p1, qw) - cubic_density(c, *p0, qw)
    div = divergence_of_flux(c, JrA, JtA)
    np.testing.assert_allclose(drho, -c.dt * div, rtol=0, atol=2e-15)
    assert np.all(Jph == 0)


def test_cubic_static_particle_radial_motion_and_moments():
    c = cfg(shape=3)
    JrA, JtA, Jph = O.deposit_one(c, 1.0, 4.3, 5.6, 4.3, 5.6, 0.0)
    assert np.all(JrA == 0) and np.all(JtA == 0) and np.all(Jph == 0)
    JrA, JtA, Jph = O.deposit_one(c, 1.0, 4.3, 5.6, 4.9, 5.6, 0.0)
    assert np.all(JtA == 0)
    AD, _ = O.areas(c)
    x0, x1, dphi, q = (4.3, 5.6), (4.8, 5.45), 0.013, -2.0
    JrA, JtA, Jph = O.deposit_one(c, q, *x0, *x1, dphi)
    assert JrA.sum() == pytest.approx(q * (x1[0] - x0[0]) / c.dt, rel=1e-12)
    assert JtA.sum() == pytest.approx(q * (x1[1] - x0[1]) / c.dt, rel=1e-12)
    assert (Jph * AD[2]).sum() == pytest.approx(q * dphi / c.dt, rel=1e-12)


def test_cubic_interpolation_reproduces_linear_fields():
    """The cubic B-spline reproduces linear data exactly (first moment), on
    every staggered lattice, away from the axis and the radial ends."""
    c = cfg(shape=3)
    stag = [(0.5, 0.0), (0.0, 0.5), (0.0, 0.0), (0.0, 0.5), (0.5, 0.0), (0.5, 0.5)]
    coef = [(0.3, 1.1, -0.7), (-2.0, 0.4, 0.9), (1.5, -0.3, 0.2), (0.1, 0.2, 0.3), (-0.6, 0.8, -1.2), (2.2, 0.5, 0.5)]
    F = []
    for (sr, st), (a0, a1, a2) in zip(stag, coef):
        col = np.arange(c.ld) - c.ng + sr
        row = np.arange(c.nth + 1) + st
        F.append(a0 + a1 * col[None, :] + a2 * row[:, None])
    for x1, x2 in [(3.3, 4.6), (2.1, 7.2), (8.9, 2.3), (5.5, 5.5)]:
        v = O.interp(c, F[:3], F[3:], x1, x2)
        ref = [a0 + a1 * x1 + a2 * x2 for (a0, a1, a2) in coef]
        np.testing.assert_allclose(v, ref, rtol=0, atol=1e-13)
    # next to the axis the mirror rows carry the parities: a constant theta
    # component averages to less than the constant, the others keep it
    G = [np.ones(O.field_shape(c)) for _ in range(6)]
    v = O.interp(c, G[:3], G[3:], 4.2, 0.6)
    for k in (0, 2, 3, 5):
        assert v[k] == pytest.approx(1.0, abs=1e-14)
    assert v[1] < 1.0 and v[4] < 1.0


def test_cubic_full_steps_conserve_charge_to_round_off():
    """Sec. 3.4's continuity with the cubic shape: push, deposit (folded at
    the axis), field update and sort keep div D - rho to round-off."""
    c = cfg(n=24, qw=(-0.05, 0.05, 0.05, 0.0), shape=3)
    D, B = O.init_fields(c, O.WALD, 1.0)
    arrs = synth.particles(c.nr, c.nth, c.r_in, c.r_out, 3000, seed=9, sigma=0.6)
    P = O.Particles(*arrs)
    P.th[0], P.u2[0] = 0.3 * c.dth, -3.0 * P.r[0]
    P.th[1], P.u2[1] = math.pi - 0.4 * c.dth, 3.0 * P.r[1]
    D0 = [x.copy() for x in D]
    P0 = P.copy()
    worst = 0.0
    for _ in range(6):
        st, P, J = O.step(c, P, D, B)
        assert st == 0
        res, rmax = _charge_residual(c, D0, P0, D, P)
        worst = max(worst, res / rmax)
    assert worst < 1e-12, worst


def test_sort_matches_stable_argsort():
    rng = np.random.default_rng(11)
    for n, nk in [(1, 5), (1000, 7), (20000, 333), (5000, 1)]:
        keys = rng.integers(0, nk + 1, size=n).astype(np.int32)
        perm, live = O.counting_sort(keys, nk)
        ref = np.argsort(keys, kind="stable")
        np.testing.assert_array_equal(perm, ref)
        assert live == np.sum(keys < nk)


def test_cell_keys_and_sort_drop_dead():
    c = cfg(n=16)
    arrs = synth.particles(c.nr, c.nth, c.r_in, c.r_out, 600, seed=1)
    P = O.Particles(*arrs)
    P.tag[5] |= O.DEAD
    rng = np.random.default_rng(2)
    P = P.take(rng.permutation(P.n))
    keys = O.cell_keys(c, P)
    x1 = np.floor(np.log(P.r / c.r_in) / c.dx1).astype(int)
    x2 = np.minimum(np.floor(P.th / c.dth).astype(int), c.nth - 1)
    dead = (P.tag & O.DEAD) != 0
    np.testing.assert_array_equal(keys[~dead], (x2 * c.nr + x1)[~dead])
    assert np.all(keys[dead] == c.nr * c.nth)
    Q = O.sort(c, P)
    assert Q.n == P.n - 1
    k2 = O.cell_keys(c, Q)
    assert np.all(np.diff(k2) >= 0)


def test_threaded_oracle_matches_one_thread():
    """The multi-threaded run of the CPU baseline computes the same step: the
    particles bit for bit, the currents and fields up to the order of the
    per-thread current sums (which the one-thread parity runs never use)."""
    from paper_2503_04558_gb300 import synth
    a = 0.9
    rin = 0.9 * O.horizon(a)
    c = O.make_cfg(32, 32, a, rin, 20.0)
    P = O.Particles(*synth.particles(32, 32, rin, 20.0, 20000, seed=3, sigma=0.3))
    out = {}
    try:
        for nt in (1, 4):
            O.set_threads(nt)
            D, B = O.init_fields(c, O.WALD, 1.0)
            Q = P.copy()
            st, J, _ = O.push_deposit(c, Q, D, B)
            O.field_update(c, D, B, J)
            out[nt] = (Q, J, D + B)
    finally:
        O.set_threads(1)
    (Q1, J1, F1), (Q4, J4, F4) = out[1], out[4]
    for x, y in ((Q1.r, Q4.r), (Q1.th, Q4.th), (Q1.u1, Q4.u1), (Q1.u2, Q4.u2), (Q1.u3, Q4.u3), (Q1.tag, Q4.tag)):
        assert np.array_equal(x, y)
    for x, y in zip(J1 + F1, J4 + F4):
        assert np.max(np.abs(x - y)) <= 1e-13 * max(np.max(np.abs(x)), 1e-300)
