"""Pins of the oracle's particle pusher (Sec. 2.2, Eqs. particle-eom,
geodesic-predictor/-corrector, boris-plus-minus, u0bar, boris-scheme) and of
the closed-form fields it is driven by in the charged-orbit checks (App. C).

Independent references: Hamilton's equations with the textbook Kerr metric
(tests/kerr_indep.py), the conserved energy, angular momentum and Carter
constant of Kerr geodesics, the printed Table 1 initial data (tests/golden),
the implicit equation the Boris scheme solves (Eq. boris-step), and for the
alternative Vay update in the FIDO frame the implicit equation of Vay's
scheme, its drift property and energy conservation in a pure magnetic
field."""
import math
import os

import numpy as np
import pytest

import oracle as O
import kerr_indep as K

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1_orbits.txt")
T1 = K.load_table1(GOLD)


def state(row):
    return np.array([row["r"], row["th"], 0.0, *row["u"]])


@pytest.mark.parametrize("y,a", [
    ([4.0, 1.2, 0.0, 0.3, -0.5, 1.7], 0.9),
    ([1.4, 0.5, 0.0, -2.0, 0.4, 0.2], 0.99),
    ([12.0, 2.2, 0.0, 0.05, 3.0, -4.0], 0.5),
    ([2.5, 1.5707963, 0.0, 0.1, 0.0, 3.0], 0.0),
])
def test_geodesic_rhs_matches_hamilton_equations(y, a):
    f = O.geodesic_rhs(a, 1.0, y)
    ref = K.hamilton_rhs(a, np.array(y))
    np.testing.assert_allclose(f[[0, 1, 2]], ref[[0, 1, 2]], rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(f[[3, 4]], ref[[3, 4]], rtol=1e-8, atol=1e-10)
    assert f[5] == 0.0


def test_table1_initial_energies_are_the_catalogue_values():
    """The four periodic orbits of Table 1 start at a radial turning point
    (u_r in BL coordinates vanishes to the printed 6 digits) and their energy
    E = -u_t comes out as a round 6-digit catalogue value; both only hold if
    the printed (u_r, u_phi, r) are Kerr-Schild covariant components."""
    for name in ["(2,0,1)", "(3,3,1)", "(3,3,2)", "(4,3,1)"]:
        row = T1[name]
        y = state(row)
        E = K.energy(row["a"], y)
        assert abs(E * 1e6 - round(E * 1e6)) < 1e-2, (name, E)
        r, a = row["r"], row["a"]
        Dl = r * r - 2 * r + a * a
        u_r_bl = y[3] + (2 * r / Dl) * (-E) + (a / Dl) * y[5]
        assert abs(u_r_bl) < 1e-6, (name, u_r_bl)


def _energy_drift(name, dt, T):
    row = T1[name]
    y0 = state(row)
    E0 = K.energy(row["a"], y0)
    n = int(round(T / dt))
    every = max(1, n // 200)
    _, traj = O.push_analytic(0, 0.0, row["a"], 0.0, 1, dt, 3, y0, n, every)
    dE = np.array([abs(K.energy(row["a"], s) - E0) for s in traj])
    return dE.mean(), traj, y0


@pytest.mark.parametrize("name", ["(2,0,1)", "(3,3,2)"])
def test_geodesic_energy_error_is_second_order(name):
    """Sec. 3.1 / Fig. orbits: the period-averaged energy error scales as dt^2."""
    e1, _, _ = _energy_drift(name, 0.02, 200.0)
    e2, _, _ = _energy_drift(name, 0.01, 200.0)
    ratio = e1 / e2
    assert 3.2 < ratio < 4.8, ratio
    assert e2 < 1e-5


def test_geodesic_conserves_u_phi_exactly_and_stays_equatorial():
    _, traj, y0 = _energy_drift("(3,3,1)", 0.01, 100.0)
    assert np.all(traj[:, 5] == y0[5])          # U_phi == 0 (P4)
    assert np.max(np.abs(traj[:, 1] - math.pi / 2)) < 1e-12
    assert np.max(np.abs(traj[:, 4])) < 1e-12


def test_geodesic_carter_constant_converges():
    """An inclined geodesic (RKA8 initial data, no field): Carter's Q drift
    falls at second order in dt."""
    row = T1["RKA8"]
    y0 = state(row)
    a = row["a"]
    Q0 = K.carter_Q(a, y0)
    drifts = []
    for dt in (0.02, 0.01):
        n = int(round(60.0 / dt))
        _, traj = O.push_analytic(0, 0.0, a, 0.0, 1, dt, 3, y0, n, n // 100)
        drifts.append(max(abs(K.carter_Q(a, s) - Q0) for s in traj))
    assert drifts[1] < 1e-4 * abs(Q0)
    assert 3.0 < drifts[0] / drifts[1] < 5.0, drifts


def _boris_residual(a, r, th, qm, dt, Dv, Bv, u):
    """Residual of the implicit Eq. boris-step with u_bar = (u + u')/2 and
    u0_bar from u^- (Eq. u0bar), written with the independent 3+1 metric."""
    alpha, beta, gam, gi = K.three_plus_one(a, r, th)
    sqrtg = math.sqrt(np.linalg.det(gam))
    up = O.boris(a, r, th, qm, dt, Dv, Bv, u)
    Dl = gam @ np.asarray(Dv)
    um = np.asarray(u) + qm * alpha * dt / 2 * Dl
    u0b = math.sqrt(1 + um @ gi @ um) / alpha
    ubar = (np.asarray(u) + up) / 2
    v = gi @ ubar
    B = np.asarray(Bv)
    cross = sqrtg * np.array([v[1] * B[2] - v[2] * B[1], v[2] * B[0] - v[0] * B[2], v[0] * B[1] - v[1] * B[0]])
    res = up - np.asarray(u) - qm * dt * (alpha * Dl + cross / u0b)
    return res, up, gi


@pytest.mark.parametrize("seed", range(6))
def test_boris_solves_the_implicit_equation(seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0, 0.999)
    r = rng.uniform(1.2, 30)
    th = rng.uniform(0.1, 3.0)
    Dv = rng.normal(size=3) * [1, 1 / r, 1 / r]
    Bv = rng.normal(size=3) * [3, 3 / r, 3 / r]
    u = rng.normal(size=3) * [2, 2 * r, 2 * r]
    res, up, _ = _boris_residual(a, r, th, rng.choice([-1.0, 1.0]), 0.05, Dv, Bv, u)
    assert np.max(np.abs(res)) < 1e-13 * max(1.0, np.max(np.abs(up)))


@pytest.mark.parametrize("seed", range(4))
def test_boris_rotation_preserves_norm_without_electric_field(seed):
    rng = np.random.default_rng(100 + seed)
    a, r, th = 0.9, rng.uniform(1.5, 10), rng.uniform(0.2, 2.9)
    Bv = rng.normal(size=3) * [10, 10 / r, 10 / r]
    u = rng.normal(size=3) * [1, r, r]
    up = O.boris(a, r, th, 1.0, 0.1, [0, 0, 0], Bv, u)
    _, _, _, gi = K.three_plus_one(a, r, th)
    n0, n1 = u @ gi @ u, up @ gi @ up
    assert abs(n1 - n0) < 1e-13 * n0


# ---------------------------------------------------------------------------
# the alternative momentum update: Vay's step in the FIDO frame (Sec. 2.2)
# ---------------------------------------------------------------------------
def _vay_residual(a, r, th, qm, dt, Dv, Bv, u):
    """Residual of Vay's implicit equation over the FIDO proper time alpha dt,
    u1 - u = (q/m) alpha dt (E + (u/Gamma + u1/Gamma1)/2 x B), in coordinate
    components with the independent 3+1 metric: E_i = gamma_ij D^j, the
    cross product e_ijk V^j B^k of the raised velocity, Gamma = sqrt(1 +
    gamma^ij u_i u_j)."""
    alpha, beta, gam, gi = K.three_plus_one(a, r, th)
    sqrtg = math.sqrt(np.linalg.det(gam))
    u = np.asarray(u, np.float64)
    u1 = O.vay(a, r, th, qm, dt, Dv, Bv, u)
    G0 = math.sqrt(1 + u @ gi @ u)
    G1 = math.sqrt(1 + u1 @ gi @ u1)
    v = gi @ (u / G0 + u1 / G1) / 2
    B = np.asarray(Bv)
    cross = sqrtg * np.array([v[1] * B[2] - v[2] * B[1], v[2] * B[0] - v[0] * B[2], v[0] * B[1] - v[1] * B[0]])
    res = u1 - u - qm * alpha * dt * (gam @ np.asarray(Dv) + cross)
    return res, u1, gi


@pytest.mark.parametrize("seed", range(6))
def test_vay_solves_its_implicit_equation(seed):
    rng = np.random.default_rng(300 + seed)
    a = rng.uniform(0, 0.999)
    r = rng.uniform(1.2, 30)
    th = rng.uniform(0.1, 3.0)
    Dv = rng.normal(size=3) * [1, 1 / r, 1 / r]
    Bv = rng.normal(size=3) * [3, 3 / r, 3 / r]
    u = rng.normal(size=3) * [2, 2 * r, 2 * r]
    res, u1, _ = _vay_residual(a, r, th, rng.choice([-1.0, 1.0]), 0.05, Dv, Bv, u)
    assert np.max(np.abs(res)) < 1e-12 * max(1.0, np.max(np.abs(u1)))


@pytest.mark.parametrize("seed", range(4))
def test_vay_preserves_norm_without_electric_field(seed):
    rng = np.random.default_rng(400 + seed)
    a, r, th = 0.9, rng.uniform(1.5, 10), rng.uniform(0.2, 2.9)
    Bv = rng.normal(size=3) * [10, 10 / r, 10 / r]
    u = rng.normal(size=3) * [1, r, r]
    u1 = O.vay(a, r, th, 1.0, 0.1, [0, 0, 0], Bv, u)
    _, _, _, gi = K.three_plus_one(a, r, th)
    n0, n1 = u @ gi @ u, u1 @ gi @ u1
    assert abs(n1 - n0) < 1e-12 * n0


def test_vay_pure_electric_kick_is_exact():
    a, r, th = 0.7, 3.3, 1.1
    alpha, _, gam, _ = K.three_plus_one(a, r, th)
    Dv = np.array([0.4, -0.07, 0.02])
    u = np.array([0.3, -1.2, 2.5])
    u1 = O.vay(a, r, th, -1.0, 0.2, Dv, [0, 0, 0], u)
    np.testing.assert_allclose(u1, u - alpha * 0.2 * (gam @ Dv), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_vay_leaves_the_drift_momentum_unchanged(seed):
    """Vay's defining property: a particle whose velocity cancels the
    electric field (E + v x B = 0, any Lorentz factor) is not accelerated.
    The field D is built from u and B with the independent metric."""
    rng = np.random.default_rng(500 + seed)
    a, r, th = rng.uniform(0, 0.99), rng.uniform(1.5, 20), rng.uniform(0.3, 2.8)
    _, _, gam, gi = K.three_plus_one(a, r, th)
    sqrtg = math.sqrt(np.linalg.det(gam))
    Bv = rng.normal(size=3) * [5, 5 / r, 5 / r]
    # a momentum perpendicular to B (frame dot product u_i B^i = 0), Gamma ~ 10^2
    u = rng.normal(size=3) * [1, r, r]
    u = u - (u @ Bv) / (Bv @ gam @ Bv) * (gam @ Bv)
    u *= 100.0 / math.sqrt(u @ gi @ u)
    G = math.sqrt(1 + u @ gi @ u)
    v = gi @ u / G
    vxB = sqrtg * np.array([v[1] * Bv[2] - v[2] * Bv[1], v[2] * Bv[0] - v[0] * Bv[2], v[0] * Bv[1] - v[1] * Bv[0]])
    Dv = -gi @ vxB   # E_i = gamma_ij D^j = -(v x B)_i
    u1 = O.vay(a, r, th, 1.0, 0.05, Dv, Bv, u)
    dv = np.max(np.abs(u1 - u))
    assert dv < 1e-11 * np.max(np.abs(u))
    # the generalized Boris step does not keep it (it averages u^- and u^+
    # with the Lorentz factor of u^-)
    db = np.max(np.abs(O.boris(a, r, th, 1.0, 0.05, Dv, Bv, u) - u))
    assert db > 1e2 * max(dv, 1e-16 * np.max(np.abs(u)))


def test_vay_and_boris_differ_at_third_order():
    """Both steps are second-order accurate for the same force, so one step
    of each differs by O(dt^3)."""
    rng = np.random.default_rng(7)
    a, r, th = 0.9, 4.0, 1.0
    Dv = rng.normal(size=3) * [1, 0.25, 0.25]
    Bv = rng.normal(size=3) * [3, 0.75, 0.75]
    u = rng.normal(size=3) * [1, 4, 4]
    diffs = []
    for dt in (0.04, 0.02, 0.01):
        diffs.append(np.max(np.abs(O.vay(a, r, th, 1.0, dt, Dv, Bv, u) - O.boris(a, r, th, 1.0, dt, Dv, Bv, u))))
    assert 6.0 < diffs[0] / diffs[1] < 10.0 and 6.0 < diffs[1] / diffs[2] < 10.0, diffs


# ---------------------------------------------------------------------------
# closed-form fields (App. C) against derivatives of their potentials
# ---------------------------------------------------------------------------
def _d(f, x, h):
    return (-f(x + 2 * h) + 8 * f(x + h) - 8 * f(x - h) + f(x - 2 * h)) / (12 * h)


@pytest.mark.parametrize("kind", [O.WALD, O.WALD_A0, O.MONOPOLE, O.SPLIT_MONOPOLE])
@pytest.mark.parametrize("r,th", [(1.6, 0.6), (3.0, 1.2), (9.0, 2.4)])
def test_closed_fields_are_derivatives_of_potentials(kind, r, th):
    a, B0 = 0.9, 1.7
    F = O.closed_fields(kind, a, B0, r, th)
    Aph = lambda rr, tt: O.closed_fields(kind, a, B0, rr, tt)["Aph"]
    At = lambda rr, tt: O.closed_fields(kind, a, B0, rr, tt)["At"]
    h = 1e-4
    # B^r = (1/sqrt(gamma)) d_theta A_phi, B^theta = -(1/sqrt(gamma)) d_r A_phi
    assert F["sgB"][0] == pytest.approx(_d(lambda t: Aph(r, t), th, h), rel=1e-8, abs=1e-10)
    assert F["sgB"][1] == pytest.approx(-_d(lambda x: Aph(x, th), r, h), rel=1e-8, abs=1e-10)
    # E_i = d_i A_t (Phi = -A_0, E = -grad Phi)
    assert F["E"][0] == pytest.approx(_d(lambda x: At(x, th), r, h), rel=1e-8, abs=1e-10)
    assert F["E"][1] == pytest.approx(_d(lambda t: At(r, t), th, h), rel=1e-8, abs=1e-10)
    # B^phi = -(1/sqrt(gamma)) d_theta A_r with the Kerr-Schild A_r obtained from
    # the Boyer-Lindquist potential by the transform of Eq. BL_KS_diff:
    # A_r^KS = -(2 r A_t + a A_phi) / Delta  (monopole: printed A_r = A_t)
    if kind in (O.WALD,):
        def Ar(t):
            Dl = r * r - 2 * r + a * a
            return -(2 * r * At(r, t) + a * Aph(r, t)) / Dl
    elif kind in (O.MONOPOLE, O.SPLIT_MONOPOLE):
        def Ar(t):
            return At(r, t)
    else:
        def Ar(t):
            return 0.0
    assert F["sgB"][2] == pytest.approx(-_d(Ar, th, h), rel=1e-7, abs=1e-9)


def test_charged_orbit_conserves_canonical_energy_and_momentum():
    """RKA3 of Table 1 in the analytic rotating Wald field (Sec. 3.1): the
    canonical E = -u_t - (q/m) A_t (Eq. ptc_energy) and L = u_phi + (q/m) A_phi
    are conserved, with drift falling at second order in dt.

    With the two half Boris steps bundled into one full step at the start of
    each step (Sec. 2.2), the stored u^n lies half a Boris kick before the
    momentum of the Strang-split scheme at x^n; the conserved quantities are
    measured on that synchronized momentum (a half Boris step applied here)."""
    row = T1["RKA3"]
    a, B0 = row["a"], row["Bz"]
    y0 = state(row)
    qm = 1.0

    def canon(y):
        F = O.closed_fields(O.WALD, a, B0, y[0], y[1])
        return K.energy(a, y) - qm * F["At"], y[5] + qm * F["Aph"]

    def sync(y, dt):
        F = O.closed_fields(O.WALD, a, B0, y[0], y[1])
        z = y.copy()
        z[3:6] = O.boris(a, y[0], y[1], qm, dt / 2, F["D"], F["B"], y[3:6])
        return z

    errs = []
    for dt in (0.004, 0.002):
        E0, L0 = canon(sync(y0, dt))
        n = int(round(40.0 / dt))
        _, traj = O.push_analytic(O.WALD, B0, a, qm, 1, dt, 3, y0, n, n // 100)
        eE = max(abs(canon(sync(s, dt))[0] - E0) for s in traj)
        eL = max(abs(canon(sync(s, dt))[1] - L0) for s in traj)
        errs.append((eE, eL))
    assert errs[1][0] < 1e-6 * abs(E0) and errs[1][1] < 1e-5 * abs(L0)
    assert 3.5 < errs[0][0] / errs[1][0] < 4.5, errs
    assert 3.5 < errs[0][1] / errs[1][1] < 4.5, errs
