"""Pins of the oracle's batched 1D spark-gap line model: the radiative pair
production prescription of Sec. 4 (threshold emission at gamma_thr with FIDO
energy eps_ph, conversion with probability 1 - exp(-tau dt), Eq.
optical-depth) on radial lines, its counter-based RNG and its deposit.

Independent references: numpy's Philox4x64-10 bit generator (the same
published algorithm, Salmon et al. SC'11), statistics of the uniform draws,
the discrete 1D continuity equation with a CIC shape of the test's own, FIDO
energies from the textbook Kerr metric (tests/kerr_indep.py), and the
conservation of E = -u_t for the theta-frozen motion (a reduced Hamiltonian
system: H = g^{mu nu} u_mu u_nu / 2 with u_theta = 0 does not depend on t)."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
import kerr_indep as K

A = 0.99
RH = 1.0 + math.sqrt(1 - A * A)


@pytest.mark.parametrize("seed", range(5))
def test_philox_matches_numpy(seed):
    rng = np.random.default_rng(seed)
    key = rng.integers(0, 2**63, size=2, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    ctr = rng.integers(1, 2**63, size=4, dtype=np.uint64)
    # numpy's Philox advances its counter by one before producing a block
    prev = ctr.copy()
    prev[0] -= np.uint64(1)
    ref = np.random.Philox(key=key, counter=prev).random_raw(4)
    np.testing.assert_array_equal(O.philox4x64(ctr, key), ref)


def test_philox_counter_carry_matches_numpy():
    key = np.array([7, 11], np.uint64)
    prev = np.array([2**64 - 1, 5, 0, 0], np.uint64)
    ref = np.random.Philox(key=key, counter=prev).random_raw(4)
    np.testing.assert_array_equal(O.philox4x64(np.array([0, 6, 0, 0], np.uint64), key), ref)


def test_uniform_draws_are_uniform_and_independent():
    u = np.array([O.uniform(42, pid, 3, 1) for pid in range(20000)])
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    v = np.array([O.uniform(42, pid, 4, 1) for pid in range(20000)])
    assert abs(np.corrcoef(u, v)[0, 1]) < 0.03
    assert np.all((u >= 0) & (u < 1))


def test_child_ids_are_distinct():
    ids = {O.child_id(p, s, k) for p in range(2000) for s in range(20) for k in range(3)}
    assert len(ids) == 2000 * 20 * 3


def cic(n, x, q):
    out = np.zeros(n + 1)
    i = int(math.floor(x))
    for k in (i, i + 1):
        if 0 <= k <= n:
            out[k] += q * max(0.0, 1 - abs(x - k))
    return out


def test_line_deposit_and_field_conserve_charge():
    """Delta[(D A)_i - (D A)_{i-1}] = sum q (S^{n+1} - S^n) at every interior
    vertex i (the imposed current I_0 cancels: it is constant along the line)."""
    L = O.make_line(64, A, 0.7, RH, 20.0, I0=3.0, gamma_thr=1e30)
    Ar = O.line_area(L)
    D = O.line_init_D(L, 50.0)
    rng = np.random.default_rng(1)
    n = 400
    x = rng.random(n) * 60 + 2
    S = O.LineState(x, rng.normal(size=n) * 2, rng.normal(size=n) * 0.5, rng.integers(0, 2, n).astype(np.uint32),
                    np.arange(n, dtype=np.uint64), 4 * n)
    x0 = S.view()["x1"].copy()
    q0 = np.where(S.view()["tag"] == 0, L.qw[0], L.qw[1])
    DA0 = D * Ar
    st, JA, c = O.line_step(L, 0, S, D)
    assert st == 0 and S.n == n   # nobody left the line in one step
    x1 = S.view()["x1"]
    dq = np.zeros(L.n + 1)
    for k in range(n):
        dq += cic(L.n, x1[k], q0[k]) - cic(L.n, x0[k], q0[k])
    DA1 = D * Ar
    ddiv = (DA1[1:] - DA1[:-1]) - (DA0[1:] - DA0[:-1])   # vertices 1..n-1
    np.testing.assert_allclose(ddiv, dq[1:L.n], rtol=0, atol=1e-12 * max(1.0, np.abs(DA0).max()))


def fido_energy(L, x1, ur, up, eps):
    r = L.r_in * math.exp(x1 * L.dx1)
    _, _, _, gi = K.three_plus_one(L.a, r, L.theta)
    u = np.array([ur, 0.0, up])
    return math.sqrt(eps + u @ gi @ u)


def test_emission_takes_eps_ph_of_fido_energy():
    L = O.make_line(128, A, 0.5, RH, 20.0, gamma_thr=50.0, eps_ph=4.0)
    D = np.zeros(L.n)
    x, ur, up = 60.3, 400.0, 3.0
    ref = O.LineState([x], [ur], [up], [1], [9], 8)
    L_no = O.make_line(128, A, 0.5, RH, 20.0, gamma_thr=1e30)
    O.line_step(L_no, 0, ref, D.copy())
    G_before = fido_energy(L, ref.x1[0], ref.ur[0], ref.up[0], 1.0)
    S = O.LineState([x], [ur], [up], [1], [9], 8)
    st, JA, c = O.line_step(L, 0, S, D.copy())
    assert st == 0 and c[0] == 1 and S.n == 2
    v = S.view()
    assert v["tag"][1] == 3 and v["id"][1] == O.child_id(9, 0, 0)
    assert fido_energy(L, v["x1"][0], v["ur"][0], v["up"][0], 1.0) == pytest.approx(G_before - 4.0, rel=1e-12)
    assert fido_energy(L, v["x1"][1], v["ur"][1], v["up"][1], 0.0) == pytest.approx(4.0, rel=1e-12)
    # photon along the emitter's momentum
    assert v["ur"][1] / v["up"][1] == pytest.approx(v["ur"][0] / v["up"][0], rel=1e-12)


def test_conversion_rate_energy_and_order():
    L = O.make_line(128, A, 0.8, RH, 20.0, tau=20.0, seed=77)
    D = np.zeros(L.n)
    n = 20000
    rng = np.random.default_rng(3)
    x = rng.random(n) * 100 + 10
    kr = np.where(rng.random(n) < 0.5, 1.0, -1.0) * 6.0
    S = O.LineState(x, kr, np.zeros(n), np.full(n, 3, np.uint32), np.arange(n, dtype=np.uint64) * 7 + 1, 4 * n)
    st, JA, c = O.line_step(L, 5, S, D)
    assert st == 0
    P = 1 - math.exp(-L.tau * L.dt)
    k = c[1]
    assert abs(k - n * P) < 5 * math.sqrt(n * P * (1 - P))
    v = S.view()
    photons = v["tag"] == 3
    assert photons.sum() == n - k and S.n == n + k
    assert np.all(photons[: n - k]) and not np.any(photons[n - k:])   # survivors first, then pairs
    kids = slice(n - k, S.n)
    assert np.array_equal(v["tag"][kids], np.tile([0, 1], k).astype(np.uint32))
    # each pair member carries half of the converted photon's FIDO energy
    e_kid = np.array([fido_energy(L, a, b, cc, 1.0) for a, b, cc in zip(v["x1"][kids], v["ur"][kids], v["up"][kids])])
    assert np.all(np.abs(e_kid - e_kid[::2].repeat(2)) < 1e-12 * e_kid)   # both members alike
    # the photon momentum along the members' direction with FIDO energy 2 Gamma_kid
    # reproduces a photon of energy 2 Gamma_kid: members carry half of it each
    for a, b, g in zip(v["x1"][kids][::2], v["ur"][kids][::2], e_kid[::2]):
        scale = 2.0 * g / math.sqrt(g * g - 1.0)
        assert fido_energy(L, a, b * scale, 0.0, 0.0) == pytest.approx(2.0 * g, rel=1e-12)
        assert 2.0 * g > 2.0


def test_frozen_theta_geodesic_conserves_energy_to_second_order():
    errs = []
    for dt in (0.02, 0.01):
        L = O.make_line(256, A, 0.9, RH, 60.0, dt=dt, qm=(0, 0, 0, 0), qw=(0, 0, 0, 0), gamma_thr=1e30)
        D = np.zeros(L.n)
        S = O.LineState([150.0], [0.3], [2.5], [1], [1], 4)
        E0 = None
        drift = 0.0
        for s in range(int(round(20.0 / dt))):
            v = S.view()
            r = L.r_in * math.exp(v["x1"][0] * L.dx1)
            E = -K.u_t(L.a, r, L.theta, [v["ur"][0], 0.0, v["up"][0]])
            E0 = E if E0 is None else E0
            drift = max(drift, abs(E - E0))
            O.line_step(L, s, S, D)
            assert S.n == 1
        errs.append(drift)
    assert errs[1] < 1e-4
    assert 3.0 < errs[0] / errs[1] < 5.0, errs
