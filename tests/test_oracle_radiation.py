"""Pins of the oracle's 2D radiation and injection (Sec. 4's emission and
conversion prescription on the 2D grid; the pair injection of the
plasma-filled Wald run, Sec. 3.4).

Independent references: FIDO energy bookkeeping with the textbook 3+1 metric
(tests/kerr_indep.py), directions of the children, the binomial statistics
of the conversion probability 1 - exp(-tau dt), charge neutrality of pair
creation, and the cell and rest frame of injected pairs."""
import math

import numpy as np
import pytest

import oracle as O
import kerr_indep as K
from paper_2503_04558_gb300 import synth

A = 0.99


def cfg(**kw):
    base = dict(qw=(-0.05, 0.05, 0.05, 0.0), radiation=1, gamma_thr=20.0, eps_ph=4.0, tau=2.0, seed=11)
    base.update(kw)
    return O.make_cfg(24, 24, A, 0.9 * O.horizon(A), 20.0, **base)


def fido(a, r, th, u):
    _, _, _, gi = K.three_plus_one(a, r, th)
    return math.sqrt(np.asarray(u) @ gi @ np.asarray(u))


def one(r, th, u, tag):
    return O.Particles(np.array([r]), np.array([th]), np.array([u[0]]), np.array([u[1]]), np.array([u[2]]),
                       np.array([tag], np.uint32))


def test_emission_conserves_fido_energy_along_the_momentum():
    c = cfg()
    r, th, u = 3.1, 1.2, np.array([25.0, -40.0, 60.0])
    G0 = math.sqrt(1 + fido(A, r, th, u) ** 2)
    st, Q, (ne, nc) = O.radiate(c, one(r, th, u, 1), 0)
    assert st == 0 and (ne, nc) == (1, 0) and Q.n == 2
    ue = np.array([Q.u1[0], Q.u2[0], Q.u3[0]])
    k = np.array([Q.u1[1], Q.u2[1], Q.u3[1]])
    G1 = math.sqrt(1 + fido(A, r, th, ue) ** 2)
    assert G1 + c.eps_ph == pytest.approx(G0, rel=1e-14)
    assert fido(A, r, th, k) == pytest.approx(c.eps_ph, rel=1e-14)
    assert np.allclose(np.cross(ue, k), 0, atol=1e-12 * np.linalg.norm(ue) * np.linalg.norm(k))
    assert np.dot(ue, k) > 0 and Q.tag[1] == 3 and Q.r[1] == r and Q.th[1] == th
    # below the threshold nothing happens
    st, Q, ev = O.radiate(c, one(r, th, u / 10, 1), 0)
    assert ev == (0, 0) and Q.n == 1


def test_conversion_splits_the_photon_energy():
    c = cfg(tau=1e9)   # P = 1 - exp(-tau dt) = 1
    r, th, k = 4.0, 0.7, np.array([3.0, 20.0, -15.0])
    e = fido(A, r, th, k)
    st, Q, (ne, nc) = O.radiate(c, one(r, th, k, 3), 5)
    assert (ne, nc) == (0, 1) and Q.n == 3 and (Q.tag[0] & O.DEAD)
    assert list(Q.tag[1:]) == [0, 1]
    for m in (1, 2):
        um = np.array([Q.u1[m], Q.u2[m], Q.u3[m]])
        assert math.sqrt(1 + fido(A, r, th, um) ** 2) == pytest.approx(e / 2, rel=1e-14)
        assert np.allclose(np.cross(um, k), 0, atol=1e-12 * np.linalg.norm(um) * np.linalg.norm(k))
    # a photon below 2 m c^2 never converts
    st, Q, ev = O.radiate(c, one(r, th, k * 1.5 / e, 3), 5)
    assert ev == (0, 0)


def test_conversion_probability_is_one_minus_exp_minus_tau_dt():
    c = cfg(tau=30.0)
    n = 40000
    P = O.Particles(np.full(n, 5.0), np.full(n, 1.0), np.full(n, 30.0), np.zeros(n), np.zeros(n),
                    np.full(n, 3, np.uint32))
    p = 1 - math.exp(-c.tau * c.dt)
    for step in (0, 1):
        st, Q, (ne, nc) = O.radiate(c, P.copy(), step)
        sd = math.sqrt(n * p * (1 - p))
        assert abs(nc - n * p) < 5 * sd, (nc, n * p)
    # keyed on (slot, step): the same step decides the same, another differs
    a = O.radiate(c, P.copy(), 3)[1].tag
    b = O.radiate(c, P.copy(), 3)[1].tag
    d = O.radiate(c, P.copy(), 4)[1].tag
    assert np.array_equal(a, b) and not np.array_equal(a[:n], d[:n])


def test_injection_where_field_aligned_electric_field_and_magnetisation_allow():
    c = cfg(radiation=0, injection=1, sigma_thr=1.0, eps_db=1e-3)
    D, B = O.init_fields(c, O.WALD, 5.0)   # the rotating Wald field has D.B != 0
    P = O.Particles(*synth.particles(c.nr, c.nth, c.r_in, c.r_out, 200, seed=2, sigma=0.1))
    st, Q, ncells = O.inject(c, P.copy(), D, B, 0)
    assert st == 0 and ncells > 0 and Q.n == P.n + 2 * ncells
    new = slice(P.n, Q.n)
    assert np.all(Q.u1[new] == 0) and np.all(Q.u2[new] == 0) and np.all(Q.u3[new] == 0)
    assert list(Q.tag[new][:2]) == [0, 1]
    # each pair shares one point: the charge density does not change
    assert np.array_equal(Q.r[new][0::2], Q.r[new][1::2]) and np.array_equal(Q.th[new][0::2], Q.th[new][1::2])
    np.testing.assert_allclose(O.rho(c, Q), O.rho(c, P), rtol=0, atol=1e-15 * np.abs(O.rho(c, P)).max())
    # no field-aligned electric field (a = 0 Wald: D = 0) -> no injection
    c0 = cfg(radiation=0, injection=1, sigma_thr=1.0, eps_db=1e-3)
    D0 = [np.zeros_like(x) for x in D]
    assert O.inject(c0, P.copy(), D0, B, 0)[2] == 0
    # a magnetisation threshold above every cell -> no injection
    ch = cfg(radiation=0, injection=1, sigma_thr=1e30, eps_db=1e-3)
    assert O.inject(ch, P.copy(), D, B, 0)[2] == 0
    # the injected points lie inside their cells, uniform within
    x1 = (np.log(Q.r[new][0::2]) - math.log(c.r_in)) / c.dx1
    x2 = Q.th[new][0::2] / c.dth
    f1, f2 = x1 - np.floor(x1), x2 - np.floor(x2)
    assert 0.3 < f1.mean() < 0.7 and 0.3 < f2.mean() < 0.7


def test_cascade_steps_conserve_charge():
    c = cfg(injection=1, sigma_thr=1.0, eps_db=1e-3, tau=200.0)
    D, B = O.init_fields(c, O.WALD, 5.0)
    P = O.Particles(*synth.particles(c.nr, c.nth, c.r_in, c.r_out, 2000, seed=3, sigma=0.3))
    P.u1[:40] = 60.0
    D0 = [x.copy() for x in D]
    P0 = P.copy()
    ev = []
    for s in range(4):
        st, P, J = O.step(c, P, D, B, step=s, events=ev)
        assert st == 0
    assert sum(e[0] for e in ev) > 0 and sum(e[1] for e in ev) > 0 and sum(e[2] for e in ev) > 0
    r0 = O.divD(c, D0) - O.rho(c, P0)
    r1 = O.divD(c, D) - O.rho(c, P)
    last = c.nr - c.damp_cells - 1
    sl = (slice(0, c.nth + 1), slice(c.ng + 1, c.ng + last + 1))
    res = np.max(np.abs(r1 - r0)[sl]) / np.max(np.abs(O.rho(c, P)[sl]))
    assert res < 1e-12, res
