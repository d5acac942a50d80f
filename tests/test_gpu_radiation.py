"""GPU parity of the 2D radiation (photon emission and pair conversion, the
prescription of Sec. 4 on the 2D grid) and of the pair injection of the
plasma-filled Wald run (Sec. 3.4), FP64 path, against the oracle on the same
seeded inputs: event counts and the order of the particles bit-exact (the
appends follow the parent order, the random numbers are keyed on the slot or
cell and the step), values to 1e-10, charge conserved to round-off."""
import math

import numpy as np
import pytest

import oracle as O
from gpu_common import configs, relerr, axis_grazers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

A99 = 0.99
RH = 1.0 + math.sqrt(1 - A99 * A99)


@pytest.fixture(scope="module")
def G():
    from paper_2503_04558_gb300 import build, grpic
    build.build()
    grpic.load()
    return grpic


def host(t):
    return t.detach().cpu().numpy()


def setup(G, n, pseed, B0, cap_factor=4, **kw):
    from paper_2503_04558_gb300 import synth
    oc, gc = configs(32, 32, A99, 0.9 * RH, 20.0, qw=(-0.02, 0.02, 0.02, 0.0), **kw)
    for k in ("radiation", "injection", "gamma_thr", "eps_ph", "tau", "sigma_thr", "eps_db", "seed"):
        setattr(gc, k, getattr(oc, k))
    ctx = G.Context(gc)
    F = G.Fields(gc)
    ctx.init_fields(F, O.WALD, B0)
    D, B = O.init_fields(oc, O.WALD, B0)
    P = O.Particles(*synth.particles(oc.nr, oc.nth, oc.r_in, oc.r_out, n, seed=pseed, sigma=0.3))
    P.u1[: n // 50] = 40.0 * P.r[: n // 50] / P.r[: n // 50]   # some energetic particles
    graze = axis_grazers(oc, P, D, B, 4)
    P = P.take(np.setdiff1d(np.arange(P.n), graze))
    S = G.ParticleSet(gc, cap_factor * P.n)
    S.load(P.r, P.th, P.u1, P.u2, P.u3, P.tag)
    return oc, gc, ctx, F, D, B, P, S


def compare(h, P, F, D, B):
    assert len(h["tag"]) == P.n
    assert np.array_equal(h["tag"], P.tag)
    for k, ref in zip(("x1", "x2", "u1", "u2", "u3"), (P.r, P.th, P.u1, P.u2, P.u3)):
        assert relerr(h[k], ref) < 1e-10, k
    for k in range(3):
        assert relerr(host(F.D[k]), D[k]) < 1e-10, ("D", k)
        assert relerr(host(F.B[k]), B[k]) < 1e-10, ("B", k)


def test_radiation_steps_match_oracle(G):
    """Four steps with emission (gamma_thr 20, eps_ph 4) and conversion
    (tau 200): the same photons, pairs and order as the oracle."""
    oc, gc, ctx, F, D, B, P, S = setup(G, 3000, 5, 2.0, radiation=1, gamma_thr=20.0, eps_ph=4.0, tau=200.0, seed=9)
    ev = []
    for s in range(4):
        st, P, _ = O.step(oc, P, D, B, step=s, events=ev)
        assert st == 0
    ctx.step(S, F, 4)
    assert ctx.sync() == 0
    print("oracle events per step (emitted, converted, injecting cells):", ev)
    assert sum(e[0] for e in ev) > 0 and sum(e[1] for e in ev) > 0
    assert S.live() == P.n
    compare(S.host(), P, F, D, B)


def test_radiation_and_injection_steps_match_oracle_and_conserve_charge(G):
    """Three steps with emission, conversion and injection (sigma_thr 1,
    eps_db 1e-3, rotating Wald B0 = 5): event counts, order and values as the
    oracle; the running charge check stays at round-off."""
    oc, gc, ctx, F, D, B, P, S = setup(G, 3000, 6, 5.0, radiation=1, injection=1, gamma_thr=20.0, eps_ph=4.0,
                                       tau=200.0, sigma_thr=1.0, eps_db=1e-3, seed=4)
    _, _, state0 = ctx.charge_check(S, F, want_state=True)
    ev = []
    for s in range(3):
        st, P, _ = O.step(oc, P, D, B, step=s, events=ev)
        assert st == 0
    ctx.step(S, F, 3)
    assert ctx.sync() == 0
    print("oracle events per step (emitted, converted, injecting cells):", ev)
    assert sum(e[2] for e in ev) > 0
    assert S.live() == P.n
    compare(S.host(), P, F, D, B)
    res, rmax, _ = ctx.charge_check(S, F, base=state0)
    assert res < 1e-12 * rmax, (res, rmax)


def test_capacity_overflow_is_reported(G):
    oc, gc, ctx, F, D, B, P, S = setup(G, 2000, 7, 5.0, cap_factor=1, injection=1, sigma_thr=1.0, eps_db=1e-3,
                                       seed=2)
    ctx.step(S, F, 1)
    assert ctx.sync() == G.EOVERFLOW
    assert S.live() <= S.a.capacity


def test_radiation_refused_where_not_built(G):
    from paper_2503_04558_gb300 import grpic as GG
    with pytest.raises(GG.GrpicError):
        GG.Context(GG.Config(16, 16, 0.9, 1.3, 20.0, precision=32, radiation=1))
