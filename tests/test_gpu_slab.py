"""theta-slab decomposition on the GPU: three slabs, each with its own
context, whole-grid fields and the particles of its rows, run one after
another in one process (messages routed in memory: no kernel waits for
another slab), through the library's decomposition entry points
(grpic_field_update_rows, grpic_halo_pack/unpack, grpic_sort_split,
grpic_particles_pack, grpic_slab_assemble).

  * FP64: after the steps the slabs' particles, concatenated in slab order,
    are the undivided oracle run's particles in the same order (cells and
    tags bit for bit, positions and momenta to 1e-10) and each slab's own
    field rows match the oracle's fields to 1e-10, on the inputs without the
    axis-grazing particles (gpu_common.axis_grazers);
  * FP32 form: the slabs against the undivided FP32 run of the library
    (fields to 1e-5 of their maximum, cells the same for at least 99.9 % of
    the particles: the two add the same currents in different orders)."""
import math

import numpy as np
import pytest

import oracle as O
from gpu_common import configs, relerr, axis_grazers, fp32_offsets

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

A = 0.9
RH = 1.0 + math.sqrt(1 - A * A)
N = 48
NSTEPS = 6
NSLAB = 3


@pytest.fixture(scope="module")
def G():
    from paper_2503_04558_gb300 import build, grpic
    build.build()
    grpic.load()
    return grpic


def case(n=20000, seed=5, precision=64):
    from paper_2503_04558_gb300 import synth
    oc, gc = configs(N, N, A, 0.9 * RH, 20.0, precision=precision)
    if precision == 32:
        gc.fp64_radius = 1.5 * RH
        gc.push_tol = 1e-6
    D, B = O.init_fields(oc, O.WALD, 1.0)
    P = O.Particles(*synth.particles(N, N, oc.r_in, oc.r_out, n, seed=seed, sigma=0.2))
    P = P.take(np.setdiff1d(np.arange(P.n), axis_grazers(oc, P, D, B, NSTEPS)))
    P = O.sort(oc, P)
    return oc, gc, D, B, P


def fp32_state(oc, P):
    cell, o1, o2 = fp32_offsets(oc, P.r, P.th)
    return (o1, o2, P.u1.astype(np.float32), P.u2.astype(np.float32), P.u3.astype(np.float32), P.tag, cell)


def make_slabs(G, oc, gc, P):
    from paper_2503_04558_gb300 import slab as SL
    from slab_oracle import split_sorted
    rows = SL.partition(oc.nth, NSLAB)
    parts = split_sorted(oc, P, rows)
    engines = {}
    for s in range(NSLAB):
        ctx = G.Context(gc)
        F = G.Fields(gc)
        ctx.init_fields(F, O.WALD, 1.0)
        S = G.ParticleSet(gc, P.n + 64)
        Q = parts[s]
        if gc.precision == 64:
            S.load(Q.r, Q.th, Q.u1, Q.u2, Q.u3, Q.tag)
        else:
            S.load(*fp32_state(oc, Q))
        engines[s] = SL.LibrarySlab(ctx, S, F)
    run = SL.SlabRun(engines, NSLAB, oc.nth, oc.n_fld_iter, SL.LocalLinks())
    return run, engines


def test_fp64_slabs_match_the_undivided_oracle_run(G):
    oc, gc, D, B, P = case()
    run, engines = make_slabs(G, oc, gc, P)
    n0 = [e.S.live() for e in engines.values()]
    for _ in range(NSTEPS):
        run.step()
    for e in engines.values():
        assert e.ctx.sync() == 0
    Pu, Du, Bu = P.copy(), [x.copy() for x in D], [x.copy() for x in B]
    for _ in range(NSTEPS):
        _, Pu, _ = O.step(oc, Pu, Du, Bu)
    hs = [e.S.host() for e in engines.values()]
    assert [e.S.live() for e in engines.values()] != n0   # particles crossed the slab edges
    got = {k: np.concatenate([h[k] for h in hs]) for k in ("x1", "x2", "u1", "u2", "u3", "tag")}
    assert len(got["x1"]) == Pu.n
    assert np.array_equal(got["tag"], Pu.tag)
    Pg = O.Particles(got["x1"], got["x2"], got["u1"], got["u2"], got["u3"], got["tag"])
    assert np.array_equal(O.cell_keys(oc, Pg), O.cell_keys(oc, Pu))
    for k, ref in (("x1", Pu.r), ("x2", Pu.th), ("u1", Pu.u1), ("u2", Pu.u2), ("u3", Pu.u3)):
        assert relerr(got[k], ref) < 1e-10, k
    for s, e in engines.items():
        j0, j1 = run.rows[s]
        for x, y in zip(e.F.D + e.F.B, Du + Bu):
            assert relerr(x.cpu().numpy()[j0:j1], y[j0:j1], floor=np.max(np.abs(y))) < 1e-10, s


def test_fp32_slabs_match_the_undivided_fp32_run(G):
    oc, gc, D, B, P = case(precision=32)
    run, engines = make_slabs(G, oc, gc, P)
    ctx = G.Context(gc)
    F = G.Fields(gc)
    ctx.init_fields(F, O.WALD, 1.0)
    S = G.ParticleSet(gc, P.n + 64)
    S.load(*fp32_state(oc, P))
    for _ in range(NSTEPS):
        run.step()
        ctx.push(S, F)
        ctx.field_update(F)
        ctx.sort(S)
    assert ctx.sync() == 0
    for e in engines.values():
        assert e.ctx.sync() == 0
    h = S.host()
    hs = [e.S.host() for e in engines.values()]
    cells = np.concatenate([x["cell"] for x in hs])
    assert abs(len(cells) - len(h["cell"])) <= 2
    m = min(len(cells), len(h["cell"]))
    assert np.mean(cells[:m] == h["cell"][:m]) >= 0.999
    for s, e in engines.items():
        j0, j1 = run.rows[s]
        for x, y in zip(e.F.D + e.F.B, F.D + F.B):
            ref = y.cpu().numpy().astype(np.float64)
            assert relerr(x.cpu().numpy()[j0:j1], ref[j0:j1], floor=np.max(np.abs(ref))) < 1e-5, s
