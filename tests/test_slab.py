"""theta-slab decomposition (the paper's multi-GPU domain decomposition,
Sec. 1) on the host: the partition, and the decomposed step driver of
paper_2503_04558_gb300/slab.py run with the oracle as each slab's engine,
against the undivided oracle run from the same sorted state.

  * three slabs in one process (messages routed in memory), and two gloo
    ranks each holding one slab (torch.distributed point-to-point);
  * after the steps the slabs' particles, concatenated in slab order, are the
    undivided run's particles in the same order: cells and tags bit for bit,
    positions and momenta to 1e-12 (the current sums near a slab edge add the
    same contributions in another order, so the fields, and through them the
    pushes, differ at rounding level);
  * each slab's own rows of D and B match the undivided fields to 1e-12;
  * the rows outside each slab's update range are NaN during its field
    update (slab_oracle.OracleSlab), so the ghost-row width is checked too.
"""
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle as O  # noqa: E402
from slab_oracle import OracleSlab, split_sorted  # noqa: E402
from paper_2503_04558_gb300 import slab as SL, synth  # noqa: E402

A = 0.9
NR = NTH = 48
NSTEPS = 6


def setup_case(n=16000, seed=2):
    rin = 0.9 * O.horizon(A)
    c = O.make_cfg(NR, NTH, A, rin, 20.0)
    D, B = O.init_fields(c, O.WALD, 1.0)
    P = O.Particles(*synth.particles(NR, NTH, rin, 20.0, n, seed=seed, sigma=0.2))
    P = O.sort(c, P)   # the decomposition keeps the state sorted by cell
    return c, P, D, B


def undivided(c, P, D, B, nsteps):
    P, D, B = P.copy(), [x.copy() for x in D], [x.copy() for x in B]
    for _ in range(nsteps):
        _, P, _ = O.step(c, P, D, B)
    return P, D, B


def run_slabs(c, P, D, B, n_slabs, which, links, nsteps, ghost=None):
    rows = SL.partition(c.nth, n_slabs)
    parts = split_sorted(c, P, rows)
    engines = {s: OracleSlab(c, parts[s], D, B) for s in which}
    run = SL.SlabRun(engines, n_slabs, c.nth, c.n_fld_iter, links, ghost=ghost)
    assert run.rows == rows
    for _ in range(nsteps):
        run.step()
    return run, engines


def check_against(c, run, engines, Pu, Du, Bu):
    for s, e in engines.items():
        assert e.status == 0
        j0, j1 = run.rows[s]
        for x, y in zip(e.D + e.B, Du + Bu):
            own = slice(j0, j1)
            assert np.all(np.isfinite(x[own]))
            assert np.max(np.abs(x[own] - y[own])) <= 1e-12 * np.max(np.abs(y)), (s, j0, j1)


def compare_particles(c, got, Pu):
    keys_u = O.cell_keys(c, Pu)
    assert got.n == Pu.n
    assert np.array_equal(O.cell_keys(c, got), keys_u)
    assert np.array_equal(got.tag, Pu.tag)
    for x, y in ((got.r, Pu.r), (got.th, Pu.th), (got.u1, Pu.u1), (got.u2, Pu.u2), (got.u3, Pu.u3)):
        assert np.max(np.abs(x - y)) <= 1e-12 * max(1.0, np.max(np.abs(y)))


def test_partition_covers_the_rows():
    for nth, ns in ((48, 2), (48, 5), (2048, 8), (64, 3)):
        rows = SL.partition(nth, ns)
        assert rows[0][0] == 0 and rows[-1][1] == nth + 1
        for (a0, a1), (b0, b1) in zip(rows, rows[1:]):
            assert a1 == b0 and a1 > a0
        sizes = [min(j1, nth) - j0 for j0, j1 in rows]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        SL.partition(48, 6, min_rows=9)
    assert [SL.ghost_rows(n) for n in (0, 1, 2, 7)] == [1, 1, 2, 4]


def test_three_slabs_in_one_process_match_the_undivided_run():
    c, P, D, B = setup_case()
    Pu, Du, Bu = undivided(c, P, D, B, NSTEPS)
    run, engines = run_slabs(c, P, D, B, 3, [0, 1, 2], SL.LocalLinks(), NSTEPS)
    check_against(c, run, engines, Pu, Du, Bu)
    got = O.Particles(*[np.concatenate([getattr(engines[s].P, k) for s in range(3)])
                        for k in ("r", "th", "u1", "u2", "u3", "tag")])
    compare_particles(c, got, Pu)
    # particles did cross the slab edges in both directions
    assert any(e.P.n != p.n for e, p in zip(engines.values(), split_sorted(c, P, run.rows)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c, P, D, B = setup_case()
        run, engines = run_slabs(c, P, D, B, world, [rank], SL.DistLinks("cpu"), NSTEPS)
        e = engines[rank]
        j0, j1 = run.rows[rank]
        q.put((rank, e.status, j0, j1, [x[j0:j1].copy() for x in e.D + e.B],
               [getattr(e.P, k).copy() for k in ("r", "th", "u1", "u2", "u3", "tag")]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_the_undivided_run():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    c, P, D, B = setup_case()
    Pu, Du, Bu = undivided(c, P, D, B, NSTEPS)
    for rank, st, j0, j1, own, _ in out:
        assert st == 0
        for x, y in zip(own, Du + Bu):
            assert np.max(np.abs(x - y[j0:j1])) <= 1e-12 * np.max(np.abs(y))
    got = O.Particles(*[np.concatenate([o[5][k] for o in out]) for k in range(6)])
    compare_particles(c, got, Pu)


def test_one_ghost_row_fewer_lets_the_outside_in():
    """With ceil((N + 1) / 2) - 1 ghost rows the NaN put outside each update
    range reaches the slabs' own rows: the width is the smallest that works."""
    c, P, D, B = setup_case(n=4000)
    run, engines = run_slabs(c, P, D, B, 3, [0, 1, 2], SL.LocalLinks(), 1, ghost=SL.ghost_rows(c.n_fld_iter) - 1)
    assert any(not np.all(np.isfinite(x[j0:j1])) for s, e in engines.items() for x in e.D + e.B
               for j0, j1 in [run.rows[s]])
