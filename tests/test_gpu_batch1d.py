"""Batched 1D spark gaps on the GPU (one persistent launch over many radial
lines) against the FP64 oracle's line model, through the C ABI.

Exact: particle order (survivors, then children in parent order), ids, the
set of photons that convert (Philox4x64-10 draws, FP64 decisions) and the
photons emitted.  Within FP32 precision: positions, momenta, J A and D^r."""
import math

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

A = 0.99
RH = 1.0 + math.sqrt(1 - A * A)


@pytest.fixture(scope="module")
def G():
    from paper_2503_04558_gb300 import build, grpic
    build.build()
    grpic.load()
    return grpic


def setup(G, nl=6, n=256, cap=20000, per_line=(500, 2000), seed=3, species=None, ur_scale=0.3, **kw):
    cfg = G.Batch1DConfig(nl, n, A, RH, 20.0, cap, **kw)
    B = G.Batch1D(cfg)
    L = G.Lines(cfg)
    rng = np.random.default_rng(seed)
    thetas = (np.arange(nl) + 0.5) * (math.pi / 2) / nl
    L.theta.copy_(torch.from_numpy(thetas))
    L.I0.copy_(torch.from_numpy(rng.normal(size=nl) * 50.0))
    B.init_fields(L)
    lines = []
    for k in range(nl):
        m = int(rng.integers(per_line[0], per_line[1]))
        x = rng.random(m) * (n - 2) + 1
        cell = np.floor(x).astype(np.int32)
        off = (x - cell).astype(np.float32)
        ur = (rng.normal(size=m) * ur_scale).astype(np.float32)
        up = (rng.normal(size=m) * 0.1).astype(np.float32)
        if species is None:
            # e-/e+ with an energetic tail (|u_r| up to ~3 gamma_thr) and photons
            tag = rng.integers(0, 3, m).astype(np.uint32)
            tag[tag == 2] = 3
            hot = rng.random(m) < 0.3
            ur[hot] = (rng.choice([-1, 1], hot.sum()) * rng.uniform(0.5, 3.0, hot.sum()) * cfg.gamma_thr
                       ).astype(np.float32)
            ph = tag == 3
            ur[ph] = (rng.choice([-1, 1], ph.sum()) * rng.uniform(3.0, 8.0, ph.sum())).astype(np.float32)
        else:
            tag = np.full(m, species).astype(np.uint32)
        pid = (np.arange(m, dtype=np.uint64) + np.uint64(k) * np.uint64(1 << 40))
        L.set_line(k, cell, off, ur, up, tag, pid)
        lines.append((cell, off, ur, up, tag, pid))
    return cfg, B, L, lines, thetas


def oracle_line(cfg, theta, I0, k_state, _unused):
    Lo = O.make_line(cfg.n_cells, cfg.a, theta, cfg.r_in, cfg.r_out, dt=cfg.dt, n_push_iter=cfg.n_push_iter,
                     qm=cfg.q_over_m, qw=cfg.q_weight, massive=cfg.massive, I0=I0, gamma_thr=cfg.gamma_thr,
                     eps_ph=cfg.eps_ph, tau=cfg.tau, seed=cfg.seed)
    cell, off, ur, up, tag, pid = k_state
    x = cell.astype(np.float64) + off.astype(np.float64)
    S = O.LineState(x, ur.astype(np.float64), up.astype(np.float64), tag, pid, cfg.capacity)
    return Lo, S


def test_initial_fields_match_oracle(G):
    cfg, B, L, lines, thetas = setup(G, nl=5, B0=123.0)
    for k in range(cfg.n_lines):
        Lo, _ = oracle_line(cfg, thetas[k], 0.0, lines[k], None)
        ref = O.line_init_D(Lo, cfg.B0)
        assert np.max(np.abs(L.D[k].cpu().numpy() - ref)) <= 1e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape", [None, (128, 2, 2)], ids=["one_cta_per_line", "cluster_of_two"])
def test_one_step_matches_oracle(G, shape):
    cfg, B, L, lines, thetas = setup(G, B0=200.0, gamma_thr=30.0, tau=40.0)
    if shape:
        B.set_launch(*shape)
    I0 = L.I0.cpu().numpy()
    B.run(L, 1, 0)
    assert B.sync() == 0
    emitted = conv = 0
    for k in range(cfg.n_lines):
        Lo, S = oracle_line(cfg, thetas[k], I0[k], lines[k], None)
        D = O.line_init_D(Lo, cfg.B0)
        st, JA, c = O.line_step(Lo, 0, S, D)
        assert st == 0
        emitted += c[0]
        conv += c[1]
        g = L.line(k)
        v = S.view()
        assert len(g["id"]) == S.n
        assert np.array_equal(g["id"], v["id"]) and np.array_equal(g["tag"], v["tag"])
        xg = g["cell"] + g["off"].astype(np.float64)
        assert np.max(np.abs(xg - v["x1"])) < 2e-4, k              # cells
        assert np.max(np.abs(g["ur"] - v["ur"]) / np.maximum(1, np.abs(v["ur"]))) < 1e-4, k
        assert np.max(np.abs(g["up"] - v["up"]) / np.maximum(1, np.abs(v["up"]))) < 1e-4, k
        ja = L.JA[k].cpu().numpy()
        assert np.max(np.abs(ja - JA)) <= 1e-3 * max(1.0, np.max(np.abs(JA))), k
        dg = L.D[k].cpu().numpy()
        assert np.max(np.abs(dg - D)) <= 1e-4 * max(1.0, np.max(np.abs(D))), k
    ev = L.events.cpu().numpy()
    assert ev[0] == emitted and ev[1] == conv
    assert emitted > 100 and conv > 100
    print("one step: photons emitted", emitted, "converted", conv)


def test_photon_conversions_are_bit_exact(G):
    """A photon-only batch: the photons that convert (Philox draw below
    1 - exp(-tau dt), FP64 energy check) are exactly the oracle's."""
    cfg, B, L, lines, thetas = setup(G, nl=4, species=3, ur_scale=8.0, tau=200.0, seed=11)
    B.run(L, 1, 7)  # global step 7
    assert B.sync() == 0
    for k in range(cfg.n_lines):
        Lo, S = oracle_line(cfg, thetas[k], 0.0, lines[k], None)
        st, JA, c = O.line_step(Lo, 7, S, np.zeros(cfg.n_cells))
        g = L.line(k)
        assert np.array_equal(g["id"], S.view()["id"]) and np.array_equal(g["tag"], S.view()["tag"])
        assert c[1] > 0


def test_many_steps_track_the_oracle_statistically(G):
    cfg, B, L, lines, thetas = setup(G, nl=3, B0=300.0, gamma_thr=20.0, tau=20.0, cap=200000, seed=5)
    I0 = L.I0.cpu().numpy()
    nsteps = 40
    B.run(L, nsteps, 0)
    assert B.sync() == 0
    for k in range(cfg.n_lines):
        Lo, S = oracle_line(cfg, thetas[k], I0[k], lines[k], None)
        D = O.line_init_D(Lo, cfg.B0)
        for s in range(nsteps):
            st, JA, c = O.line_step(Lo, s, S, D)
            assert st == 0
        n_g = int(L.count[k].item())
        print("line", k, "particles GPU", n_g, "oracle", S.n, "initial", len(lines[k][0]))
        assert S.n > 1.2 * len(lines[k][0])     # the cascade grew the line
        assert abs(n_g - S.n) <= 0.05 * S.n + 10
        tg = L.line(k)["tag"]
        assert abs((tg == 3).sum() - (S.view()["tag"] == 3).sum()) <= 0.1 * max(1, (S.view()["tag"] == 3).sum()) + 10


@pytest.mark.parametrize("shape", [None, (128, 2, 2)], ids=["one_cta_per_line", "cluster_of_two"])
def test_capacity_overflow_is_reported(G, shape):
    from paper_2503_04558_gb300 import grpic as GG
    cfg, B, L, lines, thetas = setup(G, nl=2, species=3, ur_scale=8.0, tau=1e4, cap=2000, per_line=(1900, 2000))
    if shape:
        B.set_launch(*shape)
    B.run(L, 1, 0)
    assert B.sync() == GG.EOVERFLOW
    assert int(L.count.max().item()) <= cfg.capacity


def test_tuner_picks_a_launch_shape_and_advances(G):
    cfg, B, L, lines, thetas = setup(G, nl=8)
    done, best = B.tune(L, 2, 0)
    assert B.sync() == 0
    assert best[0] in (128, 256, 512, 1024) and best[1] in (1, 2, 4) and best[2] in (1, 2)
    assert done >= 2 and done % 2 == 0


def test_graph_runs_match_direct_runs(G):
    """grpic_batch1d_run_graph (graph built on the first call, the persistent
    kernel's arguments updated on later ones) gives the lines of
    grpic_batch1d_run bit for bit, emissions and conversions included."""
    out = []
    for graph in (False, True):
        cfg, B, L, lines, thetas = setup(G, nl=6, seed=11)
        run = B.run_graph if graph else B.run
        run(L, 3, 0)
        run(L, 2, 3)
        run(L, 4, 5)
        assert B.sync() == 0
        out.append(([L.line(k) for k in range(6)], L.D.cpu().numpy().copy(), L.events.cpu().numpy().copy()))
    (l0, d0, e0), (l1, d1, e1) = out
    assert e0[0] > 0 and e0[1] > 0          # the runs emitted and converted photons
    assert np.array_equal(e0, e1)
    assert np.array_equal(d0.view(np.uint32), d1.view(np.uint32))
    for a, b in zip(l0, l1):
        for k in a:
            assert np.array_equal(a[k], b[k]), k


def test_cluster_shares_lines_like_one_cta(G):
    """Two CTAs per line (a thread-block cluster on two SMs, each pushing half
    of the line's particles, the halves' currents summed through distributed
    shared memory): after one step and after four more from a graph the
    lines hold the one-CTA run's particles in the same order with the same
    ids and tags, the same emissions and conversions happened, and positions,
    momenta and D^r agree to FP32 rounding (the current is accumulated in
    fixed point, so its sum does not depend on which CTA or warp deposits
    first)."""
    outs = []
    for shape in ((128, 2, 1), (128, 2, 2)):
        cfg, B, L, lines, thetas = setup(G, nl=6, seed=11, B0=200.0, gamma_thr=30.0, tau=40.0)
        B.set_launch(*shape)
        B.run(L, 1, 0)
        assert B.sync() == 0
        one = ([L.line(k) for k in range(cfg.n_lines)], L.D.cpu().numpy().copy(), L.events.cpu().numpy().copy())
        B.run_graph(L, 4, 1)
        assert B.sync() == 0
        many = ([L.line(k) for k in range(cfg.n_lines)], L.D.cpu().numpy().copy(), L.events.cpu().numpy().copy())
        outs.append((one, many))
    (o1, m1), (o2, m2) = outs
    assert o1[2][0] > 0 and o1[2][1] > 0           # the step emitted and converted photons
    for when, x, y in (("1 step", o1, o2), ("5 steps", m1, m2)):
        assert np.array_equal(x[2], y[2]), when   # emissions, conversions, pushes
        dd = np.max(np.abs(x[1] - y[1])) / np.max(np.abs(x[1]))
        worst = {"D": dd}
        for a, b in zip(x[0], y[0]):
            for key in ("cell", "tag", "id"):
                assert np.array_equal(a[key], b[key]), (when, key)
            xa, xb = a["cell"] + a["off"].astype(np.float64), b["cell"] + b["off"].astype(np.float64)
            worst["x"] = max(worst.get("x", 0.0), float(np.max(np.abs(xa - xb), initial=0.0)))
            for key in ("ur", "up"):
                d = np.abs(a[key] - b[key]) / np.maximum(1.0, np.abs(a[key]))
                worst[key] = max(worst.get(key, 0.0), float(np.max(d, initial=0.0)))
        print(f"cluster of two vs one CTA per line, {when}:", {k: f"{v:.1e}" for k, v in worst.items()})
        # the two kernels are separate instantiations: the compiler may fuse
        # multiply-adds differently, which moves results by FP32 rounding
        assert dd <= 1e-6 and worst["x"] <= 1e-4 and worst["ur"] <= 1e-5 and worst["up"] <= 1e-5, (when, worst)


def test_launch_shapes_are_checked(G):
    from paper_2503_04558_gb300 import grpic as GG
    cfg, B, L, lines, thetas = setup(G, nl=2)
    for bad in ((100, 1, 1), (2048, 1, 1), (256, 99, 1), (256, 1, 3), (256, 0, 1)):
        with pytest.raises(GG.GrpicError):
            B.set_launch(*bad)
    B.set_launch(1024, 1, 2)
