"""grpic_sort_noalloc: the sort by cell for callers that cannot allocate
device memory (stream capture that must not see cudaMalloc, hosts whose memory
pools own the device, plugin hosts that forbid library allocations).  Called
through the C ABI and checked against grpic_sort, which allocates its scratch
in a context; both must give the same sorted particles on two calls in a row.
The file is named to be collected last; it also runs alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2503_04558_gb300 import build, grpic
    build.build()
    grpic.load()
    return grpic


def _particles(G, cfg, n, seed):
    from paper_2503_04558_gb300 import synth
    r, th, u1, u2, u3, tag = synth.particles(cfg.n_r, cfg.n_theta, cfg.r_in, cfg.r_out, n, seed=seed, sigma=0.3)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(r))
    tag = tag[perm].copy()
    tag[::53] |= np.uint32(G.DEAD)
    return [x[perm] for x in (r, th, u1, u2, u3)] + [tag]


def _host(S):
    h = S.host()
    return [h[k] for k in ("x1", "x2", "u1", "u2", "u3", "tag")]


@pytest.mark.parametrize("precision,n_side,n", [(64, 48, 30000), (32, 48, 30000), (64, 512, 2097152),
                                               (32, 512, 2097152)])
def test_noalloc_sort_matches_context_sort_twice(G, precision, n_side, n):
    """Small grids, and the largest case the fixed scratch takes (2,097,152
    slots on 512 x 512 cells); the device's free memory is the same before and
    after the second call (nothing allocated)."""
    cfg = G.Config(n_side, n_side - 8 if n_side < 100 else n_side, 0.9, 1.2923, 30.0, precision=precision)
    assert n <= G.NOALLOC_MAX_PARTICLES and cfg.n_r * cfg.n_theta <= G.NOALLOC_MAX_CELLS
    ctx = G.Context(cfg)
    lib = G.load()
    grid = cfg.grid_c()
    ref = G.ParticleSet(cfg, n)
    nal = G.ParticleSet(cfg, n)
    for call in range(2):
        arrs = _particles(G, cfg, n, seed=11 + call)
        if precision == 64:
            ref.load(*arrs)
            nal.load(*arrs)
        else:
            cell, o1, o2 = ctx.fp32_encode(torch.from_numpy(arrs[0]).cuda(), torch.from_numpy(arrs[1]).cuda())
            st = [o1, o2] + [torch.from_numpy(a.astype(np.float32)) for a in arrs[2:5]] + [arrs[5], cell]
            ref.load(*st)
            nal.load(*st)
        ctx.sort(ref)
        nal._sc.n = nal.n
        nal._ss.n = nal.n
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        status = lib.grpic_sort_noalloc(C.byref(grid), precision, C.byref(nal._sc), C.byref(nal._ss),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert status == G.OK
        nal.sync_ptrs()
        torch.cuda.synchronize()
        if call > 0:
            # the first call of a process may load the library's fixed array
            # (module data, placed when the module loads); later calls change
            # nothing in the device's free memory
            assert torch.cuda.mem_get_info()[0] == free0
        assert ctx.sync() == 0
        assert nal.live() == ref.live()
        for a, b in zip(_host(nal), _host(ref)):
            assert np.array_equal(a, b)
        if precision == 32:
            assert np.array_equal(nal.host()["cell"], ref.host()["cell"])


def test_noalloc_rejects_sizes_beyond_its_scratch(G):
    lib = G.load()
    cfg = G.Config(1024, 1024, 0.9, 1.2923, 30.0)   # 1,048,576 cells > 262,144
    S = G.ParticleSet(cfg, 8)
    grid = cfg.grid_c()
    st = lib.grpic_sort_noalloc(C.byref(grid), 64, C.byref(S._sc), C.byref(S._ss), None)
    assert st == G.EOVERFLOW
    small = G.Config(64, 64, 0.9, 1.2923, 30.0)
    T = G.ParticleSet(small, 8)
    T._sc.n = G.NOALLOC_MAX_PARTICLES + 1
    T._sc.capacity = T._sc.n
    T._ss.capacity = T._sc.n
    st = lib.grpic_sort_noalloc(C.byref(small.grid_c()), 64, C.byref(T._sc), C.byref(T._ss), None)
    assert st == G.EOVERFLOW
