"""theta-slab domain decomposition of the GRPIC step.

The paper runs on many GPUs by cutting the domain among them and exchanging
the boundary data with MPI (Sec. 1).  Here the mesh is cut into slabs of
theta rows, one per rank.  Every rank keeps field arrays of the whole grid
(global row indices; 2048^2 fields take 0.5 GB of a GB300's 288 GB) but
pushes only the particles of its own rows [j0, j1) and updates only the rows
[j0 - G, j1 + G).  This module holds the host side: the partition, the
exchange schedule between neighbouring slabs and the step driver.  All
arithmetic on fields and particles runs in the library (the `LibrarySlab`
engine calls the entry points of include/grpic.h); this module moves
buffers between slabs and decides which rows and which slots travel.

One step of slab s (the driver runs each phase for every slab it holds
before the next phase's exchange):
  1. push its particles (the deposit zeroes and fills J);
  2. J halo reduction: the J rows outside [j0, j1) that its deposit reached
     (the cloud-in-cell window reaches one row below and two above a
     particle's row; the cubic shape two and three: HALO_J rows are sent)
     are added into their owners' rows;
  3. the owners' completed J rows fill the G ghost rows on either side;
  4. the field update of rows [j0 - G, j1 + G): a stage's D rows read the
     B rows at and below them, its B rows the D rows at and above them, so a
     wrong row outside the range moves half a row inwards per stage; with
     G = ceil((N + 1) / 2) for the 1 + N stages the rows [j0, j1) come out as
     in the undivided grid;
  5. the ghost rows of D and B are refilled from their owners;
  6. migration: a sort by cell puts the particles that left below j0 first
     and those above j1 last (a particle moves at most one row in a step);
     they travel to the neighbours, and the slab's next state is
     [arrivals from below | its own | arrivals from above], sorted again.
     Each neighbour's particles are in the undivided run's order, and a
     stable sort keeps the order of equal keys, so the slab ends with the
     undivided run's order of its particles.

Ranks are slabs.  `DistLinks` exchanges through torch.distributed
point-to-point calls (NCCL between GPUs, gloo on the host); `LocalLinks`
routes the messages of several slabs held by one process (one GPU can run
all slabs one after another: no kernel waits for another rank).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

HALO_J = 3  # J rows sent to each neighbour after the deposit


def ghost_rows(n_field_iter: int) -> int:
    """Ghost rows on each side of a slab's update range: ceil((N + 1) / 2)
    for the 1 + N field stages.  A stage's D row j reads B at rows j - 1 and
    j, its B row j reads D at rows j and j + 1 (through E_phi, H_phi and the
    theta edges of App. B), so a wrong row outside the range moves half a row
    inwards per stage.  The push's stencil reads one row beyond the slab's
    rows; those are ghost rows refilled after the update."""
    return (n_field_iter + 2) // 2


def partition(n_theta: int, n_slabs: int, min_rows: int = 1):
    """Field rows [j0, j1) of each slab, as equal as possible, the last slab
    also owning row n_theta (the theta = pi axis row of the integer-row
    components).  Particle rows of a slab: [j0, min(j1, n_theta))."""
    if n_slabs < 1 or n_theta // n_slabs < min_rows:
        raise ValueError(f"{n_slabs} slabs of at least {min_rows} rows do not fit {n_theta} rows")
    bounds = [(k * n_theta) // n_slabs for k in range(n_slabs + 1)]
    out = [(bounds[k], bounds[k + 1]) for k in range(n_slabs)]
    out[-1] = (out[-1][0], n_theta + 1)
    return out


@dataclass
class Msg:
    src: int
    dst: int
    key: str
    data: object   # a torch tensor (device for NCCL, host for gloo)


class LocalLinks:
    """Messages between slabs held by one process."""

    def round(self, out_msgs, expect):
        """out_msgs: list of Msg; expect: list of (dst, src, key, like) where
        like gives the shape and dtype of the message; returns {(dst, src,
        key): tensor}."""
        box = {(m.dst, m.src, m.key): m.data for m in out_msgs}
        return {(d, s, k): box[(d, s, k)] for d, s, k, _ in expect}


class DistLinks:
    """Messages between ranks through torch.distributed (rank = slab)."""

    def __init__(self, device=None):
        self.device = device

    def round(self, out_msgs, expect):
        import torch
        import torch.distributed as dist
        reqs = []
        got = {}
        for d, s, k, like in expect:
            buf = torch.empty(like[0], dtype=like[1], device=self.device)
            got[(d, s, k)] = buf
            reqs.append(dist.irecv(buf, s))
        for m in out_msgs:
            reqs.append(dist.isend(m.data.contiguous(), m.dst))
        for r in reqs:
            r.wait()
        return got


class SlabRun:
    """The decomposed step over the slabs this process holds.

    engines: {slab id: engine}; an engine implements push, halo_pack,
    halo_unpack, field_update_rows, sort_split, particles_pack, assemble,
    sort, halo_like(set, nrows) and particles_like(n) (shape and dtype of a
    message) -- `LibrarySlab` is the library's."""

    def __init__(self, engines: dict, n_slabs: int, n_theta: int, n_field_iter: int, links, ghost=None):
        self.e = engines
        self.n = n_slabs
        self.nth = n_theta
        self.G = ghost_rows(n_field_iter) if ghost is None else ghost
        self.rows = partition(n_theta, n_slabs, min_rows=max(self.G, HALO_J))
        self.links = links

    def _halo_round(self, fset, send_rows, add):
        """send_rows(s) -> [(dst, row0, nrows)] for each local slab; the
        receiver unpacks the same global rows."""
        out, expect = [], []
        for s, eng in self.e.items():
            for dst, r0, nr in send_rows(s):
                out.append(Msg(s, dst, f"{fset}:{r0}", eng.halo_pack(fset, r0, nr)))
        for s, eng in self.e.items():
            for src in (s - 1, s + 1):
                if 0 <= src < self.n:
                    for dst, r0, nr in send_rows(src):
                        if dst == s:
                            expect.append((s, src, f"{fset}:{r0}", eng.halo_like(fset, nr), r0, nr))
        got = self.links.round(out, [x[:4] for x in expect])
        for s, src, key, _, r0, nr in expect:
            self.e[s].halo_unpack(fset, r0, nr, got[(s, src, key)], add)

    def _reduction_rows(self, s):
        """J rows of slab s's deposit that belong to its neighbours."""
        j0, j1 = self.rows[s]
        out = []
        if s > 0:
            out.append((s - 1, max(0, j0 - HALO_J), j0 - max(0, j0 - HALO_J)))
        if s < self.n - 1:
            out.append((s + 1, j1, min(self.nth + 1, j1 + HALO_J) - j1))
        return out

    def _ghost_rows(self, s):
        """Own rows of slab s that its neighbours keep as ghost rows."""
        j0, j1 = self.rows[s]
        out = []
        if s > 0:
            out.append((s - 1, j0, min(self.G, j1 - j0)))
        if s < self.n - 1:
            out.append((s + 1, j1 - min(self.G, j1 - j0), min(self.G, j1 - j0)))
        return out

    def step(self):
        for eng in self.e.values():
            eng.push()
        self._halo_round(1, self._reduction_rows, add=True)
        self._halo_round(1, self._ghost_rows, add=False)
        for s, eng in self.e.items():
            j0, j1 = self.rows[s]
            eng.field_update_rows(max(0, j0 - self.G), min(self.nth + 1, j1 + self.G))
        self._halo_round(0, self._ghost_rows, add=False)
        self._migrate()

    def _migrate(self):
        import torch
        counts = {}
        for s, eng in self.e.items():
            j0, j1 = self.rows[s]
            counts[s] = eng.sort_split(j0, min(j1, self.nth))
        # the counts first (each receiver sizes its buffers), then the particles
        out, expect = [], []
        for s in self.e:
            lo, own, up = counts[s]
            if s > 0:
                out.append(Msg(s, s - 1, "n", torch.tensor([lo], dtype=torch.int64, device=self.e[s].msg_device)))
            if s < self.n - 1:
                out.append(Msg(s, s + 1, "n", torch.tensor([up], dtype=torch.int64, device=self.e[s].msg_device)))
            for src in (s - 1, s + 1):
                if 0 <= src < self.n:
                    expect.append((s, src, "n", ((1,), torch.int64)))
        got = self.links.round(out, expect)
        arrivals = {s: {src: int(got[(s, src, "n")].item()) for src in (s - 1, s + 1) if 0 <= src < self.n}
                    for s in self.e}
        out, expect = [], []
        for s, eng in self.e.items():
            lo, own, up = counts[s]
            if s > 0:
                out.append(Msg(s, s - 1, "p", eng.particles_pack(0, lo)))
            if s < self.n - 1:
                out.append(Msg(s, s + 1, "p", eng.particles_pack(lo + own, up)))
            for src, m in arrivals[s].items():
                expect.append((s, src, "p", eng.particles_like(m)))
        got = self.links.round(out, expect)
        for s, eng in self.e.items():
            lo, own, up = counts[s]
            n_lo = arrivals[s].get(s - 1, 0)
            n_up = arrivals[s].get(s + 1, 0)
            eng.assemble(lo, own, got.get((s, s - 1, "p")), n_lo, got.get((s, s + 1, "p")), n_up)
            eng.sort()


class LibrarySlab:
    """One slab on the GPU: a context, its particles (a ParticleSet holding
    the slab's particles) and fields of the whole grid, driven through the
    library's decomposition entry points."""

    def __init__(self, ctx, S, F, stream=None):
        import torch
        from . import grpic as G
        self.G = G
        self.ctx, self.S, self.F = ctx, S, F
        self.stream = stream
        self.lib = ctx.lib
        cfg = ctx.cfg
        self.fdt = torch.float64 if cfg.precision == 64 else torch.float32
        self.esz = 8 if cfg.precision == 64 else 4
        self.bpp = 5 * self.esz + 4 + (4 if cfg.precision == 32 else 0)   # bytes per packed particle
        self.ld = F.ld
        self.device = F.D[0].device
        self.msg_device = self.device

    def _st(self):
        return self.G._stream(self.stream)

    def _check(self, st, what):
        self.ctx._check(st, what)

    def push(self):
        self.ctx.push(self.S, self.F, self.stream)

    def halo_like(self, fset, nrows):
        return ((6 if fset == 0 else 3) * nrows * self.ld,), self.fdt

    def particles_like(self, n):
        return (n * self.bpp,), __import__("torch").uint8

    def halo_pack(self, fset, row0, nrows):
        import torch
        shape, dt = self.halo_like(fset, nrows)
        buf = torch.empty(shape, dtype=dt, device=self.device)
        fc = self.F.c()
        self._check(self.lib.grpic_halo_pack(self.ctx.h, C.byref(fc), fset, row0, nrows, C.c_void_p(buf.data_ptr()),
                                             self._st()), "grpic_halo_pack")
        return buf

    def halo_unpack(self, fset, row0, nrows, buf, add):
        fc = self.F.c()
        self._check(self.lib.grpic_halo_unpack(self.ctx.h, C.byref(fc), fset, row0, nrows,
                                               C.c_void_p(buf.data_ptr()), 1 if add else 0, self._st()),
                    "grpic_halo_unpack")

    def field_update_rows(self, j_lo, j_hi):
        fc = self.F.c()
        self._check(self.lib.grpic_field_update_rows(self.ctx.h, C.byref(fc), j_lo, j_hi, self._st()),
                    "grpic_field_update_rows")

    def sort_split(self, j_lo, j_hi):
        S = self.S
        S._sc.n = S.n
        S._ss.n = S.n
        out = (C.c_int64 * 3)()
        self._check(self.lib.grpic_sort_split(self.ctx.h, C.byref(S._sc), C.byref(S._ss), j_lo, j_hi, out,
                                              self._st()), "grpic_sort_split")
        S.sync_ptrs()
        return int(out[0]), int(out[1]), int(out[2])

    def particles_pack(self, first, n):
        import torch
        buf = torch.empty((n * self.bpp,), dtype=torch.uint8, device=self.device)
        S = self.S
        self._check(self.lib.grpic_particles_pack(self.ctx.h, C.byref(S._sc), first, n, C.c_void_p(buf.data_ptr()),
                                                  self._st()), "grpic_particles_pack")
        return buf

    def assemble(self, own_first, own_n, lower, n_lower, upper, n_upper):
        S = self.S
        lo = C.c_void_p(lower.data_ptr()) if lower is not None and n_lower > 0 else None
        up = C.c_void_p(upper.data_ptr()) if upper is not None and n_upper > 0 else None
        self._check(self.lib.grpic_slab_assemble(self.ctx.h, C.byref(S._ss), C.byref(S._sc), own_first, own_n, lo,
                                                 n_lower, up, n_upper, self._st()), "grpic_slab_assemble")
        # the other buffer now holds the state
        S.a, S.b = S.b, S.a
        S._sc, S._ss = S._ss, S._sc
        S.n = int(S._sc.n)

    def sort(self):
        self.ctx.sort(self.S, self.stream)
