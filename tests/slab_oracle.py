"""A slab engine made of the oracle, for the host tests of the theta-slab
decomposition (paper_2503_04558_gb300/slab.py): the same interface as the
library's engine, each call done with the FP64 oracle on the slab's own
particles and the whole-grid field arrays.

Test infrastructure only.  The field update of rows [lo, hi) is the oracle's
whole-grid update with every row outside [lo, hi) set to NaN first (D, B
and J) and restored afterwards: if the decomposition's ghost rows were too
few, or an exchange missing, NaN or stale values would reach the slab's own
rows."""
import numpy as np
import torch

import oracle as O

BPP = 5 * 8 + 4   # packed FP64 particle: r, theta, u_r, u_theta, u_phi, tag


def pack_particles(P, first, n):
    parts = [a[first:first + n].astype(np.float64).tobytes() for a in (P.r, P.th, P.u1, P.u2, P.u3)]
    parts.append(P.tag[first:first + n].astype(np.uint32).tobytes())
    return torch.frombuffer(bytearray(b"".join(parts)), dtype=torch.uint8) if n > 0 else torch.empty(0, dtype=torch.uint8)


def unpack_particles(buf, n):
    raw = bytes(buf.cpu().numpy().tobytes()) if n > 0 else b""
    arrs = []
    for k in range(5):
        arrs.append(np.frombuffer(raw[k * 8 * n:(k + 1) * 8 * n], dtype=np.float64).copy())
    arrs.append(np.frombuffer(raw[40 * n:44 * n], dtype=np.uint32).copy())
    return arrs


class OracleSlab:
    msg_device = "cpu"

    def __init__(self, c, P, D, B):
        self.c = c
        self.P = P
        self.D = [x.copy() for x in D]
        self.B = [x.copy() for x in B]
        self.J = O.zeros_fields(c, 3)
        self.status = 0

    # messages ---------------------------------------------------------------
    def halo_like(self, fset, nrows):
        return ((6 if fset == 0 else 3) * nrows * self.c.ld,), torch.float64

    def particles_like(self, n):
        return (n * BPP,), torch.uint8

    def _set(self, fset):
        return self.D + self.B if fset == 0 else self.J

    def halo_pack(self, fset, row0, nrows):
        return torch.from_numpy(np.concatenate([a[row0:row0 + nrows].ravel() for a in self._set(fset)]).copy())

    def halo_unpack(self, fset, row0, nrows, buf, add):
        v = buf.cpu().numpy().reshape(len(self._set(fset)), nrows, self.c.ld)
        for a, x in zip(self._set(fset), v):
            if add:
                a[row0:row0 + nrows] += x
            else:
                a[row0:row0 + nrows] = x

    # steps ------------------------------------------------------------------
    def push(self):
        st, J, _ = O.push_deposit(self.c, self.P, self.D, self.B)
        self.status = self.status or st
        self.J = J

    def field_update_rows(self, lo, hi):
        keep = [(a, a[:lo].copy(), a[hi:].copy()) for a in self.D + self.B]
        for a in self.D + self.B + self.J:
            a[:lo] = np.nan
            a[hi:] = np.nan
        O.field_update(self.c, self.D, self.B, self.J)
        for a, below, above in keep:
            a[:lo] = below
            a[hi:] = above

    def _rows(self):
        keys = O.cell_keys(self.c, self.P)
        return keys // self.c.nr

    def sort_split(self, j_lo, j_hi):
        self.P = O.sort(self.c, self.P)
        rows = self._rows()
        lo = int(np.sum(rows < j_lo))
        up = int(np.sum(rows >= j_hi))
        return lo, self.P.n - lo - up, up

    def particles_pack(self, first, n):
        return pack_particles(self.P, first, n)

    def assemble(self, own_first, own_n, lower, n_lower, upper, n_upper):
        parts = []
        if n_lower > 0:
            parts.append(unpack_particles(lower, n_lower))
        sl = slice(own_first, own_first + own_n)
        parts.append([self.P.r[sl], self.P.th[sl], self.P.u1[sl], self.P.u2[sl], self.P.u3[sl], self.P.tag[sl]])
        if n_upper > 0:
            parts.append(unpack_particles(upper, n_upper))
        cat = [np.concatenate([p[k] for p in parts]) for k in range(6)]
        self.P = O.Particles(*[x.copy() for x in cat])

    def sort(self):
        self.P = O.sort(self.c, self.P)


def split_sorted(c, P, rows):
    """The particles of each slab's rows, in the order of the sorted state P."""
    keys = O.cell_keys(c, P)
    r = keys // c.nr
    out = []
    for j0, j1 in rows:
        sel = np.where((r >= j0) & (r < min(j1, c.nth)))[0]
        out.append(P.take(sel))
    return out
