"""Seeded synthetic inputs shaped like the paper's runs.

This module is shared by the tests, the benchmark and the oracle-side checks;
it holds none of the method's arithmetic (no metric, no push, no deposit, no
field solve).  It only draws positions and momenta:

* positions uniform in logical coordinates inside each cell, the cells filled
  round-robin so that every cell gets floor or ceil of N/(2 cells) pairs; each
  position is shared by one electron (species 0) and one positron (species 1),
  so the initial charge density is exactly zero;
* r = r_in * exp(x1 * dx1), theta = x2 * dtheta (the grid map of the log-r x
  theta mesh);
* momenta: covariant u_r = s n1, u_theta = s r n2, u_phi = s r sin(theta) n3
  with n ~ N(0, 1) (flat-space coordinate scale factors), s = sigma for the
  Gaussian recipe; for the thermal recipe s*n is replaced by a momentum drawn
  from the Maxwell-Juettner distribution at temperature T (Sobol's rejection
  method as described by Zenitani 2015) with an isotropic direction.
"""
from __future__ import annotations

import math
import numpy as np


def grid_spacing(nr: int, nth: int, r_in: float, r_out: float):
    return math.log(r_out / r_in) / nr, math.pi / nth


def pair_positions(nr, nth, n_pairs, seed, cell_offset=0):
    """Logical positions (x1, x2) of n_pairs pair sites, round-robin over cells."""
    rng = np.random.Generator(np.random.Philox(seed))
    ncell = nr * nth
    k = np.arange(n_pairs, dtype=np.int64) + cell_offset
    cell = k % ncell
    i = (cell % nr).astype(np.float64)
    j = (cell // nr).astype(np.float64)
    off = rng.random((n_pairs, 2))
    return i + off[:, 0], j + off[:, 1]


def maxwell_juttner(n, T, rng):
    """|u| samples from the Maxwell-Juettner distribution (Sobol's method)."""
    out = np.empty(n)
    filled = 0
    while filled < n:
        m = max(2 * (n - filled), 1024)
        x = rng.random((m, 4))
        x = np.clip(x, 1e-300, 1.0)
        u = -T * np.log(x[:, 0] * x[:, 1] * x[:, 2])
        eta = -T * np.log(x[:, 0] * x[:, 1] * x[:, 2] * x[:, 3])
        ok = eta * eta - u * u > 1.0
        take = u[ok][: n - filled]
        out[filled:filled + take.size] = take
        filled += take.size
    return out


def particles(nr, nth, r_in, r_out, n_particles, seed=0, sigma=0.1, thermal_T=None):
    """FP64 SoA particle arrays (r, theta, u_r, u_theta, u_phi, tag) as numpy.

    n_particles is rounded down to an even number; particle 2k is an electron
    and 2k+1 a positron at the same position with independent momenta."""
    dx1, dth = grid_spacing(nr, nth, r_in, r_out)
    n_pairs = n_particles // 2
    x1, x2 = pair_positions(nr, nth, n_pairs, seed)
    x1 = np.repeat(x1, 2)
    x2 = np.repeat(x2, 2)
    r = r_in * np.exp(x1 * dx1)
    th = x2 * dth
    rng = np.random.Generator(np.random.Philox(seed + 0x9E3779B9))
    n = 2 * n_pairs
    if thermal_T is None:
        g = rng.standard_normal((n, 3)) * sigma
    else:
        mag = maxwell_juttner(n, thermal_T, rng)
        v = rng.standard_normal((n, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        g = v * mag[:, None]
    u1 = g[:, 0]
    u2 = g[:, 1] * r
    u3 = g[:, 2] * r * np.sin(th)
    tag = np.tile(np.array([0, 1], np.uint32), n_pairs)
    return r, th, u1, u2, u3, tag


def particles_torch(nr, nth, r_in, r_out, n_particles, seed=0, sigma=0.1, thermal_T=None, device="cuda",
                    chunk=1 << 24):
    """Same recipe drawn with torch on the device (large benchmark sizes); the
    random streams differ from the numpy version but the distribution is the
    same.  Returns a dict of torch tensors (float64 r, th, u1..u3; int32 tag)."""
    import torch

    dx1, dth = grid_spacing(nr, nth, r_in, r_out)
    n_pairs = n_particles // 2
    n = 2 * n_pairs
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    out = {k: torch.empty(n, dtype=torch.float64, device=device) for k in ("r", "th", "u1", "u2", "u3")}
    out["tag"] = torch.empty(n, dtype=torch.int32, device=device)
    ncell = nr * nth
    for s in range(0, n_pairs, chunk):
        e = min(n_pairs, s + chunk)
        m = e - s
        k = torch.arange(s, e, device=device, dtype=torch.int64)
        cell = k % ncell
        x1 = (cell % nr).double() + torch.rand(m, generator=gen, device=device, dtype=torch.float64)
        x2 = (cell // nr).double() + torch.rand(m, generator=gen, device=device, dtype=torch.float64)
        x1 = x1.repeat_interleave(2)
        x2 = x2.repeat_interleave(2)
        r = r_in * torch.exp(x1 * dx1)
        th = x2 * dth
        if thermal_T is None:
            g = torch.randn(2 * m, 3, generator=gen, device=device, dtype=torch.float64) * sigma
        else:
            mag = _mj_torch(2 * m, thermal_T, gen, device)
            v = torch.randn(2 * m, 3, generator=gen, device=device, dtype=torch.float64)
            v = v / v.norm(dim=1, keepdim=True)
            g = v * mag[:, None]
        sl = slice(2 * s, 2 * e)
        out["r"][sl] = r
        out["th"][sl] = th
        out["u1"][sl] = g[:, 0]
        out["u2"][sl] = g[:, 1] * r
        out["u3"][sl] = g[:, 2] * r * torch.sin(th)
        out["tag"][sl] = torch.arange(2 * m, device=device, dtype=torch.int32) % 2
    return out


def _mj_torch(n, T, gen, device):
    import torch

    out = torch.empty(n, dtype=torch.float64, device=device)
    filled = 0
    while filled < n:
        m = max(2 * (n - filled), 1024)
        x = torch.rand(m, 4, generator=gen, device=device, dtype=torch.float64).clamp_min(1e-300)
        u = -T * torch.log(x[:, 0] * x[:, 1] * x[:, 2])
        eta = -T * torch.log(x[:, 0] * x[:, 1] * x[:, 2] * x[:, 3])
        take = u[eta * eta - u * u > 1.0][: n - filled]
        out[filled:filled + take.numel()] = take
        filled += take.numel()
    return out
