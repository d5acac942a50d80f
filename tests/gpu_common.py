"""Shared helpers of the GPU parity tests: one configuration built twice, for
the oracle and for the CUDA path, from the same numbers."""
import math

import numpy as np

import oracle as O


def configs(nr, nth, a, r_in, r_out, precision=64, **kw):
    from paper_2503_04558_gb300 import grpic as G
    oc = O.make_cfg(nr, nth, a, r_in, r_out, **kw)
    gk = dict(dt=oc.dt, beta_field=oc.beta_s, n_field_iter=oc.n_fld_iter, n_push_iter=oc.n_push_iter,
              damp_cells=oc.damp_cells, damp_max=oc.damp_max, q_over_m=tuple(oc.qm), q_weight=tuple(oc.qw),
              massive=tuple(oc.massive), precision=precision)
    gc = G.Config(nr, nth, a, r_in, r_out, **gk)
    assert gc.ld == oc.ld
    return oc, gc


def relerr(x, ref, mask=None):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    if mask is not None:
        x, ref = x[mask], ref[mask]
    scale = np.max(np.abs(ref))
    if scale == 0:
        return float(np.max(np.abs(x)))
    return float(np.max(np.abs(x - ref)) / scale)


def flux_form(oc, J):
    """Oracle current densities -> integrated currents J A (the library's J)."""
    AD, _ = O.areas(oc)
    return [J[0] * AD[0], J[1] * AD[1], J[2] * AD[2]]


def logical(oc, r, th):
    return (np.log(r) - math.log(oc.r_in)) / oc.dx1, th / oc.dth
