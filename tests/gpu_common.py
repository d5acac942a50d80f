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
              massive=tuple(oc.massive), precision=precision, pusher=oc.pusher, shape_order=oc.shape)
    gc = G.Config(nr, nth, a, r_in, r_out, **gk)
    assert gc.ld == oc.ld
    return oc, gc


def relerr(x, ref, mask=None, floor=0.0):
    """max|x - ref| / max(max|ref|, floor) (max-norm relative error of an array)."""
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    if mask is not None:
        x, ref = x[mask], ref[mask]
    scale = max(np.max(np.abs(ref)), floor)
    if scale == 0:
        return float(np.max(np.abs(x)))
    return float(np.max(np.abs(x - ref)) / scale)


def flux_form(oc, J):
    """Oracle current densities -> integrated currents J A (the library's J)."""
    AD, _ = O.areas(oc)
    return [J[0] * AD[0], J[1] * AD[1], J[2] * AD[2]]


def logical(oc, r, th):
    return (np.log(r) - math.log(oc.r_in)) / oc.dx1, th / oc.dth


def fp32_offsets(oc, r, th):
    """The FP32 form's (cell, o1, o2) of FP64 positions, written out from the
    documented layout (include/grpic.h): offsets from the cell's lower edges,
    except in the last theta row, where o2 is the distance to theta = pi."""
    x1, x2 = logical(oc, r, th)
    i = np.clip(np.floor(x1), 0, oc.nr - 1)
    j = np.clip(np.floor(x2), 0, oc.nth - 1)
    o2 = np.where(j == oc.nth - 1, oc.nth - x2, x2 - j)
    return (j * oc.nr + i).astype(np.int32), (x1 - i).astype(np.float32), o2.astype(np.float32)


def fp32_logical(oc, cell, o1, o2):
    """Logical coordinates (x1, x2) of FP32-form positions (inverse of fp32_offsets)."""
    i = cell % oc.nr
    j = cell // oc.nr
    o2 = o2.astype(np.float64)
    return i + o1.astype(np.float64), np.where(j == oc.nth - 1, oc.nth - o2, j + o2)


def axis_grazers(oc, P, D, B, nsteps, theta_c=1e-3):
    """Oracle-only pre-run of nsteps full steps: indices into P of the particles
    whose path comes within theta_c of the polar axis (theta = 0 or pi).

    There gamma^{phi phi} ~ 1/sin^2(theta) makes the push ill-conditioned (the
    centrifugal barrier is not resolved by dt): a one-ulp difference between
    two libm implementations grows by orders of magnitude in one step, so two
    correct FP64 implementations cannot agree to 1e-10 on such paths."""
    P = P.copy()
    D = [x.copy() for x in D]
    B = [x.copy() for x in B]
    ids = np.arange(P.n)
    mind = np.minimum(P.th, math.pi - P.th)
    for _ in range(nsteps):
        st, J, _ = O.push_deposit(oc, P, D, B)
        O.field_update(oc, D, B, J)
        d = np.minimum(P.th, math.pi - P.th)
        mind[ids] = np.minimum(mind[ids], d)
        keys = O.cell_keys(oc, P)
        perm, live = O.counting_sort(keys, oc.nr * oc.nth)
        P = P.take(perm[:live])
        ids = ids[perm[:live]]
    return np.nonzero(mind < theta_c)[0]
