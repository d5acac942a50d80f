"""Plain FP64 CPU oracle of the GRPIC time step (arXiv:2503.04558, Sec. 2 and
App. A-C), written in C (``grpic_oracle.c``) and wrapped here with ctypes.

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only ``tests/``, ``__graft_entry__.smoke()``
and the cpu_baseline / reference leg of ``bench.py`` may import this package.
It shares no code with the CUDA path and never imports it.

Array conventions (an interface both sides implement independently):
  field arrays are float64 of shape (nth+1, ld), row j = theta index,
  column c = i + ng (ng = 2) where i is the r index of the component's own
  lattice (integer or half-integer, Fig. Yee of the paper).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grpic_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")

DEAD = np.uint32(0x80000000)
NG = 2

WALD, WALD_A0, MONOPOLE, SPLIT_MONOPOLE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc -O2 -ffp-contract=off (no FMA contraction),
    with OpenMP for the multi-threaded CPU baseline where the compiler has it
    (one thread unless set_threads says otherwise)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


class Cfg(C.Structure):
    _fields_ = [("nr", C.c_int), ("nth", C.c_int), ("ng", C.c_int), ("ld", C.c_int),
                ("a", C.c_double), ("r_in", C.c_double), ("r_out", C.c_double),
                ("dx1", C.c_double), ("dth", C.c_double),
                ("dt", C.c_double), ("beta_s", C.c_double),
                ("n_fld_iter", C.c_int), ("n_push_iter", C.c_int),
                ("damp_cells", C.c_int), ("damp_max", C.c_double),
                ("qm", C.c_double * 4), ("qw", C.c_double * 4), ("massive", C.c_int * 4),
                ("pusher", C.c_int), ("shape", C.c_int), ("radiation", C.c_int), ("injection", C.c_int),
                ("gamma_thr", C.c_double), ("eps_ph", C.c_double), ("tau", C.c_double),
                ("sigma_thr", C.c_double), ("eps_db", C.c_double), ("seed", C.c_uint64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i, l, p = C.c_double, C.c_int, C.c_long, C.c_void_p
        pc = C.POINTER(Cfg)
        sig = {
            "orc_metric_eval": (None, [d, d, d, p]),
            "orc_closed_fields": (None, [i, d, d, d, d, p]),
            "orc_gauss_legendre": (None, [p, p]),
            "orc_areas": (None, [pc, p, p, p, p, p, p]),
            "orc_init_fields": (None, [pc, i, d, p, p, p, p, p, p]),
            "orc_field_update": (None, [pc, p, p, p, p, p, p, p, p, p]),
            "orc_circulations": (None, [pc] + [p] * 12),
            "orc_geodesic_rhs": (None, [d, d, p, p]),
            "orc_boris": (None, [d, d, d, d, d, p, p, p]),
            "orc_vay": (None, [d, d, d, d, d, p, p, p]),
            "orc_w3": (d, [d]),
            "orc_push_values": (None, [d, d, i, d, i, p, p, p]),
            "orc_push_analytic": (i, [i, d, d, d, i, d, i, p, l, l, p]),
            "orc_interp": (None, [pc, p, p, p, p, p, p, d, d, p]),
            "orc_deposit_one": (None, [pc, p, p, p, d, d, d, d, d, d]),
            "orc_push_deposit": (i, [pc, l, p, p, p, p, p, p, p, p, p, p, p, p, p, p, p, p]),
            "orc_cell_keys": (None, [pc, l, p, p, p, p]),
            "orc_counting_sort": (l, [l, l, p, p]),
            "orc_radiate": (i, [pc, C.c_int64, p, l, p, p, p, p, p, p, p]),
            "orc_inject": (i, [pc, C.c_int64, p, l, p, p, p, p, p, p, p, p, p, p, p, p, p]),
            "orc_rho": (None, [pc, l, p, p, p, p]),
            "orc_divD": (None, [pc, p, p, p]),
            "orc_divB": (None, [pc, p, p, p]),
            "orc_horizon_flux": (d, [pc, p, p, p, p, p, p, i]),
            "orc_set_threads": (i, [i]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def set_threads(n: int) -> int:
    """Host threads of the push and the field update (1 = the parity
    setting); returns the count in effect (1 without OpenMP)."""
    return int(lib().orc_set_threads(int(n)))


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------
# configuration
# --------------------------------------------------------------------------
def horizon(a: float) -> float:
    """Outer horizon r_H = 1 + sqrt(1 - a^2) (M = 1)."""
    return 1.0 + math.sqrt(1.0 - a * a)


def make_cfg(nr, nth, a, r_in, r_out, dt=None, cfl=0.5, beta_s=0.53, n_fld_iter=7, n_push_iter=3,
             damp_cells=None, damp_max=0.1, qm=(-1.0, 1.0, 1.0, 0.0), qw=(-1e-3, 1e-3, 1e-3, 0.0),
             massive=(1, 1, 1, 0), pusher=0, shape=1, radiation=0, injection=0, gamma_thr=100.0, eps_ph=4.0,
             tau=2.0, sigma_thr=10.0, eps_db=1e-3, seed=0) -> Cfg:
    """Grid uniform in ln r and theta; dt from the CFL reading
    dt = cfl * min(dr, r dtheta) at r_in when not given."""
    c = Cfg()
    c.nr, c.nth, c.ng = nr, nth, NG
    c.ld = nr + 2 * NG
    c.a, c.r_in, c.r_out = a, r_in, r_out
    c.dx1 = math.log(r_out / r_in) / nr
    c.dth = math.pi / nth
    if dt is None:
        dr = r_in * (math.exp(c.dx1) - 1.0)
        dt = cfl * min(dr, r_in * c.dth)
    c.dt = dt
    c.beta_s = beta_s
    c.n_fld_iter, c.n_push_iter = n_fld_iter, n_push_iter
    c.damp_cells = max(8, nr // 32) if damp_cells is None else damp_cells
    c.damp_max = damp_max
    for k in range(4):
        c.qm[k], c.qw[k], c.massive[k] = qm[k], qw[k], massive[k]
    c.pusher = pusher
    c.shape = shape
    c.radiation, c.injection = radiation, injection
    c.gamma_thr, c.eps_ph, c.tau = gamma_thr, eps_ph, tau
    c.sigma_thr, c.eps_db, c.seed = sigma_thr, eps_db, seed
    return c


def field_shape(c: Cfg):
    return (c.nth + 1, c.ld)


def zeros_fields(c: Cfg, n=6):
    return [np.zeros(field_shape(c)) for _ in range(n)]


# --------------------------------------------------------------------------
# wrappers
# --------------------------------------------------------------------------
METRIC_KEYS = ["alpha", "beta", "g_rr", "g_rp", "g_thth", "g_pp", "gi_rr", "gi_rp", "gi_thth", "gi_pp",
               "sqrtg", "da_r", "da_th", "db_r", "db_th", "dgi_rr_r", "dgi_rr_th", "dgi_rp_r", "dgi_rp_th",
               "dgi_thth_r", "dgi_thth_th", "dgi_pp_r", "dgi_pp_th"]


def metric(a, r, th) -> dict:
    out = np.zeros(23)
    lib().orc_metric_eval(a, r, th, _p(out))
    return dict(zip(METRIC_KEYS, out))


def closed_fields(kind, a, B0, r, th) -> dict:
    out = np.zeros(16)
    lib().orc_closed_fields(kind, a, B0, r, th, _p(out))
    return {"At": out[0], "Aph": out[1], "E": out[2:5].copy(), "sgB": out[5:8].copy(),
            "D": out[10:13].copy(), "B": out[13:16].copy()}


def gauss_legendre():
    x, w = np.zeros(10), np.zeros(10)
    lib().orc_gauss_legendre(_p(x), _p(w))
    return x, w


def areas(c: Cfg):
    arrs = zeros_fields(c)
    lib().orc_areas(C.byref(c), *[_p(x) for x in arrs])
    return arrs[:3], arrs[3:]


def init_fields(c: Cfg, kind: int, B0: float):
    arrs = zeros_fields(c)
    lib().orc_init_fields(C.byref(c), kind, B0, *[_p(x) for x in arrs])
    return arrs[:3], arrs[3:]


def field_update(c: Cfg, D, B, J):
    """In place: D, B lists of 3 arrays; J list of 3 current densities."""
    lib().orc_field_update(C.byref(c), *[_p(x) for x in list(D) + list(B) + list(J)])


def circulations(c: Cfg, D, B):
    out = zeros_fields(c)
    lib().orc_circulations(C.byref(c), *[_p(x) for x in list(D) + list(B) + out])
    return out[:3], out[3:]


def geodesic_rhs(a, eps, y):
    y = np.ascontiguousarray(y, dtype=np.float64)
    f = np.zeros(6)
    lib().orc_geodesic_rhs(a, eps, _p(y), _p(f))
    return f


def boris(a, r, th, qm, dt, Dv, Bv, u):
    u = np.array(u, dtype=np.float64)
    lib().orc_boris(a, r, th, qm, dt, _p(np.asarray(Dv, np.float64)), _p(np.asarray(Bv, np.float64)), _p(u))
    return u


def w3(x) -> float:
    """The cubic B-spline weight of the third-order shape."""
    return lib().orc_w3(float(x))


def vay(a, r, th, qm, dt, Dv, Bv, u):
    """Vay's momentum update in the FIDO frame over dt (fields D, B contravariant)."""
    u = np.array(u, dtype=np.float64)
    lib().orc_vay(a, r, th, qm, dt, _p(np.asarray(Dv, np.float64)), _p(np.asarray(Bv, np.float64)), _p(u))
    return u


def push_values(a, qm, massive, dt, n_iter, Dv, Bv, y):
    y = np.array(y, dtype=np.float64)
    lib().orc_push_values(a, qm, massive, dt, n_iter, _p(np.asarray(Dv, np.float64)),
                          _p(np.asarray(Bv, np.float64)), _p(y))
    return y


def push_analytic(kind, B0, a, qm, massive, dt, n_iter, y, nsteps, every):
    y = np.array(y, dtype=np.float64)
    nsamp = nsteps // every if every > 0 else 0
    traj = np.zeros((max(nsamp, 1), 6))
    n = lib().orc_push_analytic(kind, B0, a, qm, massive, dt, n_iter, _p(y), nsteps, every, _p(traj))
    return y, traj[:n]


def interp(c: Cfg, D, B, x1, x2):
    out = np.zeros(6)
    lib().orc_interp(C.byref(c), *[_p(x) for x in list(D) + list(B)], x1, x2, _p(out))
    return out


def deposit_one(c: Cfg, qw, x1a, x2a, x1b, x2b, dphi):
    JrA, JtA, Jph = zeros_fields(c, 3)
    lib().orc_deposit_one(C.byref(c), _p(JrA), _p(JtA), _p(Jph), qw, x1a, x2a, x1b, x2b, dphi)
    return JrA, JtA, Jph


class Particles:
    """SoA particle state of the FP64 path: r, theta, covariant u_i, tag
    (species in bits 0-1, DEAD in bit 31)."""

    def __init__(self, r, th, u1, u2, u3, tag):
        self.r = np.ascontiguousarray(r, np.float64)
        self.th = np.ascontiguousarray(th, np.float64)
        self.u1 = np.ascontiguousarray(u1, np.float64)
        self.u2 = np.ascontiguousarray(u2, np.float64)
        self.u3 = np.ascontiguousarray(u3, np.float64)
        self.tag = np.ascontiguousarray(tag, np.uint32)

    @property
    def n(self):
        return self.r.shape[0]

    def copy(self):
        return Particles(self.r.copy(), self.th.copy(), self.u1.copy(), self.u2.copy(), self.u3.copy(),
                         self.tag.copy())

    def take(self, idx):
        return Particles(self.r[idx], self.th[idx], self.u1[idx], self.u2[idx], self.u3[idx], self.tag[idx])


def push_deposit(c: Cfg, P: Particles, D, B):
    """Push + deposit in place; returns (status, J list, dphi array)."""
    J = zeros_fields(c, 3)
    dphi = np.zeros(P.n)
    st = lib().orc_push_deposit(C.byref(c), P.n, _p(P.r), _p(P.th), _p(P.u1), _p(P.u2), _p(P.u3), _p(P.tag),
                                _p(dphi), *[_p(x) for x in list(D) + list(B) + J])
    return st, J, dphi


def cell_keys(c: Cfg, P: Particles):
    k = np.zeros(P.n, np.int32)
    lib().orc_cell_keys(C.byref(c), P.n, _p(P.r), _p(P.th), _p(P.tag), _p(k))
    return k


def counting_sort(keys: np.ndarray, nkeys: int):
    keys = np.ascontiguousarray(keys, np.int32)
    perm = np.zeros(keys.shape[0], np.int64)
    live = lib().orc_counting_sort(keys.shape[0], nkeys, _p(keys), _p(perm))
    return perm, live


def sort(c: Cfg, P: Particles) -> Particles:
    keys = cell_keys(c, P)
    perm, live = counting_sort(keys, c.nr * c.nth)
    return P.take(perm[:live])


def rho(c: Cfg, P: Particles):
    out = np.zeros(field_shape(c))
    lib().orc_rho(C.byref(c), P.n, _p(P.r), _p(P.th), _p(P.tag), _p(out))
    return out


def divD(c: Cfg, D):
    out = np.zeros(field_shape(c))
    lib().orc_divD(C.byref(c), _p(D[0]), _p(D[1]), _p(out))
    return out


def divB(c: Cfg, B):
    out = np.zeros(field_shape(c))
    lib().orc_divB(C.byref(c), _p(B[0]), _p(B[1]), _p(out))
    return out


def _grow(P: Particles, extra: int) -> Particles:
    pad = lambda a, fill: np.concatenate([a, np.full(extra, fill, a.dtype)])
    return Particles(pad(P.r, 1.0), pad(P.th, 1.0), pad(P.u1, 0.0), pad(P.u2, 0.0), pad(P.u3, 0.0),
                     pad(P.tag, DEAD))


def radiate(c: Cfg, P: Particles, step: int):
    """Emission and conversion after a push (slot order); children appended.
    Returns (status, P with the children, (emitted, converted))."""
    n = P.n
    Q = _grow(P, 2 * n + 2)
    np_ = C.c_long(n)
    counts = (C.c_long * 2)()
    st = lib().orc_radiate(C.byref(c), step, C.byref(np_), Q.n, _p(Q.r), _p(Q.th), _p(Q.u1), _p(Q.u2), _p(Q.u3),
                           _p(Q.tag), counts)
    return st, Q.take(np.arange(np_.value)), (counts[0], counts[1])


def inject(c: Cfg, P: Particles, D, B, step: int):
    """Pair injection after the field update (cell order); pairs appended.
    Returns (status, P with the pairs, number of cells that injected)."""
    extra = 2 * c.nr * c.nth
    Q = _grow(P, extra)
    np_ = C.c_long(P.n)
    cnt = C.c_long(0)
    st = lib().orc_inject(C.byref(c), step, C.byref(np_), Q.n, _p(Q.r), _p(Q.th), _p(Q.u1), _p(Q.u2), _p(Q.u3),
                          _p(Q.tag), *[_p(x) for x in list(D) + list(B)], C.byref(cnt))
    return st, Q.take(np.arange(np_.value)), cnt.value


def step(c: Cfg, P: Particles, D, B, do_sort=True, step=0, events=None):
    """One time step in the paper's order (Fig. stepping): push + deposit from
    fields n (then emission and conversion if c.radiation), field update
    n -> n+1 with J^{n+1/2} (then injection if c.injection), then the sort by
    cell.  `step` keys the random numbers; events (a list) receives
    (emitted, converted, injecting cells)."""
    st, J, dphi = push_deposit(c, P, D, B)
    ev = [0, 0, 0]
    if c.radiation:
        s2, P, (ev[0], ev[1]) = radiate(c, P, step)
        st = st or s2
    field_update(c, D, B, J)
    if c.injection:
        s3, P, ev[2] = inject(c, P, D, B, step)
        st = st or s3
    if events is not None:
        events.append(tuple(ev))
    if do_sort:
        P = sort(c, P)
    return st, P, J


# --------------------------------------------------------------------------
# batched 1D spark-gap line model (Sec. 4 pair production on radial lines)
# --------------------------------------------------------------------------
class Line(C.Structure):
    _fields_ = [("n", C.c_int), ("a", C.c_double), ("theta", C.c_double), ("r_in", C.c_double),
                ("r_out", C.c_double), ("dx1", C.c_double), ("dt", C.c_double), ("n_push_iter", C.c_int),
                ("qm", C.c_double * 4), ("qw", C.c_double * 4), ("massive", C.c_int * 4), ("I0", C.c_double),
                ("gamma_thr", C.c_double), ("eps_ph", C.c_double), ("tau", C.c_double), ("seed", C.c_uint64)]


def _line_sigs(lib_):
    d, i, l, p, u64 = C.c_double, C.c_int, C.c_long, C.c_void_p, C.c_uint64
    pl = C.POINTER(Line)
    sig = {
        "orc_philox4x64": (None, [p, p, p]),
        "orc_splitmix64": (u64, [u64]),
        "orc_child_id": (u64, [u64, C.c_int64, i]),
        "orc_uniform": (d, [u64, u64, C.c_int64, i]),
        "orc_line_area": (None, [pl, p]),
        "orc_line_init_D": (None, [pl, d, p]),
        "orc_line_step": (i, [pl, C.c_int64, p, l, p, p, p, p, p, p, p, p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib_, name)
        fn.restype = res
        fn.argtypes = args


def make_line(n, a, theta, r_in, r_out, dt=None, cfl=0.5, n_push_iter=3, qm=(-1.0, 1.0, 1.0, 0.0),
              qw=(-1.0, 1.0, 1.0, 0.0), massive=(1, 1, 1, 0), I0=0.0, gamma_thr=100.0, eps_ph=4.0, tau=2.0,
              seed=0) -> Line:
    L = Line()
    L.n, L.a, L.theta, L.r_in, L.r_out = n, a, theta, r_in, r_out
    L.dx1 = math.log(r_out / r_in) / n
    L.dt = cfl * r_in * (math.exp(L.dx1) - 1.0) if dt is None else dt
    L.n_push_iter = n_push_iter
    for k in range(4):
        L.qm[k], L.qw[k], L.massive[k] = qm[k], qw[k], massive[k]
    L.I0, L.gamma_thr, L.eps_ph, L.tau, L.seed = I0, gamma_thr, eps_ph, tau, seed
    return L


def philox4x64(ctr, key):
    lib_ = lib()
    _line_sigs(lib_)
    c = np.ascontiguousarray(ctr, np.uint64)
    k = np.ascontiguousarray(key, np.uint64)
    o = np.zeros(4, np.uint64)
    lib_.orc_philox4x64(_p(c), _p(k), _p(o))
    return o


def child_id(parent, step, k):
    lib_ = lib()
    _line_sigs(lib_)
    return lib_.orc_child_id(int(parent), int(step), int(k))


def uniform(seed, pid, step, event):
    lib_ = lib()
    _line_sigs(lib_)
    return lib_.orc_uniform(int(seed), int(pid), int(step), int(event))


class LineState:
    """Particles of one line: logical position x1, covariant u_r, u_phi,
    tag (species | DEAD) and 64-bit id, with room for `cap` particles."""

    def __init__(self, x1, ur, up, tag, pid, cap):
        n = len(x1)
        self.cap = int(cap)
        self.x1 = np.zeros(self.cap)
        self.ur = np.zeros(self.cap)
        self.up = np.zeros(self.cap)
        self.tag = np.zeros(self.cap, np.uint32)
        self.id = np.zeros(self.cap, np.uint64)
        self.x1[:n], self.ur[:n], self.up[:n] = x1, ur, up
        self.tag[:n], self.id[:n] = tag, pid
        self.n = n

    def view(self):
        n = self.n
        return dict(x1=self.x1[:n], ur=self.ur[:n], up=self.up[:n], tag=self.tag[:n], id=self.id[:n])


def line_area(L):
    lib_ = lib()
    _line_sigs(lib_)
    A = np.zeros(L.n)
    lib_.orc_line_area(C.byref(L), _p(A))
    return A


def line_init_D(L, B0):
    lib_ = lib()
    _line_sigs(lib_)
    D = np.zeros(L.n)
    lib_.orc_line_init_D(C.byref(L), B0, _p(D))
    return D


def line_step(L, step, S: LineState, D):
    """One step of the line model in place; returns (status, JA, counts)."""
    lib_ = lib()
    _line_sigs(lib_)
    JA = np.zeros(L.n + 2)
    counts = np.zeros(2, np.int64)
    n = C.c_long(S.n)
    st = lib_.orc_line_step(C.byref(L), step, C.byref(n), S.cap, _p(S.x1), _p(S.ur), _p(S.up), _p(S.tag),
                            _p(S.id), _p(D), _p(JA), _p(counts))
    S.n = n.value
    return st, JA, counts


# --------------------------------------------------------------------------
# differentiable form: objective and its finite-difference gradient
# --------------------------------------------------------------------------
def horizon_index(c: Cfg, a_nominal: float) -> int:
    """Vertex ring nearest the horizon of the nominal spin (the grid stays
    fixed when the spin is varied)."""
    return int(round(math.log(horizon(a_nominal) / c.r_in) / c.dx1))


def horizon_flux(c: Cfg, D, B, iH: int) -> float:
    return lib().orc_horizon_flux(C.byref(c), *[_p(x) for x in list(D) + list(B)], iH)


def flux_run(c: Cfg, P: Particles, D, B, nsteps: int, iH: int) -> float:
    """Time-averaged horizon flux over nsteps steps (push + deposit, field
    update; no sort, which only permutes particles): L = (1/N) sum_n flux(F^{n+1})."""
    P = P.copy()
    D = [x.copy() for x in D]
    B = [x.copy() for x in B]
    L = 0.0
    for _ in range(nsteps):
        st, J, _ = push_deposit(c, P, D, B)
        field_update(c, D, B, J)
        L += horizon_flux(c, D, B, iH)
    return L / nsteps
