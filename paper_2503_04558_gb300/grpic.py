"""Thin ctypes binding of libgrpic (include/grpic.h).

Argument marshalling only: every step of the time step runs in the CUDA
kernels of the library.  torch tensors provide the device memory and the
stream.  Importing this module does not need a GPU; loading the library does,
and every call fails loudly (RuntimeError) if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libgrpic.so")

OK, EINVAL, ENOMEM, ECUDA, ERANGE, ENAN, EOVERFLOW, ECONVERGE, ETIMEOUT = range(9)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ERANGE", "ENAN", "EOVERFLOW", "ECONVERGE", "ETIMEOUT"]
WALD, WALD_A0, MONOPOLE, SPLIT_MONOPOLE = 0, 1, 2, 3
DEAD = 0x80000000
NG = 2

# names the header declares (checked by the CPU test of the boundary)
EXPORTS = ["grpic_init", "grpic_init_fields", "grpic_push", "grpic_deposit", "grpic_field_update", "grpic_sort",
           "grpic_step", "grpic_step_graph", "grpic_diagnostics", "grpic_charge_check", "grpic_get_areas", "grpic_sync", "grpic_last_error", "grpic_destroy",
           "grpic_sort_noalloc", "grpic_set_timing", "grpic_get_timing", "grpic_alu_peak",
           "grpic_field_update_rows", "grpic_halo_pack", "grpic_halo_unpack", "grpic_sort_split",
           "grpic_particles_pack", "grpic_slab_assemble", "grpic_set_field_path", "grpic_fp32_encode",
           "grpic_fp32_decode", "grpic_step_host"]
NOALLOC_MAX_PARTICLES = 2097152
NOALLOC_MAX_CELLS = 262144


class Grid(C.Structure):
    _fields_ = [("n_r", C.c_int32), ("n_theta", C.c_int32), ("r_in", C.c_double), ("r_out", C.c_double),
                ("damp_cells", C.c_int32), ("damp_max", C.c_double)]


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("beta_field", C.c_double), ("n_field_iter", C.c_int32),
                ("n_push_iter", C.c_int32), ("q_over_m", C.c_double * 4), ("q_weight", C.c_double * 4),
                ("massive", C.c_int32 * 4), ("precision", C.c_int32), ("sort_every", C.c_int32),
                ("fp64_radius", C.c_double), ("push_tol", C.c_double), ("island_arith", C.c_int32),
                ("pusher", C.c_int32), ("shape_order", C.c_int32), ("radiation", C.c_int32),
                ("injection", C.c_int32), ("gamma_thr", C.c_double), ("eps_ph", C.c_double), ("tau", C.c_double),
                ("sigma_thr", C.c_double), ("eps_db", C.c_double), ("seed", C.c_uint64)]


class ParticlesC(C.Structure):
    _fields_ = [("n", C.c_int64), ("capacity", C.c_int64), ("d_count", C.c_void_p),
                ("x1", C.c_void_p), ("x2", C.c_void_p), ("u1", C.c_void_p), ("u2", C.c_void_p),
                ("u3", C.c_void_p), ("tag", C.c_void_p), ("cell", C.c_void_p)]


class FieldsC(C.Structure):
    _fields_ = [("D", C.c_void_p * 3), ("B", C.c_void_p * 3), ("J", C.c_void_p * 3), ("ld", C.c_int64)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libgrpic.so; raise if it has not been built."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgrpic.so not found at {path}: build it with __graft_entry__.build()")
    lib = C.CDLL(path)
    v, p, i, d, i64 = C.c_void_p, C.POINTER, C.c_int, C.c_double, C.c_int64
    sig = {
        "grpic_init": [i, d, p(Grid), p(Params), p(v)],
        "grpic_init_fields": [v, i, d, p(FieldsC), v],
        "grpic_push": [v, p(ParticlesC), p(FieldsC), v],
        "grpic_deposit": [v, p(ParticlesC), p(ParticlesC), v, p(FieldsC), v],
        "grpic_field_update": [v, p(FieldsC), v],
        "grpic_sort": [v, p(ParticlesC), p(ParticlesC), v],
        "grpic_step": [v, p(ParticlesC), p(ParticlesC), p(FieldsC), i, v],
        "grpic_step_graph": [v, p(ParticlesC), p(ParticlesC), p(FieldsC), i, v],
        "grpic_diagnostics": [v, p(ParticlesC), p(FieldsC), v, v, v],
        "grpic_charge_check": [v, p(ParticlesC), p(FieldsC), v, v, p(d), v],
        "grpic_get_areas": [v, v * 6, i64, v],
        "grpic_sync": [v, v],
        "grpic_sort_noalloc": [p(Grid), C.c_int32, p(ParticlesC), p(ParticlesC), v],
        "grpic_set_timing": [v, i],
        "grpic_get_timing": [v, p(d), p(i64)],
        "grpic_alu_peak": [C.c_int32, p(d), v],
        "grpic_field_update_rows": [v, p(FieldsC), C.c_int32, C.c_int32, v],
        "grpic_halo_pack": [v, p(FieldsC), C.c_int32, C.c_int32, C.c_int32, v, v],
        "grpic_halo_unpack": [v, p(FieldsC), C.c_int32, C.c_int32, C.c_int32, v, C.c_int32, v],
        "grpic_sort_split": [v, p(ParticlesC), p(ParticlesC), C.c_int32, C.c_int32, p(i64), v],
        "grpic_particles_pack": [v, p(ParticlesC), i64, i64, v, v],
        "grpic_slab_assemble": [v, p(ParticlesC), p(ParticlesC), i64, i64, v, i64, v, i64, v],
        "grpic_set_field_path": [v, C.c_int32],
        "grpic_fp32_encode": [v, i64, v, v, v, v, v, v],
        "grpic_fp32_decode": [v, i64, v, v, v, v, v, v],
        "grpic_step_host": [v, p(ParticlesC), p(ParticlesC), p(ParticlesC), p(FieldsC), p(FieldsC), i, p(i64), v],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.grpic_last_error.argtypes = [v]
    lib.grpic_last_error.restype = C.c_char_p
    lib.grpic_destroy.argtypes = [v]
    lib.grpic_destroy.restype = None
    if path == LIB_PATH:
        _lib = lib
    return lib


def alu_peak(kind: int, stream=None):
    """Measured FMA ceiling of the current device: kind 0 FP32, 1 FP64, 2
    packed FP32.  Returns (flop/s, FMA warp-instructions/s, SM count)."""
    lib = load()
    out = (C.c_double * 3)()
    st = lib.grpic_alu_peak(int(kind), out, _stream(stream))
    if st != OK:
        raise GrpicError(st, "grpic_alu_peak")
    return out[0], out[1], int(out[2])


class GrpicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


def horizon(a: float) -> float:
    return 1.0 + math.sqrt(1.0 - a * a)


@dataclass
class Config:
    """Grid + solver settings of one run.  dt defaults to
    cfl * min(dr, r dtheta) at r_in."""
    n_r: int
    n_theta: int
    a: float
    r_in: float
    r_out: float
    dt: float | None = None
    cfl: float = 0.5
    beta_field: float = 0.53
    n_field_iter: int = 7
    n_push_iter: int = 3
    damp_cells: int | None = None
    damp_max: float = 0.1
    q_over_m: tuple = (-1.0, 1.0, 1.0, 0.0)
    q_weight: tuple = (-1e-3, 1e-3, 1e-3, 0.0)
    massive: tuple = (1, 1, 1, 0)
    precision: int = 64
    sort_every: int = 1
    fp64_radius: float = 0.0
    push_tol: float = 0.0
    island_arith: int = 0     # 0 double-FP32 pairs, 1 native FP64
    pusher: int = 0           # 0 generalized Boris, 1 Vay in the FIDO frame
    shape_order: int = 1      # 1 cloud in cell, 3 cubic spline (FP64 path)
    radiation: int = 0        # 2D photon emission and pair conversion (FP64 path)
    injection: int = 0        # pair injection where sigma > sigma_thr and |D.B|/B^2 > eps_db
    gamma_thr: float = 100.0
    eps_ph: float = 4.0
    tau: float = 2.0
    sigma_thr: float = 10.0
    eps_db: float = 1e-3
    seed: int = 0

    def __post_init__(self):
        self.dx1 = math.log(self.r_out / self.r_in) / self.n_r
        self.dth = math.pi / self.n_theta
        if self.dt is None:
            dr = self.r_in * (math.exp(self.dx1) - 1.0)
            self.dt = self.cfl * min(dr, self.r_in * self.dth)
        if self.damp_cells is None:
            self.damp_cells = max(8, self.n_r // 32)
        self.ld = self.n_r + 2 * NG

    def grid_c(self):
        return Grid(self.n_r, self.n_theta, self.r_in, self.r_out, self.damp_cells, self.damp_max)

    def params_c(self):
        p = Params()
        p.dt, p.beta_field = self.dt, self.beta_field
        p.n_field_iter, p.n_push_iter = self.n_field_iter, self.n_push_iter
        for k in range(4):
            p.q_over_m[k], p.q_weight[k], p.massive[k] = self.q_over_m[k], self.q_weight[k], self.massive[k]
        p.precision, p.sort_every, p.fp64_radius = self.precision, self.sort_every, self.fp64_radius
        p.push_tol = self.push_tol
        p.island_arith = self.island_arith
        p.pusher = self.pusher
        p.shape_order = self.shape_order
        p.radiation, p.injection = self.radiation, self.injection
        p.gamma_thr, p.eps_ph, p.tau = self.gamma_thr, self.eps_ph, self.tau
        p.sigma_thr, p.eps_db, p.seed = self.sigma_thr, self.eps_db, self.seed
        return p


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Fields:
    """D, B, J on the device as (n_theta+1, ld) tensors of the run's precision."""

    def __init__(self, cfg: Config, device="cuda", ld=None):
        import torch
        dt = torch.float64 if cfg.precision == 64 else torch.float32
        self.ld = ld or cfg.ld
        shape = (cfg.n_theta + 1, self.ld)
        self.D = [torch.zeros(shape, dtype=dt, device=device) for _ in range(3)]
        self.B = [torch.zeros(shape, dtype=dt, device=device) for _ in range(3)]
        self.J = [torch.zeros(shape, dtype=dt, device=device) for _ in range(3)]

    def c(self):
        f = FieldsC()
        for k in range(3):
            f.D[k] = self.D[k].data_ptr()
            f.B[k] = self.B[k].data_ptr()
            f.J[k] = self.J[k].data_ptr()
        f.ld = self.ld
        return f


class Particles:
    """Structure-of-arrays particle buffer (one of the two sort buffers)."""

    def __init__(self, cfg: Config, capacity: int, device="cuda"):
        import torch
        fdt = torch.float64 if cfg.precision == 64 else torch.float32
        cap = max(int(capacity), 1)
        self.capacity = cap
        self.x1 = torch.zeros(cap, dtype=fdt, device=device)
        self.x2 = torch.zeros(cap, dtype=fdt, device=device)
        self.u1 = torch.zeros(cap, dtype=fdt, device=device)
        self.u2 = torch.zeros(cap, dtype=fdt, device=device)
        self.u3 = torch.zeros(cap, dtype=fdt, device=device)
        self.tag = torch.full((cap,), DEAD, dtype=torch.int64, device=device).to(torch.int32)
        self.cell = torch.zeros(cap, dtype=torch.int32, device=device) if cfg.precision == 32 else None

    def arrays(self):
        return [self.x1, self.x2, self.u1, self.u2, self.u3, self.tag, self.cell]


class HostParticles:
    """A particle state in pinned host memory (the arrays of Particles) for
    grpic_step_host; n live slots."""

    def __init__(self, cfg: Config, capacity: int):
        import torch
        fdt = torch.float64 if cfg.precision == 64 else torch.float32
        cap = max(int(capacity), 1)
        self.capacity = cap
        self.n = 0
        mk = lambda dt: torch.zeros(cap, dtype=dt, pin_memory=True)
        self.x1, self.x2, self.u1, self.u2, self.u3 = (mk(fdt) for _ in range(5))
        self.tag = mk(torch.int32)
        self.cell = mk(torch.int32) if cfg.precision == 32 else None

    def arrays(self):
        return [self.x1, self.x2, self.u1, self.u2, self.u3, self.tag, self.cell]

    def c(self):
        s = ParticlesC()
        s.n = self.n
        s.capacity = self.capacity
        s.d_count = 0
        s.x1, s.x2, s.u1, s.u2, s.u3 = (t.data_ptr() for t in (self.x1, self.x2, self.u1, self.u2, self.u3))
        s.tag = self.tag.data_ptr()
        s.cell = self.cell.data_ptr() if self.cell is not None else 0
        return s


class HostFields:
    """D and B in pinned host memory, the layout of Fields (J unused)."""

    def __init__(self, F):
        import torch
        self.ld = F.ld
        self.D = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in F.D]
        self.B = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in F.B]

    def c(self):
        f = FieldsC()
        for k in range(3):
            f.D[k] = self.D[k].data_ptr()
            f.B[k] = self.B[k].data_ptr()
            f.J[k] = 0
        f.ld = self.ld
        return f


class ParticleSet:
    """Two particle buffers (sort ping-pong), the live count on the device and
    the C struct the library sees."""

    def __init__(self, cfg: Config, capacity: int, device="cuda"):
        import torch
        self.cfg = cfg
        self.a = Particles(cfg, capacity, device)
        self.b = Particles(cfg, capacity, device)
        self.count = torch.zeros(1, dtype=torch.int64, device=device)
        self.n = 0
        self._sc = self._struct(self.a)
        self._ss = self._struct(self.b)

    def _struct(self, P):
        s = ParticlesC()
        s.n = self.n
        s.capacity = P.capacity
        s.d_count = self.count.data_ptr()
        s.x1, s.x2, s.u1, s.u2, s.u3 = (t.data_ptr() for t in (P.x1, P.x2, P.u1, P.u2, P.u3))
        s.tag = P.tag.data_ptr()
        s.cell = P.cell.data_ptr() if P.cell is not None else 0
        return s

    def load(self, x1, x2, u1, u2, u3, tag, cell=None):
        """Copy host or device arrays into the current buffer; n = len(x1)."""
        import torch
        n = int(len(x1))
        if n > self.a.capacity:
            raise ValueError("capacity exceeded")
        dev = self.a.x1.device
        self.a.x1[:n].copy_(torch.as_tensor(x1).to(dev))
        self.a.x2[:n].copy_(torch.as_tensor(x2).to(dev))
        self.a.u1[:n].copy_(torch.as_tensor(u1).to(dev))
        self.a.u2[:n].copy_(torch.as_tensor(u2).to(dev))
        self.a.u3[:n].copy_(torch.as_tensor(u3).to(dev))
        t = torch.as_tensor(tag)
        if t.dtype != torch.int32:
            t = t.to(torch.int64).to(torch.int32) if t.dtype != torch.uint32 else t.view(torch.int32)
        self.a.tag[:n].copy_(t.to(dev))
        if cell is not None:
            self.a.cell[:n].copy_(torch.as_tensor(cell).to(dev))
        self.a.tag[n:].fill_(DEAD - (1 << 32))
        self.n = n
        self.count.fill_(n)
        self._sc = self._struct(self.a)
        self._ss = self._struct(self.b)

    def sync_ptrs(self):
        """After the library swapped the array pointers, swap the Python buffers too."""
        if self._sc.x1 != self.a.x1.data_ptr():
            self.a, self.b = self.b, self.a

    def live(self) -> int:
        return int(self.count.item())

    def host(self):
        """Live particles as numpy arrays (synchronizes)."""
        n = self.live()
        out = {k: getattr(self.a, k)[:n].cpu().numpy() for k in ("x1", "x2", "u1", "u2", "u3")}
        out["tag"] = self.a.tag[:n].cpu().numpy().view("uint32")
        if self.a.cell is not None:
            out["cell"] = self.a.cell[:n].cpu().numpy()
        return out


class Context:
    """Owns one grpic_ctx (tables + scratch) for a Config."""

    def __init__(self, cfg: Config):
        import torch
        torch.cuda.current_device()
        self.lib = load()
        self.cfg = cfg
        self._g = cfg.grid_c()
        self._p = cfg.params_c()
        h = C.c_void_p()
        st = self.lib.grpic_init(0, cfg.a, C.byref(self._g), C.byref(self._p), C.byref(h))
        if st != OK:
            raise GrpicError(st, "grpic_init failed")
        self.h = h

    def _check(self, st, what):
        if st != OK:
            msg = self.lib.grpic_last_error(self.h)
            raise GrpicError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.grpic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- entry points -----------------------------------------------------
    def init_fields(self, F: Fields, kind=WALD, B0=1.0, stream=None):
        fc = F.c()
        self._check(self.lib.grpic_init_fields(self.h, kind, B0, C.byref(fc), _stream(stream)), "grpic_init_fields")

    def push(self, P: ParticleSet, F: Fields, stream=None):
        P._sc.n = P.n
        fc = F.c()
        self._check(self.lib.grpic_push(self.h, C.byref(P._sc), C.byref(fc), _stream(stream)), "grpic_push")

    def deposit(self, before: ParticleSet, after: ParticleSet, dphi, F: Fields, stream=None):
        fc = F.c()
        before._sc.n = before.n
        after._sc.n = after.n
        self._check(self.lib.grpic_deposit(self.h, C.byref(before._sc), C.byref(after._sc), _ptr(dphi), C.byref(fc),
                                           _stream(stream)), "grpic_deposit")

    def field_update(self, F: Fields, stream=None):
        fc = F.c()
        self._check(self.lib.grpic_field_update(self.h, C.byref(fc), _stream(stream)), "grpic_field_update")

    def sort(self, P: ParticleSet, stream=None):
        P._sc.n = P.n
        P._ss.n = P.n
        self._check(self.lib.grpic_sort(self.h, C.byref(P._sc), C.byref(P._ss), _stream(stream)), "grpic_sort")
        P.sync_ptrs()

    def step(self, P: ParticleSet, F: Fields, nsteps=1, stream=None):
        P._sc.n = P.n
        P._ss.n = P.n
        fc = F.c()
        self._check(self.lib.grpic_step(self.h, C.byref(P._sc), C.byref(P._ss), C.byref(fc), nsteps,
                                        _stream(stream)), "grpic_step")
        P.sync_ptrs()
        P.n = P._sc.n   # radiation or injection: the whole capacity is the slot range

    def step_host(self, H: HostParticles, P: ParticleSet, F: Fields, nsteps=1, host_fields=None, stream=None):
        """grpic_step_host: nsteps steps with the particle state in H (pinned
        host memory), P's buffers as the device copy, H.n updated to the
        live count; host_fields (HostFields) copied in and out every step
        too.  Returns (bytes host to device, bytes device to host)."""
        hc = H.c()
        P._sc.n = H.n
        P._ss.n = H.n
        fc = F.c()
        hf = host_fields.c() if host_fields is not None else None
        out = (C.c_int64 * 2)()
        self._check(self.lib.grpic_step_host(self.h, C.byref(hc), C.byref(P._sc), C.byref(P._ss),
                                             C.byref(hf) if hf is not None else None, C.byref(fc), nsteps, out,
                                             _stream(stream)), "grpic_step_host")
        H.n = hc.n
        P.sync_ptrs()
        P.n = hc.n
        return out[0], out[1]

    def fp32_encode(self, r, th, stream=None):
        """(cell, o1, o2) of the FP32 form from FP64 positions (device tensors
        r, theta); the last theta row's offset is the distance to the pole."""
        import torch
        r, th = r.contiguous(), th.contiguous()
        n = int(r.numel())
        cell = torch.empty(n, dtype=torch.int32, device=r.device)
        o1 = torch.empty(n, dtype=torch.float32, device=r.device)
        o2 = torch.empty(n, dtype=torch.float32, device=r.device)
        self._check(self.lib.grpic_fp32_encode(self.h, n, _ptr(r), _ptr(th), _ptr(cell), _ptr(o1), _ptr(o2),
                                               _stream(stream)), "grpic_fp32_encode")
        return cell, o1, o2

    def fp32_decode(self, cell, o1, o2, stream=None):
        """FP64 (r, theta) device tensors of FP32-form positions."""
        import torch
        cell, o1, o2 = cell.contiguous(), o1.contiguous(), o2.contiguous()
        n = int(cell.numel())
        r = torch.empty(n, dtype=torch.float64, device=cell.device)
        th = torch.empty(n, dtype=torch.float64, device=cell.device)
        self._check(self.lib.grpic_fp32_decode(self.h, n, _ptr(cell), _ptr(o1), _ptr(o2), _ptr(r), _ptr(th),
                                               _stream(stream)), "grpic_fp32_decode")
        return r, th

    def set_field_path(self, fused: bool):
        """FP32 field update by fused shared-memory launches (True, the
        default) or one launch per stage (False); the same operations, fields
        equal to FP32 rounding."""
        self._check(self.lib.grpic_set_field_path(self.h, 1 if fused else 0), "grpic_set_field_path")

    def set_timing(self, enable: bool):
        """Record per-phase CUDA events in every step of grpic_step."""
        self._check(self.lib.grpic_set_timing(self.h, 1 if enable else 0), "grpic_set_timing")

    def get_timing(self):
        """(push ms, field update ms, sort ms) summed over the timed steps
        since the last read, and their number; waits for the events."""
        out = (C.c_double * 3)()
        n = C.c_int64()
        self._check(self.lib.grpic_get_timing(self.h, out, C.byref(n)), "grpic_get_timing")
        return out[0], out[1], out[2], n.value

    def step_graph(self, P: ParticleSet, F: Fields, nsteps=1, stream=None):
        """grpic_step with steps 2 .. nsteps-1 replayed from a captured CUDA
        graph of two steps (nsteps >= 4; fewer run as grpic_step)."""
        P._sc.n = P.n
        P._ss.n = P.n
        fc = F.c()
        self._check(self.lib.grpic_step_graph(self.h, C.byref(P._sc), C.byref(P._ss), C.byref(fc), nsteps,
                                              _stream(stream)), "grpic_step_graph")
        P.sync_ptrs()

    def diagnostics(self, P: ParticleSet | None, F: Fields, stream=None):
        import torch
        dt = torch.float64 if self.cfg.precision == 64 else torch.float32
        shape = (self.cfg.n_theta + 1, F.ld)
        rho = torch.zeros(shape, dtype=dt, device=F.D[0].device) if P is not None else None
        div = torch.zeros(shape, dtype=dt, device=F.D[0].device)
        if P is not None:
            P._sc.n = P.n
        fc = F.c()
        self._check(self.lib.grpic_diagnostics(self.h, C.byref(P._sc) if P is not None else None, C.byref(fc),
                                               _ptr(rho), _ptr(div), _stream(stream)), "grpic_diagnostics")
        return rho, div

    def charge_check(self, P: ParticleSet | None, F: Fields, base=None, want_state=False, stream=None):
        """(max |div D - rho - base|, max |rho|) over the interior vertices in
        FP64, and this call's div D - rho (an FP64 tensor) if want_state."""
        import torch
        state = torch.zeros((self.cfg.n_theta + 1, F.ld), dtype=torch.float64, device=F.D[0].device) \
            if want_state else None
        if P is not None:
            P._sc.n = P.n
        out = (C.c_double * 2)()
        fc = F.c()
        self._check(self.lib.grpic_charge_check(self.h, C.byref(P._sc) if P is not None else None, C.byref(fc),
                                                _ptr(base), _ptr(state), out, _stream(stream)), "grpic_charge_check")
        return out[0], out[1], state

    def areas(self, stream=None):
        import torch
        ld = self.cfg.ld
        out = [torch.zeros((self.cfg.n_theta + 1, ld), dtype=torch.float64, device="cuda") for _ in range(6)]
        arr = (C.c_void_p * 6)(*[t.data_ptr() for t in out])
        self._check(self.lib.grpic_get_areas(self.h, arr, ld, _stream(stream)), "grpic_get_areas")
        return out

    def sync(self, stream=None) -> int:
        """Wait for the stream and return (and clear) the device status."""
        return self.lib.grpic_sync(self.h, _stream(stream))


# ---------------------------------------------------------------------------
# batched 1D spark gaps
# ---------------------------------------------------------------------------
class Batch1DParams(C.Structure):
    _fields_ = [("n_lines", C.c_int32), ("n_cells", C.c_int32), ("a", C.c_double), ("r_in", C.c_double),
                ("r_out", C.c_double), ("dt", C.c_double), ("n_push_iter", C.c_int32),
                ("q_over_m", C.c_double * 4), ("q_weight", C.c_double * 4), ("massive", C.c_int32 * 4),
                ("gamma_thr", C.c_double), ("eps_ph", C.c_double), ("tau", C.c_double), ("B0", C.c_double),
                ("seed", C.c_uint64), ("capacity", C.c_int64)]


class LinesC(C.Structure):
    _fields_ = [("theta", C.c_void_p), ("I0", C.c_void_p), ("D", C.c_void_p), ("JA", C.c_void_p),
                ("count", C.c_void_p), ("cell", C.c_void_p * 2), ("off", C.c_void_p * 2), ("ur", C.c_void_p * 2),
                ("up", C.c_void_p * 2), ("tag", C.c_void_p * 2), ("id", C.c_void_p * 2), ("cur", C.c_int32),
                ("events", C.c_void_p)]


def _load_b1(lib):
    v, p = C.c_void_p, C.POINTER
    for name, args in {"grpic_batch1d_init": [p(Batch1DParams), p(v)],
                       "grpic_batch1d_init_fields": [v, p(LinesC), v],
                       "grpic_batch1d_run": [v, p(LinesC), C.c_int, C.c_int64, v],
                       "grpic_batch1d_run_graph": [v, p(LinesC), C.c_int, C.c_int64, v],
                       "grpic_batch1d_tune": [v, p(LinesC), C.c_int, C.c_int64, p(C.c_int64), p(C.c_int32), v],
                       "grpic_batch1d_set_launch": [v, C.c_int32, C.c_int32, C.c_int32],
                       "grpic_batch1d_sync": [v, v]}.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.grpic_batch1d_destroy.argtypes = [v]
    lib.grpic_batch1d_destroy.restype = None


EXPORTS += ["grpic_batch1d_init", "grpic_batch1d_init_fields", "grpic_batch1d_run", "grpic_batch1d_run_graph",
            "grpic_batch1d_tune", "grpic_batch1d_set_launch",
            "grpic_batch1d_sync", "grpic_batch1d_destroy"]


@dataclass
class Batch1DConfig:
    """Batched radial lines (the spark-gap workload): n_lines lines of n_cells
    cells uniform in ln r on [r_in, r_out]; dt defaults to cfl * dr at r_in."""
    n_lines: int
    n_cells: int
    a: float
    r_in: float
    r_out: float
    capacity: int
    dt: float | None = None
    cfl: float = 0.5
    n_push_iter: int = 3
    q_over_m: tuple = (-1.0, 1.0, 1.0, 0.0)
    q_weight: tuple = (-1.0, 1.0, 1.0, 0.0)
    massive: tuple = (1, 1, 1, 0)
    gamma_thr: float = 100.0
    eps_ph: float = 4.0
    tau: float = 2.0
    B0: float = 2.0e3
    seed: int = 0

    def __post_init__(self):
        self.dx1 = math.log(self.r_out / self.r_in) / self.n_cells
        if self.dt is None:
            self.dt = self.cfl * self.r_in * (math.exp(self.dx1) - 1.0)

    def c(self):
        p = Batch1DParams()
        p.n_lines, p.n_cells, p.a, p.r_in, p.r_out, p.dt = self.n_lines, self.n_cells, self.a, self.r_in, \
            self.r_out, self.dt
        p.n_push_iter = self.n_push_iter
        for k in range(4):
            p.q_over_m[k], p.q_weight[k], p.massive[k] = self.q_over_m[k], self.q_weight[k], self.massive[k]
        p.gamma_thr, p.eps_ph, p.tau, p.B0 = self.gamma_thr, self.eps_ph, self.tau, self.B0
        p.seed, p.capacity = self.seed, self.capacity
        return p


class Lines:
    """Device state of all lines (torch tensors) and the C struct view."""

    def __init__(self, cfg: Batch1DConfig, device="cuda"):
        import torch
        nl, n, cap = cfg.n_lines, cfg.n_cells, cfg.capacity
        self.cfg = cfg
        self.theta = torch.zeros(nl, dtype=torch.float64, device=device)
        self.I0 = torch.zeros(nl, dtype=torch.float64, device=device)
        self.D = torch.zeros(nl, n, dtype=torch.float32, device=device)
        self.JA = torch.zeros(nl, n + 2, dtype=torch.float32, device=device)
        self.count = torch.zeros(nl, dtype=torch.int32, device=device)
        self.events = torch.zeros(3, dtype=torch.int64, device=device)
        self.buf = []
        for _ in range(2):
            self.buf.append(dict(cell=torch.zeros(nl, cap, dtype=torch.int32, device=device),
                                 off=torch.zeros(nl, cap, dtype=torch.float32, device=device),
                                 ur=torch.zeros(nl, cap, dtype=torch.float32, device=device),
                                 up=torch.zeros(nl, cap, dtype=torch.float32, device=device),
                                 tag=torch.zeros(nl, cap, dtype=torch.int32, device=device),
                                 id=torch.zeros(nl, cap, dtype=torch.int64, device=device)))
        self._c = LinesC()
        self._c.cur = 0
        self._refresh()

    def _refresh(self):
        c = self._c
        c.theta, c.I0, c.D, c.JA = (t.data_ptr() for t in (self.theta, self.I0, self.D, self.JA))
        c.count, c.events = self.count.data_ptr(), self.events.data_ptr()
        for b in range(2):
            c.cell[b] = self.buf[b]["cell"].data_ptr()
            c.off[b] = self.buf[b]["off"].data_ptr()
            c.ur[b] = self.buf[b]["ur"].data_ptr()
            c.up[b] = self.buf[b]["up"].data_ptr()
            c.tag[b] = self.buf[b]["tag"].data_ptr()
            c.id[b] = self.buf[b]["id"].data_ptr()

    @property
    def cur(self):
        return self._c.cur

    def set_line(self, k, cell, off, ur, up, tag, pid):
        """Write line k's particles into the current buffer (host arrays)."""
        import torch
        b = self.buf[self.cur]
        n = len(cell)
        if n > self.cfg.capacity:
            raise ValueError("capacity exceeded")
        dev = self.D.device
        b["cell"][k, :n] = torch.as_tensor(np.asarray(cell, np.int32), device=dev)
        b["off"][k, :n] = torch.as_tensor(np.asarray(off, np.float32), device=dev)
        b["ur"][k, :n] = torch.as_tensor(np.asarray(ur, np.float32), device=dev)
        b["up"][k, :n] = torch.as_tensor(np.asarray(up, np.float32), device=dev)
        b["tag"][k, :n] = torch.as_tensor(np.asarray(tag, np.uint32).view(np.int32), device=dev)
        b["id"][k, :n] = torch.as_tensor(np.asarray(pid, np.uint64).view(np.int64), device=dev)
        self.count[k] = n

    def line(self, k):
        """Line k's particles from the current buffer as numpy arrays."""
        b = self.buf[self.cur]
        n = int(self.count[k].item())
        return dict(cell=b["cell"][k, :n].cpu().numpy(), off=b["off"][k, :n].cpu().numpy(),
                    ur=b["ur"][k, :n].cpu().numpy(), up=b["up"][k, :n].cpu().numpy(),
                    tag=b["tag"][k, :n].cpu().numpy().view(np.uint32),
                    id=b["id"][k, :n].cpu().numpy().view(np.uint64))


import numpy as np  # noqa: E402  (used by Lines)


class Batch1D:
    """Owns one grpic_batch1d_ctx."""

    def __init__(self, cfg: Batch1DConfig):
        import torch
        torch.cuda.current_device()
        self.lib = load()
        _load_b1(self.lib)
        self.cfg = cfg
        self._p = cfg.c()
        h = C.c_void_p()
        st = self.lib.grpic_batch1d_init(C.byref(self._p), C.byref(h))
        if st != OK:
            raise GrpicError(st, "grpic_batch1d_init failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.grpic_batch1d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, L: Lines, stream=None):
        st = self.lib.grpic_batch1d_init_fields(self.h, C.byref(L._c), _stream(stream))
        if st != OK:
            raise GrpicError(st, "grpic_batch1d_init_fields")

    def run(self, L: Lines, nsteps, step0, stream=None):
        st = self.lib.grpic_batch1d_run(self.h, C.byref(L._c), nsteps, step0, _stream(stream))
        if st != OK:
            raise GrpicError(st, "grpic_batch1d_run")

    def run_graph(self, L: Lines, nsteps, step0, stream=None):
        st = self.lib.grpic_batch1d_run_graph(self.h, C.byref(L._c), nsteps, step0, _stream(stream))
        if st != OK:
            raise GrpicError(st, "grpic_batch1d_run_graph")

    def tune(self, L: Lines, trial_steps, step0, stream=None):
        done = C.c_int64()
        best = (C.c_int32 * 3)()
        st = self.lib.grpic_batch1d_tune(self.h, C.byref(L._c), trial_steps, step0, C.byref(done), best,
                                         _stream(stream))
        if st != OK:
            raise GrpicError(st, "grpic_batch1d_tune")
        return done.value, (best[0], best[1], best[2])

    def set_launch(self, threads: int, ctas_per_sm: int, ctas_per_line: int = 1):
        """Launch shape of later runs: threads per CTA, CTAs per SM, CTAs per
        line (2: a cluster of two CTAs shares each line)."""
        st = self.lib.grpic_batch1d_set_launch(self.h, threads, ctas_per_sm, ctas_per_line)
        if st != OK:
            raise GrpicError(st, "grpic_batch1d_set_launch")

    def sync(self, stream=None):
        return self.lib.grpic_batch1d_sync(self.h, _stream(stream))


# ---------------------------------------------------------------------------
# differentiable form: horizon Poynting flux and its adjoint (FP64 contexts)
# ---------------------------------------------------------------------------
EXPORTS += ["grpic_horizon_flux", "grpic_adjoint_field_step", "grpic_adjoint_grad", "grpic_adjoint_spin",
            "grpic_horizon_index"]


def _load_adj(lib):
    v, p = C.c_void_p, C.POINTER
    for name, args in {"grpic_horizon_flux": [v, p(FieldsC), C.c_int, p(C.c_double), v],
                       "grpic_adjoint_field_step": [v, p(FieldsC), p(FieldsC), v],
                       "grpic_adjoint_grad": [v, p(ParticlesC), p(FieldsC), C.c_int, C.c_int, C.c_int,
                                              C.c_int, p(C.c_double), v, v, v, v],
                       "grpic_adjoint_spin": [v, p(ParticlesC), C.c_int, C.c_double, C.c_int, C.c_int, C.c_int,
                                              C.c_int, p(C.c_double), v, v, p(C.c_double), v],
                       "grpic_horizon_index": [v, C.c_double, p(C.c_int32)]}.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int


def horizon_index(gctx: "Context", a_nominal: float | None = None) -> int:
    """Column nearest the outer horizon of spin a_nominal (default: the
    context's spin), from the library (grpic_horizon_index)."""
    _load_adj(gctx.lib)
    out = C.c_int32()
    a = gctx.cfg.a if a_nominal is None else a_nominal
    gctx._check(gctx.lib.grpic_horizon_index(gctx.h, float(a), C.byref(out)), "grpic_horizon_index")
    return out.value


def _fields_of(D, B, ld, J=None):
    f = FieldsC()
    for k in range(3):
        f.D[k] = D[k].data_ptr()
        f.B[k] = B[k].data_ptr()
        f.J[k] = J[k].data_ptr() if J is not None else 0
    f.ld = ld
    return f


def horizon_flux(gctx: Context, F: Fields, i_horizon: int, stream=None) -> float:
    """flux(F) = sum_j (E_th H_ph - E_ph H_th)(r_iH, theta_{j+1/2}) dtheta."""
    _load_adj(gctx.lib)
    out = C.c_double()
    fc = F.c()
    gctx._check(gctx.lib.grpic_horizon_flux(gctx.h, C.byref(fc), int(i_horizon), C.byref(out), _stream(stream)),
                "grpic_horizon_flux")
    return out.value


def adjoint_field_step(gctx: Context, lam: Fields, stream=None) -> Fields:
    """Transpose of one field update: returns a Fields holding the adjoint of
    the fields before the update (D, B) and of the integrated currents (J)."""
    _load_adj(gctx.lib)
    out = Fields(gctx.cfg, device=lam.D[0].device, ld=lam.ld)
    fi, fo = lam.c(), out.c()
    gctx._check(gctx.lib.grpic_adjoint_field_step(gctx.h, C.byref(fi), C.byref(fo), _stream(stream)),
                "grpic_adjoint_field_step")
    return out


def adjoint_grad(gctx: Context, x, tag, D, B, nsteps: int, i_horizon: int, checkpoint_every: int = 20,
                 want_grad: bool = True, ift: bool = False, want_spin: bool = False, stream=None):
    """Objective L of nsteps steps from particles x = (r, theta, u_r, u_theta,
    u_phi) (five float64 device tensors of n), tag (int32 tensor of n) and
    fields D, B (three (n_theta+1, ld) float64 tensors each).  Returns L and,
    if want_grad, the gradients (five tensors like x, six like D + B).
    ift=True differentiates the converged geodesic trapezoid (implicit-function
    theorem) instead of the correctors the push runs.  want_spin=True (needs
    want_grad) appends dL/da at fixed step-0 particles and fields (grid, dt
    and i_horizon fixed) as a fourth result."""
    import torch
    _load_adj(gctx.lib)
    n = int(x[0].numel())
    ld = int(D[0].shape[1])
    xs = [t.contiguous() for t in x]
    pc = ParticlesC()
    pc.n, pc.capacity, pc.d_count = n, max(n, 1), 0
    pc.x1, pc.x2, pc.u1, pc.u2, pc.u3 = (t.data_ptr() for t in xs)
    pc.tag = tag.data_ptr()
    pc.cell = 0
    Dc = [t.contiguous() for t in D]
    Bc = [t.contiguous() for t in B]
    fc = _fields_of(Dc, Bc, ld)
    L = C.c_double()
    gp = gf = None
    if want_grad:
        gp = [torch.empty_like(t) for t in xs]
        gf = [torch.empty_like(t) for t in Dc + Bc]
        arr_p = (C.c_void_p * 5)(*[t.data_ptr() for t in gp])
        arr_f = (C.c_void_p * 6)(*[t.data_ptr() for t in gf])
    else:
        arr_p = arr_f = None
    if want_spin and not want_grad:
        raise ValueError("want_spin needs want_grad")
    La = C.c_double()
    st = gctx.lib.grpic_adjoint_grad(gctx.h, C.byref(pc), C.byref(fc), int(nsteps), int(checkpoint_every),
                                     int(i_horizon), 1 if ift else 0, C.byref(L), arr_p, arr_f,
                                     C.byref(La) if want_spin else None, _stream(stream))
    gctx._check(st, "grpic_adjoint_grad")
    if want_spin:
        return L.value, gp, gf, La.value
    return L.value, gp, gf


def spin_gradient(gctx: "Context", x, tag, kind: int, B0: float, nsteps: int, i_horizon: int,
                  checkpoint_every: int = 20, ift: bool = False, stream=None):
    """dL/da for a run that starts from the closed-form fields `kind`, B0 of
    the context's spin (grid, dt and i_horizon held fixed): the library's
    grpic_adjoint_spin, the adjoint's part at fixed step-0 state plus the
    step-0 fields' own a-dependence.  Returns (L, dL/da, grad_p, grad_f)."""
    import torch
    _load_adj(gctx.lib)
    n = int(x[0].numel())
    xs = [t.contiguous() for t in x]
    pc = ParticlesC()
    pc.n, pc.capacity, pc.d_count = n, max(n, 1), 0
    pc.x1, pc.x2, pc.u1, pc.u2, pc.u3 = (t.data_ptr() for t in xs)
    pc.tag = tag.data_ptr()
    pc.cell = 0
    cfg = gctx.cfg
    gp = [torch.empty_like(t) for t in xs]
    gf = [torch.empty((cfg.n_theta + 1, cfg.ld), dtype=torch.float64, device=xs[0].device) for _ in range(6)]
    arr_p = (C.c_void_p * 5)(*[t.data_ptr() for t in gp])
    arr_f = (C.c_void_p * 6)(*[t.data_ptr() for t in gf])
    L, La = C.c_double(), C.c_double()
    st = gctx.lib.grpic_adjoint_spin(gctx.h, C.byref(pc), int(kind), float(B0), int(nsteps), int(checkpoint_every),
                                     int(i_horizon), 1 if ift else 0, C.byref(L), arr_p, arr_f, C.byref(La),
                                     _stream(stream))
    gctx._check(st, "grpic_adjoint_spin")
    return L.value, La.value, gp, gf


def _autograd_fn():
    import torch

    class HorizonFluxFn(torch.autograd.Function):
        """L = horizon flux objective; inputs: the five particle state
        tensors and the six field tensors at step 0.  The gradient comes from
        the hand-written adjoint (grpic_adjoint_grad), evaluated in the
        forward pass when any input needs it."""

        @staticmethod
        def forward(fctx, gctx, tag, nsteps, i_horizon, checkpoint_every, ift, *xs):
            need = any(fctx.needs_input_grad[6:])
            L, gp, gf = adjoint_grad(gctx, list(xs[:5]), tag, list(xs[5:8]), list(xs[8:11]), nsteps, i_horizon,
                                     checkpoint_every, want_grad=need, ift=ift)
            if need:
                fctx.save_for_backward(*(gp + gf))
            return torch.tensor(L, dtype=torch.float64, device=xs[0].device)

        @staticmethod
        def backward(fctx, gL):
            g = fctx.saved_tensors
            return (None,) * 6 + tuple(gL * t for t in g)

    return HorizonFluxFn


_HFN = None


def horizon_flux_objective(gctx: Context, x, tag, D, B, nsteps: int, i_horizon: int, checkpoint_every: int = 20,
                           ift: bool = False):
    """Differentiable L(x, D, B) (torch scalar); backward() fills .grad of the
    inputs that require it through the adjoint."""
    global _HFN
    if _HFN is None:
        _HFN = _autograd_fn()
    return _HFN.apply(gctx, tag, int(nsteps), int(i_horizon), int(checkpoint_every), bool(ift), *x, *D, *B)
