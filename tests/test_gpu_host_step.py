"""grpic_step_host: steps with the particle state resident in pinned host
memory (copied in, stepped, copied back every step, the two copy directions
overlapped chunk by chunk), against the same steps on device-resident
buffers.

  * FP64, 128^2 Wald, 2e5 particles, 4 steps: the host state equals the
    device-resident run's state (cells and tags bit for bit, positions and
    momenta to 1e-10: the currents are summed by atomics in either order);
  * FP32 form with the host fields copied in and out: the host fields after
    the call are the device fields bit for bit, and the call reports the
    bytes it copied;
  * FP32 form at 2.5e7 particles (two copy chunks): the host arrays are the
    device buffers' live slots bit for bit, and match a device-resident run;
  * radiation contexts are refused."""
import math

import numpy as np
import pytest

import oracle as O
from gpu_common import configs, relerr, fp32_offsets

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

A09 = 0.9
RH = 1.0 + math.sqrt(1 - A09 * A09)


@pytest.fixture(scope="module")
def G():
    from paper_2503_04558_gb300 import build, grpic
    build.build()
    grpic.load()
    return grpic


def state(oc, n, seed):
    from paper_2503_04558_gb300 import synth
    return O.Particles(*synth.particles(oc.nr, oc.nth, oc.r_in, oc.r_out, n, seed=seed, sigma=0.1))


def arrays(gc, oc, P):
    if gc.precision == 64:
        return (P.r, P.th, P.u1, P.u2, P.u3, P.tag, None)
    cell, o1, o2 = fp32_offsets(oc, P.r, P.th)
    f = np.float32
    return (o1, o2, P.u1.astype(f), P.u2.astype(f), P.u3.astype(f), P.tag, cell)


def fill_host(H, arrs):
    n = len(arrs[0])
    for t, a in zip(H.arrays(), arrs):
        if t is not None:
            t[:n].copy_(torch.from_numpy(np.ascontiguousarray(a)).view(t.dtype))
    H.n = n


def two_runs(G, gc, oc, P, nsteps, host_fields=False):
    """The device-resident run (ctx.step per step) and the host-resident one
    (one grpic_step_host call) from the same state."""
    out = []
    for mode in ("device", "host"):
        ctx = G.Context(gc)
        F = G.Fields(gc)
        ctx.init_fields(F, O.WALD, 1.0)
        S = G.ParticleSet(gc, P.n + 64)
        arrs = arrays(gc, oc, P)
        if mode == "device":
            S.load(*arrs)
            for _ in range(nsteps):
                ctx.step(S, F, 1)
            assert ctx.sync() == 0
            out.append(dict(ctx=ctx, F=F, S=S, n=S.live(), h=S.host()))
        else:
            H = G.HostParticles(gc, P.n + 64)
            fill_host(H, arrs)
            HF = None
            if host_fields:
                HF = G.HostFields(F)
                for hd, d in zip(HF.D + HF.B, F.D + F.B):
                    hd.copy_(d.cpu())
            nb = ctx.step_host(H, S, F, nsteps, host_fields=HF)
            torch.cuda.synchronize()
            assert ctx.sync() == 0
            out.append(dict(ctx=ctx, F=F, S=S, H=H, HF=HF, n=H.n, bytes=nb))
    return out


def host_dict(H):
    n = H.n
    keys = ("x1", "x2", "u1", "u2", "u3", "tag", "cell")
    out = {k: (t[:n].numpy().copy() if t is not None else None) for k, t in zip(keys, H.arrays())}
    out["tag"] = out["tag"].view(np.uint32)
    return out


def test_fp64_host_steps_match_device_steps(G):
    oc, gc = configs(128, 128, A09, 0.9 * RH, 50.0)
    P = state(oc, 200000, seed=3)
    dev, hst = two_runs(G, gc, oc, P, 4)
    assert hst["n"] == dev["n"]
    h, d = host_dict(hst["H"]), dev["h"]
    assert np.array_equal(h["tag"], d["tag"])
    Pg = O.Particles(h["x1"], h["x2"], h["u1"], h["u2"], h["u3"], h["tag"])
    Pd = O.Particles(d["x1"], d["x2"], d["u1"], d["u2"], d["u3"], d["tag"])
    assert np.array_equal(O.cell_keys(oc, Pg), O.cell_keys(oc, Pd))
    for k in ("x1", "x2", "u1", "u2", "u3"):
        assert relerr(h[k], d[k]) < 1e-10, k
    for x, y in zip(hst["F"].D + hst["F"].B, dev["F"].D + dev["F"].B):
        yy = y.cpu().numpy()
        assert relerr(x.cpu().numpy(), yy, floor=np.max(np.abs(yy))) < 1e-10


def test_fp32_host_fields_and_byte_counts(G):
    oc, gc = configs(128, 128, A09, 0.9 * RH, 50.0, precision=32)
    gc.fp64_radius = 1.5 * RH
    gc.push_tol = 1e-6
    P = state(oc, 200000, seed=4)
    dev, hst = two_runs(G, gc, oc, P, 3, host_fields=True)
    # the host fields are the device fields after the last step
    for hd, d in zip(hst["HF"].D + hst["HF"].B, hst["F"].D + hst["F"].B):
        assert torch.equal(hd, d.cpu())
    # bytes: 28 per slot each way per step (the live count before / after
    # the step), plus D and B both ways
    fbytes = 6 * (oc.nth + 1) * hst["F"].ld * 4
    b_in, b_out = hst["bytes"]
    assert b_in > 3 * fbytes and b_out > 3 * fbytes
    assert (b_in - 3 * fbytes) % 28 == 0 and (b_out - 3 * fbytes) % 28 == 0
    assert (b_out - 3 * fbytes) // 28 <= (b_in - 3 * fbytes) // 28
    n_last = (b_out - 3 * fbytes) // 28 - (b_in - 3 * fbytes) // 28 + P.n
    assert n_last == hst["n"]
    # and the state matches the device-resident run to FP32 rounding
    assert abs(hst["n"] - dev["n"]) <= 2
    h, d = host_dict(hst["H"]), dev["h"]
    m = min(len(h["cell"]), len(d["cell"]))
    assert np.mean(h["cell"][:m] == d["cell"][:m]) > 0.999
    for x, y in zip(hst["F"].D + hst["F"].B, dev["F"].D + dev["F"].B):
        yy = y.cpu().numpy().astype(np.float64)
        assert relerr(x.cpu().numpy().astype(np.float64), yy, floor=np.max(np.abs(yy))) < 1e-5


def test_fp32_host_steps_in_two_chunks(G):
    """2.5e7 particles: the slot range is copied in two chunks each way."""
    oc, gc = configs(1024, 1024, A09, 0.9 * RH, 50.0, precision=32)
    gc.fp64_radius = 1.5 * RH
    gc.push_tol = 1e-6
    n = 25_000_000
    assert n > (1 << 24)
    from paper_2503_04558_gb300 import synth
    ctx = G.Context(gc)
    F = G.Fields(gc)
    ctx.init_fields(F, O.WALD, 1.0)
    g = synth.particles_torch(oc.nr, oc.nth, oc.r_in, oc.r_out, n, seed=11, sigma=0.1, device="cuda")
    cell, o1, o2 = ctx.fp32_encode(g["r"], g["th"])
    arrs = [o1, o2, g["u1"].float(), g["u2"].float(), g["u3"].float(), g["tag"], cell]
    del g
    # device-resident reference run
    Sd = G.ParticleSet(gc, n + 64)
    Sd.load(*arrs)
    ctxd = G.Context(gc)
    Fd = G.Fields(gc)
    ctxd.init_fields(Fd, O.WALD, 1.0)
    for _ in range(2):
        ctxd.step(Sd, Fd, 1)
    assert ctxd.sync() == 0
    nd = Sd.live()
    # host-resident run
    H = G.HostParticles(gc, n + 64)
    for t, a in zip(H.arrays(), arrs):
        t[:n].copy_(a.cpu())
    H.n = n
    del arrs
    S = G.ParticleSet(gc, n + 64)
    b_in, b_out = ctx.step_host(H, S, F, 2)
    torch.cuda.synchronize()
    assert ctx.sync() == 0
    assert b_in >= 28 * n
    # the host arrays hold the device buffers' live slots
    assert H.n == S.live()
    for t, dvt in zip(H.arrays(), S.a.arrays()):
        assert torch.equal(t[:H.n], dvt[:H.n].cpu())
    # and agree with the device-resident run to FP32 rounding
    assert abs(H.n - nd) <= max(2, nd // 1000000)
    m = min(H.n, nd)
    agree = (H.cell[:m] == Sd.a.cell[:m].cpu()).float().mean().item()
    assert agree > 0.999
    for x, y in zip(F.D + F.B, Fd.D + Fd.B):
        yy = y.cpu().numpy().astype(np.float64)
        assert relerr(x.cpu().numpy().astype(np.float64), yy, floor=np.max(np.abs(yy))) < 1e-5


def test_radiation_context_is_refused(G):
    oc, gc = configs(32, 32, A09, 0.9 * RH, 20.0)
    gc.radiation = 1
    ctx = G.Context(gc)
    F = G.Fields(gc)
    ctx.init_fields(F, O.WALD, 1.0)
    S = G.ParticleSet(gc, 1024)
    H = G.HostParticles(gc, 1024)
    with pytest.raises(G.GrpicError):
        ctx.step_host(H, S, F, 1)
