"""GPU tests of the differentiable form: the hand-written adjoint of push +
deposit + field update for the time-averaged horizon Poynting flux L, through
the C ABI (grpic_adjoint_field_step, grpic_adjoint_grad, grpic_horizon_flux).

  * dot-product test of the transposed field update: it is linear, so
    <lam, F(X, J)> = <F^T lam, (X, J)> for random X, J, lam;
  * the forward objective matches the oracle's (64^2, 1e4 particles, 20 steps);
  * directional derivatives of L (random directions in the initial momenta,
    positions and fields, and the Wald strength B0) match central finite
    differences of the GPU forward and of the oracle's FP64 objective;
  * dL/da (the spin) matches central differences of L in a with the grid, dt
    and i_H held, both at fixed initial fields (the adjoint's own part) and
    with the Wald fields of each spin (its part plus grad_F0 . dF0/da);
  * the gradient does not depend on the checkpoint interval;
  * the torch.autograd.Function hands the same gradients to .grad.

The default adjoint transposes the predictor and correctors the push runs,
so it is the gradient of the computed trajectory; the implicit-function-theorem
mode differentiates the converged trapezoid and is checked where the
iteration converges (away from the polar axis, many correctors).  Central
differences of the particle terms see the kinks of the piecewise-linear CIC
weights when a perturbed path crosses a cell boundary or centre, which bounds
the agreement with them to ~1e-6 relative here."""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
from gpu_common import configs, relerr, axis_grazers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

A09 = 0.9
RH = 1.0 + math.sqrt(1 - A09 * A09)
NSTEPS = 20


@pytest.fixture(scope="module")
def G():
    from paper_2503_04558_gb300 import build, grpic
    build.build()
    grpic.load()
    return grpic


def host(t):
    return t.detach().cpu().numpy()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n_iter,damp", [(7, 0.1), (1, 0.0), (3, 0.1)])
def test_field_step_transpose_dot_product(G, n_iter, damp):
    oc, gc = configs(40, 32, A09, 0.9 * RH, 30.0, n_fld_iter=n_iter, damp_max=damp)
    ctx = G.Context(gc)
    rng = np.random.default_rng(11 + n_iter)
    X = G.Fields(gc, ld=gc.ld + 3)   # a wider stride: columns the update never touches
    for arr in X.D + X.B + X.J:
        arr.copy_(torch.from_numpy(rng.normal(size=tuple(arr.shape))))
    x0 = [host(t).copy() for t in X.D + X.B + X.J]
    ctx.field_update(X)
    assert ctx.sync() == 0
    y = [host(t) for t in X.D + X.B]
    lam = G.Fields(gc, ld=X.ld)
    for arr in lam.D + lam.B:
        arr.copy_(torch.from_numpy(rng.normal(size=tuple(arr.shape))))
    lam_h = [host(t) for t in lam.D + lam.B]
    out = G.adjoint_field_step(ctx, lam)
    g = [host(t) for t in out.D + out.B + out.J]
    lhs = sum(float(np.sum(a * b)) for a, b in zip(lam_h, y))
    rhs = sum(float(np.sum(a * b)) for a, b in zip(g, x0))
    scale = math.sqrt(sum(float(np.sum(a * a)) for a in lam_h) * sum(float(np.sum(a * a)) for a in y))
    assert abs(lhs - rhs) < 1e-12 * scale, (lhs, rhs, scale)


# ---------------------------------------------------------------------------
# the reduced case: 64^2, a = 0.9, Wald B0 = 1, 1e4 particles, 20 steps
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def case(G):
    from paper_2503_04558_gb300 import synth
    oc, gc = configs(64, 64, A09, 0.9 * RH, 20.0)
    ctx = G.Context(gc)
    F = G.Fields(gc)
    ctx.init_fields(F, O.WALD, 1.0)
    D, B = O.init_fields(oc, O.WALD, 1.0)
    P = O.Particles(*synth.particles(oc.nr, oc.nth, oc.r_in, oc.r_out, 10000, seed=0, sigma=0.1))
    graz = axis_grazers(oc, P, D, B, NSTEPS)
    P = P.take(np.setdiff1d(np.arange(P.n), graz))
    iH = O.horizon_index(oc, A09)
    assert iH == G.horizon_index(ctx)
    x = [dev(a) for a in (P.r, P.th, P.u1, P.u2, P.u3)]
    tag = dev(P.tag.view(np.int32))
    L, gp, gf = G.adjoint_grad(ctx, x, tag, F.D, F.B, NSTEPS, iH)
    return dict(oc=oc, gc=gc, ctx=ctx, F=F, D=D, B=B, P=P, iH=iH, x=x, tag=tag, L=L, gp=gp, gf=gf)


def gpu_L(G, c, x=None, D=None, B=None):
    x = c["x"] if x is None else x
    D = c["F"].D if D is None else D
    B = c["F"].B if B is None else B
    return G.adjoint_grad(c["ctx"], x, c["tag"], D, B, NSTEPS, c["iH"], want_grad=False)[0]


def test_objective_matches_oracle(G, case):
    ref = O.flux_run(case["oc"], case["P"], case["D"], case["B"], NSTEPS, case["iH"])
    assert case["L"] == pytest.approx(ref, rel=1e-10, abs=0)
    assert gpu_L(G, case) == pytest.approx(case["L"], rel=1e-12)


def test_horizon_flux_matches_oracle(G, case):
    v = G.horizon_flux(case["ctx"], case["F"], case["iH"])
    assert v == pytest.approx(O.horizon_flux(case["oc"], case["D"], case["B"], case["iH"]), rel=1e-12)


def directional(G, c, which, h, rng):
    """(adjoint prediction, GPU central difference, oracle central difference)."""
    if which in ("u", "x"):
        idx = (2, 3, 4) if which == "u" else (0, 1)
        dirs = {}
        for k in idx:
            scale = 0.1 * (1.0 if k == 2 else (c["P"].r if k == 3 else c["P"].r * np.sin(c["P"].th))) \
                if which == "u" else (1e-2 * c["P"].r if k == 0 else 1e-2)
            dirs[k] = rng.standard_normal(c["P"].n) * scale
        pred = sum(float(np.sum(host(c["gp"][k]) * d)) for k, d in dirs.items())

        def shifted(s):
            xs = [t.clone() for t in c["x"]]
            for k, d in dirs.items():
                xs[k] += s * dev(d)
            return xs

        def oracle_P(s):
            arrs = [c["P"].r, c["P"].th, c["P"].u1, c["P"].u2, c["P"].u3]
            arrs = [a + s * dirs[k] if k in dirs else a for k, a in enumerate(arrs)]
            return O.Particles(*arrs, c["P"].tag)

        fd = (gpu_L(G, c, x=shifted(h)) - gpu_L(G, c, x=shifted(-h))) / (2 * h)
        fo = (O.flux_run(c["oc"], oracle_P(h), c["D"], c["B"], NSTEPS, c["iH"]) -
              O.flux_run(c["oc"], oracle_P(-h), c["D"], c["B"], NSTEPS, c["iH"])) / (2 * h)
        return pred, fd, fo
    if which == "F":
        base = [host(t) for t in c["F"].D + c["F"].B]
        dirs = [rng.standard_normal(a.shape) * (np.abs(a).max() + 1e-3) for a in base]
        pred = sum(float(np.sum(host(g) * d)) for g, d in zip(c["gf"], dirs))

        def Fs(s):
            return [dev(a + s * d) for a, d in zip(base, dirs)]

        fp, fm = Fs(h), Fs(-h)
        fd = (gpu_L(G, c, D=fp[:3], B=fp[3:]) - gpu_L(G, c, D=fm[:3], B=fm[3:])) / (2 * h)
        Do = lambda s: [a + s * d for a, d in zip(c["D"], dirs[:3])]
        Bo = lambda s: [a + s * d for a, d in zip(c["B"], dirs[3:])]
        fo = (O.flux_run(c["oc"], c["P"], Do(h), Bo(h), NSTEPS, c["iH"]) -
              O.flux_run(c["oc"], c["P"], Do(-h), Bo(-h), NSTEPS, c["iH"])) / (2 * h)
        return pred, fd, fo
    # the Wald strength B0: the initial fields are linear in it
    pred = sum(float(np.sum(host(g) * host(f))) for g, f in zip(c["gf"], c["F"].D + c["F"].B))
    Fp, Fm = G.Fields(c["gc"]), G.Fields(c["gc"])
    c["ctx"].init_fields(Fp, O.WALD, 1.0 + h)
    c["ctx"].init_fields(Fm, O.WALD, 1.0 - h)
    fd = (gpu_L(G, c, D=Fp.D, B=Fp.B) - gpu_L(G, c, D=Fm.D, B=Fm.B)) / (2 * h)
    Dp, Bp = O.init_fields(c["oc"], O.WALD, 1.0 + h)
    Dm, Bm = O.init_fields(c["oc"], O.WALD, 1.0 - h)
    fo = (O.flux_run(c["oc"], c["P"], Dp, Bp, NSTEPS, c["iH"]) -
          O.flux_run(c["oc"], c["P"], Dm, Bm, NSTEPS, c["iH"])) / (2 * h)
    return pred, fd, fo


@pytest.mark.parametrize("which,h", [("u", 1e-6), ("x", 1e-6), ("F", 1e-6), ("B0", 1e-6)])
def test_gradient_matches_finite_differences(G, case, which, h):
    rng = np.random.default_rng({"u": 1, "x": 2, "F": 3, "B0": 4}[which])
    pred, fd, fo = directional(G, case, which, h, rng)
    print(f"{which}: adjoint {pred:.12e} gpu-fd {fd:.12e} oracle-fd {fo:.12e} "
          f"rel {abs(pred - fd) / abs(fd):.2e} {abs(pred - fo) / abs(fo):.2e}")
    assert abs(pred - fd) <= 2e-6 * abs(fd)
    assert abs(pred - fo) <= 2e-6 * abs(fo)


def test_spin_gradient_matches_finite_differences(G, case):
    h = 1e-6
    oc, gc = case["oc"], case["gc"]
    L, gp, gf, La = G.adjoint_grad(case["ctx"], case["x"], case["tag"], case["F"].D, case["F"].B, NSTEPS,
                                   case["iH"], want_spin=True)
    assert L == pytest.approx(case["L"], rel=1e-13)
    for a, b in zip(gp + gf, case["gp"] + case["gf"]):
        assert relerr(host(a), host(b)) < 1e-12

    def gpu_at(da, fixed_fields):
        c = dataclasses.replace(gc, a=A09 + da)
        ctx = G.Context(c)
        F = case["F"] if fixed_fields else G.Fields(c)
        if not fixed_fields:
            ctx.init_fields(F, O.WALD, 1.0)
        return G.adjoint_grad(ctx, case["x"], case["tag"], F.D, F.B, NSTEPS, case["iH"], want_grad=False)[0]

    def oracle_at(da, fixed_fields):
        o = O.make_cfg(oc.nr, oc.nth, A09 + da, oc.r_in, oc.r_out, dt=oc.dt, damp_cells=oc.damp_cells)
        D, B = (case["D"], case["B"]) if fixed_fields else O.init_fields(o, O.WALD, 1.0)
        return O.flux_run(o, case["P"], D, B, NSTEPS, case["iH"])

    # the adjoint's own part: metric of the pushes, tables of the updates and the flux
    fd = (gpu_at(h, True) - gpu_at(-h, True)) / (2 * h)
    fo = (oracle_at(h, True) - oracle_at(-h, True)) / (2 * h)
    print(f"dL/da at fixed F0: adjoint {La:.12e} gpu-fd {fd:.12e} oracle-fd {fo:.12e}")
    assert abs(La - fd) <= 2e-6 * abs(fd)
    assert abs(La - fo) <= 2e-6 * abs(fo)
    # with the initial Wald fields of each spin
    L2, dLda, gp2, gf2 = G.spin_gradient(case["ctx"], case["x"], case["tag"], O.WALD, 1.0, NSTEPS, case["iH"])
    assert L2 == pytest.approx(case["L"], rel=1e-13)
    for a, b in zip(gp2 + gf2, case["gp"] + case["gf"]):
        assert relerr(host(a), host(b)) < 1e-12
    fd = (gpu_at(h, False) - gpu_at(-h, False)) / (2 * h)
    fo = (oracle_at(h, False) - oracle_at(-h, False)) / (2 * h)
    print(f"dL/da: adjoint {dLda:.12e} gpu-fd {fd:.12e} oracle-fd {fo:.12e}")
    assert abs(dLda - fd) <= 2e-6 * abs(fd)
    assert abs(dLda - fo) <= 2e-6 * abs(fo)
    # checkpointing leaves it unchanged
    La7 = G.adjoint_grad(case["ctx"], case["x"], case["tag"], case["F"].D, case["F"].B, NSTEPS, case["iH"],
                         checkpoint_every=7, want_spin=True)[3]
    assert La7 == pytest.approx(La, rel=1e-10)


def test_gradient_independent_of_checkpoint_interval(G, case):
    for ck in (1, 7):
        L, gp, gf = G.adjoint_grad(case["ctx"], case["x"], case["tag"], case["F"].D, case["F"].B, NSTEPS,
                                   case["iH"], checkpoint_every=ck)
        assert L == pytest.approx(case["L"], rel=1e-13)
        for a, b in zip(gp, case["gp"]):
            assert relerr(host(a), host(b)) < 1e-10
        for a, b in zip(gf, case["gf"]):
            assert relerr(host(a), host(b)) < 1e-10


def test_autograd_function(G, case):
    x = [t.clone().requires_grad_(k >= 2) for k, t in enumerate(case["x"])]
    B0 = torch.tensor(1.0, dtype=torch.float64, device="cuda", requires_grad=True)
    unit = [t.clone() for t in case["F"].D + case["F"].B]   # the Wald field of B0 = 1
    F0 = [B0 * t for t in unit]
    L = G.horizon_flux_objective(case["ctx"], x, case["tag"], F0[:3], F0[3:], NSTEPS, case["iH"])
    L.backward()
    assert L.item() == pytest.approx(case["L"], rel=1e-13)
    for k in (2, 3, 4):
        assert relerr(host(x[k].grad), host(case["gp"][k])) < 1e-10
    ref = sum(float(np.sum(host(g) * host(f))) for g, f in zip(case["gf"], unit))
    assert float(B0.grad) == pytest.approx(ref, rel=1e-10)
    with torch.no_grad():
        L2 = G.horizon_flux_objective(case["ctx"], case["x"], case["tag"], case["F"].D, case["F"].B, NSTEPS,
                                      case["iH"])
    assert float(L2) == pytest.approx(case["L"], rel=1e-13)


def test_ift_mode_matches_the_converged_iteration(G):
    """Away from the axis and with enough correctors the trapezoid has
    converged: the implicit-function-theorem gradient equals the unrolled one
    and the central differences of L."""
    from paper_2503_04558_gb300 import synth
    oc, gc = configs(48, 48, A09, 0.9 * RH, 20.0, n_push_iter=12)
    ctx = G.Context(gc)
    F = G.Fields(gc)
    ctx.init_fields(F, O.WALD, 1.0)
    P = O.Particles(*synth.particles(oc.nr, oc.nth, oc.r_in, oc.r_out, 4000, seed=5, sigma=0.1))
    P = P.take(np.nonzero((P.th > 0.4) & (P.th < math.pi - 0.4))[0])
    iH = O.horizon_index(oc, A09)
    x = [dev(a) for a in (P.r, P.th, P.u1, P.u2, P.u3)]
    tag = dev(P.tag.view(np.int32))
    L0, g0, f0, a0 = G.adjoint_grad(ctx, x, tag, F.D, F.B, 10, iH, want_spin=True)
    L1, g1, f1, a1 = G.adjoint_grad(ctx, x, tag, F.D, F.B, 10, iH, ift=True, want_spin=True)
    assert L1 == pytest.approx(L0, rel=1e-13)   # the deposit's atomics may order sums differently
    assert a1 == pytest.approx(a0, rel=1e-8)
    errs = [relerr(host(a), host(b)) for a, b in zip(g1 + f1, g0 + f0)]
    print("ift vs unrolled:", " ".join(f"{e:.1e}" for e in errs))
    assert max(errs) < 1e-8
    rng = np.random.default_rng(8)
    d = rng.standard_normal(P.n) * 0.1
    pred = float(np.sum(host(g1[2]) * d))
    h = 1e-6

    def Lof(s):
        xs = [t.clone() for t in x]
        xs[2] += s * dev(d)
        return G.adjoint_grad(ctx, xs, tag, F.D, F.B, 10, iH, want_grad=False)[0]

    fd = (Lof(h) - Lof(-h)) / (2 * h)
    assert abs(pred - fd) <= 2e-6 * abs(fd), (pred, fd)
