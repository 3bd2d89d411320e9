"""GPU adjoint (force-VJP kernel + checkpointed reverse leapfrog) against the
oracle's reverse sweep, against central finite differences, and through the
torch.autograd.Function wrapper."""

import numpy as np
import pytest

import oracle
from paper_2511_02655_gb300 import inputs
from helpers import assert_elem_close, to_dev, to_np

pytestmark = pytest.mark.gpu

# per-element bounds (relative, cancellation guard at 1e-3 of the rms element) of the
# gradients against the oracle's reverse sweep
FP64_TOL, MIX_TOL = 1e-11, 1e-4


def _small_case(n=96, seed=21):
    x, v, m = inputs.plummer(n, seed=seed)
    m = m * np.exp(0.3 * np.random.default_rng(seed).standard_normal(n))
    t = inputs.targets(n, seed=seed + 1)
    return x, v, m, t


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, MIX_TOL)])
@pytest.mark.parametrize("T,K", [(20, 5), (17, 4), (9, 1), (12, 12), (5, 8), (1, 1)])
def test_adjoint_matches_oracle_reverse_sweep(nb, prec, tol, T, K):
    import torch
    G, eps, dt = 1.0, 0.05, 5e-3
    x, v, m, t = _small_case()
    xT, vT, _, _ = oracle.kdk(x, v, m, G, eps, dt, T)
    lx, lv = 2 * (xT - t), 0.1 * np.random.default_rng(3).standard_normal(xT.shape)
    gx_o, gv_o, gm_o = oracle.adjoint(x, v, m, G, eps, dt, T, lx, lv)
    ctx = nb.nbody_init(G=G, eps=eps, dt=dt, precision=prec, n=len(m))
    xt, vt, mt, lxt, lvt = to_dev(x, v, m, lx, lv)
    gx, gv, gm = nb.nbody_adjoint(ctx, xt, vt, mt, T, K, lxt, lvt)
    nb.nbody_sync(ctx)
    gx, gv, gm = to_np(gx, gv, gm)
    assert_elem_close(gx, gx_o, tol, "g_x0")
    assert_elem_close(gv, gv_o, tol, "g_v0")
    assert_elem_close(gm, gm_o, tol, "g_m")
    # inputs untouched
    assert np.array_equal(xt.cpu().numpy(), x) and np.array_equal(vt.cpu().numpy(), v)


def test_adjoint_zero_steps_is_identity(nb):
    x, v, m, t = _small_case(16)
    ctx = nb.nbody_init(G=1.0, eps=0.05, dt=1e-3, precision=nb.MIXED, n=16)
    lx, lv = np.ones((16, 3)), 2 * np.ones((16, 3))
    gx, gv, gm = nb.nbody_adjoint(ctx, *to_dev(x, v, m), 0, 3, *to_dev(lx, lv))
    gx, gv, gm = to_np(gx, gv, gm)
    assert np.array_equal(gx, lx) and np.array_equal(gv, lv) and np.all(gm == 0)


def test_adjoint_several_systems(nb):
    sizes = [7, 130, 0, 300]
    ens = inputs.ensemble(len(sizes), seed=5, sizes=np.array(sizes))
    off = [int(o) for o in ens.offsets]
    G, eps, dt, T, K = 1.0, 0.05, 4e-3, 10, 3
    t = inputs.targets(off[-1], seed=6)
    ctx = nb.nbody_init(G=G, eps=eps, dt=dt, precision=nb.FP64, offsets=off)
    lx_all = np.zeros((off[-1], 3))
    for s in range(len(sizes)):
        b, e = off[s], off[s + 1]
        if e > b:
            xT, _, _, _ = oracle.kdk(ens.x[b:e], ens.v[b:e], ens.m[b:e], G, eps, dt, T)
            lx_all[b:e] = 2 * (xT - t[b:e])
    gx, gv, gm = nb.nbody_adjoint(ctx, *to_dev(ens.x, ens.v, ens.m), T, K, *to_dev(lx_all, np.zeros_like(lx_all)))
    gx, gv, gm = to_np(gx, gv, gm)
    for s in range(len(sizes)):
        b, e = off[s], off[s + 1]
        if e == b:
            continue
        ox, ov, om = oracle.adjoint(ens.x[b:e], ens.v[b:e], ens.m[b:e], G, eps, dt, T, lx_all[b:e],
                                    np.zeros((e - b, 3)))
        assert_elem_close(gx[b:e], ox, FP64_TOL, f"g_x0 system {s}")
        assert_elem_close(gv[b:e], ov, FP64_TOL, f"g_v0 system {s}")
        assert_elem_close(gm[b:e], om, FP64_TOL, f"g_m system {s}")


@pytest.mark.parametrize("prec", [0, 1])
def test_autograd_function(nb, prec):
    import torch
    G, eps, dt, T, K = 1.0, 0.05, 5e-3, 12, 5
    x, v, m, t = _small_case(64, seed=40)
    ctx = nb.nbody_init(G=G, eps=eps, dt=dt, precision=prec, n=64)
    xt, vt, mt, tt = to_dev(x, v, m, t)
    x0 = xt.clone().requires_grad_(True)
    v0 = vt.clone().requires_grad_(True)
    m0 = mt.clone().requires_grad_(True)
    xT, vT = nb.NBodyAdjoint.apply(ctx, x0, v0, m0, T, K)
    loss = ((xT - tt) ** 2).sum() + 0.5 * (vT ** 2).sum()
    loss.backward()
    # the forward equals nbody_step, the backward equals nbody_adjoint
    xs, vs, a = xt.clone(), vt.clone(), torch.empty_like(xt)
    nb.nbody_step(ctx, xs, vs, mt, a, False, T)
    assert torch.equal(xs, xT.detach()) and torch.equal(vs, vT.detach())
    gx, gv, gm = nb.nbody_adjoint(ctx, xt, vt, mt, T, K, 2 * (xs - tt), vs.clone())
    for g, ref in ((gx, x0.grad), (gv, v0.grad), (gm, m0.grad)):
        assert torch.allclose(g, ref, rtol=1e-14, atol=0)
    ox, ov, om = oracle.adjoint(x, v, m, G, eps, dt, T, 2 * (xs.cpu().numpy() - t), vs.cpu().numpy())
    tol = FP64_TOL if prec == 0 else MIX_TOL
    assert_elem_close(x0.grad.cpu().numpy(), ox, tol, "x0.grad")
    assert_elem_close(v0.grad.cpu().numpy(), ov, tol, "v0.grad")
    assert_elem_close(m0.grad.cpu().numpy(), om, tol, "m.grad")


@pytest.mark.slow
def test_adjoint_n16384_200_steps_vs_finite_differences(nb):
    """N = 16384 Plummer, 200 KDK steps, dt = 1e-3, checkpoints every 20 steps; loss = sum |x_T - t|^2.
    FP64 and mixed adjoint gradients vs FP64 central differences (h = 1e-6) on 32 coordinates
    (12 positions, 12 velocities, 8 masses), relative error <= 1e-4."""
    import torch
    n, G, eps, dt, T, K = 16384, 1.0, 0.01, 1e-3, 200, 20
    x, v, m = inputs.plummer(n, seed=5)
    t = inputs.targets(n, seed=6)
    rng = np.random.default_rng(7)
    pos = [(int(i), int(c)) for i, c in zip(rng.choice(n, 12, replace=False), rng.integers(0, 3, 12))]
    vel = [(int(i), int(c)) for i, c in zip(rng.choice(n, 12, replace=False), rng.integers(0, 3, 12))]
    mas = [int(i) for i in rng.choice(n, 8, replace=False)]
    tt = to_dev(t)[0]
    # FD systems: 64 perturbed copies advanced together as one batched FP64 ensemble
    h = 1e-6
    copies_x, copies_v, copies_m = [], [], []
    for kind, items in (("x", pos), ("v", vel), ("m", [(i, None) for i in mas])):
        for i, c in items:
            for sgn in (1.0, -1.0):
                xx, vv, mm = x.copy(), v.copy(), m.copy()
                if kind == "x":
                    xx[i, c] += sgn * h
                elif kind == "v":
                    vv[i, c] += sgn * h
                else:
                    mm[i] += sgn * h
                copies_x.append(xx), copies_v.append(vv), copies_m.append(mm)
    nc = len(copies_x)
    off = [k * n for k in range(nc + 1)]
    ctxb = nb.nbody_init(G=G, eps=eps, dt=dt, precision=nb.FP64, offsets=off)
    xb, vb, mb = to_dev(np.concatenate(copies_x), np.concatenate(copies_v), np.concatenate(copies_m))
    ab = torch.empty_like(xb)
    nb.nbody_step(ctxb, xb, vb, mb, ab, False, T)
    nb.nbody_sync(ctxb)
    # L+ - L- = sum (x+ - x-) . (x+ + x- - 2t): differencing the trajectories first avoids the
    # cancellation of two ~5e4-sized sums
    xr = xb.view(nc, n, 3)
    dL = ((xr[0::2] - xr[1::2]) * (xr[0::2] + xr[1::2] - 2 * tt)).sum(dim=(1, 2)).cpu().numpy()
    fd = dL / (2 * h)
    ctxb.close()
    for prec in (nb.FP64, nb.MIXED):
        ctx = nb.nbody_init(G=G, eps=eps, dt=dt, precision=prec, n=n)
        xt, vt, mt = to_dev(x, v, m)
        xs, vs, a = xt.clone(), vt.clone(), torch.empty_like(xt)
        nb.nbody_step(ctx, xs, vs, mt, a, False, T)
        gx, gv, gm = nb.nbody_adjoint(ctx, xt, vt, mt, T, K, 2 * (xs - tt), torch.zeros_like(vs))
        nb.nbody_sync(ctx)
        gx, gv, gm = to_np(gx, gv, gm)
        ad = np.array([gx[i, c] for i, c in pos] + [gv[i, c] for i, c in vel] + [gm[i] for i in mas])
        err = np.abs(ad - fd) / np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())
        assert err.max() <= 1e-4, (prec, err.max(), np.argmax(err))
        ctx.close()


# --------------------------------------------------------------------------------------
# gradients with respect to G and eps (nbody_adjoint_params)


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, MIX_TOL)])
@pytest.mark.parametrize("T,K", [(20, 5), (9, 1), (5, 8)])
def test_adjoint_params_match_oracle(nb, prec, tol, T, K):
    import torch
    G, eps, dt = 1.3, 0.05, 5e-3
    x, v, m, t = _small_case(n=200, seed=31)
    xT, vT, _, _ = oracle.kdk(x, v, m, G, eps, dt, T)
    lx, lv = 2 * (xT - t), 0.1 * np.random.default_rng(4).standard_normal(xT.shape)
    gx_o, gv_o, gm_o, (gG_o, ge_o) = oracle.adjoint_params(x, v, m, G, eps, dt, T, lx, lv)
    ctx = nb.nbody_init(G=G, eps=eps, dt=dt, precision=prec, n=len(m))
    args = to_dev(x, v, m) + (T, K) + to_dev(lx, lv)
    gx, gv, gm, gp = nb.nbody_adjoint_params(ctx, *args)
    nb.nbody_sync(ctx)
    assert gp.shape == (1, 2)
    gG, ge = gp.cpu().numpy()[0]
    assert abs(gG - gG_o) <= tol * abs(gG_o) and abs(ge - ge_o) <= tol * abs(ge_o), (gG, gG_o, ge, ge_o)
    # the parameter sums leave the other gradients as nbody_adjoint computes them
    hx, hv, hm = nb.nbody_adjoint(ctx, *args)
    assert torch.equal(gx, hx) and torch.equal(gv, hv) and torch.equal(gm, hm)
    assert_elem_close(gx.cpu().numpy(), gx_o, tol, "g_x0")
    assert_elem_close(gv.cpu().numpy(), gv_o, tol, "g_v0")
    assert_elem_close(gm.cpu().numpy(), gm_o, tol, "g_m")


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, MIX_TOL)])
def test_adjoint_params_several_systems_and_mass_identity(nb, prec, tol):
    # per-system rows against the oracle, an empty system's row zero, and
    # G dL/dG = sum_j m_j dL/dm_j (G enters softened gravity only as G m_j) per system
    sizes = [7, 130, 0, 300]
    ens = inputs.ensemble(len(sizes), seed=8, sizes=np.array(sizes))
    off = [int(o) for o in ens.offsets]
    G, eps, dt, T, K = 0.8, 0.04, 4e-3, 10, 3
    t = inputs.targets(off[-1], seed=9)
    lx_all = np.zeros((off[-1], 3))
    for s in range(len(sizes)):
        b, e = off[s], off[s + 1]
        if e > b:
            xT, _, _, _ = oracle.kdk(ens.x[b:e], ens.v[b:e], ens.m[b:e], G, eps, dt, T)
            lx_all[b:e] = 2 * (xT - t[b:e])
    ctx = nb.nbody_init(G=G, eps=eps, dt=dt, precision=prec, offsets=off)
    gx, gv, gm, gp = nb.nbody_adjoint_params(ctx, *to_dev(ens.x, ens.v, ens.m), T, K,
                                             *to_dev(lx_all, np.zeros_like(lx_all)))
    nb.nbody_sync(ctx)
    gx, gv, gm, gp = to_np(gx, gv, gm, gp)
    for s in range(len(sizes)):
        b, e = off[s], off[s + 1]
        if e == b:
            assert np.all(gp[s] == 0)
            continue
        ox, ov, om, (oG, oe) = oracle.adjoint_params(ens.x[b:e], ens.v[b:e], ens.m[b:e], G, eps, dt, T,
                                                     lx_all[b:e], np.zeros((e - b, 3)))
        assert abs(gp[s, 0] - oG) <= tol * abs(oG) and abs(gp[s, 1] - oe) <= tol * abs(oe), (s, gp[s], oG, oe)
        assert_elem_close(gx[b:e], ox, tol, f"g_x0 system {s}")
        assert_elem_close(gv[b:e], ov, tol, f"g_v0 system {s}")
        assert_elem_close(gm[b:e], om, tol, f"g_m system {s}")
        assert abs(G * gp[s, 0] - (ens.m[b:e] * gm[b:e]).sum()) <= tol * abs(G * gp[s, 0])


def test_adjoint_params_rejects_null_and_lj(nb):
    x, v, m, t = _small_case(16)
    ctx = nb.nbody_init(G=1.0, eps=0.05, dt=1e-3, precision=nb.FP64, n=16)
    lib = nb.load()
    xt, vt, mt, lx = to_dev(x, v, m, np.ones((16, 3)))
    g = [lx.clone() for _ in range(2)] + [mt.clone()]
    ptr = lambda a: a.data_ptr()
    st = lib.nbody_adjoint_params(ctx._h, ptr(xt), ptr(vt), ptr(mt), 3, 1, ptr(lx), ptr(lx), ptr(g[0]), ptr(g[1]),
                                  ptr(g[2]), None)
    assert st == 1
    ctx2 = nb.nbody_init(law=nb.LENNARD_JONES, precision=nb.FP64, n=16, dt=1e-3)
    with pytest.raises(nb.NBodyError) as ei:
        nb.nbody_adjoint_params(ctx2, xt, vt, mt, 3, 1, lx, lx)
    assert ei.value.status == 6


@pytest.mark.slow
def test_adjoint_params_n16384_200_steps_vs_finite_differences(nb):
    """dL/dG and dL/deps at N = 16384 Plummer, 200 KDK steps, dt = 1e-3, checkpoints every 20,
    against FP64 central differences (relative step 1e-6) of the FP64 GPU trajectory; <= 1e-4."""
    import torch
    n, G, eps, dt, T, K = 16384, 1.0, 0.01, 1e-3, 200, 20
    x, v, m = inputs.plummer(n, seed=5)
    t = inputs.targets(n, seed=6)
    tt = to_dev(t)[0]

    def final_x(g, e):
        ctx = nb.nbody_init(G=g, eps=e, dt=dt, precision=nb.FP64, n=n)
        xs, vs, mt = to_dev(x, v, m)
        nb.nbody_step(ctx, xs, vs, mt, torch.empty_like(xs), False, T)
        nb.nbody_sync(ctx)
        ctx.close()
        return xs

    fd = []
    for gp, ep, gm_, em in ((G * (1 + 1e-6), eps, G * (1 - 1e-6), eps), (G, eps * (1 + 1e-6), G, eps * (1 - 1e-6))):
        xp, xm = final_x(gp, ep), final_x(gm_, em)
        dL = float(((xp - xm) * (xp + xm - 2 * tt)).sum())
        fd.append(dL / (gp - gm_ + ep - em))
    for prec in (nb.FP64, nb.MIXED):
        ctx = nb.nbody_init(G=G, eps=eps, dt=dt, precision=prec, n=n)
        xt, vt, mt = to_dev(x, v, m)
        xs, vs, a = xt.clone(), vt.clone(), torch.empty_like(xt)
        nb.nbody_step(ctx, xs, vs, mt, a, False, T)
        _, _, _, gp = nb.nbody_adjoint_params(ctx, xt, vt, mt, T, K, 2 * (xs - tt), torch.zeros_like(vs))
        nb.nbody_sync(ctx)
        ad = gp.cpu().numpy()[0]
        err = np.abs(ad - np.array(fd)) / np.abs(np.array(fd))
        assert err.max() <= 1e-4, (prec, ad, fd, err)
        ctx.close()


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("n,T,K", [(203, 12, 5), (64, 7, 7), (1, 3, 2), (517, 4, 1)])
def test_scalar_and_packed_vjp_match_oracle(nb, variant, n, T, K):
    """Both mixed VJP kernels (scalar float32, packed float32x2 over j-pairs with a padded,
    ragged last tile) against the oracle's reverse sweep, gradients and parameter gradients."""
    G, eps, dt = 1.1, 0.05, 5e-3
    x, v, m, t = _small_case(n, seed=50 + n)
    xT, vT, _, _ = oracle.kdk(x, v, m, G, eps, dt, T)
    lx, lv = 2 * (xT - t), 0.1 * np.random.default_rng(9).standard_normal(xT.shape)
    gx_o, gv_o, gm_o, (gG_o, ge_o) = oracle.adjoint_params(x, v, m, G, eps, dt, T, lx, lv)
    ctx = nb.nbody_init(G=G, eps=eps, dt=dt, precision=nb.MIXED, n=n, variant=variant)
    gx, gv, gm, gp = nb.nbody_adjoint_params(ctx, *to_dev(x, v, m), T, K, *to_dev(lx, lv))
    nb.nbody_sync(ctx)
    gx, gv, gm, gp = to_np(gx, gv, gm, gp)
    tol = MIX_TOL
    assert_elem_close(gx, gx_o, tol, "g_x0")
    assert_elem_close(gv, gv_o, tol, "g_v0")
    if n > 1:
        assert_elem_close(gm, gm_o, tol, "g_m")
        assert abs(gp[0, 0] - gG_o) <= tol * abs(gG_o)
        assert abs(gp[0, 1] - ge_o) <= tol * abs(ge_o), (gp, gG_o, ge_o)
    else:
        assert np.all(gm == 0) and np.all(gp == 0)


@pytest.mark.parametrize("variant", [1, 2])
def test_adjoint_tight_pairs_far_from_origin(nb, variant):
    """Tight pairs (separation ~ eps / 2) around |x| ~ 100, 10 KDK steps: float32 staging alone
    carries ~4e-6 absolute error in each coordinate, several % of the pair separation, and the
    pair terms of the force VJP (1/s^3, 1/s^5) would carry it into every gradient. Mixed
    gradients (x0, v0, m, G, eps) against the oracle's reverse sweep, per element."""
    rng = np.random.default_rng(11)
    npair, eps, G, dt, T, K = 200, 1e-3, 1.0, 1e-4, 10, 4
    centres = rng.normal(size=(npair, 3))
    centres = 100.0 * centres / np.linalg.norm(centres, axis=1, keepdims=True)
    x = np.concatenate([centres, centres + rng.normal(size=(npair, 3)) * 0.5 * eps])
    v = 0.05 * rng.normal(size=x.shape)
    m = np.full(2 * npair, 1e-3)
    xT, vT, _, _ = oracle.kdk(x, v, m, G, eps, dt, T)
    lx = 2 * (xT - inputs.targets(2 * npair, seed=12))
    lv = rng.normal(size=x.shape)
    gx_o, gv_o, gm_o, (gG_o, ge_o) = oracle.adjoint_params(x, v, m, G, eps, dt, T, lx, lv)
    ctx = nb.nbody_init(G=G, eps=eps, dt=dt, precision=nb.MIXED, n=2 * npair, variant=variant)
    gx, gv, gm, gp = nb.nbody_adjoint_params(ctx, *to_dev(x, v, m), T, K, *to_dev(lx, lv))
    nb.nbody_sync(ctx)
    gx, gv, gm, gp = to_np(gx, gv, gm, gp)
    assert_elem_close(gx, gx_o, MIX_TOL, "g_x0")
    assert_elem_close(gv, gv_o, MIX_TOL, "g_v0")
    assert_elem_close(gm, gm_o, MIX_TOL, "g_m")
    assert abs(gp[0, 0] - gG_o) <= MIX_TOL * abs(gG_o), (gp[0, 0], gG_o)
    assert abs(gp[0, 1] - ge_o) <= MIX_TOL * abs(ge_o), (gp[0, 1], ge_o)
