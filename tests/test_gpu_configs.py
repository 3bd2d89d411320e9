"""GPU parity at the full sizes of the reference workloads, on sampled bodies
the oracle can compute one by one, plus properties that hold at any size.

* Plummer N = 65536, eps = 0.005, dt = 5e-4, 100 KDK steps, mixed beside FP64
* two Plummer spheres, N = 1 048 576, eps = 0.002, 10 steps, mixed
* 512 independent Plummer systems, N log-uniform in [64, 16384], eps = 0.01,
  dt = 1e-3, 50 steps, one persistent launch per step replayed as a CUDA graph
"""

import numpy as np
import pytest

import oracle
from paper_2511_02655_gb300 import inputs
from helpers import assert_elem_close, force_rel_err, to_dev, to_np

pytestmark = pytest.mark.gpu

MIX_MED, MIX_MAX, FP64_TOL = 1e-6, 1e-4, 1e-12
# the 1M two-sphere case: oracle forces on this many sampled bodies (each against all N)
SAMPLE_1M = 16384


def _sampled_err(x, m, a_gpu, G, eps, k=1024, seed=17):
    idx = inputs.sample_indices(len(m), k, seed)
    a_ref, _ = oracle.forces_at(x, m, idx, G=G, eps=eps)
    return force_rel_err(a_gpu[idx], a_ref)


def test_plummer_65536_mixed_and_fp64_100_steps(nb):
    import torch
    n, G, eps, dt, T = 65536, 1.0, 0.005, 5e-4, 100
    x, v, m = inputs.plummer(n, seed=2)
    runs = {}
    for prec in (nb.MIXED, nb.FP64):
        ctx = nb.nbody_init(G=G, eps=eps, dt=dt, precision=prec, n=n, energy_every=10)
        xt, vt, mt = to_dev(x, v, m)
        at = torch.empty_like(xt)
        nb.nbody_forces(ctx, xt, mt, at)
        e0 = _sampled_err(x, m, at.cpu().numpy(), G, eps)
        E0 = nb.nbody_energy(ctx, xt, vt, mt).cpu().numpy()[0]
        log = nb.nbody_step(ctx, xt, vt, mt, at, True, T)
        nb.nbody_sync(ctx)
        xf, vf, af = to_np(xt, vt, at)
        e1 = _sampled_err(xf, m, af, G, eps, seed=18)
        runs[prec] = (e0, e1, E0, log.cpu().numpy()[:, 0, :], xf, vf)
        ctx.close()
    for prec, (e0, e1, E0, log, xf, vf) in runs.items():
        if prec == nb.FP64:
            assert e0.max() <= FP64_TOL and e1.max() <= FP64_TOL
        else:
            assert np.median(e0) <= MIX_MED and e0.max() <= MIX_MAX
            assert np.median(e1) <= MIX_MED and e1.max() <= MIX_MAX
    # energy drift of the mixed run tracks the FP64 run (both leapfrog, same dt)
    dm = (runs[nb.MIXED][3][:, 0] - runs[nb.MIXED][2][0]) / abs(runs[nb.MIXED][2][0])
    df = (runs[nb.FP64][3][:, 0] - runs[nb.FP64][2][0]) / abs(runs[nb.FP64][2][0])
    assert np.abs(df).max() < 1e-5
    assert np.abs(dm - df).max() < 1e-6
    # the FP64 GPU energy of the final state against the oracle's pair-sum energy
    ref = oracle.energy(runs[nb.FP64][4], runs[nb.FP64][5], m, G=G, eps=eps)
    assert abs(runs[nb.FP64][3][-1, 0] - ref[0]) <= 1e-12 * abs(ref[0])
    # the two trajectories stay close over 100 steps
    assert np.abs(runs[nb.MIXED][4] - runs[nb.FP64][4]).max() < 1e-6


def test_two_spheres_1m_mixed_10_steps(nb):
    import torch
    n, G, eps, dt, T = 1048576, 1.0, 0.002, 5e-4, 10
    x, v, m = inputs.two_spheres(n, seed=3)
    ctx = nb.nbody_init(G=G, eps=eps, dt=dt, precision=nb.MIXED, n=n, energy_every=10)
    xt, vt, mt = to_dev(x, v, m)
    at = torch.empty_like(xt)
    nb.nbody_forces(ctx, xt, mt, at)
    e0 = _sampled_err(x, m, at.cpu().numpy(), G, eps, k=SAMPLE_1M)
    assert np.median(e0) <= MIX_MED and e0.max() <= MIX_MAX, (np.median(e0), e0.max())
    E0 = nb.nbody_energy(ctx, xt, vt, mt).cpu().numpy()[0]
    log = nb.nbody_step(ctx, xt, vt, mt, at, True, T)
    nb.nbody_sync(ctx)
    xf, af = to_np(xt, at)
    e1 = _sampled_err(xf, m, af, G, eps, k=SAMPLE_1M, seed=19)
    assert np.median(e1) <= MIX_MED and e1.max() <= MIX_MAX, (np.median(e1), e1.max())
    E1 = log.cpu().numpy()[-1, 0]
    assert abs(E1[0] - E0[0]) <= 1e-5 * abs(E0[0])
    np.testing.assert_allclose(E1[3:6], E0[3:6], atol=1e-9)
    ctx.close()


# positions and velocities after the 50 ensemble steps against the oracle's KDK, per element
# (relative, guard 1e-3 of the rms element): the mixed force error (<= 1e-4 per body, ~1e-7
# typical) moves x by ~ t^2 |da| / 2 and v by ~ t |da| over t = 0.05
ENS_X_TOL, ENS_V_TOL = 1e-6, 1e-5
# largest relative energy drift of any system over the 50 steps (leapfrog error plus the
# mixed energy evaluation); measured maximum 9.6e-6 on GB300, bound at about 3x that
ENS_DRIFT = 3e-5


@pytest.mark.parametrize("graph", [False, True])
def test_ensemble_512_systems_50_steps(nb, graph):
    import torch
    G, eps, dt, T = 1.0, 0.01, 1e-3, 50
    ens = inputs.ensemble(512, seed=4)
    off = [int(o) for o in ens.offsets]
    flags = nb.FLAG_GRAPH if graph else 0
    ctx = nb.nbody_init(G=G, eps=eps, dt=dt, precision=nb.MIXED, offsets=off, energy_every=T, flags=flags)
    xt, vt, mt = to_dev(ens.x, ens.v, ens.m)
    at = torch.empty_like(xt)
    nb.nbody_forces(ctx, xt, mt, at)
    a0 = at.cpu().numpy()
    E0 = nb.nbody_energy(ctx, xt, vt, mt).cpu().numpy()
    log = nb.nbody_step(ctx, xt, vt, mt, at, True, T)
    nb.nbody_sync(ctx)
    xf, vf, af = to_np(xt, vt, at)
    E1 = log.cpu().numpy()[0]
    sizes = np.diff(off)
    order = np.argsort(sizes)
    # forces at the start and at the end on sampled bodies: the 20 smallest and the 3 largest systems
    for s in list(order[:20]) + list(order[-3:]):
        b, e = off[s], off[s + 1]
        k = min(256, e - b)
        for xx, aa, seed in ((ens.x[b:e], a0[b:e], 1), (xf[b:e], af[b:e], 2)):
            err = _sampled_err(xx, ens.m[b:e], aa, G, eps, k=k, seed=seed)
            assert err.max() <= MIX_MAX and np.median(err) <= MIX_MED, (s, sizes[s], err.max())
    # whole trajectories against the oracle's KDK: the 20 smallest systems and the two closest
    # to 2048 bodies; x, v per element and a per body
    near2k = [int(i) for i in np.argsort(np.abs(sizes - 2048))[:2]]
    for s in list(order[:20]) + near2k:
        b, e = off[s], off[s + 1]
        xr, vr, ar, _ = oracle.kdk(ens.x[b:e], ens.v[b:e], ens.m[b:e], G, eps, dt, T)
        assert_elem_close(xf[b:e], xr, ENS_X_TOL, f"x of system {s} (N={sizes[s]})")
        assert_elem_close(vf[b:e], vr, ENS_V_TOL, f"v of system {s} (N={sizes[s]})")
        err = force_rel_err(af[b:e], ar)
        assert err.max() <= MIX_MAX and np.median(err) <= MIX_MED, (s, sizes[s], err.max())
    # conservation per system: momentum stays ~0, energy drift small
    assert np.abs(E1[:, 3:6]).max() < 1e-9
    drift = np.abs(E1[:, 0] - E0[:, 0]) / np.abs(E0[:, 0])
    assert drift.max() < ENS_DRIFT, drift.max()
    ctx.close()
