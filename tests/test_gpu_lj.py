"""GPU parity of the Lennard-Jones pair law (the paper's Eq. 1) with reflecting
walls ("boundary checking"), against the FP64 CPU oracle."""

import numpy as np
import pytest

import oracle
from paper_2511_02655_gb300 import inputs
from helpers import assert_elem_close, force_rel_err, to_dev, to_np

pytestmark = pytest.mark.gpu

FP64_TOL, MIX_MED, MIX_MAX = 1e-12, 1e-6, 1e-4


def _lj_forces(nb, prec, x, m, **kw):
    ctx = nb.nbody_init(law=nb.LENNARD_JONES, precision=prec, n=len(m), dt=5e-3, **kw)
    xt, mt = to_dev(x, m)
    a, phi = nb.nbody_forces(ctx, xt, mt)
    nb.nbody_sync(ctx)
    return a.cpu().numpy(), phi.cpu().numpy()


@pytest.mark.parametrize("density", [0.05, 0.5])
@pytest.mark.parametrize("prec", [0, 1])
def test_lj_forces(nb, prec, density):
    x, v, m, box = inputs.lj_gas(2000, seed=7, density=density, temperature=2.0)
    m = m * np.exp(0.2 * np.random.default_rng(1).standard_normal(len(m)))
    a, phi = _lj_forces(nb, prec, x, m, lj_epsilon=1.3, lj_sigma=0.9)
    a_ref, phi_ref = oracle.lj_forces(x, m, eps_lj=1.3, sigma=0.9)
    e = force_rel_err(a, a_ref)
    # the LJ potential changes sign with r, so phi is checked per body with the guard of
    # elem_rel_err (1e-3 of the rms phi), like the forces
    if prec == nb.FP64:
        assert e.max() <= FP64_TOL
        assert_elem_close(phi, phi_ref, FP64_TOL, "phi")
    else:
        assert np.median(e) <= MIX_MED and e.max() <= MIX_MAX, (np.median(e), e.max())
        assert_elem_close(phi, phi_ref, MIX_MAX, "phi")


@pytest.mark.parametrize("variant,j_tile", [(2, 256), (2, 512), (3, 256), (3, 512)])
def test_lj_packed_variants_forces_and_steps(nb, variant, j_tile):
    """The packed Lennard-Jones kernel, uncapped (variant 2) and compiled for 6 CTAs per SM
    (variant 3), at both j-tiles the capped build has: forces and 20 steps between walls."""
    import torch
    x, v, m, box = inputs.lj_gas(3001, seed=21, density=0.05, temperature=2.0)
    kw = dict(block=128, i_per_thread=1, j_tile=j_tile, variant=variant)
    a, phi = _lj_forces(nb, nb.MIXED, x, m, **kw)
    a_ref, phi_ref = oracle.lj_forces(x, m)
    e = force_rel_err(a, a_ref)
    assert np.median(e) <= MIX_MED and e.max() <= MIX_MAX, (np.median(e), e.max())
    assert_elem_close(phi, phi_ref, MIX_MAX, "phi")
    dt, T = 5e-3, 20
    ctx = nb.nbody_init(law=nb.LENNARD_JONES, precision=nb.MIXED, n=len(m), dt=dt, box=box, energy_every=5, **kw)
    assert nb.nbody_get_tuning(ctx)["variant"] == variant
    xt, vt, mt = to_dev(x, v, m)
    at = torch.empty_like(xt)
    log = nb.nbody_step(ctx, xt, vt, mt, at, False, T)
    nb.nbody_sync(ctx)
    xr, vr, ar, logr = oracle.lj_kdk(x, v, m, 1.0, 1.0, 0.0, box, dt, T, energy_every=5)
    xg, vg, ag, lg = to_np(xt, vt, at, log)
    assert xg.min() >= 0 and xg.max() <= box
    assert np.abs(xg - xr).max() <= 1e-5
    e = force_rel_err(ag, ar)
    assert np.median(e) <= MIX_MED and e.max() <= MIX_MAX, (np.median(e), e.max())
    np.testing.assert_allclose(lg[:, 0, 0], logr[:, 0], rtol=1e-5)


@pytest.mark.parametrize("prec", [0, 1])
def test_lj_kdk_with_walls(nb, prec):
    import torch
    x, v, m, box = inputs.lj_gas(1000, seed=8, density=0.1, temperature=2.0)
    dt, T = 5e-3, 60
    ctx = nb.nbody_init(law=nb.LENNARD_JONES, precision=prec, n=1000, dt=dt, box=box, energy_every=10)
    xt, vt, mt = to_dev(x, v, m)
    at = torch.empty_like(xt)
    log = nb.nbody_step(ctx, xt, vt, mt, at, False, T)
    nb.nbody_sync(ctx)
    xr, vr, ar, logr = oracle.lj_kdk(x, v, m, 1.0, 1.0, 0.0, box, dt, T, energy_every=10)
    xg, vg, ag, lg = to_np(xt, vt, at, log)
    assert xg.min() >= 0 and xg.max() <= box
    if prec == nb.FP64:
        assert np.abs(xg - xr).max() <= 1e-10
        assert force_rel_err(ag, ar).max() <= 1e-9
        np.testing.assert_allclose(lg[:, 0, 0:3], logr[:, 0:3], rtol=1e-10)
    else:
        assert np.abs(xg - xr).max() <= 1e-5
        np.testing.assert_allclose(lg[:, 0, 0], logr[:, 0], rtol=1e-5)
    # walls reflect, so momentum is not conserved; energy is (to the leapfrog's accuracy)
    assert np.abs(lg[:, 0, 0] - lg[0, 0, 0]).max() <= 1e-3 * abs(lg[0, 0, 0])


def test_lj_paper_configuration_short_run(nb):
    """The paper's system size (10 000 particles), 20 KDK steps, FP64 GPU vs oracle."""
    import torch
    x, v, m, box = inputs.lj_gas(10000, seed=9)
    dt, T = 5e-3, 20
    ctx = nb.nbody_init(law=nb.LENNARD_JONES, precision=nb.FP64, n=10000, dt=dt, box=box)
    xt, vt, mt = to_dev(x, v, m)
    at = torch.empty_like(xt)
    nb.nbody_step(ctx, xt, vt, mt, at, False, T)
    nb.nbody_sync(ctx)
    xr, vr, ar, _ = oracle.lj_kdk(x, v, m, 1.0, 1.0, 0.0, box, dt, T)
    assert np.abs(xt.cpu().numpy() - xr).max() <= 1e-10
    idx = inputs.sample_indices(10000, 512, seed=3)
    e = force_rel_err(at.cpu().numpy()[idx], ar[idx])
    assert e.max() <= 1e-9


def test_lj_adjoint_unsupported(nb):
    x, v, m, box = inputs.lj_gas(64, seed=1)
    ctx = nb.nbody_init(law=nb.LENNARD_JONES, precision=nb.FP64, n=64, dt=1e-3)
    xt, vt, mt = to_dev(x, v, m)
    with pytest.raises(nb.NBodyError) as ei:
        nb.nbody_adjoint(ctx, xt, vt, mt, 5, 2, xt.clone(), vt.clone())
    assert ei.value.status == 6


def test_lj_graph_replay_matches_eager(nb):
    import torch
    x, v, m, box = inputs.lj_gas(3000, seed=12, density=0.1)
    outs = []
    for flags in (0, nb.FLAG_GRAPH):
        ctx = nb.nbody_init(law=nb.LENNARD_JONES, precision=nb.MIXED, n=3000, dt=5e-3, box=box, energy_every=5,
                            flags=flags, block=128, i_per_thread=1, j_tile=256, slice=512)
        xt, vt, mt = to_dev(x, v, m)
        at = torch.empty_like(xt)
        log = torch.empty((4, 1, 9), dtype=torch.float64, device="cuda")
        for _ in range(2):
            nb.nbody_step(ctx, xt, vt, mt, at, False, 20, log)
        nb.nbody_sync(ctx)
        outs.append((xt.cpu(), vt.cpu(), at.cpu(), log.cpu()))
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def test_lj_unsoftened_coincident_bodies_flag_nonfinite(nb):
    x = np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 1.0], [3.0, 1.0, 1.0]])
    ctx = nb.nbody_init(law=nb.LENNARD_JONES, precision=nb.FP64, n=3, dt=1e-3)
    nb.nbody_forces(ctx, *to_dev(x, np.ones(3)))
    with pytest.raises(nb.NBodyError) as ei:
        nb.nbody_sync(ctx)
    assert ei.value.status == 5


@pytest.mark.parametrize("graph", [False, True])
def test_lj_paper_configuration_mixed(nb, graph):
    """The paper's system (10 000 particles, density 0.05, walls) on the mixed path as the bench
    runs it (tuned tiling, energy every step, optionally replayed as a CUDA graph): forces of 1024
    sampled particles against the oracle at the start and after 40 steps, and the energy record
    against the oracle's pair sum."""
    import torch
    n = 10000
    x, v, m, box = inputs.lj_gas(n, seed=9)
    ctx = nb.nbody_init(law=nb.LENNARD_JONES, precision=nb.MIXED, n=n, dt=5e-3, box=box, energy_every=1,
                        flags=nb.FLAG_GRAPH if graph else 0)
    xt, vt, mt = to_dev(x, v, m)
    at = torch.empty_like(xt)
    nb.nbody_forces(ctx, xt, mt, at)
    idx = inputs.sample_indices(n, 1024, seed=5)
    a_ref, _ = oracle.lj_forces_at(x, m, idx)
    e = force_rel_err(at.cpu().numpy()[idx], a_ref)
    assert np.median(e) <= MIX_MED and e.max() <= MIX_MAX, (np.median(e), e.max())
    log = nb.nbody_step(ctx, xt, vt, mt, at, True, 40)
    nb.nbody_sync(ctx)
    xf, vf, af = to_np(xt, vt, at)
    assert xf.min() >= 0 and xf.max() <= box
    a_ref, _ = oracle.lj_forces_at(xf, m, idx)
    e = force_rel_err(af[idx], a_ref)
    assert np.median(e) <= MIX_MED and e.max() <= MIX_MAX, (np.median(e), e.max())
    E = oracle.lj_energy(xf, vf, m)
    assert abs(log.cpu().numpy()[-1, 0, 0] - E[0]) <= 1e-6 * abs(E[0])


@pytest.mark.parametrize("prec", [0, 1])
def test_lj_several_systems(nb, prec):
    """Independent Lennard-Jones systems in one context (one of them empty): each system's forces
    match the oracle on that system alone, so no pair crosses a system boundary."""
    sizes = [500, 0, 1201, 37]
    parts = [inputs.lj_gas(s, seed=20 + k, density=0.1) for k, s in enumerate(sizes) if s > 0]
    x = np.concatenate([p[0] for p in parts])
    m = np.concatenate([p[2] for p in parts])
    off = [0]
    for s_ in sizes:
        off.append(off[-1] + s_)
    ctx = nb.nbody_init(law=nb.LENNARD_JONES, precision=prec, offsets=off, dt=5e-3)
    xt, mt = to_dev(x, m)
    a, phi = nb.nbody_forces(ctx, xt, mt)
    nb.nbody_sync(ctx)
    a, phi = to_np(a, phi)
    for s in range(len(sizes)):
        b, e = off[s], off[s + 1]
        if e == b:
            continue
        a_ref, phi_ref = oracle.lj_forces(x[b:e], m[b:e])
        err = force_rel_err(a[b:e], a_ref)
        if prec == nb.FP64:
            assert err.max() <= FP64_TOL
        else:
            assert np.median(err) <= MIX_MED and err.max() <= MIX_MAX, (s, np.median(err), err.max())
