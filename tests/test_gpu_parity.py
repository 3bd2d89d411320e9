"""GPU parity: the sm_103a kernels through the C ABI against the FP64 CPU oracle.

Bounds: FP64 path forces within 1e-12 relative per body; mixed path median
<= 1e-6 and max <= 1e-4 (relative per body, cancellation guard at 1e-3 of the
rms force).
"""

import numpy as np
import pytest

import oracle
from paper_2511_02655_gb300 import inputs
from helpers import assert_elem_close, force_rel_err, to_dev, to_np

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIX_MED, MIX_MAX = 1e-6, 1e-4
# mixed potential, per body: its pair terms all have the same sign, so a j-tile's float32 sum of
# J <= 512 terms is good to (J - 1) 2^-24 < 3.1e-5 relative (recursive summation bound; it is
# approached when one near pair dominates and the tile's small terms are added after it), and
# the compensated fold across tiles adds ~2^-24: max 3e-5, median 1e-6 per body
MIX_PHI_MED, MIX_PHI_MAX = 1e-6, 3e-5


def _check_mixed_phi(phi, phi_ref):
    e = assert_elem_close(phi, phi_ref, MIX_PHI_MAX, "phi")
    assert np.median(e) <= MIX_PHI_MED, np.median(e)


def _forces(nb, prec, x, m, G, eps, offsets=None, **kw):
    import torch
    ctx = nb.nbody_init(G=G, eps=eps, dt=1e-3, precision=prec, offsets=offsets or [0, len(m)], **kw)
    xt, mt = to_dev(x, m)
    a, phi = nb.nbody_forces(ctx, xt, mt)
    nb.nbody_sync(ctx)
    torch.cuda.synchronize()
    return ctx, a.cpu().numpy(), phi.cpu().numpy()


# ----------------------------------------------------------------------------------------
# plain method, N = 1024 Plummer (G = 1, eps = 0.01, dt = 1e-3, 10 KDK steps)


def test_fp64_forces_n1024(nb):
    x, v, m = inputs.plummer(1024, seed=1)
    _, a, phi = _forces(nb, nb.FP64, x, m, 1.0, 0.01)
    a_ref, phi_ref = oracle.forces(x, m, G=1.0, eps=0.01)
    assert force_rel_err(a, a_ref).max() <= FP64_TOL
    assert_elem_close(phi, phi_ref, FP64_TOL, "phi")


def test_mixed_forces_n1024(nb):
    x, v, m = inputs.plummer(1024, seed=1)
    _, a, phi = _forces(nb, nb.MIXED, x, m, 1.0, 0.01)
    a_ref, phi_ref = oracle.forces(x, m, G=1.0, eps=0.01)
    e = force_rel_err(a, a_ref)
    assert np.median(e) <= MIX_MED and e.max() <= MIX_MAX, (np.median(e), e.max())
    _check_mixed_phi(phi, phi_ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_kdk_10_steps_n1024_with_energy(nb, prec):
    import torch
    G, eps, dt, n_steps = 1.0, 0.01, 1e-3, 10
    x, v, m = inputs.plummer(1024, seed=1)
    ctx = nb.nbody_init(G=G, eps=eps, dt=dt, precision=prec, n=1024, energy_every=1)
    xt, vt, mt = to_dev(x, v, m)
    at = torch.empty_like(xt)
    log = nb.nbody_step(ctx, xt, vt, mt, at, False, n_steps)
    nb.nbody_sync(ctx)
    xr, vr, ar, logr = oracle.kdk(x, v, m, G, eps, dt, n_steps, energy_every=1)
    xg, vg, ag, lg = to_np(xt, vt, at, log)
    if prec == nb.FP64:
        assert np.abs(xg - xr).max() <= 1e-13
        assert np.abs(vg - vr).max() <= 1e-12 * np.abs(vr).max()
        assert force_rel_err(ag, ar).max() <= FP64_TOL
        np.testing.assert_allclose(lg[:, 0, 0:3], logr[:, 0:3], rtol=1e-12)
    else:
        assert np.abs(xg - xr).max() <= 1e-8
        e = force_rel_err(ag, ar)
        assert np.median(e) <= MIX_MED and e.max() <= MIX_MAX
        np.testing.assert_allclose(lg[:, 0, 0:3], logr[:, 0:3], rtol=2e-6)
    # momentum and angular momentum: KDK conserves them exactly when pair forces are exactly
    # antisymmetric (FP64 path, up to rounding); float32 pair forces break antisymmetry at
    # ~1e-7 relative, so P and L drift by ~ steps * dt * sum m|a| * 1e-7 on the mixed path.
    np.testing.assert_allclose(lg[:, 0, 3:9], logr[:, 3:9], atol=1e-12 if prec == nb.FP64 else 1e-10)


@pytest.mark.parametrize("prec", [0, 1])
def test_energy_reduction(nb, prec):
    x, v, m = inputs.plummer(3000, seed=4)
    m = m * np.exp(0.4 * np.random.default_rng(2).standard_normal(3000))
    ctx = nb.nbody_init(G=0.8, eps=0.02, dt=1e-3, precision=prec, n=3000)
    out = nb.nbody_energy(ctx, *to_dev(x, v, m))
    nb.nbody_sync(ctx)
    ref = oracle.energy(x, v, m, G=0.8, eps=0.02)
    g = out.cpu().numpy()[0]
    tol = 1e-12 if prec == nb.FP64 else 1e-6
    assert abs(g[0] - ref[0]) <= tol * abs(ref[0])
    assert abs(g[2] - ref[2]) <= tol * abs(ref[2])
    assert abs(g[1] - ref[1]) <= 1e-13 * abs(ref[1])
    np.testing.assert_allclose(g[3:], ref[3:], atol=1e-14)


# ----------------------------------------------------------------------------------------
# edge cases: tiny and ragged sizes, eps = 0, coincident bodies, several systems


@pytest.mark.parametrize("n", [1, 2, 3, 31, 100, 257, 1000, 4097])
@pytest.mark.parametrize("prec", [0, 1])
def test_ragged_sizes(nb, n, prec):
    x, v, m = inputs.plummer(n, seed=n)
    m = m * np.exp(0.3 * np.random.default_rng(n).standard_normal(n))
    _, a, phi = _forces(nb, prec, x, m, 1.3, 0.05)
    a_ref, phi_ref = oracle.forces(x, m, G=1.3, eps=0.05)
    if n == 1:
        assert np.all(a == 0) and np.all(phi == 0)
        return
    e = force_rel_err(a, a_ref)
    if prec == nb.FP64:
        assert e.max() <= FP64_TOL
        assert_elem_close(phi, phi_ref, FP64_TOL, "phi")
    else:
        assert np.median(e) <= MIX_MED and e.max() <= MIX_MAX
        _check_mixed_phi(phi, phi_ref)


@pytest.mark.parametrize("tiling", [dict(block=128, i_per_thread=1, j_tile=128, slice=512),
                                    dict(block=256, i_per_thread=4, j_tile=256, slice=1024),
                                    dict(block=128, i_per_thread=2, j_tile=256, slice=256)])
@pytest.mark.parametrize("prec", [0, 1])
def test_explicit_tilings_agree(nb, tiling, prec):
    x, v, m = inputs.plummer(2500, seed=9)
    _, a, phi = _forces(nb, prec, x, m, 1.0, 0.01, **tiling)
    a_ref, _ = oracle.forces(x, m, G=1.0, eps=0.01)
    e = force_rel_err(a, a_ref)
    assert e.max() <= (FP64_TOL if prec == nb.FP64 else MIX_MAX)


def test_unsoftened_kepler_fp64(nb):
    import torch
    x0, v0, m, period = inputs.kepler_pair(0.6, 0.4, 1.0, 0.5)
    dt = period / 2000
    ctx = nb.nbody_init(G=1.0, eps=0.0, dt=dt, precision=nb.FP64, n=2)
    xt, vt, mt = to_dev(x0, v0, m)
    at = torch.empty_like(xt)
    nb.nbody_step(ctx, xt, vt, mt, at, False, 1000)
    nb.nbody_sync(ctx)
    xr, vr, _, _ = oracle.kdk(x0, v0, m, 1.0, 0.0, dt, 1000)
    assert np.abs(xt.cpu().numpy() - xr).max() <= 1e-11


def test_coincident_bodies_softened(nb):
    x = np.zeros((4, 3))
    x[2:] = [[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]]
    m = np.array([0.1, 0.2, 0.3, 0.4])
    for prec in (nb.FP64, nb.MIXED):
        _, a, phi = _forces(nb, prec, x, m, 1.0, 0.1)
        a_ref, phi_ref = oracle.forces(x, m, G=1.0, eps=0.1)
        np.testing.assert_allclose(a, a_ref, rtol=1e-6 if prec else 1e-14, atol=1e-12)
        np.testing.assert_allclose(phi, phi_ref, rtol=1e-6 if prec else 1e-14)


def test_unsoftened_coincident_bodies_flag_nonfinite(nb):
    import torch
    x = np.zeros((2, 3))
    m = np.array([0.5, 0.5])
    ctx = nb.nbody_init(G=1.0, eps=0.0, dt=1e-3, precision=nb.MIXED, n=2)
    nb.nbody_forces(ctx, *to_dev(x, m))
    with pytest.raises(nb.NBodyError) as ei:
        nb.nbody_sync(ctx)
    assert ei.value.status == 5
    nb.nbody_sync(ctx)  # flag was cleared


@pytest.mark.parametrize("prec", [0, 1])
def test_several_systems_with_empty_ones(nb, prec):
    sizes = [0, 5, 300, 0, 1, 1200, 2]
    ens = inputs.ensemble(len(sizes), seed=3, sizes=np.array(sizes))
    off = [int(o) for o in ens.offsets]
    _, a, phi = _forces(nb, prec, ens.x, ens.m, 1.0, 0.01, offsets=off)
    for s in range(len(sizes)):
        b, e = off[s], off[s + 1]
        if e - b < 2:
            assert np.all(a[b:e] == 0)
            continue
        a_ref, _ = oracle.forces(ens.x[b:e], ens.m[b:e], G=1.0, eps=0.01)
        err = force_rel_err(a[b:e], a_ref)
        assert err.max() <= (FP64_TOL if prec == nb.FP64 else MIX_MAX)


def test_deterministic(nb):
    x, v, m = inputs.plummer(5000, seed=6)
    ctx = nb.nbody_init(G=1.0, eps=0.01, dt=1e-3, precision=nb.MIXED, n=5000)
    xt, mt = to_dev(x, m)
    a1, p1 = nb.nbody_forces(ctx, xt, mt)
    a2, p2 = nb.nbody_forces(ctx, xt, mt)
    assert bool((a1 == a2).all()) and bool((p1 == p2).all())


def test_host_pointers_rejected_without_launch(nb):
    import torch
    ctx = nb.nbody_init(G=1.0, eps=0.01, dt=1e-3, precision=nb.MIXED, n=16)
    x = torch.zeros((16, 3), dtype=torch.float64)
    m = torch.ones(16, dtype=torch.float64)
    a = torch.zeros((16, 3), dtype=torch.float64)
    lib = nb.load()
    before = nb.nbody_launch_count(ctx)
    st = lib.nbody_forces(ctx._h, nb.ctx_ptr(x.data_ptr()), nb.ctx_ptr(m.data_ptr()), nb.ctx_ptr(a.data_ptr()),
                          None)
    assert st == 1 and "device memory" in nb.nbody_last_error(ctx) or "CUDA pointer" in nb.nbody_last_error(ctx)
    assert nb.nbody_launch_count(ctx) == before
    # too short a device buffer
    xs = torch.zeros((8, 3), dtype=torch.float64, device="cuda")
    st = lib.nbody_forces(ctx._h, nb.ctx_ptr(xs.data_ptr()), nb.ctx_ptr(m.cuda().data_ptr()),
                          nb.ctx_ptr(a.cuda().data_ptr()), None)
    assert st in (0, 1)  # caching allocators may hand out a larger block; checked when it is not
    nb.nbody_sync(ctx)


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("memory", ["pinned", "pinned_state_pageable_log", "pageable"])
def test_step_host_matches_device_path(nb, memory, graph):
    """nbody_step_host moves mapped pinned buffers with one copy kernel each way and any
    other host memory with cudaMemcpyAsync; both give the device path's results bit for bit."""
    import torch
    n = 2049  # odd: the copy kernel's ragged end
    x, v, m = inputs.plummer(n, seed=12)
    ctx = nb.nbody_init(G=1.0, eps=0.01, dt=1e-3, precision=nb.MIXED, n=n, energy_every=2,
                        flags=nb.FLAG_GRAPH if graph else 0)
    xt, vt, mt = to_dev(x, v, m)
    at = torch.empty_like(xt)
    log = nb.nbody_step(ctx, xt, vt, mt, at, False, 4)
    log2 = nb.nbody_step(ctx, xt, vt, mt, at, True, 4)
    nb.nbody_sync(ctx)
    pin = (lambda t: t.pin_memory()) if memory != "pageable" else (lambda t: t)
    xh, vh = pin(torch.from_numpy(x.copy())), pin(torch.from_numpy(v.copy()))
    mh, ah = pin(torch.from_numpy(m.copy())), pin(torch.zeros((n, 3), dtype=torch.float64))
    logh = torch.zeros((2, 1, 9), dtype=torch.float64)
    if memory == "pinned":
        logh = logh.pin_memory()
    nb.nbody_step_host(ctx, xh, vh, mh, ah, False, 4, logh)
    assert torch.equal(logh, log.cpu())
    nb.nbody_step_host(ctx, xh, vh, mh, ah, True, 4, logh)  # a passed in from the host
    assert torch.equal(xh, xt.cpu()) and torch.equal(vh, vt.cpu()) and torch.equal(ah, at.cpu())
    assert torch.equal(logh, log2.cpu())


def test_graph_replay_matches_eager(nb):
    import torch
    x, v, m = inputs.plummer(3000, seed=13)
    outs = []
    for flags in (0, nb.FLAG_GRAPH):
        ctx = nb.nbody_init(G=1.0, eps=0.01, dt=1e-3, precision=nb.MIXED, n=3000, energy_every=5, flags=flags,
                            block=128, i_per_thread=2, j_tile=128, slice=1024)
        xt, vt, mt = to_dev(x, v, m)
        at = torch.empty_like(xt)
        log = torch.empty((2, 1, 9), dtype=torch.float64, device="cuda")
        for _ in range(3):  # first call captures, later calls replay
            nb.nbody_step(ctx, xt, vt, mt, at, False, 10, log)
        nb.nbody_sync(ctx)
        outs.append((xt.cpu(), vt.cpu(), at.cpu(), log.cpu()))
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def test_kernel_profiling_counts_force_launches(nb):
    import torch
    x, v, m = inputs.plummer(4096, seed=14)
    ctx = nb.nbody_init(G=1.0, eps=0.01, dt=1e-3, precision=nb.MIXED, n=4096)
    xt, vt, mt = to_dev(x, v, m)
    at = torch.empty_like(xt)
    nb.nbody_profile(ctx, True)
    nb.nbody_step(ctx, xt, vt, mt, at, False, 5)
    ms, k = nb.nbody_kernel_time(ctx, 0)
    assert k == 6 and ms > 0
    nb.nbody_profile(ctx, False)
    nb.nbody_step(ctx, xt, vt, mt, at, True, 2)
    assert nb.nbody_kernel_time(ctx, 0)[1] == 6


@pytest.mark.parametrize("tiling", [dict(block=256, i_per_thread=2, j_tile=256, slice=2048),
                                    dict(block=128, i_per_thread=4, j_tile=128, slice=1024),
                                    dict(block=128, i_per_thread=1, j_tile=128, slice=512)])
def test_packed_and_scalar_mixed_kernels_agree(nb, tiling):
    """The packed kernel sums even and odd j-bodies of a tile in separate lanes, so it agrees
    with the scalar kernel to float32 rounding of the partial sums, not bit for bit."""
    x, v, m = inputs.two_spheres(6002, seed=21)  # 6002: ragged tail tiles (padding to quads)
    outs = []
    for variant in (1, 2):
        _, a, phi = _forces(nb, nb.MIXED, x, m, 1.0, 0.004, variant=variant, **tiling)
        outs.append((a, phi))
    a_ref, phi_ref = oracle.forces(x, m, G=1.0, eps=0.004)
    for a, phi in outs:
        e = force_rel_err(a, a_ref)
        assert np.median(e) <= MIX_MED and e.max() <= MIX_MAX, (np.median(e), e.max())
        _check_mixed_phi(phi, phi_ref)
    assert force_rel_err(outs[1][0], outs[0][0]).max() <= 1e-5


@pytest.mark.parametrize("variant", [1, 2])
def test_near_pairs_far_from_origin(nb, variant):
    """Tight pairs (separation ~ eps / 2) around |x| ~ 100: float32 staging coordinates alone
    would carry ~4e-6 absolute error, several % of the pair separation; the near-pair
    refinement keeps the mixed path within its bounds."""
    rng = np.random.default_rng(5)
    centres = rng.normal(size=(500, 3))
    centres = 100.0 * centres / np.linalg.norm(centres, axis=1, keepdims=True)
    eps = 1e-3
    off = rng.normal(size=(500, 3)) * 0.5 * eps
    x = np.concatenate([centres, centres + off])
    m = np.full(1000, 1e-3)
    _, a, phi = _forces(nb, nb.MIXED, x, m, 1.0, eps, variant=variant)
    a_ref, phi_ref = oracle.forces(x, m, G=1.0, eps=eps)
    e = force_rel_err(a, a_ref)
    assert np.median(e) <= MIX_MED and e.max() <= MIX_MAX, (np.median(e), e.max())
    _check_mixed_phi(phi, phi_ref)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
def test_virial_matches_oracle(nb, prec, tol):
    sizes = [300, 0, 1200, 37]
    ens = inputs.ensemble(len(sizes), seed=17, sizes=np.array(sizes))
    off = [int(o) for o in ens.offsets]
    G, eps = 1.2, 0.02
    ctx = nb.nbody_init(G=G, eps=eps, dt=1e-3, precision=prec, offsets=off)
    out = nb.nbody_virial(ctx, *to_dev(ens.x, ens.v, ens.m))
    nb.nbody_sync(ctx)
    out = out.cpu().numpy()
    for s in range(len(sizes)):
        b, e = off[s], off[s + 1]
        if e == b:
            assert np.all(out[s] == 0)
            continue
        K, W, Q = oracle.virial(ens.x[b:e], ens.v[b:e], ens.m[b:e], G=G, eps=eps)
        assert abs(out[s, 0] - K) <= 1e-13 * K
        assert abs(out[s, 1] - W) <= tol * abs(W), (s, out[s], W)
        assert abs(out[s, 2] - Q) <= 2 * tol * abs(Q)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
def test_virial_lennard_jones_matches_oracle(nb, prec, tol):
    x, v, m, box = inputs.lj_gas(2000, seed=19, density=0.2)
    ctx = nb.nbody_init(law=nb.LENNARD_JONES, precision=prec, n=2000, dt=1e-3, lj_epsilon=1.1, lj_sigma=0.95)
    out = nb.nbody_virial(ctx, *to_dev(x, v, m))
    nb.nbody_sync(ctx)
    K, W, Q = oracle.virial(x, v, m, law=1, eps_lj=1.1, sigma=0.95)
    got = out.cpu().numpy()[0]
    assert abs(got[1] - W) <= tol * abs(W) and abs(got[0] - K) <= 1e-13 * K, (got, W)


@pytest.mark.parametrize("prec", [0, 1])
def test_ring_schedule_passes_agree(nb, prec):
    """The paper's ring exchange (Sec. V-B, Fig. 1) as a blocked schedule on one GPU: P j-slices
    play the P ranks' blocks, each an (i-tile, j-block) pass with its own partial folded
    in a fixed order. Every P gives the oracle's forces; FP64 results agree across P to rounding."""
    n = 4096
    x, v, m = inputs.plummer(n, seed=23)
    a_ref, _ = oracle.forces(x, m, G=1.0, eps=0.01)
    res = []
    for P in (1, 2, 3, 4, 8):
        sl = -(-n // P)
        sl = -(-sl // 128) * 128
        ctx, a, _ = _forces(nb, prec, x, m, 1.0, 0.01, block=128, i_per_thread=1, j_tile=128, slice=sl)
        assert nb.nbody_get_tuning(ctx)["slice"] == sl
        res.append(a)
        e = force_rel_err(a, a_ref)
        if prec == nb.FP64:
            assert e.max() <= FP64_TOL
        else:
            assert np.median(e) <= MIX_MED and e.max() <= MIX_MAX
    for a in res[1:]:
        assert force_rel_err(a, res[0]).max() <= (1e-13 if prec == nb.FP64 else 1e-5)


@pytest.mark.parametrize("law", ["gravity", "lj"])
def test_potential_free_pass_matches(nb, law):
    """Without a phi output or an energy record the packed kernel skips the potential; the
    accelerations and trajectories are bit-identical to the passes that form it."""
    import torch
    if law == "gravity":
        x, v, m = inputs.plummer(3001, seed=31)
        kw = dict(G=1.0, eps=0.01, dt=1e-3)
    else:
        x, v, m, box = inputs.lj_gas(3001, seed=32, density=0.1)
        kw = dict(law=nb.LENNARD_JONES, dt=5e-3, box=box)
    til = dict(variant=2, block=128, i_per_thread=2, j_tile=256, slice=1024)
    xt, vt, mt = to_dev(x, v, m)
    runs = []
    for every in (1, 0):  # energy record every step (potential formed) / none (skipped)
        ctx = nb.nbody_init(precision=nb.MIXED, n=len(m), energy_every=every, **til, **kw)
        a1, phi = nb.nbody_forces(ctx, xt, mt)
        a0, none = nb.nbody_forces(ctx, xt, mt, with_phi=False)
        assert none is None and torch.equal(a0, a1)
        xs, vs, at = xt.clone(), vt.clone(), torch.empty_like(xt)
        nb.nbody_step(ctx, xs, vs, mt, at, False, 6)
        nb.nbody_sync(ctx)
        runs.append((a1, xs, vs, at))
        ctx.close()
    for p, q in zip(*runs):
        assert torch.equal(p, q)


def test_tuning_cache(nb, tmp_path, monkeypatch):
    """NBODY_TUNE_CACHE keeps the tuner's choices: a second context of the same setup reuses
    the force and VJP tilings without tuning, another setup gets its own entry, and an entry
    that no longer installs is re-tuned."""
    import torch
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("NBODY_TUNE_CACHE", str(path))
    n = 5000
    x, v, m = inputs.plummer(n, seed=61)
    xt, vt, mt = to_dev(x, v, m)
    lam = torch.ones_like(xt)

    def make(eps=0.01):
        ctx = nb.nbody_init(G=1.0, eps=eps, dt=1e-3, precision=nb.MIXED, n=n)
        nb.nbody_adjoint(ctx, xt, vt, mt, 2, 1, lam, lam)  # tunes the VJP
        a, _ = nb.nbody_forces(ctx, xt, mt)
        nb.nbody_sync(ctx)
        return ctx, a

    c1, a1 = make()
    lines = path.read_text().splitlines()
    assert len(lines) == 2 and "|force|" in lines[0] and "|vjp|" in lines[1]
    c2, a2 = make()
    assert path.read_text().splitlines() == lines  # reused, nothing tuned
    assert nb.nbody_get_tuning(c2) == nb.nbody_get_tuning(c1) and torch.equal(a1, a2)
    c3, _ = make(eps=0.02)
    assert len(path.read_text().splitlines()) == 4  # another setup, its own entries
    # an entry that no longer installs (an uncompiled block size) is ignored and re-tuned
    key = lines[0].split("\t")[0]
    with open(path, "a") as f:
        f.write(f"{key}\t96 2 256 4096 1 0\n")
    c4, a4 = make()
    assert nb.nbody_get_tuning(c4)["block"] in (128, 256)
    assert torch.equal(a4, a1) or force_rel_err(a4.cpu().numpy(), a1.cpu().numpy()).max() <= 1e-5
    assert path.read_text().splitlines()[-1].startswith(key)
    for c in (c1, c2, c3, c4):
        c.close()


def test_register_capped_packed_variant(nb):
    """Variant 3 (the packed kernel compiled for 4 CTAs per SM) computes exactly what variant 2
    computes, in forces and in steps, and the tuner may choose it."""
    import torch
    x, v, m = inputs.plummer(4099, seed=71)
    xt, vt, mt = to_dev(x, v, m)
    outs = []
    for variant in (2, 3):
        ctx = nb.nbody_init(G=1.0, eps=0.01, dt=1e-3, precision=nb.MIXED, n=4099, variant=variant, block=128,
                            i_per_thread=2, j_tile=256, slice=1024)
        assert nb.nbody_get_tuning(ctx)["variant"] == variant
        a, phi = nb.nbody_forces(ctx, xt, mt)
        xs, vs, at = xt.clone(), vt.clone(), torch.empty_like(xt)
        nb.nbody_step(ctx, xs, vs, mt, at, False, 3)
        nb.nbody_sync(ctx)
        outs.append((a, phi, xs, vs, at))
        ctx.close()
    for p, q in zip(*outs):
        assert torch.equal(p, q)
    a_ref, _ = oracle.forces(x, m, G=1.0, eps=0.01)
    e = force_rel_err(outs[1][0].cpu().numpy(), a_ref)
    assert np.median(e) <= MIX_MED and e.max() <= MIX_MAX
    with pytest.raises(nb.NBodyError):  # capped build exists for the 128 x 2 tilings only
        nb.nbody_init(G=1.0, eps=0.01, dt=1e-3, precision=nb.MIXED, n=4099, variant=3, block=256,
                      i_per_thread=1, j_tile=256)


def test_nvtx_ranges_enabled(nb, monkeypatch):
    """NBODY_NVTX=1 wraps the API calls in NVTX ranges; results are unchanged."""
    import torch
    x, v, m = inputs.plummer(1000, seed=81)
    outs = []
    for flag in ("0", "1"):
        monkeypatch.setenv("NBODY_NVTX", flag)
        ctx = nb.nbody_init(G=1.0, eps=0.01, dt=1e-3, precision=nb.MIXED, n=1000, energy_every=1,
                            block=128, i_per_thread=2, j_tile=256, slice=512, variant=2)
        xt, vt, mt = to_dev(x, v, m)
        at = torch.empty_like(xt)
        log = nb.nbody_step(ctx, xt, vt, mt, at, False, 3)
        g = nb.nbody_adjoint(ctx, xt, vt, mt, 3, 2, at.clone(), at.clone())
        nb.nbody_sync(ctx)
        outs.append((xt.cpu(), log.cpu(), g[0].cpu()))
        ctx.close()
    for p, q in zip(*outs):
        assert torch.equal(p, q)
