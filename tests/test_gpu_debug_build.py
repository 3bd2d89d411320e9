"""The NBODY_DEBUG build (libnbody_debug.so): every kernel checks the work items,
chunks and per-system ranges it reads against the buffers they index, skips a
failed access and latches a status bit that nbody_sync reports as
NBODY_EINTERNAL. It stands in for a device memory checker. The tiny and ragged
sizes below run every entry point of both precisions through it, in a child
process that loads the debug build, and must come back without a failed check
and with the oracle's results."""

import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
    import oracle
    import paper_2511_02655_gb300 as nb
    from paper_2511_02655_gb300 import inputs
    from helpers import elem_rel_err, force_rel_err, to_dev, to_np
    assert nb.lib_path().endswith("libnbody_debug.so") and nb.nbody_build_flags() & 1
    G, eps, dt, T = 1.1, 0.05, 2e-3, 4
    for n in (1, 2, 3, 31, 4097):
        x, v, m = inputs.plummer(n, seed=100 + n)
        for prec, ftol, gtol in ((nb.FP64, 1e-12, 1e-11), (nb.MIXED, 1e-4, 1e-4)):
            ctx = nb.nbody_init(G=G, eps=eps, dt=dt, precision=prec, n=n, energy_every=2)
            xt, vt, mt = to_dev(x, v, m)
            a, phi = nb.nbody_forces(ctx, xt, mt)
            e = nb.nbody_energy(ctx, xt, vt, mt)
            w = nb.nbody_virial(ctx, xt, vt, mt)
            xs, vs, at = xt.clone(), vt.clone(), torch.empty_like(xt)
            log = nb.nbody_step(ctx, xs, vs, mt, at, False, T)
            lam = torch.ones_like(xt)
            gx, gv, gm, gp = nb.nbody_adjoint_params(ctx, xt, vt, mt, T, 3, lam, lam)
            nb.nbody_sync(ctx)  # raises NBodyError(EINTERNAL) if an index check failed
            ctx.close()
            a_ref, phi_ref = oracle.forces(x, m, G=G, eps=eps)
            xr, vr, ar, _ = oracle.kdk(x, v, m, G, eps, dt, T)
            gxr, gvr, gmr, _ = oracle.adjoint_params(x, v, m, G, eps, dt, T, np.ones((n, 3)), np.ones((n, 3)))
            if n > 1:
                assert force_rel_err(a.cpu().numpy(), a_ref).max() <= ftol, (n, prec)
                assert force_rel_err(at.cpu().numpy(), ar).max() <= ftol, (n, prec)
            assert np.abs(xs.cpu().numpy() - xr).max() <= 1e-9 * max(1.0, np.abs(xr).max()), (n, prec)
            assert elem_rel_err(gx.cpu().numpy(), gxr).max() <= gtol, (n, prec)
            assert elem_rel_err(gv.cpu().numpy(), gvr).max() <= gtol, (n, prec)
    # several systems with empty ones, and the Lennard-Jones law with walls
    sizes = [0, 5, 130, 0, 1, 257]
    ens = inputs.ensemble(len(sizes), seed=3, sizes=np.array(sizes))
    off = [int(o) for o in ens.offsets]
    for prec in (nb.FP64, nb.MIXED):
        ctx = nb.nbody_init(G=G, eps=eps, dt=dt, precision=prec, offsets=off, energy_every=1, flags=nb.FLAG_GRAPH)
        xt, vt, mt = to_dev(ens.x, ens.v, ens.m)
        nb.nbody_step(ctx, xt, vt, mt, torch.empty_like(xt), False, 3)
        nb.nbody_sync(ctx)
        ctx.close()
    xg, vg, mg, box = inputs.lj_gas(500, seed=5, density=0.1)
    for prec in (nb.FP64, nb.MIXED):
        ctx = nb.nbody_init(law=nb.LENNARD_JONES, precision=prec, n=500, dt=5e-3, box=box, energy_every=1)
        xt, vt, mt = to_dev(xg, vg, mg)
        nb.nbody_step(ctx, xt, vt, mt, torch.empty_like(xt), False, 3)
        nb.nbody_sync(ctx)
        ctx.close()
    print("DEBUG_BUILD_OK")
""")


def test_debug_build_tiny_and_ragged_sizes():
    from paper_2511_02655_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, NBODY_DEBUG_LIB="1")
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "DEBUG_BUILD_OK" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
