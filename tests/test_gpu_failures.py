"""Failure detection without a GPU fault. Scratch-allocation failures are injected on
the host (NBODY_FAULT_ALLOC=k fails the k-th allocation of a context): whichever call
allocates reports NBODY_ENOMEM with the reason, nothing is launched on a half-built
context, destroying it returns every byte, and a fresh context works. Non-finite
results are reported by nbody_sync (see also the coincident-body tests)."""

import numpy as np
import pytest

import oracle
from paper_2511_02655_gb300 import inputs
from helpers import force_rel_err, to_dev

pytestmark = pytest.mark.gpu


def _workload(nb, torch, xt, vt, mt, lam, stage):
    """init, forces, steps with energy records, energy, virial, adjoint with parameters;
    stage[0] names the call in progress."""
    stage[0] = "init"
    ctx = nb.nbody_init(G=1.0, eps=0.02, dt=1e-3, precision=nb.MIXED, n=xt.shape[0], energy_every=2)
    try:
        stage[0] = "forces"
        a, phi = nb.nbody_forces(ctx, xt, mt)
        a0 = a.clone()
        xs, vs = xt.clone(), vt.clone()
        stage[0] = "step"
        nb.nbody_step(ctx, xs, vs, mt, a, True, 4)
        stage[0] = "energy"
        nb.nbody_energy(ctx, xs, vs, mt)
        stage[0] = "virial"
        nb.nbody_virial(ctx, xs, vs, mt)
        stage[0] = "adjoint"
        nb.nbody_adjoint_params(ctx, xt, vt, mt, 6, 3, lam, torch.zeros_like(lam))
        nb.nbody_sync(ctx)
        stage[0] = "done"
        return a0.cpu().numpy()
    finally:
        ctx.close()


def test_injected_allocation_failures(nb, monkeypatch):
    """Fail the k-th allocation for k = 1, 2, ... until a run completes: every failure is
    NBODY_ENOMEM from the call that allocates, the context gives all memory back, a fresh
    context right after is correct, and failures are seen in init and in the adjoint's
    first call (forces, steps, energies and virials allocate nothing after init)."""
    import torch
    n = 600
    x, v, m = inputs.plummer(n, seed=44)
    xt, vt, mt, lam = to_dev(x, v, m, np.ones((n, 3)))
    ref, _ = oracle.forces(x, m, G=1.0, eps=0.02)
    failed_in = []
    for k in range(1, 200):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        monkeypatch.setenv("NBODY_FAULT_ALLOC", str(k))
        stage = [None]
        try:
            a = _workload(nb, torch, xt, vt, mt, lam, stage)
        except nb.NBodyError as e:
            assert e.status == 2 and "injected allocation failure" in str(e), (k, stage[0], str(e))
            failed_in.append(stage[0])
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] >= free0 - (2 << 20), (k, stage[0])
        monkeypatch.delenv("NBODY_FAULT_ALLOC")
        a = _workload(nb, torch, xt, vt, mt, lam, [None])
        assert force_rel_err(a, ref).max() <= 1e-4
        if stage[0] == "done":
            break
    assert stage[0] == "done", "the workload never completed"
    assert set(failed_in) == {"init", "adjoint"}, failed_in


def test_first_allocation_fails_in_init(nb, monkeypatch):
    monkeypatch.setenv("NBODY_FAULT_ALLOC", "1")
    with pytest.raises(nb.NBodyError) as ei:
        nb.nbody_init(G=1.0, eps=0.02, dt=1e-3, precision=nb.FP64, n=100)
    assert ei.value.status == 2
