"""nbody_forces_noalloc, the entry point for callers that cannot allocate
device memory (it takes no context and uses a fixed static device array as
scratch), against the regular nbody_forces entry point.

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test first. It must pass both in a fresh process
and after the other tests.
"""

import ctypes

import numpy as np
import pytest

import oracle
from paper_2511_02655_gb300 import inputs
from helpers import force_rel_err, to_dev

pytestmark = pytest.mark.gpu

MIX_MED, MIX_MAX = 1e-6, 1e-4  # the mixed-path bounds used throughout the GPU tests


def _noalloc_via_abi(nb, x, m, G, eps):
    """Calls the C entry point directly; outputs are preallocated by the test."""
    import torch
    lib = nb.load()
    n = m.shape[0]
    a = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    phi = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.nbody_forces_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(m.data_ptr()), n, G, eps,
                                  ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
                                  nb.ctx_ptr(torch.cuda.current_stream().cuda_stream))
    assert st == 0, nb.nbody_last_error(None)
    torch.cuda.synchronize()
    return a, phi


def test_noalloc_matches_regular_entry_point_on_two_calls_in_a_row(nb):
    import torch
    cases = [(inputs.plummer(20000, seed=31), 1.0, 0.01), (inputs.plummer(4097, seed=32), 0.7, 0.03)]
    for (x, v, m), G, eps in cases:  # the second call reuses the static scratch left by the first
        n = m.shape[0]
        xt, mt = to_dev(x, m)
        a_na, phi_na = _noalloc_via_abi(nb, xt, mt, G, eps)
        ctx = nb.nbody_init(G=G, eps=eps, dt=1e-3, precision=nb.MIXED, n=n)
        a_ref, phi_ref = nb.nbody_forces(ctx, xt, mt)
        nb.nbody_sync(ctx)
        a_na, phi_na, a_ref, phi_ref = (t.cpu().numpy() for t in (a_na, phi_na, a_ref, phi_ref))
        e = force_rel_err(a_na, a_ref)
        assert np.median(e) <= MIX_MED and e.max() <= MIX_MAX, (np.median(e), e.max())
        assert np.abs(phi_na - phi_ref).max() <= 1e-5 * np.abs(phi_ref).max()
        # and against the FP64 oracle on a sample of bodies
        idx = inputs.sample_indices(n, 256, seed=5)
        a_or, _ = oracle.forces_at(x, m, idx, G=G, eps=eps)
        e = force_rel_err(a_na[idx], a_or)
        assert e.max() <= MIX_MAX
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_static_scratch(nb):
    import torch
    lib = nb.load()
    x = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    too_many = nb.NOALLOC_MAX_BODIES + 1
    st = lib.nbody_forces_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), too_many, 1.0,
                                  0.01, ctypes.c_void_p(x.data_ptr()), None, None)
    assert st == 1
    assert "NBODY_NOALLOC_MAX_BODIES" in nb.nbody_last_error(None)
