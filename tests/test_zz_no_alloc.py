"""nbody_forces_noalloc, the entry point for callers that cannot allocate
device memory (it takes no context and uses a fixed static device array as
scratch), against the regular nbody_forces entry point and the FP64 oracle.

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
# the mixed potential per body: max (J - 1) 2^-24 < 3e-5 for a float32 tile sum of J <= 512
# same-sign terms, median 1e-6 (as in the other GPU tests)
PHI_MED, PHI_MAX = 1e-6, 3e-5
EINVAL = 1


def _check_phi(phi, phi_ref):
    e = np.abs(np.asarray(phi) - phi_ref) / np.abs(phi_ref)
    assert np.median(e) <= PHI_MED and e.max() <= PHI_MAX, (np.median(e), e.max())


def _raw_call(nb, x, m, n, G, eps, a, phi, stream=None):
    """The C entry point with plain pointers (outputs preallocated by the caller)."""
    import torch
    lib = nb.load()
    ptr = lambda t: ctypes.c_void_p(t) if isinstance(t, int) else (None if t is None else ctypes.c_void_p(t.data_ptr()))
    s = torch.cuda.current_stream().cuda_stream if stream is None else stream
    return lib.nbody_forces_noalloc(ptr(x), ptr(m), n, G, eps, ptr(a), ptr(phi), nb.ctx_ptr(s))


def _noalloc_via_abi(nb, x, m, G, eps, with_phi=True):
    """Calls the C entry point directly; outputs are preallocated by the test."""
    import torch
    n = m.shape[0]
    a = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    phi = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda") if with_phi else None
    st = _raw_call(nb, x, m, n, G, eps, a, phi)
    assert st == 0, nb.nbody_last_error(None)
    torch.cuda.synchronize()
    return a, phi


def test_noalloc_matches_regular_entry_point_on_two_calls_in_a_row(nb):
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
        _check_phi(phi_na, phi_ref)
        # and against the FP64 oracle on a sample of bodies
        idx = inputs.sample_indices(n, 256, seed=5)
        a_or, phi_or = oracle.forces_at(x, m, idx, G=G, eps=eps)
        e = force_rel_err(a_na[idx], a_or)
        assert np.median(e) <= MIX_MED and e.max() <= MIX_MAX
        _check_phi(phi_na[idx], phi_or)
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_static_scratch(nb):
    import torch
    x = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    st = _raw_call(nb, x, x, nb.NOALLOC_MAX_BODIES + 1, 1.0, 0.01, x, None)
    assert st == EINVAL
    assert "NBODY_NOALLOC_MAX_BODIES" in nb.nbody_last_error(None)


def test_noalloc_tight_pairs_far_from_origin(nb):
    """Pairs ~eps/2 apart around |x| ~ 100: float32 staging alone carries ~4e-6 absolute error,
    several % of the separation; the refinement from the staged remainders keeps the bounds."""
    rng = np.random.default_rng(5)
    centres = rng.normal(size=(500, 3))
    centres = 100.0 * centres / np.linalg.norm(centres, axis=1, keepdims=True)
    eps = 1e-3
    x = np.concatenate([centres, centres + rng.normal(size=(500, 3)) * 0.5 * eps])
    m = np.full(1000, 1e-3)
    xt, mt = to_dev(x, m)
    a, phi = _noalloc_via_abi(nb, xt, mt, 1.0, eps)
    a_ref, phi_ref = oracle.forces(x, m, G=1.0, eps=eps)
    e = force_rel_err(a.cpu().numpy(), a_ref)
    assert np.median(e) <= MIX_MED and e.max() <= MIX_MAX, (np.median(e), e.max())
    _check_phi(phi.cpu().numpy(), phi_ref)


def test_noalloc_two_spheres_1m_sampled(nb):
    """The 1 048 576-body two-sphere input (eps = 0.002), the largest size the scratch takes,
    against the oracle on 1024 sampled bodies."""
    n, eps = nb.NOALLOC_MAX_BODIES, 0.002
    x, v, m = inputs.two_spheres(n, seed=3)
    xt, mt = to_dev(x, m)
    a, _ = _noalloc_via_abi(nb, xt, mt, 1.0, eps, with_phi=False)
    idx = inputs.sample_indices(n, 1024, seed=17)
    a_ref, _ = oracle.forces_at(x, m, idx, G=1.0, eps=eps)
    e = force_rel_err(a.cpu().numpy()[idx], a_ref)
    assert np.median(e) <= MIX_MED and e.max() <= MIX_MAX, (np.median(e), e.max())


@pytest.mark.parametrize("n", [1, 2, 3])
def test_noalloc_tiny_systems_without_phi(nb, n):
    """n = 1: only the masked self pair (a = 0, phi = 0); n = 2, 3 against the oracle; phi = NULL."""
    x, v, m = inputs.plummer(n, seed=40 + n)
    xt, mt = to_dev(x, m)
    a, _ = _noalloc_via_abi(nb, xt, mt, 1.0, 0.05, with_phi=False)
    a2, phi2 = _noalloc_via_abi(nb, xt, mt, 1.0, 0.05, with_phi=True)
    a, a2, phi2 = (t.cpu().numpy() for t in (a, a2, phi2))
    assert np.array_equal(a, a2)
    if n == 1:
        assert np.all(a == 0) and np.all(phi2 == 0)
        return
    a_ref, phi_ref = oracle.forces(x, m, G=1.0, eps=0.05)
    assert force_rel_err(a, a_ref).max() <= MIX_MAX
    _check_phi(phi2, phi_ref)


def test_noalloc_rejects_host_and_short_buffers(nb):
    """A host pointer and a device buffer shorter than n bodies are refused before any launch."""
    import torch
    n = 1000
    x, v, m = inputs.plummer(n, seed=44)
    xt, mt = to_dev(x, m)
    a = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    xh = torch.from_numpy(x.copy())
    assert _raw_call(nb, xh, mt, n, 1.0, 0.01, a, None) == EINVAL
    assert "device memory" in nb.nbody_last_error(None) or "CUDA pointer" in nb.nbody_last_error(None)
    # a buffer of its own allocation that holds n - 1 rows of a
    cudart = ctypes.CDLL("libcudart.so.13")
    p = ctypes.c_void_p()
    assert cudart.cudaMalloc(ctypes.byref(p), ctypes.c_size_t((n - 1) * 3 * 8)) == 0
    try:
        st = _raw_call(nb, xt, mt, n, 1.0, 0.01, p.value, None)
        assert st == EINVAL and "needs" in nb.nbody_last_error(None), nb.nbody_last_error(None)
    finally:
        cudart.cudaFree(p)
    # the Python wrapper checks the shapes of caller-supplied outputs as well
    with pytest.raises(ValueError):
        nb.nbody_forces_noalloc(xt, mt, 1.0, 0.01, a=torch.empty(n, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        nb.nbody_forces_noalloc(xt, mt, 1.0, 0.01, a=a.float())


def test_noalloc_python_wrapper_matches_raw_call(nb):
    import torch
    x, v, m = inputs.plummer(3001, seed=45)
    xt, mt = to_dev(x, m)
    a_raw, phi_raw = _noalloc_via_abi(nb, xt, mt, 1.2, 0.02)
    a, phi = nb.nbody_forces_noalloc(xt, mt, 1.2, 0.02, phi=torch.empty_like(mt))
    torch.cuda.synchronize()
    assert torch.equal(a, a_raw) and torch.equal(phi, phi_raw)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):  # the wrapper queues on the current stream
        a2, none = nb.nbody_forces_noalloc(xt, mt, 1.2, 0.02)
    s.synchronize()
    assert none is None and torch.equal(a2, a_raw)


def test_noalloc_second_call_leaves_free_memory_unchanged(nb):
    """After the first call on the device (which loads the device code and its static array),
    a call allocates nothing: the device's free memory is the same before and after."""
    import torch
    x, v, m = inputs.plummer(50000, seed=46)
    xt, mt = to_dev(x, m)
    a = torch.empty((50000, 3), dtype=torch.float64, device="cuda")
    phi = torch.empty(50000, dtype=torch.float64, device="cuda")
    assert _raw_call(nb, xt, mt, 50000, 1.0, 0.01, a, phi) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert _raw_call(nb, xt, mt, 50000, 1.0, 0.01, a, phi) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
