"""Shared helpers for the GPU parity tests (no method arithmetic here)."""

import numpy as np


def force_rel_err(a, a_ref, guard=1e-3):
    """Per-body relative error |a - a_ref| / |a_ref|; bodies whose reference
    force is below guard * rms(|a_ref|) are normalised by that floor instead
    (cancellation guard)."""
    a, a_ref = np.asarray(a), np.asarray(a_ref)
    nrm = np.linalg.norm(a_ref, axis=1)
    rms = np.sqrt(np.mean(nrm ** 2)) if len(nrm) else 1.0
    return np.linalg.norm(a - a_ref, axis=1) / np.maximum(nrm, guard * rms)


def to_dev(*arrs, device="cuda:0"):
    import torch
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(device) for a in arrs)


def to_np(*ts):
    return tuple(t.detach().cpu().numpy() for t in ts)


def elem_rel_err(g, g_ref, guard=1e-3):
    """Per-element relative error |g - g_ref| / max(|g_ref|, guard * rms(g_ref)), over every
    component of every body (cancellation guard as in force_rel_err)."""
    g = np.asarray(g, dtype=np.float64).ravel()
    g_ref = np.asarray(g_ref, dtype=np.float64).ravel()
    rms = np.sqrt(np.mean(g_ref ** 2)) if g_ref.size else 1.0
    return np.abs(g - g_ref) / np.maximum(np.abs(g_ref), guard * rms)


def assert_elem_close(g, g_ref, tol, what=""):
    """Every element within tol (elem_rel_err); the message names the worst element."""
    e = elem_rel_err(g, g_ref)
    if e.size:
        k = int(np.argmax(e))
        assert e[k] <= tol, f"{what}: max per-element rel err {e[k]:.3e} at flat index {k} (tol {tol:.1e})"
    return e
