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
