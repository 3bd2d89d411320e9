"""CPU oracle for the softened-gravity N-body hot path -- TEST INFRASTRUCTURE.

Plain FP64 C (``nbody_oracle.c``) reached through ctypes. Only the tests, the
smoke check and the benchmark's CPU-baseline leg use it; the GPU library
neither imports nor links it, and the two share no code. Inputs come from
``paper_2511_02655_gb300.inputs`` (initial conditions only).

What each function computes (softened Newtonian gravity in the all-pairs,
Verlet half-step, fused-energy structure of the paper's N-body miniapp,
Sec. II-A and Sec. V-B, Sec. VI):

* ``forces``      a_i = G sum_{j!=i} m_j d_ij / s_ij^3, phi_i = -G sum_{j!=i} m_j / s_ij
* ``forces_at``   the same for a subset of bodies, each against all N
* ``energy``      [E, K, U, Px, Py, Pz, Lx, Ly, Lz] with U over pairs i<j
* ``kdk``         leapfrog kick-drift-kick steps, one force evaluation per step
* ``force_vjp``   w -> (dL/dx, dL/dm) through a(x, m) for dL/da = w
* ``adjoint``     gradients of a final-state loss w.r.t. x0, v0, m through KDK
* ``virial``      (K, W, -2K/W) with the Clausius virial W = sum_{i<j} (x_i - x_j) . F_ij
* ``param_vjp``   w -> (sum_k w_k . da_k/dG, sum_k w_k . da_k/deps)
* ``adjoint_params``  ``adjoint`` plus dL/dG and dL/deps
* ``lj_*``         the same for the paper's Lennard-Jones pair law (Eq. 1):
                   a_i = F_i / m_i, phi_i = sum_j V(r_ij) / m_i, and KDK with
                   reflecting walls of the box [0, box]^3
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nbody_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            d, i64, i32, p = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
            lib.oracle_default_threads.restype = i32
            lib.oracle_forces.argtypes = [i64, p, p, d, d, p, p, i32]
            lib.oracle_forces_at.argtypes = [i64, p, p, d, d, p, i64, p, p, i32]
            lib.oracle_energy.argtypes = [i64, p, p, p, d, d, p, i32]
            lib.oracle_kdk.argtypes = [i64, p, p, p, d, d, d, i32, p, i32, i32, p, i32]
            lib.oracle_force_vjp.argtypes = [i64, p, p, p, d, d, p, p, i32]
            lib.oracle_adjoint.argtypes = [i64, p, p, p, d, d, d, i32, p, p, p, p, p, i32]
            lib.oracle_param_vjp.argtypes = [i64, p, p, p, d, d, p, i32]
            lib.oracle_virial.argtypes = [i64, p, p, p, i32, d, d, d, d, d, p, i32]
            lib.oracle_adjoint_params.argtypes = [i64, p, p, p, d, d, d, i32, p, p, p, p, p, p, i32]
            lib.oracle_lj_forces.argtypes = [i64, p, p, d, d, d, p, p, i32]
            lib.oracle_lj_forces_at.argtypes = [i64, p, p, d, d, d, p, i64, p, p, i32]
            lib.oracle_lj_energy.argtypes = [i64, p, p, p, d, d, d, p, i32]
            lib.oracle_lj_kdk.argtypes = [i64, p, p, p, d, d, d, d, d, i32, p, i32, i32, p, i32]
            for f in ("oracle_forces", "oracle_forces_at", "oracle_energy", "oracle_kdk",
                      "oracle_force_vjp", "oracle_adjoint", "oracle_param_vjp", "oracle_adjoint_params", "oracle_virial",
                      "oracle_lj_forces", "oracle_lj_forces_at",
                      "oracle_lj_energy", "oracle_lj_kdk"):
                getattr(lib, f).restype = i32
            _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


def default_threads() -> int:
    return int(_load().oracle_default_threads())


def forces(x, m, G=1.0, eps=0.0, threads=0, with_phi=True):
    """All-pairs accelerations a [N,3] and potentials phi [N] (self pair excluded)."""
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    a = np.zeros((n, 3))
    phi = np.zeros(n) if with_phi else None
    _check(_load().oracle_forces(n, _ptr(x), _ptr(m), G, eps, _ptr(a), _ptr(phi), threads), "oracle_forces")
    return (a, phi) if with_phi else a


def forces_at(x, m, idx, G=1.0, eps=0.0, threads=0):
    """a [k,3], phi [k] for the bodies ``idx`` against all N bodies."""
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    k = idx.shape[0]
    a = np.zeros((k, 3))
    phi = np.zeros(k)
    _check(_load().oracle_forces_at(n, _ptr(x), _ptr(m), G, eps, _ptr(idx), k, _ptr(a), _ptr(phi), threads),
           "oracle_forces_at")
    return a, phi


def energy(x, v, m, G=1.0, eps=0.0, threads=0):
    """[E, K, U, Px, Py, Pz, Lx, Ly, Lz] (float64[9])."""
    m = _f64(m)
    n = m.shape[0]
    x, v = _f64(x, (n, 3)), _f64(v, (n, 3))
    out = np.zeros(9)
    _check(_load().oracle_energy(n, _ptr(x), _ptr(v), _ptr(m), G, eps, _ptr(out), threads), "oracle_energy")
    return out


def kdk(x, v, m, G, eps, dt, n_steps, a=None, energy_every=0, threads=0):
    """KDK leapfrog; returns (x, v, a, energy_log) on new arrays.

    ``a`` is a(x) at entry if given (else computed); energy_log is
    [n_steps // energy_every, 9] when energy_every > 0, else None.
    """
    m = _f64(m)
    n = m.shape[0]
    x, v = _f64(x, (n, 3)).copy(), _f64(v, (n, 3)).copy()
    a_valid = a is not None
    a = _f64(a, (n, 3)).copy() if a_valid else np.zeros((n, 3))
    nrec = n_steps // energy_every if energy_every > 0 else 0
    log = np.zeros((nrec, 9)) if nrec else None
    _check(_load().oracle_kdk(n, _ptr(x), _ptr(v), _ptr(m), G, eps, dt, int(n_steps), _ptr(a), int(a_valid),
                              int(energy_every), _ptr(log), threads), "oracle_kdk")
    return x, v, a, log


def force_vjp(x, m, w, G=1.0, eps=0.0, threads=0):
    """(gx [N,3], gm [N]) = w^T d a / d(x, m)."""
    m = _f64(m)
    n = m.shape[0]
    x, w = _f64(x, (n, 3)), _f64(w, (n, 3))
    gx, gm = np.zeros((n, 3)), np.zeros(n)
    _check(_load().oracle_force_vjp(n, _ptr(x), _ptr(m), _ptr(w), G, eps, _ptr(gx), _ptr(gm), threads),
           "oracle_force_vjp")
    return gx, gm


def adjoint(x0, v0, m, G, eps, dt, n_steps, lam_xT, lam_vT, threads=0):
    """(g_x0, g_v0, g_m) for a loss with dL/dx_T = lam_xT and dL/dv_T = lam_vT."""
    m = _f64(m)
    n = m.shape[0]
    x0, v0 = _f64(x0, (n, 3)), _f64(v0, (n, 3))
    lx, lv = _f64(lam_xT, (n, 3)), _f64(lam_vT, (n, 3))
    gx, gv, gm = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    _check(_load().oracle_adjoint(n, _ptr(x0), _ptr(v0), _ptr(m), G, eps, dt, int(n_steps), _ptr(lx), _ptr(lv),
                                  _ptr(gx), _ptr(gv), _ptr(gm), threads), "oracle_adjoint")
    return gx, gv, gm


def virial(x, v, m, G=1.0, eps=0.0, threads=0, law=0, eps_lj=1.0, sigma=1.0, soft=0.0):
    """(K, W, Q): kinetic energy, Clausius virial (pair form), virial ratio -2K/W.

    law 0: softened gravity (G, eps); law 1: Lennard-Jones (eps_lj, sigma, soft)."""
    m = _f64(m)
    n = m.shape[0]
    x, v = _f64(x, (n, 3)), _f64(v, (n, 3))
    out = np.zeros(3)
    _check(_load().oracle_virial(n, _ptr(x), _ptr(v), _ptr(m), int(law), G, eps, eps_lj, sigma, soft, _ptr(out),
                                 threads), "oracle_virial")
    return out


def param_vjp(x, m, w, G=1.0, eps=0.0, threads=0):
    """(sum_k w_k . da_k/dG, sum_k w_k . da_k/deps) at positions x."""
    m = _f64(m)
    n = m.shape[0]
    x, w = _f64(x, (n, 3)), _f64(w, (n, 3))
    out = np.zeros(2)
    _check(_load().oracle_param_vjp(n, _ptr(x), _ptr(m), _ptr(w), G, eps, _ptr(out), threads), "oracle_param_vjp")
    return float(out[0]), float(out[1])


def adjoint_params(x0, v0, m, G, eps, dt, n_steps, lam_xT, lam_vT, threads=0):
    """(g_x0, g_v0, g_m, (dL/dG, dL/deps)) for a loss with dL/dx_T = lam_xT, dL/dv_T = lam_vT."""
    m = _f64(m)
    n = m.shape[0]
    x0, v0 = _f64(x0, (n, 3)), _f64(v0, (n, 3))
    lx, lv = _f64(lam_xT, (n, 3)), _f64(lam_vT, (n, 3))
    gx, gv, gm, gp = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n), np.zeros(2)
    _check(_load().oracle_adjoint_params(n, _ptr(x0), _ptr(v0), _ptr(m), G, eps, dt, int(n_steps), _ptr(lx),
                                         _ptr(lv), _ptr(gx), _ptr(gv), _ptr(gm), _ptr(gp), threads),
           "oracle_adjoint_params")
    return gx, gv, gm, (float(gp[0]), float(gp[1]))


def trajectory_loss(x0, v0, m, G, eps, dt, n_steps, target, threads=0):
    """L = sum_i |x_i(T) - t_i|^2 after n_steps KDK steps from (x0, v0)."""
    xT, _, _, _ = kdk(x0, v0, m, G, eps, dt, n_steps, threads=threads)
    return float(((xT - target) ** 2).sum())


def lj_forces(x, m, eps_lj=1.0, sigma=1.0, soft=0.0, threads=0):
    """Lennard-Jones accelerations a [N,3] and potentials per unit mass phi [N]."""
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    a, phi = np.zeros((n, 3)), np.zeros(n)
    _check(_load().oracle_lj_forces(n, _ptr(x), _ptr(m), eps_lj, sigma, soft, _ptr(a), _ptr(phi), threads),
           "oracle_lj_forces")
    return a, phi


def lj_forces_at(x, m, idx, eps_lj=1.0, sigma=1.0, soft=0.0, threads=0):
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    k = idx.shape[0]
    a, phi = np.zeros((k, 3)), np.zeros(k)
    _check(_load().oracle_lj_forces_at(n, _ptr(x), _ptr(m), eps_lj, sigma, soft, _ptr(idx), k, _ptr(a), _ptr(phi),
                                       threads), "oracle_lj_forces_at")
    return a, phi


def lj_energy(x, v, m, eps_lj=1.0, sigma=1.0, soft=0.0, threads=0):
    """[E, K, U, Px, Py, Pz, Lx, Ly, Lz] with U the Lennard-Jones pair sum."""
    m = _f64(m)
    n = m.shape[0]
    x, v = _f64(x, (n, 3)), _f64(v, (n, 3))
    out = np.zeros(9)
    _check(_load().oracle_lj_energy(n, _ptr(x), _ptr(v), _ptr(m), eps_lj, sigma, soft, _ptr(out), threads),
           "oracle_lj_energy")
    return out


def lj_kdk(x, v, m, eps_lj, sigma, soft, box, dt, n_steps, a=None, energy_every=0, threads=0):
    """KDK leapfrog of the Lennard-Jones gas with reflecting walls (box > 0); returns (x, v, a, log)."""
    m = _f64(m)
    n = m.shape[0]
    x, v = _f64(x, (n, 3)).copy(), _f64(v, (n, 3)).copy()
    a_valid = a is not None
    a = _f64(a, (n, 3)).copy() if a_valid else np.zeros((n, 3))
    nrec = n_steps // energy_every if energy_every > 0 else 0
    log = np.zeros((nrec, 9)) if nrec else None
    _check(_load().oracle_lj_kdk(n, _ptr(x), _ptr(v), _ptr(m), eps_lj, sigma, soft, box, dt, int(n_steps),
                                 _ptr(a), int(a_valid), int(energy_every), _ptr(log), threads), "oracle_lj_kdk")
    return x, v, a, log
