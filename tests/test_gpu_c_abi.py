"""The C ABI from a plain C program (tests/c_abi_client.c, built here with gcc
against include/nbody.h and linked to libnbody.so): status codes, host-pointer
rejection, forces, KDK steps, the energy reduction and the allocation-free
entry point, compared with the FP64 CPU oracle."""

import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from helpers import force_rel_err

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    import paper_2511_02655_gb300 as nb
    from paper_2511_02655_gb300 import build
    lib = build.build()
    d = tmp_path_factory.mktemp("cabi")
    exe = str(d / "c_abi_client")
    cuda = "/usr/local/cuda"
    cmd = ["gcc", "-O2", "-std=c11", "-I" + os.path.join(ROOT, "include"), "-I" + cuda + "/include",
           os.path.join(ROOT, "tests", "c_abi_client.c"), "-o", exe, lib, "-L" + cuda + "/lib64", "-lcudart", "-lm",
           "-Wl,-rpath," + os.path.dirname(lib) + ":" + cuda + "/lib64"]
    subprocess.run(cmd, check=True)
    assert nb.lib_path() == lib
    return exe


@pytest.mark.parametrize("prec", [0, 1])
def test_c_client(client, prec):
    n = 3001
    with tempfile.TemporaryDirectory() as td:
        out = os.path.join(td, "res.bin")
        r = subprocess.run([client, str(n), str(prec), out], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stdout + r.stderr
        assert r.stdout.startswith("ok")
        raw = np.fromfile(out, dtype=np.float64)
    k = 0

    def take(cnt, shape):
        nonlocal k
        a = raw[k:k + cnt].reshape(shape)
        k += cnt
        return a

    x, v, m = take(3 * n, (n, 3)), take(3 * n, (n, 3)), take(n, (n,))
    a, x1, a1, e, ana = take(3 * n, (n, 3)), take(3 * n, (n, 3)), take(3 * n, (n, 3)), take(9, (9,)), \
        take(3 * n, (n, 3))
    assert k == raw.size
    a_ref, _ = oracle.forces(x, m, G=1.0, eps=0.02)
    tol = 1e-12 if prec == 0 else 1e-4
    assert force_rel_err(a, a_ref).max() <= tol
    xr, vr, ar, _ = oracle.kdk(x, v, m, 1.0, 0.02, 1e-3, 5, a=a_ref)
    assert np.abs(x1 - xr).max() <= (1e-13 if prec == 0 else 1e-9)
    E = oracle.energy(x, v, m, G=1.0, eps=0.02)
    assert abs(e[0] - E[0]) <= (1e-12 if prec == 0 else 1e-6) * abs(E[0])
    assert force_rel_err(ana, a_ref).max() <= 1e-4
