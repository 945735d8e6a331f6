"""C-ABI surface checks that need no GPU: the library builds for sm_103a,
loads, exports every entry point include/oci.h declares, and rejects invalid
problems before touching the device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2305_13555_gb300 as pkg
import workloads
from paper_2305_13555_gb300 import build as pbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared_functions():
    names = []
    for h in HEADERS:
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(", txt, re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return pkg.load_library()


def test_header_declares_the_core_calls():
    names = _declared_functions()
    for n in ("oci_create", "oci_step", "si_step", "oci_fluxes", "oci_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", pbuild.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, re.M))
    missing = [n for n in _declared_functions() if n not in exported]
    assert not missing, missing
    # and the binding gives every one a signature
    assert not [n for n in _declared_functions() if n not in pkg.SIGNATURES]


def test_library_is_sm103a_only():
    objs = [os.path.join(pbuild.OUT_DIR, s.replace(".cu", ".o")) for s in pbuild.SOURCES]
    pbuild.build()
    for o in objs:
        r = subprocess.run(["cuobjdump", "--list-elf", o], capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("cuobjdump unavailable")
        archs = set(re.findall(r"sm_(\d+a?)", r.stdout))
        assert archs <= {"103a"}, archs


def test_strerror(lib):
    assert pkg.oci_strerror(pkg.OCI_OK) == "ok"
    assert "not converged" in pkg.oci_strerror(pkg.OCI_ENOTCONV)
    assert pkg.oci_strerror(999) == "unknown status"


def _bad(prob, **kw):
    with pytest.raises(pkg.OciError) as e:
        pkg.oci_create(prob, **kw)
    return e.value.code


@pytest.mark.parametrize("mutate", [
    lambda p: p.update(n_ord=7),
    lambda p: p.update(n_ord=258),
    lambda p: p.update(n_ord=0),
    lambda p: p.update(v=-1.0),
    lambda p: p.update(dt=0.0),
    lambda p: p["dx"].__setitem__(3, 0.0),
    lambda p: p["sigma_s"].__setitem__(2, p["sigma_t"][2] * 1.5),
    lambda p: p["sigma_t"].__setitem__(1, float("nan")),
    lambda p: p.update(bc_left=7),
    lambda p: p.update(bc_right="incident", psi_bc_right=None),
])
def test_invalid_problems_rejected_before_device_use(lib, mutate):
    p = workloads.random_small(seed=1, J=8, N=4, with_bc=False, with_psi0=False)
    mutate(p)
    assert _bad(p) == pkg.OCI_EINVAL


def test_invalid_iteration_controls(lib):
    p = workloads.random_small(seed=1, J=8, N=4)
    assert _bad(p, max_iter=0) == pkg.OCI_EINVAL
    assert _bad(p, tol=-1.0) == pkg.OCI_EINVAL
    assert _bad(p, precision=5) == pkg.OCI_EINVAL


def test_null_handle_calls(lib):
    assert lib.oci_step(None, None) == pkg.OCI_EINVAL
    assert lib.si_step(None, None) == pkg.OCI_EINVAL
    assert lib.oci_fluxes(None, None) == pkg.OCI_EINVAL
    assert lib.oci_set_iteration(None, 1e-8, 10, 0) == pkg.OCI_EINVAL
    assert lib.oci_set_halo(None, pkg.OCI_HALO_BF16) == pkg.OCI_EINVAL
    assert lib.oci_step_async(None) == pkg.OCI_EINVAL
    assert lib.oci_step_wait(None, None) == pkg.OCI_EINVAL
    assert lib.oci_fluxes_async(None, None) == pkg.OCI_EINVAL
    assert lib.oci_sync(None) == pkg.OCI_EINVAL
    lib.oci_destroy(None)
