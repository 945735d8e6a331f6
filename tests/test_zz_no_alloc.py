"""oci_nn_forward_noalloc: network inference whose scratch is a fixed array in
the library, for callers that cannot allocate device memory or pass a
workspace (see include/oci_nn.h).  Checked through the C ABI against
oci_nn_forward (caller workspace) on two calls in a row with different inputs,
so stale contents of the shared array would show; also the size limit.  Runs
alone in a fresh process or after the other tests (it builds and loads the
library itself)."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2305_13555_gb300 as pkg

pytestmark = pytest.mark.gpu

MAX_CELLS = 16384  # OCI_NN_NOALLOC_MAX_CELLS


@pytest.fixture(scope="module")
def lib():
    from paper_2305_13555_gb300 import build
    build.build()
    return pkg.load_library()


def _noalloc(lib, params, x, J, out):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.oci_nn_forward_noalloc(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(x.data_ptr()), J,
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def test_noalloc_forward_matches_workspace_forward_twice(lib):
    g = np.random.default_rng(11)
    n = pkg.oci_nn_param_count()
    params = torch.tensor(g.normal(0, 0.15, n).astype(np.float32), device="cuda")
    for J in (5000, MAX_CELLS):
        xs = [torch.tensor(g.normal(0, 1, (1, 13, J)).astype(np.float32), device="cuda") for _ in range(2)]
        ws = torch.empty(pkg.oci_nn_workspace_bytes(1, J), dtype=torch.uint8, device="cuda")
        for x in xs:  # two calls in a row, different inputs
            ref = torch.empty((1, 4, J), dtype=torch.float32, device="cuda")
            pkg.oci_nn_forward(params, x, ref, ws)
            out = torch.full((1, 4, J), float("nan"), dtype=torch.float32, device="cuda")
            assert _noalloc(lib, params, x, J, out) == 0
            torch.cuda.synchronize()
            r, o = ref.cpu().numpy(), out.cpu().numpy()
            assert np.isfinite(o).all()
            # one kernel per layer against oci_nn_forward's fused kernel, with the same
            # arithmetic per output element: bit for bit
            assert np.array_equal(o, r), np.abs(o - r).max()


def test_noalloc_call_allocates_no_device_memory(lib):
    """After the first call on the device (its set-up: the array's address), a
    call leaves the device's free memory unchanged."""
    g = np.random.default_rng(12)
    J = 4096
    params = torch.tensor(g.normal(0, 0.15, pkg.oci_nn_param_count()).astype(np.float32), device="cuda")
    x = torch.tensor(g.normal(0, 1, (1, 13, J)).astype(np.float32), device="cuda")
    out = torch.empty((1, 4, J), dtype=torch.float32, device="cuda")
    assert _noalloc(lib, params, x, J, out) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _noalloc(lib, params, x, J, out) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    x = torch.zeros((1, 13, MAX_CELLS + 1), dtype=torch.float32, device="cuda")
    out = torch.zeros((1, 4, MAX_CELLS + 1), dtype=torch.float32, device="cuda")
    params = torch.zeros(pkg.oci_nn_param_count(), dtype=torch.float32, device="cuda")
    assert _noalloc(lib, params, x, MAX_CELLS + 1, out) == pkg.OCI_EINVAL
    assert _noalloc(lib, params, x, 0, out) == pkg.OCI_EINVAL
