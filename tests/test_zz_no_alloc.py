"""The allocation-free free energy (lcbp_free_energy_noalloc) agrees with the
ordinary entry point (lcbp_free_energy) on the same Q field.

It exists for callers that cannot allocate device memory when they need the
free energy (a framework allocator owning the heap, real-time loops); its
scratch is a fixed device array instead of cudaMalloc'd memory, so repeated
calls leave the device's free memory unchanged.
This file sorts last so that a run stopping at the first failure has run
every other test before it.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lcbp():
    import torch
    from paper_0901_3293_gb300 import build
    build.build()
    from paper_0901_3293_gb300 import lcbp as L
    torch.cuda.set_device(0)
    return L


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_free_energy_matches_lattice_entry_point(lcbp, dtype):
    import torch
    nx, ny, nz = 24, 20, 18
    A0, gamma, K, q0 = 0.01, 3.1, 0.01, 2 * np.pi / 16
    lat = lcbp.Lattice(nx, ny, nz, dtype=dtype)
    lat.set_ldg(A0, gamma, K, q0)
    lat.init_q(lcbp.BPII, 0.3, noise=1e-3, seed=5)
    F_ref = lat.free_energy()
    tdt = torch.float32 if dtype == "f32" else torch.float64
    q = torch.empty((5, nz, ny, nx), dtype=tdt, device="cuda")
    lat.read_q(out=q)
    stream = torch.cuda.Stream()
    tol = 1e-12 * abs(F_ref)  # same kernel, same FP64 reduction order
    for _ in range(2):  # two calls in a row share the same scratch
        F = lcbp.free_energy_noalloc(q, nx, ny, nz, A0, gamma, K, q0, stream=stream)
        assert abs(F - F_ref) <= tol, (F, F_ref)
    # a different field afterwards: the scratch keeps no stale partial sums
    q2 = q * 0.5
    torch.cuda.synchronize()  # the lattice's stream is not ordered after torch's
    lat.set_q(q2)
    F2_ref = lat.free_energy()
    F2 = lcbp.free_energy_noalloc(q2, nx, ny, nz, A0, gamma, K, q0)
    assert abs(F2 - F2_ref) <= 1e-12 * abs(F2_ref)
    lat.close()


def test_noalloc_calls_leave_free_memory_unchanged(lcbp):
    """After a warm-up call (which looks up the scratch array's address),
    repeated calls take no device memory: cudaMemGetInfo reports the same free
    bytes before and after."""
    import torch
    nx, ny, nz = 32, 16, 12
    lat = lcbp.Lattice(nx, ny, nz, dtype="f32")
    lat.init_q(lcbp.BPII, 0.3, noise=1e-3, seed=9)
    q = torch.empty((5, nz, ny, nx), dtype=torch.float32, device="cuda")
    lat.read_q(out=q)
    args = (q, nx, ny, nz, 0.01, 3.1, 0.01, 2 * np.pi / 16)
    F0 = lcbp.free_energy_noalloc(*args)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(20):
        assert lcbp.free_energy_noalloc(*args) == F0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    lat.close()


def test_noalloc_rejects_bad_sizes(lcbp):
    import torch
    q = torch.zeros(5 * 8, dtype=torch.float32, device="cuda")
    F = ctypes.c_double()
    rc = lcbp.lib().lcbp_free_energy_noalloc(q.data_ptr(), lcbp.F32, 0, 2, 4, 0.01, 3.1, 0.01, 0.4, None,
                                             ctypes.byref(F))
    assert rc == lcbp.EINVAL
    rc = lcbp.lib().lcbp_free_energy_noalloc(q.data_ptr(), lcbp.F32, 1 << 16, 1 << 16, 2, 0.01, 3.1, 0.01, 0.4,
                                             None, ctypes.byref(F))
    assert rc == lcbp.EINVAL and b"exceed" in lcbp.lib().lcbp_last_error()
