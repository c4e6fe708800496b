"""smr_rhs_plane_waves_static: right-hand sides with no device allocation.

For callers that cannot call cudaMalloc (device memory fully reserved by
their own pool allocator, or latency-critical loops that cannot take the
synchronisation an allocation may cause).  The call keeps its intermediate
sums in a fixed 4 MiB array in device global memory instead of allocating.

Checked through the C ABI: two calls in a row, each against the allocating
entry point smr_rhs_plane_waves on the same inputs, at the tolerance the
other RHS tests use (1e-13 relative); around the second call, that neither
the device's free memory nor the stream-ordered pool's usage (read through
the driver API, so the library's own cudaMallocAsync would show) moves; and
the size limit is enforced with an error instead of an overflow.  This file
is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2407_21724_gb300 import smr, workloads


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _reference(ctx, kh, pol, n):
    b = torch.empty(n * len(kh), dtype=torch.complex128, device="cuda")
    smr.smr_rhs_plane_waves(ctx, kh, pol, b)
    torch.cuda.synchronize()
    return b.cpu().numpy()


class _Pool:
    """The device's default stream-ordered memory pool, through the driver
    API (one instance per process, whichever runtime the library links)."""
    USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8          # CUmemPool_attribute values

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), torch.cuda.current_device()) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        z = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(z)) == 0


def _static(ctx, kh, pol, n, check_no_alloc=False):
    lib = smr.lib()
    R = len(kh)
    kd = torch.tensor(np.asarray(kh, dtype=np.float64), device="cuda").contiguous()
    pd = torch.tensor(np.asarray(pol, dtype=np.complex128), device="cuda").contiguous()
    b = torch.full((n * R,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    if check_no_alloc:
        pool = _Pool()
        pool.reset_high()
        used0 = pool.get(pool.USED_MEM_CURRENT)
        free0 = torch.cuda.mem_get_info()[0]
    rc = lib.smr_rhs_plane_waves_static(ctx, R, kd.data_ptr(), pd.data_ptr(), b.data_ptr(), stream)
    assert rc == 0, lib.smr_last_error(ctx).decode()
    torch.cuda.synchronize()
    if check_no_alloc:
        assert torch.cuda.mem_get_info()[0] == free0, "device memory changed across the call"
        assert pool.get(pool.USED_MEM_HIGH) <= used0, "the call drew on the stream-ordered pool"
    return b.cpu().numpy()


@pytest.fixture(scope="module")
def scene():
    w = workloads.make("random", n=9, seed=17, modes=16)
    ctx = smr.scene_from_workload(w)
    yield ctx, smr.smr_info(ctx)["n_unknowns"]
    smr.smr_destroy(ctx)


def test_static_rhs_matches_allocating_entry_point_twice(scene):
    ctx, n = scene
    grid = workloads.incidence_grid64()
    first = grid[:5]
    second = grid[40:43]            # different R: the array keeps the first call's sums
    for i, inc in enumerate((first, second)):
        kh = [k for k, _ in inc]
        pol = [p for _, p in inc]
        # the first call on a device looks the array's address up; the
        # second must leave device memory and the pool untouched
        got = _static(ctx, kh, pol, n, check_no_alloc=(i == 1))
        ref = _reference(ctx, kh, pol, n)
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) < 1e-13


def test_static_rhs_rejects_sizes_beyond_the_array(scene):
    ctx, n = scene
    lib = smr.lib()
    info = smr.smr_info(ctx)
    # smallest R whose sums (shapes x n_psi x 2 x R x 16 bytes) exceed 4 MiB
    R = (4 << 20) // (info["n_shapes"] * info["n_psi"] * 32) + 1
    kd = torch.zeros((R, 3), dtype=torch.float64, device="cuda")
    pd = torch.zeros((R, 3), dtype=torch.complex128, device="cuda")
    b = torch.zeros(n * R, dtype=torch.complex128, device="cuda")
    rc = lib.smr_rhs_plane_waves_static(ctx, R, kd.data_ptr(), pd.data_ptr(), b.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
    assert rc == -1
    assert b"exceeds the fixed scratch" in lib.smr_last_error(ctx)
