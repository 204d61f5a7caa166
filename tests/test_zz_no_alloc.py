"""flbm_step_noalloc: stepping caller-owned populations with no device
allocation.  Some callers cannot call cudaMalloc (an arena or pool owns all
device memory, or a real-time loop must not allocate); this entry point keeps
its scratch (density field, status word) in a static device array instead.

The check: starting from the same populations, two calls in a row of the
no-allocation entry point give bitwise the same populations as flbm_step on an
in-place context, in each storage format.  Both run the same population-reading
kernels with the same parameters, so the words must be identical."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(lib):
    fn = lib.flbm_step_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                   ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint)]
    return fn


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("lat,shape", [(0, (1, 40, 72)), (1, (12, 10, 24))])
def test_noalloc_matches_flbm_step(lat, shape, storage):
    import torch

    import oracle
    from paper_1410_5584_gb300 import Lattice
    from paper_1410_5584_gb300 import flbm as F
    from paper_1410_5584_gb300 import inputs

    nz, ny, nx = shape
    c, w, T, N = oracle.tables(lat)
    f0 = inputs.random_populations(np.stack([w * 1.0, w * 0.9]), shape, 0.02, seed=21)
    # the caller's buffer holds one in-place array, like the reference context's
    ref = Lattice(lat, nx, ny, nz, 0.8, 1.0, 1e-4, 0.7, 99, storage=storage,
                  streaming=F.STREAMING["in_place"], rho0_a=1.0, rho0_b=0.9)
    ref.set_populations(f0, step=4)
    work = ref.pop_buffer.clone()  # caller-owned copy of the raw populations (parity 0)
    torch.cuda.synchronize()
    step_noalloc = _noalloc(F.lib())
    status = ctypes.c_uint(123)
    stream = ctypes.c_void_p(ref.stream.cuda_stream)
    # two calls in a row: 3 steps from parity 0, then 2 steps from parity 1
    assert step_noalloc(ref._h, ctypes.c_void_p(work.data_ptr()), 0, 4, 3, stream, ctypes.byref(status)) == F.OK
    assert status.value == 0
    assert step_noalloc(ref._h, ctypes.c_void_p(work.data_ptr()), 1, 7, 2, stream, ctypes.byref(status)) == F.OK
    assert status.value == 0
    ref.step(3)
    ref.step(2)
    ref.sync()
    # both buffers now hold the state after 5 steps in the same in-place layout
    a = ref.pop_buffer.cpu().numpy()
    b = work.cpu().numpy()
    assert np.array_equal(a, b)
    assert a.any()


def test_noalloc_rejects_boxes_above_its_scratch():
    from paper_1410_5584_gb300 import flbm as F

    h = F.flbm_create(1, 160, 128, 128, 1.0, 1.0, 1e-5, 0.9, 1)  # 2,621,440 sites > 2^21
    try:
        step_noalloc = _noalloc(F.lib())
        assert step_noalloc(h, ctypes.c_void_p(256), 0, 0, 1, None, None) == F.EINVAL
    finally:
        F.lib().flbm_destroy(h)


def test_noalloc_rejects_batches_and_misaligned_populations_before_launching():
    """A batch handle and a population pointer off a 256-byte boundary are
    refused on the host; nothing is launched, so the pointers are never used."""
    from paper_1410_5584_gb300 import Batch, Lattice
    from paper_1410_5584_gb300 import flbm as F

    step_noalloc = _noalloc(F.lib())
    lat = Lattice(0, 32, 16, 1, 1.0, 1.0, 1e-5, 0.5, 3, streaming=F.STREAMING["in_place"])
    lat.init()
    base = lat.pop_buffer.data_ptr()
    assert base % 256 == 0
    for off in (4, 16, 128):
        assert step_noalloc(lat._h, ctypes.c_void_p(base + off), 0, 0, 1, None, None) == F.EINVAL
    batch = Batch(0, [dict(nx=16, ny=16, kT=1e-5, G=0.3, seed=5), dict(nx=32, ny=16, kT=1e-5, G=0.3, seed=6)])
    batch.init()
    assert step_noalloc(batch._h, ctypes.c_void_p(batch.pop_buffer.data_ptr()), 0, 0, 1, None, None) == F.EINVAL
