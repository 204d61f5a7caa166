"""The C-ABI library loads and exports every entry point of include/flbm.h, and
its argument checks work without a GPU (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_1410_5584_gb300 import _build
from paper_1410_5584_gb300 import flbm as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(flbm_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return F.lib()


def test_every_declared_symbol_is_exported(lib):
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            names += _declared(os.path.join(ROOT, "include", h))
    assert "flbm_step" in names and "flbm_create" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_version(lib):
    assert "sm_103a" in F.version()


@pytest.mark.parametrize("args", [
    (5, 16, 16, 1, 1.0, 1.0, 1e-4, 0.0),        # unknown lattice
    (0, 16, 16, 2, 1.0, 1.0, 1e-4, 0.0),        # D2Q9 needs nz = 1
    (1, 16, 16, 1, 1.0, 1.0, 1e-4, 0.0),        # D3Q19 needs nz >= 2
    (0, 1, 16, 1, 1.0, 1.0, 1e-4, 0.0),         # dimension < 2
    (0, 16, 16, 1, 0.5, 1.0, 1e-4, 0.0),        # tau <= 1/2 (2 lb - lb^2 <= 0)
    (0, 16, 16, 1, 1.0, 0.4, 1e-4, 0.0),
    (0, 16, 16, 1, 1.0, 1.0, -1e-4, 0.0),       # kT < 0
    (0, 16, 70000, 1, 1.0, 1.0, 1e-4, 0.0),     # ny > 65535
    (1, 2048, 2048, 512, 1.0, 1.0, 1e-4, 0.0),  # N >= 2^31
    (0, 16, 16, 1, float("nan"), 1.0, 1e-4, 0.0),
])
def test_create_rejects_invalid_arguments(lib, args):
    h = ctypes.c_void_p()
    st = lib.flbm_create(*args, 1, ctypes.byref(h))
    assert st == F.EINVAL
    assert not h.value


def test_options_are_validated(lib):
    h = F.flbm_create(F.D2Q9, 8, 8, 1, 1.0, 1.0, 1e-4, 0.0, 1)
    try:
        assert lib.flbm_set_option(h, F.OPT_LAMBDA_D, 2.5) == F.EINVAL
        assert b"lambda_d" in lib.flbm_last_error(h)
        assert lib.flbm_set_option(h, 12345, 1.0) == F.EINVAL
        assert lib.flbm_set_option(h, F.OPT_LAMBDA_MODE + 2, 1.0) == F.EINVAL  # a momentum mode
        assert lib.flbm_set_option(h, F.OPT_LAMBDA_MODE + 100 + 8, 1.2) == F.OK
        assert lib.flbm_set_option(h, F.OPT_STORAGE, 3) == F.EINVAL
        assert lib.flbm_set_option(h, F.OPT_SF_AXIS, 2) == F.EINVAL  # no z axis in 2D
        assert lib.flbm_set_option(h, F.OPT_RHO0_A, -1.0) == F.EINVAL
        assert lib.flbm_step(h, 1) == F.ESTATE  # before init
        assert lib.flbm_step(h, -1) == F.EINVAL
        pb, rb = ctypes.c_size_t(), ctypes.c_size_t()
        assert lib.flbm_buffer_bytes(h, ctypes.byref(pb), ctypes.byref(rb)) == F.OK
        # two population arrays (the default streaming) of 2 species x 9 x 64 sites
        assert pb.value == 2 * (2 * 9 * 64 * 4) and rb.value == 2 * 64 * 4
        assert lib.flbm_set_option(h, F.OPT_STORAGE, 2) == F.OK
        assert lib.flbm_buffer_bytes(h, ctypes.byref(pb), None) == F.OK
        assert pb.value == 2 * (2 * 9 * 64 * 2)
        need = ctypes.c_size_t()
        assert lib.flbm_checkpoint(h, None, ctypes.byref(need)) == F.OK
        assert need.value > pb.value // 2  # a header and the current array
    finally:
        lib.flbm_destroy(h)


def test_launch_settings_are_validated_and_read_back(lib):
    """Block shape, schedule and slab options (host logic only; no GPU)."""
    h = F.flbm_create(F.D3Q19, 16, 16, 16, 1.0, 1.0, 1e-4, 0.0, 1)
    v = ctypes.c_double()
    try:
        for key, bad in ((F.OPT_BLOCK_X, 48), (F.OPT_BLOCK_X, 256), (F.OPT_BLOCK_Y, 3), (F.OPT_BLOCK_Y, 8),
                         (F.OPT_SCHEDULE, 4), (F.OPT_SLABS, 2), (F.OPT_SLABS, 4.5)):
            assert lib.flbm_set_option(h, key, bad) == F.EINVAL, (key, bad)
        assert lib.flbm_set_option(h, F.OPT_BLOCK_X, 32) == F.OK
        assert lib.flbm_set_option(h, F.OPT_BLOCK_Y, 4) == F.OK
        assert lib.flbm_set_option(h, F.OPT_BLOCK_X, 64) == F.EINVAL  # 64 x 4 > 128 sites
        assert lib.flbm_set_option(h, F.OPT_SCHEDULE, F.SCHEDULE["overlap"]) == F.OK
        assert lib.flbm_set_option(h, F.OPT_SLABS, 5) == F.OK
        for key, want in ((F.OPT_BLOCK_X, 32), (F.OPT_BLOCK_Y, 4), (F.OPT_SCHEDULE, 2), (F.OPT_SLABS, 5),
                          (F.OPT_LAMBDA_MODE + 100 + 7, 1.0)):
            assert lib.flbm_get_option(h, key, ctypes.byref(v)) == F.OK and v.value == want, key
        assert lib.flbm_get_option(h, F.OPT_GRAPH_STEPS, ctypes.byref(v)) == F.OK and v.value == 0  # off
        assert lib.flbm_get_option(h, 12345, ctypes.byref(v)) == F.EINVAL
        # the autotuner checks its arguments and the state before touching the GPU
        assert lib.flbm_autotune(h, 0, None) == F.EINVAL
        assert lib.flbm_autotune(h, 5, None) == F.ESTATE  # before init
    finally:
        lib.flbm_destroy(h)


def test_null_context_is_safe(lib):
    assert lib.flbm_last_error(None) == b""
    assert lib.flbm_step(None, 1) == F.EINVAL
    lib.flbm_destroy(None)


def test_batch_create_validates_replicas(lib):
    good = F.RepParams(8, 6, 1, 1.0, 1.0, 1e-4, 0.1, 3, 1.0, 1.0)
    bad_tau = F.RepParams(8, 6, 1, 0.5, 1.0, 1e-4, 0.1, 3, 1.0, 1.0)
    bad_rho = F.RepParams(8, 6, 1, 1.0, 1.0, 1e-4, 0.1, 3, 0.0, 1.0)
    for arr in [(F.RepParams * 2)(good, bad_tau), (F.RepParams * 1)(bad_rho)]:
        h = ctypes.c_void_p()
        assert lib.flbm_batch_create(0, len(arr), arr, ctypes.byref(h)) == F.EINVAL
        assert not h.value
    arr = (F.RepParams * 2)(good, F.RepParams(5, 7, 1, 0.9, 1.1, 1e-5, 0.2, 4, 1.0, 0.8))
    h = ctypes.c_void_p()
    assert lib.flbm_batch_create(0, 2, arr, ctypes.byref(h)) == F.OK
    try:
        n, sites = ctypes.c_int(), ctypes.c_int64()
        assert lib.flbm_batch_size(h, ctypes.byref(n), ctypes.byref(sites)) == F.OK
        assert (n.value, sites.value) == (2, 48 + 35)
        v = ctypes.c_void_p()
        assert lib.flbm_batch_replica(h, 1, ctypes.byref(v)) == F.OK
        assert lib.flbm_step(v, 1) == F.ESTATE          # views are read-only
        assert lib.flbm_set_option(v, F.OPT_SF_AXIS, 1) == F.OK
        assert lib.flbm_batch_replica(h, 2, ctypes.byref(v)) == F.EINVAL
        assert lib.flbm_set_option(h, F.OPT_GRAPH_STEPS, -1) == F.EINVAL
        lib.flbm_destroy(v)                             # a view is not destroyed on its own
    finally:
        lib.flbm_destroy(h)


def test_batch_streaming_and_schedule_options(lib):
    """Batches stream through two arrays by default (twice the population
    bytes of in place), take the streaming mode before their buffers exist,
    and accept the two-kernel (1) and tiled (3) schedules only; a schedule
    outside the enum is rejected on single boxes too (host logic only)."""
    arr = (F.RepParams * 2)(F.RepParams(8, 6, 1, 1.0, 1.0, 1e-4, 0.1, 3, 1.0, 1.0),
                            F.RepParams(5, 7, 1, 0.9, 1.1, 1e-5, 0.2, 4, 1.0, 0.8))
    h = ctypes.c_void_p()
    assert lib.flbm_batch_create(0, 2, arr, ctypes.byref(h)) == F.OK
    try:
        v = ctypes.c_double()
        assert lib.flbm_get_option(h, F.OPT_STREAMING, ctypes.byref(v)) == F.OK and v.value == 1
        pb2, rb = ctypes.c_size_t(), ctypes.c_size_t()
        assert lib.flbm_buffer_bytes(h, ctypes.byref(pb2), ctypes.byref(rb)) == F.OK
        assert pb2.value == 2 * 2 * 9 * (48 + 35) * 4
        assert lib.flbm_set_option(h, F.OPT_STREAMING, 2) == F.EINVAL
        assert lib.flbm_set_option(h, F.OPT_STREAMING, 0) == F.OK
        pb1 = ctypes.c_size_t()
        assert lib.flbm_buffer_bytes(h, ctypes.byref(pb1), ctypes.byref(rb)) == F.OK
        assert 2 * pb1.value == pb2.value
        assert lib.flbm_get_option(h, F.OPT_STREAMING, ctypes.byref(v)) == F.OK and v.value == 0
        for sched, want in ((0, F.EUNSUPPORTED), (2, F.EUNSUPPORTED), (3, F.OK), (1, F.OK), (4, F.EUNSUPPORTED)):
            assert lib.flbm_set_option(h, F.OPT_SCHEDULE, sched) == want, sched
        assert lib.flbm_set_option(h, F.OPT_SCHEDULE, 3) == F.OK
        assert lib.flbm_get_option(h, F.OPT_SCHEDULE, ctypes.byref(v)) == F.OK and v.value == 3
    finally:
        lib.flbm_destroy(h)
    g = F.flbm_create(0, 8, 6, 1, 1.0, 1.0, 1e-4, 0.5, 1)
    try:
        assert lib.flbm_set_option(g, F.OPT_SCHEDULE, 3) == F.OK
        assert lib.flbm_set_option(g, F.OPT_SCHEDULE, 4) == F.EINVAL
    finally:
        lib.flbm_destroy(g)


def _mcreate(lib, lat, ns, nx, ny, nz, tau, kT, G):
    t = (ctypes.c_double * len(tau))(*tau)
    g = (ctypes.c_double * len(G))(*G)
    h = ctypes.c_void_p()
    st = lib.flbm_mcreate(lat, ns, nx, ny, nz, t, kT, g, 7, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("lat,ns,nz,tau,kT,G", [
    (0, 1, 1, [1.0], 1e-4, [0.0]),                                       # one species
    (0, 5, 1, [1.0] * 5, 1e-4, [0.0] * 25),                              # more than four
    (0, 3, 2, [1.0] * 3, 1e-4, [0.0] * 9),                               # D2Q9 needs nz = 1
    (0, 3, 1, [1.0, 0.5, 1.0], 1e-4, [0.0] * 9),                         # tau <= 1/2
    (0, 3, 1, [1.0] * 3, -1.0, [0.0] * 9),                               # kT < 0
    (0, 3, 1, [1.0] * 3, 1e-4, [0, 0.1, 0, 0.2, 0, 0, 0, 0, 0]),         # G not symmetric
    (0, 2, 1, [1.0] * 2, 1e-4, [0, float("inf"), float("inf"), 0]),      # G not finite
    (3, 3, 1, [1.0] * 3, 1e-4, [0.0] * 9),                               # unknown lattice
])
def test_multi_create_rejects_invalid_arguments(lib, lat, ns, nz, tau, kT, G):
    st, h = _mcreate(lib, lat, ns, 8, 8, nz, tau, kT, G)
    assert st == F.EINVAL
    assert not h.value


def test_multi_options_and_order_are_validated(lib):
    st, h = _mcreate(lib, 1, 3, 8, 6, 4, [1.0, 0.8, 1.2], 1e-4, [0, 0.1, 0.2, 0.1, 0, 0.3, 0.2, 0.3, 0])
    assert st == F.OK
    try:
        assert lib.flbm_mset_option(h, F.OPT_RHO0_SPECIES + 2, 0.7) == F.OK
        assert lib.flbm_mset_option(h, F.OPT_RHO0_SPECIES + 3, 0.7) == F.EINVAL   # only 3 species
        assert lib.flbm_mset_option(h, F.OPT_RHO0_SPECIES, 0.0) == F.EINVAL
        assert lib.flbm_mset_option(h, F.OPT_KERNEL_TIMING, 2) == F.EINVAL
        assert lib.flbm_mset_option(h, F.OPT_BLOCK_X, 64) == F.OK
        assert lib.flbm_mset_option(h, F.OPT_BLOCK_Y, 4) == F.EINVAL              # 64 x 4 > 128
        assert lib.flbm_mset_option(h, F.OPT_STORAGE, 1) == F.EINVAL              # float storage only
        assert b"unknown option" in lib.flbm_mlast_error(h)
        assert lib.flbm_mstep(h, 1) == F.ESTATE                                    # before init
        v = ctypes.c_double()
        for key, want in ((F.OPT_RHO0_SPECIES + 2, 0.7), (F.OPT_BLOCK_X, 64), (F.OPT_STREAMING, 1),
                          (F.OPT_GRAPH_STEPS, 0), (F.OPT_KERNEL_TIMING, 0)):
            assert lib.flbm_mget_option(h, key, ctypes.byref(v)) == F.OK and v.value == want, key
        assert lib.flbm_mget_option(h, F.OPT_RHO0_SPECIES + 3, ctypes.byref(v)) == F.EINVAL
        step = ctypes.c_int64(-1)
        assert lib.flbm_mget_step(h, ctypes.byref(step)) == F.OK and step.value == 0
    finally:
        lib.flbm_mdestroy(h)
    assert lib.flbm_mlast_error(None) == b""
    assert lib.flbm_mstep(None, 1) == F.EINVAL
    lib.flbm_mdestroy(None)


def test_streaming_option_and_buffer_sizes(lib):
    """Two-array streaming (the default) needs twice the population bytes of
    in-place streaming; the option takes 0 or 1 (host logic only)."""
    h = F.flbm_create(1, 8, 6, 4, 1.0, 1.0, 1e-4, 0.5, 1)
    try:
        v = ctypes.c_double()
        assert lib.flbm_get_option(h, F.OPT_STREAMING, ctypes.byref(v)) == F.OK and v.value == 1
        pb2, rb2 = ctypes.c_size_t(), ctypes.c_size_t()
        assert lib.flbm_buffer_bytes(h, ctypes.byref(pb2), ctypes.byref(rb2)) == F.OK
        assert lib.flbm_set_option(h, F.OPT_STREAMING, 2) == F.EINVAL
        assert lib.flbm_set_option(h, F.OPT_STREAMING, 0) == F.OK
        pb1, rb1 = ctypes.c_size_t(), ctypes.c_size_t()
        assert lib.flbm_buffer_bytes(h, ctypes.byref(pb1), ctypes.byref(rb1)) == F.OK
        assert pb2.value == 2 * pb1.value == 2 * 2 * 19 * 8 * 6 * 4 * 4
        assert rb1.value == rb2.value
    finally:
        lib.flbm_destroy(h)


def test_graph_steps_option_on_a_single_box(lib):
    h = F.flbm_create(0, 16, 8, 1, 1.0, 1.0, 1e-4, 0.5, 1)
    try:
        v = ctypes.c_double(-1)
        assert lib.flbm_get_option(h, F.OPT_GRAPH_STEPS, ctypes.byref(v)) == F.OK and v.value == 0
        assert lib.flbm_set_option(h, F.OPT_GRAPH_STEPS, 16) == F.OK
        assert lib.flbm_get_option(h, F.OPT_GRAPH_STEPS, ctypes.byref(v)) == F.OK and v.value == 16
        assert lib.flbm_set_option(h, F.OPT_GRAPH_STEPS, -1) == F.EINVAL
        assert lib.flbm_set_option(h, F.OPT_GRAPH_STEPS, 2.5) == F.EINVAL
    finally:
        lib.flbm_destroy(h)


def test_header_is_plain_c_and_links(lib, tmp_path):
    """include/flbm.h compiles as C99 with warnings as errors, and a C program
    linked against the library runs its argument checks (no GPU needed)."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi_check.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "flbm.h"
int main(void)
{
    flbm_ctx *ctx = NULL;
    if (flbm_create(FLBM_D2Q9, 16, 16, 2, 1.0, 1.0, 1e-4, 0.5, 1, &ctx) != FLBM_EINVAL || ctx) return 1;
    if (flbm_create(FLBM_D3Q19, 8, 6, 4, 1.0, 0.8, 1e-4, 0.5, 7, &ctx) != FLBM_OK || !ctx) return 2;
    if (flbm_set_option(ctx, FLBM_OPT_STREAMING, FLBM_STREAM_IN_PLACE) != FLBM_OK) return 3;
    if (flbm_set_option(ctx, 12345, 1.0) != FLBM_EINVAL || strlen(flbm_last_error(ctx)) == 0) return 4;
    size_t pop = 0, rho = 0;
    if (flbm_buffer_bytes(ctx, &pop, &rho) != FLBM_OK || pop != (size_t)2 * 19 * 192 * 4) return 5;
    if (flbm_step(ctx, 1) != FLBM_ESTATE) return 6;
    flbm_destroy(ctx);
    double tau[3] = {1.0, 0.8, 1.25}, G[9] = {0, .3, .3, .3, 0, .3, .3, .3, 0};
    flbm_mctx *m = NULL;
    if (flbm_mcreate(FLBM_D2Q9, 3, 16, 8, 1, tau, 1e-4, G, 3, &m) != FLBM_OK || !m) return 7;
    if (flbm_mstep(m, 1) != FLBM_ESTATE) return 8;
    flbm_mdestroy(m);
    printf("%s\n", flbm_version());
    return 0;
}
""")
    exe = tmp_path / "abi_check"
    libdir = os.path.dirname(F.library_path())
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
           "-o", str(exe), "-L", libdir, "-lflbm", "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert "sm_103a" in out.stdout
