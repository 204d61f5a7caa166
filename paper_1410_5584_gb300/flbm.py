"""Python binding of the flbm C-ABI (include/flbm.h): argument marshalling only.

Every step of the lattice update runs in the CUDA kernels of ``libflbm.so``;
this module converts arguments, owns the PyTorch device buffers it attaches,
and turns status codes into exceptions.  It never falls back to a CPU path:
if the library is missing or no GPU is visible, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

D2Q9, D3Q19 = 0, 1
STORE = {"f32": 0, "f16": 1, "bf16": 2}

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, EUNSUPPORTED, ESTATE = range(8)
STATUS_NAMES = ["FLBM_OK", "FLBM_EINVAL", "FLBM_ENOMEM", "FLBM_ECUDA", "FLBM_ENONFINITE",
                "FLBM_ETIMEOUT", "FLBM_EUNSUPPORTED", "FLBM_ESTATE"]

OPT_STORAGE = 1
OPT_LAMBDA_D = 2
OPT_SDF = 3
OPT_RHO0_A = 4
OPT_RHO0_B = 5
OPT_NOISE_RHO = 7
OPT_FORCE_VELOCITY = 8
OPT_SF_AXIS = 9
OPT_KERNEL_TIMING = 10
OPT_SCHEDULE = 11
OPT_WAIT_LIMIT_MS = 12
OPT_TEST_STALL = 13
OPT_PIPE_LAG = 14
OPT_GRAPH_STEPS = 15
OPT_SLABS = 16
OPT_BLOCK_X = 17
OPT_BLOCK_Y = 18
OPT_STREAMING = 19
OPT_TEST_GENERAL_COLLIDE = 20
OPT_GHOST_NOISE = 21
OPT_DIRECT_HOST = 22
STREAMING = {"in_place": 0, "two_arrays": 1}
SCHEDULE = {"fused": 0, "two_kernels": 1, "overlap": 2, "tiled": 3}
OPT_LAMBDA_MODE = 1000
OPT_RHO0_SPECIES = 2000
OPTION_NAMES = {"storage": OPT_STORAGE, "lambda_d": OPT_LAMBDA_D, "sdf": OPT_SDF,
                "rho0_a": OPT_RHO0_A, "rho0_b": OPT_RHO0_B, "noise_rho": OPT_NOISE_RHO,
                "force_velocity": OPT_FORCE_VELOCITY, "sf_axis": OPT_SF_AXIS,
                "kernel_timing": OPT_KERNEL_TIMING, "schedule": OPT_SCHEDULE,
                "wait_limit_ms": OPT_WAIT_LIMIT_MS, "test_stall": OPT_TEST_STALL,
                "pipe_lag": OPT_PIPE_LAG, "graph_steps": OPT_GRAPH_STEPS, "slabs": OPT_SLABS,
                "block_x": OPT_BLOCK_X, "block_y": OPT_BLOCK_Y, "streaming": OPT_STREAMING,
                "test_general_collide": OPT_TEST_GENERAL_COLLIDE, "ghost_noise": OPT_GHOST_NOISE,
                "direct_host": OPT_DIRECT_HOST}


class RepParams(ctypes.Structure):
    """flbm_rep_params: one replica of a batch."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("tau_a", ctypes.c_double), ("tau_b", ctypes.c_double), ("kT", ctypes.c_double),
                ("G", ctypes.c_double), ("seed", ctypes.c_uint64), ("rho0_a", ctypes.c_double),
                ("rho0_b", ctypes.c_double)]


class FlbmError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libflbm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(the CUDA library is required; there is no CPU fallback)")
        L = ctypes.CDLL(path)
        vp, i32, i64, u64, dbl, sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                      ctypes.c_double, ctypes.c_size_t)
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        szp = ctypes.POINTER(ctypes.c_size_t)
        sig = {
            "flbm_create": (i32, [i32, i32, i32, i32, dbl, dbl, dbl, dbl, u64, ctypes.POINTER(vp)]),
            "flbm_set_option": (i32, [vp, i32, dbl]),
            "flbm_get_option": (i32, [vp, i32, dp]),
            "flbm_autotune": (i32, [vp, i32, ctypes.c_char_p]),
            "flbm_set_stream": (i32, [vp, vp]),
            "flbm_buffer_bytes": (i32, [vp, szp, szp]),
            "flbm_attach_buffers": (i32, [vp, vp, sz, vp, sz]),
            "flbm_init": (i32, [vp, dp, dp]),
            "flbm_step": (i32, [vp, i64]),
            "flbm_sync": (i32, [vp]),
            "flbm_get_step": (i32, [vp, i64p]),
            "flbm_kernel_times": (i32, [vp, dp, i64p]),
            "flbm_moments": (i32, [vp, dp, dp, dp, dp]),
            "flbm_sf_sample": (i32, [vp]),
            "flbm_structure_factor": (i32, [vp, i32, i32, dp, dp, dp, dp, i64p]),
            "flbm_sf_reset": (i32, [vp]),
            "flbm_sfk_sample": (i32, [vp]),
            "flbm_sfk": (i32, [vp, dp, dp, dp, i64p]),
            "flbm_sfk_functions": (i32, [vp, dbl, dbl, dp, dp, dp]),
            "flbm_sfk_reset": (i32, [vp]),
            "flbm_cap_sample": (i32, [vp, i32, i32]),
            "flbm_cap_spectrum": (i32, [vp, i32, dp, dp, i64p]),
            "flbm_cap_reset": (i32, [vp]),
            "flbm_get_populations": (i32, [vp, dp]),
            "flbm_set_populations": (i32, [vp, dp, i64]),
            "flbm_get_site_populations": (i32, [vp, i64p, i64, dp]),
            "flbm_checkpoint": (i32, [vp, vp, szp]),
            "flbm_restore": (i32, [vp, vp, sz]),
            "flbm_last_error": (ctypes.c_char_p, [vp]),
            "flbm_destroy": (None, [vp]),
            "flbm_version": (ctypes.c_char_p, []),
            "flbm_batch_create": (i32, [i32, i32, ctypes.POINTER(RepParams), ctypes.POINTER(vp)]),
            "flbm_batch_replica": (i32, [vp, i32, ctypes.POINTER(vp)]),
            "flbm_batch_size": (i32, [vp, ctypes.POINTER(ctypes.c_int), i64p]),
            "flbm_mcreate": (i32, [i32, i32, i32, i32, i32, dp, dbl, dp, u64, ctypes.POINTER(vp)]),
            "flbm_mset_option": (i32, [vp, i32, dbl]),
            "flbm_mget_option": (i32, [vp, i32, dp]),
            "flbm_mset_stream": (i32, [vp, vp]),
            "flbm_minit": (i32, [vp, dp]),
            "flbm_mstep": (i32, [vp, i64]),
            "flbm_msync": (i32, [vp]),
            "flbm_mkernel_times": (i32, [vp, dp, i64p]),
            "flbm_mget_step": (i32, [vp, i64p]),
            "flbm_mmoments": (i32, [vp, dp, dp, dp]),
            "flbm_mget_populations": (i32, [vp, dp]),
            "flbm_mset_populations": (i32, [vp, dp, i64]),
            "flbm_mget_site_populations": (i32, [vp, i64p, i64, dp]),
            "flbm_msf_sample": (i32, [vp, i32]),
            "flbm_mstructure_factor": (i32, [vp, i32, i32, dp, i64p]),
            "flbm_msf_reset": (i32, [vp]),
            "flbm_mcheckpoint": (i32, [vp, vp, szp]),
            "flbm_mrestore": (i32, [vp, vp, sz]),
            "flbm_mlast_error": (ctypes.c_char_p, [vp]),
            "flbm_mdestroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def version() -> str:
    return lib().flbm_version().decode()


def check(handle, status):
    if status != OK:
        msg = lib().flbm_last_error(handle).decode(errors="replace") if handle else ""
        raise FlbmError(status, msg)


def mcheck(handle, status):
    if status != OK:
        msg = lib().flbm_mlast_error(handle).decode(errors="replace") if handle else ""
        raise FlbmError(status, msg)


def flbm_create(lattice, nx, ny, nz, tau_a, tau_b, kT, G, seed):
    h = ctypes.c_void_p()
    st = lib().flbm_create(int(lattice), int(nx), int(ny), int(nz), float(tau_a), float(tau_b),
                           float(kT), float(G), int(seed) & (2**64 - 1), ctypes.byref(h))
    check(None, st)
    return h


class _Context:
    """Observation and state calls shared by single boxes, batches and replica views."""

    def sync(self):
        check(self._h, lib().flbm_sync(self._h))

    @property
    def step_count(self):
        v = ctypes.c_int64()
        check(self._h, lib().flbm_get_step(self._h, ctypes.byref(v)))
        return v.value

    def set_option(self, key, value):
        if isinstance(key, str):
            key = OPTION_NAMES[key]
        check(self._h, lib().flbm_set_option(self._h, int(key), float(value)))

    def get_option(self, key):
        if isinstance(key, str):
            key = OPTION_NAMES[key]
        v = ctypes.c_double()
        check(self._h, lib().flbm_get_option(self._h, int(key), ctypes.byref(v)))
        return v.value

    def autotune(self, steps=20, cache=None):
        """flbm_autotune: time the candidate launch settings on the current state
        (left unchanged), keep the fastest, and return them; `cache` is an
        optional JSON file of earlier choices."""
        path = None if cache is None else os.fsencode(cache)
        check(self._h, lib().flbm_autotune(self._h, int(steps), path))
        keys = ("schedule", "graph_steps") if isinstance(self, Batch) else ("schedule", "slabs", "block_x",
                                                                            "block_y", "graph_steps")
        return {k: int(self.get_option(k)) for k in keys}

    def sf_sample(self):
        check(self._h, lib().flbm_sf_sample(self._h))

    def sfk_sample(self):
        """flbm_sfk_sample: one snapshot of the structure factors at every wavevector."""
        check(self._h, lib().flbm_sfk_sample(self._h))

    def sfk_reset(self):
        check(self._h, lib().flbm_sfk_reset(self._h))

    def _sfk_shape(self):
        return (self.nz, self.ny, self.nx)

    def sfk(self):
        """(S_aa, S_ab, S_bb, nsamples): ensemble means at every wavevector,
        arrays [m_z][m_y][m_x] (numpy FFT order)."""
        out = [np.empty(self._sfk_shape()) for _ in range(3)]
        n = ctypes.c_int64()
        check(self._h, lib().flbm_sfk(self._h, *[_dp(o) for o in out], ctypes.byref(n)))
        return (*out, n.value)

    def sfk_functions(self, rho0_a, rho0_b):
        """(S_tt, S_CC, S_tC) of Eq. structurefunctions about (rho0_a, rho0_b)."""
        out = [np.empty(self._sfk_shape()) for _ in range(3)]
        check(self._h, lib().flbm_sfk_functions(self._h, float(rho0_a), float(rho0_b), *[_dp(o) for o in out]))
        return tuple(out)

    def cap_sample(self, x_liquid, x_gas):
        """flbm_cap_sample: one snapshot of the two interface heights' spectrum."""
        check(self._h, lib().flbm_cap_sample(self._h, int(x_liquid), int(x_gas)))

    def cap_spectrum(self, nk=None):
        """(S_h[m = 1..nk], h_mean[2], nsamples) of the capillary snapshots."""
        nk = self.ny // 2 if nk is None else int(nk)
        s, hm = np.empty(nk), np.empty(2)
        n = ctypes.c_int64()
        check(self._h, lib().flbm_cap_spectrum(self._h, nk, _dp(s), _dp(hm), ctypes.byref(n)))
        return s, hm, n.value

    def cap_reset(self):
        check(self._h, lib().flbm_cap_reset(self._h))

    def sf_reset(self):
        check(self._h, lib().flbm_sf_reset(self._h))

    def moments(self, fields=True):
        """(rho_a, rho_b, u[D], cons[5]) as float64 arrays [z][y][x]."""
        shp = (self.nz, self.ny, self.nx)
        ra = np.empty(self.N) if fields else None
        rb = np.empty(self.N) if fields else None
        u = np.empty(self.D * self.N) if fields else None
        cons = np.empty(5)
        check(self._h, lib().flbm_moments(self._h, _dp(ra), _dp(rb), _dp(u), _dp(cons)))
        if not fields:
            return cons
        return ra.reshape(shp), rb.reshape(shp), u.reshape((self.D,) + shp), cons

    def structure_factor(self, axis=0, nk=None):
        n_axis = (self.nx, self.ny, self.nz)[axis]
        nk = n_axis // 2 if nk is None else nk
        out = [np.empty(nk) for _ in range(4)]
        n = ctypes.c_int64()
        check(self._h, lib().flbm_structure_factor(self._h, axis, nk, *[_dp(o) for o in out], ctypes.byref(n)))
        return (*out, n.value)

    def get_populations(self):
        f = np.empty(2 * self.Q * self.N)
        check(self._h, lib().flbm_get_populations(self._h, _dp(f)))
        return f.reshape(2, self.Q, self.nz, self.ny, self.nx)

    def set_populations(self, f, step=0):
        f = np.ascontiguousarray(f, dtype=np.float64).ravel()
        if f.size != 2 * self.Q * self.N:
            raise ValueError("populations need 2 * Q values per site")
        check(self._h, lib().flbm_set_populations(self._h, _dp(f), int(step)))

    def site_populations(self, sites):
        s = np.ascontiguousarray(sites, dtype=np.int64).ravel()
        out = np.empty(s.size * 2 * self.Q)
        check(self._h, lib().flbm_get_site_populations(
            self._h, s.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), s.size, _dp(out)))
        return out.reshape(s.size, 2, self.Q)

    def checkpoint(self) -> bytes:
        n = ctypes.c_size_t()
        check(self._h, lib().flbm_checkpoint(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        check(self._h, lib().flbm_checkpoint(self._h, buf, ctypes.byref(n)))
        return buf.raw[:n.value]

    def restore(self, image: bytes):
        buf = ctypes.create_string_buffer(image, len(image))
        check(self._h, lib().flbm_restore(self._h, buf, len(image)))


class ReplicaView(_Context):
    """One replica of a Batch, for observation (moments, structure factors,
    populations).  Owned by its batch."""

    def __init__(self, batch, rep, params):
        self._batch = batch
        h = ctypes.c_void_p()
        check(batch._h, lib().flbm_batch_replica(batch._h, int(rep), ctypes.byref(h)))
        self._h = h
        self.lattice = batch.lattice
        self.nx, self.ny = params.nx, params.ny
        self.nz = 1 if self.lattice == D2Q9 else params.nz
        self.D, self.Q = batch.D, batch.Q
        self.N = self.nx * self.ny * self.nz



class Batch(_Context):
    """Many independent two-species boxes of uneven size advanced together
    (flbm_batch_create).  ``replicas`` is a list of dicts with nx, ny[, nz],
    tau_a, tau_b, kT, G, seed[, rho0_a, rho0_b]."""

    def __init__(self, lattice, replicas, storage="f32", device="cuda:0", stream=None, **options):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device visible: flbm runs on the GPU only")
        self.lattice = int(lattice)
        self.D = 2 if self.lattice == D2Q9 else 3
        self.Q = 9 if self.lattice == D2Q9 else 19
        arr = (RepParams * len(replicas))()
        for k, r in enumerate(replicas):
            arr[k] = RepParams(int(r["nx"]), int(r["ny"]), int(r.get("nz", 1)), float(r.get("tau_a", 1.0)),
                               float(r.get("tau_b", 1.0)), float(r.get("kT", 0.0)), float(r.get("G", 0.0)),
                               int(r.get("seed", 1)) & (2**64 - 1), float(r.get("rho0_a", 1.0)),
                               float(r.get("rho0_b", 1.0)))
        self._params = arr
        self._h = None
        h = ctypes.c_void_p()
        check(None, lib().flbm_batch_create(self.lattice, len(replicas), arr, ctypes.byref(h)))
        self._h = h
        n = ctypes.c_int()
        sites = ctypes.c_int64()
        check(self._h, lib().flbm_batch_size(self._h, ctypes.byref(n), ctypes.byref(sites)))
        self.nrep, self.N = n.value, sites.value
        self.sizes = [arr[k].nx * arr[k].ny * (arr[k].nz if self.lattice == D3Q19 else 1) for k in range(self.nrep)]
        self.set_option(OPT_STORAGE, STORE[storage] if isinstance(storage, str) else int(storage))
        for k, v in options.items():
            self.set_option(k, v)
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        check(self._h, lib().flbm_set_stream(self._h, ctypes.c_void_p(self.stream.cuda_stream)))
        pb, rb = ctypes.c_size_t(), ctypes.c_size_t()
        check(self._h, lib().flbm_buffer_bytes(self._h, ctypes.byref(pb), ctypes.byref(rb)))
        self.pop_buffer = torch.empty(pb.value, dtype=torch.uint8, device=self.device)
        self.rho_buffer = torch.empty(rb.value, dtype=torch.uint8, device=self.device)
        check(self._h, lib().flbm_attach_buffers(self._h, ctypes.c_void_p(self.pop_buffer.data_ptr()), pb.value,
                                                 ctypes.c_void_p(self.rho_buffer.data_ptr()), rb.value))
        self.replicas = [ReplicaView(self, k, arr[k]) for k in range(self.nrep)]

    def init(self, rho_a=None, rho_b=None):
        ra = None if rho_a is None else np.ascontiguousarray(rho_a, dtype=np.float64).ravel()
        rb = None if rho_b is None else np.ascontiguousarray(rho_b, dtype=np.float64).ravel()
        check(self._h, lib().flbm_init(self._h, _dp(ra), _dp(rb)))

    def step(self, n=1):
        check(self._h, lib().flbm_step(self._h, int(n)))

    def moments(self):
        """(rho_a, rho_b, u, cons): per-replica fields concatenated, u as
        [replica][d][site] flattened, cons summed over replicas."""
        ra, rb = np.empty(self.N), np.empty(self.N)
        u = np.empty(self.D * self.N)
        cons = np.empty(5)
        check(self._h, lib().flbm_moments(self._h, _dp(ra), _dp(rb), _dp(u), _dp(cons)))
        return ra, rb, u, cons

    def get_populations(self):
        f = np.empty(2 * self.Q * self.N)
        check(self._h, lib().flbm_get_populations(self._h, _dp(f)))
        return f

    def set_populations(self, f, step=0):
        f = np.ascontiguousarray(f, dtype=np.float64).ravel()
        check(self._h, lib().flbm_set_populations(self._h, _dp(f), int(step)))

    def close(self):
        if getattr(self, "_h", None):
            self.replicas = []
            lib().flbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lattice(_Context):
    """One two-species periodic box on the GPU (a flbm_ctx).

    Device memory for the populations and the density field comes from PyTorch
    (``torch.empty`` on ``device``) and is attached to the context; the work
    runs on ``stream`` (a ``torch.cuda.Stream``; a dedicated one by default).
    """

    def __init__(self, lattice, nx, ny, nz=1, tau_a=1.0, tau_b=1.0, kT=0.0, G=0.0, seed=1,
                 storage="f32", device="cuda:0", stream=None, **options):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device visible: flbm runs on the GPU only")
        self.lattice = int(lattice)
        self.nx, self.ny = int(nx), int(ny)
        self.nz = 1 if self.lattice == D2Q9 else int(nz)
        self.D = 2 if self.lattice == D2Q9 else 3
        self.Q = 9 if self.lattice == D2Q9 else 19
        self.N = self.nx * self.ny * self.nz
        self.device = torch.device(device)
        self._h = None
        self._h = flbm_create(self.lattice, self.nx, self.ny, self.nz, tau_a, tau_b, kT, G, seed)
        self.set_option(OPT_STORAGE, STORE[storage] if isinstance(storage, str) else int(storage))
        for k, v in options.items():
            self.set_option(k, v)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        check(self._h, lib().flbm_set_stream(self._h, ctypes.c_void_p(self.stream.cuda_stream)))
        pb, rb = ctypes.c_size_t(), ctypes.c_size_t()
        check(self._h, lib().flbm_buffer_bytes(self._h, ctypes.byref(pb), ctypes.byref(rb)))
        self.pop_buffer = torch.empty(pb.value, dtype=torch.uint8, device=self.device)
        self.rho_buffer = torch.empty(rb.value, dtype=torch.uint8, device=self.device)
        check(self._h, lib().flbm_attach_buffers(self._h, ctypes.c_void_p(self.pop_buffer.data_ptr()), pb.value,
                                                 ctypes.c_void_p(self.rho_buffer.data_ptr()), rb.value))

    # -- configuration ----------------------------------------------------
    def set_mode_rate(self, species, mode, lam):
        self.set_option(OPT_LAMBDA_MODE + 100 * int(species) + int(mode), lam)

    # -- state -------------------------------------------------------------
    def init(self, rho_a=None, rho_b=None):
        ra = None if rho_a is None else np.ascontiguousarray(rho_a, dtype=np.float64).ravel()
        rb = None if rho_b is None else np.ascontiguousarray(rho_b, dtype=np.float64).ravel()
        for a in (ra, rb):
            if a is not None and a.size != self.N:
                raise ValueError("density arrays need one value per site")
        check(self._h, lib().flbm_init(self._h, _dp(ra), _dp(rb)))

    def step(self, n=1):
        check(self._h, lib().flbm_step(self._h, int(n)))

    def kernel_times(self):
        """({'density': ms, 'collide': ms}, {'density': n, 'collide': n}) accumulated
        while the kernel_timing option was on.  With the fused schedule 'density'
        is the counter reset and 'collide' the fused step kernel."""
        ms = np.zeros(2)
        n = np.zeros(2, dtype=np.int64)
        check(self._h, lib().flbm_kernel_times(self._h, _dp(ms), n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return {"density": ms[0], "collide": ms[1]}, {"density": int(n[0]), "collide": int(n[1])}

    def close(self):
        if getattr(self, "_h", None):
            lib().flbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MultiLattice:
    """One periodic box of 2 .. 4 species (App. C-D) on the GPU (a flbm_mctx):
    per-species relaxation times ``tau``, symmetric couplings ``G``
    (nspecies x nspecies, diagonal ignored).  The context owns its device
    memory; the work runs on ``stream`` (a ``torch.cuda.Stream``; a dedicated
    one by default)."""

    def __init__(self, lattice, nspecies, nx, ny, nz=1, tau=None, kT=0.0, G=None, seed=1, rho0=None,
                 device="cuda:0", stream=None, block=None, streaming="two_arrays"):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device visible: flbm runs on the GPU only")
        self.lattice, self.ns = int(lattice), int(nspecies)
        self.nx, self.ny = int(nx), int(ny)
        self.nz = 1 if self.lattice == D2Q9 else int(nz)
        self.D = 2 if self.lattice == D2Q9 else 3
        self.Q = 9 if self.lattice == D2Q9 else 19
        self.N = self.nx * self.ny * self.nz
        tau = np.ascontiguousarray(np.ones(self.ns) if tau is None else tau, dtype=np.float64)
        G = np.ascontiguousarray(np.zeros((self.ns, self.ns)) if G is None else G, dtype=np.float64)
        if tau.size != self.ns or G.size != self.ns * self.ns:
            raise ValueError("tau needs one value per species and G nspecies x nspecies")
        self._h = None
        h = ctypes.c_void_p()
        mcheck(None, lib().flbm_mcreate(self.lattice, self.ns, self.nx, self.ny, self.nz, _dp(tau), float(kT),
                                        _dp(G.ravel()), int(seed) & (2**64 - 1), ctypes.byref(h)))
        self._h = h
        if rho0 is not None:
            for s, r in enumerate(rho0):
                self.set_option(OPT_RHO0_SPECIES + s, r)
        if block is not None:
            self.set_option(OPT_BLOCK_X, block[0])
            self.set_option(OPT_BLOCK_Y, block[1])
        self.set_option(OPT_STREAMING, STREAMING[streaming] if isinstance(streaming, str) else int(streaming))
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        mcheck(self._h, lib().flbm_mset_stream(self._h, ctypes.c_void_p(self.stream.cuda_stream)))

    def set_option(self, key, value):
        mcheck(self._h, lib().flbm_mset_option(self._h, int(key), float(value)))

    def get_option(self, key):
        v = ctypes.c_double()
        mcheck(self._h, lib().flbm_mget_option(self._h, int(key), ctypes.byref(v)))
        return v.value

    def init(self, rho=None):
        """Rest state from host densities [nspecies][z][y][x] (None: the reference densities)."""
        r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64).ravel()
        if r is not None and r.size != self.ns * self.N:
            raise ValueError("densities need nspecies values per site")
        mcheck(self._h, lib().flbm_minit(self._h, _dp(r)))

    def step(self, n=1):
        mcheck(self._h, lib().flbm_mstep(self._h, int(n)))

    def sync(self):
        mcheck(self._h, lib().flbm_msync(self._h))

    @property
    def step_count(self):
        v = ctypes.c_int64()
        mcheck(self._h, lib().flbm_mget_step(self._h, ctypes.byref(v)))
        return v.value

    def kernel_times(self):
        ms = np.zeros(2)
        n = np.zeros(2, dtype=np.int64)
        mcheck(self._h, lib().flbm_mkernel_times(self._h, _dp(ms), n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return {"density": ms[0], "collide": ms[1]}, {"density": int(n[0]), "collide": int(n[1])}

    def moments(self):
        """(rho [nspecies][z][y][x], u [D][z][y][x], cons [nspecies + 3])"""
        rho = np.empty(self.ns * self.N)
        u = np.empty(self.D * self.N)
        cons = np.empty(self.ns + 3)
        mcheck(self._h, lib().flbm_mmoments(self._h, _dp(rho), _dp(u), _dp(cons)))
        shp = (self.nz, self.ny, self.nx)
        return rho.reshape((self.ns,) + shp), u.reshape((self.D,) + shp), cons

    def sf_sample(self, axis=0):
        """Add one axis structure-factor snapshot of every species pair."""
        mcheck(self._h, lib().flbm_msf_sample(self._h, int(axis)))

    def structure_factor(self, axis=0, nk=None):
        """(S [nspecies][nspecies][nk], snapshots): means at k_m = 2 pi m / n_axis, m = 1 .. nk."""
        n = (self.nx, self.ny, self.nz)[axis]
        nk = n // 2 if nk is None else int(nk)
        S = np.empty(self.ns * self.ns * max(nk, 1))
        cnt = ctypes.c_int64()
        mcheck(self._h, lib().flbm_mstructure_factor(self._h, int(axis), nk, _dp(S), ctypes.byref(cnt)))
        return S[:self.ns * self.ns * nk].reshape(self.ns, self.ns, nk), cnt.value

    def sf_reset(self):
        mcheck(self._h, lib().flbm_msf_reset(self._h))

    def checkpoint(self) -> bytes:
        n = ctypes.c_size_t()
        mcheck(self._h, lib().flbm_mcheckpoint(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        mcheck(self._h, lib().flbm_mcheckpoint(self._h, buf, ctypes.byref(n)))
        return buf.raw[:n.value]

    def restore(self, image: bytes):
        buf = ctypes.create_string_buffer(bytes(image), len(image))
        mcheck(self._h, lib().flbm_mrestore(self._h, buf, len(image)))

    def get_populations(self):
        f = np.empty(self.ns * self.Q * self.N)
        mcheck(self._h, lib().flbm_mget_populations(self._h, _dp(f)))
        return f.reshape(self.ns, self.Q, self.nz, self.ny, self.nx)

    def site_populations(self, sites):
        """Natural-layout populations [len(sites)][nspecies][Q] of the given site indices."""
        sites = np.ascontiguousarray(sites, dtype=np.int64).ravel()
        out = np.empty(sites.size * self.ns * self.Q)
        mcheck(self._h, lib().flbm_mget_site_populations(
            self._h, sites.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), sites.size, _dp(out)))
        return out.reshape(sites.size, self.ns, self.Q)

    def set_populations(self, f, step=0):
        f = np.ascontiguousarray(f, dtype=np.float64).ravel()
        if f.size != self.ns * self.Q * self.N:
            raise ValueError("populations need nspecies * Q values per site")
        mcheck(self._h, lib().flbm_mset_populations(self._h, _dp(f), int(step)))

    def close(self):
        if getattr(self, "_h", None):
            lib().flbm_mdestroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
