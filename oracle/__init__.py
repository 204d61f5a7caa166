"""FP64 CPU oracle for the fluctuating two-species lattice Boltzmann update
(arXiv 1410.5584, Sec. V, Eqs. algorithm and lattice finalstep).

TEST INFRASTRUCTURE ONLY: the yardstick the CUDA library is checked against.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The product package never imports it and shares no
code with it; the C source is ``flbm_oracle.c`` beside this file.

This module builds the C source with gcc (plain ``-O2``, IEEE semantics, no fast
math) into ``oracle/_build/`` and binds it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

D2Q9, D3Q19 = 0, 1

# option keys (same numbers as the public C-ABI's keys)
OPT_LAMBDA_D = 2
OPT_SDF = 3
OPT_RHO0_A = 4
OPT_RHO0_B = 5
OPT_NOISE_RHO = 7
OPT_FORCE_VELOCITY = 8
OPT_GHOST_NOISE = 21
OPT_LAMBDA_MODE = 1000  # + 100 * species + mode


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liborc.so (skipped when up to date)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-std=c11", "-D_DEFAULT_SOURCE", "-O2", "-fPIC", "-shared",
                    "-fopenmp", "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            vp, i32, i64, u32, u64, dbl = (ctypes.c_void_p, ctypes.c_int, ctypes.c_long,
                                           ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            up = ctypes.POINTER(ctypes.c_uint32)
            L.orc_create.restype = vp
            L.orc_create.argtypes = [i32, i32, i32, i32, dbl, dbl, dbl, dbl, u64]
            L.orc_destroy.argtypes = [vp]
            L.orc_set_option.argtypes = [vp, i32, dbl]
            L.orc_init.argtypes = [vp, dp, dp]
            L.orc_set_f.argtypes = [vp, dp, i64]
            L.orc_get_f.argtypes = [vp, dp]
            L.orc_set_threads.argtypes = [vp, i32]
            L.orc_set_rng_origin.argtypes = [vp, i64, i64, i64, i64, i64, i64]
            L.orc_get_step.restype = i64
            L.orc_get_step.argtypes = [vp]
            L.orc_step.argtypes = [vp, i64]
            L.orc_moments.argtypes = [vp, dp, dp, dp, dp]
            L.orc_sf_sample.argtypes = [vp, i32, i32]
            L.orc_structure_factor.argtypes = [vp, dp, dp, dp, dp, ctypes.POINTER(ctypes.c_long)]
            L.orc_sf_reset.argtypes = [vp]
            L.orc_tables.argtypes = [i32, ip, ip, ip, dp, dp, dp]
            L.orc_meq.argtypes = [i32, dbl, dp, dp]
            L.orc_phi.argtypes = [i32, dbl, dp, dp, dp]
            L.orc_philox4x32_10.argtypes = [up, up, up]
            L.orc_gaussian.restype = dbl
            L.orc_gaussian.argtypes = [u64, u32, u32, u32, u32]
            L.orcm_create.restype = vp
            L.orcm_create.argtypes = [i32, i32, i32, i32, i32, dp, dbl, dp, u64]
            L.orcm_destroy.argtypes = [vp]
            L.orcm_init.argtypes = [vp, dp]
            L.orcm_set_f.argtypes = [vp, dp, i64]
            L.orcm_get_f.argtypes = [vp, dp]
            L.orcm_step.argtypes = [vp, i64]
            L.orcm_moments.argtypes = [vp, dp, dp, dp]
            L.orcm_set_rng_origin.argtypes = [vp, i64, i64, i64, i64, i64, i64]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def tables(lattice: int):
    """(c [Q,3] int, w [Q], T [Q,Q] with T[a,i], N [Q]) as built by the oracle."""
    D = ctypes.c_int()
    Q = ctypes.c_int()
    c = np.zeros(19 * 3, dtype=np.int32)
    w = np.zeros(19)
    T = np.zeros(19 * 19)
    N = np.zeros(19)
    rc = lib().orc_tables(lattice, ctypes.byref(D), ctypes.byref(Q),
                          c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w), _dp(T), _dp(N))
    assert rc == 0
    q = Q.value
    return c[:q * 3].reshape(q, 3), w[:q].copy(), T[:q * q].reshape(q, q), N[:q].copy()


def meq(lattice: int, rho: float, u) -> np.ndarray:
    u3 = np.zeros(3)
    u3[:len(u)] = u
    out = np.zeros(19)
    lib().orc_meq(lattice, rho, _dp(u3), _dp(out))
    return out[:19 if lattice == D3Q19 else 9]


def phi(lattice: int, rho: float, acc, v) -> np.ndarray:
    a3 = np.zeros(3)
    a3[:len(acc)] = acc
    v3 = np.zeros(3)
    v3[:len(v)] = v
    out = np.zeros(19)
    lib().orc_phi(lattice, rho, _dp(a3), _dp(v3), _dp(out))
    return out[:19 if lattice == D3Q19 else 9]


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def gaussian(seed: int, site: int, step: int, species: int, mode: int) -> float:
    """The standard Gaussian of mode >= 1 of a species at (site, step): its
    Gaussian n = mode - 1, from Philox4x32-10 block n // 6 cut into six 21-bit
    uniforms (orc_gaussian in flbm_oracle.c); NaN for mode 0."""
    return lib().orc_gaussian(seed, site, step, species, mode)


class MultiOracle:
    """The N-species update (App. C-D) in FP64: rates 1/tau_s per species, the
    common momentum rate N / sum tau_s, mean-field forces G[s][t] between
    different species (diagonal ignored), projected momentum noise."""

    def __init__(self, lattice, nspecies, nx, ny, nz, tau, kT, G, seed):
        self.lattice, self.ns = int(lattice), int(nspecies)
        c, w, T, N = tables(lattice)
        self.Q, self.D = len(w), 2 if lattice == D2Q9 else 3
        self.nx, self.ny = int(nx), int(ny)
        self.nz = 1 if lattice == D2Q9 else int(nz)
        self.N = self.nx * self.ny * self.nz
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        G = np.ascontiguousarray(G, dtype=np.float64).reshape(self.ns, self.ns)
        assert tau.size == self.ns
        self._h = lib().orcm_create(self.lattice, self.ns, self.nx, self.ny, self.nz, _dp(tau), float(kT),
                                    _dp(G), int(seed) & (2 ** 64 - 1))
        if not self._h:
            raise ValueError("bad multi-species oracle parameters")

    def init(self, rho=None):
        r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64).ravel()
        lib().orcm_init(self._h, _dp(r))

    def set_f(self, f, step=0):
        f = np.ascontiguousarray(f, dtype=np.float64).ravel()
        assert f.size == self.ns * self.Q * self.N
        lib().orcm_set_f(self._h, _dp(f), int(step))

    def get_f(self):
        f = np.zeros(self.ns * self.Q * self.N)
        lib().orcm_get_f(self._h, _dp(f))
        return f.reshape(self.ns, self.Q, self.nz, self.ny, self.nx)

    def set_rng_origin(self, global_shape, origin):
        """Draw the noise of local site (x, y, z) with the index of site
        (x, y, z) + origin of a periodic box of shape (nz, ny, nx)."""
        gnz, gny, gnx = global_shape
        oz, oy, ox = origin
        lib().orcm_set_rng_origin(self._h, gnx, gny, gnz, ox, oy, oz)

    def step(self, n=1):
        if lib().orcm_step(self._h, int(n)) != 0:
            raise FloatingPointError("a density became non-positive")

    def moments(self):
        """(rho [ns][z][y][x], u [D][z][y][x], cons [ns + 3])"""
        rho = np.zeros(self.ns * self.N)
        u = np.zeros(self.D * self.N)
        cons = np.zeros(self.ns + 3)
        lib().orcm_moments(self._h, _dp(rho), _dp(u), _dp(cons))
        shp = (self.nz, self.ny, self.nx)
        return rho.reshape((self.ns,) + shp), u.reshape((self.D,) + shp), cons

    def close(self):
        if getattr(self, "_h", None):
            lib().orcm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def structure_factor_full(rho_a, rho_b):
    """Structure factors of one snapshot at every lattice wavevector (the
    quantities of Eq. str-bin-hom, Sec. IV A, off the axes too).  With
    rho_hat(k) = sum_r (rho(r) - <rho>) exp(-i k.r) and k_alpha = 2 pi m_alpha /
    n_alpha: S_aa = |rho_hat_a|^2 / N, S_ab = Re(rho_hat_a conj rho_hat_b) / N,
    S_bb = |rho_hat_b|^2 / N, arrays shaped like the fields ([z][y][x], m_alpha
    in numpy FFT order; k = 0 is 0).  numpy's FFT is the library step of the
    definition."""
    a = np.asarray(rho_a, dtype=np.float64)
    b = np.asarray(rho_b, dtype=np.float64)
    n = a.size
    fa = np.fft.fftn(a - a.mean())
    fb = np.fft.fftn(b - b.mean())
    return np.abs(fa) ** 2 / n, (fa * np.conj(fb)).real / n, np.abs(fb) ** 2 / n


def structure_functions(s_aa, s_ab, s_bb, rho0_a, rho0_b):
    """(S_tt, S_CC, S_tC) of Eq. structurefunctions from the density structure
    factors: total density rho_t = rho + rho' and concentration C = rho / rho_t
    linearised about (rho0_a, rho0_b), delta rho_t = delta rho + delta rho',
    delta C = (rho0_b delta rho - rho0_a delta rho') / rho_t0^2."""
    rt = rho0_a + rho0_b
    s_tt = s_aa + 2.0 * s_ab + s_bb
    s_cc = (rho0_b ** 2 * s_aa - 2.0 * rho0_a * rho0_b * s_ab + rho0_a ** 2 * s_bb) / rt ** 4
    s_tc = (rho0_b * s_aa + (rho0_b - rho0_a) * s_ab - rho0_a * s_bb) / rt ** 2
    return s_tt, s_cc, s_tc


def interface_heights(rho_a, x_liquid, x_gas):
    """Heights of the two interfaces of a stripe (Sec. VI B): rho_a[y][x] of a
    D2Q9 box whose A-rich stripe contains column x_liquid and whose B-rich
    region contains column x_gas.  The bulk values rho_l, rho_g are the means
    of rho_a over y at those columns; in the window of columns from x_gas up
    to x_liquid (periodic) and in the one from x_liquid up to x_gas, the
    liquid fraction L(y) = sum_x (rho_a - rho_g) / (rho_l - rho_g) places the
    dividing surface (Gibbs), column x covering [x - 1/2, x + 1/2):
    h1(y) = x_liquid - 1/2 - L1(y), h2(y) = x_liquid - 1/2 + L2(y), in the
    frame of x_liquid (h1 may be negative when the window wraps).  Returns
    (h1, h2) as float arrays over y."""
    r = np.asarray(rho_a, dtype=np.float64)
    ny, nx = r.shape
    rl, rg = r[:, x_liquid].mean(), r[:, x_gas].mean()
    frac = (r - rg) / (rl - rg)
    w1 = [(x_gas + k) % nx for k in range((x_liquid - x_gas) % nx)]
    w2 = [(x_liquid + k) % nx for k in range((x_gas - x_liquid) % nx)]
    h1 = x_liquid - 0.5 - frac[:, w1].sum(axis=1)
    h2 = x_liquid - 0.5 + frac[:, w2].sum(axis=1)
    return h1, h2


def track_stripe(rho_a):
    """Bulk columns of a stripe that may have moved: with C(x) the sum over y of
    rho_a, the window of n_x/2 consecutive columns (periodic) with the largest
    sum of C holds the stripe (ties: the lowest first column x0); returns
    (x_liquid, x_gas) = (x0 + w/2, x0 + w/2 + n_x/2) mod n_x with w = n_x/2."""
    r = np.asarray(rho_a, dtype=np.float64)
    ny, nx = r.shape
    c = r.sum(axis=0)
    w = nx // 2
    sums = np.array([sum(c[(x0 + k) % nx] for k in range(w)) for x0 in range(nx)])
    x0 = int(np.argmax(sums))  # the first maximum
    xl = (x0 + w // 2) % nx
    return xl, (xl + nx // 2) % nx


def height_spectrum(h):
    """S_h(k_m) = |sum_y (h(y) - <h>) exp(-i k_m y)|^2 / n_y, k_m = 2 pi m / n_y,
    m = 1 .. n_y / 2 (the capillary spectrum of Eq. predictionspectrum per unit
    length); numpy's FFT is the library step."""
    h = np.asarray(h, dtype=np.float64)
    ny = h.size
    f = np.fft.fft(h - h.mean())
    return np.abs(f[1:ny // 2 + 1]) ** 2 / ny


class Oracle:
    """Handle on one oracle lattice (two species, periodic box)."""

    def __init__(self, lattice, nx, ny, nz, tau_a, tau_b, kT, G, seed, **options):
        self.lattice = lattice
        self.nx, self.ny = nx, ny
        self.nz = 1 if lattice == D2Q9 else nz
        self.D = 2 if lattice == D2Q9 else 3
        self.Q = 9 if lattice == D2Q9 else 19
        self.N = self.nx * self.ny * self.nz
        self._h = lib().orc_create(lattice, nx, ny, self.nz, tau_a, tau_b, kT, G, seed)
        if not self._h:
            raise MemoryError("orc_create failed")
        for k, v in options.items():
            self.set_option(k, v)

    def set_threads(self, n: int):
        """OpenMP threads for the site loops (the arithmetic is unchanged)."""
        lib().orc_set_threads(self._h, int(n))

    def set_rng_origin(self, global_shape, origin):
        """Draw the noise of local site (x, y, z) with the index of site
        (x, y, z) + origin of a periodic box of shape (nz, ny, nx)."""
        gnz, gny, gnx = global_shape
        oz, oy, ox = origin
        lib().orc_set_rng_origin(self._h, gnx, gny, gnz, ox, oy, oz)

    def set_option(self, key, value):
        if isinstance(key, str):
            key = {"lambda_d": OPT_LAMBDA_D, "sdf": OPT_SDF, "rho0_a": OPT_RHO0_A,
                   "rho0_b": OPT_RHO0_B, "noise_rho": OPT_NOISE_RHO,
                   "force_velocity": OPT_FORCE_VELOCITY, "ghost_noise": OPT_GHOST_NOISE}[key]
        if lib().orc_set_option(self._h, int(key), float(value)) != 0:
            raise ValueError(f"bad oracle option {key}")

    def set_mode_rate(self, species, mode, lam):
        self.set_option(OPT_LAMBDA_MODE + 100 * species + mode, lam)

    def init(self, rho_a=None, rho_b=None):
        ra = None if rho_a is None else np.ascontiguousarray(rho_a, dtype=np.float64).ravel()
        rb = None if rho_b is None else np.ascontiguousarray(rho_b, dtype=np.float64).ravel()
        lib().orc_init(self._h, _dp(ra), _dp(rb))

    def step(self, n=1):
        rc = lib().orc_step(self._h, int(n))
        if rc != 0:
            raise FloatingPointError(f"oracle step failed with status {rc}")

    @property
    def step_count(self):
        return lib().orc_get_step(self._h)

    def get_f(self) -> np.ndarray:
        """Populations, natural layout [species][i][z][y][x]."""
        f = np.zeros(2 * self.Q * self.N)
        lib().orc_get_f(self._h, _dp(f))
        return f.reshape(2, self.Q, self.nz, self.ny, self.nx)

    def set_f(self, f, step=0):
        f = np.ascontiguousarray(f, dtype=np.float64).ravel()
        assert f.size == 2 * self.Q * self.N
        lib().orc_set_f(self._h, _dp(f), int(step))

    def moments(self):
        ra = np.zeros(self.N)
        rb = np.zeros(self.N)
        u = np.zeros(self.D * self.N)
        cons = np.zeros(5)
        lib().orc_moments(self._h, _dp(ra), _dp(rb), _dp(u), _dp(cons))
        shp = (self.nz, self.ny, self.nx)
        return ra.reshape(shp), rb.reshape(shp), u.reshape((self.D,) + shp), cons

    def sf_sample(self, axis=0, nk=None):
        n_axis = (self.nx, self.ny, self.nz)[axis]
        nk = n_axis // 2 if nk is None else nk
        self._sf_nk = nk
        if lib().orc_sf_sample(self._h, axis, nk) != 0:
            raise ValueError("bad structure-factor axis or nk")

    def structure_factor(self):
        nk = self._sf_nk
        out = [np.zeros(nk) for _ in range(4)]
        n = ctypes.c_long()
        lib().orc_structure_factor(self._h, *[_dp(o) for o in out], ctypes.byref(n))
        return (*out, n.value)

    def sf_reset(self):
        lib().orc_sf_reset(self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
