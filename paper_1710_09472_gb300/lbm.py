"""Thin Python front end of liblbm (one context = one simulation box).

Only argument marshalling happens here: arrays are checked for dtype, size
and contiguity and handed to the C ABI as raw pointers; every step of the
method runs in the library's CUDA kernels.  Device arrays are torch tensors
(PyTorch provides device memory and the stream); host arrays may be numpy
arrays or CPU tensors.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib

try:
    import torch
except ImportError:  # pragma: no cover - torch is part of the supported stack
    torch = None


def _ptr(a, dtype, count: int, name: str):
    """Raw pointer of a contiguous array with `count` elements of `dtype`."""
    if a is None:
        return None
    if torch is not None and isinstance(a, torch.Tensor):
        tdt = {np.float32: torch.float32, np.uint8: torch.uint8, np.float64: torch.float64}[dtype]
        if a.dtype != tdt:
            raise TypeError(f"{name}: expected {tdt}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError(f"{name}: tensor must be contiguous")
        if a.numel() != count:
            raise ValueError(f"{name}: expected {count} elements, got {a.numel()}")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if a.dtype != dtype:
            raise TypeError(f"{name}: expected {np.dtype(dtype)}, got {a.dtype}")
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name}: array must be C-contiguous")
        if a.size != count:
            raise ValueError(f"{name}: expected {count} elements, got {a.size}")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"{name}: unsupported array type {type(a)}")


def weight_integrals(D: int, stat: str = "fd", theta: float = 1.0 / 270.0, mu: float = 1.0):
    """Host-side I_0..I_8 of the weight (no device needed)."""
    out = (ctypes.c_double * 5)()
    _lib.check(_lib.load().lbm_weight_integrals(int(D), _lib.STAT[stat], float(theta), float(mu), out), None,
               "lbm_weight_integrals")
    return np.array(list(out))


def density_from_mu(D: int, theta: float, mu, rho=None, stream=None):
    """rho = (pi theta)^{D/2} g_{D/2}(e^{mu/theta}) per element (FD weight),
    mu and rho float32 CUDA tensors (lbm_density_from_mu)."""
    if rho is None:
        rho = torch.empty_like(mu)
    st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    _lib.check(_lib.load().lbm_density_from_mu(int(D), float(theta), _ptr(mu, np.float32, mu.numel(), "mu"),
                                               _ptr(rho, np.float32, mu.numel(), "rho"), mu.numel(), st), None,
               "lbm_density_from_mu")
    return rho


def mu_from_density(D: int, theta: float, rho, mu=None, stream=None):
    """The inverse of density_from_mu (lbm_mu_from_density)."""
    if mu is None:
        mu = torch.empty_like(rho)
    st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    _lib.check(_lib.load().lbm_mu_from_density(int(D), float(theta), _ptr(rho, np.float32, rho.numel(), "rho"),
                                               _ptr(mu, np.float32, rho.numel(), "mu"), rho.numel(), st), None,
               "lbm_mu_from_density")
    return mu


def _vec3(v):
    if v is None:
        return None
    out = (ctypes.c_double * 3)()
    for i, x in enumerate(list(v)[:3]):
        out[i] = float(x)
    return out


class LBM:
    """A semiclassical LBM box on the current CUDA device.

    vel: "D2V9" | "D3V19" | "D3V27" | "D1V3"; dims: (nx,), (nx, ny) or (nx, ny, nz); storage: "f32" |
    "f16" | "bf16" (deviations from the rest equilibrium, collision in FP32);
    force: "term" (explicit Lorentz term) | "shift" (velocity shift);
    stat: "fd" | "be" | "mb" weight with (theta, mu)."""

    def __init__(self, vel: str, dims, tau: float, E=(0.0, 0.0, 0.0), B=(0.0, 0.0, 0.0), storage: str = "f32",
                 force: str = "term", stat: str = "fd", theta: float = 1.0 / 270.0, mu: float = 1.0,
                 rho0: float = 1.0, stream=None):
        lib = _lib.load()
        d = list(dims) + [1] * (3 - len(dims))
        self.dims = tuple(int(x) for x in d)
        self.vel, self.storage, self.force = vel, storage, force
        lat = _lib.lbm_lattice(_lib.VEL[vel], _lib.STAT[stat], float(theta), float(mu), _lib.FORCE[force],
                               float(rho0))
        dims_c = (ctypes.c_int64 * 3)(*self.dims)
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = stream.cuda_stream if stream is not None and hasattr(stream, "cuda_stream") else stream
        self._h = ctypes.c_void_p()
        st = lib.lbm_create(ctypes.byref(self._h), ctypes.byref(lat), dims_c, float(tau), _vec3(E), _vec3(B),
                            _lib.STORAGE[storage], ctypes.c_void_p(handle or 0))
        _lib.check(st, None, "lbm_create")
        info = self.info()
        self.D, self.Q, self.N = info["D"], info["Q"], info["N"]
        self.shape = tuple(reversed(self.dims[: self.D]))  # C-order array shape (.., ny, nx)

    # -- lifetime ---------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.load().lbm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- queries ------------------------------------------------------------------
    def constants(self) -> dict:
        out = (ctypes.c_double * 40)()
        _lib.check(_lib.load().lbm_constants(self._h, out, 40), self._h, "lbm_constants")
        keys = ["I0", "I2", "I4", "c0", "c1", "c2", "cbar2", "cprime2", "thetabar", "J2", "Delta2", "cs"]
        c = dict(zip(keys, list(out)[:12]))
        q = self.Q
        c["w"] = np.array(list(out)[12: 12 + q])
        return c

    def info(self) -> dict:
        out = (ctypes.c_int64 * 9)()
        _lib.check(_lib.load().lbm_info(self._h, out, 9), self._h, "lbm_info")
        keys = ["D", "Q", "nx", "ny", "nz", "N", "n_fluid", "steps", "bytes_per_population"]
        return dict(zip(keys, list(out)))

    def launch_count(self) -> int:
        return int(_lib.load().lbm_launch_count(self._h))

    # -- set-up -------------------------------------------------------------------
    def set_geometry(self, mask):
        _lib.check(_lib.load().lbm_set_geometry(self._h, _ptr(mask, np.uint8, self.N, "mask")), self._h,
                   "lbm_set_geometry")

    def set_E_field(self, E):
        p = None if E is None else _ptr(E, np.float32, self.D * self.N, "E")
        _lib.check(_lib.load().lbm_set_E_field(self._h, p), self._h, "lbm_set_E_field")

    def set_params(self, tau: float, E=None, B=None):
        _lib.check(_lib.load().lbm_set_params(self._h, float(tau), _vec3(E), _vec3(B)), self._h, "lbm_set_params")

    def set_rounding(self, stochastic: bool):
        """Stochastic (default for f16/bf16) or round-to-nearest stores."""
        _lib.check(_lib.load().lbm_set_rounding(self._h, int(bool(stochastic))), self._h, "lbm_set_rounding")

    def set_rounding_seed(self, seed: int):
        """Seed of the stochastic-rounding stream (lbm_set_rounding_seed)."""
        _lib.check(_lib.load().lbm_set_rounding_seed(self._h, int(seed) & 0xFFFFFFFF), self._h,
                   "lbm_set_rounding_seed")

    def set_local_mu(self, enable: bool = True):
        """Local chemical-potential model (lbm_set_local_mu): each cell's
        thetabar from its own density through the FD relation rho(mu)."""
        _lib.check(_lib.load().lbm_set_local_mu(self._h, 1 if enable else 0), self._h, "lbm_set_local_mu")

    def init_equilibrium(self, rho=None, u=None):
        _lib.check(_lib.load().lbm_init_equilibrium(self._h, _ptr(rho, np.float32, self.N, "rho"),
                                                    _ptr(u, np.float32, self.D * self.N, "u")), self._h,
                   "lbm_init_equilibrium")

    # -- the hot path -------------------------------------------------------------
    def step(self, n: int = 1):
        _lib.check(_lib.load().lbm_step(self._h, int(n)), self._h, "lbm_step")

    def moments(self, rho=None, j=None, totals: bool = True):
        """Fill rho[N] / j[D*N] (either may be None) and return
        (total_rho, total_j[3]) in FP64, or None when totals is False."""
        tr = ctypes.c_double(0.0) if totals else None
        tj = (ctypes.c_double * 3)() if totals else None
        st = _lib.load().lbm_moments(self._h, _ptr(rho, np.float32, self.N, "rho"),
                                     _ptr(j, np.float32, self.D * self.N, "j"),
                                     ctypes.byref(tr) if totals else None, tj)
        _lib.check(st, self._h, "lbm_moments")
        if totals:
            return tr.value, np.array(list(tj))
        return None

    def set_memory_budget(self, nbytes: int):
        """Device bytes an adjoint call with checkpoint_every=0 may allocate (0 = free memory)."""
        _lib.check(_lib.load().lbm_set_memory_budget(self._h, int(nbytes)), self._h, "lbm_set_memory_budget")

    def release_workspace(self):
        """Free the device buffers kept by earlier adjoint calls."""
        _lib.check(_lib.load().lbm_release_workspace(self._h), self._h, "lbm_release_workspace")

    def adjoint_stats(self) -> dict:
        out = (ctypes.c_int64 * 5)()
        _lib.check(_lib.load().lbm_adjoint_stats(self._h, out), self._h, "lbm_adjoint_stats")
        return {"schedule": ["segments", "binomial", "store_all"][int(out[0])], "states": int(out[1]),
                "forward_steps": int(out[2]), "reverse_steps": int(out[3]), "state_bytes": int(out[4])}

    def selftest_wait_timeout(self, clocks: int = 1 << 20) -> int:
        """Run the bounded-wait probe (lbm_selftest_wait_timeout) and return its
        raw status; LBM_ERR_TIMEOUT is the expected answer."""
        return int(_lib.load().lbm_selftest_wait_timeout(self._h, int(clocks)))

    def moment_totals_static(self, out):
        """FP64 totals into `out` (a float64 device tensor of 4) without any
        device allocation (lbm_moment_totals_static)."""
        _lib.check(_lib.load().lbm_moment_totals_static(self._h, _ptr(out, np.float64, 4, "totals")), self._h,
                   "lbm_moment_totals_static")
        return out

    def populations(self, out=None, deviation: bool = False):
        """f_a(x, t) (or the stored deviations h_a when deviation=True), Q*N FP32."""
        if out is None:
            out = np.empty(self.Q * self.N, dtype=np.float32)
        _lib.check(_lib.load().lbm_get_populations(self._h, _ptr(out, np.float32, self.Q * self.N, "f"),
                                                   int(bool(deviation))), self._h, "lbm_get_populations")
        return out

    def window_totals(self, t_begin: int, t_end: int):
        """Advance t_end steps; return the FP64 sums over the states after steps
        t_begin+1..t_end of (sum rho, sum j_x, sum j_y, sum j_z)."""
        out = (ctypes.c_double * 4)()
        _lib.check(_lib.load().lbm_window_totals(self._h, int(t_begin), int(t_end), out), self._h,
                   "lbm_window_totals")
        return np.array(list(out))

    def adjoint(self, t_begin: int, t_end: int, w_rho=None, w_j=None, checkpoint_every: int = 0, dL_dE=None,
                dL_df0=None):
        """Run t_end steps from the current state and return the gradient of
        L = sum_{t_begin < t <= t_end} sum_x w_rho rho_t + w_j . j_t:
        dict(loss, dL_dB[3], dL_dtau); dL_dE ([D*N] float64 device tensor) and
        dL_df0 ([Q*N] float32 device tensor) are filled when given."""
        dB = (ctypes.c_double * 3)()
        dtau = ctypes.c_double(0.0)
        loss = ctypes.c_double(0.0)
        st = _lib.load().lbm_adjoint(self._h, _ptr(w_rho, np.float32, self.N, "w_rho"),
                                     _ptr(w_j, np.float32, self.D * self.N, "w_j"), int(t_begin), int(t_end),
                                     int(checkpoint_every), _ptr(dL_dE, np.float64, self.D * self.N, "dL_dE"), dB,
                                     ctypes.byref(dtau), ctypes.byref(loss),
                                     _ptr(dL_df0, np.float32, self.Q * self.N, "dL_df0"))
        _lib.check(st, self._h, "lbm_adjoint")
        return {"loss": loss.value, "dL_dB": np.array(list(dB)), "dL_dtau": dtau.value}

    def save_state(self) -> bytes:
        used = ctypes.c_size_t(0)
        lib = _lib.load()
        _lib.check(lib.lbm_save_state(self._h, None, 0, ctypes.byref(used)), self._h, "lbm_save_state")
        buf = ctypes.create_string_buffer(used.value)
        _lib.check(lib.lbm_save_state(self._h, buf, used.value, ctypes.byref(used)), self._h, "lbm_save_state")
        return buf.raw

    def load_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _lib.check(_lib.load().lbm_load_state(self._h, buf, len(blob)), self._h, "lbm_load_state")


class Thermal:
    """The 1D thermal model with the fourth-order EDF (lbm_thermal_*).

    lattice: "D1V5a" | "D1V5b" | "D1V7" | "D1V7r1" | "D1V7r2"; nx cells,
    periodic; E the uniform force (velocity shift); order 2, 3 or 4; storage
    "f32" | "f16" | "bf16".  Fields are nx FP32 device tensors."""

    def __init__(self, lattice: str, nx: int, tau: float, E: float = 0.0, order: int = 4, storage: str = "f32",
                 stat: str = "fd", theta: float = 1.0 / 270.0, mu: float = 1.0, stream=None):
        lib = _lib.load()
        h = ctypes.c_void_p()
        st = None
        if stream is not None:
            st = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        _lib.check(lib.lbm_thermal_create(ctypes.byref(h), _lib.THERMAL_LATTICE[lattice], _lib.STAT[stat],
                                          float(theta), float(mu), int(nx), float(tau), float(E), int(order),
                                          _lib.STORAGE[storage], st), None, "lbm_thermal_create")
        self._h = h
        self.nx = int(nx)
        out = (ctypes.c_double * 31)()
        _lib.check(lib.lbm_thermal_constants(self._h, out, 31), self._h, "lbm_thermal_constants", thermal=True)
        v = list(out)
        self.Q = int(v[22])
        keys = ["I0", "I2", "I4", "I6", "I8", "cs", "g", "c0", "c1", "c2", "c3", "c4", "cp2", "cp3", "cp4",
                "cb2", "cb3", "cb4", "d4", "d4p", "d4b", "thetabar_w", "Q", "tau"]
        self.const = dict(zip(keys, v[:24]))
        self.w = np.array(v[24: 24 + self.Q])

    def close(self):
        if self._h:
            _lib.load().lbm_thermal_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_rounding(self, stochastic: bool, seed: int = 0):
        _lib.check(_lib.load().lbm_thermal_set_rounding(self._h, int(bool(stochastic)), int(seed) & 0xFFFFFFFF),
                   self._h, "lbm_thermal_set_rounding", thermal=True)

    def init(self, rho=None, u=None, thetabar=None):
        n = self.nx
        _lib.check(_lib.load().lbm_thermal_init(self._h, _ptr(rho, np.float32, n, "rho"), _ptr(u, np.float32, n, "u"),
                                                _ptr(thetabar, np.float32, n, "thetabar")), self._h,
                   "lbm_thermal_init", thermal=True)

    def step(self, n: int = 1):
        _lib.check(_lib.load().lbm_thermal_step(self._h, int(n)), self._h, "lbm_thermal_step", thermal=True)

    def moments(self, rho=None, j=None, energy=None, totals: bool = True):
        n = self.nx
        tot = (ctypes.c_double * 3)() if totals else None
        _lib.check(_lib.load().lbm_thermal_moments(self._h, _ptr(rho, np.float32, n, "rho"),
                                                   _ptr(j, np.float32, n, "j"),
                                                   _ptr(energy, np.float32, n, "energy"), tot), self._h,
                   "lbm_thermal_moments", thermal=True)
        return np.array(list(tot)) if totals else None

    def populations(self, out, deviation: bool = False):
        _lib.check(_lib.load().lbm_thermal_populations(self._h, _ptr(out, np.float32, self.Q * self.nx, "f"),
                                                       int(bool(deviation))), self._h, "lbm_thermal_populations",
                   thermal=True)
        return out

    def launch_count(self) -> int:
        return int(_lib.load().lbm_thermal_launch_count(self._h))
