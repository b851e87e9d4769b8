"""FP64 CPU oracle for the semiclassical lattice Boltzmann method (arXiv 1710.09472).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path never
does.  It is a thin ctypes wrapper around ``lbm_oracle.c`` (plain C, double
precision), which restates the paper step by step and shares no code with the
CUDA library.

Functions and the passages they follow:
  weight_integrals   Sec. 3, Eq. i2n-cont2 (I_2N of the weight omega)
  coefficients       Sec. 3 (c_K, cbar_K, c'_K, Delta_2K, J_2K); Sec. 9.1 (thetabar)
  Model              Sec. 8 + Table lattices-tab (lattices), Sec. 9.1 (EDF, step)
  Model.equilibrium  Sec. 9.1, Eq. feq-reduced-applied-electrons-in-metals-eq
  Model.force_term   Sec. 7, Eq. forcing-term-integrals-eq
  Model.equilibrium_thetabar, Model.step_local_mu, Model.adjoint_local_mu
                     Sec. 9.1, Eq. feq-exp-2nd-order-eq with the cell's own
                     thetabar = I_2/I_0 at its chemical potential (Sec. 5, Eq.
                     omega-feq; the lattice stays the weight's), and its
                     reverse sweep
  Model.step         Sec. 9.1 discrete Boltzmann equation (collide, then stream)
  Model.adjoint      reverse sweep of Model.step (chain rule of the above)

Fourth-order equilibrium and the 1D thermal model (``lbm_oracle4.c``):
  coefficients4      Sec. 3 (c_K for K <= 4, c'_K, cbar_K, d_4, d'_4, dbar_4)
  polynomials        Sec. 3 (P_0 .. P_4 as dense tensors)
  projections        Sec. 4 (A_0 .. A_4 of an isotropic EDF shifted by u)
  edf                Sec. 4, Eq. feq-4order-01 (the contraction to order N)
  lattice1d          Table lattices-tab (D1V5 a/b), App. A (D1V7)
  Thermal            the 1D thermal model on D1V5/D1V7 (readings in lbm_oracle4.c)
  fd_integral        Sec. 4 (g_nu of the FD/BE EDF)
  density_of_mu      Sec. 9.1, Eq. rho-def-eq; mu_of_density its inverse (Sec. 9.1.2)

Every function is pinned in tests/ against something other than itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_SRC4 = os.path.join(_HERE, "lbm_oracle4.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liblbm_oracle.so")

STAT = {"fd": 0, "be": 1, "mb": 2}
VEL = {"D1V3": 0, "D2V9": 1, "D3V15": 2, "D3V19": 3, "D3V27": 4}
FORCE = {"shift": 0, "term": 1}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC4))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, _SRC4, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    i64p = ctypes.POINTER(ctypes.c_int64)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    vp = ctypes.c_void_p
    lib.or_weight_integrals.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, dp]
    lib.or_coefficients.argtypes = [ctypes.c_int, dp, dp]
    lib.or_lattice.argtypes = [ctypes.c_int, dp, ip, dp, ip, dp]
    lib.or_model_size.restype = ctypes.c_int
    lib.or_model_init.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, dp, dp, ctypes.c_int]
    lib.or_model_constants.argtypes = [vp, dp]
    lib.or_model_velocities.argtypes = [vp, ip, ip]
    lib.or_equilibrium.argtypes = [vp, ctypes.c_double, dp, dp]
    lib.or_force_term.argtypes = [vp, ctypes.c_double, dp, dp, dp]
    lib.or_collide_cell.argtypes = [vp, dp, dp, dp]
    lib.or_equilibrium_thetabar.argtypes = [vp, ctypes.c_double, dp, ctypes.c_double, dp]
    lib.or_collide_cell_thetabar.argtypes = [vp, dp, dp, ctypes.c_double, dp]
    lib.or_step_thetabar.argtypes = [vp, i64p, u8p, dp, dp, dp, dp]
    lib.or_adjoint_thetabar.argtypes = [vp, i64p, u8p, dp, dp, dp, dp, ctypes.c_int64, ctypes.c_int64, dp, dp,
                                        dp, dp, dp, dp, dp]
    lib.or_init_equilibrium.argtypes = [vp, i64p, u8p, dp, dp, dp]
    lib.or_step.argtypes = [vp, i64p, u8p, dp, dp, dp, ctypes.c_int64]
    lib.or_moments.argtypes = [vp, i64p, u8p, dp, dp, dp, dp]
    lib.or_collide_cell_adjoint.argtypes = [vp, dp, dp, dp, dp, dp, dp, dp]
    lib.or_adjoint.argtypes = [vp, i64p, u8p, dp, dp, ctypes.c_int64, ctypes.c_int64, dp, dp, dp, dp,
                               dp, dp, dp]
    lib.or_num_threads.restype = ctypes.c_int
    lib.or_coefficients4.argtypes = [ctypes.c_int, dp, dp]
    lib.or_polynomials.argtypes = [ctypes.c_int, dp, dp, dp]
    lib.or_projections.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, ctypes.c_double, ctypes.c_double, dp]
    lib.or_edf.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, dp, ctypes.c_double, dp,
                           ctypes.c_double, ctypes.c_double]
    lib.or_edf.restype = ctypes.c_double
    lib.or_lattice1d.argtypes = [ctypes.c_int, dp, ip, dp, dp]
    lib.or_thermal_size.restype = ctypes.c_int
    lib.or_thermal_init.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int]
    lib.or_thermal_constants.argtypes = [vp, dp]
    lib.or_thermal_equilibrium.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
    lib.or_thermal_collide_cell.argtypes = [vp, dp, ctypes.c_double, dp]
    lib.or_thermal_step.argtypes = [vp, ctypes.c_int64, dp, dp, dp, ctypes.c_int64]
    lib.or_thermal_init_state.argtypes = [vp, ctypes.c_int64, dp, dp, dp, dp]
    lib.or_thermal_moments.argtypes = [vp, ctypes.c_int64, dp, dp, dp, dp, dp]
    lib.or_fd_integral.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int]
    lib.or_fd_integral.restype = ctypes.c_double
    lib.or_density_of_mu.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    lib.or_density_of_mu.restype = ctypes.c_double
    lib.or_mu_of_density.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    lib.or_mu_of_density.restype = ctypes.c_double
    _lib = lib
    return lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8p(a):
    if a is None:
        return None
    assert a.dtype == np.uint8 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def num_threads() -> int:
    return int(_load().or_num_threads())


def weight_integrals(D: int, stat: str = "fd", theta: float = 1.0 / 270.0, mu: float = 1.0,
                     nmax: int = 4) -> np.ndarray:
    """I_0, I_2, ..., I_{2 nmax} of the weight (Sec. 3, Eq. i2n-cont2)."""
    out = np.zeros(nmax + 1)
    rc = _load().or_weight_integrals(D, STAT[stat], theta, mu, nmax, _dp(out))
    if rc != 0:
        raise ValueError("bad weight-integral arguments")
    return out


def coefficients(D: int, I: np.ndarray) -> dict:
    """Second-order polynomial coefficients and thetabar (Sec. 3; Sec. 9.1)."""
    I = np.ascontiguousarray(I[:3], dtype=np.float64)
    out = np.zeros(8)
    _load().or_coefficients(D, _dp(I), _dp(out))
    keys = ["c0", "c1", "c2", "cbar2", "cprime2", "thetabar", "J2", "Delta2"]
    return dict(zip(keys, out.tolist()))


def lattice(vel: str, I: np.ndarray):
    """(e[Q,3], w[Q], opp[Q], c_s) of a lattice from Table lattices-tab; raises
    ValueError('unstable') when a weight or c_s is not positive (Sec. 8)."""
    I4 = np.zeros(5)
    I4[: len(I)] = I
    e = np.zeros(3 * 27, dtype=np.int32)
    w = np.zeros(27)
    opp = np.zeros(27, dtype=np.int32)
    cs = ctypes.c_double(0.0)
    q = _load().or_lattice(VEL[vel], _dp(I4), e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                           opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.byref(cs))
    if q == -2:
        raise ValueError("unstable")
    if q < 0:
        raise ValueError("bad lattice")
    return e[: 3 * q].reshape(q, 3).copy(), w[:q].copy(), opp[:q].copy(), cs.value


class Model:
    """A configured model: lattice + weight + tau + uniform E, B + force mode."""

    def __init__(self, vel: str = "D2V9", stat: str = "fd", theta: float = 1.0 / 270.0, mu: float = 1.0,
                 tau: float = 0.8, E=(0.0, 0.0, 0.0), B=(0.0, 0.0, 0.0), force: str = "term"):
        lib = _load()
        self._buf = ctypes.create_string_buffer(lib.or_model_size())
        E3 = np.zeros(3)
        E3[: len(E)] = E
        B3 = np.zeros(3)
        B3[: len(B)] = B
        rc = lib.or_model_init(self._buf, VEL[vel], STAT[stat], theta, mu, tau, _dp(E3), _dp(B3),
                               FORCE[force])
        if rc == -2:
            raise ValueError("unstable lattice (a weight or c_s is not positive)")
        if rc != 0:
            raise ValueError("bad model arguments")
        self.vel, self.stat, self.force, self.tau = vel, stat, force, tau
        self.theta, self.mu = theta, mu
        self.D = {"D1V3": 1, "D2V9": 2}.get(vel, 3)
        self.E = E3.copy()
        self.B = B3.copy()
        if self.D < 3:  # the model keeps only the in-plane E and B_z in 2D
            self.E[2] = 0.0
            self.B[0] = self.B[1] = 0.0
        out = np.zeros(12 + 27)
        self.Q = lib.or_model_constants(self._buf, _dp(out))
        keys = ["I0", "I2", "I4", "c0", "c1", "c2", "cbar2", "cprime2", "thetabar", "J2", "Delta2", "cs"]
        self.const = dict(zip(keys, out[:12].tolist()))
        self.w = out[12: 12 + self.Q].copy()
        e = np.zeros(3 * 27, dtype=np.int32)
        opp = np.zeros(27, dtype=np.int32)
        lib.or_model_velocities(self._buf, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        self.e = e[: 3 * self.Q].reshape(self.Q, 3).copy()
        self.opp = opp[: self.Q].copy()
        self.xi = self.e / self.const["cs"]

    # --- single-cell pieces -------------------------------------------------
    def equilibrium(self, rho: float, u) -> np.ndarray:
        u3 = np.zeros(3)
        u3[: len(u)] = u
        out = np.zeros(self.Q)
        _load().or_equilibrium(self._buf, float(rho), _dp(u3), _dp(out))
        return out

    def equilibrium_thetabar(self, rho: float, u, thetabar: float) -> np.ndarray:
        """Eq. feq-exp-2nd-order-eq with the reduced temperature as an argument."""
        u3 = np.zeros(3)
        u3[: len(u)] = u
        out = np.zeros(self.Q)
        _load().or_equilibrium_thetabar(self._buf, float(rho), _dp(u3), float(thetabar), _dp(out))
        return out

    def collide_cell_thetabar(self, fc: np.ndarray, thetabar: float, E=None) -> np.ndarray:
        fc = np.ascontiguousarray(fc, dtype=np.float64)
        E3 = np.zeros(3)
        if E is None:
            E3[:] = self._uniform_E()
        else:
            E3[: len(E)] = E
        out = np.zeros(self.Q)
        _load().or_collide_cell_thetabar(self._buf, _dp(fc), _dp(E3), float(thetabar), _dp(out))
        return out

    def force_term(self, rho: float, u, E) -> np.ndarray:
        u3 = np.zeros(3)
        u3[: len(u)] = u
        E3 = np.zeros(3)
        E3[: len(E)] = E
        out = np.zeros(self.Q)
        _load().or_force_term(self._buf, float(rho), _dp(u3), _dp(E3), _dp(out))
        return out

    def collide_cell(self, fc: np.ndarray, E=None) -> np.ndarray:
        fc = np.ascontiguousarray(fc, dtype=np.float64)
        E3 = np.zeros(3)
        if E is None:
            E3[:] = self._uniform_E()
        else:
            E3[: len(E)] = E
        out = np.zeros(self.Q)
        _load().or_collide_cell(self._buf, _dp(fc), _dp(E3), _dp(out))
        return out

    def _uniform_E(self):
        return self.E

    # --- grids ---------------------------------------------------------------
    @staticmethod
    def _dims(shape):
        n = list(shape)[::-1]  # shape is (nz, ny, nx) / (ny, nx) -> n = (nx, ny, nz)
        while len(n) < 3:
            n.append(1)
        return np.array(n, dtype=np.int64)

    def init_equilibrium(self, shape, solid, rho, u=None) -> np.ndarray:
        """f(x, 0) = f^eq(rho(x), u(x)); arrays in C order over `shape`."""
        n = self._dims(shape)
        N = int(np.prod(n))
        solid_a = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8).reshape(N)
        rho_a = np.ascontiguousarray(np.broadcast_to(rho, shape), dtype=np.float64).reshape(N)
        u_a = None
        if u is not None:
            u_a = np.ascontiguousarray(u, dtype=np.float64).reshape(self.D * N)
        f = np.zeros(self.Q * N)
        _load().or_init_equilibrium(self._buf, n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                    _u8p(solid_a), _dp(rho_a), _dp(u_a), _dp(f))
        return f

    def step(self, shape, solid, f: np.ndarray, nsteps: int, Efield=None) -> np.ndarray:
        """Advance f (Q*N, float64) in place by nsteps collide-and-stream steps."""
        n = self._dims(shape)
        N = int(np.prod(n))
        assert f.shape == (self.Q * N,)
        solid_a = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8).reshape(N)
        E_a = None if Efield is None else np.ascontiguousarray(Efield, dtype=np.float64).reshape(self.D * N)
        tmp = np.empty_like(f)
        _load().or_step(self._buf, n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _u8p(solid_a),
                        _dp(E_a), _dp(f), _dp(tmp), int(nsteps))
        return f

    def moments(self, shape, solid, f: np.ndarray):
        """(rho[shape], j[D, *shape], totals[4] = (sum rho, sum j_x, sum j_y, sum j_z))."""
        n = self._dims(shape)
        N = int(np.prod(n))
        solid_a = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8).reshape(N)
        rho = np.zeros(N)
        j = np.zeros(self.D * N)
        tot = np.zeros(4)
        _load().or_moments(self._buf, n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _u8p(solid_a),
                           _dp(np.ascontiguousarray(f)), _dp(rho), _dp(j), _dp(tot))
        return rho.reshape(shape), j.reshape((self.D,) + tuple(shape)), tot

    def local_thetabar(self, rho, rho_ref: float | None = None) -> np.ndarray:
        """thetabar(x) = I_2/I_0 at the chemical potential mu(x) of the cell:
        I_0(mu(x)) = rho(x) I_0(mu_w) / rho_ref (Sec. 9.1, Eq. rho-def-eq; the
        density is in units where rho_ref is the weight's own density, by
        default rho_ref = I_0(mu_w), i.e. physical units)."""
        return thetabar_of_density(self.D, self.stat, self.theta, self.mu, rho, rho_ref)

    def step_local_mu(self, shape, solid, f: np.ndarray, nsteps: int, Efield=None,
                      rho_ref: float | None = None) -> np.ndarray:
        """Advance f in place by nsteps steps of the model with the local
        thetabar: before each collision every fluid cell takes thetabar from
        its own density (local_thetabar), then Eq. feq-exp-2nd-order-eq."""
        n = self._dims(shape)
        N = int(np.prod(n))
        assert f.shape == (self.Q * N,)
        solid_a = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8).reshape(N)
        E_a = None if Efield is None else np.ascontiguousarray(Efield, dtype=np.float64).reshape(self.D * N)
        fluid = np.ones(N, dtype=bool) if solid_a is None else solid_a == 0
        tmp = np.empty_like(f)
        for _ in range(nsteps):
            rho = self.moments(shape, solid, f)[0].reshape(N)
            thb = np.full(N, self.const["thetabar"])
            thb[fluid] = self.local_thetabar(rho[fluid], rho_ref)
            _load().or_step_thetabar(self._buf, n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _u8p(solid_a),
                                     _dp(E_a), _dp(thb), _dp(f), _dp(tmp))
        return f

    def trajectory(self, shape, solid, f0: np.ndarray, nsteps: int, Efield=None) -> np.ndarray:
        """States f_0..f_T stacked as (T+1, Q*N)."""
        out = np.empty((nsteps + 1, f0.size))
        out[0] = f0
        f = f0.copy()
        for t in range(nsteps):
            self.step(shape, solid, f, 1, Efield)
            out[t + 1] = f
        return out

    def adjoint(self, shape, solid, states: np.ndarray, t_begin: int, t_end: int, wr=None, wj=None,
                Efield=None):
        """Reverse sweep over a stored trajectory (states[t] = f_t, t = 0..t_end).

        Loss L = sum_{t_begin < t <= t_end} sum_x wr(x) rho_t(x) + wj(x).j_t(x).
        Returns dict(loss, lam0[Q*N], gE[D, *shape], gB[3], gtau)."""
        n = self._dims(shape)
        N = int(np.prod(n))
        assert states.shape[0] >= t_end + 1
        solid_a = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8).reshape(N)
        E_a = None if Efield is None else np.ascontiguousarray(Efield, dtype=np.float64).reshape(self.D * N)
        wr_a = None if wr is None else np.ascontiguousarray(wr, dtype=np.float64).reshape(N)
        wj_a = None if wj is None else np.ascontiguousarray(wj, dtype=np.float64).reshape(self.D * N)
        st = np.ascontiguousarray(states[: t_end + 1], dtype=np.float64)
        lam0 = np.zeros(self.Q * N)
        gE = np.zeros(self.D * N)
        gB = np.zeros(3)
        gtau = np.zeros(1)
        loss = np.zeros(1)
        _load().or_adjoint(self._buf, n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _u8p(solid_a),
                           _dp(E_a), _dp(st), int(t_begin), int(t_end), _dp(wr_a), _dp(wj_a), _dp(lam0),
                           _dp(gE), _dp(gB), _dp(gtau), _dp(loss))
        return {"loss": float(loss[0]), "lam0": lam0, "gE": gE.reshape((self.D,) + tuple(shape)),
                "gB": gB, "gtau": float(gtau[0])}


    def adjoint_local_mu(self, shape, solid, states: np.ndarray, t_begin: int, t_end: int, wr=None, wj=None,
                         Efield=None, rho_ref: float | None = None):
        """Reverse sweep of step_local_mu over its stored trajectory: as
        adjoint(), with every cell's thetabar and d thetabar / d rho taken
        from its density in each state."""
        n = self._dims(shape)
        N = int(np.prod(n))
        assert states.shape[0] >= t_end + 1
        solid_a = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8).reshape(N)
        fluid = np.ones(N, dtype=bool) if solid_a is None else solid_a == 0
        thb = np.full((t_end + 1, N), self.const["thetabar"])
        dthb = np.zeros((t_end + 1, N))
        for t in range(t_end + 1):
            rho = self.moments(shape, solid, states[t])[0].reshape(N)[fluid]
            thb[t, fluid] = self.local_thetabar(rho, rho_ref)
            dthb[t, fluid] = thetabar_slope_of_density(self.D, self.stat, self.theta, self.mu, rho, rho_ref)
        E_a = None if Efield is None else np.ascontiguousarray(Efield, dtype=np.float64).reshape(self.D * N)
        wr_a = None if wr is None else np.ascontiguousarray(wr, dtype=np.float64).reshape(N)
        wj_a = None if wj is None else np.ascontiguousarray(wj, dtype=np.float64).reshape(self.D * N)
        st = np.ascontiguousarray(states[: t_end + 1], dtype=np.float64)
        lam0 = np.zeros(self.Q * N)
        gE = np.zeros(self.D * N)
        gB = np.zeros(3)
        gtau = np.zeros(1)
        loss = np.zeros(1)
        _load().or_adjoint_thetabar(self._buf, n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _u8p(solid_a),
                                    _dp(E_a), _dp(st), _dp(thb), _dp(dthb), int(t_begin), int(t_end), _dp(wr_a),
                                    _dp(wj_a), _dp(lam0), _dp(gE), _dp(gB), _dp(gtau), _dp(loss))
        return {"loss": float(loss[0]), "lam0": lam0, "gE": gE.reshape((self.D,) + tuple(shape)),
                "gB": gB, "gtau": float(gtau[0])}


# ---------------------------------------------------------------------------
# Fourth-order EDF and the 1D thermal model (lbm_oracle4.c).
# ---------------------------------------------------------------------------
COEF4_KEYS = ["c0", "c1", "c2", "c3", "c4", "cp2", "cp3", "cp4", "cb2", "cb3", "cb4", "d4", "d4p", "d4b",
              "Delta2", "Delta4", "Delta6"]
LATTICE1D = {"D1V5a": 0, "D1V5b": 1, "D1V7": 2, "D1V7r1": 3, "D1V7r2": 4}


def coefficients4(D: int, I: np.ndarray) -> np.ndarray:
    """The 17 coefficients of Sec. 3 up to K = 4 (order of COEF4_KEYS)."""
    I = np.ascontiguousarray(I[:5], dtype=np.float64)
    out = np.zeros(17)
    if _load().or_coefficients4(D, _dp(I), _dp(out)) != 0:
        raise ValueError("coefficients undefined for these weight integrals")
    return out


def _split(D, flat):
    out, off = [], 0
    for N in range(5):
        n = D ** N
        out.append(flat[off: off + n].reshape((D,) * N))
        off += n
    return out


def polynomials(D: int, co: np.ndarray, xi) -> list:
    """[P_0, P_i, P_ij, P_ijk, P_ijkl] at xi (Sec. 3)."""
    x = np.ascontiguousarray(np.asarray(xi, dtype=np.float64).reshape(D))
    flat = np.zeros(sum(D ** N for N in range(5)))
    _load().or_polynomials(D, _dp(np.ascontiguousarray(co, dtype=np.float64)), _dp(x), _dp(flat))
    return _split(D, flat)


def projections(D: int, co: np.ndarray, rho: float, u, thetabar: float, g: float) -> list:
    """[A_0, A_i, ..., A_ijkl] of Sec. 4."""
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(D))
    flat = np.zeros(sum(D ** N for N in range(5)))
    _load().or_projections(D, _dp(np.ascontiguousarray(co, dtype=np.float64)), float(rho), _dp(uu),
                           float(thetabar), float(g), _dp(flat))
    return _split(D, flat)


def edf(D: int, order: int, co: np.ndarray, w_a: float, xi_a, rho: float, u, thetabar: float, g: float) -> float:
    """Eq. feq-4order-01 truncated at `order`, at one lattice vector."""
    x = np.ascontiguousarray(np.asarray(xi_a, dtype=np.float64).reshape(D))
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(D))
    return float(_load().or_edf(D, order, _dp(np.ascontiguousarray(co, dtype=np.float64)), float(w_a), _dp(x),
                                float(rho), _dp(uu), float(thetabar), float(g)))


def lattice1d(kind: str, I: np.ndarray):
    """(e[Q], w[Q], c_s) of D1V5a/D1V5b (Table lattices-tab) or D1V7 with root
    0 (the printed closed form), 1 or 2 of its cubic (App. A)."""
    I = np.ascontiguousarray(I[:5], dtype=np.float64)
    e = np.zeros(7, dtype=np.int32)
    w = np.zeros(7)
    cs = np.zeros(1)
    q = _load().or_lattice1d(LATTICE1D[kind], _dp(I), e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                             _dp(cs))
    if q == -2:
        raise ValueError("unstable")
    if q < 0:
        raise ValueError("bad lattice")
    return e[:q].copy(), w[:q].copy(), float(cs[0])


class Thermal:
    """The 1D thermal model: fourth-order EDF (order 4 by default) with local
    thetabar on D1V5/D1V7, velocity-shift force E, periodic box."""

    def __init__(self, kind: str = "D1V7", stat: str = "fd", theta: float = 1.0 / 270.0, mu: float = 1.0,
                 tau: float = 0.8, E: float = 0.0, order: int = 4):
        lib = _load()
        self._buf = ctypes.create_string_buffer(lib.or_thermal_size())
        rc = lib.or_thermal_init(self._buf, LATTICE1D[kind], STAT[stat], theta, mu, tau, E, order)
        if rc == -2:
            raise ValueError("unstable lattice (a weight or c_s is not positive)")
        if rc != 0:
            raise ValueError("bad thermal-model arguments")
        out = np.zeros(24 + 7)
        self.Q = lib.or_thermal_constants(self._buf, _dp(out))
        self.I = out[:5].copy()
        self.cs = float(out[5])
        self.g = float(out[6])
        self.co = out[7:24].copy()
        self.w = out[24: 24 + self.Q].copy()
        self.e = {5: np.array([0, 1, -1, 3, -3]), 7: np.array([0, 1, -1, 2, -2, 3, -3])}[self.Q]
        self.xi = self.e / self.cs
        self.tau, self.E, self.order = tau, E, order

    def equilibrium(self, rho: float, u: float, thetabar: float) -> np.ndarray:
        out = np.zeros(self.Q)
        _load().or_thermal_equilibrium(self._buf, float(rho), float(u), float(thetabar), _dp(out))
        return out

    def collide_cell(self, f, E=None) -> np.ndarray:
        out = np.zeros(self.Q)
        _load().or_thermal_collide_cell(self._buf, _dp(np.ascontiguousarray(f, dtype=np.float64)),
                                        float(self.E if E is None else E), _dp(out))
        return out

    def init_state(self, rho, u, thetabar) -> np.ndarray:
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        n = rho.size
        uu = np.ascontiguousarray(np.broadcast_to(u, (n,)), dtype=np.float64)
        th = np.ascontiguousarray(np.broadcast_to(thetabar, (n,)), dtype=np.float64)
        f = np.zeros(self.Q * n)
        _load().or_thermal_init_state(self._buf, n, _dp(rho), _dp(uu), _dp(th), _dp(f))
        return f

    def step(self, f: np.ndarray, nsteps: int, Efield=None) -> np.ndarray:
        n = f.size // self.Q
        E_a = None if Efield is None else np.ascontiguousarray(Efield, dtype=np.float64)
        tmp = np.empty_like(f)
        _load().or_thermal_step(self._buf, n, _dp(E_a), _dp(f), _dp(tmp), int(nsteps))
        return f

    def moments(self, f: np.ndarray):
        """(rho[n], j[n], energy[n], totals[3]); energy = sum_a f_a xi_a^2."""
        n = f.size // self.Q
        rho, j, en, tot = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(3)
        _load().or_thermal_moments(self._buf, n, _dp(np.ascontiguousarray(f)), _dp(rho), _dp(j), _dp(en), _dp(tot))
        return rho, j, en, tot


BE_STAT = {"fd": 0, "be": 1}


def fd_integral(nu: float, eta: float, stat: str = "fd") -> float:
    """g_nu(e^eta) of the FD (or BE) distribution (Sec. 4)."""
    return float(_load().or_fd_integral(float(nu), float(eta), BE_STAT[stat]))


def density_of_mu(D: int, theta: float, mu: float, stat: str = "fd") -> float:
    """rho = (pi theta)^{D/2} g_{D/2}(e^{mu/theta}) (Sec. 9.1, Eq. rho-def-eq)."""
    return float(_load().or_density_of_mu(int(D), BE_STAT[stat], float(theta), float(mu)))


def mu_of_density(D: int, theta: float, rho: float, stat: str = "fd") -> float:
    """The inverse of density_of_mu (Sec. 9.1.2), by bisection."""
    return float(_load().or_mu_of_density(int(D), BE_STAT[stat], float(theta), float(rho)))


def thetabar_of_mu(D: int, theta: float, mu: float, stat: str = "fd") -> float:
    """thetabar = I_2 / I_0 of the FD/BE/MB distribution at (theta, mu)
    (Sec. 9.1; the weight integrals of Sec. 3, Eq. i2n-cont2)."""
    I = weight_integrals(D, stat, theta, mu, nmax=1)
    return float(I[1] / I[0])


def _thetabar_2d_closed(stat: str, theta: float, mu_w: float, r: np.ndarray) -> np.ndarray:
    """D = 2 in closed form: I_0 = pi theta g_1(z), I_2 = (theta/2) pi theta
    g_2(z), so thetabar = theta g_2(z) / (2 g_1(z)) (Sec. 9.1) with
    g_1 = ln(1 + z), g_2 = -Li_2(-z) (FD) and g_1 = -ln(1 - z), g_2 = Li_2(z)
    (BE); the cell's g_1 is r times the weight's."""
    from scipy.special import spence  # spence(x) = Li_2(1 - x)

    eta_w = mu_w / theta
    if stat == "fd":
        g1w = np.log1p(np.exp(eta_w)) if eta_w < 30 else eta_w + np.log1p(np.exp(-eta_w))
        g1 = r * g1w
        z = np.expm1(g1)
        g2 = -spence(1.0 + z)
    else:
        g1w = -np.log1p(-np.exp(eta_w))
        g1 = r * g1w
        z = -np.expm1(-g1)
        g2 = spence(1.0 - z)
    return theta * g2 / (2.0 * g1)


def thetabar_of_density(D: int, stat: str, theta: float, mu_w: float, rho, rho_ref: float | None = None):
    """thetabar of cells of density rho: I_2/I_0 at the mu with
    I_0(mu) = rho I_0(mu_w) / rho_ref (rho_ref defaults to I_0(mu_w)).  MB:
    thetabar does not depend on mu; D = 2 FD/BE: closed form; otherwise mu by
    mu_of_density and thetabar by thetabar_of_mu, cell by cell (slow)."""
    rho = np.asarray(rho, dtype=np.float64)
    if stat == "mb":
        return np.full(rho.shape, thetabar_of_mu(D, theta, mu_w, stat))
    I0w = density_of_mu(D, theta, mu_w, stat)
    r = rho / (I0w if rho_ref is None else rho_ref)
    if D == 2:
        return _thetabar_2d_closed(stat, theta, mu_w, r)
    out = np.empty(rho.shape)
    for i, ri in np.ndenumerate(r):
        out[i] = thetabar_of_mu(D, theta, mu_of_density(D, theta, ri * I0w, stat), stat)
    return out


def thetabar_slope_of_density(D: int, stat: str, theta: float, mu_w: float, rho, rho_ref: float | None = None):
    """d thetabar / d rho of thetabar_of_density.  MB: 0.  D = 2 FD/BE in
    closed form: with g_1 = r g_1w, d g_2 / d g_1 = g_1 (1 + z) / z (FD) or
    g_1 (1 - z) / z (BE), since d g_nu / dz = g_{nu-1} / z; otherwise a
    central difference of thetabar_of_density with a relative step 1e-6."""
    rho = np.asarray(rho, dtype=np.float64)
    if stat == "mb":
        return np.zeros(rho.shape)
    I0w = density_of_mu(D, theta, mu_w, stat)
    ref = I0w if rho_ref is None else rho_ref
    if D == 2:
        from scipy.special import spence

        eta_w = mu_w / theta
        r = rho / ref
        if stat == "fd":
            g1w = np.log1p(np.exp(eta_w)) if eta_w < 30 else eta_w + np.log1p(np.exp(-eta_w))
            g1 = r * g1w
            z = np.expm1(g1)
            g2 = -spence(1.0 + z)
            dg2 = g1 * (1.0 + z) / z * g1w
        else:
            g1w = -np.log1p(-np.exp(eta_w))
            g1 = r * g1w
            z = -np.expm1(-g1)
            g2 = spence(1.0 - z)
            dg2 = g1 * (1.0 - z) / z * g1w
        return 0.5 * theta * (dg2 * g1 - g2 * g1w) / g1 ** 2 / ref
    h = 1e-6 * rho
    return (thetabar_of_density(D, stat, theta, mu_w, rho + h, rho_ref)
            - thetabar_of_density(D, stat, theta, mu_w, rho - h, rho_ref)) / (2 * h)
