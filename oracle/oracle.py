"""ctypes wrapper of the plain FP64 CPU oracle (``heat_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The CUDA library never imports,
links or calls it.

The oracle computes one Peaceman-Rachford ADI step of the paper's scheme
(Sec. 3, eqs. "scheme_eq_1", "scheme_eq_2", "Lambda_r", "Lambda_z") on the
shifted grid of eq. "grid", with textbook Thomas line solves, in FP64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "heat_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libheat_oracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP over lines)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        # HEAT_ORACLE_LIB: a variant build of this oracle (the mutation test
        # compiles copies with planted mistakes and runs the pins against them).
        override = os.environ.get("HEAT_ORACLE_LIB")
        _lib = ctypes.CDLL(override if override else build())
        L = _lib
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.c_int, _D, _I, ctypes.c_int, _D, _I, ctypes.c_int, _D, _I,
                                 _I, _D, ctypes.c_int, _D, _D, _D, ctypes.c_int, ctypes.c_double]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_dims.argtypes = [ctypes.c_void_p, _I, _I]
        L.orc_grid.argtypes = [ctypes.c_void_p, _D, _D, _D, _D, _I]
        L.orc_coeffs.argtypes = [ctypes.c_void_p, _D]
        L.orc_tau_exp.restype = ctypes.c_double
        L.orc_tau_exp.argtypes = [ctypes.c_void_p]
        L.orc_get_field.argtypes = [ctypes.c_void_p, _D]
        L.orc_set_field.argtypes = [ctypes.c_void_p, _D]
        L.orc_get_half.argtypes = [ctypes.c_void_p, _D]
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int]
        L.orc_step_src.argtypes = [ctypes.c_void_p, ctypes.c_double, _D]
        L.orc_energy.argtypes = [ctypes.c_void_p, _D, _D, _D]
        L.orc_thomas.argtypes = [ctypes.c_int, _D, _D, _D, _D, _D, _D, _D]
        L.orc_pulse.restype = ctypes.c_double
        L.orc_pulse.argtypes = [ctypes.c_int] + [ctypes.c_double] * 6
        L.orc_nl_setup.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int]
        L.orc_nl_step.restype = ctypes.c_int
        L.orc_nl_step.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  _D, _I, _I]
        L.orc_nl_advance.restype = ctypes.c_int
        L.orc_nl_advance.argtypes = [ctypes.c_void_p, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int, _D]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_max_threads.restype = ctypes.c_int
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I)


def thomas(a, b, c, d):
    """Textbook Thomas solve of a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i."""
    a, b, c, d = (np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, c, d))
    n = len(b)
    x = np.empty(n)
    cw = np.empty(n)
    dw = np.empty(n)
    lib().orc_thomas(n, _dp(a), _dp(b), _dp(c), _dp(d), _dp(x), _dp(cw), _dp(dw))
    return x


def pulse(model: int, t: float, t_per: float, t_src: float, t_trs: float, xi: float = 4.0,
          zeta: float = 2.0) -> float:
    """p(t) of the paper's Sec. 2: 0 constant 1, 1 the rectangular pulse
    train (eq. "unit_model"), 2 its erf-smoothed version (eq. "trans_model")."""
    return float(lib().orc_pulse(int(model), float(t), float(t_per), float(t_src), float(t_trs), float(xi),
                                 float(zeta)))


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


class Oracle:
    """One oracle instance of a ``workloads.heat.Problem``."""

    def __init__(self, p):
        L = lib()
        self._keep = []

        def arr(x, dt):
            a = np.ascontiguousarray(x, dtype=dt)
            self._keep.append(a)
            return a

        rf, rcl = arr(p.r_faces, np.float64), arr(p.r_cells, np.int32)
        zf, zcl = arr(p.z_faces, np.float64), arr(p.z_cells, np.int32)
        bx, br = arr(np.asarray(p.boxes).reshape(-1, 4), np.float64), arr(p.box_region, np.int32)
        bc, tbc = arr(p.bc, np.int32), arr(p.T_bc, np.float64)
        k, C, q = arr(p.k, np.float64), arr(p.C, np.float64), arr(p.q, np.float64)
        self._h = L.orc_create(len(rcl), _dp(rf), _ip(rcl), len(zcl), _dp(zf), _ip(zcl),
                               len(br), _dp(bx), _ip(br), _ip(bc), _dp(tbc),
                               len(k), _dp(k), _dp(C), _dp(q), int(p.face_mean), float(p.T_init))
        nr, nz = ctypes.c_int(), ctypes.c_int()
        L.orc_dims(self._h, ctypes.byref(nr), ctypes.byref(nz))
        self.Nr, self.Nz = nr.value, nz.value
        self.problem = p

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def grid(self):
        rc, zc = np.empty(self.Nr), np.empty(self.Nz)
        hb, eb = np.empty(self.Nr), np.empty(self.Nz)
        reg = np.empty((self.Nz, self.Nr), dtype=np.int32)
        lib().orc_grid(self._h, _dp(rc), _dp(zc), _dp(hb), _dp(eb), _ip(reg))
        return dict(rc=rc, zc=zc, hbar=hb, etabar=eb, region=reg)

    def coeffs(self):
        out = np.empty((10, self.Nz, self.Nr))
        lib().orc_coeffs(self._h, _dp(out))
        names = ["Arm", "Arp", "Azm", "Azp", "Drl", "Drh", "Dzl", "Dzh", "C", "q"]
        return {n: out[a] for a, n in enumerate(names)}

    def tau_exp(self) -> float:
        return float(lib().orc_tau_exp(self._h))

    def field(self) -> np.ndarray:
        out = np.empty((self.Nz, self.Nr))
        lib().orc_get_field(self._h, _dp(out))
        return out

    def half_field(self) -> np.ndarray:
        out = np.empty((self.Nz, self.Nr))
        lib().orc_get_half(self._h, _dp(out))
        return out

    def set_field(self, T) -> None:
        a = np.ascontiguousarray(T, dtype=np.float64).reshape(self.Nz, self.Nr)
        lib().orc_set_field(self._h, _dp(a))

    def step(self, tau: float, n: int = 1) -> None:
        lib().orc_step(self._h, float(tau), int(n))

    def step_src(self, tau: float, X) -> None:
        a = np.ascontiguousarray(X, dtype=np.float64).reshape(self.Nz, self.Nr)
        lib().orc_step_src(self._h, float(tau), _dp(a))

    def energy(self):
        """(E, Phi, Q): energy, Dirichlet boundary heat flow and source power."""
        e, f, q = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        lib().orc_energy(self._h, ctypes.byref(e), ctypes.byref(f), ctypes.byref(q))
        return e.value, f.value, q.value

    # ---- temperature-dependent materials, simple iteration, adaptive tau
    def nl_setup(self, m):
        """Attach temperature-dependent material tables and the source model
        (a ``workloads.heat.NlMaterials``); the grid, regions and boundary
        conditions stay those of the problem."""
        keep = [np.ascontiguousarray(x, dtype=np.float64) for x in (m.T_knots, m.k, m.C, m.chi, m.j2)]
        self._keep.extend(keep)
        Tk, k, C, chi, j2 = keep
        R, K = Tk.shape
        lib().orc_nl_setup(self._h, R, K, _dp(Tk), _dp(k), _dp(C), _dp(chi), _dp(j2), int(m.model),
                           float(m.t_per), float(m.t_src), float(m.t_trs), float(m.xi), float(m.zeta),
                           int(self.problem.face_mean))

    def nl_step(self, t: float, tau: float, eps: float, s_max: int, X=None):
        """One step of eqs. "iter_scheme_eq_1/2" from time t (no halving).
        Returns (ok, iterations of half-step 1, of half-step 2)."""
        it1, it2 = ctypes.c_int(), ctypes.c_int()
        xp = None
        if X is not None:
            xa = np.ascontiguousarray(X, dtype=np.float64).reshape(self.Nz, self.Nr)
            self._keep.append(xa)
            xp = _dp(xa)
        ok = lib().orc_nl_step(self._h, float(t), float(tau), float(eps), int(s_max), xp, ctypes.byref(it1),
                               ctypes.byref(it2))
        return bool(ok), it1.value, it2.value

    def nl_advance(self, t: float, t_end: float, tau_base: float, tau_trs: float, eps: float, s_max: int,
                   tau_min: float, max_steps: int = 10 ** 9):
        """The evolution loop of Sec. 4 from t to t_end.  Returns (status, t,
        stats) with stats = (steps, halvings, iterations 1, iterations 2,
        smallest tau)."""
        tt = ctypes.c_double(t)
        st = np.zeros(5)
        rc = lib().orc_nl_advance(self._h, ctypes.byref(tt), float(t_end), float(tau_base), float(tau_trs),
                                  float(eps), int(s_max), float(tau_min), int(max_steps), _dp(st))
        return int(rc), tt.value, st
