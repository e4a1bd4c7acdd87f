"""Thin ctypes binding of libheat.so (C ABI declared in include/heat.h).

Argument marshalling only: every step of the ADI path runs in the library's
CUDA kernels.  PyTorch is used for device buffers and streams.  There is no
CPU fallback: if the library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libheat.so")

HEAT_OK = 0
STATUS = {0: "ok", -1: "HEAT_ERR_ARG", -2: "HEAT_ERR_CUDA", -3: "HEAT_ERR_NONFINITE",
          -4: "HEAT_ERR_TIMEOUT", -5: "HEAT_ERR_OOM", -6: "HEAT_ERR_TOO_LARGE", -7: "HEAT_ERR_NOCONV"}
PRECISION = {"fp64": 0, "fp32": 1, "fp32_refined": 2}
NUMPY_DTYPE = {"fp64": np.float64, "fp32": np.float32, "fp32_refined": np.float32}

# Every extern "C" symbol include/heat.h declares.
SYMBOLS = ["heat_create", "heat_set_dt", "heat_step", "heat_sweep", "heat_field", "heat_set_field", "heat_energy",
           "heat_info", "heat_launches_per_step", "heat_sync", "heat_destroy", "heat_strerror",
           "heat_energy_noalloc", "heat_batch_create", "heat_batch_member", "heat_batch_step", "heat_batch_sync",
           "heat_batch_tune", "heat_batch_set_tuning", "heat_batch_get_tuning", "heat_batch_launches_per_step",
           "heat_batch_destroy", "heat_batch_set_dt",
           "heat_nl_create", "heat_nl_step", "heat_nl_advance", "heat_nl_time", "heat_nl_set_time", "heat_nl_field",
           "heat_nl_half_field", "heat_nl_set_field", "heat_nl_info", "heat_nl_destroy", "heat_nl_layout",
           "heat_nl_field_packed", "heat_test_stall", "heat_set_rsweep", "heat_get_rsweep"]


class HeatError(RuntimeError):
    def __init__(self, fn, status):
        super().__init__(f"{fn} failed: {STATUS.get(status, status)}")
        self.status = status


class _Box(ctypes.Structure):
    _fields_ = [("r0", ctypes.c_double), ("r1", ctypes.c_double), ("z0", ctypes.c_double),
                ("z1", ctypes.c_double), ("region", ctypes.c_int)]


class _Geometry(ctypes.Structure):
    _fields_ = [("n_r_layers", ctypes.c_int), ("r_faces", ctypes.POINTER(ctypes.c_double)),
                ("r_cells", ctypes.POINTER(ctypes.c_int)),
                ("n_z_layers", ctypes.c_int), ("z_faces", ctypes.POINTER(ctypes.c_double)),
                ("z_cells", ctypes.POINTER(ctypes.c_int)),
                ("n_boxes", ctypes.c_int), ("boxes", ctypes.POINTER(_Box)),
                ("bc", ctypes.c_int * 4), ("T_bc", ctypes.c_double * 4)]


class _Materials(ctypes.Structure):
    _fields_ = [("n_regions", ctypes.c_int), ("k", ctypes.POINTER(ctypes.c_double)),
                ("C", ctypes.POINTER(ctypes.c_double)), ("q", ctypes.POINTER(ctypes.c_double)),
                ("T_init", ctypes.c_double)]


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("face_mean", ctypes.c_int)]


class _NlMaterials(ctypes.Structure):
    _fields_ = [("n_regions", ctypes.c_int), ("n_knots", ctypes.c_int)] + \
        [(n, ctypes.POINTER(ctypes.c_double)) for n in ("T_knots", "k", "C", "chi", "j2")] + \
        [("T_init", ctypes.c_double)]


class _Pulse(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int)] + [(n, ctypes.c_double) for n in ("t_per", "t_src", "t_trs", "xi", "zeta")]


class _NlOptions(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("s_max", ctypes.c_int), ("tau_base", ctypes.c_double),
                ("tau_trs", ctypes.c_double), ("tau_min", ctypes.c_double), ("face_mean", ctypes.c_int)]


class _NlStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("halvings", ctypes.c_longlong), ("iters1", ctypes.c_longlong),
                ("iters2", ctypes.c_longlong), ("tau_smallest", ctypes.c_double)]


_lib = None


def load():
    """Load libheat.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        L.heat_create.argtypes = [ctypes.POINTER(_Geometry), ctypes.POINTER(_Materials), ctypes.POINTER(_Options),
                                  ctypes.c_double, vp, ctypes.POINTER(vp)]
        L.heat_set_dt.argtypes = [vp, ctypes.c_double]
        L.heat_step.argtypes = [vp, ctypes.c_int]
        L.heat_sweep.argtypes = [vp, ctypes.c_int]
        L.heat_field.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int]
        L.heat_set_field.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int]
        L.heat_energy.argtypes = [vp, dp, dp, dp]
        L.heat_energy_noalloc.argtypes = [vp, dp, dp, dp]
        L.heat_info.argtypes = [vp, ip, ip, dp, dp, dp]
        L.heat_launches_per_step.argtypes = [vp]
        L.heat_sync.argtypes = [vp]
        L.heat_test_stall.argtypes = [vp, ctypes.c_int]
        L.heat_set_rsweep.argtypes = [vp, ctypes.c_int]
        L.heat_get_rsweep.argtypes = [vp]
        L.heat_destroy.argtypes = [vp]
        L.heat_destroy.restype = None
        L.heat_strerror.argtypes = [ctypes.c_int]
        L.heat_strerror.restype = ctypes.c_char_p
        L.heat_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(_Geometry), ctypes.POINTER(_Materials),
                                         ctypes.POINTER(_Options), dp, vp, ctypes.POINTER(vp)]
        L.heat_batch_member.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp)]
        L.heat_batch_set_dt.argtypes = [vp, dp]
        L.heat_batch_step.argtypes = [vp, ctypes.c_int]
        L.heat_batch_sync.argtypes = [vp]
        L.heat_batch_tune.argtypes = [vp, ctypes.c_int, dp]
        L.heat_batch_set_tuning.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.heat_batch_get_tuning.argtypes = [vp, ip, ip, ip]
        L.heat_batch_launches_per_step.argtypes = [vp]
        L.heat_batch_destroy.argtypes = [vp]
        L.heat_batch_destroy.restype = None
        L.heat_nl_create.argtypes = [ctypes.POINTER(_Geometry), ctypes.POINTER(_NlMaterials), ctypes.POINTER(_Pulse),
                                     ctypes.POINTER(_NlOptions), vp, ctypes.POINTER(vp)]
        L.heat_nl_step.argtypes = [vp, ctypes.c_double, ip, ip]
        L.heat_nl_advance.argtypes = [vp, ctypes.c_double, ctypes.c_longlong, ctypes.POINTER(_NlStats)]
        L.heat_nl_time.argtypes = [vp, dp]
        L.heat_nl_set_time.argtypes = [vp, ctypes.c_double]
        L.heat_nl_field.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int]
        L.heat_nl_half_field.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int]
        L.heat_nl_set_field.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int]
        L.heat_nl_info.argtypes = [vp, ip, ip, ctypes.POINTER(ctypes.c_longlong)]
        L.heat_nl_layout.argtypes = [vp, ip, ip, ctypes.POINTER(ctypes.c_longlong)]
        L.heat_nl_field_packed.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int]
        L.heat_nl_destroy.argtypes = [vp]
        L.heat_nl_destroy.restype = None
        _lib = L
    return _lib


def _check(fn, st):
    if st != HEAT_OK:
        raise HeatError(fn, st)


def _current_stream_handle():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _marshal(p, keep):
    """heat_geometry and heat_materials of a problem; arrays they point to go in ``keep``."""
    def arr(x, dt_):
        a = np.ascontiguousarray(x, dtype=dt_)
        keep.append(a)
        return a

    rf, rc = arr(p.r_faces, np.float64), arr(p.r_cells, np.int32)
    zf, zc = arr(p.z_faces, np.float64), arr(p.z_cells, np.int32)
    bx = np.asarray(p.boxes, dtype=np.float64).reshape(-1, 4)
    boxes = (_Box * len(bx))(*[_Box(*map(float, b), int(r)) for b, r in zip(bx, p.box_region)])
    keep.append(boxes)
    geo = _Geometry(len(rc), rf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                    rc.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                    len(zc), zf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                    zc.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(bx), boxes,
                    (ctypes.c_int * 4)(*[int(v) for v in p.bc]),
                    (ctypes.c_double * 4)(*[float(v) for v in p.T_bc]))
    k, C, q = arr(p.k, np.float64), arr(p.C, np.float64), arr(p.q, np.float64)
    mat = _Materials(len(k), k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     C.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     q.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(p.T_init))
    return geo, mat


class HeatSolver:
    """One ADI heat problem on the GPU (wraps heat_create / heat_step / ...).

    ``problem`` is any object with the attributes of ``workloads.heat.Problem``
    (r_faces, r_cells, z_faces, z_cells, boxes, box_region, bc, T_bc, k, C, q,
    T_init, face_mean).  ``stream``: a torch.cuda.Stream, or None for torch's
    current stream.
    """

    def __init__(self, problem, dt: float, precision: str = "fp64", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("HeatSolver needs a CUDA GPU; there is no CPU path")
        L = load()
        p = problem
        self._keep = []
        geo, mat = _marshal(p, self._keep)
        opt = _Options(PRECISION[precision], int(getattr(p, "face_mean", 0)))
        self.stream = stream
        sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else _current_stream_handle()
        h = ctypes.c_void_p()
        _check("heat_create", L.heat_create(ctypes.byref(geo), ctypes.byref(mat), ctypes.byref(opt),
                                            float(dt), sh, ctypes.byref(h)))
        self._h = h
        self.precision = precision
        nr, nz = ctypes.c_int(), ctypes.c_int()
        te = ctypes.c_double()
        _check("heat_info", L.heat_info(h, ctypes.byref(nr), ctypes.byref(nz), None, None, ctypes.byref(te)))
        self.Nr, self.Nz, self.tau_exp = nr.value, nz.value, te.value
        self.dt = float(dt)

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            load().heat_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API
    def set_dt(self, dt: float):
        _check("heat_set_dt", load().heat_set_dt(self._h, float(dt)))
        self.dt = float(dt)

    def step(self, n: int = 1):
        _check("heat_step", load().heat_step(self._h, int(n)))

    def sweep(self, direction: int):
        """One half-step: 0 = implicit in r (to the half layer), 1 = implicit in z."""
        _check("heat_sweep", load().heat_sweep(self._h, int(direction)))

    def sync(self):
        _check("heat_sync", load().heat_sync(self._h))

    def field(self, out=None):
        """Current temperature field.  ``out``: a CUDA float64 torch tensor of
        Nz*Nr elements (stream-ordered copy), else a new host numpy array."""
        n = self.Nr * self.Nz
        if out is not None:
            assert out.is_cuda and out.dtype.is_floating_point and out.element_size() == 8 and out.numel() == n
            _check("heat_field", load().heat_field(self._h, ctypes.c_void_p(out.data_ptr()), n, 1))
            return out
        a = np.empty((self.Nz, self.Nr), dtype=np.float64)
        _check("heat_field", load().heat_field(self._h, a.ctypes.data_as(ctypes.c_void_p), n, 0))
        return a

    def set_field(self, T):
        n = self.Nr * self.Nz
        if hasattr(T, "is_cuda") and T.is_cuda:
            assert T.element_size() == 8 and T.numel() == n and T.is_contiguous()
            _check("heat_set_field", load().heat_set_field(self._h, ctypes.c_void_p(T.data_ptr()), n, 1))
            return
        a = np.ascontiguousarray(T, dtype=np.float64).reshape(self.Nz, self.Nr)
        _check("heat_set_field", load().heat_set_field(self._h, a.ctypes.data_as(ctypes.c_void_p), n, 0))

    def energy(self):
        """(E, Phi, Q) in FP64 (see include/heat.h)."""
        e, f, q = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check("heat_energy", load().heat_energy(self._h, ctypes.byref(e), ctypes.byref(f), ctypes.byref(q)))
        return e.value, f.value, q.value

    def energy_noalloc(self):
        """(E, Phi, Q) like energy(), computed with no device allocation and
        none of the context's scratch (include/heat.h)."""
        e, f, q = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check("heat_energy_noalloc",
               load().heat_energy_noalloc(self._h, ctypes.byref(e), ctypes.byref(f), ctypes.byref(q)))
        return e.value, f.value, q.value

    def centres(self):
        rc = np.empty(self.Nr)
        zc = np.empty(self.Nz)
        _check("heat_info", load().heat_info(self._h, None, None, rc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             zc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None))
        return rc, zc

    def set_rsweep(self, kind: int):
        """Choose the r-sweep kernel (include/heat.h, heat_set_rsweep)."""
        _check("heat_set_rsweep", load().heat_set_rsweep(self._h, int(kind)))

    def rsweep(self) -> int:
        return int(load().heat_get_rsweep(self._h))

    def launches_per_step(self) -> int:
        return int(load().heat_launches_per_step(self._h))


class _MemberView(HeatSolver):
    """HeatSolver view of a batch member: the batch owns the context."""

    def close(self):
        pass


class HeatBatch:
    """A batched ensemble of independent ADI problems of one precision
    (wraps heat_batch_*).  ``problems``: list of problem objects (each with
    Nr <= 1024); ``dts``: one dt per member.  ``members[i]`` is a HeatSolver
    view of member i for field / set_field / energy / centres; stepping is
    done for all members at once by ``step``."""

    def __init__(self, problems, dts, precision: str = "fp32", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("HeatBatch needs a CUDA GPU; there is no CPU path")
        L = load()
        n = len(problems)
        self._keep = []
        geos = (_Geometry * n)()
        mats = (_Materials * n)()
        for i, p in enumerate(problems):
            geos[i], mats[i] = _marshal(p, self._keep)
        fm = {int(getattr(p, "face_mean", 0)) for p in problems}
        if len(fm) != 1:
            raise ValueError("batch members must share the face mean")
        opt = _Options(PRECISION[precision], fm.pop())
        d = np.ascontiguousarray(dts, dtype=np.float64)
        assert d.shape == (n,)
        sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else _current_stream_handle()
        h = ctypes.c_void_p()
        _check("heat_batch_create", L.heat_batch_create(n, geos, mats, ctypes.byref(opt),
                                                        d.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), sh,
                                                        ctypes.byref(h)))
        self._h = h
        self.n = n
        self.precision = precision
        self.members = []
        for i in range(n):
            c = ctypes.c_void_p()
            _check("heat_batch_member", L.heat_batch_member(h, i, ctypes.byref(c)))
            m = _MemberView.__new__(_MemberView)
            m._h, m._owner, m._keep, m.precision, m.stream = c, self, [], precision, stream
            nr, nz, te = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
            _check("heat_info", L.heat_info(c, ctypes.byref(nr), ctypes.byref(nz), None, None, ctypes.byref(te)))
            m.Nr, m.Nz, m.tau_exp, m.dt = nr.value, nz.value, te.value, float(d[i])
            self.members.append(m)
        self.cells = sum(m.Nr * m.Nz for m in self.members)

    def close(self):
        if getattr(self, "_h", None):
            for m in self.members:
                m._h = None  # member handles die with the batch
            load().heat_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_dt(self, dts):
        d = np.ascontiguousarray(dts, dtype=np.float64)
        assert d.shape == (self.n,)
        _check("heat_batch_set_dt", load().heat_batch_set_dt(self._h, d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        for m, x in zip(self.members, d):
            m.dt = float(x)

    def step(self, n: int = 1):
        _check("heat_batch_step", load().heat_batch_step(self._h, int(n)))

    def sync(self):
        _check("heat_batch_sync", load().heat_batch_sync(self._h))

    def tune(self, trial_steps: int = 5) -> float:
        """Autotune the schedule (fields are left unchanged); returns ms/step of the winner."""
        ms = ctypes.c_double()
        _check("heat_batch_tune", load().heat_batch_tune(self._h, int(trial_steps), ctypes.byref(ms)))
        return ms.value

    def set_tuning(self, rK: int = 0, band: int = 0, zwpb: int = 0):
        _check("heat_batch_set_tuning", load().heat_batch_set_tuning(self._h, int(rK), int(band), int(zwpb)))

    def tuning(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check("heat_batch_get_tuning", load().heat_batch_get_tuning(self._h, ctypes.byref(a), ctypes.byref(b),
                                                                     ctypes.byref(c)))
        return a.value, b.value, c.value

    def launches_per_step(self) -> int:
        return int(load().heat_batch_launches_per_step(self._h))


def _marshal_nl(p, m, eps, s_max, tau_base, tau_trs, tau_min, keep):
    """heat_geometry, heat_nl_materials, heat_pulse and heat_nl_options of a
    problem and its ``workloads.heat.NlMaterials``."""
    geo, _ = _marshal(p, keep)
    Tk, k, C, chi = (np.ascontiguousarray(x, dtype=np.float64) for x in (m.T_knots, m.k, m.C, m.chi))
    j2 = np.ascontiguousarray(m.j2, dtype=np.float64)
    keep.extend([Tk, k, C, chi, j2])
    R, K = Tk.shape
    dp = ctypes.POINTER(ctypes.c_double)
    mat = _NlMaterials(R, K, Tk.ctypes.data_as(dp), k.ctypes.data_as(dp), C.ctypes.data_as(dp),
                       chi.ctypes.data_as(dp), j2.ctypes.data_as(dp), float(p.T_init))
    pulse = _Pulse(int(m.model), float(m.t_per), float(m.t_src), float(m.t_trs), float(m.xi), float(m.zeta))
    opt = _NlOptions(float(eps), int(s_max), float(tau_base), float(tau_trs), float(tau_min),
                     int(getattr(p, "face_mean", 0)))
    return geo, mat, pulse, opt


class HeatNl:
    """The paper's full method on the GPU (wraps heat_nl_*): temperature-
    dependent materials, the simple iteration, adaptive tau, the pulsed
    source; FP64.  ``materials``: a ``workloads.heat.NlMaterials``."""

    def __init__(self, problem, materials, eps=1e-9, s_max=20, tau_base=1.0, tau_trs=1.0, tau_min=1e-12,
                 stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("HeatNl needs a CUDA GPU; there is no CPU path")
        L = load()
        self._keep = []
        geo, mat, pulse, opt = _marshal_nl(problem, materials, eps, s_max, tau_base, tau_trs, tau_min, self._keep)
        sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else _current_stream_handle()
        h = ctypes.c_void_p()
        _check("heat_nl_create", L.heat_nl_create(ctypes.byref(geo), ctypes.byref(mat), ctypes.byref(pulse),
                                                  ctypes.byref(opt), sh, ctypes.byref(h)))
        self._h = h
        nr, nz = ctypes.c_int(), ctypes.c_int()
        _check("heat_nl_info", L.heat_nl_info(h, ctypes.byref(nr), ctypes.byref(nz), None))
        self.Nr, self.Nz = nr.value, nz.value

    def close(self):
        if getattr(self, "_h", None):
            load().heat_nl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, tau: float):
        """One step of length tau (no halving); returns the iterations of the
        two half-steps.  Raises HeatError (HEAT_ERR_NOCONV) if s_max is not enough."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _check("heat_nl_step", load().heat_nl_step(self._h, float(tau), ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def advance(self, t_end: float, max_steps: int = 2 ** 62):
        """The evolution loop of Sec. 4 up to t_end; returns its statistics."""
        st = _NlStats()
        _check("heat_nl_advance", load().heat_nl_advance(self._h, float(t_end), int(max_steps), ctypes.byref(st)))
        return {"steps": st.steps, "halvings": st.halvings, "iters1": st.iters1, "iters2": st.iters2,
                "tau_smallest": st.tau_smallest}

    @property
    def time(self) -> float:
        t = ctypes.c_double()
        _check("heat_nl_time", load().heat_nl_time(self._h, ctypes.byref(t)))
        return t.value

    def set_time(self, t: float):
        _check("heat_nl_set_time", load().heat_nl_set_time(self._h, float(t)))

    def _get(self, fn):
        out = np.empty((self.Nz, self.Nr))
        _check(fn, getattr(load(), fn)(self._h, out.ctypes.data_as(ctypes.c_void_p), self.Nr * self.Nz, 0))
        return out

    def field(self):
        return self._get("heat_nl_field")

    def half_field(self):
        return self._get("heat_nl_half_field")

    def set_field(self, T):
        a = np.ascontiguousarray(T, dtype=np.float64).reshape(self.Nz, self.Nr)
        _check("heat_nl_set_field", load().heat_nl_set_field(self._h, a.ctypes.data_as(ctypes.c_void_p),
                                                             self.Nr * self.Nz, 0))

    def launches(self) -> int:
        n = ctypes.c_longlong()
        _check("heat_nl_info", load().heat_nl_info(self._h, None, None, ctypes.byref(n)))
        return n.value

    def layout(self):
        """(N_j per row, M_i per column, stored cells) of the packed layout."""
        Nj = np.zeros(self.Nz, dtype=np.int32)
        Mi = np.zeros(self.Nr, dtype=np.int32)
        n = ctypes.c_longlong()
        _check("heat_nl_layout", load().heat_nl_layout(self._h, Nj.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                                       Mi.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                                       ctypes.byref(n)))
        return Nj, Mi, n.value

    def field_packed(self):
        """The field in the row-packed layout (row j: its N_j cells)."""
        _, _, n = self.layout()
        out = np.empty(n)
        _check("heat_nl_field_packed", load().heat_nl_field_packed(self._h, out.ctypes.data_as(ctypes.c_void_p), n, 0))
        return out
