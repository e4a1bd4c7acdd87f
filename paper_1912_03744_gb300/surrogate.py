"""ctypes binding of the surrogate C ABI (include/surrogate.h): argument
marshalling only; every step runs in libheat.so's kernels."""
from __future__ import annotations

import ctypes

import numpy as np

from .heat import HEAT_OK, HeatError, _Options, _current_stream_handle, _marshal, load

SURR_SYMBOLS = ["surr_create", "surr_n_params", "surr_set_params", "surr_get_params", "surr_forward",
                "surr_loss_grad", "surr_adam", "surr_infer_checked", "surr_solve", "surr_train", "surr_errors",
                "surr_destroy"]


class _Dims(ctypes.Structure):
    _fields_ = [("Nz", ctypes.c_int), ("Nr", ctypes.c_int), ("C", ctypes.c_int), ("mz", ctypes.c_int),
                ("mr", ctypes.c_int), ("L", ctypes.c_int)]


_bound = False


def _lib():
    global _bound
    L = load()
    if not _bound:
        vp, dp, fp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)
        from .heat import _Geometry, _Materials
        L.surr_create.argtypes = [ctypes.POINTER(_Dims), ctypes.POINTER(_Geometry), ctypes.POINTER(_Materials),
                                  ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)]
        L.surr_n_params.argtypes = [vp]
        L.surr_n_params.restype = ctypes.c_size_t
        L.surr_set_params.argtypes = [vp, fp, ctypes.c_size_t, ctypes.c_int]
        L.surr_get_params.argtypes = [vp, fp, ctypes.c_size_t, ctypes.c_int]
        L.surr_forward.argtypes = [vp, dp, ctypes.c_int, fp, ctypes.c_int]
        L.surr_loss_grad.argtypes = [vp, dp, ctypes.c_int, fp, ctypes.c_int, dp, fp, ctypes.c_int]
        L.surr_adam.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.surr_infer_checked.argtypes = [vp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint, fp,
                                         ctypes.c_int, ip, dp]
        L.surr_solve.argtypes = [vp, dp, ctypes.c_int, fp, ctypes.c_int]
        L.surr_train.argtypes = [vp, dp, ctypes.c_int, fp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_uint, dp]
        L.surr_errors.argtypes = [vp, dp, ctypes.c_int, fp, ctypes.c_int, dp]
        L.surr_destroy.argtypes = [vp]
        L.surr_destroy.restype = None
        _bound = True
    return L


def _check(fn, st):
    if st != HEAT_OK:
        raise HeatError(fn, st)


def _ptr(x):
    """(pointer, on_device) of a numpy array or a CUDA torch tensor."""
    if hasattr(x, "is_cuda") and x.is_cuda:
        assert x.is_contiguous()
        return ctypes.c_void_p(x.data_ptr()), 1
    assert x.flags["C_CONTIGUOUS"]
    return x.ctypes.data_as(ctypes.c_void_p), 0


class Surrogate:
    """FNO surrogate of the ADI solver on one fixed cell (see include/surrogate.h).

    ``problem``: a problem object giving the geometry, heat capacities and
    T_init (its k and q are replaced per instance); ``dims``: a
    ``workloads.fno.FnoDims``-like object; ``heater``: region index of q."""

    def __init__(self, problem, dims, heater: int, dt: float, steps: int, max_batch: int = 64, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Surrogate needs a CUDA GPU; there is no CPU path")
        L = _lib()
        self._keep = []
        geo, mat = _marshal(problem, self._keep)
        d = _Dims(dims.Nz, dims.Nr, dims.C, dims.mz, dims.mr, dims.L)
        sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else _current_stream_handle()
        h = ctypes.c_void_p()
        _check("surr_create", L.surr_create(ctypes.byref(d), ctypes.byref(geo), ctypes.byref(mat), int(heater),
                                            float(dt), int(steps), int(max_batch), sh, ctypes.byref(h)))
        self._h = h
        self.dims = dims
        self.Nz, self.Nr = dims.Nz, dims.Nr
        self.max_batch = max_batch
        self.n_params = int(L.surr_n_params(h))

    def close(self):
        if getattr(self, "_h", None):
            _lib().surr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _params(params):
        p = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 7)
        return p, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def set_params(self, flat):
        if not (hasattr(flat, "is_cuda") and flat.is_cuda):
            flat = np.ascontiguousarray(flat, dtype=np.float32)
        ptr, dev = _ptr(flat)
        _check("surr_set_params", _lib().surr_set_params(self._h, ptr, self.n_params, dev))

    def get_params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        _check("surr_get_params", _lib().surr_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p),
                                                         self.n_params, 0))
        return out

    def _out(self, B, out):
        if out is None:
            out = np.empty((B, self.Nz, self.Nr), dtype=np.float32)
        return out

    def forward(self, params, out=None):
        p, pp = self._params(params)
        out = self._out(len(p), out)
        ptr, dev = _ptr(out)
        _check("surr_forward", _lib().surr_forward(self._h, pp, len(p), ptr, dev))
        return out

    def loss_grad(self, params, T_true, want_grad=True):
        p, pp = self._params(params)
        if not (hasattr(T_true, "is_cuda") and T_true.is_cuda):
            T_true = np.ascontiguousarray(T_true, dtype=np.float32)
        tp, tdev = _ptr(T_true)
        loss = ctypes.c_double()
        g = np.empty(self.n_params, dtype=np.float32) if want_grad else None
        gp = g.ctypes.data_as(ctypes.c_void_p) if want_grad else None
        _check("surr_loss_grad", _lib().surr_loss_grad(self._h, pp, len(p), tp, tdev, ctypes.byref(loss), gp, 0))
        return loss.value, g

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        _check("surr_adam", _lib().surr_adam(self._h, float(lr), float(beta1), float(beta2), float(eps)))

    def infer_checked(self, params, n_check=8, tol=0.01, seed=0, out=None):
        p, pp = self._params(params)
        out = self._out(len(p), out)
        ptr, dev = _ptr(out)
        fb, err = ctypes.c_int(), ctypes.c_double()
        _check("surr_infer_checked", _lib().surr_infer_checked(self._h, pp, len(p), int(n_check), float(tol),
                                                               int(seed), ptr, dev, ctypes.byref(fb),
                                                               ctypes.byref(err)))
        return out, bool(fb.value), err.value

    def train(self, params, fields, epochs, batch, lr, lr_min_frac=0.02, seed=0):
        """surr_train: fields is a CUDA float32 tensor [n, Nz, Nr]; returns the last epoch's mean loss."""
        p, pp = self._params(params)
        assert hasattr(fields, "is_cuda") and fields.is_cuda and fields.dtype.is_floating_point
        ptr, _ = _ptr(fields)
        loss = ctypes.c_double()
        _check("surr_train", _lib().surr_train(self._h, pp, len(p), ptr, int(epochs), int(batch), float(lr),
                                               float(lr_min_frac), int(seed), ctypes.byref(loss)))
        return loss.value

    def errors(self, params, fields):
        """surr_errors: per-sample rise-relative max error of the network against fields."""
        p, pp = self._params(params)
        if not (hasattr(fields, "is_cuda") and fields.is_cuda):
            fields = np.ascontiguousarray(fields, dtype=np.float32)
        ptr, dev = _ptr(fields)
        out = np.empty(len(p), dtype=np.float64)
        _check("surr_errors", _lib().surr_errors(self._h, pp, len(p), ptr, dev,
                                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def solve(self, params, out=None):
        p, pp = self._params(params)
        out = self._out(len(p), out)
        ptr, dev = _ptr(out)
        _check("surr_solve", _lib().surr_solve(self._h, pp, len(p), ptr, dev))
        return out
