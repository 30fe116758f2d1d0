"""Differentiable occupied-orbital energy E_occ(x, theta) of a two-orbital
adsorbate on a metal band (include/iesh.h, iesh_eocc_*), as a
torch.autograd.Function whose forward and backward run in the library's
CUDA kernels.  float64 tensors use the FP64 kernels, float32 the FP32 ones.
"""
import ctypes

import torch

from . import iesh as _I


class EOccModel:
    """Device-side bath and constants of the model (wraps iesh_eocc_ctx).

    workload: dict with M, Ne, band, Vbar[2], R[6] (see iesh_inputs.eocc_workload)."""

    def __init__(self, workload, stream=None):
        self.L = _I.load()
        m = _I._EoccModel()
        m.n_bath = int(workload["M"])
        m.n_elec = int(workload["Ne"])
        m.band_lo, m.band_hi = (float(v) for v in workload["band"])
        m.mu = float(workload.get("mu", 0.0))
        for a in range(2):
            m.vbar[a] = float(workload["Vbar"][a])
        for q in range(6):
            m.R[q] = float(workload["R"][q])
        self._m = m
        self.stream = _I.current_stream_handle() if stream is None else stream
        h = _I._vp()
        rc = self.L.iesh_eocc_create(ctypes.byref(h), ctypes.byref(m),
                                     _I._vp(self.stream) if self.stream else None)
        self._h = h
        if rc != _I.IESH_OK:
            msg = self.L.iesh_eocc_last_error(h).decode() if h.value else ""
            self.L.iesh_eocc_destroy(h)
            self._h = None
            raise _I.IeshError(f"iesh_eocc_create: {_I.STATUS_NAMES.get(rc, rc)}: {msg}")

    def close(self):
        if getattr(self, "_h", None):
            self.L.iesh_eocc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != _I.IESH_OK:
            raise _I.IeshError(f"{what}: {_I.STATUS_NAMES.get(rc, rc)}: "
                               f"{self.L.iesh_eocc_last_error(self._h).decode()}")

    @staticmethod
    def _prec(t):
        if t.dtype == torch.float64:
            return _I.PREC_FP64
        if t.dtype == torch.float32:
            return _I.PREC_MIXED
        raise TypeError("x and theta must be float64 or float32 CUDA tensors")

    def forward(self, x, theta):
        assert x.is_cuda and theta.is_cuda and x.dtype == theta.dtype
        x = x.contiguous()
        theta = theta.contiguous()
        B = x.shape[0]
        E = torch.empty(B, dtype=x.dtype, device=x.device)
        saved = torch.empty(B, 4, dtype=x.dtype, device=x.device)
        status = torch.empty(B, dtype=torch.int32, device=x.device)
        self._check(self.L.iesh_eocc_forward(self._h, B, self._prec(x), x.data_ptr(),
                                             theta.data_ptr(), E.data_ptr(), saved.data_ptr(),
                                             status.data_ptr()), "iesh_eocc_forward")
        return E, saved, status

    def backward(self, x, theta, saved, gE):
        x = x.contiguous()
        theta = theta.contiguous()
        gE = gE.contiguous().to(x.dtype)
        B = x.shape[0]
        dx = torch.empty_like(x)
        per = torch.empty(B, 16, dtype=x.dtype, device=x.device)
        dth = torch.empty(16, dtype=x.dtype, device=x.device)
        self._check(self.L.iesh_eocc_backward(self._h, B, self._prec(x), x.data_ptr(),
                                              theta.data_ptr(), saved.data_ptr(), gE.data_ptr(),
                                              dx.data_ptr(), per.data_ptr(), dth.data_ptr()),
                    "iesh_eocc_backward")
        return dx, dth


class EOcc(torch.autograd.Function):
    """E = EOcc.apply(x[B,6], theta[16], model): occupied-orbital energy per
    geometry; gradients with respect to x and theta by Hellmann-Feynman."""

    @staticmethod
    def forward(ctx, x, theta, model):
        E, saved, status = model.forward(x, theta)
        ctx.model = model
        ctx.save_for_backward(x, theta, saved)
        ctx.mark_non_differentiable(status)
        return E, status

    @staticmethod
    def backward(ctx, gE, gstatus):
        x, theta, saved = ctx.saved_tensors
        dx, dth = ctx.model.backward(x, theta, saved, gE)
        return dx, dth, None


def eocc(x, theta, model):
    """Occupied-orbital energy E[B] (differentiable in x and theta)."""
    E, _ = EOcc.apply(x, theta, model)
    return E
