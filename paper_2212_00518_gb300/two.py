"""IESH dynamics of a two-orbital adsorbate over six nuclear coordinates
(include/iesh.h, iesh2_*): ctypes marshalling only; every step runs in the
library's CUDA kernels (FP64 or the mixed-precision split)."""
import ctypes

import numpy as np

from . import iesh as _I


def model_struct(md):
    """iesh2_model from a model dictionary (iesh_inputs.two_orbital)."""
    m = _I._Model2()
    m.n_bath = int(md["M"])
    m.n_elec = int(md["Ne"])
    m.band_lo, m.band_hi = (float(v) for v in md["band"])
    m.mu = float(md.get("mu", 0.0))
    m.mass = float(md["mass"])
    m.omega = float(md["omega"])
    for i in range(6):
        m.x0[i] = float(md["x0"][i])
        m.R[i] = float(md["R"][i])
    for i in range(16):
        m.theta[i] = float(md["theta"][i])
    for a in range(2):
        m.vbar[a] = float(md["Vbar"][a])
    prof = md.get("profile")
    if prof is not None:  # own Lorentzian bath profile per orbital
        m.profile = 1
        for a in range(2):
            m.prof_center[a] = float(prof["center"][a])
            m.prof_width[a] = float(prof["width"][a])
    m.eigensolver = 1 if md.get("eigensolver") == "dense" else 0
    return m


class TwoOrbitalContext:
    """A batch of two-orbital trajectories on one GPU (wraps iesh2_ctx).
    N = M + 2 orbitals; x, p, F are [n][6]; C is [n][Ne][N], complex128
    (FP64) or complex64 (mixed precision)."""

    def __init__(self, model, max_traj, precision=_I.PREC_FP64, skip_bound=False, stream=None):
        self.L = _I.load()
        self.precision = int(precision)
        self.model = dict(model)
        self.N = int(model["M"]) + 2
        self.Ne = int(model["Ne"])
        self.max_traj = int(max_traj)
        self.n = 0
        self._m = model_struct(model)
        self.stream = _I.current_stream_handle() if stream is None else stream
        h = _I._vp()
        rc = self.L.iesh2_create(ctypes.byref(h), ctypes.byref(self._m), self.precision, self.max_traj,
                                 int(bool(skip_bound)), _I._vp(self.stream) if self.stream else None)
        self._h = h
        if rc != _I.IESH_OK:
            msg = self.L.iesh2_last_error(h).decode() if h.value else ""
            self.L.iesh2_destroy(h)
            self._h = None
            raise _I.IeshError(f"iesh2_create: {_I.STATUS_NAMES.get(rc, rc)}: {msg}")

    def close(self):
        if getattr(self, "_h", None):
            self.L.iesh2_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != _I.IESH_OK:
            raise _I.IeshError(f"{what}: {_I.STATUS_NAMES.get(rc, rc)}: "
                               f"{self.L.iesh2_last_error(self._h).decode()}")

    @property
    def cdtype(self):
        return np.complex128 if self.precision == _I.PREC_FP64 else np.complex64

    def set_state(self, x, p, occ, C):
        n = int(x.shape[0])
        self._check(self.L.iesh2_set_state(self._h, n, _I._ptr(x), _I._ptr(p), _I._ptr(occ),
                                           _I._ptr(C)), "iesh2_set_state")
        self.n = n

    def get_state(self, x=None, p=None, occ=None, C=None, status=None):
        n = self.n
        x = np.zeros((n, 6)) if x is None else x
        p = np.zeros((n, 6)) if p is None else p
        occ = np.zeros((n, self.Ne), np.int16) if occ is None else occ
        C = np.zeros((n, self.Ne, self.N), self.cdtype) if C is None else C
        status = np.zeros(n, np.uint32) if status is None else status
        self._check(self.L.iesh2_get_state(self._h, _I._ptr(x), _I._ptr(p), _I._ptr(occ), _I._ptr(C),
                                           _I._ptr(status)), "iesh2_get_state")
        return dict(x=x, p=p, occ=occ, C=C, status=status)

    def run(self, dt, n_steps, seed=0):
        self._check(self.L.iesh2_run(self._h, float(dt), int(n_steps), int(seed)), "iesh2_run")

    def eigen(self):
        """lam [n][N], Q [n][2][N] (adsorbate components), F [n][6]."""
        lam = np.zeros((self.n, self.N))
        Q = np.zeros((self.n, 2, self.N))
        F = np.zeros((self.n, 6))
        self._check(self.L.iesh2_get_eigen(self._h, lam.ctypes.data, Q.ctypes.data, F.ctypes.data),
                    "iesh2_get_eigen")
        return lam, Q, F

    def hop_probabilities(self, dt):
        g = np.zeros((self.n, self.Ne, self.N))
        self._check(self.L.iesh2_hop_probabilities(self._h, float(dt), g.ctypes.data),
                    "iesh2_hop_probabilities")
        return g

    def counters(self):
        ns = np.zeros(self.n, np.int64)
        hops = np.zeros(self.n, np.int32)
        fr = np.zeros(self.n, np.int32)
        self._check(self.L.iesh2_get_counters(self._h, ns.ctypes.data, hops.ctypes.data,
                                              fr.ctypes.data), "iesh2_get_counters")
        return ns, hops, fr

    def profile(self, enable=True):
        self._check(self.L.iesh2_profile(self._h, int(bool(enable))), "iesh2_profile")

    def profile_read(self):
        ms = np.zeros(len(_I.KERNEL_CLASSES))
        n = np.zeros(len(_I.KERNEL_CLASSES), np.int64)
        self._check(self.L.iesh2_profile_read(self._h, ms.ctypes.data, n.ctypes.data),
                    "iesh2_profile_read")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(_I.KERNEL_CLASSES)}
