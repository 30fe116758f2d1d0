"""ctypes binding of libiesh.so (the C-ABI declared in include/iesh.h).

Argument marshalling only: every step of the IESH path runs in the CUDA
kernels of the library.  There is no fallback; if the shared library is
missing or fails to load, ImportError/OSError propagate.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); they are
passed to the library by pointer, which copies with cudaMemcpyDefault.
"""
import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libiesh.so")

IESH_OK = 0
STATUS_NAMES = {0: "IESH_OK", 1: "IESH_EINVAL", 2: "IESH_ECUDA", 3: "IESH_ENOMEM",
                4: "IESH_ESTATE", 5: "IESH_EUNSUPPORTED", 6: "IESH_ENONCONV",
                7: "IESH_ESINGULAR", 8: "IESH_ENORM", 9: "IESH_ENAN"}
TRAJ_SECULAR_NONCONV = 0x1
TRAJ_SINGULAR = 0x2
TRAJ_NAN = 0x4
TRAJ_DONE = 0x8
TRAJ_PROP_RANGE = 0x10
TRAJ_TC_WAIT = 0x20
TRAJ_NORM_DRIFT = 0x40

PREC_FP64 = 0
PREC_MIXED = 1
PROP_AVERAGED = 0  # exponential of the step-averaged adiabatic generator
PROP_OVERLAP = 1   # diabatic-basis variant (overlap of the two ends' orbitals)
IESH_NOALLOC_SCRATCH_BYTES = 32 << 20
_KIND = {"harmonic": 0, "erpenbeck": 1, "morse_image": 2}
_DISC = {"gl": 0, "trapezoid": 1}


class IeshError(RuntimeError):
    pass


class _Model(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("mass", ctypes.c_double),
                ("par", ctypes.c_double * 16), ("gamma", ctypes.c_double),
                ("band_lo", ctypes.c_double), ("band_hi", ctypes.c_double),
                ("mu", ctypes.c_double), ("n_bath", ctypes.c_int), ("n_elec", ctypes.c_int),
                ("disc", ctypes.c_int), ("n_lo", ctypes.c_int), ("n_leads", ctypes.c_int),
                ("lead_mu", ctypes.c_double * 2), ("lead_n", ctypes.c_int * 2),
                ("lead_nlo", ctypes.c_int * 2), ("lead_frac", ctypes.c_double * 2)]


class _EoccModel(ctypes.Structure):
    _fields_ = [("n_bath", ctypes.c_int), ("n_elec", ctypes.c_int), ("band_lo", ctypes.c_double),
                ("band_hi", ctypes.c_double), ("mu", ctypes.c_double),
                ("vbar", ctypes.c_double * 2), ("R", ctypes.c_double * 6)]


class _Model2(ctypes.Structure):
    _fields_ = [("n_bath", ctypes.c_int), ("n_elec", ctypes.c_int), ("band_lo", ctypes.c_double),
                ("band_hi", ctypes.c_double), ("mu", ctypes.c_double), ("mass", ctypes.c_double),
                ("omega", ctypes.c_double), ("x0", ctypes.c_double * 6),
                ("theta", ctypes.c_double * 16), ("vbar", ctypes.c_double * 2),
                ("R", ctypes.c_double * 6), ("profile", ctypes.c_int),
                ("prof_center", ctypes.c_double * 2), ("prof_width", ctypes.c_double * 2),
                ("eigensolver", ctypes.c_int)]


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("skip_bound", ctypes.c_int),
                ("record_every", ctypes.c_int), ("max_records", ctypes.c_int),
                ("z_done", ctypes.c_double), ("compact_every", ctypes.c_int),
                ("propagator", ctypes.c_int), ("traj_base", ctypes.c_int64),
                ("prop_tol", ctypes.c_double), ("norm_tol", ctypes.c_double),
                ("no_deflation", ctypes.c_int)]


EXPORTS = ["iesh_create", "iesh_destroy", "iesh_bath", "iesh_init_state", "iesh_set_state",
           "iesh_get_state", "iesh_run", "iesh_get_eigen", "iesh_hop_probabilities",
           "iesh_get_counters", "iesh_get_records", "iesh_get_propagator_terms", "iesh_profile",
           "iesh_profile_read", "iesh_get_live", "iesh_set_kernel_shape",
           "iesh_get_kernel_shape", "iesh_hop_probabilities_noalloc", "iesh_eocc_create",
           "iesh_eocc_destroy", "iesh_eocc_last_error", "iesh_eocc_forward",
           "iesh_eocc_backward", "iesh_last_error", "iesh_status_string", "iesh2_create",
           "iesh2_destroy", "iesh2_last_error", "iesh2_set_state", "iesh2_get_state", "iesh2_run",
           "iesh2_get_eigen", "iesh2_hop_probabilities", "iesh2_get_counters", "iesh2_profile",
           "iesh2_profile_read", "iesh_checkpoint_bytes", "iesh_checkpoint_save",
           "iesh_checkpoint_load", "iesh_run_host", "iesh_observables", "iesh_check", "iesh_syev_work_bytes",
           "iesh_syev_batched", "iesh_ensemble_create", "iesh_ensemble_run",
           "iesh_ensemble_status", "iesh_ensemble_destroy", "iesh_ensemble_last_error",
           "iesh_diag_reciprocal"]
KERNEL_CLASSES = ["eigen", "coupling", "propagate", "hop", "other"]

_lib = None
_vp = ctypes.c_void_p


def load(path=LIB_PATH):
    """Load libiesh.so once (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libiesh.so not built at {path}; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    L.iesh_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_Model),
                              ctypes.POINTER(_Options), ctypes.c_int64, _vp]
    L.iesh_destroy.argtypes = [_vp]
    L.iesh_bath.argtypes = [_vp, _vp, _vp]
    L.iesh_init_state.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_uint64]
    L.iesh_set_state.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp]
    L.iesh_get_state.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    L.iesh_run.argtypes = [_vp, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64]
    L.iesh_get_eigen.argtypes = [_vp, _vp, _vp, _vp]
    L.iesh_hop_probabilities.argtypes = [_vp, ctypes.c_double, _vp]
    L.iesh_get_counters.argtypes = [_vp, _vp, _vp, _vp]
    L.iesh_get_records.argtypes = [_vp, _vp, _vp, _vp]
    L.iesh_get_propagator_terms.argtypes = [_vp, _vp]
    L.iesh_profile.argtypes = [_vp, ctypes.c_int]
    L.iesh_get_live.argtypes = [_vp, _vp]
    L.iesh_set_kernel_shape.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.iesh_get_kernel_shape.argtypes = [_vp, _vp, _vp, _vp]
    L.iesh_profile_read.argtypes = [_vp, _vp, _vp]
    L.iesh_hop_probabilities_noalloc.argtypes = [ctypes.POINTER(_Model), ctypes.c_int64, _vp, _vp,
                                                 _vp, _vp, _vp, _vp, ctypes.c_double, _vp, _vp,
                                                 ctypes.c_char_p, ctypes.c_size_t]
    L.iesh_eocc_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_EoccModel), _vp]
    L.iesh_eocc_destroy.argtypes = [_vp]
    L.iesh_eocc_last_error.argtypes = [_vp]
    L.iesh_eocc_last_error.restype = ctypes.c_char_p
    L.iesh_eocc_forward.argtypes = [_vp, ctypes.c_int64, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]
    L.iesh_eocc_backward.argtypes = [_vp, ctypes.c_int64, ctypes.c_int, _vp, _vp, _vp, _vp, _vp,
                                     _vp, _vp]
    L.iesh2_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_Model2), ctypes.c_int,
                               ctypes.c_int64, ctypes.c_int, _vp]
    L.iesh2_destroy.argtypes = [_vp]
    L.iesh2_last_error.argtypes = [_vp]
    L.iesh2_last_error.restype = ctypes.c_char_p
    L.iesh2_set_state.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp]
    L.iesh2_get_state.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    L.iesh2_run.argtypes = [_vp, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64]
    L.iesh2_get_eigen.argtypes = [_vp, _vp, _vp, _vp]
    L.iesh2_hop_probabilities.argtypes = [_vp, ctypes.c_double, _vp]
    L.iesh2_get_counters.argtypes = [_vp, _vp, _vp, _vp]
    L.iesh2_profile.argtypes = [_vp, ctypes.c_int]
    L.iesh2_profile_read.argtypes = [_vp, _vp, _vp]
    L.iesh_checkpoint_bytes.argtypes = [_vp, _vp]
    L.iesh_checkpoint_save.argtypes = [_vp, _vp, ctypes.c_size_t]
    L.iesh_checkpoint_load.argtypes = [_vp, _vp, ctypes.c_size_t]
    L.iesh_run_host.argtypes = [_vp, _vp, _vp, ctypes.c_size_t, ctypes.c_double, ctypes.c_int64,
                                ctypes.c_uint64, ctypes.c_int]
    L.iesh_observables.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.iesh_check.argtypes = [_vp, _vp]
    L.iesh_ensemble_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int,
                                       ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, _vp]
    L.iesh_ensemble_run.argtypes = [_vp, ctypes.c_int64]
    L.iesh_diag_reciprocal.argtypes = [ctypes.c_int64, _vp, _vp, _vp]
    L.iesh_ensemble_status.argtypes = [_vp, _vp, _vp]
    L.iesh_ensemble_destroy.argtypes = [_vp]
    L.iesh_ensemble_last_error.argtypes = [_vp]
    L.iesh_ensemble_last_error.restype = ctypes.c_char_p
    L.iesh_syev_work_bytes.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.iesh_syev_batched.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp,
                                    _vp, ctypes.c_size_t, _vp, ctypes.c_char_p, ctypes.c_size_t]
    L.iesh_last_error.argtypes = [_vp]
    L.iesh_last_error.restype = ctypes.c_char_p
    L.iesh_status_string.argtypes = [ctypes.c_int]
    L.iesh_status_string.restype = ctypes.c_char_p
    for name in EXPORTS:
        getattr(L, name).restype = getattr(L, name).restype if name in (
            "iesh_last_error", "iesh_status_string", "iesh_eocc_last_error",
            "iesh2_last_error", "iesh_ensemble_last_error") else ctypes.c_int
    L.iesh_syev_work_bytes.restype = ctypes.c_size_t
    _lib = L
    return L


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "arrays must be contiguous"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensors must be contiguous"
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def model_struct(md):
    """iesh_model from a plain model dictionary (see iesh_inputs)."""
    m = _Model()
    m.kind = _KIND[md["kind"]]
    m.mass = float(md["mass"])
    for i, v in enumerate(md["par"]):
        m.par[i] = float(v)
    m.gamma = float(md["Gamma"])
    m.band_lo, m.band_hi = (float(v) for v in md["band"])
    m.mu = float(md.get("mu", 0.0))
    m.n_bath = int(md["M"])
    m.n_elec = int(md["Ne"])
    m.disc = _DISC[md.get("disc", "gl")]
    m.n_lo = -1 if md.get("n_lo") is None else int(md["n_lo"])
    leads = md.get("leads")
    if leads:
        m.n_leads = len(leads)
        for i, (mu_l, n_lo, n_l, frac) in enumerate(leads):
            m.lead_mu[i] = float(mu_l)
            m.lead_nlo[i] = int(n_lo)
            m.lead_n[i] = int(n_l)
            m.lead_frac[i] = float(frac)
    return m


def current_stream_handle():
    """cudaStream_t of torch's current stream on the current device (0 if no torch CUDA)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


class Context:
    """A batch of IESH trajectories on one GPU (wraps iesh_ctx)."""

    def __init__(self, model, max_traj, precision=PREC_FP64, skip_bound=False, record_every=0,
                 max_records=0, z_done=0.0, compact_every=0, stream=None, propagator=PROP_AVERAGED,
                 traj_base=0, prop_tol=0.0, norm_tol=0.0, deflation=True):
        self.L = load()
        self.model = dict(model)
        self.N = int(model["M"]) + 1
        self.Ne = int(model["Ne"])
        self.precision = precision
        self.max_traj = int(max_traj)
        self.n = 0
        self._m = model_struct(model)
        self.propagator = int(propagator)
        self.deflation = bool(deflation)
        self._o = _Options(precision, int(bool(skip_bound)), int(record_every), int(max_records),
                           float(z_done), int(compact_every), self.propagator, int(traj_base),
                           float(prop_tol), float(norm_tol), int(not deflation))
        self.stream = current_stream_handle() if stream is None else stream
        h = _vp()
        rc = self.L.iesh_create(ctypes.byref(h), ctypes.byref(self._m), ctypes.byref(self._o),
                                self.max_traj, _vp(self.stream) if self.stream else None)
        self._h = h
        if rc != IESH_OK:
            msg = self.L.iesh_last_error(h).decode() if h.value else ""
            self.L.iesh_destroy(h)
            self._h = None
            raise IeshError(f"iesh_create: {STATUS_NAMES.get(rc, rc)}: {msg}")

    def close(self):
        if getattr(self, "_h", None):
            self.L.iesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != IESH_OK:
            raise IeshError(f"{what}: {STATUS_NAMES.get(rc, rc)}: "
                            f"{self.L.iesh_last_error(self._h).decode()}")

    @property
    def cdtype(self):
        return np.complex128 if self.precision == PREC_FP64 else np.complex64

    # -------------------------------------------------------------- state
    def bath(self):
        eps = np.zeros(self.N - 1)
        z0 = np.zeros(self.N - 1)
        self._check(self.L.iesh_bath(self._h, eps.ctypes.data, z0.ctypes.data), "iesh_bath")
        return eps, z0

    def init_state(self, n, x0=None, p0=None, occ0=None, kT_nuc=0.0, kT_el=0.0, seed=0):
        self._check(self.L.iesh_init_state(self._h, int(n), _ptr(x0), _ptr(p0), _ptr(occ0),
                                           float(kT_nuc), float(kT_el), int(seed)),
                    "iesh_init_state")
        self.n = int(n)

    def set_state(self, x, p, occ, C):
        n = int(x.shape[0])
        self._check(self.L.iesh_set_state(self._h, n, _ptr(x), _ptr(p), _ptr(occ), _ptr(C)),
                    "iesh_set_state")
        self.n = n

    def get_state(self, x=None, p=None, occ=None, C=None, status=None):
        """Copy the state out; by default into new host numpy arrays."""
        n = self.n
        x = np.zeros(n) if x is None else x
        p = np.zeros(n) if p is None else p
        occ = np.zeros((n, self.Ne), np.int16) if occ is None else occ
        C = np.zeros((n, self.Ne, self.N), self.cdtype) if C is None else C
        status = np.zeros(n, np.uint32) if status is None else status
        self._check(self.L.iesh_get_state(self._h, _ptr(x), _ptr(p), _ptr(occ), _ptr(C),
                                          _ptr(status)), "iesh_get_state")
        return dict(x=x, p=p, occ=occ, C=C, status=status)

    def run(self, dt, n_steps, seed=0):
        self._check(self.L.iesh_run(self._h, float(dt), int(n_steps), int(seed)), "iesh_run")

    def eigen(self):
        lam = np.zeros((self.n, self.N))
        q0 = np.zeros((self.n, self.N))
        F = np.zeros(self.n)
        self._check(self.L.iesh_get_eigen(self._h, lam.ctypes.data, q0.ctypes.data,
                                          F.ctypes.data), "iesh_get_eigen")
        return lam, q0, F

    def hop_probabilities(self, dt):
        g = np.zeros((self.n, self.Ne, self.N))
        self._check(self.L.iesh_hop_probabilities(self._h, float(dt), g.ctypes.data),
                    "iesh_hop_probabilities")
        return g

    def counters(self):
        ns = np.zeros(self.n, np.int64)
        hops = np.zeros(self.n, np.int32)
        fr = np.zeros(self.n, np.int32)
        self._check(self.L.iesh_get_counters(self._h, ns.ctypes.data, hops.ctypes.data,
                                             fr.ctypes.data), "iesh_get_counters")
        return ns, hops, fr

    def live_count(self):
        n = ctypes.c_int64(0)
        self._check(self.L.iesh_get_live(self._h, ctypes.addressof(n)), "iesh_get_live")
        return n.value

    def set_kernel_shape(self, cheb_ept=0, cheb_G=0, hop_threads=0):
        """Propagator and hop kernel shapes (0 = built-in choice).  FP64:
        cheb_ept 1 or 2 with G column groups.  Mixed: cheb_ept 4 with G
        (SIMT kernel) or cheb_ept 8, G 1 (tensor-core kernel, N <= 128,
        Ne <= 56; the default where eligible)."""
        self._check(self.L.iesh_set_kernel_shape(self._h, int(cheb_ept), int(cheb_G),
                                                 int(hop_threads)), "iesh_set_kernel_shape")

    def kernel_shape(self):
        """(cheb_ept, cheb_G, hop_threads) in effect; cheb_ept 8 = tensor cores."""
        e, g, h = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        self._check(self.L.iesh_get_kernel_shape(self._h, ctypes.addressof(e), ctypes.addressof(g),
                                                 ctypes.addressof(h)), "iesh_get_kernel_shape")
        return e.value, g.value, h.value

    def propagator_terms(self):
        K = np.zeros(self.n, np.int32)
        self._check(self.L.iesh_get_propagator_terms(self._h, K.ctypes.data),
                    "iesh_get_propagator_terms")
        return K

    def profile(self, enable=True):
        """Switch per-kernel CUDA-event timing on (resetting it) or off."""
        self._check(self.L.iesh_profile(self._h, int(bool(enable))), "iesh_profile")

    def profile_read(self):
        """{kernel class: (ms summed, launches)} since profiling was switched on."""
        ms = np.zeros(len(KERNEL_CLASSES))
        n = np.zeros(len(KERNEL_CLASSES), np.int64)
        self._check(self.L.iesh_profile_read(self._h, ms.ctypes.data, n.ctypes.data),
                    "iesh_profile_read")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES)}

    def checkpoint_bytes(self):
        b = ctypes.c_size_t(0)
        self._check(self.L.iesh_checkpoint_bytes(self._h, ctypes.addressof(b)),
                    "iesh_checkpoint_bytes")
        return b.value

    def checkpoint_save(self, buf=None):
        """Write the checkpoint of the whole batch into `buf` (host numpy
        uint8 array or CUDA tensor), by default a new host array."""
        nb = self.checkpoint_bytes()
        buf = np.zeros(nb, np.uint8) if buf is None else buf
        size = buf.nbytes if isinstance(buf, np.ndarray) else buf.numel() * buf.element_size()
        self._check(self.L.iesh_checkpoint_save(self._h, _ptr(buf), int(size)),
                    "iesh_checkpoint_save")
        return buf

    def run_host(self, src, dst, dt, n_steps, seed=0, chunks=0):
        """Advance the batch held in the host checkpoint `src` by n_steps and
        write the result to `dst` (may be `src`), copies overlapped with the
        steps over `chunks` trajectory ranges (iesh_run_host)."""
        size = src.nbytes if isinstance(src, np.ndarray) else src.numel() * src.element_size()
        self._check(self.L.iesh_run_host(self._h, _ptr(src), _ptr(dst), int(size), float(dt), int(n_steps),
                                         int(seed), int(chunks)), "iesh_run_host")
        hdr = np.asarray(src[:64].cpu() if hasattr(src, "cpu") else src[:64]).view(np.int64)
        self.n = int(hdr[3])

    def checkpoint_load(self, buf):
        size = buf.nbytes if isinstance(buf, np.ndarray) else buf.numel() * buf.element_size()
        self._check(self.L.iesh_checkpoint_load(self._h, _ptr(buf), int(size)),
                    "iesh_checkpoint_load")
        hdr = np.asarray(buf[:64].cpu() if hasattr(buf, "cpu") else buf[:64]).view(np.int64)
        self.n = int(hdr[3])

    def observables(self):
        """Per trajectory: kinetic energy, potential energy U0 + sum of the
        occupied eigenvalues, occupied-surface and wavefunction impurity
        populations."""
        out = [np.zeros(self.n) for _ in range(4)]
        self._check(self.L.iesh_observables(self._h, *(o.ctypes.data for o in out)),
                    "iesh_observables")
        return dict(ke=out[0], epot=out[1], pop_sh=out[2], pop_wf=out[3])

    def check(self):
        """(status code, OR of the status words, per-bit trajectory counts)."""
        bits = np.zeros(9, np.uint32)
        rc = self.L.iesh_check(self._h, bits.ctypes.data)
        if rc not in (0, 6, 7, 8, 9):
            self._check(rc, "iesh_check")
        return STATUS_NAMES.get(rc, rc), int(bits[0]), bits[1:].copy()

    def records(self, max_records):
        sh = np.zeros((max_records, self.n))
        wf = np.zeros((max_records, self.n))
        nr = ctypes.c_int64(0)
        self._check(self.L.iesh_get_records(self._h, sh.ctypes.data, wf.ctypes.data,
                                            ctypes.addressof(nr)), "iesh_get_records")
        return sh[: nr.value], wf[: nr.value]


def hop_probabilities_noalloc(model, x, p, occ, C, lam, q0, dt, g, stream=None):
    """Hop probabilities g[n][Ne][N] into the caller's device array `g`, with
    no device allocation (see iesh_hop_probabilities_noalloc in iesh.h).
    All arrays are CUDA tensors; C is complex128 [n][Ne][N]."""
    L = load()
    m = model_struct(model)
    err = ctypes.create_string_buffer(512)
    s = current_stream_handle() if stream is None else stream
    rc = L.iesh_hop_probabilities_noalloc(ctypes.byref(m), int(x.shape[0]), _ptr(x), _ptr(p),
                                          _ptr(occ), _ptr(C), _ptr(lam), _ptr(q0), float(dt),
                                          _ptr(g), _vp(s) if s else None, err, len(err))
    if rc != IESH_OK:
        raise IeshError(f"iesh_hop_probabilities_noalloc: {STATUS_NAMES.get(rc, rc)}: "
                        f"{err.value.decode()}")


class Ensemble:
    """Contexts advanced together by one device-side loop (wraps
    iesh_ensemble): every context by `chunk` steps per iteration, work lists
    compacted on the device, until no trajectory is live or the step cap."""

    def __init__(self, contexts, dt, chunk, seed=0, stream=None):
        self.L = load()
        self.contexts = list(contexts)
        arr = (_vp * len(self.contexts))(*[c._h.value for c in self.contexts])
        self.stream = current_stream_handle() if stream is None else stream
        h = _vp()
        rc = self.L.iesh_ensemble_create(ctypes.byref(h), arr, len(self.contexts), float(dt),
                                         int(chunk), int(seed), _vp(self.stream) if self.stream else None)
        self._h = h
        if rc != IESH_OK:
            msg = self.L.iesh_ensemble_last_error(h).decode() if h.value else ""
            self.L.iesh_ensemble_destroy(h)
            self._h = None
            raise IeshError(f"iesh_ensemble_create: {STATUS_NAMES.get(rc, rc)}: {msg}")

    def _check(self, rc, what):
        if rc != IESH_OK:
            raise IeshError(f"{what}: {STATUS_NAMES.get(rc, rc)}: "
                            f"{self.L.iesh_ensemble_last_error(self._h).decode()}")

    def run(self, max_steps):
        """One graph launch (asynchronous)."""
        self._check(self.L.iesh_ensemble_run(self._h, int(max_steps)), "iesh_ensemble_run")

    def status(self):
        """(loop steps so far, live trajectories after the last chunk)."""
        s, l = ctypes.c_int64(0), ctypes.c_int64(0)
        self._check(self.L.iesh_ensemble_status(self._h, ctypes.addressof(s), ctypes.addressof(l)),
                    "iesh_ensemble_status")
        return s.value, l.value

    def close(self):
        if getattr(self, "_h", None):
            self.L.iesh_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def syev_batched(A, lam, V=None, info=None, work=None, stream=None):
    """Eigenvalues lam [B][n] (ascending) and eigenvector rows V [B][n][n] of
    the symmetric matrices A [B][n][n] (CUDA tensors, float64 or float32; see
    iesh_syev_batched in iesh.h).  work: a CUDA uint8 tensor of at least
    iesh_syev_work_bytes bytes (allocated here when None)."""
    import torch
    L = load()
    B, n = int(A.shape[0]), int(A.shape[1])
    prec = PREC_FP64 if A.dtype == torch.float64 else PREC_MIXED
    need = L.iesh_syev_work_bytes(B, n, prec, int(V is not None))
    if work is None:
        work = torch.empty(max(need, 1), dtype=torch.uint8, device=A.device)
    err = ctypes.create_string_buffer(512)
    s = current_stream_handle() if stream is None else stream
    rc = L.iesh_syev_batched(B, n, prec, _ptr(A), _ptr(lam), _ptr(V), _ptr(info), _ptr(work),
                             int(work.numel()), _vp(s) if s else None, err, len(err))
    if rc != IESH_OK:
        raise IeshError(f"iesh_syev_batched: {STATUS_NAMES.get(rc, rc)}: {err.value.decode()}")


def vbar(model):
    return math.sqrt(model["Gamma"] / (2 * math.pi))
