"""TEST INFRASTRUCTURE ONLY: ctypes front end of the plain FP64 CPU oracle.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It never imports the CUDA package; both
are fed the same plain model dictionaries and seeded inputs.

A model dictionary holds
  kind   'harmonic' | 'erpenbeck' | 'morse_image'
  mass   nuclear mass (a.u.)
  par    model constants in a.u. (see iesh_oracle.c, orc_model_eval)
  Gamma  wide-band hybridisation (a.u.), V_k = sqrt(Gamma/2pi) sqrt(w_k) f(x)
  band   (a, b) band edges
  mu     split point of the Gauss-Legendre discretisation
  M, Ne  bath states and electrons
  disc   'gl' (split Gauss-Legendre, Appendix A) or 'trapezoid'
  leads  optional list of (mu_lead, n_lo, n_states, gamma_fraction): each lead is
         discretised on the band with its own split, the couplings scaled by
         sqrt(gamma_fraction); the leads are merged in ascending energy.

Coefficient matrices here are [n_traj][N][Ne] complex128 (row = orbital);
the CUDA library's layout is [n_traj][Ne][N] and the tests transpose.
"""
import ctypes
import math
import os

import numpy as np

from . import build_oracle

_KIND = {"harmonic": 0, "erpenbeck": 1, "morse_image": 2}
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        L.orc_gauss_legendre.argtypes = [ctypes.c_int, _dp, _dp]
        L.orc_bath.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_int, _dp, _dp]
        L.orc_jacobi_sym.argtypes = [ctypes.c_int, _dp, _dp, _dp]
        L.orc_jacobi_herm.argtypes = [ctypes.c_int, _vp, _dp, _vp]
        L.orc_model_eval_x.argtypes = [ctypes.c_int, ctypes.c_double, _dp, ctypes.c_double, _dp]
        L.orc_eigen_x.argtypes = [ctypes.c_int, ctypes.c_double, _dp, ctypes.c_double,
                                  ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double, _ip,
                                  _dp, _dp, _dp, _dp, _dp]
        L.orc_propagate.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp,
                                    _dp, ctypes.c_double, ctypes.c_double, _vp]
        L.orc_det_x.argtypes = [ctypes.c_int, _vp, _dp]
        L.orc_inverse.argtypes = [ctypes.c_int, _vp, _vp]
        L.orc_hop_probs_x.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _vp, _dp, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, _dp, _dp, _vp]
        L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.orc_hop_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64]
        L.orc_hop_uniform.restype = ctypes.c_double
        L.orc_sample_nuclear.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, _dp, _dp]
        L.orc_sample_occupations.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                             ctypes.c_int, _dp, ctypes.c_double, _ip]
        L.orc_run.argtypes = [ctypes.c_int, ctypes.c_double, _dp, ctypes.c_double, ctypes.c_int,
                              ctypes.c_int, _dp, _dp, ctypes.c_int64, _dp, _dp, _dp, _ip, _vp,
                              ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                              ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _u32p, _i64p,
                              _i64p, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _i64p]
        L.orc_step_one.argtypes = [ctypes.c_int, ctypes.c_double, _dp, ctypes.c_double,
                                   ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _ip, _vp,
                                   ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_int, _dp, _dp, _ip, _dp, ctypes.c_int]
        L.orc_propagate_overlap.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp,
                                            ctypes.c_double, _vp]
        L.orc_select.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _dp, ctypes.c_double]
        L.orc_run2.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, ctypes.c_double,
                               ctypes.c_double, _dp, ctypes.c_int64, _dp, _dp, _dp, _ip, _vp,
                               ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, _u32p, _i64p, _i64p, _dp]
        L.orc_eigen2.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, ctypes.c_double,
                                 ctypes.c_double, _dp, _dp, _ip, _dp, _dp, _dp, _dp]
        L.orc_eocc.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_int64,
                               _dp, _dp, _dp, _dp, _dp]
        L.orc_run2g.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_double,
                                ctypes.c_double, _dp, ctypes.c_int64, _dp, _dp, _dp, _ip, _vp,
                                ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, _u32p, _i64p, _i64p,
                                _dp, _dp]
        L.orc_eigen2g.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_double,
                                  ctypes.c_double, _dp, _dp, _ip, _dp, _dp, _dp, _dp, _dp]
        L.orc_syev.argtypes = [ctypes.c_int64, ctypes.c_int, _dp, _dp, _dp]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _c(a, t=np.float64):
    return np.ascontiguousarray(a, dtype=t)


# ---------------------------------------------------------------- bath / model
def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    rc = lib().orc_gauss_legendre(n, _d(x), _d(w))
    assert rc == 0
    return x, w


def _lead_bath(disc, n, a, b, mu, n_lo):
    eps = np.zeros(n)
    w = np.zeros(n)
    rc = lib().orc_bath({"gl": 0, "trapezoid": 1}[disc], n, a, b, mu,
                        -1 if n_lo is None else int(n_lo), _d(eps), _d(w))
    assert rc == 0
    return eps, w


def bath(model):
    """Bath energies eps[M] (ascending) and sqrt-weights sqw[M] (Appendix A)."""
    a, b = model["band"]
    leads = model.get("leads")
    if not leads:
        eps, w = _lead_bath(model.get("disc", "gl"), model["M"], a, b, model.get("mu", 0.0),
                            model.get("n_lo"))
        return eps, np.sqrt(w)
    es, ss = [], []
    for (mu_l, n_lo, n_l, frac) in leads:
        e, w = _lead_bath(model.get("disc", "gl"), n_l, a, b, mu_l, n_lo)
        es.append(e)
        ss.append(np.sqrt(w * frac))
    eps = np.concatenate(es)
    sqw = np.concatenate(ss)
    order = np.argsort(eps, kind="stable")
    return eps[order], sqw[order]


def _par(model):
    p = np.zeros(16)
    par = np.asarray(model["par"], dtype=np.float64)
    p[: len(par)] = par
    return p


def vbar(model):
    return math.sqrt(model["Gamma"] / (2.0 * math.pi))


def model_eval(model, x):
    """(U0, dU0, h, dh, f, df) at x."""
    out = np.zeros(6)
    p = _par(model)
    lib().orc_model_eval_x(_KIND[model["kind"]], model["mass"], _d(p), float(x), _d(out))
    return out


class _Bound:
    def __init__(self, model):
        self.model = model
        self.kind = _KIND[model["kind"]]
        self.mass = float(model["mass"])
        self.par = _par(model)
        self.Vbar = vbar(model)
        self.M = int(model["M"])
        self.Ne = int(model["Ne"])
        self.N = self.M + 1
        self.eps, self.sqw = bath(model)


def bind(model):
    return _Bound(model)


def eigen(model_or_bound, x, occ=None):
    """lam[N], Q[N][N] (column i = orbital i), T, d, F at position x."""
    B = model_or_bound if isinstance(model_or_bound, _Bound) else _Bound(model_or_bound)
    N = B.N
    lam = np.zeros(N)
    Q = np.zeros((N, N))
    T = np.zeros((N, N))
    d = np.zeros((N, N))
    F = np.zeros(1)
    occp = None
    if occ is not None:
        occ = _c(occ, np.int32)
        occp = occ.ctypes.data_as(_ip)
    rc = lib().orc_eigen_x(B.kind, B.mass, _d(B.par), B.Vbar, B.M, B.Ne, _d(B.eps), _d(B.sqw),
                           float(x), occp, _d(lam), _d(Q), _d(T), _d(d), _d(F))
    assert rc == 0, "Jacobi did not converge"
    return lam, Q, T, d, float(F[0])


# ------------------------------------------------------------------ linear algebra
def jacobi_sym(A):
    A = _c(A).copy()
    n = A.shape[0]
    ev = np.zeros(n)
    V = np.zeros((n, n))
    rc = lib().orc_jacobi_sym(n, _d(A), _d(ev), _d(V))
    assert rc == 0
    return ev, V


def jacobi_herm(A):
    A = _c(A, np.complex128).copy()
    n = A.shape[0]
    ev = np.zeros(n)
    V = np.zeros((n, n), dtype=np.complex128)
    rc = lib().orc_jacobi_herm(n, A.ctypes.data, _d(ev), V.ctypes.data)
    assert rc == 0
    return ev, V


def det(S):
    S = _c(S, np.complex128)
    r = np.zeros(2)
    lib().orc_det_x(S.shape[0], S.ctypes.data, _d(r))
    return complex(r[0], r[1])


def inverse(S):
    S = _c(S, np.complex128)
    out = np.zeros_like(S)
    rc = lib().orc_inverse(S.shape[0], S.ctypes.data, out.ctypes.data)
    assert rc == 0
    return out


def propagate(lam0, d0, v0, lam1, d1, v1, dt, C):
    """Exponential integrator over one step; C is [N][Ne] complex, returned new."""
    C = _c(C, np.complex128).copy()
    N, Ne = C.shape
    rc = lib().orc_propagate(N, Ne, _d(_c(lam0)), _d(_c(d0)), float(v0), _d(_c(lam1)),
                             _d(_c(d1)), float(v1), float(dt), C.ctypes.data)
    assert rc == 0
    return C


def hop_probs(occ, C, d, v, dt, brute=False):
    """g[Ne][N], Re(R)[Ne][N], det S for coefficients C[N][Ne]."""
    C = _c(C, np.complex128)
    N, Ne = C.shape
    occ = _c(occ, np.int32)
    g = np.zeros((Ne, N))
    R = np.zeros((Ne, N))
    ds = np.zeros(2)
    rc = lib().orc_hop_probs_x(N, Ne, occ.ctypes.data_as(_ip), C.ctypes.data, _d(_c(d)),
                               float(v), float(dt), int(brute), _d(g), _d(R), ds.ctypes.data)
    return g, R, complex(ds[0], ds[1]), rc


def select(occ, g, zeta):
    """(a, m) chosen by the uniform zeta from g[Ne][N], or None."""
    g = _c(g)
    Ne, N = g.shape
    occ = _c(occ, np.int32)
    r = lib().orc_select(N, Ne, occ.ctypes.data_as(_ip), _d(g), float(zeta))
    return None if r < 0 else divmod(r, N)


# ---------------------------------------------------------------------- random
def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return list(o)


def hop_uniform(seed, traj, n):
    return lib().orc_hop_uniform(seed, traj, n)


def sample_nuclear(seed, traj, mass, omega, x_eq, kT, wigner=False):
    x = np.zeros(1)
    p = np.zeros(1)
    lib().orc_sample_nuclear(seed, traj, mass, omega, x_eq, kT, int(wigner), _d(x), _d(p))
    return float(x[0]), float(p[0])


def sample_occupations(seed, traj, lam, Ne, kT):
    lam = _c(lam)
    occ = np.zeros(Ne, dtype=np.int32)
    rc = lib().orc_sample_occupations(seed, traj, lam.shape[0], Ne, _d(lam), float(kT),
                                      occ.ctypes.data_as(_ip))
    assert rc == 0
    return occ


# ---------------------------------------------------------------------- dynamics
def unit_coefficients(N, occ):
    """C[N][Ne] with electron j in orbital occ[j]."""
    Ne = len(occ)
    C = np.zeros((N, Ne), dtype=np.complex128)
    for j, o in enumerate(occ):
        C[o, j] = 1.0
    return C


def step_one(model_or_bound, x, p, occ, C, dt, seed, traj, n, brute=False, prop=0):
    """One step of one trajectory from (x, p, occ, C[N][Ne]).  prop 0: the
    exponential of the averaged adiabatic generator; prop 1: the
    diabatic-basis (overlap) propagator.

    Returns dict with the new state and the step's g[Ne][N], zeta, hop flag."""
    B = model_or_bound if isinstance(model_or_bound, _Bound) else _Bound(model_or_bound)
    xa = np.array([x], dtype=np.float64)
    pa = np.array([p], dtype=np.float64)
    Fa = np.zeros(1)
    occ = _c(occ, np.int32).copy()
    C = _c(C, np.complex128).copy()
    g = np.zeros((B.Ne, B.N))
    zeta = np.zeros(1)
    hop = np.zeros(1, dtype=np.int32)
    lam = np.zeros(B.N)
    st = lib().orc_step_one(B.kind, B.mass, _d(B.par), B.Vbar, B.M, B.Ne, _d(B.eps), _d(B.sqw),
                            _d(xa), _d(pa), _d(Fa), occ.ctypes.data_as(_ip), C.ctypes.data,
                            float(dt), int(seed), int(traj), int(n), int(brute), _d(g),
                            _d(zeta), hop.ctypes.data_as(_ip), _d(lam), int(prop))
    return dict(x=float(xa[0]), p=float(pa[0]), F=float(Fa[0]), occ=occ, C=C, g=g,
                zeta=float(zeta[0]), hop=int(hop[0]), lam=lam, status=st)


def run(model_or_bound, x, p, occ, C, dt, n_steps, seed, step0=0, brute=False,
        record_every=0, n_threads=None, prop=0, z_done=0.0):
    """Advance a batch: x, p [n]; occ [n][Ne]; C [n][N][Ne].  prop selects the
    electronic propagator (0 averaged-generator exponential, 1 overlap).  With
    z_done > 0 a trajectory stops at the end of the first step with
    x > z_done (status bit 8); "steps" holds the steps each one took.
    Returns a dict."""
    B = model_or_bound if isinstance(model_or_bound, _Bound) else _Bound(model_or_bound)
    x = _c(x).copy()
    p = _c(p).copy()
    n = x.shape[0]
    occ = _c(occ, np.int32).copy()
    C = _c(C, np.complex128).copy()
    assert occ.shape == (n, B.Ne) and C.shape == (n, B.N, B.Ne)
    F = np.zeros(n)
    status = np.zeros(n, dtype=np.uint32)
    hops = np.zeros(n, dtype=np.int64)
    frus = np.zeros(n, dtype=np.int64)
    lam = np.zeros((n, B.N))
    steps = np.zeros(n, dtype=np.int64)
    n_rec = int(n_steps // record_every) if record_every else 0
    psh = np.zeros((max(n_rec, 1), n))
    pwf = np.zeros((max(n_rec, 1), n))
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    lib().orc_run(B.kind, B.mass, _d(B.par), B.Vbar, B.M, B.Ne, _d(B.eps), _d(B.sqw), n, _d(x),
                  _d(p), _d(F), occ.ctypes.data_as(_ip), C.ctypes.data, float(dt), int(n_steps),
                  int(seed), int(step0), int(brute), int(record_every), n_rec, _d(psh), _d(pwf),
                  status.ctypes.data_as(_u32p), hops.ctypes.data_as(_i64p),
                  frus.ctypes.data_as(_i64p), _d(lam), int(n_threads), int(prop), float(z_done),
                  steps.ctypes.data_as(_i64p))
    return dict(x=x, p=p, F=F, occ=occ, C=C, status=status, hops=hops, frustrated=frus,
                lam=lam, pop_sh=psh[:n_rec], pop_wf=pwf[:n_rec], steps=steps)


def propagate_overlap(lam0, Q0, lam1, Q1, dt, C):
    """C[N][Ne] <- exp(-i L1 dt/2) Q1^T Q0 exp(-i L0 dt/2) C (reading R15)."""
    N = len(lam0)
    C = _c(C, np.complex128).copy()
    lib().orc_propagate_overlap(N, C.shape[1], _d(_c(lam0)), _d(_c(Q0)), _d(_c(lam1)), _d(_c(Q1)),
                                float(dt), C.ctypes.data)
    return C


# ----------------------------------------------------- two-orbital dynamics
def _two_bath(md):
    eps, sqw = bath(dict(band=md["band"], M=md["M"], mu=0.0, disc="gl"))
    return _c(eps), _c(sqw)


def two_couplings(md, eps, sqw):
    """Vk[2][M]: coupling of adsorbate orbital a to bath state k at f_a = 1.
    Without a "profile" entry both orbitals couple as Vbar_a sqrt(w_k)
    (parallel border vectors, reading R16); with profile = dict(center,
    width) orbital a's coupling carries its own Lorentzian energy profile,
    Vbar_a sqrt(w_k) / sqrt(1 + ((eps_k - center_a) / width_a)^2)
    (reading R17)."""
    Vbar = _c(md["Vbar"])
    prof = md.get("profile")
    if prof is None:
        return np.vstack([Vbar[0] * sqw, Vbar[1] * sqw])
    out = np.zeros((2, eps.shape[0]))
    for a in range(2):
        u = (eps - prof["center"][a]) / prof["width"][a]
        out[a] = Vbar[a] * sqw / np.sqrt(1.0 + u * u)
    return out


def eigen2(md, x, occ, Qref=None):
    """Two-orbital model at x[6]: lam[N], Q[N][N], d[6][N][N], F[6] (N = M + 2).
    With an own bath profile per orbital (md["profile"], reading R17) the
    eigenvectors are signed by their overlap with Qref [N][N] (the previous
    step's) when given, else by the rule of R16."""
    eps, sqw = _two_bath(md)
    if md.get("profile") is not None:
        N = md["M"] + 2
        Vk = _c(two_couplings(md, eps, sqw))
        lam, Q, d, F = np.zeros(N), np.zeros((N, N)), np.zeros((6, N, N)), np.zeros(6)
        lib().orc_eigen2g(md["M"], md["Ne"], _d(eps), _d(Vk), _d(_c(md["R"])), _d(_c(md["theta"])),
                          float(md["mass"]), float(md["omega"]), _d(_c(md["x0"])), _d(_c(x)),
                          _c(occ, np.int32).ctypes.data_as(_ip),
                          None if Qref is None else _d(_c(Qref)), _d(lam), _d(Q), _d(d), _d(F))
        return lam, Q, d, F
    N = md["M"] + 2
    lam, Q, d, F = np.zeros(N), np.zeros((N, N)), np.zeros((6, N, N)), np.zeros(6)
    lib().orc_eigen2(md["M"], md["Ne"], _d(eps), _d(sqw), _d(_c(md["Vbar"])), _d(_c(md["R"])),
                     _d(_c(md["theta"])), float(md["mass"]), float(md["omega"]), _d(_c(md["x0"])),
                     _d(_c(x)), _c(occ, np.int32).ctypes.data_as(_ip), _d(lam), _d(Q), _d(d), _d(F))
    return lam, Q, d, F


def run2(md, x, p, occ, C, dt, n_steps, seed):
    """Two-orbital IESH batch: x, p [n][6]; occ [n][Ne]; C [n][N][Ne]."""
    eps, sqw = _two_bath(md)
    x = _c(x).copy()
    p = _c(p).copy()
    n = x.shape[0]
    occ = _c(occ, np.int32).copy()
    C = _c(C, np.complex128).copy()
    N = md["M"] + 2
    F = np.zeros((n, 6))
    status = np.zeros(n, np.uint32)
    hops = np.zeros(n, np.int64)
    frus = np.zeros(n, np.int64)
    lam = np.zeros((n, N))
    if md.get("profile") is not None:
        Vk = _c(two_couplings(md, eps, sqw))
        Qad = np.zeros((n, 2, N))
        lib().orc_run2g(md["M"], md["Ne"], _d(eps), _d(Vk), _d(_c(md["R"])), _d(_c(md["theta"])),
                        float(md["mass"]), float(md["omega"]), _d(_c(md["x0"])), n, _d(x), _d(p),
                        _d(F), occ.ctypes.data_as(_ip), C.ctypes.data, float(dt), int(n_steps),
                        int(seed), status.ctypes.data_as(_u32p), hops.ctypes.data_as(_i64p),
                        frus.ctypes.data_as(_i64p), _d(lam), _d(Qad))
        return dict(x=x, p=p, F=F, occ=occ, C=C, status=status, hops=hops, frustrated=frus,
                    lam=lam, Qad=Qad)
    lib().orc_run2(md["M"], md["Ne"], _d(eps), _d(sqw), _d(_c(md["Vbar"])), _d(_c(md["R"])),
                   _d(_c(md["theta"])), float(md["mass"]), float(md["omega"]), _d(_c(md["x0"])), n,
                   _d(x), _d(p), _d(F), occ.ctypes.data_as(_ip), C.ctypes.data, float(dt), int(n_steps),
                   int(seed), status.ctypes.data_as(_u32p), hops.ctypes.data_as(_i64p),
                   frus.ctypes.data_as(_i64p), _d(lam))
    return dict(x=x, p=p, F=F, occ=occ, C=C, status=status, hops=hops, frustrated=frus, lam=lam)


# ------------------------------------------------------------- occupied energy
def eocc(eps, sqw, Vbar, R, x, theta, Ne, grad=True):
    """E[B], dE/dx[B][6], dE/dtheta[B][16] for the two-orbital model."""
    eps = _c(eps)
    sqw = _c(sqw)
    Vbar = _c(Vbar)
    R = _c(R)
    x = _c(x).reshape(-1, 6)
    theta = _c(theta)
    B = x.shape[0]
    E = np.zeros(B)
    dx = np.zeros((B, 6)) if grad else None
    dth = np.zeros((B, 16)) if grad else None
    rc = lib().orc_eocc(eps.shape[0], Ne, _d(eps), _d(sqw), _d(Vbar), _d(R), B, _d(x),
                        _d(theta), _d(E), _d(dx) if grad else None, _d(dth) if grad else None)
    assert rc == 0
    return E, dx, dth


# -------------------------------------------------- dense symmetric eigenproblem
def syev(A):
    """Eigenvalues ascending lam [B][n] and unit eigenvectors as rows V
    [B][n][n] of the symmetric matrices A [B][n][n] (cyclic Jacobi), each
    eigenvector signed so that its largest-magnitude component is positive."""
    A = _c(A)
    B, n, _ = A.shape
    lam = np.zeros((B, n))
    V = np.zeros((B, n, n))
    rc = lib().orc_syev(B, n, _d(A), _d(lam), _d(V))
    return lam, V, rc
