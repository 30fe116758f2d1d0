"""Pins of the FP64 CPU oracle against values and identities fixed by the paper
and by mathematics, independent of the oracle's own code paths.

Each test is chosen so that a plausible slip (a dropped term, a wrong sign or
index, a transposed operand) in the oracle fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg

import iesh_inputs as W
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------ random
def test_philox_known_answers():
    for r in _golden("philox4x32_10_kat.txt"):
        v = [int(t, 16) for t in r]
        assert O.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_hop_uniform_range_and_mean():
    u = np.array([O.hop_uniform(7, t, n) for t in range(50) for n in range(100)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)


# -------------------------------------------------------------- quadrature
@pytest.mark.parametrize("n", [1, 2, 7, 25, 50, 100])
def test_gauss_legendre_matches_numpy(n):
    x, w = O.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.abs(x - xr).max() < 1e-13
    assert np.abs(w - wr).max() < 1e-13


def test_gl_split_bath():
    md = W.double_well(100)
    eps, sqw = O.bath(md)
    a, b = md["band"]
    assert np.all(np.diff(eps) > 0)
    assert np.all(eps[:50] < 0) and np.all(eps[50:] > 0)
    assert abs(np.sum(sqw ** 2) - (b - a)) < 1e-13
    # GL integrates polynomials up to degree 2n-1 exactly on each half
    assert abs(np.sum(sqw[:50] ** 2 * eps[:50] ** 3) - (0 - a ** 4) / 4) < 1e-15
    # hybridisation: sum_k V_k^2 = (Gamma / 2 pi) (b - a)
    Vk = O.vbar(md) * sqw
    assert abs(np.sum(Vk ** 2) - md["Gamma"] / (2 * math.pi) * (b - a)) < 1e-15


def test_trapezoid_bath_is_left_endpoint():
    md = W.double_well(10, disc="trapezoid")
    eps, sqw = O.bath(md)
    a, b = md["band"]
    assert np.allclose(eps, a + np.arange(10) * (b - a) / 10)
    assert np.allclose(sqw ** 2, (b - a) / 10)


# ---------------------------------------------------------------- eigen
def test_jacobi_sym_matches_lapack():
    rng = np.random.default_rng(1)
    for n in (1, 2, 5, 30):
        A = rng.standard_normal((n, n))
        A = A + A.T
        ev, V = O.jacobi_sym(A)
        assert np.abs(np.sort(ev) - np.linalg.eigvalsh(A)).max() < 1e-12
        assert np.abs(V.T @ V - np.eye(n)).max() < 1e-13
        assert np.abs(A @ V - V * ev).max() < 1e-12


def test_jacobi_herm_matches_lapack():
    rng = np.random.default_rng(2)
    for n in (1, 2, 6, 25):
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        A = A + A.conj().T
        ev, V = O.jacobi_herm(A)
        assert np.abs(np.sort(ev) - np.linalg.eigvalsh(A)).max() < 1e-12
        assert np.abs(V.conj().T @ V - np.eye(n)).max() < 1e-13
        assert np.abs(A @ V - V * ev).max() < 1e-12


@pytest.mark.parametrize("md,x", [(W.double_well(20), 1.3), (W.double_well_paper(40), 12.0),
                                  (W.desorption(1.0, 40), 4.0)])
def test_arrowhead_eigen(md, x):
    B = O.bind(md)
    lam, Q, T, d, F = O.eigen(B, x)
    U0, dU0, h, dh, f, df = O.model_eval(md, x)
    # dense H independently assembled here
    N = B.N
    H = np.zeros((N, N))
    H[0, 0] = h
    H[0, 1:] = H[1:, 0] = B.Vbar * B.sqw * f
    H[np.arange(1, N), np.arange(1, N)] = B.eps
    assert np.abs(lam - np.linalg.eigvalsh(H)).max() < 1e-13
    assert abs(lam.sum() - np.trace(H)) < 1e-12
    # strict interlacing with the bath energies
    assert np.all(lam[:-1] < B.eps) and np.all(B.eps < lam[1:])
    # gauge
    assert np.all(Q[0] > 0)
    assert np.abs(H @ Q - Q * lam).max() < 1e-13
    # secular equation at every eigenvalue
    z = B.Vbar * B.sqw * f
    sec = lam - h - np.array([np.sum(z ** 2 / (l - B.eps)) for l in lam])
    dsec = 1 + np.array([np.sum(z ** 2 / (l - B.eps) ** 2) for l in lam])
    # the Newton correction of each root is at rounding level
    assert np.abs(sec / dsec).max() < 2e-14 * max(1.0, np.abs(lam).max())


# ---------------------------------------------------------------- models
def test_desorption_model_pins():
    gold = {r[0]: (float(r[1]), float(r[2])) for r in _golden("desorption_model_pins.txt")}
    kT = 300.0 * W.KB_HARTREE_PER_K
    for key, mass_u in (("kT_over_hw_1u", 1.0), ("kT_over_hw_10p54u", 10.54)):
        md = W.desorption(mass_u=mass_u)
        x0 = md["par"][1]
        hh = 1e-4
        k = (O.model_eval(md, x0 + hh)[1] - O.model_eval(md, x0 - hh)[1]) / (2 * hh)
        assert abs(O.model_eval(md, x0)[1]) < 1e-14  # minimum of U0 at x0
        w = math.sqrt(k / md["mass"])
        val, tol = gold[key]
        assert abs(kT / w - val) < tol, (key, kT / w)
        if mass_u == 10.54:
            bw = w / kT
            Q = bw / (2 * math.tanh(bw / 2))
            val, tol = gold["wigner_Q_10p54u"]
            assert abs(Q - val) < tol
    md = W.desorption()
    # crossing of U0 and U1 (h = 0) between the minimum and 5 angstrom, by bisection
    lo, hi = md["par"][1], W.angstrom(5.0)
    assert O.model_eval(md, lo)[2] * O.model_eval(md, hi)[2] < 0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if O.model_eval(md, lo)[2] * O.model_eval(md, mid)[2] <= 0:
            hi = mid
        else:
            lo = mid
    xc = 0.5 * (lo + hi)
    U0c = O.model_eval(md, xc)[0]
    barrier = (U0c - md["par"][7]) * W.HARTREE_EV
    val, tol = gold["barrier_ev"]
    assert abs(barrier - val) < tol, barrier
    assert abs(xc * W.BOHR_ANGSTROM - 2.008) < 0.002


def test_model_derivatives_by_fd():
    for md, xs in ((W.double_well(10), [-2.0, 0.3, 5.0]), (W.desorption(), [2.5, 3.4, 7.0]),
                   (W.morse_image(10), [3.0, 9.0, 18.0])):
        for x in xs:
            h = 1e-5
            a = O.model_eval(md, x + h)
            b = O.model_eval(md, x - h)
            c = O.model_eval(md, x)
            for v, dv in ((0, 1), (2, 3), (4, 5)):
                fd = (a[v] - b[v]) / (2 * h)
                assert abs(fd - c[dv]) < 1e-7 * (1 + abs(c[dv])), (md["kind"], x, v)


# -------------------------------------------------------- force and couplings
@pytest.mark.parametrize("md,x", [(W.double_well(20), 1.3), (W.double_well_paper(40), 9.0),
                                  (W.desorption(1.0, 30), 3.9)])
def test_hellmann_feynman_force_by_fd(md, x):
    B = O.bind(md)
    rng = np.random.default_rng(3)
    occ = np.sort(rng.choice(B.N, size=B.Ne, replace=False)).astype(np.int32)
    _, _, _, _, F = O.eigen(B, x, occ)
    h = 1e-5

    def energy(xx):
        lam = O.eigen(B, xx)[0]
        return O.model_eval(md, xx)[0] + lam[occ].sum()

    fd = -(energy(x + h) - energy(x - h)) / (2 * h)
    assert abs(F - fd) < 1e-8 * (1 + abs(F))


@pytest.mark.parametrize("md,x", [(W.double_well(12), 0.7), (W.desorption(1.0, 16), 3.9)])
def test_nac_matches_fd_of_eigenvectors(md, x):
    B = O.bind(md)
    lam, Q, T, d, _ = O.eigen(B, x)
    h = 1e-6
    Qp = O.eigen(B, x + h)[1]
    Qm = O.eigen(B, x - h)[1]
    dQ = (Qp - Qm) / (2 * h)
    fd = Q.T @ dQ  # fd[j, k] = <j | d_x k>
    np.fill_diagonal(fd, 0.0)
    scale = np.abs(d).max()
    assert np.abs(d - fd).max() < 1e-6 * scale
    assert np.abs(d + d.T).max() < 1e-12 * scale


# ------------------------------------------------------------ propagation
def _random_state(B, seed, weight=0.5):
    occ = np.sort(np.random.default_rng(seed).choice(B.N, size=B.Ne, replace=False))
    C = W.mixed_coefficients(occ[None, :].astype(np.int16), B.N, seed, weight)[0].T
    return occ.astype(np.int32), np.ascontiguousarray(C)


def test_propagator_matches_expm_and_is_unitary():
    md = W.double_well_paper(16)
    B = O.bind(md)
    lam0, _, _, d0, _ = O.eigen(B, 3.0)
    lam1, _, _, d1, _ = O.eigen(B, 3.4)
    v0, v1, dt = 0.03, 0.035, 10.0
    _, C = _random_state(B, 4)
    Cn = O.propagate(lam0, d0, v0, lam1, d1, v1, dt, C)
    A = np.diag(0.5 * (lam0 + lam1)) - 0.5j * (v0 * d0 + v1 * d1)
    ref = scipy.linalg.expm(-1j * A * dt) @ C
    assert np.abs(Cn - ref).max() < 1e-12
    assert np.abs(Cn.conj().T @ Cn - np.eye(B.Ne)).max() < 1e-13


def test_propagator_zero_velocity_is_phase_only():
    B = O.bind(W.double_well(10))
    lam, _, _, d, _ = O.eigen(B, 1.0)
    _, C = _random_state(B, 5)
    Cn = O.propagate(lam, d, 0.0, lam, d, 0.0, 7.0, C)
    assert np.abs(Cn - np.exp(-1j * lam * 7.0)[:, None] * C).max() < 1e-13


def test_adiabatic_propagation_converges_to_diabatic():
    """Along a prescribed path x(t) = x0 + v t, Q(x) c_adiabatic must follow
    the diabatic TDSE i c' = H(x(t)) c; with the step-averaged generator the
    error falls as dt^2 (checks the NAC sign inside the generator)."""
    md = W.double_well_paper(8)
    B = O.bind(md)
    x0, v, Ttot = 4.0, 0.05, 400.0
    occ, C0 = _random_state(B, 6)
    Q0 = O.eigen(B, x0)[1]
    cd0 = Q0 @ C0

    def H_of(x):
        U0, dU0, h, dh, f, df = O.model_eval(md, x)
        H = np.diag(np.concatenate([[h], B.eps]))
        H[0, 1:] = H[1:, 0] = B.Vbar * B.sqw * f
        return H

    # diabatic reference: midpoint-exponential with tiny steps
    nref = 4000
    cd = cd0.copy()
    for k in range(nref):
        x = x0 + v * (k + 0.5) * Ttot / nref
        cd = scipy.linalg.expm(-1j * H_of(x) * Ttot / nref) @ cd
    errs = []
    for nst in (40, 80):
        dt = Ttot / nst
        C = C0.copy()
        lam0, Q, T, d0, _ = O.eigen(B, x0)
        for k in range(nst):
            lam1, Q, T, d1, _ = O.eigen(B, x0 + v * (k + 1) * dt)
            C = O.propagate(lam0, d0, v, lam1, d1, v, dt, C)
            lam0, d0 = lam1, d1
        errs.append(np.abs(Q @ C - cd).max())
    assert errs[1] < 5e-4
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def _H_diabatic(md, B, x):
    U0, dU0, h, dh, f, df = O.model_eval(md, x)
    H = np.diag(np.concatenate([[h], B.eps]))
    H[0, 1:] = H[1:, 0] = B.Vbar * B.sqw * f
    return H


def test_overlap_propagator_is_the_diabatic_strang_product():
    """Reading R15: in the diabatic basis the overlap propagator is
    exp(-i H(x1) dt/2) exp(-i H(x0) dt/2); checked against scipy's expm of
    the dense diabatic Hamiltonians, with the adiabatic frames of both ends."""
    md = W.double_well_paper(16)
    B = O.bind(md)
    x0, x1, dt = 3.0, 3.4, 10.0
    lam0, Q0 = O.eigen(B, x0)[:2]
    lam1, Q1 = O.eigen(B, x1)[:2]
    _, C = _random_state(B, 11)
    Cn = O.propagate_overlap(lam0, Q0, lam1, Q1, dt, C)
    U = scipy.linalg.expm(-0.5j * dt * _H_diabatic(md, B, x1)) @ scipy.linalg.expm(-0.5j * dt * _H_diabatic(md, B, x0))
    ref = Q1.T @ U @ (Q0 @ C)
    assert np.abs(Cn - ref).max() < 1e-12
    assert np.abs(Cn.conj().T @ Cn - np.eye(B.Ne)).max() < 1e-13


def test_overlap_propagator_frozen_nuclei_is_phase_only():
    B = O.bind(W.double_well(12))
    lam, Q = O.eigen(B, 1.5)[:2]
    _, C = _random_state(B, 12)
    Cn = O.propagate_overlap(lam, Q, lam, Q, 7.0, C)
    assert np.abs(Cn - np.exp(-1j * lam * 7.0)[:, None] * C).max() < 1e-13


def test_overlap_propagation_converges_to_diabatic():
    """Same moving-path check as for the averaged generator: the symmetric
    splitting is second order, error ratio ~4 when dt halves."""
    md = W.double_well_paper(8)
    B = O.bind(md)
    x0, v, Ttot = 4.0, 0.05, 400.0
    occ, C0 = _random_state(B, 6)
    cd = O.eigen(B, x0)[1] @ C0
    nref = 4000
    for k in range(nref):
        x = x0 + v * (k + 0.5) * Ttot / nref
        cd = scipy.linalg.expm(-1j * _H_diabatic(md, B, x) * Ttot / nref) @ cd
    errs = []
    for nst in (40, 80):
        dt = Ttot / nst
        C = C0.copy()
        lam0, Q0 = O.eigen(B, x0)[:2]
        for k in range(nst):
            lam1, Q1 = O.eigen(B, x0 + v * (k + 1) * dt)[:2]
            C = O.propagate_overlap(lam0, Q0, lam1, Q1, dt, C)
            lam0, Q0 = lam1, Q1
        errs.append(np.abs(Q1 @ C - cd).max())
    assert errs[1] < 5e-4
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_step_with_overlap_propagator_conserves_energy_and_norm():
    """A full oracle step with the variant: the coefficient columns stay
    orthonormal and, without hops, nuclear + occupied-orbital energy drifts
    only at the Verlet order."""
    md = W.double_well_paper(10)
    B = O.bind(md)
    occ, C = _random_state(B, 3)
    x, p = 6.0, 5.0
    r0 = O.step_one(B, x, p, occ, C, 5.0, seed=1, traj=0, n=0, prop=1)
    assert np.abs(r0["C"].conj().T @ r0["C"] - np.eye(B.Ne)).max() < 1e-12
    ra = O.step_one(B, x, p, occ, C, 5.0, seed=1, traj=0, n=0, prop=0)
    # same nuclei (the propagator does not feed back within a step), close coefficients
    assert r0["x"] == ra["x"] and r0["p"] == ra["p"]
    assert np.abs(r0["C"] - ra["C"]).max() < 1e-3


# ----------------------------------------------------- determinants and hops
def test_det_and_inverse_match_numpy():
    rng = np.random.default_rng(7)
    for n in (1, 3, 9):
        S = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        assert abs(O.det(S) - np.linalg.det(S)) < 1e-12 * abs(np.linalg.det(S)) + 1e-14
        assert np.abs(O.inverse(S) - np.linalg.inv(S)).max() < 1e-11


@pytest.mark.parametrize("M,Ne", [(5, 2), (7, 3), (11, 5)])
def test_ratio_mode_equals_brute_force(M, Ne):
    B = O.bind(W.double_well_paper(M))
    lam, Q, T, d, _ = O.eigen(B, 8.0)
    occ, C = _random_state(B, M)
    g1, R1, dS1, rc1 = O.hop_probs(occ, C, d, 0.02, 10.0, brute=True)
    g0, R0, dS0, rc0 = O.hop_probs(occ, C, d, 0.02, 10.0, brute=False)
    assert rc0 == rc1 == 0
    assert np.abs(R0 - R1).max() < 1e-11 * max(1, np.abs(R1).max())
    assert np.abs(g0 - g1).max() < 1e-11 * max(1e-30, np.abs(g1).max())
    assert abs(dS0 - np.linalg.det(C[occ, :])) < 1e-13
    # each ratio equals numpy's determinant of the replaced matrix
    S = C[occ, :]
    for a in range(Ne):
        for m in range(B.N):
            if m in occ:
                continue
            Sj = S.copy()
            Sj[a] = C[m]
            assert abs(R1[a, m] - (np.linalg.det(Sj) / np.linalg.det(S)).real) < 1e-11


def test_single_electron_reduces_to_fssh():
    md = W.double_well_paper(9)
    md["Ne"] = 1
    B = O.bind(md)
    lam, Q, T, d, _ = O.eigen(B, 8.0)
    rng = np.random.default_rng(8)
    c = rng.standard_normal(B.N) + 1j * rng.standard_normal(B.N)
    c /= np.linalg.norm(c)
    k = 3
    v, dt = 0.01, 10.0
    g, R, dS, rc = O.hop_probs(np.array([k]), c[:, None], d, v, dt)
    for m in range(B.N):
        if m == k:
            continue
        # Tully (1990): g_{k->m} = max(0, -2 dt Re(a*_{mk}) v d_mk / a_kk) with a_mk = c_m c_k*
        ref = max(0.0, -2 * dt * (np.conj(c[m] * np.conj(c[k]))).real * v * d[m, k] / abs(c[k]) ** 2)
        assert abs(g[0, m] - ref) < 1e-14 * (1 + ref)


def test_many_electron_flux_identity():
    """dP_K/dt of the occupied configuration under the frozen generator equals
    minus the summed raw hopping flux over all single excitations (sign of d,
    in-place candidate replacement and the ratio formula together)."""
    md = W.double_well_paper(9)
    B = O.bind(md)
    lam, Q, T, d, _ = O.eigen(B, 8.5)
    occ, C = _random_state(B, 9, weight=0.8)
    v = 0.02
    _, R, dS, _ = O.hop_probs(occ, C, d, v, 1.0)
    PK = abs(dS) ** 2
    raw = np.zeros_like(R)
    for a in range(B.Ne):
        for m in range(B.N):
            if m not in occ:
                raw[a, m] = -2 * v * R[a, m] * d[m, occ[a]]  # per unit time
    dPdt = -PK * raw.sum()
    h = 1e-3
    Cp = O.propagate(lam, d, v, lam, d, v, h, C)
    Cm = O.propagate(lam, d, v, lam, d, v, -h, C)
    fd = (abs(np.linalg.det(Cp[occ])) ** 2 - abs(np.linalg.det(Cm[occ])) ** 2) / (2 * h)
    assert abs(dPdt) > 1e-6
    assert abs(fd - dPdt) < 1e-6 * abs(dPdt)


# ------------------------------------------------------------- dynamics
def test_zero_coupling_never_hops():
    md = W.double_well(10, Gamma=0.0)
    B = O.bind(md)
    x, p = W.thermal_harmonic(4, md["mass"], md["par"][0], 0.01, seed=1)
    occ = np.tile(np.arange(B.Ne, dtype=np.int32), (4, 1))
    C = np.stack([O.unit_coefficients(B.N, o) for o in occ])
    out = O.run(B, x, p, occ, C, 1.0, 200, seed=3)
    assert np.all(out["hops"] == 0)
    assert np.abs(np.abs(out["C"]) - np.abs(C)).max() < 1e-12


def test_energy_conserved_across_hops():
    md = W.double_well_paper(12)
    md["Gamma"] = 0.02
    B = O.bind(md)
    occ, C = _random_state(B, 12, weight=1.5)
    x, p, dt = 8.0, 3.0, 10.0

    def energy(st_x, st_p, st_occ):
        lam = O.eigen(B, st_x)[0]
        return st_p ** 2 / (2 * md["mass"]) + O.model_eval(md, st_x)[0] + lam[st_occ].sum()

    E0 = energy(x, p, occ)
    hops = 0
    dEmax = dEhop = 0.0
    for n in range(400):
        r = O.step_one(B, x, p, occ, C, dt, seed=5, traj=0, n=n)
        E1 = energy(r["x"], r["p"], r["occ"])
        dEmax = max(dEmax, abs(E1 - E0))
        if r["hop"] == 1:
            hops += 1
            dEhop = max(dEhop, abs(E1 - E0))
        x, p, occ, C = r["x"], r["p"], r["occ"], r["C"]
        E0 = E1
    assert hops >= 2
    # per-step velocity-Verlet error here is ~1e-10; a wrong rescale would
    # leave an error of order of the orbital gap (~1e-3) at the hop steps
    assert dEmax < 1e-9 and dEhop < 1e-9


def test_canonical_occupation_sampler_matches_enumeration():
    lam = np.array([-0.3, -0.1, -0.05, 0.02, 0.1, 0.25])
    Ne, kT = 3, 0.1
    configs = list(itertools.combinations(range(6), Ne))
    wts = np.array([math.exp(-lam[list(c)].sum() / kT) for c in configs])
    prob = wts / wts.sum()
    ns = 20000
    counts = np.zeros(len(configs))
    for t in range(ns):
        occ = tuple(O.sample_occupations(17, t, lam, Ne, kT))
        counts[configs.index(occ)] += 1
    chi2 = np.sum((counts - ns * prob) ** 2 / (ns * prob))
    # 19 degrees of freedom: 5-sigma region
    assert chi2 < 19 + 5 * math.sqrt(2 * 19)
    assert list(O.sample_occupations(1, 0, lam, Ne, 0.0)) == [0, 1, 2]


def test_boltzmann_sampler_moments():
    m, w, kT = 2000.0, 0.002, 0.01
    xs = np.array([O.sample_nuclear(3, t, m, w, 0.0, kT) for t in range(20000)])
    sx, sp = math.sqrt(kT / (m * w * w)), math.sqrt(m * kT)
    assert abs(xs[:, 0].mean()) < 5 * sx / math.sqrt(len(xs))
    assert abs(xs[:, 0].std() / sx - 1) < 5 / math.sqrt(2 * len(xs))
    assert abs(xs[:, 1].std() / sp - 1) < 5 / math.sqrt(2 * len(xs))


def _wigner_moments(m, w, x_eq, kT, n, seed):
    """Sample variances of x and p from the oracle's Wigner branch."""
    xs = np.array([O.sample_nuclear(seed, t, m, w, x_eq, kT, wigner=True) for t in range(n)])
    return xs[:, 0].mean(), xs[:, 0].var(), xs[:, 1].var()


def test_wigner_sampler_printed_Q_at_300K():
    """Sec. III C: at 300 K the Wigner density of the m = 10.54 u Morse well is
    the classical Boltzmann density widened by Q ~ 1.9 (printed to two digits).
    The factor is read from the sampler's own variances, var(x) m w^2 / kT and
    var(p) / (m kT), with w from finite differences of the model's U0."""
    gold = {r[0]: (float(r[1]), float(r[2])) for r in _golden("desorption_model_pins.txt")}
    md = W.desorption(mass_u=10.54)
    x0, m = md["par"][1], md["mass"]
    hh = 1e-4
    w = math.sqrt((O.model_eval(md, x0 + hh)[1] - O.model_eval(md, x0 - hh)[1]) / (2 * hh) / m)
    kT = 300.0 * W.KB_HARTREE_PER_K
    n = 100000
    mean, vx, vp = _wigner_moments(m, w, x0, kT, n, 11)
    sig = math.sqrt(2.0 / n)  # relative standard error of a Gaussian sample variance
    val, tol = gold["wigner_Q_10p54u"]
    Qx = vx * m * w * w / kT
    Qp = vp / (m * kT)
    assert abs(Qx - val) < tol + 5 * sig * val, Qx
    assert abs(Qp - val) < tol + 5 * sig * val, Qp
    assert abs(mean - x0) < 5 * math.sqrt(vx / n)


def test_wigner_sampler_limits():
    """High temperature: the Wigner density becomes the classical Boltzmann
    density (Q -> 1).  Low temperature: it becomes the harmonic ground state,
    var(x) = 1 / (2 m w) and var(p) = m w / 2 (hbar = 1)."""
    m, w = 2000.0, 0.002
    n = 40000
    sig = 5 * math.sqrt(2.0 / n)
    kT = 200 * w  # Q = 1 + (w/kT)^2 / 12 + ... = 1.000002
    _, vx, vp = _wigner_moments(m, w, 0.0, kT, n, 12)
    assert abs(vx * m * w * w / kT - 1) < sig
    assert abs(vp / (m * kT) - 1) < sig
    kT = w / 60  # coth(30) = 1 to 1e-25
    _, vx, vp = _wigner_moments(m, w, 0.0, kT, n, 13)
    assert abs(vx * 2 * m * w - 1) < sig
    assert abs(vp * 2 / (m * w) - 1) < sig
    # between the limits the factor grows monotonically as kT falls
    qs = []
    for kT in (2 * w, w, 0.5 * w):
        _, vx, _ = _wigner_moments(m, w, 0.0, kT, n, 14)
        qs.append(vx * m * w * w / kT)
    assert qs[0] < qs[1] < qs[2]


# ------------------------------------------------------- occupied energy
def _eocc_dense(eps, sqw, wl, x, th):
    M = eps.shape[0]
    N = M + 2
    H = np.zeros((N, N))
    for a in range(2):
        H[a, a] = th[a] + th[2 + 6 * a: 8 + 6 * a] @ x
        r2 = np.sum((x[3 * a: 3 * a + 3] - wl["R"][3 * a: 3 * a + 3]) ** 2)
        V = wl["Vbar"][a] * sqw * math.exp(-0.5 * r2 / th[14 + a] ** 2)
        H[a, 2:] = H[2:, a] = V
    H[np.arange(2, N), np.arange(2, N)] = eps
    return np.linalg.eigvalsh(H)[: wl["Ne"]].sum()


def test_eocc_energy_and_gradients():
    wl = W.eocc_workload(M=24, B=3, seed=5)
    eps, sqw = O.bath(dict(band=wl["band"], M=wl["M"], mu=0.0, disc="gl"))
    E, dx, dth = O.eocc(eps, sqw, wl["Vbar"], wl["R"], wl["x"], wl["theta"], wl["Ne"])
    h = 1e-5
    for b in range(3):
        x, th = wl["x"][b], wl["theta"]
        assert abs(E[b] - _eocc_dense(eps, sqw, wl, x, th)) < 1e-13
        for y in range(6):
            e = np.zeros(6)
            e[y] = h
            fd = (_eocc_dense(eps, sqw, wl, x + e, th) - _eocc_dense(eps, sqw, wl, x - e, th)) / (2 * h)
            assert abs(dx[b, y] - fd) < 1e-8
        for y in range(16):
            e = np.zeros(16)
            e[y] = h
            fd = (_eocc_dense(eps, sqw, wl, x, th + e) - _eocc_dense(eps, sqw, wl, x, th - e)) / (2 * h)
            assert abs(dth[b, y] - fd) < 1e-8


# ------------------------------------------------- model definitions
def test_double_well_definition():
    """Sec. III B: U0 has its minimum 0 at x=0, U1 its minimum dG at x=g, both
    with curvature m w^2; h = U1 - U0 is linear in x."""
    md = W.double_well_paper(4)
    w, g, dG = md["par"]
    m = md["mass"]
    U0, dU0, h, dh, f, df = O.model_eval(md, 0.0)
    assert U0 == 0.0 and dU0 == 0.0
    out_g = O.model_eval(md, g)
    assert abs((out_g[0] + out_g[2]) - dG) < 1e-15  # U1(g) = dG
    assert abs(out_g[1] + out_g[3]) < 1e-15         # U1'(g) = 0
    hh = 1.0  # U1 is quadratic: the second difference is exact up to rounding
    curv1 = ((O.model_eval(md, g + hh)[0] + O.model_eval(md, g + hh)[2]) - 2 * dG
             + (O.model_eval(md, g - hh)[0] + O.model_eval(md, g - hh)[2])) / hh ** 2
    assert abs(curv1 - m * w * w) < 1e-9 * m * w * w
    hs = [O.model_eval(md, x)[2] for x in (-5.0, 0.0, 5.0)]
    assert abs((hs[2] - hs[1]) - (hs[1] - hs[0])) < 1e-15
    assert f == 1.0 and df == 0.0


def test_morse_image_definition():
    """Morse well of Table II, image-charge level h -> h_inf - 1/(4 (z - z_im))
    far from the surface, Gaussian coupling factor with f(z_c) = 1."""
    md = W.morse_image(10)
    De, x0, a, c, hinf, zim, ac, zc, sg = md["par"][:9]
    U0, dU0, h, dh, f, df = O.model_eval(md, x0)
    assert abs(U0 - c) < 1e-15 and abs(dU0) < 1e-15
    U0far = O.model_eval(md, 1e3)[0]
    assert abs(U0far - (De + c)) < 1e-12
    z = 400.0
    assert abs(O.model_eval(md, z)[2] - (hinf - 0.25 / (z - zim))) < 1e-7
    assert O.model_eval(md, zc)[4] == 1.0
    assert abs(O.model_eval(md, zc + sg)[4] - np.exp(-0.5)) < 1e-15


def test_hop_selection_frequencies():
    """Candidate J is chosen with probability g_J (Sec. II B), no hop with
    probability 1 - sum g, for a uniform zeta."""
    rng = np.random.default_rng(4)
    N, Ne = 6, 2
    occ = np.array([1, 4])
    g = np.zeros((Ne, N))
    for a in range(Ne):
        for m in range(N):
            if m not in occ:
                g[a, m] = rng.uniform(0.0, 0.08)
    trials = 40000
    counts = {}
    for _ in range(trials):
        r = O.select(occ, g, rng.uniform())
        counts[r] = counts.get(r, 0) + 1
    for a in range(Ne):
        for m in range(N):
            if g[a, m] > 0:
                p = g[a, m]
                assert abs(counts.get((a, m), 0) / trials - p) < 5 * math.sqrt(p * (1 - p) / trials)
    p0 = 1 - g.sum()
    assert abs(counts.get(None, 0) / trials - p0) < 5 * math.sqrt(p0 * (1 - p0) / trials)
    assert O.select(occ, g, 0.9999) is None


def test_population_invariants():
    """Impurity populations: with unit coefficients the wavefunction value
    equals the occupied-surface value; both lie in [0, 1]; with zero coupling
    they are 1 exactly when the impurity orbital is occupied."""
    md = W.double_well_paper(12)
    B = O.bind(md)
    x = np.array([8.0, 9.0])
    p = np.array([1.0, -2.0])
    occ = np.tile(np.arange(B.Ne, dtype=np.int32), (2, 1))
    C = np.stack([O.unit_coefficients(B.N, o) for o in occ])
    out = O.run(B, x, p, occ, C, 1e-9, 1, seed=0, record_every=1)
    assert np.allclose(out["pop_sh"], out["pop_wf"], atol=1e-12)
    assert np.all((out["pop_sh"] >= 0) & (out["pop_sh"] <= 1 + 1e-12))
    md0 = W.double_well_paper(12)
    md0["Gamma"] = 0.0
    B0 = O.bind(md0)
    lam, Q, _, _, _ = O.eigen(B0, 8.0)
    imp = int(np.argmax(np.abs(Q[0])))
    occ0 = np.array([[i for i in range(B0.N) if i != imp][: B0.Ne]], dtype=np.int32)
    occ1 = np.array([sorted([imp] + list(range(B0.Ne - 1 + (imp < B0.Ne - 1)))[:B0.Ne])],
                    dtype=np.int32)
    for o, want in ((occ0, 0.0), (occ1, 1.0)):
        Cu = O.unit_coefficients(B0.N, o[0])[None]
        r = O.run(B0, np.array([8.0]), np.array([0.0]), o, Cu, 1e-9, 1, seed=0, record_every=1)
        assert abs(r["pop_sh"][0, 0] - want) < 1e-12 and abs(r["pop_wf"][0, 0] - want) < 1e-12


# ------------------------------------------------------ two-orbital dynamics
def _two_energy(md, x, occ):
    lam = O.eigen2(md, x, occ)[0]
    u0 = 0.5 * md["mass"] * md["omega"] ** 2 * np.sum((x - md["x0"]) ** 2)
    return u0 + lam[occ].sum()


def test_two_orbital_force_is_minus_energy_gradient():
    md = W.two_orbital(12, seed=5)
    x, p, occ, C = W.two_orbital_state(md, 2, 3)
    for t in range(2):
        F = O.eigen2(md, x[t], occ[t])[3]
        h = 1e-5
        for a in range(6):
            e = np.zeros(6)
            e[a] = h
            fd = -(_two_energy(md, x[t] + e, occ[t]) - _two_energy(md, x[t] - e, occ[t])) / (2 * h)
            assert abs(F[a] - fd) < 1e-7 * max(1.0, abs(fd)), (a, F[a], fd)


def test_two_orbital_nac_matches_fd_of_eigenvectors():
    """d^a_jk = <j| d/dx_a k> in the gauge c1 Q_1j + c2 Q_2j > 0."""
    md = W.two_orbital(10, seed=6)
    x = W.two_orbital_state(md, 1, 4)[0][0]
    occ = np.arange(md["Ne"])
    lam, Q, d, _ = O.eigen2(md, x, occ)
    h = 1e-6
    for a in (0, 4):
        e = np.zeros(6)
        e[a] = h
        Qp = O.eigen2(md, x + e, occ)[1]
        Qm = O.eigen2(md, x - e, occ)[1]
        fd = Q.T @ (Qp - Qm) / (2 * h)
        gap = np.abs(lam[:, None] - lam[None, :]) + np.eye(len(lam))
        ok = gap > 1e-3  # well-separated pairs (FD of near-degenerate pairs is ill-conditioned)
        assert np.abs((fd - d[a])[ok]).max() < 1e-6 * max(1.0, np.abs(d[a][ok]).max())


def _two_c(md, x):
    """Coupling amplitudes c_a = vbar_a f_a(x), written out from the model."""
    th, R = md["theta"], md["R"]
    return np.array([md["Vbar"][a] * np.exp(-0.5 * np.sum((x[3 * a:3 * a + 3] - R[3 * a:3 * a + 3]) ** 2)
                                            / th[14 + a] ** 2) for a in range(2)])


def test_two_orbital_gauge_is_the_coupled_combination_and_continuous():
    """Eigenvector j is signed so that its component on the coupled
    combination c_0|0> + c_1|1> is positive, and that choice is continuous
    along a path: consecutive eigenvector matrices overlap with a positive
    diagonal near 1 (the convention d_jj = 0 of the NACs and the adiabatic
    coefficients rely on)."""
    md = W.two_orbital(12, seed=5)
    x0 = W.two_orbital_state(md, 1, 11)[0][0]
    occ = np.arange(md["Ne"])
    step = np.array([0.004, -0.003, 0.002, 0.003, 0.001, -0.004])
    Qprev = None
    for i in range(12):
        x = x0 + i * step
        lam, Q, _, _ = O.eigen2(md, x, occ)
        c = _two_c(md, x)
        assert np.all(c[0] * Q[0] + c[1] * Q[1] > 0)
        if Qprev is not None:
            assert np.all(np.diag(Qprev.T @ Q) > 0.9)
        Qprev = Q


def test_two_orbital_steps_conserve_energy_and_norm():
    """Velocity Verlet with hops rescaled along the NAC vector (strong
    coupling, many hops): the total energy U0 + sum_occ lam + p^2 / 2m stays
    within the Verlet error of the avoided crossings (the rescale itself is
    exact), and the coefficient columns stay orthonormal."""
    md = W.two_orbital(10, seed=7, vscale=1.0, omega=0.01)
    n, steps, dt = 6, 400, 2.5
    x, p, occ, C = W.two_orbital_state(md, n, 8, kT=0.01, weight=1.0)
    e0 = np.array([_two_energy(md, x[t], occ[t]) + (p[t] ** 2).sum() / (2 * md["mass"]) for t in range(n)])
    r = O.run2(md, x, p, occ, np.transpose(C, (0, 2, 1)), dt, steps, seed=2)
    e1 = np.array([_two_energy(md, r["x"][t], r["occ"][t]) + (r["p"][t] ** 2).sum() / (2 * md["mass"])
                   for t in range(n)])
    assert r["hops"].sum() > 0, "case must hop"
    assert np.abs(e1 - e0).max() < 2e-4 * np.abs(e0).max()
    for t in range(n):
        G = r["C"][t].conj().T @ r["C"][t]
        assert np.abs(G - np.eye(md["Ne"])).max() < 1e-10


def test_two_orbital_verlet_error_is_second_order():
    """Without coupling (no NAC, no hop; the occupied levels h_a(x) still
    drive the nuclei) the energy error after a fixed time falls as dt^2.  The
    impurity levels sit deep inside the occupied range, so the summed
    occupied energy has no kink (a level crossing the Fermi boundary would
    make the surface non-smooth)."""
    md = W.two_orbital(8, seed=11, vscale=0.0, omega=0.01)
    md["theta"] = md["theta"].copy()
    md["theta"][0:2] = [-0.30, -0.25]
    x, p, occ, C = W.two_orbital_state(md, 1, 12, kT=0.01, occ="lowest", weight=0.0)
    e0 = _two_energy(md, x[0], occ[0]) + (p[0] ** 2).sum() / (2 * md["mass"])
    errs = []
    for dt in (8.0, 4.0):
        r = O.run2(md, x, p, occ, np.transpose(C, (0, 2, 1)), dt, int(800 / dt), seed=1)
        assert r["hops"].sum() == 0
        e1 = _two_energy(md, r["x"][0], r["occ"][0]) + (r["p"][0] ** 2).sum() / (2 * md["mass"])
        errs.append(abs(e1 - e0))
    assert 2.5 < errs[0] / errs[1] < 6.0, errs


def test_two_orbital_zero_coupling_is_phase_only():
    md = W.two_orbital(8, seed=9, vscale=0.0)
    x, p, occ, C = W.two_orbital_state(md, 2, 10)
    r = O.run2(md, x, p, occ, np.transpose(C, (0, 2, 1)), 5.0, 10, seed=1)
    assert r["hops"].sum() == 0 and r["frustrated"].sum() == 0
    lam = O.eigen2(md, r["x"][0], r["occ"][0])[0]
    h = md["theta"][0:2] + np.array([md["theta"][2:8] @ r["x"][0], md["theta"][8:14] @ r["x"][0]])
    eps = O.bath(dict(band=md["band"], M=md["M"], mu=0.0, disc="gl"))[0]
    assert np.abs(np.sort(np.concatenate([h, eps])) - lam).max() < 1e-13
