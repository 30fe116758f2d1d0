"""Pins of the oracle's dense symmetric eigensolver and of the two-orbital
model with an own bath profile per adsorbate orbital (non-parallel border
vectors, reading R17), on the CPU.

What fixes them besides the oracle itself:
  - eigenpairs: LAPACK (numpy.linalg.eigh) on the same matrices;
  - the model's Hamiltonian: eigenvalues of an independently assembled H;
  - forces: central finite differences of the occupied energy (Hellmann-
    Feynman, Sec. II B);
  - nonadiabatic couplings: finite differences of the gauge-fixed
    eigenvectors (d_jk = <j|d_y k>, reading R1);
  - the gauge: continuity along a path (overlap of consecutive eigenvectors
    near +1);
  - the parallel limit: with flat profiles the model is the pinned
    two-orbital model of reading R16 and the runs agree;
  - energy conservation across hops.
"""
import math

import numpy as np

import iesh_inputs as W
from oracle import oracle as O


def _signed(V):
    """Rows of V signed so that the largest-magnitude entry is positive."""
    V = V.copy()
    for j in range(V.shape[0]):
        k = int(np.argmax(np.abs(V[j])))
        if V[j, k] < 0:
            V[j] = -V[j]
    return V


def test_dense_eigensolver_matches_lapack():
    for n, B in ((1, 2), (2, 3), (7, 4), (33, 3), (64, 2)):
        A = W.random_symmetric(B, n, seed=n)
        lam, V, rc = O.syev(A)
        assert rc == 0
        for b in range(B):
            w, U = np.linalg.eigh(A[b])
            scale = np.abs(w).max()
            assert np.abs(lam[b] - w).max() <= 1e-12 * scale
            assert np.abs(V[b] - _signed(U.T)).max() <= 1e-10
            # the definition: A v = lambda v for every row
            assert np.abs(A[b] @ V[b].T - V[b].T * lam[b]).max() <= 1e-11 * scale


def test_dense_eigensolver_degenerate_and_diagonal():
    A = np.diag([3.0, -1.0, 2.0, -1.0])[None]
    lam, V, rc = O.syev(A)
    assert rc == 0
    assert np.array_equal(lam[0], np.array([-1.0, -1.0, 2.0, 3.0]))
    assert np.allclose(np.abs(V[0] @ V[0].T), np.eye(4), atol=1e-14)


def _H(md, x):
    """Independent assembly of the own-profile two-orbital Hamiltonian."""
    eps, sqw = O.bath(dict(band=md["band"], M=md["M"], mu=0.0, disc="gl"))
    M, N = md["M"], md["M"] + 2
    th = md["theta"]
    H = np.zeros((N, N))
    for a in range(2):
        H[a, a] = th[a] + np.dot(th[2 + 6 * a: 8 + 6 * a], x)
        r2 = np.sum((x[3 * a: 3 * a + 3] - md["R"][3 * a: 3 * a + 3]) ** 2)
        f = math.exp(-0.5 * r2 / th[14 + a] ** 2)
        lor = 1.0 / np.sqrt(1.0 + ((eps - md["profile"]["center"][a]) / md["profile"]["width"][a]) ** 2)
        H[a, 2:] = H[2:, a] = md["Vbar"][a] * sqw * lor * f
    H[np.arange(2, N), np.arange(2, N)] = eps
    return H


def _occ_energy(md, x, occ):
    U0 = 0.5 * md["mass"] * md["omega"] ** 2 * np.sum((x - md["x0"]) ** 2)
    return U0 + np.linalg.eigvalsh(_H(md, x))[occ].sum()


def test_profiled_model_is_not_parallel_and_flat_profile_is():
    md = W.two_orbital_profiled(20, seed=5)
    eps, sqw = O.bath(dict(band=md["band"], M=md["M"], mu=0.0, disc="gl"))
    V = O.two_couplings(md, eps, sqw)
    cos = abs(V[0] @ V[1]) / (np.linalg.norm(V[0]) * np.linalg.norm(V[1]))
    assert cos < 0.95
    flat = dict(md, profile=dict(center=[0.0, 0.0], width=[1e30, 1e30]))
    V = O.two_couplings(flat, eps, sqw)
    assert np.allclose(V, np.vstack([md["Vbar"][0] * sqw, md["Vbar"][1] * sqw]), rtol=1e-15)


def test_profiled_eigenpairs_forces_and_nac():
    md = W.two_orbital_profiled(16, seed=5)
    N, Ne = md["M"] + 2, md["Ne"]
    x, p, occ, C = W.two_orbital_state(md, 2, 3, kT=0.01)
    for t in range(2):
        lam, Q, d, F = O.eigen2(md, x[t], occ[t])
        H = _H(md, x[t])
        w = np.linalg.eigvalsh(H)
        assert np.abs(lam - w).max() <= 1e-12 * np.abs(w).max()
        assert np.abs(H @ Q - Q * lam).max() <= 1e-12 * np.abs(w).max()
        assert np.abs(Q.T @ Q - np.eye(N)).max() <= 1e-12
        h = 1e-5
        for y in range(6):
            e = np.zeros(6)
            e[y] = h
            fd = -(_occ_energy(md, x[t] + e, occ[t]) - _occ_energy(md, x[t] - e, occ[t])) / (2 * h)
            assert abs(F[y] - fd) <= 1e-7 * (1 + abs(fd)), (y, F[y], fd)
            # d_jk = <j| d_y k> from the eigenvectors at x +- h, signed by
            # overlap with those at x
            _, Qp, _, _ = O.eigen2(md, x[t] + e, occ[t], Qref=Q)
            _, Qm, _, _ = O.eigen2(md, x[t] - e, occ[t], Qref=Q)
            dfd = Q.T @ (Qp - Qm) / (2 * h)
            gaps = np.abs(lam[:, None] - lam[None, :])
            ok = gaps > 1e-3 * np.abs(lam).max()  # finite differences resolve these pairs
            err = np.abs(d[y] - dfd)[ok].max()
            assert err <= 1e-6 * max(1.0, np.abs(d[y][ok]).max()), (y, err)
            assert np.abs(d[y] + d[y].T).max() <= 1e-9 * max(1.0, np.abs(d[y]).max())


def test_profiled_gauge_is_continuous_along_a_path():
    md = W.two_orbital_profiled(16, seed=5)
    x, _, occ, _ = W.two_orbital_state(md, 1, 7, kT=0.01)
    direction = np.random.default_rng(2).standard_normal(6)
    direction /= np.linalg.norm(direction)
    _, Q, _, _ = O.eigen2(md, x[0], occ[0])
    for s in range(1, 60):
        _, Qn, _, _ = O.eigen2(md, x[0] + 0.02 * s * direction, occ[0], Qref=Q)
        ov = np.einsum("rj,rj->j", Q, Qn)
        assert ov.min() > 0.9, (s, ov.min())
        Q = Qn


def test_flat_profiles_reproduce_the_parallel_model_run():
    md = W.two_orbital(12, seed=5)
    md["Vbar"] = 3.0 * np.asarray(md["Vbar"])
    flat = dict(md, profile=dict(center=[0.0, 0.0], width=[1e30, 1e30]))
    x, p, occ, C = W.two_orbital_state(md, 3, 11, kT=0.01, weight=0.8)
    Ct = np.transpose(C, (0, 2, 1))
    a = O.run2(md, x, p, occ, Ct, 2.0, 40, 5)
    b = O.run2(flat, x, p, occ, Ct, 2.0, 40, 5)
    assert np.array_equal(a["occ"], b["occ"]) and np.array_equal(a["hops"], b["hops"])
    assert np.abs(a["x"] - b["x"]).max() <= 1e-12 * np.abs(a["x"]).max()
    assert np.abs(a["C"] - b["C"]).max() <= 1e-10


def test_profiled_run_conserves_energy_through_hops():
    md = W.two_orbital_profiled(12, seed=5)
    md["Vbar"] = 4.0 * np.asarray(md["Vbar"])
    n = 6
    x, p, occ, C = W.two_orbital_state(md, n, 21, kT=0.02, weight=1.0)
    # dt = 0.5: the velocity-Verlet fluctuation (about 1e-6 here, O(dt^2)) stays
    # far below the orbital gaps (~1e-2) that a wrong rescale would leave
    r = O.run2(md, x, p, occ, np.transpose(C, (0, 2, 1)), 0.5, 600, 9)
    assert r["hops"].sum() > 0, "case must hop"
    for t in range(n):
        E0 = _occ_energy(md, x[t], occ[t]) + np.sum(p[t] ** 2) / (2 * md["mass"])
        E1 = _occ_energy(md, r["x"][t], r["occ"][t]) + np.sum(r["p"][t] ** 2) / (2 * md["mass"])
        assert abs(E1 - E0) <= 5e-6, (t, E0, E1)
    # unitary propagation: orthonormal coefficient columns
    for t in range(n):
        G = r["C"][t].conj().T @ r["C"][t]
        assert np.abs(G - np.eye(md["Ne"])).max() <= 1e-9


def test_continuity_gauge_through_a_level_crossing():
    """Parallel couplings (reading R16), a straight path on which the two
    adsorbate levels cross (h_0 = h_1, where the coupling t of |-> to |+>
    vanishes): the R16 sign rule alone flips the |->-like eigenvector, the
    continuity gauge used after set-up (reading R17) keeps every overlap of
    consecutive eigenvectors near +1, and a run across the crossing agrees
    with the flat-profile model, which always signs by continuity."""
    md = W.two_orbital(40, seed=6, vscale=1.0)
    x, p, occ, C = W.two_orbital_state(md, 6, 31, weight=0.8)
    th = md["theta"]
    r = O.run2(md, x, p, occ, np.transpose(C, (0, 2, 1)), 2.0, 1, 2)
    x0, x1 = r["x"][3], O.run2(md, x, p, occ, np.transpose(C, (0, 2, 1)), 2.0, 2, 2)["x"][3]
    dh = lambda y: th[0] + th[2:8] @ y - th[1] - th[8:14] @ y
    assert dh(x0) * dh(x1) < 0, "the path must cross h_0 = h_1"
    flat = dict(md, profile=dict(center=[0.0, 0.0], width=[1e30, 1e30]))
    _, Qa, _, _ = O.eigen2(flat, x0, occ[3])
    _, Qr, _, _ = O.eigen2(md, x1, occ[3])  # R16 rule alone at x1
    _, Qc, _, _ = O.eigen2(flat, x1, occ[3], Qref=Qa)  # continuity
    assert np.einsum("rj,rj->j", Qa, Qr).min() < -0.9
    assert np.einsum("rj,rj->j", Qa, Qc).min() > 0.9
    Ct = np.transpose(C, (0, 2, 1))
    a = O.run2(md, x, p, occ, Ct, 2.0, 20, 2)
    b = O.run2(flat, x, p, occ, Ct, 2.0, 20, 2)
    assert np.array_equal(a["occ"], b["occ"])
    assert np.abs(a["C"] - b["C"]).max() <= 1e-10
