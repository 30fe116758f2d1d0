"""GPU parity of the two-orbital, six-coordinate IESH dynamics (iesh2_*)
with the FP64 oracle (dense Jacobi eigenpairs, T^y = Q^T dH/dy Q by
matrix products, the same step in six dimensions).

The GPU path takes the eigenpairs from the rank-two arrowhead's secular
equation (one extra pole at h_-) and the couplings from their closed form,
so agreement checks the reduction as well as the kernels.  Tolerances are
those of the one-coordinate FP64 path: eigenvalues 1e-12 (the band is
[-0.5, 0.5]), components 1e-11, forces 1e-10 relative; per step 1e-10 on C;
over 100 steps with hops 1e-9 on C and identical occupations and hop
counts."""
import numpy as np
import pytest

import iesh_inputs as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_2212_00518_gb300 import build as B
    B.build()
    from paper_2212_00518_gb300 import two
    return two


def _ctx(P, md, x, p, occ, C, **kw):
    ctx = P.TwoOrbitalContext(md, x.shape[0], **kw)
    ctx.set_state(x, p, occ.astype(np.int16), C)
    return ctx


def _one_coupling(M):
    md = W.two_orbital(M, seed=5)
    md["Vbar"] = np.array([md["Vbar"][0], 0.0])
    return md


CASES = {
    "M12": W.two_orbital(12, seed=5),
    "M40": W.two_orbital(40, seed=6),
    "M100": W.two_orbital(100, seed=7, Ne=48),
    "strong": W.two_orbital(16, seed=7, vscale=3.0),
    "one_coupling": _one_coupling(20),
    "no_coupling": W.two_orbital(20, seed=9, vscale=0.0),
}


@pytest.mark.parametrize("name", list(CASES))
def test_eigenpairs_and_forces(P, name):
    md = CASES[name]
    n = 5
    x, p, occ, C = W.two_orbital_state(md, n, 11)
    ctx = _ctx(P, md, x, p, occ, C)
    lam, Q, F = ctx.eigen()
    assert np.all(ctx.get_state()["status"] == 0)
    for t in range(n):
        rl, rQ, _, rF = O.eigen2(md, x[t], occ[t])
        assert np.abs(lam[t] - rl).max() <= 1e-12
        assert np.abs(Q[t] - rQ[0:2]).max() <= 1e-11
        assert np.abs(F[t] - rF).max() <= 1e-10 * max(1.0, np.abs(rF).max())


@pytest.mark.parametrize("name", ["M12", "M40", "strong", "one_coupling"])
def test_hop_probabilities(P, name):
    """g_{a->m} with v . d at the state's velocity, against the oracle's
    determinant ratios with the velocity-projected NAC matrix."""
    md = CASES[name]
    n, dt = 4, 20.0
    x, p, occ, C = W.two_orbital_state(md, n, 13, weight=0.6)
    ctx = _ctx(P, md, x, p, occ, C)
    g = ctx.hop_probabilities(dt)
    for t in range(n):
        d = O.eigen2(md, x[t], occ[t])[2]
        dv = np.tensordot(p[t] / md["mass"], d, axes=1)
        gref = O.hop_probs(occ[t], C[t].T, dv, 1.0, dt)[0]
        assert np.abs(gref).max() > 0
        assert np.abs(g[t] - gref).max() <= 1e-10 * np.abs(gref).max()


@pytest.mark.parametrize("name", list(CASES))
def test_one_step(P, name):
    md = CASES[name]
    n, dt = 6, 5.0
    x, p, occ, C = W.two_orbital_state(md, n, 17, weight=0.6)
    ctx = _ctx(P, md, x, p, occ, C)
    ctx.run(dt, 1, seed=3)
    st = ctx.get_state()
    ref = O.run2(md, x, p, occ, np.transpose(C, (0, 2, 1)), dt, 1, seed=3)
    assert np.all(st["status"] == 0)
    assert np.array_equal(st["occ"], ref["occ"])
    assert np.abs(st["x"] - ref["x"]).max() <= 1e-12 * (1 + np.abs(ref["x"]).max())
    assert np.abs(st["p"] - ref["p"]).max() <= 1e-11 * (1 + np.abs(ref["p"]).max())
    assert np.abs(np.transpose(st["C"], (0, 2, 1)) - ref["C"]).max() <= 1e-10


@pytest.mark.parametrize("name", ["M12", "strong", "one_coupling"])
def test_100_steps_with_hops(P, name):
    """Trajectories with hops (strong coupling, large coefficients off the
    occupied set): identical occupations and hop counts, and C, x, p within
    the FP64 tolerance after 100 steps."""
    md = CASES[name]
    n, steps, dt = 8, 100, 5.0
    x, p, occ, C = W.two_orbital_state(md, n, 19, kT=0.01, weight=1.0)
    ctx = _ctx(P, md, x, p, occ, C)
    ctx.run(dt, steps, seed=5)
    st = ctx.get_state()
    ns, hops, frus = ctx.counters()
    ref = O.run2(md, x, p, occ, np.transpose(C, (0, 2, 1)), dt, steps, seed=5)
    assert ref["hops"].sum() > 0, "case must hop"
    assert np.all(ns == steps)
    assert np.array_equal(st["occ"], ref["occ"])
    assert np.array_equal(hops, ref["hops"].astype(np.int32))
    assert np.array_equal(frus, ref["frustrated"].astype(np.int32))
    assert np.abs(st["x"] - ref["x"]).max() <= 1e-10 * np.abs(ref["x"]).max()
    assert np.abs(st["p"] - ref["p"]).max() <= 1e-9 * np.abs(ref["p"]).max()
    assert np.abs(np.transpose(st["C"], (0, 2, 1)) - ref["C"]).max() <= 1e-9
    lam, _, F = ctx.eigen()
    assert np.abs(F - ref["F"]).max() <= 1e-9 * np.abs(ref["F"]).max()
    assert np.abs(lam - ref["lam"]).max() <= 1e-11


def test_empty_batch(P):
    md = CASES["M12"]
    N = md["M"] + 2
    ctx = P.TwoOrbitalContext(md, 4)
    z = np.zeros((0, 6))
    ctx.set_state(z, z, np.zeros((0, md["Ne"]), np.int16), np.zeros((0, md["Ne"], N), np.complex128))
    ctx.run(5.0, 3, seed=1)
    assert ctx.get_state()["x"].shape == (0, 6)


def test_energy_conserved_with_hops_on_gpu(P):
    """Energy U0 + sum_occ lam + |p|^2 / 2m over 400 steps of a strongly
    coupled batch: the rescale is exact and the Verlet error small; the
    coefficient columns stay orthonormal."""
    md = W.two_orbital(16, seed=7, vscale=3.0)
    n, steps, dt = 64, 400, 2.0
    x, p, occ, C = W.two_orbital_state(md, n, 23, kT=0.01, weight=1.0)
    ctx = _ctx(P, md, x, p, occ, C)

    def energy():
        st = ctx.get_state()
        lam = ctx.eigen()[0]
        u0 = 0.5 * md["mass"] * md["omega"] ** 2 * ((st["x"] - md["x0"]) ** 2).sum(1)
        return u0 + np.take_along_axis(lam, st["occ"].astype(np.int64), 1).sum(1) + \
            (st["p"] ** 2).sum(1) / (2 * md["mass"])

    e0 = energy()
    ctx.run(dt, steps, seed=9)
    e1 = energy()
    assert ctx.counters()[1].sum() > 0
    assert np.abs(e1 - e0).max() < 1e-3 * np.abs(e0).max()
    Cn = ctx.get_state()["C"]
    G = np.einsum("tei,tfi->tef", Cn.conj(), Cn)
    assert np.abs(G - np.eye(md["Ne"])[None]).max() < 1e-10


# ------------------------------------------------------------ mixed precision
# FP64 eigenpairs, forces, probabilities and rescale; FP32 coefficients,
# generator, propagation (3xTF32 tensor cores for N <= 128, Ne <= 56) and
# overlap LU.  Bounds as for the one-coordinate mixed path.
def _mixed(P, md, x, p, occ, C):
    C32 = C.astype(np.complex64)
    ctx = _ctx(P, md, x, p, occ, C32, precision=1)
    return ctx, C32.astype(np.complex128)


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_eigenpairs_and_forces(P, name):
    """The mixed path's secular sums over the bath poles run in double-float
    (about 48 bits): eigenvalues within 1e-12 of the band, components 1e-11,
    forces 1e-10 relative."""
    md = CASES[name]
    n = 5
    x, p, occ, C = W.two_orbital_state(md, n, 11)
    ctx, _ = _mixed(P, md, x, p, occ, C)
    ctx.run(2.0, 3, seed=1)  # warm-started roots as well
    st = ctx.get_state()
    lam, Q, F = ctx.eigen()
    assert np.all(st["status"] == 0)
    for t in range(n):
        rl, rQ, _, rF = O.eigen2(md, st["x"][t], st["occ"][t])
        assert np.abs(lam[t] - rl).max() <= 1e-12
        assert np.abs(Q[t] - rQ[0:2]).max() <= 1e-11
        assert np.abs(F[t] - rF).max() <= 1e-10 * max(1.0, np.abs(rF).max())


@pytest.mark.parametrize("name", ["M12", "M40", "strong", "one_coupling"])
def test_mixed_hop_probabilities(P, name):
    md = CASES[name]
    n, dt = 4, 20.0
    x, p, occ, C = W.two_orbital_state(md, n, 13, weight=0.6)
    ctx, Cr = _mixed(P, md, x, p, occ, C)
    g = ctx.hop_probabilities(dt)
    for t in range(n):
        d = O.eigen2(md, x[t], occ[t])[2]
        dv = np.tensordot(p[t] / md["mass"], d, axes=1)
        gref = O.hop_probs(occ[t], Cr[t].T, dv, 1.0, dt)[0]
        assert np.abs(g[t] - gref).max() <= 2e-6 * np.abs(gref).max()


@pytest.mark.parametrize("name", ["M12", "M40", "M100", "strong", "one_coupling", "no_coupling"])
def test_mixed_one_step(P, name):
    md = CASES[name]
    n, dt = 6, 5.0
    x, p, occ, C = W.two_orbital_state(md, n, 17, weight=0.6)
    ctx, Cr = _mixed(P, md, x, p, occ, C)
    ctx.run(dt, 1, seed=3)
    st = ctx.get_state()
    ref = O.run2(md, x, p, occ, np.transpose(Cr, (0, 2, 1)), dt, 1, seed=3)
    assert np.all(st["status"] == 0)
    assert np.array_equal(st["occ"], ref["occ"])
    assert np.abs(st["x"] - ref["x"]).max() <= 1e-12 * (1 + np.abs(ref["x"]).max())
    assert np.abs(st["p"] - ref["p"]).max() <= 1e-11 * (1 + np.abs(ref["p"]).max())
    assert np.abs(np.transpose(st["C"], (0, 2, 1)) - ref["C"]).max() <= 1e-6


@pytest.mark.parametrize("name", ["M12", "strong"])
def test_mixed_100_steps(P, name):
    """Hop decisions agree unless a uniform falls within the FP32 error of a
    cumulative boundary: at least 7 of 8 trajectories identical; on those, C
    within 3e-5 after 100 steps."""
    md = CASES[name]
    n, steps, dt = 8, 100, 5.0
    x, p, occ, C = W.two_orbital_state(md, n, 19, kT=0.01, weight=1.0)
    ctx, Cr = _mixed(P, md, x, p, occ, C)
    ctx.run(dt, steps, seed=5)
    st = ctx.get_state()
    _, hops, _ = ctx.counters()
    ref = O.run2(md, x, p, occ, np.transpose(Cr, (0, 2, 1)), dt, steps, seed=5)
    assert ref["hops"].sum() > 0
    same = [t for t in range(n) if np.array_equal(st["occ"][t], ref["occ"][t]) and hops[t] == ref["hops"][t]]
    assert len(same) >= n - 1
    Cg = np.transpose(st["C"], (0, 2, 1))
    assert np.abs(Cg[same] - ref["C"][same]).max() <= 3e-5
    assert np.abs(st["x"][same] - ref["x"][same]).max() <= 1e-6 * np.abs(ref["x"]).max()


def test_mixed_large_system_shared_rows_and_simt(P):
    """N = 142 orbitals, Ne = 71: past the register Gauss-Jordan kernel and
    the tensor-core propagator, so the mixed path runs the Gauss-Jordan
    kernel with the rows past 128 in shared memory (its six-coordinate
    variant) and the SIMT FP32 propagator; one step against the oracle."""
    md = W.two_orbital(140, seed=8, Ne=71)
    n, dt = 4, 5.0
    x, p, occ, C = W.two_orbital_state(md, n, 29, weight=0.6)
    ctx, Cr = _mixed(P, md, x, p, occ, C)
    g = ctx.hop_probabilities(dt)
    for t in range(n):
        d = O.eigen2(md, x[t], occ[t])[2]
        dv = np.tensordot(p[t] / md["mass"], d, axes=1)
        gref = O.hop_probs(occ[t], Cr[t].T, dv, 1.0, dt)[0]
        assert np.abs(g[t] - gref).max() <= 2e-6 * np.abs(gref).max()
    ctx.run(dt, 1, seed=3)
    st = ctx.get_state()
    ref = O.run2(md, x, p, occ, np.transpose(Cr, (0, 2, 1)), dt, 1, seed=3)
    assert np.all(st["status"] == 0)
    assert np.array_equal(st["occ"], ref["occ"])
    assert np.abs(np.transpose(st["C"], (0, 2, 1)) - ref["C"]).max() <= 1e-6
