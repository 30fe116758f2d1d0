"""GPU checks of the deflated propagators.

When the top eigenvalue of the step's generator lies apart from the rest of
the spectrum (Gershgorin discs and interlacing), the Chebyshev series of
exp(-i dt Abar) (Sec. II C) runs over the bulk interval only, from c - a u
(a = u^H c), and the component along the isolated eigenvector is propagated
exactly.  Both forms compute the same exponential to within the series
tolerance (1e-15 per step in FP64), so:
  - a deflating context and one with deflation off agree to 1e-12 in C per
    step and take identical hop decisions;
  - trajectories whose series length did not change took the plain path and
    give identical bits;
  - on the double well (adsorbate level above the band) the series is at
    least two terms shorter for every trajectory;
  - the deflated path matches the oracle's one-step propagation to 1e-12;
  - every FP64 propagator shape gives the same bits (the start value and the
    end term are formed per entry, in a fixed order).
The mixed path's kernels are held to its one-step bound (C 1e-6).
"""
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
    import paper_2212_00518_gb300 as pkg
    return pkg


def _state(md, n, seed):
    N = md["M"] + 1
    kT = np.array([0.005, 0.0075, 0.01])[np.arange(n) % 3]
    x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], kT, seed=seed)
    occ = W.lowest_occupations(n, md["Ne"])
    C = W.mixed_coefficients(occ, N, seed + 1, 0.3)
    return x, p, occ, C


def _pair(P, md, n, x, p, occ, C, steps, seed=0):
    out = []
    for defl in (True, False):
        ctx = P.Context(md, n, deflation=defl)
        ctx.set_state(x, p, occ, C)
        ctx.run(1.0, steps, seed=seed)
        st = ctx.get_state()
        st["K"] = np.asarray(ctx.propagator_terms()).copy()
        st["hops"] = ctx.counters()[1]
        ctx.close()
        out.append(st)
    return out


@pytest.mark.parametrize("M", [100, 200])
def test_double_well_series_shorter_and_same_dynamics(P, M):
    md = W.double_well(M)
    n = 256
    x, p, occ, C = _state(md, n, 7 + M)
    d1, f1 = _pair(P, md, n, x, p, occ, C, 1)
    assert np.all(d1["status"] == 0) and np.all(f1["status"] == 0)
    assert np.all(d1["K"] <= f1["K"] - 2), (d1["K"].max(), f1["K"].min())
    assert np.array_equal(d1["occ"], f1["occ"])
    assert np.abs(d1["C"] - f1["C"]).max() <= 1e-12
    d, f = _pair(P, md, n, x, p, occ, C, 30, seed=3)
    assert np.array_equal(d["occ"], f["occ"]) and np.array_equal(d["hops"], f["hops"])
    assert np.abs(d["x"] - f["x"]).max() <= 1e-11 * (np.abs(f["x"]).max() + 1.0)
    assert np.abs(d["p"] - f["p"]).max() <= 1e-11 * np.abs(f["p"]).max()
    assert np.abs(d["C"] - f["C"]).max() <= 30e-12


def test_deflated_step_matches_oracle(P):
    md = W.double_well(100)
    n = 64
    x, p, occ, C = _state(md, n, 19)
    ctx = P.Context(md, n)
    ctx.set_state(x, p, occ, C)
    ctx.run(1.0, 1, seed=0)
    st = ctx.get_state()
    K = ctx.propagator_terms()
    ctx.close()
    assert K.max() <= 10
    B = O.bind(md)
    for t in (0, 1, 17, 40, 63):
        r = O.step_one(B, x[t], p[t], occ[t].astype(np.int32), C[t].T, 1.0, seed=0, traj=t, n=0)
        assert np.array_equal(st["occ"][t], r["occ"]), t
        assert abs(st["x"][t] - r["x"]) <= 1e-13 * (abs(r["x"]) + 1.0), t
        assert abs(st["p"][t] - r["p"]) <= 1e-10 * (abs(r["p"]) + 1e-3), t
        assert np.abs(st["C"][t].T - r["C"]).max() <= 1e-12, t


def test_unchanged_series_length_gives_identical_bits(P):
    """A wide band (the desorption model, 64 eV) puts the adsorbate level
    inside the spectrum's hull at most positions: where the deflated series
    is not shorter the plain path runs, bit for bit."""
    md = W.desorption(M=100)
    n = 128
    N = md["M"] + 1
    rng = np.random.default_rng(5)
    x = md["par"][1] + 0.2 * rng.standard_normal(n)
    p = 2.0 * rng.standard_normal(n)
    occ = W.lowest_occupations(n, md["Ne"])
    C = W.mixed_coefficients(occ, N, 6, 0.3)
    d, f = _pair(P, md, n, x, p, occ, C, 1)
    same = d["K"] == f["K"]
    assert np.all(d["K"] <= f["K"])
    assert np.all((~same) <= (d["K"] <= f["K"] - 2))
    assert np.array_equal(d["C"][same], f["C"][same])
    assert np.abs(d["C"] - f["C"]).max() <= 1e-12


def test_every_shape_gives_the_same_bits(P):
    from paper_2212_00518_gb300 import tuning
    md = W.double_well(60)
    n = 48
    x, p, occ, C = _state(md, n, 23)
    ref = None
    for ept, G in tuning.cheb_candidates(md["M"] + 1, md["Ne"], precision=P.PREC_FP64):
        ctx = P.Context(md, n)
        ctx.set_kernel_shape(ept, G, 0)
        ctx.set_state(x, p, occ, C)
        ctx.run(1.0, 3, seed=1)
        Cs = ctx.get_state()["C"]
        assert ctx.propagator_terms().max() <= 10
        ctx.close()
        if ref is None:
            ref = Cs
        assert np.array_equal(Cs, ref), (ept, G)


def _pair_mixed(P, md, n, x, p, occ, C, steps, shape=None, seed=0):
    out = []
    for defl in (True, False):
        ctx = P.Context(md, n, precision=P.PREC_MIXED, deflation=defl)
        if shape:
            ctx.set_kernel_shape(*shape, 0)
        ctx.set_state(x, p, occ, C.astype(np.complex64))
        ctx.run(1.0, steps, seed=seed)
        st = ctx.get_state()
        st["K"] = np.asarray(ctx.propagator_terms()).copy()
        st["hops"] = ctx.counters()[1]
        ctx.close()
        out.append(st)
    return out


@pytest.mark.parametrize("M,shape", [(200, None), (100, (4, 3)), (100, (32, 2))])
def test_mixed_deflation(P, M, shape):
    """The SIMT propagator (the default at M = 200, shapes 4 and 32) deflates
    with the FP32 eigenvector: the series is at least two terms shorter (or,
    where the FP32 iteration does not reach its residual, unchanged), the
    step agrees with the plain series within the mixed path's one-step bound
    (C 1e-6) and with the oracle's FP64 step within the same bound."""
    md = W.double_well(M)
    n = 128
    x, p, occ, C = _state(md, n, 29 + M)
    d, f = _pair_mixed(P, md, n, x, p, occ, C, 1, shape)
    assert np.all(d["status"] == 0) and np.all(f["status"] == 0)
    shorter = d["K"] <= f["K"] - 2
    assert np.all(shorter | (d["K"] == f["K"]))
    assert shorter.mean() >= 0.95, shorter.mean()
    assert np.array_equal(d["occ"], f["occ"])
    assert np.abs(d["C"] - f["C"]).max() <= 1e-6
    B = O.bind(md)
    C32 = C.astype(np.complex64).astype(np.complex128)
    for t in (0, 5, 64, 127):
        r = O.step_one(B, x[t], p[t], occ[t].astype(np.int32), C32[t].T, 1.0, seed=0, traj=t, n=0)
        assert np.array_equal(d["occ"][t], r["occ"]), t
        assert np.abs(d["C"][t].T - r["C"]).max() <= 1e-6, t


def test_mixed_deflation_many_steps(P):
    """30 steps: deflated and plain mixed runs take the same hops and stay
    within the accumulated bound (30 x 1e-6)."""
    md = W.double_well(200)
    n = 256
    x, p, occ, C = _state(md, n, 71)
    d, f = _pair_mixed(P, md, n, x, p, occ, C, 30, seed=2)
    assert np.array_equal(d["occ"], f["occ"]) and np.array_equal(d["hops"], f["hops"])
    assert np.abs(d["C"] - f["C"]).max() <= 30e-6
    assert np.abs(d["p"] - f["p"]).max() <= 1e-5 * np.abs(f["p"]).max()


@pytest.mark.parametrize("shape", [None, (8, 1)])
def test_tensor_core_paths_do_not_deflate(P, shape):
    """The tensor-core propagators (FP16 split, the default at M = 100;
    3xTF32, shape 8) keep the full interval: deflating and plain contexts
    take the same series and give the same bits."""
    md = W.double_well(100)
    n = 64
    x, p, occ, C = _state(md, n, 83)
    d, f = _pair_mixed(P, md, n, x, p, occ, C, 2, shape)
    assert np.array_equal(d["K"], f["K"])
    assert np.array_equal(d["C"], f["C"])


def _dt_pair(P, md, n, x, p, occ, C, dt, precision, shape=None):
    out = []
    for defl in (True, False):
        ctx = P.Context(md, n, precision=precision, deflation=defl)
        if shape:
            ctx.set_kernel_shape(*shape, 0)
        ctx.set_state(x, p, occ, C if precision == P.PREC_FP64 else C.astype(np.complex64))
        ctx.run(dt, 1, seed=0)
        st = ctx.get_state()
        st["K"] = np.asarray(ctx.propagator_terms()).copy()
        ctx.close()
        out.append(st)
    return out


def test_amplification_guard(P):
    """With a long time step the bulk series amplifies the u direction by
    |J_0| + 2 sum |J_k| |T_k(mu_x)| (about 50 at dt = 3, 3e4 at dt = 8 on the
    double well): FP64 deflates at dt = 3 (bound 1e3) and keeps the full
    interval at dt = 8, bit for bit; the FP32 SIMT path keeps it at dt = 3
    (bound 16)."""
    md = W.double_well(100)
    n = 32
    x, p, occ, C = _state(md, n, 91)
    d, f = _dt_pair(P, md, n, x, p, occ, C, 3.0, P.PREC_FP64)
    assert np.all(d["K"] <= f["K"] - 2)
    assert np.abs(d["C"] - f["C"]).max() <= 1e-12
    d, f = _dt_pair(P, md, n, x, p, occ, C, 8.0, P.PREC_FP64)
    assert np.array_equal(d["K"], f["K"]) and np.array_equal(d["C"], f["C"])
    d, f = _dt_pair(P, md, n, x, p, occ, C, 3.0, P.PREC_MIXED, shape=(4, 3))
    assert np.array_equal(d["K"], f["K"]) and np.array_equal(d["C"], f["C"])


@pytest.mark.parametrize("precision,shape", [(0, None), (1, (4, 3))])
def test_resume_is_bit_exact_while_deflating(P, precision, shape):
    """The deflation record is rebuilt every step from the state, so a run
    split by a checkpoint gives the same bits as the undivided run."""
    md = W.double_well(100)
    n = 48
    x, p, occ, C = _state(md, n, 97)
    C = C if precision == P.PREC_FP64 else C.astype(np.complex64)

    def ctx():
        c = P.Context(md, n, precision=precision)
        if shape:
            c.set_kernel_shape(*shape, 0)
        return c

    a = ctx()
    a.set_state(x, p, occ, C)
    a.run(1.0, 8, seed=4)
    ref = a.get_state()
    assert a.propagator_terms().max() <= (10 if precision == 0 else 6)
    a.close()
    b = ctx()
    b.set_state(x, p, occ, C)
    b.run(1.0, 4, seed=4)
    blob = b.checkpoint_save()
    b.close()
    c = ctx()
    c.checkpoint_load(blob)
    c.run(1.0, 4, seed=4)
    st = c.get_state()
    c.close()
    for k in ("x", "p", "occ", "C", "status"):
        assert np.array_equal(st[k], ref[k]), k
