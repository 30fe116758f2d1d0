"""GPU (sm_103a) parity of the FP64 CUDA path with the FP64 CPU oracle, from
shared seeded states, through the C-ABI.

Tolerance (FP64 path): 1e-10 relative to the natural scale of each quantity
-- the largest |lambda| for eigenvalues, the unit norm of eigenvectors and
coefficient columns, the largest term of the force sum, the largest hop
probability of the batch -- and bit-exact for occupations and hop counts.
"""
import numpy as np
import pytest

import iesh_inputs as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_2212_00518_gb300 import build as B
    B.build()
    import paper_2212_00518_gb300 as pkg
    return pkg


MODELS = {
    "dw20": (W.double_well(20), 0.01, 1.0),
    "dw100": (W.double_well(100), 0.01, 1.0),
    "paper40": (W.double_well_paper(40), 5 * 9.5e-4, 10.0),
    "paper40trap": (W.double_well_paper(40, disc="trapezoid"), 5 * 9.5e-4, 10.0),
    "desorb50": (W.desorption(1.0, 50), None, 4.0),
    "image50": (W.morse_image(50), None, 4.0),
}


def _positions(md, n, seed):
    rng = np.random.default_rng(seed)
    if md["kind"] == "harmonic":
        w = md["par"][0]
        kT = 0.01 if w > 1e-3 else 5 * 9.5e-4
        x, p = W.thermal_harmonic(n, md["mass"], w, kT, seed)
        if w < 1e-3:
            x = x + 8.0  # near the crossing of the paper double well
        return x, p
    x = rng.uniform(W.angstrom(1.6), W.angstrom(6.0), n)
    p = rng.normal(0.0, np.sqrt(md["mass"] * 0.02), n)
    return x, p


def _state(md, n, seed, weight=0.5):
    N, Ne = md["M"] + 1, md["Ne"]
    x, p = _positions(md, n, seed)
    occ = W.random_occupations(n, N, Ne, seed + 1)
    C = W.mixed_coefficients(occ, N, seed + 2, weight)
    return x, p, occ, C


def _close(a, b, scale, rtol=RTOL, what=""):
    err = np.max(np.abs(np.asarray(a) - np.asarray(b)))
    assert err <= rtol * scale, f"{what}: max error {err:.3e} > {rtol:.0e} x {scale:.3e}"


# ------------------------------------------------------------------ bath
@pytest.mark.parametrize("name", ["dw100", "paper40", "paper40trap", "image50"])
def test_bath_matches_oracle(P, name):
    md = MODELS[name][0]
    ctx = P.Context(md, 1)
    eps, z0 = ctx.bath()
    B = O.bind(md)
    _close(eps, B.eps, np.abs(B.eps).max(), 1e-14, "eps")
    _close(z0, B.Vbar * B.sqw, np.abs(z0).max(), 1e-13, "z0")


def test_two_lead_bath(P):
    md = W.morse_image(50, bias=0.1)
    ctx = P.Context(md, 1)
    eps, z0 = ctx.bath()
    B = O.bind(md)
    _close(eps, B.eps, np.abs(B.eps).max(), 1e-14, "eps")
    _close(z0, B.Vbar * B.sqw, np.abs(z0).max(), 1e-13, "z0")


# --------------------------------------------------------------- eigen
@pytest.mark.parametrize("name", list(MODELS))
def test_eigen_and_force_parity(P, name):
    md = MODELS[name][0]
    n = 12
    x, p, occ, C = _state(md, n, 11)
    ctx = P.Context(md, n)
    ctx.set_state(x, p, occ, C)
    lam, q0, F = ctx.eigen()
    B = O.bind(md)
    for t in range(n):
        l_o, Q_o, T_o, d_o, F_o = O.eigen(B, x[t], occ[t].astype(np.int32))
        _close(lam[t], l_o, np.abs(l_o).max(), RTOL, f"lambda traj {t}")
        _close(q0[t], Q_o[0], 1.0, RTOL, f"q0 traj {t}")
        fscale = abs(O.model_eval(md, x[t])[1]) + np.abs(np.diag(T_o)[occ[t]]).sum()
        _close(F[t], F_o, fscale, RTOL, f"force traj {t}")


# ----------------------------------------------------- hop probabilities
@pytest.mark.parametrize("name", ["dw20", "paper40", "desorb50"])
def test_hop_probability_parity(P, name):
    md, _, dt = MODELS[name]
    n = 8
    x, p, occ, C = _state(md, n, 21, weight=0.8)
    ctx = P.Context(md, n)
    ctx.set_state(x, p, occ, C)
    g = ctx.hop_probabilities(dt)
    B = O.bind(md)
    for t in range(n):
        _, _, _, d_o, _ = O.eigen(B, x[t])
        g_o, _, _, rc = O.hop_probs(occ[t], C[t].T, d_o, p[t] / md["mass"], dt)
        assert rc == 0
        _close(g[t], g_o, max(np.abs(g_o).max(), 1e-300), 1e-9, f"g traj {t}")


# ---------------------------------------------------------- one step
@pytest.mark.parametrize("name", list(MODELS))
def test_one_step_parity(P, name):
    md, _, dt = MODELS[name]
    n = 8
    x, p, occ, C = _state(md, n, 31, weight=0.6)
    ctx = P.Context(md, n)
    ctx.set_state(x, p, occ, C)
    ctx.run(dt, 1, seed=9)
    st = ctx.get_state()
    assert np.all(st["status"] == 0)
    B = O.bind(md)
    for t in range(n):
        r = O.step_one(B, x[t], p[t], occ[t].astype(np.int32), C[t].T, dt, seed=9, traj=t, n=0)
        assert np.array_equal(st["occ"][t], r["occ"]), f"occupations traj {t}"
        _close(st["x"][t], r["x"], abs(r["x"]) + 1.0, 1e-13, f"x traj {t}")
        _close(st["p"][t], r["p"], abs(r["p"]) + 1e-3, 1e-10, f"p traj {t}")
        _close(st["C"][t].T, r["C"], 1.0, RTOL, f"C traj {t}")


# -------------------------------------------------------- many steps
def test_hop_decisions_identical_tiny_case(P):
    """Hop-rich tiny case (paper double well, M=8): identical hop decisions
    over many steps on the shared Philox stream."""
    md = W.double_well_paper(8)
    md["Gamma"] = 0.02
    n, steps, dt = 32, 300, 10.0
    x, p, occ, C = _state(md, n, 41, weight=1.0)
    ctx = P.Context(md, n)
    ctx.set_state(x, p, occ, C)
    ctx.run(dt, steps, seed=123)
    st = ctx.get_state()
    ns, hops, fr = ctx.counters()
    ref = O.run(O.bind(md), x, p, occ.astype(np.int32), np.transpose(C, (0, 2, 1)), dt, steps,
                seed=123)
    assert np.all(ns == steps)
    assert hops.sum() > 0, "case must hop"
    assert np.array_equal(hops, ref["hops"])
    assert np.array_equal(fr, ref["frustrated"])
    assert np.array_equal(st["occ"], ref["occ"])
    _close(st["x"], ref["x"], np.abs(ref["x"]).max(), 1e-9, "x")
    _close(np.transpose(st["C"], (0, 2, 1)), ref["C"], 1.0, 1e-8, "C")


def test_config1_run_parity(P):
    """The small measured configuration: M=20, Ne=10, 16 trajectories, kT=0.01,
    dt=1, 1000 steps, seed 0, lowest orbitals occupied."""
    md = W.double_well(20)
    n, steps = 16, 1000
    x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], 0.01, seed=0)
    occ = W.lowest_occupations(n, md["Ne"])
    C = W.unit_coefficients(occ, md["M"] + 1)
    ctx = P.Context(md, n)
    ctx.set_state(x, p, occ, C)
    ctx.run(1.0, steps, seed=0)
    st = ctx.get_state()
    ref = O.run(O.bind(md), x, p, occ.astype(np.int32), np.transpose(C, (0, 2, 1)), 1.0, steps,
                seed=0)
    assert np.array_equal(st["occ"], ref["occ"])
    _close(st["x"], ref["x"], np.abs(ref["x"]).max(), RTOL, "x")
    _close(st["p"], ref["p"], np.abs(ref["p"]).max(), RTOL, "p")
    _close(np.transpose(st["C"], (0, 2, 1)), ref["C"], 1.0, 1e-9, "C")


def test_zero_coupling_phases_only(P):
    md = W.double_well(20, Gamma=0.0)
    n = 8
    x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], 0.01, seed=3)
    occ = W.lowest_occupations(n, md["Ne"])
    C = W.mixed_coefficients(occ, md["M"] + 1, 4, 0.5)
    ctx = P.Context(md, n)
    ctx.set_state(x, p, occ, C)
    ctx.run(1.0, 200, seed=1)
    st = ctx.get_state()
    _, hops, fr = ctx.counters()
    assert hops.sum() == 0 and fr.sum() == 0
    _close(np.abs(st["C"]), np.abs(C), 1.0, 1e-12, "|C|")


def test_skip_bound_keeps_decisions(P):
    md = W.double_well_paper(12)
    n, steps, dt = 32, 200, 10.0
    x, p, occ, C = _state(md, n, 51, weight=0.3)
    out = []
    for skip in (False, True):
        ctx = P.Context(md, n, skip_bound=skip)
        ctx.set_state(x, p, occ, C)
        ctx.run(dt, steps, seed=5)
        out.append((ctx.get_state(), ctx.counters()))
    (s0, c0), (s1, c1) = out
    assert np.array_equal(c0[1], c1[1])
    assert np.array_equal(s0["occ"], s1["occ"])
    assert np.array_equal(s0["x"], s1["x"])
    assert np.array_equal(s0["C"], s1["C"])


def test_thermal_initial_conditions_match_oracle_samplers(P):
    md = W.double_well(20)
    n, seed, kT, kTe = 64, 77, 0.01, 0.05
    ctx = P.Context(md, n)
    ctx.init_state(n, kT_nuc=kT, kT_el=kTe, seed=seed)
    st = ctx.get_state()
    lam, _, _ = ctx.eigen()
    B = O.bind(md)
    for t in range(n):
        xo, po = O.sample_nuclear(seed, t, md["mass"], md["par"][0], 0.0, kT)
        assert abs(st["x"][t] - xo) < 1e-12 * (1 + abs(xo))
        assert abs(st["p"][t] - po) < 1e-12 * (1 + abs(po))
        lam_o = O.eigen(B, st["x"][t])[0]
        occ_o = O.sample_occupations(seed, t, lam_o, md["Ne"], kTe)
        assert np.array_equal(st["occ"][t], occ_o), t
    # unit coefficients
    N = md["M"] + 1
    assert np.array_equal(st["C"], W.unit_coefficients(st["occ"], N))


def test_records_match_oracle(P):
    md = W.double_well_paper(12)
    n, steps, dt, every = 8, 60, 10.0, 20
    x, p, occ, C = _state(md, n, 61, weight=0.5)
    ctx = P.Context(md, n, record_every=every, max_records=steps // every)
    ctx.set_state(x, p, occ, C)
    ctx.run(dt, steps, seed=2)
    sh, wf = ctx.records(steps // every)
    ref = O.run(O.bind(md), x, p, occ.astype(np.int32), np.transpose(C, (0, 2, 1)), dt, steps,
                seed=2, record_every=every)
    assert sh.shape == ref["pop_sh"].shape
    _close(sh, ref["pop_sh"], 1.0, 1e-9, "P_d surface")
    _close(wf, ref["pop_wf"], 1.0, 1e-9, "P_d wavefunction")


def test_state_errors(P):
    md = W.double_well(20)
    ctx = P.Context(md, 4)
    with pytest.raises(P.IeshError, match="ESTATE"):
        ctx.run(1.0, 1)
    with pytest.raises(P.IeshError, match="EINVAL"):
        ctx.init_state(5)


# ------------------------------------------- full benchmark size, sampled
def test_full_size_one_step_sampled(P):
    """The benchmark workload (M=100, Ne=50, 4096 trajectories, dt=1) in the
    launch configuration the benchmark times: one step from a shared state,
    checked against the oracle on a sample of trajectories."""
    md = W.double_well(100)
    n = 4096
    kT = np.array([0.005, 0.0075, 0.01])[np.arange(n) % 3]
    x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], kT, seed=2)
    occ = W.lowest_occupations(n, md["Ne"])
    C = W.mixed_coefficients(occ[:64], md["M"] + 1, 3, 0.3)
    C = np.concatenate([C] * (n // 64))
    ctx = P.Context(md, n)
    ctx.set_state(x, p, occ, C)
    ctx.run(1.0, 1, seed=0)
    st = ctx.get_state()
    assert np.all(st["status"] == 0)
    B = O.bind(md)
    for t in (0, 1, 777, 2048, 4095):
        r = O.step_one(B, x[t], p[t], occ[t].astype(np.int32), C[t].T, 1.0, seed=0, traj=t, n=0)
        assert np.array_equal(st["occ"][t], r["occ"])
        _close(st["x"][t], r["x"], abs(r["x"]) + 1.0, 1e-13, "x")
        _close(st["p"][t], r["p"], abs(r["p"]) + 1e-3, RTOL, "p")
        _close(st["C"][t].T, r["C"], 1.0, RTOL, "C")
