"""GPU parity of the diabatic-basis (overlap) propagator variant with the FP64
oracle's own restatement (dense Jacobi eigenvectors, O = Q1^T Q0).

The GPU builds O from the closed form of the arrowhead (no eigenvectors):
the off-diagonal entries from the secular equation at both ends of the step,
the diagonal from orthogonality.  FP64 tolerances as for the main path:
per step 1e-10 relative on x, p and 1e-10 on C; over 100 steps 1e-9 on C.
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


def _state(md, n, seed, weight=0.6, shift=0.0):
    N, Ne = md["M"] + 1, md["Ne"]
    x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], 0.01, seed)
    occ = W.random_occupations(n, N, Ne, seed + 1)
    C = W.mixed_coefficients(occ, N, seed + 2, weight)
    return x + shift, p, occ, C


def _strong_paper(M):
    md = W.double_well_paper(M)
    md["Gamma"] = 0.02
    return md


CASES = {
    "paper40": (W.double_well_paper(40), 10.0, 8.0),
    "strong12": (_strong_paper(12), 10.0, 8.0),
    "dw100": (W.double_well(100), 1.0, 0.0),
}


@pytest.mark.parametrize("name", list(CASES))
def test_overlap_one_step(P, name):
    md, dt, shift = CASES[name]
    n = 6
    x, p, occ, C = _state(md, n, 5, 0.6, shift)
    B = O.bind(md)
    ctx = P.Context(md, n, propagator=P.iesh.PROP_OVERLAP)
    ctx.set_state(x, p, occ, C)
    ctx.run(dt, 1, seed=9)
    st = ctx.get_state()
    for t in range(n):
        r = O.step_one(B, x[t], p[t], occ[t].astype(np.int32), C[t].T, dt, seed=9, traj=t, n=0, prop=1)
        assert np.array_equal(st["occ"][t], r["occ"])
        assert abs(st["x"][t] - r["x"]) <= 1e-12 * (1 + abs(r["x"]))
        assert abs(st["p"][t] - r["p"]) <= 1e-12 * (1 + abs(r["p"]))
        assert np.abs(st["C"][t].T - r["C"]).max() <= 1e-10


@pytest.mark.parametrize("name", ["paper40", "strong12"])
def test_overlap_100_steps(P, name):
    md, dt, shift = CASES[name]
    n, steps, every = 8, 100, 20
    x, p, occ, C = _state(md, n, 7, 0.6, shift)
    ctx = P.Context(md, n, record_every=every, max_records=steps // every, propagator=P.iesh.PROP_OVERLAP)
    ctx.set_state(x, p, occ, C)
    ctx.run(dt, steps, seed=3)
    st = ctx.get_state()
    sh, wf = ctx.records(steps // every)
    ref = O.run(O.bind(md), x, p, occ.astype(np.int32), np.transpose(C, (0, 2, 1)), dt, steps, seed=3,
                record_every=every, prop=1)
    assert np.array_equal(st["occ"], ref["occ"])
    assert np.array_equal(ctx.counters()[1], ref["hops"].astype(np.int32))
    assert np.abs(np.transpose(st["C"], (0, 2, 1)) - ref["C"]).max() <= 1e-9
    assert np.abs(st["x"] - ref["x"]).max() <= 1e-10 * np.abs(ref["x"]).max()
    assert np.abs(wf - ref["pop_wf"]).max() <= 1e-10
    assert np.abs(sh - ref["pop_sh"]).max() <= 1e-10


def test_overlap_scattering_model_matches_oracle(P):
    """Two-lead Morse + image-charge model: the coupling factor f(x) changes
    along the path, so both Cauchy coefficients a and b are active."""
    md = W.morse_image(20, bias=0.1)
    n = 6
    rng = np.random.default_rng(9)
    e = rng.uniform(W.ev(0.2), W.ev(1.5), n)
    x = np.full(n, W.angstrom(5.0))
    p = -np.sqrt(2 * md["mass"] * e)
    occ = W.lowest_occupations(n, md["Ne"])
    C = W.mixed_coefficients(occ, 21, 3, 0.4)
    dt = 0.1 * W.FS_AU
    ctx = P.Context(md, n, propagator=P.iesh.PROP_OVERLAP)
    ctx.set_state(x, p, occ, C)
    ctx.run(dt, 150, seed=8)
    st = ctx.get_state()
    ref = O.run(O.bind(md), x, p, occ.astype(np.int32), np.transpose(C, (0, 2, 1)), dt, 150, seed=8, prop=1)
    assert np.all(st["status"] == 0)
    assert np.array_equal(st["occ"], ref["occ"])
    assert np.abs(st["x"] - ref["x"]).max() <= 1e-9 * np.abs(ref["x"]).max()
    assert np.abs(np.transpose(st["C"], (0, 2, 1)) - ref["C"]).max() <= 1e-8


def test_overlap_agrees_with_averaged_generator_at_small_steps(P):
    """Both propagators are second order: one step of dt = 0.5 from the same
    state differs by O(dt^3) in C, and both keep the columns orthonormal."""
    md = W.double_well(60)
    n = 8
    x, p, occ, C = _state(md, n, 21, 0.8)
    out = []
    for prop in (P.iesh.PROP_AVERAGED, P.iesh.PROP_OVERLAP):
        ctx = P.Context(md, n, propagator=prop)
        ctx.set_state(x, p, occ, C)
        ctx.run(0.5, 1, seed=1)
        out.append(ctx.get_state()["C"])
        ctx.close()
    for Cn in out:
        G = np.einsum("tei,tfi->tef", Cn.conj(), Cn)
        assert np.abs(G - np.eye(md["Ne"])[None]).max() < 1e-12
    assert np.abs(out[0] - out[1]).max() < 1e-6


def test_overlap_is_fp64_only(P):
    with pytest.raises(P.iesh.IeshError):
        P.Context(W.double_well(10), 4, precision=P.PREC_MIXED, propagator=P.iesh.PROP_OVERLAP)
