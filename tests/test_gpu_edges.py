"""Edge cases on the GPU: an empty batch, the largest system the library
accepts (N = 256 orbitals, Ne = 112 electrons) on every path, one electron
(the two-state surface-hopping limit), and a singular overlap matrix S."""
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


def _state(md, n, seed, weight=0.5, shift=0.0):
    N, Ne = md["M"] + 1, md["Ne"]
    x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], 0.01, seed)
    occ = W.random_occupations(n, N, Ne, seed + 1)
    C = W.mixed_coefficients(occ, N, seed + 2, weight)
    return x + shift, p, occ, C


def test_empty_batch(P):
    md = W.double_well(20)
    for prec in (0, 1):
        ctx = P.Context(md, 4, precision=prec)
        z = np.zeros(0)
        occ = np.zeros((0, md["Ne"]), np.int16)
        C = np.zeros((0, md["Ne"], 21), np.complex128 if prec == 0 else np.complex64)
        ctx.set_state(z, z, occ, C)
        ctx.run(1.0, 3, seed=1)
        st = ctx.get_state()
        assert st["x"].shape == (0,) and ctx.live_count() == 0
        ctx.close()


@pytest.mark.parametrize("path", ["fp64", "mixed", "overlap"])
def test_largest_system_one_step(P, path):
    """M = 255 (N = 256, the orbital limit) with Ne = 112 (the hop-kernel
    limit): the hop LU fills most of the shared memory of a 512-thread CTA,
    the propagators run their widest shapes."""
    md = W.double_well_paper(255)
    md["Ne"] = 112
    md["Gamma"] = 0.02
    n = 2
    x, p, occ, C = _state(md, n, 31, 0.5, shift=8.0)
    prec = 1 if path == "mixed" else 0
    prop = 1 if path == "overlap" else 0
    ctx = P.Context(md, n, precision=prec, propagator=prop)
    ctx.set_state(x, p, occ, C if prec == 0 else C.astype(np.complex64))
    g = ctx.hop_probabilities(10.0)
    ctx.run(10.0, 1, seed=4)
    st = ctx.get_state()
    assert np.all(st["status"] == 0)
    B = O.bind(md)
    tolC = 2e-6 if prec else 1e-10
    for t in range(n):
        d = O.eigen(B, x[t])[3]
        gref = O.hop_probs(occ[t], C[t].T, d, p[t] / md["mass"], 10.0)[0]
        assert np.abs(g[t] - gref).max() <= (2e-6 if prec else 1e-10) * max(np.abs(gref).max(), 1e-300)
        r = O.step_one(B, x[t], p[t], occ[t].astype(np.int32), C[t].T, 10.0, seed=4, traj=t, n=0, prop=prop)
        assert np.array_equal(st["occ"][t], r["occ"])
        assert abs(st["x"][t] - r["x"]) <= 1e-12 * (1 + abs(r["x"]))
        assert np.abs(st["C"][t].T - r["C"]).max() <= tolC


@pytest.mark.parametrize("prec", [0, 1])
def test_one_electron_limit(P, prec):
    """Ne = 1: the hop ratio reduces to c_m / c_k (two-state FSSH per
    candidate); 200 steps with hops against the oracle."""
    md = W.double_well_paper(10)
    md["Ne"] = 1
    md["Gamma"] = 0.02
    n, steps, dt = 16, 200, 10.0
    x, p, occ, C = _state(md, n, 41, 1.0, shift=8.0)
    ctx = P.Context(md, n, precision=prec)
    ctx.set_state(x, p, occ, C if prec == 0 else C.astype(np.complex64))
    ctx.run(dt, steps, seed=5)
    st = ctx.get_state()
    _, hops, _ = ctx.counters()
    ref = O.run(O.bind(md), x, p, occ.astype(np.int32), np.transpose(C, (0, 2, 1)), dt, steps, seed=5)
    assert ref["hops"].sum() > 0
    same = [np.array_equal(st["occ"][t], ref["occ"][t]) and hops[t] == ref["hops"][t] for t in range(n)]
    if prec == 0:
        assert all(same)
        assert np.abs(np.transpose(st["C"], (0, 2, 1)) - ref["C"]).max() <= 1e-9
    else:
        assert np.mean(same) >= 0.9


@pytest.mark.parametrize("prec", [0, 1])
def test_singular_overlap_flags_and_keeps_going(P, prec):
    """An electron with no weight on the occupied orbitals makes a column of
    S = C[s, :] exactly zero.  Without coupling the propagation only changes
    phases, so S stays singular through the step: the trajectory is flagged
    IESH_TRAJ_SINGULAR, takes no hop, and the rest of the batch is
    unaffected."""
    md = W.double_well(20)
    md["Gamma"] = 0.0
    n = 4
    x, p, occ, C = _state(md, n, 51, 0.5)
    free = [m for m in range(21) if m not in set(occ[1].tolist())]
    C[1, 0, :] = 0.0
    C[1, 0, free[0]] = 1.0
    ctx = P.Context(md, n, precision=prec)
    ctx.set_state(x, p, occ, C if prec == 0 else C.astype(np.complex64))
    ctx.run(1.0, 1, seed=2)
    st = ctx.get_state()
    _, hops, _ = ctx.counters()
    assert st["status"][1] & P.iesh.TRAJ_SINGULAR
    assert hops[1] == 0
    assert np.all(st["status"][[0, 2, 3]] == 0)
    assert np.all(np.isfinite(st["x"])) and np.all(np.isfinite(st["C"]))
