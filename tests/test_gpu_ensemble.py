"""Ensemble observables of the GPU paths against the FP64 oracle on matched
ensembles (same seeded initial conditions, same Philox hop stream):
desorption probability of the desorption model (Sec. III C, threshold
5 angstrom) and impurity populations of the paper's double well
(Sec. III B), for the FP64 and the mixed-precision paths, within three
binomial / sample standard errors; and identical hop decisions of the FP64
path on a tiny hop-rich case over 10^4 steps.
"""
import math

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


@pytest.mark.parametrize("precision", [0, 1])
def test_desorption_probability_matches_oracle(P, precision):
    md = W.desorption(1.0, 16, band_ev=16.0, mu_ev=0.0)
    n, steps, seed = 128, 1000, 11
    kT = 300 * W.KB_HARTREE_PER_K
    ctx = P.Context(md, n, precision=precision)
    ctx.init_state(n, kT_nuc=kT, kT_el=0.0, seed=seed)  # Wigner sample on the device
    st0 = ctx.get_state()
    ctx.run(0.1 * W.FS_AU, steps, seed=3)
    st = ctx.get_state()
    B = O.bind(md)
    w = math.sqrt(2 * md["par"][0] * md["par"][2] ** 2 / md["mass"])
    x0, p0 = zip(*[O.sample_nuclear(seed, t, md["mass"], w, md["par"][1], kT, True) for t in range(n)])
    x0, p0 = np.array(x0), np.array(p0)
    assert np.abs(st0["x"] - x0).max() < 1e-10
    occ = np.tile(np.arange(B.Ne, dtype=np.int32), (n, 1))
    C = np.stack([O.unit_coefficients(B.N, o) for o in occ])
    ref = O.run(B, x0, p0, occ, C, 0.1 * W.FS_AU, steps, seed=3)
    thr = W.angstrom(5.0)
    pg, po = np.mean(st["x"] > thr), np.mean(ref["x"] > thr)
    assert po > 0.02, "ensemble must desorb"
    se = math.sqrt(max(po * (1 - po), 1.0 / n) / n)
    assert abs(pg - po) <= 3 * math.sqrt(2) * se, (pg, po)


@pytest.mark.parametrize("precision", [0, 1])
def test_double_well_populations_match_oracle(P, precision):
    md = W.double_well_paper(12)
    n, steps, every = 64, 400, 100
    kT = 5 * 9.5e-4
    x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], kT, seed=21)
    occ = W.lowest_occupations(n, md["Ne"])
    C = W.unit_coefficients(occ, md["M"] + 1)
    ctx = P.Context(md, n, precision=precision, record_every=every, max_records=steps // every)
    ctx.set_state(x, p, occ, C if precision == 0 else C.astype(np.complex64))
    ctx.run(100.0, steps, seed=4)
    sh, wf = ctx.records(steps // every)
    ref = O.run(O.bind(md), x, p, occ.astype(np.int32), np.transpose(C, (0, 2, 1)), 100.0, steps,
                seed=4, record_every=every)
    for a, b in ((sh, ref["pop_sh"]), (wf, ref["pop_wf"])):
        se = np.sqrt(np.maximum(b.var(axis=1), 1e-12) / n)
        assert np.all(np.abs(a.mean(axis=1) - b.mean(axis=1)) <= 3 * np.sqrt(2) * se)


def test_identical_hop_decisions_over_ten_thousand_steps(P):
    md = W.double_well_paper(8)
    md["Gamma"] = 0.02
    n, steps, dt = 32, 10000, 10.0
    x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], 5 * 9.5e-4, seed=41)
    x = x + 8.0
    occ = W.random_occupations(n, 9, 4, 42)
    C = W.mixed_coefficients(occ, 9, 43, 1.0)
    ctx = P.Context(md, n)
    ctx.set_state(x, p, occ, C)
    ctx.run(dt, steps, seed=123)
    st = ctx.get_state()
    _, hops, fr = ctx.counters()
    ref = O.run(O.bind(md), x, p, occ.astype(np.int32), np.transpose(C, (0, 2, 1)), dt, steps,
                seed=123)
    assert hops.sum() > 50
    assert np.array_equal(hops, ref["hops"]) and np.array_equal(fr, ref["frustrated"])
    assert np.array_equal(st["occ"], ref["occ"])


@pytest.mark.parametrize("precision", [0, 1])
def test_desorption_curve_matches_oracle(P, precision):
    """P_des(t) of Sec. III C: the fraction of trajectories that have passed
    x > 5 angstrom by time t, from the library's finished-trajectory flag and
    step counters, against the oracle's first-passage steps on matched
    ensembles (Wigner 300 K nuclei and canonical 300 K electrons sampled on
    the device; the same states start the oracle)."""
    md = W.desorption(1.0, 16, band_ev=16.0, mu_ev=0.0)
    n, steps, seed = 128, 1000, 11
    kT = 300 * W.KB_HARTREE_PER_K
    thr = W.angstrom(5.0)
    dt = 0.1 * W.FS_AU
    ctx = P.Context(md, n, precision=precision, z_done=thr)
    ctx.init_state(n, kT_nuc=kT, kT_el=kT, seed=seed)
    st0 = ctx.get_state()
    ctx.run(dt, steps, seed=3)
    st = ctx.get_state()
    ns = ctx.counters()[0]
    C0 = np.transpose(st0["C"].astype(np.complex128), (0, 2, 1))
    ref = O.run(O.bind(md), st0["x"], st0["p"], st0["occ"].astype(np.int32), C0, dt, steps, seed=3,
                z_done=thr)
    done_g = (st["status"] & P.iesh.TRAJ_DONE) != 0
    done_o = (ref["status"] & 8) != 0
    assert done_o.mean() > 0.02, "ensemble must desorb"
    for t_fs in (25, 50, 75, 100):
        k = int(round(t_fs * W.FS_AU / dt))
        pg = np.mean(done_g & (ns <= k))
        po = np.mean(done_o & (ref["steps"] <= k))
        se = math.sqrt(max(po * (1 - po), 1.0 / n) / n)
        assert abs(pg - po) <= 3 * math.sqrt(2) * se, (t_fs, pg, po)


@pytest.mark.parametrize("precision", [0, 1])
def test_scattering_energy_loss_matches_oracle(P, precision):
    """Sec. III D scattering on the desorption model: start at 5 angstrom
    toward the surface with E_inc = 1 eV, electrons at 0 K, stop on the
    rebound through 5 angstrom; the kinetic-energy loss of the rebounded
    trajectories against the oracle's (matched ensembles, 3 standard errors)."""
    n, E_inc = 64, 1.0
    md, x, p, occ, C = W.erpenbeck_scattering(n, E_inc, M=16, band_ev=16.0)
    thr = W.angstrom(5.0)
    dt = 0.1 * W.FS_AU
    steps = 3000  # 300 fs
    ctx = P.Context(md, n, precision=precision, z_done=thr)
    ctx.set_state(x, p, occ, C if precision == 0 else C.astype(np.complex64))
    ctx.run(dt, steps, seed=5)
    st = ctx.get_state()
    ref = O.run(O.bind(md), x, p, occ.astype(np.int32), np.transpose(C, (0, 2, 1)), dt, steps, seed=5,
                z_done=thr)
    done_g = (st["status"] & P.iesh.TRAJ_DONE) != 0
    done_o = (ref["status"] & 8) != 0
    assert done_o.mean() > 0.9 and done_g.mean() > 0.9
    e_inc = W.ev(E_inc)
    lg = e_inc - st["p"][done_g] ** 2 / (2 * md["mass"])
    lo = e_inc - ref["p"][done_o] ** 2 / (2 * md["mass"])
    se = math.sqrt(max(lo.var(), 1e-12) / len(lo))
    assert abs(lg.mean() - lo.mean()) <= 3 * math.sqrt(2) * se + 1e-9 * e_inc, (lg.mean(), lo.mean())
