"""Boundary features of the C-ABI on the GPU: bit-exact resume from a
checkpoint, global trajectory ids in the Philox counters (a batch split over
contexts reproduces the undivided batch), the norm-drift status bit and the
batch status summary, and the per-trajectory observables against the oracle."""
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


def _hop_rich(n, seed):
    """Paper double well with strong coupling near the crossing: hops occur."""
    md = W.double_well_paper(8)
    md["Gamma"] = 0.02
    N, Ne = md["M"] + 1, md["Ne"]
    x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], 5 * 9.5e-4, seed)
    x = x + 8.0
    occ = W.random_occupations(n, N, Ne, seed + 1)
    C = W.mixed_coefficients(occ, N, seed + 2, 1.0)
    return md, x, p, occ, C


def _same_state(a, b):
    sa, sb = a.get_state(), b.get_state()
    for k in ("x", "p", "occ", "C", "status"):
        assert np.array_equal(sa[k], sb[k]), k
    for u, v in zip(a.counters(), b.counters()):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("where", ["host", "device"])
def test_checkpoint_resume_is_bit_exact(P, precision, where):
    import torch
    md, x, p, occ, C = _hop_rich(16, 51)
    C = C.astype(np.complex128 if precision == 0 else np.complex64)
    dt, seed = 10.0, 77
    full = P.Context(md, 16, precision=precision, record_every=50, max_records=40)
    full.set_state(x, p, occ, C)
    full.run(dt, 1000, seed)
    assert full.counters()[1].sum() > 0, "case must hop"

    half = P.Context(md, 16, precision=precision, record_every=50, max_records=40)
    half.set_state(x, p, occ, C)
    half.run(dt, 500, seed)
    if where == "host":
        blob = half.checkpoint_save()
    else:
        blob = torch.zeros(half.checkpoint_bytes(), dtype=torch.uint8, device="cuda")
        half.checkpoint_save(blob)
    half.close()
    resumed = P.Context(md, 16, precision=precision, record_every=50, max_records=40)
    resumed.checkpoint_load(blob)
    resumed.run(dt, 500, seed)
    _same_state(full, resumed)
    ra, rb = full.records(40), resumed.records(40)
    assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])


def test_checkpoint_rejects_other_shapes(P):
    md, x, p, occ, C = _hop_rich(4, 3)
    a = P.Context(md, 4)
    a.set_state(x, p, occ, C)
    blob = a.checkpoint_save()
    other = dict(md, M=10, Ne=5)
    b = P.Context(other, 4)
    with pytest.raises(P.IeshError, match="EINVAL"):
        b.checkpoint_load(blob)
    small = P.Context(md, 2)
    with pytest.raises(P.IeshError, match="EINVAL"):
        small.checkpoint_load(blob)
    bad = blob.copy()
    bad[0] = 0
    with pytest.raises(P.IeshError, match="EINVAL"):
        a.checkpoint_load(bad)


@pytest.mark.parametrize("precision", [0, 1])
def test_split_batch_with_trajectory_ids_reproduces_whole(P, precision):
    """Thermal nuclei, canonical electrons and hop uniforms keyed by global
    trajectory ids: [0, n/2) and [n/2, n) in two contexts equal one context."""
    md = W.double_well_paper(8)
    md["Gamma"] = 0.02
    n, h = 24, 12
    N = md["M"] + 1
    kT = 5 * 9.5e-4
    whole = P.Context(md, n, precision=precision)
    whole.init_state(n, kT_nuc=kT, kT_el=2 * kT, seed=5)
    parts = []
    for base in (0, h):
        c = P.Context(md, h, precision=precision, traj_base=base)
        c.init_state(h, kT_nuc=kT, kT_el=2 * kT, seed=5)
        parts.append(c)
    sw = whole.get_state()
    for k, c in enumerate(parts):  # samples drawn with global ids
        s = c.get_state()
        sl = slice(k * h, (k + 1) * h)
        for key in ("x", "p", "occ", "C"):
            assert np.array_equal(s[key], sw[key][sl]), key
    # the second part's nuclei are the oracle's samples for global ids h..n-1
    st1 = parts[1].get_state()
    for t in range(h):
        xo, po = O.sample_nuclear(5, h + t, md["mass"], md["par"][0], 0.0, kT)
        assert abs(st1["x"][t] - xo) <= 1e-12 * abs(xo) + 1e-15
        assert abs(st1["p"][t] - po) <= 1e-12 * abs(po) + 1e-15
    # hop-rich continuation: near the crossing with coherent coefficients
    x = sw["x"] + 8.0
    C = W.mixed_coefficients(sw["occ"], N, 6, 1.0).astype(sw["C"].dtype)
    whole.set_state(x, sw["p"], sw["occ"], C)
    for k, c in enumerate(parts):
        sl = slice(k * h, (k + 1) * h)
        c.set_state(x[sl].copy(), sw["p"][sl].copy(), sw["occ"][sl].copy(), C[sl].copy())
    for c in [whole] + parts:
        c.run(10.0, 300, seed=9)
    sw = whole.get_state()
    cw = whole.counters()
    for k, c in enumerate(parts):
        s = c.get_state()
        sl = slice(k * h, (k + 1) * h)
        for key in ("x", "p", "occ", "C", "status"):
            assert np.array_equal(s[key], sw[key][sl]), key
        for u, v in zip(c.counters(), cw):
            assert np.array_equal(u, v[sl])
    assert cw[1].sum() > 0, "case must hop"


def test_norm_drift_bit_and_status_summary(P):
    md, x, p, occ, C = _hop_rich(8, 61)
    ok = P.Context(md, 8)
    ok.set_state(x, p, occ, C)
    ok.run(10.0, 20, seed=1)
    code, bits, counts = ok.check()
    assert code == "IESH_OK" and not bits & P.iesh.TRAJ_NORM_DRIFT
    # a deliberately loose Chebyshev truncation loses unitarity
    loose = P.Context(md, 8, prop_tol=1e-2)
    loose.set_state(x, p, occ, C)
    loose.run(10.0, 20, seed=1)
    code, bits, counts = loose.check()
    st = loose.get_state()["status"]
    assert code == "IESH_ENORM"
    assert bits & P.iesh.TRAJ_NORM_DRIFT
    assert counts[6] == np.count_nonzero(st & P.iesh.TRAJ_NORM_DRIFT) > 0
    # the bit is sticky until the state is replaced
    loose.set_state(x, p, occ, C)
    assert loose.check()[0] == "IESH_OK"


@pytest.mark.parametrize("precision", [0, 1])
def test_observables_match_oracle(P, precision):
    md = W.desorption(1.0, 50)
    n = 8
    N, Ne = md["M"] + 1, md["Ne"]
    rng = np.random.default_rng(71)
    x = rng.uniform(W.angstrom(1.6), W.angstrom(6.0), n)
    p = rng.normal(0.0, np.sqrt(md["mass"] * 0.02), n)
    occ = W.random_occupations(n, N, Ne, 72)
    C = W.mixed_coefficients(occ, N, 73, 0.6)
    C = C.astype(np.complex128 if precision == 0 else np.complex64)
    ctx = P.Context(md, n, precision=precision)
    ctx.set_state(x, p, occ, C)
    ob = ctx.observables()
    B = O.bind(md)
    tol = 1e-10 if precision == 0 else 1e-6
    for t in range(n):
        lam, Q, _, _, _ = O.eigen(B, x[t])
        U0 = O.model_eval(md, x[t])[0]
        s = occ[t]
        assert abs(ob["ke"][t] - p[t] ** 2 / (2 * md["mass"])) <= 1e-15 * ob["ke"][t]
        ep = U0 + lam[s].sum()
        assert abs(ob["epot"][t] - ep) <= 1e-10 * (abs(U0) + np.abs(lam[s]).sum())
        assert abs(ob["pop_sh"][t] - np.sum(Q[0, s] ** 2)) <= 1e-10
        wf = np.sum(np.abs(Q[0] @ C[t].T.astype(np.complex128)) ** 2)
        assert abs(ob["pop_wf"][t] - wf) <= tol


def test_total_energy_conserved_through_hops(P):
    """KE + epot of the observables call is conserved along the run, across
    accepted hops (velocity Verlet: O(dt^2) fluctuation only)."""
    md, x, p, occ, C = _hop_rich(16, 81)
    ctx = P.Context(md, 16)
    ctx.set_state(x, p, occ, C)
    ob = ctx.observables()
    E0 = ob["ke"] + ob["epot"]
    ctx.run(10.0, 400, seed=3)
    assert ctx.counters()[1].sum() > 0
    ob = ctx.observables()
    E1 = ob["ke"] + ob["epot"]
    assert np.abs(E1 - E0).max() < 1e-6 * np.abs(E0).max() + 1e-7
