"""GPU parity of the mixed-precision path (IESH_PREC_MIXED) with the FP64 oracle.

Mixed path: eigen iteration (with double-float pole sums), forces, the hop
selection and the rescale in FP64; coupling generator, Chebyshev propagation,
coefficients and the determinant ratios in FP32 (a Gauss-Jordan elimination
in registers for N <= 128, Ne <= 56, with the rows past 128 in shared memory
for N <= 256, Ne <= 112, the couplings in g also FP32; an LU with
substitutions when a hop CTA size is set).  The
propagator runs on the tensor cores (3xTF32, tcgen05) for N <= 128 and
Ne <= 56 and as a register-tiled SIMT kernel otherwise, or when a propagator
shape (4, G) is set; both are checked here.  Stated error per output (against the FP64 oracle,
from shared states; measured values on GB300 in brackets):
  hop probabilities g      relative to max g        2e-6   [3.8e-7]
  coefficients C, 1 step   absolute (unit columns)  1e-6   [1.8e-7]
  coefficients C, 100 steps                         3e-5   [7.4e-6]
  wavefunction P_d, 100 steps                       2e-5   [5.6e-6]
  occupied-surface P_d, x, p, force                 FP64 tolerance when the hop
                                                    decisions agree (they do here)
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


CASES = {
    "paper40": (W.double_well_paper(40), 10.0, 8.0),
    "dw100": (W.double_well(100), 1.0, 0.0),
    "dw200": (W.double_well(200), 1.0, 0.0),
}


def _state(md, n, seed, weight, shift):
    N, Ne = md["M"] + 1, md["Ne"]
    x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], 0.01, seed)
    occ = W.random_occupations(n, N, Ne, seed + 1)
    C = W.mixed_coefficients(occ, N, seed + 2, weight)
    return x + shift, p, occ, C


@pytest.mark.parametrize("name,kernel", [(k, "default") for k in CASES] +
                         [("dw100", "simt"), ("paper40", "simt"), ("dw200", "simt")])
def test_mixed_one_step(P, name, kernel):
    md, dt, shift = CASES[name]
    n = 8
    x, p, occ, C = _state(md, n, 5, 0.6, shift)
    B = O.bind(md)
    ctx = P.Context(md, n, precision=P.PREC_MIXED)
    if kernel == "simt":
        ctx.set_kernel_shape(4, 1, 0)
    else:
        assert ctx.kernel_shape()[0] in ((8, 16) if md["M"] + 1 <= 128 else (4,))
    ctx.set_state(x, p, occ, C.astype(np.complex64))
    g = ctx.hop_probabilities(dt)
    gref = []
    for t in range(n):
        d_o = O.eigen(B, x[t])[3]
        gref.append(O.hop_probs(occ[t], C[t].T, d_o, p[t] / md["mass"], dt)[0])
    gref = np.array(gref)
    assert np.abs(g - gref).max() <= 2e-6 * np.abs(gref).max()
    ctx.run(dt, 1, seed=9)
    st = ctx.get_state()
    for t in range(n):
        r = O.step_one(B, x[t], p[t], occ[t].astype(np.int32), C[t].T, dt, seed=9, traj=t, n=0)
        assert np.array_equal(st["occ"][t], r["occ"])
        assert abs(st["x"][t] - r["x"]) <= 1e-13 * (1 + abs(r["x"]))
        assert np.abs(st["C"][t].T - r["C"]).max() <= 1e-6


@pytest.mark.parametrize("M,Ne,n", [(128, 1, 6), (200, 100, 4), (200, 33, 4), (160, 80, 4), (255, 112, 2),
                                     (120, 60, 4)])
def test_mixed_large_and_ragged_shapes(P, M, Ne, n):
    """Mixed step on shapes past the tensor-core kernel (N > 128 or
    Ne > 56): one orbital past a 128-row tile (N = 129, Ne = 1), the M = 200
    bath with Ne = 100 and with a ragged Ne = 33, Ne = 80 at N = 161, the
    largest sizes (N = 256, Ne = 112) and N = 121 with Ne = 60 > 56.  The
    SIMT propagator and the Gauss-Jordan kernel with shared-memory rows serve
    them; one step against the oracle, and the hop probabilities against the
    LU kernel's."""
    md = W.double_well(M, Ne)
    N = M + 1
    x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], 0.01, 21)
    occ = W.random_occupations(n, N, Ne, 22)
    C = W.mixed_coefficients(occ, N, 23, 0.6)
    B = O.bind(md)
    ctx = P.Context(md, n, precision=P.PREC_MIXED)
    assert ctx.kernel_shape()[0] == (32 if N > 224 else 4)
    ctx.set_state(x, p, occ, C.astype(np.complex64))
    g_gj = ctx.hop_probabilities(1.0)
    ctx.set_kernel_shape(0, 0, 512)
    g_lu = ctx.hop_probabilities(1.0)
    ctx.set_kernel_shape(0, 0, 0)
    assert np.abs(g_gj - g_lu).max() <= 2e-6 * max(np.abs(g_lu).max(), 1e-300)
    ctx.run(1.0, 1, seed=4)
    st = ctx.get_state()
    ctx.close()
    assert np.all(st["status"] == 0)
    for t in range(n):
        r = O.step_one(B, x[t], p[t], occ[t].astype(np.int32), C[t].T, 1.0, seed=4, traj=t, n=0)
        assert np.array_equal(st["occ"][t], r["occ"])
        assert abs(st["x"][t] - r["x"]) <= 1e-13 * (1 + abs(r["x"]))
        assert np.abs(st["C"][t].T - r["C"]).max() <= 1e-6


@pytest.mark.parametrize("name", ["paper40", "dw100", "dw200"])
def test_mixed_hop_kernels_agree(P, name):
    """The mixed path's two ratio algorithms: the built-in Gauss-Jordan
    elimination (in registers for N <= 128, Ne <= 56; with the rows past 128
    in shared memory up to N = 256, Ne = 112) and the LU kernel (chosen by a
    hop CTA size of 256 or 512 threads) each match the oracle's hop
    probabilities within the mixed bound, and so each other."""
    md, dt, shift = CASES[name]
    n = 8
    x, p, occ, C = _state(md, n, 15, 0.6, shift)
    B = O.bind(md)
    gref = np.array([O.hop_probs(occ[t], C[t].T, O.eigen(B, x[t])[3], p[t] / md["mass"], dt)[0]
                     for t in range(n)])
    got = {}
    for hop in (0, 256, 512):
        ctx = P.Context(md, n, precision=P.PREC_MIXED)
        ctx.set_kernel_shape(0, 0, hop)
        ctx.set_state(x, p, occ, C.astype(np.complex64))
        got[hop] = ctx.hop_probabilities(dt)
        ctx.close()
        assert np.abs(got[hop] - gref).max() <= 2e-6 * np.abs(gref).max(), hop
    assert np.abs(got[0] - got[256]).max() <= 2e-6 * np.abs(gref).max()
    assert np.abs(got[256] - got[512]).max() <= 1e-7 * np.abs(gref).max()


@pytest.mark.parametrize("name,kernel", [("paper40", "default"), ("dw100", "default"), ("dw100", "simt"),
                                         ("dw200", "default")])
def test_mixed_100_steps(P, name, kernel):
    md, dt, shift = CASES[name]
    n, steps, every = 8, 100, 20
    if md["M"] + 1 > 128:  # the FP64 oracle takes about 0.1 s per step here
        n, steps, every = 4, 40, 20
    x, p, occ, C = _state(md, n, 5, 0.6, shift)
    B = O.bind(md)
    ctx = P.Context(md, n, precision=P.PREC_MIXED, record_every=every, max_records=steps // every)
    if kernel == "simt":
        ctx.set_kernel_shape(4, 1, 0)
    ctx.set_state(x, p, occ, C.astype(np.complex64))
    ctx.run(dt, steps, seed=3)
    st = ctx.get_state()
    sh, wf = ctx.records(steps // every)
    _, F = ctx.eigen()[1:]
    ref = O.run(B, x, p, occ.astype(np.int32), np.transpose(C, (0, 2, 1)), dt, steps, seed=3,
                record_every=every)
    assert np.array_equal(st["occ"], ref["occ"])
    assert np.abs(np.transpose(st["C"], (0, 2, 1)) - ref["C"]).max() <= 3e-5
    assert np.abs(wf - ref["pop_wf"]).max() <= 2e-5
    assert np.abs(sh - ref["pop_sh"]).max() <= 1e-10
    assert np.abs(st["x"] - ref["x"]).max() <= 1e-10 * np.abs(ref["x"]).max()
    assert np.abs(st["p"] - ref["p"]).max() <= 1e-10 * np.abs(ref["p"]).max()
    Fo = np.array([O.eigen(B, st["x"][t], st["occ"][t].astype(np.int32))[4] for t in range(n)])
    assert np.abs(F - Fo).max() <= 1e-10 * (np.abs(Fo).max() + 1e-3)


def test_mixed_hop_decisions_on_hop_rich_case(P):
    """Strong-coupling paper double well: mixed and FP64 paths take the same
    hop decisions as the oracle over 200 steps (g agrees to ~1e-7 relative,
    so only uniforms within that distance of a boundary could differ)."""
    md = W.double_well_paper(8)
    md["Gamma"] = 0.02
    n, steps, dt = 32, 200, 10.0
    x, p, occ, C = _state(md, n, 41, 1.0, 8.0)
    ctx = P.Context(md, n, precision=P.PREC_MIXED)
    ctx.set_state(x, p, occ, C.astype(np.complex64))
    ctx.run(dt, steps, seed=123)
    st = ctx.get_state()
    _, hops, fr = ctx.counters()
    ref = O.run(O.bind(md), x, p, occ.astype(np.int32), np.transpose(C, (0, 2, 1)), dt, steps,
                seed=123)
    assert ref["hops"].sum() > 0
    agree = np.mean([np.array_equal(st["occ"][t], ref["occ"][t]) and hops[t] == ref["hops"][t]
                     for t in range(n)])
    assert agree >= 0.9, agree


@pytest.mark.parametrize("name", ["paper40", "dw100", "dw200"])
def test_mixed_eigenpairs_double_float_accuracy(P, name):
    """The mixed path forms the secular pole sums in double-float arithmetic
    (about 48 bits).  Stated error of the eigenpairs against the oracle's
    Jacobi eigenpairs: 1e-12 relative for lambda, 1e-11 for q0, after a
    cold start and after 5 warm-started steps."""
    md, dt, shift = CASES[name]
    n = 4
    x, p, occ, C = _state(md, n, 17, 0.5, shift)
    B = O.bind(md)
    ctx = P.Context(md, n, precision=P.PREC_MIXED)
    ctx.set_state(x, p, occ, C.astype(np.complex64))
    for steps in (0, 5):
        if steps:
            ctx.run(dt, steps, seed=1)
        xs = ctx.get_state()["x"]
        lam, q0, _ = ctx.eigen()
        for t in range(n):
            lo, Qo = O.eigen(B, xs[t])[:2]
            scale = np.abs(lo).max()
            assert np.abs(lam[t] - lo).max() <= 1e-12 * scale
            assert np.abs(q0[t] - Qo[0]).max() <= 1e-11


def test_mixed_two_lead_eigenpairs(P):
    md = W.morse_image(50, bias=0.1)
    n = 4
    x = np.linspace(W.angstrom(1.8), W.angstrom(6.0), n)
    p = np.zeros(n)
    occ = W.lowest_occupations(n, md["Ne"])
    C = W.unit_coefficients(occ, 51).astype(np.complex64)
    ctx = P.Context(md, n, precision=P.PREC_MIXED)
    ctx.set_state(x, p, occ, C)
    lam, q0, _ = ctx.eigen()
    B = O.bind(md)
    for t in range(n):
        lo, Qo = O.eigen(B, x[t])[:2]
        assert np.abs(lam[t] - lo).max() <= 1e-12 * np.abs(lo).max()
        assert np.abs(q0[t] - Qo[0]).max() <= 1e-11


@pytest.mark.parametrize("M,Ne,n", [(200, 100, 6), (255, 112, 3), (128, 1, 5), (160, 80, 4), (200, 33, 4)])
def test_mixed_two_quad_propagator_identical(P, M, Ne, n):
    """The SIMT propagator with two row quads per thread (shape 32) computes
    every entry with the same FP32 operations in the same order as the
    one-quad kernel (shape 4), so one step gives bit-identical states; and
    both agree with the oracle at the mixed bounds."""
    md = W.double_well(M, Ne)
    N = M + 1
    x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], 0.01, 31)
    occ = W.random_occupations(n, N, Ne, 32)
    C = W.mixed_coefficients(occ, N, 33, 0.6).astype(np.complex64)
    out = {}
    for ept in (4, 32):
        ctx = P.Context(md, n, precision=P.PREC_MIXED)
        ctx.set_state(x, p, occ, C)
        ctx.set_kernel_shape(ept, 1, 0)
        ctx.run(1.0, 2, seed=6)
        out[(ept, 1)] = ctx.get_state()
        ctx.close()
    ctx = P.Context(md, n, precision=P.PREC_MIXED)
    ctx.set_state(x, p, occ, C)
    ctx.set_kernel_shape(32, 3, 0)
    ctx.run(1.0, 2, seed=6)
    out[(32, 3)] = ctx.get_state()
    ctx.close()
    a = out[(4, 1)]
    for key in ((32, 1), (32, 3)):
        b = out[key]
        assert np.array_equal(a["C"], b["C"]), key
        assert np.array_equal(a["occ"], b["occ"]) and np.array_equal(a["x"], b["x"]), key
    B = O.bind(md)
    ctx = P.Context(md, n, precision=P.PREC_MIXED)
    ctx.set_state(x, p, occ, C)
    ctx.set_kernel_shape(32, 2, 0)
    ctx.run(1.0, 1, seed=4)
    st = ctx.get_state()
    ctx.close()
    for t in range(n):
        r = O.step_one(B, x[t], p[t], occ[t].astype(np.int32), C[t].T.astype(np.complex128), 1.0, seed=4,
                       traj=t, n=0)
        assert np.array_equal(st["occ"][t], r["occ"])
        assert np.abs(st["C"][t].T - r["C"]).max() <= 1e-6


@pytest.mark.parametrize("M,Ne,n", [(100, 50, 6), (20, 10, 8), (110, 50, 4), (64, 1, 4), (9, 4, 3)])
def test_mixed_fp16_tensor_core_propagator(P, M, Ne, n):
    """The tensor-core propagator on FP16 split operands (shape 16: scaled
    hi + lo FP16 pairs, about 22 bits each, the Chebyshev sum in tensor
    memory): one step against the oracle at the mixed bounds, and against
    the 3xTF32 kernel where that one fits (both within about 2^-22 of |W||T|
    per order; at N = 111 only the FP16 kernel's shared memory fits)."""
    md = W.double_well(M, Ne)
    N = M + 1
    x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], 0.01, 41)
    occ = W.random_occupations(n, N, Ne, 42)
    C = W.mixed_coefficients(occ, N, 43, 0.6).astype(np.complex64)
    out = {}
    for ept in (8, 16):
        ctx = P.Context(md, n, precision=P.PREC_MIXED)
        ctx.set_state(x, p, occ, C)
        try:
            ctx.set_kernel_shape(ept, 1, 0)
        except P.IeshError:
            assert ept == 8 and M == 110
            ctx.close()
            continue
        ctx.run(1.0, 1, seed=4)
        out[ept] = ctx.get_state()
        ctx.close()
    st = out[16]
    assert np.all(st["status"] == 0)
    if 8 in out:
        assert np.abs(st["C"] - out[8]["C"]).max() <= 2e-6
    B = O.bind(md)
    for t in range(n):
        r = O.step_one(B, x[t], p[t], occ[t].astype(np.int32), C[t].T.astype(np.complex128), 1.0, seed=4,
                       traj=t, n=0)
        assert np.array_equal(st["occ"][t], r["occ"])
        assert abs(st["x"][t] - r["x"]) <= 1e-13 * (1 + abs(r["x"]))
        assert np.abs(st["C"][t].T - r["C"]).max() <= 1e-6
