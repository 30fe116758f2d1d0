"""GPU parity at the benchmark's full sizes, in the launch configurations the
benchmark times, on sampled trajectories.

The two workloads are the double-well IESH batches:
- M = 100, Ne = 50, 4096 trajectories;
- M = 200, Ne = 100, 8192 trajectories.

Each test takes one step from a shared seeded state, FP64 and mixed, and checks
sampled trajectories against the oracle's step, one trajectory at a time. The
first, middle and last trajectories are always sampled. The coefficients start
near the occupied orbitals with every amplitude nonzero, so the propagation and
the hop probabilities do real work.

Tolerances:
- FP64: 1e-10 relative to each quantity's scale; occupations bit-exact.
- Mixed: the one-step bounds of the mixed path. Positions are within
  1e-13 relative, because the force is FP64 and taken before the FP32
  propagation. Momenta are within 1e-6, the stated bound for forces from the
  double-float secular sums. C is within 1e-6. Occupations are bit-exact.
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


def _workload(M, n, seed):
    """The benchmark's batch: kT cycling over 0.005, 0.0075, 0.01; thermal
    nuclei; lowest occupations; coefficients near them (64 distinct ones
    tiled over the batch to keep the set-up cheap)."""
    md = W.double_well(M)
    kT = np.array([0.005, 0.0075, 0.01])[np.arange(n) % 3]
    x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], kT, seed=seed)
    occ = W.lowest_occupations(n, md["Ne"])
    C = W.mixed_coefficients(occ[:64], md["M"] + 1, seed + 1, 0.3)
    C = np.concatenate([C] * (n // 64))
    return md, x, p, occ, C


def _check(P, md, x, p, occ, C, precision, samples, rtol_c, rtol_p):
    n = x.shape[0]
    ctx = P.Context(md, n, precision=precision)
    ctx.set_state(x, p, occ, C if precision == P.PREC_FP64 else C.astype(np.complex64))
    ctx.run(1.0, 1, seed=0)
    st = ctx.get_state()
    ctx.close()
    assert np.all(st["status"] == 0)
    B = O.bind(md)
    Cref = C if precision == P.PREC_FP64 else C.astype(np.complex64).astype(np.complex128)
    for t in samples:
        r = O.step_one(B, x[t], p[t], occ[t].astype(np.int32), Cref[t].T, 1.0, seed=0, traj=t, n=0)
        assert np.array_equal(st["occ"][t], r["occ"]), t
        assert abs(st["x"][t] - r["x"]) <= 1e-13 * (abs(r["x"]) + 1.0), t
        assert abs(st["p"][t] - r["p"]) <= rtol_p * (abs(r["p"]) + 1e-3), t
        err = np.abs(st["C"][t].T - r["C"]).max()
        assert err <= rtol_c, (t, err)


def test_config3_fp64_one_step_sampled(P):
    md, x, p, occ, C = _workload(200, 8192, 31)
    _check(P, md, x, p, occ, C, P.PREC_FP64, (0, 1, 4095, 8191), 1e-10, 1e-10)


def test_config2_mixed_one_step_sampled(P):
    md, x, p, occ, C = _workload(100, 4096, 41)
    _check(P, md, x, p, occ, C, P.PREC_MIXED, (0, 1, 777, 2048, 4095), 1e-6, 1e-6)


def test_config3_mixed_one_step_sampled(P):
    md, x, p, occ, C = _workload(200, 8192, 51)
    _check(P, md, x, p, occ, C, P.PREC_MIXED, (0, 3, 4096, 8191), 1e-6, 1e-6)
