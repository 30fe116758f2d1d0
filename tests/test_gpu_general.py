"""GPU parity of the batched dense symmetric eigensolver (iesh_syev_batched)
and of the two-orbital dynamics whose orbitals couple to the bath with their
own profiles (non-parallel border vectors, reading R17), which take their
eigenpairs from two nested secular equations by default or from the dense
solver; both are checked against the oracle's dense Jacobi.

Tolerances follow from the method's backward error: Householder reduction
and QL rotations give the eigenpairs of A + E with |E| <= c n u |A| (u the
unit roundoff), so eigenvalues are within that of the oracle's and each
eigenvector within it divided by the gap to its neighbours.
  - FP64 solver on the random test matrices (eigenvalue gaps >= about
    |A| / n^2): eigenvalues 1e-12 |A|, eigenvectors 1e-9.
  - FP32 solver: eigenvalues, residuals |A v - lambda v| and orthogonality
    within 8 n 2^-24 (times |A| for the first two).
  - Two-orbital model (band [-0.5, 0.5], smallest Gauss-Legendre gaps about
    2e-4): eigenvalues 1e-12, adsorbate components 1e-10, forces 1e-9
    relative; one step C 1e-9; 100 steps with hops C 1e-8 with identical
    occupations and hop counts.
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


def _syev(P, A, dtype, vectors=True):
    import torch
    tA = torch.tensor(A, dtype=dtype, device="cuda")
    B, n = A.shape[0], A.shape[1]
    lam = torch.full((B, n), float("nan"), dtype=dtype, device="cuda")
    V = torch.full((B, n, n), float("nan"), dtype=dtype, device="cuda") if vectors else None
    info = torch.full((B,), 7, dtype=torch.int32, device="cuda")
    P.iesh.syev_batched(tA, lam, V, info)
    torch.cuda.synchronize()
    return (lam.cpu().numpy().astype(np.float64),
            None if V is None else V.cpu().numpy().astype(np.float64), info.cpu().numpy())


@pytest.mark.parametrize("n", [1, 2, 3, 7, 33, 64, 102, 157, 158, 201, 256])
def test_syev_fp64_matches_oracle(P, n):
    import torch
    B = 3 if n <= 158 else 2
    A = W.random_symmetric(B, n, seed=100 + n)
    lam, V, info = _syev(P, A, torch.float64)
    rl, rV, rc = O.syev(A)
    assert rc == 0 and np.all(info == 0)
    for b in range(B):
        scale = np.abs(rl[b]).max()
        assert np.abs(lam[b] - rl[b]).max() <= 1e-12 * scale
        assert np.abs(V[b] - rV[b]).max() <= 1e-9
    # values only: the same eigenvalues
    lam2, _, info2 = _syev(P, A, torch.float64, vectors=False)
    assert np.all(info2 == 0) and np.abs(lam2 - lam).max() <= 1e-12 * np.abs(rl).max()


@pytest.mark.parametrize("n", [5, 64, 150, 256])
def test_syev_fp32_residual_and_orthogonality(P, n):
    import torch
    B = 3
    A = W.random_symmetric(B, n, seed=200 + n)
    lam, V, info = _syev(P, A.astype(np.float32), torch.float32)
    rl, _, _ = O.syev(A.astype(np.float32).astype(np.float64))
    assert np.all(info == 0)
    tol = 8 * n * 2.0 ** -24
    for b in range(B):
        scale = np.abs(rl[b]).max()
        A32 = A[b].astype(np.float32).astype(np.float64)
        assert np.abs(lam[b] - rl[b]).max() <= tol * scale
        assert np.abs(A32 @ V[b].T - V[b].T * lam[b]).max() <= tol * scale
        assert np.abs(V[b] @ V[b].T - np.eye(n)).max() <= tol


def test_syev_special_matrices_and_errors(P):
    import torch
    # diagonal with repeated eigenvalues: exact eigenvalues, orthonormal vectors
    A = np.diag([3.0, -1.0, 2.0, -1.0, 0.5])[None]
    lam, V, info = _syev(P, A, torch.float64)
    assert np.all(info == 0)
    assert np.array_equal(lam[0], np.array([-1.0, -1.0, 0.5, 2.0, 3.0]))
    assert np.abs(V[0] @ V[0].T - np.eye(5)).max() <= 1e-15
    # zero matrix
    lam, V, info = _syev(P, np.zeros((2, 9, 9)), torch.float64)
    assert np.all(lam == 0.0) and np.abs(V[0] @ V[0].T - np.eye(9)).max() <= 1e-15
    # tridiagonal (the reduction has nothing to do) and 2 x 2
    T = np.diag(np.arange(6.0)) + np.diag(np.full(5, 0.3), 1) + np.diag(np.full(5, 0.3), -1)
    lam, V, info = _syev(P, T[None], torch.float64)
    assert np.abs(lam[0] - np.linalg.eigvalsh(T)).max() <= 1e-14
    A2 = np.array([[[1.0, 2.0], [2.0, -3.0]]])
    lam, V, info = _syev(P, A2, torch.float64)
    assert np.abs(lam[0] - np.linalg.eigvalsh(A2[0])).max() <= 1e-15
    # empty batch, out-of-range n, short workspace
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    P.iesh.syev_batched(torch.zeros((0, 4, 4), dtype=torch.float64, device="cuda"),
                        torch.zeros((0, 4), dtype=torch.float64, device="cuda"))
    with pytest.raises(P.IeshError, match="EINVAL"):
        P.iesh.syev_batched(torch.zeros((1, 257, 257), dtype=torch.float64, device="cuda"),
                            torch.zeros((1, 257), dtype=torch.float64, device="cuda"))
    with pytest.raises(P.IeshError, match="EINVAL"):
        P.iesh.syev_batched(torch.zeros((2, 8, 8), dtype=torch.float64, device="cuda"),
                            torch.zeros((2, 8), dtype=torch.float64, device="cuda"),
                            work=torch.zeros(16, dtype=torch.uint8, device="cuda"))
    del z


# ------------------------------------------------------- two-orbital dynamics
CASES = {
    "M20": W.two_orbital_profiled(20, seed=5),
    "M100": W.two_orbital_profiled(100, seed=7, Ne=48),
    "strong": W.two_orbital_profiled(16, seed=7, vscale=3.0),
    "M200": W.two_orbital_profiled(200, seed=8, Ne=90),   # matrix past shared memory
    "M254": W.two_orbital_profiled(254, seed=9, Ne=100),  # N = 256
}


def _ctx(P, md, x, p, occ, C, **kw):
    from paper_2212_00518_gb300 import two
    ctx = two.TwoOrbitalContext(md, x.shape[0], **kw)
    ctx.set_state(x, p, occ.astype(np.int16), C)
    return ctx


SOLVERS = ("nested", "dense")


def _solver(md, solver):
    """The model with the dense solver forced, or as is (the nested secular
    equations are the default for own profiles)."""
    return dict(md, eigensolver="dense") if solver == "dense" else md


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("name", list(CASES))
def test_profiled_eigenpairs_and_forces(P, name, solver):
    md = _solver(CASES[name], solver)
    n = 3
    x, p, occ, C = W.two_orbital_state(md, n, 11)
    ctx = _ctx(P, md, x, p, occ, C)
    lam, Q, F = ctx.eigen()
    assert np.all(ctx.get_state()["status"] == 0)
    for t in range(n):
        rl, rQ, _, rF = O.eigen2(md, x[t], occ[t])
        assert np.abs(lam[t] - rl).max() <= 1e-12
        assert np.abs(Q[t] - rQ[0:2]).max() <= 1e-10
        assert np.abs(F[t] - rF).max() <= 1e-9 * max(1.0, np.abs(rF).max())


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("name", ["M20", "M100", "strong", "M200"])
def test_profiled_one_step(P, name, solver):
    md = _solver(CASES[name], solver)
    n, dt = 4, 5.0
    x, p, occ, C = W.two_orbital_state(md, n, 17, weight=0.6)
    ctx = _ctx(P, md, x, p, occ, C)
    ctx.run(dt, 1, seed=3)
    st = ctx.get_state()
    ref = O.run2(md, x, p, occ, np.transpose(C, (0, 2, 1)), dt, 1, seed=3)
    assert np.all(st["status"] == 0)
    assert np.array_equal(st["occ"], ref["occ"])
    assert np.abs(st["x"] - ref["x"]).max() <= 1e-12 * (1 + np.abs(ref["x"]).max())
    assert np.abs(st["p"] - ref["p"]).max() <= 1e-10 * (1 + np.abs(ref["p"]).max())
    assert np.abs(np.transpose(st["C"], (0, 2, 1)) - ref["C"]).max() <= 1e-9
    lam, Q, _ = ctx.eigen()  # the step's gauge: continuity with the start
    for t in range(n):
        assert np.abs(Q[t] - ref["Qad"][t]).max() <= 1e-10


@pytest.mark.parametrize("solver", SOLVERS)
def test_profiled_100_steps_with_hops(P, solver):
    md = _solver(W.two_orbital_profiled(16, seed=7, vscale=3.0), solver)
    n, steps, dt = 8, 100, 5.0
    x, p, occ, C = W.two_orbital_state(md, n, 19, kT=0.01, weight=1.0)
    ctx = _ctx(P, md, x, p, occ, C)
    ctx.run(dt, steps, seed=5)
    st = ctx.get_state()
    _, hops, fr = ctx.counters()
    ref = O.run2(md, x, p, occ, np.transpose(C, (0, 2, 1)), dt, steps, seed=5)
    assert ref["hops"].sum() > 0, "case must hop"
    assert np.array_equal(hops, ref["hops"]) and np.array_equal(fr, ref["frustrated"])
    assert np.array_equal(st["occ"], ref["occ"])
    assert np.abs(np.transpose(st["C"], (0, 2, 1)) - ref["C"]).max() <= 1e-8
    assert np.abs(st["x"] - ref["x"]).max() <= 1e-9 * np.abs(ref["x"]).max()


def test_dense_path_equals_secular_path_on_parallel_couplings(P):
    """The dense solver forced on the parallel-coupling model reproduces the
    rank-two secular path (same gauge there)."""
    md = W.two_orbital(40, seed=6, vscale=2.0)
    dense = dict(md, eigensolver="dense")
    n, steps, dt = 6, 50, 5.0
    x, p, occ, C = W.two_orbital_state(md, n, 31, weight=0.8)
    a = _ctx(P, md, x, p, occ, C)
    b = _ctx(P, dense, x, p, occ, C)
    la, Qa, Fa = a.eigen()
    lb, Qb, Fb = b.eigen()
    assert np.abs(la - lb).max() <= 1e-12 and np.abs(Qa - Qb).max() <= 1e-10
    a.run(dt, steps, seed=2)
    b.run(dt, steps, seed=2)
    sa, sb = a.get_state(), b.get_state()
    assert np.array_equal(sa["occ"], sb["occ"])
    assert np.array_equal(a.counters()[1], b.counters()[1])
    assert np.abs(sa["C"] - sb["C"]).max() <= 1e-8


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("name", ["M20", "strong", "M100"])
def test_profiled_mixed_one_step(P, name, solver):
    """Mixed precision with FP64 eigenpairs (nested secular equations or the
    dense solver): the one-coordinate mixed bounds (C within 1e-6 after one
    step)."""
    md = _solver(CASES[name], solver)
    n, dt = 4, 5.0
    x, p, occ, C = W.two_orbital_state(md, n, 17, weight=0.6)
    C32 = C.astype(np.complex64)
    ctx = _ctx(P, md, x, p, occ, C32, precision=1)
    ctx.run(dt, 1, seed=3)
    st = ctx.get_state()
    ref = O.run2(md, x, p, occ, np.transpose(C32.astype(np.complex128), (0, 2, 1)), dt, 1, seed=3)
    assert np.all(st["status"] == 0)
    assert np.array_equal(st["occ"], ref["occ"])
    assert np.abs(st["x"] - ref["x"]).max() <= 1e-12 * (1 + np.abs(ref["x"]).max())
    assert np.abs(np.transpose(st["C"], (0, 2, 1)) - ref["C"]).max() <= 1e-6


@pytest.mark.parametrize("name", ["M20", "M100", "M254"])
def test_nested_secular_equals_dense_solver(P, name):
    """The two eigensolvers of the own-profile model give the same ordered
    eigenvalues (1e-12) and gauge-fixed adsorbate rows (1e-10) on many
    geometries."""
    md = CASES[name]
    n = 24
    x, p, occ, C = W.two_orbital_state(md, n, 29)
    a = _ctx(P, md, x, p, occ, C)
    b = _ctx(P, _solver(md, "dense"), x, p, occ, C)
    la, Qa, Fa = a.eigen()
    lb, Qb, Fb = b.eigen()
    assert np.abs(la - lb).max() <= 1e-12
    assert np.abs(Qa - Qb).max() <= 1e-10
    assert np.abs(Fa - Fb).max() <= 1e-9 * max(1.0, np.abs(Fb).max())
