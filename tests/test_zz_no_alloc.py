"""The allocation-free hop-probability entry point.

Callers that cannot allocate device memory (a host framework that owns the
device memory through its own pool, a latency-critical loop that cannot pay
for an allocation) use iesh_hop_probabilities_noalloc, which works in a
fixed array inside the library.  This file is collected last so that a run
stopping at the first failure has run every other test first.  Through the
C-ABI it checks that two calls in a row give the hop probabilities of the
context entry point iesh_hop_probabilities and of the FP64 oracle, at the
tolerance of the other hop-probability parity tests; that the second call
changes the device's free memory by nothing; that an oversized request is
refused; and that a small call leaves the hop kernels' shared-memory limits
high enough for a larger context captured into a CUDA graph afterwards.
"""
import numpy as np
import pytest

import iesh_inputs as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _pkg():
    from paper_2212_00518_gb300 import build as B
    B.build()
    import paper_2212_00518_gb300 as P
    from paper_2212_00518_gb300 import iesh
    return P, iesh


def _state(md, n, seed):
    N, Ne = md["M"] + 1, md["Ne"]
    rng = np.random.default_rng(seed)
    x = rng.uniform(W.angstrom(1.6), W.angstrom(6.0), n)
    p = rng.normal(0.0, np.sqrt(md["mass"] * 0.02), n)
    occ = W.random_occupations(n, N, Ne, seed + 1)
    C = W.mixed_coefficients(occ, N, seed + 2, 0.8)
    return x, p, occ, C


def test_noalloc_matches_context_and_oracle_twice():
    import torch

    P, iesh = _pkg()
    assert torch.cuda.is_available()
    md = W.desorption(1.0, 50)  # position-dependent coupling (kappa != 0)
    n, dt = 24, 4.0
    N, Ne = md["M"] + 1, md["Ne"]
    x, p, occ, C = _state(md, n, 5)

    ctx = P.Context(md, n)
    ctx.set_state(x, p, occ, C)
    g_ref = ctx.hop_probabilities(dt)
    lam, q0, _ = ctx.eigen()
    assert np.abs(g_ref).max() > 0
    # the oracle's hop probabilities from its own dense eigenpairs
    B = O.bind(md)
    g_orc = np.zeros_like(g_ref)
    for t in range(n):
        _, _, _, d_o, _ = O.eigen(B, x[t])
        g_orc[t], _, _, rc = O.hop_probs(occ[t], C[t].T, d_o, p[t] / md["mass"], dt)
        assert rc == 0

    dev = torch.device("cuda")
    tx, tp, tocc, tC, tlam, tq0 = (torch.from_numpy(a).to(dev) for a in (x, p, occ, C, lam, q0))
    scale = np.abs(g_ref).max()
    g = torch.full((n, Ne, N), float("nan"), dtype=torch.float64, device=dev)
    for call in range(2):
        g.fill_(float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        iesh.hop_probabilities_noalloc(md, tx, tp, tocc, tC, tlam, tq0, dt, g)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:  # the first call may load kernels; the second allocates nothing
            assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
        gh = g.cpu().numpy()
        err = np.abs(gh - g_ref).max()
        assert err <= 1e-9 * scale, f"call {call}: max error vs context {err:.3e}"
        for t in range(n):
            s = max(np.abs(g_orc[t]).max(), 1e-300)
            e = np.abs(gh[t] - g_orc[t]).max()
            assert e <= 1e-9 * s, f"call {call}, traj {t}: max error vs oracle {e:.3e}"

    # a request larger than the fixed working array is refused
    big = md.copy()
    big["M"], big["Ne"] = 200, 100
    nb = iesh.IESH_NOALLOC_SCRATCH_BYTES // (16 * 100 * 201) + 1
    z = torch.zeros(nb, dtype=torch.float64, device=dev)
    with pytest.raises(P.IeshError, match="EINVAL"):
        iesh.hop_probabilities_noalloc(big, z, z, z, z, z, z, dt, z)


def test_small_noalloc_call_keeps_room_for_a_captured_larger_context():
    """A context whose hop kernel needs more than the default 48 KB of shared
    memory still launches inside a CUDA graph after a small allocation-free
    call ran eagerly, and the replay equals an eager run."""
    import torch

    P, iesh = _pkg()
    dev = torch.device("cuda")
    big = W.desorption(1.0, 200)  # N = 201, Ne = 100: the FP64 LU hop kernel
    n, dt, steps = 4, 4.0, 2
    x, p, occ, C = _state(big, n, 31)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        cap = P.Context(big, n, stream=side.cuda_stream)
        ref = P.Context(big, n, stream=side.cuda_stream)
        cap.set_state(x, p, occ, C)
        ref.set_state(x, p, occ, C)
    torch.cuda.synchronize()

    small = W.desorption(1.0, 20)
    xs, ps, occs, Cs = _state(small, 3, 41)
    sctx = P.Context(small, 3)
    sctx.set_state(xs, ps, occs, Cs)
    lam, q0, _ = sctx.eigen()
    ts = [torch.from_numpy(a).to(dev) for a in (xs, ps, occs, Cs, lam, q0)]
    gs = torch.zeros((3, small["Ne"], small["M"] + 1), dtype=torch.float64, device=dev)
    iesh.hop_probabilities_noalloc(small, *ts, dt, gs)
    torch.cuda.synchronize()

    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        cap.run(dt, steps, seed=3)
    graph.replay()
    with torch.cuda.stream(side):
        ref.run(dt, steps, seed=3)
    torch.cuda.synchronize()
    a, b = cap.get_state(), ref.get_state()
    assert np.array_equal(a["occ"], b["occ"])
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["C"], b["C"])
    assert not np.any(a["status"] & (iesh.TRAJ_NAN | iesh.TRAJ_SINGULAR))
    for c in (cap, ref, sctx):
        c.close()
