"""The allocation-free hop-probability entry point.

Callers that cannot allocate device memory (a host framework that owns the
device memory through its own pool, a latency-critical loop that cannot pay
for an allocation) use iesh_hop_probabilities_noalloc, which works in a
fixed array inside the library.  This file is collected last so that a run
stopping at the first failure has run every other test first.  It checks,
through the C-ABI, that two calls in a row give the same hop probabilities
as the context entry point iesh_hop_probabilities, at the tolerance of the
other hop-probability parity tests, and that an oversized request is refused.
"""
import numpy as np
import pytest

import iesh_inputs as W

pytestmark = pytest.mark.gpu


def test_noalloc_matches_context_entry_point_twice():
    import torch

    from paper_2212_00518_gb300 import build as B
    B.build()
    import paper_2212_00518_gb300 as P
    from paper_2212_00518_gb300 import iesh

    assert torch.cuda.is_available()
    md = W.desorption(1.0, 50)  # position-dependent coupling (kappa != 0)
    n, dt = 24, 4.0
    N, Ne = md["M"] + 1, md["Ne"]
    rng = np.random.default_rng(5)
    x = rng.uniform(W.angstrom(1.6), W.angstrom(6.0), n)
    p = rng.normal(0.0, np.sqrt(md["mass"] * 0.02), n)
    occ = W.random_occupations(n, N, Ne, 6)
    C = W.mixed_coefficients(occ, N, 7, 0.8)

    ctx = P.Context(md, n)
    ctx.set_state(x, p, occ, C)
    g_ref = ctx.hop_probabilities(dt)
    lam, q0, _ = ctx.eigen()
    assert np.abs(g_ref).max() > 0

    dev = torch.device("cuda")
    tx = torch.from_numpy(x).to(dev)
    tp = torch.from_numpy(p).to(dev)
    tocc = torch.from_numpy(occ).to(dev)
    tC = torch.from_numpy(C).to(dev)
    tlam = torch.from_numpy(lam).to(dev)
    tq0 = torch.from_numpy(q0).to(dev)
    scale = np.abs(g_ref).max()
    for call in range(2):
        g = torch.full((n, Ne, N), float("nan"), dtype=torch.float64, device=dev)
        iesh.hop_probabilities_noalloc(md, tx, tp, tocc, tC, tlam, tq0, dt, g)
        torch.cuda.synchronize()
        err = np.abs(g.cpu().numpy() - g_ref).max()
        assert err <= 1e-9 * scale, f"call {call}: max error {err:.3e}"

    # a request larger than the fixed working array is refused
    big = md.copy()
    big["M"], big["Ne"] = 200, 100
    nb = iesh.IESH_NOALLOC_SCRATCH_BYTES // (16 * 100 * 201) + 1
    z = torch.zeros(nb, dtype=torch.float64, device=dev)
    with pytest.raises(P.IeshError, match="EINVAL"):
        iesh.hop_probabilities_noalloc(big, z, z, z, z, z, z, dt, z)
