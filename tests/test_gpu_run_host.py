"""iesh_run_host: a batch held in host memory advanced with the copies
overlapped with the steps, over trajectory ranges.

It must give the same bytes as iesh_checkpoint_load + iesh_run +
iesh_checkpoint_save of the whole batch. The step kernels treat
trajectories independently, so cutting the batch into ranges changes no
arithmetic. Checked for FP64 and mixed, for several range counts (including
ranges of unequal size and more ranges than fit evenly), with the output in
place and in a separate pinned buffer, and for the refusals.
"""
import numpy as np
import pytest

import iesh_inputs as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_2212_00518_gb300 import build as B
    B.build()
    import paper_2212_00518_gb300 as pkg
    return pkg


def _state(md, n, seed):
    N = md["M"] + 1
    kT = np.array([0.005, 0.0075, 0.01])[np.arange(n) % 3]
    x, p = W.thermal_harmonic(n, md["mass"], md["par"][0], kT, seed=seed)
    occ = W.lowest_occupations(n, md["Ne"])
    C = W.mixed_coefficients(occ, N, seed + 1, 0.3)
    return x, p, occ, C


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("chunks", [1, 3, 7])
def test_run_host_equals_load_run_save(P, precision, chunks):
    import torch
    md = W.double_well(100)
    n = 101  # not a multiple of the range counts
    x, p, occ, C = _state(md, n, 11)
    C = C if precision == P.PREC_FP64 else C.astype(np.complex64)
    a = P.Context(md, n, precision=precision)
    a.set_state(x, p, occ, C)
    a.run(1.0, 2, seed=3)
    blob = a.checkpoint_save()
    ref = P.Context(md, n, precision=precision)
    ref.checkpoint_load(blob)
    ref.run(1.0, 3, seed=3)
    want = ref.checkpoint_save()
    want_state = ref.get_state()
    ref.close()
    b = P.Context(md, n, precision=precision)
    src = torch.from_numpy(blob.copy()).pin_memory()
    dst = torch.zeros_like(src).pin_memory()
    b.run_host(src, dst, 1.0, 3, seed=3, chunks=chunks)
    assert np.array_equal(dst.numpy(), want)
    got = b.get_state()
    for k in ("x", "p", "occ", "C", "status"):
        assert np.array_equal(got[k], want_state[k]), k
    # in place, twice: the same as six steps
    c = P.Context(md, n, precision=precision)
    buf = torch.from_numpy(blob.copy()).pin_memory()
    c.run_host(buf, buf, 1.0, 3, seed=3, chunks=chunks)
    assert np.array_equal(buf.numpy(), want)
    c.run_host(buf, buf, 1.0, 3, seed=3, chunks=chunks)
    ref = P.Context(md, n, precision=precision)
    ref.checkpoint_load(blob)
    ref.run(1.0, 6, seed=3)
    assert np.array_equal(buf.numpy(), ref.checkpoint_save())
    for ctx in (a, b, c, ref):
        ctx.close()


def test_run_host_refusals(P):
    md = W.double_well(20)
    n = 8
    x, p, occ, C = _state(md, n, 21)
    a = P.Context(md, n)
    a.set_state(x, p, occ, C)
    blob = a.checkpoint_save()
    # records on: not trajectory-major
    r = P.Context(md, n, record_every=1, max_records=4)
    with pytest.raises(P.iesh.IeshError):
        r.run_host(blob, blob.copy(), 1.0, 1)
    # another model size
    other = P.Context(W.double_well(30), n)
    with pytest.raises(P.iesh.IeshError):
        other.run_host(blob, blob.copy(), 1.0, 1)
    # device buffers: the call is for host memory
    import torch
    dev = torch.from_numpy(blob).cuda()
    with pytest.raises(P.iesh.IeshError):
        a.run_host(dev, dev, 1.0, 1)
    for ctx in (a, r, other):
        ctx.close()
