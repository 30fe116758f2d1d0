"""GPU parity of the differentiable occupied-orbital energy E_occ(x, theta)
(two adsorbate orbitals on a Gauss-Legendre band, six coordinates, 16
parameters) with the FP64 oracle's dense Jacobi diagonalisation, with
central finite differences (h = 1e-5), and through torch.autograd.

Stated tolerances: FP64 kernels 1e-10 relative (energies) and 1e-9 of the
largest gradient component; FP32 kernels (the fast forward) 2e-6 relative
for E and 1e-3 of the largest gradient component against the FP64 oracle.
"""
import numpy as np
import pytest

import iesh_inputs as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_2212_00518_gb300 import build as B
    B.build()
    from paper_2212_00518_gb300 import eocc as E
    return torch, E


def _oracle(wl, x, theta):
    eps, sqw = O.bath(dict(band=wl["band"], M=wl["M"], mu=0.0, disc="gl"))
    return O.eocc(eps, sqw, wl["Vbar"], wl["R"], x, theta, wl["Ne"])


@pytest.mark.parametrize("M,B", [(24, 8), (40, 6), (300, 2)])
def test_eocc_fp64_matches_oracle(env, M, B):
    torch, E = env
    wl = W.eocc_workload(M=M, B=B, seed=5)
    model = E.EOccModel(wl)
    x = torch.tensor(wl["x"], device="cuda")
    th = torch.tensor(wl["theta"], device="cuda")
    Eg, saved, status = model.forward(x, th)
    assert int(status.abs().sum()) == 0
    gE = torch.ones(B, dtype=torch.float64, device="cuda")
    dx, dth = model.backward(x, th, saved, gE)
    Eo, dxo, dtho = _oracle(wl, wl["x"], wl["theta"])
    scale = np.abs(Eo).max()
    assert np.abs(Eg.cpu().numpy() - Eo).max() <= 1e-10 * scale
    gs = max(np.abs(dxo).max(), np.abs(dtho).max())
    assert np.abs(dx.cpu().numpy() - dxo).max() <= 1e-9 * gs
    assert np.abs(dth.cpu().numpy() - dtho.sum(0)).max() <= 1e-9 * gs * B


def test_eocc_gradients_match_finite_differences(env):
    torch, E = env
    wl = W.eocc_workload(M=300, B=8, seed=5)
    model = E.EOccModel(wl)
    x = torch.tensor(wl["x"], device="cuda")
    th = torch.tensor(wl["theta"], device="cuda")
    _, saved, _ = model.forward(x, th)
    dx, _ = model.backward(x, th, saved, torch.ones(8, dtype=torch.float64, device="cuda"))
    h = 1e-5
    for al in range(6):
        e = torch.zeros_like(x)
        e[:, al] = h
        fd = (model.forward(x + e, th)[0] - model.forward(x - e, th)[0]) / (2 * h)
        assert torch.abs(fd - dx[:, al]).max().item() < 1e-7
    # parameter gradients of the summed energy
    _, saved, _ = model.forward(x, th)
    _, dth = model.backward(x, th, saved, torch.ones(8, dtype=torch.float64, device="cuda"))
    for p in range(16):
        e = torch.zeros_like(th)
        e[p] = h
        fd = (model.forward(x, th + e)[0].sum() - model.forward(x, th - e)[0].sum()) / (2 * h)
        assert abs(fd.item() - dth[p].item()) < 1e-6, p


def test_eocc_fp32_forward_error(env):
    torch, E = env
    wl = W.eocc_workload(M=300, B=3, seed=5)
    model = E.EOccModel(wl)
    x = torch.tensor(wl["x"], device="cuda", dtype=torch.float32)
    th = torch.tensor(wl["theta"], device="cuda", dtype=torch.float32)
    Ef, saved, status = model.forward(x, th)
    assert int(status.abs().sum()) == 0
    dx, dth = model.backward(x, th, saved, torch.ones(3, dtype=torch.float32, device="cuda"))
    # the oracle at the FP32-rounded inputs
    Eo, dxo, dtho = _oracle(wl, x.double().cpu().numpy(), th.double().cpu().numpy())
    assert np.abs(Ef.double().cpu().numpy() - Eo).max() <= 2e-6 * np.abs(Eo).max()
    gs = max(np.abs(dxo).max(), np.abs(dtho).max())
    assert np.abs(dx.double().cpu().numpy() - dxo).max() <= 1e-3 * gs
    assert np.abs(dth.double().cpu().numpy() - dtho.sum(0)).max() <= 1e-3 * gs * 3


def test_eocc_autograd(env):
    torch, E = env
    wl = W.eocc_workload(M=40, B=5, seed=7)
    model = E.EOccModel(wl)
    x = torch.tensor(wl["x"], device="cuda", requires_grad=True)
    th = torch.tensor(wl["theta"], device="cuda", requires_grad=True)
    w = torch.linspace(0.5, 1.5, 5, dtype=torch.float64, device="cuda")
    loss = (E.eocc(x, th, model) * w).sum()
    loss.backward()
    Eo, dxo, dtho = _oracle(wl, wl["x"], wl["theta"])
    wn = w.cpu().numpy()
    assert abs(loss.item() - (Eo * wn).sum()) < 1e-10 * np.abs(Eo).sum()
    assert np.abs(x.grad.cpu().numpy() - dxo * wn[:, None]).max() < 1e-9
    assert np.abs(th.grad.cpu().numpy() - (dtho * wn[:, None]).sum(0)).max() < 1e-8


def test_eocc_full_size_sampled(env):
    """65536 geometries, M=300, Ne=151 (the differentiable-energy workload),
    FP64 and FP32 forward + backward; sampled geometries against the oracle."""
    torch, E = env
    wl = W.eocc_workload(M=300, B=65536, seed=5)
    model = E.EOccModel(wl)
    x = torch.tensor(wl["x"], device="cuda")
    th = torch.tensor(wl["theta"], device="cuda")
    Eg, saved, status = model.forward(x, th)
    assert int(status.abs().sum()) == 0
    dx, _ = model.backward(x, th, saved, torch.ones(65536, dtype=torch.float64, device="cuda"))
    Ef, _, st32 = model.forward(x.float(), th.float())
    assert int(st32.abs().sum()) == 0
    idx = [0, 12345, 65535]
    Eo, dxo, _ = _oracle(wl, wl["x"][idx], wl["theta"])
    assert np.abs(Eg.cpu().numpy()[idx] - Eo).max() <= 1e-10 * np.abs(Eo).max()
    assert np.abs(dx.cpu().numpy()[idx] - dxo).max() <= 1e-9 * np.abs(dxo).max()
    assert np.abs(Ef.double().cpu().numpy() - Eg.cpu().numpy()).max() <= 1e-5 * np.abs(Eo).max()
