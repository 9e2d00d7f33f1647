"""hk.CrossSectionFn: the adjoint kernel behind torch.autograd, end to end.

loss = sum_k sum_i g_k,i sigma_k,i for a few (T, P) points of one species;
loss.backward() must give dL/dT, dL/dP per point and dL/dS_ref, dL/dgamma_ref
per line equal to the FP64 oracle's gradient (chain rule of Sect. 2.2 /
2.2.2 through S(T), alpha_D(T), Gamma_L(T, P) and w'(z), with upstream
gradient g) within the gradient tolerance: 1e-4 relative per point, 1e-4
relative L2 per line.
"""
import numpy as np
import pytest

import oracle
from paper_2101_02005_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Q = synth.partition_function
QREF = float(Q(296.0))


@pytest.fixture(scope="module")
def hk():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2101_02005_gb300 import build
    build.build()
    from paper_2101_02005_gb300 import hk
    hk.lib()
    return hk


def test_autograd_function_matches_oracle_gradient(hk):
    w = synth.config(0, scale=0.03)                # 300 lines, 0-3000 cm^-1 @ 0.1, cut 25
    L = w.species[0]
    grid = hk.make_grid(*w.grid.astuple())
    opts = hk.make_opts(QREF, w.cut, hk.HK_FP32C)
    D = hk.DeviceLines.from_host(L)
    pts = [(1000.0, 1.0), (450.0, 0.02), (2200.0, 7.0)]
    dev = torch.device("cuda")
    T = torch.tensor([t for t, _ in pts], dtype=torch.float64, device=dev, requires_grad=True)
    P = torch.tensor([p for _, p in pts], dtype=torch.float64, device=dev, requires_grad=True)
    S_ref = D.S_ref.clone().requires_grad_(True)
    gam = D.gamma_ref.clone().requires_grad_(True)
    sigma = hk.CrossSectionFn.apply(T, P, S_ref, gam, D, grid, opts,
                                    lambda t: float(Q(t)), lambda t: float(synth.dlnQ_dT(t)))
    hk.hk_sync_status()
    assert sigma.shape == (len(pts), w.grid.nbins)
    g = torch.from_numpy(np.random.default_rng(11).standard_normal(
        (len(pts), w.grid.nbins)).astype(np.float32)).to(dev)
    loss = (g.to(sigma.dtype) * sigma).sum()
    loss.backward()
    hk.hk_sync_status()
    assert T.grad.dtype == torch.float64 and T.grad.device == T.device
    assert S_ref.grad.shape == S_ref.shape and gam.grad.shape == gam.shape

    oS, oG = np.zeros(L.n), np.zeros(L.n)
    gn = g.cpu().numpy().astype(np.float64)
    for k, (t, p) in enumerate(pts):
        _, _, oT, oP = oracle.backward(L.as_oracle(), w.grid.astuple(),
                                       (t, p, float(Q(t)), QREF, float(synth.dlnQ_dT(t))),
                                       w.cut, gn[k], oS, oG)
        assert abs(T.grad[k].item() - oT) <= 1e-4 * abs(oT), (k, T.grad[k].item(), oT)
        assert abs(P.grad[k].item() - oP) <= 1e-4 * abs(oP), (k, P.grad[k].item(), oP)
    dS = S_ref.grad.double().cpu().numpy()
    dG = gam.grad.double().cpu().numpy()
    eS = np.linalg.norm(dS - oS) / np.linalg.norm(oS)
    eG = np.linalg.norm(dG - oG) / np.linalg.norm(oG)
    assert eS <= 1e-4 and eG <= 1e-4, (eS, eG)

    # the forward values themselves: sigma_k against the oracle at each point
    from parity import assert_sigma_close
    for k, (t, p) in enumerate(pts):
        ref = oracle.cross_section(L.as_oracle(), w.grid.astuple(), (t, p, float(Q(t)), QREF),
                                   w.cut)
        assert_sigma_close(sigma[k].detach().double().cpu().numpy(), ref, f"autograd fwd {k}")
