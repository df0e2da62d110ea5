"""GPU parity of the differentiable filter (spl_diff_forward / spl_diff_backward, FilterLoss) against the FP64
autograd oracle (oracle/diff_oracle.py, pinned to the C oracle and to finite differences).

Tolerances. Forward states and readouts: relative 1e-4 as for the filter. Loss: relative 1e-4. Gradients are
sums over pixels x candidates x frames of FP32 products (here ~5e5 terms per component, with cancellation between
positive and negative contributions), so each component is compared with an absolute tolerance of 2e-3 times the
largest component of the same gradient plus 1e-3 relative."""
import numpy as np
import pytest
import torch

import paper_2004_09211_gb300 as spl
from paper_2004_09211_gb300 import synth

from parity import check_close

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _inputs(H, W, T, N, seed, L=24):
    h, peak = synth.asymmetric_irf(L=L)
    sc = synth.moving_scene(H, W, N, peak + 6, T - L + peak - 6, seed, n_objects=2)
    g = torch.Generator().manual_seed(seed)
    zs = []
    for n in range(N):
        mean = synth.expected_counts(torch.from_numpy(sc.depth[n]), torch.from_numpy(sc.signal[n]) * 3.0, 0.02,
                                     torch.from_numpy(h), peak, T)
        zs.append(torch.poisson(mean, generator=g).numpy())
    return h, peak, zs, [d.astype(np.float64) for d in sc.depth]


def _gpu_z(zs, T):
    pitch = synth.pad_pitch(T)
    z = torch.stack([torch.from_numpy(np.ascontiguousarray(x).reshape(-1, T).astype(np.int32)) for x in zs])
    return synth.pitched(z.to(torch.uint16), pitch).contiguous().to(DEV)


def _check_grad(g, o, name):
    g = np.asarray(g, np.float64).reshape(-1)
    o = np.asarray(o, np.float64).reshape(-1)
    tol = 2e-3 * np.abs(o).max() + 1e-3 * np.abs(o)
    bad = np.nonzero(np.abs(g - o) > tol)[0]
    assert bad.size == 0, f"{name}: {bad[:6]} gpu {g[bad[:6]]} oracle {o[bad[:6]]} (max |oracle| {np.abs(o).max():.3g})"


@pytest.mark.parametrize("beta,tau", [(0.45, 0.5), (0.8, 1.0)])
def test_diff_matches_fp64_autograd(beta, tau):
    from oracle import diff_oracle as dor
    H, W, T, N = 6, 7, 160, 4
    h, peak, zs, refs = _inputs(H, W, T, N, seed=71)
    nu = np.array([0.05, 0.1, 0.0, 0.15, 0.4, 0.2, 0.0, 0.1, 0.0])
    ref = dor.gradients(h, beta, nu, zs, refs, peak, sigma_rw2=3.0, tau=tau)
    prm = spl.make_params(H, W, T, len(h), peak, beta=beta, sigma_rw2=3.0, nu=nu)
    z = _gpu_z(zs, T)
    d_ref = torch.from_numpy(np.stack(refs).reshape(N, -1).astype(np.float32)).to(DEV)
    hd = torch.from_numpy(h).to(DEV)
    fw = spl.spl_diff_forward(prm, z, hd, tau, d_ref=d_ref)
    bw = spl.spl_diff_backward(prm, z, hd, tau, d_ref, fw["mu_states"], fw["var_states"], scratch=fw["scratch"])
    torch.cuda.synchronize()
    for n in range(N):
        m, v, ds = ref["frames"][n]
        check_close(fw["mu_states"][n + 1].cpu().numpy(), m, f"mu frame {n}")
        check_close(fw["var_states"][n + 1].cpu().numpy(), v, f"var frame {n}", atol=1e-6)
        check_close(fw["dsoft"][n].cpu().numpy(), ds, f"dsoft frame {n}")
    check_close(fw["loss"].cpu().numpy(), [ref["loss"]], "loss")
    _check_grad(bw["grad_h"].cpu().numpy(), ref["grad_h"], "grad_h")
    _check_grad(bw["grad_beta"].cpu().numpy(), [ref["grad_beta"]], "grad_beta")
    _check_grad(bw["grad_nu"].cpu().numpy(), ref["grad_nu"], "grad_nu")


def test_diff_backward_is_bitwise_reproducible_and_autograd_wired():
    H, W, T, N = 9, 8, 200, 3
    h, peak, zs, refs = _inputs(H, W, T, N, seed=72)
    z = _gpu_z(zs, T)
    d_ref = torch.from_numpy(np.stack(refs).reshape(N, -1).astype(np.float32)).to(DEV)
    geom = dict(H=H, W=W, T=T, peak=peak, sigma_rw2=3.0)
    grads = []
    for _ in range(2):
        ht = torch.from_numpy(h).to(DEV).requires_grad_(True)
        bt = torch.tensor(0.5, device=DEV, requires_grad=True)
        nt = torch.tensor(spl.cross_weights(0.5), device=DEV, requires_grad=True)
        loss = spl.FilterLoss.apply(ht, bt, nt, z, d_ref, geom, 0.5)
        loss.sum().backward()
        grads.append((ht.grad.clone(), bt.grad.clone(), nt.grad.clone(), loss.detach().clone()))
    for name, a, b in zip(("grad_h", "grad_beta", "grad_nu", "loss"), grads[0], grads[1]):
        assert torch.equal(a, b), f"{name}: max |diff| {(a - b).abs().max().item():.3g}, run 1 {a[:4].tolist()}"
    assert torch.isfinite(grads[0][0]).all() and torch.isfinite(grads[0][2]).all()
