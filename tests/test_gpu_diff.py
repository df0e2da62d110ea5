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


def _check_grad(g, o, name, floor=2e-5):
    """Per component: relative 1e-4, with an absolute floor of `floor` times the largest component of the same
    gradient for components that nearly cancel (see the module docstring)."""
    g = np.asarray(g, np.float64).reshape(-1)
    o = np.asarray(o, np.float64).reshape(-1)
    scale = np.abs(o).max()
    tol = floor * scale + 1e-4 * np.abs(o)
    err = np.abs(g - o)
    bad = np.nonzero(err > tol)[0]
    worst = float((err / np.maximum(np.abs(o), 1e-300)).max())
    assert bad.size == 0, (f"{name}: {bad[:6]} gpu {g[bad[:6]]} oracle {o[bad[:6]]} (max |oracle| {scale:.3g}, "
                           f"largest error / max |oracle| {float(err.max() / scale):.3g}, worst relative {worst:.3g})")


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


def test_diff_forward_off_centre_posteriors():
    """From a broad prior state (every pixel N(x0, 50^2)), 3-6 photons in one bin 3.0-3.6 prior standard deviations
    away: the maximiser sits on the photons while most of the mass stays under the prior, so for about a third of
    the pixels (checked on the oracle) the posterior mean lies more than two standard deviations from the
    maximiser, about which the forward pass centres its moment sums (the variance's relative rounding error grows
    like 1e-7 (1 + m1^2 / var): about 1e-6 here). States and readouts of two frames against the FP64 oracle's
    frames from the same initial state."""
    from oracle import diff_oracle as dor
    H, W, T, beta, tau, sigma_rw2 = 5, 6, 500, 0.5, 0.5, 3.0
    h, peak = synth.asymmetric_irf(L=24)
    nu = synth.cross_weights(0.5)
    rng = np.random.default_rng(91)
    dmin, dmax = peak, T - len(h) + peak
    x0 = 0.5 * (dmin + dmax)
    mu0 = np.full((H, W), x0, np.float32)
    var0 = np.full((H, W), 2500.0, np.float32)
    z = np.zeros((H, W, T))
    for y in range(H):
        for x in range(W):
            d = int(round(x0 + rng.choice([-1, 1]) * rng.uniform(3.0, 3.6) * 50))
            z[y, x, d] += int(rng.integers(3, 7))  # the IRF maximum of a surface at depth d falls in bin d
    t = lambda a: torch.as_tensor(a, dtype=torch.float64)
    ref, m, v = [], t(mu0), t(var0)
    for _ in range(2):
        m, v, ds = dor.frame(t(h), t(beta), t(nu), t(z), m, v, peak, dmin, dmax, sigma_rw2, tau)
        ref.append((m.numpy(), v.numpy(), ds.numpy()))
    # the regime: posterior mean more than two standard deviations from the maximiser of ell
    g = t(h).clamp(min=1e-300) ** beta
    C = t(z).unfold(-1, len(h), 1)[..., dmin - peak:dmax - peak + 1, :] @ g
    cm, cv = dor._stencil_components(t(mu0), t(var0), t(nu), sigma_rw2, dmin, dmax)
    e = torch.arange(dmin, dmax + 1, dtype=torch.float64).view(1, 1, -1, 1) - cm.unsqueeze(2)
    lp = torch.logsumexp(torch.log(t(nu)).view(1, 1, 1, 9) - 0.5 * torch.log(2 * np.pi * cv).unsqueeze(2)
                         - e * e / (2 * cv.unsqueeze(2)), -1)
    am = ((beta + 1) / beta * C + lp).argmax(-1).numpy() + dmin
    m1 = ref[0][0] - am
    assert (m1 * m1 > 4 * ref[0][1] + 1).sum() >= 8
    prm = spl.make_params(H, W, T, len(h), peak, beta=beta, sigma_rw2=sigma_rw2, nu=nu)
    ms = torch.empty(3, H * W, device=DEV)
    vs = torch.empty(3, H * W, device=DEV)
    ms[0] = torch.from_numpy(mu0.reshape(-1)).to(DEV)
    vs[0] = torch.from_numpy(var0.reshape(-1)).to(DEV)
    fw = spl.spl_diff_forward(prm, _gpu_z([z, z], T), torch.from_numpy(h).to(DEV), tau, mu_states=ms, var_states=vs)
    torch.cuda.synchronize()
    for n in range(2):
        check_close(ms[n + 1].cpu().numpy(), ref[n][0], f"mu frame {n}")
        check_close(vs[n + 1].cpu().numpy(), ref[n][1], f"var frame {n}", atol=1e-6)
        check_close(fw["dsoft"][n].cpu().numpy(), ref[n][2], f"dsoft frame {n}")


def test_diff_gradients_at_the_differentiable_workload_shape():
    """The gradient test at the differentiable workload's own shape: 48-tap IRF, T = 1024, 20 frames, tau = 0.5,
    beta = 0.5, the workload's scene and photon generator (SBR 0.1), on a 12 x 12 crop of its 128 x 128 frames that
    a moving object crosses (the crop is the input of both sides). Forward states and readouts of every frame, the
    loss, and every component of the three gradients against the FP64 autograd oracle. The weights are the cross
    with 0.02 on the diagonals: where every weighted component of a pixel's prior underflows next to an unweighted
    one, the oracle's plain log-sum-exp returns log 0 and autograd a NaN gradient, so zero weights are left to
    the small-shape test above."""
    from oracle import diff_oracle as dor
    Hf = Wf = 128
    N, T, L, c = 20, 1024, 48, 12
    h, peak = synth.asymmetric_irf(L=L)
    sc = synth.moving_scene(Hf, Wf, N, peak + 8, T - L + peak - 8, 5)
    g = torch.Generator().manual_seed(5)
    y0, x0 = 96, 64  # every pixel of this crop changes depth every frame
    zs, refs = [], []
    for n in range(N):
        mean = synth.expected_counts(torch.from_numpy(sc.depth[n]), torch.from_numpy(sc.signal[n]),
                                     float(sc.signal[n].mean()) / (0.1 * T), torch.from_numpy(h), peak, T)
        z = torch.poisson(mean, generator=g).numpy()
        zs.append(np.ascontiguousarray(z[y0:y0 + c, x0:x0 + c]))
        refs.append(sc.depth[n][y0:y0 + c, x0:x0 + c].astype(np.float64))
    beta, tau = 0.5, 0.5
    nu = synth.cross_weights(0.5).astype(np.float64)
    nu[[0, 2, 6, 8]] = 0.02
    ref = dor.gradients(h, beta, nu, zs, refs, peak, sigma_rw2=3.0, tau=tau)
    assert np.isfinite(ref["grad_h"]).all() and np.isfinite(ref["grad_nu"]).all()
    prm = spl.make_params(c, c, T, L, peak, beta=beta, sigma_rw2=3.0, nu=nu)
    zd = _gpu_z(zs, T)
    d_ref = torch.from_numpy(np.stack(refs).reshape(N, -1).astype(np.float32)).to(DEV)
    hd = torch.from_numpy(h).to(DEV)
    fw = spl.spl_diff_forward(prm, zd, hd, tau, d_ref=d_ref)
    bw = spl.spl_diff_backward(prm, zd, hd, tau, d_ref, fw["mu_states"], fw["var_states"], scratch=fw["scratch"])
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
