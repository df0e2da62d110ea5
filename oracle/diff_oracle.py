"""FP64 differentiable oracle of the online filter with a soft-argmax readout (plain PyTorch CPU autograd).

TEST INFRASTRUCTURE: imported only by tests/ and bench.py's CPU-baseline leg; never by the CUDA library.

It restates, with torch float64 tensor operations on the CPU, the same definitions the C oracle (spl_oracle.c)
implements with loops, so that it can be differentiated by autograd:
  g_j = h_j^beta (0 where h_j <= 0); C(d) = sum_j g_j z[d - peak + j]                       (Eq. beta_div2)
  prior(d) = sum_k nu_k N(d; m_k, s2_k) over the 3x3 stencil (informative neighbour: its previous mean and
  variance + sigma_RW^2; otherwise the weakly informative Gaussian)                          (Eq. predict)
  ell(d) = lambda C(d) + log prior(d), lambda = (beta + 1) / beta                            (Eq. approx_post)
  mu = sum w d, var = sum w (d - mu)^2 with w = softmax(ell)                                  (Eq. KL_div)
  readout d_soft = sum softmax(ell / tau) d; tau = 1 gives mu (the paper's estimator).
Loss = mean over frames and pixels of (d_soft - d_ref)^2. All pixels present, none faulty.
Pinned by tests/test_oracle_pins.py: its mu and var equal the C oracle's filter step, its tau = 1 readout equals mu,
and its autograd gradient equals central finite differences of its own loss.
"""
from __future__ import annotations

import math

import torch


def _stencil_components(mu_prev, var_prev, nu, sigma_rw2, dmin, dmax):
    """Per-pixel stencil entries (m_k, s2_k) for k = 0..8, [H, W, 9] each; out-of-frame -> flat Gaussian."""
    H, W = mu_prev.shape
    flat_m = 0.5 * (dmin + dmax)
    flat_v = (dmax - dmin) ** 2 / 12.0
    mp = torch.nn.functional.pad(mu_prev, (1, 1, 1, 1), value=flat_m)
    vp = torch.nn.functional.pad(var_prev, (1, 1, 1, 1), value=flat_v)
    ms, vs = [], []
    for k in range(9):
        dy, dx = k // 3 - 1, k % 3 - 1
        ms.append(mp[1 + dy:1 + dy + H, 1 + dx:1 + dx + W])
        vs.append(vp[1 + dy:1 + dy + H, 1 + dx:1 + dx + W] + sigma_rw2)
    return torch.stack(ms, -1), torch.stack(vs, -1)


def frame(h, beta, nu, z, mu_prev, var_prev, peak, dmin, dmax, sigma_rw2, tau):
    """One frame: returns (mu, var, d_soft), each [H, W]."""
    L = h.numel()
    H, W, T = z.shape
    d = torch.arange(dmin, dmax + 1, dtype=torch.float64)
    g = torch.where(h > 0, torch.clamp(h, min=1e-300) ** beta, torch.zeros_like(h))
    windows = z.unfold(-1, L, 1)[..., dmin - peak:dmax - peak + 1, :]      # [H, W, D, L]: z[d - peak + j]
    C = windows @ g                                                        # [H, W, D]
    lam = (beta + 1.0) / beta
    m, s2 = _stencil_components(mu_prev, var_prev, nu, sigma_rw2, dmin, dmax)  # [H, W, 9]
    e = d.view(1, 1, -1, 1) - m.unsqueeze(2)                                # [H, W, D, 9]
    logN = -0.5 * torch.log(2 * math.pi * s2).unsqueeze(2) - e * e / (2 * s2.unsqueeze(2))
    mx = logN.max(-1, keepdim=True).values.detach()
    lp = mx.squeeze(-1) + torch.log((nu.view(1, 1, 1, 9) * torch.exp(logN - mx)).sum(-1))
    ell = lam * C + lp
    w = torch.softmax(ell, -1)
    mu = (w * d).sum(-1)
    var = (w * (d - mu.unsqueeze(-1)) ** 2).sum(-1)
    wt = torch.softmax(ell / tau, -1)
    dsoft = (wt * d).sum(-1)
    return mu, var, dsoft


def sequence_loss(h, beta, nu, zs, d_refs, peak, dmin, dmax, sigma_rw2, tau):
    """Loss over frames from the flat initial state; returns (loss, [(mu, var, d_soft) per frame])."""
    H, W, _ = zs[0].shape
    mu = torch.full((H, W), 0.5 * (dmin + dmax), dtype=torch.float64)
    var = torch.full((H, W), (dmax - dmin) ** 2 / 12.0, dtype=torch.float64)
    total = 0.0
    outs = []
    for z, dr in zip(zs, d_refs):
        mu, var, ds = frame(h, beta, nu, z, mu, var, peak, dmin, dmax, sigma_rw2, tau)
        total = total + ((ds - dr) ** 2).sum()
        outs.append((mu, var, ds))
    return total / (len(zs) * H * W), outs


def gradients(h, beta, nu, zs, d_refs, peak, dmin=None, dmax=None, sigma_rw2=3.0, tau=0.5):
    """Loss and its gradient with respect to (h, beta, nu) by autograd, all float64."""
    T = zs[0].shape[-1]
    L = len(h)
    dmin = peak if dmin is None else dmin
    dmax = T - L + peak if dmax is None else dmax
    ht = torch.tensor(h, dtype=torch.float64, requires_grad=True)
    bt = torch.tensor(float(beta), dtype=torch.float64, requires_grad=True)
    nt = torch.tensor(nu, dtype=torch.float64, requires_grad=True)
    zt = [torch.as_tensor(z, dtype=torch.float64) for z in zs]
    dt = [torch.as_tensor(x, dtype=torch.float64) for x in d_refs]
    loss, outs = sequence_loss(ht, bt, nt, zt, dt, peak, dmin, dmax, sigma_rw2, tau)
    loss.backward()
    return dict(loss=float(loss), grad_h=ht.grad.numpy(), grad_beta=bt.grad.item(), grad_nu=nt.grad.numpy(),
                frames=[tuple(x.detach().numpy() for x in o) for o in outs])


def loss_value(h, beta, nu, zs, d_refs, peak, dmin=None, dmax=None, sigma_rw2=3.0, tau=0.5):
    T = zs[0].shape[-1]
    L = len(h)
    dmin = peak if dmin is None else dmin
    dmax = T - L + peak if dmax is None else dmax
    with torch.no_grad():
        loss, _ = sequence_loss(torch.as_tensor(h, dtype=torch.float64), torch.tensor(float(beta), dtype=torch.float64),
                                torch.as_tensor(nu, dtype=torch.float64),
                                [torch.as_tensor(z, dtype=torch.float64) for z in zs],
                                [torch.as_tensor(x, dtype=torch.float64) for x in d_refs], peak, dmin, dmax, sigma_rw2,
                                tau)
    return float(loss)
