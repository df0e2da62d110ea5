"""GPU checks of the differentiable filter at the full size of its workload (128 x 128 pixels x 20 frames,
T = 1024, 48-tap IRF, tau = 0.5, the benchmark's scene and photon generator). The states and readouts of the first
frames are compared at sampled pixels with the FP64 autograd oracle on dependency-cone crops (the crops reproduce
the oracle's full image: checked on the host). The gradients are sums over every pixel and frame, so at this size
they are checked for the properties that hold at any size: finite, and bitwise the same on a second backward pass."""
import numpy as np
import pytest
import torch

import paper_2004_09211_gb300 as spl
from paper_2004_09211_gb300 import synth

from parity import check_close

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _diff_job_inputs(device, H=128, W=128, N=20, T=1024, L=48, seed=5):
    """The differentiable job's inputs: IRF, peak, pitched uint16 histograms [N, P, pitch] on `device`, reference
    depths [N, P]."""
    h, peak = synth.asymmetric_irf(L=L)
    sc = synth.moving_scene(H, W, N, peak + 8, T - L + peak - 8, seed)
    gen = torch.Generator(device=device).manual_seed(seed)
    hd = torch.from_numpy(h).to(device)
    pitch = synth.pad_pitch(T)
    zs = []
    for n in range(N):
        mean = synth.expected_counts(torch.from_numpy(sc.depth[n]).to(device), torch.from_numpy(sc.signal[n]).to(device),
                                     float(sc.signal[n].mean()) / (0.1 * T), hd, peak, T)
        zs.append(synth.pitched(synth.poisson_histograms(mean, gen).reshape(-1, T), pitch))
    z = torch.stack(zs).contiguous()
    d_ref = torch.from_numpy(sc.depth.reshape(N, -1).astype(np.float32)).to(device)
    return h, peak, z, d_ref


def _crop_frames(h, peak, z_host, H, W, T, y, x, K, beta, nu, sigma_rw2, tau):
    """The autograd oracle's frames 0..K-1 at pixel (y, x) from a (2K+1)^2 crop (clipped at the edges) that starts
    from the flat state: a list of (mu, var, d_soft) per frame."""
    from oracle import diff_oracle as dor
    t = lambda a: torch.as_tensor(a, dtype=torch.float64)
    L = len(h)
    dmin, dmax = peak, T - L + peak
    y0, y1 = max(0, y - K), min(H, y + K + 1)
    x0, x1 = max(0, x - K), min(W, x + K + 1)
    m = torch.full((y1 - y0, x1 - x0), 0.5 * (dmin + dmax), dtype=torch.float64)
    v = torch.full((y1 - y0, x1 - x0), (dmax - dmin) ** 2 / 12.0, dtype=torch.float64)
    out = []
    for n in range(K):
        zc = z_host[n].reshape(H, W, -1)[y0:y1, x0:x1, :T].astype(np.float64)
        m, v, ds = dor.frame(t(h), t(beta), t(nu), t(zc), m, v, peak, dmin, dmax, sigma_rw2, tau)
        out.append((float(m[y - y0, x - x0]), float(v[y - y0, x - x0]), float(ds[y - y0, x - x0])))
    return out


def test_full_size_differentiable_job():
    H = W = 128
    N, T, L, K = 20, 1024, 48, 3
    beta, tau, sigma_rw2 = 0.5, 0.5, 3.0
    h, peak, z, d_ref = _diff_job_inputs(DEV, H, W, N, T, L)
    prm = spl.make_params(H, W, T, L, peak, beta=beta, sigma_rw2=sigma_rw2)
    hd = torch.from_numpy(h).to(DEV)
    fw = spl.spl_diff_forward(prm, z, hd, tau, d_ref=d_ref)
    grads = []
    for _ in range(2):
        bw = spl.spl_diff_backward(prm, z, hd, tau, d_ref, fw["mu_states"], fw["var_states"], scratch=fw["scratch"])
        grads.append({k: bw[k].clone() for k in ("grad_h", "grad_beta", "grad_nu")})
    torch.cuda.synchronize()
    assert torch.isfinite(fw["loss"]).all()
    for k in grads[0]:
        assert torch.isfinite(grads[0][k]).all(), k
        assert torch.equal(grads[0][k], grads[1][k]), k
    z_host = [z[n].cpu().numpy() for n in range(K)]
    mu_s, var_s, ds_s = fw["mu_states"].cpu().numpy(), fw["var_states"].cpu().numpy(), fw["dsoft"].cpu().numpy()
    nu = synth.cross_weights(0.5)
    for (y, x) in [(0, 0), (127, 127), (0, 90), (64, 64), (17, 101)]:
        p = y * W + x
        for n, (m, v, ds) in enumerate(_crop_frames(h, peak, z_host, H, W, T, y, x, K, beta, nu, sigma_rw2, tau)):
            what = f"pixel ({y},{x}) frame {n}"
            check_close(mu_s[n + 1, p:p + 1], [m], f"{what} mu")
            check_close(var_s[n + 1, p:p + 1], [v], f"{what} var", atol=1e-6)
            check_close(ds_s[n, p:p + 1], [ds], f"{what} d_soft")
