"""GPU parity of the tensor-core (tcgen05) data term, spl_depth_cost_tc, on FP16 histograms.

Tolerance: each powered tap g = h^beta is carried as two FP16 parts of g * 2^15 (about 22 significant bits, relative
error <= 2^-22 per tap) and the products of exact integer counts with them are exact in FP32; the FP32 accumulation
of at most 2 * 208 products adds a few units in the last place. C is therefore compared with relative 1e-5 plus an
absolute 1e-6 * max C (the parity tolerance of the FP32 path is 1e-4 relative)."""
import numpy as np
import pytest
import torch

import paper_2004_09211_gb300 as spl
from paper_2004_09211_gb300 import synth

from parity import check_argmax, check_close

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _f16_hist(z, T):
    zt = torch.from_numpy(np.ascontiguousarray(z).reshape(-1, T).astype(np.float32)).to(torch.float16)
    return synth.pitched(zt, synth.pad_pitch(T)).to(DEV)


@pytest.mark.parametrize("P,T,L,beta,dlo,dhi", [
    (130, 700, 64, 0.5, None, None),       # ragged pixel tile, 64 taps (the mixed-precision workload's IRF length)
    (256, 1000, 48, 0.2, 60, 900),          # sub-range of depths: dmin - peak not a multiple of 8
    (77, 333, 1, 1.0, None, None),          # one tap, odd T (padded pitch)
    (129, 900, 128, 0.7, None, None),       # largest IRF
    (300, 4096, 64, 0.5, None, None),       # the mixed-precision workload's T
])
def test_tc_cost_matches_oracle(orc, P, T, L, beta, dlo, dhi):
    rng = np.random.default_rng(P + T + L)
    if L >= 48:
        h, peak = synth.stretched_irf(synth.asymmetric_irf(L=48)[0], L)
    else:
        h = np.ones(L, np.float32) / L
        peak = 0
    q = orc.params(T, L, peak, dlo, dhi, beta=beta)
    z = rng.poisson(0.05, size=(P, T)).astype(np.float64)
    for p in range(P):
        d = int(rng.integers(q.dmin, q.dmax + 1))
        z[p, d - peak:d - peak + L] += rng.poisson(40 * h)
    z = np.minimum(z, 2048)
    prm = spl.make_params(1, P, T, L, peak, dlo, dhi, beta=beta)
    hd = torch.from_numpy(np.asarray(h, np.float32)).to(DEV)
    zt = _f16_hist(z, T)
    cost, am = spl.spl_depth_cost_tc(prm, zt, hd)
    torch.cuda.synchronize()
    assert spl.spl_tc_status() == 0
    C = orc.cost(q, h, z)
    check_close(cost.cpu().numpy(), C, "C (tensor cores)", rtol=1e-5, atol=1e-6 * C.max())
    check_argmax(am.cpu().numpy(), C.argmax(1) + q.dmin, C, q.dmin, "argmax C (tensor cores)")
    # the FP32 CUDA-core path on the same FP16 input agrees as well
    c32, a32 = spl.spl_depth_cost(prm, zt, hd)
    torch.cuda.synchronize()
    check_close(cost.cpu().numpy(), c32.cpu().numpy(), "C tensor vs FP32 cores", rtol=1e-5, atol=1e-6 * C.max())
