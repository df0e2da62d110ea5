"""The allocation-free batched step (spl_batch_step_noalloc), called through the C ABI.

It serves callers that cannot allocate device memory through CUDA (their memory comes from someone else's pool,
or their loop must never enter cudaMalloc): they pass descriptors, inputs and outputs in memory they own, and the
library's working memory is a fixed array compiled into it. This test checks that two calls in a row give the same
results as the plan-based spl_batch_step (the existing entry point) on the same data, within the parity tolerance
of the other GPU tests, and that an over-capacity request is refused on the host. The file is named so pytest
collects it last; it also passes on its own in a fresh process (its first call does the one-time set-up).
"""
import ctypes as ct

import numpy as np
import pytest
import torch

import paper_2004_09211_gb300 as spl
from paper_2004_09211_gb300 import _abi, synth

from parity import check_close

pytestmark = pytest.mark.gpu
DEV = "cuda"
N_FRAMES = 2


def _sequences():
    g3 = synth.gaussian_irf(3.0, 12)
    asy = synth.asymmetric_irf(L=48)
    specs = [(9, 14, 512, g3, 0.5, 3.0), (16, 8, 400, asy, 0.3, 2.0), (4, 33, 700, asy, 1.0, 4.0)]
    seqs = []
    for s, (H, W, T, (h, peak), beta, s2) in enumerate(specs):
        L = len(h)
        sc = synth.moving_scene(H, W, N_FRAMES, peak + 4, T - L + peak - 4, 60 + s, n_objects=2)
        frames = [synth.toa_lists(sc.depth[n], np.full((H, W), 3.0), 12.0 / T, h, peak, T, 600 + 10 * s + n)
                  for n in range(N_FRAMES)]
        prm = spl.make_params(H, W, T, L, peak, beta=beta, sigma_rw2=s2)
        seqs.append(dict(prm=prm, h=torch.from_numpy(h).to(DEV), P=H * W,
                         frames=[(torch.from_numpy(o).to(DEV), torch.from_numpy(b).to(DEV)) for o, b in frames]))
    return seqs


def _buffers(q):
    P = q["P"]
    st = dict(mu=[torch.empty(P, device=DEV) for _ in range(N_FRAMES + 1)],
              var=[torch.empty(P, device=DEV) for _ in range(N_FRAMES + 1)])
    outs = [dict(argmax=torch.empty(P, dtype=torch.int32, device=DEV), refl=torch.empty(P, device=DEV),
                 bg=torch.empty(P, device=DEV)) for _ in range(N_FRAMES)]
    spl.spl_state_init(q["prm"], st["mu"][0], st["var"][0])
    return st, outs


def _frame(q, st, outs, n):
    off, bins = q["frames"][n]
    return dict(h=q["h"], offsets=off, bins=bins, mu_in=st["mu"][n], var_in=st["var"][n], mu_out=st["mu"][n + 1],
                var_out=st["var"][n + 1], **outs[n])


def _desc_arrays(seqs, frames):
    """Host array of spl_seq_desc and the same bytes in device memory owned by the caller (a torch tensor)."""
    host = (_abi.spl_seq_desc * len(seqs))()
    for i, (q, fr) in enumerate(zip(seqs, frames)):
        host[i].prm = q["prm"]
        for k, dt in spl._FRAME_KEYS.items():
            setattr(host[i].f, k, spl._dev(fr.get(k), k, dt))
    raw = bytes(ct.string_at(ct.addressof(host), ct.sizeof(host)))
    dev = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(DEV)
    return host, dev


def test_noalloc_step_matches_plan_step_on_two_calls():
    lib = _abi.load()
    seqs = _sequences()
    # existing entry point: a plan with one slot per frame
    ref = [_buffers(q) for q in seqs]
    plan = spl.spl_batch_create([q["prm"] for q in seqs], nslots=N_FRAMES)
    try:
        for n in range(N_FRAMES):
            spl.spl_batch_set(plan, n, [_frame(q, *ref[i], n) for i, q in enumerate(seqs)])
        for n in range(N_FRAMES):
            spl.spl_batch_step(plan, n)
        torch.cuda.synchronize()
        assert spl.spl_batch_status(plan) == 0
    finally:
        spl.spl_batch_destroy(plan)

    # allocation-free entry point, two calls in a row (frame 1 starts from frame 0's output)
    mine = [_buffers(q) for q in seqs]
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    descs = [_desc_arrays(seqs, [_frame(q, *mine[i], n) for i, q in enumerate(seqs)]) for n in range(N_FRAMES)]
    torch.cuda.synchronize()
    for n in range(N_FRAMES):
        host, dev = descs[n]
        if n == 1:  # the set-up of the first call is done: from here on the call may not take device memory
            free_before = torch.cuda.mem_get_info()[0]
        st = lib.spl_batch_step_noalloc(host, dev.data_ptr(), len(seqs), 32, status.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
        assert st == _abi.SPL_OK, lib.spl_last_error()
        torch.cuda.synchronize()
        if n == 1:
            assert torch.cuda.mem_get_info()[0] >= free_before, "the second call took device memory"
        for i in range(len(seqs)):
            a_st, a_out = ref[i]
            b_st, b_out = mine[i]
            check_close(b_st["mu"][n + 1].cpu().numpy(), a_st["mu"][n + 1].cpu().numpy(), f"call {n} seq {i} mu")
            check_close(b_st["var"][n + 1].cpu().numpy(), a_st["var"][n + 1].cpu().numpy(), f"call {n} seq {i} var",
                        atol=1e-6)
            check_close(b_out[n]["refl"].cpu().numpy(), a_out[n]["refl"].cpu().numpy(), f"call {n} seq {i} refl",
                        atol=1e-6)
            check_close(b_out[n]["bg"].cpu().numpy(), a_out[n]["bg"].cpu().numpy(), f"call {n} seq {i} bg",
                        atol=1e-9)
            np.testing.assert_array_equal(b_out[n]["argmax"].cpu().numpy(), a_out[n]["argmax"].cpu().numpy())
    assert int(status.item()) == 0


def test_noalloc_rejects_more_sequences_than_its_fixed_scratch():
    lib = _abi.load()
    n = _abi.SPL_NOALLOC_MAX_SEQ + 1
    host = (_abi.spl_seq_desc * n)()
    st = lib.spl_batch_step_noalloc(host, 0x1000, n, 32, None, None)
    assert st == _abi.SPL_EINVAL
    assert "capacity" in lib.spl_last_error().decode()


def test_noalloc_refuses_a_device_descriptor_wider_than_its_host_copy():
    """The host copy of the descriptors sizes the kernel's shared-memory slices and the kernel reads the device copy:
    a device descriptor with more candidates than any host descriptor is refused on the device (its outputs set to
    NaN, SPL_BATCH_DESC_MISMATCH raised) instead of overrunning the slice; the other sequences are unaffected."""
    lib = _abi.load()
    seqs = _sequences()
    mine = [_buffers(q) for q in seqs]
    frames = [_frame(q, *mine[i], 0) for i, q in enumerate(seqs)]
    host, dev = _desc_arrays(seqs, frames)
    Ds = [q["prm"].dmax - q["prm"].dmin + 1 for q in seqs]
    w = int(np.argmax(Ds))  # the widest sequence: its host copy is made to claim 41 candidates
    host[w].prm.dmax = host[w].prm.dmin + 40
    assert Ds[w] > max([41] + [d for i, d in enumerate(Ds) if i != w])
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    st = lib.spl_batch_step_noalloc(host, dev.data_ptr(), len(seqs), 32, status.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert st == _abi.SPL_OK, lib.spl_last_error()
    torch.cuda.synchronize()
    assert int(status.item()) & _abi.SPL_BATCH_DESC_MISMATCH
    assert torch.isnan(mine[w][0]["mu"][1]).all()
    for i in range(len(seqs)):
        if i != w:
            assert torch.isfinite(mine[i][0]["mu"][1]).all()
