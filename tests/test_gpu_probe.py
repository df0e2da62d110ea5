"""GPU sanity of the arithmetic-throughput probes (spl_probe_throughput) that the ALU and issue rooflines are quoted
against: every kind runs, writes finite chain results, records positive cycle counts, and the FFMA probe reaches a
plausible fraction of the architectural rate (one warp-instruction per scheduler per clock)."""
import ctypes as ct

import numpy as np
import pytest
import torch

from paper_2004_09211_gb300 import _abi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_probe_runs_and_measures(kind):
    lib = _abi.load()
    nb, opt = ct.c_int(0), ct.c_longlong(0)
    iters = 256
    assert lib.spl_probe_throughput(kind, 4, iters, None, None, ct.byref(nb), ct.byref(opt), None) == _abi.SPL_OK
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert nb.value == 4 * nsm and opt.value == iters * 128
    sink = torch.empty(nb.value * 256, device="cuda")
    cyc = torch.zeros(nb.value, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for rep in range(2):
        e0.record(s)
        st = lib.spl_probe_throughput(kind, 4, iters, ct.c_void_p(sink.data_ptr()), ct.c_void_p(cyc.data_ptr()),
                                      ct.byref(nb), ct.byref(opt), ct.c_void_p(s.cuda_stream))
        e1.record(s)
        assert st == _abi.SPL_OK, lib.spl_last_error()
    torch.cuda.synchronize()
    assert torch.isfinite(sink).all()
    assert (cyc > 0).all()
    if kind == 0:  # FFMA: operations per second against 128 per clock per SM at 2.2 GHz (an upper bound)
        rate = nb.value * 256 * opt.value / (e0.elapsed_time(e1) / 1e3)
        assert 0.2 < rate / (128 * nsm * 2.2e9) < 1.0
