"""Host-side checks of the C ABI (no GPU): the library builds and loads, exports every entry point that
include/spl.h declares, and rejects invalid arguments on the host before anything is launched."""
import ctypes as ct
import os
import re

import pytest

from paper_2004_09211_gb300 import _abi, make_params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"SPL_API\s+[\w\s\*]+?\b(spl_\w+)\s*\(", src)
    return names


def test_every_declared_symbol_is_exported():
    lib = _abi.load()
    names = declared_entry_points()
    assert len(names) >= 7
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported by libspl.so"
        assert n in _abi.SIGNATURES, f"{n} has no ctypes signature in the binding"


def test_version_and_empty_error():
    lib = _abi.load()
    assert b"sm_103a" in lib.spl_version()


def _call_cost(prm, data=0x1000, pitch=None, fmt=_abi.SPL_HIST_U16, h=0x2000, cost=0x3000, argmax=0x4000):
    lib = _abi.load()
    hz = _abi.spl_hist()
    hz.fmt = fmt
    hz.data = data
    hz.pitch = prm.T if pitch is None else pitch
    st = lib.spl_depth_cost(ct.byref(prm), ct.byref(hz), h, cost, argmax, None)
    return st, lib.spl_last_error().decode()


@pytest.mark.parametrize("mut, needle", [
    (dict(dmin=5), "full-support"),                 # below peak
    (dict(dmax=10_000), "full-support"),
    (dict(beta=0.0), "beta"),
    (dict(beta=float("nan")), "beta"),
    (dict(L=0), "L must"),
    (dict(T=10, L=20), "T (10) must be >= L"),
    (dict(peak=30), "peak"),
    (dict(H=0), "H and W"),
])
def test_invalid_parameters_rejected_on_host(mut, needle):
    kw = dict(H=4, W=4, T=64, L=25, peak=12, dmin=12, dmax=51, beta=0.5)
    kw.update(mut)
    prm = make_params(kw["H"], kw["W"], kw["T"], kw["L"], kw["peak"], kw["dmin"], kw["dmax"], beta=kw["beta"])
    st, msg = _call_cost(prm)
    assert st == _abi.SPL_EINVAL, (st, msg)
    assert needle in msg


def test_histogram_layout_rejected_on_host():
    prm = make_params(4, 4, 60, 25, 12)
    assert _call_cost(prm, pitch=59)[0] == _abi.SPL_EINVAL                  # pitch < T
    st, msg = _call_cost(prm, pitch=60)                                       # 120 B rows: not 16-B multiple
    assert st == _abi.SPL_EINVAL and "16 bytes" in msg
    assert _call_cost(prm, pitch=64, data=0x1008)[0] == _abi.SPL_EINVAL      # misaligned base
    assert _call_cost(prm, pitch=64, fmt=7)[0] == _abi.SPL_EINVAL
    assert _call_cost(prm, pitch=64, data=0)[0] == _abi.SPL_EINVAL
    assert _call_cost(prm, pitch=64, cost=0, argmax=0)[0] == _abi.SPL_EINVAL


def test_unsupported_sizes_reported():
    prm = make_params(4, 4, 600, 200, 100)
    st, msg = _call_cost(prm, pitch=600)
    assert st == _abi.SPL_EUNSUPPORTED and "not supported" in msg


@pytest.mark.parametrize("entry", ["spl_filter_step", "spl_filter_step_fp32"])
def test_filter_argument_checks(entry):
    lib = _abi.load()
    fn = getattr(lib, entry)
    prm = make_params(4, 4, 64, 25, 12, sigma_rw2=0.0)
    hz = _abi.spl_hist(_abi.SPL_HIST_U16, 0x1000, 64)
    st = fn(ct.byref(prm), ct.byref(hz), 0x2000, 0x3000, 0x4000, None, None, None, 0x5000, 0x6000, None, None, None,
            None)
    assert st == _abi.SPL_EINVAL and "sigma_rw2" in lib.spl_last_error().decode()
    prm = make_params(4, 4, 64, 25, 12, nu=[0] * 9)
    st = fn(ct.byref(prm), ct.byref(hz), 0x2000, 0x3000, 0x4000, None, None, None, 0x5000, 0x6000, None, None, None,
            None)
    assert st == _abi.SPL_EINVAL and "sum to 0" in lib.spl_last_error().decode()
    prm = make_params(4, 4, 64, 25, 12)
    st = fn(ct.byref(prm), ct.byref(hz), 0x2000, 0x3000, 0x4000, None, None, None, 0x3000, 0x6000, None, None, None,
            None)
    assert st == _abi.SPL_EINVAL and "alias" in lib.spl_last_error().decode()
    st = fn(ct.byref(prm), ct.byref(hz), 0x2000, 0x3000, 0x4000, None, None, None, 0x5000, 0x6000, None, 0x7000, None,
            None)
    assert st == _abi.SPL_EINVAL and "refl and bg" in lib.spl_last_error().decode()


def test_pi_and_init_argument_checks():
    lib = _abi.load()
    prm = make_params(4, 4, 64, 25, 12)
    assert lib.spl_pi_propagate(ct.byref(prm), 0x1000, None, 0x1000, None) == _abi.SPL_EINVAL
    assert lib.spl_state_init(ct.byref(prm), None, 0x1000, None) == _abi.SPL_EINVAL
    assert lib.spl_pi_propagate(None, 0x1000, None, 0x2000, None) == _abi.SPL_EINVAL


def test_batch_argument_checks():
    """Batch plans validate every sequence's parameters on the host before touching the device."""
    lib = _abi.load()
    good = make_params(4, 4, 64, 25, 12)
    bad = make_params(4, 4, 64, 25, 12, beta=-1.0)
    arr = (_abi.spl_params * 2)(good, bad)
    h = ct.c_void_p()
    assert lib.spl_batch_create(arr, 2, 1, ct.byref(h)) == _abi.SPL_EINVAL
    assert "sequence 1" in lib.spl_last_error().decode()
    assert lib.spl_batch_create(arr, 0, 1, ct.byref(h)) == _abi.SPL_EINVAL
    assert lib.spl_batch_create(arr, 1, 0, ct.byref(h)) == _abi.SPL_EINVAL
    assert lib.spl_batch_create(arr, 1, 1, None) == _abi.SPL_EINVAL
    assert lib.spl_batch_step(None, 0, None) == _abi.SPL_EINVAL
    assert lib.spl_batch_set(None, 0, None) == _abi.SPL_EINVAL
    assert lib.spl_batch_tune(None, 0, None) == _abi.SPL_EINVAL
    assert lib.spl_batch_info(None, None, None, None, None) == _abi.SPL_EINVAL
    assert lib.spl_batch_class_info(None, 0, None, None, None, None, None) == _abi.SPL_EINVAL
    assert lib.spl_batch_status(None, None) == _abi.SPL_EINVAL


def test_tensor_core_argument_checks():
    """spl_depth_cost_tc takes FP16 histograms only, spl_filter_step_tc FP16 or uint16 ones; both check the filter
    arguments like spl_filter_step, all on the host."""
    lib = _abi.load()
    prm = make_params(4, 4, 64, 25, 12)
    hz_u16 = _abi.spl_hist(_abi.SPL_HIST_U16, 0x1000, 64)
    hz_f16 = _abi.spl_hist(_abi.SPL_HIST_F16, 0x1000, 64)
    hz_f32 = _abi.spl_hist(_abi.SPL_HIST_F32, 0x1000, 64)
    st = lib.spl_depth_cost_tc(ct.byref(prm), ct.byref(hz_u16), 0x2000, 0x3000, None, None)
    assert st == _abi.SPL_EINVAL and "FP16" in lib.spl_last_error().decode()
    st = lib.spl_depth_cost_tc(ct.byref(prm), ct.byref(hz_f16), 0x2000, None, None, None)
    assert st == _abi.SPL_EINVAL and "nothing to compute" in lib.spl_last_error().decode()
    st = lib.spl_filter_step_tc(ct.byref(prm), ct.byref(hz_f32), 0x2000, 0x3000, 0x4000, None, None, None, 0x5000,
                                0x6000, None, None, None, None)
    assert st == _abi.SPL_EINVAL and "FP16 or uint16" in lib.spl_last_error().decode()
    st = lib.spl_filter_step_tc(ct.byref(prm), ct.byref(hz_f16), 0x2000, 0x3000, 0x4000, None, None, None, 0x3000,
                                0x6000, None, None, None, None)
    assert st == _abi.SPL_EINVAL and "alias" in lib.spl_last_error().decode()
    st = lib.spl_filter_step_tc(ct.byref(prm), ct.byref(hz_f16), 0x2000, 0x3000, 0x4000, None, None, None, 0x5000,
                                0x6000, None, 0x7000, None, None)
    assert st == _abi.SPL_EINVAL and "refl and bg" in lib.spl_last_error().decode()
    bad = make_params(4, 4, 64, 25, 12, sigma_rw2=0.0)
    st = lib.spl_filter_step_tc(ct.byref(bad), ct.byref(hz_f16), 0x2000, 0x3000, 0x4000, None, None, None, 0x5000,
                                0x6000, None, None, None, None)
    assert st == _abi.SPL_EINVAL and "sigma_rw2" in lib.spl_last_error().decode()
    assert lib.spl_tc_status(None) == _abi.SPL_EINVAL


def test_fine_grid_argument_checks():
    """spl_depth_estimate_fine: S in 1..16, the fine grid fits a warp's shared memory; checked on the host."""
    lib = _abi.load()
    prm = make_params(4, 4, 1500, 48, 5)
    hz = _abi.spl_hist(_abi.SPL_HIST_U16, 0x1000, 1504)
    st = lib.spl_depth_estimate_fine(ct.byref(prm), 0, ct.byref(hz), 0x2000, None, None, None, 0x3000, 0x4000, None)
    assert st == _abi.SPL_EINVAL and "S must be" in lib.spl_last_error().decode()
    st = lib.spl_depth_estimate_fine(ct.byref(prm), 17, ct.byref(hz), 0x2000, None, None, None, 0x3000, 0x4000, None)
    assert st == _abi.SPL_EINVAL
    st = lib.spl_depth_estimate_fine(ct.byref(prm), 16, ct.byref(hz), 0x2000, None, None, None, 0x3000, 0x4000, None)
    assert st == _abi.SPL_EUNSUPPORTED and "16384" in lib.spl_last_error().decode()
    st = lib.spl_depth_estimate_fine(ct.byref(prm), 4, ct.byref(hz), 0x2000, 0x5000, None, None, 0x3000, 0x4000, None)
    assert st == _abi.SPL_EINVAL and "prior_mu and prior_var" in lib.spl_last_error().decode()


def test_detect_argument_checks():
    """spl_filter_step_detect requires pi, refl and bg, keeps the filter's checks, and pi must not alias pi0;
    all decided on the host."""
    lib = _abi.load()
    prm = make_params(4, 4, 64, 25, 12)
    hz = _abi.spl_hist(_abi.SPL_HIST_U16, 0x1000, 64)
    #                    prm, z, h, mu_in, var_in, present_in, faulty, pi0, mu_out, var_out, argmax, pi, present, refl, bg
    st = lib.spl_filter_step_detect(ct.byref(prm), ct.byref(hz), 0x2000, 0x3000, 0x4000, None, None, None, 0x5000,
                                    0x6000, 0xa000, None, None, 0x7000, 0x8000, None)
    assert st == _abi.SPL_EINVAL and "argmax, pi, refl and bg" in lib.spl_last_error().decode()
    st = lib.spl_filter_step_detect(ct.byref(prm), ct.byref(hz), 0x2000, 0x3000, 0x4000, None, None, None, 0x5000,
                                    0x6000, None, 0x9000, None, 0x7000, 0x8000, None)
    assert st == _abi.SPL_EINVAL and "argmax, pi, refl and bg" in lib.spl_last_error().decode()
    st = lib.spl_filter_step_detect(ct.byref(prm), ct.byref(hz), 0x2000, 0x3000, 0x4000, None, None, 0x9000, 0x5000,
                                    0x6000, 0xa000, 0x9000, None, 0x7000, 0x8000, None)
    assert st == _abi.SPL_EINVAL and "alias pi0" in lib.spl_last_error().decode()
    st = lib.spl_filter_step_detect(ct.byref(prm), ct.byref(hz), 0x2000, 0x3000, 0x4000, None, None, None, 0x3000,
                                    0x6000, 0xa000, 0x9000, None, 0x7000, 0x8000, None)
    assert st == _abi.SPL_EINVAL and "alias" in lib.spl_last_error().decode()
    bad = make_params(4, 4, 64, 25, 12, beta=-1.0)
    st = lib.spl_filter_step_detect(ct.byref(bad), ct.byref(hz), 0x2000, 0x3000, 0x4000, None, None, None, 0x5000,
                                    0x6000, 0xa000, 0x9000, None, 0x7000, 0x8000, None)
    assert st == _abi.SPL_EINVAL


def test_multispectral_argument_checks():
    """spl_depth_estimate_msl: nbands in 1..SPL_MAX_BANDS, mu and var required, prior both or neither, the single-band
    parameter and layout checks; all decided on the host."""
    lib = _abi.load()
    prm = make_params(4, 4, 64, 25, 12)
    hz = _abi.spl_hist(_abi.SPL_HIST_U16, 0x1000, 64)
    #                    prm, nbands, z, h, prior_mu, prior_var, argmax, mu, var, cost, stream
    for nb in (0, _abi.SPL_MAX_BANDS + 1):
        st = lib.spl_depth_estimate_msl(ct.byref(prm), nb, ct.byref(hz), 0x2000, None, None, None, 0x3000, 0x4000,
                                        None, None)
        assert st == _abi.SPL_EINVAL and "nbands" in lib.spl_last_error().decode()
    st = lib.spl_depth_estimate_msl(ct.byref(prm), 2, ct.byref(hz), 0x2000, None, None, None, None, 0x4000, None, None)
    assert st == _abi.SPL_EINVAL and "mu and var" in lib.spl_last_error().decode()
    st = lib.spl_depth_estimate_msl(ct.byref(prm), 2, ct.byref(hz), 0x2000, 0x5000, None, None, 0x3000, 0x4000, None,
                                    None)
    assert st == _abi.SPL_EINVAL and "prior_mu and prior_var" in lib.spl_last_error().decode()
    st = lib.spl_depth_estimate_msl(ct.byref(prm), 2, ct.byref(hz), None, None, None, None, 0x3000, 0x4000, None, None)
    assert st == _abi.SPL_EINVAL and "h is NULL" in lib.spl_last_error().decode()
    bad = _abi.spl_hist(_abi.SPL_HIST_U16, 0x1000, 68)  # 136-byte rows
    st = lib.spl_depth_estimate_msl(ct.byref(prm), 2, ct.byref(bad), 0x2000, None, None, None, 0x3000, 0x4000, None,
                                    None)
    assert st == _abi.SPL_EINVAL and "16 bytes" in lib.spl_last_error().decode()
    out = make_params(4, 4, 64, 25, 12, dmin=5)
    st = lib.spl_depth_estimate_msl(ct.byref(out), 2, ct.byref(hz), 0x2000, None, None, None, 0x3000, 0x4000, None,
                                    None)
    assert st == _abi.SPL_EINVAL and "full-support" in lib.spl_last_error().decode()


def test_throughput_probe_size_query():
    """spl_probe_throughput answers its size query on the host (no launch without buffers) and rejects bad kinds."""
    lib = _abi.load()
    nb, opt = ct.c_int(0), ct.c_longlong(0)
    assert lib.spl_probe_throughput(7, 4, 16, None, None, ct.byref(nb), ct.byref(opt), None) == _abi.SPL_EINVAL
    assert lib.spl_probe_throughput(0, 0, 16, None, None, ct.byref(nb), ct.byref(opt), None) == _abi.SPL_EINVAL


@pytest.mark.parametrize("args, needle", [
    (dict(offsets=None), "offsets"),
    (dict(bins=None), "bins is NULL"),
    (dict(nph=-1), "nphotons"),
    (dict(out=None), "out is NULL"),
    (dict(out=0x3008), "16-byte aligned"),
    (dict(pitch=60), "pitch"),
    (dict(pitch=68), "pitch"),
    (dict(T=9000, pitch=9000), "not supported"),
])
def test_toa_histogram_argument_checks(args, needle):
    """spl_toa_histogram checks its arguments on the host (nothing is launched): offsets and out are required,
    bins unless there are no photons, out 16-byte aligned, pitch >= T and a multiple of 8, T <= SPL_MAX_BINS."""
    lib = _abi.load()
    kw = dict(offsets=0x1000, bins=0x2000, nph=10, out=0x3000, pitch=64, T=64)
    kw.update(args)
    prm = make_params(4, 4, kw["T"], 1, 0)
    st = lib.spl_toa_histogram(ct.byref(prm), kw["offsets"], kw["bins"], kw["nph"], kw["out"], kw["pitch"], None)
    assert st in (_abi.SPL_EINVAL, _abi.SPL_EUNSUPPORTED)
    assert needle in lib.spl_last_error().decode()
    assert lib.spl_toa_status(None) == _abi.SPL_EINVAL


def test_toa_histogram_binding_refuses_host_tensors():
    """The binding passes device pointers only: host tensors are refused before anything reaches the library."""
    import torch
    import paper_2004_09211_gb300 as spl
    prm = make_params(2, 2, 64, 1, 0)
    off = torch.zeros(5, dtype=torch.int32)
    bins = torch.zeros(0, dtype=torch.uint16)
    with pytest.raises(TypeError, match="CUDA tensor"):
        spl.spl_toa_histogram(prm, off, bins, out=torch.zeros((4, 64), dtype=torch.int32).to(torch.uint16))
