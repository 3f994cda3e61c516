"""The allocation-free refit entry point (tpc_refit_noalloc).

Callers that cannot allocate device memory at refit time -- inside a CUDA
graph capture, in a real-time loop, or under a framework whose allocator owns
the device -- use tpc_refit_noalloc, which keeps its working memory in a fixed
device array. This test calls it through the C ABI twice in a row (two
different track sets, so the shared array is reused) and compares each result
with the context-based tpc_refit of the same tracks, within the refit
tolerance used by the other parity tests.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from pipeline import RTOL, rel_err, tracker

pytestmark = pytest.mark.gpu


def _noalloc(tr, ts, yc, zc, row, flags):
    import torch
    from paper_1811_11481_b300 import binding
    L = binding.load_library()
    nt = ts.numel() - 1
    na = yc.numel()
    dev = tr.dev
    out = dict(params=torch.full((nt, 5), float("nan"), device=dev),
               cov=torch.full((nt, 15), float("nan"), device=dev),
               chi2=torch.full((nt,), float("nan"), device=dev),
               ndf=torch.full((nt,), -7, dtype=torch.int32, device=dev),
               status=torch.full((nt,), -7, dtype=torch.int32, device=dev))
    geo = synth.geometry()
    rx = np.ascontiguousarray(geo.row_x, np.float32)
    g = binding.tpc_geometry(rx.size, rx.ctypes.data_as(C.POINTER(C.c_float)),
                             float(geo.tan_half), float(geo.drift_length), float(geo.bz))
    P = lambda t: C.c_void_p(t.data_ptr())
    st = L.tpc_refit_noalloc(C.byref(g), None, C.c_void_p(torch.cuda.current_stream().cuda_stream),
                             nt, na, P(ts), P(yc), P(zc), P(row), P(flags), P(out["params"]),
                             P(out["cov"]), P(out["chi2"]), P(out["ndf"]), P(out["status"]))
    assert st == 0, st
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _reference(geo, ev, ts, ci, tc):
    """The context path on the same tracks: calibrated inputs and refit."""
    import torch
    tr = tracker(geo)
    tr.set_calib()
    cl = tr.upload(ev)
    tr.load(cl)
    tr.set_tracks(torch.as_tensor(ts.astype(np.int32)), torch.as_tensor(ci.astype(np.int32)),
                  torch.as_tensor(tc))
    r = tr.refit()
    yc, zc = tr.calibrated()
    ref = {k: v.cpu().numpy() for k, v in r.items()}
    idx = torch.as_tensor(ci.astype(np.int64), device=tr.dev)
    inputs = dict(ts=torch.as_tensor(ts.astype(np.int32), device=tr.dev), yc=yc.contiguous(),
                  zc=zc.contiguous(), row=cl["row"][idx].contiguous(),
                  flags=cl["flags"][idx].contiguous())
    return tr, ref, inputs


def _compare(got, ref):
    assert np.array_equal(got["status"], ref["status"])
    ok = ref["status"] == 0
    assert ok.sum() > 0
    np.testing.assert_array_equal(got["ndf"][ok], ref["ndf"][ok])
    e = rel_err(got["params"][ok].astype(np.float64), ref["params"][ok].astype(np.float64))
    assert np.all(e <= RTOL), e.max(0)
    np.testing.assert_allclose(got["chi2"][ok], ref["chi2"][ok], rtol=1e-4, atol=1e-4)


def test_noalloc_refit_matches_context_refit_twice():
    geo = synth.geometry()
    ev = synth.make_tiny(seed=41, n_tracks=400, central=True, noise_frac=0.05)
    ts, ci, tc, _ = synth.truth_tracks(ev, 20)
    # first call: all tracks
    tr, ref, inp = _reference(geo, ev, ts, ci, tc)
    got = _noalloc(tr, inp["ts"], inp["yc"], inp["zc"], inp["row"], inp["flags"])
    _compare(got, ref)
    # second call: a different, smaller track set reusing the same scratch
    k = (ts.size - 1) // 2
    ts2 = (ts[k:] - ts[k]).astype(np.uint32)
    ci2 = ci[ts[k]:]
    tr2, ref2, inp2 = _reference(geo, ev, ts2, ci2, tc[k:])
    got2 = _noalloc(tr2, inp2["ts"], inp2["yc"], inp2["zc"], inp2["row"], inp2["flags"])
    _compare(got2, ref2)


def test_noalloc_rejects_oversized_input_before_any_work():
    from paper_1811_11481_b300 import binding
    L = binding.load_library()
    geo = synth.geometry()
    rx = np.ascontiguousarray(geo.row_x, np.float32)
    g = binding.tpc_geometry(rx.size, rx.ctypes.data_as(C.POINTER(C.c_float)),
                             float(geo.tan_half), float(geo.drift_length), float(geo.bz))
    too_many = (1 << 20) + 1
    st = L.tpc_refit_noalloc(C.byref(g), None, None, 10, too_many, *([None] * 10))
    assert st == 2  # TPC_ERR_CAPACITY
