"""CUDA-graph capture and replay of a whole step through the C ABI."""
import ctypes as C

import pytest

import synth
from paper_1811_11481_b300.binding import TPC_GRAD_CALIB_SIZE, TpcError, Tracker
from paper_1811_11481_b300.config import default_params

pytestmark = pytest.mark.gpu


def _step_buffers(torch, dev, n):
    cap = n // 10 + 1
    return dict(params=torch.zeros(cap, 5, device=dev), cov=torch.zeros(cap, 15, device=dev),
                x=torch.zeros(cap, device=dev), chi2=torch.zeros(cap, device=dev),
                ndf=torch.zeros(cap, dtype=torch.int32, device=dev),
                status=torch.zeros(cap, dtype=torch.int32, device=dev),
                rej=torch.zeros(n + 1, dtype=torch.uint8, device=dev),
                ones=torch.ones(cap, device=dev), gy=torch.zeros(n + 1, device=dev),
                gz=torch.zeros(n + 1, device=dev),
                gc=torch.zeros(TPC_GRAD_CALIB_SIZE, dtype=torch.float64, device=dev))


def _step(tr, cl, b):
    P = lambda t: C.c_void_p(t.data_ptr())
    L, h = tr.L, tr.h
    tr.load(cl)
    assert L.tpc_find_tracks_async(h) == 0
    assert L.tpc_refit(h, 1, P(b["params"]), P(b["cov"]), P(b["x"]), P(b["chi2"]), P(b["ndf"]),
                       P(b["status"]), P(b["rej"])) == 0
    assert L.tpc_refit_backward(h, P(b["ones"]), P(b["gy"]), P(b["gz"]), P(b["gc"])) == 0


def test_graph_replay_equals_direct_run():
    import torch
    geo = synth.geometry()
    ev = synth.make_batched(seed=38, n_events=8, lo=20, hi=400)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        tr = Tracker(geo, default_params(), stream=stream)
        tr.set_calib()
        cl = tr.upload(ev)
        b = _step_buffers(torch, tr.dev, ev.n)
        _step(tr, cl, b)                      # allocates every buffer
        nt, na, _ = tr.counts()
        ref = {k: v.clone() for k, v in b.items()}
        for k, v in b.items():
            if v.dtype.is_floating_point and k != "ones":
                v.fill_(float("nan"))
        stream.synchronize()
        tr.graph_begin()
        # a synchronising call is refused while capturing
        with pytest.raises(TpcError) as ei:
            tr.counts()
        assert ei.value.status == 5
        _step(tr, cl, b)                      # recorded, not run
        tr.graph_end()
        tr.graph_launch()
        tr.graph_launch()                     # replay twice
        stream.synchronize()
        nt2, na2, _ = tr.counts()
    assert (nt2, na2) == (nt, na) and nt > 0
    for k in ("params", "cov", "chi2", "ndf", "status"):
        assert torch.equal(b[k][:nt], ref[k][:nt]), k
    assert torch.equal(b["rej"][:na], ref["rej"][:na])
    assert torch.equal(b["gy"][:na], ref["gy"][:na])
    # the calibration gradient sums in fixed point: reproducible bit for bit
    assert torch.equal(b["gc"], ref["gc"])
    assert torch.equal(b["gz"][:na], ref["gz"][:na])


def test_allocation_during_capture_is_refused():
    import torch
    geo = synth.geometry()
    ev = synth.make_tiny(seed=39, n_tracks=30)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        tr = Tracker(geo, default_params(), stream=stream)
        tr.set_calib()
        cl = tr.upload(ev)
        stream.synchronize()
        tr.graph_begin()
        with pytest.raises(TpcError) as ei:
            tr.load(cl)                       # first load allocates
        assert ei.value.status == 5
        tr.graph_end()                        # nothing was recorded
        stream.synchronize()
        # the context is usable afterwards
        tr.load(cl)
        tr.find()
        assert tr.n_tracks > 0
