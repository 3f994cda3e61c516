"""Frames in flight: two contexts on their own CUDA streams, their calls
issued interleaved so that their kernels overlap on the GPU, give outputs
bit-identical to the same frames run one after the other on one context
(tracks, refit, adjoint)."""
import numpy as np
import pytest

import synth
from pipeline import tracker

pytestmark = pytest.mark.gpu


def _frames():
    return [synth.make_tiny(seed=81, n_tracks=500, central=True, noise_frac=0.1, mode="time",
                            tf_start=1.0e6, n_coll=3),
            synth.make_tiny(seed=82, n_tracks=400, central=True, noise_frac=0.1)]


def _collect(tr, r, g):
    f = tr.tracks()
    out = {k: v.cpu().numpy() for k, v in f.items()}
    out.update({"r_" + k: v.cpu().numpy() for k, v in r.items()})
    out.update(gy=g[0].cpu().numpy(), gz=g[1].cpu().numpy(), gc=g[2].cpu().numpy())
    return out


def test_frames_in_flight_equal_serial_frames():
    import torch
    geo = synth.geometry()
    evs = _frames()
    # serial: one context, frame after frame
    tr = tracker(geo)
    tr.set_calib()
    want = []
    for ev in evs:
        tr.load(tr.upload(ev))
        tr.find()
        r = tr.refit(save_for_backward=True)
        g = tr.refit_backward(torch.ones(tr.n_tracks, device=tr.dev))
        want.append(_collect(tr, r, g))
    # in flight: one context per frame, each on its own stream, calls
    # interleaved (asynchronous find), three rounds
    from paper_1811_11481_b300.binding import Tracker
    from paper_1811_11481_b300.config import default_params
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    trs = [Tracker(geo, default_params(), stream=s) for s in streams]
    cls = []
    for t, ev in zip(trs, evs):
        t.set_calib()
        cls.append(t.upload(ev))
    for _ in range(3):
        for t, cl in zip(trs, cls):
            t.load(cl)
        for t in trs:
            t.find_async()
        rs = [t.refit(save_for_backward=True, n_tracks=None) for t in trs]
    torch.cuda.synchronize()
    for t, r, w in zip(trs, rs, want):
        t.counts()
        g = t.refit_backward(torch.ones(t.n_tracks, device=t.dev))
        got = _collect(t, r, g)
        assert set(got) == set(w)
        for k in w:
            assert np.array_equal(got[k], w[k], equal_nan=True), k
