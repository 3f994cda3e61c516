"""Launch-shape tuning: every tuning gives the same outputs bit for bit, the
autotuner picks among its candidates, and invalid tunings are refused."""
import numpy as np
import pytest

import synth
from paper_1811_11481_b300.binding import TpcError
from pipeline import tracker

pytestmark = pytest.mark.gpu

# corners of the tuning space (the autotuner's candidates lie inside)
TUNINGS = [
    dict(grid_tau=0.125, grid_ny_max=1, tracklet_block=64, tracklet_per_sm=1, tracklet_regs=0),
    dict(grid_tau=0.25, grid_ny_max=16, tracklet_block=128, tracklet_per_sm=0, tracklet_regs=96),
    dict(grid_tau=4.0, grid_ny_max=64, tracklet_block=256, tracklet_per_sm=0, tracklet_regs=96),
    dict(grid_tau=16.0, grid_ny_max=8, tracklet_block=128, tracklet_per_sm=2, tracklet_regs=96),
    dict(grid_tau=1.0, grid_ny_max=16, tracklet_block=64, tracklet_per_sm=0, tracklet_regs=96),
]


def _run(tr, cl):
    import torch
    tr.load(cl)
    out = tr.find()
    r = tr.refit(save_for_backward=True)
    nt = tr.n_tracks
    gy, gz, gc = tr.refit_backward(torch.ones(max(nt, 1)))
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res.update({k: v[:nt].cpu().numpy() for k, v in r.items() if k != "rej"})
    res.update(gy=gy.cpu().numpy(), gz=gz.cpu().numpy(), gc=gc.cpu().numpy())
    return res


def _same(a, b):
    assert a.keys() == b.keys()
    for k in a:
        assert np.array_equal(a[k], b[k], equal_nan=True), k


@pytest.mark.parametrize("mode", ["event", "time"])
def test_outputs_do_not_depend_on_tuning(mode):
    geo = synth.geometry()
    ev = synth.make_tiny(seed=61, n_tracks=400, sectors=(0, 5, 20, 33), noise_frac=0.1,
                         mode=mode, n_coll=3 if mode == "time" else 1)
    tr = tracker(geo)
    tr.set_calib()
    cl = tr.upload(ev)
    ref = _run(tr, cl)
    assert tr.n_tracks > 20
    for t in TUNINGS:
        tr.set_tuning(**t)
        assert tr.get_tuning() == pytest.approx(t)
        _same(_run(tr, cl), ref)


def test_autotune_chooses_a_candidate_and_keeps_results():
    geo = synth.geometry()
    ev = synth.make_batched(seed=62, n_events=6, lo=50, hi=800)
    tr = tracker(geo)
    tr.set_calib()
    cl = tr.upload(ev)
    ref = _run(tr, cl)
    t = tr.autotune(repeats=2)
    assert t["grid_tau"] in (0.25, 0.5, 1.0, 2.0, 4.0)
    assert t["grid_ny_max"] in (8, 16, 32)
    assert t["tracklet_block"] in (64, 128, 256)
    assert t["tracklet_per_sm"] in (0, 1, 2, 4)
    assert t["tracklet_regs"] in (0, 96)
    assert tr.get_tuning() == t
    # the batch stays loaded and found with the chosen tuning
    nt, na, _ = tr.counts()
    assert (nt, na) == (len(ref["track_start"]) - 1, len(ref["cluster_idx"]))
    _same(_run(tr, cl), ref)


def test_invalid_tuning_is_refused():
    tr = tracker(synth.geometry())
    good = tr.get_tuning()
    for bad in (dict(grid_tau=0.0), dict(grid_tau=100.0), dict(grid_ny_max=0),
                dict(tracklet_block=96), dict(tracklet_block=512), dict(tracklet_per_sm=-1),
                dict(tracklet_regs=64), dict(tracklet_regs=-1)):
        with pytest.raises(TpcError) as ei:
            tr.set_tuning(**bad)
        assert ei.value.status == 1
        assert tr.get_tuning() == good
    with pytest.raises(TpcError) as ei:
        tr.autotune()                     # nothing loaded
    assert ei.value.status == 5
