"""tpc_find_tracks_batched: several cluster sets loaded as one batch.

The parts are concatenated in order, each part's events numbered after the
events of the parts before it. On the same clusters in the same order the
call must give exactly the tracks of tpc_find_tracks on the concatenated
batch; a time frame split into two parts by sector (sectors are
independent, Sec. 2) must give the same tracks as the whole frame.
"""
import numpy as np
import pytest

import synth
from pipeline import canonical_tracks, tracker

pytestmark = pytest.mark.gpu


def _reorder(ev, perm):
    for k in ("y", "z", "t", "row", "sector", "flags", "event", "pad", "segment", "label"):
        v = getattr(ev, k, None)
        if v is not None and np.ndim(v) == 1 and len(v) == ev.n:
            setattr(ev, k, v[perm])
    return ev


def _part(cl, idx, n_events=1, event=None):
    import torch
    ix = torch.as_tensor(idx, device=cl["y"].device)
    d = dict(mode=cl["mode"], n_events=n_events, tf_start=cl["tf_start"], pads=cl["pads"])
    for k in ("y", "z", "t", "row", "sector", "flags"):
        d[k] = cl[k][ix].contiguous() if cl.get(k) is not None else None
    d["event"] = event
    return d


def _tracks(out):
    return canonical_tracks(out["track_start"].cpu().numpy(), out["cluster_idx"].cpu().numpy(),
                            out["start_hit"].cpu().numpy(), out["t_coll"].cpu().numpy())


def test_batched_call_equals_one_batch():
    geo = synth.geometry()
    ev = synth.make_batched(seed=34, n_events=5, lo=5, hi=150)
    ev = _reorder(ev, np.argsort(ev.event, kind="stable"))
    tr = tracker(geo)
    tr.set_calib()
    cl = tr.upload(ev)
    tr.load(cl)
    whole = tr.find()
    r_whole = {k: v.cpu().numpy() for k, v in tr.refit().items()}
    parts = [_part(cl, np.nonzero(ev.event == k)[0]) for k in range(ev.n_events)]
    tr2 = tracker(geo)
    tr2.set_calib()
    got = tr2.find_batched(parts)
    for k in ("track_start", "cluster_idx", "t_coll", "start_hit"):
        assert np.array_equal(got[k].cpu().numpy(), whole[k].cpu().numpy()), k
    r_got = {k: v.cpu().numpy() for k, v in tr2.refit().items()}
    for k in ("params", "chi2", "status"):
        assert np.array_equal(r_got[k], r_whole[k]), k


def test_time_frame_split_by_sector_gives_the_same_tracks():
    import torch
    geo = synth.geometry()
    ev = synth.make_tiny(seed=32, n_tracks=250, central=True, noise_frac=0.15, mode="time",
                         tf_start=1.0e6, n_coll=4)
    lo = (ev.sector % 18) < 9
    ev = _reorder(ev, np.concatenate([np.nonzero(lo)[0], np.nonzero(~lo)[0]]))
    lo = (ev.sector % 18) < 9
    tr = tracker(geo)
    tr.set_calib()
    cl = tr.upload(ev)
    tr.load(cl)
    sw, lw, tw = _tracks(tr.find())
    tr2 = tracker(geo)
    tr2.set_calib()
    parts = [_part(cl, np.nonzero(lo)[0]), _part(cl, np.nonzero(~lo)[0])]
    sg, lg, tg = _tracks(tr2.find_batched(parts))
    assert len(lw) > 0
    assert np.array_equal(sg, sw)
    for a, b in zip(lg, lw):
        assert np.array_equal(a, b)
    assert np.array_equal(tg, tw)


def test_batched_call_rejects_inconsistent_parts():
    from paper_1811_11481_b300.binding import TpcError
    geo = synth.geometry()
    ev = synth.make_batched(seed=34, n_events=2, lo=5, hi=20)
    tr = tracker(geo)
    tr.set_calib()
    cl = tr.upload(ev)
    a = _part(cl, np.arange(ev.n))
    b = dict(a, mode=1, t=a["y"].double(), z=None)
    with pytest.raises(TpcError):
        tr.find_batched([a, b])
