"""Native pad coordinates (the paper's next step after Sec. 4: tracking in
native pad, row and time coordinates, transformed on the fly): the CUDA path
fed with pad positions against the oracle fed with the same pads — every
discrete stage up to counted near-ties; refit within the tolerance; gradient per pad within 1e-3
relative norm — and against the CUDA path fed with the transformed y."""
import numpy as np
import pytest

import oracle
import synth
from oracle import parity
from paper_1811_11481_b300.config import default_params
from pipeline import RTOL, rel_err, tracker

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["event", "time"])
def test_native_pads_parity(mode):
    import torch
    geo = synth.geometry()
    cal = synth.nominal_calib()
    if mode == "time":
        cal.spline = synth.random_distortion(np.random.default_rng(10), 0.8)
    ev = synth.make_tiny(seed=53, n_tracks=300, central=True, mode=mode, tf_start=1.0e6,
                         n_coll=2, noise_frac=0.1, calib=cal)
    tr = tracker(geo)
    tr.set_calib(cal.vdrift, cal.t0, cal.spline)
    tr.load(tr.upload(ev, pads=True))
    g = {k: v.cpu().numpy() for k, v in tr.find().items()}
    g["up"], g["dn"], g["upc"], g["dnc"] = [t.cpu().numpy() for t in tr.links()]
    g["tracklets"] = {k: v.cpu().numpy() for k, v in tr.tracklets().items()}
    r = tr.refit(save_for_backward=True)
    nt = tr.n_tracks
    w = torch.linspace(0.5, 1.5, nt, device=tr.dev)
    gy, gz, gc = [t.cpu().numpy() for t in tr.refit_backward(w)]
    o = oracle.Oracle(ev, geo, default_params(), cal, pads=True)
    print(f"native pads, {mode}: {parity.find(o, g, mode == 'time')}")
    ts = g["track_start"].astype(np.int64)
    assert nt > 100
    ref = o.refit(g["track_start"], g["cluster_idx"], g["t_coll"], prec=64)
    gotr = {k: v.cpu().numpy() for k, v in r.items()}
    same = np.array([np.array_equal(gotr["rej"][ts[k]:ts[k + 1]], ref["rej"][ts[k]:ts[k + 1]])
                     for k in range(nt)])
    ok = (gotr["status"] == 0) & (ref["status"] == 0) & same
    assert ok.sum() > 0.95 * nt
    e = rel_err(gotr["params"][ok].astype(np.float64), ref["params"][ok])
    assert np.all(e <= RTOL), e.max(0)
    ry, rz, rc = o.refit_grad(g["track_start"], g["cluster_idx"], g["t_coll"], ref["seeds"],
                              gotr["rej"], w.cpu().numpy().astype(np.float64))
    m = np.repeat((gotr["status"] == 0) & (ref["status"] == 0), np.diff(ts))
    for a, b in ((gy, ry), (gz, rz)):
        assert np.linalg.norm(a[m] - b[m]) / np.linalg.norm(b[m]) < 1e-3
    # the same event given in cm (the transformed y): the same tracks bit for bit
    row = ev.row.astype(np.int64)
    ev.y[:] = ((ev.pad - geo.pad_center[row]) * geo.pad_width[row]).astype(np.float32)
    tr2 = tracker(geo)
    tr2.set_calib(cal.vdrift, cal.t0, cal.spline)
    tr2.load(tr2.upload(ev))
    g2 = {k: v.cpu().numpy() for k, v in tr2.find().items()}
    for k in ("track_start", "cluster_idx", "t_coll", "start_hit"):
        np.testing.assert_array_equal(g2[k], g[k], err_msg=k)
    r2 = tr2.refit()
    for k in ("params", "chi2", "status"):
        assert torch.equal(r2[k], r[k]), k


def test_native_pads_need_the_pad_tables():
    import torch
    from paper_1811_11481_b300.binding import TpcError
    geo = synth.geometry()
    geo_nopad = synth.Geometry(row_x=geo.row_x, tan_half=geo.tan_half,
                               drift_length=geo.drift_length, bz=geo.bz)
    ev = synth.make_tiny(seed=54, n_tracks=20)
    tr = tracker(geo_nopad)
    tr.set_calib()
    with pytest.raises(TpcError) as ei:
        tr.load(tr.upload(ev, pads=True))
    assert ei.value.status == 1
