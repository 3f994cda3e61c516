"""Vertex pseudo-measurements in the refit and its adjoint (tpc_set_vertex)
against the FP64 oracle: truth tracks of a distorted time frame, the first
outgoing leg of each particle with its vertex z (the other legs without),
parameters at the beam line, chi2 and ndf within the refit tolerance, and
the adjoint within 1e-3 relative norm of the oracle's tape gradient per
block (clusters, v_drift, t0, spline)."""
import numpy as np
import pytest

import oracle
import synth
from paper_1811_11481_b300.config import default_params
from pipeline import RTOL, rel_err, tracker

pytestmark = pytest.mark.gpu


def _vertex_tracks(ev, min_hits=40):
    ts, ci, tc, sids = synth.truth_tracks(ev, min_hits)
    lab = ev.label[ci[ts[:-1].astype(np.int64)]]
    zv = np.asarray(ev.part["zv"], np.float64)[lab]
    zv[sids % 4 != 0] = np.nan
    return ts, ci, tc, zv


def test_vertex_refit_and_adjoint_match_the_oracle():
    import torch
    geo = synth.geometry()
    cal = synth.nominal_calib()
    cal.spline = synth.random_distortion(np.random.default_rng(12), 0.8)
    ev = synth.make_tiny(seed=38, n_tracks=300, central=True, mode="time", tf_start=1.0e6,
                         n_coll=2, calib=cal)
    ts, ci, tc, zv = _vertex_tracks(ev)
    tr = tracker(geo)
    tr.set_calib(cal.vdrift, cal.t0, cal.spline)
    tr.load(tr.upload(ev))
    tr.set_tracks(torch.as_tensor(ts.astype(np.int32)), torch.as_tensor(ci.astype(np.int32)),
                  torch.as_tensor(tc))
    tr.set_vertex(torch.as_tensor(zv.astype(np.float32)), 0.01)
    r = {k: v.cpu().numpy() for k, v in tr.refit(save_for_backward=True).items()}
    o = oracle.Oracle(ev, geo, default_params(), cal)
    ref = o.refit(ts, ci, tc, prec=64, zv=zv.astype(np.float32).astype(np.float64))
    has = ~np.isnan(zv)
    ok = (r["status"] == 0) & (ref["status"] == 0)
    same = np.array([np.array_equal(r["rej"][ts[k]:ts[k + 1]], ref["rej"][ts[k]:ts[k + 1]])
                     for k in range(ts.size - 1)])
    sel = ok & same
    assert sel.sum() > 0.98 * ok.sum() and (sel & has).sum() > 100
    # the vertex was used (state at the beam line) exactly where the oracle used it
    assert np.array_equal(r["x"][sel] == 0.0, ref["x"][sel] == 0.0)
    assert np.all(r["x"][sel & ~has] != 0.0)
    e = rel_err(r["params"][sel].astype(np.float64), ref["params"][sel])
    assert np.all(e <= RTOL), e.max(0)
    np.testing.assert_array_equal(r["ndf"][sel], ref["ndf"][sel])
    np.testing.assert_allclose(r["chi2"][sel], ref["chi2"][sel], rtol=2e-3, atol=1e-2)
    w = torch.linspace(0.5, 1.5, ts.size - 1, device=tr.dev)
    gy, gz, gc = [t.cpu().numpy() for t in tr.refit_backward(w)]
    ry, rz, rc = o.refit_grad(ts, ci, tc, ref["seeds"], r["rej"],
                              w.cpu().numpy().astype(np.float64),
                              zv=zv.astype(np.float32).astype(np.float64))
    m = np.repeat(ok, np.diff(ts.astype(np.int64)))
    for a, b in ((gy, ry), (gz, rz)):
        assert np.linalg.norm(a[m] - b[m]) / np.linalg.norm(b[m]) < 1e-3
    # v_drift and t0: sums over clusters whose terms largely cancel (without
    # a vertex exactly, for t0), each compared with the sum of its terms'
    # magnitudes (rz is per drift time); the spline block by relative norm
    ci64 = ci.astype(np.int64)
    drift = np.abs(ev.t[ci64] - cal.t0 - np.repeat(tc, np.diff(ts.astype(np.int64))))
    scales = (np.sum(np.abs(rz[m]) * drift[m]) / cal.vdrift, np.sum(np.abs(rz[m])))
    for k, scale in enumerate(scales):
        assert abs(gc[k] - rc[k]) <= 1e-3 * scale, (k, gc[k], rc[k], scale)
    err = np.linalg.norm(gc[2:] - rc[2:]) / np.linalg.norm(rc[2:])
    assert err < 1e-3, err


def test_vertex_state_errors():
    import torch
    from paper_1811_11481_b300.binding import TpcError
    geo = synth.geometry()
    ev = synth.make_tiny(seed=39, n_tracks=40, central=True, mode="time", tf_start=1.0e6)
    ts, ci, tc, zv = _vertex_tracks(ev)
    tr = tracker(geo)
    tr.set_calib()
    tr.load(tr.upload(ev))
    tr.set_tracks(torch.as_tensor(ts.astype(np.int32)), torch.as_tensor(ci.astype(np.int32)),
                  torch.as_tensor(tc))
    with pytest.raises(TpcError) as ei:
        tr.set_vertex(torch.as_tensor(zv.astype(np.float32)), 0.0)
    assert ei.value.status == 1
    tr.refit(save_for_backward=True)
    tr.set_vertex(torch.as_tensor(zv.astype(np.float32)), 0.01)
    # vertices set after the saved refit: the adjoint refuses
    with pytest.raises(TpcError) as ei:
        tr.refit_backward(torch.ones(ts.size - 1, device=tr.dev))
    assert ei.value.status == 5
