"""The full field in the final refit (Sec. 3: Bx, By and a three-dimensional
polynomial field) on the GPU against the FP64 oracle, on particles traced
through a non-uniform solenoid-like field."""
import numpy as np
import pytest

import oracle
import synth
from paper_1811_11481_b300.config import default_params
from pipeline import RTOL, refit_tolerance, rel_err

pytestmark = pytest.mark.gpu


def _tracker(geo, field):
    from paper_1811_11481_b300.binding import Tracker
    return Tracker(geo, default_params(), field=field)


@pytest.mark.parametrize("mode", ["event", "time"])
def test_field_refit_matches_the_oracle(mode):
    import torch
    from synth.field import solenoid_field
    geo = synth.geometry()
    f = solenoid_field(eps=0.04)
    ev = synth.make_tiny(seed=64, n_tracks=400, central=True, mode=mode, tf_start=1.0e6,
                         n_coll=2, noise_frac=0.05, field=f)
    tr = _tracker(geo, f)
    tr.set_calib()
    tr.load(tr.upload(ev))
    g = {k: v.cpu().numpy() for k, v in tr.find().items()}
    r = {k: v.cpu().numpy() for k, v in tr.refit().items()}
    nt = tr.n_tracks
    o = oracle.Oracle(ev, geo, default_params(), synth.nominal_calib(), field=f)
    ref = o.refit(g["track_start"], g["cluster_idx"], g["t_coll"], prec=64)
    ts = g["track_start"].astype(np.int64)
    same = np.array([np.array_equal(r["rej"][ts[k]:ts[k + 1]], ref["rej"][ts[k]:ts[k + 1]])
                     for k in range(nt)])
    assert np.mean(r["status"] == ref["status"]) > 0.99
    ok = (r["status"] == 0) & (ref["status"] == 0) & same
    assert ok.sum() > 0.95 * np.sum(ref["status"] == 0) and ok.sum() > 200
    e = rel_err(r["params"][ok].astype(np.float64), ref["params"][ok])
    tol, mirror = refit_tolerance(o, g["track_start"], g["cluster_idx"], g["t_coll"], ref, ok)
    print(f"field {mode}: max error {e.max(0)}, FP32 mirror {mirror}")
    assert np.all(e <= tol), (e.max(0), tol)
    assert np.mean(np.all(e <= RTOL, axis=1)) > 0.99
    np.testing.assert_allclose(r["chi2"][ok], ref["chi2"][ok], rtol=2e-3, atol=1e-2)
    # the uniform-field refit of the same tracks is farther from the oracle's
    # full-field fit in q/pT
    tr2 = _tracker(geo, None)
    tr2.set_calib()
    tr2.load(tr2.upload(ev))
    tr2.find()
    ru = {k: v.cpu().numpy() for k, v in tr2.refit().items()}
    ok2 = ok & (ru["status"] == 0)
    eu = rel_err(ru["params"][ok2].astype(np.float64), ref["params"][ok2])[:, 4]
    assert np.median(eu) > 10 * np.median(e[:, 4])


@pytest.mark.parametrize("merged", [False, True])
def test_field_adjoint_matches_the_oracle_gradient(merged):
    """The adjoint of the full-field refit (reverse sweep through the
    Runge-Kutta sub-steps and the local Bz of the helix part) against the
    oracle's reverse-mode tape through the same transport, on truth tracks
    per sector and merged across sectors."""
    import torch
    from synth.field import solenoid_field
    geo = synth.geometry()
    f = solenoid_field(eps=0.04)
    ev = synth.make_tiny(seed=65, n_tracks=300, central=True, field=f, noise_frac=0.0)
    ts, ci, tc, _ = synth.truth_tracks(ev, 30, merged=merged)
    tr = _tracker(geo, f)
    tr.set_calib()
    tr.load(tr.upload(ev))
    tr.set_tracks(torch.as_tensor(ts.astype(np.int32)), torch.as_tensor(ci.astype(np.int32)),
                  torch.as_tensor(tc))
    r = {k: v.cpu().numpy() for k, v in tr.refit(save_for_backward=True).items()}
    nt = ts.size - 1
    w = torch.linspace(0.5, 1.5, nt, device=tr.dev)
    gy, gz, _ = [t.cpu().numpy() for t in tr.refit_backward(w)]
    o = oracle.Oracle(ev, geo, default_params(), synth.nominal_calib(), field=f)
    ref = o.refit(ts, ci, tc, prec=64)
    ry, rz, _ = o.refit_grad(ts, ci, tc, ref["seeds"], r["rej"],
                             w.cpu().numpy().astype(np.float64))
    ok = (r["status"] == 0) & (ref["status"] == 0)
    assert ok.sum() > (40 if merged else 150)   # merged loopers reach s_max
    m = np.repeat(ok, np.diff(ts.astype(np.int64)))
    for a, b in ((gy, ry), (gz, rz)):
        assert np.linalg.norm(a[m] - b[m]) / np.linalg.norm(b[m]) < 1e-3
