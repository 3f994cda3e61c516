"""The full field in the final refit (Sec. 3: Bx, By and a three-dimensional
polynomial field) on the GPU against the FP64 oracle, on particles traced
through a non-uniform solenoid-like field."""
import numpy as np
import pytest

import oracle
import synth
from paper_1811_11481_b300.config import default_params
from pipeline import RTOL, rel_err

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
    assert np.all(e <= RTOL), e.max(0)
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


def test_adjoint_in_the_field_is_refused():
    import torch
    from paper_1811_11481_b300.binding import TpcError
    from synth.field import solenoid_field
    geo = synth.geometry()
    f = solenoid_field(eps=0.04)
    ev = synth.make_tiny(seed=65, n_tracks=50, central=True, field=f)
    tr = _tracker(geo, f)
    tr.set_calib()
    tr.load(tr.upload(ev))
    tr.find()
    tr.refit(save_for_backward=True)
    with pytest.raises(TpcError) as ei:
        tr.refit_backward(torch.ones(tr.n_tracks, device=tr.dev))
    assert ei.value.status == 5
