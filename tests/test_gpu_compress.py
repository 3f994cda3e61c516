"""Track-model compression (Sec. 5) on the GPU against the oracle: residuals
and decoded clusters bit for bit (integer residuals decided in single
precision) on found tracks, on tracks merged across sectors and with native
pad input; the oracle's decoder reproduces the GPU's decoded clusters from
the GPU's residuals alone."""
import numpy as np
import pytest

import oracle
import synth
from paper_1811_11481_b300.config import default_params
from pipeline import tracker

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode,pads", [("event", False), ("time", False), ("time", True)])
def test_residuals_exact(mode, pads):
    import torch
    geo = synth.geometry()
    ev = synth.make_tiny(seed=57, n_tracks=300, central=True, mode=mode, tf_start=1.0e6,
                         n_coll=2, noise_frac=0.1)
    tr = tracker(geo)
    tr.set_calib()
    tr.load(tr.upload(ev, pads=pads))
    g = {k: v.cpu().numpy() for k, v in tr.find().items()}
    o = oracle.Oracle(ev, geo, default_params(), synth.nominal_calib(), pads=pads)
    sets = [(g["track_start"], g["cluster_idx"], g["t_coll"])]
    ts, ci, tc, _ = synth.truth_tracks(ev, 40, merged=True)
    sets.append((ts, ci, tc))
    for k, (ts, ci, tt) in enumerate(sets):
        if k == 1:
            tr.set_tracks(torch.as_tensor(ts.astype(np.int32)),
                          torch.as_tensor(ci.astype(np.int32)), torch.as_tensor(tt))
        got = {kk: v.cpu().numpy() for kk, v in tr.compress(qy=0.01, qz=0.013).items()}
        want = o.compress(ts, ci, tt, qy=0.01, qz=0.013)
        assert ci.size > 1000
        for kk in ("ry", "rz", "dy", "dz"):
            np.testing.assert_array_equal(got[kk], want[kk], err_msg=kk)
        dy, dz = o.decompress(ts, ci, got["ry"], got["rz"], qy=0.01, qz=0.013)
        np.testing.assert_array_equal(dy, got["dy"])
        np.testing.assert_array_equal(dz, got["dz"])


def test_invalid_steps_are_refused():
    import torch
    from paper_1811_11481_b300.binding import TpcError
    geo = synth.geometry()
    tr = tracker(geo)
    tr.set_calib()
    tr.load(tr.upload(synth.make_tiny(seed=58, n_tracks=20)))
    tr.find()
    for q in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(TpcError) as ei:
            tr.compress(qy=q)
        assert ei.value.status == 1
