"""Many small random cases through the CUDA path against the oracle: every
discrete output of the finder stage by stage (links and tracklets up to
counted near-ties, cleaned links, start hits and tracks exactly) and the
merge on the oracle's states exactly, whatever the mode, the sectors, the
noise, the batching and the cluster flags."""
import numpy as np
import pytest

import oracle
import synth
from oracle import parity
from paper_1811_11481_b300.config import default_params
from pipeline import tracker

pytestmark = pytest.mark.gpu


def _case(seed):
    rng = np.random.default_rng(1000 + seed)
    mode = "time" if rng.random() < 0.5 else "event"
    kind = rng.integers(0, 3)
    if kind == 0:
        ev = synth.make_tiny(seed=seed, n_tracks=int(rng.integers(20, 400)), central=True,
                             mode=mode, tf_start=1.0e6, n_coll=int(rng.integers(1, 4)),
                             noise_frac=float(rng.uniform(0.0, 0.4)))
    elif kind == 1:
        secs = tuple(int(s) for s in rng.choice(36, size=int(rng.integers(1, 5)), replace=False))
        ev = synth.make_tiny(seed=seed, n_tracks=int(rng.integers(10, 200)), sectors=secs,
                             mode=mode, tf_start=1.0e6, noise_frac=float(rng.uniform(0.0, 0.5)))
    else:
        ev = synth.make_batched(seed=seed, n_events=int(rng.integers(2, 6)), lo=5, hi=200)
    pick = rng.random(ev.n) < 0.1
    ev.flags[pick] = rng.integers(1, 32, size=int(pick.sum())).astype(np.uint8)
    return ev


@pytest.mark.parametrize("seed", range(12))
def test_random_cases(seed):
    import torch
    geo = synth.geometry()
    ev = _case(seed)
    tr = tracker(geo)
    tr.set_calib()
    tr.load(tr.upload(ev))
    g = {k: v.cpu().numpy() for k, v in tr.find().items()}
    g["up"], g["dn"], g["upc"], g["dnc"] = [t.cpu().numpy() for t in tr.links()]
    g["tracklets"] = {k: v.cpu().numpy() for k, v in tr.tracklets().items()}
    o = oracle.Oracle(ev, geo, default_params(), synth.nominal_calib())
    print(f"case {seed}: {parity.find(o, g, ev.mode == 'time')}")
    ts = g["track_start"].astype(np.int64)
    if ts.size < 3:
        return
    # merge on the oracle's states of these segments
    r = o.refit(g["track_start"], g["cluster_idx"], g["t_coll"], prec=64)
    st = dict(params=r["params"].astype(np.float32), cov=r["cov"].astype(np.float32),
              x=r["x"].astype(np.float32), status=r["status"].astype(np.int32))
    m = o.merge(g["track_start"], g["cluster_idx"], g["t_coll"], st["params"], st["cov"],
                st["x"], st["status"], prec=32)
    nx = tr.merge({k: torch.as_tensor(v) for k, v in st.items()})["next"].cpu().numpy()
    np.testing.assert_array_equal(nx, m["next"])
