"""The search grid at the limits of one pad-row bucket (one event, sector and
row): a row holding more clusters than the common sort tile (4096) goes
through the large-tile sort, and its bins (16-bit offsets from the row's
bucket start) must give the oracle's discrete outputs; a row holding more
than the large tile (16384) is reported as a capacity error by the next
synchronising call, and the context stays usable."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from oracle import parity
from paper_1811_11481_b300.config import default_params
from pipeline import tracker

pytestmark = pytest.mark.gpu


def _crowded(n_extra, seed, row=70, sector=3):
    """A small event-mode event of one sector with n_extra uniform noise
    clusters added to one pad row (inside the sector's acceptance, on its
    side of the central electrode)."""
    ev = synth.make_tiny(seed=seed, n_tracks=60, sectors=(sector,), noise_frac=0.1)
    geo = synth.geometry()
    rng = np.random.default_rng(seed)
    half = float(geo.row_x[row]) * float(geo.tan_half)
    y = rng.uniform(-half, half, n_extra).astype(np.float32)
    side = 1.0 if sector < 18 else -1.0
    z = (side * rng.uniform(2.0, 245.0, n_extra)).astype(np.float32)
    nan = np.full(n_extra, np.nan)

    def cat(a, b):
        return np.concatenate([a, b.astype(a.dtype)])
    return dataclasses.replace(
        ev, y=cat(ev.y, y), z=cat(ev.z, z), row=cat(ev.row, np.full(n_extra, row)),
        sector=cat(ev.sector, np.full(n_extra, sector)), flags=cat(ev.flags, np.zeros(n_extra)),
        event=cat(ev.event, np.zeros(n_extra)), label=cat(ev.label, np.full(n_extra, -1)),
        segment=cat(ev.segment, np.full(n_extra, -1)), y_true=cat(ev.y_true, nan),
        z_true=cat(ev.z_true, nan), s_true=cat(ev.s_true, nan), tl_true=cat(ev.tl_true, nan),
        q_true=cat(ev.q_true, nan))


@pytest.mark.parametrize("grid_tau", [0.25, 1.0])
def test_crowded_row_through_the_large_tile_sort(grid_tau):
    """6,000 clusters in one row: links, cleaned links, start hits,
    tracklets and tracks as the oracle's (stage by stage, up to counted
    near-ties)."""
    geo = synth.geometry()
    ev = _crowded(6000, seed=91)
    tr = tracker(geo)
    tr.set_calib()
    tr.set_tuning(grid_tau=grid_tau, grid_ny_max=16)
    tr.load(tr.upload(ev))
    g = {k: v.cpu().numpy() for k, v in tr.find().items()}
    g["up"], g["dn"], g["upc"], g["dnc"] = [x.cpu().numpy() for x in tr.links()]
    g["tracklets"] = {k: v.cpu().numpy() for k, v in tr.tracklets().items()}
    o = oracle.Oracle(ev, geo, default_params(), synth.nominal_calib())
    print(f"crowded row, {grid_tau} per bin: {parity.find(o, g, False)}")
    assert g["track_start"].size > 1


def test_row_beyond_the_large_tile_is_a_capacity_error():
    from paper_1811_11481_b300.binding import TpcError
    geo = synth.geometry()
    tr = tracker(geo)
    tr.set_calib()
    tr.load(tr.upload(_crowded(17000, seed=92)))
    with pytest.raises(TpcError) as ei:
        tr.find()
    assert ei.value.status == 2  # TPC_ERR_CAPACITY
    # the context stays usable
    ev = synth.make_tiny(seed=93, n_tracks=40)
    tr.load(tr.upload(ev))
    tr.find()
    assert tr.n_tracks > 0
