"""The near-tie parity checker (oracle/parity.py) and the oracle's decision
margins, on the CPU.

The margin of a neighbour-finder decision is pinned by moving the three
clusters of a constructed triplet along the margin's direction: the link
must hold just short of the margin and flip just beyond it. The checker must
accept the oracle's own outputs, count a planted difference at a near-tie,
and reject planted differences at clear decisions and in the exact stages.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import parity


class _Mini:
    """Hand-built clusters in one sector (event mode)."""

    def __init__(self, rows, ys, zs):
        self.mode = "event"
        self.row = np.asarray(rows, np.uint8)
        self.y = np.asarray(ys, np.float32)
        self.z = np.asarray(zs, np.float32)
        n = self.y.size
        self.sector = np.zeros(n, np.uint8)
        self.flags = np.zeros(n, np.uint8)
        self.event = np.zeros(n, np.uint32)
        self.n_events = 1
        self.tf_start = 0.0
        self.t = None


def _link(geo, params, ys):
    ev = _Mini([50, 51, 49], ys, [0.0, 0.0, 0.0])
    o = oracle.Oracle(ev, geo, params, synth.nominal_calib())
    up, dn, m = o.neighbours(64, margin=True)
    return up[0], dn[0], m[0]


def test_link_margin_is_the_distance_to_the_deviation_cut(geo, params):
    """Hit at row 50, up candidate on its line, down candidate a bit inside
    the deviation cut: the margin times x is the distance the three points
    must move together (steepest direction) to leave the cut."""
    x = geo.row_x.astype(np.float64)
    dmax = float(np.float32(params["nb_dmax"]))
    a = np.sqrt(dmax) - 2e-3
    up, dn, m = _link(geo, params, [0.0, 0.0, a])
    assert (up, dn) == (1, 2)
    f = float(np.float32(x[50] - x[49])) / float(np.float32(x[51] - x[50]))
    kf = 1.0 + f * f + (1.0 + f) ** 2
    unit = np.array([-(1.0 + f), f, 1.0]) / np.sqrt(kf)      # (h, u, d) in y
    delta = m * float(np.float32(x[50]))
    assert 0.5e-3 < delta < 2e-3
    for t, linked in ((0.98 * delta, True), (1.02 * delta, False)):
        ys = np.array([0.0, 0.0, a]) + t * unit
        u2, d2, _ = _link(geo, params, ys.astype(np.float32).tolist())
        assert ((u2, d2) == (1, 2)) == linked, (t, u2, d2)


def test_exact_tie_has_zero_margin(geo, params):
    # mirror-symmetric candidates: two pairs with the same deviation
    ev = _Mini([60, 61, 61, 59, 59], [0.0, 0.1, -0.1, 0.1, -0.1], [0.0] * 5)
    o = oracle.Oracle(ev, geo, params, synth.nominal_calib())
    _, _, m = o.neighbours(64, margin=True)
    assert m[0] == 0.0


@pytest.fixture(scope="module")
def small(geo, params):
    ev = synth.make_tiny(seed=31, n_tracks=600, central=True, noise_frac=0.1)
    o = oracle.Oracle(ev, geo, params, synth.nominal_calib())
    up, dn = o.neighbours(32)
    upc, dnc = o.clean(up, dn)
    starts = o.start_hits(upc, dnc)
    tl = o.tracklets(upc, starts, 32)
    tr = o.select(starts, tl)
    g = dict(up=up, dn=dn, upc=upc, dnc=dnc,
             tracklets=dict(start_hit=starts, nh=tl["nh"], hits=tl["hits"], that=tl["that"]),
             track_start=tr["track_start"], cluster_idx=tr["cluster_idx"], t_coll=tr["that"],
             start_hit=tr["start_hit"])
    return o, g


def _copy(g):
    return {k: ({kk: vv.copy() for kk, vv in v.items()} if isinstance(v, dict) else v.copy())
            for k, v in g.items()}


def test_checker_accepts_the_oracles_own_outputs(small):
    o, g = small
    r = parity.find(o, g, time_mode=False)
    assert r["links"]["near_ties"] == 0 and r["tracklets"]["near_ties"] == 0
    assert r["tracks"] > 100


def test_checker_counts_a_near_tie_link_and_rejects_a_clear_one(small):
    o, g = small
    _, _, m = o.neighbours(64, margin=True)
    linked = np.nonzero(g["up"] >= 0)[0]
    near = linked[m[linked] < parity.NEAR_TIE]
    clear = linked[m[linked] > 100 * parity.NEAR_TIE]
    assert near.size > 0 and clear.size > 0
    h = _copy(g)
    h["up"][near[0]] = -1
    h["dn"][near[0]] = -1
    r = parity.links(o, h["up"], h["dn"])
    assert r["near_ties"] == 1 and r["max_margin"] < parity.NEAR_TIE
    h = _copy(g)
    h["up"][clear[0]] = -1
    with pytest.raises(parity.ParityError):
        parity.links(o, h["up"], h["dn"])


def test_checker_rejects_a_changed_tracklet_and_changed_tracks(small):
    o, g = small
    tl = g["tracklets"]
    t64 = o.tracklets(g["upc"], tl["start_hit"], 64, margin=True)
    k = int(np.nonzero((tl["nh"] > 20) & (t64["margin"] > 100 * parity.NEAR_TIE))[0][0])
    h = _copy(g)
    r = int(np.nonzero(h["tracklets"]["hits"][k] >= 0)[0][5])
    h["tracklets"]["hits"][k, r] = -1
    h["tracklets"]["nh"][k] -= 1
    with pytest.raises(parity.ParityError):
        parity.tracklets(o, h["upc"], h["tracklets"]["start_hit"], h["tracklets"]["nh"],
                         h["tracklets"]["hits"], h["tracklets"]["that"], False)
    # a cluster moved from one track to the next: the selection differs
    h = _copy(g)
    ts = h["track_start"].astype(np.int64)
    h["cluster_idx"][ts[1]] = h["cluster_idx"][ts[1] + 1]
    with pytest.raises(parity.ParityError):
        parity.tracks(o, tl["start_hit"], tl["nh"], tl["hits"], tl["that"], h["track_start"],
                      h["cluster_idx"], h["t_coll"], h["start_hit"])
    # cleaning and start hits are exact
    h = _copy(g)
    h["upc"][np.nonzero(h["upc"] >= 0)[0][0]] = -1
    with pytest.raises(parity.ParityError):
        parity.cleaned(o, h["up"], h["dn"], h["upc"], h["dnc"])
    with pytest.raises(parity.ParityError):
        parity.start_hits(o, g["upc"], g["dnc"], tl["start_hit"][1:])
