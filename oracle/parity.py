"""Parity of discrete outputs up to near-ties (TEST INFRASTRUCTURE ONLY).

Only the tests and ``__graft_entry__.smoke()`` use this module. It compares
the discrete outputs of another implementation of the method (given as
numpy arrays) with the oracle's, stage by stage on the same inputs, and
imports nothing of that implementation.

An implementation that rounds differently from the oracle's single-precision
mirror may take a decision the other way only where the decision is a
near-tie: where the float64 oracle's decision margin (oracle.cpp: the
distance the cluster positions would have to move to reverse a window, cut
or nearest-candidate decision, relative to the pad row's x, and the
distance of |sin(phi)| from its limit) is below NEAR_TIE. Those differences
are counted; the count must stay below MAX_RATE of the decisions taken.
Every other difference fails. Stages whose inputs are the other
implementation's outputs and whose work is integer (link cleaning, start
hits, selection) must agree exactly.
"""
from __future__ import annotations

import numpy as np

NEAR_TIE = 1e-5
MAX_RATE = 1e-4


class ParityError(AssertionError):
    pass


def _check(cond, msg):
    if not cond:
        raise ParityError(msg)


def links(o, up, dn, n_rows=152, hits=None):
    """Neighbour links (a4) against the oracle's single-precision links, of
    every cluster or of the sampled 'hits' (up, dn given for those). Returns
    the counts; raises ParityError on a difference that is not a near-tie or
    on too many near-ties."""
    up = np.asarray(up, np.int32)
    dn = np.asarray(dn, np.int32)
    hits = np.arange(o.n) if hits is None else np.asarray(hits, np.int64)
    ou, od = o.neighbours(32, hits=hits)
    d = np.nonzero((up != ou) | (dn != od))[0]
    diff = hits[d]
    rows = np.asarray(o.row, np.int64)[hits]
    decisions = int(np.count_nonzero((rows >= 1) & (rows + 1 < n_rows)))
    margins = np.empty(0)
    if diff.size:
        _, _, margins = o.neighbours(64, hits=diff, margin=True)
        bad = diff[margins >= NEAR_TIE]
        _check(bad.size == 0, f"links differ beyond near-ties at hits {bad[:10]} "
                              f"(margins {margins[margins >= NEAR_TIE][:10]})")
    _check(diff.size <= MAX_RATE * decisions,
           f"{diff.size} near-tie link differences in {decisions} decisions")
    return dict(near_ties=int(diff.size), decisions=decisions,
                max_margin=float(margins.max()) if margins.size else 0.0)


def cleaned(o, up, dn, upc, dnc):
    """Link cleaning (a5) of the given links: exact."""
    cu, cd = o.clean(up, dn)
    _check(np.array_equal(cu, upc) and np.array_equal(cd, dnc), "cleaned links differ")


def start_hits(o, upc, dnc, starts):
    """Start hits (a6) of the given cleaned links: exact (as a set)."""
    want = o.start_hits(upc, dnc)
    _check(np.array_equal(np.sort(np.asarray(starts, np.int64)), want), "start hits differ")


def tracklets(o, upc, starts, nh, hits, that, time_mode, sample=None):
    """Tracklets (a7) built by the oracle from the given cleaned links and
    start hits (in the given order) against the given ones: hit tables and
    counts equal up to near-ties; collision times (a continuous float64
    output of the single-precision seed fit) as close to the float64
    oracle's as the oracle's own single-precision mirror is. sample: indices
    of the start hits to check (all when None)."""
    starts = np.asarray(starts, np.int64)
    idx = np.arange(starts.size) if sample is None else np.asarray(sample, np.int64)
    st = starts[idx]
    t32 = o.tracklets(upc, st, 32)
    t64 = o.tracklets(upc, st, 64, margin=True)
    nh = np.asarray(nh)[idx]
    hits = np.asarray(hits)[idx]
    that = np.asarray(that)[idx]
    diff = np.nonzero((nh != t32["nh"]) | np.any(hits != t32["hits"], axis=1))[0]
    decisions = int(t64["decisions"].sum())
    m = t64["margin"][diff]
    bad = diff[m >= NEAR_TIE]
    _check(bad.size == 0, f"tracklets differ beyond near-ties: start hits {st[bad][:10]} "
                          f"(margins {m[m >= NEAR_TIE][:10]})")
    _check(diff.size <= MAX_RATE * decisions,
           f"{diff.size} near-tie tracklet differences in {decisions} decisions")
    t_err = None
    if time_mode:
        ok = (nh >= 0) & (t32["nh"] >= 0) & (t64["nh"] >= 0)
        e_got = np.abs(that[ok] - t64["that"][ok])
        e_32 = np.abs(t32["that"][ok] - t64["that"][ok])
        q = [50, 90, 99, 100]
        pg, p32 = np.percentile(e_got, q), np.percentile(e_32, q)
        _check(np.all(pg <= 3.0 * p32 + 1e-6),
               f"collision times: percentiles {q} of |t - t64| {pg} against the "
               f"single-precision mirror's {p32} (us)")
        t_err = dict(percentiles=q, got=pg.tolist(), mirror=p32.tolist())
    else:
        _check(np.all(that[nh >= 0] == 0.0), "collision time set in event mode")
    return dict(near_ties=int(diff.size), decisions=decisions, checked=int(idx.size),
                max_margin=float(m.max()) if m.size else 0.0, that=t_err)


def tracks(o, starts, nh, hits, that, track_start, cluster_idx, track_that, start_hit):
    """Selection (a8) of the given tracklets: exact. The given tracks are
    compared in the order of their start hits."""
    t = o.select(starts, dict(nh=np.asarray(nh, np.int32), hits=np.asarray(hits, np.int32),
                              that=np.asarray(that, np.float64)))
    got = canonical(track_start, cluster_idx, start_hit, track_that)
    want = canonical(t["track_start"], t["cluster_idx"], t["start_hit"], t["that"])
    _check(np.array_equal(got[0], want[0]), "tracks differ (start hits)")
    for a, b in zip(got[1], want[1]):
        _check(np.array_equal(a, b), "track clusters differ")
    _check(np.array_equal(got[2], want[2]), "track collision times differ")
    return int(got[0].size)


def canonical(track_start, cluster_idx, start_hit, that):
    """Tracks ordered by their start hit (input index)."""
    ts = np.asarray(track_start, np.int64)
    order = np.argsort(np.asarray(start_hit, np.int64), kind="stable")
    lists = [np.asarray(cluster_idx[ts[k]:ts[k + 1]], np.int64) for k in order]
    return np.asarray(start_hit, np.int64)[order], lists, np.asarray(that)[order]


def find(o, g, time_mode, n_rows=152, sample=None):
    """Every discrete stage of a find (a4-a8) stage by stage: g holds the
    other implementation's up, dn, upc, dnc, its tracklets (start_hit, nh,
    hits, that) and tracks (track_start, cluster_idx, t_coll, start_hit).
    Returns the near-tie counts."""
    lk = links(o, g["up"], g["dn"], n_rows)
    cleaned(o, g["up"], g["dn"], g["upc"], g["dnc"])
    tl = g["tracklets"]
    start_hits(o, g["upc"], g["dnc"], tl["start_hit"])
    tk = tracklets(o, g["upc"], tl["start_hit"], tl["nh"], tl["hits"], tl["that"], time_mode,
                   sample)
    n = tracks(o, tl["start_hit"], tl["nh"], tl["hits"], tl["that"], g["track_start"],
               g["cluster_idx"], g["t_coll"], g["start_hit"])
    return dict(links=lk, tracklets=tk, tracks=n)
