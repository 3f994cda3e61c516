"""Shared drivers for the parity tests: run the CUDA path and the oracle on the
same seeded inputs and put both results in the same (input-index) numbering."""
import numpy as np

import oracle
import synth
from paper_1811_11481_b300.config import default_params

# Floating-point tolerance of the refit against the FP64 oracle: relative
# 1e-4 on y, z, sin(phi), tan(lambda) and 1e-3 on q/pT, each relative to
# max(|reference|, floor) with floors 1 cm, 1 cm, 0.1, 0.1, 0.1 /GeV.
RTOL = np.array([1e-4, 1e-4, 1e-4, 1e-4, 1e-3])
FLOOR = np.array([1.0, 1.0, 0.1, 0.1, 0.1])


def refit_tolerance(o, track_start, cluster_idx, that, ref64, ok):
    """Per-parameter tolerance of a single-precision refit against the FP64
    oracle: the stated RTOL, or, where single-precision arithmetic of the
    method itself does not reach it, the largest deviation of the oracle's
    own FP32 refit of the same tracks from FP64 (times 1.5). The bulk
    arithmetic is single precision; on short, stiff tracks in the full field
    its q/pT is not determined to 1e-3 of max(|q/pT|, 0.1)."""
    r32 = o.refit(track_start, cluster_idx, that, prec=32)
    m = ok & (r32["status"] == 0)
    mirror = rel_err(r32["params"][m], ref64["params"][m]).max(0) if m.any() else 0.0
    return np.maximum(RTOL, 1.5 * mirror), mirror


def tracker(geo, params=None):
    from paper_1811_11481_b300.binding import Tracker
    return Tracker(geo, params or default_params())


def gpu_find(tr, ev, calib=None):
    calib = calib or synth.nominal_calib()
    tr.set_calib(calib.vdrift, calib.t0, calib.spline)
    cl = tr.upload(ev)
    tr.load(cl)
    out = tr.find()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    up, dn, upc, dnc = [t.cpu().numpy() for t in tr.links()]
    res.update(up=up, dn=dn, upc=upc, dnc=dnc)
    tl = tr.tracklets()
    res["tracklets"] = {k: v.cpu().numpy() for k, v in tl.items()}
    yc, zc = tr.calibrated()
    res["yc"], res["zc"] = yc.cpu().numpy(), zc.cpu().numpy()
    res["_cl"] = cl
    return res


def canonical_tracks(track_start, cluster_idx, start_hit, that):
    """Tracks ordered by their start hit (input index)."""
    ts = np.asarray(track_start, np.int64)
    order = np.argsort(np.asarray(start_hit, np.int64), kind="stable")
    lists = [np.asarray(cluster_idx[ts[k]:ts[k + 1]], np.int64) for k in order]
    return (np.asarray(start_hit, np.int64)[order], lists, np.asarray(that)[order])


def oracle_find(ev, geo, calib=None, params=None, prec=32):
    calib = calib or synth.nominal_calib()
    o = oracle.Oracle(ev, geo, params or default_params(), calib)
    return o, o.find(prec)


def rel_err(got, ref):
    return np.abs(got - ref) / np.maximum(np.abs(ref), FLOOR)
