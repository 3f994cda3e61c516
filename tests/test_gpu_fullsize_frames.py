"""Parity at the full sizes of the benchmark's other workloads: the 50-collision
continuous-readout time frame (11.1M clusters, float64 times) and the batch
of 64 events of uneven size (9.5M clusters), each run in the launch shapes
the autotuner picks for it in bench.py (128-thread tracklet blocks with the
128-register cap).

As for the central event (test_gpu_fullsize.py), the oracle recomputes
sampled outputs one by one (links of sampled hits, tracklets of sampled start
hits, refits and gradients of sampled tracks) and the cheap whole-array steps
completely (link cleaning, start hits, selection, calibration transform),
each fed with the GPU's inputs of that step.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import parity
from paper_1811_11481_b300.config import default_params
from pipeline import RTOL, rel_err, tracker

pytestmark = pytest.mark.gpu

TUNING = dict(grid_tau=0.5, grid_ny_max=8, tracklet_block=128, tracklet_per_sm=0,
              tracklet_regs=96)


def _make(name):
    if name == "timeframe":
        return synth.make_timeframe(seed=2, n_coll=50)
    return synth.make_batched(seed=3)


@pytest.fixture(scope="module", params=["timeframe", "batched"])
def big(request):
    geo = synth.geometry()
    ev = _make(request.param)
    tr = tracker(geo)
    tr.set_calib()
    tr.set_tuning(**TUNING)
    cl = tr.upload(ev)
    tr.load(cl)
    out = tr.find()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    g["up"], g["dn"], g["upc"], g["dnc"] = [t.cpu().numpy() for t in tr.links()]
    g["tl"] = {k: v.cpu().numpy() for k, v in tr.tracklets().items()}
    yc, zc = tr.calibrated()
    g["yc"], g["zc"] = yc.cpu().numpy(), zc.cpu().numpy()
    o = oracle.Oracle(ev, geo, default_params(), synth.nominal_calib())
    return dict(name=request.param, ev=ev, tr=tr, g=g, o=o, rng=np.random.default_rng(98))


def test_size_is_the_benchmarks(big):
    ev, g = big["ev"], big["g"]
    assert ev.n > 9_000_000
    assert g["track_start"].size - 1 > 150_000
    if big["name"] == "timeframe":
        assert ev.mode == "time" and ev.n_events == 1
    else:
        assert ev.n_events == 64


def test_sampled_links(big):
    g, o, ev = big["g"], big["o"], big["ev"]
    hits = big["rng"].choice(ev.n, 4000, replace=False)
    r = parity.links(o, g["up"][hits], g["dn"][hits], hits=hits)
    print(f"sampled links: {r}")


def test_cleaning_and_start_hits_whole(big):
    g, o = big["g"], big["o"]
    upc, dnc = o.clean(g["up"], g["dn"])
    assert np.array_equal(upc, g["upc"]) and np.array_equal(dnc, g["dnc"])
    starts = o.start_hits(upc, dnc)
    assert np.array_equal(starts, np.sort(g["tl"]["start_hit"].astype(np.int64)))


def test_sampled_tracklets(big):
    g, o = big["g"], big["o"]
    tl = g["tl"]
    k = big["rng"].choice(tl["start_hit"].size, 300, replace=False)
    r = parity.tracklets(o, g["upc"], tl["start_hit"], tl["nh"], tl["hits"], tl["that"],
                         big["ev"].mode == "time", sample=k)
    print(f"sampled tracklets: {r}")


def test_selection_whole(big):
    g, o = big["g"], big["o"]
    tl = g["tl"]
    order = np.argsort(tl["start_hit"].astype(np.int64))
    sel = o.select(tl["start_hit"][order].astype(np.int64),
                   dict(nh=np.ascontiguousarray(tl["nh"][order]),
                        hits=np.ascontiguousarray(tl["hits"][order]),
                        that=np.ascontiguousarray(tl["that"][order])))
    ts = g["track_start"].astype(np.int64)
    got = {int(s): (g["cluster_idx"][ts[i]:ts[i + 1]], g["t_coll"][i])
           for i, s in enumerate(g["start_hit"])}
    rts = sel["track_start"].astype(np.int64)
    assert len(got) == rts.size - 1
    for i, s in enumerate(sel["start_hit"]):
        c, t = got[int(s)]
        assert np.array_equal(c, sel["cluster_idx"][rts[i]:rts[i + 1]])
        assert t == sel["that"][i]
    ci = g["cluster_idx"]
    assert np.unique(ci).size == ci.size


def test_calibration_whole(big):
    g, o = big["g"], big["o"]
    ts = g["track_start"].astype(np.int64)
    that = np.repeat(g["t_coll"], np.diff(ts))
    yc, zc = o.calibrate(g["cluster_idx"], that, prec=32)
    assert np.array_equal(g["yc"], yc.astype(np.float32))
    assert np.array_equal(g["zc"], zc.astype(np.float32))


def test_sampled_refits_and_gradients(big):
    import torch
    g, o, tr, ev = big["g"], big["o"], big["tr"], big["ev"]
    r = tr.refit(save_for_backward=True)
    got = {k: v.cpu().numpy() for k, v in r.items()}
    nt = got["chi2"].size
    ts = g["track_start"].astype(np.int64)
    k = np.sort(big["rng"].choice(nt, 400, replace=False))
    sts = np.concatenate([[0], np.cumsum(np.diff(ts)[k])]).astype(np.uint32)
    sci = np.concatenate([g["cluster_idx"][ts[i]:ts[i + 1]] for i in k])
    ref = o.refit(sts, sci, g["t_coll"][k], prec=64)
    ok = (got["status"][k] == 0) & (ref["status"] == 0)
    same = np.array([np.array_equal(got["rej"][ts[i]:ts[i + 1]], ref["rej"][sts[j]:sts[j + 1]])
                     for j, i in enumerate(k)])
    assert np.mean(got["status"][k] == ref["status"]) > 0.99 and np.mean(same[ok]) > 0.98
    m = ok & same
    e = rel_err(got["params"][k][m].astype(np.float64), ref["params"][m])
    assert np.all(e <= RTOL), e.max(0)
    # gradients of L = sum over 60 sampled tracks of chi2
    kk = k[np.nonzero(m)[0][:60]]
    w = torch.zeros(nt, device=tr.dev)
    w[torch.as_tensor(kk, device=tr.dev)] = 1.0
    gy, gz, gc = [t.cpu().numpy() for t in tr.refit_backward(w)]
    sts2 = np.concatenate([[0], np.cumsum(np.diff(ts)[kk])]).astype(np.uint32)
    sci2 = np.concatenate([g["cluster_idx"][ts[i]:ts[i + 1]] for i in kk])
    ref2 = o.refit(sts2, sci2, g["t_coll"][kk], prec=64)
    rej2 = np.concatenate([got["rej"][ts[i]:ts[i + 1]] for i in kk])
    ry, rz, rc = o.refit_grad(sts2, sci2, g["t_coll"][kk], ref2["seeds"], rej2, np.ones(kk.size))
    py = np.concatenate([gy[ts[i]:ts[i + 1]] for i in kk])
    pz = np.concatenate([gz[ts[i]:ts[i + 1]] for i in kk])
    assert np.linalg.norm(py - ry) / np.linalg.norm(ry) < 1e-3
    assert np.linalg.norm(pz - rz) / np.linalg.norm(rz) < 1e-3
    if ev.mode == "time":
        # v_drift and t0: sums whose terms partly cancel (the drift distance
        # is nearly linear along a track), compared with the sum of their
        # terms' magnitudes (pz is per drift time); the spline coefficients
        # (at zero distortion) by relative norm
        cal = synth.nominal_calib()
        that2 = np.concatenate([np.full(ts[i + 1] - ts[i], g["t_coll"][i]) for i in kk])
        drift = np.abs(ev.t[sci2.astype(np.int64)] - cal.t0 - that2)
        scales = (np.sum(np.abs(rz) * drift) / cal.vdrift, np.sum(np.abs(rz)))
        for q, scale in enumerate(scales):
            assert abs(gc[q] - rc[q]) <= 1e-3 * scale, (q, gc[q], rc[q], scale)
        err = np.linalg.norm(gc[2:] - rc[2:]) / np.linalg.norm(rc[2:])
        assert err < 1e-3, err
    rest = np.ones(gy.size, bool)
    for i in kk:
        rest[ts[i]:ts[i + 1]] = False
    assert np.all(gy[rest] == 0) and np.all(gz[rest] == 0)
