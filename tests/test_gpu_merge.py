"""Segment merging (Sec. 2, second phase) on the GPU against the oracle.

On the same segment states (the oracle's FP64 refit rounded to float32) the
links, their chi2 and the merged track set must equal the oracle's FP32
merge bit for bit. End to end (GPU finder, GPU refit, GPU merge) the
decisions are taken on states that agree with the oracle's FP64 refit
within the refit tolerance: at most 1% of the links may differ; merged
tracks that both sides form are refitted (across sector frames) within the
refit tolerance.
"""
import numpy as np
import pytest

import synth
from pipeline import RTOL, rel_err, tracker

pytestmark = pytest.mark.gpu


def _event(mode, seed=41, n_coll=3):
    return synth.make_tiny(seed=seed, n_tracks=300, central=True, mode=mode, noise_frac=0.1,
                           tf_start=1.0e6, n_coll=n_coll)


def _oracle(ev, geo):
    import oracle
    from paper_1811_11481_b300.config import default_params
    return oracle.Oracle(ev, geo, default_params(), synth.nominal_calib())


@pytest.fixture(scope="module")
def geo():
    return synth.geometry()


@pytest.mark.parametrize("mode", ["event", "time"])
def test_links_exact_on_the_same_states(geo, mode):
    import torch
    ev = _event(mode)
    o = _oracle(ev, geo)
    seg = o.find(prec=32)["tracks"]
    ts, ci, tt = seg["track_start"], seg["cluster_idx"], seg["that"]
    r = o.refit(ts, ci, tt, prec=64)
    st = dict(params=r["params"].astype(np.float32), cov=r["cov"].astype(np.float32),
              x=r["x"].astype(np.float32), status=r["status"].astype(np.int32))
    want = o.merge(ts, ci, tt, st["params"], st["cov"], st["x"], st["status"], prec=32)
    tr = tracker(geo)
    tr.set_calib()
    tr.load(tr.upload(ev))
    tr.set_tracks(torch.as_tensor(ts.astype(np.int32)), torch.as_tensor(ci.astype(np.int32)),
                  torch.as_tensor(tt), torch.as_tensor(seg["start_hit"].astype(np.int32)))
    got = tr.merge({k: torch.as_tensor(v) for k, v in st.items()})
    nx = got["next"].cpu().numpy()
    assert (want["next"] >= 0).sum() > 300
    np.testing.assert_array_equal(nx, want["next"])
    np.testing.assert_array_equal(got["link_chi2"].cpu().numpy(),
                                  want["link_chi2"].astype(np.float32))
    mt = {k: v.cpu().numpy() for k, v in got["tracks"].items()}
    np.testing.assert_array_equal(mt["track_start"], want["track_start"].astype(np.int32))
    np.testing.assert_array_equal(mt["cluster_idx"], want["cluster_idx"].astype(np.int32))
    np.testing.assert_array_equal(mt["t_coll"], want["that"])
    np.testing.assert_array_equal(mt["start_hit"], seg["start_hit"][want["head"]])
    assert tr.n_tracks == want["track_start"].size - 1


def test_batched_events_are_not_linked_across_events(geo):
    """Segments of different events (same sectors, same rows) stay apart."""
    import torch
    ev = synth.make_batched(seed=45, n_events=4, lo=150, hi=300)
    o = _oracle(ev, geo)
    seg = o.find(prec=32)["tracks"]
    ts, ci, tt = seg["track_start"], seg["cluster_idx"], seg["that"]
    r = o.refit(ts, ci, tt, prec=64)
    st = dict(params=r["params"].astype(np.float32), cov=r["cov"].astype(np.float32),
              x=r["x"].astype(np.float32), status=r["status"].astype(np.int32))
    want = o.merge(ts, ci, tt, st["params"], st["cov"], st["x"], st["status"], prec=32)
    tr = tracker(geo)
    tr.set_calib()
    tr.load(tr.upload(ev))
    tr.set_tracks(torch.as_tensor(ts.astype(np.int32)), torch.as_tensor(ci.astype(np.int32)),
                  torch.as_tensor(tt))
    nx = tr.merge({k: torch.as_tensor(v) for k, v in st.items()})["next"].cpu().numpy()
    np.testing.assert_array_equal(nx, want["next"])
    ev_of = ev.event[ci[ts[:-1].astype(np.int64)]]
    lk = np.nonzero(nx >= 0)[0]
    assert lk.size > 50 and np.all(ev_of[lk] == ev_of[nx[lk]])


@pytest.mark.parametrize("mode", ["event", "time"])
def test_find_refit_merge_refit_end_to_end(geo, mode):
    """GPU chain against the oracle chain; segments are matched by their
    start hit (the finders emit the same segments up to the consequences of
    counted near-ties, at most 1 %)."""
    import torch
    ev = _event(mode, seed=46, n_coll=2)
    o = _oracle(ev, geo)
    seg = o.find(prec=32)["tracks"]
    ts, ci, tt = seg["track_start"], seg["cluster_idx"], seg["that"]
    r = o.refit(ts, ci, tt, prec=64)
    want = o.merge(ts, ci, tt, r["params"], r["cov"], r["x"], r["status"], prec=32)
    tr = tracker(geo)
    tr.set_calib()
    tr.load(tr.upload(ev))
    g = {k: v.cpu().numpy() for k, v in tr.find().items()}
    rg = tr.refit()
    got = tr.merge(rg)
    gnx = got["next"].cpu().numpy()
    # the same segments, numbered differently
    o_of = {int(h): k for k, h in enumerate(seg["start_hit"])}
    perm = np.array([o_of.get(int(h), -1) for h in g["start_hit"]])
    assert np.sum(perm < 0) <= 0.01 * perm.size
    gl = {(perm[i], perm[j]) for i, j in enumerate(gnx) if j >= 0}
    ol = {(i, int(j)) for i, j in enumerate(want["next"]) if j >= 0}
    assert len(ol) > 300
    # link decisions taken on states that differ within the refit tolerance
    assert len(gl ^ ol) <= 0.01 * len(ol), (len(gl ^ ol), len(ol))
    # the merged tracks that both sides form
    rm = tr.refit()
    mt = {k: v.cpu().numpy() for k, v in got["tracks"].items()}
    ref_o = o.refit(want["track_start"], want["cluster_idx"], want["that"], prec=64)
    key_o = {tuple(want["cluster_idx"][want["track_start"][k]:want["track_start"][k + 1]]): k
             for k in range(want["track_start"].size - 1)}
    n_mt = mt["track_start"].size - 1
    n_same = sum(1 for k in range(n_mt)
                 if tuple(mt["cluster_idx"][mt["track_start"][k]:mt["track_start"][k + 1]]
                          .astype(np.uint32)) in key_o)
    assert n_same > 0.97 * n_mt * np.mean(ref_o["status"] == 0)
    # the refit of the CUDA path's merged set on its own inputs (its
    # collision times, compared separately with the tracklets): within the
    # tolerance of the FP64 oracle's refit of the same tracks
    ref = o.refit(mt["track_start"], mt["cluster_idx"], mt["t_coll"], prec=64)
    pg = rm["params"].cpu().numpy()[:n_mt]
    ok = (rm["status"].cpu().numpy()[:n_mt] == 0) & (ref["status"] == 0)
    e = rel_err(pg[ok].astype(np.float64), ref["params"][ok])
    assert np.all(e <= RTOL), e.max(0)


def test_merge_of_an_empty_set_and_of_failed_segments(geo):
    import torch
    ev = _event("event", seed=47, n_coll=1)
    tr = tracker(geo)
    tr.set_calib()
    tr.load(tr.upload(ev))
    z = lambda *s: torch.zeros(*s)
    tr.set_tracks(torch.zeros(1, dtype=torch.int32), torch.zeros(0, dtype=torch.int32),
                  torch.zeros(0, dtype=torch.float64))
    out = tr.merge(dict(params=z(0, 5), cov=z(0, 15), x=z(0), status=z(0).int()))
    assert tr.n_tracks == 0 and out["next"].numel() == 0
    # every segment failed: nothing is linked, the set is unchanged
    g = {k: v.cpu().numpy() for k, v in tr.find().items()}
    n = tr.n_tracks
    rg = tr.refit()
    rg["status"][:] = 1
    out = tr.merge(rg)
    assert tr.n_tracks == n and np.all(out["next"].cpu().numpy() == -1)
    mt = {k: v.cpu().numpy() for k, v in out["tracks"].items()}
    np.testing.assert_array_equal(mt["track_start"], g["track_start"])
    np.testing.assert_array_equal(mt["cluster_idx"], g["cluster_idx"])


def test_refined_time_exact_on_the_same_states(geo):
    """Collision times refined from the same float32 states (some with a z
    offset, so that the shift back inside the drift volume acts) equal the
    oracle's FP32 refinement bit for bit."""
    import torch
    ev = _event("time", seed=48, n_coll=2)
    ts, ci, tc, _ = synth.truth_tracks(ev, 40, merged=True)
    o = _oracle(ev, geo)
    r = o.refit(ts, ci, tc, prec=64)
    p = r["params"].copy()
    rng = np.random.default_rng(3)
    p[:, 1] += rng.choice([0.0, 0.0, -120.0, 120.0], size=p.shape[0])
    st = dict(params=p.astype(np.float32), x=r["x"].astype(np.float32),
              status=r["status"].astype(np.int32))
    want = o.refine_time(ts, ci, tc, st["params"], st["x"], st["status"], prec=32)
    assert np.sum(want != tc) > 100
    tr = tracker(geo)
    tr.set_calib()
    tr.load(tr.upload(ev))
    tr.set_tracks(torch.as_tensor(ts.astype(np.int32)), torch.as_tensor(ci.astype(np.int32)),
                  torch.as_tensor(tc))
    got = tr.refine_time({k: torch.as_tensor(v) for k, v in st.items()}).cpu().numpy()
    np.testing.assert_array_equal(got, want)
    # and the track set now carries them
    np.testing.assert_array_equal(tr.tracks()["t_coll"].cpu().numpy(), want)


def test_full_chain_with_time_refinement(geo):
    """Time frame: find, refit, merge, refit, refine the collision times,
    refit. The GPU chain against the oracle chain on the merged tracks both
    form: times within 2 ns (the refit tolerance carried to the closest
    approach: 1e-4 on tan(lambda) over at most 250 cm, plus 1e-4 cm on z,
    over v_drift), final parameters within the refit tolerance."""
    ev = _event("time", seed=49, n_coll=3)
    o = _oracle(ev, geo)
    seg = o.find(prec=32)["tracks"]
    ts, ci, tt = seg["track_start"], seg["cluster_idx"], seg["that"]
    r = o.refit(ts, ci, tt, prec=64)
    m = o.merge(ts, ci, tt, r["params"], r["cov"], r["x"], r["status"], prec=32)
    r2 = o.refit(m["track_start"], m["cluster_idx"], m["that"], prec=64)
    th = o.refine_time(m["track_start"], m["cluster_idx"], m["that"], r2["params"], r2["x"],
                       r2["status"], prec=64)
    r3 = o.refit(m["track_start"], m["cluster_idx"], th, prec=64)
    tr = tracker(geo)
    tr.set_calib()
    tr.load(tr.upload(ev))
    tr.find()
    tr.merge(tr.refit())
    gth = tr.refine_time(tr.refit()).cpu().numpy()
    g3 = tr.refit()
    mt = {k: v.cpu().numpy() for k, v in tr.tracks().items()}
    key_o = {tuple(m["cluster_idx"][m["track_start"][k]:m["track_start"][k + 1]]): k
             for k in range(m["track_start"].size - 1)}
    pg, sg = g3["params"].cpu().numpy(), g3["status"].cpu().numpy()
    dt, errs = [], []
    for k in range(mt["track_start"].size - 1):
        c = tuple(mt["cluster_idx"][mt["track_start"][k]:mt["track_start"][k + 1]].astype(np.uint32))
        ko = key_o.get(c)
        if ko is None or sg[k] != 0 or r3["status"][ko] != 0 or r2["status"][ko] != 0:
            continue
        dt.append(abs(gth[k] - th[ko]))
        errs.append(rel_err(pg[k].astype(np.float64), r3["params"][ko]))
    assert len(dt) > 300
    assert max(dt) < 2e-3, max(dt)
    assert np.all(np.array(errs) <= RTOL), np.array(errs).max(0)


def _chain_buffers(torch, dev, n):
    cap = n // 10 + 1
    f = lambda *s: torch.zeros(*s, device=dev)
    i32 = lambda *s: torch.zeros(*s, dtype=torch.int32, device=dev)
    mk = lambda: dict(params=f(cap, 5), cov=f(cap, 15), x=f(cap), chi2=f(cap), ndf=i32(cap),
                      status=i32(cap), rej=torch.zeros(n + 1, dtype=torch.uint8, device=dev))
    return dict(seg=mk(), r1=mk(), r2=mk(), next=i32(cap), lchi=f(cap),
                t=torch.zeros(cap, dtype=torch.float64, device=dev))


def _chain(tr, cl, b):
    """find, refit the segments, merge (asynchronous), refit, refine the
    collision times, refit: only asynchronous calls."""
    import ctypes as C
    P = lambda t: C.c_void_p(t.data_ptr())
    L, h = tr.L, tr.h
    fit = lambda o: L.tpc_refit(h, 0, P(o["params"]), P(o["cov"]), P(o["x"]), P(o["chi2"]),
                                P(o["ndf"]), P(o["status"]), P(o["rej"]))
    tr.load(cl)
    assert L.tpc_find_tracks_async(h) == 0
    assert fit(b["seg"]) == 0
    s = b["seg"]
    assert L.tpc_merge_tracks_async(h, P(s["params"]), P(s["cov"]), P(s["x"]), P(s["status"]),
                                    P(b["next"]), P(b["lchi"])) == 0
    assert fit(b["r1"]) == 0
    r = b["r1"]
    assert L.tpc_refine_time(h, P(r["params"]), P(r["x"]), P(r["status"]), P(b["t"])) == 0
    assert fit(b["r2"]) == 0


def test_async_merge_and_captured_chain_equal_the_synchronous_merge(geo):
    """The asynchronous merge gives the synchronous merge's set bit for bit,
    and the whole chain replays from a CUDA graph with the same outputs."""
    import torch
    from paper_1811_11481_b300.binding import Tracker
    from paper_1811_11481_b300.config import default_params
    ev = _event("time", seed=50, n_coll=2)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        tr = Tracker(geo, default_params(), stream=stream)
        tr.set_calib()
        cl = tr.upload(ev)
        # synchronous reference
        tr.load(cl)
        tr.find()
        seg = tr.refit()
        m = tr.merge(seg)
        ref = {k: v.cpu().numpy() for k, v in tr.tracks().items()}
        ref_next = m["next"].cpu().numpy()
        nseg = ref_next.size
        b = _chain_buffers(torch, tr.dev, ev.n)
        # the asynchronous merge alone
        tr.load(cl)
        tr.find()
        seg2 = tr.refit()
        tr.merge_async(seg2, b["next"], b["lchi"])
        got = {k: v.cpu().numpy() for k, v in tr.tracks().items()}
        for k in ref:
            np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
        np.testing.assert_array_equal(b["next"][:nseg].cpu().numpy(), ref_next)
        np.testing.assert_array_equal(b["lchi"][:nseg].cpu().numpy(),
                                      m["link_chi2"].cpu().numpy())
        # the chain, directly (allocates every buffer), then from a graph
        _chain(tr, cl, b)
        nt, na, _ = tr.counts()
        direct = {k: v.clone() for k, v in b["r2"].items()}
        t_direct = b["t"][:nt].clone()
        for o in (b["r1"], b["r2"]):
            for v in o.values():
                if v.dtype.is_floating_point:
                    v.fill_(float("nan"))
        stream.synchronize()
        tr.graph_begin()
        _chain(tr, cl, b)                     # recorded, not run
        tr.graph_end()
        tr.graph_launch()
        stream.synchronize()
        assert tr.counts()[:2] == (nt, na)
    for k in ("params", "cov", "chi2", "ndf", "status"):
        assert torch.equal(b["r2"][k][:nt], direct[k][:nt]), k
    assert torch.equal(b["t"][:nt], t_direct)
    assert nt < nseg and nt > 0
