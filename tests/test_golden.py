"""Stored fixtures under tests/golden/.

paper_facts.txt  numbers the paper states (cited there): the header,
                 geometry and defaults must agree with them.
tiny_event_oracle.json  the oracle's links, tracks and refit on one small
                 seeded event, written by tests/golden/make_golden.py (which
                 calls only the oracle): the oracle must still reproduce it
                 (CPU), and the CUDA path must match it (GPU) -- discrete
                 outputs exactly, refit parameters within the parity
                 tolerance.
"""
import json
import os
import re
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")
ROOT = os.path.dirname(HERE)
sys.path.insert(0, GOLD)
import make_golden  # noqa: E402


def _facts():
    out = {}
    for line in open(os.path.join(GOLD, "paper_facts.txt")):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (s.strip() for s in line.split("="))
            out[k] = int(v)
    return out


def _golden():
    with open(os.path.join(GOLD, "tiny_event_oracle.json")) as fh:
        return json.load(fh)


def test_paper_facts_fix_header_geometry_and_defaults():
    import synth
    from paper_1811_11481_b300.config import default_params
    f = _facts()
    hdr = open(os.path.join(ROOT, "include", "tpc.h")).read()
    assert int(re.search(r"#define TPC_N_SECTORS (\d+)", hdr).group(1)) == f["n_sectors"]
    geo = synth.geometry()
    assert geo.n_sectors == f["n_sectors"]
    assert geo.row_x.size == f["n_rows"]
    assert int(re.search(r"#define TPC_MAX_ROWS (\d+)", hdr).group(1)) >= f["n_rows"]
    p = default_params()
    assert p["seed_max_hits"] == f["segment_hits_max"]


def test_seed_segments_have_the_papers_length():
    # the fitted segment of a tracklet is its chain of links from the start
    # hit, at most seed_max_hits long and at least 3 hits (start-hit rule):
    # on the golden event most segments have 4 to 10 hits
    import oracle
    import synth
    from paper_1811_11481_b300.config import default_params
    f = _facts()
    p = default_params()
    o = oracle.Oracle(make_golden.event(), synth.geometry(), p, synth.nominal_calib())
    r = o.find(32)
    upc = r["upc"]
    lens = []
    for h in r["starts"]:
        n, x = 1, int(h)
        while upc[x] >= 0 and n < p["seed_max_hits"]:
            x = int(upc[x])
            n += 1
        lens.append(n)
    lens = np.array(lens)
    assert lens.size > 10
    assert lens.min() >= 3 and lens.max() <= f["segment_hits_max"]
    assert np.mean((lens >= f["segment_hits_min"]) & (lens <= f["segment_hits_max"])) > 0.5


def test_oracle_reproduces_golden():
    g = _golden()
    d = make_golden.compute()
    assert d["recipe"] == g["recipe"] and d["n_clusters"] == g["n_clusters"]
    for k in ("up", "dn", "track_start", "cluster_idx", "start_hit", "ndf", "status"):
        assert d[k] == g[k], k
    for k in ("params", "chi2"):
        a, b = np.asarray(d[k]), np.asarray(g[k])
        assert np.allclose(a, b, rtol=1e-12, atol=1e-12), k
    assert len(g["track_start"]) - 1 >= 10


@pytest.mark.gpu
def test_cuda_path_matches_golden():
    import synth
    import torch
    from paper_1811_11481_b300.binding import Tracker
    from paper_1811_11481_b300.config import default_params
    g = _golden()
    ev = make_golden.event()
    assert ev.n == g["n_clusters"]
    tr = Tracker(synth.geometry(), default_params())
    tr.set_calib()
    tr.load(tr.upload(ev))
    out = tr.find()
    up, dn, _, _ = [t.cpu().numpy() for t in tr.links()]
    # links equal the stored ones except near-ties of the float64 oracle
    import oracle
    from oracle import parity
    diff = np.nonzero((up != np.asarray(g["up"])) | (dn != np.asarray(g["dn"])))[0]
    if diff.size:
        o = oracle.Oracle(ev, synth.geometry(), default_params(), synth.nominal_calib())
        _, _, m = o.neighbours(64, hits=diff, margin=True)
        assert np.all(m < parity.NEAR_TIE), (diff, m)
    ts = out["track_start"].cpu().numpy()
    ci = out["cluster_idx"].cpu().numpy()
    sh = out["start_hit"].cpu().numpy()
    got = {int(s): ci[ts[k]:ts[k + 1]].tolist() for k, s in enumerate(sh)}
    gts, gci = g["track_start"], g["cluster_idx"]
    want = {int(s): gci[gts[k]:gts[k + 1]] for k, s in enumerate(g["start_hit"])}
    differ = sum(1 for k in set(got) | set(want) if got.get(k) != want.get(k))
    print(f"golden event: {diff.size} near-tie links, {differ} of {len(want)} tracks differ")
    assert differ <= 0.01 * len(want)
    sh = np.array([s for s in sh if got[int(s)] == want.get(int(s))], np.int64)
    keep = {int(s) for s in sh}
    r = tr.refit()
    torch.cuda.synchronize()
    # golden tracks (those found alike) in the CUDA path's order
    allsh = out["start_hit"].cpu().numpy()
    rows = np.array([k for k, s in enumerate(allsh) if int(s) in keep], np.int64)
    pos = {int(s): k for k, s in enumerate(g["start_hit"])}
    order = np.array([pos[int(s)] for s in allsh[rows]])
    ref = np.asarray(g["params"])[order]
    st = r["status"].cpu().numpy()[rows]
    ok = (st == 0) & (np.asarray(g["status"])[order] == 0)
    assert ok.sum() >= 10
    p = r["params"].cpu().numpy()[rows][ok]
    e = np.abs(p - ref[ok]) / np.maximum(np.abs(ref[ok]), np.array([1, 1, 0.1, 0.1, 0.1]))
    assert np.all(e <= np.array([1e-4, 1e-4, 1e-4, 1e-4, 1e-3])), e.max(0)
