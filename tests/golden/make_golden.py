"""Write tests/golden/tiny_event_oracle.json: the oracle's result on one
small seeded event (test infrastructure; calls only the oracle and the
seeded input generator).

The event: synth.make_tiny(seed=3, n_tracks=24, sectors=(0, 21),
noise_frac=0.05), event mode, nominal calibration, default cut values.
Stored: the neighbour links and the tracks of the FP32-mirror finder
(Sec. 2, phase 1), and the FP64 refit of every track (Sec. 3, three-pass
Kalman refit with outlier rejection).

Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

RECIPE = dict(seed=3, n_tracks=24, sectors=[0, 21], noise_frac=0.05)
OUT = os.path.join(HERE, "tiny_event_oracle.json")


def event():
    import synth
    return synth.make_tiny(seed=RECIPE["seed"], n_tracks=RECIPE["n_tracks"],
                           sectors=tuple(RECIPE["sectors"]), noise_frac=RECIPE["noise_frac"])


def compute():
    import oracle
    import synth
    from paper_1811_11481_b300.config import default_params
    geo = synth.geometry()
    ev = event()
    o = oracle.Oracle(ev, geo, default_params(), synth.nominal_calib())
    f = o.find(32)
    tr = f["tracks"]
    r = o.refit(tr["track_start"], tr["cluster_idx"], tr["that"], prec=64)
    return dict(
        source="oracle (FP32 mirror for links and tracks, Sec. 2 phase 1; FP64 three-pass "
               "refit, Sec. 3), written by tests/golden/make_golden.py",
        recipe=RECIPE, n_clusters=int(ev.n),
        up=f["up"].tolist(), dn=f["dn"].tolist(),
        track_start=tr["track_start"].tolist(), cluster_idx=tr["cluster_idx"].tolist(),
        start_hit=tr["start_hit"].tolist(),
        params=r["params"].tolist(), chi2=r["chi2"].tolist(), ndf=r["ndf"].tolist(),
        status=r["status"].tolist())


if __name__ == "__main__":
    d = compute()
    with open(OUT, "w") as fh:
        json.dump(d, fh, separators=(",", ":"))
        fh.write("\n")
    print(f"wrote {OUT}: {d['n_clusters']} clusters, {len(d['track_start']) - 1} tracks")
