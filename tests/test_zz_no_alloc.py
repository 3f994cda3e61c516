"""The allocation-free refit entry point (tpc_refit_noalloc).

Callers that cannot allocate device memory at refit time -- inside a CUDA
graph capture, in a real-time loop, or under a framework whose allocator owns
the device -- use tpc_refit_noalloc, which keeps its working memory in a fixed
device array. These tests call it through the C ABI: twice in a row (two
different track sets, so the shared array is reused) against the
context-based tpc_refit of the same tracks and against the FP64 oracle,
within the refit tolerance used by the other parity tests; then the edge
cases (invalid track ranges and rows, no flags, no tracks, exactly the
largest accepted size, a full-field geometry, an oversized input).
"""
import ctypes as C

import numpy as np
import pytest

import synth
from pipeline import RTOL, rel_err, tracker

pytestmark = pytest.mark.gpu

MAX_ASSIGNED = 1 << 20


def _geometry(field=None):
    from paper_1811_11481_b300 import binding
    geo = synth.geometry()
    rx = np.ascontiguousarray(geo.row_x, np.float32)
    keep = [rx]
    fp = None
    if field is not None:
        fld = np.ascontiguousarray(field, np.float32).reshape(-1)
        keep.append(fld)
        fp = fld.ctypes.data_as(C.POINTER(C.c_float))
    g = binding.tpc_geometry(rx.size, rx.ctypes.data_as(C.POINTER(C.c_float)),
                             float(geo.tan_half), float(geo.drift_length), float(geo.bz),
                             None, None, fp)
    return g, keep


def _call(ts, yc, zc, row, flags, n_assigned=None, field=None, expect=0):
    """tpc_refit_noalloc on device tensors; outputs pre-filled with sentinels."""
    import torch
    from paper_1811_11481_b300 import binding
    L = binding.load_library()
    nt = ts.numel() - 1
    na = yc.numel() if n_assigned is None else n_assigned
    dev = yc.device
    out = dict(params=torch.full((max(nt, 1), 5), float("nan"), device=dev),
               cov=torch.full((max(nt, 1), 15), float("nan"), device=dev),
               chi2=torch.full((max(nt, 1),), float("nan"), device=dev),
               ndf=torch.full((max(nt, 1),), -7, dtype=torch.int32, device=dev),
               status=torch.full((max(nt, 1),), -7, dtype=torch.int32, device=dev))
    g, keep = _geometry(field)
    P = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    st = L.tpc_refit_noalloc(C.byref(g), None, C.c_void_p(torch.cuda.current_stream().cuda_stream),
                             nt, na, P(ts), P(yc), P(zc), P(row), P(flags), P(out["params"]),
                             P(out["cov"]), P(out["chi2"]), P(out["ndf"]), P(out["status"]))
    assert st == expect, st
    torch.cuda.synchronize()
    del keep
    return {k: v.cpu().numpy() for k, v in out.items()}


def _reference(geo, ev, ts, ci, tc):
    """The context path on the same tracks: calibrated inputs and refit."""
    import torch
    tr = tracker(geo)
    tr.set_calib()
    cl = tr.upload(ev)
    tr.load(cl)
    tr.set_tracks(torch.as_tensor(ts.astype(np.int32)), torch.as_tensor(ci.astype(np.int32)),
                  torch.as_tensor(tc))
    r = tr.refit()
    yc, zc = tr.calibrated()
    ref = {k: v.cpu().numpy() for k, v in r.items()}
    idx = torch.as_tensor(ci.astype(np.int64), device=tr.dev)
    inputs = dict(ts=torch.as_tensor(ts.astype(np.int32), device=tr.dev), yc=yc.contiguous(),
                  zc=zc.contiguous(), row=cl["row"][idx].contiguous(),
                  flags=cl["flags"][idx].contiguous())
    return tr, ref, inputs


def _compare(got, ref):
    assert np.array_equal(got["status"], ref["status"])
    ok = ref["status"] == 0
    assert ok.sum() > 0
    np.testing.assert_array_equal(got["ndf"][ok], ref["ndf"][ok])
    e = rel_err(got["params"][ok].astype(np.float64), ref["params"][ok].astype(np.float64))
    assert np.all(e <= RTOL), e.max(0)
    np.testing.assert_allclose(got["chi2"][ok], ref["chi2"][ok], rtol=1e-4, atol=1e-4)


def _compare_oracle(got, geo, ev, ts, ci, tc):
    """Against the FP64 oracle's refit of the same tracks (the oracle
    calibrates the clusters itself)."""
    import oracle
    from paper_1811_11481_b300.config import default_params
    o = oracle.Oracle(ev, geo, default_params(), synth.nominal_calib())
    ref = o.refit(ts, ci, tc, prec=64)
    ok = (got["status"] == 0) & (ref["status"] == 0)
    assert np.mean(got["status"] == ref["status"]) > 0.99
    same = np.array([np.array_equal(got["ndf"][k:k + 1], ref["ndf"][k:k + 1])
                     for k in range(ts.size - 1)])
    sel = ok & same
    assert sel.sum() > 0.98 * ok.sum() > 0
    e = rel_err(got["params"][sel].astype(np.float64), ref["params"][sel])
    assert np.all(e <= RTOL), e.max(0)
    np.testing.assert_allclose(got["chi2"][sel], ref["chi2"][sel], rtol=2e-3, atol=1e-2)


@pytest.fixture(scope="module")
def tiny():
    geo = synth.geometry()
    ev = synth.make_tiny(seed=41, n_tracks=400, central=True, noise_frac=0.05)
    ts, ci, tc, _ = synth.truth_tracks(ev, 20)
    return geo, ev, ts, ci, tc


def test_noalloc_refit_matches_context_refit_and_oracle_twice(tiny):
    geo, ev, ts, ci, tc = tiny
    # first call: all tracks
    tr, ref, inp = _reference(geo, ev, ts, ci, tc)
    got = _call(inp["ts"], inp["yc"], inp["zc"], inp["row"], inp["flags"])
    _compare(got, ref)
    _compare_oracle(got, geo, ev, ts, ci, tc)
    # second call: a different, smaller track set reusing the same scratch
    k = (ts.size - 1) // 2
    ts2 = (ts[k:] - ts[k]).astype(np.uint32)
    ci2 = ci[ts[k]:]
    tr2, ref2, inp2 = _reference(geo, ev, ts2, ci2, tc[k:])
    got2 = _call(inp2["ts"], inp2["yc"], inp2["zc"], inp2["row"], inp2["flags"])
    _compare(got2, ref2)
    _compare_oracle(got2, geo, ev, ts2, ci2, tc[k:])


def test_noalloc_invalid_ranges_and_rows_give_status_3(tiny):
    import torch
    geo, ev, ts, ci, tc = tiny
    tr, ref, inp = _reference(geo, ev, ts, ci, tc)
    na = int(ts[-1])
    T = lambda a: torch.as_tensor(np.asarray(a, np.int32), device=tr.dev)
    a0, a1, a2 = int(ts[4]), int(ts[5]), int(ts[6])
    # track 0 = truth track 5, track 1 reversed, track 2 = truth track 4
    # (ranges do not overlap), track 3 ends beyond the assigned clusters
    bad_ts = T([a1, a2, a0, a1, na + 3])
    got = _call(bad_ts, inp["yc"], inp["zc"], inp["row"], inp["flags"])
    assert got["status"][1] == 3 and got["status"][3] == 3
    assert got["chi2"][1] == 0 and got["ndf"][1] == 0 and got["chi2"][3] == 0
    for k, t in ((0, 5), (2, 4)):
        assert got["status"][k] == ref["status"][t]
        if ref["status"][t] != 0:
            continue
        e = rel_err(got["params"][k].astype(np.float64), ref["params"][t].astype(np.float64))
        assert np.all(e <= RTOL), e
    # a row beyond the geometry inside truth track 7
    row = inp["row"].clone()
    row[int(ts[7]) + 2] = 200
    got = _call(inp["ts"], inp["yc"], inp["zc"], row, inp["flags"])
    assert got["status"][7] == 3 and got["chi2"][7] == 0 and got["ndf"][7] == 0
    others = np.arange(ts.size - 1) != 7
    assert np.array_equal(got["status"][others], ref["status"][others])


def test_noalloc_without_flags_equals_zero_flags(tiny):
    import torch
    geo, ev, ts, ci, tc = tiny
    tr, ref, inp = _reference(geo, ev, ts, ci, tc)
    zero = torch.zeros_like(inp["flags"])
    a = _call(inp["ts"], inp["yc"], inp["zc"], inp["row"], zero)
    b = _call(inp["ts"], inp["yc"], inp["zc"], inp["row"], None)
    for k in a:
        assert np.array_equal(a[k], b[k], equal_nan=True), k


def test_noalloc_no_tracks_writes_nothing(tiny):
    import torch
    geo, ev, ts, ci, tc = tiny
    tr, ref, inp = _reference(geo, ev, ts, ci, tc)
    got = _call(inp["ts"][:1], inp["yc"], inp["zc"], inp["row"], inp["flags"])
    assert np.isnan(got["chi2"]).all() and (got["status"] == -7).all()


def test_noalloc_at_the_largest_accepted_size(tiny):
    """Exactly TPC_NOALLOC_MAX_ASSIGNED assigned clusters: the truth tracks
    tiled until the array is full; every copy refits like the first."""
    import torch
    geo, ev, ts, ci, tc = tiny
    tr, ref, inp = _reference(geo, ev, ts, ci, tc)
    na = int(ts[-1])
    reps = MAX_ASSIGNED // na
    pad = MAX_ASSIGNED - reps * na
    tile = lambda t: torch.cat([t.repeat(reps), t[:pad]])
    yc, zc, row, flags = (tile(inp[k]) for k in ("yc", "zc", "row", "flags"))
    assert yc.numel() == MAX_ASSIGNED
    base = ts[:-1].astype(np.int64)
    big_ts = np.concatenate([base + r * na for r in range(reps)] + [[reps * na]])
    got = _call(torch.as_tensor(big_ts.astype(np.int32), device=tr.dev), yc, zc, row, flags)
    nt = ts.size - 1
    one = _call(inp["ts"], inp["yc"], inp["zc"], inp["row"], inp["flags"])
    for r in (0, reps // 2, reps - 1):
        sl = slice(r * nt, (r + 1) * nt)
        for k in ("status", "ndf", "params", "chi2"):
            assert np.array_equal(got[k][sl], one[k], equal_nan=True), (r, k)
    # one more cluster is refused before any work
    more = torch.cat([yc, yc[:1]])
    _call(torch.as_tensor(big_ts.astype(np.int32), device=tr.dev), more, more, tile(inp["row"]),
          None, n_assigned=MAX_ASSIGNED + 1, expect=2)


def test_noalloc_refuses_a_full_field_geometry(tiny):
    from synth.field import solenoid_field
    geo, ev, ts, ci, tc = tiny
    tr, ref, inp = _reference(geo, ev, ts, ci, tc)
    got = _call(inp["ts"], inp["yc"], inp["zc"], inp["row"], inp["flags"],
                field=solenoid_field(), expect=1)
    assert (got["status"] == -7).all()


def test_noalloc_rejects_oversized_input_before_any_work():
    from paper_1811_11481_b300 import binding
    L = binding.load_library()
    g, keep = _geometry()
    too_many = MAX_ASSIGNED + 1
    st = L.tpc_refit_noalloc(C.byref(g), None, None, 10, too_many, *([None] * 10))
    assert st == 2  # TPC_ERR_CAPACITY
