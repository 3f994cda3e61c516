"""CPU oracle of the TPC hot path (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It wraps ``liborc.so`` (built from
``oracle.cpp`` with g++, strict IEEE: no FMA contraction, no fast-math) with
ctypes. It shares no code with the CUDA library and does not import it.

Every input (clusters, geometry, calibration, cut values) is passed in; the
oracle keeps no defaults of its own for the method's parameters.

Parity unpinned: the numerical values of the cellular-automaton cuts are
readings (Sec. 2 and Sec. 4 of the paper give none); the tests pin the
arithmetic with closed forms, brute force and library routines.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.cpp")
# TPC_ORACLE_LIB: a prebuilt library to load instead (the mutation tests
# build variants of oracle.cpp with a planted mistake and run the pins on them)
LIB = os.environ.get("TPC_ORACLE_LIB") or os.path.join(HERE, "liborc.so")
N_SPLINE = 36 * 2 * 8 * 8 * 8

CXXFLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", "-fopenmp"]


def build(force=False):
    """Compile liborc.so (g++, IEEE-strict)."""
    if os.environ.get("TPC_ORACLE_LIB"):
        return LIB
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cmd = ["g++", *CXXFLAGS, SRC, "-o", LIB]
    subprocess.check_call(cmd)
    return LIB


class _Geom(C.Structure):
    _fields_ = [("row_x", C.POINTER(C.c_float)), ("n_rows", C.c_int32),
                ("tan_half", C.c_float), ("drift_length", C.c_float), ("bz", C.c_float),
                ("pad_width", C.POINTER(C.c_float)), ("pad_center", C.POINTER(C.c_float)),
                ("field", C.POINTER(C.c_float))]


class _Params(C.Structure):
    _fields_ = [("sigma", C.c_float), ("shared_scale", C.c_float),
                ("nb_wy", C.c_float), ("nb_wz", C.c_float), ("nb_teta", C.c_float),
                ("nb_ty", C.c_float),
                ("nb_dmax", C.c_float), ("chi2_pick", C.c_float),
                ("max_miss", C.c_int32), ("max_gap", C.c_int32),
                ("min_track_hits", C.c_int32), ("s_max", C.c_float),
                ("inward_cov_scale", C.c_float), ("c0t", C.c_float * 5),
                ("c0r", C.c_float * 5), ("chi2_out", C.c_float),
                ("min_acc_reject", C.c_int32), ("refit_inflate", C.c_float),
                ("seed_max_hits", C.c_int32), ("chi2_merge", C.c_float),
                ("split_scale", C.c_float), ("single_row_scale", C.c_float),
                ("single_time_scale", C.c_float), ("edge_scale", C.c_float)]


class _Calib(C.Structure):
    _fields_ = [("vdrift", C.c_double), ("t0", C.c_double), ("tf_start", C.c_double),
                ("spline", C.POINTER(C.c_float)), ("spl_x0", C.c_float),
                ("spl_dx", C.c_float)]


class _Clusters(C.Structure):
    _fields_ = [("n", C.c_int64), ("mode", C.c_int32), ("n_events", C.c_int32),
                ("y", C.POINTER(C.c_float)), ("z", C.POINTER(C.c_float)),
                ("t", C.POINTER(C.c_double)), ("row", C.POINTER(C.c_uint8)),
                ("sector", C.POINTER(C.c_uint8)), ("flags", C.POINTER(C.c_uint8)),
                ("event", C.POINTER(C.c_uint32)), ("pads", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        vp = C.c_void_p
        L.orc_create.restype = vp
        L.orc_create.argtypes = [C.POINTER(_Geom), C.POINTER(_Params), C.POINTER(_Calib),
                                 C.POINTER(_Clusters)]
        L.orc_destroy.argtypes = [vp]
        L.orc_seed_z.argtypes = [vp, C.c_int, vp]
        L.orc_calibrate.argtypes = [vp, C.c_int, C.c_int64, vp, vp, vp, vp]
        L.orc_spline.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, vp]
        L.orc_neighbours.argtypes = [vp, C.c_int, vp, C.c_int64, vp, vp, vp]
        L.orc_clean.argtypes = [vp, vp, vp, vp, vp]
        L.orc_start_hits.restype = C.c_int64
        L.orc_start_hits.argtypes = [vp, vp, vp, vp]
        L.orc_tracklets.argtypes = [vp, C.c_int, vp, C.c_int64, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_select.restype = C.c_int64
        L.orc_select.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, vp, vp, vp,
                                 C.c_int64, C.c_int64]
        L.orc_refit.argtypes = [vp, C.c_int, C.c_int64, vp, vp, vp, vp, vp, C.c_int, vp,
                                vp, vp, vp, vp, vp, vp, vp, C.c_double]
        L.orc_refit_grad.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                     C.c_double]
        L.orc_propagate.restype = C.c_int
        L.orc_propagate.argtypes = [vp, vp, C.c_double, C.c_double, vp, vp, vp]
        L.orc_refit_points.restype = C.c_int
        L.orc_refit_points.argtypes = [vp, C.c_int64, vp, vp, vp, C.c_double, vp, vp, vp, vp,
                                       vp]
        L.orc_set_joseph.argtypes = [vp, C.c_int]
        L.orc_jacobian.restype = C.c_int
        L.orc_jacobian.argtypes = [vp, vp, C.c_double, C.c_double, vp, vp]
        L.orc_update.argtypes = [vp, vp, C.c_double, C.c_double, C.c_double, C.c_double,
                                 vp, vp, vp]
        L.orc_merge.restype = C.c_int64
        L.orc_merge.argtypes = [vp, C.c_int, C.c_int64, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                vp, vp, vp, vp]
        L.orc_compress.argtypes = [vp, C.c_int64, vp, vp, vp, C.c_float, C.c_float, vp, vp, vp,
                                   vp]
        L.orc_decompress.argtypes = [vp, C.c_int64, vp, vp, C.c_float, C.c_float, vp, vp, vp, vp]
        L.orc_refine_time.argtypes = [vp, C.c_int, C.c_int64, vp, vp, vp, vp, vp, vp, vp]
        L.orc_propagate_field.restype = C.c_int
        L.orc_propagate_field.argtypes = [vp, vp, C.c_double, C.c_double, C.c_double, vp, vp,
                                          vp]
        L.orc_rotate.restype = C.c_int
        L.orc_rotate.argtypes = [vp, vp, C.c_double, C.c_double, vp, vp, vp, vp]
        L.orc_dca_z.restype = C.c_double
        L.orc_dca_z.argtypes = [vp, vp, C.c_double]
        L.orc_threads.restype = C.c_int
        L.orc_threads.argtypes = [C.c_int]
        L.orc_arc_factor.restype = C.c_double
        L.orc_arc_factor.argtypes = [C.c_int, C.c_double]
        L.orc_arc_deriv.restype = C.c_double
        L.orc_arc_deriv.argtypes = [C.c_int, C.c_double]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def threads(n=0):
    """Set the oracle's thread count (n >= 1; loops over hits, start hits,
    tracks and clusters run in parallel) and return the count in force."""
    return lib().orc_threads(int(n))


def arc_factor(h, prec=64):
    """asin(h)/h as the oracle evaluates it (prec 32: the FP32 sequence)."""
    return lib().orc_arc_factor(prec, float(h))


def arc_deriv(h, prec=64):
    return lib().orc_arc_deriv(prec, float(h))


class Oracle:
    """Oracle bound to one batch of clusters.

    ev: object with y, z or t, row, sector, flags, event, mode, n_events
    geo: object with row_x (float32[152]), tan_half, drift_length, bz
    params: dict of the method's cut values (names as in OrcParams)
    calib: object with vdrift, t0, spline ([36][2][8][8][8] float32)
    """

    def __init__(self, ev, geo, params, calib, tf_start=None, spl_x0=85.0, spl_dx=160.0,
                 pads=False, field=None):
        L = lib()
        self._keep = []
        k = self._keep
        self.n = int(ev.y.shape[0])
        self.n_rows = int(len(geo.row_x))
        rowx = np.ascontiguousarray(geo.row_x, np.float32)
        k.append(rowx)
        fp = lambda a: a.ctypes.data_as(C.POINTER(C.c_float)) if a is not None else None
        pw = pc = None
        if pads:
            pw = np.ascontiguousarray(geo.pad_width, np.float32)
            pc = np.ascontiguousarray(geo.pad_center, np.float32)
            k.extend([pw, pc])
        fld = None
        if field is not None:
            fld = np.ascontiguousarray(field, np.float32).reshape(-1)
            assert fld.size == 30
            k.append(fld)
        self.g = _Geom(fp(rowx), self.n_rows, float(geo.tan_half), float(geo.drift_length),
                       float(geo.bz), fp(pw), fp(pc), fp(fld))
        p = _Params()
        for name, _t in _Params._fields_:
            v = params[name]
            if name in ("c0t", "c0r"):
                setattr(p, name, (C.c_float * 5)(*[float(x) for x in v]))
            else:
                setattr(p, name, v)
        self.p = p
        spl = np.ascontiguousarray(calib.spline, np.float32).reshape(-1)
        assert spl.size == N_SPLINE
        k.append(spl)
        tfs = float(getattr(ev, "tf_start", 0.0) if tf_start is None else tf_start)
        self.c = _Calib(float(calib.vdrift), float(calib.t0), tfs,
                        spl.ctypes.data_as(C.POINTER(C.c_float)), spl_x0, spl_dx)
        mode = 0 if ev.mode == "event" else 1
        # with pads, the native pad positions take the place of y
        y = np.ascontiguousarray(ev.pad if pads else ev.y, np.float32)
        z = np.ascontiguousarray(ev.z, np.float32) if mode == 0 else None
        t = np.ascontiguousarray(ev.t, np.float64) if mode == 1 else None
        row = np.ascontiguousarray(ev.row, np.uint8)
        sec = np.ascontiguousarray(ev.sector, np.uint8)
        flg = np.ascontiguousarray(ev.flags, np.uint8)
        evt = np.ascontiguousarray(ev.event, np.uint32)
        k.extend([y, z, t, row, sec, flg, evt])
        self.row = row
        cast = lambda a, T: (a.ctypes.data_as(C.POINTER(T)) if a is not None else None)
        self.cl = _Clusters(self.n, mode, int(ev.n_events), cast(y, C.c_float),
                            cast(z, C.c_float), cast(t, C.c_double), cast(row, C.c_uint8),
                            cast(sec, C.c_uint8), cast(flg, C.c_uint8), cast(evt, C.c_uint32),
                            1 if pads else 0)
        self.mode = mode
        self.h = L.orc_create(C.byref(self.g), C.byref(self.p), C.byref(self.c),
                              C.byref(self.cl))

    def close(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- a2
    def seed_z(self, prec=32):
        out = np.empty(self.n, np.float32 if prec == 32 else np.float64)
        lib().orc_seed_z(self.h, prec, _p(out))
        return out

    def calibrate(self, idx, that, prec=64):
        idx = np.ascontiguousarray(idx, np.uint32)
        that = np.ascontiguousarray(np.broadcast_to(that, idx.shape), np.float64)
        yc = np.empty(idx.size)
        zc = np.empty(idx.size)
        lib().orc_calibrate(self.h, prec, idx.size, _p(idx), _p(that), _p(yc), _p(zc))
        return yc, zc

    def spline(self, sector, x, y, az):
        sector = np.ascontiguousarray(sector, np.int32)
        x, y, az = (np.ascontiguousarray(a, np.float64) for a in (x, y, az))
        dy = np.empty(x.size)
        dz = np.empty(x.size)
        lib().orc_spline(self.h, x.size, _p(sector), _p(x), _p(y), _p(az), _p(dy), _p(dz))
        return dy, dz

    # --- a4-a6
    def neighbours(self, prec=32, hits=None, margin=False):
        """Links (up, dn) of every cluster or of 'hits'; with margin (FP64
        only) also each hit's smallest decision margin."""
        if hits is not None:
            hits = np.ascontiguousarray(hits, np.int64)
            m = hits.size
        else:
            m = self.n
        up = np.empty(m, np.int32)
        dn = np.empty(m, np.int32)
        mg = np.empty(m) if margin else None
        assert not margin or prec == 64
        lib().orc_neighbours(self.h, prec, _p(hits), m, _p(up), _p(dn), _p(mg))
        return (up, dn, mg) if margin else (up, dn)

    def clean(self, up, dn):
        up = np.ascontiguousarray(up, np.int32)
        dn = np.ascontiguousarray(dn, np.int32)
        upc = np.empty_like(up)
        dnc = np.empty_like(dn)
        lib().orc_clean(self.h, _p(up), _p(dn), _p(upc), _p(dnc))
        return upc, dnc

    def start_hits(self, upc, dnc):
        out = np.empty(self.n, np.int64)
        m = lib().orc_start_hits(self.h, _p(np.ascontiguousarray(upc, np.int32)),
                                 _p(np.ascontiguousarray(dnc, np.int32)), _p(out))
        return out[:m].copy()

    # --- a7
    def tracklets(self, upc, starts, prec=32, margin=False):
        """One tracklet per start hit; with margin (FP64 only) also each
        tracklet's smallest decision margin and its number of decisions."""
        starts = np.ascontiguousarray(starts, np.int64)
        m = starts.size
        nh = np.empty(m, np.int32)
        hits = np.empty((m, self.n_rows), np.int32)
        that = np.empty(m)
        state = np.empty((m, 5))
        x = np.empty(m)
        mg = np.empty(m) if margin else None
        nd = np.empty(m, np.int64) if margin else None
        assert not margin or prec == 64
        lib().orc_tracklets(self.h, prec, _p(np.ascontiguousarray(upc, np.int32)), m,
                            _p(starts), _p(nh), _p(hits), _p(that), _p(state), _p(x), _p(mg),
                            _p(nd))
        out = dict(nh=nh, hits=hits, that=that, state=state, x=x)
        if margin:
            out.update(margin=mg, decisions=nd)
        return out

    # --- a8
    def select(self, starts, tl):
        starts = np.ascontiguousarray(starts, np.int64)
        m = starts.size
        cap_t = self.n // max(1, int(self.p.min_track_hits)) + 2
        ts = np.zeros(cap_t + 1, np.uint32)
        ci = np.zeros(self.n + 1, np.uint32)
        tt = np.zeros(cap_t)
        tid = np.zeros(cap_t, np.int64)
        nt = lib().orc_select(self.h, m, _p(starts), _p(tl["nh"]), _p(tl["hits"]),
                              _p(tl["that"]), _p(ts), _p(ci), _p(tt), _p(tid), cap_t, self.n)
        assert nt >= 0
        return dict(track_start=ts[:nt + 1].copy(), cluster_idx=ci[:ts[nt]].copy(),
                    that=tt[:nt].copy(), start_hit=tid[:nt].copy())

    def find(self, prec=32):
        """Sec. 2 phase 1 end to end: links, cleaning, start hits, tracklets, selection."""
        up, dn = self.neighbours(prec)
        upc, dnc = self.clean(up, dn)
        starts = self.start_hits(upc, dnc)
        tl = self.tracklets(upc, starts, prec)
        tr = self.select(starts, tl)
        return dict(up=up, dn=dn, upc=upc, dnc=dnc, starts=starts, tracklets=tl, tracks=tr)

    # --- a9-a10
    def refit(self, track_start, cluster_idx, that, prec=64, seeds=None, rej=None, zv=None,
              vsigma=0.01):
        """Three-pass refit of the tracks (CSR); zv: optional vertex z per
        track (NaN: none) with error vsigma (cm)."""
        ts = np.ascontiguousarray(track_start, np.uint32)
        ci = np.ascontiguousarray(cluster_idx, np.uint32)
        that = np.ascontiguousarray(that, np.float64)
        nt = ts.size - 1
        frozen = rej is not None
        rj = np.ascontiguousarray(rej, np.uint8).copy() if frozen else np.zeros(ci.size, np.uint8)
        sd = None if seeds is None else np.ascontiguousarray(seeds, np.float64)
        so = np.empty((nt, 5))
        out = dict(params=np.empty((nt, 5)), cov=np.empty((nt, 15)), x=np.empty(nt),
                   chi2=np.empty(nt), ndf=np.empty(nt, np.int32),
                   status=np.empty(nt, np.int32))
        zvv = None if zv is None else np.ascontiguousarray(zv, np.float64)
        lib().orc_refit(self.h, prec, nt, _p(ts), _p(ci), _p(that), _p(sd), _p(so),
                        int(frozen), _p(rj), _p(out["params"]), _p(out["cov"]), _p(out["x"]),
                        _p(out["chi2"]), _p(out["ndf"]), _p(out["status"]), _p(zvv),
                        float(vsigma) ** 2)
        out["rej"] = rj
        out["seeds"] = so
        return out

    # --- a11
    def refit_grad(self, track_start, cluster_idx, that, seeds, rej, g=None, zv=None,
                   vsigma=0.01):
        ts = np.ascontiguousarray(track_start, np.uint32)
        ci = np.ascontiguousarray(cluster_idx, np.uint32)
        nt = ts.size - 1
        g = np.ones(nt) if g is None else np.ascontiguousarray(g, np.float64)
        gy = np.zeros(ci.size)
        gz = np.zeros(ci.size)
        gc = np.zeros(2 + N_SPLINE)
        lib().orc_refit_grad(self.h, nt, _p(ts), _p(ci), _p(np.ascontiguousarray(that, np.float64)),
                             _p(np.ascontiguousarray(seeds, np.float64)),
                             _p(np.ascontiguousarray(rej, np.uint8)), _p(g), _p(gy), _p(gz), _p(gc),
                             _p(None if zv is None else np.ascontiguousarray(zv, np.float64)),
                             float(vsigma) ** 2)
        return gy, gz, gc

    # --- Sec. 2 second phase: segment merging
    def merge(self, track_start, cluster_idx, that, params, cov, x, status, prec=32):
        """Links between segments and the merged track set; params, cov, x,
        status: the segments' refitted states at their innermost cluster."""
        ts = np.ascontiguousarray(track_start, np.uint32)
        ci = np.ascontiguousarray(cluster_idx, np.uint32)
        nt = ts.size - 1
        f64 = lambda a, shp: np.ascontiguousarray(np.asarray(a, np.float64).reshape(shp))
        nxt = np.empty(nt, np.int32)
        lc = np.empty(nt)
        ots = np.zeros(nt + 1, np.uint32)
        oci = np.zeros(max(ci.size, 1), np.uint32)
        oth = np.zeros(max(nt, 1))
        ohd = np.zeros(max(nt, 1), np.int64)
        m = lib().orc_merge(self.h, prec, nt, _p(ts), _p(ci), _p(f64(that, (nt,))),
                            _p(f64(params, (nt, 5))), _p(f64(cov, (nt, 15))),
                            _p(f64(x, (nt,))), _p(np.ascontiguousarray(status, np.int32)),
                            _p(nxt), _p(lc), _p(ots), _p(oci), _p(oth), _p(ohd))
        return dict(next=nxt, link_chi2=lc, track_start=ots[:m + 1].copy(),
                    cluster_idx=oci[:ci.size].copy(), that=oth[:m].copy(), head=ohd[:m].copy())

    def refine_time(self, track_start, cluster_idx, that, params, x, status, prec=32):
        """Collision times refined from the tracks' fits (time-frame mode)."""
        ts = np.ascontiguousarray(track_start, np.uint32)
        nt = ts.size - 1
        out = np.empty(nt)
        lib().orc_refine_time(self.h, prec, nt, _p(ts),
                              _p(np.ascontiguousarray(cluster_idx, np.uint32)),
                              _p(np.ascontiguousarray(that, np.float64)),
                              _p(np.ascontiguousarray(np.reshape(params, (nt, 5)), np.float64)),
                              _p(np.ascontiguousarray(x, np.float64)),
                              _p(np.ascontiguousarray(status, np.int32)), _p(out))
        return out

    # --- Sec. 5: track-model compression
    def compress(self, track_start, cluster_idx, that, qy=0.01, qz=0.01):
        """Residuals (ry, rz) of the track set's clusters and the decoded
        clusters (dy, dz)."""
        ts = np.ascontiguousarray(track_start, np.uint32)
        ci = np.ascontiguousarray(cluster_idx, np.uint32)
        nt = ts.size - 1
        ry = np.zeros(ci.size, np.int32)
        rz = np.zeros(ci.size, np.int32)
        dy = np.zeros(ci.size, np.float32)
        dz = np.zeros(ci.size, np.float32)
        lib().orc_compress(self.h, nt, _p(ts), _p(ci), _p(np.ascontiguousarray(that, np.float64)),
                           float(qy), float(qz), _p(ry), _p(rz), _p(dy), _p(dz))
        return dict(ry=ry, rz=rz, dy=dy, dz=dz)

    def decompress(self, track_start, cluster_idx, ry, rz, qy=0.01, qz=0.01):
        ts = np.ascontiguousarray(track_start, np.uint32)
        ci = np.ascontiguousarray(cluster_idx, np.uint32)
        dy = np.zeros(ci.size, np.float32)
        dz = np.zeros(ci.size, np.float32)
        lib().orc_decompress(self.h, ts.size - 1, _p(ts), _p(ci), float(qy), float(qz),
                             _p(np.ascontiguousarray(ry, np.int32)),
                             _p(np.ascontiguousarray(rz, np.int32)), _p(dy), _p(dz))
        return dy, dz

    # --- single-step helpers
    def propagate(self, state, x1, x2, cov=None):
        s = np.ascontiguousarray(state, np.float64)
        cv = np.eye(5) if cov is None else np.ascontiguousarray(cov, np.float64)
        so = np.empty(5)
        co = np.empty((5, 5))
        ok = lib().orc_propagate(self.h, _p(s), float(x1), float(x2), _p(cv), _p(so), _p(co))
        return (so, co) if ok else (None, None)

    def refit_points(self, x, y, z, var, details=False):
        """FP64 refit of explicit points (three-point seed); with details also
        the state each pass starts from (x, parameters, 5x5 covariance) and
        the final covariance (5x5)."""
        x, y, z = (np.ascontiguousarray(a, np.float64) for a in (x, y, z))
        p = np.empty(5)
        ch = np.empty(1)
        nd = np.empty(1, np.int32)
        pr = np.empty((3, 21))
        cv = np.empty(15)
        stt = lib().orc_refit_points(self.h, x.size, _p(x), _p(y), _p(z), float(var), _p(p),
                                     _p(ch), _p(nd), _p(pr), _p(cv))
        if not details:
            return stt, p, float(ch[0]), int(nd[0])

        def sym(v):
            m = np.zeros((5, 5))
            m[np.tril_indices(5)] = v
            return m + np.tril(m, -1).T
        priors = [dict(x=pr[k, 0], p=pr[k, 1:6].copy(), C=sym(pr[k, 6:])) for k in range(3)]
        return stt, p, float(ch[0]), int(nd[0]), priors, sym(cv)

    def set_joseph(self, on=True):
        """Covariance update of the refit in the Joseph form (on) or the
        short form (off, the default)."""
        lib().orc_set_joseph(self.h, int(bool(on)))

    def rotate(self, state, x, dalpha, cov=None):
        """The state re-expressed in a frame rotated by dalpha (and its
        covariance, 5x5); (None, None, None) when the rotation fails."""
        s = np.ascontiguousarray(state, np.float64)
        cv = np.eye(5) if cov is None else np.ascontiguousarray(cov, np.float64)
        so = np.empty(5)
        co = np.empty((5, 5))
        xo = np.empty(1)
        ok = lib().orc_rotate(self.h, _p(s), float(x), float(dalpha), _p(cv), _p(so), _p(xo),
                              _p(co))
        return (so, float(xo[0]), co) if ok else (None, None, None)

    def propagate_field(self, state, x1, x2, alpha, cov=None):
        """Transport in the full field in the frame rotated by alpha."""
        s = np.ascontiguousarray(state, np.float64)
        cv = np.eye(5) if cov is None else np.ascontiguousarray(cov, np.float64)
        so = np.empty(5)
        co = np.empty((5, 5))
        ok = lib().orc_propagate_field(self.h, _p(s), float(x1), float(x2), float(alpha),
                                       _p(cv), _p(so), _p(co))
        return (so, co) if ok else (None, None)

    def jacobian(self, state, x1, x2):
        so = np.empty(5)
        J = np.empty((5, 5))
        ok = lib().orc_jacobian(self.h, _p(np.ascontiguousarray(state, np.float64)), float(x1),
                                float(x2), _p(so), _p(J))
        return (so, J) if ok else (None, None)

    @staticmethod
    def update(state, cov, my, mz, vy, vz):
        so = np.empty(5)
        co = np.empty((5, 5))
        ch = np.empty(1)
        lib().orc_update(_p(np.ascontiguousarray(state, np.float64)),
                         _p(np.ascontiguousarray(cov, np.float64)), float(my), float(mz),
                         float(vy), float(vz), _p(so), _p(co), _p(ch))
        return so, co, float(ch[0])

    def dca_z(self, state, x):
        return lib().orc_dca_z(self.h, _p(np.ascontiguousarray(state, np.float64)), float(x))
