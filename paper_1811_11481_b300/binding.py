"""ctypes binding of libtpc.so (include/tpc.h), argument marshalling only.

Functions keep the C names (tpc_create, tpc_load_clusters, ...). ``Tracker``
wraps one context with torch tensors as device memory and the current torch
stream as the work stream. There is no fallback: without the built library,
or without a CUDA device, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtpc.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "tpc.h")

TPC_MAX_ROWS = 160
TPC_SPLINE_SIZE = 36 * 2 * 8 * 8 * 8
TPC_GRAD_CALIB_SIZE = 2 + TPC_SPLINE_SIZE
STATUS = {0: "TPC_OK", 1: "TPC_ERR_ARG", 2: "TPC_ERR_CAPACITY", 3: "TPC_ERR_CUDA",
          4: "TPC_ERR_TIMEOUT", 5: "TPC_ERR_STATE", 6: "TPC_ERR_NUMERIC"}


class TpcError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


class tpc_geometry(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("row_x", C.POINTER(C.c_float)),
                ("tan_half", C.c_float), ("drift_length", C.c_float), ("bz", C.c_float),
                ("pad_width", C.POINTER(C.c_float)), ("pad_center", C.POINTER(C.c_float)),
                ("field", C.POINTER(C.c_float))]


class tpc_params(C.Structure):
    _fields_ = [("sigma", C.c_float), ("shared_scale", C.c_float), ("nb_wy", C.c_float),
                ("nb_wz", C.c_float), ("nb_teta", C.c_float), ("nb_ty", C.c_float),
                ("nb_dmax", C.c_float), ("chi2_pick", C.c_float), ("max_miss", C.c_int32),
                ("max_gap", C.c_int32), ("min_track_hits", C.c_int32), ("s_max", C.c_float),
                ("inward_cov_scale", C.c_float), ("c0t", C.c_float * 5),
                ("c0r", C.c_float * 5), ("chi2_out", C.c_float),
                ("min_acc_reject", C.c_int32), ("refit_inflate", C.c_float),
                ("seed_max_hits", C.c_int32), ("chi2_merge", C.c_float),
                ("split_scale", C.c_float), ("single_row_scale", C.c_float),
                ("single_time_scale", C.c_float), ("edge_scale", C.c_float)]


class tpc_calib(C.Structure):
    _fields_ = [("vdrift", C.c_double), ("t0", C.c_double), ("spline", C.c_void_p),
                ("spl_x0", C.c_float), ("spl_dx", C.c_float)]


class tpc_clusters(C.Structure):
    _fields_ = [("n", C.c_int64), ("mode", C.c_int32), ("n_events", C.c_int32),
                ("tf_start", C.c_double), ("y", C.c_void_p), ("z", C.c_void_p),
                ("t", C.c_void_p), ("row", C.c_void_p), ("sector", C.c_void_p),
                ("flags", C.c_void_p), ("event", C.c_void_p), ("pads", C.c_int32)]


class tpc_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double)]


class tpc_tuning(C.Structure):
    _fields_ = [("grid_tau", C.c_float), ("grid_ny_max", C.c_int32),
                ("tracklet_block", C.c_int32), ("tracklet_per_sm", C.c_int32),
                ("tracklet_regs", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class tpc_tracks(C.Structure):
    _fields_ = [("n_tracks", C.c_int64), ("n_assigned", C.c_int64),
                ("track_start", C.c_void_p), ("cluster_idx", C.c_void_p),
                ("t_coll", C.c_void_p), ("start_hit", C.c_void_p)]


_PROTOS = {
    "tpc_default_params": (None, [C.POINTER(tpc_params)]),
    "tpc_create": (C.c_int, [C.POINTER(tpc_geometry), C.POINTER(tpc_params), C.c_void_p,
                             C.POINTER(C.c_void_p)]),
    "tpc_destroy": (None, [C.c_void_p]),
    "tpc_get_tuning": (C.c_int, [C.c_void_p, C.POINTER(tpc_tuning)]),
    "tpc_profile_only": (C.c_int, [C.c_void_p, C.c_char_p]),
    "tpc_set_tuning": (C.c_int, [C.c_void_p, C.POINTER(tpc_tuning)]),
    "tpc_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(tpc_tuning)]),
    "tpc_set_calib": (C.c_int, [C.c_void_p, C.POINTER(tpc_calib)]),
    "tpc_load_clusters": (C.c_int, [C.c_void_p, C.POINTER(tpc_clusters)]),
    "tpc_find_tracks": (C.c_int, [C.c_void_p, C.POINTER(tpc_tracks)]),
    "tpc_find_tracks_async": (C.c_int, [C.c_void_p]),
    "tpc_find_tracks_batched": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32,
                                          C.POINTER(tpc_tracks)]),
    "tpc_set_tracks": (C.c_int, [C.c_void_p, C.POINTER(tpc_tracks)]),
    "tpc_get_tracks": (C.c_int, [C.c_void_p, C.POINTER(tpc_tracks)]),
    "tpc_refit": (C.c_int, [C.c_void_p, C.c_int] + [C.c_void_p] * 7),
    "tpc_refit_backward": (C.c_int, [C.c_void_p] + [C.c_void_p] * 4),
    "tpc_set_vertex": (C.c_int, [C.c_void_p, C.c_void_p, C.c_float]),
    "tpc_merge_tracks": (C.c_int, [C.c_void_p] + [C.c_void_p] * 6 + [C.POINTER(tpc_tracks)]),
    "tpc_merge_tracks_async": (C.c_int, [C.c_void_p] + [C.c_void_p] * 6),
    "tpc_refine_time": (C.c_int, [C.c_void_p] + [C.c_void_p] * 4),
    "tpc_compress_tracks": (C.c_int, [C.c_void_p, C.c_float, C.c_float] + [C.c_void_p] * 4),
    "tpc_sync": (C.c_int, [C.c_void_p]),
    "tpc_get_counts": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int64)]),
    "tpc_get_links": (C.c_int, [C.c_void_p] + [C.c_void_p] * 4),
    "tpc_get_tracklets": (C.c_int, [C.c_void_p, C.c_int64] + [C.c_void_p] * 4),
    "tpc_get_calibrated": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "tpc_get_grid": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "tpc_last_error": (C.c_char_p, [C.c_void_p]),
    "tpc_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "tpc_graph_begin": (C.c_int, [C.c_void_p]),
    "tpc_graph_end": (C.c_int, [C.c_void_p]),
    "tpc_graph_launch": (C.c_int, [C.c_void_p]),
    "tpc_refit_noalloc": (C.c_int, [C.POINTER(tpc_geometry), C.POINTER(tpc_params), C.c_void_p,
                                    C.c_int64, C.c_int64] + [C.c_void_p] * 10),
    "tpc_profile_read": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int64)]),
}

_lib = None


def declared_functions():
    """Names of the functions include/tpc.h declares."""
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:tpc_status|void|const char\*)\s+(tpc_\w+)\s*\(",
                                 src, re.M)))


def load_library(path=LIB_PATH):
    """Load libtpc.so; raises if it has not been built (no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with python -m paper_1811_11481_b300.build")
    L = C.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def default_params_struct():
    p = tpc_params()
    load_library().tpc_default_params(C.byref(p))
    return p


def params_struct(d):
    p = tpc_params()
    for name, _ in tpc_params._fields_:
        v = d[name]
        if name in ("c0t", "c0r"):
            setattr(p, name, (C.c_float * 5)(*[float(x) for x in v]))
        else:
            setattr(p, name, v)
    return p


class Tracker:
    """One library context bound to the current CUDA device and torch stream."""

    def __init__(self, geo, params=None, stream=None, field=None):
        import torch
        self.torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("libtpc needs a CUDA device")
        self.L = load_library()
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream or torch.cuda.current_stream()
        self.row_x = np.ascontiguousarray(geo.row_x, np.float32)
        self.n_rows = int(self.row_x.size)
        fp = lambda a: a.ctypes.data_as(C.POINTER(C.c_float)) if a is not None else None
        self.pad_w = (np.ascontiguousarray(geo.pad_width, np.float32)
                      if getattr(geo, "pad_width", None) is not None else None)
        self.pad_c = (np.ascontiguousarray(geo.pad_center, np.float32)
                      if getattr(geo, "pad_center", None) is not None else None)
        self.field = (np.ascontiguousarray(field, np.float32).reshape(-1)
                      if field is not None else None)
        g = tpc_geometry(self.n_rows, fp(self.row_x), float(geo.tan_half),
                         float(geo.drift_length), float(geo.bz), fp(self.pad_w), fp(self.pad_c),
                         fp(self.field))
        p = params_struct(params) if params is not None else None
        h = C.c_void_p()
        st = self.L.tpc_create(C.byref(g), C.byref(p) if p is not None else None,
                               C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != 0:
            raise TpcError(st, "tpc_create")
        self.h = h
        self._keep = {}
        self.n = 0
        self.n_tracks = None
        self.n_assigned = None

    def close(self):
        if getattr(self, "h", None):
            self.L.tpc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st, what):
        if st != 0:
            raise TpcError(st, f"{what}: {self.L.tpc_last_error(self.h).decode()}")

    # ----------------------------------------------------------- inputs
    def set_calib(self, vdrift=2.58, t0=0.0, spline=None, spl_x0=85.0, spl_dx=160.0):
        torch = self.torch
        sp = None
        if spline is not None:
            sp = torch.as_tensor(np.asarray(spline, np.float32).reshape(-1)
                                 if not isinstance(spline, torch.Tensor) else spline,
                                 device=self.dev).float().contiguous()
            assert sp.numel() == TPC_SPLINE_SIZE
        self._keep["spline"] = sp
        c = tpc_calib(float(vdrift), float(t0), sp.data_ptr() if sp is not None else None,
                      float(spl_x0), float(spl_dx))
        self._ck(self.L.tpc_set_calib(self.h, C.byref(c)), "tpc_set_calib")

    def upload(self, ev, pads=False):
        """Copy an event's cluster arrays to device tensors; with pads, the
        native pad positions (ev.pad) take the place of y."""
        torch = self.torch
        d = dict(mode=0 if ev.mode == "event" else 1, n_events=int(ev.n_events),
                 tf_start=float(ev.tf_start), pads=1 if pads else 0)
        d["y"] = torch.as_tensor(np.ascontiguousarray(ev.pad if pads else ev.y, np.float32),
                                 device=self.dev)
        d["z"] = (torch.as_tensor(np.ascontiguousarray(ev.z, np.float32), device=self.dev)
                  if d["mode"] == 0 else None)
        d["t"] = (torch.as_tensor(np.ascontiguousarray(ev.t, np.float64), device=self.dev)
                  if d["mode"] == 1 else None)
        for k in ("row", "sector", "flags"):
            d[k] = torch.as_tensor(np.ascontiguousarray(getattr(ev, k), np.uint8), device=self.dev)
        d["event"] = torch.as_tensor(np.ascontiguousarray(ev.event, np.int32).view(np.int32),
                                     device=self.dev)
        return d

    def load(self, cl):
        """cl: dict of device tensors (y, z or t, row, sector, flags, event) + mode,
        n_events, tf_start. The tensors are kept alive until the next load."""
        self._keep["clusters"] = cl
        n = int(cl["y"].numel())
        s = tpc_clusters(n, int(cl["mode"]), int(cl.get("n_events", 1)),
                         float(cl.get("tf_start", 0.0)), cl["y"].data_ptr(),
                         cl["z"].data_ptr() if cl.get("z") is not None else None,
                         cl["t"].data_ptr() if cl.get("t") is not None else None,
                         cl["row"].data_ptr(), cl["sector"].data_ptr(),
                         cl["flags"].data_ptr() if cl.get("flags") is not None else None,
                         cl["event"].data_ptr() if cl.get("event") is not None else None,
                         int(cl.get("pads", 0)))
        self.n = n
        self._ck(self.L.tpc_load_clusters(self.h, C.byref(s)), "tpc_load_clusters")
        self.n_tracks = None

    # ----------------------------------------------------------- finding
    def find(self):
        """Run the finder; returns the track CSR as torch tensors (copies)."""
        torch = self.torch
        t = tpc_tracks()
        self._ck(self.L.tpc_find_tracks(self.h, C.byref(t)), "tpc_find_tracks")
        self.n_tracks, self.n_assigned = int(t.n_tracks), int(t.n_assigned)
        view = self._tracks_view(t)
        self.cluster_idx = view["cluster_idx"]
        return view

    def find_batched(self, parts):
        """Load several cluster sets (dicts as returned by upload) as one
        batch, concatenated in order, and run the finder; returns the track
        CSR in the concatenated cluster numbering (copies)."""
        arr = (tpc_clusters * len(parts))()
        for i, cl in enumerate(parts):
            arr[i] = tpc_clusters(
                int(cl["y"].numel()), int(cl["mode"]), int(cl.get("n_events", 1)),
                float(cl.get("tf_start", 0.0)), cl["y"].data_ptr(),
                cl["z"].data_ptr() if cl.get("z") is not None else None,
                cl["t"].data_ptr() if cl.get("t") is not None else None,
                cl["row"].data_ptr(), cl["sector"].data_ptr(),
                cl["flags"].data_ptr() if cl.get("flags") is not None else None,
                cl["event"].data_ptr() if cl.get("event") is not None else None,
                int(cl.get("pads", 0)))
        t = tpc_tracks()
        self._ck(self.L.tpc_find_tracks_batched(self.h, C.cast(arr, C.c_void_p), len(parts),
                                                C.byref(t)), "tpc_find_tracks_batched")
        self._keep["clusters"] = None
        self.n = sum(int(cl["y"].numel()) for cl in parts)
        self.n_tracks, self.n_assigned = int(t.n_tracks), int(t.n_assigned)
        view = self._tracks_view(t)
        self.cluster_idx = view["cluster_idx"]
        return view

    def find_async(self):
        self._ck(self.L.tpc_find_tracks_async(self.h), "tpc_find_tracks_async")
        self.n_tracks = None

    def counts(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        self._ck(self.L.tpc_get_counts(self.h, C.byref(a), C.byref(b), C.byref(c)),
                 "tpc_get_counts")
        self.n_tracks, self.n_assigned = a.value, b.value
        return a.value, b.value, c.value

    def _tracks_view(self, t):
        torch = self.torch
        nt, na = int(t.n_tracks), int(t.n_assigned)
        out = dict(track_start=torch.empty(nt + 1, dtype=torch.int32, device=self.dev),
                   cluster_idx=torch.empty(max(na, 1), dtype=torch.int32, device=self.dev)[:na],
                   t_coll=torch.empty(max(nt, 1), dtype=torch.float64, device=self.dev)[:nt],
                   start_hit=torch.empty(max(nt, 1), dtype=torch.int32, device=self.dev)[:nt])
        cu = torch.cuda
        for key, src, nbytes in (("track_start", t.track_start, 4 * (nt + 1)),
                                 ("cluster_idx", t.cluster_idx, 4 * na),
                                 ("t_coll", t.t_coll, 8 * nt),
                                 ("start_hit", t.start_hit, 4 * nt)):
            if nbytes:
                _memcpy_d2d(out[key].data_ptr(), src, nbytes, self.stream)
        return out

    def tracks(self):
        """The context's current track set (copies)."""
        t = tpc_tracks()
        self._ck(self.L.tpc_get_tracks(self.h, C.byref(t)), "tpc_get_tracks")
        self.n_tracks, self.n_assigned = int(t.n_tracks), int(t.n_assigned)
        return self._tracks_view(t)

    def set_tracks(self, track_start, cluster_idx, t_coll, start_hit=None):
        ts = track_start.to(self.dev, self.torch.int32).contiguous()
        ci = cluster_idx.to(self.dev, self.torch.int32).contiguous()
        tc = t_coll.to(self.dev, self.torch.float64).contiguous()
        sh = start_hit.to(self.dev, self.torch.int32).contiguous() if start_hit is not None else None
        self._keep["tracks"] = (ts, ci, tc, sh)
        t = tpc_tracks(ts.numel() - 1, ci.numel(), ts.data_ptr(), ci.data_ptr(), tc.data_ptr(),
                       sh.data_ptr() if sh is not None else None)
        self._ck(self.L.tpc_set_tracks(self.h, C.byref(t)), "tpc_set_tracks")
        self.n_tracks, self.n_assigned = int(t.n_tracks), int(t.n_assigned)
        self.cluster_idx = ci

    # ----------------------------------------------------------- refit
    def refit(self, save_for_backward=False, n_tracks=None, n_assigned=None):
        torch = self.torch
        nt = self.n_tracks if n_tracks is None else n_tracks
        na = self.n_assigned if n_assigned is None else n_assigned
        if nt is None:
            nt, na, _ = self.counts()
        f = lambda *s: torch.empty(*s, dtype=torch.float32, device=self.dev)
        out = dict(params=f(max(nt, 1), 5), cov=f(max(nt, 1), 15), x=f(max(nt, 1)),
                   chi2=f(max(nt, 1)),
                   ndf=torch.empty(max(nt, 1), dtype=torch.int32, device=self.dev),
                   status=torch.empty(max(nt, 1), dtype=torch.int32, device=self.dev),
                   rej=torch.empty(max(na, 1), dtype=torch.uint8, device=self.dev))
        self._ck(self.L.tpc_refit(self.h, int(bool(save_for_backward)), _ptr(out["params"]),
                                  _ptr(out["cov"]), _ptr(out["x"]), _ptr(out["chi2"]),
                                  _ptr(out["ndf"]), _ptr(out["status"]), _ptr(out["rej"])),
                 "tpc_refit")
        for k in ("params", "cov", "x", "chi2", "ndf", "status"):
            out[k] = out[k][:nt]
        out["rej"] = out["rej"][:na]
        return out

    def set_vertex(self, z_vertex, sigma=0.01):
        """Vertex pseudo-measurements (device float32 tensor [n_tracks], NaN =
        none) for the refits of the current track set; None switches them
        off. The tensor is kept alive here until the next call."""
        if z_vertex is None:
            self._keep["vertex"] = None
            self._ck(self.L.tpc_set_vertex(self.h, None, 0.0), "tpc_set_vertex")
            return
        z = z_vertex.to(self.dev, self.torch.float32).contiguous()
        self._keep["vertex"] = z
        self._ck(self.L.tpc_set_vertex(self.h, _ptr(z), float(sigma)), "tpc_set_vertex")

    def refit_backward(self, dl_dchi2):
        torch = self.torch
        na = self.n_assigned
        g = dl_dchi2.to(self.dev, torch.float32).contiguous()
        gy = torch.empty(max(na, 1), dtype=torch.float32, device=self.dev)
        gz = torch.empty(max(na, 1), dtype=torch.float32, device=self.dev)
        gc = torch.empty(TPC_GRAD_CALIB_SIZE, dtype=torch.float64, device=self.dev)
        self._ck(self.L.tpc_refit_backward(self.h, _ptr(g), _ptr(gy), _ptr(gz), _ptr(gc)),
                 "tpc_refit_backward")
        return gy[:na], gz[:na], gc

    # ----------------------------------------------------------- merging
    def merge(self, seg):
        """Merge the current track set (sector segments) using their refit
        outputs seg (params, cov, x, status as returned by refit); the merged
        tracks become the track set. Returns next (continuation of each
        segment or -1) and link_chi2 as tensors."""
        torch = self.torch
        nt = int(seg["status"].numel())
        nx = torch.empty(max(nt, 1), dtype=torch.int32, device=self.dev)
        lc = torch.empty(max(nt, 1), dtype=torch.float32, device=self.dev)
        c = lambda k, dt: seg[k].to(self.dev, dt).contiguous()
        ins = (c("params", torch.float32), c("cov", torch.float32), c("x", torch.float32),
               c("status", torch.int32))
        t = tpc_tracks()
        self._ck(self.L.tpc_merge_tracks(self.h, *[_ptr(a) for a in ins], _ptr(nx), _ptr(lc),
                                         C.byref(t)), "tpc_merge_tracks")
        self.n_tracks, self.n_assigned = int(t.n_tracks), int(t.n_assigned)
        self._merged_view = self._tracks_view(t)
        self.cluster_idx = self._merged_view["cluster_idx"]
        return dict(next=nx[:nt], link_chi2=lc[:nt], tracks=self._merged_view)

    def merge_async(self, seg, next_out=None, link_chi2=None):
        """tpc_merge_tracks_async: no synchronisation, counts stay on the
        device (counts() reads them). seg: refit outputs of the segments."""
        torch = self.torch
        c = lambda k, dt: seg[k].to(self.dev, dt).contiguous()
        ins = (c("params", torch.float32), c("cov", torch.float32), c("x", torch.float32),
               c("status", torch.int32))
        self._keep["merge"] = ins
        self._ck(self.L.tpc_merge_tracks_async(self.h, *[_ptr(a) for a in ins], _ptr(next_out),
                                               _ptr(link_chi2)), "tpc_merge_tracks_async")
        self.n_tracks = None

    def compress(self, qy=0.01, qz=0.01):
        """Track-model residuals (ry, rz) and decoded clusters (dy, dz) of the
        current track set, per assigned cluster in track order."""
        torch = self.torch
        na = self.n_assigned if self.n_assigned is not None else self.counts()[1]
        i32 = lambda: torch.empty(max(na, 1), dtype=torch.int32, device=self.dev)
        f32 = lambda: torch.empty(max(na, 1), dtype=torch.float32, device=self.dev)
        out = dict(ry=i32(), rz=i32(), dy=f32(), dz=f32())
        self._ck(self.L.tpc_compress_tracks(self.h, float(qy), float(qz), _ptr(out["ry"]),
                                            _ptr(out["rz"]), _ptr(out["dy"]), _ptr(out["dz"])),
                 "tpc_compress_tracks")
        return {k: v[:na] for k, v in out.items()}

    def refine_time(self, fit):
        """Refine the collision times of the current track set from its refit
        outputs fit (params, x, status); returns the times."""
        torch = self.torch
        nt = int(fit["status"].numel())
        out = torch.empty(max(nt, 1), dtype=torch.float64, device=self.dev)
        c = lambda k, dt: fit[k].to(self.dev, dt).contiguous()
        ins = (c("params", torch.float32), c("x", torch.float32), c("status", torch.int32))
        self._keep["refine"] = ins
        self._ck(self.L.tpc_refine_time(self.h, *[_ptr(a) for a in ins], _ptr(out)),
                 "tpc_refine_time")
        return out[:nt]

    def sync(self):
        self._ck(self.L.tpc_sync(self.h), "tpc_sync")

    # ----------------------------------------------------------- graphs
    def graph_begin(self):
        self._ck(self.L.tpc_graph_begin(self.h), "tpc_graph_begin")

    def graph_end(self):
        self._ck(self.L.tpc_graph_end(self.h), "tpc_graph_end")

    def graph_launch(self):
        self._ck(self.L.tpc_graph_launch(self.h), "tpc_graph_launch")

    # ----------------------------------------------------------- accounting
    def profile(self, enable=True):
        """Reset kernel accounting; with enable, time every kernel with events."""
        self._ck(self.L.tpc_profile(self.h, int(bool(enable))), "tpc_profile")

    def profile_only(self, kernel=None):
        """Time only the launches of `kernel` (None: every kernel)."""
        self._ck(self.L.tpc_profile_only(self.h, kernel.encode() if kernel else None),
                 "tpc_profile_only")

    def profile_read(self):
        """{kernel: (launches, total_ms)} and the total launch count."""
        buf = (tpc_kernel_stat * 64)()
        n = C.c_int32()
        tot = C.c_int64()
        self._ck(self.L.tpc_profile_read(self.h, buf, 64, C.byref(n), C.byref(tot)),
                 "tpc_profile_read")
        return ({buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms))
                 for i in range(min(n.value, 64))}, int(tot.value))

    # ----------------------------------------------------------- tuning
    def get_tuning(self):
        t = tpc_tuning()
        self._ck(self.L.tpc_get_tuning(self.h, C.byref(t)), "tpc_get_tuning")
        return t.as_dict()

    def set_tuning(self, **kw):
        t = tpc_tuning(**{**self.get_tuning(), **kw})
        self._ck(self.L.tpc_set_tuning(self.h, C.byref(t)), "tpc_set_tuning")

    def autotune(self, repeats=3):
        """Search launch shapes on the loaded batch; returns the chosen tuning."""
        t = tpc_tuning()
        self._ck(self.L.tpc_autotune(self.h, int(repeats), C.byref(t)), "tpc_autotune")
        return t.as_dict()

    # ----------------------------------------------------------- introspection
    def links(self):
        torch = self.torch
        o = [torch.empty(max(self.n, 1), dtype=torch.int32, device=self.dev) for _ in range(4)]
        self._ck(self.L.tpc_get_links(self.h, *[_ptr(t) for t in o]), "tpc_get_links")
        return [t[:self.n] for t in o]

    def tracklets(self):
        torch = self.torch
        _, _, ntl = self.counts()
        m = max(ntl, 1)
        sh = torch.empty(m, dtype=torch.int32, device=self.dev)
        nh = torch.empty(m, dtype=torch.int32, device=self.dev)
        th = torch.empty(m, dtype=torch.float64, device=self.dev)
        hits = torch.empty(m, self.n_rows, dtype=torch.int32, device=self.dev)
        self._ck(self.L.tpc_get_tracklets(self.h, ntl, _ptr(sh), _ptr(nh), _ptr(th), _ptr(hits)),
                 "tpc_get_tracklets")
        return dict(start_hit=sh[:ntl], nh=nh[:ntl], that=th[:ntl], hits=hits[:ntl])

    def calibrated(self):
        torch = self.torch
        na = self.n_assigned if self.n_assigned is not None else self.counts()[1]
        yc = torch.empty(max(na, 1), dtype=torch.float32, device=self.dev)
        zc = torch.empty(max(na, 1), dtype=torch.float32, device=self.dev)
        self._ck(self.L.tpc_get_calibrated(self.h, _ptr(yc), _ptr(zc)), "tpc_get_calibrated")
        return yc[:na], zc[:na]

    def grid(self, n_events=1):
        torch = self.torch
        K = n_events * 36 * self.n_rows
        order = torch.empty(max(self.n, 1), dtype=torch.int32, device=self.dev)
        rs = torch.empty(K + 1, dtype=torch.int32, device=self.dev)
        self._ck(self.L.tpc_get_grid(self.h, _ptr(order), _ptr(rs)), "tpc_get_grid")
        return order[:self.n], rs


def _memcpy_d2d(dst, src, nbytes, stream):
    """Device-to-device copy on the given torch stream (via torch)."""
    import torch
    src_t = _wrap_ptr(src, nbytes)
    dst_t = _wrap_ptr(dst, nbytes)
    with torch.cuda.stream(stream):
        dst_t.copy_(src_t, non_blocking=True)


def _wrap_ptr(ptr, nbytes):
    """A uint8 torch tensor viewing nbytes of device memory at ptr (no ownership)."""
    import torch

    class _CAI:
        def __init__(self, p, n):
            self.__cuda_array_interface__ = dict(shape=(n,), typestr="|u1", data=(p, False),
                                                 version=3, strides=None)
    return torch.as_tensor(_CAI(int(ptr), int(nbytes)))
