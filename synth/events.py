"""Synthetic ALICE-TPC-like events, seeded, as flat structure-of-arrays.

Geometry (Sec. 2, Fig. 2 caption of the paper): 36 trapezoidal sectors, 18 in
azimuth on each side of the central electrode, 152 pad rows. The row radii,
drift length and field are not given in the paper; the values used here are
85-245 cm (uniform), 250 cm and Bz = 0.5 T.

Every helix starts at the beam line (x = y = 0, z = z_v). In the global frame
its transverse projection is a circle through the origin; the generator finds
the arc length at which it crosses each sector's pad-row plane in closed form
and records one cluster per crossing that lies inside the sector acceptance
and inside |z| <= L. Particles that reach the outer radius leave the detector;
particles whose diameter is smaller than the outer radius loop for up to two
turns (Sec. 4, low-pT loopers).

Continuous readout (Sec. 4): in time-frame mode a cluster carries the absolute
drift time t = t_coll + t0 + (L - |z|) / v_drift as float64 microseconds
instead of z.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.interpolate as si

C_LIGHT = 2.99792458e-3  # curvature [1/cm] per (q/pT [1/GeV]) per Tesla

N_SECTORS = 36
N_ROWS = 152
SPLINE_N = 8  # control points per axis of the distortion spline


@dataclass
class Geometry:
    row_x: np.ndarray            # float32[152], plane positions in cm
    tan_half: np.float32         # tan(10 deg) as float32
    drift_length: np.float32     # L, cm
    bz: np.float32               # Tesla
    n_sectors: int = N_SECTORS
    n_rows: int = N_ROWS
    pad_width: np.ndarray | None = None   # float32[152] pad pitch (cm)
    pad_center: np.ndarray | None = None  # float32[152] pad position of y = 0

    @property
    def tan_half64(self) -> float:
        return float(self.tan_half)


def geometry() -> Geometry:
    r = np.arange(N_ROWS, dtype=np.float64)
    row_x = (85.0 + r * 160.0 / 151.0).astype(np.float32)
    tan_half = np.float32(math.tan(math.pi / 18.0))
    # native pads: 4 mm pitch on the inner 63 rows, 6 mm outside; pad 0 at the
    # sector's lower edge, so y = 0 lies at ceil(x tan(10 deg) / pitch)
    pad_width = np.where(r < 63, 0.4, 0.6).astype(np.float32)
    pad_center = np.ceil(row_x.astype(np.float64) * float(tan_half) /
                         pad_width).astype(np.float32)
    return Geometry(row_x=row_x, tan_half=tan_half, drift_length=np.float32(250.0),
                    bz=np.float32(0.5), pad_width=pad_width, pad_center=pad_center)


def pad_positions(geo: Geometry, y, row):
    """Native pad positions (pads, continuous) of local y (cm) on the rows."""
    row = np.asarray(row, np.int64)
    return (np.asarray(y, np.float64) / geo.pad_width[row] + geo.pad_center[row]).astype(
        np.float32)


def sector_alpha(k):
    """Rotation angle of sector k's local frame (sectors k and k+18 share it)."""
    return ((np.asarray(k) % 18) + 0.5) * (math.pi / 9.0)


def sector_side(k):
    return np.where(np.asarray(k) < 18, 1.0, -1.0)


@dataclass
class Calib:
    vdrift: float = 2.58          # cm / us
    t0: float = 0.0               # us
    spline: np.ndarray = field(default_factory=lambda: np.zeros(
        (N_SECTORS, 2, SPLINE_N, SPLINE_N, SPLINE_N), np.float32))
    # spline[sector][component (0: dy, 1: dz)][iw (|z|)][iv (y/x)][iu (x)]

    def copy(self) -> "Calib":
        return Calib(self.vdrift, self.t0, self.spline.copy())


def nominal_calib() -> Calib:
    return Calib()


@dataclass
class Event:
    """Clusters (SoA, float32 coordinates) plus Monte-Carlo truth."""
    mode: str                     # "event" (z given) or "time" (t given)
    y: np.ndarray                 # float32
    z: np.ndarray | None          # float32 (event mode)
    t: np.ndarray | None          # float64 (time mode), microseconds
    row: np.ndarray               # uint8
    sector: np.ndarray            # uint8
    flags: np.ndarray             # uint8
    event: np.ndarray             # uint32 event index inside a batch
    tf_start: float               # time-frame start, us (time mode)
    n_events: int
    calib_true: Calib
    # truth
    label: np.ndarray             # int32 particle id, -1 for noise
    segment: np.ndarray           # int64 id of (particle, sector, leg), -1 noise
    y_true: np.ndarray            # float64 local y on the helix
    z_true: np.ndarray            # float64 global z on the helix
    s_true: np.ndarray            # float64 sin(phi) in the fitter convention
    tl_true: np.ndarray           # float64 tan(lambda) in the fitter convention
    q_true: np.ndarray            # float64 q/pT in the fitter convention
    t_coll: np.ndarray            # float64 per particle collision time
    part: dict                    # per-particle arrays
    info: dict = field(default_factory=dict)
    pad: np.ndarray | None = None  # float32 native pad positions of y

    @property
    def n(self) -> int:
        return int(self.y.shape[0])


# ---------------------------------------------------------------------------
# particles
# ---------------------------------------------------------------------------

def gen_particles_single_sector(rng, n, sector=0, bz=0.5):
    """Helices whose azimuth at mid radius (165 cm) is uniform in the sector."""
    a = sector_alpha(sector)
    half = math.pi / 18.0
    pt = 0.1 + rng.exponential(0.5, n)
    q = rng.choice([-1.0, 1.0], n)
    kap = C_LIGHT * bz * q / pt
    bend = np.sign(kap) * np.arcsin(np.minimum(1.0, 165.0 * np.abs(kap) / 2.0))
    return dict(
        pt=pt,
        phi0=a + rng.uniform(-half, half, n) + bend,
        eta=rng.uniform(0.05, 0.9, n),
        q=q,
        zv=np.zeros(n),
    )


def gen_particles_central(rng, n, zv_spread=5.0, pmin=0.05, index=19.0 / 9.0,
                          pmax=50.0):
    # Pareto pT spectrum with pdf ~ pT^-index above pmin (mean 0.5 GeV)
    pt = pmin * rng.uniform(0.0, 1.0, n) ** (-1.0 / (index - 1.0))
    pt = np.minimum(pt, pmax)
    return dict(
        pt=pt,
        phi0=rng.uniform(0.0, 2.0 * math.pi, n),
        eta=rng.uniform(-0.9, 0.9, n),
        q=rng.choice([-1.0, 1.0], n),
        zv=rng.uniform(-zv_spread, zv_spread, n),
    )


def _concat_parts(parts):
    keys = parts[0].keys()
    return {k: np.concatenate([p[k] for p in parts]) for k in keys}


# ---------------------------------------------------------------------------
# helix / pad-row crossings in the global frame
# ---------------------------------------------------------------------------

def _crossings(geo: Geometry, p: dict, chunk=4000):
    """All (particle, sector, row, leg) crossings inside the acceptance."""
    kB = C_LIGHT * float(geo.bz)
    L = float(geo.drift_length)
    tanA = math.tan(math.pi / 18.0)
    row_x = geo.row_x.astype(np.float64)
    rho_in = float(row_x[0])
    rho_out = float(row_x[-1]) / math.cos(math.pi / 18.0) + 1.0
    sw = math.pi / 9.0

    pt, phi0, q = p["pt"], p["phi0"], p["q"]
    tanl = np.sinh(p["eta"])
    kap = kB * q / pt
    ak = np.abs(kap)
    lo = np.arcsin(np.minimum(1.0, rho_in * ak / 2.0))
    loops = 2.0 / ak < rho_out
    hi = np.where(loops, math.pi - lo, np.arcsin(np.minimum(1.0, rho_out * ak / 2.0)))
    sg = np.sign(kap)
    a1 = phi0 - sg * lo
    a2 = phi0 - sg * hi
    amin = np.minimum(a1, a2) - 0.01
    amax = np.maximum(a1, a2) + 0.01
    klo = np.floor(amin / sw).astype(np.int64)
    khi = np.floor(amax / sw).astype(np.int64)
    nk = np.minimum(khi - klo + 1, 18)
    # arc length at which the particle leaves through the outer radius
    l_exit = np.where(loops, np.inf,
                      2.0 * np.arcsin(np.minimum(1.0, rho_out * ak / 2.0)) / ak)

    out = []
    ip_all = np.repeat(np.arange(pt.shape[0]), nk)
    off = np.concatenate([np.arange(v) for v in nk]) if len(nk) else np.zeros(0, np.int64)
    ks_all = np.mod(np.repeat(klo, nk) + off, 18)
    for c0 in range(0, ip_all.shape[0], chunk):
        ip = ip_all[c0:c0 + chunk][:, None, None, None]
        ks = ks_all[c0:c0 + chunk][:, None, None, None]
        al = (ks + 0.5) * sw
        xr = row_x[None, :, None, None]
        br = np.arange(2)[None, None, :, None]
        turn = np.arange(2)[None, None, None, :]
        kp = kap[ip]
        f0 = phi0[ip]
        w = kp * xr - np.sin(f0 - al)
        ok = np.abs(w) <= 1.0
        ws = np.clip(w, -1.0, 1.0)
        asw = np.arcsin(ws)
        psi = np.where(br == 0, al - asw, al - math.pi + asw)
        dlt = f0 - psi
        two_pi = 2.0 * math.pi
        dm = np.where(kp > 0, np.mod(dlt, two_pi), -np.mod(-dlt, two_pi))
        period = two_pi / np.abs(kp)
        larc = dm / kp + turn * period
        half = 0.5 * dm
        s_half = np.sin(half) / kp
        X = 2.0 * np.cos(f0 - half) * s_half
        Y = 2.0 * np.sin(f0 - half) * s_half
        ylo = -X * np.sin(al) + Y * np.cos(al)
        Z = p["zv"][ip] + tanl[ip] * larc
        ok = ok & (np.abs(ylo) <= xr * tanA) & (np.abs(Z) <= L)
        ok = ok & (larc >= 0.0) & (larc <= l_exit[ip])
        idx = np.nonzero(ok)
        if idx[0].size == 0:
            continue
        b = np.broadcast_to(br, ok.shape)[idx]
        tt = np.broadcast_to(turn, ok.shape)[idx]
        ipp = np.broadcast_to(ip, ok.shape)[idx]
        kk = np.broadcast_to(ks, ok.shape)[idx]
        rr = np.broadcast_to(np.arange(N_ROWS)[None, :, None, None], ok.shape)[idx]
        Zs = np.broadcast_to(Z, ok.shape)[idx]
        sec = kk + 18 * (Zs < 0.0)
        wv = np.broadcast_to(w, ok.shape)[idx]
        sgn = np.where(b == 0, 1.0, -1.0)
        out.append(dict(
            ip=ipp, sector=sec, row=rr, y=np.broadcast_to(ylo, ok.shape)[idx], z=Zs,
            s=np.where(b == 0, -wv, wv),
            tl=sgn * tanl[ipp], qpt=sgn * q[ipp] / pt[ipp],
            leg=2 * tt + b, larc=np.broadcast_to(larc, ok.shape)[idx],
        ))
    if not out:
        z0 = np.zeros(0)
        return dict(ip=z0.astype(np.int64), sector=z0.astype(np.int64),
                    row=z0.astype(np.int64), y=z0, z=z0, s=z0, tl=z0, qpt=z0,
                    leg=z0.astype(np.int64), larc=z0)
    return {k: np.concatenate([o[k] for o in out]) for k in out[0]}


# ---------------------------------------------------------------------------
# distortion spline (scipy tensor-product B-spline, independent evaluator)
# ---------------------------------------------------------------------------

def _knots():
    return (np.arange(SPLINE_N + 4, dtype=np.float64) - 3.0) / (SPLINE_N - 3)


def _spline_args(geo, x, y, az):
    tanA = float(geo.tan_half)
    u = np.clip((x - 85.0) / 160.0, 0.0, 1.0)
    v = np.clip((y / x + tanA) / (2.0 * tanA), 0.0, 1.0)
    w = np.clip(az / float(geo.drift_length), 0.0, 1.0)
    return u, v, w


def eval_distortion(geo, spline, sector, x, y, az):
    """(dy, dz) of the distortion spline; scipy NdBSpline evaluation."""
    u, v, w = _spline_args(geo, x, y, az)
    t = _knots()
    out = np.zeros((2, x.shape[0]))
    for k in np.unique(sector):
        m = sector == k
        pts = np.stack([w[m], v[m], u[m]], axis=1)
        for c in range(2):
            coef = spline[k, c].astype(np.float64)
            if not np.any(coef):
                continue
            bs = si.NdBSpline((t, t, t), coef, 3, extrapolate=False)
            out[c, m] = bs(pts)
    return out[0], out[1]


def random_distortion(rng, max_abs=1.0):
    """Per-sector coefficients U(-1, 1) scaled so that max |Delta| <= max_abs."""
    c = rng.uniform(-1.0, 1.0, (N_SECTORS, 2, SPLINE_N, SPLINE_N, SPLINE_N))
    c *= max_abs / np.max(np.abs(c))
    return c.astype(np.float32)


# ---------------------------------------------------------------------------
# assembling events
# ---------------------------------------------------------------------------

def make_event(rng, geo: Geometry, parts: list, mode="event", t_colls=None,
               noise_frac=0.0, calib: Calib | None = None, sigma=0.1,
               tf_start=0.0, keep_sectors=None, event_ids=None,
               distortion_iters=8, field=None):
    """Build one batch of clusters.

    parts: list of particle dicts, one per collision (event).
    t_colls: collision time per collision (time mode).
    event_ids: batch-event index per collision (default: all 0).
    field: coefficients [3][10] of a non-uniform field (synth/field.py):
    particles are traced through it (outgoing legs only) instead of
    intersecting helices in the uniform geo.bz.
    """
    calib = calib or nominal_calib()
    ncol = len(parts)
    if t_colls is None:
        t_colls = np.zeros(ncol)
    if event_ids is None:
        event_ids = np.zeros(ncol, np.int64)
    sizes = [len(p["pt"]) for p in parts]
    allp = _concat_parts(parts)
    col_of = np.repeat(np.arange(ncol), sizes)
    allp["t_coll"] = np.asarray(t_colls, np.float64)[col_of]
    allp["event"] = np.asarray(event_ids)[col_of]
    if field is None:
        cr = _crossings(geo, allp)
    else:
        from .field import crossings_in_field
        cr = crossings_in_field(geo, allp, field)
    if keep_sectors is not None:
        m = np.isin(cr["sector"], np.asarray(keep_sectors))
        cr = {k: v[m] for k, v in cr.items()}
    n_sig = cr["y"].shape[0]
    L = float(geo.drift_length)
    x_sig = geo.row_x.astype(np.float64)[cr["row"]]
    y_t = cr["y"] + sigma * rng.standard_normal(n_sig)
    z_t = cr["z"] + sigma * rng.standard_normal(n_sig)
    side = sector_side(cr["sector"])
    # distortion: measured m with m + Delta(m) = smeared true position
    y_m, z_m = y_t.copy(), z_t.copy()
    if np.any(calib.spline):
        for _ in range(distortion_iters):
            dy, dz = eval_distortion(geo, calib.spline, cr["sector"], x_sig, y_m,
                                     np.abs(z_m))
            y_m = y_t - dy
            z_m = z_t - dz
    ev_of = allp["event"][cr["ip"]]
    tc_of = allp["t_coll"][cr["ip"]]

    # noise clusters
    n_noise = int(round(noise_frac * n_sig))
    if keep_sectors is not None:
        nsec = rng.choice(np.asarray(keep_sectors), n_noise)
    else:
        nsec = rng.integers(0, N_SECTORS, n_noise)
    nrow = rng.integers(0, N_ROWS, n_noise)
    nx = geo.row_x.astype(np.float64)[nrow]
    tanA = float(geo.tan_half)
    ny = rng.uniform(-1.0, 1.0, n_noise) * nx * tanA
    nside = sector_side(nsec)
    nev = rng.integers(0, max(1, int(np.max(event_ids)) + 1), n_noise)
    if mode == "event":
        nz = nside * rng.uniform(0.0, L, n_noise)
        nt = None
    else:
        tmin = float(np.min(t_colls)) if ncol else tf_start
        tmax = float(np.max(t_colls)) + L / calib.vdrift if ncol else tf_start
        nt = rng.uniform(tmin, tmax, n_noise) + calib.t0
        nz = None

    y = np.concatenate([y_m, ny]).astype(np.float32)
    row = np.concatenate([cr["row"], nrow]).astype(np.uint8)
    sector = np.concatenate([cr["sector"], nsec]).astype(np.uint8)
    event = np.concatenate([ev_of, nev]).astype(np.uint32)
    if mode == "event":
        z = np.concatenate([z_m, nz]).astype(np.float32)
        t = None
    else:
        t_sig = tc_of + calib.t0 + (L - side * z_m) / calib.vdrift
        t = np.concatenate([t_sig, nt]).astype(np.float64)
        z = None
    nn = n_noise
    seg = (cr["ip"].astype(np.int64) * N_SECTORS + cr["sector"]) * 4 + cr["leg"]
    return Event(
        mode=mode, y=y, z=z, t=t, row=row, sector=sector,
        flags=np.zeros(n_sig + nn, np.uint8), event=event, tf_start=tf_start,
        n_events=int(np.max(event_ids)) + 1 if ncol else 1,
        calib_true=calib.copy(),
        label=np.concatenate([cr["ip"], -np.ones(nn, np.int64)]).astype(np.int32),
        segment=np.concatenate([seg, -np.ones(nn, np.int64)]),
        y_true=np.concatenate([cr["y"], np.full(nn, np.nan)]),
        z_true=np.concatenate([cr["z"], np.full(nn, np.nan)]),
        s_true=np.concatenate([cr["s"], np.full(nn, np.nan)]),
        tl_true=np.concatenate([cr["tl"], np.full(nn, np.nan)]),
        q_true=np.concatenate([cr["qpt"], np.full(nn, np.nan)]),
        t_coll=allp["t_coll"], part=allp, pad=pad_positions(geo, y, row),
        info=dict(n_signal=n_sig, n_noise=nn, sigma=sigma,
                  larc=np.concatenate([cr["larc"], np.full(nn, np.nan)]),
                  z_meas=np.concatenate([z_m, np.full(nn, np.nan)]),
                  y_meas=np.concatenate([y_m, np.full(nn, np.nan)])),
    )


def truth_tracks(ev: Event, min_hits=40, merged=False):
    """Truth-assigned tracks: one per (particle, sector, leg) segment, or with
    merged=True one per (particle, leg, side) across sectors.

    Returns CSR (track_start uint32[n+1], cluster_idx uint32[...], clusters in
    increasing row order -- for merged tracks: along the path, rows
    increasing), the collision time per track and the segment (or merged
    track) ids.
    """
    if merged:
        return _truth_tracks_merged(ev, min_hits)
    sig = np.nonzero(ev.segment >= 0)[0]
    seg = ev.segment[sig]
    order = np.lexsort((ev.row[sig], seg))
    sig = sig[order]
    seg = seg[order]
    if sig.size == 0:
        return (np.zeros(1, np.uint32), np.zeros(0, np.uint32), np.zeros(0),
                np.zeros(0, np.int64))
    starts = np.concatenate([[0], np.nonzero(np.diff(seg))[0] + 1, [seg.size]])
    lens = np.diff(starts)
    keep = lens >= min_hits
    ts, ci, tc, sids = [0], [], [], []
    for a, b, k in zip(starts[:-1], starts[1:], keep):
        if not k:
            continue
        idx = sig[a:b]
        ci.append(idx)
        ts.append(ts[-1] + idx.size)
        tc.append(ev.t_coll[ev.label[idx[0]]])
        sids.append(seg[a])
    return (np.asarray(ts, np.uint32),
            np.concatenate(ci).astype(np.uint32) if ci else np.zeros(0, np.uint32),
            np.asarray(tc, np.float64), np.asarray(sids, np.int64))


def _truth_tracks_merged(ev: Event, min_hits):
    sig = np.nonzero(ev.segment >= 0)[0]
    seg = ev.segment[sig]
    leg = seg % 4
    side = (ev.sector[sig] >= 18).astype(np.int64)
    mid = (ev.label[sig].astype(np.int64) * 4 + leg) * 2 + side
    # along the path: outgoing branches (even leg) cross the rows outward,
    # incoming ones inward; order so that rows increase
    larc = ev.info["larc"][sig]
    key2 = np.where(leg % 2 == 0, larc, -larc)
    order = np.lexsort((key2, mid))
    sig, mid = sig[order], mid[order]
    if sig.size == 0:
        return (np.zeros(1, np.uint32), np.zeros(0, np.uint32), np.zeros(0),
                np.zeros(0, np.int64))
    starts = np.concatenate([[0], np.nonzero(np.diff(mid))[0] + 1, [mid.size]])
    ts, ci, tc, ids = [0], [], [], []
    for a, b in zip(starts[:-1], starts[1:]):
        if b - a < min_hits:
            continue
        idx = sig[a:b]
        if np.any(np.diff(ev.row[idx].astype(np.int64)) < 0):
            idx = idx[np.argsort(ev.row[idx], kind="stable")]
        ci.append(idx)
        ts.append(ts[-1] + idx.size)
        tc.append(ev.t_coll[ev.label[idx[0]]])
        ids.append(mid[a])
    return (np.asarray(ts, np.uint32),
            np.concatenate(ci).astype(np.uint32) if ci else np.zeros(0, np.uint32),
            np.asarray(tc, np.float64), np.asarray(ids, np.int64))


# ---------------------------------------------------------------------------
# the workload configurations
# ---------------------------------------------------------------------------

def make_single_sector(seed=0, n_tracks=200):
    """Single sector, 200 helices from the origin, no noise, event mode."""
    rng = np.random.default_rng(seed)
    geo = geometry()
    p = gen_particles_single_sector(rng, n_tracks, sector=0)
    return make_event(rng, geo, [p], mode="event", keep_sectors=[0])


def make_central(seed=1, n_tracks=10000, noise_frac=0.10, field=None):
    """One central Pb-Pb-like event: 36 sectors, 10k primaries, 10% noise
    (with field: traced through that non-uniform field, outgoing legs)."""
    rng = np.random.default_rng(seed)
    geo = geometry()
    p = gen_particles_central(rng, n_tracks)
    return make_event(rng, geo, [p], mode="event", noise_frac=noise_frac, field=field)


def make_timeframe(seed=2, n_coll=50, mean_mult=2000, rate_khz=50.0,
                   noise_frac=0.15, tf_start=1.0e6, calib=None):
    """Continuous-readout time frame of overlapping collisions (time mode)."""
    rng = np.random.default_rng(seed)
    geo = geometry()
    calib = calib or nominal_calib()
    gaps = rng.exponential(1000.0 / rate_khz, n_coll)
    t_colls = tf_start + np.cumsum(gaps)
    mult = np.maximum(1, np.round(rng.exponential(mean_mult, n_coll))).astype(int)
    parts = [gen_particles_central(rng, m) for m in mult]
    ev = make_event(rng, geo, parts, mode="time", t_colls=t_colls,
                    noise_frac=noise_frac, calib=calib, tf_start=tf_start)
    ev.info["t_colls"] = t_colls
    ev.info["mult"] = mult
    return ev


def make_batched(seed=3, n_events=64, lo=20, hi=10000, noise_frac=0.10):
    """Many events of uneven size (log-uniform track counts), one batch."""
    rng = np.random.default_rng(seed)
    geo = geometry()
    mult = np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), n_events))).astype(int)
    parts = [gen_particles_central(rng, m) for m in mult]
    ev = make_event(rng, geo, parts, mode="event", noise_frac=noise_frac,
                    event_ids=np.arange(n_events))
    ev.info["mult"] = mult
    return ev


def make_adjoint(seed=4, n_events=10, n_tracks=10000, tf_start=1.0e6,
                 spacing_us=200.0):
    """Calibration-recovery workload.

    Ten central events in time mode, generated with the TRUE calibration
    (v_drift +0.5 %, t0 +0.05 us, a per-sector distortion spline with
    max |Delta| <= 1 cm); reconstruction starts from the nominal calibration.
    """
    rng = np.random.default_rng(seed)
    geo = geometry()
    nom = nominal_calib()
    true = Calib(vdrift=nom.vdrift * 1.005, t0=nom.t0 + 0.05,
                 spline=random_distortion(rng, 1.0))
    t_colls = tf_start + spacing_us * (1.0 + np.arange(n_events))
    parts = [gen_particles_central(rng, n_tracks) for _ in range(n_events)]
    ev = make_event(rng, geo, parts, mode="time", t_colls=t_colls,
                    noise_frac=0.0, calib=true, tf_start=tf_start)
    ev.info["t_colls"] = t_colls
    return ev


def make_tiny(seed=5, n_tracks=20, sectors=(0,), noise_frac=0.0, mode="event",
              central=False, calib=None, tf_start=0.0, n_coll=1, sigma=0.1, field=None,
              pt=None):
    """Small cases for tests: a few tracks in chosen sectors. pt (GeV/c):
    give every particle this transverse momentum (pt=1000: tracks straight
    to 5e-3 cm over the rows, for a tracker run without field)."""
    rng = np.random.default_rng(seed)
    geo = geometry()
    parts = []
    for _ in range(n_coll):
        if central:
            parts.append(gen_particles_central(rng, n_tracks))
        else:
            ps = [gen_particles_single_sector(rng, max(1, n_tracks // len(sectors)),
                                              sector=s % 18) for s in sectors]
            pp = _concat_parts(ps)
            if any(s >= 18 for s in sectors):
                flip = np.isin(np.arange(len(pp["eta"])) % len(sectors),
                               [i for i, s in enumerate(sectors) if s >= 18])
                pp["eta"] = np.where(flip, -pp["eta"], pp["eta"])
            parts.append(pp)
        if pt is not None:
            parts[-1]["pt"] = np.full_like(parts[-1]["pt"], float(pt))
    t_colls = tf_start + 10.0 * (1.0 + np.arange(n_coll)) if mode == "time" else None
    ev = make_event(rng, geo, parts, mode=mode, t_colls=t_colls,
                    noise_frac=noise_frac, calib=calib, tf_start=tf_start,
                    keep_sectors=None if central else list(sectors), sigma=sigma,
                    field=field)
    return ev


CONFIGS = {
    "single_sector": make_single_sector,
    "central": make_central,
    "timeframe": make_timeframe,
    "batched": make_batched,
    "adjoint": make_adjoint,
}


def make_config(name, **kw):
    return CONFIGS[name](**kw)
