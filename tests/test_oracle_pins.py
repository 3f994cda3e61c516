"""Pins of the CPU oracle against references that are not the oracle itself.

Each test checks one piece of the oracle against something independent: the
generator's global-frame helix (closed-form circle/plane intersection),
central finite differences, the information form of the Kalman update
(numpy.linalg), scipy's B-spline and least-squares routines, closed forms
and brute-force constructions whose answer is known.
"""
import math

import numpy as np
import pytest
import scipy.optimize as so
import scipy.stats as st

import oracle
import synth
from synth.events import eval_distortion

KB = 2.99792458e-3 * 0.5


def _oracle(ev, geo, params, calib=None, **kw):
    return oracle.Oracle(ev, geo, params, calib or synth.nominal_calib(), **kw)


# ---------------------------------------------------------------- arc length
@pytest.mark.parametrize("prec,rtol", [(64, 2e-15), (32, 6e-7)])
def test_arc_factor_matches_asin(prec, rtol):
    for h in np.concatenate([np.linspace(-0.999, 0.999, 401), [1e-9, -1e-6, 0.124999, 0.125, 0.5]]):
        ref = math.asin(h) / h
        assert abs(oracle.arc_factor(h, prec) - ref) <= rtol * ref, h


@pytest.mark.parametrize("prec,rtol", [(64, 1e-8), (32, 2e-4)])
def test_arc_derivative_is_derivative(prec, rtol):
    # B(h) = d/dh [asin(h)/h]; compare with a central difference of asin(h)/h
    for h in np.linspace(-0.95, 0.95, 77):
        e = 1e-5
        fd = (math.asin(h + e) / (h + e) - math.asin(h - e) / (h - e)) / (2 * e) if abs(h) > 2e-5 else 0.0
        b = oracle.arc_deriv(h, prec)
        assert abs(b - fd) <= rtol * max(abs(fd), 1e-3), (h, b, fd)


# ------------------------------------------------------ helix propagation
def test_propagation_matches_generator_helix(geo, params):
    ev = synth.make_tiny(seed=11, n_tracks=60, sectors=(0, 7, 20), sigma=0.0)
    o = _oracle(ev, geo, params)
    seg = ev.segment
    checked = 0
    worst = np.zeros(5)
    for s in np.unique(seg[seg >= 0]):
        idx = np.nonzero(seg == s)[0]
        idx = idx[np.argsort(ev.row[idx])]
        if idx.size < 20 or np.max(np.abs(ev.s_true[idx])) >= params["s_max"]:
            continue
        a, b = idx[0], idx[-1]
        for (i, j) in [(a, b), (b, a), (idx[3], idx[4])]:
            s0 = [ev.y_true[i], ev.z_true[i], ev.s_true[i], ev.tl_true[i], ev.q_true[i]]
            out, _ = o.propagate(s0, geo.row_x[ev.row[i]], geo.row_x[ev.row[j]])
            assert out is not None
            ref = [ev.y_true[j], ev.z_true[j], ev.s_true[j], ev.tl_true[j], ev.q_true[j]]
            worst = np.maximum(worst, np.abs(out - ref))
            checked += 1
    assert checked > 50
    assert worst[0] < 1e-9 and worst[1] < 1e-9, worst
    assert worst[2] < 1e-12 and worst[3] == 0 and worst[4] == 0, worst


def test_jacobian_matches_finite_differences(geo, params):
    ev = synth.make_tiny(seed=12, n_tracks=4)
    o = _oracle(ev, geo, params)
    rng = np.random.default_rng(0)
    for _ in range(40):
        s0 = np.array([rng.uniform(-5, 5), rng.uniform(-50, 50), rng.uniform(-0.6, 0.6),
                       rng.uniform(-1, 1), rng.uniform(-8, 8)])
        x1 = rng.uniform(85, 245)
        x2 = x1 + rng.choice([-1, 1]) * rng.uniform(0.5, 8)
        out, J = o.jacobian(s0, x1, x2)
        if out is None:
            continue
        for k in range(5):
            e = 1e-6 * max(1.0, abs(s0[k]))
            sp = s0.copy(); sp[k] += e
            sm = s0.copy(); sm[k] -= e
            op, _ = o.jacobian(sp, x1, x2)
            om, _ = o.jacobian(sm, x1, x2)
            fd = (op - om) / (2 * e)
            np.testing.assert_allclose(J[:, k], fd, rtol=1e-6, atol=1e-8)


def test_covariance_transport_is_JCJt(geo, params):
    ev = synth.make_tiny(seed=12, n_tracks=4)
    o = _oracle(ev, geo, params)
    rng = np.random.default_rng(1)
    A = rng.normal(size=(5, 5))
    C = A @ A.T + np.eye(5)
    s0 = np.array([1.0, 20.0, 0.2, 0.3, 2.0])
    out, J = o.jacobian(s0, 100.0, 103.0)
    out2, C2 = o.propagate(s0, 100.0, 103.0, C)
    np.testing.assert_allclose(out2, out, rtol=0, atol=0)
    np.testing.assert_allclose(C2, J @ C @ J.T, rtol=1e-13, atol=1e-13)


# ----------------------------------------------------------- Kalman update
def test_update_equals_information_form():
    rng = np.random.default_rng(2)
    H = np.zeros((2, 5)); H[0, 0] = 1; H[1, 1] = 1
    for _ in range(20):
        A = rng.normal(size=(5, 5))
        C = A @ A.T + 0.1 * np.eye(5)
        p = rng.normal(size=5)
        m = rng.normal(size=2)
        V = np.diag(rng.uniform(0.005, 0.05, 2))
        p2, C2, chi2 = oracle.Oracle.update(p, C, m[0], m[1], V[0, 0], V[1, 1])
        Ci = np.linalg.inv(C)
        Cn = np.linalg.inv(Ci + H.T @ np.linalg.inv(V) @ H)
        pn = Cn @ (Ci @ p + H.T @ np.linalg.inv(V) @ m)
        r = m - H @ p
        S = H @ C @ H.T + V
        np.testing.assert_allclose(p2, pn, rtol=1e-9, atol=1e-10)
        np.testing.assert_allclose(C2, Cn, rtol=1e-8, atol=1e-10)
        assert abs(chi2 - r @ np.linalg.solve(S, r)) < 1e-10 * max(1, chi2)


# --------------------------------------------------------------- the refit
def _truth_refit(ev, geo, params, min_hits=40, prec=64):
    ts, ci, tc, sids = synth.truth_tracks(ev, min_hits)
    o = _oracle(ev, geo, params)
    r = o.refit(ts, ci, np.zeros(ts.size - 1), prec=prec)
    inner = ci[ts[:-1]]
    return o, ts, ci, r, inner


def test_noise_free_refit_returns_generating_helix(geo, params):
    ev = synth.make_tiny(seed=13, n_tracks=80, sectors=(0, 9), sigma=0.0)
    o, ts, ci, r, inner = _truth_refit(ev, geo, params)
    ok = r["status"] == 0
    assert ok.sum() >= 50
    truth = np.stack([ev.y_true, ev.z_true, ev.s_true, ev.tl_true, ev.q_true], 1)[inner]
    np.testing.assert_allclose(r["x"][ok], geo.row_x[ev.row[inner]][ok].astype(np.float64))
    d = np.abs(r["params"][ok] - truth[ok])
    # clusters are float32: compare with the helix through the rounded points
    assert np.max(d[:, 0]) < 2e-5 and np.max(d[:, 1]) < 2e-5, np.max(d, 0)
    assert np.max(d[:, 2]) < 1e-6 and np.max(d[:, 3]) < 1e-6
    assert np.max(d[:, 4] / np.abs(truth[ok, 4])) < 2e-4
    assert np.all(r["rej"] == 0)


def test_refit_of_exact_points_is_exact(geo, params):
    """Float64 points exactly on a generated helix refit to it within 1e-9."""
    ev = synth.make_tiny(seed=14, n_tracks=40, sectors=(0,), sigma=0.0)
    o = _oracle(ev, geo, params)
    ts, ci, tc, sids = synth.truth_tracks(ev, 60)
    n = 0
    for k in range(ts.size - 1):
        idx = ci[ts[k]:ts[k + 1]]
        if np.max(np.abs(ev.s_true[idx])) > 0.9:
            continue
        x = geo.row_x[ev.row[idx]].astype(np.float64)
        stt, p, chi2, ndf = o.refit_points(x, ev.y_true[idx], ev.z_true[idx], 0.01)
        assert stt == 0
        i = idx[0]
        truth = np.array([ev.y_true[i], ev.z_true[i], ev.s_true[i], ev.tl_true[i], ev.q_true[i]])
        assert np.all(np.abs(p - truth) < 1e-9 * np.array([1, 1, 1, 1, max(1, abs(truth[4]))])), (
            p - truth)
        assert chi2 < 1e-12 and ndf == 2 * idx.size
        n += 1
    assert n >= 10


def test_zero_field_refit_of_a_straight_line_is_exact(geo, params):
    """The degenerate case Bz = 0 (straight tracks, q/pT not observable, held
    at 0): float64 points on straight lines refit to the line within 1e-9."""
    import dataclasses
    geo0 = dataclasses.replace(geo, bz=np.float32(0.0))
    o = _oracle(synth.make_tiny(seed=14, n_tracks=4, sectors=(0,), sigma=0.0), geo0, params)
    rng = np.random.default_rng(21)
    x = geo.row_x.astype(np.float64)
    for _ in range(10):
        s, t = rng.uniform(-0.3, 0.3), rng.uniform(-1.0, 1.0)
        y0, z0 = rng.uniform(-5.0, 5.0), rng.uniform(-100.0, 100.0)
        c = np.sqrt(1.0 - s * s)
        y = y0 + (x - x[0]) * (s / c)
        z = z0 + (x - x[0]) * (t / c)
        stt, p, chi2, ndf = o.refit_points(x, y, z, 0.01)
        assert stt == 0
        assert np.all(np.abs(p - np.array([y0, z0, s, t, 0.0])) < 1e-9), p
        assert p[4] == 0.0 and chi2 < 1e-12 and ndf == 2 * x.size


def _helix_at_planes(p, x0, xs, kB=KB):
    """Independent helix model: circle through (x0, y0) with direction phi,
    curvature kB*q, intersected with planes x = xs; z advances with arc length."""
    y0, z0, s, t, q = p
    kap = kB * q
    c = math.sqrt(1 - s * s)
    if abs(kap) < 1e-12:
        ys = y0 + (xs - x0) * s / c
        ls = (xs - x0) / c
        return ys, z0 + t * ls
    # centre of curvature: clockwise for kap > 0
    xc, yc = x0 + s / kap, y0 - c / kap
    R = 1 / abs(kap)
    dx = xs - xc
    dy = np.sqrt(R * R - dx * dx)
    # branch continuous with the start point
    sgn = np.sign(y0 - yc)
    ys = yc + sgn * dy
    ang0 = math.atan2(y0 - yc, x0 - xc)
    ang = np.arctan2(ys - yc, xs - xc)
    dang = np.angle(np.exp(1j * (ang0 - ang)))  # clockwise positive for kap>0
    ls = dang / kap
    return ys, z0 + t * ls


def _ls_fit(geo, e, idx, p_start, sigma=0.1):
    x = geo.row_x[e.row[idx]].astype(np.float64)
    y = e.y[idx].astype(np.float64)
    z = e.z[idx].astype(np.float64)
    x0 = x[0]

    def res(p):
        yy, zz = _helix_at_planes(p, x0, x)
        return np.concatenate([(yy - y) / sigma, (zz - z) / sigma])
    sol = so.least_squares(res, p_start, xtol=1e-15, ftol=1e-15, gtol=1e-15,
                           x_scale=np.array([0.1, 0.1, 1e-3, 1e-3, 1e-2]))
    return sol.x


def test_refit_agrees_with_least_squares(geo, params):
    """Pass 3 of the refit (Sec. 3) starts from pass 2's state with its
    covariance inflated; its result is the extended Kalman filter's estimate
    of the minimum of chi2 over the clusters plus that starting state as a
    pseudo-measurement. Against Gauss-Newton on the same objective with an
    independent helix model (scipy), on helices with sigma = 0.1 cm: within
    1e-3 sigma in the median and 2e-2 sigma at most (the filter linearises at
    its running estimate once, which leaves ~1e-2 sigma on the most curved of
    40 tracks; without the pseudo-measurement the two differ by up to ~3 % of
    sigma, which is the prior's weight, not an error)."""
    ev = synth.make_tiny(seed=15, n_tracks=40, sectors=(0,))
    ts, ci, tc, sids = synth.truth_tracks(ev, 50)
    o = _oracle(ev, geo, params)
    dev = []
    for k in range(ts.size - 1):
        idx = ci[ts[k]:ts[k + 1]]
        xs = geo.row_x[ev.row[idx]].astype(np.float64)
        ys, zs = ev.y[idx].astype(np.float64), ev.z[idx].astype(np.float64)
        stt, p, chi2, ndf, pri, C = o.refit_points(xs, ys, zs, 0.01, details=True)
        if stt != 0 or ndf != 2 * xs.size:
            continue
        pr = pri[2]
        L = np.linalg.cholesky(np.linalg.inv(pr["C"]))

        def res(q):
            yy, zz = _helix_at_planes(q, xs[0], xs)
            yn, zn = _helix_at_planes(q, xs[0], np.array([pr["x"]]))
            sn = q[2] - KB * q[4] * (pr["x"] - xs[0])
            d = np.array([yn[0], zn[0], sn, q[3], q[4]]) - pr["p"]
            return np.concatenate([(yy - ys) / 0.1, (zz - zs) / 0.1, L.T @ d])
        sol = so.least_squares(res, p, xtol=1e-15, ftol=1e-15, gtol=1e-15,
                               x_scale=np.array([0.1, 0.1, 1e-3, 1e-3, 1e-2]))
        dev.append(np.abs(p - sol.x) / np.sqrt(np.diag(C)))
    dev = np.array(dev)
    assert dev.shape[0] >= 15
    assert np.all(dev < 2e-2), dev.max(0)
    assert np.all(np.median(dev, 0) < 1e-3), np.median(dev, 0)


def test_zero_field_refit_is_least_squares_with_the_priors(geo, params):
    """Information-filter identity (Sec. 3 refit, no field): for tracks on
    the sector's centre line (y = 0, so sin(phi) stays 0 and the transport
    is linear in (z, tan(lambda)); with sin(phi) != 0 it is not linear even
    without a field), each pass equals weighted linear least squares of the
    noisy z measurements with the state the pass starts from (the seed with
    the prior covariance C0 in pass 1, then the previous pass's state with
    its inflated covariance) as a pseudo-measurement: state, covariance and
    chi2 to 1e-12 relative."""
    import dataclasses
    geo0 = dataclasses.replace(geo, bz=np.float32(0.0))
    o = _oracle(synth.make_tiny(seed=14, n_tracks=4, sectors=(0,), sigma=0.0), geo0, params)
    rng = np.random.default_rng(5)
    x = geo.row_x.astype(np.float64)
    sig = 0.1
    for _ in range(10):
        t, z0 = rng.uniform(-1, 1), rng.uniform(-100, 100)
        z = z0 + (x - x[0]) * t + rng.normal(0, sig, x.size)
        stt, p, chi2, ndf, pri, C = o.refit_points(x, np.zeros_like(x), z, sig * sig,
                                                   details=True)
        assert stt == 0 and ndf == 2 * x.size
        assert p[0] == 0.0 and p[2] == 0.0 and p[4] == 0.0
        # pass 1 starts from the seed with the prior covariance C0
        np.testing.assert_array_equal(np.diag(pri[0]["C"]), np.float32(params["c0r"]))
        for k, xr in enumerate((x[0], x[-1], x[0])):        # plane each pass ends at
            pr = pri[k]
            Pi = np.linalg.inv(pr["C"][np.ix_([1, 3], [1, 3])])
            F = np.array([[1.0, pr["x"] - xr], [0.0, 1.0]])  # (z, t) at xr -> prior plane
            H = np.stack([np.ones_like(x), x - xr], 1)
            A = H.T @ H / sig ** 2 + F.T @ Pi @ F
            sol = np.linalg.solve(A, H.T @ z / sig ** 2 + F.T @ Pi @ pr["p"][[1, 3]])
            if k < 2:   # the next pass starts from this one's state
                nxt = pri[k + 1]
                np.testing.assert_allclose(nxt["p"][[1, 3]], sol, rtol=1e-12, atol=1e-12)
                cov_next = nxt["C"][np.ix_([1, 3], [1, 3])] / params["refit_inflate"]
                np.testing.assert_allclose(cov_next, np.linalg.inv(A), rtol=1e-12)
        np.testing.assert_allclose(p[[1, 3]], sol, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(C[np.ix_([1, 3], [1, 3])], np.linalg.inv(A), rtol=1e-12)
        r = z - H @ sol
        d = F @ sol - pr["p"][[1, 3]]
        assert abs(chi2 - (r @ r / sig ** 2 + d @ Pi @ d)) <= 1e-12 * chi2


def test_joseph_form_equals_the_short_form(geo, params):
    """The Joseph form of the covariance update and the short form used by
    the refit are the same update in exact arithmetic: in float64 the refit
    of truth tracks gives the same parameters (1e-10) and covariances
    (1e-8); in float32 the Joseph form stays at least as close to float64."""
    ev = synth.make_tiny(seed=16, n_tracks=300, sectors=(0, 5, 19))
    ts, ci, tc, _ = synth.truth_tracks(ev, 40)
    o = _oracle(ev, geo, params)
    short64 = o.refit(ts, ci, tc, prec=64)
    short32 = o.refit(ts, ci, tc, prec=32, seeds=short64["seeds"])
    o.set_joseph(True)
    jos64 = o.refit(ts, ci, tc, prec=64, seeds=short64["seeds"])
    jos32 = o.refit(ts, ci, tc, prec=32, seeds=short64["seeds"])
    o.set_joseph(False)
    ok = (short64["status"] == 0) & (jos64["status"] == 0)
    assert ok.sum() > 100
    assert np.array_equal(short64["rej"], jos64["rej"])
    np.testing.assert_allclose(jos64["params"][ok], short64["params"][ok], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(jos64["cov"][ok], short64["cov"][ok], rtol=1e-8, atol=1e-14)
    np.testing.assert_allclose(jos64["chi2"][ok], short64["chi2"][ok], rtol=1e-10)
    ok32 = ok & (short32["status"] == 0) & (jos32["status"] == 0)
    e_s = np.abs(short32["params"][ok32] - short64["params"][ok32]).max(0)
    e_j = np.abs(jos32["params"][ok32] - short64["params"][ok32]).max(0)
    assert np.all(e_j <= 2.0 * e_s + 1e-7), (e_j, e_s)


def test_refit_pulls_and_chi2(geo, params):
    ev = synth.make_tiny(seed=16, n_tracks=600, sectors=(0, 5, 11, 19, 30))
    o, ts, ci, r, inner = _truth_refit(ev, geo, params, min_hits=40)
    ok = (r["status"] == 0)
    for k in np.nonzero(ok)[0]:
        if np.any(r["rej"][ts[k]:ts[k + 1]]):
            ok[k] = False
    truth = np.stack([ev.y_true, ev.z_true, ev.s_true, ev.tl_true, ev.q_true], 1)[inner]
    C = r["cov"]
    diag = C[:, [0, 2, 5, 9, 14]]
    pulls = (r["params"][ok] - truth[ok]) / np.sqrt(diag[ok])
    N = pulls.shape[0]
    assert N > 300
    m = pulls.mean(0)
    s = pulls.std(0)
    assert np.all(np.abs(m) < 4 / math.sqrt(N)), m
    assert np.all(np.abs(s - 1) < 4 / math.sqrt(2 * N)), s
    u = st.chi2.cdf(r["chi2"][ok], r["ndf"][ok] - 5)
    assert st.kstest(u, "uniform").pvalue > 1e-3


# ------------------------------------------------------------ time -> z
def test_time_to_z_round_trip(geo, params):
    ev = synth.make_tiny(seed=17, n_tracks=30, sectors=(0, 20), mode="time", tf_start=1.0e6,
                         n_coll=3)
    o = _oracle(ev, geo, params)
    sig = np.nonzero(ev.label >= 0)[0]
    tcoll = ev.t_coll[ev.label[sig]]
    yc, zc = o.calibrate(sig, tcoll, prec=64)
    assert np.max(np.abs(zc - ev.info["z_meas"][sig])) < 1e-9
    assert np.max(np.abs(yc - ev.y[sig])) == 0
    z32 = o.seed_z(32)
    z64 = o.seed_z(64)
    # the float32 seeding coordinate is the correctly rounded float64 one
    np.testing.assert_array_equal(z32, z64.astype(np.float32))
    # and equals the linear time scaling with the time-frame start as reference
    sg = np.where(ev.sector < 18, 1.0, -1.0)
    ref = sg * (250.0 - 2.58 * (ev.t - ev.tf_start))
    assert np.max(np.abs(z64 - ref)) < 1e-7


# --------------------------------------------------------------- spline
def test_spline_matches_scipy_bspline(geo, params):
    rng = np.random.default_rng(3)
    cal = synth.nominal_calib()
    cal.spline = synth.random_distortion(rng, 1.0)
    ev = synth.make_tiny(seed=18, n_tracks=2)
    o = _oracle(ev, geo, params, cal)
    m = 4000
    sec = rng.integers(0, 36, m)
    x = rng.uniform(85, 245, m)
    y = rng.uniform(-1, 1, m) * x * math.tan(math.pi / 18)
    az = rng.uniform(0, 250, m)
    dy, dz = o.spline(sec, x, y, az)
    ry, rz = eval_distortion(geo, cal.spline, sec, x, y, az)
    np.testing.assert_allclose(dy, ry, atol=1e-12)
    np.testing.assert_allclose(dz, rz, atol=1e-12)


def test_spline_partition_of_unity_and_linear_precision(geo, params):
    ev = synth.make_tiny(seed=18, n_tracks=2)
    cal = synth.nominal_calib()
    spl = np.zeros_like(cal.spline)
    spl[:, 0] = 1.0                                    # constant 1 in dy
    g = (np.arange(8) - 1.0) / 5.0                     # Greville abscissae
    spl[:, 1] = g[None, None, None, :]                 # dz = u (linear in x)
    cal.spline = spl.astype(np.float32)
    o = _oracle(ev, geo, params, cal)
    rng = np.random.default_rng(4)
    x = rng.uniform(85, 245, 500)
    y = rng.uniform(-0.15, 0.15, 500) * x
    az = rng.uniform(0, 250, 500)
    dy, dz = o.spline(np.zeros(500, np.int32), x, y, az)
    np.testing.assert_allclose(dy, 1.0, atol=1e-6)
    np.testing.assert_allclose(dz, (x - 85.0) / 160.0, atol=2e-7)


# ------------------------------------------------------------------ DCA
def test_dca_of_primary_helix_is_vertex(geo, params):
    ev = synth.make_tiny(seed=19, n_tracks=40, sectors=(0, 3), sigma=0.0, central=False)
    ev.part["zv"][:] = 0.0
    o = _oracle(ev, geo, params)
    rng = np.random.default_rng(5)
    first_leg = np.nonzero((ev.segment >= 0) & (ev.segment % 4 == 0))[0]
    for i in rng.choice(first_leg, 60, replace=False):
        s0 = [ev.y_true[i], ev.z_true[i], ev.s_true[i], ev.tl_true[i], ev.q_true[i]]
        zd = o.dca_z(s0, geo.row_x[ev.row[i]])
        zv = ev.part["zv"][ev.label[i]]
        assert abs(zd - zv) < 1e-6, (zd, zv)


# ------------------------------------------------------ neighbour finder
class _Mini:
    """Hand-built clusters in one sector."""

    def __init__(self, rows, ys, zs):
        self.mode = "event"
        self.row = np.asarray(rows, np.uint8)
        self.y = np.asarray(ys, np.float32)
        self.z = np.asarray(zs, np.float32)
        n = self.y.size
        self.sector = np.zeros(n, np.uint8)
        self.flags = np.zeros(n, np.uint8)
        self.event = np.zeros(n, np.uint32)
        self.n_events = 1
        self.tf_start = 0.0
        self.t = None


def test_neighbours_on_constructed_lines(geo, params):
    x = geo.row_x.astype(np.float64)
    # a straight line through rows 10, 11, 12 plus distractors in the outer rows
    ys = [2.0, 2.0 + 0.3 * (x[11] - x[10]), 2.0 + 0.3 * (x[12] - x[10]),
          2.0 + 0.3 * (x[12] - x[10]) + 0.4,  # displaced by 0.4 cm in y (D = 0.16)
          2.0 - 0.3 * (x[10] - x[9]) * 0 - 0.3 * (x[10] - x[9]),  # true continuation in row 9
          30.0]                                # far away
    zs = [10.0, 10.0 + 0.5 * (x[11] - x[10]), 10.0 + 0.5 * (x[12] - x[10]),
          10.0 + 0.5 * (x[12] - x[10]), 10.0 - 0.5 * (x[10] - x[9]), 10.0]
    rows = [10, 11, 12, 12, 9, 11]
    ev = _Mini(rows, ys, zs)
    o = _oracle(ev, geo, params)
    up, dn = o.neighbours(32)
    upd, dnd = o.neighbours(64)
    # hit 1 (row 11): down = 0, up = 2 (the exact line, not the displaced 3)
    assert (up[1], dn[1]) == (2, 0)
    # hit 0 (row 10): down = 4 (row 9), up = 1
    assert (up[0], dn[0]) == (1, 4)
    # row 12 and row 9 hits have no row on one side within reach -> no links
    assert up[2] == -1 and up[4] == -1
    # the far cluster has no neighbours
    assert up[5] == -1 and dn[5] == -1
    np.testing.assert_array_equal(up, upd)
    np.testing.assert_array_equal(dn, dnd)


def test_neighbours_prefer_smaller_deviation_and_respect_windows(geo, params):
    x = geo.row_x.astype(np.float64)
    h_y, h_z = 0.0, 0.0
    dxu, dxd = x[51] - x[50], x[50] - x[49]
    # two up candidates and two down candidates; pairs (u0,d0) exact, others off
    ys = [h_y, 0.0, 0.2, 0.0, 0.25, 0.0]
    zs = [h_z, 0.0, 0.0, 0.0, 0.0, dxu * params["nb_teta"] + params["nb_wz"] + 0.01]
    rows = [50, 51, 51, 49, 49, 51]
    ev = _Mini(rows, ys, zs)
    o = _oracle(ev, geo, params)
    up, dn = o.neighbours(32)
    assert (up[0], dn[0]) == (1, 3)
    # cluster 5 is outside the eta window of hit 0: never its up link
    assert up[0] != 5


def test_neighbour_tie_goes_to_lowest_pair(geo, params):
    # mirror-symmetric candidates give identical deviations
    ys = [0.0, 0.1, -0.1, 0.1, -0.1]
    zs = [0.0, 0.0, 0.0, 0.0, 0.0]
    rows = [60, 61, 61, 59, 59]
    ev = _Mini(rows, ys, zs)
    o = _oracle(ev, geo, params)
    up, dn = o.neighbours(32)
    # D(u=1, d=4) = D(u=2, d=3) exactly (symmetric); lowest pair (1, 4) wins
    assert (up[0], dn[0]) == (1, 4)


# ------------------------------------------------ CA invariants, end to end
def test_ca_invariants_and_efficiency_single_sector(geo, params):
    ev = synth.make_single_sector()
    o = _oracle(ev, geo, params)
    f = o.find(32)
    up, dn, upc, dnc = f["up"], f["dn"], f["upc"], f["dnc"]
    # every kept link is mutual and connects adjacent rows of one sector
    k = np.nonzero(upc >= 0)[0]
    assert np.all(dnc[upc[k]] == k)
    assert np.all(ev.row[upc[k]] == ev.row[k] + 1)
    # start hits are chain heads of chains with >= 3 hits
    s = f["starts"]
    assert np.all(dnc[s] < 0) and np.all(upc[s] >= 0) and np.all(upc[upc[s]] >= 0)
    tr = f["tracks"]
    ci = tr["cluster_idx"]
    assert np.unique(ci).size == ci.size, "a cluster is in two tracks"
    lens = np.diff(tr["track_start"].astype(np.int64))
    assert np.all(lens >= params["min_track_hits"])
    # tracks: clusters in increasing row order, one sector
    for a, b in zip(tr["track_start"][:-1], tr["track_start"][1:]):
        r = ev.row[ci[a:b]]
        assert np.all(np.diff(r.astype(int)) > 0)
    # the tracklet with the globally largest weight keeps all its hits
    tl = f["tracklets"]
    w = tl["nh"].astype(np.int64) * 2**32 + (2**32 - 1 - s)
    top = np.argmax(w)
    top_hits = tl["hits"][top][tl["hits"][top] >= 0]
    assert np.isin(top_hits, ci).all()
    # sanity bound on an isolated, noise-free sector
    seg = ev.segment
    from collections import Counter
    matched, fake = set(), 0
    for a, b in zip(tr["track_start"][:-1], tr["track_start"][1:]):
        c = Counter(seg[ci[a:b]])
        m, cnt = c.most_common(1)[0]
        if m < 0 or cnt < 0.9 * (b - a):
            fake += 1
        else:
            matched.add(m)
    cnt = Counter(seg[seg >= 0])
    findable = [q for q, c in cnt.items() if c >= 70]
    eff = np.mean([q in matched for q in findable])
    assert eff >= 0.99 and fake == 0, (eff, fake)


# ------------------------------------------------------------- adjoint
def test_gradient_matches_finite_differences(geo, params):
    rng = np.random.default_rng(6)
    cal = synth.nominal_calib()
    cal.spline = synth.random_distortion(rng, 0.5)
    ev = synth.make_tiny(seed=20, n_tracks=6, sectors=(2,), mode="time", tf_start=1.0e6,
                         calib=cal)
    ts, ci, tc, sids = synth.truth_tracks(ev, 40)
    nt = min(3, ts.size - 1)
    ts = ts[:nt + 1]
    ci = ci[:ts[-1]]
    tc = tc[:nt]
    o = _oracle(ev, geo, params, cal)
    r = o.refit(ts, ci, tc, prec=64)
    seeds, rej = r["seeds"], r["rej"]
    g = np.array([1.0, 0.7, 1.3])[:nt]
    gy, gz, gc = o.refit_grad(ts, ci, tc, seeds, rej, g)

    def loss(ev_mod=None, cal_mod=None):
        oo = _oracle(ev_mod or ev, geo, params, cal_mod or cal)
        rr = oo.refit(ts, ci, tc, prec=64, seeds=seeds, rej=rej)
        oo.close()
        return float(np.sum(g * rr["chi2"]))

    class Ev:
        pass

    def perturbed(field, i, e):
        E = Ev()
        for k in ("mode", "row", "sector", "flags", "event", "n_events", "tf_start", "z"):
            setattr(E, k, getattr(ev, k))
        E.y = ev.y.copy()
        E.t = ev.t.copy()
        getattr(E, field)[i] += e
        return E

    # cluster coordinates (y is float32 in storage: use a large step)
    for q in [0, 7, ts[1] + 3]:
        i = ci[q]
        ey = 1e-2
        fd = (loss(perturbed("y", i, ey)) - loss(perturbed("y", i, -ey))) / (2 * ey)
        assert abs(fd - gy[q]) < 2e-3 * max(1, abs(fd)), (q, fd, gy[q])
        et = 1e-5
        fd = (loss(perturbed("t", i, et)) - loss(perturbed("t", i, -et))) / (2 * et)
        assert abs(fd - gz[q]) < 1e-4 * max(1, abs(fd)), (q, fd, gz[q])
    # vdrift and t0
    for k, name, e in [(0, "vdrift", 1e-7), (1, "t0", 1e-6)]:
        cp, cm = cal.copy(), cal.copy()
        setattr(cp, name, getattr(cal, name) + e)
        setattr(cm, name, getattr(cal, name) - e)
        fd = (loss(cal_mod=cp) - loss(cal_mod=cm)) / (2 * e)
        assert abs(fd - gc[k]) < 1e-5 * max(1, abs(fd)), (name, fd, gc[k])
    # spline coefficients with the largest gradients
    flat = cal.spline.reshape(-1)
    for j in np.argsort(-np.abs(gc[2:]))[:4]:
        e = 1e-3
        cp, cm = cal.copy(), cal.copy()
        cp.spline.reshape(-1)[j] = flat[j] + e
        cm.spline.reshape(-1)[j] = flat[j] - e
        fd = (loss(cal_mod=cp) - loss(cal_mod=cm)) / (2 * e)
        assert abs(fd - gc[2 + j]) < 1e-3 * max(1, abs(fd)), (j, fd, gc[2 + j])


def test_spline_gradient_at_zero_coefficients(geo, params):
    """An all-zero spline adds nothing, but its coefficients have a gradient."""
    cal = synth.nominal_calib()
    ev = synth.make_tiny(seed=21, n_tracks=5, sectors=(3,), mode="time", tf_start=1.0e6)
    ts, ci, tc, sids = synth.truth_tracks(ev, 40)
    ts, ci, tc = ts[:3], ci[:ts[2]], tc[:2]
    o = _oracle(ev, geo, params, cal)
    r = o.refit(ts, ci, tc, prec=64)
    gy, gz, gc = o.refit_grad(ts, ci, tc, r["seeds"], r["rej"], np.ones(2))
    assert np.count_nonzero(gc[2:]) > 0
    for j in np.argsort(-np.abs(gc[2:]))[:3]:
        e = 1e-3
        losses = []
        for sgn in (1, -1):
            cm = cal.copy()
            cm.spline.reshape(-1)[j] = sgn * e
            oo = _oracle(ev, geo, params, cm)
            losses.append(float(np.sum(oo.refit(ts, ci, tc, prec=64, seeds=r["seeds"],
                                                 rej=r["rej"])["chi2"])))
        fd = (losses[0] - losses[1]) / (2 * e)
        assert abs(fd - gc[2 + j]) < 1e-3 * max(1, abs(fd)), (j, fd, gc[2 + j])


# ------------------------------------------------------ tracklet constructor
@pytest.mark.parametrize("mode", ["event", "time"])
def test_tracklets_match_python_reference(geo, params, mode):
    """The oracle's tracklet constructor against a second implementation of
    its steps (tests/tracklet_reference.py) on a small noisy event: hit
    tables, hit counts, collision times and final states."""
    import tracklet_reference
    calib = synth.nominal_calib()
    kw = dict(n_coll=3, tf_start=1.0e6) if mode == "time" else {}
    ev = synth.make_tiny(seed=41, n_tracks=40, sectors=(2, 25), noise_frac=0.3, mode=mode,
                         **kw)
    o = _oracle(ev, geo, params, calib)
    f = o.find(64)
    ref = tracklet_reference.tracklets(o, ev, geo, params, calib, f["upc"], f["starts"])
    tl = f["tracklets"]
    assert len(f["starts"]) > 40
    np.testing.assert_array_equal(tl["nh"], ref["nh"])
    np.testing.assert_array_equal(tl["hits"], ref["hits"])
    np.testing.assert_allclose(tl["that"], ref["that"], rtol=0, atol=1e-9)
    ok = ref["nh"] >= 0
    np.testing.assert_allclose(tl["x"][ok], ref["x"][ok], rtol=0, atol=1e-12)
    np.testing.assert_allclose(tl["state"][ok], ref["state"][ok], rtol=1e-12, atol=1e-12)


# ------------------------------------------- time -> z with calibration offsets
def test_time_to_z_round_trip_with_offsets(geo, params):
    """Drift velocity and t0 away from nominal: calibrated z from the true
    collision time equals the generator's z (Sec. 4 transform)."""
    cal = synth.nominal_calib()
    cal.vdrift *= 1.01
    cal.t0 = 0.07
    ev = synth.make_tiny(seed=19, n_tracks=30, sectors=(4, 30), mode="time", tf_start=1.0e6,
                         n_coll=2, calib=cal)
    o = _oracle(ev, geo, params, cal)
    sig = np.nonzero(ev.label >= 0)[0]
    yc, zc = o.calibrate(sig, ev.t_coll[ev.label[sig]], prec=64)
    assert np.max(np.abs(zc - ev.info["z_meas"][sig])) < 1e-9
    # a wrong t0 or drift velocity shows up in z
    o2 = _oracle(ev, geo, params, synth.nominal_calib())
    _, zc2 = o2.calibrate(sig, ev.t_coll[ev.label[sig]], prec=64)
    assert np.max(np.abs(zc2 - ev.info["z_meas"][sig])) > 0.1


# ----------------------------------------------------- refit outlier rules
def test_refit_rejection_follows_pass_order(geo, params):
    """Constructed outliers on a noise-free helix (Sec. 3): pass 1 runs inward
    from the outermost cluster and may reject only after min_acc_reject
    accepted clusters; pass 2 runs outward. A 1 cm (10 sigma) outlier third
    from the outer end is accepted by pass 1 (2 accepted before it) and
    rejected by pass 2; one at the sixth position of pass 1 (5 accepted
    before it) is rejected by pass 1; one at the fifth (4 before it) is
    accepted by pass 1 (it then drags the state, so that later clusters of
    pass 1 are rejected) and rejected by pass 2."""
    ev = synth.make_tiny(seed=23, n_tracks=6, sectors=(7,), sigma=0.0)
    ts, ci, tc, _ = synth.truth_tracks(ev, 60)
    o_plain = _oracle(ev, geo, params)
    r0 = o_plain.refit(ts, ci, tc, prec=64)
    k = int(np.nonzero(r0["status"] == 0)[0][0])      # a track that refits
    a, b = int(ts[k]), int(ts[k + 1])
    n = b - a
    one = (np.array([0, n], np.uint32), ci[a:b].copy(), tc[k:k + 1].copy())
    y = ev.y.copy()
    for pos, expect, alone in [(n - 3, 2, True), (n - 6, 1, True), (n - 5, 2, False)]:
        ev.y[:] = y
        ev.y[one[1][pos]] += np.float32(1.0)
        o = _oracle(ev, geo, params)
        r = o.refit(*one, prec=64)
        rej = r["rej"][:n]
        assert r["status"][0] == 0
        assert rej[pos] == expect, (pos, rej[pos], expect)
        if alone:
            assert np.count_nonzero(rej) == 1
    ev.y[:] = y
    assert np.count_nonzero(o_plain.refit(*one, prec=64)["rej"][:n]) == 0


def test_neighbour_deviation_cut_is_inclusive(geo, params):
    """A down hit exactly at the deviation cut (D = nb_dmax, exact in
    floating point) is linked; one just beyond is not."""
    assert params["nb_dmax"] == 0.5
    ys = [1.0, 1.0, 1.5, 1.0]
    zs = [10.0, 10.0, 10.5, 10.0]
    rows = [70, 71, 69, 72]
    o = _oracle(_Mini(rows, ys, zs), geo, params)
    up, dn = o.neighbours(32)
    # u straight above h: prediction (1.0, 10.0) in row 69, D = 0.25 + 0.25
    assert (up[0], dn[0]) == (1, 2)
    zs2 = [10.0, 10.0, 10.5 + 1e-3, 10.0]
    up2, dn2 = _oracle(_Mini(rows, ys, zs2), geo, params).neighbours(32)
    assert (up2[0], dn2[0]) == (-1, -1)


# ------------------------------------------------------------ selector rules
def test_selector_weights_and_gaps(geo, params):
    """Constructed tracklet tables with known answers (Sec. 3 shared
    clusters): a shared cluster goes to the tracklet with more hits, on equal
    hit counts to the lower start index; a track keeps at least
    min_track_hits clusters with no gap above max_gap rows."""
    R = geo.row_x.size
    nmin, gmax = params["min_track_hits"], params["max_gap"]
    ev = _Mini([5] * 200, [0.0] * 200, [0.0] * 200)
    o = _oracle(ev, geo, params)

    def table(rows_list):
        hits = -np.ones((len(rows_list), R), np.int32)
        for k, rs in enumerate(rows_list):
            for r, j in rs:
                hits[k, r] = j
        nh = np.array([len(rs) for rs in rows_list], np.int32)
        return dict(nh=nh, hits=hits, that=np.zeros(len(rows_list)))

    # A (start 7) and B (start 3), 12 hits each, sharing cluster 50 in row 20
    A = [(20 + i, 40 + i) for i in range(12)]          # clusters 40..51, 50 at row 30
    B = [(25 + i, 100 + i) for i in range(12)]
    B[5] = (30, 50)                                     # the shared cluster, same row
    tr = o.select(np.array([7, 3]), table([A, B]))
    lists = [list(tr["cluster_idx"][tr["track_start"][k]:tr["track_start"][k + 1]])
             for k in range(len(tr["track_start"]) - 1)]
    # equal hit counts: start 3 (B) wins cluster 50; A keeps 11 >= min hits
    assert 50 in lists[1] and 50 not in lists[0]
    # one more hit on A: A wins it
    A2 = A + [(32, 150)]
    tr = o.select(np.array([7, 3]), table([A2, B]))
    lists = [list(tr["cluster_idx"][tr["track_start"][k]:tr["track_start"][k + 1]])
             for k in range(len(tr["track_start"]) - 1)]
    assert 50 in lists[0] and all(50 not in l for l in lists[1:])
    # gaps: max_gap empty rows inside a track are allowed, one more is not
    ok = [(10 + i, i) for i in range(nmin - 1)] + [(10 + nmin - 1 + gmax, 90)]
    bad = [(10 + i, 60 + i) for i in range(nmin - 1)] + [(10 + nmin + gmax, 99)]
    tr = o.select(np.array([1, 2]), table([ok, bad]))
    assert len(tr["track_start"]) - 1 == 1
    assert list(tr["cluster_idx"]) == [j for _, j in ok]


# -------------------------------------------------- special-cluster errors
SCALE_OF_BIT = {0x01: "split_scale", 0x02: "single_row_scale", 0x04: "single_time_scale",
                0x08: "edge_scale", 0x10: "shared_scale"}


@pytest.mark.parametrize("flags", [0x01, 0x02, 0x04, 0x08, 0x10, 0x09, 0x1f])
def test_special_clusters_have_scaled_errors(geo, params, flags):
    """Flagged clusters have their error scaled by the factor of each flag
    bit (Sec. 3: special clusters get larger errors): flagging every cluster
    of a track leaves the least-squares estimate unchanged and divides chi2
    by the square of the product of the factors (up to the weak prior of the
    first pass)."""
    ev = synth.make_tiny(seed=29, n_tracks=10, sectors=(11,))
    ts, ci, tc, _ = synth.truth_tracks(ev, 60)
    o = _oracle(ev, geo, params)
    r = o.refit(ts, ci, tc, prec=64)
    ev.flags[:] = flags
    o2 = _oracle(ev, geo, params)
    r2 = o2.refit(ts, ci, tc, prec=64)
    ev.flags[:] = 0
    ok = (r["status"] == 0) & (r2["status"] == 0)
    assert ok.sum() >= 3
    s = np.prod([params[v] for b, v in SCALE_OF_BIT.items() if flags & b])
    ratio = r2["chi2"][ok] / r["chi2"][ok]
    np.testing.assert_allclose(ratio, 1.0 / (s * s), rtol=2e-2)
    np.testing.assert_allclose(r2["params"][ok], r["params"][ok], rtol=0, atol=2e-3 * s)


# ------------------------------------------- tracks across sectors (rotation)
def test_rotation_is_the_same_helix_and_its_covariance_transform(geo, params):
    """A state re-expressed in a rotated frame is the same helix at the same
    point: the global position and direction agree, rotating back returns the
    state, and the covariance transform is J C J^T with J taken by finite
    differences of (rotate, then follow the helix back to the rotated
    reference plane)."""
    ev = synth.make_tiny(seed=12, n_tracks=4)
    o = _oracle(ev, geo, params)
    rng = np.random.default_rng(3)
    n_ok = 0
    for _ in range(60):
        s0 = np.array([rng.uniform(-20, 20), rng.uniform(-50, 50), rng.uniform(-0.5, 0.5),
                       rng.uniform(-1, 1), rng.uniform(-5, 5)])
        x0 = rng.uniform(90, 240)
        d = rng.choice([-1, 1]) * math.pi / 9
        s1, x1, _ = o.rotate(s0, x0, d)
        if s1 is None:
            continue
        n_ok += 1
        # same point and direction in the global frame (frames differ by d)
        X0, Y0 = x0, s0[0]
        X1 = x1 * math.cos(d) - s1[0] * math.sin(d)
        Y1 = x1 * math.sin(d) + s1[0] * math.cos(d)
        assert abs(X1 - X0) < 1e-10 and abs(Y1 - Y0) < 1e-10
        assert abs(math.asin(s1[2]) + d - math.asin(s0[2])) < 1e-12
        assert s1[1] == s0[1] and s1[3] == s0[3] and s1[4] == s0[4]
        back, xb, _ = o.rotate(s1, x1, -d)
        np.testing.assert_allclose(back, s0, rtol=0, atol=1e-12)
        assert abs(xb - x0) < 1e-10
        # Jacobian at the rotated reference plane x1, by finite differences
        J = np.zeros((5, 5))
        for k in range(5):
            e = 1e-6 * max(1.0, abs(s0[k]))
            outs = []
            for sg in (1, -1):
                sp = s0.copy()
                sp[k] += sg * e
                r1, xr, _ = o.rotate(sp, x0, d)
                r2, _ = o.propagate(r1, xr, x1)
                outs.append(r2)
            J[:, k] = (outs[0] - outs[1]) / (2 * e)
        A = rng.normal(size=(5, 5))
        C = A @ A.T + np.eye(5)
        _, _, C1 = o.rotate(s0, x0, d, C)
        np.testing.assert_allclose(C1, J @ C @ J.T, rtol=1e-6, atol=1e-8)
    assert n_ok >= 40


def _merged_truth(geo, params, **kw):
    ev = synth.make_central(**kw)
    ts, ci, tc, ids = synth.truth_tracks(ev, 40, merged=True)
    multi = np.array([np.unique(ev.sector[ci[a:b]]).size > 1
                      for a, b in zip(ts[:-1], ts[1:])])
    return ev, ts, ci, tc, multi


def test_noise_free_helix_across_sectors_refits_to_truth(geo, params):
    """Exact clusters of helices that cross sector boundaries: the refit,
    rotating its state at every change of sector, returns the generating
    parameters at the innermost cluster in that cluster's frame."""
    ev, ts, ci, tc, multi = _merged_truth(geo, params, seed=7, n_tracks=400, noise_frac=0.0)
    ev.y[:] = ev.y_true.astype(np.float32)
    ev.z[:] = ev.z_true.astype(np.float32)
    o = _oracle(ev, geo, params)
    r = o.refit(ts, ci, tc, prec=64)
    ok = multi & (r["status"] == 0)
    assert ok.sum() >= 20
    inner = ci[ts[:-1].astype(np.int64)]
    truth = np.stack([ev.y_true, ev.z_true, ev.s_true, ev.tl_true, ev.q_true], 1)[inner]
    d = np.abs(r["params"][ok] - truth[ok])
    assert np.max(d[:, 0]) < 2e-5 and np.max(d[:, 1]) < 2e-5, np.max(d, 0)
    assert np.max(d[:, 2]) < 1e-6 and np.max(d[:, 3]) < 1e-6
    assert np.max(d[:, 4] / np.abs(truth[ok, 4])) < 2e-4
    np.testing.assert_allclose(r["x"][ok], geo.row_x[ev.row[inner]][ok].astype(np.float64))


def test_gradient_across_sectors_matches_finite_differences(geo, params):
    """The tape-derived gradient of a multi-sector refit (rotations included)
    against central finite differences of the cluster coordinates."""
    ev, ts, ci, tc, multi = _merged_truth(geo, params, seed=8, n_tracks=300, noise_frac=0.0)
    o = _oracle(ev, geo, params)
    r = o.refit(ts, ci, tc, prec=64)
    ks = np.nonzero(multi & (r["status"] == 0))[0][:2]
    assert ks.size == 2
    sel_ts = [0]
    sel_ci = []
    for k in ks:
        sel_ci.append(ci[ts[k]:ts[k + 1]])
        sel_ts.append(sel_ts[-1] + sel_ci[-1].size)
    ts2, ci2, tc2 = np.array(sel_ts, np.uint32), np.concatenate(sel_ci), tc[ks]
    r2 = o.refit(ts2, ci2, tc2, prec=64)
    g = np.array([1.0, 0.6])
    gy, gz, gc = o.refit_grad(ts2, ci2, tc2, r2["seeds"], r2["rej"], g)

    def loss(y, z):
        ev.y[:], ev.z[:] = y, z
        oo = _oracle(ev, geo, params)
        rr = oo.refit(ts2, ci2, tc2, prec=64, seeds=r2["seeds"], rej=r2["rej"])
        oo.close()
        return float(np.sum(g * rr["chi2"]))

    y0, z0 = ev.y.copy(), ev.z.copy()
    for q in [0, 5, ts2[1] - 1, ts2[1] + 4]:
        i = ci2[q]
        e = 1e-2
        yp, ym = y0.copy(), y0.copy()
        yp[i] += e
        ym[i] -= e
        fd = (loss(yp, z0) - loss(ym, z0)) / (2 * e)
        assert abs(fd - gy[q]) < 2e-3 * max(1, abs(fd)), (q, fd, gy[q])
        zp, zm = z0.copy(), z0.copy()
        zp[i] += e
        zm[i] -= e
        fd = (loss(y0, zp) - loss(y0, zm)) / (2 * e)
        assert abs(fd - gz[q]) < 2e-3 * max(1, abs(fd)), (q, fd, gz[q])
    ev.y[:], ev.z[:] = y0, z0


# ------------------------------------------------ segment merging (Sec. 2)
def _segment_key(ev):
    """Particle and leg of each cluster (-1 for noise)."""
    key = ev.label.astype(np.int64) * 4 + np.where(ev.segment >= 0, ev.segment % 4, 0)
    key[ev.label < 0] = -1
    return key


@pytest.mark.parametrize("mode", ["event", "time"])
def test_merge_links_segments_of_one_particle(geo, params, mode):
    """Found and refitted sector segments of a central event (three
    collisions): every link joins two segments of the same particle leg,
    nearly every pair of consecutive segments of a leg is linked, and the
    link chi2 follows a chi2 distribution of 5 degrees of freedom (the
    covariances are consistent)."""
    ev = synth.make_tiny(seed=41, n_tracks=300, central=True, mode=mode, noise_frac=0.1,
                         tf_start=1.0e6, n_coll=3)
    o = _oracle(ev, geo, params)
    tr = o.find(prec=32)["tracks"]
    ts, ci, tt = tr["track_start"], tr["cluster_idx"], tr["that"]
    r = o.refit(ts, ci, tt, prec=64)
    m = o.merge(ts, ci, tt, r["params"], r["cov"], r["x"], r["status"])
    nt = ts.size - 1
    key = _segment_key(ev)
    lab = np.array([np.bincount(k[k >= 0]).argmax() if (k >= 0).any() else -1
                    for k in (key[ci[ts[j]:ts[j + 1]]] for j in range(nt))])
    nx = m["next"]
    links = np.nonzero(nx >= 0)[0]
    assert links.size > 300
    assert np.all(lab[links] == lab[nx[links]]) and np.all(lab[links] >= 0)
    assert 4.5 < m["link_chi2"][links].mean() < 6.0
    assert np.all(m["link_chi2"][links] <= params["chi2_merge"])
    # consecutive segments of a leg (same side, both refitted)
    first_row = ev.row[ci[ts[:-1].astype(np.int64)]]
    side = ev.sector[ci[ts[:-1].astype(np.int64)]] // 18
    pairs = linked = 0
    for k in np.unique(lab[lab >= 0]):
        segs = [j for j in np.nonzero(lab == k)[0] if r["status"][j] == 0]
        segs.sort(key=lambda j: first_row[j])
        for a, b in zip(segs[:-1], segs[1:]):
            if side[a] == side[b]:
                pairs += 1
                linked += nx[a] == b
    assert linked >= 0.99 * pairs and pairs > 300
    # the merged track set: chains of segments from a segment without
    # predecessor, in the order of that segment
    heads = np.setdiff1d(np.arange(nt), nx[links])
    np.testing.assert_array_equal(m["head"], heads)
    assert m["track_start"].size - 1 == nt - links.size
    for t, h in enumerate(heads):
        chain = [h]
        while nx[chain[-1]] >= 0:
            chain.append(nx[chain[-1]])
        want = np.concatenate([ci[ts[j]:ts[j + 1]] for j in chain])
        np.testing.assert_array_equal(m["cluster_idx"][m["track_start"][t]:m["track_start"][t + 1]],
                                      want)
        assert m["that"][t] == tt[h]


def _pick_clusters(ev, sector, rows):
    """One cluster of the given sector on each of the given rows."""
    out = []
    for r in rows:
        idx = np.nonzero((ev.sector == sector) & (ev.row == r))[0]
        assert idx.size, (sector, r)
        out.append(idx[0])
    return np.array(out, np.uint32)


def _spd(rng, scale):
    A = rng.normal(size=(5, 5))
    return (A @ A.T + np.eye(5)) * scale


def _packed(C):
    return np.array([C[i, j] for i in range(5) for j in range(i + 1)])


def test_merge_chi2_is_the_quadratic_form_and_rules(geo, params):
    """Constructed segments with known states: the link chi2 equals
    d^T (C_i' + C_j)^-1 d with C_i' the rotated and transported covariance
    (numpy solve); only segments on the same side, in the same or a
    neighbouring sector frame and starting beyond the predecessor's last
    row are compared; of two predecessors of one segment the one with the
    smaller chi2 is linked."""
    ev = synth.make_tiny(seed=43, n_tracks=300, sectors=(3, 4, 5, 22), noise_frac=0.9)
    o = _oracle(ev, geo, params)
    rng = np.random.default_rng(5)
    rx = geo.row_x.astype(np.float64)
    p0 = np.array([3.0, 20.0, 0.15, 0.3, 0.8])
    C_a = _spd(rng, 1e-5)
    C_b = _spd(rng, 1e-5)
    # B: the exact continuation of p0 in the frame of sector 4 at row 70
    p1, x1, _ = o.rotate(p0, rx[40], math.pi / 9)
    p_b, _ = o.propagate(p1, x1, rx[70])
    p_b40, _ = o.propagate(p1, x1, rx[40])
    q5, x5, _ = o.rotate(p0, rx[40], 2 * math.pi / 9)
    p_b5, _ = o.propagate(q5, x5, rx[70])

    def chi2_of(p):
        q1, y1, C1 = o.rotate(p, rx[40], math.pi / 9, C_a)
        q2, C2 = o.propagate(q1, y1, rx[70], C1)
        d = q2 - p_b
        return d @ np.linalg.solve(C2 + C_b, d)

    u = np.array([0.002, -0.003, 1e-4, 2e-4, 0.001])
    p_a = p0 + u * math.sqrt(2.0 / chi2_of(p0 + u))     # chi2 about 2
    p_a2 = p0 + u * math.sqrt(8.0 / chi2_of(p0 + u))    # chi2 about 8
    want = chi2_of(p_a)
    segs = [  # sector, rows, state, covariance, x of the state
        (3, range(10, 41), p_a, C_a, rx[40]),           # 0: A
        (4, range(70, 100), p_b, C_b, rx[70]),          # 1: B, continuation of A
        (4, range(40, 75), p_b40, C_b, rx[40]),         # 2: starts on A's last row
        (5, range(70, 100), p_b5, C_b, rx[70]),         # 3: two frames away
        (22, range(70, 100), p_b, C_b, rx[70]),         # 4: other side
        (3, range(11, 41), p_a2, C_a, rx[40]),          # 5: A', a worse predecessor of B
    ]

    def run(sel):
        cs = [_pick_clusters(ev, segs[k][0], segs[k][1]) for k in sel]
        ts = np.concatenate([[0], np.cumsum([c.size for c in cs])]).astype(np.uint32)
        return o.merge(ts, np.concatenate(cs), np.zeros(len(sel)),
                       np.array([segs[k][2] for k in sel]),
                       np.array([_packed(segs[k][3]) for k in sel]),
                       np.array([segs[k][4] for k in sel]), np.zeros(len(sel), np.int32),
                       prec=64)

    m = run(range(6))
    assert list(m["next"]) == [1, -1, -1, -1, -1, -1]
    assert abs(m["link_chi2"][0] - want) < 1e-9 * want, (m["link_chi2"][0], want)
    # A' alone is linked to B, with a larger chi2
    m = run([5, 1])
    assert m["next"][0] == 1 and want < m["link_chi2"][0] <= params["chi2_merge"]
    # segments 2, 3, 4 carry exact continuations of A's helix but are never
    # compared with A
    for k in (2, 3, 4):
        assert list(run([0, k])["next"]) == [-1, -1], k
    # a predecessor farther off is not linked
    segs[0] = (3, range(10, 41), p0 + u * math.sqrt(40.0 / chi2_of(p0 + u)), C_a, rx[40])
    assert run([0, 1])["next"][0] == -1


def test_merge_expresses_z_with_the_predecessors_time(geo, params):
    """Time-frame mode: segment j's z was obtained with its own collision
    time; the clusters' calibration with i's time shifts it by a constant,
    which the merge takes into account (chi2 about 0 for an exact
    continuation whose z is given in j's time)."""
    ev = synth.make_tiny(seed=44, n_tracks=200, sectors=(3, 4), noise_frac=0.9, mode="time",
                         tf_start=1.0e6, n_coll=2)
    o = _oracle(ev, geo, params)
    rng = np.random.default_rng(6)
    rx = geo.row_x.astype(np.float64)
    c_a = _pick_clusters(ev, 3, range(10, 41))
    c_b = _pick_clusters(ev, 4, range(70, 100))
    th_a, th_b = 1.0e6 + 12.0, 1.0e6 + 31.0
    # the z offset between the two time bases, from the calibration itself
    za, _ = o.calibrate(c_b[:1], th_a)[1], None
    zb = o.calibrate(c_b[:1], th_b)[1]
    dz = float(za[0] - zb[0])
    assert abs(dz) > 10.0
    p_a = np.array([3.0, 20.0, 0.15, 0.3, 0.8])
    C_a = _spd(rng, 1e-3)
    p1, x1, C1 = o.rotate(p_a, rx[40], math.pi / 9, C_a)
    p_b, _ = o.propagate(p1, x1, rx[70], C1)
    p_b = p_b - np.array([0.0, dz, 0.0, 0.0, 0.0])   # B's z in its own time base
    ts = np.array([0, c_a.size, c_a.size + c_b.size], np.uint32)
    m = o.merge(ts, np.concatenate([c_a, c_b]), np.array([th_a, th_b]), np.array([p_a, p_b]),
                np.array([_packed(C_a), _packed(_spd(rng, 1e-3))]), np.array([rx[40], rx[70]]),
                np.zeros(2, np.int32), prec=64)
    assert m["next"][0] == 1 and m["link_chi2"][0] < 1e-8, m["link_chi2"]


# ------------------------------- collision time after merging (Sec. 4)
def _timeframe_truth(geo, params, seed):
    ev = synth.make_tiny(seed=seed, n_tracks=200, central=True, mode="time", tf_start=1.0e6,
                         n_coll=2, sigma=0.0)
    ts, ci, tc, ids = synth.truth_tracks(ev, 40, merged=True)
    first = ci[ts[:-1].astype(np.int64)]
    leg0 = (ids // 2) % 4 == 0
    zv = ev.part["zv"][ev.label[first]]
    return ev, ts, ci, tc, leg0, zv, first


def test_refined_time_puts_the_vertex_of_primaries_at_zero(geo, params):
    """Exact clusters of primaries, refitted with a collision time 0.7 us
    off: the refined time is the one at which the fitted helix's closest
    approach lies at z = 0, i.e. the true time shifted by the vertex z
    (t - sg z_v / v_drift), independently of the starting error."""
    ev, ts, ci, tc, leg0, zv, first = _timeframe_truth(geo, params, seed=48)
    cal = synth.nominal_calib()
    o = _oracle(ev, geo, params)
    t_start = tc + 0.7
    r = o.refit(ts, ci, t_start, prec=64)
    th = o.refine_time(ts, ci, t_start, r["params"], r["x"], r["status"], prec=64)
    sg = np.where(ev.sector[first] < 18, 1.0, -1.0)
    want = tc - sg * zv / cal.vdrift
    # tracks away from both ends of the drift volume (no shift inside needed)
    L = geo.drift_length
    inside = np.array([np.all((np.abs(ev.z_true[ci[a:b]]) > 6.0) &
                              (np.abs(ev.z_true[ci[a:b]]) < L - 6.0))
                       for a, b in zip(ts[:-1], ts[1:])])
    ok = leg0 & inside & (r["status"] == 0)
    assert ok.sum() >= 50
    assert np.max(np.abs(th[ok] - want[ok])) < 1e-6, np.max(np.abs(th[ok] - want[ok]))
    # failed refits and the event mode keep their time
    assert np.all(th[r["status"] != 0] == t_start[r["status"] != 0])


def test_refined_time_keeps_every_cluster_inside_the_drift_volume(geo, params):
    """When the closest-approach estimate would put clusters outside the
    drift volume (a state with a z offset, as for a secondary), the refined
    time is that estimate moved into the set of times for which every
    cluster's drift time lies in [0, L / v_drift]."""
    ev, ts, ci, tc, leg0, zv, first = _timeframe_truth(geo, params, seed=49)
    cal = synth.nominal_calib()
    o = _oracle(ev, geo, params)
    r = o.refit(ts, ci, tc, prec=64)
    ok = np.nonzero(r["status"] == 0)[0]
    T = float(geo.drift_length) / cal.vdrift
    moved = 0
    for off in (-120.0, 120.0):
        p = r["params"].copy()
        p[:, 1] += off
        th = o.refine_time(ts, ci, tc, p, r["x"], r["status"], prec=64)
        for k in ok:
            d = ev.t[ci[ts[k]:ts[k + 1]]] - cal.t0
            sg = 1.0 if ev.sector[first[k]] < 18 else -1.0
            est = tc[k] - sg * o.dca_z(p[k], r["x"][k]) / cal.vdrift
            lo, hi = d.min(), d.max()
            assert hi - lo <= T
            assert abs(th[k] - np.clip(est, hi - T, lo)) < 1e-9, (k, th[k], est, lo, hi - T)
            tau = d - th[k]
            assert tau.min() >= -1e-9 and tau.max() <= T + 1e-9
            moved += est != np.clip(est, hi - T, lo)
    assert moved >= 50


# ------------------------------------- native pad coordinates (next step)
def test_native_pads_give_the_same_tracking_as_their_positions(geo, params):
    """Native pad positions are turned into y = (pad - centre) * pitch of the
    cluster's row in single precision: the oracle fed with pads finds the
    same tracks and fits the same parameters as the oracle fed with those y
    values (numpy float32), the pads reproduce the generator's y within float
    rounding, and the gradient per pad is the gradient per cm times the
    pitch, checked by finite differences of a pad."""
    ev = synth.make_tiny(seed=52, n_tracks=150, central=True, mode="time", tf_start=1.0e6,
                         n_coll=2, noise_frac=0.05)
    row = ev.row.astype(np.int64)
    y_pad = ((ev.pad - geo.pad_center[row]) * geo.pad_width[row]).astype(np.float32)
    assert np.max(np.abs(y_pad - ev.y)) < 2e-5
    on = _oracle(ev, geo, params, pads=True)
    fn = on.find(prec=32)
    y0 = ev.y.copy()
    ev.y[:] = y_pad
    os_ = _oracle(ev, geo, params)
    fs = os_.find(prec=32)
    for k in ("up", "dn", "starts"):
        np.testing.assert_array_equal(fn[k], fs[k])
    for k in ("track_start", "cluster_idx", "that"):
        np.testing.assert_array_equal(fn["tracks"][k], fs["tracks"][k])
    tr = fn["tracks"]
    ts, ci, tt = tr["track_start"], tr["cluster_idx"], tr["that"]
    rn = on.refit(ts, ci, tt, prec=64)
    rs = os_.refit(ts, ci, tt, prec=64)
    np.testing.assert_array_equal(rn["params"], rs["params"])
    w = np.linspace(0.5, 1.5, ts.size - 1)
    gn = on.refit_grad(ts, ci, tt, rn["seeds"], rn["rej"], w)
    gs = os_.refit_grad(ts, ci, tt, rs["seeds"], rs["rej"], w)
    np.testing.assert_allclose(gn[0], gs[0] * geo.pad_width[row[ci]], rtol=1e-12, atol=0)
    np.testing.assert_array_equal(gn[1], gs[1])
    ev.y[:] = y0
    # finite differences of one pad position
    k = int(np.argmax(np.abs(gn[0])))
    i = ci[k]
    e = 1e-3

    def loss(p):
        p0 = ev.pad[i]
        ev.pad[i] = p
        oo = _oracle(ev, geo, params, pads=True)
        rr = oo.refit(ts, ci, tt, prec=64, seeds=rn["seeds"], rej=rn["rej"])
        oo.close()
        ev.pad[i] = p0
        return float(np.sum(w * rr["chi2"]))

    p0 = float(ev.pad[i])
    fd = (loss(np.float32(p0 + e)) - loss(np.float32(p0 - e))) / (
        float(np.float32(p0 + e)) - float(np.float32(p0 - e)))
    assert abs(fd - gn[0][k]) < 2e-2 * abs(gn[0][k]), (fd, gn[0][k])


# ------------------------------- track-model compression (Sec. 5)
def _entropy(a):
    _, cnt = np.unique(a, return_counts=True)
    p = cnt / cnt.sum()
    return float(-(p * np.log2(p)).sum())


@pytest.mark.parametrize("mode", ["event", "time"])
def test_compression_round_trip_is_exact_and_lossless_to_half_a_step(geo, params, mode):
    """Residuals of the clusters of found tracks and of truth tracks across
    sectors: a decoder running on the residuals alone (and the rows and
    sectors) reproduces the encoder's decoded clusters bit for bit, and every
    decoded cluster lies within half a quantisation step of the measured
    (distorted) one; the residual entropy is far below that of the absolute
    positions."""
    ev = synth.make_tiny(seed=55, n_tracks=300, central=True, mode=mode, tf_start=1.0e6,
                         n_coll=2, noise_frac=0.1)
    o = _oracle(ev, geo, params)
    tr = o.find(prec=32)["tracks"]
    sets = [(tr["track_start"], tr["cluster_idx"], tr["that"])]
    ts, ci, tc, _ = synth.truth_tracks(ev, 40, merged=True)
    sets.append((ts, ci, tc))
    cal = synth.nominal_calib()
    for q, qz in ((0.01, 0.013), (0.037, 0.02)):
        for ts, ci, tt in sets:
            c = o.compress(ts, ci, tt, qy=q, qz=qz)
            dy, dz = o.decompress(ts, ci, c["ry"], c["rz"], qy=q, qz=qz)
            np.testing.assert_array_equal(dy, c["dy"])
            np.testing.assert_array_equal(dz, c["dz"])
            my = ev.y[ci]
            if mode == "event":
                mz = ev.z[ci]
            else:
                that = np.repeat(tt, np.diff(ts.astype(np.int64)))
                sg = np.where(ev.sector[ci] < 18, 1.0, -1.0)
                mz = sg * (float(geo.drift_length) - cal.vdrift * ((ev.t[ci] - cal.t0) - that))
            assert np.max(np.abs(c["dy"] - my)) <= 0.5 * q * (1 + 1e-3) + 1e-5
            assert np.max(np.abs(c["dz"] - mz)) <= 0.5 * qz * (1 + 1e-3) + 3e-5
            first = np.zeros(ci.size, bool)
            first[ts[:-1].astype(np.int64)] = True
            if q == 0.01:
                assert _entropy(c["ry"][~first]) < _entropy(np.rint(my / q)) - 4.0
                assert _entropy(c["rz"][~first]) < _entropy(np.rint(mz / qz)) - 2.0


def test_compression_residuals_of_exact_helices_are_small(geo, params):
    """Clusters exactly on their helices: from the sixth cluster of a run on,
    the filter's prediction misses by the quantisation noise of the decoded
    clusters only, so the residuals are a few steps at most."""
    ev = synth.make_tiny(seed=56, n_tracks=200, central=True, noise_frac=0.0, sigma=0.0)
    ts, ci, tc, _ = synth.truth_tracks(ev, 40)
    o = _oracle(ev, geo, params)
    c = o.compress(ts, ci, tc, qy=0.01, qz=0.01)
    pos = np.concatenate([np.arange(b - a) for a, b in zip(ts[:-1].astype(np.int64),
                                                           ts[1:].astype(np.int64))])
    # away from |sin(phi)| = 0.95, where the transport stops and the previous
    # cluster becomes the prediction
    late = (pos >= 5) & (np.abs(ev.s_true[ci]) < 0.9)
    r = np.abs(np.concatenate([c["ry"][late], c["rz"][late]]))
    assert late.sum() > 5000
    assert np.percentile(r, 99) <= 4 and r.max() <= 8, (np.percentile(r, 99), r.max())


# -------------------------------------------- full field (Sec. 3)
def _field_event(eps, seed, n=300):
    from synth.field import solenoid_field
    f = solenoid_field(eps=eps)
    ev = synth.make_tiny(seed=seed, n_tracks=n, central=True, sigma=0.0, field=f)
    ev.y[:] = ev.y_true.astype(np.float32)
    ev.z[:] = ev.z_true.astype(np.float32)
    return ev, f


def test_field_transport_in_a_uniform_field_is_the_helix(geo, params):
    """With no inhomogeneity the Runge-Kutta transport in the field gives the
    exact helix and its covariance transport."""
    ev, f = _field_event(0.0, 61, n=20)
    o = _oracle(ev, geo, params, field=f)
    rng = np.random.default_rng(4)
    n_ok = 0
    for _ in range(40):
        s0 = np.array([rng.uniform(-20, 20), rng.uniform(-100, 100), rng.uniform(-0.6, 0.6),
                       rng.uniform(-1, 1), rng.uniform(-3, 3)])
        x0 = rng.uniform(90, 200)
        x1 = x0 + rng.uniform(-30, 30)
        A = rng.normal(size=(5, 5))
        C = A @ A.T + np.eye(5)
        a, ca = o.propagate_field(s0, x0, x1, rng.uniform(0, 2 * math.pi), C)
        b, cb = o.propagate(s0, x0, x1, C)
        if b is None:
            continue
        n_ok += 1
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-8)
        np.testing.assert_allclose(ca, cb, rtol=1e-12, atol=1e-12)
    assert n_ok >= 30


def test_field_transport_follows_the_traced_particles(geo, params):
    """In a non-uniform field (4 % solenoid-like inhomogeneity with radial
    components) the transport from one row crossing of a traced particle to
    a later one reproduces the tracer's crossing (the generator integrates
    the Lorentz force in arc length in the global frame, an independent
    implementation)."""
    ev, f = _field_event(0.04, 62)
    o = _oracle(ev, geo, params, field=f)
    truth = np.stack([ev.y_true, ev.z_true, ev.s_true, ev.tl_true, ev.q_true], 1)
    checked = 0
    worst = np.zeros(5)
    for s in np.unique(ev.segment[ev.segment >= 0])[:400]:
        idx = np.nonzero(ev.segment == s)[0]
        idx = idx[np.argsort(ev.row[idx])]
        if idx.size < 30:
            continue
        i, j = idx[2], idx[-3]
        al = synth.sector_alpha(ev.sector[i])
        got, _ = o.propagate_field(truth[i], geo.row_x[ev.row[i]], geo.row_x[ev.row[j]], al)
        if got is None:
            continue
        d = np.abs(got - truth[j])
        d[4] /= abs(truth[j][4])
        worst = np.maximum(worst, d)
        checked += 1
    assert checked >= 50
    assert worst[0] < 2e-5 and worst[1] < 2e-5, worst
    assert worst[2] < 1e-6 and worst[3] < 1e-6 and worst[4] < 1e-6, worst


def test_field_refit_removes_the_momentum_bias(geo, params):
    """Exact clusters of particles traced through the non-uniform field: the
    refit in the full field returns the generating parameters, the refit in
    the uniform field (Bz only, as before Sec. 3's change) is biased in
    q/pT."""
    ev, f = _field_event(0.04, 63)
    ts, ci, tc, _ = synth.truth_tracks(ev, 40)
    inner = ci[ts[:-1].astype(np.int64)]
    truth = np.stack([ev.y_true, ev.z_true, ev.s_true, ev.tl_true, ev.q_true], 1)[inner]
    rf = _oracle(ev, geo, params, field=f).refit(ts, ci, tc, prec=64)
    ru = _oracle(ev, geo, params).refit(ts, ci, tc, prec=64)
    ok = (rf["status"] == 0) & (ru["status"] == 0)
    assert ok.sum() >= 100
    df = np.abs(rf["params"][ok] - truth[ok])
    assert np.max(df[:, 0]) < 1e-4 and np.max(df[:, 1]) < 1e-4, df.max(0)
    assert np.max(df[:, 2]) < 1e-5 and np.max(df[:, 3]) < 1e-5, df.max(0)
    qf = df[:, 4] / np.abs(truth[ok, 4])
    qu = np.abs(ru["params"][ok, 4] - truth[ok, 4]) / np.abs(truth[ok, 4])
    assert np.max(qf) < 1e-4, np.max(qf)
    assert np.median(qu) > 20 * np.median(qf) and np.max(qu) > 3e-3, (np.median(qu), np.max(qu))


# ------------------------------------------------ vertex pseudo-measurement
def _vertex_tracks(ev, min_hits=40):
    """Truth tracks and their vertex z: only a particle's first outgoing leg
    passes through its vertex (later legs of a looper reach the beam line on
    another turn), so the other legs get NaN (no vertex)."""
    ts, ci, tc, sids = synth.truth_tracks(ev, min_hits)
    lab = ev.label[ci[ts[:-1].astype(np.int64)]]
    zv = np.asarray(ev.part["zv"], np.float64)[lab]
    zv[sids % 4 != 0] = np.nan
    return ts, ci, tc, zv


def test_vertex_refit_of_a_noise_free_primary_is_its_helix_at_the_beam_line(geo, params):
    """With exact clusters and the true vertex the fit ends at the beam line
    (x = 0) on the generating helix: y = 0, z = the vertex z, and the
    direction and curvature the pinned transport gives there; chi2 ~ 0."""
    ev = synth.make_tiny(seed=27, n_tracks=30, sectors=(3,), sigma=0.0)
    ts, ci, tc, zv = _vertex_tracks(ev)
    o = _oracle(ev, geo, params)
    r = o.refit(ts, ci, tc, prec=64, zv=zv, vsigma=0.01)
    n = 0
    for k in range(ts.size - 1):
        if r["status"][k] != 0 or r["x"][k] != 0.0 or np.isnan(zv[k]):
            continue
        i = int(ci[ts[k]])
        x0 = float(geo.row_x[ev.row[i]])
        truth = np.array([ev.y_true[i], ev.z_true[i], ev.s_true[i], ev.tl_true[i],
                          ev.q_true[i]])
        want, _ = o.propagate(truth, x0, 0.0)
        assert abs(want[0]) < 1e-9 and abs(want[1] - zv[k]) < 1e-9
        np.testing.assert_allclose(r["params"][k], want, rtol=0, atol=1e-6)
        # (cluster coordinates are stored in float32)
        assert r["chi2"][k] < 1e-6 and r["ndf"][k] == 2 * (ts[k + 1] - ts[k]) + 2
        n += 1
    assert n >= 15


def test_vertex_breaks_the_drift_velocity_and_t0_degeneracy(geo, params):
    """Reading of how v_drift and t0 become determinable: a change of t0
    shifts every cluster of a track along z by the same amount, which the
    track's z0 absorbs, so without a vertex the summed chi2 of the refit does
    not change; a change of v_drift by a factor 1 + e moves z by an affine
    map that z0 and tan(lambda) absorb, except that the measurement noise
    along z is scaled by 1 + e too, so chi2 changes by at most ~2e of itself.
    With the vertex z fixed both raise chi2 (a triggered event with a known
    vertex)."""
    ev = synth.make_tiny(seed=28, n_tracks=200, central=True, mode="time", tf_start=1.0e6,
                         n_coll=2)
    ts, ci, tc, zv = _vertex_tracks(ev)
    nom = synth.nominal_calib()

    def total(dv, dt0, use_zv):
        cal = synth.nominal_calib()
        cal.vdrift = nom.vdrift * (1.0 + dv)
        cal.t0 = nom.t0 + dt0
        o = _oracle(ev, geo, params, cal)
        r = o.refit(ts, ci, tc, prec=64, zv=zv if use_zv else None)
        o.close()
        return r["chi2"][r["status"] == 0].sum(), (r["status"] == 0).sum()

    c0, n0 = total(0.0, 0.0, False)
    v0, m0 = total(0.0, 0.0, True)
    assert n0 > 100 and m0 == n0
    for dv, dt0, flat in ((2e-3, 0.0, 2.5 * 2e-3), (0.0, 0.02, 1e-6)):
        c, n = total(dv, dt0, False)
        v, m = total(dv, dt0, True)
        assert n == n0 and m == m0
        print(f"dv {dv} dt0 {dt0}: without vertex {(c - c0) / c0:.2e}, with {(v - v0) / v0:.2e}")
        assert abs(c - c0) < flat * c0, (dv, dt0, c, c0)
        assert (v - v0) - abs(c - c0) > 1e-3 * v0, (dv, dt0, v, v0, c, c0)


def test_vertex_gradient_matches_finite_differences(geo, params):
    """The tape gradient of the refit with vertices (drift velocity, t0, a
    cluster's drift time) against central differences of the FP64 refit."""
    ev = synth.make_tiny(seed=29, n_tracks=8, sectors=(4,), mode="time", tf_start=1.0e6)
    ts, ci, tc, zv = _vertex_tracks(ev)
    nt = min(3, ts.size - 1)
    ts, ci, tc, zv = ts[:nt + 1], ci[:ts[nt]], tc[:nt], zv[:nt]
    cal = synth.nominal_calib()
    o = _oracle(ev, geo, params, cal)
    r = o.refit(ts, ci, tc, prec=64, zv=zv)
    assert np.sum(r["x"] == 0.0) >= 2
    gy, gz, gc = o.refit_grad(ts, ci, tc, r["seeds"], r["rej"], np.ones(nt), zv=zv)

    def loss(vd, t0, dt=None):
        c = synth.nominal_calib()
        c.vdrift, c.t0 = vd, t0
        e = ev
        if dt is not None:
            class E:
                pass
            e = E()
            for k in ("mode", "row", "sector", "flags", "event", "n_events", "tf_start", "z",
                      "y"):
                setattr(e, k, getattr(ev, k))
            e.t = ev.t.copy()
            e.t[dt[0]] += dt[1]
        oo = _oracle(e, geo, params, c)
        rr = oo.refit(ts, ci, tc, prec=64, seeds=r["seeds"], rej=r["rej"], zv=zv)
        oo.close()
        return float(rr["chi2"].sum())

    for k, e in ((0, 1e-7), (1, 1e-6)):
        a = [cal.vdrift, cal.t0]
        a[k] += e
        b = [cal.vdrift, cal.t0]
        b[k] -= e
        fd = (loss(*a) - loss(*b)) / (2 * e)
        assert abs(fd - gc[k]) < 1e-4 * max(1.0, abs(fd)), (k, fd, gc[k])
    q = 2
    i = int(ci[q])
    fd = (loss(cal.vdrift, cal.t0, (i, 1e-5)) - loss(cal.vdrift, cal.t0, (i, -1e-5))) / 2e-5
    assert abs(fd - gz[q]) < 1e-4 * max(1.0, abs(fd)), (fd, gz[q])
