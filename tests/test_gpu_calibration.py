"""Calibration recovery by gradient descent on the adjoint refit (with and
without vertex pseudo-measurements), and the torch.autograd.Function against
finite differences of the GPU forward."""
import numpy as np
import pytest

import synth
from pipeline import tracker

pytestmark = pytest.mark.gpu


def _setup(seed=50, n_tracks=1500, max_abs=1.0, vertex=False, n_coll=2):
    """A time frame generated with a distorted calibration (v_drift +0.5 %,
    t0 +0.05 us, a per-sector spline up to max_abs cm), its truth tracks
    loaded; with vertex, each particle's first outgoing leg gets its vertex z
    as a pseudo-measurement (the other legs none)."""
    import torch
    rng = np.random.default_rng(seed)
    nom = synth.nominal_calib()
    true = synth.Calib(vdrift=nom.vdrift * 1.005, t0=nom.t0 + 0.05,
                       spline=synth.random_distortion(rng, max_abs))
    ev = synth.make_tiny(seed=seed, n_tracks=n_tracks, central=True, mode="time",
                         tf_start=1.0e6, n_coll=n_coll, calib=true)
    ts, ci, tc, sids = synth.truth_tracks(ev, 40)
    geo = synth.geometry()
    tr = tracker(geo)
    tr.set_calib()
    cl = tr.upload(ev)
    tr.load(cl)
    tr.set_tracks(torch.as_tensor(ts.astype(np.int32)), torch.as_tensor(ci.astype(np.int32)),
                  torch.as_tensor(tc))
    if vertex:
        lab = ev.label[ci[ts[:-1].astype(np.int64)]]
        zv = np.asarray(ev.part["zv"], np.float64)[lab]
        zv[sids % 4 != 0] = np.nan
        tr.set_vertex(torch.as_tensor(zv.astype(np.float32)), 0.01)
    tr.truth = (ev, ts, ci, tc)
    return tr, cl, nom, true


def _loss(tr, cl, theta):
    from paper_1811_11481_b300.autograd import RefitChi2
    chi2 = RefitChi2.apply(theta, cl["y"], cl["t"], tr)
    return float(chi2.sum()) / tr.ndf_sum


def test_gradient_descent_recovers_injected_distortion():
    """All of v_drift, t0 and the spline from the nominal calibration, with
    vertex pseudo-measurements and a small Tikhonov term: chi2/ndf returns
    to within 1 % of its value with the true calibration and the calibrated
    cluster positions' error in the part no track can absorb falls >= 5x
    (>= 10x at the adjoint workload's 100k tracks, bench.py --workload
    adjoint)."""
    import bench
    from paper_1811_11481_b300.autograd import calib_vector, recover_calibration
    tr, cl, nom, true = _setup(n_tracks=8000, vertex=True, n_coll=3)
    dev = tr.dev
    th_true = calib_vector(true.vdrift, true.t0, true.spline, dev)
    th_nom = calib_vector(nom.vdrift, nom.t0, nom.spline, dev)
    l_true = _loss(tr, cl, th_true)
    l_nom = _loss(tr, cl, th_nom)
    assert l_true < 1.2 and l_nom > 1.5 * l_true, (l_true, l_nom)
    theta, hist = recover_calibration(tr, th_nom, steps=400, lr_spline=0.02, lr_vdrift=1e-3,
                                      lr_t0=1e-3, tikhonov=1e-5)
    l_end = _loss(tr, cl, theta)
    ev, ts, ci, tc = tr.truth
    geo = synth.geometry()
    e_nom = bench.identifiable_error(geo, ev, ts, ci, tc, th_nom.cpu().numpy(),
                                     th_true.cpu().numpy())
    e_end = bench.identifiable_error(geo, ev, ts, ci, tc, theta.cpu().numpy(),
                                     th_true.cpu().numpy())
    print("chi2/ndf true %.4f nominal %.4f recovered %.4f; identifiable position error "
          "%.4f -> %.4f cm" % (l_true, l_nom, l_end, e_nom, e_end))
    assert abs(l_end / l_true - 1.0) < 0.01, (l_true, l_end, hist[::40])
    assert e_end < e_nom / 5.0, (e_nom, e_end)


@pytest.mark.parametrize("which", [0, 1])
def test_vertex_makes_drift_velocity_or_t0_recoverable(which):
    """With vertex pseudo-measurements and the spline known, v_drift (which
    0) or t0 (which 1), the other at its true value, from its nominal value
    by bounded L-BFGS: the error falls >= 10x. (Both together keep one
    nearly free combination, dt0 = dv L / v^2, which leaves the z of the
    vertex plane unchanged; only the vertices' z spread holds it.)"""
    from paper_1811_11481_b300.autograd import calib_vector, fit_drift_and_t0
    tr, cl, nom, true = _setup(n_tracks=8000, vertex=True, n_coll=3)
    v0 = nom.vdrift if which == 0 else true.vdrift
    t00 = nom.t0 if which == 1 else true.t0
    th0 = calib_vector(v0, t00, true.spline, tr.dev)
    theta = fit_drift_and_t0(tr, th0, free=(which == 0, which == 1))
    err = abs(float(theta[which]) - (true.vdrift, true.t0)[which])
    start = abs((nom.vdrift, nom.t0)[which] - (true.vdrift, true.t0)[which])
    print(f"{('v_drift', 't0')[which]}: error {err / start:.4f} of the initial")
    assert err < 0.1 * start, (err, start)


def test_autograd_gradient_matches_finite_difference_of_gpu_forward():
    import torch
    from paper_1811_11481_b300.autograd import RefitChi2, calib_vector
    tr, cl, nom, true = _setup(seed=51, n_tracks=300, max_abs=0.5)
    theta = calib_vector(nom.vdrift, nom.t0, true.spline * 0.5, tr.dev).requires_grad_(True)
    y = cl["y"]
    chi2 = RefitChi2.apply(theta, y, cl["t"], tr)
    chi2.sum().backward()
    g = theta.grad.detach().cpu().numpy()
    # directional derivative along the spline block of the gradient, central
    # difference of the float32 forward
    d = torch.zeros_like(theta)
    d[2:] = theta.grad[2:]
    d = d / d.norm()
    e = 0.01
    with torch.no_grad():
        lp = float(RefitChi2.apply(theta + e * d, y, cl["t"], tr).double().sum())
        lm = float(RefitChi2.apply(theta - e * d, y, cl["t"], tr).double().sum())
    fd = (lp - lm) / (2 * e)
    an = float(np.dot(g, d.cpu().numpy()))
    assert abs(fd - an) < 2e-2 * max(1.0, abs(fd)), (fd, an)
