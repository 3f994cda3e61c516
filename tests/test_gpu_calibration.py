"""Calibration recovery by gradient descent on the adjoint refit, and the
torch.autograd.Function against finite differences of the GPU forward."""
import numpy as np
import pytest

import synth
from pipeline import tracker

pytestmark = pytest.mark.gpu


def _setup(seed=50, n_tracks=1500, max_abs=1.0):
    import torch
    rng = np.random.default_rng(seed)
    nom = synth.nominal_calib()
    true = synth.Calib(vdrift=nom.vdrift * 1.005, t0=nom.t0 + 0.05,
                       spline=synth.random_distortion(rng, max_abs))
    ev = synth.make_tiny(seed=seed, n_tracks=n_tracks, central=True, mode="time",
                         tf_start=1.0e6, n_coll=2, calib=true)
    ts, ci, tc, _ = synth.truth_tracks(ev, 40)
    geo = synth.geometry()
    tr = tracker(geo)
    tr.set_calib()
    cl = tr.upload(ev)
    tr.load(cl)
    tr.set_tracks(torch.as_tensor(ts.astype(np.int32)), torch.as_tensor(ci.astype(np.int32)),
                  torch.as_tensor(tc))
    return tr, cl, nom, true


def _loss(tr, cl, theta):
    from paper_1811_11481_b300.autograd import RefitChi2
    chi2 = RefitChi2.apply(theta, cl["y"], cl["t"], tr)
    return float(chi2.sum()) / tr.ndf_sum


def test_gradient_descent_recovers_injected_distortion():
    import torch
    from paper_1811_11481_b300.autograd import calib_vector, recover_calibration
    tr, cl, nom, true = _setup()
    dev = tr.dev
    th_true = calib_vector(true.vdrift, true.t0, true.spline, dev)
    th_nom = calib_vector(nom.vdrift, nom.t0, nom.spline, dev)
    l_true = _loss(tr, cl, th_true)
    l_nom = _loss(tr, cl, th_nom)
    assert l_true < 1.2 and l_nom > 1.5 * l_true, (l_true, l_nom)
    theta, hist = recover_calibration(tr, th_nom, steps=200, lr_spline=0.02)
    l_end = _loss(tr, cl, theta)
    print("chi2/ndf true %.4f nominal %.4f recovered %.4f" % (l_true, l_nom, l_end))
    assert hist[-1] < hist[0]
    # chi2/ndf returns close to its value with the true calibration
    assert l_end < l_true * 1.05, (l_true, l_end, hist[::20])


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
