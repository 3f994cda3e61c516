"""The three-pass refit as a differentiable torch function.

``RefitChi2.apply(theta, y, zt, tracker)`` returns the pass-3 chi2 of every
track of the tracker's current track set. ``theta`` is the calibration
vector [v_drift, t0, spline (36 x 2 x 8 x 8 x 8)] (float64); ``y`` and
``zt`` are the loaded cluster coordinates (y, and t in time-frame mode or z
in event mode) -- the very tensors given to ``tracker.load``. The backward
pass is the library's adjoint (tpc_refit_backward): the track assignment,
the rejected clusters and the seed states are held fixed.
"""
import torch

from .binding import TPC_GRAD_CALIB_SIZE


class RefitChi2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, y, zt, tracker):
        if theta.numel() != TPC_GRAD_CALIB_SIZE:
            raise ValueError("theta must hold v_drift, t0 and the 36864 spline coefficients")
        cl = tracker._keep.get("clusters")
        if cl is None or cl["y"].data_ptr() != y.data_ptr():
            raise ValueError("y must be the tensor loaded into the tracker")
        ztl = cl["t"] if cl.get("t") is not None else cl["z"]
        if ztl.data_ptr() != zt.data_ptr():
            raise ValueError("zt must be the loaded t (time frame) or z (event) tensor")
        vt = theta[:2].detach().double().cpu()
        tracker.set_calib(vdrift=float(vt[0]), t0=float(vt[1]),
                          spline=theta[2:].detach().float().contiguous())
        out = tracker.refit(save_for_backward=True)
        tracker.ndf_sum = int(out["ndf"].sum())
        ctx.tracker = tracker
        ctx.shapes = (y.shape, y.dtype, zt.shape, zt.dtype, theta.dtype)
        return out["chi2"].clone()

    @staticmethod
    def backward(ctx, g_chi2):
        tr = ctx.tracker
        ys, yd, zs, zd, td = ctx.shapes
        gy, gz, gc = tr.refit_backward(g_chi2.float().contiguous())
        idx = tr.cluster_idx.long()
        grad_y = torch.zeros(ys, dtype=yd, device=gy.device).index_add_(0, idx, gy.to(yd))
        grad_zt = torch.zeros(zs, dtype=zd, device=gz.device).index_add_(0, idx, gz.to(zd))
        return gc.to(td), grad_y, grad_zt, None


def calib_vector(vdrift, t0, spline, device):
    """theta = [v_drift, t0, spline...] as float64 on device."""
    s = torch.as_tensor(spline, dtype=torch.float64, device=device).reshape(-1)
    head = torch.tensor([float(vdrift), float(t0)], dtype=torch.float64, device=device)
    return torch.cat([head, s])


def recover_calibration(tracker, theta0, steps=200, lr_spline=0.02, lr_vdrift=0.0,
                        lr_t0=0.0, tikhonov=0.0, callback=None):
    """Gradient descent (Adam, cosine-annealed) on the calibration,
    minimising the summed chi2 over ndf of the tracker's track set plus
    tikhonov * |spline|^2 (the minimum-norm choice along directions chi2 does
    not see). Returns the final theta and the loss history. A block moves
    only with a nonzero learning rate: without vertex pseudo-measurements
    (Tracker.set_vertex) v_drift and t0 are degenerate with every track's z0
    and tan(lambda); with them and a free spline, they still share the
    effect of each sector's constant and z-linear spline modes."""
    cl = tracker._keep["clusters"]
    y = cl["y"]
    zt = cl["t"] if cl.get("t") is not None else cl["z"]
    vd = theta0[0:1].clone().requires_grad_(True)
    t0 = theta0[1:2].clone().requires_grad_(True)
    spline = theta0[2:].clone().requires_grad_(True)
    groups = [{"params": [p], "lr": lr} for p, lr in ((spline, lr_spline), (vd, lr_vdrift),
                                                       (t0, lr_t0)) if lr > 0]
    opt = torch.optim.Adam(groups)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, steps)
    hist = []
    for it in range(steps):
        opt.zero_grad()
        theta = torch.cat([vd, t0, spline])
        chi2 = RefitChi2.apply(theta, y, zt, tracker)
        loss = chi2.sum() / max(1, tracker.ndf_sum)
        total = loss + tikhonov * (spline * spline).sum() if tikhonov > 0 else loss
        total.backward()
        opt.step()
        sched.step()
        hist.append(float(loss.detach()))
        if callback:
            callback(it, hist[-1])
    return torch.cat([vd, t0, spline]).detach(), hist


def fit_drift_and_t0(tracker, theta0, free=(True, True), iters=60, scale=(0.01, 0.1),
                     bound=5.0):
    """Drift velocity and/or t0 (free), the rest held at theta0's: bounded
    L-BFGS (scipy's L-BFGS-B) in units of `scale` (cm/us, us) within
    +-bound units of theta0, minimising the summed chi2 over ndf with the
    adjoint's gradient. The bound keeps the search where the tracks' fits
    converge: far off, failing tracks would leave the sum and lower the
    loss. With vertex pseudo-measurements each of the two alone has a clear
    minimum; together, the change dt0 = dv L / v^2 (which keeps the z of the
    vertex plane) is held only by the spread of the vertices' z. Returns the
    final theta."""
    import numpy as np
    from scipy.optimize import minimize
    cl = tracker._keep["clusters"]
    y = cl["y"]
    zt = cl["t"] if cl.get("t") is not None else cl["z"]
    base = theta0.detach().clone()
    sc = np.asarray(scale, np.float64) * np.asarray(free, np.float64)

    def f(u):
        du = torch.as_tensor(u * sc, dtype=torch.float64, device=base.device)
        head = (base[:2] + du).clone().requires_grad_(True)
        theta = torch.cat([head, base[2:]])
        chi2 = RefitChi2.apply(theta, y, zt, tracker)
        loss = chi2.sum() / max(1, tracker.ndf_sum)
        loss.backward()
        return float(loss), head.grad.detach().cpu().numpy() * sc
    res = minimize(f, np.zeros(2), jac=True, method="L-BFGS-B",
                   bounds=[(-bound, bound)] * 2, options=dict(maxiter=iters))
    du = torch.as_tensor(res.x * sc, dtype=torch.float64, device=base.device)
    return torch.cat([base[:2] + du, base[2:]])
