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
                        lr_t0=0.0, callback=None):
    """Gradient descent (Adam) on the calibration, minimising the summed chi2
    over ndf of the tracker's track set; returns the final theta and the loss
    history. v_drift and t0 only move with a nonzero learning rate: without a
    vertex constraint they are degenerate with the track z0 and tan(lambda)."""
    cl = tracker._keep["clusters"]
    y = cl["y"]
    zt = cl["t"] if cl.get("t") is not None else cl["z"]
    head = theta0[:2].clone().requires_grad_(True)
    spline = theta0[2:].clone().requires_grad_(True)
    groups = [{"params": [spline], "lr": lr_spline}]
    if lr_vdrift > 0 or lr_t0 > 0:
        groups.append({"params": [head], "lr": max(lr_vdrift, lr_t0)})
    opt = torch.optim.Adam(groups)
    hist = []
    for it in range(steps):
        opt.zero_grad()
        theta = torch.cat([head, spline])
        chi2 = RefitChi2.apply(theta, y, zt, tracker)
        loss = chi2.sum() / max(1, tracker.ndf_sum)
        loss.backward()
        opt.step()
        hist.append(float(loss.detach()))
        if callback:
            callback(it, hist[-1])
    return torch.cat([head, spline]).detach(), hist
