"""A non-uniform solenoid field and particles traced through it.

The field is a quadratic polynomial in the global coordinates (X, Y, Z) in
metres (the form the library takes: ten monomials 1, X, Y, Z, X^2, XY, XZ,
Y^2, YZ, Z^2 per component); the solenoid-like model here,

    Bz = B0 (1 + eps (Z^2 - (X^2 + Y^2) / 2) / Lm^2),
    Bx = -B0 eps X Z / Lm^2,   By = -B0 eps Y Z / Lm^2,

is free of divergence and curl. Particles are traced by a fourth-order
Runge-Kutta integration of the Lorentz force in arc length (1 cm steps) in
the global frame; the crossings with the pad-row planes of each sector are
found on the cubic Hermite interpolant of each step. Only the outgoing leg
of each particle is traced (it stops when it turns back towards the beam
line, leaves the drift volume, or passes the outermost row).
"""
from __future__ import annotations

import math

import numpy as np

C_LIGHT = 2.99792458e-3  # GeV/c per (T cm)
MONOMIALS = ("1", "X", "Y", "Z", "XX", "XY", "XZ", "YY", "YZ", "ZZ")


def solenoid_field(b0=0.5, eps=0.04, lm=2.5):
    """Coefficients [3][10] of (Bx, By, Bz) in T, variables in metres."""
    a = np.zeros((3, 10), np.float64)
    a[0, 6] = -b0 * eps / lm ** 2          # Bx: XZ
    a[1, 8] = -b0 * eps / lm ** 2          # By: YZ
    a[2, 0] = b0                           # Bz: 1
    a[2, 4] = -0.5 * b0 * eps / lm ** 2    # Bz: XX
    a[2, 7] = -0.5 * b0 * eps / lm ** 2    # Bz: YY
    a[2, 9] = b0 * eps / lm ** 2           # Bz: ZZ
    return a.astype(np.float32)


def field_at(coef, X, Y, Z):
    """(Bx, By, Bz) at global positions in cm (numpy, float64)."""
    c = np.asarray(coef, np.float64)
    x, y, z = (np.asarray(v, np.float64) * 0.01 for v in (X, Y, Z))
    one = np.ones_like(x)
    m = np.stack([one, x, y, z, x * x, x * y, x * z, y * y, y * z, z * z])
    return np.tensordot(c, m, axes=(1, 0))


def _deriv(coef, P, U, kq):
    B = field_at(coef, P[0], P[1], P[2])
    dU = kq * np.stack([U[1] * B[2] - U[2] * B[1], U[2] * B[0] - U[0] * B[2],
                        U[0] * B[1] - U[1] * B[0]])
    return U, dU


def crossings_in_field(geo, p, coef, step=1.0):
    """Crossings of the outgoing leg of each particle with the pad-row planes:
    the same fields as the helix crossings of events.py (leg 0 only)."""
    n = p["pt"].shape[0]
    row_x = geo.row_x.astype(np.float64)
    tanA = math.tan(math.pi / 18.0)
    L = float(geo.drift_length)
    rho_out = float(row_x[-1]) / math.cos(math.pi / 18.0) + 1.0
    sw = math.pi / 9.0
    tanl = np.sinh(p["eta"])
    cl = 1.0 / np.sqrt(1.0 + tanl ** 2)
    P = np.stack([np.zeros(n), np.zeros(n), p["zv"].astype(np.float64)])
    U = np.stack([np.cos(p["phi0"]) * cl, np.sin(p["phi0"]) * cl, tanl * cl])
    qp = p["q"] / (p["pt"] / cl)            # q/|p|
    kq = C_LIGHT * qp
    active = np.ones(n, bool)
    larc = np.zeros(n)
    out = {k: [] for k in ("ip", "sector", "row", "y", "z", "s", "tl", "qpt", "leg", "larc")}
    h = step
    for _ in range(2000):
        if not active.any():
            break
        idx = np.nonzero(active)[0]
        P0, U0, k = P[:, idx], U[:, idx], kq[idx]
        # RK4 in arc length
        d1p, d1u = _deriv(coef, P0, U0, k)
        d2p, d2u = _deriv(coef, P0 + 0.5 * h * d1p, U0 + 0.5 * h * d1u, k)
        d3p, d3u = _deriv(coef, P0 + 0.5 * h * d2p, U0 + 0.5 * h * d2u, k)
        d4p, d4u = _deriv(coef, P0 + h * d3p, U0 + h * d3u, k)
        P1 = P0 + h / 6.0 * (d1p + 2 * d2p + 2 * d3p + d4p)
        U1 = U0 + h / 6.0 * (d1u + 2 * d2u + 2 * d3u + d4u)
        U1 = U1 / np.linalg.norm(U1, axis=0)
        # crossings of the row planes of the sectors at both ends of the step
        a0 = np.arctan2(P0[1], P0[0])
        a1 = np.arctan2(P1[1], P1[0])
        secs = np.stack([np.floor(a0 / sw), np.floor(a1 / sw)]).astype(np.int64) % 18
        for which in range(2):
            ks = secs[which]
            if which == 1:
                ks = np.where(secs[1] == secs[0], -1, ks)
            al = (ks + 0.5) * sw
            ca, sa = np.cos(al), np.sin(al)
            x0 = P0[0] * ca + P0[1] * sa
            x1 = P1[0] * ca + P1[1] * sa
            r0 = np.searchsorted(row_x, x0, side="right")
            r1 = np.searchsorted(row_x, x1, side="right")
            for dr in range(3):
                r = r0 + dr
                sel = (ks >= 0) & (r < r1) & (r < row_x.size) & (x1 > x0)
                if not sel.any():
                    continue
                j = np.nonzero(sel)[0]
                xr = row_x[r[j]]
                # cubic Hermite of the local x along the step; Newton for tau
                p0, p1 = P0[:, j], P1[:, j]
                m0, m1 = U0[:, j] * h, U1[:, j] * h
                c_, s_ = ca[j], sa[j]

                def herm(t):
                    t2, t3 = t * t, t * t * t
                    h00, h10 = 2 * t3 - 3 * t2 + 1, t3 - 2 * t2 + t
                    h01, h11 = -2 * t3 + 3 * t2, t3 - t2
                    pos = h00 * p0 + h10 * m0 + h01 * p1 + h11 * m1
                    d00, d10 = 6 * t2 - 6 * t, 3 * t2 - 4 * t + 1
                    d01, d11 = -6 * t2 + 6 * t, 3 * t2 - 2 * t
                    der = d00 * p0 + d10 * m0 + d01 * p1 + d11 * m1
                    return pos, der

                tau = (xr - x0[j]) / (x1[j] - x0[j])
                for _it in range(6):
                    pos, der = herm(tau)
                    fx = pos[0] * c_ + pos[1] * s_ - xr
                    dfx = der[0] * c_ + der[1] * s_
                    tau = tau - fx / dfx
                pos, der = herm(tau)
                u = der / np.linalg.norm(der, axis=0)
                ylo = -pos[0] * s_ + pos[1] * c_
                ulx = u[0] * c_ + u[1] * s_
                uly = -u[0] * s_ + u[1] * c_
                rho_u = np.sqrt(ulx ** 2 + uly ** 2)
                ok = (np.abs(ylo) <= xr * tanA) & (np.abs(pos[2]) <= L) & (ulx > 0)
                if not ok.any():
                    continue
                jj = j[ok]
                ip = idx[jj]
                Zc = pos[2][ok]
                out["ip"].append(ip)
                out["sector"].append(ks[jj] + 18 * (Zc < 0.0))
                out["row"].append(r[jj])
                out["y"].append(ylo[ok])
                out["z"].append(Zc)
                out["s"].append((uly / rho_u)[ok])
                out["tl"].append((u[2] / rho_u)[ok])
                out["qpt"].append((qp[ip] / rho_u[ok]))
                out["leg"].append(np.zeros(ip.size, np.int64))
                out["larc"].append(larc[ip] + tau[ok] * h)
        P[:, idx], U[:, idx] = P1, U1
        larc[idx] += h
        rho1 = np.hypot(P1[0], P1[1])
        vr = (P1[0] * U1[0] + P1[1] * U1[1])
        stop = (rho1 > rho_out) | (np.abs(P1[2]) > L) | ((vr < 0) & (rho1 > 1.0))
        active[idx[stop]] = False
    res = {k: (np.concatenate(v) if v else np.zeros(0)) for k, v in out.items()}
    for k in ("ip", "sector", "row", "leg"):
        res[k] = res[k].astype(np.int64)
    return res
