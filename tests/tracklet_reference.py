"""A second, plain-Python implementation of the tracklet constructor (Sec. 2
seed and following; Sec. 3 inward pass through the seed; Sec. 4 closest
approach -> collision time, calibrated coordinates), written from the steps
of the method for small inputs. It uses the oracle's helix transport and
Kalman update (pinned on their own against the generator, finite
differences and the information form) and brute force over the clusters of
a row, so that it checks the oracle's control flow: the seed, the phases,
the pick-up rule, the miss counting and the inward covariance scaling.

Float64 throughout; distortion-free calibration (the spline is pinned
separately).
"""
import math

import numpy as np


def _seed_two_points(x0, y0, z0, x1, y1, z1, c0):
    dx, dy, dz = x1 - x0, y1 - y0, z1 - z0
    dl = math.sqrt(dx * dx + dy * dy)
    return np.array([y0, z0, dy / dl, dz / dl, 0.0]), np.diag(c0), x0


def tracklets(o, ev, geo, params, calib, upc, starts):
    """Per start hit: hit count (-1 if the seed fit fails), hit rows (input
    index or -1 per row), collision time, and the state at its innermost
    pick (state, x)."""
    n_rows = len(geo.row_x)
    rx = np.asarray(geo.row_x, np.float64)
    zs = o.seed_z(64)
    sg32 = float(np.float32(params["sigma"]))
    sig2 = sg32 * sg32
    c0t = np.asarray(params["c0t"], np.float32).astype(np.float64)
    # clusters of each (event, sector, row), increasing input index
    rows = {}
    ev_id = ev.event if ev.event is not None else np.zeros(ev.n, np.int64)
    for i in range(ev.n):
        rows.setdefault((int(ev_id[i]), int(ev.sector[i]), int(ev.row[i])), []).append(i)

    def prop(p, C, x, x2):
        p2, C2 = o.propagate(p, x, x2, C)
        return (None, None) if p2 is None else (p2, C2)

    def update(p, C, my, mz):
        p2, C2, _ = o.update(p, C, my, mz, sig2, sig2)
        return p2, C2

    out_nh, out_hits, out_that, out_state, out_x = [], [], [], [], []
    for h0 in starts:
        hits = -np.ones(n_rows, np.int64)
        chain = [int(h0)]
        while upc[chain[-1]] >= 0 and len(chain) < params["seed_max_hits"]:
            chain.append(int(upc[chain[-1]]))
        e, sec = int(ev_id[h0]), int(ev.sector[h0])
        xs = [rx[ev.row[h]] for h in chain]
        # seed fit in seeding coordinates
        p, C, x = _seed_two_points(xs[0], float(ev.y[chain[0]]), zs[chain[0]], xs[-1],
                                   float(ev.y[chain[-1]]), zs[chain[-1]], c0t)
        failed = False
        for k, h in enumerate(chain):
            p, C = prop(p, C, x, xs[k])
            if p is None:
                failed = True
                break
            x = xs[k]
            p, C = update(p, C, float(ev.y[h]), zs[h])
        if failed:
            out_nh.append(-1), out_hits.append(hits), out_that.append(0.0)
            out_state.append(np.zeros(5)), out_x.append(0.0)
            continue
        # collision time from the closest approach (time mode)
        that = 0.0
        if ev.mode == "time":
            sg = 1.0 if sec < 18 else -1.0
            that = ev.tf_start - (sg * o.dca_z(p, x)) / calib.vdrift

        def cal(j):
            """Calibrated position once the collision time is known (Sec. 4):
            z from the drift time, t = t_coll + t0 + (L - |z|) / v_drift."""
            if ev.mode != "time":
                return float(ev.y[j]), zs[j]
            sg = 1.0 if ev.sector[j] < 18 else -1.0
            zeta = calib.vdrift * ((float(ev.t[j]) - calib.t0) - that)
            return float(ev.y[j]), sg * (float(np.float32(geo.drift_length)) - zeta)
        # seed fit in calibrated coordinates
        yz = [cal(h) for h in chain]
        p, C, x = _seed_two_points(xs[0], yz[0][0], yz[0][1], xs[-1], yz[-1][0], yz[-1][1],
                                   c0t)
        for k in range(len(chain)):
            p, C = prop(p, C, x, xs[k])
            if p is None:
                failed = True
                break
            x = xs[k]
            p, C = update(p, C, *yz[k])
        if failed:
            out_nh.append(-1), out_hits.append(hits), out_that.append(0.0)
            out_state.append(np.zeros(5)), out_x.append(0.0)
            continue

        def pick(p, C, r):
            vy = C[0, 0] + sig2
            vz = C[1, 1] + sig2
            best, bd = -1, 0.0
            for j in rows.get((e, sec, r), []):
                yc, zc = cal(j)
                ry, rz = yc - p[0], zc - p[1]
                d2 = (ry * ry) / vy + (rz * rz) / vz
                if not d2 <= params["chi2_pick"]:
                    continue
                if best < 0 or d2 < bd:
                    best, bd = j, d2
            return best

        # outward from the seed end
        best_state = (p.copy(), C.copy(), x)
        rlast = int(ev.row[chain[-1]])
        miss = 0
        for r in range(rlast + 1, n_rows):
            q, Q = prop(p, C, x, rx[r])
            if q is None:
                break
            p, C, x = q, Q, rx[r]
            j = pick(p, C, r)
            if j >= 0:
                p, C = update(p, C, *cal(j))
                best_state = (p.copy(), C.copy(), x)
                rlast = r
                miss = 0
            else:
                miss += 1
                if miss >= params["max_miss"]:
                    break
        # inward from the outermost pick, through the seed, covariance scaled
        p, C, x = best_state
        C = C * float(np.float32(params["inward_cov_scale"]))
        inner = (p.copy(), x)
        nh, miss = 0, 0
        for r in range(rlast, -1, -1):
            q, Q = prop(p, C, x, rx[r])
            if q is None:
                break
            p, C, x = q, Q, rx[r]
            j = pick(p, C, r)
            if j >= 0:
                p, C = update(p, C, *cal(j))
                hits[r] = j
                nh += 1
                miss = 0
                inner = (p.copy(), x)
            else:
                miss += 1
                if miss >= params["max_miss"]:
                    break
        out_nh.append(nh), out_hits.append(hits), out_that.append(that)
        out_state.append(inner[0]), out_x.append(inner[1])
    return dict(nh=np.array(out_nh), hits=np.array(out_hits), that=np.array(out_that),
                state=np.array(out_state), x=np.array(out_x))
