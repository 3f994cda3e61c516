#!/usr/bin/env python
"""Throughput of the TPC hot path on B300: clusters/s tracked.

One step = load a batch (bucketing, seeding transform, search grid), find
tracks (neighbours, link cleaning, start hits, tracklets, selection,
calibration transform), refit them (3 passes, saved for the adjoint) and run
the adjoint refit (gradient of the summed chi2 w.r.t. cluster coordinates and
calibration). Default workload: a 50 kHz continuous-readout time frame of 50
min-bias Pb-Pb-like collisions (11.1M clusters, float64 drift times, seed 2),
synthetic; `--workload central` runs one central event instead.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank processes its own independent event (seed 1 + rank):
weak scaling with no collective on the data path; the barrier and the
max-over-ranks timing use torch.distributed.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 126 * 1024 * 1024
METRIC = "TPC clusters/s tracked (CA+Kalman) on 1 B300; adjoint refit time vs fwd"
UNIT = "clusters/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="timeframe",
                    choices=["central", "timeframe", "batched", "single_sector", "adjoint"])
    ap.add_argument("--collisions", type=int, default=50,
                    help="collisions of the time-frame workload (50: the headline frame)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--field", action="store_true",
                    help="central event traced through a non-uniform field, refit (and "
                         "adjoint) in it")
    ap.add_argument("--pads", action="store_true",
                    help="give the clusters as native pad positions instead of y in cm")
    ap.add_argument("--no-merge", action="store_true",
                    help="skip the merging and compression stages measured after the "
                         "timed region")
    ap.add_argument("--no-recovery", action="store_true",
                    help="adjoint workload: skip the calibration recovery after the timing")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes instead of tuning them on the workload")
    ap.add_argument("--tuning", default=None,
                    help="launch shapes as JSON (tpc_tuning fields), instead of autotuning")
    ap.add_argument("--graph", action="store_true",
                    help="replay each step as one captured CUDA graph")
    ap.add_argument("--streams", type=int, default=2,
                    help="frames in flight: contexts on their own CUDA streams, each with its "
                         "own frame of the workload (1: one context, serial steps)")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="only run W+K steps with kernel timing (for ncu launch lists)")
    return ap.parse_args()


def make_workload(name, rank, collisions=50, field=None, frame=0):
    """The workload of this rank; frame k > 0 is another frame of the same
    kind (seed offset by 1000 k) for the k-th context in flight."""
    import synth
    rank = rank + 1000 * frame
    if name == "central":
        ev = synth.make_central(seed=1 + rank, field=field)
        cfg = dict(workload="central Pb-Pb-like event: 36 sectors x 152 rows, 10000 primaries "
                            "(pT power law, mean 0.5 GeV), 10% noise, event mode", seed=1 + rank)
        if field is not None:
            cfg["workload"] += ("; particles traced through a solenoid-like field with 4 % "
                                "inhomogeneity and radial components (outgoing legs), refit "
                                "in that full field")
    elif name == "timeframe":
        ev = synth.make_timeframe(seed=2 + rank, n_coll=collisions)
        cfg = dict(workload=f"50 kHz continuous-readout time frame: {collisions} collisions, "
                            "multiplicity Exp(2000), 15% noise, float64 times", seed=2 + rank)
    elif name == "batched":
        ev = synth.make_batched(seed=3 + rank)
        cfg = dict(workload="64 events, log-uniform 20..10000 tracks, one batch", seed=3 + rank)
    else:
        ev = synth.make_single_sector(seed=rank)
        cfg = dict(workload="single sector, 200 helices", seed=rank)
    cfg.update(n_clusters=int(ev.n), n_events=int(ev.n_events), mode=ev.mode)
    return ev, cfg


# ---------------------------------------------------------------- clocks
class Clocks:
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=[], samples=0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, f[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return dict(sm_mhz=float(np.median(sm)) if sm else None,
                    sm_max_mhz=float(max(smax)) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


# -------------------------------------------------------- byte model
def algorithmic_bytes(kernel, c):
    """Compulsory DRAM bytes of one launch (reads + writes of its inputs and
    outputs once; re-reads served on chip are not counted)."""
    n, mode, nt, na, ntl, nh = c["n"], c["mode"], c["n_tracks"], c["n_assigned"], \
        c["n_tracklets"], c["sum_nh"]
    zt = 8 if mode == 1 else 4
    ev = 4 if c["n_events"] > 1 else 0
    model = {
        "k_hist": n * (2 + zt + ev + 4),
        "k_scatter": n * (2 + ev + 4 + 4 + 4 + 8),
        "k_row_sort": n * (4 + 8 + 8 + 4 + 4 + 4),
        "k_neighbours": n * (12 + 8),
        "k_clean": n * (8 + 8),
        "k_write_starts": n * 8 + ntl * 8,
        # grid coordinates and input index once; per tracklet its start, seed
        # end, hit count, collision time and row range; per hit its row entry
        "k_tracklets": n * 12 + ntl * (8 + 16) + nh * 4,
        "k_tl_weight": ntl * 12 + nh * (4 + 8 + 8),
        "k_select_count": ntl * (4 + 4 + 8 + 8) + nh * (4 + 8),
        "k_select_write": ntl * 24 + nh * (4 + 8) + na * 12 + nt * 16,
        "k_calib": na * (4 + 4 + 8 + 4 + zt + 3 + 12),
        "k_interleave": na * (4 + 12 + 12),
        "k_refit": na * (12 + 1) + nt * (5 + 15 + 4) * 4,
        "k_refit_bwd": na * (12 + 1 + 8) + nt * 4,
        "k_calib_grad": na * (8 + 8 + 8 + 4 + zt + 2 + 8 + 8),
    }
    return model.get(kernel)


def aggregate(total_ms, units, dist=None, device="cpu"):
    """Whole-job timing over ranks: the slowest rank's time and the sum of the
    units (clusters) every rank processed; returns (max_ms, units_sum,
    units_per_second). Without torch.distributed initialised: this rank's."""
    if dist is not None and dist.is_available() and dist.is_initialized() and \
            dist.get_world_size() > 1:
        import torch
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        u = torch.tensor([float(units)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        total_ms, units = float(t.item()), float(u.item())
    return total_ms, units, units / (total_ms / 1000.0)


def _ncu_entry(fname, kernel):
    """The entry of 'kernel' in a committed ncu summary (profiles/fname), or
    None when the kernel's sources changed since that capture."""
    import hashlib
    p = os.path.join(ROOT, "profiles", fname)
    if not os.path.exists(p):
        return None
    e = json.load(open(p))["kernels"].get(kernel)
    if not e:
        return None
    src = os.path.join(ROOT, "paper_1811_11481_b300", "csrc")
    for f, h in e["sources"].items():
        fp = os.path.join(src, f)
        if not os.path.exists(fp) or hashlib.sha256(open(fp, "rb").read()).hexdigest()[:16] != h:
            return None
    return e


def ncu_traffic(kernel, units):
    """DRAM bytes (read + write) of one launch of 'kernel' that processes
    'units' (dict of unit counts), from the committed ncu capture scaled by
    the units the capture processed; None when the sources changed."""
    e = _ncu_entry("ncu_traffic.json", kernel)
    if not e or e.get("unit") not in units:
        return None
    return e["bytes_per_unit"] * units[e["unit"]]


def ncu_flops(kernel, units):
    """Executed single-precision floating-point operations of one launch of
    'kernel' (FFMA counted as 2, FADD and FMUL as 1, from ncu's SASS
    instruction counters), scaled from the capture by the launch's units;
    None when the sources changed since the capture."""
    e = _ncu_entry("ncu_alu.json", kernel)
    if not e or e.get("unit") not in units:
        return None
    return e["flops_per_unit"] * units[e["unit"]]


def alu_peak_gflops(sms, sm_mhz):
    """FP32 peak of the GPU at the sampled SM clock: SMs x 128 FP32 lanes x 2
    operations per fused multiply-add x clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e9


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=float(d["hbm_gbs"]), source="measured",
                    sm_max_mhz=float(d.get("sm_max_mhz", 2032.0)))
    return dict(hbm_gbs=6400.0, source="fallback", sm_max_mhz=2032.0)


# ------------------------------------------------------------- our arm
def track_quality(ev, track_start, cluster_idx, min_findable=70, purity=0.9):
    """Efficiency, fake and clone rates of found tracks against the
    generator's truth segments (one per particle, sector and leg): a segment
    with at least min_findable clusters is findable; a track matches the
    segment of the majority of its clusters if that majority is at least
    `purity` of them, and is fake otherwise."""
    ts = np.asarray(track_start, np.int64)
    nt = ts.size - 1
    if nt <= 0:
        return dict(efficiency=0.0, fake_rate=0.0, clone_rate=0.0, findable=0, tracks=0)
    seg = np.asarray(ev.segment, np.int64)[np.asarray(cluster_idx, np.int64)]
    lens = np.diff(ts)
    tid = np.repeat(np.arange(nt), lens)
    M = int(seg.max()) + 2
    key, cnt = np.unique(tid * M + (seg + 1), return_counts=True)
    ktid, kseg = key // M, key % M - 1
    order = np.lexsort((-cnt, ktid))
    first = order[np.r_[True, ktid[order][1:] != ktid[order][:-1]]]
    maj_seg, maj_cnt = kseg[first], cnt[first]
    good = (maj_seg >= 0) & (maj_cnt >= purity * lens[ktid[first]])
    matched, per = np.unique(maj_seg[good], return_counts=True)
    truth = np.bincount(np.asarray(ev.segment, np.int64)[np.asarray(ev.segment) >= 0])
    findable = np.nonzero(truth >= min_findable)[0]
    eff = float(np.isin(findable, matched).mean()) if findable.size else 0.0
    return dict(efficiency=eff, fake_rate=float((~good).sum() / nt),
                clone_rate=float((per - 1).sum() / nt), findable=int(findable.size), tracks=nt,
                definition=f"findable: >= {min_findable} clusters of one (particle, sector, leg); "
                           f"matched: >= {int(purity * 100)}% of a track's clusters from it")


def merged_quality(ev, track_start, cluster_idx, min_findable=70, purity=0.9, cover=0.8):
    """How many particle legs that cross sector boundaries are found whole:
    a leg (particle, leg, side) with at least min_findable clusters in two
    or more sector frames is findable; it is found whole when one track has
    at least `purity` of its clusters from it and holds at least `cover` of
    the leg's clusters."""
    seg = np.asarray(ev.segment, np.int64)
    lab = np.asarray(ev.label, np.int64)
    side = (np.asarray(ev.sector) >= 18).astype(np.int64)
    key = np.where(seg >= 0, (lab * 4 + seg % 4) * 2 + side, -1)
    sig = key >= 0
    K = int(key.max()) + 1 if sig.any() else 1
    size = np.bincount(key[sig], minlength=K)
    frames = np.zeros(K, np.int64)
    fk = np.unique(key[sig] * 18 + np.asarray(ev.sector)[sig] % 18)
    np.add.at(frames, fk // 18, 1)
    findable = np.nonzero((size >= min_findable) & (frames >= 2))[0]
    ts = np.asarray(track_start, np.int64)
    ci = np.asarray(cluster_idx, np.int64)
    whole = set()
    for t in range(ts.size - 1):
        k = key[ci[ts[t]:ts[t + 1]]]
        if k.size == 0:
            continue
        v, c = np.unique(k, return_counts=True)
        j = np.argmax(c)
        if v[j] >= 0 and c[j] >= purity * k.size and c[j] >= cover * size[v[j]]:
            whole.add(int(v[j]))
    return dict(findable=int(findable.size),
                found_whole=float(np.isin(findable, list(whole)).mean()) if findable.size else 0.0)


def merge_stage(tr, cl, ev, flush, stream, reps=5):
    """Sector merging and collision-time refinement after the per-sector
    refit (Sec. 2 second phase, Sec. 4), on the same batch: find, refit,
    merge, refit, refine the times (time-frame mode), refit."""
    import torch

    def ev_pair():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    acc = dict(merge_ms=0.0, merged_refit_ms=0.0, refine_ms=0.0, final_refit_ms=0.0)
    info = {}
    for rep in range(reps):
        tr.load(cl)
        tr.find()
        seg = tr.refit()
        if rep == 0:
            t0 = tr.tracks()
            info["segments"] = tr.n_tracks
            info["before"] = merged_quality(ev, t0["track_start"].cpu().numpy(),
                                            t0["cluster_idx"].cpu().numpy())
        flush.fill_(1.0)
        spans = {}
        a, b = ev_pair()
        a.record(stream)
        m = tr.merge(seg)
        b.record(stream)
        spans["merge_ms"] = (a, b)
        a, b = ev_pair()
        a.record(stream)
        r1 = tr.refit()
        b.record(stream)
        spans["merged_refit_ms"] = (a, b)
        a, b = ev_pair()
        a.record(stream)
        tr.refine_time(r1)
        b.record(stream)
        spans["refine_ms"] = (a, b)
        a, b = ev_pair()
        a.record(stream)
        r2 = tr.refit()
        b.record(stream)
        spans["final_refit_ms"] = (a, b)
        torch.cuda.synchronize()
        for k, (a, b) in spans.items():
            acc[k] += a.elapsed_time(b) / reps
        if rep == 0:
            nx = m["next"]
            info["links"] = int((nx >= 0).sum().item())
            info["merged_tracks"] = tr.n_tracks
            t1 = tr.tracks()
            info["after"] = merged_quality(ev, t1["track_start"].cpu().numpy(),
                                           t1["cluster_idx"].cpu().numpy())
            info["refit_ok"] = float((r2["status"] == 0).float().mean().item())
    return dict(acc, **info, reps=reps,
                note="after the timed region, on the same batch; merge_ms brackets the "
                     "synchronous tpc_merge_tracks call (segment copies, kernels, count "
                     "read-back); quality: legs crossing sector boundaries found whole "
                     "by one track before and after merging")


def merge_chain(tr, cl, n, flush, stream, steps):
    """The full chain of the widened path as one CUDA graph per step: load,
    find, refit of the segments, merge (asynchronous), refit, collision-time
    refinement, refit; timed over `steps` replays with the L2 flushed
    before each (after the headline's timed region)."""
    import ctypes as C
    import torch
    P = lambda t: C.c_void_p(t.data_ptr())
    L, h = tr.L, tr.h
    cap = n // 10 + 1
    dev = tr.dev
    f = lambda *s: torch.zeros(*s, device=dev)
    i32 = lambda *s: torch.zeros(*s, dtype=torch.int32, device=dev)
    mk = lambda: dict(params=f(cap, 5), cov=f(cap, 15), x=f(cap), chi2=f(cap), ndf=i32(cap),
                      status=i32(cap), rej=torch.zeros(n + 1, dtype=torch.uint8, device=dev))
    seg, r1, r2 = mk(), mk(), mk()

    def ck(st, what):
        if st != 0:
            raise RuntimeError(f"{what}: status {st}: {L.tpc_last_error(h).decode()}")

    def fit(o):
        ck(L.tpc_refit(h, 0, P(o["params"]), P(o["cov"]), P(o["x"]), P(o["chi2"]), P(o["ndf"]),
                       P(o["status"]), P(o["rej"])), "refit")

    def step():
        tr.load(cl)
        ck(L.tpc_find_tracks_async(h), "find")
        fit(seg)
        ck(L.tpc_merge_tracks_async(h, P(seg["params"]), P(seg["cov"]), P(seg["x"]),
                                    P(seg["status"]), None, None), "merge")
        fit(r1)
        ck(L.tpc_refine_time(h, P(r1["params"]), P(r1["x"]), P(r1["status"]), None), "refine")
        fit(r2)

    for _ in range(3):
        step()
    tr.counts()                      # reports a capacity error of the asynchronous merge
    torch.cuda.synchronize()
    tr.graph_begin()
    step()
    tr.graph_end()
    tr.graph_launch()
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tr.graph_launch()
        b.record(stream)
        times.append((a, b))
    torch.cuda.synchronize()
    nt, na, _ = tr.counts()
    ms = float(np.mean([a.elapsed_time(b) for a, b in times]))
    return dict(value=n / (ms / 1000.0), unit=UNIT, ms_per_step=ms, steps=steps,
                merged_tracks=nt, refit_ok=float((r2["status"][:nt] == 0).float().mean().item()),
                note="one CUDA graph per step: load, find, refit, merge, refit, collision-time "
                     "refinement, refit; L2 flushed before each replay")


def _entropy_bits(a):
    _, c = np.unique(a, return_counts=True)
    p = c / c.sum()
    return float(-(p * np.log2(p)).sum())


def compression_stage(tr, cl, flush, stream, reps=5, qy=0.01, qz=0.01):
    """Track-model compression of the found tracks (Sec. 5): the encoder
    kernel timed with CUDA events (after the headline's timed region), and
    the empirical entropy of the residuals against that of the quantised
    absolute positions."""
    import torch
    tr.load(cl)
    tr.find()
    tr.compress(qy, qz)                                  # allocates
    acc = 0.0
    for _ in range(reps):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = tr.compress(qy, qz)
        b.record(stream)
        b.synchronize()
        acc += a.elapsed_time(b)
    ms = acc / reps
    ry, rz = out["ry"].cpu().numpy(), out["rz"].cpu().numpy()
    dy, dz = out["dy"].cpu().numpy(), out["dz"].cpu().numpy()
    ts = tr.tracks()["track_start"].cpu().numpy().astype(np.int64)
    first = np.zeros(ry.size, bool)
    first[ts[:-1]] = True
    res_bits = _entropy_bits(ry[~first]) + _entropy_bits(rz[~first])
    abs_bits = _entropy_bits(np.rint(dy / qy).astype(np.int64)) + \
        _entropy_bits(np.rint(dz / qz).astype(np.int64))
    na = int(ry.size)
    return dict(ms=ms, assigned_clusters=na, clusters_per_s=na / (ms / 1000.0),
                step_cm=[qy, qz], residual_bits_per_cluster=res_bits,
                absolute_bits_per_cluster=abs_bits, entropy_ratio=abs_bits / res_bits,
                note="k_compress on the found tracks (one thread per track), CUDA events, "
                     "L2 flushed; empirical entropies of the (y, z) residuals after the first "
                     "cluster of each track and of the quantised absolute positions")


def run_ours(args):
    import torch
    import torch.distributed as dist
    import synth
    from paper_1811_11481_b300.binding import Tracker, TPC_GRAD_CALIB_SIZE

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    geo = synth.geometry()
    field = None
    if args.field:
        if args.workload != "central":
            raise SystemExit("--field: the central workload only")
        from synth.field import solenoid_field
        field = solenoid_field()
    ev, cfg = make_workload(args.workload, rank, args.collisions, field)
    work = torch.cuda.Stream()
    torch.cuda.set_stream(work)
    tr = Tracker(geo, stream=work, field=field)
    tr.set_calib()
    cl = tr.upload(ev, pads=args.pads)
    if args.pads:
        cfg = dict(cfg, coordinates="native pad positions, turned into cm on the fly")
    L, h = tr.L, tr.h
    if args.tuning:
        tr.set_tuning(**json.loads(args.tuning))
        tuning, how = tr.get_tuning(), "given"
    elif not args.no_autotune:
        # launch shapes tuned on this workload, before and outside the timed region
        tr.load(cl)
        tuning, how = tr.autotune(repeats=3), "autotuned"
    else:
        tuning, how = tr.get_tuning(), "default"
    # the other frames in flight: one context each, on its own stream, with
    # the same launch shapes
    others = []
    for k in range(1, max(1, args.streams)):
        ev_k, cfg_k = make_workload(args.workload, rank, args.collisions, field, frame=k)
        st_k = torch.cuda.Stream()
        tr_k = Tracker(geo, stream=st_k, field=field)
        tr_k.set_calib()
        tr_k.set_tuning(**{f: tuning[f] for f in ("grid_tau", "grid_ny_max", "tracklet_block",
                                                  "tracklet_per_sm", "tracklet_regs")})
        others.append(dict(ev=ev_k, seed=cfg_k["seed"], stream=st_k, tr=tr_k,
                           cl=tr_k.upload(ev_k, pads=args.pads)))
    n = ev.n
    cap_tr = n // 10 + 1
    dev = tr.dev
    out = dict(params=torch.empty(cap_tr, 5, device=dev), cov=torch.empty(cap_tr, 15, device=dev),
               x=torch.empty(cap_tr, device=dev), chi2=torch.empty(cap_tr, device=dev),
               ndf=torch.empty(cap_tr, dtype=torch.int32, device=dev),
               status=torch.empty(cap_tr, dtype=torch.int32, device=dev),
               rej=torch.empty(n + 1, dtype=torch.uint8, device=dev))
    ones = torch.ones(cap_tr, device=dev)
    gy = torch.empty(n + 1, device=dev)
    gz = torch.empty(n + 1, device=dev)
    gc = torch.empty(TPC_GRAD_CALIB_SIZE, dtype=torch.float64, device=dev)
    import ctypes as C
    P = lambda t: C.c_void_p(t.data_ptr())
    stream = torch.cuda.current_stream()

    def ck(st, what):
        if st != 0:
            raise RuntimeError(f"{what}: status {st}: {L.tpc_last_error(h).decode()}")

    def step(refit=True, backward=True):
        tr.load(cl)
        ck(L.tpc_find_tracks_async(h), "find")
        if refit:
            ck(L.tpc_refit(h, 1, P(out["params"]), P(out["cov"]), P(out["x"]), P(out["chi2"]),
                           P(out["ndf"]), P(out["status"]), P(out["rej"])), "refit")
        if backward:
            ck(L.tpc_refit_backward(h, P(ones), P(gy), P(gz), P(gc)), "backward")

    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    # warm-up (allocations happen here), then a count check
    for _ in range(max(3, args.warmup)):
        step()
    if args.graph:
        work.synchronize()
        tr.graph_begin()
        step()
        tr.graph_end()
        direct_step = step

        def step(refit=True, backward=True):
            if refit and backward:
                tr.graph_launch()
            else:
                direct_step(refit, backward)
        step()
    if args.profile_steps:
        # steady-state steps only: for ncu launch lists and captures
        tr.profile(True)
        for _ in range(args.profile_steps):
            step()
        kstats, launches = tr.profile_read()
        nt_p, na_p, _ = tr.counts()
        nh_p = int(tr.tracklets()["nh"].clamp(min=0).sum().item())
        # the units one step of this context processes: ncu figures per
        # launch divided by these give the per-unit figures of the summaries
        print(json.dumps(dict(profile_steps=args.profile_steps, launches=launches,
                              units=dict(cluster=int(ev.n), tracklet_hit=nh_p,
                                         assigned_cluster=int(na_p), track=int(nt_p)),
                              kernels={k: v for k, v in kstats.items()})))
        return
    nt, na, ntl = tr.counts()
    tl = tr.tracklets()
    sum_nh = int(tl["nh"].clamp(min=0).sum().item())
    found = tr.find()
    quality = track_quality(ev, found["track_start"].cpu().numpy(),
                            found["cluster_idx"].cpu().numpy())

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- per-kernel breakdown: a separate pass with every launch timed
    n_prof = min(args.steps, 20)
    prof_step = direct_step if args.graph else step
    tr.profile(True)
    for _ in range(n_prof):
        flush.fill_(1.0)
        prof_step()
    kstats_all, _ = tr.profile_read()
    tr.profile(False)
    dom = max(kstats_all, key=lambda k: kstats_all[k][1]) if kstats_all else None

    # ---- timed region: device-resident inputs, L2 flushed before each step;
    # only the dominant kernel carries CUDA events (for its roofline)
    clocks = Clocks(local)
    clocks.start()
    t_end = time.time() + 1.5  # keep the GPU busy while the sampler starts
    while time.time() < t_end:
        step()
    tr.profile(True)
    tr.profile_only(dom)
    barrier()
    times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        times.append((e0, e1))
    barrier()
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in times]
    kstats, launches = tr.profile_read()
    tr.profile_only(None)
    tr.profile(False)
    total_ms, units, value = aggregate(float(np.sum(ms)), n * args.steps, dist, dev)

    # ---- the same steps replayed as one CUDA graph each, without the
    # per-kernel events of the timed region above (reported beside it)
    graph_replay = None
    if not args.graph:
        work.synchronize()
        tr.graph_begin()
        step()
        tr.graph_end()
        tr.graph_launch()
        barrier()
        gtimes = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tr.graph_launch()
            e1.record(stream)
            gtimes.append((e0, e1))
        barrier()
        g_ms, _, g_value = aggregate(float(np.sum([a.elapsed_time(b) for a, b in gtimes])),
                                     n * args.steps, dist, dev)
        graph_replay = dict(value=g_value, unit=UNIT, ms_per_step=g_ms / args.steps,
                            steps=args.steps, note="one CUDA graph per step, L2 flushed "
                            "before each, no per-kernel events")

    # ---- forward-only vs adjoint timing (phases of the same step)
    def phase_time(fn, reps=5):
        torch.cuda.synchronize()
        acc = 0.0
        for _ in range(reps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            acc += a.elapsed_time(b)
        return acc / reps
    step()
    torch.cuda.synchronize()
    t_fwd = phase_time(lambda: ck(L.tpc_refit(h, 1, P(out["params"]), P(out["cov"]), P(out["x"]),
                                              P(out["chi2"]), P(out["ndf"]), P(out["status"]),
                                              P(out["rej"])), "refit"))
    t_fwd_nosave = phase_time(lambda: ck(L.tpc_refit(h, 0, P(out["params"]), P(out["cov"]),
                                                     P(out["x"]), P(out["chi2"]), P(out["ndf"]),
                                                     P(out["status"]), P(out["rej"])), "refit"))
    # a saved refit through a direct call (a graph replay does not update the
    # context's host-side record of what was saved)
    ck(L.tpc_refit(h, 1, P(out["params"]), P(out["cov"]), P(out["x"]), P(out["chi2"]),
                   P(out["ndf"]), P(out["status"]), P(out["rej"])), "refit")
    t_bwd = phase_time(lambda: ck(L.tpc_refit_backward(h, P(ones), P(gy), P(gz), P(gc)), "bwd"))

    # ---- find + refit without the adjoint: load, find, refit (no
    # checkpoints), the quantity the HBM target of the method is stated on
    def fr_step():
        tr.load(cl)
        ck(L.tpc_find_tracks_async(h), "find")
        ck(L.tpc_refit(h, 0, P(out["params"]), P(out["cov"]), P(out["x"]), P(out["chi2"]),
                       P(out["ndf"]), P(out["status"]), P(out["rej"])), "refit")
    for _ in range(3):
        fr_step()
    tr.profile(True)
    barrier()
    fr_times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fr_step()
        e1.record(stream)
        fr_times.append((e0, e1))
    barrier()
    fr_kstats, _ = tr.profile_read()
    tr.profile(False)
    fr_ms, _, fr_value = aggregate(float(np.sum([a.elapsed_time(b) for a, b in fr_times])),
                                   n * args.steps, dist, dev)
    fr_ms /= args.steps

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        host = {k: (v.cpu().pin_memory() if v is not None else None) for k, v in cl.items()
                if hasattr(v, "cpu")}
        res_h = torch.empty(cap_tr * 6 + 8, dtype=torch.float32).pin_memory()
        cnt_h = torch.empty(3, dtype=torch.int64)
        h2d = sum(v.numel() * v.element_size() for v in host.values() if v is not None)
        d2h = res_h.numel() * 4
        # two device copies of the inputs: while a step runs on one, the
        # next step's inputs are copied into the other on a copy stream
        bufs = [cl, {k: (torch.empty_like(v) if hasattr(v, "copy_") else v)
                     for k, v in cl.items()}]
        cstream = torch.cuda.Stream()
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        free = [torch.cuda.Event(), torch.cuda.Event()]

        def put(i):
            with torch.cuda.stream(cstream):
                cstream.wait_event(free[i % 2])
                for k, v in host.items():
                    if v is not None:
                        bufs[i % 2][k].copy_(v, non_blocking=True)
                ready[i % 2].record(cstream)

        def run(buf):
            tr.load(buf)
            ck(L.tpc_find_tracks_async(h), "find")
            ck(L.tpc_refit(h, 1, P(out["params"]), P(out["cov"]), P(out["x"]), P(out["chi2"]),
                           P(out["ndf"]), P(out["status"]), P(out["rej"])), "refit")
            ck(L.tpc_refit_backward(h, P(ones), P(gy), P(gz), P(gc)), "backward")

        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for f in free:
            f.record(stream)
        put(0)
        for i in range(args.steps):
            if i + 1 < args.steps:
                put(i + 1)
            stream.wait_event(ready[i % 2])
            run(bufs[i % 2])
            free[i % 2].record(stream)
            res_h[:cap_tr * 5].view(cap_tr, 5).copy_(out["params"], non_blocking=True)
            res_h[cap_tr * 5:cap_tr * 6].copy_(out["chi2"], non_blocking=True)
        b.record(stream)
        barrier()
        _, _, e2e_value = aggregate(a.elapsed_time(b), n * args.steps, dist, dev)
        e2e = dict(value=e2e_value, unit=UNIT,
                   h2d_bytes_per_step=int(h2d), d2h_bytes_per_step=int(d2h),
                   note="inputs copied from pinned host memory every step on a second "
                        "stream into one of two device buffers (overlapping the previous "
                        "step), track parameters and chi2 copied back every step")

    # ---- frames in flight: every context runs its own frame on its own
    # stream; a step issues one full pass per context, the step ends when
    # all have finished (inputs resident, L2 flushed before each step)
    pipe = None
    if others:
        pipe = pipelined(args, torch, dist, dev, flush, stream,
                         [dict(ev=ev, seed=cfg["seed"], stream=stream, tr=tr, cl=cl)] + others,
                         barrier)

    # ---- rooflines of the top kernels: HBM (algorithmic bytes) and FP32 ALU
    # (executed single-precision operations from the ncu capture, scaled by
    # the launch's units); the dominant kernel's bound is the one it is
    # closer to
    counts = dict(n=n, mode=1 if ev.mode == "time" else 0, n_tracks=nt, n_assigned=na,
                  n_tracklets=ntl, sum_nh=sum_nh, n_events=ev.n_events)
    units = dict(cluster=n, tracklet_hit=sum_nh, assigned_cluster=na, track=nt)
    peaks = load_peaks()
    sm_mhz = clk["sm_mhz"] or peaks["sm_max_mhz"]
    alu_peak = alu_peak_gflops(torch.cuda.get_device_properties(dev).multi_processor_count,
                               sm_mhz)
    tot = sum(v[1] for v in kstats_all.values()) or 1.0

    def kernel_roofs(k, per_launch_ms):
        ab = algorithmic_bytes(k, counts)
        gbs = ab / (per_launch_ms / 1000.0) / 1e9 if ab else None
        hbm = dict(bound="hbm", achieved=gbs, peak=peaks["hbm_gbs"], unit="GB/s",
                   frac=(gbs / peaks["hbm_gbs"]) if gbs else None,
                   traffic=ncu_traffic(k, units), algorithmic_bytes=ab,
                   peak_source=peaks["source"] + " (burst copy)")
        fl = ncu_flops(k, units)
        gfl = fl / (per_launch_ms / 1000.0) / 1e9 if fl else None
        alu = dict(bound="alu", achieved=gfl, peak=alu_peak, unit="GFLOP/s",
                   frac=(gfl / alu_peak) if gfl else None, flops=fl,
                   traffic=ncu_traffic(k, units),
                   peak_source=f"148 SMs x 128 FP32 lanes x 2 x sampled SM clock "
                               f"{sm_mhz:.0f} MHz",
                   flops_source="executed FP32 operations per unit from the ncu capture "
                                "(profiles/ncu_alu.json; FFMA = 2), null once the kernel "
                                "changed")
        return hbm, alu

    roof = None
    alu_kernels = {}
    for k in ("k_tracklets", "k_refit", "k_refit_bwd"):
        if k in kstats_all:
            nl, kms = kstats_all[k]
            hb, al = kernel_roofs(k, kms / nl)
            alu_kernels[k] = dict(ms_per_launch=kms / nl, alu=al, hbm=hb)
    if dom and dom in kstats:
        nl, kms = kstats[dom]
        per_launch_ms = kms / nl
        hb, al = kernel_roofs(dom, per_launch_ms)
        main, other = (al, hb) if (al["frac"] or 0.0) > (hb["frac"] or 0.0) else (hb, al)
        roof = dict(main, kernel=dom, ms_per_launch=per_launch_ms,
                    share=kstats_all[dom][1] / tot,
                    timing="CUDA events around each of its launches in the timed region",
                    bound_choice="the resource the kernel is closer to: larger fraction of "
                                 "HBM (algorithmic bytes) and FP32 ALU (executed operations)",
                    other=other)
    kernels = {k: dict(launches=v[0], ms_per_step=v[1] / n_prof, share=v[1] / tot)
               for k, v in sorted(kstats_all.items(), key=lambda kv: -kv[1][1])}

    def step_bytes_of(ks, nsteps):
        b = 0
        for k, v in ks.items():
            ab = None if k.startswith("k_row_sort") else algorithmic_bytes(k, counts)
            if ab:
                b += ab * v[0] / nsteps          # launches per step
        if any(k.startswith("k_row_sort") for k in ks):
            b += algorithmic_bytes("k_row_sort", counts)
        return b

    # the whole step against the HBM roofline: the algorithmic bytes of every
    # modelled kernel of a step over the step's time
    step_bytes = step_bytes_of(kstats_all, n_prof)
    step_ms = total_ms / args.steps
    step_gbs = step_bytes / (step_ms / 1000.0) / 1e9
    step_hbm = dict(algorithmic_bytes=step_bytes, achieved=step_gbs, unit="GB/s",
                    peak=peaks["hbm_gbs"], frac=step_gbs / peaks["hbm_gbs"],
                    note="algorithmic bytes of all modelled kernels of one step (times "
                         "their launches per step; the row sorts together once) over the "
                         "step time, of measured HBM copy bandwidth")
    # find + refit: the method's own 180 bytes per cluster (compulsory
    # reads and writes of the hot path's steps) and this code's kernel model
    fr_bytes = step_bytes_of(fr_kstats, args.steps)
    fr_s = fr_ms / 1000.0
    find_refit = dict(
        value=fr_value, unit=UNIT, ms_per_step=fr_ms, steps=args.steps,
        hbm_180=dict(bytes_per_cluster=180, achieved=180 * n / fr_s / 1e9, unit="GB/s",
                     peak=peaks["hbm_gbs"], frac=180 * n / fr_s / 1e9 / peaks["hbm_gbs"],
                     frac_of_nominal_8tbs=180 * n / fr_s / 1e9 / 8000.0),
        hbm_kernels=dict(algorithmic_bytes=fr_bytes, achieved=fr_bytes / fr_s / 1e9,
                         unit="GB/s", frac=fr_bytes / fr_s / 1e9 / peaks["hbm_gbs"]),
        note="load, find and refit (no checkpoints, no adjoint) per step, L2 flushed "
             "before each, CUDA events; hbm_180: 180 algorithmic bytes per cluster for "
             "the hot path's steps; hbm_kernels: the per-kernel model of this code")

    compression = None if args.no_merge else compression_stage(tr, cl, flush, stream)
    merge = None if args.no_merge else merge_stage(tr, cl, ev, flush, stream)
    if merge is not None:
        merge["chain"] = merge_chain(tr, cl, n, flush, stream, min(args.steps, 50))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(ev, geo, secs=sample_sectors(ev))

    serial = dict(value=value, unit=UNIT, ms_per_step=total_ms / args.steps,
                  graph_replay=graph_replay, find_refit=dict(value=fr_value, ms_per_step=fr_ms),
                  e2e=e2e, note="one context, one frame per step (the timed region of the "
                                "per-kernel events)")
    step_ms = total_ms / args.steps
    head_value, head_ms, head_e2e = value, step_ms, e2e
    head_cfg = dict(cfg)
    if pipe is not None:
        head_value, head_ms, head_e2e = pipe["value"], pipe["ms_per_step"], pipe["e2e"]
        graph_replay = pipe["graph_replay"]
        head_cfg["workload"] = (f"{len(others) + 1} frames in flight, each on its own context "
                                f"and CUDA stream: " + cfg["workload"])
        head_cfg["seed"] = pipe["seeds"]
        head_cfg["n_clusters"] = pipe["clusters_per_step"]
        find_refit = dict(find_refit, value=pipe["find_refit"]["value"],
                          ms_per_step=pipe["find_refit"]["ms_per_step"],
                          hbm_180=pipe["find_refit"]["hbm_180"],
                          serial=dict(value=fr_value, ms_per_step=fr_ms,
                                      hbm_180=find_refit["hbm_180"]))
    line = dict(metric=METRIC, value=head_value, unit=UNIT, n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=head_ms, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f32 (f64 timestamps and gradient sums)",
                data="synthetic",
                config=dict(head_cfg, l2="flushed before every timed step (256 MB write)",
                            tuning=dict(tuning, chosen=how),
                            parallelism=f"replicas x{world}, independent frames per GPU",
                            launch="one CUDA graph per step" if args.graph else "stream launches"),
                serial=serial, pipeline=pipe and {k: v for k, v in pipe.items()
                                                  if k not in ("e2e", "find_refit")},
                tracks_per_s=aggregate(total_ms, nt * args.steps, dist, dev)[2],
                n_tracks=nt, n_assigned=na, n_tracklets=ntl,
                refit_fwd_ms=t_fwd, refit_fwd_nosave_ms=t_fwd_nosave, adjoint_ms=t_bwd,
                adjoint_vs_fwd=(t_bwd / t_fwd_nosave if t_bwd is not None and t_fwd_nosave > 0
                                else None),
                roofline=roof, step_hbm=step_hbm, find_refit=find_refit,
                alu_roofline=alu_kernels, kernels=kernels,
                kernels_timing=f"separate pass of {n_prof} steps with every launch timed",
                gpu_launches=launches,
                graph_replay=graph_replay, track_quality=quality, merge_stage=merge,
                compression=compression,
                clocks=clk, e2e=head_e2e, cpu_baseline=cpu)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------ frames in flight
def pipelined(args, torch, dist, dev, flush, stream0, ctxs, barrier):
    """Throughput with one frame per context in flight on its own stream.
    ctxs: dicts with ev, seed, stream, tr (a Tracker on that stream), cl
    (device inputs). Returns the timed step (load, find, refit with
    checkpoints, adjoint), its graph replay, find + refit, and the end to
    end through host buffers."""
    import ctypes as C
    from paper_1811_11481_b300.binding import TPC_GRAD_CALIB_SIZE
    P = lambda t: C.c_void_p(t.data_ptr())
    for c in ctxs:
        n = c["ev"].n
        cap = n // 10 + 1
        f = lambda *sh, **kw: torch.empty(*sh, device=dev, **kw)
        c["out"] = dict(params=f(cap, 5), cov=f(cap, 15), x=f(cap), chi2=f(cap),
                        ndf=f(cap, dtype=torch.int32), status=f(cap, dtype=torch.int32),
                        rej=f(n + 1, dtype=torch.uint8))
        c["ones"] = torch.ones(cap, device=dev)
        c["gy"], c["gz"] = f(n + 1), f(n + 1)
        c["gc"] = f(TPC_GRAD_CALIB_SIZE, dtype=torch.float64)

    def issue(c, save=True, backward=True):
        tr, o = c["tr"], c["out"]
        L, h = tr.L, tr.h

        def ck(st, what):
            if st != 0:
                raise RuntimeError(f"{what}: status {st}: {L.tpc_last_error(h).decode()}")
        tr.load(c["cl"])
        ck(L.tpc_find_tracks_async(h), "find")
        ck(L.tpc_refit(h, int(save), P(o["params"]), P(o["cov"]), P(o["x"]), P(o["chi2"]),
                       P(o["ndf"]), P(o["status"]), P(o["rej"])), "refit")
        if backward:
            ck(L.tpc_refit_backward(h, P(c["ones"]), P(c["gy"]), P(c["gz"]), P(c["gc"])),
               "backward")

    def timed(run_one, steps):
        evs = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream0)
            for c in ctxs[1:]:
                c["stream"].wait_event(e0)
            for c in ctxs:
                run_one(c)
            for c in ctxs[1:]:
                d = torch.cuda.Event()
                d.record(c["stream"])
                stream0.wait_event(d)
            e1.record(stream0)
            evs.append((e0, e1))
        barrier()
        return float(np.sum([a.elapsed_time(b) for a, b in evs]))

    units = sum(c["ev"].n for c in ctxs)
    for _ in range(max(3, args.warmup)):
        for c in ctxs:
            issue(c)
    barrier()
    ms = timed(issue, args.steps)
    tot, _, value = aggregate(ms, units * args.steps, dist, dev)
    res = dict(value=value, unit=UNIT, ms_per_step=tot / args.steps, frames=len(ctxs),
               seeds=[c["seed"] for c in ctxs], clusters_per_step=units,
               note="one frame per context in flight, each context on its own CUDA stream; "
                    "a step is one full pass (load, find, refit with checkpoints, adjoint) of "
                    "every frame; L2 flushed before each step")
    # the same as one captured graph per context
    for c in ctxs:
        c["stream"].synchronize()
        c["tr"].graph_begin()
        issue(c)
        c["tr"].graph_end()
    barrier()
    g_ms = timed(lambda c: c["tr"].graph_launch(), args.steps)
    g_tot, _, g_value = aggregate(g_ms, units * args.steps, dist, dev)
    res["graph_replay"] = dict(value=g_value, unit=UNIT, ms_per_step=g_tot / args.steps,
                               steps=args.steps, note="one CUDA graph per context and step")
    # find + refit (no checkpoints, no adjoint)
    fr_ms = timed(lambda c: issue(c, save=False, backward=False), args.steps)
    fr_tot, _, fr_value = aggregate(fr_ms, units * args.steps, dist, dev)
    fr_s = fr_tot / args.steps / 1000.0
    peak = load_peaks()["hbm_gbs"]
    res["find_refit"] = dict(value=fr_value, ms_per_step=fr_tot / args.steps,
                             hbm_180=dict(bytes_per_cluster=180,
                                          achieved=180 * units / fr_s / 1e9, unit="GB/s",
                                          peak=peak, frac=180 * units / fr_s / 1e9 / peak,
                                          frac_of_nominal_8tbs=180 * units / fr_s / 1e9 / 8000.0))
    # end to end: each context copies its next frame from pinned host memory
    # on its own copy stream into one of two device buffers while the
    # current one runs, and copies the track parameters and chi2 back
    res["e2e"] = None
    if not args.no_e2e:
        h2d = d2h = 0
        for c in ctxs:
            c["host"] = {k: v.cpu().pin_memory() for k, v in c["cl"].items()
                         if hasattr(v, "cpu") and v is not None}
            cap = c["out"]["chi2"].numel()
            c["res_h"] = torch.empty(cap * 6, dtype=torch.float32).pin_memory()
            c["bufs"] = [c["cl"], {k: (torch.empty_like(v) if hasattr(v, "copy_") else v)
                                   for k, v in c["cl"].items()}]
            c["cstream"] = torch.cuda.Stream()
            c["ready"] = [torch.cuda.Event(), torch.cuda.Event()]
            c["free"] = [torch.cuda.Event(), torch.cuda.Event()]
            h2d += sum(v.numel() * v.element_size() for v in c["host"].values())
            d2h += c["res_h"].numel() * 4

        def put(c, i):
            with torch.cuda.stream(c["cstream"]):
                c["cstream"].wait_event(c["free"][i % 2])
                for k, v in c["host"].items():
                    c["bufs"][i % 2][k].copy_(v, non_blocking=True)
                c["ready"][i % 2].record(c["cstream"])

        def run(c, i):
            s = c["stream"]
            s.wait_event(c["ready"][i % 2])
            c["cl_saved"] = c["cl"]
            c["cl"] = c["bufs"][i % 2]
            issue(c)
            c["cl"] = c["cl_saved"]
            c["free"][i % 2].record(s)
            cap = c["out"]["chi2"].numel()
            with torch.cuda.stream(s):
                c["res_h"][:cap * 5].view(cap, 5).copy_(c["out"]["params"], non_blocking=True)
                c["res_h"][cap * 5:].copy_(c["out"]["chi2"], non_blocking=True)

        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream0)
        for c in ctxs:
            c["stream"].wait_event(a)
            c["cstream"].wait_event(a)
            for f in c["free"]:
                f.record(c["stream"])
            put(c, 0)
        for i in range(args.steps):
            for c in ctxs:
                if i + 1 < args.steps:
                    put(c, i + 1)
                run(c, i)
        for c in ctxs[1:]:
            d = torch.cuda.Event()
            d.record(c["stream"])
            stream0.wait_event(d)
        b.record(stream0)
        barrier()
        _, _, e_value = aggregate(a.elapsed_time(b), units * args.steps, dist, dev)
        res["e2e"] = dict(value=e_value, unit=UNIT, h2d_bytes_per_step=int(h2d),
                          d2h_bytes_per_step=int(d2h),
                          note="every step each context's frame is copied from pinned host "
                               "memory on that context's copy stream into one of two device "
                               "buffers (overlapping its previous step and the other "
                               "contexts), run, and its track parameters and chi2 copied back")
    return res


# ---------------------------------------------------------- CPU baseline
def _subset(ev, secs):
    class S:
        pass
    m = np.isin(ev.sector, secs)
    s = S()
    for k in ("mode", "n_events", "tf_start"):
        setattr(s, k, getattr(ev, k))
    for k in ("y", "z", "t", "row", "sector", "flags", "event"):
        v = getattr(ev, k)
        setattr(s, k, None if v is None else v[m])
    return s, int(m.sum())


def sample_sectors(ev, target=300_000):
    """The first sectors of the workload holding at least `target` clusters
    (a bounded sample: about 20 s of single-thread oracle work)."""
    cnt = np.bincount(np.asarray(ev.sector, np.int64), minlength=36)
    secs, tot = [], 0
    for k in range(36):
        secs.append(k)
        tot += int(cnt[k])
        if tot >= target:
            break
    return secs


def oracle_pass(ev, geo, secs):
    """One pass of the oracle as it stands over sectors 'secs' of the
    workload: find (FP32 mirror), refit (FP64) and tape gradient. Returns
    (clusters, seconds)."""
    import oracle
    import synth
    from paper_1811_11481_b300.config import default_params
    sub, n = _subset(ev, secs)
    t0 = time.time()
    o = oracle.Oracle(sub, geo, default_params(), synth.nominal_calib())
    f = o.find(32)
    tr = f["tracks"]
    r = o.refit(tr["track_start"], tr["cluster_idx"], tr["that"], prec=64)
    o.refit_grad(tr["track_start"], tr["cluster_idx"], tr["that"], r["seeds"], r["rej"])
    dt = time.time() - t0
    o.close()
    return n, dt


def cpu_baseline(ev, geo, secs):
    """The oracle as it stands on the sectors 'secs' of the same workload,
    on all host cores (its loops over hits, start hits, tracks and clusters
    in parallel) and on one."""
    import oracle
    ncores = os.cpu_count() or 1
    oracle.threads(ncores)
    used = oracle.threads()
    n, dt = oracle_pass(ev, geo, secs)
    oracle.threads(1)
    n1, dt1 = oracle_pass(ev, geo, secs)
    oracle.threads(ncores)
    what = (f"sectors {secs[0]}..{secs[-1]} of the same workload ({n} clusters): find (FP32 "
            f"mirror) + refit (FP64) + tape-AD gradient")
    return dict(value=n / dt, unit=UNIT, cores=used, kind="oracle", host_cores=ncores,
                sample=f"{what}, {dt:.1f} s on {used} threads",
                single_thread=dict(value=n1 / dt1, unit=UNIT, cores=1, seconds=dt1),
                speedup_all_cores=dt1 / dt)


# ------------------------------------------------------- reference arm
def run_reference(args):
    """The reference arm: the oracle as it stands on the host cores (all of
    them), each step one sector of the same workload, rotating over the
    sectors."""
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    import oracle
    import synth
    geo = synth.geometry()
    wl = "timeframe" if args.workload == "adjoint" else args.workload
    ev, cfg = make_workload(wl, 0, args.collisions)
    ncores = os.cpu_count() or 1
    oracle.threads(ncores)
    used = oracle.threads()
    for w in range(args.warmup):
        oracle_pass(ev, geo, [w % 36])
    tot_n, tot_t = 0, 0.0
    for k in range(args.steps):
        n, dt = oracle_pass(ev, geo, [k % 36])
        tot_t += dt
        tot_n += n
    v = tot_n / tot_t
    cb = dict(value=v, unit=UNIT, cores=used, kind="oracle", host_cores=ncores,
              sample=f"one sector of the workload per step (sector k mod 36 at step k), "
                     f"find (FP32 mirror) + refit (FP64) + tape-AD gradient, {used} threads")
    line = dict(impl="reference", metric=METRIC, value=v, unit=UNIT,
                n_gpus=int(os.environ.get("WORLD_SIZE", args.gpus)), steps=args.steps,
                warmup=args.warmup, ms_per_step=1000.0 * tot_t / args.steps,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64 (oracle)",
                data="synthetic", config=cfg, cpu_baseline=cb,
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))


def identifiable_error(geo, ev, ts, ci, tc, theta, theta_true):
    """RMS (cm) over the assigned clusters of the error of their calibrated
    positions under theta against theta_true (time-frame mode), after
    removing from each track the part its own fit absorbs: a least-squares
    parabola in x from the error in y (the helix's offset, direction and
    curvature), a straight line in x from the error in z. The calibration
    parameters move freely along the directions this leaves out (reading of
    the identifiable subspace); spline values by the generator's evaluator."""
    from synth.events import eval_distortion
    ts = np.asarray(ts, np.int64)
    ci = np.asarray(ci, np.int64)
    lens = np.diff(ts)
    st = ts[:-1]
    x = np.asarray(geo.row_x, np.float64)[ev.row[ci]]
    sec = ev.sector[ci].astype(np.int64)
    sg = np.where(sec < 18, 1.0, -1.0)
    tcl = np.repeat(np.asarray(tc, np.float64), lens)
    L = float(geo.drift_length)
    y = ev.y[ci].astype(np.float64)

    def positions(th):
        th = np.asarray(th, np.float64)
        z = sg * (L - th[0] * ((ev.t[ci] - th[1]) - tcl))
        dy, dz = eval_distortion(geo, th[2:].astype(np.float32).reshape(36, 2, 8, 8, 8), sec, x,
                                 y, np.abs(z))
        return y + dy, z + dz

    def resid(e, deg):
        xm = np.repeat(np.add.reduceat(x, st) / lens, lens)
        u = (x - xm) / 100.0
        P = np.stack([u ** k for k in range(deg + 1)], 1)
        A = np.stack([np.stack([np.add.reduceat(P[:, i] * P[:, j], st) for j in range(deg + 1)],
                               1) for i in range(deg + 1)], 1)
        b = np.stack([np.add.reduceat(P[:, i] * e, st) for i in range(deg + 1)], 1)
        c = np.linalg.solve(A + 1e-12 * np.eye(deg + 1), b[..., None])[..., 0]
        return e - np.einsum("nk,nk->n", P, np.repeat(c, lens, axis=0))

    Y, Z = positions(theta)
    Yt, Zt = positions(theta_true)
    ry, rz = resid(Y - Yt, 2), resid(Z - Zt, 1)
    return float(np.sqrt((ry @ ry + rz @ rz) / (2 * ry.size)))


def recovery(tr, ev, geo, ts, ci, tc, sids, steps=600, tikhonov=1e-6):
    """Calibration recovery on the adjoint workload: vertex pseudo-
    measurements for each particle's first outgoing leg, then gradient
    descent on v_drift, t0 and the spline from the nominal calibration.
    Reports chi2/ndf against the true calibration's and the identifiable
    position error before and after."""
    import torch
    import synth
    from paper_1811_11481_b300.autograd import RefitChi2, calib_vector, recover_calibration
    lab = ev.label[np.asarray(ci, np.int64)[np.asarray(ts[:-1], np.int64)]]
    zv = np.asarray(ev.part["zv"], np.float64)[lab]
    zv[np.asarray(sids) % 4 != 0] = np.nan
    tr.set_vertex(torch.as_tensor(zv.astype(np.float32)), 0.01)
    nom, true = synth.nominal_calib(), ev.calib_true
    cl = tr._keep["clusters"]
    th_nom = calib_vector(nom.vdrift, nom.t0, nom.spline, tr.dev)
    th_true = calib_vector(true.vdrift, true.t0, true.spline, tr.dev)

    def chi2ndf(th):
        with torch.no_grad():
            c = RefitChi2.apply(th, cl["y"], cl["t"], tr)
        return float(c.sum()) / max(1, tr.ndf_sum)
    l_true, l_nom = chi2ndf(th_true), chi2ndf(th_nom)
    t0 = time.time()
    theta, hist = recover_calibration(tr, th_nom, steps=steps, lr_spline=0.02, lr_vdrift=1e-3,
                                      lr_t0=1e-3, tikhonov=tikhonov)
    secs = time.time() - t0
    l_end = chi2ndf(theta)
    th_n, th_t, th_e = (a.cpu().numpy() for a in (th_nom, th_true, theta))
    e_nom = identifiable_error(geo, ev, ts, ci, tc, th_n, th_t)
    e_end = identifiable_error(geo, ev, ts, ci, tc, th_e, th_t)
    tr.set_vertex(None)
    return dict(tracks=int(len(ts) - 1), vertex_tracks=int(np.sum(~np.isnan(zv))),
                steps=steps, tikhonov=tikhonov, seconds=secs,
                chi2ndf_true=l_true, chi2ndf_nominal=l_nom, chi2ndf_recovered=l_end,
                chi2ndf_vs_true=l_end / l_true,
                identifiable_error_cm=dict(nominal=e_nom, recovered=e_end,
                                           reduction=e_nom / e_end),
                vdrift_error_left=abs(th_e[0] - true.vdrift) / abs(nom.vdrift - true.vdrift),
                t0_error_left=abs(th_e[1] - true.t0) / abs(nom.t0 - true.t0),
                note="vertex z of each particle's first outgoing leg as a pseudo-measurement "
                     "(sigma 0.01 cm), Adam on v_drift, t0 and the spline from the nominal "
                     "calibration with a Tikhonov term on the spline; the identifiable error "
                     "is the calibrated positions' error left after each track's own fit "
                     "absorbs what it can (v_drift and t0 alone remain degenerate with each "
                     "sector's constant and z-linear spline modes)")


def run_adjoint(args):
    """Adjoint-refit workload: ten central events in continuous readout,
    generated with a distorted calibration (v_drift +0.5 %, t0 +0.05 us, a
    per-sector spline up to 1 cm); truth-assigned tracks of at least 30
    clusters (~100k) with fixed assignments. A step is the refit with
    checkpoints (calibration transform included: the calibration is set again
    each step, as a calibration loop does) and the adjoint back to the
    cluster coordinates and the calibration, at a calibration halfway between
    nominal and true (so that the spline is evaluated and differentiated)."""
    import torch
    import torch.distributed as dist
    import synth
    from paper_1811_11481_b300.binding import TPC_GRAD_CALIB_SIZE, Tracker
    local = int(os.environ.get("LOCAL_RANK", 0))
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    geo = synth.geometry()
    ev = synth.make_adjoint(seed=4 + rank)
    ts, ci, tc, sids = synth.truth_tracks(ev, 30)
    nom, true = synth.nominal_calib(), ev.calib_true
    work = torch.cuda.Stream()
    torch.cuda.set_stream(work)
    tr = Tracker(geo, stream=work)
    tr.set_calib(0.5 * (nom.vdrift + true.vdrift), 0.5 * (nom.t0 + true.t0),
                 0.5 * np.asarray(true.spline, np.float32))
    cl = tr.upload(ev)
    tr.load(cl)
    dev = tr.dev
    tr.set_tracks(torch.as_tensor(ts.astype(np.int32), device=dev),
                  torch.as_tensor(ci.astype(np.int32), device=dev),
                  torch.as_tensor(tc, device=dev))
    nt, na = ts.size - 1, int(ts[-1])
    L, h = tr.L, tr.h
    import ctypes as C
    P = lambda t: C.c_void_p(t.data_ptr())
    f32 = lambda *sh: torch.empty(*sh, device=dev)
    out = dict(params=f32(nt, 5), cov=f32(nt, 15), x=f32(nt), chi2=f32(nt),
               ndf=torch.empty(nt, dtype=torch.int32, device=dev),
               status=torch.empty(nt, dtype=torch.int32, device=dev),
               rej=torch.empty(na, dtype=torch.uint8, device=dev))
    ones, gy, gz = torch.ones(nt, device=dev), f32(na), f32(na)
    gc = torch.empty(TPC_GRAD_CALIB_SIZE, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def ck(st, what):
        if st != 0:
            raise RuntimeError(f"{what}: status {st}: {L.tpc_last_error(h).decode()}")

    def fwd(save):
        ck(L.tpc_refit(h, int(save), P(out["params"]), P(out["cov"]), P(out["x"]),
                       P(out["chi2"]), P(out["ndf"]), P(out["status"]), P(out["rej"])), "refit")

    def bwd():
        ck(L.tpc_refit_backward(h, P(ones), P(gy), P(gz), P(gc)), "backward")

    # a step of a calibration loop sets the calibration it differentiates at
    # (here always the same values), so the refit re-applies the transform
    from paper_1811_11481_b300.binding import tpc_calib
    spl = torch.as_tensor(0.5 * np.asarray(true.spline, np.float32).reshape(-1), device=dev)
    cal = tpc_calib(0.5 * (nom.vdrift + true.vdrift), 0.5 * (nom.t0 + true.t0),
                    spl.data_ptr(), 85.0, 160.0)

    def setc():
        ck(L.tpc_set_calib(h, C.byref(cal)), "set_calib")

    def step():
        setc()
        fwd(True)
        bwd()

    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn, k):
        ev_ = []
        for _ in range(k):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            ev_.append((a, b))
        torch.cuda.synchronize()
        return float(np.sum([a.elapsed_time(b) for a, b in ev_]))

    for _ in range(max(3, args.warmup)):
        step()
    clocks = Clocks(local)
    clocks.start()
    t_end = time.time() + 1.5
    while time.time() < t_end:
        step()
    tr.profile(True)
    torch.cuda.synchronize()
    total = timed(step, args.steps)
    clk = clocks.stop()
    kstats, launches = tr.profile_read()
    tr.profile(False)
    t_fwd = timed(lambda: (setc(), fwd(False)), 20) / 20
    t_fwd_save = timed(lambda: (setc(), fwd(True)), 20) / 20
    fwd(True)
    t_bwd = timed(bwd, 20) / 20
    total_ms, _, value = aggregate(total, na * args.steps, dist, dev)
    st = out["status"].cpu().numpy()
    rec = None
    if not args.no_recovery and rank == 0:
        rec = recovery(tr, ev, geo, ts, ci, tc, sids)
    kernels = {k: dict(launches=v[0], ms_per_step=v[1] / args.steps)
               for k, v in sorted(kstats.items(), key=lambda kv: -kv[1][1])}
    line = dict(metric=METRIC, value=value, unit="assigned clusters/s", n_gpus=world,
                steps=args.steps, warmup=args.warmup, ms_per_step=total_ms / args.steps,
                higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32 (f64 timestamps and gradient sums)", data="synthetic",
                config=dict(workload="adjoint refit: 10 central events, continuous readout, "
                                     "injected calibration error, truth tracks >= 30 clusters",
                            seed=4 + rank, n_clusters=int(ev.n), n_tracks=nt, n_assigned=na,
                            calib="halfway between nominal and true (spline active), set "
                                  "again every step as in a calibration loop, so the refit "
                                  "re-applies the calibration transform",
                            l2="flushed before every timed step (256 MB write)"),
                tracks_per_s=aggregate(total, nt * args.steps, dist, dev)[2],
                refit_fwd_ms=t_fwd, refit_fwd_save_ms=t_fwd_save, adjoint_ms=t_bwd,
                adjoint_vs_fwd=t_bwd / t_fwd if t_fwd > 0 else None,
                fit_status_ok=float((st == 0).mean()), kernels=kernels, gpu_launches=launches,
                clocks=clk, recovery=rec)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
