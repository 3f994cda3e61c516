// Track-model compression (arXiv:1811.11481 Sec. 5: for the entropy
// reduction of the TPC data only the residuals of the clusters attached to
// tracks are stored, with respect to the track model, and the track is fitted
// in the distorted coordinate system so that calibration effects stay out of
// the residuals).
//
// Along each track (clusters in row order; the model restarts where the
// sector frame changes) the first cluster of a run is stored as quantised
// absolute (y, z), the second as the quantised difference to the first, and
// from then on the tracklet filter (straight-line seed through the first two
// decoded clusters, helix transport, Kalman update with each decoded
// cluster) predicts (y, z) at the next row: the residual is
// round((measured - predicted) / q). Every step works on the decoded
// cluster (prediction + residual * q), so that a decoder running the same
// arithmetic on the residuals reproduces the decoded clusters exactly; where
// the transport fails the prediction is the previous decoded cluster and the
// filter restarts. Measured z in the time-frame mode: the drift time turned
// into z with the track's collision time, without the distortion correction.
//
// k_compress  one thread per track.
//
// Compiled with -fmad=false and IEEE division and square root: the residuals
// are integers decided in single precision with one rounding per written
// operation.
#include "tpc_impl.h"

namespace tpc {
namespace {

constexpr int kCB = 128;
inline int nblk(int64_t n, int b) { return (int)((n + b - 1) / b); }

__global__ void __launch_bounds__(kCB) k_compress(Geo g, Cal c, ClIn cl, Params p, float qy,
                                                  float qz, int64_t cap_tr, const uint32_t* cnt,
                                                  const uint32_t* track_start,
                                                  const uint32_t* cluster_idx,
                                                  const double* t_coll, int32_t* ry_out,
                                                  int32_t* rz_out, float* dy_out,
                                                  float* dz_out) {
  int T = blockIdx.x * blockDim.x + threadIdx.x;
  int nt = (int)cnt[kCntTracks];
  if ((int64_t)nt > cap_tr) nt = (int)cap_tr;
  if (T >= nt) return;
  const float iqy = 1.0f / qy, iqz = 1.0f / qz;
  const float sig2 = p.sigma * p.sigma;
  uint32_t a = track_start[T], b = track_start[T + 1];
  double that = t_coll[T];
  float st[5], C[15], x = 0.0f;
  int frame = -1, j = 0;
  bool model = false;
  float px = 0.0f, pyd = 0.0f, pzd = 0.0f;  // previous decoded cluster
  for (uint32_t k = a; k < b; ++k) {
    uint32_t i = cluster_idx[k];
    int s = cl.sector[i], r = cl.row[i];
    int f = s % 18;
    float xr = g.rx[r];
    if (f != frame) {
      frame = f;
      j = 0;
      model = false;
    }
    float my = cluster_y(g, cl, i);
    float mz = abs_z(g, c, cl.mode, cl.mode == 0 ? cl.z[i] : 0.0f, cl.mode == 1 ? cl.t[i] : 0.0,
                     s, that);
    float prey = 0.0f, prez = 0.0f;
    bool absolute = j == 0;
    if (j >= 2 && model && propagate(g.kB, p.s_max, st, C, x, xr)) {
      prey = st[0];
      prez = st[1];
    } else if (!absolute) {
      prey = pyd;
      prez = pzd;
      model = false;
    }
    int32_t ry = (int32_t)nearbyintf((my - prey) * iqy);
    int32_t rz = (int32_t)nearbyintf((mz - prez) * iqz);
    float dy = prey + (float)ry * qy;
    float dz = prez + (float)rz * qz;
    ry_out[k] = ry;
    rz_out[k] = rz;
    if (dy_out) dy_out[k] = dy;
    if (dz_out) dz_out[k] = dz;
    if (j >= 1) {
      if (!model) {
        // (re)start: seed through the previous and this decoded cluster, then
        // the filter takes this cluster
        seed_two_points(st, C, x, p.c0t, px, pyd, pzd, xr, dy, dz);
        model = propagate(g.kB, p.s_max, st, C, x, xr);
      }
      if (model) apply_update(st, C, innovation(st, C, dy, dz, sig2, sig2));
    }
    px = xr;
    pyd = dy;
    pzd = dz;
    ++j;
  }
}

}  // namespace

void launch_compress(Prof* P, const Geo& g, const Cal& c, const ClIn& cl, const Params& p,
                     float qy, float qz, int64_t cap_tr, const uint32_t* cnt, const TrackBuf& tb,
                     int32_t* ry, int32_t* rz, float* dy, float* dz, cudaStream_t s) {
  if (cap_tr <= 0) return;
  TPC_LAUNCH(P, "k_compress", s,
             k_compress<<<nblk(cap_tr, kCB), kCB, 0, s>>>(g, c, cl, p, qy, qz, cap_tr, cnt,
                                                          tb.track_start, tb.cluster_idx,
                                                          tb.t_coll, ry, rz, dy, dz));
}

}  // namespace tpc
