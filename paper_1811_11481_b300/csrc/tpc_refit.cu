// Final Kalman refit (arXiv:1811.11481 Sec. 3) and its adjoint.
//
// k_refit      one thread per track: three-point circle seed, then three
//              passes (inward, outward, inward) of the full Kalman filter
//              with rejection of clusters whose predicted chi2 exceeds the
//              cut; passes 2 and 3 start from the previous pass's covariance
//              times refit_inflate. With checkpointing, the filter state
//              before every step is stored for the adjoint.
// k_refit_bwd  one thread per track: reverse sweep over the three passes
//              (rejections and seed held fixed), recomputing each step from
//              its checkpoint. The transport Jacobian depends on the state,
//              so its second-order term is formed with a forward-mode dual
//              number in (sin phi, tan lambda, q/pT).
// k_calib_grad one warp per range of assigned clusters: chain rule through
//              the calibration transform (drift time to z, distortion
//              spline); spline gradients summed in registers per cell and
//              added to 64-bit fixed-point totals, so that the gradient is
//              reproducible bit for bit.
// k_calib_reduce sums the float64 (v_drift, t0) partials in block order and
//              converts the spline sums back to float64.
#include "tpc_impl.h"
#include "tpc_refit_core.cuh"

namespace tpc {
namespace {

constexpr int kB = 128;

RefitCfg make_cfg(const Geo& g, const Params& p) {
  RefitCfg c;
  c.kB = g.kB;
  c.s_max = p.s_max;
  c.sigma = p.sigma;
  c.flag_scale[0] = p.split_scale;
  c.flag_scale[1] = p.single_row_scale;
  c.flag_scale[2] = p.single_time_scale;
  c.flag_scale[3] = p.edge_scale;
  c.flag_scale[4] = p.shared_scale;
  c.chi2_out = p.chi2_out;
  c.refit_inflate = p.refit_inflate;
  c.min_acc_reject = p.min_acc_reject;
  for (int i = 0; i < 5; ++i) c.c0r[i] = p.c0r[i];
  set_frame_rotations(c);
  c.field_on = g.field_on;
  for (int i = 0; i < 30; ++i) c.field[i] = g.field[i];
  return c;
}

// Counting sort of the tracks by decreasing cluster count, so that the
// threads of a warp run tracks of similar length.
constexpr int kLenBins = 256;
__global__ void k_len_init(uint32_t* hist) {
  int i = threadIdx.x;
  hist[i] = 0u;
  hist[kLenBins + i] = 0u;
}
__device__ __forceinline__ int len_bin(const uint32_t* ts, int T) {
  uint32_t n = ts[T + 1] - ts[T];
  return kLenBins - 1 - (int)(n < (uint32_t)(kLenBins - 1) ? n : (uint32_t)(kLenBins - 1));
}
__global__ void k_len_hist(const uint32_t* cnt, const uint32_t* ts, uint32_t* hist) {
  int T = blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= (int)cnt[kCntTracks]) return;
  warp_counter_add1(hist, (uint32_t)len_bin(ts, T));
}
__global__ void k_len_scan(uint32_t* hist) {
  __shared__ uint32_t s[kLenBins];
  int i = threadIdx.x;
  s[i] = hist[i];
  __syncthreads();
  if (i == 0) {
    uint32_t acc = 0;
    for (int k = 0; k < kLenBins; ++k) {
      uint32_t v = s[k];
      s[k] = acc;
      acc += v;
    }
  }
  __syncthreads();
  hist[i] = s[i];
}
__global__ void k_len_scatter(const uint32_t* cnt, const uint32_t* ts, uint32_t* hist,
                              uint32_t* order, uint32_t* slot, uint8_t* multi) {
  int T = blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= (int)cnt[kCntTracks]) return;
  int b = len_bin(ts, T);
  uint32_t pos = hist[b] + warp_counter_add1(hist + kLenBins, (uint32_t)b);
  order[pos] = (uint32_t)T;
  slot[T] = pos;
  multi[T] = 0;  // set by k_interleave for tracks across sector frames
}

// Longest track of each warp of thread slots.
__global__ void k_warp_len(const uint32_t* cnt, const uint32_t* ts, const uint32_t* order,
                           uint32_t* wlen) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int nt = (int)cnt[kCntTracks];
  uint32_t n = 0;
  if (tid < nt) {
    int T = (int)order[tid];
    n = ts[T + 1] - ts[T];
  }
  uint32_t m = __reduce_max_sync(0xffffffffu, n);
  if ((threadIdx.x & 31) == 0 && tid < nt) wlen[tid >> 5] = m;
}

// Single block: exclusive scan of the warp lengths.
__global__ void k_warp_scan(const uint32_t* cnt, const uint32_t* wlen, uint32_t* wbase) {
  __shared__ uint32_t carry;
  __shared__ uint32_t ws[32];
  int nw = ((int)cnt[kCntTracks] + 31) / 32;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  for (int b0 = 0; b0 < nw; b0 += blockDim.x) {
    int i = b0 + threadIdx.x;
    uint32_t v = i < nw ? wlen[i] : 0u;
    uint32_t x = v;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
      uint32_t s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0u;
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      ws[lane] = s;
    }
    __syncthreads();
    uint32_t excl = (w > 0 ? ws[w - 1] : 0u) + x - v;
    if (i < nw) wbase[i] = carry + excl;
    __syncthreads();
    if (threadIdx.x == 0) carry += ws[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) wbase[nw] = carry;
}

__device__ __forceinline__ Lay warp_layout(const uint32_t* wbase, const uint32_t* wlen, int tid) {
  int w = tid >> 5, lane = tid & 31;
  Lay l;
  l.base = (size_t)wbase[w] * 32 + lane;
  l.stride = 32;
  l.L = (int)wlen[w];
  l.ck_base = (size_t)3 * wbase[w] * 32 * kCk + lane;
  l.ck_step = 32 * kCk;
  l.ck_comp = 32;
  return l;
}

// Copy each track's calibrated clusters into the warp-interleaved layout.
// One thread per assigned cluster: reads are coalesced, each value goes to
// its place in its warp's interleaved block.
__global__ void k_interleave(const uint32_t* cnt, TrackIn in, const uint32_t* asg_track,
                             const uint32_t* slot, const uint32_t* wbase, float* w_yc,
                             float* w_zc, uint32_t* w_meta, uint8_t* multi) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= (int)cnt[kCntAssigned]) return;
  uint32_t T = asg_track[j];
  if (T >= cnt[kCntTracks]) return;
  uint32_t sl = slot[T];
  uint32_t a = in.track_start[T];
  size_t pos = ((size_t)wbase[sl >> 5] + (j - a)) * 32 + (sl & 31);
  uint32_t m = in.meta[j];
  w_yc[pos] = in.yc[j];
  w_zc[pos] = in.zc[j];
  w_meta[pos] = m;
  if (frame_of(m) != frame_of(in.meta[a])) multi[T] = 1;
}

template <bool kField>
__global__ void __launch_bounds__(kB) k_refit(Geo g, RefitCfg p, const uint32_t* cnt,
                                               const uint32_t* order, const uint32_t* wbase,
                                               const uint32_t* wlen, const uint32_t* track_start,
                                               TrackIn win, float* seed_out, uint8_t* rej,
                                               int32_t* status, float* ckpt, int save,
                                               float* o_params, float* o_cov, float* o_x,
                                               float* o_chi2, int32_t* o_ndf, int32_t* o_status,
                                               uint8_t* o_rej, const uint8_t* multi,
                                               const float* vz, float vvar, float* vck,
                                               uint32_t* err) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (int)cnt[kCntTracks]) return;
  int T = (int)order[tid];
  uint32_t a = track_start[T];
  uint32_t b = track_start[T + 1];
  if (b < a || b > cnt[kCntAssigned]) {  // invalid CSR: leave the track alone
    status[T] = 3;
    if (o_status) o_status[T] = 3;
    atomicOr(err, kErrArg);
    return;
  }
  int n = (int)(b - a);
  Lay ly = warp_layout(wbase, wlen, tid);
  Vertex vx{vz ? vz[T] : NAN, vvar, (vz && save) ? vck + (size_t)T * kVtxCk : nullptr};
  RefitOut o = refit_track<kField>(g, p, win, ly, n, rej, seed_out + (size_t)T * 5,
                                   save ? ckpt : nullptr, multi[T] != 0, vx);
  if (o.status == 0 && !(fabsf(o.chi2) < 1.0e30f && fabsf(o.st[4]) < 1.0e30f))
    atomicOr(err, kErrNumeric);
  if (o.status != 0) {
    o.chi2 = 0.0f;
    o.ndf = 0;
  }
  status[T] = o.status;
  if (o_status) o_status[T] = o.status;
  if (o_params)
#pragma unroll
    for (int i = 0; i < 5; ++i) o_params[(size_t)T * 5 + i] = o.st[i];
  if (o_cov)
#pragma unroll
    for (int i = 0; i < 15; ++i) o_cov[(size_t)T * 15 + i] = o.C[i];
  if (o_x) o_x[T] = o.x;
  if (o_chi2) o_chi2[T] = o.chi2;
  if (o_ndf) o_ndf[T] = o.ndf;
  if (o_rej)
    for (int k = 0; k < n; ++k) o_rej[a + k] = rej[ly.at(k)];
}

template <bool kField>
__global__ void __launch_bounds__(kB) k_refit_bwd(Geo g, RefitCfg p, const uint32_t* cnt,
                                                   const uint32_t* order, const uint32_t* wbase,
                                                   const uint32_t* wlen,
                                                   const uint32_t* track_start, TrackIn win,
                                                   const uint8_t* rej, const int32_t* status,
                                                   const float* ckpt, const float* dl_dchi2,
                                                   float* gyc, float* gzc, const uint8_t* multi,
                                                   const float* vz, float vvar, float* vck,
                                                   uint32_t* gmax) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (int)cnt[kCntTracks]) return;
  int T = (int)order[tid];
  if (status[T] == 3) return;
  int n = (int)(track_start[T + 1] - track_start[T]);
  Lay ly = warp_layout(wbase, wlen, tid);
  if (status[T] != 0) {
    for (int k = 0; k < n; ++k) {
      gyc[ly.at(k)] = 0.0f;
      gzc[ly.at(k)] = 0.0f;
    }
    return;
  }
  Vertex vx{vz ? vz[T] : NAN, vvar, vz ? vck + (size_t)T * kVtxCk : nullptr};
  refit_backward_track<kField>(g, p, win, ly, n, rej, ckpt, dl_dchi2[T], gyc, gzc,
                               multi[T] != 0, vx);
  // largest |gradient| (as float bits, so that NaN ranks above infinity)
  uint32_t m = 0u;
  for (int k = 0; k < n; ++k) {
    m = max(m, __float_as_uint(fabsf(gyc[ly.at(k)])));
    m = max(m, __float_as_uint(fabsf(gzc[ly.at(k)])));
  }
  if (m) atomicMax(gmax, m);
}

// Fixed-point exponent of the spline-gradient sums: every partial sum of
// coefficient contributions is bounded by n_assigned * max|gradient| (the
// B-spline weights of a point sum to one), which is kept below 2^61.
// Returns false when that maximum is not finite.
__device__ __forceinline__ bool grad_fixed_exponent(uint32_t gmax_bits, int n_asg, int& k) {
  float m = __uint_as_float(gmax_bits);
  if (!isfinite(m)) return false;
  k = 0;
  if (m > 0.0f) {
    int e = 0;
    frexp((double)m * (double)(n_asg > 0 ? n_asg : 1), &e);
    k = 61 - e;
  }
  return true;
}

// Chain rule through the calibration transform (Sec. 4): calibrated (y, z)
// -> raw (y, t or z), v_drift, t0 and the spline coefficients.
// v * 2^kx rounded to the nearest integer (ties away from zero), by integer
// arithmetic on the float's fields. |v| * 2^kx < 2^62 by the choice of kx.
__device__ __forceinline__ long long to_fixed(float v, int kx) {
  uint32_t b = __float_as_uint(v);
  int ex = (int)((b >> 23) & 0xffu);
  long long m = (long long)(b & 0x7fffffu);
  if (ex) m |= 0x800000ll;
  int sh = (ex ? ex : 1) - 150 + kx;
  long long q;
  if (sh >= 0) q = m << sh;
  else if (sh > -26) q = (m + (1ll << (-sh - 1))) >> (-sh);
  else q = 0;
  return (b >> 31) ? -q : q;
}

// One warp per contiguous range of assigned clusters (tracks are contiguous
// and row-ordered in it). Lanes first take one cluster each: its coordinate
// gradients through the calibration, its spline cell and B-spline weights.
// The warp then walks the clusters in order; lane l owns two of the 64
// coefficients of the current cell (and both components) and sums their
// contributions in registers while the cell stays the same, which along a
// track it does for many rows. On a change of cell the sums go into the
// warp's table of the current sector in shared memory (each lane adds to its
// own entries, no atomics); the table goes to the global 64-bit fixed-point
// totals when the sector changes and at the end (tracks are grouped by
// sector, so a warp flushes one or two tables). Every sum has a fixed order
// and integer additions commute, so the gradient is reproducible bit for
// bit. Four blocks per SM (64 registers, 48 KB of shared memory each).
constexpr int kCgThreads = 256;
__global__ void __launch_bounds__(kCgThreads, 4) k_calib_grad(
    Geo g, Cal c, ClIn cl, const uint32_t* cnt, const uint32_t* cluster_idx,
    const uint32_t* asg_track, const uint32_t* track_start, const uint32_t* slot,
    const uint32_t* wbase, const double* t_coll, const float* gyc, const float* gzc,
    const uint32_t* gmax, float* grad_y, float* grad_zt, unsigned long long* acc_spline,
    double* part_cal) {
  constexpr int kComp = kSpl * kSpl * kSpl;
  __shared__ double red[2][kCgThreads / 32];
  __shared__ float sw[kCgThreads / 32][32][15];  // per lane: weights, gradient, cell
  __shared__ float tabs[kCgThreads / 32][2 * kComp];  // per warp: one sector's sums
  int n = (int)cnt[kCntAssigned];
  int kx = 0;
  // a non-finite gradient leaves the spline sums to k_calib_reduce (NaN)
  const bool fixed_ok = grad_fixed_exponent(*gmax, n, kx);
  const bool spl_on = c.spl_bound[2] > 0.0f;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nwarps = gridDim.x * (kCgThreads / 32);
  const int gw = blockIdx.x * (kCgThreads / 32) + w;
  int per = (n + nwarps - 1) / nwarps;
  int jb = gw * per, je = min(n, jb + per);
  // (v_drift, t0) partial sums of this lane, in a fixed order; the lanes'
  // sums are added in float64
  float avd = 0.0f, at0 = 0.0f;
  // single precision after the drift time: double precision runs at a small
  // fraction of the single-precision rate, and the gradient needs no more
  const float vf = (float)c.vdrift;
  const float kS = (float)(kSpl - 3);
  // this lane's two coefficients of a cell: (w, v, u) offsets (cc, bb, aa)
  // with cc = lane / 16 and cc + 2
  const int aa = lane & 3, bb = (lane >> 2) & 3, cc1 = lane >> 4;
  const int off1 = (cc1 * kSpl + bb) * kSpl + aa;
  const int off2 = off1 + 2 * kSpl * kSpl;
  float a01 = 0.f, a02 = 0.f, a11 = 0.f, a12 = 0.f;  // [component][coefficient]
  int cur = -1;                                        // cell base of the sums
  float* tab = tabs[w];
  int tsec = -1;  // sector of the warp's table
  for (int e = lane; e < 2 * kComp; e += 32) tab[e] = 0.0f;
  __syncwarp();
  // the table into the global totals (all lanes, converged)
  auto flush_table = [&]() {
    __syncwarp();
    unsigned long long* acc = acc_spline + (size_t)tsec * 2 * kComp;
    for (int e = lane; e < 2 * kComp; e += 32) {
      const long long q = to_fixed(tab[e], kx);
      if (q != 0) atomicAdd(&acc[e], (unsigned long long)q);
      tab[e] = 0.0f;
    }
    __syncwarp();
  };
  // the cell's sums into the table (all lanes, converged: cur is the same on
  // every lane); a cell's coefficients lie in its sector's 2 * kComp: base
  // (iw * kSpl + iv) * kSpl + iu with iu, iv, iw <= kSpl - 4, plus offsets
  // below 3 * (kSpl^2 + kSpl + 1)
  auto flush = [&]() {
    const int sec = cur / (2 * kComp);
    if (sec != tsec) {
      if (tsec >= 0) flush_table();
      tsec = sec;
    }
    const int lc = cur - sec * 2 * kComp;
    tab[lc + off1] += a01;
    tab[lc + off2] += a02;
    tab[lc + kComp + off1] += a11;
    tab[lc + kComp + off2] += a12;
    a01 = a02 = a11 = a12 = 0.f;
  };
  for (int b0 = jb; b0 < je; b0 += 32) {
    int j = b0 + lane;
    bool valid = j < je;
    float by = 0.0f, bz = 0.0f;
    int o0 = 0;
    float bu[4] = {0.f, 0.f, 0.f, 0.f}, bv[4] = {0.f, 0.f, 0.f, 0.f};
    float bw[4] = {0.f, 0.f, 0.f, 0.f};
    if (valid) {
      uint32_t i = cluster_idx[j];
      uint32_t T = asg_track[j];
      double that = t_coll[T];
      uint32_t sl = slot[T];
      size_t wpos = ((size_t)wbase[sl >> 5] + (j - track_start[T])) * 32 + (sl & 31);
      int r = cl.row[i], s = cl.sector[i];
      float x = g.rx[r];
      float y = cluster_y(g, cl, i);
      // absolute z (Sec. 4): the drift time in float64 (t and the collision
      // time are large absolute times), the rest in float32
      const float sgf = s < 18 ? 1.0f : -1.0f;
      const float dtf = cl.mode == 1 ? (float)((cl.t[i] - c.t0) - that) : 0.0f;
      float za = cl.mode == 0 ? cl.z[i] : sgf * (g.L - vf * dtf);
      by = gyc[wpos];
      bz = gzc[wpos];
      float ur = (x - c.spl_x0) / c.spl_dx;
      float vr = (y / x + g.tan_half) / (2.0f * g.tan_half);
      float wr = fabsf(za) / g.L;
      float u = clamp01(ur), v = clamp01(vr), wv = clamp01(wr);
      int iu, iv, iw;
      float fu, fv, fw;
      spline_split(u, iu, fu);
      spline_split(v, iv, fv);
      spline_split(wv, iw, fw);
      spline_basis(fu, bu);
      spline_basis(fv, bv);
      spline_basis(fw, bw);
      o0 = s * 2 * kComp + (iw * kSpl + iv) * kSpl + iu;
      // gradient through the distortion itself: d(spline)/d(y, z) of both
      // components (zero when no coefficient is set: the forward then skips
      // the spline too), and the drift-time chain for v_drift and t0
      float dvdy = (vr > 0.0f && vr < 1.0f) ? 1.0f / (x * (2.0f * g.tan_half)) : 0.0f;
      float dwdz = (wr > 0.0f && wr < 1.0f) ? (za >= 0.0f ? 1.0f : -1.0f) / g.L : 0.0f;
      float dbv[4], dbw[4];
      auto dbasis = [](float f, float d[4]) {
        float gg = 1.0f - f;
        d[0] = -0.5f * gg * gg;
        d[1] = 0.5f * (3.0f * f * f - 4.0f * f);
        d[2] = 0.5f * (-3.0f * f * f + 2.0f * f + 1.0f);
        d[3] = 0.5f * f * f;
      };
      dbasis(fv, dbv);
      dbasis(fw, dbw);
      // tensor-product derivatives, summed innermost axis first (u, then v,
      // then w): 4 x 4 partial sums over u shared by both derivatives
      float dval_dv[2] = {0.f, 0.f}, dval_dw[2] = {0.f, 0.f};
      for (int cp = 0; cp < (spl_on ? 2 : 0); ++cp) {
        const float* cf = c.spline + (s * 2 + cp) * kComp;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          float tv = 0.f, tdv = 0.f;
#pragma unroll
          for (int b2 = 0; b2 < 4; ++b2) {
            const float* row = cf + ((iw + cc) * kSpl + (iv + b2)) * kSpl + iu;
            float su = bu[0] * row[0] + bu[1] * row[1] + bu[2] * row[2] + bu[3] * row[3];
            tv += bv[b2] * su;
            tdv += dbv[b2] * su;
          }
          dval_dv[cp] += bw[cc] * tdv;
          dval_dw[cp] += dbw[cc] * tv;
        }
      }
      float dDy_dy = dval_dv[0] * kS * dvdy, dDz_dy = dval_dv[1] * kS * dvdy;
      float dDy_dz = dval_dw[0] * kS * dwdz, dDz_dz = dval_dw[1] * kS * dwdz;
      float gy = by * (1.0f + dDy_dy) + bz * dDz_dy;
      float gza = by * dDy_dz + bz * (1.0f + dDz_dz);
      grad_y[j] = cl.pads ? gy * g.pw[r] : gy;  // per pad for native input
      if (cl.mode == 1) {
        grad_zt[j] = gza * (-sgf * vf);
        avd += gza * (-sgf * dtf);
        at0 += gza * (sgf * vf);
      } else {
        grad_zt[j] = gza;
      }
    }
    // spline coefficient gradients, one cluster at a time in cluster order:
    // each lane publishes its cluster's cell, gradient and B-spline weights
    // in shared memory, each lane then reads the four weights of its own
    // coefficients
    float* mine = sw[w][lane];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      mine[q] = bu[q];
      mine[4 + q] = bv[q];
      mine[8 + q] = bw[q];
    }
    mine[12] = by;
    mine[13] = bz;
    mine[14] = __int_as_float(o0);
    __syncwarp();
    unsigned am = __ballot_sync(0xffffffffu, valid && fixed_ok && (by != 0.0f || bz != 0.0f));
    while (am) {
      int src = __ffs(am) - 1;
      am &= am - 1;
      const float* sc = sw[w][src];
      int o = __float_as_int(sc[14]);
      if (o != cur) {  // uniform over the warp
        if (cur >= 0) flush();
        cur = o;
      }
      float cy = sc[12], cz = sc[13];
      float uv = sc[4 + bb] * sc[aa];
      float p1 = sc[8 + cc1] * uv;
      float p2 = sc[10 + cc1] * uv;
      a01 += cy * p1;
      a02 += cy * p2;
      a11 += cz * p1;
      a12 += cz * p2;
    }
    __syncwarp();
  }
  if (cur >= 0) flush();
  if (tsec >= 0) flush_table();
  // block reduction in float64, in a fixed order
  double dvd = (double)avd, dt0 = (double)at0;
  for (int o = 16; o > 0; o >>= 1) {
    dvd += __shfl_down_sync(0xffffffffu, dvd, o);
    dt0 += __shfl_down_sync(0xffffffffu, dt0, o);
  }
  if (lane == 0) {
    red[0][w] = dvd;
    red[1][w] = dt0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int q = 0; q < kCgThreads / 32; ++q) {
      s0 += red[0][q];
      s1 += red[1][q];
    }
    part_cal[blockIdx.x * 2 + 0] = s0;
    part_cal[blockIdx.x * 2 + 1] = s1;
  }
}

__global__ void k_calib_reduce(int nblk, const uint32_t* cnt, const uint32_t* gmax,
                               const unsigned long long* acc_spline, const double* part_cal,
                               double* grad_calib) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0 && threadIdx.x < 64) {
    // (v_drift, t0): warp w sums component w over the blocks, lane-strided,
    // then a fixed-order tree; both fixed, so the sum is reproducible
    int comp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double a = 0.0;
    for (int b = lane; b < nblk; b += 32) a += part_cal[b * 2 + comp];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) grad_calib[comp] = a;
  }
  if (i < 2 || i >= TPC_GRAD_CALIB_SIZE) return;
  double s = 0.0;
  {
    int kx = 0;
    if (grad_fixed_exponent(*gmax, (int)cnt[kCntAssigned], kx)) {
      s = ldexp((double)(long long)acc_spline[i - 2], -kx);
    } else {
      s = __longlong_as_double(0x7ff8000000000000ll);
    }
  }
  grad_calib[i] = s;
}

inline int nblk(int64_t n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

void launch_refit(Prof* P, const Geo& g, const Params& p, int64_t cap_tr, const uint32_t* cnt,
                  const TrackBuf& tb, RefitBuf& rb, bool save, float* params, float* cov,
                  float* x, float* chi2, int32_t* ndf, int32_t* status, uint8_t* rej,
                  uint32_t* err, cudaStream_t s) {
  if (cap_tr <= 0) return;
  TrackIn in{tb.track_start, tb.yc, tb.zc, tb.meta};
  TrackIn win{tb.track_start, rb.w_yc, rb.w_zc, rb.w_meta};
  int nb = nblk(cap_tr, 256);
  TPC_LAUNCH(P, "k_len_init", s, k_len_init<<<1, kLenBins, 0, s>>>(rb.len_hist));
  TPC_LAUNCH(P, "k_len_hist", s, k_len_hist<<<nb, 256, 0, s>>>(cnt, tb.track_start, rb.len_hist));
  TPC_LAUNCH(P, "k_len_scan", s, k_len_scan<<<1, kLenBins, 0, s>>>(rb.len_hist));
  TPC_LAUNCH(P, "k_len_scatter", s,
             k_len_scatter<<<nb, 256, 0, s>>>(cnt, tb.track_start, rb.len_hist, rb.order,
                                               rb.slot, rb.multi));
  TPC_LAUNCH(P, "k_warp_len", s,
             k_warp_len<<<nb, 256, 0, s>>>(cnt, tb.track_start, rb.order, rb.wlen));
  TPC_LAUNCH(P, "k_warp_scan", s, k_warp_scan<<<1, 1024, 0, s>>>(cnt, rb.wlen, rb.wbase));
  TPC_LAUNCH(P, "k_interleave", s,
             k_interleave<<<nblk(tb.cap_asg, 256), 256, 0, s>>>(cnt, in, tb.asg_track, rb.slot,
                                                                 rb.wbase, rb.w_yc, rb.w_zc,
                                                                 rb.w_meta, rb.multi));
  if (g.field_on)
    TPC_LAUNCH(P, "k_refit_field", s,
               k_refit<true><<<nblk(cap_tr, kB), kB, 0, s>>>(
                   g, make_cfg(g, p), cnt, rb.order, rb.wbase, rb.wlen, tb.track_start, win,
                   rb.seed, rb.rej, rb.status, rb.ckpt, save ? 1 : 0, params, cov, x, chi2, ndf,
                   status, rej, rb.multi, rb.vz, rb.vvar, rb.vck, err));
  else
    TPC_LAUNCH(P, "k_refit", s,
               k_refit<false><<<nblk(cap_tr, kB), kB, 0, s>>>(
                   g, make_cfg(g, p), cnt, rb.order, rb.wbase, rb.wlen, tb.track_start, win,
                   rb.seed, rb.rej, rb.status, rb.ckpt, save ? 1 : 0, params, cov, x, chi2, ndf,
                   status, rej, rb.multi, rb.vz, rb.vvar, rb.vck, err));
}

void launch_refit_backward(Prof* P, const Geo& g, const Cal& c, const Params& p, const ClIn& cl,
                           int64_t cap_tr, int64_t cap_asg, const uint32_t* cnt,
                           const TrackBuf& tb, RefitBuf& rb, const float* dl_dchi2,
                           float* grad_y, float* grad_zt, double* grad_calib, cudaStream_t s) {
  TrackIn win{tb.track_start, rb.w_yc, rb.w_zc, rb.w_meta};
  cudaMemsetAsync(rb.gmax, 0, sizeof(uint32_t), s);
  cudaMemsetAsync(rb.acc_spline, 0, sizeof(unsigned long long) * TPC_SPLINE_SIZE, s);
  if (cap_tr > 0)
    TPC_LAUNCH(P, g.field_on ? "k_refit_bwd_field" : "k_refit_bwd", s,
               (g.field_on ? k_refit_bwd<true> : k_refit_bwd<false>)<<<nblk(cap_tr, kB), kB, 0,
                                                                       s>>>(
                   g, make_cfg(g, p), cnt, rb.order, rb.wbase, rb.wlen, tb.track_start, win,
                   rb.rej, rb.status, rb.ckpt, dl_dchi2, rb.gyc, rb.gzc, rb.multi, rb.vz,
                   rb.vvar, rb.vck, rb.gmax));
  TPC_LAUNCH(P, "k_calib_grad", s,
             k_calib_grad<<<kCalibGradBlocks, kCgThreads, 0, s>>>(
                 g, c, cl, cnt, tb.cluster_idx, tb.asg_track, tb.track_start, rb.slot, rb.wbase,
                 tb.t_coll, rb.gyc, rb.gzc, rb.gmax, grad_y, grad_zt, rb.acc_spline,
                 rb.part_cal));
  TPC_LAUNCH(P, "k_calib_reduce", s,
             k_calib_reduce<<<nblk(TPC_GRAD_CALIB_SIZE, 256), 256, 0, s>>>(
                 kCalibGradBlocks, cnt, rb.gmax, rb.acc_spline, rb.part_cal, grad_calib));
}

}  // namespace tpc
