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
// k_calib_grad persistent blocks: chain rule through the calibration
//              transform (drift time to z, distortion spline); spline
//              gradients accumulate in shared memory per block.
// k_calib_reduce sums the per-block partials in float64.
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
  c.shared_scale = p.shared_scale;
  c.chi2_out = p.chi2_out;
  c.refit_inflate = p.refit_inflate;
  c.min_acc_reject = p.min_acc_reject;
  for (int i = 0; i < 5; ++i) c.c0r[i] = p.c0r[i];
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
  atomicAdd(&hist[len_bin(ts, T)], 1u);
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
                              uint32_t* order, uint32_t* slot) {
  int T = blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= (int)cnt[kCntTracks]) return;
  int b = len_bin(ts, T);
  uint32_t pos = hist[b] + atomicAdd(&hist[kLenBins + b], 1u);
  order[pos] = (uint32_t)T;
  slot[T] = pos;
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
__global__ void k_interleave(const uint32_t* cnt, TrackIn in, const uint32_t* order,
                             const uint32_t* wbase, const uint32_t* wlen, float* w_yc,
                             float* w_zc, uint32_t* w_meta) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (int)cnt[kCntTracks]) return;
  int T = (int)order[tid];
  uint32_t a = in.track_start[T];
  uint32_t b = in.track_start[T + 1];
  if (b < a || b > cnt[kCntAssigned]) return;
  Lay ly = warp_layout(wbase, wlen, tid);
  for (int k = 0; k < (int)(b - a); ++k) {
    w_yc[ly.at(k)] = in.yc[a + k];
    w_zc[ly.at(k)] = in.zc[a + k];
    w_meta[ly.at(k)] = in.meta[a + k];
  }
}

__global__ void __launch_bounds__(kB) k_refit(Geo g, RefitCfg p, const uint32_t* cnt,
                                               const uint32_t* order, const uint32_t* wbase,
                                               const uint32_t* wlen, const uint32_t* track_start,
                                               TrackIn win, float* seed_out, uint8_t* rej,
                                               int32_t* status, float* ckpt, int save,
                                               float* o_params, float* o_cov, float* o_x,
                                               float* o_chi2, int32_t* o_ndf, int32_t* o_status,
                                               uint8_t* o_rej, uint32_t* err) {
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
  RefitOut o = refit_track(g, p, win, ly, n, rej, seed_out + (size_t)T * 5, save ? ckpt : nullptr);
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

__global__ void __launch_bounds__(kB) k_refit_bwd(Geo g, RefitCfg p, const uint32_t* cnt,
                                                   const uint32_t* order, const uint32_t* wbase,
                                                   const uint32_t* wlen,
                                                   const uint32_t* track_start, TrackIn win,
                                                   const uint8_t* rej, const int32_t* status,
                                                   const float* ckpt, const float* dl_dchi2,
                                                   float* gyc, float* gzc) {
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
  refit_backward_track(g, p, win, ly, n, rej, ckpt, dl_dchi2[T], gyc, gzc);
}

// Chain rule through the calibration transform (Sec. 4): calibrated (y, z)
// -> raw (y, t or z), v_drift, t0 and the spline coefficients.
__global__ void __launch_bounds__(512) k_calib_grad(Geo g, Cal c, ClIn cl, const uint32_t* cnt,
                                                     const uint32_t* cluster_idx,
                                                     const uint32_t* asg_track,
                                                     const uint32_t* track_start,
                                                     const uint32_t* slot, const uint32_t* wbase,
                                                     const double* t_coll, const float* gyc,
                                                     const float* gzc, float* grad_y,
                                                     float* grad_zt, float* part_spline,
                                                     double* part_cal) {
  extern __shared__ float sacc[];
  __shared__ double red[2][16];
  const int NS = TPC_SPLINE_SIZE;
  // the spline's coefficient gradient is formed even when all coefficients
  // are zero (the forward then adds exactly zero)
  bool spl_on = true;
  for (int i = threadIdx.x; i < NS; i += blockDim.x) sacc[i] = 0.0f;
  __syncthreads();
  int n = (int)cnt[kCntAssigned];
  int per = (n + gridDim.x - 1) / gridDim.x;
  int j0 = blockIdx.x * per, j1 = min(n, j0 + per);
  int len = j1 - j0;
  int nthr = blockDim.x;
  double avd = 0.0, at0 = 0.0;
  // lane-strided order so that the lanes of a warp work on different tracks
  int lanes = 32, warps = nthr / 32;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int sub = (len + lanes - 1) / lanes;
  for (int k = w; k < sub; k += warps) {
    int jj = lane * sub + k;
    if (jj >= len) continue;
    int j = j0 + jj;
    uint32_t i = cluster_idx[j];
    uint32_t T = asg_track[j];
    double that = t_coll[T];
    uint32_t sl = slot[T];
    size_t wpos = ((size_t)wbase[sl >> 5] + (j - track_start[T])) * 32 + (sl & 31);
    int r = cl.row[i], s = cl.sector[i];
    float x = g.row_x[r];
    float y = cl.y[i];
    float za = abs_z(g, c, cl.mode, cl.mode == 0 ? cl.z[i] : 0.0f, cl.mode == 1 ? cl.t[i] : 0.0,
                     s, that);
    float by = gyc[wpos], bz = gzc[wpos];
    float gy = by, gza = bz;
    if (spl_on) {
      float ur = (x - c.spl_x0) / c.spl_dx;
      float vr = (y / x + g.tan_half) / (2.0f * g.tan_half);
      float wr = fabsf(za) / g.L;
      float u = clamp01(ur), v = clamp01(vr), w = clamp01(wr);
      float dvdy = (vr > 0.0f && vr < 1.0f) ? 1.0f / (x * (2.0f * g.tan_half)) : 0.0f;
      float dwdz = (wr > 0.0f && wr < 1.0f) ? (za >= 0.0f ? 1.0f : -1.0f) / g.L : 0.0f;
      int iu, iv, iw;
      float fu, fv, fw;
      spline_split(u, iu, fu);
      spline_split(v, iv, fv);
      spline_split(w, iw, fw);
      float bu[4], bv[4], bw[4], dbv[4], dbw[4];
      spline_basis(fu, bu);
      spline_basis(fv, bv);
      spline_basis(fw, bw);
      auto dbasis = [](float f, float d[4]) {
        float gg = 1.0f - f;
        d[0] = -0.5f * gg * gg;
        d[1] = 0.5f * (3.0f * f * f - 4.0f * f);
        d[2] = 0.5f * (-3.0f * f * f + 2.0f * f + 1.0f);
        d[3] = 0.5f * f * f;
      };
      dbasis(fv, dbv);
      dbasis(fw, dbw);
      const float kS = (float)(kSpl - 3);
      float dval_dv[2] = {0.f, 0.f}, dval_dw[2] = {0.f, 0.f};
      for (int comp = 0; comp < 2; ++comp) {
        float cb = comp == 0 ? by : bz;
        int base = ((s * 2 + comp) * kSpl) * kSpl * kSpl;
        const float* cf = c.spline + base;
        for (int cc = 0; cc < 4; ++cc)
          for (int bb = 0; bb < 4; ++bb) {
            int o = ((iw + cc) * kSpl + (iv + bb)) * kSpl + iu;
            for (int aa = 0; aa < 4; ++aa) {
              float coef = cf[o + aa];
              dval_dv[comp] += bw[cc] * dbv[bb] * bu[aa] * coef;
              dval_dw[comp] += dbw[cc] * bv[bb] * bu[aa] * coef;
              if (cb != 0.0f) atomicAdd(&sacc[base + o + aa], cb * (bw[cc] * bv[bb] * bu[aa]));
            }
          }
      }
      float dDy_dy = dval_dv[0] * kS * dvdy, dDz_dy = dval_dv[1] * kS * dvdy;
      float dDy_dz = dval_dw[0] * kS * dwdz, dDz_dz = dval_dw[1] * kS * dwdz;
      gy = by * (1.0f + dDy_dy) + bz * dDz_dy;
      gza = by * dDy_dz + bz * (1.0f + dDz_dz);
    }
    grad_y[j] = gy;
    if (cl.mode == 1) {
      double sg = s < 18 ? 1.0 : -1.0;
      grad_zt[j] = (float)((double)gza * (-sg * c.vdrift));
      avd += (double)gza * (-sg * ((cl.t[i] - c.t0) - that));
      at0 += (double)gza * (sg * c.vdrift);
    } else {
      grad_zt[j] = gza;
    }
  }
  // block reduction of the float64 sums
  for (int o = 16; o > 0; o >>= 1) {
    avd += __shfl_down_sync(0xffffffffu, avd, o);
    at0 += __shfl_down_sync(0xffffffffu, at0, o);
  }
  if (lane == 0) {
    red[0][w] = avd;
    red[1][w] = at0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int q = 0; q < warps; ++q) {
      s0 += red[0][q];
      s1 += red[1][q];
    }
    part_cal[blockIdx.x * 2 + 0] = s0;
    part_cal[blockIdx.x * 2 + 1] = s1;
  }
  float* ps = part_spline + (size_t)blockIdx.x * NS;
  for (int i = threadIdx.x; i < NS; i += blockDim.x) ps[i] = sacc[i];
}

__global__ void k_calib_reduce(int nblk, const float* part_spline, const double* part_cal,
                               double* grad_calib) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= TPC_GRAD_CALIB_SIZE) return;
  double s = 0.0;
  if (i < 2) {
    for (int b = 0; b < nblk; ++b) s += part_cal[b * 2 + i];
  } else {
    for (int b = 0; b < nblk; ++b) s += (double)part_spline[(size_t)b * TPC_SPLINE_SIZE + (i - 2)];
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
                                               rb.slot));
  TPC_LAUNCH(P, "k_warp_len", s,
             k_warp_len<<<nb, 256, 0, s>>>(cnt, tb.track_start, rb.order, rb.wlen));
  TPC_LAUNCH(P, "k_warp_scan", s, k_warp_scan<<<1, 1024, 0, s>>>(cnt, rb.wlen, rb.wbase));
  TPC_LAUNCH(P, "k_interleave", s,
             k_interleave<<<nb, 256, 0, s>>>(cnt, in, rb.order, rb.wbase, rb.wlen, rb.w_yc,
                                              rb.w_zc, rb.w_meta));
  TPC_LAUNCH(P, "k_refit", s,
             k_refit<<<nblk(cap_tr, kB), kB, 0, s>>>(g, make_cfg(g, p), cnt, rb.order, rb.wbase,
                                                     rb.wlen, tb.track_start, win, rb.seed,
                                                     rb.rej, rb.status, rb.ckpt, save ? 1 : 0,
                                                     params, cov, x, chi2, ndf, status, rej,
                                                     err));
}

void launch_refit_backward(Prof* P, const Geo& g, const Cal& c, const Params& p, const ClIn& cl,
                           int64_t cap_tr, int64_t cap_asg, const uint32_t* cnt,
                           const TrackBuf& tb, RefitBuf& rb, const float* dl_dchi2,
                           float* grad_y, float* grad_zt, double* grad_calib, cudaStream_t s) {
  TrackIn win{tb.track_start, rb.w_yc, rb.w_zc, rb.w_meta};
  if (cap_tr > 0)
    TPC_LAUNCH(P, "k_refit_bwd", s,
               k_refit_bwd<<<nblk(cap_tr, kB), kB, 0, s>>>(g, make_cfg(g, p), cnt, rb.order,
                                                           rb.wbase, rb.wlen, tb.track_start,
                                                           win, rb.rej, rb.status, rb.ckpt,
                                                           dl_dchi2, rb.gyc, rb.gzc));
  size_t smem = TPC_SPLINE_SIZE * sizeof(float);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_calib_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  TPC_LAUNCH(P, "k_calib_grad", s,
             k_calib_grad<<<kCalibGradBlocks, 512, smem, s>>>(
                 g, c, cl, cnt, tb.cluster_idx, tb.asg_track, tb.track_start, rb.slot, rb.wbase,
                 tb.t_coll, rb.gyc, rb.gzc, grad_y, grad_zt, rb.part_spline, rb.part_cal));
  TPC_LAUNCH(P, "k_calib_reduce", s,
             k_calib_reduce<<<nblk(TPC_GRAD_CALIB_SIZE, 256), 256, 0, s>>>(
                 kCalibGradBlocks, rb.part_spline, rb.part_cal, grad_calib));
}

}  // namespace tpc
