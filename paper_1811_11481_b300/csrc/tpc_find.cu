// Track finding on the GPU (arXiv:1811.11481 Sec. 2 and Sec. 4).
//
// Compiled with -fmad=false: every decision (windows, argmins, pick-up cuts)
// is taken on single-precision values rounded once per written operation.
//
// Data flow of one batch (all on the context's stream, no host round trip):
//   k_hist      cluster -> (event, sector, row) bucket counts, seed z (Sec. 4
//               time scaling), per (event, side) z range
//   k_scan_rows bucket offsets, grid z geometry
//   k_scatter   input index into its bucket
//   k_row_sort  one block per pad-row bucket: sort by (bin, input index) in
//               shared memory, write the grid-ordered SoA and bin offsets
//   k_neighbours one thread per hit: best (up, down) pair (Sec. 2 CA)
//   k_clean     mutual links only (Sec. 2 "evolution"), start-hit counts
//   k_write_starts ordered start-hit list
//   k_tracklets one thread per start hit: chain fit, closest approach ->
//               collision time, calibrated refit of the seed, outward and
//               inward following with pick-up (Sec. 2, 3, 4)
//   k_select_*  shared-cluster resolution and ordered track emission
//   k_calib     calibrated coordinates of the assigned clusters (Sec. 4)
#include <cstdio>

#include "tpc_impl.h"

namespace tpc {
namespace {

constexpr int kB256 = 256;

__device__ __forceinline__ int32_t f2ord(float f) {
  int32_t i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int32_t i) {
  return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff);
}

// Block-wide exclusive scan of one uint32 per thread (blockDim.x <= 1024).
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sum[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[w] = x;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  if (w == 0) {
    uint32_t s = lane < nw ? warp_sum[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) warp_sum[lane] = s;
  }
  __syncthreads();
  uint32_t base = w > 0 ? warp_sum[w - 1] : 0u;
  if (total) *total = warp_sum[nw - 1];
  uint32_t r = base + x - v;
  __syncthreads();
  return r;
}

// ------------------------------------------------------------- a1, a2, a3
__global__ void k_init_load(int K, int n_events, uint32_t* cnt, uint32_t* fill, int32_t* zmm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < K) {
    cnt[i] = 0u;
    fill[i] = 0u;
  }
  if (i < n_events * 2) {
    zmm[2 * i] = f2ord(3.0e38f);
    zmm[2 * i + 1] = f2ord(-3.0e38f);
  }
}

__global__ void k_hist(Geo g, Cal c, ClIn cl, uint32_t* cnt, float* zs_in, int32_t* zmm,
                       uint32_t* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cl.n) return;
  int r = cl.row[i], s = cl.sector[i];
  int e = cl.event ? (int)cl.event[i] : 0;
  if (r >= g.n_rows || s >= kNS || e >= cl.n_events) {
    atomicOr(err, kErrArg);
    zs_in[i] = 0.0f;
    return;
  }
  float zs = seed_z(g, c, cl.mode, cl.mode == 0 ? cl.z[i] : 0.0f, cl.mode == 1 ? cl.t[i] : 0.0, s);
  zs_in[i] = zs;
  if (!(fabsf(zs) < 1.0e30f)) {
    atomicOr(err, kErrArg);
    return;
  }
  int key = (e * kNS + s) * g.n_rows + r;
  atomicAdd(&cnt[key], 1u);
  int side = e * 2 + (s >= 18 ? 1 : 0);
  int32_t o = f2ord(zs);
  if (o < zmm[2 * side]) atomicMin(&zmm[2 * side], o);
  if (o > zmm[2 * side + 1]) atomicMax(&zmm[2 * side + 1], o);
}

// Single block: bucket offsets and z-bin geometry per (event, side).
__global__ void k_scan_rows(int K, int n_events, GridDims gd, const uint32_t* cnt,
                            uint32_t* row_start, const int32_t* zmm, float* zr) {
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  for (int base = 0; base < K; base += blockDim.x) {
    int i = base + threadIdx.x;
    uint32_t v = i < K ? cnt[i] : 0u;
    uint32_t tot;
    uint32_t ex = block_excl_scan(v, &tot);
    if (i < K) row_start[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) row_start[K] = carry;
  for (int i = threadIdx.x; i < n_events * 2; i += blockDim.x) {
    float lo = ord2f(zmm[2 * i]), hi = ord2f(zmm[2 * i + 1]);
    if (!(hi >= lo)) {
      zr[2 * i] = 0.0f;
      zr[2 * i + 1] = 0.0f;
    } else {
      float z0 = lo - gd.z_margin;
      float span = (hi + gd.z_margin) - z0;
      zr[2 * i] = z0;
      zr[2 * i + 1] = (float)gd.nz / span;
    }
  }
}

__global__ void k_scatter(Geo g, ClIn cl, const uint32_t* row_start, uint32_t* fill,
                          uint32_t* perm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cl.n) return;
  int r = cl.row[i], s = cl.sector[i];
  int e = cl.event ? (int)cl.event[i] : 0;
  if (r >= g.n_rows || s >= kNS || e >= cl.n_events) return;
  int key = (e * kNS + s) * g.n_rows + r;
  uint32_t pos = row_start[key] + atomicAdd(&fill[key], 1u);
  perm[pos] = (uint32_t)i;
}

__device__ __forceinline__ int bin_y(const Geo& g, const GridDims& gd, int r, float y) {
  float hw = g.row_x[r] * g.tan_half + gd.y_margin;
  float v = (y + hw) * ((float)gd.ny / (2.0f * hw));
  int iy = (int)floorf(v);
  return iy < 0 ? 0 : (iy >= gd.ny ? gd.ny - 1 : iy);
}
__device__ __forceinline__ int bin_z(const GridDims& gd, const float* zr, int side, float z) {
  float v = (z - zr[2 * side]) * zr[2 * side + 1];
  int iz = (int)floorf(v);
  if (!(v == v)) iz = 0;
  return iz < 0 ? 0 : (iz >= gd.nz ? gd.nz - 1 : iz);
}

// One block per (event, sector, row) bucket: bitonic sort of (bin, input index)
// keys in shared memory, then the grid-ordered SoA and the bin offsets.
__global__ void k_row_sort(Geo g, ClIn cl, GridDims gd, const uint32_t* row_start,
                           const uint32_t* perm, const float* zs_in, const float* zr, float2* gyz,
                           double* gt, uint32_t* gorig, uint32_t* gseg,
                           uint32_t* bin_start, uint32_t* err) {
  extern __shared__ unsigned long long keys[];
  int seg = blockIdx.x;
  uint32_t start = row_start[seg];
  int n = (int)(row_start[seg + 1] - start);
  uint32_t* bs = bin_start + (size_t)seg * (gd.nb + 1);
  if (n == 0) {
    for (int b = threadIdx.x; b <= gd.nb; b += blockDim.x) bs[b] = start;
    return;
  }
  if (n > kSortTile) {
    if (threadIdx.x == 0) atomicOr(err, kErrCapRow);
    for (int b = threadIdx.x; b <= gd.nb; b += blockDim.x) bs[b] = start;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      uint32_t i = perm[start + j];
      gyz[start + j] = make_float2(cl.y[i], zs_in[i]);
      if (cl.mode == 1) gt[start + j] = cl.t[i];
      gorig[start + j] = i;
      gseg[start + j] = (uint32_t)seg;
    }
    return;
  }
  int r = seg % g.n_rows;
  int es = seg / g.n_rows;
  int e = es / kNS, s = es % kNS;
  int side = e * 2 + (s >= 18 ? 1 : 0);
  int P = 1;
  while (P < n) P <<= 1;
  for (int j = threadIdx.x; j < P; j += blockDim.x) {
    unsigned long long k = ~0ull;
    if (j < n) {
      uint32_t i = perm[start + j];
      int b = bin_z(gd, zr, side, zs_in[i]) * gd.ny + bin_y(g, gd, r, cl.y[i]);
      k = ((unsigned long long)(uint32_t)b << 32) | i;
    }
    keys[j] = k;
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          unsigned long long a = keys[i], b = keys[ixj];
          bool up = (i & k) == 0;
          if ((a > b) == up) {
            keys[i] = b;
            keys[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    unsigned long long k = keys[j];
    uint32_t i = (uint32_t)(k & 0xffffffffu);
    int b = (int)(k >> 32);
    int bprev = j > 0 ? (int)(keys[j - 1] >> 32) : -1;
    for (int q = bprev + 1; q <= b; ++q) bs[q] = start + j;
    if (j == n - 1)
      for (int q = b + 1; q <= gd.nb; ++q) bs[q] = start + n;
    gyz[start + j] = make_float2(cl.y[i], zs_in[i]);
    if (cl.mode == 1) gt[start + j] = cl.t[i];
    gorig[start + j] = i;
    gseg[start + j] = (uint32_t)seg;
  }
}

// Range of grid bins [iy0, iy1] x [iz0, iz1] covering a (y, z) box of row seg.
struct Box {
  int iy0, iy1, iz0, iz1;
};
__device__ __forceinline__ Box make_box(const Geo& g, const GridDims& gd, const float* zr,
                                        int r, int side, float ylo, float yhi, float zlo,
                                        float zhi) {
  Box b;
  b.iy0 = bin_y(g, gd, r, ylo);
  b.iy1 = bin_y(g, gd, r, yhi);
  b.iz0 = bin_z(gd, zr, side, zlo);
  b.iz1 = bin_z(gd, zr, side, zhi);
  return b;
}

// ------------------------------------------------------- a4: neighbour finder
// For hit h in row r: the pair (u in row r+1, d in row r-1) inside the slope
// windows whose d lies closest to the straight line through h and u; ties go
// to the lowest pair of input indices.
__global__ void k_neighbours(Geo g, Params p, GridDims gd, const uint32_t* nvalid,
                             const float2* __restrict__ gyz, const uint32_t* __restrict__ gorig,
                             const uint32_t* gseg, const uint32_t* bin_start, const float* zr,
                             int32_t* up, int32_t* dn) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= (int)*nvalid) return;
  int seg = (int)gseg[h];
  int r = seg % g.n_rows;
  int32_t bu = -1, bd = -1;
  if (r >= 1 && r + 1 < g.n_rows) {
    int es = seg / g.n_rows;
    int e = es / kNS, s = es % kNS;
    int side = e * 2 + (s >= 18 ? 1 : 0);
    float xh = g.row_x[r], xu = g.row_x[r + 1], xd = g.row_x[r - 1];
    float2 hh = gyz[h];
    float yh = hh.x, zh = hh.y;
    float dxu = xu - xh, dxd = xh - xd;
    float wy_u = dxu * p.nb_ty + p.nb_wy;
    float wy_d = dxd * p.nb_ty + p.nb_wy;
    float wz_u = dxu * p.nb_teta + p.nb_wz;
    float wz_d = dxd * p.nb_teta + p.nb_wz;
    float f = dxd / dxu;
    const float eps = 1.0e-3f;
    Box BU = make_box(g, gd, zr, r + 1, side, yh - wy_u - eps, yh + wy_u + eps, zh - wz_u - eps,
                      zh + wz_u + eps);
    Box BD = make_box(g, gd, zr, r - 1, side, yh - wy_d - eps, yh + wy_d + eps, zh - wz_d - eps,
                      zh + wz_d + eps);
    const uint32_t* bsu = bin_start + (size_t)(seg + 1) * (gd.nb + 1);
    const uint32_t* bsd = bin_start + (size_t)(seg - 1) * (gd.nb + 1);
    bool found = false;
    float best = 0.0f;
    uint32_t bou = 0, bod = 0;
    for (int iz = BU.iz0; iz <= BU.iz1; ++iz) {
      uint32_t u0 = bsu[iz * gd.ny + BU.iy0], u1 = bsu[iz * gd.ny + BU.iy1 + 1];
      for (uint32_t u = u0; u < u1; ++u) {
        float2 uu = gyz[u];
        float yu = uu.x, zu = uu.y;
        if (!(fabsf(yu - yh) <= wy_u)) continue;
        if (!(fabsf(zu - zh) <= wz_u)) continue;
        float py = yh - (yu - yh) * f;
        float pz = zh - (zu - zh) * f;
        uint32_t ou = gorig[u];
        for (int jz = BD.iz0; jz <= BD.iz1; ++jz) {
          uint32_t d0 = bsd[jz * gd.ny + BD.iy0], d1 = bsd[jz * gd.ny + BD.iy1 + 1];
          for (uint32_t d = d0; d < d1; ++d) {
            float2 dd = gyz[d];
            float yd = dd.x, zd = dd.y;
            if (!(fabsf(yd - yh) <= wy_d)) continue;
            if (!(fabsf(zd - zh) <= wz_d)) continue;
            float ey = yd - py, ez = zd - pz;
            float D = ey * ey + ez * ez;
            if (!(D <= p.nb_dmax)) continue;
            uint32_t od = gorig[d];
            if (!found || D < best || (D == best && (ou < bou || (ou == bou && od < bod)))) {
              found = true;
              best = D;
              bou = ou;
              bod = od;
              bu = (int32_t)u;
              bd = (int32_t)d;
            }
          }
        }
      }
    }
  }
  up[h] = bu;
  dn[h] = bd;
}

// --------------------------------------------------- a5, a6: cleaning, starts
__device__ __forceinline__ bool is_start(const int32_t* upc, const int32_t* dnc, int h) {
  int u = upc[h];
  return dnc[h] < 0 && u >= 0 && upc[u] >= 0;
}

__global__ void k_clean(const uint32_t* nvalid, const int32_t* up, const int32_t* dn,
                        int32_t* upc, int32_t* dnc, uint32_t* blk_cnt) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  int n = (int)*nvalid;
  uint32_t st = 0;
  if (h < n) {
    int u = up[h], d = dn[h];
    int uc = (u >= 0 && dn[u] == h) ? u : -1;
    int dc = (d >= 0 && up[d] == h) ? d : -1;
    upc[h] = uc;
    dnc[h] = dc;
    if (dc < 0 && uc >= 0) {
      int uu = up[uc];
      st = (uu >= 0 && dn[uu] == uc) ? 1u : 0u;
    }
  }
  uint32_t c = __syncthreads_count(st);
  if (threadIdx.x == 0) blk_cnt[blockIdx.x] = c;
}

// Single block: exclusive scan of per-block counts (two arrays), totals to
// cnt[slot_a], cnt[slot_b]; totals above cap raise err_bit and are clamped.
__global__ void k_scan_blocks(int nblk, const uint32_t* a, uint32_t* off_a, const uint32_t* b,
                              uint32_t* off_b, uint32_t* cnt, int slot_a, int slot_b,
                              uint32_t cap_a, uint32_t cap_b, uint32_t* err, uint32_t err_bit) {
  __shared__ uint32_t carry_a, carry_b;
  if (threadIdx.x == 0) {
    carry_a = 0u;
    carry_b = 0u;
  }
  __syncthreads();
  for (int base = 0; base < nblk; base += blockDim.x) {
    int i = base + threadIdx.x;
    uint32_t va = i < nblk ? a[i] : 0u;
    uint32_t ta;
    uint32_t ea = block_excl_scan(va, &ta);
    uint32_t vb = 0u, tb = 0u, eb = 0u;
    if (b) {
      vb = i < nblk ? b[i] : 0u;
      eb = block_excl_scan(vb, &tb);
    }
    if (i < nblk) {
      off_a[i] = carry_a + ea;
      if (b) off_b[i] = carry_b + eb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry_a += ta;
      carry_b += tb;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    off_a[nblk] = carry_a;
    uint32_t ca = carry_a, cb = carry_b;
    if (ca > cap_a) {
      atomicOr(err, err_bit);
      ca = cap_a;
    }
    if (b && cb > cap_b) {
      atomicOr(err, err_bit);
      cb = cap_b;
    }
    cnt[slot_a] = ca;
    if (b) {
      off_b[nblk] = carry_b;
      cnt[slot_b] = cb;
    }
  }
}

__global__ void k_write_starts(const uint32_t* nvalid, const int32_t* upc, const int32_t* dnc,
                               const uint32_t* blk_off, uint32_t cap, uint32_t* starts) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  int n = (int)*nvalid;
  uint32_t st = (h < n && is_start(upc, dnc, h)) ? 1u : 0u;
  uint32_t ex = block_excl_scan(st, nullptr);
  if (st) {
    uint32_t pos = blk_off[blockIdx.x] + ex;
    if (pos < cap) starts[pos] = (uint32_t)h;
  }
}

// ------------------------------------------------------ a7: tracklets
struct Grid {
  const float2* gyz;
  const double* gt;
  const uint32_t* gorig;
  const uint32_t* bin_start;
  const float* zr;
};

// Nearest cluster of row r (calibrated frame) by the normalised distance,
// inside the pick-up cut; ties to the lowest input index. Returns grid
// position or -1, and the calibrated coordinates of the pick.
__device__ int pick(const Geo& g, const Cal& c, const Params& p, const GridDims& gd,
                    const Grid& G, int mode, int ev, int sec, int r, const float st[5],
                    const float C[15], double that, float shift, bool spl_on, float dymax,
                    float dzmax, float& ycb, float& zcb) {
  int seg = (ev * kNS + sec) * g.n_rows + r;
  int side = ev * 2 + (sec >= 18 ? 1 : 0);
  float sig2 = p.sigma * p.sigma;
  float vy = C[0] + sig2, vz = C[2] + sig2;
  float wy = sqrtf(p.chi2_pick * vy), wz = sqrtf(p.chi2_pick * vz);
  float eps = 0.01f + 1.0e-6f * fabsf(shift);
  float yp = st[0], zp = st[1] - shift;
  Box B = make_box(g, gd, G.zr, r, side, yp - wy - dymax - eps, yp + wy + dymax + eps,
                   zp - wz - dzmax - eps, zp + wz + dzmax + eps);
  const uint32_t* __restrict__ bs = G.bin_start + (size_t)seg * (gd.nb + 1);
  int best = -1;
  float bd = 0.0f;
  for (int izb = B.iz0; izb <= B.iz1; izb += 4) {
    // bin offsets of up to four z rows of the box, loaded together
    uint32_t lo[4], hi[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int iz = izb + q;
      bool in = iz <= B.iz1;
      lo[q] = in ? __ldg(bs + iz * gd.ny + B.iy0) : 0u;
      hi[q] = in ? __ldg(bs + iz * gd.ny + B.iy1 + 1) : 0u;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      for (uint32_t j = lo[q]; j < hi[q]; ++j) {
        float2 yz = __ldg(G.gyz + j);
        double tj = mode == 1 ? __ldg(G.gt + j) : 0.0;
        float yc, zc;
        calibrate(g, c, spl_on, mode, sec, r, yz.x, yz.y, tj, that, yc, zc);
        float ry = yc - st[0];
        float rz = zc - st[1];
        float d2 = (ry * ry) / vy + (rz * rz) / vz;
        if (!(d2 <= p.chi2_pick)) continue;
        bool take = best < 0 || d2 < bd;
        if (!take && d2 == bd) take = __ldg(G.gorig + j) < __ldg(G.gorig + best);
        if (take) {
          best = (int)j;
          bd = d2;
          ycb = yc;
          zcb = zc;
        }
      }
    }
  }
  return best;
}

__global__ void __launch_bounds__(128) k_tracklets(Geo g, Cal c, Params p, GridDims gd, Grid G,
                                                  int mode, const int32_t* upc,
                                                  const uint32_t* gseg, const uint32_t* starts,
                                                  const uint32_t* cnt, int32_t* nh_out,
                                                  int32_t* hits, double* that_out,
                                                  unsigned long long* weight) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int)cnt[kCntStart]) return;
  int32_t* H = hits + (size_t)t * g.n_rows;
  for (int r = 0; r < g.n_rows; ++r) H[r] = -1;
  nh_out[t] = -1;
  that_out[t] = 0.0;
  int h0 = (int)starts[t];
  int seg0 = (int)gseg[h0];
  int r0 = seg0 % g.n_rows;
  int es = seg0 / g.n_rows;
  int ev = es / kNS, sec = es % kNS;
  const float sig2 = p.sigma * p.sigma;
  bool spl_on = c.spl_bound[2] > 0.0f;
  float dymax = spl_on ? c.spl_bound[0] : 0.0f;
  float dzmax = spl_on ? c.spl_bound[1] : 0.0f;
  // the seed: the first segment of at most seed_max_hits linked hits
  int hl = h0, rl = r0, nseed = 1;
  while (upc[hl] >= 0 && nseed < p.seed_max_hits) {
    hl = upc[hl];
    ++rl;
    ++nseed;
  }
  float st[5], C[15], x;
  // seed fit in seeding coordinates
  float2 yz0 = G.gyz[h0], yzl = G.gyz[hl];
  seed_two_points(st, C, x, p.c0t, g.row_x[r0], yz0.x, yz0.y, g.row_x[rl], yzl.x, yzl.y);
  {
    int h = h0, r = r0;
    while (true) {
      if (!propagate(g.kB, p.s_max, st, C, x, g.row_x[r])) return;
      float2 yz = G.gyz[h];
      apply_update(st, C, innovation(st, C, yz.x, yz.y, sig2, sig2));
      if (h == hl) break;
      h = upc[h];
      ++r;
    }
  }
  double that = 0.0;
  float shift = 0.0f;
  if (mode == 1) {
    float zd = dca_z(g.kB, st, x);
    double sg = sec < 18 ? 1.0 : -1.0;
    that = c.tf_start - (sg * (double)zd) / c.vdrift;
    shift = (float)(sg * c.vdrift * (that - c.tf_start));
  }
  // seed fit in calibrated coordinates
  {
    float y0, z0, y1, z1;
    calibrate(g, c, spl_on, mode, sec, r0, yz0.x, yz0.y, mode == 1 ? G.gt[h0] : 0.0, that, y0,
              z0);
    calibrate(g, c, spl_on, mode, sec, rl, yzl.x, yzl.y, mode == 1 ? G.gt[hl] : 0.0, that, y1,
              z1);
    seed_two_points(st, C, x, p.c0t, g.row_x[r0], y0, z0, g.row_x[rl], y1, z1);
    int h = h0, r = r0;
    while (true) {
      if (!propagate(g.kB, p.s_max, st, C, x, g.row_x[r])) return;
      float yc, zc;
      float2 yz = G.gyz[h];
      calibrate(g, c, spl_on, mode, sec, r, yz.x, yz.y, mode == 1 ? G.gt[h] : 0.0, that, yc, zc);
      apply_update(st, C, innovation(st, C, yc, zc, sig2, sig2));
      if (h == hl) break;
      h = upc[h];
      ++r;
    }
  }
  // outward following
  float bst[5], bC[15], bx = x;
#pragma unroll
  for (int i = 0; i < 5; ++i) bst[i] = st[i];
#pragma unroll
  for (int i = 0; i < 15; ++i) bC[i] = C[i];
  int rlast = rl;
  int miss = 0;
  for (int r = rl + 1; r < g.n_rows; ++r) {
    if (!propagate(g.kB, p.s_max, st, C, x, g.row_x[r])) break;
    float yc, zc;
    int j = pick(g, c, p, gd, G, mode, ev, sec, r, st, C, that, shift, spl_on, dymax, dzmax, yc,
                 zc);
    if (j >= 0) {
      apply_update(st, C, innovation(st, C, yc, zc, sig2, sig2));
#pragma unroll
      for (int i = 0; i < 5; ++i) bst[i] = st[i];
#pragma unroll
      for (int i = 0; i < 15; ++i) bC[i] = C[i];
      bx = x;
      rlast = r;
      miss = 0;
    } else if (++miss >= p.max_miss) {
      break;
    }
  }
  // inward following through the seed
#pragma unroll
  for (int i = 0; i < 5; ++i) st[i] = bst[i];
#pragma unroll
  for (int i = 0; i < 15; ++i) C[i] = bC[i] * p.inward_cov_scale;
  x = bx;
  int nh = 0;
  miss = 0;
  for (int r = rlast; r >= 0; --r) {
    if (!propagate(g.kB, p.s_max, st, C, x, g.row_x[r])) break;
    float yc, zc;
    int j = pick(g, c, p, gd, G, mode, ev, sec, r, st, C, that, shift, spl_on, dymax, dzmax, yc,
                 zc);
    if (j >= 0) {
      apply_update(st, C, innovation(st, C, yc, zc, sig2, sig2));
      H[r] = j;
      ++nh;
      miss = 0;
    } else if (++miss >= p.max_miss) {
      break;
    }
  }
  nh_out[t] = nh;
  that_out[t] = that;
  if (nh >= p.min_track_hits) {
    unsigned long long w = ((unsigned long long)(uint32_t)nh << 32) |
                           (unsigned long long)(0xffffffffu - G.gorig[h0]);
    for (int r = 0; r < g.n_rows; ++r)
      if (H[r] >= 0) atomicMax(&weight[H[r]], w);
  }
}

// --------------------------------------------------- a8: tracklet selection
__global__ void k_select_count(int n_rows, const Params p, const uint32_t* cnt,
                               const int32_t* nh, const int32_t* hits, const uint32_t* starts,
                               const uint32_t* gorig, const unsigned long long* weight,
                               uint32_t* nkeep, uint32_t* blk_tr, uint32_t* blk_cl) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t emit = 0, kept = 0;
  if (t < (int)cnt[kCntStart] && nh[t] >= p.min_track_hits) {
    unsigned long long w = ((unsigned long long)(uint32_t)nh[t] << 32) |
                           (unsigned long long)(0xffffffffu - gorig[starts[t]]);
    const int32_t* H = hits + (size_t)t * n_rows;
    int lastr = -1, maxgap = 0, k = 0;
    for (int r = 0; r < n_rows; ++r) {
      int j = H[r];
      if (j < 0 || weight[j] != w) continue;
      if (lastr >= 0) maxgap = max(maxgap, r - lastr - 1);
      lastr = r;
      ++k;
    }
    if (k >= p.min_track_hits && maxgap <= p.max_gap) {
      emit = 1;
      kept = (uint32_t)k;
    }
  }
  if (t < (int)cnt[kCntStart]) nkeep[t] = kept;
  uint32_t tot_tr, tot_cl;
  block_excl_scan(emit, &tot_tr);
  block_excl_scan(kept, &tot_cl);
  if (threadIdx.x == 0) {
    blk_tr[blockIdx.x] = tot_tr;
    blk_cl[blockIdx.x] = tot_cl;
  }
}

__global__ void k_select_write(int n_rows, const uint32_t* cnt, const int32_t* hits,
                               const uint32_t* starts, const double* that,
                               const uint32_t* gorig, const unsigned long long* weight,
                               const int32_t* nh, const uint32_t* nkeep, const uint32_t* off_tr,
                               const uint32_t* off_cl, int64_t cap_tr, int64_t cap_asg,
                               uint32_t* track_start, uint32_t* cluster_idx, uint32_t* asg_track,
                               double* t_coll, uint32_t* start_hit) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t kept = (t < (int)cnt[kCntStart]) ? nkeep[t] : 0u;
  uint32_t emit = kept > 0 ? 1u : 0u;
  uint32_t ex_tr = block_excl_scan(emit, nullptr);
  uint32_t ex_cl = block_excl_scan(kept, nullptr);
  if (!emit) return;
  uint32_t id = off_tr[blockIdx.x] + ex_tr;
  uint32_t o = off_cl[blockIdx.x] + ex_cl;
  if ((int64_t)id >= cap_tr || (int64_t)(o + kept) > cap_asg) return;
  unsigned long long w = ((unsigned long long)(uint32_t)nh[t] << 32) |
                         (unsigned long long)(0xffffffffu - gorig[starts[t]]);
  track_start[id] = o;
  t_coll[id] = that[t];
  start_hit[id] = gorig[starts[t]];
  const int32_t* H = hits + (size_t)t * n_rows;
  for (int r = 0; r < n_rows; ++r) {
    int j = H[r];
    if (j < 0 || weight[j] != w) continue;
    cluster_idx[o] = gorig[j];
    asg_track[o] = id;
    ++o;
  }
}

__global__ void k_track_end(const uint32_t* cnt, uint32_t* track_start) {
  track_start[cnt[kCntTracks]] = cnt[kCntAssigned];
}

// ---------------------------------------------------- a9: calibration
__global__ void k_calib(Geo g, Cal c, ClIn cl, const uint32_t* cnt, const uint32_t* cluster_idx,
                        const uint32_t* asg_track, const double* t_coll, float* yc, float* zc,
                        uint32_t* meta, uint32_t* err) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= (int)cnt[kCntAssigned]) return;
  uint32_t i = cluster_idx[j];
  if (i >= (uint32_t)cl.n || cl.row[i] >= g.n_rows || cl.sector[i] >= kNS) {
    atomicOr(err, kErrArg);
    yc[j] = 0.0f;
    zc[j] = 0.0f;
    meta[j] = 0u;
    return;
  }
  double that = t_coll[asg_track[j]];
  int r = cl.row[i], s = cl.sector[i];
  bool spl_on = c.spl_bound[2] > 0.0f;
  float a, b;
  calibrate(g, c, spl_on, cl.mode, s, r, cl.y[i], cl.mode == 0 ? cl.z[i] : 0.0f,
            cl.mode == 1 ? cl.t[i] : 0.0, that, a, b);
  yc[j] = a;
  zc[j] = b;
  uint32_t fl = cl.flags ? cl.flags[i] : 0u;
  meta[j] = (uint32_t)r | (fl << 8) | ((uint32_t)s << 16);
}

// Track id of every assigned cluster of caller-given tracks; an invalid CSR
// (decreasing offsets, offsets beyond n_assigned) raises the argument error.
__global__ void k_asg_track(const uint32_t* cnt, const uint32_t* track_start,
                            uint32_t* asg_track, uint32_t* err) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int)cnt[kCntTracks]) return;
  uint32_t a = track_start[t], b = track_start[t + 1];
  if (b < a || b > cnt[kCntAssigned] || (t == 0 && a != 0)) {
    atomicOr(err, kErrArg);
    return;
  }
  for (uint32_t j = a; j < b; ++j) asg_track[j] = (uint32_t)t;
}

__global__ void k_spline_bound(const float* spline, float* bound) {
  __shared__ float m0[256], m1[256];
  float a = 0.0f, b = 0.0f;
  constexpr int kPer = kSpl * kSpl * kSpl;
  for (int i = threadIdx.x; i < kNS * 2 * kPer; i += blockDim.x) {
    float v = fabsf(spline[i]);
    if ((i / kPer) % 2 == 0) a = fmaxf(a, v);
    else b = fmaxf(b, v);
  }
  m0[threadIdx.x] = a;
  m1[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      m0[threadIdx.x] = fmaxf(m0[threadIdx.x], m0[threadIdx.x + o]);
      m1[threadIdx.x] = fmaxf(m1[threadIdx.x], m1[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bound[0] = m0[0];
    bound[1] = m1[0];
    bound[2] = (m0[0] > 0.0f || m1[0] > 0.0f) ? 1.0f : 0.0f;
  }
}

// -------------------------------------------------------- introspection
__global__ void k_export_links(const uint32_t* nvalid, const uint32_t* gorig, const int32_t* up,
                               const int32_t* dn, const int32_t* upc, const int32_t* dnc,
                               int32_t* oup, int32_t* odn, int32_t* oupc, int32_t* odnc) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= (int)*nvalid) return;
  uint32_t i = gorig[h];
  auto cv = [&](int32_t v) { return v >= 0 ? (int32_t)gorig[v] : -1; };
  if (oup) oup[i] = cv(up[h]);
  if (odn) odn[i] = cv(dn[h]);
  if (oupc) oupc[i] = cv(upc[h]);
  if (odnc) odnc[i] = cv(dnc[h]);
}

__global__ void k_export_tracklets(int n_rows, int64_t n_cap, const uint32_t* cnt,
                                   const uint32_t* gorig, const uint32_t* starts,
                                   const int32_t* nh, const double* that, const int32_t* hits,
                                   uint32_t* o_start, int32_t* o_nh, double* o_that,
                                   int32_t* o_hits) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int)cnt[kCntStart] || t >= n_cap) return;
  if (o_start) o_start[t] = gorig[starts[t]];
  if (o_nh) o_nh[t] = nh[t];
  if (o_that) o_that[t] = that[t];
  if (o_hits)
    for (int r = 0; r < n_rows; ++r) {
      int j = hits[(size_t)t * n_rows + r];
      o_hits[(size_t)t * n_rows + r] = j >= 0 ? (int32_t)gorig[j] : -1;
    }
}

inline int nblk(int64_t n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

// ======================================================================
// launchers
// ======================================================================
void launch_load(Prof* P, const Geo& g, const Cal& c, const ClIn& cl, const GridDims& gd, int K,
                 FindBuf& b, uint32_t* err, cudaStream_t s) {
  int init_n = K > cl.n_events * 2 ? K : cl.n_events * 2;
  TPC_LAUNCH(P, "k_init_load", s, k_init_load<<<nblk(init_n, kB256), kB256, 0, s>>>(K, cl.n_events, b.cnt, b.fill, b.zmm));
  if (cl.n > 0)
    TPC_LAUNCH(P, "k_hist", s,
               k_hist<<<nblk(cl.n, kB256), kB256, 0, s>>>(g, c, cl, b.cnt, b.zs_in, b.zmm, err));
  TPC_LAUNCH(P, "k_scan_rows", s, k_scan_rows<<<1, 1024, 0, s>>>(K, cl.n_events, gd, b.cnt, b.row_start, b.zmm, b.zr));
  if (cl.n > 0)
    TPC_LAUNCH(P, "k_scatter", s,
               k_scatter<<<nblk(cl.n, kB256), kB256, 0, s>>>(g, cl, b.row_start, b.fill, b.perm));
  size_t smem = kSortTile * sizeof(unsigned long long);
  TPC_LAUNCH(P, "k_row_sort", s, k_row_sort<<<K, 512, smem, s>>>(g, cl, gd, b.row_start, b.perm, b.zs_in, b.zr, b.gyz,
                                   b.gt, b.gorig, b.gseg, b.bin_start, err));
}

void launch_find(Prof* P, const Geo& g, const Cal& c, const Params& p, const ClIn& cl,
                 const GridDims& gd, int K, FindBuf& b, TrackBuf& tb, uint32_t* cnt,
                 uint32_t* err, cudaStream_t s) {
  int n = cl.n;
  int nb = nblk(n, kB256);
  if (n > 0) {
    const uint32_t* nv = b.row_start + K;
    TPC_LAUNCH(P, "k_neighbours", s, k_neighbours<<<nb, kB256, 0, s>>>(g, p, gd, nv, b.gyz, b.gorig, b.gseg, b.bin_start,
                                      b.zr, b.up, b.dn));
    TPC_LAUNCH(P, "k_clean", s, k_clean<<<nb, kB256, 0, s>>>(nv, b.up, b.dn, b.upc, b.dnc, b.blk_a));
  }
  TPC_LAUNCH(P, "k_scan_blocks", s, k_scan_blocks<<<1, 1024, 0, s>>>(n > 0 ? nb : 0, b.blk_a, b.off_a, nullptr, nullptr, cnt,
                                   kCntStart, 0, (uint32_t)b.cap_tl, 0u, err, kErrCapStart));
  if (n > 0)
    TPC_LAUNCH(P, "k_write_starts", s, k_write_starts<<<nb, kB256, 0, s>>>(b.row_start + K, b.upc, b.dnc, b.off_a,
                                        (uint32_t)b.cap_tl, b.starts));
  cudaMemsetAsync(b.weight, 0, sizeof(unsigned long long) * (size_t)(n > 0 ? n : 1), s);
  Grid G{b.gyz, b.gt, b.gorig, b.bin_start, b.zr};
  int ntl_blk = nblk(b.cap_tl, 128);
  TPC_LAUNCH(P, "k_tracklets", s, k_tracklets<<<ntl_blk, 128, 0, s>>>(g, c, p, gd, G, cl.mode, b.upc, b.gseg, b.starts, cnt, b.nh,
                                      b.hits, b.that, b.weight));
  int nsel = nblk(b.cap_tl, kB256);
  TPC_LAUNCH(P, "k_select_count", s, k_select_count<<<nsel, kB256, 0, s>>>(g.n_rows, p, cnt, b.nh, b.hits, b.starts, b.gorig,
                                        b.weight, b.nkeep, b.blk_a, b.blk_b));
  TPC_LAUNCH(P, "k_scan_blocks", s, k_scan_blocks<<<1, 1024, 0, s>>>(nsel, b.blk_a, b.off_a, b.blk_b, b.off_b, cnt, kCntTracks,
                                   kCntAssigned, (uint32_t)tb.cap_tr, (uint32_t)tb.cap_asg, err,
                                   kErrCapTrack));
  TPC_LAUNCH(P, "k_select_write", s, k_select_write<<<nsel, kB256, 0, s>>>(g.n_rows, cnt, b.hits, b.starts, b.that, b.gorig,
                                        b.weight, b.nh, b.nkeep, b.off_a, b.off_b, tb.cap_tr,
                                        tb.cap_asg, tb.track_start, tb.cluster_idx, tb.asg_track,
                                        tb.t_coll, tb.start_hit));
  TPC_LAUNCH(P, "k_track_end", s, k_track_end<<<1, 1, 0, s>>>(cnt, tb.track_start));
  TPC_LAUNCH(P, "k_calib", s, k_calib<<<nblk(tb.cap_asg, kB256), kB256, 0, s>>>(g, c, cl, cnt, tb.cluster_idx, tb.asg_track,
                                                    tb.t_coll, tb.yc, tb.zc, tb.meta, err));
}

void launch_set_tracks(Prof* P, const Geo& g, const Cal& c, const ClIn& cl, int64_t n_tracks,
                       int64_t n_asg, TrackBuf& tb, uint32_t* cnt, uint32_t* err, cudaStream_t s) {
  if (n_tracks > 0)
    TPC_LAUNCH(P, "k_asg_track", s, k_asg_track<<<nblk(n_tracks, kB256), kB256, 0, s>>>(cnt, tb.track_start, tb.asg_track, err));
  if (n_asg > 0)
    TPC_LAUNCH(P, "k_calib", s, k_calib<<<nblk(n_asg, kB256), kB256, 0, s>>>(g, c, cl, cnt, tb.cluster_idx, tb.asg_track,
                                                 tb.t_coll, tb.yc, tb.zc, tb.meta, err));
}

void launch_spline_bound(const float* spline, float* bound, cudaStream_t s) {
  k_spline_bound<<<1, 256, 0, s>>>(spline, bound);
}

void launch_export_links(const FindBuf& b, int n, int K, int32_t* up, int32_t* dn, int32_t* upc,
                         int32_t* dnc, cudaStream_t s) {
  if (n > 0)
    k_export_links<<<nblk(n, kB256), kB256, 0, s>>>(b.row_start + K, b.gorig, b.up, b.dn, b.upc,
                                                    b.dnc, up, dn, upc, dnc);
}

void launch_export_tracklets(const FindBuf& b, int n_rows, int64_t n_cap, const uint32_t* cnt,
                             uint32_t* start_hit, int32_t* nh, double* that, int32_t* hits,
                             cudaStream_t s) {
  int64_t m = n_cap < b.cap_tl ? n_cap : b.cap_tl;
  if (m > 0)
    k_export_tracklets<<<nblk(m, kB256), kB256, 0, s>>>(n_rows, m, cnt, b.gorig, b.starts, b.nh,
                                                        b.that, b.hits, start_hit, nh, that,
                                                        hits);
}

}  // namespace tpc
