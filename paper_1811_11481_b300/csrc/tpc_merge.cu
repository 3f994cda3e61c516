// Segment merging (arXiv:1811.11481 Sec. 2, second phase: the track segments
// found in the individual sectors are merged before the final fit).
//
// A segment is described by its refitted state at its innermost cluster (in
// its sector's frame), its pad-row range and its collision time. Segment j
// may continue segment i when both converged, lie in the same event and on
// the same side, j's sector frame is i's or a neighbour of it, and j starts
// on a pad row beyond i's last one. i's state is rotated into j's frame and
// transported to j's innermost x; in the time-frame mode j's z is expressed
// with i's collision time; the pair's chi2 is d^T (C_i' + C_j)^-1 d over the
// five parameters (Cholesky). Pairs whose tan(lambda) or q/pT differ by more
// than sqrt(2 chi2_merge) standard deviations of the difference are not
// compared. i -> j is a link when chi2 <= chi2_merge, j is i's best
// continuation and i is j's best predecessor (smallest chi2, then smallest
// index). Merged tracks are the chains of links from segments without
// predecessor, in the order of their first segment, which gives them its
// collision time and start hit.
//
// k_mg_copy    the segments copied aside (the merged set replaces them).
// k_mg_info    one thread per segment: bucket (event, sector), row range,
//              participation; bucket histogram.
// k_mg_bucket  one block: bucket offsets.
// k_mg_scatter one thread per segment: segment lists per bucket.
// k_mg_sort    one block per bucket: segments in classes of tan(lambda)
//              variance, sorted by tan(lambda) inside a class.
// k_mg_cand    one warp per segment: the segments of the three candidate
//              buckets inside its tan(lambda) window of each variance class
//              (binary searches, one per lane) that pass the prefilter,
//              appended to a pair list.
// k_mg_eval    one thread per pair: chi2; 64-bit atomic minima (chi2 bits,
//              index) give each segment its best continuation and its best
//              predecessor.
// k_mg_link    mutual best -> link.
// k_mg_len     chain length of each first segment, block-local scans.
// k_mg_top     one block: block offsets, track and cluster totals.
// k_mg_write   one warp per first segment: the merged track's clusters.
//
// Compiled with -fmad=false and IEEE division and square root: the chi2 that
// decides a link is computed with one rounding per written operation.
#include "tpc_impl.h"
#include "tpc_refit_core.cuh"

namespace tpc {
namespace {

constexpr int kMB = 256;    // threads per block of the per-segment kernels
constexpr int kScanB = 1024;  // threads per block of the scans
inline int nblk(int64_t n, int b) { return (int)((n + b - 1) / b); }

struct SegIn {
  const uint32_t* ts;     // segment CSR (copy of the track set)
  const uint32_t* ci;
  const double* that;
  const float* params;    // [n][5] refitted state at the innermost cluster
  const float* cov;       // [n][15] packed lower triangle
  const float* x;         // [n]
  const int32_t* status;  // [n]
};

constexpr uint32_t kTakesPart = 0x80000000u;

// The segments (the current track set) copied aside, so that the merged set
// can be written in their place; their count kept for the merge kernels
// (the track count is replaced by the merged count). Counts are read on the
// device and bounded by the capacities.
__global__ void k_mg_copy(int64_t cap_tr, int64_t cap_asg, const uint32_t* cnt, TrackBuf tb,
                          uint32_t* seg_ts, uint32_t* seg_ci, double* seg_that,
                          uint32_t* seg_hit, uint32_t* nseg) {
  uint32_t n = cnt[kCntTracks], na = cnt[kCntAssigned];
  if ((int64_t)n > cap_tr) n = (uint32_t)cap_tr;
  if ((int64_t)na > cap_asg) na = (uint32_t)cap_asg;
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  if (t == 0) *nseg = n;
  for (size_t k = t; k <= n; k += stride) seg_ts[k] = tb.track_start[k];
  for (size_t k = t; k < n; k += stride) {
    seg_that[k] = tb.t_coll[k];
    seg_hit[k] = tb.start_hit[k];
  }
  for (size_t k = t; k < na; k += stride) seg_ci[k] = tb.cluster_idx[k];
}

__global__ void k_mg_info(const uint32_t* nseg, ClIn cl, SegIn s, uint32_t* info,
                          uint32_t* rows, uint32_t* bk_cnt, unsigned long long* best_in,
                          unsigned long long* best_out, uint8_t* has_in) {
  int n = (int)*nseg;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t w = 0u;
  if (i < n) {
    best_in[i] = ~0ull;
    best_out[i] = ~0ull;
    has_in[i] = 0;
    uint32_t a = s.ts[i], b = s.ts[i + 1];
    uint32_t r = 0u;
    if (b > a) {
      uint32_t f = s.ci[a], l = s.ci[b - 1];
      uint32_t ev = cl.event ? cl.event[f] : 0u;
      uint32_t bk = ev * TPC_N_SECTORS + cl.sector[f];
      // clusters with an invalid event or sector (reported at load) stay out
      bool ok = s.status[i] == 0 && ev < (uint32_t)cl.n_events && cl.sector[f] < TPC_N_SECTORS;
      w = ok ? (bk | kTakesPart) : 0u;
      r = (uint32_t)cl.row[f] | ((uint32_t)cl.row[l] << 16);
    }
    info[i] = w;
    rows[i] = r;
  }
  // one atomic per bucket and warp (neighbouring segments share buckets)
  uint32_t peers = __match_any_sync(0xffffffffu, w);
  if ((w & kTakesPart) && (threadIdx.x & 31) == __ffs(peers) - 1)
    atomicAdd(&bk_cnt[w & ~kTakesPart], (uint32_t)__popc(peers));
}

// Exclusive scan of v over a block of kScanB threads; returns the prefix and
// writes the block total to *total.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t ws[kScanB / 32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < kScanB / 32 ? ws[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kScanB / 32) ws[lane] = t;
  }
  __syncthreads();
  uint32_t incl = x + (w > 0 ? ws[w - 1] : 0u);
  *total = ws[kScanB / 32 - 1];
  __syncthreads();
  return incl - v;
}

// Exclusive scan of a[0..m) in place by one block, a[m] = total.
__device__ void block_scan_inplace(uint32_t* a, int m) {
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  for (int base = 0; base < m; base += kScanB) {
    int i = base + (int)threadIdx.x;
    uint32_t v = i < m ? a[i] : 0u;
    uint32_t tot;
    uint32_t ex = block_exclusive_scan(v, &tot);
    uint32_t c = carry;
    if (i < m) a[i] = c + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry = c + tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) a[m] = carry;
}

__global__ void __launch_bounds__(kScanB) k_mg_bucket(int nb, uint32_t* bk_cnt, uint32_t* bk_fill) {
  block_scan_inplace(bk_cnt, nb);  // counts -> offsets
  for (int i = threadIdx.x; i < nb; i += kScanB) bk_fill[i] = 0u;
}

__global__ void k_mg_scatter(const uint32_t* nseg, const uint32_t* info,
                             const uint32_t* bk_start, uint32_t* bk_fill, uint32_t* bk_seg) {
  int n = (int)*nseg;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t w = i < n ? info[i] : 0u;
  // one atomic per bucket and warp
  uint32_t peers = __match_any_sync(0xffffffffu, w);
  int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
  uint32_t base = 0u;
  if ((w & kTakesPart) && lane == leader)
    base = atomicAdd(&bk_fill[w & ~kTakesPart], (uint32_t)__popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (!(w & kTakesPart)) return;
  uint32_t bk = w & ~kTakesPart;
  bk_seg[bk_start[bk] + base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)i;
}

// Each bucket's segments are grouped into classes of tan(lambda) variance and
// sorted by tan(lambda) inside a class (one block per bucket, bitonic sort in
// shared memory): a segment then searches, class by class, only the window
// of tan(lambda) that its prefilter admits against the class's largest
// variance. The prefilter data of the candidates (tan(lambda), q/pT, their
// variances, first row) are stored in sorted order next to each other.
// Buckets above kBucketSortMax stay unsorted and are scanned whole.
constexpr int kBucketSortMax = 16384;
constexpr int kSortThreads = 1024;
constexpr int kVarClasses = 4;
// upper tan(lambda) variance of the classes but the last (2^-20, 2^-17, 2^-14)
__constant__ float kClassVar[kVarClasses - 1] = {9.5367431640625e-07f, 7.62939453125e-06f,
                                                 6.103515625e-05f};

// Sort key of a float: increasing with the value; every NaN after +inf.
__device__ __forceinline__ uint32_t orderable(float f) {
  uint32_t u = f == f ? __float_as_uint(f) : 0x7fffffffu;
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ int var_class(float v) {
  int c = 0;
#pragma unroll
  for (int k = 0; k < kVarClasses - 1; ++k) c += v > kClassVar[k] ? 1 : 0;
  return c;
}

__global__ void __launch_bounds__(kSortThreads) k_mg_sort(const uint32_t* bk_start,
                                                          uint32_t* bk_seg, float4* bk_v,
                                                          float* bk_t, uint32_t* bk_rlo,
                                                          uint32_t* bk_cls,
                                                          const uint32_t* rows,
                                                          const float* params,
                                                          const float* cov) {
  extern __shared__ unsigned long long sk[];
  int b = blockIdx.x;
  uint32_t a = bk_start[b], e = bk_start[b + 1];
  int m = (int)(e - a);
  if (m > kBucketSortMax) {
    // unsorted: everything in the last class, which is scanned whole
    if (threadIdx.x <= kVarClasses)
      bk_cls[(size_t)b * (kVarClasses + 1) + threadIdx.x] = threadIdx.x == kVarClasses ? e : a;
    for (int i = threadIdx.x; i < m; i += kSortThreads) {
      uint32_t j = bk_seg[a + i];
      bk_v[a + i] = make_float4(params[(size_t)j * 5 + 3], params[(size_t)j * 5 + 4],
                                cov[(size_t)j * 15 + 9], cov[(size_t)j * 15 + 14]);
      bk_t[a + i] = params[(size_t)j * 5 + 3];
      bk_rlo[a + i] = rows[j] & 0xffffu;
    }
    return;
  }
  int np = 1;
  while (np < m) np <<= 1;
  int cnt[kVarClasses];
#pragma unroll
  for (int c = 0; c < kVarClasses; ++c) cnt[c] = 0;
  for (int i = threadIdx.x; i < np; i += kSortThreads) {
    if (i < m) {
      uint32_t j = bk_seg[a + i];
      int c = var_class(cov[(size_t)j * 15 + 9]);
      ++cnt[c];
      sk[i] = ((unsigned long long)c << 62) |
              ((unsigned long long)orderable(params[(size_t)j * 5 + 3]) << 30) | j;
    } else {
      sk[i] = ~0ull;
    }
  }
  // class boundaries
  __shared__ int ccount[kVarClasses];
  if (threadIdx.x < kVarClasses) ccount[threadIdx.x] = 0;
  __syncthreads();
#pragma unroll
  for (int c = 0; c < kVarClasses; ++c)
    if (cnt[c]) atomicAdd(&ccount[c], cnt[c]);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t o = a;
    for (int c = 0; c < kVarClasses; ++c) {
      bk_cls[(size_t)b * (kVarClasses + 1) + c] = o;
      o += (uint32_t)ccount[c];
    }
    bk_cls[(size_t)b * (kVarClasses + 1) + kVarClasses] = o;
  }
  for (int k = 2; k <= np; k <<= 1)
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int i = threadIdx.x; i < np; i += kSortThreads) {
        int l = i ^ jj;
        if (l > i) {
          unsigned long long x = sk[i], y = sk[l];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            sk[i] = y;
            sk[l] = x;
          }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < m; i += kSortThreads) {
    uint32_t j = (uint32_t)(sk[i] & 0x3fffffffull);
    bk_seg[a + i] = j;
    bk_v[a + i] = make_float4(params[(size_t)j * 5 + 3], params[(size_t)j * 5 + 4],
                              cov[(size_t)j * 15 + 9], cov[(size_t)j * 15 + 14]);
    bk_t[a + i] = params[(size_t)j * 5 + 3];
    bk_rlo[a + i] = rows[j] & 0xffffu;
  }
}

struct MergeCfg {
  RefitCfg rc;   // kB, s_max and the frame rotations
  float cut;     // chi2_merge
  int mode;      // 1: time frame
  double vdrift;
};

// chi2 of "j continues i"; false when the pair is not compared or fails.
__device__ bool pair_chi2(const MergeCfg& m, int side, const float pi[5], const float Ci[15],
                          float xi, double thi, int fi, const float* pj, const float* Cj,
                          float xj, double thj, int fj, float& chi2) {
#pragma unroll
  for (int k = 3; k <= 4; ++k) {
    int d = sidx(k, k);
    float dd = pi[k] - pj[k];
    if (dd * dd > (2.0f * m.cut) * (Ci[d] + Cj[d])) return false;
  }
  float p[5], C[15];
#pragma unroll
  for (int k = 0; k < 5; ++k) p[k] = pi[k];
#pragma unroll
  for (int k = 0; k < 15; ++k) C[k] = Ci[k];
  float x = xi;
  if (fj != fi) {
    int r = frame_step(fi, fj);
    if (!rotate_frame(m.rc.kB, m.rc.s_max, m.rc.rot_c[r], m.rc.rot_s[r], p, C, x)) return false;
  }
  if (!propagate(m.rc.kB, m.rc.s_max, p, C, x, xj)) return false;
  float shift = 0.0f;
  if (m.mode == 1) {
    double sg = side == 0 ? 1.0 : -1.0;
    shift = (float)(sg * m.vdrift * (thi - thj));
  }
  float d[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) d[k] = p[k] - pj[k];
  d[1] = p[1] - (pj[1] + shift);
  float L[5][5];
#pragma unroll
  for (int a = 0; a < 5; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      float acc = C[sidx(a, b)] + Cj[sidx(a, b)];
#pragma unroll
      for (int k = 0; k < b; ++k) acc = acc - L[a][k] * L[b][k];
      if (a == b) {
        if (!(acc > 0.0f)) return false;
        L[a][a] = sqrtf(acc);
      } else {
        L[a][b] = acc / L[b][b];
      }
    }
  float w[5];
#pragma unroll
  for (int a = 0; a < 5; ++a) {
    float acc = d[a];
#pragma unroll
    for (int k = 0; k < a; ++k) acc = acc - L[a][k] * w[k];
    w[a] = acc / L[a][a];
  }
  float ch = 0.0f;
#pragma unroll
  for (int a = 0; a < 5; ++a) ch = ch + w[a] * w[a];
  chi2 = ch;
  return ch <= m.cut;
}

// Candidate pairs. One warp per segment i: lanes 0..11 each find one
// candidate range (three buckets times four variance classes; in the sorted
// classes the window of tan(lambda) that the prefilter admits, by binary
// search), so that the searches run side by side; then the warp scans the
// concatenated ranges 128 candidates at a time and appends the pairs that
// pass the prefilter to a list (one atomic per warp and step). The chi2 of
// the pairs is the long part and runs in k_mg_eval, one thread per pair:
// here most lanes would idle while one evaluates.
constexpr int kRanges = 3 * kVarClasses;
constexpr int kPerLane = 4;  // candidates per lane and step, their loads issued together

__global__ void __launch_bounds__(kMB) k_mg_cand(const uint32_t* nseg, float cut,
                                                 const float* params,
                                                 const float* cov, const uint32_t* info,
                                                 const uint32_t* rows, const uint32_t* bk_seg,
                                                 const float4* bk_v, const float* bk_t,
                                                 const uint32_t* bk_rlo,
                                                 const uint32_t* bk_cls, uint2* pairs,
                                                 uint32_t cap_pairs, uint32_t* n_pairs) {
  __shared__ uint32_t r_first[kMB / 32][kRanges], r_pre[kMB / 32][kRanges + 1];
  int n = (int)*nseg;
  int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  if (i >= n) return;
  uint32_t wi = info[i];
  if (!(wi & kTakesPart)) return;
  uint32_t bk = wi & ~kTakesPart;
  int sec = (int)(bk % TPC_N_SECTORS);
  uint32_t ev0 = bk - (uint32_t)sec;
  int side = sec / 18, fi = sec % 18;
  int rhi = (int)(rows[i] >> 16);
  const float ti = params[(size_t)i * 5 + 3], qi = params[(size_t)i * 5 + 4];
  const float vti = cov[(size_t)i * 15 + 9], vqi = cov[(size_t)i * 15 + 14];
  const float lim = 2.0f * cut;
  // the candidate ranges, one per lane
  uint32_t len = 0u;
  if (lane < kRanges) {
    int df = lane / kVarClasses, c = lane % kVarClasses;
    int fj = df == 0 ? fi : (df == 1 ? (fi + 1) % 18 : (fi + 17) % 18);
    const uint32_t* cls = bk_cls + (size_t)(ev0 + (uint32_t)(side * 18 + fj)) * (kVarClasses + 1);
    uint32_t q0 = cls[c], q1 = cls[c + 1];
    if (c < kVarClasses - 1 && q0 < q1) {
      // the prefilter's tan(lambda) bound with the class's largest variance,
      // widened against rounding: a superset of the admitted
      float w = sqrtf(lim * (vti + kClassVar[c])) * 1.001f + 1e-6f;
      float lo = ti - w, hi = ti + w;
      uint32_t l = q0, r = q1;
      while (l < r) {  // first entry not below lo
        uint32_t mid = (l + r) >> 1;
        if (bk_t[mid] < lo)
          l = mid + 1;
        else
          r = mid;
      }
      q0 = l;
      r = q1;
      while (l < r) {  // first entry beyond hi (NaN counts as beyond)
        uint32_t mid = (l + r) >> 1;
        if (!(bk_t[mid] <= hi))
          r = mid;
        else
          l = mid + 1;
      }
      q1 = l;
    }
    len = q1 > q0 ? q1 - q0 : 0u;
    r_first[wl][lane] = q0;
  }
  uint32_t incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane < kRanges) r_pre[wl][lane] = incl - len;
  uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  if (lane == 0) r_pre[wl][kRanges] = total;
  __syncwarp();
  int k = 0;  // the lane's current range
  for (uint32_t base = 0; base < total; base += 32 * kPerLane) {
    uint32_t qq[kPerLane];
    bool in[kPerLane];
#pragma unroll
    for (int u = 0; u < kPerLane; ++u) {
      uint32_t g = base + (uint32_t)(u * 32 + lane);
      in[u] = g < total;
      qq[u] = 0u;
      if (in[u]) {
        while (r_pre[wl][k + 1] <= g) ++k;
        qq[u] = r_first[wl][k] + (g - r_pre[wl][k]);
      }
    }
    uint32_t rl[kPerLane], jj[kPerLane];
    float4 v[kPerLane];
#pragma unroll
    for (int u = 0; u < kPerLane; ++u) {
      rl[u] = in[u] ? bk_rlo[qq[u]] : 0u;
      v[u] = in[u] ? bk_v[qq[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
      jj[u] = in[u] ? bk_seg[qq[u]] : 0u;
    }
    uint32_t msk[kPerLane], cnt = 0u;
#pragma unroll
    for (int u = 0; u < kPerLane; ++u) {
      // the prefilter of pair_chi2, on the same values
      float dt = ti - v[u].x, dq = qi - v[u].y;
      bool pass = in[u] && (int)rl[u] > rhi && !(dt * dt > lim * (vti + v[u].z)) &&
                  !(dq * dq > lim * (vqi + v[u].w)) && (int)jj[u] != i;
      msk[u] = __ballot_sync(0xffffffffu, pass);
      cnt += __popc(msk[u]);
    }
    if (cnt == 0) continue;
    uint32_t at = 0;
    if (lane == 0) at = atomicAdd(n_pairs, cnt);
    at = __shfl_sync(0xffffffffu, at, 0);
    uint32_t below = (1u << lane) - 1u;
#pragma unroll
    for (int u = 0; u < kPerLane; ++u) {
      uint32_t p = at + __popc(msk[u] & below);
      if ((msk[u] >> lane) & 1u && p < cap_pairs) pairs[p] = make_uint2((uint32_t)i, jj[u]);
      at += __popc(msk[u]);
    }
  }
}

// chi2 of each candidate pair (one thread per pair), folded into i's best
// continuation and j's best predecessor (64-bit atomic minimum of chi2 bits
// and index: the smallest chi2, then the smallest index).
__global__ void __launch_bounds__(kMB) k_mg_eval(MergeCfg m, SegIn s, const uint32_t* info,
                                                 const uint2* pairs, uint32_t cap_pairs,
                                                 const uint32_t* n_pairs,
                                                 unsigned long long* best_in,
                                                 unsigned long long* best_out) {
  uint32_t np = *n_pairs;
  if (np > cap_pairs) np = cap_pairs;
  uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += stride) {
    uint2 e = pairs[p];
    uint32_t i = e.x, j = e.y;
    uint32_t bki = info[i] & ~kTakesPart, bkj = info[j] & ~kTakesPart;
    int seci = (int)(bki % TPC_N_SECTORS), secj = (int)(bkj % TPC_N_SECTORS);
    float pi[5], Ci[15];
#pragma unroll
    for (int k = 0; k < 5; ++k) pi[k] = s.params[(size_t)i * 5 + k];
#pragma unroll
    for (int k = 0; k < 15; ++k) Ci[k] = s.cov[(size_t)i * 15 + k];
    float chi2;
    if (!pair_chi2(m, seci / 18, pi, Ci, s.x[i], s.that[i], seci % 18, s.params + (size_t)j * 5,
                   s.cov + (size_t)j * 15, s.x[j], s.that[j], secj % 18, chi2))
      continue;
    unsigned long long cb = (unsigned long long)__float_as_uint(chi2) << 32;
    atomicMin(&best_out[i], cb | j);
    atomicMin(&best_in[j], cb | i);
  }
}

__global__ void k_mg_link(const uint32_t* nseg, const unsigned long long* best_in,
                          const unsigned long long* best_out, int32_t* next, int32_t* next_out,
                          float* link_chi2, uint8_t* has_in, const uint32_t* n_pairs,
                          uint32_t cap_pairs, uint32_t* err) {
  int n = (int)*nseg;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  // pairs beyond the list's capacity were dropped: the links are incomplete
  if (i == 0 && *n_pairs > cap_pairs) atomicOr(err, kErrCapPairs);
  if (i >= n) return;
  unsigned long long b = best_out[i];
  int32_t nx = -1;
  float c = 0.0f;
  if (b != ~0ull) {
    uint32_t j = (uint32_t)b;
    if ((uint32_t)best_in[j] == (uint32_t)i) {
      nx = (int32_t)j;
      c = __uint_as_float((uint32_t)(b >> 32));
      has_in[j] = 1;
    }
  }
  next[i] = nx;
  if (next_out) next_out[i] = nx;
  if (link_chi2) link_chi2[i] = c;
}

// Chains are acyclic and at most one segment per pad row long: along a link
// the first row strictly increases.
__global__ void __launch_bounds__(kScanB) k_mg_len(const uint32_t* nseg, const uint32_t* ts,
                                                   const int32_t* next, const uint8_t* has_in,
                                                   uint32_t* hpos, uint32_t* cpos,
                                                   uint32_t* blk_h, uint32_t* blk_c) {
  int n = (int)*nseg;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t h = 0u, len = 0u;
  if (i < n && !has_in[i]) {
    h = 1u;
    int s = i;
    for (int k = 0; s >= 0 && k <= TPC_MAX_ROWS; ++k) {
      len += ts[s + 1] - ts[s];
      s = next[s];
    }
  }
  uint32_t th, tc;
  uint32_t eh = block_exclusive_scan(h, &th);
  uint32_t ec = block_exclusive_scan(len, &tc);
  if (i < n) {
    hpos[i] = eh;
    cpos[i] = ec;
  }
  if (threadIdx.x == 0) {
    blk_h[blockIdx.x] = th;
    blk_c[blockIdx.x] = tc;
  }
}

__global__ void __launch_bounds__(kScanB) k_mg_top(int nb, uint32_t* blk_h, uint32_t* blk_c,
                                                   uint32_t* cnt, uint32_t* track_start) {
  block_scan_inplace(blk_h, nb);
  block_scan_inplace(blk_c, nb);
  if (threadIdx.x == 0) {
    cnt[kCntTracks] = blk_h[nb];
    track_start[blk_h[nb]] = blk_c[nb];
  }
}

__global__ void k_mg_write(const uint32_t* nseg, SegIn s, const uint32_t* seg_hit,
                           const int32_t* next,
                           const uint8_t* has_in, const uint32_t* hpos, const uint32_t* cpos,
                           const uint32_t* blk_h, const uint32_t* blk_c, TrackBuf tb) {
  int n = (int)*nseg;
  int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (i >= n || has_in[i]) return;
  int blk = i / kScanB;
  uint32_t t = blk_h[blk] + hpos[i];
  uint32_t o = blk_c[blk] + cpos[i];
  if (lane == 0) {
    tb.track_start[t] = o;
    tb.t_coll[t] = s.that[i];
    tb.start_hit[t] = seg_hit[i];
  }
  int sg = i;
  for (int k = 0; sg >= 0 && k <= TPC_MAX_ROWS; ++k) {
    uint32_t a = s.ts[sg], len = s.ts[sg + 1] - a;
    for (uint32_t q = lane; q < len; q += 32) {
      tb.cluster_idx[o + q] = s.ci[a + q];
      tb.asg_track[o + q] = t;
    }
    o += len;
    sg = next[sg];
  }
}

// Collision time after merging (time-frame mode, Sec. 4): the closest
// approach of the fitted helix to the beam line is moved to z = 0, then the
// time is clipped so that every cluster's drift time t - t0 - that lies in
// [0, L / v_drift] (the lower bound wins when both apply). One warp per
// track: lanes reduce the range of t - t0 over the clusters.
__global__ void k_refine_time(int cap, Geo g, Cal c, ClIn cl, const uint32_t* cnt,
                              const uint32_t* ts, const uint32_t* ci, const float* params,
                              const float* x, const int32_t* status, double* t_coll,
                              double* t_out) {
  int lane = threadIdx.x & 31;
  int n = (int)cnt[kCntTracks];
  if (n > cap) n = cap;
  int nw = (int)((gridDim.x * (size_t)blockDim.x) >> 5);
  for (int T = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5); T < n; T += nw) {
    uint32_t a = ts[T], b = ts[T + 1];
    double th = t_coll[T];
    if (cl.mode == 1 && status[T] == 0 && b > a) {
      double lo = cl.t[ci[a]] - c.t0, hi = lo;
      for (uint32_t q = a + lane; q < b; q += 32) {
        double d = cl.t[ci[q]] - c.t0;
        lo = fmin(lo, d);
        hi = fmax(hi, d);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      }
      float p[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) p[k] = params[(size_t)T * 5 + k];
      float z0 = dca_z(g.kB, p, x[T]);
      double sg = cl.sector[ci[a]] < 18 ? 1.0 : -1.0;
      th = th - (sg * (double)z0) / c.vdrift;
      double tmax = (double)g.L / c.vdrift;
      if (hi - th > tmax) th = th + ((hi - th) - tmax);
      if (lo - th < 0.0) th = th + (lo - th);
    }
    if (lane == 0) {
      t_coll[T] = th;
      if (t_out) t_out[T] = th;
    }
  }
}

}  // namespace

void setup_merge_kernels() {
  cudaFuncSetAttribute(k_mg_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(kBucketSortMax * sizeof(unsigned long long)));
}

void launch_refine_time(Prof* P, const Geo& g, const Cal& c, const ClIn& cl, int64_t cap_tr,
                        const uint32_t* cnt, TrackBuf& tb, const float* params, const float* x,
                        const int32_t* status, double* t_out, cudaStream_t s) {
  if (cap_tr <= 0) return;
  int blocks = nblk(cap_tr * 32, kMB);
  if (blocks > 64 * 148) blocks = 64 * 148;  // grid-stride beyond 64 blocks per SM
  TPC_LAUNCH(P, "k_refine_time", s,
             k_refine_time<<<blocks, kMB, 0, s>>>((int)cap_tr, g, c, cl, cnt, tb.track_start,
                                                  tb.cluster_idx, params, x, status, tb.t_coll,
                                                  t_out));
}

void launch_merge(Prof* P, const Geo& g, const Params& p, const Cal& c, const ClIn& cl,
                  int64_t cap_n, bool copy, TrackBuf& tb, MergeBuf& mb, const float* params,
                  const float* cov, const float* x, const int32_t* status, int32_t* next_out,
                  float* link_chi2, uint32_t* cnt, uint32_t* err, cudaStream_t s) {
  if (cap_n <= 0) return;
  int nb = cl.n_events * TPC_N_SECTORS;
  SegIn si{mb.seg_ts, mb.seg_ci, mb.seg_that, params, cov, x, status};
  MergeCfg m;
  m.rc = RefitCfg{};
  m.rc.kB = g.kB;
  m.rc.s_max = p.s_max;
  set_frame_rotations(m.rc);
  m.cut = p.chi2_merge;
  m.mode = cl.mode;
  m.vdrift = c.vdrift;
  int64_t cap_asg = tb.cap_asg < mb.cap_asg ? tb.cap_asg : mb.cap_asg;
  if (copy)
    TPC_LAUNCH(P, "k_mg_copy", s,
               k_mg_copy<<<16 * 148, kMB, 0, s>>>(cap_n, cap_asg, cnt, tb, mb.seg_ts, mb.seg_ci,
                                                  mb.seg_that, mb.seg_hit, mb.n_seg));
  cudaMemsetAsync(mb.n_pairs, 0, sizeof(uint32_t), s);
  cudaMemsetAsync(mb.bk_cnt, 0, sizeof(uint32_t) * (nb + 1), s);
  TPC_LAUNCH(P, "k_mg_info", s,
             k_mg_info<<<nblk(cap_n, kMB), kMB, 0, s>>>(mb.n_seg, cl, si, mb.info, mb.rows,
                                                        mb.bk_cnt, mb.best_in, mb.best_out,
                                                        mb.has_in));
  TPC_LAUNCH(P, "k_mg_bucket", s, k_mg_bucket<<<1, kScanB, 0, s>>>(nb, mb.bk_cnt, mb.bk_fill));
  TPC_LAUNCH(P, "k_mg_scatter", s,
             k_mg_scatter<<<nblk(cap_n, kMB), kMB, 0, s>>>(mb.n_seg, mb.info, mb.bk_cnt,
                                                           mb.bk_fill, mb.bk_seg));
  TPC_LAUNCH(P, "k_mg_sort", s,
             k_mg_sort<<<nb, kSortThreads, kBucketSortMax * sizeof(unsigned long long), s>>>(
                 mb.bk_cnt, mb.bk_seg, mb.bk_v, mb.bk_t, mb.bk_rlo, mb.bk_cls, mb.rows, params,
                 cov));
  TPC_LAUNCH(P, "k_mg_cand", s,
             k_mg_cand<<<nblk(cap_n * 32, kMB), kMB, 0, s>>>(
                 mb.n_seg, m.cut, params, cov, mb.info, mb.rows, mb.bk_seg, mb.bk_v, mb.bk_t,
                 mb.bk_rlo, mb.bk_cls, mb.pairs, (uint32_t)mb.cap_pairs, mb.n_pairs));
  TPC_LAUNCH(P, "k_mg_eval", s,
             k_mg_eval<<<4 * 148, kMB, 0, s>>>(m, si, mb.info, mb.pairs, (uint32_t)mb.cap_pairs,
                                               mb.n_pairs, mb.best_in, mb.best_out));
  TPC_LAUNCH(P, "k_mg_link", s,
             k_mg_link<<<nblk(cap_n, kMB), kMB, 0, s>>>(mb.n_seg, mb.best_in, mb.best_out,
                                                        mb.next, next_out, link_chi2, mb.has_in,
                                                        mb.n_pairs, (uint32_t)mb.cap_pairs,
                                                        err));
  int nsb = nblk(cap_n, kScanB);
  TPC_LAUNCH(P, "k_mg_len", s,
             k_mg_len<<<nsb, kScanB, 0, s>>>(mb.n_seg, mb.seg_ts, mb.next, mb.has_in, mb.hpos,
                                             mb.cpos, mb.blk_h, mb.blk_c));
  TPC_LAUNCH(P, "k_mg_top", s,
             k_mg_top<<<1, kScanB, 0, s>>>(nsb, mb.blk_h, mb.blk_c, cnt, tb.track_start));
  TPC_LAUNCH(P, "k_mg_write", s,
             k_mg_write<<<nblk(cap_n * 32, kMB), kMB, 0, s>>>(mb.n_seg, si, mb.seg_hit, mb.next,
                                                              mb.has_in, mb.hpos, mb.cpos,
                                                              mb.blk_h, mb.blk_c, tb));
}

}  // namespace tpc
