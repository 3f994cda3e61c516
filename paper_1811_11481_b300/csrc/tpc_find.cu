// Track finding on the GPU (arXiv:1811.11481 Sec. 2 and Sec. 4).
//
// Compiled with -fmad=false: the neighbour finder's windows and argmins are
// taken on single-precision values rounded once per written operation; the
// tracklet constructor's Kalman steps use the explicit Fast arithmetic of
// tpc_math.cuh (fused multiply-adds, approximate reciprocals), the same bits
// whatever the launch shape.
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

// Row histogram, seeding z and the z range of each (event, side). A fixed
// grid strides over the clusters; the z range is first reduced per block in
// shared memory (the global minimum and maximum would otherwise take one
// contended atomic per cluster), for up to kHistSides (event, side) pairs.
constexpr int kHistSides = 2048;
__global__ void __launch_bounds__(256) k_hist(Geo g, Cal c, ClIn cl, uint32_t* cnt,
                                              float* zs_in, int32_t* zmm, uint32_t* err) {
  __shared__ int32_t smin[kHistSides], smax[kHistSides];
  const int nsides = cl.n_events * 2;
  const bool local = nsides <= kHistSides;
  if (local)
    for (int q = threadIdx.x; q < nsides; q += blockDim.x) {
      smin[q] = f2ord(3.0e38f);
      smax[q] = f2ord(-3.0e38f);
    }
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cl.n; i += gridDim.x * blockDim.x) {
    int r = cl.row[i], s = cl.sector[i];
    int e = cl.event ? (int)cl.event[i] : 0;
    if (r >= g.n_rows || s >= kNS || e >= cl.n_events) {
      atomicOr(err, kErrArg);
      zs_in[i] = 0.0f;
      continue;
    }
    float zs = seed_z(g, c, cl.mode, cl.mode == 0 ? cl.z[i] : 0.0f,
                      cl.mode == 1 ? cl.t[i] : 0.0, s);
    zs_in[i] = zs;
    if (!(fabsf(zs) < 1.0e30f)) {
      atomicOr(err, kErrArg);
      continue;
    }
    int key = (e * kNS + s) * g.n_rows + r;
    atomicAdd(&cnt[key], 1u);
    int side = e * 2 + (s >= 18 ? 1 : 0);
    int32_t o = f2ord(zs);
    if (local) {
      if (o < smin[side]) atomicMin(&smin[side], o);
      if (o > smax[side]) atomicMax(&smax[side], o);
    } else {
      if (o < zmm[2 * side]) atomicMin(&zmm[2 * side], o);
      if (o > zmm[2 * side + 1]) atomicMax(&zmm[2 * side + 1], o);
    }
  }
  __syncthreads();
  if (local)
    for (int q = threadIdx.x; q < nsides; q += blockDim.x) {
      if (smin[q] != f2ord(3.0e38f)) atomicMin(&zmm[2 * q], smin[q]);
      if (smax[q] != f2ord(-3.0e38f)) atomicMax(&zmm[2 * q + 1], smax[q]);
    }
}

// Single block: bucket offsets, the z range of each (event, side) and the bin
// geometry of each (event, sector): ny x nz bins of about tau clusters each,
// square in (y, z) on average, shared by the rows of the sector.
// Many buckets (a batch of events): the bucket offsets in three steps, so
// that no single block walks all of them: k_rows_local scans each block's
// counts (row_start holds block-local offsets, blk the block totals),
// k_scan_rows scans blk into block offsets (and reads row_start through
// them), k_rows_add adds them.
constexpr int kRowScanBlock = 1024;
constexpr int kRowScanSplit = 8 * kRowScanBlock;  // buckets above which the scan is split
__global__ void __launch_bounds__(kRowScanBlock) k_rows_local(int K, const uint32_t* cnt,
                                                              uint32_t* row_start, uint32_t* blk) {
  int i = blockIdx.x * kRowScanBlock + threadIdx.x;
  uint32_t v = i < K ? cnt[i] : 0u;
  uint32_t tot;
  uint32_t ex = block_excl_scan(v, &tot);
  if (i < K) row_start[i] = ex;
  if (threadIdx.x == 0) blk[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kRowScanBlock) k_rows_add(int K, const uint32_t* blk,
                                                            uint32_t* row_start) {
  int i = blockIdx.x * kRowScanBlock + threadIdx.x;
  if (i < K) row_start[i] += blk[blockIdx.x];
}

// nblk_rows == 0: the bucket offsets are scanned here from cnt; otherwise
// row_start holds block-local offsets and blk the nblk_rows block totals,
// which are scanned here in place (k_rows_add then completes row_start).
__global__ void k_scan_rows(Geo g, int K, int n_events, GridDims gd, const uint32_t* cnt,
                            uint32_t* row_start, int nblk_rows, uint32_t* blk,
                            const int32_t* zmm, float* zr, uint2* es_dims, uint32_t* n_bins) {
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  const int nscan = nblk_rows > 0 ? nblk_rows : K;
  uint32_t* dst = nblk_rows > 0 ? blk : row_start;
  for (int base = 0; base < nscan; base += blockDim.x) {
    int i = base + threadIdx.x;
    uint32_t v = i < nscan ? (nblk_rows > 0 ? blk[i] : cnt[i]) : 0u;
    uint32_t tot;
    uint32_t ex = block_excl_scan(v, &tot);
    __syncthreads();
    if (i < nscan) dst[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  const uint32_t total = carry;
  if (threadIdx.x == 0) row_start[K] = total;
  __syncthreads();
  // final offset of bucket i (i <= K)
  auto rs = [&](int i) -> uint32_t {
    if (nblk_rows == 0 || i >= K) return row_start[i];
    return row_start[i] + blk[i / kRowScanBlock];
  };
  for (int i = threadIdx.x; i < n_events * 2; i += blockDim.x) {
    float lo = ord2f(zmm[2 * i]), hi = ord2f(zmm[2 * i + 1]);
    if (!(hi >= lo)) {
      zr[2 * i] = 0.0f;
      zr[2 * i + 1] = 0.0f;
    } else {
      float z0 = lo - gd.z_margin;
      float span = (hi + gd.z_margin) - z0;
      zr[2 * i] = z0;
      zr[2 * i + 1] = 1.0f / span;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  int nes = n_events * kNS;
  int R = g.n_rows;
  float xm = g.rx[R / 2];
  float W = 2.0f * (xm * g.tan_half + gd.y_margin);
  for (int base = 0; base < nes; base += blockDim.x) {
    int es = base + threadIdx.x;
    uint32_t sz = 0u;
    uint32_t dims = 1u | (1u << 16);
    if (es < nes) {
      uint32_t tot = rs((es + 1) * R) - rs(es * R);
      int nbt = (int)((float)tot / ((float)R * gd.tau));
      if (nbt < 1) nbt = 1;
      if (nbt > gd.nb_max) nbt = gd.nb_max;
      int side = (es / kNS) * 2 + ((es % kNS) >= 18 ? 1 : 0);
      float invspan = zr[2 * side + 1];
      float H = invspan > 0.0f ? 1.0f / invspan : 1.0f;
      int ny = (int)(sqrtf((float)nbt * W / H) + 0.5f);
      if (ny < 1) ny = 1;
      if (ny > gd.ny_max) ny = gd.ny_max;
      if (ny > nbt) ny = nbt;
      int nz = nbt / ny;
      if (nz < 1) nz = 1;
      dims = (uint32_t)ny | ((uint32_t)nz << 16);
      sz = (uint32_t)R * (uint32_t)(ny * nz + 1);
    }
    uint32_t tot;
    uint32_t ex = block_excl_scan(sz, &tot);
    if (es < nes) es_dims[es] = make_uint2(carry + ex, dims);
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_bins = carry;
}

// Local y (cm) of a grid coordinate. With native pad input (the next step
// the paper names after Sec. 4: tracking in native pad, row and time
// coordinates, transformed to space on the fly) the grid keeps each
// cluster's pad position, and every kernel that reads one turns it into cm
// with the row's pad pitch and centre (two roundings, as for the input).
// The conversion of one row, loaded once by its reader: the pad centre and
// pitch, or 0 and 1 without pads ((v - 0) * 1 is v exactly).
struct RowPad {
  float c, w;
  __device__ __forceinline__ float y(float v) const { return (v - c) * w; }
};
__device__ __forceinline__ RowPad row_pad(const Geo& g, int pads, int r) {
  return pads ? RowPad{g.pc[r], g.pw[r]} : RowPad{0.0f, 1.0f};
}
__device__ __forceinline__ float grid_y(const Geo& g, int pads, int r, float v) {
  return row_pad(g, pads, r).y(v);
}

// Bucket order: the input index and, alongside, (y or pad position, seeding
// z), so that the row sorts read their clusters contiguously.
__global__ void k_scatter(Geo g, ClIn cl, const uint32_t* row_start, const float* zs_in,
                          uint32_t* fill, uint32_t* perm, float2* pyz) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cl.n) return;
  int r = cl.row[i], s = cl.sector[i];
  int e = cl.event ? (int)cl.event[i] : 0;
  if (r >= g.n_rows || s >= kNS || e >= cl.n_events) return;
  int key = (e * kNS + s) * g.n_rows + r;
  uint32_t pos = row_start[key] + atomicAdd(&fill[key], 1u);
  perm[pos] = (uint32_t)i;
  pyz[pos] = make_float2(cl.y[i], zs_in[i]);
}

// Search-grid geometry of one (event, sector): tables of nb + 1 bin offsets
// per row starting at base + row * (nb + 1).
struct Bins {
  uint32_t base;
  int ny, nz, nb;
};
__device__ __forceinline__ Bins es_bins(const uint2* es_dims, int es) {
  uint2 d = es_dims[es];
  Bins b;
  b.base = d.x;
  b.ny = (int)(d.y & 0xffffu);
  b.nz = (int)(d.y >> 16);
  b.nb = b.ny * b.nz;
  return b;
}
// Bin of a coordinate. The same function places the clusters and bounds
// the search boxes, so it need not be correctly rounded: the boxes carry a
// margin (>= 0.01 cm) far above its error, and it is monotone in y.
__device__ __forceinline__ int bin_y(const Geo& g, const GridDims& gd, int r, int ny, float y) {
  float hw = g.rx[r] * g.tan_half + gd.y_margin;
  float v = (y + hw) * __fdividef((float)ny, 2.0f * hw);
  int iy = (int)floorf(v);
  if (!(v == v)) iy = 0;
  return iy < 0 ? 0 : (iy >= ny ? ny - 1 : iy);
}
__device__ __forceinline__ int bin_z(const float* zr, int side, int nz, float z) {
  float v = (z - zr[2 * side]) * ((float)nz * zr[2 * side + 1]);
  int iz = (int)floorf(v);
  if (!(v == v)) iz = 0;
  return iz < 0 ? 0 : (iz >= nz ? nz - 1 : iz);
}

// Sort key of a cluster in its bucket: bin, then input index, then its slot
// j in the bucket (unique already; carried to find its (y, z) after sorting).
__device__ __forceinline__ unsigned long long sort_key(int b, uint32_t i, int j) {
  return ((unsigned long long)(uint32_t)b << 46) | ((unsigned long long)i << 15) | (uint32_t)j;
}
__device__ __forceinline__ int key_bin(unsigned long long k) { return (int)(k >> 46); }
__device__ __forceinline__ uint32_t key_index(unsigned long long k) {
  return (uint32_t)((k >> 15) & 0x7fffffffu);
}
__device__ __forceinline__ uint32_t key_slot(unsigned long long k) {
  return (uint32_t)(k & 0x7fffu);
}

// Bitonic sort of one (event, sector, row) bucket by (bin, input index) in
// shared memory (keys[] holds 'tile' entries), then the grid-ordered SoA and
// the bin offsets of the bucket.
__device__ void sort_bucket(const Geo& g, const GridDims& gd, const Bins& B, int seg,
                            uint32_t start, int n, const uint32_t* perm, const float2* pyz,
                            const float* zr, float2* gyz, uint32_t* gorig, uint32_t* gseg,
                            uint16_t* bs, unsigned long long* keys) {
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
      float2 v = pyz[start + j];
      int b = bin_z(zr, side, B.nz, v.y) * B.ny + bin_y(g, gd, r, B.ny, grid_y(g, gd.pads, r, v.x));
      k = sort_key(b, i, j);
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
    int b = key_bin(k);
    int bprev = j > 0 ? key_bin(keys[j - 1]) : -1;
    for (int q = bprev + 1; q <= b; ++q) bs[q] = (uint16_t)j;
    if (j == n - 1)
      for (int q = b + 1; q <= B.nb; ++q) bs[q] = (uint16_t)n;
    gyz[start + j] = pyz[start + key_slot(k)];
    gorig[start + j] = key_index(k);
    gseg[start + j] = (uint32_t)seg;
  }
}

// Block counting sort of one row bucket by bin, then by input index inside
// each bin: the same order as sort_bucket's (bin, input index) keys, in
// O(n + bins) work. Shared memory: per bin a counter (turned into offsets),
// per cluster its input index, bin and sorted slot. Returns false, before
// writing anything, when a bin holds more than kCountBinMax clusters (the
// per-bin insertion sort would be slow); the caller then uses sort_bucket.
constexpr int kCountBinMax = 64;
__device__ bool count_sort_bucket(const Geo& g, const GridDims& gd, const Bins& B, int seg,
                                  uint32_t start, int n, int tile, const uint32_t* perm,
                                  const float2* pyz, const float* zr, float2* gyz,
                                  uint32_t* gorig, uint32_t* gseg, uint16_t* bs,
                                  uint32_t* smem) {
  __shared__ uint32_t maxc;
  uint32_t* arr = smem;                 // [nb] counts, then bin ends
  uint32_t* si = arr + B.nb;            // [tile] input index, bucket order
  uint32_t* out = si + tile;            // [tile] bucket slot, sorted
  uint16_t* kb = reinterpret_cast<uint16_t*>(out + tile);  // [tile] bin
  int r = seg % g.n_rows;
  int es = seg / g.n_rows;
  int e = es / kNS, s = es % kNS;
  int side = e * 2 + (s >= 18 ? 1 : 0);
  for (int q = threadIdx.x; q < B.nb; q += blockDim.x) arr[q] = 0u;
  if (threadIdx.x == 0) maxc = 0u;
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    uint32_t i = perm[start + j];
    float2 v = pyz[start + j];
    int b = bin_z(zr, side, B.nz, v.y) * B.ny + bin_y(g, gd, r, B.ny, grid_y(g, gd.pads, r, v.x));
    si[j] = i;
    kb[j] = (uint16_t)b;
    atomicAdd(&arr[b], 1u);
  }
  __syncthreads();
  // exclusive scan of the counts: each thread takes a run of consecutive
  // bins, one block scan of the runs' sums (an odd run length keeps the
  // threads' strided reads on distinct shared-memory banks)
  {
    const int per = ((B.nb + (int)blockDim.x - 1) / (int)blockDim.x) | 1;
    const int q0 = (int)threadIdx.x * per;
    uint32_t sum = 0u, mx = 0u;
    for (int k = 0; k < per; ++k) {
      const int q = q0 + k;
      if (q < B.nb) {
        const uint32_t v = arr[q];
        sum += v;
        mx = v > mx ? v : mx;
      }
    }
    if (mx > kCountBinMax) atomicMax(&maxc, mx);
    uint32_t run = block_excl_scan(sum, nullptr);
    for (int k = 0; k < per; ++k) {
      const int q = q0 + k;
      if (q < B.nb) {
        const uint32_t v = arr[q];
        arr[q] = run;
        run += v;
      }
    }
  }
  __syncthreads();
  if (maxc > (uint32_t)kCountBinMax) return false;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    uint32_t pos = atomicAdd(&arr[kb[j]], 1u);
    out[pos] = (uint32_t)j;
  }
  __syncthreads();
  // arr[b] is now the end of bin b; input-index order inside each bin
  for (int b = threadIdx.x; b < B.nb; b += blockDim.x) {
    int lo = b > 0 ? (int)arr[b - 1] : 0, hi = (int)arr[b];
    for (int a = lo + 1; a < hi; ++a) {
      uint32_t v = out[a], iv = si[v];
      int c = a - 1;
      while (c >= lo && si[out[c]] > iv) {
        out[c + 1] = out[c];
        --c;
      }
      out[c + 1] = v;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q <= B.nb; q += blockDim.x)
    bs[q] = (uint16_t)(q > 0 ? arr[q - 1] : 0u);
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    uint32_t jj = out[j];
    gyz[start + j] = pyz[start + jj];
    gorig[start + j] = si[jj];
    gseg[start + j] = (uint32_t)seg;
  }
  return true;
}

// Bucket too large for any tile: copied unsorted, its bins left empty (the
// capacity error is raised).
__device__ void copy_bucket_unsorted(int nb, int seg, uint32_t start, int n,
                                     const uint32_t* perm, const float2* pyz, float2* gyz,
                                     uint32_t* gorig, uint32_t* gseg, uint16_t* bs) {
  for (int b = threadIdx.x; b <= nb; b += blockDim.x) bs[b] = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    gyz[start + j] = pyz[start + j];
    gorig[start + j] = perm[start + j];
    gseg[start + j] = (uint32_t)seg;
  }
}

// Small buckets (<= 256 clusters): one warp each, 8 per block, bitonic sort
// in a 256-entry shared tile per warp. Buckets up to 4096 clusters are listed
// for the 4096-entry block sort, larger ones for the 16384-entry sort.
constexpr int kWarpTile = 256;
__global__ void k_row_sort_warp(Geo g, GridDims gd, int K, const uint32_t* row_start,
                                const uint2* es_dims, const uint32_t* perm, const float2* pyz,
                                const float* zr, float2* gyz, uint32_t* gorig, uint32_t* gseg,
                                uint16_t* bin_start, uint32_t* mid_list, uint32_t* mid_count,
                                uint32_t* big_list, uint32_t* big_count) {
  __shared__ unsigned long long tiles[8][kWarpTile];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int seg = blockIdx.x * 8 + w;
  if (seg >= K) return;
  uint32_t start = row_start[seg];
  int n = (int)(row_start[seg + 1] - start);
  int r = seg % g.n_rows;
  int es = seg / g.n_rows;
  Bins B = es_bins(es_dims, es);
  uint16_t* bs = bin_start + B.base + (size_t)r * (B.nb + 1);
  if (n == 0) {
    for (int q = lane; q <= B.nb; q += 32) bs[q] = 0;
    return;
  }
  if (n > kSortTile) {
    if (lane == 0) big_list[atomicAdd(big_count, 1u)] = (uint32_t)seg;
    return;
  }
  if (n > kWarpTile) {
    if (lane == 0) mid_list[atomicAdd(mid_count, 1u)] = (uint32_t)seg;
    return;
  }
  unsigned long long* keys = tiles[w];
  int e = es / kNS, sc = es % kNS;
  int side = e * 2 + (sc >= 18 ? 1 : 0);
  int P = 1;
  while (P < n) P <<= 1;
  for (int j = lane; j < P; j += 32) {
    unsigned long long k = ~0ull;
    if (j < n) {
      uint32_t i = perm[start + j];
      float2 v = pyz[start + j];
      int b = bin_z(zr, side, B.nz, v.y) * B.ny + bin_y(g, gd, r, B.ny, grid_y(g, gd.pads, r, v.x));
      k = sort_key(b, i, j);
    }
    keys[j] = k;
  }
  __syncwarp();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < P; i += 32) {
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
      __syncwarp();
    }
  }
  for (int j = lane; j < n; j += 32) {
    unsigned long long k = keys[j];
    int b = key_bin(k);
    int bprev = j > 0 ? key_bin(keys[j - 1]) : -1;
    for (int q = bprev + 1; q <= b; ++q) bs[q] = (uint16_t)j;
    if (j == n - 1)
      for (int q = b + 1; q <= B.nb; ++q) bs[q] = (uint16_t)n;
    gyz[start + j] = pyz[start + key_slot(k)];
    gorig[start + j] = key_index(k);
    gseg[start + j] = (uint32_t)seg;
  }
}

// Listed buckets, persistent blocks; 'tile' entries of shared memory.
__global__ void k_row_sort_list(Geo g, GridDims gd, int tile, const uint32_t* row_start,
                                const uint2* es_dims, const uint32_t* perm, const float2* pyz,
                                const float* zr, float2* gyz, uint32_t* gorig, uint32_t* gseg,
                                uint16_t* bin_start, const uint32_t* list, const uint32_t* count,
                                uint32_t* err) {
  extern __shared__ unsigned long long keys[];
  uint32_t* words = reinterpret_cast<uint32_t*>(keys);
  int nl = (int)*count;
  for (int q = blockIdx.x; q < nl; q += gridDim.x) {
    int seg = (int)list[q];
    uint32_t start = row_start[seg];
    int n = (int)(row_start[seg + 1] - start);
    int r = seg % g.n_rows;
    Bins B = es_bins(es_dims, seg / g.n_rows);
    uint16_t* bs = bin_start + B.base + (size_t)r * (B.nb + 1);
    if (n > tile) {
      if (threadIdx.x == 0) atomicOr(err, kErrCapRow);
      copy_bucket_unsorted(B.nb, seg, start, n, perm, pyz, gyz, gorig, gseg, bs);
    } else if (!count_sort_bucket(g, gd, B, seg, start, n, tile, perm, pyz, zr, gyz,
                                  gorig, gseg, bs, words)) {
      sort_bucket(g, gd, B, seg, start, n, perm, pyz, zr, gyz, gorig, gseg, bs, keys);
    }
    __syncthreads();
  }
}

// Range of grid bins [iy0, iy1] x [iz0, iz1] covering a (y, z) box of row seg.
struct Box {
  int iy0, iy1, iz0, iz1;
};
__device__ __forceinline__ Box make_box(const Geo& g, const GridDims& gd, const float* zr,
                                        const Bins& B, int r, int side, float ylo, float yhi,
                                        float zlo, float zhi) {
  Box b;
  b.iy0 = bin_y(g, gd, r, B.ny, ylo);
  b.iy1 = bin_y(g, gd, r, B.ny, yhi);
  b.iz0 = bin_z(zr, side, B.nz, zlo);
  b.iz1 = bin_z(zr, side, B.nz, zhi);
  return b;
}

// ------------------------------------------------------- a4: neighbour finder
// For hit h in row r: the pair (u in row r+1, d in row r-1) inside the slope
// windows whose d lies closest to the straight line through h and u; ties go
// to the lowest pair of input indices. Held to 64 registers: four blocks per
// SM instead of three hide more of the dependent grid loads.
__global__ void __launch_bounds__(256, 4) k_neighbours(Geo g, Params p, GridDims gd, const uint2* es_dims,
                             const uint32_t* nvalid,
                             const float2* __restrict__ gyz, const uint32_t* __restrict__ gorig,
                             const uint32_t* gseg, const uint16_t* bin_start,
                             const uint32_t* row_start, const float* zr, int32_t* up,
                             int32_t* dn) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= (int)*nvalid) return;
  int seg = (int)gseg[h];
  int r = seg % g.n_rows;
  int32_t bu = -1, bd = -1;
  if (r >= 1 && r + 1 < g.n_rows) {
    int es = seg / g.n_rows;
    int e = es / kNS, s = es % kNS;
    int side = e * 2 + (s >= 18 ? 1 : 0);
    float xh = g.rx[r], xu = g.rx[r + 1], xd = g.rx[r - 1];
    float2 hh = gyz[h];
    const RowPad pu = row_pad(g, gd.pads, r + 1), pd = row_pad(g, gd.pads, r - 1);
    float yh = grid_y(g, gd.pads, r, hh.x), zh = hh.y;
    float dxu = xu - xh, dxd = xh - xd;
    float wy_u = dxu * p.nb_ty + p.nb_wy;
    float wy_d = dxd * p.nb_ty + p.nb_wy;
    float wz_u = dxu * p.nb_teta + p.nb_wz;
    float wz_d = dxd * p.nb_teta + p.nb_wz;
    float f = dxd / dxu;
    const float eps = 1.0e-3f;
    Bins BB = es_bins(es_dims, es);
    Box BU = make_box(g, gd, zr, BB, r + 1, side, yh - wy_u - eps, yh + wy_u + eps,
                      zh - wz_u - eps, zh + wz_u + eps);
    Box BD = make_box(g, gd, zr, BB, r - 1, side, yh - wy_d - eps, yh + wy_d + eps,
                      zh - wz_d - eps, zh + wz_d + eps);
    // bin offsets from the bucket starts of rows r + 1 and r - 1
    const uint16_t* bsu = bin_start + BB.base + (size_t)(r + 1) * (BB.nb + 1);
    const uint16_t* bsd = bin_start + BB.base + (size_t)(r - 1) * (BB.nb + 1);
    const uint32_t ru = row_start[seg + 1], rd = row_start[seg - 1];
    // the down candidates inside their windows, once per hit (the windows
    // do not depend on the up candidate); beyond kNd of them the down box
    // is scanned again for each up candidate
    constexpr int kNd = 6;
    float cy[kNd], cz[kNd];
    uint32_t cj[kNd];
    int nd = 0;
    for (int jz = BD.iz0; jz <= BD.iz1; ++jz) {
      uint32_t d0 = rd + bsd[jz * BB.ny + BD.iy0], d1 = rd + bsd[jz * BB.ny + BD.iy1 + 1];
      for (uint32_t d = d0; d < d1; ++d) {
        float2 dd = gyz[d];
        float yd = pd.y(dd.x), zd = dd.y;
        if (!(fabsf(yd - yh) <= wy_d)) continue;
        if (!(fabsf(zd - zh) <= wz_d)) continue;
#pragma unroll
        for (int q = 0; q < kNd; ++q)
          if (q == nd) {
            cy[q] = yd;
            cz[q] = zd;
            cj[q] = d;
          }
        ++nd;
      }
    }
    bool found = false;
    float best = 0.0f;
    // a candidate pair against the best so far: smaller deviation, on an
    // exact tie the lower (up, down) input-index pair (indices loaded then)
    auto consider = [&](uint32_t u, uint32_t d, float D) {
      bool take = !found || D < best;
      if (!take && D == best) {
        uint32_t ou = gorig[u], od = gorig[d], bou = gorig[bu], bod = gorig[bd];
        take = ou < bou || (ou == bou && od < bod);
      }
      if (take) {
        found = true;
        best = D;
        bu = (int32_t)u;
        bd = (int32_t)d;
      }
    };
    for (int iz = BU.iz0; nd > 0 && iz <= BU.iz1; ++iz) {
      uint32_t u0 = ru + bsu[iz * BB.ny + BU.iy0], u1 = ru + bsu[iz * BB.ny + BU.iy1 + 1];
      for (uint32_t u = u0; u < u1; ++u) {
        float2 uu = gyz[u];
        float yu = pu.y(uu.x), zu = uu.y;
        if (!(fabsf(yu - yh) <= wy_u)) continue;
        if (!(fabsf(zu - zh) <= wz_u)) continue;
        float py = yh - (yu - yh) * f;
        float pz = zh - (zu - zh) * f;
        if (nd <= kNd) {
#pragma unroll
          for (int q = 0; q < kNd; ++q) {
            if (q >= nd) break;
            float ey = cy[q] - py, ez = cz[q] - pz;
            float D = ey * ey + ez * ez;
            if (D <= p.nb_dmax) consider(u, cj[q], D);
          }
        } else {
          for (int jz = BD.iz0; jz <= BD.iz1; ++jz) {
            uint32_t d0 = rd + bsd[jz * BB.ny + BD.iy0], d1 = rd + bsd[jz * BB.ny + BD.iy1 + 1];
            for (uint32_t d = d0; d < d1; ++d) {
              float2 dd = gyz[d];
              float yd = pd.y(dd.x), zd = dd.y;
              if (!(fabsf(yd - yh) <= wy_d)) continue;
              if (!(fabsf(zd - zh) <= wz_d)) continue;
              float ey = yd - py, ez = zd - pz;
              float D = ey * ey + ez * ez;
              if (D <= p.nb_dmax) consider(u, d, D);
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
  // each thread takes kPer consecutive entries per pass: a serial sum of
  // its entries, one block scan of the sums, then its entries' offsets
  constexpr int kPer = 8;
  const int span = blockDim.x * kPer;
  for (int base = 0; base < nblk; base += span) {
    const int i0 = base + threadIdx.x * kPer;
    uint32_t va[kPer], vb[kPer];
    uint32_t sa = 0u, sb = 0u;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      int i = i0 + q;
      va[q] = i < nblk ? a[i] : 0u;
      vb[q] = (b && i < nblk) ? b[i] : 0u;
      sa += va[q];
      sb += vb[q];
    }
    uint32_t ta;
    uint32_t ea = block_excl_scan(sa, &ta);
    uint32_t tb = 0u, eb = 0u;
    if (b) eb = block_excl_scan(sb, &tb);
    uint32_t ra = carry_a + ea, rb = carry_b + eb;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      int i = i0 + q;
      if (i < nblk) {
        off_a[i] = ra;
        if (b) off_b[i] = rb;
      }
      ra += va[q];
      rb += vb[q];
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

// Also the last hit of each start hit's seed: the first seed_max_hits hits
// of its chain of cleaned links.
__global__ void k_write_starts(const uint32_t* nvalid, const int32_t* upc, const int32_t* dnc,
                               const uint32_t* blk_off, uint32_t cap, int seed_max_hits,
                               uint32_t* starts, uint32_t* seed_end) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  int n = (int)*nvalid;
  uint32_t st = (h < n && is_start(upc, dnc, h)) ? 1u : 0u;
  uint32_t ex = block_excl_scan(st, nullptr);
  if (st) {
    uint32_t pos = blk_off[blockIdx.x] + ex;
    if (pos < cap) {
      starts[pos] = (uint32_t)h;
      int hl = h, nseed = 1;
      while (upc[hl] >= 0 && nseed < seed_max_hits) {
        hl = upc[hl];
        ++nseed;
      }
      seed_end[pos] = (uint32_t)hl;
    }
  }
}

// ------------------------------------------------------ a7: tracklets
struct Grid {
  const float2* gyz;  // (y or pad position, seeding z)
  const uint32_t* gorig;
  const uint16_t* bin_start;  // per row, from the row's bucket start
  const uint32_t* row_start;  // bucket starts
  const float* zr;
  int32_t pads;       // gyz.x holds pad positions
};

// Calibrated position of a candidate during following (Sec. 4): the seeding z
// shifted by the offset of the estimated collision time, then the space-point
// correction at the shifted position.
__device__ __forceinline__ void calibrate_follow(const Geo& g, const Cal& c, bool spl_on, int sec,
                                                 int r, float y, float zs, float shift,
                                                 float& yc, float& zc) {
  float za = zs + shift;
  if (spl_on) {
    float d[2];
    spline_eval(g, c, sec, g.rx[r], y, fabsf(za), d);
    yc = y + d[0];
    zc = za + d[1];
  } else {
    yc = y;
    zc = za;
  }
}

enum : int { kOut = 2, kIn = 3, kDone = 4 };

// The measurement of one following step: the nearest cluster of row r
// (calibrated frame) by the normalised distance inside the pick-up cut, ties
// to the lowest input index. Returns the grid position or -1, and the
// calibrated coordinates. The candidate loop is flattened over up to four z
// rows of bins.
__device__ int step_measurement(const Geo& g, const Cal& c, const Params& p, const GridDims& gd,
                                const Bins& BB, const Grid& G, int ev, int sec, int r,
                                const float st[5], const float C[15], float shift, bool spl_on,
                                float dymax, float dzmax, float& ycb, float& zcb) {
  int side = ev * 2 + (sec >= 18 ? 1 : 0);
  float sig2 = p.sigma * p.sigma;
  float vy = C[0] + sig2, vz = C[2] + sig2;
  float ivy = Fast::rcp(vy), ivz = Fast::rcp(vz);
  // window half-widths bound the search box only (the cut below decides):
  // a fast square root is enough
  float qy = p.chi2_pick * vy, qz = p.chi2_pick * vz;
  float wy = qy * rsqrtf(qy), wz = qz * rsqrtf(qz);
  float eps = 0.01f + 1.0e-6f * fabsf(shift);
  float yp = st[0], zp = st[1] - shift;
  Box B = make_box(g, gd, G.zr, BB, r, side, yp - wy - dymax - eps, yp + wy + dymax + eps,
                   zp - wz - dzmax - eps, zp + wz + dzmax + eps);
  const uint16_t* __restrict__ bs = G.bin_start + BB.base + (size_t)r * (BB.nb + 1);
  const uint32_t rb0 = __ldg(G.row_start + (size_t)(ev * kNS + sec) * g.n_rows + r);
  const RowPad rp = row_pad(g, G.pads, r);
  int best = -1;
  float bd = 0.0f;
  for (int izb = B.iz0; izb <= B.iz1; izb += 4) {
    // bin offsets of up to four z rows of the box, loaded together
    uint32_t lo[4], hi[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int iz = izb + q;
      bool in = iz <= B.iz1;
      lo[q] = in ? rb0 + __ldg(bs + iz * BB.ny + B.iy0) : 0u;
      hi[q] = in ? rb0 + __ldg(bs + iz * BB.ny + B.iy1 + 1) : 0u;
    }
    const uint32_t c0 = hi[0] - lo[0], c1 = c0 + (hi[1] - lo[1]), c2 = c1 + (hi[2] - lo[2]);
    const uint32_t total = c2 + (hi[3] - lo[3]);
    for (uint32_t k = 0; k < total; ++k) {
      uint32_t j = k < c0 ? lo[0] + k
                 : k < c1 ? lo[1] + (k - c0)
                 : k < c2 ? lo[2] + (k - c1)
                          : lo[3] + (k - c2);
      float2 yz = __ldg(G.gyz + j);
      float yc, zc;
      calibrate_follow(g, c, spl_on, sec, r, rp.y(yz.x), yz.y, shift, yc, zc);
      float ry = yc - st[0];
      float rz = zc - st[1];
      float d2 = Fast::fma(rz * rz, ivz, (ry * ry) * ivy);
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
  return best;
}

// Tracklet constructor, part 1: the seed of every start hit, one thread
// each. The chain hits h0 .. hl are fitted in seeding coordinates; in
// continuous readout the closest approach to the beam line gives the
// collision time (Sec. 4) and the seed is fitted again in calibrated
// coordinates (also with a distortion map in event mode). Each hit is one
// transport and one update in the arithmetic of the following, so a seed
// gets the same bits as if the following kernel had fitted it. Writes the
// seed state at the seed's last hit, the collision time, the final outputs of
// seeds that fail, and the number of rows the seed's helix can still cross
// inside the sector (outward to its exit, then inward to row 0), counted
// into the histogram that orders the following longest first.
constexpr int kSeedStride = 24;   // floats per seed: p[5], C[15], x, ok flag, padding
constexpr int kLenBuckets = 512;  // predicted steps, capped
__global__ void k_tl_seed(Geo g, Cal c, Params p, Grid G, int mode, const int32_t* upc,
                          const uint32_t* gseg, const uint32_t* starts,
                          const uint32_t* seed_end, const uint32_t* cnt, float* seed_st,
                          uint32_t* pred, uint32_t* hist, int32_t* nh_out, double* that_out,
                          uint32_t* range_out) {
  const int ntl = (int)cnt[kCntStart];
  const float sig2 = p.sigma * p.sigma;
  const bool spl_on = c.spl_bound[2] > 0.0f;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntl; t += gridDim.x * blockDim.x) {
    const int h0 = (int)starts[t], hl = (int)seed_end[t];
    const int seg0 = (int)gseg[h0];
    const int rl = (int)gseg[hl] % g.n_rows, r0 = seg0 % g.n_rows;
    const int sec = (seg0 / g.n_rows) % kNS;
    float2 yz0 = G.gyz[h0], yzl = G.gyz[hl];
    yz0.x = grid_y(g, G.pads, r0, yz0.x);
    yzl.x = grid_y(g, G.pads, rl, yzl.x);
    float st[5], C[15], x;
    seed_two_points(st, C, x, p.c0t, g.rx[r0], yz0.x, yz0.y, g.rx[rl], yzl.x, yzl.y);
    double that = 0.0;
    float shift = 0.0f;
    bool ok = true;
    const bool second = mode == 1 || spl_on;
    for (int pass = 0; ok && pass < (second ? 2 : 1); ++pass) {
      if (pass == 1) {
        if (mode == 1) {
          float zd = dca_z(g.kB, st, x);
          double sg = sec < 18 ? 1.0 : -1.0;
          that = c.tf_start - (sg * (double)zd) / c.vdrift;
          shift = (float)(sg * c.vdrift * (that - c.tf_start));
        }
        float y0, z0, y1, z1;
        calibrate_follow(g, c, spl_on, sec, r0, yz0.x, yz0.y, shift, y0, z0);
        calibrate_follow(g, c, spl_on, sec, rl, yzl.x, yzl.y, shift, y1, z1);
        seed_two_points(st, C, x, p.c0t, g.rx[r0], y0, z0, g.rx[rl], y1, z1);
      }
      int h = h0, r = r0;
      while (true) {
        if (!propagate<Fast>(g.kB, p.s_max, st, C, x, g.rx[r])) {
          ok = false;
          break;
        }
        float2 yz = __ldg(G.gyz + h);
        yz.x = grid_y(g, G.pads, r, yz.x);
        float my = yz.x, mz = yz.y;
        if (pass == 1) calibrate_follow(g, c, spl_on, sec, r, yz.x, yz.y, shift, my, mz);
        apply_update<Fast>(st, C, innovation<Fast>(st, C, my, mz, sig2, sig2));
        if (h == hl) break;
        h = upc[h];
        ++r;
      }
    }
    uint32_t len = 0;
    if (!ok) {
      nh_out[t] = -1;
      that_out[t] = 0.0;
      range_out[t] = 1u;
      seed_st[(size_t)t * kSeedStride + 21] = 0.0f;
    } else {
      float* o = seed_st + (size_t)t * kSeedStride;
#pragma unroll
      for (int i = 0; i < 5; ++i) o[i] = st[i];
#pragma unroll
      for (int i = 0; i < 15; ++i) o[5 + i] = C[i];
      o[20] = x;
      o[21] = 1.0f;
      that_out[t] = that;
      // rows the seed's helix crosses inside the sector with |sin(phi)| below
      // its limit: outward from the seed end, then inward from there
      const float kap = g.kB * st[4];
      const float c1 = Fast::sqrt(Fast::fma(-st[2], st[2], 1.0f));
      auto inside = [&](int rr) {
        float xr = g.rx[rr], dx = xr - x;
        float s2 = Fast::fma(-kap, dx, st[2]);
        if (!(fabsf(s2) < p.s_max)) return false;
        float c2 = Fast::sqrt(Fast::fma(-s2, s2, 1.0f));
        float yr = Fast::fma(dx, Fast::div(st[2] + s2, c1 + c2), st[0]);
        return fabsf(yr) <= Fast::fma(xr, g.tan_half, 2.0f);
      };
      // (in steps of four rows: an ordering key needs no finer count)
      int rend = rl;
      while (rend + 4 < g.n_rows && inside(rend + 4)) rend += 4;
      int rin = rend;
      while (rin - 4 >= 0 && inside(rin - 4)) rin -= 4;
      len = (uint32_t)((rend - rl) + (rend - rin) + 2);
    }
    if (len >= (uint32_t)kLenBuckets) len = kLenBuckets - 1;
    pred[t] = len;
    warp_counter_add1(hist, kLenBuckets - 1 - len);
  }
}

// Following order, longest predicted first: bucket offsets of the histogram
// (one block), then each tracklet's place (its position inside a bucket is
// arbitrary; every tracklet's result is independent of the order).
__global__ void k_tl_order_scan(uint32_t* hist) {
  __shared__ uint32_t tot;
  uint32_t v = threadIdx.x < kLenBuckets ? hist[threadIdx.x] : 0u;
  uint32_t e = block_excl_scan(v, &tot);
  if (threadIdx.x < kLenBuckets) hist[threadIdx.x] = e;
}
__global__ void k_tl_order(const uint32_t* cnt, const uint32_t* pred, uint32_t* cursor,
                           uint32_t* order) {
  const int ntl = (int)cnt[kCntStart];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntl; t += gridDim.x * blockDim.x)
    order[warp_counter_add1(cursor, kLenBuckets - 1 - pred[t])] = (uint32_t)t;
}

// Tracklet constructor, part 2: the following, as a persistent step machine.
// Every iteration of the loop transports the state to the next row and
// updates it with the picked cluster, so the threads of a warp execute the
// same instructions whatever phase their tracklet is in; a thread whose
// tracklet ends takes the next one from a queue in the order above, so the
// lanes of a warp stay busy while work is left and the long tracklets are not
// the last to start.
//   phase 2: outward following from the seed end
//   phase 3: inward following from the outermost pick down to row 0
// kCap: the launch bound asks for 640 resident threads per SM (blocks of 64
// or 128), which holds the kernel to 96 registers per thread (no spills, the
// best state being in shared memory): 20 warps per SM instead of 16, for the
// workloads with more tracklets than resident threads. Without it (a minimum
// of 0 blocks: no occupancy target) the compiler takes 128.
template <int BS, bool kCap>
__global__ void __launch_bounds__(BS, kCap ? 640 / BS : 0) k_tracklets(Geo g, Cal c, Params p, GridDims gd, Grid G,
                                                  const uint2* es_dims, int mode,
                                                  const uint32_t* gseg, const uint32_t* starts,
                                                  const uint32_t* seed_end, const uint32_t* cnt,
                                                  const float* seed_st, const uint32_t* order,
                                                  int32_t* nh_out, int32_t* hits,
                                                  uint32_t* range_out, const double* that_in,
                                                  uint32_t* queue) {
  const int ntl = (int)cnt[kCntStart];
  const float sig2 = p.sigma * p.sigma;
  const bool spl_on = c.spl_bound[2] > 0.0f;
  const float dymax = spl_on ? c.spl_bound[0] : 0.0f;
  const float dzmax = spl_on ? c.spl_bound[1] : 0.0f;
  // the state at the outermost pick (the inward pass starts from it), one
  // column per thread in shared memory: it is written on every outward pick
  // and read once, and keeping it out of the registers lets more warps stay
  // resident
  __shared__ float s_best[21][BS];
  float* bst = &s_best[0][threadIdx.x];  // element i at bst[i * BS]
  int t = -1;
  int32_t* H = nullptr;
  int ev = 0, sec = 0;
  Bins BB{0u, 1, 1, 1};
  float st[5], C[15], x = 0.0f;
  float shift = 0.0f;
  int phase = kDone, r = 0, rlast = 0, miss = 0, nh = 0;
  int rlo = 0;
  while (true) {
    if (phase == kDone) {
      if (t >= 0) {
        // the current tracklet: hit count and the rows [rlo, rlast] its
        // inward pass visited (hits[] holds those rows); its collision time
        // was written with the seed
        nh_out[t] = nh;
        range_out[t] = (uint32_t)rlo | ((uint32_t)rlast << 16);
      }
      const int q = (int)atomicAdd(queue, 1u);
      if (q >= ntl) break;
      t = (int)order[q];
      const int h0 = (int)starts[t];
      const int seg0 = (int)gseg[h0];
      const int rl = (int)gseg[seed_end[t]] % g.n_rows;
      const float* so = seed_st + (size_t)t * kSeedStride;
      if (so[21] == 0.0f) {
        // a failed seed: its outputs are written already
        t = -1;
        continue;
      }
      const double that = that_in[t];
      H = hits + (size_t)t * g.n_rows;
      int es = seg0 / g.n_rows;
      ev = es / kNS;
      sec = es % kNS;
      BB = es_bins(es_dims, es);
#pragma unroll
      for (int i = 0; i < 5; ++i) st[i] = so[i];
#pragma unroll
      for (int i = 0; i < 15; ++i) C[i] = so[5 + i];
      x = so[20];
      shift = 0.0f;
      if (mode == 1) {
        double sg = sec < 18 ? 1.0 : -1.0;
        shift = (float)(sg * c.vdrift * (that - c.tf_start));
      }
      rlast = rl;
      rlo = rl + 1;
      miss = 0;
      nh = 0;
      phase = kOut;
      r = rl + 1;
      if (r >= g.n_rows) {
        // nothing outward: the inward pass starts from the seed
#pragma unroll
        for (int i = 0; i < 15; ++i) C[i] = C[i] * p.inward_cov_scale;
        r = rlast;
        phase = kIn;
      } else {
#pragma unroll
        for (int i = 0; i < 5; ++i) bst[i * BS] = st[i];
#pragma unroll
        for (int i = 0; i < 15; ++i) bst[(5 + i) * BS] = C[i];
        bst[20 * BS] = x;
      }
    }
    bool ok = propagate<Fast>(g.kB, p.s_max, st, C, x, g.rx[r]);
    bool have = false;
    float my = 0.0f, mz = 0.0f;
    int j = -1;
    if (ok) {
      j = step_measurement(g, c, p, gd, BB, G, ev, sec, r, st, C, shift, spl_on, dymax, dzmax,
                           my, mz);
      have = j >= 0;
      if (have) apply_update<Fast>(st, C, innovation<Fast>(st, C, my, mz, sig2, sig2));
    }
    bool start_in = false;
    if (phase == kOut) {
      if (!ok) {
        start_in = true;
      } else {
        if (have) {
#pragma unroll
          for (int i = 0; i < 5; ++i) bst[i * BS] = st[i];
#pragma unroll
          for (int i = 0; i < 15; ++i) bst[(5 + i) * BS] = C[i];
          bst[20 * BS] = x;
          rlast = r;
          miss = 0;
        } else if (++miss >= p.max_miss) {
          start_in = true;
        }
        if (!start_in && ++r >= g.n_rows) start_in = true;
      }
    } else {  // kIn
      if (!ok) {
        phase = kDone;
      } else {
        H[r] = have ? j : -1;
        rlo = r;
        if (have) {
          ++nh;
          miss = 0;
        } else if (++miss >= p.max_miss) {
          phase = kDone;
        }
        if (phase != kDone && --r < 0) phase = kDone;
      }
    }
    if (start_in) {
#pragma unroll
      for (int i = 0; i < 5; ++i) st[i] = bst[i * BS];
#pragma unroll
      for (int i = 0; i < 15; ++i) C[i] = bst[(5 + i) * BS] * p.inward_cov_scale;
      x = bst[20 * BS];
      r = rlast;
      rlo = rlast + 1;
      miss = 0;
      phase = kIn;
    }
  }
}

// --------------------------------------------------- a8: tracklet selection
// Every cluster keeps the largest weight (hit count, then the lowest start
// hit) of the tracklets of at least min_track_hits hits that picked it
// (Sec. 3, tracklet selection). One warp per tracklet.
__global__ void k_tl_weight(int n_rows, int min_track_hits, const uint32_t* cnt,
                            const int32_t* nh, const int32_t* hits, const uint32_t* range,
                            const uint32_t* starts, const uint32_t* gorig,
                            unsigned long long* weight) {
  const int ntl = (int)cnt[kCntStart];
  const int lane = threadIdx.x & 31;
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < ntl; t += nw) {
    int n = nh[t];
    if (n < min_track_hits) continue;
    unsigned long long w = ((unsigned long long)(uint32_t)n << 32) |
                           (unsigned long long)(0xffffffffu - gorig[starts[t]]);
    uint32_t rg = range[t];
    int rlo = (int)(rg & 0xffffu), rhi = (int)(rg >> 16);
    const int32_t* H = hits + (size_t)t * n_rows;
    for (int r = rlo + lane; r <= rhi; r += 32) {
      int j = H[r];
      if (j >= 0) atomicMax(&weight[j], w);
    }
  }
}

// One warp per tracklet of at least min_track_hits hits: the lanes test 32
// rows at a time for the hits whose cluster weight is the tracklet's own;
// the track is kept if it keeps min_track_hits of them with no gap above
// max_gap rows.
__global__ void k_select_count(int n_rows, const Params p, const uint32_t* cnt,
                               const int32_t* nh, const int32_t* hits, const uint32_t* range,
                               const uint32_t* starts, const uint32_t* gorig,
                               const unsigned long long* weight, uint32_t* nkeep) {
  const int ntl = (int)cnt[kCntStart];
  const int lane = threadIdx.x & 31;
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < ntl; t += nw) {
    uint32_t kept = 0;
    int n = nh[t];
    if (n >= p.min_track_hits) {
      unsigned long long w = ((unsigned long long)(uint32_t)n << 32) |
                             (unsigned long long)(0xffffffffu - gorig[starts[t]]);
      const int32_t* H = hits + (size_t)t * n_rows;
      uint32_t rg = range[t];
      int rlo = (int)(rg & 0xffffu), rhi = (int)(rg >> 16);
      int lastr = -1, maxgap = 0, k = 0;
      for (int r0 = rlo; r0 <= rhi; r0 += 32) {
        int r = r0 + lane;
        bool own = false;
        if (r <= rhi) {
          int j = H[r];
          own = j >= 0 && weight[j] == w;
        }
        unsigned m = __ballot_sync(0xffffffffu, own);
        k += __popc(m);
        // gap before each kept row: to the previous kept lane of this chunk,
        // else to the last kept row of the chunks before
        int gap = 0;
        if (own) {
          unsigned below = m & ((1u << lane) - 1u);
          int prev = below ? r0 + 31 - __clz(below) : lastr;
          if (prev >= 0) gap = r - prev - 1;
        }
        maxgap = max(maxgap, __reduce_max_sync(0xffffffffu, gap));
        if (m) lastr = r0 + 31 - __clz(m);
      }
      if (k >= p.min_track_hits && maxgap <= p.max_gap) kept = (uint32_t)k;
    }
    if (lane == 0) nkeep[t] = kept;
  }
}

// Per block of 256 tracklets: counts of emitted tracks and kept clusters for
// the ordered compaction; the start hit's (event, sector, row) and input
// index for the order of emission, and the list of large groups.
__global__ void k_select_sum(const uint32_t* cnt, const uint32_t* nkeep, const uint32_t* starts,
                             const uint32_t* gorig, const uint32_t* gseg, uint32_t* tkey,
                             uint32_t* tseg, uint32_t* grp_list, uint32_t* grp_count,
                             uint32_t cap_grp, uint32_t* blk_tr, uint32_t* blk_cl) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int ntl = (int)cnt[kCntStart];
  uint32_t kept = 0;
  if (t < ntl) {
    kept = nkeep[t];
    uint32_t h0 = starts[t];
    uint32_t seg = gseg[h0];
    tkey[t] = gorig[h0];
    tseg[t] = seg;
    if ((t == 0 || gseg[starts[t - 1]] != seg) && t + kSmallGroup < ntl &&
        gseg[starts[t + kSmallGroup]] == seg) {
      uint32_t q = atomicAdd(grp_count, 1u);
      if (q < cap_grp) grp_list[q] = (uint32_t)t;
    }
  }
  uint32_t tot_tr, tot_cl;
  block_excl_scan(kept ? 1u : 0u, &tot_tr);
  block_excl_scan(kept, &tot_cl);
  if (threadIdx.x == 0) {
    blk_tr[blockIdx.x] = tot_tr;
    blk_cl[blockIdx.x] = tot_cl;
  }
}

// Emission order inside the groups of more than kSmallGroup tracklets: one
// block per group sorts the emitted tracklets by start-hit input index
// (bitonic sort in shared memory) and stores, per tracklet, how far its track
// moves from the tracklet order: delta_id (tracks) and delta_o (clusters).
// Groups of more than kRankTile emitted tracklets are marked (kUnranked) and
// left to the scan in k_select_write.
constexpr uint32_t kUnranked = 0x80000000u;
constexpr size_t kRankSmem = (size_t)kRankTile * (sizeof(unsigned long long) + 3 * sizeof(uint32_t));
__global__ void __launch_bounds__(1024) k_group_rank(const uint32_t* cnt, const uint32_t* tkey,
                                                     const uint32_t* tseg, const uint32_t* nkeep,
                                                     const uint32_t* grp_list,
                                                     const uint32_t* grp_count, uint32_t cap_grp,
                                                     int32_t* delta_id, int32_t* delta_o) {
  extern __shared__ unsigned long long skey[];           // [kRankTile]
  uint32_t* sidx = reinterpret_cast<uint32_t*>(skey + kRankTile);  // local index
  uint32_t* skept = sidx + kRankTile;                     // kept, index order
  uint32_t* spre = skept + kRankTile;                     // kept prefix, index order
  __shared__ uint32_t carry_n, carry_k;
  const int ntl = (int)cnt[kCntStart];
  const uint32_t ng = min(*grp_count, cap_grp);
  for (uint32_t gi = blockIdx.x; gi < ng; gi += gridDim.x) {
    const int head = (int)grp_list[gi];
    const uint32_t seg = tseg[head];
    // end of the group: tseg is non-decreasing
    int lo = head, hi = ntl;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (tseg[mid] == seg) lo = mid;
      else hi = mid;
    }
    const int m = hi - head;
    // emitted tracklets in index order, with their cluster-count prefix
    if (threadIdx.x == 0) carry_n = carry_k = 0u;
    __syncthreads();
    for (int b0 = 0; b0 < m; b0 += blockDim.x) {
      int u = b0 + threadIdx.x;
      uint32_t k = u < m ? nkeep[head + u] : 0u;
      uint32_t tn, tk;
      uint32_t en = block_excl_scan(k ? 1u : 0u, &tn);
      uint32_t ek = block_excl_scan(k, &tk);
      uint32_t pos = carry_n + en;
      if (k && pos < (uint32_t)kRankTile) {
        skey[pos] = ((unsigned long long)tkey[head + u] << 32) | pos;
        sidx[pos] = (uint32_t)u;
        skept[pos] = k;
        spre[pos] = carry_k + ek;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        carry_n += tn;
        carry_k += tk;
      }
      __syncthreads();
    }
    const uint32_t M = carry_n;
    if (M > (uint32_t)kRankTile) {
      for (int u = threadIdx.x; u < m; u += blockDim.x)
        if (nkeep[head + u]) delta_id[head + u] = (int32_t)kUnranked;
      __syncthreads();
      continue;
    }
    int P = 1;
    while (P < (int)M) P <<= 1;
    for (int j = (int)M + threadIdx.x; j < P; j += blockDim.x) skey[j] = ~0ull;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
          int ixj = i ^ j;
          if (ixj > i) {
            unsigned long long a = skey[i], b = skey[ixj];
            bool up = (i & k) == 0;
            if ((a > b) == up) {
              skey[i] = b;
              skey[ixj] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    // sorted rank r: clusters of the tracks ranked before it
    if (threadIdx.x == 0) carry_k = 0u;
    __syncthreads();
    for (int r0 = 0; r0 < (int)M; r0 += blockDim.x) {
      int r = r0 + threadIdx.x;
      uint32_t pos = r < (int)M ? (uint32_t)(skey[r] & 0xffffffffu) : 0u;
      uint32_t k = r < (int)M ? skept[pos] : 0u;
      uint32_t tk;
      uint32_t ek = block_excl_scan(k, &tk);
      if (r < (int)M) {
        int u = head + (int)sidx[pos];
        delta_id[u] = r - (int32_t)pos;
        delta_o[u] = (int32_t)(carry_k + ek) - (int32_t)spre[pos];
      }
      __syncthreads();
      if (threadIdx.x == 0) carry_k += tk;
      __syncthreads();
    }
  }
}

// Tracks are emitted in a canonical order: by (event, sector, row) of the
// start hit, then by its input index -- not by its position in the search
// grid, which depends on the grid's tuning. Tracklets of one (event, sector,
// row) are contiguous in the start list (it follows the row buckets), so a
// track's place is its tracklet's place corrected inside that group.
__global__ void k_select_write(int n_rows, const uint32_t* cnt, const int32_t* hits,
                               const uint32_t* range, const uint32_t* starts,
                               const uint32_t* tkey, const uint32_t* tseg,
                               const int32_t* delta_id, const int32_t* delta_o, const double* that,
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
  uint32_t id = off_tr[blockIdx.x] + ex_tr;
  uint32_t o = off_cl[blockIdx.x] + ex_cl;
  if (emit) {
    const int ntl = (int)cnt[kCntStart];
    const uint32_t seg = tseg[t];
    // size of the group, counted up to kSmallGroup + 1
    int nb = 0, na = 0;
    while (nb + na < kSmallGroup && t - nb - 1 >= 0 && tseg[t - nb - 1] == seg) ++nb;
    while (nb + na < kSmallGroup && t + na + 1 < ntl && tseg[t + na + 1] == seg) ++na;
    bool small = nb + na < kSmallGroup;
    if (!small && delta_id[t] != (int32_t)kUnranked) {
      id = (uint32_t)((int32_t)id + delta_id[t]);
      o = (uint32_t)((int32_t)o + delta_o[t]);
    } else {
      const uint32_t me = tkey[t];
      uint32_t n_before = 0, k_before = 0, n_less = 0, k_less = 0;
      for (int u = t - 1; u >= 0 && tseg[u] == seg; --u) {
        uint32_t ku = nkeep[u];
        if (!ku) continue;
        ++n_before;
        k_before += ku;
        if (tkey[u] < me) {
          ++n_less;
          k_less += ku;
        }
      }
      for (int u = t + 1; u < ntl && tseg[u] == seg; ++u) {
        uint32_t ku = nkeep[u];
        if (ku && tkey[u] < me) {
          ++n_less;
          k_less += ku;
        }
      }
      id = id - n_before + n_less;
      o = o - k_before + k_less;
    }
  }
  bool ok = emit && (int64_t)id < cap_tr && (int64_t)(o + kept) <= cap_asg;
  unsigned long long w = 0ull;
  uint32_t rg = 0u;
  if (ok) {
    uint32_t h0 = gorig[starts[t]];
    w = ((unsigned long long)(uint32_t)nh[t] << 32) | (unsigned long long)(0xffffffffu - h0);
    track_start[id] = o;
    t_coll[id] = that[t];
    start_hit[id] = h0;
    rg = range[t];
  }
  // the kept clusters in row order, the warp's tracks one after the other
  // with the lanes on 32 rows at a time
  const int lane = threadIdx.x & 31;
  unsigned todo = __ballot_sync(0xffffffffu, ok);
  while (todo) {
    int src = __ffs(todo) - 1;
    todo &= todo - 1;
    int ts = __shfl_sync(0xffffffffu, t, src);
    uint32_t tid = __shfl_sync(0xffffffffu, id, src);
    uint32_t oo = __shfl_sync(0xffffffffu, o, src);
    uint32_t rr = __shfl_sync(0xffffffffu, rg, src);
    unsigned long long ww = __shfl_sync(0xffffffffu, w, src);
    int rlo = (int)(rr & 0xffffu), rhi = (int)(rr >> 16);
    const int32_t* H = hits + (size_t)ts * n_rows;
    for (int r0 = rlo; r0 <= rhi; r0 += 32) {
      int r = r0 + lane;
      int j = -1;
      if (r <= rhi) {
        j = H[r];
        if (j >= 0 && weight[j] != ww) j = -1;
      }
      unsigned m = __ballot_sync(0xffffffffu, j >= 0);
      if (j >= 0) {
        uint32_t pos = oo + __popc(m & ((1u << lane) - 1u));
        cluster_idx[pos] = gorig[j];
        asg_track[pos] = tid;
      }
      oo += __popc(m);
    }
  }
}

__global__ void k_track_end(const uint32_t* cnt, uint32_t* track_start) {
  track_start[cnt[kCntTracks]] = cnt[kCntAssigned];
}

// ---------------------------------------------------- a9: calibration
// (held to 32 registers: eight blocks per SM for its gathers)
__global__ void __launch_bounds__(256, 8) k_calib(Geo g, Cal c, ClIn cl, const uint32_t* cnt, const uint32_t* cluster_idx,
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
  calibrate(g, c, spl_on, cl.mode, s, r, cluster_y(g, cl, i), cl.mode == 0 ? cl.z[i] : 0.0f,
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
                                   const uint32_t* range, uint32_t* o_start, int32_t* o_nh,
                                   double* o_that, int32_t* o_hits) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int)cnt[kCntStart] || t >= n_cap) return;
  if (o_start) o_start[t] = gorig[starts[t]];
  if (o_nh) o_nh[t] = nh[t];
  if (o_that) o_that[t] = that[t];
  if (o_hits) {
    uint32_t rg = range[t];
    int rlo = (int)(rg & 0xffffu), rhi = (int)(rg >> 16);
    for (int r = 0; r < n_rows; ++r) {
      int j = (r >= rlo && r <= rhi) ? hits[(size_t)t * n_rows + r] : -1;
      o_hits[(size_t)t * n_rows + r] = j >= 0 ? (int32_t)gorig[j] : -1;
    }
  }
}

inline int nblk(int64_t n, int b) { return (int)((n + b - 1) / b); }

// Shared memory of a block sort of up to `tile` clusters: the larger of the
// bitonic keys and the counting sort's arrays.
inline size_t sort_smem(int tile, int nb_max) {
  size_t bitonic = (size_t)tile * sizeof(unsigned long long);
  size_t counting = (size_t)nb_max * 4 + (size_t)tile * (4 + 4 + 2);
  return bitonic > counting ? bitonic : counting;
}

}  // namespace

// ======================================================================
// launchers
// ======================================================================
void launch_load(Prof* P, const Geo& g, const Cal& c, const ClIn& cl, const GridDims& gd, int K,
                 FindBuf& b, uint32_t* err, cudaStream_t s) {
  int init_n = K > cl.n_events * 2 ? K : cl.n_events * 2;
  TPC_LAUNCH(P, "k_init_load", s,
             k_init_load<<<nblk(init_n, kB256), kB256, 0, s>>>(K, cl.n_events, b.cnt, b.fill,
                                                               b.zmm));
  if (cl.n > 0)
    TPC_LAUNCH(P, "k_hist", s,
               k_hist<<<min(nblk(cl.n, kB256), 8 * 148), kB256, 0, s>>>(g, c, cl, b.cnt, b.zs_in,
                                                                        b.zmm, err));
  const int nblk_rows = K > kRowScanSplit ? nblk(K, kRowScanBlock) : 0;
  if (nblk_rows > 0)
    TPC_LAUNCH(P, "k_rows_local", s,
               k_rows_local<<<nblk_rows, kRowScanBlock, 0, s>>>(K, b.cnt, b.row_start,
                                                                b.row_blk));
  TPC_LAUNCH(P, "k_scan_rows", s,
             k_scan_rows<<<1, 1024, 0, s>>>(g, K, cl.n_events, gd, b.cnt, b.row_start, nblk_rows,
                                            b.row_blk, b.zmm, b.zr, b.es_dims, b.n_bins));
  if (nblk_rows > 0)
    TPC_LAUNCH(P, "k_rows_add", s,
               k_rows_add<<<nblk_rows, kRowScanBlock, 0, s>>>(K, b.row_blk, b.row_start));
  if (cl.n > 0)
    TPC_LAUNCH(P, "k_scatter", s,
               k_scatter<<<nblk(cl.n, kB256), kB256, 0, s>>>(g, cl, b.row_start, b.zs_in, b.fill,
                                                             b.perm, b.pyz));
  cudaMemsetAsync(b.list_counts, 0, 2 * sizeof(uint32_t), s);
  TPC_LAUNCH(P, "k_row_sort_warp", s,
             k_row_sort_warp<<<nblk(K, 8), 256, 0, s>>>(g, gd, K, b.row_start, b.es_dims,
                                                        b.perm, b.pyz, b.zr, b.gyz, b.gorig,
                                                        b.gseg, b.bin_start, b.mid_list,
                                                        b.list_counts, b.big_list,
                                                        b.list_counts + 1));
  size_t smem = sort_smem(kSortTile, gd.nb_max);
  TPC_LAUNCH(P, "k_row_sort_mid", s,
             k_row_sort_list<<<4 * 148, 512, smem, s>>>(g, gd, kSortTile, b.row_start,
                                                        b.es_dims, b.perm, b.pyz, b.zr, b.gyz,
                                                        b.gorig, b.gseg, b.bin_start, b.mid_list,
                                                        b.list_counts, err));
  size_t smem_big = sort_smem(kSortTileBig, gd.nb_max);
  TPC_LAUNCH(P, "k_row_sort_big", s,
             k_row_sort_list<<<148, 1024, smem_big, s>>>(g, gd, kSortTileBig, b.row_start,
                                                         b.es_dims, b.perm, b.pyz, b.zr, b.gyz,
                                                         b.gorig, b.gseg, b.bin_start,
                                                         b.big_list, b.list_counts + 1, err));
}

void setup_find_kernels() {
  cudaFuncSetAttribute(k_group_rank, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRankSmem);
  cudaFuncSetAttribute(k_row_sort_list, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sort_smem(kSortTileBig, kGridBinsMax));
}

template <bool kCap>
cudaError_t tracklet_occupancy(int* per, int block) {
  return block == 64    ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k_tracklets<64, kCap>, 64, 0)
         : block == 256 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k_tracklets<256, kCap>, 256, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k_tracklets<128, kCap>, 128, 0);
}

int tracklet_blocks_per_sm(int block, int regs) {
  int per = 0;
  cudaError_t e = regs == 96 ? tracklet_occupancy<true>(&per, block)
                              : tracklet_occupancy<false>(&per, block);
  return e == cudaSuccess ? per : 0;
}

void launch_find(Prof* P, const Geo& g, const Cal& c, const Params& p, const ClIn& cl,
                 const GridDims& gd, const Shapes& sh, int K, FindBuf& b, TrackBuf& tb,
                 uint32_t* cnt, uint32_t* err, cudaStream_t s) {
  int n = cl.n;
  int nb = nblk(n, kB256);
  if (n > 0) {
    const uint32_t* nv = b.row_start + K;
    TPC_LAUNCH(P, "k_neighbours", s, k_neighbours<<<nb, kB256, 0, s>>>(g, p, gd, b.es_dims, nv, b.gyz, b.gorig, b.gseg, b.bin_start,
                                      b.row_start, b.zr, b.up, b.dn));
    TPC_LAUNCH(P, "k_clean", s, k_clean<<<nb, kB256, 0, s>>>(nv, b.up, b.dn, b.upc, b.dnc, b.blk_a));
  }
  TPC_LAUNCH(P, "k_scan_blocks", s, k_scan_blocks<<<1, 1024, 0, s>>>(n > 0 ? nb : 0, b.blk_a, b.off_a, nullptr, nullptr, cnt,
                                   kCntStart, 0, (uint32_t)b.cap_tl, 0u, err, kErrCapStart));
  if (n > 0)
    TPC_LAUNCH(P, "k_write_starts", s, k_write_starts<<<nb, kB256, 0, s>>>(b.row_start + K, b.upc, b.dnc, b.off_a,
                                        (uint32_t)b.cap_tl, p.seed_max_hits, b.starts, b.seed_end));
  cudaMemsetAsync(b.weight, 0, sizeof(unsigned long long) * (size_t)(n > 0 ? n : 1), s);
  Grid G{b.gyz, b.gorig, b.bin_start, b.row_start, b.zr, gd.pads};
  // seeds, then the following order (longest predicted first)
  cudaMemsetAsync(b.tl_hist, 0, sizeof(uint32_t) * kLenBuckets, s);
  TPC_LAUNCH(P, "k_tl_seed", s,
             k_tl_seed<<<min(nblk(b.cap_tl, 128), 64 * 148), 128, 0, s>>>(
                 g, c, p, G, cl.mode, b.upc, b.gseg, b.starts, b.seed_end, cnt, b.seed_st,
                 b.tl_pred, b.tl_hist, b.nh, b.that, b.range));
  TPC_LAUNCH(P, "k_tl_order_scan", s, k_tl_order_scan<<<1, kLenBuckets, 0, s>>>(b.tl_hist));
  TPC_LAUNCH(P, "k_tl_order", s,
             k_tl_order<<<min(nblk(b.cap_tl, kB256), 16 * 148), kB256, 0, s>>>(
                 cnt, b.tl_pred, b.tl_hist, b.tl_order));
  // persistent grid: the tuned number of resident blocks, or fewer for a
  // small capacity
  cudaMemsetAsync(b.queue, 0, sizeof(uint32_t), s);
#define TPC_TRACKLETS(BS, CAP)                                                              \
  {                                                                                        \
    int nbk = nblk(b.cap_tl, BS);                                                          \
    if (sh.tl_grid > 0 && nbk > sh.tl_grid) nbk = sh.tl_grid;                              \
    TPC_LAUNCH(P, "k_tracklets", s,                                                        \
               (k_tracklets<BS, CAP><<<nbk, BS, 0, s>>>(                                   \
                   g, c, p, gd, G, b.es_dims, cl.mode, b.gseg, b.starts, b.seed_end, cnt,   \
                   b.seed_st, b.tl_order, b.nh, b.hits, b.range, b.that, b.queue)));       \
  }
  const bool cap = sh.tl_regs == 96;
  if (sh.tl_block == 64) {
    if (cap) TPC_TRACKLETS(64, true) else TPC_TRACKLETS(64, false)
  } else if (sh.tl_block == 256) {
    if (cap) TPC_TRACKLETS(256, true) else TPC_TRACKLETS(256, false)
  } else {
    if (cap) TPC_TRACKLETS(128, true) else TPC_TRACKLETS(128, false)
  }
#undef TPC_TRACKLETS
  TPC_LAUNCH(P, "k_tl_weight", s,
             k_tl_weight<<<min(nblk(b.cap_tl * 32, kB256), 16 * 148), kB256, 0, s>>>(
                 g.n_rows, p.min_track_hits, cnt, b.nh, b.hits, b.range, b.starts, b.gorig,
                 b.weight));
  int nsel = nblk(b.cap_tl, kB256);
  cudaMemsetAsync(b.grp_count, 0, sizeof(uint32_t), s);
  TPC_LAUNCH(P, "k_select_count", s,
             k_select_count<<<min(nblk(b.cap_tl * 32, kB256), 16 * 148), kB256, 0, s>>>(
                 g.n_rows, p, cnt, b.nh, b.hits, b.range, b.starts, b.gorig, b.weight, b.nkeep));
  TPC_LAUNCH(P, "k_select_sum", s,
             k_select_sum<<<nsel, kB256, 0, s>>>(cnt, b.nkeep, b.starts, b.gorig, b.gseg, b.tkey,
                                                 b.tseg, b.grp_list, b.grp_count, b.cap_grp,
                                                 b.blk_a, b.blk_b));
  TPC_LAUNCH(P, "k_group_rank", s,
             k_group_rank<<<2 * 148, 1024, kRankSmem, s>>>(cnt, b.tkey, b.tseg, b.nkeep,
                                                          b.grp_list, b.grp_count, b.cap_grp,
                                                          b.delta_id, b.delta_o));
  TPC_LAUNCH(P, "k_scan_blocks", s, k_scan_blocks<<<1, 1024, 0, s>>>(nsel, b.blk_a, b.off_a, b.blk_b, b.off_b, cnt, kCntTracks,
                                   kCntAssigned, (uint32_t)tb.cap_tr, (uint32_t)tb.cap_asg, err,
                                   kErrCapTrack));
  TPC_LAUNCH(P, "k_select_write", s, k_select_write<<<nsel, kB256, 0, s>>>(g.n_rows, cnt, b.hits, b.range, b.starts, b.tkey, b.tseg, b.delta_id, b.delta_o, b.that, b.gorig,
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

void launch_calib(Prof* P, const Geo& g, const Cal& c, const ClIn& cl, int64_t cap_asg,
                  TrackBuf& tb, uint32_t* cnt, uint32_t* err, cudaStream_t s) {
  if (cap_asg > 0)
    TPC_LAUNCH(P, "k_calib", s,
               k_calib<<<nblk(cap_asg, kB256), kB256, 0, s>>>(g, c, cl, cnt, tb.cluster_idx,
                                                              tb.asg_track, tb.t_coll, tb.yc,
                                                              tb.zc, tb.meta, err));
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
                                                        b.that, b.hits, b.range, start_hit, nh,
                                                        that, hits);
}

}  // namespace tpc
