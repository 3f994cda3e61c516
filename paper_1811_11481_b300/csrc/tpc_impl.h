// Internal declarations shared by the CUDA translation units and the C ABI.
#pragma once

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "tpc.h"
#include "tpc_math.cuh"

namespace tpc {

// device error word bits
enum : uint32_t {
  kErrArg = 1u,           // invalid cluster field
  kErrCapStart = 2u,      // start-hit / tracklet buffer overflow
  kErrCapRow = 4u,        // a pad-row bucket exceeds the sort tile
  kErrCapTrack = 8u,      // track buffer overflow
  kErrNumeric = 16u,      // non-finite fit output
  kErrTimeout = 32u,      // a bounded wait gave up
  kErrCapPairs = 64u,     // merge candidate-pair list overflow
};

// device counters (uint32 each)
enum : int {
  kCntStart = 0,     // start hits (= tracklets)
  kCntTracks = 1,    // emitted tracks
  kCntAssigned = 2,  // clusters assigned to tracks
  kCntSize = 8,
};

struct Params {
  float sigma, shared_scale, nb_wy, nb_wz, nb_teta, nb_ty, nb_dmax, chi2_pick;
  int32_t max_miss, max_gap, min_track_hits;
  float s_max, inward_cov_scale;
  float c0t[5], c0r[5];
  float chi2_out;
  int32_t min_acc_reject;
  float refit_inflate;
  int32_t seed_max_hits;
  float chi2_merge;
  float split_scale, single_row_scale, single_time_scale, edge_scale;
};

// Search-grid parameters of a batch. The bin geometry itself (ny x nz bins
// per row, the same for all rows of an (event, sector)) is chosen on the
// device from the sector's occupancy.
struct GridDims {
  float tau;              // target clusters per bin
  int32_t nb_max;         // bins per row at most
  int32_t ny_max;         // bins along y at most
  float y_margin;         // cm beyond the sector edge
  float z_margin;         // cm beyond the (event, side) z range
  int32_t pads;           // the grid keeps native pad positions in place of y
};

// Cluster input as the kernels see it (device pointers).
struct ClIn {
  int32_t n;
  int32_t mode;
  int32_t n_events;
  const float* y;
  const float* z;
  const double* t;
  const uint8_t* row;
  const uint8_t* sector;
  const uint8_t* flags;
  const uint32_t* event;
  int32_t pads;  // y holds native pad positions
};

// Local y (cm) of cluster i: the input y, or its native pad position turned
// into cm with the row's pad pitch (single precision, two roundings).
TPC_HD float cluster_y(const Geo& g, const ClIn& cl, int64_t i) {
  if (!cl.pads) return cl.y[i];
  int r = cl.row[i];
  return (cl.y[i] - g.pc[r]) * g.pw[r];
}

// Buffers of the finder (device).
struct FindBuf {
  // bucketing
  uint32_t* cnt;        // [K] cluster count per (event, sector, row)
  uint32_t* row_start;  // [K + 1]
  uint32_t* fill;       // [K]
  uint32_t* row_blk;    // [K / 1024 + 1] block totals, then offsets, of the split bucket scan
  int32_t* zmm;         // [n_events * 2 * 2] ordered-int min/max of seed z per side
  float* zr;            // [n_events * 2 * 2] z0, 1/dz per (event, side)
  float* zs_in;         // [n] seed z in input order
  uint32_t* perm;       // [n] input index in bucket order
  float2* pyz;          // [n] (y, seeding z) in bucket order
  // grid order (bucket, bin, input index)
  float2* gyz;          // [n] (y, seed z)
  uint32_t* gorig;      // [n] input index
  uint32_t* gseg;       // [n] bucket (event*36 + sector)*n_rows + row
  uint16_t* bin_start;  // [cap_bins] per row: nb + 1 bin offsets from the row's bucket start
  uint2* es_dims;       // [n_events * 36]: table base, ny | nz << 16
  uint32_t* n_bins;     // [1] bin-table entries used
  uint32_t* mid_list;   // [K] buckets for the 4096-entry block sort
  uint32_t* big_list;   // [K] buckets for the 16384-entry block sort
  uint32_t* list_counts;  // [2]
  // links (grid positions)
  int32_t* up;
  int32_t* dn;
  int32_t* upc;
  int32_t* dnc;
  // compaction scratch
  uint32_t* blk_a;      // [n_blocks]
  uint32_t* blk_b;
  uint32_t* off_a;      // [n_blocks + 1]
  uint32_t* off_b;
  // tracklets
  uint32_t* starts;     // [cap_tl] grid position of the start hit
  int32_t* nh;          // [cap_tl]
  int32_t* hits;        // [cap_tl * n_rows] grid positions
  double* that;         // [cap_tl]
  unsigned long long* weight;  // [n]
  uint32_t* nkeep;      // [cap_tl]
  uint32_t* queue;      // [1] next start hit of the persistent tracklet kernel
  uint32_t* seed_end;   // [cap_tl] last hit of each start hit's seed
  uint32_t* range;      // [cap_tl] rows lo | hi << 16 of hits[] the tracklet wrote
  float* seed_st;       // [cap_tl * 24] seed state (p, C, x) and an ok flag per tracklet
  uint32_t* tl_pred;    // [cap_tl] predicted following steps of each tracklet
  uint32_t* tl_order;   // [cap_tl] tracklets in following order (longest predicted first)
  uint32_t* tl_hist;    // [512] tracklets per predicted length, then bucket offsets
  uint32_t* tkey;       // [cap_tl] input index of the start hit
  uint32_t* tseg;       // [cap_tl] (event, sector, row) segment of the start hit
  int32_t* delta_id;    // [cap_tl] track-order shift inside large groups
  int32_t* delta_o;     // [cap_tl] cluster-offset shift inside large groups
  uint32_t* grp_list;   // [cap_grp] first tracklet of each large group
  uint32_t* grp_count;  // [1]
  uint32_t cap_grp;
  int64_t cap_tl;
};

// The current track set (device).
struct TrackBuf {
  uint32_t* track_start;  // [cap_tr + 1]
  uint32_t* cluster_idx;  // [cap_asg]
  uint32_t* asg_track;    // [cap_asg]
  double* t_coll;         // [cap_tr]
  uint32_t* start_hit;    // [cap_tr]
  float* yc;              // [cap_asg] calibrated
  float* zc;              // [cap_asg]
  uint32_t* meta;         // [cap_asg] row | flags << 8 | sector << 16
  int64_t cap_tr, cap_asg;
};

// The refit runs one track per thread over tracks sorted by decreasing length;
// per-cluster data and checkpoints are stored warp-interleaved: element k of
// lane l of warp w at (wbase[w] + k) * 32 + l, so that each step of a warp is
// one coalesced access.
struct RefitBuf {
  uint32_t* order;        // [cap_tr] thread slot -> track, decreasing length
  uint32_t* slot;         // [cap_tr] track -> thread slot
  uint32_t* wlen;         // [cap_warp] longest track of each warp
  uint32_t* wbase;        // [cap_warp + 1] first interleaved row of each warp
  uint32_t* len_hist;     // [1024] length histogram and fill counters
  float* w_yc;            // [cap_w] interleaved calibrated y
  float* w_zc;            // [cap_w]
  uint32_t* w_meta;       // [cap_w]
  float* seed;            // [cap_tr * 5]
  uint8_t* rej;           // [cap_w] interleaved rejection pass
  int32_t* status;        // [cap_tr]
  uint8_t* multi;         // [cap_tr] track across sector frames
  float* ckpt;            // [3 * cap_w * 20]
  float* gyc;             // [cap_w] dL/d(calibrated y), interleaved
  float* gzc;             // [cap_w]
  int64_t cap_w;          // interleaved capacity: cap_asg + 32 * 257
  unsigned long long* acc_spline;  // [TPC_SPLINE_SIZE] fixed-point spline-gradient sums
  uint32_t* gmax;         // [1] largest |coordinate gradient| (float bits)
  double* part_cal;       // [n_part_blocks * 2]
  int64_t cap_ckpt;
  // vertex pseudo-measurements (tpc_set_vertex): the caller's z per track
  // (NaN: none) or null, their variance, and the states entering the vertex
  // step of the saved refit
  const float* vz;
  float vvar;
  float* vck;             // [cap_vck * 24]
  int64_t cap_vck;
};

// Segment merging (tpc_merge.cu): a copy of the segments being merged and
// the link search state (device).
struct MergeBuf {
  uint32_t* seg_ts;     // [cap_tr + 1] segment CSR
  uint32_t* seg_ci;     // [cap_asg]
  double* seg_that;     // [cap_tr]
  uint32_t* seg_hit;    // [cap_tr]
  uint32_t* info;       // [cap_tr] bucket (event * 36 + sector) | 1 << 31 when taking part
  uint32_t* rows;       // [cap_tr] first row | last row << 16
  uint32_t* bk_cnt;     // [cap_bk + 1] bucket counts, then offsets
  uint32_t* bk_fill;    // [cap_bk]
  uint32_t* bk_seg;     // [cap_tr] segments by bucket, variance class, tan(lambda)
  float4* bk_v;         // [cap_tr] their tan(lambda), q/pT and the two variances
  float* bk_t;          // [cap_tr] their tan(lambda) alone (binary searches)
  uint32_t* bk_rlo;     // [cap_tr] their first row
  uint32_t* bk_cls;     // [cap_bk * 5] class boundaries of each bucket
  unsigned long long* best_in;   // [cap_tr] chi2 bits << 32 | best predecessor
  unsigned long long* best_out;  // [cap_tr] chi2 bits << 32 | best continuation
  uint2* pairs;         // [cap_pairs] candidate pairs (i, j) that pass the prefilter
  uint32_t* n_pairs;    // [1] pairs found (may exceed cap_pairs: then merged again)
  uint32_t* n_seg;      // [1] segments being merged
  int64_t cap_pairs;
  int32_t* next;        // [cap_tr] linked continuation or -1
  uint8_t* has_in;      // [cap_tr] has a linked predecessor
  uint32_t* hpos;       // [cap_tr] block-local merged-track index of a first segment
  uint32_t* cpos;       // [cap_tr] block-local cluster offset
  uint32_t* blk_h;      // [cap_tr / 1024 + 2] block totals, then offsets
  uint32_t* blk_c;      // [cap_tr / 1024 + 2]
  int64_t cap_tr, cap_asg, cap_bk;
};

// Per-context kernel accounting: every launch is counted; with timing on, a
// pair of CUDA events on the launch stream brackets each kernel.
struct Prof {
  bool on = false;
  int64_t launches = 0;
  struct Rec {
    const char* name;
    cudaEvent_t a, b;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  std::map<std::string, std::pair<int64_t, double>> stats;  // name -> (launches, ms)
  const char* cur = nullptr;
  cudaEvent_t ev() {
    cudaEvent_t e;
    if (!pool.empty()) {
      e = pool.back();
      pool.pop_back();
    } else {
      cudaEventCreate(&e);
    }
    return e;
  }
  std::string only;          // when set, only launches of this kernel are timed
  bool timed_last = false;   // the last begin() recorded an event pair
  void begin(const char* name, cudaStream_t s) {
    ++launches;
    timed_last = on && (only.empty() || only == name);
    if (!timed_last) return;
    Rec r{name, ev(), ev()};
    cudaEventRecord(r.a, s);
    pending.push_back(r);
  }
  void end(cudaStream_t s) {
    if (!timed_last || pending.empty()) return;
    cudaEventRecord(pending.back().b, s);
  }
  // Requires the stream to be synchronised.
  void collect() {
    for (auto& r : pending) {
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, r.a, r.b);
      auto& st = stats[r.name];
      st.first += 1;
      st.second += ms;
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    pending.clear();
  }
  ~Prof() {
    for (auto& r : pending) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

#define TPC_LAUNCH(P, NAME, S, ...) \
  do {                              \
    if (P) (P)->begin(NAME, S);     \
    __VA_ARGS__;                    \
    if (P) (P)->end(S);             \
  } while (0)

constexpr int kGridBinsMax = 8192;  // search-grid bins per row at most
constexpr int kSmallGroup = 64;  // start-hit groups up to this size are ranked by a scan
constexpr int kRankTile = 8192;   // emitted tracklets a block ranks in shared memory
constexpr int kSortTile = 4096;      // pad-row bucket tile of the common sort
constexpr int kSortTileBig = 16384;  // tile of the large-bucket sort (128 KB)
constexpr int kCalibGradBlocks = 4 * 148;

#ifdef __CUDACC__
// atomicAdd(&ctr[key], 1) for every active lane, one atomic per distinct key
// of the warp: the lanes with the same key take consecutive values in lane
// order after the group leader's add. Returns the lane's value. Called by
// converged lanes (the active mask is the set of callers).
__device__ __forceinline__ uint32_t warp_counter_add1(uint32_t* ctr, uint32_t key) {
  const unsigned act = __activemask();
  const unsigned peers = __match_any_sync(act, key);
  const int lane = (int)(threadIdx.x & 31);
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0u;
  if (lane == leader) base = atomicAdd(&ctr[key], (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  return base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}
#endif

// launchers (tpc_find.cu)
void launch_load(Prof* P, const Geo& g, const Cal& c, const ClIn& cl, const GridDims& gd, int K,
                 FindBuf& b, uint32_t* err, cudaStream_t s);
// Launch shapes chosen by the autotuner (none of them changes a result).
struct Shapes {
  int tl_block = 128;    // tracklet kernel threads per block (64, 128, 256)
  int tl_grid = 0;       // persistent tracklet grid (0: one block per 128 tracklets)
  int tl_regs = 0;       // tracklet kernel register cap (0: compiler's choice, 96)
};
// Resident blocks per SM of the tracklet kernel at a block size.
int tracklet_blocks_per_sm(int block, int regs);
// Kernel attributes (shared-memory limits), once per context.
void setup_find_kernels();
void launch_find(Prof* P, const Geo& g, const Cal& c, const Params& p, const ClIn& cl,
                 const GridDims& gd, const Shapes& sh, int K, FindBuf& b, TrackBuf& tb,
                 uint32_t* cnt, uint32_t* err, cudaStream_t s);
void launch_set_tracks(Prof* P, const Geo& g, const Cal& c, const ClIn& cl, int64_t n_tracks,
                       int64_t n_asg, TrackBuf& tb, uint32_t* cnt, uint32_t* err, cudaStream_t s);
void launch_calib(Prof* P, const Geo& g, const Cal& c, const ClIn& cl, int64_t cap_asg,
                  TrackBuf& tb, uint32_t* cnt, uint32_t* err, cudaStream_t s);
void launch_spline_bound(const float* spline, float* bound, cudaStream_t s);
void launch_export_links(const FindBuf& b, int n, int K, int32_t* up, int32_t* dn, int32_t* upc,
                         int32_t* dnc, cudaStream_t s);
void launch_export_tracklets(const FindBuf& b, int n_rows, int64_t n_cap, const uint32_t* cnt,
                             uint32_t* start_hit, int32_t* nh, double* that, int32_t* hits,
                             cudaStream_t s);

// Host-side check of a geometry as every entry point that takes one
// accepts it: 3 .. TPC_MAX_ROWS pad rows with strictly increasing plane
// positions, a positive half-opening tangent and a positive drift length.
inline bool geometry_valid(const tpc_geometry* geo) {
  if (!geo || !geo->row_x || geo->n_rows < 3 || geo->n_rows > TPC_MAX_ROWS) return false;
  for (int r = 1; r < geo->n_rows; ++r)
    if (!(geo->row_x[r] > geo->row_x[r - 1])) return false;
  return geo->tan_half > 0.0f && geo->drift_length > 0.0f;
}

// launchers (tpc_refit.cu)
void launch_refit(Prof* P, const Geo& g, const Params& p, int64_t cap_tr, const uint32_t* cnt,
                  const TrackBuf& tb, RefitBuf& rb, bool save, float* params, float* cov,
                  float* x, float* chi2, int32_t* ndf, int32_t* status, uint8_t* rej,
                  uint32_t* err, cudaStream_t s);
void launch_refit_backward(Prof* P, const Geo& g, const Cal& c, const Params& p, const ClIn& cl,
                           int64_t cap_tr, int64_t cap_asg, const uint32_t* cnt,
                           const TrackBuf& tb, RefitBuf& rb, const float* dl_dchi2,
                           float* grad_y, float* grad_zt, double* grad_calib, cudaStream_t s);

// launcher (tpc_merge.cu): merges the current track set of tb (at most
// cap_n segments; counts read on the device; refitted states params, cov,
// x, status), writes the merged set into tb and its count into
// cnt[kCntTracks]; next_out and link_chi2 (may be null) receive each
// segment's link and its chi2; a candidate-pair overflow sets kErrCapPairs
// in err. copy = false merges again the segments copied by the previous
// call (after a pair-list overflow).
void launch_merge(Prof* P, const Geo& g, const Params& p, const Cal& c, const ClIn& cl,
                  int64_t cap_n, bool copy, TrackBuf& tb, MergeBuf& mb, const float* params,
                  const float* cov, const float* x, const int32_t* status, int32_t* next_out,
                  float* link_chi2, uint32_t* cnt, uint32_t* err, cudaStream_t s);
// Kernel attributes of the merge (shared-memory limit), once per context.
void setup_merge_kernels();
// launcher (tpc_compress.cu): residuals of the track set's clusters against
// the track model (and the decoded clusters; dy, dz may be null).
void launch_compress(Prof* P, const Geo& g, const Cal& c, const ClIn& cl, const Params& p,
                     float qy, float qz, int64_t cap_tr, const uint32_t* cnt, const TrackBuf& tb,
                     int32_t* ry, int32_t* rz, float* dy, float* dz, cudaStream_t s);
// Collision times of the track set refined from its fit (time-frame mode),
// written to tb.t_coll and t_out (may be null).
void launch_refine_time(Prof* P, const Geo& g, const Cal& c, const ClIn& cl, int64_t cap_tr,
                        const uint32_t* cnt, TrackBuf& tb, const float* params, const float* x,
                        const int32_t* status, double* t_out, cudaStream_t s);

}  // namespace tpc
