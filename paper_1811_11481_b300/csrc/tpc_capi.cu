// C ABI of the library (declared in include/tpc.h).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <string>

#include "tpc_impl.h"

using namespace tpc;

struct tpc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  Geo geo{};
  Params prm{};
  tpc_params prm_c{};
  Cal cal{};
  float* d_rowx = nullptr;       // [TPC_MAX_ROWS] pad-row positions
  float* d_pads = nullptr;       // [2 * TPC_MAX_ROWS] pad pitch and centre per row
  float* d_spline = nullptr;
  float* d_spl_bound = nullptr;
  uint32_t* d_err = nullptr;
  uint32_t* d_cnt = nullptr;
  uint32_t* h_pinned = nullptr;  // [kCntSize + 1]: counters and error word
  // batch
  ClIn cl{};
  bool loaded = false;
  int K = 0;
  GridDims gd{};
  tpc_tuning tune{1.0f, 16, 128, 0, 0};
  Shapes sh{};
  int sms = 0;
  FindBuf fb{};
  TrackBuf tb{};
  RefitBuf rb{};
  MergeBuf mb{};
  // concatenated inputs of tpc_find_tracks_batched (library-owned)
  struct {
    float* y = nullptr;
    float* z = nullptr;
    double* t = nullptr;
    uint8_t *row = nullptr, *sector = nullptr, *flags = nullptr;
    uint32_t* event = nullptr;
    int64_t cap = 0;
  } bb;
  Prof prof;
  // capacities
  int64_t cap_n = 0, cap_K = 0, cap_bins = 0, cap_blk = 0, cap_ev = 0;
  int64_t tl_factor = 8;  // cap_tl = n / tl_factor (halved on overflow)
  int64_t cap_tr_alloc = 0, cap_asg_alloc = 0, cap_ckpt_alloc = 0;
  bool tracks_valid = false;
  bool saved = false;
  bool part_alloc = false;
  const float* saved_vz = nullptr;  // vertex array of the saved refit
  bool capturing = false;
  int64_t calib_version = 0;        // incremented by tpc_set_calib
  int64_t refit_calib_version = -1;  // calibration of the saved refit
  int64_t coords_calib_version = -1;  // calibration of the track set's yc, zc
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int64_t graph_kernels = 0;     // kernel launches recorded in the graph
  int64_t launches_before = 0;
  bool prof_was_on = false;
  std::string err;
};

namespace {

tpc_status fail(tpc_ctx* c, tpc_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

#define CK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ == cudaErrorStreamCaptureUnsupported)                                     \
      return fail(ctx, TPC_ERR_STATE, "allocation during graph capture: run the sequence "  \
                                      "once before capturing");                       \
    if (e_ != cudaSuccess)                                                           \
      return fail(ctx, TPC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

thread_local bool g_capturing_alloc_guard = false;  // set while a context captures

template <class T>
cudaError_t grow(T*& p, int64_t& cap, int64_t need) {
  if (need <= cap && p) return cudaSuccess;
  if (g_capturing_alloc_guard) return cudaErrorStreamCaptureUnsupported;
  if (p) cudaFree(p);
  p = nullptr;
  int64_t c = need > 0 ? need : 1;
  cudaError_t e = cudaMalloc((void**)&p, sizeof(T) * (size_t)c);
  cap = e == cudaSuccess ? c : 0;
  return e;
}

template <class T>
cudaError_t alloc(T*& p, int64_t n) {
  if (g_capturing_alloc_guard) return cudaErrorStreamCaptureUnsupported;
  if (p) cudaFree(p);
  p = nullptr;
  return cudaMalloc((void**)&p, sizeof(T) * (size_t)(n > 0 ? n : 1));
}

void copy_params(const tpc_params& s, Params& d) {
  d.sigma = s.sigma;
  d.shared_scale = s.shared_scale;
  d.nb_wy = s.nb_wy;
  d.nb_wz = s.nb_wz;
  d.nb_teta = s.nb_teta;
  d.nb_ty = s.nb_ty;
  d.nb_dmax = s.nb_dmax;
  d.chi2_pick = s.chi2_pick;
  d.max_miss = s.max_miss;
  d.max_gap = s.max_gap;
  d.min_track_hits = s.min_track_hits;
  d.s_max = s.s_max;
  d.inward_cov_scale = s.inward_cov_scale;
  for (int i = 0; i < 5; ++i) {
    d.c0t[i] = s.c0t[i];
    d.c0r[i] = s.c0r[i];
  }
  d.chi2_out = s.chi2_out;
  d.min_acc_reject = s.min_acc_reject;
  d.refit_inflate = s.refit_inflate;
  d.seed_max_hits = s.seed_max_hits;
  d.chi2_merge = s.chi2_merge;
  d.split_scale = s.split_scale;
  d.single_row_scale = s.single_row_scale;
  d.single_time_scale = s.single_time_scale;
  d.edge_scale = s.edge_scale;
}

std::string err_text(uint32_t e) {
  std::string s;
  if (e & kErrArg) s += "invalid cluster field (row, sector, event or time); ";
  if (e & kErrCapStart) s += "start-hit buffer overflow (retry enlarges it); ";
  if (e & kErrCapRow) s += "a pad-row bucket exceeds 16384 clusters; ";
  if (e & kErrCapTrack) s += "track buffer overflow; ";
  if (e & kErrNumeric) s += "non-finite value in a refit; ";
  if (e & kErrTimeout) s += "a bounded device wait gave up; ";
  if (e & kErrCapPairs)
    s += "merge candidate-pair list overflow (tpc_merge_tracks enlarges it); ";
  return s;
}

tpc_status status_of(uint32_t e) {
  if (e & kErrArg) return TPC_ERR_ARG;
  if (e & (kErrCapStart | kErrCapRow | kErrCapTrack | kErrCapPairs)) return TPC_ERR_CAPACITY;
  if (e & kErrTimeout) return TPC_ERR_TIMEOUT;
  if (e & kErrNumeric) return TPC_ERR_NUMERIC;
  return TPC_OK;
}

// Read counters and error word (synchronises the stream).
tpc_status read_back(tpc_ctx* ctx) {
  if (ctx->capturing) return fail(ctx, TPC_ERR_STATE, "synchronising call during graph capture");
  CK(cudaMemcpyAsync(ctx->h_pinned, ctx->d_cnt, sizeof(uint32_t) * kCntSize,
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(ctx->h_pinned + kCntSize, ctx->d_err, sizeof(uint32_t),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  uint32_t e = ctx->h_pinned[kCntSize];
  if (e) {
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), ctx->stream));
    if (e & kErrCapStart) ctx->tl_factor = ctx->tl_factor > 1 ? ctx->tl_factor / 2 : 1;
    return fail(ctx, status_of(e), err_text(e));
  }
  return TPC_OK;
}

// Launch shapes from the tuning: the persistent tracklet grid is the SM
// count times the resident blocks per SM (capped by tracklet_per_sm).
void apply_tuning(tpc_ctx* ctx) {
  const tpc_tuning& t = ctx->tune;
  ctx->sh.tl_block = t.tracklet_block;
  ctx->sh.tl_regs = t.tracklet_regs;
  int per = tracklet_blocks_per_sm(t.tracklet_block, t.tracklet_regs);
  if (t.tracklet_per_sm > 0 && t.tracklet_per_sm < per) per = t.tracklet_per_sm;
  ctx->sh.tl_grid = (ctx->sms > 0 && per > 0) ? ctx->sms * per : 0;
}

bool valid_block(int b) { return b == 64 || b == 128 || b == 256; }

tpc_status ensure_track_buffers(tpc_ctx* ctx, int64_t cap_tr, int64_t cap_asg) {
  TrackBuf& t = ctx->tb;
  RefitBuf& rb = ctx->rb;
  if (cap_tr > ctx->cap_tr_alloc) {
    CK(alloc(t.track_start, cap_tr + 1));
    CK(alloc(t.t_coll, cap_tr));
    CK(alloc(t.start_hit, cap_tr));
    CK(alloc(rb.seed, cap_tr * 5));
    CK(alloc(rb.order, cap_tr));
    CK(alloc(rb.slot, cap_tr));
    CK(alloc(rb.wlen, cap_tr / 32 + 2));
    CK(alloc(rb.wbase, cap_tr / 32 + 3));
    CK(alloc(rb.status, cap_tr));
    CK(alloc(rb.multi, cap_tr));
    ctx->cap_tr_alloc = cap_tr;
  }
  if (cap_asg > ctx->cap_asg_alloc) {
    int64_t cap_w = cap_asg + 32 * 257;
    CK(alloc(t.cluster_idx, cap_asg));
    CK(alloc(t.asg_track, cap_asg));
    CK(alloc(t.yc, cap_asg));
    CK(alloc(t.zc, cap_asg));
    CK(alloc(t.meta, cap_asg));
    CK(alloc(rb.w_yc, cap_w));
    CK(alloc(rb.w_zc, cap_w));
    CK(alloc(rb.w_meta, cap_w));
    CK(alloc(rb.rej, cap_w));
    CK(alloc(rb.gyc, cap_w));
    CK(alloc(rb.gzc, cap_w));
    rb.cap_w = cap_w;
    ctx->cap_asg_alloc = cap_asg;
  }
  t.cap_tr = cap_tr;
  t.cap_asg = cap_asg;
  return TPC_OK;
}

tpc_status ensure_tracklets(tpc_ctx* ctx) {
  int64_t n = ctx->cl.n;
  int64_t cap = n / ctx->tl_factor + 1024;
  if (cap > n + 1) cap = n + 1;
  FindBuf& b = ctx->fb;
  if (cap > b.cap_tl) {
    CK(alloc(b.starts, cap));
    CK(alloc(b.seed_end, cap));
    CK(alloc(b.range, cap));
    CK(alloc(b.seed_st, cap * 24));
    CK(alloc(b.tl_pred, cap));
    CK(alloc(b.tl_order, cap));
    if (!b.tl_hist) CK(alloc(b.tl_hist, 512));
    CK(alloc(b.tkey, cap));
    CK(alloc(b.tseg, cap));
    CK(alloc(b.delta_id, cap));
    CK(alloc(b.delta_o, cap));
    b.cap_grp = (uint32_t)(cap / (kSmallGroup + 1) + 1);
    CK(alloc(b.grp_list, (int64_t)b.cap_grp));
    CK(alloc(b.nh, cap));
    CK(alloc(b.hits, cap * (int64_t)ctx->geo.n_rows));
    CK(alloc(b.that, cap));
    CK(alloc(b.nkeep, cap));
    b.cap_tl = cap;
    int64_t nblk = (cap + 255) / 256 + 1;
    if (nblk > ctx->cap_blk) {
      int64_t tmp = 0;
      CK(grow(b.blk_a, tmp, nblk));
      tmp = 0;
      CK(grow(b.blk_b, tmp, nblk));
      tmp = 0;
      CK(grow(b.off_a, tmp, nblk + 1));
      tmp = 0;
      CK(grow(b.off_b, tmp, nblk + 1));
      ctx->cap_blk = nblk;
    }
  }
  return TPC_OK;
}

}  // namespace

extern "C" {

void tpc_default_params(tpc_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->sigma = 0.1f;
  p->shared_scale = 2.0f;
  p->nb_wy = 0.5f;
  p->nb_wz = 0.5f;
  p->nb_teta = (float)std::sinh(1.0);
  p->nb_ty = 1.0f;
  p->nb_dmax = 0.5f;
  p->chi2_pick = 16.0f;
  p->max_miss = 4;
  p->max_gap = 4;
  p->min_track_hits = 10;
  p->s_max = 0.95f;
  p->inward_cov_scale = 4.0f;
  const float c0t[5] = {0.01f, 0.01f, 1.0f, 1.0f, 100.0f};
  const float c0r[5] = {1.0f, 1.0f, 0.1f, 0.1f, 10.0f};
  for (int i = 0; i < 5; ++i) {
    p->c0t[i] = c0t[i];
    p->c0r[i] = c0r[i];
  }
  p->chi2_out = 25.0f;
  p->min_acc_reject = 5;
  p->refit_inflate = 100.0f;
  p->seed_max_hits = 10;
  p->chi2_merge = 30.0f;
  p->split_scale = 1.5f;
  p->single_row_scale = 1.5f;
  p->single_time_scale = 1.5f;
  p->edge_scale = 2.0f;
}

tpc_status tpc_create(const tpc_geometry* geo, const tpc_params* params, void* stream,
                      tpc_ctx** out) {
  if (!out) return TPC_ERR_ARG;
  *out = nullptr;
  if (!geometry_valid(geo)) return TPC_ERR_ARG;
  tpc_ctx* ctx = new tpc_ctx();
  if (cudaGetDevice(&ctx->device) != cudaSuccess) {
    delete ctx;
    return TPC_ERR_CUDA;
  }
  ctx->stream = (cudaStream_t)stream;
  Geo& g = ctx->geo;
  std::memset(&g, 0, sizeof(g));
  g.n_rows = geo->n_rows;
  g.tan_half = geo->tan_half;
  g.L = geo->drift_length;
  g.bz = geo->bz;
  g.kB = (float)2.99792458e-3 * geo->bz;
  if (params) ctx->prm_c = *params;
  else tpc_default_params(&ctx->prm_c);
  copy_params(ctx->prm_c, ctx->prm);
  tpc_status st = TPC_OK;
  auto chk = [&](cudaError_t e) {
    if (e != cudaSuccess && st == TPC_OK) {
      st = TPC_ERR_CUDA;
      ctx->err = cudaGetErrorString(e);
    }
  };
  chk(cudaMalloc(&ctx->d_rowx, sizeof(float) * TPC_MAX_ROWS));
  chk(cudaMalloc(&ctx->d_spline, sizeof(float) * TPC_SPLINE_SIZE));
  chk(cudaMalloc(&ctx->d_spl_bound, sizeof(float) * 4));
  chk(cudaMalloc(&ctx->d_err, sizeof(uint32_t)));
  chk(cudaMalloc(&ctx->d_cnt, sizeof(uint32_t) * kCntSize));
  chk(cudaMalloc(&ctx->rb.len_hist, sizeof(uint32_t) * 1024));
  chk(cudaMalloc(&ctx->fb.list_counts, sizeof(uint32_t) * 2));
  chk(cudaMalloc(&ctx->fb.n_bins, sizeof(uint32_t)));
  chk(cudaMalloc(&ctx->fb.queue, sizeof(uint32_t)));
  chk(cudaMalloc(&ctx->fb.grp_count, sizeof(uint32_t)));
  chk(cudaMallocHost(&ctx->h_pinned, sizeof(uint32_t) * (kCntSize + 1)));
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev);
  }
  apply_tuning(ctx);
  setup_find_kernels();
  setup_merge_kernels();
  if (st != TPC_OK) {
    tpc_destroy(ctx);
    return st;
  }
  chk(cudaMemcpy(ctx->d_rowx, geo->row_x, sizeof(float) * geo->n_rows, cudaMemcpyHostToDevice));
  g.rx = ctx->d_rowx;
  if (geo->field) {
    g.field_on = 1;
    for (int i = 0; i < 30; ++i) g.field[i] = geo->field[i];
  }
  if (geo->pad_width && geo->pad_center) {
    chk(cudaMalloc(&ctx->d_pads, sizeof(float) * 2 * TPC_MAX_ROWS));
    chk(cudaMemcpy(ctx->d_pads, geo->pad_width, sizeof(float) * geo->n_rows,
                   cudaMemcpyHostToDevice));
    chk(cudaMemcpy(ctx->d_pads + TPC_MAX_ROWS, geo->pad_center, sizeof(float) * geo->n_rows,
                   cudaMemcpyHostToDevice));
    g.pw = ctx->d_pads;
    g.pc = ctx->d_pads + TPC_MAX_ROWS;
  }
  chk(cudaMemsetAsync(ctx->d_spline, 0, sizeof(float) * TPC_SPLINE_SIZE, ctx->stream));
  chk(cudaMemsetAsync(ctx->d_spl_bound, 0, sizeof(float) * 4, ctx->stream));
  chk(cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), ctx->stream));
  chk(cudaMemsetAsync(ctx->d_cnt, 0, sizeof(uint32_t) * kCntSize, ctx->stream));
  ctx->cal.vdrift = 2.58;
  ctx->cal.t0 = 0.0;
  ctx->cal.tf_start = 0.0;
  ctx->cal.spline = ctx->d_spline;
  ctx->cal.spl_bound = ctx->d_spl_bound;
  ctx->cal.spl_x0 = 85.0f;
  ctx->cal.spl_dx = 160.0f;
  if (st != TPC_OK) {
    tpc_destroy(ctx);
    return st;
  }
  *out = ctx;
  return TPC_OK;
}

void tpc_destroy(tpc_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  void* ptrs[] = {ctx->d_rowx, ctx->d_pads, ctx->d_spline, ctx->d_spl_bound, ctx->d_err, ctx->d_cnt,
                  ctx->fb.cnt, ctx->fb.row_start, ctx->fb.fill, ctx->fb.row_blk, ctx->fb.zmm, ctx->fb.zr,
                  ctx->fb.zs_in, ctx->fb.perm, ctx->fb.pyz, ctx->fb.gyz,
                  ctx->fb.gorig, ctx->fb.gseg, ctx->fb.bin_start, ctx->fb.big_list, ctx->fb.mid_list, ctx->fb.list_counts,
                  ctx->fb.n_bins, ctx->fb.es_dims, ctx->fb.queue, ctx->fb.up, ctx->fb.dn,
                  ctx->fb.upc, ctx->fb.dnc, ctx->fb.blk_a, ctx->fb.blk_b, ctx->fb.off_a,
                  ctx->fb.off_b, ctx->fb.starts, ctx->fb.seed_end, ctx->fb.range, ctx->fb.seed_st, ctx->fb.tl_pred, ctx->fb.tl_order, ctx->fb.tl_hist, ctx->fb.tkey, ctx->fb.tseg, ctx->fb.delta_id, ctx->fb.delta_o, ctx->fb.grp_list, ctx->fb.grp_count, ctx->fb.nh, ctx->fb.hits, ctx->fb.that,
                  ctx->fb.weight, ctx->fb.nkeep, ctx->tb.track_start, ctx->tb.cluster_idx,
                  ctx->tb.asg_track, ctx->tb.t_coll, ctx->tb.start_hit, ctx->tb.yc, ctx->tb.zc,
                  ctx->tb.meta, ctx->rb.seed, ctx->rb.order, ctx->rb.slot, ctx->rb.wlen, ctx->rb.wbase, ctx->rb.len_hist,
                  ctx->rb.w_yc, ctx->rb.w_zc, ctx->rb.w_meta, ctx->rb.rej, ctx->rb.status, ctx->rb.multi, ctx->rb.ckpt,
                  ctx->rb.gyc, ctx->rb.gzc, ctx->rb.acc_spline, ctx->rb.gmax, ctx->rb.part_cal,
                  ctx->mb.seg_ts, ctx->mb.seg_ci, ctx->mb.seg_that, ctx->mb.seg_hit,
                  ctx->mb.info, ctx->mb.rows, ctx->mb.bk_cnt, ctx->mb.bk_fill, ctx->mb.bk_seg,
                  ctx->mb.bk_v, ctx->mb.bk_t, ctx->mb.bk_rlo, ctx->mb.bk_cls,
                  ctx->mb.best_in, ctx->mb.best_out, ctx->mb.next, ctx->mb.has_in,
                  ctx->mb.pairs, ctx->mb.n_pairs, ctx->mb.n_seg,
                  ctx->mb.hpos, ctx->mb.cpos, ctx->mb.blk_h, ctx->mb.blk_c,
                  ctx->bb.y, ctx->bb.z, ctx->bb.t, ctx->bb.row, ctx->bb.sector, ctx->bb.flags,
                  ctx->bb.event, ctx->rb.vck};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  delete ctx;
}

tpc_status tpc_set_calib(tpc_ctx* ctx, const tpc_calib* calib) {
  if (!ctx || !calib) return fail(ctx, TPC_ERR_ARG, "null argument");
  if (!(calib->vdrift > 0.0) || !(calib->spl_dx != 0.0f))
    return fail(ctx, TPC_ERR_ARG, "vdrift must be > 0 and spl_dx != 0");
  ctx->cal.vdrift = calib->vdrift;
  ctx->cal.t0 = calib->t0;
  ctx->cal.spl_x0 = calib->spl_x0;
  ctx->cal.spl_dx = calib->spl_dx;
  if (calib->spline) {
    CK(cudaMemcpyAsync(ctx->d_spline, calib->spline, sizeof(float) * TPC_SPLINE_SIZE,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  } else {
    CK(cudaMemsetAsync(ctx->d_spline, 0, sizeof(float) * TPC_SPLINE_SIZE, ctx->stream));
  }
  launch_spline_bound(ctx->d_spline, ctx->d_spl_bound, ctx->stream);
  CK(cudaGetLastError());
  ++ctx->calib_version;
  return TPC_OK;
}

tpc_status prepare_load(tpc_ctx* ctx, int n_events);

tpc_status tpc_load_clusters(tpc_ctx* ctx, const tpc_clusters* in) {
  if (!ctx || !in) return fail(ctx, TPC_ERR_ARG, "null argument");
  if (in->n < 0 || in->n >= (int64_t)1 << 31) return fail(ctx, TPC_ERR_ARG, "n out of range");
  if (in->mode != 0 && in->mode != 1) return fail(ctx, TPC_ERR_ARG, "mode must be 0 or 1");
  if (in->n_events < 1 || in->n_events > 4096) return fail(ctx, TPC_ERR_ARG, "n_events");
  if (in->n > 0 && (!in->y || !in->row || !in->sector || (in->mode == 0 && !in->z) ||
                    (in->mode == 1 && !in->t)))
    return fail(ctx, TPC_ERR_ARG, "missing cluster array");
  if (in->n_events > 1 && in->n > 0 && !in->event)
    return fail(ctx, TPC_ERR_ARG, "event array required for n_events > 1");
  if (in->pads != 0 && in->pads != 1) return fail(ctx, TPC_ERR_ARG, "pads must be 0 or 1");
  if (in->pads && !ctx->geo.pw)
    return fail(ctx, TPC_ERR_ARG, "native pad positions need the geometry's pad tables");
  ctx->cl.n = (int32_t)in->n;
  ctx->cl.mode = in->mode;
  ctx->cl.n_events = in->n_events;
  ctx->cl.y = in->y;
  ctx->cl.z = in->z;
  ctx->cl.t = in->t;
  ctx->cl.row = in->row;
  ctx->cl.sector = in->sector;
  ctx->cl.flags = in->flags;
  ctx->cl.event = in->event;
  ctx->cl.pads = in->pads;
  ctx->cal.tf_start = in->mode == 1 ? in->tf_start : 0.0;
  ctx->K = in->n_events * TPC_N_SECTORS * ctx->geo.n_rows;
  return prepare_load(ctx, in->n_events);
}

// Capacities for the loaded batch and the load kernels (row bucketing, search
// grid). Also used by the autotuner to rebuild the grid of the same batch.
tpc_status prepare_load(tpc_ctx* ctx, int n_events) {
  int64_t n = ctx->cl.n;
  int K = ctx->K;
  // search grid: the tuned clusters per bin, geometry chosen on the device
  ctx->gd.tau = ctx->tune.grid_tau;
  ctx->gd.nb_max = kGridBinsMax;
  ctx->gd.ny_max = ctx->tune.grid_ny_max;
  ctx->gd.y_margin = 2.0f;
  ctx->gd.pads = ctx->cl.pads;
  ctx->gd.z_margin = 1.0f;
  FindBuf& b = ctx->fb;
  if (n > ctx->cap_n || ctx->cap_n == 0) {
    int64_t c = n > 0 ? n : 1;
    CK(alloc(b.zs_in, c));
    CK(alloc(b.perm, c));
    CK(alloc(b.pyz, c));
    CK(alloc(b.gyz, c));
    CK(alloc(b.gorig, c));
    CK(alloc(b.gseg, c));
    CK(alloc(b.up, c));
    CK(alloc(b.dn, c));
    CK(alloc(b.upc, c));
    CK(alloc(b.dnc, c));
    CK(alloc(b.weight, c));
    ctx->cap_n = c;
    int64_t nblk = (c + 255) / 256 + 1;
    if (nblk > ctx->cap_blk) {
      int64_t tmp = 0;
      CK(grow(b.blk_a, tmp, nblk));
      tmp = 0;
      CK(grow(b.blk_b, tmp, nblk));
      tmp = 0;
      CK(grow(b.off_a, tmp, nblk + 1));
      tmp = 0;
      CK(grow(b.off_b, tmp, nblk + 1));
      ctx->cap_blk = nblk;
    }
  }
  if (K > ctx->cap_K) {
    CK(alloc(b.big_list, K));
    CK(alloc(b.mid_list, K));
    CK(alloc(b.cnt, K));
    CK(alloc(b.row_start, (int64_t)K + 1));
    CK(alloc(b.fill, K));
    CK(alloc(b.row_blk, (int64_t)K / 1024 + 1));
    ctx->cap_K = K;
  }
  if (n_events > ctx->cap_ev) {
    CK(alloc(b.zmm, (int64_t)n_events * 4));
    CK(alloc(b.zr, (int64_t)n_events * 4));
    CK(alloc(b.es_dims, (int64_t)n_events * TPC_N_SECTORS));
    ctx->cap_ev = n_events;
  }
  // per row: nb + 1 <= total / (rows * tau) + ny_max + 1 entries
  int64_t nbins = (int64_t)((double)n / ctx->gd.tau) + (int64_t)K * (ctx->gd.ny_max + 2) + 64;
  if (nbins > ctx->cap_bins) {
    CK(alloc(b.bin_start, nbins));
    ctx->cap_bins = nbins;
  }
  tpc_status st = ensure_tracklets(ctx);
  if (st != TPC_OK) return st;
  st = ensure_track_buffers(ctx, n / (ctx->prm.min_track_hits > 0 ? ctx->prm.min_track_hits : 1) + 1,
                            n + 1);
  if (st != TPC_OK) return st;
  launch_load(&ctx->prof, ctx->geo, ctx->cal, ctx->cl, ctx->gd, K, b, ctx->d_err, ctx->stream);
  CK(cudaGetLastError());
  ctx->loaded = true;
  ctx->tracks_valid = false;
  ctx->saved = false;
  return TPC_OK;
}

tpc_status tpc_find_tracks_async(tpc_ctx* ctx) {
  if (ctx) ctx->rb.vz = nullptr;  // a new track set: no vertices
  if (!ctx) return TPC_ERR_ARG;
  if (!ctx->loaded) return fail(ctx, TPC_ERR_STATE, "no batch loaded");
  tpc_status st = ensure_tracklets(ctx);
  if (st != TPC_OK) return st;
  launch_find(&ctx->prof, ctx->geo, ctx->cal, ctx->prm, ctx->cl, ctx->gd, ctx->sh, ctx->K, ctx->fb, ctx->tb,
              ctx->d_cnt, ctx->d_err, ctx->stream);
  CK(cudaGetLastError());
  ctx->coords_calib_version = ctx->calib_version;
  ctx->tracks_valid = true;
  ctx->saved = false;
  return TPC_OK;
}

tpc_status tpc_find_tracks(tpc_ctx* ctx, tpc_tracks* out) {
  tpc_status st = tpc_find_tracks_async(ctx);
  if (st != TPC_OK) return st;
  st = read_back(ctx);
  if (st == TPC_ERR_CAPACITY && (ctx->h_pinned[kCntSize] & kErrCapStart)) {
    // retry once with a larger tracklet buffer
    st = tpc_find_tracks_async(ctx);
    if (st != TPC_OK) return st;
    st = read_back(ctx);
  }
  if (st != TPC_OK) return st;
  if (out) {
    out->n_tracks = ctx->h_pinned[kCntTracks];
    out->n_assigned = ctx->h_pinned[kCntAssigned];
    out->track_start = ctx->tb.track_start;
    out->cluster_idx = ctx->tb.cluster_idx;
    out->t_coll = ctx->tb.t_coll;
    out->start_hit = ctx->tb.start_hit;
  }
  return TPC_OK;
}

namespace {
// Event index of each cluster of one part of a batched call: the part's own
// index (0 when it has none) shifted by the events of the parts before it.
__global__ void k_batch_event(int64_t n, const uint32_t* ev_in, uint32_t offset, uint32_t* out) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = offset + (ev_in ? ev_in[j] : 0u);
}
}  // namespace

tpc_status tpc_find_tracks_batched(tpc_ctx* ctx, const tpc_clusters* ev, int32_t n_parts,
                                   tpc_tracks* out) {
  if (!ctx || !ev) return fail(ctx, TPC_ERR_ARG, "null argument");
  if (ctx->capturing) return fail(ctx, TPC_ERR_STATE, "tpc_find_tracks_batched synchronises");
  if (n_parts < 1) return fail(ctx, TPC_ERR_ARG, "n_parts must be >= 1");
  int64_t n = 0;
  int64_t n_events = 0;
  for (int32_t i = 0; i < n_parts; ++i) {
    const tpc_clusters& c = ev[i];
    if (c.n < 0 || c.n_events < 1) return fail(ctx, TPC_ERR_ARG, "part: n or n_events");
    if (c.mode != ev[0].mode || c.pads != ev[0].pads)
      return fail(ctx, TPC_ERR_ARG, "parts differ in mode or pads");
    if (c.mode == 1 && c.tf_start != ev[0].tf_start)
      return fail(ctx, TPC_ERR_ARG, "parts of a time-frame batch need the same tf_start");
    if (c.n > 0 && (!c.y || !c.row || !c.sector || (c.mode == 0 && !c.z) ||
                    (c.mode == 1 && !c.t)))
      return fail(ctx, TPC_ERR_ARG, "part: missing cluster array");
    if (c.n_events > 1 && c.n > 0 && !c.event)
      return fail(ctx, TPC_ERR_ARG, "part: event array required for n_events > 1");
    n += c.n;
    n_events += c.n_events;
  }
  if (n >= (int64_t)1 << 31) return fail(ctx, TPC_ERR_ARG, "n out of range");
  if (n_events > 4096) return fail(ctx, TPC_ERR_ARG, "more than 4096 events");
  const int mode = ev[0].mode;
  auto& B = ctx->bb;
  if (n > B.cap || !B.y) {
    int64_t c = n > 0 ? n : 1;
    CK(alloc(B.y, c));
    CK(alloc(B.z, c));
    CK(alloc(B.t, c));
    CK(alloc(B.row, c));
    CK(alloc(B.sector, c));
    CK(alloc(B.flags, c));
    CK(alloc(B.event, c));
    B.cap = c;
  }
  cudaStream_t s = ctx->stream;
  int64_t off = 0;
  uint32_t ev_off = 0;
  for (int32_t i = 0; i < n_parts; ++i) {
    const tpc_clusters& c = ev[i];
    if (c.n > 0) {
      size_t m = (size_t)c.n;
      CK(cudaMemcpyAsync(B.y + off, c.y, 4 * m, cudaMemcpyDeviceToDevice, s));
      if (mode == 0) CK(cudaMemcpyAsync(B.z + off, c.z, 4 * m, cudaMemcpyDeviceToDevice, s));
      else CK(cudaMemcpyAsync(B.t + off, c.t, 8 * m, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(B.row + off, c.row, m, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(B.sector + off, c.sector, m, cudaMemcpyDeviceToDevice, s));
      if (c.flags) CK(cudaMemcpyAsync(B.flags + off, c.flags, m, cudaMemcpyDeviceToDevice, s));
      else CK(cudaMemsetAsync(B.flags + off, 0, m, s));
      k_batch_event<<<(unsigned)((c.n + 255) / 256), 256, 0, s>>>(
          c.n, c.n_events > 1 ? c.event : nullptr, ev_off, B.event + off);
      CK(cudaGetLastError());
    }
    off += c.n;
    ev_off += (uint32_t)c.n_events;
  }
  tpc_clusters all{};
  all.n = n;
  all.mode = mode;
  all.n_events = (int32_t)n_events;
  all.tf_start = ev[0].tf_start;
  all.y = B.y;
  all.z = mode == 0 ? B.z : nullptr;
  all.t = mode == 1 ? B.t : nullptr;
  all.row = B.row;
  all.sector = B.sector;
  all.flags = B.flags;
  all.event = B.event;
  all.pads = ev[0].pads;
  tpc_status st = tpc_load_clusters(ctx, &all);
  if (st != TPC_OK) return st;
  return tpc_find_tracks(ctx, out);
}

tpc_status tpc_get_tracks(tpc_ctx* ctx, tpc_tracks* out) {
  if (!ctx || !out) return fail(ctx, TPC_ERR_ARG, "null argument");
  if (!ctx->tracks_valid) return fail(ctx, TPC_ERR_STATE, "no track set");
  tpc_status st = read_back(ctx);
  if (st != TPC_OK) return st;
  out->n_tracks = ctx->h_pinned[kCntTracks];
  out->n_assigned = ctx->h_pinned[kCntAssigned];
  out->track_start = ctx->tb.track_start;
  out->cluster_idx = ctx->tb.cluster_idx;
  out->t_coll = ctx->tb.t_coll;
  out->start_hit = ctx->tb.start_hit;
  return TPC_OK;
}

tpc_status tpc_set_tracks(tpc_ctx* ctx, const tpc_tracks* t) {
  if (ctx) ctx->rb.vz = nullptr;  // a new track set: no vertices
  if (!ctx || !t) return fail(ctx, TPC_ERR_ARG, "null argument");
  if (ctx->capturing) return fail(ctx, TPC_ERR_STATE, "tpc_set_tracks synchronises");
  if (!ctx->loaded) return fail(ctx, TPC_ERR_STATE, "no batch loaded");
  if (t->n_tracks < 0 || t->n_assigned < 0 || t->n_assigned > ctx->cl.n ||
      (t->n_tracks > 0 && (!t->track_start || !t->cluster_idx || !t->t_coll)))
    return fail(ctx, TPC_ERR_ARG, "invalid track set");
  tpc_status st = ensure_track_buffers(ctx, t->n_tracks > ctx->tb.cap_tr ? t->n_tracks : ctx->tb.cap_tr,
                                       t->n_assigned > ctx->tb.cap_asg ? t->n_assigned : ctx->tb.cap_asg);
  if (st != TPC_OK) return st;
  if (t->n_tracks > 0) {
    CK(cudaMemcpyAsync(ctx->tb.track_start, t->track_start, sizeof(uint32_t) * (t->n_tracks + 1),
                       cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->tb.cluster_idx, t->cluster_idx, sizeof(uint32_t) * t->n_assigned,
                       cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->tb.t_coll, t->t_coll, sizeof(double) * t->n_tracks,
                       cudaMemcpyDeviceToDevice, ctx->stream));
    if (t->start_hit)
      CK(cudaMemcpyAsync(ctx->tb.start_hit, t->start_hit, sizeof(uint32_t) * t->n_tracks,
                         cudaMemcpyDeviceToDevice, ctx->stream));
  }
  ctx->h_pinned[kCntTracks] = (uint32_t)t->n_tracks;
  ctx->h_pinned[kCntAssigned] = (uint32_t)t->n_assigned;
  CK(cudaMemcpyAsync(ctx->d_cnt + kCntTracks, ctx->h_pinned + kCntTracks, sizeof(uint32_t) * 2,
                     cudaMemcpyHostToDevice, ctx->stream));
  launch_set_tracks(&ctx->prof, ctx->geo, ctx->cal, ctx->cl, t->n_tracks, t->n_assigned, ctx->tb,
                    ctx->d_cnt, ctx->d_err, ctx->stream);
  CK(cudaGetLastError());
  ctx->coords_calib_version = ctx->calib_version;
  // the pinned words are read by the copy above: keep them stable
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->tracks_valid = true;
  ctx->saved = false;
  return TPC_OK;
}

tpc_status tpc_refit(tpc_ctx* ctx, int save_for_backward, float* params, float* cov, float* x,
                     float* chi2, int32_t* ndf, int32_t* status, uint8_t* rej) {
  if (!ctx) return TPC_ERR_ARG;
  if (!ctx->tracks_valid) return fail(ctx, TPC_ERR_STATE, "no track set");
  if (save_for_backward) {
    int64_t need = 3 * ctx->rb.cap_w * 20;
    if (need > ctx->cap_ckpt_alloc) {
      CK(alloc(ctx->rb.ckpt, need));
      ctx->cap_ckpt_alloc = need;
    }
    if (ctx->rb.vz && ctx->tb.cap_tr > ctx->rb.cap_vck) {
      CK(alloc(ctx->rb.vck, ctx->tb.cap_tr * 24));
      ctx->rb.cap_vck = ctx->tb.cap_tr;
    }
  }
  // the current calibration applies to the refit inputs (Sec. 4): the
  // calibrated coordinates are recomputed when it changed since the track
  // set's were
  if (ctx->coords_calib_version != ctx->calib_version) {
    launch_calib(&ctx->prof, ctx->geo, ctx->cal, ctx->cl, ctx->tb.cap_asg, ctx->tb, ctx->d_cnt,
                 ctx->d_err, ctx->stream);
    ctx->coords_calib_version = ctx->calib_version;
  }
  launch_refit(&ctx->prof, ctx->geo, ctx->prm, ctx->tb.cap_tr, ctx->d_cnt, ctx->tb, ctx->rb,
               save_for_backward != 0, params, cov, x, chi2, ndf, status, rej, ctx->d_err,
               ctx->stream);
  CK(cudaGetLastError());
  ctx->saved = save_for_backward != 0;
  ctx->saved_vz = ctx->rb.vz;
  ctx->refit_calib_version = ctx->calib_version;
  return TPC_OK;
}

tpc_status tpc_set_vertex(tpc_ctx* ctx, const float* z_vertex, float sigma) {
  if (!ctx) return TPC_ERR_ARG;
  if (ctx->capturing) return fail(ctx, TPC_ERR_STATE, "tpc_set_vertex while capturing");
  if (!z_vertex) {
    ctx->rb.vz = nullptr;
    return TPC_OK;
  }
  if (!(sigma > 0.0f)) return fail(ctx, TPC_ERR_ARG, "vertex sigma must be > 0");
  if (ctx->geo.field_on)
    return fail(ctx, TPC_ERR_ARG, "the vertex pseudo-measurement needs the uniform field");
  if (!ctx->tracks_valid) return fail(ctx, TPC_ERR_STATE, "no track set");
  ctx->rb.vz = z_vertex;
  ctx->rb.vvar = sigma * sigma;
  return TPC_OK;
}

namespace {
tpc_status ensure_merge_buffers(tpc_ctx* ctx, int64_t n_tr, int64_t n_asg) {
  MergeBuf& m = ctx->mb;
  int64_t nb = (int64_t)ctx->cl.n_events * TPC_N_SECTORS;
  if (n_tr > m.cap_tr) {
    int64_t c = n_tr + n_tr / 4 + 1024;
    CK(alloc(m.seg_ts, c + 1));
    CK(alloc(m.seg_that, c));
    CK(alloc(m.seg_hit, c));
    CK(alloc(m.info, c));
    CK(alloc(m.rows, c));
    CK(alloc(m.bk_seg, c));
    CK(alloc(m.bk_v, c));
    CK(alloc(m.bk_t, c));
    CK(alloc(m.bk_rlo, c));
    CK(alloc(m.best_in, c));
    CK(alloc(m.best_out, c));
    CK(alloc(m.next, c));
    CK(alloc(m.pairs, 32 * c + 65536));
    m.cap_pairs = 32 * c + 65536;
    if (!m.n_pairs) CK(alloc(m.n_pairs, 1));
    if (!m.n_seg) CK(alloc(m.n_seg, 1));
    CK(alloc(m.has_in, c));
    CK(alloc(m.hpos, c));
    CK(alloc(m.cpos, c));
    CK(alloc(m.blk_h, c / 1024 + 2));
    CK(alloc(m.blk_c, c / 1024 + 2));
    m.cap_tr = c;
  }
  if (n_asg > m.cap_asg) {
    int64_t c = n_asg + n_asg / 4 + 1024;
    CK(alloc(m.seg_ci, c));
    m.cap_asg = c;
  }
  if (nb > m.cap_bk) {
    CK(alloc(m.bk_cnt, nb + 1));
    CK(alloc(m.bk_fill, nb));
    CK(alloc(m.bk_cls, nb * 5));
    m.cap_bk = nb;
  }
  return TPC_OK;
}
}  // namespace

tpc_status tpc_merge_tracks_async(tpc_ctx* ctx, const float* params, const float* cov,
                                  const float* x, const int32_t* status, int32_t* next,
                                  float* link_chi2) {
  if (ctx) ctx->rb.vz = nullptr;  // a new track set: no vertices
  if (!ctx) return TPC_ERR_ARG;
  if (!ctx->tracks_valid) return fail(ctx, TPC_ERR_STATE, "no track set");
  if (!params || !cov || !x || !status) return fail(ctx, TPC_ERR_ARG, "null segment state");
  TrackBuf& t = ctx->tb;
  tpc_status st = ensure_merge_buffers(ctx, t.cap_tr, t.cap_asg);
  if (st != TPC_OK) return st;
  launch_merge(&ctx->prof, ctx->geo, ctx->prm, ctx->cal, ctx->cl, t.cap_tr, true, t, ctx->mb,
               params, cov, x, status, next, link_chi2, ctx->d_cnt, ctx->d_err, ctx->stream);
  // the merged set's calibrated coordinates (Sec. 4)
  launch_calib(&ctx->prof, ctx->geo, ctx->cal, ctx->cl, t.cap_asg, t, ctx->d_cnt, ctx->d_err,
               ctx->stream);
  CK(cudaGetLastError());
  ctx->coords_calib_version = ctx->calib_version;
  ctx->saved = false;
  return TPC_OK;
}

tpc_status tpc_merge_tracks(tpc_ctx* ctx, const float* params, const float* cov, const float* x,
                            const int32_t* status, int32_t* next, float* link_chi2,
                            tpc_tracks* out) {
  if (!ctx) return TPC_ERR_ARG;
  if (ctx->capturing) return fail(ctx, TPC_ERR_STATE, "tpc_merge_tracks synchronises");
  if (!ctx->tracks_valid) return fail(ctx, TPC_ERR_STATE, "no track set");
  ctx->rb.vz = nullptr;  // a new track set: no vertices
  tpc_status st = read_back(ctx);  // segment and cluster counts
  if (st != TPC_OK) return st;
  int64_t nt = ctx->h_pinned[kCntTracks], na = ctx->h_pinned[kCntAssigned];
  if (nt > 0 && (!params || !cov || !x || !status))
    return fail(ctx, TPC_ERR_ARG, "null segment state");
  st = ensure_merge_buffers(ctx, nt, na);
  if (st != TPC_OK) return st;
  MergeBuf& m = ctx->mb;
  TrackBuf& t = ctx->tb;
  if (nt > 0) {
    // the candidate-pair list has a capacity: when the pairs that pass the
    // prefilter exceed it, it grows and the merge runs again on the copied
    // segments
    for (int attempt = 0;; ++attempt) {
      launch_merge(&ctx->prof, ctx->geo, ctx->prm, ctx->cal, ctx->cl, nt, attempt == 0, t, m,
                   params, cov, x, status, next, link_chi2, ctx->d_cnt, ctx->d_err, ctx->stream);
      CK(cudaGetLastError());
      uint32_t np = 0;
      CK(cudaMemcpyAsync(&np, m.n_pairs, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      if ((int64_t)np <= m.cap_pairs) break;
      if (attempt > 0) return fail(ctx, TPC_ERR_CAPACITY, "merge candidate pairs overflow");
      CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), ctx->stream));  // the overflow bit
      m.cap_pairs = (int64_t)np + np / 4 + 65536;
      CK(alloc(m.pairs, m.cap_pairs));
    }
    // the merged set's calibrated coordinates (Sec. 4)
    launch_calib(&ctx->prof, ctx->geo, ctx->cal, ctx->cl, t.cap_asg, t, ctx->d_cnt, ctx->d_err,
                 ctx->stream);
    CK(cudaGetLastError());
    ctx->coords_calib_version = ctx->calib_version;
  }
  st = read_back(ctx);
  if (st != TPC_OK) return st;
  ctx->saved = false;
  if (out) {
    out->n_tracks = ctx->h_pinned[kCntTracks];
    out->n_assigned = ctx->h_pinned[kCntAssigned];
    out->track_start = t.track_start;
    out->cluster_idx = t.cluster_idx;
    out->t_coll = t.t_coll;
    out->start_hit = t.start_hit;
  }
  return TPC_OK;
}

tpc_status tpc_compress_tracks(tpc_ctx* ctx, float qy, float qz, int32_t* ry, int32_t* rz,
                               float* dy, float* dz) {
  if (!ctx) return TPC_ERR_ARG;
  if (!ctx->tracks_valid) return fail(ctx, TPC_ERR_STATE, "no track set");
  if (!ry || !rz) return fail(ctx, TPC_ERR_ARG, "null residual output");
  if (!(qy > 0.0f) || !(qz > 0.0f) || !std::isfinite(qy) || !std::isfinite(qz))
    return fail(ctx, TPC_ERR_ARG, "quantisation steps must be positive");
  launch_compress(&ctx->prof, ctx->geo, ctx->cal, ctx->cl, ctx->prm, qy, qz, ctx->tb.cap_tr,
                  ctx->d_cnt, ctx->tb, ry, rz, dy, dz, ctx->stream);
  CK(cudaGetLastError());
  return TPC_OK;
}

tpc_status tpc_refine_time(tpc_ctx* ctx, const float* params, const float* x,
                           const int32_t* status, double* t_coll_out) {
  if (!ctx) return TPC_ERR_ARG;
  if (!ctx->tracks_valid) return fail(ctx, TPC_ERR_STATE, "no track set");
  if (!params || !x || !status) return fail(ctx, TPC_ERR_ARG, "null track state");
  TrackBuf& t = ctx->tb;
  launch_refine_time(&ctx->prof, ctx->geo, ctx->cal, ctx->cl, t.cap_tr, ctx->d_cnt, t, params, x,
                     status, t_coll_out, ctx->stream);
  // the clusters' calibrated coordinates with the new times (Sec. 4)
  launch_calib(&ctx->prof, ctx->geo, ctx->cal, ctx->cl, t.cap_asg, t, ctx->d_cnt, ctx->d_err,
               ctx->stream);
  CK(cudaGetLastError());
  ctx->coords_calib_version = ctx->calib_version;
  ctx->saved = false;
  return TPC_OK;
}

tpc_status tpc_refit_backward(tpc_ctx* ctx, const float* dl_dchi2, float* grad_y, float* grad_zt,
                              double* grad_calib) {
  if (!ctx) return TPC_ERR_ARG;
  if (!ctx->saved) return fail(ctx, TPC_ERR_STATE, "refit_backward needs a saved refit");
  if (ctx->refit_calib_version != ctx->calib_version)
    return fail(ctx, TPC_ERR_STATE, "calibration changed since the saved refit");
  if (ctx->saved_vz != ctx->rb.vz)
    return fail(ctx, TPC_ERR_STATE, "vertex set or cleared since the saved refit");
  if (!dl_dchi2 || !grad_y || !grad_zt || !grad_calib)
    return fail(ctx, TPC_ERR_ARG, "null output");
  if (!ctx->part_alloc) {
    CK(alloc(ctx->rb.acc_spline, (int64_t)TPC_SPLINE_SIZE));
    CK(alloc(ctx->rb.gmax, (int64_t)1));
    CK(alloc(ctx->rb.part_cal, (int64_t)kCalibGradBlocks * 2));
    ctx->part_alloc = true;
  }
  launch_refit_backward(&ctx->prof, ctx->geo, ctx->cal, ctx->prm, ctx->cl, ctx->tb.cap_tr, ctx->tb.cap_asg,
                        ctx->d_cnt, ctx->tb, ctx->rb, dl_dchi2, grad_y, grad_zt, grad_calib,
                        ctx->stream);
  CK(cudaGetLastError());
  return TPC_OK;
}

tpc_status tpc_graph_begin(tpc_ctx* ctx) {
  if (!ctx) return TPC_ERR_ARG;
  if (ctx->capturing) return fail(ctx, TPC_ERR_STATE, "already capturing");
  if (!ctx->stream) return fail(ctx, TPC_ERR_STATE, "graph capture needs a non-default stream");
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->prof.collect();
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  ctx->capturing = true;
  g_capturing_alloc_guard = true;
  ctx->prof_was_on = ctx->prof.on;
  ctx->prof.on = false;  // no event pairs inside the graph
  ctx->launches_before = ctx->prof.launches;
  return TPC_OK;
}

tpc_status tpc_graph_end(tpc_ctx* ctx) {
  if (!ctx) return TPC_ERR_ARG;
  if (!ctx->capturing) return fail(ctx, TPC_ERR_STATE, "not capturing");
  ctx->capturing = false;
  g_capturing_alloc_guard = false;
  ctx->graph_kernels = ctx->prof.launches - ctx->launches_before;
  ctx->prof.launches = ctx->launches_before;
  ctx->prof.on = ctx->prof_was_on;
  cudaGraph_t gr = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->stream, &gr);
  if (e != cudaSuccess || !gr)
    return fail(ctx, TPC_ERR_STATE, std::string("capture failed: ") + cudaGetErrorString(e) +
                                        " (run the sequence once before capturing)");
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  ctx->graph = gr;
  ctx->graph_exec = nullptr;
  CK(cudaGraphInstantiate(&ctx->graph_exec, gr, 0));
  return TPC_OK;
}

tpc_status tpc_graph_launch(tpc_ctx* ctx) {
  if (!ctx) return TPC_ERR_ARG;
  if (!ctx->graph_exec) return fail(ctx, TPC_ERR_STATE, "no captured graph");
  CK(cudaGraphLaunch(ctx->graph_exec, ctx->stream));
  ctx->prof.launches += ctx->graph_kernels;
  return TPC_OK;
}

tpc_status tpc_sync(tpc_ctx* ctx) {
  if (!ctx) return TPC_ERR_ARG;
  return read_back(ctx);
}

tpc_status tpc_get_counts(tpc_ctx* ctx, int64_t* n_tracks, int64_t* n_assigned,
                          int64_t* n_tracklets) {
  if (!ctx) return TPC_ERR_ARG;
  tpc_status st = read_back(ctx);
  if (n_tracks) *n_tracks = ctx->h_pinned[kCntTracks];
  if (n_assigned) *n_assigned = ctx->h_pinned[kCntAssigned];
  if (n_tracklets) *n_tracklets = ctx->h_pinned[kCntStart];
  return st;
}

tpc_status tpc_get_links(tpc_ctx* ctx, int32_t* up, int32_t* dn, int32_t* upc, int32_t* dnc) {
  if (!ctx) return TPC_ERR_ARG;
  if (!ctx->tracks_valid) return fail(ctx, TPC_ERR_STATE, "run tpc_find_tracks first");
  int n = ctx->cl.n;
  int32_t* outs[4] = {up, dn, upc, dnc};
  for (int32_t* o : outs)
    if (o && n > 0) CK(cudaMemsetAsync(o, 0xff, sizeof(int32_t) * n, ctx->stream));
  launch_export_links(ctx->fb, n, ctx->K, up, dn, upc, dnc, ctx->stream);
  CK(cudaGetLastError());
  return TPC_OK;
}

tpc_status tpc_get_tracklets(tpc_ctx* ctx, int64_t n_cap, uint32_t* start_hit, int32_t* n_hits,
                             double* t_coll, int32_t* hits) {
  if (!ctx) return TPC_ERR_ARG;
  if (!ctx->tracks_valid) return fail(ctx, TPC_ERR_STATE, "run tpc_find_tracks first");
  launch_export_tracklets(ctx->fb, ctx->geo.n_rows, n_cap, ctx->d_cnt, start_hit, n_hits, t_coll,
                          hits, ctx->stream);
  CK(cudaGetLastError());
  return TPC_OK;
}

tpc_status tpc_get_calibrated(tpc_ctx* ctx, float* yc, float* zc) {
  if (!ctx) return TPC_ERR_ARG;
  if (!ctx->tracks_valid) return fail(ctx, TPC_ERR_STATE, "no track set");
  tpc_status st = read_back(ctx);
  if (st != TPC_OK) return st;
  size_t m = ctx->h_pinned[kCntAssigned];
  if (m) {
    if (yc) CK(cudaMemcpyAsync(yc, ctx->tb.yc, sizeof(float) * m, cudaMemcpyDeviceToDevice, ctx->stream));
    if (zc) CK(cudaMemcpyAsync(zc, ctx->tb.zc, sizeof(float) * m, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  return TPC_OK;
}

tpc_status tpc_get_grid(tpc_ctx* ctx, uint32_t* order, uint32_t* row_start) {
  if (!ctx) return TPC_ERR_ARG;
  if (!ctx->loaded) return fail(ctx, TPC_ERR_STATE, "no batch loaded");
  if (order && ctx->cl.n > 0)
    CK(cudaMemcpyAsync(order, ctx->fb.gorig, sizeof(uint32_t) * ctx->cl.n, cudaMemcpyDeviceToDevice,
                       ctx->stream));
  if (row_start)
    CK(cudaMemcpyAsync(row_start, ctx->fb.row_start, sizeof(uint32_t) * (ctx->K + 1),
                       cudaMemcpyDeviceToDevice, ctx->stream));
  return TPC_OK;
}

tpc_status tpc_profile(tpc_ctx* ctx, int enable) {
  if (!ctx) return TPC_ERR_ARG;
  if (ctx->capturing) return fail(ctx, TPC_ERR_STATE, "tpc_profile synchronises");
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->prof.collect();
  ctx->prof.stats.clear();
  ctx->prof.launches = 0;
  ctx->prof.on = enable != 0;
  return TPC_OK;
}

tpc_status tpc_profile_only(tpc_ctx* ctx, const char* kernel) {
  if (!ctx) return TPC_ERR_ARG;
  ctx->prof.only = kernel ? kernel : "";
  return TPC_OK;
}

tpc_status tpc_profile_read(tpc_ctx* ctx, tpc_kernel_stat* out, int32_t cap, int32_t* n_out,
                            int64_t* launches) {
  if (!ctx) return TPC_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->prof.collect();
  int32_t k = 0;
  for (auto& kv : ctx->prof.stats) {
    if (out && k < cap) {
      std::memset(out[k].name, 0, sizeof(out[k].name));
      std::strncpy(out[k].name, kv.first.c_str(), sizeof(out[k].name) - 1);
      out[k].launches = kv.second.first;
      out[k].total_ms = kv.second.second;
    }
    ++k;
  }
  if (n_out) *n_out = k;
  if (launches) *launches = ctx->prof.launches;
  return TPC_OK;
}

const char* tpc_last_error(const tpc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

}  // extern "C"

// ---------------------------------------------------------------- tuning
tpc_status tpc_get_tuning(const tpc_ctx* ctx, tpc_tuning* out) {
  if (!ctx || !out) return TPC_ERR_ARG;
  *out = ctx->tune;
  return TPC_OK;
}

tpc_status tpc_set_tuning(tpc_ctx* ctx, const tpc_tuning* in) {
  if (!ctx || !in) return fail(ctx, TPC_ERR_ARG, "null argument");
  if (ctx->capturing) return fail(ctx, TPC_ERR_STATE, "tuning changes during graph capture");
  if (!(in->grid_tau >= 0.125f && in->grid_tau <= 16.0f) || in->grid_ny_max < 1 ||
      in->grid_ny_max > 64 || !valid_block(in->tracklet_block) || in->tracklet_per_sm < 0 ||
      in->tracklet_per_sm > 64 || (in->tracklet_regs != 0 && in->tracklet_regs != 96))
    return fail(ctx, TPC_ERR_ARG, "tuning out of range");
  ctx->tune = *in;
  apply_tuning(ctx);
  return TPC_OK;
}

namespace {

// Median device time (ms) of `repeats` runs of op after one untimed run.
template <class Op>
tpc_status time_median(tpc_ctx* ctx, int repeats, Op op, float* ms_out) {
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return fail(ctx, TPC_ERR_CUDA, "event create");
  }
  std::vector<float> t;
  tpc_status st = TPC_OK;
  for (int i = 0; i <= repeats && st == TPC_OK; ++i) {
    cudaEventRecord(a, ctx->stream);
    st = op();
    cudaEventRecord(b, ctx->stream);
    if (st == TPC_OK) st = read_back(ctx);
    float ms = 0.0f;
    if (st == TPC_OK && cudaEventElapsedTime(&ms, a, b) == cudaSuccess && i > 0) t.push_back(ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != TPC_OK) return st;
  std::sort(t.begin(), t.end());
  *ms_out = t.empty() ? 0.0f : t[t.size() / 2];
  return TPC_OK;
}

}  // namespace

tpc_status tpc_autotune(tpc_ctx* ctx, int32_t repeats, tpc_tuning* out) {
  if (!ctx) return TPC_ERR_ARG;
  if (ctx->capturing) return fail(ctx, TPC_ERR_STATE, "autotune during graph capture");
  if (!ctx->loaded) return fail(ctx, TPC_ERR_STATE, "no batch loaded");
  if (repeats < 1) repeats = 3;
  if (repeats > 50) repeats = 50;
  // the tuner's own launches are not traced
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->prof.collect();
  bool prof_on = ctx->prof.on;
  int64_t launches = ctx->prof.launches;
  ctx->prof.on = false;
  // settle the tracklet capacity on this batch (one retry on overflow)
  tpc_status st = tpc_find_tracks(ctx, nullptr);
  int n_events = ctx->cl.n_events;
  auto load_find = [&]() -> tpc_status {
    tpc_status s = prepare_load(ctx, n_events);
    return s == TPC_OK ? tpc_find_tracks_async(ctx) : s;
  };
  auto find = [&]() -> tpc_status { return tpc_find_tracks_async(ctx); };
  // one parameter at a time, in pipeline order; each keeps the best so far
  const float taus[] = {0.25f, 0.5f, 1.0f, 2.0f, 4.0f};
  const int nys[] = {8, 16, 32};
  // the tracklet kernel's block size and register cap together: which block
  // size is fastest depends on the cap (the 96-register build holds 640
  // threads per SM with blocks of 64 or 128 only)
  const int blocks[] = {64, 128, 256, 64, 128};
  const int regs[] = {0, 0, 0, 96, 96};
  const int pers[] = {0, 1, 2, 4};
  tpc_tuning best = ctx->tune;
  auto trial = [&](tpc_tuning cand, int which, float* ms) -> tpc_status {
    ctx->tune = cand;
    apply_tuning(ctx);
    return which == 0 ? time_median(ctx, repeats, load_find, ms)
                      : time_median(ctx, repeats, find, ms);
  };
  for (int knob = 0; knob < 4 && st == TPC_OK; ++knob) {
    float best_ms = 0.0f;
    tpc_tuning keep = best;
    int nc = knob == 0 ? 5 : knob == 1 ? 3 : knob == 2 ? 5 : 4;
    for (int k = 0; k < nc && st == TPC_OK; ++k) {
      tpc_tuning cand = best;
      if (knob == 0) cand.grid_tau = taus[k];
      else if (knob == 1) cand.grid_ny_max = nys[k];
      else if (knob == 2) {
        cand.tracklet_block = blocks[k];
        cand.tracklet_regs = regs[k];
      } else if (knob == 3) {
        int mx = tracklet_blocks_per_sm(cand.tracklet_block, cand.tracklet_regs);
        if (pers[k] > 0 && pers[k] >= mx) continue;  // same as "as many as fit"
        cand.tracklet_per_sm = pers[k];
      }
      float ms = 0.0f;
      st = trial(cand, knob <= 1 ? 0 : 1, &ms);
      if (st == TPC_OK && (best_ms == 0.0f || ms < best_ms)) {
        best_ms = ms;
        keep = cand;
      }
    }
    best = keep;
  }
  // leave the batch loaded and found with the chosen tuning
  ctx->tune = best;
  apply_tuning(ctx);
  if (st == TPC_OK) st = prepare_load(ctx, n_events);
  if (st == TPC_OK) st = tpc_find_tracks(ctx, nullptr);
  if (st == TPC_OK) CK(cudaStreamSynchronize(ctx->stream));
  ctx->prof.on = prof_on;
  ctx->prof.launches = launches;
  if (out) *out = best;
  return st;
}
