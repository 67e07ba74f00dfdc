// C ABI: contexts, workspace layout and the entry points of include/gs.h.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "gs_context.cuh"
#include "gs_launch.cuh"
#include "gs_sort.cuh"

namespace gs {

unsigned long long g_launches = 0;
int g_pdl = 1;

namespace {

constexpr size_t kAlign = 256;
// widest image: the binning keeps 8 warps x 4 tile rows x 2 counters per tile
// column in shared memory (128 KB at 512 tile columns, the limit)
constexpr int kMaxWidth = 8192;
constexpr int kMaxTileCols = 512;



struct Carver {
  char *base;
  size_t off = 0;
  bool dry;
  template <class T>
  T *take(size_t count) {
    off = (off + kAlign - 1) / kAlign * kAlign;
    T *p = dry ? nullptr : reinterpret_cast<T *>(base + off);
    off += sizeof(T) * (count ? count : 1);
    return p;
  }
};

void layout(const gs_limits &lim, Carver &c, Workspace &ws) {
  const size_t N = (size_t)lim.max_surfels;
  const size_t P = (size_t)lim.max_width * (size_t)lim.max_height;
  // the ROI grid (16 pixels) and the finest rasterizer grid the context serves
  const size_t roi_tiles =
      (size_t)((lim.max_width + kTile - 1) / kTile) * (size_t)((lim.max_height + kTile - 1) / kTile);
  const int msh = min_tshift(lim), mts = 1 << msh;
  const size_t rtx = (size_t)((lim.max_width + mts - 1) >> msh), rty = (size_t)((lim.max_height + mts - 1) >> msh);
  const size_t tiles = rtx * rty > roi_tiles ? rtx * rty : roi_tiles;
  const size_t I = (size_t)lim.max_instances;
  const size_t Ie[2] = {I, lim.max_instances_aff > 0 ? (size_t)lim.max_instances_aff : I};
  const int paths = lim.paths ? lim.paths : GS_PATH_ALL;
  const bool stereo = paths & GS_PATH_STEREO, reuse = paths & GS_PATH_REUSE, repair = paths & GS_PATH_REPAIR;
  const size_t table_max = tiles * bin_chunks(lim.max_surfels);
  size_t scan_n = N > P ? N : P;
  if (table_max > scan_n) scan_n = table_max;
  ws.cams = c.take<CamBlock>(1);
  ws.ctr = c.take<Counters>(1);
  for (int e = 0; e < 2; ++e) {
    ws.rec[e] = c.take<float4>(4 * N);
    ws.rect[e] = c.take<ushort4>(N);
    ws.bounds[e] = c.take<float4>(N);  // the rasterizer's per-warp culling reads them
    ws.cnt[e] = c.take<uint32_t>(N);
    ws.zkey[e] = c.take<uint32_t>(N);
  }
  ws.uval = c.take<uint32_t>(N);
  ws.bin_warp_surfels = bin_warp_surfels(lim.max_surfels);
  ws.bin_nch = bin_chunks(lim.max_surfels);
  const size_t table = tiles * ws.bin_nch;
  ws.cnt_bin = c.take<uint32_t>(lim.keep_intermediates ? N : 1);
  // a band-list entry covers at least one span of its surfel, so the spans'
  // capacity bounds the entries too
  for (int e = 0; e < 2; ++e) ws.band_pool_cap[e] = (uint32_t)(Ie[e] < 8 * N ? Ie[e] + 1024 : 8 * N + 1024);
  const size_t rs_words = radix_status_words(N);
  for (int e = 0; e < 2; ++e) {  // one binning scratch per eye
    BinScratch &b = ws.bin[e];
    for (int k = 0; k < 2; ++k) {
      b.dkey[k] = c.take<uint32_t>(N);
      b.dval[k] = c.take<uint32_t>(N);
    }
    b.ival = c.take<uint32_t>(Ie[e]);
    b.ikey = c.take<uint32_t>(lim.keep_intermediates ? Ie[e] : 1);
    b.bin_table = c.take<uint4>(table);
    b.band_pool = reinterpret_cast<BandEntry *>(c.take<char>(kBandEntryBytes * ws.band_pool_cap[e]));
    b.band_lists = c.take<uint2>(band_list_words(lim.max_surfels, (int)rty));  // the binning runs on the raster grid
    b.bin_offs = c.take<uint32_t>(table);
    b.ranges = c.take<uint2>(tiles);
    b.rmask = c.take<uint8_t>(tiles);
    b.items = c.take<uint32_t>(tiles);
    b.items16 = c.take<uint32_t>(1 + roi_tiles);
    b.lpt = c.take<uint32_t>(1 + tiles);
    b.rqueue = c.take<uint32_t>(2);
    b.mask_sat = c.take<uint32_t>((rty + 1) * (rtx + 1));
    b.mask_clip = c.take<uint16_t>(2 * rty * rtx);
    b.rs_hist = c.take<uint32_t>(2 * kRsPasses * 256);
    b.rs_status = c.take<unsigned long long>(rs_words);
    b.rs_ctl = c.take<uint32_t>(4);
    b.scan_tiles = c.take<unsigned long long>(scan_tiles(scan_n));
    ws.n_rs_status = rs_words;
    ws.n_scan_tiles = scan_tiles(scan_n);
    b.scan_ticket = c.take<uint32_t>(4);
  }
  ws.tile_mask = c.take<uint8_t>(tiles);
  ws.strip_mask = c.take<uint8_t>(tiles);
  ws.strip_rgb = c.take<float>(reuse ? 3 * P : 1);
  for (int e = 0; e < 2; ++e) {
    ws.row_off[e] = c.take<uint32_t>(N);
    ws.spans[e] = c.take<uint2>(Ie[e]);
  }
  ws.warpbuf = c.take<unsigned long long>(stereo ? P : 1);
  ws.warp_depth = c.take<float>(stereo ? P : 1);
  ws.cls = c.take<uint8_t>(stereo ? P : 1);
  ws.labels = c.take<int32_t>(stereo ? P : 1);
  ws.cc_list = c.take<uint32_t>(stereo ? P : 1);
  ws.slots = c.take<uint32_t>(stereo ? P + 1 : 1);
  ws.rects = c.take<int4>((size_t)lim.max_rects);
  ws.rp_master = c.take<float>(kRepairParams);
  ws.rp_grad = c.take<float>(kRepairParams);
  ws.rp_m = c.take<float>(kRepairParams);
  ws.rp_v = c.take<float>(kRepairParams);
  ws.rp_wpack = c.take<uint8_t>(92160);
  ws.rp_bias = c.take<float>(6 * 32);
  ws.rp_wpack8 = c.take<uint8_t>(50688);
  ws.rp_wpackT = c.take<uint8_t>(82944);
  ws.rp_sx = c.take<float>(6 * 32);
  ws.rp_sw = c.take<float>(6 * 32);
  ws.rp_amax = c.take<uint32_t>(6 * 32);
  ws.rp_feat = c.take<uint4>(repair ? P : 1);
  ws.rp_fill = c.take<float>(repair ? 3 * P : 1);
  ws.rp_gate = c.take<float>(tiles);
  ws.rp_skip = c.take<uint8_t>(tiles);
  ws.rp_list = c.take<uint32_t>(tiles);
  ws.rp_nlist = c.take<uint32_t>(1);
  ws.ssim_part = c.take<double>(ssim_partials(lim.max_width, lim.max_height));
  ws.strips = c.take<int32_t>(16);
  ws.drange = c.take<float>(2);
  ws.widths = c.take<int32_t>(4);
  ws.max_surfels = lim.max_surfels;
  ws.max_w = lim.max_width;
  ws.max_h = lim.max_height;
  ws.max_rects = lim.max_rects;
  ws.max_tiles = (int)tiles;
  ws.min_tshift = msh;
  ws.max_instances = (int64_t)I;
  ws.max_inst[0] = (int64_t)Ie[0];
  ws.max_inst[1] = (int64_t)Ie[1];
  ws.paths = paths;
  ws.max_pixels = (int64_t)P;
  ws.keep_intermediates = lim.keep_intermediates;
  ws.host_img = c.take<float>(lim.host_outputs ? 8 * P : 1);
}

bool limits_ok(const gs_limits *lim) {
  return lim && lim->max_surfels >= 0 && lim->max_width > 0 && lim->max_height > 0 && lim->max_instances > 0 &&
         lim->max_instances < (int64_t(1) << 30) && lim->max_instances_aff >= 0 &&
         lim->max_instances_aff < (int64_t(1) << 30) && lim->paths >= 0 && lim->paths <= GS_PATH_ALL &&
         lim->max_rects > 0 &&
         (int64_t)lim->max_width * lim->max_height < (int64_t(1) << 31) && lim->max_surfels < (1 << 30) &&
         lim->max_width <= kMaxWidth && lim->max_height <= kMaxWidth &&
         (lim->min_tile == 0 || lim->min_tile == 8 || lim->min_tile == 16 || lim->min_tile == 32) &&
         ((lim->max_width + (1 << min_tshift(*lim)) - 1) >> min_tshift(*lim)) <= kMaxTileCols;
}

__global__ void reset_counters_kernel(Counters *c) {
  griddep_wait();
  if (threadIdx.x == 0) {
    c->n_vis[0] = c->n_vis[1] = 0;
    c->n_inst[0] = c->n_inst[1] = 0;
    c->n_sort[0] = c->n_sort[1] = 0;
    c->n_rows[0] = c->n_rows[1] = 0;
    c->n_band[0] = c->n_band[1] = 0;
    c->n_union = 0;
    c->n_items[0] = c->n_items[1] = 0;
    c->dmin_bits = 0x7f800000u;
    c->dmax_bits = 0u;
    c->n_rects = 0;
    c->n_centre = 0;
    c->pairs[0] = c->pairs[1] = 0ull;
    c->contrib[0] = c->contrib[1] = 0ull;
  }
}

}  // namespace

// log2 of the smallest rasterizer tile edge a context is sized for (0 = 16)
int min_tshift(const gs_limits &lim) { return lim.min_tile == 8 ? 3 : lim.min_tile == 32 ? 5 : 4; }

size_t workspace_bytes(const gs_limits &lim) {
  Carver c{nullptr, 0, true};
  Workspace ws;
  layout(lim, c, ws);
  return c.off + kAlign;
}

bool carve_workspace(const gs_limits &lim, void *base, size_t bytes, Workspace *ws) {
  if (workspace_bytes(lim) > bytes + kAlign) return false;
  Carver c{reinterpret_cast<char *>(base), 0, false};
  layout(lim, c, *ws);
  return c.off <= bytes;
}

}  // namespace gs

using namespace gs;

static void release_slot(GraphSlot &g) {
  if (g.valid) {
    cudaGraphExecDestroy(g.exec);
    cudaGraphDestroy(g.graph);
  }
  g.valid = false;
}


// The CUDA error behind the last GS_ERR_CUDA of this host thread.
static thread_local cudaError_t g_last_cuda_error = cudaSuccess;
static thread_local int g_last_cuda_line = 0;
static thread_local char g_last_cuda_text[160];
static thread_local const char *g_last_cuda_file = "gs_api.cu";

static gs_status cuda_fail_at(int line, cudaError_t e) {
  g_last_cuda_error = e != cudaSuccess ? e : cudaErrorUnknown;
  g_last_cuda_line = line;
  g_last_cuda_file = "gs_api.cu";
  return GS_ERR_CUDA;
}
#define cuda_fail(e) cuda_fail_at(__LINE__, (e))

namespace gs {
gs_status record_cuda_failure(const char *file, int line, cudaError_t e) {
  cuda_fail_at(line, e);
  g_last_cuda_file = file;
  return GS_ERR_CUDA;
}
}  // namespace gs

static gs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? GS_OK : cuda_fail(e); }

namespace gs {

bool scene_ok(const gs_context *ctx, const gs_scene *sc) {
  if (!sc || sc->n < 0 || sc->n > ctx->lim.max_surfels || sc->sh_degree < 0 || sc->sh_degree > 3) return false;
  if (sc->primitive != 0 && sc->primitive != 1) return false;
  if (sc->n == 0) return true;
  if (!sc->pos || !sc->quat || !sc->scale || !sc->opacity || !sc->sh) return false;
  // float4 loads need 16-byte alignment; surfel scales are read as float2,
  // ellipsoid scales as float4
  const uintptr_t scale_align = sc->primitive ? 15 : 7;
  if (((uintptr_t)sc->pos & 15) || ((uintptr_t)sc->quat & 15) || ((uintptr_t)sc->scale & scale_align) ||
      ((uintptr_t)sc->opacity & 3))
    return false;
  if (sc->sh_degree == 3 && ((uintptr_t)sc->sh & 15)) return false;
  return true;
}

bool intr_ok(const gs_context *ctx, const gs_intrinsics *in) {
  return in && in->width > 0 && in->height > 0 && in->width <= ctx->lim.max_width &&
         in->height <= ctx->lim.max_height && in->fx > 0 && in->fy > 0 && in->width < 65536 * kTile &&
         in->height < 65536 * kTile;
}

PoseArgs pose_args(const gs_pose *a, const gs_pose *b, const gs_intrinsics *in, const RasterConfig &rc,
                   const RasterConfig *rc1) {
  PoseArgs pa;
  memset(&pa, 0, sizeof(pa));
  pa.tshift = raster_tshift(rc);
  pa.tshift1 = raster_tshift(rc1 ? *rc1 : rc);
  memcpy(pa.R[0], a->R, sizeof(double) * 9);
  memcpy(pa.t[0], a->t, sizeof(double) * 3);
  if (b) {
    memcpy(pa.R[1], b->R, sizeof(double) * 9);
    memcpy(pa.t[1], b->t, sizeof(double) * 3);
  }
  pa.neyes = b ? 2 : 1;
  pa.parallel = 0;
  if (b && memcmp(a->R, b->R, sizeof(double) * 9) == 0) {
    // baseline along the optical axis (column 2 of R)?
    double d[3], along = 0.0, len2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      d[k] = b->t[k] - a->t[k];
      along += d[k] * a->R[k * 3 + 2];
      len2 += d[k] * d[k];
    }
    pa.parallel = fabs(along) <= 1e-12 + 1e-9 * sqrt(len2) ? 1 : 0;
  }
  pa.fx = in->fx; pa.fy = in->fy; pa.cx = in->cx; pa.cy = in->cy;
  pa.W = in->width; pa.H = in->height;
  return pa;
}

// The buffers a stereo call with these parameters needs are in the workspace.
bool paths_ok(const gs_context *ctx, const gs_roi_params *roi) {
  const int p = ctx->ws.paths;
  if (!(p & GS_PATH_STEREO)) return false;
  if (roi->depth_mode == 2 && !(p & GS_PATH_REUSE)) return false;
  return roi->repair_mode == 0 || (p & GS_PATH_REPAIR);
}

bool outputs_ok(const gs_outputs *o) { return o && o->rgb_dom && o->depth_dom && o->trans_dom && o->rgb_aff; }

bool roi_ok(int gap_thresh, const gs_roi_params *roi) {
  if (!roi || gap_thresh < 0 || roi->margin < 0 || roi->samples_per_edge < 2 || roi->samples_per_edge > 1 << 20 ||
      roi->depth_mode < 0 || roi->depth_mode > 2)
    return false;
  return roi->repair_mode >= 0 && roi->repair_mode <= 3 && roi->gate_tau > 0.f && roi->gate_tau < 1.f;
}

// The optional outputs in one kernel: the class map (16 bytes at a time when
// both buffers allow it), the rectangles the frame found (not the whole
// capacity), their count and the edge widths.
__global__ void outputs_kernel(const uint8_t *__restrict__ cls, uint8_t *__restrict__ cls_out, size_t npix,
                               const int4 *__restrict__ rects, int4 *__restrict__ rects_out, uint32_t cap,
                               const Counters *__restrict__ ctr, int32_t *__restrict__ count_out,
                               const int32_t *__restrict__ widths, int32_t *__restrict__ widths_out) {
  griddep_wait();
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  if (cls_out) {
    const bool vec = (((uintptr_t)cls | (uintptr_t)cls_out) & 15u) == 0;
    const size_t nv = vec ? npix / 16 : 0;
    for (size_t i = tid; i < nv; i += stride)
      reinterpret_cast<uint4 *>(cls_out)[i] = reinterpret_cast<const uint4 *>(cls)[i];
    for (size_t i = nv * 16 + tid; i < npix; i += stride) cls_out[i] = cls[i];
  }
  const uint32_t nr = min(ctr->n_rects, cap);
  if (rects_out)
    for (size_t i = tid; i < nr; i += stride) rects_out[i] = rects[i];
  if (tid == 0 && count_out) *count_out = (int32_t)ctr->n_rects;
  if (tid < 4 && widths_out) widths_out[tid] = widths[tid];
}

cudaError_t copy_optional(gs_context *ctx, const gs_outputs *out, int W, int H) {
  if (!out->cls_aff && !out->roi_rects && !out->roi_count && !out->edge_widths) return cudaSuccess;
  const size_t npix = (size_t)W * H;
  const int64_t grid = ((int64_t)npix / 16 + 255) / 256;
  const int64_t cap = sm_grid_cap(4);
  launch_k(outputs_kernel, (unsigned)(grid < 1 ? 1 : grid > cap ? cap : grid), 256, 0, ctx->stream,
           (const uint8_t *)ctx->ws.cls, out->cls_aff, npix, (const int4 *)ctx->ws.rects,
           reinterpret_cast<int4 *>(out->roi_rects), (uint32_t)ctx->lim.max_rects, (const Counters *)ctx->ws.ctr,
           out->roi_count, (const int32_t *)ctx->ws.widths, out->edge_widths);
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_reset_counters(Counters *c, cudaStream_t s) {
  launch_k(reset_counters_kernel, 1, 32, 0, s, c);
  GS_LAUNCHED(1);
  return cudaGetLastError();
}

}  // namespace gs

extern "C" {

const char *gs_status_str(gs_status s) {
  switch (s) {
    case GS_OK: return "ok";
    case GS_ERR_BAD_ARG: return "bad argument";
    case GS_ERR_CAPACITY: return "device buffer capacity exceeded";
    case GS_ERR_TIMEOUT: return "bounded device loop gave up";
    case GS_ERR_CUDA: return "CUDA runtime error";
    case GS_ERR_WORKSPACE: return "workspace too small";
    case GS_ERR_NOT_LOADED: return "no repair network loaded";
  }
  return "unknown status";
}

unsigned long long gs_kernel_launches(void) { return g_launches; }

void gs_set_programmatic_launch(int enable) { g_pdl = enable ? 1 : 0; }
int gs_programmatic_launch(void) { return g_pdl; }

const char *gs_last_cuda_error(void) {
  snprintf(g_last_cuda_text, sizeof(g_last_cuda_text), "%s (%s:%d)", cudaGetErrorString(g_last_cuda_error),
           g_last_cuda_file, g_last_cuda_line);
  return g_last_cuda_text;
}

gs_status gs_workspace_size(const gs_limits *lim, size_t *bytes) {
  if (!limits_ok(lim) || !bytes) return GS_ERR_BAD_ARG;
  *bytes = workspace_bytes(*lim);
  return GS_OK;
}

gs_status gs_context_create(gs_context **out, const gs_limits *lim, void *workspace, size_t workspace_bytes_,
                            void *stream) {
  if (!out || !limits_ok(lim) || !workspace) return GS_ERR_BAD_ARG;
  if (((uintptr_t)workspace & 255) != 0) return GS_ERR_BAD_ARG;
  if (workspace_bytes(*lim) > workspace_bytes_) return GS_ERR_WORKSPACE;
  gs_context *ctx = new (std::nothrow) gs_context;
  if (!ctx) return GS_ERR_BAD_ARG;
  memset(ctx, 0, sizeof(*ctx));
  ctx->lim = *lim;
  ctx->stream = (cudaStream_t)stream;
  ctx->use_graphs = 1;
  ctx->rc = lim->min_tile == 32 ? RasterConfig{32, 8, 128} : RasterConfig{16, 4, 128};
  if (!carve_workspace(*lim, workspace, workspace_bytes_, &ctx->ws)) {
    delete ctx;
    return GS_ERR_WORKSPACE;
  }
  const int msh = min_tshift(*lim);
  cudaError_t e = prepare_binning((lim->max_width + (1 << msh) - 1) >> msh);
  if (e == cudaSuccess) e = prepare_repair();
  if (e == cudaSuccess) e = prepare_reproject();
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaMemsetAsync(ctx->ws.bin[k].rqueue, 0, 2 * sizeof(uint32_t), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ws.bin[k].scan_ticket, 0, 4 * sizeof(uint32_t), ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(ctx->ws.bin[k].scan_tiles, 0, sizeof(unsigned long long) * ctx->ws.n_scan_tiles, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(ctx->ws.bin[k].rs_status, 0, sizeof(unsigned long long) * ctx->ws.n_rs_status, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ws.bin[k].rs_hist, 0, sizeof(uint32_t) * kRsPasses * 256, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ws.bin[k].rs_ctl, 0, sizeof(uint32_t) * 4, ctx->stream);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ws.ctr, 0, sizeof(Counters), ctx->stream);
  if (e != cudaSuccess) {
    delete ctx;
    return cuda_fail(e);
  }
  *out = ctx;
  return GS_OK;
}

gs_status gs_context_destroy(gs_context *ctx) {
  if (!ctx) return GS_ERR_BAD_ARG;
  for (int i = 0; i < kMaxMarks; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  for (int k = 0; k < 3; ++k) release_slot(ctx->graphs[k]);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_edge) cudaEventDestroy(ctx->ev_edge);
  if (ctx->ev_strip) cudaEventDestroy(ctx->ev_strip);
  if (ctx->ev_net) cudaEventDestroy(ctx->ev_net);
  if (ctx->copy) cudaStreamDestroy(ctx->copy);
  if (ctx->rows) cudaStreamDestroy(ctx->rows);
  if (ctx->ev_rfork) cudaEventDestroy(ctx->ev_rfork);
  if (ctx->ev_rjoin) cudaEventDestroy(ctx->ev_rjoin);
  if (ctx->ev_hfork) cudaEventDestroy(ctx->ev_hfork);
  if (ctx->ev_hjoin) cudaEventDestroy(ctx->ev_hjoin);
  delete ctx;
  return GS_OK;
}

gs_status gs_context_set_profiling(gs_context *ctx, int enable) {
  if (!ctx) return GS_ERR_BAD_ARG;
  ctx->profiling = enable ? 1 : 0;
  return GS_OK;
}

gs_status gs_context_stage_times(gs_context *ctx, float *ms, int max_stages, int *n_stages) {
  if (!ctx || !ms || max_stages < 0) return GS_ERR_BAD_ARG;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_fail(cudaGetLastError());
  int n = ctx->nmarks > 1 ? ctx->nmarks - 1 : 0;
  if (n > max_stages) n = max_stages;
  for (int i = 0; i < n; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ctx->ev[i], ctx->ev[i + 1]) != cudaSuccess) return cuda_fail(cudaGetLastError());
    ms[i] = t;
  }
  if (n_stages) *n_stages = n;
  return GS_OK;
}

gs_status gs_context_set_stream(gs_context *ctx, void *stream) {
  if (!ctx) return GS_ERR_BAD_ARG;
  ctx->stream = (cudaStream_t)stream;
  return GS_OK;
}

gs_status gs_context_set_counting(gs_context *ctx, int enable) {
  if (!ctx) return GS_ERR_BAD_ARG;
  ctx->counting = enable ? 1 : 0;
  return GS_OK;
}

gs_status gs_context_usage(gs_context *ctx, gs_usage *u) {
  if (!ctx || !u) return GS_ERR_BAD_ARG;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  Counters c;
  if ((e = cudaMemcpy(&c, ctx->ws.ctr, sizeof(c), cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(e);
  for (int k = 0; k < 2; ++k) {
    u->binned[k] = c.n_vis[k];
    u->instances[k] = c.n_inst[k];
    u->spans[k] = c.n_rows[k];
    u->band_entries[k] = c.n_band[k];
  }
  return GS_OK;
}

gs_status gs_context_check(gs_context *ctx, int *device_status) {
  if (!ctx) return GS_ERR_BAD_ARG;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  uint32_t st = 0;
  e = cudaMemcpy(&st, &ctx->ws.ctr->status, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e);
  const uint32_t zero = 0;
  e = cudaMemcpy(&ctx->ws.ctr->status, &zero, sizeof(zero), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e);
  int code = GS_OK;
  if (st & kStCapacity) code = GS_ERR_CAPACITY;
  else if (st & kStTimeout) code = GS_ERR_TIMEOUT;
  if (device_status) *device_status = code;
  return GS_OK;
}

// Stage timing: with profiling on, an event is recorded on the context's stream
// at each stage boundary (slot 0 before the first kernel).
static void mark(gs_context *ctx, int slot) {
  if (!ctx->profiling || slot >= kMaxMarks) return;
  if (!ctx->ev[slot] && cudaEventCreate(&ctx->ev[slot]) != cudaSuccess) return;
  if (ctx->capturing) cudaEventRecordWithFlags(ctx->ev[slot], ctx->stream, cudaEventRecordExternal);
  else cudaEventRecord(ctx->ev[slot], ctx->stream);
  ctx->nmarks = slot + 1 > ctx->nmarks ? slot + 1 : ctx->nmarks;
}

// One eye through the persistent rasterizer (a table of one frame).
// The stream and events on which a binning computes its row spans beside its
// compaction and depth sort (created on first use); null if they cannot be.
static const SideRows *side_rows(gs_context *ctx) {
  static thread_local SideRows r;
  if (!ctx->rows || !ctx->ev_rfork || !ctx->ev_rjoin) {
    cudaError_t e = ctx->rows ? cudaSuccess : cudaStreamCreateWithFlags(&ctx->rows, cudaStreamNonBlocking);
    if (e == cudaSuccess && !ctx->ev_rfork) e = cudaEventCreateWithFlags(&ctx->ev_rfork, cudaEventDisableTiming);
    if (e == cudaSuccess && !ctx->ev_rjoin) e = cudaEventCreateWithFlags(&ctx->ev_rjoin, cudaEventDisableTiming);
    if (e != cudaSuccess) {  // the binnings then compute their spans in stream order
      cudaGetLastError();
      return nullptr;
    }
  }
  r = SideRows{ctx->rows, ctx->ev_rfork, ctx->ev_rjoin};
  return &r;
}

// One frame in the persistent rasterizer, its tiles taken longest list first.
// Tiles that read a coarser grid's lists keep their order: the four children
// of a parent share its length, and the measured gain did not pay for the sort.
static cudaError_t raster_one(gs_context *ctx, const RasterFrame &f, const RasterConfig *rc = nullptr) {
  RasterTable t;
  t.n = 1;
  t.f[0] = f;
  if (!f.rshift) {
    const cudaError_t e = launch_lpt_order(t.f[0], ctx->ws.bin[f.eye].lpt, ctx->stream);
    if (e != cudaSuccess) return e;
  }
  return launch_raster(t, rc ? *rc : ctx->rc, ctx->counting != 0, ctx->ws.bin[f.eye].rqueue, ctx->stream);
}

static gs_status render_eye_full(gs_context *ctx, const gs_scene *scene, int eye, int W, int H, float3 bg,
                                 float *rgb, float *depth, float *trans, bool stats, int slot, int order,
                                 unsigned long long *winit = nullptr) {
  const Workspace &ws = ctx->ws;
  cudaStream_t s = ctx->stream;
  const int sh = raster_tshift(ctx->rc), ts = 1 << sh;
  const int tx = (W + ts - 1) >> sh, ty = (H + ts - 1) >> sh;
  ctx->last_tiles = tx * ty;
  cudaError_t e = launch_binning(ws, eye, scene->n, tx, ty, nullptr, s, order, nullptr, 0, 0, 4, side_rows(ctx));
  if (e != cudaSuccess) return cuda_fail(e);
  mark(ctx, slot);
  RasterFrame f = raster_frame(ws, eye, W, H, sh, nullptr, bg, rgb, depth, trans, nullptr, stats);
  f.winit = winit;  // the stereo call's warp buffer, cleared pixel by pixel
  e = raster_one(ctx, f);
  mark(ctx, slot + 1);
  return cuda_status(e);
}

static gs_status begin_call(gs_context *ctx, const gs_scene *scene, const PoseArgs &pa) {
  cudaStream_t s = ctx->stream;
  ctx->nmarks = 0;
  cudaError_t e = launch_reset_counters(ctx->ws.ctr, s);
  if (e == cudaSuccess) e = launch_setup_cams(pa, ctx->ws.cams, s);
  if (e != cudaSuccess) return cuda_fail(e);
  mark(ctx, 0);  // the first stage is the preprocessing kernel alone
  e = launch_preprocess(*scene, ctx->ws, pa.neyes, pa.W, pa.H, s);
  mark(ctx, 1);
  return cuda_status(e);
}

}  // extern "C"

// ---------------------------------------------------------------- CUDA graphs
//
// Each entry point enqueues the same kernel sequence for a given scene, image
// size, output set and parameter set; only the poses (and focal lengths) change
// between frames, and they reach the device through the arguments of the FP64
// set-up kernel alone. The first call with a new configuration enqueues its
// kernels one by one (so every kernel is loaded before any capture); the second
// captures the sequence into a graph on an internal stream; later calls patch
// the set-up kernel's arguments in the instantiated graph and replay it on the
// caller's stream. When the caller's stream is itself being captured, kernels
// are enqueued directly (they become part of the caller's graph).

static bool direct_launch(gs_context *ctx) {
  if (!ctx->use_graphs) return true;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess) return true;
  return cs != cudaStreamCaptureStatusNone;
}

template <class Enqueue>
static gs_status run_graph(gs_context *ctx, int kind, const void *key, size_t key_len, const PoseArgs &pa,
                           Enqueue &&enqueue) {
  if (direct_launch(ctx)) return enqueue(pa);
  GraphSlot &g = ctx->graphs[kind];
  if (key_len > sizeof(g.key)) return enqueue(pa);
  const bool same = g.key_len == key_len && memcmp(g.key, key, key_len) == 0;
  const bool hit = g.valid && same;
  if (!same) {
    // a configuration seen for the first time runs kernel by kernel: every
    // kernel is then loaded before the next call captures the sequence
    release_slot(g);
    memcpy(g.key, key, key_len);
    g.key_len = key_len;
    return enqueue(pa);
  }
  if (!hit) {
    release_slot(g);
    if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return cuda_fail(cudaGetLastError());
    cudaStream_t user = ctx->stream;
    if (cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return cuda_fail(cudaGetLastError());
    const unsigned long long l0 = g_launches;
    ctx->stream = ctx->cap_stream;
    ctx->capturing = 1;
    const gs_status st = enqueue(pa);
    ctx->stream = user;
    ctx->capturing = 0;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    g.launches = g_launches - l0;
    g_launches = l0;
    if (st != GS_OK || e != cudaSuccess || !graph) {
      if (graph) cudaGraphDestroy(graph);
      return st != GS_OK ? st : cuda_fail(e);
    }
    // the set-up kernel node, whose arguments carry the poses
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    cudaGraphNode_t *nodes = (cudaGraphNode_t *)malloc(sizeof(cudaGraphNode_t) * (nn ? nn : 1));
    cudaGraphGetNodes(graph, nodes, &nn);
    g.setup_node = nullptr;
    for (size_t i = 0; i < nn && !g.setup_node; ++i) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
      cudaKernelNodeParams kp;
      if (cudaGraphKernelNodeGetParams(nodes[i], &kp) == cudaSuccess && kp.func == setup_cams_kernel_ptr())
        g.setup_node = nodes[i];
    }
    free(nodes);
    const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
    if (ie != cudaSuccess || !g.setup_node) {
      if (ie == cudaSuccess) cudaGraphExecDestroy(g.exec);
      cudaGraphDestroy(graph);
      return cuda_fail(ie != cudaSuccess ? ie : cudaErrorInvalidKernelImage);
    }
    g.graph = graph;
    memcpy(g.key, key, key_len);
    g.key_len = key_len;
    g.nmarks = ctx->nmarks;
    g.valid = true;
  } else {
    PoseArgs arg = pa;
    CamBlock *cams = ctx->ws.cams;
    void *args[2] = {(void *)&arg, (void *)&cams};
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.func = const_cast<void *>(setup_cams_kernel_ptr());
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = args;
    if (cudaGraphExecKernelNodeSetParams(g.exec, g.setup_node, &kp) != cudaSuccess) return cuda_fail(cudaGetLastError());
  }
  const cudaError_t le = cudaGraphLaunch(g.exec, ctx->stream);
  g_launches += g.launches;
  ctx->nmarks = g.nmarks;
  return cuda_status(le);
}


static void key_common(KeyBuilder &kb, gs_context *ctx, int kind, const gs_scene *scene, const gs_intrinsics *intr) {
  kb.add(kind);
  kb.add_scene(*scene);
  kb.add(intr->width);
  kb.add(intr->height);
  kb.add(ctx->counting);
  kb.add(ctx->profiling);
  kb.add(ctx->rc);
}

extern "C" {

gs_status gs_render_mono(gs_context *ctx, const gs_scene *scene, const gs_pose *pose, const gs_intrinsics *intr,
                         const float *bg, float *rgb, float *depth, float *trans) {
  if (!ctx || !pose || !scene_ok(ctx, scene) || !intr_ok(ctx, intr) || !rgb) return GS_ERR_BAD_ARG;
  if (!(ctx->ws.paths & GS_PATH_MONO)) return GS_ERR_BAD_ARG;
  const float3 b = bg ? make_float3(bg[0], bg[1], bg[2]) : make_float3(0.f, 0.f, 0.f);
  const PoseArgs pa = pose_args(pose, nullptr, intr, ctx->rc);
  KeyBuilder kb;
  key_common(kb, ctx, 0, scene, intr);
  kb.add(b);
  kb.add(rgb);
  kb.add(depth);
  kb.add(trans);
  return run_graph(ctx, 0, kb.buf, kb.len, pa, [&](const PoseArgs &p) -> gs_status {
    gs_status st = begin_call(ctx, scene, p);
    if (st != GS_OK) return st;
    return render_eye_full(ctx, scene, 0, intr->width, intr->height, b, rgb, depth, trans, false, 2, kOrderOwn);
  });
}

// The second stream and events of depth_mode 2 (created on first use).
static gs_status ensure_side(gs_context *ctx) {
  // each object is created once; one that failed is retried on the next call
  cudaError_t e = ctx->side ? cudaSuccess : cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
  if (e == cudaSuccess && !ctx->ev_fork) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess && !ctx->ev_edge) e = cudaEventCreateWithFlags(&ctx->ev_edge, cudaEventDisableTiming);
  if (e == cudaSuccess && !ctx->ev_strip) e = cudaEventCreateWithFlags(&ctx->ev_strip, cudaEventDisableTiming);
  if (e == cudaSuccess && !ctx->ev_net) e = cudaEventCreateWithFlags(&ctx->ev_net, cudaEventDisableTiming);
  return cuda_status(e);
}

// The copy stream and events of gs_render_stereo_host (created on first use).
static gs_status ensure_copy(gs_context *ctx) {
  cudaError_t e = ctx->copy ? cudaSuccess : cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking);
  if (e == cudaSuccess && !ctx->ev_hfork) e = cudaEventCreateWithFlags(&ctx->ev_hfork, cudaEventDisableTiming);
  if (e == cudaSuccess && !ctx->ev_hjoin) e = cudaEventCreateWithFlags(&ctx->ev_hjoin, cudaEventDisableTiming);
  return cuda_status(e);
}

// Host destinations of the two RGB images (gs_render_stereo_host), or none.
struct HostCopy {
  float *dom, *aff;
};

static gs_status stereo_impl(gs_context *ctx, const gs_scene *scene, const gs_pose *pose_dom,
                             const gs_pose *pose_aff, const gs_intrinsics *intr, int gap_thresh,
                             const gs_roi_params *roi, const gs_outputs *out, const HostCopy *hc);

gs_status gs_render_stereo(gs_context *ctx, const gs_scene *scene, const gs_pose *pose_dom, const gs_pose *pose_aff,
                           const gs_intrinsics *intr, int gap_thresh, const gs_roi_params *roi,
                           const gs_outputs *out) {
  return stereo_impl(ctx, scene, pose_dom, pose_aff, intr, gap_thresh, roi, out, nullptr);
}

static bool page_locked(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear a sticky-free error from an unknown pointer
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

gs_status gs_render_stereo_host(gs_context *ctx, const gs_scene *scene, const gs_pose *pose_dom,
                                const gs_pose *pose_aff, const gs_intrinsics *intr, int gap_thresh,
                                const gs_roi_params *roi, float *host_rgb_dom, float *host_rgb_aff) {
  if (!ctx || !ctx->lim.host_outputs || !intr_ok(ctx, intr)) return GS_ERR_BAD_ARG;
  if (!page_locked(host_rgb_dom) || !page_locked(host_rgb_aff)) return GS_ERR_BAD_ARG;
  const gs_status st = ensure_copy(ctx);
  if (st != GS_OK) return st;
  const size_t P = (size_t)intr->width * intr->height;
  float *img = ctx->ws.host_img;
  gs_outputs out{};
  out.rgb_dom = img;
  out.depth_dom = img + 3 * P;
  out.trans_dom = img + 4 * P;
  out.rgb_aff = img + 5 * P;
  const HostCopy hc{host_rgb_dom, host_rgb_aff};
  return stereo_impl(ctx, scene, pose_dom, pose_aff, intr, gap_thresh, roi, &out, &hc);
}

static gs_status stereo_impl(gs_context *ctx, const gs_scene *scene, const gs_pose *pose_dom,
                             const gs_pose *pose_aff, const gs_intrinsics *intr, int gap_thresh,
                             const gs_roi_params *roi, const gs_outputs *out, const HostCopy *hc) {
  if (!ctx || !pose_dom || !pose_aff || !roi || !scene_ok(ctx, scene) || !intr_ok(ctx, intr) || !outputs_ok(out))
    return GS_ERR_BAD_ARG;
  if (!roi_ok(gap_thresh, roi) || !paths_ok(ctx, roi)) return GS_ERR_BAD_ARG;
  if ((roi->repair_mode == 1 && !ctx->rp_loaded) || (roi->repair_mode == 2 && !ctx->rp_fp8)) return GS_ERR_NOT_LOADED;
  const int W = intr->width, H = intr->height;
  // the ROI re-render (Stage 4) runs in its own rasterizer configuration when
  // one is set. Its tile edge is also the affiliated eye's binning grid, except
  // that 16-pixel ROI tiles under a coarser dominant grid are binned on the
  // dominant grid and rendered from their parent tiles' lists (the masked
  // 16-pixel tiles, without the unmasked pixels of a coarse tile)
  const RasterConfig rc1 = ctx->has_rc_roi ? ctx->rc_roi : ctx->rc;
  const int rsh = raster_tshift(rc1), dsh = raster_tshift(ctx->rc);
  const bool parent = rsh == 4 && dsh > 4;
  const int sh = parent ? dsh : rsh, ts = 1 << sh;
  const int tx = (W + ts - 1) >> sh, ty = (H + ts - 1) >> sh;
  RasterConfig rcb = rc1;  // the ROI binning grid
  rcb.tile = ts;
  const PoseArgs pa = pose_args(pose_dom, pose_aff, intr, ctx->rc, &rcb);
  // depth_mode 2 reuses the depth range the previous stereo call measured; the
  // first call measures it (mode 0)
  gs_roi_params r = *roi;
  const bool reuse = roi->depth_mode == 2 && ctx->have_range;
  if (roi->depth_mode == 2 && !reuse) r.depth_mode = 0;
  // learned repair without the depth-range reuse: the network runs on the second
  // stream beside the ROI binning (which reads the ROI mask the network leaves
  // unchanged); the rasterizer then skips the tiles whose gate passed
  const bool net_side = (r.repair_mode == 1 || r.repair_mode == 2) && !reuse;
  if (reuse || net_side) {
    const gs_status st = ensure_side(ctx);
    if (st != GS_OK) return st;
  }
  KeyBuilder kb;
  key_common(kb, ctx, 1, scene, intr);
  kb.add(gap_thresh);
  kb.add(r);
  kb.add(*out);
  kb.add(pa.parallel);  // selects the depth-order path of the affiliated eye
  kb.add(rc1);
  kb.add(hc ? hc->dom : nullptr);  // host copies are nodes of the captured graph
  kb.add(hc ? hc->aff : nullptr);
  const gs_status res = run_graph(ctx, 1, kb.buf, kb.len, pa, [&](const PoseArgs &p) -> gs_status {
    gs_status st = begin_call(ctx, scene, p);
    if (st != GS_OK) return st;
    const float3 black = make_float3(0.f, 0.f, 0.f);
    const Workspace &ws = ctx->ws;
    cudaError_t e = cudaSuccess;
    // the affiliated eye's masked re-render: the binning grid's masked tiles, or
    // the masked 16-pixel tiles, each from its parent tile's list
    auto roi_frame = [&](const uint8_t *mask, float *rgb, uint8_t *cls) {
      RasterFrame f = raster_frame(ws, 1, W, H, sh, mask, black, rgb, nullptr, nullptr, cls, false);
      if (parent) {
        const RasterFrame fine = raster_frame(ws, 1, W, H, 4, mask, black, rgb, nullptr, nullptr, cls, false);
        f.tiles_x = fine.tiles_x;
        f.ntiles = fine.ntiles;
        f.tshift = 4;
        f.roi = nullptr;  // the listed tiles are masked whole
        f.items = ws.bin[1].items16 + 1;
        f.n_items = ws.bin[1].items16;
        f.rshift = sh - 4;
        f.rtiles_x = tx;
      }
      return f;
    };
    if (reuse) {
      // With the previous frame's depth range the edge strips (Eq. 6-8) are known
      // before the dominant eye is rendered: a second stream bins and renders the
      // affiliated eye's strip tiles (into a scratch image) while the dominant
      // eye is binned and rendered.
      cudaStream_t sd = ctx->side;
      if ((e = cudaEventRecord(ctx->ev_fork, ctx->stream)) == cudaSuccess) e = cudaStreamWaitEvent(sd, ctx->ev_fork, 0);
      if (e == cudaSuccess) e = launch_edge_roi(ws, r, ws.strip_mask, true, sd);
      if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_edge, sd);
      if (e == cudaSuccess)
        e = sh != 4 ? launch_binning(ws, 1, scene->n, tx, ty, ws.bin[1].rmask, sd, kOrderOwn, ws.strip_mask, W, H, sh)
                    : launch_binning(ws, 1, scene->n, tx, ty, ws.strip_mask, sd, kOrderOwn);
      if (e == cudaSuccess) {
        RasterTable t;
        t.n = 1;
        t.f[0] = roi_frame(ws.strip_mask, ws.strip_rgb, nullptr);
        e = launch_raster(t, rc1, ctx->counting != 0, ws.bin[1].rqueue, sd);
      }
      if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_strip, sd);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    // Stage 1: dominant eye, RGB + depth proxy (+ the per-frame depth range)
    // without a reused depth range the dominant eye's rasterizer also clears the
    // warp buffer (the two eyes share the image size)
    st = render_eye_full(ctx, scene, 0, W, H, black, out->rgb_dom, out->depth_dom, out->trans_dom, true, 2,
                         p.parallel ? kOrderUnion : kOrderOwn, reuse ? nullptr : ws.warpbuf);
    if (st != GS_OK) return st;
    if (hc) {  // the dominant eye is final: copy it out beside Stages 2-4
      if ((e = cudaEventRecord(ctx->ev_hfork, ctx->stream)) == cudaSuccess)
        e = cudaStreamWaitEvent(ctx->copy, ctx->ev_hfork, 0);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(hc->dom, out->rgb_dom, sizeof(float) * 3 * (size_t)W * H, cudaMemcpyDeviceToHost,
                            ctx->copy);
      if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_hjoin, ctx->copy);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    // Stages 2-3: warp, edge ROIs, gaps
    if (reuse) {
      e = launch_warp(ws, W, H, out->depth_dom, out->trans_dom, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->ev_edge, 0);
      if (e == cudaSuccess) e = launch_classify(ws, W, H, gap_thresh, r, out->rgb_dom, out->rgb_aff, ctx->stream);
    } else {
      e = launch_warp_classify(ws, W, H, gap_thresh, r, out->rgb_dom, out->depth_dom, out->trans_dom, out->rgb_aff,
                               ctx->stream, true);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    if (r.repair_mode != 0) {  // the repair network's inputs, kept for gs_repair_features
      if ((e = repair_features(ws, W, H, out->rgb_aff, ws.rp_feat, ctx->stream)) != cudaSuccess) return cuda_fail(e);
    }
    mark(ctx, 4);
    // Step 2: connected centre holes -> ROIs
    if (r.enable_center) {
      if ((e = launch_centre_rois(ws, W, H, r.margin, ctx->stream)) != cudaSuccess) return cuda_fail(e);
    }
    // learned repair: tiles with holes whose gate passes take the network fill
    // and leave the ROI tile mask
    if (net_side) {
      if ((e = cudaEventRecord(ctx->ev_fork, ctx->stream)) == cudaSuccess)
        e = cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
      if (e == cudaSuccess)
        e = repair_stereo(ws, W, H, r.gate_tau, out->rgb_aff, ctx->side, r.repair_mode == 2, ws.rp_skip);
      if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_net, ctx->side);
      if (e != cudaSuccess) return cuda_fail(e);
    } else if (r.repair_mode == 1 || r.repair_mode == 2) {
      if ((e = repair_stereo(ws, W, H, r.gate_tau, out->rgb_aff, ctx->stream, r.repair_mode == 2)) != cudaSuccess)
        return cuda_fail(e);
    }
    if (reuse) {  // the strip tiles are rendered already
      const int rtiles = ((W + kTile - 1) / kTile) * ((H + kTile - 1) / kTile);
      if ((e = cudaStreamWaitEvent(ctx->stream, ctx->ev_strip, 0)) == cudaSuccess)
        e = launch_mask_minus(ws.tile_mask, ws.strip_mask, rtiles, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    mark(ctx, 5);
    // Stage 4: targeted re-rasterisation of the ROI tiles of the affiliated eye
    // (the ROI mask lives on the 16-pixel grid; other tile edges bin on a copy
    // on their own grid)
    ctx->last_tiles = tx * ty;
    const int aorder = p.parallel ? kOrderReuse : kOrderOwn;
    // (with depth_mode 2 the strip binning of this eye ran on the second stream:
    // its spans stay in stream order)
    const SideRows *sr = reuse ? nullptr : side_rows(ctx);
    e = sh != 4 ? launch_binning(ws, 1, scene->n, tx, ty, ws.bin[1].rmask, ctx->stream, aorder, ws.tile_mask, W, H, sh,
                                 sr)
                : launch_binning(ws, 1, scene->n, tx, ty, ws.tile_mask, ctx->stream, aorder, nullptr, 0, 0, 4, sr);
    if (e != cudaSuccess) return cuda_fail(e);
    mark(ctx, 6);
    RasterFrame rf = roi_frame(ws.tile_mask, out->rgb_aff, ws.cls);
    if (net_side) {  // join the network; its gated tiles keep the fill
      if ((e = cudaStreamWaitEvent(ctx->stream, ctx->ev_net, 0)) != cudaSuccess) return cuda_fail(e);
      rf.skip = ws.rp_skip;
    }
    e = raster_one(ctx, rf, &rc1);
    if (e == cudaSuccess && reuse) e = launch_strip_composite(ws, W, H, ws.strip_rgb, out->rgb_aff, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    mark(ctx, 7);
    e = copy_optional(ctx, out, W, H);
    if (e == cudaSuccess && hc) {  // the affiliated eye, then join the dominant eye's copy
      e = cudaMemcpyAsync(hc->aff, out->rgb_aff, sizeof(float) * 3 * (size_t)W * H, cudaMemcpyDeviceToHost,
                          ctx->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->ev_hjoin, 0);
    }
    mark(ctx, 8);
    return cuda_status(e);
  });
  if (res == GS_OK) ctx->have_range = 1;
  return res;
}

gs_status gs_render_two_pass(gs_context *ctx, const gs_scene *scene, const gs_pose *pose_dom,
                             const gs_pose *pose_aff, const gs_intrinsics *intr, const gs_outputs *out) {
  if (!ctx || !pose_dom || !pose_aff || !scene_ok(ctx, scene) || !intr_ok(ctx, intr) || !outputs_ok(out))
    return GS_ERR_BAD_ARG;
  if (!(ctx->ws.paths & GS_PATH_MONO)) return GS_ERR_BAD_ARG;
  const int W = intr->width, H = intr->height;
  const PoseArgs pa = pose_args(pose_dom, pose_aff, intr, ctx->rc);
  KeyBuilder kb;
  key_common(kb, ctx, 2, scene, intr);
  kb.add(*out);
  kb.add(pa.parallel);
  return run_graph(ctx, 2, kb.buf, kb.len, pa, [&](const PoseArgs &p) -> gs_status {
    gs_status st = begin_call(ctx, scene, p);
    if (st != GS_OK) return st;
    const float3 black = make_float3(0.f, 0.f, 0.f);
    st = render_eye_full(ctx, scene, 0, W, H, black, out->rgb_dom, out->depth_dom, out->trans_dom, false, 2,
                         p.parallel ? kOrderUnion : kOrderOwn);
    if (st != GS_OK) return st;
    return render_eye_full(ctx, scene, 1, W, H, black, out->rgb_aff, nullptr, nullptr, false, 4,
                           p.parallel ? kOrderReuse : kOrderOwn);
  });
}

gs_status gs_context_set_raster(gs_context *ctx, const gs_raster_config *rc) {
  if (!ctx || !rc) return GS_ERR_BAD_ARG;
  const RasterConfig c{rc->tile, rc->pix, rc->batch};
  if (!raster_config_ok(c) || raster_tshift(c) < ctx->ws.min_tshift) return GS_ERR_BAD_ARG;
  ctx->rc = c;
  return GS_OK;
}

gs_status gs_context_set_raster_roi(gs_context *ctx, const gs_raster_config *rc) {
  if (!ctx) return GS_ERR_BAD_ARG;
  if (!rc) {
    ctx->has_rc_roi = 0;
    return GS_OK;
  }
  const RasterConfig c{rc->tile, rc->pix, rc->batch};
  if (!raster_config_ok(c) || raster_tshift(c) < ctx->ws.min_tshift) return GS_ERR_BAD_ARG;
  ctx->rc_roi = c;
  ctx->has_rc_roi = 1;
  return GS_OK;
}

gs_status gs_context_get_raster_roi(gs_context *ctx, gs_raster_config *rc, int *is_set) {
  if (!ctx || !rc) return GS_ERR_BAD_ARG;
  const RasterConfig &c = ctx->has_rc_roi ? ctx->rc_roi : ctx->rc;
  rc->tile = c.tile;
  rc->pix = c.pix;
  rc->batch = c.batch;
  if (is_set) *is_set = ctx->has_rc_roi;
  return GS_OK;
}

gs_status gs_context_get_raster(gs_context *ctx, gs_raster_config *rc) {
  if (!ctx || !rc) return GS_ERR_BAD_ARG;
  rc->tile = ctx->rc.tile;
  rc->pix = ctx->rc.pix;
  rc->batch = ctx->rc.batch;
  return GS_OK;
}

gs_status gs_ssim(gs_context *ctx, const float *img, const float *ref, int width, int height, int channels,
                  float *ssim) {
  if (!ctx || !img || !ref || !ssim || width <= 0 || height <= 0 || width > ctx->lim.max_width ||
      height > ctx->lim.max_height || channels < 1 || channels > 3)
    return GS_ERR_BAD_ARG;
  return cuda_status(launch_ssim(img, ref, width, height, channels, ctx->ws.ssim_part, ssim, ctx->stream));
}

gs_status gs_centre_rois(gs_context *ctx, const uint8_t *cls, int width, int height, int margin, int32_t *rects,
                         int32_t *count, uint8_t *tile_mask) {
  if (!ctx || !cls || !rects || !count || width <= 0 || height <= 0 || width > ctx->lim.max_width ||
      height > ctx->lim.max_height || margin < 0)
    return GS_ERR_BAD_ARG;
  if (!(ctx->ws.paths & GS_PATH_STEREO)) return GS_ERR_BAD_ARG;
  const Workspace &ws = ctx->ws;
  // without a caller mask the tiles land in the workspace's ROI mask
  cudaError_t e = launch_centre_rois_of(ws, cls, width, height, margin, tile_mask ? tile_mask : ws.tile_mask,
                                        ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(rects, ws.rects, sizeof(int4) * (size_t)ws.max_rects, cudaMemcpyDeviceToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(count, &ws.ctr->n_rects, sizeof(uint32_t), cudaMemcpyDeviceToDevice, ctx->stream);
  return cuda_status(e);
}

gs_status gs_context_set_graphs(gs_context *ctx, int enable) {
  if (!ctx) return GS_ERR_BAD_ARG;
  ctx->use_graphs = enable ? 1 : 0;
  return GS_OK;
}

gs_status gs_context_buffer(gs_context *ctx, int which, void **dev_ptr, size_t *bytes, int64_t *count) {
  if (!ctx || !dev_ptr) return GS_ERR_BAD_ARG;
  const Workspace &ws = ctx->ws;
  const size_t N = (size_t)ws.max_surfels, P = (size_t)ws.max_pixels;
  Counters c;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_fail(cudaGetLastError());
  if (cudaMemcpy(&c, ws.ctr, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return cuda_fail(cudaGetLastError());
  void *p = nullptr;
  size_t b = 0;
  int64_t n = -1;
  const int nt = ws.max_tiles;
  const int eye = (which & GS_BUF_EYE1) ? 1 : 0;
  // the last binning is the affiliated eye's when it ran, else the dominant eye's
  const int last = c.n_vis[1] || c.n_inst[1] ? 1 : 0;
  const size_t I = (size_t)ws.max_inst[last];
  switch (which & ~GS_BUF_EYE1) {
    case GS_BUF_RECORDS: p = ws.rec[eye]; b = 64 * N; n = (int64_t)N; break;
    case GS_BUF_RECTS: p = ws.rect[eye]; b = 8 * N; n = (int64_t)N; break;
    case GS_BUF_BOUNDS: p = ws.bounds[eye]; b = 16 * N; n = (int64_t)N; break;
    case GS_BUF_COUNTS: p = ws.cnt[eye]; b = 4 * N; n = (int64_t)N; break;
    case GS_BUF_DEPTH_ORDER: p = ws.bin[last].dval[0]; b = 4 * N; n = c.n_vis[last]; break;
    case GS_BUF_INST_KEYS:
      if (!ws.keep_intermediates) return GS_ERR_BAD_ARG;
      p = ws.bin[last].ikey; b = 4 * I; n = c.n_sort[last]; break;
    case GS_BUF_INST_VALS: p = ws.bin[last].ival; b = 4 * I; n = c.n_sort[last]; break;
    case GS_BUF_RANGES: p = ws.bin[last].ranges; b = 8 * (size_t)nt; n = nt; break;
    case GS_BUF_WARP:
      if (!(ws.paths & GS_PATH_STEREO)) return GS_ERR_BAD_ARG;
      p = ws.warpbuf; b = 8 * P; n = (int64_t)P; break;
    case GS_BUF_TILE_MASK: p = ws.tile_mask; b = (size_t)nt; n = nt; break;
    case GS_BUF_DEPTH_RANGE: p = ws.drange; b = 8; n = 2; break;
    case GS_BUF_STRIPS: p = ws.strips; b = 64; n = 16; break;
    case GS_BUF_WARP_DEPTH:
      if (!(ws.paths & GS_PATH_STEREO)) return GS_ERR_BAD_ARG;
      p = ws.warp_depth; b = 4 * P; n = (int64_t)P; break;
    case GS_BUF_PAIRS: p = &ws.ctr->pairs[0]; b = 32; n = 4; break;
    case GS_BUF_BIN_COUNTS:
      if (!ws.keep_intermediates) return GS_ERR_BAD_ARG;
      p = ws.cnt_bin; b = 4 * N; n = (int64_t)N; break;
    default: return GS_ERR_BAD_ARG;
  }
  *dev_ptr = p;
  if (bytes) *bytes = b;
  if (count) *count = n;
  return GS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- learned repair
extern "C" {

gs_status gs_repair_load(gs_context *ctx, const float *weights, int64_t count) {
  if (!ctx || !weights || count != kRepairParams) return GS_ERR_BAD_ARG;
  const Workspace &ws = ctx->ws;
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(ws.rp_master, weights, sizeof(float) * kRepairParams, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws.rp_m, 0, sizeof(float) * kRepairParams, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws.rp_v, 0, sizeof(float) * kRepairParams, s);
  if (e == cudaSuccess) e = repair_pack(ws, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host array may go away after the call
  if (e != cudaSuccess) return cuda_fail(e);
  ctx->rp_loaded = 1;
  ctx->rp_fp8 = 0;  // the FP8 image belongs to the previous weights
  ctx->rp_step = 0;
  return GS_OK;
}

gs_status gs_repair_steps(gs_context *ctx, int *steps) {
  if (!ctx || !steps) return GS_ERR_BAD_ARG;
  if (!ctx->rp_loaded) return GS_ERR_NOT_LOADED;
  *steps = ctx->rp_step;
  return GS_OK;
}

gs_status gs_repair_load_state(gs_context *ctx, const float *weights, const float *m, const float *v, int64_t count,
                               int steps) {
  if (!ctx || !weights || !m || !v || count != kRepairParams || steps < 0) return GS_ERR_BAD_ARG;
  const Workspace &ws = ctx->ws;
  cudaStream_t s = ctx->stream;
  const size_t bytes = sizeof(float) * kRepairParams;
  cudaError_t e = cudaMemcpyAsync(ws.rp_master, weights, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ws.rp_m, m, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ws.rp_v, v, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = repair_pack(ws, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host arrays may go away after the call
  if (e != cudaSuccess) return cuda_fail(e);
  ctx->rp_loaded = 1;
  ctx->rp_fp8 = 0;
  ctx->rp_step = steps;
  return GS_OK;
}

gs_status gs_repair_read(gs_context *ctx, int which, float *out, int64_t count) {
  if (!ctx || !out || count != kRepairParams || which < 0 || which > 3) return GS_ERR_BAD_ARG;
  if (!ctx->rp_loaded) return GS_ERR_NOT_LOADED;
  const float *src = which == 0 ? ctx->ws.rp_master : which == 1 ? ctx->ws.rp_grad : which == 2 ? ctx->ws.rp_m
                                                                                                : ctx->ws.rp_v;
  cudaError_t e = cudaMemcpyAsync(out, src, sizeof(float) * kRepairParams, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  return cuda_status(e);
}

gs_status gs_repair_features(gs_context *ctx, int width, int height, uint16_t *feat) {
  if (!ctx || !feat || width <= 0 || height <= 0 || width > ctx->lim.max_width || height > ctx->lim.max_height ||
      ((uintptr_t)feat & 15) || !(ctx->ws.paths & GS_PATH_REPAIR))
    return GS_ERR_BAD_ARG;
  return cuda_status(cudaMemcpyAsync(feat, ctx->ws.rp_feat, (size_t)width * height * 16, cudaMemcpyDeviceToDevice,
                                     ctx->stream));
}

gs_status gs_repair_infer(gs_context *ctx, const uint16_t *feat, int frames, int width, int height,
                          const uint32_t *tiles, int n_tiles, float *fill, float *gate, int fp8) {
  if (!ctx || !feat || !tiles || !gate || frames <= 0 || frames > 255 || width <= 0 || height <= 0 ||
      width > 4095 * 16 || height > 4095 * 16 || n_tiles < 0 || ((uintptr_t)feat & 15) || (fp8 != 0 && fp8 != 1))
    return GS_ERR_BAD_ARG;
  if (!ctx->rp_loaded || (fp8 && !ctx->rp_fp8)) return GS_ERR_NOT_LOADED;
  return cuda_status(repair_forward(ctx->ws, (const uint4 *)feat, width, height, tiles, nullptr, (uint32_t)n_tiles,
                                    fill, gate, nullptr, nullptr, ctx->stream, fp8 != 0, nullptr));
}

gs_status gs_repair_calibrate_fp8(gs_context *ctx, const uint16_t *feat, int frames, int width, int height,
                                  const uint32_t *tiles, int n_tiles) {
  if (!ctx || !feat || !tiles || frames <= 0 || frames > 255 || width <= 0 || height <= 0 || width > 4095 * 16 ||
      height > 4095 * 16 || n_tiles <= 0 || ((uintptr_t)feat & 15) || (int64_t)n_tiles > 3 * ctx->ws.max_pixels ||
      !(ctx->ws.paths & GS_PATH_REPAIR))
    return GS_ERR_BAD_ARG;
  if (!ctx->rp_loaded) return GS_ERR_NOT_LOADED;
  cudaError_t e = repair_calibrate_fp8(ctx->ws, (const uint4 *)feat, width, height, tiles, (uint32_t)n_tiles,
                                       ctx->ws.rp_fill, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  ctx->rp_fp8 = 1;
  return GS_OK;
}

gs_status gs_repair_read_fp8_scales(gs_context *ctx, float *out) {
  if (!ctx || !out) return GS_ERR_BAD_ARG;
  if (!ctx->rp_fp8) return GS_ERR_NOT_LOADED;
  cudaError_t e = cudaMemcpyAsync(out, ctx->ws.rp_sx, sizeof(float) * 6 * 32, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out + 6 * 32, ctx->ws.rp_sw, sizeof(float) * 6 * 32, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  return cuda_status(e);
}

gs_status gs_repair_train_scratch_size(int n_tiles, size_t *bytes) {
  if (n_tiles <= 0 || !bytes) return GS_ERR_BAD_ARG;
  *bytes = repair_train_scratch_bytes(n_tiles);
  return GS_OK;
}

gs_status gs_repair_train_step(gs_context *ctx, const gs_repair_batch *b, const gs_adamw *opt, float *loss) {
  if (!ctx || !b || !opt || !b->feat || !b->target || !b->plain || !b->tiles || !b->scratch || b->n_tiles <= 0 ||
      b->frames <= 0 || b->frames > 255 || b->width <= 0 || b->height <= 0 || b->width > 4095 * 16 ||
      b->height > 4095 * 16 || ((uintptr_t)b->feat & 15) || !(opt->lr >= 0.f))
    return GS_ERR_BAD_ARG;
  if (!ctx->rp_loaded) return GS_ERR_NOT_LOADED;
  RepairBatch rb{(const uint4 *)b->feat, b->target, b->plain, b->width, b->height, b->tiles, b->n_tiles, b->scratch};
  if (opt->lr > 0.f) {
    ++ctx->rp_step;
    ctx->rp_fp8 = 0;  // the weights change; the FP8 image needs a new calibration
  }
  RepairOpt ro{opt->lr, opt->beta1, opt->beta2, opt->eps, opt->weight_decay, opt->gate_weight,
               ctx->rp_step > 0 ? ctx->rp_step : 1};
  return cuda_status(repair_train_step(ctx->ws, rb, ro, loss, ctx->stream));
}

}  // extern "C"
