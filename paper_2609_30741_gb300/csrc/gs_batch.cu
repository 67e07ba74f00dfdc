// Batched stereo rendering and the rasterizer autotuner (a serving mode with no
// counterpart in the paper, which renders one stereo frame at a time).
//
// A batch renders up to kRasterFrames stereo frames - scenes of different
// surfel counts and image sizes - in one call. Every frame owns a context (its
// "slot": workspace, counters, repair weights), so the per-frame stages run side
// by side: the call forks one stream per frame for preprocessing and binning,
// joins them for ONE persistent rasterizer launch over the dominant eyes of all
// frames, forks again for warp, hole classification, ROIs and the ROI binning,
// and joins for ONE persistent rasterizer launch over the ROI tiles of all
// frames. The second call with a configuration captures this fork/join DAG into
// a CUDA graph; later calls patch the poses into the per-frame FP64 set-up
// nodes and replay it. Each frame's result equals what gs_render_stereo gives
// for it alone with the same rasterizer configuration, bit for bit.
//
// The autotuner times every rasterizer configuration (tile edge, block shape,
// records per shared-memory stage) on the caller's frames and keeps the
// fastest; results are cached per (GPU, frame shapes) for the process and can
// be saved to and loaded from a text file.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "gs_context.cuh"

using namespace gs;

namespace {

constexpr int kBatchMarks = 6;

struct BatchGraph {
  bool valid;
  unsigned char key[2048];
  size_t key_len;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  cudaGraphNode_t setup[kRasterFrames];  // per frame: the FP64 set-up kernel node
  unsigned long long launches;
};

void release(BatchGraph &g) {
  if (g.valid) {
    cudaGraphExecDestroy(g.exec);
    cudaGraphDestroy(g.graph);
  }
  g.valid = false;
}

}  // namespace

struct gs_batch {
  gs_context *slot[kRasterFrames];
  int n_slots;
  cudaStream_t stream;                 // the caller's stream
  cudaStream_t cap_stream;             // internal capture origin
  cudaStream_t side[kRasterFrames];    // one per frame
  cudaEvent_t fork[3], join[kRasterFrames];
  cudaEvent_t ev[kBatchMarks];
  RasterConfig rc;
  int use_graphs, counting, profiling, nmarks;
  cudaStream_t cur;                    // where the call's main-line work goes
  int capturing;
  BatchGraph graphs[3];                // stereo, two-pass, mono
};

static gs_status bfail(int line, cudaError_t e) {
  return record_cuda_failure("gs_batch.cu", line, e != cudaSuccess ? e : cudaErrorUnknown);
}
#define BFAIL(e) bfail(__LINE__, (e))
#define BTRY(x)                                  \
  do {                                           \
    const cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) return BFAIL(e_);     \
  } while (0)

static void bmark(gs_batch *b, int k) {
  if (!b->profiling || k >= kBatchMarks) return;
  if (b->capturing) cudaEventRecordWithFlags(b->ev[k], b->cur, cudaEventRecordExternal);
  else cudaEventRecord(b->ev[k], b->cur);
  b->nmarks = k + 1 > b->nmarks ? k + 1 : b->nmarks;
}

// Every frame's stream waits for the main line; the slots' contexts are pointed
// at their streams for the enqueues that follow.
static cudaError_t fork_frames(gs_batch *b, int n, int which) {
  cudaError_t e = cudaEventRecord(b->fork[which], b->cur);
  for (int f = 0; f < n && e == cudaSuccess; ++f) {
    e = cudaStreamWaitEvent(b->side[f], b->fork[which], 0);
    b->slot[f]->stream = b->side[f];
    b->slot[f]->capturing = b->capturing;
  }
  return e;
}

static cudaError_t join_frames(gs_batch *b, int n) {
  cudaError_t e = cudaSuccess;
  for (int f = 0; f < n && e == cudaSuccess; ++f) {
    e = cudaEventRecord(b->join[f], b->side[f]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cur, b->join[f], 0);
  }
  return e;
}

struct FrameGeom {
  int W, H, sh, tx, ty;
  PoseArgs pa;
};

static FrameGeom geom(const gs_batch *b, const gs_frame &fr) {
  FrameGeom g;
  g.W = fr.intr.width;
  g.H = fr.intr.height;
  g.sh = raster_tshift(b->rc);
  g.tx = (g.W + (1 << g.sh) - 1) >> g.sh;
  g.ty = (g.H + (1 << g.sh) - 1) >> g.sh;
  g.pa = pose_args(&fr.pose_dom, &fr.pose_aff, &fr.intr, b->rc);
  return g;
}

// Stages 1-4 of every frame; two_pass: the comparator (both eyes in full).
static gs_status enqueue_batch(gs_batch *b, const gs_frame *frames, int n, const FrameGeom *g, int gap_thresh,
                               const gs_roi_params *roi, bool two_pass) {
  const float3 black = make_float3(0.f, 0.f, 0.f);
  bmark(b, 0);
  // per frame: pose set-up, both eyes' preprocessing, dominant binning
  BTRY(fork_frames(b, n, 0));
  for (int f = 0; f < n; ++f) {
    gs_context *ctx = b->slot[f];
    cudaStream_t s = ctx->stream;
    BTRY(launch_reset_counters(ctx->ws.ctr, s));
    BTRY(launch_setup_cams(g[f].pa, ctx->ws.cams, s));
    BTRY(launch_preprocess(*frames[f].scene, ctx->ws, 2, g[f].W, g[f].H, s));
    BTRY(launch_binning(ctx->ws, 0, frames[f].scene->n, g[f].tx, g[f].ty, nullptr, s,
                        g[f].pa.parallel ? kOrderUnion : kOrderOwn));
  }
  BTRY(join_frames(b, n));
  bmark(b, 1);
  // one persistent rasterizer launch over every dominant eye
  RasterTable t;
  t.n = n;
  for (int f = 0; f < n; ++f) {
    const gs_outputs &o = frames[f].out;
    t.f[f] = raster_frame(b->slot[f]->ws, 0, g[f].W, g[f].H, g[f].sh, nullptr, black, o.rgb_dom, o.depth_dom,
                          o.trans_dom, nullptr, !two_pass);
  }
  BTRY(launch_raster(t, b->rc, b->counting != 0, b->slot[0]->ws.bin[0].rqueue, b->cur));
  bmark(b, 2);
  // per frame: warp, edge ROIs, gaps, centre ROIs, repair, ROI binning (or the
  // affiliated eye's full binning for the comparator)
  BTRY(fork_frames(b, n, 1));
  for (int f = 0; f < n; ++f) {
    gs_context *ctx = b->slot[f];
    cudaStream_t s = ctx->stream;
    const gs_outputs &o = frames[f].out;
    const int order = g[f].pa.parallel ? kOrderReuse : kOrderOwn;
    if (two_pass) {
      BTRY(launch_binning(ctx->ws, 1, frames[f].scene->n, g[f].tx, g[f].ty, nullptr, s, order));
      continue;
    }
    BTRY(launch_warp_classify(ctx->ws, g[f].W, g[f].H, gap_thresh, *roi, o.rgb_dom, o.depth_dom, o.trans_dom,
                              o.rgb_aff, s));
    if (roi->repair_mode != 0) BTRY(repair_features(ctx->ws, g[f].W, g[f].H, o.rgb_aff, ctx->ws.rp_feat, s));
    if (roi->enable_center) BTRY(launch_centre_rois(ctx->ws, g[f].W, g[f].H, roi->margin, s));
    if (roi->repair_mode == 1 || roi->repair_mode == 2)
      BTRY(repair_stereo(ctx->ws, g[f].W, g[f].H, roi->gate_tau, o.rgb_aff, s, roi->repair_mode == 2));
    if (g[f].sh != 4)
      BTRY(launch_binning(ctx->ws, 1, frames[f].scene->n, g[f].tx, g[f].ty, ctx->ws.bin[1].rmask, s, order,
                          ctx->ws.tile_mask, g[f].W, g[f].H, g[f].sh));
    else
      BTRY(launch_binning(ctx->ws, 1, frames[f].scene->n, g[f].tx, g[f].ty, ctx->ws.tile_mask, s, order));
  }
  BTRY(join_frames(b, n));
  bmark(b, 3);
  // one persistent rasterizer launch over every frame's ROI tiles (or every
  // affiliated eye in full)
  for (int f = 0; f < n; ++f) {
    const Workspace &ws = b->slot[f]->ws;
    t.f[f] = two_pass ? raster_frame(ws, 1, g[f].W, g[f].H, g[f].sh, nullptr, black, frames[f].out.rgb_aff, nullptr,
                                     nullptr, nullptr, false)
                      : raster_frame(ws, 1, g[f].W, g[f].H, g[f].sh, ws.tile_mask, black, frames[f].out.rgb_aff,
                                     nullptr, nullptr, ws.cls, false);
  }
  BTRY(launch_raster(t, b->rc, b->counting != 0, b->slot[0]->ws.bin[1].rqueue, b->cur));
  bmark(b, 4);
  if (!two_pass) {
    for (int f = 0; f < n; ++f) {
      gs_context *ctx = b->slot[f];
      ctx->stream = b->cur;
      BTRY(copy_optional(ctx, &frames[f].out, g[f].W, g[f].H));
    }
  }
  bmark(b, 5);
  return GS_OK;
}

// One eye per frame in full (gs_render_mono_batch): per frame pose set-up,
// preprocessing and binning on the frame's stream, then one rasterizer launch.
static gs_status enqueue_mono(gs_batch *b, const gs_mono_frame *frames, int n, const FrameGeom *g) {
  bmark(b, 0);
  BTRY(fork_frames(b, n, 0));
  for (int f = 0; f < n; ++f) {
    gs_context *ctx = b->slot[f];
    cudaStream_t s = ctx->stream;
    BTRY(launch_reset_counters(ctx->ws.ctr, s));
    BTRY(launch_setup_cams(g[f].pa, ctx->ws.cams, s));
    BTRY(launch_preprocess(*frames[f].scene, ctx->ws, 1, g[f].W, g[f].H, s));
    BTRY(launch_binning(ctx->ws, 0, frames[f].scene->n, g[f].tx, g[f].ty, nullptr, s, kOrderOwn));
  }
  BTRY(join_frames(b, n));
  bmark(b, 1);
  RasterTable t;
  t.n = n;
  for (int f = 0; f < n; ++f) {
    const gs_mono_frame &fr = frames[f];
    t.f[f] = raster_frame(b->slot[f]->ws, 0, g[f].W, g[f].H, g[f].sh, nullptr,
                          make_float3(fr.bg[0], fr.bg[1], fr.bg[2]), fr.rgb, fr.depth, fr.trans, nullptr, false);
  }
  BTRY(launch_raster(t, b->rc, b->counting != 0, b->slot[0]->ws.bin[0].rqueue, b->cur));
  bmark(b, 2);
  return GS_OK;
}

// Direct enqueue, or capture / patch / replay of the call's graph (as the
// single-frame entry points do, with one set-up node per frame).
template <class Enqueue>
static gs_status batch_run(gs_batch *b, int kind, const KeyBuilder &kb, const FrameGeom *g, int n, Enqueue &&enq) {
  cudaStream_t saved[kRasterFrames];
  int saved_cap[kRasterFrames];
  for (int f = 0; f < n; ++f) {
    saved[f] = b->slot[f]->stream;
    saved_cap[f] = b->slot[f]->capturing;
  }
  auto restore = [&]() {
    for (int f = 0; f < n; ++f) {
      b->slot[f]->stream = saved[f];
      b->slot[f]->capturing = saved_cap[f];
    }
    b->cur = b->stream;
    b->capturing = 0;
  };
  auto direct = [&]() {
    b->cur = b->stream;
    b->capturing = 0;
    const gs_status st = enq();
    restore();
    return st;
  };
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (!b->use_graphs || cudaStreamIsCapturing(b->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone ||
      kb.len > sizeof(b->graphs[kind].key))
    return direct();
  BatchGraph &gr = b->graphs[kind];
  const bool same = gr.key_len == kb.len && memcmp(gr.key, kb.buf, kb.len) == 0;
  if (!same) {  // first call of a configuration: kernel by kernel
    release(gr);
    memcpy(gr.key, kb.buf, kb.len);
    gr.key_len = kb.len;
    return direct();
  }
  if (!gr.valid) {
    if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return BFAIL(cudaGetLastError());
    const unsigned long long l0 = g_launches;
    b->cur = b->cap_stream;
    b->capturing = 1;
    const gs_status st = enq();
    restore();
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
    gr.launches = g_launches - l0;
    g_launches = l0;
    if (st != GS_OK || e != cudaSuccess || !graph) {
      if (graph) cudaGraphDestroy(graph);
      return st != GS_OK ? st : BFAIL(e);
    }
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn ? nn : 1);
    cudaGraphGetNodes(graph, nodes.data(), &nn);
    int found = 0;
    for (int f = 0; f < n; ++f) gr.setup[f] = nullptr;
    for (size_t i = 0; i < nn; ++i) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nodes[i], &ty) != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
      cudaKernelNodeParams kp;
      if (cudaGraphKernelNodeGetParams(nodes[i], &kp) != cudaSuccess || kp.func != setup_cams_kernel_ptr()) continue;
      const CamBlock *cams = *(CamBlock *const *)kp.kernelParams[1];
      for (int f = 0; f < n; ++f)
        if (b->slot[f]->ws.cams == cams && !gr.setup[f]) {
          gr.setup[f] = nodes[i];
          ++found;
        }
    }
    const cudaError_t ie = found == n ? cudaGraphInstantiate(&gr.exec, graph, 0) : cudaErrorInvalidKernelImage;
    if (ie != cudaSuccess) {
      cudaGraphDestroy(graph);
      return BFAIL(ie);
    }
    gr.graph = graph;
    gr.valid = true;
  } else {
    for (int f = 0; f < n; ++f) {
      PoseArgs arg = g[f].pa;
      CamBlock *cams = b->slot[f]->ws.cams;
      void *args[2] = {(void *)&arg, (void *)&cams};
      cudaKernelNodeParams kp;
      memset(&kp, 0, sizeof(kp));
      kp.func = const_cast<void *>(setup_cams_kernel_ptr());
      kp.gridDim = dim3(1);
      kp.blockDim = dim3(32);
      kp.kernelParams = args;
      if (cudaGraphExecKernelNodeSetParams(gr.exec, gr.setup[f], &kp) != cudaSuccess) return BFAIL(cudaGetLastError());
    }
  }
  const cudaError_t le = cudaGraphLaunch(gr.exec, b->stream);
  g_launches += gr.launches;
  if (b->profiling) b->nmarks = kBatchMarks;
  return le == cudaSuccess ? GS_OK : BFAIL(le);
}

static gs_status check_frames(gs_batch *b, const gs_frame *frames, int n, const gs_roi_params *roi) {
  if (!frames || n <= 0 || n > b->n_slots) return GS_ERR_BAD_ARG;
  for (int f = 0; f < n; ++f) {
    gs_context *ctx = b->slot[f];
    const gs_frame &fr = frames[f];
    if (!scene_ok(ctx, fr.scene) || !intr_ok(ctx, &fr.intr) || !outputs_ok(&fr.out)) return GS_ERR_BAD_ARG;
    if (raster_tshift(b->rc) < ctx->ws.min_tshift) return GS_ERR_BAD_ARG;
    if (roi ? !paths_ok(ctx, roi) : !(ctx->ws.paths & GS_PATH_MONO)) return GS_ERR_BAD_ARG;
    if (roi && ((roi->repair_mode == 1 && !ctx->rp_loaded) || (roi->repair_mode == 2 && !ctx->rp_fp8)))
      return GS_ERR_NOT_LOADED;
  }
  return GS_OK;
}

static void key_frames(KeyBuilder &kb, gs_batch *b, int kind, const gs_frame *frames, int n, const FrameGeom *g) {
  kb.add(kind);
  kb.add(n);
  kb.add(b->rc);
  kb.add(b->counting);
  kb.add(b->profiling);
  for (int f = 0; f < n; ++f) {
    kb.add_scene(*frames[f].scene);
    kb.add(frames[f].intr.width);
    kb.add(frames[f].intr.height);
    kb.add(frames[f].out);
    kb.add(g[f].pa.parallel);
  }
}

// ---------------------------------------------------------------- tuning cache
namespace {

struct TuneEntry {
  gs_raster_config rc;
  float ms;
};

std::mutex g_tune_mu;
std::map<std::string, TuneEntry> g_tune;

std::string device_tag() {
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string name(p.name);
  for (char &c : name)
    if (c == ' ' || c == '|' || c == '\t') c = '_';
  char buf[96];
  snprintf(buf, sizeof(buf), "|sm%d%d|%dsm", p.major, p.minor, p.multiProcessorCount);
  return name + buf;
}

// Shape of a frame for the cache: image size, surfel count bucket (log2), SH degree.
std::string frame_tag(const gs_frame &fr) {
  char buf[64];
  const int n = fr.scene ? fr.scene->n : 0;
  int bucket = 0;
  while ((1LL << bucket) < (long long)n) ++bucket;
  snprintf(buf, sizeof(buf), "%dx%d:n2^%d:sh%d", fr.intr.width, fr.intr.height, bucket,
           fr.scene ? fr.scene->sh_degree : 0);
  return buf;
}

std::string tune_key(const char *mode, const gs_frame *frames, int n) {
  std::vector<std::string> tags;
  for (int f = 0; f < n; ++f) tags.push_back(frame_tag(frames[f]));
  std::sort(tags.begin(), tags.end());
  std::string k = device_tag() + "|" + mode + "|";
  for (size_t i = 0; i < tags.size(); ++i) k += (i ? "," : "") + tags[i];
  return k;
}

}  // namespace

extern "C" {

gs_status gs_batch_create(gs_batch **out, gs_context *const *slots, int n_slots, void *stream) {
  if (!out || !slots || n_slots <= 0 || n_slots > kRasterFrames) return GS_ERR_BAD_ARG;
  for (int f = 0; f < n_slots; ++f) {
    if (!slots[f]) return GS_ERR_BAD_ARG;
    for (int k = 0; k < f; ++k)
      if (slots[k] == slots[f]) return GS_ERR_BAD_ARG;  // every frame needs its own workspace
  }
  gs_batch *b = new (std::nothrow) gs_batch;
  if (!b) return GS_ERR_BAD_ARG;
  memset(b, 0, sizeof(*b));
  b->n_slots = n_slots;
  for (int f = 0; f < n_slots; ++f) b->slot[f] = slots[f];
  b->stream = (cudaStream_t)stream;
  b->cur = b->stream;
  b->use_graphs = 1;
  int msh = 4;
  for (int f = 0; f < n_slots; ++f) msh = std::max(msh, slots[f]->ws.min_tshift);
  b->rc = msh == 5 ? RasterConfig{32, 8, 128} : RasterConfig{16, 4, 128};
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  for (int f = 0; f < n_slots && e == cudaSuccess; ++f) {
    e = cudaStreamCreateWithFlags(&b->side[f], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[f], cudaEventDisableTiming);
  }
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&b->fork[k], cudaEventDisableTiming);
  for (int k = 0; k < kBatchMarks && e == cudaSuccess; ++k) e = cudaEventCreate(&b->ev[k]);
  if (e != cudaSuccess) {
    gs_batch_destroy(b);
    return BFAIL(e);
  }
  *out = b;
  return GS_OK;
}

gs_status gs_batch_destroy(gs_batch *b) {
  if (!b) return GS_ERR_BAD_ARG;
  for (int k = 0; k < 3; ++k) release(b->graphs[k]);
  for (int f = 0; f < kRasterFrames; ++f) {
    if (b->side[f]) cudaStreamDestroy(b->side[f]);
    if (b->join[f]) cudaEventDestroy(b->join[f]);
  }
  for (int k = 0; k < 3; ++k)
    if (b->fork[k]) cudaEventDestroy(b->fork[k]);
  for (int k = 0; k < kBatchMarks; ++k)
    if (b->ev[k]) cudaEventDestroy(b->ev[k]);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
  return GS_OK;
}

gs_status gs_batch_set_raster(gs_batch *b, const gs_raster_config *rc) {
  if (!b || !rc) return GS_ERR_BAD_ARG;
  const RasterConfig c{rc->tile, rc->pix, rc->batch};
  if (!raster_config_ok(c)) return GS_ERR_BAD_ARG;
  for (int f = 0; f < b->n_slots; ++f)
    if (raster_tshift(c) < b->slot[f]->ws.min_tshift) return GS_ERR_BAD_ARG;
  b->rc = c;
  return GS_OK;
}

gs_status gs_batch_get_raster(gs_batch *b, gs_raster_config *rc) {
  if (!b || !rc) return GS_ERR_BAD_ARG;
  rc->tile = b->rc.tile;
  rc->pix = b->rc.pix;
  rc->batch = b->rc.batch;
  return GS_OK;
}

gs_status gs_batch_set_graphs(gs_batch *b, int enable) {
  if (!b) return GS_ERR_BAD_ARG;
  b->use_graphs = enable ? 1 : 0;
  return GS_OK;
}

gs_status gs_batch_set_counting(gs_batch *b, int enable) {
  if (!b) return GS_ERR_BAD_ARG;
  b->counting = enable ? 1 : 0;
  return GS_OK;
}

gs_status gs_batch_set_profiling(gs_batch *b, int enable) {
  if (!b) return GS_ERR_BAD_ARG;
  b->profiling = enable ? 1 : 0;
  b->nmarks = 0;
  return GS_OK;
}

gs_status gs_batch_stage_times(gs_batch *b, float *ms, int max_stages, int *n_stages) {
  if (!b || !ms || max_stages < 0) return GS_ERR_BAD_ARG;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return BFAIL(cudaGetLastError());
  int n = b->nmarks > 1 ? b->nmarks - 1 : 0;
  if (n > max_stages) n = max_stages;
  for (int i = 0; i < n; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, b->ev[i], b->ev[i + 1]) != cudaSuccess) return BFAIL(cudaGetLastError());
    ms[i] = t;
  }
  if (n_stages) *n_stages = n;
  return GS_OK;
}

gs_status gs_batch_check(gs_batch *b, int *device_status) {
  if (!b) return GS_ERR_BAD_ARG;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return BFAIL(cudaGetLastError());
  int worst = GS_OK;
  for (int f = 0; f < b->n_slots; ++f) {
    uint32_t st = 0;
    const uint32_t zero = 0;
    if (cudaMemcpy(&st, &b->slot[f]->ws.ctr->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&b->slot[f]->ws.ctr->status, &zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess)
      return BFAIL(cudaGetLastError());
    if ((st & kStCapacity) && worst == GS_OK) worst = GS_ERR_CAPACITY;
    if ((st & kStTimeout) && worst == GS_OK) worst = GS_ERR_TIMEOUT;
  }
  if (device_status) *device_status = worst;
  return GS_OK;
}

gs_status gs_render_stereo_batch(gs_batch *b, const gs_frame *frames, int n_frames, int gap_thresh,
                                 const gs_roi_params *roi_in) {
  if (!b || !roi_ok(gap_thresh, roi_in)) return GS_ERR_BAD_ARG;
  const gs_status cs = check_frames(b, frames, n_frames, roi_in);
  if (cs != GS_OK) return cs;
  // depth_mode 2 (the previous call's range) needs a previous call on every
  // slot; until then every frame measures its own (mode 0)
  gs_roi_params rr = *roi_in;
  if (rr.depth_mode == 2)
    for (int f = 0; f < n_frames; ++f)
      if (!b->slot[f]->have_range) rr.depth_mode = 0;
  const gs_roi_params *roi = &rr;
  FrameGeom g[kRasterFrames];
  for (int f = 0; f < n_frames; ++f) g[f] = geom(b, frames[f]);
  KeyBuilder kb;
  key_frames(kb, b, 0, frames, n_frames, g);
  kb.add(gap_thresh);
  kb.add(*roi);
  const gs_status res = batch_run(b, 0, kb, g, n_frames,
                                  [&]() { return enqueue_batch(b, frames, n_frames, g, gap_thresh, roi, false); });
  if (res == GS_OK)
    for (int f = 0; f < n_frames; ++f) b->slot[f]->have_range = 1;
  return res;
}

gs_status gs_render_mono_batch(gs_batch *b, const gs_mono_frame *frames, int n_frames) {
  if (!b || !frames || n_frames <= 0 || n_frames > b->n_slots) return GS_ERR_BAD_ARG;
  FrameGeom g[kRasterFrames];
  for (int f = 0; f < n_frames; ++f) {
    gs_context *ctx = b->slot[f];
    const gs_mono_frame &fr = frames[f];
    if (!scene_ok(ctx, fr.scene) || !intr_ok(ctx, &fr.intr) || !fr.rgb) return GS_ERR_BAD_ARG;
    if (raster_tshift(b->rc) < ctx->ws.min_tshift || !(ctx->ws.paths & GS_PATH_MONO)) return GS_ERR_BAD_ARG;
    g[f].W = fr.intr.width;
    g[f].H = fr.intr.height;
    g[f].sh = raster_tshift(b->rc);
    g[f].tx = (g[f].W + (1 << g[f].sh) - 1) >> g[f].sh;
    g[f].ty = (g[f].H + (1 << g[f].sh) - 1) >> g[f].sh;
    g[f].pa = pose_args(&fr.pose, nullptr, &fr.intr, b->rc);
  }
  KeyBuilder kb;
  kb.add(2);
  kb.add(n_frames);
  kb.add(b->rc);
  kb.add(b->counting);
  kb.add(b->profiling);
  for (int f = 0; f < n_frames; ++f) {
    kb.add_scene(*frames[f].scene);
    kb.add(frames[f].intr.width);
    kb.add(frames[f].intr.height);
    kb.add(frames[f].bg);
    kb.add(frames[f].rgb);
    kb.add(frames[f].depth);
    kb.add(frames[f].trans);
  }
  return batch_run(b, 2, kb, g, n_frames, [&]() { return enqueue_mono(b, frames, n_frames, g); });
}

gs_status gs_render_two_pass_batch(gs_batch *b, const gs_frame *frames, int n_frames) {
  if (!b) return GS_ERR_BAD_ARG;
  const gs_status cs = check_frames(b, frames, n_frames, nullptr);
  if (cs != GS_OK) return cs;
  FrameGeom g[kRasterFrames];
  for (int f = 0; f < n_frames; ++f) g[f] = geom(b, frames[f]);
  KeyBuilder kb;
  key_frames(kb, b, 1, frames, n_frames, g);
  return batch_run(b, 1, kb, g, n_frames, [&]() { return enqueue_batch(b, frames, n_frames, g, 0, nullptr, true); });
}

}  // extern "C"

// ---------------------------------------------------------------- autotuner

// Times `call` (which enqueues one frame set on `s`) for each configuration that
// `apply` accepts: two untimed calls (the first enqueues kernel by kernel, the
// second captures the graph), then `reps` calls, each between CUDA events; the
// median is the configuration's time. A configuration whose calls fail or
// overflow a device buffer gets ms = -1.
template <class Apply, class Call, class Check>
static gs_status tune_loop(cudaStream_t s, int reps, int min_tshift, Apply &&apply, Call &&call, Check &&check,
                           gs_tune_result *results, int max_results, int *n_results, gs_raster_config *best,
                           float *best_ms) {
  static const int shapes[7][2] = {{8, 1}, {8, 2}, {16, 2}, {16, 4}, {32, 2}, {32, 4}, {32, 8}};
  static const int batches[4] = {32, 64, 128, 256};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return BFAIL(cudaGetLastError());
  std::vector<float> t(reps);
  int nr = 0;
  gs_raster_config win{0, 0, 0};
  float win_ms = INFINITY;
  gs_status err = GS_OK;
  for (int si = 0; si < 7 && err == GS_OK; ++si) {
    for (int bi = 0; bi < 4 && err == GS_OK; ++bi) {
      const gs_raster_config rc{shapes[si][0], shapes[si][1], batches[bi]};
      if (raster_tshift(RasterConfig{rc.tile, rc.pix, rc.batch}) < min_tshift) continue;
      if (apply(rc) != GS_OK) continue;
      float ms = -1.f;
      gs_status st = call();
      if (st == GS_OK) st = call();
      int dev = GS_OK;
      if (st == GS_OK) st = check(&dev);
      const bool ran = st == GS_OK && dev == GS_OK;  // (check clears the status it reports)
      for (int r = 0; r < reps && ran && st == GS_OK; ++r) {
        if (cudaEventRecord(e0, s) != cudaSuccess) st = BFAIL(cudaGetLastError());
        if (st == GS_OK) st = call();
        if (st == GS_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&t[r], e0, e1) != cudaSuccess))
          st = BFAIL(cudaGetLastError());
      }
      if (ran && st == GS_OK) st = check(&dev);
      if (st == GS_ERR_CUDA) err = st;  // the context is unusable: stop
      if (ran && st == GS_OK && dev == GS_OK) {
        std::sort(t.begin(), t.end());
        ms = t[reps / 2];
        if (ms < win_ms) {
          win_ms = ms;
          win = rc;
        }
      }
      if (results && nr < max_results) results[nr] = gs_tune_result{rc, ms};
      ++nr;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (n_results) *n_results = nr < max_results ? nr : max_results;
  if (err != GS_OK) return err;
  if (!(win_ms < INFINITY)) return GS_ERR_CAPACITY;  // no configuration ran
  if (best) *best = win;
  if (best_ms) *best_ms = win_ms;
  return GS_OK;
}

static bool cache_get(const std::string &k, gs_raster_config *rc, float *ms) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(k);
  if (it == g_tune.end()) return false;
  *rc = it->second.rc;
  if (ms) *ms = it->second.ms;
  return true;
}

static void cache_put(const std::string &k, const gs_raster_config &rc, float ms) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[k] = TuneEntry{rc, ms};
}

extern "C" {

static const char *tune_mode(const gs_roi_params *roi) {
  return !roi ? "two-pass" : roi->repair_mode ? "stereo-learned" : "stereo";
}

gs_status gs_autotune_batch(gs_batch *b, const gs_frame *frames, int n_frames, int gap_thresh,
                            const gs_roi_params *roi, int reps, int use_cache, gs_tune_result *results,
                            int max_results, int *n_results, gs_raster_config *best, float *best_ms) {
  if (!b || (roi && !roi_ok(gap_thresh, roi)) || reps <= 0 || reps > 1000 || max_results < 0) return GS_ERR_BAD_ARG;
  const gs_status cs = check_frames(b, frames, n_frames, roi);
  if (cs != GS_OK) return cs;
  if (n_results) *n_results = 0;
  const std::string key = tune_key(tune_mode(roi), frames, n_frames);
  gs_raster_config rc;
  float ms = -1.f;
  int msh = 0;
  for (int f = 0; f < n_frames; ++f) msh = std::max(msh, b->slot[f]->ws.min_tshift);
  if (use_cache && cache_get(key, &rc, &ms) && gs_batch_set_raster(b, &rc) == GS_OK) {
    if (best) *best = rc;
    if (best_ms) *best_ms = ms;
    return GS_OK;
  }
  const RasterConfig old = b->rc;
  const gs_status st = tune_loop(
      b->stream, reps, msh, [&](const gs_raster_config &c) { return gs_batch_set_raster(b, &c); },
      [&]() {
        return roi ? gs_render_stereo_batch(b, frames, n_frames, gap_thresh, roi)
                   : gs_render_two_pass_batch(b, frames, n_frames);
      },
      [&](int *dev) { return gs_batch_check(b, dev); }, results, max_results, n_results, &rc, &ms);
  if (st != GS_OK) {
    b->rc = old;
    return st;
  }
  gs_batch_set_raster(b, &rc);
  cache_put(key, rc, ms);
  if (best) *best = rc;
  if (best_ms) *best_ms = ms;
  return GS_OK;
}

gs_status gs_autotune_stereo(gs_context *ctx, const gs_scene *scene, const gs_pose *pose_dom, const gs_pose *pose_aff,
                             const gs_intrinsics *intr, int gap_thresh, const gs_roi_params *roi,
                             const gs_outputs *out, int reps, int use_cache, gs_tune_result *results,
                             int max_results, int *n_results, gs_raster_config *best, float *best_ms) {
  if (!ctx || !pose_dom || !pose_aff || (roi && !roi_ok(gap_thresh, roi)) || !scene_ok(ctx, scene) ||
      !intr_ok(ctx, intr) || !outputs_ok(out) || reps <= 0 || reps > 1000 || max_results < 0)
    return GS_ERR_BAD_ARG;
  if (roi ? !paths_ok(ctx, roi) : !(ctx->ws.paths & GS_PATH_MONO)) return GS_ERR_BAD_ARG;
  if (n_results) *n_results = 0;
  gs_frame fr;
  fr.scene = scene;
  fr.pose_dom = *pose_dom;
  fr.pose_aff = *pose_aff;
  fr.intr = *intr;
  fr.out = *out;
  const std::string key = tune_key(tune_mode(roi), &fr, 1);
  gs_raster_config rc;
  float ms = -1.f;
  if (use_cache && cache_get(key, &rc, &ms) && gs_context_set_raster(ctx, &rc) == GS_OK) {
    if (best) *best = rc;
    if (best_ms) *best_ms = ms;
    return GS_OK;
  }
  const RasterConfig old = ctx->rc;
  const gs_status st = tune_loop(
      ctx->stream, reps, ctx->ws.min_tshift, [&](const gs_raster_config &c) { return gs_context_set_raster(ctx, &c); },
      [&]() {
        return roi ? gs_render_stereo(ctx, scene, pose_dom, pose_aff, intr, gap_thresh, roi, out)
                   : gs_render_two_pass(ctx, scene, pose_dom, pose_aff, intr, out);
      },
      [&](int *dev) { return gs_context_check(ctx, dev); }, results, max_results, n_results, &rc, &ms);
  if (st != GS_OK) {
    ctx->rc = old;
    return st;
  }
  gs_context_set_raster(ctx, &rc);
  cache_put(key, rc, ms);
  if (best) *best = rc;
  if (best_ms) *best_ms = ms;
  return GS_OK;
}

gs_status gs_tune_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  return GS_OK;
}

gs_status gs_tune_cache_size(int *n) {
  if (!n) return GS_ERR_BAD_ARG;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  *n = (int)g_tune.size();
  return GS_OK;
}

gs_status gs_tune_cache_put(const char *key, const gs_raster_config *rc, float ms) {
  if (!key || !rc || !*key || strlen(key) > 4000) return GS_ERR_BAD_ARG;
  for (const char *c = key; *c; ++c)
    if (*c == ' ' || *c == '\n' || *c == '\t') return GS_ERR_BAD_ARG;
  if (!raster_config_ok(RasterConfig{rc->tile, rc->pix, rc->batch})) return GS_ERR_BAD_ARG;
  cache_put(key, *rc, ms);
  return GS_OK;
}

gs_status gs_tune_cache_get(const char *key, gs_raster_config *rc, float *ms) {
  if (!key || !rc) return GS_ERR_BAD_ARG;
  return cache_get(key, rc, ms) ? GS_OK : GS_ERR_NOT_LOADED;
}

// One entry per line: key tile pix batch ms.
gs_status gs_tune_cache_save(const char *path) {
  if (!path) return GS_ERR_BAD_ARG;
  FILE *fp = fopen(path, "w");
  if (!fp) return GS_ERR_BAD_ARG;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto &kv : g_tune)
    fprintf(fp, "%s %d %d %d %.6g\n", kv.first.c_str(), kv.second.rc.tile, kv.second.rc.pix, kv.second.rc.batch,
            (double)kv.second.ms);
  return fclose(fp) == 0 ? GS_OK : GS_ERR_BAD_ARG;
}

// Adds (or replaces) the entries of a saved file; a malformed line rejects the
// whole file and changes nothing.
gs_status gs_tune_cache_load(const char *path) {
  if (!path) return GS_ERR_BAD_ARG;
  FILE *fp = fopen(path, "r");
  if (!fp) return GS_ERR_BAD_ARG;
  std::vector<std::pair<std::string, TuneEntry>> got;
  char line[4200];
  bool ok = true;
  while (ok && fgets(line, sizeof(line), fp)) {
    const size_t len = strlen(line);
    if (len == 0 || (len == 1 && line[0] == '\n')) continue;
    if (line[len - 1] != '\n' && !feof(fp)) {
      ok = false;
      break;
    }
    char key[4100];
    int t = 0, p = 0, bt = 0;
    double ms = 0.0;
    char extra[2];
    if (sscanf(line, "%4099s %d %d %d %lf %1s", key, &t, &p, &bt, &ms, extra) != 5 ||
        !raster_config_ok(RasterConfig{t, p, bt})) {
      ok = false;
      break;
    }
    got.push_back({key, TuneEntry{gs_raster_config{t, p, bt}, (float)ms}});
  }
  fclose(fp);
  if (!ok) return GS_ERR_BAD_ARG;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto &kv : got) g_tune[kv.first] = kv.second;
  return GS_OK;
}

}  // extern "C"
