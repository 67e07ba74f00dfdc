// Internal: the context object behind gs_context and the host helpers that the
// entry points of gs_api.cu and gs_batch.cu share.
#pragma once

#include "gs_internal.cuh"

constexpr int kMaxMarks = 16;

// One captured kernel sequence per entry point.
struct GraphSlot {
  bool valid;
  unsigned char key[512];
  size_t key_len;
  cudaGraph_t graph;             // kept alive: setup_node belongs to it
  cudaGraphExec_t exec;
  cudaGraphNode_t setup_node;
  unsigned long long launches;  // kernels in the graph
  int nmarks;
};

struct gs_context {
  gs::Workspace ws;
  gs_limits lim;
  cudaStream_t stream;
  int counting;
  int last_tiles;  // tile count of the last binning (selects the sorted buffer)
  int profiling;
  int nmarks;
  cudaEvent_t ev[kMaxMarks];
  int use_graphs;
  int capturing;
  cudaStream_t cap_stream;
  GraphSlot graphs[3];  // mono, stereo, two-pass
  gs::RasterConfig rc;  // persistent rasterizer: tile edge, pixels per thread, records per stage
  gs::RasterConfig rc_roi;  // the ROI re-render's (Stage 4), when has_rc_roi
  int has_rc_roi;
  int rp_loaded;        // repair network weights present
  int rp_fp8;           // FP8 scales and weights calibrated for the current weights
  int rp_step;          // AdamW steps taken
  int have_range;       // a stereo call has measured a depth range (depth_mode 2 can reuse it)
  cudaStream_t side;    // second stream of a stereo call with depth_mode 2
  cudaEvent_t ev_fork, ev_edge, ev_strip;
  cudaEvent_t ev_net;    // learned repair on the second stream: the network is done
  cudaStream_t copy;    // gs_render_stereo_host: the dominant eye's copy to the host
  cudaStream_t rows;    // the binnings' row spans beside their compaction and sort
  cudaEvent_t ev_rfork, ev_rjoin;
  cudaEvent_t ev_hfork, ev_hjoin;
};

namespace gs {

// Byte key of everything a captured sequence depends on besides the poses.
struct KeyBuilder {
  unsigned char buf[2048];
  size_t len = 0;
  template <class T>
  void add(const T &v) {
    if (len + sizeof(T) <= sizeof(buf)) memcpy(buf + len, &v, sizeof(T));
    len += sizeof(T);
  }
  // field by field: the struct's tail padding is not part of the key
  void add_scene(const gs_scene &s) {
    add(s.pos); add(s.quat); add(s.scale); add(s.opacity); add(s.sh);
    add(s.n); add(s.sh_degree); add(s.primitive);
  }
};

bool scene_ok(const gs_context *ctx, const gs_scene *sc);
bool intr_ok(const gs_context *ctx, const gs_intrinsics *in);
bool outputs_ok(const gs_outputs *o);
// gs_roi_params and gap threshold of a stereo call (not the repair weights)
bool roi_ok(int gap_thresh, const gs_roi_params *roi);
bool paths_ok(const gs_context *ctx, const gs_roi_params *roi);
PoseArgs pose_args(const gs_pose *a, const gs_pose *b, const gs_intrinsics *in, const RasterConfig &rc,
                   const RasterConfig *rc1 = nullptr);
cudaError_t launch_reset_counters(Counters *c, cudaStream_t s);
// Copies the optional stereo outputs (class map, ROI rectangles, counts) on ctx->stream.
cudaError_t copy_optional(gs_context *ctx, const gs_outputs *out, int W, int H);
int min_tshift(const gs_limits &lim);

}  // namespace gs
