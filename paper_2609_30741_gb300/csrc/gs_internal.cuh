// Internal declarations shared by the CUDA translation units of the renderer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

namespace gs {

// ROI grid: the ROI generator aligns its rectangles to 16x16 tiles (Sec. 3.5),
// whatever tile edge the rasterizer runs with (8, 16 or 32 pixels).
constexpr int kTile = 16;
constexpr float kZNear = 0.2f;       // near plane, metres
constexpr float kAlphaMax = 0.99f;   // alpha clamp
constexpr float kTMin = 1e-4f;       // transmittance stop
// log2(1/255): a contribution with log2(o * Ghat) below this is skipped
constexpr float kLog2AlphaMin = -7.9943534368588579f;
// -log2(e) / 2: Ghat = exp(-rho / 2) = 2^(rho * kNegHalfLog2e)
constexpr float kNegHalfLog2e = -0.72134752044448170f;
// the bounds of a surfel's support are grown by this many pixels so that the
// float32 blend never evaluates a contributing pair outside its tile rectangle
constexpr float kBoundPad = 1.0e-2f;
// Low-pass factor that switches the surfel low-pass term off (ellipsoids): any
// non-zero pixel offset gives a term above every record's support radius.
constexpr float kNoLowpass = 3.0e38f;

constexpr uint32_t kClsHole = 1, kClsGap = 2, kClsCentre = 4, kClsStrip = 8, kClsRender = 16,
                   kClsNet = 32;

// Device status bits (mapped to gs_status by the host).
constexpr uint32_t kStCapacity = 1, kStTimeout = 2;

struct EyeCam {
  float R[9];       // world -> camera rotation, row-major: X_c = R P + t
  float t[3];
  float centre[3];  // camera centre in world coordinates (SH view direction)
  float fx, fy, cx, cy;
  int W, H, tiles_x, tiles_y;  // tiles of the rasterizer grid
  int tshift;                   // rasterizer tile edge = 1 << tshift pixels
};

struct CamBlock {
  EyeCam eye[2];
  float Rrel[9];  // dominant camera -> affiliated camera: X_a = Rrel X_d + trel
  float trel[3];
};

// Host-side copy of what the FP64 set-up kernel needs.
struct PoseArgs {
  double R[2][9];
  double t[2][3];
  double fx, fy, cx, cy;
  int W, H;
  int neyes;
  int parallel;  // the eyes share orientation and the baseline lies in the image plane
  int tshift;    // rasterizer tile edge = 1 << tshift pixels (the dominant eye)
  int tshift1;   // the affiliated eye's (its ROI re-render may use another tile edge)
};

struct Counters {
  uint32_t status;
  uint32_t n_vis[2];     // visible (binned) surfels of the last binning per eye
  uint32_t n_inst[2];    // instances requested per eye (may exceed capacity)
  uint32_t dmin_bits, dmax_bits;  // range of the normalised depth (positive float bits)
  uint32_t n_rects;      // centre components found
  uint32_t n_sort[2];    // instances actually binned per eye (capacity-clamped)
  uint32_t n_rows[2];    // (surfel, tile row) spans per eye
  uint32_t n_band[2];    // (surfel, band) list entries of the last binning per eye
  uint32_t n_union;      // surfels in the dominant binning's depth order (both eyes' visible set)
  uint32_t n_items[2];   // rasterizer tiles listed by the last masked binning per eye
  uint32_t prev_range[2];// float bits of the last measured depth range (reused by depth_mode 2)
  uint32_t n_chunks[2];  // binning chunks holding binned surfels, per eye (at least 1)
  uint32_t n_table[2];   // (tile, chunk) entries the binning's table scan covers, per eye
  uint32_t n_centre;     // centre-hole pixels listed by the classification
  unsigned long long pairs[2];    // evaluated (pixel, surfel) pairs per eye (counting mode)
  unsigned long long contrib[2];  // of which contributed (alpha >= 1/255, before termination)
};

// The per-surfel blend record, 64 bytes = 4 float4:
//  r0 = (c.x, c.y, r_c^2, z_c)            projected centre, support radius^2
//                                         2 ln(255 o) (alpha >= 1/255 iff rho <= it),
//                                         centre depth
//  r1 = (V1, -V0, -U1, U0)                p.xy = [dx dy] * these (see preprocess)
//  r2 = (Az, Bz, Cz, dz_u)                p.z = Az + dx Bz + dy Cz; depth slope along u
//  r3 = (dz_v, r, g, b)                   depth slope along v; colour
struct Record {
  float4 r0, r1, r2, r3;
};

// Scratch of one eye's binning and rasterization. Each eye has its own, so the
// affiliated eye can be binned and rasterized while the dominant eye's binning
// and rasterizer run on another stream.
struct BinScratch {
  uint32_t *dkey[2], *dval[2];  // depth sort double buffers
  uint4 *bin_table;             // [tile][chunk] per-warp instance counts (8 x 16 bits)
  struct BandEntry *band_pool;  // (surfel, band) entries of every warp's lists
  uint2 *band_lists;            // [chunk][band][warp]: first entry, entries
  uint32_t *bin_offs;           // their tile-major exclusive scan
  uint32_t *ival;               // surfel id per instance, grouped by tile, depth order inside
  uint32_t *ikey;               // tile id per instance (keep_intermediates)
  uint2 *ranges;                // per rasterizer tile: [first, end) of its instances
  uint8_t *rmask;               // the binning's mask on the rasterizer grid (tile edge 8 or 32)
  uint32_t *items;              // rasterizer tiles of the last masked binning
  uint32_t *items16;            // [1 + 16-pixel tiles]: count, then the masked 16-pixel tiles
  uint32_t *lpt;                // [1 + tiles]: count, then the rasterizer's tiles, longest list first
  uint32_t *rqueue;             // persistent rasterizer work counter and exit ticket
  uint32_t *mask_sat;           // summed-area table of the mask [tiles_y + 1][tiles_x + 1]
  uint16_t *mask_clip;          // [2][tiles_y][tiles_x]: next / previous masked tile of the row (0xffff: none)
  uint32_t *rs_hist;            // radix sort: [4][256] digit counts, then [4][256] digit bases
  unsigned long long *rs_status;// radix sort look-back words [tiles][256]
  uint32_t *rs_ctl;             // radix sort control words (zero at creation)
  unsigned long long *scan_tiles;  // look-back tile words of the other scans
  uint32_t *scan_ticket;        // scan control words {tile counter, exit counter, epoch}
};

// Views of the caller-owned workspace.
struct Workspace {
  CamBlock *cams;
  Counters *ctr;
  float4 *rec[2];
  ushort4 *rect[2];
  float4 *bounds[2];
  uint32_t *cnt[2];             // tiles of each surfel's bounding rectangle (0 = culled)
  uint32_t *zkey[2];            // float bits of the centre depth per surfel and eye
  uint32_t *cnt_bin;            // tiles each surfel reaches in the last binning (keep_intermediates)
  uint32_t *uval;               // depth-ordered union of both eyes' binned surfels (dominant keys)
  uint32_t band_pool_cap[2];     // per eye
  BinScratch bin[2];            // per eye
  uint8_t *tile_mask;           // ROI mask on the 16-pixel grid
  uint8_t *strip_mask;          // edge-strip tiles of a reused depth range (16-pixel grid)
  float *strip_rgb;             // [3][pixels] the affiliated eye's strip tiles, rendered ahead
  uint32_t *row_off[2];         // per surfel and eye: slot of its first rectangle row in spans
  uint2 *spans[2];              // per (surfel, tile row): tile ranges [a0, a1] u [c0, c1], 4 x 16 bits
  // scans outside the binning (centre ROIs, repair tile lists) use bin[0]'s scratch
  unsigned long long *warpbuf;
  float *warp_depth;
  uint8_t *cls;
  int32_t *labels;
  uint32_t *cc_list;            // the frame's centre-hole pixels (classification order)
  uint32_t *slots;              // scan of component roots (+1)
  int4 *rects;                  // centre ROI rectangles
  int32_t *strips;              // [4][4]
  float *drange;                // [2]
  int32_t *widths;              // [4]
  // learned repair network
  float *rp_master, *rp_grad, *rp_m, *rp_v;  // FP32 parameters, gradients, AdamW moments
  uint8_t *rp_wpack;            // BF16 B-operand images of the six layers
  uint8_t *rp_wpack8;           // FP8 (e4m3) B-operand images
  uint8_t *rp_wpackT;           // BF16 flipped, transposed images of layers 1-5 (input gradients)
  float *rp_sx, *rp_sw;         // FP8 input scales and output-channel weight scales, [6][32] each
  uint32_t *rp_amax;            // calibration maxima of the layer inputs [6][32]
  float *rp_bias;               // [6][32]
  uint4 *rp_feat;               // [pixels] 8 x bf16 features of the affiliated eye
  float *rp_fill;               // [3][pixels] network fill
  float *rp_gate;               // [tiles] gate logit per listed tile
  uint8_t *rp_skip;             // [16-pixel tiles] the network's fill was taken
  uint32_t *rp_list, *rp_nlist; // listed tiles and their number
  double *ssim_part;            // per-(tile, channel) SSIM sums
  // limits
  int max_surfels, max_w, max_h, max_rects, max_tiles;  // max_tiles: rasterizer tiles at min_tshift
  int min_tshift;               // smallest rasterizer tile edge the buffers hold (log2)
  int64_t max_instances, max_pixels;  // max_instances: the dominant eye's
  int64_t max_inst[2];          // instance and span capacity per eye
  int paths;                    // GS_PATH_* bits the buffers serve
  int keep_intermediates;
  uint32_t bin_warp_surfels, bin_nch;  // binning chunk geometry (see launch_binning)
  int prim;                     // primitive of the prepared records (gs_scene.primitive), set by launch_preprocess
  float *host_img;              // gs_render_stereo_host's device images: rgb_dom, depth, trans, rgb_aff [8][pixels]
  size_t n_scan_tiles, n_rs_status;  // look-back words of scan_tiles and rs_status
};

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Host-side count of the kernels this library has enqueued (diagnostics).
extern unsigned long long g_launches;
#define GS_LAUNCHED(n) (::gs::g_launches += (n))

// Records a CUDA runtime error for gs_last_cuda_error (file:line of the caller)
// and returns GS_ERR_CUDA.
gs_status record_cuda_failure(const char *file, int line, cudaError_t e);

size_t workspace_bytes(const gs_limits &lim);
bool carve_workspace(const gs_limits &lim, void *base, size_t bytes, Workspace *ws);

// ---- launches (each returns the launch error) ----
cudaError_t launch_setup_cams(const PoseArgs &pa, CamBlock *cams, cudaStream_t s);
// Address of the set-up kernel (its graph node carries the per-frame poses).
const void *setup_cams_kernel_ptr();
cudaError_t launch_preprocess(const gs_scene &sc, Workspace &ws, int neyes, int W, int H,
                              cudaStream_t s);
// Bins the visible surfels of `eye` (restricted to tile_mask when given) into
// sorted per-tile instance lists and their ranges. Depth order:
//   kOrderOwn     sort this eye's binned surfels by their own keys;
//   kOrderUnion   (dominant eye of a parallel two-eye call) sort every surfel
//                 either eye bins by the dominant keys and keep that order in
//                 ws.uval;
//   kOrderReuse   (affiliated eye after kOrderUnion) filter the kept order: for
//                 a parallel rig both eyes' depth keys are identical, so the
//                 filtered order is the affiliated (depth, index) order.
enum BinOrder { kOrderOwn = 0, kOrderUnion = 1, kOrderReuse = 2 };
// roi16 (with W x H the image and tshift the rasterizer's log2 tile edge): the
// ROI mask on the 16-pixel grid from which the binning derives its own mask on
// the rasterizer grid into tile_mask (then ws.bin[eye].rmask); null when
// tile_mask is given directly (or no mask).
// rows (optional): a second stream and two events on which the row spans are
// computed beside the compaction and the depth sort (forked after the mask
// tables, joined before the band lists); null: on s, after the compaction.
struct SideRows {
  cudaStream_t stream;
  cudaEvent_t fork, join;
};
cudaError_t launch_binning(const Workspace &ws, int eye, int n, int tiles_x, int tiles_y,
                           const uint8_t *tile_mask, cudaStream_t s, int order = kOrderOwn,
                           const uint8_t *roi16 = nullptr, int W = 0, int H = 0, int tshift = 4,
                           const SideRows *rows = nullptr);
// Chunk geometry of the binning for a surfel capacity, and the one-time
// shared-memory opt-in of its kernel for the widest image.
uint32_t bin_warp_surfels(int max_surfels);
uint32_t bin_chunks(int max_surfels);
size_t band_list_words(int max_surfels, int max_tiles_y);
constexpr size_t kBandEntryBytes = 12;
cudaError_t prepare_binning(int max_tiles_x);
// ---- learned repair network ----
constexpr int kRepairParams = 39908;
struct RepairBatch {
  const uint4 *feat;     // [frames][H][W] 8 x bf16
  const float *target;   // [frames][3][H][W]
  const float *plain;    // [frames][3][H][W]
  int W, H;
  const uint32_t *tiles; // frame << 24 | ty << 12 | tx
  int n_tiles;
  void *scratch;         // repair_train_scratch_bytes(n_tiles)
};
struct RepairOpt {
  float lr, beta1, beta2, eps, weight_decay, gate_weight;
  int step;
};
cudaError_t prepare_repair();
cudaError_t prepare_reproject();
// The classification's centre-hole list of a caller-given class map, then the
// component labelling into ws.rects (gs_centre_rois).
cudaError_t launch_centre_rois_of(const Workspace &ws, const uint8_t *cls, int W, int H, int margin,
                                  uint8_t *tile_mask, cudaStream_t s);
size_t repair_train_scratch_bytes(int n_tiles);
cudaError_t repair_pack(const Workspace &ws, cudaStream_t s);
// Features from the warp buffer and the affiliated image after hole
// classification (rgb_aff before the ROI re-render).
cudaError_t repair_features(const Workspace &ws, int W, int H, const float *rgb_aff, uint4 *feat, cudaStream_t s);
// sm_share: the percentage of the multiprocessors the persistent grid may hold
// (less when other work runs beside it).
cudaError_t repair_forward(const Workspace &ws, const uint4 *feat, int W, int H, const uint32_t *tiles,
                           const uint32_t *n_ptr, uint32_t n_max, float *fill, float *gate, float *out4,
                           uint4 *acts, cudaStream_t s, bool fp8 = false, uint32_t *amax = nullptr,
                           int sm_share = 100);
// FP8 scales from the BF16 network's activation maxima over the listed tiles,
// then the e4m3 weight images.
cudaError_t repair_calibrate_fp8(const Workspace &ws, const uint4 *feat, int W, int H, const uint32_t *tiles,
                                 uint32_t n_tiles, float *gate_scratch, cudaStream_t s);
// Tile list, network and gated merge for the affiliated eye of the last warp
// (features already in ws.rp_feat). Gated tiles leave ws.tile_mask, or, with
// skip given, are flagged there instead (the ROI mask stays as it is, so the
// ROI binning can read it while the network runs on another stream).
cudaError_t repair_stereo(const Workspace &ws, int W, int H, float gate_tau, float *rgb_aff, cudaStream_t s,
                          bool fp8 = false, uint8_t *skip = nullptr);
cudaError_t repair_train_step(const Workspace &ws, const RepairBatch &b, const RepairOpt &o, float *host_loss,
                              cudaStream_t s);

// ---- persistent rasterizer ----
// One launch blends the tiles of up to kRasterFrames (frame, eye) images: its
// CTAs stay resident and take (frame, tile) work items from a device counter.
constexpr int kRasterFrames = 32;
struct RasterFrame {
  const uint2 *ranges;      // per rasterizer tile: [first, end) into ids
  const uint32_t *ids;      // surfel id per instance, grouped by tile, depth order inside
  const float4 *rec;        // this eye's blend records
  const float4 *box;        // their screen bounds xmin, xmax, ymin, ymax (conservative)
  const uint8_t *roi;       // 16-pixel ROI mask: only its pixels are written, or null
  const uint8_t *skip;      // 16-pixel tiles another step filled: not written, or null
  const uint32_t *items;    // listed tiles, or null: every tile in raster order
  int rshift, rtiles_x;     // > 0: the tile lists are those of a grid 1 << rshift times coarser
                            // (rtiles_x columns), each raster tile reads its parent's list
  const uint32_t *n_items;  // device count of the listed tiles
  float *rgb, *depth, *trans;  // [3][H][W], [H][W] (or null), [H][W] (or null)
  uint8_t *cls;             // class map: written pixels get kClsRender, or null
  unsigned long long *winit;  // warp buffer cleared (no sample) at every written pixel, or null
  Counters *ctr;            // depth range and pair counts of this frame
  float bg[3];
  int W, H, tiles_x, ntiles, tshift;
  int eye;
  int stats;                // 1: record the range of D / (1 - T) over pixels with coverage >= 0.5
  float lowpass;            // rho2 = lowpass |x - c|^2: 2 for surfels, kNoLowpass for ellipsoids
  uint32_t n_rec;           // records available (ids beyond are ignored)
};
struct RasterTable {
  RasterFrame f[kRasterFrames];
  int n;
};
// Tile edge, pixels per thread (the block has tile^2 / pix threads) and surfel
// records per shared-memory stage.
struct RasterConfig {
  int tile, pix, batch;
};
// Streaming multiprocessors of the current device (cached per device; 0 on error).
int sm_count();
// Grid cap for grid-stride kernels: `per_sm` CTAs per multiprocessor (152 SMs
// when the device cannot be queried).
inline int sm_grid_cap(int per_sm) {
  const int n = sm_count();
  return (n > 0 ? n : 152) * per_sm;
}
bool raster_config_ok(const RasterConfig &c);
int raster_tshift(const RasterConfig &c);
// `queue` holds two words that are zero between launches (the launch's last CTA
// clears them).
cudaError_t launch_raster(const RasterTable &t, const RasterConfig &c, bool count_pairs, uint32_t *queue,
                          cudaStream_t s);
// Rewrites f's work items as a list of its tiles, longest surfel list first,
// into buf (1 + f.ntiles words: the count, then the tiles); the images do not
// depend on the order.
cudaError_t launch_lpt_order(RasterFrame &f, uint32_t *buf, cudaStream_t s);
// Fills a RasterFrame for eye `eye` of a workspace; mask: 16-pixel ROI mask of a
// masked pass (the listed tiles of the last masked binning), or null.
RasterFrame raster_frame(const Workspace &ws, int eye, int W, int H, int tshift, const uint8_t *mask, float3 bg,
                         float *rgb, float *depth, float *trans, uint8_t *cls, bool stats);
// Mean SSIM of a [C][H][W] image against a reference (11 x 11 Gaussian window,
// zero padding) into *out (device); part: ssim_partials() doubles.
size_t ssim_partials(int max_w, int max_h);
cudaError_t launch_ssim(const float *a, const float *b, int W, int H, int C, double *part, float *out,
                        cudaStream_t s);
// The stages of launch_warp_classify one by one: the warp (clears the warp
// buffer and the ROI mask first), the edge ROI (into `mask`: ORed into the
// cleared ROI mask, or every tile assigned when `assign`), and the
// classification (which also keeps this frame's measured depth range for the
// next frame's depth_mode 2).
cudaError_t launch_warp(const Workspace &ws, int W, int H, const float *depth_dom, const float *trans_dom,
                        cudaStream_t s);
// Value of an empty warp-buffer entry (no source pixel landed there).
constexpr unsigned long long kNoSample = ~0ull;
cudaError_t launch_edge_roi(const Workspace &ws, const gs_roi_params &roi, uint8_t *mask, bool assign,
                            cudaStream_t s);
cudaError_t launch_classify(const Workspace &ws, int W, int H, int gap_thresh, const gs_roi_params &roi,
                            const float *rgb_dom, float *rgb_aff, cudaStream_t s);
// Strip tiles of an image rendered ahead -> the affiliated image (and class bits).
cudaError_t launch_strip_composite(const Workspace &ws, int W, int H, const float *src, float *rgb_aff,
                                   cudaStream_t s);
cudaError_t launch_mask_minus(uint8_t *mask, const uint8_t *minus, int n, cudaStream_t s);
// Warp, edge ROIs, hole classification and gap filling (writes rgb_aff and cls).
// cleared = true: the dominant eye's rasterizer has cleared the warp buffer
// (RasterFrame::winit), and the edge ROI assigns every tile of the ROI mask
// instead of adding its strips to a cleared mask.
cudaError_t launch_warp_classify(const Workspace &ws, int W, int H, int gap_thresh, const gs_roi_params &roi,
                                 const float *rgb_dom, const float *depth_dom, const float *trans_dom,
                                 float *rgb_aff, cudaStream_t s, bool cleared = false);
// Connected centre holes -> ROI rectangles -> tile mask.
cudaError_t launch_centre_rois(const Workspace &ws, int W, int H, int margin, cudaStream_t s);

}  // namespace gs
