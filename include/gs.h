/*
 * gs.h - C ABI of a GB300 (sm_103a) renderer for binocular 2D Gaussian
 * splatting by reprojection and selective patching (Zhu & Zhou, "From Mono to
 * Stereo: Accelerating Binocular Gaussian Splatting via Reprojection and
 * Selective Patching").
 *
 * The library renders the dominant eye in full (Sec. 3.1 Stage 1), warps it to
 * the affiliated eye with the depth proxy (Stage 2, Eq. 3-5), sorts the holes
 * into interpolated gaps and regions of interest (Stage 3, Sec. 3.5) and
 * re-rasterises only the tiles of those regions (Stage 4). Every stage runs in
 * this library's CUDA kernels on the caller's stream.
 *
 * Conventions
 *   - All scene and image pointers are DEVICE pointers owned by the caller; the
 *     library never frees them. Host structs (poses, intrinsics, parameters) are
 *     read during the call only.
 *   - Scene arrays, float32, structure of arrays:
 *       pos[n][4] surfel centre p_k (x, y, z, unused pad), 16-byte aligned
 *       quat[n][4] rotation (w, x, y, z), any non-zero norm (Sec. 3.3, Eq. 1)
 *       scale[n][2] in-plane scales (s_u, s_v) (Eq. 1) of a surfel scene, or
 *       scale[n][4] axis scales (s_x, s_y, s_z, unused pad) of an ellipsoid
 *       scene (primitive 1, below), 16-byte aligned
 *       opacity[n]
 *       sh[n][(sh_degree+1)^2][3] real SH colour coefficients, degree 0..3
 *   - Poses are camera-to-world, double precision: P_world = R X_cam + t with
 *     R row-major (Eq. 4). Camera axes: x right, y down, z forward.
 *   - Intrinsics: pinhole K = [[fx,0,cx],[0,fy,cy],[0,0,1]] (Eq. 3); pixel
 *     centres at integer coordinates, so a centred principal point is
 *     ((W-1)/2, (H-1)/2). Both eyes share the intrinsics.
 *   - Images are planar float32: rgb[3][H][W], depth[H][W], trans[H][W].
 *     depth is the unnormalised depth proxy D = sum_i d_i w_i with
 *     w_i = alpha_i T_i (Stage 1); trans is the final transmittance T.
 *   - Calls are asynchronous on the context's stream. A call returns GS_OK once
 *     its kernels are enqueued; errors found on the device (an instance buffer
 *     too small, a bounded wait that ran out) are recorded in a device status
 *     word that gs_context_check() reads back.
 *
 * Rendering rule (the 2DGS rasterizer conventions; the paper does not restate
 * them): alpha = min(0.99, o * Ghat) with Ghat = max(G(u,v), exp(-|x-c|^2))
 * (Eq. 2 plus the 2DGS low-pass term); contributions with alpha < 1/255 are
 * skipped; a pixel stops before the contribution that would bring T below
 * 1e-4; surfels are ordered by their float32 camera depth, ties by index.
 * A surfel is culled when its quaternion is zero, 255 o < 1, its centre is
 * within 0.2 m of the camera plane, or its support square reaches that plane.
 *
 * Ellipsoid scenes (gs_scene.primitive = 1): the 3D Gaussians of 3DGS, the
 * other backbone the method accepts (Sec. 3.2: any Gaussian splatting variant
 * with per-pixel depth), in the EWA splatting convention of the 3DGS
 * rasterizer. Covariance Sigma = Rq diag(s^2) Rq^T; screen covariance
 * Sigma2D = J W Sigma W^T J^T + 0.3 I with W the world-to-camera rotation and
 * J = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]] at the centre (unclamped);
 * alpha = min(0.99, o exp(-d^T Sigma2D^-1 d / 2)), d the pixel offset from the
 * projected centre, with no further low-pass term; the depth d_i of every
 * contribution is the centre's camera depth. Ordering, the 1/255 and 1e-4
 * rules and the z_near cull of the centre are those of surfels.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GS_OK = 0,
  GS_ERR_BAD_ARG = 1,   /* a NULL pointer, a size out of the context's limits, ... */
  GS_ERR_CAPACITY = 2,  /* a device buffer was too small (instances, ROI rectangles) */
  GS_ERR_TIMEOUT = 3,   /* a bounded device loop gave up; results are incomplete */
  GS_ERR_CUDA = 4,      /* a CUDA runtime call failed */
  GS_ERR_WORKSPACE = 5, /* the workspace is smaller than gs_workspace_size() asks */
  GS_ERR_NOT_LOADED = 6 /* no repair network has been loaded */
} gs_status;

typedef struct gs_context gs_context;

typedef struct {
  const float *pos, *quat, *scale, *opacity, *sh;
  int n;
  int sh_degree;
  int primitive; /* 0: 2D surfels (scale[n][2]); 1: 3D ellipsoids (scale[n][4]) */
} gs_scene;

typedef struct {
  double R[9];
  double t[3];
} gs_pose;

typedef struct {
  double fx, fy, cx, cy;
  int width, height;
} gs_intrinsics;

/* Adaptive ROI generator settings (Sec. 3.5). */
typedef struct {
  int margin;           /* m in Eq. 7-8 and Step 2; the paper fixes 32 */
  int samples_per_edge; /* N boundary samples per image edge (>= 2) */
  int enable_center;    /* Step 2 (centre ROIs) on/off, chosen before rendering */
  int depth_mode;       /* 0: d_min/d_max = per-frame range of the normalised depth
                           D/(1-T) over pixels with coverage 1-T >= 0.5; 1: fixed;
                           2: the range the previous stereo call of this context
                           measured (temporal reuse along a head trajectory; the
                           paper leaves continuous head motion to future work,
                           Sec. 4.6 and Sec. 5): the edge strips are then
                           known before the dominant eye is rendered, and
                           gs_render_stereo renders the affiliated eye's strip
                           tiles on a second stream meanwhile. The result equals
                           mode 1 with that range. A context's first call, with
                           no previous range, measures it (mode 0). */
  float d_min, d_max;   /* the two depth hypotheses when depth_mode = 1 */
  int repair_mode;      /* 0: plain interpolation + ROI re-render; 1: learned repair
                           in BF16; 2: learned repair in FP8 (both need
                           gs_repair_load); 3: plain output, plus the repair
                           network's features for gs_repair_features */
  float gate_tau;       /* learned repair: a tile uses the network fill when
                           sigmoid(gate logit) >= gate_tau, else the plain path */
} gs_roi_params;

/* Outputs of the stereo and two-pass calls (device pointers, caller-owned). */
typedef struct {
  float *rgb_dom, *depth_dom, *trans_dom; /* dominant eye, [3][H][W], [H][W], [H][W] */
  float *rgb_aff;                         /* affiliated eye, [3][H][W] */
  uint8_t *cls_aff;   /* optional [H][W] class bits: 1 hole after the warp, 2 gap
                         (interpolated), 4 centre hole, 8 inside an edge strip,
                         16 re-rendered tile, 32 filled by the repair network */
  int32_t *roi_rects; /* optional [max_rects][4] centre ROIs x0, y0, x1, y1 (half-open
                         pixels, tile aligned), in the order of each component's
                         smallest linear pixel index; only the first
                         min(count, max_rects) entries are written */
  int32_t *roi_count; /* optional [1]: number of centre components found */
  int32_t *edge_widths; /* optional [4]: left, right, top, bottom widths (Eq. 7-8) */
} gs_outputs;

/* Upper bounds a context is sized for. */
typedef struct {
  int max_surfels;
  int max_width, max_height; /* each <= 8192 */
  int64_t max_instances; /* (surfel, tile) pairs per eye; < 2^30 */
  int max_rects;         /* centre ROI rectangles */
  int keep_intermediates;/* 1: also store per-surfel float bounds, per-instance tile
                            ids and per-surfel tile counts for inspection */
  int min_tile;          /* smallest rasterizer tile edge the context will run: 8, 16
                            or 32 (0 = 16); max_width / min_tile <= 512 */
  int host_outputs;      /* 1: the workspace also holds the device images that
                            gs_render_stereo_host renders into (32 B per pixel) */
  int64_t max_instances_aff; /* (surfel, tile) pairs and (surfel, tile row) spans
                            of the affiliated eye (0 = max_instances). A context
                            that serves only gs_render_stereo needs room for the
                            ROI tiles alone (Stage 4 re-renders only them) */
  int paths;             /* which entry points the context serves, GS_PATH_* bits
                            (0 = all); buffers only other paths use are left
                            out of the workspace, and a call on a path the
                            context was not sized for returns GS_ERR_BAD_ARG */
} gs_limits;

/* gs_limits.paths bits. MONO: gs_render_mono and gs_render_two_pass (full
 * renders of one or both eyes). STEREO: gs_render_stereo(_host) with
 * depth_mode 0 or 1 and repair_mode 0: the warp, class, component and ROI
 * buffers (25 B per pixel). REUSE: depth_mode 2 (the affiliated eye's strip
 * image, 12 B per pixel). REPAIR: the learned repair (repair_mode 1-3, the
 * gs_repair_* calls): features and fill (28 B per pixel). */
#define GS_PATH_MONO 1
#define GS_PATH_STEREO 2
#define GS_PATH_REUSE 4
#define GS_PATH_REPAIR 8
#define GS_PATH_ALL 15

/* Work counts of a context's last call, for sizing a context to a workload:
 * per eye the binned surfels, the (surfel, tile) instances, the (surfel, tile
 * row) spans and the (surfel, band of 4 tile rows) list entries the binning
 * produced (counted also when they overflowed a capacity). */
typedef struct {
  int64_t binned[2], instances[2], spans[2], band_entries[2];
} gs_usage;

/* Synchronises the context's stream and reads the counts of its last call. */
gs_status gs_context_usage(gs_context *ctx, gs_usage *usage);

/* Bytes of device workspace a context with these limits needs. */
gs_status gs_workspace_size(const gs_limits *lim, size_t *bytes);

/* Creates a context on the current device. `workspace` is a caller-owned device
 * allocation of at least gs_workspace_size() bytes (256-byte aligned) that the
 * context uses for all scratch; the context allocates no device memory itself.
 * `stream` is a cudaStream_t (NULL = the legacy default stream). */
gs_status gs_context_create(gs_context **out, const gs_limits *lim, void *workspace,
                            size_t workspace_bytes, void *stream);
gs_status gs_context_destroy(gs_context *ctx);
gs_status gs_context_set_stream(gs_context *ctx, void *stream);

/* Synchronises the context's stream, returns the device status word (0 = no
 * error, else a GS_ERR_* code) in *device_status and clears it. */
gs_status gs_context_check(gs_context *ctx, int *device_status);

/* Full render of one eye (Sec. 3.1 Stage 1): RGB, depth proxy and transmittance
 * from the same blending weights. bg: host float[3] background or NULL (black). */
gs_status gs_render_mono(gs_context *ctx, const gs_scene *scene, const gs_pose *pose,
                         const gs_intrinsics *intr, const float *bg, float *rgb, float *depth,
                         float *trans);

/* The method (Sec. 3.1-3.5, the pipeline of Sec. 4.3): full dominant render,
 * forward warp to the affiliated eye with a depth test, edge ROIs (Eq. 6-8),
 * gaps of at most gap_thresh pixels interpolated, centre ROIs (optional), and
 * re-rasterisation of the ROI tiles only. Black background. */
gs_status gs_render_stereo(gs_context *ctx, const gs_scene *scene, const gs_pose *pose_dom,
                           const gs_pose *pose_aff, const gs_intrinsics *intr, int gap_thresh,
                           const gs_roi_params *roi, const gs_outputs *out);

/* gs_render_stereo with both eyes' RGB images delivered to HOST memory, for a
 * frame loop that ends on the host (a display or an encoder). The pipeline
 * renders into the context's own device images (gs_limits.host_outputs = 1).
 * The dominant eye is final after Stage 1, so its image is copied out on a
 * second stream while Stages 2-4 run; the affiliated eye's image follows
 * Stage 4.
 *   host_rgb_dom, host_rgb_aff: [3][H][W] float32 in page-locked host memory
 *     (cudaHostAlloc, cudaMallocHost or cudaHostRegister); other host memory,
 *     device memory or NULL gives GS_ERR_BAD_ARG.
 * Asynchronous like gs_render_stereo: the host images are complete once the
 * context's stream is synchronised (gs_context_check does that). The depth,
 * transmittance and class images stay in the workspace (gs_context_buffer). */
gs_status gs_render_stereo_host(gs_context *ctx, const gs_scene *scene, const gs_pose *pose_dom,
                                const gs_pose *pose_aff, const gs_intrinsics *intr, int gap_thresh,
                                const gs_roi_params *roi, float *host_rgb_dom, float *host_rgb_aff);

/* The sequential two-pass reference of Sec. 4.3: full dominant render, then a
 * full affiliated render, built from the same kernels. Black background. */
gs_status gs_render_two_pass(gs_context *ctx, const gs_scene *scene, const gs_pose *pose_dom,
                             const gs_pose *pose_aff, const gs_intrinsics *intr,
                             const gs_outputs *out);

/* ---- Learned hole repair (no counterpart in the paper: the paper repairs holes
 * by interpolation and ROI re-rendering only, Sec. 3.1 Stage 3 and Sec. 3.5).
 *
 * A small network fills the holes the forward warp leaves and decides, per
 * 16x16 tile, whether its fill replaces that tile's plain repair:
 *   features per affiliated pixel (8 x bf16, channels 6 and 7 zero):
 *     0-2 the affiliated image after hole classification: the warped colour, at
 *     holes outside the edge strips the method's own fill (gap interpolation,
 *     else the row/column fill), 0 at holes inside the strips; 3 inverse depth
 *     1/z of the winner (0 at holes and background samples); 4 hole mask;
 *     5 min(distance to the nearest hole, 8) / 8 in pixels;
 *   network: six 3x3 convolutions (cross-correlation, zero padding at the image
 *     border) 6 -> 32 -> 32 -> 32 -> 32 -> 32 -> 4, ReLU after the first five,
 *     BF16 weights and activations, FP32 accumulation on the tensor cores;
 *     outputs 0-2 are a correction added to feature channels 0-2 (the fill =
 *     features + correction), output 3 a gate logit;
 *   gate: the mean of output 3 over a tile's pixels; with repair_mode = 1 in
 *     gs_render_stereo the network runs on the ROI tiles that hold a hole
 *     outside the edge strips, and such a tile whose sigmoid(gate) >= gate_tau
 *     takes max(fill, 0) at its hole pixels (class bit 32) and is not
 *     re-rendered; every other tile keeps the plain path.
 * Parameters: GS_REPAIR_PARAMS floats in the canonical order: for each layer,
 * W[c_out][3][3][c_in] then b[c_out]. */
#define GS_REPAIR_PARAMS 39908

/* Copies the FP32 parameters (host array) into the context (synchronises its
 * stream), resets the AdamW state and packs the BF16 weights. */
gs_status gs_repair_load(gs_context *ctx, const float *weights, int64_t count);

/* Reads back the FP32 parameters (which = 0), the gradients of the last
 * training step (which = 1), or the AdamW first (which = 2) and second (which =
 * 3) moments into a host array of GS_REPAIR_PARAMS floats; synchronises the
 * stream. */
gs_status gs_repair_read(gs_context *ctx, int which, float *out, int64_t count);

/* Training checkpoints: the AdamW steps taken since the last gs_repair_load
 * (the bias correction's step count), and the restore of a saved state: the
 * parameters, both moments (host arrays of GS_REPAIR_PARAMS floats) and the
 * step count; packs the BF16 weights and synchronises the stream. A training
 * run resumed from a state read with gs_repair_read (which = 0, 2, 3) and
 * gs_repair_steps continues exactly as the uninterrupted run (the training
 * step is deterministic). */
gs_status gs_repair_steps(gs_context *ctx, int *steps);
gs_status gs_repair_load_state(gs_context *ctx, const float *weights, const float *m, const float *v,
                               int64_t count, int steps);

/* The features of the last gs_render_stereo call on this context made with
 * repair_mode != 0 (same width and height), copied to feat: device [H][W][8]
 * bf16, 16-byte aligned. repair_mode = 3 computes them without running the
 * network (training data). */
gs_status gs_repair_features(gs_context *ctx, int width, int height, uint16_t *feat);

/* Runs the network on listed tiles of a stack of feature images.
 * feat: device [frames][H][W][8] bf16; tiles: device uint32 entries
 * frame << 24 | tile_y << 12 | tile_x (16x16 tiles); fill: device
 * [frames][3][H][W] (written inside the listed tiles; may be NULL); gate: device
 * float[n_tiles], the mean gate logit of each listed tile. fp8 = 1 runs the
 * e4m3 network (needs gs_repair_calibrate_fp8). */
gs_status gs_repair_infer(gs_context *ctx, const uint16_t *feat, int frames, int width, int height,
                          const uint32_t *tiles, int n_tiles, float *fill, float *gate, int fp8);

/* FP8 (e4m3) network, FP32 accumulation with per-channel scales. Calibration
 * runs the BF16 network over the listed tiles and records, per layer and input
 * channel, the largest |input|; the input scale sx = max / 448 (the largest
 * finite e4m3 value) is folded into the weights W' = W * sx, which are stored
 * per output channel as e4m3(W' / sw) with sw = max |W'| / 448. A layer computes
 * y = sw * sum(codes) + b in FP32, then ReLU and the next layer's e4m3 input.
 * Needed by gs_repair_infer(fp8 = 1) and gs_render_stereo(repair_mode = 2);
 * loading weights or a training step with lr > 0 invalidates it. */
gs_status gs_repair_calibrate_fp8(gs_context *ctx, const uint16_t *feat, int frames, int width, int height,
                                  const uint32_t *tiles, int n_tiles);
/* The calibrated scales: out (host float[384]) = sx[6][32] then sw[6][32]. */
gs_status gs_repair_read_fp8_scales(gs_context *ctx, float *out);

/* One training step on listed tiles: forward (keeping activations), loss, FP32
 * gradients, and an AdamW update of the FP32 parameters when lr > 0 (lr = 0
 * leaves them unchanged and only computes gradients).
 * Loss = mean over the tiles' hole pixels of |fill - target| (averaged over RGB)
 *      + gate_weight * mean over tiles of BCE(sigmoid(gate), label), where the
 *        label is 1 when, over the tile's hole pixels, max(fill, 0) scores a PSNR
 *        against the target of at least 30 dB and at most 0.5 dB below that of
 *        the plain image at the same pixels.
 * loss (host float[4], may be NULL): total, L1 term, BCE term, share of positive
 * labels; reading it synchronises the stream. */
typedef struct {
  const uint16_t *feat;  /* device [frames][H][W][8] bf16 */
  const float *target;   /* device [frames][3][H][W]: full affiliated render */
  const float *plain;    /* device [frames][3][H][W]: plain-method affiliated image */
  int frames, width, height;
  const uint32_t *tiles; /* device, as for gs_repair_infer */
  int n_tiles;
  void *scratch;         /* device, gs_repair_train_scratch_size() bytes */
} gs_repair_batch;
typedef struct {
  float lr, beta1, beta2, eps, weight_decay, gate_weight;
} gs_adamw;
gs_status gs_repair_train_scratch_size(int n_tiles, size_t *bytes);
gs_status gs_repair_train_step(gs_context *ctx, const gs_repair_batch *batch, const gs_adamw *opt, float *loss);

/* Allocation-free forward warp (no counterpart in the paper; a deployment aid).
 *
 * For callers that cannot allocate device memory: a plugin or compositor inside
 * a host application that owns the GPU memory pool and forbids allocations from
 * outside it, or a frame loop with a hard deadline where a cudaMalloc could stall
 * or fail. It needs no gs_context and no workspace, and calls no cudaMalloc,
 * cudaFree or other allocating routine. It computes the depth-tested forward warp
 * of the stereo pipeline (the same arithmetic and tie-breaking as
 * gs_render_stereo's warp stage): every dominant pixel with coverage 1 - T >= 0.5
 * is unprojected with depth D / (1 - T), moved to the affiliated camera and
 * projected to pixel (floor(u + 0.5), floor(v + 0.5)); other pixels travel as
 * background samples at infinite depth; the nearest sample wins, then the
 * smallest source index.
 *
 * Inputs (device pointers, the dominant eye's gs_render_* outputs, planar):
 *   rgb_dom float[3][H][W], depth_dom float[H][W] (D), trans_dom float[H][W] (T);
 *   pose_dom, pose_aff, intr: host structs (both eyes share intr).
 * Outputs (device pointers, caller-owned):
 *   rgb_warp float[3][H][W]: the winner's colour, 0 at holes;
 *   depth_warp float[H][W] (may be NULL): the winner's camera-space depth in the
 *     affiliated eye, +inf for a background sample, 0 at holes;
 *   hole uint8[H][W] (may be NULL): 1 where no sample landed.
 *
 * Scratch: one 64-bit key per pixel in a static device array of
 * GS_WARP_NOALLOC_MAX_PIXELS entries (32 MiB), held by every device that loads
 * this library until the process exits. Frames with more pixels return
 * GS_ERR_CAPACITY. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture. The call clears the array's first W*H keys before
 * it scatters, so no state carries over from an earlier call; but every call on
 * a device shares the one array, so calls that overlap on the GPU (other streams,
 * other host threads) race and give wrong results: serialise them.
 * Asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream).
 * Errors: GS_ERR_BAD_ARG (NULL input or output, non-positive size or focal
 * length), GS_ERR_CAPACITY (W*H above the limit), GS_ERR_CUDA (lookup or launch
 * failure; see gs_last_cuda_error). */
#define GS_WARP_NOALLOC_MAX_PIXELS (1 << 22)
gs_status gs_warp_noalloc(const float *rgb_dom, const float *depth_dom, const float *trans_dom,
                          const gs_pose *pose_dom, const gs_pose *pose_aff, const gs_intrinsics *intr,
                          float *rgb_warp, float *depth_warp, uint8_t *hole, void *stream);

/* Intermediate buffers of the last call, for inspection by tests. *dev_ptr points
 * into the workspace; *count is the element count the call produced (read from
 * the device, so this synchronises the stream). DEPTH_ORDER, INST_KEYS,
 * INST_VALS and RANGES hold the last binning of the call (the affiliated eye's
 * ROI binning after gs_render_stereo or gs_render_two_pass). */
typedef enum {
  GS_BUF_RECORDS = 0,     /* float4[eye][max_surfels][4]: per-surfel blend records */
  GS_BUF_RECTS = 1,       /* uint16x4[eye][max_surfels]: tile rect tx0, ty0, tx1, ty1 */
  GS_BUF_BOUNDS = 2,      /* float4[eye][max_surfels]: xmin, xmax, ymin, ymax (screen bounds) */
  GS_BUF_COUNTS = 3,      /* uint32[eye][max_surfels]: tiles touched per surfel (0 = culled) */
  GS_BUF_DEPTH_ORDER = 4, /* uint32[max_surfels]: surfel ids of the last binning in depth order */
  GS_BUF_INST_KEYS = 5,   /* uint32[max_instances]: tile id per instance, sorted (keep_intermediates) */
  GS_BUF_INST_VALS = 6,   /* uint32[max_instances]: surfel id per instance: tile by tile, depth order */
  GS_BUF_RANGES = 7,      /* uint32x2[tiles]: [start, end) of each tile's instances */
  GS_BUF_WARP = 8,        /* uint64[pixels]: (float depth bits << 32) | source index, ~0 = hole */
  GS_BUF_TILE_MASK = 9,   /* uint8[tiles]: tiles of the ROI re-render */
  GS_BUF_DEPTH_RANGE = 10,/* float[2]: d_min, d_max used by the edge ROI */
  GS_BUF_STRIPS = 11,     /* int32[4][4]: edge strips x0, y0, x1, y1 (left, right, top, bottom) */
  GS_BUF_WARP_DEPTH = 12, /* float[pixels]: warped depth (+inf background, 0 hole) */
  GS_BUF_PAIRS = 13,      /* uint64[2]: evaluated (pixel, surfel) pairs per eye, when counting */
  GS_BUF_BIN_COUNTS = 14, /* uint32[max_surfels]: tiles each surfel's support reaches in the
                             last binning (within the ROI tile mask for the ROI pass;
                             keep_intermediates) */
  GS_BUF_EYE1 = 0x100     /* OR into RECORDS/RECTS/BOUNDS/COUNTS for the affiliated eye */
} gs_buffer_id;

gs_status gs_context_buffer(gs_context *ctx, int which, void **dev_ptr, size_t *bytes,
                            int64_t *count);

/* 1: the blend kernels count evaluated (pixel, surfel) pairs, and those that
 * contributed, into GS_BUF_PAIRS (uint64 evaluated[2], contributed[2]). */
gs_status gs_context_set_counting(gs_context *ctx, int enable);

/* SSIM of an image against a reference (the structural similarity that Table 2
 * reports beside PSNR), in the convention of the 2DGS/3DGS evaluation code:
 * 11 x 11 Gaussian window with sigma 1.5, same-size filtering with zero
 * padding, C1 = 0.01^2, C2 = 0.03^2 (dynamic range 1), averaged over every
 * pixel of every channel. img, ref: device [channels][height][width] float32
 * (channels 1..3), within the context's size limits; *ssim: device float,
 * written on the context's stream (float32 arithmetic, double-precision sum
 * in a fixed order). */
gs_status gs_ssim(gs_context *ctx, const float *img, const float *ref, int width, int height, int channels,
                  float *ssim);

/* Centre ROIs of a caller-given class map (Sec. 3.1 Stage 3, Step 2, the step
 * gs_render_stereo runs after its classification): the 4-connected components
 * of the pixels whose class has GS_CLS_CENTRE set, each component's bounding box
 * grown by `margin` pixels, aligned outward to the 16-pixel tile grid and
 * clipped to the image.
 *   cls        device uint8[height][width], the classes of gs_outputs.cls_aff
 *              (only the GS_CLS_CENTRE bit is read), within the size limits;
 *   rects      device int32[max_rects][4]: x0, y0, x1, y1 (x1, y1 exclusive) per
 *              component, in increasing order of the component's first pixel in
 *              row-major order; entries past the count are left unspecified;
 *   count      device int32: the number of components, which may exceed the
 *              context's max_rects (then only max_rects are written and
 *              gs_context_check reports GS_ERR_CAPACITY);
 *   tile_mask  optional device uint8[ceil(height/16)][ceil(width/16)]: 1 is
 *              written on every tile of a rectangle (nothing is cleared).
 * Needs the stereo path (GS_PATH_STEREO). Asynchronous on the context's stream. */
gs_status gs_centre_rois(gs_context *ctx, const uint8_t *cls, int width, int height, int margin, int32_t *rects,
                         int32_t *count, uint8_t *tile_mask);

/* Rasterizer configuration (no counterpart in the paper, which fixes 16x16
 * tiles for the ROI grid, Sec. 3.5; the tile edge of the rasterizer itself is a
 * free choice of the 2DGS/3DGS tile rasterizer it builds on).
 *   tile  8, 16 or 32: edge of the rasterizer's square tiles, pixels; at least
 *         the context's min_tile. The ROI generator keeps the 16-pixel grid:
 *         with 32-pixel tiles only the pixels of ROI 16-pixel tiles are written.
 *   pix   pixels per thread, i.e. the block shape (tile^2 / pix threads): 1 or 2
 *         at tile 8, 2 or 4 at tile 16, 2, 4 or 8 at tile 32.
 *   batch 32, 64, 128 or 256 surfel records per shared-memory stage.
 * Every configuration produces the same images bit for bit; they differ in
 * speed only. The default is {16, 4, 128} ({32, 8, 128} when min_tile = 32).
 * Returns GS_ERR_BAD_ARG for any other value. */
typedef struct {
  int tile, pix, batch;
} gs_raster_config;
gs_status gs_context_set_raster(gs_context *ctx, const gs_raster_config *rc);
gs_status gs_context_get_raster(gs_context *ctx, gs_raster_config *rc);

/* The configuration of gs_render_stereo's ROI re-render (Sec. 3.1 Stage 4): the
 * affiliated eye's ROI tiles are binned and blended on its tile grid, which may
 * differ from the dominant eye's (the ROI mask lives on 16-pixel tiles, so
 * 16-pixel tiles render exactly the ROI tiles). A 16-pixel ROI tile under a
 * coarser dominant grid is binned on the dominant grid and blended from its
 * parent tile's list (fewer, shorter binning passes; only the masked 16-pixel
 * tiles blended). NULL clears it: the ROI re-render then uses
 * gs_context_set_raster's configuration. The images do not depend on it. get
 * returns the configuration the ROI re-render uses and, in *is_set, whether one
 * of its own is set. */
gs_status gs_context_set_raster_roi(gs_context *ctx, const gs_raster_config *rc);
gs_status gs_context_get_raster_roi(gs_context *ctx, gs_raster_config *rc, int *is_set);

/* ---------------------------------------------------------------------------
 * Batched rendering (a serving mode; the paper renders one stereo frame at a
 * time, Sec. 4.3).
 *
 * A batch renders up to GS_BATCH_MAX_FRAMES stereo frames - of different
 * scenes, surfel counts and image sizes - in one call. Frame f runs in slot f:
 * a context the caller created with limits that fit that frame, whose
 * workspace, counters and repair weights it uses (a slot serves one frame per
 * call). The per-frame stages (pose set-up, preprocessing, binning, warp, hole
 * classification, ROIs, repair) run on one stream per frame; each rasterizer
 * pass is ONE persistent launch over all frames: the dominant eyes, then the ROI
 * tiles. From the second call with a configuration on, the whole call is one
 * CUDA graph replay on the batch's stream (poses are patched in). Frame f's
 * outputs equal those of gs_render_stereo (gs_render_two_pass) on slot f with
 * the batch's rasterizer configuration, bit for bit. A slot must not be used by
 * another call while a batch call using it is in flight.
 *
 * gs_batch_create: slots are n_slots distinct contexts (1..GS_BATCH_MAX_FRAMES);
 *   stream is a cudaStream_t (NULL = legacy default stream). The batch owns CUDA
 *   streams and events (no device memory) and starts with the default rasterizer
 *   configuration. gs_batch_destroy releases them; the slots stay the caller's.
 * gs_render_stereo_batch: frames[0..n_frames) with n_frames <= n_slots; the
 *   gap threshold and ROI parameters apply to every frame. Errors: BAD_ARG (a
 *   frame that does not fit its slot, an invalid parameter), NOT_LOADED
 *   (repair_mode 1 or 2 on a slot without weights / FP8 calibration), CUDA.
 * gs_batch_check: synchronises the batch's stream; *device_status is the worst
 *   device status of the slots (cleared). */
#define GS_BATCH_MAX_FRAMES 32
typedef struct gs_batch gs_batch;
typedef struct {
  const gs_scene *scene;            /* device SoA, as for gs_render_stereo */
  gs_pose pose_dom, pose_aff;
  gs_intrinsics intr;
  gs_outputs out;                   /* caller-owned device outputs of this frame */
} gs_frame;
gs_status gs_batch_create(gs_batch **out, gs_context *const *slots, int n_slots, void *stream);
gs_status gs_batch_destroy(gs_batch *b);
gs_status gs_batch_set_raster(gs_batch *b, const gs_raster_config *rc); /* tile >= every slot's min_tile */
gs_status gs_batch_get_raster(gs_batch *b, gs_raster_config *rc);
gs_status gs_batch_set_graphs(gs_batch *b, int enable);
gs_status gs_batch_set_counting(gs_batch *b, int enable); /* pair counts land in each slot's GS_BUF_PAIRS */
/* With profiling on, stage times of the last call (synchronises): per-frame
 * set-up + preprocessing + dominant binning, dominant rasterizer launch,
 * per-frame warp .. ROI binning, ROI rasterizer launch, outputs. */
gs_status gs_batch_set_profiling(gs_batch *b, int enable);
gs_status gs_batch_stage_times(gs_batch *b, float *ms, int max_stages, int *n_stages);
gs_status gs_batch_check(gs_batch *b, int *device_status);
gs_status gs_render_stereo_batch(gs_batch *b, const gs_frame *frames, int n_frames, int gap_thresh,
                                 const gs_roi_params *roi);
/* The sequential comparator (Sec. 4.3) in the same batched mode: both eyes of
 * every frame rendered in full (rgb_dom, depth_dom, trans_dom, rgb_aff). */
gs_status gs_render_two_pass_batch(gs_batch *b, const gs_frame *frames, int n_frames);

/* Full renders of single eyes in one call (as gs_render_mono, frame f in slot
 * f): pose set-up, preprocessing and binning of every frame side by side, then
 * one rasterizer launch over all of them. With a stereo pair's two eyes as two
 * frames this is the concurrent two-eye comparator (the paper leaves concurrent
 * and multiview references to future work, Sec. 4.6 and Sec. 5): the two-pass
 * render without its sequential order. rgb is required; depth, trans optional. */
typedef struct {
  const gs_scene *scene;
  gs_pose pose;
  gs_intrinsics intr;
  float bg[3];
  float *rgb, *depth, *trans; /* device [3][H][W], [H][W], [H][W] */
} gs_mono_frame;
gs_status gs_render_mono_batch(gs_batch *b, const gs_mono_frame *frames, int n_frames);

/* ---------------------------------------------------------------------------
 * Rasterizer autotuner. Runs the call - gs_render_stereo(_batch) with `roi`, or
 * the two-pass comparator gs_render_two_pass(_batch) when roi is NULL (gap
 * threshold unused) - on the caller's inputs once per rasterizer configuration
 * the slots allow (two untimed calls, then `reps` calls timed with CUDA events
 * on the call's stream; the median counts) and leaves the fastest set on the
 * batch / context. results[0..*n_results) gets
 * every configuration tried with its median ms (-1: the configuration
 * overflowed a buffer or failed). Results are cached for the process under a
 * key of the GPU (name, compute capability, SM count) and the frames' shapes
 * (image size, surfel-count power-of-two bucket, SH degree; stereo with plain
 * or learned repair, or two-pass); with use_cache = 1 a cached entry is applied without timing
 * (*n_results = 0). The outputs of the tuned calls are overwritten. */
typedef struct {
  gs_raster_config rc;
  float ms;
} gs_tune_result;
gs_status gs_autotune_batch(gs_batch *b, const gs_frame *frames, int n_frames, int gap_thresh,
                            const gs_roi_params *roi, int reps, int use_cache, gs_tune_result *results,
                            int max_results, int *n_results, gs_raster_config *best, float *best_ms);
gs_status gs_autotune_stereo(gs_context *ctx, const gs_scene *scene, const gs_pose *pose_dom,
                             const gs_pose *pose_aff, const gs_intrinsics *intr, int gap_thresh,
                             const gs_roi_params *roi, const gs_outputs *out, int reps, int use_cache,
                             gs_tune_result *results, int max_results, int *n_results,
                             gs_raster_config *best, float *best_ms);
/* The process-wide tuning cache (host only; no GPU needed). Text file, one
 * entry per line: "<key> <tile> <pix> <batch> <ms>", keys without blanks.
 * Loading merges a file's entries (a malformed file changes nothing and gives
 * BAD_ARG); get gives NOT_LOADED for a missing key. */
gs_status gs_tune_cache_save(const char *path);
gs_status gs_tune_cache_load(const char *path);
gs_status gs_tune_cache_clear(void);
gs_status gs_tune_cache_size(int *n);
gs_status gs_tune_cache_put(const char *key, const gs_raster_config *rc, float ms);
gs_status gs_tune_cache_get(const char *key, gs_raster_config *rc, float *ms);

/* 1 (the default): the first call of an entry point with a given scene, image
 * size, output set and parameters captures its kernels into a CUDA graph, and
 * later calls only patch the poses into it and replay it on the context's
 * stream. 0: every call enqueues its kernels one by one. Calls made while the
 * context's stream is being captured by the caller always enqueue directly. */
gs_status gs_context_set_graphs(gs_context *ctx, int enable);

/* 1: record a CUDA event on the context's stream at every stage boundary of the
 * following calls (the paper reports a per-stage time breakdown, Sec. 4.5). */
gs_status gs_context_set_profiling(gs_context *ctx, int enable);

/* Milliseconds of each stage of the last profiled call (synchronises the stream):
 *   gs_render_stereo:   preprocess, bin dominant, blend dominant, warp + edge ROI +
 *                       gaps, centre ROIs, bin ROI tiles, blend ROI tiles, outputs
 *   gs_render_two_pass: preprocess, bin dominant, blend dominant, bin affiliated,
 *                       blend affiliated
 *   gs_render_mono:     preprocess, bin, blend
 * "preprocess" is the preprocessing kernel alone: the counter reset and the FP64
 * camera set-up before it belong to no stage. */
gs_status gs_context_stage_times(gs_context *ctx, float *ms, int max_stages, int *n_stages);

const char *gs_status_str(gs_status s);

/* Text of the CUDA runtime error behind the last GS_ERR_CUDA returned on the
 * calling host thread. */
const char *gs_last_cuda_error(void);

/* 1 (the default): the library launches its kernels with programmatic dependent
 * launch, so a kernel is set up while its predecessor in the stream (or graph)
 * drains; every kernel waits for its predecessor's completion before touching
 * memory, so results do not depend on this switch. 0: plain launches.
 * Process-wide; affects graphs captured afterwards. */
void gs_set_programmatic_launch(int enable);
int gs_programmatic_launch(void);

/* Number of CUDA kernels this library has enqueued since it was loaded, over all
 * contexts and threads (diagnostics; host-side count, no synchronisation). */
unsigned long long gs_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
