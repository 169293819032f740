/*
 * libpifu — C ABI of a GB300 (sm_103a) implementation of the pixel-aligned
 * implicit occupancy field, its coarse-to-fine surface localization and
 * mesh-free direct rendering, after Li et al., "Monocular Real-Time
 * Volumetric Performance Capture" (arXiv 2007.13988):
 *
 *   Sec. 3.1, Eq. 1   O(P) = f_O(Phi(P_xy, g_O(I)), P_z)          occupancy
 *   Sec. 3.1, Eq. 2   T(P) = f_T(Phi(P_xy, g_T), Phi(P_xy, g_O), P_z)  colour
 *   Sec. 3.2          "Octree-based Robust Surface Localization"
 *   Sec. 3.2, Eq. 3   "Mesh-free Rendering"
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *   library never frees them and keeps none of them after a call returns.
 *   Host pointers are read during the call only.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Work is enqueued on it; the calls that need a host decision
 *   (pifu_localize, pifu_render) synchronise it internally, the graph forms
 *   once per call, and pifu_frame_async not at all (its device-side errors
 *   wait for pifu_frame_wait).
 * - Every call returns a pifu_status.  Errors detectable on the host return
 *   before any work is enqueued.  A CUDA error returns PIFU_ERR_CUDA and
 *   leaves the context usable only if the CUDA context itself survived.
 * - A context is bound to the device that was current at pifu_create and is
 *   not thread-safe: one thread (or external serialisation) per context.
 * - Feature maps are channel-last [H][W][C], C a multiple of 4, base
 *   address 16-byte aligned.
 * - Volume NDC is [-1, 1]^3.  A level of resolution N (cells per axis) has
 *   N+1 nodes per axis at x_i = -1 + 2 i / N; node (i, j, k) has linear index
 *   (k (N+1) + j) (N+1) + i (x fastest).
 * - calib: 3x4 row-major affine map from volume NDC to the input view
 *   (u, v, z_in); (u, v) index the feature map, z_in is the MLP's depth
 *   input ("P_z" of Eq. 1).
 */
#ifndef PIFU_H
#define PIFU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pifu_ctx pifu_ctx;

typedef enum {
    PIFU_OK = 0,
    PIFU_ERR_ARG = -1,            /* bad pointer, size, alignment or shape      */
    PIFU_ERR_FORMAT = -2,         /* weight blob malformed                       */
    PIFU_ERR_CUDA = -3,           /* a CUDA call failed                          */
    PIFU_ERR_OOM = -4,            /* device allocation failed                    */
    PIFU_ERR_NOT_CONVERGED = -5,  /* conflict loop hit pifu_levels.max_rounds    */
    PIFU_ERR_TIMEOUT = -6,        /* a bounded device wait gave up               */
    PIFU_ERR_STATE = -7,          /* call order violated (e.g. render first)     */
    PIFU_ERR_UNSUPPORTED = -8,    /* valid request outside what is implemented   */
    PIFU_ERR_CAPACITY = -9        /* graph form: a device-side count exceeded a
                                     fixed capacity (use pifu_localize/render)   */
} pifu_status;

typedef enum { PIFU_F32 = 0, PIFU_BF16 = 1 } pifu_dtype;

/* MLP arithmetic.  FP32: plain single precision (SIMT FFMA).  BF16: tcgen05
 * tensor cores, BF16 weights and activations, FP32 accumulation.  MIXED:
 * BF16, then every occupancy within `margin` of 0.5 evaluated again in FP32
 * (the decision threshold is where low precision can change a result).
 * FP8: as BF16, but among f_O's leading hidden layers with at least 512
 * outputs (at full size the 1024- and 512-wide layers, 78% of its
 * arithmetic) the first writes its output in E4M3 (per-tensor scale), and
 * each later one reads it as E4M3 operands against E4M3 weights
 * (per-output-channel scales; kind::f8f6f4) while its input-row columns stay
 * BF16, all with FP32 accumulation; needs pifu_calibrate_fp8 first.  FP8_MIXED: FP8, then the FP32 re-evaluation of
 * MIXED.  The colour MLP runs in BF16 in the FP8 forms. */
typedef enum {
    PIFU_PREC_FP32 = 0,
    PIFU_PREC_BF16 = 1,
    PIFU_PREC_MIXED = 2,
    PIFU_PREC_FP8_MIXED = 3,
    PIFU_PREC_FP8 = 4
} pifu_precision;

/* A channel-last feature map g(I) in device memory: data[(j W + i) C + c]. */
typedef struct {
    const void* data;   /* device pointer, 16-byte aligned                    */
    int32_t H, W, C;    /* H, W >= 1; C a multiple of 4                         */
    int32_t dtype;      /* pifu_dtype: F32, or BF16 (read as float; storage    *
                         * precision only -- the arithmetic is unchanged)      */
} pifu_fmap;

/* Coarse-to-fine schedule (Sec. 3.2): dense evaluation at n0 cells per axis,
 * then num_levels-1 refinements doubling the resolution each time. */
typedef struct {
    int32_t n0;          /* power of two, >= 2                                 */
    int32_t num_levels;  /* 1 .. 8; finest n0 << (num_levels-1) <= 512         */
    int32_t precision;   /* pifu_precision                                     */
    int32_t max_rounds;  /* cap on conflict rounds per level (<= 0: 4096)      */
    float margin;        /* MIXED, FP8_MIXED: FP32 re-evaluation band |o - 0.5| < margin */
    int32_t use_surrogate;    /* 1: coarse levels evaluate the trained f_S first  */
    float surrogate_margin;   /* f_S occupancies within this of 0.5 fall back to f_O */
    int32_t subdivision;      /* pifu_subdivision (0: the method of Sec. 3.2)     */
    float threshold;          /* PIFU_SUBDIV_THRESHOLD: deviation threshold >= 0  */
} pifu_levels;

/* Rule that picks the nodes of a finer level to evaluate (pifu_localize
 * only; the graph forms take METHOD alone).  The two octree baselines the
 * paper compares against in Fig. 3 run one evaluation pass per level, with
 * no dilation and no conflict rounds:
 *  BINARIZED  evaluate the nodes whose tri-linear interpolation of the
 *             binarized coarser level is neither 0 nor 1; the others keep
 *             that 0 / 1;
 *  THRESHOLD  give every node the tri-linear interpolation of the coarser
 *             level's continuous values and evaluate it when those corner
 *             values deviate from their mean by more than `threshold`
 *             (values_dev then holds a value at every node).
 * The acceleration factor of Fig. 3 is (n + 1)^3 / pifu_volume.n_eval. */
typedef enum {
    PIFU_SUBDIV_METHOD = 0,
    PIFU_SUBDIV_BINARIZED = 1,
    PIFU_SUBDIV_THRESHOLD = 2
} pifu_subdivision;

/* Target view of the render: the volume is aligned with it (Sec. 3.2), so
 * pixel (i, j) looks along -z through x = (2i+1)/width - 1,
 * y = (2j+1)/height - 1.
 * final_level 0: the ray samples the localized volume (N cells) at its depth
 * nodes, bilinearly between the four node columns around the pixel.
 * final_level 1: the paper's view-culled final level at twice the localized
 * resolution (Sec. 3.2; square power-of-two images): along each pixel column
 * the binarized localized level is upsampled tri-linearly to the 2N + 1
 * depth nodes of the next level; the nodes behind the nearest fully inside
 * one are shadow nodes; the remaining ambiguous nodes (0 < upsampled < 1) are
 * evaluated with f_O in the localization's arithmetic; the first inside node
 * after binarization and its predecessor give the surface.  No conflict loop
 * runs at this level.  The evaluations are counted in the volume's
 * evals_per_level[num_levels]. */
typedef struct {
    int32_t width, height;
    float background[3];  /* B of Eq. 3                                        */
    int32_t precision;    /* pifu_precision of the colour MLP                   */
    int32_t final_level;  /* 0 or 1 (see above)                                 */
} pifu_camera;

/* Result of pifu_localize: views into context memory, valid until the next
 * pifu_localize or pifu_destroy on the same context.  Bitsets use one
 * 32-bit word row per (k, j): bit i of row (k, j) is word
 * (k (N+1) + j) row_words + (i >> 5), bit (i & 31); padding bits are 0. */
typedef struct {
    int32_t n;                    /* finest resolution (cells per axis)        */
    int32_t num_levels;
    int32_t row_words;            /* ceil((n+1) / 32)                          */
    const uint32_t* occ_bits_dev; /* binarized finest level (o >= 0.5)         */
    const uint32_t* eval_bits_dev;/* nodes the network evaluated at the finest */
    const float* values_dev;      /* dense [(n+1)^3]; meaningful where the eval
                                     bit is set (the network's occupancy)      */
    int64_t n_eval;               /* network evaluations over all levels       */
    int64_t evals_per_level[8];
    int64_t candidates_per_level[8]; /* boundary candidates (before dilation)  */
    int64_t rechecked_per_level[8];  /* MIXED: evaluations redone in FP32       */
    int64_t fallback_per_level[8];   /* surrogate: evaluations redone by f_O    */
    int32_t conflict_rounds[8];
} pifu_volume;

/* Parse a weight blob (host memory, copied) holding the occupancy MLP f_O
 * and the colour MLP f_T, and upload it to the current device.
 * Blob format (little-endian): "PIFU", u32 version = 1, u32 n_nets = 2, then
 * per net: u32 kind (0 occupancy/sigmoid, 1 colour/tanh), u32 d_in,
 * u32 n_layers, f32 leaky slope, u32 widths[n_layers], u32 skip_mask
 * (bit l: layer l reads [h_{l-1}, x]), then per layer f32 W[width][fan_in]
 * row-major and f32 b[width].  Hidden widths must be multiples of 8 and the
 * output width 1 (f_O) or 3 (f_T).
 * The occupancy net may instead be the paper's final CBN + SoftZ network
 * (Appendix, "Depth Representation", Eq. 7, and "Pixel-aligned 3D
 * Lifting", Eq. 8): u32 kind = 2, u32 C (feature channels), u32 n_z (SoftZ
 * channels), u32 K (width), u32 n_blocks, f32 eps, then f32 Wz[K][n_z],
 * bz[K], and per block Gg[K][C], gg[K], Gb[K][C], gb[K], mu[K], var[K]
 * (running statistics), W[K_out][K], b[K_out] with K_out = K except 1 for
 * the last block.  The network computes h = Wz Z + bz, then per block
 * a = ReLU((Gg c + gg) (h - mu) / sqrt(var + eps) + Gb c + gb), h = W a + b,
 * and O = sigmoid(h).  Limits: C and K multiples of 8, n_z >= 2,
 * n_blocks 1 .. 8.  Such a context serves pifu_query, pifu_query_ex (FP32,
 * BF16, MIXED), pifu_localize, pifu_render, pifu_frame and pifu_frames
 * (BF16, MIXED); the FP8 forms and the surrogate return
 * PIFU_ERR_UNSUPPORTED.  The blob is validated completely on the
 * host before any CUDA call.  Errors: PIFU_ERR_FORMAT, PIFU_ERR_UNSUPPORTED
 * (hidden width not a multiple of 8), PIFU_ERR_OOM, PIFU_ERR_CUDA,
 * PIFU_ERR_ARG (null pointers). */
int pifu_create(const void* weight_blob, size_t bytes, pifu_ctx** out);

/* Release the context and all its device memory (after waiting for the
 * device when pifu_frame_async frames are pending).  NULL is a no-op. */
void pifu_destroy(pifu_ctx* ctx);

/* Eq. 1 at m arbitrary points: occ_dev[p] = O(pts_dev[3p .. 3p+2]).
 * pts_dev: device float32 [m][3] in volume NDC; occ_dev: device float32 [m].
 * m = 0 is a no-op.  Asynchronous on `stream`. */
int pifu_query(pifu_ctx* ctx, const pifu_fmap* occ_map, const float calib[12],
               const float* pts_dev, int64_t m, float* occ_dev, void* stream);

/* pifu_query with a choice of MLP arithmetic (pifu_precision).  BF16 and
 * MIXED need hidden widths that are multiples of 64 (else
 * PIFU_ERR_UNSUPPORTED); the FP8 forms need pifu_calibrate_fp8 (else
 * PIFU_ERR_STATE); MIXED and FP8_MIXED re-evaluate occupancies within
 * `margin` (0 .. 0.5) of 0.5 in FP32 and synchronise the stream once per
 * 65,536 points.  A bounded device wait that gave up is reported as
 * PIFU_ERR_TIMEOUT by the next synchronising call. */
int pifu_query_ex(pifu_ctx* ctx, const pifu_fmap* occ_map, const float calib[12],
                  const float* pts_dev, int64_t m, float* occ_dev, int precision, float margin,
                  void* stream);

/* Eq. 2 at m points: rgb_dev[3p + c] = (tanh(f_T) + 1) / 2.  col_map may be
 * NULL when f_T reads only [Phi(g_O), P_z]; otherwise its input is
 * [Phi(g_T), Phi(g_O), P_z].  Asynchronous on `stream`. */
int pifu_query_colour(pifu_ctx* ctx, const pifu_fmap* occ_map, const pifu_fmap* col_map,
                      const float calib[12], const float* pts_dev, int64_t m,
                      float* rgb_dev, void* stream);

/* Sec. 3.2 coarse-to-fine localization of the 0.5 level set of Eq. 1.
 * Level 0 is evaluated densely.  Every finer level binarizes the coarser one
 * at 0.5, interpolates it tri-linearly onto the new nodes, evaluates the
 * nodes whose interpolated value is neither 0 nor 1 together with their
 * 26-neighbourhood, then repeatedly evaluates the unevaluated
 * 26-neighbours of nodes whose binarized prediction disagrees with the
 * binarized interpolation, until there are none.  Unevaluated nodes keep the
 * interpolated 0/1.  Synchronises `stream` (the loop length is decided on
 * the host).  *out receives views of the finest level and the counters.
 * Errors: PIFU_ERR_ARG, PIFU_ERR_NOT_CONVERGED, PIFU_ERR_OOM, PIFU_ERR_CUDA,
 * PIFU_ERR_UNSUPPORTED (precision not available). */
int pifu_localize(pifu_ctx* ctx, const pifu_fmap* occ_map, const float calib[12],
                  const pifu_levels* levels, void* stream, pifu_volume* out);

/* Sec. 3.2 mesh-free render of the last localized volume (Eq. 3).  Each
 * pixel's ray samples the bilinear (x, y) interpolation of the node values
 * at every depth node from the observer (z = +1) backwards; the first sample
 * >= 0.5 marks the surface, whose depth is the linear 0.5 crossing between it
 * and the previous sample (z = +1 if it is the first).  Hit pixels get
 * T(P(q), I) of Eq. 2, misses the background and mask 0.
 * depth_dev: float32 [height][width] (NaN on misses); rgb_dev: float32
 * [height][width][3]; mask_dev: uint8 [height][width].  Any of the three may
 * be NULL if not wanted.  Requires a prior successful pifu_localize
 * (PIFU_ERR_STATE otherwise).  Synchronises `stream`. */
int pifu_render(pifu_ctx* ctx, const pifu_camera* cam, const pifu_fmap* occ_map,
                const pifu_fmap* col_map, const float calib[12], void* stream,
                float* depth_dev, float* rgb_dev, uint8_t* mask_dev);

/* One frame -- pifu_localize followed by pifu_render -- as a CUDA graph
 * (Sec. 3.2: localization, then mesh-free render; one launch per frame).
 * The first call with a given argument set (map pointers and shapes,
 * calibration, levels, camera, output pointers) captures the graph; later
 * calls with the same set relaunch it.  Batch sizes stay on the device: the
 * MLP launches read them from the counters the selection kernels write, and
 * each level's conflict loop is a conditional WHILE node.  The stream is
 * synchronised once, at the end, to read the counters into *out.
 * Tensor-core forms only (levels->precision BF16, MIXED, FP8 or FP8_MIXED;
 * the colour MLP runs in BF16).  Fixed capacities: 1,048,576 points per
 * evaluation batch and pixels per render; a frame that exceeds one
 * returns PIFU_ERR_CAPACITY (its outputs are then invalid and the
 * host-driven pifu_localize + pifu_render handle it).  Other errors as in
 * pifu_localize / pifu_render.  The last volume is then available to
 * pifu_render and pifu_sync_stats as after pifu_localize. */
int pifu_frame(pifu_ctx* ctx, const pifu_fmap* occ_map, const pifu_fmap* col_map,
               const float calib[12], const pifu_levels* levels, const pifu_camera* cam,
               void* stream, float* depth_dev, float* rgb_dev, uint8_t* mask_dev,
               pifu_volume* out);

/* pifu_frame without the host waiting on it (Sec. 3.2's frame, one graph
 * launch; Sec. 4 keeps frames flowing through its pipeline, and this lets a
 * caller enqueue frame i+1 -- and the copies around it -- while frame i
 * runs).  Arguments, the graph, its capture rule and the host-side checks
 * are pifu_frame's; `out` is read by pifu_frame_wait instead.
 * The call returns once the frame's graph is enqueued on `stream`: it does
 * not synchronise the stream and reads no counter.  (The first call with a
 * new argument set still captures the graph; with frames in flight it then
 * waits for them first.)  The frame's device-side errors (a capacity, the
 * round cap, a bounded wait that gave up) are latched on the device and
 * reported by pifu_frame_wait; frames enqueued after a failing one have
 * undefined outputs.  The frames of one context share its workspaces, so
 * they must all go to one stream (stream order serialises them), and no
 * other call may use the context until pifu_frame_wait (pifu_frame returns
 * PIFU_ERR_STATE meanwhile).  Returns PIFU_OK or a host-detected error, in
 * which case nothing was enqueued. */
int pifu_frame_async(pifu_ctx* ctx, const pifu_fmap* occ_map, const pifu_fmap* col_map,
                     const float calib[12], const pifu_levels* levels, const pifu_camera* cam,
                     void* stream, float* depth_dev, float* rgb_dev, uint8_t* mask_dev);

/* Waits for the frames pifu_frame_async enqueued on `stream` since the last
 * wait.  If any of them latched a device-side error, returns the code
 * pifu_frame gives for the union of their error bits (PIFU_ERR_CAPACITY
 * before PIFU_ERR_NOT_CONVERGED before PIFU_ERR_TIMEOUT) and clears them (the
 * device counters are reset, as after a failed pifu_frame); otherwise PIFU_OK.
 * *out (may be NULL) receives the last frame's volume view and counters, as
 * from pifu_frame, and that volume is then available to pifu_render and
 * pifu_sync_stats.  PIFU_ERR_STATE when no frame is pending. */
int pifu_frame_wait(pifu_ctx* ctx, void* stream, pifu_volume* out);

/* ---- Lockstep batch of frames (not in the paper) ------------------------------
 * Localization + render of B independent frames (1 <= B <= 64) that advance
 * together.  Every level's set-up, dilation and compaction runs over all B
 * frames at once.  Every evaluation batch is one device-sized list of
 * (frame, node) keys for all frames, so one persistent tensor-core launch per
 * MLP layer serves all B frames.  A level's conflict loop runs while any
 * frame has a frontier (the rounds of the batch are those of its slowest
 * frame).  Each frame's binarized volume and evaluated set equal what
 * pifu_frame computes for it alone; its values agree to BF16 rounding (a
 * round of at most 256 points, which the MIXED forms evaluate in FP32
 * outright, can be tiny in one form and not in the other).
 * The B frames' pipeline is one CUDA graph, captured per argument set: B, the
 * maps' shapes and types, levels, camera and output pointers.  The map
 * pointers and calibrations are read on the device, so consecutive batches
 * with new maps relaunch the same graph.
 *   occ_maps[f], col_maps[f]  frame f's maps (device pointers; the same shape
 *                             and type for all f; col_maps may be null)
 *   calibs                    B x 12 floats (host), frame f's calibration
 *   depth_dev, rgb_dev, mask_dev  [B][height][width] (rgb x3) device outputs,
 *                             each may be null
 *   out                       B volumes (views into the context, valid until
 *                             the next pifu_frames): per-level evaluation and
 *                             candidate counts of each frame; conflict_rounds,
 *                             rechecked_per_level and fallback_per_level are
 *                             the batch's.
 * Synchronises `stream` once.  Precisions and errors as pifu_frame;
 * PIFU_ERR_CAPACITY when one round's keys exceed the batch capacity
 * (B x 2^18 rounded up to a power of two, between 2^20 and 2^22) or
 * B x width x height exceeds 2^22. */
int pifu_frames(pifu_ctx* ctx, int B, const pifu_fmap* occ_maps, const pifu_fmap* col_maps,
                const float* calibs, const pifu_levels* levels, const pifu_camera* cam,
                void* stream, float* depth_dev, float* rgb_dev, uint8_t* mask_dev,
                pifu_volume* out);

/* ---- Stream of frames through a device work queue (not in the paper) ---------
 * Localization + render of F independent frames (1 <= F <= 4096), held in
 * `slots` concurrent frame slots (1 <= slots <= 16, slots x width x height
 * <= 2^22), in ONE graph launch.  On the device the graph loops over rounds;
 * in each round every slot takes one step of the method (Sec. 3.2) for the
 * frame it holds: a frame taken from the queue evaluates its dense level 0;
 * a level whose frontier is empty advances to the next level (binarize,
 * interpolate, candidates, their 26-ring) or, at the finest level, to the
 * render (Eq. 3) and colour (Eq. 2) of the frame, after which the slot takes
 * the next frame of the queue; otherwise the level runs its next conflict
 * round.  All slots' points of a round -- whatever level each slot is at --
 * go through one gather and one persistent tensor-core launch per MLP layer.
 * So every frame makes the decisions, and runs the conflict rounds, it makes
 * alone (its binarized volume and evaluated set equal pifu_frame's), and a
 * frame that needs few rounds does not wait for the slowest one.
 *   occ_maps[f], col_maps[f]  frame f's maps (device; one shape and type for
 *                             all f; col_maps may be null)
 *   calibs                    F x 12 floats (host)
 *   depth_dev, rgb_dev, mask_dev  [F][height][width] (rgb x3) device
 *                             outputs, each may be null
 *   occ_bits_dev              optional [F][(n+1)^2 row_words] words: each
 *                             frame's binarized finest level (the bitset
 *                             layout of pifu_volume)
 *   out                       F volumes (may be null): per-level evaluation
 *                             and candidate counts and conflict rounds of
 *                             each frame; rechecked_per_level[0] and
 *                             fallback_per_level[0] hold the stream's
 *                             totals; the bitset and value views show the
 *                             last frame each slot held (valid until the
 *                             next pifu_stream) and are null for the others
 *   times                     F entries (may be null): when each frame was
 *                             taken from the queue and when its render
 *                             ended, in ms after the first frame was taken
 *                             (device clock), the slot that held it and the
 *                             rounds the whole stream ran
 * The graph is captured per argument set (F, slots, the maps' shapes and
 * types, levels, camera, output pointers); the map pointers and calibrations
 * are read on the device, so later calls with new maps relaunch it.
 * Synchronises `stream` once.  Precisions as pifu_frame; the CBN + SoftZ
 * network and final_level 1 return PIFU_ERR_UNSUPPORTED.  Errors:
 * PIFU_ERR_ARG, PIFU_ERR_CAPACITY (a round's points beyond the key list,
 * max(2^20, slots x 2^18) rounded up to a power of two), PIFU_ERR_NOT_CONVERGED
 * (a level over max_rounds), PIFU_ERR_STATE, PIFU_ERR_OOM, PIFU_ERR_CUDA. */
typedef struct {
    float admit_ms;          /* taken from the queue, after the first frame was  */
    float done_ms;           /* render finished, after the first frame was taken */
    int32_t slot;            /* the slot that held the frame                     */
    int32_t stream_rounds;   /* rounds the whole stream ran (same for all)        */
} pifu_frame_time;

int pifu_stream(pifu_ctx* ctx, int F, const pifu_fmap* occ_maps, const pifu_fmap* col_maps,
                const float* calibs, int slots, const pifu_levels* levels,
                const pifu_camera* cam, void* stream, float* depth_dev, float* rgb_dev,
                uint8_t* mask_dev, uint32_t* occ_bits_dev, pifu_volume* out,
                pifu_frame_time* times);

/* ---- Tile autotuner (not in the paper) ----------------------------------------
 * Times every tensor-core hidden layer of f_O and f_T (and of f_O's E4M3
 * layers once calibrated) on a batch of `rows` points (128 .. 2^22) with each
 * tile form allowed for it, keeps the fastest, and invalidates captured
 * graphs.  A form is given by its tile code:
 *   64, 128, 256  one CTA per 128-row x BN-column output tile, BN = the code
 *                 (dividing the layer's width);
 *   512           the CTA-pair form: two CTAs (a cluster of 2) share a
 *                 256-row x 256-column tile through cta_group::2 MMAs, each
 *                 holding half of the tile's operands (BF16 layers whose
 *                 width 256 divides).
 * The layer into whose epilogue the last layer is fused keeps its code (BN =
 * its width).  The contents of the activation workspaces are whatever they
 * hold (only the timing matters).  Writes the chosen code and the mean ms per
 * launch of each tuned layer, in order (f_O layers, each E4M3 form before the
 * BF16 form, then f_T), into bn_out / ms_out (up to n_max entries, either may
 * be null) and their number into *n_layers.  Synchronises `stream`. */
int pifu_autotune(pifu_ctx* ctx, int64_t rows, void* stream, int32_t* bn_out, double* ms_out,
                  int n_max, int* n_layers);

/* ---- Layer schedule (not in the paper) ----------------------------------------
 * PIFU_SCHED_PER_LAYER (the default): one launch per tensor-core hidden
 * layer.  PIFU_SCHED_CHAINED: a BF16 batch runs all hidden layers of the
 * network, with the last layer fused, in ONE persistent launch.
 * Rows move through the layers in groups of 128-row blocks, so a layer reads
 * activations the layer before wrote shortly earlier, and the tiles of one
 * layer fill the last wave of another.  It applies when the last layer can be
 * fused, the network has at most 4 hidden layers whose widths sum to at most
 * 2048, and no layer uses the CTA-pair form; otherwise the per-layer
 * launches run.  The results are the same bits either way.  Invalidates
 * captured graphs; no device work.  Errors: PIFU_ERR_ARG. */
enum pifu_schedule { PIFU_SCHED_PER_LAYER = 0, PIFU_SCHED_CHAINED = 1 };
int pifu_set_schedule(pifu_ctx* ctx, int schedule);

/* Arithmetic of the MIXED forms' FP32 passes: the re-evaluation of
 * occupancies within the margin of 0.5 and batches of at most 256 points
 * (not in the paper, which evaluates every point once; Sec. 3.2 needs only
 * the decision at 0.5 to be the network's).
 *   PIFU_RECHECK_TENSOR (default): a pass of more than 192 points runs f_O's
 *     hidden layers on the tensor cores with every FP32 operand split into
 *     two TF32 values, hi = tf32(v) and lo = tf32(v - hi), and each product
 *     formed as hi*hi + hi*lo + lo*hi (Ootomo and Yokota's split-TF32
 *     method), FP32 accumulation and an FP32 last layer: within about 2e-5
 *     of the FP64 network in occupancy (the FP32 SIMT network: about 1e-6).
 *     The whole network is one cooperative launch.  Needs hidden widths
 *     that are multiples of 128, the last one 128 wide, and a one-output
 *     last layer reading only it.  A pass of at most 64 points runs the
 *     network in FP32 FFMA as one cooperative launch over every SM (each
 *     hidden layer's neurons split over the SMs, a grid barrier between
 *     layers), whose latency is the lowest there; passes between the two
 *     sizes, and networks neither form takes (and the CBN network), use
 *     the FP32 form's SIMT network.
 *     The first MIXED call of a context reserves its workspace: 16,384
 *     points x (2 d_in + 4 widest hidden width) floats, 256 points x 2
 *     widest hidden width floats, plus 17 MB.
 *   PIFU_RECHECK_SIMT: the FP32 form's SIMT network (FFMA, clusters of
 *     CTAs) for every pass.
 *   PIFU_RECHECK_TENSOR_ALL: the split-TF32 network for every pass, small
 *     ones included (where PIFU_RECHECK_TENSOR allows it).
 * Invalidates captured graphs; no device work.  Errors: PIFU_ERR_ARG. */
enum pifu_recheck { PIFU_RECHECK_TENSOR = 0, PIFU_RECHECK_SIMT = 1, PIFU_RECHECK_TENSOR_ALL = 2 };
int pifu_set_recheck(pifu_ctx* ctx, int form);

/* Test hook for the bounded device waits (not in the paper).  With starve =
 * 1, two cross-CTA waits each wait for one arrival more than there are: the
 * split-TF32 kernels' split-K wait (the units of a tile waiting for each
 * other's partial tiles) and the whole-GPU FP32 kernel's grid barrier (which
 * then issues each layer's weight copies after the barrier, so no bulk copy
 * or MMA is in flight at either wait).  Each gives up after a few thousand
 * polls and latches the context's error word; the next synchronising call
 * returns PIFU_ERR_TIMEOUT and puts the kernels' counters back, so the
 * context stays usable.  starve = 0 (the default)
 * restores normal operation.  Results computed while starving are not
 * meaningful.  Invalidates captured graphs; no device work.  Errors:
 * PIFU_ERR_ARG. */
int pifu_test_starve_wait(pifu_ctx* ctx, int starve);

/* Sets the tile code of every tuned layer, in pifu_autotune's order: codes[i]
 * for layer i, n = the number of layers pifu_autotune reports (for instance a
 * saved autotuner result).  A code must be allowed for its layer as above
 * (E4M3 forms: 64, 128 or 256); the fused layer must keep its code.  Results
 * do not depend on the codes.  Invalidates captured graphs; no device work.
 * Errors: PIFU_ERR_ARG (n or a code not allowed; nothing is changed). */
int pifu_set_tiles(pifu_ctx* ctx, const int32_t* codes, int n);

/* ---- FP8 form of f_O (not in the paper) --------------------------------------
 * Calibrates and builds the FP8 layers used by PIFU_PREC_FP8 and
 * PIFU_PREC_FP8_MIXED: f_O's hidden outputs that an E4M3 layer reads are
 * evaluated in FP32 at the (n0+1)^3 nodes of the dense coarsest grid of this
 * feature map and calibration; their activation scales are their absolute
 * maxima / 448 (the largest E4M3 value; larger values saturate).  A later
 * layer's E4M3 weights are divided by their per-output-channel absolute
 * maxima / 448 (s_w), its BF16 input-row weights by s_w times the scale of
 * its E4M3 input, so that both segments share one accumulator, multiplied
 * back in the epilogue.  The scales stay with the context until the next
 * call.  Synchronises `stream`.
 * Errors: PIFU_ERR_ARG (map/calibration/n0), PIFU_ERR_UNSUPPORTED (f_O has no
 * tensor-core form, or fewer than two leading hidden layers with >= 512
 * outputs whose widths are multiples of 128), PIFU_ERR_CUDA / PIFU_ERR_OOM. */
int pifu_calibrate_fp8(pifu_ctx* ctx, const pifu_fmap* occ_map, const float calib[12], int n0,
                       void* stream);

/* ---- Learned surrogate f_S (not in the paper) -------------------------------
 * A small MLP of f_O's family, f_S: d_in -> h1 -> h2 -> 1 (leaky-ReLU,
 * sigmoid, no skips), distilled from f_O and used by pifu_localize at the
 * coarse levels (pifu_levels.use_surrogate): points whose f_S occupancy lies
 * within surrogate_margin of 0.5 are evaluated again by f_O; the finest level
 * always uses f_O.  Trained by the library's kernels: FP32 forward, the mean
 * binary cross-entropy of Sec. 3.1 against f_O's occupancy, back-propagation
 * and Adam (beta 0.9 / 0.999, eps 1e-8; the optimiser of the appendix).
 * Parameters are exchanged in the blob's order: per layer W[n_out][fan_in]
 * row-major, then b[n_out]. */

/* Create (or re-create) f_S with Kaiming-uniform weights from `seed` and
 * zero biases; h1, h2 multiples of 64 in 64 .. 1024. */
int pifu_surrogate_init(pifu_ctx* ctx, int h1, int h2, uint64_t seed);

/* Distillation tuples at m points: x_dev [m][ldx] float32 receives the rows
 * f_O and f_S read ([Phi(g_O), P_z] zero-padded to ldx = d_in rounded up to
 * 8), o_dev [m] f_O's occupancy in FP32.  Asynchronous on `stream`. */
int pifu_surrogate_samples(pifu_ctx* ctx, const pifu_fmap* occ_map, const float calib[12],
                           const float* pts_dev, int64_t m, float* x_dev, float* o_dev,
                           void* stream);

/* f_S's occupancy at m points (as pifu_query_ex, precision FP32 or BF16). */
int pifu_surrogate_query(pifu_ctx* ctx, const pifu_fmap* occ_map, const float calib[12],
                         const float* pts_dev, int64_t m, float* occ_dev, int precision,
                         void* stream);

/* Loss and gradient of f_S on one batch (x_dev [B][ldx], y_dev [B] targets in
 * [0, 1]); grad_host (may be NULL) receives the gradient in the parameter
 * order, loss_host the mean BCE.  Synchronises `stream`. */
int pifu_surrogate_grad(pifu_ctx* ctx, const float* x_dev, const float* y_dev, int64_t B,
                        float* grad_host, double* loss_host, void* stream);

/* `steps` Adam steps with learning rate lr over consecutive batches of
 * `batch` rows of (x_dev, y_dev) (m rows, wrapping around); loss_host[0] and
 * [1] receive the first and the last batch loss.  Synchronises `stream`. */
int pifu_surrogate_train(pifu_ctx* ctx, const float* x_dev, const float* y_dev, int64_t m,
                         int batch, int steps, float lr, double* loss_host, void* stream);

/* Point OHEM (Sec. 3.3, Eq. 6) for f_S's training tuples: every tuple m
 * carries w_m = 1 / (exp(-L_BCE(m) / alpha) + beta), the inverse of its
 * sampling probability, recomputed from its loss whenever it is in a batch;
 * batches are drawn with probability w_m / sum w (inverse-CDF search of the
 * float64 prefix sums, one splitmix64 uniform per draw from the counter
 * seed ^ (step << 32) ^ draw, top 53 bits).
 * pifu_surrogate_ohem_init: weights of m tuples set to 1 (after
 * pifu_surrogate_init, which drops them).  pifu_surrogate_ohem_weights:
 * host copy of the m weights (set = 0) or upload (set = 1).
 * pifu_surrogate_ohem_sample: B indices into idx_dev by the current weights
 * for (seed, step).  pifu_surrogate_train_ohem: as pifu_surrogate_train with
 * the batches drawn so, re-weighting each drawn tuple from its loss under the
 * parameters before that step's Adam update; needs the weights for the same
 * m.  The paper's constants are alpha = 0.7, beta = 0. */
int pifu_surrogate_ohem_init(pifu_ctx* ctx, int64_t m);
int pifu_surrogate_ohem_weights(pifu_ctx* ctx, float* host, int64_t n, int set);
int pifu_surrogate_ohem_sample(pifu_ctx* ctx, uint64_t seed, int step, int B, int* idx_dev,
                               void* stream);
int pifu_surrogate_train_ohem(pifu_ctx* ctx, const float* x_dev, const float* y_dev, int64_t m,
                              int batch, int steps, float lr, float alpha, float beta,
                              uint64_t seed, double* loss_host, void* stream);

/* Copy f_S's n parameters to (set = 0) or from (set != 0) host memory;
 * n must equal the parameter count. */
int pifu_surrogate_params(pifu_ctx* ctx, float* host, int64_t n, int set);

/* Copy the counters of the last pifu_localize into *out (host). */
int pifu_sync_stats(pifu_ctx* ctx, pifu_volume* out);

/* Static description of a status code. */
const char* pifu_status_string(int status);

/* Kernel classes counted and timed by the profiler. */
typedef enum {
    PIFU_K_GATHER = 0,      /* projection + bilinear gather (MLP input rows)      */
    PIFU_K_MLP_HIDDEN = 1,  /* hidden MLP layers on the tensor cores (tcgen05)    */
    PIFU_K_MLP_LAST = 2,    /* last MLP layer + activation + epilogue             */
    PIFU_K_LEVEL = 3,       /* level set-up (dense set-up / classify, popcount)   */
    PIFU_K_SELECT = 4,      /* 26-dilation, selection and compaction              */
    PIFU_K_RENDER = 5,      /* ray first crossing                                 */
    PIFU_K_MLP_F32 = 6,     /* hidden MLP layers in FP32 (SIMT FFMA)              */
    PIFU_K_CBN_TC = 7,      /* the CBN + SoftZ occupancy network on tcgen05       */
    PIFU_K_COUNT = 8
} pifu_kernel_class;

/* Per-class totals since the last pifu_profile call.  `launches` counts
 * every kernel launch of the class (always on).  `ms` sums CUDA-event
 * durations measured on the launching stream around each launch (profiling
 * on only).  `flops` and `bytes` are the ALGORITHMIC work of those launches
 * (unpadded MLP shapes: 2 K N flops per point and layer; bitset, value and
 * output bytes a launch must move at least), for roofline fractions. */
typedef struct {
    int64_t launches;
    double ms;
    double flops;
    double bytes;
} pifu_kernel_stats;

/* Reset the counters and switch event timing on (enable != 0) or off. */
int pifu_profile(pifu_ctx* ctx, int enable);

/* Resolve pending timing events (waits for them) and copy the totals of all
 * PIFU_K_COUNT classes into out[0 .. PIFU_K_COUNT). */
int pifu_profile_read(pifu_ctx* ctx, pifu_kernel_stats* out);

/* Occupancy query that allocates nothing (the paper has no counterpart; this
 * is a deployment aid).  It is meant for callers that cannot call cudaMalloc
 * -- code embedded in an application whose own allocator owns all device
 * memory, or running where device allocation is not permitted -- and so
 * cannot create a context either (pifu_create allocates).
 *
 * Same result as pifu_query: occ_dev[p] = O(pts_dev[3p .. 3p+2]) (Eq. 1),
 * with the occupancy MLP read from weight_blob_dev, a device copy of the
 * weight blob (format as in pifu_create) placed by the caller in memory it
 * owns (4-byte aligned, not modified).  weight_blob is the host copy of the
 * same bytes, read for the layer shapes only.  pts_dev, occ_dev and the map
 * are the caller's, as in pifu_query.  Asynchronous on `stream`.
 *
 * Scratch: the MLP activations use one fixed 16 MiB device array inside the
 * library, which every GPU that loads the library holds until the process
 * exits.  It bounds the points of one call: m <= 4194304 / (ldx + 2 h)
 * with ldx = d_in rounded up to 8 and h the widest hidden layer (1,814
 * points for the 257-1024-512-256-128-1 network, 14,169 for 33-128-64-1);
 * a larger m returns PIFU_ERR_ARG before any work is enqueued.
 * All calls share the array: calls that overlap on the GPU (other streams,
 * other threads) race and must be serialised by the caller.  Each call looks
 * the array's device address up (cudaGetSymbolAddress) on the current device
 * (inside a stream capture: the address its last call outside one found);
 * make the first call on a device before any stream capture.  With CUDA's
 * lazy module loading (the default), the first call on a device also loads
 * the library's device code and its static arrays there, the 16 MiB array
 * included: make it while that much device memory is still free (for
 * instance before the application's allocator reserves the rest).  Apart
 * from that one-time load no call allocates memory, host or device.
 * Errors: PIFU_ERR_ARG, PIFU_ERR_FORMAT, PIFU_ERR_UNSUPPORTED (bf16 map),
 * PIFU_ERR_CUDA. */
int pifu_query_noalloc(const void* weight_blob, size_t bytes, const void* weight_blob_dev,
                       const pifu_fmap* occ_map, const float calib[12],
                       const float* pts_dev, int64_t m, float* occ_dev, void* stream);

/* Text of the last CUDA error seen by this context ("" if none).  The
 * pointer stays valid until the next call on the context. */
const char* pifu_last_error(const pifu_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PIFU_H */
