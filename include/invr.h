/*
 * invr.h -- C ABI of the B300 (sm_103a) hot path of Instant-NVR: per-ray-sample
 * evaluation of the deformed hash-grid radiance field (warp -> hash encoding -> MLPs ->
 * volume rendering), forward and training backward.
 *
 * The calls follow the paper's statement of the back-end's problem (Sec. 3 "Neural
 * Rendering Back-end" and Sec. 4.2): per frame the back-end receives the tracked human
 * motion {dq_i^t} on the deformation-graph nodes x_i and the object pose T^t; it keeps a
 * canonical hash-grid radiance field per branch (H^h, E^h_g, E^h_c for the human,
 * H^o, E^o_g, E^o_c for the object), trains them on key-frame rays and renders novel
 * views, combining the two branches by depth (Sec. 4.3).
 *
 * General rules
 *   - Every pointer named *_dev is device memory on the context's device, owned by the
 *     caller; the library never frees it.  Host pointers are named without the suffix.
 *   - Streams are passed as `invr_stream` (a cudaStream_t; NULL = the legacy default
 *     stream).  Calls enqueue work and return; argument errors are reported
 *     synchronously by the return code, device-side conditions (non-finite values) by a
 *     device status word that invr_ctx_sync() reads.
 *   - Handles are not thread-safe; use one handle from one host thread at a time.
 *   - Layouts are structure-of-arrays: rays [3][R], node positions [3][N], node dual
 *     quaternions [8][N] as (real w,x,y,z ; dual w,x,y,z), hash tables [L][T][F], MLP
 *     weights W1..W5 row-major [out][in] concatenated.
 *   - No exception crosses this boundary.  On error the last error text is kept in the
 *     context (invr_last_error_detail).
 */
#ifndef INVR_H
#define INVR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct invr_ctx_s* invr_ctx;     /* device, workspace, status word              */
typedef struct invr_field_s* invr_field; /* hash tables + MLP weights + grads + Adam    */
typedef struct invr_graph_s* invr_graph; /* deformation-graph nodes and per-frame poses */
typedef struct invr_deform_s* invr_deform; /* pose-conditioned deformation net + its optimiser state */
typedef void* invr_stream;               /* cudaStream_t                                */

typedef enum {
    INVR_OK = 0,
    INVR_E_ARG = -1,        /* invalid argument (size, pointer, unsupported shape)   */
    INVR_E_OOM = -2,        /* device allocation failed                               */
    INVR_E_CUDA = -3,       /* a CUDA runtime call failed (text in last_error_detail) */
    INVR_E_TIMEOUT = -4,    /* a bounded device-side wait gave up                     */
    INVR_E_NONFINITE = -5,  /* a kernel produced a NaN/Inf output                      */
    INVR_E_STATE = -6       /* call out of order (e.g. backward without forward)       */
} invr_status;

typedef enum {
    INVR_FP32 = 0,      /* every step in FP32                                        */
    INVR_MLP_FP16 = 1,  /* MLP GEMMs on tensor cores, FP16 operands, FP32 accumulate   */
    INVR_MLP_BF16 = 2   /* MLP GEMMs on tensor cores, BF16 operands, FP32 accumulate   */
} invr_precision;

/* ------------------------------------------------------------------ context */
/* Create a context on CUDA device `device`.  Owns the sample workspace (grown on demand,
 * or sized once by invr_ctx_reserve) and a device status word. */
invr_status invr_ctx_create(invr_ctx* out, int device);
invr_status invr_ctx_destroy(invr_ctx ctx);

/* Size the workspace once for calls of up to max_rays rays in total (summed over views and
 * batches) and max_samples occupied samples per ray on average; afterwards the workspace
 * never grows, so later calls allocate nothing (needed before capturing calls into a CUDA
 * graph).  A call with more rays returns INVR_E_ARG; a call whose occupied samples exceed
 * the reserved slots is detected on the device, skips its sample work and makes the next
 * invr_ctx_sync return INVR_E_STATE. */
invr_status invr_ctx_reserve(invr_ctx ctx, int64_t max_rays, int max_samples);

/* Wait for `stream`, then read and clear the device status word, reporting the first of:
 * INVR_E_TIMEOUT if a bounded device wait gave up, INVR_E_STATE if a call's occupied samples
 * overflowed a reserved workspace, INVR_E_NONFINITE if a kernel flagged a non-finite output
 * since the last sync; else INVR_OK.
 * After a timeout the kernel waits (bounded again) for its own MMAs and copies in flight
 * before it frees its tensor memory.  If that drain finished, the context stays usable: the
 * outputs of the calls since the last sync are undefined, later calls are correct.  If the
 * drain gave up too, the detail text (invr_last_error_detail) says so ("drain"): tensor-core
 * work may then have written tensor or shared memory after the CTA released it, so results
 * of any kernel that shared those SMs are undefined and the context should be destroyed. */
invr_status invr_ctx_sync(invr_ctx ctx, invr_stream stream);

/* Per-kernel timing with CUDA events recorded on the launching stream around every kernel
 * launch of the library (off by default).  enable != 0 starts a new record (clearing the
 * old one).  invr_ctx_timing synchronises the device, then fills up to max entries:
 * names[i] (static strings), total milliseconds ms[i] and launch counts launches[i], one
 * entry per kernel name; it returns the number of entries (or a negative invr_status). */
invr_status invr_ctx_enable_timing(invr_ctx ctx, int enable);
int invr_ctx_timing(invr_ctx ctx, const char** names, double* ms, int64_t* launches, int max);

const char* invr_status_string(invr_status s);
/* Copy the text of the context's last error (NUL-terminated, truncated to n bytes). */
invr_status invr_last_error_detail(invr_ctx ctx, char* buf, size_t n);

/* ------------------------------------------------------------------ fields */
/* One canonical radiance field (Sec. 4.2, "Separated instant neural representation"):
 * a multiresolution hash encoding H (L levels of T = 2^log2_T entries of F features,
 * level resolution floor(N_min growth^l)) feeding the geometry MLP E_g
 * (mlp_in -> mlp_hidden -> mlp_hidden -> geo_out, ReLU, density exp(o_0)) and the colour
 * MLP E_c (o_1..o_{geo_out-1} -> col_hidden -> 3, ReLU then sigmoid), no biases.
 * Supported: L*F = mlp_in in {16, 32}, F = 2, L <= 16, mlp_hidden = col_hidden = 64,
 * geo_out = 16, 10 <= log2_T <= 24.  Other shapes return INVR_E_ARG. */
typedef struct {
    int L, log2_T, F, N_min;
    double growth;
    int mlp_in, mlp_hidden, geo_out, col_hidden;
    invr_precision prec;
} invr_field_desc;

/* Allocates parameters (tables + weights), gradients and Adam moments (zeroed, step 0),
 * and a 36 KB scratch copy of the weights that every FP32 MLP forward on this field
 * rewrites before use (so two calls that evaluate one FP32 field at the same time on
 * different streams must not see different weights).  Parameters are undefined until
 * invr_field_set_params. */
invr_status invr_field_create(invr_ctx ctx, const invr_field_desc* desc, invr_field* out);
invr_status invr_field_destroy(invr_field field);

/* Copy parameters in: tables_dev [L][T][F] and weights_dev (W1..W5) FP32. */
invr_status invr_field_set_params(invr_field field, const float* tables_dev, const float* weights_dev,
                                  invr_stream stream);
/* Copy parameters and optimiser state out; any pointer may be NULL.  Adam moments are laid
 * out as tables then weights (L*T*F + n_weights floats).  *step (host) receives the number
 * of Adam steps taken (read after the stream's prior work completes). */
invr_status invr_field_get_params(invr_field field, float* tables_dev, float* weights_dev, float* adam_m_dev,
                                  float* adam_v_dev, int64_t* step, invr_stream stream);
/* Copy src's parameters (tables and weights, not gradients or Adam state) into dst, on
 * `stream`; both fields must have the same description apart from precision.  Used to give a
 * renderer a snapshot of a field that another stream keeps training. */
invr_status invr_field_copy_params(invr_field dst, invr_field src, invr_stream stream);
/* Copy the accumulated gradients out (same layouts as the parameters); either may be NULL. */
invr_status invr_field_get_grads(invr_field field, float* grad_tables_dev, float* grad_weights_dev,
                                 invr_stream stream);
invr_status invr_field_zero_grads(invr_field field, invr_stream stream);
/* Number of weights of W1..W5 for a description (host-side helper). */
int64_t invr_field_weight_count(const invr_field_desc* desc);

/* ------------------------------------------------------------------ deformation graph */
/* Embedded-deformation graph W = {dq_i, x_i} (Sec. 4.1, Eq. 2): n_nodes canonical nodes,
 * K nearest deformed nodes blended per sample with weights exp(-|v - x_i^t|^2 / radius^2)
 * (radius 0.1 in the paper), poses for n_frames frames.  Requires 1 <= K <= 8,
 * K <= n_nodes <= 65535. */
typedef struct {
    int n_nodes, K;
    float radius;
    int n_frames;
} invr_graph_desc;

invr_status invr_graph_create(invr_ctx ctx, const invr_graph_desc* desc, const float* x_canon_dev,
                              invr_graph* out);
/* Set frame `frame`'s motion (Sec. 4.2, Eq. 4): node dual quaternions dq_dev [8][N]
 * (canonical -> live) and deformed node positions x_live_dev [3][N] (x_i^t = dq_i^t x_i,
 * the tracker's output).  The library copies both and builds, on `stream`, its
 * per-frame nearest-node candidate grid over the live nodes (128^3 cells: sorted lists of
 * up to 64 entries (128 for K > 4) plus a 32-byte head per cell, ~576 MiB per frame at
 * K <= 4, through a 64^3 scratch grid owned by the graph: calls on one graph must be
 * ordered, i.e. issued on one stream or synchronised). */
invr_status invr_graph_set_pose(invr_graph graph, int frame, const float* dq_dev, const float* x_live_dev,
                                invr_stream stream);
invr_status invr_graph_destroy(invr_graph graph);

/* Look-up-table neighbour search (Sec. 4.2, "On-the-fly Radiance Fields"), the paper's
 * approximate O(1) replacement of the K-nearest-node query of the human warp.
 * invr_graph_enable_lut builds, asynchronously on `stream`, a canonical KNN field of
 * resolution^3 voxels over [-1,1]^3 (each voxel's K nearest canonical nodes; 512 in the
 * paper) and, for every frame already posed, a live index field: each canonical voxel
 * centre is carried to live space by the forward warp of Eq. 2 and its index stored in the
 * live voxel it lands in (several: the smallest index; outside the box: dropped).  Every
 * later invr_graph_set_pose rebuilds its frame's live field.  While a graph has tables,
 * warps of views on it take each sample's K nodes from the canonical voxel stored in its
 * live voxel (ordered by live distance, ties to the lower index); samples in a live voxel
 * that received no canonical voxel use the exact search.  Device memory: resolution^3 x K x
 * 2 bytes once plus resolution^3 x 4 bytes per posed frame (1 GiB + 512 MiB per frame at
 * 512 and K = 4).  resolution: a power of two in [4, 1024], else INVR_E_ARG; not during
 * stream capture (INVR_E_STATE).  Calling it again rebuilds at the new resolution.
 * invr_graph_disable_lut frees the tables (after a device synchronisation); warps return
 * to the exact search.  invr_graph_get_lut copies the canonical field ([G^3][K] uint16,
 * voxel x + G (y + G z)) and/or one frame's live field ([G^3] uint32, 0xFFFFFFFF = none)
 * into caller device buffers (either may be NULL); INVR_E_STATE without tables. */
invr_status invr_graph_enable_lut(invr_graph graph, int resolution, invr_stream stream);
invr_status invr_graph_disable_lut(invr_graph graph);
invr_status invr_graph_get_lut(invr_graph graph, int frame, uint16_t* canon_dev, uint32_t* live_dev,
                               invr_stream stream);

/* ------------------------------------------------------------------ rendering */
/* ---------------------------------------------------------- deformation net */
/* Pose-conditioned deformation net (Sec. 4.2, after Eq. 4; sizes of Sec. 4.4): the warped
 * human point v_t = DQB^{-1}(v) v is hash-encoded with the net's own tables (L levels x
 * F = 2 features, 32 in the paper), concatenated with the frame's pose theta (pose_dim,
 * 72), passed through n_hidden ReLU layers of width `hidden` (4 x 128) and a linear layer
 * giving the residual displacement delta v (3); the human field is then evaluated at
 * v_c = v_t + delta v.  No biases.  Weights, row-major [out][in], concatenated:
 * W_1 [hidden][L*F + pose_dim], W_2..W_n [hidden][hidden], W_out [3][hidden].  Training
 * (invr_train_step and its halves) back-propagates through v_c into the net's tables and
 * weights and updates them with the same Adam step as the fields.  Supported: F = 2,
 * L*F a multiple of 8 up to 32, hidden a multiple of 16 up to 128, 1 <= n_hidden <= 4,
 * pose_dim <= 128; else INVR_E_ARG.  prec: INVR_FP32 runs the net in FP32; INVR_MLP_FP16 and
 * INVR_MLP_BF16 run it on the tensor cores with FP16 / BF16 operands and FP32 accumulation,
 * forward and backward
 * (then L*F = 32, hidden = 128, pose_dim <= 80, and one training call takes at most one such
 * net; training keeps ~2.1 KB of operand tiles per sample slot of the workspace).  The net's
 * precision is independent of the field's. */
typedef struct {
    int L, log2_T, F, N_min;
    double growth;
    int pose_dim, hidden, n_hidden;
    invr_precision prec;
} invr_deform_desc;

invr_status invr_deform_create(invr_ctx ctx, const invr_deform_desc* desc, invr_deform* out);
invr_status invr_deform_destroy(invr_deform deform);
/* tables [L][2^log2_T][F] and weights (layout above), device, copied in / out. */
invr_status invr_deform_set_params(invr_deform deform, const float* tables_dev, const float* weights_dev,
                                   invr_stream stream);
invr_status invr_deform_get_params(invr_deform deform, float* tables_dev, float* weights_dev, invr_stream stream);
/* Accumulated gradients (cleared by the Adam step, or by invr_deform_zero_grads). */
invr_status invr_deform_get_grads(invr_deform deform, float* grad_tables_dev, float* grad_weights_dev,
                                  invr_stream stream);
invr_status invr_deform_zero_grads(invr_deform deform, invr_stream stream);

/* One field seen in one frame: the human field through `graph` at `frame` (inverse
 * dual-quaternion-blend warp, Eq. 4), or, when graph == NULL, the object field through
 * the rigid pose rigid_dq (host pointer to 8 floats: unit dual quaternion canonical ->
 * live, Sec. 4.1 "Object Rigid Tracking"; its values are copied at call time).
 * occupancy_dev: live-space 128^3 bitfield over [-1,1]^3 (bit x + 128(y + 128 z) set =
 * occupied; samples in empty cells have zero density and are not evaluated) or NULL. */
typedef struct {
    invr_field field;
    invr_graph graph;
    int frame;
    const float* rigid_dq;
    const uint32_t* occupancy_dev;
    /* pose-conditioned deformation net (human field only; NULL: none) and the pose theta^t
     * of this view's frame (device, deform's pose_dim floats): v_c = v_t + delta v.  The
     * render and training calls run it; the per-point calls (invr_warp_points,
     * invr_query_points, invr_query_points_noalloc, invr_occupancy_update) reject a view
     * that has one with INVR_E_ARG. */
    invr_deform deform;
    const float* pose_dev;
} invr_field_view;

/* Volume rendering of n_rays rays (Sec. 3, "share volumetric rendering"): each ray is
 * clipped to [-1,1]^3 and sampled at n_samples uniform midpoints; per view the samples
 * are composited front to back, stopping after the first sample whose transmittance
 * falls below t_eps.  With two views (view 0 = human, view 1 = object) the nearer field
 * by expected depth is laid over the farther (Sec. 4.3).  Outputs: rgba_dev [4][R]
 * (colour on a black background and opacity) and depth_dev [R] (opacity-weighted depth
 * sum; divide by opacity for the expected depth).  1 <= n_samples <= 1024. */
typedef struct {
    int64_t n_rays;
    const float* o_dev;  /* [3][R] */
    const float* d_dev;  /* [3][R] */
    int n_samples;
    float t_eps;
    int n_views;         /* 1 or 2 */
    const invr_field_view* views;
    float* rgba_dev;     /* [4][R] */
    float* depth_dev;    /* [R]    */
} invr_render_args;

invr_status invr_render_rays(invr_ctx ctx, const invr_render_args* args, invr_stream stream);

/* Joint per-sample compositing of the two views of `args` (n_views = 2: the human field,
 * then the object field), the alternative to laying one field's image over the other's
 * (Sec. 4.3 composes the two images by depth; this mixes them inside the volume): both
 * fields are sampled at the same t_j, densities add and colours mix in proportion to
 * density, sigma = sigma_h + sigma_o, c = (sigma_h c_h + sigma_o c_o) / sigma (a field whose
 * occupancy bit is clear contributes sigma = 0), and the mixture is composited front to
 * back with early termination.  Outputs as invr_render_rays; n_views != 2 is INVR_E_ARG. */
invr_status invr_render_rays_joint(invr_ctx ctx, const invr_render_args* args, invr_stream stream);

/* Density-driven maintenance of a view's 128^3 live-space occupancy bitfield (the layout of
 * invr_field_view.occupancy_dev).  The density at every cell centre ((i + 1/2) 2/128 - 1 per
 * axis) is evaluated through the view's warp (its frame's pose), encoding and MLPs; then per
 * cell density_dev[c] = max(decay * density_dev[c], sigma) and the bit of cell c
 * (x + 128 (y + 128 z); bit c & 31 of word c >> 5) is set iff density_dev[c] > threshold.
 * The view's own occupancy_dev is not read.  density_dev: [128^3] floats, caller-owned,
 * updated in place (start from zeros); bits_dev: [65536] words, written.  The paper takes
 * the occupied space as given; this keeps it current as the fields train and the poses
 * change.  Asynchronous on `stream`; scratch of ~350 MB is taken from the stream-ordered
 * allocator.  decay outside [0, 1] or null pointers: INVR_E_ARG. */
invr_status invr_occupancy_update(invr_ctx ctx, const invr_field_view* view, float decay, float threshold,
                                  float* density_dev, uint32_t* bits_dev, invr_stream stream);

/* ------------------------------------------------------------------ training */
/* Training losses.
 *  INVR_LOSS_HUBER: Huber penalty (threshold huber_delta) of rendered colour minus target,
 *    averaged over all rays of all batches and the 3 channels.
 *  INVR_LOSS_PAPER: the paper's photometric and depth losses (Sec. 4.4, Implementation
 *    Details), summed over all rays of all batches:
 *      sum_r ||M(r) (C_hat(r) - C(r))||_2 + depth_weight * sum_r |M(r) (D_hat(r) - D(r))|
 *    with C_hat the rendered colour, D_hat = sum_j T_j alpha_j t_j the rendered depth,
 *    C(r) the target colour, D(r) the sensor depth and M(r) >= 0 the mask of the field's
 *    actor (human or object, so each field is supervised by its own mask).  Where the
 *    colour error is exactly 0 its gradient is taken as 0; sign(0) = 0 for the depth. */
typedef enum { INVR_LOSS_HUBER = 0, INVR_LOSS_PAPER = 1 } invr_loss;

/* One training step over key-frame ray batches (Sec. 4.2 "On-the-fly Radiance Fields",
 * key frames of Sec. 4.2): each batch is one field seen in one frame (n_views = 1; its
 * rgba_dev/depth_dev may be NULL or receive the rendered values).  targets_dev holds each
 * batch's [3][R_b] target colours back to back; for INVR_LOSS_PAPER, masks_dev (or NULL
 * for M = 1) and depths_dev hold each batch's [R_b] masks and sensor depths back to back.
 * The backward pass recomputes per-sample MLP activations, scatter-adds hash-table
 * gradients, and Adam (lr, beta1, beta2, adam_eps, bias-corrected) then updates every
 * parameter of every field used.  loss_dev (device, 1 float) receives the loss.  At most
 * 16 batches.  An unknown loss, or INVR_LOSS_PAPER without depths_dev, is INVR_E_ARG. */
typedef struct {
    int n_batches;
    const invr_render_args* batches;
    const float* targets_dev;
    float huber_delta;
    float lr, beta1, beta2, adam_eps;
    float* loss_dev;
    int loss;                   /* invr_loss */
    const float* masks_dev;     /* per batch [R_b], back to back; NULL = 1 */
    const float* depths_dev;    /* per batch [R_b], back to back */
    float depth_weight;
} invr_train_args;

invr_status invr_train_step(invr_ctx ctx, const invr_train_args* args, invr_stream stream);

/* The forward and backward halves of invr_train_step, for autograd front ends:
 * forward_train renders every batch, writes loss_dev and keeps the per-sample state in the
 * context's workspace; backward adds dLoss/dparams (scaled by grad_scale) into each
 * field's gradient buffers; invr_field_adam applies one Adam step from the gradient
 * buffer and zeroes it. */
invr_status invr_field_forward_train(invr_ctx ctx, const invr_train_args* args, invr_stream stream);
invr_status invr_field_backward(invr_ctx ctx, const invr_train_args* args, float grad_scale, invr_stream stream);
invr_status invr_field_adam(invr_field field, float lr, float beta1, float beta2, float eps, invr_stream stream);

/* Autotuner of the launch shapes (CTAs per SM of the warp, encoding and gradient-scatter
 * kernels, the level resolution up to which gradient runs are summed per warp before the
 * atomics, whether the forward warps and encodes in one fused kernel per field or in two
 * staged kernels, and the fused kernel's work-item size): coordinate descent, each candidate
 * timed with CUDA events on `stream` over forward_train + backward of `args` (best of 2
 * after a warm-up run).  Parameters are not changed (no Adam step); the gradients it
 * accumulates are cleared.  The chosen shapes are kept in the context for all later calls.
 * Synchronises `stream`; not during capture. */
invr_status invr_ctx_autotune(invr_ctx ctx, const invr_train_args* args, invr_stream stream);
#define INVR_TUNE_N 6
/* The context's launch shapes: out[INVR_TUNE_N] = {warp CTAs/SM, encode CTAs/SM, scatter
 * CTAs/SM, aggregation resolution, fused warp + encoding (1) or staged (0), samples per work
 * item of the fused kernel (128 or 256)}. */
invr_status invr_ctx_get_tune(invr_ctx ctx, int* out);
/* Set the launch shapes directly (e.g. ones an earlier autotune returned): in[INVR_TUNE_N]
 * as for invr_ctx_get_tune.  CTAs per SM in [1, 32], aggregation resolution in [0, 2^20]
 * (0: no level sums runs), fused 0 or 1, work item 128 or 256.  INVR_E_ARG on a value out
 * of range; the context is then unchanged.  Views with a deformation net always run staged.
 * A new context starts at {4, 32, 8, 128, 1, 128}. */
invr_status invr_ctx_set_tune(invr_ctx ctx, const int* in);
/* Polls of each bounded device-side wait (the tensor-core kernels' mbarrier waits) before
 * the kernel gives up, records INVR_E_TIMEOUT in the status word, lets its in-flight work
 * finish (its own drain wait, bounded by 2^22 polls whatever this setting), frees its tensor
 * memory and returns.  Default 2^22 (a few seconds).  0 makes every such wait give up at
 * once, which exercises the failure path without a fault. */
invr_status invr_ctx_set_wait_limit(invr_ctx ctx, uint32_t polls);

/* ------------------------------------------------------------------ single steps */
/* Samples of n_rays rays as the renderer takes them: count_dev [R] occupied samples per
 * ray, t_dev [R][n_samples] and p_dev [3][R][n_samples] hold each ray's occupied samples
 * in its first count slots (remaining slots untouched).  occupancy_dev may be NULL. */
invr_status invr_ray_samples(invr_ctx ctx, int64_t n_rays, const float* o_dev, const float* d_dev, int n_samples,
                             const uint32_t* occupancy_dev, int32_t* count_dev, float* t_dev, float* p_dev,
                             invr_stream stream);
/* Warp n live points p_dev [3][n] to canonical vc_dev [3][n] through `view` (Eq. 4 or
 * the rigid pose).  knn_ids_dev [K][n] (may be NULL) receives the selected node ids,
 * nearest first (human view only). */
invr_status invr_warp_points(invr_ctx ctx, const invr_field_view* view, int64_t n, const float* p_dev,
                             float* vc_dev, int32_t* knn_ids_dev, invr_stream stream);
/* Hash-encode n canonical points x_dev [3][n]: feat_dev [L*F][n]; idx_dev [L*8][n] (may be
 * NULL) receives the table slot of each level's 8 cell corners (bit 0 = +x, 1 = +y, 2 = +z). */
invr_status invr_encode_points(invr_ctx ctx, invr_field field, int64_t n, const float* x_dev, float* feat_dev,
                               uint32_t* idx_dev, invr_stream stream);
/* Evaluate the MLPs on n feature vectors feat_dev [mlp_in][n]: out_dev [4][n] = (sigma,r,g,b). */
invr_status invr_mlp_points(invr_ctx ctx, invr_field field, int64_t n, const float* feat_dev, float* out_dev,
                            invr_stream stream);
/* Warp + encode + MLPs at n live points p_dev [3][n]: out_dev [4][n] = (sigma,r,g,b). */
invr_status invr_query_points(invr_ctx ctx, const invr_field_view* view, int64_t n, const float* p_dev,
                              float* out_dev, invr_stream stream);

/* ------------------------------------------------------------------ no allocation */
/* Not part of the paper's method (the paper has no counterpart): a variant of
 * invr_query_points for callers that cannot call cudaMalloc -- for example code that runs
 * inside a host framework which owns all device memory through its own pool, or a
 * real-time loop where an allocation (and the synchronisation it can imply) is not
 * allowed.  Inputs, outputs and results are those of invr_query_points.  Its scratch
 * (canonical positions and encoding features, (3 + mlp_in) floats per point) lives in one
 * fixed device array of 35 x INVR_NOALLOC_MAX_POINTS floats (9.2 MB) compiled into the
 * library.  invr_ctx_create, which allocates anyway, sets the query up on its device: it
 * looks up the array's device address and loads the code of the kernels the query launches
 * (with lazy module loading both would otherwise happen at the first query).  From then on
 * the device holds the array until the process exits, and the query itself allocates
 * nothing, on its first call too.  All calls share the one array and each call overwrites
 * it: calls that overlap on the GPU (other streams, other host threads) race, so the caller
 * must serialise them.  n > INVR_NOALLOC_MAX_POINTS returns INVR_E_ARG. */
#define INVR_NOALLOC_MAX_POINTS 65536
invr_status invr_query_points_noalloc(invr_ctx ctx, const invr_field_view* view, int64_t n, const float* p_dev,
                                      float* out_dev, invr_stream stream);

/* ---- L2 ceiling probes (measurement helpers; the paper has no counterpart) -------------
 * The hash tables of a field with T = 2^19 (64 MiB) stay resident in L2, so the encoding's
 * gathers and the backward's scatter-add are bound by L2 rather than HBM.  These calls
 * launch one kernel each, asynchronously on `stream`, that the caller times with events:
 *  - invr_probe_l2_read: `passes` coalesced 16-byte reads of every element of buf_dev
 *    (n_floats floats, a multiple of 4, 16-byte aligned; choose n_floats * 4 bytes below
 *    the L2 size and warm it first).  Bytes read = passes * n_floats * 4.  sink_dev: one
 *    float the kernel may write (never, for finite contents of buf_dev).
 *  - invr_probe_l2_atomic: n_ops vector float atomic adds of +1.0 per component, width
 *    4 (16-byte float4) or 2 (8-byte float2), at pseudo-random entries of table_dev
 *    (n_floats floats, a multiple of 4, 16-byte aligned).  Payload = n_ops * width * 4 B.
 *  - invr_probe_l2_gather: n_ops loads of width 8 (32 bytes; table_dev 32-byte aligned and
 *    n_floats a multiple of 8), 4 (float4) or 2 (float2) at the same pseudo-random entries
 *    (the encoding's gathers); sink_dev as for the read probe.
 * Bad sizes or null pointers return INVR_E_ARG. */
invr_status invr_probe_l2_read(invr_ctx ctx, const float* buf_dev, int64_t n_floats, int passes, float* sink_dev,
                               invr_stream stream);
invr_status invr_probe_l2_atomic(invr_ctx ctx, float* table_dev, int64_t n_floats, int width, int64_t n_ops,
                                 invr_stream stream);
invr_status invr_probe_l2_gather(invr_ctx ctx, const float* table_dev, int64_t n_floats, int width, int64_t n_ops,
                                 float* sink_dev, invr_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* INVR_H */
