// Internal structures and device helpers of the sm_103a hot path.
//
// Every launch receives a `Plan` by value (__grid_constant__): the view table (one entry
// per field-in-a-frame), the sample-workspace pointers and the sizes.  Nothing is copied
// host->device per call, so a whole render or train step can be captured in a CUDA graph.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace invr {

constexpr int kMaxViews = 16;   // batches per call (8 key frames x 2 fields)
constexpr int kMaxL = 16;       // hash levels
constexpr int kWtF32 = 9216;    // floats of the FP32 MLP's padded transposed weights
// A 16-bit field's MLP weights as the render forward's and the backward's shared-memory image:
// W1..W5 (padded) as 16-bit K-major operands.
constexpr int kW16Bytes = 18432;
constexpr int kF = 2;           // features per level
constexpr int kMaxIn = kMaxL * kF;
constexpr int kHidden = 64;
constexpr int kGeoOut = 16;
constexpr int kColHidden = 64;
constexpr int kOccRes = 128;    // occupancy grid resolution over [-1,1]^3
constexpr int kTile = 128;      // sample tile: every view's sample range is padded to it
constexpr int kKnnG = 128;      // nearest-node candidate grid resolution over [-1,1]^3
constexpr uint16_t kKnnOverflow = 0xFFFF;
// Candidate-list entries are (r bound << 16) | node id; ids are < 65535, so id 0xFFFF marks
// the end of a list (kKnnEnd) and, in a cell's head with bound 0, a list that overflowed its
// capacity (kKnnHeadOverflow: the cell's points scan every node).
constexpr uint32_t kKnnEnd = 0xFFFFFFFFu;
constexpr uint32_t kKnnHeadOverflow = 0x0000FFFFu;
constexpr int kKnnHead = 8;     // entries of a cell's list kept in its 32-byte head
constexpr int kKnnMaxCap = 128;  // largest candidate list capacity (a multiple of 32)
constexpr int kRayBitWords = 32;   // 1024 samples per ray at most
constexpr uint32_t kLutEmpty = 0xFFFFFFFFu;
constexpr int kTicketSlots = 16;   // work counters: one per persistent launch kind
constexpr int kTicketSplitFwd = 0;   // + 1 for the FP16 instantiation
constexpr int kTicketWarp = 2;       // k_warp's chunks
constexpr int kLossHuber = 0;      // values of invr_loss
constexpr int kLossPaper = 1;

// Device status word bits (read and cleared by invr_ctx_sync).
constexpr unsigned kStatusNonFinite = 1u;
constexpr unsigned kStatusTimeout = 2u;
constexpr unsigned kStatusOverflow = 4u;
// A kernel whose bounded wait gave up then waits (bounded again) for its own MMAs and copies
// in flight before it frees its tensor memory; this bit says that second wait gave up too,
// so that work may still have been writing the CTA's tensor and shared memory as it exited.
constexpr unsigned kStatusDrainTimeout = 8u;

enum MlpKind : int { kMlpF32 = 0, kMlpF16 = 1, kMlpBF16 = 2 };

struct FieldDev {
  const float* tables;      // [L][T][F]
  const float* weights;     // W1..W5 FP32, row-major [out][in]
  float* wt_f32;            // [9216]: the FP32 MLP's padded weights, transposed per layer (written
                            // by each FP32 forward launch from `weights`), or null
  uint8_t* w16;             // [kW16Bytes]: a 16-bit field's weight image (written from `weights` before
                            // each tensor-core forward), or null
  float* grad_tables;       // [L][T][F]
  float* grad_weights;      // W1..W5
  int L, log2T, mlp_in, mlp_kind;
  int res[kMaxL];           // level resolutions N_l
  uint32_t dense_mask;      // bit l: level l stored densely
};

struct WarpDev {
  int mode;                 // 0 = rigid pose, 1 = dual-quaternion blend of K nodes
  float R[9];               // rigid: rotation (row-major) and translation of the pose
  float t[3];
  const float4* x_live;     // [N] (x, y, z, 0)
  const float4* dq;         // [N][2] (real, dual)
  const uint32_t* cand;     // [G^3][cap] candidate entries per grid cell: (r bound << 16) | node id, ascending,
                            // kKnnEnd after the last one (when shorter than cap)
  const uint32_t* cand_head;  // [G^3][kKnnHead] the first entries of each cell's list (kKnnEnd past its
                              // end; kKnnHeadOverflow: scan all nodes); null: no grid
  int n_nodes, K, cap;
  float inv_r2;             // 1 / radius^2
  // look-up-table neighbour search (Sec. 4.2); lut_live == null: exact search
  int lut_res;              // G
  const uint16_t* lut_canon;  // [G^3][K] canonical KNN field
  const uint32_t* lut_live;   // [G^3] live voxel -> canonical voxel, kLutEmpty = none
};

// Pose-conditioned deformation net of a human view (Sec. 4.2): its hash encoding, FP32
// weights W_1 [hidden][n_feat + pose_dim], W_2..W_n [hidden][hidden], W_out [3][hidden].
struct DeformDev {
  const float* weights;
  float* grad_weights;
  float* dw_scratch;        // [num_sms][n_w]: per-CTA weight-gradient partials of the backward
  const float* pose;        // [pose_dim] theta of the view's frame
  float* pose_bias;         // [hidden] W_1[:, n_feat:] theta (computed per call)
  FieldDev enc;             // the net's own hash encoding (F = 2; mlp_kind F32, mlp_in = n_feat)
  int n_feat, pose_dim, hidden, n_hidden, n_w;
  int tc;                   // 0: FP32 SIMT; on the tensor cores with 1: FP16, 2: BF16 operands
};

struct ViewDev {
  const float* o;           // [3][n_rays]
  const float* d;           // [3][n_rays]
  const uint32_t* occ;      // 128^3 bits or null
  const float* target;      // [3][n_rays] (training) or null
  const float* mask;        // [n_rays] M(r) of the paper's losses, or null (= 1)
  const float* depth_target;  // [n_rays] sensor depth of the paper's depth loss
  float* rgba_out;          // [4][n_rays] per-view output (training) or null
  float* depth_out;         // [n_rays] or null
  int64_t n_rays;
  int64_t ray_begin;        // first global ray index of this view
  int scan_block_begin;     // first scan block of this view
  FieldDev field;
  WarpDev warp;
  int has_deform;
  DeformDev deform;
};

struct Workspace {
  int32_t* ray_count;       // [R] occupied samples per ray
  uint32_t* ray_bits;       // [kRayBitWords][R_cap] occupancy bit of every sample of the ray
  int32_t* ray_first;       // [R] first sample slot of the ray
  int32_t* ray_used;        // [R] samples composited (early termination)
  float* ray_out;           // [5][R] C, A, D per global ray
  int32_t* block_sums;      // [n_scan_blocks]
  int32_t* view_base;       // [kMaxViews + 1] padded sample base per view; [n_views] = total
  int32_t* view_count;      // [kMaxViews] occupied samples per view (before padding)
  int32_t* occ_box;         // [kMaxViews][6] bounds of the occupied cells per view (lo xyz, -hi xyz)
  int32_t* s_ray;           // [S] global ray id of each sample, -1 = padding
  float* s_t;               // [S] sample depth t_j
  float* s_pos;             // [3][S] live position
  float* s_vc;              // [3][S] canonical position
  void* feat;               // [kMaxIn][S] FP32 feature-major, or 16-bit tiles (feat16_offset)
  float* out;               // [4][S] sigma, r, g, b
  float* dout;              // [4][S] dL/d o_0, dL/d z_rgb
  float* dfeat;             // [mlp_in][S]
  uint32_t* mlp_mask;       // [6][S] training: ReLU decisions of H1, H2, H4 (tensor-core fields)
  float* loss_part;         // [n loss blocks]
  uint32_t* tickets;        // [kTicketSlots] work counters of the persistent kernels (zeroed before each launch)
  // deformation net (allocated when a call has one)
  float* s_vt;              // [3][S] v_t, the warp before the net
  float* feat_d;            // [n_feat][S] the net's hash features
  float* dvc;               // [3][S] dL/dv_c (scaled like dfeat)
  float* dfeat_d;           // [n_feat][S] dL/d(net features)
  // tensor-core training of a net: per 128-sample tile, 16-bit operand tiles in the
  // K-major MMA layout (32 KB per [128 x 128] tile; tile T of layer l at l * S_cap/128 + T)
  uint8_t* def_x;           // [S/128] x [128 x 32]  the net's input features
  uint8_t* def_h;           // [kDeformMaxLayers][S/128] x [128 x 128]  ReLU outputs h_1..h_n
  uint8_t* def_g;           // [kDeformMaxLayers][S/128] x [128 x 128]  dL/d(pre-activation) of h_1..h_n
  uint8_t* def_gout;        // [S/128] x [128 x 16]  dL/d(delta v), padded to 16 columns
  int64_t S_cap;            // sample slots
  int64_t R_cap;            // ray slots
};

// Launch shapes the autotuner chooses: CTAs per SM of the grid-stride kernels.
struct Tune {
  int warp_ctas_per_sm = 4;
  int encode_ctas_per_sm = 32;
  int encode_bwd_ctas_per_sm = 8;
  int agg_res = 128;
  int fused = 1;            // warp + encoding in one kernel per field (k_warp_encode), else staged
  int chunk = 128;          // samples per work item of the fused kernel (128 or 256)
};

struct Plan {
  int n_views;
  int n_samples;
  float t_eps;
  int n_scan_blocks;
  int64_t total_rays;
  float loss_norm;          // Huber: 1 / (3 * total_rays); the paper's losses: 1
  float huber_delta;
  int loss_kind;            // INVR_LOSS_HUBER or INVR_LOSS_PAPER
  float depth_weight;
  float grad_scale;
  int agg_res;              // levels with N_l <= agg_res aggregate gradient runs per warp
  int view_lo, view_hi;     // views processed by the per-field launches ([0, n_views) by default)
  int has_deform;           // some view has a deformation net
  int deform_store;         // training: the tensor-core forward keeps its operand tiles
  int feat_split;           // training: 16-bit fields' features also as remainder tiles
  int march_coop;           // training: the march count tests a warp's rays in turn (rays in random order)
  uint32_t wait_limit;      // polls per bounded device wait
  Tune tune;                // launch shapes (autotuned per context)
  Workspace ws;
  unsigned* status;         // device status word
  ViewDev v[kMaxViews];
};

// ------------------------------------------------------------------ FP32 recipes
// The discrete decisions (sample positions, occupancy cell, hash cell, nearest-node key)
// use explicitly rounded single-precision operations (no contraction into FMA), so that
// they are reproducible by any implementation performing the same rounded operations.

__device__ __forceinline__ bool ray_box(float3 o, float3 d, int n_samples, float& tn, float& dt) {
  float tnear = -INFINITY, tfar = INFINITY;
  const float oo[3] = {o.x, o.y, o.z};
  const float dd[3] = {d.x, d.y, d.z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (dd[a] == 0.0f) {
      if (oo[a] < -1.0f || oo[a] > 1.0f) return false;
      continue;
    }
    float t0 = __fdiv_rn(__fsub_rn(-1.0f, oo[a]), dd[a]);
    float t1 = __fdiv_rn(__fsub_rn(1.0f, oo[a]), dd[a]);
    float lo = t0 < t1 ? t0 : t1;
    float hi = t0 < t1 ? t1 : t0;
    if (lo > tnear) tnear = lo;
    if (hi < tfar) tfar = hi;
  }
  tn = tnear > 0.0f ? tnear : 0.0f;
  if (!(tfar > tn)) return false;
  dt = __fdiv_rn(__fsub_rn(tfar, tn), (float)n_samples);
  return true;
}

__device__ __forceinline__ float sample_t(float tn, float dt, int j) {
  return __fadd_rn(tn, __fmul_rn(__fadd_rn((float)j, 0.5f), dt));
}

__device__ __forceinline__ float3 sample_p(float3 o, float3 d, float t) {
  return make_float3(__fadd_rn(o.x, __fmul_rn(t, d.x)), __fadd_rn(o.y, __fmul_rn(t, d.y)),
                     __fadd_rn(o.z, __fmul_rn(t, d.z)));
}

__device__ __forceinline__ int grid_cell(float x, int res) {
  float q = __fmul_rn(__fmul_rn(__fadd_rn(x, 1.0f), 0.5f), (float)res);
  int i = (int)floorf(q);
  return i < 0 ? 0 : (i > res - 1 ? res - 1 : i);
}

__device__ __forceinline__ bool occupied(const uint32_t* bits, float3 p) {
  uint32_t idx = (uint32_t)grid_cell(p.x, kOccRes) +
                 kOccRes * ((uint32_t)grid_cell(p.y, kOccRes) + kOccRes * (uint32_t)grid_cell(p.z, kOccRes));
  return (__ldg(bits + (idx >> 5)) >> (idx & 31u)) & 1u;
}

// Hash-level cell of one coordinate: u = clamp((x+1)/2, 0, 1), q = u N, c = min(floor q, N-1)
// (the FP32 decision).  The fraction q - c is evaluated as x N/2 + (N/2 - c) with a single
// rounding (N/2 - c is exact), so it is accurate to ~1e-7 even where q ~ 2000 has an FP32
// spacing of 1.2e-4; it may fall a rounding step outside [0,1] next to a cell boundary,
// where the trilinear blend is continuous.
__device__ __forceinline__ int level_cell(float x, int res, float& frac) {
  float u = __fmul_rn(__fadd_rn(x, 1.0f), 0.5f);
  u = fminf(fmaxf(u, 0.0f), 1.0f);
  float q = __fmul_rn(u, (float)res);
  int c = (int)floorf(q);
  c = c > res - 1 ? res - 1 : c;
  const float half = 0.5f * (float)res;
  const float xc = fminf(fmaxf(x, -1.0f), 1.0f);
  frac = __fmaf_rn(xc, half, half - (float)c);
  return c;
}

__device__ __forceinline__ uint32_t vertex_index(uint32_t x, uint32_t y, uint32_t z, int res, bool dense,
                                                 uint32_t tmask) {
  if (dense) {
    uint32_t n = (uint32_t)res + 1u;
    return x + y * n + z * n * n;
  }
  return ((x * 1u) ^ (y * 2654435761u) ^ (z * 805459861u)) & tmask;
}

__device__ __forceinline__ float knn_key(float3 p, float4 x) {
  float dx = __fsub_rn(p.x, x.x), dy = __fsub_rn(p.y, x.y), dz = __fsub_rn(p.z, x.z);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// View of a global ray / of a padded sample slot (linear search over <= 16 views).
__device__ __forceinline__ int view_of_ray(const Plan& P, int64_t g) {
  int v = 0;
  while (v + 1 < P.n_views && g >= P.v[v + 1].ray_begin) ++v;
  return v;
}

__device__ __forceinline__ int view_of_slot(const int32_t* view_base, int n_views, int64_t s) {
  int v = 0;
  while (v + 1 < n_views && s >= view_base[v + 1]) ++v;
  return v;
}

// View cursor for slots visited in increasing order (a CTA's tiles): advances v to the view
// of slot s, reading the view bases from a copy in shared memory.
__device__ __forceinline__ int advance_view(const int32_t* vb, int n_views, int64_t s, int v) {
  while (v + 1 < n_views && s >= (int64_t)vb[v + 1]) ++v;
  return v;
}

__device__ __forceinline__ void flag_status(unsigned* status, unsigned bit) { atomicOr(status, bit); }

// Grid-stride walk over the work items b = chunk * L + l (level fastest) of the encoding
// kernels, b = blockIdx.x, blockIdx.x + gridDim.x, ..., kept as (chunk, l) so that no step
// divides.
struct ItemWalk {
  int64_t chunk;
  int l, L, dc, dl;
  __device__ __forceinline__ explicit ItemWalk(int levels)
      : chunk(blockIdx.x / levels), l(blockIdx.x % levels), L(levels), dc(gridDim.x / levels), dl(gridDim.x % levels) {}
  __device__ __forceinline__ void next() {
    chunk += dc;
    l += dl;
    if (l >= L) {
      l -= L;
      ++chunk;
    }
  }
};

// 16-bit encoding features of a tensor-core field.  Each 128-sample tile T is the first
// MMA's A operand [128 x K] (K = mlp_in) in the K-major no-swizzle layout: 16 row groups of
// 8 samples, K * 16 bytes each.  Row group g of tile T sits at byte g * 4 * S_cap + T * 512
// of the feature buffer, inside the columns that the FP32 feature-major layout gives the
// same samples, so views of different precisions in one call never overlap; with S_cap a
// multiple of kTile every row group starts on a 16-byte boundary (the tile is one TMA box,
// see encode_feat16_map).
__host__ __device__ constexpr size_t feat16_group_offset(int64_t S_cap, int64_t tile, int g) {
  return (size_t)g * 4 * (size_t)S_cap + (size_t)tile * 512;
}

// TMA tensor map over the 16-bit feature tiles of a buffer with S_cap slots for K = in
// features: 3-D, innermost the in * 16 bytes of a row group (as 16-bit elements), then the
// tile (stride 512 B), then the 16 row groups (stride 4 * S_cap B); a box {in * 8, 1, 16} at
// (0, T, 0) is tile T in the MMA's K-major layout.  `map` points to a CUtensorMap.  Returns
// false if the driver's encoder is unavailable or rejects the map.
bool encode_feat16_map(void* map, const void* feat, int64_t S_cap, int in);

// Byte offset of the remainder tiles (training of a 16-bit field: each feature's 16-bit
// value plus the 16-bit remainder of its rounding, tc::split2): the same layout 16 FP32
// feature rows further, inside the tile's own columns again.
__host__ __device__ constexpr size_t feat16_lo_offset(int64_t S_cap) { return (size_t)64 * (size_t)S_cap; }

// Byte offset of feature k of sample s (k even: the pair k, k+1 is one 32-bit word).
__host__ __device__ constexpr size_t feat16_offset(int64_t S_cap, int64_t s, int k) {
  return feat16_group_offset(S_cap, s >> 7, (int)((s & 127) >> 3)) + (size_t)((k >> 3) * 128) +
         (size_t)((s & 7) * 16) + (size_t)((k & 7) * 2);
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------------------------ launchers
// Each returns cudaGetLastError() of its launches.
cudaError_t launch_march_count(const Plan& P, cudaStream_t s);
cudaError_t launch_scan(const Plan& P, cudaStream_t s);
cudaError_t launch_march_emit(const Plan& P, cudaStream_t s);
cudaError_t launch_warp(const Plan& P, int num_sms, cudaStream_t s);
cudaError_t launch_encode(const Plan& P, int num_sms, cudaStream_t s);
cudaError_t launch_encode_bwd(const Plan& P, int num_sms, cudaStream_t s);
cudaError_t launch_encode_by_field(const Plan& P, int num_sms, cudaStream_t s);
cudaError_t launch_encode_bwd_by_field(const Plan& P, int num_sms, cudaStream_t s);
cudaError_t launch_warp_encode_by_field(const Plan& P, int num_sms, cudaStream_t s);
cudaError_t launch_mlp_fwd_f32(const Plan& P, int num_sms, cudaStream_t s);
cudaError_t launch_mlp_bwd_f32(const Plan& P, int num_sms, cudaStream_t s);
bool plan_has_kind(const Plan& P, int kind);
cudaError_t launch_mlp_fwd_tc(const Plan& P, int num_sms, cudaStream_t s);
// training forward of the 16-bit fields: split products, ReLU decisions to ws.mlp_mask
cudaError_t launch_mlp_fwd_split_tc(const Plan& P, int num_sms, cudaStream_t s);
cudaError_t launch_mlp_bwd_tc(const Plan& P, int num_sms, cudaStream_t s);
// Rewrite the weight images (FieldDev::w16) of every 16-bit field of the plan.
cudaError_t launch_prep_w16_plan(const Plan& P, cudaStream_t s);
cudaError_t launch_mlp_points_tc(const FieldDev& f, int64_t n, const float* feat, float* out, unsigned* status,
                                 uint32_t wait_limit, int num_sms, cudaStream_t s);
constexpr uint32_t kDefaultWaitLimit = 1u << 22;  // polls of try_wait: a few seconds
cudaError_t launch_composite_joint(const Plan& P, int64_t n_rays, float* rgba, float* depth, cudaStream_t s);
cudaError_t launch_composite_render(const Plan& P, int64_t n_rays, float* rgba, float* depth, cudaStream_t s);
cudaError_t launch_composite_train(const Plan& P, float* loss, cudaStream_t s);
cudaError_t launch_adam(float* params, const float* grads_in, float* grads_zero, float* m, float* v, int64_t n,
                        const int64_t* step_dev, float lr, float b1, float b2, float eps, cudaStream_t s);
cudaError_t launch_step_increment(int64_t* step_dev, cudaStream_t s);

// graph preprocessing
cudaError_t launch_graph_pack(const float* dq_soa, const float* x_soa, int n, float4* dq_out, float4* x_out,
                              cudaStream_t s);
// candidate grid of resolution kKnnG, through a kKnnG/2 grid (coarse, coarse_n: scratch of
// (kKnnG/2)^3 x kKnnCoarseCapFactor * cap and (kKnnG/2)^3 entries)
constexpr int kKnnCoarseCapFactor = 4;
cudaError_t launch_knn_grid_build(const float4* x_live, int n, int K, int cap, uint16_t* coarse, uint16_t* coarse_n,
                                  uint32_t* cand, uint32_t* cand_head, int num_sms, cudaStream_t s);

// single-step entry points
cudaError_t launch_ray_samples(int64_t n_rays, const float* o, const float* d, int n_samples, const uint32_t* occ,
                               int32_t* count, float* t, float* p, cudaStream_t s);
cudaError_t launch_warp_points(const WarpDev& w, int64_t n, const float* p, float* vc, int32_t* ids,
                               cudaStream_t s);
cudaError_t launch_encode_points(const FieldDev& f, int64_t n, const float* x, float* feat, uint32_t* idx,
                                 cudaStream_t s);
cudaError_t launch_mlp_points_f32(const FieldDev& f, int64_t n, const float* feat, float* out, int num_sms,
                                  cudaStream_t s);

// Load the code of the point-query kernels (warp, encoding, both MLP paths) now: with lazy
// module loading their first launch would otherwise load it, allocating device memory.
cudaError_t preload_warp_points();
cudaError_t preload_encode_points();
cudaError_t preload_mlp_points_f32();
cudaError_t preload_mlp_points_tc();
// Set up the no-allocation point query on the current device `dev`: look up its scratch
// array's device address and load the kernels it launches (called by invr_ctx_create).
cudaError_t noalloc_prepare(int dev);

// deformation net
cudaError_t launch_deform_forward(const Plan& P, int num_sms, cudaStream_t s);
cudaError_t launch_deform_forward_tc(const Plan& P, int num_sms, cudaStream_t s);
cudaError_t launch_deform_backward_tc(const Plan& P, int num_sms, cudaStream_t s);
constexpr int kDeformTcMaxPose = 80;   // pose columns of the tensor-core weight gradient
cudaError_t launch_encode_dx(const Plan& P, int num_sms, cudaStream_t s);
cudaError_t launch_deform_backward(const Plan& P, int num_sms, cudaStream_t s);
cudaError_t launch_deform_reduce(const DeformDev& D, int n_parts, cudaStream_t s);
constexpr int kDeformMaxFeat = 32;
constexpr int kDeformMaxHidden = 128;
constexpr int kDeformMaxLayers = 4;
constexpr int kDeformMaxPose = 128;

// occupancy maintenance
cudaError_t launch_occ_centres(float* p, int64_t n, cudaStream_t s);
cudaError_t launch_occ_update(const float* sigma, int64_t n, float decay, float threshold, float* density,
                              uint32_t* bits, cudaStream_t s);

// look-up-table neighbour search (Sec. 4.2)
cudaError_t launch_pack_points(const float* x_soa, int n, float4* out, cudaStream_t s);
cudaError_t launch_lut_canon(const float4* x_canon, int n, int K, const uint32_t* cand, const uint32_t* cand_head,
                             int cap, int G, uint16_t* canon, int num_sms, cudaStream_t s);
cudaError_t launch_lut_live(const float4* x_canon, const float4* dq, int n, int K, float inv_r2, int G,
                            const uint16_t* canon, uint32_t* live, int num_sms, cudaStream_t s);

// L2 ceiling probes (measurement only)
cudaError_t launch_probe_l2_read(const float* buf, int64_t n_floats, int passes, float* sink, int num_sms,
                                 cudaStream_t s);
cudaError_t launch_probe_l2_atomic(float* table, int64_t n_floats, int width, int64_t n_ops, int num_sms,
                                   cudaStream_t s);
cudaError_t launch_probe_l2_gather(const float* table, int64_t n_floats, int width, int64_t n_ops, float* sink,
                                   int num_sms, cudaStream_t s);

}  // namespace invr
