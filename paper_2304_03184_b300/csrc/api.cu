// C ABI of the hot path: handles, argument checks, workspace, and the launch sequences of
// render_rays / train_step.  See include/invr.h for the contract of each call.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "invr.h"
#include "invr_internal.cuh"

using namespace invr;

struct invr_ctx_s {
  int device = 0;
  int num_sms = 148;
  Workspace ws{};
  int64_t cap_R = 0, cap_S = 0;
  bool cap_train = false;
  bool cap_fixed = false;   // set by invr_ctx_reserve: never grow, overflow is flagged on device
  Tune tune;
  uint32_t wait_limit = kDefaultWaitLimit;
  unsigned* status = nullptr;
  float* pose_bias = nullptr;  // [kMaxViews][kDeformMaxHidden] per-view first-layer pose terms
  int64_t cap_deform = 0;      // sample slots of the deformation-net buffers
  std::string err;
  // per-kernel event timing (invr_ctx_enable_timing)
  bool timing = false;
  struct Rec {
    const char* name;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  // side stream of the backward: one field's gradient scatter beside the other's MLP backward
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // state kept between invr_field_forward_train and invr_field_backward
  bool fwd_valid = false;
  Plan fwd_plan{};
  std::vector<int64_t> fwd_sig;
};

struct invr_field_s {
  invr_ctx ctx = nullptr;
  invr_field_desc desc{};
  int64_t n_tab = 0, n_w = 0;
  float* params = nullptr;  // tables then weights
  float* grads = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  int64_t* step = nullptr;  // device step counter
  float* wt = nullptr;      // [kWtF32] the FP32 MLP's transposed weights (scratch of its forward)
  uint8_t* w16 = nullptr;   // [kW16Bytes] the tensor-core MLPs' weight images (16-bit fields)
  int res[kMaxL] = {};
  uint32_t dense_mask = 0;
};

struct invr_deform_s {
  invr_ctx ctx = nullptr;
  invr_deform_desc desc{};
  int64_t n_tab = 0, n_w = 0;
  float* params = nullptr;  // tables then weights
  float* grads = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  int64_t* step = nullptr;
  float* scratch = nullptr; // [num_sms][n_w] weight-gradient partials of the backward
  int res[kMaxL] = {};
  uint32_t dense_mask = 0;
};

struct invr_graph_s {
  invr_ctx ctx = nullptr;
  invr_graph_desc desc{};
  float* x_canon = nullptr;
  struct Frame {
    float4* x_live = nullptr;
    float4* dq = nullptr;
    uint32_t* cand = nullptr;
    uint32_t* cand_head = nullptr;  // [G^3][kKnnHead] the lists' heads
    uint32_t* lut_live = nullptr;   // [G^3] live index field of this frame
    bool set = false;
  };
  std::vector<Frame> frames;
  int cap = 0;  // 0: no candidate grid (scan all nodes)
  uint16_t* coarse = nullptr;    // scratch of the two-level candidate-grid build
  uint16_t* coarse_n = nullptr;
  // look-up-table neighbour search (Sec. 4.2); lut_res == 0: exact search
  int lut_res = 0;
  uint16_t* lut_canon = nullptr;   // [G^3][K] canonical KNN field
  float4* x_canon4 = nullptr;      // canonical nodes, packed
  uint32_t* canon_cand = nullptr;  // candidate grid over the canonical nodes
  uint32_t* canon_cand_head = nullptr;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Brackets one launch with events on its stream when timing is enabled.
struct Timed {
  invr_ctx ctx;
  cudaStream_t s;
  invr_ctx_s::Rec rec{};
  Timed(invr_ctx c, const char* name, cudaStream_t st) : ctx(c), s(st) {
    if (!ctx->timing) return;
    rec.name = name;
    cudaEventCreate(&rec.a);
    cudaEventCreate(&rec.b);
    cudaEventRecord(rec.a, s);
  }
  ~Timed() {
    if (!ctx->timing) return;
    cudaEventRecord(rec.b, s);
    ctx->recs.push_back(rec);
  }
};

#define TIMED(ctx, name, s, call) \
  [&]() -> cudaError_t {          \
    Timed t_(ctx, name, s);       \
    return (call);                \
  }()

void clear_timing(invr_ctx ctx) {
  for (auto& r : ctx->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  ctx->recs.clear();
}

invr_status fail(invr_ctx ctx, invr_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

#define INVR_CUDA(ctx, call)                                                                     \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? INVR_E_OOM : INVR_E_CUDA,             \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                           \
  } while (0)

template <class T>
cudaError_t dmalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

int level_resolution(int N_min, double growth, int l) {
  return (int)std::floor((double)N_min * std::pow(growth, (double)l));
}

int64_t weight_count(int in, int hidden, int geo, int col) {
  return (int64_t)hidden * in + (int64_t)hidden * hidden + (int64_t)geo * hidden + (int64_t)col * (geo - 1) +
         3LL * col;
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &st);
  return st != cudaStreamCaptureStatusNone;
}

void free_workspace(Workspace& w) {
  void* ptrs[] = {w.ray_count, w.ray_bits, w.ray_first, w.ray_used, w.ray_out, w.block_sums, w.view_base, w.s_ray,
                  w.s_t, w.s_pos, w.s_vc, w.feat, w.out, w.dout, w.dfeat, w.mlp_mask, w.loss_part, w.tickets,
                  w.s_vt, w.feat_d, w.dvc, w.dfeat_d, w.def_x, w.def_h, w.def_g, w.def_gout};
  for (void* p : ptrs) dfree(p);
  w = Workspace{};
}

// Grow the workspace to hold R rays and S sample slots (and the training buffers).
invr_status ensure_workspace(invr_ctx ctx, int64_t R, int64_t S, bool train, cudaStream_t stream) {
  if (R <= ctx->cap_R && S <= ctx->cap_S && (!train || ctx->cap_train)) return INVR_OK;
  if (ctx->cap_fixed) {
    // a reserved workspace never grows: more rays is an argument error, more samples than
    // reserved is detected on the device (status word, reported by invr_ctx_sync)
    if (R > ctx->cap_R) return fail(ctx, INVR_E_ARG, "more rays than reserved with invr_ctx_reserve");
    if (train && !ctx->cap_train) return fail(ctx, INVR_E_STATE, "reserved workspace has no training buffers");
    return INVR_OK;
  }
  if (capturing(stream))
    return fail(ctx, INVR_E_STATE, "workspace too small during stream capture: call invr_ctx_reserve first");
  R = std::max(R, ctx->cap_R);
  S = std::max(S, ctx->cap_S);
  S = (S + kTile - 1) / kTile * kTile;  // 16-byte aligned row groups of the 16-bit feature tiles
  train = train || ctx->cap_train;
  INVR_CUDA(ctx, cudaDeviceSynchronize());
  free_workspace(ctx->ws);
  ctx->cap_R = ctx->cap_S = 0;
  ctx->cap_train = false;
  Workspace& w = ctx->ws;
  const int64_t blocks = R / 1024 + kMaxViews + 1;
  INVR_CUDA(ctx, dmalloc(&w.ray_count, R));
  INVR_CUDA(ctx, dmalloc(&w.ray_bits, (size_t)R * kRayBitWords));
  INVR_CUDA(ctx, dmalloc(&w.ray_first, R));
  INVR_CUDA(ctx, dmalloc(&w.ray_used, R));
  INVR_CUDA(ctx, dmalloc(&w.ray_out, 5 * R));
  INVR_CUDA(ctx, dmalloc(&w.block_sums, blocks));
  INVR_CUDA(ctx, dmalloc(&w.view_base, 2 * (kMaxViews + 1) + 6 * kMaxViews));
  w.view_count = w.view_base + kMaxViews + 1;
  w.occ_box = w.view_base + 2 * (kMaxViews + 1);
  INVR_CUDA(ctx, dmalloc(&w.s_ray, S));
  INVR_CUDA(ctx, dmalloc(&w.s_t, S));
  INVR_CUDA(ctx, dmalloc(&w.s_pos, 3 * S));
  INVR_CUDA(ctx, dmalloc(&w.s_vc, 3 * S));
  float* feat = nullptr;
  INVR_CUDA(ctx, dmalloc(&feat, (size_t)kMaxIn * S));
  w.feat = feat;
  INVR_CUDA(ctx, dmalloc(&w.out, 4 * S));
  INVR_CUDA(ctx, dmalloc(&w.loss_part, R / 32 + 1));
  INVR_CUDA(ctx, dmalloc(&w.tickets, kTicketSlots));
  if (train) {
    INVR_CUDA(ctx, dmalloc(&w.dout, 4 * S));
    INVR_CUDA(ctx, dmalloc(&w.dfeat, (size_t)kMaxIn * S));
    INVR_CUDA(ctx, dmalloc(&w.mlp_mask, (size_t)6 * S));
  }
  w.S_cap = S;
  w.R_cap = R;
  ctx->cap_R = R;
  ctx->cap_S = S;
  ctx->cap_train = train;
  ctx->cap_deform = 0;
  ctx->fwd_valid = false;
  return INVR_OK;
}

// The deformation-net buffers (v_t, the net's features, dL/dv_c, dL/d features), sized like
// the sample slots; allocated the first time a call has a net.
invr_status ensure_deform_workspace(invr_ctx ctx, cudaStream_t stream) {
  Workspace& w = ctx->ws;
  if (ctx->cap_deform >= w.S_cap && w.s_vt) return INVR_OK;
  if (capturing(stream))
    return fail(ctx, INVR_E_STATE, "deformation-net buffers missing during stream capture: run one call first");
  INVR_CUDA(ctx, cudaDeviceSynchronize());
  dfree(w.s_vt); dfree(w.feat_d); dfree(w.dvc); dfree(w.dfeat_d);
  dfree(w.def_x); dfree(w.def_h); dfree(w.def_g); dfree(w.def_gout);
  w.def_x = w.def_h = w.def_g = w.def_gout = nullptr;
  const int64_t S = w.S_cap;
  INVR_CUDA(ctx, dmalloc(&w.s_vt, 3 * S));
  INVR_CUDA(ctx, dmalloc(&w.feat_d, (size_t)kDeformMaxFeat * S));
  INVR_CUDA(ctx, dmalloc(&w.dvc, 3 * S));
  INVR_CUDA(ctx, dmalloc(&w.dfeat_d, (size_t)kDeformMaxFeat * S));
  ctx->cap_deform = S;
  return INVR_OK;
}

// Operand tiles of the tensor-core training of a net (2,144 bytes per sample slot).
invr_status ensure_deform_tc_workspace(invr_ctx ctx, cudaStream_t stream) {
  Workspace& w = ctx->ws;
  if (w.def_h) return INVR_OK;
  if (capturing(stream))
    return fail(ctx, INVR_E_STATE, "deformation-net buffers missing during stream capture: run one call first");
  INVR_CUDA(ctx, cudaDeviceSynchronize());
  const size_t tiles = (size_t)(w.S_cap / kTile);
  INVR_CUDA(ctx, dmalloc(&w.def_x, tiles * kTile * kDeformMaxFeat * 2));
  INVR_CUDA(ctx, dmalloc(&w.def_h, (size_t)kDeformMaxLayers * tiles * kTile * kDeformMaxHidden * 2));
  INVR_CUDA(ctx, dmalloc(&w.def_g, (size_t)kDeformMaxLayers * tiles * kTile * kDeformMaxHidden * 2));
  INVR_CUDA(ctx, dmalloc(&w.def_gout, tiles * kTile * 16 * 2));
  return INVR_OK;
}

DeformDev deform_dev(invr_ctx ctx, invr_deform d, const float* pose, int view) {
  DeformDev D{};
  const invr_deform_desc& q = d->desc;
  D.weights = d->params + d->n_tab;
  D.grad_weights = d->grads + d->n_tab;
  D.dw_scratch = d->scratch;
  D.pose = pose;
  D.pose_bias = ctx->pose_bias + (int64_t)view * kDeformMaxHidden;
  D.enc.tables = d->params;
  D.enc.weights = nullptr;
  D.enc.wt_f32 = nullptr;
  D.enc.w16 = nullptr;
  D.enc.grad_tables = d->grads;
  D.enc.grad_weights = nullptr;
  D.enc.L = q.L;
  D.enc.log2T = q.log2_T;
  D.enc.mlp_in = q.L * q.F;
  D.enc.mlp_kind = kMlpF32;
  for (int l = 0; l < kMaxL; ++l) D.enc.res[l] = d->res[l];
  D.enc.dense_mask = d->dense_mask;
  D.n_feat = q.L * q.F;
  D.pose_dim = q.pose_dim;
  D.hidden = q.hidden;
  D.n_hidden = q.n_hidden;
  D.n_w = (int)d->n_w;
  D.tc = q.prec == INVR_MLP_BF16 ? 2 : (q.prec == INVR_MLP_FP16 ? 1 : 0);
  return D;
}

FieldDev field_dev(invr_field f) {
  FieldDev F{};
  F.tables = f->params;
  F.weights = f->params + f->n_tab;
  F.wt_f32 = f->wt;
  F.w16 = f->w16;
  F.grad_tables = f->grads;
  F.grad_weights = f->grads + f->n_tab;
  F.L = f->desc.L;
  F.log2T = f->desc.log2_T;
  F.mlp_in = f->desc.mlp_in;
  F.mlp_kind = (int)f->desc.prec;
  for (int l = 0; l < kMaxL; ++l) F.res[l] = f->res[l];
  F.dense_mask = f->dense_mask;
  return F;
}

// Rotation and translation of a (renormalised) unit dual quaternion, in double.
void dq_rigid(const float* dq, float R[9], float t[3]) {
  double b[8];
  for (int i = 0; i < 8; ++i) b[i] = dq[i];
  const double n = std::sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2] + b[3] * b[3]);
  double r[4], d[4], dot = 0.0;
  for (int i = 0; i < 4; ++i) {
    r[i] = b[i] / n;
    d[i] = b[4 + i] / n;
  }
  for (int i = 0; i < 4; ++i) dot += r[i] * d[i];
  for (int i = 0; i < 4; ++i) d[i] -= dot * r[i];
  const double w = r[0], x = r[1], y = r[2], z = r[3];
  const double M[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z),     2 * (x * z + w * y),
                       2 * (x * y + w * z),     1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                       2 * (x * z - w * y),     2 * (y * z + w * x),     1 - 2 * (x * x + y * y)};
  for (int i = 0; i < 9; ++i) R[i] = (float)M[i];
  // t = 2 vec(d r^*)
  t[0] = (float)(2.0 * (-d[0] * x + d[1] * w - d[2] * z + d[3] * y));
  t[1] = (float)(2.0 * (-d[0] * y + d[1] * z + d[2] * w - d[3] * x));
  t[2] = (float)(2.0 * (-d[0] * z - d[1] * y + d[2] * x + d[3] * w));
}

invr_status warp_dev(invr_ctx ctx, const invr_field_view& v, WarpDev& W) {
  W = WarpDev{};
  if (!v.graph) {
    if (!v.rigid_dq) return fail(ctx, INVR_E_ARG, "view without graph needs rigid_dq (8 host floats)");
    W.mode = 0;
    dq_rigid(v.rigid_dq, W.R, W.t);
    return INVR_OK;
  }
  invr_graph g = v.graph;
  if (g->ctx != ctx) return fail(ctx, INVR_E_ARG, "graph belongs to another context");
  if (v.frame < 0 || v.frame >= (int)g->frames.size()) return fail(ctx, INVR_E_ARG, "frame out of range");
  const auto& fr = g->frames[v.frame];
  if (!fr.set) return fail(ctx, INVR_E_STATE, "frame pose not set (invr_graph_set_pose)");
  W.mode = 1;
  W.x_live = fr.x_live;
  W.dq = fr.dq;
  W.cand = fr.cand;
  W.cand_head = fr.cand_head;
  W.n_nodes = g->desc.n_nodes;
  W.K = g->desc.K;
  W.cap = g->cap;
  W.inv_r2 = 1.0f / (g->desc.radius * g->desc.radius);
  if (g->lut_res > 0) {
    W.lut_res = g->lut_res;
    W.lut_canon = g->lut_canon;
    W.lut_live = fr.lut_live;
  }
  return INVR_OK;
}

invr_status check_field(invr_ctx ctx, invr_field f) {
  if (!f) return fail(ctx, INVR_E_ARG, "null field");
  if (f->ctx != ctx) return fail(ctx, INVR_E_ARG, "field belongs to another context");
  return INVR_OK;
}

// Build the plan of a call: one entry per view (render) or per batch (training).
invr_status build_plan(invr_ctx ctx, const std::vector<const invr_render_args*>& rays,
                       const std::vector<const invr_field_view*>& views, int n_samples, float t_eps, Plan& P) {
  P = Plan{};
  const int nv = (int)views.size();
  if (nv < 1 || nv > kMaxViews) return fail(ctx, INVR_E_ARG, "1..16 views/batches per call");
  if (n_samples < 1 || n_samples > 1024) return fail(ctx, INVR_E_ARG, "n_samples must be in [1, 1024]");
  P.n_views = nv;
  P.view_lo = 0;
  P.view_hi = nv;
  P.wait_limit = ctx->wait_limit;
  P.n_samples = n_samples;
  P.t_eps = t_eps;
  P.tune = ctx->tune;
  P.agg_res = ctx->tune.agg_res;
  P.grad_scale = 1.0f;
  int64_t ray_begin = 0;
  int blocks = 0;
  for (int i = 0; i < nv; ++i) {
    const invr_render_args* a = rays[i];
    const invr_field_view& v = *views[i];
    if (a->n_rays < 0) return fail(ctx, INVR_E_ARG, "n_rays < 0");
    if (a->n_rays > 0 && (!a->o_dev || !a->d_dev)) return fail(ctx, INVR_E_ARG, "null ray pointer");
    invr_status st = check_field(ctx, v.field);
    if (st != INVR_OK) return st;
    ViewDev& V = P.v[i];
    V.o = a->o_dev;
    V.d = a->d_dev;
    V.occ = v.occupancy_dev;
    V.n_rays = a->n_rays;
    V.ray_begin = ray_begin;
    V.scan_block_begin = blocks;
    V.field = field_dev(v.field);
    st = warp_dev(ctx, v, V.warp);
    if (st != INVR_OK) return st;
    if (v.deform) {
      if (v.deform->ctx != ctx) return fail(ctx, INVR_E_ARG, "deformation net belongs to another context");
      if (!v.graph) return fail(ctx, INVR_E_ARG, "a deformation net needs the human view (graph != NULL)");
      if (!v.pose_dev) return fail(ctx, INVR_E_ARG, "a deformation net needs pose_dev");
      V.has_deform = 1;
      V.deform = deform_dev(ctx, v.deform, v.pose_dev, i);
      P.has_deform = 1;
    }
    ray_begin += a->n_rays;
    blocks += (int)((a->n_rays + 1023) / 1024);
  }
  P.total_rays = ray_begin;
  P.n_scan_blocks = blocks;
  P.status = ctx->status;
  return INVR_OK;
}

// Run `launch` on plan copies that see the deformation net's encoding as each view's
// field, v_t as the positions and the net's feature buffers, once per run of consecutive
// views with a net (views without one are outside the runs).
template <class Launch>
cudaError_t deform_runs(const Plan& P, bool backward, Launch launch) {
  for (int lo = 0; lo < P.n_views;) {
    if (!P.v[lo].has_deform) {
      ++lo;
      continue;
    }
    int hi = lo + 1;
    while (hi < P.n_views && P.v[hi].has_deform) ++hi;
    Plan Q = P;
    Q.view_lo = lo;
    Q.view_hi = hi;
    for (int v = lo; v < hi; ++v) Q.v[v].field = P.v[v].deform.enc;
    Q.ws.s_vc = P.ws.s_vt;
    Q.ws.feat = P.ws.feat_d;
    Q.ws.dfeat = P.ws.dfeat_d;
    if (backward) Q.grad_scale = 1.0f;  // dL/df of the net already carries the scale
    cudaError_t e = launch(Q);
    if (e != cudaSuccess) return e;
    lo = hi;
  }
  return cudaSuccess;
}

cudaError_t run_deform_and_encode(invr_ctx ctx, const Plan& P, cudaStream_t s);

cudaError_t run_forward(invr_ctx ctx, const Plan& P, cudaStream_t s) {
  cudaError_t e;
  if ((e = TIMED(ctx, "march_count", s, launch_march_count(P, s))) != cudaSuccess) return e;
  if ((e = TIMED(ctx, "scan", s, launch_scan(P, s))) != cudaSuccess) return e;
  if ((e = TIMED(ctx, "march_emit", s, launch_march_emit(P, s))) != cudaSuccess) return e;
  if (P.tune.fused && !P.has_deform) {
    if ((e = TIMED(ctx, "warp_encode", s, launch_warp_encode_by_field(P, ctx->num_sms, s))) != cudaSuccess) return e;
  } else {
    if ((e = TIMED(ctx, "warp", s, launch_warp(P, ctx->num_sms, s))) != cudaSuccess) return e;
    if ((e = run_deform_and_encode(ctx, P, s)) != cudaSuccess) return e;
  }
  if (plan_has_kind(P, kMlpF32) && (e = TIMED(ctx, "mlp_fwd", s, launch_mlp_fwd_f32(P, ctx->num_sms, s))) != cudaSuccess)
    return e;
  if (plan_has_kind(P, kMlpF16) || plan_has_kind(P, kMlpBF16)) {
    if ((e = TIMED(ctx, "prep_w16", s, launch_prep_w16_plan(P, s))) != cudaSuccess) return e;
    e = P.feat_split ? TIMED(ctx, "mlp_fwd_tc", s, launch_mlp_fwd_split_tc(P, ctx->num_sms, s))
                     : TIMED(ctx, "mlp_fwd_tc", s, launch_mlp_fwd_tc(P, ctx->num_sms, s));
  }
  return e;
}

// The staged forward after the warp: the deformation net (if any view has one), then the
// field's encoding.
cudaError_t run_deform_and_encode(invr_ctx ctx, const Plan& P, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (P.has_deform) {
    // v_t = the warp; the net's features of v_t; v_c = v_t + delta v (written over s_vc)
    if ((e = cudaMemcpyAsync(P.ws.s_vt, P.ws.s_vc, 3 * P.ws.S_cap * sizeof(float), cudaMemcpyDeviceToDevice, s)) !=
        cudaSuccess)
      return e;
    if ((e = TIMED(ctx, "deform_encode", s, deform_runs(P, false, [&](const Plan& Q) {
                     return launch_encode(Q, ctx->num_sms, s);
                   }))) != cudaSuccess)
      return e;
    if ((e = TIMED(ctx, "deform_fwd", s, launch_deform_forward(P, ctx->num_sms, s))) != cudaSuccess) return e;
  }
  return TIMED(ctx, "encode", s, launch_encode_by_field(P, ctx->num_sms, s));
}

invr_status check_desc(invr_ctx ctx, const invr_field_desc* d) {
  if (!d) return fail(ctx, INVR_E_ARG, "null field desc");
  if (d->F != kF) return fail(ctx, INVR_E_ARG, "F must be 2");
  if (d->L < 1 || d->L > kMaxL) return fail(ctx, INVR_E_ARG, "L must be in [1, 16]");
  if (d->mlp_in != d->L * d->F || (d->mlp_in != 16 && d->mlp_in != 32))
    return fail(ctx, INVR_E_ARG, "mlp_in must equal L*F and be 16 or 32");
  if (d->mlp_hidden != kHidden || d->col_hidden != kColHidden || d->geo_out != kGeoOut)
    return fail(ctx, INVR_E_ARG, "mlp_hidden = col_hidden = 64 and geo_out = 16 are supported");
  if (d->log2_T < 10 || d->log2_T > 24) return fail(ctx, INVR_E_ARG, "log2_T must be in [10, 24]");
  if (d->N_min < 1 || !(d->growth >= 1.0)) return fail(ctx, INVR_E_ARG, "N_min >= 1 and growth >= 1 required");
  if (d->prec != INVR_FP32 && d->prec != INVR_MLP_FP16 && d->prec != INVR_MLP_BF16)
    return fail(ctx, INVR_E_ARG, "unknown precision");
  if (level_resolution(d->N_min, d->growth, d->L - 1) > (1 << 20))
    return fail(ctx, INVR_E_ARG, "finest level resolution above 2^20");
  return INVR_OK;
}

static_assert(kLossHuber == INVR_LOSS_HUBER && kLossPaper == INVR_LOSS_PAPER, "loss codes");

std::vector<int64_t> signature(const invr_train_args* a) {
  std::vector<int64_t> s{a->n_batches, a->loss};
  for (int b = 0; b < a->n_batches; ++b) {
    s.push_back(a->batches[b].n_rays);
    s.push_back((int64_t)(uintptr_t)a->batches[b].views[0].field);
  }
  return s;
}

invr_status train_forward(invr_ctx ctx, const invr_train_args* a, cudaStream_t s) {
  if (!a || a->n_batches < 1 || a->n_batches > kMaxViews || !a->batches)
    return fail(ctx, INVR_E_ARG, "1..16 batches per training call");
  if (!a->targets_dev || !a->loss_dev) return fail(ctx, INVR_E_ARG, "null targets_dev or loss_dev");
  if (a->loss != INVR_LOSS_HUBER && a->loss != INVR_LOSS_PAPER) return fail(ctx, INVR_E_ARG, "unknown loss");
  if (a->loss == INVR_LOSS_PAPER && !a->depths_dev)
    return fail(ctx, INVR_E_ARG, "the paper's depth loss needs depths_dev");
  std::vector<const invr_render_args*> rays;
  std::vector<const invr_field_view*> views;
  const int ns = a->batches[0].n_samples;
  const float te = a->batches[0].t_eps;
  for (int b = 0; b < a->n_batches; ++b) {
    const invr_render_args& r = a->batches[b];
    if (r.n_views != 1 || !r.views) return fail(ctx, INVR_E_ARG, "each training batch has exactly one view");
    if (r.n_samples != ns || r.t_eps != te) return fail(ctx, INVR_E_ARG, "batches must share n_samples and t_eps");
  }
  // Batches of the same field are laid out next to each other (stable order), so that the
  // per-field launches of the encoding and the gradient scatter each keep one field's
  // tables and gradients in L2.
  std::vector<int> order;
  std::vector<invr_field> seen;
  for (int b = 0; b < a->n_batches; ++b) {
    invr_field f = a->batches[b].views[0].field;
    if (std::find(seen.begin(), seen.end(), f) == seen.end()) seen.push_back(f);
  }
  for (invr_field f : seen)
    for (int b = 0; b < a->n_batches; ++b)
      if (a->batches[b].views[0].field == f) order.push_back(b);
  std::vector<int64_t> target_off(a->n_batches, 0);
  for (int b = 1; b < a->n_batches; ++b) target_off[b] = target_off[b - 1] + a->batches[b - 1].n_rays;
  for (int b : order) {
    rays.push_back(&a->batches[b]);
    views.push_back(&a->batches[b].views[0]);
  }
  Plan P;
  invr_status st = build_plan(ctx, rays, views, ns, te, P);
  if (st != INVR_OK) return st;
  if (P.total_rays == 0) return fail(ctx, INVR_E_ARG, "training call without rays");
  for (int i = 0; i < a->n_batches; ++i) {
    const int b = order[i];
    P.v[i].target = a->targets_dev + 3 * target_off[b];
    P.v[i].mask = a->loss == INVR_LOSS_PAPER && a->masks_dev ? a->masks_dev + target_off[b] : nullptr;
    P.v[i].depth_target = a->loss == INVR_LOSS_PAPER ? a->depths_dev + target_off[b] : nullptr;
    P.v[i].rgba_out = a->batches[b].rgba_dev;
    P.v[i].depth_out = a->batches[b].depth_dev;
  }
  P.loss_kind = a->loss;
  P.loss_norm = a->loss == INVR_LOSS_HUBER ? (float)(1.0 / (3.0 * (double)P.total_rays)) : 1.0f;
  P.huber_delta = a->huber_delta;
  P.depth_weight = a->depth_weight;
  st = ensure_workspace(ctx, P.total_rays, P.total_rays * ns + (int64_t)P.n_views * kTile, true, s);
  if (st != INVR_OK) return st;
  if (P.has_deform && (st = ensure_deform_workspace(ctx, s)) != INVR_OK) return st;
  const DeformDev* tc_net = nullptr;
  for (int v = 0; v < P.n_views; ++v) {
    if (!P.v[v].has_deform || !P.v[v].deform.tc) continue;
    if (tc_net && tc_net->weights != P.v[v].deform.weights)
      return fail(ctx, INVR_E_ARG, "one training call takes at most one tensor-core deformation net");
    tc_net = &P.v[v].deform;
  }
  if (tc_net) {
    if ((st = ensure_deform_tc_workspace(ctx, s)) != INVR_OK) return st;
    P.deform_store = 1;
  }
  P.feat_split = 1;  // 16-bit fields train on split products (values plus rounding remainders)
  P.march_coop = 1;  // training batches draw their rays in random order
  P.ws = ctx->ws;
  INVR_CUDA(ctx, run_forward(ctx, P, s));
  INVR_CUDA(ctx, TIMED(ctx, "composite_train", s, launch_composite_train(P, a->loss_dev, s)));
  ctx->fwd_plan = P;
  ctx->fwd_sig = signature(a);
  ctx->fwd_valid = true;
  return INVR_OK;
}

// Adam of the side field on the side stream (a training step's backward only): set by
// invr_train_step, which then skips that field's update.
struct SideAdam {
  float lr, b1, b2, eps;
  invr_field done = nullptr;
};

invr_status train_backward(invr_ctx ctx, const invr_train_args* a, float scale, cudaStream_t s,
                           SideAdam* side_adam = nullptr) {
  if (!a || !ctx->fwd_valid || signature(a) != ctx->fwd_sig)
    return fail(ctx, INVR_E_STATE, "invr_field_backward needs the matching invr_field_forward_train first");
  Plan P = ctx->fwd_plan;
  P.grad_scale = scale;
  // Two fields, both on the tensor cores, no deformation net, no per-kernel timing: the MLP
  // backward of the field with fewer rays runs first, and that field's gradient scatter then
  // runs on the context's side stream beside the other field's MLP backward (the scatter is
  // bound by the L2's atomics, the MLP backward by its MMA chain; a scatter CTA fits beside
  // two MLP CTAs on an SM); the side stream is joined before returning.  Within a training
  // step (side_adam set) the side field's Adam update follows its scatter on the side stream,
  // beside the other field's scatter (0.08 ms per batched step).
  int split = 1;
  while (split < P.n_views && P.v[split].field.tables == P.v[0].field.tables) ++split;
  bool two = split < P.n_views;
  for (int v = split + 1; v < P.n_views; ++v) two = two && P.v[v].field.tables == P.v[split].field.tables;
  if (two && !ctx->timing && !P.has_deform && !plan_has_kind(P, kMlpF32)) {
    int64_t r0 = 0, r1 = 0;
    for (int v = 0; v < P.n_views; ++v) (v < split ? r0 : r1) += P.v[v].n_rays;
    Plan A = P, B = P;  // A: the side field
    A.view_lo = r0 <= r1 ? 0 : split;
    A.view_hi = r0 <= r1 ? split : P.n_views;
    B.view_lo = r0 <= r1 ? split : 0;
    B.view_hi = r0 <= r1 ? P.n_views : split;
    INVR_CUDA(ctx, launch_mlp_bwd_tc(A, ctx->num_sms, s));
    INVR_CUDA(ctx, cudaEventRecord(ctx->ev_fork, s));
    INVR_CUDA(ctx, launch_mlp_bwd_tc(B, ctx->num_sms, s));
    A.grad_scale = B.grad_scale = 1.0f;  // dL/dfeat already carries the scale
    INVR_CUDA(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
    INVR_CUDA(ctx, launch_encode_bwd(A, ctx->num_sms, ctx->side));
    if (side_adam) {  // the side field's update, beside the other field's scatter
      for (int b = 0; b < a->n_batches && !side_adam->done; ++b) {
        invr_field f = a->batches[b].views[0].field;
        if (f->params == P.v[A.view_lo].field.tables && !a->batches[b].views[0].deform) side_adam->done = f;
      }
      if (invr_field f = side_adam->done) {
        INVR_CUDA(ctx, launch_step_increment(f->step, ctx->side));
        INVR_CUDA(ctx, launch_adam(f->params, f->grads, f->grads, f->m, f->v, f->n_tab + f->n_w, f->step,
                                   side_adam->lr, side_adam->b1, side_adam->b2, side_adam->eps, ctx->side));
      }
    }
    INVR_CUDA(ctx, cudaEventRecord(ctx->ev_join, ctx->side));
    INVR_CUDA(ctx, launch_encode_bwd(B, ctx->num_sms, s));
    INVR_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev_join, 0));
    return INVR_OK;
  }
  if (plan_has_kind(P, kMlpF32)) INVR_CUDA(ctx, TIMED(ctx, "mlp_bwd", s, launch_mlp_bwd_f32(P, ctx->num_sms, s)));
  if (plan_has_kind(P, kMlpF16) || plan_has_kind(P, kMlpBF16))
    INVR_CUDA(ctx, TIMED(ctx, "mlp_bwd_tc", s, launch_mlp_bwd_tc(P, ctx->num_sms, s)));
  P.grad_scale = 1.0f;  // dL/dfeat already carries the scale
  if (P.has_deform) {
    // dL/dv_c through the field's encoding, then back through the net into its weights
    // (per-CTA partials, summed per net) and its tables
    INVR_CUDA(ctx, TIMED(ctx, "encode_dx", s, launch_encode_dx(P, ctx->num_sms, s)));
    std::vector<const DeformDev*> nets;
    for (int v = 0; v < P.n_views; ++v) {
      if (!P.v[v].has_deform) continue;
      bool seen = false;
      for (const DeformDev* q : nets) seen = seen || q->dw_scratch == P.v[v].deform.dw_scratch;
      if (!seen) nets.push_back(&P.v[v].deform);
    }
    for (const DeformDev* q : nets)
      INVR_CUDA(ctx, cudaMemsetAsync(q->dw_scratch, 0, (size_t)ctx->num_sms * q->n_w * sizeof(float), s));
    bool simt = false, tcn = false;
    for (int v = 0; v < P.n_views; ++v)
      if (P.v[v].has_deform) (P.v[v].deform.tc ? tcn : simt) = true;
    if (simt) INVR_CUDA(ctx, TIMED(ctx, "deform_bwd", s, launch_deform_backward(P, ctx->num_sms, s)));
    if (tcn) INVR_CUDA(ctx, TIMED(ctx, "deform_bwd_tc", s, launch_deform_backward_tc(P, ctx->num_sms, s)));
    for (const DeformDev* q : nets) INVR_CUDA(ctx, launch_deform_reduce(*q, ctx->num_sms, s));
    INVR_CUDA(ctx, TIMED(ctx, "deform_encode_bwd", s, deform_runs(P, true, [&](const Plan& Q) {
                           return launch_encode_bwd(Q, ctx->num_sms, s);
                         })));
  }
  INVR_CUDA(ctx, TIMED(ctx, "encode_bwd", s, launch_encode_bwd_by_field(P, ctx->num_sms, s)));
  return INVR_OK;
}

invr_status adam_step(invr_field f, float lr, float b1, float b2, float eps, cudaStream_t s) {
  invr_ctx ctx = f->ctx;
  INVR_CUDA(ctx, TIMED(ctx, "step_increment", s, launch_step_increment(f->step, s)));
  INVR_CUDA(ctx, TIMED(ctx, "adam", s,
                       launch_adam(f->params, f->grads, f->grads, f->m, f->v, f->n_tab + f->n_w, f->step, lr, b1,
                                   b2, eps, s)));
  return INVR_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* invr_status_string(invr_status s) {
  switch (s) {
    case INVR_OK: return "ok";
    case INVR_E_ARG: return "invalid argument";
    case INVR_E_OOM: return "out of device memory";
    case INVR_E_CUDA: return "CUDA error";
    case INVR_E_TIMEOUT: return "device wait timed out";
    case INVR_E_NONFINITE: return "non-finite value produced";
    case INVR_E_STATE: return "call out of order";
  }
  return "unknown status";
}

invr_status invr_ctx_create(invr_ctx* out, int device) {
  if (!out) return INVR_E_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return INVR_E_ARG;
  DeviceGuard guard(device);
  invr_ctx ctx = new invr_ctx_s();
  ctx->device = device;
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&ctx->status, sizeof(unsigned)) != cudaSuccess || cudaMemset(ctx->status, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&ctx->pose_bias, sizeof(float) * kMaxViews * kDeformMaxHidden) != cudaSuccess) {
    dfree(ctx->status);
    delete ctx;
    return INVR_E_OOM;
  }
  // the no-allocation query's scratch array and kernels are loaded here, where allocating is allowed
  if (noalloc_prepare(device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    dfree(ctx->status);
    dfree(ctx->pose_bias);
    delete ctx;
    return INVR_E_CUDA;
  }
  *out = ctx;
  return INVR_OK;
}

invr_status invr_ctx_destroy(invr_ctx ctx) {
  if (!ctx) return INVR_E_ARG;
  DeviceGuard guard(ctx->device);
  cudaDeviceSynchronize();
  clear_timing(ctx);
  free_workspace(ctx->ws);
  cudaEventDestroy(ctx->ev_fork);
  cudaEventDestroy(ctx->ev_join);
  cudaStreamDestroy(ctx->side);
  dfree(ctx->status);
  dfree(ctx->pose_bias);
  delete ctx;
  return INVR_OK;
}

invr_status invr_ctx_reserve(invr_ctx ctx, int64_t max_rays, int max_samples) {
  if (!ctx || max_rays < 0 || max_samples < 1 || max_samples > 1024) return fail(ctx, INVR_E_ARG, "bad reserve sizes");
  DeviceGuard guard(ctx->device);
  ctx->cap_fixed = false;
  ctx->cap_R = ctx->cap_S = 0;  // force a fresh allocation of exactly the reserved size
  ctx->cap_train = false;
  invr_status st = ensure_workspace(ctx, max_rays, max_rays * max_samples + (int64_t)kMaxViews * kTile, true, nullptr);
  if (st == INVR_OK) ctx->cap_fixed = true;
  return st;
}

invr_status invr_ctx_autotune(invr_ctx ctx, const invr_train_args* a, invr_stream stream) {
  if (!ctx || !a) return INVR_E_ARG;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (capturing(s)) return fail(ctx, INVR_E_STATE, "autotune cannot run during stream capture");
  const bool timing_was = ctx->timing;
  // time forward + backward (no optimiser step, parameters unchanged) per candidate
  auto measure = [&](float& ms) -> invr_status {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    ctx->timing = false;
    invr_status st = INVR_OK;
    float best = 1e30f;
    for (int rep = 0; rep < 3 && st == INVR_OK; ++rep) {
      cudaEventRecord(e0, s);
      st = train_forward(ctx, a, s);
      if (st == INVR_OK) st = train_backward(ctx, a, 1.0f, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float t = 0.0f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep > 0) best = std::min(best, t);  // first repetition warms caches
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ms = best;
    return st;
  };
  Tune best = ctx->tune;
  float best_ms = 0.0f;
  invr_status st = measure(best_ms);
  // coordinate descent over the launch shapes: the forward's structure first
  // (staged; fused with 256- or 128-sample work items: fused + 2 * (chunk == 128)),
  // then the grid sizes and the aggregation threshold
  const int form_c[] = {0, 1, 3}, warp_c[] = {2, 3, 4}, enc_c[] = {4, 8, 16, 32}, bwd_c[] = {1, 2, 4, 8},
            agg_c[] = {0, 64, 128, 256, 512, 1024};
  const int* dims[] = {form_c, warp_c, enc_c, bwd_c, agg_c};
  const int dim_n[] = {3, 3, 4, 4, 6};
  for (int dim = 0; dim < 5 && st == INVR_OK; ++dim) {
    const int* cands = dims[dim];
    const int n = dim_n[dim];
    if (dim == 1 && best.fused) continue;  // the staged warp's grid only matters to the staged path
    for (int i = 0; i < n && st == INVR_OK; ++i) {
      Tune t = best;
      if (dim == 0) {
        const int form = cands[i];
        if (t.fused == (form & 1) && (!t.fused || t.chunk == ((form & 2) ? 128 : 256))) continue;
        t.fused = form & 1;
        t.chunk = (form & 2) ? 128 : 256;
        ctx->tune = t;
        float ms = 0.0f;
        st = measure(ms);
        if (st == INVR_OK && ms < best_ms) {
          best_ms = ms;
          best = t;
        }
        continue;
      }
      int* slot = dim == 1 ? &t.warp_ctas_per_sm
                : dim == 2 ? &t.encode_ctas_per_sm : dim == 3 ? &t.encode_bwd_ctas_per_sm : &t.agg_res;
      if (*slot == cands[i]) continue;
      *slot = cands[i];
      ctx->tune = t;
      float ms = 0.0f;
      st = measure(ms);
      if (st == INVR_OK && ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
  }
  ctx->tune = best;
  ctx->timing = timing_was;
  ctx->fwd_valid = false;
  if (st != INVR_OK) return st;
  // the timed backward passes accumulated gradients: clear them
  for (int b = 0; b < a->n_batches; ++b) {
    invr_field f = a->batches[b].views[0].field;
    INVR_CUDA(ctx, cudaMemsetAsync(f->grads, 0, (f->n_tab + f->n_w) * sizeof(float), s));
  }
  INVR_CUDA(ctx, cudaStreamSynchronize(s));
  return INVR_OK;
}

invr_status invr_ctx_set_tune(invr_ctx ctx, const int* in) {
  if (!ctx) return INVR_E_ARG;
  if (!in) return fail(ctx, INVR_E_ARG, "null tune array");
  for (int i = 0; i < 3; ++i)
    if (in[i] < 1 || in[i] > 32) return fail(ctx, INVR_E_ARG, "CTAs per SM must be in [1, 32]");
  if (in[3] < 0 || in[3] > (1 << 20)) return fail(ctx, INVR_E_ARG, "aggregation resolution must be in [0, 2^20]");
  if (in[4] != 0 && in[4] != 1) return fail(ctx, INVR_E_ARG, "fused must be 0 or 1");
  if (in[5] != 128 && in[5] != 256) return fail(ctx, INVR_E_ARG, "the fused work item must be 128 or 256 samples");
  ctx->tune.warp_ctas_per_sm = in[0];
  ctx->tune.encode_ctas_per_sm = in[1];
  ctx->tune.encode_bwd_ctas_per_sm = in[2];
  ctx->tune.agg_res = in[3];
  ctx->tune.fused = in[4];
  ctx->tune.chunk = in[5];
  ctx->fwd_valid = false;
  return INVR_OK;
}

invr_status invr_ctx_set_wait_limit(invr_ctx ctx, uint32_t polls) {
  if (!ctx) return INVR_E_ARG;
  ctx->wait_limit = polls;
  return INVR_OK;
}

invr_status invr_ctx_get_tune(invr_ctx ctx, int* out) {
  if (!ctx || !out) return INVR_E_ARG;
  out[0] = ctx->tune.warp_ctas_per_sm;
  out[1] = ctx->tune.encode_ctas_per_sm;
  out[2] = ctx->tune.encode_bwd_ctas_per_sm;
  out[3] = ctx->tune.agg_res;
  out[4] = ctx->tune.fused;
  out[5] = ctx->tune.chunk;
  return INVR_OK;
}

invr_status invr_ctx_sync(invr_ctx ctx, invr_stream stream) {
  if (!ctx) return INVR_E_ARG;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  INVR_CUDA(ctx, cudaStreamSynchronize(s));
  unsigned st = 0;
  INVR_CUDA(ctx, cudaMemcpy(&st, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  INVR_CUDA(ctx, cudaMemset(ctx->status, 0, sizeof(unsigned)));
  // root causes first: a timed-out or skipped stage leaves later stages reading stale values
  if (st & kStatusDrainTimeout)
    return fail(ctx, INVR_E_TIMEOUT,
                "a bounded device wait gave up, and so did the drain of the kernel's own tensor-core work: "
                "results since the last sync are undefined and tensor memory may have been written after release; "
                "destroy this context");
  if (st & kStatusTimeout) return fail(ctx, INVR_E_TIMEOUT, "a bounded device wait gave up");
  if (st & kStatusOverflow) return fail(ctx, INVR_E_STATE, "sample workspace overflow");
  if (st & kStatusNonFinite) return fail(ctx, INVR_E_NONFINITE, "a kernel produced a non-finite output");
  return INVR_OK;
}

invr_status invr_ctx_enable_timing(invr_ctx ctx, int enable) {
  if (!ctx) return INVR_E_ARG;
  DeviceGuard guard(ctx->device);
  cudaDeviceSynchronize();
  clear_timing(ctx);
  ctx->timing = enable != 0;
  return INVR_OK;
}

int invr_ctx_timing(invr_ctx ctx, const char** names, double* ms, int64_t* launches, int max) {
  if (!ctx || max < 0) return INVR_E_ARG;
  DeviceGuard guard(ctx->device);
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(ctx, INVR_E_CUDA, "synchronize failed");
  int n = 0;
  for (const auto& r : ctx->recs) {
    float t = 0.0f;
    cudaEventElapsedTime(&t, r.a, r.b);
    int i = 0;
    while (i < n && std::strcmp(names[i], r.name) != 0) ++i;
    if (i == n) {
      if (n == max) continue;
      names[n] = r.name;
      ms[n] = 0.0;
      launches[n] = 0;
      ++n;
    }
    ms[i] += t;
    launches[i] += 1;
  }
  return n;
}

invr_status invr_last_error_detail(invr_ctx ctx, char* buf, size_t n) {
  if (!ctx || !buf || n == 0) return INVR_E_ARG;
  std::snprintf(buf, n, "%s", ctx->err.c_str());
  return INVR_OK;
}

int64_t invr_field_weight_count(const invr_field_desc* d) {
  if (!d) return -1;
  return weight_count(d->mlp_in, d->mlp_hidden, d->geo_out, d->col_hidden);
}

invr_status invr_field_create(invr_ctx ctx, const invr_field_desc* desc, invr_field* out) {
  if (!ctx || !out) return INVR_E_ARG;
  *out = nullptr;
  invr_status st = check_desc(ctx, desc);
  if (st != INVR_OK) return st;
  DeviceGuard guard(ctx->device);
  invr_field f = new invr_field_s();
  f->ctx = ctx;
  f->desc = *desc;
  f->n_tab = (int64_t)desc->L * ((int64_t)1 << desc->log2_T) * desc->F;
  f->n_w = weight_count(desc->mlp_in, desc->mlp_hidden, desc->geo_out, desc->col_hidden);
  for (int l = 0; l < desc->L; ++l) {
    f->res[l] = level_resolution(desc->N_min, desc->growth, l);
    const int64_t v = (int64_t)f->res[l] + 1;
    if (v * v * v <= ((int64_t)1 << desc->log2_T)) f->dense_mask |= 1u << l;
  }
  const int64_t n = f->n_tab + f->n_w;
  if (dmalloc(&f->params, n) != cudaSuccess || dmalloc(&f->grads, n) != cudaSuccess ||
      dmalloc(&f->m, n) != cudaSuccess || dmalloc(&f->v, n) != cudaSuccess || dmalloc(&f->step, 1) != cudaSuccess ||
      dmalloc(&f->wt, kWtF32) != cudaSuccess || dmalloc(&f->w16, kW16Bytes) != cudaSuccess) {
    dfree(f->params); dfree(f->grads); dfree(f->m); dfree(f->v); dfree(f->step); dfree(f->wt); dfree(f->w16);
    delete f;
    return fail(ctx, INVR_E_OOM, "field allocation failed");
  }
  cudaMemset(f->grads, 0, n * sizeof(float));
  cudaMemset(f->m, 0, n * sizeof(float));
  cudaMemset(f->v, 0, n * sizeof(float));
  cudaMemset(f->step, 0, sizeof(int64_t));
  INVR_CUDA(ctx, cudaDeviceSynchronize());
  *out = f;
  return INVR_OK;
}

invr_status invr_field_destroy(invr_field f) {
  if (!f) return INVR_E_ARG;
  DeviceGuard guard(f->ctx->device);
  cudaDeviceSynchronize();
  dfree(f->params); dfree(f->grads); dfree(f->m); dfree(f->v); dfree(f->step); dfree(f->wt); dfree(f->w16);
  delete f;
  return INVR_OK;
}

invr_status invr_field_set_params(invr_field f, const float* tables_dev, const float* weights_dev, invr_stream stream) {
  if (!f) return INVR_E_ARG;
  invr_ctx ctx = f->ctx;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (tables_dev) INVR_CUDA(ctx, cudaMemcpyAsync(f->params, tables_dev, f->n_tab * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (weights_dev)
    INVR_CUDA(ctx, cudaMemcpyAsync(f->params + f->n_tab, weights_dev, f->n_w * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return INVR_OK;
}

invr_status invr_field_get_params(invr_field f, float* tables_dev, float* weights_dev, float* m_dev, float* v_dev,
                                  int64_t* step, invr_stream stream) {
  if (!f) return INVR_E_ARG;
  invr_ctx ctx = f->ctx;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = f->n_tab + f->n_w;
  if (tables_dev) INVR_CUDA(ctx, cudaMemcpyAsync(tables_dev, f->params, f->n_tab * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (weights_dev)
    INVR_CUDA(ctx, cudaMemcpyAsync(weights_dev, f->params + f->n_tab, f->n_w * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (m_dev) INVR_CUDA(ctx, cudaMemcpyAsync(m_dev, f->m, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (v_dev) INVR_CUDA(ctx, cudaMemcpyAsync(v_dev, f->v, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (step) {
    INVR_CUDA(ctx, cudaStreamSynchronize(s));
    INVR_CUDA(ctx, cudaMemcpy(step, f->step, sizeof(int64_t), cudaMemcpyDeviceToHost));
  }
  return INVR_OK;
}

invr_status invr_field_copy_params(invr_field dst, invr_field src, invr_stream stream) {
  if (!dst || !src) return INVR_E_ARG;
  invr_ctx ctx = dst->ctx;
  if (src->ctx->device != ctx->device) return fail(ctx, INVR_E_ARG, "fields on different devices");
  if (dst->n_tab != src->n_tab || dst->n_w != src->n_w || dst->desc.L != src->desc.L ||
      dst->desc.N_min != src->desc.N_min || dst->desc.growth != src->desc.growth)
    return fail(ctx, INVR_E_ARG, "field descriptions differ");
  DeviceGuard guard(ctx->device);
  INVR_CUDA(ctx, cudaMemcpyAsync(dst->params, src->params, (src->n_tab + src->n_w) * sizeof(float),
                                 cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
  return INVR_OK;
}

invr_status invr_field_get_grads(invr_field f, float* gt_dev, float* gw_dev, invr_stream stream) {
  if (!f) return INVR_E_ARG;
  invr_ctx ctx = f->ctx;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (gt_dev) INVR_CUDA(ctx, cudaMemcpyAsync(gt_dev, f->grads, f->n_tab * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (gw_dev)
    INVR_CUDA(ctx, cudaMemcpyAsync(gw_dev, f->grads + f->n_tab, f->n_w * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return INVR_OK;
}

invr_status invr_field_zero_grads(invr_field f, invr_stream stream) {
  if (!f) return INVR_E_ARG;
  invr_ctx ctx = f->ctx;
  DeviceGuard guard(ctx->device);
  INVR_CUDA(ctx, cudaMemsetAsync(f->grads, 0, (f->n_tab + f->n_w) * sizeof(float), static_cast<cudaStream_t>(stream)));
  return INVR_OK;
}

invr_status invr_graph_create(invr_ctx ctx, const invr_graph_desc* desc, const float* x_canon_dev, invr_graph* out) {
  if (!ctx || !out || !desc) return INVR_E_ARG;
  *out = nullptr;
  if (desc->K < 1 || desc->K > 8 || desc->n_nodes < desc->K || desc->n_nodes > 65535)
    return fail(ctx, INVR_E_ARG, "need 1 <= K <= 8 and K <= n_nodes <= 65535");
  if (desc->n_frames < 1 || !(desc->radius > 0.0f)) return fail(ctx, INVR_E_ARG, "need n_frames >= 1 and radius > 0");
  DeviceGuard guard(ctx->device);
  invr_graph g = new invr_graph_s();
  g->ctx = ctx;
  g->desc = *desc;
  g->frames.resize(desc->n_frames);
  g->cap = desc->n_nodes <= 64 ? 0 : (desc->K <= 4 ? 64 : 128);
  if (dmalloc(&g->x_canon, 3 * (size_t)desc->n_nodes) != cudaSuccess) {
    delete g;
    return fail(ctx, INVR_E_OOM, "graph allocation failed");
  }
  if (x_canon_dev)
    INVR_CUDA(ctx, cudaMemcpy(g->x_canon, x_canon_dev, 3 * (size_t)desc->n_nodes * sizeof(float), cudaMemcpyDeviceToDevice));
  *out = g;
  return INVR_OK;
}

invr_status invr_graph_set_pose(invr_graph g, int frame, const float* dq_dev, const float* x_live_dev, invr_stream stream) {
  if (!g) return INVR_E_ARG;
  invr_ctx ctx = g->ctx;
  if (frame < 0 || frame >= (int)g->frames.size()) return fail(ctx, INVR_E_ARG, "frame out of range");
  if (!dq_dev || !x_live_dev) return fail(ctx, INVR_E_ARG, "null pose pointer");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto& fr = g->frames[frame];
  const int N = g->desc.n_nodes;
  if (!fr.x_live) {
    if (capturing(s)) return fail(ctx, INVR_E_STATE, "first pose of a frame cannot be set during capture");
    INVR_CUDA(ctx, dmalloc(&fr.x_live, N));
    INVR_CUDA(ctx, dmalloc(&fr.dq, 2 * (size_t)N));
    if (g->cap > 0) {
      const size_t cells = (size_t)kKnnG * kKnnG * kKnnG;
      INVR_CUDA(ctx, dmalloc(&fr.cand, cells * g->cap));
      INVR_CUDA(ctx, dmalloc(&fr.cand_head, cells * kKnnHead));
    }
  }
  INVR_CUDA(ctx, TIMED(ctx, "graph_pack", s, launch_graph_pack(dq_dev, x_live_dev, N, fr.dq, fr.x_live, s)));
  if (g->cap > 0) {
    if (!g->coarse) {
      if (capturing(s)) return fail(ctx, INVR_E_STATE, "first pose of a graph cannot be set during capture");
      const size_t cc = (size_t)(kKnnG / 2) * (kKnnG / 2) * (kKnnG / 2);
      INVR_CUDA(ctx, dmalloc(&g->coarse, cc * kKnnCoarseCapFactor * g->cap));
      INVR_CUDA(ctx, dmalloc(&g->coarse_n, cc));
    }
    INVR_CUDA(ctx, TIMED(ctx, "knn_grid_build", s,
                         launch_knn_grid_build(fr.x_live, N, g->desc.K, g->cap, g->coarse, g->coarse_n, fr.cand,
                                               fr.cand_head, ctx->num_sms, s)));
  }
  if (g->lut_res > 0) {
    const size_t G3 = (size_t)g->lut_res * g->lut_res * g->lut_res;
    if (!fr.lut_live) {
      if (capturing(s)) return fail(ctx, INVR_E_STATE, "first pose of a frame cannot be set during capture");
      INVR_CUDA(ctx, dmalloc(&fr.lut_live, G3));
    }
    INVR_CUDA(ctx, TIMED(ctx, "lut_live", s,
                         launch_lut_live(g->x_canon4, fr.dq, N, g->desc.K, 1.0f / (g->desc.radius * g->desc.radius),
                                         g->lut_res, g->lut_canon, fr.lut_live, ctx->num_sms, s)));
  }
  fr.set = true;
  return INVR_OK;
}

static void free_lut(invr_graph g) {
  for (auto& fr : g->frames) {
    dfree(fr.lut_live);
    fr.lut_live = nullptr;
  }
  dfree(g->lut_canon); dfree(g->x_canon4); dfree(g->canon_cand); dfree(g->canon_cand_head);
  g->lut_canon = nullptr; g->x_canon4 = nullptr; g->canon_cand = nullptr; g->canon_cand_head = nullptr;
  g->lut_res = 0;
}

invr_status invr_graph_enable_lut(invr_graph g, int resolution, invr_stream stream) {
  if (!g) return INVR_E_ARG;
  invr_ctx ctx = g->ctx;
  if (resolution < 4 || resolution > 1024 || (resolution & (resolution - 1)))
    return fail(ctx, INVR_E_ARG, "table resolution must be a power of two in [4, 1024]");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (capturing(s)) return fail(ctx, INVR_E_STATE, "tables cannot be built during capture");
  if (g->lut_res > 0) {
    cudaDeviceSynchronize();
    free_lut(g);
  }
  const int N = g->desc.n_nodes, K = g->desc.K;
  const size_t G3 = (size_t)resolution * resolution * resolution;
  if (dmalloc(&g->lut_canon, G3 * K) != cudaSuccess || dmalloc(&g->x_canon4, (size_t)N) != cudaSuccess) {
    free_lut(g);
    return fail(ctx, INVR_E_OOM, "table allocation failed");
  }
  if (g->cap > 0) {
    const size_t cells = (size_t)kKnnG * kKnnG * kKnnG;
    if (dmalloc(&g->canon_cand, cells * g->cap) != cudaSuccess || dmalloc(&g->canon_cand_head, cells * kKnnHead) != cudaSuccess) {
      free_lut(g);
      return fail(ctx, INVR_E_OOM, "table allocation failed");
    }
  }
  for (auto& fr : g->frames) {
    if (fr.set && dmalloc(&fr.lut_live, G3) != cudaSuccess) {
      free_lut(g);
      return fail(ctx, INVR_E_OOM, "table allocation failed");
    }
  }
  g->lut_res = resolution;
  INVR_CUDA(ctx, launch_pack_points(g->x_canon, N, g->x_canon4, s));
  if (g->cap > 0) {
    if (!g->coarse) {
      const size_t cc = (size_t)(kKnnG / 2) * (kKnnG / 2) * (kKnnG / 2);
      INVR_CUDA(ctx, dmalloc(&g->coarse, cc * kKnnCoarseCapFactor * g->cap));
      INVR_CUDA(ctx, dmalloc(&g->coarse_n, cc));
    }
    INVR_CUDA(ctx, launch_knn_grid_build(g->x_canon4, N, K, g->cap, g->coarse, g->coarse_n, g->canon_cand,
                                         g->canon_cand_head, ctx->num_sms, s));
  }
  INVR_CUDA(ctx, TIMED(ctx, "lut_canon", s,
                       launch_lut_canon(g->x_canon4, N, K, g->canon_cand, g->canon_cand_head, g->cap, resolution,
                                        g->lut_canon, ctx->num_sms, s)));
  for (auto& fr : g->frames) {
    if (!fr.set) continue;
    INVR_CUDA(ctx, TIMED(ctx, "lut_live", s,
                         launch_lut_live(g->x_canon4, fr.dq, N, K, 1.0f / (g->desc.radius * g->desc.radius),
                                         resolution, g->lut_canon, fr.lut_live, ctx->num_sms, s)));
  }
  return INVR_OK;
}

invr_status invr_graph_disable_lut(invr_graph g) {
  if (!g) return INVR_E_ARG;
  DeviceGuard guard(g->ctx->device);
  cudaDeviceSynchronize();
  free_lut(g);
  return INVR_OK;
}

invr_status invr_graph_get_lut(invr_graph g, int frame, uint16_t* canon_dev, uint32_t* live_dev, invr_stream stream) {
  if (!g) return INVR_E_ARG;
  invr_ctx ctx = g->ctx;
  if (g->lut_res == 0) return fail(ctx, INVR_E_STATE, "graph has no tables (invr_graph_enable_lut)");
  if (frame < 0 || frame >= (int)g->frames.size()) return fail(ctx, INVR_E_ARG, "frame out of range");
  if (live_dev && !g->frames[frame].lut_live) return fail(ctx, INVR_E_STATE, "frame pose not set");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t G3 = (size_t)g->lut_res * g->lut_res * g->lut_res;
  if (canon_dev)
    INVR_CUDA(ctx, cudaMemcpyAsync(canon_dev, g->lut_canon, G3 * g->desc.K * sizeof(uint16_t),
                                   cudaMemcpyDeviceToDevice, s));
  if (live_dev)
    INVR_CUDA(ctx, cudaMemcpyAsync(live_dev, g->frames[frame].lut_live, G3 * sizeof(uint32_t),
                                   cudaMemcpyDeviceToDevice, s));
  return INVR_OK;
}

invr_status invr_graph_destroy(invr_graph g) {
  if (!g) return INVR_E_ARG;
  DeviceGuard guard(g->ctx->device);
  cudaDeviceSynchronize();
  free_lut(g);
  for (auto& fr : g->frames) {
    dfree(fr.x_live); dfree(fr.dq); dfree(fr.cand); dfree(fr.cand_head);
  }
  dfree(g->coarse); dfree(g->coarse_n);
  dfree(g->x_canon);
  delete g;
  return INVR_OK;
}

static invr_status render(invr_ctx ctx, const invr_render_args* a, bool joint, invr_stream stream) {
  if (!ctx || !a) return INVR_E_ARG;
  if (a->n_views < 1 || a->n_views > 2 || !a->views) return fail(ctx, INVR_E_ARG, "render takes 1 or 2 views");
  if (joint && a->n_views != 2) return fail(ctx, INVR_E_ARG, "joint compositing takes 2 views");
  if (a->n_rays > 0 && (!a->rgba_dev || !a->depth_dev)) return fail(ctx, INVR_E_ARG, "null output pointer");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (a->n_rays == 0) return INVR_OK;
  std::vector<const invr_render_args*> rays(a->n_views, a);
  std::vector<const invr_field_view*> views;
  for (int v = 0; v < a->n_views; ++v) views.push_back(&a->views[v]);
  Plan P;
  invr_status st = build_plan(ctx, rays, views, a->n_samples, a->t_eps, P);
  if (st != INVR_OK) return st;
  st = ensure_workspace(ctx, P.total_rays, P.total_rays * a->n_samples + (int64_t)P.n_views * kTile, false, s);
  if (st != INVR_OK) return st;
  if (P.has_deform && (st = ensure_deform_workspace(ctx, s)) != INVR_OK) return st;
  P.ws = ctx->ws;
  ctx->fwd_valid = false;
  INVR_CUDA(ctx, run_forward(ctx, P, s));
  if (joint) {
    INVR_CUDA(ctx, TIMED(ctx, "composite_joint", s, launch_composite_joint(P, a->n_rays, a->rgba_dev, a->depth_dev, s)));
  } else {
    INVR_CUDA(ctx, TIMED(ctx, "composite_render", s,
                         launch_composite_render(P, a->n_rays, a->rgba_dev, a->depth_dev, s)));
  }
  return INVR_OK;
}

invr_status invr_render_rays(invr_ctx ctx, const invr_render_args* a, invr_stream stream) {
  return render(ctx, a, false, stream);
}

invr_status invr_render_rays_joint(invr_ctx ctx, const invr_render_args* a, invr_stream stream) {
  return render(ctx, a, true, stream);
}

invr_status invr_field_forward_train(invr_ctx ctx, const invr_train_args* a, invr_stream stream) {
  if (!ctx) return INVR_E_ARG;
  DeviceGuard guard(ctx->device);
  return train_forward(ctx, a, static_cast<cudaStream_t>(stream));
}

invr_status invr_field_backward(invr_ctx ctx, const invr_train_args* a, float grad_scale, invr_stream stream) {
  if (!ctx) return INVR_E_ARG;
  DeviceGuard guard(ctx->device);
  return train_backward(ctx, a, grad_scale, static_cast<cudaStream_t>(stream));
}

invr_status invr_field_adam(invr_field f, float lr, float b1, float b2, float eps, invr_stream stream) {
  if (!f) return INVR_E_ARG;
  DeviceGuard guard(f->ctx->device);
  return adam_step(f, lr, b1, b2, eps, static_cast<cudaStream_t>(stream));
}

invr_status invr_train_step(invr_ctx ctx, const invr_train_args* a, invr_stream stream) {
  if (!ctx) return INVR_E_ARG;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  invr_status st = train_forward(ctx, a, s);
  if (st != INVR_OK) return st;
  SideAdam side{a->lr, a->beta1, a->beta2, a->adam_eps};
  st = train_backward(ctx, a, 1.0f, s, &side);
  if (st != INVR_OK) return st;
  std::vector<invr_field> done;
  if (side.done) done.push_back(side.done);
  std::vector<invr_deform> nets;
  for (int b = 0; b < a->n_batches; ++b) {
    invr_field f = a->batches[b].views[0].field;
    invr_deform d = a->batches[b].views[0].deform;
    if (d && std::find(nets.begin(), nets.end(), d) == nets.end()) {
      nets.push_back(d);
      INVR_CUDA(ctx, TIMED(ctx, "step_increment", s, launch_step_increment(d->step, s)));
      INVR_CUDA(ctx, TIMED(ctx, "adam", s,
                           launch_adam(d->params, d->grads, d->grads, d->m, d->v, d->n_tab + d->n_w, d->step, a->lr,
                                       a->beta1, a->beta2, a->adam_eps, s)));
    }
    if (std::find(done.begin(), done.end(), f) != done.end()) continue;
    done.push_back(f);
    st = adam_step(f, a->lr, a->beta1, a->beta2, a->adam_eps, s);
    if (st != INVR_OK) return st;
  }
  return INVR_OK;
}

invr_status invr_deform_create(invr_ctx ctx, const invr_deform_desc* desc, invr_deform* out) {
  if (!ctx || !out || !desc) return INVR_E_ARG;
  *out = nullptr;
  const invr_deform_desc& q = *desc;
  if (q.F != 2 || q.L < 1 || q.L > kMaxL || q.L * q.F > kDeformMaxFeat || (q.L * q.F) % 8 || q.log2_T < 4 ||
      q.log2_T > 24 || q.N_min < 2 || !(q.growth >= 1.0) || q.hidden < 16 || q.hidden > kDeformMaxHidden ||
      q.hidden % 16 || q.n_hidden < 1 || q.n_hidden > kDeformMaxLayers || q.pose_dim < 0 ||
      q.pose_dim > kDeformMaxPose)
    return fail(ctx, INVR_E_ARG,
                "deformation net: F = 2, L*F a multiple of 8 up to 32, hidden a multiple of 16 up to 128, "
                "1..4 hidden layers, pose_dim <= 128");
  if (q.prec != INVR_FP32 && q.prec != INVR_MLP_FP16 && q.prec != INVR_MLP_BF16)
    return fail(ctx, INVR_E_ARG, "unknown precision");
  if (q.prec != INVR_FP32 && (q.hidden != kDeformMaxHidden || q.L * q.F != kDeformMaxFeat ||
                              q.pose_dim > kDeformTcMaxPose))
    return fail(ctx, INVR_E_ARG, "a tensor-core deformation net has 32 features, hidden 128 and pose_dim <= 80");
  DeviceGuard guard(ctx->device);
  invr_deform d = new invr_deform_s();
  d->ctx = ctx;
  d->desc = q;
  d->n_tab = (int64_t)q.L * ((int64_t)1 << q.log2_T) * q.F;
  d->n_w = (int64_t)q.hidden * (q.L * q.F + q.pose_dim) + (int64_t)(q.n_hidden - 1) * q.hidden * q.hidden +
           3 * (int64_t)q.hidden;
  for (int l = 0; l < q.L; ++l) {
    d->res[l] = level_resolution(q.N_min, q.growth, l);
    const int64_t v = (int64_t)d->res[l] + 1;
    if (v * v * v <= ((int64_t)1 << q.log2_T)) d->dense_mask |= 1u << l;
  }
  const int64_t n = d->n_tab + d->n_w;
  if (dmalloc(&d->params, n) != cudaSuccess || dmalloc(&d->grads, n) != cudaSuccess ||
      dmalloc(&d->m, n) != cudaSuccess || dmalloc(&d->v, n) != cudaSuccess || dmalloc(&d->step, 1) != cudaSuccess ||
      dmalloc(&d->scratch, (size_t)ctx->num_sms * d->n_w) != cudaSuccess) {
    dfree(d->params); dfree(d->grads); dfree(d->m); dfree(d->v); dfree(d->step); dfree(d->scratch);
    delete d;
    return fail(ctx, INVR_E_OOM, "deformation net allocation failed");
  }
  cudaMemset(d->params, 0, n * sizeof(float));
  cudaMemset(d->grads, 0, n * sizeof(float));
  cudaMemset(d->m, 0, n * sizeof(float));
  cudaMemset(d->v, 0, n * sizeof(float));
  cudaMemset(d->step, 0, sizeof(int64_t));
  INVR_CUDA(ctx, cudaDeviceSynchronize());
  *out = d;
  return INVR_OK;
}

invr_status invr_deform_destroy(invr_deform d) {
  if (!d) return INVR_E_ARG;
  DeviceGuard guard(d->ctx->device);
  cudaDeviceSynchronize();
  dfree(d->params); dfree(d->grads); dfree(d->m); dfree(d->v); dfree(d->step); dfree(d->scratch);
  delete d;
  return INVR_OK;
}

invr_status invr_deform_set_params(invr_deform d, const float* tables, const float* weights, invr_stream stream) {
  if (!d) return INVR_E_ARG;
  invr_ctx ctx = d->ctx;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (tables) INVR_CUDA(ctx, cudaMemcpyAsync(d->params, tables, d->n_tab * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (weights)
    INVR_CUDA(ctx, cudaMemcpyAsync(d->params + d->n_tab, weights, d->n_w * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return INVR_OK;
}

invr_status invr_deform_get_params(invr_deform d, float* tables, float* weights, invr_stream stream) {
  if (!d) return INVR_E_ARG;
  invr_ctx ctx = d->ctx;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (tables) INVR_CUDA(ctx, cudaMemcpyAsync(tables, d->params, d->n_tab * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (weights)
    INVR_CUDA(ctx, cudaMemcpyAsync(weights, d->params + d->n_tab, d->n_w * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return INVR_OK;
}

invr_status invr_deform_get_grads(invr_deform d, float* gt, float* gw, invr_stream stream) {
  if (!d) return INVR_E_ARG;
  invr_ctx ctx = d->ctx;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (gt) INVR_CUDA(ctx, cudaMemcpyAsync(gt, d->grads, d->n_tab * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (gw) INVR_CUDA(ctx, cudaMemcpyAsync(gw, d->grads + d->n_tab, d->n_w * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return INVR_OK;
}

invr_status invr_deform_zero_grads(invr_deform d, invr_stream stream) {
  if (!d) return INVR_E_ARG;
  invr_ctx ctx = d->ctx;
  DeviceGuard guard(ctx->device);
  INVR_CUDA(ctx, cudaMemsetAsync(d->grads, 0, (d->n_tab + d->n_w) * sizeof(float), static_cast<cudaStream_t>(stream)));
  return INVR_OK;
}

invr_status invr_ray_samples(invr_ctx ctx, int64_t n_rays, const float* o, const float* d, int n_samples,
                             const uint32_t* occ, int32_t* count, float* t, float* p, invr_stream stream) {
  if (!ctx || n_rays < 0 || n_samples < 1 || n_samples > 1024) return fail(ctx, INVR_E_ARG, "bad ray_samples sizes");
  if (n_rays > 0 && (!o || !d || !count || !t || !p)) return fail(ctx, INVR_E_ARG, "null pointer");
  DeviceGuard guard(ctx->device);
  INVR_CUDA(ctx, launch_ray_samples(n_rays, o, d, n_samples, occ, count, t, p, static_cast<cudaStream_t>(stream)));
  return INVR_OK;
}

invr_status invr_probe_l2_read(invr_ctx ctx, const float* buf, int64_t n_floats, int passes, float* sink,
                               invr_stream stream) {
  if (!ctx || !buf || !sink || n_floats < 4 || n_floats % 4 || passes < 1 || (uintptr_t)buf % 16)
    return fail(ctx, INVR_E_ARG, "bad probe_l2_read arguments");
  DeviceGuard guard(ctx->device);
  INVR_CUDA(ctx, launch_probe_l2_read(buf, n_floats, passes, sink, ctx->num_sms, static_cast<cudaStream_t>(stream)));
  return INVR_OK;
}

invr_status invr_probe_l2_gather(invr_ctx ctx, const float* table, int64_t n_floats, int width, int64_t n_ops,
                                 float* sink, invr_stream stream) {
  if (!ctx || !table || !sink || n_floats < 4 || n_floats % 4 || n_floats / 2 > 0xFFFFFFFFll ||
      (width != 2 && width != 4 && width != 8) || n_ops < 0 || (uintptr_t)table % 16 ||
      (width == 8 && (n_floats % 8 || (uintptr_t)table % 32)))
    return fail(ctx, INVR_E_ARG, "bad probe_l2_gather arguments");
  DeviceGuard guard(ctx->device);
  INVR_CUDA(ctx, launch_probe_l2_gather(table, n_floats, width, n_ops, sink, ctx->num_sms,
                                        static_cast<cudaStream_t>(stream)));
  return INVR_OK;
}

invr_status invr_probe_l2_atomic(invr_ctx ctx, float* table, int64_t n_floats, int width, int64_t n_ops,
                                 invr_stream stream) {
  if (!ctx || !table || n_floats < 4 || n_floats % 4 || n_floats / 2 > 0xFFFFFFFFll || (width != 2 && width != 4) ||
      n_ops < 0 || (uintptr_t)table % 16)
    return fail(ctx, INVR_E_ARG, "bad probe_l2_atomic arguments");
  DeviceGuard guard(ctx->device);
  INVR_CUDA(ctx, launch_probe_l2_atomic(table, n_floats, width, n_ops, ctx->num_sms, static_cast<cudaStream_t>(stream)));
  return INVR_OK;
}

invr_status invr_warp_points(invr_ctx ctx, const invr_field_view* view, int64_t n, const float* p, float* vc,
                             int32_t* ids, invr_stream stream) {
  if (!ctx || !view || n < 0) return fail(ctx, INVR_E_ARG, "bad warp_points arguments");
  if (view->deform) return fail(ctx, INVR_E_ARG, "per-point calls do not run the deformation net");
  if (n > 0 && (!p || !vc)) return fail(ctx, INVR_E_ARG, "null pointer");
  DeviceGuard guard(ctx->device);
  WarpDev W;
  invr_status st = warp_dev(ctx, *view, W);
  if (st != INVR_OK) return st;
  INVR_CUDA(ctx, launch_warp_points(W, n, p, vc, W.mode == 1 ? ids : nullptr, static_cast<cudaStream_t>(stream)));
  return INVR_OK;
}

invr_status invr_encode_points(invr_ctx ctx, invr_field f, int64_t n, const float* x, float* feat, uint32_t* idx,
                               invr_stream stream) {
  if (!ctx || n < 0) return fail(ctx, INVR_E_ARG, "bad encode_points arguments");
  invr_status st = check_field(ctx, f);
  if (st != INVR_OK) return st;
  if (n > 0 && (!x || !feat)) return fail(ctx, INVR_E_ARG, "null pointer");
  DeviceGuard guard(ctx->device);
  INVR_CUDA(ctx, launch_encode_points(field_dev(f), n, x, feat, idx, static_cast<cudaStream_t>(stream)));
  return INVR_OK;
}

invr_status invr_mlp_points(invr_ctx ctx, invr_field f, int64_t n, const float* feat, float* out, invr_stream stream) {
  if (!ctx || n < 0) return fail(ctx, INVR_E_ARG, "bad mlp_points arguments");
  invr_status st = check_field(ctx, f);
  if (st != INVR_OK) return st;
  if (n > 0 && (!feat || !out)) return fail(ctx, INVR_E_ARG, "null pointer");
  DeviceGuard guard(ctx->device);
  const FieldDev F = field_dev(f);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (F.mlp_kind == kMlpF32)
    INVR_CUDA(ctx, launch_mlp_points_f32(F, n, feat, out, ctx->num_sms, s));
  else
    INVR_CUDA(ctx, launch_mlp_points_tc(F, n, feat, out, ctx->status, ctx->wait_limit, ctx->num_sms, s));
  return INVR_OK;
}

invr_status invr_query_points(invr_ctx ctx, const invr_field_view* view, int64_t n, const float* p, float* out,
                              invr_stream stream) {
  if (!ctx || !view || n < 0) return fail(ctx, INVR_E_ARG, "bad query_points arguments");
  if (view->deform) return fail(ctx, INVR_E_ARG, "per-point calls do not run the deformation net");
  invr_status st = check_field(ctx, view->field);
  if (st != INVR_OK) return st;
  if (n == 0) return INVR_OK;
  if (!p || !out) return fail(ctx, INVR_E_ARG, "null pointer");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  WarpDev W;
  st = warp_dev(ctx, *view, W);
  if (st != INVR_OK) return st;
  float *vc = nullptr, *feat = nullptr;
  INVR_CUDA(ctx, cudaMallocAsync(reinterpret_cast<void**>(&vc), 3 * n * sizeof(float), s));
  INVR_CUDA(ctx, cudaMallocAsync(reinterpret_cast<void**>(&feat), (size_t)view->field->desc.mlp_in * n * sizeof(float), s));
  const FieldDev F = field_dev(view->field);
  cudaError_t e = launch_warp_points(W, n, p, vc, nullptr, s);
  if (e == cudaSuccess) e = launch_encode_points(F, n, vc, feat, nullptr, s);
  if (e == cudaSuccess)
    e = F.mlp_kind == kMlpF32 ? launch_mlp_points_f32(F, n, feat, out, ctx->num_sms, s)
                              : launch_mlp_points_tc(F, n, feat, out, ctx->status, ctx->wait_limit, ctx->num_sms, s);
  cudaFreeAsync(vc, s);
  cudaFreeAsync(feat, s);
  INVR_CUDA(ctx, e);
  return INVR_OK;
}

invr_status invr_occupancy_update(invr_ctx ctx, const invr_field_view* view, float decay, float threshold,
                                  float* density, uint32_t* bits, invr_stream stream) {
  if (!ctx || !view) return INVR_E_ARG;
  if (!density || !bits) return fail(ctx, INVR_E_ARG, "null density or bits");
  if (view->deform) return fail(ctx, INVR_E_ARG, "per-point calls do not run the deformation net");
  if (!(decay >= 0.0f && decay <= 1.0f)) return fail(ctx, INVR_E_ARG, "decay must lie in [0, 1]");
  invr_status st = check_field(ctx, view->field);
  if (st != INVR_OK) return st;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  WarpDev W;
  st = warp_dev(ctx, *view, W);
  if (st != INVR_OK) return st;
  const int64_t n = (int64_t)kOccRes * kOccRes * kOccRes;
  const FieldDev F = field_dev(view->field);
  float *p = nullptr, *vc = nullptr, *feat = nullptr, *out = nullptr;
  INVR_CUDA(ctx, cudaMallocAsync(reinterpret_cast<void**>(&p), 3 * n * sizeof(float), s));
  INVR_CUDA(ctx, cudaMallocAsync(reinterpret_cast<void**>(&vc), 3 * n * sizeof(float), s));
  INVR_CUDA(ctx, cudaMallocAsync(reinterpret_cast<void**>(&feat), (size_t)view->field->desc.mlp_in * n * sizeof(float), s));
  INVR_CUDA(ctx, cudaMallocAsync(reinterpret_cast<void**>(&out), 4 * n * sizeof(float), s));
  cudaError_t e = TIMED(ctx, "occ_centres", s, launch_occ_centres(p, n, s));
  if (e == cudaSuccess) e = TIMED(ctx, "warp_points", s, launch_warp_points(W, n, p, vc, nullptr, s));
  if (e == cudaSuccess) e = TIMED(ctx, "encode_points", s, launch_encode_points(F, n, vc, feat, nullptr, s));
  if (e == cudaSuccess)
    e = TIMED(ctx, "mlp_points", s,
              F.mlp_kind == kMlpF32 ? launch_mlp_points_f32(F, n, feat, out, ctx->num_sms, s)
                                    : launch_mlp_points_tc(F, n, feat, out, ctx->status, ctx->wait_limit,
                                                           ctx->num_sms, s));
  if (e == cudaSuccess) e = TIMED(ctx, "occ_update", s, launch_occ_update(out, n, decay, threshold, density, bits, s));
  cudaFreeAsync(p, s);
  cudaFreeAsync(vc, s);
  cudaFreeAsync(feat, s);
  cudaFreeAsync(out, s);
  INVR_CUDA(ctx, e);
  return INVR_OK;
}

}  // extern "C"

// Helpers for entry points defined in other files (the no-allocation query).
namespace invr {

invr_status resolve_point_query(invr_ctx ctx, const invr_field_view* view, WarpDev& W, FieldDev& F, int& device,
                                int& num_sms, unsigned*& status, uint32_t& wait_limit) {
  if (!ctx || !view) return INVR_E_ARG;
  if (view->deform) return fail(ctx, INVR_E_ARG, "per-point calls do not run the deformation net");
  invr_status st = check_field(ctx, view->field);
  if (st != INVR_OK) return st;
  st = warp_dev(ctx, *view, W);
  if (st != INVR_OK) return st;
  F = field_dev(view->field);
  device = ctx->device;
  num_sms = ctx->num_sms;
  status = ctx->status;
  wait_limit = ctx->wait_limit;
  return INVR_OK;
}

invr_status record_error(invr_ctx ctx, invr_status st, const char* msg) { return fail(ctx, st, msg); }

}  // namespace invr
