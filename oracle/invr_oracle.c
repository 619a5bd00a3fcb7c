/*
 * invr_oracle.c -- plain, slow FP64 CPU oracle of the deformed hash-grid radiance field
 * of Instant-NVR (Sec. 4.2): warp a live-space sample to canonical space (Eq. 4 for the
 * human field, the tracked rigid pose for the object field), multiresolution hash
 * encoding, geometry and colour MLPs, front-to-back volume rendering, the Huber colour
 * loss, its analytic gradient, and Adam.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg use it.  It
 * shares no code, header, table or constant generator with the CUDA library.
 *
 * Conventions
 *   - Everything continuous is computed in double precision.
 *   - Discrete decisions (sample positions, occupancy cell, nearest-node selection, hash
 *     cell) follow fixed FP32 operation sequences written below with C `float` and
 *     compiled with -ffp-contract=off, so that any FP32 implementation that performs the
 *     same rounded operations takes the same decisions.
 *   - Layouts: rays SoA [3][R]; node positions [3][N]; node dual quaternions [8][N] as
 *     (real w,x,y,z ; dual w,x,y,z); hash tables [L][T][F]; MLP weights W1..W5 row-major
 *     [out][in], concatenated.
 *   - Parity pins: see the header of oracle.py and the tests named there.  Every function
 *     below is pinned by at least one test except where its comment says otherwise.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_L 32
#define ORC_MAX_F 8
#define ORC_MAX_K 16
#define ORC_MAX_W 256   /* widest MLP layer */
#define ORC_OCC_RES 128

/* ----------------------------------------------------------------------- descriptions */
typedef struct {
    int L, log2_T, F, N_min;
    double growth;
    int mlp_in, hidden, geo_out, col_hidden;
    const double* tables;   /* [L][T][F] */
    const double* weights;  /* W1[hidden][in] W2[hidden][hidden] W3[geo][hidden]
                               W4[col_hidden][geo-1] W5[3][col_hidden] */
} orc_field;

typedef struct {
    int n_nodes, K;
    double radius;          /* influence radius r of Eq. 2 (0.1 in the paper) */
    const float* x_live;    /* deformed node positions x_i^t = dq_i^t x_i, [3][N] */
    const float* dq;        /* node motions dq_i^t, [8][N] */
    /* look-up-table neighbour search (Sec. 4.2, "On-the-fly Radiance Fields"); unused
     * when lut_live is NULL */
    int lut_res;                /* G: G^3 voxels over [-1,1]^3 in both spaces */
    const uint16_t* lut_canon;  /* [G^3][K] canonical KNN field */
    const uint32_t* lut_live;   /* [G^3] live voxel -> canonical voxel, ORC_LUT_EMPTY = none */
} orc_graph;

#define ORC_LUT_EMPTY 0xFFFFFFFFu

/* Pose-conditioned deformation net (Sec. 4.2 Eq. 4 and the text after it; sizes from
 * Sec. 4.4): its own hash encoding of the warped point (L levels x F features, 32 in the
 * paper) concatenated with the pose (72), n_hidden ReLU layers of width `hidden` (4 x 128),
 * a linear output of the residual displacement (3); no biases. */
typedef struct orc_deform_s {
    int L, log2_T, F, N_min;
    double growth;
    int pose_dim, hidden, n_hidden;
    const double* tables;   /* [L][T][F] */
    const double* weights;  /* W_1 [hidden][L*F + pose_dim], W_2..W_n [hidden][hidden], W_out [3][hidden] */
} orc_deform;

typedef struct {
    const orc_field* field;
    const orc_graph* graph;     /* NULL: rigid (object) field */
    const float* rigid_dq;      /* [8] canonical -> live pose T^t, used when graph == NULL */
    const uint32_t* occupancy;  /* live-space 128^3 bitfield, or NULL for none */
    const struct orc_deform_s* deform;  /* pose-conditioned deformation net, or NULL */
    const float* pose;          /* [pose_dim] pose theta^t of this view's frame */
} orc_view;

typedef struct {
    int64_t n_rays;
    const float* o;             /* [3][R] */
    const float* d;             /* [3][R] */
    const orc_view* view;
    const float* target;        /* [3][R] */
    double* grad_tables;        /* accumulates dLoss/dtables of view->field */
    double* grad_weights;       /* accumulates dLoss/dweights of view->field */
    const float* mask;          /* [R] M(r) of the paper's losses, NULL = 1 */
    const float* depth;         /* [R] sensor depth D(r) of the paper's depth loss */
    double* grad_deform_tables;   /* accumulates dLoss/d(deformation-net tables), if any */
    double* grad_deform_weights;  /* accumulates dLoss/d(deformation-net weights), if any */
} orc_batch;

/* ---------------------------------------------------------------- hash-grid geometry */
/* Level resolution N_l = floor(N_min * b^l) (multiresolution hash encoding of
 * Instant-NGP, which Sec. 4.2 adopts for H^h and H^o). */
int orc_level_res(int N_min, double growth, int l)
{
    return (int)floor((double)N_min * pow(growth, (double)l));
}

/* A level is stored densely when its (N_l+1)^3 vertices fit the table of T entries. */
int orc_level_dense(int res, int log2_T)
{
    int64_t v = (int64_t)(res + 1);
    return v * v * v <= ((int64_t)1 << log2_T);
}

/* Table slot of integer vertex (x,y,z) on a level of resolution res: dense row-major
 * x + y(N+1) + z(N+1)^2, else the spatial hash (x*1 ^ y*2654435761 ^ z*805459861) mod T
 * with 32-bit wrap-around. */
uint32_t orc_vertex_index(int res, int log2_T, uint32_t x, uint32_t y, uint32_t z)
{
    uint32_t T = 1u << log2_T;
    if (orc_level_dense(res, log2_T)) {
        uint32_t n = (uint32_t)res + 1u;
        return x + y * n + z * n * n;
    }
    uint32_t h = (x * 1u) ^ (y * 2654435761u) ^ (z * 805459861u);
    return h & (T - 1u);
}

/* Cell of one coordinate on a level (FP32 decision): u = (x+1)/2 clamped to [0,1],
 * q = u N_l, c = min(floor(q), N_l - 1). */
static int orc_level_cell(double x, int res)
{
    float u = ((float)x + 1.0f) * 0.5f;
    u = u < 0.0f ? 0.0f : (u > 1.0f ? 1.0f : u);
    float q = u * (float)res;
    int c = (int)floorf(q);
    return c > res - 1 ? res - 1 : c;
}

/* ------------------------------------------------------------------- ray sampling */
/* Slab intersection of the ray with the box [-1,1]^3 (FP32 decision).  Returns 0 on a
 * miss; otherwise t_n = max(0, t_near), t_f = t_far and the uniform step
 * dt = (t_f - t_n) / n_samples. */
int orc_ray_setup(const float o[3], const float d[3], int n_samples, float* t_n, float* dt)
{
    float tnear = -INFINITY, tfar = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0f) {
            if (o[a] < -1.0f || o[a] > 1.0f) return 0;
            continue;
        }
        float t0 = (-1.0f - o[a]) / d[a];
        float t1 = (1.0f - o[a]) / d[a];
        float lo = t0 < t1 ? t0 : t1;
        float hi = t0 < t1 ? t1 : t0;
        if (lo > tnear) tnear = lo;
        if (hi < tfar) tfar = hi;
    }
    float tn = tnear > 0.0f ? tnear : 0.0f;
    if (!(tfar > tn)) return 0;
    *t_n = tn;
    *dt = (tfar - tn) / (float)n_samples;
    return 1;
}

/* Midpoint sample j: t_j = t_n + (j + 1/2) dt, p_j = o + t_j d (FP32, no fused ops). */
void orc_sample(const float o[3], const float d[3], float t_n, float dt, int j, float* t, float p[3])
{
    float tj = t_n + ((float)j + 0.5f) * dt;
    for (int a = 0; a < 3; ++a) {
        float s = tj * d[a];
        p[a] = o[a] + s;
    }
    *t = tj;
}

/* Occupancy bit of the 128^3 live-space cell holding p (FP32 decision). */
int orc_occupied(const uint32_t* bits, const float p[3])
{
    int c[3];
    for (int a = 0; a < 3; ++a) {
        float q = (p[a] + 1.0f) * 0.5f * (float)ORC_OCC_RES;
        int i = (int)floorf(q);
        c[a] = i < 0 ? 0 : (i > ORC_OCC_RES - 1 ? ORC_OCC_RES - 1 : i);
    }
    uint32_t idx = (uint32_t)c[0] + ORC_OCC_RES * ((uint32_t)c[1] + ORC_OCC_RES * (uint32_t)c[2]);
    return (int)((bits[idx >> 5] >> (idx & 31u)) & 1u);
}

/* --------------------------------------------------------------- dual quaternions */
static void quat_mul(const double a[4], const double b[4], double out[4])
{
    /* Hamilton product, (w, x, y, z) */
    double w = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    double x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    double y = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    double z = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    out[0] = w; out[1] = x; out[2] = y; out[3] = z;
}

/* Rotation R and translation t of a unit dual quaternion: R = R(q_r),
 * t = 2 vec(q_d q_r^*). */
static void dq_to_rt(const double qr[4], const double qd[4], double R[9], double t[3])
{
    double w = qr[0], x = qr[1], y = qr[2], z = qr[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
    double conj[4] = {qr[0], -qr[1], -qr[2], -qr[3]};
    double m[4];
    quat_mul(qd, conj, m);
    t[0] = 2.0 * m[1]; t[1] = 2.0 * m[2]; t[2] = 2.0 * m[3];
}

/* Normalise a blended dual quaternion b = (b_r, b_d): q_r = b_r/|b_r|,
 * q_d = b_d/|b_r| - (q_r . b_d/|b_r|) q_r, so that |q_r| = 1 and q_r . q_d = 0. */
void orc_dq_normalize(const double b[8], double qr[4], double qd[4])
{
    double n = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2] + b[3] * b[3]);
    double dn[4], dot = 0.0;
    for (int k = 0; k < 4; ++k) {
        qr[k] = b[k] / n;
        dn[k] = b[4 + k] / n;
    }
    for (int k = 0; k < 4; ++k) dot += qr[k] * dn[k];
    for (int k = 0; k < 4; ++k) qd[k] = dn[k] - dot * qr[k];
}

/* SE3(dq) p = R p + t (forward motion of Eq. 2; used for x_i^t = dq_i^t x_i). */
void orc_dq_apply(const double qr[4], const double qd[4], const double p[3], double out[3])
{
    double R[9], t[3];
    dq_to_rt(qr, qd, R, t);
    for (int a = 0; a < 3; ++a)
        out[a] = R[3 * a + 0] * p[0] + R[3 * a + 1] * p[1] + R[3 * a + 2] * p[2] + t[a];
}

/* SE3(dq)^{-1} p = R^T (p - t) (the inverse warp of Eq. 4). */
void orc_dq_apply_inverse(const double qr[4], const double qd[4], const double p[3], double out[3])
{
    double R[9], t[3], q[3];
    dq_to_rt(qr, qd, R, t);
    for (int a = 0; a < 3; ++a) q[a] = p[a] - t[a];
    for (int a = 0; a < 3; ++a)
        out[a] = R[0 * 3 + a] * q[0] + R[1 * 3 + a] * q[1] + R[2 * 3 + a] * q[2];
}

/* --------------------------------------------------------------- nearest nodes */
/* The K deformed nodes nearest to p, by brute force over all N nodes.  Selection key
 * (FP32 decision): ((dx*dx)+(dy*dy))+(dz*dz) with d = p - x_i^t; ties go to the lower
 * node index.  Output sorted ascending by (key, index). */
void orc_knn(const orc_graph* g, const float p[3], int* ids, float* keys)
{
    int N = g->n_nodes, K = g->K;
    for (int k = 0; k < K; ++k) { keys[k] = INFINITY; ids[k] = -1; }
    for (int i = 0; i < N; ++i) {
        float dx = p[0] - g->x_live[0 * N + i];
        float dy = p[1] - g->x_live[1 * N + i];
        float dz = p[2] - g->x_live[2 * N + i];
        float key = ((dx * dx) + (dy * dy)) + (dz * dz);
        if (!(key < keys[K - 1])) continue;
        int pos = K - 1;
        while (pos > 0 && keys[pos - 1] > key) {
            keys[pos] = keys[pos - 1];
            ids[pos] = ids[pos - 1];
            --pos;
        }
        keys[pos] = key;
        ids[pos] = i;
    }
}

/* ---------------------------------------- look-up-table neighbour search (Sec. 4.2) */
/* The paper replaces the O(N) neighbour query by tables: a canonical KNN field of G^3
 * voxels (G = 512 there) holding each voxel's K nearest canonical nodes, built once; per
 * frame every canonical voxel centre is carried to live space by the forward warp of
 * Eq. 2 (its own K nodes blended) and its index is stored in the live voxel it lands in;
 * a sample then reads its live voxel, the canonical voxel stored there, and that voxel's
 * K nodes, and blends them as in Eq. 4.
 *
 * Readings where the paper is silent: several canonical voxels landing in one live voxel
 * leave the smallest canonical index; canonical voxels carried outside [-1,1]^3 are
 * dropped; a sample whose live voxel received none (a hole) uses the exact K nearest
 * deformed nodes.  The integer results (voxel of a point, KNN ids, live voxel of a warped
 * centre) are decided in single precision by the recipes below, so that any
 * implementation performing the same rounded operations builds identical tables; the
 * exponential of the blend weights is computed by Cody-Waite range reduction
 * (x = n ln2 + r, ln2 split in a short high part and a low part, |r| <= ln2/2) and the
 * degree-6 Taylor polynomial of e^r by Horner's rule, scaled by 2^n, for x <= 0; it is 0
 * where n < -125 (x below about -86.6), a weight negligible next to the nearest node's 1. */
static float orc_lut_exp(float x)
{
    float n = rintf(x * 1.44269504f);
    if (n < -125.0f) return 0.0f;
    float r = (x - n * 0.693145752f) - n * 1.42860682e-06f;
    float p = 1.38888889e-03f;    /* 1/6! ... 1/3!: decimal literals, no constant folding */
    p = p * r + 8.33333333e-03f;
    p = p * r + 4.16666667e-02f;
    p = p * r + 1.66666667e-01f;
    p = p * r + 0.5f;
    p = p * r + 1.0f;
    p = p * r + 1.0f;
    union { uint32_t u; float f; } scale;
    scale.u = (uint32_t)((int)n + 127) << 23;
    return p * scale.f;
}

/* Centre of voxel i of G along one axis: (i + 1/2) (2/G) - 1 (exact for G a power of 2). */
static float orc_lut_centre(int i, int G)
{
    return ((float)i + 0.5f) * (2.0f / (float)G) - 1.0f;
}

/* Voxel of one coordinate: floor(((x + 1) * 0.5) * G); -1 when outside [0, G). */
static int orc_lut_cell(float x, int G)
{
    float q = ((x + 1.0f) * 0.5f) * (float)G;
    float f = floorf(q);
    return (f >= 0.0f && f < (float)G) ? (int)f : -1;
}

/* Canonical KNN field: for every voxel centre the K nearest canonical nodes x_i, same key
 * and tie rule as orc_knn, ids ascending by (key, id).  out [G^3][K], voxel x + G(y + G z). */
void orc_lut_canon_knn(int n_nodes, int K, const float* x_canon, int G, uint16_t* out)
{
    orc_graph cg = {n_nodes, K, 0.0, x_canon, NULL, 0, NULL, NULL};
    int64_t n = (int64_t)G * G * G;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; ++v) {
        float c[3] = {orc_lut_centre((int)(v % G), G), orc_lut_centre((int)((v / G) % G), G),
                      orc_lut_centre((int)(v / ((int64_t)G * G)), G)};
        int ids[ORC_MAX_K];
        float keys[ORC_MAX_K];
        orc_knn(&cg, c, ids, keys);
        for (int k = 0; k < K; ++k) out[v * K + k] = (uint16_t)ids[k];
    }
}

/* Forward warp (Eq. 2) of canonical point c by the blend of its K canonical neighbours
 * ids (ascending by canonical key), single-precision recipe: weights
 * exp((key_0 - key_k) / r^2) with key_k = |c - x_k|^2 (the shift by the nearest key cancels
 * in the normalisation), sign alignment to the nearest node, blend, normalisation
 * q_r = b_r/|b_r|, q_d = b_d/|b_r| - (q_r.b_d/|b_r|) q_r, then R(q_r) c + t with
 * t = 2 vec(q_d q_r^*). */
static void orc_lut_forward(int N, int K, float radius, const float* x_canon, const float* dq, const int* ids,
                            const float c[3], float out[3])
{
    float keys[ORC_MAX_K];
    for (int k = 0; k < K; ++k) {
        float dx = c[0] - x_canon[0 * N + ids[k]];
        float dy = c[1] - x_canon[1 * N + ids[k]];
        float dz = c[2] - x_canon[2 * N + ids[k]];
        keys[k] = ((dx * dx) + (dy * dy)) + (dz * dz);
    }
    float inv_r2 = 1.0f / (radius * radius);
    float ref[4];
    for (int a = 0; a < 4; ++a) ref[a] = dq[a * N + ids[0]];
    float b[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < K; ++k) {
        const int i = ids[k];
        float w = orc_lut_exp((keys[0] - keys[k]) * inv_r2);
        float dot = (((dq[0 * N + i] * ref[0]) + (dq[1 * N + i] * ref[1])) + (dq[2 * N + i] * ref[2])) +
                    (dq[3 * N + i] * ref[3]);
        if (dot < 0.0f) w = -w;
        for (int a = 0; a < 8; ++a) b[a] = b[a] + w * dq[a * N + i];
    }
    float nr = sqrtf((((b[0] * b[0]) + (b[1] * b[1])) + (b[2] * b[2])) + (b[3] * b[3]));
    float qr[4], dn[4];
    for (int a = 0; a < 4; ++a) {
        qr[a] = b[a] / nr;
        dn[a] = b[4 + a] / nr;
    }
    float dot = (((qr[0] * dn[0]) + (qr[1] * dn[1])) + (qr[2] * dn[2])) + (qr[3] * dn[3]);
    float qd[4];
    for (int a = 0; a < 4; ++a) qd[a] = dn[a] - dot * qr[a];
    /* q_r = (w, u), q_d = (s, v): vec(q_d q_r^*) = w v - s u - v x u */
    float w = qr[0], u[3] = {qr[1], qr[2], qr[3]}, sd = qd[0], v[3] = {qd[1], qd[2], qd[3]};
    float vxu[3] = {(v[1] * u[2]) - (v[2] * u[1]), (v[2] * u[0]) - (v[0] * u[2]), (v[0] * u[1]) - (v[1] * u[0])};
    float t[3];
    for (int a = 0; a < 3; ++a) t[a] = 2.0f * (((w * v[a]) - (sd * u[a])) - vxu[a]);
    /* R(q_r) c = c + w tt + u x tt with tt = 2 (u x c) */
    float tt[3] = {2.0f * ((u[1] * c[2]) - (u[2] * c[1])), 2.0f * ((u[2] * c[0]) - (u[0] * c[2])),
                   2.0f * ((u[0] * c[1]) - (u[1] * c[0]))};
    float uxt[3] = {(u[1] * tt[2]) - (u[2] * tt[1]), (u[2] * tt[0]) - (u[0] * tt[2]),
                    (u[0] * tt[1]) - (u[1] * tt[0])};
    for (int a = 0; a < 3; ++a) out[a] = ((c[a] + (w * tt[a])) + uxt[a]) + t[a];
}

/* Live index field of one frame: every canonical voxel k, in increasing order, forward
 * warped (orc_lut_forward with its K canonical neighbours and the frame's motions dq) and
 * stored in the live voxel it lands in unless that voxel already holds a smaller index
 * (so each live voxel keeps the smallest k).  live [G^3]. */
void orc_lut_live_index(int n_nodes, int K, float radius, const float* x_canon, const float* dq, int G,
                        const uint16_t* canon, uint32_t* live)
{
    int64_t n = (int64_t)G * G * G;
    for (int64_t v = 0; v < n; ++v) live[v] = ORC_LUT_EMPTY;
    for (int64_t k = 0; k < n; ++k) {
        float c[3] = {orc_lut_centre((int)(k % G), G), orc_lut_centre((int)((k / G) % G), G),
                      orc_lut_centre((int)(k / ((int64_t)G * G)), G)};
        int ids[ORC_MAX_K];
        for (int j = 0; j < K; ++j) ids[j] = canon[k * K + j];
        float q[3];
        orc_lut_forward(n_nodes, K, radius, x_canon, dq, ids, c, q);
        int cx = orc_lut_cell(q[0], G), cy = orc_lut_cell(q[1], G), cz = orc_lut_cell(q[2], G);
        if (cx < 0 || cy < 0 || cz < 0) continue;
        int64_t f = cx + (int64_t)G * (cy + (int64_t)G * cz);
        if (live[f] == ORC_LUT_EMPTY) live[f] = (uint32_t)k;
    }
}

/* Neighbour set of a live point: with tables, the K nodes of the canonical voxel stored
 * in p's live voxel (p's voxel clamped into the grid), ordered by the same live key and
 * tie rule as orc_knn; without tables or in a hole, the exact K nearest (orc_knn).
 * Returns 1 when the tables supplied the set. */
int orc_neighbours(const orc_graph* g, const float p[3], int* ids, float* keys)
{
    if (!g->lut_live) {
        orc_knn(g, p, ids, keys);
        return 0;
    }
    int G = g->lut_res, N = g->n_nodes, K = g->K;
    int c[3];
    for (int a = 0; a < 3; ++a) {
        int i = (int)floorf(((p[a] + 1.0f) * 0.5f) * (float)G);
        c[a] = i < 0 ? 0 : (i > G - 1 ? G - 1 : i);
    }
    uint32_t k = g->lut_live[c[0] + (int64_t)G * (c[1] + (int64_t)G * c[2])];
    if (k == ORC_LUT_EMPTY) {
        orc_knn(g, p, ids, keys);
        return 0;
    }
    for (int j = 0; j < K; ++j) {
        keys[j] = INFINITY;
        ids[j] = -1;
    }
    for (int j = 0; j < K; ++j) {
        int i = g->lut_canon[(int64_t)k * K + j];
        float dx = p[0] - g->x_live[0 * N + i];
        float dy = p[1] - g->x_live[1 * N + i];
        float dz = p[2] - g->x_live[2 * N + i];
        float key = ((dx * dx) + (dy * dy)) + (dz * dz);
        int pos = K - 1;
        while (pos > 0 && (keys[pos - 1] > key || (keys[pos - 1] == key && ids[pos - 1] > i))) {
            keys[pos] = keys[pos - 1];
            ids[pos] = ids[pos - 1];
            --pos;
        }
        keys[pos] = key;
        ids[pos] = i;
    }
    return 1;
}

/* Dual-quaternion blend of the K nearest deformed nodes (Eq. 2 blending, applied with
 * the deformed nodes as in Eq. 4).  Weights w_i = exp(-|p - x_i^t|^2 / r^2), evaluated
 * shifted by the nearest node's squared distance (the common factor cancels in the
 * normalisation and the shift avoids underflow far from the nodes).  Each node's
 * quaternion is sign-aligned to the nearest node's real part before summing. */
void orc_blend(const orc_graph* g, const float p[3], double qr[4], double qd[4], int* ids_out)
{
    int ids[ORC_MAX_K];
    float keys[ORC_MAX_K];
    int N = g->n_nodes, K = g->K;
    orc_neighbours(g, p, ids, keys);
    double d2[ORC_MAX_K];
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a) {
            double diff = (double)p[a] - (double)g->x_live[a * N + ids[k]];
            s += diff * diff;
        }
        d2[k] = s;
    }
    double r2 = g->radius * g->radius;
    double ref[4];
    for (int c = 0; c < 4; ++c) ref[c] = g->dq[c * N + ids[0]];
    double b[8] = {0};
    for (int k = 0; k < K; ++k) {
        double w = exp(-(d2[k] - d2[0]) / r2);
        double dot = 0.0;
        for (int c = 0; c < 4; ++c) dot += (double)g->dq[c * N + ids[k]] * ref[c];
        double s = dot < 0.0 ? -1.0 : 1.0;
        for (int c = 0; c < 8; ++c) b[c] += s * w * (double)g->dq[c * N + ids[k]];
    }
    orc_dq_normalize(b, qr, qd);
    if (ids_out)
        for (int k = 0; k < K; ++k) ids_out[k] = ids[k];
}

/* Live -> canonical warp of one sample before the deformation net: Eq. 4 for the human
 * field (v^h_t), the inverse of the tracked rigid pose for the object field. */
static void orc_warp_vt(const orc_view* v, const float p[3], double vc[3])
{
    double qr[4], qd[4];
    if (v->graph) {
        orc_blend(v->graph, p, qr, qd, NULL);
    } else {
        double b[8];
        for (int c = 0; c < 8; ++c) b[c] = v->rigid_dq[c];
        orc_dq_normalize(b, qr, qd);
    }
    double pd[3] = {p[0], p[1], p[2]};
    orc_dq_apply_inverse(qr, qd, pd, vc);
}

/* ---------------------------------------------------------------- hash encoding */
/* Multiresolution hash encoding of canonical point x: per level, trilinear interpolation
 * of the F-vectors stored at the 8 corners of the cell holding x.  Output level-major
 * feat[l*F + f].  Optional outputs: the 8 table slots and weights per level (corner bit
 * 0 = +x, bit 1 = +y, bit 2 = +z). */
void orc_encode(const orc_field* fd, const double x[3], double* feat, uint32_t* idx_out, double* w_out)
{
    int L = fd->L, F = fd->F;
    int64_t T = (int64_t)1 << fd->log2_T;
    for (int l = 0; l < L; ++l) {
        int res = orc_level_res(fd->N_min, fd->growth, l);
        int c[3];
        double fr[3];
        for (int a = 0; a < 3; ++a) {
            c[a] = orc_level_cell(x[a], res);
            double u = (x[a] + 1.0) * 0.5;
            u = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
            fr[a] = u * (double)res - (double)c[a];
        }
        for (int f = 0; f < F; ++f) feat[l * F + f] = 0.0;
        for (int corner = 0; corner < 8; ++corner) {
            int bx = corner & 1, by = (corner >> 1) & 1, bz = (corner >> 2) & 1;
            double w = (bx ? fr[0] : 1.0 - fr[0]) * (by ? fr[1] : 1.0 - fr[1]) * (bz ? fr[2] : 1.0 - fr[2]);
            uint32_t idx = orc_vertex_index(res, fd->log2_T, (uint32_t)(c[0] + bx),
                                            (uint32_t)(c[1] + by), (uint32_t)(c[2] + bz));
            const double* e = fd->tables + ((int64_t)l * T + idx) * F;
            for (int f = 0; f < F; ++f) feat[l * F + f] += w * e[f];
            if (idx_out) idx_out[l * 8 + corner] = idx;
            if (w_out) w_out[l * 8 + corner] = w;
        }
    }
}

/* Derivative of the encoding with respect to the point: dx[a] = sum_l sum_f dfeat[l F + f]
 * d feat[l F + f] / d x_a.  Per level, d/dx_a of the trilinear weight of a corner is the
 * product of the other two axes' weights times +-1 (corner bit set / clear) times N_l / 2
 * (q = (x + 1)/2 N_l); an axis whose u = (x + 1)/2 lies outside [0, 1] is clamped and
 * contributes 0.  Parity pinned against the affine-table closed form and central
 * differences of orc_encode. */
void orc_encode_dx(const orc_field* fd, const double x[3], const double* dfeat, double dx[3])
{
    int L = fd->L, F = fd->F;
    int64_t T = (int64_t)1 << fd->log2_T;
    dx[0] = dx[1] = dx[2] = 0.0;
    for (int l = 0; l < L; ++l) {
        int res = orc_level_res(fd->N_min, fd->growth, l);
        int c[3];
        double fr[3], scale[3];
        for (int a = 0; a < 3; ++a) {
            c[a] = orc_level_cell(x[a], res);
            double u = (x[a] + 1.0) * 0.5;
            scale[a] = (u < 0.0 || u > 1.0) ? 0.0 : 0.5 * (double)res;
            u = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
            fr[a] = u * (double)res - (double)c[a];
        }
        for (int corner = 0; corner < 8; ++corner) {
            int b[3] = {corner & 1, (corner >> 1) & 1, (corner >> 2) & 1};
            double w1[3];
            for (int a = 0; a < 3; ++a) w1[a] = b[a] ? fr[a] : 1.0 - fr[a];
            uint32_t idx = orc_vertex_index(res, fd->log2_T, (uint32_t)(c[0] + b[0]), (uint32_t)(c[1] + b[1]),
                                            (uint32_t)(c[2] + b[2]));
            const double* e = fd->tables + ((int64_t)l * T + idx) * F;
            double g = 0.0;
            for (int f = 0; f < F; ++f) g += dfeat[l * F + f] * e[f];
            for (int a = 0; a < 3; ++a) {
                double dw = (b[a] ? 1.0 : -1.0) * scale[a];
                for (int o = 0; o < 3; ++o)
                    if (o != a) dw *= w1[o];
                dx[a] += dw * g;
            }
        }
    }
}

/* ------------------------------------------------------------ deformation net */
static void dense(const double* W, const double* x, int out, int in, double* y, int relu);

#define ORC_MAX_DIN 256
#define ORC_MAX_DW 256
#define ORC_MAX_DH 8

typedef struct {
    double vt[3];                  /* the point v^h_t the net reads */
    double x[ORC_MAX_DIN];         /* [hash features of v^h_t, pose] */
    double h[ORC_MAX_DH][ORC_MAX_DW];
    double dv[3];                  /* delta v^h */
} orc_dact;

static void orc_deform_field(const orc_deform* d, orc_field* fd)
{
    memset(fd, 0, sizeof(*fd));
    fd->L = d->L; fd->log2_T = d->log2_T; fd->F = d->F; fd->N_min = d->N_min; fd->growth = d->growth;
    fd->tables = d->tables;
}

/* delta v^h of the point vt under pose theta: encode vt with the net's own tables,
 * append the pose, ReLU layers, linear output. */
void orc_deform_forward(const orc_deform* d, const float* pose, const double vt[3], orc_dact* a)
{
    orc_field fd;
    orc_deform_field(d, &fd);
    int LF = d->L * d->F, in = LF + d->pose_dim, H = d->hidden;
    for (int k = 0; k < 3; ++k) a->vt[k] = vt[k];
    orc_encode(&fd, vt, a->x, NULL, NULL);
    for (int k = 0; k < d->pose_dim; ++k) a->x[LF + k] = pose[k];
    const double* W = d->weights;
    dense(W, a->x, H, in, a->h[0], 1);
    W += (int64_t)H * in;
    for (int k = 1; k < d->n_hidden; ++k) {
        dense(W, a->h[k - 1], H, H, a->h[k], 1);
        W += (int64_t)H * H;
    }
    dense(W, a->h[d->n_hidden - 1], 3, H, a->dv, 0);
}

/* Backward of the net for dL/d(delta v) = ddv: weight gradients added to dW (same layout
 * as the weights), dL/d(hash features) written to dfeat [L*F]. */
static void orc_deform_backward(const orc_deform* d, const orc_dact* a, const double ddv[3], double* dW,
                                double* dfeat)
{
    int LF = d->L * d->F, in = LF + d->pose_dim, H = d->hidden, n = d->n_hidden;
    int64_t off[ORC_MAX_DH + 1];
    off[0] = 0;
    off[1] = (int64_t)H * in;
    for (int k = 2; k <= n; ++k) off[k] = off[k - 1] + (int64_t)H * H;
    const double* W = d->weights;
    double g[ORC_MAX_DW], gp[ORC_MAX_DW];
    /* output layer */
    for (int o = 0; o < 3; ++o)
        for (int k = 0; k < H; ++k) dW[off[n] + o * H + k] += ddv[o] * a->h[n - 1][k];
    for (int k = 0; k < H; ++k) {
        double s = 0.0;
        for (int o = 0; o < 3; ++o) s += W[off[n] + o * H + k] * ddv[o];
        g[k] = a->h[n - 1][k] > 0.0 ? s : 0.0;
    }
    /* hidden layers n-1 .. 1: g = dL/d(pre-activation of layer k) */
    for (int k = n - 1; k >= 1; --k) {
        for (int o = 0; o < H; ++o)
            for (int i = 0; i < H; ++i) dW[off[k] + o * H + i] += g[o] * a->h[k - 1][i];
        for (int i = 0; i < H; ++i) {
            double s = 0.0;
            for (int o = 0; o < H; ++o) s += W[off[k] + o * H + i] * g[o];
            gp[i] = a->h[k - 1][i] > 0.0 ? s : 0.0;
        }
        for (int i = 0; i < H; ++i) g[i] = gp[i];
    }
    /* first layer */
    for (int o = 0; o < H; ++o)
        for (int i = 0; i < in; ++i) dW[o * in + i] += g[o] * a->x[i];
    for (int i = 0; i < LF; ++i) {
        double s = 0.0;
        for (int o = 0; o < H; ++o) s += W[o * in + i] * g[o];
        dfeat[i] = s;
    }
}

/* Live -> canonical warp of one sample: v^h_t by Eq. 4, then, with a deformation net,
 * v^h_c = v^h_t + delta v^h (Sec. 4.2); the object field's rigid inverse pose. */
void orc_warp(const orc_view* v, const float p[3], double vc[3])
{
    orc_warp_vt(v, p, vc);
    if (v->graph && v->deform) {
        orc_dact a;
        orc_deform_forward(v->deform, v->pose, vc, &a);
        for (int k = 0; k < 3; ++k) vc[k] += a.dv[k];
    }
}

/* ------------------------------------------------------------------------ MLPs */
typedef struct {
    double feat[ORC_MAX_L * ORC_MAX_F];
    double h1[ORC_MAX_W], h2[ORC_MAX_W], o[ORC_MAX_W], h4[ORC_MAX_W], z[3];
    double sigma, rgb[3];
} orc_act;

static void orc_weight_views(const orc_field* fd, const double* base, const double* W[5])
{
    int in = fd->mlp_in, h = fd->hidden, g = fd->geo_out, ch = fd->col_hidden;
    W[0] = base;
    W[1] = W[0] + (size_t)h * in;
    W[2] = W[1] + (size_t)h * h;
    W[3] = W[2] + (size_t)g * h;
    W[4] = W[3] + (size_t)ch * (g - 1);
}

static void dense(const double* W, const double* x, int out, int in, double* y, int relu)
{
    for (int i = 0; i < out; ++i) {
        double s = 0.0;
        for (int k = 0; k < in; ++k) s += W[(size_t)i * in + k] * x[k];
        y[i] = (relu && s < 0.0) ? 0.0 : s;
    }
}

/* Geometry MLP E_g: in -> hidden -> hidden -> geo_out (ReLU hidden, no biases), density
 * sigma = exp(o_0); colour MLP E_c: o_1..o_{geo_out-1} -> col_hidden (ReLU) -> 3,
 * sigmoid (Sec. 4.2, "geometry MLP" and "color MLP"). */
void orc_mlp_forward(const orc_field* fd, orc_act* a)
{
    const double* W[5];
    orc_weight_views(fd, fd->weights, W);
    dense(W[0], a->feat, fd->hidden, fd->mlp_in, a->h1, 1);
    dense(W[1], a->h1, fd->hidden, fd->hidden, a->h2, 1);
    dense(W[2], a->h2, fd->geo_out, fd->hidden, a->o, 0);
    dense(W[3], a->o + 1, fd->col_hidden, fd->geo_out - 1, a->h4, 1);
    dense(W[4], a->h4, 3, fd->col_hidden, a->z, 0);
    a->sigma = exp(a->o[0]);
    for (int c = 0; c < 3; ++c) a->rgb[c] = 1.0 / (1.0 + exp(-a->z[c]));
}

/* Reverse-mode pass through both MLPs.  Inputs: dL/dsigma and dL/drgb of one sample.
 * Accumulates dL/dW into dW (same layout as the weights) and writes dL/dfeat. */
static void orc_mlp_backward(const orc_field* fd, const orc_act* a, double dsigma, const double drgb[3],
                             double* dW, double* dfeat)
{
    const double* W[5];
    double* G[5];
    orc_weight_views(fd, fd->weights, W);
    orc_weight_views(fd, dW, (const double**)G);
    int in = fd->mlp_in, h = fd->hidden, g = fd->geo_out, ch = fd->col_hidden;
    double dz[3], dh4[ORC_MAX_W], dout[ORC_MAX_W], dh2[ORC_MAX_W], dh1[ORC_MAX_W];
    for (int c = 0; c < 3; ++c) dz[c] = drgb[c] * a->rgb[c] * (1.0 - a->rgb[c]);
    for (int c = 0; c < 3; ++c)
        for (int j = 0; j < ch; ++j) G[4][(size_t)c * ch + j] += dz[c] * a->h4[j];
    for (int j = 0; j < ch; ++j) {
        double s = 0.0;
        for (int c = 0; c < 3; ++c) s += W[4][(size_t)c * ch + j] * dz[c];
        dh4[j] = a->h4[j] > 0.0 ? s : 0.0;
    }
    for (int i = 0; i < ch; ++i)
        for (int j = 0; j < g - 1; ++j) G[3][(size_t)i * (g - 1) + j] += dh4[i] * a->o[1 + j];
    for (int j = 0; j < g - 1; ++j) {
        double s = 0.0;
        for (int i = 0; i < ch; ++i) s += W[3][(size_t)i * (g - 1) + j] * dh4[i];
        dout[1 + j] = s;
    }
    dout[0] = dsigma * a->sigma;
    for (int i = 0; i < g; ++i)
        for (int j = 0; j < h; ++j) G[2][(size_t)i * h + j] += dout[i] * a->h2[j];
    for (int j = 0; j < h; ++j) {
        double s = 0.0;
        for (int i = 0; i < g; ++i) s += W[2][(size_t)i * h + j] * dout[i];
        dh2[j] = a->h2[j] > 0.0 ? s : 0.0;
    }
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < h; ++j) G[1][(size_t)i * h + j] += dh2[i] * a->h1[j];
    for (int j = 0; j < h; ++j) {
        double s = 0.0;
        for (int i = 0; i < h; ++i) s += W[1][(size_t)i * h + j] * dh2[i];
        dh1[j] = a->h1[j] > 0.0 ? s : 0.0;
    }
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < in; ++j) G[0][(size_t)i * in + j] += dh1[i] * a->feat[j];
    for (int j = 0; j < in; ++j) {
        double s = 0.0;
        for (int i = 0; i < h; ++i) s += W[0][(size_t)i * in + j] * dh1[i];
        dfeat[j] = s;
    }
}

/* One sample through the field: warp -> encode -> MLPs. */
static void orc_eval_sample(const orc_view* v, const float p[3], orc_act* a, uint32_t* idx, double* w)
{
    double vc[3];
    orc_warp(v, p, vc);
    orc_encode(v->field, vc, a->feat, idx, w);
    orc_mlp_forward(v->field, a);
}

/* ------------------------------------------------------------------ compositing */
typedef struct {
    float t;          /* sample depth t_j */
    float p[3];       /* sample position */
    double sigma, rgb[3];
    double T;         /* transmittance before the sample */
    double alpha;
} orc_rec;

/* Front-to-back alpha compositing of one ray through one field (the volume rendering
 * shared by both fields, Sec. 3 and 4.2):
 *   alpha_j = 1 - exp(-sigma_j dt), T_{j+1} = T_j (1 - alpha_j),
 *   C = sum T_j alpha_j c_j, A = sum T_j alpha_j, D = sum T_j alpha_j t_j,
 * over the samples that the occupancy grid keeps (empty cells have sigma = 0), stopping
 * after the first sample with T_{j+1} < t_eps.  Returns the number of composited
 * samples and fills rec[] (if non-NULL) with them. */
static int orc_composite_ray(const orc_view* v, const float o[3], const float d[3], int n_samples,
                             double t_eps, double out[5], orc_rec* rec, double* T_end)
{
    float tn, dt;
    for (int c = 0; c < 5; ++c) out[c] = 0.0;
    if (T_end) *T_end = 1.0;
    if (!orc_ray_setup(o, d, n_samples, &tn, &dt)) return 0;
    double T = 1.0;
    int n = 0;
    orc_act a;
    for (int j = 0; j < n_samples; ++j) {
        float t, p[3];
        orc_sample(o, d, tn, dt, j, &t, p);
        if (v->occupancy && !orc_occupied(v->occupancy, p)) continue;
        orc_eval_sample(v, p, &a, NULL, NULL);
        double alpha = 1.0 - exp(-a.sigma * (double)dt);
        double w = T * alpha;
        for (int c = 0; c < 3; ++c) out[c] += w * a.rgb[c];
        out[3] += w;
        out[4] += w * (double)t;
        if (rec) {
            rec[n].t = t;
            rec[n].p[0] = p[0]; rec[n].p[1] = p[1]; rec[n].p[2] = p[2];
            rec[n].sigma = a.sigma;
            for (int c = 0; c < 3; ++c) rec[n].rgb[c] = a.rgb[c];
            rec[n].T = T;
            rec[n].alpha = alpha;
        }
        ++n;
        T = T * (1.0 - alpha);
        if (T < t_eps) break;
    }
    if (T_end) *T_end = T;
    return n;
}

/* Render n_rays rays through n_views fields.  Per view v: rgba_v[v][4][R] = (C, A) and
 * depth_v[v][R] = D, n_used[v][R] samples composited, T_end[v][R] final transmittance.
 * With two views (human = view 0, object = view 1) the nearer field, by expected depth
 * D/A (compared as D_h A_o <= D_o A_h, ties to the human), is laid over the farther:
 * C = C_n + (1 - A_n) C_f, A = A_n + (1 - A_n) A_f, D = D_n + (1 - A_n) D_f (Sec. 4.3,
 * "combine the RGB images according to the depth occlusion"). */
void orc_render(int64_t n_rays, const float* o, const float* d, int n_samples, double t_eps,
                int n_views, const orc_view* views, double* rgba_v, double* depth_v, int* n_used,
                double* T_end, double* rgba, double* depth)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < n_rays; ++r) {
        float ro[3] = {o[r], o[n_rays + r], o[2 * n_rays + r]};
        float rd[3] = {d[r], d[n_rays + r], d[2 * n_rays + r]};
        double res[2][5];
        for (int v = 0; v < n_views; ++v) {
            double te;
            int n = orc_composite_ray(&views[v], ro, rd, n_samples, t_eps, res[v], NULL, &te);
            for (int c = 0; c < 4; ++c) rgba_v[((int64_t)v * 4 + c) * n_rays + r] = res[v][c];
            depth_v[(int64_t)v * n_rays + r] = res[v][4];
            n_used[(int64_t)v * n_rays + r] = n;
            T_end[(int64_t)v * n_rays + r] = te;
        }
        double out[5];
        if (n_views == 1) {
            for (int c = 0; c < 5; ++c) out[c] = res[0][c];
        } else {
            int human_near = res[0][4] * res[1][3] <= res[1][4] * res[0][3];
            const double* nr = res[human_near ? 0 : 1];
            const double* fr = res[human_near ? 1 : 0];
            for (int c = 0; c < 5; ++c) out[c] = nr[c] + (1.0 - nr[3]) * fr[c];
        }
        for (int c = 0; c < 4; ++c) rgba[(int64_t)c * n_rays + r] = out[c];
        depth[r] = out[4];
    }
}

/* Joint per-sample compositing of the human field (view 0) and the object field (view 1)
 * along each ray, the alternative to laying one field's image over the other's: both
 * fields are sampled at the same t_j (same ray, same sample count), so at every sample the
 * densities add and the colours mix in proportion to density,
 *   sigma = sigma_h + sigma_o,  c = (sigma_h c_h + sigma_o c_o) / sigma,
 * a field whose occupancy bit is clear contributing sigma = 0 there, and the mixture is
 * composited front to back with early termination (T < t_eps) as for one field.
 * rgba[4][R], depth[R]; n_used[R] samples composited (samples where either field is occupied). */
void orc_render_joint(int64_t n_rays, const float* o, const float* d, int n_samples, double t_eps,
                      const orc_view* views, double* rgba, double* depth, int* n_used)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < n_rays; ++r) {
        float ro[3] = {o[r], o[n_rays + r], o[2 * n_rays + r]};
        float rd[3] = {d[r], d[n_rays + r], d[2 * n_rays + r]};
        double out[5] = {0, 0, 0, 0, 0};
        int n = 0;
        float tn, dt;
        if (orc_ray_setup(ro, rd, n_samples, &tn, &dt)) {
            double T = 1.0;
            for (int j = 0; j < n_samples; ++j) {
                float t, p[3];
                orc_sample(ro, rd, tn, dt, j, &t, p);
                double sig[2] = {0.0, 0.0}, col[2][3] = {{0, 0, 0}, {0, 0, 0}};
                int any = 0;
                for (int v = 0; v < 2; ++v) {
                    if (views[v].occupancy && !orc_occupied(views[v].occupancy, p)) continue;
                    orc_act a;
                    orc_eval_sample(&views[v], p, &a, NULL, NULL);
                    sig[v] = a.sigma;
                    for (int c = 0; c < 3; ++c) col[v][c] = a.rgb[c];
                    any = 1;
                }
                if (!any) continue;
                double sigma = sig[0] + sig[1];
                double alpha = 1.0 - exp(-sigma * (double)dt);
                double w = T * alpha;
                for (int c = 0; c < 3; ++c) {
                    double mix = sigma > 0.0 ? (sig[0] * col[0][c] + sig[1] * col[1][c]) / sigma : 0.0;
                    out[c] += w * mix;
                }
                out[3] += w;
                out[4] += w * (double)t;
                ++n;
                T = T * (1.0 - alpha);
                if (T < t_eps) break;
            }
        }
        for (int c = 0; c < 4; ++c) rgba[(int64_t)c * n_rays + r] = out[c];
        depth[r] = out[4];
        n_used[r] = n;
    }
}

/* ---------------------------------------------------------------- occupancy grid */
/* Density-driven maintenance of a view's 128^3 live-space occupancy bitfield (the given
 * bitfield of the hot path, kept up to date per frame): the density at every cell centre
 * ((i + 1/2) 2/128 - 1 per axis, FP32 recipe) is evaluated through the view's warp, encoding
 * and MLPs; density[c] = max(decay * density[c], sigma); the bit of cell c (index
 * x + 128 (y + 128 z), bit c & 31 of word c >> 5) is set iff density[c] > threshold. */
void orc_occupancy_update(const orc_view* v, double decay, double threshold, double* density, uint32_t* bits)
{
    const int G = ORC_OCC_RES;
    const int64_t n = (int64_t)G * G * G;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
        float p[3];
        int64_t ijk[3] = {c % G, (c / G) % G, c / ((int64_t)G * G)};
        for (int a = 0; a < 3; ++a) p[a] = ((float)ijk[a] + 0.5f) * (2.0f / (float)G) - 1.0f;
        orc_act act;
        orc_eval_sample(v, p, &act, NULL, NULL);
        double dn = decay * density[c];
        density[c] = dn > act.sigma ? dn : act.sigma;
    }
    for (int64_t w = 0; w < n / 32; ++w) {
        uint32_t m = 0;
        for (int b = 0; b < 32; ++b)
            if (density[w * 32 + b] > threshold) m |= 1u << b;
        bits[w] = m;
    }
}

/* ------------------------------------------------------------------ loss + gradient */
/* Huber penalty with threshold delta and its derivative. */
double orc_huber(double x, double delta)
{
    double ax = fabs(x);
    return ax <= delta ? 0.5 * x * x : delta * (ax - 0.5 * delta);
}

static double orc_huber_grad(double x, double delta)
{
    if (fabs(x) <= delta) return x;
    return x > 0.0 ? delta : -delta;
}

static void add_atomic(double* p, double v)
{
#pragma omp atomic
    *p += v;
}

/* Loss = mean over all rays of all batches and the 3 channels of Huber(C - target),
 * and (if grads != 0) its gradient with respect to every hash-table entry and MLP
 * weight, accumulated into each batch's grad_tables / grad_weights.
 *
 * Gradient of the compositing (per ray, samples k <= n that were composited):
 *   dC/dc_j     = T_j alpha_j
 *   dC/dsigma_j = dt (T_{j+1} c_j - (C - sum_{k<=j} T_k alpha_k c_k)),
 * then sigma = exp(o_0), c = sigmoid(z), the MLP chain rule, and the trilinear weights
 * scatter dL/dfeat into the 8 corner entries of every level. */
/* Per-ray loss and its derivatives dl/dC (3) and dl/dD of the rendered colour C and depth D.
 * Huber (kind 0): sum over the 3 channels of the Huber penalty of C - target, scaled by
 * `norm`.  The paper's losses (kind 1, Sec. 4.4 Implementation Details): the colour term
 * ||M (C_hat - C)||_2, the Euclidean norm of the masked colour error (its gradient is taken
 * as 0 where the error is exactly 0), plus depth_weight times the depth term
 * |M (D_hat - D)|, the L1 norm of the masked depth error (sign(0) = 0); summed over rays. */
static double orc_ray_loss(int kind, const orc_batch* B, int64_t r, const double out[5], double huber_delta,
                           double norm, double depth_weight, double dC[3], double* dD)
{
    int64_t R = B->n_rays;
    double e[3];
    for (int c = 0; c < 3; ++c) e[c] = out[c] - (double)B->target[(int64_t)c * R + r];
    *dD = 0.0;
    if (kind == 0) {
        double l = 0.0;
        for (int c = 0; c < 3; ++c) {
            l += orc_huber(e[c], huber_delta);
            dC[c] = orc_huber_grad(e[c], huber_delta) * norm;
        }
        return l;
    }
    double M = B->mask ? (double)B->mask[r] : 1.0;
    double n = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    for (int c = 0; c < 3; ++c) dC[c] = n > 0.0 ? M * e[c] / n : 0.0;
    double ed = out[4] - (double)B->depth[r];
    double sgn = ed > 0.0 ? 1.0 : (ed < 0.0 ? -1.0 : 0.0);
    *dD = depth_weight * M * sgn;
    return M * n + depth_weight * M * fabs(ed);
}

double orc_train_loss_grad(int n_batches, const orc_batch* batches, int n_samples, double t_eps,
                           double huber_delta, int grads, int loss_kind, double depth_weight)
{
    int64_t total = 0;
    for (int b = 0; b < n_batches; ++b) total += batches[b].n_rays;
    /* Huber: mean over rays and channels; the paper's losses: sum over rays */
    double norm = loss_kind == 0 ? 1.0 / (3.0 * (double)total) : 1.0;
    double loss = 0.0;
    for (int b = 0; b < n_batches; ++b) {
        const orc_batch* B = &batches[b];
        const orc_view* v = B->view;
        const orc_field* fd = v->field;
        int64_t R = B->n_rays;
        int64_t T = (int64_t)1 << fd->log2_T;
        int nw = fd->hidden * fd->mlp_in + fd->hidden * fd->hidden + fd->geo_out * fd->hidden +
                 fd->col_hidden * (fd->geo_out - 1) + 3 * fd->col_hidden;
        const orc_deform* def = v->graph ? v->deform : NULL;
        int nwd = 0;
        orc_field dfd;
        int64_t Td = 0;
        if (def) {
            nwd = def->hidden * (def->L * def->F + def->pose_dim) + (def->n_hidden - 1) * def->hidden * def->hidden +
                  3 * def->hidden;
            orc_deform_field(def, &dfd);
            Td = (int64_t)1 << def->log2_T;
        }
        double bl = 0.0;
#pragma omp parallel reduction(+ : bl)
        {
            orc_rec* rec = (orc_rec*)malloc(sizeof(orc_rec) * (size_t)n_samples);
            double* dW = grads ? (double*)calloc((size_t)nw, sizeof(double)) : NULL;
            double* dWd = (grads && def) ? (double*)calloc((size_t)nwd, sizeof(double)) : NULL;
#pragma omp for schedule(dynamic, 16)
            for (int64_t r = 0; r < R; ++r) {
                float ro[3] = {B->o[r], B->o[R + r], B->o[2 * R + r]};
                float rd[3] = {B->d[r], B->d[R + r], B->d[2 * R + r]};
                double out[5];
                int n = orc_composite_ray(v, ro, rd, n_samples, t_eps, out, rec, NULL);
                double dC[3], dD;
                bl += orc_ray_loss(loss_kind, B, r, out, huber_delta, norm, depth_weight, dC, &dD);
                if (!grads) continue;
                float tn, dt;
                if (!orc_ray_setup(ro, rd, n_samples, &tn, &dt)) continue;
                double prefix[3] = {0.0, 0.0, 0.0}, prefix_d = 0.0;
                for (int k = 0; k < n; ++k) {
                    const orc_rec* s = &rec[k];
                    double w = s->T * s->alpha;
                    double T_next = s->T * (1.0 - s->alpha);
                    double dsigma = 0.0, drgb[3];
                    for (int c = 0; c < 3; ++c) {
                        prefix[c] += w * s->rgb[c];
                        double rest = out[c] - prefix[c];
                        dsigma += dC[c] * (double)dt * (T_next * s->rgb[c] - rest);
                        drgb[c] = dC[c] * w;
                    }
                    /* depth D = sum T_j alpha_j t_j: the same adjoint with c_j -> t_j */
                    prefix_d += w * (double)s->t;
                    dsigma += dD * (double)dt * (T_next * (double)s->t - (out[4] - prefix_d));
                    orc_act a;
                    uint32_t idx[ORC_MAX_L * 8];
                    double cw[ORC_MAX_L * 8], dfeat[ORC_MAX_L * ORC_MAX_F];
                    orc_eval_sample(v, s->p, &a, idx, cw);
                    orc_mlp_backward(fd, &a, dsigma, drgb, dW, dfeat);
                    for (int l = 0; l < fd->L; ++l)
                        for (int corner = 0; corner < 8; ++corner) {
                            double wc = cw[l * 8 + corner];
                            double* gp = B->grad_tables + ((int64_t)l * T + idx[l * 8 + corner]) * fd->F;
                            for (int f = 0; f < fd->F; ++f) add_atomic(&gp[f], wc * dfeat[l * fd->F + f]);
                        }
                    if (def) {
                        /* v_c = v_t + delta v: dL/d(delta v) = dL/dv_c, the encoding's
                         * derivative in the point; then back through the net and into
                         * its tables at v_t */
                        double vt[3], vcn[3], dx[3], dfd_feat[ORC_MAX_DIN];
                        orc_dact da;
                        orc_warp_vt(v, s->p, vt);
                        orc_deform_forward(def, v->pose, vt, &da);
                        for (int k = 0; k < 3; ++k) vcn[k] = vt[k] + da.dv[k];
                        orc_encode_dx(fd, vcn, dfeat, dx);
                        orc_deform_backward(def, &da, dx, dWd, dfd_feat);
                        uint32_t didx[ORC_MAX_L * 8];
                        double dcw[ORC_MAX_L * 8], dfe[ORC_MAX_L * ORC_MAX_F];
                        orc_encode(&dfd, vt, dfe, didx, dcw);
                        for (int l = 0; l < def->L; ++l)
                            for (int corner = 0; corner < 8; ++corner) {
                                double wc = dcw[l * 8 + corner];
                                double* gp = B->grad_deform_tables + ((int64_t)l * Td + didx[l * 8 + corner]) * def->F;
                                for (int f = 0; f < def->F; ++f) add_atomic(&gp[f], wc * dfd_feat[l * def->F + f]);
                            }
                    }
                }
            }
            if (grads)
                for (int i = 0; i < nw; ++i) add_atomic(&B->grad_weights[i], dW[i]);
            if (dWd)
                for (int i = 0; i < nwd; ++i) add_atomic(&B->grad_deform_weights[i], dWd[i]);
            free(dWd);
            free(dW);
            free(rec);
        }
        loss += bl;
    }
    return loss * norm;
}

/* Adam (bias-corrected) on n parameters at step `step` (1-based):
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, p -= lr m_hat / (sqrt(v_hat) + eps). */
void orc_adam(int64_t n, double* p, const double* g, double* m, double* v, int64_t step, double lr,
              double b1, double b2, double eps)
{
    double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* ------------------------------------------------------------ per-point entry points */
/* Samples of R rays: hit[R], t_n[R], dt[R], t[R][S], p[3][R][S] (FP32 recipe). */
void orc_ray_samples(int64_t n_rays, const float* o, const float* d, int n_samples, int* hit, float* t_n,
                     float* dt, float* t, float* p)
{
    int64_t RS = n_rays * n_samples;
    for (int64_t r = 0; r < n_rays; ++r) {
        float ro[3] = {o[r], o[n_rays + r], o[2 * n_rays + r]};
        float rd[3] = {d[r], d[n_rays + r], d[2 * n_rays + r]};
        float tn = 0.0f, step = 0.0f;
        hit[r] = orc_ray_setup(ro, rd, n_samples, &tn, &step);
        t_n[r] = tn;
        dt[r] = step;
        for (int j = 0; j < n_samples; ++j) {
            float tj = 0.0f, pj[3] = {0.0f, 0.0f, 0.0f};
            if (hit[r]) orc_sample(ro, rd, tn, step, j, &tj, pj);
            t[r * n_samples + j] = tj;
            for (int a = 0; a < 3; ++a) p[a * RS + r * n_samples + j] = pj[a];
        }
    }
}

/* Occupancy bits of n points p[3][n]. */
void orc_occupied_points(const uint32_t* bits, int64_t n, const float* p, int* out)
{
    for (int64_t i = 0; i < n; ++i) {
        float q[3] = {p[i], p[n + i], p[2 * n + i]};
        out[i] = orc_occupied(bits, q);
    }
}

/* Nearest-node ids/keys [K][n] of n points p[3][n]. */
void orc_knn_points(const orc_graph* g, int64_t n, const float* p, int* ids, float* keys)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        float q[3] = {p[i], p[n + i], p[2 * n + i]};
        int id[ORC_MAX_K];
        float ky[ORC_MAX_K];
        orc_knn(g, q, id, ky);
        for (int k = 0; k < g->K; ++k) {
            ids[(int64_t)k * n + i] = id[k];
            keys[(int64_t)k * n + i] = ky[k];
        }
    }
}

/* Neighbour sets of n points p[3][n] (orc_neighbours): ids [K][n]; from_lut[n] = 1 where the
 * tables supplied the set, 0 where the exact search did. */
void orc_neighbour_points(const orc_graph* g, int64_t n, const float* p, int* ids, int* from_lut)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        float q[3] = {p[i], p[n + i], p[2 * n + i]};
        int id[ORC_MAX_K];
        float ky[ORC_MAX_K];
        from_lut[i] = orc_neighbours(g, q, id, ky);
        for (int k = 0; k < g->K; ++k) ids[(int64_t)k * n + i] = id[k];
    }
}

/* delta v of n points vt[3][n] under pose: dv[3][n] (deformation net forward). */
void orc_deform_points(const orc_deform* d, const float* pose, int64_t n, const double* vt, double* dv)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double q[3] = {vt[i], vt[n + i], vt[2 * n + i]};
        orc_dact a;
        orc_deform_forward(d, pose, q, &a);
        for (int k = 0; k < 3; ++k) dv[k * n + i] = a.dv[k];
    }
}

/* Encoding derivative of n points x[3][n] for dfeat [L*F][n]: dx[3][n]. */
void orc_encode_dx_points(const orc_field* fd, int64_t n, const double* x, const double* dfeat, double* dx)
{
    int LF = fd->L * fd->F;
    for (int64_t i = 0; i < n; ++i) {
        double q[3] = {x[i], x[n + i], x[2 * n + i]}, g[ORC_MAX_L * ORC_MAX_F], r[3];
        for (int k = 0; k < LF; ++k) g[k] = dfeat[(int64_t)k * n + i];
        orc_encode_dx(fd, q, g, r);
        for (int a = 0; a < 3; ++a) dx[a * n + i] = r[a];
    }
}

/* The table exponential of n arguments (for its error-bound pin). */
void orc_lut_exp_points(int64_t n, const float* x, float* out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_lut_exp(x[i]);
}

/* Forward warp (single-precision recipe) of n canonical points c[3][n] with neighbour ids
 * [n][K] (ascending by canonical key): out[3][n]. */
void orc_lut_forward_points(int n_nodes, int K, float radius, const float* x_canon, const float* dq, int64_t n,
                            const float* c, const int* ids, float* out)
{
    for (int64_t i = 0; i < n; ++i) {
        float q[3] = {c[i], c[n + i], c[2 * n + i]}, r[3];
        orc_lut_forward(n_nodes, K, radius, x_canon, dq, ids + i * K, q, r);
        for (int a = 0; a < 3; ++a) out[a * n + i] = r[a];
    }
}

/* Warp n points p[3][n] to canonical vc[3][n]; optionally the blended, normalised dual
 * quaternion qb[8][n] (human field only; identity for the rigid field). */
void orc_warp_points(const orc_view* v, int64_t n, const float* p, double* vc, double* qb)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        float q[3] = {p[i], p[n + i], p[2 * n + i]};
        double out[3];
        orc_warp(v, q, out);
        for (int a = 0; a < 3; ++a) vc[(int64_t)a * n + i] = out[a];
        if (qb) {
            double qr[4] = {1, 0, 0, 0}, qd[4] = {0, 0, 0, 0};
            if (v->graph) orc_blend(v->graph, q, qr, qd, NULL);
            for (int c = 0; c < 4; ++c) {
                qb[(int64_t)c * n + i] = qr[c];
                qb[(int64_t)(4 + c) * n + i] = qd[c];
            }
        }
    }
}

/* Forward motion of n points by one unit dual quaternion dq[8]: out = R p + t. */
void orc_dq_apply_points(const double* dq, int64_t n, const double* p, double* out)
{
    double b[8], qr[4], qd[4];
    for (int c = 0; c < 8; ++c) b[c] = dq[c];
    orc_dq_normalize(b, qr, qd);
    for (int64_t i = 0; i < n; ++i) {
        double q[3] = {p[i], p[n + i], p[2 * n + i]}, r[3];
        orc_dq_apply(qr, qd, q, r);
        for (int a = 0; a < 3; ++a) out[(int64_t)a * n + i] = r[a];
    }
}

/* Hash-encode n canonical points x[3][n]: feat[L*F][n]; optional idx[L*8][n], w[L*8][n]. */
void orc_encode_points(const orc_field* fd, int64_t n, const double* x, double* feat, uint32_t* idx, double* w)
{
    int LF = fd->L * fd->F, L8 = fd->L * 8;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double q[3] = {x[i], x[n + i], x[2 * n + i]};
        double f[ORC_MAX_L * ORC_MAX_F], ww[ORC_MAX_L * 8];
        uint32_t id[ORC_MAX_L * 8];
        orc_encode(fd, q, f, id, ww);
        for (int k = 0; k < LF; ++k) feat[(int64_t)k * n + i] = f[k];
        for (int k = 0; k < L8; ++k) {
            if (idx) idx[(int64_t)k * n + i] = id[k];
            if (w) w[(int64_t)k * n + i] = ww[k];
        }
    }
}

/* MLPs on n feature vectors feat[in][n]: out[4][n] = (sigma, r, g, b). */
void orc_mlp_points(const orc_field* fd, int64_t n, const double* feat, double* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        orc_act a;
        for (int k = 0; k < fd->mlp_in; ++k) a.feat[k] = feat[(int64_t)k * n + i];
        orc_mlp_forward(fd, &a);
        out[i] = a.sigma;
        for (int c = 0; c < 3; ++c) out[(int64_t)(1 + c) * n + i] = a.rgb[c];
    }
}

/* Field query at n live points p[3][n] (warp -> encode -> MLPs): out[4][n]. */
void orc_query_points(const orc_view* v, int64_t n, const float* p, double* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        float q[3] = {p[i], p[n + i], p[2 * n + i]};
        orc_act a;
        orc_eval_sample(v, q, &a, NULL, NULL);
        out[i] = a.sigma;
        for (int c = 0; c < 3; ++c) out[(int64_t)(1 + c) * n + i] = a.rgb[c];
    }
}
