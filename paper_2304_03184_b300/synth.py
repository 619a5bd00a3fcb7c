"""Seeded synthetic inputs shaped like the paper's capture (human + hand-held object).

This module draws the inputs of the hot path and nothing else: pinhole rays, the
deformation graph's canonical nodes and per-node rigid motions (the tracker's output,
Sec. 4.1), one rigid object pose (Sec. 4.1, "Object Rigid Tracking"), hash tables, MLP
weights, 128^3 occupancy bitfields and smooth target colours.  It holds none of the
method's arithmetic (no warp, encoding, MLP or compositing); the CUDA path and the FP64
oracle both consume the arrays it returns.

Recipes (all seeded with numpy's PCG64):
  * camera: eye at distance 2.5 looking at the origin, up +y, vertical fov 50 deg, pixel
    centres (i+1/2, j+1/2), pixel order row-major; rays are rounded once to FP32.
  * graph: Fibonacci-sphere points scaled to an ellipsoid with semi-axes (0.4, 0.8, 0.3)
    (a standing person ~1.6 m tall in a [-1,1]^3 box); each node's motion is a rotation
    about a uniform random axis by U(0, 15 deg) plus a translation uniform in the
    0.05-ball.  The motion is given as a unit dual quaternion (real part q_r, dual part
    q_d = 1/2 (0,t) q_r) and the live node position x_live = R x + t is computed with the
    Rodrigues rotation matrix in FP64 and rounded once to FP32.
  * object: rotation by 30 deg about a random axis plus a translation of length 0.2 in a
    random direction; its canonical centre is (0.55, 0, 0).
  * occupancy (live space, 128^3 over [-1,1]^3, bit x + 128 (y + 128 z)): human cells whose
    centre lies within 0.12 of a live node; object cells whose centre lies inside the
    sphere of radius 0.25 about the posed object centre.
  * hash tables U(-0.5, 0.5); MLP weights Xavier-uniform U(+-sqrt(6/(fan_in+fan_out))).
  * target colours: 0.5 + 0.45 sin(a_k . d + b_k) per channel k, smooth in the ray
    direction d (a stand-in for the paper's RGB captures, which are not available).
  * deformation net (Sec. 4.2, sizes of Sec. 4.4): tables U(-0.5, 0.5), Xavier weights with
    the output layer scaled by 0.05 (|delta v| ~ 1e-2); pose: 24 axis-angle joints with
    components U(-0.3, 0.3) rad.
  * sensor depth and mask per training ray (stand-ins for the RGBD depth and the
    segmentation masks): first hit of the canonical body ellipsoid (human batches) or of
    the posed object sphere (object batches); mask 1 on a hit, else depth 0 and mask 0.
    Computed from the rays alone, so they draw no random numbers.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

OCC_RES = 128
ELLIPSOID = (0.4, 0.8, 0.3)
OBJECT_CENTRE = (0.55, 0.0, 0.0)
OBJECT_RADIUS = 0.25


# --------------------------------------------------------------------------- containers
@dataclasses.dataclass
class FieldDesc:
    L: int
    log2_T: int
    F: int
    N_min: int
    growth: float
    hidden: int = 64
    geo_out: int = 16
    col_hidden: int = 64

    @property
    def mlp_in(self) -> int:
        return self.L * self.F

    @property
    def T(self) -> int:
        return 1 << self.log2_T

    def n_table_params(self) -> int:
        return self.L * self.T * self.F

    def weight_shapes(self):
        """(rows, cols) of W1..W5, each stored row-major [out][in]."""
        return [(self.hidden, self.mlp_in), (self.hidden, self.hidden),
                (self.geo_out, self.hidden), (self.col_hidden, self.geo_out - 1),
                (3, self.col_hidden)]

    def n_weight_params(self) -> int:
        return sum(r * c for r, c in self.weight_shapes())


@dataclasses.dataclass
class FieldParams:
    desc: FieldDesc
    tables: np.ndarray   # float32 [L][T][F]
    weights: np.ndarray  # float32 flat, W1..W5 row-major


@dataclasses.dataclass
class Graph:
    x_canon: np.ndarray  # float32 [3][N]
    dq: np.ndarray       # float32 [8][N]  (q_r w,x,y,z ; q_d w,x,y,z)
    x_live: np.ndarray   # float32 [3][N]
    K: int
    radius: float


@dataclasses.dataclass
class DeformDesc:
    """Pose-conditioned deformation net: its own hash encoding (L x F features) of the
    warped point, concatenated with the pose (pose_dim), n_hidden ReLU layers of width
    hidden, a linear 3-vector output."""
    L: int = 16
    log2_T: int = 19
    F: int = 2
    N_min: int = 16
    growth: float = 1.38
    pose_dim: int = 72
    hidden: int = 128
    n_hidden: int = 4

    @property
    def T(self) -> int:
        return 1 << self.log2_T

    @property
    def n_in(self) -> int:
        return self.L * self.F + self.pose_dim

    def weight_shapes(self):
        return ([(self.hidden, self.n_in)] + [(self.hidden, self.hidden)] * (self.n_hidden - 1)
                + [(3, self.hidden)])

    def n_weight_params(self) -> int:
        return sum(r * c for r, c in self.weight_shapes())


@dataclasses.dataclass
class DeformParams:
    desc: DeformDesc
    tables: np.ndarray   # float32 [L][T][F]
    weights: np.ndarray  # float32 flat, W_1..W_n, W_out row-major


@dataclasses.dataclass
class View:
    """One field seen through one frame's motion: graph is None for the rigid field."""
    field: FieldParams
    graph: Optional[Graph] = None
    rigid_dq: Optional[np.ndarray] = None   # float32 [8], canonical -> live
    occupancy: Optional[np.ndarray] = None  # uint32 [128^3 / 32]
    deform: Optional[DeformParams] = None   # human field only
    pose: Optional[np.ndarray] = None       # float32 [pose_dim], the frame's pose


@dataclasses.dataclass
class Rays:
    o: np.ndarray  # float32 [3][R]
    d: np.ndarray  # float32 [3][R]

    @property
    def n(self) -> int:
        return self.o.shape[1]


# --------------------------------------------------------------------------- geometry inputs
def look_at_basis(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)):
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    true_up = np.cross(right, fwd)
    return right, true_up, fwd


def pinhole_rays(width: int, height: int, fov_y_deg: float, eye, target=(0.0, 0.0, 0.0)) -> Rays:
    """Rays through pixel centres of a pinhole camera, row-major pixel order."""
    right, up, fwd = look_at_basis(eye, target)
    f = 0.5 * height / math.tan(math.radians(fov_y_deg) * 0.5)
    i, j = np.meshgrid(np.arange(width, dtype=np.float64), np.arange(height, dtype=np.float64))
    x = (i.ravel() + 0.5 - 0.5 * width) / f
    y = -(j.ravel() + 0.5 - 0.5 * height) / f
    d = x[:, None] * right[None] + y[:, None] * up[None] + fwd[None]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(np.asarray(eye, np.float64), d.shape)
    return Rays(np.ascontiguousarray(o.T, np.float32), np.ascontiguousarray(d.T, np.float32))


def ring_rays(n_cams: int, width: int, height: int, fov_y_deg: float, dist: float) -> Rays:
    """All pixels of n_cams cameras on a horizontal ring of radius dist around the origin."""
    os_, ds = [], []
    for c in range(n_cams):
        a = 2.0 * math.pi * c / n_cams
        r = pinhole_rays(width, height, fov_y_deg, (dist * math.sin(a), 0.0, dist * math.cos(a)))
        os_.append(r.o)
        ds.append(r.d)
    return Rays(np.concatenate(os_, axis=1), np.concatenate(ds, axis=1))


def subset_rays(rays: Rays, idx: np.ndarray) -> Rays:
    return Rays(np.ascontiguousarray(rays.o[:, idx]), np.ascontiguousarray(rays.d[:, idx]))


def fibonacci_ellipsoid(n: int, semi_axes=ELLIPSOID) -> np.ndarray:
    k = np.arange(n, dtype=np.float64)
    y = 1.0 - 2.0 * (k + 0.5) / n
    rad = np.sqrt(np.maximum(0.0, 1.0 - y * y))
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    p = np.stack([np.cos(phi) * rad, y, np.sin(phi) * rad])
    return p * np.asarray(semi_axes, np.float64)[:, None]


def random_axes(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def random_in_ball(rng: np.random.Generator, n: int, radius: float) -> np.ndarray:
    dirs = random_axes(rng, n)
    r = radius * rng.uniform(0.0, 1.0, size=n) ** (1.0 / 3.0)
    return dirs * r[:, None]


def rodrigues(axis: np.ndarray, angle: float) -> np.ndarray:
    kx, ky, kz = axis
    Kx = np.array([[0.0, -kz, ky], [kz, 0.0, -kx], [-ky, kx, 0.0]])
    return np.eye(3) + math.sin(angle) * Kx + (1.0 - math.cos(angle)) * (Kx @ Kx)


def motion_dual_quaternion(axis: np.ndarray, angle: float, t: np.ndarray) -> np.ndarray:
    """Unit dual quaternion of x -> R(axis, angle) x + t: q_r = (cos a/2, sin a/2 axis),
    q_d = 1/2 (0, t) q_r (Hamilton product).  Encodes the tracker's motion input."""
    h = 0.5 * angle
    qr = np.array([math.cos(h), *(math.sin(h) * np.asarray(axis, np.float64))])
    tw, tv = 0.0, np.asarray(t, np.float64)
    qd_w = tw * qr[0] - np.dot(tv, qr[1:])
    qd_v = tw * qr[1:] + qr[0] * tv + np.cross(tv, qr[1:])
    return np.concatenate([qr, 0.5 * np.array([qd_w, *qd_v])])


def make_graph(rng: np.random.Generator, n_nodes: int, K: int, max_deg: float = 15.0,
               max_t: float = 0.05, radius: float = 0.1) -> Graph:
    xc = fibonacci_ellipsoid(n_nodes)
    xc32 = xc.astype(np.float32)
    axes = random_axes(rng, n_nodes)
    angles = np.radians(rng.uniform(0.0, max_deg, size=n_nodes))
    trans = random_in_ball(rng, n_nodes, max_t)
    dq = np.zeros((8, n_nodes))
    xl = np.zeros((3, n_nodes))
    for i in range(n_nodes):
        dq[:, i] = motion_dual_quaternion(axes[i], angles[i], trans[i])
        xl[:, i] = rodrigues(axes[i], angles[i]) @ xc32[:, i].astype(np.float64) + trans[i]
    return Graph(xc32, dq.astype(np.float32), xl.astype(np.float32), K, radius)


def repose_graph(rng: np.random.Generator, g: Graph, max_deg: float = 15.0, max_t: float = 0.05) -> Graph:
    """A fresh per-frame pose of the same canonical graph (same node count, K, radius)."""
    n = g.x_canon.shape[1]
    axes = random_axes(rng, n)
    angles = np.radians(rng.uniform(0.0, max_deg, size=n))
    trans = random_in_ball(rng, n, max_t)
    dq = np.zeros((8, n))
    xl = np.zeros((3, n))
    for i in range(n):
        dq[:, i] = motion_dual_quaternion(axes[i], angles[i], trans[i])
        xl[:, i] = rodrigues(axes[i], angles[i]) @ g.x_canon[:, i].astype(np.float64) + trans[i]
    return Graph(g.x_canon, dq.astype(np.float32), xl.astype(np.float32), g.K, g.radius)


def _hamilton(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return np.array([a[0] * b[0] - np.dot(a[1:], b[1:]), *(a[0] * b[1:] + b[0] * a[1:] + np.cross(a[1:], b[1:]))])


def articulated_pose(rng: np.random.Generator, g: Graph, max_deg: float = 15.0, max_t: float = 0.05,
                     max_twist: float = 30.0) -> Graph:
    """A spatially coherent per-frame pose of the canonical graph: a twist about the
    vertical axis through the origin whose angle grows linearly with height (beta y/0.8,
    clamped, beta ~ U(-max_twist, max_twist) deg), followed by one global motion (random axis,
    U(0, max_deg) deg about the origin, translation uniform in the max_t ball).  Nearby
    nodes get nearby motions, as the tracker's regularised motion field does (unlike
    repose_graph, which moves every node independently)."""
    n = g.x_canon.shape[1]
    axis = random_axes(rng, 1)[0]
    ang = math.radians(rng.uniform(0.0, max_deg))
    t = random_in_ball(rng, 1, max_t)[0]
    beta = math.radians(rng.uniform(-max_twist, max_twist))
    qg = np.array([math.cos(0.5 * ang), *(math.sin(0.5 * ang) * axis)])
    Rg = rodrigues(axis, ang)
    dq = np.zeros((8, n))
    xl = np.zeros((3, n))
    ey = np.array([0.0, 1.0, 0.0])
    for i in range(n):
        x = g.x_canon[:, i].astype(np.float64)
        a = beta * min(1.0, max(-1.0, x[1] / 0.8))
        qr = _hamilton(qg, np.array([math.cos(0.5 * a), 0.0, math.sin(0.5 * a), 0.0]))
        qd = 0.5 * _hamilton(np.array([0.0, *t]), qr)
        dq[:, i] = np.concatenate([qr, qd])
        xl[:, i] = Rg @ (rodrigues(ey, a) @ x) + t
    return Graph(g.x_canon, dq.astype(np.float32), xl.astype(np.float32), g.K, g.radius)


def make_object_pose(rng: np.random.Generator, angle_deg: float = 30.0, t_len: float = 0.2):
    """(dual quaternion float32[8], R, t) of the object's canonical -> live motion."""
    axis = random_axes(rng, 1)[0]
    t = random_axes(rng, 1)[0] * t_len
    ang = math.radians(angle_deg)
    return motion_dual_quaternion(axis, ang, t).astype(np.float32), rodrigues(axis, ang), t


# --------------------------------------------------------------------------- occupancy
def _cell_centres(res: int = OCC_RES) -> np.ndarray:
    c = -1.0 + (np.arange(res) + 0.5) * (2.0 / res)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")   # x fastest
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def pack_bits(mask: np.ndarray) -> np.ndarray:
    """bool[res^3] (index x + res (y + res z)) -> uint32 words, bit i&31 of word i>>5."""
    m = mask.reshape(-1, 32).astype(np.uint64)
    w = (m << np.arange(32, dtype=np.uint64)[None, :]).sum(axis=1)
    return w.astype(np.uint32)


def occupancy_near_nodes(x_live: np.ndarray, dist: float = 0.12) -> np.ndarray:
    from scipy.spatial import cKDTree
    tree = cKDTree(x_live.T.astype(np.float64))
    d, _ = tree.query(_cell_centres(), k=1, distance_upper_bound=dist * 1.5)
    return pack_bits(d <= dist)


def occupancy_sphere(centre, radius: float = OBJECT_RADIUS) -> np.ndarray:
    c = _cell_centres()
    return pack_bits(np.sum((c - np.asarray(centre)[None]) ** 2, axis=1) <= radius * radius)


# --------------------------------------------------------------------------- field parameters
def xavier_weights(rng: np.random.Generator, desc: FieldDesc) -> np.ndarray:
    parts = []
    for rows, cols in desc.weight_shapes():
        a = math.sqrt(6.0 / (rows + cols))
        parts.append(rng.uniform(-a, a, size=rows * cols))
    return np.concatenate(parts).astype(np.float32)


def make_field(rng: np.random.Generator, desc: FieldDesc) -> FieldParams:
    tables = rng.uniform(-0.5, 0.5, size=(desc.L, desc.T, desc.F)).astype(np.float32)
    return FieldParams(desc, tables, xavier_weights(rng, desc))


def make_deform(rng: np.random.Generator, desc: DeformDesc = DeformDesc(), out_scale: float = 0.05) -> DeformParams:
    """Deformation net: tables U(-0.5, 0.5), Xavier-uniform weights, the output layer
    scaled by out_scale so that the residual displacement is a small correction of the
    warp (|delta v| of order 1e-2)."""
    tables = rng.uniform(-0.5, 0.5, size=(desc.L, desc.T, desc.F)).astype(np.float32)
    parts = []
    shapes = desc.weight_shapes()
    for k, (o, i) in enumerate(shapes):
        a = math.sqrt(6.0 / (i + o))
        w = rng.uniform(-a, a, size=(o, i))
        if k == len(shapes) - 1:
            w *= out_scale
        parts.append(w.ravel())
    return DeformParams(desc, tables, np.concatenate(parts).astype(np.float32))


def make_pose(rng: np.random.Generator, pose_dim: int = 72, max_angle: float = 0.3) -> np.ndarray:
    """A body pose theta: pose_dim / 3 joints as axis-angle vectors with components
    U(-max_angle, max_angle) rad (the shape of an SMPL pose; the SMPL model is not used)."""
    return rng.uniform(-max_angle, max_angle, size=pose_dim).astype(np.float32)


def sensor_depth_mask(rays: Rays, centre, axes) -> Tuple[np.ndarray, np.ndarray]:
    """Stand-in for the RGBD sensor and the segmentation mask of one actor: the distance
    along each (unit-direction) ray to its first hit of an ellipsoid (centre, semi-axes),
    and a mask that is 1 where the ray hits it; depth 0 and mask 0 elsewhere."""
    c = np.asarray(centre, np.float64)[:, None]
    a = np.asarray(axes, np.float64)[:, None]
    o = (rays.o.astype(np.float64) - c) / a
    d = rays.d.astype(np.float64) / a
    qa = np.sum(d * d, axis=0)
    qb = 2.0 * np.sum(o * d, axis=0)
    qc = np.sum(o * o, axis=0) - 1.0
    disc = qb * qb - 4.0 * qa * qc
    hit = disc >= 0.0
    t = np.where(hit, (-qb - np.sqrt(np.where(hit, disc, 0.0))) / (2.0 * qa), 0.0)
    hit &= t > 0.0
    return np.where(hit, 1.0, 0.0).astype(np.float32), np.where(hit, t, 0.0).astype(np.float32)


def target_colours(rng: np.random.Generator, rays: Rays) -> np.ndarray:
    a = rng.normal(scale=3.0, size=(3, 3))
    b = rng.uniform(0.0, 2.0 * math.pi, size=3)
    d = rays.d.astype(np.float64)
    return (0.5 + 0.45 * np.sin(a @ d + b[:, None])).astype(np.float32)


# --------------------------------------------------------------------------- workloads
CFG1_FIELD = FieldDesc(L=8, log2_T=14, F=2, N_min=16, growth=1.5)
CFG2_FIELD = FieldDesc(L=16, log2_T=19, F=2, N_min=16, growth=1.38)
CFG5_FIELD = FieldDesc(L=16, log2_T=21, F=2, N_min=16, growth=1.38)


@dataclasses.dataclass
class RenderWorkload:
    name: str
    rays: Rays
    views: List[View]
    n_samples: int
    t_eps: float = 1e-4


@dataclasses.dataclass
class TrainBatch:
    rays: Rays
    view: View
    target: np.ndarray  # float32 [3][R]
    mask: Optional[np.ndarray] = None    # float32 [R], 1 where the ray sees the field's actor
    depth: Optional[np.ndarray] = None   # float32 [R], sensor depth along the ray (0 = none)


@dataclasses.dataclass
class TrainWorkload:
    name: str
    batches: List[TrainBatch]
    fields: List[FieldParams]
    n_samples: int
    t_eps: float = 1e-4
    huber_delta: float = 0.1
    lr: float = 1e-2
    beta1: float = 0.9
    beta2: float = 0.99
    adam_eps: float = 1e-15


def plain_forward(seed: int = 1, res: int = 64, n_samples: int = 64) -> RenderWorkload:
    """Single human field, no occupancy: 64x64 rays, 64 samples, L=8, T=2^14, 64 nodes, K=4."""
    rng = np.random.default_rng(seed)
    rays = pinhole_rays(res, res, 50.0, (0.0, 0.0, 2.5))
    field = make_field(rng, CFG1_FIELD)
    graph = make_graph(rng, 64, K=4)
    return RenderWorkload("plain_forward_64x64_s64_L8_T2^14_N64", rays,
                          [View(field, graph=graph)], n_samples)


def two_field_render(seed: int = 2, width: int = 512, height: int = 512, n_samples: int = 128,
                     field_desc: FieldDesc = CFG2_FIELD, n_nodes: int = 2048, K: int = 4) -> RenderWorkload:
    """Human (DQB-warped) + object (rigid) fields with occupancy skipping, depth-composited."""
    rng = np.random.default_rng(seed)
    rays = pinhole_rays(width, height, 50.0, (0.0, 0.0, 2.5))
    human = make_field(rng, field_desc)
    obj = make_field(rng, field_desc)
    graph = make_graph(rng, n_nodes, K=K)
    odq, oR, ot = make_object_pose(rng)
    centre = oR @ np.asarray(OBJECT_CENTRE) + ot
    views = [View(human, graph=graph, occupancy=occupancy_near_nodes(graph.x_live)),
             View(obj, rigid_dq=odq, occupancy=occupancy_sphere(centre))]
    return RenderWorkload(f"two_field_render_{width}x{height}_s{n_samples}_L{field_desc.L}"
                          f"_T2^{field_desc.log2_T}_N{n_nodes}_K{K}", rays, views, n_samples)


def train_step_workload(seed: int = 3, n_rays: int = 1 << 18, n_samples: int = 128,
                        image: int = 512, field_desc: FieldDesc = CFG2_FIELD,
                        n_nodes: int = 2048, K: int = 4) -> TrainWorkload:
    """Human field of the two-field render, n_rays drawn from 4 ring cameras, Huber loss."""
    rng = np.random.default_rng(seed)
    field = make_field(rng, field_desc)
    graph = make_graph(rng, n_nodes, K=K)
    all_rays = ring_rays(4, image, image, 50.0, 2.5)
    idx = np.sort(rng.choice(all_rays.n, size=n_rays, replace=False))
    idx = rng.permutation(idx)
    rays = subset_rays(all_rays, idx)
    view = View(field, graph=graph, occupancy=occupancy_near_nodes(graph.x_live))
    batch = TrainBatch(rays, view, target_colours(rng, rays), *sensor_depth_mask(rays, (0, 0, 0), ELLIPSOID))
    return TrainWorkload(f"train_step_{n_rays}rays_s{n_samples}_L{field_desc.L}_T2^{field_desc.log2_T}"
                         f"_N{n_nodes}", [batch], [field], n_samples)


def keyframe_batch_workload(seed: int = 4, n_frames: int = 8, n_samples: int = 128,
                            log2_rays=(14.0, 18.0), image: int = 512,
                            field_desc: FieldDesc = CFG2_FIELD, n_nodes: int = 2048) -> TrainWorkload:
    """n_frames key frames x (human, object): per-frame graph pose and object pose, ray
    counts floor(2^U(14,18)) per frame per field, drawn from 4 ring cameras."""
    rng = np.random.default_rng(seed)
    human = make_field(rng, field_desc)
    obj = make_field(rng, field_desc)
    base = make_graph(rng, n_nodes, K=4)
    all_rays = ring_rays(4, image, image, 50.0, 2.5)
    batches = []
    for _ in range(n_frames):
        g = repose_graph(rng, base)
        odq, oR, ot = make_object_pose(rng)
        centre = oR @ np.asarray(OBJECT_CENTRE) + ot
        hv = View(human, graph=g, occupancy=occupancy_near_nodes(g.x_live))
        ov = View(obj, rigid_dq=odq, occupancy=occupancy_sphere(centre))
        for v, (c, ax) in ((hv, ((0, 0, 0), ELLIPSOID)), (ov, (centre, (OBJECT_RADIUS,) * 3))):
            n = int(math.floor(2.0 ** rng.uniform(*log2_rays)))
            idx = rng.choice(all_rays.n, size=n, replace=False)
            rays = subset_rays(all_rays, idx)
            batches.append(TrainBatch(rays, v, target_colours(rng, rays), *sensor_depth_mask(rays, c, ax)))
    name = f"keyframe_batch_{n_frames}frames_x2fields_s{n_samples}"
    if tuple(log2_rays) != (14.0, 18.0):
        name += f"_rays2^{log2_rays[0]:g}-2^{log2_rays[1]:g}"
    return TrainWorkload(name, batches, [human, obj], n_samples)
