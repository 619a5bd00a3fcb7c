"""ctypes front end of the FP64 CPU oracle (invr_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by the
CPU-baseline leg of bench.py, never by the product package.  It marshals numpy arrays
into the C oracle and back; all arithmetic lives in invr_oracle.c.

What pins each oracle function (tests/test_oracle_pins.py, run with -m "not gpu"):
  ray setup / samples   axis-aligned ray closed form (t_n, t_f, dt, midpoints), misses,
                        samples inside the box and strictly increasing
  occupancy lookup      integer cell of hand-placed points; bit packing round trip
  level resolution      hand-computed table of floor(16 * 1.5^l) (tests/golden)
  vertex index          dense levels: bijection onto [0,(N+1)^3); hashed levels: the
                        published primes (tests/golden) via Python integers, the +x
                        XOR-1 adjacency, range [0,T)
  trilinear encoding    affine tables reproduce the affine function exactly; at vertices
                        the stored entry is returned exactly
  nearest nodes         numpy lexsort of float32 keys over all nodes
  DQ blend / warp       |q_r| = 1 and q_r.q_d = 0; K=1 returns the node's own inverse
                        motion; equal motions everywhere give that rigid motion; the
                        identity motion gives v_c = p; sign flips of node quaternions do
                        not change the result; x_live = R x + t of the input generator
  rigid warp            R orthonormal, round trip T^-1 T p = p
  look-up-table search  table exponential within 4e-7 of exp; canonical KNN field = numpy
                        lexsort per voxel; identity motion maps every voxel to itself; a
                        one-voxel translation shifts the live index by one; the FP32
                        forward-warp recipe within 2e-6 of an FP64 blend computed in the
                        test; live index = brute-force smallest canonical voxel per cell
                        (FP64, cell-face cases exempt); table neighbour sets give the
                        exact warp wherever they equal the exact K nearest, holes use
                        the exact set
  MLPs                  zero weights give sigma = 1, c = 1/2; numpy matmul chain
  compositing           constant density closed forms for A, C, D; single sample;
                        early-termination bound; identity deformation equals the rigid
                        field at p; depth ordering cases of the two-field composition
  loss / gradient       Huber closed form; central finite differences in FP64 of the
                        loss on 64 parameters
  paper's losses        constant-density closed form of the masked colour L2 norm plus
                        the masked depth L1 term (Sec. 4.4); central differences; a binary
                        mask equals cutting the batch down to the masked-in rays
  Adam                  first and second steps in closed form
  joint compositing     an empty second field reproduces the single-field render; two
                        constant fields (sigma = 1 each, c = 1/2) give A = 1 - exp(-2 L)
  deformation net       forward = numpy matmul chain on the hash features and pose; a
                        zero output layer leaves the warp unchanged; the encoding's point
                        derivative = the affine-table closed form and central differences;
                        training gradients of the net's tables and weights and of the
                        field through v_c = v_t + delta v by central differences
  occupancy update      a field built so that sigma = exp(max(a.x + b, 0)) exactly (affine
                        dense level, identity-like first layers) gives that density at
                        every cell centre; decay keeps max(decay d, sigma); bits = d > thr
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "invr_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP32 decisions need -ffp-contract=off)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", LIB + ".tmp", SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(LIB)
        _declare(_lib)
    return _lib


# ----------------------------------------------------------------------- C structs
class CField(C.Structure):
    _fields_ = [("L", C.c_int), ("log2_T", C.c_int), ("F", C.c_int), ("N_min", C.c_int),
                ("growth", C.c_double), ("mlp_in", C.c_int), ("hidden", C.c_int),
                ("geo_out", C.c_int), ("col_hidden", C.c_int),
                ("tables", C.POINTER(C.c_double)), ("weights", C.POINTER(C.c_double))]


class CGraph(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("K", C.c_int), ("radius", C.c_double),
                ("x_live", C.POINTER(C.c_float)), ("dq", C.POINTER(C.c_float)),
                ("lut_res", C.c_int), ("lut_canon", C.POINTER(C.c_uint16)),
                ("lut_live", C.POINTER(C.c_uint32))]


class CDeform(C.Structure):
    _fields_ = [("L", C.c_int), ("log2_T", C.c_int), ("F", C.c_int), ("N_min", C.c_int),
                ("growth", C.c_double), ("pose_dim", C.c_int), ("hidden", C.c_int), ("n_hidden", C.c_int),
                ("tables", C.POINTER(C.c_double)), ("weights", C.POINTER(C.c_double))]


class CView(C.Structure):
    _fields_ = [("field", C.POINTER(CField)), ("graph", C.POINTER(CGraph)),
                ("rigid_dq", C.POINTER(C.c_float)), ("occupancy", C.POINTER(C.c_uint32)),
                ("deform", C.POINTER(CDeform)), ("pose", C.POINTER(C.c_float))]


class CBatch(C.Structure):
    _fields_ = [("n_rays", C.c_int64), ("o", C.POINTER(C.c_float)), ("d", C.POINTER(C.c_float)),
                ("view", C.POINTER(CView)), ("target", C.POINTER(C.c_float)),
                ("grad_tables", C.POINTER(C.c_double)), ("grad_weights", C.POINTER(C.c_double)),
                ("mask", C.POINTER(C.c_float)), ("depth", C.POINTER(C.c_float)),
                ("grad_deform_tables", C.POINTER(C.c_double)), ("grad_deform_weights", C.POINTER(C.c_double))]


def _declare(L):
    P = C.c_void_p
    L.orc_level_res.argtypes = [C.c_int, C.c_double, C.c_int]
    L.orc_level_res.restype = C.c_int
    L.orc_level_dense.argtypes = [C.c_int, C.c_int]
    L.orc_level_dense.restype = C.c_int
    L.orc_vertex_index.argtypes = [C.c_int, C.c_int, C.c_uint32, C.c_uint32, C.c_uint32]
    L.orc_vertex_index.restype = C.c_uint32
    L.orc_huber.argtypes = [C.c_double, C.c_double]
    L.orc_huber.restype = C.c_double
    L.orc_render.argtypes = [C.c_int64, P, P, C.c_int, C.c_double, C.c_int, P, P, P, P, P, P, P]
    L.orc_render.restype = None
    L.orc_deform_points.argtypes = [P, P, C.c_int64, P, P]
    L.orc_encode_dx_points.argtypes = [P, C.c_int64, P, P, P]
    L.orc_render_joint.argtypes = [C.c_int64, P, P, C.c_int, C.c_double, P, P, P, P]
    L.orc_occupancy_update.argtypes = [P, C.c_double, C.c_double, P, P]
    L.orc_lut_canon_knn.argtypes = [C.c_int, C.c_int, P, C.c_int, P]
    L.orc_lut_live_index.argtypes = [C.c_int, C.c_int, C.c_float, P, P, C.c_int, P, P]
    L.orc_lut_exp_points.argtypes = [C.c_int64, P, P]
    L.orc_lut_forward_points.argtypes = [C.c_int, C.c_int, C.c_float, P, P, C.c_int64, P, P, P]
    L.orc_neighbour_points.argtypes = [P, C.c_int64, P, P, P]
    L.orc_train_loss_grad.argtypes = [C.c_int, P, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                      C.c_double]
    L.orc_train_loss_grad.restype = C.c_double
    L.orc_adam.argtypes = [C.c_int64, P, P, P, P, C.c_int64, C.c_double, C.c_double, C.c_double,
                           C.c_double]
    L.orc_ray_samples.argtypes = [C.c_int64, P, P, C.c_int, P, P, P, P, P]
    L.orc_occupied_points.argtypes = [P, C.c_int64, P, P]
    L.orc_knn_points.argtypes = [P, C.c_int64, P, P, P]
    L.orc_warp_points.argtypes = [P, C.c_int64, P, P, P]
    L.orc_dq_apply_points.argtypes = [P, C.c_int64, P, P]
    L.orc_encode_points.argtypes = [P, C.c_int64, P, P, P, P]
    L.orc_mlp_points.argtypes = [P, C.c_int64, P, P]
    L.orc_query_points.argtypes = [P, C.c_int64, P, P]


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- object wrappers
class Field:
    """FP64 copy of one field's parameters (tables [L][T][F], weights W1..W5)."""

    def __init__(self, desc, tables, weights):
        self.desc = desc
        self.tables = _f64(tables).reshape(-1)
        self.weights = _f64(weights).reshape(-1)
        self._c = CField(desc.L, desc.log2_T, desc.F, desc.N_min, float(desc.growth), desc.mlp_in,
                         desc.hidden, desc.geo_out, desc.col_hidden,
                         self.tables.ctypes.data_as(C.POINTER(C.c_double)),
                         self.weights.ctypes.data_as(C.POINTER(C.c_double)))

    @classmethod
    def from_params(cls, fp):
        return cls(fp.desc, fp.tables, fp.weights)


class Graph:
    """Deformed nodes x_live [3][N] and motions dq [8][N] of one frame.  With lut=(G, canon,
    live) the neighbour sets come from the look-up tables (lut_canon_knn, lut_live_index)
    instead of the exact search."""

    def __init__(self, x_live, dq, K: int, radius: float, lut=None):
        self.x_live = _f32(x_live)
        self.dq = _f32(dq)
        self._c = CGraph(self.x_live.shape[1], K, float(radius),
                         self.x_live.ctypes.data_as(C.POINTER(C.c_float)),
                         self.dq.ctypes.data_as(C.POINTER(C.c_float)), 0, None, None)
        self.lut = None
        if lut is not None:
            G, canon, live = lut
            self.lut = (int(G), np.ascontiguousarray(canon, np.uint16), np.ascontiguousarray(live, np.uint32))
            self._c.lut_res = self.lut[0]
            self._c.lut_canon = self.lut[1].ctypes.data_as(C.POINTER(C.c_uint16))
            self._c.lut_live = self.lut[2].ctypes.data_as(C.POINTER(C.c_uint32))

    @classmethod
    def from_synth(cls, g, lut=None):
        return cls(g.x_live, g.dq, g.K, g.radius, lut)


LUT_EMPTY = 0xFFFFFFFF


def deform_points(deform: Deform, pose, vt) -> np.ndarray:
    """delta v [3][n] of points vt [3][n] under pose (deformation net forward)."""
    vt = _f64(vt)
    pose = _f32(pose)
    dv = np.zeros_like(vt)
    lib().orc_deform_points(C.byref(deform._c), _p(pose), vt.shape[1], _p(vt), _p(dv))
    return dv


def encode_dx_points(field: Field, x, dfeat) -> np.ndarray:
    """Encoding derivative: dx [3][n] = sum over features dfeat [L*F][n] x d feat / d x."""
    x, dfeat = _f64(x), _f64(dfeat)
    dx = np.zeros_like(x)
    lib().orc_encode_dx_points(C.byref(field._c), x.shape[1], _p(x), _p(dfeat), _p(dx))
    return dx


def lut_canon_knn(x_canon, K: int, G: int) -> np.ndarray:
    """Canonical KNN field [G^3][K] (uint16 node ids, ascending by key)."""
    x = _f32(x_canon)
    out = np.zeros((G ** 3, K), np.uint16)
    lib().orc_lut_canon_knn(x.shape[1], K, _p(x), G, _p(out))
    return out


def lut_live_index(x_canon, dq, K: int, radius: float, G: int, canon) -> np.ndarray:
    """Live index field [G^3] (uint32 canonical voxel per live voxel, LUT_EMPTY = none)."""
    x, q = _f32(x_canon), _f32(dq)
    canon = np.ascontiguousarray(canon, np.uint16)
    live = np.zeros(G ** 3, np.uint32)
    lib().orc_lut_live_index(x.shape[1], K, float(radius), _p(x), _p(q), G, _p(canon), _p(live))
    return live


def lut_exp(x) -> np.ndarray:
    x = _f32(x)
    out = np.zeros_like(x)
    lib().orc_lut_exp_points(x.size, _p(x), _p(out))
    return out


def lut_forward_points(x_canon, dq, K: int, radius: float, c, ids) -> np.ndarray:
    """Single-precision forward warp of canonical points c [3][n] by neighbours ids [n][K]."""
    x, q, c = _f32(x_canon), _f32(dq), _f32(c)
    ids = np.ascontiguousarray(ids, np.int32)
    out = np.zeros_like(c)
    lib().orc_lut_forward_points(x.shape[1], K, float(radius), _p(x), _p(q), c.shape[1], _p(c), _p(ids), _p(out))
    return out


def neighbour_points(graph: Graph, p):
    """Neighbour ids [K][n] of live points and whether the tables supplied each set."""
    p = _f32(p)
    n = p.shape[1]
    ids = np.zeros((graph._c.K, n), np.int32)
    from_lut = np.zeros(n, np.int32)
    lib().orc_neighbour_points(C.byref(graph._c), n, _p(p), _p(ids), _p(from_lut))
    return ids, from_lut.astype(bool)


class Deform:
    """FP64 copy of a pose-conditioned deformation net (tables [L][T][F], weights W_1..W_out)."""

    def __init__(self, desc, tables, weights):
        self.desc = desc
        self.tables = _f64(tables).reshape(-1)
        self.weights = _f64(weights).reshape(-1)
        self._c = CDeform(desc.L, desc.log2_T, desc.F, desc.N_min, float(desc.growth), desc.pose_dim, desc.hidden,
                          desc.n_hidden, self.tables.ctypes.data_as(C.POINTER(C.c_double)),
                          self.weights.ctypes.data_as(C.POINTER(C.c_double)))

    @classmethod
    def from_params(cls, dp):
        return cls(dp.desc, dp.tables, dp.weights)


class View:
    def __init__(self, field: Field, graph: Optional[Graph] = None, rigid_dq=None, occupancy=None,
                 deform: Optional[Deform] = None, pose=None):
        self.field, self.graph, self.deform = field, graph, deform
        self.rigid_dq = None if rigid_dq is None else _f32(rigid_dq)
        self.occupancy = None if occupancy is None else np.ascontiguousarray(occupancy, np.uint32)
        self.pose = None if pose is None else _f32(pose)
        self._c = CView(C.pointer(field._c), C.pointer(graph._c) if graph is not None else None,
                        self.rigid_dq.ctypes.data_as(C.POINTER(C.c_float)) if self.rigid_dq is not None else None,
                        self.occupancy.ctypes.data_as(C.POINTER(C.c_uint32)) if self.occupancy is not None else None,
                        C.pointer(deform._c) if deform is not None else None,
                        self.pose.ctypes.data_as(C.POINTER(C.c_float)) if self.pose is not None else None)

    @classmethod
    def from_synth(cls, v, field: Optional[Field] = None, deform: Optional[Deform] = None):
        f = field if field is not None else Field.from_params(v.field)
        g = Graph.from_synth(v.graph) if v.graph is not None else None
        d = deform if deform is not None else (Deform.from_params(v.deform) if v.deform is not None else None)
        return cls(f, g, v.rigid_dq, v.occupancy, d, v.pose)


# ------------------------------------------------------------------------- calls
def level_res(N_min: int, growth: float, l: int) -> int:
    return lib().orc_level_res(N_min, growth, l)


def level_dense(res: int, log2_T: int) -> bool:
    return bool(lib().orc_level_dense(res, log2_T))


def vertex_index(res: int, log2_T: int, x: int, y: int, z: int) -> int:
    return lib().orc_vertex_index(res, log2_T, x, y, z)


def huber(x: float, delta: float) -> float:
    return lib().orc_huber(x, delta)


def ray_samples(o, d, n_samples: int):
    o, d = _f32(o), _f32(d)
    R = o.shape[1]
    hit = np.zeros(R, np.int32)
    tn = np.zeros(R, np.float32)
    dt = np.zeros(R, np.float32)
    t = np.zeros((R, n_samples), np.float32)
    p = np.zeros((3, R, n_samples), np.float32)
    lib().orc_ray_samples(R, _p(o), _p(d), n_samples, _p(hit), _p(tn), _p(dt), _p(t), _p(p))
    return hit, tn, dt, t, p


def occupied_points(bits, p) -> np.ndarray:
    bits = np.ascontiguousarray(bits, np.uint32)
    p = _f32(p)
    out = np.zeros(p.shape[1], np.int32)
    lib().orc_occupied_points(_p(bits), p.shape[1], _p(p), _p(out))
    return out


def knn_points(graph: Graph, p):
    p = _f32(p)
    n = p.shape[1]
    K = graph._c.K
    ids = np.zeros((K, n), np.int32)
    keys = np.zeros((K, n), np.float32)
    lib().orc_knn_points(C.byref(graph._c), n, _p(p), _p(ids), _p(keys))
    return ids, keys


def warp_points(view: View, p, with_blend: bool = False):
    p = _f32(p)
    n = p.shape[1]
    vc = np.zeros((3, n))
    qb = np.zeros((8, n)) if with_blend else None
    lib().orc_warp_points(C.byref(view._c), n, _p(p), _p(vc), _p(qb))
    return (vc, qb) if with_blend else vc


def dq_apply_points(dq, p) -> np.ndarray:
    dq, p = _f64(dq), _f64(p)
    out = np.zeros_like(p)
    lib().orc_dq_apply_points(_p(dq), p.shape[1], _p(p), _p(out))
    return out


def encode_points(field: Field, x, with_index: bool = False):
    x = _f64(x)
    n = x.shape[1]
    d = field.desc
    feat = np.zeros((d.L * d.F, n))
    idx = np.zeros((d.L * 8, n), np.uint32) if with_index else None
    w = np.zeros((d.L * 8, n)) if with_index else None
    lib().orc_encode_points(C.byref(field._c), n, _p(x), _p(feat), _p(idx), _p(w))
    return (feat, idx, w) if with_index else feat


def mlp_points(field: Field, feat) -> np.ndarray:
    feat = _f64(feat)
    n = feat.shape[1]
    out = np.zeros((4, n))
    lib().orc_mlp_points(C.byref(field._c), n, _p(feat), _p(out))
    return out


def query_points(view: View, p) -> np.ndarray:
    p = _f32(p)
    n = p.shape[1]
    out = np.zeros((4, n))
    lib().orc_query_points(C.byref(view._c), n, _p(p), _p(out))
    return out


class RenderResult:
    def __init__(self, rgba, depth, rgba_v, depth_v, n_used, T_end):
        self.rgba, self.depth = rgba, depth
        self.rgba_v, self.depth_v, self.n_used, self.T_end = rgba_v, depth_v, n_used, T_end


def render(o, d, n_samples: int, t_eps: float, views: Sequence[View]) -> RenderResult:
    o, d = _f32(o), _f32(d)
    R = o.shape[1]
    V = len(views)
    assert V in (1, 2)
    arr = (CView * V)(*[v._c for v in views])
    rgba_v = np.zeros((V, 4, R))
    depth_v = np.zeros((V, R))
    n_used = np.zeros((V, R), np.int32)
    T_end = np.zeros((V, R))
    rgba = np.zeros((4, R))
    depth = np.zeros(R)
    lib().orc_render(R, _p(o), _p(d), n_samples, t_eps, V, C.cast(arr, C.c_void_p), _p(rgba_v),
                     _p(depth_v), _p(n_used), _p(T_end), _p(rgba), _p(depth))
    return RenderResult(rgba, depth, rgba_v, depth_v, n_used, T_end)


def render_joint(o, d, n_samples: int, t_eps: float, human: View, obj: View):
    """Joint per-sample compositing of the two fields: (rgba [4][R], depth [R], n_used [R])."""
    o, d = _f32(o), _f32(d)
    R = o.shape[1]
    arr = (CView * 2)(human._c, obj._c)
    rgba = np.zeros((4, R))
    depth = np.zeros(R)
    n_used = np.zeros(R, np.int32)
    lib().orc_render_joint(R, _p(o), _p(d), n_samples, t_eps, C.cast(arr, C.c_void_p), _p(rgba), _p(depth),
                           _p(n_used))
    return rgba, depth, n_used


def occupancy_update(view: View, decay: float, threshold: float, density=None):
    """One density-driven update of the 128^3 live-space occupancy: (density [128^3] FP64,
    bits [65536] uint32).  `density` (updated in place if given) starts at zero otherwise."""
    n = OCC_RES ** 3
    density = np.zeros(n) if density is None else density
    assert density.dtype == np.float64 and density.shape == (n,)
    bits = np.zeros(n // 32, np.uint32)
    lib().orc_occupancy_update(C.byref(view._c), decay, threshold, _p(density), _p(bits))
    return density, bits


OCC_RES = 128


class TrainBatch:
    """One key-frame batch: rays o, d [3][R], the field view, target colour [3][R] and, for
    the paper's losses, the mask M(r) [R] (None = 1) and sensor depth D(r) [R]."""

    def __init__(self, o, d, view: View, target, mask=None, depth=None):
        self.o, self.d, self.target = _f32(o), _f32(d), _f32(target)
        self.mask = None if mask is None else _f32(mask)
        self.depth = None if depth is None else _f32(depth)
        self.view = view


LOSS_KINDS = {"huber": 0, "paper": 1}


def train_loss_grad(batches: List[TrainBatch], n_samples: int, t_eps: float, huber_delta: float,
                    grads: bool = True, loss: str = "huber", depth_weight: float = 1.0):
    """Returns (loss, {id(field): (grad_tables, grad_weights)}).  loss = "huber" (mean
    Huber penalty over rays x channels) or "paper" (Sec. 4.4: sum over rays of the masked
    colour L2 norm plus depth_weight x the masked depth L1 norm)."""
    kind = LOSS_KINDS[loss]
    if kind == 1 and any(b.depth is None for b in batches):
        raise ValueError("the paper's depth loss needs every batch's sensor depth")
    out = {}
    cb = []
    for b in batches:
        f = b.view.field
        if id(f) not in out:
            out[id(f)] = (np.zeros_like(f.tables), np.zeros_like(f.weights))
        gt, gw = out[id(f)]
        dgt = dgw = None
        dn = b.view.deform
        if dn is not None:
            if id(dn) not in out:
                out[id(dn)] = (np.zeros_like(dn.tables), np.zeros_like(dn.weights))
            dgt, dgw = out[id(dn)]
        cb.append(CBatch(b.o.shape[1], b.o.ctypes.data_as(C.POINTER(C.c_float)),
                         b.d.ctypes.data_as(C.POINTER(C.c_float)), C.pointer(b.view._c),
                         b.target.ctypes.data_as(C.POINTER(C.c_float)),
                         gt.ctypes.data_as(C.POINTER(C.c_double)), gw.ctypes.data_as(C.POINTER(C.c_double)),
                         None if b.mask is None else b.mask.ctypes.data_as(C.POINTER(C.c_float)),
                         None if b.depth is None else b.depth.ctypes.data_as(C.POINTER(C.c_float)),
                         None if dgt is None else dgt.ctypes.data_as(C.POINTER(C.c_double)),
                         None if dgw is None else dgw.ctypes.data_as(C.POINTER(C.c_double))))
    arr = (CBatch * len(cb))(*cb)
    value = lib().orc_train_loss_grad(len(cb), C.cast(arr, C.c_void_p), n_samples, t_eps, huber_delta,
                                      1 if grads else 0, kind, depth_weight)
    return value, out


def adam(p, g, m, v, step: int, lr: float, b1: float, b2: float, eps: float):
    """In-place Adam on float64 arrays p, m, v with gradient g."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64(g)
    lib().orc_adam(p.size, _p(p), _p(g), _p(m), _p(v), step, lr, b1, b2, eps)
