"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms, brute
force with numpy, invariants, published constants (tests/golden), or library routines.
None of these tests needs a GPU.
"""
import math
import os

import numpy as np
import pytest

from paper_2304_03184_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def tiny_field(rng, L=2, log2_T=10, F=2, N_min=2, growth=1.5, zero=False):
    desc = synth.FieldDesc(L=L, log2_T=log2_T, F=F, N_min=N_min, growth=growth)
    fp = synth.make_field(rng, desc)
    if zero:
        fp.weights[:] = 0.0
    return fp


# ------------------------------------------------------------------ ray sampling
def test_axis_aligned_ray_closed_form(oracle):
    o = np.array([[0.0], [0.0], [2.5]], np.float32)
    d = np.array([[0.0], [0.0], [-1.0]], np.float32)
    hit, tn, dt, t, p = oracle.ray_samples(o, d, 64)
    assert hit[0] == 1
    assert tn[0] == 1.5 and dt[0] == 2.0 / 64
    j = np.arange(64)
    np.testing.assert_array_equal(t[0], 1.5 + (j + 0.5) * (2.0 / 64))
    np.testing.assert_array_equal(p[2, 0], 2.5 - t[0])
    np.testing.assert_array_equal(p[0, 0], 0.0)


def test_ray_inside_box_starts_at_zero_and_misses(oracle):
    o = np.array([[0.2, 0.0, 0.0], [0.1, 0.0, 5.0], [-0.3, 2.5, 0.0]], np.float32)
    d = np.array([[1.0, 1.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 1.0]], np.float32)
    hit, tn, dt, t, p = oracle.ray_samples(o, d, 8)
    # ray 0 starts inside: t_n = 0, exits x = 1 at t = 0.8
    assert hit[0] == 1 and tn[0] == 0.0
    assert abs(dt[0] * 8 - 0.8) < 1e-6
    # ray 1: z = 2.5 outside the slab and d_z = 0; ray 2: y = 5 outside, d_y = 0
    assert hit[1] == 0 and hit[2] == 0


def test_oblique_rays_samples_inside_box_and_increasing(oracle):
    rays = synth.pinhole_rays(16, 16, 50.0, (0.3, -0.2, 2.5))
    hit, tn, dt, t, p = oracle.ray_samples(rays.o, rays.d, 32)
    assert hit.sum() > 100
    h = hit.astype(bool)
    assert np.all(np.diff(t[h], axis=1) > 0)
    assert np.all(np.abs(p[:, h]) <= 1.0 + 1e-5)
    # midpoint rule: first and last samples half a step from the ends
    tf = tn + dt * 32
    np.testing.assert_allclose(t[h, 0], tn[h] + 0.5 * dt[h], rtol=1e-6)
    np.testing.assert_allclose(t[h, -1], tf[h] - 0.5 * dt[h], rtol=1e-5)
    # positions are o + t d
    o64, d64 = rays.o.astype(np.float64), rays.d.astype(np.float64)
    np.testing.assert_allclose(p[:, h], o64[:, h, None] + t[None, h] * d64[:, h, None], atol=2e-6)


# ---------------------------------------------------------------------- occupancy
def test_occupancy_cell_lookup(oracle):
    mask = np.zeros(128 ** 3, bool)
    cell = (5, 77, 126)
    mask[cell[0] + 128 * (cell[1] + 128 * cell[2])] = True
    bits = synth.pack_bits(mask)
    centre = [-1.0 + (c + 0.5) / 64.0 for c in cell]
    lo = [-1.0 + c / 64.0 for c in cell]                # exact lower corner -> that cell
    hi = [-1.0 + (c + 1) / 64.0 for c in cell]          # exact upper corner -> next cell
    pts = np.array([centre, lo, hi, [centre[0], centre[1], 1.0], [centre[0], centre[1], 3.0]],
                   np.float32).T
    got = oracle.occupied_points(bits, pts)
    # z = 1.0 and z = 3.0 clamp to cell 127, which is empty
    assert list(got) == [1, 1, 0, 0, 0]
    mask2 = np.zeros(128 ** 3, bool)
    mask2[127 + 128 * (0 + 128 * 127)] = True
    got2 = oracle.occupied_points(synth.pack_bits(mask2), np.array([[1.5], [-7.0], [1.0]], np.float32))
    assert got2[0] == 1


# ------------------------------------------------------------------- hash geometry
def test_level_resolution_golden(oracle):
    for n_min, g, l, res in _golden_rows("level_resolution.txt"):
        assert oracle.level_res(int(n_min), float(g), int(l)) == int(res)


def test_dense_hash_switch(oracle):
    # dense iff (N_l+1)^3 <= T: levels 0-1 (L=8, T=2^14, b=1.5), 0-4 (T=2^19, b=1.38),
    # 0-6 (T=2^21, b=1.38)
    for growth, log2_T, n_dense in ((1.5, 14, 2), (1.38, 19, 5), (1.38, 21, 7)):
        flags = [oracle.level_dense(oracle.level_res(16, growth, l), log2_T) for l in range(8)]
        assert flags == [True] * n_dense + [False] * (8 - n_dense)


def test_dense_index_is_bijection(oracle):
    res, log2_T = 5, 10
    n = res + 1
    seen = set()
    for z in range(n):
        for y in range(n):
            for x in range(n):
                seen.add(oracle.vertex_index(res, log2_T, x, y, z))
    assert seen == set(range(n ** 3))
    # steps of 1 along x and N+1 along y
    assert oracle.vertex_index(res, log2_T, 3, 2, 1) - oracle.vertex_index(res, log2_T, 2, 2, 1) == 1
    assert oracle.vertex_index(res, log2_T, 2, 3, 1) - oracle.vertex_index(res, log2_T, 2, 2, 1) == n


def test_hashed_index_published_primes(oracle):
    primes = {k: int(v) for k, v in _golden_rows("hash_primes.txt")}
    res, log2_T = 20, 10
    T = 1 << log2_T
    assert not oracle.level_dense(res, log2_T)
    rng = np.random.default_rng(0)
    for x, y, z in rng.integers(0, res + 1, size=(500, 3)):
        h = ((int(x) * primes["pi1"]) ^ (int(y) * primes["pi2"]) ^ (int(z) * primes["pi3"])) % (1 << 32)
        assert oracle.vertex_index(res, log2_T, int(x), int(y), int(z)) == h % T
    # 32-bit wrap-around on a big level
    big = 2005
    for x, y, z in ((2005, 2005, 2005), (1, 1999, 7)):
        h = ((x * primes["pi1"]) ^ (y * primes["pi2"]) ^ (z * primes["pi3"])) % (1 << 32)
        assert oracle.vertex_index(big, 19, x, y, z) == h % (1 << 19)


def test_hashed_index_x_adjacency_and_range(oracle):
    res, log2_T = 300, 12
    for y, z in ((0, 0), (5, 9), (299, 1)):
        for x in range(0, 300, 2):
            a = oracle.vertex_index(res, log2_T, x, y, z)
            b = oracle.vertex_index(res, log2_T, x + 1, y, z)
            assert b == a ^ 1 and 0 <= a < (1 << log2_T)


def test_trilinear_reproduces_affine_function(oracle):
    rng = np.random.default_rng(1)
    fp = tiny_field(rng, L=2, log2_T=10, F=2, N_min=2, growth=1.5)
    d = fp.desc
    tables = np.zeros((d.L, d.T, d.F))
    coef = rng.normal(size=(d.L, d.F, 4))
    for l in range(d.L):
        res = oracle.level_res(d.N_min, d.growth, l)
        assert oracle.level_dense(res, d.log2_T)
        for z in range(res + 1):
            for y in range(res + 1):
                for x in range(res + 1):
                    i = oracle.vertex_index(res, d.log2_T, x, y, z)
                    tables[l, i] = coef[l, :, 0] + coef[l, :, 1:] @ np.array([x, y, z], float)
    f = oracle.Field(d, tables, fp.weights)
    pts = rng.uniform(-1.1, 1.1, size=(3, 200))          # outside the box u clamps to [0,1]
    feat = oracle.encode_points(f, pts)
    for l in range(d.L):
        res = oracle.level_res(d.N_min, d.growth, l)
        q = np.clip((pts + 1.0) * 0.5, 0.0, 1.0) * res
        want = coef[l, :, 0:1] + coef[l, :, 1:] @ q
        np.testing.assert_allclose(feat[l * d.F:(l + 1) * d.F], want, atol=1e-12)


def test_encoding_at_vertices_returns_entries(oracle):
    rng = np.random.default_rng(2)
    fp = synth.make_field(rng, synth.CFG1_FIELD)
    d = fp.desc
    f = oracle.Field.from_params(fp)
    # level 0 has N_0 = 16: vertices at -1 + k/8 are exact in binary
    ks = rng.integers(0, 17, size=(3, 50))
    pts = -1.0 + ks / 8.0
    feat = oracle.encode_points(f, pts)
    for i in range(50):
        x, y, z = (int(v) for v in ks[:, i])
        slot = oracle.vertex_index(16, d.log2_T, x, y, z)
        np.testing.assert_array_equal(feat[0:2, i], fp.tables[0, slot].astype(np.float64))
        # the finer levels are exact too wherever the point is one of their vertices
        for l in range(1, d.L):
            res = oracle.level_res(d.N_min, d.growth, l)
            q = (pts[:, i] + 1.0) * 0.5 * res
            if np.all(q == np.round(q)):
                v = [int(c) for c in np.minimum(q, res)]
                s = oracle.vertex_index(res, d.log2_T, *v)
                np.testing.assert_array_equal(feat[2 * l:2 * l + 2, i], fp.tables[l, s].astype(np.float64))


# ----------------------------------------------------------------- nearest nodes
def test_knn_matches_numpy_lexsort(oracle):
    rng = np.random.default_rng(3)
    N, K = 50, 4
    x = rng.uniform(-0.5, 0.5, size=(3, N)).astype(np.float32)
    x[:, 10] = x[:, 3]     # exact duplicates -> ties resolved to the lower index
    x[:, 40] = x[:, 3]
    g = oracle.Graph(x, np.tile(np.array([1, 0, 0, 0, 0, 0, 0, 0], np.float32)[:, None], (1, N)), K, 0.1)
    pts = rng.uniform(-0.6, 0.6, size=(3, 300)).astype(np.float32)
    pts[:, 0] = x[:, 3]
    ids, keys = oracle.knn_points(g, pts)
    for i in range(pts.shape[1]):
        dx = pts[0, i] - x[0]
        dy = pts[1, i] - x[1]
        dz = pts[2, i] - x[2]
        key = (dx * dx + dy * dy) + dz * dz      # numpy float32 arithmetic, no fusion
        order = np.lexsort((np.arange(N), key))[:K]
        np.testing.assert_array_equal(ids[:, i], order)
        np.testing.assert_array_equal(keys[:, i], key[order])
    assert list(ids[:3, 0]) == [3, 10, 40]


# ------------------------------------------------------------- dual quaternions
def _graph_view(oracle, g, field=None):
    rng = np.random.default_rng(9)
    f = field or oracle.Field.from_params(tiny_field(rng))
    return oracle.View(f, graph=oracle.Graph.from_synth(g))


def test_generator_live_nodes_are_dq_motion(oracle):
    rng = np.random.default_rng(4)
    g = synth.make_graph(rng, 40, K=4)
    for i in range(40):
        got = oracle.dq_apply_points(g.dq[:, i], g.x_canon[:, i:i + 1])
        np.testing.assert_allclose(got[:, 0], g.x_live[:, i], atol=2e-7)


def test_blend_is_unit_dual_quaternion(oracle):
    rng = np.random.default_rng(5)
    g = synth.make_graph(rng, 64, K=4)
    v = _graph_view(oracle, g)
    pts = rng.uniform(-0.9, 0.9, size=(3, 500)).astype(np.float32)
    _, qb = oracle.warp_points(v, pts, with_blend=True)
    np.testing.assert_allclose(np.sum(qb[:4] ** 2, axis=0), 1.0, atol=1e-12)
    np.testing.assert_allclose(np.sum(qb[:4] * qb[4:], axis=0), 0.0, atol=1e-12)


def test_k1_inverts_own_node_motion(oracle):
    rng = np.random.default_rng(6)
    g = synth.make_graph(rng, 64, K=1)
    v = _graph_view(oracle, g)
    vc = oracle.warp_points(v, g.x_live)
    np.testing.assert_allclose(vc, g.x_canon.astype(np.float64), atol=1e-6)


def test_equal_motions_give_that_rigid_motion(oracle):
    rng = np.random.default_rng(7)
    g = synth.make_graph(rng, 64, K=4)
    axis = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    t = np.array([0.04, -0.02, 0.01])
    dq = synth.motion_dual_quaternion(axis, math.radians(12.0), t)
    g.dq = np.tile(dq.astype(np.float32)[:, None], (1, 64))
    v = _graph_view(oracle, g)
    pts = rng.uniform(-0.9, 0.9, size=(3, 300)).astype(np.float32)
    vc = oracle.warp_points(v, pts)
    R = synth.rodrigues(axis, math.radians(12.0))
    # inverse motion from the single-precision quaternion: R^T (p - t) to float32 accuracy
    want = R.T @ (pts.astype(np.float64) - t[:, None])
    np.testing.assert_allclose(vc, want, atol=2e-6)


def test_two_node_blend_closed_form(oracle):
    """Two nodes rotating about one axis through the origin by angles a1, a2: the blend is
    the rotation about that axis by phi with tan(phi/2) = (w1 sin(a1/2) + w2 sin(a2/2)) /
    (w1 cos(a1/2) + w2 cos(a2/2)), w_i = exp(-|p - x_i|^2 / r^2) (Eq. 2, r from the paper)."""
    r = float(dict(_golden_rows("paper_constants.txt"))["radius"])
    axis = np.array([0.0, 0.0, 1.0])
    a1, a2 = math.radians(10.0), math.radians(-7.0)
    dq = np.stack([synth.motion_dual_quaternion(axis, a, np.zeros(3)) for a in (a1, a2)], axis=1)
    x = np.array([[0.10, 0.16], [0.05, 0.02], [0.0, 0.01]], np.float32)
    g = synth.Graph(x, dq.astype(np.float32), x, K=2, radius=r)
    v = oracle.View(oracle.Field.from_params(tiny_field(np.random.default_rng(0))),
                    graph=oracle.Graph.from_synth(g))
    pts = np.array([[0.12, 0.13, 0.11], [0.04, 0.03, 0.05], [0.0, 0.01, -0.01]], np.float32)
    vc = oracle.warp_points(v, pts)
    for i in range(3):
        p = pts[:, i].astype(np.float64)
        w = np.exp(-np.sum((p[:, None] - x.astype(np.float64)) ** 2, axis=0) / r ** 2)
        h = dq.astype(np.float32).astype(np.float64)
        phi = 2.0 * math.atan2(w[0] * h[3, 0] + w[1] * h[3, 1], w[0] * h[0, 0] + w[1] * h[0, 1])
        want = synth.rodrigues(axis, phi).T @ p
        np.testing.assert_allclose(vc[:, i], want, atol=1e-12)


def test_identity_motion_is_identity_warp(oracle):
    rng = np.random.default_rng(8)
    g = synth.make_graph(rng, 64, K=4)
    g.dq = np.tile(np.array([1, 0, 0, 0, 0, 0, 0, 0], np.float32)[:, None], (1, 64))
    v = _graph_view(oracle, g)
    pts = rng.uniform(-1, 1, size=(3, 300)).astype(np.float32)
    np.testing.assert_allclose(oracle.warp_points(v, pts), pts.astype(np.float64), atol=1e-14)


def test_quaternion_sign_flip_is_same_motion(oracle):
    rng = np.random.default_rng(10)
    g = synth.make_graph(rng, 64, K=4)
    v = _graph_view(oracle, g)
    pts = rng.uniform(-0.9, 0.9, size=(3, 300)).astype(np.float32)
    a = oracle.warp_points(v, pts)
    flip = rng.uniform(size=64) < 0.5
    g.dq[:, flip] *= -1.0
    b = oracle.warp_points(_graph_view(oracle, g), pts)
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_rigid_warp_round_trip(oracle):
    rng = np.random.default_rng(11)
    dq, R, t = synth.make_object_pose(rng)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
    f = oracle.Field.from_params(tiny_field(rng))
    v = oracle.View(f, rigid_dq=dq)
    pts = rng.uniform(-1, 1, size=(3, 200)).astype(np.float32)
    vc = oracle.warp_points(v, pts)
    np.testing.assert_allclose(vc, R.T @ (pts.astype(np.float64) - t[:, None]), atol=2e-6)
    back = oracle.dq_apply_points(dq, vc)
    np.testing.assert_allclose(back, pts.astype(np.float64), atol=1e-12)


# -------------------------------------------------------------------------- MLPs
def test_zero_weights_give_unit_density_half_grey(oracle):
    rng = np.random.default_rng(12)
    f = oracle.Field.from_params(tiny_field(rng, zero=True))
    out = oracle.mlp_points(f, rng.normal(size=(f.desc.mlp_in, 20)))
    np.testing.assert_array_equal(out[0], 1.0)
    np.testing.assert_array_equal(out[1:], 0.5)


def test_mlp_matches_numpy_matmul_chain(oracle):
    rng = np.random.default_rng(13)
    fp = synth.make_field(rng, synth.CFG1_FIELD)
    f = oracle.Field.from_params(fp)
    feat = rng.normal(size=(16, 64))
    Ws, off = [], 0
    for r, c in fp.desc.weight_shapes():
        Ws.append(fp.weights[off:off + r * c].astype(np.float64).reshape(r, c))
        off += r * c
    relu = lambda a: np.maximum(a, 0.0)
    o = Ws[2] @ relu(Ws[1] @ relu(Ws[0] @ feat))
    z = Ws[4] @ relu(Ws[3] @ o[1:])
    want = np.concatenate([np.exp(o[:1]), 1.0 / (1.0 + np.exp(-z))])
    np.testing.assert_allclose(oracle.mlp_points(f, feat), want, rtol=1e-12, atol=1e-14)


# -------------------------------------------------------------------- compositing
def test_constant_density_closed_form(oracle):
    rng = np.random.default_rng(14)
    fp = tiny_field(rng, zero=True)                      # sigma = 1, c = 1/2 everywhere
    g = synth.make_graph(rng, 16, K=4)
    v = oracle.View(oracle.Field.from_params(fp), graph=oracle.Graph.from_synth(g))
    rays = synth.pinhole_rays(12, 12, 50.0, (0.0, 0.0, 2.5))
    N = 48
    res = oracle.render(rays.o, rays.d, N, 1e-4, [v])
    hit, tn, dt, _, _ = oracle.ray_samples(rays.o, rays.d, N)
    h = hit.astype(bool)
    D = dt.astype(np.float64)
    Lr = N * D
    np.testing.assert_allclose(res.rgba[3], np.where(h, 1.0 - np.exp(-Lr), 0.0), atol=1e-13)
    np.testing.assert_allclose(res.rgba[:3], np.broadcast_to(0.5 * res.rgba[3], (3, res.rgba.shape[1])), atol=1e-13)
    # depth: sum_j e^{-j D} (1 - e^{-D}) (t_n + (j+1/2) D), arithmetico-geometric series
    q = np.exp(-D)
    s0 = (1 - q ** N) / (1 - np.where(h, q, 0.5))
    s1 = q * (1 - N * q ** (N - 1) + (N - 1) * q ** N) / (1 - np.where(h, q, 0.5)) ** 2
    want_D = (1 - q) * ((tn + 0.5 * D) * s0 + D * s1)
    # sample depths t_j are FP32 values (relative rounding <= 2^-24 each)
    np.testing.assert_allclose(res.depth[h], want_D[h], rtol=1e-7)
    assert np.all(res.n_used[0][h] == N)


def test_single_sample_alpha(oracle):
    rng = np.random.default_rng(15)
    fp = tiny_field(rng, zero=True)
    v = oracle.View(oracle.Field.from_params(fp), rigid_dq=np.array([1, 0, 0, 0, 0, 0, 0, 0], np.float32))
    rays = synth.pinhole_rays(6, 6, 50.0, (0.0, 0.0, 2.5))
    res = oracle.render(rays.o, rays.d, 1, 0.0, [v])
    hit, tn, dt, _, _ = oracle.ray_samples(rays.o, rays.d, 1)
    np.testing.assert_allclose(res.rgba[3], np.where(hit > 0, 1.0 - np.exp(-dt.astype(np.float64)), 0.0),
                               atol=1e-15)


def _dense_view(oracle, rng, scale=25.0):
    fp = synth.make_field(rng, synth.CFG1_FIELD)
    d = fp.desc
    off = d.hidden * d.mlp_in + d.hidden * d.hidden
    fp.weights[off:off + d.hidden] *= scale               # row 0 of W3 drives log-density
    g = synth.make_graph(rng, 64, K=4)
    return oracle.View(oracle.Field.from_params(fp), graph=oracle.Graph.from_synth(g))


def test_early_termination_bound(oracle):
    rng = np.random.default_rng(16)
    v = _dense_view(oracle, rng)
    rays = synth.pinhole_rays(24, 24, 50.0, (0.0, 0.0, 2.5))
    a = oracle.render(rays.o, rays.d, 64, 1e-4, [v])
    b = oracle.render(rays.o, rays.d, 64, 0.0, [v])
    assert np.any(a.n_used[0] < b.n_used[0])               # termination happened
    assert np.max(np.abs(a.rgba[:4] - b.rgba[:4])) <= 1e-4
    assert np.all(a.T_end[0][a.n_used[0] < b.n_used[0]] < 1e-4)


def test_identity_deformation_equals_static_field(oracle):
    rng = np.random.default_rng(17)
    fp = synth.make_field(rng, synth.CFG1_FIELD)
    f = oracle.Field.from_params(fp)
    g = synth.make_graph(rng, 64, K=4)
    g.dq = np.tile(np.array([1, 0, 0, 0, 0, 0, 0, 0], np.float32)[:, None], (1, 64))
    human = oracle.View(f, graph=oracle.Graph.from_synth(g))
    static = oracle.View(f, rigid_dq=np.array([1, 0, 0, 0, 0, 0, 0, 0], np.float32))
    rays = synth.pinhole_rays(16, 16, 50.0, (0.0, 0.0, 2.5))
    a = oracle.render(rays.o, rays.d, 32, 1e-4, [human])
    b = oracle.render(rays.o, rays.d, 32, 1e-4, [static])
    np.testing.assert_allclose(a.rgba, b.rgba, atol=1e-13)
    np.testing.assert_allclose(a.depth, b.depth, atol=1e-13)


def test_two_field_depth_composition(oracle):
    rng = np.random.default_rng(18)
    ident = np.array([1, 0, 0, 0, 0, 0, 0, 0], np.float32)
    dense = _dense_view(oracle, rng, scale=60.0)
    front = np.zeros(128 ** 3, bool)
    back = np.zeros(128 ** 3, bool)
    zc = -1.0 + (np.arange(128) + 0.5) / 64.0
    zz = np.repeat(zc, 128 * 128)                         # z of each cell, x fastest
    front[zz > 0.3] = True
    back[zz < -0.3] = True
    rays = synth.pinhole_rays(10, 10, 30.0, (0.0, 0.0, 2.5))
    human_front = oracle.View(dense.field, graph=dense.graph, occupancy=synth.pack_bits(front))
    obj = oracle.View(oracle.Field.from_params(synth.make_field(rng, synth.CFG1_FIELD)), rigid_dq=ident,
                      occupancy=synth.pack_bits(back))
    r = oracle.render(rays.o, rays.d, 64, 0.0, [human_front, obj])
    # nearer (human, z > 0.3) is laid over the farther; an opaque near layer hides the far one
    opaque = r.rgba_v[0][3] > 1.0 - 1e-9
    assert opaque.sum() > 10
    np.testing.assert_allclose(r.rgba[:, opaque], r.rgba_v[0][:, opaque], atol=1e-9)
    # swap depths: the object in front now hides the human behind it
    human_back = oracle.View(dense.field, graph=dense.graph, occupancy=synth.pack_bits(back))
    obj_front = oracle.View(obj.field, rigid_dq=ident, occupancy=synth.pack_bits(front))
    s = oracle.render(rays.o, rays.d, 64, 0.0, [human_back, obj_front])
    assert np.all(s.depth_v[1] * s.rgba_v[0][3] <= s.depth_v[0] * s.rgba_v[1][3] + 1e-12)
    transparent_front = s.rgba_v[1][3] < 1e-12
    np.testing.assert_allclose(s.rgba[:, transparent_front], s.rgba_v[0][:, transparent_front], atol=1e-12)
    # an empty field changes nothing
    empty = oracle.View(obj.field, rigid_dq=ident, occupancy=synth.pack_bits(np.zeros(128 ** 3, bool)))
    e = oracle.render(rays.o, rays.d, 64, 0.0, [human_front, empty])
    np.testing.assert_allclose(e.rgba, e.rgba_v[0], atol=0)


# ------------------------------------------------------------------- loss + grads
def test_huber_closed_form(oracle):
    assert abs(oracle.huber(0.05, 0.1) - 0.00125) < 1e-17
    assert abs(oracle.huber(0.3, 0.1) - 0.025) < 1e-17
    assert abs(oracle.huber(-0.3, 0.1) - 0.025) < 1e-17
    assert oracle.huber(0.0, 0.1) == 0.0


def _small_train(oracle, rng, n_rays=48, n_samples=24):
    fp = synth.make_field(rng, synth.FieldDesc(L=4, log2_T=10, F=2, N_min=4, growth=1.6))
    g = synth.make_graph(rng, 32, K=4)
    rays = synth.subset_rays(synth.ring_rays(4, 16, 16, 50.0, 2.5), rng.choice(4 * 256, n_rays, replace=False))
    tgt = synth.target_colours(rng, rays)
    f = oracle.Field.from_params(fp)
    v = oracle.View(f, graph=oracle.Graph.from_synth(g))
    return f, [oracle.TrainBatch(rays.o, rays.d, v, tgt)], n_samples


def test_gradients_match_central_differences(oracle):
    rng = np.random.default_rng(19)
    f, batches, S = _small_train(oracle, rng)
    _check_central_differences(oracle, rng, f, batches, S)


def _check_central_differences(oracle, rng, f, batches, S, **kw):
    loss, grads = oracle.train_loss_grad(batches, S, 0.0, 0.1, **kw)
    gt, gw = grads[id(f)]
    assert loss > 0
    hit = np.flatnonzero(np.abs(gt) > 1e-3 * np.abs(gt).max())
    pick_t = rng.choice(hit, 40, replace=False)
    pick_w = rng.choice(np.flatnonzero(np.abs(gw) > 1e-3 * np.abs(gw).max()), 24, replace=False)
    def fd(arr, i, h):
        old = arr[i]
        arr[i] = old + h
        lp, _ = oracle.train_loss_grad(batches, S, 0.0, 0.1, grads=False, **kw)
        arr[i] = old - h
        lm, _ = oracle.train_loss_grad(batches, S, 0.0, 0.1, grads=False, **kw)
        arr[i] = old
        return (lp - lm) / (2 * h)

    # central differences: round-off ~ eps * loss / h, truncation O(h^2).  A ReLU or
    # Huber kink within h of the parameter makes the two step sizes disagree; such
    # parameters are skipped (at most a few of the 64).
    eps = np.finfo(np.float64).eps
    skipped = 0
    for arr, picks, g in ((f.tables, pick_t, gt), (f.weights, pick_w, gw)):
        for i in picks:
            f1, f2 = fd(arr, i, 1e-5), fd(arr, i, 1e-6)
            if abs(f1 - f2) > 1e-4 * abs(f2) + 100 * eps * loss / 1e-6:
                skipped += 1
                continue
            assert abs(f2 - g[i]) <= 1e-5 * abs(g[i]) + 50 * eps * loss / 1e-6, (i, f2, g[i])
    assert skipped <= 4


# ------------------------------------------------------- the paper's losses (Sec. 4.4)
def _with_sensor(oracle, batches, rng, p_mask=0.7):
    """Copies of the batches with a random binary mask and sensor depths in the box's range."""
    out = []
    for b in batches:
        R = b.o.shape[1]
        mask = (rng.uniform(size=R) < p_mask).astype(np.float32)
        depth = rng.uniform(1.5, 3.5, size=R).astype(np.float32)
        out.append(oracle.TrainBatch(b.o, b.d, b.view, b.target, mask, depth))
    return out


def test_paper_loss_constant_density_closed_form(oracle):
    """sigma = 1, c = 1/2 everywhere: C_hat = A/2 per channel with A = 1 - exp(-(t_f - t_n)),
    D_hat the arithmetico-geometric series of the constant-density pin, so the loss is
    sum_r M_r (||A_r/2 - C_r||_2 + w |D_hat_r - D_r|) in closed form."""
    rng = np.random.default_rng(41)
    fp = tiny_field(rng, zero=True)
    g = synth.make_graph(rng, 16, K=4)
    v = oracle.View(oracle.Field.from_params(fp), graph=oracle.Graph.from_synth(g))
    rays = synth.pinhole_rays(10, 10, 50.0, (0.0, 0.0, 2.5))
    N, R = 40, rays.n
    hit, tn, dt, _, _ = oracle.ray_samples(rays.o, rays.d, N)
    h = hit.astype(bool)
    D = dt.astype(np.float64)
    A = np.where(h, 1.0 - np.exp(-N * D), 0.0)
    q = np.exp(-D)
    s0 = (1 - q ** N) / (1 - np.where(h, q, 0.5))
    s1 = q * (1 - N * q ** (N - 1) + (N - 1) * q ** N) / (1 - np.where(h, q, 0.5)) ** 2
    Dh = np.where(h, (1 - q) * ((tn + 0.5 * D) * s0 + D * s1), 0.0)
    target = np.stack([np.full(R, 0.1), np.full(R, 0.25), np.full(R, 0.6)]).astype(np.float32)
    mask = (rng.uniform(size=R) < 0.6).astype(np.float32)
    depth = rng.uniform(1.5, 3.5, size=R).astype(np.float32)
    w = 0.7
    b = oracle.TrainBatch(rays.o, rays.d, v, target, mask, depth)
    loss, _ = oracle.train_loss_grad([b], N, 0.0, 0.1, grads=False, loss="paper", depth_weight=w)
    e = 0.5 * A[None, :] - target.astype(np.float64)
    want = np.sum(mask * (np.sqrt(np.sum(e * e, axis=0)) + w * np.abs(Dh - depth)))
    assert abs(loss - want) <= 1e-9 * want


def test_paper_loss_gradients_match_central_differences(oracle):
    rng = np.random.default_rng(43)
    f, batches, S = _small_train(oracle, rng)
    batches = _with_sensor(oracle, batches, rng)
    _check_central_differences(oracle, rng, f, batches, S, loss="paper", depth_weight=0.5)


def test_paper_loss_mask_selects_rays(oracle):
    """M(r) in {0,1} selects rays: the masked loss and gradients equal those of the batch
    cut down to the rays with M = 1 (unmasked); an all-zero mask gives zero everything."""
    rng = np.random.default_rng(47)
    f, batches, S = _small_train(oracle, rng)
    (b,) = _with_sensor(oracle, batches, rng, p_mask=0.5)
    keep = b.mask > 0
    sub = oracle.TrainBatch(b.o[:, keep], b.d[:, keep], b.view, b.target[:, keep], None, b.depth[keep])
    l1, g1 = oracle.train_loss_grad([b], S, 0.0, 0.1, loss="paper", depth_weight=0.3)
    l2, g2 = oracle.train_loss_grad([sub], S, 0.0, 0.1, loss="paper", depth_weight=0.3)
    assert abs(l1 - l2) <= 1e-12 * l2
    for x, y in zip(g1[id(f)], g2[id(f)]):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-12 * np.abs(y).max())
    zero = oracle.TrainBatch(b.o, b.d, b.view, b.target, np.zeros_like(b.mask), b.depth)
    l0, g0 = oracle.train_loss_grad([zero], S, 0.0, 0.1, loss="paper")
    assert l0 == 0.0 and all(np.all(x == 0.0) for x in g0[id(f)])


# -------------------------------------------------------------------------- Adam
def test_adam_constant_gradient_steps_by_lr_sign(oracle):
    rng = np.random.default_rng(20)
    p0 = rng.normal(size=100)
    g = rng.normal(size=100)
    p, m, v = p0.copy(), np.zeros(100), np.zeros(100)
    for step in (1, 2, 3):
        oracle.adam(p, g, m, v, step, 1e-2, 0.9, 0.99, 1e-15)
        # with a constant gradient m_hat = g and v_hat = g^2 at every step
        np.testing.assert_allclose(p, p0 - step * 1e-2 * np.sign(g), atol=1e-12)
    np.testing.assert_allclose(m, (1 - 0.9 ** 3) * g, rtol=1e-12)
    np.testing.assert_allclose(v, (1 - 0.99 ** 3) * g * g, rtol=1e-12)
    # zero gradient from zero state: no motion
    q, m0, v0 = p0.copy(), np.zeros(100), np.zeros(100)
    oracle.adam(q, np.zeros(100), m0, v0, 1, 1e-2, 0.9, 0.99, 1e-15)
    np.testing.assert_array_equal(q, p0)


# ------------------------------------- look-up-table neighbour search (Sec. 4.2)
def test_lut_exp_error_bound(oracle):
    """The tables' exponential (Cody-Waite reduction + degree-6 Taylor) stays within
    4e-7 relative of exp on [-86, 0], is exact at 0, and is 0 below -86.6 (2^-125)."""
    x = np.linspace(-86.0, 0.0, 200001).astype(np.float32)
    got = oracle.lut_exp(x).astype(np.float64)
    want = np.exp(x.astype(np.float64))
    assert np.max(np.abs(got - want) / want) <= 4e-7
    assert oracle.lut_exp(np.zeros(1, np.float32))[0] == 1.0
    assert np.all(oracle.lut_exp(np.array([-87.0, -200.0, -1e30], np.float32)) == 0.0)


def _centres(G):
    c = ((np.arange(G, dtype=np.float32) + np.float32(0.5)) * np.float32(2.0 / G) - np.float32(1.0)).astype(np.float32)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()])       # voxel x + G (y + G z)


def test_lut_canonical_field_matches_lexsort(oracle):
    rng = np.random.default_rng(51)
    G, K = 8, 4
    x = rng.uniform(-0.9, 0.9, size=(3, 40)).astype(np.float32)
    canon = oracle.lut_canon_knn(x, K, G)
    c = _centres(G)
    for v in range(G ** 3):
        d = (c[:, v:v + 1] - x).astype(np.float32)
        key = ((d[0] * d[0]) + (d[1] * d[1])) + (d[2] * d[2])
        order = np.lexsort((np.arange(x.shape[1]), key))[:K]
        assert list(canon[v]) == list(order), v


def _identity_graph(g):
    g.dq[:] = np.array([1, 0, 0, 0, 0, 0, 0, 0], np.float32)[:, None]
    g.x_live[:] = g.x_canon
    return g


def test_lut_identity_motion_maps_each_voxel_to_itself(oracle):
    rng = np.random.default_rng(52)
    G = 16
    g = _identity_graph(synth.make_graph(rng, 48, K=4))
    canon = oracle.lut_canon_knn(g.x_canon, 4, G)
    live = oracle.lut_live_index(g.x_canon, g.dq, 4, g.radius, G, canon)
    assert np.array_equal(live, np.arange(G ** 3, dtype=np.uint32))


def test_lut_one_voxel_translation_shifts_the_index(oracle):
    """Every node translated by one voxel along +x: canonical voxel (x, y, z) lands in live
    voxel (x+1, y, z), so live[f] = f - 1 and the x = 0 plane stays empty."""
    rng = np.random.default_rng(53)
    G = 16
    g = synth.make_graph(rng, 48, K=4)
    g.dq[:] = np.array([1, 0, 0, 0, 0, 1.0 / G, 0, 0], np.float32)[:, None]   # q_d = 1/2 (0, t) q_r
    canon = oracle.lut_canon_knn(g.x_canon, 4, G)
    live = oracle.lut_live_index(g.x_canon, g.dq, 4, g.radius, G, canon).reshape(G, G, G)   # [z][y][x]
    f = np.arange(G ** 3, dtype=np.int64).reshape(G, G, G)
    assert np.all(live[:, :, 0] == oracle.LUT_EMPTY)
    assert np.array_equal(live[:, :, 1:].astype(np.int64), f[:, :, 1:] - 1)


def _fp64_forward(oracle, g, ids, c):
    """FP64 forward warp of Eq. 2 from scratch: weights exp(-|c - x_i|^2 / r^2) over the
    given canonical neighbours, sign alignment, blend, then the oracle's pinned SE3 apply
    (which normalises)."""
    x = g.x_canon.astype(np.float64)
    q = g.dq.astype(np.float64)
    n = c.shape[1]
    b = np.zeros((8, n))
    d2 = np.stack([np.sum((c.astype(np.float64) - x[:, ids[:, k]]) ** 2, axis=0) for k in range(ids.shape[1])])
    ref = q[:4, ids[:, 0]]
    for k in range(ids.shape[1]):
        w = np.exp(-(d2[k] - d2[0]) / g.radius ** 2)
        s = np.where(np.sum(q[:4, ids[:, k]] * ref, axis=0) < 0, -1.0, 1.0)
        b += s * w * q[:, ids[:, k]]
    c64 = c.astype(np.float64)
    return np.concatenate([oracle.dq_apply_points(b[:, i], c64[:, i:i + 1]) for i in range(n)], axis=1)


def test_lut_forward_warp_matches_fp64(oracle):
    rng = np.random.default_rng(54)
    G = 16
    g = synth.make_graph(rng, 64, K=4)
    canon = oracle.lut_canon_knn(g.x_canon, 4, G)
    c = _centres(G)
    got = oracle.lut_forward_points(g.x_canon, g.dq, 4, g.radius, c, canon.astype(np.int32))
    want = _fp64_forward(oracle, g, canon.astype(np.int64), c)
    assert np.max(np.abs(got - want)) <= 2e-6


def test_lut_live_index_brute_force(oracle):
    """Each live voxel holds the smallest canonical voxel whose FP64 forward warp lands in
    it, and empty voxels receive none; voxels warped to within 1e-5 of a cell face (where
    single and double precision may pick different cells) are exempt."""
    rng = np.random.default_rng(55)
    G = 12
    g = synth.make_graph(rng, 48, K=4)
    canon = oracle.lut_canon_knn(g.x_canon, 4, G)
    live = oracle.lut_live_index(g.x_canon, g.dq, 4, g.radius, G, canon).astype(np.int64)
    pos = _fp64_forward(oracle, g, canon.astype(np.int64), _centres(G))
    q = (pos + 1.0) * 0.5 * G
    fl = np.floor(q)
    ambiguous = np.any(np.minimum(q - fl, fl + 1 - q) < 1e-5 * G, axis=0)
    inside = np.all((fl >= 0) & (fl < G), axis=0)
    cell = (fl[0] + G * (fl[1] + G * fl[2])).astype(np.int64)
    assert ambiguous.sum() < 0.01 * G ** 3
    want = np.full(G ** 3, -1, np.int64)
    for k in np.flatnonzero(inside & ~ambiguous)[::-1]:     # descending: the smallest k wins
        want[cell[k]] = k
    empty = live == oracle.LUT_EMPTY
    for f in range(G ** 3):
        if want[f] >= 0:
            assert not empty[f] and (live[f] == want[f] or (live[f] < want[f] and ambiguous[live[f]])), f
        elif not empty[f]:
            assert ambiguous[live[f]], f
    assert empty.sum() > 0 and (~empty).sum() > 0.5 * G ** 3


def test_lut_neighbours_and_warp(oracle):
    """Neighbour sets from the tables: under identity motion they are the canonical field's
    entry of the point's voxel; under motion, where a set equals the exact K nearest the
    warp is identical to the exact warp, and points in empty live voxels use the exact set."""
    rng = np.random.default_rng(56)
    G = 32
    gi = _identity_graph(synth.make_graph(rng, 64, K=4))
    canon_i = oracle.lut_canon_knn(gi.x_canon, 4, G)
    live_i = oracle.lut_live_index(gi.x_canon, gi.dq, 4, gi.radius, G, canon_i)
    p = rng.uniform(-0.95, 0.95, size=(3, 3000)).astype(np.float32)
    ids, from_lut = oracle.neighbour_points(oracle.Graph.from_synth(gi, (G, canon_i, live_i)), p)
    assert from_lut.all()
    vox = np.floor(((p + np.float32(1)) * np.float32(0.5)) * np.float32(G)).astype(np.int64)
    v = vox[0] + G * (vox[1] + G * vox[2])
    assert np.array_equal(np.sort(ids, axis=0), np.sort(canon_i[v].T.astype(np.int32), axis=0))

    g = synth.make_graph(rng, 64, K=4)
    canon = oracle.lut_canon_knn(g.x_canon, 4, G)
    live = oracle.lut_live_index(g.x_canon, g.dq, 4, g.radius, G, canon)
    lut_graph = oracle.Graph.from_synth(g, (G, canon, live))
    exact_graph = oracle.Graph.from_synth(g)
    near = g.x_live[:, rng.integers(0, 64, 3000)] + rng.normal(scale=0.05, size=(3, 3000)).astype(np.float32)
    ids_l, from_lut = oracle.neighbour_points(lut_graph, near)
    ids_e, _ = oracle.knn_points(exact_graph, near)
    f = oracle.Field.from_params(tiny_field(rng))
    vc_l = oracle.warp_points(oracle.View(f, graph=lut_graph), near)
    vc_e = oracle.warp_points(oracle.View(f, graph=exact_graph), near)
    same = np.all(ids_l == ids_e, axis=0)
    assert 0.3 < same.mean() < 1.0                 # an approximation that is mostly right
    assert np.array_equal(vc_l[:, same], vc_e[:, same])
    assert np.array_equal(ids_l[:, ~from_lut], ids_e[:, ~from_lut])
    holes = live == oracle.LUT_EMPTY
    vox = np.floor(((np.clip(near, -1, 1) + np.float32(1)) * np.float32(0.5)) * np.float32(G)).astype(np.int64)
    vox = np.clip(vox, 0, G - 1)
    assert np.array_equal(~from_lut, holes[vox[0] + G * (vox[1] + G * vox[2])])


# ----------------------------------- joint compositing and occupancy maintenance
def test_joint_compositing_with_an_empty_field_is_the_single_render(oracle):
    rng = np.random.default_rng(71)
    w = synth.two_field_render(width=24, height=24, n_samples=48, n_nodes=256)
    hv = oracle.View.from_synth(w.views[0])
    ov = oracle.View.from_synth(w.views[1])
    empty = oracle.View(ov.field, rigid_dq=w.views[1].rigid_dq, occupancy=np.zeros(128 ** 3 // 32, np.uint32))
    rgba, depth, n_used = oracle.render_joint(w.rays.o, w.rays.d, w.n_samples, w.t_eps, hv, empty)
    ref = oracle.render(w.rays.o, w.rays.d, w.n_samples, w.t_eps, [hv])
    assert ref.rgba[3].max() > 0.2
    np.testing.assert_allclose(rgba, ref.rgba, rtol=0, atol=1e-14)
    np.testing.assert_allclose(depth, ref.depth, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(n_used, ref.n_used[0])


def test_joint_compositing_two_constant_fields_closed_form(oracle):
    """sigma = 1 and c = 1/2 in both fields, no occupancy: the mixture has sigma = 2 and
    c = 1/2, so A = 1 - exp(-2 (t_f - t_n)) and C = A/2 per channel."""
    rng = np.random.default_rng(72)
    f1 = oracle.Field.from_params(tiny_field(rng, zero=True))
    f2 = oracle.Field.from_params(tiny_field(rng, zero=True))
    g = synth.make_graph(rng, 16, K=4)
    dq, _, _ = synth.make_object_pose(rng)
    hv = oracle.View(f1, graph=oracle.Graph.from_synth(g))
    ov = oracle.View(f2, rigid_dq=dq)
    rays = synth.pinhole_rays(10, 10, 50.0, (0.0, 0.0, 2.5))
    N = 40
    rgba, depth, n_used = oracle.render_joint(rays.o, rays.d, N, 0.0, hv, ov)
    hit, tn, dt, _, _ = oracle.ray_samples(rays.o, rays.d, N)
    h = hit.astype(bool)
    A = np.where(h, 1.0 - np.exp(-2.0 * N * dt.astype(np.float64)), 0.0)
    np.testing.assert_allclose(rgba[3], A, rtol=0, atol=1e-13)
    np.testing.assert_allclose(rgba[:3], np.broadcast_to(0.5 * A, (3, rays.n)), rtol=0, atol=1e-13)
    assert np.all(n_used[h] == N) and np.all(n_used[~h] == 0)


def _affine_density_field(oracle, a0, a):
    """A field with sigma(x) = exp(max(a0 + a . q, 0)) exactly, q = clamp((x+1)/2, 0, 1) N_0:
    level 0 (dense) holds the affine function of the vertex coordinates in feature 0, and
    the first layers pass feature 0 through (W1[0][0] = W2[0][0] = W3[0][0] = 1, all other
    weights 0, so c = 1/2)."""
    rng = np.random.default_rng(0)
    fp = tiny_field(rng, zero=True)
    d = fp.desc
    tables = np.zeros((d.L, d.T, d.F))
    res = oracle.level_res(d.N_min, d.growth, 0)
    assert oracle.level_dense(res, d.log2_T)
    for z in range(res + 1):
        for y in range(res + 1):
            for x in range(res + 1):
                tables[0, oracle.vertex_index(res, d.log2_T, x, y, z), 0] = a0 + np.dot(a, [x, y, z])
    weights = np.zeros(d.n_weight_params())
    shapes = d.weight_shapes()
    off = 0
    for k, (r, c) in enumerate(shapes):
        if k < 3:
            weights[off] = 1.0                            # W_k[0][0]
        off += r * c
    return oracle.Field(d, tables, weights), res


def test_occupancy_update_affine_density(oracle):
    a0, a = -1.0, np.array([0.5, 0.2, -0.3])
    f, res = _affine_density_field(oracle, a0, a)
    ident = np.array([1, 0, 0, 0, 0, 0, 0, 0], np.float32)
    v = oracle.View(f, rigid_dq=ident)
    G = oracle.OCC_RES
    c = (np.arange(G, dtype=np.float32) + np.float32(0.5)) * np.float32(2.0 / G) - np.float32(1.0)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    q = np.stack([x.ravel(), y.ravel(), z.ravel()]).astype(np.float64)
    q = np.clip((q + 1.0) * 0.5, 0.0, 1.0) * res
    want = np.exp(np.maximum(a0 + a @ q, 0.0))
    thr = 1.2
    dens, bits = oracle.occupancy_update(v, 0.9, thr)
    np.testing.assert_allclose(dens, want, rtol=1e-12)
    np.testing.assert_array_equal(bits, synth.pack_bits(want > thr))
    assert 0 < (want > thr).mean() < 1
    # a second update with a constant-density field (sigma = 1) and decay 1/2
    zero = oracle.View(oracle.Field.from_params(tiny_field(np.random.default_rng(1), zero=True)), rigid_dq=ident)
    dens2, bits2 = oracle.occupancy_update(zero, 0.5, thr, dens.copy())
    np.testing.assert_allclose(dens2, np.maximum(0.5 * want, 1.0), rtol=1e-12)
    np.testing.assert_array_equal(bits2, synth.pack_bits(np.maximum(0.5 * want, 1.0) > thr))


# ------------------------------------------- pose-conditioned deformation net (Sec. 4.2)
TINY_DEFORM = synth.DeformDesc(L=2, log2_T=10, F=2, N_min=2, growth=1.5, pose_dim=6, hidden=16, n_hidden=3)


def test_deform_forward_matches_numpy_chain(oracle):
    rng = np.random.default_rng(91)
    dp = synth.make_deform(rng, TINY_DEFORM, out_scale=1.0)
    d = dp.desc
    pose = synth.make_pose(rng, d.pose_dim)
    vt = rng.uniform(-0.9, 0.9, size=(3, 50))
    got = oracle.deform_points(oracle.Deform.from_params(dp), pose, vt)
    enc = oracle.Field(synth.FieldDesc(L=d.L, log2_T=d.log2_T, F=d.F, N_min=d.N_min, growth=d.growth),
                       dp.tables, np.zeros(1))
    feat = oracle.encode_points(enc, vt)
    x = np.concatenate([feat, np.repeat(pose.astype(np.float64)[:, None], vt.shape[1], axis=1)])
    W, off = [], 0
    for r, c in d.weight_shapes():
        W.append(dp.weights[off:off + r * c].astype(np.float64).reshape(r, c))
        off += r * c
    h = x
    for k in range(d.n_hidden):
        h = np.maximum(W[k] @ h, 0.0)
    np.testing.assert_allclose(got, W[-1] @ h, rtol=1e-12, atol=1e-14)
    assert np.abs(got).max() > 1e-3


def test_deform_zero_output_layer_leaves_the_warp(oracle):
    rng = np.random.default_rng(92)
    dp = synth.make_deform(rng, TINY_DEFORM, out_scale=0.0)
    g = synth.make_graph(rng, 32, K=4)
    f = oracle.Field.from_params(tiny_field(rng))
    p = rng.uniform(-0.9, 0.9, size=(3, 300)).astype(np.float32)
    with_net = oracle.View(f, graph=oracle.Graph.from_synth(g), deform=oracle.Deform.from_params(dp),
                           pose=synth.make_pose(rng, TINY_DEFORM.pose_dim))
    plain = oracle.View(f, graph=oracle.Graph.from_synth(g))
    np.testing.assert_array_equal(oracle.warp_points(with_net, p), oracle.warp_points(plain, p))


def test_encode_point_derivative_affine_closed_form(oracle):
    """Dense levels holding an affine function of the vertex coordinates: d feat / d x_a =
    coef_a N_l / 2 inside the box and 0 along an axis clamped outside it."""
    rng = np.random.default_rng(93)
    fp = tiny_field(rng, L=2, log2_T=10, F=2, N_min=2, growth=1.5)
    d = fp.desc
    tables = np.zeros((d.L, d.T, d.F))
    coef = rng.normal(size=(d.L, d.F, 4))
    for l in range(d.L):
        res = oracle.level_res(d.N_min, d.growth, l)
        for z in range(res + 1):
            for y in range(res + 1):
                for x in range(res + 1):
                    tables[l, oracle.vertex_index(res, d.log2_T, x, y, z)] = coef[l, :, 0] + coef[l, :, 1:] @ [x, y, z]
    f = oracle.Field(d, tables, fp.weights)
    pts = rng.uniform(-0.95, 0.95, size=(3, 100))
    pts[1, :10] = 1.3                                   # y clamped for the first ten points
    dfeat = rng.normal(size=(d.L * d.F, 100))
    dx = oracle.encode_dx_points(f, pts, dfeat)
    want = np.zeros((3, 100))
    for l in range(d.L):
        res = oracle.level_res(d.N_min, d.growth, l)
        for fi in range(d.F):
            want += np.outer(coef[l, fi, 1:], dfeat[l * d.F + fi]) * 0.5 * res
    want[1, :10] = 0.0
    np.testing.assert_allclose(dx, want, rtol=1e-11, atol=1e-11)


def test_encode_point_derivative_central_differences(oracle):
    rng = np.random.default_rng(94)
    fp = synth.make_field(rng, synth.FieldDesc(L=4, log2_T=10, F=2, N_min=4, growth=1.6))
    f = oracle.Field.from_params(fp)
    pts = rng.uniform(-0.9, 0.9, size=(3, 60))
    dfeat = rng.normal(size=(8, 60))
    dx = oracle.encode_dx_points(f, pts, dfeat)
    h = 1e-7
    checked = 0
    for a in range(3):
        e = np.zeros((3, 1))
        e[a] = h
        fp_ = np.sum(dfeat * oracle.encode_points(f, pts + e), axis=0)
        fm_ = np.sum(dfeat * oracle.encode_points(f, pts - e), axis=0)
        fd = (fp_ - fm_) / (2 * h)
        # a cell face within h of a point makes the encoding's derivative jump; skip those
        ok = np.ones(60, bool)
        for l in range(4):
            res = oracle.level_res(4, 1.6, l)
            q = (pts[a] + 1.0) * 0.5 * res
            ok &= np.abs(q - np.round(q)) > 1e-4
        np.testing.assert_allclose(dx[a, ok], fd[ok], rtol=1e-6, atol=1e-6)
        checked += ok.sum()
    assert checked > 120


def test_deform_gradients_match_central_differences(oracle):
    """Training through v_c = v_t + delta v: the analytic gradients of the net's tables and of
    every weight layer, and of the field's own parameters, against central differences."""
    rng = np.random.default_rng(95)
    fp = synth.make_field(rng, synth.FieldDesc(L=4, log2_T=10, F=2, N_min=4, growth=1.6))
    dp = synth.make_deform(rng, TINY_DEFORM, out_scale=0.5)
    g = synth.make_graph(rng, 32, K=4)
    rays = synth.subset_rays(synth.ring_rays(4, 16, 16, 50.0, 2.5), rng.choice(4 * 256, 48, replace=False))
    f = oracle.Field.from_params(fp)
    dn = oracle.Deform.from_params(dp)
    v = oracle.View(f, graph=oracle.Graph.from_synth(g), deform=dn, pose=synth.make_pose(rng, TINY_DEFORM.pose_dim))
    batches = [oracle.TrainBatch(rays.o, rays.d, v, synth.target_colours(rng, rays))]
    S = 24
    loss, grads = oracle.train_loss_grad(batches, S, 0.0, 0.1)
    dgt, dgw = grads[id(dn)]
    gt, gw = grads[id(f)]
    assert np.abs(dgt).max() > 0 and np.abs(dgw).max() > 0

    def fd(arr, i, h):
        old = arr[i]
        arr[i] = old + h
        lp, _ = oracle.train_loss_grad(batches, S, 0.0, 0.1, grads=False)
        arr[i] = old - h
        lm, _ = oracle.train_loss_grad(batches, S, 0.0, 0.1, grads=False)
        arr[i] = old
        return (lp - lm) / (2 * h)

    eps = np.finfo(np.float64).eps
    offs = np.cumsum([0] + [r * c for r, c in TINY_DEFORM.weight_shapes()])
    picks = [(dn.tables, i, dgt) for i in rng.choice(np.flatnonzero(np.abs(dgt) > 1e-3 * np.abs(dgt).max()), 16,
                                                      replace=False)]
    for k in range(len(offs) - 1):                       # every layer of the net
        seg = np.arange(offs[k], offs[k + 1])
        seg = seg[np.abs(dgw[seg]) > 1e-3 * np.abs(dgw[seg]).max()]
        picks += [(dn.weights, i, dgw) for i in rng.choice(seg, 6, replace=False)]
    picks += [(f.tables, i, gt) for i in rng.choice(np.flatnonzero(np.abs(gt) > 1e-3 * np.abs(gt).max()), 8,
                                                     replace=False)]
    picks += [(f.weights, i, gw) for i in rng.choice(np.flatnonzero(np.abs(gw) > 1e-3 * np.abs(gw).max()), 8,
                                                      replace=False)]
    skipped = 0
    for arr, i, g_ in picks:
        f1, f2 = fd(arr, i, 1e-5), fd(arr, i, 1e-6)
        if abs(f1 - f2) > 1e-4 * abs(f2) + 100 * eps * loss / 1e-6:
            skipped += 1
            continue
        assert abs(f2 - g_[i]) <= 1e-5 * abs(g_[i]) + 50 * eps * loss / 1e-6, (i, f2, g_[i])
    assert skipped <= 5, skipped
