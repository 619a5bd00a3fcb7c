"""Look-up-table neighbour search (Sec. 4.2, "On-the-fly Radiance Fields") on the GPU
against the oracle: both tables bit for bit where the oracle builds them whole, sampled
rows and entries at the paper's 512^3, neighbour ids bit for bit, and the warp, render
and gradients through the tables within the FP32 tolerances."""
import numpy as np
import pytest

from paper_2304_03184_b300 import synth

pytestmark = pytest.mark.gpu

COLOUR_TOL = 1e-5
GRAD_RTOL_WARP = 1e-2


@pytest.fixture(scope="module")
def env(oracle):
    import torch
    from paper_2304_03184_b300 import build
    build.build()
    import paper_2304_03184_b300 as invr
    assert torch.cuda.is_available()
    ctx = invr.Context(0)
    yield invr, ctx, oracle
    torch.cuda.synchronize()


def cu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def as_u16(a):
    return np.asarray(a).astype(np.int64) & 0xFFFF


def as_u32(a):
    return np.asarray(a).astype(np.int64) & 0xFFFFFFFF


def gpu_graph(invr, ctx, g, G=None):
    graph = invr.Graph(ctx, g.x_canon.shape[1], g.K, g.radius, 1, cu(g.x_canon))
    graph.set_pose(0, cu(g.dq), cu(g.x_live))
    if G:
        graph.enable_lut(G)
    return graph


def oracle_tables(oracle, g, G):
    canon = oracle.lut_canon_knn(g.x_canon, g.K, G)
    live = oracle.lut_live_index(g.x_canon, g.dq, g.K, g.radius, G, canon)
    return canon, live


@pytest.mark.parametrize("n_nodes,K,G", [(64, 4, 32), (2048, 4, 64), (4096, 8, 32)])
def test_lut_tables_bit_exact(env, n_nodes, K, G):
    invr, ctx, oracle = env
    rng = np.random.default_rng(61)
    g = synth.make_graph(rng, n_nodes, K=K)
    graph = gpu_graph(invr, ctx, g, G)
    canon_g, live_g = (host(x) for x in graph.get_lut(0))
    canon_o, live_o = oracle_tables(oracle, g, G)
    np.testing.assert_array_equal(as_u16(canon_g), canon_o.astype(np.int64))
    np.testing.assert_array_equal(as_u32(live_g), live_o.astype(np.int64))
    empty = live_o == oracle.LUT_EMPTY
    assert 0 < empty.sum() < G ** 3


def test_lut_follows_set_pose(env):
    """Tables enabled before the pose is set, then a new pose: the live field follows."""
    invr, ctx, oracle = env
    rng = np.random.default_rng(62)
    g = synth.make_graph(rng, 512, K=4)
    graph = invr.Graph(ctx, 512, 4, g.radius, 2, cu(g.x_canon))
    graph.enable_lut(32)
    graph.set_pose(1, cu(g.dq), cu(g.x_live))
    g2 = synth.repose_graph(rng, g)
    graph.set_pose(1, cu(g2.dq), cu(g2.x_live))
    _, live_g = graph.get_lut(1)
    _, live_o = oracle_tables(oracle, g2, 32)
    np.testing.assert_array_equal(as_u32(host(live_g)), live_o.astype(np.int64))
    with pytest.raises(invr.InvrError):
        graph.get_lut(0)                                  # frame 0 was never posed
    with pytest.raises(invr.InvrError):
        graph.enable_lut(48)                              # not a power of two
    graph.disable_lut()
    ctx.sync()


def _probe(rng, g, n=4000):
    near = g.x_live[:, rng.integers(0, g.x_live.shape[1], n)] + rng.normal(scale=0.05, size=(3, n))
    far = rng.uniform(-1.0, 1.0, size=(3, 500))
    return np.concatenate([near, far], axis=1).astype(np.float32)


def test_lut_neighbours_and_warp_match_oracle(env):
    invr, ctx, oracle = env
    rng = np.random.default_rng(63)
    G = 64
    g = synth.make_graph(rng, 2048, K=4)
    graph = gpu_graph(invr, ctx, g, G)
    field = synth.make_field(rng, synth.CFG1_FIELD)
    view = invr.View(invr.Field.from_synth(ctx, field), graph)
    p = _probe(rng, g)
    vc, ids = invr.warp_points(ctx, view, cu(p), with_ids=True)
    og = oracle.Graph.from_synth(g, (G,) + oracle_tables(oracle, g, G))
    oids, from_lut = oracle.neighbour_points(og, p)
    np.testing.assert_array_equal(host(ids), oids)
    ov = oracle.View(oracle.Field.from_params(field), graph=og)
    np.testing.assert_allclose(host(vc), oracle.warp_points(ov, p), rtol=0, atol=2e-6)
    exact, _ = oracle.knn_points(oracle.Graph.from_synth(g), p)
    # the synthetic motions rotate each node independently about the origin, so the live
    # field tears: a third of these probe points fall in holes and use the exact search
    agree = np.all(oids == exact, axis=0).mean()
    assert from_lut.mean() > 0.5 and 0.3 < agree < 1.0, (from_lut.mean(), agree)


def test_lut_render_and_gradients_match_oracle(env):
    invr, ctx, oracle = env
    G = 64
    tw = synth.train_step_workload(seed=64, n_rays=1024)
    b = tw.batches[0]
    g = b.view.graph
    graph = gpu_graph(invr, ctx, g, G)
    fp = tw.fields[0]
    field = invr.Field.from_synth(ctx, fp)
    occ = cu(b.view.occupancy)
    view = invr.View(field, graph, 0, None, occ)
    og = oracle.Graph.from_synth(g, (G,) + oracle_tables(oracle, g, G))
    of = oracle.Field.from_params(fp)
    ov = oracle.View(of, graph=og, occupancy=b.view.occupancy)
    o, d = cu(b.rays.o), cu(b.rays.d)
    rgba, depth = invr.render_rays(ctx, o, d, tw.n_samples, tw.t_eps, [view])
    ref = oracle.render(b.rays.o, b.rays.d, tw.n_samples, tw.t_eps, [ov])
    assert ref.rgba[3].max() > 0.1
    np.testing.assert_allclose(host(rgba), ref.rgba, rtol=0, atol=COLOUR_TOL)
    tb = invr.TrainBatches([(o, d, view, cu(b.target))], tw.n_samples, tw.t_eps, tw.huber_delta)
    loss = invr.forward_train(ctx, tb)
    invr.backward(ctx, tb)
    ctx.sync()
    oloss, ograds = oracle.train_loss_grad([oracle.TrainBatch(b.rays.o, b.rays.d, ov, b.target)], tw.n_samples,
                                           tw.t_eps, tw.huber_delta)
    assert abs(float(host(loss)[0]) - oloss) <= 1e-5 * oloss
    gt, gw = (host(x) for x in field.get_grads())
    ogt, ogw = ograds[id(of)]
    for got, want, what in ((gt, ogt, "tables"), (gw, ogw, "weights")):
        assert np.linalg.norm(got - want) <= GRAD_RTOL_WARP * np.linalg.norm(want), what


def test_lut_full_size_sampled(env):
    """The paper's 512^3 tables for the 2048-node graph: sampled canonical rows equal the
    oracle's brute-force K nearest of the voxel centre; sampled live entries hold a voxel
    whose forward warp (the oracle's single-precision recipe) lands in that live voxel; the
    neighbour ids of sampled live points follow from the two tables (or, in holes, equal
    the exact K nearest)."""
    invr, ctx, oracle = env
    import torch
    rng = np.random.default_rng(65)
    G = 512
    g = synth.make_graph(rng, 2048, K=4)
    graph = gpu_graph(invr, ctx, g, G)
    canon_d, live_d = graph.get_lut(0)
    ctx.sync()

    def centres(v):
        v = np.asarray(v, np.int64)
        ijk = np.stack([v % G, (v // G) % G, v // (G * G)])
        return ((ijk.astype(np.float32) + np.float32(0.5)) * np.float32(2.0 / G) - np.float32(1.0)).astype(np.float32)

    vox = rng.integers(0, G ** 3, 3000)
    rows = as_u16(host(canon_d[cu(vox)]))
    canon_graph = oracle.Graph(g.x_canon, g.dq, g.K, g.radius)
    want, _ = oracle.knn_points(canon_graph, centres(vox))
    np.testing.assert_array_equal(rows, want.T.astype(np.int64))

    filled = torch.nonzero(live_d != -1).flatten()
    assert 0.5 * G ** 3 < filled.numel() < G ** 3
    f = host(filled[cu(rng.integers(0, filled.numel(), 3000))]).astype(np.int64)
    k = as_u32(host(live_d[cu(f)]))
    krows = as_u16(host(canon_d[cu(k)]))
    q = oracle.lut_forward_points(g.x_canon, g.dq, g.K, g.radius, centres(k), krows.astype(np.int32))
    cell = np.floor(((q + np.float32(1)) * np.float32(0.5)) * np.float32(G)).astype(np.int64)
    np.testing.assert_array_equal(cell[0] + G * (cell[1] + G * cell[2]), f)

    field = synth.make_field(rng, synth.CFG1_FIELD)
    view = invr.View(invr.Field.from_synth(ctx, field), graph)
    p = _probe(rng, g)
    _, ids = invr.warp_points(ctx, view, cu(p), with_ids=True)
    ids = host(ids)
    pv = np.clip(np.floor(((p + np.float32(1)) * np.float32(0.5)) * np.float32(G)).astype(np.int64), 0, G - 1)
    pf = pv[0] + G * (pv[1] + G * pv[2])
    kp = as_u32(host(live_d[cu(pf)]))
    hole = kp == 0xFFFFFFFF
    exact, _ = oracle.knn_points(oracle.Graph.from_synth(g), p)
    np.testing.assert_array_equal(ids[:, hole], exact[:, hole])
    cand = as_u16(host(canon_d[cu(np.where(hole, 0, kp))]))          # [n][K]
    x = g.x_live
    for i in np.flatnonzero(~hole):
        d = (p[:, i:i + 1] - x[:, cand[i]]).astype(np.float32)
        key = ((d[0] * d[0]) + (d[1] * d[1])) + d[2] * d[2]
        order = np.lexsort((cand[i], key))
        np.testing.assert_array_equal(ids[:, i], cand[i][order])
    graph.disable_lut()
    ctx.sync()
