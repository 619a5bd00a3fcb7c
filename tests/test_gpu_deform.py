"""Pose-conditioned deformation net (Sec. 4.2) on the GPU against the oracle: renders,
training loss and gradients of the field and of the net's tables and weights, the Adam
step, and the zero-output identity."""
import numpy as np
import pytest

from paper_2304_03184_b300 import synth

pytestmark = pytest.mark.gpu

COLOUR_TOL = 1e-5
GRAD_RTOL = 1e-3        # identity motion: both sides start the net from the same v_t
GRAD_RTOL_WARP = 1e-2   # through the FP32 warp (see test_gpu_parity)


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


MIXED_COLOUR_TOL = 2e-3


class Human:
    """A human view with a deformation net on both sides."""

    def __init__(self, invr, ctx, oracle, sv, dp, pose, prec=0, field=None, ofield=None, net=None, onet=None,
                 net_prec=0):
        self.field = field or invr.Field.from_synth(ctx, sv.field, prec)
        g = sv.graph
        self.graph = invr.Graph(ctx, g.x_canon.shape[1], g.K, g.radius, 1, cu(g.x_canon))
        self.graph.set_pose(0, cu(g.dq), cu(g.x_live))
        self.occ = cu(sv.occupancy) if sv.occupancy is not None else None
        self.net = net or invr.Deform.from_synth(ctx, dp, net_prec)
        self.pose = cu(pose)
        self.view = invr.View(self.field, self.graph, 0, None, self.occ, self.net, self.pose)
        self.onet = onet or oracle.Deform.from_params(dp)
        self.oview = oracle.View(ofield or oracle.Field.from_params(sv.field), graph=oracle.Graph.from_synth(g),
                                 occupancy=sv.occupancy, deform=self.onet, pose=pose)


def _render_workload(rng):
    w = synth.two_field_render(width=64, height=64, n_samples=96)
    return w, synth.make_deform(rng), synth.make_pose(rng)


def test_deform_render_matches_oracle(env):
    invr, ctx, oracle = env
    rng = np.random.default_rng(101)
    w, dp, pose = _render_workload(rng)
    hum = Human(invr, ctx, oracle, w.views[0], dp, pose)
    rgba, depth = invr.render_rays(ctx, cu(w.rays.o), cu(w.rays.d), w.n_samples, w.t_eps, [hum.view])
    ctx.sync()
    ref = oracle.render(w.rays.o, w.rays.d, w.n_samples, w.t_eps, [hum.oview])
    assert ref.rgba[3].max() > 0.3
    np.testing.assert_allclose(host(rgba), ref.rgba, rtol=0, atol=COLOUR_TOL)
    # the net changes the image (|delta v| ~ 1e-2)
    plain = oracle.render(w.rays.o, w.rays.d, w.n_samples, w.t_eps, [oracle.View.from_synth(w.views[0])])
    assert np.abs(plain.rgba - ref.rgba).max() > 1e-3


@pytest.mark.parametrize("field_prec,net_prec", [("fp32", "fp16"), ("bf16", "fp16"), ("bf16", "bf16")])
def test_deform_tensor_core_forward_matches_oracle(env, field_prec, net_prec):
    """The net's forward on the tensor cores (FP16 or BF16 split operands, FP32 accumulation):
    renders within 1e-5 with an FP32 field, within the mixed-precision colour tolerance with a
    BF16 field."""
    invr, ctx, oracle = env
    rng = np.random.default_rng(107)
    w, dp, pose = _render_workload(rng)
    code = invr.INVR_MLP_BF16 if field_prec == "bf16" else invr.INVR_FP32
    ncode = invr.INVR_MLP_BF16 if net_prec == "bf16" else invr.INVR_MLP_FP16
    hum = Human(invr, ctx, oracle, w.views[0], dp, pose, prec=code, net_prec=ncode)
    rgba, _ = invr.render_rays(ctx, cu(w.rays.o), cu(w.rays.d), w.n_samples, w.t_eps, [hum.view])
    ctx.sync()
    ref = oracle.render(w.rays.o, w.rays.d, w.n_samples, w.t_eps, [hum.oview])
    # with an FP32 field the split-product net is as exact as the FP32 one (measured 9e-7)
    tol = COLOUR_TOL if field_prec == "fp32" else MIXED_COLOUR_TOL
    np.testing.assert_allclose(host(rgba), ref.rgba, rtol=0, atol=tol)


# The net on the tensor cores, trained.  Its forward forms every product from 16-bit values
# plus the 16-bit remainders of their rounding (activations in tensor memory, weights in shared
# memory), so delta v -- and with it v_c, at which the rough hash-grid field is differentiated
# -- is as exact as in FP32; the adjoint chain runs in 16 bit.  Measured: the net's gradients
# within 0.005-0.010 of the oracle's per weight matrix and 0.007-0.010 over its tables, the
# field's tables within 0.002-0.003, in both FP16 and BF16 (with single-rounded 16-bit
# operands they were 0.09-0.15 and 0.28-0.54).
NET_TC_RTOL = {"fp16": (3e-2, 3e-2, 1e-2), "bf16": (3e-2, 3e-2, 1e-2)}   # net weights, net tables, field tables


@pytest.mark.parametrize("net_prec", ["fp16", "bf16"])
def test_deform_tensor_core_training(env, net_prec):
    invr, ctx, oracle = env
    rng = np.random.default_rng(108)
    tw = synth.train_step_workload(seed=18, n_rays=1024)
    dp, pose = synth.make_deform(rng), synth.make_pose(rng)
    ncode = invr.INVR_MLP_BF16 if net_prec == "bf16" else invr.INVR_MLP_FP16
    tb, gfields, ofields, net, onet, obatches, keep = _train(env, tw, dp, [pose], net_prec=ncode)
    loss = invr.forward_train(ctx, tb)
    invr.backward(ctx, tb)
    ctx.sync()
    oloss, ograds = oracle.train_loss_grad(obatches, tw.n_samples, tw.t_eps, tw.huber_delta)
    assert abs(float(host(loss)[0]) - oloss) <= 1e-5 * oloss
    w_tol, t_tol, f_tol = NET_TC_RTOL[net_prec]
    gt, gw = (host(x) for x in net.get_grads())
    ogt, ogw = ograds[id(onet)]
    off = 0
    for k, (r, c) in enumerate(dp.desc.weight_shapes()):
        e = _rel(gw[off:off + r * c], ogw[off:off + r * c])
        assert e <= w_tol, (k, e)
        off += r * c
    assert _rel(gt, ogt) <= t_tol
    fp = tw.fields[0]
    ft, fw = (host(x) for x in gfields[id(fp)].get_grads())
    oft, ofw = ograds[id(ofields[id(fp)])]
    assert _rel(fw, ofw) <= 1e-2 and _rel(ft, oft) <= f_tol


def test_deform_tensor_core_wait_timeout_recovered(env):
    """The net's tensor-core kernels (forward, adjoint chain, weight-gradient pipeline) with
    every bounded wait giving up at once: INVR_E_TIMEOUT at the next sync and no fault (each
    kernel retires its MMAs and copies in flight before freeing tensor memory); with the
    default limit the same context then matches the oracle's loss again."""
    invr, ctx, oracle = env
    rng = np.random.default_rng(121)
    tw = synth.train_step_workload(seed=21, n_rays=512)
    dp, pose = synth.make_deform(rng), synth.make_pose(rng)
    tb, gfields, ofields, net, onet, obatches, keep = _train(env, tw, dp, [pose], net_prec=invr.INVR_MLP_FP16)
    ctx.set_wait_limit(0)
    try:
        invr.forward_train(ctx, tb)
        invr.backward(ctx, tb)
        with pytest.raises(invr.InvrError, match="TIMEOUT"):
            ctx.sync()
    finally:
        ctx.set_wait_limit(1 << 22)
    loss = invr.forward_train(ctx, tb)
    ctx.sync()
    oloss, _ = oracle.train_loss_grad(obatches, tw.n_samples, tw.t_eps, tw.huber_delta, grads=False)
    assert abs(float(host(loss)[0]) - oloss) <= 1e-3 * oloss


def test_deform_zero_output_layer_is_the_plain_warp(env):
    invr, ctx, oracle = env
    rng = np.random.default_rng(102)
    w, dp, pose = _render_workload(rng)
    dp.weights[-3 * dp.desc.hidden:] = 0.0
    hum = Human(invr, ctx, oracle, w.views[0], dp, pose)
    plain_view = invr.View(hum.field, hum.graph, 0, None, hum.occ)
    a, _ = invr.render_rays(ctx, cu(w.rays.o), cu(w.rays.d), w.n_samples, w.t_eps, [hum.view])
    b, _ = invr.render_rays(ctx, cu(w.rays.o), cu(w.rays.d), w.n_samples, w.t_eps, [plain_view])
    ctx.sync()
    np.testing.assert_array_equal(host(a), host(b))


def _train(env, tw, dp, poses, loss="huber", net_prec=0):
    invr, ctx, oracle = env
    ofields = {id(fp): oracle.Field.from_params(fp) for fp in tw.fields}
    gfields = {id(fp): invr.Field.from_synth(ctx, fp) for fp in tw.fields}
    net, onet = invr.Deform.from_synth(ctx, dp, net_prec), oracle.Deform.from_params(dp)
    batches, obatches, keep = [], [], []
    k = 0
    for b in tw.batches:
        sv = b.view
        if sv.graph is not None:
            side = Human(invr, ctx, oracle, sv, dp, poses[k], field=gfields[id(sv.field)],
                         ofield=ofields[id(sv.field)], net=net, onet=onet)
            k += 1
            view, oview = side.view, side.oview
        else:
            f = gfields[id(sv.field)]
            occ = cu(sv.occupancy) if sv.occupancy is not None else None
            side = (f, occ)
            view = invr.View(f, None, 0, sv.rigid_dq, occ)
            oview = oracle.View.from_synth(sv, field=ofields[id(sv.field)])
        keep.append(side)
        batches.append((cu(b.rays.o), cu(b.rays.d), view, cu(b.target)))
        obatches.append(oracle.TrainBatch(b.rays.o, b.rays.d, oview, b.target))
    tb = invr.TrainBatches(batches, tw.n_samples, tw.t_eps, tw.huber_delta, tw.lr, tw.beta1, tw.beta2, tw.adam_eps)
    return tb, gfields, ofields, net, onet, obatches, keep


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _check_net_grads(net, onet, ograds, rtol):
    gt, gw = (host(x) for x in net.get_grads())
    ogt, ogw = ograds[id(onet)]
    assert np.abs(ogw).max() > 0
    d = onet.desc
    off = 0
    for k, (r, c) in enumerate(d.weight_shapes()):
        assert _rel(gw[off:off + r * c], ogw[off:off + r * c]) <= rtol, (k, _rel(gw[off:off + r * c], ogw[off:off + r * c]))
        off += r * c
    per = d.T * d.F
    for l in range(d.L):
        sl = slice(l * per, (l + 1) * per)
        if np.abs(ogt[sl]).max() > 0:
            assert _rel(gt[sl], ogt[sl]) <= rtol, (l, _rel(gt[sl], ogt[sl]))


@pytest.mark.parametrize("identity", [True, False])
def test_deform_training_gradients_match_oracle(env, identity):
    invr, ctx, oracle = env
    rng = np.random.default_rng(103)
    tw = synth.train_step_workload(seed=13, n_rays=1024)
    if identity:
        g = tw.batches[0].view.graph
        g.dq[:] = np.array([1, 0, 0, 0, 0, 0, 0, 0], np.float32)[:, None]
        g.x_live[:] = g.x_canon
    dp, pose = synth.make_deform(rng), synth.make_pose(rng)
    tb, gfields, ofields, net, onet, obatches, keep = _train(env, tw, dp, [pose])
    loss = invr.forward_train(ctx, tb)
    invr.backward(ctx, tb)
    ctx.sync()
    oloss, ograds = oracle.train_loss_grad(obatches, tw.n_samples, tw.t_eps, tw.huber_delta)
    assert abs(float(host(loss)[0]) - oloss) <= 1e-5 * oloss
    rtol = GRAD_RTOL if identity else GRAD_RTOL_WARP
    fp = tw.fields[0]
    gt, gw = (host(x) for x in gfields[id(fp)].get_grads())
    ogt, ogw = ograds[id(ofields[id(fp)])]
    assert _rel(gw, ogw) <= rtol and _rel(gt, ogt) <= rtol
    _check_net_grads(net, onet, ograds, 10 * rtol)


def test_deform_keyframes_two_fields(env):
    """Key frames of the human (one shared net, one pose per frame) and the object field in
    one call: loss and the net's gradients against the oracle."""
    invr, ctx, oracle = env
    rng = np.random.default_rng(104)
    tw = synth.keyframe_batch_workload(n_frames=2, log2_rays=(9.0, 10.0))
    dp = synth.make_deform(rng)
    poses = [synth.make_pose(rng) for _ in range(2)]
    tb, gfields, ofields, net, onet, obatches, keep = _train(env, tw, dp, poses)
    loss = invr.forward_train(ctx, tb)
    invr.backward(ctx, tb)
    ctx.sync()
    oloss, ograds = oracle.train_loss_grad(obatches, tw.n_samples, tw.t_eps, tw.huber_delta)
    assert abs(float(host(loss)[0]) - oloss) <= 1e-5 * oloss
    _check_net_grads(net, onet, ograds, 10 * GRAD_RTOL_WARP)


def test_deform_train_step_updates_the_net(env):
    invr, ctx, oracle = env
    rng = np.random.default_rng(105)
    tw = synth.train_step_workload(seed=15, n_rays=512)
    dp, pose = synth.make_deform(rng), synth.make_pose(rng)
    tb, gfields, ofields, net, onet, obatches, keep = _train(env, tw, dp, [pose])
    t0, w0 = (host(x) for x in net.get_params())
    losses = [float(host(invr.train_step(ctx, tb))[0]) for _ in range(3)]
    ctx.sync()
    t1, w1 = (host(x) for x in net.get_params())
    assert np.abs(w1 - w0).max() > 0 and np.abs(t1 - t0).max() > 0
    gt, gw = (host(x) for x in net.get_grads())
    assert np.abs(gw).max() == 0.0 and np.abs(gt).max() == 0.0     # Adam clears the gradients
    assert losses[-1] < losses[0]


def test_deform_rejected_by_point_calls(env):
    invr, ctx, oracle = env
    rng = np.random.default_rng(106)
    w, dp, pose = _render_workload(rng)
    hum = Human(invr, ctx, oracle, w.views[0], dp, pose)
    with pytest.raises(invr.InvrError):
        invr.warp_points(ctx, hum.view, cu(np.zeros((3, 8), np.float32)))
    with pytest.raises(invr.InvrError):
        invr.Deform(ctx, L=16, hidden=200)
    ctx.sync()
