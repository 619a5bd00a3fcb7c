"""invr_query_points_noalloc, the query entry point that allocates no device memory (for
callers that cannot call cudaMalloc), checked through the C ABI against the allocating
invr_query_points on two calls in a row.  Collected last on purpose."""
import numpy as np
import pytest

from paper_2304_03184_b300 import synth

pytestmark = pytest.mark.gpu

COLOUR_TOL = 1e-5


@pytest.fixture(scope="module")
def ctx_env():
    import torch
    from paper_2304_03184_b300 import build
    build.build()
    import paper_2304_03184_b300 as invr
    assert torch.cuda.is_available()
    return invr, invr.Context(0)


def _cu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _views(invr, ctx, rng):
    human = synth.make_field(rng, synth.CFG2_FIELD)
    g = synth.make_graph(rng, 2048, K=4)
    graph = invr.Graph(ctx, 2048, 4, g.radius, 1, _cu(g.x_canon))
    graph.set_pose(0, _cu(g.dq), _cu(g.x_live))
    obj = synth.make_field(rng, synth.CFG1_FIELD)
    dq, _, _ = synth.make_object_pose(rng)
    fh, fo = invr.Field.from_synth(ctx, human), invr.Field.from_synth(ctx, obj)
    return (fh, graph, invr.View(fh, graph)), (fo, invr.View(fo, rigid_dq=dq)), g


def test_noalloc_query_matches_allocating_query(ctx_env):
    invr, ctx = ctx_env
    rng = np.random.default_rng(40)
    (fh, graph, hv), (fo, ov), g = _views(invr, ctx, rng)
    # call 1: the largest allowed batch through the human field; call 2: a smaller, ragged
    # batch through the object field, so stale scratch from call 1 would show
    near = g.x_live[:, rng.integers(0, 2048, invr.NOALLOC_MAX_POINTS)] + rng.normal(
        scale=0.05, size=(3, invr.NOALLOC_MAX_POINTS))
    for view, pts in ((hv, near.astype(np.float32)),
                      (ov, rng.uniform(-1, 1, size=(3, 1001)).astype(np.float32))):
        p = _cu(pts)
        want = invr.query_points(ctx, view, p)
        got = invr.query_points_noalloc(ctx, view, p)
        ctx.sync()
        np.testing.assert_allclose(got.cpu().numpy(), want.cpu().numpy(), rtol=0, atol=COLOUR_TOL)


def test_noalloc_query_mixed_precision_field(ctx_env):
    """A field with a 16-bit MLP goes through the tensor-core MLP in both entry points."""
    invr, ctx = ctx_env
    rng = np.random.default_rng(42)
    fp = synth.make_field(rng, synth.CFG1_FIELD)
    f = invr.Field.from_synth(ctx, fp, invr.INVR_MLP_BF16)
    dq, _, _ = synth.make_object_pose(rng)
    view = invr.View(f, rigid_dq=dq)
    p = _cu(rng.uniform(-1, 1, size=(3, 3000)).astype(np.float32))
    want = invr.query_points(ctx, view, p)
    got = invr.query_points_noalloc(ctx, view, p)
    ctx.sync()
    assert np.isfinite(want.cpu().numpy()).all()
    np.testing.assert_allclose(got.cpu().numpy(), want.cpu().numpy(), rtol=0, atol=COLOUR_TOL)


def test_noalloc_query_rejects_oversize(ctx_env):
    invr, ctx = ctx_env
    rng = np.random.default_rng(41)
    (_, _, hv), _, _ = _views(invr, ctx, rng)
    p = _cu(np.zeros((3, invr.NOALLOC_MAX_POINTS + 1), np.float32))
    with pytest.raises(invr.InvrError, match="INVR_NOALLOC_MAX_POINTS"):
        invr.query_points_noalloc(ctx, hv, p)


def _pool_attr(rt, pool, attr):
    err, v = rt.cudaMemPoolGetAttribute(pool, attr)
    assert err == rt.cudaError_t.cudaSuccess
    return int(v)


def test_noalloc_query_allocates_nothing(ctx_env):
    """What the entry point is for: a call, including the first one on a new context, leaves
    the device's memory use unchanged.  Checked around two calls per MLP path (FP32 and BF16
    tensor cores) with the output pre-allocated by the caller: the device's free memory
    (a cudaMalloc or a lazily loaded module would lower it), the high-water mark of the
    device's default stream-ordered pool (cudaMallocAsync) and torch's allocator peak."""
    invr, _ = ctx_env
    import torch
    from cuda.bindings import driver as drv, runtime as rt
    ctx = invr.Context(0)                    # sets the query up (address lookup, kernel loads)
    rng = np.random.default_rng(43)
    (fh, graph, hv), (fo, ov), g = _views(invr, ctx, rng)
    fb = invr.Field.from_synth(ctx, synth.make_field(rng, synth.CFG1_FIELD), invr.INVR_MLP_BF16)
    dq, _, _ = synth.make_object_pose(rng)
    bv = invr.View(fb, rigid_dq=dq)
    p = _cu(rng.uniform(-1, 1, size=(3, 5000)).astype(np.float32))
    out = torch.empty((4, 5000), device="cuda")
    torch.cuda.synchronize()
    err, pool = rt.cudaDeviceGetDefaultMemPool(0)
    assert err == rt.cudaError_t.cudaSuccess
    high = rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemHigh
    used = rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemCurrent
    err, = rt.cudaMemPoolSetAttribute(pool, high, drv.cuuint64_t(0))   # high mark := current use
    assert err == rt.cudaError_t.cudaSuccess
    used0 = _pool_attr(rt, pool, used)
    torch.cuda.reset_peak_memory_stats()
    peak0 = torch.cuda.max_memory_allocated()
    free0 = torch.cuda.mem_get_info()[0]
    for view in (hv, bv, hv, bv):
        invr.query_points_noalloc(ctx, view, p, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert _pool_attr(rt, pool, high) == used0
    assert torch.cuda.max_memory_allocated() == peak0
    want = invr.query_points(ctx, bv, p)
    ctx.sync()
    np.testing.assert_allclose(out.cpu().numpy(), want.cpu().numpy(), rtol=0, atol=COLOUR_TOL)
