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
