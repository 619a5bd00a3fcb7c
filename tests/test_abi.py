"""C-ABI checks that need no GPU: the library builds and loads, exports every function
include/invr.h declares, the ctypes mirrors match the C struct layouts, and host-side
argument checks reject bad calls without touching a device."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "invr.h")


@pytest.fixture(scope="module")
def invr():
    from paper_2304_03184_b300 import build
    build.build()
    import paper_2304_03184_b300 as pkg
    pkg.lib()
    return pkg


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(invr_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("invr_render_rays", "invr_train_step", "invr_graph_create", "invr_graph_set_pose",
                     "invr_field_create", "invr_ctx_create"):
        assert required in names


def test_library_exports_every_declared_symbol(invr):
    out = subprocess.check_output(["nm", "-D", "--defined-only", invr.LIB_PATH], text=True)
    exported = set(re.findall(r"\sT\s+(invr_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert sorted(declared_functions()) == invr.exported_symbols()


LAYOUT_C = r"""
#include <stdio.h>
#include <stddef.h>
#include "invr.h"
#define F(T, m) printf(#T "." #m " %zu\n", offsetof(T, m));
int main(void) {
  printf("invr_field_desc %zu\n", sizeof(invr_field_desc));
  F(invr_field_desc, growth) F(invr_field_desc, mlp_in) F(invr_field_desc, prec)
  printf("invr_graph_desc %zu\n", sizeof(invr_graph_desc));
  F(invr_graph_desc, radius) F(invr_graph_desc, n_frames)
  printf("invr_field_view %zu\n", sizeof(invr_field_view));
  F(invr_field_view, frame) F(invr_field_view, rigid_dq) F(invr_field_view, occupancy_dev)
  F(invr_field_view, deform) F(invr_field_view, pose_dev)
  printf("invr_deform_desc %zu\n", sizeof(invr_deform_desc));
  F(invr_deform_desc, growth) F(invr_deform_desc, pose_dim) F(invr_deform_desc, n_hidden) F(invr_deform_desc, prec)
  printf("invr_render_args %zu\n", sizeof(invr_render_args));
  F(invr_render_args, n_samples) F(invr_render_args, t_eps) F(invr_render_args, views) F(invr_render_args, depth_dev)
  printf("invr_train_args %zu\n", sizeof(invr_train_args));
  F(invr_train_args, targets_dev) F(invr_train_args, huber_delta) F(invr_train_args, loss_dev)
  F(invr_train_args, loss) F(invr_train_args, masks_dev) F(invr_train_args, depths_dev)
  F(invr_train_args, depth_weight)
  return 0;
}
"""


def test_ctypes_struct_layouts_match_header(invr, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        k, v = line.split()
        got[k] = int(v)
    for name in ("invr_field_desc", "invr_graph_desc", "invr_field_view", "invr_render_args", "invr_train_args",
                 "invr_deform_desc"):
        cls = getattr(invr, name)
        assert C.sizeof(cls) == got[name], name
        for key, off in got.items():
            if key.startswith(name + "."):
                assert getattr(cls, key.split(".")[1]).offset == off, key


def test_status_strings_and_weight_count(invr):
    L = invr.lib()
    assert L.invr_status_string(0) == b"ok"
    assert L.invr_status_string(-1) == b"invalid argument"
    d = invr.field_desc(8, 14, N_min=16, growth=1.5)
    assert L.invr_field_weight_count(C.byref(d)) == 7296       # 16->64->64->16, 15->64->3
    d = invr.field_desc(16, 19, N_min=16, growth=1.38)
    assert L.invr_field_weight_count(C.byref(d)) == 8320


def test_host_argument_checks_need_no_device(invr):
    L = invr.lib()
    h = C.c_void_p()
    # an impossible device index is rejected before any device work
    assert L.invr_ctx_create(C.byref(h), 10_000) == -1
    assert L.invr_ctx_create(None, 0) == -1
    assert L.invr_ctx_destroy(None) == -1
    assert L.invr_render_rays(None, None, None) == -1
    assert L.invr_train_step(None, None, None) == -1
    assert L.invr_field_create(None, None, None) == -1
    assert L.invr_graph_set_pose(None, 0, None, None, None) == -1
    buf = C.create_string_buffer(8)
    assert L.invr_last_error_detail(None, buf, 8) == -1
