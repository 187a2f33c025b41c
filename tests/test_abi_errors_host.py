"""CPU-only checks of the boundary's argument validation: every call below must
return BSP_ERR_INVALID_ARG with a message before it touches the GPU (no CUDA
call is made on these paths, so they run without a device)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def bsp():
    from paper_1810_02719_gb300 import build
    build.build()
    from paper_1810_02719_gb300 import bsp as b
    return b


def _invalid(bsp, fn, *args, match=None, **kw):
    with pytest.raises(bsp.BspError) as e:
        fn(*args, **kw)
    assert e.value.code == bsp.BSP_ERR_INVALID_ARG
    msg = bsp.bsp_last_error()
    assert msg
    if match:
        assert match in msg, msg


def test_mesh_calls_reject_a_null_mesh(bsp):
    E = np.zeros((8, 3), np.float32)
    codes = np.zeros((8, 3), np.uint16)
    rng = np.zeros((1, 3, 2), np.float32)
    _invalid(bsp, bsp.bsp_quantize, None, E, 3, 12, codes, rng, match="NULL")
    _invalid(bsp, bsp.bsp_dequantize, None, codes, rng, 3, 12, E, match="NULL")
    _invalid(bsp, bsp.bsp_bits_per_vertex, None, 12, match="NULL")
    with pytest.raises(bsp.BspError):
        bsp.bsp_get_stats(None)


def test_nmsve_arguments(bsp):
    X = np.zeros((4, 3))
    tri = np.array([[0, 1, 2]], np.int32)
    _invalid(bsp, bsp.bsp_nmsve, X, X, bsp.BSP_DT_BF16, 4, tri, 1, match="dtype")
    _invalid(bsp, bsp.bsp_nmsve, X, X, bsp.BSP_DT_F64, 0, tri, 1, match="out of range")
    _invalid(bsp, bsp.bsp_nmsve, X, X, bsp.BSP_DT_F64, 4, tri, -1, match="out of range")
    _invalid(bsp, bsp.bsp_nmsve, X, None, bsp.BSP_DT_F64, 4, tri, 1, match="NULL")
    _invalid(bsp, bsp.bsp_nmsve, X, X, bsp.BSP_DT_F64, 4, None, 1, match="NULL")


def test_fine_denoise_arguments(bsp):
    X = np.zeros((4, 3))
    out = np.zeros_like(X)
    tri = np.array([[0, 1, 2]], np.int32)
    for ss, sr in [(0.0, 0.3), (0.1, 0.0), (-1.0, 0.3), (np.inf, 0.3), (0.1, np.nan)]:
        _invalid(bsp, bsp.bsp_fine_denoise, X, out, bsp.BSP_DT_F64, 4, tri, 1, ss, sr, 1, 1,
                 match="sigma")
    _invalid(bsp, bsp.bsp_fine_denoise, X, out, bsp.BSP_DT_F64, 4, tri, 1, 0.1, 0.3, -1, 1,
             match="iteration")
    _invalid(bsp, bsp.bsp_fine_denoise, X, out, bsp.BSP_DT_BF16, 4, tri, 1, 0.1, 0.3, 1, 1,
             match="dtype")
    _invalid(bsp, bsp.bsp_fine_denoise, X, None, bsp.BSP_DT_F64, 4, tri, 1, 0.1, 0.3, 1, 1,
             match="NULL")
    _invalid(bsp, bsp.bsp_normal_angle_error, X, X, bsp.BSP_DT_BF16, 4, tri, 1, match="dtype")
    _invalid(bsp, bsp.bsp_normal_angle_error, X, X, bsp.BSP_DT_F32, 0, tri, 1,
             match="out of range")


def test_onorm_noalloc_size_limits(bsp):
    Y = np.zeros((4096, 8), np.float32)
    Q = np.zeros_like(Y)
    _invalid(bsp, bsp.bsp_onorm_noalloc, Y, Q, 4096, 8, match="2048")
    _invalid(bsp, bsp.bsp_onorm_noalloc, Y, Q, 128, 65, match="2048")
    _invalid(bsp, bsp.bsp_onorm_noalloc, Y, Q, 4, 8, match="c <= n")
    _invalid(bsp, bsp.bsp_onorm_noalloc, None, Q, 4, 2, match="required")


def test_mesh_options_are_checked_before_the_device(bsp):
    from paper_1810_02719_gb300 import synth
    xyz, faces = synth.torus(8)
    ptr, verts = synth.tile_partition(8, 4)
    parent = synth.raster_chain(len(ptr) - 1)
    bad = [dict(delta=0.0), dict(delta=-1.0), dict(z=0), dict(precision=3),
           dict(weight_mode=5), dict(cg_rtol=0.0), dict(cg_max_steps=0), dict(cols_per_cta=3)]
    for kw in bad:
        _invalid(bsp, bsp.bsp_mesh_create, xyz, faces, ptr, verts, parent, bsp.make_opts(**kw))
    _invalid(bsp, bsp.bsp_mesh_create, xyz, faces, ptr, verts, parent, bsp.make_opts(), n=0,
             match="positive")


# every entry point that takes a mesh handle, checked straight through ctypes
# (the Python wrappers are bypassed so that the library's own check is seen)
MESH_CALLS = ["bsp_get_edges", "bsp_get_block_csr", "bsp_set_edge_weights", "bsp_oi_track",
              "bsp_oi_track_dynamic", "bsp_get_block_c", "bsp_get_basis", "bsp_project",
              "bsp_reconstruct", "bsp_reconstruct_bf16", "bsp_spmm", "bsp_set_profiling",
              "bsp_get_kernel_times", "bsp_filter_forward", "bsp_filter_backward",
              "bsp_autotune", "bsp_quantize", "bsp_dequantize", "bsp_bits_per_vertex",
              "bsp_merge_overlapped", "bsp_oi_track_paper_doi", "bsp_get_stats"]


def test_every_mesh_call_rejects_a_null_handle_before_the_device(bsp):
    import ctypes as C
    ints = (C.c_int32, C.c_int64, C.c_uint64)
    for name in MESH_CALLS:
        f = getattr(bsp._lib, name)
        args = []
        for t in f.argtypes:
            if t in ints:
                args.append(1)
            elif t is C.c_double:
                args.append(1.0)
            else:
                args.append(None)        # the handle and every buffer: NULL
        rc = f(*args)
        assert rc == bsp.BSP_ERR_INVALID_ARG, (name, rc)
        assert bsp.bsp_last_error(), name
    # destroying a NULL handle is a no-op
    assert bsp._lib.bsp_mesh_destroy(None) == bsp.BSP_OK
    # the list above covers every exported call that takes a mesh handle
    no_mesh = {"bsp_opts_default", "bsp_mesh_create", "bsp_mesh_create_edges",
               "bsp_mesh_destroy", "bsp_last_error", "bsp_onorm_noalloc", "bsp_nmsve",
               "bsp_fine_denoise", "bsp_normal_angle_error"}
    assert set(bsp.exported_symbols()) == set(MESH_CALLS) | no_mesh
