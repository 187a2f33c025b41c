"""Thin ctypes binding of libbsp.so (the C ABI in include/bsp.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Functions keep the C names; arrays may be NumPy arrays (host)
or torch tensors (host or CUDA).  There is no CPU fallback: importing this
module fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libbsp.so")

BSP_OK = 0
BSP_ERR_INVALID_ARG = 1
BSP_ERR_OOM = 2
BSP_ERR_CUDA = 3
BSP_ERR_NUMERICAL = 4
BSP_ERR_TIMEOUT = 5
BSP_ERR_NOT_CONVERGED = 6

BSP_PREC_F32, BSP_PREC_F64, BSP_PREC_MIXED = 0, 1, 2
BSP_W_COMBINATORIAL, BSP_W_EDGE, BSP_W_INV_SQ_DIST = 0, 1, 2
BSP_SCHED_AUTO, BSP_SCHED_WAVES = 0, 1
BSP_DT_F32, BSP_DT_F64, BSP_DT_BF16 = 0, 1, 2

_STATUS = {0: "BSP_OK", 1: "BSP_ERR_INVALID_ARG", 2: "BSP_ERR_OOM", 3: "BSP_ERR_CUDA",
           4: "BSP_ERR_NUMERICAL", 5: "BSP_ERR_TIMEOUT", 6: "BSP_ERR_NOT_CONVERGED"}


class bsp_opts(C.Structure):
    _fields_ = [("delta", C.c_double), ("z", C.c_int32), ("weight_mode", C.c_int32),
                ("literal_degree", C.c_int32), ("precision", C.c_int32),
                ("cg_rtol", C.c_double), ("cg_max_steps", C.c_int32),
                ("rayleigh_ritz", C.c_int32), ("cols_per_cta", C.c_int32),
                ("use_graph", C.c_int32), ("schedule", C.c_int32),
                ("wait_limit_ms", C.c_int32), ("withhold_block", C.c_int32),
                ("cg_rows_per_lane", C.c_int32)]


class bsp_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("k", C.c_int32), ("nnz", C.c_int64),
                ("intra_edges", C.c_int64), ("max_block", C.c_int32), ("levels", C.c_int32),
                ("cg_steps_total", C.c_int64), ("cg_steps_max", C.c_int32),
                ("not_converged", C.c_int32), ("gpu_launches", C.c_int32),
                ("jacobi_sweeps", C.c_int32)]


class BspError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with "
                          "paper_1810_02719_gb300.build.build() (nvcc, sm_103a)")
    lib = C.CDLL(_LIB_PATH)
    P, I32, I64, D, U64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_uint64
    sig = {
        "bsp_opts_default": (None, [C.POINTER(bsp_opts)]),
        "bsp_mesh_create": (C.c_int, [P, I64, P, I64, P, P, I32, P, C.POINTER(bsp_opts),
                                      C.POINTER(P)]),
        "bsp_mesh_create_edges": (C.c_int, [P, I64, P, I64, P, P, I32, P, C.POINTER(bsp_opts),
                                            C.POINTER(P)]),
        "bsp_mesh_destroy": (C.c_int, [P]),
        "bsp_get_stats": (C.c_int, [P, C.POINTER(bsp_stats)]),
        "bsp_get_edges": (C.c_int, [P, P, C.POINTER(I64)]),
        "bsp_get_block_csr": (C.c_int, [P, I32, P, P, P, P, C.POINTER(I64)]),
        "bsp_set_edge_weights": (C.c_int, [P, P, I64]),
        "bsp_oi_track": (C.c_int, [P, I32, I32, P, P]),
        "bsp_oi_track_dynamic": (C.c_int, [P, P, D, I32, I32, I32, I32, U64, P, P, P, P]),
        "bsp_get_block_c": (C.c_int, [P, P]),
        "bsp_get_basis": (C.c_int, [P, I32, P, C.POINTER(I32)]),
        "bsp_project": (C.c_int, [P, P, I32, I32, P, P]),
        "bsp_reconstruct": (C.c_int, [P, P, I32, P, P]),
        "bsp_spmm": (C.c_int, [P, P, P, I32, P]),
        "bsp_last_error": (C.c_char_p, []),
        "bsp_set_profiling": (C.c_int, [P, I32]),
        "bsp_get_kernel_times": (C.c_int, [P, P, P, I32]),
        "bsp_onorm_noalloc": (C.c_int, [P, P, I32, I32, P]),
        "bsp_merge_overlapped": (C.c_int, [P, P, I64, P, I32, I32, P, P]),
        "bsp_oi_track_paper_doi": (C.c_int, [P, P, I32, D, D, I32, I32, I32, P, P, P, P]),
        "bsp_filter_forward": (C.c_int, [P, I32, I32, P, P, P, P]),
        "bsp_filter_backward": (C.c_int, [P, P, P, P, P, P]),
        "bsp_reconstruct_bf16": (C.c_int, [P, P, I32, P, P]),
        "bsp_autotune": (C.c_int, [P, I32, I32, P, I32, P, C.POINTER(I32), P]),
        "bsp_quantize": (C.c_int, [P, P, I32, I32, P, P, P]),
        "bsp_dequantize": (C.c_int, [P, P, P, I32, I32, P, P]),
        "bsp_bits_per_vertex": (C.c_int, [P, I32, C.POINTER(D)]),
        "bsp_nmsve": (C.c_int, [P, P, I32, I64, P, I64, P, P]),
        "bsp_fine_denoise": (C.c_int, [P, P, P, I32, I64, P, I64, D, D, I32, I32, P]),
        "bsp_normal_angle_error": (C.c_int, [P, P, I32, I64, P, I64, C.POINTER(D), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
LIB_PATH = _LIB_PATH


def exported_symbols():
    """Names the binding resolves in libbsp.so."""
    return ["bsp_opts_default", "bsp_mesh_create", "bsp_mesh_create_edges", "bsp_mesh_destroy",
            "bsp_get_stats", "bsp_get_edges", "bsp_get_block_csr", "bsp_set_edge_weights",
            "bsp_oi_track", "bsp_oi_track_dynamic", "bsp_get_block_c", "bsp_get_basis",
            "bsp_project", "bsp_reconstruct", "bsp_spmm", "bsp_last_error",
            "bsp_set_profiling", "bsp_get_kernel_times", "bsp_onorm_noalloc",
            "bsp_filter_forward", "bsp_filter_backward", "bsp_reconstruct_bf16",
            "bsp_autotune", "bsp_quantize", "bsp_dequantize", "bsp_bits_per_vertex",
            "bsp_nmsve", "bsp_fine_denoise", "bsp_normal_angle_error", "bsp_merge_overlapped",
            "bsp_oi_track_paper_doi"]


def _check(code):
    if code != BSP_OK:
        raise BspError(code, _lib.bsp_last_error().decode())


def _ptr(a):
    """Raw pointer of a NumPy array or torch tensor (must be contiguous); None -> NULL."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _i32(a):
    if isinstance(a, np.ndarray) or a is None or not hasattr(a, "data_ptr"):
        return None if a is None else np.ascontiguousarray(a, dtype=np.int32)
    return a.contiguous()


def _f64(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.contiguous()
    return np.ascontiguousarray(a, dtype=np.float64)


def bsp_opts_default() -> bsp_opts:
    o = bsp_opts()
    _lib.bsp_opts_default(C.byref(o))
    return o


def make_opts(**kw) -> bsp_opts:
    o = bsp_opts_default()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


# per handle: the mesh's real type and block sizes, so that the readers below
# size their host buffers from the mesh itself (the library writes n_b rows of
# the mesh's precision; a smaller or narrower buffer would be overrun)
_MESHES = {}


def _remember(h, opts, block_ptr):
    prec = opts.precision if opts is not None else bsp_opts_default().precision
    _MESHES[h] = (np.float64 if prec == BSP_PREC_F64 else np.float32,
                  np.diff(np.asarray(block_ptr, dtype=np.int64)))


def _mesh_real(mesh, real, what):
    info = _MESHES.get(mesh)
    if info is None:
        if real is None:
            raise ValueError(f"{what}: unknown mesh handle; pass real=")
        return real
    if real is not None and np.dtype(real) != np.dtype(info[0]):
        raise ValueError(f"{what}: the mesh holds {np.dtype(info[0])}, not {np.dtype(real)}")
    return info[0]


def _check_rows(mesh, b, n_b, what):
    info = _MESHES.get(mesh)
    if info is not None and not (0 <= b < info[1].size and int(info[1][b]) == int(n_b)):
        raise ValueError(f"{what}: block {b} has {int(info[1][b]) if 0 <= b < info[1].size else '?'} "
                         f"rows, not {n_b}")


def bsp_mesh_create(xyz, faces, block_ptr, block_verts, parent, opts=None, n=None):
    """Create a mesh from faces; returns an opaque handle (int)."""
    xyz = _f64(xyz)
    faces, block_ptr = _i32(faces), _i32(block_ptr)
    block_verts, parent = _i32(block_verts), _i32(parent)
    if n is None:
        n = int(block_verts.shape[0])
    h = C.c_void_p()
    _check(_lib.bsp_mesh_create(_ptr(xyz), n, _ptr(faces), int(faces.shape[0]), _ptr(block_ptr),
                                _ptr(block_verts), int(block_ptr.shape[0]) - 1, _ptr(parent),
                                C.byref(opts) if opts is not None else None, C.byref(h)))
    _remember(h.value, opts, block_ptr)
    return h.value


def bsp_mesh_create_edges(xyz, edges, block_ptr, block_verts, parent, opts=None, n=None):
    xyz = _f64(xyz)
    edges, block_ptr = _i32(edges), _i32(block_ptr)
    block_verts, parent = _i32(block_verts), _i32(parent)
    if n is None:
        n = int(block_verts.shape[0])
    h = C.c_void_p()
    _check(_lib.bsp_mesh_create_edges(_ptr(xyz), n, _ptr(edges), int(edges.shape[0]),
                                      _ptr(block_ptr), _ptr(block_verts),
                                      int(block_ptr.shape[0]) - 1, _ptr(parent),
                                      C.byref(opts) if opts is not None else None, C.byref(h)))
    _remember(h.value, opts, block_ptr)
    return h.value


def bsp_mesh_destroy(mesh):
    _MESHES.pop(mesh, None)
    _check(_lib.bsp_mesh_destroy(mesh))


def bsp_get_stats(mesh) -> dict:
    st = bsp_stats()
    _check(_lib.bsp_get_stats(mesh, C.byref(st)))
    return {f: getattr(st, f) for f, _ in bsp_stats._fields_}


def bsp_get_edges(mesh) -> np.ndarray:
    E = C.c_int64()
    _check(_lib.bsp_get_edges(mesh, None, C.byref(E)))
    out = np.empty((E.value, 2), dtype=np.int32)
    _check(_lib.bsp_get_edges(mesh, _ptr(out), C.byref(E)))
    return out


def bsp_get_block_csr(mesh, b, n_b, real=None):
    """Block b's CSR (row pointers, local columns, off-diagonal weights,
    diagonal) in the mesh's precision (real: that dtype or None)."""
    real = _mesh_real(mesh, real, "bsp_get_block_csr")
    _check_rows(mesh, b, n_b, "bsp_get_block_csr")
    nnz = C.c_int64()
    _check(_lib.bsp_get_block_csr(mesh, b, None, None, None, None, C.byref(nnz)))
    rp = np.empty(n_b + 1, np.int32)
    cols = np.empty(nnz.value, np.int32)
    vals = np.empty(nnz.value, real)
    diag = np.empty(n_b, real)
    _check(_lib.bsp_get_block_csr(mesh, b, _ptr(rp), _ptr(cols), _ptr(vals), _ptr(diag),
                                  C.byref(nnz)))
    return rp, cols, vals, diag


def bsp_set_edge_weights(mesh, w):
    _check(_lib.bsp_set_edge_weights(mesh, _ptr(w), int(w.shape[0])))


def bsp_oi_track(mesh, c, t_max, V0_roots, stream=None):
    _check(_lib.bsp_oi_track(mesh, c, t_max, _ptr(V0_roots), _stream_ptr(stream)))


def bsp_autotune(mesh, c, t_max, V0_roots, reps=3, stream=None):
    """Time the CG layouts (columns per CTA 0, 2, 4, 8) on fixed-c tracking of this
    mesh and keep the fastest; returns (chosen, {candidate: median ms or -1})."""
    times = np.zeros(4, np.float64)
    chosen = C.c_int32()
    _check(_lib.bsp_autotune(mesh, c, t_max, _ptr(V0_roots), reps, _ptr(times), C.byref(chosen),
                             _stream_ptr(stream)))
    return chosen.value, dict(zip((0, 2, 4, 8), times.tolist()))


def bsp_oi_track_dynamic(mesh, X, rel_tol, c_min, c_max, c_step, t_max, seed, V0_roots,
                         forced_c=None, c_out=None, stream=None):
    forced_c = _i32(forced_c)
    _check(_lib.bsp_oi_track_dynamic(mesh, _ptr(X), rel_tol, c_min, c_max, c_step, t_max,
                                     seed, _ptr(V0_roots), _ptr(forced_c), _ptr(c_out),
                                     _stream_ptr(stream)))


def bsp_get_block_c(mesh, k) -> np.ndarray:
    out = np.empty(k, np.int32)
    _check(_lib.bsp_get_block_c(mesh, _ptr(out)))
    return out


def bsp_get_basis(mesh, b, n_b, real=None) -> np.ndarray:
    """Block b's basis [n_b x c_b] in the mesh's precision (real: that dtype or None)."""
    real = _mesh_real(mesh, real, "bsp_get_basis")
    _check_rows(mesh, b, n_b, "bsp_get_basis")
    c = C.c_int32()
    _check(_lib.bsp_get_basis(mesh, b, None, C.byref(c)))
    U = np.empty((n_b, c.value), real)
    _check(_lib.bsp_get_basis(mesh, b, _ptr(U), C.byref(c)))
    return U


def bsp_project(mesh, X, x_dtype, cols, E_out, stream=None):
    _check(_lib.bsp_project(mesh, _ptr(X), x_dtype, cols, _ptr(E_out), _stream_ptr(stream)))


def bsp_reconstruct(mesh, E, cols, X_out, stream=None):
    _check(_lib.bsp_reconstruct(mesh, _ptr(E), cols, _ptr(X_out), _stream_ptr(stream)))


def bsp_reconstruct_bf16(mesh, E, cols, X_out, stream=None):
    _check(_lib.bsp_reconstruct_bf16(mesh, _ptr(E), cols, _ptr(X_out), _stream_ptr(stream)))


def bsp_quantize(mesh, E, cols, bits, codes, rng, stream=None):
    """codes (uint16 [sum c_b x cols]) and ranges (real [k x cols x 2]) of E."""
    _check(_lib.bsp_quantize(mesh, _ptr(E), cols, bits, _ptr(codes), _ptr(rng),
                             _stream_ptr(stream)))


def bsp_dequantize(mesh, codes, rng, cols, bits, E_out, stream=None):
    _check(_lib.bsp_dequantize(mesh, _ptr(codes), _ptr(rng), cols, bits, _ptr(E_out),
                               _stream_ptr(stream)))


def bsp_bits_per_vertex(mesh, bits) -> float:
    out = C.c_double()
    _check(_lib.bsp_bits_per_vertex(mesh, bits, C.byref(out)))
    return out.value


def bsp_nmsve(X, X_rec, dtype, n, faces, m, stream=None):
    """(NMSVE, ||v - v~||, ||GL(v) - GL(v~)||) of two n x 3 coordinate arrays."""
    out = np.zeros(3, np.float64)
    faces = _i32(faces)
    _check(_lib.bsp_nmsve(_ptr(X), _ptr(X_rec), dtype, n, _ptr(faces), m, _ptr(out),
                          _stream_ptr(stream)))
    return float(out[0]), float(out[1]), float(out[2])


def bsp_fine_denoise(X, X_out, dtype, n, faces, m, sigma_s, sigma_r, normal_iters,
                     vertex_iters, normals_out=None, stream=None):
    """Bilateral normal filter + vertex fitting of an n x 3 mesh (fine denoising step)."""
    faces = _i32(faces)
    _check(_lib.bsp_fine_denoise(_ptr(X), _ptr(X_out), _ptr(normals_out), dtype, n, _ptr(faces),
                                 m, float(sigma_s), float(sigma_r), normal_iters, vertex_iters,
                                 _stream_ptr(stream)))


def bsp_normal_angle_error(X, X_ref, dtype, n, faces, m, stream=None) -> float:
    """Mean angle (degrees) between corresponding face normals of two meshes."""
    faces = _i32(faces)
    out = C.c_double()
    _check(_lib.bsp_normal_angle_error(_ptr(X), _ptr(X_ref), dtype, n, _ptr(faces), m,
                                       C.byref(out), _stream_ptr(stream)))
    return out.value


def bsp_spmm(mesh, P, Y, c, stream=None):
    _check(_lib.bsp_spmm(mesh, _ptr(P), _ptr(Y), c, _stream_ptr(stream)))


KERNEL_CLASSES = ["init", "cg", "gram", "reduce", "chol", "panel", "rr", "jacobi", "project",
                  "recon", "spmm", "dyn", "oi"]


def bsp_set_profiling(mesh, on):
    _check(_lib.bsp_set_profiling(mesh, 1 if on else 0))


def bsp_get_kernel_times(mesh) -> dict:
    """{class: (total_ms, launches)} accumulated while profiling was on."""
    n = len(KERNEL_CLASSES)
    ms = np.zeros(n, np.float64)
    cnt = np.zeros(n, np.int32)
    _check(_lib.bsp_get_kernel_times(mesh, _ptr(ms), _ptr(cnt), n))
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_CLASSES)}


def bsp_onorm_noalloc(Y, Q, n, c, stream=None):
    """Allocation-free Q = Onorm(Y) of one block (device float [n x c] buffers owned
    by the caller), for callers that must not allocate device memory while running.

    Torch tensors must be contiguous float32 CUDA tensors of at least n * c
    elements; with ``stream=None`` the call runs on the current torch stream of
    Y's device, so it is ordered after the work that wrote Y.  Other objects
    (raw pointers, NumPy arrays) go to the library unchanged, which rejects
    anything that is not device memory of the current device.
    """
    tensors = [(name, t) for name, t in (("Y", Y), ("Q", Q)) if hasattr(t, "data_ptr")]
    if tensors:
        import torch
        for name, t in tensors:
            if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
            if t.numel() < n * c:
                raise ValueError(f"{name} holds {t.numel()} elements, fewer than n * c")
        if stream is None and hasattr(Y, "data_ptr"):
            stream = torch.cuda.current_stream(Y.device)
    _check(_lib.bsp_onorm_noalloc(_ptr(Y), _ptr(Q), n, c, _stream_ptr(stream)))


def bsp_oi_track_paper_doi(mesh, X, c0, eps_l, eps_h, c_min, c_max, t_cap, V0_roots,
                           stream=None):
    """The paper's dynamic OI (Sec. 5, Algorithm 2, one column at a time, two
    thresholds); returns (c per block, iterations per block) as int32 arrays."""
    k = bsp_get_stats(mesh)["k"]
    c = np.empty(k, np.int32)
    its = np.empty(k, np.int32)
    _check(_lib.bsp_oi_track_paper_doi(mesh, _ptr(X), c0, float(eps_l), float(eps_h), c_min,
                                       c_max, t_cap, _ptr(V0_roots), _ptr(c), _ptr(its),
                                       _stream_ptr(stream)))
    return c, its


def bsp_merge_overlapped(mesh, orig, n_orig, X_copies, x_dtype, cols, X_out, stream=None):
    """Algorithm 3 (Sec. 6.1): degree-weighted mean of every vertex's copies in an
    expanded (one vertex per part and copy) mesh; orig maps copies to vertices."""
    _check(_lib.bsp_merge_overlapped(mesh, _ptr(_i32(orig)), int(n_orig), _ptr(X_copies),
                                     x_dtype, cols, _ptr(X_out), _stream_ptr(stream)))


def bsp_filter_forward(mesh, c, t_max, V0_roots, X, X_out, stream=None):
    _check(_lib.bsp_filter_forward(mesh, c, t_max, _ptr(V0_roots), _ptr(X), _ptr(X_out),
                                   _stream_ptr(stream)))


def bsp_filter_backward(mesh, G, X, dX, dW, stream=None):
    _check(_lib.bsp_filter_backward(mesh, _ptr(G), _ptr(X), _ptr(dX), _ptr(dW),
                                    _stream_ptr(stream)))


def bsp_last_error() -> str:
    return _lib.bsp_last_error().decode()
