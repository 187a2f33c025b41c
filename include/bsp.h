/*
 * bsp.h — C ABI of the GB300 (sm_103a) library for block-based spectral
 * processing of triangle meshes with orthogonal iterations (OI).
 *
 * Method: Arvanitis, Lalos, Moustakas, "Block-Based Spectral Processing of
 * Static and Dynamic 3D Meshes using Orthogonal Iterations".  A mesh
 * M = (V, F) (Sec. 3) is split into k blocks (Sec. 4); for each block b the
 * library assembles the graph Laplacian L[b] = D - C (Sec. 3, Eqs. for L and
 * C), tracks the c lowest-frequency eigenvectors U_c[b] by orthogonal
 * iterations U(t) = Onorm(R^z U(t-1)), R = (L[b] + delta I)^-1, warm-started
 * from the parent block's basis (Sec. 4, Algorithm 1), optionally chooses c
 * per block for a reconstruction-quality target (Sec. 5, Algorithm 2), and
 * projects/reconstructs coordinates E = U^T v, v~ = U E (Sec. 3 GFT;
 * Sec. 7.1 compression; Sec. 7.2 coarse denoising; Sec. 7.3 all frames of a
 * dynamic mesh with one basis).  Around that path it offers the codec and
 * quality measures the paper evaluates (q-bit quantisation of the
 * coefficients, bits per vertex, NMSVE, the mean face-normal angle; Sec. 8)
 * and the fine denoising step after the coarse one (Sec. 7.2).
 *
 * Conventions for every entry point:
 *  - Returns a bsp_status; no C++ exception crosses this boundary.  On error,
 *    bsp_last_error() returns a thread-local message for the failing call.
 *  - Pointer arguments marked "host or device" may point to host memory
 *    (pageable or pinned) or to device memory of the current CUDA device; the
 *    library detects which with cudaPointerGetAttributes and copies as needed.
 *    Such calls are synchronous with respect to host buffers.
 *  - "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Every call returns only after its work on that stream has
 *    finished, so its status covers numerical failures detected on the GPU.
 *  - Matrices are row-major.  "real" means float when the mesh precision is
 *    BSP_PREC_F32 or BSP_PREC_MIXED and double when it is BSP_PREC_F64.
 *  - The caller owns every buffer it passes; the library copies what it keeps.
 *  - Different meshes may be used from different host threads at the same
 *    time; one mesh must not be used by two threads at once (the library's
 *    per-call scratch and error message are per thread; bsp_onorm_noalloc
 *    documents its own shared scratch).
 *  - Blocks are numbered 0..k-1 and must be topologically sorted:
 *    parent[b] < b, or parent[b] = -1 for a root (Sec. 4: "the subsequent ones
 *    are processed in a topologically sorted order").
 */
#ifndef BSP_H_
#define BSP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bsp_status {
  BSP_OK = 0,
  BSP_ERR_INVALID_ARG = 1,   /* bad index, non-covering partition, c > n_b, delta <= 0, ... */
  BSP_ERR_OOM = 2,           /* device allocation failed */
  BSP_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  BSP_ERR_NUMERICAL = 4,     /* Gram matrix not positive definite, NaN/Inf */
  BSP_ERR_TIMEOUT = 5,       /* a bounded device wait expired */
  BSP_ERR_NOT_CONVERGED = 6  /* a CG solve hit its step cap; results are still written */
} bsp_status;

typedef enum bsp_precision {
  BSP_PREC_F32 = 0,    /* FP32 everywhere, including Gram accumulation and Cholesky */
  BSP_PREC_F64 = 1,    /* FP64 everywhere */
  BSP_PREC_MIXED = 2   /* FP32 vectors/solves/projection; FP64 Gram accumulation and Cholesky */
} bsp_precision;

typedef enum bsp_weight_mode {
  BSP_W_COMBINATORIAL = 0,  /* C_ij = 1 on every edge */
  BSP_W_EDGE = 1,           /* C_ij = per-edge weight, initially 1, set by bsp_set_edge_weights */
  BSP_W_INV_SQ_DIST = 2     /* C_ij = 1 / ||v_i - v_j||^2 (Sec. 3, Eq. for C) */
} bsp_weight_mode;

typedef enum bsp_dtype {
  BSP_DT_F32 = 0,
  BSP_DT_F64 = 1,
  BSP_DT_BF16 = 2
} bsp_dtype;

typedef struct bsp_opts {
  double delta;            /* shift delta > 0 in R = (L + delta I)^-1 (Sec. 4). Default 1e-2. */
  int32_t z;               /* power z >= 1 of R (Sec. 4). Default 1. */
  int32_t weight_mode;     /* bsp_weight_mode. Default BSP_W_COMBINATORIAL. */
  int32_t literal_degree;  /* 1: D_ii = |N(i)| as printed in Sec. 3; 0: D_ii = sum_j C_ij. Default 0. */
  int32_t precision;       /* bsp_precision. Default BSP_PREC_MIXED. */
  double cg_rtol;          /* CG stop: ||r_j|| <= cg_rtol * ||b_j|| per column. Default 1e-6 (1e-12 for F64). */
  int32_t cg_max_steps;    /* CG step cap per solve. Default 2000. */
  int32_t rayleigh_ritz;   /* 1: Rayleigh-Ritz after the OI steps of each block (ascending order). Default 1. */
  int32_t cols_per_cta;    /* CG column-slab width (1, 2, 4 or 8); 0 = automatic. */
  int32_t use_graph;       /* 1: run the tracking schedules (fixed c, dynamic c, the paper's
                              dynamic OI) as CUDA graphs, captured on the first call and
                              replayed while the parameters stay the same; the dynamic
                              schedules decide their rounds on the device (conditional
                              nodes).  0: the same launches from the host.  Default 1. */
  int32_t schedule;        /* bsp_schedule: how the fixed-c schedule runs.  Default BSP_SCHED_AUTO. */
  int32_t wait_limit_ms;   /* bound of a device-side wait for a block computed by another
                              cluster of the persistent engine; on expiry the call returns
                              BSP_ERR_TIMEOUT.  Default 2000. */
  int32_t withhold_block;  /* test hook: block b >= 0 waits for a parent flag that is never
                              set (the wait runs out: BSP_ERR_TIMEOUT).  Default -1 (none). */
  int32_t cg_rows_per_lane; /* tile shape of the batched CG (one column per team of warps):
                              8 = 8 rows per lane, each row's neighbour indices in registers
                              (unweighted meshes of degree <= 8, blocks <= 2,048 rows; teams
                              twice as wide), 16 = 16 rows per lane, the pattern in shared
                              memory.  0 = automatic (8 where it applies).  bsp_autotune
                              sets it. */
} bsp_opts;

/* Execution of the fixed-c schedule (bsp_oi_track, FP32 precision).
 *   BSP_SCHED_AUTO   persistent cluster engine when the shapes fit (c <= 64,
 *                    blocks <= 1,024 rows, <= 16 neighbours per vertex, t_max >= 1),
 *                    per-wave launches otherwise;
 *   BSP_SCHED_WAVES  per-wave launches only (one CG and one Onorm launch per
 *                    level of the block DAG). */
typedef enum { BSP_SCHED_AUTO = 0, BSP_SCHED_WAVES = 1 } bsp_schedule;

typedef struct bsp_stats {
  int64_t n;               /* vertices */
  int32_t k;               /* blocks */
  int64_t nnz;             /* stored off-diagonal entries over all blocks (2 x intra-block edges) */
  int64_t intra_edges;     /* intra-block edges */
  int32_t max_block;       /* largest n_b */
  int32_t levels;          /* depth of the block forest (number of dependent waves) */
  int64_t cg_steps_total;  /* CG steps summed over all CTAs' slabs in the last tracking call */
  int32_t cg_steps_max;    /* largest step count of one solve in the last tracking call */
  int32_t not_converged;   /* solves that hit cg_max_steps in the last tracking call */
  int32_t gpu_launches;    /* kernels launched by the last tracking/projection call */
  int32_t jacobi_sweeps;   /* Rayleigh-Ritz Jacobi sweeps summed over blocks, last tracking call */
} bsp_stats;

typedef struct bsp_mesh bsp_mesh;

/* Fill *opts with the defaults listed above. */
void bsp_opts_default(bsp_opts* opts);

/*
 * Create a partitioned mesh and assemble every block's Laplacian on the GPU
 * (Sec. 3 L = D - C; Sec. 4 block processing; Sec. 6.1 a block only sees its
 * own edges).  Edges are the sides of the faces (Sec. 3); an edge belongs to
 * block b when both end points lie in b.
 *   xyz         host or device, double [n x 3]; may be NULL unless
 *               weight_mode = BSP_W_INV_SQ_DIST.
 *   faces       host or device, int32 [m x 3], vertex ids in [0, n).
 *   block_ptr   host or device, int32 [k + 1], block_ptr[0] = 0, non-decreasing,
 *               block_ptr[k] = n: the partition must cover every vertex once.
 *   block_verts host or device, int32 [n]: block b's vertices in their local
 *               order are block_verts[block_ptr[b] .. block_ptr[b+1]).
 *   parent      host or device, int32 [k]: warm-start parent, parent[b] < b or -1.
 *   opts        host; NULL = defaults.
 *   out         receives the new mesh; *out = NULL on error.
 * Errors: BSP_ERR_INVALID_ARG (index out of range, vertex missing or repeated,
 * block larger than 65535, parent not earlier), BSP_ERR_OOM, BSP_ERR_CUDA.
 */
int bsp_mesh_create(const double* xyz, int64_t n, const int32_t* faces, int64_t m,
                    const int32_t* block_ptr, const int32_t* block_verts, int32_t k,
                    const int32_t* parent, const bsp_opts* opts, bsp_mesh** out);

/* As bsp_mesh_create, from an explicit edge list (host or device int32 [E x 2])
 * instead of faces; for graphs that are not triangle meshes (paths, cycles). */
int bsp_mesh_create_edges(const double* xyz, int64_t n, const int32_t* edges, int64_t E,
                          const int32_t* block_ptr, const int32_t* block_verts, int32_t k,
                          const int32_t* parent, const bsp_opts* opts, bsp_mesh** out);

/* Release every device buffer of the mesh.  NULL is accepted. */
int bsp_mesh_destroy(bsp_mesh* mesh);

/* Mesh sizes and counters of the last call. */
int bsp_get_stats(const bsp_mesh* mesh, bsp_stats* stats);

/*
 * Intra-block edge list in the library's canonical order: by block, then by
 * local pair (i, j), i < j, lexicographically.  edges_out: host or device
 * int32 [E_intra x 2] of GLOBAL vertex ids (NULL to query only); *E_out
 * receives E_intra.  This is the order of bsp_set_edge_weights.
 */
int bsp_get_edges(const bsp_mesh* mesh, int32_t* edges_out, int64_t* E_out);

/*
 * Per-block assembled Laplacian of block b in CSR form (for checking the
 * assembly against Sec. 3's definition).  row_ptr: int32 [n_b + 1]; cols:
 * int32 [nnz_b] local column ids ascending per row; vals: real [nnz_b] = C_ij;
 * diag: real [n_b] = D_ii.  All host or device; pass NULL to skip an array;
 * *nnz_b receives the entry count.
 */
int bsp_get_block_csr(const bsp_mesh* mesh, int32_t b, int32_t* row_ptr, int32_t* cols,
                      void* vals, void* diag, int64_t* nnz_b);

/*
 * Replace the edge weights C_ij (mesh created with BSP_W_EDGE), in the order of
 * bsp_get_edges; D_ii is re-derived.  w: host or device real [E].
 * Errors: BSP_ERR_INVALID_ARG if the mode is not BSP_W_EDGE or E mismatches.
 */
int bsp_set_edge_weights(bsp_mesh* mesh, const void* w, int64_t E);

/*
 * Fixed-c orthogonal iterations over all blocks (Sec. 4, Algorithm 1).
 * For every block in topological order: U(0) = Onorm(start); t_max times
 * U(t) = Onorm(R^z U(t-1)) with R^z applied by z conjugate-gradient solves
 * with (L + delta I) (Sec. 4: R^z U is computed with sparse linear solvers);
 * optional Rayleigh-Ritz.  start = the parent's final basis (rows mapped
 * r -> floor(r n_parent / n_b) when sizes differ), or, for a root, its rows
 * of V0_roots.  Independent blocks (same forest depth) run concurrently.
 *   c        1 <= c <= min over blocks of n_b, c <= 128 (c <= 64 with BSP_PREC_F64).
 *   t_max    >= 0 OI steps per block.
 *   V0_roots host or device real [sum over roots of n_b, c]: the roots' start
 *            matrices concatenated in block order; any full-rank matrices.
 * Results stay on the device (bsp_get_basis, bsp_project).  On a chain the
 * FP32 schedule runs the persistent engine over consecutive ranges of blocks
 * with each range's second CholeskyQR pass and Rayleigh-Ritz beside the next
 * range; the call returns once every block is done.
 * Errors: BSP_ERR_INVALID_ARG, BSP_ERR_NUMERICAL, BSP_ERR_NOT_CONVERGED, BSP_ERR_CUDA.
 */
int bsp_oi_track(bsp_mesh* mesh, int32_t c, int32_t t_max, const void* V0_roots, void* stream);

/*
 * The paper's own dynamic OI (Sec. 5, Algorithm 2), one column at a time with
 * two thresholds.  Per block, each iteration applies one Algorithm 1 step
 * U = Onorm(R^z U) and measures e = sum over x, y, z of (X_b - U U^T X_b)
 * (Eq. residual).  Branch directions as the text states them (the printed
 * algorithm swaps them): ||e|| > eps_h grows U by the column e/||e|| (the next
 * step's Onorm of R^z [U, e/||e||] is Eq. newU); ||e|| < eps_l keeps the
 * first c - 1 columns; anything else stops the block.  The width stays in
 * [c_min, min(c_max, n_b)] (a branch that would leave it stops instead), at
 * most t_cap iterations run, and a basis still carrying an appended column at
 * the cap is orthonormalised once more.  A root starts from its rows of
 * V0_roots (c0 columns), a child from its parent's final basis and width (rows
 * mapped r -> floor(r n_parent / n_b) when sizes differ).  The decisions are
 * taken in FP64.
 *   X         host or device real [n x 3] coordinates (global vertex order).
 *   c0        1 <= c_min <= c0 <= c_max <= 128 (<= 64 with BSP_PREC_F64),
 *             c0 <= every n_b.
 *   eps_l, eps_h  0 < eps_l <= eps_h: absolute thresholds on ||e||.
 *   t_cap     >= 1 iterations at most per block.
 *   V0_roots  host or device real [sum over roots of n_b, c0].
 *   c_out     host or device int32 [k] or NULL: final widths c_b.
 *   iters_out host or device int32 [k] or NULL: iterations run per block.
 * The iterations are decided on the device (no read-back between them); the
 * widths and iteration counts are read back once at the end.
 * Errors: BSP_ERR_INVALID_ARG, BSP_ERR_NUMERICAL, BSP_ERR_NOT_CONVERGED, BSP_ERR_CUDA.
 */
int bsp_oi_track_paper_doi(bsp_mesh* mesh, const void* X, int32_t c0, double eps_l, double eps_h,
                           int32_t c_min, int32_t c_max, int32_t t_cap, const void* V0_roots,
                           int32_t* c_out, int32_t* iters_out, void* stream);

/*
 * Dynamic-c orthogonal iterations (Sec. 5, Algorithm 2; quality-target reading).
 * Per block: start at c_parent (roots: c_min); run Algorithm 1 and
 * Rayleigh-Ritz; choose the smallest j in {c_step, 2 c_step, ...} with
 * ||X_b - U_j U_j^T X_b||_F <= rel_tol ||X_b||_F (shrink = Ritz prefix); if none,
 * grow by c_step columns [e/||e||, counter-hash columns] with e the residual
 * summed over x, y, z (Sec. 5, Eq. residual and Eq. newU), orthonormalise and
 * repeat, up to c_max.
 *   X        host or device real [n x 3] coordinates.
 *   V0_roots host or device real [sum over roots of n_b, c_min].
 *   forced_c host or device int32 [k] or NULL: when forced_c[b] >= 0 it replaces
 *            the decision of block b (replay hook).
 *   c_out    host or device int32 [k] or NULL: chosen c_b.
 * Requires c_min, c_max multiples of c_step, c_max <= 128.  The rounds are
 * decided on the device (no read-back between them); the widths are read
 * back once at the end.
 */
int bsp_oi_track_dynamic(bsp_mesh* mesh, const void* X, double rel_tol, int32_t c_min,
                         int32_t c_max, int32_t c_step, int32_t t_max, uint64_t seed,
                         const void* V0_roots, const int32_t* forced_c, int32_t* c_out,
                         void* stream);

/* Chosen c_b of every block after the last tracking call: host or device int32 [k]. */
int bsp_get_block_c(const bsp_mesh* mesh, int32_t* c_out);

/*
 * Basis U_c[b] of block b after tracking: host or device real [n_b x c_b]
 * (row-major, local vertex order).  *c receives c_b (U may be NULL to query).
 */
int bsp_get_basis(const bsp_mesh* mesh, int32_t b, void* U, int32_t* c);

/*
 * Spectral coefficients E[b] = U_c[b]^T X_b for every block (Sec. 3 GFT;
 * Sec. 7.1 encoder; Sec. 7.3 all frames at once).
 *   X       host or device [n x cols] with cols = 3 F (F frames of xyz per
 *           vertex row), element type x_dtype (BSP_DT_BF16 only with F32/MIXED).
 *   E_out   host or device real [sum_b c_b x cols], blocks concatenated in order.
 */
int bsp_project(bsp_mesh* mesh, const void* X, int32_t x_dtype, int32_t cols, void* E_out,
                void* stream);

/*
 * Reconstruction v~[b] = U_c[b] E[b] scattered to the global vertex rows
 * (Sec. 7.1 decoder; Sec. 7.2 coarse denoising v^ = U U^T v).
 *   E       host or device real [sum_b c_b x cols].
 *   X_out   host or device real [n x cols].
 */
int bsp_reconstruct(bsp_mesh* mesh, const void* E, int32_t cols, void* X_out, void* stream);

/*
 * Reconstruction X~[b] = U[b] E[b] on tcgen05 tensor cores with BF16 operands
 * (U and E rounded to bfloat16) and FP32 accumulation and output, for wide
 * coordinate matrices (all frames of a dynamic mesh, Sec. 7.3).
 *   E      device float [sum_b c_b x cols]; X_out device float [n x cols].
 * Requires F32 or MIXED precision and c <= 128.  (bsp_project takes the
 * tensor-core path itself when x_dtype is BSP_DT_BF16, cols % 8 == 0,
 * cols >= 64 and X is 16-byte aligned.)  Both build a BF16 copy of the bases
 * (n x pad16(c), kept on the mesh until the next tracking call).
 * Errors: BSP_ERR_INVALID_ARG, BSP_ERR_TIMEOUT, BSP_ERR_CUDA.
 */
int bsp_reconstruct_bf16(bsp_mesh* mesh, const float* E, int32_t cols, float* X_out, void* stream);

/*
 * Standalone operator product Y = (L + delta I) P for all blocks at once (the
 * sparse x tall-skinny kernel inside every CG step of R^z U, Sec. 4).
 *   P, Y    device real [n x c], rows in block order (row block_ptr[b] + i is
 *           local vertex i of block b).  1 <= c <= 128.
 */
int bsp_spmm(bsp_mesh* mesh, const void* P, void* Y, int32_t c, void* stream);

/*
 * Overlapped submeshes (Sec. 6.1, Algorithm 3): merge every vertex's copies
 * into one position, the average of the copies weighted by the vertex's
 * degree in each part (its number of neighbours in the part's induced
 * subgraph).  Parts that share vertices are given to the library as an
 * expanded mesh with one vertex per (part, vertex) copy, each part's induced
 * edges re-indexed to its copies (so every copy lies in one block); tracking,
 * projection and reconstruction run on that mesh as usual, and this call
 * merges the reconstructed copies.  A copy's weight is its CSR row length in
 * this mesh.  A vertex whose copies all have degree 0 takes the plain mean of
 * its copies; a vertex with no copy gets 0.  Each vertex's copies are summed
 * in ascending copy order (deterministic).
 *   mesh      the expanded mesh (n = number of copies).
 *   orig      host or device int32 [n]: the vertex of every copy, in [0, n_orig).
 *   n_orig    number of vertices of the original mesh.
 *   X_copies  host or device [n x cols] in the expanded mesh's vertex order (as
 *             bsp_reconstruct writes it), element type x_dtype (BSP_DT_F32 or
 *             BSP_DT_F64); the caller owns it.
 *   X_out     host or device [n_orig x cols], same element type; caller-owned.
 *   stream    cudaStream_t as void*; the call synchronises it.
 * Errors: BSP_ERR_INVALID_ARG (NULL, n_orig < 1, cols < 1, dtype, an orig
 * entry outside [0, n_orig)), BSP_ERR_OOM, BSP_ERR_CUDA.
 */
int bsp_merge_overlapped(const bsp_mesh* mesh, const int32_t* orig, int64_t n_orig,
                         const void* X_copies, int32_t x_dtype, int32_t cols, void* X_out,
                         void* stream);

/*
 * Block low-pass filter X^ = U U^T X (Sec. 7.2, coarse denoising) made
 * differentiable (not in the paper): every block runs t_max steps of
 * Algorithm 1 on L(w) = D(w) - C(w), where the per-edge weights w are those of
 * bsp_set_edge_weights (BSP_W_EDGE; the paper's combinatorial L at w = 1),
 * with Onorm after every step and no Rayleigh-Ritz; the start of a block is
 * its parent's final basis, treated as a constant (no gradient flows into
 * the parent).  All steps are checkpointed on the device for the backward.
 *   c, t_max   columns (1 <= c <= 64) and unrolled steps (>= 1).
 *   V0_roots   host or device real [sum over roots of n_b, c].
 *   X, X_out   host or device real [n x 3].
 * Requires opts.z = 1.  The bases become the mesh's tracked bases.
 */
int bsp_filter_forward(bsp_mesh* mesh, int32_t c, int32_t t_max, const void* V0_roots,
                       const void* X, void* X_out, void* stream);

/*
 * Gradients of a loss through the last bsp_filter_forward: given
 * G = dLoss/dX^ (device real [n x 3]) and the filter input X (device real
 * [n x 3]), writes dX = U U^T G (device real [n x 3]) and dW = dLoss/dw
 * (device real [E_intra], order of bsp_get_edges).  The adjoint solves with
 * (L + delta I) by the same CG (one solve per unrolled step) and uses
 * dLoss/dA = -Lambda Y^T for A = L(w) + delta I.
 */
int bsp_filter_backward(bsp_mesh* mesh, const void* G, const void* X, void* dX, void* dW,
                        void* stream);

/* Kernel classes reported by bsp_get_kernel_times, in this order. */
typedef enum bsp_kernel_class {
  BSP_KC_INIT = 0,     /* start matrices (root rows / parent row transfer) */
  BSP_KC_CG = 1,       /* fused CG solves of (L + delta I)^z Y = V */
  BSP_KC_GRAM = 2,     /* panel Gram partials of Onorm */
  BSP_KC_REDUCE = 3,   /* panel-partial reductions */
  BSP_KC_CHOL = 4,     /* c x c Cholesky + triangular inverse */
  BSP_KC_PANEL = 5,    /* panel x (c x c) products: Q = Y R^-1, V Q_H */
  BSP_KC_RR = 6,       /* H = V^T L V partials */
  BSP_KC_JACOBI = 7,   /* c x c Jacobi eigensolve of H */
  BSP_KC_PROJECT = 8,  /* E = U^T X */
  BSP_KC_RECON = 9,    /* X~ = U E */
  BSP_KC_SPMM = 10,    /* standalone (L + delta I) P */
  BSP_KC_DYN = 11,     /* dynamic-c decision and growth */
  BSP_KC_COUNT = 12
} bsp_kernel_class;

/*
 * Per-kernel-class timing (not part of the paper's method: instrumentation).
 * While on, every launch made by this mesh's calls is bracketed by CUDA events
 * recorded on the launching stream, and the fixed-c schedule runs eagerly
 * instead of as a CUDA graph; the kernels themselves are unchanged.  Turning it
 * on or off clears the accumulated times.
 */
int bsp_set_profiling(bsp_mesh* mesh, int32_t on);

/* Accumulated milliseconds and launch counts per class since profiling was
 * switched on; ms_out and launches_out are host arrays of n_classes entries
 * (either may be NULL). */
int bsp_get_kernel_times(const bsp_mesh* mesh, double* ms_out, int32_t* launches_out,
                         int32_t n_classes);

/*
 * Autotuner for the tile shape of the solves (no counterpart in the paper):
 * times fixed-c tracking of this mesh (bsp_oi_track with c, t_max and the
 * given root starts, reps timed runs after one warm-up, median) for each
 * candidate CG layout -- the batched team CG in size buckets (0), timed with
 * 8 and with 16 rows per lane (cg_rows_per_lane; 16 only where the 8-row
 * form does not apply), and column slabs of 2, 4 and 8 columns per CTA --
 * and keeps the fastest (cols_per_cta and cg_rows_per_lane) in the mesh's
 * options for later tracking calls (fixed and dynamic c).  With the FP32
 * schedule on the persistent engine the layouts are not used (a chain's
 * timings then differ only by noise).
 *   times_ms  host double [4] or NULL: median ms per candidate, in the order
 *             0, 2, 4, 8 (for 0 the faster of its rows-per-lane forms; a
 *             candidate whose shared memory does not fit the mesh's largest
 *             block reports -1).
 *   chosen    host int32 or NULL: the kept columns-per-CTA value.
 * The tracked bases afterwards are those of the last run.  Errors: as
 * bsp_oi_track.
 */
int bsp_autotune(bsp_mesh* mesh, int32_t c, int32_t t_max, const void* V0_roots, int32_t reps,
                 double* times_ms, int32_t* chosen, void* stream);

/*
 * Allocation-free orthonormalisation of one block (no counterpart in the
 * paper: an interface for callers that may not allocate device memory).
 * Q = Onorm(Y) by CholeskyQR2 in FP32 (the same fused kernel that Onorm uses
 * inside bsp_oi_track), for callers that cannot call cudaMalloc while they
 * run: a cudaMalloc can synchronise the whole device and has no latency
 * bound, which a streaming pipeline orthonormalising submeshes as they
 * arrive cannot afford, and some host applications own all device memory
 * through their own allocator.  This call allocates nothing: its scratch is
 * a fixed static device array of about 145 KiB (every GPU that loads the
 * library holds it until the process exits).
 *   Y, Q     device float [n x c], row-major (Q may alias Y); the caller owns
 *            both.  Both must be device (or managed) memory of the current
 *            device: a host pointer, or another GPU's, returns
 *            BSP_ERR_INVALID_ARG before any GPU work.
 *   n, c     1 <= c <= n, n <= 2048, c <= 64; larger sizes return
 *            BSP_ERR_INVALID_ARG without touching the GPU.
 *   stream   cudaStream_t as void* (NULL: the legacy default stream).  Every
 *            call copies its five parameters from host memory into the
 *            scratch array and synchronises this stream before it returns.
 * The first call on each device looks up the scratch array's device address
 * and configures the kernel.  All calls share the one scratch array: calls
 * that overlap on the GPU (other host threads, other streams) race and must
 * be serialised by the caller.  Errors: BSP_ERR_INVALID_ARG,
 * BSP_ERR_NUMERICAL (rank-deficient Y), BSP_ERR_CUDA.
 */
int bsp_onorm_noalloc(const float* Y, float* Q, int32_t n, int32_t c, void* stream);

/*
 * Compression codec of the spectral coefficients (Sec. 7.1; quantisation and
 * bit count as Sec. 8 evaluates it): every block's
 * coefficients are coded with `bits` bits per value by a uniform scalar
 * quantiser.  The paper fixes the bit count (q_c = 12) but not the range;
 * here each (block, column) pair has its own range [lo, hi] = [min, max] of
 * that column over the block's c_b coefficient rows, returned as side
 * information:
 *     s = (2^bits - 1) / (hi - lo),   code = clamp(rint((e - lo) s), 0, 2^bits - 1)
 * with rint rounding half to even, every operation rounded on its own in the
 * coefficients' precision (real), s = 0 (all codes 0) when hi = lo or when s
 * overflows.  Codes for NaN coefficients are unspecified.
 *   E       host or device real [sum_b c_b x cols], blocks concatenated in
 *           order (the layout of bsp_project's output for the tracked c_b).
 *   bits    1 .. 16.
 *   codes   host or device uint16 [sum_b c_b x cols].
 *   range   host or device real [k x cols x 2]: (lo, hi) of block b, column j
 *           at index 2 (b cols + j).
 * Errors: BSP_ERR_INVALID_ARG (no tracking call yet, bad cols or bits),
 * BSP_ERR_OOM, BSP_ERR_CUDA.
 */
int bsp_quantize(bsp_mesh* mesh, const void* E, int32_t cols, int32_t bits, uint16_t* codes,
                 void* range, void* stream);

/*
 * Inverse of bsp_quantize (the decoder of Sec. 7.1):
 *     e~ = lo + code (hi - lo) / (2^bits - 1)
 * each operation rounded on its own in real precision.
 *   codes, range   as written by bsp_quantize (host or device).
 *   E_out          host or device real [sum_b c_b x cols].
 */
int bsp_dequantize(bsp_mesh* mesh, const uint16_t* codes, const void* range, int32_t cols,
                   int32_t bits, void* E_out, void* stream);

/*
 * Bits per vertex of the coefficient stream for xyz coordinates (Sec. 8):
 * bpv = 3 bits (sum_b c_b) / n, the paper's 3 q_c c k / n with the tracked
 * c_b of every block; like the paper, it leaves out the connectivity and the
 * quantiser ranges (side information of 2 k reals per coordinate).
 */
int bsp_bits_per_vertex(const bsp_mesh* mesh, int32_t bits, double* bpv);

/*
 * Normalised mean square visual error between a mesh and its reconstruction
 * (Sec. 8, the NMSVE formula; mesh-wide, independent of any partition):
 *     out[0] = (out[1] + out[2]) / (2 n)
 *     out[1] = ||v - v~||            over all 3 n coordinates
 *     out[2] = ||GL(v) - GL(v~)||    GL(v)_i = v_i - sum_j v_j / d_ij / sum_j 1 / d_ij
 * with j over the distinct mesh neighbours of vertex i (edges of all faces)
 * and d_ij the edge length in the geometry GL is applied to; neighbours at
 * distance 0 get no weight, and a vertex without weighted neighbours has
 * GL(v)_i = v_i.  The paper prints the norms unsquared and the result in dB
 * without a conversion; the value here is the formula as printed, linear.
 * Accumulated in FP64 on the device.
 *   X, X_rec   host or device [n x 3] of `dtype` (BSP_DT_F32 or BSP_DT_F64).
 *   faces      host or device int32 [m x 3], vertex ids in [0, n).
 *   out        host double [3].
 * Errors: BSP_ERR_INVALID_ARG (face index out of range, bad sizes or dtype),
 * BSP_ERR_OOM, BSP_ERR_CUDA.  Allocates its own scratch and synchronises.
 */
int bsp_nmsve(const void* X, const void* X_rec, int32_t dtype, int64_t n, const int32_t* faces,
              int64_t m, double* out, void* stream);

/*
 * Fine denoising step of the coarse-to-fine denoising (Sec. 7.2), applied
 * after the coarse step v^ = U U^T v (bsp_reconstruct) or to any mesh:
 *  1. face normals, centroids and areas of X (Sec. 7.2, face normal equation;
 *     a degenerate face has normal 0 and area 0);
 *  2. normal_iters passes of the bilateral normal filter (Eqs. BF, Wm, Wn)
 *         n_i <- normalise( sum_j A_j exp(-||m_i - m_j||^2 / (2 sigma_s^2))
 *                                      exp(-||n_i - n_j||^2 / (2 sigma_r^2)) n_j )
 *     over the faces j that share a vertex with face i (i included), each
 *     pass on the previous pass's normals with the centroids and areas of X;
 *     a face whose sum vanishes keeps its normal;
 *  3. vertex_iters updates (Eqs. iter1, iter2)
 *         v <- v + (1 / |F_v|) sum_{z in F_v} n_z [n_z . (m_z - v)]
 *     with the centroids m_z at the current positions, all vertices moving
 *     from the previous iterate; a vertex in no face stays.
 * Arithmetic in the precision of `dtype` (exp as the CUDA math library
 * computes it).
 *   X, X_out      host or device [n x 3] of dtype (BSP_DT_F32 or BSP_DT_F64);
 *                 X is copied to the device first, so X_out may alias X.
 *   normals_out   NULL, or host or device [m x 3] of dtype: the filtered normals.
 *   faces         host or device int32 [m x 3], vertex ids in [0, n).
 *   sigma_s, sigma_r  kernel widths, positive; iterations >= 0.
 * Errors: BSP_ERR_INVALID_ARG (bad index, sizes, dtype or widths),
 * BSP_ERR_OOM, BSP_ERR_CUDA.  Allocates its own scratch and synchronises.
 */
int bsp_fine_denoise(const void* X, void* X_out, void* normals_out, int32_t dtype, int64_t n,
                     const int32_t* faces, int64_t m, double sigma_s, double sigma_r,
                     int32_t normal_iters, int32_t vertex_iters, void* stream);

/*
 * theta of the evaluation (Sec. 8): the mean over faces of the angle between
 * the normal of a face in X and in X_ref (same faces), atan2(||n x n'||,
 * n . n'), in degrees; faces degenerate in either mesh are left out (0 if
 * none is left).  Accumulated in FP64.
 *   X, X_ref   host or device [n x 3] of dtype (BSP_DT_F32 or BSP_DT_F64).
 *   faces      host or device int32 [m x 3].
 *   theta_deg  host double.
 */
int bsp_normal_angle_error(const void* X, const void* X_ref, int32_t dtype, int64_t n,
                           const int32_t* faces, int64_t m, double* theta_deg, void* stream);

/* Thread-local message describing the last failure on this thread ("" if none). */
const char* bsp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BSP_H_ */
