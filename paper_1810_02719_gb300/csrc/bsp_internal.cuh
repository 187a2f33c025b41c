// Internal declarations shared by the library's translation units.
//
// Device data layout ("block order"): the rows of every per-vertex array are
// the blocks' vertices concatenated, block b occupying rows
// [bptr[b], bptr[b+1]) in its local order.  Per-block CSR of the off-diagonal
// part of L[b] = D - C (Sec. 3): rowptr (global offsets, int32 [n+1]),
// col (uint16 local column ids, ascending per row), wt (real per entry, or
// null for unit weights), diag (real D_ii per row).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <array>
#include <vector>

#include "../../include/bsp.h"

namespace bsp {

// ---------------------------------------------------------------- status bits
// Device-side status word (OR-ed by kernels, read by the host after a call).
enum : int {
  ST_NUMERICAL = 1 << 0,      // Gram/Cholesky breakdown or NaN
  ST_NOT_CONVERGED = 1 << 1,  // a CG solve hit its step cap
  ST_BAD_INDEX = 1 << 2,      // assembly saw an out-of-range vertex id
  ST_DUP_VERTEX = 1 << 3,     // assembly saw a vertex in two blocks
  ST_DEGREE = 1 << 4,         // a row's neighbour list overflowed
  ST_TIMEOUT = 1 << 5,        // a bounded device wait expired
  ST_CG_BREAKDOWN = 1 << 6,   // a CG recurrence lost positivity ((p, A p) <= 0)
};

struct CgStats {
  unsigned long long steps_total;
  int steps_max;
  int not_converged;
  int jacobi_sweeps;
};

// ---------------------------------------------------------------- profiling
// Kernel classes for the optional per-class timing (CUDA events recorded on
// the launching stream around every launch, eager mode only).
enum KernelClass : int {
  KC_INIT = 0, KC_CG, KC_GRAM, KC_REDUCE, KC_CHOL, KC_PANEL, KC_RR, KC_JACOBI,
  KC_PROJECT, KC_RECON, KC_SPMM, KC_DYN, KC_OI, KC_COUNT
};
struct Profiler {
  std::vector<cudaEvent_t> ev[KC_COUNT];  // pairs (start, stop)
};
extern thread_local Profiler* g_prof;
inline void prof_begin(int cls, cudaStream_t s) {
  if (!g_prof) return;
  cudaEvent_t e;
  cudaEventCreate(&e);
  cudaEventRecord(e, s);
  g_prof->ev[cls].push_back(e);
}
inline void prof_end(int cls, cudaStream_t s) {
  if (!g_prof) return;
  cudaEvent_t e;
  cudaEventCreate(&e);
  cudaEventRecord(e, s);
  g_prof->ev[cls].push_back(e);
}

// ---------------------------------------------------------------- helpers
#define BSP_DEV __device__ __forceinline__

template <typename T>
BSP_DEV T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Let `kernel` use all the opt-in shared memory left next to its static shared
// memory.  Leaves no error behind in the runtime's last-error state.
template <typename K>
inline void set_max_dynamic_smem(K kernel) {
  cudaFuncAttributes fa;
  int dev = 0, optin = 0;
  if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         optin - (int)fa.sharedSizeBytes);
  cudaGetLastError();
}

// Thin tuple of the device-side mesh arrays passed to kernels by value.
template <typename T>
struct MeshView {
  const int32_t* bptr;     // [k+1]
  const int32_t* rowptr;   // [n+1]
  const uint16_t* col;     // [nnz]
  const T* wt;             // [nnz] or nullptr (unit weights)
  const T* diag;           // [n]
};

// ---------------------------------------------------------------- launchers
// Assembly (bsp_assemble.cu)
struct AssemblyOut {
  int32_t* rowptr = nullptr;
  uint16_t* col = nullptr;
  int32_t* eoff = nullptr;      // [n+1] canonical edge id offset per row
  int32_t* blk_row = nullptr;   // [n] block of each row
  int64_t nnz = 0;
  int64_t intra_edges = 0;
};
// Returns a bsp_status; fills `out` with device arrays owned by the caller.
int assemble_pattern(int64_t n, const int32_t* d_tri, int64_t m, int arity,
                     const int32_t* d_bptr, const int32_t* d_verts, int32_t k,
                     AssemblyOut* out, int* d_status, cudaStream_t s, std::string* err);
// out[0..n] = exclusive scan of in[0..n-1], out[n] = total (also returned on
// the host); synchronises s.
int exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int* d_status, cudaStream_t s,
                   long long* h_total);
template <typename T>
void launch_weights(int64_t n, const int32_t* bptr, const int32_t* blk_row, const int32_t* verts,
                    const int32_t* rowptr, const uint16_t* col, const double* xyz, int mode,
                    int literal, T* wt, T* diag, cudaStream_t s);
template <typename T>
void launch_set_weights(int64_t n, const int32_t* bptr, const int32_t* blk_row,
                        const int32_t* rowptr, const uint16_t* col, const int32_t* eoff,
                        const T* w_edges, int literal, T* wt, T* diag, cudaStream_t s);
void launch_edges_out(int64_t n, const int32_t* bptr, const int32_t* blk_row, const int32_t* verts,
                      const int32_t* rowptr, const uint16_t* col, const int32_t* eoff,
                      int32_t* edges, cudaStream_t s);

// Standalone SpMM (bsp_cg.cu)
template <typename T>
void launch_spmm(int64_t n, const MeshView<T>& mv, const int32_t* blk_row, T delta, const T* P,
                 T* Y, int c, cudaStream_t s);

// Fused CG solve of (L + delta I)^z Y = V per (block, column slab) (bsp_cg.cu)
struct CgArgs {
  const int32_t* batch; int nbatch;
  const int32_t* cb;        // [k] columns per block
  int ld;                   // row stride of V and Y
  int z; double delta; double rtol; int max_steps;
  int* status; CgStats* stats;
  int max_deg = 0;          // largest row degree of the mesh (selects the register-ELL kernel)
  // right-hand sides read from the rows of block vsrc[b] instead of block b
  // (a warm start read in place from a same-size parent); nullptr: own rows
  const int32_t* vsrc = nullptr;
  // [k] per-block flags: a CTA whose block has live[b] == 0 returns at once
  // (the device-driven dynamic-c rounds); nullptr: every block of the batch
  const int32_t* live = nullptr;
  // team CG tile shape: 8 or 16 rows per lane (0: 8 where the register form applies)
  int rows_per_lane = 0;
};
extern bool g_disable_cg1;  // force the shared-memory CG kernel (A/B checks)
template <typename T>
int launch_cg(const MeshView<T>& mv, const T* V, T* Y, const CgArgs& a, int cs, int max_nb,
              int c_max, cudaStream_t s);
// Batched one-column-per-CTA CG (bsp_cg.cu): the batch sorted by size bucket
// (rows per thread 1, 4, 8, 16), bucket_off[0..4] (host) delimiting the
// buckets and bucket_rows[q] the largest block of bucket q.
constexpr int kCgBuckets = 5;  // size buckets: up to 256, 512, 1,024, 2,048, 4,096 rows
int cg_bucket(int nb);   // -1 when the block is too large (> 4,096 rows)
// Streams and events on which the buckets of one batched CG launch run side
// by side (fork from the launching stream, join back into it).
struct CgFork {
  cudaStream_t aux[kCgBuckets - 1] = {};
  cudaEvent_t fork = nullptr, join[kCgBuckets - 1] = {};
};
// Team CG (bsp_cgt.cu): one column per team of 1-8 warps, the pattern in
// shared memory once per CTA; blocks up to 4,096 rows, degrees up to 16.
bool cgt_fits(int max_nb, int max_deg, int real_bytes, bool weighted);
bool cgt_reg(int max_nb, int max_deg, bool weighted);   // the 8-rows-per-lane register form applies
template <typename T>
int launch_cgt(const MeshView<T>& mv, const T* V, T* Y, const CgArgs& a, int max_nb, int c_max,
               cudaStream_t s);
void configure_cgt_kernels();
bool cg1_fits(int max_nb, int max_deg, int real_bytes, bool weighted);
template <typename T>
int launch_cg_buckets(const MeshView<T>& mv, const T* V, T* Y, const CgArgs& a,
                      const int* bucket_off, const int* bucket_rows, int c_max, cudaStream_t s,
                      const CgFork* fork = nullptr);
template <typename T>
int cg_smem_bytes(int cs, int max_nb);
void configure_cg_kernels();
void configure_dense_kernels();

// Dense small-matrix kernels (bsp_dense.cu)
struct DenseArgs {
  const int32_t* batch; int nbatch;
  const int32_t* bptr;
  const int32_t* cb;        // [k] columns per block
  int ld;                   // row stride of the n x c_cap matrices
  int cmax;                 // largest c in the batch (grid sizing)
  int max_nb;               // largest n_b in the batch
  int* status;
  int* sweeps = nullptr;    // optional: Jacobi sweeps performed (summed)
  const int32_t* live = nullptr;  // as CgArgs::live
};
template <typename T, typename TA>
int launch_cholqr2(const DenseArgs& a, const T* Y, T* Q, TA* Gp, T* Rsm, cudaStream_t s,
                   int* launches, int passes = 2);
template <typename T, typename TA>
int launch_rayleigh_ritz(const DenseArgs& a, const MeshView<T>& mv, T* V, TA* Gp, T* Rsm,
                         T* theta, cudaStream_t s, int* launches);
int dense_chunk_rows(int cpad, int real_bytes);
// Fused cluster Onorm (bsp_fused.cu); BSP_ERR_INVALID_ARG when the shape does not fit.
template <typename T, typename TA>
int launch_cholqr2_fused(const DenseArgs& a, const T* Y, T* Q, TA* Gp, int maxch, cudaStream_t s,
                         int passes);
void configure_fused_kernels();
template <typename T, typename TA>
int launch_reduce_chol(const DenseArgs& a, int CH, int maxch, const TA* Gp, TA* G, T* Rsm,
                       cudaStream_t s);
// One CholeskyQR pass with both contractions on the tensor cores (bsp_tcqr.cu;
// FP32 operands, c <= 64); BSP_ERR_INVALID_ARG when the shape does not fit.
bool tcqr_fits(int cmax, int real_bytes);
template <typename TA>
int launch_cholqr_pass_tc(const DenseArgs& a, const float* Y, float* Q, TA* Gp, float* Rsm,
                          cudaStream_t s, int* launches);
void configure_tcqr_kernels();
void set_last_error(const char* msg);  // message for bsp_last_error() on this thread
extern bool g_disable_fused;  // force the multi-kernel Onorm (A/B checks)

// Persistent cluster engine of the fixed-c schedule (bsp_oi_cluster.cu): every
// block's solves and CholeskyQR2 on chip, blocks in topological order, one
// cluster of ceil(c / 4) CTAs per dependency path, bounded waits on the
// parents' ready flags between clusters.
struct OiClusterArgs {
  const int32_t* order; int nblocks;   // blocks in topological (wave) order
  int k;                               // blocks of the mesh (ready has k + 2 slots)
  const int32_t* parent; const int32_t* root_off;
  const float* starts;                 // roots' start rows, [root rows x c]
  float* U; int ld; int c;
  int t_max; int z; double delta; double rtol; int max_steps;
  int* ready;                          // [k] flags, [k] abort word, [k + 1] never set
  int* status; CgStats* stats;
  long long wait_limit_us;             // bound of one wait for a parent's flag
  int withhold;                        // test hook: this block's wait never sees its flag
  int rpm = 0;                         // panel rows per CTA (set by the launcher)
};
extern bool g_disable_oi_cluster;      // force the per-wave launches (A/B checks)
bool oi_cluster_fits(int c, int t_max, int max_nb, int max_deg, int min_nb);
// Outside any stream capture: sets the kernel's attributes and returns in
// *nclusters how many clusters run at once (at most max_wave);
// BSP_ERR_INVALID_ARG when the cluster shape cannot be resident (the caller
// falls back to the per-wave launches).
int prepare_oi_cluster(const MeshView<float>& mv, int c, int max_nb, int max_deg, int max_wave,
                       int* nclusters);
int launch_oi_cluster(const MeshView<float>& mv, const OiClusterArgs& a, int max_nb, int max_deg,
                      int nclusters, cudaStream_t s);

// Projection / reconstruction (bsp_proj.cu)
struct ProjArgs {
  const int32_t* bptr; const int32_t* verts; const int32_t* cb; const int32_t* eoff;
  int k; int ld; int cmax; int max_nb; int cols;
};
template <typename T>
int launch_project(const ProjArgs& a, const T* U, const void* X, int x_dtype, T* E,
                   cudaStream_t s);
template <typename T>
int launch_reconstruct(const ProjArgs& a, const T* U, const T* E, T* X, cudaStream_t s);
// tcgen05 tensor-core versions, BF16 operands, FP32 accumulation (bsp_tc.cu);
// Ub is the BF16 copy of the basis written by launch_basis_bf16 (pad16(cmax)
// columns per row, zero past each block's c).
int launch_basis_bf16(const ProjArgs& a, const float* U, void* Ub, cudaStream_t s);
int launch_project_tc(const ProjArgs& a, const void* Ub, const void* X, float* E, int* status,
                      cudaStream_t s);
int launch_recon_tc(const ProjArgs& a, const void* Ub, const float* E, int64_t erows, void* Eb,
                    float* X, int* status, cudaStream_t s);
void configure_tc_kernels();

// Tiled operator product (bsp_spmm.cu): chunks of up to 64 rows inside a
// block, each with the row range [lo, hi] that its neighbours reach (8 int32
// per chunk in the table).
void configure_spmm_kernels();
void configure_dyn_kernels();
std::vector<int32_t> spmm_chunk_rows(const std::vector<int32_t>& bptr);
void launch_spmm_ranges(const MeshView<float>& mv_any, const int32_t* blk_row, int32_t* chunks,
                        int nchunks, cudaStream_t s);
template <typename T>
int launch_spmm_tiled(const MeshView<T>& mv, const int32_t* chunks, int nchunks, int max_span,
                      int max_nnz, T delta, const T* P, T* Y, int c, cudaStream_t s);

// Coefficient quantiser and NMSVE (bsp_codec.cu).  ceoff: [k + 1] row offsets
// of the blocks' coefficients; range: [k x cols x 2] (lo, hi).
template <typename T>
int launch_quantize(const int32_t* ceoff, int k, const T* E, int cols, int bits, uint16_t* codes,
                    T* range, cudaStream_t s);
template <typename T>
int launch_dequantize(const int32_t* ceoff, int k, const uint16_t* codes, const T* range, int cols,
                      int bits, T* E, cudaStream_t s);
void launch_nm_count(int64_t m, const int32_t* faces, int64_t n, int32_t* cnt, int* status,
                     cudaStream_t s);
void launch_nm_fill(int64_t m, const int32_t* faces, int64_t n, const int32_t* off, int32_t* cur,
                    int32_t* nbr, cudaStream_t s);
template <typename T>
int launch_nm_err(int64_t n, const int32_t* off, const int32_t* nbr, const T* X, const T* Xr,
                  double* acc, cudaStream_t s);

// Fine denoising and normal-angle metric (bsp_denoise.cu).  The vertex -> face
// table: counts (status bit ST_BAD_INDEX on a bad face), then after a scan the
// fill and a per-vertex sort.
void launch_vf_table(int64_t m, const int32_t* faces, int64_t n, int32_t* cnt, int* status,
                     cudaStream_t s);
void launch_vf_fill(int64_t m, const int32_t* faces, int64_t n, const int32_t* off, int32_t* cur,
                    int32_t* vf, cudaStream_t s);
template <typename T>
int launch_fine_denoise(int64_t n, int64_t m, const int32_t* faces, const int32_t* off,
                        const int32_t* vf, T* X0, T* X1, T* n0, T* n1, T* cen, T* area,
                        double sigma_s, double sigma_r, int normal_iters, int vertex_iters,
                        T** X_final, T** n_final, cudaStream_t s);
template <typename T>
int launch_normal_angle(int64_t m, const int32_t* faces, const T* X, const T* Xr, double* acc,
                        unsigned long long* cnt, cudaStream_t s);

// Start matrices and dynamic-c helpers (bsp_dyn.cu)
template <typename T>
void launch_init_starts(const int32_t* batch, int nbatch, const int32_t* bptr,
                        const int32_t* parent, const int32_t* root_off, const int32_t* cb,
                        const int32_t* cpar, const T* starts, int ld_start, T* U, int ld,
                        int max_nb, int cmax, cudaStream_t s, const T* Usrc = nullptr);
// live (optional, [k]): the decision clears live[b] unless block b grows
// (not met and below min(c_max, n_b rounded down to c_step)); the growth step
// skips blocks with live[b] == 0 and advances round[b] of the others.
template <typename T, typename TA>
int launch_dyn_decide(const int32_t* batch, int nbatch, const int32_t* bptr, const int32_t* verts,
                      const T* X, const T* U, int ld, int32_t* cb, int32_t* action,
                      const int32_t* forced, double tol, int c_step, int c_max, T* gcol,
                      TA* rho_out, int max_nb, cudaStream_t s, int32_t* live = nullptr);
template <typename T, typename TA>
int launch_dyn_grow(const int32_t* batch, int nbatch, const int32_t* bptr, int32_t* cb,
                    int32_t* round, T* U, int ld, const T* gcol, uint64_t seed,
                    int c_step, int max_nb, cudaStream_t s, const int32_t* live = nullptr);

// Device-side control of the dynamic-c schedule: one wave's state between
// rounds.  A graph replays the rounds under conditional nodes (a WHILE over
// rounds, a SWITCH over width classes) whose values these kernels set; the
// eager path reads the same fields back instead.
struct DynCtl {
  int cls_start;                 // width class of the wave's start bases
  int cls_round;                 // width class of the next round (largest live width)
  int more;                      // another round follows
  int rounds;                    // rounds run in this wave
  unsigned long long launches;   // kernels launched by the schedule (summed over the call)
};
// Wave start: widths (root c_min, child min(parent width, c_max, n_b rounded
// down)), parent widths, live = 1, round = 0; the start's width class.
// Launch counts: ctl->launches += start_launches[class] + 1.
int launch_dyn_wave_init(const int32_t* wave, int nw, const int32_t* bptr, const int32_t* parent,
                         int32_t* cb, int32_t* cpar, int32_t* live, int32_t* round, int c_min,
                         int c_max, int c_step, int cls_width, int ncls,
                         const unsigned* start_launches, DynCtl* ctl, int set_handle,
                         cudaGraphConditionalHandle h_start, cudaStream_t s);
// Round class: the largest width among live blocks -> ctl->cls_round and the
// SWITCH handle; ctl->launches += round_launches[class] + base (base: this
// kernel and the round's end, 2; a final class with no end kernel, 1).
int launch_dyn_class(const int32_t* wave, int nw, const int32_t* cb, const int32_t* live,
                     int cls_width, int ncls, const unsigned* round_launches, DynCtl* ctl,
                     int set_handle, cudaGraphConditionalHandle h_round, cudaStream_t s,
                     unsigned base = 2);
// Round end: ctl->more = any live block and fewer than max_rounds rounds run;
// sets the WHILE handle.
int launch_dyn_next(const int32_t* wave, int nw, const int32_t* live, int max_rounds, DynCtl* ctl,
                    int set_handle, cudaGraphConditionalHandle h_while, cudaStream_t s);

// Overlapped parts (bsp_overlap.cu): copy weights and copy counts per vertex,
// then (after a scan of the counts) the per-vertex copy lists in copy order,
// then the degree-weighted mean of Algorithm 3 (Sec. 6.1).
int launch_ov_table(int64_t rows, const int32_t* verts, const int32_t* rowptr, const int32_t* orig,
                    int64_t n_orig, float* w, int32_t* cnt, int* status, cudaStream_t s);
int launch_ov_fill(int64_t rows, const int32_t* orig, int64_t n_orig, const int32_t* off,
                   int32_t* cur, int32_t* list, cudaStream_t s);
template <typename T>
int launch_ov_merge(int64_t n_orig, int cols, const int32_t* off, const int32_t* list,
                    const float* w, const T* Xc, T* Xo, cudaStream_t s);

// The paper's dynamic OI (Sec. 5, Algorithm 2): per block of the batch, the
// summed residual e and the grow / shrink / stop decision (bsp_dyn.cu).
// live (optional): blocks with live[b] == 0 are skipped and a stopping block
// clears its flag; ctl (optional): the iteration number is ctl->rounds + 1
// instead of t (device-driven rounds).
template <typename T>
int launch_doi_decide(const int32_t* batch, int nbatch, const int32_t* bptr, const int32_t* verts,
                      const T* X, T* U, int ld, int32_t* cb, int32_t* done, int t, double eps_l,
                      double eps_h, int c_min, int c_max, T* gcol, double* enorm, cudaStream_t s,
                      int32_t* live = nullptr, const struct DynCtl* ctl = nullptr);

// Adjoint of the low-pass filter (bsp_adjoint.cu)
struct AdjointArgs {
  const int32_t* batch; int k;          // all blocks
  const int32_t* bptr; const int32_t* cb; const int32_t* verts;
  const int32_t* blk_row; const int32_t* eoff;
  int64_t n; int64_t n_edges; int ld; int c; int t_max; int max_nb;
  const void* X; const void* G;         // device [n x 3]
  const void* ckV; const void* ckY;     // checkpoints: V_0..V_t, Y_1..Y_t, each [n x ld]
  void* ws_gp; void* ws_thin; void* ws_rows;
  void* dW;                             // device [n_edges]
  int* status; CgStats* cgstats;
  int z; double delta; double rtol; int max_steps; int max_deg; int cs;
};
int adjoint_maxch(int max_nb);
template <typename T, typename TA>
int launch_filter_backward(const AdjointArgs& aa, const MeshView<T>& mv, cudaStream_t s);
void configure_adjoint_kernels();

}  // namespace bsp

// ---------------------------------------------------------------- the mesh
struct bsp_mesh {
  int64_t n = 0;
  int32_t k = 0;
  bsp_opts opts{};
  int real_bytes = 4;
  int32_t max_nb = 0, min_nb = 0;
  int32_t max_deg = 0;     // largest number of intra-block neighbours of a vertex
  int64_t nnz = 0, intra_edges = 0;
  std::vector<int32_t> h_bptr, h_parent, h_level, h_root_off, h_c;
  std::vector<std::vector<int32_t>> waves;
  std::vector<int32_t> h_wave_list;      // all waves concatenated
  std::vector<int32_t> h_wave_off;       // [levels+1]
  std::vector<std::array<int, bsp::kCgBuckets + 1>> wave_bucket;  // CG size-bucket offsets per wave
  std::vector<std::array<int, bsp::kCgBuckets>> wave_bucket_rows;  // largest block per bucket
  bsp::CgFork cg_fork;   // side streams of the batched CG (created before the first capture)
  cudaStream_t post_stream = nullptr;   // deferred work of the engine's ranges
  cudaEvent_t post_ev[2] = {nullptr, nullptr};
  int64_t root_rows = 0;
  // device arrays
  int32_t *d_bptr = nullptr, *d_verts = nullptr, *d_rowptr = nullptr, *d_eoff = nullptr,
          *d_blk_row = nullptr, *d_parent = nullptr, *d_root_off = nullptr,
          *d_waves = nullptr, *d_cb = nullptr, *d_cpar = nullptr, *d_ceoff = nullptr;
  uint16_t* d_col = nullptr;
  void* d_wt = nullptr;
  void* d_diag = nullptr;
  int* d_status = nullptr;
  bsp::CgStats* d_cgstats = nullptr;
  // tracking state and workspace
  int32_t c_cap = 0;       // row stride (columns) of d_U / d_Y
  bool tracked = false;
  void* d_U = nullptr;
  void* d_Y = nullptr;
  void* d_starts = nullptr;
  void* d_Gp = nullptr;
  void* d_Rsm = nullptr;
  void* d_theta = nullptr;
  size_t cap_U = 0, cap_starts = 0, cap_Gp = 0, cap_Rsm = 0, cap_theta = 0;
  // dynamic-c workspace
  int32_t *d_action = nullptr, *d_round = nullptr, *d_forced = nullptr;
  void* d_gcol = nullptr;
  void* d_rho = nullptr;
  void* d_X = nullptr;
  size_t cap_X = 0;
  // BF16 copy of the tracked bases for the tensor-core projection and
  // reconstruction; rebuilt on first use after every tracking call
  void* d_Ubf = nullptr;
  size_t cap_Ubf = 0;
  bool ubf_valid = false;
  int* d_ready = nullptr;              // cluster engine: ready flags + abort word
  size_t cap_ready = 0;
  int engine_c = -1, engine_ncl = 0;   // engine prepared for width c: clusters (0: not usable)
  int32_t* d_spmm_chunks = nullptr;   // tiled operator product: 8 int32 per chunk
  int spmm_nchunks = 0, spmm_max_span = 0, spmm_max_nnz = 0;
  void* d_Ebf = nullptr;   // BF16 copy of the coefficients of a reconstruction call
  size_t cap_Ebf = 0;
  // Rayleigh-Ritz of the fixed-c schedule: block groups (offsets into the
  // wave order, largest block of each) and their workspace
  std::vector<int32_t> rr_group, rr_wmax;
  void* d_Gp_rr = nullptr;
  void* d_Rsm_rr = nullptr;
  void* d_theta_rr = nullptr;
  size_t cap_Gp_rr = 0, cap_Rsm_rr = 0, cap_theta_rr = 0;
  // graph cache for the fixed-c schedule
  cudaGraphExec_t graph_exec = nullptr;
  int graph_c = -1, graph_t = -1, graph_launches = 0, graph_cs = -1, graph_rpl = -1;
  cudaStream_t graph_stream = nullptr;
  // dynamic-c schedule: device state and its graph (conditional nodes), keyed
  // by the call's parameters
  int32_t* d_live = nullptr;
  bsp::DynCtl* d_dynctl = nullptr;
  unsigned* d_dyn_launches = nullptr;  // per wave: start and round launch counts per class
  size_t cap_dyn_launches = 0;
  cudaGraphExec_t dyn_exec = nullptr;
  std::vector<double> dyn_key;
  cudaGraphExec_t doi_exec = nullptr;   // the paper's dynamic OI, same machinery
  std::vector<double> doi_key;
  cudaStream_t dyn_stream[2] = {nullptr, nullptr};
  bsp_stats stats{};
  // low-pass filter checkpoints (last bsp_filter_forward)
  void* d_ckV = nullptr;
  void* d_ckY = nullptr;
  void* d_adj_gp = nullptr;
  void* d_adj_thin = nullptr;
  void* d_adj_rows = nullptr;
  size_t cap_ckV = 0, cap_ckY = 0, cap_adj_gp = 0, cap_adj_thin = 0, cap_adj_rows = 0;
  int filter_c = 0, filter_t = -1;
  // optional per-kernel-class timing (eager launches, CUDA events)
  int profiling = 0;
  double prof_ms[bsp::KC_COUNT] = {};
  int32_t prof_n[bsp::KC_COUNT] = {};
};
