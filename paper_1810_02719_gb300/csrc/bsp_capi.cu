// C ABI of the library (declared in include/bsp.h): argument checking, device
// buffers, the schedule of kernels over the block forest, and CUDA-graph
// capture of the fixed-c schedule.
//
// Schedule (Sec. 4, Algorithm 1, blocks in topological order): blocks at the
// same depth of the warm-start forest are independent and form one wave; a
// wave runs as one launch of each kernel with the wave's blocks on the grid's
// y axis.  Per wave: start matrices (root rows or row-transferred parent
// basis) -> Onorm where the start is not already orthonormal -> t_max times
// {CG solve of (L + delta I)^z Y = V; Onorm (CholeskyQR2)} -> Rayleigh-Ritz.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "bsp_internal.cuh"

using namespace bsp;

namespace bsp {
thread_local Profiler* g_prof = nullptr;
}

namespace {
thread_local std::string g_err;
}

namespace bsp {
// The thread-local message returned by bsp_last_error().
void set_last_error(const char* msg) { g_err = msg; }
}

namespace {

// Collects the events of a profiled call after its stream has synchronised.
struct ProfScope {
  bsp_mesh* M;
  Profiler P;
  explicit ProfScope(bsp_mesh* m) : M(m) {
    if (M && M->profiling) g_prof = &P;
  }
  ~ProfScope() {
    if (!M || !M->profiling) return;
    g_prof = nullptr;
    for (int c = 0; c < KC_COUNT; ++c) {
      auto& v = P.ev[c];
      for (size_t i = 0; i + 1 < v.size(); i += 2) {
        float ms = 0.f;
        if (cudaEventSynchronize(v[i + 1]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, v[i], v[i + 1]) == cudaSuccess) {
          M->prof_ms[c] += ms;
          M->prof_n[c] += 1;
        }
      }
      for (auto e : v) cudaEventDestroy(e);
    }
    cudaGetLastError();
  }
};

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CU(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(BSP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Copy `bytes` of host data into a host-or-device destination (synchronises s).
int to_host_or_device(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return BSP_OK;
  CU(cudaStreamSynchronize(s));
  if (is_device_ptr(dst)) {
    CU(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice));
  } else {
    std::memcpy(dst, src, bytes);
  }
  return BSP_OK;
}

// Copy `bytes` from a host-or-device pointer into a device buffer.
int to_device(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return BSP_OK;
  cudaMemcpyKind kind = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CU(cudaMemcpyAsync(dst, src, bytes, kind, s));
  return BSP_OK;
}

// Copy from a device buffer to a host-or-device destination.
int from_device(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return BSP_OK;
  cudaMemcpyKind kind = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CU(cudaMemcpyAsync(dst, src, bytes, kind, s));
  return BSP_OK;
}

// Read a host-or-device array into a host vector.
template <typename V>
int read_host(std::vector<V>& out, const V* src, size_t count) {
  out.resize(count);
  if (count == 0) return BSP_OK;
  if (is_device_ptr(src)) {
    CU(cudaMemcpy(out.data(), src, count * sizeof(V), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(out.data(), src, count * sizeof(V));
  }
  return BSP_OK;
}

// ensure() replaced a buffer during this thread's current call (cached graphs go stale)
thread_local bool g_realloc = false;

int ensure(void** p, size_t* cap, size_t bytes) {
  if (*cap >= bytes && *p) return BSP_OK;
  g_realloc = true;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    return fail(BSP_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  *cap = bytes;
  return BSP_OK;
}

void configure_once() {
  static std::once_flag flag;
  std::call_once(flag, [] {
    configure_cg_kernels();
    configure_cgt_kernels();
    configure_tcqr_kernels();
    configure_dense_kernels();
    configure_adjoint_kernels();
    configure_tc_kernels();
    configure_spmm_kernels();
    configure_dyn_kernels();
  });
}

// Sort a batch by the size bucket of the batched CG (cg_bucket; blocks too
// large last) and return the bucket offsets off[0..kCgBuckets] and the
// largest block of every bucket.
void sort_by_bucket(const bsp_mesh* M, std::vector<int32_t>& list, int* off, int* rows) {
  auto nb = [&](int b) { return M->h_bptr[b + 1] - M->h_bptr[b]; };
  auto key = [&](int b) {
    const int q = cg_bucket(nb(b));
    return q < 0 ? kCgBuckets : q;
  };
  std::stable_sort(list.begin(), list.end(), [&](int a, int b) { return key(a) < key(b); });
  off[0] = 0;
  for (int q = 0; q < kCgBuckets; ++q) {
    int cnt = 0, mx = 0;
    for (int b : list)
      if (key(b) == q) {
        ++cnt;
        mx = std::max(mx, nb(b));
      }
    off[q + 1] = off[q] + cnt;
    rows[q] = mx;
  }
}

// The batched CG (team kernel, or one column per CTA), launched per size
// bucket, for batches of several blocks (automatic column choice only; slab
// widths set by the caller keep the shared-memory slab kernel).
bool use_buckets(const bsp_mesh* M, int nbatch, int wmax) {
  return M->opts.cols_per_cta == 0 && nbatch >= 2 &&
         (cgt_fits(wmax, M->max_deg, M->real_bytes, M->d_wt != nullptr) ||
          cg1_fits(wmax, M->max_deg, M->real_bytes, M->d_wt != nullptr));
}

int pad4(int c) { return (c + 3) & ~3; }

void release(bsp_mesh* m) {
  void* ptrs[] = {m->d_bptr, m->d_verts, m->d_rowptr, m->d_eoff, m->d_blk_row, m->d_parent,
                  m->d_root_off, m->d_waves, m->d_cb, m->d_cpar, m->d_ceoff, m->d_col,
                  m->d_wt, m->d_diag, m->d_status, m->d_cgstats, m->d_U, m->d_Y, m->d_starts,
                  m->d_Gp, m->d_Rsm, m->d_theta, m->d_action, m->d_round, m->d_forced,
                  m->d_gcol, m->d_rho, m->d_X, m->d_Gp_rr, m->d_Rsm_rr, m->d_theta_rr,
                  m->d_ckV, m->d_ckY,
                  m->d_adj_gp, m->d_adj_thin, m->d_adj_rows, m->d_Ubf, m->d_Ebf,
                  m->d_spmm_chunks, m->d_ready, m->d_live, m->d_dynctl, m->d_dyn_launches};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (m->graph_exec) cudaGraphExecDestroy(m->graph_exec);
  if (m->dyn_exec) cudaGraphExecDestroy(m->dyn_exec);
  if (m->doi_exec) cudaGraphExecDestroy(m->doi_exec);
  if (m->graph_stream) cudaStreamDestroy(m->graph_stream);
  for (cudaStream_t q : m->dyn_stream)
    if (q) cudaStreamDestroy(q);
  for (int q = 0; q < kCgBuckets - 1; ++q) {
    if (m->cg_fork.aux[q]) cudaStreamDestroy(m->cg_fork.aux[q]);
    if (m->cg_fork.join[q]) cudaEventDestroy(m->cg_fork.join[q]);
  }
  if (m->cg_fork.fork) cudaEventDestroy(m->cg_fork.fork);
  if (m->post_stream) cudaStreamDestroy(m->post_stream);
  for (cudaEvent_t e : m->post_ev)
    if (e) cudaEventDestroy(e);
}

int stream_error_status(bsp_mesh* m, cudaStream_t s) {
  CU(cudaStreamSynchronize(s));
  int st = 0;
  CgStats cs{};
  CU(cudaMemcpy(&st, m->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(&cs, m->d_cgstats, sizeof(CgStats), cudaMemcpyDeviceToHost));
  m->stats.cg_steps_total = (int64_t)cs.steps_total;
  m->stats.cg_steps_max = cs.steps_max;
  m->stats.not_converged = cs.not_converged;
  m->stats.jacobi_sweeps = cs.jacobi_sweeps;
  if (st & ST_NUMERICAL)
    return fail(BSP_ERR_NUMERICAL, "Gram matrix not positive definite or non-finite values");
  if (st & ST_CG_BREAKDOWN)
    return fail(BSP_ERR_NUMERICAL, "CG breakdown: (p, A p) <= 0 or a non-finite recurrence");
  if (st & ST_TIMEOUT) return fail(BSP_ERR_TIMEOUT, "a bounded device wait expired");
  if (st & ST_NOT_CONVERGED)
    return fail(BSP_ERR_NOT_CONVERGED,
                std::to_string(cs.not_converged) + " CG solves hit the step cap");
  return BSP_OK;
}

// ------------------------------------------------------------------ create
int create_common(const double* xyz, int64_t n, const int32_t* tri, int64_t m, int arity,
                  const int32_t* block_ptr, const int32_t* block_verts, int32_t k,
                  const int32_t* parent, const bsp_opts* opts, bsp_mesh** out) {
  if (!out) return fail(BSP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n <= 0 || k <= 0 || m < 0) return fail(BSP_ERR_INVALID_ARG, "n, k must be positive");
  if (!tri && m > 0) return fail(BSP_ERR_INVALID_ARG, "faces/edges is NULL");
  if (!block_ptr || !block_verts || !parent)
    return fail(BSP_ERR_INVALID_ARG, "block_ptr, block_verts and parent are required");
  if (n > INT32_MAX / 2) return fail(BSP_ERR_INVALID_ARG, "n too large");
  bsp_opts o;
  bsp_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.delta > 0.0)) return fail(BSP_ERR_INVALID_ARG, "delta must be positive");
  if (o.z < 1) return fail(BSP_ERR_INVALID_ARG, "z must be >= 1");
  if (o.precision < 0 || o.precision > 2) return fail(BSP_ERR_INVALID_ARG, "bad precision");
  if (o.weight_mode < 0 || o.weight_mode > 2) return fail(BSP_ERR_INVALID_ARG, "bad weight mode");
  if (o.weight_mode == BSP_W_INV_SQ_DIST && !xyz)
    return fail(BSP_ERR_INVALID_ARG, "inverse-square-distance weights need xyz");
  if (!(o.cg_rtol > 0.0)) return fail(BSP_ERR_INVALID_ARG, "cg_rtol must be positive");
  if (o.cg_max_steps < 1) return fail(BSP_ERR_INVALID_ARG, "cg_max_steps must be >= 1");
  if (o.cols_per_cta != 0 && o.cols_per_cta != 1 && o.cols_per_cta != 2 && o.cols_per_cta != 4 &&
      o.cols_per_cta != 8)
    return fail(BSP_ERR_INVALID_ARG, "cols_per_cta must be 0, 1, 2, 4 or 8");
  configure_once();

  bsp_mesh* M = new (std::nothrow) bsp_mesh();
  if (!M) return fail(BSP_ERR_OOM, "host allocation failed");
  M->n = n;
  M->k = k;
  M->opts = o;
  M->real_bytes = o.precision == BSP_PREC_F64 ? 8 : 4;
  int rc = BSP_OK;
  cudaStream_t s = 0;
  auto bail = [&](int code) {
    release(M);
    delete M;
    return code;
  };
  // host-side validation of the partition and the block order
  if ((rc = read_host(M->h_bptr, block_ptr, (size_t)k + 1)) != BSP_OK) return bail(rc);
  if ((rc = read_host(M->h_parent, parent, (size_t)k)) != BSP_OK) return bail(rc);
  if (M->h_bptr[0] != 0 || M->h_bptr[k] != n)
    return bail(fail(BSP_ERR_INVALID_ARG, "block_ptr must start at 0 and end at n"));
  M->max_nb = 0;
  M->min_nb = INT32_MAX;
  for (int b = 0; b < k; ++b) {
    int nb = M->h_bptr[b + 1] - M->h_bptr[b];
    if (nb <= 0) return bail(fail(BSP_ERR_INVALID_ARG, "empty or decreasing block " + std::to_string(b)));
    if (nb > 65535) return bail(fail(BSP_ERR_INVALID_ARG, "block larger than 65535 vertices"));
    M->max_nb = std::max(M->max_nb, nb);
    M->min_nb = std::min(M->min_nb, nb);
    int p = M->h_parent[b];
    if (p >= b || p < -1)
      return bail(fail(BSP_ERR_INVALID_ARG, "parent[" + std::to_string(b) + "] must be -1 or < b"));
  }
  // waves: depth in the forest
  M->h_level.assign(k, 0);
  M->h_root_off.assign(k, -1);
  int levels = 0;
  for (int b = 0; b < k; ++b) {
    int p = M->h_parent[b];
    M->h_level[b] = p < 0 ? 0 : M->h_level[p] + 1;
    levels = std::max(levels, M->h_level[b] + 1);
    if (p < 0) {
      M->h_root_off[b] = (int32_t)M->root_rows;
      M->root_rows += M->h_bptr[b + 1] - M->h_bptr[b];
    }
  }
  M->waves.assign(levels, {});
  for (int b = 0; b < k; ++b) M->waves[M->h_level[b]].push_back(b);
  M->wave_bucket.assign(levels, {});
  M->wave_bucket_rows.assign(levels, {});
  for (int l = 0; l < levels; ++l)
    sort_by_bucket(M, M->waves[l], M->wave_bucket[l].data(), M->wave_bucket_rows[l].data());
  M->h_wave_off.assign(levels + 1, 0);
  for (int l = 0; l < levels; ++l) {
    M->h_wave_off[l + 1] = M->h_wave_off[l] + (int32_t)M->waves[l].size();
    for (int b : M->waves[l]) M->h_wave_list.push_back(b);
  }
  // device copies of the inputs
  int32_t* d_tri = nullptr;
  double* d_xyz = nullptr;
  auto dmalloc = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  if (!dmalloc((void**)&M->d_bptr, sizeof(int32_t) * (k + 1)) ||
      !dmalloc((void**)&M->d_verts, sizeof(int32_t) * n) ||
      !dmalloc((void**)&M->d_parent, sizeof(int32_t) * k) ||
      !dmalloc((void**)&M->d_root_off, sizeof(int32_t) * k) ||
      !dmalloc((void**)&M->d_waves, sizeof(int32_t) * 3 * k) ||
      !dmalloc((void**)&M->d_cb, sizeof(int32_t) * k) ||
      !dmalloc((void**)&M->d_cpar, sizeof(int32_t) * k) ||
      !dmalloc((void**)&M->d_ceoff, sizeof(int32_t) * (k + 1)) ||
      !dmalloc((void**)&M->d_status, sizeof(int)) ||
      !dmalloc((void**)&M->d_cgstats, sizeof(CgStats)) ||
      !dmalloc((void**)&d_tri, sizeof(int32_t) * arity * (m > 0 ? m : 1)))
    return bail(fail(BSP_ERR_OOM, "device allocation failed"));
  auto cleanup_inputs = [&]() {
    if (d_tri) cudaFree(d_tri);
    if (d_xyz) cudaFree(d_xyz);
  };
  if ((rc = to_device(M->d_bptr, M->h_bptr.data(), sizeof(int32_t) * (k + 1), s)) ||
      (rc = to_device(M->d_verts, block_verts, sizeof(int32_t) * n, s)) ||
      (rc = to_device(M->d_parent, M->h_parent.data(), sizeof(int32_t) * k, s)) ||
      (rc = to_device(M->d_root_off, M->h_root_off.data(), sizeof(int32_t) * k, s)) ||
      (rc = to_device(M->d_waves, M->h_wave_list.data(), sizeof(int32_t) * k, s)) ||
      (rc = to_device(d_tri, tri, sizeof(int32_t) * arity * m, s))) {
    cleanup_inputs();
    return bail(rc);
  }
  cudaMemsetAsync(M->d_status, 0, sizeof(int), s);
  AssemblyOut ao;
  std::string err;
  rc = assemble_pattern(n, d_tri, m, arity, M->d_bptr, M->d_verts, k, &ao, M->d_status, s, &err);
  M->d_rowptr = ao.rowptr;
  M->d_col = ao.col;
  M->d_eoff = ao.eoff;
  M->d_blk_row = ao.blk_row;
  if (rc != BSP_OK) {
    cleanup_inputs();
    return bail(fail(rc, err.empty() ? "assembly failed" : err));
  }
  M->nnz = ao.nnz;
  M->intra_edges = ao.intra_edges;
  {
    std::vector<int32_t> rp(n + 1);
    if (cudaMemcpy(rp.data(), M->d_rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cleanup_inputs();
      return bail(fail(BSP_ERR_CUDA, "copy of row pointers failed"));
    }
    for (int64_t i = 0; i < n; ++i) M->max_deg = std::max(M->max_deg, rp[i + 1] - rp[i]);
  }
  // weights and degrees
  const int rb = M->real_bytes;
  if (!dmalloc(&M->d_diag, (size_t)rb * n)) {
    cleanup_inputs();
    return bail(fail(BSP_ERR_OOM, "device allocation failed"));
  }
  if (o.weight_mode != BSP_W_COMBINATORIAL) {
    if (!dmalloc(&M->d_wt, (size_t)rb * (M->nnz > 0 ? M->nnz : 1))) {
      cleanup_inputs();
      return bail(fail(BSP_ERR_OOM, "device allocation failed"));
    }
  }
  if (o.weight_mode == BSP_W_INV_SQ_DIST) {
    if (!dmalloc((void**)&d_xyz, sizeof(double) * 3 * n) ||
        to_device(d_xyz, xyz, sizeof(double) * 3 * n, s) != BSP_OK) {
      cleanup_inputs();
      return bail(fail(BSP_ERR_OOM, "device allocation failed"));
    }
  }
  if (rb == 8)
    launch_weights<double>(n, M->d_bptr, M->d_blk_row, M->d_verts, M->d_rowptr, M->d_col, d_xyz,
                           o.weight_mode, o.literal_degree, (double*)M->d_wt, (double*)M->d_diag, s);
  else
    launch_weights<float>(n, M->d_bptr, M->d_blk_row, M->d_verts, M->d_rowptr, M->d_col, d_xyz,
                          o.weight_mode, o.literal_degree, (float*)M->d_wt, (float*)M->d_diag, s);
  cudaError_t e = cudaStreamSynchronize(s);
  cleanup_inputs();
  if (e != cudaSuccess) return bail(fail(BSP_ERR_CUDA, cudaGetErrorString(e)));
  M->stats.n = n;
  M->stats.k = k;
  M->stats.nnz = M->nnz;
  M->stats.intra_edges = M->intra_edges;
  M->stats.max_block = M->max_nb;
  M->stats.levels = levels;
  // side stream and events of the deferred work of the engine's ranges
  if (cudaStreamCreateWithFlags(&M->post_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&M->post_ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&M->post_ev[1], cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(BSP_ERR_CUDA, "stream creation failed"));
  // side streams of the batched CG (bucket launches run side by side)
  for (int q = 0; q < kCgBuckets - 1; ++q)
    if (cudaStreamCreateWithFlags(&M->cg_fork.aux[q], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&M->cg_fork.join[q], cudaEventDisableTiming) != cudaSuccess)
      return bail(fail(BSP_ERR_CUDA, "stream creation failed"));
  if (cudaEventCreateWithFlags(&M->cg_fork.fork, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(BSP_ERR_CUDA, "event creation failed"));
  *out = M;
  return BSP_OK;
}

// ------------------------------------------------------------------ tracking
template <typename T>
MeshView<T> view(const bsp_mesh* M) {
  MeshView<T> v;
  v.bptr = M->d_bptr;
  v.rowptr = M->d_rowptr;
  v.col = M->d_col;
  v.wt = (const T*)M->d_wt;
  v.diag = (const T*)M->d_diag;
  return v;
}

int pick_cs(const bsp_mesh* M, int nbatch, int c, int rb) {
  int cs = M->opts.cols_per_cta;
  if (cs == 0) {
    cs = 8;
    while (cs > 1 && (int64_t)nbatch * ((c + cs - 1) / cs) * 2 <= 152) cs /= 2;
  }
  while (cs > 1 && (size_t)4 * M->max_nb * cs * rb > 200 * 1024) cs /= 2;
  return cs;
}

// Workspace for `cmax` columns over batches of up to `maxbatch` blocks.
template <typename T, typename TA>
int ensure_workspace(bsp_mesh* M, int c_cap, int maxbatch) {
  const int cpad = pad4(c_cap);
  const int CH = dense_chunk_rows(cpad, (int)sizeof(T));
  const int maxch = (M->max_nb + CH - 1) / CH;
  const size_t gp = ((size_t)maxbatch * maxch * cpad * cpad + (size_t)maxbatch * cpad * cpad) *
                    sizeof(TA);
  int rc;
  g_realloc = false;
  if ((rc = ensure(&M->d_U, &M->cap_U, (size_t)M->n * c_cap * sizeof(T))) != BSP_OK) return rc;
  if (!M->d_Y || M->c_cap != c_cap) {
    g_realloc = true;
    if (M->d_Y) cudaFree(M->d_Y);
    M->d_Y = nullptr;
    if (cudaMalloc(&M->d_Y, (size_t)M->n * c_cap * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return fail(BSP_ERR_OOM, "device allocation failed");
    }
  }
  if ((rc = ensure(&M->d_Gp, &M->cap_Gp, gp)) != BSP_OK) return rc;
  if ((rc = ensure(&M->d_Rsm, &M->cap_Rsm, (size_t)maxbatch * cpad * cpad * sizeof(T))) != BSP_OK)
    return rc;
  if ((rc = ensure(&M->d_theta, &M->cap_theta, (size_t)maxbatch * cpad * sizeof(T))) != BSP_OK)
    return rc;
  if ((M->c_cap != c_cap || g_realloc) && M->graph_exec) {
    cudaGraphExecDestroy(M->graph_exec);
    M->graph_exec = nullptr;
  }
  if ((M->c_cap != c_cap || g_realloc) && M->dyn_exec) {
    cudaGraphExecDestroy(M->dyn_exec);
    M->dyn_exec = nullptr;
  }
  if ((M->c_cap != c_cap || g_realloc) && M->doi_exec) {
    cudaGraphExecDestroy(M->doi_exec);
    M->doi_exec = nullptr;
  }
  M->c_cap = c_cap;
  return BSP_OK;
}

// Rayleigh-Ritz of the fixed-c schedule runs after the last wave over all
// blocks: consecutive blocks of the wave order are grouped so that a group's
// partial Grams stay within kRRBytes (a larger block forms a group alone).
constexpr size_t kRRBytes = (size_t)512 << 20;

template <typename T, typename TA>
int ensure_rr_groups(bsp_mesh* M, int c) {
  const int cpad = pad4(c);
  const int CH = dense_chunk_rows(cpad, (int)sizeof(T));
  const size_t mat = (size_t)cpad * cpad * sizeof(TA);
  M->rr_group.assign(1, 0);
  M->rr_wmax.clear();
  size_t gp = 0;
  int nmax = 0, wmax = 0;
  for (int q = 0; q < M->k; ++q) {
    const int b = M->h_wave_list[q];
    const int w = std::max(wmax, M->h_bptr[b + 1] - M->h_bptr[b]);
    const int n = q - M->rr_group.back() + 1;
    const size_t bytes = (size_t)n * ((w + CH - 1) / CH + 1) * mat;
    if (n > 1 && bytes > kRRBytes) {   // close the group before block q
      M->rr_wmax.push_back(wmax);
      M->rr_group.push_back(q);
      wmax = M->h_bptr[b + 1] - M->h_bptr[b];
      gp = std::max(gp, (size_t)((wmax + CH - 1) / CH + 1) * mat);
      nmax = std::max(nmax, 1);
      continue;
    }
    wmax = w;
    gp = std::max(gp, bytes);
    nmax = std::max(nmax, n);
  }
  M->rr_wmax.push_back(wmax);
  M->rr_group.push_back(M->k);
  int rc;
  if ((rc = ensure(&M->d_Gp_rr, &M->cap_Gp_rr, gp)) != BSP_OK ||
      (rc = ensure(&M->d_Rsm_rr, &M->cap_Rsm_rr, (size_t)nmax * cpad * cpad * sizeof(T))) != BSP_OK ||
      (rc = ensure(&M->d_theta_rr, &M->cap_theta_rr, (size_t)nmax * cpad * sizeof(T))) != BSP_OK)
    return rc;
  return BSP_OK;
}

// The fixed-c schedule for the blocks at positions [pos0, pos1) of the wave
// order in one launch of the persistent cluster engine (FP32).  The ready
// flags are cleared with the first range.  BSP_ERR_INVALID_ARG: the engine's
// cluster shape cannot be resident here (the caller falls back to the
// per-wave launches).
int enqueue_engine(bsp_mesh* M, int c, int t_max, cudaStream_t s, int* launches, int pos0,
                   int pos1) {
  int maxwave = 0;
  for (auto& w : M->waves) maxwave = std::max(maxwave, (int)w.size());
  if (pos0 == 0 && (maxwave > 1 || M->opts.withhold_block >= 0))
    CU(cudaMemsetAsync(M->d_ready, 0, sizeof(int) * (M->k + 2), s));
  OiClusterArgs oa;
  oa.order = M->d_waves + pos0;
  oa.nblocks = pos1 - pos0;
  oa.k = M->k;
  oa.parent = M->d_parent;
  oa.root_off = M->d_root_off;
  oa.starts = (const float*)M->d_starts;
  oa.U = (float*)M->d_U;
  oa.ld = M->c_cap;
  oa.c = c;
  oa.t_max = t_max;
  oa.z = M->opts.z;
  oa.delta = M->opts.delta;
  oa.rtol = M->opts.cg_rtol;
  oa.max_steps = M->opts.cg_max_steps;
  oa.ready = M->d_ready;
  oa.status = M->d_status;
  oa.stats = M->d_cgstats;
  oa.wait_limit_us = (long long)M->opts.wait_limit_ms * 1000;
  oa.withhold = M->opts.withhold_block;
  const int rc = launch_oi_cluster(view<float>(M), oa, M->max_nb, M->max_deg, M->engine_ncl, s);
  if (rc == BSP_OK) ++*launches;
  return rc;
}

// Engine launches over a chain (every block's parent is the block before it
// in the wave order, or none) are split into consecutive ranges so that the
// deferred work of a range (the second CholeskyQR pass and Rayleigh-Ritz) runs
// on a side stream while the engine works through the next range: the engine
// holds one cluster of SMs, the deferred kernels use the others.  A block's
// basis is read by its child only, which (at a range boundary) loads it from
// U at the start of the next launch; so the deferred work of range i stops
// one block short of it and that block goes with range i + 1.  Ranges of 128
// blocks, the last 128 in 64, 32, 16, 16 (a short tail after the engine).
// Returns the range ends, or {k} when the schedule does not split.
std::vector<int> engine_ranges(const bsp_mesh* M) {
  const int k = M->k;
  std::vector<int> ends;
  bool chain = M->engine_ncl == 1 && k >= 256;
  for (int q = 1; q < k && chain; ++q) {
    const int b = M->h_wave_list[q], p = M->h_parent[b];
    chain = p < 0 || p == M->h_wave_list[q - 1];
  }
  if (!chain || M->opts.withhold_block >= 0 || !M->post_stream) return {k};
  const int tail[] = {64, 32, 16, 16};
  int front = k;
  for (int t : tail) front -= t;
  for (int pos = 128; pos < front; pos += 128) ends.push_back(pos);
  int pos = front;
  for (int t : tail) {
    ends.push_back(pos);
    pos += t;
  }
  ends.push_back(k);
  return ends;
}

// Deferred work for the blocks at positions [q0, q1) of the wave order: the
// second CholeskyQR pass (engine schedule) and Rayleigh-Ritz, per block
// group of ensure_rr_groups() intersected with the range.
template <typename T, typename TA>
int enqueue_deferred(bsp_mesh* M, int c, bool engine, int q0, int q1, cudaStream_t s,
                     int* launches) {
  int rc;
  for (size_t g = 0; g + 1 < M->rr_group.size(); ++g) {
    const int g0 = std::max(M->rr_group[g], q0), g1 = std::min(M->rr_group[g + 1], q1);
    if (g0 >= g1) continue;
    int wmax = 0;
    for (int q = g0; q < g1; ++q) {
      const int b = M->h_wave_list[q];
      wmax = std::max(wmax, M->h_bptr[b + 1] - M->h_bptr[b]);
    }
    DenseArgs da{M->d_waves + g0, g1 - g0, M->d_bptr, M->d_cb, M->c_cap, c, wmax, M->d_status};
    if (engine) {
      // the second pass on the tensor cores where it fits (FP32, c <= 64)
      rc = BSP_ERR_INVALID_ARG;
      if constexpr (sizeof(T) == 4 && sizeof(TA) == 4) {
        if (tcqr_fits(c, 4))
          rc = launch_cholqr_pass_tc<float>(da, (float*)M->d_U, (float*)M->d_U,
                                            (float*)M->d_Gp_rr, (float*)M->d_Rsm_rr, s, launches);
      }
      if (rc == BSP_ERR_INVALID_ARG)
        rc = launch_cholqr2<T, TA>(da, (T*)M->d_U, (T*)M->d_U, (TA*)M->d_Gp_rr, (T*)M->d_Rsm_rr,
                                   s, launches, 1);
      if (rc) return fail(rc, "launch failed (second CholeskyQR pass)");
    }
    if (!M->opts.rayleigh_ritz) continue;
    da.sweeps = &M->d_cgstats->jacobi_sweeps;
    rc = launch_rayleigh_ritz<T, TA>(da, view<T>(M), (T*)M->d_U, (TA*)M->d_Gp_rr, (T*)M->d_Rsm_rr,
                                     (T*)M->d_theta_rr, s, launches);
    if (rc) return fail(rc, "launch failed (Rayleigh-Ritz)");
  }
  return BSP_OK;
}

// Enqueue the fixed-c schedule on stream s; returns a status, counts launches.
template <typename T, typename TA>
int enqueue_fixed(bsp_mesh* M, int c, int t_max, cudaStream_t s, int* launches) {
  const MeshView<T> mv = view<T>(M);
  const int levels = (int)M->waves.size();
  T* U = (T*)M->d_U;
  T* Y = (T*)M->d_Y;
  int rc;
  bool engine = false;
  if constexpr (sizeof(T) == 4 && sizeof(TA) == 4) {
    if (M->opts.schedule == BSP_SCHED_AUTO && M->engine_c == c && M->engine_ncl > 0 &&
        oi_cluster_fits(c, t_max, M->max_nb, M->max_deg, M->min_nb)) {
      const std::vector<int> ends = engine_ranges(M);
      if (ends.size() > 1) {
        // engine ranges on s; each range's deferred work (one block short) on
        // the side stream, serialised there (shared workspace), joined at the end
        int pos = 0, done = 0;
        for (size_t i = 0; i < ends.size(); ++i) {
          if ((rc = enqueue_engine(M, c, t_max, s, launches, pos, ends[i])) != BSP_OK)
            return fail(rc, "launch failed (cluster engine)");
          pos = ends[i];
          const int upto = i + 1 < ends.size() ? pos - 1 : pos;
          CU(cudaEventRecord(M->post_ev[0], s));
          CU(cudaStreamWaitEvent(M->post_stream, M->post_ev[0], 0));
          if ((rc = enqueue_deferred<T, TA>(M, c, true, done, upto, M->post_stream, launches)))
            return rc;
          done = upto;
        }
        CU(cudaEventRecord(M->post_ev[1], M->post_stream));
        CU(cudaStreamWaitEvent(s, M->post_ev[1], 0));
        return BSP_OK;
      }
      if ((rc = enqueue_engine(M, c, t_max, s, launches, 0, M->k)) != BSP_OK)
        return fail(rc, "launch failed (cluster engine)");
      engine = true;
    }
  }
  for (int l = 0; l < levels && !engine; ++l) {
    const int nbw = (int)M->waves[l].size();
    const int32_t* batch = M->d_waves + M->h_wave_off[l];
    int wmax = 0;
    for (int b : M->waves[l]) wmax = std::max(wmax, M->h_bptr[b + 1] - M->h_bptr[b]);
    // Onorm of the start where it is not already an orthonormal basis: roots and
    // children whose size differs from their parent's.
    std::vector<int32_t> need;
    for (int b : M->waves[l]) {
      int p = M->h_parent[b];
      if (p < 0 || (M->h_bptr[b + 1] - M->h_bptr[b]) != (M->h_bptr[p + 1] - M->h_bptr[p]))
        need.push_back(b);
    }
    // a wave of same-size warm starts reads its starts in place (the parents'
    // rows) in its first solve: no start copy
    const int sub = t_max * M->opts.z;
    const bool in_place = need.empty() && l > 0 && sub > 0;
    if (!in_place) {
      launch_init_starts<T>(batch, nbw, M->d_bptr, M->d_parent, M->d_root_off, M->d_cb, M->d_cb,
                            (const T*)M->d_starts, c, U, M->c_cap, wmax, c, s);
      ++*launches;
    }
    DenseArgs da{batch, nbw, M->d_bptr, M->d_cb, M->c_cap, c, wmax, M->d_status};
    if (!need.empty()) {
      DenseArgs dn = da;
      if ((int)need.size() != nbw) {
        // sub-batch staged by stage_onorm_lists() in the second third of d_waves
        dn.batch = M->d_waves + M->k + M->h_wave_off[l];
        dn.nbatch = (int)need.size();
      }
      if ((rc = launch_cholqr2<T, TA>(dn, U, U, (TA*)M->d_Gp, (T*)M->d_Rsm, s, launches)))
        return fail(rc, "launch failed (Onorm of start)");
    }
    // S^z V is applied as z solves with an Onorm after each: the span is that
    // of R^z V (Onorm keeps the span), and every solve sees a well-conditioned
    // input (R^z V itself loses rank in FP32 once ((lambda_c + delta)/delta)^z
    // nears 1/u).
    CgArgs ca{batch, nbw, M->d_cb, M->c_cap, 1, M->opts.delta, M->opts.cg_rtol,
              M->opts.cg_max_steps, M->d_status, M->d_cgstats, M->max_deg};
    ca.rows_per_lane = M->opts.cg_rows_per_lane;
    const int cs = pick_cs(M, nbw, c, sizeof(T));
    const bool buckets = use_buckets(M, nbw, wmax);
    // Onorm placement.  Only the span matters between steps (span(S Q) =
    // span(S Y) for Q = Onorm(Y)), so Onorm is there to keep the next solve's
    // input well conditioned.  A random (root) or row-transferred start needs
    // it after every solve; a warm start from a same-size parent is close to
    // the block's eigenbasis, which S maps to nearly orthogonal columns, so
    // two solves share one Onorm (S^2 V0 stays far inside what CholeskyQR2
    // handles).  Solves between two Onorms run in one CG launch (every column
    // goes straight on to its next solve).  Intermediate Onorms take one
    // Cholesky-QR pass, the last one the full CholeskyQR2.
    const bool warm = need.empty();
    for (int t = 0; t < sub;) {
      const int g = (warm && t + 1 < sub) ? 2 : 1;   // solves before the next Onorm
      CgArgs cg = ca;
      cg.z = g;
      if (t == 0 && in_place) cg.vsrc = M->d_parent;
      rc = buckets ? launch_cg_buckets<T>(mv, U, Y, cg, M->wave_bucket[l].data(),
                                          M->wave_bucket_rows[l].data(), c, s, &M->cg_fork)
                   : launch_cg<T>(mv, U, Y, cg, cs, wmax, c, s);
      if (rc) return fail(rc, "CG launch failed (block too large for shared memory?)");
      ++*launches;
      t += g;
      const int passes = t == sub ? 2 : 1;
      if ((rc = launch_cholqr2<T, TA>(da, Y, U, (TA*)M->d_Gp, (T*)M->d_Rsm, s, launches, passes)))
        return fail(rc, "launch failed (Onorm)");
    }
  }
  // The engine leaves every block's basis after one CholeskyQR pass (same
  // span, orthonormal to O(kappa^2 u)); the second pass, which no later block
  // needs, runs here batched over all blocks.  Rayleigh-Ritz does not change
  // the spans the chain depends on, and no later wave reads its rotation: it
  // also runs once after the last wave.  Both use the groups of
  // ensure_rr_groups().
  if (engine || M->opts.rayleigh_ritz)
    return enqueue_deferred<T, TA>(M, c, engine, 0, M->k, s, launches);
  return BSP_OK;
}

// Blocks of each wave whose start needs Onorm (roots, and children whose size
// differs from the parent's), written to d_waves[k + wave offset ...].
int stage_onorm_lists(bsp_mesh* M) {
  for (int l = 0; l < (int)M->waves.size(); ++l) {
    std::vector<int32_t> need;
    for (int b : M->waves[l]) {
      int p = M->h_parent[b];
      if (p < 0 || (M->h_bptr[b + 1] - M->h_bptr[b]) != (M->h_bptr[p + 1] - M->h_bptr[p]))
        need.push_back(b);
    }
    if (!need.empty() && need.size() != M->waves[l].size())
      CU(cudaMemcpy(M->d_waves + M->k + M->h_wave_off[l], need.data(),
                    sizeof(int32_t) * need.size(), cudaMemcpyHostToDevice));
  }
  return BSP_OK;
}

template <typename T, typename TA>
int track_fixed(bsp_mesh* M, int c, int t_max, const void* V0, cudaStream_t s) {
  if (c < 1 || c > 128) return fail(BSP_ERR_INVALID_ARG, "c must be in [1, 128]");
  if (c > M->min_nb) return fail(BSP_ERR_INVALID_ARG, "c exceeds the smallest block size");
  if (t_max < 0) return fail(BSP_ERR_INVALID_ARG, "t_max must be >= 0");
  if (!V0) return fail(BSP_ERR_INVALID_ARG, "V0_roots is NULL");
  if (sizeof(T) == 8 && c > 64) return fail(BSP_ERR_INVALID_ARG, "FP64 precision supports c <= 64");
  int maxbatch = 0;
  for (auto& w : M->waves) maxbatch = std::max(maxbatch, (int)w.size());
  int rc;
  if ((rc = ensure_workspace<T, TA>(M, c, maxbatch)) != BSP_OK) return rc;
  g_realloc = false;
  if ((rc = ensure(&M->d_starts, &M->cap_starts, (size_t)M->root_rows * c * sizeof(T))) != BSP_OK)
    return rc;
  if ((rc = ensure((void**)&M->d_ready, &M->cap_ready, sizeof(int) * (M->k + 2))) != BSP_OK)
    return rc;
  if (sizeof(T) == 4 && sizeof(TA) == 4 && M->engine_c != c) {
    // the engine's attributes and residency, before any capture
    int maxwave = 0;
    for (auto& w : M->waves) maxwave = std::max(maxwave, (int)w.size());
    M->engine_ncl = 0;
    if (oi_cluster_fits(c, std::max(t_max, 1), M->max_nb, M->max_deg, M->min_nb) &&
        prepare_oi_cluster(view<float>(M), c, M->max_nb, M->max_deg, maxwave, &M->engine_ncl) !=
            BSP_OK)
      M->engine_ncl = 0;
    M->engine_c = c;
  }
  if ((rc = ensure_rr_groups<T, TA>(M, c)) != BSP_OK) return rc;
  if (g_realloc && M->graph_exec) {
    cudaGraphExecDestroy(M->graph_exec);
    M->graph_exec = nullptr;
  }
  // copy the roots' start matrices (before any graph launch)
  if ((rc = to_device(M->d_starts, V0, (size_t)M->root_rows * c * sizeof(T), s)) != BSP_OK)
    return rc;
  M->h_c.assign(M->k, c);
  std::vector<int32_t> ce(M->k + 1, 0);
  for (int b = 0; b < M->k; ++b) ce[b + 1] = ce[b] + c;
  CU(cudaMemcpyAsync(M->d_cb, M->h_c.data(), sizeof(int32_t) * M->k, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(M->d_ceoff, ce.data(), sizeof(int32_t) * (M->k + 1), cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(M->d_status, 0, sizeof(int), s));
  CU(cudaMemsetAsync(M->d_cgstats, 0, sizeof(CgStats), s));
  int launches = 0;
  if ((rc = stage_onorm_lists(M)) != BSP_OK) return rc;
  if (M->opts.use_graph && !M->profiling) {
    if (!M->graph_exec || M->graph_c != c || M->graph_t != t_max ||
        M->graph_cs != M->opts.cols_per_cta || M->graph_rpl != M->opts.cg_rows_per_lane) {
      if (M->graph_exec) {
        cudaGraphExecDestroy(M->graph_exec);
        M->graph_exec = nullptr;
      }
      if (!M->graph_stream) CU(cudaStreamCreateWithFlags(&M->graph_stream, cudaStreamNonBlocking));
      CU(cudaStreamSynchronize(s));
      cudaGraph_t g;
      CU(cudaStreamBeginCapture(M->graph_stream, cudaStreamCaptureModeThreadLocal));
      rc = enqueue_fixed<T, TA>(M, c, t_max, M->graph_stream, &launches);
      cudaError_t ce2 = cudaStreamEndCapture(M->graph_stream, &g);
      if (rc != BSP_OK) {
        if (ce2 == cudaSuccess) cudaGraphDestroy(g);
        return rc;
      }
      if (ce2 != cudaSuccess) return fail(BSP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce2));
      // node priorities as launched (the engine above its side-stream work)
      cudaError_t ie = cudaGraphInstantiate(&M->graph_exec, g, cudaGraphInstantiateFlagUseNodePriority);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) return fail(BSP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
      M->graph_c = c;
      M->graph_t = t_max;
      M->graph_cs = M->opts.cols_per_cta;
      M->graph_rpl = M->opts.cg_rows_per_lane;
      M->graph_launches = launches;
    }
    CU(cudaGraphLaunch(M->graph_exec, s));
    launches = M->graph_launches;
  } else {
    rc = enqueue_fixed<T, TA>(M, c, t_max, s, &launches);
    if (rc != BSP_OK) return rc;
  }
  M->stats.gpu_launches = launches;
  M->tracked = true;
  M->ubf_valid = false;
  return stream_error_status(M, s);
}

// Per-block state of the dynamic schedules (allocated once per mesh, each
// buffer on its first use).
int ensure_dyn_state(bsp_mesh* M) {
  struct Buf { void** p; size_t bytes; };
  const Buf bufs[] = {{(void**)&M->d_action, sizeof(int32_t) * M->k},
                      {(void**)&M->d_round, sizeof(int32_t) * M->k},
                      {(void**)&M->d_forced, sizeof(int32_t) * M->k},
                      {(void**)&M->d_rho, sizeof(double) * M->k},
                      {(void**)&M->d_gcol, sizeof(double) * M->n},
                      {(void**)&M->d_live, sizeof(int32_t) * M->k},
                      {(void**)&M->d_dynctl, sizeof(DynCtl)}};
  for (const Buf& b : bufs)
    if (!*b.p && cudaMalloc(b.p, b.bytes) != cudaSuccess) {
      *b.p = nullptr;
      cudaGetLastError();
      return fail(BSP_ERR_OOM, "device allocation failed");
    }
  return BSP_OK;
}

// ---------------------------------------------------------- dynamic c
// The dynamic-c schedule (Sec. 5, Algorithm 2, with the reading of
// oi_dynamic_block: rounds of Algorithm 1 + Rayleigh-Ritz, the smallest
// passing prefix width, else c_step more columns) runs device-driven: per
// block, live[b] says whether it still grows; the decision kernel clears it,
// every kernel of a round skips blocks that are no longer live, and two
// one-CTA kernels per round reduce the wave's state to "another round?" and
// "largest live width".  No decision goes back to the host between rounds.
// With use_graph the whole call is one CUDA graph: per wave, a SWITCH node
// over width classes for the start, then a WHILE node over rounds whose body
// is a SWITCH over width classes (launches sized for the largest live width,
// a multiple of c_step = kDynClass), the conditions set by those kernels.  Without it
// (or while profiling, or when the forest has too many levels for one graph)
// the host replays the same launches, reading the class and the "another
// round" flag back after each control kernel.
constexpr int kDynClass = 8;
constexpr int kDynMaxRounds = 64;
constexpr size_t kDynMaxBodies = 256;   // waves x width classes captured in one graph

struct DynParams {
  int c_min, c_max, c_step, t_max;
  double tol;
  uint64_t seed;
  const int32_t* forced;   // device copy or nullptr
};

int dyn_classes(int c_max) { return (c_max + kDynClass - 1) / kDynClass; }
int dyn_class_width(int q, int c_max) { return std::min((q + 1) * kDynClass, c_max); }

int wave_rows(const bsp_mesh* M, int l) {
  int w = 0;
  for (int b : M->waves[l]) w = std::max(w, M->h_bptr[b + 1] - M->h_bptr[b]);
  return w;
}

// Start of wave l at widths <= cm: start matrices (roots: their rows of the
// start matrix; children: the parent's basis, rows transferred) and Onorm.
template <typename T, typename TA>
int enqueue_dyn_start(bsp_mesh* M, int l, int cm, const DynParams& p, cudaStream_t s,
                      int* launches) {
  const int32_t* wave = M->d_waves + M->h_wave_off[l];
  const int nw = (int)M->waves[l].size(), wmax = wave_rows(M, l);
  T* U = (T*)M->d_U;
  launch_init_starts<T>(wave, nw, M->d_bptr, M->d_parent, M->d_root_off, M->d_cb, M->d_cpar,
                        (const T*)M->d_starts, p.c_min, U, M->c_cap, wmax, cm, s);
  ++*launches;
  DenseArgs da{wave, nw, M->d_bptr, M->d_cb, M->c_cap, cm, wmax, M->d_status};
  return launch_cholqr2<T, TA>(da, U, U, (TA*)M->d_Gp, (T*)M->d_Rsm, s, launches);
}

// One round of wave l for the live blocks, widths <= cm: t_max steps of z
// solves with an Onorm after each, Rayleigh-Ritz, the decision, and for the
// blocks that grow: c_step new columns and an Onorm at widths <= cm + c_step.
template <typename T, typename TA>
int enqueue_dyn_round(bsp_mesh* M, int l, int cm, const DynParams& p, cudaStream_t s,
                      int* launches) {
  const int32_t* wave = M->d_waves + M->h_wave_off[l];
  const int nw = (int)M->waves[l].size(), wmax = wave_rows(M, l);
  const MeshView<T> mv = view<T>(M);
  T* U = (T*)M->d_U;
  T* Y = (T*)M->d_Y;
  int rc;
  DenseArgs da{wave, nw, M->d_bptr, M->d_cb, M->c_cap, cm, wmax, M->d_status};
  da.live = M->d_live;
  CgArgs ca{wave, nw, M->d_cb, M->c_cap, 1, M->opts.delta, M->opts.cg_rtol, M->opts.cg_max_steps,
            M->d_status, M->d_cgstats, M->max_deg};
  ca.rows_per_lane = M->opts.cg_rows_per_lane;
  ca.live = M->d_live;
  const int cs = pick_cs(M, nw, cm, sizeof(T));
  const bool buckets = use_buckets(M, nw, wmax);
  for (int t = 0; t < p.t_max * M->opts.z; ++t) {   // z solves per step, Onorm after each
    rc = buckets ? launch_cg_buckets<T>(mv, U, Y, ca, M->wave_bucket[l].data(),
                                        M->wave_bucket_rows[l].data(), cm, s, &M->cg_fork)
                 : launch_cg<T>(mv, U, Y, ca, cs, wmax, cm, s);
    if (rc) return fail(rc, "CG launch failed");
    ++*launches;
    if ((rc = launch_cholqr2<T, TA>(da, Y, U, (TA*)M->d_Gp, (T*)M->d_Rsm, s, launches)))
      return fail(rc, "launch failed");
  }
  da.sweeps = &M->d_cgstats->jacobi_sweeps;
  if ((rc = launch_rayleigh_ritz<T, TA>(da, mv, U, (TA*)M->d_Gp, (T*)M->d_Rsm, (T*)M->d_theta, s,
                                        launches)))
    return fail(rc, "launch failed");
  if ((rc = launch_dyn_decide<T, TA>(wave, nw, M->d_bptr, M->d_verts, (const T*)M->d_X, U,
                                     M->c_cap, M->d_cb, M->d_action, p.forced, p.tol, p.c_step,
                                     p.c_max, (T*)M->d_gcol, (TA*)M->d_rho, wmax, s, M->d_live)))
    return fail(rc, "launch failed");
  ++*launches;
  if ((rc = launch_dyn_grow<T, TA>(wave, nw, M->d_bptr, M->d_cb, M->d_round, U, M->c_cap,
                                   (const T*)M->d_gcol, p.seed, p.c_step, wmax, s, M->d_live)))
    return fail(rc, "launch failed");
  ++*launches;
  DenseArgs dg = da;
  dg.sweeps = nullptr;
  dg.cmax = std::min(cm + p.c_step, p.c_max);
  if ((rc = launch_cholqr2<T, TA>(dg, U, U, (TA*)M->d_Gp, (T*)M->d_Rsm, s, launches)))
    return fail(rc, "launch failed");
  return BSP_OK;
}

// A conditional node after the current capture frontier of s (which then
// continues after the node); its body graphs in *bodies.
int add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                    unsigned size, std::vector<cudaGraph_t>* bodies) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CU(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd));
  if (st != cudaStreamCaptureStatusActive) return fail(BSP_ERR_CUDA, "stream is not capturing");
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = size;
  cudaGraphNode_t node;
  CU(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
  bodies->assign(np.conditional.phGraph_out, np.conditional.phGraph_out + size);
  CU(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return BSP_OK;
}

// A device-driven wave schedule: per wave, an init kernel (widths, live
// flags, the start's width class), the start at its width class, rounds while
// a block is live, and optionally a final body for the blocks still live
// after the last round.  Bodies are enqueued per width class q (launches
// sized for widths <= the class width) by the callbacks; the control kernels
// choose the class and whether another round runs.
struct WaveSchedule {
  int ncls = 0;         // width classes
  int max_rounds = 0;   // bound of the round loop
  bool has_final = false;
  // init(l, counts of wave l, handle, set_handle, stream): launches the wave's init kernel
  std::function<int(int, const unsigned*, int, cudaGraphConditionalHandle, cudaStream_t)> init;
  // start / round / final (l, q, stream, launches)
  std::function<int(int, int, cudaStream_t, int*)> start, round, final_;
};

// Launch-count table of a schedule: per wave, [start | round | final] x ncls.
size_t wave_counts_size(const bsp_mesh* M, const WaveSchedule& w) {
  return (M->waves.size() + 1) * 3 * (size_t)w.ncls;
}

// The whole schedule as one CUDA graph: per wave a SWITCH over width classes
// for the start, a WHILE over rounds whose body is a SWITCH over width classes
// (the class and the loop condition set on the device), and for a final body
// one more class kernel and SWITCH.  counts: launches of every body.
int build_wave_graph(bsp_mesh* M, const WaveSchedule& w, std::vector<unsigned>* counts,
                     cudaGraphExec_t* exec) {
  const int ncls = w.ncls;
  const int levels = (int)M->waves.size();
  counts->assign(wave_counts_size(M, w), 0u);
  cudaStream_t s0 = M->graph_stream, s1 = M->dyn_stream[0], s2 = M->dyn_stream[1];
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
  cudaGraph_t g;
  CU(cudaGraphCreate(&g, 0));
  auto abort_capture = [&](int rc) {
    for (cudaStream_t q : {s2, s1, s0}) {
      cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
      cudaStreamIsCapturing(q, &st);
      if (st != cudaStreamCaptureStatusNone) {
        cudaGraph_t t = nullptr;
        cudaStreamEndCapture(q, &t);
      }
    }
    cudaGraphDestroy(g);
    cudaGetLastError();
    return rc;
  };
  // capture the bodies of a SWITCH node, one per class, on stream cs
  auto capture_bodies = [&](std::vector<cudaGraph_t>& bodies, cudaStream_t cs,
                            const std::function<int(int, int, cudaStream_t, int*)>& fn, int l,
                            unsigned* cnt) -> int {
    for (int q = 0; q < ncls; ++q) {
      int n = 0, rc;
      if (cudaStreamBeginCaptureToGraph(cs, bodies[q], nullptr, nullptr, 0, mode) != cudaSuccess)
        return fail(BSP_ERR_CUDA, "graph capture failed to start");
      if ((rc = fn(l, q, cs, &n))) return rc;
      cudaGraph_t t;
      if (cudaStreamEndCapture(cs, &t) != cudaSuccess) return fail(BSP_ERR_CUDA, "graph capture");
      cnt[q] = (unsigned)n;
    }
    return BSP_OK;
  };
  if (cudaStreamBeginCaptureToGraph(s0, g, nullptr, nullptr, 0, mode) != cudaSuccess)
    return abort_capture(fail(BSP_ERR_CUDA, "graph capture failed to start"));
  int rc = BSP_OK;
  for (int l = 0; l < levels; ++l) {
    const int32_t* wave = M->d_waves + M->h_wave_off[l];
    const int nw = (int)M->waves[l].size();
    const unsigned* dcnt = M->d_dyn_launches + (size_t)l * 3 * ncls;
    unsigned* hcnt = counts->data() + (size_t)l * 3 * ncls;
    cudaGraphConditionalHandle h_start, h_while, h_round, h_final;
    if (cudaGraphConditionalHandleCreate(&h_start, g, 0, 0) != cudaSuccess ||
        cudaGraphConditionalHandleCreate(&h_while, g, 1, cudaGraphCondAssignDefault) != cudaSuccess ||
        (w.has_final && cudaGraphConditionalHandleCreate(&h_final, g, 0, 0) != cudaSuccess))
      return abort_capture(fail(BSP_ERR_CUDA, "conditional handle"));
    if ((rc = w.init(l, dcnt, 1, h_start, s0))) return abort_capture(fail(rc, "launch failed"));
    std::vector<cudaGraph_t> sb, wb, rb, fb;
    if ((rc = add_conditional(s0, h_start, cudaGraphCondTypeSwitch, ncls, &sb)) ||
        (rc = capture_bodies(sb, s1, w.start, l, hcnt)))
      return abort_capture(rc);
    if ((rc = add_conditional(s0, h_while, cudaGraphCondTypeWhile, 1, &wb))) return abort_capture(rc);
    if (cudaGraphConditionalHandleCreate(&h_round, wb[0], 0, 0) != cudaSuccess ||
        cudaStreamBeginCaptureToGraph(s1, wb[0], nullptr, nullptr, 0, mode) != cudaSuccess)
      return abort_capture(fail(BSP_ERR_CUDA, "graph capture failed to start"));
    if ((rc = launch_dyn_class(wave, nw, M->d_cb, M->d_live, kDynClass, ncls, dcnt + ncls,
                               M->d_dynctl, 1, h_round, s1, 2)))
      return abort_capture(fail(rc, "launch failed"));
    if ((rc = add_conditional(s1, h_round, cudaGraphCondTypeSwitch, ncls, &rb)) ||
        (rc = capture_bodies(rb, s2, w.round, l, hcnt + ncls)))
      return abort_capture(rc);
    if ((rc = launch_dyn_next(wave, nw, M->d_live, w.max_rounds, M->d_dynctl, 1, h_while, s1)))
      return abort_capture(fail(rc, "launch failed"));
    cudaGraph_t t;
    if (cudaStreamEndCapture(s1, &t) != cudaSuccess)
      return abort_capture(fail(BSP_ERR_CUDA, "graph capture"));
    if (w.has_final) {
      if ((rc = launch_dyn_class(wave, nw, M->d_cb, M->d_live, kDynClass, ncls, dcnt + 2 * ncls,
                                 M->d_dynctl, 1, h_final, s0, 1)))
        return abort_capture(fail(rc, "launch failed"));
      if ((rc = add_conditional(s0, h_final, cudaGraphCondTypeSwitch, ncls, &fb)) ||
          (rc = capture_bodies(fb, s1, w.final_, l, hcnt + 2 * ncls)))
        return abort_capture(rc);
    }
  }
  cudaGraph_t t;
  if (cudaStreamEndCapture(s0, &t) != cudaSuccess)
    return abort_capture(fail(BSP_ERR_CUDA, "graph capture"));
  const cudaError_t ie = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess)
    return fail(BSP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
  return BSP_OK;
}

// The same schedule launched from the host: control values read back after
// each control kernel (one synchronisation per kernel; profiling mode, or a
// forest with too many levels for one graph).  The device's launch counter
// counts only the control kernels here; *launches gets the bodies'.
int run_wave_eager(bsp_mesh* M, const WaveSchedule& w, cudaStream_t s, int* launches) {
  const int ncls = w.ncls;
  const unsigned* zeros = M->d_dyn_launches + (size_t)M->waves.size() * 3 * ncls;
  DynCtl ctl;
  auto read_ctl = [&]() -> int {
    CU(cudaMemcpyAsync(&ctl, M->d_dynctl, sizeof(DynCtl), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return BSP_OK;
  };
  int rc;
  for (int l = 0; l < (int)M->waves.size(); ++l) {
    const int32_t* wave = M->d_waves + M->h_wave_off[l];
    const int nw = (int)M->waves[l].size();
    if ((rc = w.init(l, zeros, 0, 0, s))) return fail(rc, "launch failed");
    if ((rc = read_ctl())) return rc;
    if (ctl.cls_start < ncls && (rc = w.start(l, ctl.cls_start, s, launches))) return rc;
    for (;;) {
      if ((rc = launch_dyn_class(wave, nw, M->d_cb, M->d_live, kDynClass, ncls, zeros,
                                 M->d_dynctl, 0, 0, s, 2)))
        return fail(rc, "launch failed");
      if ((rc = read_ctl())) return rc;
      if (ctl.cls_round < ncls && (rc = w.round(l, ctl.cls_round, s, launches))) return rc;
      if ((rc = launch_dyn_next(wave, nw, M->d_live, w.max_rounds, M->d_dynctl, 0, 0, s)))
        return fail(rc, "launch failed");
      if ((rc = read_ctl())) return rc;
      if (!ctl.more) break;
    }
    if (w.has_final) {
      if ((rc = launch_dyn_class(wave, nw, M->d_cb, M->d_live, kDynClass, ncls, zeros,
                                 M->d_dynctl, 0, 0, s, 1)))
        return fail(rc, "launch failed");
      if ((rc = read_ctl())) return rc;
      if (ctl.cls_round < ncls && (rc = w.final_(l, ctl.cls_round, s, launches))) return rc;
    }
  }
  return BSP_OK;
}

// The schedule of one call: the cached graph (rebuilt when the key, a buffer
// or the bodies' layout changed) or the host-driven replay.
int run_wave_schedule(bsp_mesh* M, const WaveSchedule& w, const std::vector<double>& key,
                      bool realloc, cudaGraphExec_t* exec, std::vector<double>* cached_key,
                      cudaStream_t s, int* launches) {
  const size_t ncounts = wave_counts_size(M, w);
  const bool graph_fits = M->waves.size() * (size_t)w.ncls <= kDynMaxBodies;
  if (M->opts.use_graph && !M->profiling && graph_fits) {
    if (*exec && (realloc || key != *cached_key)) {
      cudaGraphExecDestroy(*exec);
      *exec = nullptr;
    }
    if (!*exec) {
      if (!M->graph_stream) CU(cudaStreamCreateWithFlags(&M->graph_stream, cudaStreamNonBlocking));
      for (auto& q : M->dyn_stream)
        if (!q) CU(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
      CU(cudaStreamSynchronize(s));
      std::vector<unsigned> counts;
      int rc;
      if ((rc = build_wave_graph(M, w, &counts, exec)) != BSP_OK) return rc;
      counts.resize(ncounts, 0u);   // the host-driven replay's zero counts at the end
      CU(cudaMemcpy(M->d_dyn_launches, counts.data(), ncounts * sizeof(unsigned),
                    cudaMemcpyHostToDevice));
      *cached_key = key;
    }
    CU(cudaGraphLaunch(*exec, s));
    return BSP_OK;
  }
  CU(cudaMemsetAsync(M->d_dyn_launches + (ncounts - 3 * w.ncls), 0, 3 * w.ncls * sizeof(unsigned), s));
  return run_wave_eager(M, w, s, launches);
}

template <typename T, typename TA>
int track_dynamic(bsp_mesh* M, const void* X, double tol, int c_min, int c_max, int c_step,
                  int t_max, uint64_t seed, const void* V0, const int32_t* forced,
                  int32_t* c_out, cudaStream_t s) {
  if (c_step < 8 || c_step > 8) return fail(BSP_ERR_INVALID_ARG, "c_step must be 8");
  if (c_min < c_step || c_min % c_step || c_max % c_step || c_max < c_min || c_max > 128)
    return fail(BSP_ERR_INVALID_ARG, "need c_step <= c_min <= c_max <= 128, multiples of c_step");
  if (c_min > M->min_nb) return fail(BSP_ERR_INVALID_ARG, "c_min exceeds the smallest block");
  if (!(tol > 0)) return fail(BSP_ERR_INVALID_ARG, "rel_tol must be positive");
  if (!X || !V0) return fail(BSP_ERR_INVALID_ARG, "X and V0_roots are required");
  if (sizeof(T) == 8 && c_max > 64) return fail(BSP_ERR_INVALID_ARG, "FP64 precision supports c <= 64");
  int maxbatch = 0;
  for (auto& w : M->waves) maxbatch = std::max(maxbatch, (int)w.size());
  int rc;
  if ((rc = ensure_workspace<T, TA>(M, c_max, maxbatch)) != BSP_OK) return rc;
  bool realloc = g_realloc;
  if ((rc = ensure(&M->d_starts, &M->cap_starts, (size_t)M->root_rows * c_min * sizeof(T))) != BSP_OK)
    return rc;
  if ((rc = ensure(&M->d_X, &M->cap_X, (size_t)M->n * 3 * sizeof(T))) != BSP_OK) return rc;
  DynParams p{c_min, c_max, c_step, t_max, tol, seed, nullptr};
  WaveSchedule w;
  w.ncls = dyn_classes(c_max);
  w.max_rounds = kDynMaxRounds;
  w.init = [&](int l, const unsigned* cnt, int set, cudaGraphConditionalHandle h,
                cudaStream_t q) -> int {
    return launch_dyn_wave_init(M->d_waves + M->h_wave_off[l], (int)M->waves[l].size(), M->d_bptr,
                                M->d_parent, M->d_cb, M->d_cpar, M->d_live, M->d_round, c_min,
                                c_max, c_step, kDynClass, w.ncls, cnt, M->d_dynctl, set, h, q);
  };
  w.start = [&](int l, int q, cudaStream_t st, int* n) -> int {
    return enqueue_dyn_start<T, TA>(M, l, dyn_class_width(q, c_max), p, st, n);
  };
  w.round = [&](int l, int q, cudaStream_t st, int* n) -> int {
    return enqueue_dyn_round<T, TA>(M, l, dyn_class_width(q, c_max), p, st, n);
  };
  if ((rc = ensure((void**)&M->d_dyn_launches, &M->cap_dyn_launches,
                   wave_counts_size(M, w) * sizeof(unsigned))) != BSP_OK)
    return rc;
  if ((rc = ensure_dyn_state(M)) != BSP_OK) return rc;
  p.forced = forced ? M->d_forced : nullptr;   // allocated by ensure_dyn_state on first use
  realloc = realloc || g_realloc;
  if ((rc = to_device(M->d_starts, V0, (size_t)M->root_rows * c_min * sizeof(T), s)) != BSP_OK)
    return rc;
  if ((rc = to_device(M->d_X, X, (size_t)M->n * 3 * sizeof(T), s)) != BSP_OK) return rc;
  if (forced && (rc = to_device(M->d_forced, forced, sizeof(int32_t) * M->k, s)) != BSP_OK)
    return rc;
  CU(cudaMemsetAsync(M->d_status, 0, sizeof(int), s));
  CU(cudaMemsetAsync(M->d_cgstats, 0, sizeof(CgStats), s));
  CU(cudaMemsetAsync(M->d_dynctl, 0, sizeof(DynCtl), s));
  int launches = 0;
  // the graph holds one start and one round body per wave and width class: a
  // forest of a few deep levels captures once and replays cheaply, a long
  // chain of single-block waves would not (host-driven replay instead)
  const std::vector<double> key = {(double)sizeof(T), (double)sizeof(TA), (double)c_min,
                                   (double)c_max, (double)c_step, (double)t_max, tol,
                                   (double)(seed >> 32), (double)(seed & 0xffffffffu),
                                   forced ? 1.0 : 0.0, (double)M->opts.z, M->opts.delta,
                                   M->opts.cg_rtol, (double)M->opts.cg_max_steps,
                                   (double)M->opts.cols_per_cta,
                                   (double)M->opts.cg_rows_per_lane, (double)M->c_cap};
  if ((rc = run_wave_schedule(M, w, key, realloc, &M->dyn_exec, &M->dyn_key, s, &launches)))
    return rc;
  // the chosen widths and the launch count: one read-back at the end
  std::vector<int32_t>& hc = M->h_c;
  hc.assign(M->k, 0);
  DynCtl ctl;
  CU(cudaMemcpyAsync(hc.data(), M->d_cb, sizeof(int32_t) * M->k, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(&ctl, M->d_dynctl, sizeof(DynCtl), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  std::vector<int32_t> ce(M->k + 1, 0);
  for (int b = 0; b < M->k; ++b) ce[b + 1] = ce[b] + hc[b];
  CU(cudaMemcpyAsync(M->d_ceoff, ce.data(), sizeof(int32_t) * (M->k + 1), cudaMemcpyHostToDevice, s));
  if (c_out) {
    if (is_device_ptr(c_out)) CU(cudaMemcpyAsync(c_out, M->d_cb, sizeof(int32_t) * M->k,
                                                 cudaMemcpyDeviceToDevice, s));
    else std::memcpy(c_out, hc.data(), sizeof(int32_t) * M->k);
  }
  M->stats.gpu_launches = (int)(ctl.launches + (unsigned long long)launches);
  M->tracked = true;
  M->ubf_valid = false;
  return stream_error_status(M, s);
}

// ------------------------------------------------------- low-pass filter
// Forward: Algorithm 1 without Rayleigh-Ritz, every step checkpointed
// (V_0..V_t in d_ckV, Y_1..Y_t in d_ckY; Onorm by CholeskyQR2 at every step),
// then X_out = U U^T X.  The next block's start is the parent's V_t.
// The paper's dynamic OI (Sec. 5, Algorithm 2) with the text's branch
// directions: per block, each iteration applies one Algorithm 1 step
// U = Onorm(R^z U) and measures the summed residual e; ||e|| > eps_h grows U
// by e/||e||, ||e|| < eps_l drops its last column, anything else stops the
// block; the width stays in [c_min, min(c_max, n_b)], at most t_cap
// iterations run, and a basis still carrying an appended column at the cap
// is orthonormalised once more.  A root starts from its rows of V0 (c0
// columns), a child from its parent's final basis and width.  The blocks of a
// DAG level run as one batch, device-driven like the step-8 dynamic c: a
// live flag per block (cleared by the decision when the block stops), the
// iteration number read on the device, the round loop and the width class
// of each iteration decided by the control kernels; the whole call is one
// CUDA graph (WHILE over iterations, SWITCH over width classes, a final
// SWITCH for the blocks still running at the cap).
template <typename T, typename TA>
int track_doi(bsp_mesh* M, const void* X, int c0, double eps_l, double eps_h, int c_min,
              int c_max, int t_cap, const void* V0, int32_t* c_out, int32_t* iters_out,
              cudaStream_t s) {
  if (!X || !V0) return fail(BSP_ERR_INVALID_ARG, "X and V0_roots are required");
  if (c_min < 1 || c0 < c_min || c_max < c0 || c_max > 128)
    return fail(BSP_ERR_INVALID_ARG, "need 1 <= c_min <= c0 <= c_max <= 128");
  if (sizeof(T) == 8 && c_max > 64) return fail(BSP_ERR_INVALID_ARG, "FP64 precision supports c <= 64");
  if (c0 > M->min_nb) return fail(BSP_ERR_INVALID_ARG, "c0 exceeds the smallest block");
  if (!(eps_l > 0) || !(eps_h >= eps_l)) return fail(BSP_ERR_INVALID_ARG, "need 0 < eps_l <= eps_h");
  if (t_cap < 1) return fail(BSP_ERR_INVALID_ARG, "t_cap must be >= 1");
  int maxbatch = 0;
  for (auto& w : M->waves) maxbatch = std::max(maxbatch, (int)w.size());
  int rc;
  if ((rc = ensure_workspace<T, TA>(M, c_max, maxbatch)) != BSP_OK) return rc;
  bool realloc = g_realloc;
  if ((rc = ensure(&M->d_starts, &M->cap_starts, (size_t)M->root_rows * c0 * sizeof(T))) != BSP_OK)
    return rc;
  if ((rc = ensure(&M->d_X, &M->cap_X, (size_t)M->n * 3 * sizeof(T))) != BSP_OK) return rc;
  const MeshView<T> mv = view<T>(M);
  T* U = (T*)M->d_U;
  T* Y = (T*)M->d_Y;
  WaveSchedule w;
  w.ncls = dyn_classes(c_max);
  w.max_rounds = t_cap;
  w.has_final = true;
  auto wave_rows_of = [&](int l) { return wave_rows(M, l); };
  // wave start: root c0, child min(parent width, c_max, n_b) (c_step 1)
  w.init = [&](int l, const unsigned* cnt, int set, cudaGraphConditionalHandle h,
                cudaStream_t q) -> int {
    return launch_dyn_wave_init(M->d_waves + M->h_wave_off[l], (int)M->waves[l].size(), M->d_bptr,
                                M->d_parent, M->d_cb, M->d_cpar, M->d_live, M->d_round, c0, c_max,
                                1, kDynClass, w.ncls, cnt, M->d_dynctl, set, h, q);
  };
  w.start = [&](int l, int q, cudaStream_t st, int* n) -> int {
    const int32_t* wave = M->d_waves + M->h_wave_off[l];
    launch_init_starts<T>(wave, (int)M->waves[l].size(), M->d_bptr, M->d_parent, M->d_root_off,
                          M->d_cb, M->d_cpar, (const T*)M->d_starts, c0, U, M->c_cap,
                          wave_rows_of(l), dyn_class_width(q, c_max), st);
    ++*n;
    return BSP_OK;
  };
  // one iteration: U = Onorm(R^z U) (z solves, an Onorm after each), then the
  // decision (grow by e/||e||, drop the last column, or stop)
  w.round = [&](int l, int q, cudaStream_t st, int* n) -> int {
    const int32_t* wave = M->d_waves + M->h_wave_off[l];
    const int nw = (int)M->waves[l].size(), wmax = wave_rows_of(l);
    const int cm = dyn_class_width(q, c_max);
    int rc2;
    DenseArgs da{wave, nw, M->d_bptr, M->d_cb, M->c_cap, cm, wmax, M->d_status};
    da.live = M->d_live;
    CgArgs ca{wave, nw, M->d_cb, M->c_cap, 1, M->opts.delta, M->opts.cg_rtol,
              M->opts.cg_max_steps, M->d_status, M->d_cgstats, M->max_deg};
    ca.rows_per_lane = M->opts.cg_rows_per_lane;
    ca.live = M->d_live;
    const int cs = pick_cs(M, nw, cm, sizeof(T));
    for (int zz = 0; zz < M->opts.z; ++zz) {
      if ((rc2 = launch_cg<T>(mv, U, Y, ca, cs, wmax, cm, st)))
        return fail(rc2, "CG launch failed (block too large for shared memory?)");
      ++*n;
      if ((rc2 = launch_cholqr2<T, TA>(da, Y, U, (TA*)M->d_Gp, (T*)M->d_Rsm, st, n)))
        return fail(rc2, "launch failed (Onorm)");
    }
    if ((rc2 = launch_doi_decide<T>(wave, nw, M->d_bptr, M->d_verts, (const T*)M->d_X, U,
                                    M->c_cap, M->d_cb, M->d_action, 0, eps_l, eps_h, c_min, c_max,
                                    (T*)M->d_gcol, (double*)M->d_rho, st, M->d_live, M->d_dynctl)))
      return fail(rc2, "launch failed (decision)");
    ++*n;
    return BSP_OK;
  };
  // blocks still running at the iteration cap: one more Onorm
  w.final_ = [&](int l, int q, cudaStream_t st, int* n) -> int {
    const int32_t* wave = M->d_waves + M->h_wave_off[l];
    DenseArgs da{wave, (int)M->waves[l].size(), M->d_bptr, M->d_cb, M->c_cap,
                 dyn_class_width(q, c_max), wave_rows_of(l), M->d_status};
    da.live = M->d_live;
    const int rc2 = launch_cholqr2<T, TA>(da, U, U, (TA*)M->d_Gp, (T*)M->d_Rsm, st, n);
    return rc2 ? fail(rc2, "launch failed (Onorm)") : BSP_OK;
  };
  if ((rc = ensure((void**)&M->d_dyn_launches, &M->cap_dyn_launches,
                   wave_counts_size(M, w) * sizeof(unsigned))) != BSP_OK)
    return rc;
  if ((rc = ensure_dyn_state(M)) != BSP_OK) return rc;
  realloc = realloc || g_realloc;
  if ((rc = to_device(M->d_starts, V0, (size_t)M->root_rows * c0 * sizeof(T), s)) != BSP_OK)
    return rc;
  if ((rc = to_device(M->d_X, X, (size_t)M->n * 3 * sizeof(T), s)) != BSP_OK) return rc;
  CU(cudaMemsetAsync(M->d_action, 0, sizeof(int32_t) * M->k, s));   // stop iteration per block
  CU(cudaMemsetAsync(M->d_status, 0, sizeof(int), s));
  CU(cudaMemsetAsync(M->d_cgstats, 0, sizeof(CgStats), s));
  CU(cudaMemsetAsync(M->d_dynctl, 0, sizeof(DynCtl), s));
  int launches = 0;
  const std::vector<double> key = {(double)sizeof(T), (double)sizeof(TA), (double)c0, eps_l, eps_h,
                                   (double)c_min, (double)c_max, (double)t_cap, (double)M->opts.z,
                                   M->opts.delta, M->opts.cg_rtol, (double)M->opts.cg_max_steps,
                                   (double)M->opts.cols_per_cta,
                                   (double)M->opts.cg_rows_per_lane, (double)M->c_cap};
  if ((rc = run_wave_schedule(M, w, key, realloc, &M->doi_exec, &M->doi_key, s, &launches)))
    return rc;
  // widths, stop iterations and the launch count: one read-back at the end
  std::vector<int32_t>& hc = M->h_c;
  hc.assign(M->k, 0);
  std::vector<int32_t> its(M->k, 0);
  DynCtl ctl;
  CU(cudaMemcpyAsync(hc.data(), M->d_cb, sizeof(int32_t) * M->k, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(its.data(), M->d_action, sizeof(int32_t) * M->k, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(&ctl, M->d_dynctl, sizeof(DynCtl), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  for (auto& t : its)
    if (t == 0) t = t_cap;   // still running at the cap
  std::vector<int32_t> ce(M->k + 1, 0);
  for (int b = 0; b < M->k; ++b) ce[b + 1] = ce[b] + hc[b];
  CU(cudaMemcpyAsync(M->d_ceoff, ce.data(), sizeof(int32_t) * (M->k + 1), cudaMemcpyHostToDevice, s));
  if (c_out && (rc = to_host_or_device(c_out, hc.data(), sizeof(int32_t) * M->k, s)) != BSP_OK)
    return rc;
  if (iters_out && (rc = to_host_or_device(iters_out, its.data(), sizeof(int32_t) * M->k, s)) != BSP_OK)
    return rc;
  M->stats.gpu_launches = (int)(ctl.launches + (unsigned long long)launches);
  M->tracked = true;
  M->ubf_valid = false;
  return stream_error_status(M, s);
}

template <typename T, typename TA>
int filter_forward(bsp_mesh* M, int c, int t_max, const void* V0, cudaStream_t s) {
  if (c < 1 || c > 64 || c > M->min_nb)
    return fail(BSP_ERR_INVALID_ARG, "the filter takes 1 <= c <= 64, c <= smallest block");
  if (t_max < 1) return fail(BSP_ERR_INVALID_ARG, "t_max must be >= 1");
  if (sizeof(T) == 8 && c > 64) return fail(BSP_ERR_INVALID_ARG, "FP64 precision supports c <= 64");
  int maxbatch = 0;
  for (auto& w : M->waves) maxbatch = std::max(maxbatch, (int)w.size());
  int rc;
  if ((rc = ensure_workspace<T, TA>(M, c, maxbatch)) != BSP_OK) return rc;
  const size_t nc = (size_t)M->n * c;
  if ((rc = ensure(&M->d_ckV, &M->cap_ckV, (t_max + 1) * nc * sizeof(T))) ||
      (rc = ensure(&M->d_ckY, &M->cap_ckY, t_max * nc * sizeof(T))) ||
      (rc = ensure(&M->d_starts, &M->cap_starts, (size_t)M->root_rows * c * sizeof(T))))
    return rc;
  if ((rc = to_device(M->d_starts, V0, (size_t)M->root_rows * c * sizeof(T), s))) return rc;
  M->h_c.assign(M->k, c);
  std::vector<int32_t> ce(M->k + 1, 0);
  for (int b = 0; b < M->k; ++b) ce[b + 1] = ce[b] + c;
  CU(cudaMemcpyAsync(M->d_cb, M->h_c.data(), sizeof(int32_t) * M->k, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(M->d_ceoff, ce.data(), sizeof(int32_t) * (M->k + 1), cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(M->d_status, 0, sizeof(int), s));
  CU(cudaMemsetAsync(M->d_cgstats, 0, sizeof(CgStats), s));
  if ((rc = stage_onorm_lists(M)) != BSP_OK) return rc;
  const MeshView<T> mv = view<T>(M);
  T* ckV = (T*)M->d_ckV;
  T* ckY = (T*)M->d_ckY;
  int launches = 0;
  for (int l = 0; l < (int)M->waves.size(); ++l) {
    const int nbw = (int)M->waves[l].size();
    const int32_t* batch = M->d_waves + M->h_wave_off[l];
    int wmax = 0;
    for (int b : M->waves[l]) wmax = std::max(wmax, M->h_bptr[b + 1] - M->h_bptr[b]);
    launch_init_starts<T>(batch, nbw, M->d_bptr, M->d_parent, M->d_root_off, M->d_cb, M->d_cb,
                          (const T*)M->d_starts, c, ckV, c, wmax, c, s, ckV + t_max * nc);
    ++launches;
    std::vector<int32_t> need;
    for (int b : M->waves[l]) {
      int p = M->h_parent[b];
      if (p < 0 || (M->h_bptr[b + 1] - M->h_bptr[b]) != (M->h_bptr[p + 1] - M->h_bptr[p]))
        need.push_back(b);
    }
    DenseArgs da{batch, nbw, M->d_bptr, M->d_cb, c, c, wmax, M->d_status};
    if (!need.empty()) {
      DenseArgs dn = da;
      if ((int)need.size() != nbw) {
        dn.batch = M->d_waves + M->k + M->h_wave_off[l];
        dn.nbatch = (int)need.size();
      }
      if ((rc = launch_cholqr2<T, TA>(dn, ckV, ckV, (TA*)M->d_Gp, (T*)M->d_Rsm, s, &launches)))
        return fail(rc, "launch failed (Onorm of start)");
    }
    CgArgs ca{batch, nbw, M->d_cb, c, M->opts.z, M->opts.delta, M->opts.cg_rtol,
              M->opts.cg_max_steps, M->d_status, M->d_cgstats, M->max_deg};
    ca.rows_per_lane = M->opts.cg_rows_per_lane;
    const int cs = pick_cs(M, nbw, c, sizeof(T));
    for (int t = 1; t <= t_max; ++t) {
      if ((rc = launch_cg<T>(mv, ckV + (t - 1) * nc, ckY + (t - 1) * nc, ca, cs, wmax, c, s)))
        return fail(rc, "CG launch failed");
      ++launches;
      if ((rc = launch_cholqr2<T, TA>(da, ckY + (t - 1) * nc, ckV + t * nc, (TA*)M->d_Gp,
                                      (T*)M->d_Rsm, s, &launches)))
        return fail(rc, "launch failed (Onorm)");
    }
  }
  // the final bases become the mesh's tracked bases (ld = c)
  CU(cudaMemcpyAsync(M->d_U, ckV + t_max * nc, nc * sizeof(T), cudaMemcpyDeviceToDevice, s));
  M->filter_c = c;
  M->filter_t = t_max;
  M->tracked = true;
  M->ubf_valid = false;
  M->stats.gpu_launches = launches;
  return stream_error_status(M, s);
}

template <typename T, typename TA>
int filter_backward(bsp_mesh* M, const T* dG, const T* dX, T* dW, cudaStream_t s) {
  const int c = M->filter_c, t_max = M->filter_t;
  const int cpad = (c + 3) & ~3;
  const int maxch = adjoint_maxch(M->max_nb);
  const size_t nc = (size_t)M->n * c;
  int rc;
  if ((rc = ensure(&M->d_adj_gp, &M->cap_adj_gp,
                   ((size_t)M->k * maxch * cpad * cpad + 2 * (size_t)M->k * cpad * cpad) * sizeof(TA))) ||
      (rc = ensure(&M->d_adj_thin, &M->cap_adj_thin, (size_t)M->k * 3 * 128 * 2 * sizeof(T))) ||
      (rc = ensure(&M->d_adj_rows, &M->cap_adj_rows, 3 * nc * sizeof(T))))
    return rc;
  CU(cudaMemsetAsync(M->d_status, 0, sizeof(int), s));
  CU(cudaMemsetAsync(M->d_cgstats, 0, sizeof(CgStats), s));
  AdjointArgs aa;
  aa.batch = M->d_waves;
  aa.k = M->k;
  aa.bptr = M->d_bptr;
  aa.cb = M->d_cb;
  aa.verts = M->d_verts;
  aa.blk_row = M->d_blk_row;
  aa.eoff = M->d_eoff;
  aa.n = M->n;
  aa.n_edges = M->intra_edges;
  aa.ld = c;
  aa.c = c;
  aa.t_max = t_max;
  aa.max_nb = M->max_nb;
  aa.X = dX;
  aa.G = dG;
  aa.ckV = M->d_ckV;
  aa.ckY = M->d_ckY;
  aa.ws_gp = M->d_adj_gp;
  aa.ws_thin = M->d_adj_thin;
  aa.ws_rows = M->d_adj_rows;
  aa.dW = dW;
  aa.status = M->d_status;
  aa.cgstats = M->d_cgstats;
  aa.z = M->opts.z;
  aa.delta = M->opts.delta;
  aa.rtol = M->opts.cg_rtol;
  aa.max_steps = M->opts.cg_max_steps;
  aa.max_deg = M->max_deg;
  aa.cs = pick_cs(M, M->k, c, sizeof(T));
  if ((rc = launch_filter_backward<T, TA>(aa, view<T>(M), s))) return fail(rc, "adjoint launch failed");
  return stream_error_status(M, s);
}

// --------------------------------------------------------- scratch buffers
struct Scratch {
  void* p = nullptr;
  size_t cap = 0;
};
thread_local Scratch g_scratch[3];

int scratch(int slot, size_t bytes, void** out) {
  int rc = ensure(&g_scratch[slot].p, &g_scratch[slot].cap, bytes);
  *out = g_scratch[slot].p;
  return rc;
}

// Device buffers of one synchronous call, freed when it returns.
struct DevBufs {
  std::vector<void*> p;
  ~DevBufs() {
    for (void* q : p) cudaFree(q);
  }
  void* get(size_t bytes) {
    void* q = nullptr;
    if (cudaMalloc(&q, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    p.push_back(q);
    return q;
  }
};

// X_out = U U^T X for n x 3 coordinates (real type), through the projection
// and reconstruction kernels; X and X_out host or device.
int bsp_reconstruct_projected(bsp_mesh* M, const void* X, void* X_out, cudaStream_t s) {
  const int rb = M->real_bytes;
  int64_t erows = 0;
  int cmax = 0;
  for (int b = 0; b < M->k; ++b) {
    erows += M->h_c[b];
    cmax = std::max(cmax, M->h_c[b]);
  }
  const void* dX = X;
  int rc;
  if (!is_device_ptr(X)) {
    void* t;
    if ((rc = scratch(0, (size_t)M->n * 3 * rb, &t))) return rc;
    CU(cudaMemcpyAsync(t, X, (size_t)M->n * 3 * rb, cudaMemcpyHostToDevice, s));
    dX = t;
  }
  void* dE;
  if ((rc = scratch(1, (size_t)erows * 3 * rb, &dE))) return rc;
  void* dO = X_out;
  const bool host_out = !is_device_ptr(X_out);
  if (host_out && (rc = scratch(2, (size_t)M->n * 3 * rb, &dO))) return rc;
  ProjArgs pa{M->d_bptr, M->d_verts, M->d_cb, M->d_ceoff, M->k, M->c_cap, cmax, M->max_nb, 3};
  if (rb == 8) {
    rc = launch_project<double>(pa, (const double*)M->d_U, dX, BSP_DT_F64, (double*)dE, s);
    if (!rc) rc = launch_reconstruct<double>(pa, (const double*)M->d_U, (const double*)dE, (double*)dO, s);
  } else {
    rc = launch_project<float>(pa, (const float*)M->d_U, dX, BSP_DT_F32, (float*)dE, s);
    if (!rc) rc = launch_reconstruct<float>(pa, (const float*)M->d_U, (const float*)dE, (float*)dO, s);
  }
  if (rc) return fail(rc, "projection launch failed");
  if (host_out) CU(cudaMemcpyAsync(X_out, dO, (size_t)M->n * 3 * rb, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return BSP_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

void bsp_opts_default(bsp_opts* o) {
  if (!o) return;
  o->delta = 1e-2;
  o->z = 1;
  o->weight_mode = BSP_W_COMBINATORIAL;
  o->literal_degree = 0;
  o->precision = BSP_PREC_MIXED;
  o->cg_rtol = 1e-6;
  o->cg_max_steps = 2000;
  o->rayleigh_ritz = 1;
  o->cols_per_cta = 0;
  o->use_graph = 1;
  o->schedule = BSP_SCHED_AUTO;
  o->wait_limit_ms = 2000;
  o->withhold_block = -1;
  o->cg_rows_per_lane = 0;
}

const char* bsp_last_error(void) { return g_err.c_str(); }

int bsp_mesh_create(const double* xyz, int64_t n, const int32_t* faces, int64_t m,
                    const int32_t* block_ptr, const int32_t* block_verts, int32_t k,
                    const int32_t* parent, const bsp_opts* opts, bsp_mesh** out) {
  g_err.clear();
  return create_common(xyz, n, faces, m, 3, block_ptr, block_verts, k, parent, opts, out);
}

int bsp_mesh_create_edges(const double* xyz, int64_t n, const int32_t* edges, int64_t E,
                          const int32_t* block_ptr, const int32_t* block_verts, int32_t k,
                          const int32_t* parent, const bsp_opts* opts, bsp_mesh** out) {
  g_err.clear();
  return create_common(xyz, n, edges, E, 2, block_ptr, block_verts, k, parent, opts, out);
}

int bsp_mesh_destroy(bsp_mesh* mesh) {
  if (!mesh) return BSP_OK;
  cudaDeviceSynchronize();
  release(mesh);
  delete mesh;
  return BSP_OK;
}

int bsp_get_stats(const bsp_mesh* mesh, bsp_stats* st) {
  if (!mesh || !st) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  *st = mesh->stats;
  return BSP_OK;
}

int bsp_get_edges(const bsp_mesh* M, int32_t* edges_out, int64_t* E_out) {
  g_err.clear();
  if (!M) return fail(BSP_ERR_INVALID_ARG, "mesh is NULL");
  if (E_out) *E_out = M->intra_edges;
  if (!edges_out) return BSP_OK;
  void* tmp;
  int rc = scratch(0, sizeof(int32_t) * 2 * (M->intra_edges > 0 ? M->intra_edges : 1), &tmp);
  if (rc) return rc;
  launch_edges_out(M->n, M->d_bptr, M->d_blk_row, M->d_verts, M->d_rowptr, M->d_col, M->d_eoff,
                   (int32_t*)tmp, 0);
  if ((rc = from_device(edges_out, tmp, sizeof(int32_t) * 2 * M->intra_edges, 0))) return rc;
  CU(cudaStreamSynchronize(0));
  return BSP_OK;
}

int bsp_get_block_csr(const bsp_mesh* M, int32_t b, int32_t* row_ptr, int32_t* cols, void* vals,
                      void* diag, int64_t* nnz_b) {
  g_err.clear();
  if (!M || b < 0 || b >= M->k) return fail(BSP_ERR_INVALID_ARG, "bad mesh or block id");
  const int r0 = M->h_bptr[b], nb = M->h_bptr[b + 1] - r0;
  std::vector<int32_t> rp(nb + 1);
  CU(cudaMemcpy(rp.data(), M->d_rowptr + r0, sizeof(int32_t) * (nb + 1), cudaMemcpyDeviceToHost));
  const int64_t e0 = rp[0], ne = rp[nb] - rp[0];
  if (nnz_b) *nnz_b = ne;
  int rc;
  if (row_ptr) {
    for (auto& v : rp) v -= (int32_t)e0;
    if (is_device_ptr(row_ptr)) CU(cudaMemcpy(row_ptr, rp.data(), sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice));
    else std::memcpy(row_ptr, rp.data(), sizeof(int32_t) * (nb + 1));
  }
  if (cols) {
    std::vector<uint16_t> c16(ne);
    CU(cudaMemcpy(c16.data(), M->d_col + e0, sizeof(uint16_t) * ne, cudaMemcpyDeviceToHost));
    std::vector<int32_t> c32(c16.begin(), c16.end());
    if (is_device_ptr(cols)) CU(cudaMemcpy(cols, c32.data(), sizeof(int32_t) * ne, cudaMemcpyHostToDevice));
    else std::memcpy(cols, c32.data(), sizeof(int32_t) * ne);
  }
  const int rb = M->real_bytes;
  if (vals) {
    if (M->d_wt) {
      if ((rc = from_device(vals, (const char*)M->d_wt + e0 * rb, (size_t)ne * rb, 0))) return rc;
    } else {
      std::vector<double> ones(ne, 1.0);
      std::vector<float> onesf(ne, 1.0f);
      const void* src = rb == 8 ? (const void*)ones.data() : (const void*)onesf.data();
      if (is_device_ptr(vals)) CU(cudaMemcpy(vals, src, (size_t)ne * rb, cudaMemcpyHostToDevice));
      else std::memcpy(vals, src, (size_t)ne * rb);
    }
  }
  if (diag) {
    if ((rc = from_device(diag, (const char*)M->d_diag + (size_t)r0 * rb, (size_t)nb * rb, 0))) return rc;
  }
  CU(cudaStreamSynchronize(0));
  return BSP_OK;
}

int bsp_set_edge_weights(bsp_mesh* M, const void* w, int64_t E) {
  g_err.clear();
  if (!M || !w) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (M->opts.weight_mode != BSP_W_EDGE)
    return fail(BSP_ERR_INVALID_ARG, "mesh was not created with BSP_W_EDGE");
  if (E != M->intra_edges) return fail(BSP_ERR_INVALID_ARG, "edge count mismatch");
  const int rb = M->real_bytes;
  void* tmp;
  int rc = scratch(0, (size_t)rb * (E > 0 ? E : 1), &tmp);
  if (rc) return rc;
  if ((rc = to_device(tmp, w, (size_t)rb * E, 0))) return rc;
  if (rb == 8)
    launch_set_weights<double>(M->n, M->d_bptr, M->d_blk_row, M->d_rowptr, M->d_col, M->d_eoff,
                               (const double*)tmp, M->opts.literal_degree, (double*)M->d_wt,
                               (double*)M->d_diag, 0);
  else
    launch_set_weights<float>(M->n, M->d_bptr, M->d_blk_row, M->d_rowptr, M->d_col, M->d_eoff,
                              (const float*)tmp, M->opts.literal_degree, (float*)M->d_wt,
                              (float*)M->d_diag, 0);
  CU(cudaStreamSynchronize(0));
  return BSP_OK;
}

int bsp_oi_track(bsp_mesh* M, int32_t c, int32_t t_max, const void* V0, void* stream) {
  g_err.clear();
  if (!M) return fail(BSP_ERR_INVALID_ARG, "mesh is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope ps(M);
  switch (M->opts.precision) {
    case BSP_PREC_F64: return track_fixed<double, double>(M, c, t_max, V0, s);
    case BSP_PREC_F32: return track_fixed<float, float>(M, c, t_max, V0, s);
    default: return track_fixed<float, double>(M, c, t_max, V0, s);
  }
}

int bsp_autotune(bsp_mesh* M, int32_t c, int32_t t_max, const void* V0, int32_t reps,
                 double* times_ms, int32_t* chosen, void* stream) {
  g_err.clear();
  if (!M) return fail(BSP_ERR_INVALID_ARG, "mesh is NULL");
  if (reps < 1) return fail(BSP_ERR_INVALID_ARG, "reps must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  // (columns per CTA, team CG rows per lane): the team CG in both tile shapes
  // (the 8-row form only where it applies), then the column slabs
  struct Cand { int cs, rpl, slot; };
  std::vector<Cand> cands;
  if (cgt_reg(std::min(M->max_nb, 2048), M->max_deg, M->d_wt != nullptr))
    cands.push_back({0, 8, 0});   // buckets up to 2,048 rows take the register form
  cands.push_back({0, 16, 0});
  for (int q = 1; q < 4; ++q) cands.push_back({1 << q, 0, q});
  const int keep_cs = M->opts.cols_per_cta, keep_rpl = M->opts.cg_rows_per_lane;
  double best = -1.0;
  Cand best_c{keep_cs, keep_rpl, -1};
  if (times_ms)
    for (int q = 0; q < 4; ++q) times_ms[q] = -1.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  int rc = BSP_OK;
  for (const Cand& cd : cands) {
    M->opts.cols_per_cta = cd.cs;
    M->opts.cg_rows_per_lane = cd.rpl;
    double ms_med = -1.0;
    rc = bsp_oi_track(M, c, t_max, V0, stream);   // warm-up (captures the schedule)
    if (rc == BSP_OK) {
      std::vector<double> ts;
      for (int r = 0; r < reps && rc == BSP_OK; ++r) {
        cudaEventRecord(e0, s);
        rc = bsp_oi_track(M, c, t_max, V0, stream);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ts.push_back(ms);
      }
      if (rc == BSP_OK) {
        std::sort(ts.begin(), ts.end());
        ms_med = ts[ts.size() / 2];
      }
    }
    if (rc == BSP_ERR_INVALID_ARG && cd.cs != 0) {
      rc = BSP_OK;   // this slab does not fit the mesh's blocks: not a candidate
      cudaGetLastError();
    }
    if (rc != BSP_OK) break;
    if (times_ms && ms_med >= 0 && (times_ms[cd.slot] < 0 || ms_med < times_ms[cd.slot]))
      times_ms[cd.slot] = ms_med;
    if (ms_med >= 0 && (best < 0 || ms_med < best)) {
      best = ms_med;
      best_c = cd;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  M->opts.cols_per_cta = rc == BSP_OK ? best_c.cs : keep_cs;
  M->opts.cg_rows_per_lane = rc == BSP_OK ? best_c.rpl : keep_rpl;
  if (chosen) *chosen = M->opts.cols_per_cta;
  if (rc != BSP_OK) return rc;
  g_err.clear();
  return BSP_OK;
}

int bsp_oi_track_paper_doi(bsp_mesh* M, const void* X, int32_t c0, double eps_l, double eps_h,
                           int32_t c_min, int32_t c_max, int32_t t_cap, const void* V0,
                           int32_t* c_out, int32_t* iters_out, void* stream) {
  g_err.clear();
  if (!M) return fail(BSP_ERR_INVALID_ARG, "mesh is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope ps(M);
  switch (M->opts.precision) {
    case BSP_PREC_F64:
      return track_doi<double, double>(M, X, c0, eps_l, eps_h, c_min, c_max, t_cap, V0, c_out,
                                       iters_out, s);
    case BSP_PREC_F32:
      return track_doi<float, float>(M, X, c0, eps_l, eps_h, c_min, c_max, t_cap, V0, c_out,
                                     iters_out, s);
    default:
      return track_doi<float, double>(M, X, c0, eps_l, eps_h, c_min, c_max, t_cap, V0, c_out,
                                      iters_out, s);
  }
}

int bsp_oi_track_dynamic(bsp_mesh* M, const void* X, double rel_tol, int32_t c_min,
                         int32_t c_max, int32_t c_step, int32_t t_max, uint64_t seed,
                         const void* V0, const int32_t* forced_c, int32_t* c_out, void* stream) {
  g_err.clear();
  if (!M) return fail(BSP_ERR_INVALID_ARG, "mesh is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope ps(M);
  switch (M->opts.precision) {
    case BSP_PREC_F64:
      return track_dynamic<double, double>(M, X, rel_tol, c_min, c_max, c_step, t_max, seed, V0,
                                           forced_c, c_out, s);
    case BSP_PREC_F32:
      return track_dynamic<float, float>(M, X, rel_tol, c_min, c_max, c_step, t_max, seed, V0,
                                         forced_c, c_out, s);
    default:
      return track_dynamic<float, double>(M, X, rel_tol, c_min, c_max, c_step, t_max, seed, V0,
                                          forced_c, c_out, s);
  }
}

int bsp_get_block_c(const bsp_mesh* M, int32_t* c_out) {
  g_err.clear();
  if (!M || !c_out) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (!M->tracked) return fail(BSP_ERR_INVALID_ARG, "no tracking call yet");
  if (is_device_ptr(c_out)) CU(cudaMemcpy(c_out, M->h_c.data(), sizeof(int32_t) * M->k, cudaMemcpyHostToDevice));
  else std::memcpy(c_out, M->h_c.data(), sizeof(int32_t) * M->k);
  return BSP_OK;
}

int bsp_get_basis(const bsp_mesh* M, int32_t b, void* U, int32_t* c) {
  g_err.clear();
  if (!M || b < 0 || b >= M->k) return fail(BSP_ERR_INVALID_ARG, "bad mesh or block id");
  if (!M->tracked) return fail(BSP_ERR_INVALID_ARG, "no tracking call yet");
  const int cb = M->h_c[b];
  if (c) *c = cb;
  if (!U) return BSP_OK;
  const int rb = M->real_bytes;
  const int r0 = M->h_bptr[b], nb = M->h_bptr[b + 1] - r0;
  cudaMemcpyKind kind = is_device_ptr(U) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CU(cudaMemcpy2D(U, (size_t)cb * rb, (const char*)M->d_U + (size_t)r0 * M->c_cap * rb,
                  (size_t)M->c_cap * rb, (size_t)cb * rb, nb, kind));
  return BSP_OK;
}

// BF16 copy of the tracked bases (tensor-core operand), built once per tracking call.
int ensure_basis_bf16(bsp_mesh* M, const ProjArgs& pa, cudaStream_t s, int* launched) {
  const int np = (pa.cmax + 15) & ~15;
  const size_t cap0 = M->cap_Ubf;
  int rc;
  *launched = 0;
  if ((rc = ensure(&M->d_Ubf, &M->cap_Ubf, (size_t)M->n * np * 2)) != BSP_OK) return rc;
  if (M->cap_Ubf != cap0) M->ubf_valid = false;
  if (M->ubf_valid) return BSP_OK;
  if ((rc = launch_basis_bf16(pa, (const float*)M->d_U, M->d_Ubf, s)) != BSP_OK) return rc;
  M->ubf_valid = true;
  *launched = 1;
  return BSP_OK;
}

int bsp_project(bsp_mesh* M, const void* X, int32_t x_dtype, int32_t cols, void* E_out,
                void* stream) {
  g_err.clear();
  if (!M || !X || !E_out) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (!M->tracked) return fail(BSP_ERR_INVALID_ARG, "no tracking call yet");
  if (cols < 1) return fail(BSP_ERR_INVALID_ARG, "cols must be >= 1");
  if (x_dtype == BSP_DT_BF16 && M->real_bytes == 8)
    return fail(BSP_ERR_INVALID_ARG, "bf16 input needs F32 or MIXED precision");
  cudaStream_t s = (cudaStream_t)stream;
  const int rb = M->real_bytes;
  const size_t xb = x_dtype == BSP_DT_BF16 ? 2 : x_dtype == BSP_DT_F64 ? 8 : 4;
  if (x_dtype < 0 || x_dtype > 2) return fail(BSP_ERR_INVALID_ARG, "bad x_dtype");
  int64_t erows = 0;
  int cmax = 0;
  for (int b = 0; b < M->k; ++b) {
    erows += M->h_c[b];
    cmax = std::max(cmax, M->h_c[b]);
  }
  const void* dX = X;
  int rc;
  if (!is_device_ptr(X)) {
    void* t;
    if ((rc = scratch(0, (size_t)M->n * cols * xb, &t))) return rc;
    CU(cudaMemcpyAsync(t, X, (size_t)M->n * cols * xb, cudaMemcpyHostToDevice, s));
    dX = t;
  }
  void* dE = E_out;
  const bool host_out = !is_device_ptr(E_out);
  if (host_out && (rc = scratch(1, (size_t)erows * cols * rb, &dE))) return rc;
  ProjArgs pa{M->d_bptr, M->d_verts, M->d_cb, M->d_ceoff, M->k, M->c_cap, cmax, M->max_nb, cols};
  ProfScope ps(M);
  bool tc = false;
  int conv = 0;
  if (x_dtype == BSP_DT_BF16 && rb == 4 && cols % 8 == 0 && cols >= 64 && cmax <= 256 &&
      (uintptr_t)dX % 16 == 0) {
    CU(cudaMemsetAsync(M->d_status, 0, sizeof(int), s));
    if ((rc = ensure_basis_bf16(M, pa, s, &conv)) != BSP_OK) return fail(rc, "basis conversion failed");
    rc = launch_project_tc(pa, M->d_Ubf, dX, (float*)dE, M->d_status, s);
    tc = rc == BSP_OK;
  }
  if (!tc) {
    rc = rb == 8 ? launch_project<double>(pa, (const double*)M->d_U, dX, x_dtype, (double*)dE, s)
                 : launch_project<float>(pa, (const float*)M->d_U, dX, x_dtype, (float*)dE, s);
  }
  if (rc) return fail(rc, "projection launch failed");
  if (host_out) CU(cudaMemcpyAsync(E_out, dE, (size_t)erows * cols * rb, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  M->stats.gpu_launches = 1 + conv;
  if (tc) {
    int st = 0;
    CU(cudaMemcpy(&st, M->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & ST_TIMEOUT) return fail(BSP_ERR_TIMEOUT, "a bounded device wait expired");
  }
  return BSP_OK;
}

int bsp_reconstruct(bsp_mesh* M, const void* E, int32_t cols, void* X_out, void* stream) {
  g_err.clear();
  if (!M || !E || !X_out) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (!M->tracked) return fail(BSP_ERR_INVALID_ARG, "no tracking call yet");
  if (cols < 1) return fail(BSP_ERR_INVALID_ARG, "cols must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  const int rb = M->real_bytes;
  int64_t erows = 0;
  int cmax = 0;
  for (int b = 0; b < M->k; ++b) {
    erows += M->h_c[b];
    cmax = std::max(cmax, M->h_c[b]);
  }
  const void* dE = E;
  int rc;
  if (!is_device_ptr(E)) {
    void* t;
    if ((rc = scratch(1, (size_t)erows * cols * rb, &t))) return rc;
    CU(cudaMemcpyAsync(t, E, (size_t)erows * cols * rb, cudaMemcpyHostToDevice, s));
    dE = t;
  }
  void* dX = X_out;
  const bool host_out = !is_device_ptr(X_out);
  if (host_out && (rc = scratch(2, (size_t)M->n * cols * rb, &dX))) return rc;
  ProjArgs pa{M->d_bptr, M->d_verts, M->d_cb, M->d_ceoff, M->k, M->c_cap, cmax, M->max_nb, cols};
  ProfScope ps(M);
  rc = rb == 8 ? launch_reconstruct<double>(pa, (const double*)M->d_U, (const double*)dE, (double*)dX, s)
               : launch_reconstruct<float>(pa, (const float*)M->d_U, (const float*)dE, (float*)dX, s);
  if (rc) return fail(rc, "reconstruction launch failed");
  if (host_out) CU(cudaMemcpyAsync(X_out, dX, (size_t)M->n * cols * rb, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  M->stats.gpu_launches = 1;
  return BSP_OK;
}

int bsp_reconstruct_bf16(bsp_mesh* M, const float* E, int32_t cols, float* X_out, void* stream) {
  g_err.clear();
  if (!M || !E || !X_out) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (!M->tracked) return fail(BSP_ERR_INVALID_ARG, "no tracking call yet");
  if (M->real_bytes != 4) return fail(BSP_ERR_INVALID_ARG, "needs F32 or MIXED precision");
  if (cols < 1) return fail(BSP_ERR_INVALID_ARG, "cols must be >= 1");
  if (!is_device_ptr(E) || !is_device_ptr(X_out))
    return fail(BSP_ERR_INVALID_ARG, "bsp_reconstruct_bf16 takes device pointers");
  int cmax = 0;
  for (int b = 0; b < M->k; ++b) cmax = std::max(cmax, M->h_c[b]);
  if (cmax > 128) return fail(BSP_ERR_INVALID_ARG, "c must be <= 128");
  cudaStream_t s = (cudaStream_t)stream;
  ProjArgs pa{M->d_bptr, M->d_verts, M->d_cb, M->d_ceoff, M->k, M->c_cap, cmax, M->max_nb, cols};
  ProfScope ps(M);
  CU(cudaMemsetAsync(M->d_status, 0, sizeof(int), s));
  int conv = 0;
  int rc = ensure_basis_bf16(M, pa, s, &conv);
  if (rc) return fail(rc, "basis conversion failed");
  int64_t erows = 0;
  for (int b = 0; b < M->k; ++b) erows += M->h_c[b];
  const size_t ebytes = (size_t)erows * (((size_t)cols + 7) & ~(size_t)7) * 2;
  if ((rc = ensure(&M->d_Ebf, &M->cap_Ebf, ebytes > 0 ? ebytes : 16)) != BSP_OK)
    return fail(rc, "out of device memory");
  rc = launch_recon_tc(pa, M->d_Ubf, E, erows, M->d_Ebf, X_out, M->d_status, s);
  if (rc) return fail(rc, "reconstruction launch failed");
  CU(cudaStreamSynchronize(s));
  int st = 0;
  CU(cudaMemcpy(&st, M->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st & ST_TIMEOUT) return fail(BSP_ERR_TIMEOUT, "a bounded device wait expired");
  M->stats.gpu_launches = 2 + conv;
  return BSP_OK;
}

int bsp_merge_overlapped(const bsp_mesh* M, const int32_t* orig, int64_t n_orig,
                         const void* X_copies, int32_t x_dtype, int32_t cols, void* X_out,
                         void* stream) {
  g_err.clear();
  if (!M || !orig || !X_copies || !X_out) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (n_orig < 1 || n_orig > INT32_MAX) return fail(BSP_ERR_INVALID_ARG, "n_orig out of range");
  if (cols < 1) return fail(BSP_ERR_INVALID_ARG, "cols must be >= 1");
  if (x_dtype != BSP_DT_F32 && x_dtype != BSP_DT_F64)
    return fail(BSP_ERR_INVALID_ARG, "x_dtype must be BSP_DT_F32 or BSP_DT_F64");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = M->n;
  const size_t eb = x_dtype == BSP_DT_F64 ? 8 : 4;
  // workspace: status, orig (device copy), copy weights, counts, offsets, cursors, lists
  const size_t ints = 4 + (size_t)n + (size_t)n + 3 * ((size_t)n_orig + 1) + (size_t)n;
  void* wsp;
  int rc;
  if ((rc = scratch(0, ints * sizeof(int32_t), &wsp))) return rc;
  int32_t* st = static_cast<int32_t*>(wsp);
  int32_t* d_orig = st + 4;
  float* w = reinterpret_cast<float*>(d_orig + n);
  int32_t* cnt = reinterpret_cast<int32_t*>(w + n);
  int32_t* off = cnt + n_orig + 1;
  int32_t* cur = off + n_orig + 1;
  int32_t* list = cur + n_orig + 1;
  const int32_t* orig_dev = orig;
  if (!is_device_ptr(orig)) {
    CU(cudaMemcpyAsync(d_orig, orig, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    orig_dev = d_orig;
  }
  CU(cudaMemsetAsync(st, 0, sizeof(int32_t), s));
  if ((rc = launch_ov_table(n, M->d_verts, M->d_rowptr, orig_dev, n_orig, w, cnt, st, s)))
    return fail(rc, "launch failed (copy table)");
  int h_st = 0;
  CU(cudaMemcpyAsync(&h_st, st, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  long long total = 0;
  if ((rc = exclusive_scan(cnt, off, n_orig, st, s, &total)) != BSP_OK) return rc;  // synchronises s
  if (h_st & ST_BAD_INDEX) return fail(BSP_ERR_INVALID_ARG, "orig holds a vertex id outside [0, n_orig)");
  if ((rc = launch_ov_fill(n, orig_dev, n_orig, off, cur, list, s)))
    return fail(rc, "launch failed (copy lists)");
  const void* dXc = X_copies;
  if (!is_device_ptr(X_copies)) {
    void* t;
    if ((rc = scratch(1, (size_t)n * cols * eb, &t))) return rc;
    CU(cudaMemcpyAsync(t, X_copies, (size_t)n * cols * eb, cudaMemcpyHostToDevice, s));
    dXc = t;
  }
  void* dXo = X_out;
  const bool host_out = !is_device_ptr(X_out);
  if (host_out && (rc = scratch(2, (size_t)n_orig * cols * eb, &dXo))) return rc;
  rc = eb == 8 ? launch_ov_merge<double>(n_orig, cols, off, list, w, (const double*)dXc,
                                         (double*)dXo, s)
               : launch_ov_merge<float>(n_orig, cols, off, list, w, (const float*)dXc,
                                        (float*)dXo, s);
  if (rc) return fail(rc, "launch failed (merge)");
  if (host_out) CU(cudaMemcpyAsync(X_out, dXo, (size_t)n_orig * cols * eb, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return BSP_OK;
}

int bsp_spmm(bsp_mesh* M, const void* P, void* Y, int32_t c, void* stream) {
  g_err.clear();
  if (!M || !P || !Y) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (c < 1 || c > 128) return fail(BSP_ERR_INVALID_ARG, "c must be in [1, 128]");
  if (!is_device_ptr(P) || !is_device_ptr(Y))
    return fail(BSP_ERR_INVALID_ARG, "bsp_spmm takes device pointers");
  cudaStream_t s = (cudaStream_t)stream;
  if (!M->d_spmm_chunks) {
    // chunk table, once per mesh: rows on the host, neighbour ranges on the device
    std::vector<int32_t> ch = spmm_chunk_rows(M->h_bptr);
    const int nch = (int)(ch.size() / 8);
    void* d = nullptr;
    if (cudaMalloc(&d, sizeof(int32_t) * (ch.empty() ? 8 : ch.size())) != cudaSuccess) {
      cudaGetLastError();
      return fail(BSP_ERR_OOM, "device allocation failed");
    }
    CU(cudaMemcpy(d, ch.data(), sizeof(int32_t) * ch.size(), cudaMemcpyHostToDevice));
    launch_spmm_ranges(view<float>(M), M->d_blk_row, (int32_t*)d, nch, 0);
    CU(cudaMemcpy(ch.data(), d, sizeof(int32_t) * ch.size(), cudaMemcpyDeviceToHost));
    int span = 0, mnnz = 0;
    for (int q = 0; q < nch; ++q) {
      span = std::max(span, ch[8 * q + 3] - ch[8 * q + 2] + 1);
      mnnz = std::max(mnnz, ch[8 * q + 5]);
    }
    M->d_spmm_chunks = (int32_t*)d;
    M->spmm_nchunks = nch;
    M->spmm_max_span = span;
    M->spmm_max_nnz = mnnz;
  }
  ProfScope ps(M);
  int rc;
  if (M->real_bytes == 8) {
    rc = launch_spmm_tiled<double>(view<double>(M), M->d_spmm_chunks, M->spmm_nchunks, M->spmm_max_span,
                                   M->spmm_max_nnz, M->opts.delta, (const double*)P, (double*)Y, c, s);
    if (rc == BSP_ERR_INVALID_ARG)
      launch_spmm<double>(M->n, view<double>(M), M->d_blk_row, M->opts.delta, (const double*)P,
                          (double*)Y, c, s);
  } else {
    rc = launch_spmm_tiled<float>(view<float>(M), M->d_spmm_chunks, M->spmm_nchunks, M->spmm_max_span,
                                  M->spmm_max_nnz, (float)M->opts.delta, (const float*)P, (float*)Y, c, s);
    if (rc == BSP_ERR_INVALID_ARG)
      launch_spmm<float>(M->n, view<float>(M), M->d_blk_row, (float)M->opts.delta, (const float*)P,
                         (float*)Y, c, s);
  }
  CU(cudaGetLastError());
  M->stats.gpu_launches = 1;
  return BSP_OK;
}

int bsp_filter_forward(bsp_mesh* M, int32_t c, int32_t t_max, const void* V0_roots,
                       const void* X, void* X_out, void* stream) {
  g_err.clear();
  if (!M || !V0_roots || !X || !X_out) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (M->opts.z != 1) return fail(BSP_ERR_INVALID_ARG, "the filter adjoint supports z = 1");
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope ps(M);
  int rc;
  switch (M->opts.precision) {
    case BSP_PREC_F64: rc = filter_forward<double, double>(M, c, t_max, V0_roots, s); break;
    case BSP_PREC_F32: rc = filter_forward<float, float>(M, c, t_max, V0_roots, s); break;
    default: rc = filter_forward<float, double>(M, c, t_max, V0_roots, s); break;
  }
  if (rc != BSP_OK) return rc;
  return bsp_reconstruct_projected(M, X, X_out, s);
}

int bsp_filter_backward(bsp_mesh* M, const void* G, const void* X, void* dX, void* dW,
                        void* stream) {
  g_err.clear();
  if (!M || !G || !X || !dX || !dW) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (M->filter_t < 1) return fail(BSP_ERR_INVALID_ARG, "call bsp_filter_forward first");
  if (!is_device_ptr(G) || !is_device_ptr(X) || !is_device_ptr(dX) || !is_device_ptr(dW))
    return fail(BSP_ERR_INVALID_ARG, "bsp_filter_backward takes device pointers");
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope ps(M);
  int rc = bsp_reconstruct_projected(M, G, dX, s);   // dL/dX = U U^T G
  if (rc != BSP_OK) return rc;
  switch (M->opts.precision) {
    case BSP_PREC_F64:
      return filter_backward<double, double>(M, (const double*)G, (const double*)X, (double*)dW, s);
    case BSP_PREC_F32:
      return filter_backward<float, float>(M, (const float*)G, (const float*)X, (float*)dW, s);
    default:
      return filter_backward<float, double>(M, (const float*)G, (const float*)X, (float*)dW, s);
  }
}

int bsp_set_profiling(bsp_mesh* M, int32_t on) {
  g_err.clear();
  if (!M) return fail(BSP_ERR_INVALID_ARG, "mesh is NULL");
  M->profiling = on ? 1 : 0;
  for (int c = 0; c < KC_COUNT; ++c) {
    M->prof_ms[c] = 0.0;
    M->prof_n[c] = 0;
  }
  return BSP_OK;
}

int bsp_get_kernel_times(const bsp_mesh* M, double* ms_out, int32_t* launches_out,
                         int32_t n_classes) {
  g_err.clear();
  if (!M || n_classes < 0) return fail(BSP_ERR_INVALID_ARG, "bad argument");
  for (int c = 0; c < n_classes && c < KC_COUNT; ++c) {
    if (ms_out) ms_out[c] = M->prof_ms[c];
    if (launches_out) launches_out[c] = M->prof_n[c];
  }
  return BSP_OK;
}

int bsp_quantize(bsp_mesh* M, const void* E, int32_t cols, int32_t bits, uint16_t* codes,
                 void* range, void* stream) {
  g_err.clear();
  if (!M || !E || !codes || !range) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (!M->tracked) return fail(BSP_ERR_INVALID_ARG, "no tracking call yet");
  if (cols < 1) return fail(BSP_ERR_INVALID_ARG, "cols must be >= 1");
  if (bits < 1 || bits > 16) return fail(BSP_ERR_INVALID_ARG, "bits must be in [1, 16]");
  cudaStream_t s = (cudaStream_t)stream;
  const int rb = M->real_bytes;
  int64_t erows = 0;
  for (int b = 0; b < M->k; ++b) erows += M->h_c[b];
  const size_t ne = (size_t)erows * cols, nr = (size_t)M->k * cols * 2;
  int rc;
  const void* dE = E;
  if (!is_device_ptr(E)) {
    void* t;
    if ((rc = scratch(0, ne * rb, &t))) return rc;
    CU(cudaMemcpyAsync(t, E, ne * rb, cudaMemcpyHostToDevice, s));
    dE = t;
  }
  void* dC = codes;
  const bool host_codes = !is_device_ptr(codes);
  if (host_codes && (rc = scratch(1, ne * sizeof(uint16_t), &dC))) return rc;
  void* dR = range;
  const bool host_range = !is_device_ptr(range);
  if (host_range && (rc = scratch(2, nr * rb, &dR))) return rc;
  rc = rb == 8 ? launch_quantize<double>(M->d_ceoff, M->k, (const double*)dE, cols, bits,
                                         (uint16_t*)dC, (double*)dR, s)
               : launch_quantize<float>(M->d_ceoff, M->k, (const float*)dE, cols, bits,
                                        (uint16_t*)dC, (float*)dR, s);
  if (rc) return fail(rc, "quantiser launch failed");
  if (host_codes) CU(cudaMemcpyAsync(codes, dC, ne * sizeof(uint16_t), cudaMemcpyDeviceToHost, s));
  if (host_range) CU(cudaMemcpyAsync(range, dR, nr * rb, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  M->stats.gpu_launches = 1;
  return BSP_OK;
}

int bsp_dequantize(bsp_mesh* M, const uint16_t* codes, const void* range, int32_t cols,
                   int32_t bits, void* E_out, void* stream) {
  g_err.clear();
  if (!M || !codes || !range || !E_out) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (!M->tracked) return fail(BSP_ERR_INVALID_ARG, "no tracking call yet");
  if (cols < 1) return fail(BSP_ERR_INVALID_ARG, "cols must be >= 1");
  if (bits < 1 || bits > 16) return fail(BSP_ERR_INVALID_ARG, "bits must be in [1, 16]");
  cudaStream_t s = (cudaStream_t)stream;
  const int rb = M->real_bytes;
  int64_t erows = 0;
  for (int b = 0; b < M->k; ++b) erows += M->h_c[b];
  const size_t ne = (size_t)erows * cols, nr = (size_t)M->k * cols * 2;
  int rc;
  const void* dC = codes;
  if (!is_device_ptr(codes)) {
    void* t;
    if ((rc = scratch(0, ne * sizeof(uint16_t), &t))) return rc;
    CU(cudaMemcpyAsync(t, codes, ne * sizeof(uint16_t), cudaMemcpyHostToDevice, s));
    dC = t;
  }
  const void* dR = range;
  if (!is_device_ptr(range)) {
    void* t;
    if ((rc = scratch(2, nr * rb, &t))) return rc;
    CU(cudaMemcpyAsync(t, range, nr * rb, cudaMemcpyHostToDevice, s));
    dR = t;
  }
  void* dE = E_out;
  const bool host_out = !is_device_ptr(E_out);
  if (host_out && (rc = scratch(1, ne * rb, &dE))) return rc;
  rc = rb == 8 ? launch_dequantize<double>(M->d_ceoff, M->k, (const uint16_t*)dC,
                                           (const double*)dR, cols, bits, (double*)dE, s)
               : launch_dequantize<float>(M->d_ceoff, M->k, (const uint16_t*)dC,
                                          (const float*)dR, cols, bits, (float*)dE, s);
  if (rc) return fail(rc, "dequantiser launch failed");
  if (host_out) CU(cudaMemcpyAsync(E_out, dE, ne * rb, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  M->stats.gpu_launches = 1;
  return BSP_OK;
}

int bsp_bits_per_vertex(const bsp_mesh* M, int32_t bits, double* bpv) {
  g_err.clear();
  if (!M || !bpv) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (!M->tracked) return fail(BSP_ERR_INVALID_ARG, "no tracking call yet");
  if (bits < 1 || bits > 16) return fail(BSP_ERR_INVALID_ARG, "bits must be in [1, 16]");
  int64_t csum = 0;
  for (int b = 0; b < M->k; ++b) csum += M->h_c[b];
  *bpv = 3.0 * bits * (double)csum / (double)M->n;
  return BSP_OK;
}

int bsp_nmsve(const void* X, const void* X_rec, int32_t dtype, int64_t n, const int32_t* faces,
              int64_t m, double* out, void* stream) {
  g_err.clear();
  if (!X || !X_rec || !out || (m > 0 && !faces)) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (n < 1 || n >= INT32_MAX || m < 0 || m > INT32_MAX / 2)
    return fail(BSP_ERR_INVALID_ARG, "n or m out of range");
  if (dtype != BSP_DT_F32 && dtype != BSP_DT_F64)
    return fail(BSP_ERR_INVALID_ARG, "dtype must be BSP_DT_F32 or BSP_DT_F64");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t xb = dtype == BSP_DT_F64 ? 8 : 4;
  DevBufs bufs;
  const void* dX = X;
  const void* dXr = X_rec;
  const int32_t* dF = faces;
  if (!is_device_ptr(X)) {
    void* t = bufs.get((size_t)n * 3 * xb);
    if (!t) return fail(BSP_ERR_OOM, "device allocation failed");
    CU(cudaMemcpyAsync(t, X, (size_t)n * 3 * xb, cudaMemcpyHostToDevice, s));
    dX = t;
  }
  if (!is_device_ptr(X_rec)) {
    void* t = bufs.get((size_t)n * 3 * xb);
    if (!t) return fail(BSP_ERR_OOM, "device allocation failed");
    CU(cudaMemcpyAsync(t, X_rec, (size_t)n * 3 * xb, cudaMemcpyHostToDevice, s));
    dXr = t;
  }
  if (m > 0 && !is_device_ptr(faces)) {
    void* t = bufs.get((size_t)m * 3 * sizeof(int32_t));
    if (!t) return fail(BSP_ERR_OOM, "device allocation failed");
    CU(cudaMemcpyAsync(t, faces, (size_t)m * 3 * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    dF = (const int32_t*)t;
  }
  // [status, pad] [acc0, acc1] then cnt, off, cur: n + 1 ints each
  char* w = (char*)bufs.get(32 + 3 * (size_t)(n + 1) * sizeof(int32_t));
  if (!w) return fail(BSP_ERR_OOM, "device allocation failed");
  int* d_status = (int*)w;
  double* d_acc = (double*)(w + 16);
  int32_t* cnt = (int32_t*)(w + 32);
  int32_t* off = cnt + (n + 1);
  int32_t* cur = off + (n + 1);
  CU(cudaMemsetAsync(w, 0, 32 + 3 * (size_t)(n + 1) * sizeof(int32_t), s));
  if (m > 0) launch_nm_count(m, dF, n, cnt, d_status, s);
  long long total = 0;
  int rc = exclusive_scan(cnt, off, n, d_status, s, &total);
  if (rc) return fail(rc, "scan failed");
  int st = 0;
  CU(cudaMemcpy(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st & ST_BAD_INDEX) return fail(BSP_ERR_INVALID_ARG, "face vertex index out of range");
  if (st) return fail(BSP_ERR_INVALID_ARG, "too many neighbour entries");
  int32_t* nbr = (int32_t*)bufs.get((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  if (!nbr) return fail(BSP_ERR_OOM, "device allocation failed");
  if (m > 0) launch_nm_fill(m, dF, n, off, cur, nbr, s);
  rc = dtype == BSP_DT_F64
           ? launch_nm_err<double>(n, off, nbr, (const double*)dX, (const double*)dXr, d_acc, s)
           : launch_nm_err<float>(n, off, nbr, (const float*)dX, (const float*)dXr, d_acc, s);
  if (rc) return fail(rc, "NMSVE launch failed");
  double acc[2];
  CU(cudaMemcpyAsync(acc, d_acc, sizeof(acc), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  out[1] = std::sqrt(acc[0]);
  out[2] = std::sqrt(acc[1]);
  out[0] = (out[1] + out[2]) / (2.0 * (double)n);
  return BSP_OK;
}

int bsp_fine_denoise(const void* X, void* X_out, void* normals_out, int32_t dtype, int64_t n,
                     const int32_t* faces, int64_t m, double sigma_s, double sigma_r,
                     int32_t normal_iters, int32_t vertex_iters, void* stream) {
  g_err.clear();
  if (!X || !X_out || (m > 0 && !faces)) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (n < 1 || n >= INT32_MAX || m < 0 || m > INT32_MAX / 3)
    return fail(BSP_ERR_INVALID_ARG, "n or m out of range");
  if (dtype != BSP_DT_F32 && dtype != BSP_DT_F64)
    return fail(BSP_ERR_INVALID_ARG, "dtype must be BSP_DT_F32 or BSP_DT_F64");
  if (!(sigma_s > 0) || !(sigma_r > 0) || !std::isfinite(sigma_s) || !std::isfinite(sigma_r))
    return fail(BSP_ERR_INVALID_ARG, "sigma_s and sigma_r must be positive and finite");
  if (normal_iters < 0 || vertex_iters < 0)
    return fail(BSP_ERR_INVALID_ARG, "iteration counts must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t xb = dtype == BSP_DT_F64 ? 8 : 4;
  DevBufs bufs;
  const size_t xbytes = (size_t)n * 3 * xb, fbytes = (size_t)(m > 0 ? m : 1) * 3 * xb;
  char* X0 = (char*)bufs.get(xbytes);
  char* X1 = (char*)bufs.get(xbytes);
  char* N0 = (char*)bufs.get(fbytes);
  char* N1 = (char*)bufs.get(fbytes);
  char* cen = (char*)bufs.get(fbytes);
  char* area = (char*)bufs.get((size_t)(m > 0 ? m : 1) * xb);
  char* w = (char*)bufs.get(16 + 3 * (size_t)(n + 1) * sizeof(int32_t));
  if (!X0 || !X1 || !N0 || !N1 || !cen || !area || !w)
    return fail(BSP_ERR_OOM, "device allocation failed");
  int* d_status = (int*)w;
  int32_t* cnt = (int32_t*)(w + 16);
  int32_t* off = cnt + (n + 1);
  int32_t* cur = off + (n + 1);
  CU(cudaMemsetAsync(w, 0, 16 + 3 * (size_t)(n + 1) * sizeof(int32_t), s));
  int rc;
  if ((rc = to_device(X0, X, xbytes, s)) != BSP_OK) return rc;
  const int32_t* dF = faces;
  if (m > 0 && !is_device_ptr(faces)) {
    void* t = bufs.get((size_t)m * 3 * sizeof(int32_t));
    if (!t) return fail(BSP_ERR_OOM, "device allocation failed");
    CU(cudaMemcpyAsync(t, faces, (size_t)m * 3 * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    dF = (const int32_t*)t;
  }
  launch_vf_table(m, dF, n, cnt, d_status, s);
  long long total = 0;
  if ((rc = exclusive_scan(cnt, off, n, d_status, s, &total)) != BSP_OK) return fail(rc, "scan failed");
  int st = 0;
  CU(cudaMemcpy(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st & ST_BAD_INDEX) return fail(BSP_ERR_INVALID_ARG, "face vertex index out of range");
  if (st) return fail(BSP_ERR_INVALID_ARG, "too many face entries");
  int32_t* vf = (int32_t*)bufs.get((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  if (!vf) return fail(BSP_ERR_OOM, "device allocation failed");
  launch_vf_fill(m, dF, n, off, cur, vf, s);
  void* Xf = nullptr;
  void* Nf = nullptr;
  if (dtype == BSP_DT_F64) {
    double *xf, *nf;
    rc = launch_fine_denoise<double>(n, m, dF, off, vf, (double*)X0, (double*)X1, (double*)N0,
                                     (double*)N1, (double*)cen, (double*)area, sigma_s, sigma_r,
                                     normal_iters, vertex_iters, &xf, &nf, s);
    Xf = xf;
    Nf = nf;
  } else {
    float *xf, *nf;
    rc = launch_fine_denoise<float>(n, m, dF, off, vf, (float*)X0, (float*)X1, (float*)N0,
                                    (float*)N1, (float*)cen, (float*)area, sigma_s, sigma_r,
                                    normal_iters, vertex_iters, &xf, &nf, s);
    Xf = xf;
    Nf = nf;
  }
  if (rc) return fail(rc, "fine denoising launch failed");
  if ((rc = from_device(X_out, Xf, xbytes, s)) != BSP_OK) return rc;
  if (normals_out && m > 0 && (rc = from_device(normals_out, Nf, (size_t)m * 3 * xb, s)) != BSP_OK)
    return rc;
  CU(cudaStreamSynchronize(s));
  return BSP_OK;
}

int bsp_normal_angle_error(const void* X, const void* X_ref, int32_t dtype, int64_t n,
                           const int32_t* faces, int64_t m, double* theta_deg, void* stream) {
  g_err.clear();
  if (!X || !X_ref || !theta_deg || (m > 0 && !faces))
    return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (n < 1 || n >= INT32_MAX || m < 0 || m > INT32_MAX / 3)
    return fail(BSP_ERR_INVALID_ARG, "n or m out of range");
  if (dtype != BSP_DT_F32 && dtype != BSP_DT_F64)
    return fail(BSP_ERR_INVALID_ARG, "dtype must be BSP_DT_F32 or BSP_DT_F64");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t xb = dtype == BSP_DT_F64 ? 8 : 4;
  const size_t xbytes = (size_t)n * 3 * xb;
  DevBufs bufs;
  const void* dX = X;
  const void* dXr = X_ref;
  const int32_t* dF = faces;
  if (!is_device_ptr(X)) {
    void* t = bufs.get(xbytes);
    if (!t) return fail(BSP_ERR_OOM, "device allocation failed");
    CU(cudaMemcpyAsync(t, X, xbytes, cudaMemcpyHostToDevice, s));
    dX = t;
  }
  if (!is_device_ptr(X_ref)) {
    void* t = bufs.get(xbytes);
    if (!t) return fail(BSP_ERR_OOM, "device allocation failed");
    CU(cudaMemcpyAsync(t, X_ref, xbytes, cudaMemcpyHostToDevice, s));
    dXr = t;
  }
  if (m > 0 && !is_device_ptr(faces)) {
    void* t = bufs.get((size_t)m * 3 * sizeof(int32_t));
    if (!t) return fail(BSP_ERR_OOM, "device allocation failed");
    CU(cudaMemcpyAsync(t, faces, (size_t)m * 3 * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    dF = (const int32_t*)t;
  }
  // face indices are checked by the vertex -> face count (nothing else is kept)
  char* w = (char*)bufs.get(32 + (size_t)(n + 1) * sizeof(int32_t));
  if (!w) return fail(BSP_ERR_OOM, "device allocation failed");
  int* d_status = (int*)w;
  double* d_acc = (double*)(w + 8);
  unsigned long long* d_cnt = (unsigned long long*)(w + 16);
  CU(cudaMemsetAsync(w, 0, 32 + (size_t)(n + 1) * sizeof(int32_t), s));
  launch_vf_table(m, dF, n, (int32_t*)(w + 32), d_status, s);
  int st = 0;
  CU(cudaMemcpyAsync(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (st & ST_BAD_INDEX) return fail(BSP_ERR_INVALID_ARG, "face vertex index out of range");
  int rc = dtype == BSP_DT_F64
               ? launch_normal_angle<double>(m, dF, (const double*)dX, (const double*)dXr, d_acc,
                                             d_cnt, s)
               : launch_normal_angle<float>(m, dF, (const float*)dX, (const float*)dXr, d_acc,
                                            d_cnt, s);
  if (rc) return fail(rc, "normal angle launch failed");
  double acc = 0.0;
  unsigned long long c = 0;
  CU(cudaMemcpyAsync(&acc, d_acc, sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(&c, d_cnt, sizeof(c), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  *theta_deg = c ? acc / (double)c * (180.0 / 3.14159265358979323846) : 0.0;
  return BSP_OK;
}

}  // extern "C"
