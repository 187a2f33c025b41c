// Per-block Laplacian assembly on the GPU (Sec. 3: edges derived from F,
// L = D - C; Sec. 4: the mesh is split into k blocks, each processed on its
// own; Sec. 6.1: a block sees only its own edges).
//
// Pipeline (integer work, once per mesh, deterministic result):
//   1. row_of[v]: the block-order row of every vertex (checks range/duplicates)
//   2. count half-edges per row for every face side whose ends share a block
//   3. exclusive scan -> neighbour-slot offsets; scatter neighbour local ids
//   4. per row: sort + unique the neighbour list (faces share sides)
//   5. exclusive scan of unique counts -> rowptr; compact into uint16 cols
//   6. per row: count of neighbours with a larger local id -> scan -> canonical
//      edge ids (block, i, j), i < j, lexicographic
#include <climits>
#include <cstdio>

#include "bsp_internal.cuh"

namespace bsp {
namespace {

constexpr int kScanTile = 1024;  // elements per CTA in the scan (256 threads x 4)

__global__ void k_scan_tiles(const int32_t* in, int32_t* out, long long* tsum, int64_t n) {
  __shared__ long long warp_tot[8];
  int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * 4;
  long long v[4];
  long long s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[i] = (base + i < n) ? (long long)in[base + i] : 0;
    s += v[i];
  }
  // inclusive warp scan of the thread sums
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  long long woff = 0;
  for (int i = 0; i < w; ++i) woff += warp_tot[i];
  long long excl = woff + incl - s;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (base + i < n) out[base + i] = (int32_t)excl;  // tile-local, fixed up below
    excl += v[i];
  }
  if (threadIdx.x == blockDim.x - 1) tsum[blockIdx.x] = woff + incl;
}

// One CTA: exclusive scan of the tile sums in place; writes the grand total.
__global__ void k_scan_sums(long long* tsum, int64_t ntiles, long long* total) {
  __shared__ long long warp_tot[32];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t b0 = 0; b0 < ntiles; b0 += blockDim.x) {
    int64_t i = b0 + threadIdx.x;
    long long s = i < ntiles ? tsum[i] : 0;
    long long incl = s;
    for (int o = 1; o < 32; o <<= 1) {
      long long t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    long long woff = 0;
    for (int j = 0; j < w; ++j) woff += warp_tot[j];
    long long c0 = carry;
    if (i < ntiles) tsum[i] = c0 + woff + incl - s;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long t = 0;
      for (int j = 0; j < nw; ++j) t += warp_tot[j];
      carry = c0 + t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int32_t* out, const long long* tsum, int64_t n, const long long* total,
                           int* status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    long long v = (long long)out[i] + tsum[i / kScanTile];
    out[i] = (int32_t)v;
  }
  if (i == 0) {
    long long t = *total;
    if (t > INT_MAX) atomicOr(status, ST_DEGREE);
    out[n] = (int32_t)t;
  }
}

}  // namespace

// out[0..n] = exclusive scan of in[0..n-1]; out[n] = total.  Returns the total on the host.
int exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int* d_status, cudaStream_t s,
                   long long* h_total) {
  int64_t ntiles = (n + kScanTile - 1) / kScanTile;
  if (ntiles == 0) ntiles = 1;
  long long* tmp = nullptr;
  if (cudaMalloc(&tmp, sizeof(long long) * (ntiles + 1)) != cudaSuccess) return BSP_ERR_OOM;
  k_scan_tiles<<<(unsigned)ntiles, 256, 0, s>>>(in, out, tmp, n);
  k_scan_sums<<<1, 1024, 0, s>>>(tmp, ntiles, tmp + ntiles);
  k_scan_add<<<ceil_div(n > 0 ? n : 1, 256), 256, 0, s>>>(out, tmp, n, tmp + ntiles, d_status);
  cudaError_t e = cudaMemcpyAsync(h_total, tmp + ntiles, sizeof(long long),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(tmp);
  return e == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

namespace {

__global__ void k_rows(int32_t k, const int32_t* bptr, int32_t* blk_row) {
  int b = blockIdx.x;
  for (int r = bptr[b] + threadIdx.x; r < bptr[b + 1]; r += blockDim.x) blk_row[r] = b;
}

__global__ void k_locate(int64_t n, const int32_t* verts, int32_t* row_of, int* status) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = verts[r];
    if (v < 0 || v >= n) {
      atomicOr(status, ST_BAD_INDEX);
      continue;
    }
    int old = atomicExch(&row_of[v], (int32_t)r);
    if (old != -1) atomicOr(status, ST_DUP_VERTEX);
  }
}

// Side s of element f: (tri[f*arity + s], tri[f*arity + (s+1) % arity]).
// For faces (arity 3) this lists the three sides; for edges (arity 2) one side.
__device__ __forceinline__ bool side_rows(int64_t e, int arity, const int32_t* tri, int64_t n,
                                          const int32_t* row_of, const int32_t* blk_row,
                                          int32_t* ru, int32_t* rv, int* status) {
  int per = arity == 3 ? 3 : 1;
  int64_t f = e / per;
  int s = (int)(e % per);
  int32_t u = tri[f * arity + s];
  int32_t v = tri[f * arity + (s + 1) % arity];
  if (u < 0 || u >= n || v < 0 || v >= n) {
    atomicOr(status, ST_BAD_INDEX);
    return false;
  }
  if (u == v) return false;
  int32_t a = row_of[u], b = row_of[v];
  if (a < 0 || b < 0) return false;
  if (blk_row[a] != blk_row[b]) return false;
  *ru = a;
  *rv = b;
  return true;
}

__global__ void k_count(int64_t nside, int arity, const int32_t* tri, int64_t n,
                        const int32_t* row_of, const int32_t* blk_row, int32_t* cnt, int* status) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nside;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t a, b;
    if (side_rows(e, arity, tri, n, row_of, blk_row, &a, &b, status)) {
      atomicAdd(&cnt[a], 1);
      atomicAdd(&cnt[b], 1);
    }
  }
}

__global__ void k_fill(int64_t nside, int arity, const int32_t* tri, int64_t n,
                       const int32_t* row_of, const int32_t* blk_row, const int32_t* bptr,
                       const int32_t* off, int32_t* cur, int32_t* nbr, int* status) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nside;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t a, b;
    if (side_rows(e, arity, tri, n, row_of, blk_row, &a, &b, status)) {
      int32_t base = bptr[blk_row[a]];
      int pa = atomicAdd(&cur[a], 1);
      int pb = atomicAdd(&cur[b], 1);
      nbr[off[a] + pa] = b - base;
      nbr[off[b] + pb] = a - base;
    }
  }
}

__global__ void k_sort_unique(int64_t n, const int32_t* off, int32_t* nbr, const int32_t* bptr,
                              const int32_t* blk_row, int32_t* ucnt, int32_t* up) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t* a = nbr + off[r];
    int len = off[r + 1] - off[r];
    for (int i = 1; i < len; ++i) {  // insertion sort: lists are short
      int32_t x = a[i];
      int j = i - 1;
      while (j >= 0 && a[j] > x) {
        a[j + 1] = a[j];
        --j;
      }
      a[j + 1] = x;
    }
    int u = 0;
    for (int i = 0; i < len; ++i)
      if (u == 0 || a[i] != a[u - 1]) a[u++] = a[i];
    int32_t me = (int32_t)(r - bptr[blk_row[r]]);
    int cu = 0;
    for (int i = 0; i < u; ++i) cu += a[i] > me;
    ucnt[r] = u;
    up[r] = cu;
  }
}

__global__ void k_compact(int64_t n, const int32_t* off, const int32_t* nbr, const int32_t* rowptr,
                          uint16_t* col) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int len = rowptr[r + 1] - rowptr[r];
    const int32_t* a = nbr + off[r];
    uint16_t* o = col + rowptr[r];
    for (int i = 0; i < len; ++i) o[i] = (uint16_t)a[i];
  }
}

template <typename T>
__global__ void k_weights(int64_t n, const int32_t* bptr, const int32_t* blk_row,
                          const int32_t* verts, const int32_t* rowptr, const uint16_t* col,
                          const double* xyz, int mode, int literal, T* wt, T* diag) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t base = bptr[blk_row[r]];
    double sum = 0.0;
    int cnt = 0;
    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
      double w = 1.0;
      if (mode == BSP_W_INV_SQ_DIST) {
        int32_t u = verts[r], v = verts[base + col[p]];
        double dx = xyz[3 * (int64_t)u] - xyz[3 * (int64_t)v];
        double dy = xyz[3 * (int64_t)u + 1] - xyz[3 * (int64_t)v + 1];
        double dz = xyz[3 * (int64_t)u + 2] - xyz[3 * (int64_t)v + 2];
        w = 1.0 / (dx * dx + dy * dy + dz * dz);
      }
      if (wt) wt[p] = (T)w;
      sum += w;
      ++cnt;
    }
    diag[r] = literal ? (T)cnt : (T)sum;
  }
}

// Rank of local id `j` among the larger-than-`i` neighbours of row r (sorted).
__device__ __forceinline__ int upper_rank(const uint16_t* c, int len, int up, int j) {
  int first = len - up;  // first entry above the row's own id
  int lo = first, hi = len - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if ((int)c[mid] < j) lo = mid + 1; else hi = mid;
  }
  return lo - first;
}

template <typename T>
__global__ void k_set_weights(int64_t n, const int32_t* bptr, const int32_t* blk_row,
                              const int32_t* rowptr, const uint16_t* col, const int32_t* eoff,
                              const T* w_edges, int literal, T* wt, T* diag) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t base = bptr[blk_row[r]];
    int i = (int)(r - base);
    double sum = 0.0;
    int cnt = 0;
    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
      int j = col[p];
      int64_t rr = j > i ? r : base + j;      // the row that owns edge (min, max)
      int other = j > i ? j : i;
      int len = rowptr[rr + 1] - rowptr[rr];
      int up = eoff[rr + 1] - eoff[rr];
      int e = eoff[rr] + upper_rank(col + rowptr[rr], len, up, other);
      T w = w_edges[e];
      wt[p] = w;
      sum += (double)w;
      ++cnt;
    }
    diag[r] = literal ? (T)cnt : (T)sum;
  }
}

__global__ void k_edges_out(int64_t n, const int32_t* bptr, const int32_t* blk_row,
                            const int32_t* verts, const int32_t* rowptr, const uint16_t* col,
                            const int32_t* eoff, int32_t* edges) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t base = bptr[blk_row[r]];
    int i = (int)(r - base);
    int e = eoff[r];
    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
      int j = col[p];
      if (j > i) {
        edges[2 * (int64_t)e] = verts[r];
        edges[2 * (int64_t)e + 1] = verts[base + j];
        ++e;
      }
    }
  }
}

inline unsigned grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

int assemble_pattern(int64_t n, const int32_t* d_tri, int64_t m, int arity,
                     const int32_t* d_bptr, const int32_t* d_verts, int32_t k,
                     AssemblyOut* out, int* d_status, cudaStream_t s, std::string* err) {
  int32_t *row_of = nullptr, *cnt = nullptr, *off = nullptr, *cur = nullptr, *nbr = nullptr,
          *ucnt = nullptr, *up = nullptr;
  int rc = BSP_OK;
  long long total = 0, nnz = 0, nedge = 0;
  int64_t nside = m * (arity == 3 ? 3 : 1);
  auto fail = [&](int code, const char* msg) {
    if (err) *err = msg;
    rc = code;
  };
  do {
    if (cudaMalloc(&out->blk_row, sizeof(int32_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&row_of, sizeof(int32_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&cnt, sizeof(int32_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&off, sizeof(int32_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&cur, sizeof(int32_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&ucnt, sizeof(int32_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&up, sizeof(int32_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&out->rowptr, sizeof(int32_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&out->eoff, sizeof(int32_t) * (n + 1)) != cudaSuccess) {
      fail(BSP_ERR_OOM, "device allocation failed during assembly");
      break;
    }
    cudaMemsetAsync(row_of, 0xff, sizeof(int32_t) * (n + 1), s);
    cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n + 1), s);
    cudaMemsetAsync(cur, 0, sizeof(int32_t) * (n + 1), s);
    k_rows<<<k, 256, 0, s>>>(k, d_bptr, out->blk_row);
    k_locate<<<grid_for(n), 256, 0, s>>>(n, d_verts, row_of, d_status);
    k_count<<<grid_for(nside), 256, 0, s>>>(nside, arity, d_tri, n, row_of, out->blk_row, cnt,
                                            d_status);
    rc = exclusive_scan(cnt, off, n, d_status, s, &total);
    if (rc != BSP_OK) break;
    int st = 0;
    cudaMemcpy(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (st & (ST_BAD_INDEX | ST_DUP_VERTEX | ST_DEGREE)) {
      fail(BSP_ERR_INVALID_ARG, (st & ST_BAD_INDEX) ? "vertex index out of range"
                                : (st & ST_DUP_VERTEX) ? "a vertex appears in more than one block slot"
                                : "too many neighbour entries");
      break;
    }
    if (cudaMalloc(&nbr, sizeof(int32_t) * (total > 0 ? total : 1)) != cudaSuccess) {
      fail(BSP_ERR_OOM, "device allocation failed during assembly");
      break;
    }
    k_fill<<<grid_for(nside), 256, 0, s>>>(nside, arity, d_tri, n, row_of, out->blk_row, d_bptr,
                                           off, cur, nbr, d_status);
    k_sort_unique<<<grid_for(n), 256, 0, s>>>(n, off, nbr, d_bptr, out->blk_row, ucnt, up);
    rc = exclusive_scan(ucnt, out->rowptr, n, d_status, s, &nnz);
    if (rc != BSP_OK) break;
    rc = exclusive_scan(up, out->eoff, n, d_status, s, &nedge);
    if (rc != BSP_OK) break;
    if (cudaMalloc(&out->col, sizeof(uint16_t) * (nnz > 0 ? nnz : 1)) != cudaSuccess) {
      fail(BSP_ERR_OOM, "device allocation failed during assembly");
      break;
    }
    k_compact<<<grid_for(n), 256, 0, s>>>(n, off, nbr, out->rowptr, out->col);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      fail(BSP_ERR_CUDA, "CUDA error during assembly");
      break;
    }
    out->nnz = nnz;
    out->intra_edges = nedge;
  } while (0);
  cudaFree(row_of);
  cudaFree(cnt);
  cudaFree(off);
  cudaFree(cur);
  cudaFree(nbr);
  cudaFree(ucnt);
  cudaFree(up);
  return rc;
}

template <typename T>
void launch_weights(int64_t n, const int32_t* bptr, const int32_t* blk_row, const int32_t* verts,
                    const int32_t* rowptr, const uint16_t* col, const double* xyz, int mode,
                    int literal, T* wt, T* diag, cudaStream_t s) {
  k_weights<T><<<grid_for(n), 256, 0, s>>>(n, bptr, blk_row, verts, rowptr, col, xyz, mode,
                                           literal, wt, diag);
}

template <typename T>
void launch_set_weights(int64_t n, const int32_t* bptr, const int32_t* blk_row,
                        const int32_t* rowptr, const uint16_t* col, const int32_t* eoff,
                        const T* w_edges, int literal, T* wt, T* diag, cudaStream_t s) {
  k_set_weights<T><<<grid_for(n), 256, 0, s>>>(n, bptr, blk_row, rowptr, col, eoff, w_edges,
                                               literal, wt, diag);
}

void launch_edges_out(int64_t n, const int32_t* bptr, const int32_t* blk_row, const int32_t* verts,
                      const int32_t* rowptr, const uint16_t* col, const int32_t* eoff,
                      int32_t* edges, cudaStream_t s) {
  k_edges_out<<<grid_for(n), 256, 0, s>>>(n, bptr, blk_row, verts, rowptr, col, eoff, edges);
}

template void launch_weights<float>(int64_t, const int32_t*, const int32_t*, const int32_t*,
                                    const int32_t*, const uint16_t*, const double*, int, int,
                                    float*, float*, cudaStream_t);
template void launch_weights<double>(int64_t, const int32_t*, const int32_t*, const int32_t*,
                                     const int32_t*, const uint16_t*, const double*, int, int,
                                     double*, double*, cudaStream_t);
template void launch_set_weights<float>(int64_t, const int32_t*, const int32_t*, const int32_t*,
                                        const uint16_t*, const int32_t*, const float*, int,
                                        float*, float*, cudaStream_t);
template void launch_set_weights<double>(int64_t, const int32_t*, const int32_t*, const int32_t*,
                                         const uint16_t*, const int32_t*, const double*, int,
                                         double*, double*, cudaStream_t);

}  // namespace bsp
