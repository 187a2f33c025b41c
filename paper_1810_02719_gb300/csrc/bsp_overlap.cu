// Overlapped submeshes (Sec. 6.1, Algorithm 3): when parts share vertices,
// every part reconstructs its own copy of each of its vertices, and a vertex's
// final position is the average of its copies, each weighted by the vertex's
// degree inside that part (its number of neighbours in the part's induced
// subgraph).  A vertex whose copies all have degree 0 takes the plain mean of
// its copies; a vertex in no part is 0.
//
// The library keeps every vertex in one block, so overlapped parts are given
// as an expanded mesh with one vertex per (part, vertex) copy; `orig` maps a
// copy to its vertex.  The merge is a gather: the copies of each vertex are
// listed (count, scan, fill, then each list sorted by copy id so the sum has a
// fixed order) and one thread per (vertex, column) forms the weighted mean.
#include "bsp_internal.cuh"

namespace bsp {
namespace {

constexpr int kT = 256;

// Copy weights (degree of the copy in its block = stored off-diagonal entries
// of its CSR row) by copy id, and the number of copies of every vertex.
__global__ void k_ov_count(int64_t rows, const int32_t* __restrict__ verts,
                           const int32_t* __restrict__ rowptr, const int32_t* __restrict__ orig,
                           int64_t n_orig, float* __restrict__ w, int32_t* __restrict__ cnt,
                           int* status) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = verts[r];               // copy id of this row
    w[v] = (float)(rowptr[r + 1] - rowptr[r]);
    const int32_t o = orig[v];
    if (o < 0 || o >= n_orig) {
      atomicOr(status, ST_BAD_INDEX);
      continue;
    }
    atomicAdd(cnt + o, 1);
  }
}

__global__ void k_ov_fill(int64_t rows, const int32_t* __restrict__ orig, int64_t n_orig,
                          const int32_t* __restrict__ off, int32_t* __restrict__ cur,
                          int32_t* __restrict__ list) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < rows;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = orig[v];
    if (o < 0 || o >= n_orig) continue;
    list[off[o] + atomicAdd(cur + o, 1)] = (int32_t)v;
  }
}

// Each vertex's copies in ascending copy id (insertion sort: a vertex has a
// handful of copies).
__global__ void k_ov_sort(int64_t n_orig, const int32_t* __restrict__ off,
                          int32_t* __restrict__ list) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_orig;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int a = off[o], b = off[o + 1];
    for (int i = a + 1; i < b; ++i) {
      const int32_t x = list[i];
      int j = i - 1;
      while (j >= a && list[j] > x) {
        list[j + 1] = list[j];
        --j;
      }
      list[j + 1] = x;
    }
  }
}

template <typename T>
__global__ void k_ov_merge(int64_t n_orig, int cols, const int32_t* __restrict__ off,
                           const int32_t* __restrict__ list, const float* __restrict__ w,
                           const T* __restrict__ Xc, T* __restrict__ Xo) {
  const int64_t total = n_orig * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = e / cols;
    const int j = (int)(e - o * cols);
    const int a = off[o], b = off[o + 1];
    T num = 0, den = 0, plain = 0;
    for (int i = a; i < b; ++i) {
      const int32_t v = list[i];
      const T x = Xc[(size_t)v * cols + j];
      const T wv = (T)w[v];
      num += wv * x;
      den += wv;
      plain += x;
    }
    T out = 0;
    if (den > T(0)) out = num / den;
    else if (b > a) out = plain / (T)(b - a);
    Xo[(size_t)o * cols + j] = out;
  }
}

int grid_for(int64_t work) {
  const int64_t g = (work + kT - 1) / kT;
  return (int)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

}  // namespace

int launch_ov_table(int64_t rows, const int32_t* verts, const int32_t* rowptr, const int32_t* orig,
                    int64_t n_orig, float* w, int32_t* cnt, int* status, cudaStream_t s) {
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)n_orig, s);
  k_ov_count<<<grid_for(rows), kT, 0, s>>>(rows, verts, rowptr, orig, n_orig, w, cnt, status);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

int launch_ov_fill(int64_t rows, const int32_t* orig, int64_t n_orig, const int32_t* off,
                   int32_t* cur, int32_t* list, cudaStream_t s) {
  cudaMemsetAsync(cur, 0, sizeof(int32_t) * (size_t)n_orig, s);
  k_ov_fill<<<grid_for(rows), kT, 0, s>>>(rows, orig, n_orig, off, cur, list);
  k_ov_sort<<<grid_for(n_orig), kT, 0, s>>>(n_orig, off, list);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

template <typename T>
int launch_ov_merge(int64_t n_orig, int cols, const int32_t* off, const int32_t* list,
                    const float* w, const T* Xc, T* Xo, cudaStream_t s) {
  k_ov_merge<T><<<grid_for(n_orig * cols), kT, 0, s>>>(n_orig, cols, off, list, w, Xc, Xo);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

template int launch_ov_merge<float>(int64_t, int, const int32_t*, const int32_t*, const float*,
                                    const float*, float*, cudaStream_t);
template int launch_ov_merge<double>(int64_t, int, const int32_t*, const int32_t*, const float*,
                                     const double*, double*, cudaStream_t);

}  // namespace bsp
