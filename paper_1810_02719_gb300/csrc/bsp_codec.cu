// Compression codec of the spectral coefficients (Sec. 7.1) and its quality
// metric.
//
//  * Quantisation: the coefficients E[b] of every block are coded with q bits
//    per value by a uniform scalar quantiser (Sec. 8, the bits-per-vertex
//    formula with q_c = 12).  The paper does not state the quantiser's range;
//    here every (block, column) pair has its own [lo, hi] = [min, max] over
//    the block's c_b coefficients, sent as side information:
//        s = (2^q - 1) / (hi - lo),  code = clamp(rint((e - lo) s), 0, 2^q - 1)
//        e~ = lo + code (hi - lo) / (2^q - 1)
//    evaluated in the coefficients' own precision with every operation
//    rounded on its own (no contraction into FMA), so that the codes are a
//    deterministic function of the inputs.
//  * NMSVE (Sec. 8): (||v - v~|| + ||GL(v) - GL(v~)||) / (2 n) over the 3 n
//    coordinates, with the geometric Laplacian
//        GL(v_i) = v_i - sum_j v_j / d_ij / sum_j 1 / d_ij
//    over the mesh neighbours j of i (all faces, across block borders) and
//    d_ij the edge length in the geometry GL is applied to.  Accumulated in
//    FP64.
#include "bsp_internal.cuh"

namespace bsp {
namespace {

constexpr int kQT = 128;   // quantiser: threads per CTA, one coefficient column each
constexpr int kNT = 256;   // NMSVE: threads per CTA

__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float rint_even(float a) { return rintf(a); }
__device__ __forceinline__ double rint_even(double a) { return rint(a); }
__device__ __forceinline__ bool finite_pos(float a) { return a > 0.f && a <= 3.402823466e38f; }
__device__ __forceinline__ bool finite_pos(double a) { return a > 0.0 && a <= 1.7976931348623157e308; }

// grid (k, ceil(cols / kQT)): CTA (b, y) codes columns y kQT .. of block b.
// Reads each column of the block twice (range, then codes; the second pass
// hits L2).
template <typename T>
__global__ void __launch_bounds__(kQT) k_quantize(const int32_t* __restrict__ ceoff,
                                                  const T* __restrict__ E, int cols, int bits,
                                                  uint16_t* __restrict__ codes,
                                                  T* __restrict__ range) {
  const int b = blockIdx.x;
  const int j = blockIdx.y * kQT + threadIdx.x;
  if (j >= cols) return;
  const int r0 = ceoff[b], r1 = ceoff[b + 1];
  T lo = T(0), hi = T(0);
  if (r1 > r0) lo = hi = E[(size_t)r0 * cols + j];
  for (int r = r0 + 1; r < r1; ++r) {
    const T e = E[(size_t)r * cols + j];
    lo = e < lo ? e : lo;
    hi = e > hi ? e : hi;
  }
  range[((size_t)b * cols + j) * 2] = lo;
  range[((size_t)b * cols + j) * 2 + 1] = hi;
  const T qmax = T((1u << bits) - 1u);
  T s = T(0);
  if (hi > lo) {
    s = div_rn(qmax, sub_rn(hi, lo));
    if (!finite_pos(s)) s = T(0);   // range too narrow to scale: every code 0
  }
  for (int r = r0; r < r1; ++r) {
    T q = rint_even(mul_rn(sub_rn(E[(size_t)r * cols + j], lo), s));
    q = q < T(0) ? T(0) : (q > qmax ? qmax : q);
    codes[(size_t)r * cols + j] = (uint16_t)q;
  }
}

template <typename T>
__global__ void __launch_bounds__(kQT) k_dequantize(const int32_t* __restrict__ ceoff,
                                                    const uint16_t* __restrict__ codes,
                                                    const T* __restrict__ range, int cols,
                                                    int bits, T* __restrict__ E) {
  const int b = blockIdx.x;
  const int j = blockIdx.y * kQT + threadIdx.x;
  if (j >= cols) return;
  const int r0 = ceoff[b], r1 = ceoff[b + 1];
  const T lo = range[((size_t)b * cols + j) * 2];
  const T hi = range[((size_t)b * cols + j) * 2 + 1];
  const T qmax = T((1u << bits) - 1u);
  const T step = div_rn(sub_rn(hi, lo), qmax);
  for (int r = r0; r < r1; ++r)
    E[(size_t)r * cols + j] = add_rn(lo, mul_rn(T(codes[(size_t)r * cols + j]), step));
}

// Half-edge counts of every vertex over the face sides (a side shared by two
// faces is counted twice; duplicates are skipped when the lists are read).
__global__ void k_nm_count(int64_t m, const int32_t* __restrict__ faces, int64_t n,
                           int32_t* cnt, int* status) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = e / 3;
    const int s = (int)(e - 3 * f);
    const int32_t u = faces[3 * f + s], v = faces[3 * f + (s + 1) % 3];
    if (u < 0 || u >= n || v < 0 || v >= n) {
      atomicOr(status, ST_BAD_INDEX);
      continue;
    }
    if (u == v) continue;
    atomicAdd(&cnt[u], 1);
    atomicAdd(&cnt[v], 1);
  }
}

__global__ void k_nm_fill(int64_t m, const int32_t* __restrict__ faces, int64_t n,
                          const int32_t* __restrict__ off, int32_t* cur, int32_t* nbr) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = e / 3;
    const int s = (int)(e - 3 * f);
    const int32_t u = faces[3 * f + s], v = faces[3 * f + (s + 1) % 3];
    if (u < 0 || u >= n || v < 0 || v >= n || u == v) continue;
    nbr[off[u] + atomicAdd(&cur[u], 1)] = v;
    nbr[off[v] + atomicAdd(&cur[v], 1)] = u;
  }
}

// GL(X)_i for one vertex: X_i minus the inverse-edge-length weighted mean of
// its distinct neighbours (neighbours at distance 0 carry no weight; with no
// weighted neighbour GL is X_i itself).
template <typename T>
__device__ __forceinline__ void geometric_laplacian(const T* __restrict__ X, int64_t i,
                                    const int32_t* __restrict__ nbr, int e0, int e1,
                                    double gl[3]) {
  const double xi[3] = {(double)X[3 * i], (double)X[3 * i + 1], (double)X[3 * i + 2]};
  double sw = 0.0, sx[3] = {0.0, 0.0, 0.0};
  for (int e = e0; e < e1; ++e) {
    const int32_t j = nbr[e];
    bool seen = false;
    for (int p = e0; p < e; ++p) seen |= nbr[p] == j;
    if (seen) continue;
    const double xj[3] = {(double)X[3 * (int64_t)j], (double)X[3 * (int64_t)j + 1],
                          (double)X[3 * (int64_t)j + 2]};
    const double d0 = xi[0] - xj[0], d1 = xi[1] - xj[1], d2 = xi[2] - xj[2];
    const double d = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    if (!(d > 0.0)) continue;
    const double w = 1.0 / d;
    sw += w;
    sx[0] += w * xj[0];
    sx[1] += w * xj[1];
    sx[2] += w * xj[2];
  }
  for (int a = 0; a < 3; ++a) gl[a] = sw > 0.0 ? xi[a] - sx[a] / sw : xi[a];
}

// acc[0] += sum_i ||X_i - Xr_i||^2, acc[1] += sum_i ||GL(X)_i - GL(Xr)_i||^2
template <typename T>
__global__ void __launch_bounds__(kNT) k_nm_err(int64_t n, const int32_t* __restrict__ off,
                                                const int32_t* __restrict__ nbr,
                                                const T* __restrict__ X,
                                                const T* __restrict__ Xr, double* acc) {
  double a = 0.0, g = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double gx[3], gr[3];
    geometric_laplacian(X, i, nbr, off[i], off[i + 1], gx);
    geometric_laplacian(Xr, i, nbr, off[i], off[i + 1], gr);
    for (int c = 0; c < 3; ++c) {
      const double d = (double)X[3 * i + c] - (double)Xr[3 * i + c];
      a += d * d;
      g += (gx[c] - gr[c]) * (gx[c] - gr[c]);
    }
  }
  __shared__ double sa[kNT / 32], sg[kNT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    g += __shfl_xor_sync(0xffffffffu, g, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sa[threadIdx.x >> 5] = a;
    sg[threadIdx.x >> 5] = g;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kNT / 32; ++w) {
      a += sa[w];
      g += sg[w];
    }
    atomicAdd(&acc[0], a);
    atomicAdd(&acc[1], g);
  }
}

unsigned grid_cap(int64_t items, int threads) {
  int64_t g = (items + threads - 1) / threads;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

template <typename T>
int launch_quantize(const int32_t* ceoff, int k, const T* E, int cols, int bits, uint16_t* codes,
                    T* range, cudaStream_t s) {
  if (k < 1 || cols < 1) return BSP_OK;
  dim3 grid(k, (cols + kQT - 1) / kQT);
  k_quantize<T><<<grid, kQT, 0, s>>>(ceoff, E, cols, bits, codes, range);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

template <typename T>
int launch_dequantize(const int32_t* ceoff, int k, const uint16_t* codes, const T* range, int cols,
                      int bits, T* E, cudaStream_t s) {
  if (k < 1 || cols < 1) return BSP_OK;
  dim3 grid(k, (cols + kQT - 1) / kQT);
  k_dequantize<T><<<grid, kQT, 0, s>>>(ceoff, codes, range, cols, bits, E);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

void launch_nm_count(int64_t m, const int32_t* faces, int64_t n, int32_t* cnt, int* status,
                     cudaStream_t s) {
  k_nm_count<<<grid_cap(3 * m, 256), 256, 0, s>>>(m, faces, n, cnt, status);
}

void launch_nm_fill(int64_t m, const int32_t* faces, int64_t n, const int32_t* off, int32_t* cur,
                    int32_t* nbr, cudaStream_t s) {
  k_nm_fill<<<grid_cap(3 * m, 256), 256, 0, s>>>(m, faces, n, off, cur, nbr);
}

template <typename T>
int launch_nm_err(int64_t n, const int32_t* off, const int32_t* nbr, const T* X, const T* Xr,
                  double* acc, cudaStream_t s) {
  k_nm_err<T><<<grid_cap(n, kNT), kNT, 0, s>>>(n, off, nbr, X, Xr, acc);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

template int launch_quantize<float>(const int32_t*, int, const float*, int, int, uint16_t*,
                                    float*, cudaStream_t);
template int launch_quantize<double>(const int32_t*, int, const double*, int, int, uint16_t*,
                                     double*, cudaStream_t);
template int launch_dequantize<float>(const int32_t*, int, const uint16_t*, const float*, int, int,
                                      float*, cudaStream_t);
template int launch_dequantize<double>(const int32_t*, int, const uint16_t*, const double*, int,
                                       int, double*, cudaStream_t);
template int launch_nm_err<float>(int64_t, const int32_t*, const int32_t*, const float*,
                                  const float*, double*, cudaStream_t);
template int launch_nm_err<double>(int64_t, const int32_t*, const int32_t*, const double*,
                                   const double*, double*, cudaStream_t);

}  // namespace bsp
