// Graph Fourier transform per block (Sec. 3: v_bar = U^T v, v = U v_bar),
// used as the encoder E[b] = U_c[b]^T v[b] and decoder v~[b] = U_c[b] E[b] of
// block-based compression (Sec. 7.1), the coarse low-pass filter
// v^ = U U^T v (Sec. 7.2), and for all frames of a dynamic mesh at once with
// one basis per block (Sec. 7.3).
//
// SIMT tiled kernels: one CTA per (block, 64 x 64 output tile), 4 x 4 outputs
// per thread, the reduction dimension staged through shared memory in
// 32-row panels.  X rows are gathered through the block's vertex list.
// Narrow right-hand sides (at most 4 columns, e.g. xyz) take kernels that
// stream the basis once instead (one CTA per block; lanes across the basis
// columns, warps across the rows), whose cost is the read of U.
#include <cuda_bf16.h>

#include <type_traits>

#include "bsp_internal.cuh"

namespace bsp {
namespace {

constexpr int kTile = 64;
constexpr int kKc = 32;

// Input element -> compute type T (bf16 widens exactly to float).
template <typename T, typename XT>
BSP_DEV T to_real(XT v) {
  if constexpr (std::is_same<XT, __nv_bfloat16>::value) return (T)__bfloat162float(v);
  else return (T)v;
}

// E_b[cr][cc] = sum_i U_b[i][cr] X[v_i][cc]
template <typename T, typename XT>
__global__ void __launch_bounds__(256) k_project(ProjArgs a, const T* __restrict__ U,
                                                 const XT* __restrict__ X, T* __restrict__ E) {
  __shared__ __align__(16) T Us[kKc][kTile];
  __shared__ __align__(16) T Xs[kKc][kTile];
  const int b = blockIdx.z;
  const int c = a.cb[b];
  const int cr0 = blockIdx.y * kTile, cc0 = blockIdx.x * kTile;
  if (cr0 >= c) return;
  const int r0 = a.bptr[b], nb = a.bptr[b + 1] - r0;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int k0 = 0; k0 < nb; k0 += kKc) {
    for (int t = threadIdx.x; t < kKc * kTile; t += 256) {
      int i = t / kTile, j = t % kTile;
      int row = k0 + i;
      T u = 0, x = 0;
      if (row < nb) {
        if (cr0 + j < c) u = U[(size_t)(r0 + row) * a.ld + cr0 + j];
        if (cc0 + j < a.cols) x = to_real<T, XT>(X[(size_t)a.verts[r0 + row] * a.cols + cc0 + j]);
      }
      Us[i][j] = u;
      Xs[i][j] = x;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kKc; ++kk) {
      T ua[4], xb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) ua[i] = Us[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) xb[j] = Xs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += ua[i] * xb[j];
    }
    __syncthreads();
  }
  const size_t eb = (size_t)a.eoff[b];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int cr = cr0 + ty * 4 + i;
    if (cr >= c) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int cc = cc0 + tx * 4 + j;
      if (cc < a.cols) E[(eb + cr) * a.cols + cc] = acc[i][j];
    }
  }
}

// X[v_i][cc] = sum_l U_b[i][l] E_b[l][cc]
template <typename T>
__global__ void __launch_bounds__(256) k_reconstruct(ProjArgs a, const T* __restrict__ U,
                                                     const T* __restrict__ E, T* __restrict__ X) {
  __shared__ __align__(16) T Us[kTile][kKc + 1];
  __shared__ __align__(16) T Es[kKc][kTile];
  const int b = blockIdx.z;
  const int c = a.cb[b];
  const int r0 = a.bptr[b], nb = a.bptr[b + 1] - r0;
  const int row0 = blockIdx.y * kTile, cc0 = blockIdx.x * kTile;
  if (row0 >= nb) return;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const size_t eb = (size_t)a.eoff[b];
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int l0 = 0; l0 < c; l0 += kKc) {
    for (int t = threadIdx.x; t < kTile * kKc; t += 256) {
      int i = t / kKc, l = t % kKc;
      int row = row0 + i;
      Us[i][l] = (row < nb && l0 + l < c) ? U[(size_t)(r0 + row) * a.ld + l0 + l] : T(0);
    }
    for (int t = threadIdx.x; t < kKc * kTile; t += 256) {
      int l = t / kTile, j = t % kTile;
      Es[l][j] = (l0 + l < c && cc0 + j < a.cols) ? E[(eb + l0 + l) * a.cols + cc0 + j] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int l = 0; l < kKc; ++l) {
      T ua[4], eb4[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) ua[i] = Us[ty * 4 + i][l];
#pragma unroll
      for (int j = 0; j < 4; ++j) eb4[j] = Es[l][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += ua[i] * eb4[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int row = row0 + ty * 4 + i;
    if (row >= nb) continue;
    const size_t orow = (size_t)a.verts[r0 + row] * a.cols;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int cc = cc0 + tx * 4 + j;
      if (cc < a.cols) X[orow + cc] = acc[i][j];
    }
  }
}

constexpr int kNW = 8;     // warps per CTA of the narrow kernels
constexpr int kNCol = 4;   // right-hand-side columns they take
constexpr int kNQ = 4;     // basis columns per lane: c <= 128
constexpr int kNU = 4;     // rows in flight per warp

// E_b[j][cc] = sum_i U_b[i][j] X[v_i][cc] for cols <= 4: lane l of warp w
// accumulates columns j = l + 32 q over rows i = w + 8 m (4 rows per
// iteration in flight); the 8 warps' partial sums are added in warp order.
template <typename T, typename XT>
__global__ void __launch_bounds__(32 * kNW) k_project_narrow(ProjArgs a, const T* __restrict__ U,
                                                              const XT* __restrict__ X,
                                                              T* __restrict__ E) {
  __shared__ T red[kNW][32 * kNQ * kNCol];
  const int b = blockIdx.x;
  const int c = a.cb[b], cols = a.cols;
  const int r0 = a.bptr[b], nb = a.bptr[b + 1] - r0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T acc[kNQ][kNCol];
#pragma unroll
  for (int q = 0; q < kNQ; ++q)
#pragma unroll
    for (int cc = 0; cc < kNCol; ++cc) acc[q][cc] = 0;
  for (int i0 = w; i0 < nb; i0 += kNW * kNU) {
    T u[kNU][kNQ], x[kNU][kNCol];
#pragma unroll
    for (int m = 0; m < kNU; ++m) {
      const int i = i0 + kNW * m;
      const bool ok = i < nb;
      const size_t xr = ok ? (size_t)__ldg(a.verts + r0 + i) * cols : 0;
#pragma unroll
      for (int cc = 0; cc < kNCol; ++cc)
        x[m][cc] = (ok && cc < cols) ? to_real<T, XT>(X[xr + cc]) : T(0);
#pragma unroll
      for (int q = 0; q < kNQ; ++q) {
        const int j = lane + 32 * q;
        u[m][q] = (ok && j < c) ? __ldg(U + (size_t)(r0 + i) * a.ld + j) : T(0);
      }
    }
#pragma unroll
    for (int m = 0; m < kNU; ++m)
#pragma unroll
      for (int q = 0; q < kNQ; ++q)
#pragma unroll
        for (int cc = 0; cc < kNCol; ++cc) acc[q][cc] += u[m][q] * x[m][cc];
  }
#pragma unroll
  for (int q = 0; q < kNQ; ++q)
#pragma unroll
    for (int cc = 0; cc < kNCol; ++cc) red[w][(lane + 32 * q) * kNCol + cc] = acc[q][cc];
  __syncthreads();
  const size_t eb = (size_t)a.eoff[b];
  for (int t = threadIdx.x; t < c * cols; t += 32 * kNW) {
    const int j = t / cols, cc = t - j * cols;
    T sum = 0;
#pragma unroll
    for (int ww = 0; ww < kNW; ++ww) sum += red[ww][j * kNCol + cc];
    E[(eb + j) * cols + cc] = sum;
  }
}

// X[v_i][cc] = sum_j U_b[i][j] E_b[j][cc] for cols <= 4: E_b in shared
// memory, warp w takes rows i = w + 8 m (4 in flight), lane l the columns
// j = l + 32 q; the row's sums are finished with a butterfly over the warp.
template <typename T>
__global__ void __launch_bounds__(32 * kNW) k_reconstruct_narrow(ProjArgs a,
                                                                  const T* __restrict__ U,
                                                                  const T* __restrict__ E,
                                                                  T* __restrict__ X) {
  __shared__ T Es[32 * kNQ][kNCol + 1];   // padded: lane-strided reads hit distinct banks
  const int b = blockIdx.x;
  const int c = a.cb[b], cols = a.cols;
  const int r0 = a.bptr[b], nb = a.bptr[b + 1] - r0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t eb = (size_t)a.eoff[b];
  for (int t = threadIdx.x; t < 32 * kNQ * kNCol; t += 32 * kNW) {
    const int j = t / kNCol, cc = t - j * kNCol;
    Es[j][cc] = (j < c && cc < cols) ? E[(eb + j) * cols + cc] : T(0);
  }
  __syncthreads();
  for (int i0 = w; i0 < nb; i0 += kNW * kNU) {
    T u[kNU][kNQ];
#pragma unroll
    for (int m = 0; m < kNU; ++m) {
      const int i = i0 + kNW * m;
#pragma unroll
      for (int q = 0; q < kNQ; ++q) {
        const int j = lane + 32 * q;
        u[m][q] = (i < nb && j < c) ? __ldg(U + (size_t)(r0 + i) * a.ld + j) : T(0);
      }
    }
#pragma unroll
    for (int m = 0; m < kNU; ++m) {
      T p[kNCol];
#pragma unroll
      for (int cc = 0; cc < kNCol; ++cc) {
        T v = 0;
#pragma unroll
        for (int q = 0; q < kNQ; ++q) v += u[m][q] * Es[lane + 32 * q][cc];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        p[cc] = v;
      }
      const int i = i0 + kNW * m;
      if (i < nb && lane < cols) {
        T out = p[0];
#pragma unroll
        for (int cc = 1; cc < kNCol; ++cc)
          if (lane == cc) out = p[cc];
        X[(size_t)a.verts[r0 + i] * cols + lane] = out;
      }
    }
  }
}

}  // namespace

template <typename T>
int launch_project(const ProjArgs& a, const T* U, const void* X, int x_dtype, T* E,
                   cudaStream_t s) {
  dim3 grid((a.cols + kTile - 1) / kTile, (a.cmax + kTile - 1) / kTile, a.k);
  if (a.cols <= kNCol && a.cmax <= 32 * kNQ &&
      (x_dtype == BSP_DT_F32 || x_dtype == BSP_DT_F64)) {
    prof_begin(KC_PROJECT, s);
    if (x_dtype == BSP_DT_F32)
      k_project_narrow<T, float><<<a.k, 32 * kNW, 0, s>>>(a, U, (const float*)X, E);
    else
      k_project_narrow<T, double><<<a.k, 32 * kNW, 0, s>>>(a, U, (const double*)X, E);
    prof_end(KC_PROJECT, s);
    return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
  }
  prof_begin(KC_PROJECT, s);
  if (x_dtype == BSP_DT_BF16) {
    if (sizeof(T) != 4) return BSP_ERR_INVALID_ARG;
    k_project<T, __nv_bfloat16><<<grid, 256, 0, s>>>(a, U, (const __nv_bfloat16*)X, E);
  } else if (x_dtype == BSP_DT_F32) {
    k_project<T, float><<<grid, 256, 0, s>>>(a, U, (const float*)X, E);
  } else if (x_dtype == BSP_DT_F64) {
    k_project<T, double><<<grid, 256, 0, s>>>(a, U, (const double*)X, E);
  } else {
    prof_end(KC_PROJECT, s);
    return BSP_ERR_INVALID_ARG;
  }
  prof_end(KC_PROJECT, s);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

template <typename T>
int launch_reconstruct(const ProjArgs& a, const T* U, const T* E, T* X, cudaStream_t s) {
  dim3 grid((a.cols + kTile - 1) / kTile, (a.max_nb + kTile - 1) / kTile, a.k);
  prof_begin(KC_RECON, s);
  if (a.cols <= kNCol && a.cmax <= 32 * kNQ)
    k_reconstruct_narrow<T><<<a.k, 32 * kNW, 0, s>>>(a, U, E, X);
  else
    k_reconstruct<T><<<grid, 256, 0, s>>>(a, U, E, X);
  prof_end(KC_RECON, s);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

template int launch_project<float>(const ProjArgs&, const float*, const void*, int, float*,
                                   cudaStream_t);
template int launch_project<double>(const ProjArgs&, const double*, const void*, int, double*,
                                    cudaStream_t);
template int launch_reconstruct<float>(const ProjArgs&, const float*, const float*, float*,
                                       cudaStream_t);
template int launch_reconstruct<double>(const ProjArgs&, const double*, const double*, double*,
                                        cudaStream_t);

}  // namespace bsp
