// Device helpers shared by the dense small-matrix kernels (bsp_dense.cu) and
// the fused cluster Onorm (bsp_fused.cu).
#pragma once

#include <cmath>

#include "bsp_internal.cuh"

namespace bsp {
namespace dev {

constexpr int kDT = 256;

__host__ __device__ inline int pad4(int c) { return (c + 3) & ~3; }

template <typename T>
BSP_DEV void stage_panel(const T* __restrict__ A, int ld, int row0, int nr, int c, int cpad,
                         int CH, T* S) {
  for (int t = threadIdx.x; t < CH * cpad; t += blockDim.x) {
    int i = t / cpad, j = t - i * cpad;
    S[t] = (i < nr && j < c) ? A[(size_t)(row0 + i) * ld + j] : T(0);
  }
}

template <typename T>
BSP_DEV void ld4(const T* p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
    double2 a = *reinterpret_cast<const double2*>(p);
    double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
}

template <typename T>
BSP_DEV void st4(T* p, const T* v) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
  }
}

// 1/sqrt(x) for x > 0 without a divide or a square root: an FP32 seed from
// rsqrtf refined by Newton-Raphson steps y <- y (3 - x y^2) / 2 (two steps
// take the ~2^-23 seed error below 2^-52 for FP64).  Used on the Cholesky's
// dependent chain, where the FP64 divide and square root cost most.
template <typename TA>
BSP_DEV TA rsqrt_newton(TA x) {
  if constexpr (sizeof(TA) == 4) {
    return rsqrtf(x);
  } else {
    TA y = (TA)rsqrtf((float)x);
    y = y * (TA(1.5) - TA(0.5) * x * y * y);
    y = y * (TA(1.5) - TA(0.5) * x * y * y);
    return y;
  }
}

// out[i][j] (cpad x cpad, TA) = sum_r S[r][i] * S2[r][j] over the panel's CH rows,
// in 4x4 register tiles; `upper` computes only tiles with ti <= tj.
template <typename T, typename TA>
BSP_DEV void panel_gram(const T* S, const T* S2, int CH, int cpad, bool upper, TA* out) {
  const int nt = cpad / 4;
  for (int u = threadIdx.x; u < nt * nt; u += blockDim.x) {
    const int ti = u / nt, tj = u - ti * nt;
    if (upper && ti > tj) continue;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0;
    for (int r = 0; r < CH; ++r) {
      T a[4], b[4];
      ld4(S + r * cpad + 4 * ti, a);
      ld4(S2 + r * cpad + 4 * tj, b);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) out[(4 * ti + i) * cpad + 4 * tj + j] = (TA)acc[i][j];
  }
}

// Width of the zero-padded R used by chol_inverse, and the size of its A
// workspace in TA elements: the scaled Gram (cpad^2 TA) and, after the
// factorization, R^-1 plus temporaries (1.5 CP^2 T).
__host__ __device__ inline int chol_cp(int c) { return c <= 32 ? 32 : (c <= 64 ? 64 : 128); }
template <typename T, typename TA>
__host__ __device__ inline int chol_a_elems(int cpad, int cp) {
  const int a = cpad * cpad;
  const int b = (int)((3 * (size_t)cp * cp * sizeof(T) / 2 + sizeof(TA) - 1) / sizeof(TA));
  return ((a > b ? a : b) + 1) & ~1;
}

// Cluster-wide barrier with release/acquire ordering; the fence makes global
// writes (partial Grams) visible GPU-wide before the release.
BSP_DEV void cluster_barrier() {
  __threadfence();
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

}  // namespace dev
}  // namespace bsp
