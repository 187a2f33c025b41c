// Fine denoising after the coarse spectral step (Sec. 7.2) and the mean
// face-normal angle of the evaluation (Sec. 8).
//
//  * Face geometry of a mesh (Sec. 7.2, face normal equation): unit normal
//    n_i = (v2 - v1) x (v3 - v1) / ||.||, centroid m_i, area A_i = ||.|| / 2;
//    a degenerate face has normal 0 and area 0.
//  * Bilateral normal filter (Sec. 7.2, Eqs. BF, Wm, Wn):
//        n_i <- normalise( sum_{j in N(f_i)} A_j K_s(m_i, m_j) K_r(n_i, n_j) n_j )
//    with Gaussian K_s, K_r of widths sigma_s, sigma_r and N(f_i) the faces
//    that share a vertex with f_i (f_i included); repeated passes filter the
//    previous pass's normals with the input mesh's centroids and areas.
//  * Vertex fitting (Sec. 7.2, Eqs. iter1, iter2):
//        v <- v + (1 / |F_v|) sum_{z in F_v} n_z [n_z . (m_z - v)]
//    with face centroids m_z at the current positions, every vertex moving
//    from the previous iterate (two position buffers).
//  * theta (Sec. 8): mean over faces of atan2(||n x n'||, n . n') between the
//    normals of two meshes with the same faces, in degrees, faces degenerate
//    in either mesh left out.
// Face rings come from a vertex -> face table (counts, scan, fill, then each
// list sorted so that every run sums in the same order).
#include "bsp_internal.cuh"

namespace bsp {
namespace {

constexpr int kDT = 256;

unsigned grid_for(int64_t items) {
  int64_t g = (items + kDT - 1) / kDT;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

__device__ __forceinline__ float exp_t(float x) { return expf(x); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }

// Faces incident to each vertex, each distinct vertex of a face counted once.
__global__ void k_vf_count(int64_t m, const int32_t* __restrict__ faces, int64_t n, int32_t* cnt,
                           int* status) {
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < m;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = faces[3 * f], b = faces[3 * f + 1], c = faces[3 * f + 2];
    if (a < 0 || a >= n || b < 0 || b >= n || c < 0 || c >= n) {
      atomicOr(status, ST_BAD_INDEX);
      continue;
    }
    atomicAdd(&cnt[a], 1);
    if (b != a) atomicAdd(&cnt[b], 1);
    if (c != a && c != b) atomicAdd(&cnt[c], 1);
  }
}

__global__ void k_vf_fill(int64_t m, const int32_t* __restrict__ faces,
                          const int32_t* __restrict__ off, int32_t* cur, int32_t* vf) {
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < m;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = faces[3 * f], b = faces[3 * f + 1], c = faces[3 * f + 2];
    vf[off[a] + atomicAdd(&cur[a], 1)] = (int32_t)f;
    if (b != a) vf[off[b] + atomicAdd(&cur[b], 1)] = (int32_t)f;
    if (c != a && c != b) vf[off[c] + atomicAdd(&cur[c], 1)] = (int32_t)f;
  }
}

// Insertion sort of every vertex's face list (a handful of entries).
__global__ void k_vf_sort(int64_t n, const int32_t* __restrict__ off, int32_t* vf) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int32_t* a = vf + off[v];
    const int len = off[v + 1] - off[v];
    for (int i = 1; i < len; ++i) {
      const int32_t x = a[i];
      int j = i - 1;
      while (j >= 0 && a[j] > x) {
        a[j + 1] = a[j];
        --j;
      }
      a[j + 1] = x;
    }
  }
}

template <typename T>
__global__ void k_face_geom(int64_t m, const int32_t* __restrict__ faces, const T* __restrict__ X,
                            T* __restrict__ nrm, T* __restrict__ cen, T* __restrict__ area) {
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < m;
       f += (int64_t)gridDim.x * blockDim.x) {
    const T* p = X + 3 * (int64_t)faces[3 * f];
    const T* q = X + 3 * (int64_t)faces[3 * f + 1];
    const T* r = X + 3 * (int64_t)faces[3 * f + 2];
    const T e1[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
    const T e2[3] = {r[0] - p[0], r[1] - p[1], r[2] - p[2]};
    const T cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                     e1[0] * e2[1] - e1[1] * e2[0]};
    const T len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    for (int k = 0; k < 3; ++k) {
      nrm[3 * f + k] = len > T(0) ? cr[k] / len : T(0);
      cen[3 * f + k] = (p[k] + q[k] + r[k]) / T(3);
    }
    area[f] = len / T(2);
  }
}

// One pass of the bilateral filter: nin -> nout.
template <typename T>
__global__ void __launch_bounds__(kDT) k_normal_filter(int64_t m, const int32_t* __restrict__ faces,
                                                      const int32_t* __restrict__ off,
                                                      const int32_t* __restrict__ vf,
                                                      const T* __restrict__ cen,
                                                      const T* __restrict__ area,
                                                      const T* __restrict__ nin,
                                                      T* __restrict__ nout, T inv2ss, T inv2sr) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t vi[3] = {faces[3 * i], faces[3 * i + 1], faces[3 * i + 2]};
    const T ci[3] = {cen[3 * i], cen[3 * i + 1], cen[3 * i + 2]};
    const T ni[3] = {nin[3 * i], nin[3 * i + 1], nin[3 * i + 2]};
    T acc[3] = {T(0), T(0), T(0)};
    for (int k = 0; k < 3; ++k) {
      if ((k >= 1 && vi[k] == vi[0]) || (k == 2 && vi[2] == vi[1])) continue;
      for (int e = off[vi[k]]; e < off[vi[k] + 1]; ++e) {
        const int64_t j = vf[e];
        // a face met through an earlier corner of f_i was counted there
        bool seen = false;
        for (int k2 = 0; k2 < k; ++k2)
          seen |= faces[3 * j] == vi[k2] || faces[3 * j + 1] == vi[k2] || faces[3 * j + 2] == vi[k2];
        if (seen) continue;
        const T dc0 = ci[0] - cen[3 * j], dc1 = ci[1] - cen[3 * j + 1], dc2 = ci[2] - cen[3 * j + 2];
        const T nj[3] = {nin[3 * j], nin[3 * j + 1], nin[3 * j + 2]};
        const T dn0 = ni[0] - nj[0], dn1 = ni[1] - nj[1], dn2 = ni[2] - nj[2];
        const T w = area[j] * exp_t(-(dc0 * dc0 + dc1 * dc1 + dc2 * dc2) * inv2ss -
                                    (dn0 * dn0 + dn1 * dn1 + dn2 * dn2) * inv2sr);
        acc[0] += w * nj[0];
        acc[1] += w * nj[1];
        acc[2] += w * nj[2];
      }
    }
    const T len = sqrt(acc[0] * acc[0] + acc[1] * acc[1] + acc[2] * acc[2]);
    for (int k = 0; k < 3; ++k) nout[3 * i + k] = len > T(0) ? acc[k] / len : ni[k];
  }
}

// One vertex-fitting iteration: Xin -> Xout with the filtered normals.
template <typename T>
__global__ void __launch_bounds__(kDT) k_vertex_fit(int64_t n, const int32_t* __restrict__ faces,
                                                   const int32_t* __restrict__ off,
                                                   const int32_t* __restrict__ vf,
                                                   const T* __restrict__ nrm,
                                                   const T* __restrict__ Xin, T* __restrict__ Xout) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const T p[3] = {Xin[3 * v], Xin[3 * v + 1], Xin[3 * v + 2]};
    const int e0 = off[v], e1 = off[v + 1];
    T acc[3] = {T(0), T(0), T(0)};
    for (int e = e0; e < e1; ++e) {
      const int64_t z = vf[e];
      const T* a = Xin + 3 * (int64_t)faces[3 * z];
      const T* b = Xin + 3 * (int64_t)faces[3 * z + 1];
      const T* c = Xin + 3 * (int64_t)faces[3 * z + 2];
      const T nz[3] = {nrm[3 * z], nrm[3 * z + 1], nrm[3 * z + 2]};
      T d = T(0);
      for (int k = 0; k < 3; ++k) d += nz[k] * ((a[k] + b[k] + c[k]) / T(3) - p[k]);
      for (int k = 0; k < 3; ++k) acc[k] += nz[k] * d;
    }
    for (int k = 0; k < 3; ++k) Xout[3 * v + k] = e1 > e0 ? p[k] + acc[k] / T(e1 - e0) : p[k];
  }
}

__device__ __forceinline__ bool unit_normal(const double* p, const double* q, const double* r,
                                            double nrm[3]) {
  const double e1[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
  const double e2[3] = {r[0] - p[0], r[1] - p[1], r[2] - p[2]};
  const double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                        e1[0] * e2[1] - e1[1] * e2[0]};
  const double len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
  if (!(len > 0.0)) return false;
  for (int k = 0; k < 3; ++k) nrm[k] = cr[k] / len;
  return true;
}

// acc[0] += sum of angles (radians) over faces normal in both meshes; cnt += their count
template <typename T>
__global__ void __launch_bounds__(kDT) k_normal_angle(int64_t m, const int32_t* __restrict__ faces,
                                                     const T* __restrict__ X,
                                                     const T* __restrict__ Xr, double* acc,
                                                     unsigned long long* cnt) {
  double s = 0.0;
  unsigned long long c = 0;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < m;
       f += (int64_t)gridDim.x * blockDim.x) {
    double P[3][3], Q[3][3];
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) {
        P[k][d] = (double)X[3 * (int64_t)faces[3 * f + k] + d];
        Q[k][d] = (double)Xr[3 * (int64_t)faces[3 * f + k] + d];
      }
    double a[3], b[3];
    if (!unit_normal(P[0], P[1], P[2], a) || !unit_normal(Q[0], Q[1], Q[2], b)) continue;
    // products rounded on their own: identical normals give a cross product
    // of exactly 0 (an FMA would leave the rounding residue of one product)
    const double cx = __dsub_rn(__dmul_rn(a[1], b[2]), __dmul_rn(a[2], b[1]));
    const double cy = __dsub_rn(__dmul_rn(a[2], b[0]), __dmul_rn(a[0], b[2]));
    const double cz = __dsub_rn(__dmul_rn(a[0], b[1]), __dmul_rn(a[1], b[0]));
    s += atan2(sqrt(cx * cx + cy * cy + cz * cz), a[0] * b[0] + a[1] * b[1] + a[2] * b[2]);
    ++c;
  }
  __shared__ double ss[kDT / 32];
  __shared__ unsigned long long sc[kDT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    ss[threadIdx.x >> 5] = s;
    sc[threadIdx.x >> 5] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kDT / 32; ++w) {
      s += ss[w];
      c += sc[w];
    }
    atomicAdd(acc, s);
    atomicAdd(cnt, c);
  }
}

}  // namespace

void launch_vf_table(int64_t m, const int32_t* faces, int64_t n, int32_t* cnt, int* status,
                     cudaStream_t s) {
  if (m > 0) k_vf_count<<<grid_for(m), kDT, 0, s>>>(m, faces, n, cnt, status);
}

void launch_vf_fill(int64_t m, const int32_t* faces, int64_t n, const int32_t* off, int32_t* cur,
                    int32_t* vf, cudaStream_t s) {
  if (m > 0) k_vf_fill<<<grid_for(m), kDT, 0, s>>>(m, faces, off, cur, vf);
  k_vf_sort<<<grid_for(n), kDT, 0, s>>>(n, off, vf);
}

template <typename T>
int launch_fine_denoise(int64_t n, int64_t m, const int32_t* faces, const int32_t* off,
                        const int32_t* vf, T* X0, T* X1, T* n0, T* n1, T* cen, T* area,
                        double sigma_s, double sigma_r, int normal_iters, int vertex_iters,
                        T** X_final, T** n_final, cudaStream_t s) {
  *X_final = X0;
  *n_final = n0;
  if (m > 0) {
    k_face_geom<T><<<grid_for(m), kDT, 0, s>>>(m, faces, X0, n0, cen, area);
    const T inv2ss = T(1.0 / (2.0 * sigma_s * sigma_s));
    const T inv2sr = T(1.0 / (2.0 * sigma_r * sigma_r));
    for (int it = 0; it < normal_iters; ++it) {
      k_normal_filter<T><<<grid_for(m), kDT, 0, s>>>(m, faces, off, vf, cen, area, *n_final,
                                                     *n_final == n0 ? n1 : n0, inv2ss, inv2sr);
      *n_final = *n_final == n0 ? n1 : n0;
    }
    for (int it = 0; it < vertex_iters; ++it) {
      k_vertex_fit<T><<<grid_for(n), kDT, 0, s>>>(n, faces, off, vf, *n_final, *X_final,
                                                  *X_final == X0 ? X1 : X0);
      *X_final = *X_final == X0 ? X1 : X0;
    }
  }
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

template <typename T>
int launch_normal_angle(int64_t m, const int32_t* faces, const T* X, const T* Xr, double* acc,
                        unsigned long long* cnt, cudaStream_t s) {
  if (m > 0) k_normal_angle<T><<<grid_for(m), kDT, 0, s>>>(m, faces, X, Xr, acc, cnt);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

template int launch_fine_denoise<float>(int64_t, int64_t, const int32_t*, const int32_t*,
                                        const int32_t*, float*, float*, float*, float*, float*,
                                        float*, double, double, int, int, float**, float**,
                                        cudaStream_t);
template int launch_fine_denoise<double>(int64_t, int64_t, const int32_t*, const int32_t*,
                                         const int32_t*, double*, double*, double*, double*,
                                         double*, double*, double, double, int, int, double**,
                                         double**, cudaStream_t);
template int launch_normal_angle<float>(int64_t, const int32_t*, const float*, const float*,
                                        double*, unsigned long long*, cudaStream_t);
template int launch_normal_angle<double>(int64_t, const int32_t*, const double*, const double*,
                                         double*, unsigned long long*, cudaStream_t);

}  // namespace bsp
