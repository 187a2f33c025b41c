// Onorm and Rayleigh-Ritz for batches of blocks (Sec. 4, Onorm equations).
//
// Onorm is computed as CholeskyQR2: G = Y^T Y, G = R^T R, Q = Y R^-1, twice.
// It produces the same Q as the paper's Householder QR in exact arithmetic
// (diag(R) > 0 fixes the signs; both keep the nested column spans).  Data is
// processed in panels of CH rows staged in shared memory:
//   k_gram        per-panel partial Gram matrices (FP32 products, TA = the
//                 accumulation type; one conversion per panel)
//   k_reduce      sums the panels of each block in a fixed order (deterministic)
//   k_chol        one CTA per block: Jacobi-scaled Cholesky G = R^T R in TA,
//                 then R^-1 by back substitution; flags breakdown
//   k_panel_mul   Q panel = Y panel x M (M = R^-1 upper triangular, or a full
//                 c x c rotation), optionally fused with the next Gram panel
// Rayleigh-Ritz (not in the paper): H = V^T L V (k_rr), c x c symmetric
// eigensolve by cyclic Jacobi (k_jacobi), V <- V Q_H (k_panel_mul).
#include <cfloat>
#include <cmath>

#include "bsp_internal.cuh"

namespace bsp {
namespace {

constexpr int kDT = 256;
constexpr int kJacobiSweeps = 20;

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

template <typename T, typename TA>
__global__ void __launch_bounds__(kDT) k_gram(DenseArgs a, const T* __restrict__ Y, int CH,
                                              int maxch, TA* __restrict__ Gp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);
  const int b = a.batch[blockIdx.y];
  const int c = a.cb[b];
  const int cpad = pad4(a.cmax);
  const int r0 = a.bptr[b], nb = a.bptr[b + 1] - r0;
  const int row0 = blockIdx.x * CH;
  if (row0 >= nb) return;
  stage_panel(Y, a.ld, r0 + row0, min(CH, nb - row0), c, cpad, CH, S);
  __syncthreads();
  TA* out = Gp + ((size_t)blockIdx.y * maxch + blockIdx.x) * cpad * cpad;
  panel_gram<T, TA>(S, S, CH, cpad, true, out);
}

// G[slot] = sum over the block's panels (fixed order), entries (i, j) < cpad.
template <typename TA>
__global__ void k_reduce(DenseArgs a, int CH, int maxch, bool upper, const TA* __restrict__ Gp,
                         TA* __restrict__ G) {
  const int b = a.batch[blockIdx.y];
  const int cpad = pad4(a.cmax);
  const int nb = a.bptr[b + 1] - a.bptr[b];
  const int nch = (nb + CH - 1) / CH;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= cpad * cpad) return;
  const int i = e / cpad, j = e - i * cpad;
  if (upper && i > j) return;
  const TA* src = Gp + (size_t)blockIdx.y * maxch * cpad * cpad + e;
  TA s = 0;
  for (int ch = 0; ch < nch; ++ch) s += src[(size_t)ch * cpad * cpad];
  G[(size_t)blockIdx.y * cpad * cpad + e] = s;
}

// Cholesky G = R^T R (upper R) after Jacobi scaling, then M = R^-1 (upper) in T.
// smem: A [cpad x cpad] TA, X [cpad x cpad] T, d [cpad] TA.
template <typename T, typename TA>
__global__ void __launch_bounds__(kDT) k_chol(DenseArgs a, const TA* __restrict__ G,
                                              T* __restrict__ Mout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = a.batch[blockIdx.x];
  const int c = a.cb[b];
  const int cpad = pad4(a.cmax);
  TA* A = reinterpret_cast<TA*>(smem_raw);
  T* X = reinterpret_cast<T*>(A + cpad * cpad);
  TA* d = reinterpret_cast<TA*>(X + cpad * cpad);
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  const TA* g = G + (size_t)blockIdx.x * cpad * cpad;
  for (int t = threadIdx.x; t < c; t += blockDim.x) {
    TA v = g[t * cpad + t];
    if (!(v > TA(0)) || !isfinite((double)v)) {
      fail = 1;
      v = TA(1);
    }
    d[t] = TA(1) / sqrt(v);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    int i = e / c, j = e - i * c;
    A[i * cpad + j] = i <= j ? g[i * cpad + j] * d[i] * d[j] : TA(0);
  }
  __syncthreads();
  for (int k = 0; k < c; ++k) {
    if (threadIdx.x == 0) {
      TA p = A[k * cpad + k];
      if (!(p > TA(0)) || !isfinite((double)p)) {
        fail = 1;
        p = TA(1);
      }
      A[k * cpad + k] = sqrt(p);
    }
    __syncthreads();
    const TA rkk = A[k * cpad + k];
    for (int j = k + 1 + threadIdx.x; j < c; j += blockDim.x) A[k * cpad + j] /= rkk;
    __syncthreads();
    const int m = c - k - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      int i = k + 1 + t / m, j = k + 1 + t % m;
      if (i <= j) A[i * cpad + j] -= A[k * cpad + i] * A[k * cpad + j];
    }
    __syncthreads();
  }
  // X = R^-1 (upper) by back substitution, one column per thread, in T.
  for (int j = threadIdx.x; j < cpad; j += blockDim.x) {
    for (int i = cpad - 1; i >= 0; --i) {
      T v = 0;
      if (j < c && i <= j) {
        T s = (i == j) ? T(1) : T(0);
        for (int l = i + 1; l <= j; ++l) s -= (T)A[i * cpad + l] * X[l * cpad + j];
        v = s / (T)A[i * cpad + i];
      }
      X[i * cpad + j] = v;
    }
  }
  __syncthreads();
  // undo the scaling: R_full = R_s D^-1  =>  R_full^-1 = D R_s^-1
  T* M = Mout + (size_t)blockIdx.x * cpad * cpad;
  const bool bad = fail != 0;
  for (int e = threadIdx.x; e < cpad * cpad; e += blockDim.x) {
    int i = e / cpad, j = e - i * cpad;
    T v = (i < c && j < c) ? (T)d[i] * X[e] : T(0);
    if (bad) v = (i == j && i < c) ? T(1) : T(0);
    M[e] = v;
  }
  if (bad && threadIdx.x == 0) atomicOr(a.status, ST_NUMERICAL);
}

// Out panel = Y panel (CH x c) x M (c x c); written to Q (may alias Y: every
// CTA reads its own rows before writing them).  UPPER skips M's zero part.
// GRAM also writes the Gram partial of the output panel.
template <typename T, typename TA, bool UPPER, bool GRAM>
__global__ void __launch_bounds__(kDT) k_panel_mul(DenseArgs a, const T* Y, T* Q,
                                                   const T* __restrict__ Msm, int CH, int maxch,
                                                   TA* __restrict__ Gp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = a.batch[blockIdx.y];
  const int c = a.cb[b];
  const int cpad = pad4(a.cmax);
  const int r0 = a.bptr[b], nb = a.bptr[b + 1] - r0;
  const int row0 = blockIdx.x * CH;
  if (row0 >= nb) return;
  const int nr = min(CH, nb - row0);
  T* S = reinterpret_cast<T*>(smem_raw);
  T* O = S + CH * cpad;
  T* M = O + CH * cpad;
  stage_panel(Y, a.ld, r0 + row0, nr, c, cpad, CH, S);
  const T* msrc = Msm + (size_t)blockIdx.y * cpad * cpad;
  for (int e = threadIdx.x; e < cpad * cpad; e += blockDim.x) M[e] = msrc[e];
  __syncthreads();
  const int nti = CH / 4, ntj = cpad / 4;
  for (int u = threadIdx.x; u < nti * ntj; u += blockDim.x) {
    const int ti = u / ntj, tj = u - ti * ntj;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0;
    const int kend = UPPER ? min(cpad, 4 * tj + 4) : cpad;
    for (int kk = 0; kk < kend; kk += 4) {
      T sa[4][4], mb[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i) ld4(S + (4 * ti + i) * cpad + kk, sa[i]);
#pragma unroll
      for (int q = 0; q < 4; ++q) ld4(M + (kk + q) * cpad + 4 * tj, mb[q]);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += sa[i][q] * mb[q][j];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) O[(4 * ti + i) * cpad + 4 * tj + j] = acc[i][j];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < CH * cpad; t += blockDim.x) {
    int i = t / cpad, j = t - i * cpad;
    if (i < nr && j < c) Q[(size_t)(r0 + row0 + i) * a.ld + j] = O[t];
  }
  if constexpr (GRAM) {
    // rows past nr are zero in S, hence in O: they add nothing
    TA* out = Gp + ((size_t)blockIdx.y * maxch + blockIdx.x) * cpad * cpad;
    panel_gram<T, TA>(O, O, CH, cpad, true, out);
  }
}

// Partial H = V_panel^T (L V)_panel: (L V) rows from the block's CSR, neighbour
// rows of V read from global memory.
template <typename T, typename TA>
__global__ void __launch_bounds__(kDT) k_rr(DenseArgs a, MeshView<T> mv, const T* __restrict__ V,
                                            int CH, int maxch, TA* __restrict__ Gp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = a.batch[blockIdx.y];
  const int c = a.cb[b];
  const int cpad = pad4(a.cmax);
  const int r0 = a.bptr[b], nb = a.bptr[b + 1] - r0;
  const int row0 = blockIdx.x * CH;
  if (row0 >= nb) return;
  const int nr = min(CH, nb - row0);
  T* S = reinterpret_cast<T*>(smem_raw);
  T* W = S + CH * cpad;
  stage_panel(V, a.ld, r0 + row0, nr, c, cpad, CH, S);
  for (int t = threadIdx.x; t < CH * cpad; t += blockDim.x) {
    int i = t / cpad, j = t - i * cpad;
    T v = 0;
    if (i < nr && j < c) {
      const int64_t gr = r0 + row0 + i;
      v = mv.diag[gr] * V[gr * a.ld + j];
      for (int e = mv.rowptr[gr]; e < mv.rowptr[gr + 1]; ++e) {
        const T w = mv.wt ? mv.wt[e] : T(1);
        v -= w * V[(int64_t)(r0 + mv.col[e]) * a.ld + j];
      }
    }
    W[t] = v;
  }
  __syncthreads();
  TA* out = Gp + ((size_t)blockIdx.y * maxch + blockIdx.x) * cpad * cpad;
  panel_gram<T, TA>(S, W, CH, cpad, false, out);
}

// Cyclic Jacobi eigensolve of H = (G + G^T)/2 (c x c) in T; writes the
// eigenvectors sorted by ascending eigenvalue into Q_out (cpad x cpad) and
// the eigenvalues into theta (cpad).  Round-robin pairing gives c/2 disjoint
// rotations per round.
template <typename T, typename TA>
__global__ void __launch_bounds__(kDT) k_jacobi(DenseArgs a, const TA* __restrict__ G,
                                                T* __restrict__ Qout, T* __restrict__ theta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = a.batch[blockIdx.x];
  const int c = a.cb[b];
  const int cpad = pad4(a.cmax);
  const int ne = (c + 1) & ~1;  // even size for round-robin pairing (dummy index if c is odd)
  const int ld = cpad + 1;      // padded stride against bank conflicts
  T* H = reinterpret_cast<T*>(smem_raw);
  T* Qm = H + cpad * ld;
  T* cs = Qm + cpad * ld;
  T* sn = cs + cpad / 2 + 1;
  int* pp = reinterpret_cast<int*>(sn + cpad / 2 + 1);
  int* qq = pp + cpad / 2 + 1;
  const TA* g = G + (size_t)blockIdx.x * cpad * cpad;
  for (int e = threadIdx.x; e < ne * ne; e += blockDim.x) {
    int i = e / ne, j = e - i * ne;
    T v;
    if (i < c && j < c) v = (T)(0.5 * ((double)g[i * cpad + j] + (double)g[j * cpad + i]));
    else v = (i == j) ? (T)1e30 : T(0);
    H[i * ld + j] = v;
    Qm[i * ld + j] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  const T eps = sizeof(T) == 4 ? (T)1e-7 : (T)1e-15;
  // absolute floor for pairs next to the (near-)zero Ritz value of L's null space
  __shared__ T hscale;
  __shared__ int rotated;
  if (threadIdx.x == 0) {
    T m = 0;
    for (int i = 0; i < c; ++i) m = fmax(m, fabs(H[i * ld + i]));
    hscale = m;
  }
  __syncthreads();
  const T floor_abs = eps * (T)1e-2 * hscale;
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int rnd = 0; rnd < ne - 1; ++rnd) {
      for (int m = threadIdx.x; m < ne / 2; m += blockDim.x) {
        // round-robin: position 0 fixed, others rotate
        auto player = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + rnd) % (ne - 1); };
        int p = player(m), q = player(ne - 1 - m);
        if (p > q) { int t = p; p = q; q = t; }
        T hpq = H[p * ld + q], hpp = H[p * ld + p], hqq = H[q * ld + q];
        T cth = 1, sth = 0;
        if (fabs(hpq) > eps * sqrt(fabs(hpp * hqq)) && fabs(hpq) > floor_abs) {
          rotated = 1;
          T tau = (hqq - hpp) / (2 * hpq);
          T t = (tau >= 0 ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
          cth = T(1) / sqrt(T(1) + t * t);
          sth = t * cth;
        }
        pp[m] = p; qq[m] = q; cs[m] = cth; sn[m] = sth;
      }
      __syncthreads();
      // rows p, q  <-  J^T H
      for (int t = threadIdx.x; t < (ne / 2) * ne; t += blockDim.x) {
        int m = t / ne, k = t - m * ne;
        int p = pp[m], q = qq[m];
        T cth = cs[m], sth = sn[m];
        T hp = H[p * ld + k], hq = H[q * ld + k];
        H[p * ld + k] = cth * hp - sth * hq;
        H[q * ld + k] = sth * hp + cth * hq;
      }
      __syncthreads();
      // columns p, q  <-  H J ; eigenvectors Q <- Q J
      for (int t = threadIdx.x; t < (ne / 2) * ne; t += blockDim.x) {
        int m = t / ne, k = t - m * ne;
        int p = pp[m], q = qq[m];
        T cth = cs[m], sth = sn[m];
        T hp = H[k * ld + p], hq = H[k * ld + q];
        H[k * ld + p] = cth * hp - sth * hq;
        H[k * ld + q] = sth * hp + cth * hq;
        T qp = Qm[k * ld + p], qv = Qm[k * ld + q];
        Qm[k * ld + p] = cth * qp - sth * qv;
        Qm[k * ld + q] = sth * qp + cth * qv;
      }
      __syncthreads();
    }
    __syncthreads();
    const int any = rotated;
    __syncthreads();  // every thread has read the flag before thread 0 resets it
    if (!any) break;
  }
  // sort ascending: rank of each eigenvalue (ties broken by index)
  T* Qo = Qout + (size_t)blockIdx.x * cpad * cpad;
  T* th = theta + (size_t)blockIdx.x * cpad;
  for (int i = threadIdx.x; i < cpad; i += blockDim.x) {
    if (i >= c) {
      th[i] = 0;
      continue;
    }
    T li = H[i * ld + i];
    int rank = 0;
    for (int j = 0; j < c; ++j) {
      T lj = H[j * ld + j];
      rank += (lj < li) || (lj == li && j < i);
    }
    th[rank] = li;
    for (int k = 0; k < cpad; ++k) Qo[k * cpad + rank] = k < c ? Qm[k * ld + i] : T(0);
  }
  for (int e = threadIdx.x; e < cpad * (cpad - c); e += blockDim.x) {  // zero padding columns
    int k = e / (cpad - c), j = c + e % (cpad - c);
    Qo[k * cpad + j] = 0;
  }
}

template <typename T, typename TA>
size_t panel_smem(int CH, int cpad) {
  return (size_t)(2 * CH * cpad + cpad * cpad) * sizeof(T);
}

template <typename T, typename TA>
void configure_one() {
  set_max_dynamic_smem(k_gram<T, TA>);
  set_max_dynamic_smem(k_chol<T, TA>);
  set_max_dynamic_smem(k_panel_mul<T, TA, true, true>);
  set_max_dynamic_smem(k_panel_mul<T, TA, true, false>);
  set_max_dynamic_smem(k_panel_mul<T, TA, false, false>);
  set_max_dynamic_smem(k_rr<T, TA>);
  set_max_dynamic_smem(k_jacobi<T, TA>);
}

}  // namespace

int dense_chunk_rows(int cpad, int rb) {
  const int opts[3] = {128, 64, 32};
  for (int ch : opts)
    if ((size_t)(2 * ch * cpad + cpad * cpad) * rb <= 200 * 1024) return ch;
  return 16;
}

void configure_dense_kernels() {
  configure_one<float, float>();
  configure_one<float, double>();
  configure_one<double, double>();
}

// One Onorm: G1 = Y^T Y (TA), Cholesky (TA), Q1 = Y R1^-1 fused with G2 = Q1^T Q1
// (T), Cholesky (T), Q = Q1 R2^-1.  Q may alias Y.
template <typename T, typename TA>
int launch_cholqr2(const DenseArgs& a, const T* Y, T* Q, TA* Gp, T* Rsm, cudaStream_t s,
                   int* launches) {
  const int cpad = pad4(a.cmax);
  const int CH = dense_chunk_rows(cpad, sizeof(T));
  const int maxch = (a.max_nb + CH - 1) / CH;
  // partial-Gram area first, reduced Gram after it (both in the Gp workspace)
  TA* G = Gp + (size_t)a.nbatch * maxch * cpad * cpad;
  T* Gp2raw = reinterpret_cast<T*>(Gp);  // pass 2 partials in T reuse the same area
  T* G2 = Gp2raw + (size_t)a.nbatch * maxch * cpad * cpad;
  dim3 gp(maxch, a.nbatch);
  const size_t sm_panel = (size_t)CH * cpad * sizeof(T);
  prof_begin(KC_GRAM, s);
  k_gram<T, TA><<<gp, kDT, sm_panel, s>>>(a, Y, CH, maxch, Gp);
  prof_end(KC_GRAM, s);
  dim3 gr((cpad * cpad + kDT - 1) / kDT, a.nbatch);
  prof_begin(KC_REDUCE, s);
  k_reduce<TA><<<gr, kDT, 0, s>>>(a, CH, maxch, true, Gp, G);
  prof_end(KC_REDUCE, s);
  const size_t sm_chol_a = (size_t)cpad * cpad * sizeof(TA) + (size_t)cpad * cpad * sizeof(T) +
                           (size_t)cpad * sizeof(TA) + 16;
  prof_begin(KC_CHOL, s);
  k_chol<T, TA><<<a.nbatch, kDT, sm_chol_a, s>>>(a, G, Rsm);
  prof_end(KC_CHOL, s);
  const size_t sm_mul = panel_smem<T, TA>(CH, cpad);
  prof_begin(KC_PANEL, s);
  k_panel_mul<T, T, true, true><<<gp, kDT, sm_mul, s>>>(a, Y, Q, Rsm, CH, maxch, Gp2raw);
  prof_end(KC_PANEL, s);
  prof_begin(KC_REDUCE, s);
  k_reduce<T><<<gr, kDT, 0, s>>>(a, CH, maxch, true, Gp2raw, G2);
  prof_end(KC_REDUCE, s);
  const size_t sm_chol_b = (size_t)cpad * cpad * sizeof(T) * 2 + (size_t)cpad * sizeof(T) + 16;
  prof_begin(KC_CHOL, s);
  k_chol<T, T><<<a.nbatch, kDT, sm_chol_b, s>>>(a, G2, Rsm);
  prof_end(KC_CHOL, s);
  prof_begin(KC_PANEL, s);
  k_panel_mul<T, T, true, false><<<gp, kDT, sm_mul, s>>>(a, Q, Q, Rsm, CH, maxch, (T*)nullptr);
  prof_end(KC_PANEL, s);
  if (launches) *launches += 7;
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

template <typename T, typename TA>
int launch_rayleigh_ritz(const DenseArgs& a, const MeshView<T>& mv, T* V, TA* Gp, T* Rsm,
                         T* theta, cudaStream_t s, int* launches) {
  const int cpad = pad4(a.cmax);
  const int CH = dense_chunk_rows(cpad, sizeof(T));
  const int maxch = (a.max_nb + CH - 1) / CH;
  TA* G = Gp + (size_t)a.nbatch * maxch * cpad * cpad;
  dim3 gp(maxch, a.nbatch);
  prof_begin(KC_RR, s);
  k_rr<T, TA><<<gp, kDT, (size_t)2 * CH * cpad * sizeof(T), s>>>(a, mv, V, CH, maxch, Gp);
  prof_end(KC_RR, s);
  dim3 gr((cpad * cpad + kDT - 1) / kDT, a.nbatch);
  prof_begin(KC_REDUCE, s);
  k_reduce<TA><<<gr, kDT, 0, s>>>(a, CH, maxch, false, Gp, G);
  prof_end(KC_REDUCE, s);
  const size_t ldp = cpad + 1;
  const size_t sm_j = (size_t)2 * cpad * ldp * sizeof(T) + (size_t)2 * (cpad / 2 + 1) * sizeof(T) +
                      (size_t)2 * (cpad / 2 + 1) * sizeof(int) + 16;
  prof_begin(KC_JACOBI, s);
  k_jacobi<T, TA><<<a.nbatch, kDT, sm_j, s>>>(a, G, Rsm, theta);
  prof_end(KC_JACOBI, s);
  prof_begin(KC_PANEL, s);
  k_panel_mul<T, T, false, false><<<gp, kDT, panel_smem<T, TA>(CH, cpad), s>>>(
      a, V, V, Rsm, CH, maxch, (T*)nullptr);
  prof_end(KC_PANEL, s);
  if (launches) *launches += 4;
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

template int launch_cholqr2<float, double>(const DenseArgs&, const float*, float*, double*,
                                           float*, cudaStream_t, int*);
template int launch_cholqr2<float, float>(const DenseArgs&, const float*, float*, float*, float*,
                                          cudaStream_t, int*);
template int launch_cholqr2<double, double>(const DenseArgs&, const double*, double*, double*,
                                            double*, cudaStream_t, int*);
template int launch_rayleigh_ritz<float, double>(const DenseArgs&, const MeshView<float>&,
                                                 float*, double*, float*, float*, cudaStream_t,
                                                 int*);
template int launch_rayleigh_ritz<float, float>(const DenseArgs&, const MeshView<float>&, float*,
                                                float*, float*, float*, cudaStream_t, int*);
template int launch_rayleigh_ritz<double, double>(const DenseArgs&, const MeshView<double>&,
                                                  double*, double*, double*, double*,
                                                  cudaStream_t, int*);

}  // namespace bsp
