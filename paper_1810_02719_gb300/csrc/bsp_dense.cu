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

#include "bsp_dense_dev.cuh"

namespace bsp {
namespace {

using namespace dev;
constexpr int kJacobiSweeps = 20;

template <typename T, typename TA>
__global__ void __launch_bounds__(kDT) k_gram(DenseArgs a, const T* __restrict__ Y, int CH,
                                              int maxch, TA* __restrict__ Gp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);
  const int b = a.batch[blockIdx.y];
  if (a.live && !a.live[b]) return;
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
  if (a.live && !a.live[b]) return;
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

// M = R^-1 (upper, T, cpad x cpad) for G = R^T R with G given by its upper
// triangle g (type TG, stride cpad, global or shared memory); the Cholesky
// runs in TA after Jacobi scaling D G D, D = diag(G)^-1/2.  Shared workspace:
// A [cpad x cpad] TA (scaled G, updated in place), d [2 cpad] TA (scaling,
// then the pivot row), Rr [CP x CP] T (R, zero-padded to the width CP >= c, a
// power of two >= 32).  A must hold max(cpad^2 TA, 1.5 CP^2 T) bytes: R^-1
// and its temporaries reuse it after the factorization.  *fail (shared) is set
// on a non-positive or non-finite pivot; M is then the identity.  Called by
// all threads; ends with a barrier.
//
// Factorization: right-looking, two barriers per column; the trailing update
// of column k is tiled over a 16 x 16 thread grid (balanced, division-free).
template <typename T, typename TA, typename TG, int CP>
BSP_DEV void chol_inverse(const TG* g, int c, int cpad, TA* A, TA* d, T* Rr, T* M, int* fail) {
  for (int t = threadIdx.x; t < CP * CP; t += blockDim.x) Rr[t] = T(0);
  for (int t = threadIdx.x; t < c; t += blockDim.x) {
    TA v = (TA)g[t * cpad + t];
    if (!(v > TA(0)) || !isfinite((double)v)) {
      *fail = 1;
      v = TA(1);
    }
    d[t] = rsqrt_newton(v);
  }
  __syncthreads();
  for (int i = threadIdx.x >> 5; i < c; i += blockDim.x >> 5)
    for (int jj = (threadIdx.x & 31) + i; jj < c; jj += 32)  // upper triangle only
      A[i * cpad + jj] = (TA)g[i * cpad + jj] * d[i] * d[jj];
  __syncthreads();
  TA* lrow = d + cpad;  // scaled pivot row (TA)
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 (256 threads)
  for (int k = 0; k < c; ++k) {
    if (ty == 0) {
      TA piv = A[k * cpad + k];
      if (!(piv > TA(0)) || !isfinite((double)piv)) {
        *fail = 1;
        piv = TA(1);
      }
      const TA inv = rsqrt_newton(piv);
      for (int jj = k + tx; jj < c; jj += 16) {
        const TA lj = A[k * cpad + jj] * inv;
        lrow[jj] = lj;
        Rr[k * CP + jj] = (T)lj;
      }
    }
    __syncthreads();
    for (int i = k + 1 + ty; i < c; i += 16) {
      const TA li = lrow[i];
      int j0 = k + 1 + tx;
      if (j0 < i) j0 += ((i - j0 + 15) >> 4) << 4;   // first j >= i in this thread's lane
      for (int jj = j0; jj < c; jj += 16) A[i * cpad + jj] -= li * lrow[jj];
    }
    __syncthreads();
  }
  // R^-1 by recursive blocking: rows/columns >= c act as the identity; the 16 x
  // 16 diagonal blocks are inverted by per-thread back substitution (thread =
  // column, 16 registers), then levels s = 16, 32, ... combine block pairs with
  // X12 = -X11 R12 X22 as two small shared-memory GEMMs (four barriers/level).
  T* X = reinterpret_cast<T*>(A);             // CP x CP
  T* W = X + CP * CP;                         // CP x CP / 2 temporaries
  for (int i = threadIdx.x; i < CP; i += blockDim.x)
    if (i >= c) Rr[i * CP + i] = T(1);
  for (int t = threadIdx.x; t < CP * CP; t += blockDim.x) X[t] = T(0);
  __syncthreads();
  if (threadIdx.x < CP) {
    const int q0 = threadIdx.x & ~15, jl = threadIdx.x & 15;
    T x[16];
#pragma unroll
    for (int i = 15; i >= 0; --i) {
      T sum = (i == jl) ? T(1) : T(0);
#pragma unroll
      for (int l = i + 1; l < 16; ++l) sum -= Rr[(q0 + i) * CP + q0 + l] * x[l];
      x[i] = sum / Rr[(q0 + i) * CP + q0 + i];
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) X[(q0 + i) * CP + q0 + jl] = i <= jl ? x[i] : T(0);
  }
  __syncthreads();
  for (int sz = 16; sz < CP; sz <<= 1) {
    int lg = 0;
    while ((1 << lg) < sz) ++lg;
    const int npair = CP / (2 * sz), tot = npair * sz * sz;
    // W = R12 X22 for every pair (blocks at o = m 2 sz)
    for (int u = threadIdx.x; u < tot; u += blockDim.x) {
      const int m = u >> (2 * lg), rem = u & (sz * sz - 1);
      const int i = rem >> lg, jj = rem & (sz - 1);
      const int o = m * 2 * sz;
      T acc = 0;
      for (int l = 0; l < sz; ++l) acc += Rr[(o + i) * CP + o + sz + l] * X[(o + sz + l) * CP + o + sz + jj];
      W[u] = acc;
    }
    __syncthreads();
    // X12 = -X11 W
    for (int u = threadIdx.x; u < tot; u += blockDim.x) {
      const int m = u >> (2 * lg), rem = u & (sz * sz - 1);
      const int i = rem >> lg, jj = rem & (sz - 1);
      const int o = m * 2 * sz;
      T acc = 0;
      for (int l = 0; l < sz; ++l) acc += X[(o + i) * CP + o + l] * W[(m * sz + l) * sz + jj];
      X[(o + i) * CP + o + sz + jj] = -acc;
    }
    __syncthreads();
  }
  // M = D R_s^-1 (undo the Jacobi scaling)
  const bool bad = *fail != 0;
  for (int i = threadIdx.x >> 5; i < cpad; i += blockDim.x >> 5)
    for (int jj = threadIdx.x & 31; jj < cpad; jj += 32) {
      T v = (i < c && jj < c && i <= jj) ? (T)d[i] * X[i * CP + jj] : T(0);
      if (bad) v = (i == jj && i < c) ? T(1) : T(0);
      M[i * cpad + jj] = v;
    }
  __syncthreads();
}

// Dispatch on the compile-time width.
template <typename T, typename TA, typename TG>
BSP_DEV void chol_inverse_any(const TG* g, int c, int cpad, TA* A, TA* d, T* Rr, T* M, int* fail) {
  if (c <= 32) chol_inverse<T, TA, TG, 32>(g, c, cpad, A, d, Rr, M, fail);
  else if (c <= 64) chol_inverse<T, TA, TG, 64>(g, c, cpad, A, d, Rr, M, fail);
  else chol_inverse<T, TA, TG, 128>(g, c, cpad, A, d, Rr, M, fail);
}

// Cholesky + inverse for each block of the batch (one CTA per block): the
// Gram in TG, the factorization in TA.
template <typename T, typename TA, typename TG = TA>
__global__ void __launch_bounds__(kDT) k_chol(DenseArgs a, const TG* __restrict__ G,
                                              T* __restrict__ Mout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = a.batch[blockIdx.x];
  if (a.live && !a.live[b]) return;
  const int c = a.cb[b];
  const int cpad = pad4(a.cmax);
  TA* A = reinterpret_cast<TA*>(smem_raw);
  TA* d = A + chol_a_elems<T, TA>(cpad, chol_cp(cpad));
  T* Rr = reinterpret_cast<T*>(d + 2 * cpad);
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  chol_inverse_any<T, TA, TG>(G + (size_t)blockIdx.x * cpad * cpad, c, cpad, A, d, Rr,
                              Mout + (size_t)blockIdx.x * cpad * cpad, &fail);
  if (fail && threadIdx.x == 0) atomicOr(a.status, ST_NUMERICAL);
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
  if (a.live && !a.live[b]) return;
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
  if (a.live && !a.live[b]) return;
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
  if (a.live && !a.live[b]) return;
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
  // Rounding in T leaves off-diagonal noise of order eps * ||H||: pairs below
  // that floor are treated as converged.
  const T floor_abs = (T)8 * eps * hscale;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  int sweeps = 0;
  // per-round "some pair rotates" flags in three rotating slots: round r sets
  // slot r % 3 and clears slot (r + 1) % 3 before its first barrier, so the
  // next round's writers (past that barrier) never race the clearing, and a
  // round without rotations skips its two update phases and their barriers
  __shared__ int rot[3];
  if (threadIdx.x < 3) rot[threadIdx.x] = 0;
  int rr = 0;
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    // any pair above threshold?  (checked before the sweep: a nearly diagonal
    // H, the common case for a warm-started block, costs one pass)
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int i = warp; i < c; i += nwarp)
      for (int jj = i + 1 + lane; jj < c; jj += 32) {
        const T hij = H[i * ld + jj];
        if (fabs(hij) > eps * sqrt(fabs(H[i * ld + i] * H[jj * ld + jj])) && fabs(hij) > floor_abs)
          rotated = 1;
      }
    __syncthreads();
    const int any = rotated;
    if (!any) break;
    ++sweeps;
    for (int rnd = 0; rnd < ne - 1; ++rnd, rr = rr == 2 ? 0 : rr + 1) {
      if (threadIdx.x == 0) rot[rr == 2 ? 0 : rr + 1] = 0;
      for (int m = threadIdx.x; m < ne / 2; m += blockDim.x) {
        // round-robin: position 0 fixed, the others rotate by one per round
        int p = m == 0 ? 0 : 1 + (m - 1 + rnd) % (ne - 1);
        int q = 1 + (ne - 2 - m + rnd) % (ne - 1);
        if (p > q) { int t = p; p = q; q = t; }
        T hpq = H[p * ld + q], hpp = H[p * ld + p], hqq = H[q * ld + q];
        T cth = 1, sth = 0;
        if (fabs(hpq) > eps * sqrt(fabs(hpp * hqq)) && fabs(hpq) > floor_abs) {
          T tau = (hqq - hpp) / (2 * hpq);
          T t = (tau >= 0 ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
          cth = T(1) / sqrt(T(1) + t * t);
          sth = t * cth;
          rot[rr] = 1;
        }
        pp[m] = p; qq[m] = q; cs[m] = cth; sn[m] = sth;
      }
      __syncthreads();
      if (!rot[rr]) continue;   // uniform: nothing to rotate this round
      // rows p, q  <-  J^T H   (warp per pair, lane per column)
      for (int m = warp; m < ne / 2; m += nwarp) {
        const int p = pp[m], q = qq[m];
        const T cth = cs[m], sth = sn[m];
        if (sth == T(0)) continue;
        for (int k = lane; k < ne; k += 32) {
          const T hp = H[p * ld + k], hq = H[q * ld + k];
          H[p * ld + k] = cth * hp - sth * hq;
          H[q * ld + k] = sth * hp + cth * hq;
        }
      }
      __syncthreads();
      // columns p, q  <-  H J ; eigenvectors Q <- Q J
      for (int m = warp; m < ne / 2; m += nwarp) {
        const int p = pp[m], q = qq[m];
        const T cth = cs[m], sth = sn[m];
        if (sth == T(0)) continue;
        for (int k = lane; k < ne; k += 32) {
          const T hp = H[k * ld + p], hq = H[k * ld + q];
          H[k * ld + p] = cth * hp - sth * hq;
          H[k * ld + q] = sth * hp + cth * hq;
          const T qp = Qm[k * ld + p], qv = Qm[k * ld + q];
          Qm[k * ld + p] = cth * qp - sth * qv;
          Qm[k * ld + q] = sth * qp + cth * qv;
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0 && a.sweeps) atomicAdd(a.sweeps, sweeps);
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
  set_max_dynamic_smem(k_chol<T, T, TA>);
  set_max_dynamic_smem(k_panel_mul<T, TA, true, true>);
  set_max_dynamic_smem(k_panel_mul<T, TA, true, false>);
  set_max_dynamic_smem(k_panel_mul<T, TA, false, false>);
  set_max_dynamic_smem(k_rr<T, TA>);
  set_max_dynamic_smem(k_jacobi<T, TA>);
}

}  // namespace

bool g_disable_fused = false;

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
  configure_fused_kernels();
}

// One Onorm: G1 = Y^T Y (TA), Cholesky (TA), Q1 = Y R1^-1 fused with G2 = Q1^T Q1
// (TA), Cholesky (TA), Q = Q1 R2^-1.  Q may alias Y.
template <typename T, typename TA>
int launch_cholqr2(const DenseArgs& a, const T* Y, T* Q, TA* Gp, T* Rsm, cudaStream_t s,
                   int* launches, int passes) {
  const int cpad = pad4(a.cmax);
  const int CH = dense_chunk_rows(cpad, sizeof(T));
  const int maxch = (a.max_nb + CH - 1) / CH;
  // Fused path (c <= 64): one cluster launch per batch of blocks.
  if (cpad <= 64 && !g_disable_fused) {
    const int rc = launch_cholqr2_fused<T, TA>(a, Y, Q, Gp, maxch, s, passes);
    if (rc != BSP_ERR_INVALID_ARG) {
      if (launches) *launches += 1;
      return rc;
    }
  }
  // partial-Gram area first, reduced Gram after it (both in the Gp workspace)
  TA* G = Gp + (size_t)a.nbatch * maxch * cpad * cpad;
  dim3 gp(maxch, a.nbatch);
  const size_t sm_panel = (size_t)CH * cpad * sizeof(T);
  prof_begin(KC_GRAM, s);
  k_gram<T, TA><<<gp, kDT, sm_panel, s>>>(a, Y, CH, maxch, Gp);
  prof_end(KC_GRAM, s);
  dim3 gr((cpad * cpad + kDT - 1) / kDT, a.nbatch);
  prof_begin(KC_REDUCE, s);
  k_reduce<TA><<<gr, kDT, 0, s>>>(a, CH, maxch, true, Gp, G);
  prof_end(KC_REDUCE, s);
  const int cpw = chol_cp(cpad);
  const size_t sm_chol_a = (size_t)(chol_a_elems<T, TA>(cpad, cpw) + 2 * cpad) * sizeof(TA) +
                           (size_t)cpw * cpw * sizeof(T);
  prof_begin(KC_CHOL, s);
  k_chol<T, TA><<<a.nbatch, kDT, sm_chol_a, s>>>(a, G, Rsm);
  prof_end(KC_CHOL, s);
  const size_t sm_mul = panel_smem<T, TA>(CH, cpad);
  if (passes < 2) {
    prof_begin(KC_PANEL, s);
    k_panel_mul<T, T, true, false><<<gp, kDT, sm_mul, s>>>(a, Y, Q, Rsm, CH, maxch, (T*)nullptr);
    prof_end(KC_PANEL, s);
    if (launches) *launches += 4;
    return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
  }
  // pass 2: the Gram of Q1 accumulates in TA; it is I + O(kappa u), so its
  // Cholesky runs in T
  prof_begin(KC_PANEL, s);
  k_panel_mul<T, TA, true, true><<<gp, kDT, sm_mul, s>>>(a, Y, Q, Rsm, CH, maxch, Gp);
  prof_end(KC_PANEL, s);
  prof_begin(KC_REDUCE, s);
  k_reduce<TA><<<gr, kDT, 0, s>>>(a, CH, maxch, true, Gp, G);
  prof_end(KC_REDUCE, s);
  const size_t sm_chol_b = (size_t)(chol_a_elems<T, T>(cpad, cpw) + 2 * cpad) * sizeof(T) +
                           (size_t)cpw * cpw * sizeof(T);
  prof_begin(KC_CHOL, s);
  k_chol<T, T, TA><<<a.nbatch, kDT, sm_chol_b, s>>>(a, G, Rsm);
  prof_end(KC_CHOL, s);
  prof_begin(KC_PANEL, s);
  k_panel_mul<T, T, true, false><<<gp, kDT, sm_mul, s>>>(a, Q, Q, Rsm, CH, maxch, (T*)nullptr);
  prof_end(KC_PANEL, s);
  if (launches) *launches += 7;
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

// Chunk Grams -> G (fixed order), then M = D R^-1 per block: the middle of one
// CholeskyQR pass whose chunk products run elsewhere (bsp_tcqr.cu).
template <typename T, typename TA>
int launch_reduce_chol(const DenseArgs& a, int CH, int maxch, const TA* Gp, TA* G, T* Rsm,
                       cudaStream_t s) {
  const int cpad = pad4(a.cmax);
  dim3 gr((cpad * cpad + kDT - 1) / kDT, a.nbatch);
  prof_begin(KC_REDUCE, s);
  k_reduce<TA><<<gr, kDT, 0, s>>>(a, CH, maxch, true, Gp, G);
  prof_end(KC_REDUCE, s);
  const int cpw = chol_cp(cpad);
  const size_t sm = (size_t)(chol_a_elems<T, TA>(cpad, cpw) + 2 * cpad) * sizeof(TA) +
                    (size_t)cpw * cpw * sizeof(T);
  prof_begin(KC_CHOL, s);
  k_chol<T, TA><<<a.nbatch, kDT, sm, s>>>(a, G, Rsm);
  prof_end(KC_CHOL, s);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}
template int launch_reduce_chol<float, float>(const DenseArgs&, int, int, const float*, float*,
                                              float*, cudaStream_t);
template int launch_reduce_chol<float, double>(const DenseArgs&, int, int, const double*, double*,
                                               float*, cudaStream_t);

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

template int launch_cholqr2<float, double>(const DenseArgs&, const float*, float*, double*, float*, cudaStream_t, int*, int);
template int launch_cholqr2<float, float>(const DenseArgs&, const float*, float*, float*, float*,
                                          cudaStream_t, int*, int);
template int launch_cholqr2<double, double>(const DenseArgs&, const double*, double*, double*, double*, cudaStream_t, int*, int);
template int launch_rayleigh_ritz<float, double>(const DenseArgs&, const MeshView<float>&,
                                                 float*, double*, float*, float*, cudaStream_t,
                                                 int*);
template int launch_rayleigh_ritz<float, float>(const DenseArgs&, const MeshView<float>&, float*,
                                                float*, float*, float*, cudaStream_t, int*);
template int launch_rayleigh_ritz<double, double>(const DenseArgs&, const MeshView<double>&,
                                                  double*, double*, double*, double*,
                                                  cudaStream_t, int*);

}  // namespace bsp
