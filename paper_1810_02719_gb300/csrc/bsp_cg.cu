// The iteration operator S = R^z, R = (L + delta I)^-1 (Sec. 4, below
// Algorithm 1), applied to a block's subspace V with conjugate gradients: the
// paper computes R^z U with sparse linear-system solvers.  Every CG step costs
// one product (L + delta I) P, the sparse x tall-skinny kernel that this file
// also exposes on its own (k_spmm) for all blocks at once.
//
// k_cg: one CTA per (block, slab of CS columns).  The columns of V are
// independent right-hand sides, so a CTA runs its slab's whole CG on chip:
// p, x, r and q live in shared memory as [row][CS] arrays, neighbour rows of p
// are read from shared memory, and the only global traffic is the block's
// sparsity pattern (L1/L2 resident) plus V in and Y out.  Initial guess
// x0 = b / (theta + delta) with theta + delta the Rayleigh quotient of
// (L + delta I) for that column: exact when b is an eigenvector, which is what
// a warm start from the previous block's Ritz basis approaches.
#include <cstdio>

#include "bsp_internal.cuh"

namespace bsp {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// ---- row I/O helpers: CS contiguous values in shared memory
template <typename T, int CS>
BSP_DEV void lds_row(const T* s, T (&v)[CS]) {
  if constexpr (sizeof(T) * CS % 16 == 0) {
    constexpr int NV = sizeof(T) * CS / 16;
    const float4* s4 = reinterpret_cast<const float4*>(s);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      float4 t = s4[i];
      const T* tp = reinterpret_cast<const T*>(&t);
#pragma unroll
      for (int j = 0; j < 16 / (int)sizeof(T); ++j) v[i * (16 / sizeof(T)) + j] = tp[j];
    }
  } else {
#pragma unroll
    for (int j = 0; j < CS; ++j) v[j] = s[j];
  }
}

template <typename T, int CS>
BSP_DEV void sts_row(T* s, const T (&v)[CS]) {
  if constexpr (sizeof(T) * CS % 16 == 0) {
    constexpr int NV = sizeof(T) * CS / 16;
    float4* s4 = reinterpret_cast<float4*>(s);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      float4 t;
      T* tp = reinterpret_cast<T*>(&t);
#pragma unroll
      for (int j = 0; j < 16 / (int)sizeof(T); ++j) tp[j] = v[i * (16 / sizeof(T)) + j];
      s4[i] = t;
    }
  } else {
#pragma unroll
    for (int j = 0; j < CS; ++j) s[j] = v[j];
  }
}

// Sum each of the N per-thread values over the CTA; every thread gets the sums.
// Two alternating buffers make one __syncthreads per reduction sufficient.
template <typename T, int N>
BSP_DEV void block_sum(T (&v)[N], T (*red)[kWarps][N], int& buf) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < N; ++j) v[j] = warp_sum(v[j]);
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < N; ++j) red[buf][w][j] = v[j];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < N; ++j) {
    T s = 0;
#pragma unroll
    for (int i = 0; i < kWarps; ++i) s += red[buf][i][j];
    v[j] = s;
  }
  buf ^= 1;
}

// q_i = (D_ii + delta) p_i - sum_j C_ij p_j  for one local row i (p in smem).
template <typename T, int CS>
BSP_DEV void apply_row(const MeshView<T>& mv, int r0, int i, T delta, const T* p, T (&q)[CS]) {
  const int64_t gr = r0 + i;
  const T dd = mv.diag[gr] + delta;
  T pi[CS];
  lds_row<T, CS>(p + (size_t)i * CS, pi);
#pragma unroll
  for (int j = 0; j < CS; ++j) q[j] = dd * pi[j];
  const int e0 = __ldg(mv.rowptr + gr), e1 = __ldg(mv.rowptr + gr + 1);
  for (int e = e0; e < e1; ++e) {
    const int nj = __ldg(mv.col + e);
    const T w = mv.wt ? mv.wt[e] : T(1);
    T pj[CS];
    lds_row<T, CS>(p + (size_t)nj * CS, pj);
#pragma unroll
    for (int j = 0; j < CS; ++j) q[j] -= w * pj[j];
  }
}

template <typename T, int CS>
__global__ void __launch_bounds__(kThreads) k_cg(MeshView<T> mv, const T* __restrict__ V,
                                                 T* __restrict__ Y, CgArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // separate double-buffered reduction arrays for the 2CS- and CS-wide sums,
  // so consecutive reductions of different widths never alias
  __shared__ T red2[2][kWarps][2 * CS];
  __shared__ T red1[2][kWarps][CS];
  const int b = a.batch[blockIdx.y];
  if (a.live && !a.live[b]) return;
  const int c = a.cb[b];
  const int j0 = blockIdx.x * CS;
  if (j0 >= c) return;
  const int ncol = min(CS, c - j0);
  const int r0 = mv.bptr[b];
  const int nb = mv.bptr[b + 1] - r0;
  T* p = reinterpret_cast<T*>(smem_raw);
  T* x = p + (size_t)nb * CS;
  T* r = x + (size_t)nb * CS;
  T* q = r + (size_t)nb * CS;
  const T delta = (T)a.delta;
  const T rtol2 = (T)(a.rtol * a.rtol);
  int buf1 = 0, buf2 = 0;

  // right-hand side b = V slab (zero-padded past ncol)
  const int rv = a.vsrc ? mv.bptr[a.vsrc[b]] : r0;
  for (int i = threadIdx.x; i < nb; i += kThreads) {
    T v[CS];
#pragma unroll
    for (int j = 0; j < CS; ++j) v[j] = j < ncol ? V[(size_t)(rv + i) * a.ld + j0 + j] : T(0);
    sts_row<T, CS>(p + (size_t)i * CS, v);
  }
  __syncthreads();

  int steps_all = 0, steps_max = 0;
  bool unconverged = false, bad = false;
  for (int sol = 0; sol < a.z; ++sol) {
    // q = A b; scalars ||b||^2 and b^T A b
    T s2[2 * CS];
#pragma unroll
    for (int j = 0; j < 2 * CS; ++j) s2[j] = 0;
    for (int i = threadIdx.x; i < nb; i += kThreads) {
      T qi[CS], pi[CS];
      apply_row<T, CS>(mv, r0, i, delta, p, qi);
      lds_row<T, CS>(p + (size_t)i * CS, pi);
      sts_row<T, CS>(q + (size_t)i * CS, qi);
#pragma unroll
      for (int j = 0; j < CS; ++j) {
        s2[j] += pi[j] * pi[j];
        s2[CS + j] += pi[j] * qi[j];
      }
    }
    block_sum<T, 2 * CS>(s2, red2, buf2);
    T g[CS], bn2[CS], rr[CS];
#pragma unroll
    for (int j = 0; j < CS; ++j) {
      bn2[j] = s2[j];
      g[j] = s2[CS + j] > T(0) ? s2[j] / s2[CS + j] : T(0);
      rr[j] = 0;
    }
    // x0 = g b, r0 = b - g A b, p0 = r0
    for (int i = threadIdx.x; i < nb; i += kThreads) {
      T pi[CS], qi[CS], xi[CS], ri[CS];
      lds_row<T, CS>(p + (size_t)i * CS, pi);
      lds_row<T, CS>(q + (size_t)i * CS, qi);
#pragma unroll
      for (int j = 0; j < CS; ++j) {
        xi[j] = g[j] * pi[j];
        ri[j] = pi[j] - g[j] * qi[j];
        rr[j] += ri[j] * ri[j];
      }
      sts_row<T, CS>(x + (size_t)i * CS, xi);
      sts_row<T, CS>(r + (size_t)i * CS, ri);
      sts_row<T, CS>(p + (size_t)i * CS, ri);   // own row only: no hazard
    }
    {
      T t[CS];
#pragma unroll
      for (int j = 0; j < CS; ++j) t[j] = rr[j];
      block_sum<T, CS>(t, red1, buf1);
#pragma unroll
      for (int j = 0; j < CS; ++j) rr[j] = t[j];
    }
    __syncthreads();  // p fully written before the first product

    int steps = 0;
    for (;;) {
      bool done[CS];
      bool all = true;
#pragma unroll
      for (int j = 0; j < CS; ++j) {
        done[j] = (j >= ncol) || !(rr[j] > rtol2 * bn2[j]);
        all = all && done[j];
      }
      if (all) break;
      if (steps >= a.max_steps) {
        unconverged = true;
        break;
      }
      T pq[CS];
#pragma unroll
      for (int j = 0; j < CS; ++j) pq[j] = 0;
      for (int i = threadIdx.x; i < nb; i += kThreads) {
        T qi[CS], pi[CS];
        apply_row<T, CS>(mv, r0, i, delta, p, qi);
        lds_row<T, CS>(p + (size_t)i * CS, pi);
        sts_row<T, CS>(q + (size_t)i * CS, qi);
#pragma unroll
        for (int j = 0; j < CS; ++j) pq[j] += pi[j] * qi[j];
      }
      block_sum<T, CS>(pq, red1, buf1);
      T al[CS], rn[CS];
#pragma unroll
      for (int j = 0; j < CS; ++j) {
        if (!done[j] && !(pq[j] > T(0))) bad = true;
        al[j] = (done[j] || !(pq[j] > T(0))) ? T(0) : rr[j] / pq[j];
        rn[j] = 0;
      }
      for (int i = threadIdx.x; i < nb; i += kThreads) {
        T pi[CS], qi[CS], xi[CS], ri[CS];
        lds_row<T, CS>(p + (size_t)i * CS, pi);
        lds_row<T, CS>(q + (size_t)i * CS, qi);
        lds_row<T, CS>(x + (size_t)i * CS, xi);
        lds_row<T, CS>(r + (size_t)i * CS, ri);
#pragma unroll
        for (int j = 0; j < CS; ++j) {
          xi[j] += al[j] * pi[j];
          ri[j] -= al[j] * qi[j];
          rn[j] += ri[j] * ri[j];
        }
        sts_row<T, CS>(x + (size_t)i * CS, xi);
        sts_row<T, CS>(r + (size_t)i * CS, ri);
      }
      block_sum<T, CS>(rn, red1, buf1);
      // p = r + beta p (own rows; all neighbour reads of p finished before the
      // two reductions above)
      T be[CS];
#pragma unroll
      for (int j = 0; j < CS; ++j) {
        be[j] = (done[j] || !(rr[j] > T(0))) ? T(0) : rn[j] / rr[j];
        if (!done[j]) rr[j] = rn[j];
      }
      for (int i = threadIdx.x; i < nb; i += kThreads) {
        T pi[CS], ri[CS];
        lds_row<T, CS>(p + (size_t)i * CS, pi);
        lds_row<T, CS>(r + (size_t)i * CS, ri);
#pragma unroll
        for (int j = 0; j < CS; ++j) pi[j] = ri[j] + be[j] * pi[j];
        sts_row<T, CS>(p + (size_t)i * CS, pi);
      }
      __syncthreads();
      ++steps;
    }
    steps_all += steps;
    steps_max = max(steps_max, steps);
    if (sol + 1 < a.z) {  // next right-hand side: this solution
      for (int i = threadIdx.x; i < nb; i += kThreads) {
        T xi[CS];
        lds_row<T, CS>(x + (size_t)i * CS, xi);
        sts_row<T, CS>(p + (size_t)i * CS, xi);
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < nb; i += kThreads) {
    T xi[CS];
    lds_row<T, CS>(x + (size_t)i * CS, xi);
#pragma unroll
    for (int j = 0; j < CS; ++j)
      if (j < ncol) Y[(size_t)(r0 + i) * a.ld + j0 + j] = xi[j];
  }
  if (threadIdx.x == 0) {
    atomicAdd(&a.stats->steps_total, (unsigned long long)steps_all);
    atomicMax(&a.stats->steps_max, steps_max);
    if (unconverged) {
      atomicAdd(&a.stats->not_converged, 1);
      atomicOr(a.status, ST_NOT_CONVERGED);
    }
    if (bad) atomicOr(a.status, ST_CG_BREAKDOWN);
  }
}

// ---- standalone SpMM: Y = (L + delta I) P over all rows of all blocks.
// LPR lanes per row, each lane owning 16-byte vectors v = lane, lane+LPR, ...
template <typename T, int LPR>
__global__ void __launch_bounds__(256) k_spmm_vec(int64_t n, MeshView<T> mv,
                                                  const int32_t* __restrict__ blk_row, T delta,
                                                  const T* __restrict__ P, T* __restrict__ Y,
                                                  int c) {
  constexpr int VE = 16 / sizeof(T);
  const int nv = c / VE;
  const int lane = threadIdx.x % LPR;
  const int64_t rows_per_iter = (int64_t)gridDim.x * (blockDim.x / LPR);
  for (int64_t row = (int64_t)blockIdx.x * (blockDim.x / LPR) + threadIdx.x / LPR; row < n;
       row += rows_per_iter) {
    const int64_t base = mv.bptr[__ldg(blk_row + row)];
    const int e0 = __ldg(mv.rowptr + row), e1 = __ldg(mv.rowptr + row + 1);
    const T dd = mv.diag[row] + delta;
    for (int v = lane; v < nv; v += LPR) {
      float4 t = __ldg(reinterpret_cast<const float4*>(P + row * c) + v);
      T* tp = reinterpret_cast<T*>(&t);
      T acc[VE];
#pragma unroll
      for (int j = 0; j < VE; ++j) acc[j] = dd * tp[j];
      for (int e = e0; e < e1; ++e) {
        const int64_t nr = base + __ldg(mv.col + e);
        const T w = mv.wt ? mv.wt[e] : T(1);
        float4 u = __ldg(reinterpret_cast<const float4*>(P + nr * c) + v);
        T* up = reinterpret_cast<T*>(&u);
#pragma unroll
        for (int j = 0; j < VE; ++j) acc[j] -= w * up[j];
      }
      float4 o;
      T* op = reinterpret_cast<T*>(&o);
#pragma unroll
      for (int j = 0; j < VE; ++j) op[j] = acc[j];
      reinterpret_cast<float4*>(Y + row * c)[v] = o;
    }
  }
}

template <typename T>
__global__ void k_spmm_scalar(int64_t n, MeshView<T> mv, const int32_t* __restrict__ blk_row,
                              T delta, const T* __restrict__ P, T* __restrict__ Y, int c) {
  const int64_t total = n * c;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = t / c;
    const int j = (int)(t % c);
    const int64_t base = mv.bptr[blk_row[row]];
    T acc = (mv.diag[row] + delta) * P[row * c + j];
    for (int e = mv.rowptr[row]; e < mv.rowptr[row + 1]; ++e) {
      const T w = mv.wt ? mv.wt[e] : T(1);
      acc -= w * P[(base + mv.col[e]) * c + j];
    }
    Y[row * c + j] = acc;
  }
}


// ---- one column per CTA, latency-optimised (the warm-started chain, and the
// batches of dynamic c, whose growth columns start from random vectors).
// Chronopoulos-Gear CG: one fused reduction of (r, r) and (A r, r) per step and
// two barriers; each thread keeps its rows' x, r, p, s = A p, w = A r in
// registers, only r goes through shared memory for the neighbour reads.
// Rows: i = threadIdx.x + 256 m, m < MAXR.  The rows' pattern (ELL, width
// ELLW) sits in registers for MAXR <= 4 (blocks up to 1,024 rows) and in
// shared memory for larger blocks (SMEM_ELL: padded entries point at a zero
// slot of the shared vector, so every row does ELLW branch-free updates).
template <typename T, int MAXR, int ELLW, bool SMEM_ELL>
__global__ void __launch_bounds__(kThreads) k_cg1(MeshView<T> mv, const T* __restrict__ V,
                                                  T* __restrict__ Y, CgArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T red[2][kWarps][2];
  const int b = a.batch[blockIdx.y];
  if (a.live && !a.live[b]) return;
  const int col = blockIdx.x;
  if (col >= a.cb[b]) return;
  const int r0 = mv.bptr[b];
  const int nb = mv.bptr[b + 1] - r0;
  constexpr int CAP = MAXR * kThreads;            // rows this instantiation holds
  constexpr int RSN = SMEM_ELL ? CAP + 4 : 0;     // shared vector incl. the zero slot
  T* rs = reinterpret_cast<T*>(smem_raw);
  // SMEM_ELL layout after rs: diagonal + delta [CAP], weights [CAP][ELLW]
  // (weighted meshes only), neighbour indices [CAP][ELLW]
  T* sdd = rs + RSN;
  T* swt = sdd + (SMEM_ELL ? CAP : 0);
  uint16_t* snb = reinterpret_cast<uint16_t*>(swt + ((SMEM_ELL && mv.wt) ? (size_t)CAP * ELLW : 0));
  const T delta = (T)a.delta;
  const T rtol2 = (T)(a.rtol * a.rtol);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int RR = SMEM_ELL ? 1 : MAXR;          // rows whose pattern is in registers
  uint16_t nbr[RR][ELLW];
  T wt[RR][ELLW];
  T dd[RR];
  int deg[RR];
#pragma unroll
  for (int m = 0; m < MAXR; ++m) {
    const int i = threadIdx.x + kThreads * m;
    const int q = SMEM_ELL ? 0 : m;
    int dg = 0;
    T d0 = 0;
    uint16_t nl[ELLW];
    T wl[ELLW];
#pragma unroll
    for (int e = 0; e < ELLW; ++e) { nl[e] = SMEM_ELL ? (uint16_t)CAP : 0; wl[e] = 0; }
    if (i < nb) {
      const int e0 = mv.rowptr[r0 + i], e1 = mv.rowptr[r0 + i + 1];
      dg = e1 - e0;
      d0 = mv.diag[r0 + i] + delta;
#pragma unroll
      for (int e = 0; e < ELLW; ++e)
        if (e < dg) {
          nl[e] = mv.col[e0 + e];
          wl[e] = mv.wt ? mv.wt[e0 + e] : T(1);
        }
    }
    if constexpr (SMEM_ELL) {
      sdd[i] = d0;
#pragma unroll
      for (int e = 0; e < ELLW; ++e) {
        snb[(size_t)i * ELLW + e] = nl[e];
        if (mv.wt) swt[(size_t)i * ELLW + e] = wl[e];
      }
    } else {
      deg[q] = dg;
      dd[q] = d0;
#pragma unroll
      for (int e = 0; e < ELLW; ++e) { nbr[q][e] = nl[e]; wt[q][e] = wl[e]; }
    }
  }
  if constexpr (SMEM_ELL) {
    if (threadIdx.x == 0) rs[CAP] = T(0);          // the padded entries' target
  }
  int buf = 0;
  // sum of two per-thread values over the CTA (one barrier, double buffered)
  auto reduce2 = [&](T u, T v, T& su, T& sv) {
    u = warp_sum(u);
    v = warp_sum(v);
    if (lane == 0) { red[buf][w][0] = u; red[buf][w][1] = v; }
    __syncthreads();
    su = 0; sv = 0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) { su += red[buf][q][0]; sv += red[buf][q][1]; }
    buf ^= 1;
  };
  // out_m = (D + delta) v_m - sum C v_nbr, v taken from rs (shared)
  auto apply = [&](const T (&v)[MAXR], T (&out)[MAXR]) {
#pragma unroll
    for (int m = 0; m < MAXR; ++m) {
      if constexpr (SMEM_ELL) {
        const int i = threadIdx.x + kThreads * m;
        T acc = 0;
        if (i < nb) {
          acc = sdd[i] * v[m];
          uint16_t nl[ELLW];
          if constexpr (ELLW == 8) {
            const uint4 q = *reinterpret_cast<const uint4*>(snb + (size_t)i * ELLW);
            const uint16_t* qp = reinterpret_cast<const uint16_t*>(&q);
#pragma unroll
            for (int e = 0; e < 8; ++e) nl[e] = qp[e];
          } else {
#pragma unroll
            for (int e = 0; e < ELLW; ++e) nl[e] = snb[(size_t)i * ELLW + e];
          }
          if (mv.wt) {
#pragma unroll
            for (int e = 0; e < ELLW; ++e) acc -= swt[(size_t)i * ELLW + e] * rs[nl[e]];
          } else {
#pragma unroll
            for (int e = 0; e < ELLW; ++e) acc -= rs[nl[e]];
          }
        }
        out[m] = acc;
      } else {
        T acc = dd[m] * v[m];
#pragma unroll
        for (int e = 0; e < ELLW; ++e)
          if (e < deg[m]) acc -= wt[m][e] * rs[nbr[m][e]];
        out[m] = acc;
      }
    }
  };
  T bvec[MAXR], x[MAXR], r[MAXR], p[MAXR], sv[MAXR], wv[MAXR];
  const int rv = a.vsrc ? mv.bptr[a.vsrc[b]] : r0;   // rows of the right-hand side
#pragma unroll
  for (int m = 0; m < MAXR; ++m) {
    const int i = threadIdx.x + kThreads * m;
    bvec[m] = i < nb ? V[(size_t)(rv + i) * a.ld + col] : T(0);
  }
  int steps_all = 0, steps_max = 0;
  bool unconverged = false, bad = false;
  for (int sol = 0; sol < a.z; ++sol) {
    // initial guess x0 = b (b, b) / (b, A b)
#pragma unroll
    for (int m = 0; m < MAXR; ++m) {
      const int i = threadIdx.x + kThreads * m;
      if (i < nb) rs[i] = bvec[m];
    }
    __syncthreads();
    apply(bvec, wv);
    T bb = 0, bab = 0;
#pragma unroll
    for (int m = 0; m < MAXR; ++m) { bb += bvec[m] * bvec[m]; bab += bvec[m] * wv[m]; }
    T sbb, sbab;
    reduce2(bb, bab, sbb, sbab);
    const T g = sbab > T(0) ? sbb / sbab : T(0);
    const T bn2 = sbb;
#pragma unroll
    for (int m = 0; m < MAXR; ++m) {
      x[m] = g * bvec[m];
      r[m] = bvec[m] - g * wv[m];
    }
    // w0 = A r0 ; gamma = (r, r), delta = (w, r)
#pragma unroll
    for (int m = 0; m < MAXR; ++m) {
      const int i = threadIdx.x + kThreads * m;
      if (i < nb) rs[i] = r[m];
    }
    __syncthreads();
    apply(r, wv);
    T gl = 0, dl = 0;
#pragma unroll
    for (int m = 0; m < MAXR; ++m) { gl += r[m] * r[m]; dl += wv[m] * r[m]; }
    T gam, dlt;
    reduce2(gl, dl, gam, dlt);
    T alpha = dlt > T(0) ? gam / dlt : T(0);
#pragma unroll
    for (int m = 0; m < MAXR; ++m) { p[m] = r[m]; sv[m] = wv[m]; }
    int steps = 0;
    while (gam > rtol2 * bn2) {
      if (steps >= a.max_steps) { unconverged = true; break; }
      if (!(dlt > T(0))) { bad = true; break; }
#pragma unroll
      for (int m = 0; m < MAXR; ++m) {
        x[m] += alpha * p[m];
        r[m] -= alpha * sv[m];
      }
#pragma unroll
      for (int m = 0; m < MAXR; ++m) {
        const int i = threadIdx.x + kThreads * m;
        if (i < nb) rs[i] = r[m];
      }
      __syncthreads();
      apply(r, wv);
      gl = 0; dl = 0;
#pragma unroll
      for (int m = 0; m < MAXR; ++m) { gl += r[m] * r[m]; dl += wv[m] * r[m]; }
      T gnew, dnew;
      reduce2(gl, dl, gnew, dnew);
      ++steps;
      if (!(gnew > rtol2 * bn2)) { gam = gnew; break; }
      const T beta = gnew / gam;
      const T den = dnew - beta * gnew / alpha;
      alpha = den > T(0) ? gnew / den : T(0);
      if (!(den > T(0))) bad = true;
      gam = gnew;
      dlt = den;
#pragma unroll
      for (int m = 0; m < MAXR; ++m) {
        p[m] = r[m] + beta * p[m];
        sv[m] = wv[m] + beta * sv[m];
      }
    }
    steps_all += steps;
    steps_max = max(steps_max, steps);
#pragma unroll
    for (int m = 0; m < MAXR; ++m) bvec[m] = x[m];   // next right-hand side (z > 1)
    __syncthreads();  // rs is rewritten by the next solve
  }
#pragma unroll
  for (int m = 0; m < MAXR; ++m) {
    const int i = threadIdx.x + kThreads * m;
    if (i < nb) Y[(size_t)(r0 + i) * a.ld + col] = x[m];
  }
  if (threadIdx.x == 0) {
    atomicAdd(&a.stats->steps_total, (unsigned long long)steps_all);
    atomicMax(&a.stats->steps_max, steps_max);
    if (unconverged) {
      atomicAdd(&a.stats->not_converged, 1);
      atomicOr(a.status, ST_NOT_CONVERGED);
    }
    if (bad) atomicOr(a.status, ST_CG_BREAKDOWN);
  }
}

// Shared memory of a k_cg1 launch: the shared vector, and for SMEM_ELL the
// diagonal, the weights (weighted meshes) and the neighbour indices.
template <typename T, int MAXR, int ELLW, bool SMEM_ELL>
size_t cg1_smem(int max_nb, bool weighted) {
  if (!SMEM_ELL) return (size_t)max_nb * sizeof(T);
  const size_t cap = (size_t)MAXR * kThreads;
  return (cap + 4 + cap) * sizeof(T) + (weighted ? cap * ELLW * sizeof(T) : 0) +
         cap * ELLW * sizeof(uint16_t);
}

template <typename T, int MAXR, int ELLW, bool SMEM_ELL>
int launch_cg1_t(const MeshView<T>& mv, const T* V, T* Y, const CgArgs& a, int max_nb, int c_max,
                 cudaStream_t s) {
  dim3 grid(c_max, a.nbatch);
  const size_t smem = cg1_smem<T, MAXR, ELLW, SMEM_ELL>(max_nb, mv.wt != nullptr);
  if (smem > 220 * 1024) return BSP_ERR_INVALID_ARG;
  k_cg1<T, MAXR, ELLW, SMEM_ELL><<<grid, kThreads, smem, s>>>(mv, V, Y, a);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

// One-column-per-CTA CG for rows up to 4,096 and degrees up to 16: the
// instantiation by rows per thread (1, 4 in registers; 8, 16 in shared memory).
template <typename T>
int launch_cg1_rows(const MeshView<T>& mv, const T* V, T* Y, const CgArgs& a, int max_nb,
                    int c_max, cudaStream_t s) {
  const int mr = (max_nb + kThreads - 1) / kThreads;
  const bool w8 = a.max_deg <= 8;
  if (mr <= 1) return w8 ? launch_cg1_t<T, 1, 8, false>(mv, V, Y, a, max_nb, c_max, s)
                         : launch_cg1_t<T, 1, 16, false>(mv, V, Y, a, max_nb, c_max, s);
  if (mr <= 4) return w8 ? launch_cg1_t<T, 4, 8, false>(mv, V, Y, a, max_nb, c_max, s)
                         : launch_cg1_t<T, 4, 16, false>(mv, V, Y, a, max_nb, c_max, s);
  if (mr <= 8) return w8 ? launch_cg1_t<T, 8, 8, true>(mv, V, Y, a, max_nb, c_max, s)
                         : launch_cg1_t<T, 8, 16, true>(mv, V, Y, a, max_nb, c_max, s);
  return w8 ? launch_cg1_t<T, 16, 8, true>(mv, V, Y, a, max_nb, c_max, s)
            : launch_cg1_t<T, 16, 16, true>(mv, V, Y, a, max_nb, c_max, s);
}

template <typename T, int CS>
int launch_cg_cs(const MeshView<T>& mv, const T* V, T* Y, const CgArgs& a, int max_nb, int c_max,
                 cudaStream_t s) {
  size_t smem = (size_t)4 * max_nb * CS * sizeof(T);
  if (smem > 227 * 1024) return BSP_ERR_INVALID_ARG;
  dim3 grid((c_max + CS - 1) / CS, a.nbatch);
  prof_begin(KC_CG, s);
  k_cg<T, CS><<<grid, kThreads, smem, s>>>(mv, V, Y, a);
  prof_end(KC_CG, s);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

}  // namespace

bool g_disable_cg1 = false;

// Opt every CG instantiation in to the full 227 KB of dynamic shared memory.
void configure_cg_kernels() {
  set_max_dynamic_smem(k_cg<float, 1>);
  set_max_dynamic_smem(k_cg<float, 2>);
  set_max_dynamic_smem(k_cg<float, 4>);
  set_max_dynamic_smem(k_cg<float, 8>);
  set_max_dynamic_smem(k_cg<double, 1>);
  set_max_dynamic_smem(k_cg<double, 2>);
  set_max_dynamic_smem(k_cg<double, 4>);
  set_max_dynamic_smem(k_cg<double, 8>);
  set_max_dynamic_smem(k_cg1<float, 8, 8, true>);
  set_max_dynamic_smem(k_cg1<float, 8, 16, true>);
  set_max_dynamic_smem(k_cg1<float, 16, 8, true>);
  set_max_dynamic_smem(k_cg1<float, 16, 16, true>);
  set_max_dynamic_smem(k_cg1<double, 8, 8, true>);
  set_max_dynamic_smem(k_cg1<double, 8, 16, true>);
  set_max_dynamic_smem(k_cg1<double, 16, 8, true>);
  set_max_dynamic_smem(k_cg1<double, 16, 16, true>);
}

// Whether the one-column-per-CTA CG holds a block of max_nb rows (its shared
// memory within the opt-in limit).
bool cg1_fits(int max_nb, int max_deg, int real_bytes, bool weighted) {
  if (max_deg <= 0 || max_deg > 16 || max_nb > 16 * kThreads) return false;
  const int mr = (max_nb + kThreads - 1) / kThreads;
  const size_t rows = mr <= 1 ? 1 : mr <= 4 ? 4 : mr <= 8 ? 8 : 16;
  if (rows <= 4) return true;
  const size_t cap = rows * kThreads, ellw = max_deg <= 8 ? 8 : 16;
  const size_t bytes = (2 * cap + 4) * real_bytes + (weighted ? cap * ellw * real_bytes : 0) +
                       cap * ellw * 2;
  return bytes <= 220 * 1024;
}

// Size bucket of a block for the batched CG: up to 256, 512, 1,024, 2,048
// and 4,096 rows (the team CG's team sizes), -1 when the block is too large.
int cg_bucket(int nb) {
  return nb <= 256 ? 0 : nb <= 512 ? 1 : nb <= 1024 ? 2 : nb <= 2048 ? 3 : nb <= 4096 ? 4 : -1;
}

// CG over a batch sorted by size bucket (bucket_off[q] .. bucket_off[q + 1] of
// a.batch holds bucket q): one launch per non-empty bucket, each sized for
// its own largest block; the team kernel where its shared memory fits, else
// one column per CTA.  With `fork`, the buckets after the first run on side
// streams concurrently with it (each launch ends on its slowest column; side
// by side their tails overlap), joined back into s before the return.
template <typename T>
int launch_cg_buckets(const MeshView<T>& mv, const T* V, T* Y, const CgArgs& a,
                      const int* bucket_off, const int* bucket_rows, int c_max, cudaStream_t s,
                      const CgFork* fork) {
  if (!(a.max_deg > 0 && a.max_deg <= 16)) return BSP_ERR_INVALID_ARG;
  prof_begin(KC_CG, s);
  int rc = BSP_OK;
  int used[kCgBuckets] = {};
  bool forked = false;
  for (int q = 0, side = 0; q < kCgBuckets && rc == BSP_OK; ++q) {
    const int n = bucket_off[q + 1] - bucket_off[q];
    if (n <= 0) continue;
    cudaStream_t st = s;
    if (fork && side > 0) {
      if (!forked) {
        if (cudaEventRecord(fork->fork, s) != cudaSuccess) return BSP_ERR_CUDA;
        forked = true;
      }
      st = fork->aux[side - 1];
      if (cudaStreamWaitEvent(st, fork->fork, 0) != cudaSuccess) return BSP_ERR_CUDA;
      used[side - 1] = 1;
    }
    ++side;
    CgArgs sub = a;
    sub.batch = a.batch + bucket_off[q];
    sub.nbatch = n;
    rc = cgt_fits(bucket_rows[q], a.max_deg, sizeof(T), mv.wt != nullptr)
             ? launch_cgt<T>(mv, V, Y, sub, bucket_rows[q], c_max, st)
             : launch_cg1_rows<T>(mv, V, Y, sub, bucket_rows[q], c_max, st);
  }
  for (int k = 0; k < kCgBuckets - 1; ++k)
    if (used[k]) {
      if (cudaEventRecord(fork->join[k], fork->aux[k]) != cudaSuccess ||
          cudaStreamWaitEvent(s, fork->join[k], 0) != cudaSuccess)
        return BSP_ERR_CUDA;
    }
  prof_end(KC_CG, s);
  return rc;
}

template <typename T>
int cg_smem_bytes(int cs, int max_nb) {
  return 4 * max_nb * cs * (int)sizeof(T);
}

template <typename T>
int launch_cg(const MeshView<T>& mv, const T* V, T* Y, const CgArgs& a, int cs, int max_nb,
              int c_max, cudaStream_t s) {
  // one column per CTA when the pattern fits its ELL forms
  if (cs == 1 && cg1_fits(max_nb, a.max_deg, sizeof(T), mv.wt != nullptr) && !g_disable_cg1) {
    prof_begin(KC_CG, s);
    const int rc = launch_cg1_rows<T>(mv, V, Y, a, max_nb, c_max, s);
    prof_end(KC_CG, s);
    return rc;
  }
  switch (cs) {
    case 1: return launch_cg_cs<T, 1>(mv, V, Y, a, max_nb, c_max, s);
    case 2: return launch_cg_cs<T, 2>(mv, V, Y, a, max_nb, c_max, s);
    case 4: return launch_cg_cs<T, 4>(mv, V, Y, a, max_nb, c_max, s);
    case 8: return launch_cg_cs<T, 8>(mv, V, Y, a, max_nb, c_max, s);
    default: return BSP_ERR_INVALID_ARG;
  }
}

template <typename T>
void launch_spmm(int64_t n, const MeshView<T>& mv, const int32_t* blk_row, T delta, const T* P,
                 T* Y, int c, cudaStream_t s) {
  constexpr int VE = 16 / sizeof(T);
  const bool vec = (c % VE == 0) && ((uintptr_t)P % 16 == 0) && ((uintptr_t)Y % 16 == 0);
  prof_begin(KC_SPMM, s);
  if (vec) {
    int nv = c / VE;
    int lpr = 1;
    while (lpr < nv && lpr < 32) lpr <<= 1;
    int rows_per_cta = 256 / lpr;
    int64_t g = (n + rows_per_cta - 1) / rows_per_cta;
    if (g > 152 * 64) g = 152 * 64;
    unsigned grid = (unsigned)(g < 1 ? 1 : g);
    switch (lpr) {
      case 1: k_spmm_vec<T, 1><<<grid, 256, 0, s>>>(n, mv, blk_row, delta, P, Y, c); break;
      case 2: k_spmm_vec<T, 2><<<grid, 256, 0, s>>>(n, mv, blk_row, delta, P, Y, c); break;
      case 4: k_spmm_vec<T, 4><<<grid, 256, 0, s>>>(n, mv, blk_row, delta, P, Y, c); break;
      case 8: k_spmm_vec<T, 8><<<grid, 256, 0, s>>>(n, mv, blk_row, delta, P, Y, c); break;
      case 16: k_spmm_vec<T, 16><<<grid, 256, 0, s>>>(n, mv, blk_row, delta, P, Y, c); break;
      default: k_spmm_vec<T, 32><<<grid, 256, 0, s>>>(n, mv, blk_row, delta, P, Y, c); break;
    }
  } else {
    int64_t g = (n * c + 255) / 256;
    if (g > 152 * 64) g = 152 * 64;
    k_spmm_scalar<T><<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(n, mv, blk_row, delta, P, Y, c);
  }
  prof_end(KC_SPMM, s);
}

template int cg_smem_bytes<float>(int, int);
template int cg_smem_bytes<double>(int, int);
template int launch_cg<float>(const MeshView<float>&, const float*, float*, const CgArgs&, int,
                              int, int, cudaStream_t);
template int launch_cg<double>(const MeshView<double>&, const double*, double*, const CgArgs&,
                               int, int, int, cudaStream_t);
template int launch_cg_buckets<float>(const MeshView<float>&, const float*, float*,
                                      const CgArgs&, const int*, const int*, int, cudaStream_t,
                                      const CgFork*);
template int launch_cg_buckets<double>(const MeshView<double>&, const double*, double*,
                                       const CgArgs&, const int*, const int*, int, cudaStream_t,
                                       const CgFork*);
template void launch_spmm<float>(int64_t, const MeshView<float>&, const int32_t*, float,
                                 const float*, float*, int, cudaStream_t);
template void launch_spmm<double>(int64_t, const MeshView<double>&, const int32_t*, double,
                                  const double*, double*, int, cudaStream_t);

}  // namespace bsp
