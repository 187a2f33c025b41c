// Fused Onorm: CholeskyQR2 of every block of a batch in one cluster launch
// (Sec. 4, Onorm; same Q as Householder QR in exact arithmetic).
//
// One cluster of P <= 8 CTAs per block: CTA p holds a panel of the block's
// rows in shared memory for both passes; partial Grams go through L2, a
// distributed fixed-order reduction forms the c x c Gram, and every CTA
// factorizes it itself, so the CTAs only meet at cluster barriers.  The
// Cholesky runs in one warp in registers (FP32) or, for an FP64-accumulated
// first pass, block-wide in FP64; Q = Y R^-1 is a row-wise forward
// substitution on the resident panel.
#include "bsp_dense_dev.cuh"

namespace bsp {
namespace {

using namespace dev;

// Scratch next to the panel: the Gram half-sums (cpad^2) and the Cholesky's
// double-buffered block rows (8 (CP + 4)); a multiple of 4 keeps the
// following arrays aligned.
__host__ __device__ inline int fused_half_elems(int cpad, int cp) {
  const int a = cpad * cpad, b = 8 * (cp + 4);
  return ((a > b ? a : b) + 3) & ~3;
}

// One block step of chol_cols (rows KB..KB+3).  A template recursion over
// KB keeps every register index a compile-time constant (an unrolled loop
// of this size is not unrolled fully, and the column would go to local memory).
template <int CP, int KB>
BSP_DEV void chol_step(float (&a)[CP], int c, int j, float* lbuf, bool& bad) {
  constexpr int B = 4;
  constexpr int LD = CP + 4;
  if (KB < c) {   // uniform over the CP threads
    float* buf = lbuf + ((KB / B) & 1) * (B * LD);
#pragma unroll
    for (int q = 0; q < B; ++q) buf[q * LD + j] = a[KB + q];
    asm volatile("bar.sync 1, %0;" ::"r"(CP) : "memory");
    float r4[B][B], inv[B];
#pragma unroll
    for (int q = 0; q < B; ++q) {
      float sq = buf[q * LD + KB + q];
#pragma unroll
      for (int p = 0; p < q; ++p) sq -= r4[p][q] * r4[p][q];
      const bool ok = sq > 0.f && isfinite(sq);
      bad = bad || !ok;
      inv[q] = ok ? rsqrtf(sq) : 1.f;
      r4[q][q] = ok ? sq * inv[q] : 1.f;
#pragma unroll
      for (int r = q + 1; r < B; ++r) {
        float t = buf[q * LD + KB + r];
#pragma unroll
        for (int p = 0; p < q; ++p) t -= r4[p][q] * r4[p][r];
        r4[q][r] = t * inv[q];
      }
    }
    float l[B], w[B];
#pragma unroll
    for (int q = 0; q < B; ++q) {
      float t = a[KB + q];
#pragma unroll
      for (int p = 0; p < q; ++p) t -= r4[p][q] * l[p];
      l[q] = t * inv[q];
    }
#pragma unroll
    for (int q = B - 1; q >= 0; --q) {
      float t = l[q];
#pragma unroll
      for (int p = q + 1; p < B; ++p) t -= r4[q][p] * w[p];
      w[q] = t * inv[q];
    }
#pragma unroll
    for (int q = 0; q < B; ++q) a[KB + q] = l[q];
#pragma unroll
    for (int i = KB + B; i < CP; ++i) {
      float t = a[i];
#pragma unroll
      for (int q = 0; q < B; ++q) t -= buf[q * LD + i] * w[q];
      a[i] = t;
    }
  }
  if constexpr (KB + 4 < CP) chol_step<CP, KB + 4>(a, c, j, lbuf, bad);
}
// Cholesky of the Jacobi-scaled Gram in FP32 by CP threads (CP/32 warps),
// blocked by 4: thread j keeps column j of the symmetric A in registers.
// Block step kb publishes rows kb..kb+3 (a_{kb+q, j} from thread j) in a
// double-buffered shared area, one named barrier over the CP threads; then
// every thread factorises the 4 x 4 pivot block D = R4^T R4 itself, forms its
// entries of R's rows kb..kb+3, l = R4^-T p_j (p_j its published values), and
// applies the Schur update a_ij -= p_i^T D^-1 p_j = sum_q p_i[q] w_j[q] with
// w_j = D^-1 p_j (i >= kb + 4).  Entries below the diagonal of column j are
// never read back or written out.  Rows/columns >= c act as the identity.
// Writes R (upper, stride CP) to Rr and 1/R_jj to rinv.  Called by threads
// 0..CP-1 only; lbuf holds 8 (CP + 4) floats.
template <typename TG, int CP>
BSP_DEV void chol_cols(const TG* g, int c, int cpad, const float* dsc, float* Rr, float* rinv,
                       float* lbuf, int* fail) {
  constexpr int B = 4;
  constexpr int LD = CP + 4;
  const int j = threadIdx.x;
  float a[CP];
#pragma unroll
  for (int i = 0; i < CP; ++i) {
    float v = i == j ? 1.f : 0.f;
    if (i < c && j < c) v = (float)g[min(i, j) * cpad + max(i, j)] * dsc[i] * dsc[j];
    a[i] = v;
  }
  bool bad = false;
  chol_step<CP, 0>(a, c, j, lbuf, bad);
#pragma unroll
  for (int i = 0; i < CP; ++i) Rr[i * CP + j] = i <= j ? a[i] : 0.f;
  rinv[j] = 1.f / Rr[j * CP + j];
  if (bad && j == 0) *fail = 1;
}


// Block-level Cholesky (any TA), for the FP64-accumulated pass: the balanced
// factorization of chol_inverse without the inverse; writes R (T, stride CP,
// identity past c) to Rr and 1/R_jj to rinv.  All threads; ends with a barrier.
template <typename T, typename TA, typename TG, int CP>
BSP_DEV void chol_block(const TG* g, int c, int cpad, TA* A, TA* dsc, TA* lrow, T* Rr, T* rinv,
                        int* fail) {
  for (int t = threadIdx.x; t < CP * CP; t += blockDim.x) Rr[t] = T(0);
  for (int i = threadIdx.x >> 5; i < c; i += blockDim.x >> 5)
    for (int jj = (threadIdx.x & 31) + i; jj < c; jj += 32)
      A[i * cpad + jj] = (TA)g[i * cpad + jj] * dsc[i] * dsc[jj];
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
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
      if (j0 < i) j0 += ((i - j0 + 15) >> 4) << 4;
      for (int jj = j0; jj < c; jj += 16) A[i * cpad + jj] -= li * lrow[jj];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < CP; i += blockDim.x) {
    if (i >= c) Rr[i * CP + i] = T(1);
    rinv[i] = T(1) / (i < c ? Rr[i * CP + i] : T(1));
  }
  __syncthreads();
}

// Forward substitution Q R = Y D on the panel in shared memory: the Onorm
// output Q = Y D R_s^-1 = Y R^-1 without forming R^-1.  Blocked over 16
// columns: for column block J, a GEMM-style update with all threads
// (rows x 16 outputs, 8 per thread), then a per-row 16 x 16 triangular solve.
// All threads; ends with a barrier.
template <typename T, int CP>
BSP_DEV void trsm_rows(T* S, int rows, int cpad, int ldS, int c, const T* Rr, const T* rinv,
                       const float* dscf, const double* dscd) {
  // scale the columns by D (zero past c)
  for (int r = threadIdx.x >> 5; r < rows; r += blockDim.x >> 5)
    for (int jj = threadIdx.x & 31; jj < cpad; jj += 32)
      S[r * ldS + jj] = jj < c ? S[r * ldS + jj] * (dscd ? (T)dscd[jj] : (T)dscf[jj]) : T(0);
  __syncthreads();
#pragma unroll 1
  for (int J = 0; J < CP / 16; ++J) {
    const int j0 = 16 * J;
    if (j0 >= cpad) break;
    if (J > 0) {
      // S[r, j0 + 8h .. +7] -= S[r, 0:j0] R[0:j0, j0 + 8h .. +7]
      for (int t = threadIdx.x; t < rows * 2; t += blockDim.x) {
        const int r = t >> 1, h = t & 1;
        T acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = 0;
        for (int l = 0; l < j0; ++l) {
          const T sv = S[r * ldS + l];
#pragma unroll
          for (int q = 0; q < 8; ++q) acc[q] += sv * Rr[l * CP + j0 + 8 * h + q];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (j0 + 8 * h + q < cpad) S[r * ldS + j0 + 8 * h + q] -= acc[q];
      }
      __syncthreads();
    }
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
      T q[16];
      T* row = S + r * ldS + j0;   // 16-byte aligned: ldS and j0 are multiples of 4
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        T t4[4] = {T(0), T(0), T(0), T(0)};
        if (j0 + 4 * v < cpad) ld4(row + 4 * v, t4);
#pragma unroll
        for (int e = 0; e < 4; ++e) q[4 * v + e] = t4[e];
      }
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        T s0 = q[jj];
#pragma unroll
        for (int l = 0; l < jj; ++l) s0 -= q[l] * Rr[(j0 + l) * CP + j0 + jj];
        q[jj] = s0 * rinv[j0 + jj];
      }
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if (j0 + 4 * v < cpad) st4(row + 4 * v, q + 4 * v);
    }
    __syncthreads();
  }
}

// Stage rows [row0, row0 + nr) x [0, c) of A (stride ld) into S [rows x cpad]
// (row stride ldS), zero padded.  Aligned rows go by 16-byte asynchronous
// copies, all in flight at once (consecutive threads take consecutive pieces
// of a row: coalesced); the caller's barrier follows the final wait.
template <typename T>
BSP_DEV void stage_rows(const T* __restrict__ A, int ld, int row0, int nr, int c, int cpad,
                        int rows, T* S, int ldS) {
  constexpr int VE = 16 / sizeof(T);
  const bool vec = (ld % VE == 0) && (cpad % VE == 0) && (c % VE == 0) &&
                   ((uintptr_t)A % 16 == 0);
  if (vec) {
    const int per = cpad / VE;
    for (int t = threadIdx.x; t < rows * per; t += blockDim.x) {
      const int r = t / per, v = t - r * per;
      T* dst = S + r * ldS + v * VE;
      if (r < nr && v * VE < c) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(dst)),
                     "l"(A + (size_t)(row0 + r) * ld + v * VE));
      } else {
        *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = threadIdx.x >> 5; r < rows; r += nw) {
      T* dst = S + r * ldS;
      const T* src = A + (size_t)(row0 + r) * ld;
      for (int j = lane; j < cpad; j += 32) dst[j] = (r < nr && j < c) ? src[j] : T(0);
    }
  }
}

// Upper-triangle Gram of the panel S (rows x cpad) into out (TA, cpad x
// cpad): tiles of 4 x 4, the rows split in two halves so that every thread
// has work; the halves are added through shared memory scratch `half` (T).
template <typename T, typename TA>
BSP_DEV void panel_gram_split(const T* S, int rows, int cpad, int ldS, T* half, TA* out) {
  const int nt = cpad / 4;
  const int nup = nt * (nt + 1) / 2;
  const int items = 2 * nup;
  const int hr = rows / 2;   // rows is a multiple of 4
  T acc[2][4][4];
  int tiles[2] = {-1, -1};
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int it = threadIdx.x + q * blockDim.x;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[q][i][j] = 0;
    if (it >= items) continue;
    const int h = it >= nup ? 1 : 0;
    int u = it - h * nup;
    // upper tile u -> (ti, tj), row-major over ti <= tj
    int ti = 0;
    while (u >= nt - ti) { u -= nt - ti; ++ti; }
    const int tj = ti + u;
    tiles[q] = (ti * nt + tj) * 2 + h;
#pragma unroll 4
    for (int r = h * hr; r < (h + 1) * hr; ++r) {
      T a4[4], b4[4];
      ld4(S + r * ldS + 4 * ti, a4);
      ld4(S + r * ldS + 4 * tj, b4);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[q][i][j] += a4[i] * b4[j];
    }
  }
  // second halves park their sums in `half`, first halves add them
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (tiles[q] < 0 || (tiles[q] & 1) == 0) continue;
    const int t = tiles[q] >> 1, ti = t / nt, tj = t - ti * nt;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) half[(4 * ti + i) * cpad + 4 * tj + j] = acc[q][i][j];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (tiles[q] < 0 || (tiles[q] & 1) == 1) continue;
    const int t = tiles[q] >> 1, ti = t / nt, tj = t - ti * nt;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int e = (4 * ti + i) * cpad + 4 * tj + j;
        out[e] = (TA)acc[q][i][j] + (TA)half[e];
      }
  }
}

// CholeskyQR2 of one block per cluster of P CTAs (c <= 64).  CTA p keeps rows
// [p RP, (p+1) RP) of Y in shared memory for both passes; partial Grams go
// through L2 (Gpart), a distributed fixed-order reduction forms G (Gfin), and
// every CTA factorizes G itself (identical inputs, identical results), so the
// only inter-CTA steps are cluster barriers.  Every pass accumulates in TA;
// when TA is double the first pass factorizes in FP64 (block-level); the
// second pass's Gram is I + O(kappa u), whose Cholesky runs in registers in
// FP32 like every pass of the FP32 mode.  Q = Y R^-1 by row-wise forward substitution.
template <typename T, typename TA, int CP>
__global__ void __launch_bounds__(kDT) k_cholqr2_cluster(DenseArgs a, const T* Y, T* Q, int P,
                                                         int rp_max, TA* Gpart, TA* Gfin,
                                                         int passes) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int slot = blockIdx.y;
  const int b = a.batch[slot];
  if (a.live && !a.live[b]) return;
  const int c = a.cb[b];
  const int cpad = pad4(a.cmax);
  const int p = blockIdx.x;
  const int r0 = a.bptr[b], nb = a.bptr[b + 1] - r0;
  const int RP = (nb + P - 1) / P;
  const int row0 = p * RP;
  const int nr = max(0, min(RP, nb - row0));
  const int ldS = cpad + 4;                              // padded: conflict-free row-parallel access
  T* S = reinterpret_cast<T*>(smem_raw);                 // rp_max x ldS
  T* half = S + rp_max * ldS;                            // scratch: Gram halves, pivot row
  T* Rr = half + fused_half_elems(cpad, CP);             // CP x CP
  T* rinv = Rr + CP * CP;                                // CP
  TA* dsc = reinterpret_cast<TA*>(rinv + CP);            // cpad (scaling), then pivot row
  TA* A = dsc + 2 * cpad;                                // cpad x cpad (FP64 pass only)
  float* dscf = reinterpret_cast<float*>(A + cpad * cpad);
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  stage_rows(Y, a.ld, r0 + row0, nr, c, cpad, rp_max, S, ldS);
  __syncthreads();
  const size_t cc = (size_t)cpad * cpad;
  TA* gf = Gfin + (size_t)slot * cc;
  for (int pass = 0; pass < passes; ++pass) {
    panel_gram_split<T, TA>(S, rp_max, cpad, ldS, half, Gpart + ((size_t)slot * P + p) * cc);
    cluster_barrier();
    for (int e = p * blockDim.x + threadIdx.x; e < cpad * cpad; e += P * blockDim.x) {
      const int i = e / cpad, jj = e - i * cpad;
      if (i > jj) continue;
      TA sum = 0;
      for (int q = 0; q < P; ++q) sum += Gpart[((size_t)slot * P + q) * cc + e];
      gf[e] = sum;
    }
    cluster_barrier();
    // Jacobi scaling d_i = G_ii^-1/2
    for (int t = threadIdx.x; t < cpad; t += blockDim.x) {
      TA v = t < c ? gf[t * cpad + t] : TA(1);
      if (!(v > TA(0)) || !isfinite((double)v)) {
        fail = 1;
        v = TA(1);
      }
      dsc[t] = TA(1) / sqrt(v);
      dscf[t] = (float)dsc[t];
    }
    __syncthreads();
    if constexpr (sizeof(T) == 8) {
      chol_block<T, TA, TA, CP>(gf, c, cpad, A, dsc, dsc + cpad, Rr, rinv, &fail);
    } else {
      if (sizeof(TA) == 8 && pass == 0) {   // MIXED: the first pass factorises in FP64
        chol_block<T, TA, TA, CP>(gf, c, cpad, A, dsc, dsc + cpad, Rr, rinv, &fail);
      } else {
        if (threadIdx.x < CP)
          chol_cols<TA, CP>(gf, c, cpad, dscf, Rr, rinv, reinterpret_cast<float*>(half), &fail);
        __syncthreads();
      }
    }
    if (fail) {  // uniform: identity factor, flagged below
      for (int t = threadIdx.x; t < CP * CP; t += blockDim.x) Rr[t] = (t / CP == t % CP) ? T(1) : T(0);
      for (int t = threadIdx.x; t < CP; t += blockDim.x) rinv[t] = T(1);
      for (int t = threadIdx.x; t < cpad; t += blockDim.x) { dsc[t] = TA(1); dscf[t] = 1.f; }
      __syncthreads();
    }
    trsm_rows<T, CP>(S, rp_max, cpad, ldS, c, Rr, rinv, dscf,
                     sizeof(T) == 8 ? reinterpret_cast<const double*>(dsc) : nullptr);
    cluster_barrier();  // every CTA has read Gfin before the next pass rewrites it
  }
  for (int i = threadIdx.x >> 5; i < nr; i += blockDim.x >> 5)
    for (int jj = threadIdx.x & 31; jj < c; jj += 32)
      Q[(size_t)(r0 + row0 + i) * a.ld + jj] = S[i * ldS + jj];
  if (fail && threadIdx.x == 0 && p == 0) atomicOr(a.status, ST_NUMERICAL);
}

template <typename T, typename TA>
size_t fused_smem(int rp_max, int cpad) {
  const int cp = chol_cp(cpad);
  return (size_t)(rp_max * (cpad + 4) + fused_half_elems(cpad, cp) + cp * cp + cp) * sizeof(T) +
         (size_t)(2 * cpad + cpad * cpad) * sizeof(TA) + (size_t)cpad * sizeof(float) + 16;
}


}  // namespace

template <typename T, typename TA>
int launch_cholqr2_fused(const DenseArgs& a, const T* Y, T* Q, TA* Gp, int maxch, cudaStream_t s,
                         int passes) {
  const int cpad = pad4(a.cmax);
  int P = (a.max_nb + 127) / 128;
  P = P < 1 ? 1 : (P > 8 ? 8 : P);
  const int rp_max = pad4((a.max_nb + P - 1) / P);
  const size_t sm = fused_smem<T, TA>(rp_max, cpad);
  if (cpad > 64 || rp_max > 256 || P > maxch || sm > 200 * 1024) return BSP_ERR_INVALID_ARG;
  TA* Gpart = Gp;
  TA* Gfin = Gp + (size_t)a.nbatch * maxch * cpad * cpad;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P, a.nbatch, 1);
  cfg.blockDim = dim3(kDT, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  prof_begin(KC_CHOL, s);
  cudaError_t e = cpad <= 32
      ? cudaLaunchKernelEx(&cfg, k_cholqr2_cluster<T, TA, 32>, a, Y, Q, P, rp_max, Gpart, Gfin, passes)
      : cudaLaunchKernelEx(&cfg, k_cholqr2_cluster<T, TA, 64>, a, Y, Q, P, rp_max, Gpart, Gfin, passes);
  prof_end(KC_CHOL, s);
  return e == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

void configure_fused_kernels() {
  set_max_dynamic_smem(k_cholqr2_cluster<float, float, 32>);
  set_max_dynamic_smem(k_cholqr2_cluster<float, float, 64>);
  set_max_dynamic_smem(k_cholqr2_cluster<float, double, 32>);
  set_max_dynamic_smem(k_cholqr2_cluster<float, double, 64>);
  set_max_dynamic_smem(k_cholqr2_cluster<double, double, 32>);
  set_max_dynamic_smem(k_cholqr2_cluster<double, double, 64>);
}

template int launch_cholqr2_fused<float, float>(const DenseArgs&, const float*, float*, float*, int, cudaStream_t, int);
template int launch_cholqr2_fused<float, double>(const DenseArgs&, const float*, float*, double*, int, cudaStream_t, int);
template int launch_cholqr2_fused<double, double>(const DenseArgs&, const double*, double*,
                                                  double*, int, cudaStream_t, int);

}  // namespace bsp
