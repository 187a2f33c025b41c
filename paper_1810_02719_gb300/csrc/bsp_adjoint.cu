// Adjoint of the block low-pass filter x -> U U^T x (the coarse denoising
// filter of Sec. 7.2) with respect to the coordinates and to per-edge weights
// of L(w) = D(w) - C(w), through t_max unrolled steps of Algorithm 1 (Sec. 4)
// whose start is detached.  Not in the paper.
//
// The loss depends on U only through span(U), and each step's span only
// through the previous span, so with Y_t = S V_{t-1}, Y_t = V_t R_t and the
// incoming gradient Vbar_t of V_t:
//   Ybar_t   = (Vbar_t - V_t (V_t^T Vbar_t)) R_t^-T        (QR adjoint, span form)
//   Lambda_t = S Ybar_t                                    (one more solve per step)
//   dL/dA    = -Lambda_t Y_t^T, A = L(w) + delta I          (solve adjoint)
//   dL/dw_e += -sum_cols (Lambda_t[i] - Lambda_t[j]) (Y_t[i] - Y_t[j])   for e = (i, j)
//   Vbar_{t-1} = Lambda_t
// starting from Vbar_T = G (X^T V_T) + X (G^T V_T) for dL/dX^ = G; and
// dL/dX = U U^T G.  Kernels here do the thin products and the row updates;
// the solves reuse the CG kernels and the c x c products the panel kernels.
#include "bsp_dense_dev.cuh"

namespace bsp {
namespace {

using namespace dev;
constexpr int kAT = 256;
constexpr int kMaxC = 128;  // thin-product row width (the filter itself takes c <= 64)

// out[slot][d][j] = sum_i A[verts[r0 + i]][d] * V[r0 + i][j], d < 3 (one CTA per block)
template <typename T, typename TA>
__global__ void __launch_bounds__(kAT) k_thin_cross(const int32_t* batch, const int32_t* bptr,
                                                    const int32_t* verts, const T* __restrict__ A,
                                                    const T* __restrict__ V, int ld, int c,
                                                    T* __restrict__ out) {
  __shared__ TA part[kAT / 32][3 * 32];
  const int slot = blockIdx.x;
  const int b = batch[slot];
  const int r0 = bptr[b], nb = bptr[b + 1] - r0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int q = 0; q * 32 < c; ++q) {
    const int j = q * 32 + lane;
    TA e0 = 0, e1 = 0, e2 = 0;
    for (int i = w; i < nb; i += kAT / 32) {
      const T v = j < c ? V[(size_t)(r0 + i) * ld + j] : T(0);
      const T* a = A + (size_t)verts[r0 + i] * 3;
      e0 += (TA)(v * a[0]);
      e1 += (TA)(v * a[1]);
      e2 += (TA)(v * a[2]);
    }
    part[w][3 * lane] = e0;
    part[w][3 * lane + 1] = e1;
    part[w][3 * lane + 2] = e2;
    __syncthreads();
    if (threadIdx.x < 96) {
      TA s = 0;
      for (int ww = 0; ww < kAT / 32; ++ww) s += part[ww][threadIdx.x];
      const int jj = q * 32 + threadIdx.x / 3, d = threadIdx.x % 3;
      if (jj < c) out[((size_t)slot * 3 + d) * kMaxC + jj] = (T)s;
    }
    __syncthreads();
  }
}

// Vbar_T[i] = G[v_i] (X^T V) + X[v_i] (G^T V)   (rows of every block in the batch)
template <typename T>
__global__ void k_vbar_init(const int32_t* batch, const int32_t* bptr, const int32_t* verts,
                            const T* __restrict__ G, const T* __restrict__ X,
                            const T* __restrict__ XtV, const T* __restrict__ GtV, int ld, int c,
                            T* __restrict__ Vbar) {
  const int slot = blockIdx.y;
  const int b = batch[slot];
  const int r0 = bptr[b], nb = bptr[b + 1] - r0;
  const T* xt = XtV + (size_t)slot * 3 * kMaxC;
  const T* gt = GtV + (size_t)slot * 3 * kMaxC;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nb * c; t += gridDim.x * blockDim.x) {
    const int i = t / c, j = t - i * c;
    const T* g = G + (size_t)verts[r0 + i] * 3;
    const T* x = X + (size_t)verts[r0 + i] * 3;
    T v = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) v += g[d] * xt[d * kMaxC + j] + x[d] * gt[d * kMaxC + j];
    Vbar[(size_t)(r0 + i) * ld + j] = v;
  }
}

// Ybar = (Vbar - V C) R^-T per row, with C = V^T Vbar and R (upper, c x c) per
// block: z = vbar - v C, then y R^T = z by back substitution.  One thread per
// row; C and R staged in shared memory.
template <typename T, typename TA>
__global__ void __launch_bounds__(kAT) k_ybar(const int32_t* batch, const int32_t* bptr,
                                              const T* __restrict__ Vbar, const T* __restrict__ V,
                                              const TA* __restrict__ Cm, const TA* __restrict__ Rm,
                                              int ld, int c, T* __restrict__ Ybar) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int slot = blockIdx.y;
  const int b = batch[slot];
  const int r0 = bptr[b], nb = bptr[b + 1] - r0;
  const int cpad = pad4(c);
  T* Cs = reinterpret_cast<T*>(smem_raw);
  T* Rs = Cs + cpad * cpad;
  T* z = Rs + cpad * cpad;  // per-thread row scratch: kAT x cpad
  for (int e = threadIdx.x; e < cpad * cpad; e += blockDim.x) {
    Cs[e] = (T)Cm[(size_t)slot * cpad * cpad + e];
    Rs[e] = (T)Rm[(size_t)slot * cpad * cpad + e];
  }
  __syncthreads();
  T* zr = z + threadIdx.x * cpad;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    const T* vr = V + (size_t)(r0 + i) * ld;
    const T* qr = Vbar + (size_t)(r0 + i) * ld;
    for (int k = 0; k < c; ++k) {
      T s = qr[k];
      for (int j = 0; j < c; ++j) s -= vr[j] * Cs[j * cpad + k];
      zr[k] = s;
    }
    // y R^T = z  <=>  y_k = (z_k - sum_{j > k} R_kj y_j) / R_kk, k = c-1 .. 0
    for (int k = c - 1; k >= 0; --k) {
      T s = zr[k];
      for (int j = k + 1; j < c; ++j) s -= Rs[k * cpad + j] * zr[j];
      zr[k] = s / Rs[k * cpad + k];
    }
    T* yr = Ybar + (size_t)(r0 + i) * ld;
    for (int k = 0; k < c; ++k) yr[k] = zr[k];
  }
}

// dW[e] += -sum_k (Lam[i][k] - Lam[j][k]) (Y[i][k] - Y[j][k]) for every edge
// e = (i, j), i < j, owned by row i (no two threads touch the same edge).
template <typename T>
__global__ void k_edge_grad(int64_t n, const int32_t* bptr, const int32_t* blk_row,
                            const int32_t* rowptr, const uint16_t* col, const int32_t* eoff,
                            const T* __restrict__ Lam, const T* __restrict__ Y, int ld, int c,
                            T* __restrict__ dW) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t base = bptr[blk_row[r]];
    const int i = (int)(r - base);
    int e = eoff[r];
    const T* li = Lam + (size_t)r * ld;
    const T* yi = Y + (size_t)r * ld;
    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
      const int j = col[p];
      if (j <= i) continue;
      const T* lj = Lam + (size_t)(base + j) * ld;
      const T* yj = Y + (size_t)(base + j) * ld;
      T s = 0;
      for (int k = 0; k < c; ++k) s += (li[k] - lj[k]) * (yi[k] - yj[k]);
      dW[e] -= s;
      ++e;
    }
  }
}

// out (c x c per block, TA) = A^T B over the block's rows: panel partials, then
// a fixed-order reduction (deterministic).
template <typename T, typename TA>
__global__ void __launch_bounds__(kDT) k_cross_partial(DenseArgs a, const T* __restrict__ A,
                                                       const T* __restrict__ B, int CH, int maxch,
                                                       TA* __restrict__ Gp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = a.batch[blockIdx.y];
  const int c = a.cb[b];
  const int cpad = pad4(a.cmax);
  const int r0 = a.bptr[b], nb = a.bptr[b + 1] - r0;
  const int row0 = blockIdx.x * CH;
  if (row0 >= nb) return;
  T* SA = reinterpret_cast<T*>(smem_raw);
  T* SB = SA + CH * cpad;
  stage_panel(A, a.ld, r0 + row0, min(CH, nb - row0), c, cpad, CH, SA);
  stage_panel(B, a.ld, r0 + row0, min(CH, nb - row0), c, cpad, CH, SB);
  __syncthreads();
  panel_gram<T, TA>(SA, SB, CH, cpad, false, Gp + ((size_t)blockIdx.y * maxch + blockIdx.x) * cpad * cpad);
}

template <typename TA>
__global__ void k_cross_reduce(DenseArgs a, int CH, int maxch, const TA* __restrict__ Gp,
                               TA* __restrict__ out) {
  const int b = a.batch[blockIdx.y];
  const int cpad = pad4(a.cmax);
  const int nb = a.bptr[b + 1] - a.bptr[b];
  const int nch = (nb + CH - 1) / CH;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= cpad * cpad) return;
  TA s = 0;
  for (int ch = 0; ch < nch; ++ch) s += Gp[((size_t)blockIdx.y * maxch + ch) * cpad * cpad + e];
  out[(size_t)blockIdx.y * cpad * cpad + e] = s;
}

template <typename T, typename TA>
void launch_cross(const DenseArgs& a, const T* A, const T* B, TA* Gp, int maxch, TA* out,
                  cudaStream_t s) {
  const int cpad = pad4(a.cmax);
  const int CH = 64;
  dim3 g((a.max_nb + CH - 1) / CH, a.nbatch);
  k_cross_partial<T, TA><<<g, kDT, (size_t)2 * CH * cpad * sizeof(T), s>>>(a, A, B, CH, maxch, Gp);
  dim3 gr((cpad * cpad + 255) / 256, a.nbatch);
  k_cross_reduce<TA><<<gr, 256, 0, s>>>(a, CH, maxch, Gp, out);
}

}  // namespace

// Work sizes for launch_filter_backward's workspace (elements of TA / T).
int adjoint_maxch(int max_nb) { return (max_nb + 63) / 64; }

template <typename T, typename TA>
int launch_filter_backward(const AdjointArgs& aa, const MeshView<T>& mv, cudaStream_t s) {
  const int c = aa.c, cpad = pad4(c);
  const int maxch = adjoint_maxch(aa.max_nb);
  if (c > 64) return BSP_ERR_INVALID_ARG;
  DenseArgs da{aa.batch, aa.k, aa.bptr, aa.cb, aa.ld, c, aa.max_nb, aa.status};
  TA* Gp = reinterpret_cast<TA*>(aa.ws_gp);
  TA* Cm = Gp + (size_t)aa.k * maxch * cpad * cpad;
  TA* Rm = Cm + (size_t)aa.k * cpad * cpad;
  T* XtV = reinterpret_cast<T*>(aa.ws_thin);
  T* GtV = XtV + (size_t)aa.k * 3 * kMaxC;
  const size_t nc = (size_t)aa.n * aa.ld;
  const T* VT = reinterpret_cast<const T*>(aa.ckV) + (size_t)aa.t_max * nc;
  T* Vbar = reinterpret_cast<T*>(aa.ws_rows);
  T* Ybar = Vbar + nc;
  T* Lam = Ybar + nc;
  // Vbar_T = G (X^T V_T) + X (G^T V_T)
  k_thin_cross<T, TA><<<aa.k, kAT, 0, s>>>(aa.batch, aa.bptr, aa.verts, (const T*)aa.X, VT, aa.ld,
                                           c, XtV);
  k_thin_cross<T, TA><<<aa.k, kAT, 0, s>>>(aa.batch, aa.bptr, aa.verts, (const T*)aa.G, VT, aa.ld,
                                           c, GtV);
  dim3 gi((aa.max_nb * c + 255) / 256 < 64 ? (aa.max_nb * c + 255) / 256 : 64, aa.k);
  k_vbar_init<T><<<gi, 256, 0, s>>>(aa.batch, aa.bptr, aa.verts, (const T*)aa.G, (const T*)aa.X,
                                    XtV, GtV, aa.ld, c, Vbar);
  cudaMemsetAsync(aa.dW, 0, sizeof(T) * aa.n_edges, s);
  CgArgs ca{aa.batch, aa.k, aa.cb, aa.ld, aa.z, aa.delta, aa.rtol, aa.max_steps, aa.status,
            aa.cgstats, aa.max_deg};
  const size_t ysm = ((size_t)2 * cpad * cpad + (size_t)kAT * cpad) * sizeof(T);
  for (int t = aa.t_max; t >= 1; --t) {
    const T* Vt = reinterpret_cast<const T*>(aa.ckV) + (size_t)t * nc;
    const T* Yt = reinterpret_cast<const T*>(aa.ckY) + (size_t)(t - 1) * nc;
    launch_cross<T, TA>(da, Vt, Yt, Gp, maxch, Rm, s);      // R_t = V_t^T Y_t
    launch_cross<T, TA>(da, Vt, Vbar, Gp, maxch, Cm, s);    // C = V_t^T Vbar_t
    dim3 gy((aa.max_nb + kAT - 1) / kAT, aa.k);
    k_ybar<T, TA><<<gy, kAT, ysm, s>>>(aa.batch, aa.bptr, Vbar, Vt, Cm, Rm, aa.ld, c, Ybar);
    int rc = launch_cg<T>(mv, Ybar, Lam, ca, aa.cs, aa.max_nb, c, s);  // Lambda_t = S Ybar_t
    if (rc) return rc;
    int64_t g = (aa.n + 255) / 256;
    k_edge_grad<T><<<(unsigned)(g > 4096 ? 4096 : g), 256, 0, s>>>(
        aa.n, aa.bptr, aa.blk_row, mv.rowptr, mv.col, aa.eoff, Lam, Yt, aa.ld, c, (T*)aa.dW);
    std::swap(Vbar, Lam);   // Vbar_{t-1} = Lambda_t
  }
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

void configure_adjoint_kernels() {
  set_max_dynamic_smem(k_cross_partial<float, float>);
  set_max_dynamic_smem(k_cross_partial<float, double>);
  set_max_dynamic_smem(k_cross_partial<double, double>);
  set_max_dynamic_smem(k_ybar<float, float>);
  set_max_dynamic_smem(k_ybar<float, double>);
  set_max_dynamic_smem(k_ybar<double, double>);
}

template int launch_filter_backward<float, float>(const AdjointArgs&, const MeshView<float>&,
                                                  cudaStream_t);
template int launch_filter_backward<float, double>(const AdjointArgs&, const MeshView<float>&,
                                                   cudaStream_t);
template int launch_filter_backward<double, double>(const AdjointArgs&, const MeshView<double>&,
                                                    cudaStream_t);

}  // namespace bsp
