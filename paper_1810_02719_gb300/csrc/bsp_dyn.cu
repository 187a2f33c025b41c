// Start matrices for Algorithm 1 and the decision/growth steps of dynamic OI
// (Sec. 4 warm start; Sec. 5, Algorithm 2, Eq. residual and Eq. newU).
//
// k_init_starts  U_b <- rows of the root start matrices, or the parent's basis
//                with row r taken from row floor(r n_parent / n_b)
// k_dyn_decide   one CTA per block: E = U^T X (3 columns), then for every
//                prefix width j = c_step, 2 c_step, ... the relative residual
//                rho(j) = ||X - U_j U_j^T X||_F / ||X||_F (direct, not Parseval);
//                picks the smallest passing j, or asks for growth; also writes
//                the residual e = sum over x, y, z of (X - U U^T X) for growth
// k_dyn_grow     appends [e/||e||, counter-hash columns] projected off span(U)
#include <cstdint>

#include "bsp_internal.cuh"

namespace bsp {
namespace {

constexpr int kT = 256;
constexpr int kMaxChk = 128 / 8 + 1;   // prefix checkpoints for c_step >= 8
constexpr int kMaxC = 128;
constexpr int kRowsInFlight = 4;       // rows whose loads a warp issues together

template <typename T>
__global__ void k_init_starts(const int32_t* batch, const int32_t* bptr, const int32_t* parent,
                              const int32_t* root_off, const int32_t* cb, const int32_t* cpar,
                              const T* starts, int ld_start, T* U, int ld, const T* Usrc) {
  const int b = batch[blockIdx.y];
  const int c = cb[b];
  const int r0 = bptr[b], nb = bptr[b + 1] - r0;
  const int p = parent[b];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nb * c; t += gridDim.x * blockDim.x) {
    const int i = t / c, j = t - i * c;
    T v;
    if (p < 0) {
      v = starts[(size_t)(root_off[b] + i) * ld_start + j];
    } else {
      const int rp0 = bptr[p], np = bptr[p + 1] - rp0;
      const int src = (int)(((int64_t)i * np) / nb);
      v = j < cpar[b] ? Usrc[(size_t)(rp0 + src) * ld + j] : T(0);
    }
    U[(size_t)(r0 + i) * ld + j] = v;
  }
}

// SplitMix64 output function (Steele, Lea, Flood 2014) chained over the
// counter (seed, block, round, row, col); top 53 bits -> u in [0,1) -> 2u - 1.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__device__ __forceinline__ double hash_uniform(uint64_t seed, uint64_t blk, uint64_t rnd,
                                               uint64_t row, uint64_t col) {
  const uint64_t g = 0x9E3779B97F4A7C15ull;
  uint64_t h = seed;
  h = mix64(h + g * (blk + 1));
  h = mix64(h + g * (rnd + 1));
  h = mix64(h + g * (row + 1));
  h = mix64(h + g * (col + 1));
  return 2.0 * ((double)(h >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

template <typename T, typename TA>
BSP_DEV TA block_reduce(TA v, TA* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  TA s = 0;
  for (int w = 0; w < kT / 32; ++w) s += red[w];
  return s;
}

// action: 0 = accepted (cb[b] set to the chosen width), 1 = grow, 2 = accepted at c_max
template <typename T, typename TA>
__global__ void __launch_bounds__(kT) k_dyn_decide(const int32_t* batch, const int32_t* bptr,
                                                   const int32_t* verts, const T* __restrict__ X,
                                                   const T* __restrict__ U, int ld, int32_t* cb,
                                                   int32_t* action, const int32_t* forced,
                                                   double tol, int c_step, int c_max, T* gcol,
                                                   TA* rho_out, int32_t* live) {
  __shared__ TA Ered[kT / 32][3 * 32];
  __shared__ T Es[kMaxC][3];
  __shared__ TA res[kMaxChk];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  T* Xs = reinterpret_cast<T*>(dyn_smem);   // the block's coordinates, local order [nb x 3]
  const int b = batch[blockIdx.x];
  if (live && !live[b]) return;
  const int c = cb[b];
  const int r0 = bptr[b], nb = bptr[b + 1] - r0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // gather the block's coordinates once (all rows in flight together)
  for (int t = threadIdx.x; t < nb * 3; t += kT) {
    const int i = t / 3, k = t - i * 3;
    Xs[t] = X[(size_t)verts[r0 + i] * 3 + k];
  }
  __syncthreads();
  // E = U^T X: lanes own columns j = lane + 32 q, warps split the rows
  for (int q = 0; q * 32 < c; ++q) {
    const int j = q * 32 + lane;
    TA e0 = 0, e1 = 0, e2 = 0;
    T f0 = 0, f1 = 0, f2 = 0;
    int cnt = 0;
    // rows w, w + 8, ... in order; four rows' loads in flight per iteration
    for (int i0 = w; i0 < nb; i0 += kRowsInFlight * (kT / 32)) {
      T u[kRowsInFlight];
#pragma unroll
      for (int m = 0; m < kRowsInFlight; ++m) {
        const int i = i0 + m * (kT / 32);
        u[m] = (i < nb && j < c) ? U[(size_t)(r0 + i) * ld + j] : T(0);
      }
#pragma unroll
      for (int m = 0; m < kRowsInFlight; ++m) {
        const int i = i0 + m * (kT / 32);
        if (i < nb) {
          const T* x = Xs + i * 3;
          f0 += u[m] * x[0];
          f1 += u[m] * x[1];
          f2 += u[m] * x[2];
          if (++cnt == 32) {  // FP32 partial sums over 32 rows, accumulated in TA
            e0 += f0; e1 += f1; e2 += f2;
            f0 = f1 = f2 = 0;
            cnt = 0;
          }
        }
      }
    }
    e0 += f0; e1 += f1; e2 += f2;
    Ered[w][3 * lane] = e0;
    Ered[w][3 * lane + 1] = e1;
    Ered[w][3 * lane + 2] = e2;
    __syncthreads();
    if (threadIdx.x < 96) {
      TA s = 0;
      for (int ww = 0; ww < kT / 32; ++ww) s += Ered[ww][threadIdx.x];
      const int jj = q * 32 + threadIdx.x / 3;
      if (jj < c) Es[jj][threadIdx.x % 3] = (T)s;
    }
    __syncthreads();
  }
  // residual norms at every checkpoint width; ||X||^2
  const int nchk = c / c_step;
  __shared__ T accs[kMaxChk][kT];
  T xx = 0;
  // c is a multiple of c_step = 8: one checkpoint per 8-column segment.  The
  // segments' partial sums are independent (no long dependent chain); every
  // thread keeps its checkpoint sums in its own column of accs (shared).
  for (int q = 0; q < nchk; ++q) accs[q][threadIdx.x] = 0;
  for (int i = threadIdx.x; i < nb; i += kT) {
    const T* x = Xs + i * 3;
    const T x0 = x[0], x1 = x[1], x2 = x[2];
    xx += x0 * x0 + x1 * x1 + x2 * x2;
    T h0 = 0, h1 = 0, h2 = 0;
    const T* u = U + (size_t)(r0 + i) * ld;
    for (int q = 0; q < nchk; ++q) {
      T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const T ul = u[q * 8 + e];
        s0 += ul * Es[q * 8 + e][0];
        s1 += ul * Es[q * 8 + e][1];
        s2 += ul * Es[q * 8 + e][2];
      }
      h0 += s0;
      h1 += s1;
      h2 += s2;
      const T d0 = x0 - h0, d1 = x1 - h1, d2 = x2 - h2;
      accs[q][threadIdx.x] += d0 * d0 + d1 * d1 + d2 * d2;
    }
    gcol[(size_t)(r0 + i)] = (x0 - h0) + (x1 - h1) + (x2 - h2);
  }
  // ||X||^2 and every checkpoint residual, reduced together (per warp by the
  // same butterfly as block_reduce, then over the warps in warp order); each
  // checkpoint's ratio by its own thread
  __shared__ TA wred[kT / 32][kMaxChk + 1];
  __shared__ TA ratio[kMaxChk];
  {
    const TA v = warp_sum((TA)xx);
    if (lane == 0) wred[w][kMaxChk] = v;
    for (int q = 0; q < nchk; ++q) {
      const TA u = warp_sum((TA)accs[q][threadIdx.x]);
      if (lane == 0) wred[w][q] = u;
    }
  }
  __syncthreads();
  TA xnorm2 = 0;
  for (int ww = 0; ww < kT / 32; ++ww) xnorm2 += wred[ww][kMaxChk];
  if (threadIdx.x < nchk) {
    TA sq = 0;
    for (int ww = 0; ww < kT / 32; ++ww) sq += wred[ww][threadIdx.x];
    res[threadIdx.x] = sq;
    ratio[threadIdx.x] = xnorm2 > 0 ? sqrt(sq / xnorm2) : TA(0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int fc = forced ? forced[b] : -1;
    int act = 1, cj = c;
    TA rho = 0;
    if (fc >= 0) {
      if (fc <= c || c >= c_max) {
        cj = fc < c ? fc : c;
        act = 0;
        const int q = cj / c_step - 1;
        rho = q >= 0 ? ratio[q] : TA(0);
      }
    } else {
      for (int q = 0; q < nchk; ++q) {
        const TA r = ratio[q];
        if (r <= (TA)tol) {
          act = 0;
          cj = (q + 1) * c_step;
          rho = r;
          break;
        }
        rho = r;
      }
      if (act == 1 && c >= c_max) act = 2;
    }
    action[b] = act;
    if (act == 0) cb[b] = cj;
    rho_out[b] = rho;
    if (live) {
      const int cmaxb = min(c_max, (nb / c_step) * c_step);
      live[b] = (act == 1 && c < cmaxb) ? 1 : 0;
    }
  }
}

// Append c_step columns at position c = cb[b]: [e/||e||, hash columns], all
// projected off the current basis U[:, :c] (one classical Gram-Schmidt sweep;
// the Onorm that follows re-orthonormalises).  Updates cb[b] += c_step and
// round[b] += 1 (the hash counter of the next growth).
template <typename T, typename TA>
__global__ void __launch_bounds__(kT) k_dyn_grow(const int32_t* batch, const int32_t* bptr,
                                                 int32_t* cb, int32_t* round, T* U, int ld,
                                                 const T* __restrict__ gcol, uint64_t seed,
                                                 int c_step, const int32_t* live) {
  __shared__ TA red[kT / 32];
  __shared__ T Cm[kMaxC][8];              // U^T G, c x c_step (c_step <= 8)
  __shared__ T part[kT / 32][32 * 8];     // per-warp partial products (one 32-column slice)
  const int b = batch[blockIdx.x];
  if (live && !live[b]) return;
  const int c = cb[b];
  const int r0 = bptr[b], nb = bptr[b + 1] - r0;
  const int rnd = round[b];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // ||e||
  T ee = 0;
  for (int i = threadIdx.x; i < nb; i += kT) {
    const T e = gcol[r0 + i];
    ee += e * e;
  }
  const TA en = sqrt(block_reduce<T, TA>((TA)ee, red));
  const T inv = en > 0 ? (T)(1.0 / (double)en) : T(0);
  // write the raw growth block into columns [c, c + c_step)
  for (int t = threadIdx.x; t < nb * c_step; t += kT) {
    const int i = t / c_step, g = t - i * c_step;
    T v = g == 0 ? gcol[r0 + i] * inv
                 : (T)hash_uniform(seed, (uint64_t)b, (uint64_t)rnd, (uint64_t)i, (uint64_t)g);
    U[(size_t)(r0 + i) * ld + c + g] = v;
  }
  __syncthreads();
  // Cm = U[:, :c]^T G, 32 columns of U at a time
  for (int q = 0; q * 32 < c; ++q) {
    const int j = q * 32 + lane;
    T a[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) a[g] = 0;
    for (int i0 = w; i0 < nb; i0 += kRowsInFlight * (kT / 32)) {
      T u[kRowsInFlight], gv[kRowsInFlight][8];
#pragma unroll
      for (int m = 0; m < kRowsInFlight; ++m) {
        const int i = i0 + m * (kT / 32);
        const T* row = U + (size_t)(r0 + (i < nb ? i : 0)) * ld;
        u[m] = (i < nb && j < c) ? row[j] : T(0);
#pragma unroll
        for (int g = 0; g < 8; ++g) gv[m][g] = (i < nb && g < c_step) ? row[c + g] : T(0);
      }
#pragma unroll
      for (int m = 0; m < kRowsInFlight; ++m)
#pragma unroll
        for (int g = 0; g < 8; ++g) a[g] += u[m] * gv[m][g];
    }
#pragma unroll
    for (int g = 0; g < 8; ++g) part[w][lane * 8 + g] = a[g];
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * 8; t += kT) {
      T s = 0;
      for (int ww = 0; ww < kT / 32; ++ww) s += part[ww][t];
      const int jj = q * 32 + t / 8;
      if (jj < c) Cm[jj][t % 8] = s;
    }
    __syncthreads();
  }
  // G -= U[:, :c] Cm (c a multiple of 8; four independent partial sums)
  for (int t = threadIdx.x; t < nb * c_step; t += kT) {
    const int i = t / c_step, g = t - i * c_step;
    T* row = U + (size_t)(r0 + i) * ld;
    T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int l = 0; l < c; l += 4) {
      s0 += row[l] * Cm[l][g];
      s1 += row[l + 1] * Cm[l + 1][g];
      s2 += row[l + 2] * Cm[l + 2][g];
      s3 += row[l + 3] * Cm[l + 3][g];
    }
    row[c + g] -= (s0 + s1) + (s2 + s3);
  }
  if (threadIdx.x == 0) {
    cb[b] = c + c_step;
    round[b] = rnd + 1;
  }
}

// ---- device-side control of the dynamic-c rounds (one CTA per wave)
constexpr int kCT = 256;

BSP_DEV int block_max(int v, int* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int m = red[0];
  for (int w = 1; w < kCT / 32; ++w) m = max(m, red[w]);
  return m;
}

// width class of the largest width: ceil(c / cls_width) - 1, clamped to the
// classes built (a width above every class selects none: no body runs)
BSP_DEV int width_class(int cmax, int cls_width, int ncls) {
  const int q = (cmax + cls_width - 1) / cls_width - 1;
  return q < 0 ? 0 : (q < ncls ? q : ncls);
}

__global__ void __launch_bounds__(kCT) k_dyn_wave_init(
    const int32_t* wave, int nw, const int32_t* bptr, const int32_t* parent, int32_t* cb,
    int32_t* cpar, int32_t* live, int32_t* round, int c_min, int c_max, int c_step, int cls_width,
    int ncls, const unsigned* start_launches, DynCtl* ctl, int set_handle,
    cudaGraphConditionalHandle h_start) {
  __shared__ int red[kCT / 32];
  int mx = 0;
  for (int i = threadIdx.x; i < nw; i += kCT) {
    const int b = wave[i];
    const int p = parent[b];
    const int nb = bptr[b + 1] - bptr[b];
    const int cmaxb = min(c_max, (nb / c_step) * c_step);
    const int c = p < 0 ? c_min : min(cb[p], cmaxb);
    cb[b] = c;
    cpar[b] = p < 0 ? 0 : cb[p];
    live[b] = 1;
    round[b] = 0;
    mx = max(mx, c);
  }
  mx = block_max(mx, red);
  if (threadIdx.x == 0) {
    const int q = width_class(mx, cls_width, ncls);
    ctl->cls_start = q;
    ctl->rounds = 0;
    ctl->more = 1;
    ctl->launches += 1 + (q < ncls ? start_launches[q] : 0u);
    if (set_handle) cudaGraphSetConditional(h_start, (unsigned)q);
  }
}

__global__ void __launch_bounds__(kCT) k_dyn_class(const int32_t* wave, int nw, const int32_t* cb,
                                                   const int32_t* live, int cls_width, int ncls,
                                                   const unsigned* round_launches, unsigned base,
                                                   DynCtl* ctl, int set_handle,
                                                   cudaGraphConditionalHandle h_round) {
  __shared__ int red[kCT / 32];
  int mx = 0;
  for (int i = threadIdx.x; i < nw; i += kCT) {
    const int b = wave[i];
    if (live[b]) mx = max(mx, cb[b]);
  }
  mx = block_max(mx, red);
  if (threadIdx.x == 0) {
    const int q = width_class(mx, cls_width, ncls);
    ctl->cls_round = q;
    ctl->launches += base + (q < ncls ? round_launches[q] : 0u);
    if (set_handle) cudaGraphSetConditional(h_round, (unsigned)q);
  }
}

__global__ void __launch_bounds__(kCT) k_dyn_next(const int32_t* wave, int nw,
                                                  const int32_t* live, int max_rounds, DynCtl* ctl,
                                                  int set_handle,
                                                  cudaGraphConditionalHandle h_while) {
  __shared__ int red[kCT / 32];
  int any = 0;
  for (int i = threadIdx.x; i < nw; i += kCT) any |= live[wave[i]] ? 1 : 0;
  any = block_max(any, red);
  if (threadIdx.x == 0) {
    const int r = ctl->rounds + 1;
    ctl->rounds = r;
    const int more = (any && r < max_rounds) ? 1 : 0;
    ctl->more = more;
    if (set_handle) cudaGraphSetConditional(h_while, (unsigned)more);
  }
}

// The paper's dynamic OI (Sec. 5, Algorithm 2): one decision per iteration
// for every block of the batch.  E = U^T X and e = sum over x, y, z of
// (X - U E) (Eq. residual), products in T over 32-row chunks accumulated in
// FP64, ||e|| in FP64.  Then, branch directions as the text states them:
// ||e|| > eps_h and c < min(c_max, n_b): column c of U becomes e/||e|| (the
// next step's Onorm of R^z [U, e/||e||] is Eq. newU) and cb[b] = c + 1;
// ||e|| < eps_l and c > c_min: cb[b] = c - 1 (the first c - 1 columns stay);
// otherwise done[b] = t (the block stops).  enorm[b] = ||e||.
template <typename T>
__global__ void __launch_bounds__(kT) k_doi_decide(const int32_t* batch, const int32_t* bptr,
                                                   const int32_t* verts, const T* __restrict__ X,
                                                   T* U, int ld, int32_t* cb, int32_t* done,
                                                   int t_arg, double eps_l, double eps_h, int c_min,
                                                   int c_max, T* gcol, double* enorm,
                                                   int32_t* live, const DynCtl* ctl) {
  __shared__ double Ered[kT / 32][3 * 32];
  __shared__ T Es[kMaxC][3];
  __shared__ double red[kT / 32];
  __shared__ int s_act;
  const int b = batch[blockIdx.x];
  if (live && !live[b]) return;
  // the iteration number: the argument, or (device-driven rounds) the rounds
  // already run in this wave plus one
  const int t = ctl ? ctl->rounds + 1 : t_arg;
  const int c = cb[b];
  const int r0 = bptr[b], nb = bptr[b + 1] - r0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int q = 0; q * 32 < c; ++q) {
    const int j = q * 32 + lane;
    double e0 = 0, e1 = 0, e2 = 0;
    T f0 = 0, f1 = 0, f2 = 0;
    int cnt = 0;
    for (int i = w; i < nb; i += kT / 32) {
      const T u = j < c ? U[(size_t)(r0 + i) * ld + j] : T(0);
      const T* x = X + (size_t)verts[r0 + i] * 3;
      f0 += u * x[0];
      f1 += u * x[1];
      f2 += u * x[2];
      if (++cnt == 32) {
        e0 += f0; e1 += f1; e2 += f2;
        f0 = f1 = f2 = 0;
        cnt = 0;
      }
    }
    e0 += f0; e1 += f1; e2 += f2;
    Ered[w][3 * lane] = e0;
    Ered[w][3 * lane + 1] = e1;
    Ered[w][3 * lane + 2] = e2;
    __syncthreads();
    if (threadIdx.x < 96) {
      double sum = 0;
      for (int ww = 0; ww < kT / 32; ++ww) sum += Ered[ww][threadIdx.x];
      const int jj = q * 32 + threadIdx.x / 3;
      if (jj < c) Es[jj][threadIdx.x % 3] = (T)sum;
    }
    __syncthreads();
  }
  double ee = 0;
  for (int i = threadIdx.x; i < nb; i += kT) {
    const T* x = X + (size_t)verts[r0 + i] * 3;
    const T* u = U + (size_t)(r0 + i) * ld;
    T h0 = 0, h1 = 0, h2 = 0;
    for (int j = 0; j < c; ++j) {
      const T uj = u[j];
      h0 += uj * Es[j][0];
      h1 += uj * Es[j][1];
      h2 += uj * Es[j][2];
    }
    const double e = ((double)x[0] - (double)h0) + ((double)x[1] - (double)h1) +
                     ((double)x[2] - (double)h2);
    gcol[r0 + i] = (T)e;
    ee += e * e;
  }
  const double n2 = block_reduce<T, double>(ee, red);
  if (threadIdx.x == 0) {
    const double ne = sqrt(n2);
    const int cmx = c_max < nb ? c_max : nb;
    int act = 0;
    if (ne > eps_h && c < cmx) act = 1;
    else if (ne < eps_l && c > c_min) act = 2;
    if (act == 1) cb[b] = c + 1;
    else if (act == 2) cb[b] = c - 1;
    else done[b] = t;
    if (live && act == 0) live[b] = 0;
    enorm[b] = ne;
    s_act = act;
  }
  __syncthreads();
  if (s_act == 1) {
    const double inv = 1.0 / sqrt(n2);
    for (int i = threadIdx.x; i < nb; i += kT)
      U[(size_t)(r0 + i) * ld + c] = (T)((double)gcol[r0 + i] * inv);
  }
}

}  // namespace

template <typename T>
void launch_init_starts(const int32_t* batch, int nbatch, const int32_t* bptr,
                        const int32_t* parent, const int32_t* root_off, const int32_t* cb,
                        const int32_t* cpar, const T* starts, int ld_start, T* U, int ld,
                        int max_nb, int cmax, cudaStream_t s, const T* Usrc) {
  const int per = max_nb * cmax;
  dim3 grid((per + 255) / 256 < 64 ? (per + 255) / 256 : 64, nbatch);
  prof_begin(KC_INIT, s);
  k_init_starts<T><<<grid, 256, 0, s>>>(batch, bptr, parent, root_off, cb, cpar, starts, ld_start,
                                        U, ld, Usrc ? Usrc : U);
  prof_end(KC_INIT, s);
}

template <typename T, typename TA>
int launch_dyn_decide(const int32_t* batch, int nbatch, const int32_t* bptr, const int32_t* verts,
                      const T* X, const T* U, int ld, int32_t* cb, int32_t* action,
                      const int32_t* forced, double tol, int c_step, int c_max, T* gcol,
                      TA* rho_out, int max_nb, cudaStream_t s, int32_t* live) {
  if (c_step < 8 || c_max > kMaxC) return BSP_ERR_INVALID_ARG;
  const size_t smem = (size_t)max_nb * 3 * sizeof(T);
  if (smem > 160 * 1024) return BSP_ERR_INVALID_ARG;
  prof_begin(KC_DYN, s);
  k_dyn_decide<T, TA><<<nbatch, kT, smem, s>>>(batch, bptr, verts, X, U, ld, cb, action, forced,
                                               tol, c_step, c_max, gcol, rho_out, live);
  prof_end(KC_DYN, s);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

void configure_dyn_kernels() {
  set_max_dynamic_smem(k_dyn_decide<float, float>);
  set_max_dynamic_smem(k_dyn_decide<float, double>);
  set_max_dynamic_smem(k_dyn_decide<double, double>);
}

template <typename T, typename TA>
int launch_dyn_grow(const int32_t* batch, int nbatch, const int32_t* bptr, int32_t* cb,
                    int32_t* round, T* U, int ld, const T* gcol, uint64_t seed,
                    int c_step, int max_nb, cudaStream_t s, const int32_t* live) {
  if (c_step > 8) return BSP_ERR_INVALID_ARG;
  prof_begin(KC_DYN, s);
  k_dyn_grow<T, TA><<<nbatch, kT, 0, s>>>(batch, bptr, cb, round, U, ld, gcol, seed, c_step,
                                          live);
  prof_end(KC_DYN, s);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

int launch_dyn_wave_init(const int32_t* wave, int nw, const int32_t* bptr, const int32_t* parent,
                         int32_t* cb, int32_t* cpar, int32_t* live, int32_t* round, int c_min,
                         int c_max, int c_step, int cls_width, int ncls,
                         const unsigned* start_launches, DynCtl* ctl, int set_handle,
                         cudaGraphConditionalHandle h_start, cudaStream_t s) {
  k_dyn_wave_init<<<1, kCT, 0, s>>>(wave, nw, bptr, parent, cb, cpar, live, round, c_min, c_max,
                                    c_step, cls_width, ncls, start_launches, ctl, set_handle,
                                    h_start);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

int launch_dyn_class(const int32_t* wave, int nw, const int32_t* cb, const int32_t* live,
                     int cls_width, int ncls, const unsigned* round_launches, DynCtl* ctl,
                     int set_handle, cudaGraphConditionalHandle h_round, cudaStream_t s,
                     unsigned base) {
  k_dyn_class<<<1, kCT, 0, s>>>(wave, nw, cb, live, cls_width, ncls, round_launches, base, ctl,
                                set_handle, h_round);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

int launch_dyn_next(const int32_t* wave, int nw, const int32_t* live, int max_rounds, DynCtl* ctl,
                    int set_handle, cudaGraphConditionalHandle h_while, cudaStream_t s) {
  k_dyn_next<<<1, kCT, 0, s>>>(wave, nw, live, max_rounds, ctl, set_handle, h_while);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

template <typename T>
int launch_doi_decide(const int32_t* batch, int nbatch, const int32_t* bptr, const int32_t* verts,
                      const T* X, T* U, int ld, int32_t* cb, int32_t* done, int t, double eps_l,
                      double eps_h, int c_min, int c_max, T* gcol, double* enorm, cudaStream_t s,
                      int32_t* live, const DynCtl* ctl) {
  if (c_max > kMaxC) return BSP_ERR_INVALID_ARG;
  prof_begin(KC_DYN, s);
  k_doi_decide<T><<<nbatch, kT, 0, s>>>(batch, bptr, verts, X, U, ld, cb, done, t, eps_l, eps_h,
                                        c_min, c_max, gcol, enorm, live, ctl);
  prof_end(KC_DYN, s);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}
template int launch_doi_decide<float>(const int32_t*, int, const int32_t*, const int32_t*,
                                      const float*, float*, int, int32_t*, int32_t*, int, double,
                                      double, int, int, float*, double*, cudaStream_t, int32_t*,
                                      const DynCtl*);
template int launch_doi_decide<double>(const int32_t*, int, const int32_t*, const int32_t*,
                                       const double*, double*, int, int32_t*, int32_t*, int,
                                       double, double, int, int, double*, double*, cudaStream_t,
                                       int32_t*, const DynCtl*);

template void launch_init_starts<float>(const int32_t*, int, const int32_t*, const int32_t*,
                                        const int32_t*, const int32_t*, const int32_t*,
                                        const float*, int, float*, int, int, int, cudaStream_t,
                                        const float*);
template void launch_init_starts<double>(const int32_t*, int, const int32_t*, const int32_t*,
                                         const int32_t*, const int32_t*, const int32_t*,
                                         const double*, int, double*, int, int, int,
                                         cudaStream_t, const double*);
template int launch_dyn_decide<float, double>(const int32_t*, int, const int32_t*, const int32_t*,
                                              const float*, const float*, int, int32_t*, int32_t*,
                                              const int32_t*, double, int, int, float*, double*,
                                              int, cudaStream_t, int32_t*);
template int launch_dyn_decide<float, float>(const int32_t*, int, const int32_t*, const int32_t*,
                                             const float*, const float*, int, int32_t*, int32_t*,
                                             const int32_t*, double, int, int, float*, float*, int,
                                             cudaStream_t, int32_t*);
template int launch_dyn_decide<double, double>(const int32_t*, int, const int32_t*,
                                               const int32_t*, const double*, const double*, int,
                                               int32_t*, int32_t*, const int32_t*, double, int,
                                               int, double*, double*, int, cudaStream_t, int32_t*);
template int launch_dyn_grow<float, double>(const int32_t*, int, const int32_t*, int32_t*,
                                            int32_t*, float*, int, const float*, uint64_t,
                                            int, int, cudaStream_t, const int32_t*);
template int launch_dyn_grow<float, float>(const int32_t*, int, const int32_t*, int32_t*,
                                           int32_t*, float*, int, const float*, uint64_t,
                                           int, int, cudaStream_t, const int32_t*);
template int launch_dyn_grow<double, double>(const int32_t*, int, const int32_t*, int32_t*,
                                             int32_t*, double*, int, const double*, uint64_t,
                                             int, int, cudaStream_t, const int32_t*);

}  // namespace bsp
