// One CholeskyQR pass of Onorm (Sec. 4, Onorm equations) with both
// contractions on the tensor cores (tcgen05, kind::tf32), FP32 path, c <= 64:
//   k_gram_tc  G_chunk = Y_chunk^T Y_chunk for every 128-row chunk of a block
//   k_reduce   (bsp_dense.cu) sums the chunks in a fixed order
//   k_chol     (bsp_dense.cu) M = D R^-1 of the Jacobi-scaled Cholesky
//   k_mul_tc   Q_chunk = Y_chunk M
// TF32 keeps 11 significant bits, so every operand x is split in three:
// hi = x rounded to TF32, mid = (x - hi) rounded to TF32, lo = x - hi - mid
// (exact in FP32; the MMA reads its leading 11 bits).  A product is
// accumulated as hi*hi + hi*mid + mid*hi + mid*mid + hi*lo + lo*hi: the terms
// left out are below 2^-33 relative, so the result is as accurate as the
// FP32 accumulation in tensor memory that sums it.
//
// Operands are staged by all threads from global memory into shared memory
// in the K-major, non-swizzled core-matrix layout for 4-byte elements
// (core matrix = 8 rows x 16 bytes = 8 x 4 elements, contiguous 128 bytes;
// neighbouring core matrices 128 bytes apart along K, (K / 4) 128 bytes apart
// along M or N).  One thread issues the MMAs and commits them to an mbarrier;
// the four warps read the accumulator with tcgen05.ld (warp w: lanes
// 32 w .. 32 w + 31).  Every mbarrier wait is bounded: on expiry the kernel
// records ST_TIMEOUT, writes nothing, still frees its tensor memory and
// returns.
#include "bsp_dense_dev.cuh"

namespace bsp {
namespace {

using namespace dev;

constexpr int kTQ = 128;          // threads per CTA (4 warps: the 128 TMEM lanes)
constexpr int kCH = 128;          // rows per chunk (the dense path's chunk for FP32, c <= 128)
constexpr long kSpinQ = 1L << 26; // bounded mbarrier wait (iterations)

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t a, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((a & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major.
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
               ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(saddr(mbar)));
}

__device__ __forceinline__ bool wait_bounded(uint64_t* mbar, uint32_t phase) {
  uint32_t done = 0;
  for (long it = 0; it < kSpinQ && !done; ++it) {
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(done) : "r"(saddr(mbar)), "r"(phase));
  }
  return done != 0;
}

__device__ __forceinline__ void ld16(uint32_t addr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
               "%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                 "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_get(uint32_t* dst, int cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               ::"r"(saddr(dst)), "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_put(uint32_t tmem, int cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

__device__ __forceinline__ float round_tf32(float x) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  return __uint_as_float(h);
}

// x = hi + mid + lo: hi and mid rounded to TF32 (nearest, ties away); the
// two subtractions are exact in FP32
__device__ __forceinline__ void split3(float x, float& hi, float& mid, float& lo) {
  hi = round_tf32(x);
  const float r = x - hi;
  mid = round_tf32(r);
  lo = r - mid;
}

// D (+)= A B over one K-step from the three parts of A and of B (descriptors
// of the hi, mid, lo copies)
__device__ __forceinline__ void mma6(uint32_t tmem, const uint64_t (&da)[3], const uint64_t (&db)[3],
                                     uint32_t idesc, bool first) {
  mma_tf32(tmem, da[0], db[0], idesc, first ? 0u : 1u);
  mma_tf32(tmem, da[0], db[1], idesc, 1u);
  mma_tf32(tmem, da[1], db[0], idesc, 1u);
  mma_tf32(tmem, da[1], db[1], idesc, 1u);
  mma_tf32(tmem, da[0], db[2], idesc, 1u);
  mma_tf32(tmem, da[2], db[0], idesc, 1u);
}

// Element (r, k) of a K-major tile with K extent kx (a multiple of 4), in floats.
__device__ __forceinline__ int kmaj4(int r, int k, int kx) {
  return ((r >> 3) * (kx >> 2) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

__device__ __forceinline__ int tmem_columns(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : 128; }

// G_chunk = Y_chunk^T Y_chunk: M = 128 (the accumulator's row i in TMEM lane
// i), N = c rounded up to 16 (<= 64), K = 128 rows.  A (M x K) and B (N x K)
// are both Y_chunk^T in K-major form: one staged buffer (hi and lo copies)
// serves as both operands.  Its rows past c are not staged: they reach only
// accumulator rows and columns that are not read.
template <typename TA>
__global__ void __launch_bounds__(kTQ) k_gram_tc(DenseArgs a, const float* __restrict__ Y,
                                                 int maxch, TA* __restrict__ Gp) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int b = a.batch[blockIdx.y];
  if (a.live && !a.live[b]) return;
  const int c = a.cb[b];
  const int cpad = pad4(a.cmax);
  const int r0 = a.bptr[b], nb = a.bptr[b + 1] - r0;
  const int row0 = blockIdx.x * kCH;
  if (row0 >= nb) return;   // uniform per CTA, before any tensor-memory use
  const int tid = threadIdx.x, warp = tid >> 5;
  const int Np = (cpad + 7) & ~7;           // staged rows: 8 .. 64
  const int Nm = (Np + 15) & ~15;           // MMA N for M = 128
  const int cols = tmem_columns(Nm);
  float* Ap = reinterpret_cast<float*>(smem_raw);    // hi, mid, lo: 3 x (128 x kCH), K-major
  if (warp == 0) tmem_get(&tmem_base, cols);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // stage: element (m, k) = Y[row0 + k][m] (0 past the block's rows and c)
  for (int t = tid; t < kCH * Np; t += kTQ) {
    const int k = t / Np, m = t - k * Np;
    const float x = (row0 + k < nb && m < c) ? Y[(size_t)(r0 + row0 + k) * a.ld + m] : 0.f;
    float hi, mid, lo;
    split3(x, hi, mid, lo);
    const int o = kmaj4(m, k, kCH);
    Ap[o] = hi;
    Ap[128 * kCH + o] = mid;
    Ap[2 * 128 * kCH + o] = lo;
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    const uint32_t idesc = idesc_tf32(128, Nm);
    const uint32_t base = saddr(Ap), part = 128 * kCH * 4, sbo = (kCH / 4) * 128;
#pragma unroll 1
    for (int q = 0; q < kCH / 8; ++q) {
      uint64_t d[3];
#pragma unroll
      for (int h = 0; h < 3; ++h) d[h] = sdesc(base + h * part + q * 256, 128, sbo);
      mma6(tmem, d, d, idesc, q == 0);
    }
    commit(&mbar);
  }
  // one outcome per warp: the tensor-memory loads below are warp-aligned
  const bool ok = __all_sync(0xffffffffu, wait_bounded(&mbar, 0));
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok && warp < 2) {   // Gram rows < 64 live in lanes 0 .. 63
    const int i = tid;    // Gram row (lane)
    TA* out = Gp + ((size_t)blockIdx.y * maxch + blockIdx.x) * cpad * cpad;
    for (int c0 = 0; c0 < Np; c0 += 16) {
      float v[16];
      ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (i < cpad && c0 + j < cpad) out[i * cpad + c0 + j] = (TA)v[j];
    }
  }
  if (!ok && tid == 0) atomicOr(a.status, ST_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) tmem_put(tmem, cols);
}

// Q_chunk = Y_chunk M (M = cpad x cpad, upper triangular, row-major): M = 128
// rows, N = Np columns, K = Np.  A = Y_chunk (K-major: a row's columns are its
// K); B[n][k] = M[k][n] (K-major: M transposed).  The result goes through
// shared memory (row stride Np + 1) so that rows leave as coalesced segments.
// Q may alias Y: the CTA has staged its rows before it writes them.
__global__ void __launch_bounds__(kTQ) k_mul_tc(DenseArgs a, const float* Y, float* Q,
                                                const float* __restrict__ Msm) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int b = a.batch[blockIdx.y];
  if (a.live && !a.live[b]) return;
  const int c = a.cb[b];
  const int cpad = pad4(a.cmax);
  const int r0 = a.bptr[b], nb = a.bptr[b + 1] - r0;
  const int row0 = blockIdx.x * kCH;
  if (row0 >= nb) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Np = (cpad + 7) & ~7;
  const int Nm = (Np + 15) & ~15;           // MMA N for M = 128 (multiple of 16)
  const int cols = tmem_columns(Nm);
  float* Ap = reinterpret_cast<float*>(smem_raw);    // hi, mid, lo: 3 x (kCH x 64)
  float* Bp = Ap + 3 * kCH * 64;                     // hi, mid, lo: 3 x (64 x 64)
  float* out = Ap;                                   // reused after the MMAs: kCH x (Np + 1)
  if (warp == 0) tmem_get(&tmem_base, cols);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  const int nr = min(kCH, nb - row0);
  for (int t = tid; t < kCH * Np; t += kTQ) {
    const int m = t / Np, k = t - m * Np;
    const float x = (m < nr && k < c) ? Y[(size_t)(r0 + row0 + m) * a.ld + k] : 0.f;
    float hi, mid, lo;
    split3(x, hi, mid, lo);
    const int o = kmaj4(m, k, Np);
    Ap[o] = hi;
    Ap[kCH * 64 + o] = mid;
    Ap[2 * kCH * 64 + o] = lo;
  }
  const float* msrc = Msm + (size_t)blockIdx.y * cpad * cpad;
  for (int t = tid; t < Nm * Np; t += kTQ) {
    const int n = t / Np, k = t - n * Np;
    const float x = (n < cpad && k < cpad) ? msrc[k * cpad + n] : 0.f;
    float hi, mid, lo;
    split3(x, hi, mid, lo);
    const int o = kmaj4(n, k, Np);
    Bp[o] = hi;
    Bp[64 * 64 + o] = mid;
    Bp[2 * 64 * 64 + o] = lo;
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    const uint32_t idesc = idesc_tf32(128, Nm);
    const uint32_t abase = saddr(Ap), bbase = saddr(Bp), sbo = (Np / 4) * 128;
#pragma unroll 1
    for (int q = 0; q < Np / 8; ++q) {
      uint64_t da[3], db[3];
#pragma unroll
      for (int h = 0; h < 3; ++h) {
        da[h] = sdesc(abase + h * kCH * 64 * 4 + q * 256, 128, sbo);
        db[h] = sdesc(bbase + h * 64 * 64 * 4 + q * 256, 128, sbo);
      }
      mma6(tmem, da, db, idesc, q == 0);
    }
    commit(&mbar);
  }
  // one outcome per warp: the tensor-memory loads below are warp-aligned
  const bool ok = __all_sync(0xffffffffu, wait_bounded(&mbar, 0));
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();   // every thread past the wait: the operand buffers are free
  const int os = Np + 1;
  if (ok) {
    for (int c0 = 0; c0 < Np; c0 += 16) {
      float v[16];
      ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (c0 + j < Np) out[tid * os + c0 + j] = v[j];
    }
  }
  __syncthreads();
  if (ok) {
    for (int r = warp; r < nr; r += kTQ / 32) {
      float* dst = Q + (size_t)(r0 + row0 + r) * a.ld;
      for (int j = lane; j < c; j += 32) dst[j] = out[r * os + j];
    }
  }
  if (!ok && tid == 0) atomicOr(a.status, ST_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) tmem_put(tmem, cols);
}

constexpr size_t kGramSmem = (size_t)3 * 128 * kCH * sizeof(float);                 // 192 KB
constexpr size_t kMulSmem = (size_t)(3 * kCH * 64 + 3 * 64 * 64) * sizeof(float);     // 144 KB

}  // namespace

void configure_tcqr_kernels() {
  set_max_dynamic_smem(k_gram_tc<float>);
  set_max_dynamic_smem(k_gram_tc<double>);
  set_max_dynamic_smem(k_mul_tc);
}

bool tcqr_fits(int cmax, int real_bytes) { return real_bytes == 4 && dev::pad4(cmax) <= 64; }

template <typename TA>
int launch_cholqr_pass_tc(const DenseArgs& a, const float* Y, float* Q, TA* Gp, float* Rsm,
                          cudaStream_t s, int* launches) {
  if (!tcqr_fits(a.cmax, 4)) return BSP_ERR_INVALID_ARG;
  const int cpad = dev::pad4(a.cmax);
  const int maxch = (a.max_nb + kCH - 1) / kCH;
  TA* G = Gp + (size_t)a.nbatch * maxch * cpad * cpad;
  dim3 gp(maxch, a.nbatch);
  prof_begin(KC_GRAM, s);
  k_gram_tc<TA><<<gp, kTQ, kGramSmem, s>>>(a, Y, maxch, Gp);
  prof_end(KC_GRAM, s);
  int rc = launch_reduce_chol<float, TA>(a, kCH, maxch, Gp, G, Rsm, s);
  if (rc != BSP_OK) return rc;
  prof_begin(KC_PANEL, s);
  k_mul_tc<<<gp, kTQ, kMulSmem, s>>>(a, Y, Q, Rsm);
  prof_end(KC_PANEL, s);
  if (launches) *launches += 4;
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

template int launch_cholqr_pass_tc<float>(const DenseArgs&, const float*, float*, float*, float*,
                                          cudaStream_t, int*);
template int launch_cholqr_pass_tc<double>(const DenseArgs&, const float*, float*, double*, float*,
                                            cudaStream_t, int*);

}  // namespace bsp
