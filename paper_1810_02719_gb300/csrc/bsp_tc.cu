// Tensor-core (tcgen05) projection and reconstruction for wide coordinate
// matrices: all frames of a dynamic mesh with one basis per block (Sec. 7.3),
// E[b] = U[b]^T X[b] and X~[b] = U[b] E[b] (Sec. 3 GFT / inverse GFT).
//
// BF16 operands (kind::f16), FP32 accumulation in tensor memory.  Operands are
// staged by all threads from global memory into shared memory in the
// K-major, non-swizzled core-matrix layout (8 rows x 16 bytes per core
// matrix; neighbouring core matrices 128 bytes apart along K and 1024 bytes
// apart along M/N), one elected thread issues the MMAs and commits them to an
// mbarrier, and four warps read the accumulator back with tcgen05.ld.  Every
// mbarrier wait is bounded: on expiry the kernel records an error, still
// frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "bsp_internal.cuh"

namespace bsp {
namespace {

constexpr int kTT = 256;         // threads per CTA
constexpr int kM = 128;          // MMA M (rows of D = TMEM lanes)
constexpr int kKC = 64;          // K chunk per pipeline stage (4 MMAs of K = 16)
constexpr long kSpin = 1L << 26; // bounded mbarrier wait (iterations)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N)
// byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Element (r, k) of a K-major tile with K extent kc, in elements.
__device__ __forceinline__ int kmaj(int r, int k, int kc) {
  return ((r >> 3) * (kc >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
               ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(smem_u32(mbar)));
}

// Bounded wait for the given phase of an mbarrier; returns false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t phase) {
  uint32_t done = 0;
  for (long it = 0; it < kSpin && !done; ++it) {
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(done) : "r"(smem_u32(mbar)), "r"(phase));
  }
  return done != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t addr, float (&v)[16]) {
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

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, int cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               ::"r"(smem_u32(dst)), "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_free(uint32_t tmem, int cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

// E^T tile = X^T U for block b = blockIdx.y and frame-columns [m0, m0 + 128):
// A[m][k] = X[verts[r0 + k]][m0 + m] (bf16), B[n][k] = U[r0 + k][n] (fp32 -> bf16),
// K over the block's vertices in chunks of 64 (two pipeline stages).
__global__ void __launch_bounds__(kTT) k_project_tc(ProjArgs a, const float* __restrict__ U,
                                                    const __nv_bfloat16* __restrict__ X,
                                                    float* __restrict__ E, int NP, int tcols,
                                                    int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(smem_raw);     // 2 x kM x kKC
  __nv_bfloat16* sB = sA + 2 * kM * kKC;                               // 2 x NP x kKC
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int b = blockIdx.y;
  const int c = a.cb[b];
  const int r0 = a.bptr[b], nb = a.bptr[b + 1] - r0;
  const int m0 = blockIdx.x * kM;
  const int cols = a.cols;
  if (warp == 0) tmem_alloc(&tmem_base, tcols);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_bf16(kM, NP);
  const int nchunk = (nb + kKC - 1) / kKC;
  uint32_t phase[2] = {0, 0};
  bool ok = true;
  for (int ch = 0; ch < nchunk; ++ch) {
    const int s = ch & 1;
    if (ch >= 2) {  // the MMAs that read this stage two chunks ago must be done
      if (!mbar_wait(&mbar[s], phase[s])) ok = false;
      phase[s] ^= 1;
    }
    __nv_bfloat16* tA = sA + s * kM * kKC;
    __nv_bfloat16* tB = sB + s * NP * kKC;
    const int k0 = ch * kKC;
    // A: 8 consecutive frame-columns of one vertex row per 16-byte load
    for (int t = tid; t < kKC * (kM / 8); t += kTT) {
      const int k = t / (kM / 8), mg = (t % (kM / 8)) * 8;
      const int row = k0 + k;
      __nv_bfloat16 v[8];
      if (row < nb && m0 + mg + 8 <= cols) {
        const uint4 q = *reinterpret_cast<const uint4*>(X + (size_t)a.verts[r0 + row] * cols + m0 + mg);
        const __nv_bfloat16* qv = reinterpret_cast<const __nv_bfloat16*>(&q);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = qv[j];
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          v[j] = (row < nb && m0 + mg + j < cols)
                     ? X[(size_t)a.verts[r0 + row] * cols + m0 + mg + j]
                     : __float2bfloat16(0.f);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) tA[kmaj(mg + j, k, kKC)] = v[j];
    }
    // B: the basis rows, converted to bf16 (zero past c and past the block)
    for (int t = tid; t < kKC * NP; t += kTT) {
      const int k = t / NP, n = t % NP;
      const int row = k0 + k;
      const float u = (row < nb && n < c) ? U[(size_t)(r0 + row) * a.ld + n] : 0.f;
      tB[kmaj(n, k, kKC)] = __float2bfloat16(u);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int q = 0; q < kKC / 16; ++q) {
        const uint64_t da = smem_desc(smem_u32(tA) + q * 256, 128, 1024);
        const uint64_t db = smem_desc(smem_u32(tB) + q * 256, 128, 1024);
        mma_bf16(tmem, da, db, idesc, (ch > 0 || q > 0) ? 1u : 0u);
      }
      mma_commit(&mbar[s]);
    }
  }
  // drain: the last commit of each stage in use
  for (int s = 0; s < 2 && s < nchunk; ++s) {
    if (!mbar_wait(&mbar[s], phase[s])) ok = false;
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok && warp < 4 && nchunk > 0) {
    const int m = warp * 32 + (tid & 31);
    const size_t eb = (size_t)a.eoff[b];
    for (int c0 = 0; c0 < NP; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (c0 + j < c && m0 + m < cols) E[(eb + c0 + j) * cols + m0 + m] = v[j];
    }
  }
  if (!ok && tid == 0) atomicOr(status, ST_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) tmem_free(tmem, tcols);
}

// X~ tile = U E for block b = blockIdx.z, vertex rows [m0, m0 + 128) and
// columns [n0, n0 + 128): A[m][k] = U[r0 + m0 + m][k], B[n][k] = E[eoff + k][n0 + n],
// K = c padded to KP (a multiple of 16) in one stage.
__global__ void __launch_bounds__(kTT) k_recon_tc(ProjArgs a, const float* __restrict__ U,
                                                  const float* __restrict__ E,
                                                  float* __restrict__ X, int KP, int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int NT = 128;
  __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(smem_raw);  // kM x KP
  __nv_bfloat16* sB = sA + kM * KP;                                 // NT x KP
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int b = blockIdx.z;
  const int c = a.cb[b];
  const int r0 = a.bptr[b], nb = a.bptr[b + 1] - r0;
  const int m0 = blockIdx.y * kM, n0 = blockIdx.x * NT;
  const int cols = a.cols;
  if (m0 >= nb) return;  // uniform per CTA, before any tensor-memory use
  if (warp == 0) tmem_alloc(&tmem_base, NT);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  const size_t eb = (size_t)a.eoff[b];
  for (int t = tid; t < kM * KP; t += kTT) {
    const int m = t / KP, k = t % KP;
    const float u = (m0 + m < nb && k < c) ? U[(size_t)(r0 + m0 + m) * a.ld + k] : 0.f;
    sA[kmaj(m, k, KP)] = __float2bfloat16(u);
  }
  for (int t = tid; t < KP * NT; t += kTT) {
    const int k = t / NT, n = t % NT;
    const float e = (k < c && n0 + n < cols) ? E[(eb + k) * cols + n0 + n] : 0.f;
    sB[kmaj(n, k, KP)] = __float2bfloat16(e);
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    const uint32_t idesc = idesc_bf16(kM, NT);
    for (int q = 0; q < KP / 16; ++q) {
      const uint64_t da = smem_desc(smem_u32(sA) + q * 256, 128, (KP / 8) * 128);
      const uint64_t db = smem_desc(smem_u32(sB) + q * 256, 128, (KP / 8) * 128);
      mma_bf16(tmem, da, db, idesc, q > 0 ? 1u : 0u);
    }
    mma_commit(&mbar);
  }
  const bool ok = mbar_wait(&mbar, 0);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok && warp < 4) {
    const int m = warp * 32 + (tid & 31);
    const bool live = m0 + m < nb;
    float* xo = live ? X + (size_t)a.verts[r0 + m0 + m] * cols : nullptr;
    for (int c0 = 0; c0 < NT; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
      if (!live) continue;
      if (n0 + c0 + 16 <= cols && (cols & 3) == 0) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(xo + n0 + c0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (n0 + c0 + j < cols) xo[n0 + c0 + j] = v[j];
      }
    }
  }
  if (!ok && tid == 0) atomicOr(status, ST_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) tmem_free(tmem, NT);
}

inline int pad16(int c) { return (c + 15) & ~15; }
inline int tmem_cols(int n) {
  int t = 32;
  while (t < n) t <<= 1;
  return t;
}

}  // namespace

void configure_tc_kernels() {
  set_max_dynamic_smem(k_project_tc);
  set_max_dynamic_smem(k_recon_tc);
}

// E = U^T X with X in bf16 on tensor cores; needs cols % 8 == 0 and c <= 256.
int launch_project_tc(const ProjArgs& a, const float* U, const void* X, float* E, int* status,
                      cudaStream_t s) {
  const int NP = pad16(a.cmax);
  if (a.cols % 8 != 0 || NP > 256) return BSP_ERR_INVALID_ARG;
  const size_t smem = (size_t)2 * (kM + NP) * kKC * sizeof(__nv_bfloat16);
  dim3 grid((a.cols + kM - 1) / kM, a.k);
  prof_begin(KC_PROJECT, s);
  k_project_tc<<<grid, kTT, smem, s>>>(a, U, (const __nv_bfloat16*)X, E, NP, tmem_cols(NP), status);
  prof_end(KC_PROJECT, s);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

// X = U E with bf16 operands on tensor cores (FP32 accumulation and output); c <= 128.
int launch_recon_tc(const ProjArgs& a, const float* U, const float* E, float* X, int* status,
                    cudaStream_t s) {
  const int KP = pad16(a.cmax);
  if (KP > 128) return BSP_ERR_INVALID_ARG;
  // at least 60 KB of shared memory per CTA keeps <= 3 CTAs (384 tensor-memory
  // columns) per SM, so tcgen05.alloc never waits for another CTA
  size_t smem = (size_t)(kM + 128) * KP * sizeof(__nv_bfloat16);
  if (smem < 60 * 1024) smem = 60 * 1024;
  dim3 grid((a.cols + 127) / 128, (a.max_nb + kM - 1) / kM, a.k);
  prof_begin(KC_RECON, s);
  k_recon_tc<<<grid, kTT, smem, s>>>(a, U, E, X, KP, status);
  prof_end(KC_RECON, s);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

}  // namespace bsp
