// Tensor-core (tcgen05) projection and reconstruction for wide coordinate
// matrices: all frames of a dynamic mesh with one basis per block (Sec. 7.3),
// E[b] = U[b]^T X[b] and X~[b] = U[b] E[b] (Sec. 3 GFT / inverse GFT).
//
// BF16 operands (kind::f16), FP32 accumulation in tensor memory.  Operands are
// staged from global memory into shared memory by 16-byte asynchronous
// copies, in the canonical core-matrix layouts (non-swizzled: 8 rows x 16
// bytes per core matrix; or, for the projection's gathered coordinate rows,
// 128-byte swizzled atoms of 8 rows x 128 bytes), one elected thread issues
// the MMAs and commits them to an mbarrier, and four warps read the
// accumulator back with tcgen05.ld.  Every mbarrier wait is bounded: on
// expiry the kernel records an error, skips its later waits, still frees its
// tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "bsp_internal.cuh"

namespace bsp {
namespace {

constexpr int kTT = 256;         // threads per CTA
constexpr int kM = 128;          // MMA M (rows of D = TMEM lanes)
constexpr int kKC = 64;          // projection K chunk per ring stage (4 MMAs of K = 16)
constexpr long kSpin = 1L << 26; // bounded mbarrier wait (iterations)
constexpr int kS = 3;            // projection ring depth
constexpr int kD = 1;            // projection: chunks a copying thread runs ahead of its arrivals
constexpr int kProd = kTT - 32;  // projection: copying threads (warps 1-7)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N)
// byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// The same with the 128-byte swizzle (layout type 2): for an MN-major operand,
// atoms of 8 K-rows x 128 bytes (64 elements along MN, row k's 16-byte piece
// j stored at piece j ^ (k & 7)), lbo = the stride between atoms along MN,
// sbo = the stride between 8-row groups along K.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return smem_desc(saddr, lbo, sbo) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
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

// Bounded wait for the given phase of an mbarrier; returns false on expiry,
// and at once when `ok` is already false (a thread whose earlier wait expired
// skips the rest instead of spinning again).
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t phase, bool ok = true) {
  if (!ok) return false;
  uint32_t done = 0;
  for (long it = 0; it < kSpin && !done; ++it) {
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(done) : "r"(smem_u32(mbar)), "r"(phase));
  }
  return done != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}\n"
               ::"r"(smem_u32(mbar)) : "memory");
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

// 16-byte global -> shared copy on the asynchronous copy path; src_bytes = 0
// writes zeros without reading.
__device__ __forceinline__ void cp16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
               "r"(src_bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

// Element offsets inside the non-swizzled layouts (core matrix = 8 x 16 bytes):
//  K-major  (r, k), K extent kc:  core (r/8, k/8) at ((r/8)(kc/8) + k/8) * 64,
//           row r%8 holds 8 consecutive k;  LBO = 128 B (K), SBO = (kc/8) 128 B (rows).
//  MN-major (r, k), MN extent R:  core (r/8, k/8) at ((k/8)(R/8) + r/8) * 64,
//           row k%8 holds 8 consecutive r;  LBO = (R/8) 128 B (K), SBO = 128 B (MN).
__device__ __forceinline__ int mnmaj(int r, int k, int R) {
  return ((k >> 3) * (R >> 3) + (r >> 3)) * 64 + (k & 7) * 8 + (r & 7);
}

// Instruction descriptor with operand majorness: bit 15 (A) / bit 16 (B) set
// for MN-major.
__device__ __forceinline__ uint32_t idesc_bf16_major(int M, int N, int a_mn, int b_mn) {
  return idesc_bf16(M, N) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16);
}

// Ub[r][j] = bf16(U[r][j]) for j < c_b of the row's block, 0 for c_b <= j < NP:
// the basis as a tensor-core operand (rows in block order, NP columns).
__global__ void k_basis_bf16(ProjArgs a, const float* __restrict__ U, __nv_bfloat16* __restrict__ Ub,
                             int NP) {
  const int b = blockIdx.y;
  const int r0 = a.bptr[b], nb = a.bptr[b + 1] - r0, c = a.cb[b];
  const int g = NP / 8;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nb * g; t += gridDim.x * blockDim.x) {
    const int r = t / g, j0 = (t - r * g) * 8;
    const float* src = U + (size_t)(r0 + r) * a.ld + j0;
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = __float2bfloat16(j0 + e < c ? src[e] : 0.f);
    *reinterpret_cast<uint4*>(Ub + (size_t)(r0 + r) * NP + j0) = *reinterpret_cast<const uint4*>(v);
  }
}

// Eb[r][n] = bf16(E[r][n]) for n < cols, 0 for cols <= n < colsP (colsP =
// cols rounded up to 8, so that every 16-byte piece of an Eb row is aligned).
__global__ void k_coef_bf16(const float* __restrict__ E, __nv_bfloat16* __restrict__ Eb, int64_t rows,
                            int cols, int colsP) {
  const int g = colsP / 8;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < rows * g;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / g;
    const int n0 = (int)(t - r * g) * 8;
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = __float2bfloat16(n0 + e < cols ? E[r * cols + n0 + e] : 0.f);
    *reinterpret_cast<uint4*>(Eb + r * colsP + n0) = *reinterpret_cast<const uint4*>(v);
  }
}

// E^T tile = X^T U for block b = blockIdx.y and frame-columns [m0, m0 + 128):
// A[m][k] = X[verts[r0 + k]][m0 + m] and B[n][k] = Ub[r0 + k][n], both
// MN-major.  K runs over the block's vertices in chunks of 64 through a ring
// of 3 stages.  Warps 1-7 copy: 16 consecutive threads take one gathered X
// row's 256 bytes (coalesced), written into 128-byte swizzled atoms (atom
// (k / 8, m / 64) at 1024 (2 (k / 8) + m / 64) bytes, conflict-free); the
// basis rows go to the non-swizzled core-matrix layout.  Each copying thread
// waits for the stage's release (the MMA commit of the chunk that last read
// it), copies, and one chunk later waits for its own copies, fences them for
// the tensor core's proxy and arrives on the stage's full barrier.  Lane 0 of
// warp 0 waits on the full barriers and issues the MMAs.  No CTA barrier per
// chunk.
__global__ void __launch_bounds__(kTT) k_project_tc(ProjArgs a, const __nv_bfloat16* __restrict__ Ub,
                                                    const __nv_bfloat16* __restrict__ X,
                                                    float* __restrict__ E, int NP, int tcols,
                                                    int* status) {
  constexpr int S = kS, D = kD;
  static_assert(D < S, "a copying thread runs fewer chunks ahead than the ring holds");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int stageA = kM * kKC, stageB = NP * kKC;                     // elements
  // swizzled atoms need 1024-byte alignment: the launch adds 1024 bytes of slack
  const uint32_t raw = smem_u32(smem_raw);
  __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(smem_raw + (((raw + 1023u) & ~1023u) - raw));
  __nv_bfloat16* sB = sA + S * stageA;                                 // S x NP x kKC
  int32_t* sv = reinterpret_cast<int32_t*>(sB + S * stageB);           // the block's vertex ids
  __shared__ __align__(8) uint64_t full[kS], empty[kS];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int b = blockIdx.y;
  const int c = a.cb[b];
  const int r0 = a.bptr[b], nb = a.bptr[b + 1] - r0;
  const int m0 = blockIdx.x * kM;
  const int cols = a.cols;
  if (warp == 0) tmem_alloc(&tmem_base, tcols);
  // vertex ids once per CTA: the row gathers below then need no dependent
  // global load before each copy
  for (int t = tid; t < nb; t += kTT) sv[t] = a.verts[r0 + t];
  if (tid < S) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[tid])), "r"(kProd));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[tid])));
  }
  if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const int nchunk = (nb + kKC - 1) / kKC;
  const int gB = NP / 8;
  bool ok = true;
  if (warp > 0) {
    const int p = tid - 32;
    for (int ch = 0; ch < nchunk + D; ++ch) {
      if (ch < nchunk) {
        const int st = ch % S, k0 = ch * kKC;
        if (ch >= S && !mbar_wait(&empty[st], ((ch / S) - 1) & 1, ok)) ok = false;
        __nv_bfloat16* tA = sA + st * stageA;
        __nv_bfloat16* tB = sB + st * stageB;
        for (int it = p; it < kKC * (kM / 8); it += kProd) {
          const int k = it >> 4, mg = it & 15, row = k0 + k;
          const bool okr = row < nb && m0 + 8 * mg < cols;
          const __nv_bfloat16* src = okr ? X + (size_t)sv[row] * cols + m0 + 8 * mg : X;
          const int ma = mg >> 3, jj = mg & 7;
          cp16(tA + ((k >> 3) * 2 + ma) * 512 + (k & 7) * 64 + ((jj ^ (k & 7)) * 8), src,
               okr ? 16 : 0);
        }
        // basis: item -> (k % 8 fastest, piece, k / 8)
        for (int it = p; it < kKC * gB; it += kProd) {
          const int q = it >> 3, k = (it & 7) + 8 * (q / gB), ng = q % gB;
          const int row = k0 + k;
          const bool okr = row < nb;
          const __nv_bfloat16* src = okr ? Ub + (size_t)(r0 + row) * NP + 8 * ng : Ub;
          cp16(tB + mnmaj(8 * ng, k, NP), src, okr ? 16 : 0);
        }
      }
      cp_commit();
      if (ch >= D) {
        cp_wait<D>();   // this thread's copies of chunk ch - D have landed
        asm volatile("fence.proxy.async.shared::cta;");
        mbar_arrive(&full[(ch - D) % S]);
      }
    }
    cp_wait<0>();
  } else {
    // lanes 1-31 of warp 0 wait at the warp barrier (no spinning beside the
    // issuing lane)
    if (tid == 0) {
      const uint32_t idesc = idesc_bf16_major(kM, NP, 1, 1);
      for (int ch = 0; ch < nchunk; ++ch) {
        const int st = ch % S;
        if (!mbar_wait(&full[st], (ch / S) & 1, ok)) ok = false;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t aBase = smem_u32(sA + st * stageA), bBase = smem_u32(sB + st * stageB);
#pragma unroll
        for (int q = 0; q < kKC / 16; ++q) {
          const uint64_t da = smem_desc_sw128(aBase + q * 4096, 1024, 2048);
          const uint64_t db = smem_desc(bBase + q * 2 * gB * 128, gB * 128, 128);
          mma_bf16(tmem, da, db, idesc, (ch > 0 || q > 0) ? 1u : 0u);
        }
        mma_commit(&empty[st]);
      }
    }
    __syncwarp();
  }
  // every thread: the last commit covers every MMA issued before it
  if (nchunk > 0 && !mbar_wait(&empty[(nchunk - 1) % S], ((nchunk - 1) / S) & 1, ok)) ok = false;
  __syncwarp();
  ok = __all_sync(0xffffffffu, ok);   // one outcome per warp: tcgen05.ld is warp-aligned
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok && nchunk > 0) {
    // warp w reads lanes 32 (w % 4) .. + 31; warps 0-3 and 4-7 split the columns
    const int m = (warp & 3) * 32 + (tid & 31);
    const size_t eb = (size_t)a.eoff[b];
    for (int c0 = (warp >> 2) * 16; c0 < NP; c0 += 32) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (c0 + j < c && m0 + m < cols) E[(eb + c0 + j) * cols + m0 + m] = v[j];
    }
  }
  if (!ok) atomicOr(status, ST_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) tmem_free(tmem, tcols);
}

// X~ rows [m0, m0 + 128) of block b = blockIdx.y (m0 = 128 blockIdx.x) for
// all columns: A[m][k] = Ub[r0 + m0 + m][k] (K-major, resident for the whole
// CTA), B[n][k] = Eb[eoff + k][n0 + n] (MN-major), one 128-column tile after
// the other.  Both operands arrive by 16-byte asynchronous copies; the B tile
// of the next column tile is in flight while the current one drains.  The
// accumulator is double-buffered in tensor memory (2 x 128 columns), so the
// MMAs of tile j run while tile j - 1 drains: tcgen05.ld -> shared staging
// (row stride 132 floats, conflict-free) -> full 512-byte row segments to
// global memory.
constexpr int kNT = 128;
constexpr int kOS = kNT + 4;   // staging row stride (floats)
__global__ void __launch_bounds__(kTT) k_recon_tc(ProjArgs a, const __nv_bfloat16* __restrict__ Ub,
                                                  const __nv_bfloat16* __restrict__ Eb, int colsP,
                                                  float* __restrict__ X, int KP, int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(smem_raw);  // kM x KP
  __nv_bfloat16* sB = sA + kM * KP;                                 // 2 x kNT x KP
  float* out = reinterpret_cast<float*>(sB + 2 * kNT * KP);         // kM x kOS
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int32_t sv[kM];   // the tile's vertex ids
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.y;
  const int c = a.cb[b];
  const int r0 = a.bptr[b], nb = a.bptr[b + 1] - r0;
  const int m0 = blockIdx.x * kM;
  const int cols = a.cols;
  if (m0 >= nb) return;  // uniform per CTA, before any tensor-memory use
  if (warp == 0) tmem_alloc(&tmem_base, 2 * kNT);
  if (tid < kM) sv[tid] = m0 + tid < nb ? a.verts[r0 + m0 + tid] : 0;
  if (tid < 2) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[tid])));
  if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;");
  const size_t eb = (size_t)a.eoff[b];
  const int gA = KP / 8;
  // A: 128 rows x KP/8 pieces; item -> (row % 8 fastest, piece, row / 8)
  for (int it = tid; it < kM * gA; it += kTT) {
    const int q = it >> 3, m = (it & 7) + 8 * (q / gA), kg = q % gA;
    const bool ok = m0 + m < nb;
    const __nv_bfloat16* src = ok ? Ub + (size_t)(r0 + m0 + m) * KP + 8 * kg : Ub;
    cp16(sA + ((m >> 3) * gA + kg) * 64 + (m & 7) * 8, src, ok ? 16 : 0);
  }
  // B tile j: KP rows x 16 pieces of 8 columns; item -> (k % 8 fastest, piece, k / 8)
  auto issue_B = [&](int j) {
    const int n0 = j * kNT;
    __nv_bfloat16* tB = sB + (j & 1) * kNT * KP;
    for (int it = tid; it < KP * (kNT / 8); it += kTT) {
      const int k = (it & 7) + 8 * (it >> 7), ng = (it >> 3) & 15;
      const int n = n0 + 8 * ng;
      const bool ok = k < c && n < colsP;
      const __nv_bfloat16* src = ok ? Eb + (eb + k) * colsP + n : Eb;
      cp16(tB + mnmaj(8 * ng, k, kNT), src, ok ? 16 : 0);
    }
  };
  const int ntiles = (cols + kNT - 1) / kNT;
  issue_B(0);
  cp_commit();   // group 0: A and B tile 0
  const bool vec = (cols & 3) == 0 && ((uintptr_t)X & 15) == 0;
  bool ok = true;
  for (int j = 0; j < ntiles; ++j) {
    // B tile j + 1 goes to the buffer that the MMAs of tile j - 1 read
    if (j >= 1 && !mbar_wait(&mbar[(j - 1) & 1], ((j - 1) >> 1) & 1)) ok = false;
    if (j + 1 < ntiles) issue_B(j + 1);
    cp_commit();
    cp_wait<1>();  // this thread's copies of tile j (and A) have landed
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t idesc = idesc_bf16_major(kM, kNT, 0, 1);
      const uint32_t aBase = smem_u32(sA), bBase = smem_u32(sB + (j & 1) * kNT * KP);
      for (int q = 0; q < KP / 16; ++q) {
        const uint64_t da = smem_desc(aBase + q * 256, 128, gA * 128);
        const uint64_t db = smem_desc(bBase + q * 2 * (kNT / 8) * 128, (kNT / 8) * 128, 128);
        mma_bf16(tmem_base + (uint32_t)((j & 1) * kNT), da, db, idesc, q > 0 ? 1u : 0u);
      }
      mma_commit(&mbar[j & 1]);
    }
    // drain tile j - 1 (its MMAs were waited for above), then, after the
    // loop, the last tile
    const int last = (j == ntiles - 1);
    for (int jj = (j >= 1 ? j - 1 : j); jj <= j; ++jj) {
      if (jj == j && !last) break;
      if (jj == j && !mbar_wait(&mbar[jj & 1], (jj >> 1) & 1)) ok = false;
      const int n0 = jj * kNT;
      asm volatile("tcgen05.fence::after_thread_sync;");
      __syncthreads();  // the previous drain's readers are done with `out`
      const int m = (warp & 3) * 32 + lane;
      const int cbase = (warp >> 2) * 64;
#pragma unroll
      for (int c0 = 0; c0 < 64; c0 += 16) {
        float v[16];
        tmem_ld16(tmem_base + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((jj & 1) * kNT + cbase + c0), v);
#pragma unroll
        for (int e = 0; e < 16; e += 4)
          *reinterpret_cast<float4*>(out + m * kOS + cbase + c0 + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      const int width = min(kNT, cols - n0);
      if (ok && vec) {
        // the warp's 16 rows: every shared-memory load first, then the
        // 16-byte stores (no load -> store dependency per row); width is a
        // multiple of 4 here (cols % 4 == 0, n0 % 128 == 0)
        constexpr int kRW = kM / (kTT / 32);   // rows per warp
        const int nv = width >> 2;
        float4 buf[kRW];
        int vid[kRW];
#pragma unroll
        for (int i = 0; i < kRW; ++i) {
          const int r = warp + (kTT / 32) * i;
          const bool live = lane < nv && m0 + r < nb;
          buf[i] = live ? reinterpret_cast<const float4*>(out + r * kOS)[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
          vid[i] = live ? sv[r] : 0;
        }
#pragma unroll
        for (int i = 0; i < kRW; ++i) {
          const int r = warp + (kTT / 32) * i;
          if (lane < nv && m0 + r < nb)
            reinterpret_cast<float4*>(X + (size_t)vid[i] * cols + n0)[lane] = buf[i];
        }
      } else if (ok) {
        for (int r = warp; r < kM; r += kTT / 32) {
          if (m0 + r >= nb) break;
          float* dst = X + (size_t)sv[r] * cols + n0;
          const float* srow = out + r * kOS;
          for (int e = lane; e < width; e += 32) dst[e] = srow[e];
        }
      }
    }
  }
  cp_wait<0>();
  if (!ok && tid == 0) atomicOr(status, ST_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) tmem_free(tmem_base, 2 * kNT);
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

// Ub = bf16 copy of the basis, NP = pad16(cmax) columns, zero past each c_b.
int launch_basis_bf16(const ProjArgs& a, const float* U, void* Ub, cudaStream_t s) {
  const int NP = pad16(a.cmax);
  const int per = a.max_nb * (NP / 8);
  dim3 grid((per + 255) / 256, a.k);
  k_basis_bf16<<<grid, 256, 0, s>>>(a, U, (__nv_bfloat16*)Ub, NP);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

// E = U^T X with X in bf16 on tensor cores; Ub from launch_basis_bf16; needs
// cols % 8 == 0 and c <= 256.
int launch_project_tc(const ProjArgs& a, const void* Ub, const void* X, float* E, int* status,
                      cudaStream_t s) {
  const int NP = pad16(a.cmax);
  if (a.cols % 8 != 0 || NP > 256) return BSP_ERR_INVALID_ARG;
  const size_t smem = (size_t)kS * (kM + NP) * kKC * sizeof(__nv_bfloat16) +
                      (size_t)a.max_nb * sizeof(int32_t) + 1024;   // + alignment slack
  if (smem > 220 * 1024) return BSP_ERR_INVALID_ARG;
  dim3 grid((a.cols + kM - 1) / kM, a.k);
  prof_begin(KC_PROJECT, s);
  k_project_tc<<<grid, kTT, smem, s>>>(a, (const __nv_bfloat16*)Ub, (const __nv_bfloat16*)X, E, NP,
                                       tmem_cols(NP), status);
  prof_end(KC_PROJECT, s);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

// X = U E with bf16 operands on tensor cores (FP32 accumulation and output);
// Ub from launch_basis_bf16, Eb scratch of erows x pad8(cols) bf16; c <= 128.
int launch_recon_tc(const ProjArgs& a, const void* Ub, const float* E, int64_t erows, void* Eb,
                    float* X, int* status, cudaStream_t s) {
  const int KP = pad16(a.cmax);
  if (KP > 128) return BSP_ERR_INVALID_ARG;
  const int colsP = (a.cols + 7) & ~7;
  const int64_t pieces = erows * (colsP / 8);
  if (pieces > 0) {
    const int grid = (int)std::min<int64_t>((pieces + 255) / 256, 152 * 16);
    k_coef_bf16<<<grid, 256, 0, s>>>(E, (__nv_bfloat16*)Eb, erows, a.cols, colsP);
  }
  // at least 80 KB of shared memory per CTA keeps <= 2 CTAs (512 tensor-memory
  // columns) per SM, so tcgen05.alloc never waits for another CTA
  size_t smem = (size_t)3 * kNT * KP * sizeof(__nv_bfloat16) + (size_t)kM * kOS * sizeof(float);
  if (smem < 80 * 1024) smem = 80 * 1024;
  dim3 grid((a.max_nb + kM - 1) / kM, a.k);
  prof_begin(KC_RECON, s);
  k_recon_tc<<<grid, kTT, smem, s>>>(a, (const __nv_bfloat16*)Ub, (const __nv_bfloat16*)Eb, colsP, X,
                                     KP, status);
  prof_end(KC_RECON, s);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

}  // namespace bsp
