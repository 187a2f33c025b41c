// Tiled operator product Y = (L + delta I) P over all blocks (the sparse x
// tall-skinny product inside every solve of S = R^z, Sec. 4).
//
// Rows are cut into chunks of up to 64 rows inside one block.  A chunk's
// neighbour rows lie in a contiguous range [lo, hi] of the block (its
// bandwidth in local order), computed once per mesh.  One CTA per chunk
// stages P[lo..hi] into shared memory with 16-byte asynchronous copies
// (consecutive threads copy consecutive 16-byte pieces: fully coalesced, and
// every P row is read from HBM about once) and, while they fly, the chunk's
// pattern with columns rebased to rows of the staged range and the diagonal;
// then every row of
// the chunk is formed from shared memory only, LPR lanes per row (the row's
// 16-byte vectors, LPR not necessarily a power of two) with one vector each, and written out whole.  Several CTAs per SM overlap
// one chunk's copies with another's arithmetic.
#include <algorithm>

#include "bsp_internal.cuh"

namespace bsp {
namespace {

constexpr int kChunk = 64;    // rows per chunk
constexpr int kST = 256;      // threads per CTA

// lo/hi (global rows) of every chunk: the chunk's own rows and all their
// neighbours.  chunks[4 q + 0..1] = (first row, rows) in, [4 q + 2..3] out.
__global__ void k_spmm_ranges(MeshView<float> mv_any, const int32_t* __restrict__ blk_row,
                              int32_t* chunks, int nchunks) {
  const int q = blockIdx.x;
  if (q >= nchunks) return;
  const int row0 = chunks[4 * q], nr = chunks[4 * q + 1];
  const int base = mv_any.bptr[blk_row[row0]];
  int lo = row0, hi = row0 + nr - 1;
  for (int i = threadIdx.x; i < nr; i += blockDim.x) {
    const int row = row0 + i;
    for (int e = mv_any.rowptr[row]; e < mv_any.rowptr[row + 1]; ++e) {
      const int nrw = base + mv_any.col[e];
      lo = min(lo, nrw);
      hi = max(hi, nrw);
    }
  }
  __shared__ int slo[kST / 32], shi[kST / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    slo[threadIdx.x >> 5] = lo;
    shi[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      lo = min(lo, slo[w]);
      hi = max(hi, shi[w]);
    }
    chunks[4 * q + 2] = lo;
    chunks[4 * q + 3] = hi;
  }
}

__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src));
}

template <typename T, int LPR>
__global__ void __launch_bounds__(kST) k_spmm_tile(MeshView<T> mv, const int32_t* __restrict__ blk_row,
                                                  const int32_t* __restrict__ chunks, int span_elems,
                                                  int max_nnz, T delta, const T* __restrict__ P,
                                                  T* __restrict__ Y, int c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int VE = 16 / sizeof(T);
  T* S = reinterpret_cast<T*>(smem_raw);                                  // P[lo..hi]
  T* sdd = S + span_elems;                                                 // D + delta [kChunk]
  T* sw = sdd + kChunk;                                                    // weights (weighted)
  int32_t* sptr = reinterpret_cast<int32_t*>(sw + (mv.wt ? max_nnz : 0));  // kChunk + 1
  uint16_t* scol = reinterpret_cast<uint16_t*>(sptr + kChunk + 1);         // max_nnz
  const int q = blockIdx.x;
  const int row0 = chunks[4 * q], nr = chunks[4 * q + 1];
  const int lo = chunks[4 * q + 2], hi = chunks[4 * q + 3];
  // stage P[lo..hi]: (hi - lo + 1) c elements in 16-byte pieces
  const int pieces = (hi - lo + 1) * c / VE;
  const float4* src = reinterpret_cast<const float4*>(P + (size_t)lo * c);
  float4* dst = reinterpret_cast<float4*>(S);
  for (int t = threadIdx.x; t < pieces; t += kST) cp16(dst + t, src + t);
  asm volatile("cp.async.commit_group;" ::: "memory");
  // the chunk's pattern (row pointers rebased to the chunk, local columns,
  // weights) while the copies are in flight
  const int ebase = mv.rowptr[row0];
  const int nnz = mv.rowptr[row0 + nr] - ebase;
  for (int t = threadIdx.x; t <= nr; t += kST) {
    sptr[t] = mv.rowptr[row0 + t] - ebase;
    if (t < nr) sdd[t] = mv.diag[row0 + t] + delta;
  }
  const int shift = mv.bptr[blk_row[row0]] - lo;   // local column -> row of S
  for (int t = threadIdx.x; t < nnz; t += kST) {
    scol[t] = (uint16_t)(mv.col[ebase + t] + shift);
    if (mv.wt) sw[t] = mv.wt[ebase + t];
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int nv = c / VE;
  const int lane = threadIdx.x % LPR;
  for (int r = threadIdx.x / LPR; r < nr; r += kST / LPR) {
    const int row = row0 + r;
    const int e0 = sptr[r], e1 = sptr[r + 1];
    const T dd = sdd[r];
    for (int v = lane; v < nv; v += LPR) {
      float4 t = reinterpret_cast<const float4*>(S + (size_t)(row - lo) * c)[v];
      T* tp = reinterpret_cast<T*>(&t);
      T acc[VE];
#pragma unroll
      for (int j = 0; j < VE; ++j) acc[j] = dd * tp[j];
#pragma unroll 4
      for (int e = e0; e < e1; ++e) {
        const T w = mv.wt ? sw[e] : T(1);
        float4 u = reinterpret_cast<const float4*>(S + (size_t)scol[e] * c)[v];
        T* up = reinterpret_cast<T*>(&u);
#pragma unroll
        for (int j = 0; j < VE; ++j) acc[j] -= w * up[j];
      }
      float4 o;
      T* op = reinterpret_cast<T*>(&o);
#pragma unroll
      for (int j = 0; j < VE; ++j) op[j] = acc[j];
      reinterpret_cast<float4*>(Y + (size_t)row * c)[v] = o;
    }
  }
}

template <typename T, int LPR>
void launch_tile(const MeshView<T>& mv, const int32_t* blk_row, const int32_t* chunks, int nchunks,
                 int span_elems, int max_nnz, size_t smem, T delta, const T* P, T* Y, int c,
                 cudaStream_t s) {
  k_spmm_tile<T, LPR><<<nchunks, kST, smem, s>>>(mv, blk_row, chunks, span_elems, max_nnz, delta,
                                                 P, Y, c);
}

}  // namespace

void configure_spmm_kernels() {
  set_max_dynamic_smem(k_spmm_tile<float, 1>);
  set_max_dynamic_smem(k_spmm_tile<float, 2>);
  set_max_dynamic_smem(k_spmm_tile<float, 4>);
  set_max_dynamic_smem(k_spmm_tile<float, 8>);
  set_max_dynamic_smem(k_spmm_tile<float, 12>);
  set_max_dynamic_smem(k_spmm_tile<float, 16>);
  set_max_dynamic_smem(k_spmm_tile<float, 24>);
  set_max_dynamic_smem(k_spmm_tile<float, 32>);
  set_max_dynamic_smem(k_spmm_tile<double, 1>);
  set_max_dynamic_smem(k_spmm_tile<double, 2>);
  set_max_dynamic_smem(k_spmm_tile<double, 4>);
  set_max_dynamic_smem(k_spmm_tile<double, 8>);
  set_max_dynamic_smem(k_spmm_tile<double, 12>);
  set_max_dynamic_smem(k_spmm_tile<double, 16>);
  set_max_dynamic_smem(k_spmm_tile<double, 24>);
  set_max_dynamic_smem(k_spmm_tile<double, 32>);
}

// Chunk table (4 int32 per chunk) of a mesh with the given block pointers:
// the first row and row count of every chunk; the ranges follow on the device.
std::vector<int32_t> spmm_chunk_rows(const std::vector<int32_t>& bptr) {
  std::vector<int32_t> ch;
  for (size_t b = 0; b + 1 < bptr.size(); ++b)
    for (int r = bptr[b]; r < bptr[b + 1]; r += kChunk) {
      ch.push_back(r);
      ch.push_back(std::min(kChunk, bptr[b + 1] - r));
      ch.push_back(0);
      ch.push_back(0);
    }
  return ch;
}

void launch_spmm_ranges(const MeshView<float>& mv_any, const int32_t* blk_row, int32_t* chunks,
                        int nchunks, cudaStream_t s) {
  if (nchunks > 0) k_spmm_ranges<<<nchunks, kST, 0, s>>>(mv_any, blk_row, chunks, nchunks);
}

// Tiled product; returns BSP_ERR_INVALID_ARG when the shapes do not suit it
// (rows not a multiple of 16 bytes, unaligned buffers, a chunk range larger
// than shared memory), so that the caller takes the untiled kernel.
template <typename T>
int launch_spmm_tiled(const MeshView<T>& mv, const int32_t* blk_row, const int32_t* chunks,
                      int nchunks, int max_span, int max_nnz, T delta, const T* P, T* Y, int c,
                      cudaStream_t s) {
  constexpr int VE = 16 / sizeof(T);
  if (c % VE != 0 || (uintptr_t)P % 16 != 0 || (uintptr_t)Y % 16 != 0) return BSP_ERR_INVALID_ARG;
  const int span = max_span * c;   // elements of the staged range
  const size_t smem = (size_t)(span + kChunk) * sizeof(T) + (mv.wt ? (size_t)max_nnz * sizeof(T) : 0) +
                      (size_t)(kChunk + 1) * sizeof(int32_t) + (size_t)max_nnz * sizeof(uint16_t) + 16;
  if (smem > 200 * 1024 || nchunks < 1 || max_span > 65535) return BSP_ERR_INVALID_ARG;
  // lanes per row: the 16-byte vectors of a row, rounded up to a listed width
  const int nv = c / VE;
  static const int kL[] = {1, 2, 4, 8, 12, 16, 24, 32};
  int lpr = 32;
  for (int w : kL)
    if (w >= nv) { lpr = w; break; }
  prof_begin(KC_SPMM, s);
#define BSP_TILE(L) launch_tile<T, L>(mv, blk_row, chunks, nchunks, span, max_nnz, smem, delta, P, Y, c, s)
  switch (lpr) {
    case 1: BSP_TILE(1); break;
    case 2: BSP_TILE(2); break;
    case 4: BSP_TILE(4); break;
    case 8: BSP_TILE(8); break;
    case 12: BSP_TILE(12); break;
    case 16: BSP_TILE(16); break;
    case 24: BSP_TILE(24); break;
    default: BSP_TILE(32); break;
  }
#undef BSP_TILE
  prof_end(KC_SPMM, s);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

template int launch_spmm_tiled<float>(const MeshView<float>&, const int32_t*, const int32_t*, int,
                                      int, int, float, const float*, float*, int, cudaStream_t);
template int launch_spmm_tiled<double>(const MeshView<double>&, const int32_t*, const int32_t*,
                                       int, int, int, double, const double*, double*, int,
                                       cudaStream_t);

}  // namespace bsp
