// Tiled operator product Y = (L + delta I) P over all blocks (the sparse x
// tall-skinny product inside every solve of S = R^z, Sec. 4).
//
// Rows are cut into chunks of up to 64 rows inside one block.  A chunk's
// neighbour rows lie in a contiguous range [lo, hi] of the block (its
// bandwidth in local order), computed once per mesh together with the
// chunk's first edge, edge count and column shift, so that a chunk needs no
// dependent global load before its copies can start.
//
// One CTA per chunk stages P[lo..hi] into shared memory with 16-byte
// asynchronous copies (consecutive threads copy consecutive 16-byte pieces:
// fully coalesced; neighbouring chunks run on neighbouring CTAs, so the halo
// rows they share come from L2) and, while they fly, the chunk's pattern with
// columns rebased to rows of the staged range and the diagonal; all of its
// addresses follow from the chunk's table entry.  Then every row of the chunk
// is formed from shared memory only, LPR lanes per row (the row's 16-byte
// vectors, LPR not necessarily a power of two) with one vector each, and
// written out whole.  Several CTAs per SM overlap one chunk's copies with
// another's arithmetic.
#include <algorithm>

#include "bsp_internal.cuh"

namespace bsp {
namespace {

constexpr int kChunk = 64;    // rows per chunk
constexpr int kST = 256;      // threads per CTA

// Completes the chunk table: chunks[8 q + 0..1] = (first row, rows) in;
// [8 q + 2..6] = lo, hi (global rows reached by the chunk and its
// neighbours), first edge, edge count, and the shift from a local column to
// a row of the staged range [lo, hi].
__global__ void k_spmm_ranges(MeshView<float> mv_any, const int32_t* __restrict__ blk_row,
                              int32_t* chunks, int nchunks) {
  const int q = blockIdx.x;
  if (q >= nchunks) return;
  const int row0 = chunks[8 * q], nr = chunks[8 * q + 1];
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
    const int e0 = mv_any.rowptr[row0];
    chunks[8 * q + 2] = lo;
    chunks[8 * q + 3] = hi;
    chunks[8 * q + 4] = e0;
    chunks[8 * q + 5] = mv_any.rowptr[row0 + nr] - e0;
    chunks[8 * q + 6] = base - lo;
    chunks[8 * q + 7] = 0;
  }
}

__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// One chunk's table entry.
struct ChunkMeta {
  int row0, nr, lo, hi, e0, nnz, shift;
};
__device__ __forceinline__ ChunkMeta load_meta(const int32_t* chunks, int q) {
  const int4 a = __ldg(reinterpret_cast<const int4*>(chunks) + 2 * q);
  const int4 b = __ldg(reinterpret_cast<const int4*>(chunks) + 2 * q + 1);
  return {a.x, a.y, a.z, a.w, b.x, b.y, b.z};
}

// Shared-memory stage: P[lo..hi] (span_elems), D + delta [kChunk], weights
// [max_nnz] (weighted meshes), row pointers [kChunk + 1], rebased columns
// [max_nnz].
template <typename T>
struct Stage {
  T* S;
  T* dd;
  T* w;
  int32_t* ptr;
  uint16_t* col;
  BSP_DEV Stage(unsigned char* base, int span_elems, int max_nnz, bool weighted) {
    S = reinterpret_cast<T*>(base);
    dd = S + span_elems;
    w = dd + kChunk;
    ptr = reinterpret_cast<int32_t*>(w + (weighted ? max_nnz : 0));
    col = reinterpret_cast<uint16_t*>(ptr + kChunk + 1);
  }
};

template <typename T, int LPR>
BSP_DEV void form_rows(const MeshView<T>& mv, const ChunkMeta& m, const Stage<T>& st,
                       T* __restrict__ Y, int c) {
  constexpr int VE = 16 / sizeof(T);
  const int nv = c / VE;
  const int lane = threadIdx.x % LPR;
  for (int r = threadIdx.x / LPR; r < m.nr; r += kST / LPR) {
    const int row = m.row0 + r;
    const int e0 = st.ptr[r], e1 = st.ptr[r + 1];
    const T dd = st.dd[r];
    for (int v = lane; v < nv; v += LPR) {
      float4 t = reinterpret_cast<const float4*>(st.S + (size_t)(row - m.lo) * c)[v];
      T* tp = reinterpret_cast<T*>(&t);
      T acc[VE];
#pragma unroll
      for (int j = 0; j < VE; ++j) acc[j] = dd * tp[j];
#pragma unroll 4
      for (int e = e0; e < e1; ++e) {
        const T w = mv.wt ? st.w[e] : T(1);
        float4 u = reinterpret_cast<const float4*>(st.S + (size_t)st.col[e] * c)[v];
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
__global__ void __launch_bounds__(kST) k_spmm_tile(MeshView<T> mv, const int32_t* __restrict__ chunks,
                                                  int span_elems, int max_nnz, T delta,
                                                  const T* __restrict__ P, T* __restrict__ Y, int c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int VE = 16 / sizeof(T);
  const Stage<T> st(smem_raw, span_elems, max_nnz, mv.wt != nullptr);
  const ChunkMeta m = load_meta(chunks, blockIdx.x);
  // P[lo..hi]: (hi - lo + 1) c elements in 16-byte pieces
  const int pieces = (m.hi - m.lo + 1) * c / VE;
  const float4* src = reinterpret_cast<const float4*>(P + (size_t)m.lo * c);
  float4* dst = reinterpret_cast<float4*>(st.S);
  for (int t = threadIdx.x; t < pieces; t += kST) cp16(dst + t, src + t);
  cp_commit();
  // the pattern while the copies are in flight: row pointers rebased to the
  // chunk, columns rebased to rows of the staged range, weights, diagonal
  for (int t = threadIdx.x; t <= m.nr; t += kST) {
    st.ptr[t] = __ldg(mv.rowptr + m.row0 + t) - m.e0;
    if (t < m.nr) st.dd[t] = __ldg(mv.diag + m.row0 + t) + delta;
  }
  for (int t = threadIdx.x; t < m.nnz; t += kST) {
    st.col[t] = (uint16_t)(__ldg(mv.col + m.e0 + t) + m.shift);
    if (mv.wt) st.w[t] = __ldg(mv.wt + m.e0 + t);
  }
  cp_wait<0>();
  __syncthreads();
  form_rows<T, LPR>(mv, m, st, Y, c);
}

template <typename T, int LPR>
void launch_tile(const MeshView<T>& mv, const int32_t* chunks, int nchunks, int span_elems,
                 int max_nnz, size_t smem, T delta, const T* P, T* Y, int c, cudaStream_t s) {
  k_spmm_tile<T, LPR><<<nchunks, kST, smem, s>>>(mv, chunks, span_elems, max_nnz, delta, P, Y, c);
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

// Chunk table (8 int32 per chunk) of a mesh with the given block pointers:
// the first row and row count of every chunk; the rest follows on the device.
std::vector<int32_t> spmm_chunk_rows(const std::vector<int32_t>& bptr) {
  std::vector<int32_t> ch;
  for (size_t b = 0; b + 1 < bptr.size(); ++b)
    for (int r = bptr[b]; r < bptr[b + 1]; r += kChunk) {
      ch.push_back(r);
      ch.push_back(std::min(kChunk, bptr[b + 1] - r));
      for (int z = 0; z < 6; ++z) ch.push_back(0);
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
int launch_spmm_tiled(const MeshView<T>& mv, const int32_t* chunks, int nchunks, int max_span,
                      int max_nnz, T delta, const T* P, T* Y, int c, cudaStream_t s) {
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
#define BSP_TILE(L) launch_tile<T, L>(mv, chunks, nchunks, span, max_nnz, smem, delta, P, Y, c, s)
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

template int launch_spmm_tiled<float>(const MeshView<float>&, const int32_t*, int, int, int, float,
                                      const float*, float*, int, cudaStream_t);
template int launch_spmm_tiled<double>(const MeshView<double>&, const int32_t*, int, int, int,
                                       double, const double*, double*, int, cudaStream_t);

}  // namespace bsp
