// Persistent cluster engine for the fixed-c OI schedule (Sec. 4, Algorithm 1,
// with the warm start of each submesh from the previous one's subspace).
//
// One thread-block cluster of P = ceil(c / 4) CTAs owns one dependency path
// of the block DAG at a time and runs every step of a block on chip, in one
// launch for the whole schedule:
//
//   * the z t_max solves (L + delta I) Y = V of S = R^z (Sec. 4, below
//     Algorithm 1), by Chronopoulos-Gear CG: CTA q owns columns 4q .. 4q+3
//     of the block for all its rows, so a solve never leaves the CTA (one
//     CTA-wide reduction of 8 scalars per step, neighbour rows gathered from
//     a shared-memory copy of the residual, the pattern held as ELL in
//     registers);
//   * Onorm (Sec. 4) by CholeskyQR2: the solves' output is re-distributed
//     through distributed shared memory so that CTA q owns a panel of rows
//     with all columns; partial Grams are summed across the cluster by a
//     reduce-scatter and broadcast; every CTA factorises the c x c Gram
//     itself (identical inputs, identical results), with the factor's
//     inverse built alongside on the identity, and applies it to its panel.
//     This is one CholeskyQR pass: its output spans the same subspace and is
//     orthonormal to O(kappa^2 u), which is all the next solve needs.  The
//     second pass, which only restores orthonormality to working precision,
//     runs after the engine, batched over all blocks (the host enqueues it);
//   * the orthonormal panel goes back to the column layout in the CTAs'
//     shared memory, where the next block of the path reads its start (same
//     size: row r of the child starts from row r of the parent), and to U in
//     HBM.
//
// Several clusters run independent paths of a forest; a block whose parent
// was processed by another cluster waits for the parent's ready flag with a
// bounded wait (globaltimer deadline): on expiry the cluster stops, flags
// ST_TIMEOUT and sets an abort word that every other waiter also honours.
// Every decision that steers a cluster barrier is uniform over the cluster.
#include "bsp_internal.cuh"

namespace bsp {
namespace {

constexpr int kNT = 512;                 // threads per CTA (16 warps)
constexpr int kWarps = kNT / 32;
constexpr int kCMax = 64;                // widest basis (16 CTAs x 4 columns)
constexpr int kLDA = kCMax + 4;          // row stride of the c x c work matrices

// ---------------------------------------------------------------- cluster helpers
BSP_DEV uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
BSP_DEV uint32_t remote(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
BSP_DEV void st_remote4(uint32_t a, float4 v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};"
               ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}
BSP_DEV void st_remote(uint32_t a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
BSP_DEV void st_remote_i(uint32_t a, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
BSP_DEV float ld_remote(uint32_t a) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}
// All threads of all CTAs of the cluster; orders shared (local and remote)
// and global accesses before it against those after it, cluster-wide.
BSP_DEV void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
BSP_DEV uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
BSP_DEV uint32_t cluster_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
BSP_DEV uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
BSP_DEV int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
BSP_DEV void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------- CTA reduction
// Sum 8 per-thread values over the CTA; every thread receives the 8 sums.
// Within a warp the values are halved at each butterfly level (xor 16, 8, 4
// keep one half each), so lane l ends with the warp sum of value
// 4 b4 + 2 b3 + b2 (b = bits of l) after 9 shuffles; lanes 4m write them, one
// barrier, then every warp reads the 16 x 8 partials (one float4 per lane)
// and reduces them the same way.  `red` holds 2 x 16 x 8 floats; `buf`
// alternates so one barrier per reduction suffices.
BSP_DEV void reduce8(float (&v)[8], float* red, int& buf) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float h[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool up = lane & 16;
    const float send = up ? v[k] : v[k + 4], keep = up ? v[k + 4] : v[k];
    h[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float g[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const bool up = lane & 8;
    const float send = up ? h[k] : h[k + 2], keep = up ? h[k + 2] : h[k];
    g[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float t;
  {
    const bool up = lane & 4;
    const float send = up ? g[0] : g[1], keep = up ? g[1] : g[0];
    t = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  float* rb = red + buf * (kWarps * 8);
  if ((lane & 3) == 0) rb[w * 8 + ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1)] = t;
  __syncthreads();
  // lane l: warps (l & 15), values 4 (l >> 4) .. +3
  const float4 q = *reinterpret_cast<const float4*>(rb + (lane & 15) * 8 + (lane >> 4) * 4);
  float a[4] = {q.x, q.y, q.z, q.w};
  float b2[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const bool up = lane & 8;
    const float send = up ? a[k] : a[k + 2], keep = up ? a[k + 2] : a[k];
    b2[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  {
    const bool up = lane & 4;
    const float send = up ? b2[0] : b2[1], keep = up ? b2[1] : b2[0];
    t = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  // lane l holds value 4 b4 + 2 b3 + b2; gather all 8
#pragma unroll
  for (int k = 0; k < 8; ++k)
    v[k] = __shfl_sync(0xffffffffu, t, ((k >> 2) << 4) | (((k >> 1) & 1) << 3) | ((k & 1) << 2));
  buf ^= 1;
}

// ---------------------------------------------------------------- block pattern
// Rows i = threadIdx.x + kNT m of the block, m < MAXR.  ELL of the
// off-diagonal part of L: local neighbour ids (padding -> CAP, the zero slot
// of the shared vector), weights (WEIGHTED only), D_ii + delta.
template <int MAXR, int ELLW, bool WEIGHTED>
struct Pattern {
  uint16_t nb[MAXR][ELLW];
  float wt[WEIGHTED ? MAXR : 1][WEIGHTED ? ELLW : 1];
  float dd[MAXR];

  float nrm;   // Gershgorin bound of ||L + delta I||_2 over the block (same in every thread)

  // Loads the rows' pattern and forms nrm with one CTA-wide max (scratch: 16
  // floats, two barriers).
  BSP_DEV void load(const MeshView<float>& mv, int r0, int nbk, float delta, float* scratch) {
    constexpr int CAP = MAXR * kNT;
    float bound = 0.f;
#pragma unroll
    for (int m = 0; m < MAXR; ++m) {
      const int i = threadIdx.x + kNT * m;
      int e0 = 0, dg = 0;
      dd[m] = 0.f;
      if (i < nbk) {
        e0 = __ldg(mv.rowptr + r0 + i);
        dg = __ldg(mv.rowptr + r0 + i + 1) - e0;
        dd[m] = __ldg(mv.diag + r0 + i) + delta;
      }
      float row = dd[m];
#pragma unroll
      for (int e = 0; e < ELLW; ++e) {
        const bool ok = e < dg;
        nb[m][e] = ok ? __ldg(mv.col + e0 + e) : (uint16_t)CAP;
        if constexpr (WEIGHTED) {
          wt[m][e] = ok ? __ldg(mv.wt + e0 + e) : 0.f;
          row += fabsf(wt[m][e]);
        } else {
          row += ok ? 1.f : 0.f;
        }
      }
      bound = fmaxf(bound, row);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bound = fmaxf(bound, __shfl_xor_sync(0xffffffffu, bound, o));
    if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = bound;
    __syncthreads();
    nrm = 0.f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) nrm = fmaxf(nrm, scratch[w]);
    __syncthreads();
  }

  // out = (L + delta I) v for the 4 columns, v's neighbour rows from rs
  BSP_DEV void apply(const float4* rs, const float (&v)[MAXR][4], float (&out)[MAXR][4]) const {
#pragma unroll
    for (int m = 0; m < MAXR; ++m) {
      float a0 = dd[m] * v[m][0], a1 = dd[m] * v[m][1], a2 = dd[m] * v[m][2], a3 = dd[m] * v[m][3];
#pragma unroll
      for (int e = 0; e < ELLW; ++e) {
        const float4 p = rs[nb[m][e]];
        if constexpr (WEIGHTED) {
          const float w = wt[m][e];
          a0 -= w * p.x; a1 -= w * p.y; a2 -= w * p.z; a3 -= w * p.w;
        } else {
          a0 -= p.x; a1 -= p.y; a2 -= p.z; a3 -= p.w;
        }
      }
      out[m][0] = a0; out[m][1] = a1; out[m][2] = a2; out[m][3] = a3;
    }
  }
};

template <int MAXR>
BSP_DEV void put_rows(float4* rs, const float (&v)[MAXR][4], int nbk) {
#pragma unroll
  for (int m = 0; m < MAXR; ++m) {
    const int i = threadIdx.x + kNT * m;
    if (i < nbk) rs[i] = make_float4(v[m][0], v[m][1], v[m][2], v[m][3]);
  }
}

struct CgCount {
  long long total = 0;
  int max = 0;
  bool unconverged = false, breakdown = false;
};

// g solves A x = b for the CTA's 4 columns (A = L + delta I): the first
// right-hand side is in rs (column layout), the next one is the previous
// solution.  ncol: columns of this CTA that exist (the rest stay 0).
// Returns the last solution in x.  Leaves rs in use: callers synchronise
// before rewriting it.
// Stopping rule per column: ||r|| <= max(rtol ||b||, u (||b|| + ||A|| ||x0||)),
// u = 2^-24.  The second term is the level below which an FP32 residual
// b - A x cannot be computed (its rounding error is of that size), so
// iterating further only shrinks the recursively updated residual, not the
// error of x; it matters for the columns whose solution is much larger than
// the right-hand side (the lowest ones, x ~ b / delta).  ||A|| is bounded by
// the block's Gershgorin radius and x0 = b (b, b) / (b, A b).
template <int MAXR, int ELLW, bool WEIGHTED>
BSP_DEV void cg_group(const Pattern<MAXR, ELLW, WEIGHTED>& pat, float4* rs, float* red, int& buf,
                      int nbk, int ncol, int g, float rtol2, int max_steps,
                      float (&x)[MAXR][4], CgCount& cnt) {
  float bv[MAXR][4], r[MAXR][4], p[MAXR][4], s[MAXR][4], w[MAXR][4];
#pragma unroll
  for (int m = 0; m < MAXR; ++m) {
    const int i = threadIdx.x + kNT * m;
    const float4 t = i < nbk ? rs[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    bv[m][0] = t.x; bv[m][1] = t.y; bv[m][2] = t.z; bv[m][3] = t.w;
  }
  for (int sol = 0; sol < g; ++sol) {
    if (sol > 0) {
      __syncthreads();                 // every gather of the previous solve is done
      put_rows<MAXR>(rs, bv, nbk);
      __syncthreads();
    }
    // x0 = b (b, b) / (b, A b)
    pat.apply(rs, bv, w);
    float sums[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float bb = 0.f, bab = 0.f;
#pragma unroll
      for (int m = 0; m < MAXR; ++m) { bb += bv[m][j] * bv[m][j]; bab += bv[m][j] * w[m][j]; }
      sums[j] = bb;
      sums[4 + j] = bab;
    }
    reduce8(sums, red, buf);
    float bn2[4], alpha[4], gam[4], dlt[4];
    bool act[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float gf = sums[4 + j] > 0.f ? __fdividef(sums[j], sums[4 + j]) : 0.f;
      const float nb = sqrtf(sums[j]);
      const float fl = 5.9604645e-8f * nb * (1.f + pat.nrm * fabsf(gf));   // u (||b|| + ||A|| ||x0||)
      bn2[j] = fmaxf(rtol2 * sums[j], fl * fl);
#pragma unroll
      for (int m = 0; m < MAXR; ++m) {
        x[m][j] = gf * bv[m][j];
        r[m][j] = bv[m][j] - gf * w[m][j];
      }
    }
    put_rows<MAXR>(rs, r, nbk);        // the gathers above finished before reduce8's barrier
    __syncthreads();
    pat.apply(rs, r, w);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float gl = 0.f, dl = 0.f;
#pragma unroll
      for (int m = 0; m < MAXR; ++m) { gl += r[m][j] * r[m][j]; dl += w[m][j] * r[m][j]; }
      sums[j] = gl;
      sums[4 + j] = dl;
    }
    reduce8(sums, red, buf);
    bool any = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      gam[j] = sums[j];
      dlt[j] = sums[4 + j];
      alpha[j] = dlt[j] > 0.f ? __fdividef(gam[j], dlt[j]) : 0.f;
      act[j] = j < ncol && gam[j] > bn2[j];
      any = any || act[j];
#pragma unroll
      for (int m = 0; m < MAXR; ++m) { p[m][j] = r[m][j]; s[m][j] = w[m][j]; }
    }
    int steps = 0, col_steps = 0;
    // converged columns keep x and r (step length 0); no branches on the columns
    while (any) {
      if (steps >= max_steps) { cnt.unconverged = true; break; }
      float ae[4], be[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bool ok = act[j] && dlt[j] > 0.f;   // (p, A p) <= 0: the recurrence broke down
        cnt.breakdown = cnt.breakdown || (act[j] && !ok);
        act[j] = ok;
        col_steps += ok ? 1 : 0;
        ae[j] = ok ? alpha[j] : 0.f;
      }
#pragma unroll
      for (int m = 0; m < MAXR; ++m)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          x[m][j] += ae[j] * p[m][j];
          r[m][j] -= ae[j] * s[m][j];
        }
      put_rows<MAXR>(rs, r, nbk);
      __syncthreads();
      pat.apply(rs, r, w);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float gl = 0.f, dl = 0.f;
#pragma unroll
        for (int m = 0; m < MAXR; ++m) { gl += r[m][j] * r[m][j]; dl += w[m][j] * r[m][j]; }
        sums[j] = gl;
        sums[4 + j] = dl;
      }
      reduce8(sums, red, buf);
      ++steps;
      any = false;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float gnew = sums[j], dnew = sums[4 + j];
        const bool go = act[j] && gnew > bn2[j];
        const float beta = go ? __fdividef(gnew, gam[j]) : 0.f;
        const float den = go ? dnew - beta * __fdividef(gnew, alpha[j]) : 1.f;
        const bool ok = go && den > 0.f;
        cnt.breakdown = cnt.breakdown || (go && !ok);
        alpha[j] = ok ? __fdividef(gnew, den) : 0.f;
        gam[j] = ok ? gnew : gam[j];
        dlt[j] = ok ? den : dlt[j];
        act[j] = ok;
        be[j] = ok ? beta : 0.f;
        any = any || ok;
      }
#pragma unroll
      for (int m = 0; m < MAXR; ++m)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          p[m][j] = r[m][j] + be[j] * p[m][j];
          s[m][j] = w[m][j] + be[j] * s[m][j];
        }
    }
    cnt.total += col_steps;
    cnt.max = max(cnt.max, steps);
#pragma unroll
    for (int m = 0; m < MAXR; ++m)
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[m][j] = x[m][j];
  }
}

// ---------------------------------------------------------------- Onorm pieces
// Shared-memory work area of one CTA for the c x c part of CholeskyQR2.
struct Dense {
  float* Gp;     // [64 x 64] partial Gram of this CTA's panel (also the T buffer of the inverse)
  float* A;      // [64 x kLDA] the summed Gram, then R (upper)
  float* M;      // [64 x kLDA] the right factor applied to the panel
  float4* PT;    // [144] rows K..K+7 of R, per column at col8(j) (Cholesky panel)
  float* dinv;   // [2 x 64] inverses of R's 8 x 8 diagonal blocks (alternating)
  float* dsc;    // [64] Jacobi scaling
  float* red;    // 2 x 16 x 8 reduction buffer
  int* ctl;      // [8] cluster-uniform control words
};

// Partial Gram Gp = S^T S of the panel (nr rows, cpad columns, row stride ldp):
// upper 4 x 4 tiles only, each tile split over 4 lanes by row residue mod 4
// and summed by shuffles (lane part p ends with tile row p).
BSP_DEV void gram_partial(const float* S, int nr, int ldp, int cpad, float* Gp) {
  const int nt = cpad >> 2, ntile = nt * (nt + 1) / 2, items = ntile * 4;
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < items; base += kNT) {
    if (base + (threadIdx.x & ~31) >= items) break;     // whole warp past the end
    const int it = base + threadIdx.x;
    const bool valid = it < items;
    const int part = it & 3;
    int u = valid ? (it >> 2) : 0, ti = 0;
    while (u >= nt - ti) { u -= nt - ti; ++ti; }
    const int tj = ti + u;
    float acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.f;
    if (valid) {
      for (int r = part; r < nr; r += 4) {
        const float4 a = *reinterpret_cast<const float4*>(S + r * ldp + 4 * ti);
        const float4 b = *reinterpret_cast<const float4*>(S + r * ldp + 4 * tj);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[4 * i + j] += av[i] * bv[j];
      }
    }
    // 16 values over 4 lanes: keep rows {0,1} / {2,3} by bit 1, then one row by bit 0
    float h[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const bool up = lane & 2;
      const float send = up ? acc[k] : acc[k + 8], keep = up ? acc[k + 8] : acc[k];
      h[k] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    float o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool up = lane & 1;
      const float send = up ? h[k] : h[k + 4], keep = up ? h[k + 4] : h[k];
      o[k] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
    }
    if (valid) {
      const int row = 4 * ti + ((lane >> 1) & 1) * 2 + (lane & 1);
      *reinterpret_cast<float4*>(Gp + row * 64 + 4 * tj) = make_float4(o[0], o[1], o[2], o[3]);
    }
  }
}

// Every CTA's A (upper triangle, rows 0 .. cpad-1) = sum over the P CTAs of
// their Gp, in rank order.  CTA q sums rows 4q .. 4q+3 (columns >= 4q) and
// writes them into all P CTAs.  Caller: cluster_sync before (partials
// complete) and after (rows delivered).
BSP_DEV void gram_allreduce(const Dense& d, int q, int P, int cpad) {
  const int w = cpad - 4 * q, cnt = 4 * w;
  const uint32_t gp = smem_addr(d.Gp), aa = smem_addr(d.A);
  for (int e = threadIdx.x; e < cnt; e += kNT) {
    const int row = 4 * q + e / w, col = 4 * q + e % w;
    const uint32_t off = (uint32_t)(row * 64 + col) * 4u;
    float s = 0.f;
    for (int src = 0; src < P; ++src) s += ld_remote(remote(gp + off, src));
    const uint32_t offa = (uint32_t)(row * kLDA + col) * 4u;
    for (int dst = 0; dst < P; ++dst) st_remote(remote(aa + offa, dst), s);
  }
}

BSP_DEV float dot4(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
BSP_DEV float dot8(const float4* a, const float4* b) { return dot4(a[0], b[0]) + dot4(a[1], b[1]); }
// Column j's 8 values in the per-column panels PT / BT: float4 index 2j + j/4
// (16 bytes of skew every 4 columns, so the column groups 4 t that one warp
// reads for different tiles t fall into different shared-memory banks).
BSP_DEV int col8(int j) { return 2 * j + (j >> 2); }

// Cholesky of the symmetric 8 x 8 diagonal block of A at (K, K) (upper
// entries, already updated) by one thread, in registers: writes W = R^-1
// (upper, row-major 8 x 8, zeros below) to w.  A non-positive or non-finite
// pivot is replaced by 1 and reported in *fail.
BSP_DEV void factor8(const float* A, int K, float* w, int* fail) {
  float R[8][8], W[8][8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {   // whole rows as float4 (only r >= q is used)
    const float4 a0 = *reinterpret_cast<const float4*>(A + (K + q) * kLDA + K);
    const float4 a1 = *reinterpret_cast<const float4*>(A + (K + q) * kLDA + K + 4);
    R[q][0] = a0.x; R[q][1] = a0.y; R[q][2] = a0.z; R[q][3] = a0.w;
    R[q][4] = a1.x; R[q][5] = a1.y; R[q][6] = a1.z; R[q][7] = a1.w;
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float sq = R[q][q];
#pragma unroll
    for (int p = 0; p < q; ++p) sq -= R[p][q] * R[p][q];
    if (!(sq > 0.f) || !isfinite(sq)) { *fail = 1; sq = 1.f; }
    const float rq = rsqrtf(sq);
    R[q][q] = sq * rq;
    W[q][q] = rq;
#pragma unroll
    for (int r = q + 1; r < 8; ++r) {
      float t = R[q][r];
#pragma unroll
      for (int p = 0; p < q; ++p) t -= R[p][q] * R[p][r];
      R[q][r] = t * rq;
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int r = q + 1; r < 8; ++r) {
      float t = 0.f;
#pragma unroll
      for (int p = q; p < r; ++p) t += W[q][p] * R[p][r];
      W[q][r] = -t * W[r][r];
    }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float row[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) row[r] = r >= q ? W[q][r] : 0.f;
    *reinterpret_cast<float4*>(w + 8 * q) = make_float4(row[0], row[1], row[2], row[3]);
    *reinterpret_cast<float4*>(w + 8 * q + 4) = make_float4(row[4], row[5], row[6], row[7]);
  }
}

// Upper-triangle tile (ti, tj) of a T x T tile grid, ti <= tj, from its
// row-major index u (closed form, corrected by at most one step).
BSP_DEV void upper_tile(int T, int u, int& ti, int& tj) {
  const float b = 2.f * T + 1.f;
  int t = (int)(0.5f * (b - sqrtf(fmaxf(b * b - 8.f * u, 0.f))));
  auto off = [T](int r) { return r * T - (r * (r - 1)) / 2; };
  if (t > 0 && off(t) > u) --t;
  if (t + 1 < T && off(t + 1) <= u) ++t;
  ti = t;
  tj = t + (u - off(t));
}

// M = D R^-1 for the Jacobi-scaled Cholesky D G D = R^T R (G in A's upper
// triangle, rows and columns >= c already the identity; padded to a multiple
// of 8 with the identity).  Right-looking, blocked by 8.  The elimination
// that turns D G D into R is applied to the identity alongside (B, lower
// triangular, in M's storage), which leaves B = R^-T: no separate inversion.
// Per block step: W = R_KK^-1 is known; the threads of the columns form the
// block's 8 rows of R (PT) and of B (BT); then warp 0 updates the next
// diagonal block and one lane factorises it in registers, while the other
// warps update the trailing part of A and the rows of B below the block.
// Two barriers per block step.  Ends with a barrier.
BSP_DEV void chol_inverse(const Dense& d, int cpad) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cp8 = (cpad + 7) & ~7, nt = cp8 >> 3;
  float* A = d.A;
  float* B = d.M;
  float4* PT = d.PT;                                // 8 rows of R per column at col8(j)
  float4* BT = reinterpret_cast<float4*>(d.Gp);     // 8 new rows of B per column
  for (int i = tid; i < cp8; i += kNT) {
    float sc = 1.f;
    if (i < cpad) {
      const float g = A[i * kLDA + i];
      const bool ok = g > 0.f && isfinite(g);
      if (!ok) d.ctl[1] = 1;
      sc = ok ? rsqrtf(g) : 1.f;
    }
    d.dsc[i] = sc;
  }
  __syncthreads();
  for (int i = warp; i < cp8; i += kWarps)
    for (int j = lane; j < cp8; j += 32) {
      if (i >= cpad || j >= cpad) A[i * kLDA + j] = i == j ? 1.f : 0.f;
      else if (j >= i) A[i * kLDA + j] *= d.dsc[i] * d.dsc[j];
      B[i * kLDA + j] = i == j ? 1.f : 0.f;
    }
  __syncthreads();
  if (tid == 0) factor8(A, 0, d.dinv, &d.ctl[1]);
  __syncthreads();
  for (int kb = 0; kb < nt; ++kb) {
    const int K = 8 * kb;
    const float* W = d.dinv + (kb & 1) * 64;
    // rows K..K+7 of R (A columns > K+7) and of B (B columns <= K+7): x <- W^T x
    if (tid < cp8) {
      const int j = tid;
      const bool inB = j < K + 8;
      const float* src = inB ? B : A;
      float a[8], r[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = src[(K + q) * kLDA + j];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float t = 0.f;
#pragma unroll
        for (int p = 0; p <= q; ++p) t += W[p * 8 + q] * a[p];
        r[q] = t;
      }
      const float4 lo = make_float4(r[0], r[1], r[2], r[3]), hi = make_float4(r[4], r[5], r[6], r[7]);
      if (inB) {
#pragma unroll
        for (int q = 0; q < 8; ++q) B[(K + q) * kLDA + j] = r[q];
        BT[col8(j)] = lo;
        BT[col8(j) + 1] = hi;
      } else {
        PT[col8(j)] = lo;
        PT[col8(j) + 1] = hi;
        // a column of the next diagonal block updates its own diagonal entry
        // (the rest of that block is warp 0's below)
        if (j >= K + 8 && j < K + 16) A[j * kLDA + j] -= dot4(lo, lo) + dot4(hi, hi);
      }
    }
    __syncthreads();
    if (kb + 1 == nt) break;
    const int K8 = K + 8;
    if (warp == 0) {
      // next diagonal block: its 28 strictly upper entries, one per lane
      // (row q holds 7 - q of them), then one lane factorises it
      if (lane < 28) {
        const int e = lane;
        const int q = (e >= 7) + (e >= 13) + (e >= 18) + (e >= 22) + (e >= 25) + (e >= 27);
        const int r = q + 1 + e - (7 * q - (q * (q - 1)) / 2);
        A[(K8 + q) * kLDA + K8 + r] -= dot8(PT + col8(K8 + q), PT + col8(K8 + r));
      }
      __syncwarp();
      if (lane == 0) factor8(A, K8, d.dinv + ((kb + 1) & 1) * 64, &d.ctl[1]);
    } else {
      const int t0 = K8 >> 2, T = (cp8 >> 2) - t0;    // trailing 4 x 4 tile grid
      const int na = 4 * (T * (T + 1) / 2 - 3);        // but the next diagonal block's 3 tiles
      const int nb = (cp8 - K8) * (K8 >> 2);           // B rows below x column groups
      const float inv_g = 1.f / (float)(K8 >> 2);
      for (int it = tid - 32; it < na + nb; it += kNT - 32) {
        if (it < na) {
          // skip tiles (0,0), (0,1) (u = 0, 1) and (1,1) (u = T)
          int u = (it >> 2) + 2;
          if (u >= T) ++u;
          int ti, tj;
          upper_tile(T, u, ti, tj);
          const int i = 4 * (t0 + ti) + (it & 3), j0 = 4 * (t0 + tj);
          const float4* pi = PT + col8(i);
          float4 v = *reinterpret_cast<float4*>(A + i * kLDA + j0);
          v.x -= dot8(pi, PT + col8(j0));
          v.y -= dot8(pi, PT + col8(j0 + 1));
          v.z -= dot8(pi, PT + col8(j0 + 2));
          v.w -= dot8(pi, PT + col8(j0 + 3));
          *reinterpret_cast<float4*>(A + i * kLDA + j0) = v;
        } else {
          const int e = it - na;
          const int row = __float2int_rz(((float)e + 0.5f) * inv_g);
          const int g = e - row * (K8 >> 2);
          const int i = K8 + row, j0 = 4 * g;
          const float4* pi = PT + col8(i);
          float4 v = *reinterpret_cast<float4*>(B + i * kLDA + j0);
          v.x -= dot8(pi, BT + col8(j0));
          v.y -= dot8(pi, BT + col8(j0 + 1));
          v.z -= dot8(pi, BT + col8(j0 + 2));
          v.w -= dot8(pi, BT + col8(j0 + 3));
          *reinterpret_cast<float4*>(B + i * kLDA + j0) = v;
        }
      }
    }
    __syncthreads();
  }
  // B = R^-T (lower); M = D R^-1 = D B^T in the same storage, lower part zero
  for (int i = warp; i < cpad; i += kWarps)
    for (int j = i + lane; j < cpad; j += 32) {
      const float bji = B[j * kLDA + i];
      B[i * kLDA + j] = d.dsc[i] * bji;
      if (j > i) B[j * kLDA + i] = 0.f;
    }
  __syncthreads();
}

// S <- S M for the panel (nr rows, cpad columns; M upper triangular).  Warp
// items = (column group of 4, chunk of 64 rows); lane = pair of rows.  Every
// warp has at most 2 items (checked by the launcher).  Ends with a barrier.
BSP_DEV void apply_right(float* S, int nr, int ldp, int cpad, const float* M) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ng = cpad >> 2, nch = (nr + 63) >> 6, items = ng * nch;
  float acc[2][2][4];
  int its[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int it = w + kWarps * s;
    its[s] = it;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[s][q][j] = 0.f;
    if (it >= items) continue;
    const int grp = it % ng, ch = it / ng;
    const int r = ch * 64 + 2 * lane;
    const bool v0 = r < nr, v1 = r + 1 < nr;
    const int kend = 4 * grp + 4;
    for (int k = 0; k < kend; k += 4) {
      const float4 sa = v0 ? *reinterpret_cast<const float4*>(S + r * ldp + k) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 sb = v1 ? *reinterpret_cast<const float4*>(S + (r + 1) * ldp + k) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float xa[4] = {sa.x, sa.y, sa.z, sa.w}, xb[4] = {sb.x, sb.y, sb.z, sb.w};
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const float4 m = *reinterpret_cast<const float4*>(M + (k + kk) * kLDA + 4 * grp);
        acc[s][0][0] += xa[kk] * m.x; acc[s][0][1] += xa[kk] * m.y;
        acc[s][0][2] += xa[kk] * m.z; acc[s][0][3] += xa[kk] * m.w;
        acc[s][1][0] += xb[kk] * m.x; acc[s][1][1] += xb[kk] * m.y;
        acc[s][1][2] += xb[kk] * m.z; acc[s][1][3] += xb[kk] * m.w;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int it = its[s];
    if (it >= items) continue;
    const int grp = it % ng, ch = it / ng;
    const int r = ch * 64 + 2 * lane;
    if (r < nr)
      *reinterpret_cast<float4*>(S + r * ldp + 4 * grp) =
          make_float4(acc[s][0][0], acc[s][0][1], acc[s][0][2], acc[s][0][3]);
    if (r + 1 < nr)
      *reinterpret_cast<float4*>(S + (r + 1) * ldp + 4 * grp) =
          make_float4(acc[s][1][0], acc[s][1][1], acc[s][1][2], acc[s][1][3]);
  }
  __syncthreads();
}

// ---------------------------------------------------------------- the kernel
template <int MAXR, int ELLW, bool WEIGHTED>
__global__ void __launch_bounds__(kNT, 1) k_oi_cluster(MeshView<float> mv, OiClusterArgs a) {
  constexpr int CAP = MAXR * kNT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = (int)cluster_size(), q = (int)cluster_rank();
  const int cl = blockIdx.x / P, ncl = gridDim.x / P;
  const int c = a.c, cpad = 4 * P, ldp = cpad + 4;
  const int tid = threadIdx.x;
  // shared memory carve-up (the launcher sizes it the same way)
  float4* rs = reinterpret_cast<float4*>(smem_raw);              // [CAP + 1] column layout
  float* S = reinterpret_cast<float*>(rs + CAP + 1);              // [rpm x ldp] row panel
  Dense d;
  d.Gp = S + a.rpm * ldp;
  d.A = d.Gp + 64 * 64;
  d.M = d.A + 64 * kLDA;
  d.PT = reinterpret_cast<float4*>(d.M + 64 * kLDA);
  d.dinv = reinterpret_cast<float*>(d.PT + 144);
  d.dsc = d.dinv + 128;
  d.red = d.dsc + 64;
  d.ctl = reinterpret_cast<int*>(d.red + 2 * kWarps * 8 + kWarps);
  if (tid < 8) d.ctl[tid] = 0;
  if (tid == 0) rs[CAP] = make_float4(0.f, 0.f, 0.f, 0.f);    // ELL padding target
  const float rtol2 = (float)(a.rtol * a.rtol);
  const bool flags = ncl > 1 || a.withhold >= 0;
  int* abort_word = a.ready + a.k;
  int* never_set = a.ready + a.k + 1;
  int buf = 0, failed = 0;
  CgCount cnt;
  int prev = -1;
  Pattern<MAXR, ELLW, WEIGHTED> pat;
  cluster_sync();   // every CTA of the cluster runs before any remote access

  // Onorm of the panels (nr rows each) in `passes` CholeskyQR passes; then the
  // result goes back to the column layout (rs of every CTA) and, when
  // `write_u`, to U.
  auto onorm = [&](int r0, int rp, int nr, int passes, bool write_u) {
    for (int pass = 0; pass < passes; ++pass) {
      gram_partial(S, nr, ldp, cpad, d.Gp);
      cluster_sync();
      gram_allreduce(d, q, P, cpad);
      cluster_sync();
      for (int i = c + tid; i < cpad; i += kNT) d.A[i * kLDA + i] = 1.f;   // padded columns
      if (tid == 0) d.ctl[1] = 0;
      __syncthreads();
      chol_inverse(d, cpad);
      if (d.ctl[1]) failed = 1;
      apply_right(S, nr, ldp, cpad, d.M);
    }
    // back to the column layout: row lr of this panel -> rs[q rp + lr] of CTA grp
    const uint32_t rsa = smem_addr(rs);
    for (int e = tid; e < nr * P; e += kNT) {
      const int lr = e / P, grp = e - lr * P;
      const float4 v = *reinterpret_cast<const float4*>(S + lr * ldp + 4 * grp);
      st_remote4(remote(rsa + (uint32_t)(q * rp + lr) * 16u, grp), v);
    }
    if (write_u) {
      float* U = a.U + (size_t)(r0 + q * rp) * a.ld;
      if ((a.ld & 3) == 0 && (c & 3) == 0) {
        const int g4 = c >> 2;
        for (int e = tid; e < nr * g4; e += kNT) {
          const int lr = e / g4, grp = e - lr * g4;
          *reinterpret_cast<float4*>(U + (size_t)lr * a.ld + 4 * grp) =
              *reinterpret_cast<const float4*>(S + lr * ldp + 4 * grp);
        }
      } else {
        for (int e = tid; e < nr * c; e += kNT) {
          const int lr = e / c, j = e - lr * c;
          U[(size_t)lr * a.ld + j] = S[lr * ldp + j];
        }
      }
      if (flags) __threadfence();
    }
    cluster_sync();
  };

  for (int pos = cl; pos < a.nblocks; pos += ncl) {
    const int b = a.order[pos];
    const int r0 = mv.bptr[b], nbk = mv.bptr[b + 1] - r0;
    const int p = a.parent[b];
    const int np = p >= 0 ? mv.bptr[p + 1] - mv.bptr[p] : 0;
    const bool warm = p >= 0 && np == nbk;
    const int rp = (nbk + P - 1) / P;                       // panel rows per CTA
    const int nr = max(0, min(rp, nbk - q * rp));
    // bounded wait for a parent computed by another cluster (uniform decision)
    if (p >= 0 && (p != prev || b == a.withhold) && flags) {
      if (q == 0 && tid == 0) {
        const int* flag = b == a.withhold ? never_set : a.ready + p;
        const uint64_t deadline = global_ns() + (uint64_t)a.wait_limit_us * 1000ull;
        int go = 1;
        while (!ld_acquire(flag)) {
          if (ld_acquire(abort_word)) { go = 0; break; }
          if (global_ns() > deadline) {
            go = 0;
            atomicOr(a.status, ST_TIMEOUT);
            st_release(abort_word, 1);
            break;
          }
          __nanosleep(256);
        }
        for (int r = 0; r < P; ++r) st_remote_i(remote(smem_addr(d.ctl), r), go);
      }
      cluster_sync();
      if (!d.ctl[0]) break;
    }
    pat.load(mv, r0, nbk, (float)a.delta, d.red + 2 * kWarps * 8);
    const int sub = a.t_max * a.z;
    if (!warm) {
      // start rows into the panel: a root's supplied start, or the parent's
      // rows transferred by r -> floor(r n_p / n_b)
      for (int e = tid; e < nr * cpad; e += kNT) {
        const int lr = e / cpad, j = e - lr * cpad;
        const int i = q * rp + lr;
        float v = 0.f;
        if (j < c) {
          if (p < 0) v = a.starts[(size_t)(a.root_off[b] + i) * c + j];
          else v = __ldcg(a.U + (size_t)(mv.bptr[p] + (int)(((long long)i * np) / nbk)) * a.ld + j);
        }
        S[lr * ldp + j] = v;
      }
      __syncthreads();
      onorm(r0, rp, nr, 1, false);
    } else if (p != prev) {
      // same-size parent computed elsewhere: its rows, this CTA's 4 columns
      const float* Up = a.U + (size_t)mv.bptr[p] * a.ld;
      for (int i = tid; i < nbk; i += kNT) {
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = 4 * q + j < c ? __ldcg(Up + (size_t)i * a.ld + 4 * q + j) : 0.f;
        rs[i] = make_float4(v[0], v[1], v[2], v[3]);
      }
      __syncthreads();
    }
    // else: the parent was this cluster's previous block; its basis is in rs
    const int ncol = min(4, max(0, c - 4 * q));
    for (int t = 0; t < sub;) {
      const int g = (warm && t + 1 < sub) ? 2 : 1;
      float x[MAXR][4];
      cg_group<MAXR, ELLW, WEIGHTED>(pat, rs, d.red, buf, nbk, ncol, g, rtol2, a.max_steps, x, cnt);
      // solutions to the row panels: row i -> CTA i / rp, panel row i % rp, columns 4q..4q+3
      const uint32_t sa = smem_addr(S);
#pragma unroll
      for (int m = 0; m < MAXR; ++m) {
        const int i = tid + kNT * m;
        if (i < nbk) {
          const int o = i / rp, lr = i - o * rp;
          st_remote4(remote(sa + (uint32_t)(lr * ldp + 4 * q) * 4u, o),
                     make_float4(x[m][0], x[m][1], x[m][2], x[m][3]));
        }
      }
      cluster_sync();
      t += g;
      onorm(r0, rp, nr, 1, t == sub);
    }
    if (flags && q == 0 && tid == 0) st_release(a.ready + b, 1);
    prev = b;
  }
  cluster_sync();
  if (tid == 0) {
    atomicAdd(&a.stats->steps_total, (unsigned long long)cnt.total);
    atomicMax(&a.stats->steps_max, cnt.max);
    if (cnt.unconverged) {
      atomicAdd(&a.stats->not_converged, 1);
      atomicOr(a.status, ST_NOT_CONVERGED);
    }
    if (cnt.breakdown) atomicOr(a.status, ST_CG_BREAKDOWN);
    if (failed) atomicOr(a.status, ST_NUMERICAL);
  }
}

template <int MAXR>
size_t oi_cluster_smem(int P, int rpm) {
  const int ldp = 4 * P + 4;
  return (size_t)(MAXR * kNT + 1) * 16 + (size_t)rpm * ldp * 4 + 64 * 64 * 4 + 2 * 64 * kLDA * 4 +
         144 * 16 + 128 * 4 + 64 * 4 + (2 * kWarps * 8 + kWarps) * 4 + 8 * 4;
}

template <int MAXR, int ELLW, bool W>
int launch_t(const MeshView<float>& mv, const OiClusterArgs& a, int P, int ncl, bool query,
             cudaStream_t s, int* nclusters) {
  const size_t sm = oi_cluster_smem<MAXR>(P, a.rpm);
  if (sm > 220 * 1024) return BSP_ERR_INVALID_ARG;
  auto kern = k_oi_cluster<MAXR, ELLW, W>;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  // highest scheduling priority: work running beside the engine (the deferred
  // kernels of the previous range) yields SMs to the engine's next cluster
  static const int top_priority = [] {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return greatest;
  }();
  attr[1].id = cudaLaunchAttributePriority;
  attr[1].val.priority = top_priority;
  cfg.blockDim = dim3(kNT, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (query) {   // outside any stream capture: attributes and residency
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cfg.gridDim = dim3(P, 1, 1);
    int active = 0;
    if (cudaOccupancyMaxActiveClusters(&active, kern, &cfg) != cudaSuccess || active < 1) {
      cudaGetLastError();
      return BSP_ERR_INVALID_ARG;   // this cluster shape cannot be resident
    }
    *nclusters = std::max(1, std::min(ncl, active));
    return BSP_OK;
  }
  cfg.gridDim = dim3(P * ncl, 1, 1);
  cfg.numAttrs = 2;
  prof_begin(KC_OI, s);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, mv, a);
  prof_end(KC_OI, s);
  return e == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

template <int MAXR, int ELLW>
int launch_w(const MeshView<float>& mv, const OiClusterArgs& a, int P, int ncl, bool query,
             cudaStream_t s, int* nclusters) {
  return mv.wt ? launch_t<MAXR, ELLW, true>(mv, a, P, ncl, query, s, nclusters)
               : launch_t<MAXR, ELLW, false>(mv, a, P, ncl, query, s, nclusters);
}

int dispatch(const MeshView<float>& mv, OiClusterArgs a, int max_nb, int max_deg, int ncl,
             bool query, cudaStream_t s, int* nclusters) {
  const int P = (a.c + 3) / 4;
  a.rpm = (((max_nb + P - 1) / P) + 3) & ~3;
  const bool two = max_nb > kNT;
  const int w = max_deg <= 6 ? 6 : max_deg <= 8 ? 8 : 16;   // ELL width
  if (!two) return w == 6 ? launch_w<1, 6>(mv, a, P, ncl, query, s, nclusters)
                   : w == 8 ? launch_w<1, 8>(mv, a, P, ncl, query, s, nclusters)
                            : launch_w<1, 16>(mv, a, P, ncl, query, s, nclusters);
  return w == 6 ? launch_w<2, 6>(mv, a, P, ncl, query, s, nclusters)
       : w == 8 ? launch_w<2, 8>(mv, a, P, ncl, query, s, nclusters)
                : launch_w<2, 16>(mv, a, P, ncl, query, s, nclusters);
}

}  // namespace

bool g_disable_oi_cluster = false;

bool oi_cluster_fits(int c, int t_max, int max_nb, int max_deg, int min_nb) {
  if (g_disable_oi_cluster) return false;
  if (c < 1 || c > kCMax || t_max < 1 || max_nb > 2 * kNT || max_deg > 16) return false;
  const int P = (c + 3) / 4;
  // a CTA's panel must hold ceil(n_b / P) rows, apply_right at most 2 items per warp
  const int rp = (max_nb + P - 1) / P;
  if (((rp + 63) / 64) * P > 2 * kWarps) return false;
  return min_nb >= 1;
}

int prepare_oi_cluster(const MeshView<float>& mv, int c, int max_nb, int max_deg, int max_wave,
                       int* nclusters) {
  OiClusterArgs a{};
  a.c = c;
  return dispatch(mv, a, max_nb, max_deg, max_wave, true, nullptr, nclusters);
}

int launch_oi_cluster(const MeshView<float>& mv, const OiClusterArgs& a, int max_nb, int max_deg,
                      int nclusters, cudaStream_t s) {
  int unused = 0;
  return dispatch(mv, a, max_nb, max_deg, nclusters, false, s, &unused);
}

}  // namespace bsp
