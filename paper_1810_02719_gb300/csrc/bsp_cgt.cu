// Batched CG for S = (L + delta I)^-1 (Sec. 4, below Algorithm 1), one column
// per team of TW warps.
//
// A CTA of 8 warps takes 8 / TW consecutive columns of one block.  The block's
// pattern sits in shared memory once per CTA.  It is stored as ELL transposed
// (entry e of all rows contiguous), with padded entries aimed at a zero slot;
// the diagonal plus delta sits beside it.  Each team keeps the rows
// i = lane + 32 (w + TW m), m < R, of x, r, p, s = A p and w = A r in
// registers, and its current r in a shared vector for the neighbour reads.
// The iteration is Chronopoulos-Gear: per step one product and one fused
// reduction of (r, r) and (A r, r).  The reduction is done by warp shuffles,
// and for TW > 1 across the team's warps through shared memory and a named
// barrier.  Inside the iteration no barrier spans the CTA, so its columns run
// independently: a column that converges frees nothing but also waits for
// nothing, and a team of one warp synchronises with __syncwarp only.
//
// Two forms.  Unweighted meshes of degree <= 8 up to 2,048 rows keep each
// row's neighbour indices (packed two per register) and diagonal in registers
// too, 8 rows per lane: teams of 1, 2, 4, 8 warps up to 256, 512, 1,024,
// 2,048 rows.  The neighbour reads are then the only shared-memory loads of
// the product.  Otherwise the pattern stays in shared memory, 16 rows per
// lane (teams of 1, 2, 4, 8 warps up to 512, 1,024, 2,048, 4,096 rows).  The
// stopping rule and the initial guess (x0 = b (b, b) / (b, A b)) are those of
// the one-column-per-CTA kernel in bsp_cg.cu.
#include "bsp_internal.cuh"

namespace bsp {
namespace {

constexpr int kWarpsCta = 8;
constexpr int kThreadsCta = 32 * kWarpsCta;

BSP_DEV void team_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <typename T>
BSP_DEV T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Shared memory of one CTA: diagonal [CAP] T, weights [ELLW][CAP] T
// (weighted meshes), team vectors [NT][CAP + 1] T, neighbours [ELLW][CAP] u16;
// with the pattern in registers (REG) only the team vectors.
template <typename T, int TW, int R, int ELLW, bool REG>
constexpr size_t cgt_smem(bool weighted) {
  constexpr size_t CAP = 32 * TW * R, NT = kWarpsCta / TW;
  if (REG) return NT * (CAP + 1) * sizeof(T);
  return CAP * sizeof(T) + (weighted ? ELLW * CAP * sizeof(T) : 0) + NT * (CAP + 1) * sizeof(T) +
         ELLW * CAP * sizeof(uint16_t);
}

// Two CTAs per SM in FP32 (x, r, p, s, w of 16 rows in 128 registers); one
// in FP64, whose registers would otherwise spill.
template <typename T, int TW, int R, int ELLW, bool REG>
__global__ void __launch_bounds__(kThreadsCta, sizeof(T) == 4 ? 2 : 1)
    k_cgt(MeshView<T> mv, const T* __restrict__ V, T* __restrict__ Y, CgArgs a) {
  constexpr int CAP = 32 * TW * R;
  constexpr int NT = kWarpsCta / TW;
  static_assert(!REG || ELLW % 2 == 0, "indices are packed in pairs");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T tred[2][kWarpsCta][2];
  const int b = a.batch[blockIdx.y];
  if (a.live && !a.live[b]) return;
  const int c = a.cb[b];
  const int col0 = blockIdx.x * NT;
  if (col0 >= c) return;
  const int r0 = mv.bptr[b], nb = mv.bptr[b + 1] - r0;
  const bool weighted = mv.wt != nullptr;
  T* sdd = reinterpret_cast<T*>(smem_raw);
  T* swt = sdd + (REG ? 0 : CAP);
  T* svec = swt + (weighted && !REG ? ELLW * CAP : 0);
  uint16_t* snb = reinterpret_cast<uint16_t*>(svec + NT * (CAP + 1));
  const T delta = (T)a.delta;
  const int dmax = a.max_deg < ELLW ? a.max_deg : ELLW;   // uniform: entries past it skipped
  for (int i = threadIdx.x; i < CAP && !REG; i += kThreadsCta) {
    T d0 = 0;
    int dg = 0, e0 = 0;
    if (i < nb) {
      e0 = mv.rowptr[r0 + i];
      dg = mv.rowptr[r0 + i + 1] - e0;
      d0 = mv.diag[r0 + i] + delta;
    }
    sdd[i] = d0;
#pragma unroll
    for (int e = 0; e < ELLW; ++e) {
      const bool ok = e < dg;
      snb[e * CAP + i] = ok ? (uint16_t)mv.col[e0 + e] : (uint16_t)CAP;
      if (weighted) swt[e * CAP + i] = ok ? mv.wt[e0 + e] : T(0);
    }
  }
  if (threadIdx.x < NT) svec[threadIdx.x * (CAP + 1) + CAP] = T(0);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int team = warp / TW, wt = warp - team * TW;
  const int col = col0 + team;
  if (col >= c) return;   // the whole team leaves; no CTA-wide barrier follows
  T* vec = svec + team * (CAP + 1);
  const T rtol2 = (T)(a.rtol * a.rtol);

  auto row = [&](int m) { return lane + 32 * (wt + TW * m); };
  // REG: the team's rows' diagonal + delta and neighbour indices (two per word)
  constexpr int RP = REG ? R : 1, EP = REG ? ELLW / 2 : 1;
  T rdd[RP];
  uint32_t rnb[RP][EP];
  if constexpr (REG) {
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int i = row(m);
      int dg = 0, e0 = 0;
      rdd[m] = T(0);
      if (i < nb) {
        e0 = mv.rowptr[r0 + i];
        dg = mv.rowptr[r0 + i + 1] - e0;
        rdd[m] = mv.diag[r0 + i] + delta;
      }
#pragma unroll
      for (int e = 0; e < ELLW / 2; ++e) {
        const uint32_t lo = 2 * e < dg ? (uint32_t)mv.col[e0 + 2 * e] : (uint32_t)CAP;
        const uint32_t hi = 2 * e + 1 < dg ? (uint32_t)mv.col[e0 + 2 * e + 1] : (uint32_t)CAP;
        rnb[m][e] = lo | (hi << 16);
      }
    }
  }
  auto sync_vec = [&]() {
    if constexpr (TW == 1) __syncwarp();
    else team_barrier(1 + team, 32 * TW);
  };
  int buf = 0;
  auto team_sum2 = [&](T u, T v, T& su, T& sv) {
    u = warp_sum_t(u);
    v = warp_sum_t(v);
    if constexpr (TW == 1) {
      su = u;
      sv = v;
    } else {
      if (lane == 0) {
        tred[buf][warp][0] = u;
        tred[buf][warp][1] = v;
      }
      team_barrier(1 + team, 32 * TW);
      su = 0;
      sv = 0;
#pragma unroll
      for (int k = 0; k < TW; ++k) {
        su += tred[buf][team * TW + k][0];
        sv += tred[buf][team * TW + k][1];
      }
      buf ^= 1;
    }
  };
  // out_m = (D + delta) v_m - sum_e C v_nbr, v read from vec
  auto apply = [&](const T (&v)[R], T (&out)[R]) {
    if constexpr (REG) {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        T acc = rdd[m] * v[m];
#pragma unroll
        for (int e = 0; e < ELLW / 2; ++e) {
          const uint32_t w = rnb[m][e];
          acc -= vec[w & 0xffffu];
          acc -= vec[w >> 16];
        }
        out[m] = acc;
      }
      return;
    }
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int i = row(m);
      T acc = sdd[i] * v[m];
#pragma unroll
      for (int e = 0; e < ELLW; ++e) {
        if (e < dmax) {
          const T nv = vec[snb[e * CAP + i]];
          if (weighted) acc -= swt[e * CAP + i] * nv;
          else acc -= nv;
        }
      }
      out[m] = acc;
    }
  };
  auto put = [&](const T (&v)[R]) {
#pragma unroll
    for (int m = 0; m < R; ++m) vec[row(m)] = v[m];
  };

  T x[R], r[R], p[R], sv[R], wv[R];
  const int rv = a.vsrc ? mv.bptr[a.vsrc[b]] : r0;   // rows of the right-hand side
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int i = row(m);
    r[m] = i < nb ? V[(size_t)(rv + i) * a.ld + col] : T(0);
  }
  int steps_all = 0, steps_max = 0;
  bool unconverged = false, bad = false;
  for (int sol = 0; sol < a.z; ++sol) {
    // right-hand side in r: x0 = b (b, b) / (b, A b)
    put(r);
    sync_vec();
    apply(r, wv);
    T bb = 0, bab = 0;
#pragma unroll
    for (int m = 0; m < R; ++m) {
      bb += r[m] * r[m];
      bab += r[m] * wv[m];
    }
    T sbb, sbab;
    team_sum2(bb, bab, sbb, sbab);
    const T g = sbab > T(0) ? sbb / sbab : T(0);
    const T bn2 = sbb;
#pragma unroll
    for (int m = 0; m < R; ++m) {
      x[m] = g * r[m];
      r[m] -= g * wv[m];
    }
    put(r);
    sync_vec();
    apply(r, wv);
    T gl = 0, dl = 0;
#pragma unroll
    for (int m = 0; m < R; ++m) {
      gl += r[m] * r[m];
      dl += wv[m] * r[m];
    }
    T gam, dlt;
    team_sum2(gl, dl, gam, dlt);
    T alpha = dlt > T(0) ? gam / dlt : T(0);
#pragma unroll
    for (int m = 0; m < R; ++m) {
      p[m] = r[m];
      sv[m] = wv[m];
    }
    int steps = 0;
    while (gam > rtol2 * bn2) {
      if (steps >= a.max_steps) {
        unconverged = true;
        break;
      }
      if (!(dlt > T(0))) {
        bad = true;
        break;
      }
#pragma unroll
      for (int m = 0; m < R; ++m) {
        x[m] += alpha * p[m];
        r[m] -= alpha * sv[m];
      }
      put(r);
      sync_vec();
      apply(r, wv);
      gl = 0;
      dl = 0;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        gl += r[m] * r[m];
        dl += wv[m] * r[m];
      }
      T gnew, dnew;
      team_sum2(gl, dl, gnew, dnew);
      ++steps;
      if (!(gnew > rtol2 * bn2)) {
        gam = gnew;
        break;
      }
      const T beta = gnew / gam;
      const T den = dnew - beta * gnew / alpha;
      alpha = den > T(0) ? gnew / den : T(0);
      if (!(den > T(0))) bad = true;
      gam = gnew;
      dlt = den;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        p[m] = r[m] + beta * p[m];
        sv[m] = wv[m] + beta * sv[m];
      }
    }
    steps_all += steps;
    steps_max = max(steps_max, steps);
#pragma unroll
    for (int m = 0; m < R; ++m) r[m] = x[m];   // next right-hand side (z > 1)
  }
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int i = row(m);
    if (i < nb) Y[(size_t)(r0 + i) * a.ld + col] = x[m];
  }
  if (wt == 0 && lane == 0) {
    atomicAdd(&a.stats->steps_total, (unsigned long long)steps_all);
    atomicMax(&a.stats->steps_max, steps_max);
    if (unconverged) {
      atomicAdd(&a.stats->not_converged, 1);
      atomicOr(a.status, ST_NOT_CONVERGED);
    }
    if (bad) atomicOr(a.status, ST_CG_BREAKDOWN);
  }
}

template <typename T, int TW, int R, int ELLW, bool REG>
int launch_t(const MeshView<T>& mv, const T* V, T* Y, const CgArgs& a, int c_max,
             cudaStream_t s) {
  constexpr int NT = kWarpsCta / TW;
  const size_t smem = cgt_smem<T, TW, R, ELLW, REG>(mv.wt != nullptr);
  if (smem > 220 * 1024) return BSP_ERR_INVALID_ARG;
  dim3 grid((c_max + NT - 1) / NT, a.nbatch);
  k_cgt<T, TW, R, ELLW, REG><<<grid, kThreadsCta, smem, s>>>(mv, V, Y, a);
  return cudaGetLastError() == cudaSuccess ? BSP_OK : BSP_ERR_CUDA;
}

template <typename T, int ELLW>
int launch_rows(const MeshView<T>& mv, const T* V, T* Y, const CgArgs& a, int max_nb, int c_max,
                cudaStream_t s) {
  if (max_nb <= 512) return launch_t<T, 1, 16, ELLW, false>(mv, V, Y, a, c_max, s);
  if (max_nb <= 1024) return launch_t<T, 2, 16, ELLW, false>(mv, V, Y, a, c_max, s);
  if (max_nb <= 2048) return launch_t<T, 4, 16, ELLW, false>(mv, V, Y, a, c_max, s);
  if (max_nb <= 4096) return launch_t<T, 8, 16, ELLW, false>(mv, V, Y, a, c_max, s);
  return BSP_ERR_INVALID_ARG;
}

template <typename T, int ELLW>
int launch_rows_reg(const MeshView<T>& mv, const T* V, T* Y, const CgArgs& a, int max_nb,
                    int c_max, cudaStream_t s) {
  if (max_nb <= 256) return launch_t<T, 1, 8, ELLW, true>(mv, V, Y, a, c_max, s);
  if (max_nb <= 512) return launch_t<T, 2, 8, ELLW, true>(mv, V, Y, a, c_max, s);
  if (max_nb <= 1024) return launch_t<T, 4, 8, ELLW, true>(mv, V, Y, a, c_max, s);
  return launch_t<T, 8, 8, ELLW, true>(mv, V, Y, a, c_max, s);
}

template <typename T, int ELLW>
void configure_t() {
  set_max_dynamic_smem(k_cgt<T, 1, 16, ELLW, false>);
  set_max_dynamic_smem(k_cgt<T, 2, 16, ELLW, false>);
  set_max_dynamic_smem(k_cgt<T, 4, 16, ELLW, false>);
  set_max_dynamic_smem(k_cgt<T, 8, 16, ELLW, false>);
}

}  // namespace

void configure_cgt_kernels() {
  configure_t<float, 8>();
  configure_t<float, 16>();
  configure_t<double, 8>();
  configure_t<double, 16>();
}

// The register form applies (unweighted, degree <= 8, up to 2,048 rows).
bool cgt_reg(int max_nb, int max_deg, bool weighted) {
  return !weighted && max_deg > 0 && max_deg <= 8 && max_nb <= 2048;
}

// Whether the team kernel holds blocks of up to max_nb rows of degree <= max_deg.
bool cgt_fits(int max_nb, int max_deg, int real_bytes, bool weighted) {
  if (max_deg <= 0 || max_deg > 16 || max_nb > 4096) return false;
  if (cgt_reg(max_nb, max_deg, weighted)) return true;   // 8 KB per team vector at most
  const size_t tw = max_nb <= 512 ? 1 : max_nb <= 1024 ? 2 : max_nb <= 2048 ? 4 : 8;
  const size_t r = 16, cap = 32 * tw * r, nt = kWarpsCta / tw;
  const size_t ellw = max_deg <= 8 ? 8 : 16;
  const size_t bytes = cap * real_bytes + (weighted ? ellw * cap * real_bytes : 0) +
                       nt * (cap + 1) * real_bytes + ellw * cap * 2;
  return bytes <= 220 * 1024;
}

template <typename T>
int launch_cgt(const MeshView<T>& mv, const T* V, T* Y, const CgArgs& a, int max_nb, int c_max,
               cudaStream_t s) {
  if (!(a.max_deg > 0 && a.max_deg <= 16)) return BSP_ERR_INVALID_ARG;
  if (a.rows_per_lane != 16 && cgt_reg(max_nb, a.max_deg, mv.wt != nullptr))
    return a.max_deg <= 6 ? launch_rows_reg<T, 6>(mv, V, Y, a, max_nb, c_max, s)
                          : launch_rows_reg<T, 8>(mv, V, Y, a, max_nb, c_max, s);
  return a.max_deg <= 8 ? launch_rows<T, 8>(mv, V, Y, a, max_nb, c_max, s)
                        : launch_rows<T, 16>(mv, V, Y, a, max_nb, c_max, s);
}

template int launch_cgt<float>(const MeshView<float>&, const float*, float*, const CgArgs&, int,
                               int, cudaStream_t);
template int launch_cgt<double>(const MeshView<double>&, const double*, double*, const CgArgs&,
                                int, int, cudaStream_t);

}  // namespace bsp
