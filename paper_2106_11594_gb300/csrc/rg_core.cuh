// rg_core.cuh -- the phases of one rank-Greville block update, written once for two
// execution teams: the whole grid of a cooperative launch (one stream on the GPU,
// synchronised by bounded grid barriers) and a single CTA (one instance of a batch).
// A Team provides id() / size() (this worker and the number of workers; work items are
// strided over workers) and sync() (a barrier over the team that returns false if a
// bounded wait ran out).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "rg_internal.cuh"

namespace rg {

struct CallArgs {
  const double* Gamma;  // k x m
  const double* y;      // k
  long long k;
  uint8_t* indep;       // k or null
};

struct GridTeam {
  int* ctrl;
  __device__ __forceinline__ int id() const { return blockIdx.x; }
  __device__ __forceinline__ int size() const { return gridDim.x; }
  __device__ __forceinline__ bool sync() const { return grid_barrier(ctrl); }
};

struct CtaTeam {
  __device__ __forceinline__ int id() const { return 0; }
  __device__ __forceinline__ int size() const { return 1; }
  __device__ __forceinline__ bool sync() const {
    __syncthreads();
    return true;
  }
};


// ---------------------------------------------------------------------------------------
// Phase 1: gamma. Warp item = (group of JW block rows, one basis row i). The basis row is
// Ct_i (general) or Q_i (orthonormal); F32 projects with the FP32 copy of Q.
// ---------------------------------------------------------------------------------------
template <class Team, bool F32>
__device__ void phase_gamma(const Team& T, const StreamDev& S, const double* __restrict__ gam, int row_lo,
                            int row_hi, int r, const double* __restrict__ basis64) {
  const int nrows = row_hi - row_lo;
  if (nrows <= 0 || r <= 0) return;
  const int m = S.m, ld = S.ld;
  const int ngroups = (nrows + JW - 1) / JW;
  const long long nitems = (long long)ngroups * r;
  const int lane = threadIdx.x & 31;
  const long long wstride = (long long)T.size() * NWARP;
  for (long long it = (long long)T.id() * NWARP + (threadIdx.x >> 5); it < nitems;
       it += wstride) {
    const int grp = (int)(it / r);
    const int i = (int)(it - (long long)grp * r);
    const int jbase = row_lo + grp * JW;
    const int nj = min(JW, row_hi - jbase);
    if (F32) {
      float acc[JW];
#pragma unroll
      for (int a = 0; a < JW; ++a) acc[a] = 0.f;
      const float* q = S.Qf + (size_t)i * ld;
      for (int c = lane; c < m; c += 32) {
        const float qv = __ldcg(q + c);
#pragma unroll
        for (int a = 0; a < JW; ++a)
          if (a < nj) acc[a] = fmaf(qv, (float)__ldg(gam + (size_t)(jbase + a) * m + c), acc[a]);
      }
#pragma unroll
      for (int a = 0; a < JW; ++a) {
        const float v = warp_sumf(acc[a]);
        if (lane == 0 && a < nj) S.G[(size_t)(jbase + a) * S.r_max + i] = (double)v;
      }
    } else {
      double acc[JW];
#pragma unroll
      for (int a = 0; a < JW; ++a) acc[a] = 0.0;
      const double* q = basis64 + (size_t)i * ld;
      for (int c = lane; c < m; c += 32) {
        const double qv = __ldcg(q + c);
#pragma unroll
        for (int a = 0; a < JW; ++a)
          if (a < nj) acc[a] = fma(qv, __ldg(gam + (size_t)(jbase + a) * m + c), acc[a]);
      }
#pragma unroll
      for (int a = 0; a < JW; ++a) {
        const double v = warp_sum(acc[a]);
        if (lane == 0 && a < nj) S.G[(size_t)(jbase + a) * S.r_max + i] = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Phase 2: rejection. CTA item = (RJ block rows) x (MC columns); one thread per
// (row, column). Writes per-chunk partial sums of ||Gamma_r||^2 and ||Gamma||^2 and, when
// Rout != null, the FP64 rejection vectors (row j at Rout[(j - row_lo) * ld]).
// ---------------------------------------------------------------------------------------
template <class Team, bool F32>
__device__ void phase_reject(const Team& T, const StreamDev& S, const double* __restrict__ gam, int row_lo,
                             int row_hi, int r, const double* __restrict__ back64,
                             double* __restrict__ Rout) {
  const int nrows = row_hi - row_lo;
  if (nrows <= 0) return;
  const int m = S.m, ld = S.ld, nmc = S.nmc;
  const int ngroups = (nrows + RJ - 1) / RJ;
  const long long nitems = (long long)ngroups * nmc;
  __shared__ double red_s[NWARP], red_t[NWARP];
  const int jj = threadIdx.x / MC;
  const int cc = threadIdx.x % MC;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (long long it = T.id(); it < nitems; it += T.size()) {
    const int grp = (int)(it / nmc);
    const int mc = (int)(it - (long long)grp * nmc);
    const int j = row_lo + grp * RJ + jj;
    const int c = mc * MC + cc;
    double sv = 0.0, tv = 0.0;
    if (j < row_hi && c < m) {
      const double gv = __ldg(gam + (size_t)j * m + c);
      const double* gj = S.G + (size_t)j * S.r_max;
      if (F32) {
        float acc = (float)gv;
        for (int i = 0; i < r; ++i)
          acc = fmaf(-__ldcg(S.Qf + (size_t)i * ld + c), (float)__ldcg(gj + i), acc);
        sv = (double)acc * (double)acc;
      } else {
        double acc = gv;
        for (int i = 0; i < r; ++i) acc = fma(-__ldcg(back64 + (size_t)i * ld + c), __ldcg(gj + i), acc);
        sv = acc * acc;
        if (Rout) Rout[(size_t)(j - row_lo) * ld + c] = acc;
      }
      tv = gv * gv;
    }
    sv = warp_sum(sv);
    tv = warp_sum(tv);
    __syncthreads();
    if (lane == 0) {
      red_s[warp] = sv;
      red_t[warp] = tv;
    }
    __syncthreads();
    // MC = 64 columns per row = 2 warps per row
    if (threadIdx.x < RJ) {
      const int jr = row_lo + grp * RJ + threadIdx.x;
      if (jr < row_hi) {
        S.spart[(size_t)jr * nmc + mc] = red_s[2 * threadIdx.x] + red_s[2 * threadIdx.x + 1];
        S.tpart[(size_t)jr * nmc + mc] = red_t[2 * threadIdx.x] + red_t[2 * threadIdx.x + 1];
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Phase 3 (CTA 0): reduce the partial norms, decide every row, find the first row that
// needs the sequential section (independent, FP32 candidate, or non-finite).
// ---------------------------------------------------------------------------------------
template <bool MIXED>
__device__ void phase_decide(const StreamDev& S, const CallArgs& A, long long j0, int b, int r) {
  __shared__ int q0;
  if (threadIdx.x == 0) q0 = b;
  __syncthreads();
  const int nmc = S.nmc;
  double tc = S.tau_lo;
  if (MIXED && S.test_mode == 0 && S.tol > 0.0) tc = fmax(tc, 0.5 * S.tol);
  for (int j = threadIdx.x; j < b; j += NT) {
    double s = 0.0, t = 0.0;
    for (int c = 0; c < nmc; ++c) {
      s += __ldcg(S.spart + (size_t)j * nmc + c);
      t += __ldcg(S.tpart + (size_t)j * nmc + c);
    }
    S.s[j] = s;
    S.t[j] = t;
    const double yv = __ldg(A.y + j0 + j);
    bool special = !isfinite(t) || !isfinite(yv);
    if (!special) {
      if (MIXED) special = s > tc * tc * t;
      else special = is_independent(s, t, r, S.m, S.tol, S.test_mode);
    }
    if (special) atomicMin(&q0, j);
  }
  __syncthreads();
  if (threadIdx.x == 0) S.ctrl[CTRL_Q0] = q0;
}

// ---------------------------------------------------------------------------------------
// Blocked Sherman-Morrison (Woodbury) update of P^-1 and w for dependent block rows
// [a, a + len) whose gammas (length r) are in S.G. Every CTA calls it (grid phases).
// Returns false if a grid barrier timed out.
// ---------------------------------------------------------------------------------------
template <class Team>
__device__ bool woodbury(const Team& T, const StreamDev& S, const CallArgs& A, long long j0, int a, int len,
                         int r) {
  const int lane = threadIdx.x & 31;
  const long long gw = (long long)T.id() * NWARP + (threadIdx.x >> 5);
  const long long wstride = (long long)T.size() * NWARP;
  const long long gt = (long long)T.id() * NT + threadIdx.x;
  const long long tstride = (long long)T.size() * NT;
  const int rm = S.r_max;
  __shared__ double Ls[SB * SB];
  __shared__ double zs[SB];
  for (int s0 = a; s0 < a + len; s0 += SB) {
    const int q = min(SB, a + len - s0);
    if (r == 0) continue;  // zero rows with an empty basis: K = 0, nothing changes
    // W1: zeta_j = P^-1 gamma_j (Zt row j), D_j = y_j - gamma_j^T w
    {
      const long long nitems = (long long)r * q + q;
      for (long long it = gw; it < nitems; it += wstride) {
        double acc = 0.0;
        if (it < (long long)r * q) {
          const int jj = (int)(it / r), i = (int)(it - (long long)jj * r);
          const double* g = S.G + (size_t)(s0 + jj) * rm;
          const double* p = S.Pinv + (size_t)i * rm;
          for (int l = lane; l < r; l += 32) acc = fma(__ldcg(p + l), __ldcg(g + l), acc);
          acc = warp_sum(acc);
          if (lane == 0) S.Zt[(size_t)jj * rm + i] = acc;
        } else {
          const int jj = (int)(it - (long long)r * q);
          const double* g = S.G + (size_t)(s0 + jj) * rm;
          for (int l = lane; l < r; l += 32) acc = fma(__ldcg(g + l), __ldcg(S.w + l), acc);
          acc = warp_sum(acc);
          if (lane == 0) S.D[jj] = __ldg(A.y + j0 + s0 + jj) - acc;
        }
      }
    }
    if (!T.sync()) return false;
    // W2: M = I + G^T Z (lower triangle)
    {
      const long long nitems = (long long)q * q;
      for (long long it = gw; it < nitems; it += wstride) {
        const int p = (int)(it / q), p2 = (int)(it - (long long)p * q);
        if (p2 > p) continue;
        const double* g = S.G + (size_t)(s0 + p) * rm;
        const double* z = S.Zt + (size_t)p2 * rm;
        double acc = 0.0;
        for (int l = lane; l < r; l += 32) acc = fma(__ldcg(g + l), __ldcg(z + l), acc);
        acc = warp_sum(acc);
        if (lane == 0) S.M[p * SB + p2] = acc + (p == p2 ? 1.0 : 0.0);
      }
    }
    if (!T.sync()) return false;
    // W3a (CTA 0): Cholesky M = L L^T and a = M^-1 D
    if (T.id() == 0) {
      for (int e = threadIdx.x; e < q * q; e += NT) {
        const int p = e / q, p2 = e - p * q;
        Ls[p * SB + p2] = (p2 <= p) ? __ldcg(S.M + p * SB + p2) : 0.0;
      }
      if (threadIdx.x < q) zs[threadIdx.x] = __ldcg(S.D + threadIdx.x);
      __syncthreads();
      for (int kk = 0; kk < q; ++kk) {
        if (threadIdx.x == 0) {
          const double d = Ls[kk * SB + kk];
          if (!(d > 0.0) || !isfinite(d)) atomicOr(S.ctrl + CTRL_STATUS, ST_NONFINITE);
          Ls[kk * SB + kk] = sqrt(fmax(d, 1e-300));
        }
        __syncthreads();
        const double lkk = Ls[kk * SB + kk];
        for (int p = kk + 1 + threadIdx.x; p < q; p += NT) Ls[p * SB + kk] /= lkk;
        __syncthreads();
        const int rem = q - kk - 1;
        for (int e = threadIdx.x; e < rem * rem; e += NT) {
          const int p = kk + 1 + e / rem, p2 = kk + 1 + e % rem;
          if (p2 <= p) Ls[p * SB + p2] -= Ls[p * SB + kk] * Ls[p2 * SB + kk];
        }
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        for (int p = 0; p < q; ++p) {  // forward: L z = D
          double v = zs[p];
          for (int p2 = 0; p2 < p; ++p2) v -= Ls[p * SB + p2] * zs[p2];
          zs[p] = v / Ls[p * SB + p];
        }
        for (int p = q - 1; p >= 0; --p) {  // backward: L^T a = z
          double v = zs[p];
          for (int p2 = p + 1; p2 < q; ++p2) v -= Ls[p2 * SB + p] * zs[p2];
          zs[p] = v / Ls[p * SB + p];
        }
      }
      __syncthreads();
      for (int e = threadIdx.x; e < q * q; e += NT) {
        const int p = e / q, p2 = e - p * q;
        S.M[p * SB + p2] = Ls[p * SB + p2];
      }
      if (threadIdx.x < q) S.aw[threadIdx.x] = zs[threadIdx.x];
    }
    if (!T.sync()) return false;
    // W3b: Wt = L^-1 Z^T column by column; w += Z a
    for (long long i = gt; i < r; i += tstride) {
      double wi = __ldcg(S.w + i);
      for (int p = 0; p < q; ++p) {
        const double zpi = __ldcg(S.Zt + (size_t)p * rm + i);
        wi = fma(zpi, __ldcg(S.aw + p), wi);
        double v = zpi;
        for (int p2 = 0; p2 < p; ++p2) v -= __ldcg(S.M + p * SB + p2) * __ldcg(S.Wt + (size_t)p2 * rm + i);
        S.Wt[(size_t)p * rm + i] = v / __ldcg(S.M + p * SB + p);
      }
      S.w[i] = wi;
    }
    if (!T.sync()) return false;
    // W4: P^-1 <- P^-1 - Wt^T Wt
    {
      const long long nitems = (long long)r * r;
      for (long long it = gt; it < nitems; it += tstride) {
        const int i = (int)(it / r), l = (int)(it - (long long)i * r);
        double acc = 0.0;
        for (int p = 0; p < q; ++p)
          acc = fma(__ldcg(S.Wt + (size_t)p * rm + i), __ldcg(S.Wt + (size_t)p * rm + l), acc);
        S.Pinv[(size_t)i * rm + l] = __ldcg(S.Pinv + (size_t)i * rm + l) - acc;
      }
    }
    if (!T.sync()) return false;
  }
  return true;
}

// Block-wide sum (all threads get the result).
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[NWARP];
  __shared__ double tot;
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < NWARP; ++i) a += red[i];
    tot = a;
  }
  __syncthreads();
  return tot;
}

// ---------------------------------------------------------------------------------------
// Sequential section scan (CTA 0): rows [q0, bend) with FP64 G and R (R row j at
// S.R[(j - q0) * ld]). Decides each row in order, fixes up the later rows of the section
// after each append, records segments and the data of every append.
// ---------------------------------------------------------------------------------------
template <bool ORTHO>
__device__ void phase_scan(const StreamDev& S, const CallArgs& A, long long j0, int q0, int bend,
                           int r) {
  const int m = S.m, ld = S.ld, rm = S.r_max;
  // dec: 0 dependent, 1 independent, -1 stop (error)
  __shared__ int nseg, nind, applied, r_cur, dec;
  __shared__ double sh_s;
  if (threadIdx.x == 0) {
    nseg = 0;
    nind = 0;
    applied = bend;
    r_cur = r;
  }
  __syncthreads();
  const long long base_row = __ldcg(S.rows_seen);
  for (int j = q0; j < bend; ++j) {
    const double* Rj = S.R + (size_t)(j - q0) * ld;
    double part = 0.0;
    for (int c = threadIdx.x; c < m; c += NT) {
      const double v = __ldcg(Rj + c);
      part = fma(v, v, part);
    }
    const double s = block_sum(part);  // ||Gamma_r||^2 after the in-block fix-ups
    const double t = __ldcg(S.t + j);
    const double yv = __ldg(A.y + j0 + j);
    const int rc = r_cur;
    if (threadIdx.x == 0) {
      int d = 0;
      if (!isfinite(t) || !isfinite(yv) || !isfinite(s)) {
        atomicOr(S.ctrl + CTRL_STATUS, ST_NONFINITE);
        d = -1;
      } else if (is_independent(s, t, rc, m, S.tol, S.test_mode)) {
        d = 1;
        if (rc >= rm) {
          atomicOr(S.ctrl + CTRL_STATUS, ST_CAPACITY);
          d = -1;
        }
      }
      if (d < 0) {
        applied = j;
      } else {
        S.rowflag[j] = (uint8_t)(d + 1);
        bool extended = false;
        if (d == 0 && nseg > 0) {
          int* sg = S.seg + 3 * (nseg - 1);
          if (sg[0] == SEG_DEP && sg[1] + sg[2] == j) {
            sg[2] += 1;
            extended = true;
          }
        }
        if (!extended) {
          int* nw = S.seg + 3 * nseg;
          nw[0] = d ? SEG_IND : SEG_DEP;
          nw[1] = j;
          nw[2] = 1;
          nseg += 1;
        }
      }
      dec = d;
      sh_s = s;
    }
    __syncthreads();
    if (dec < 0) break;
    if (dec == 1) {  // independent row: record the append, fix up the later rows
      const int q = nind;
      const double scale = ORTHO ? 1.0 / sqrt(sh_s) : 1.0 / sh_s;
      double* Kq = S.Kv + (size_t)q * ld;
      for (int c = threadIdx.x; c < m; c += NT) Kq[c] = __ldcg(Rj + c) * scale;
      const double* gj = S.G + (size_t)j * rm;
      for (int i = threadIdx.x; i < rc; i += NT) S.Gind[(size_t)q * rm + i] = __ldcg(gj + i);
      if (threadIdx.x == 0) {
        S.jind[q] = j;
        S.alpha[q] = 1.0 / sqrt(sh_s);
        S.basis_rows[rc] = base_row + j;
        if (!ORTHO) {  // general variant: P^-1 <- diag(P^-1, 1), w <- [w; y]
          for (int i = 0; i < rc; ++i) {
            S.Pinv[(size_t)rc * rm + i] = 0.0;
            S.Pinv[(size_t)i * rm + rc] = 0.0;
          }
          S.Pinv[(size_t)rc * rm + rc] = 1.0;
          S.w[rc] = yv;
        }
      }
      __syncthreads();
      const double sj = sh_s, sq = sqrt(sh_s);
      for (int jt = j + 1; jt < bend; ++jt) {
        double* Rt = S.R + (size_t)(jt - q0) * ld;
        double part2 = 0.0;
        for (int c = threadIdx.x; c < m; c += NT) part2 = fma(__ldcg(Rj + c), __ldcg(Rt + c), part2);
        const double kap = block_sum(part2) / sj;  // K_j^T Gamma_r,t
        for (int c = threadIdx.x; c < m; c += NT) Rt[c] = fma(-kap, __ldcg(Rj + c), __ldcg(Rt + c));
        double* gt = S.G + (size_t)jt * rm;
        if (!ORTHO)
          for (int i = threadIdx.x; i < rc; i += NT) gt[i] = fma(-kap, __ldcg(gj + i), __ldcg(gt + i));
        if (threadIdx.x == 0) gt[rc] = ORTHO ? kap * sq : kap;
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        nind = q + 1;
        r_cur = rc + 1;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    S.ctrl[CTRL_NSEG] = nseg;
    S.ctrl[CTRL_NIND] = nind;
    S.ctrl[CTRL_APPLIED] = applied;
    S.ctrl[CTRL_RNEW] = r_cur;
  }
}

// Orthonormal variant, independent row (Section 2.2): with zeta = P^-1 gamma,
// P^-1 <- [[P^-1, -alpha zeta], [-alpha zeta^T, alpha^2 (1 + gamma^T zeta)]] and
// w <- [w; alpha (y - gamma^T w)]. CTA 0 only.
__device__ __forceinline__ void ortho_border(const StreamDev& S, const double* gam, double alpha, double yv, int r) {
  const int rm = S.r_max;
  double gz_part = 0.0, gw_part = 0.0;
  for (int i = threadIdx.x; i < r; i += NT) {
    double z = 0.0;
    for (int l = 0; l < r; ++l) z = fma(__ldcg(S.Pinv + (size_t)i * rm + l), __ldcg(gam + l), z);
    S.Zt[i] = z;  // scratch row 0
    gz_part = fma(__ldcg(gam + i), z, gz_part);
    gw_part = fma(__ldcg(gam + i), __ldcg(S.w + i), gw_part);
  }
  const double gz = block_sum(gz_part);
  const double gw = block_sum(gw_part);
  __syncthreads();
  for (int i = threadIdx.x; i < r; i += NT) {
    const double v = -alpha * S.Zt[i];
    S.Pinv[(size_t)i * rm + r] = v;
    S.Pinv[(size_t)r * rm + i] = v;
  }
  if (threadIdx.x == 0) {
    S.Pinv[(size_t)r * rm + r] = alpha * alpha * (1.0 + gz);
    S.w[r] = alpha * (yv - gw);
  }
  __syncthreads();
}

// Appends of the sequential section, applied by the whole grid.
// General variant: Ct_final[i] = base_i - sum_{q >= qmin(i)} Gind[q][i] K_q with
// base_i = Ct[i] (i < r) or K_{i-r}, qmin(i) = max(0, i - r + 1); C[r + q] = Gamma_{jind[q]}.
// Orthonormal variant: Q[r + q] = alpha_q Gamma_r (already scaled in Kv) and its FP32 copy.
template <class Team, bool ORTHO>
__device__ void phase_append(const Team& T, const StreamDev& S, const CallArgs& A, long long j0, int r, int nind) {
  const int m = S.m, ld = S.ld, rm = S.r_max;
  const long long gt = (long long)T.id() * NT + threadIdx.x;
  const long long tstride = (long long)T.size() * NT;
  if (ORTHO) {
    const long long n = (long long)nind * m;
    for (long long e = gt; e < n; e += tstride) {
      const int q = (int)(e / m), c = (int)(e - (long long)q * m);
      const double v = __ldcg(S.Kv + (size_t)q * ld + c);
      S.C[(size_t)(r + q) * ld + c] = v;
      S.Qf[(size_t)(r + q) * ld + c] = (float)v;
    }
    return;
  }
  const int rnew = r + nind;
  const long long n = (long long)rnew * m;
  for (long long e = gt; e < n; e += tstride) {
    const int i = (int)(e / m), c = (int)(e - (long long)i * m);
    double v = (i < r) ? __ldcg(S.Ct + (size_t)i * ld + c) : __ldcg(S.Kv + (size_t)(i - r) * ld + c);
    const int qmin = max(0, i - r + 1);
    for (int q = qmin; q < nind; ++q)
      v = fma(-__ldcg(S.Gind + (size_t)q * rm + i), __ldcg(S.Kv + (size_t)q * ld + c), v);
    S.Ct[(size_t)i * ld + c] = v;
  }
  const long long n2 = (long long)nind * m;
  for (long long e = gt; e < n2; e += tstride) {
    const int q = (int)(e / m), c = (int)(e - (long long)q * m);
    const int j = __ldcg(S.jind + q);
    S.C[(size_t)(r + q) * ld + c] = __ldg(A.Gamma + (size_t)(j0 + j) * m + c);
  }
}


// ---------------------------------------------------------------------------------------
// Apply the k rows of one call to one stream, team-wide. Returns false if a bounded team
// barrier gave up (the status word then holds ST_TIMEOUT). Every worker of the team runs
// the same control flow; decisions made by worker 0 are read back after a barrier.
// ---------------------------------------------------------------------------------------
template <class Team, bool MIXED>
__device__ bool process_rows(const Team& T, const StreamDev& S, const CallArgs& A) {
  __shared__ int sh[8];
  long long j0 = 0;
  while (j0 < A.k) {
    if (threadIdx.x == 0) {
      sh[0] = ld_acquire_i32(S.ctrl + CTRL_STATUS);
      sh[1] = ld_acquire_i32(S.ctrl + CTRL_R);
      sh[2] = ld_acquire_i32(S.ctrl + CTRL_KB);
    }
    __syncthreads();
    if (sh[0] != 0) break;
    const int r = sh[1];
    const int kb0 = sh[2];
    const int b = (int)min((long long)kb0, A.k - j0);
    const double* gam = A.Gamma + (size_t)j0 * S.m;
    __syncthreads();
    // 1-2: project every row of the block against the block-start basis
    phase_gamma<Team, MIXED>(T, S, gam, 0, b, r, MIXED ? S.C : S.Ct);
    if (!T.sync()) return false;
    phase_reject<Team, MIXED>(T, S, gam, 0, b, r, S.C, nullptr);
    if (!T.sync()) return false;
    // 3: decide
    if (T.id() == 0) phase_decide<MIXED>(S, A, j0, b, r);
    if (!T.sync()) return false;
    if (threadIdx.x == 0) sh[3] = ld_acquire_i32(S.ctrl + CTRL_Q0);
    __syncthreads();
    const int q0 = sh[3];
    // 4: leading dependent run
    if (q0 > 0 && !woodbury(T, S, A, j0, 0, q0, r)) return false;
    int applied = b, rnew = r;
    if (q0 < b) {
      // 5: sequential section, in FP64
      const int bend = min(b, q0 + SLOW_MAX);
      phase_gamma<Team, false>(T, S, gam, q0, bend, r, MIXED ? S.C : S.Ct);
      if (!T.sync()) return false;
      phase_reject<Team, false>(T, S, gam, q0, bend, r, S.C, S.R);
      if (!T.sync()) return false;
      if (T.id() == 0) phase_scan<MIXED>(S, A, j0, q0, bend, r);
      if (!T.sync()) return false;
      if (threadIdx.x == 0) {
        sh[4] = ld_acquire_i32(S.ctrl + CTRL_NSEG);
        sh[5] = ld_acquire_i32(S.ctrl + CTRL_APPLIED);
        sh[6] = ld_acquire_i32(S.ctrl + CTRL_RNEW);
        sh[7] = ld_acquire_i32(S.ctrl + CTRL_NIND);
      }
      __syncthreads();
      const int nseg = sh[4];
      applied = sh[5];
      rnew = sh[6];
      const int nind = sh[7];
      int rs = r, qi = 0;
      for (int sgi = 0; sgi < nseg; ++sgi) {
        const int kind = __ldcg(S.seg + 3 * sgi), first = __ldcg(S.seg + 3 * sgi + 1),
                  cnt = __ldcg(S.seg + 3 * sgi + 2);
        if (kind == SEG_DEP) {
          if (!woodbury(T, S, A, j0, first, cnt, rs)) return false;
        } else {
          if (MIXED) {
            if (T.id() == 0)
              ortho_border(S, S.Gind + (size_t)qi * S.r_max, __ldcg(S.alpha + qi),
                           __ldg(A.y + j0 + first), rs);
            if (!T.sync()) return false;
          }
          rs += 1;
          qi += 1;
        }
      }
      if (nind > 0) {
        phase_append<Team, MIXED>(T, S, A, j0, r, nind);
        if (!T.sync()) return false;
      }
    }
    // finalize the block (worker 0): flags, counters, rank, next block size
    if (T.id() == 0) {
      if (A.indep)
        for (int j = threadIdx.x; j < applied; j += NT)
          A.indep[j0 + j] = (j < q0) ? 0 : (uint8_t)(__ldcg(S.rowflag + j) - 1);
      if (threadIdx.x == 0) {
        *S.rows_seen = __ldcg(S.rows_seen) + applied;
        S.ctrl[CTRL_R] = rnew;
        S.ctrl[CTRL_KB] = (q0 < b) ? min(KB_MIN, S.kb_max) : min(2 * kb0, S.kb_max);
      }
    }
    if (!T.sync()) return false;
    j0 += applied;
  }
  return true;
}

}  // namespace rg
