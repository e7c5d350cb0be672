// rg_core.cuh -- the phases of one rank-Greville block update, written once for two
// execution teams: the whole grid of a cooperative launch (one stream on the GPU,
// synchronised by bounded grid barriers) and a single CTA (one instance of a batch).
// A Team provides id() / size() (this worker and the number of workers; work items are
// strided over workers) and sync() (a barrier over the team that returns false if a
// bounded wait ran out).
//
// State (Section 2.1): the basis C (or Q), its dual Ct, and the small matrices in
// information form: P = B^T B (so P^-1 of Algorithm 1 is its inverse) and the solution
// coordinates w = w_b + P^-1 u with X = Ct^T w (from A^+ = Ct^T P^-1 B^T). A dependent row
// (Theorem 6, dependent case; Theorem 5) adds gamma gamma^T to P and gamma (y - gamma^T w_b)
// to u: P^-1 <- P^-1 - zeta zeta^T / (1 + gamma^T zeta) is exactly the inverse of
// P <- P + gamma gamma^T (Sherman-Morrison, Eq. label_eq_sherman_morrison), and
// w_new = w_b + P_new^-1 (u + gamma (y - gamma^T w_b)) holds for any base w_b. An
// independent row extends the state (Theorem 6, independent case): general variant
// P <- diag(P, 1), w_b <- [w_b; y], u <- [u; 0]; orthonormal variant (Section 2.2)
// P <- diag(P, 0) + g g^T with g = [gamma; 1/alpha], w_b <- [w_b; 0], u <- [u; 0] +
// g (y - gamma^T w_b). P^-1 and w are formed (Cholesky of P) only when X or an export is
// requested, so no sequential small solve sits on the row path.
//
// Data written by one worker and read by another within a launch is always read with
// __ldcg (L2), never through the non-coherent L1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <type_traits>

#include "rg_internal.cuh"
#include "rg_tc.cuh"

namespace rg {

struct CallArgs {
  const double* Gamma;  // k x m
  const double* y;      // k
  long long k;
  uint8_t* indep;       // k or null
};

struct GridTeam {
  int* ctrl;
  int bar_off = CTRL_BAR_COUNT;  // control word of the barrier's arrival counter
  __device__ __forceinline__ int id() const { return blockIdx.x; }
  __device__ __forceinline__ int size() const { return gridDim.x; }
  __device__ __forceinline__ bool sync() const { return grid_barrier(ctrl, bar_off); }
};

struct CtaTeam {
  __device__ __forceinline__ int id() const { return 0; }
  __device__ __forceinline__ int size() const { return 1; }
  __device__ __forceinline__ bool sync() const {
    __syncthreads();
    return true;
  }
};

// Work-item numbering that deals consecutive items to different workers first, so that a
// phase with few items still spreads over every SM (FP64 throughput is per SM).
template <class Team>
__device__ __forceinline__ long long rr_warp(const Team& T) {
  return (long long)(threadIdx.x >> 5) * T.size() + T.id();
}
template <class Team>
__device__ __forceinline__ long long rr_thread(const Team& T) {
  return (long long)threadIdx.x * T.size() + T.id();
}

// 1/sqrt(d) for d > 0: single-precision seed refined by two Newton-Raphson steps
// y <- y (3 - d y^2) / 2 (quadratic convergence: ~2^-22 -> ~2^-44 -> rounding level).
// Falls back to 1/sqrt outside the single-precision range.
__device__ __forceinline__ double rsqrt_nr(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double y = (double)rsqrtf((float)d);
  const double h = 0.5 * d;
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return y;
}

// 1/d for d > 0: single-precision seed refined by two Newton-Raphson steps
// y <- y (2 - d y) (quadratic convergence, as for rsqrt_nr); 1/d outside that range.
__device__ __forceinline__ double rcp_nr(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / d;
  double y = (double)(1.0f / (float)d);
  y = y * fma(-d, y, 2.0);
  y = y * fma(-d, y, 2.0);
  return y;
}

// CTA-wide sum; every thread gets the result.
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

// One shared-memory pool per CTA for the larger working arrays of the phases below; the
// phases that use it are separated by barriers, so they never overlap.
constexpr int POOL_DOUBLES = 4352;  // 34 KiB: a 64 x 64 tile plus 4 rows of 64
static_assert(32 * 33 + GRAM_RMAX <= POOL_DOUBLES, "solve staging must fit the pool");
static_assert(3 * 32 * 33 <= POOL_DOUBLES, "Cholesky tiles must fit the pool");
static_assert(64 * MC + RJ * 64 <= POOL_DOUBLES, "rejection tiles must fit the pool");
__device__ __forceinline__ double* smem_pool() {
  __shared__ __align__(16) double pool[POOL_DOUBLES];
  return pool;
}

// Butterfly all-reduce of 32 values across the 32 lanes of a warp: on entry every lane
// holds v[0..31]; on exit lane l holds in v[0] the sum over lanes of v[l]. Each of the
// five stages exchanges half of the remaining values (16 + 8 + 4 + 2 + 1 shuffles), and
// the adds within a stage are independent, so the FP64 add latency overlaps.
__device__ __forceinline__ void warp_transpose_sum32(double (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int k = 0; k < off; ++k) {
      const double send = upper ? v[k] : v[k + off];
      const double keep = upper ? v[k + off] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
}

// Generalisation to N = 2^k <= 32 values per lane (type V): the first k stages split the
// values by lane bits 4, 3, ..., the remaining 5 - k stages are plain butterflies. On
// exit lane l holds in v[0] the total for value index (l >> (5 - k)) mod N, bit-reversed
// order not needed: index = sum of lane bits 4..(5-k) weighted N/2, N/4, ..., 1.
template <typename V, int N>
__device__ __forceinline__ V warp_transpose_sum(V (&v)[N]) {
  const int lane = threadIdx.x & 31;
  int cur = N;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    if (cur > 1) {
      const bool upper = (lane & off) != 0;
      const int half = cur >> 1;
#pragma unroll
      for (int k = 0; k < N / 2; ++k) {
        if (k < half) {
          const V send = upper ? v[k] : v[k + half];
          const V keep = upper ? v[k + half] : v[k];
          v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
      }
      cur = half;
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
    }
  }
  return v[0];
}
// Value index held by this lane after warp_transpose_sum<V, N>.
template <int N>
__device__ __forceinline__ int transpose_sum_index() {
  const int lane = threadIdx.x & 31;
  int idx = 0, w = N >> 1;
#pragma unroll
  for (int off = 16; off >= 1 && w >= 1; off >>= 1, w >>= 1)
    if (lane & off) idx += w;
  return idx;
}

// =======================================================================================
// Projection of a block of rows against the block-start basis
// =======================================================================================

// gamma_j = Ct Gamma_j (general) or Q Gamma_j (orthonormal) for rows [row_lo, row_hi).
// Warp item = (NJ rows) x (NI basis rows), dealt round robin over the workers; the lanes
// stride over the m columns and the NJ x NI partial sums are combined by one butterfly
// transpose-reduction. FP64: NJ = 8, NI = 1 (FP64 adds are scarce on this part, so the
// reduction is kept to ~3% of the FMAs). F32 (FP32 copy of Q): NJ = 4, NI = 8, FP32
// accumulation, each FP64 input element converted once per item.
template <class Team, bool F32>
__device__ void phase_gamma(const Team& T, const StreamDev& S, const double* __restrict__ gam,
                            int row_lo, int row_hi, int r, const double* __restrict__ basis64) {
  constexpr int NJ = F32 ? 4 : 8, NI = F32 ? 8 : 1, N = NJ * NI;
  using V = typename std::conditional<F32, float, double>::type;
  const int nrows = row_hi - row_lo;
  if (nrows <= 0 || r <= 0) return;
  const int m = S.m, ld = S.ld, rm = S.r_max;
  const int nj = (nrows + NJ - 1) / NJ, ni = (r + NI - 1) / NI;
  const long long nitems = (long long)nj * ni;
  const long long wstride = (long long)T.size() * NWARP;
  const int lane = threadIdx.x & 31;
  for (long long it = rr_warp(T); it < nitems; it += wstride) {
    const int gj = (int)(it / ni), gi = (int)(it - (long long)gj * ni);
    const int j0 = row_lo + gj * NJ, i0 = gi * NI;
    V acc[N];
#pragma unroll
    for (int q = 0; q < N; ++q) acc[q] = V(0);
#pragma unroll 8
    for (int c = lane; c < m; c += 32) {
      V gv[NJ], bv[NI];
#pragma unroll
      for (int a = 0; a < NJ; ++a) gv[a] = (j0 + a < row_hi) ? (V)__ldg(gam + (size_t)(j0 + a) * m + c) : V(0);
#pragma unroll
      for (int bb = 0; bb < NI; ++bb) {
        if (F32) bv[bb] = (i0 + bb < r) ? (V)__ldcg(S.Qf + (size_t)(i0 + bb) * ld + c) : V(0);
        else bv[bb] = (i0 + bb < r) ? (V)__ldcg(basis64 + (size_t)(i0 + bb) * ld + c) : V(0);
      }
#pragma unroll
      for (int a = 0; a < NJ; ++a)
#pragma unroll
        for (int bb = 0; bb < NI; ++bb) acc[a * NI + bb] = fma(bv[bb], gv[a], acc[a * NI + bb]);
    }
    const V tot = warp_transpose_sum<V, N>(acc);
    const int q = transpose_sum_index<N>();
    // the lanes holding index q are those with equal high bits; the lowest one writes
    const int low_bits = 32 / N;  // lanes sharing an index: low (5 - log2 N) bits free
    if ((lane & (low_bits - 1)) == 0) {
      const int a = q / NI, bb = q - a * NI;
      if (j0 + a < row_hi && i0 + bb < r) S.G[(size_t)(j0 + a) * rm + i0 + bb] = (double)tot;
    }
  }
}

// Small FP64 blocks: the same products with CTA items of 4 rows x 2 basis rows whose
// columns are split over the 8 warps (warp w takes columns 32 w + lane + 256 k), so that
// every SM sub-partition has FP64 work even when there are fewer items than warps (one
// warp per item would leave three of an SM's four FP64 units idle). The 8 partial sums of
// each lane are combined by a butterfly transpose-reduction, then across the warps in
// shared memory.
template <class Team>
__device__ void phase_gamma_cta(const Team& T, const StreamDev& S, const double* __restrict__ gam,
                                int row_lo, int row_hi, int r, const double* __restrict__ basis64) {
  constexpr int NJ = 4, NI = 2, N = NJ * NI;
  const int nrows = row_hi - row_lo;
  if (nrows <= 0 || r <= 0) return;
  const int m = S.m, ld = S.ld, rm = S.r_max;
  const int nj = (nrows + NJ - 1) / NJ, ni = (r + NI - 1) / NI;
  const long long nitems = (long long)nj * ni;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ double red[NWARP][N];
  for (long long it = T.id(); it < nitems; it += T.size()) {
    const int gj = (int)(it / ni), gi = (int)(it - (long long)gj * ni);
    const int j0 = row_lo + gj * NJ, i0 = gi * NI;
    double acc[N];
#pragma unroll
    for (int q = 0; q < N; ++q) acc[q] = 0.0;
#pragma unroll 4
    for (int c = warp * 32 + lane; c < m; c += NT) {
      double gv[NJ], bv[NI];
#pragma unroll
      for (int a = 0; a < NJ; ++a) gv[a] = (j0 + a < row_hi) ? __ldg(gam + (size_t)(j0 + a) * m + c) : 0.0;
#pragma unroll
      for (int bb = 0; bb < NI; ++bb) bv[bb] = (i0 + bb < r) ? __ldcg(basis64 + (size_t)(i0 + bb) * ld + c) : 0.0;
#pragma unroll
      for (int a = 0; a < NJ; ++a)
#pragma unroll
        for (int bb = 0; bb < NI; ++bb) acc[a * NI + bb] = fma(bv[bb], gv[a], acc[a * NI + bb]);
    }
    const double tot = warp_transpose_sum<double, N>(acc);
    const int q = transpose_sum_index<N>();
    if ((lane & (32 / N - 1)) == 0) red[warp][q] = tot;
    __syncthreads();
    if (threadIdx.x < N) {
      double v = 0.0;
#pragma unroll
      for (int w2 = 0; w2 < NWARP; ++w2) v += red[w2][threadIdx.x];
      const int a = threadIdx.x / NI, bb = threadIdx.x - a * NI;
      if (j0 + a < row_hi && i0 + bb < r) S.G[(size_t)(j0 + a) * rm + i0 + bb] = v;
    }
    __syncthreads();
  }
}

// Small blocks on grid teams: CTA tile = JT rows x BT basis rows (BT in {1, 2, 4, 8}, from
// small_gamma_bt). Warp w takes basis row w % BT of the tile over the column range w / BT of
// NWARP / BT equal ranges, so the four SM sub-partitions (warp w on w % 4), each with its
// own FP64 unit, get equal shares of every tile. The lanes stride over the range with the
// JT row sums in registers (each basis element loaded serves JT rows); one butterfly
// transpose-reduction combines them across the lanes and the ranges are added in shared
// memory in a fixed order. A warp does 4 m BT / 256 FMAs per lane before its 6 adds, where
// phase_gamma_cta does 32 before 9.
template <class Team, bool F32, int JT>
__device__ void phase_gamma_small(const Team& T, const StreamDev& S, const double* __restrict__ gam,
                                  int row_lo, int row_hi, int r, const double* __restrict__ basis64, int BT) {
  using V = typename std::conditional<F32, float, double>::type;
  const int nrows = row_hi - row_lo;
  if (nrows <= 0 || r <= 0) return;
  const int m = S.m, ld = S.ld, rm = S.r_max;
  const int ntb = (r + BT - 1) / BT, ntj = (nrows + JT - 1) / JT;
  const long long ntiles = (long long)ntj * ntb;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nseg = NWARP / BT, seg = warp / BT, bb = warp - seg * BT;
  const int len = ((m + nseg - 1) / nseg + 31) & ~31;  // columns per range (multiple of 32)
  const int c_lo = seg * len, c_hi = min(m, c_lo + len);
  __shared__ double red[NWARP][JT];
  for (long long it = T.id(); it < ntiles; it += T.size()) {
    const int tj = (int)(it / ntb), tb = (int)(it - (long long)tj * ntb);
    const int j0 = row_lo + tj * JT, i = tb * BT + bb;
    const bool iok = i < r;
    const double* gp = gam + (size_t)j0 * m;
    V acc[JT];
#pragma unroll
    for (int a = 0; a < JT; ++a) acc[a] = V(0);
#pragma unroll 8
    for (int c = c_lo + lane; c < c_hi; c += 32) {
      V gv[JT];
#pragma unroll
      for (int a = 0; a < JT; ++a) gv[a] = (j0 + a < row_hi) ? (V)__ldg(gp + (size_t)a * m + c) : V(0);
      V bv;
      if (F32) bv = iok ? (V)__ldcg(S.Qf + (size_t)i * ld + c) : V(0);
      else bv = iok ? (V)__ldcg(basis64 + (size_t)i * ld + c) : V(0);
#pragma unroll
      for (int a = 0; a < JT; ++a) acc[a] = fma(bv, gv[a], acc[a]);
    }
    const V tot = warp_transpose_sum<V, JT>(acc);
    const int q = transpose_sum_index<JT>();
    if ((lane & (32 / JT - 1)) == 0) red[warp][q] = (double)tot;
    __syncthreads();
    if (threadIdx.x < JT * BT) {
      const int a = threadIdx.x / BT, b2 = threadIdx.x - a * BT;
      double v = 0.0;
      for (int s2 = 0; s2 < nseg; ++s2) v += red[s2 * BT + b2][a];
      const int ii = tb * BT + b2;
      if (j0 + a < row_hi && ii < r) S.G[(size_t)(j0 + a) * rm + ii] = v;
    }
    __syncthreads();
  }
}

// Basis rows per tile of phase_gamma_small for ntj row groups, rank r and nw workers. FP64:
// the fewest FMAs per sub-partition (rounds x BT), ties to the larger BT (fewer adds and
// rounds); FP32, where the FMAs are cheap: the fewest rounds, ties to the smaller BT (less
// data per CTA).
__device__ __forceinline__ int small_gamma_bt(int ntj, int r, int nw, bool f32) {
  int best = 1;
  long long bc = -1;
  for (int bt = 1; bt <= NWARP; bt <<= 1) {
    const long long tiles = (long long)ntj * ((r + bt - 1) / bt);
    const long long rounds = (tiles + nw - 1) / nw;
    const long long cost = f32 ? rounds * 16 + bt : rounds * bt * 16 - bt;
    if (bc < 0 || cost < bc) {
      bc = cost;
      best = bt;
    }
  }
  return best;
}

template <class Team, bool F32>
__device__ __forceinline__ void phase_gamma_small_any(const Team& T, const StreamDev& S, const double* gam,
                                                      int row_lo, int row_hi, int r, const double* basis64) {
  const int nrows = row_hi - row_lo;
  const int jt = nrows >= 4 ? 4 : (nrows >= 2 ? 2 : 1);
  const int bt = small_gamma_bt((nrows + jt - 1) / jt, r, T.size(), F32);
  if (jt == 4) phase_gamma_small<Team, F32, 4>(T, S, gam, row_lo, row_hi, r, basis64, bt);
  else if (jt == 2) phase_gamma_small<Team, F32, 2>(T, S, gam, row_lo, row_hi, r, basis64, bt);
  else phase_gamma_small<Team, F32, 1>(T, S, gam, row_lo, row_hi, r, basis64, bt);
}

// FP32 screen of mixed mode: true if the row is certainly dependent (relative rejection
// at most tc). Rows whose squared norm leaves the range where FP32 squares and sums are
// exact enough (including zero rows) are not screened: the FP64 section decides them.
__device__ __forceinline__ bool fp32_screen_dependent(double s, double t, double tc) {
  return t > 1e-30 && t < 1e30 && s <= tc * tc * t;
}

// TMA prefetch of the basis tile of a CTA's first rejection item (grid teams, small blocks):
// rows [0, rc) x columns [mc MC, mc MC + MC) of C (FP64) or of the FP32 copy of Q (mixed
// mode), one bulk copy per basis row into the shared-memory pool, issued before the
// projection so that the copies overlap it and the barrier after it. A copy stops at the
// row stride ld (a multiple of 4 elements, so every copy is a multiple of 16 bytes and
// starts on a 16-byte boundary of the 256-byte aligned state); the columns >= m it brings
// are never used. phase_reject then waits for the tile (bounded) instead of staging it.
struct RejPrefetch {
  unsigned long long* bar;  // mbarrier: one arrival with the expected bytes per prefetch
  uint32_t* ph;             // parity of its next completion (per thread)
};

// One bulk copy (TMA) of `bytes` from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Every thread waits for the completion of parity ph of the mbarrier (bounded); the CTA
// agrees on the outcome. On success the parity advances; false if the wait gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t& ph) {
  bool done = mbar_try_wait(bar, ph);
  if (!done) {
    const unsigned long long t0 = global_ns();
    while (!(done = mbar_try_wait(bar, ph)))
      if (global_ns() - t0 > WAIT_LIMIT_NS) break;
  }
  if (!__syncthreads_and(done ? 1 : 0)) return false;
  ph ^= 1u;
  return true;
}

template <bool F32>
__device__ __forceinline__ void rej_prefetch(const StreamDev& S, int mc, int rc, unsigned long long* bar) {
  fence_async_smem();  // earlier generic accesses of the pool before the asynchronous writes
  __syncthreads();
  if (threadIdx.x < 32) {
    constexpr int ES = F32 ? 4 : 8;
    const uint32_t bytes = (uint32_t)(min(MC, S.ld - mc * MC) * ES);
    if (threadIdx.x == 0)
      asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                       smem_u32(bar)),
                   "r"(bytes * (uint32_t)rc)
                   : "memory");
    __syncwarp();
    const char* src = F32 ? reinterpret_cast<const char*>(S.Qf) : reinterpret_cast<const char*>(S.C);
    src += (size_t)mc * MC * ES;
    char* dst = reinterpret_cast<char*>(smem_pool());
    for (int ii = threadIdx.x; ii < rc; ii += 32)
      bulk_g2s(dst + (size_t)ii * MC * ES, src + (size_t)ii * S.ld * ES, bytes, bar);
  }
}

// The rank decisions of a small block fused into its rejection phase (grid teams): the CTA
// whose item completes a row group's partial norms (one counter per group, control words
// CTRL_GRP..) sums the group's partials in a fixed order, decides its rows as decide_rows
// does, stores s and t, lowers CTRL_Q0 to the first row that needs the sequential section,
// and clears the counter for the next block. After the phase's barrier every CTA reads
// CTRL_Q0 instead of reducing and deciding every row itself.
struct FusedDecide {
  const double* y;  // the block's targets
  double tc;        // mixed mode: floor of the FP32 screen
};

// The fused decision (FusedDecide) of row group grp, rows [jb, min(jb + rb, row_hi)), called by
// every thread of an item once its partial norms are written (by threads [0, rb)).
template <bool F32>
__device__ __forceinline__ void fused_decide(const StreamDev& S, const FusedDecide* fd, int grp, int jb, int rb,
                                             int row_hi, int r) {
  const int nmc = S.nmc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ int last_s;
  if (threadIdx.x < rb) __threadfence();  // the partials before the counter
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last_s = atomicAdd(S.ctrl + CTRL_GRP + grp, 1) == nmc - 1;
  }
  __syncthreads();
  if (last_s) {
    __threadfence();
    // one warp per row: lanes load the partials (all in flight together), a butterfly sums
    // them in a fixed order
    for (int a = warp; a < rb; a += NWARP) {
      const int jr = jb + a;
      if (jr >= row_hi) continue;
      double sv = 0.0, tv = 0.0;
      for (int c = lane; c < nmc; c += 32) {
        sv += __ldcg(S.spart + (size_t)jr * nmc + c);
        tv += __ldcg(S.tpart + (size_t)jr * nmc + c);
      }
      sv = warp_sum(sv);
      tv = warp_sum(tv);
      if (lane == 0) {
        S.s[jr] = sv;
        S.t[jr] = tv;
        const double yv = __ldg(fd->y + jr);
        bool special = !isfinite(tv) || !isfinite(yv);
        if (!special) {
          if (F32) special = !fp32_screen_dependent(sv, tv, fd->tc);
          else special = is_independent(sv, tv, r, S.m, S.tol, S.test_mode);
        }
        if (special) atomicMin(S.ctrl + CTRL_Q0, jr);
      }
    }
    if (threadIdx.x == 0) S.ctrl[CTRL_GRP + grp] = 0;
  }
}

// Gamma_r = Gamma_j - B^T gamma_j with B = C (general) or Q (orthonormal). CTA item =
// (4 RPT rows) x (MC columns): thread (row lane rl, column cc) handles rows rl, rl + 4,
// ..., so each staged basis tile serves 4 RPT rows. The basis tile (RC ranks x MC
// columns) and the gamma slice are staged in shared memory per chunk of RC ranks. RPT = 1
// spreads small blocks over many CTAs; RPT = 8 is used for large blocks. Writes per-chunk
// partial sums of ||Gamma_r||^2 and ||Gamma||^2 and, when Rout != null, the FP64
// rejections (row j at Rout[(j - row_lo) * ld]). The partial sums are FP64 in FP64 mode;
// in the FP32 screen of mixed mode they are FP32 sums over the MC columns of a chunk (the
// screen only compares s against tau_lo^2 t, and FP64 arithmetic is 1/64 of FP32 here).
template <class Team, bool F32, int RPT>
__device__ void phase_reject(const Team& T, const StreamDev& S, const double* __restrict__ gam,
                             int row_lo, int row_hi, int r, const double* __restrict__ back64,
                             double* __restrict__ Rout, const FusedDecide* fd = nullptr,
                             const RejPrefetch* pf = nullptr) {
  using V = typename std::conditional<F32, float, double>::type;
  constexpr int RB = 4 * RPT;                          // rows per item
  constexpr int RC = (F32 || RPT == 1) ? 64 : 32;      // ranks per staged chunk
  static_assert(RC * MC * sizeof(V) / 8 + RB * RC * sizeof(V) / 8 <= POOL_DOUBLES, "pool");
  const int nrows = row_hi - row_lo;
  if (nrows <= 0) return;
  const int m = S.m, ld = S.ld, nmc = S.nmc, rm = S.r_max;
  const int ngroups = (nrows + RB - 1) / RB;
  const long long nitems = (long long)ngroups * nmc;
  __shared__ double red_s[NWARP][RPT], red_t[NWARP][RPT];
  V* Bt = reinterpret_cast<V*>(smem_pool());  // RC x MC basis tile
  V* Gs = Bt + RC * MC;                        // RB x RC gamma slice
  const int cc = threadIdx.x % MC;
  const int rl = threadIdx.x / MC;             // 0..3
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (long long it = T.id(); it < nitems; it += T.size()) {
    const int grp = (int)(it / nmc);
    const int mc = (int)(it - (long long)grp * nmc);
    const int jb = row_lo + grp * RB;
    const int c = mc * MC + cc;
    double gv[RPT];
    V acc[RPT][2];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int j = jb + rl + 4 * q;
      gv[q] = (j < row_hi && c < m) ? __ldg(gam + (size_t)j * m + c) : 0.0;
      acc[q][0] = (V)gv[q];
      acc[q][1] = V(0);
    }
    for (int i0 = 0; i0 < r; i0 += RC) {
      const int rc = min(RC, r - i0);
      const bool prefetched = pf && i0 == 0 && it == T.id();  // see RejPrefetch
      __syncthreads();
      if (!prefetched) {
#pragma unroll 8
        for (int e = threadIdx.x; e < rc * MC; e += NT) {
          const int ii = e / MC, c2 = mc * MC + (e - ii * MC);
          if (F32) Bt[e] = (c2 < m) ? (V)__ldcg(S.Qf + (size_t)(i0 + ii) * ld + c2) : V(0);
          else Bt[e] = (c2 < m) ? (V)__ldcg(back64 + (size_t)(i0 + ii) * ld + c2) : V(0);
        }
      }
#pragma unroll 4
      for (int e = threadIdx.x; e < RB * rc; e += NT) {
        const int a = e / rc, ii = e - a * rc;
        const int ja = jb + a;
        Gs[a * RC + ii] = (ja < row_hi) ? (V)__ldcg(S.G + (size_t)ja * rm + i0 + ii) : V(0);
      }
      if (prefetched && !mbar_wait(pf->bar, *pf->ph)) {
        // the tile never arrived: flag the failure, wait once more (bounded) for the copies
        // in flight, and go on with whatever the pool holds (the status word stops the call)
        if (threadIdx.x == 0) atomicOr(S.ctrl + CTRL_STATUS, ST_TIMEOUT);
        uint32_t p2 = *pf->ph;
        if (mbar_wait(pf->bar, p2)) *pf->ph = p2;
      }
      __syncthreads();
      int ii = 0;
      for (; ii + 1 < rc; ii += 2) {
        const V b0 = Bt[ii * MC + cc], b1 = Bt[(ii + 1) * MC + cc];
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          const V* g = Gs + (rl + 4 * q) * RC;
          acc[q][0] = fma(-b0, g[ii], acc[q][0]);
          acc[q][1] = fma(-b1, g[ii + 1], acc[q][1]);
        }
      }
      if (ii < rc) {
        const V b0 = Bt[ii * MC + cc];
#pragma unroll
        for (int q = 0; q < RPT; ++q) acc[q][0] = fma(-b0, Gs[(rl + 4 * q) * RC + ii], acc[q][0]);
      }
    }
    V sv[RPT], tv[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int j = jb + rl + 4 * q;
      const bool valid = (j < row_hi && c < m);
      const V a = acc[q][0] + acc[q][1];
      const V g = (V)gv[q];
      sv[q] = valid ? a * a : V(0);
      tv[q] = valid ? g * g : V(0);
      if (!F32 && Rout && valid) Rout[(size_t)(j - row_lo) * ld + c] = (double)a;
    }
    // per warp: the 32 columns of its row lane; lanes reduce the RPT rows at once
    V ts, tt;
    int qi = 0;
    if (RPT == 1) {
      ts = sv[0];
      tt = tv[0];
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        ts += __shfl_xor_sync(0xffffffffu, ts, off);
        tt += __shfl_xor_sync(0xffffffffu, tt, off);
      }
    } else {
      ts = warp_transpose_sum<V, RPT>(sv);
      tt = warp_transpose_sum<V, RPT>(tv);
      qi = transpose_sum_index<RPT>();
    }
    __syncthreads();
    if ((lane & (32 / RPT - 1)) == 0) {
      red_s[warp][qi] = (double)ts;
      red_t[warp][qi] = (double)tt;
    }
    __syncthreads();
    if (threadIdx.x < RB) {  // row a = rl + 4 q: warps 2 rl and 2 rl + 1 hold its columns
      const int a = threadIdx.x, rla = a & 3, q = a >> 2;
      const int jr = jb + a;
      if (jr < row_hi) {
        S.spart[(size_t)jr * nmc + mc] = red_s[2 * rla][q] + red_s[2 * rla + 1][q];
        S.tpart[(size_t)jr * nmc + mc] = red_t[2 * rla][q] + red_t[2 * rla + 1][q];
      }
    }
    if (fd) fused_decide<F32>(S, fd, grp, jb, RB, row_hi, r);
  }
}

// Blocks of at most 16 rows on grid teams: CTA item = 1 row x MC columns (the 4-row items
// of phase_reject would carry empty rows). Thread (warp w, lane) takes column 8 w +
// (lane mod 8) of the item and every fourth rank from lane / 8 on, so it does a quarter of
// the FMAs of a 4-row item's thread; two shuffles combine the quarters. The partial norms
// per (row, column chunk), the basis-tile prefetch and the fused decision are those of
// phase_reject.
template <class Team, bool F32>
__device__ void phase_reject_row(const Team& T, const StreamDev& S, const double* __restrict__ gam,
                                 int row_lo, int row_hi, int r, const double* __restrict__ back64,
                                 const FusedDecide* fd, const RejPrefetch* pf) {
  using V = typename std::conditional<F32, float, double>::type;
  constexpr int RC = 64;  // ranks per staged chunk, as phase_reject with 4-row items
  static_assert(RC * MC * sizeof(V) / 8 + RC * sizeof(V) / 8 <= POOL_DOUBLES, "pool");
  const int nrows = row_hi - row_lo;
  if (nrows <= 0) return;
  const int m = S.m, ld = S.ld, nmc = S.nmc, rm = S.r_max;
  const long long nitems = (long long)nrows * nmc;
  __shared__ double red_s[NWARP], red_t[NWARP];
  V* Bt = reinterpret_cast<V*>(smem_pool());  // RC x MC basis tile
  V* Gs = Bt + RC * MC;                        // RC gammas of the row
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cc = warp * 8 + (lane & 7), qr = lane >> 3;
  for (long long it = T.id(); it < nitems; it += T.size()) {
    const int grp = (int)(it / nmc);
    const int mc = (int)(it - (long long)grp * nmc);
    const int j = row_lo + grp;
    const int c = mc * MC + cc;
    const double gv = (c < m) ? __ldg(gam + (size_t)j * m + c) : 0.0;
    V acc = (qr == 0) ? (V)gv : V(0);
    for (int i0 = 0; i0 < r; i0 += RC) {
      const int rc = min(RC, r - i0);
      const bool prefetched = pf && i0 == 0 && it == T.id();  // see RejPrefetch
      __syncthreads();
      if (!prefetched) {
#pragma unroll 8
        for (int e = threadIdx.x; e < rc * MC; e += NT) {
          const int ii = e / MC, c2 = mc * MC + (e - ii * MC);
          if (F32) Bt[e] = (c2 < m) ? (V)__ldcg(S.Qf + (size_t)(i0 + ii) * ld + c2) : V(0);
          else Bt[e] = (c2 < m) ? (V)__ldcg(back64 + (size_t)(i0 + ii) * ld + c2) : V(0);
        }
      }
      for (int e = threadIdx.x; e < rc; e += NT) Gs[e] = (V)__ldcg(S.G + (size_t)j * rm + i0 + e);
      if (prefetched && !mbar_wait(pf->bar, *pf->ph)) {
        if (threadIdx.x == 0) atomicOr(S.ctrl + CTRL_STATUS, ST_TIMEOUT);
        uint32_t p2 = *pf->ph;
        if (mbar_wait(pf->bar, p2)) *pf->ph = p2;
      }
      __syncthreads();
      // ranks qr, qr + 4, ...: the four lane groups read four different banks of Gs
      V a0 = V(0), a1 = V(0);
      int ii = qr;
      for (; ii + 4 < rc; ii += 8) {
        a0 = fma(-Bt[ii * MC + cc], Gs[ii], a0);
        a1 = fma(-Bt[(ii + 4) * MC + cc], Gs[ii + 4], a1);
      }
      if (ii < rc) a0 = fma(-Bt[ii * MC + cc], Gs[ii], a0);
      acc += a0 + a1;
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 8);
    acc += __shfl_xor_sync(0xffffffffu, acc, 16);
    const bool own = qr == 0 && c < m;  // lanes 0-7 hold the warp's 8 columns
    V two[2] = {own ? acc * acc : V(0), own ? (V)gv * (V)gv : V(0)};
    const V tot = warp_transpose_sum<V, 2>(two);
    const int qi = transpose_sum_index<2>();
    if ((lane & 15) == 0) {
      if (qi == 0) red_s[warp] = (double)tot;
      else red_t[warp] = (double)tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sv = 0.0, tv = 0.0;
#pragma unroll
      for (int w = 0; w < NWARP; ++w) {
        sv += red_s[w];
        tv += red_t[w];
      }
      S.spart[(size_t)j * nmc + mc] = sv;
      S.tpart[(size_t)j * nmc + mc] = tv;
    }
    if (fd) fused_decide<F32>(S, fd, grp, j, 1, row_hi, r);
    else __syncthreads();  // red_s / red_t are free for the next item
  }
}

// Mixed mode, large blocks: gamma with the block's rows staged once in shared memory,
// converted to FP32 (CTA item = GR rows x all basis rows; warp w takes basis rows
// w, w + NWARP, ...; lanes stride over the columns; FP32 accumulation).
template <class Team>
__device__ void phase_gamma_f32_staged(const Team& T, const StreamDev& S, const double* __restrict__ gam,
                                       int row_lo, int row_hi, int r, int GR) {
  const int m = S.m, ld = S.ld, rm = S.r_max;
  float* Gf = reinterpret_cast<float*>(smem_pool());  // GR x m
  const int ngroups = (row_hi - row_lo + GR - 1) / GR;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int it = T.id(); it < ngroups; it += T.size()) {
    const int j0 = row_lo + it * GR;
    const int nj = min(GR, row_hi - j0);
    __syncthreads();
#pragma unroll 8
    for (int e = threadIdx.x; e < GR * m; e += NT) {
      const int a = e / m, c = e - a * m;
      Gf[e] = (a < nj) ? (float)__ldg(gam + (size_t)(j0 + a) * m + c) : 0.f;
    }
    __syncthreads();
    for (int i = warp; i < r; i += NWARP) {
      const float* q = S.Qf + (size_t)i * ld;
      float acc[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) acc[a] = 0.f;
#pragma unroll 4
      for (int c = lane; c < m; c += 32) {
        const float qv = __ldcg(q + c);
#pragma unroll
        for (int a = 0; a < 8; ++a)
          if (a < GR) acc[a] = fmaf(qv, Gf[a * m + c], acc[a]);
      }
      const float tot = warp_transpose_sum<float, 8>(acc);
      const int a = transpose_sum_index<8>();
      if ((lane & 3) == 0 && a < nj) S.G[(size_t)(j0 + a) * rm + i] = (double)tot;
    }
  }
}

// A-priori errors D_j = y_j - gamma_j^T w_b of rows [0, b) (Theorems 4/5 with the
// solution in base coordinates). Warp items, one row each. In the variants of Section 2.2
// every append extends w_b with 0, so w_b = 0 and D_j = y_j (no FP64 products).
template <class Team>
__device__ void phase_dall(const Team& T, const StreamDev& S, const CallArgs& A, long long j0, int b,
                           int r, int w_first = 0) {
  if (S.ortho || S.orthog) {
    const long long tstride = (long long)T.size() * NT;
    const int wid = (T.id() - w_first + T.size()) % T.size();
    for (long long j = (long long)wid * NT + threadIdx.x; j < b; j += tstride) S.Dall[j] = __ldg(A.y + j0 + j);
    return;
  }
  // rows are dealt to the workers starting at w_first (the ones another phase leaves idle)
  const int lane = threadIdx.x & 31;
  const long long wstride = (long long)T.size() * NWARP;
  const int wid = (T.id() - w_first + T.size()) % T.size();
  for (long long j = (long long)wid * NWARP + (threadIdx.x >> 5); j < b; j += wstride) {
    const double* g = S.G + (size_t)j * S.r_max;
    const double yv = __ldg(A.y + j0 + j);
    double acc = 0.0;
    for (int l = lane; l < r; l += 32) acc = fma(__ldcg(g + l), __ldcg(S.wb + l), acc);
    acc = warp_sum(acc);
    if (lane == 0) S.Dall[j] = yv - acc;
  }
}


// Reduce the partial norms of rows [0, b), decide every row and return the first row that
// needs the sequential section (independent, FP32 candidate, or non-finite). Every CTA that
// calls it gets the same answer (same data, same summation order); with `publish` the CTA
// also stores s, t and the answer for the later phases.
template <bool MIXED>
__device__ int decide_rows(const StreamDev& S, const CallArgs& A, long long j0, int b, int r,
                           bool publish) {
  __shared__ int q0;
  if (threadIdx.x == 0) q0 = b;
  __syncthreads();
  const int nmc = S.nmc;
  double tc = S.tau_lo;
  if (MIXED && S.test_mode == 0 && S.tol > 0.0) tc = fmax(tc, 0.5 * S.tol);
  // a warp takes rows warp, warp + NWARP, warp + 2 NWARP, warp + 3 NWARP of each group of
  // 4 NWARP rows; all loads are issued first, then one butterfly transpose-reduction sums
  // the 8 values (s and t of 4 rows) across the lanes (chunks) and lane group p decides
  // row p / 2
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int jb = 0; jb < b; jb += 4 * NWARP) {
    double v[8], y4[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = jb + q * NWARP + warp;
      v[2 * q] = 0.0;
      v[2 * q + 1] = 0.0;
      y4[q] = (j < b) ? __ldg(A.y + j0 + j) : 0.0;
      if (j < b)
        for (int c = lane; c < nmc; c += 32) {
          v[2 * q] += __ldcg(S.spart + (size_t)j * nmc + c);
          v[2 * q + 1] += __ldcg(S.tpart + (size_t)j * nmc + c);
        }
    }
    const double tot8 = warp_transpose_sum<double, 8>(v);
    const int idx = transpose_sum_index<8>();  // value index held by this lane
    // pair (s, t) of row q sits in value indices 2q, 2q + 1: fetch t from the partner lane
    const double other = __shfl_xor_sync(0xffffffffu, tot8, 32 / 8 * 1);
    if ((idx & 1) == 0 && (lane & (32 / 8 - 1)) == 0) {
      const int q = idx >> 1;
      const int j = jb + q * NWARP + warp;
      if (j < b) {
        const double s = tot8, t = other;
        if (publish) {
          S.s[j] = s;
          S.t[j] = t;
        }
        const double yv = (q == 0) ? y4[0] : (q == 1) ? y4[1] : (q == 2) ? y4[2] : y4[3];
        bool special = !isfinite(t) || !isfinite(yv);
        if (!special) {
          if (MIXED) special = !fp32_screen_dependent(s, t, tc);
          else special = is_independent(s, t, r, S.m, S.tol, S.test_mode);
        }
        if (special) atomicMin(&q0, j);
      }
    }
  }
  __syncthreads();
  const int res = q0;
  if (publish && threadIdx.x == 0) S.ctrl[CTRL_Q0] = res;
  __syncthreads();
  return res;
}

// Team-parallel form for large blocks: every warp decides rows (dealt round robin) and
// lowers CTRL_Q0 with atomicMin; CTRL_Q0 must hold b beforehand (set in an earlier phase).
// Stores s and t of every row.
template <class Team, bool MIXED>
__device__ void decide_rows_team(const Team& T, const StreamDev& S, const CallArgs& A, long long j0,
                                 int b, int r) {
  const int nmc = S.nmc;
  double tc = S.tau_lo;
  if (MIXED && S.test_mode == 0 && S.tol > 0.0) tc = fmax(tc, 0.5 * S.tol);
  const int lane = threadIdx.x & 31;
  const long long wstride = (long long)T.size() * NWARP;
  for (long long j = rr_warp(T); j < b; j += wstride) {
    double s = 0.0, t = 0.0;
    for (int c = lane; c < nmc; c += 32) {
      s += __ldcg(S.spart + (size_t)j * nmc + c);
      t += __ldcg(S.tpart + (size_t)j * nmc + c);
    }
    s = warp_sum(s);
    t = warp_sum(t);
    if (lane == 0) {
      S.s[j] = s;
      S.t[j] = t;
      const double yv = __ldg(A.y + j0 + j);
      bool special = !isfinite(t) || !isfinite(yv);
      if (!special) {
        if (MIXED) special = !fp32_screen_dependent(s, t, tc);
        else special = is_independent(s, t, r, S.m, S.tol, S.test_mode);
      }
      if (special) atomicMin(S.ctrl + CTRL_Q0, (int)j);
    }
  }
}

// =======================================================================================
// Dependent rows: P += gamma gamma^T, u += gamma D for rows of a run whose D are in S.Dall.
// =======================================================================================

// Short runs: one thread per entry of P (and of u), dealt round robin over the workers,
// up to EMAX entries per thread per pass; the gamma rows of the run (and their D) are
// staged in shared memory in row chunks. Ranks whose gamma rows do not fit the pool read
// G from L2 directly. F32 (mixed mode): the gammas are FP32 values held in FP64 (exact
// conversions) and every entry is a compensated FP32 sum (FABsum).
template <class Team, bool F32>
__device__ void acc_rows(const Team& T, const StreamDev& S, const double* Gsrc, const double* Dsrc, int a,
                         int len, int r, int w_lo) {
  using V = typename std::conditional<F32, float, double>::type;
  const int rm = S.r_max;
  if (T.id() < w_lo) return;  // workers [w_lo, size) take part
  const int nw = T.size() - w_lo;
  const long long tstride = (long long)nw * NT;
  const long long nP = (long long)r * r, ntot = nP + r;
  constexpr int EMAX = 4;
  constexpr int POOL_V = POOL_DOUBLES * (int)(sizeof(double) / sizeof(V));
  constexpr int DW = F32 ? 2 : 1;  // words per staged D (hi, lo in mixed mode)
  const bool staged = (r + DW) <= (POOL_V - 64);
  V* Gs = reinterpret_cast<V*>(smem_pool());
  const int rows_per = staged ? max(1, min(len, (POOL_V - 64) / (r + DW))) : 1;
  V* Ds = Gs + (size_t)rows_per * r;  // D (FP64 mode) or D hi at [jj], D lo at [rows_per + jj]
  auto gload = [&](const double* p) -> V {
    if constexpr (F32) return d2f_rz(__ldcg(p));  // exact: the value is an FP32 number
    else return __ldcg(p);
  };
  for (long long base = 0; base < ntot; base += (long long)EMAX * tstride) {
    V acc[EMAX];
    CompSum cs[F32 ? EMAX : 1];
    double old[EMAX];  // current P / u entries, loaded before the products
#pragma unroll
    for (int q = 0; q < EMAX; ++q) acc[q] = V(0);
    const long long e0 = base + (long long)threadIdx.x * nw + (T.id() - w_lo);
#pragma unroll
    for (int q = 0; q < EMAX; ++q) {
      const long long e = e0 + (long long)q * tstride;
      old[q] = 0.0;
      if (e < nP) {
        const int i = (int)(e / r), l = (int)(e - (long long)i * r);
        old[q] = __ldcg(S.P + (size_t)i * rm + l);
      } else if (e < ntot) {
        old[q] = __ldcg(S.u + (e - nP));
      }
    }
    for (int jb = a; jb < a + len; jb += rows_per) {
      const int nr = min(rows_per, a + len - jb);
      if (staged) {
        __syncthreads();
#pragma unroll 8
        for (int e = threadIdx.x; e < nr * r; e += NT) {
          const int jj = e / r, i = e - jj * r;
          Gs[e] = gload(Gsrc + (size_t)(jb + jj) * rm + i);
        }
        for (int e = threadIdx.x; e < nr; e += NT) {
          if constexpr (F32) split_d(__ldcg(Dsrc + jb + e), Ds[e], Ds[rows_per + e]);
          else Ds[e] = __ldcg(Dsrc + jb + e);
        }
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < EMAX; ++q) {
        const long long e = e0 + (long long)q * tstride;
        if (e >= ntot) continue;
        const bool isP = e < nP;
        const int i = isP ? (int)(e / r) : (int)(e - nP);
        const int l = isP ? (int)(e - (long long)i * r) : 0;
        auto gi_of = [&](int jj) -> V { return staged ? Gs[jj * r + i] : gload(Gsrc + (size_t)(jb + jj) * rm + i); };
        auto gl_of = [&](int jj) -> V { return staged ? Gs[jj * r + l] : gload(Gsrc + (size_t)(jb + jj) * rm + l); };
        if constexpr (F32) {
          // FABsum: FP32 blocks of FAB_B rows (two independent FMA chains), each block
          // sum added to the compensated pair
          auto term = [&](float acc, int jj) -> float {
            const float gi = gi_of(jj);
            if (isP) return fmaf(gi, gl_of(jj), acc);
            float dh, dl;
            if (staged) {
              dh = Ds[jj];
              dl = Ds[rows_per + jj];
            } else {
              split_d(__ldcg(Dsrc + jb + jj), dh, dl);
            }
            return fmaf(gi, dh, fmaf(gi, dl, acc));
          };
          for (int j1 = 0; j1 < nr; j1 += FAB_B) {
            const int j2 = min(nr, j1 + FAB_B);
            float x0 = 0.f, x1 = 0.f;
            int jj = j1;
            for (; jj + 1 < j2; jj += 2) {
              x0 = term(x0, jj);
              x1 = term(x1, jj + 1);
            }
            if (jj < j2) x0 = term(x0, jj);
            cs[q].add(x0 + x1);
          }
        } else {
          auto gterm = [&](int jj) -> V {
            const V gi = gi_of(jj);
            const V gl = isP ? gl_of(jj) : (staged ? Ds[jj] : __ldcg(Dsrc + jb + jj));
            return gi * gl;
          };
          V x0 = V(0), x1 = V(0), x2 = V(0), x3 = V(0);  // four independent chains
          int jj = 0;
          for (; jj + 3 < nr; jj += 4) {
            x0 += gterm(jj);
            x1 += gterm(jj + 1);
            x2 += gterm(jj + 2);
            x3 += gterm(jj + 3);
          }
          for (; jj < nr; ++jj) x0 += gterm(jj);
          acc[q] += (x0 + x1) + (x2 + x3);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < EMAX; ++q) {
      const long long e = e0 + (long long)q * tstride;
      if (e >= ntot) continue;
      double add;
      if constexpr (F32) add = cs[q].value();
      else add = (double)acc[q];
      if (e < nP) {
        const int i = (int)(e / r), l = (int)(e - (long long)i * r);
        S.P[(size_t)i * rm + l] = old[q] + add;
      } else {
        S.u[e - nP] = old[q] + add;
      }
    }
  }
}

// Long runs, step 1: partial Gram sums per chunk of rows; CTA item = (16 x 16 tile pair
// with ti <= tl, chunk). Diagonal tiles also accumulate sum_j gamma_j D_j for their rows.
// F32 (mixed mode): compensated FP32 sums (FABsum; D as an FP32 hi/lo pair).
template <class Team, bool F32>
__device__ void gram_partials(const Team& T, const StreamDev& S, int a, int len, int r, int nch) {
  using V = typename std::conditional<F32, float, double>::type;
  V(*gi_s)[17] = reinterpret_cast<V(*)[17]>(smem_pool());
  V(*gl_s)[17] = gi_s + 32;
  V* d_s = reinterpret_cast<V*>(gl_s + 32);
  V* dl_s = d_s + 32;  // D lo (mixed mode)
  const int rm = S.r_max;
  const int nt = (r + 15) / 16;
  const int npairs = nt * (nt + 1) / 2;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int per = (len + nch - 1) / nch;
  auto gload = [&](const double* p) -> V {
    if constexpr (F32) return d2f_rz(__ldcg(p));  // exact: the value is an FP32 number
    else return __ldcg(p);
  };
  for (int it = T.id(); it < npairs * nch; it += T.size()) {
    const int c = it / npairs;
    int pr = it - c * npairs, ti = 0;
    while (pr >= nt - ti) {
      pr -= nt - ti;
      ++ti;
    }
    const int tl = ti + pr;
    const int jlo = a + c * per, jhi = min(a + len, jlo + per);
    V acc = V(0), uacc = V(0);
    CompSum pc, uc;
    for (int jb = jlo; jb < jhi; jb += 32) {
      __syncthreads();
#pragma unroll 2
      for (int e = threadIdx.x; e < 32 * 16; e += NT) {
        const int jj = e >> 4, cc = e & 15;
        const int j = jb + jj, i = ti * 16 + cc, l = tl * 16 + cc;
        gi_s[jj][cc] = (j < jhi && i < r) ? gload(S.G + (size_t)j * rm + i) : V(0);
        gl_s[jj][cc] = (j < jhi && l < r) ? gload(S.G + (size_t)j * rm + l) : V(0);
      }
      if (threadIdx.x < 32) {
        const bool ok = jb + threadIdx.x < jhi;
        if constexpr (F32) {
          float h = 0.f, l = 0.f;
          if (ok) split_d(__ldcg(S.Dall + jb + threadIdx.x), h, l);
          d_s[threadIdx.x] = h;
          dl_s[threadIdx.x] = l;
        } else {
          d_s[threadIdx.x] = ok ? __ldcg(S.Dall + jb + threadIdx.x) : V(0);
        }
      }
      __syncthreads();
      if constexpr (F32) {  // FABsum: FP32 blocks of FAB_B rows, compensated block sums
#pragma unroll
        for (int j1 = 0; j1 < 32; j1 += FAB_B) {
          float x0 = 0.f, x1 = 0.f;
#pragma unroll
          for (int jj = j1; jj < j1 + FAB_B; jj += 2) {
            x0 = fmaf(gi_s[jj][ty], gl_s[jj][tx], x0);
            x1 = fmaf(gi_s[jj + 1][ty], gl_s[jj + 1][tx], x1);
          }
          pc.add(x0 + x1);
          if (tx == 0) {
            float y0 = 0.f;
#pragma unroll
            for (int jj = j1; jj < j1 + FAB_B; ++jj)
              y0 = fmaf(gi_s[jj][ty], d_s[jj], fmaf(gi_s[jj][ty], dl_s[jj], y0));
            uc.add(y0);
          }
        }
      } else {
#pragma unroll 8
        for (int jj = 0; jj < 32; ++jj) {
          acc = fma(gi_s[jj][ty], gl_s[jj][tx], acc);
          if (tx == 0) uacc = fma(gi_s[jj][ty], d_s[jj], uacc);
        }
      }
    }
    const int i = ti * 16 + ty, l = tl * 16 + tx;
    double* Pc = S.Pp + (size_t)c * r * r;
    double pv, uv;
    if constexpr (F32) {
      pv = pc.value();
      uv = uc.value();
    } else {
      pv = acc;
      uv = uacc;
    }
    if (i < r && l < r) Pc[(size_t)i * r + l] = pv;
    if (ti == tl && tx == 0 && i < r) S.up[(size_t)c * rm + i] = uv;
  }
}

// Long runs, step 2: P += sum_c partials (both triangles), u += sum_c up.
template <class Team>
__device__ void gram_reduce(const Team& T, const StreamDev& S, int r, int nch) {
  const int rm = S.r_max;
  const long long tstride = (long long)T.size() * NT;
  const long long nP = (long long)r * r;
  for (long long e = rr_thread(T); e < nP + r; e += tstride) {
    if (e < nP) {
      const int i = (int)(e / r), l = (int)(e - (long long)i * r);
      const bool upper = (i >> 4) <= (l >> 4);
      const size_t src = upper ? (size_t)i * r + l : (size_t)l * r + i;
      double acc = 0.0;
      for (int c = 0; c < nch; ++c) acc += __ldcg(S.Pp + (size_t)c * r * r + src);
      const size_t o = (size_t)i * rm + l;
      S.P[o] = __ldcg(S.P + o) + acc;
    } else {
      const int i = (int)(e - nP);
      double acc = 0.0;
      for (int c = 0; c < nch; ++c) acc += __ldcg(S.up + (size_t)c * rm + i);
      S.u[i] = __ldcg(S.u + i) + acc;
    }
  }
}

// The grid team's tensor-core chunk path: P (both triangles) and u += the per-CTA staging
// slots [0, nslot) of the fused dependent-run sums (slot c: packed triangle at
// S.Pp + c r (r + 1) / 2, sums of gamma_j y_j at S.up + c r), added in slot order.
template <class Team>
__device__ void gram_reduce_slots(const Team& T, const StreamDev& S, int r, int nslot) {
  const int rm = S.r_max;
  const long long ntri = (long long)r * (r + 1) / 2;
  const long long tstride = (long long)T.size() * NT;
  for (long long e = rr_thread(T); e < ntri + r; e += tstride) {
    double acc = 0.0;
    if (e < ntri) {
      for (int c = 0; c < nslot; ++c) acc += __ldcg(S.Pp + (size_t)c * ntri + e);
      int rem = (int)e, i = 0;
      while (rem >= r - i) {
        rem -= r - i;
        ++i;
      }
      const int l = i + rem;
      S.P[(size_t)i * rm + l] = __ldcg(S.P + (size_t)i * rm + l) + acc;
      if (l != i) S.P[(size_t)l * rm + i] = __ldcg(S.P + (size_t)l * rm + i) + acc;
    } else {
      const int i = (int)(e - ntri);
      for (int c = 0; c < nslot; ++c) acc += __ldcg(S.up + (size_t)c * r + i);
      S.u[i] = __ldcg(S.u + i) + acc;
    }
  }
}

template <class Team, bool F32>
__device__ __forceinline__ void acc_small(const Team& T, const StreamDev& S, int a, int len, int r) {
  acc_rows<Team, F32>(T, S, S.G, S.Dall, a, len, r, 0);
}

// A run of dependent rows [a, a + len): short runs directly, long runs through chunked
// partial sums. Returns false if a team barrier gave up. The caller syncs afterwards.
// F32 (mixed mode): the per-chunk sums of gamma gamma^T and gamma D are compensated FP32
// sums (FABsum) of the FP32 projections, added to the FP64 P and u.
template <class Team, bool F32>
__device__ bool dep_run(const Team& T, const StreamDev& S, int a, int len, int r) {
  if (len <= 0 || r == 0) return true;
  const size_t rr = (size_t)r * r;
  if (len > SMALL_B && S.Pp && S.pp_cap >= rr) {
    int nch = (int)min((size_t)NCH_MAX, S.pp_cap / rr);
    nch = max(1, min(nch, (len + GRAM_CHUNK - 1) / GRAM_CHUNK));
    gram_partials<Team, F32>(T, S, a, len, r, nch);
    if (!T.sync()) return false;
    gram_reduce(T, S, r, nch);
    return true;
  }
  acc_small<Team, F32>(T, S, a, len, r);
  return true;
}

// =======================================================================================
// Sequential section: rows [q0, bend) (at most SLOW_MAX) with FP64 coordinates in S.G and
// FP64 rejections in S.R (row j at S.R[(j - q0) * ld]). Rows are decided in order; after
// an append the later rejections of the section lose the new direction
// (Gamma_r,t -= kappa_t Gamma_r,j with kappa_t = Gamma_r,j^T Gamma_r,t / s_j, modified
// Gram-Schmidt, valid because Gamma_r,j is orthogonal to span(C)).
//
// The columns are split over the first nact = min(workers, ceil(m / NT)) workers. Per row
// every column owner forms its part of s_j = ||Gamma_r,j||^2 and of the dot products with
// the later rows, the parts are summed (across the warps of a CTA in shared memory; across
// CTAs through S.Sp, double-buffered by row parity, after a barrier over the nact workers
// only, always in the same order), and every owner takes the same decision. Each thread
// keeps its column of the section's rejections in registers when it owns one column
// (REG), otherwise they stay in shared memory (S.Rs, when they fit) or in S.R.
// Only decisions, kappa_t, the new basis rows K and the append records are produced in the
// row loop; worker 0 then replays the appends on the coordinates of the section's rows
// (gamma_t <- [gamma_t - kappa_t gamma_j; kappa_t], orthonormal: [gamma_t; kappa_t sqrt(s_j)])
// in one pass in which every thread owns one coordinate, and forms the a-priori errors
// D_t = y_t - gamma_t^T w_b with w_b as it stands when row t is reached.
// Publishes {applied, r_new, n_ind} in CTRL_APPLIED / CTRL_RNEW / CTRL_NIND; the caller
// reads them after its next team barrier. Returns false if a bounded wait gave up.
// =======================================================================================
__device__ __forceinline__ bool sub_barrier(int* ctrl, int sub_off, int n, unsigned long long& target) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(ctrl + sub_off);
    target += (unsigned long long)n;
    red_release_add_u64(cnt, 1ull);
    if (ld_acquire_u64(cnt) < target) {
      const unsigned long long t0 = global_ns();
      while (ld_acquire_u64(cnt) < target) {
        if (global_ns() - t0 > WAIT_LIMIT_NS) {
          atomicOr(ctrl + CTRL_STATUS, ST_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

// Sums this worker's 32 partials (one set per thread) over the CTA and over the nact
// column owners; the result lands in tot[0..31] for every thread of every owner.
template <class Team>
__device__ __forceinline__ bool scan_exchange(const Team& T, const StreamDev& S, double (&v)[32], int nact,
                                              int parity, unsigned long long& bar_target, double* tot,
                                              double (*wred)[32], bool warp_active, int nlive) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // a warp without columns holds zeros; with at most 16 live values (the later rows of the
  // section) a 16-value butterfly does (15 FP64 adds instead of 31)
  if (!warp_active) {
    wred[warp][lane] = 0.0;
  } else if (nlive <= 16) {
    double h[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) h[k] = v[k];
    const double t16 = warp_transpose_sum<double, 16>(h);
    const int q = transpose_sum_index<16>();
    if ((lane & 1) == 0) wred[warp][q] = t16;
    if (lane >= 16) wred[warp][lane] = 0.0;  // values 16..31: not live
  } else {
    warp_transpose_sum32(v);  // lane l holds the warp's sum of value l
    wred[warp][lane] = v[0];
  }
  __syncthreads();
  double a = 0.0;
  if (threadIdx.x < 32) {
#pragma unroll
    for (int w2 = 0; w2 < NWARP; ++w2) a += wred[w2][threadIdx.x];
  }
  if (nact > 1) {
    double* Sp = S.Sp + (size_t)parity * S.sp_stride;
    if (threadIdx.x < 32) Sp[(size_t)T.id() * 32 + threadIdx.x] = a;
    if (!sub_barrier(S.ctrl, S.sub_off, nact, bar_target)) return false;
    if (threadIdx.x < 32) {
      a = 0.0;
      for (int w2 = 0; w2 < nact; ++w2) a += __ldcg(Sp + (size_t)w2 * 32 + threadIdx.x);
    }
  }
  if (threadIdx.x < 32) tot[threadIdx.x] = a;
  __syncthreads();
  return true;
}

template <class Team, int VAR>
__device__ bool scan_team(const Team& T, const StreamDev& S, const CallArgs& A, long long j0, int q0,
                          int bend, int r) {
  constexpr bool ORTHO = VAR == VAR_ORTHONORMAL;
  // the new basis row kept in Kv: general K = Gamma_r / s (the new dual row), orthonormal
  // Gamma_r / sqrt(s), orthogonal Gamma_r itself
  auto kv_scale = [](double is, double rsq) -> double {
    return VAR == VAR_ORTHONORMAL ? rsq : (VAR == VAR_ORTHOGONAL ? 1.0 : is);
  };
  const int m = S.m, ld = S.ld, rm = S.r_max;
  const int nrow = bend - q0;
  // grid teams: one warp per CTA owns 32 columns (registers), so that the FP64 work of a
  // row (partials, their reduction, the fix-ups) spreads over ceil(m / 32) SMs; otherwise
  // (one-CTA teams, or m beyond 32 columns per CTA) every thread owns columns
  constexpr bool kGrid = std::is_same<Team, GridTeam>::value;
  const long long nwarp_cols = ((long long)m + 31) / 32;
  const bool reg = kGrid && nwarp_cols <= T.size() && nwarp_cols <= 20 * NWARP;
  const int nact = reg ? (int)nwarp_cols : (int)min((long long)T.size(), ((long long)m + NT - 1) / NT);
  __shared__ double tot[32];
  __shared__ double wred[NWARP][32];
  __shared__ double ts[32], ys[32], sq_s[32];  // t_j, y_j, sqrt(s_j) of the section rows
  __shared__ int flag_s[32];
  __shared__ int dec_s;
  __shared__ double is_s, rsq_s;  // 1 / s_j and 1 / sqrt(s_j) of an independent row
  const int tid = threadIdx.x;
  int rc = r, nind = 0, applied = bend;
  if (T.id() < nact) {
    const long long base_row = __ldcg(S.rows_seen);
    if (tid < 32) {
      ts[tid] = (tid < nrow) ? __ldcg(S.t + q0 + tid) : 0.0;
      ys[tid] = (tid < nrow) ? __ldg(A.y + j0 + q0 + tid) : 0.0;
      flag_s[tid] = 0;
    }
    __shared__ unsigned long long bar_target_s;
    if (tid == 0 && nact > 1) {
      const unsigned long long c = ld_acquire_u64(reinterpret_cast<unsigned long long*>(S.ctrl + S.sub_off));
      bar_target_s = (c / (unsigned long long)nact) * (unsigned long long)nact;
    }
    __syncthreads();
    unsigned long long bar_target = bar_target_s;
    const long long cstride = (long long)nact * NT;
    // decision of row jj (thread 0), records (worker 0), kappa of the later rows
    auto decide = [&](int jj) -> int {
      const int j = q0 + jj;
      if (tid == 0) {
        const double s = tot[0], t = ts[jj], yv = ys[jj];
        int d = 0;
        if (!isfinite(t) || !isfinite(yv) || !isfinite(s)) d = -1;
        else if (is_independent(s, t, rc, m, S.tol, S.test_mode)) d = (rc >= rm) ? -2 : 1;
        // the reciprocals are formed once, here, by Newton-Raphson (FP64 division and
        // square root are long dependent chains on this part)
        const double is = (d == 1) ? rcp_nr(s) : 0.0, rsq = (d == 1) ? rsqrt_nr(s) : 0.0;
        if (T.id() == 0) {
          if (d < 0) {
            atomicOr(S.ctrl + CTRL_STATUS, d == -1 ? ST_NONFINITE : ST_CAPACITY);
          } else {
            flag_s[jj] = d + 1;
            S.rowflag[j] = (uint8_t)(d + 1);
            sq_s[jj] = s * rsq;
            if (d == 1) {
              S.jind[nind] = j;
              S.alpha[nind] = rsq;
              S.basis_rows[rc] = base_row + j;
              S.wb[rc] = VAR == VAR_GENERAL ? yv : 0.0;  // w_b <- [w_b; y] (general), [w_b; 0] (Section 2.2)
            }
          }
        }
        is_s = is;
        rsq_s = rsq;
        dec_s = d;
      }
      __syncthreads();
      const int d = dec_s;
      if (d == 1 && T.id() == 0 && tid >= 1 && tid < 32 && jj + tid < nrow)
        S.Kap[nind * SLOW_MAX + jj + tid] = tot[tid] * is_s;
      return d;
    };
    if constexpr (kGrid) {
      static_assert(4 * NWARP == SLOW_MAX, "four section rows per warp");
      if (reg) {
      // Each CTA owns 32 columns (lane = column); warp w holds the rejections of section
      // rows 4w .. 4w + 3 on them, so the FP64 work of a row (its products with the later
      // rows and their fix-ups) is spread over the 8 warps and the SM's four FP64 units.
      const int lane = tid & 31, warp = tid >> 5;
      const long long c = (long long)T.id() * 32 + lane;
      const bool colv = c < m;
      __shared__ double rcur[32];   // the current row's rejection on the CTA's columns
      __shared__ double cpart[32];  // the CTA's part of R_jj . R_t for section rows t
      double Rw[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int t = 4 * warp + i;
        Rw[i] = (colv && t < nrow) ? __ldcg(S.R + (size_t)t * ld + c) : 0.0;
      }
      for (int jj = 0; jj < nrow; ++jj) {
        if (warp == (jj >> 2)) {
          const int i = jj & 3;
          rcur[lane] = i == 0 ? Rw[0] : i == 1 ? Rw[1] : i == 2 ? Rw[2] : Rw[3];
        }
        __syncthreads();
        const double rj = rcur[lane];
        double v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = (4 * warp + i >= jj) ? rj * Rw[i] : 0.0;
        warp_transpose_sum<double, 4>(v);
        if ((lane & 7) == 0) cpart[4 * warp + transpose_sum_index<4>()] = v[0];
        __syncthreads();
        if (tid < 32) {  // lane k: row jj + k
          const double pv = (jj + tid < 32) ? cpart[jj + tid] : 0.0;
          if (nact > 1) S.Sp[(size_t)(jj & 1) * S.sp_stride + (size_t)T.id() * 32 + tid] = pv;
          else tot[tid] = pv;
        }
        if (nact > 1) {
          if (!sub_barrier(S.ctrl, S.sub_off, nact, bar_target)) return false;
          // value k = lane, summed over the owners w = warp, warp + NWARP, ... (a fixed
          // pairwise tree, all loads issued first: up to 20 owners per warp), then over
          // the warps; every CTA sums in the same order
          const double* Sp = S.Sp + (size_t)(jj & 1) * S.sp_stride;
          double pv[20];
#pragma unroll
          for (int q = 0; q < 20; ++q) {
            const int w2 = warp + q * NWARP;
            pv[q] = (w2 < nact) ? __ldcg(Sp + (size_t)w2 * 32 + lane) : 0.0;
          }
#pragma unroll
          for (int h = 16; h >= 1; h >>= 1)
#pragma unroll
            for (int q = 0; q < h; ++q)
              if (q + h < 20) pv[q] += pv[q + h];
          wred[warp][lane] = pv[0];
          __syncthreads();
          if (tid < 32) {
            const double a0 = wred[0][tid] + wred[1][tid], a1 = wred[2][tid] + wred[3][tid];
            const double a2 = wred[4][tid] + wred[5][tid], a3 = wred[6][tid] + wred[7][tid];
            tot[tid] = (a0 + a1) + (a2 + a3);
          }
        }
        __syncthreads();
        const int d = decide(jj);
        if (d < 0) {
          applied = q0 + jj;
          break;
        }
        if (d == 1) {
          const double is = is_s;
          const double scale = kv_scale(is, rsq_s);
          if (warp == 0 && colv) S.Kv[(size_t)nind * ld + c] = rj * scale;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int t = 4 * warp + i;
            if (t > jj) Rw[i] = fma(-tot[t - jj] * is, rj, Rw[i]);
          }
          ++rc;
          ++nind;
        }
      }
      }
    }
    if (!reg) {
      // rejections in shared memory (row stride m) when they fit, else in S.R (global,
      // read through L2 since other CTAs wrote it); `rsm` selects plain shared-memory loads
      double* Rb = S.R;
      long long ldr = ld;
      bool rsm = false;
      if (nact == 1 && S.Rs && (long long)nrow * m <= S.rs_cap) {
        for (long long e = tid; e < (long long)nrow * m; e += NT) {
          const long long k = e / m, c = e - k * m;
          S.Rs[e] = __ldcg(S.R + (size_t)k * ld + c);
        }
        __syncthreads();
        Rb = S.Rs;
        ldr = m;
        rsm = true;
      }
      auto rload = [&](const double* p) -> double { return rsm ? *p : __ldcg(p); };
      const long long col0 = (long long)T.id() * NT + tid;
      if (rsm) {
        // One CTA holds every column, the rejections in shared memory: warp w owns section
        // rows w, w + 8, w + 16, w + 24. Per row jj each warp forms the products of its rows
        // t >= jj with row jj (lanes over the columns, one 4-value butterfly; the owner of jj
        // gets s_jj), so no sum across warps is needed; after the decision each warp fixes
        // up its own later rows.
        const int lane = tid & 31, warp = tid >> 5;
        for (int jj = 0; jj < nrow; ++jj) {
          const double* rj = Rb + (size_t)jj * ldr;
          double v[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            v[i] = 0.0;
            const int t = warp + NWARP * i;
            if (t >= jj && t < nrow) {  // the warp's live rows only (the test is warp-uniform)
              const double* rt = Rb + (size_t)t * ldr;
              double a0 = 0.0, a1 = 0.0;
              int c = lane;
              for (; c + 32 < m; c += 64) {
                a0 = fma(rj[c], rt[c], a0);
                a1 = fma(rj[c + 32], rt[c + 32], a1);
              }
              if (c < m) a0 = fma(rj[c], rt[c], a0);
              v[i] = a0 + a1;
            }
          }
          warp_transpose_sum<double, 4>(v);
          if ((lane & 7) == 0) {  // lanes 8 q .. 8 q + 7 hold the total of row warp + NWARP q
            const int t = warp + NWARP * transpose_sum_index<4>();
            if (t >= jj && t < nrow) tot[t - jj] = v[0];
          }
          __syncthreads();
          const int d = decide(jj);
          if (d < 0) {
            applied = q0 + jj;
            break;
          }
          if (d == 1) {
            const double is = is_s;
            const double scale = kv_scale(is, rsq_s);
            for (int c = tid; c < m; c += NT) S.Kv[(size_t)nind * ld + c] = rj[c] * scale;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int t = warp + NWARP * i;
              if (t > jj && t < nrow) {
                const double nk = -tot[t - jj] * is;
                double* rt = Rb + (size_t)t * ldr;
                for (int c = lane; c < m; c += 32) rt[c] = fma(nk, rj[c], rt[c]);
              }
            }
            ++rc;
            ++nind;
          }
          __syncthreads();  // the fixed-up rows before the next row's products
        }
      } else
      for (int jj = 0; jj < nrow; ++jj) {
        double v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = 0.0;
        for (long long c = col0; c < m; c += cstride) {
          const double rj = rload(Rb + (size_t)jj * ldr + c);
#pragma unroll
          for (int k = 0; k < 32; ++k)
            if (jj + k < nrow) v[k] = fma(rj, rload(Rb + (size_t)(jj + k) * ldr + c), v[k]);
        }
        const bool wact = (long long)T.id() * NT + (threadIdx.x & ~31) < m;  // the warp owns columns
        if (!scan_exchange(T, S, v, nact, jj & 1, bar_target, tot, wred, wact, nrow - jj)) return false;
        const int d = decide(jj);
        if (d < 0) {
          applied = q0 + jj;
          break;
        }
        if (d == 1) {
          const double is = is_s;
          const double scale = kv_scale(is, rsq_s);
          __shared__ double negk[32];  // -kappa_t of the later rows, formed once
          if (tid < 32) negk[tid] = -tot[tid] * is;
          __syncthreads();
          for (long long c = col0; c < m; c += cstride) {
            const double rj = rload(Rb + (size_t)jj * ldr + c);
            S.Kv[(size_t)nind * ld + c] = rj * scale;
#pragma unroll
            for (int k = 1; k < 32; ++k)
              if (jj + k < nrow) {
                double* rt = Rb + (size_t)(jj + k) * ldr + c;
                *rt = fma(negk[k], rj, rload(rt));
              }
          }
          ++rc;
          ++nind;
        }
      }
    }
  }
  if (T.id() == 0) {
    // replay the appends on the coordinates: thread = coordinate i (of the final rank rc);
    // the kappas are staged in the shared pool first
    const int napp = applied - q0;
    __syncthreads();
    double* kap_s = smem_pool();
    for (int e = tid; e < nind * SLOW_MAX; e += NT) kap_s[e] = __ldcg(S.Kap + e);
    __syncthreads();
    for (int i0 = 0; i0 < rc; i0 += NT) {
      const int i = i0 + tid;
      double g[32];
#pragma unroll
      for (int tt = 0; tt < 32; ++tt) g[tt] = (tt < napp && i < r) ? __ldcg(S.G + (size_t)(q0 + tt) * rm + i) : 0.0;
      int rcv = r, q = 0;
#pragma unroll
      for (int tt = 0; tt < 32; ++tt) {
        if (tt < napp) {
          if (i < rcv) S.G[(size_t)(q0 + tt) * rm + i] = g[tt];
          if (flag_s[tt] == 2) {
            if (i < rcv) S.Gind[(size_t)q * rm + i] = g[tt];
            const double sq = sq_s[tt];
#pragma unroll
            for (int t2 = tt + 1; t2 < 32; ++t2) {
              if (t2 < napp) {
                const double kap = kap_s[q * SLOW_MAX + t2];
                if (i < rcv) {  // general: the raw row also has components on the old basis
                  if (VAR == VAR_GENERAL) g[t2] = fma(-kap, g[tt], g[t2]);
                } else if (i == rcv) {  // coordinate on the new basis row
                  g[t2] = ORTHO ? kap * sq : kap;
                }
              }
            }
            ++rcv;
            ++q;
          }
        }
      }
    }
    __syncthreads();
    // a-priori errors: one warp per row, w_b entries below the rank the row saw
    const int lane = tid & 31, warp = tid >> 5;
    for (int tt = warp; tt < napp; tt += NWARP) {
      int rk = r;
      for (int u2 = 0; u2 < tt; ++u2) rk += (flag_s[u2] == 2);
      const double* g = S.G + (size_t)(q0 + tt) * rm;
      double acc = 0.0;
      for (int l = lane; l < rk; l += 32) acc = fma(__ldcg(g + l), __ldcg(S.wb + l), acc);
      acc = warp_sum(acc);
      if (lane == 0) S.Dall[q0 + tt] = ys[tt] - acc;
    }
    if (tid == 0) {
      S.ctrl[CTRL_APPLIED] = applied;
      S.ctrl[CTRL_RNEW] = rc;
      S.ctrl[CTRL_NIND] = nind;
    }
  }
  return true;
}

// Apply the sequential section's rows [q0, q0 + napp) to P and u (team-wide, one thread
// per entry of the new r_new x r_new P and of u). Rows are taken in order with the rank
// r_j each saw: a dependent row adds gamma_j gamma_j^T on the leading r_j x r_j block and
// gamma_j D_j to u; an independent row opens entry r_j (general: P_jj = 1; orthonormal and
// orthogonal: adds g g^T with g = [gamma_j; 1/alpha_j] and g D_j to u, alpha_j = 1 for the
// orthogonal variant).
template <class Team, int VAR>
__device__ void section_apply_pu(const Team& T, const StreamDev& S, int q0, int napp, int r,
                                 int rnew) {
  const int rm = S.r_max;
  // per-row data of the section, staged once per CTA: flag, rank the row saw, append index,
  // 1/alpha of an appended row (one FP64 division per row, not per entry) and D
  __shared__ int fl_s[SLOW_MAX], rj_s[SLOW_MAX], q_s[SLOW_MAX];
  __shared__ double ia_s[SLOW_MAX], d_s[SLOW_MAX], al_s[SLOW_MAX];
  __syncthreads();
  if (threadIdx.x < napp) {
    fl_s[threadIdx.x] = __ldcg(S.rowflag + q0 + threadIdx.x);
    d_s[threadIdx.x] = __ldcg(S.Dall + q0 + threadIdx.x);
    if (VAR == VAR_ORTHONORMAL) al_s[threadIdx.x] = __ldcg(S.alpha + threadIdx.x);
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // the rank each row saw and its append index (integers only)
    int rj = r, q = 0;
    for (int jj = 0; jj < napp; ++jj) {
      rj_s[jj] = rj;
      q_s[jj] = q;
      if (fl_s[jj] != 1) {
        ++rj;
        ++q;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < napp)  // one division per appended row, all rows at once
    ia_s[threadIdx.x] = (VAR == VAR_ORTHONORMAL && fl_s[threadIdx.x] != 1) ? 1.0 / al_s[q_s[threadIdx.x]] : 1.0;
  __syncthreads();
  // the section rows' coordinate vectors g_j (gamma_j up to the rank the row saw; an
  // appended row of the variants of Section 2.2 adds 1/alpha_j after them; zero beyond),
  // staged once in the shared pool when they fit; the sums below run in the same order
  // either way
  const bool staged = (long long)napp * rnew <= POOL_DOUBLES;
  double* gs = smem_pool();
  if (staged) {
    for (int e = threadIdx.x; e < napp * rnew; e += NT) {
      const int jj = e / rnew, i = e - jj * rnew;
      const int rj = rj_s[jj];
      double v = 0.0;
      if (fl_s[jj] == 1) {
        if (i < rj) v = __ldcg(S.G + (size_t)(q0 + jj) * rm + i);
      } else if (VAR != VAR_GENERAL) {
        if (i < rj) v = __ldcg(S.Gind + (size_t)q_s[jj] * rm + i);
        else if (i == rj) v = ia_s[jj];
      }
      gs[e] = v;
    }
    __syncthreads();
  }
  const long long tstride = (long long)T.size() * NT;
  const long long nP = (long long)rnew * rnew;
  for (long long e = rr_thread(T); e < nP + rnew; e += tstride) {
    const bool isP = e < nP;
    const int i = isP ? (int)(e / rnew) : (int)(e - nP);
    const int l = isP ? (int)(e - (long long)i * rnew) : 0;
    double acc = 0.0;
    if (staged) {
      for (int jj = 0; jj < napp; ++jj) {
        const double gi = gs[jj * rnew + i];
        acc = fma(gi, isP ? gs[jj * rnew + l] : d_s[jj], acc);
        if (VAR == VAR_GENERAL && fl_s[jj] != 1 && isP && i == rj_s[jj] && l == rj_s[jj]) acc += 1.0;
      }
    } else
    for (int jj = 0; jj < napp; ++jj) {
      const int rj = rj_s[jj];
      const double* g = S.G + (size_t)(q0 + jj) * rm;
      if (fl_s[jj] == 1) {  // dependent
        if (isP) {
          if (i < rj && l < rj) acc = fma(__ldcg(g + i), __ldcg(g + l), acc);
        } else if (i < rj) {
          acc = fma(__ldcg(g + i), d_s[jj], acc);
        }
      } else {  // independent: opens entry rj
        if (VAR != VAR_GENERAL) {  // g = [gamma_j; 1/alpha_j], alpha = 1 (orthogonal)
          const double ia = ia_s[jj];
          const double* gq = S.Gind + (size_t)q_s[jj] * rm;
          const double gi = (i < rj) ? __ldcg(gq + i) : (i == rj ? ia : 0.0);
          if (isP) {
            const double gl = (l < rj) ? __ldcg(gq + l) : (l == rj ? ia : 0.0);
            acc = fma(gi, gl, acc);
          } else {
            acc = fma(gi, d_s[jj], acc);
          }
        } else if (isP && i == rj && l == rj) {
          acc += 1.0;
        }
      }
    }
    if (isP) {
      const size_t o = (size_t)i * rm + l;
      const double base = (i < r && l < r) ? __ldcg(S.P + o) : 0.0;
      S.P[o] = base + acc;
    } else {
      const double base = (i < r) ? __ldcg(S.u + i) : 0.0;
      S.u[i] = base + acc;
    }
  }
}

// Appends of the sequential section to the basis, team-wide.
// Orthogonal variant: C[r + q] = Gamma_r,q and Ct[r + q] = Gamma_r,q / ||Gamma_r,q||^2.
// General variant: Ct_final[i] = base_i - sum_{q >= qmin(i)} Gind[q][i] K_q with
// base_i = Ct[i] (i < r) or K_{i-r}, qmin(i) = max(0, i - r + 1); C[r + q] = Gamma_{jind[q]}.
// Orthonormal variant: Q[r + q] = alpha_q Gamma_r (already scaled in Kv) and, with FP32
// projections, its FP32 copy.
template <class Team, int VAR>
__device__ void section_apply_basis(const Team& T, const StreamDev& S, const CallArgs& A, long long j0,
                                    int r, int nind) {
  const int m = S.m, ld = S.ld, rm = S.r_max;
  const long long gt = (long long)T.id() * NT + threadIdx.x;
  const long long tstride = (long long)T.size() * NT;
  if (VAR == VAR_ORTHOGONAL) {  // C[r + q] = Gamma_r (in Kv), Ct[r + q] = Gamma_r / s; old rows kept
    const long long n = (long long)nind * m;
    for (long long e = gt; e < n; e += tstride) {
      const int q = (int)(e / m), c = (int)(e - (long long)q * m);
      const double v = __ldcg(S.Kv + (size_t)q * ld + c);
      const double a = __ldcg(S.alpha + q);  // 1 / sqrt(s)
      S.C[(size_t)(r + q) * ld + c] = v;
      S.Ct[(size_t)(r + q) * ld + c] = v * a * a;
    }
    return;
  }
  if (VAR == VAR_ORTHONORMAL) {
    const long long n = (long long)nind * m;
    for (long long e = gt; e < n; e += tstride) {
      const int q = (int)(e / m), c = (int)(e - (long long)q * m);
      const double v = __ldcg(S.Kv + (size_t)q * ld + c);
      S.C[(size_t)(r + q) * ld + c] = v;
      if (S.Qf) S.Qf[(size_t)(r + q) * ld + c] = (float)v;
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

// =======================================================================================
// Apply the k rows of one call to one stream, team-wide. Returns false if a bounded team
// barrier gave up (the status word then holds ST_TIMEOUT). Every worker runs the same
// control flow; values decided by worker 0 are read back after a barrier.
//
// Block of b rows: gamma | rejections, norms and a-priori errors | then
//  * b <= SMALL_B, all rows dependent: every worker decides redundantly and accumulates
//    into P and u at once (two barriers per block, none after the last block);
//  * otherwise: worker 0 decides; the dependent run before the first special row is
//    accumulated; from that row the sequential FP64 section applies the rank changes.
// =======================================================================================
// Growth factor of the block size after a block whose rows were all dependent (it falls
// back to KB_MIN after a rank change): 2, except for mixed mode on the whole GPU, where
// blocks of TC_GRID_MIN rows and more go to the tensor cores and are reached sooner with 4.
template <class Team, bool F32>
__device__ __forceinline__ int kb_growth() {
  return (F32 && std::is_same<Team, GridTeam>::value) ? 4 : 2;
}

// Steps 4 and 5 of a block whose rows [0, b) (call rows j0 + [0, b)) have their gamma in
// S.G, their norms in S.s / S.t and their a-priori errors in S.Dall, and whose first row
// that needs the sequential section is q0 (b if none): the dependent run before q0 (unless
// run_done: the tensor-core projection already added it to P and u), the
// FP64 section from q0 (rank tests in order, appends, fix-ups of the later rows), and the
// block's bookkeeping (flags, counters, rank, next block size), followed by a team barrier.
// Returns the rows applied, or -1 if a bounded team barrier gave up.
template <class Team, bool F32, int VAR>
__device__ int block_tail(const Team& T, const StreamDev& S, const CallArgs& A, long long j0, int b,
                          int r, int q0, int kb0, bool run_done = false) {
  constexpr bool ORTHO = VAR == VAR_ORTHONORMAL;  // the projection basis is C itself
  __shared__ int shc[3];
  const double* gam = A.Gamma + (size_t)j0 * S.m;
  // 4: dependent run before the first special row (unless already summed: run_done)
  if (q0 > 0 && !run_done && !dep_run<Team, F32>(T, S, 0, q0, r)) return -1;
  int applied = b, rnew = r;
  if (q0 < b) {
    // 5: sequential section, in FP64 (rows [q0, bend)); its rows never overlap the run
    const int bend = min(b, q0 + SLOW_MAX);
    if (std::is_same<Team, GridTeam>::value)
      phase_gamma_small_any<Team, false>(T, S, gam, q0, bend, r, ORTHO ? S.C : S.Ct);
    else if ((long long)((bend - q0 + 7) / 8) * r < 4LL * NWARP * T.size())
      phase_gamma_cta(T, S, gam, q0, bend, r, ORTHO ? S.C : S.Ct);
    else
      phase_gamma<Team, false>(T, S, gam, q0, bend, r, ORTHO ? S.C : S.Ct);
    if (!T.sync()) return -1;
    // one-CTA teams: the section's rows as one 32-row item per column chunk (its items run
    // one after another there, so fewer, larger items)
    if constexpr (std::is_same<Team, CtaTeam>::value) phase_reject<Team, false, 8>(T, S, gam, q0, bend, r, S.C, S.R);
    else phase_reject<Team, false, 1>(T, S, gam, q0, bend, r, S.C, S.R);
    if (!T.sync()) return -1;
    if (!scan_team<Team, VAR>(T, S, A, j0, q0, bend, r)) return -1;
    // the scan may have used the dynamic shared memory that caches the tensor-core B tiles
    if (S.tcx && threadIdx.x == 0) reinterpret_cast<TcCtx*>(S.tcx)->cq = nullptr;
    if (!T.sync()) return -1;
    if (threadIdx.x == 0) {
      shc[0] = __ldcg(S.ctrl + CTRL_APPLIED);  // published before the barrier above
      shc[1] = __ldcg(S.ctrl + CTRL_RNEW);
      shc[2] = __ldcg(S.ctrl + CTRL_NIND);
    }
    __syncthreads();
    applied = shc[0];
    rnew = shc[1];
    const int nind = shc[2];
    section_apply_pu<Team, VAR>(T, S, q0, applied - q0, r, rnew);
    if (nind > 0) section_apply_basis<Team, VAR>(T, S, A, j0, r, nind);
  }
  // finalize the block (worker 0): flags, counters, rank, next block size
  if (T.id() == 0) {
    if (A.indep)
      for (int j = threadIdx.x; j < applied; j += NT)
        A.indep[j0 + j] = (j < q0) ? 0 : (uint8_t)(__ldcg(S.rowflag + j) - 1);
    if (threadIdx.x == 0) {
      *S.rows_seen = __ldcg(S.rows_seen) + applied;
      S.ctrl[CTRL_R] = rnew;
      S.ctrl[CTRL_KB] = (q0 < b) ? min(KB_MIN, S.kb_max) : min(kb_growth<Team, F32>() * kb0, S.kb_max);
      S.ctrl[CTRL_PEND] = 1;
      S.ctrl[CTRL_PEND_ROWS] = 0;
    }
  }
  if (!T.sync()) return -1;
  return applied;
}

// TCG: the kernel carries the tensor-core chunk path of large mixed-mode blocks on a grid
// team (stream_tc_kernel); the other grid kernels leave it out.
template <class Team, bool F32, int VAR = (F32 ? VAR_ORTHONORMAL : VAR_GENERAL), bool TCG = false>
__device__ bool process_rows(const Team& T, const StreamDev& S, const CallArgs& A) {
  constexpr bool ORTHO = VAR == VAR_ORTHONORMAL;  // the projection basis is C itself
  __shared__ int sh[8];
  constexpr bool kGridTeam = std::is_same<Team, GridTeam>::value;
  __shared__ __align__(8) unsigned long long pf_bar;  // rejection-tile prefetch (RejPrefetch)
  uint32_t pf_ph = 0;
  if (kGridTeam && threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&pf_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // grid teams: the call's first rows (up to a small block) into L2 while the control
  // words are read, each CTA asking for its share
  if (kGridTeam && threadIdx.x == 0) {
    const size_t bytes = (size_t)min(A.k, (long long)SMALL_B) * S.m * 8;
    const size_t share = ((bytes + T.size() - 1) / T.size() + 255) & ~(size_t)255;
    const size_t off = share * T.id();
    if (off < bytes) l2_prefetch(reinterpret_cast<const char*>(A.Gamma) + off, min(share, bytes - off));
  }
  long long j0 = 0;
  while (j0 < A.k) {
    if (threadIdx.x == 0) {  // written before the last barrier or by an earlier launch
      sh[0] = __ldcg(S.ctrl + CTRL_STATUS);
      sh[1] = __ldcg(S.ctrl + CTRL_R);
      sh[2] = __ldcg(S.ctrl + CTRL_KB);
      sh[4] = S.Gpend ? __ldcg(S.ctrl + CTRL_PEND_ROWS) : 0;
    }
    __syncthreads();
    if (sh[0] != 0) break;
    const int r = sh[1];
    const int kb0 = sh[2];
    const int b = (int)min((long long)kb0, A.k - j0);
    const bool last = (j0 + b == A.k);
    const double* gam = A.Gamma + (size_t)j0 * S.m;
    __syncthreads();
    // mixed mode, one CTA per stream: projection, rejection norms and the FP32 screen on
    // the tensor cores (q0 = first row the screen cannot clear)
    int q0 = -2;
    bool gram_done = false;  // the dependent-run sums were fused into the projection
    if constexpr (F32 && std::is_same<Team, CtaTeam>::value) {
      if (S.tcx && r >= 1 && r <= TC_RMAX) {
        double tcut = S.tau_lo;
        if (S.test_mode == 0 && S.tol > 0.0) tcut = fmax(tcut, 0.5 * S.tol);
        __shared__ bool gd;
        const bool want_gram = S.Pp && S.pp_cap >= (size_t)r * r && S.up;
        q0 = tc_project_block(reinterpret_cast<TcCtx*>(S.tcx), S, gam, A.y + j0, b, r, tcut, A.k - j0,
                              reinterpret_cast<float*>(smem_pool()), want_gram, &gd,
                              TcOut{0, S.Pp, S.up, true, true});
        if (q0 < 0) return false;
        gram_done = gd;
        phase_dall(T, S, A, j0, b, r);
        if (!T.sync()) return false;
      }
    }
    // mixed mode, whole GPU, blocks of at least TC_GRID_MIN rows: the same tensor-core
    // projection, each CTA taking 128-row chunks of the block (q0 = the first row that any
    // chunk's screen cannot clear; the CTAs' fused sums are reduced when there is none)
    if constexpr (F32 && kGridTeam && TCG) {
      if (S.tcx && b >= TC_GRID_MIN && r >= 1 && r <= TC_RMAX) {
        double tcut = S.tau_lo;
        if (S.test_mode == 0 && S.tol > 0.0) tcut = fmax(tcut, 0.5 * S.tol);
        const int nchunk = (b + TC_M - 1) / TC_M;
        const int nslot = min(T.size(), nchunk);
        const size_t ntri = (size_t)r * (r + 1) / 2;
        const bool want_gram = S.Pp && S.up && (size_t)nslot * ntri <= S.pp_cap &&
                               (size_t)nslot * r <= (size_t)NCH_MAX * S.r_max;
        __shared__ bool gd;
        int q_loc = b;
        bool sums_ok = want_gram, first = true;
        for (int ch = T.id(); ch < nchunk; ch += T.size()) {
          const int c0 = ch * TC_M, nr = min(TC_M, b - c0);
          const int q = tc_project_block(reinterpret_cast<TcCtx*>(S.tcx), S, gam + (size_t)c0 * S.m,
                                         A.y + j0 + c0, nr, r, tcut, A.k - j0 - c0,
                                         reinterpret_cast<float*>(smem_pool()), want_gram, &gd,
                                         TcOut{c0, want_gram ? S.Pp + (size_t)T.id() * ntri : nullptr,
                                               want_gram ? S.up + (size_t)T.id() * r : nullptr, first, false});
          if (q < 0) return false;
          if (q < nr) q_loc = min(q_loc, c0 + q);
          sums_ok = sums_ok && gd;
          first = false;
        }
        if (threadIdx.x == 0 && T.id() < nslot) {  // this CTA's first special row, sums usable
          S.spart[2 * T.id()] = (double)q_loc;
          S.spart[2 * T.id() + 1] = sums_ok ? 1.0 : 0.0;
        }
        if (!T.sync()) return false;
        __shared__ int q_all;
        if (threadIdx.x == 0) q_all = b;
        __syncthreads();
        bool ok_mine = true;
        for (int c = threadIdx.x; c < nslot; c += NT) {
          const int qc = (int)__ldcg(S.spart + 2 * c);
          if (qc < b) atomicMin(&q_all, qc);
          ok_mine = ok_mine && __ldcg(S.spart + 2 * c + 1) != 0.0;
        }
        const bool ok_all = __syncthreads_and(ok_mine ? 1 : 0) != 0;
        q0 = q_all;
        if (want_gram && ok_all && q0 == b) {
          gram_reduce_slots(T, S, r, nslot);
          gram_done = true;
        }
        phase_dall(T, S, A, j0, b, r);
        if (!T.sync()) return false;
      }
    }
    if (q0 == -2) {
      // 1: gamma of every row against the block-start basis
      if (T.id() == 0 && threadIdx.x == 0) S.ctrl[CTRL_Q0] = b;
      // larger items only while they still give every worker at least two
      const bool big_rej = (long long)(b / 32) * S.nmc >= 2LL * T.size();
      const int gr = min(8, (int)((POOL_DOUBLES * 2) / max(S.m, 1)));  // FP32 rows that fit
      // grid teams, small blocks: the basis tile of this CTA's first rejection item comes
      // in by TMA while the projection runs
      // FP64: one-row rejection items (phase_reject_row) when they take fewer FMA
      // instructions per SM sub-partition over the grid's rounds: 48 per round (16 FMAs and
      // the combining adds per thread) against 128 for the 4-row items (FP32 FMAs are cheap:
      // mixed mode keeps the 4-row items)
      bool row_rej = false;
      if (!F32 && kGridTeam && b <= 16 && r > 0) {
        const long long r1 = ((long long)b * S.nmc + T.size() - 1) / T.size();
        const long long r4 = ((long long)((b + 3) / 4) * S.nmc + T.size() - 1) / T.size();
        row_rej = r1 * 48 < r4 * 128;
      }
      const long long rej_items = row_rej ? (long long)b * S.nmc : (long long)((b + 3) / 4) * S.nmc;
      const bool pf_on = kGridTeam && b <= SMALL_B && !big_rej && r > 0 && (long long)T.id() < rej_items;
      if (pf_on) rej_prefetch<F32>(S, (int)(T.id() % S.nmc), min(64, r), &pf_bar);
      RejPrefetch pfv{&pf_bar, &pf_ph};
      if (kGridTeam && b <= SMALL_B)
        phase_gamma_small_any<Team, F32>(T, S, gam, 0, b, r, ORTHO ? S.C : S.Ct);
      else if (F32 && gr >= 1 && (long long)(b / gr) >= 2LL * T.size())
        phase_gamma_f32_staged(T, S, gam, 0, b, r, gr);
      else if (!F32 && (long long)((b + 7) / 8) * r < 4LL * NWARP * T.size())
        phase_gamma_cta(T, S, gam, 0, b, r, ORTHO ? S.C : S.Ct);  // few warp items: split each over a CTA
      else
        phase_gamma<Team, F32>(T, S, gam, 0, b, r, ORTHO ? S.C : S.Ct);
      if (!T.sync()) {
        if (pf_on) mbar_wait(&pf_bar, pf_ph);  // no copy may be in flight at exit
        return false;
      }
      // 2: rejections and norms (grid teams, small blocks: with the decisions fused in);
      // a-priori errors against w_b
      const bool fuse = kGridTeam && b <= SMALL_B && (b + 3) / 4 <= 16;
      FusedDecide fdv{A.y + j0, S.tau_lo};
      if (F32 && S.test_mode == 0 && S.tol > 0.0) fdv.tc = fmax(fdv.tc, 0.5 * S.tol);
      if (big_rej) phase_reject<Team, F32, 8>(T, S, gam, 0, b, r, S.C, nullptr, fuse ? &fdv : nullptr);
      else if (!F32 && row_rej) phase_reject_row<Team, false>(T, S, gam, 0, b, r, S.C, fuse ? &fdv : nullptr,
                                                              pf_on ? &pfv : nullptr);
      else phase_reject<Team, F32, 1>(T, S, gam, 0, b, r, S.C, nullptr, fuse ? &fdv : nullptr,
                                      pf_on ? &pfv : nullptr);
      // CTAs beyond the rejection items take the a-priori errors and the previous call's
      // deferred P/u update
      const long long nrej = row_rej ? (long long)b * S.nmc
                                     : (long long)((b + 4 * (big_rej ? 8 : 1) - 1) / (4 * (big_rej ? 8 : 1))) * S.nmc;
      const int w_lo = (int)min(nrej, (long long)max(0, T.size() - 16));
      phase_dall(T, S, A, j0, b, r, w_lo);
      if (sh[4] > 0) acc_rows<Team, F32>(T, S, S.Gpend, S.Dpend, 0, sh[4], r, w_lo);
      if (!T.sync()) return false;
      // 3: decide
      if (b <= SMALL_B) {
        if (fuse) {
          if (threadIdx.x == 0) sh[3] = __ldcg(S.ctrl + CTRL_Q0);  // decided before the barrier
          __syncthreads();
          q0 = sh[3];
        } else {
          q0 = decide_rows<F32>(S, A, j0, b, r, T.id() == 0);
        }
        if (q0 == b) {  // fast finish: every row dependent
          const bool defer = S.defer && last && j0 == 0;  // the call's only block
          if (!defer) acc_small<Team, F32>(T, S, 0, b, r);
          if (T.id() == 0) {
            if (A.indep)
              for (int j = threadIdx.x; j < b; j += NT) A.indep[j0 + j] = 0;
            if (threadIdx.x == 0) {
              *S.rows_seen = __ldcg(S.rows_seen) + b;
              S.ctrl[CTRL_KB] = min(kb_growth<Team, F32>() * kb0, S.kb_max);
              S.ctrl[CTRL_PEND] = 1;
              S.ctrl[CTRL_PEND_ROWS] = defer ? b : 0;
            }
          }
          if (!last && !T.sync()) return false;
          j0 += b;
          continue;
        }
      } else {
        decide_rows_team<Team, F32>(T, S, A, j0, b, r);
        if (!T.sync()) return false;
        if (threadIdx.x == 0) sh[3] = __ldcg(S.ctrl + CTRL_Q0);
        __syncthreads();
        q0 = sh[3];
      }
    }
    const int applied = block_tail<Team, F32, VAR>(T, S, A, j0, b, r, q0, kb0, gram_done);
    if (applied < 0) return false;
    j0 += applied;
  }
  return true;
}

// =======================================================================================
// On-demand forms: w = w_b + P^-1 u (solution) and P^-1 (export). Dense helpers for one
// CTA (all threads): Cholesky of P in the workspace Lw and solves with it.
// =======================================================================================

// In-place lower Cholesky of A (n x n, row stride lda), 32-wide panels: each diagonal
// block is factored in shared memory by the whole CTA, the panel below by row-wise
// substitution, the trailing matrix updated in 32 x 32 tiles. Returns false if a pivot
// was not positive.
static __device__ bool cta_cholesky(double* A, int n, int lda) {
  double* Dk = smem_pool();
  double(*Pi)[33] = reinterpret_cast<double(*)[33]>(Dk + 32 * 33);
  double(*Pj)[33] = Pi + 32;
  __shared__ double invd[32];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += 32) {
    const int kb = min(32, n - k0);
    for (int e = threadIdx.x; e < kb * kb; e += NT) {
      const int i = e / kb, j = e - i * kb;
      Dk[i * 33 + j] = (j <= i) ? __ldcg(A + (size_t)(k0 + i) * lda + k0 + j) : 0.0;
    }
    __syncthreads();
    for (int kk = 0; kk < kb; ++kk) {
      if (threadIdx.x == 0) {
        const double d = Dk[kk * 33 + kk];
        if (!(d > 0.0) || !isfinite(d)) bad = 1;
        const double y = rsqrt_nr(fmax(d, 1e-300));
        Dk[kk * 33 + kk] = d * y;
        invd[kk] = y;
      }
      __syncthreads();
      const double y = invd[kk];
      for (int i = kk + 1 + threadIdx.x; i < kb; i += NT) Dk[i * 33 + kk] *= y;
      __syncthreads();
      const int rem = kb - kk - 1;
      for (int e = threadIdx.x; e < rem * rem; e += NT) {
        const int i = kk + 1 + e / rem, j = kk + 1 + e % rem;
        if (j <= i) Dk[i * 33 + j] -= Dk[i * 33 + kk] * Dk[j * 33 + kk];
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < kb * kb; e += NT) {
      const int i = e / kb, j = e - i * kb;
      if (j <= i) A[(size_t)(k0 + i) * lda + k0 + j] = Dk[i * 33 + j];
    }
    // panel below: L[i, k0:k0+kb] = A[i, k0:k0+kb] L_kk^-T (one thread per row)
    for (int i = k0 + kb + threadIdx.x; i < n; i += NT) {
      double v[32];
      double* row = A + (size_t)i * lda + k0;
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = (j < kb) ? __ldcg(row + j) : 0.0;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (j < kb) {
          double x = v[j];
          for (int t = 0; t < j; ++t) x -= v[t] * Dk[j * 33 + t];
          v[j] = x * invd[j];
        }
      }
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < kb) row[j] = v[j];
    }
    __syncthreads();
    // trailing update A[i][j] -= sum_t L[i][k0+t] L[j][k0+t], lower triangle, 32x32 tiles
    const int t0 = k0 + kb;
    const int ntile = (n - t0 + 31) / 32;
    for (int tt = 0; tt < ntile * ntile; ++tt) {
      const int bi = tt / ntile, bj = tt - bi * ntile;
      if (bj > bi) continue;
      for (int e = threadIdx.x; e < 32 * 32; e += NT) {
        const int a = e >> 5, t = e & 31;
        const int ri = t0 + bi * 32 + a, rj = t0 + bj * 32 + a;
        Pi[a][t] = (ri < n && t < kb) ? __ldcg(A + (size_t)ri * lda + k0 + t) : 0.0;
        Pj[a][t] = (rj < n && t < kb) ? __ldcg(A + (size_t)rj * lda + k0 + t) : 0.0;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < 32 * 32; e += NT) {
        const int a = e >> 5, b2 = e & 31;
        const int ri = t0 + bi * 32 + a, rj = t0 + bj * 32 + b2;
        if (ri < n && rj < n && rj <= ri) {
          double acc = 0.0;
          for (int t = 0; t < kb; ++t) acc = fma(Pi[a][t], Pj[b2][t], acc);
          double* dst = A + (size_t)ri * lda + rj;
          *dst = __ldcg(dst) - acc;
        }
      }
      __syncthreads();
    }
  }
  __syncthreads();
  return bad == 0;
}

// x <- (L L^T)^-1 x for the factor of cta_cholesky; n <= GRAM_RMAX (x staged in shared
// memory). xin is read with __ldcg, the result goes to xout. Each 32-wide diagonal block
// is staged in shared memory with the reciprocals of its diagonal (one rsqrt_nr of the
// squared pivot each), so the sequential steps multiply instead of divide.
static __device__ void cta_chol_solve(const double* L, int n, int lda, const double* xin,
                                      double* xout) {
  __shared__ double dinv[32];
  double* Db = smem_pool();  // 32 x 33 diagonal block
  double* xs = Db + 32 * 33;  // n <= GRAM_RMAX entries (fits the pool)
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += NT) xs[i] = __ldcg(xin + i);
  const int lane = threadIdx.x & 31;
  for (int pass = 0; pass < 2; ++pass) {  // forward L y = x, then backward L^T z = y
    const int nblk = (n + 31) / 32;
    for (int bi = 0; bi < nblk; ++bi) {
      const int k0 = (pass == 0 ? bi : nblk - 1 - bi) * 32;
      const int kb = min(32, n - k0);
      __syncthreads();
      for (int e = threadIdx.x; e < kb * kb; e += NT) {
        const int i = e / kb, j = e - i * kb;
        Db[i * 33 + j] = (j <= i) ? __ldcg(L + (size_t)(k0 + i) * lda + k0 + j) : 0.0;
      }
      __syncthreads();
      if (threadIdx.x < kb) {
        const double d = Db[threadIdx.x * 33 + threadIdx.x];
        dinv[threadIdx.x] = rsqrt_nr(d * d);
      }
      __syncthreads();
      if (threadIdx.x < 32) {
        double v = (lane < kb) ? xs[k0 + lane] : 0.0;
        if (pass == 0) {
          for (int p = 0; p < kb; ++p) {
            const double vp = __shfl_sync(0xffffffffu, v, p) * dinv[p];
            if (lane == p) v = vp;
            if (lane > p && lane < kb) v -= Db[lane * 33 + p] * vp;
          }
        } else {
          for (int p = kb - 1; p >= 0; --p) {
            const double vp = __shfl_sync(0xffffffffu, v, p) * dinv[p];
            if (lane == p) v = vp;
            if (lane < p) v -= Db[p * 33 + lane] * vp;
          }
        }
        if (lane < kb) xs[k0 + lane] = v;
      }
      __syncthreads();
      if (pass == 0) {
        for (int i = k0 + kb + threadIdx.x; i < n; i += NT) {
          double acc = 0.0;
          const double* row = L + (size_t)i * lda + k0;
          for (int t = 0; t < kb; ++t) acc = fma(__ldcg(row + t), xs[k0 + t], acc);
          xs[i] -= acc;
        }
      } else {
        for (int i = threadIdx.x; i < k0; i += NT) {
          double acc = 0.0;
          for (int t = 0; t < kb; ++t) acc = fma(__ldcg(L + (size_t)(k0 + t) * lda + i), xs[k0 + t], acc);
          xs[i] -= acc;
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += NT) xout[i] = xs[i];
  __syncthreads();
}

// w = w_b + P^-1 u, by one CTA: Lw = chol(P), then the two triangular solves. Ranks above
// GRAM_RMAX are refused with ST_BADARG (no shared-memory staging for them).
static __device__ void form_w(const StreamDev& S, int r) {
  const int rm = S.r_max;
  if (r == 0) return;
  if (r > GRAM_RMAX) {
    if (threadIdx.x == 0) atomicOr(S.ctrl + CTRL_STATUS, ST_BADARG);
    return;
  }
  for (long long e = threadIdx.x; e < (long long)r * r; e += NT) {
    const int i = (int)(e / r), l = (int)(e - (long long)i * r);
    S.Lw[(size_t)i * rm + l] = __ldcg(S.P + (size_t)i * rm + l);
  }
  __syncthreads();
  if (!cta_cholesky(S.Lw, r, rm) && threadIdx.x == 0) atomicOr(S.ctrl + CTRL_STATUS, ST_NONFINITE);
  cta_chol_solve(S.Lw, r, rm, S.u, S.w);
  for (int i = threadIdx.x; i < r; i += NT) S.w[i] = __ldcg(S.w + i) + __ldcg(S.wb + i);
  __syncthreads();
}

// P^-1 from the factor in Lw (after form_w), team-wide: worker c solves for columns
// c, c + size, ... (column l of P^-1 = (L L^T)^-1 e_l, stored as row l: P^-1 is symmetric).
template <class Team>
__device__ void form_pinv(const Team& T, const StreamDev& S, int r) {
  const int rm = S.r_max;
  if (r == 0 || r > GRAM_RMAX) return;
  for (int l = T.id(); l < r; l += T.size()) {
    double* out = S.Pinv + (size_t)l * rm;
    for (int i = threadIdx.x; i < r; i += NT) out[i] = (i == l) ? 1.0 : 0.0;
    __syncthreads();
    cta_chol_solve(S.Lw, r, rm, out, out);
  }
}

}  // namespace rg
