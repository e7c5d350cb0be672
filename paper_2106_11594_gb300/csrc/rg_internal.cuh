// rg_internal.cuh -- device-side state layout and helpers shared by the CUDA kernels of
// librg.so. Not part of the public ABI (include/rg.h is).
#pragma once

#include <cfloat>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rg {

constexpr int NT = 256;          // threads per CTA in every kernel
constexpr int NWARP = NT / 32;   // warps per CTA
constexpr int SMALL_B = 64;      // blocks up to this many rows take the two-barrier path
constexpr int SLOW_MAX = 32;     // rows per sequential rank-change section
constexpr int KB_MIN = 64;       // internal block size right after a rank change
constexpr int JW = 4;            // observation rows per warp tile in the gamma phase
constexpr int RJ = 4;            // observation rows per CTA item in the rejection phase
constexpr int MC = NT / RJ;      // columns per CTA item in the rejection phase (64)
constexpr int NCH_MAX = 64;      // row chunks of the Gram path
constexpr int GRAM_CHUNK = 128;  // rows per Gram-path chunk (at least)
constexpr int GRAM_RMAX = 2048;  // the Gram path is used for ranks up to this
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;  // bounded waits: 2 s

// Rank factorizations kept (template parameter VAR of the update): Algorithm 1's general
// variant (C = selected rows, Ct its dual basis) and the two variants of Section 2.2 --
// orthonormal (alpha = 1/||Gamma_r||: C = Q, its own dual) and orthogonal (alpha = 1:
// C holds the raw rejections, Ct the same rows over their squared norms).
enum : int { VAR_GENERAL = 0, VAR_ORTHONORMAL = 1, VAR_ORTHOGONAL = 2 };

// Device status bits (mapped to rg_status on the host).
enum : int { ST_NONFINITE = 1, ST_CAPACITY = 2, ST_TIMEOUT = 4, ST_BADARG = 8 };

// Control words of one stream (device memory).
enum : int {
  CTRL_R = 0,          // current rank r
  CTRL_STATUS = 1,     // sticky error bits
  CTRL_BAR_COUNT = 2,  // grid barrier arrival counter (64 bits: words 2 and 3)
  CTRL_KB = 4,         // adaptive internal block size
  CTRL_Q0 = 5,         // block plan: first row that needs the sequential section
  CTRL_APPLIED = 7,    // block plan: rows of the block that were applied
  CTRL_RNEW = 8,       // block plan: rank after the block
  CTRL_NIND = 9,       // block plan: independent rows found in the block
  CTRL_PEND = 10,      // 1: u holds a correction not yet folded into w
  CTRL_PEND_ROWS = 11, // rows of the previous call whose P/u update was deferred (in Gpend)
  CTRL_SUB_COUNT = 32, // barrier counter of the sequential section's column owners (words
                       // 32-33, a cache line apart from the grid barrier's counter)
  CTRL_GRP = 40,       // 16 words: per-row-group item counters of the decision fused into
                       // the rejection phase of small blocks (idle between blocks: zero)
  CTRL_N = 64
};

// Everything a kernel needs to know about one stream. Plain pointers into device
// memory owned by the host-side rg_state. Two algebraic variants:
//  * general (FP64 mode by default): C = selected observation rows, Ct = dual basis
//    (Ct C^T = I), Algorithm 1 of the paper;
//  * orthonormal (mixed mode, or FP64 mode on request): C = Q with orthonormal rows
//    spanning the same space (Section 2.2, alpha = 1/||Gamma_r||), so the dual basis is
//    Q itself; in mixed mode an FP32 copy Qf feeds the FP32 projections.
struct StreamDev {
  int m, ld, r_max, kb_max;
  int mixed;      // 1: FP32 projections (implies the orthonormal variant)
  int ortho;      // 1: orthonormal variant (Ct is C itself)
  int orthog;     // 1: orthogonal variant (C and Ct both kept, as in the general variant)
  int test_mode;  // 0 REL, 2 PAPER
  int bar_off = CTRL_BAR_COUNT;  // control words of the grid barrier and of the section's
  int sub_off = CTRL_SUB_COUNT;  // barrier used by this launch (each counter stays a multiple
                                 // of its team size between launches)
  double tol;     // <= 0: paper default (m^2 r + m r + m) eps_M
  double tau_lo;  // mixed mode: FP32 relative-rejection floor below which rows are dependent
  double* C;      // r_max x ld
  double* Ct;     // r_max x ld (general variant only)
  float* Qf;      // r_max x ld (mixed only)
  double* Pinv;   // r_max x r_max: P^-1, formed on demand (export)
  double* P;      // r_max x r_max: Gram matrix B^T B (information form of P^-1)
  double* wb;     // r_max: base coordinates w_b
  double* u;      // r_max: accumulated correction, w = w_b + P^-1 u
  double* w;      // r_max: w, formed on demand (solution, export); X = Ct^T w
  long long* basis_rows;  // r_max
  long long* rows_seen;   // [1]
  int* ctrl;              // CTRL_N ints
  // scratch of one internal block
  double* G;      // kb_max x r_max: gamma of each row of the block (row-major by row)
  double* spart;  // kb_max x nmc: partial ||Gamma_r||^2 per column chunk
  double* tpart;  // kb_max x nmc: partial ||Gamma||^2 per column chunk
  int nmc;        // column chunks = ceil(m / MC)
  double* s;      // kb_max
  double* t;      // kb_max
  uint8_t* rowflag;   // kb_max: 1 = dependent, 2 = independent (per row of the block)
  double* R;      // SLOW_MAX x ld: FP64 rejections of the sequential section
  double* Kv;     // SLOW_MAX x ld: new dual rows K (general) or new Q rows (orthonormal)
  double* Gind;   // SLOW_MAX x r_max: gamma (fixed up) of each independent row
  double* alpha;  // SLOW_MAX: 1/||Gamma_r|| of each independent row of the section
  int* jind;      // SLOW_MAX: block row of each independent row
  double* Dall;   // kb_max: a-priori errors y_j - gamma_j^T w_b of the block's rows
  double* Pp;     // pp_cap doubles: Gram partials, chunk c at Pp + c * r * r
  size_t pp_cap;
  double* up;     // NCH_MAX x r_max: partial sums of gamma_j D_j per chunk
  double* Lw;     // r_max x r_max: Cholesky workspace (solution, export)
  double* Sp;     // 2 x sp_stride: per-worker partial sums of the sequential section
  size_t sp_stride;  // >= 32 x (number of workers)
  void* tcx;      // tensor-core context of the CTA (struct TcCtx in shared memory) or null
  // Deferred P/u update of small calls: a call of at most SMALL_B rows that ends with all
  // rows dependent leaves its gammas (G) and a-priori errors (Dall) in place and records
  // their count in CTRL_PEND_ROWS; the next call (whose G/Dall are the host's other pair
  // of buffers, and whose Gpend/Dpend point here) folds them into P and u on CTAs that the
  // rejection phase leaves idle, and rg_solution/rg_export fold them first.
  double* Gpend;  // gammas of the pending rows (SMALL_B x r_max) or null (no deferral)
  double* Dpend;  // their a-priori errors
  int defer;      // 1: this call may defer (its G/Dall are a pending-capable pair)
  double* Kap;    // SLOW_MAX x SLOW_MAX: kappa of the section's later rows per append
  double* Rs;     // shared memory for the section's rejections (one-CTA team) or null
  long long rs_cap;  // doubles available at Rs
};

// FP64 -> FP32 by integer operations, rounding toward zero (FP64<->FP32 conversion
// instructions issue on the FP64 pipe, 1/64 of the FP32 rate on this part). Magnitudes
// below the FP32 normal range give a signed zero, above it a signed infinity; NaN stays
// NaN.
__device__ __forceinline__ float d2f_rz(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ex = hi & 0x7FF00000u, sign = hi & 0x80000000u;
  unsigned f = sign | ((((hi & 0x7FFFFFFFu) - (896u << 20)) << 3) | (lo >> 29));
  if (ex < (897u << 20)) f = sign;
  if (ex >= (1151u << 20)) f = sign | 0x7F800000u | ((ex == 0x7FF00000u && ((hi & 0xFFFFFu) | lo)) ? 0x400000u : 0u);
  return __uint_as_float(f);
}

// FP32 -> FP64 (exact) by integer operations for normal numbers, zero, infinity and NaN;
// FP32 subnormals take the conversion instruction.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xFFu, sign = u & 0x80000000u, man = u & 0x7FFFFFu;
  if (ex == 0u) return man ? (double)f : __hiloint2double((int)sign, 0);
  const unsigned hex = (ex == 0xFFu) ? 0x7FF00000u : ((ex + 896u) << 20);
  return __hiloint2double((int)(sign | hex | (man >> 3)), (int)(man << 29));
}

// Compensated FP32 accumulation for mixed mode's Gram sums: blocked summation (FABsum;
// Blanchard, Higham and Mary, "A class of fast and accurate summation algorithms", SIAM J.
// Sci. Comput. 42, 2020). The products of FAB_B consecutive rows are summed in FP32 by
// plain FMAs, and each block sum is added to a pair (s, c) by Knuth's TwoSum, so the error
// bound is about FAB_B units of FP32 rounding whatever the length of the run (plain FP32
// accumulation grows with it), for ~1.75 FP32 operations per product. The _rn intrinsics
// keep the compiler from fusing or reordering the TwoSum steps. The pair is added to the
// FP64 state as s + c.
constexpr int FAB_B = 8;
struct CompSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = __fadd_rn(s, x);
    const float z = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z)));
    s = t;
  }
  __device__ __forceinline__ double value() const { return f2d_exact(s) + f2d_exact(c); }
};

// An FP64 a-priori error D as two FP32 words (D ~ hi + lo to ~48 bits; hi truncated, the
// remainder D - hi is exact in FP64), so that gamma D enters the FP32 sums as two products.
__device__ __forceinline__ void split_d(double d, float& hi, float& lo) {
  hi = d2f_rz(d);
  lo = d2f_rz(d - f2d_exact(hi));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_i32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident), on a monotonic 64-bit
// arrival counter (control words CTRL_BAR_COUNT..+1) that is a multiple of gridDim.x
// between barriers: each CTA adds 1 with an atomic that returns the old value, which
// fixes the barrier's target ((old / gridDim.x + 1) gridDim.x: no CTA can arrive at the
// next barrier before this one completes), and waits with acquire loads until the counter
// reaches it. No per-launch initialisation is needed.
// The wait is bounded: after WAIT_LIMIT_NS the CTA records ST_TIMEOUT and returns false.
__device__ __forceinline__ void grid_barrier_init(int* /*ctrl*/) {}
__device__ __forceinline__ unsigned long long atom_release_add_u64(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.release.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}
__device__ __forceinline__ bool grid_barrier(int* ctrl, int bar_off = CTRL_BAR_COUNT) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(ctrl + bar_off);
    const unsigned long long old = atom_release_add_u64(cnt, 1ull);
    const unsigned long long target = (old / gridDim.x + 1) * gridDim.x;
    if (ld_acquire_u64(cnt) < target) {
      const unsigned long long t0 = global_ns();
      while (ld_acquire_u64(cnt) < target) {
        const unsigned long long dt = global_ns() - t0;
        if (dt > WAIT_LIMIT_NS) {
          atomicOr(ctrl + CTRL_STATUS, ST_TIMEOUT);
          ok = 0;
          break;
        }
        if (dt > 4000) __nanosleep(256);  // long waits (a few CTAs busy) poll gently
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

// Rank test of Eq. label_eq_eps in squared form. s = ||Gamma_r||^2, t = ||Gamma||^2.
__device__ __forceinline__ bool is_independent(double s, double t, int r, int m, double tol,
                                               int test_mode) {
  double eps = tol;
  if (!(eps > 0.0)) {
    const double md = (double)m, rd = (double)r;
    eps = (md * md * rd + md * rd + md) * DBL_EPSILON;
  }
  const double e2 = eps * eps;
  if (test_mode == 2) return !(s < e2 || s < e2 * t);
  return s > e2 * t;
}

}  // namespace rg
