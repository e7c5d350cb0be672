// rg_tc.cuh -- the block projection of mixed mode on the fifth-generation tensor cores
// (tcgen05.mma, kind::tf32, FP32 accumulators in tensor memory).
//
// For a chunk of up to 128 rows of a block (Section 3's block of observations, all
// projected against the block-start basis Q, which dependent rows leave unchanged by
// Theorem 6) one CTA computes
//   G = Gamma_c Q^T          (128 x r: the coordinates gamma_j of the rows, Section 2.2)
//   R = Gamma_c - G Q        (128 x m: the rejections, Eq. label_eq_schur_complement)
// and from R the squared norms s_j = ||Gamma_r,j||^2 and t_j = ||Gamma_j||^2 of the FP32
// screen of mixed mode. Both products are dense contractions (K = m, then K = r) and run as
// 3xTF32: every FP32 operand x is split into hi = x rounded to TF32 and lo = x - hi, and
// A B = Ahi Bhi + Ahi Blo + Alo Bhi, which keeps the product error near FP32 rounding
// (one TF32 product alone would leave a rejection noise of ~1e-3 |Gamma|, far above the
// screen's floor tau_lo).
//
// Operands are staged by all threads into shared memory in the no-swizzle K-major
// core-matrix layout (core matrix = 8 rows x 16 bytes, 128 contiguous bytes; the next
// core matrix along K at +128 B, the next 8-row group at +1024 B for a 32-wide K slice);
// one thread issues the MMAs and commits them to an mbarrier; the accumulators are read
// back with tcgen05.ld (32x32b shape: thread = row). Waits on the mbarrier are bounded.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rg_internal.cuh"

namespace rg {

constexpr int TC_M = 128;      // rows per chunk (MMA M)
constexpr int TC_K = 32;       // K slice: 32 TF32 elements = 128 bytes per row
constexpr int TC_N2 = 64;      // columns of m per second-product slice (MMA N)
constexpr int TC_RMAX = 128;   // ranks handled (first-product N = r rounded up to 16)
constexpr int TC_TILE = TC_M * TC_K;            // floats per operand tile (16 KiB)
constexpr int TC_SMEM = 4 * TC_TILE * 4 + 1024;  // Ahi, Alo, Bhi, Blo + alignment slack
// mixed-mode batch kernels (one CTA per SM) take more: Ahi, Alo, then either Bhi, Blo or a
// cache of every B tile of the instance's current basis (both products), kept while the
// basis does not change
constexpr int TC_SMEM_MIXED = 180 * 1024;
constexpr int TC_TMEM_COLS = 512;  // D1: columns [0, 128); D2 slices: 64 columns each from 128
constexpr int TC_NG2 = 6;          // second-product column slices issued together (6 x 64 = 384)

// Per-CTA tensor-core context (shared memory, written once by the kernel prologue except
// `phase`, which thread 0 stores back at the end of every projection).
struct TcCtx {
  float* Ahi;
  float* Alo;
  float* Bhi;  // per-slice B tiles (uncached mode); the cache starts here too
  float* Blo;
  unsigned long long* bar;  // mbarrier: one arrival per commit
  uint32_t tmem;            // tensor-memory base (lane 0, column 0)
  uint32_t phase;           // parity of the next completion of `bar`
  int cache_cap;            // floats available for the B-tile cache at Bhi (0: none)
  const float* cq;          // basis whose tiles are cached (with rank cr), or null
  int cr;
  int ng2;                  // second-product column slices issued per commit (1..TC_NG2)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Blocks of at least this many rows of a single mixed-mode stream take the tensor-core
// chunk path on the whole GPU (every SM gets a 128-row chunk from 152 x 128 / 2 rows on).
constexpr int TC_GRID_MIN = 8192;

// Offset (floats) of element (row, k) in a tile with a 32-wide K slice.
__host__ __device__ __forceinline__ int tc_off(int row, int k) {
  return (row >> 3) * 256 + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

// Shared-memory matrix descriptor: start address, leading byte offset 128 (K direction),
// stride byte offset 1024 (8-row groups), fixed version bits, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: D FP32, A and B TF32, both K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Every thread waits for the completion of parity `ph` of the mbarrier (bounded); the CTA
// agrees on the outcome. On success the parity advances; false if the wait gave up.
__device__ __forceinline__ bool tc_wait(unsigned long long* bar, uint32_t& ph) {
  bool done = mbar_try_wait(bar, ph);
  if (!done) {
    const unsigned long long t0 = global_ns();
    while (!(done = mbar_try_wait(bar, ph)))
      if (global_ns() - t0 > WAIT_LIMIT_NS) break;
  }
  if (!__syncthreads_and(done ? 1 : 0)) return false;
  ph ^= 1u;
  tc_fence_after();
  return true;
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// hi = x rounded to TF32 (10 explicit mantissa bits), lo = x - hi (exact in FP32).
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
  lo = x - hi;
}

// One 32-wide K slice of D (+)= A B^T as 3xTF32 (four K steps of 8), issued by one thread.
__device__ __forceinline__ void tc_slice_mma_at(const float* Ahi, const float* Alo, const float* Bhi,
                                                const float* Blo, uint32_t d, int N, bool first) {
  const uint32_t id = tc_idesc(TC_M, N);
  const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const uint32_t o = (uint32_t)s * 256u;  // 8 TF32 = two core matrices along K
    tc_mma(d, tc_desc(ah + o), tc_desc(bh + o), id, (first && s == 0) ? 0u : 1u);
    tc_mma(d, tc_desc(ah + o), tc_desc(bl + o), id, 1u);
    tc_mma(d, tc_desc(al + o), tc_desc(bh + o), id, 1u);
  }
}
__device__ __forceinline__ void tc_slice_mma(const TcCtx& X, uint32_t d, int N, bool first) {
  tc_slice_mma_at(X.Ahi, X.Alo, X.Bhi, X.Blo, d, N, first);
}

// A = rows [0, 128) x columns [k0, k0 + 32) of an FP64 row-major matrix (valid rows <
// nrows, valid columns < m; the rest zero), in two steps so that the loads of the next
// slice can be in flight while the tensor cores work on the current one: tc_load_a puts
// this thread's 16 elements in registers (FP32), tc_store_a splits and stores them. Warp w
// takes the 4 columns [4w, 4w + 4) of all 16 row groups; a warp access covers 8 rows x 4
// columns, so its 32 lanes hit 32 distinct banks.
// The 16 loads are all issued before any value is used (raw FP64 kept in registers), so
// they are in flight together; the conversion happens in tc_store_a.
__device__ __forceinline__ void tc_load_a(double (&v)[16], const double* __restrict__ src, int m, int nrows,
                                          int k0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rl = lane >> 2, c = k0 + warp * 4 + (lane & 3);
  const bool cok = c < m;
  const double* p = src + (size_t)rl * m + c;
#pragma unroll
  for (int rg = 0; rg < 16; ++rg)
    v[rg] = (cok && rg * 8 + rl < nrows) ? __ldg(p + (size_t)rg * 8 * m) : 0.0;
}
__device__ __forceinline__ void tc_store_a(const TcCtx& X, const double (&v)[16]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int o0 = warp * 32 + (lane >> 2) * 4 + (lane & 3);
#pragma unroll
  for (int rg = 0; rg < 16; ++rg) {
    float h, l;
    tf32_split(d2f_rz(v[rg]), h, l);
    X.Ahi[o0 + rg * 256] = h;
    X.Alo[o0 + rg * 256] = l;
  }
}

// Stages B = rows [0, nrow) (multiple of 8) x columns [k0, k0 + 32) of the FP32 basis Qf
// (rows >= r and columns >= m zero).
__device__ __forceinline__ void tc_stage_q_to(float* Bhi, float* Blo, const float* __restrict__ Qf, int ld,
                                              int m, int r, int nrow, int k0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rl = lane >> 2, kl = lane & 3;
  // warp w takes column group kg = w of the row groups rg < nrow / 8 (at most 16); all
  // loads are issued before the stores
  const int c = k0 + warp * 4 + kl;
  const int ngr = nrow >> 3;
  float x[16];
#pragma unroll
  for (int rg = 0; rg < 16; ++rg) {
    const int row = rg * 8 + rl;
    x[rg] = (rg < ngr && row < r && c < m) ? __ldcg(Qf + (size_t)row * ld + c) : 0.f;
  }
  const int o0 = warp * 32 + rl * 4 + kl;
#pragma unroll
  for (int rg = 0; rg < 16; ++rg) {
    if (rg < ngr) {
      float h, l;
      tf32_split(x[rg], h, l);
      Bhi[o0 + rg * 256] = h;
      Blo[o0 + rg * 256] = l;
    }
  }
}
__device__ __forceinline__ void tc_stage_q(const TcCtx& X, const float* __restrict__ Qf, int ld, int m,
                                           int r, int nrow, int k0) {
  tc_stage_q_to(X.Bhi, X.Blo, Qf, ld, m, r, nrow, k0);
}

// Stages B = Q^T slice for the second product: row n < 64 is column c0 + n of Q, K index
// k is basis row k1 + k (zero beyond r or m). Threads [t_lo, t_lo + 128) take part.
__device__ __forceinline__ void tc_stage_qt_to(float* Bhi, float* Blo, const float* __restrict__ Qf, int ld,
                                               int m, int r, int c0, int k1, int t_lo) {
  const int t = threadIdx.x - t_lo;
  const int lane = t & 31, warp = t >> 5;  // 4 warps
  const int rl = lane >> 2, kl = lane & 3;
  float x[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int it = warp + 4 * q;
    const int rg = it >> 3, kg = it & 7;
    const int n = rg * 8 + rl, i = k1 + kg * 4 + kl, c = c0 + n;
    x[q] = (i < r && c < m) ? __ldcg(Qf + (size_t)i * ld + c) : 0.f;
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int it = warp + 4 * q;
    const int rg = it >> 3, kg = it & 7;
    float h, l;
    tf32_split(x[q], h, l);
    const int o = rg * 256 + kg * 32 + rl * 4 + kl;
    Bhi[o] = h;
    Blo[o] = l;
  }
}
__device__ __forceinline__ void tc_stage_qt(const TcCtx& X, const float* __restrict__ Qf, int ld, int m,
                                            int r, int c0, int k1, int t_lo) {
  tc_stage_qt_to(X.Bhi, X.Blo, Qf, ld, m, r, c0, k1, t_lo);
}

__device__ __forceinline__ uint32_t dyn_smem_bytes() {
  uint32_t x;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(x));
  return x;
}

// The CTA's tensor-core context over `smem_bytes` of dynamic shared memory at dyn_base
// (1024-byte aligned): warp 0 allocates TC_TMEM_COLS columns of tensor memory (one CTA per
// SM, so they are always free), thread 0 initialises the mbarrier and lays out the operand
// tiles Ahi, Alo, Bhi, Blo, the rest after Bhi being the B-tile cache. Every thread calls
// it; tc_ctx_release frees the tensor memory before the CTA exits.
__device__ __forceinline__ void tc_ctx_init(TcCtx* tcx, unsigned long long* bar, uint32_t* tmem_slot,
                                            float* dyn_base, int smem_bytes, int ng2 = TC_NG2) {
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    tcx->Ahi = dyn_base;
    tcx->Alo = dyn_base + TC_TILE;
    tcx->Bhi = dyn_base + 2 * TC_TILE;
    tcx->Blo = dyn_base + 3 * TC_TILE;
    tcx->bar = bar;
    tcx->phase = 0;
    tcx->cache_cap = (smem_bytes - 1024) / 4 - 2 * TC_TILE;
    tcx->cq = nullptr;
    tcx->cr = -1;
    tcx->ng2 = min(max(ng2, 1), TC_NG2);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x == 0) tcx->tmem = *tmem_slot;
  __syncthreads();
}
__device__ __forceinline__ void tc_ctx_release(const TcCtx* tcx) {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tcx->tmem), "r"(TC_TMEM_COLS));
}

// Asks the TMA unit to pull the bytes [p, p + bytes) of global memory into L2 ahead of their
// use (cp.async.bulk.prefetch: nothing is written to shared memory and nothing waits on it).
// The range is shrunk inward to 16-byte boundaries, so no byte outside it is touched; it is
// issued in pieces of at most 32 KiB.
__device__ __forceinline__ void l2_prefetch(const void* p, size_t bytes) {
  uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
  const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
  for (; a + 16 <= e; a += 32768) {
    const uint32_t n = (uint32_t)((e - a) < 32768 ? (e - a) : 32768);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(n) : "memory");
  }
}

// A wait gave up: wait once more (bounded) for the MMAs in flight, so that the caller can
// release its shared and tensor memory, record ST_TIMEOUT and report failure.
__device__ __forceinline__ int tc_timeout(const StreamDev& S, TcCtx* Xp, uint32_t ph) {
  if (tc_wait(Xp->bar, ph) && threadIdx.x == 0) Xp->phase = ph;
  if (threadIdx.x == 0) atomicOr(S.ctrl + CTRL_STATUS, ST_TIMEOUT);
  __syncthreads();
  return -1;
}

// Block rows [0, b) against the basis (rank 1 <= r <= TC_RMAX), mixed mode, one CTA (navail:
// rows available from gam on, for the L2 prefetch of the rows that come next):
// writes S.G (FP64 copies of the FP32 gammas), S.s and S.t, and returns the first row
// that the FP32 screen cannot declare dependent (b if none), or -1 if a bounded wait gave
// up (ST_TIMEOUT is then set in the status word; MMAs may still be in flight). The rows
// are Gamma[j * m ...] of `gam`, their targets y[j].
// Dependent-run sums of one chunk, fused into the projection (gsm != null): the chunk's
// FP32 gammas are in gsm (row j at gsm + j (r + 1)), its targets as FP32 hi/lo
// pairs after them; each thread sums entries of the upper triangle of sum_j gamma_j
// gamma_j^T and of sum_j gamma_j y_j (in the variants of Section 2.2 the a-priori error is
// y_j, since w_b = 0) over the chunk's rows with FABsum, and adds them to FP64 staging sums:
// pp (the triangle, packed by rows) and upp (first: the staging's first chunk).
constexpr int TC_GRAM_RMAX = 64;  // staging in the shared pool up to this rank (above it: see
                                  // tc_project_block)
__device__ __forceinline__ void tc_chunk_gram(double* __restrict__ pp, double* __restrict__ upp, const float* gsm,
                                              int nrows, int r, bool first) {
  const int ldg = r + 1;
  const float* dh = gsm + TC_M * ldg;
  const float* dl = dh + TC_M;
  const int ntri = r * (r + 1) / 2;
  for (int e = threadIdx.x; e < ntri + r; e += NT) {
    int i, l;
    if (e < ntri) {  // (i, l), i <= l, rows of the triangle one after another
      int rem = e;
      i = 0;
      while (rem >= r - i) {
        rem -= r - i;
        ++i;
      }
      l = i + rem;
    } else {
      i = e - ntri;
      l = -1;
    }
    // FP32 blocks of FAB_B rows in two FMA chains, unrolled so that the block's shared-memory
    // loads issue together; block sums compensated
    CompSum cs;
    const float* ga = gsm + i;
    const float* gb = gsm + (l >= 0 ? l : 0);
    int j1 = 0;
    for (; j1 + FAB_B <= nrows; j1 += FAB_B) {
      float x0 = 0.f, x1 = 0.f;
      if (l >= 0) {
#pragma unroll
        for (int j = j1; j < j1 + FAB_B; j += 2) {
          x0 = fmaf(ga[j * ldg], gb[j * ldg], x0);
          x1 = fmaf(ga[(j + 1) * ldg], gb[(j + 1) * ldg], x1);
        }
      } else {
#pragma unroll
        for (int j = j1; j < j1 + FAB_B; j += 2) {
          x0 = fmaf(ga[j * ldg], dh[j], fmaf(ga[j * ldg], dl[j], x0));
          x1 = fmaf(ga[(j + 1) * ldg], dh[j + 1], fmaf(ga[(j + 1) * ldg], dl[j + 1], x1));
        }
      }
      cs.add(x0 + x1);
    }
    if (j1 < nrows) {  // the last, partial block
      float x = 0.f;
      for (int j = j1; j < nrows; ++j)
        x = (l >= 0) ? fmaf(ga[j * ldg], gb[j * ldg], x) : fmaf(ga[j * ldg], dh[j], fmaf(ga[j * ldg], dl[j], x));
      cs.add(x);
    }
    double* dst = (e < ntri) ? pp + e : upp + i;
    *dst = (first ? 0.0 : *dst) + cs.value();
  }
}

// Where tc_project_block's rows land and where its fused dependent-run sums go. A one-CTA
// team projects a whole block (jb = 0) and commits the sums to P and u itself when every
// row is dependent; a CTA of a grid team projects chunks of a block (jb = the chunk's
// first row), sums into its own staging slot across its chunks (first: its first chunk)
// and leaves the reduction over the slots to the team.
struct TcOut {
  int jb;        // block row of the first row: G, s and t are written at jb + j
  double* pp;    // staging triangle (null: no fused sums)
  double* upp;   // staging sums of gamma_j y_j
  bool first;    // the staging starts with this call
  bool commit;   // add the staging to P and u when every row is dependent
};

static __device__ int tc_project_block(TcCtx* Xp, const StreamDev& S, const double* __restrict__ gam,
                                const double* __restrict__ y, int b, int r, double tc, long long navail,
                                float* pool, bool want_gram, bool* gram_done, const TcOut& O) {
  __shared__ int q0_s;
  const TcCtx X = *Xp;
  uint32_t ph = X.phase;
  __shared__ float red_s[TC_M], red_t[TC_M];
  const int m = S.m, ld = S.ld, rm = S.r_max;
  const int n1 = (r + 15) & ~15;             // first-product N (16..128)
  const int nks = (m + TC_K - 1) / TC_K;     // K slices of the first product
  const int nns = (m + TC_N2 - 1) / TC_N2;   // N slices of the second product
  const int nk2 = (r + TC_K - 1) / TC_K;     // K slices of the second product
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, half = warp >> 2;
  const uint32_t d1 = X.tmem, d2 = X.tmem + 128u;
  const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
  if (threadIdx.x == 0) q0_s = b;
  // B-tile cache: tile (hi, lo) of first-product slice ks at cache + ks * 2 * n1 * 32,
  // second-product tile (ns, k2) after them at + (ns * nk2 + k2) * 2 * 64 * 32
  const int b1 = n1 * TC_K, b2 = TC_N2 * TC_K;  // floats per hi (or lo) tile
  const bool cached = (long long)nks * 2 * b1 + (long long)nns * nk2 * 2 * b2 <= X.cache_cap;
  float* const cache1 = X.Bhi;
  float* const cache2 = X.Bhi + (size_t)nks * 2 * b1;
  if (cached && !(X.cq == S.Qf && X.cr == r)) {
    for (int ks = 0; ks < nks; ++ks)
      tc_stage_q_to(cache1 + (size_t)ks * 2 * b1, cache1 + (size_t)ks * 2 * b1 + b1, S.Qf, ld, m, r, n1, ks * TC_K);
    const int h = threadIdx.x >= 128 ? 1 : 0;  // the two halves take alternate tiles
    for (int tix = h; tix < nns * nk2; tix += 2) {
      const int ns = tix / nk2, k2 = tix - ns * nk2;
      float* t = cache2 + (size_t)tix * 2 * b2;
      tc_stage_qt_to(t, t + b2, S.Qf, ld, m, r, ns * TC_N2, k2 * TC_K, 128 * h);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      Xp->cq = S.Qf;
      Xp->cr = r;
    }
  }
  // staging of the fused dependent-run sums (tc_chunk_gram): the chunk's FP32 gammas and
  // targets go to the shared pool up to rank TC_GRAM_RMAX; above it, to the dynamic shared
  // memory after the per-slice B tiles, which is free whenever the B-tile cache is not in use
  // (always the case above rank 64, where the cache no longer fits)
  float* gsm = nullptr;
  if (want_gram && O.pp) {
    if (r <= TC_GRAM_RMAX) gsm = pool;
    else if (!cached && TC_M * (r + 1) + 2 * TC_M <= X.cache_cap - 2 * TC_TILE) gsm = X.Bhi + 2 * TC_TILE;
  }
  if (threadIdx.x == 0) l2_prefetch(gam, (size_t)min(TC_M, b) * m * 8);
  for (int row0 = 0; row0 < b; row0 += TC_M) {
    const int nrows = min(TC_M, b - row0);
    const double* src = gam + (size_t)row0 * m;
    // the next chunk's rows (of this block, or the first of the next block) into L2 while
    // this chunk is projected
    if (threadIdx.x == 0 && row0 + TC_M < navail)
      l2_prefetch(src + (size_t)TC_M * m, (size_t)min((long long)TC_M, navail - row0 - TC_M) * m * 8);
    // ---- first product: G = Gamma_c Q^T over K slices of m; the next slice's rows are
    // loaded while the tensor cores work on the current one
    double av[16];
    tc_load_a(av, src, m, nrows, 0);
    for (int ks = 0; ks < nks; ++ks) {
      tc_store_a(X, av);
      if (!cached) tc_stage_q(X, S.Qf, ld, m, r, n1, ks * TC_K);
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (threadIdx.x == 0) {
        tc_fence_after();
        if (cached) {
          const float* t = cache1 + (size_t)ks * 2 * b1;
          tc_slice_mma_at(X.Ahi, X.Alo, t, t + b1, d1, n1, ks == 0);
        } else {
          tc_slice_mma(X, d1, n1, ks == 0);
        }
        tc_commit(X.bar);
      }
      if (ks + 1 < nks) tc_load_a(av, src, m, nrows, (ks + 1) * TC_K);
      if (!tc_wait(X.bar, ph)) return tc_timeout(S, Xp, ph);
    }
    // ---- G to global (FP64), threads of warps 0-3 own rows; with the fused dependent-run
    // sums also the FP32 gammas and the targets to shared memory
    const int row = quarter * 32 + lane;
    if (half == 0) {
      for (int i0 = 0; i0 < n1; i0 += 32) {
        float g[32];
        tmem_ld32(d1 + lane_base + (uint32_t)i0, g);
        if (row < nrows) {
          double* gout = S.G + (size_t)(O.jb + row0 + row) * rm;
#pragma unroll
          for (int q = 0; q < 32; ++q)
            if (i0 + q < r) gout[i0 + q] = f2d_exact(g[q]);
          if (gsm) {
#pragma unroll
            for (int q = 0; q < 32; ++q)
              if (i0 + q < r) gsm[row * (r + 1) + i0 + q] = g[q];
          }
        }
      }
      if (gsm && row < nrows) {
        float h, l;
        split_d(__ldg(y + row0 + row), h, l);
        gsm[TC_M * (r + 1) + row] = h;
        gsm[TC_M * (r + 1) + TC_M + row] = l;
      }
    }
    if (gsm) {
      __syncthreads();
      tc_chunk_gram(O.pp, O.upp, gsm, nrows, r, O.first && row0 == 0);
    }
    // ---- second product per 64-column slice: GQ, then R = Gamma - GQ and the norms
    float s_acc = 0.f, t_acc = 0.f;
    auto epilogue = [&](int ns, uint32_t dcol) {
      // warp w reads lanes of its quarter, columns [32 half, 32 half + 32) of the slice
      const int c0 = ns * TC_N2;
      float gq[32];
      tmem_ld32(X.tmem + lane_base + dcol + (uint32_t)(half * 32), gq);
      if (row < nrows) {
        const double* xr = src + (size_t)row * m;
        const int cb = c0 + half * 32;
#pragma unroll
        for (int h2 = 0; h2 < 32; h2 += 16) {
          double xv[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) xv[q] = (cb + h2 + q < m) ? __ldg(xr + cb + h2 + q) : 0.0;
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const float xf = d2f_rz(xv[q]);
            const float rv = (cb + h2 + q < m) ? xf - gq[h2 + q] : 0.f;
            s_acc = fmaf(rv, rv, s_acc);
            t_acc = fmaf(xf, xf, t_acc);
          }
        }
      }
    };
    if (cached && nk2 == 1) {
      // A = G staged once; up to X.ng2 column slices issued back to back into their own
      // accumulators (independent MMA chains), one commit and one wait per group
      if (half == 0) {
        float g[32];
        tmem_ld32(d1 + lane_base, g);
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          float h, l;
          tf32_split(q < r ? g[q] : 0.f, h, l);
          const int o = tc_off(row, q);
          X.Ahi[o] = h;
          X.Alo[o] = l;
        }
      }
      for (int g0 = 0; g0 < nns; g0 += X.ng2) {
        const int ng = min(X.ng2, nns - g0);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
          tc_fence_after();
          for (int q = 0; q < ng; ++q) {
            const float* t = cache2 + (size_t)(g0 + q) * 2 * b2;
            tc_slice_mma_at(X.Ahi, X.Alo, t, t + b2, d2 + (uint32_t)(q * TC_N2), TC_N2, true);
          }
          tc_commit(X.bar);
        }
        if (!tc_wait(X.bar, ph)) return tc_timeout(S, Xp, ph);
        for (int q = 0; q < ng; ++q) epilogue(g0 + q, 128u + (uint32_t)(q * TC_N2));
        tc_fence_before();
        __syncthreads();  // the accumulators are free again
        tc_fence_after();
      }
    } else
    for (int ns = 0; ns < nns; ++ns) {
      const int c0 = ns * TC_N2;
      for (int k2 = 0; k2 < nk2; ++k2) {
        if (half == 0) {
          if (nk2 > 1 || ns == 0) {  // A = G slice (unchanged across column slices if r <= 32)
            float g[32];
            tmem_ld32(d1 + lane_base + (uint32_t)(k2 * TC_K), g);
#pragma unroll
            for (int q = 0; q < 32; ++q) {
              float h, l;
              tf32_split(k2 * TC_K + q < r ? g[q] : 0.f, h, l);
              const int o = tc_off(row, q);
              X.Ahi[o] = h;
              X.Alo[o] = l;
            }
          }
        } else if (!cached) {
          tc_stage_qt(X, S.Qf, ld, m, r, c0, k2 * TC_K, 128);
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
          tc_fence_after();
          if (cached) {
            const float* t = cache2 + (size_t)(ns * nk2 + k2) * 2 * b2;
            tc_slice_mma_at(X.Ahi, X.Alo, t, t + b2, d2, TC_N2, k2 == 0);
          } else {
            tc_slice_mma(X, d2, TC_N2, k2 == 0);
          }
          tc_commit(X.bar);
        }
        if (!tc_wait(X.bar, ph)) return tc_timeout(S, Xp, ph);
      }
      epilogue(ns, 128u);
      tc_fence_before();
      __syncthreads();  // D2 and the staging buffers are free again
      tc_fence_after();
    }
    // ---- combine the two column halves of each row, store s, t, screen
    if (half == 1) {
      red_s[row] = s_acc;
      red_t[row] = t_acc;
    }
    __syncthreads();
    if (half == 0 && row < nrows) {
      const double s = (double)(s_acc + red_s[row]), t = (double)(t_acc + red_t[row]);
      const int j = row0 + row;
      S.s[O.jb + j] = s;
      S.t[O.jb + j] = t;
      const double yv = __ldg(y + j);
      if (!isfinite(yv) || !(t > 1e-30 && t < 1e30 && s <= tc * tc * t)) atomicMin(&q0_s, j);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) Xp->phase = ph;
  const int q0 = q0_s;
  __syncthreads();
  // every row of the block dependent: its fused sums go to P (both triangles) and u
  if (gsm && O.commit && q0 == b) {
    const int ntri = r * (r + 1) / 2;
    for (int e = threadIdx.x; e < ntri + r; e += NT) {
      if (e < ntri) {
        int rem = e, i = 0;
        while (rem >= r - i) {
          rem -= r - i;
          ++i;
        }
        const int l = i + rem;
        const double v = __ldcg(O.pp + e);
        S.P[(size_t)i * rm + l] = __ldcg(S.P + (size_t)i * rm + l) + v;
        if (l != i) S.P[(size_t)l * rm + i] = __ldcg(S.P + (size_t)l * rm + i) + v;
      } else {
        const int i = e - ntri;
        S.u[i] = __ldcg(S.u + i) + __ldcg(O.upp + i);
      }
    }
  }
  if (threadIdx.x == 0) *gram_done = gsm != nullptr && q0 == b;
  __syncthreads();
  return q0;
}

}  // namespace rg
