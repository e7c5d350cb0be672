// rg_batch.cu -- many independent rank-Greville streams of uneven shape in ONE persistent
// kernel, plus the batched half of the C ABI.
//
// Each instance b (m_b columns, capacity r_max_b) owns its state (C, Ct or the FP32 copy
// of Q, P^-1, w, basis rows) in one arena. Persistent CTAs pop instances from an atomic
// work counter over an order sorted by estimated cost n_b m_b min(n_b, r_max_b),
// longest first, and apply all rows of the instance with the same block phases as the
// single-stream kernel (rg_core.cuh), the team being the CTA itself. Each CTA owns a
// scratch slab sized for the largest instance. There is no spin-wait anywhere here.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/rg.h"
#include "rg_adjoint.cuh"
#include "rg_core.cuh"
#include "rg_host.h"

namespace rg {

struct BatchDev {
  int B, mixed, ortho, orthog, test_mode, kb_max, ld_max, r_max_max, nmc_max;
  int kb_cap;  // rows of block scratch laid out per CTA (kb_max <= kb_cap)
  int tc_group;  // mixed mode: second-product column slices issued per commit (1..TC_NG2)
  double tol, tau_lo;
  const int* m;               // B
  const int* r_max;           // B
  const long long* soff;      // B: byte offset of the instance state in `state`
  const long long* xoff_def;  // B + 1: packed solution offsets by m_b
  char* state;
  int* ctrl;                  // B x CTRL_N
  long long* rows_seen;       // B
  char* scratch;              // one slab per CTA
  size_t scratch_stride;
  int* order;                 // B
  int* queue;                 // [1]
  int* bstatus;               // [1] OR of the instances' status bits
};

__host__ __device__ inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// Instance state layout; fills S's state pointers when base != null. Returns bytes.
__host__ __device__ inline size_t inst_layout(int m, int ld, int rmax, int mixed, int ortho, char* base,
                                              StreamDev* S) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off = al256(off + bytes);
    return p;
  };
  char* C = take((size_t)rmax * ld * 8);
  char* Ct = ortho ? nullptr : take((size_t)rmax * ld * 8);
  char* Qf = mixed ? take((size_t)rmax * ld * 4) : nullptr;
  char* P = take((size_t)rmax * rmax * 8);
  char* wb = take((size_t)rmax * 8);
  char* u = take((size_t)rmax * 8);
  char* w = take((size_t)rmax * 8);
  char* basis = take((size_t)rmax * 8);
  if (S) {
    S->C = (double*)C;
    S->Ct = (double*)Ct;
    S->Qf = (float*)Qf;
    S->Pinv = nullptr;
    S->P = (double*)P;
    S->wb = (double*)wb;
    S->u = (double*)u;
    S->w = (double*)w;
    S->basis_rows = (long long*)basis;
  }
  (void)m;
  return off;
}

// Per-CTA scratch layout (sized with the batch maxima). Returns bytes.
__host__ __device__ inline size_t scratch_layout(int kb, int ldm, int rmm, int nmcm, char* base,
                                                 StreamDev* S) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off = al256(off + bytes);
    return p;
  };
  char* G = take((size_t)kb * rmm * 8);
  char* sp = take((size_t)kb * nmcm * 8);
  char* tp = take((size_t)kb * nmcm * 8);
  char* s = take((size_t)kb * 8);
  char* t = take((size_t)kb * 8);
  char* rf = take((size_t)kb);
  char* R = take((size_t)SLOW_MAX * ldm * 8);
  char* Kv = take((size_t)SLOW_MAX * ldm * 8);
  char* Gind = take((size_t)SLOW_MAX * rmm * 8);
  char* alpha = take((size_t)SLOW_MAX * 8);
  char* jind = take((size_t)SLOW_MAX * 4);
  char* Dall = take((size_t)kb * 8);
  char* Pp = take((size_t)rmm * rmm * 8);  // one chunk: a CTA team gains nothing from more
  char* up = take((size_t)NCH_MAX * rmm * 8);
  char* Lw = take((size_t)rmm * rmm * 8);
  char* Kap = take((size_t)SLOW_MAX * SLOW_MAX * 8);
  char* Sp = take((size_t)2 * 32 * 8);  // one worker (the CTA)
  if (S) {
    S->Sp = (double*)Sp;
    S->sp_stride = 32;
    S->Dall = (double*)Dall;
    S->Pp = (double*)Pp;
    S->pp_cap = (size_t)rmm * rmm;
    S->up = (double*)up;
    S->Lw = (double*)Lw;
    S->Kap = (double*)Kap;
    S->G = (double*)G;
    S->spart = (double*)sp;
    S->tpart = (double*)tp;
    S->s = (double*)s;
    S->t = (double*)t;
    S->rowflag = (uint8_t*)rf;
    S->R = (double*)R;
    S->Kv = (double*)Kv;
    S->Gind = (double*)Gind;
    S->alpha = (double*)alpha;
    S->jind = (int*)jind;
  }
  return off;
}

// Dynamic shared memory (TC_SMEM bytes in FP64 mode, TC_SMEM_MIXED in mixed mode) holds
// the rejections of a sequential section when they fit and, in mixed mode, the operand
// tiles and the B-tile cache of the tensor-core projection (never in use at the same
// time). Mixed mode also sets up the
// CTA's tensor-core context: one mbarrier and TC_TMEM_COLS columns of tensor memory (one
// CTA per SM in mixed mode, so the 512 columns of an SM always suffice). FP64 mode runs two
// CTAs per SM; mixed mode one, with the register budget that its staging needs.
template <bool MIXED, int VAR>
__global__ void __launch_bounds__(NT, MIXED ? 1 : 2) batch_kernel(BatchDev D, const double* __restrict__ Gp,
                                                   const int64_t* __restrict__ roff,
                                                   const int64_t* __restrict__ eoff,
                                                   const double* __restrict__ yp, uint8_t* indep) {
  __shared__ int item;
  __shared__ TcCtx tcx;
  __shared__ __align__(8) unsigned long long tc_bar;
  __shared__ uint32_t tc_tmem;
  extern __shared__ __align__(1024) unsigned char dyn_smem[];
  float* const dyn_base = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~static_cast<uintptr_t>(1023));
  if (MIXED) tc_ctx_init(&tcx, &tc_bar, &tc_tmem, dyn_base, TC_SMEM_MIXED, D.tc_group);
  StreamDev S{};
  S.tcx = MIXED ? (void*)&tcx : nullptr;
  S.Rs = reinterpret_cast<double*>(dyn_base);
  S.rs_cap = ((MIXED ? TC_SMEM_MIXED : TC_SMEM) - 1024) / 8;
  constexpr bool ORTHO = VAR == VAR_ORTHONORMAL;
  S.mixed = MIXED;
  S.ortho = ORTHO;
  S.orthog = VAR == VAR_ORTHOGONAL;
  S.test_mode = D.test_mode;
  S.tol = D.tol;
  S.tau_lo = D.tau_lo;
  S.kb_max = D.kb_max;
  scratch_layout(D.kb_cap, D.ld_max, D.r_max_max, D.nmc_max,
                 D.scratch + (size_t)blockIdx.x * D.scratch_stride, &S);
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(D.queue, 1);
    __syncthreads();
    const int it = item;
    __syncthreads();
    if (it >= D.B) break;
    const int b = D.order[it];
    const int m = D.m[b];
    const long long n = roff[b + 1] - roff[b];
    if (n <= 0) continue;
    if (eoff[b + 1] - eoff[b] != n * (long long)m) {
      if (threadIdx.x == 0) {
        atomicOr(D.ctrl + (size_t)b * CTRL_N + CTRL_STATUS, ST_BADARG);
        atomicOr(D.bstatus, ST_BADARG);
      }
      continue;
    }
    S.m = m;
    S.ld = (m + 3) / 4 * 4;
    S.r_max = D.r_max[b];
    S.nmc = (m + MC - 1) / MC;
    inst_layout(m, S.ld, S.r_max, MIXED, ORTHO, D.state + D.soff[b], &S);
    S.ctrl = D.ctrl + (size_t)b * CTRL_N;
    S.rows_seen = D.rows_seen + b;
    CallArgs A{Gp + eoff[b], yp + roff[b], n, indep ? indep + roff[b] : nullptr};
    const bool ok = process_rows<CtaTeam, MIXED, VAR>(CtaTeam{}, S, A);
    __syncthreads();
    if (threadIdx.x == 0) {
      const int st = ld_acquire_i32(S.ctrl + CTRL_STATUS);
      if (st) atomicOr(D.bstatus, st);
    }
    if (!ok) break;  // a bounded wait gave up: stop taking work
  }
  if (MIXED) tc_ctx_release(&tcx);
}

// FP32 projections always come with the orthonormal variant.
static const void* batch_kernel_ptr(int mixed, int ortho, int orthog) {
  if (mixed) return (const void*)batch_kernel<true, VAR_ORTHONORMAL>;
  if (ortho) return (const void*)batch_kernel<false, VAR_ORTHONORMAL>;
  if (orthog) return (const void*)batch_kernel<false, VAR_ORTHOGONAL>;
  return (const void*)batch_kernel<false, VAR_GENERAL>;
}

// Longest-first order of the instances for this call (single CTA, bitonic sort in shared
// memory for B <= 16384; larger batches keep index order). Also resets the work counter.
__global__ void order_kernel(BatchDev D, const int64_t* __restrict__ roff) {
  extern __shared__ unsigned long long keys[];
  const int B = D.B;
  if (threadIdx.x == 0) *D.queue = 0;
  if (B > 16384) {
    for (int b = threadIdx.x; b < B; b += blockDim.x) D.order[b] = b;
    return;
  }
  int P = 1;
  while (P < B) P <<= 1;
  for (int b = threadIdx.x; b < P; b += blockDim.x) {
    unsigned long long key = ~0ull;
    if (b < B) {
      const long long n = roff[b + 1] - roff[b];
      const long long m = D.m[b];
      const long long r = min((long long)D.r_max[b], max(n, 1ll));
      double cost = (double)max(n, 0ll) * (double)m * (double)r;
      const double cap = 8.796093022207e12;  // 2^43
      if (cost > cap - 1.0) cost = cap - 1.0;
      const unsigned long long c = (unsigned long long)cost;
      key = ((((1ull << 43) - 1) - c) << 20) | (unsigned long long)b;  // descending cost
    }
    keys[b] = key;
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const unsigned long long a = keys[i], c = keys[l];
          if ((a > c) == up) {
            keys[i] = c;
            keys[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int b = threadIdx.x; b < B; b += blockDim.x) D.order[b] = (int)(keys[b] & 0xFFFFFull);
}

// One CTA per instance (strided): w = w_b + P^-1 u in the CTA's scratch slab, then X.
__global__ void __launch_bounds__(NT, 2) batch_solution_kernel(BatchDev D, double* X, const int64_t* xoff,
                                                              int64_t* ranks) {
  StreamDev S{};
  scratch_layout(D.kb_cap, D.ld_max, D.r_max_max, D.nmc_max,
                 D.scratch + (size_t)blockIdx.x * D.scratch_stride, &S);
  for (int b = blockIdx.x; b < D.B; b += gridDim.x) {
    const int m = D.m[b];
    const int ld = (m + 3) / 4 * 4;
    S.m = m;
    S.ld = ld;
    S.r_max = D.r_max[b];
    S.ctrl = D.ctrl + (size_t)b * CTRL_N;
    inst_layout(m, ld, D.r_max[b], D.mixed, D.ortho, D.state + D.soff[b], &S);
    const int r = D.ctrl[(size_t)b * CTRL_N + CTRL_R];
    __syncthreads();
    form_w(S, r);
    const double* Bm = D.ortho ? S.C : S.Ct;
    const long long x0 = xoff ? xoff[b] : D.xoff_def[b];
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
      double acc = 0.0;
      for (int i = 0; i < r; ++i) acc = fma(Bm[(size_t)i * ld + c], S.w[i], acc);
      X[x0 + c] = acc;
    }
    if (ranks && threadIdx.x == 0) ranks[b] = r;
  }
}

// Adjoint of every instance's solution (one CTA per instance, strided): w and the
// Cholesky factor of P (form_w), then adjoint_run with the CTA as the team. Workspace wk:
// 4 m-vectors per instance at 4 x_off, 7 r_max_max-vectors per instance, 3 n-vectors per
// instance at 3 row_off.
__global__ void __launch_bounds__(NT, 2) batch_adjoint_kernel(BatchDev D, const double* __restrict__ Gp,
                                                              const int64_t* __restrict__ roff,
                                                              const int64_t* __restrict__ eoff,
                                                              const double* __restrict__ yp,
                                                              const double* __restrict__ gp,
                                                              const int64_t* __restrict__ xoff, double* gAp,
                                                              double* gyp, double* wk, long long sum_m) {
  StreamDev S{};
  scratch_layout(D.kb_cap, D.ld_max, D.r_max_max, D.nmc_max,
                 D.scratch + (size_t)blockIdx.x * D.scratch_stride, &S);
  double* wm = wk;
  double* wr = wk + 4 * sum_m;
  double* wn = wr + (size_t)7 * D.r_max_max * D.B;
  for (int b = blockIdx.x; b < D.B; b += gridDim.x) {
    const int m = D.m[b];
    const long long n = roff[b + 1] - roff[b];
    if (n < 0 || eoff[b + 1] - eoff[b] != n * (long long)m) {
      if (threadIdx.x == 0) {
        atomicOr(D.ctrl + (size_t)b * CTRL_N + CTRL_STATUS, ST_BADARG);
        atomicOr(D.bstatus, ST_BADARG);
      }
      continue;
    }
    S.m = m;
    S.ld = (m + 3) / 4 * 4;
    S.r_max = D.r_max[b];
    S.mixed = D.mixed;
    S.ortho = D.ortho;
    S.orthog = D.orthog;
    S.ctrl = D.ctrl + (size_t)b * CTRL_N;
    inst_layout(m, S.ld, S.r_max, D.mixed, D.ortho, D.state + D.soff[b], &S);
    const int r = D.ctrl[(size_t)b * CTRL_N + CTRL_R];
    __syncthreads();
    form_w(S, r);
    const long long x0 = xoff ? xoff[b] : D.xoff_def[b];
    const long long xw = D.xoff_def[b];
    AdjArgs J{};
    J.A = Gp + eoff[b];
    J.y = yp + roff[b];
    J.n = n;
    J.g = gp + x0;
    J.gA = gAp + eoff[b];
    J.gy = gyp + roff[b];
    J.X = wm + 4 * xw;
    J.Aph = J.X + m;
    J.gperp = J.Aph + m;
    J.v = J.gperp + m;
    double* rv = wr + (size_t)7 * D.r_max_max * b;
    J.a = rv;
    J.c = rv + D.r_max_max;
    J.e = rv + 2 * D.r_max_max;
    J.al = rv + 3 * D.r_max_max;
    J.be = rv + 4 * D.r_max_max;
    J.bth = rv + 5 * D.r_max_max;
    J.de = rv + 6 * D.r_max_max;
    J.h = wn + 3 * roff[b];
    J.z = J.h + n;
    J.rho = J.z + n;
    J.part = nullptr;
    J.nrc = 1;
    adjoint_run<CtaTeam>(CtaTeam{}, S, J, r);
    __syncthreads();
  }
}

__global__ void batch_reset_kernel(BatchDev D, int kb0) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < D.B; b += gridDim.x * blockDim.x) {
    int* c = D.ctrl + (size_t)b * CTRL_N;
    for (int i = 0; i < CTRL_N; ++i) c[i] = 0;
    c[CTRL_KB] = kb0;
    D.rows_seen[b] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *D.bstatus = 0;
}

__global__ void batch_clear_status_kernel(BatchDev D) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < D.B; b += gridDim.x * blockDim.x)
    D.ctrl[(size_t)b * CTRL_N + CTRL_STATUS] &= ST_TIMEOUT;
  if (blockIdx.x == 0 && threadIdx.x == 0) *D.bstatus &= ST_TIMEOUT;
}

}  // namespace rg

using namespace rg;

struct rg_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  BatchDev D{};
  int grid = 0;
  void* arena = nullptr;
  std::vector<int> m, r_max;
};

namespace {
int kb0_of(const BatchDev& D) { return std::min(KB_MIN, D.kb_max); }
bool valid_batch(rg_batch* bt) { return bt && bt->arena; }
}  // namespace

extern "C" {

rg_status rg_batch_init(rg_batch** out, int64_t B, const int64_t* m, double tol, int flags,
                        const int64_t* r_max, void* cuda_stream) {
  if (!out) return fail(RG_EINVAL, "rg_batch_init: out is NULL");
  *out = nullptr;
  if (B <= 0 || B > (1 << 20)) return fail(RG_EINVAL, "rg_batch_init: B = %lld out of range", (long long)B);
  if (!m) return fail(RG_EINVAL, "rg_batch_init: m is NULL");
  if (std::isnan(tol)) return fail(RG_EINVAL, "rg_batch_init: tol is NaN");
  if (flags & ~(RG_MIXED | RG_TEST_PAPER | RG_ORTHONORMAL | RG_ORTHOGONAL))
    return fail(RG_EINVAL, "rg_batch_init: unknown flags %d", flags);
  if ((flags & RG_ORTHOGONAL) && (flags & (RG_MIXED | RG_ORTHONORMAL)))
    return fail(RG_EINVAL, "rg_batch_init: RG_ORTHOGONAL excludes RG_MIXED and RG_ORTHONORMAL");
  rg_batch* bt = new (std::nothrow) rg_batch();
  if (!bt) return fail(RG_ENOMEM, "rg_batch_init: host allocation failed");
  bt->m.resize(B);
  bt->r_max.resize(B);
  int mmax = 0, rmm = 0;
  for (int64_t b = 0; b < B; ++b) {
    if (m[b] <= 0 || m[b] > (1 << 16)) {
      delete bt;
      return fail(RG_EINVAL, "rg_batch_init: m[%lld] = %lld out of range", (long long)b, (long long)m[b]);
    }
    long long rb = r_max ? r_max[b] : m[b];
    if (rb <= 0 || rb > m[b]) rb = m[b];
    bt->m[b] = (int)m[b];
    bt->r_max[b] = (int)rb;
    mmax = std::max(mmax, (int)m[b]);
    rmm = std::max(rmm, (int)rb);
  }
  cudaError_t e = cudaGetDevice(&bt->device);
  if (e != cudaSuccess) {
    delete bt;
    return cuda_fail(e, "rg_batch_init: no CUDA device");
  }
  bt->stream = (cudaStream_t)cuda_stream;
  BatchDev& D = bt->D;
  D.B = (int)B;
  D.mixed = (flags & RG_MIXED) ? 1 : 0;
  D.ortho = (flags & (RG_MIXED | RG_ORTHONORMAL)) ? 1 : 0;
  D.orthog = (flags & RG_ORTHOGONAL) ? 1 : 0;
  D.test_mode = (flags & RG_TEST_PAPER) ? 2 : 0;
  D.tol = tol;
  D.tau_lo = 1e-5;
  D.ld_max = (mmax + 3) / 4 * 4;
  D.r_max_max = rmm;
  D.nmc_max = (mmax + MC - 1) / MC;
  int kb = 512;  // layout capacity; the default block cap is 256 (rg_batch_set_block_rows)
  while (kb > 32 && (size_t)kb * rmm * 8 > (size_t)4 << 20) kb /= 2;
  D.kb_cap = kb;
  D.kb_max = std::min(kb, 256);
  D.tc_group = TC_NG2;
  int nsm = 0, per = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, bt->device);
  const int dyn = D.mixed ? TC_SMEM_MIXED : TC_SMEM;
  const void* kfn = batch_kernel_ptr(D.mixed, D.ortho, D.orthog);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  if (e == cudaSuccess)  // up to two CTAs of ~105 KiB each per SM
    e = cudaFuncSetAttribute(kfn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kfn, NT, dyn);
  if (e != cudaSuccess || per <= 0) {
    delete bt;
    return e != cudaSuccess ? cuda_fail(e, "rg_batch_init: occupancy") : fail(RG_ECUDA, "rg_batch_init: no occupancy");
  }
  per = std::min(per, D.mixed ? 512 / TC_TMEM_COLS : 2);  // tensor memory: 512 columns per SM
  bt->grid = std::min<long long>((long long)nsm * per, B);
  // host-side layout
  std::vector<long long> soff(B), xoff(B + 1, 0);
  size_t state_bytes = 0;
  for (int64_t b = 0; b < B; ++b) {
    soff[b] = (long long)state_bytes;
    const int ld = (bt->m[b] + 3) / 4 * 4;
    state_bytes += inst_layout(bt->m[b], ld, bt->r_max[b], D.mixed, D.ortho, nullptr, nullptr);
    xoff[b + 1] = xoff[b] + bt->m[b];
  }
  StreamDev tmp{};
  D.scratch_stride = al256(scratch_layout(D.kb_cap, D.ld_max, D.r_max_max, D.nmc_max, nullptr, &tmp));
  size_t off = 0;
  auto place = [&](size_t bytes) {
    const size_t o = off;
    off = al256(off + bytes);
    return o;
  };
  const size_t o_m = place(B * 4), o_r = place(B * 4), o_soff = place(B * 8), o_xoff = place((B + 1) * 8),
               o_ctrl = place((size_t)B * CTRL_N * 4), o_rows = place(B * 8), o_order = place(B * 4),
               o_q = place(4), o_bs = place(4), o_state = place(state_bytes),
               o_scr = place(D.scratch_stride * (size_t)bt->grid);
  e = cudaMalloc(&bt->arena, off);
  if (e != cudaSuccess) {
    delete bt;
    return cuda_fail(e, "rg_batch_init: cudaMalloc");
  }
  char* base = (char*)bt->arena;
  D.m = (int*)(base + o_m);
  D.r_max = (int*)(base + o_r);
  D.soff = (long long*)(base + o_soff);
  D.xoff_def = (long long*)(base + o_xoff);
  D.ctrl = (int*)(base + o_ctrl);
  D.rows_seen = (long long*)(base + o_rows);
  D.order = (int*)(base + o_order);
  D.queue = (int*)(base + o_q);
  D.bstatus = (int*)(base + o_bs);
  D.state = base + o_state;
  D.scratch = base + o_scr;
  e = cudaMemsetAsync(bt->arena, 0, off, bt->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync((void*)D.m, bt->m.data(), B * 4, cudaMemcpyHostToDevice, bt->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync((void*)D.r_max, bt->r_max.data(), B * 4, cudaMemcpyHostToDevice, bt->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync((void*)D.soff, soff.data(), B * 8, cudaMemcpyHostToDevice, bt->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync((void*)D.xoff_def, xoff.data(), (B + 1) * 8, cudaMemcpyHostToDevice, bt->stream);
  if (e == cudaSuccess) {
    batch_reset_kernel<<<(B + 255) / 256, 256, 0, bt->stream>>>(D, kb0_of(D));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(bt->stream);  // host vectors go out of scope
  if (e == cudaSuccess && B <= 16384)
    e = cudaFuncSetAttribute(order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * 8);
  if (e != cudaSuccess) {
    cudaFree(bt->arena);
    delete bt;
    return cuda_fail(e, "rg_batch_init: initialising the batch");
  }
  *out = bt;
  return RG_OK;
}

rg_status rg_batch_add_rows(rg_batch* bt, const double* Gamma_packed, const int64_t* row_offsets,
                            const int64_t* elem_offsets, const double* y_packed, uint8_t* indep_out) {
  NvtxRange nvtx_range("rg_batch_add_rows");
  if (!valid_batch(bt)) return fail(RG_EINVAL, "rg_batch_add_rows: invalid batch");
  if (!Gamma_packed || !row_offsets || !elem_offsets || !y_packed)
    return fail(RG_EINVAL, "rg_batch_add_rows: NULL argument");
  const BatchDev& D = bt->D;
  int P = 1;
  while (P < D.B) P <<= 1;
  const size_t shm = D.B <= 16384 ? (size_t)P * 8 : 0;
  order_kernel<<<1, 1024, shm, bt->stream>>>(D, row_offsets);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "rg_batch_add_rows: order kernel");
  if (indep_out) {
    // rows not applied keep 0xFF; the total row count is only known on the device, so the
    // kernel writes every applied row and the rest are left as the caller initialised them
  }
  if (D.mixed)
    batch_kernel<true, VAR_ORTHONORMAL><<<bt->grid, NT, TC_SMEM_MIXED, bt->stream>>>(
        D, Gamma_packed, row_offsets, elem_offsets, y_packed, indep_out);
  else if (D.ortho)
    batch_kernel<false, VAR_ORTHONORMAL><<<bt->grid, NT, TC_SMEM, bt->stream>>>(
        D, Gamma_packed, row_offsets, elem_offsets, y_packed, indep_out);
  else if (D.orthog)
    batch_kernel<false, VAR_ORTHOGONAL><<<bt->grid, NT, TC_SMEM, bt->stream>>>(
        D, Gamma_packed, row_offsets, elem_offsets, y_packed, indep_out);
  else
    batch_kernel<false, VAR_GENERAL><<<bt->grid, NT, TC_SMEM, bt->stream>>>(
        D, Gamma_packed, row_offsets, elem_offsets, y_packed, indep_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "rg_batch_add_rows: launch");
  return RG_OK;
}

rg_status rg_batch_solution(rg_batch* bt, double* X_packed, const int64_t* x_offsets, int64_t* ranks_out) {
  NvtxRange nvtx_range("rg_batch_solution");
  if (!valid_batch(bt)) return fail(RG_EINVAL, "rg_batch_solution: invalid batch");
  if (!X_packed) return fail(RG_EINVAL, "rg_batch_solution: X is NULL");
  batch_solution_kernel<<<bt->grid, NT, 0, bt->stream>>>(bt->D, X_packed, x_offsets, ranks_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "rg_batch_solution: launch");
  return RG_OK;
}

rg_status rg_batch_sync(rg_batch* bt) {
  if (!valid_batch(bt)) return fail(RG_EINVAL, "rg_batch_sync: invalid batch");
  int bits = 0;
  cudaError_t e = cudaMemcpyAsync(&bits, bt->D.bstatus, 4, cudaMemcpyDeviceToHost, bt->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(bt->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_batch_sync");
  if (bits) {
    batch_clear_status_kernel<<<(bt->D.B + 255) / 256, 256, 0, bt->stream>>>(bt->D);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rg_batch_sync: clearing status");
  }
  return status_from_bits(bits);
}

rg_status rg_batch_reset(rg_batch* bt) {
  if (!valid_batch(bt)) return fail(RG_EINVAL, "rg_batch_reset: invalid batch");
  batch_reset_kernel<<<(bt->D.B + 255) / 256, 256, 0, bt->stream>>>(bt->D, kb0_of(bt->D));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "rg_batch_reset");
  return RG_OK;
}

rg_status rg_batch_adjoint(rg_batch* bt, const double* Gamma_packed, const int64_t* row_offsets,
                           const int64_t* elem_offsets, const double* y_packed, int64_t total_rows,
                           const double* g_packed, const int64_t* x_offsets, double* gA_packed,
                           double* gy_packed) {
  NvtxRange nvtx_range("rg_batch_adjoint");
  if (!valid_batch(bt)) return fail(RG_EINVAL, "rg_batch_adjoint: invalid batch");
  if (total_rows < 0) return fail(RG_EINVAL, "rg_batch_adjoint: total_rows < 0");
  if (!row_offsets || !elem_offsets || !g_packed || (total_rows > 0 && (!Gamma_packed || !y_packed || !gA_packed || !gy_packed)))
    return fail(RG_EINVAL, "rg_batch_adjoint: NULL buffer");
  const BatchDev& D = bt->D;
  long long sum_m = 0;
  for (int b = 0; b < D.B; ++b) sum_m += bt->m[b];
  const size_t doubles = (size_t)4 * sum_m + (size_t)7 * D.r_max_max * D.B + (size_t)3 * std::max<int64_t>(total_rows, 1);
  double* wk = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&wk, doubles * sizeof(double), bt->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_batch_adjoint: workspace");
  batch_adjoint_kernel<<<bt->grid, NT, 0, bt->stream>>>(D, Gamma_packed, row_offsets, elem_offsets, y_packed,
                                                        g_packed, x_offsets, gA_packed, gy_packed, wk, sum_m);
  e = cudaGetLastError();
  const cudaError_t e2 = cudaFreeAsync(wk, bt->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_batch_adjoint: launch");
  if (e2 != cudaSuccess) return cuda_fail(e2, "rg_batch_adjoint: workspace release");
  return RG_OK;
}

rg_status rg_batch_set_stream(rg_batch* bt, void* cuda_stream) {
  if (!valid_batch(bt)) return fail(RG_EINVAL, "rg_batch_set_stream: invalid batch");
  cudaError_t e = cudaStreamSynchronize(bt->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_batch_set_stream");
  bt->stream = (cudaStream_t)cuda_stream;
  return RG_OK;
}

rg_status rg_batch_set_screen(rg_batch* bt, double tau_lo) {
  if (!valid_batch(bt)) return fail(RG_EINVAL, "rg_batch_set_screen: invalid batch");
  if (!(tau_lo > 0.0 && tau_lo < 1.0)) return fail(RG_EINVAL, "rg_batch_set_screen: tau_lo = %g outside (0, 1)", tau_lo);
  bt->D.tau_lo = tau_lo;
  return RG_OK;
}

rg_status rg_batch_set_block_rows(rg_batch* bt, int64_t rows, int64_t* rows_out) {
  if (!valid_batch(bt)) return fail(RG_EINVAL, "rg_batch_set_block_rows: invalid batch");
  if (rows > 0) {
    if (rows < 32 || rows > bt->D.kb_cap)
      return fail(RG_EINVAL, "rg_batch_set_block_rows: %lld outside [32, %d]", (long long)rows, bt->D.kb_cap);
    bt->D.kb_max = (int)rows;
  }
  if (rows_out) *rows_out = bt->D.kb_max;
  return RG_OK;
}

rg_status rg_batch_set_tc_group(rg_batch* bt, int64_t group, int64_t* group_out) {
  if (!valid_batch(bt)) return fail(RG_EINVAL, "rg_batch_set_tc_group: invalid batch");
  if (group > 0) {
    if (group > TC_NG2)
      return fail(RG_EINVAL, "rg_batch_set_tc_group: %lld outside [1, %d]", (long long)group, TC_NG2);
    bt->D.tc_group = (int)group;
  }
  if (group_out) *group_out = bt->D.tc_group;
  return RG_OK;
}

rg_status rg_batch_free(rg_batch* bt) {
  if (!bt) return RG_OK;
  cudaStreamSynchronize(bt->stream);
  if (bt->arena) cudaFree(bt->arena);
  delete bt;
  return RG_OK;
}

}  // extern "C"
