// rg_stream.cu -- rank-Greville update of ONE stream on the whole GPU.
//
// One rg_add_rows call is one cooperative persistent launch (one CTA per SM) that walks
// the call's rows in internal blocks (process_rows in rg_core.cuh). Per block of b rows:
//
//  1. gamma  : gamma_j = Ct Gamma_j (Q Gamma_j in the variants of Section 2.2) for all rows
//              of the block against the block-start basis (Eq. label_eq_gnplusoneproj).
//              Blocks of up to 64 rows: CTA tiles of up to 4 rows x BT basis rows whose
//              columns are split evenly over the SM's four sub-partitions.
//  2. reject : Gamma_r = Gamma_j - C^T gamma_j with the partial norms of s_j = ||Gamma_r||^2
//              and t_j = ||Gamma_j||^2 per 64-column chunk, in FP64 (Section 2.1, Eq.
//              label_eq_schur_complement). For small blocks, each item's basis tile arrives
//              by bulk copy (TMA) during step 1, and the CTA that completes a row group sums
//              its partials and takes the group's rank decisions.
//  3. decide : rank test of Eq. label_eq_eps on every row. Dependent rows leave C and Ct
//              unchanged (Theorem 6, dependent case), so every row before the first
//              independent row is decided correctly against the block-start basis.
//  4. update : the dependent run before the first special row goes into the information
//              form P += sum gamma gamma^T, u += sum gamma (y - gamma^T w_b) (rg_core.cuh);
//              a call of one small block defers it to the next launch, which folds it in
//              on the CTAs the rejection leaves idle.
//  5. rank changes: from the first independent (or, in mixed mode, candidate) row on, up
//              to SLOW_MAX rows are re-projected in FP64 and scanned in order: rank test,
//              append (Theorem 6, independent case) and a fix-up of the later rows of the
//              section (their rejections lose the new direction: Gamma_r,t -= kappa
//              Gamma_r,j), then the section's P/u update and one low-rank update of C and Ct.
//
// The solution is kept in coordinates w = w_b + P^-1 u (X = Ct^T w, from
// A^+ = Ct^T P^-1 B^T, Section 2.1); P^-1 and w are formed (Cholesky of P) only when X or
// an export is requested.
//
// FP64 mode keeps the general factorization of Algorithm 1 (C = selected rows, Ct its dual
// basis), or either variant of Section 2.2 (RG_ORTHONORMAL, RG_ORTHOGONAL). Mixed mode keeps
// the orthonormal variant (alpha = 1/||Gamma_r||: Ct = C = Q), projects in FP32 against an
// FP32 copy of Q, and re-decides in FP64 every row whose FP32 relative rejection exceeds the
// floor tau_lo. Its calls of at least TC_GRID_MIN rows run in stream_tc_kernel, where blocks
// of that size project 128-row chunks per CTA on the tensor cores (3xTF32, rg_tc.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <stdint.h>

#include "rg_core.cuh"

namespace rg {

template <bool F32, int VAR>
__global__ void __launch_bounds__(NT, 1) stream_kernel(StreamDev S, CallArgs A) {
  grid_barrier_init(S.ctrl);
  process_rows<GridTeam, F32, VAR>(GridTeam{S.ctrl}, S, A);
}

// Mixed mode, calls of at least TC_GRID_MIN rows: a separate instantiation, launched with
// TC_SMEM bytes of dynamic shared memory for the tensor-core chunk path (the small-call
// kernel keeps its whole L1); each CTA holds its tensor-memory columns for the call.
__global__ void __launch_bounds__(NT, 1) stream_tc_kernel(StreamDev S, CallArgs A) {
  __shared__ TcCtx tcx;
  __shared__ __align__(8) unsigned long long tc_bar;
  __shared__ uint32_t tc_tmem;
  extern __shared__ __align__(1024) unsigned char dyn_smem[];
  grid_barrier_init(S.ctrl);
  const bool tc_on = dyn_smem_bytes() >= (uint32_t)TC_SMEM;
  if (tc_on) {
    float* const dyn_base = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~static_cast<uintptr_t>(1023));
    tc_ctx_init(&tcx, &tc_bar, &tc_tmem, dyn_base, TC_SMEM);
    S.tcx = &tcx;
  }
  process_rows<GridTeam, true, VAR_ORTHONORMAL, true>(GridTeam{S.ctrl}, S, A);
  if (tc_on) tc_ctx_release(&tcx);
}

// Folds the P/u update deferred by the last small call (if any) into P and u: every CTA
// takes entries; the next kernel on the stream (form_w_kernel, export_prep_kernel) clears
// the pending count.
template <bool MIXED>
__global__ void __launch_bounds__(NT, 1) flush_pending_kernel(StreamDev S) {
  const int np = S.ctrl[CTRL_PEND_ROWS];
  if (np > 0 && S.Gpend) acc_rows<GridTeam, MIXED>(GridTeam{S.ctrl}, S, S.Gpend, S.Dpend, 0, np, S.ctrl[CTRL_R], 0);
}

// w = w_b + P^-1 u (one CTA), then X = Ct^T w (general) or Q^T w (orthonormal).
__global__ void __launch_bounds__(NT, 1) form_w_kernel(StreamDev S) {
  if (threadIdx.x == 0) S.ctrl[CTRL_PEND_ROWS] = 0;
  form_w(S, S.ctrl[CTRL_R]);
}
__global__ void solution_kernel(StreamDev S, double* X) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= S.m) return;
  const int r = S.ctrl[CTRL_R];
  const double* B = S.ortho ? S.C : S.Ct;
  double acc = 0.0;
  for (int i = 0; i < r; ++i) acc = fma(B[(size_t)i * S.ld + c], S.w[i], acc);
  X[c] = acc;
}

// For an export: w and P^-1 (CTA 0 factors P and forms w, then every CTA solves for some
// columns of P^-1).
__global__ void __launch_bounds__(NT, 1) export_prep_kernel(StreamDev S) {
  grid_barrier_init(S.ctrl);
  const int r = ld_acquire_i32(S.ctrl + CTRL_R);
  if (blockIdx.x == 0 && threadIdx.x == 0) S.ctrl[CTRL_PEND_ROWS] = 0;
  if (blockIdx.x == 0) form_w(S, r);
  if (!grid_barrier(S.ctrl)) return;
  form_pinv(GridTeam{S.ctrl}, S, r);
}

// Export helpers (compact copies with row stride m / r).
__global__ void export_kernel(StreamDev S, double* C, double* Ct, double* Pinv, double* w,
                              long long* basis) {
  const int r = S.ctrl[CTRL_R];
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long str = (long long)gridDim.x * blockDim.x;
  const long long nm = (long long)r * S.m;
  for (long long e = tid; e < nm; e += str) {
    const int i = (int)(e / S.m), c = (int)(e - (long long)i * S.m);
    if (C) C[e] = S.C[(size_t)i * S.ld + c];
    if (Ct) Ct[e] = S.ortho ? S.C[(size_t)i * S.ld + c] : S.Ct[(size_t)i * S.ld + c];
  }
  for (long long e = tid; e < (long long)r * r; e += str) {
    const int i = (int)(e / r), l = (int)(e - (long long)i * r);
    if (Pinv) Pinv[e] = S.Pinv[(size_t)i * S.r_max + l];
  }
  for (long long e = tid; e < r; e += str) {
    if (w) w[e] = S.w[e];
    if (basis) basis[e] = S.basis_rows[e];
  }
}

// ---------------------------------------------------------------------------------------
// Snapshots of the factorization (checkpoint / resume, and gradients through intermediate
// solutions): a header followed by the used rows of C, Ct (general variant), the FP32 copy
// of Q (mixed mode), the leading r x r block of P, and w_b, u and the basis-row indices.
// The buffer is laid out for r_max (its size is fixed at init); only rows below the rank,
// read on the device, are copied.
// ---------------------------------------------------------------------------------------
constexpr unsigned SNAP_MAGIC = 0x52475331u;  // "RGS1"

struct SnapHeader {
  unsigned magic;
  int m, ld, r_max, mixed, ortho, orthog;
  int r, kb, pend;
  long long rows_seen;
};
static_assert(sizeof(SnapHeader) <= 256, "snapshot header");

struct SnapLayout {
  size_t C, Ct, Qf, P, wb, u, basis, bytes;
};

__host__ __device__ inline SnapLayout snap_layout(int ld, int rm, int mixed, int ortho) {
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  SnapLayout L{};
  size_t off = 256;
  L.C = off;
  off += al((size_t)rm * ld * 8);
  L.Ct = ortho ? 0 : off;
  if (!ortho) off += al((size_t)rm * ld * 8);
  L.Qf = mixed ? off : 0;
  if (mixed) off += al((size_t)rm * ld * 4);
  L.P = off;
  off += al((size_t)rm * rm * 8);
  L.wb = off;
  off += al((size_t)rm * 8);
  L.u = off;
  off += al((size_t)rm * 8);
  L.basis = off;
  off += al((size_t)rm * 8);
  L.bytes = off;
  return L;
}

size_t snapshot_bytes(const StreamDev& S) { return snap_layout(S.ld, S.r_max, S.mixed, S.ortho).bytes; }

// Copies the state into buf (grid-stride; rows below the rank only). Runs after the
// deferred P/u update has been folded (flush_pending_kernel), so it also clears the
// pending count, as form_w_kernel does.
__global__ void snapshot_kernel(StreamDev S, unsigned char* buf) {
  const SnapLayout L = snap_layout(S.ld, S.r_max, S.mixed, S.ortho);
  const int r = S.ctrl[CTRL_R];
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long str = (long long)gridDim.x * blockDim.x;
  const long long nrow = (long long)r * S.ld;
  double* C = reinterpret_cast<double*>(buf + L.C);
  double* Ct = reinterpret_cast<double*>(buf + L.Ct);
  float* Qf = reinterpret_cast<float*>(buf + L.Qf);
  for (long long e = tid; e < nrow; e += str) {
    C[e] = S.C[e];
    if (!S.ortho) Ct[e] = S.Ct[e];
    if (S.mixed) Qf[e] = S.Qf[e];
  }
  double* P = reinterpret_cast<double*>(buf + L.P);
  for (long long e = tid; e < (long long)r * r; e += str) {
    const int i = (int)(e / r), l = (int)(e - (long long)i * r);
    P[(size_t)i * S.r_max + l] = S.P[(size_t)i * S.r_max + l];
  }
  double* wb = reinterpret_cast<double*>(buf + L.wb);
  double* u = reinterpret_cast<double*>(buf + L.u);
  long long* basis = reinterpret_cast<long long*>(buf + L.basis);
  for (long long e = tid; e < r; e += str) {
    wb[e] = S.wb[e];
    u[e] = S.u[e];
    basis[e] = S.basis_rows[e];
  }
  if (tid == 0) {
    SnapHeader H{};
    H.magic = SNAP_MAGIC;
    H.m = S.m;
    H.ld = S.ld;
    H.r_max = S.r_max;
    H.mixed = S.mixed;
    H.ortho = S.ortho;
    H.orthog = S.orthog;
    H.r = r;
    H.kb = S.ctrl[CTRL_KB];
    H.pend = S.ctrl[CTRL_PEND];
    H.rows_seen = *S.rows_seen;
    *reinterpret_cast<SnapHeader*>(buf) = H;
    S.ctrl[CTRL_PEND_ROWS] = 0;
  }
}

// The inverse copy. A header that does not match the state (other m, r_max or variant, or
// not a snapshot) sets ST_BADARG and leaves the state unchanged.
__global__ void restore_kernel(StreamDev S, const unsigned char* buf) {
  const SnapHeader H = *reinterpret_cast<const SnapHeader*>(buf);
  const bool ok = H.magic == SNAP_MAGIC && H.m == S.m && H.ld == S.ld && H.r_max == S.r_max &&
                  H.mixed == S.mixed && H.ortho == S.ortho && H.orthog == S.orthog && H.r >= 0 &&
                  H.r <= S.r_max;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (!ok) {
    if (tid == 0) atomicOr(S.ctrl + CTRL_STATUS, ST_BADARG);
    return;
  }
  const SnapLayout L = snap_layout(S.ld, S.r_max, S.mixed, S.ortho);
  const int r = H.r;
  const long long str = (long long)gridDim.x * blockDim.x;
  const long long nrow = (long long)r * S.ld;
  const double* C = reinterpret_cast<const double*>(buf + L.C);
  const double* Ct = reinterpret_cast<const double*>(buf + L.Ct);
  const float* Qf = reinterpret_cast<const float*>(buf + L.Qf);
  for (long long e = tid; e < nrow; e += str) {
    S.C[e] = C[e];
    if (!S.ortho) S.Ct[e] = Ct[e];
    if (S.mixed) S.Qf[e] = Qf[e];
  }
  const double* P = reinterpret_cast<const double*>(buf + L.P);
  for (long long e = tid; e < (long long)r * r; e += str) {
    const int i = (int)(e / r), l = (int)(e - (long long)i * r);
    S.P[(size_t)i * S.r_max + l] = P[(size_t)i * S.r_max + l];
  }
  const double* wb = reinterpret_cast<const double*>(buf + L.wb);
  const double* u = reinterpret_cast<const double*>(buf + L.u);
  const long long* basis = reinterpret_cast<const long long*>(buf + L.basis);
  for (long long e = tid; e < r; e += str) {
    S.wb[e] = wb[e];
    S.u[e] = u[e];
    S.basis_rows[e] = basis[e];
  }
  if (tid == 0) {
    S.ctrl[CTRL_R] = r;
    S.ctrl[CTRL_KB] = H.kb;
    S.ctrl[CTRL_PEND] = H.pend;
    S.ctrl[CTRL_PEND_ROWS] = 0;
    S.ctrl[CTRL_STATUS] = 0;
    *S.rows_seen = H.rows_seen;
  }
}

cudaError_t launch_snapshot(const StreamDev& S, void* buf, cudaStream_t stream) {
  snapshot_kernel<<<64, NT, 0, stream>>>(S, (unsigned char*)buf);
  return cudaGetLastError();
}

cudaError_t launch_restore(const StreamDev& S, const void* buf, cudaStream_t stream) {
  restore_kernel<<<64, NT, 0, stream>>>(S, (const unsigned char*)buf);
  return cudaGetLastError();
}

// Host-side launch helpers (declared in rg_host.h).
// FP32 projections always come with the orthonormal variant.
static const void* stream_kernel_ptr(int mixed, int ortho, int orthog) {
  if (mixed) return (const void*)stream_kernel<true, VAR_ORTHONORMAL>;
  if (ortho) return (const void*)stream_kernel<false, VAR_ORTHONORMAL>;
  if (orthog) return (const void*)stream_kernel<false, VAR_ORTHOGONAL>;
  return (const void*)stream_kernel<false, VAR_GENERAL>;
}

cudaError_t launch_stream(const StreamDev& S, const double* Gamma, const double* y, long long k,
                          uint8_t* indep, int grid, cudaStream_t stream) {
  CallArgs A{Gamma, y, k, indep};
  StreamDev Sc = S;
  void* args[] = {(void*)&Sc, (void*)&A};
  if (S.mixed && k >= TC_GRID_MIN)
    return cudaLaunchCooperativeKernel((const void*)stream_tc_kernel, dim3(grid), dim3(NT), args, TC_SMEM,
                                       stream);
  return cudaLaunchCooperativeKernel(stream_kernel_ptr(S.mixed, S.ortho, S.orthog), dim3(grid), dim3(NT),
                                     args, 0, stream);
}

cudaError_t stream_grid_size(int mixed, int ortho, int orthog, int* grid) {
  int dev = 0, nsm = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, stream_kernel_ptr(mixed, ortho, orthog), NT, 0);
  if (e != cudaSuccess) return e;
  if (mixed) {  // the kernel of large calls, with the tensor-core chunk path's operand tiles
    int per_tc = 0;
    e = cudaFuncSetAttribute((const void*)stream_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_tc, (const void*)stream_tc_kernel, NT, TC_SMEM);
    if (e != cudaSuccess) return e;
    per = std::min(per, per_tc);
  }
  *grid = std::min(nsm, 1024) * (per >= 1 ? 1 : 0);  // the section scan holds <= 1024 workers
  return cudaSuccess;
}

cudaError_t launch_flush(const StreamDev& S, int grid, cudaStream_t stream) {
  if (!S.Gpend) return cudaSuccess;
  if (S.mixed) flush_pending_kernel<true><<<grid, NT, 0, stream>>>(S);
  else flush_pending_kernel<false><<<grid, NT, 0, stream>>>(S);
  return cudaGetLastError();
}

cudaError_t launch_export_prep(const StreamDev& S, int grid, cudaStream_t stream) {
  StreamDev Sc = S;
  void* args[] = {(void*)&Sc};
  return cudaLaunchCooperativeKernel((const void*)export_prep_kernel, dim3(grid), dim3(NT), args,
                                     0, stream);
}

cudaError_t launch_solution(const StreamDev& S, double* X, cudaStream_t stream) {
  form_w_kernel<<<1, NT, 0, stream>>>(S);
  solution_kernel<<<(S.m + NT - 1) / NT, NT, 0, stream>>>(S, X);
  return cudaGetLastError();
}

cudaError_t launch_export(const StreamDev& S, double* C, double* Ct, double* Pinv, double* w,
                          long long* basis, cudaStream_t stream) {
  export_kernel<<<64, NT, 0, stream>>>(S, C, Ct, Pinv, w, basis);
  return cudaGetLastError();
}

}  // namespace rg
