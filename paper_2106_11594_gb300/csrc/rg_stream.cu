// rg_stream.cu -- rank-Greville update of ONE stream on the whole GPU.
//
// One rg_add_rows call is one cooperative persistent launch (one CTA per SM) that walks
// the call's rows in internal blocks (rg_core.cuh). Per block of b rows:
//
//  1. gamma  : gamma_j = Ct Gamma_j for all rows of the block against the block-start
//              basis (Eq. label_eq_gnplusoneproj). Warp tiles, warp-shuffle reductions.
//  2. reject : Gamma_r = Gamma_j - C^T gamma_j, with s_j = ||Gamma_r||^2 and
//              t_j = ||Gamma_j||^2 accumulated in FP64 (Section 2.1, Eq.
//              label_eq_schur_complement).
//  3. decide : rank test of Eq. label_eq_eps on every row. Dependent rows leave C and Ct
//              unchanged (Theorem 6, dependent case), so every row before the first
//              independent row is decided correctly against the block-start basis.
//  4. update : the leading run of dependent rows is applied to P^-1 and w in steps of up
//              to SB rows with the blocked form of the Sherman-Morrison update of
//              Eq. label_eq_Pnplusoneinv_lindep_update (the Woodbury identity):
//              Z = P^-1 G, M = I + G^T Z, P^-1 <- P^-1 - Z M^-1 Z^T, w <- w + Z M^-1 (y - G^T w),
//              which equals SB successive single-row updates in exact arithmetic.
//  5. rank changes: from the first independent (or, in mixed mode, candidate) row on, up
//              to SLOW_MAX rows are re-projected in FP64 and scanned in order by one CTA:
//              rank test, append (Theorem 6, independent case) and an in-block fix-up of
//              the later rows of the section (their rejections lose the new direction:
//              Gamma_r,t -= kappa Gamma_r,j with kappa = K_j^T Gamma_r,t). The dependent
//              runs between appends go through step 4; the appends to C and Ct are applied
//              as one low-rank product afterwards.
//
// The solution is kept in coordinates w (X = Ct^T w, which follows from
// A^+ = Ct^T P^-1 B^T, Section 2.1): the a-priori error is y - Gamma^T X = y - gamma^T w,
// a dependent row adds zeta (y - gamma^T w) / (1 + gamma^T zeta) to w (Theorem 5) and an
// independent row appends y to w (Theorem 4). X is materialised on request.
//
// FP64 mode keeps the general factorization of Algorithm 1 (C = selected rows, Ct its dual
// basis). Mixed mode keeps the orthonormal variant of Section 2.2 (alpha = 1/||Gamma_r||:
// Ct = C = Q), projects in FP32 against an FP32 copy of Q, and re-decides every row whose
// FP32 relative rejection exceeds the floor tau_lo in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <stdint.h>

#include "rg_core.cuh"

namespace rg {

template <bool F32, bool ORTHO>
__global__ void __launch_bounds__(NT, 1) stream_kernel(StreamDev S, CallArgs A) {
  grid_barrier_init(S.ctrl);
  process_rows<GridTeam, F32, ORTHO>(GridTeam{S.ctrl}, S, A);
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

// Host-side launch helpers (declared in rg_host.h).
// FP32 projections always come with the orthonormal variant.
static const void* stream_kernel_ptr(int mixed, int ortho) {
  if (mixed) return (const void*)stream_kernel<true, true>;
  return ortho ? (const void*)stream_kernel<false, true> : (const void*)stream_kernel<false, false>;
}

cudaError_t launch_stream(const StreamDev& S, const double* Gamma, const double* y, long long k,
                          uint8_t* indep, int grid, cudaStream_t stream) {
  CallArgs A{Gamma, y, k, indep};
  StreamDev Sc = S;
  void* args[] = {(void*)&Sc, (void*)&A};
  return cudaLaunchCooperativeKernel(stream_kernel_ptr(S.mixed, S.ortho), dim3(grid), dim3(NT),
                                     args, 0, stream);
}

cudaError_t stream_grid_size(int mixed, int ortho, int* grid) {
  int dev = 0, nsm = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, stream_kernel_ptr(mixed, ortho), NT, 0);
  if (e != cudaSuccess) return e;
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
