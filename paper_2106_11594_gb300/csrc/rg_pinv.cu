// rg_pinv.cu -- rg_pinv: the pseudoinverse A_n^+ of the rows a stream has taken, formed from
// the stream's current factorization.
//
// Theorems label_th_pinv_indep and label_th_pinv_lindep update A^+ one row at a time
// (A^+ <- [A^+ - K b^T, K], an O(mn) outer product per row). On the GPU the same matrix is
// formed after any call from the factorization the least-squares path already keeps
// (Section 2.1): A^+ = D^T P^-1 B^T with D the dual basis Ct (general variant) or Q
// (orthonormal variant) and B = A D^T, since A = B C and A^+ = Ct^T P^-1 B^T. In order:
//
//   1. flush the deferred P/u update, factor P and form P^-1 (export_prep_kernel);
//   2. F = D^T P^-1                       (m x r, 2 m r^2 flop)
//   3. B = A D^T                          (n x r, 2 n m r flop)   -- dgemm_nt
//   4. A^+ = F B^T                        (m x n, 2 m n r flop)   -- dgemm_nt
//
// 4 m n r flop in FP64 for the whole matrix instead of 2 m n per row for n rows: cheaper
// whenever more than 2r rows arrive between two requests, and with no sequential
// dependency between rows. Every step is FP64 on the CUDA cores (the FP64 tensor rate of
// this part is far below its FP64 FMA rate).
#include <cuda_runtime.h>
#include <stdint.h>

#include "rg_core.cuh"
#include "rg_host.h"

namespace rg {

// F[c][l] = sum_k D[k][c] Pinv[k][l]  (thread = (c, l); D rows are ld apart).
__global__ void pinv_f_kernel(const double* D, int ld, const double* Pinv, int rm, int m, int r,
                              double* F) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)m * r) return;
  const int l = (int)(e / m), c = (int)(e - (long long)l * m);
  double acc = 0.0;
  for (int k = 0; k < r; ++k) acc = fma(__ldg(D + (size_t)k * ld + c), __ldg(Pinv + (size_t)k * rm + l), acc);
  F[(size_t)c * r + l] = acc;
}

// C (M x N, row-major, ldc) = A (M x K, lda) * B (N x K, ldb)^T in FP64; K is the contiguous
// index of both operands. 64 x 64 tiles over 256 threads (a 4 x 4 register tile each, rows
// ty + 16 i and columns tx + 16 j so that a warp's shared-memory reads are conflict-free),
// K in slices of 16 staged through shared memory. FP64 FMA bound: per slice a CTA does
// 65536 FMAs against 16 KiB of operand loads.
constexpr int GB = 64, GK = 16;
__global__ void __launch_bounds__(256, 2) dgemm_nt(const double* __restrict__ A, long long lda,
                                                   const double* __restrict__ B, long long ldb,
                                                   double* __restrict__ C, long long ldc, long long M,
                                                   long long N, int K) {
  __shared__ double As[GK][GB + 1];
  __shared__ double Bs[GK][GB + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const long long tiles_n = (N + GB - 1) / GB;  // one-dimensional grid: tile (ti, tj)
  const long long i0 = (long long)(blockIdx.x / tiles_n) * GB, j0 = (long long)(blockIdx.x % tiles_n) * GB;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  // loader: 1024 elements per operand tile, 4 per thread; kk fastest (128-byte row pieces)
  const int lk = tid & 15, lr = tid >> 4;  // lr in 0..15, rows lr + 16 q
  for (int k0 = 0; k0 < K; k0 += GK) {
    const int kk = k0 + lk;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long ia = i0 + lr + 16 * q, jb = j0 + lr + 16 * q;
      As[lk][lr + 16 * q] = (ia < M && kk < K) ? __ldg(A + ia * lda + kk) : 0.0;
      Bs[lk][lr + 16 * q] = (jb < N && kk < K) ? __ldg(B + jb * ldb + kk) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GK; ++k) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[k][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const long long i = i0 + ty + 16 * a;
    if (i >= M) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const long long j = j0 + tx + 16 * b;
      if (j < N) C[i * ldc + j] = acc[a][b];
    }
  }
}

static cudaError_t launch_dgemm_nt(const double* A, long long lda, const double* B, long long ldb,
                                   double* C, long long ldc, long long M, long long N, int K,
                                   cudaStream_t stream) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const long long tiles = ((N + GB - 1) / GB) * ((M + GB - 1) / GB);
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  dgemm_nt<<<(unsigned)tiles, 256, 0, stream>>>(A, lda, B, ldb, C, ldc, M, N, K);
  return cudaGetLastError();
}

// Steps 2-4 (the caller has flushed the deferred update and formed P^-1 with
// export_prep_kernel). wk holds (m + n) r doubles.
cudaError_t launch_pinv(const StreamDev& S, const double* A, long long n, double* Apinv, long long ld,
                        int r, double* wk, cudaStream_t stream) {
  const long long m = S.m;
  double* F = wk;                   // m x r
  double* Bm = wk + (size_t)m * r;  // n x r
  const double* D = S.ortho ? S.C : S.Ct;
  cudaError_t e = cudaSuccess;
  if (r > 0) {
    const long long items = m * r;
    pinv_f_kernel<<<(unsigned)((items + NT - 1) / NT), NT, 0, stream>>>(D, S.ld, S.Pinv, S.r_max, (int)m, r, F);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_dgemm_nt(A, m, D, S.ld, Bm, r, n, r, (int)m, stream);
  }
  if (e == cudaSuccess) e = launch_dgemm_nt(F, r, Bm, r, Apinv, ld, m, n, r, stream);
  return e;
}

}  // namespace rg
