// rg_noalloc.cu -- rg_solve_noalloc: solve one stream from scratch without allocating.
//
// Some callers cannot call cudaMalloc: a latency-critical loop where cudaMalloc's implicit
// device synchronisation is not acceptable, or a host application whose device memory is
// owned entirely by its own allocator. This entry point runs the same cooperative
// single-stream kernel as rg_add_rows, but its state and scratch live in one fixed,
// file-scope device array (RG_NOALLOC_BYTES) that every GPU loading the library holds
// until the process exits. The caller passes the rows, the targets and the output X.
//
// The array is shared by every call: each call first clears the control words the kernel
// needs zeroed, and calls that overlap on the GPU (other streams, other host threads)
// race on it. The host-side address of the array comes from cudaGetSymbolAddress, taken
// once per device with that device current; the first call on a device does this set-up,
// so that first call should come before any stream capture.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/rg.h"
#include "rg_core.cuh"
#include "rg_host.h"

#define RG_NOALLOC_BYTES (8u << 20)

namespace rg {

static __device__ __align__(256) unsigned char g_noalloc_scratch[RG_NOALLOC_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};
int g_noalloc_grid[kMaxDevices] = {};

size_t al(size_t x) { return (x + 255) / 256 * 256; }

// Lays the state and scratch of one stream out in the fixed array (base may be null to
// measure). Returns the bytes needed.
size_t noalloc_layout(StreamDev& S, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off = al(off + bytes);
    return p;
  };
  const size_t ld = (size_t)S.ld, rm = (size_t)S.r_max, kb = (size_t)S.kb_max;
  S.C = (double*)take(rm * ld * 8);
  S.Ct = S.ortho ? nullptr : (double*)take(rm * ld * 8);
  S.Qf = S.mixed ? (float*)take(rm * ld * 4) : nullptr;
  S.Pinv = nullptr;
  S.P = (double*)take(rm * rm * 8);
  S.wb = (double*)take(rm * 8);
  S.u = (double*)take(rm * 8);
  S.w = (double*)take(rm * 8);
  S.basis_rows = (long long*)take(rm * 8);
  S.rows_seen = (long long*)take(8);
  S.ctrl = (int*)take(CTRL_N * 4);
  S.G = (double*)take(kb * rm * 8);
  S.spart = (double*)take(kb * (size_t)S.nmc * 8);
  S.tpart = (double*)take(kb * (size_t)S.nmc * 8);
  S.s = (double*)take(kb * 8);
  S.t = (double*)take(kb * 8);
  S.rowflag = (uint8_t*)take(kb);
  S.R = (double*)take((size_t)SLOW_MAX * ld * 8);
  S.Kv = (double*)take((size_t)SLOW_MAX * ld * 8);
  S.Gind = (double*)take((size_t)SLOW_MAX * rm * 8);
  S.alpha = (double*)take(SLOW_MAX * 8);
  S.jind = (int*)take(SLOW_MAX * 4);
  S.Dall = (double*)take(kb * 8);
  S.Lw = (double*)take(rm * rm * 8);
  S.Kap = (double*)take((size_t)SLOW_MAX * SLOW_MAX * 8);
  S.Rs = nullptr;
  S.rs_cap = 0;
  S.sp_stride = (size_t)32 * std::min<size_t>((ld + 31) / 32, 1024);  // <= 1024 workers
  S.Sp = (double*)take(2 * S.sp_stride * 8);
  S.Pp = nullptr;  // no chunked partial sums here: long runs accumulate directly
  S.pp_cap = 0;
  S.up = nullptr;
  return off;
}

}  // namespace

template <bool F32, int VAR>
__global__ void __launch_bounds__(NT, 1) noalloc_kernel(StreamDev S, CallArgs A) {
  grid_barrier_init(S.ctrl);
  process_rows<GridTeam, F32, VAR>(GridTeam{S.ctrl}, S, A);
}

// FP32 projections always come with the orthonormal variant. v: 0 general, 1 orthonormal
// (FP64), 2 mixed, 3 orthogonal.
static const void* noalloc_kernel_ptr(int v) {
  if (v == 2) return (const void*)noalloc_kernel<true, VAR_ORTHONORMAL>;
  if (v == 1) return (const void*)noalloc_kernel<false, VAR_ORTHONORMAL>;
  if (v == 3) return (const void*)noalloc_kernel<false, VAR_ORTHOGONAL>;
  return (const void*)noalloc_kernel<false, VAR_GENERAL>;
}

// Clears what must start at zero before each call: the control words (rank, status,
// grid-barrier counter and generation, block plan) and the row counter.
__global__ void noalloc_reset_kernel(int* ctrl, long long* rows_seen, int kb0) {
  for (int i = threadIdx.x; i < CTRL_N; i += blockDim.x) ctrl[i] = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    ctrl[CTRL_KB] = kb0;
    *rows_seen = 0;
  }
}

// One CTA: w = w_b + P^-1 u, then X = Ct^T w (or Q^T w).
__global__ void __launch_bounds__(NT, 1) noalloc_solution_kernel(StreamDev S, double* X) {
  const int r = S.ctrl[CTRL_R];
  form_w(S, r);
  const double* B = S.ortho ? S.C : S.Ct;
  for (int c = threadIdx.x; c < S.m; c += NT) {
    double acc = 0.0;
    for (int i = 0; i < r; ++i) acc = fma(__ldcg(B + (size_t)i * S.ld + c), __ldcg(S.w + i), acc);
    X[c] = acc;
  }
}

}  // namespace rg

using namespace rg;

extern "C" rg_status rg_solve_noalloc(const double* Gamma, const double* y, int64_t n, int64_t m,
                                      double tol, int flags, int64_t r_max, double* X,
                                      int64_t* rank_out, void* cuda_stream) {
  NvtxRange nvtx_range("rg_solve_noalloc");
  if (m <= 0 || m > (1 << 24)) return fail(RG_EINVAL, "rg_solve_noalloc: m = %lld out of range", (long long)m);
  if (n < 0) return fail(RG_EINVAL, "rg_solve_noalloc: n = %lld < 0", (long long)n);
  if ((n > 0 && (!Gamma || !y)) || !X) return fail(RG_EINVAL, "rg_solve_noalloc: NULL buffer");
  if (std::isnan(tol)) return fail(RG_EINVAL, "rg_solve_noalloc: tol is NaN");
  if (flags & ~(RG_MIXED | RG_TEST_PAPER | RG_ORTHONORMAL | RG_ORTHOGONAL))
    return fail(RG_EINVAL, "rg_solve_noalloc: unknown flags %d", flags);
  if ((flags & RG_ORTHOGONAL) && (flags & (RG_MIXED | RG_ORTHONORMAL)))
    return fail(RG_EINVAL, "rg_solve_noalloc: RG_ORTHOGONAL excludes RG_MIXED and RG_ORTHONORMAL");
  if (r_max <= 0 || r_max > m) r_max = m;
  StreamDev S{};
  S.m = (int)m;
  S.ld = (int)((m + 3) / 4 * 4);
  S.r_max = (int)r_max;
  S.mixed = (flags & RG_MIXED) ? 1 : 0;
  S.ortho = (flags & (RG_MIXED | RG_ORTHONORMAL)) ? 1 : 0;
  S.orthog = (flags & RG_ORTHOGONAL) ? 1 : 0;
  S.test_mode = (flags & RG_TEST_PAPER) ? 2 : 0;
  S.tol = tol;
  S.tau_lo = 1e-5;
  S.nmc = (int)((m + MC - 1) / MC);
  // the largest internal block (power of two, 32..1024) whose layout fits the array
  size_t need = 0;
  int kb = 1024;
  for (; kb >= 32; kb /= 2) {
    S.kb_max = kb;
    need = noalloc_layout(S, nullptr);
    if (need <= RG_NOALLOC_BYTES) break;
  }
  if (kb < 32)
    return fail(RG_EINVAL,
                "rg_solve_noalloc: m = %lld with r_max = %lld needs %zu bytes of state and "
                "scratch at the smallest block size; the fixed maximum is %u bytes (lower r_max "
                "or use rg_init)", (long long)m, (long long)r_max, need, (unsigned)RG_NOALLOC_BYTES);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "rg_solve_noalloc: no CUDA device");
  if (dev < 0 || dev >= 64) return fail(RG_EINVAL, "rg_solve_noalloc: device ordinal %d unsupported", dev);
  void* base = nullptr;
  int grid = 0;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {  // once per device, with that device current
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "rg_solve_noalloc: cudaGetSymbolAddress");
      int nsm = 0, per[4] = {0, 0, 0, 0};
      e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      for (int v = 0; v < 4 && e == cudaSuccess; ++v)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per[v], noalloc_kernel_ptr(v), NT, 0);
      if (e != cudaSuccess) return cuda_fail(e, "rg_solve_noalloc: occupancy query");
      if (per[0] < 1 || per[1] < 1 || per[2] < 1 || per[3] < 1)
        return fail(RG_ECUDA, "rg_solve_noalloc: kernel cannot be resident");
      g_noalloc_grid[dev] = std::min(nsm, 1024);
      g_noalloc_ptr[dev] = p;
    }
    base = g_noalloc_ptr[dev];
    grid = g_noalloc_grid[dev];
  }
  noalloc_layout(S, (char*)base);
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  noalloc_reset_kernel<<<1, 32, 0, stream>>>(S.ctrl, S.rows_seen, std::min(KB_MIN, S.kb_max));
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "rg_solve_noalloc: reset launch");
  if (n > 0) {
    CallArgs A{Gamma, y, n, nullptr};
    void* args[] = {(void*)&S, (void*)&A};
    const int v = S.mixed ? 2 : (S.ortho ? 1 : (S.orthog ? 3 : 0));
    e = cudaLaunchCooperativeKernel(noalloc_kernel_ptr(v), dim3(grid), dim3(NT), args, 0,
                                    stream);
    if (e != cudaSuccess) return cuda_fail(e, "rg_solve_noalloc: launch");
  }
  noalloc_solution_kernel<<<1, NT, 0, stream>>>(S, X);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "rg_solve_noalloc: solution launch");
  if (rank_out) {
    int ctl[2] = {0, 0};
    e = cudaMemcpyAsync(ctl, S.ctrl, 2 * sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "rg_solve_noalloc: reading the result");
    *rank_out = ctl[CTRL_R];
    return status_from_bits(ctl[CTRL_STATUS]);
  }
  return RG_OK;
}
