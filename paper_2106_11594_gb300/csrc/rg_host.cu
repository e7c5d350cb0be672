// rg_host.cu -- host side of the C ABI declared in include/rg.h (single streams).
//
// Owns the device memory of a stream, validates arguments before anything is enqueued,
// launches the kernels of rg_stream.cu on the state's stream and maps the device status
// word to rg_status. There is no CPU fallback: every path runs the CUDA kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/rg.h"
#include "rg_adjoint.cuh"
#include "rg_host.h"
#include "rg_internal.cuh"

namespace rg {
thread_local std::string g_last_error;

rg_status fail(rg_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

rg_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear the sticky-free error so later calls start clean
  return fail(e == cudaErrorMemoryAllocation ? RG_ENOMEM : RG_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

rg_status status_from_bits(int bits) {
  if (bits & ST_TIMEOUT)
    return fail(RG_ETIMEOUT, "a bounded device-side wait gave up; reset the state");
  if (bits & ST_BADARG) return fail(RG_EINVAL, "inconsistent offsets found on the device");
  if (bits & ST_NONFINITE)
    return fail(RG_ENONFINITE, "a row or target was not finite (or a numerical breakdown "
                               "made a Woodbury denominator non-positive); the rows from it "
                               "on were not applied");
  if (bits & ST_CAPACITY)
    return fail(RG_ECAPACITY, "an independent row arrived at rank == r_max; the rows from it "
                              "on were not applied");
  return RG_OK;
}

__global__ void reset_kernel(int* ctrl, long long* rows_seen, int kb0) {
  for (int i = threadIdx.x; i < CTRL_N; i += blockDim.x) ctrl[i] = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    ctrl[CTRL_KB] = kb0;
    *rows_seen = 0;
  }
}

// Keeps the timeout bit (the state stays unusable until reset), clears the others.
__global__ void clear_status_kernel(int* ctrl) {
  ctrl[CTRL_STATUS] &= ST_TIMEOUT;
}

}  // namespace rg

using namespace rg;

struct rg_state {
  int device = 0;
  cudaStream_t stream = nullptr;
  StreamDev S{};
  int grid = 0;
  void* arena = nullptr;  // one device allocation for everything
  size_t arena_bytes = 0;
  // staging for the host-buffer entry points (allocated on first use)
  double* stage = nullptr;  // two slots of stage_rows rows (and targets) each
  uint8_t* stage_ind = nullptr;
  cudaStream_t copy_stream = nullptr;  // host-to-device copies of the host entry point
  cudaEvent_t copied[2] = {nullptr, nullptr};    // slot s holds the rows of its latest copy
  cudaEvent_t consumed[2] = {nullptr, nullptr};  // the call that read slot s has finished
  int slot = 0;
  long long stage_rows = 0;
  double* xbuf = nullptr;
  // two small (SMALL_B-row) gamma / a-priori-error buffers used alternately by calls of at
  // most SMALL_B rows, so that one call's deferred P/u update survives into the next
  double* Gs[2] = {nullptr, nullptr};
  double* Ds[2] = {nullptr, nullptr};
  int last_small = 1;  // buffer of the most recent small call
};

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Carver {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t n) {
    off = align_up(off, 256);
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += n * sizeof(T);
    return p;
  }
};

// Lays out every device buffer of a stream; with base == nullptr it only measures.
size_t carve(StreamDev& S, char* base, double** gs = nullptr, double** ds = nullptr) {
  Carver cv{base};
  const size_t ld = (size_t)S.ld, rm = (size_t)S.r_max, kb = (size_t)S.kb_max;
  S.C = cv.take<double>(rm * ld);
  S.Ct = S.ortho ? nullptr : cv.take<double>(rm * ld);
  S.Qf = S.mixed ? cv.take<float>(rm * ld) : nullptr;
  S.Pinv = cv.take<double>(rm * rm);
  S.P = cv.take<double>(rm * rm);
  S.wb = cv.take<double>(rm);
  S.u = cv.take<double>(rm);
  S.w = cv.take<double>(rm);
  S.basis_rows = cv.take<long long>(rm);
  S.rows_seen = cv.take<long long>(1);
  S.ctrl = cv.take<int>(CTRL_N);
  S.G = cv.take<double>(kb * rm);
  S.spart = cv.take<double>(kb * (size_t)S.nmc);
  S.tpart = cv.take<double>(kb * (size_t)S.nmc);
  S.s = cv.take<double>(kb);
  S.t = cv.take<double>(kb);
  S.rowflag = cv.take<uint8_t>(kb);
  S.R = cv.take<double>((size_t)SLOW_MAX * ld);
  S.Kv = cv.take<double>((size_t)SLOW_MAX * ld);
  S.Gind = cv.take<double>((size_t)SLOW_MAX * rm);
  S.alpha = cv.take<double>(SLOW_MAX);
  S.jind = cv.take<int>(SLOW_MAX);
  S.Dall = cv.take<double>(kb);
  S.Pp = cv.take<double>(S.pp_cap);
  S.up = cv.take<double>((size_t)NCH_MAX * rm);
  S.Lw = cv.take<double>(rm * rm);
  S.Kap = cv.take<double>((size_t)SLOW_MAX * SLOW_MAX);
  S.Rs = nullptr;
  S.rs_cap = 0;
  S.sp_stride = (size_t)32 * std::min<size_t>((ld + 31) / 32, 1024);  // <= 1024 workers
  S.Sp = cv.take<double>(2 * S.sp_stride);
  for (int h = 0; h < 2; ++h) {
    double* g = cv.take<double>((size_t)SMALL_B * rm);
    double* d = cv.take<double>((size_t)SMALL_B);
    if (gs) gs[h] = g;
    if (ds) ds[h] = d;
  }
  return align_up(cv.off, 256);
}

bool valid_state(rg_state* st) { return st != nullptr && st->arena != nullptr; }

// The state as one rg_add_rows call of k rows sees it: calls of at most SMALL_B rows use
// the two small buffers alternately (and may defer their P/u update), larger calls the
// main block scratch; both fold a pending update left by the previous small call.
StreamDev call_view(rg_state* st, long long k) {
  StreamDev S = st->S;
  if (k <= SMALL_B) {
    const int h = 1 - st->last_small;
    S.G = st->Gs[h];
    S.Dall = st->Ds[h];
    S.Gpend = st->Gs[1 - h];
    S.Dpend = st->Ds[1 - h];
    S.defer = 1;
    st->last_small = h;
  } else {
    S.Gpend = st->Gs[st->last_small];
    S.Dpend = st->Ds[st->last_small];
    S.defer = 0;
  }
  return S;
}

// The view for rg_solution / rg_export / rg_adjoint: pending rows of the last small call.
StreamDev flush_view(rg_state* st) {
  StreamDev S = st->S;
  S.Gpend = st->Gs[st->last_small];
  S.Dpend = st->Ds[st->last_small];
  S.defer = 0;
  return S;
}

rg_status pending_status(rg_state* st, bool clear) {
  int bits = 0;
  cudaError_t e = cudaMemcpyAsync(&bits, st->S.ctrl + CTRL_STATUS, sizeof(int),
                                  cudaMemcpyDeviceToHost, st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading the device status");
  if (bits && clear) {
    clear_status_kernel<<<1, 1, 0, st->stream>>>(st->S.ctrl);
    cudaError_t e2 = cudaGetLastError();
    if (e2 != cudaSuccess) return cuda_fail(e2, "clearing the device status");
  }
  return status_from_bits(bits);
}

}  // namespace

extern "C" {

const char* rg_last_error(void) { return g_last_error.c_str(); }

const char* rg_version(void) { return "rank-greville-gb300 0.1 (sm_103a)"; }

rg_status rg_init(rg_state** out, int64_t m, double tol, int flags, int64_t r_max,
                  void* cuda_stream) {
  if (!out) return fail(RG_EINVAL, "rg_init: out is NULL");
  *out = nullptr;
  if (m <= 0 || m > (1 << 24)) return fail(RG_EINVAL, "rg_init: m = %lld out of range", (long long)m);
  if (std::isnan(tol)) return fail(RG_EINVAL, "rg_init: tol is NaN");
  if (flags & ~(RG_MIXED | RG_TEST_PAPER | RG_ORTHONORMAL | RG_ORTHOGONAL))
    return fail(RG_EINVAL, "rg_init: unknown flags %d", flags);
  if ((flags & RG_ORTHOGONAL) && (flags & (RG_MIXED | RG_ORTHONORMAL)))
    return fail(RG_EINVAL, "rg_init: RG_ORTHOGONAL excludes RG_MIXED and RG_ORTHONORMAL");
  if (r_max <= 0 || r_max > m) r_max = m;
  rg_state* st = new (std::nothrow) rg_state();
  if (!st) return fail(RG_ENOMEM, "rg_init: host allocation failed");
  cudaError_t e = cudaGetDevice(&st->device);
  if (e != cudaSuccess) {
    delete st;
    return cuda_fail(e, "rg_init: no CUDA device");
  }
  st->stream = (cudaStream_t)cuda_stream;
  StreamDev& S = st->S;
  S.m = (int)m;
  S.ld = (int)align_up((size_t)m, 4);
  S.r_max = (int)r_max;
  S.mixed = (flags & RG_MIXED) ? 1 : 0;
  S.ortho = (flags & (RG_MIXED | RG_ORTHONORMAL)) ? 1 : 0;
  S.orthog = (flags & RG_ORTHOGONAL) ? 1 : 0;
  S.test_mode = (flags & RG_TEST_PAPER) ? 2 : 0;
  S.tol = tol;
  S.tau_lo = 1e-5;
  S.nmc = (int)((m + MC - 1) / MC);
  // internal block: large enough to fill the GPU (mixed mode: to give every SM tensor-core
  // chunks), bounded so the scratch stays small
  long long kb = S.mixed ? 32768 : 4096;
  while (kb > 256 && (double)kb * (double)r_max * 8.0 > 256.0 * (1 << 20)) kb /= 2;
  S.kb_max = (int)kb;
  {  // Gram-path partials: at least one chunk at full rank, up to NCH_MAX, <= 128 MiB
    const size_t rr = (size_t)r_max * (size_t)r_max;
    S.pp_cap = std::max(rr, std::min(rr * NCH_MAX, (size_t)16 << 20));
  }
  st->arena_bytes = carve(S, nullptr);
  e = cudaMalloc(&st->arena, st->arena_bytes);
  if (e != cudaSuccess) {
    delete st;
    return cuda_fail(e, "rg_init: cudaMalloc of the state");
  }
  carve(S, (char*)st->arena, st->Gs, st->Ds);
  e = stream_grid_size(S.mixed, S.ortho, S.orthog, &st->grid);
  if (e != cudaSuccess || st->grid <= 0) {
    cudaFree(st->arena);
    delete st;
    return e != cudaSuccess ? cuda_fail(e, "rg_init: occupancy query")
                            : fail(RG_ECUDA, "rg_init: kernel cannot be made resident");
  }
  e = cudaMemsetAsync(st->arena, 0, st->arena_bytes, st->stream);
  if (e == cudaSuccess) {
    reset_kernel<<<1, 32, 0, st->stream>>>(S.ctrl, S.rows_seen, std::min(KB_MIN, S.kb_max));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaFree(st->arena);
    delete st;
    return cuda_fail(e, "rg_init: initialising the state");
  }
  *out = st;
  return RG_OK;
}

rg_status rg_add_rows(rg_state* st, const double* Gamma, const double* y, int64_t k,
                      uint8_t* indep_out) {
  NvtxRange nvtx_range("rg_add_rows");
  if (!valid_state(st)) return fail(RG_EINVAL, "rg_add_rows: invalid state");
  if (k < 0) return fail(RG_EINVAL, "rg_add_rows: k = %lld < 0", (long long)k);
  if (k == 0) return RG_OK;
  if (!Gamma || !y) return fail(RG_EINVAL, "rg_add_rows: NULL rows or targets");
  cudaError_t e = cudaSuccess;
  if (indep_out) e = cudaMemsetAsync(indep_out, 0xFF, (size_t)k, st->stream);
  if (e == cudaSuccess) e = launch_stream(call_view(st, k), Gamma, y, k, indep_out, st->grid, st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_add_rows: launch");
  return RG_OK;
}

rg_status rg_add_rows_host(rg_state* st, const double* Gamma, const double* y, int64_t k,
                           uint8_t* indep_out) {
  NvtxRange nvtx_range("rg_add_rows_host");
  if (!valid_state(st)) return fail(RG_EINVAL, "rg_add_rows_host: invalid state");
  if (k < 0) return fail(RG_EINVAL, "rg_add_rows_host: k = %lld < 0", (long long)k);
  if (k == 0) return RG_OK;
  if (!Gamma || !y) return fail(RG_EINVAL, "rg_add_rows_host: NULL rows or targets");
  const long long m = st->S.m;
  if (st->stage_rows == 0) {  // first use: all of the staging resources, or none
    long long rows = std::max<long long>(1, (32ll << 20) / (8 * (m + 1)));
    cudaError_t e = cudaSuccess;
    if (!st->stage) e = cudaMalloc(&st->stage, 2 * (size_t)rows * (size_t)(m + 1) * 8);
    if (e == cudaSuccess && !st->stage_ind) e = cudaMalloc(&st->stage_ind, (size_t)rows);
    if (e == cudaSuccess && !st->copy_stream)
      e = cudaStreamCreateWithFlags(&st->copy_stream, cudaStreamNonBlocking);
    for (int h = 0; h < 2 && e == cudaSuccess; ++h) {
      if (!st->copied[h]) e = cudaEventCreateWithFlags(&st->copied[h], cudaEventDisableTiming);
      if (e == cudaSuccess && !st->consumed[h])
        e = cudaEventCreateWithFlags(&st->consumed[h], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(st->consumed[h], st->stream);
    }
    // on failure what was created stays owned by the state (rg_free releases it) and the
    // next call retries the rest
    if (e != cudaSuccess) return cuda_fail(e, "rg_add_rows_host: staging allocation");
    st->stage_rows = rows;
  }
  // Two staging slots: the rows of one chunk are copied on the copy stream while the
  // previous chunk's (or call's) update runs on the state's stream; a slot is refilled
  // only after the update that read it has finished. The call returns once its last copy
  // is done (the host buffers may then be reused); the update itself is asynchronous
  // unless indep_out is requested.
  cudaError_t e = cudaSuccess;
  int last = -1;
  for (long long c0 = 0; c0 < k; c0 += st->stage_rows) {
    const long long n = std::min(st->stage_rows, (long long)k - c0);
    const int h = st->slot;
    st->slot ^= 1;
    double* dG = st->stage + (size_t)h * st->stage_rows * (size_t)(m + 1);
    double* dy = dG + (size_t)st->stage_rows * (size_t)m;
    e = cudaStreamWaitEvent(st->copy_stream, st->consumed[h], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dG, Gamma + (size_t)c0 * m, (size_t)n * m * 8, cudaMemcpyHostToDevice, st->copy_stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dy, y + c0, (size_t)n * 8, cudaMemcpyHostToDevice, st->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(st->copied[h], st->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st->stream, st->copied[h], 0);
    if (e != cudaSuccess) return cuda_fail(e, "rg_add_rows_host: copy to device");
    rg_status s = rg_add_rows(st, dG, dy, n, indep_out ? st->stage_ind : nullptr);
    if (s != RG_OK) return s;
    e = cudaEventRecord(st->consumed[h], st->stream);
    if (e == cudaSuccess && indep_out) {
      e = cudaMemcpyAsync(indep_out + c0, st->stage_ind, (size_t)n, cudaMemcpyDeviceToHost, st->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);  // stage_ind is reused
    }
    if (e != cudaSuccess) return cuda_fail(e, "rg_add_rows_host: copy to host");
    last = h;
  }
  if (last >= 0) e = cudaEventSynchronize(st->copied[last]);
  if (e != cudaSuccess) return cuda_fail(e, "rg_add_rows_host: synchronise");
  return RG_OK;
}

rg_status rg_solution(rg_state* st, double* X, int64_t* rank_out) {
  NvtxRange nvtx_range("rg_solution");
  if (!valid_state(st)) return fail(RG_EINVAL, "rg_solution: invalid state");
  if (!X) return fail(RG_EINVAL, "rg_solution: X is NULL");
  cudaError_t e = launch_flush(flush_view(st), st->grid, st->stream);
  if (e == cudaSuccess) e = launch_solution(st->S, X, st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_solution: launch");
  if (rank_out) return rg_rank(st, rank_out);
  return RG_OK;
}

rg_status rg_adjoint(rg_state* st, const double* A, const double* y, int64_t n, const double* g,
                     double* gA, double* gy, double* X) {
  NvtxRange nvtx_range("rg_adjoint");
  if (!valid_state(st)) return fail(RG_EINVAL, "rg_adjoint: invalid state");
  if (n < 0) return fail(RG_EINVAL, "rg_adjoint: n = %lld < 0", (long long)n);
  if (!g || (n > 0 && (!A || !y || !gA || !gy)))
    return fail(RG_EINVAL, "rg_adjoint: NULL buffer");
  const StreamDev& S = st->S;
  const long long m = S.m, rm = S.r_max;
  const int nrc = (int)std::max<long long>(1, std::min<long long>(
      (n + 255) / 256, std::max<long long>(1, 4LL * st->grid / ((m + NT - 1) / NT))));
  // scratch: X, A^+ h, g_perp, A^T h (m each), seven r_max vectors, h, z, rho (n each),
  // row-chunk partials (nrc x m)
  const size_t doubles = (size_t)4 * m + 7 * (size_t)rm + 3 * (size_t)std::max<int64_t>(n, 1) + (size_t)nrc * m;
  double* wk = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&wk, doubles * sizeof(double), st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_adjoint: workspace");
  AdjArgs J{};
  J.A = A;
  J.y = y;
  J.n = n;
  J.g = g;
  J.gA = gA;
  J.gy = gy;
  double* p = wk;
  J.X = p; p += m;
  J.Aph = p; p += m;
  J.gperp = p; p += m;
  J.v = p; p += m;
  J.a = p; p += rm;
  J.c = p; p += rm;
  J.e = p; p += rm;
  J.al = p; p += rm;
  J.be = p; p += rm;
  J.bth = p; p += rm;
  J.de = p; p += rm;
  J.h = p; p += std::max<int64_t>(n, 1);
  J.z = p; p += std::max<int64_t>(n, 1);
  J.rho = p; p += std::max<int64_t>(n, 1);
  J.part = p;
  J.nrc = nrc;
  e = launch_flush(flush_view(st), st->grid, st->stream);
  if (e == cudaSuccess) e = launch_solution(S, J.X, st->stream);  // w and the Cholesky factor of P
  if (e == cudaSuccess) e = launch_adjoint(S, J, st->grid, st->stream);
  if (e == cudaSuccess && X) e = cudaMemcpyAsync(X, J.X, m * sizeof(double), cudaMemcpyDeviceToDevice, st->stream);
  const cudaError_t e2 = cudaFreeAsync(wk, st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_adjoint: launch");
  if (e2 != cudaSuccess) return cuda_fail(e2, "rg_adjoint: workspace release");
  return RG_OK;
}

rg_status rg_pinv(rg_state* st, const double* A, int64_t n, double* Apinv, int64_t ld) {
  NvtxRange nvtx_range("rg_pinv");
  if (!valid_state(st)) return fail(RG_EINVAL, "rg_pinv: invalid state");
  if (n < 0) return fail(RG_EINVAL, "rg_pinv: n = %lld < 0", (long long)n);
  if (n > 0 && (!A || !Apinv)) return fail(RG_EINVAL, "rg_pinv: NULL buffer");
  if (ld < n) return fail(RG_EINVAL, "rg_pinv: ld = %lld < n = %lld", (long long)ld, (long long)n);
  int64_t r = 0;
  rg_status s = rg_rank(st, &r);  // synchronises; a stream stopped by an error keeps a valid state
  if (s != RG_OK && s != RG_ECAPACITY && s != RG_ENONFINITE) return s;
  if (r > GRAM_RMAX) return fail(RG_EINVAL, "rg_pinv: rank %lld above %d", (long long)r, GRAM_RMAX);
  if (n == 0) return RG_OK;
  const size_t doubles = (size_t)std::max<long long>(1, ((long long)st->S.m + n) * r);
  double* wk = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&wk, doubles * sizeof(double), st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_pinv: workspace");
  e = launch_flush(flush_view(st), st->grid, st->stream);
  if (e == cudaSuccess) e = launch_export_prep(st->S, st->grid, st->stream);  // P^-1 from P
  if (e == cudaSuccess) e = launch_pinv(st->S, A, n, Apinv, ld, (int)r, wk, st->stream);
  const cudaError_t e2 = cudaFreeAsync(wk, st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_pinv: launch");
  if (e2 != cudaSuccess) return cuda_fail(e2, "rg_pinv: workspace release");
  return RG_OK;
}

rg_status rg_solution_host(rg_state* st, double* X, int64_t* rank_out) {
  NvtxRange nvtx_range("rg_solution_host");
  if (!valid_state(st)) return fail(RG_EINVAL, "rg_solution_host: invalid state");
  if (!X) return fail(RG_EINVAL, "rg_solution_host: X is NULL");
  if (!st->xbuf) {
    cudaError_t e = cudaMalloc(&st->xbuf, (size_t)st->S.m * 8);
    if (e != cudaSuccess) return cuda_fail(e, "rg_solution_host: allocation");
  }
  cudaError_t e = launch_flush(flush_view(st), st->grid, st->stream);
  if (e == cudaSuccess) e = launch_solution(st->S, st->xbuf, st->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(X, st->xbuf, (size_t)st->S.m * 8, cudaMemcpyDeviceToHost, st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_solution_host");
  if (rank_out) return rg_rank(st, rank_out);
  e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_solution_host: synchronise");
  return pending_status(st, true);
}

rg_status rg_rank(rg_state* st, int64_t* rank_out) {
  if (!valid_state(st) || !rank_out) return fail(RG_EINVAL, "rg_rank: invalid argument");
  int r = 0;
  cudaError_t e = cudaMemcpyAsync(&r, st->S.ctrl + CTRL_R, sizeof(int), cudaMemcpyDeviceToHost,
                                  st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_rank");
  *rank_out = r;
  return pending_status(st, true);
}

rg_status rg_rows_seen(rg_state* st, int64_t* rows_out) {
  if (!valid_state(st) || !rows_out) return fail(RG_EINVAL, "rg_rows_seen: invalid argument");
  long long n = 0;
  cudaError_t e = cudaMemcpyAsync(&n, st->S.rows_seen, sizeof(long long),
                                  cudaMemcpyDeviceToHost, st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_rows_seen");
  *rows_out = n;
  return RG_OK;
}

rg_status rg_sync(rg_state* st) {
  if (!valid_state(st)) return fail(RG_EINVAL, "rg_sync: invalid state");
  return pending_status(st, true);
}

rg_status rg_reset(rg_state* st) {
  if (!valid_state(st)) return fail(RG_EINVAL, "rg_reset: invalid state");
  reset_kernel<<<1, 32, 0, st->stream>>>(st->S.ctrl, st->S.rows_seen, std::min(KB_MIN, st->S.kb_max));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "rg_reset");
  return RG_OK;
}

rg_status rg_export(rg_state* st, double* C, double* Ct, double* Pinv, double* w,
                    int64_t* basis_rows, int64_t capacity, int64_t* rank_out) {
  NvtxRange nvtx_range("rg_export");
  if (!valid_state(st)) return fail(RG_EINVAL, "rg_export: invalid state");
  int64_t r = 0;
  rg_status s = rg_rank(st, &r);
  if (s != RG_OK && s != RG_ECAPACITY && s != RG_ENONFINITE) return s;
  if (r > capacity) return fail(RG_EINVAL, "rg_export: rank %lld exceeds capacity %lld",
                                (long long)r, (long long)capacity);
  cudaError_t e = cudaSuccess;
  e = launch_flush(flush_view(st), st->grid, st->stream);
  if (e == cudaSuccess) e = launch_export_prep(st->S, st->grid, st->stream);  // forms w and P^-1 from P
  if (e == cudaSuccess) e = launch_export(st->S, C, Ct, Pinv, w, (long long*)basis_rows, st->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_export");
  if (rank_out) *rank_out = r;
  return RG_OK;
}

rg_status rg_snapshot_size(rg_state* st, int64_t* bytes_out) {
  if (!valid_state(st) || !bytes_out) return fail(RG_EINVAL, "rg_snapshot_size: invalid argument");
  *bytes_out = (int64_t)snapshot_bytes(st->S);
  return RG_OK;
}

rg_status rg_snapshot(rg_state* st, void* buf, int64_t bytes) {
  NvtxRange nvtx_range("rg_snapshot");
  if (!valid_state(st)) return fail(RG_EINVAL, "rg_snapshot: invalid state");
  if (!buf) return fail(RG_EINVAL, "rg_snapshot: buf is NULL");
  if ((uintptr_t)buf % 256) return fail(RG_EINVAL, "rg_snapshot: buf is not 256-byte aligned");
  const size_t need = snapshot_bytes(st->S);
  if (bytes < (int64_t)need)
    return fail(RG_EINVAL, "rg_snapshot: %lld bytes given, %zu needed", (long long)bytes, need);
  cudaError_t e = launch_flush(flush_view(st), st->grid, st->stream);
  if (e == cudaSuccess) e = launch_snapshot(st->S, buf, st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_snapshot: launch");
  return RG_OK;
}

rg_status rg_restore(rg_state* st, const void* buf, int64_t bytes) {
  NvtxRange nvtx_range("rg_restore");
  if (!valid_state(st)) return fail(RG_EINVAL, "rg_restore: invalid state");
  if (!buf) return fail(RG_EINVAL, "rg_restore: buf is NULL");
  if ((uintptr_t)buf % 256) return fail(RG_EINVAL, "rg_restore: buf is not 256-byte aligned");
  const size_t need = snapshot_bytes(st->S);
  if (bytes < (int64_t)need)
    return fail(RG_EINVAL, "rg_restore: %lld bytes given, %zu needed", (long long)bytes, need);
  cudaError_t e = launch_restore(st->S, buf, st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_restore: launch");
  return RG_OK;
}

rg_status rg_set_stream(rg_state* st, void* cuda_stream) {
  if (!valid_state(st)) return fail(RG_EINVAL, "rg_set_stream: invalid state");
  cudaError_t e = cudaStreamSynchronize(st->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rg_set_stream");
  st->stream = (cudaStream_t)cuda_stream;
  return RG_OK;
}

rg_status rg_set_screen(rg_state* st, double tau_lo) {
  if (!valid_state(st)) return fail(RG_EINVAL, "rg_set_screen: invalid state");
  if (!(tau_lo > 0.0 && tau_lo < 1.0)) return fail(RG_EINVAL, "rg_set_screen: tau_lo = %g outside (0, 1)", tau_lo);
  st->S.tau_lo = tau_lo;
  return RG_OK;
}

rg_status rg_free(rg_state* st) {
  if (!st) return RG_OK;
  cudaStreamSynchronize(st->stream);
  if (st->copy_stream) cudaStreamSynchronize(st->copy_stream);
  if (st->arena) cudaFree(st->arena);
  if (st->stage) cudaFree(st->stage);
  for (int h = 0; h < 2; ++h) {
    if (st->copied[h]) cudaEventDestroy(st->copied[h]);
    if (st->consumed[h]) cudaEventDestroy(st->consumed[h]);
  }
  if (st->copy_stream) cudaStreamDestroy(st->copy_stream);
  if (st->stage_ind) cudaFree(st->stage_ind);
  if (st->xbuf) cudaFree(st->xbuf);
  delete st;
  return RG_OK;
}

}  // extern "C"
