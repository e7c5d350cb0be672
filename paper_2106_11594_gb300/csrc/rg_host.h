// rg_host.h -- launch helpers shared between the host files of librg.so (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>

#include <nvtx3/nvToolsExt.h>

#include "../../include/rg.h"
#include "rg_internal.cuh"

namespace rg {

// NVTX range around one C ABI call (header-only NVTX3: a no-op unless a profiler such as
// Nsight attaches its injection library), so that the calls show up on a timeline.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

rg_status fail(rg_status code, const char* fmt, ...);
rg_status cuda_fail(cudaError_t e, const char* what);
rg_status status_from_bits(int bits);

cudaError_t launch_stream(const StreamDev& S, const double* Gamma, const double* y, long long k,
                          uint8_t* indep, int grid, cudaStream_t stream);
cudaError_t stream_grid_size(int mixed, int ortho, int orthog, int* grid);
cudaError_t launch_export_prep(const StreamDev& S, int grid, cudaStream_t stream);
cudaError_t launch_flush(const StreamDev& S, int grid, cudaStream_t stream);
cudaError_t launch_solution(const StreamDev& S, double* X, cudaStream_t stream);
cudaError_t launch_export(const StreamDev& S, double* C, double* Ct, double* Pinv, double* w,
                          long long* basis, cudaStream_t stream);
cudaError_t launch_pinv(const StreamDev& S, const double* A, long long n, double* Apinv, long long ld,
                        int r, double* wk, cudaStream_t stream);
size_t snapshot_bytes(const StreamDev& S);
cudaError_t launch_snapshot(const StreamDev& S, void* buf, cudaStream_t stream);
cudaError_t launch_restore(const StreamDev& S, const void* buf, cudaStream_t stream);
struct AdjArgs;
cudaError_t launch_adjoint(const StreamDev& S, const AdjArgs& J, int grid, cudaStream_t stream);

}  // namespace rg
