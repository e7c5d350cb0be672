// rg_adjoint.cu -- the adjoint of one stream's solution: one cooperative launch (one CTA
// per SM, bounded grid barriers) running adjoint_run over the whole grid.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rg_adjoint.cuh"
#include "rg_host.h"

namespace rg {

__global__ void __launch_bounds__(NT, 1) adjoint_kernel(StreamDev S, AdjArgs J) {
  grid_barrier_init(S.ctrl);
  adjoint_run<GridTeam>(GridTeam{S.ctrl}, S, J, S.ctrl[CTRL_R]);
}

cudaError_t launch_adjoint(const StreamDev& S, const AdjArgs& J, int grid, cudaStream_t stream) {
  void* args[] = {(void*)&S, (void*)&J};
  return cudaLaunchCooperativeKernel((const void*)adjoint_kernel, dim3(grid), dim3(NT), args, 0, stream);
}

}  // namespace rg
