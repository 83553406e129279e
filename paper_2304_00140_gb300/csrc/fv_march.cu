// fv_march.cu -- dispatch of the fused 2D stage kernel on the register type
// (the instantiations live in fv_march_f.cu and fv_march_d.cu).
#include "fv_launch.h"
#include "fv_march.cuh"

namespace tfv {

cudaError_t launch_march_f(int nc, int mode, int var, const MarchArgs& A, int grid, cudaStream_t s);
cudaError_t launch_march_d(int nc, int mode, int var, const MarchArgs& A, int grid, cudaStream_t s);
cudaError_t launch_march_fc(int nc, int mode, int var, const MarchArgs& A, int grid, cudaStream_t s);
int march_occupancy_f(int nc, int mode, int var);
int march_occupancy_fc(int nc, int mode, int var);
int march_occupancy_d(int nc, int mode, int var);

cudaError_t launch_march(int nc, int mixed, int mode, int var, const MarchArgs& A, int grid, cudaStream_t s)
{
    // the fused CFL speed (MARCH_CFL) exists in the FP32 form only
    if (mode & MARCH_CFL) return mixed ? launch_march_fc(nc, mode, var, A, grid, s) : cudaErrorInvalidValue;
    return mixed ? launch_march_f(nc, mode, var, A, grid, s) : launch_march_d(nc, mode, var, A, grid, s);
}

int march_occupancy(int nc, int mixed, int mode, int var)
{
    if (mode & MARCH_CFL) return mixed ? march_occupancy_fc(nc, mode, var) : 0;
    return mixed ? march_occupancy_f(nc, mode, var) : march_occupancy_d(nc, mode, var);
}

}  // namespace tfv
