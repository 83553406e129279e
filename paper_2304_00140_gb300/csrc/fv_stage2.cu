// fv_stage2.cu -- 2D instantiations of the stage kernel.
#include "fv_launch.h"

namespace tfv {

template <int NC, typename R>
static cudaError_t go2(const StageArgs& A, int grid, size_t smem, cudaStream_t s)
{
    stage_kernel<2, NC, R><<<grid, TileShape<2>::NT, smem, s>>>(A);
    return cudaGetLastError();
}

template <int NC, typename R>
static cudaError_t attr2(size_t smem)
{
    return cudaFuncSetAttribute(stage_kernel<2, NC, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_stage2(int nc, int mixed, const StageArgs& A, int grid, size_t smem, cudaStream_t s)
{
    if (nc == 2) return mixed ? go2<2, float>(A, grid, smem, s) : go2<2, double>(A, grid, smem, s);
    if (nc == 3) return mixed ? go2<3, float>(A, grid, smem, s) : go2<3, double>(A, grid, smem, s);
    return cudaErrorInvalidValue;
}

cudaError_t set_smem2(int nc, int mixed, size_t smem)
{
    if (nc == 2) return mixed ? attr2<2, float>(smem) : attr2<2, double>(smem);
    if (nc == 3) return mixed ? attr2<3, float>(smem) : attr2<3, double>(smem);
    return cudaErrorInvalidValue;
}

size_t smem2(int nc, int mixed, int nprim)
{
    if (nc == 2) return mixed ? stage_smem_bytes<2, 2, float>(nprim) : stage_smem_bytes<2, 2, double>(nprim);
    return mixed ? stage_smem_bytes<2, 3, float>(nprim) : stage_smem_bytes<2, 3, double>(nprim);
}

template <int NC, typename R>
static int occ2(size_t smem)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_kernel<2, NC, R>, TileShape<2>::NT, smem) != cudaSuccess) return 1;
    return n < 1 ? 1 : n;
}

int occupancy2(int nc, int mixed, size_t smem)
{
    if (nc == 2) return mixed ? occ2<2, float>(smem) : occ2<2, double>(smem);
    return mixed ? occ2<3, float>(smem) : occ2<3, double>(smem);
}

}  // namespace tfv
