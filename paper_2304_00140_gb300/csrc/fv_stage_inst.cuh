// fv_stage_inst.cuh -- instantiations of the stage kernel for one
// (dimension, precision) pair over every candidate tile and 2 or 3
// components; included by the fv_stage_*.cu translation units, which define
// FV_ND, FV_REAL and FV_SUFFIX.
#include "fv_launch.h"

namespace tfv {

#define FV_CAT2(a, b) a##b
#define FV_CAT(a, b) FV_CAT2(a, b)

namespace {
// I < NTILES: stiffened-gas / ideal-gas closure, tile I;
// I == NTILES: Peng-Robinson closure on tile 0
template <int I> constexpr int tile_of() { return I < NTILES ? I : 0; }
template <int I> constexpr bool pr_of() { return I >= NTILES; }

template <int NC, int I>
cudaError_t go(const StageArgs& A, int grid, size_t smem, cudaStream_t s)
{
    constexpr TileDef t = tile_def(FV_ND, tile_of<I>());
    stage_kernel<FV_ND, NC, FV_REAL, t.x, t.y, t.z, t.nt, pr_of<I>()><<<grid, t.nt, smem, s>>>(A);
    return cudaGetLastError();
}
template <int NC, int I>
cudaError_t attr(size_t smem)
{
    constexpr TileDef t = tile_def(FV_ND, tile_of<I>());
    return cudaFuncSetAttribute(stage_kernel<FV_ND, NC, FV_REAL, t.x, t.y, t.z, t.nt, pr_of<I>()>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
template <int NC, int I>
int occ(size_t smem)
{
    constexpr TileDef t = tile_def(FV_ND, tile_of<I>());
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, stage_kernel<FV_ND, NC, FV_REAL, t.x, t.y, t.z, t.nt, pr_of<I>()>, t.nt, smem) != cudaSuccess)
        return 0;
    return n;
}
template <int NC, int I>
size_t bytes(int nprim)
{
    constexpr TileDef t = tile_def(FV_ND, tile_of<I>());
    return stage_smem_bytes<FV_ND, NC, FV_REAL, t.x, t.y, t.z>(nprim);
}
}  // namespace

// `tile` is the candidate index, NTILES selects the Peng-Robinson kernel
#define FV_TILE_SWITCH(fn, ...)                                                    \
    switch (tile) {                                                                \
    case 0: return nc == 2 ? fn<2, 0>(__VA_ARGS__) : fn<3, 0>(__VA_ARGS__);        \
    case 1: return nc == 2 ? fn<2, 1>(__VA_ARGS__) : fn<3, 1>(__VA_ARGS__);        \
    case 2: return nc == 2 ? fn<2, 2>(__VA_ARGS__) : fn<3, 2>(__VA_ARGS__);        \
    case 3: return nc == 2 ? fn<2, 3>(__VA_ARGS__) : fn<3, 3>(__VA_ARGS__);        \
    default: return nc == 2 ? fn<2, NTILES>(__VA_ARGS__) : fn<3, NTILES>(__VA_ARGS__); \
    }

cudaError_t FV_CAT(launch_stage_, FV_SUFFIX)(int nc, int tile, const StageArgs& A, int grid, size_t smem,
                                             cudaStream_t s)
{
    FV_TILE_SWITCH(go, A, grid, smem, s)
}
cudaError_t FV_CAT(set_smem_, FV_SUFFIX)(int nc, int tile, size_t smem) { FV_TILE_SWITCH(attr, smem) }
int FV_CAT(occupancy_, FV_SUFFIX)(int nc, int tile, size_t smem) { FV_TILE_SWITCH(occ, smem) }
size_t FV_CAT(smem_, FV_SUFFIX)(int nc, int tile, int nprim) { FV_TILE_SWITCH(bytes, nprim) }

}  // namespace tfv
