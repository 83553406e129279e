// fv_stage_inst.cuh -- instantiations of the stage kernel for one
// (dimension, precision) pair over every candidate tile and 2 or 3
// components; included by the fv_stage_*.cu translation units, which define
// FV_ND, FV_REAL and FV_SUFFIX.  Register types: double for the FP64 form;
// float2 (float-float) for the mixed form of a context, plus double on the
// default tile for the mixed no-alloc entry point.
#include "fv_launch.h"

namespace tfv {

#define FV_CAT2(a, b) a##b
#define FV_CAT(a, b) FV_CAT2(a, b)

namespace {
// kernel variant I (see NVARIANTS): tile, closure and limiter pair
template <int I> constexpr int tile_of() { return variant_tile(FV_ND, I); }
template <int I> constexpr int cl_of()
{
    return (I == NTILES || I == NTILES + 2) ? CL_PR : (I == NTILES + 4 ? CL_BARO : CL_SG);
}
template <int I> constexpr int lim_of() { return I <= NTILES ? LIM_TABLE42 : LIM_RUNTIME; }
template <int I> constexpr bool visc_of() { return I == NTILES + 3; }
template <int FF> struct RegOf { using type = double; };
template <> struct RegOf<1> { using type = float2; };

#define FV_KERNEL(NC, I, FF)                                                                  \
    stage_kernel<FV_ND, NC, FV_REAL, tile_def(FV_ND, tile_of<I>()).x, tile_def(FV_ND, tile_of<I>()).y, \
                 tile_def(FV_ND, tile_of<I>()).z, tile_def(FV_ND, tile_of<I>()).nt,                    \
                 tile_def(FV_ND, tile_of<I>()).mb, tile_def(FV_ND, tile_of<I>()).nb, cl_of<I>(),       \
                 lim_of<I>(), visc_of<I>(), typename RegOf<FF>::type>

template <int NC, int I, int FF>
cudaError_t go(const StageArgs& A, int grid, size_t smem, cudaStream_t s)
{
    FV_KERNEL(NC, I, FF)<<<grid, tile_def(FV_ND, tile_of<I>()).nt, smem, s>>>(A);
    return cudaGetLastError();
}
template <int NC, int I, int FF>
cudaError_t attr(size_t smem)
{
    return cudaFuncSetAttribute(FV_KERNEL(NC, I, FF), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
template <int NC, int I, int FF>
int occ(size_t smem)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, FV_KERNEL(NC, I, FF), tile_def(FV_ND, tile_of<I>()).nt,
                                                      smem) != cudaSuccess)
        return 0;
    return n;
}
template <int NC, int I, int FF>
size_t bytes(int nprim)
{
    constexpr TileDef t = tile_def(FV_ND, tile_of<I>());
    // the stiffened-gas run-time-limiter variant carries the capillary jump model
    return stage_smem_bytes<FV_ND, NC, FV_REAL, t.x, t.y, t.z, t.nb>(nprim, I == NTILES + 1);
}
}  // namespace

// FP64 form: double registers on every variant (FF = 0).  Mixed form: float2
// registers on every variant (ff = 1) or double registers on the three
// stiffened-gas tile-0 variants (ff = 0, the no-alloc entry point).
#define FV_NC(fn, I, FF, ...) (nc == 2 ? fn<2, I, FF>(__VA_ARGS__) : fn<3, I, FF>(__VA_ARGS__))
#if FV_IS_FLOAT
#define FV_FF 1
#else
#define FV_FF 0
#endif
#define FV_TILE_SWITCH(fn, ...)                                                   \
    static_assert(NTILES == 4 && NVARIANTS == 9, "variant switch below lists nine variants");            \
    if (FV_IS_FLOAT && !ff)                                                       \
        return tile == NTILES + 1   ? FV_NC(fn, NTILES + 1, 0, __VA_ARGS__)        \
               : tile == NTILES + 3 ? FV_NC(fn, NTILES + 3, 0, __VA_ARGS__)        \
                                    : FV_NC(fn, 0, 0, __VA_ARGS__);                \
    switch (tile) {                                                               \
    case 0: return FV_NC(fn, 0, FV_FF, __VA_ARGS__);                              \
    case 1: return FV_NC(fn, 1, FV_FF, __VA_ARGS__);                              \
    case 2: return FV_NC(fn, 2, FV_FF, __VA_ARGS__);                              \
    case 3: return FV_NC(fn, 3, FV_FF, __VA_ARGS__);                              \
    case NTILES: return FV_NC(fn, NTILES, FV_FF, __VA_ARGS__);                    \
    case NTILES + 1: return FV_NC(fn, NTILES + 1, FV_FF, __VA_ARGS__);            \
    case NTILES + 2: return FV_NC(fn, NTILES + 2, FV_FF, __VA_ARGS__);            \
    case NTILES + 3: return FV_NC(fn, NTILES + 3, FV_FF, __VA_ARGS__);            \
    default: return FV_NC(fn, NTILES + 4, FV_FF, __VA_ARGS__);                    \
    }

cudaError_t FV_CAT(launch_stage_, FV_SUFFIX)(int nc, int tile, int ff, const StageArgs& A, int grid, size_t smem,
                                             cudaStream_t s)
{
    FV_TILE_SWITCH(go, A, grid, smem, s)
}
cudaError_t FV_CAT(set_smem_, FV_SUFFIX)(int nc, int tile, int ff, size_t smem) { FV_TILE_SWITCH(attr, smem) }
int FV_CAT(occupancy_, FV_SUFFIX)(int nc, int tile, int ff, size_t smem) { FV_TILE_SWITCH(occ, smem) }
size_t FV_CAT(smem_, FV_SUFFIX)(int nc, int tile, int ff, int nprim) { FV_TILE_SWITCH(bytes, nprim) }

}  // namespace tfv
