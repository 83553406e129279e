// fv_march_inst.cuh -- instantiations and launchers of the fused 2D stage
// kernel (fv_march.cuh) for one register type; included by fv_march_f.cu
// (FP32 arithmetic, float-float registers) and fv_march_d.cu (FP64), which
// define FV_MR, FV_MQ and FV_MSUFFIX.
#include "fv_launch.h"
#include "fv_march.cuh"

namespace tfv {

#define FV_MCAT2(a, b) a##b
#define FV_MCAT(a, b) FV_MCAT2(a, b)

namespace {
// variant v: 0 Table 4.2 limiter pair, 2 limiter pair read at run time; both
// sized for 4 (FP32) or 2 (FP64) resident blocks of 4 warps per SM (5 or 6
// FP32 blocks, at 96 or 80 registers, spill and were slower on the
// 2048 x 1024 shock-bubble); the viscous modes, which keep two more values
// per window row, for 3 FP32 blocks
template <int V, typename R, int M> constexpr int mb_of()
{
    return sizeof(R) == 4 ? ((M & MARCH_VISC) ? 3 : 4) : 2;
}
template <int V> constexpr int lim_of() { return V == 2 ? LIM_RUNTIME : LIM_TABLE42; }

#define FV_MARCH(NC, V, M) march2d_kernel<NC, FV_MR, MARCH_WARPS, mb_of<V, FV_MR, M>(), lim_of<V>(), M, FV_MQ>

template <int NC, int V, int M>
cudaError_t go(const MarchArgs& A, int grid, cudaStream_t s)
{
    FV_MARCH(NC, V, M)<<<grid, 32 * MARCH_WARPS, 0, s>>>(A);
    return cudaGetLastError();
}
template <int NC, int V, int M>
int occ()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, FV_MARCH(NC, V, M), 32 * MARCH_WARPS, 0) != cudaSuccess)
        return 0;
    return n;
}
#undef FV_MARCH

template <int NC, int M>
cudaError_t go_v(int var, const MarchArgs& A, int grid, cudaStream_t s)
{
    if (var == 2) return go<NC, 2, M>(A, grid, s);
    return go<NC, 0, M>(A, grid, s);
}
template <int NC, int M>
int occ_v(int var)
{
    if (var == 2) return occ<NC, 2, M>();
    return occ<NC, 0, M>();
}
}  // namespace

// the barotropic modes (MARCH_BARO) exist in the FP32-mixed form only
#ifdef FV_MBARO
#define FV_MBARO_CASE(fn, m, ...) \
    case m: return nc == 2 ? fn<2, m>(__VA_ARGS__) : fn<3, m>(__VA_ARGS__);
#else
#define FV_MBARO_CASE(fn, m, ...)
#endif

#ifndef FV_MCFL
// the scheme modes (MARCH_ILES | MARCH_CSF | MARCH_VISC bits)
#define FV_MODE_SWITCH(fn, ...)                                                   \
    switch (mode) {                                                               \
    case 0: return nc == 2 ? fn<2, 0>(__VA_ARGS__) : fn<3, 0>(__VA_ARGS__);        \
    case 1: return nc == 2 ? fn<2, 1>(__VA_ARGS__) : fn<3, 1>(__VA_ARGS__);        \
    case 2: return nc == 2 ? fn<2, 2>(__VA_ARGS__) : fn<3, 2>(__VA_ARGS__);        \
    case 3: return nc == 2 ? fn<2, 3>(__VA_ARGS__) : fn<3, 3>(__VA_ARGS__);        \
    case 4: return nc == 2 ? fn<2, 4>(__VA_ARGS__) : fn<3, 4>(__VA_ARGS__);        \
    case 5: return nc == 2 ? fn<2, 5>(__VA_ARGS__) : fn<3, 5>(__VA_ARGS__);        \
    case 6: return nc == 2 ? fn<2, 6>(__VA_ARGS__) : fn<3, 6>(__VA_ARGS__);        \
    case 7: return nc == 2 ? fn<2, 7>(__VA_ARGS__) : fn<3, 7>(__VA_ARGS__);        \
    FV_MBARO_CASE(fn, 16, __VA_ARGS__)                                            \
    default: return FV_MBAD;                                                      \
    }
#else
// the last-stage modes with the fused CFL speed (MARCH_CFL | MARCH_ILES | MARCH_CSF)
#define FV_MODE_SWITCH(fn, ...)                                                   \
    switch (mode) {                                                               \
    case 8: return nc == 2 ? fn<2, 8>(__VA_ARGS__) : fn<3, 8>(__VA_ARGS__);        \
    case 9: return nc == 2 ? fn<2, 9>(__VA_ARGS__) : fn<3, 9>(__VA_ARGS__);        \
    case 10: return nc == 2 ? fn<2, 10>(__VA_ARGS__) : fn<3, 10>(__VA_ARGS__);     \
    case 11: return nc == 2 ? fn<2, 11>(__VA_ARGS__) : fn<3, 11>(__VA_ARGS__);     \
    FV_MBARO_CASE(fn, 24, __VA_ARGS__)                                            \
    default: return FV_MBAD;                                                      \
    }
#endif

cudaError_t FV_MCAT(launch_march_, FV_MSUFFIX)(int nc, int mode, int var, const MarchArgs& A, int grid,
                                                cudaStream_t s)
{
#define FV_MBAD cudaErrorInvalidValue
    FV_MODE_SWITCH(go_v, var, A, grid, s)
#undef FV_MBAD
}
int FV_MCAT(march_occupancy_, FV_MSUFFIX)(int nc, int mode, int var)
{
#define FV_MBAD 0
    FV_MODE_SWITCH(occ_v, var)
#undef FV_MBAD
}

}  // namespace tfv
