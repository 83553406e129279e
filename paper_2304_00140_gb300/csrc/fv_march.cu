// fv_march.cu -- instantiations and launchers of the fused 2D stage kernel
// (fv_march.cuh): FP64 (double registers) and mixed (float-float registers)
// forms, 2 or 3 components, the Table 4.2 limiter pair as constants or a
// limiter pair read at run time, and two register budgets.
#include "fv_launch.h"
#include "fv_march.cuh"

namespace tfv {

namespace {
// variant v: 0 / 1 Table 4.2 pair with 4 / 5 (FP32) or 2 / 3 (FP64)
// resident blocks of 4 warps per SM; 2 run-time limiter pair, 4 (2) blocks
template <int V, typename R> constexpr int mb_of() { return sizeof(R) == 4 ? (V == 1 ? 5 : 4) : (V == 1 ? 3 : 2); }
template <int V> constexpr int lim_of() { return V == 2 ? LIM_RUNTIME : LIM_TABLE42; }

#define FV_MARCH(NC, R, V, Q) march2d_kernel<NC, R, MARCH_WARPS, mb_of<V, R>(), lim_of<V>(), Q>

template <int NC, typename R, int V, typename Q>
cudaError_t go(const MarchArgs& A, int grid, cudaStream_t s)
{
    FV_MARCH(NC, R, V, Q)<<<grid, 32 * MARCH_WARPS, 0, s>>>(A);
    return cudaGetLastError();
}
template <int NC, typename R, int V, typename Q>
int occ()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, FV_MARCH(NC, R, V, Q), 32 * MARCH_WARPS, 0) != cudaSuccess)
        return 0;
    return n;
}
#undef FV_MARCH

template <int NC, int V>
cudaError_t go_f(int mixed, const MarchArgs& A, int grid, cudaStream_t s)
{
    return mixed ? go<NC, float, V, float2>(A, grid, s) : go<NC, double, V, double>(A, grid, s);
}
template <int NC, int V>
int occ_f(int mixed)
{
    return mixed ? occ<NC, float, V, float2>() : occ<NC, double, V, double>();
}
}  // namespace

#define FV_MARCH_SWITCH(fn, ...)                                                  \
    switch (var) {                                                                \
    case 0: return nc == 2 ? fn<2, 0>(__VA_ARGS__) : fn<3, 0>(__VA_ARGS__);        \
    case 1: return nc == 2 ? fn<2, 1>(__VA_ARGS__) : fn<3, 1>(__VA_ARGS__);        \
    default: return nc == 2 ? fn<2, 2>(__VA_ARGS__) : fn<3, 2>(__VA_ARGS__);       \
    }

cudaError_t launch_march(int nc, int mixed, int var, const MarchArgs& A, int grid, cudaStream_t s)
{
    FV_MARCH_SWITCH(go_f, mixed, A, grid, s)
}

int march_occupancy(int nc, int mixed, int var) { FV_MARCH_SWITCH(occ_f, mixed) }

}  // namespace tfv
