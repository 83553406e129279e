// fv_zmarch.cu -- instantiations and launchers of the z-marching 3D stage
// kernel (fv_zmarch.cuh): FP32-mixed form (and the FP64 form's variants 1
// and 2, one block per SM), 2 or 3 components.
// Variants: 0 / 1 / 3 / 4 / 5 Table 4.2 limiter pair with 320 / 256 / 352 /
// 416 / 288 threads (352 covers a plane's 18 x 18 sensor and smoothing cells
// in one round; a plane's 26 face tasks take 13 warps two rounds each, 9
// warps three); 2 a limiter pair read at run time, 320 threads.  Two
// resident blocks per SM (the plane ring takes about 100 KB of shared
// memory).  With the viscous and gravity terms (visc = 1) variants 1 and 2
// only; FP64 variants 1, 2, 4 and 5.
#include <type_traits>

#include "fv_launch.h"
#include "fv_zmarch.cuh"

namespace tfv {

namespace {
template <int V> constexpr int nt_of() { return V == 1 ? 256 : (V == 3 ? 352 : (V == 4 ? 416 : (V == 5 ? 288 : 320))); }
template <int V> constexpr int lim_of() { return V == 2 ? LIM_RUNTIME : LIM_TABLE42; }
// D = 1: the FP64 form (double registers and plane ring, one resident block per SM)
#define FV_ZK(NC, V, VI, D)                                                                               \
    zmarch_kernel<NC, nt_of<V>(), (D ? 1 : 2), lim_of<V>(), VI, typename std::conditional<(D != 0), double, float2>::type>

template <int NC, int V, int VI, int D>
cudaError_t go(const ZArgs& A, int grid, size_t smem, cudaStream_t s)
{
    FV_ZK(NC, V, VI, D)<<<grid, nt_of<V>(), smem, s>>>(A);
    return cudaGetLastError();
}
template <int NC, int V, int VI, int D>
cudaError_t attr(size_t smem)
{
    return cudaFuncSetAttribute(FV_ZK(NC, V, VI, D), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
template <int NC, int V, int VI, int D>
int occ(size_t smem)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, FV_ZK(NC, V, VI, D), nt_of<V>(), smem) != cudaSuccess)
        return 0;
    return n;
}
#undef FV_ZK
}  // namespace

// FV_ZBAD: the value for a variant without an instantiation (viscous: 1 and
// 2; FP64: 1, 2, 4 and 5 without the viscous terms)
#define FV_ZSWITCH(fn, ...)                                                                        \
    if (fp64) {                                                                                    \
        if (visc) return FV_ZBAD;                                                                  \
        switch (var) {                                                                             \
        case 1: return nc == 2 ? fn<2, 1, 0, 1>(__VA_ARGS__) : fn<3, 1, 0, 1>(__VA_ARGS__);         \
        case 2: return nc == 2 ? fn<2, 2, 0, 1>(__VA_ARGS__) : fn<3, 2, 0, 1>(__VA_ARGS__);         \
        case 4: return nc == 2 ? fn<2, 4, 0, 1>(__VA_ARGS__) : fn<3, 4, 0, 1>(__VA_ARGS__);         \
        case 5: return nc == 2 ? fn<2, 5, 0, 1>(__VA_ARGS__) : fn<3, 5, 0, 1>(__VA_ARGS__);         \
        default: return FV_ZBAD;                                                                   \
        }                                                                                          \
    }                                                                                              \
    if (visc) {                                                                                    \
        switch (var) {                                                                             \
        case 1: return nc == 2 ? fn<2, 1, 1, 0>(__VA_ARGS__) : fn<3, 1, 1, 0>(__VA_ARGS__);         \
        case 2: return nc == 2 ? fn<2, 2, 1, 0>(__VA_ARGS__) : fn<3, 2, 1, 0>(__VA_ARGS__);         \
        default: return FV_ZBAD;                                                                   \
        }                                                                                          \
    }                                                                                              \
    switch (var) {                                                                                 \
    case 1: return nc == 2 ? fn<2, 1, 0, 0>(__VA_ARGS__) : fn<3, 1, 0, 0>(__VA_ARGS__);             \
    case 2: return nc == 2 ? fn<2, 2, 0, 0>(__VA_ARGS__) : fn<3, 2, 0, 0>(__VA_ARGS__);             \
    case 3: return nc == 2 ? fn<2, 3, 0, 0>(__VA_ARGS__) : fn<3, 3, 0, 0>(__VA_ARGS__);             \
    case 4: return nc == 2 ? fn<2, 4, 0, 0>(__VA_ARGS__) : fn<3, 4, 0, 0>(__VA_ARGS__);             \
    case 5: return nc == 2 ? fn<2, 5, 0, 0>(__VA_ARGS__) : fn<3, 5, 0, 0>(__VA_ARGS__);             \
    default: return nc == 2 ? fn<2, 0, 0, 0>(__VA_ARGS__) : fn<3, 0, 0, 0>(__VA_ARGS__);            \
    }

cudaError_t launch_zmarch(int nc, int var, int visc, int fp64, const ZArgs& A, int grid, size_t smem, cudaStream_t s)
{
#define FV_ZBAD cudaErrorInvalidValue
    FV_ZSWITCH(go, A, grid, smem, s)
#undef FV_ZBAD
}
cudaError_t zmarch_set_smem(int nc, int var, int visc, int fp64, size_t smem)
{
#define FV_ZBAD cudaErrorInvalidValue
    FV_ZSWITCH(attr, smem)
#undef FV_ZBAD
}
int zmarch_occupancy(int nc, int var, int visc, int fp64, size_t smem)
{
#define FV_ZBAD 0
    FV_ZSWITCH(occ, smem)
#undef FV_ZBAD
}
int zmarch_threads(int var) { return var == 1 ? 256 : (var == 3 ? 352 : (var == 4 ? 416 : (var == 5 ? 288 : 320))); }
size_t zmarch_smem(int nc, int nprim, int fp64)
{
    const int es = fp64 ? 8 : 4;
    return nc == 2 ? zm_smem_bytes<2>(nprim, es) : zm_smem_bytes<3>(nprim, es);
}

}  // namespace tfv
