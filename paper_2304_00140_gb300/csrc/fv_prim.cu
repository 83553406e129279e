// fv_prim.cu -- primitive-update kernel instantiations, state I/O and
// diagnostics kernels, and the (ndim, ncomp, precision) dispatch.
#include "fv_launch.h"

namespace tfv {

#define FV_DECL(sfx)                                                                                  \
    cudaError_t launch_stage_##sfx(int nc, int tile, const StageArgs& A, int grid, size_t smem, cudaStream_t s); \
    cudaError_t set_smem_##sfx(int nc, int tile, size_t smem);                                                \
    int occupancy_##sfx(int nc, int tile, size_t smem);                                                       \
    size_t smem_##sfx(int nc, int tile, int nprim);
FV_DECL(2d)
FV_DECL(2f)
FV_DECL(3d)
FV_DECL(3f)
#undef FV_DECL

#define FV_PICK(fn, ...)                                                                 \
    (nd == 2 ? (mixed ? fn##_2f(__VA_ARGS__) : fn##_2d(__VA_ARGS__))                    \
             : (mixed ? fn##_3f(__VA_ARGS__) : fn##_3d(__VA_ARGS__)))

cudaError_t launch_stage(int nd, int nc, int mixed, int tile, const StageArgs& A, int grid, size_t smem,
                         cudaStream_t s)
{
    return FV_PICK(launch_stage, nc, tile, A, grid, smem, s);
}
size_t stage_smem(int nd, int nc, int mixed, int tile, int nprim) { return FV_PICK(smem, nc, tile, nprim); }
cudaError_t stage_set_smem(int nd, int nc, int mixed, int tile, size_t smem)
{
    return FV_PICK(set_smem, nc, tile, smem);
}
int stage_occupancy(int nd, int nc, int mixed, int tile, size_t smem)
{
    return FV_PICK(occupancy, nc, tile, smem);
}

int prim_occupancy(int nd, int nc, int mixed);

template <int ND, int NC, typename R>
static cudaError_t gop(const PrimArgs& A, int grid, cudaStream_t s)
{
    if (A.P.pr) prim_kernel<ND, NC, R, true><<<grid, 256, 0, s>>>(A);
    else prim_kernel<ND, NC, R, false><<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_prim(int nd, int nc, int mixed, const PrimArgs& A, int grid, cudaStream_t s)
{
    if (nd == 2 && nc == 2) return mixed ? gop<2, 2, float>(A, grid, s) : gop<2, 2, double>(A, grid, s);
    if (nd == 2 && nc == 3) return mixed ? gop<2, 3, float>(A, grid, s) : gop<2, 3, double>(A, grid, s);
    if (nd == 3 && nc == 2) return mixed ? gop<3, 2, float>(A, grid, s) : gop<3, 2, double>(A, grid, s);
    if (nd == 3 && nc == 3) return mixed ? gop<3, 3, float>(A, grid, s) : gop<3, 3, double>(A, grid, s);
    return cudaErrorInvalidValue;
}

template <int ND, int NC, typename R>
static int pocc()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, prim_kernel<ND, NC, R, false>, 256, 0) != cudaSuccess)
        return 1;
    return n < 1 ? 1 : n;
}

int prim_occupancy(int nd, int nc, int mixed)
{
    if (nd == 2 && nc == 2) return mixed ? pocc<2, 2, float>() : pocc<2, 2, double>();
    if (nd == 2 && nc == 3) return mixed ? pocc<2, 3, float>() : pocc<2, 3, double>();
    if (nd == 3 && nc == 2) return mixed ? pocc<3, 2, float>() : pocc<3, 2, double>();
    return mixed ? pocc<3, 3, float>() : pocc<3, 3, double>();
}

// ----------------------------------------------------------- state I/O
// primitive (u, p, T, Y) -> conserved through the FP64 closure (Eq. 3-5)
template <int ND, int NC>
__global__ void prim_to_cons_kernel(IoArgs A)
{
    constexpr int NV = ND + NC + 1;
    const CaseDesc& C = A.cases[A.icase];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < A.ncell;
         i += (long long)gridDim.x * blockDim.x) {
        double w[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) w[v] = A.in[v * A.ncell + i];
        double rho, e, c;
        const bool ok = A.P.pr ? tdu<NC, double, true>(A.P, w[ND] - A.P.p_ref, w[ND + 1], w + ND + 2, rho, e, c)
                               : tdu<NC, double, false>(A.P, w[ND] - A.P.p_ref, w[ND + 1], w + ND + 2, rho, e, c);
        if (!ok) set_err(A.err, ERR_NONPHYS);
        double ke = 0.0;
#pragma unroll
        for (int d = 0; d < ND; ++d) ke += 0.5 * w[d] * w[d];
        const long long o = C.qoff + i;
        A.out[o] = rho;
#pragma unroll
        for (int d = 0; d < ND; ++d) A.out[(1 + d) * A.P.ntot_q + o] = rho * w[d];
        A.out[(1 + ND) * A.P.ntot_q + o] = rho * (e + ke);
#pragma unroll
        for (int k = 0; k < NC - 1; ++k) A.out[(2 + ND + k) * A.P.ntot_q + o] = rho * w[ND + 2 + k];
    }
}

// conserved register -> primitive (u, p, T, Y) through the FP64 recovery
template <int ND, int NC>
__global__ void cons_to_prim_kernel(IoArgs A)
{
    constexpr int NV = ND + NC + 1;
    const CaseDesc& C = A.cases[A.icase];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < A.ncell;
         i += (long long)gridDim.x * blockDim.x) {
        double qc[NV], w[NV], rho, T, p;
        const long long o = C.qoff + i;
#pragma unroll
        for (int v = 0; v < NV; ++v) qc[v] = A.in[v * A.P.ntot_q + o];
        const int st = A.P.pr ? prim_recover<ND, NC, double, true>(A.P, qc, w, rho, T, p, 0.0)
                              : prim_recover<ND, NC, double, false>(A.P, qc, w, rho, T, p, 0.0);
        if (st) set_err(A.err, st);
        w[ND] = p;
#pragma unroll
        for (int v = 0; v < NV; ++v) A.out[v * A.ncell + i] = w[v];
    }
}

static int io_grid(long long n) { long long g = (n + 255) / 256; return (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g)); }

cudaError_t launch_prim_to_cons(int nd, int nc, const IoArgs& A, cudaStream_t s)
{
    const int g = io_grid(A.ncell);
    if (nd == 2 && nc == 2) prim_to_cons_kernel<2, 2><<<g, 256, 0, s>>>(A);
    else if (nd == 2 && nc == 3) prim_to_cons_kernel<2, 3><<<g, 256, 0, s>>>(A);
    else if (nd == 3 && nc == 2) prim_to_cons_kernel<3, 2><<<g, 256, 0, s>>>(A);
    else if (nd == 3 && nc == 3) prim_to_cons_kernel<3, 3><<<g, 256, 0, s>>>(A);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_cons_to_prim(int nd, int nc, const IoArgs& A, cudaStream_t s)
{
    const int g = io_grid(A.ncell);
    if (nd == 2 && nc == 2) cons_to_prim_kernel<2, 2><<<g, 256, 0, s>>>(A);
    else if (nd == 2 && nc == 3) cons_to_prim_kernel<2, 3><<<g, 256, 0, s>>>(A);
    else if (nd == 3 && nc == 2) cons_to_prim_kernel<3, 2><<<g, 256, 0, s>>>(A);
    else if (nd == 3 && nc == 3) cons_to_prim_kernel<3, 3><<<g, 256, 0, s>>>(A);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// ---------------------------------------------------------- diagnostics
// per-block Kahan partial sums of every field of one case
__global__ void totals_kernel(int nv, const double* q, long long ntot_q, long long off, long long ncell,
                              double* partial)
{
    __shared__ double ss[256], sc[256];
    for (int v = 0; v < nv; ++v) {
        double s = 0.0, c = 0.0;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell;
             i += (long long)gridDim.x * blockDim.x) {
            const double y = q[v * ntot_q + off + i] - c;
            const double t = s + y;
            c = (t - s) - y;
            s = t;
        }
        ss[threadIdx.x] = s;
        sc[threadIdx.x] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            double S = 0.0, Cc = 0.0;
            for (int k = 0; k < blockDim.x; ++k) {
                const double y = (ss[k] - sc[k]) - Cc;
                const double t = S + y;
                Cc = (t - S) - y;
                S = t;
            }
            partial[v * gridDim.x + blockIdx.x] = S;
        }
        __syncthreads();
    }
}

cudaError_t launch_totals(int nv, const double* q, long long ntot_q, long long off, long long ncell,
                          double* partial, int nblk, cudaStream_t s)
{
    totals_kernel<<<nblk, 256, 0, s>>>(nv, q, ntot_q, off, ncell, partial);
    return cudaGetLastError();
}

// READING (no CFL rule in the paper): dt = CFL / max_i sum_d (|u_d| + c)/dx_d
__global__ void dt_kernel(int ncases, unsigned long long* smax, double* dt, double* t, double cfl, int* err)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncases; c += gridDim.x * blockDim.x) {
        const double m = __longlong_as_double((long long)smax[c]);
        const double d = cfl / m;
        if (!(m > 0.0) || !isfinite(d)) set_err(err, ERR_NONPHYS);
        dt[c] = d;
        t[c] += d;
        smax[c] = 0ull;
    }
}

cudaError_t launch_dt(int ncases, unsigned long long* smax, double* dt, double* t, double cfl, int* err,
                      cudaStream_t s)
{
    dt_kernel<<<(ncases + 255) / 256, 256, 0, s>>>(ncases, smax, dt, t, cfl, err);
    return cudaGetLastError();
}

__global__ void fill_kernel(double* x, int n, double v)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = v;
}

cudaError_t launch_fill(double* x, int n, double v, cudaStream_t s)
{
    fill_kernel<<<(n + 255) / 256, 256, 0, s>>>(x, n, v);
    return cudaGetLastError();
}

}  // namespace tfv
