// fv_prim.cu -- primitive-update kernel instantiations, state I/O and
// diagnostics kernels, and the (ndim, ncomp, precision) dispatch.
#include <algorithm>
#include <cstdint>

#include "fv_launch.h"

namespace tfv {

#define FV_DECL(sfx)                                                                                  \
    cudaError_t launch_stage_##sfx(int nc, int tile, int ff, const StageArgs& A, int grid, size_t smem,       \
                                   cudaStream_t s);                                                           \
    cudaError_t set_smem_##sfx(int nc, int tile, int ff, size_t smem);                                        \
    int occupancy_##sfx(int nc, int tile, int ff, size_t smem);                                               \
    size_t smem_##sfx(int nc, int tile, int ff, int nprim);
FV_DECL(2d)
FV_DECL(2f)
FV_DECL(3d)
FV_DECL(3f)
#undef FV_DECL

#define FV_PICK(fn, ...)                                                                 \
    (nd == 2 ? (mixed ? fn##_2f(__VA_ARGS__) : fn##_2d(__VA_ARGS__))                    \
             : (mixed ? fn##_3f(__VA_ARGS__) : fn##_3d(__VA_ARGS__)))

cudaError_t launch_stage(int nd, int nc, int mixed, int tile, const StageArgs& A, int grid, size_t smem,
                         cudaStream_t s, int ff)
{
    return FV_PICK(launch_stage, nc, tile, ff, A, grid, smem, s);
}
size_t stage_smem(int nd, int nc, int mixed, int tile, int nprim, int ff)
{
    return FV_PICK(smem, nc, tile, ff, nprim);
}
cudaError_t stage_set_smem(int nd, int nc, int mixed, int tile, size_t smem, int ff)
{
    return FV_PICK(set_smem, nc, tile, ff, smem);
}
int stage_occupancy(int nd, int nc, int mixed, int tile, size_t smem, int ff)
{
    return FV_PICK(occupancy, nc, tile, ff, smem);
}

int prim_occupancy(int nd, int nc, int mixed);

template <int ND, int NC, typename R, typename Q>
static cudaError_t gop(const PrimArgs& A, int grid, cudaStream_t s)
{
    if (A.P.pr) prim_kernel<ND, NC, R, CL_PR, Q><<<grid, 256, 0, s>>>(A);
    else if (A.P.baro) prim_kernel<ND, NC, R, CL_BARO, Q><<<grid, 256, 0, s>>>(A);
    else prim_kernel<ND, NC, R, CL_SG, Q><<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

template <int ND, int NC>
static cudaError_t gop2(int mixed, int ff, const PrimArgs& A, int grid, cudaStream_t s)
{
    if (!mixed) return gop<ND, NC, double, double>(A, grid, s);
    return ff ? gop<ND, NC, float, float2>(A, grid, s) : gop<ND, NC, float, double>(A, grid, s);
}

cudaError_t launch_prim(int nd, int nc, int mixed, const PrimArgs& A, int grid, cudaStream_t s, int ff)
{
    if (nd == 2 && nc == 2) return gop2<2, 2>(mixed, ff, A, grid, s);
    if (nd == 2 && nc == 3) return gop2<2, 3>(mixed, ff, A, grid, s);
    if (nd == 3 && nc == 2) return gop2<3, 2>(mixed, ff, A, grid, s);
    if (nd == 3 && nc == 3) return gop2<3, 3>(mixed, ff, A, grid, s);
    return cudaErrorInvalidValue;
}

template <int ND, int NC, typename R>
static int pocc()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, prim_kernel<ND, NC, R, false, double>, 256, 0) !=
        cudaSuccess)
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

// ------------------------------------------------------ sensor flags dump
// App. D flag of every interior cell of one case from the primitive arrays
// (written by a primitive pass), through the stage kernel's sensor function
template <int ND, typename R, int CL>
__global__ void sensor_dump_kernel(DevParams P, const CaseDesc* cases, int icase, const R* prim, long long ncell,
                                   unsigned char* out)
{
    const CaseDesc& C = cases[icase];
    const long long st[3] = {1, C.gp, (long long)C.gp * C.g[1]};
    R ci[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) ci[d] = pick<R>(C.idx[d], C.fidx[d]);
    const R* base = prim + C.poff;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell;
         i += (long long)gridDim.x * blockDim.x) {
        const long long x = i % C.n[0], y = (i / C.n[0]) % C.n[1], z = i / ((long long)C.n[0] * C.n[1]);
        const long long h = (ND == 3 ? (z + 2) * st[2] : 0) + (y + 2) * st[1] + (x + 2);
        out[i] = sensor_flag<ND, R, CL, long long>(P, base, P.ntot_p, h, st, ci);
    }
}

cudaError_t launch_sensor_dump(int nd, int mixed, const DevParams& P, const CaseDesc* cases, int icase,
                               const void* prim, long long ncell, unsigned char* out, cudaStream_t s)
{
    const int g = (int)std::min<long long>(4096, (ncell + 255) / 256);
    const bool b = P.baro != 0;
#define FV_DUMP(ND_, R_)                                                                                      \
    (b ? sensor_dump_kernel<ND_, R_, CL_BARO><<<g, 256, 0, s>>>(P, cases, icase, static_cast<const R_*>(prim),  \
                                                                ncell, out)                                    \
       : sensor_dump_kernel<ND_, R_, CL_SG><<<g, 256, 0, s>>>(P, cases, icase, static_cast<const R_*>(prim),    \
                                                              ncell, out))
    if (nd == 2) { if (mixed) FV_DUMP(2, float); else FV_DUMP(2, double); }
    else { if (mixed) FV_DUMP(3, float); else FV_DUMP(3, double); }
#undef FV_DUMP
    return cudaGetLastError();
}

// ----------------------------------------------------------- state I/O
// register store / load of one conserved value (FP64 or float-float)
__device__ __forceinline__ void reg_put(double* r, long long i, double x) { r[i] = x; }
__device__ __forceinline__ void reg_put(float2* r, long long i, double x) { r[i] = ff_from_double(x); }

// primitive (u, p, T, Y) -> conserved through the FP64 closure (Eq. 3-5)
template <int ND, int NC, typename Q>
__global__ void prim_to_cons_kernel(IoArgs A)
{
    constexpr int NV = ND + NC + 1;
    const CaseDesc& C = A.cases[A.icase];
    const double* in = static_cast<const double*>(A.in);
    Q* out = static_cast<Q*>(A.out);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < A.ncell;
         i += (long long)gridDim.x * blockDim.x) {
        double w[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) w[v] = in[v * A.ncell + i];
        double rho, e, c;
        const bool ok =
            A.P.pr     ? tdu<NC, double, CL_PR>(A.P, w[ND] - A.P.p_ref, w[ND + 1], w + ND + 2, rho, e, c)
            : A.P.baro ? tdu<NC, double, CL_BARO>(A.P, w[ND] - A.P.p_ref, w[ND + 1], w + ND + 2, rho, e, c)
                       : tdu<NC, double, CL_SG>(A.P, w[ND] - A.P.p_ref, w[ND + 1], w + ND + 2, rho, e, c);
        if (!ok) set_err(A.err, ERR_NONPHYS);
        double ke = 0.0;
#pragma unroll
        for (int d = 0; d < ND; ++d) ke += 0.5 * w[d] * w[d];
        const long long o = C.qoff + i;
        reg_put(out, o, rho);
#pragma unroll
        for (int d = 0; d < ND; ++d) reg_put(out, (1 + d) * A.P.ntot_q + o, rho * w[d]);
        reg_put(out, (1 + ND) * A.P.ntot_q + o, rho * (e + ke));
#pragma unroll
        for (int k = 0; k < NC - 1; ++k) reg_put(out, (2 + ND + k) * A.P.ntot_q + o, rho * w[ND + 2 + k]);
    }
}

// conserved register -> primitive (u, p, T, Y) through the FP64 recovery
template <int ND, int NC, typename Q>
__global__ void cons_to_prim_kernel(IoArgs A)
{
    constexpr int NV = ND + NC + 1;
    const CaseDesc& C = A.cases[A.icase];
    const Q* in = static_cast<const Q*>(A.in);
    double* out = static_cast<double*>(A.out);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < A.ncell;
         i += (long long)gridDim.x * blockDim.x) {
        double qc[NV], w[NV], rho, T, p;
        const long long o = C.qoff + i;
#pragma unroll
        for (int v = 0; v < NV; ++v) qc[v] = qv_d(in[v * A.P.ntot_q + o]);
        const int st = A.P.pr     ? prim_recover<ND, NC, double, CL_PR, double>(A.P, qc, w, rho, T, p, 0.0)
                       : A.P.baro ? prim_recover<ND, NC, double, CL_BARO, double>(A.P, qc, w, rho, T, p, 0.0)
                                  : prim_recover<ND, NC, double, CL_SG, double>(A.P, qc, w, rho, T, p, 0.0);
        if (st) set_err(A.err, st);
        w[ND] = p;
#pragma unroll
        for (int v = 0; v < NV; ++v) out[v * A.ncell + i] = w[v];
    }
}

// conserved case-local doubles <-> float-float registers
// Case-local conserved doubles [nv][ncell] <-> the registers (field stride
// ntot_q, case offset off).  One grid row (blockIdx.y) per field.  `in` /
// `out` may be device memory or page-locked host memory mapped into the
// device's address space (read and written over the host link directly).
// Over the host link a thread keeps several independent 16-byte accesses in
// flight (IO_UNROLL pairs of values per iteration) when every field starts on
// a 16-byte boundary (even cell counts and offsets); otherwise one value at a
// time.
constexpr int IO_UNROLL = 4;
__device__ __forceinline__ float4 ff_pair(double2 x)
{
    const float2 a = ff_from_double(x.x), b = ff_from_double(x.y);
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ double2 dd_pair(float4 x) { return make_double2(qv_d(make_float2(x.x, x.y)), qv_d(make_float2(x.z, x.w))); }

__global__ void split_kernel(const double* __restrict__ in, long long ncell, float2* __restrict__ reg, long long ntot_q,
                             long long off, int vec)
{
    const int v = blockIdx.y;
    const double* src = in + v * ncell;
    float2* dst = reg + v * ntot_q + off;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
    if (!vec) {
        for (long long c = t0; c < ncell; c += nt) dst[c] = ff_from_double(src[c]);
        return;
    }
    const long long np = ncell / 2;
    const double2* s2 = reinterpret_cast<const double2*>(src);
    float4* d2 = reinterpret_cast<float4*>(dst);
    for (long long c = t0; c < np; c += nt * IO_UNROLL) {
        double2 x[IO_UNROLL];
#pragma unroll
        for (int u = 0; u < IO_UNROLL; ++u) {
            const long long i = c + u * nt;
            x[u] = i < np ? s2[i] : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int u = 0; u < IO_UNROLL; ++u) {
            const long long i = c + u * nt;
            if (i < np) d2[i] = ff_pair(x[u]);
        }
    }
}
__global__ void join_kernel(const float2* __restrict__ reg, long long ntot_q, long long off, long long ncell,
                            double* __restrict__ out, int vec)
{
    const int v = blockIdx.y;
    const float2* src = reg + v * ntot_q + off;
    double* dst = out + v * ncell;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
    if (!vec) {
        for (long long c = t0; c < ncell; c += nt) dst[c] = qv_d(src[c]);
        return;
    }
    const long long np = ncell / 2;
    const float4* s2 = reinterpret_cast<const float4*>(src);
    double2* d2 = reinterpret_cast<double2*>(dst);
    for (long long c = t0; c < np; c += nt * IO_UNROLL) {
        float4 x[IO_UNROLL];
#pragma unroll
        for (int u = 0; u < IO_UNROLL; ++u) {
            const long long i = c + u * nt;
            x[u] = i < np ? s2[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < IO_UNROLL; ++u) {
            const long long i = c + u * nt;
            if (i < np) d2[i] = dd_pair(x[u]);
        }
    }
}
// FP64 registers: plain field copies in (to_reg = 1) or out
__global__ void copy_fields_kernel(const double* __restrict__ in, long long in_stride, double* __restrict__ out,
                                   long long out_stride, long long ncell, int vec)
{
    const int v = blockIdx.y;
    const double* src = in + v * in_stride;
    double* dst = out + v * out_stride;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
    if (!vec) {
        for (long long c = t0; c < ncell; c += nt) dst[c] = src[c];
        return;
    }
    const long long np = ncell / 2;
    const double2* s2 = reinterpret_cast<const double2*>(src);
    double2* d2 = reinterpret_cast<double2*>(dst);
    for (long long c = t0; c < np; c += nt * IO_UNROLL) {
        double2 x[IO_UNROLL];
#pragma unroll
        for (int u = 0; u < IO_UNROLL; ++u) {
            const long long i = c + u * nt;
            x[u] = i < np ? s2[i] : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int u = 0; u < IO_UNROLL; ++u) {
            const long long i = c + u * nt;
            if (i < np) d2[i] = x[u];
        }
    }
}

// All cases at once: `in` / `out` hold each case's [nv][ncell] block in case
// order (case c's block starts at nv * qoff_c).  Grid rows walk the cases.
template <bool FF>
__global__ void all_cases_kernel(int nv, int ncases, const CaseDesc* cases, const double* host, void* reg,
                                 long long ntot_q, int to_reg)
{
    // field by field (no index division per element): the case's block of
    // the host array is [nv][cells], the register field v starts at v ntot_q
    for (int c = blockIdx.y; c < ncases; c += gridDim.y) {
        const CaseDesc& C = cases[c];
        const long long nc = (long long)C.n[0] * C.n[1] * C.n[2];
        const long long base = nv * C.qoff;
        for (int v = 0; v < nv; ++v) {
            const long long hb = base + v * nc, rb = v * ntot_q + C.qoff;
            for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nc;
                 i += (long long)gridDim.x * blockDim.x) {
                if (FF) {
                    float2* q = static_cast<float2*>(reg);
                    if (to_reg) q[rb + i] = ff_from_double(host[hb + i]);
                    else const_cast<double*>(host)[hb + i] = qv_d(q[rb + i]);
                } else {
                    double* q = static_cast<double*>(reg);
                    if (to_reg) q[rb + i] = host[hb + i];
                    else const_cast<double*>(host)[hb + i] = q[rb + i];
                }
            }
        }
    }
}

cudaError_t launch_all_cases(int nv, int ncases, const CaseDesc* cases, long long max_cells, const double* host,
                             void* reg, long long ntot_q, int ff, int to_reg, cudaStream_t s)
{
    long long gx = (max_cells + 255) / 256;
    gx = gx > 64 ? 64 : (gx < 1 ? 1 : gx);
    const dim3 g((unsigned)gx, (unsigned)(ncases > 65535 ? 65535 : ncases));
    if (ff) all_cases_kernel<true><<<g, 256, 0, s>>>(nv, ncases, cases, host, reg, ntot_q, to_reg);
    else all_cases_kernel<false><<<g, 256, 0, s>>>(nv, ncases, cases, host, reg, ntot_q, to_reg);
    return cudaGetLastError();
}

static int io_grid(long long n) { long long g = (n + 255) / 256; return (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g)); }
static dim3 field_grid(long long ncell, int nv)
{
    long long g = (ncell + 255) / 256;
    g = g > 2048 ? 2048 : (g < 1 ? 1 : g);
    return dim3((unsigned)g, (unsigned)nv);
}

// the 16-byte path: both arrays' field starts on 16-byte boundaries
static int io_vec(const void* a, const void* b, long long sa, long long sb, long long esize)
{
    const uintptr_t m = reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b);
    return ((m & 15) == 0 && ((sa * esize) & 15) == 0 && ((sb * esize) & 15) == 0) ? 1 : 0;
}
static dim3 io_field_grid(long long ncell, int nv, int vec)
{
    const long long n = vec ? (ncell / 2 + IO_UNROLL - 1) / IO_UNROLL : ncell;
    return field_grid(n, nv);
}
cudaError_t launch_split(int nv, const double* in, long long ncell, void* reg, long long ntot_q, long long off,
                         cudaStream_t s)
{
    float2* r = static_cast<float2*>(reg) + off;
    const int vec = io_vec(in, r, ncell, ntot_q, 8) && (ncell % 2 == 0);
    split_kernel<<<io_field_grid(ncell, nv, vec), 256, 0, s>>>(in, ncell, static_cast<float2*>(reg), ntot_q, off, vec);
    return cudaGetLastError();
}
cudaError_t launch_join(int nv, const void* reg, long long ntot_q, long long off, long long ncell, double* out,
                        cudaStream_t s)
{
    const float2* r = static_cast<const float2*>(reg) + off;
    const int vec = io_vec(r, out, ntot_q, ncell, 8) && (ncell % 2 == 0);
    join_kernel<<<io_field_grid(ncell, nv, vec), 256, 0, s>>>(static_cast<const float2*>(reg), ntot_q, off, ncell, out,
                                                               vec);
    return cudaGetLastError();
}
cudaError_t launch_copy_fields(int nv, const double* in, long long in_stride, double* out, long long out_stride,
                               long long ncell, cudaStream_t s)
{
    const int vec = io_vec(in, out, in_stride, out_stride, 8) && (ncell % 2 == 0);
    copy_fields_kernel<<<io_field_grid(ncell, nv, vec), 256, 0, s>>>(in, in_stride, out, out_stride, ncell, vec);
    return cudaGetLastError();
}

template <typename Q>
static cudaError_t p2c(int nd, int nc, const IoArgs& A, cudaStream_t s)
{
    const int g = io_grid(A.ncell);
    if (nd == 2 && nc == 2) prim_to_cons_kernel<2, 2, Q><<<g, 256, 0, s>>>(A);
    else if (nd == 2 && nc == 3) prim_to_cons_kernel<2, 3, Q><<<g, 256, 0, s>>>(A);
    else if (nd == 3 && nc == 2) prim_to_cons_kernel<3, 2, Q><<<g, 256, 0, s>>>(A);
    else if (nd == 3 && nc == 3) prim_to_cons_kernel<3, 3, Q><<<g, 256, 0, s>>>(A);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}
template <typename Q>
static cudaError_t c2p(int nd, int nc, const IoArgs& A, cudaStream_t s)
{
    const int g = io_grid(A.ncell);
    if (nd == 2 && nc == 2) cons_to_prim_kernel<2, 2, Q><<<g, 256, 0, s>>>(A);
    else if (nd == 2 && nc == 3) cons_to_prim_kernel<2, 3, Q><<<g, 256, 0, s>>>(A);
    else if (nd == 3 && nc == 2) cons_to_prim_kernel<3, 2, Q><<<g, 256, 0, s>>>(A);
    else if (nd == 3 && nc == 3) cons_to_prim_kernel<3, 3, Q><<<g, 256, 0, s>>>(A);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_prim_to_cons(int nd, int nc, const IoArgs& A, cudaStream_t s, int ff)
{
    return ff ? p2c<float2>(nd, nc, A, s) : p2c<double>(nd, nc, A, s);
}

cudaError_t launch_cons_to_prim(int nd, int nc, const IoArgs& A, cudaStream_t s, int ff)
{
    return ff ? c2p<float2>(nd, nc, A, s) : c2p<double>(nd, nc, A, s);
}

// ---------------------------------------------------------- diagnostics
// per-block Kahan partial sums of every field of one case
template <typename Q>
__global__ void totals_kernel(int nv, const Q* q, long long ntot_q, long long off, long long ncell,
                              double* partial)
{
    __shared__ double ss[256], sc[256];
    for (int v = 0; v < nv; ++v) {
        double s = 0.0, c = 0.0;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell;
             i += (long long)gridDim.x * blockDim.x) {
            const double y = qv_d(q[v * ntot_q + off + i]) - c;
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

cudaError_t launch_totals(int nv, const void* q, long long ntot_q, long long off, long long ncell,
                          double* partial, int nblk, cudaStream_t s, int ff)
{
    if (ff) totals_kernel<float2><<<nblk, 256, 0, s>>>(nv, static_cast<const float2*>(q), ntot_q, off, ncell, partial);
    else totals_kernel<double><<<nblk, 256, 0, s>>>(nv, static_cast<const double*>(q), ntot_q, off, ncell, partial);
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

cudaError_t launch_kappa(int nd, int mixed, const PrimArgs& A, int grid, cudaStream_t s)
{
    if (nd == 2) {
        if (mixed) kappa_kernel<2, float><<<grid, 256, 0, s>>>(A);
        else kappa_kernel<2, double><<<grid, 256, 0, s>>>(A);
    } else {
        if (mixed) kappa_kernel<3, float><<<grid, 256, 0, s>>>(A);
        else kappa_kernel<3, double><<<grid, 256, 0, s>>>(A);
    }
    return cudaGetLastError();
}

// one block: the largest signal speed over every case (positive doubles order
// like their bit patterns), then the common dt
__global__ void dt_group_kernel(int ncases, unsigned long long* smax, double* dt, double* t, double cfl, int* err)
{
    __shared__ unsigned long long m;
    if (threadIdx.x == 0) m = 0ull;
    __syncthreads();
    for (int c = threadIdx.x; c < ncases; c += blockDim.x) atomicMax(&m, smax[c]);
    __syncthreads();
    const double mm = __longlong_as_double((long long)m);
    const double d = cfl / mm;
    if (threadIdx.x == 0 && (!(mm > 0.0) || !isfinite(d))) set_err(err, ERR_NONPHYS);
    for (int c = threadIdx.x; c < ncases; c += blockDim.x) {
        dt[c] = d;
        t[c] += d;
        smax[c] = 0ull;
    }
}

cudaError_t launch_dt(int ncases, unsigned long long* smax, double* dt, double* t, double cfl, int* err,
                      cudaStream_t s, bool grouped)
{
    if (grouped)
        dt_group_kernel<<<1, 256, 0, s>>>(ncases, smax, dt, t, cfl, err);
    else
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
