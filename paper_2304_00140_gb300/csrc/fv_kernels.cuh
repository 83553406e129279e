// fv_kernels.cuh -- the CUDA kernels of one low-storage Runge-Kutta stage.
//
//   prim_kernel   boundary update + primitive/thermodynamic update
//                 (Algorithm 1, last two lines) over each case's ghosted box,
//                 optionally with the per-case CFL maximum (warp shuffles,
//                 then one atomicMax per block).
//   stage_kernel  one fused pass per tile: halo tile of primitives in shared
//                 memory, App. D sensor, reconstruction + TDU + all-Mach flux
//                 for every face of the tile (all directions), CSF source,
//                 flux divergence and the LSRK register update in FP64.
// Both walk a work list of (case, tile origin) items so one launch serves a
// single grid or a batch of uneven cases.
#pragma once

#include "fv_device.cuh"

namespace tfv {

struct PrimArgs {
    DevParams P;
    const CaseDesc* cases;
    const int4* items;
    int nitems;
    const void* q;            // conserved register read (double or float2; field stride P.ntot_q)
    void* prim;               // R[nprim][ntot_p]
    const double* in_u;       // inflow velocities (device) or null
    unsigned long long* smax; // per-case max wave speed bits, or null
    int* err;
};

struct StageArgs {
    DevParams P;
    const CaseDesc* cases;
    const int4* items;
    int nitems;
    const void* prim;
    const void* tmaps;        // per-case TMA descriptors of the primitive arrays for this tile, or null (cp.async)
    const void* q0;           // registers: double (FP64 form) or float2 (float-float, mixed form)
    void* qout;
    const double* dt;         // per-case dt
    double a;                 // LSRK coefficient a_k
    int* err;
};

// Tile of the prim kernel (one thread per ghosted cell, 256 threads).
template <int ND> struct TileShape;
template <> struct TileShape<2> { static constexpr int X = 32, Y = 8, Z = 1, NT = 256; };
template <> struct TileShape<3> { static constexpr int X = 32, Y = 4, Z = 2, NT = 256; };

// Candidate tiles of the stage kernel, chosen per workload by the autotuner.
// NT (threads) is sized so the tile's faces take about two or three full
// rounds; tile 0 is the default.
// mb: resident blocks per SM the register allocation is sized for
// (__launch_bounds__), trading registers for latency hiding; nb: halo tile
// buffers of the FP32 form (2: the next item's tile loads while this one
// computes; 1: half the shared memory, more resident blocks).
struct TileDef { int x, y, z, nt, mb, nb; };
constexpr int NTILES = 4;
constexpr TileDef TILES2[NTILES] = {{32, 8, 1, 288, 2, 2}, {32, 8, 1, 288, 3, 2}, {16, 16, 1, 288, 3, 2},
                                    {16, 16, 1, 288, 2, 2}};
// 3D: 16x8x4 recomputes fewer faces at tile edges (3.44 a cell against 3.56
// for 16x4x4) with a smaller halo, at one block per SM
constexpr TileDef TILES3[NTILES] = {{32, 4, 2, 256, 2, 1}, {16, 4, 4, 320, 2, 1}, {16, 8, 2, 320, 2, 1},
                                    {16, 8, 4, 544, 1, 1}};
constexpr TileDef tile_def(int nd, int i) { return nd == 2 ? TILES2[i] : TILES3[i]; }

// Kernel variants of the stage kernel: 0 .. NTILES-1 stiffened/ideal-gas
// closure with the Table 4.2 limiter pair on tile i; NTILES Peng-Robinson with
// that pair on tile 0; NTILES+1 / NTILES+2 stiffened-gas / Peng-Robinson with
// any limiter pair (read at run time) on tile 0; NTILES+3 stiffened-gas with
// any limiter pair plus the viscous, heat-flux and gravity terms, tile 0;
// NTILES+4 the barotropic closure with any limiter pair, tile 0.
constexpr int NVARIANTS = NTILES + 5;
// tile of variant v: the viscous 3D variant (twelve primitive fields with the
// App. D and CSF fields) takes the 16x4x4 tile, whose halo fits in shared memory
// (3D viscous and run-time-limiter variants, which hold the most primitive
// fields and, with the capillary jump model, the jump halves of every face,
// take the 16 x 4 x 4 tile so that the FP64 halo tile fits shared memory)
constexpr int variant_tile(int nd, int v)
{
    return v < NTILES ? v : ((v == NTILES + 3 || v == NTILES + 1) && nd == 3 ? 1 : 0);
}

__device__ __forceinline__ int map_index(int n, int i, int bclo, int bchi, int& flip, int& inflow)
{
    flip = 0;
    inflow = 0;
    if (i >= 0 && i < n) return i;
    // a side shared with a neighbouring block of the same grid: the two ghost
    // layers are stored next to the block's cells (filled by the exchange)
    if ((i < 0 && bclo == BC_HALO) || (i >= n && bchi == BC_HALO)) return i;
    if (i < 0) {
        int s = -1 - i;
        if (s > n - 1) s = n - 1;
        if (bclo == 0) return ((i % n) + n) % n;
        if (bclo == 1) { flip = 1; return s; }
        if (bclo == 3) { inflow = 1; return s; }
        return 0;
    }
    int s = 2 * n - 1 - i;
    if (s < 0) s = 0;
    if (bchi == 0) return i % n;
    if (bchi == 1) { flip = 1; return s; }
    return n - 1;
}

// Asynchronous global->shared copies (cp.async, zero-filled when invalid) so
// the next work item's halo tile loads while the current one computes.
__device__ __forceinline__ void cp_async_elem(float* dst, const float* src, bool valid)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(src), "r"(valid ? 4 : 0));
}
__device__ __forceinline__ void cp_async_elem(double* dst, const double* src, bool valid)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(src), "r"(valid ? 8 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Tensor memory access (TMA): one bulk tensor copy brings a whole halo tile
// (all primitive fields) into shared memory and signals an mbarrier with the
// byte count.  Waits are bounded (see tma_wait).
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned a, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned a, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned a, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(a), "r"(parity)
                 : "memory");
    return ok != 0;
}
// the descriptor (global memory, written by the host) as seen by the tensormap proxy
__device__ __forceinline__ void tmap_acquire(const void* tmap)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(tmap) : "memory");
}
// generic-proxy accesses of shared memory before async-proxy (TMA) writes
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// 4D tile load [x, y, z, field] at the given coordinates; x * element size is
// a multiple of 16 bytes (tile origins are multiples of 16 cells)
__device__ __forceinline__ void tma_load_4d(unsigned dst, const void* tmap, int x, int y, int z, int f, unsigned mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(dst), "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(f), "r"(mbar)
        : "memory");
}
// bounded wait for phase `parity` of an mbarrier: false after ~2^22 polls
// (each poll may suspend the thread for a while), far beyond any copy time
constexpr int TMA_WAIT_POLLS = 1 << 22;
__device__ __forceinline__ bool tma_wait(unsigned a, unsigned parity, int polls = TMA_WAIT_POLLS)
{
    for (int i = 0; i < polls; ++i)
        if (mbar_try_wait(a, parity)) return true;
    return false;
}

constexpr int TMAP_BYTES = 128;   // one CUtensorMap

// halo-tile buffers of the stage kernel: two (prefetch the next item) in the
// FP32 form, one in the FP64 form (FP64-pipe bound; keeps 3D tiles in shared memory)
template <typename R, int NB> constexpr int tile_buffers() { return sizeof(R) == 4 ? NB : 1; }
// elements between two halo-tile buffers: nprim x HC rounded up to 128 bytes
template <typename R, int HC> __host__ __device__ inline int tile_buffer_stride(int nprim)
{
    const int bytes = (nprim * HC * int(sizeof(R)) + 127) & ~127;
    return bytes / int(sizeof(R));
}

// Encoded liquid volume fraction (see the prim kernel): 1 when e is the
// negated gas fraction (sign bit set, including -0 for pure liquid), else 0.
__device__ __forceinline__ float liq_side(float e) { return signbit(e) ? 1.f : 0.f; }
__device__ __forceinline__ double liq_side(double e) { return signbit(e) ? 1.0 : 0.0; }

// LSRK register update q^k = q^0 + a dt R (FP64, or compensated FP32)
__device__ __forceinline__ double lsrk_update(double q0, double adt, float, double Rv) { return q0 + adt * Rv; }
__device__ __forceinline__ double lsrk_update(double q0, double adt, float, float Rv) { return q0 + adt * double(Rv); }
__device__ __forceinline__ float2 lsrk_update(float2 q0, double, float adtf, float Rv) { return ff_add_f(q0, adtf * Rv); }

__device__ __forceinline__ void set_err(int* err, int bit)
{
    if (err) atomicOr(err, bit);
}

// ----------------------------------------------------------------- prims
template <int ND, int NC, typename R, int CL, typename Q>
__global__ void __launch_bounds__(256) prim_kernel(PrimArgs A)
{
    const Q* const qreg = static_cast<const Q*>(A.q);
    constexpr int NV = ND + NC + 1;
    using TS = TileShape<ND>;
    const DevParams& P = A.P;
    R* prim = static_cast<R*>(A.prim);
    const int tx = threadIdx.x % TS::X, ty = (threadIdx.x / TS::X) % TS::Y, tz = threadIdx.x / (TS::X * TS::Y);
    __shared__ R wmax[8];
    for (int it = blockIdx.x; it < A.nitems; it += gridDim.x) {
        const int4 wi = A.items[it];
        const CaseDesc& C = A.cases[wi.x];
        const int gc[3] = {wi.y + tx, wi.z + ty, wi.w + tz};   // ghosted coordinates
        R speed = R(0);
        const bool valid = gc[0] < C.g[0] && gc[1] < C.g[1] && gc[2] < C.g[2];
        if (valid) {
            int src[3], flip[3], infl[3];
            bool interior = true;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (d < ND) {
                    const int i = gc[d] - 2;
                    interior = interior && i >= 0 && i < C.n[d];
                    src[d] = map_index(C.n[d], i, C.bc[d][0], C.bc[d][1], flip[d], infl[d]);
                } else {
                    src[d] = 0; flip[d] = 0; infl[d] = 0;
                }
            }
            bool in_disc = false;
            if (infl[0]) {
                const double y = (src[1] + C.org[1] + 0.5) * C.dx[1] - C.in_yc;
                const double z = ND == 3 ? (src[2] + C.org[2] + 0.5) * C.dx[2] - C.in_zc : 0.0;
                if (y * y + z * z <= C.in_r2) { in_disc = true; src[0] = 0; flip[0] = 0; }
                else flip[0] = 1;
            }
            // case-local indices fit 32 bits; field strides advance a pointer
            const Q* qp = qreg + C.qoff + ((src[2] * C.n[1] + src[1]) * C.n[0] + src[0]);
            Q qc[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) { qc[v] = *qp; qp += P.ntot_q; }
            R w[NV], T, pabs, rho;
            // prim == null: CFL pass only (the fused stage kernel recovers its own primitives)
            R* const pp0 = prim ? prim + C.poff + ((gc[2] * C.g[1] + gc[1]) * C.gp + gc[0]) : nullptr;
            // Peng-Robinson Newton starts from this cell's previous temperature
            const double T0 = (CL == CL_PR && pp0) ? double(pp0[(ND + 1) * P.ntot_p]) : 0.0;
            const int rst = prim_recover<ND, NC, R, CL, Q>(P, qc, w, rho, T, pabs, T0);
            bool ok = rst == 0;
            if (rst == ERR_NONCONV) set_err(A.err, ERR_NONCONV);
#pragma unroll
            for (int d = 0; d < ND; ++d) if (flip[d]) w[d] = -w[d];
            if (in_disc) {
                const long long fc = (long long)src[2] * C.n[1] + src[1];
                const long long fn = C.in_ustride;
#pragma unroll
                for (int a = 0; a < ND; ++a) w[a] = R(C.in_uoff >= 0 ? A.in_u[C.in_uoff + a * fn + fc] : C.in_u0[a]);
                w[ND + 1] = R(C.in_T);
#pragma unroll
                for (int k = 0; k < NC - 1; ++k) w[ND + 2 + k] = R(C.in_Y[k]);
            }
            R rr = rho, cs = R(0);
            const bool need_c = P.aux_rc || A.smax || in_disc;
            if (need_c) {
                R e;
                ok = tdu<NC, R, CL>(P, w[ND], w[ND + 1], w + ND + 2, rr, e, cs) && ok;
                if (!in_disc) rr = rho;
            }
            if (!ok && rst != ERR_NONCONV) set_err(A.err, ERR_NONPHYS);
            R mu_c = R(0), kc_c = R(0);
            if (CL == CL_SG && P.visc) {
                // Eq. 2-8 with no vapour: mixture viscosity = sum_k alpha_k mu_k with
                // alpha_k = rho Y_k / rho_k (Eq. A.1.4); the conductivity mixed alike
                R s = R(0);
#pragma unroll
                for (int k = 0; k < NC - 1; ++k) s += clip01(w[ND + 2 + k]);
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    const R Yk = (k == NC - 1) ? clip01(R(1) - s) : clip01(w[ND + 2 + k]);
                    const R a = fdiv(rr * Yk * K<R>(P).gm1cv[k] * w[ND + 1], K<R>(P).Pk[k] + w[ND]);
                    mu_c += a * K<R>(P).mu[k];
                    kc_c += a * K<R>(P).kc[k];
                }
                if (pp0) {
                    pp0[P.i_mu * P.ntot_p] = mu_c;
                    pp0[P.i_kc * P.ntot_p] = kc_c;
                }
            }
            if (pp0) {
                R* o = pp0;
#pragma unroll
                for (int v = 0; v < NV; ++v) { *o = w[v]; o += P.ntot_p; }
            }
            if (pp0 && P.aux_rc) {
                pp0[P.i_rho * P.ntot_p] = rr;
                pp0[P.i_c * P.ntot_p] = cs;
            }
            if constexpr (CL == CL_BARO) {
                // liquid-vapour phase fraction (encoded as below, for the gas
                // sensor) and the vapour fraction of Eq. 2-7
                R alm, ag;
                const R av = baro_vapour<NC, R>(P, w[ND], rr, w + ND + 2, &alm, &ag);
                if (pp0 && P.aux_al) pp0[P.i_al * P.ntot_p] = (alm <= ag) ? alm : -ag;
                if (pp0) pp0[P.i_av * P.ntot_p] = av;
            } else if (pp0 && P.aux_al) {
                // liquid volume fraction (Eq. A.1.4/A.1.5) stored as the smaller
                // side: e = alpha_l if alpha_l <= alpha_g, else -alpha_g
                // (alpha_g = 1 - alpha_l from the gas terms), so differences of
                // near-1 liquid fractions keep full precision:
                //   alpha_l = e + [e < 0]
                R s = R(0), al = R(0), ag = R(0);
#pragma unroll
                for (int k = 0; k < NC - 1; ++k) s += clip01(w[ND + 2 + k]);
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    const R Yk = (k == NC - 1) ? clip01(R(1) - s) : clip01(w[ND + 2 + k]);
                    const R a = fdiv(rr * Yk * K<R>(P).gm1cv[k] * w[ND + 1], K<R>(P).Pk[k] + w[ND]);
                    if (k == P.liquid) al = a; else ag += a;
                }
                pp0[P.i_al * P.ntot_p] = (al <= ag) ? al : -ag;
            }
            if (A.smax && interior) {
                R s = R(0);
#pragma unroll
                for (int d = 0; d < ND; ++d) s += (fabs(w[d]) + cs) * pick<R>(C.idx[d], C.fidx[d]);
                if (CL == CL_SG && P.visc) {
                    // diffusive limit: 2 D sum_d 1/dx_d^2, D = max(4/3 mu, k_c / cv_min) / rho
                    R i2 = R(0);
#pragma unroll
                    for (int d = 0; d < ND; ++d) i2 += pick<R>(C.idx[d], C.fidx[d]) * pick<R>(C.idx[d], C.fidx[d]);
                    s += R(2) * fdiv(fmax(R(4.0 / 3.0) * mu_c, kc_c * K<R>(P).icvmin), rr) * i2;
                }
                speed = s;
            }
        }
        if (A.smax) {
            // block maximum, one atomic per block and case
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) speed = fmax(speed, __shfl_xor_sync(0xffffffffu, speed, o));
            if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = speed;
            __syncthreads();
            if (threadIdx.x == 0) {
                R m = R(0);
                for (int i = 0; i < 8; ++i) m = fmax(m, wmax[i]);
                // positive doubles order like their bit patterns
                atomicMax(A.smax + wi.x, (unsigned long long)__double_as_longlong(double(m)));
            }
            __syncthreads();
        }
    }
}

// App. D cell sensor (Eq. D.4) of cell h of a block of primitives (field
// stride fs, neighbour strides st): the Ducros ratio from central
// differences, the variation of the gas volume fraction (from the encoded
// liquid fraction) and, for the barotropic closure, of the vapour fraction;
// 1 if one of them exceeds its threshold.  Used by the stage kernel on its
// halo tile and by the flags diagnostic on the primitive arrays.
template <int ND, typename R, int CL, typename I>
__device__ __forceinline__ unsigned char sensor_flag(const DevParams& P, const R* sp, I fs, I h, const I* st,
                                                     const R* ci)
{
    const ConstT<R>& Kc = K<R>(P);
    R g[3][3];
    R tg = R(0), tv = R(0);
    const R* ea = sp + P.i_al * fs;
    const R e0 = ea[h];
    const R o0 = liq_side(e0);
#pragma unroll
    for (int bd = 0; bd < ND; ++bd) {
        const I hp = h + st[bd], hm = h - st[bd];
        const R inv2dx = R(0.5) * ci[bd];
#pragma unroll
        for (int a = 0; a < ND; ++a) g[a][bd] = (sp[a * fs + hp] - sp[a * fs + hm]) * inv2dx;
        // |delta alpha_gas| = |delta alpha_l| from the encoded fractions
        const R em = ea[hm], ep = ea[hp];
        tg += fabs((e0 - em) + (o0 - liq_side(em))) + fabs((ep - e0) + (liq_side(ep) - o0));
        if (CL == CL_BARO) {
            // theta^alpha: the same variation of the vapour fraction
            const R* va = sp + P.i_av * fs;
            tv += fabs(va[h] - va[hm]) + fabs(va[hp] - va[h]);
        }
    }
    R div = R(0);
#pragma unroll
    for (int a = 0; a < ND; ++a) div += g[a][a];
    R curl2;
    if (ND == 3) {
        const R wx = g[2][1] - g[1][2], wy = g[0][2] - g[2][0], wz = g[1][0] - g[0][1];
        curl2 = wx * wx + wy * wy + wz * wz;
    } else {
        const R wz = g[1][0] - g[0][1];
        curl2 = wz * wz;
    }
    const R d2 = div * div;
    const R thD = fdiv(d2, d2 + curl2 + Kc.eps_ducros);
    return (thD > Kc.thr_ducros || tg > Kc.thr_gas || (CL == CL_BARO && tv > Kc.thr_vap)) ? 1 : 0;
}

// Height-function curvature (Sec. 3.5 option) of cell hc from the encoded
// liquid fraction ea (strides st): 5-cell columns along the axis where the
// fraction varies most (an exact tie goes to the lower axis), heights
// H over the 3 (3x3) neighbouring columns, kappa = -H''/(1+H'^2)^{3/2} in 2D and
// -(H_xx (1+H_y^2) + H_yy (1+H_x^2) - 2 H_xy H_x H_y)/(1+H_x^2+H_y^2)^{3/2} in 3D.
template <int ND, typename R>
__device__ __forceinline__ R hf_kappa(const R* ea, int hc, const int* st, const R* cdx)
{
    auto A = [&](int h) { const R e = ea[h]; return e + liq_side(e); };
    int dir = 0;
    R gmax = R(-1);
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        const R g = fdiv(fabs(A(hc + st[d]) - A(hc - st[d])), R(2) * cdx[d]);
        if (g > gmax) { gmax = g; dir = d; }
    }
    // transverse axes t0 (and t1 in 3D)
    const int t0 = dir == 0 ? 1 : 0;
    const int t1 = dir == 2 ? 1 : 2;
    const int sd = st[dir], s0 = st[t0], s1 = ND == 3 ? st[t1] : 0;
    R H[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (ND == 2 && b != 1) { H[a][b] = R(0); continue; }
            const int c = hc + (a - 1) * s0 + (b - 1) * s1;
            R h = R(0);
#pragma unroll
            for (int m = -2; m <= 2; ++m) h += A(c + m * sd) * cdx[dir];
            H[a][b] = h;
        }
    const R d1 = cdx[t0];
    const R Hx = fdiv(H[2][1] - H[0][1], R(2) * d1);
    const R Hxx = fdiv(H[2][1] + H[0][1] - R(2) * H[1][1], d1 * d1);
    if (ND == 2) {
        const R q = R(1) + Hx * Hx;
        return -fdiv(Hxx, q * sq_rt(q));
    }
    const R d2 = cdx[t1];
    const R Hy = fdiv(H[1][2] - H[1][0], R(2) * d2);
    const R Hyy = fdiv(H[1][2] + H[1][0] - R(2) * H[1][1], d2 * d2);
    const R Hxy = fdiv(H[2][2] - H[2][0] - H[0][2] + H[0][0], R(4) * d1 * d2);
    const R q = R(1) + Hx * Hx + Hy * Hy;
    return -fdiv(Hxx * (R(1) + Hy * Hy) + Hyy * (R(1) + Hx * Hx) - R(2) * Hxy * Hx * Hy, q * sq_rt(q));
}

// Curvature of the CSF force (Sec. 3.5) at the cell hc of the encoded liquid
// fraction ea (strides SY, SZ): one pass of the Gaussian kernel (Eq. 3-9) on
// the cell and its neighbours, unit normals at the cell's vertices from the
// smoothed fraction, kappa = -div n -- the stage kernel's formulas and
// operation order, for the curvature pass of the capillary-jump model.
template <int ND, typename R>
__device__ __forceinline__ R smoothed_enc(const R* ea, int hc, int SY, int SZ)
{
    R s = R(0), W1 = R(0);
    if (ND == 2) {
#pragma unroll
        for (int b = -1; b <= 1; ++b)
#pragma unroll
            for (int a = -1; a <= 1; ++a) {
                const R wt = R((b == 0 ? 2 : 1) * (a == 0 ? 2 : 1));
                const R e = ea[hc + b * SY + a];
                s += wt * e;
                W1 += wt * liq_side(e);
            }
    } else {
#pragma unroll
        for (int c = -1; c <= 1; ++c)
#pragma unroll
            for (int b = -1; b <= 1; ++b)
#pragma unroll
                for (int a = -1; a <= 1; ++a) {
                    const R wt = R((c == 0 ? 2 : 1) * (b == 0 ? 2 : 1) * (a == 0 ? 2 : 1));
                    const R e = ea[hc + c * SZ + b * SY + a];
                    s += wt * e;
                    W1 += wt * liq_side(e);
                }
    }
    const R norm = R(ND == 2 ? 16 : 64);
    return (s + W1 > R(0.5) * norm) ? -(((norm - W1) - s) / norm) : (s + W1) / norm;
}

template <int ND, typename R>
__device__ __forceinline__ R kappa_smoothed(const DevParams& P, const R* ea, int hc, int SY, int SZ, const R* ci,
                                            const R* cdx)
{
    constexpr int nc = 1 << ND;
    const ConstT<R>& Kc = K<R>(P);
    R dxmin = cdx[0];
#pragma unroll
    for (int d = 1; d < ND; ++d) dxmin = fmin(dxmin, cdx[d]);
    const R gthr = Kc.grad_eps / dxmin;
    // smoothed fractions of the cell's 3^ND block (offsets -1 .. 1)
    R sa[ND == 3 ? 27 : 9];
#pragma unroll
    for (int c = 0; c < (ND == 3 ? 3 : 1); ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a)
                sa[(c * 3 + b) * 3 + a] =
                    smoothed_enc<ND, R>(ea, hc + (ND == 3 ? (c - 1) * SZ : 0) + (b - 1) * SY + (a - 1), SY, SZ);
    R kappa = R(0);
#pragma unroll
    for (int vtx = 0; vtx < nc; ++vtx) {
        const int ox = vtx & 1, oy = (vtx >> 1) & 1, oz = (vtx >> 2) & 1;
        R g[3] = {R(0), R(0), R(0)}, go[3] = {R(0), R(0), R(0)};
#pragma unroll
        for (int cc = 0; cc < nc; ++cc) {
            const int bx = cc & 1, by = (cc >> 1) & 1, bz = (cc >> 2) & 1;
            const R e = sa[((ND == 3 ? oz + bz : 0) * 3 + oy + by) * 3 + ox + bx];
            const R oc = liq_side(e);
            g[0] += bx ? e : -e; go[0] += bx ? oc : -oc;
            g[1] += by ? e : -e; go[1] += by ? oc : -oc;
            if (ND == 3) { g[2] += bz ? e : -e; go[2] += bz ? oc : -oc; }
        }
        R mag2 = R(0);
#pragma unroll
        for (int d = 0; d < ND; ++d) { g[d] = (g[d] + go[d]) * ci[d] * R(2.0 / nc); mag2 += g[d] * g[d]; }
        const R mag = sq_rt(mag2);
        const R inv = (mag > gthr) ? frcp(mag) : R(0);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            const R nd_ = g[d] * inv;
            const int od = d == 0 ? ox : (d == 1 ? oy : oz);
            kappa -= (od ? nd_ : -nd_) * ci[d] * R(2.0 / nc);
        }
    }
    return kappa;
}

// Curvature pass of the capillary-jump surface tension (Sec. 3.5 jump
// model): the CSF curvature (smoothed-fraction normals, or the height
// function) of every ghosted cell into the primitive field i_kap; a ghost
// cell takes the curvature of the interior cell the boundary update maps it
// to.  Runs after the primitive pass, on its work list.
template <int ND, typename R>
__global__ void __launch_bounds__(256) kappa_kernel(PrimArgs A)
{
    using TS = TileShape<ND>;
    const DevParams& P = A.P;
    R* prim = static_cast<R*>(A.prim);
    const int tx = threadIdx.x % TS::X, ty = (threadIdx.x / TS::X) % TS::Y, tz = threadIdx.x / (TS::X * TS::Y);
    for (int it = blockIdx.x; it < A.nitems; it += gridDim.x) {
        const int4 wi = A.items[it];
        const CaseDesc& C = A.cases[wi.x];
        const int gc[3] = {wi.y + tx, wi.z + ty, wi.w + tz};
        if (!(gc[0] < C.g[0] && gc[1] < C.g[1] && gc[2] < C.g[2])) continue;
        int src[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int flip, infl;
            src[d] = d < ND ? map_index(C.n[d], gc[d] - 2, C.bc[d][0], C.bc[d][1], flip, infl) : 0;
        }
        const int SY = C.gp, SZ = C.gp * C.g[1];
        R* const base = prim + C.poff;
        const R* ea = base + (long long)P.i_al * P.ntot_p;
        const int hm = (ND == 3 ? (src[2] + 2) * SZ : 0) + (src[1] + 2) * SY + src[0] + 2;
        const R ci[3] = {pick<R>(C.idx[0], C.fidx[0]), pick<R>(C.idx[1], C.fidx[1]), pick<R>(C.idx[2], C.fidx[2])};
        const R cdx[3] = {pick<R>(C.dx[0], C.fdx[0]), pick<R>(C.dx[1], C.fdx[1]), pick<R>(C.dx[2], C.fdx[2])};
        R kap;
        if (P.hf) {
            const int st3[3] = {1, SY, SZ};
            kap = hf_kappa<ND, R>(ea, hm, st3, cdx);
        } else {
            kap = kappa_smoothed<ND, R>(P, ea, hm, SY, SZ, ci, cdx);
        }
        const int h = (ND == 3 ? gc[2] * SZ : 0) + gc[1] * SY + gc[0];
        base[(long long)P.i_kap * P.ntot_p + h] = kap;
    }
}

// Eq. 2-2 stress and heat-flux terms, added to the flux F of the face between
// cells L and R = L + e_D (visc_core: from the face's velocity gradient g,
// the two cells' u, mu, k_c, T; visc_face: from halo cells hl and hl + e_D
// with halo strides st): momentum -tau_{D a} with
// tau = mu (grad u + grad u^T - 2/3 (div u) I), energy -(u . tau)_D - k_c dT/dx_D.
// A derivative along D is the two cells' difference; along another direction
// the mean of the two cells' central differences; u, mu and k_c at the face
// are the two cells' means.
template <int ND, int D, typename R>
__device__ __forceinline__ void visc_core(const R (&g)[ND][ND], const R* uL, const R* uR, R muL, R muR, R kcL,
                                          R kcR, R TL, R TR, R ciD, R* F)
{
    R div = R(0);
#pragma unroll
    for (int a = 0; a < ND; ++a) div += g[a][a];
    const R mu = R(0.5) * (muL + muR);
    const R kc = R(0.5) * (kcL + kcR);
    R utau = R(0);
#pragma unroll
    for (int a = 0; a < ND; ++a) {
        R tau = mu * (g[a][D] + g[D][a]);
        if (a == D) tau -= R(2.0 / 3.0) * mu * div;
        F[1 + a] -= tau;
        utau += R(0.5) * (uL[a] + uR[a]) * tau;
    }
    F[1 + ND] -= utau + kc * ((TR - TL) * ciD);
}

template <int ND, int D, typename R>
__device__ __forceinline__ void visc_face(const DevParams& P, const R* sp, int HC, int hl, const int* st,
                                          const R* ci, R* F)
{
    const int hr = hl + st[D];
    R g[ND][ND];   // g[a][b] = d u_a / d x_b at the face
#pragma unroll
    for (int b = 0; b < ND; ++b)
#pragma unroll
        for (int a = 0; a < ND; ++a) {
            const R* u = sp + a * HC;
            if (b == D) g[a][b] = (u[hr] - u[hl]) * ci[D];
            else g[a][b] = ((u[hl + st[b]] - u[hl - st[b]]) + (u[hr + st[b]] - u[hr - st[b]])) * (R(0.25) * ci[b]);
        }
    R uL[ND], uR[ND];
#pragma unroll
    for (int a = 0; a < ND; ++a) { uL[a] = sp[a * HC + hl]; uR[a] = sp[a * HC + hr]; }
    const R* T = sp + (ND + 1) * HC;
    visc_core<ND, D, R>(g, uL, uR, sp[P.i_mu * HC + hl], sp[P.i_mu * HC + hr], sp[P.i_kc * HC + hl],
                        sp[P.i_kc * HC + hr], T[hl], T[hr], ci[D], F);
}

// ------------------------------------------------------------------ stage
template <int ND, int NC, typename R, int TX, int TY, int TZ, int NT, int MB, int NB, int CL, int LIM, bool VISC,
          typename Q>
__global__ void __launch_bounds__(NT, MB) stage_kernel(StageArgs A)
{
    const Q* const q0reg = static_cast<const Q*>(A.q0);
    Q* const qoreg = static_cast<Q*>(A.qout);
    constexpr int NV = ND + NC + 1;
    constexpr int NCELL = TX * TY * TZ;
    constexpr int HX = TX + 4, HY = TY + 4, HZ = (ND == 3) ? TZ + 4 : 1;
    constexpr int HC = HX * HY * HZ;
    constexpr int SX = 1, SY = HX, SZ = HX * HY;
    const DevParams& P = A.P;
    const R* prim = static_cast<const R*>(A.prim);

    extern __shared__ __align__(128) unsigned char smem_raw[];
    // halo tiles [NBUF][nprim][HC], each buffer on a 128-byte boundary (TMA destination)
    R* const spbuf = reinterpret_cast<R*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int bstride = tile_buffer_stride<R, HC>(P.nprim);
    constexpr int NFX = (TX + 1) * TY * TZ, NFY = TX * (TY + 1) * TZ, NFZ = TX * TY * (TZ + 1);
    R* const sfx = spbuf + tile_buffers<R, NB>() * bstride;   // fluxes per direction [NV][faces]
    R* const sfy = sfx + NV * NFX;
    R* const sfz = sfy + NV * NFY;
    R* extra = (ND == 2) ? sfz : sfz + NV * NFZ;
    // CSF scratch: smoothed alpha on the tile +1 halo and vertex normals
    constexpr int AX = TX + 2, AY = TY + 2, AZ = (ND == 3) ? TZ + 2 : 1;
    constexpr int VX = TX + 1, VY = TY + 1, VZ = (ND == 3) ? TZ + 1 : 1;
    R* sa = extra;                        // [AZ][AY][AX]
    R* sn = sa + AX * AY * AZ;            // [ND][VZ][VY][VX]
    unsigned char* sflag = reinterpret_cast<unsigned char*>(sn + ND * VX * VY * VZ);  // [HC]
    // capillary-jump model (the stiffened-gas variant with run-time limiters
    // carries it): the jump halves J/2 and u* J/2 of every face [2][faces]
    constexpr bool CJK = LIM == LIM_RUNTIME && CL == CL_SG && !VISC;
    constexpr int NFALL = NFX + NFY + (ND == 3 ? NFZ : 0);
    R* const sg = reinterpret_cast<R*>((reinterpret_cast<uintptr_t>(sflag + HC) + 15) & ~uintptr_t(15));

    const ConstT<R>& Kc = K<R>(P);
    const int tid = threadIdx.x;
    // TMA mode: one bulk tensor copy per tile, completion on an mbarrier per buffer
    const bool tma = A.tmaps != nullptr;
    __shared__ __align__(8) unsigned long long mbar[2];
    const unsigned mb[2] = {smem_addr(&mbar[0]), smem_addr(&mbar[1])};
    const unsigned tile_bytes = unsigned(HC * P.nprim * sizeof(R));
    unsigned phase = 0;   // bit b: parity of buffer b's next completion
    if (tma) {
        if (tid == 0) {
            mbar_init(mb[0], 1);
            mbar_init(mb[1], 1);
            mbar_init_fence();
        }
        __syncthreads();
    }
    // halo tile of primitives of item `item` (ghosted coordinates x0 .. x0+HX-1)
    auto issue_tile = [&](int item, int b) {
        R* const buf = spbuf + b * bstride;
        if (tma) {
            if (tid == 0 && item < A.nitems) {
                const int4 wn = A.items[item];
                const void* tm = static_cast<const unsigned char*>(A.tmaps) + size_t(wn.x) * TMAP_BYTES;
                tmap_acquire(tm);
                fence_async_smem();
                mbar_expect_tx(mb[b], tile_bytes);
                tma_load_4d(smem_addr(buf), tm, wn.y, wn.z, wn.w, 0, mb[b]);
            }
            return;
        }
        if (item < A.nitems) {
            const int4 wn = A.items[item];
            const CaseDesc& Cn = A.cases[wn.x];
            const int g0 = Cn.g[0], g1 = Cn.g[1], g2 = Cn.g[2], gp = Cn.gp;
            const R* const base = prim + Cn.poff;
            for (int h = tid; h < HC; h += NT) {
                const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
                const int gx = wn.y + hx, gy = wn.z + hy, gz = wn.w + hz;
                const bool ok = gx < g0 && gy < g1 && gz < g2;
                const R* src = ok ? base + ((gz * g1 + gy) * gp + gx) : prim;
                R* dst = buf + h;
                for (int v = 0; v < P.nprim; ++v) {
                    cp_async_elem(dst, src, ok);
                    dst += HC;
                    src += ok ? P.ntot_p : 0;
                }
            }
        }
        cp_async_commit();
    };
    constexpr int NBUF = tile_buffers<R, NB>();
    int cur = 0;
    if (NBUF == 2) issue_tile(blockIdx.x, 0);
    for (int it = blockIdx.x; it < A.nitems; it += gridDim.x) {
        const int4 wi = A.items[it];
        const CaseDesc& C = A.cases[wi.x];
        const int x0 = wi.y, y0 = wi.z, z0 = wi.w;
        R* const sp = spbuf + cur * bstride;
        if (NBUF == 2) {
            // the next item's tile goes to the other buffer while this one computes
            issue_tile(it + gridDim.x, cur ^ 1);
        } else {
            issue_tile(it, 0);
        }
        const int vx = min(TX, C.n[0] - x0), vy = min(TY, C.n[1] - y0), vz = (ND == 3) ? min(TZ, C.n[2] - z0) : 1;
        R ci[3], cdx[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) { ci[d] = pick<R>(C.idx[d], C.fidx[d]); cdx[d] = pick<R>(C.dx[d], C.fdx[d]); }
        // this thread's cell: prefetch q0 so its latency hides behind the face work
        const int cx = tid % TX, cy = (tid / TX) % TY, cz = tid / (TX * TY);
        const bool own = tid < NCELL && cx < vx && cy < vy && cz < vz;
        const long long gcell = C.qoff + (((z0 + cz) * C.n[1] + (y0 + cy)) * C.n[0] + (x0 + cx));
        Q q0r[NV];
        {
            const Q* qp = q0reg + gcell;
#pragma unroll
            for (int v = 0; v < NV; ++v) { q0r[v] = own ? *qp : Q{}; qp += P.ntot_q; }
        }
        if (tma) {
            const bool ok = tma_wait(mb[cur], (phase >> cur) & 1u);
            phase ^= 1u << cur;
            if (__syncthreads_or(!ok)) {
                // a copy did not complete: report, let the other buffer's copy
                // (if one was issued) finish within the same bound, and stop
                if (tid == 0) {
                    set_err(A.err, ERR_TIMEOUT);
                    if (NBUF == 2 && it + gridDim.x < A.nitems) tma_wait(mb[cur ^ 1], (phase >> (cur ^ 1)) & 1u);
                }
                return;
            }
        } else {
            if (NBUF == 2) cp_async_wait_prev(); else cp_async_wait_all();
            __syncthreads();
        }
        // ---- App. D cell sensor on the tile + 1 halo
        if (P.iles) {
            const int st3[3] = {SX, SY, SZ};
            for (int h = tid; h < HC; h += NT) {
                const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
                unsigned char fl = 0;
                const bool in = hx >= 1 && hx <= vx + 2 && hy >= 1 && hy <= vy + 2 &&
                                (ND == 2 || (hz >= 1 && hz <= vz + 2));
                if (in) fl = sensor_flag<ND, R, CL, int>(P, sp, HC, h, st3, ci);
                sflag[h] = fl;
            }
        }
        // ---- CSF: smoothed alpha (Eq. 3-9) on tile + 1 halo
        if (P.csf) {
            for (int h = tid; h < AX * AY * AZ; h += NT) {
                const int ax = h % AX, ay = (h / AX) % AY, az = h / (AX * AY);
                const int hc = (ax + 1) * SX + (ay + 1) * SY + (ND == 3 ? (az + 1) * SZ : 0);
                const R* al = sp + P.i_al * HC;
                // weighted sum of the encoded fractions plus the exact integer
                // weight W1 of the liquid-side cells; encoded result
                R s = R(0), W1 = R(0);
                if (ND == 2) {
#pragma unroll
                    for (int b = -1; b <= 1; ++b) {
#pragma unroll
                        for (int a = -1; a <= 1; ++a) {
                            const R wt = R((b == 0 ? 2 : 1) * (a == 0 ? 2 : 1));
                            const R e = al[hc + b * SY + a];
                            s += wt * e;
                            W1 += wt * liq_side(e);
                        }
                    }
                } else {
#pragma unroll
                    for (int c = -1; c <= 1; ++c)
#pragma unroll
                        for (int b = -1; b <= 1; ++b)
#pragma unroll
                            for (int a = -1; a <= 1; ++a) {
                                const R wt = R((c == 0 ? 2 : 1) * (b == 0 ? 2 : 1) * (a == 0 ? 2 : 1));
                                const R e = al[hc + c * SZ + b * SY + a];
                                s += wt * e;
                                W1 += wt * liq_side(e);
                            }
                }
                const R norm = R(ND == 2 ? 16 : 64);
                // liquid side stored as -(alpha_g~), a signed zero for pure liquid
                s = (s + W1 > R(0.5) * norm) ? -(((norm - W1) - s) / norm) : (s + W1) / norm;
                sa[h] = s;
            }
        }
        __syncthreads();
        // ---- faces of all directions, in the full tile's layout (compile-time
        // index decode); faces outside a ragged tile's valid part are skipped
        constexpr int NFACE = NFX + NFY + (ND == 3 ? NFZ : 0);
        for (int f = tid; f < NFACE; f += NT) {
            int d, fx, fy, fz, fi;
            bool valid;
            if (f < NFX) {
                d = 0; fi = f;
                fx = f % (TX + 1); fy = (f / (TX + 1)) % TY; fz = f / ((TX + 1) * TY);
                valid = fx <= vx && fy < vy && fz < vz;
            } else if (f < NFX + NFY) {
                d = 1; fi = f - NFX;
                fx = fi % TX; fy = (fi / TX) % (TY + 1); fz = fi / (TX * (TY + 1));
                valid = fx < vx && fy <= vy && fz < vz;
            } else {
                d = 2; fi = f - NFX - NFY;
                fx = fi % TX; fy = (fi / TX) % TY; fz = fi / (TX * TY);
                valid = fx < vx && fy < vy && fz <= vz;
            }
            if (!valid) continue;
            // cell i-1 of the stencil in halo coordinates
            int hx = fx + 2, hy = fy + 2, hz = (ND == 3) ? fz + 2 : 0;
            int st;
            if (d == 0) { hx -= 2; st = SX; } else if (d == 1) { hy -= 2; st = SY; } else { hz -= 2; st = SZ; }
            const int h0 = hx * SX + hy * SY + hz * SZ;
            R ws[4][NV];
            R r4[4], c4[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
#pragma unroll
                for (int v = 0; v < NV; ++v) ws[s][v] = sp[v * HC + h0 + s * st];
            }
            int fl = 1;
            R a4[4];
            if constexpr (CL == CL_BARO) {
                // cell densities and vapour fractions of the liquid-vapour THINC
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    r4[s] = sp[P.i_rho * HC + h0 + s * st];
                    c4[s] = sp[P.i_c * HC + h0 + s * st];
                    a4[s] = sp[P.i_av * HC + h0 + s * st];
                }
            } else if (P.iles) {
#pragma unroll
                for (int s = 1; s <= 2; ++s) {
                    r4[s] = sp[P.i_rho * HC + h0 + s * st];
                    c4[s] = sp[P.i_c * HC + h0 + s * st];
                }
            }
            if (P.iles) fl = (sflag[h0 + st] | sflag[h0 + 2 * st]) ? 1 : 0;
            R F[NV];
            bool ok;
            if constexpr (CJK) {
                if (P.capj) {
                    // J = sigma kappa_f (alpha_i+1 - alpha_i): cell curvatures and
                    // liquid fractions of the face's two cells
                    const R* al = sp + P.i_al * HC;
                    const R* kp = sp + P.i_kap * HC;
                    const R eL = al[h0 + st], eR = al[h0 + 2 * st];
                    const R J = Kc.sigma * R(0.5) * (kp[h0 + st] + kp[h0 + 2 * st]) *
                                ((eR + liq_side(eR)) - (eL + liq_side(eL)));
                    R us;
                    ok = face_flux<ND, NC, R, CL, LIM, -1, 1>(P, d, ws, r4, c4, fl, F, a4, J, &us);
                    const int fo = (d == 0 ? 0 : (d == 1 ? NFX : NFX + NFY)) + fi;
                    sg[fo] = R(0.5) * J;
                    sg[NFALL + fo] = R(0.5) * J * us;
                } else {
                    ok = face_flux<ND, NC, R, CL, LIM>(P, d, ws, r4, c4, fl, F, a4);
                }
            } else {
                ok = face_flux<ND, NC, R, CL, LIM>(P, d, ws, r4, c4, fl, F, a4);
            }
            if (!ok) set_err(A.err, ERR_NONPHYS);
            if (VISC && P.visc) {
                const int sts[3] = {SX, SY, SZ};
                if (d == 0) visc_face<ND, 0>(P, sp, HC, h0 + st, sts, ci, F);
                else if (d == 1) visc_face<ND, 1>(P, sp, HC, h0 + st, sts, ci, F);
                else visc_face<ND, ND - 1>(P, sp, HC, h0 + st, sts, ci, F);   // d == 2 (3D only)
            }
            // store at face index fi (= (fx, fy, fz)) of the full tile face array
            const int nfd = d == 0 ? NFX : (d == 1 ? NFY : NFZ);
            R* const dst = d == 0 ? sfx : (d == 1 ? sfy : sfz);
#pragma unroll
            for (int v = 0; v < NV; ++v) dst[v * nfd + fi] = F[v];
        }
        // ---- CSF vertex normals from the smoothed alpha (Fig. 3.3)
        if (P.csf) {
            R dxmin = cdx[0];
#pragma unroll
            for (int d = 1; d < ND; ++d) dxmin = fmin(dxmin, cdx[d]);
            const R gthr = Kc.grad_eps / dxmin;
            for (int h = tid; h < VX * VY * VZ; h += NT) {
                const int ix = h % VX, iy = (h / VX) % VY, iz = h / (VX * VY);
                // vertex between smoothed cells (ix-1+1 .. ix+1) in sa coordinates: cells ix, ix+1
                R g[3] = {R(0), R(0), R(0)}, go[3] = {R(0), R(0), R(0)};
                const int nc = 1 << ND;
#pragma unroll
                for (int cc = 0; cc < (1 << ND); ++cc) {
                    const int bx = cc & 1, by = (cc >> 1) & 1, bz = (cc >> 2) & 1;
                    // alpha~ = e + [e on the liquid side]; the offsets sum exactly
                    const R e = sa[((ND == 3 ? iz + bz : 0) * AY + iy + by) * AX + ix + bx];
                    const R oc = liq_side(e);
                    g[0] += bx ? e : -e; go[0] += bx ? oc : -oc;
                    g[1] += by ? e : -e; go[1] += by ? oc : -oc;
                    if (ND == 3) { g[2] += bz ? e : -e; go[2] += bz ? oc : -oc; }
                }
                R mag2 = R(0);
#pragma unroll
                for (int d = 0; d < ND; ++d) { g[d] = (g[d] + go[d]) * ci[d] * R(2.0 / nc); mag2 += g[d] * g[d]; }
                const R mag = sq_rt(mag2);
                const R inv = (mag > gthr) ? frcp(mag) : R(0);
#pragma unroll
                for (int d = 0; d < ND; ++d) sn[(d * VZ + iz) * VY * VX + iy * VX + ix] = g[d] * inv;
            }
        }
        __syncthreads();
        // ---- divergence, CSF source, LSRK update (FP64 registers)
        {
            if (own) {
                R S[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) S[v] = R(0);
                if (P.csf) {
                    R kappa = R(0);
                    R ga[3] = {R(0), R(0), R(0)};
                    const int nc = 1 << ND;
                    const R* al = sp + P.i_al * HC;
                    const int hc = (cx + 2) * SX + (cy + 2) * SY + (ND == 3 ? (cz + 2) * SZ : 0);
#pragma unroll
                    for (int vtx = 0; vtx < (1 << ND); ++vtx) {
                        const int ox = vtx & 1, oy = (vtx >> 1) & 1, oz = (vtx >> 2) & 1;
                        const int vi = ((ND == 3 ? cz + oz : 0) * VY + cy + oy) * VX + cx + ox;
                        R gu[3] = {R(0), R(0), R(0)}, gou[3] = {R(0), R(0), R(0)};
#pragma unroll
                        for (int cc = 0; cc < (1 << ND); ++cc) {
                            const int bx = cc & 1, by = (cc >> 1) & 1, bz = (cc >> 2) & 1;
                            const int o = hc + (ox - 1 + bx) * SX + (oy - 1 + by) * SY + (ND == 3 ? (oz - 1 + bz) * SZ : 0);
                            const R e = al[o], oc = liq_side(e);
                            gu[0] += bx ? e : -e; gou[0] += bx ? oc : -oc;
                            gu[1] += by ? e : -e; gou[1] += by ? oc : -oc;
                            if (ND == 3) { gu[2] += bz ? e : -e; gou[2] += bz ? oc : -oc; }
                        }
#pragma unroll
                        for (int d = 0; d < ND; ++d) gu[d] += gou[d];
#pragma unroll
                        for (int d = 0; d < ND; ++d) {
                            const R nd_ = sn[(d * VZ + (ND == 3 ? cz + oz : 0)) * VY * VX + (cy + oy) * VX + cx + ox];
                            const int od = d == 0 ? ox : (d == 1 ? oy : oz);
                            kappa -= (od ? nd_ : -nd_) * ci[d] * R(2.0 / nc);
                            ga[d] += gu[d] * ci[d] * R(2.0 / nc);
                        }
                        (void)vi;
                    }
                    if (P.hf) {
                        const int st3[3] = {SX, SY, SZ};
                        kappa = hf_kappa<ND, R>(al, hc, st3, cdx);
                    }
                    R udg = R(0);
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        ga[d] *= R(1.0 / nc);
                        S[1 + d] = Kc.sigma * kappa * ga[d];
                        udg += sp[d * HC + hc] * ga[d];
                    }
                    S[1 + ND] = Kc.sigma * kappa * udg;
                }
                if (VISC && P.grav) {
                    // Eq. 2-2 Q: rho g (momentum), rho u . g (energy)
                    const int hc = (cx + 2) * SX + (cy + 2) * SY + (ND == 3 ? (cz + 2) * SZ : 0);
                    const R rho = sp[P.i_rho * HC + hc];
                    R ug = R(0);
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        S[1 + d] += rho * Kc.grav[d];
                        ug += sp[d * HC + hc] * Kc.grav[d];
                    }
                    S[1 + ND] += rho * ug;
                }
                const double adt = A.a * A.dt[wi.x];
                const float adtf = float(adt);
                const int fxl = (cz * TY + cy) * (TX + 1) + cx;
                const int fyl = (cz * (TY + 1) + cy) * TX + cx;
                const int fzl = (cz * TY + cy) * TX + cx;
                Q* qo = qoreg + gcell;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    R div = (sfx[v * NFX + fxl + 1] - sfx[v * NFX + fxl]) * ci[0];
                    div += (sfy[v * NFY + fyl + TX] - sfy[v * NFY + fyl]) * ci[1];
                    if (ND == 3) div += (sfz[v * NFZ + fzl + TX * TY] - sfz[v * NFZ + fzl]) * ci[2];
                    R Rv = S[v] - div;
                    if constexpr (CJK) {
                        // the jump halves of the cell's two faces per direction:
                        // normal momentum and energy
                        if (P.capj && v >= 1 && v <= 1 + ND) {
                            const int lo[3] = {fxl, NFX + fyl, NFX + NFY + fzl};
                            const int step[3] = {1, TX, TX * TY};
#pragma unroll
                            for (int d = 0; d < ND; ++d) {
                                if (v != 1 + ND && v != 1 + d) continue;
                                const R* g = sg + (v == 1 + ND ? NFALL : 0);
                                Rv += (g[lo[d] + step[d]] + g[lo[d]]) * ci[d];
                            }
                        }
                    }
                    *qo = lsrk_update(q0r[v], adt, adtf, Rv);
                    qo += P.ntot_q;
                }
            }
        }
        __syncthreads();
        if (NBUF == 2) cur ^= 1;
    }
}

// dynamic shared memory of stage_kernel
template <int ND, int NC, typename R, int TX, int TY, int TZ, int NB>
inline size_t stage_smem_bytes(int nprim, bool capj_faces = false)
{
    constexpr int NV = ND + NC + 1;
    constexpr int HC = (TX + 4) * (TY + 4) * ((ND == 3) ? TZ + 4 : 1);
    constexpr int NFX = (TX + 1) * TY * TZ, NFY = TX * (TY + 1) * TZ, NFZ = TX * TY * (TZ + 1);
    constexpr int AC = (TX + 2) * (TY + 2) * ((ND == 3) ? TZ + 2 : 1);
    constexpr int VC = (TX + 1) * (TY + 1) * ((ND == 3) ? TZ + 1 : 1);
    size_t n = tile_buffers<R, NB>() * (size_t)tile_buffer_stride<R, HC>(nprim) +
               (size_t)NV * (NFX + NFY + (ND == 3 ? NFZ : 0)) + AC + ND * VC;
    // + the capillary jump halves of every face (aligned after the flags)
    const size_t cj = capj_faces ? 2 * (size_t)(NFX + NFY + (ND == 3 ? NFZ : 0)) * sizeof(R) + 16 : 0;
    return n * sizeof(R) + HC + 16 + 128 + cj;   // + alignment of the buffers to 128 bytes
}

}  // namespace tfv
