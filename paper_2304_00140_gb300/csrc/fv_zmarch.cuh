// fv_zmarch.cuh -- 3D stage kernel that marches along z (FP32-mixed form,
// stiffened/ideal-gas closure): the same sensor (App. D, Eq. D.4),
// reconstruction + TDU + all-Mach flux (Sec. 3.2-3.3), CSF source (Sec. 3.5,
// Eq. 3-9/3-10) and LSRK update (Sec. 3.1) as the tiled stage kernel, with
// the same formulas in the same order, but organised per z-plane.
//
// A block owns a TX x TY column of cells and walks up a chunk of z-planes.
// The primitives of planes z-1 .. z+2 (with a 2-cell halo in x and y) sit in
// a ring of four shared-memory slots; each step brings in one new plane with
// one TMA copy.  A step has two phases, each closed by a block barrier:
// (1) the vertex normals and z-face fluxes between z and z+1 and the x- and
// y-faces of plane z; (2) the update of plane z, then (once plane z+3 has
// arrived) the sensor flags and smoothed fractions of plane z+2 for the next
// step.  The flags, smoothed fractions, normals and z-fluxes of the planes
// below are kept in two-slot rings.  Every face is computed once (the tiled kernel computes
// a tile's edge faces twice), and the +1 halo work of the sensor and the
// smoothing is in x and y only.  VISC instantiations add the Eq. 2-2 stress
// and heat flux at every face (the tiled kernel's face gradients: the planes
// below and above give the z differences of x- and y-faces) and the gravity
// source in the update.
#pragma once

#include <type_traits>

#include "fv_kernels.cuh"

namespace tfv {

struct ZArgs {
    DevParams P;
    const CaseDesc* cases;
    const int4* items;        // (case, x0, y0, z0): a TX x TY column, planes z0 .. z0+zc-1
    int nitems;
    int zc;                   // planes per item
    const void* tmaps;        // per case: TMA descriptor of the primitives, box (TX+4) x (TY+4) x 1 x nprim
    const void* q0;           // registers (float-float)
    void* qout;
    const double* dt;
    double a;
    int* err;
};

constexpr int ZM_TX = 16, ZM_TY = 16;

// elements between two plane slots: nprim x HXY values of es bytes rounded up to 128 bytes
__host__ __device__ inline int zm_slot_stride(int nprim, int hxy, int es)
{
    return ((nprim * hxy * es + 127) & ~127) / es;
}

// dynamic shared memory of the kernel with es-byte values (4 FP32-mixed, 8 FP64)
template <int NC>
inline size_t zm_smem_bytes(int nprim, int es)
{
    constexpr int TX = ZM_TX, TY = ZM_TY, NV = 3 + NC + 1;
    constexpr int HX = TX + 4, HY = TY + 4, HXY = HX * HY, AXY = (TX + 2) * (TY + 2), VXY = (TX + 1) * (TY + 1);
    constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1), TXY = TX * TY;
    const size_t vals = 4 * (size_t)zm_slot_stride(nprim, HXY, es) + NV * (NFX + NFY) + 2 * NV * TXY + 2 * AXY +
                        2 * 2 * 3 * VXY;
    return vals * es + 2 * HXY + 128;
}

// Eq. 2-2 stress and heat flux of the face between cell L = (plane cl, index
// hl) and R = (cr, hr) along D, with the tiled kernel's face gradients in its
// order; dnL / upL, dnR / upR: the planes below and above L and R (x- and
// y-faces; a z-face's cells are in two planes and need none)
template <int D, typename R>
__device__ __forceinline__ void zm_visc_face(const DevParams& P, int HXY, int HX, const R* cl, int hl, const R* cr,
                                             int hr, const R* dnL, const R* upL, const R* dnR, const R* upR,
                                             const R* ci, R* F)
{
    R g[3][3];   // g[a][b] = d u_a / d x_b at the face
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const R* uL = cl + a * HXY;
            const R* uR = cr + a * HXY;
            if (b == D) {
                g[a][b] = (uR[hr] - uL[hl]) * ci[D];
            } else if (b < 2) {
                const int sb = b == 0 ? 1 : HX;
                g[a][b] = ((uL[hl + sb] - uL[hl - sb]) + (uR[hr + sb] - uR[hr - sb])) * (R(0.25) * ci[b]);
            } else {
                g[a][b] = ((upL[a * HXY + hl] - dnL[a * HXY + hl]) + (upR[a * HXY + hr] - dnR[a * HXY + hr])) *
                          (R(0.25) * ci[b]);
            }
        }
    R uL[3], uR[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) { uL[a] = cl[a * HXY + hl]; uR[a] = cr[a * HXY + hr]; }
    visc_core<3, D, R>(g, uL, uR, cl[P.i_mu * HXY + hl], cr[P.i_mu * HXY + hr], cl[P.i_kc * HXY + hl],
                       cr[P.i_kc * HXY + hr], cl[4 * HXY + hl], cr[4 * HXY + hr], ci[D], F);
}

template <int NC, int NT, int MB, int LIM, int VISC, typename Q>
__global__ void __launch_bounds__(NT, MB) zmarch_kernel(ZArgs A)
{
    // FP32 arithmetic on float-float registers, or FP64 throughout
    using R = typename std::conditional<IsFF<Q>::value, float, double>::type;
    constexpr int ND = 3, NV = ND + NC + 1;
    constexpr int TX = ZM_TX, TY = ZM_TY;
    constexpr int HX = TX + 4, HY = TY + 4, HXY = HX * HY;
    constexpr int AX = TX + 2, AY = TY + 2, AXY = AX * AY;
    constexpr int VX = TX + 1, VY = TY + 1, VXY = VX * VY;
    constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1), TXY = TX * TY;
    // face tasks: 32 faces of one direction each (x, y, then z)
    constexpr int TKX = (NFX + 31) / 32, TKY = (NFY + 31) / 32, NTASK = TKX + TKY + TXY / 32;
    static_assert(TXY % 32 == 0 && NT % 32 == 0, "whole warps");
    static_assert(NT >= TXY, "one thread per cell of the column in the update");
    const DevParams& P = A.P;
    const ConstT<R>& Kc = K<R>(P);
    const Q* const q0reg = static_cast<const Q*>(A.q0);
    Q* const qoreg = static_cast<Q*>(A.qout);
    const int tid = threadIdx.x;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    R* const PR = reinterpret_cast<R*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int SS = zm_slot_stride(P.nprim, HXY, int(sizeof(R)));
    R* const FX = PR + 4 * SS;                 // [NV][NFX] x-faces of the plane
    R* const FY = FX + NV * NFX;               // [NV][NFY] y-faces of the plane
    R* const FZ = FY + NV * NFY;               // [2][NV][TXY] z-faces, slot of the plane above the face
    R* const AT = FZ + 2 * NV * TXY;           // [2][AXY] smoothed fractions
    R* const NRM = AT + 2 * AXY;               // [2][3][VXY] vertex normals, slot of the plane above the vertex
    R* const GRD = NRM + 2 * 3 * VXY;          // [2][3][VXY] unsmoothed-fraction vertex gradients, same slots
    unsigned char* const FLAG = reinterpret_cast<unsigned char*>(GRD + 2 * 3 * VXY);   // [2][HXY]
    auto slot4 = [](int p) { return (p + 8) & 3; };
    auto slot2 = [](int p) { return (p + 8) & 1; };
    auto plane = [&](int p) { return PR + slot4(p) * SS; };

    __shared__ __align__(8) unsigned long long mbar[4];
    const unsigned mbar0 = smem_addr(&mbar[0]);
    auto mb = [&](int s) { return mbar0 + 8u * unsigned(s); };
    const unsigned plane_bytes = unsigned(HXY * P.nprim * sizeof(R));
    unsigned phase = 0;   // bit s: parity of slot s's next completion
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) mbar_init(mb(i), 1);
        mbar_init_fence();
    }
    __syncthreads();

    for (int it = blockIdx.x; it < A.nitems; it += gridDim.x) {
        const int4 wi = A.items[it];
        const CaseDesc& C = A.cases[wi.x];
        const int x0 = wi.y, y0 = wi.z, z0 = wi.w;
        const int z1 = min(z0 + A.zc, C.n[2]);
        const int vx = min(TX, C.n[0] - x0), vy = min(TY, C.n[1] - y0);
        const void* const tm = static_cast<const unsigned char*>(A.tmaps) + size_t(wi.x) * TMAP_BYTES;
        R ci[3], cdx[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) { ci[d] = pick<R>(C.idx[d], C.fidx[d]); cdx[d] = pick<R>(C.dx[d], C.fdx[d]); }
        const R gthr = Kc.grad_eps / fmin(cdx[0], fmin(cdx[1], cdx[2]));

        // plane p (interior index, >= -2) into its slot; its ghosted z index is p + 2
        auto issue = [&](int p) {
            if (tid == 0) {
                tmap_acquire(tm);
                fence_async_smem();
                mbar_expect_tx(mb(slot4(p)), plane_bytes);
                tma_load_4d(smem_addr(plane(p)), tm, x0, y0, p + 2, 0, mb(slot4(p)));
            }
        };
        // bounded wait for plane p; false (uniformly) if any thread gave up
        auto wait = [&](int p) -> bool {
            const int s = slot4(p);
            const bool ok = tma_wait(mb(s), (phase >> s) & 1u);
            phase ^= 1u << s;
            return !__syncthreads_or(!ok);
        };
        auto timeout = [&]() {
            if (tid == 0) set_err(A.err, ERR_TIMEOUT);
        };

        // App. D sensor of plane p on the tile + 1 halo in x and y (planes p-1 .. p+1 present)
        // (i0: this thread's first cell, a permutation of the thread indices)
        auto sensor_plane = [&](int p, int i0) {
            const R* const sp = plane(p);
            const R* const sm = plane(p - 1);
            const R* const su = plane(p + 1);
            unsigned char* const fl = FLAG + slot2(p) * HXY;
            for (int i = i0; i < AXY; i += NT) {
                const int hx = i % AX + 1, hy = i / AX + 1;
                if (hx > vx + 2 || hy > vy + 2) continue;
                const int h = hy * HX + hx;
                R g[3][3];
                R tg = R(0);
                const R* const ea = sp + P.i_al * HXY;
                const R e0 = ea[h];
                const R o0 = liq_side(e0);
#pragma unroll
                for (int bd = 0; bd < 3; ++bd) {
                    const R* pp;
                    const R* pm;
                    int hp, hm;
                    if (bd == 0) { pp = sp; pm = sp; hp = h + 1; hm = h - 1; }
                    else if (bd == 1) { pp = sp; pm = sp; hp = h + HX; hm = h - HX; }
                    else { pp = su; pm = sm; hp = h; hm = h; }
                    const R inv2dx = R(0.5) * ci[bd];
#pragma unroll
                    for (int a = 0; a < 3; ++a) g[a][bd] = (pp[a * HXY + hp] - pm[a * HXY + hm]) * inv2dx;
                    const R em = pm[P.i_al * HXY + hm], ep = pp[P.i_al * HXY + hp];
                    tg += fabs((e0 - em) + (o0 - liq_side(em))) + fabs((ep - e0) + (liq_side(ep) - o0));
                }
                R div = R(0);
#pragma unroll
                for (int a = 0; a < 3; ++a) div += g[a][a];
                const R wx = g[2][1] - g[1][2], wy = g[0][2] - g[2][0], wz = g[1][0] - g[0][1];
                const R curl2 = wx * wx + wy * wy + wz * wz;
                const R d2 = div * div;
                const R thD = fdiv(d2, d2 + curl2 + Kc.eps_ducros);
                fl[h] = (thD > Kc.thr_ducros || tg > Kc.thr_gas) ? 1 : 0;
            }
        };
        // CSF smoothed fraction (Eq. 3-9) of plane p on the tile + 1 halo in x and y
        auto smooth_plane = [&](int p, int i0) {
            R* const at = AT + slot2(p) * AXY;
            for (int i = i0; i < AXY; i += NT) {
                const int ax = i % AX, ay = i / AX;
                const int hc = (ay + 1) * HX + ax + 1;
                R s = R(0), W1 = R(0);
#pragma unroll
                for (int c = -1; c <= 1; ++c) {
                    const R* const al = plane(p + c) + P.i_al * HXY;
#pragma unroll
                    for (int b = -1; b <= 1; ++b)
#pragma unroll
                        for (int a = -1; a <= 1; ++a) {
                            const R wt = R((c == 0 ? 2 : 1) * (b == 0 ? 2 : 1) * (a == 0 ? 2 : 1));
                            const R e = al[hc + b * HX + a];
                            s += wt * e;
                            W1 += wt * liq_side(e);
                        }
                }
                const R norm = R(64);
                at[i] = (s + W1 > R(0.5) * norm) ? -(((norm - W1) - s) / norm) : (s + W1) / norm;
            }
        };
        // vertex normals between planes p and p+1 and the unsmoothed-fraction
        // gradient sums at the same vertices (both stored in the slot of p+1)
        auto normals = [&](int p) {
            const R* const alo = AT + slot2(p) * AXY;
            const R* const ahi = AT + slot2(p + 1) * AXY;
            R* const nr = NRM + slot2(p + 1) * 3 * VXY;
            R* const gr = GRD + slot2(p + 1) * 3 * VXY;
            const R* const elo = plane(p) + P.i_al * HXY;
            const R* const ehi = plane(p + 1) + P.i_al * HXY;
            for (int i = tid; i < VXY; i += NT) {
                const int ix = i % VX, iy = i / VX;
                {
                    // cells (ix-1+bx, iy-1+by) of planes p, p+1 (the update's order)
                    R gu[3] = {R(0), R(0), R(0)}, gou[3] = {R(0), R(0), R(0)};
                    const int h = (iy + 1) * HX + ix + 1;
#pragma unroll
                    for (int cc = 0; cc < 8; ++cc) {
                        const int bx = cc & 1, by = (cc >> 1) & 1, bz = (cc >> 2) & 1;
                        const R e = (bz ? ehi : elo)[h + bx + by * HX], oc = liq_side(e);
                        gu[0] += bx ? e : -e; gou[0] += bx ? oc : -oc;
                        gu[1] += by ? e : -e; gou[1] += by ? oc : -oc;
                        gu[2] += bz ? e : -e; gou[2] += bz ? oc : -oc;
                    }
#pragma unroll
                    for (int d = 0; d < 3; ++d) gr[d * VXY + i] = gu[d] + gou[d];
                }
                R g[3] = {R(0), R(0), R(0)}, go[3] = {R(0), R(0), R(0)};
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) {
                    const int bx = cc & 1, by = (cc >> 1) & 1, bz = (cc >> 2) & 1;
                    const R e = (bz ? ahi : alo)[(iy + by) * AX + ix + bx];
                    const R oc = liq_side(e);
                    g[0] += bx ? e : -e; go[0] += bx ? oc : -oc;
                    g[1] += by ? e : -e; go[1] += by ? oc : -oc;
                    g[2] += bz ? e : -e; go[2] += bz ? oc : -oc;
                }
                R mag2 = R(0);
#pragma unroll
                for (int d = 0; d < 3; ++d) { g[d] = (g[d] + go[d]) * ci[d] * R(2.0 / 8); mag2 += g[d] * g[d]; }
                const R mag = sq_rt(mag2);
                const R inv = (mag > gthr) ? frcp(mag) : R(0);
#pragma unroll
                for (int d = 0; d < 3; ++d) nr[d * VXY + i] = g[d] * inv;
            }
        };
        // face f (0-based within its direction) of direction d (x- and y-faces
        // of plane p, or the z-face between planes p and p+1, stored in the slot
        // of p+1): the four stencil cells as offsets into the plane ring, the
        // sensor flags and impedance inputs of the middle two; one code path
        // for the three directions
        auto face_task = [&](int d, int f, int p) {
            int fx, fy, h0, sh;
            if (d == 0) {
                fx = f % (TX + 1); fy = f / (TX + 1);
                if (f >= NFX || fx > vx || fy >= vy) return;
                h0 = (fy + 2) * HX + fx; sh = 1;
            } else if (d == 1) {
                fx = f % TX; fy = f / TX;
                if (f >= NFY || fx >= vx || fy > vy) return;
                h0 = fy * HX + fx + 2; sh = HX;
            } else {
                fx = f % TX; fy = f / TX;
                if (fx >= vx || fy >= vy) return;
                h0 = (fy + 2) * HX + fx + 2; sh = 0;
            }
            int off[4];
#pragma unroll
            for (int st = 0; st < 4; ++st) off[st] = slot4(d == 2 ? p - 1 + st : p) * SS + h0 + st * sh;
            R ws[4][NV];
            R r4[4], c4[4];
#pragma unroll
            for (int st = 0; st < 4; ++st)
#pragma unroll
                for (int v = 0; v < NV; ++v) ws[st][v] = PR[off[st] + v * HXY];
            int fl = 1;
            if (P.iles) {
#pragma unroll
                for (int st = 1; st <= 2; ++st) {
                    r4[st] = PR[off[st] + P.i_rho * HXY];
                    c4[st] = PR[off[st] + P.i_c * HXY];
                }
                const int h1 = h0 + sh, h2 = h0 + 2 * sh;
                fl = (FLAG[slot2(p) * HXY + h1] | FLAG[slot2(d == 2 ? p + 1 : p) * HXY + h2]) ? 1 : 0;
            }
            R F[NV];
            if (!face_flux<ND, NC, R, false, LIM>(P, d, ws, r4, c4, fl, F)) set_err(A.err, ERR_NONPHYS);
            if (VISC && P.visc) {
                const R* const pz = plane(p);
                const int h1 = h0 + sh, h2 = h0 + 2 * sh;
                if (d == 0)
                    zm_visc_face<0, R>(P, HXY, HX, pz, h1, pz, h2, plane(p - 1), plane(p + 1), plane(p - 1),
                                       plane(p + 1), ci, F);
                else if (d == 1)
                    zm_visc_face<1, R>(P, HXY, HX, pz, h1, pz, h2, plane(p - 1), plane(p + 1), plane(p - 1),
                                       plane(p + 1), ci, F);
                else
                    zm_visc_face<2, R>(P, HXY, HX, pz, h1, plane(p + 1), h1, nullptr, nullptr, nullptr, nullptr, ci, F);
            }
            R* const dst = d == 0 ? FX + f : (d == 1 ? FY + f : FZ + slot2(p + 1) * NV * TXY + f);
            const int ds = d == 0 ? NFX : (d == 1 ? NFY : TXY);
#pragma unroll
            for (int v = 0; v < NV; ++v) dst[v * ds] = F[v];
        };

        // ---- prologue: planes z0-2 .. z0+1, sensor and smoothed fractions of
        // planes z0-1 and z0; the loop's first pass (z = z0-1) computes the
        // normals and z-faces between them and nothing else of plane z0-1
        issue(z0 - 2);
        issue(z0 - 1);
        issue(z0);
        issue(z0 + 1);
        bool ok = true;
        for (int p = z0 - 2; p <= z0 + 1; ++p) ok = wait(p) && ok;
        if (!ok) { timeout(); return; }
        if (P.iles) { sensor_plane(z0 - 1, tid); sensor_plane(z0, tid); }
        if (P.csf) { smooth_plane(z0 - 1, tid); smooth_plane(z0, tid); }
        __syncthreads();

        const double adt = A.a * A.dt[wi.x];
        const float adtf = float(adt);
        const int cx = tid % TX, cy = tid / TX;
        // the case's fields in registers (the loop stores to q^k, which the
        // compiler cannot tell apart from the case table)
        const long long qoff = C.qoff;
        const int n0 = C.n[0], n1 = C.n[1];
        // the threads without a cell to update take the first sensor and
        // smoothing cells of the next plane; the sensor's and the smoothing's
        // cells beyond the first round go to different threads
        const int rot = tid >= TXY ? tid - TXY : tid + (NT - TXY);
        constexpr int XTRA = AXY > NT ? AXY - NT : 0;
        const int rot_s = rot >= XTRA ? rot - XTRA : rot + (NT - XTRA);
        for (int z = z0 - 1; z < z1; ++z) {
            const bool upd = z >= z0;
            const bool own = upd && tid < TXY && cx < vx && cy < vy;
            const long long gcell = qoff + (((long long)(upd ? z : z0) * n1 + (y0 + cy)) * n0 + (x0 + cx));
            Q q0r[NV];
            {
                const Q* qp = q0reg + gcell;
#pragma unroll
                for (int v = 0; v < NV; ++v) { q0r[v] = own ? *qp : Q{}; qp += P.ntot_q; }
            }
            // planes z-1 .. z+2 and the flags and smoothed fractions of planes z
            // and z+1 are in place (previous step or prologue).
            // normals between z and z+1; x- and y-faces of plane z; z-faces between z and z+1
            if (P.csf) normals(z);
            {
                // faces in warp tasks of 32 faces of one direction (no warp
                // runs two directions' code one after the other); the last
                // warps take the extra tasks, the first ones any extra vertex
                // normals above
                const int lane = tid & 31;
                for (int t = NT / 32 - 1 - (tid >> 5); t < NTASK; t += NT / 32) {
                    const int d = t < TKX ? 0 : (t < TKX + TKY ? 1 : 2);
                    const int f = (t - (d == 0 ? 0 : (d == 1 ? TKX : TKX + TKY))) * 32 + lane;
                    if (!upd && d != 2) continue;
                    if constexpr (sizeof(R) == 8) {
                        // FP64: one copy of the face code (the direction's
                        // selects are integer work beside the FP64 pipe)
                        face_task(d, f, z);
                    } else {
                        // FP32: the direction at compile time in each copy
                        if (d == 0) face_task(0, f, z);
                        else if (d == 1) face_task(1, f, z);
                        else face_task(2, f, z);
                    }
                }
            }
            __syncthreads();
            // plane z-1 is no longer read: its slot takes plane z+3 while the update runs
            const bool more = z + 1 < z1;
            if (more) issue(z + 3);
            // divergence, CSF source and LSRK update of plane z
            if (own) {
                R S[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) S[v] = R(0);
                const int hc = (cy + 2) * HX + cx + 2;
                if (P.csf) {
                    R kappa = R(0);
                    R ga[3] = {R(0), R(0), R(0)};
#pragma unroll
                    for (int vtx = 0; vtx < 8; ++vtx) {
                        const int ox = vtx & 1, oy = (vtx >> 1) & 1, oz = (vtx >> 2) & 1;
                        const int vi = (cy + oy) * VX + cx + ox;
                        const R* const gr = GRD + slot2(z + oz) * 3 * VXY + vi;
                        const R gu[3] = {gr[0], gr[VXY], gr[2 * VXY]};
                        const R* const nr = NRM + slot2(z + oz) * 3 * VXY + vi;
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            const R nd_ = nr[d * VXY];
                            const int od = d == 0 ? ox : (d == 1 ? oy : oz);
                            kappa -= (od ? nd_ : -nd_) * ci[d] * R(2.0 / 8);
                            ga[d] += gu[d] * ci[d] * R(2.0 / 8);
                        }
                    }
                    R udg = R(0);
                    const R* const pz = plane(z);
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        ga[d] *= R(1.0 / 8);
                        S[1 + d] = Kc.sigma * kappa * ga[d];
                        udg += pz[d * HXY + hc] * ga[d];
                    }
                    S[1 + ND] = Kc.sigma * kappa * udg;
                }
                if (VISC && P.grav) {
                    // Eq. 2-2 Q: rho g (momentum), rho u . g (energy)
                    const R* const pz = plane(z);
                    const R rho = pz[P.i_rho * HXY + hc];
                    R ug = R(0);
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        S[1 + d] += rho * Kc.grav[d];
                        ug += pz[d * HXY + hc] * Kc.grav[d];
                    }
                    S[1 + ND] += rho * ug;
                }
                const int fxl = cy * (TX + 1) + cx, fyl = cy * TX + cx, c = cy * TX + cx;
                const R* const fzl = FZ + slot2(z) * NV * TXY;
                const R* const fzu = FZ + slot2(z + 1) * NV * TXY;
                Q* qo = qoreg + gcell;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    R div = (FX[v * NFX + fxl + 1] - FX[v * NFX + fxl]) * ci[0];
                    div += (FY[v * NFY + fyl + TX] - FY[v * NFY + fyl]) * ci[1];
                    div += (fzu[v * TXY + c] - fzl[v * TXY + c]) * ci[2];
                    const R Rv = S[v] - div;
                    *qo = lsrk_update(q0r[v], adt, adtf, Rv);
                    qo += P.ntot_q;
                }
            }
            // then, for the next step, plane z+3 and the flags and smoothed
            // fractions of plane z+2 (they overwrite plane z's, read last in
            // this step's faces); one barrier closes the step
            bool ok_next = true;
            if (more) {
                const int sl = slot4(z + 3);
                ok_next = tma_wait(mb(sl), (phase >> sl) & 1u);
                phase ^= 1u << sl;
                if (ok_next) {
                    if (P.iles) sensor_plane(z + 2, rot);
                    if (P.csf) smooth_plane(z + 2, rot_s);
                }
            }
            if (__syncthreads_or(!ok_next)) { timeout(); return; }
        }
        __syncthreads();   // the next item's prologue rewrites every ring
    }
}

}  // namespace tfv
