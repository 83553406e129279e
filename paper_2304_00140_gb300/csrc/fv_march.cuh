// fv_march.cuh -- fused stage kernel for 2D grids with the stiffened/ideal-gas
// closure: one pass per LSRK stage that reads the stage's input register
// q^{k-1}, recovers the primitives (App. B) with the boundary update,
// evaluates the App. D sensor (Eq. D.4) and the CSF source (Sec. 3.5,
// Eq. 3-9/3-10), reconstructs, does the TDU and the all-Mach flux on every
// face and writes q^k = q^0 + a_k dt R (Algorithm 1, Sec. 3.1).
//
// Layout of the work: each warp owns a strip of 32 columns -- lanes 2..29 are
// the strip's cells, lanes 0, 1, 30, 31 its halo -- and marches along y over
// a chunk of rows, keeping the four rows y-1 .. y+2 in registers.  Neighbours
// in x come from other lanes (warp shuffles); per-row quantities that the
// next row needs (the y-flux, the sensor flag, the smoothed fraction and the
// vertex normals of the row's upper edge) are carried in registers.  The
// kernel uses no shared memory and no block barrier, and no primitive field
// goes through HBM.  Every formula follows the tiled kernel's operation
// order, so both give the same sensor decisions and the same rounding.
#pragma once

#include "fv_kernels.cuh"

namespace tfv {

struct MarchArgs {
    DevParams P;
    const CaseDesc* cases;
    const int4* items;        // (case, first strip column, first row, rows)
    int nitems;
    const void* qin;          // q^{k-1} (double or float2; field stride P.ntot_q)
    const void* q0;           // q^0
    void* qout;               // q^k
    const double* in_u;       // inflow velocities (device) or null
    const double* dt;         // per-case dt
    double a;                 // LSRK coefficient a_k
    int* err;
    unsigned long long* smax; // MARCH_CFL: per-case max wave speed bits of q^k (the next step's CFL input)
};

constexpr int MARCH_COLS = 28;   // cells per strip (32 lanes minus 2 + 2 halo)
// scheme features of a fused-kernel instantiation (MARCH_VISC: the Eq. 2-2
// stress, heat-flux and gravity terms)
constexpr int MARCH_ILES = 1, MARCH_CSF = 2, MARCH_VISC = 4;
// MARCH_CFL (last stage, plain viscosity-free modes): the kernel also
// recovers the primitives of the q^k it writes and accumulates the CFL wave
// speed sum_d (|u_d| + c) / dx_d of every interior cell into smax, as the
// CFL pass of the next step would from the same values, so that pass is
// left out
constexpr int MARCH_CFL = 8;
// MARCH_BARO (plain mode, FP32-mixed form): the barotropic closure (Sec.
// 2.2) with the liquid-vapour density THINC (Sec. 3.4): each window row also
// carries the cell density, sound speed and vapour fraction of Eq. 2-7, as
// the primitive pass writes them for the tiled kernel
constexpr int MARCH_BARO = 16;

// Inflow-disc test of an x-low ghost cell in source row iy (FP64, the same
// expression as the primitive pass).  Not inlined: only lanes on an inflow
// boundary call it, and inlined the compiler evaluated it on every row.
static __device__ __noinline__ bool march_in_disc(const CaseDesc& C, int iy)
{
    const double yy = (iy + C.org[1] + 0.5) * C.dx[1] - C.in_yc;
    return yy * yy <= C.in_r2;
}

// one row of the window: primitives, and for App. D / CSF the cell density,
// sound speed and encoded liquid fraction (e = alpha_l, or -alpha_g when the
// gas is the smaller side; see the primitive pass)
template <int NV, typename R> struct MRow {
    R w[NV];
    R rho, c, e;
    R mu, kc;    // mixture viscosity and conductivity (viscous mode)
    R av;        // vapour fraction (barotropic mode)
};

template <int NC, typename R, int NWARP, int MB, int LIM, int MODE, typename Q>
__global__ void __launch_bounds__(32 * NWARP, MB) march2d_kernel(MarchArgs A)
{
    constexpr int ND = 2, NV = ND + NC + 1;
    constexpr bool ILES = (MODE & MARCH_ILES) != 0, CSF = (MODE & MARCH_CSF) != 0, AUX = ILES || CSF;
    constexpr bool VISC = (MODE & MARCH_VISC) != 0;
    constexpr bool CFLM = (MODE & MARCH_CFL) != 0;
    constexpr bool BARO = (MODE & MARCH_BARO) != 0;
    constexpr int CL = BARO ? CL_BARO : CL_SG;
    static_assert(!(CFLM && VISC), "the fused CFL speed has no diffusive term");
    static_assert(!(BARO && (AUX || VISC)), "the barotropic mode is plain");
    const DevParams& P = A.P;
    const ConstT<R>& Kc = K<R>(P);
    // q^{k-1} never aliases q^k (the stages go q0 -> qA -> qB -> qA -> q0)
    const Q* __restrict__ const qin = static_cast<const Q*>(A.qin);
    const Q* const q0reg = static_cast<const Q*>(A.q0);
    Q* const qoreg = static_cast<Q*>(A.qout);
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (int it = blockIdx.x * NWARP + (threadIdx.x >> 5); it < A.nitems; it += gridDim.x * NWARP) {
        const int4 wi = A.items[it];
        const CaseDesc& C = A.cases[wi.x];
        // the case's fields in registers (the row loop stores to q^k, which the
        // compiler cannot tell apart from the case table)
        const int n0 = C.n[0], n1 = C.n[1];
        const int bcy0 = C.bc[1][0], bcy1 = C.bc[1][1];
        const long long qoff = C.qoff;
        // this lane's column and its boundary mapping (fixed along the strip)
        const int col = wi.y - 2 + lane;
        int fx, inx;
        const int ix = map_index(n0, col, C.bc[0][0], C.bc[0][1], fx, inx);
        const bool own_col = lane >= 2 && lane < 30 && col < n0;
        const bool own_right = lane >= 1 && lane < 29 && col + 1 < n0;   // lane + 1 owns a cell
        const R ci0 = pick<R>(C.idx[0], C.fidx[0]), ci1 = pick<R>(C.idx[1], C.fidx[1]);
        const Q* __restrict__ const qcase = qin + qoff;

        // a row enters the window in two parts: its conserved values are
        // fetched one row ahead (fetch_row) and recovered when it enters
        // (recover_row), ghosts through the boundary update exactly as the
        // primitive pass does it
        struct RowRef { int iy, fy, disc; };
        auto fetch_row = [&](int y, Q* qc, RowRef& rr) {
            int iny;
            rr.iy = map_index(n1, y, bcy0, bcy1, rr.fy, iny);
            rr.disc = inx ? (march_in_disc(C, rr.iy) ? 1 : 0) : 0;
            const Q* qp = qcase + (rr.iy * n0 + (rr.disc ? 0 : ix));
#pragma unroll
            for (int v = 0; v < NV; ++v) { qc[v] = *qp; qp += P.ntot_q; }
        };
        // non-physical states met by this lane in this work item (reported once
        // at its end instead of at every face)
        bool bad = false;
        auto recover_row = [&](const Q* qc, const RowRef& rr, MRow<NV, R>& row) {
            R* const w = row.w;
            R rho, T, pabs;
            const int rst = prim_recover<ND, NC, R, CL, Q>(P, qc, w, rho, T, pabs, 0.0);
            bool ok = rst == 0;
            if (rst == ERR_NONCONV) set_err(A.err, ERR_NONCONV);
            if (inx ? !rr.disc : fx) w[0] = -w[0];
            if (rr.fy) w[1] = -w[1];
            if (rr.disc) {
                const long long fc = rr.iy, fn = C.in_ustride;
#pragma unroll
                for (int a = 0; a < ND; ++a) w[a] = R(C.in_uoff >= 0 ? A.in_u[C.in_uoff + a * fn + fc] : C.in_u0[a]);
                w[ND + 1] = R(C.in_T);
#pragma unroll
                for (int k = 0; k < NC - 1; ++k) w[ND + 2 + k] = R(C.in_Y[k]);
            }
            R rr_ = rho, cs = R(0);
            if (ILES || BARO || rr.disc) {
                R e_;
                ok = tdu<NC, R, CL>(P, w[ND], w[ND + 1], w + ND + 2, rr_, e_, cs) && ok;
                if (!rr.disc) rr_ = rho;
            }
            bad = bad || (!ok && rst != ERR_NONCONV);
            row.rho = rr_;
            row.c = cs;
            if constexpr (BARO) row.av = baro_vapour<NC, R>(P, w[ND], rr_, w + ND + 2);
            if (AUX) {
                R s = R(0), al = R(0), ag = R(0);
#pragma unroll
                for (int k = 0; k < NC - 1; ++k) s += clip01(w[ND + 2 + k]);
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    const R Yk = (k == NC - 1) ? clip01(R(1) - s) : clip01(w[ND + 2 + k]);
                    const R a = fdiv(rr_ * Yk * Kc.gm1cv[k] * w[ND + 1], Kc.Pk[k] + w[ND]);
                    if (k == P.liquid) al = a; else ag += a;
                }
                row.e = (al <= ag) ? al : -ag;
            } else {
                row.e = R(0);
            }
            if (VISC) {
                // Eq. 2-8 with no vapour, as the primitive pass computes it
                R s = R(0), mu = R(0), kc = R(0);
#pragma unroll
                for (int k = 0; k < NC - 1; ++k) s += clip01(w[ND + 2 + k]);
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    const R Yk = (k == NC - 1) ? clip01(R(1) - s) : clip01(w[ND + 2 + k]);
                    const R a = fdiv(rr_ * Yk * Kc.gm1cv[k] * w[ND + 1], Kc.Pk[k] + w[ND]);
                    mu += a * Kc.mu[k];
                    kc += a * Kc.kc[k];
                }
                row.mu = mu;
                row.kc = kc;
            }
        };
        auto shl = [&](R v) { return __shfl_up_sync(FULL, v, 1); };     // value of lane - 1
        auto shr = [&](R v) { return __shfl_down_sync(FULL, v, 1); };   // value of lane + 1
        // Eq. 2-2 stress and heat flux of the y face between window rows 1 and 2
        // and of the x face between this lane's and the next lane's cell of row
        // 1, with the tiled kernel's face gradients and operation order
        auto visc_y = [&](const MRow<NV, R>* Wr, R* F) {
            R g[2][2];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                g[a][1] = (Wr[2].w[a] - Wr[1].w[a]) * ci1;
                g[a][0] = ((shr(Wr[1].w[a]) - shl(Wr[1].w[a])) + (shr(Wr[2].w[a]) - shl(Wr[2].w[a]))) * (R(0.25) * ci0);
            }
            visc_core<2, 1, R>(g, Wr[1].w, Wr[2].w, Wr[1].mu, Wr[2].mu, Wr[1].kc, Wr[2].kc, Wr[1].w[ND + 1],
                               Wr[2].w[ND + 1], ci1, F);
        };
        auto visc_x = [&](const MRow<NV, R>* Wr, R* F) {
            R g[2][2], uR[2];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                uR[a] = shr(Wr[1].w[a]);
                g[a][0] = (uR[a] - Wr[1].w[a]) * ci0;
                const R dL = Wr[2].w[a] - Wr[0].w[a];
                g[a][1] = (dL + shr(dL)) * (R(0.25) * ci1);
            }
            visc_core<2, 0, R>(g, Wr[1].w, uR, Wr[1].mu, shr(Wr[1].mu), Wr[1].kc, shr(Wr[1].kc), Wr[1].w[ND + 1],
                               shr(Wr[1].w[ND + 1]), ci0, F);
        };

        // App. D cell sensor f (Eq. D.4) of window row m (rows m-1 .. m+1)
        auto sensor = [&](const MRow<NV, R>* Wr, int m) -> int {
            R g[2][2];
            R tg = R(0);
            const R e0 = Wr[m].e;
            const R o0 = liq_side(e0);
            {
                const R inv2dx = R(0.5) * ci0;
#pragma unroll
                for (int a = 0; a < ND; ++a) g[a][0] = (shr(Wr[m].w[a]) - shl(Wr[m].w[a])) * inv2dx;
                const R em = shl(e0), ep = shr(e0);
                tg += fabs((e0 - em) + (o0 - liq_side(em))) + fabs((ep - e0) + (liq_side(ep) - o0));
            }
            {
                const R inv2dx = R(0.5) * ci1;
#pragma unroll
                for (int a = 0; a < ND; ++a) g[a][1] = (Wr[m + 1].w[a] - Wr[m - 1].w[a]) * inv2dx;
                const R em = Wr[m - 1].e, ep = Wr[m + 1].e;
                tg += fabs((e0 - em) + (o0 - liq_side(em))) + fabs((ep - e0) + (liq_side(ep) - o0));
            }
            R div = R(0);
#pragma unroll
            for (int a = 0; a < ND; ++a) div += g[a][a];
            const R wz = g[1][0] - g[0][1];
            const R curl2 = wz * wz;
            const R d2 = div * div;
            const R thD = fdiv(d2, d2 + curl2 + Kc.eps_ducros);
            return (thD > Kc.thr_ducros || tg > Kc.thr_gas) ? 1 : 0;
        };
        // CSF smoothed fraction (Eq. 3-9) of window row m, encoded like e
        auto smooth = [&](const MRow<NV, R>* Wr, int m) -> R {
            R s = R(0), W1 = R(0);
#pragma unroll
            for (int b = -1; b <= 1; ++b) {
                const R ec = Wr[m + b].e;
                const R el = shl(ec), er = shr(ec);
                const R wb = R(b == 0 ? 2 : 1);
                s += wb * el;
                W1 += wb * liq_side(el);
                s += (R(2) * wb) * ec;
                W1 += (R(2) * wb) * liq_side(ec);
                s += wb * er;
                W1 += wb * liq_side(er);
            }
            const R norm = R(16);
            return (s + W1 > R(0.5) * norm) ? -(((norm - W1) - s) / norm) : (s + W1) / norm;
        };
        const R cdx0 = pick<R>(C.dx[0], C.fdx[0]), cdx1 = pick<R>(C.dx[1], C.fdx[1]);
        const R gthr = Kc.grad_eps / fmin(cdx0, cdx1);
        // vertex between this lane's and the next lane's cells of two rows,
        // values (lo row: a0, a1 = lane+1; hi row: b0, b1): gradient sums of
        // the encoded fraction with the liquid-side offsets summed apart
        auto vgrad = [&](R a0, R a1, R b0, R b1, R* gu) {
            R g0 = R(0), g1 = R(0), o0 = R(0), o1 = R(0);
            const R ev[4] = {a0, a1, b0, b1};
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int bx = cc & 1, by = (cc >> 1) & 1;
                const R e = ev[cc], oc = liq_side(e);
                g0 += bx ? e : -e; o0 += bx ? oc : -oc;
                g1 += by ? e : -e; o1 += by ? oc : -oc;
            }
            gu[0] = g0 + o0;
            gu[1] = g1 + o1;
        };
        // unit normal at that vertex from the smoothed fractions of two rows
        auto vnormal = [&](R alo, R ahi, R* n) {
            R g[2];
            vgrad(alo, shr(alo), ahi, shr(ahi), g);
            g[0] = g[0] * ci0 * R(0.5);
            g[1] = g[1] * ci1 * R(0.5);
            R mag2 = R(0);
            mag2 += g[0] * g[0];
            mag2 += g[1] * g[1];
            const R mag = sq_rt(mag2);
            const R inv = (mag > gthr) ? frcp(mag) : R(0);
            n[0] = g[0] * inv;
            n[1] = g[1] * inv;
        };

        const int y0 = wi.z, y1 = min(wi.z + wi.w, n1);
        MRow<NV, R> W[4];
        {
            Q qc[NV];
            RowRef rr;
#pragma unroll
            for (int m = 0; m < 4; ++m) { fetch_row(y0 - 2 + m, qc, rr); recover_row(qc, rr, W[m]); }
        }
        // carried per-row quantities of row y
        int flag_y = 1;          // App. D sensor
        R at_y = R(0);           // smoothed fraction
        R nlo[2] = {R(0), R(0)}; // unit normal at the vertex (lane + 1/2, y - 1/2)
        R r4[4] = {R(0), R(0), R(0), R(0)}, c4[4] = {R(0), R(0), R(0), R(0)};
        R a4[4] = {R(0), R(0), R(0), R(0)};   // vapour fractions (barotropic mode)
        // barotropic mode: densities and vapour fractions of the four cells of a y-face's stencil
        auto baro_y = [&]() {
#pragma unroll
            for (int s = 0; s < 4; ++s) { r4[s] = W[s].rho; a4[s] = W[s].av; }
        };
        R Fy[NV];
        {
            int flag_lo = 1;
            if (ILES) { flag_lo = sensor(W, 1); flag_y = sensor(W, 2); }
            if (CSF) {
                const R at_lo = smooth(W, 1);
                at_y = smooth(W, 2);
                vnormal(at_lo, at_y, nlo);
            }
            R ws[4][NV];
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int v = 0; v < NV; ++v) ws[s][v] = W[s].w[v];
            if (ILES) { r4[1] = W[1].rho; r4[2] = W[2].rho; c4[1] = W[1].c; c4[2] = W[2].c; }
            if (BARO) baro_y();
            const bool ok = face_flux<ND, NC, R, CL, LIM, ILES ? 1 : 0>(P, 1, ws, r4, c4, flag_lo | flag_y, Fy, a4);
            bad = bad || (!ok && own_col);
            if (VISC && P.visc) visc_y(W, Fy);
        }
        const double adt = A.a * A.dt[wi.x];
        const float adtf = float(adt);
        R speed = R(0);    // MARCH_CFL: largest wave speed sum of this lane's cells
        Q qn[NV];          // conserved values of the next row to enter the window
        RowRef rn;
        fetch_row(y0 + 2, qn, rn);
        for (int y = y0; y < y1; ++y) {
            // q^0 of this lane's cell, loaded early so its latency hides
            Q q0r[NV];
            const long long gcell = qoff + ((long long)y * n0 + (own_col ? col : 0));
            {
                const Q* qp = q0reg + gcell;
#pragma unroll
                for (int v = 0; v < NV; ++v) { q0r[v] = own_col ? *qp : Q{}; qp += P.ntot_q; }
            }
            // advance the window: rows y-1 .. y+2; fetch row y+3 for the next round
            W[0] = W[1];
            W[1] = W[2];
            W[2] = W[3];
            recover_row(qn, rn, W[3]);
            if (y + 1 < y1) fetch_row(y + 3, qn, rn);
            // sensor of row y+1 (the y face needs rows y and y+1)
            int flag_up = 1;
            if (ILES) flag_up = sensor(W, 2);
            // y face y+1/2
            R Fyn[NV];
            {
                R ws[4][NV];
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int v = 0; v < NV; ++v) ws[s][v] = W[s].w[v];
                if (ILES) { r4[1] = W[1].rho; r4[2] = W[2].rho; c4[1] = W[1].c; c4[2] = W[2].c; }
                if (BARO) baro_y();
                const bool ok = face_flux<ND, NC, R, CL, LIM, ILES ? 1 : 0>(P, 1, ws, r4, c4, flag_y | flag_up, Fyn,
                                                                           a4);
                bad = bad || (!ok && own_col);
                if (VISC && P.visc) visc_y(W, Fyn);
            }
            // x face between this lane's cell and the next, row y
            R Fx[NV];
            {
                R ws[4][NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    ws[1][v] = W[1].w[v];
                    ws[0][v] = shl(W[1].w[v]);
                    ws[2][v] = shr(W[1].w[v]);
                    ws[3][v] = __shfl_down_sync(FULL, W[1].w[v], 2);
                }
                int fl = 1;
                if (ILES) {
                    r4[1] = W[1].rho; r4[2] = shr(W[1].rho);
                    c4[1] = W[1].c; c4[2] = shr(W[1].c);
                    fl = flag_y | __shfl_down_sync(FULL, flag_y, 1);
                }
                if (BARO) {
                    r4[1] = W[1].rho; r4[0] = shl(W[1].rho); r4[2] = shr(W[1].rho);
                    r4[3] = __shfl_down_sync(FULL, W[1].rho, 2);
                    a4[1] = W[1].av; a4[0] = shl(W[1].av); a4[2] = shr(W[1].av);
                    a4[3] = __shfl_down_sync(FULL, W[1].av, 2);
                }
                const bool ok = face_flux<ND, NC, R, CL, LIM, ILES ? 1 : 0>(P, 0, ws, r4, c4, fl, Fx, a4);
                bad = bad || (!ok && (own_col || own_right));
                if (VISC && P.visc) visc_x(W, Fx);
            }
            // CSF source of this lane's cell (momentum, energy)
            R S[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) S[v] = R(0);
            if (CSF) {
                const R at_up = smooth(W, 2);
                R nhi[2];
                vnormal(at_y, at_up, nhi);
                // unsmoothed-fraction gradients at the two right-hand vertices
                R glo[2], ghi[2];
                vgrad(W[0].e, shr(W[0].e), W[1].e, shr(W[1].e), glo);
                vgrad(W[1].e, shr(W[1].e), W[2].e, shr(W[2].e), ghi);
                // the cell's vertices in the tiled kernel's order: (-,-), (+,-), (-,+), (+,+)
                const R nv[4][2] = {{shl(nlo[0]), shl(nlo[1])}, {nlo[0], nlo[1]},
                                    {shl(nhi[0]), shl(nhi[1])}, {nhi[0], nhi[1]}};
                const R gv[4][2] = {{shl(glo[0]), shl(glo[1])}, {glo[0], glo[1]},
                                    {shl(ghi[0]), shl(ghi[1])}, {ghi[0], ghi[1]}};
                R kappa = R(0), ga[2] = {R(0), R(0)};
                const R cis[2] = {ci0, ci1};
#pragma unroll
                for (int vtx = 0; vtx < 4; ++vtx) {
                    const int ox = vtx & 1, oy = (vtx >> 1) & 1;
#pragma unroll
                    for (int d = 0; d < 2; ++d) {
                        const int od = d == 0 ? ox : oy;
                        kappa -= (od ? nv[vtx][d] : -nv[vtx][d]) * cis[d] * R(0.5);
                        ga[d] += gv[vtx][d] * cis[d] * R(0.5);
                    }
                }
                R udg = R(0);
#pragma unroll
                for (int d = 0; d < 2; ++d) {
                    ga[d] *= R(0.25);
                    S[1 + d] = Kc.sigma * kappa * ga[d];
                    udg += W[1].w[d] * ga[d];
                }
                S[1 + ND] = Kc.sigma * kappa * udg;
                at_y = at_up;
                nlo[0] = nhi[0];
                nlo[1] = nhi[1];
            }
            if (VISC && P.grav) {
                // Eq. 2-2 Q: rho g (momentum), rho u . g (energy), the stage's input rho
                const R rho = W[1].rho;
                R ug = R(0);
#pragma unroll
                for (int d = 0; d < 2; ++d) {
                    S[1 + d] += rho * Kc.grav[d];
                    ug += W[1].w[d] * Kc.grav[d];
                }
                S[1 + ND] += rho * ug;
            }
            // divergence and LSRK update of this lane's cell
            Q* qo = qoreg + gcell;
            Q qk[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const R Fxm = shl(Fx[v]);
                R div = (Fx[v] - Fxm) * ci0;
                div += (Fyn[v] - Fy[v]) * ci1;
                const R Rv = S[v] - div;
                qk[v] = lsrk_update(q0r[v], adt, adtf, Rv);
                if (own_col) *qo = qk[v];
                qo += P.ntot_q;
                Fy[v] = Fyn[v];
            }
            if (CFLM && own_col) {
                // the CFL pass's recovery and sound speed of this interior cell
                R w[NV], rho, T, pabs, rr_, e_, cs;
                const int rst = prim_recover<ND, NC, R, CL, Q>(P, qk, w, rho, T, pabs, 0.0);
                if (rst == ERR_NONCONV) set_err(A.err, ERR_NONCONV);
                const bool ok = tdu<NC, R, CL>(P, w[ND], w[ND + 1], w + ND + 2, rr_, e_, cs) && rst == 0;
                bad = bad || (!ok && rst != ERR_NONCONV);
                const R cis[2] = {ci0, ci1};
                R sp = R(0);
#pragma unroll
                for (int d = 0; d < ND; ++d) sp += (fabs(w[d]) + cs) * cis[d];
                speed = fmax(speed, sp);
            }
            flag_y = flag_up;
        }
        if (bad) set_err(A.err, ERR_NONPHYS);
        if (CFLM) {
            // warp maximum, one atomic per work item (positive doubles order like their bit patterns)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) speed = fmax(speed, __shfl_xor_sync(FULL, speed, o));
            if (lane == 0) atomicMax(A.smax + wi.x, (unsigned long long)__double_as_longlong(double(speed)));
        }
    }
}

}  // namespace tfv
