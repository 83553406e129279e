// fv_march.cuh -- fused stage kernel for 2D grids in plain mode (no App. D
// switch, no CSF, stiffened/ideal-gas closure): one pass per LSRK stage that
// reads the stage's input register q^{k-1}, recovers the primitives (App. B)
// with the boundary update, reconstructs, does the TDU and the all-Mach flux
// on every face and writes q^k = q^0 + a_k dt R (Algorithm 1, Sec. 3.1).
//
// Layout of the work: each warp owns a strip of 32 columns -- lanes 2..29 are
// the strip's cells, lanes 0, 1, 30, 31 its halo -- and marches along y over
// a chunk of rows, keeping the four rows of the y-face stencil in registers.
// The x-face stencil comes from neighbouring lanes (warp shuffles), the y-face
// flux of the previous row is carried in registers, so the kernel uses no
// shared memory and no block barrier, and no primitive field goes through HBM.
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
};

constexpr int MARCH_COLS = 28;   // cells per strip (32 lanes minus 2 + 2 halo)

// Inflow-disc test of an x-low ghost cell in source row iy (FP64, the same
// expression as the primitive pass).  Not inlined: only lanes on an inflow
// boundary call it, and inlined the compiler evaluated it on every row.
static __device__ __noinline__ bool march_in_disc(const CaseDesc& C, int iy)
{
    const double yy = (iy + 0.5) * C.dx[1] - C.in_yc;
    return yy * yy <= C.in_r2;
}

template <int NC, typename R, int NWARP, int MB, int LIM, typename Q>
__global__ void __launch_bounds__(32 * NWARP, MB) march2d_kernel(MarchArgs A)
{
    constexpr int ND = 2, NV = ND + NC + 1;
    const DevParams& P = A.P;
    const Q* const qin = static_cast<const Q*>(A.qin);
    const Q* const q0reg = static_cast<const Q*>(A.q0);
    Q* const qoreg = static_cast<Q*>(A.qout);
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (int it = blockIdx.x * NWARP + (threadIdx.x >> 5); it < A.nitems; it += gridDim.x * NWARP) {
        const int4 wi = A.items[it];
        const CaseDesc& C = A.cases[wi.x];
        const int n0 = C.n[0], n1 = C.n[1];
        // this lane's column and its boundary mapping (fixed along the strip)
        const int col = wi.y - 2 + lane;
        int fx, inx;
        const int ix = map_index(n0, col, C.bc[0][0], C.bc[0][1], fx, inx);
        const bool own_col = lane >= 2 && lane < 30 && col < n0;
        const bool own_right = lane >= 1 && lane < 29 && col + 1 < n0;   // lane + 1 owns a cell
        const R ci0 = pick<R>(C.idx[0], C.fidx[0]), ci1 = pick<R>(C.idx[1], C.fidx[1]);
        const Q* const qcase = qin + C.qoff;

        // primitives (u, v, p', T, Y) of this lane's cell in row y, ghosts
        // through the boundary update exactly as the primitive pass does it;
        // the row's conserved values are fetched one row ahead (fetch_row)
        // and recovered when the row enters the window (recover_row)
        struct RowRef { int iy, fy, disc; };
        auto fetch_row = [&](int y, Q* qc, RowRef& rr) {
            int iny;
            rr.iy = map_index(n1, y, C.bc[1][0], C.bc[1][1], rr.fy, iny);
            rr.disc = inx ? (march_in_disc(C, rr.iy) ? 1 : 0) : 0;
            const Q* qp = qcase + (rr.iy * n0 + (rr.disc ? 0 : ix));
#pragma unroll
            for (int v = 0; v < NV; ++v) { qc[v] = *qp; qp += P.ntot_q; }
        };
        auto recover_row = [&](const Q* qc, const RowRef& rr, R* w) {
            R rho, T, pabs;
            const int rst = prim_recover<ND, NC, R, false, Q>(P, qc, w, rho, T, pabs, 0.0);
            if (rst) set_err(A.err, rst == ERR_NONCONV ? ERR_NONCONV : ERR_NONPHYS);
            if (inx ? !rr.disc : fx) w[0] = -w[0];
            if (rr.fy) w[1] = -w[1];
            if (rr.disc) {
                const long long fc = rr.iy, fn = n1;
#pragma unroll
                for (int a = 0; a < ND; ++a) w[a] = R(C.in_uoff >= 0 ? A.in_u[C.in_uoff + a * fn + fc] : C.in_u0[a]);
                w[ND + 1] = R(C.in_T);
#pragma unroll
                for (int k = 0; k < NC - 1; ++k) w[ND + 2 + k] = R(C.in_Y[k]);
                R r_, e_, c_;
                if (!tdu<NC, R, false>(P, w[ND], w[ND + 1], w + ND + 2, r_, e_, c_)) set_err(A.err, ERR_NONPHYS);
            }
        };
        auto load_row = [&](int y, R* w) {
            Q qc[NV];
            RowRef rr;
            fetch_row(y, qc, rr);
            recover_row(qc, rr, w);
        };

        const int y0 = wi.z, y1 = min(wi.z + wi.w, n1);
        R W[4][NV];
        load_row(y0 - 2, W[0]);
        load_row(y0 - 1, W[1]);
        load_row(y0, W[2]);
        load_row(y0 + 1, W[3]);
        R r4[4], c4[4];   // App. D impedance inputs (unused in plain mode)
        R Fy[NV];
        {
            const bool ok = face_flux<ND, NC, R, false, LIM>(P, 1, W, r4, c4, 1, Fy);
            if (!ok && own_col) set_err(A.err, ERR_NONPHYS);
        }
        const double adt = A.a * A.dt[wi.x];
        const float adtf = float(adt);
        Q qn[NV];          // conserved values of the next row to enter the window
        RowRef rn;
        fetch_row(y0 + 2, qn, rn);
        for (int y = y0; y < y1; ++y) {
            // q^0 of this lane's cell, loaded early so its latency hides
            Q q0r[NV];
            const long long gcell = C.qoff + ((long long)y * n0 + (own_col ? col : 0));
            {
                const Q* qp = q0reg + gcell;
#pragma unroll
                for (int v = 0; v < NV; ++v) { q0r[v] = own_col ? *qp : Q{}; qp += P.ntot_q; }
            }
            // advance the window: rows y-1 .. y+2; fetch row y+3 for the next round
#pragma unroll
            for (int v = 0; v < NV; ++v) { W[0][v] = W[1][v]; W[1][v] = W[2][v]; W[2][v] = W[3][v]; }
            recover_row(qn, rn, W[3]);
            if (y + 1 < y1) fetch_row(y + 3, qn, rn);
            // y face y+1/2
            R Fyn[NV];
            {
                const bool ok = face_flux<ND, NC, R, false, LIM>(P, 1, W, r4, c4, 1, Fyn);
                if (!ok && own_col) set_err(A.err, ERR_NONPHYS);
            }
            // x face between this lane's cell and the next, row y
            R ws[4][NV], Fx[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                ws[1][v] = W[1][v];
                ws[0][v] = __shfl_up_sync(FULL, W[1][v], 1);
                ws[2][v] = __shfl_down_sync(FULL, W[1][v], 1);
                ws[3][v] = __shfl_down_sync(FULL, W[1][v], 2);
            }
            {
                const bool ok = face_flux<ND, NC, R, false, LIM>(P, 0, ws, r4, c4, 1, Fx);
                if (!ok && (own_col || own_right)) set_err(A.err, ERR_NONPHYS);
            }
            // divergence and LSRK update of this lane's cell
            Q* qo = qoreg + gcell;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const R Fxm = __shfl_up_sync(FULL, Fx[v], 1);
                R div = (Fx[v] - Fxm) * ci0;
                div += (Fyn[v] - Fy[v]) * ci1;
                const R Rv = R(0) - div;
                if (own_col) *qo = lsrk_update(q0r[v], adt, adtf, Rv);
                qo += P.ntot_q;
                Fy[v] = Fyn[v];
            }
        }
    }
}

}  // namespace tfv
