// fv_api.cu -- the C ABI (include/thinc_fv.h): context set-up, device memory
// layout, work lists, the stage sequence and its CUDA-graph replay.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/thinc_fv.h"
#include "fv_march.cuh"
#include "fv_zmarch.cuh"
#include "fv_launch.h"

using namespace tfv;

namespace {

// Jameson-Schmidt-Turkel four-stage low-storage coefficients (the paper
// names a four-stage low-storage Runge-Kutta scheme without coefficients).
const double LSRK_A[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
    size_t cases, items_stage, items_prim, items_march, q0, qa, qb, prim, io, smax, dt, t, err, in_u, partial, tmaps,
        items_z, tmaps_z, total;
    int n_items_stage, n_items_prim, n_items_march, n_items_z;
    long long ntot_q, ntot_p, max_cells, n_in_u;
};

constexpr int MARCH_CHUNK_MIN = 16;                  // shortest row chunk of a fused-kernel work item
constexpr int MARCH_CHUNKS[3] = {16, 32, 64};        // row chunks the tuner tries
constexpr int ZM_CHUNKS[3] = {16, 32, 64};           // z-plane chunks of the z-marching kernel

int tile_x(int nd) { return nd == 2 ? TileShape<2>::X : TileShape<3>::X; }
int tile_y(int nd) { return nd == 2 ? TileShape<2>::Y : TileShape<3>::Y; }
int tile_z(int nd) { return nd == 2 ? TileShape<2>::Z : TileShape<3>::Z; }

long long ntiles(const int* ext, int nd)
{
    long long t = 1;
    const int ts[3] = {tile_x(nd), tile_y(nd), tile_z(nd)};
    for (int d = 0; d < 3; ++d) t *= (ext[d] + ts[d] - 1) / ts[d];
    return t;
}

// A grid split into slabs along its last dimension (Sec. 3.1's compact
// stencil needs two ghost layers): each slab is a case of the context whose
// sides towards its neighbours are BC_HALO.  Their two ghost layers are
// stored next to the slab's cells in every conserved register and copied
// from the neighbour before each stage; every slab takes the whole grid's dt.
struct SplitInfo {
    int last = 0;                      // split dimension (ndim - 1)
    std::vector<int> row0;             // first row (plane) of each slab in the grid
    std::vector<int> nbr_lo, nbr_hi;   // neighbouring slab across each side, -1 = grid boundary
    double dx[3] = {1.0, 1.0, 1.0};    // the grid's cell sizes (slabs use them as they are)
    long long in_stride = 0;           // ny nz of the grid's inflow array, 0 = none
};

}  // namespace

struct fv_ctx {
    int ncases = 0, nd = 0, nc = 0, nv = 0, nprim = 0, mixed = 0;
    int ff = 0;                             // float-float LSRK registers (the mixed form of a context)
    DevParams P{};
    std::vector<fv_grid> grids;
    std::vector<CaseDesc> cases;
    Layout L{};
    unsigned char* base = nullptr;
    bool owns = false;
    CaseDesc* d_cases = nullptr;
    int4* d_items_stage = nullptr;
    int4* d_items_prim = nullptr;
    double *Q0 = nullptr, *QA = nullptr, *QB = nullptr;
    void* prim = nullptr;
    double* io = nullptr;
    unsigned long long* smax = nullptr;
    double* dt = nullptr;
    double* t = nullptr;
    int* err = nullptr;
    double* in_u = nullptr;
    double* partial = nullptr;
    cudaStream_t stream = nullptr;          // user stream (0 = legacy default)
    cudaStream_t cap = nullptr;             // private stream used for graph capture
    // pipelined state I/O: device staging copies of the whole state moved by
    // the copy engines on their own streams (uploads and downloads apart), so
    // host transfers overlap the steps on the context's stream
    // two staging slots each way, so that a copy never waits for the
    // conversion of the one before it: upload slot i % 2, download slot i % 2
    double* stage_up[2] = {nullptr, nullptr};
    double* stage_down[2] = {nullptr, nullptr};
    cudaStream_t up_stream = nullptr, down_stream = nullptr;
    cudaEvent_t ev_up_done[2] = {nullptr, nullptr}, ev_up_free[2] = {nullptr, nullptr};
    cudaEvent_t ev_down_ready[2] = {nullptr, nullptr}, ev_down_done[2] = {nullptr, nullptr};
    int up_next = 0, up_slot = 0, down_next = 0;   // next upload slot, the pending upload's slot, next download slot
    bool up_pending = false;
    size_t smem = 0;
    int stage_grid = 0, prim_grid = 0, n_items_cur = 0;
    float tune_ms[NTILES] = {0.f, 0.f, 0.f, 0.f};
    int tile = 0;                           // stage-kernel tile (TILES2 / TILES3 index)
    // fused stage kernel (2D plain mode): one pass per stage, no primitive pass
    bool fused_ok = false;                  // the context's scheme has a fused kernel
    bool fused = false;                     // the fused kernel is in use
    int mvar = 0, chunk = 0, march_grid = 0, n_items_march = 0;
    int4* d_items_march = nullptr;
    // TMA halo-tile loads of the tiled kernel: one descriptor per case for the current tile
    unsigned char* d_tmaps = nullptr;
    bool tma = false;
    // z-marching 3D stage kernel (FP32-mixed, stiffened/ideal gas, TMA planes)
    bool zm_ok = false, zm = false;
    int zvar = 0, zchunk = 0, zm_grid = 0, n_items_z = 0;
    size_t zm_smem = 0;
    int4* d_items_z = nullptr;
    unsigned char* d_tmaps_z = nullptr;
    float zm_ms = 0.f;
    float march_ms = 0.f, prim_ms = 0.f;
    size_t smem_max = 0;                    // opt-in shared memory per block of the device
    bool tuned = false;
    int nsm = 0;
    // captured steps per (cfl, cold): a cold step starts with the CFL pass, a
    // warm one takes the wave speeds the previous step's last fused stage left
    std::vector<std::pair<std::pair<double, bool>, cudaGraphExec_t>> graphs;
    // smax holds the wave speeds of the current q^n (a fused last stage wrote
    // them and no state write came after)
    bool smax_fresh = false;
    bool cfl_fuse = true;                   // FV_FUSED_CFL=0 in the environment: always the CFL pass
    long long launches = 0;
    std::string msg;
    bool profiling = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof;   // (kind, (start, stop))
    bool split = false;                     // the cases are slabs of one grid
    SplitInfo sp;
};

static fv_status exchange(fv_ctx* x, double* reg, cudaStream_t s);

static fv_status fail(fv_ctx* c, fv_status s, const char* fmt, const char* arg = "")
{
    if (c) {
        char buf[512];
        snprintf(buf, sizeof buf, fmt, arg);
        c->msg = buf;
    }
    return s;
}

static fv_status cuda_fail(fv_ctx* c, cudaError_t e, const char* where)
{
    if (c) c->msg = std::string(where) + ": " + cudaGetErrorString(e);
    return FV_ERR_CUDA;
}

#define CK(ctx, call)                                             \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
    } while (0)

// ------------------------------------------------------------------ checks
// Argument checks shared by fv_init and fv_rk_stage_noalloc: nullptr when
// the arguments are valid, else a static description (nothing allocated).
static const char* check_args(int ncases, const fv_grid* g, const fv_components* cm, const fv_eos* eos)
{
    if (ncases < 1 || !g || !cm || !eos) return "null argument or ncases < 1";
    const int nd = g[0].ndim;
    if (nd != 2 && nd != 3) return "ndim must be 2 or 3";
    for (int c = 0; c < ncases; ++c) {
        if (g[c].ndim != nd) return "all cases must share ndim";
        for (int d = 0; d < 3; ++d) {
            const int want1 = d >= nd;
            if (g[c].n[d] < 1 || (want1 && g[c].n[d] != 1)) return "bad cell counts";
            if (d < nd && !(g[c].hi[d] > g[c].lo[d])) return "hi must exceed lo";
            if (d < nd) {
                for (int s = 0; s < 2; ++s)
                    if (g[c].bc[d][s] < 0 || g[c].bc[d][s] > 3) return "bad boundary kind";
                if ((g[c].bc[d][0] == FV_BC_PERIODIC) != (g[c].bc[d][1] == FV_BC_PERIODIC))
                    return "periodic boundaries must pair";
                if ((d > 0 && g[c].bc[d][0] == FV_BC_INFLOW) || g[c].bc[d][1] == FV_BC_INFLOW)
                    return "inflow only on the x-low side";
            }
        }
        // each extent and the cell count within 2^31 (checked without overflow),
        // so that every ghosted extent n + 4 and every cell index fits the
        // kernels' int and 64-bit arithmetic
        const long long lim = 1LL << 31;
        if (g[c].n[0] > lim - 8 || g[c].n[1] > lim - 8 || g[c].n[2] > lim - 8) return "case too large";
        const long long n01 = (long long)g[c].n[0] * g[c].n[1];
        if (n01 > lim || n01 * g[c].n[2] > lim) return "case too large";
    }
    if (cm->ncomp < 2 || cm->ncomp > 3) return "ncomp must be 2 or 3";
    if (cm->liquid < 0 || cm->liquid >= cm->ncomp) return "bad liquid index";
    int npr = 0, nbaro = 0;
    for (int k = 0; k < cm->ncomp; ++k) {
        npr += cm->comp[k].kind == FV_PR;
        nbaro += cm->comp[k].kind == FV_BARO;
    }
    if (nbaro > 0) {
        // barotropic closure (Sec. 2.2): the liquid-vapour component at
        // `liquid`, isothermal ideal gases elsewhere
        if (nbaro != cm->ncomp) return "barotropic components cannot mix with other closures";
        for (int k = 0; k < cm->ncomp; ++k) {
            const fv_component& c = cm->comp[k];
            if (k == cm->liquid) {
                if (!(c.psat > 0.0) || !(c.rho_sl > 0.0) || !(c.rho_sv > 0.0) || !(c.rho_sv < c.rho_sl) ||
                    !(c.cl > 0.0) || !std::isfinite(c.psat * c.rho_sl * c.cl))
                    return "bad barotropic liquid constants";
            } else if (!(c.rt > 0.0) || !std::isfinite(c.rt)) return "bad barotropic gas constant R T_ref";
            if (c.mu != 0.0 || c.kc != 0.0) return "viscous terms need stiffened-gas / ideal-gas components";
        }
        if (eos->sigma > 0.0) return "CSF needs stiffened-gas / ideal-gas components";
        for (int c = 0; c < ncases; ++c)
            if (g[c].bc[0][0] == FV_BC_INFLOW) return "the inflow disc needs stiffened-gas / ideal-gas components";
        if (!std::isfinite(eos->thr_vap)) return "bad vapour sensor threshold";
    } else if (npr == cm->ncomp) {
        // Peng-Robinson mixture (Eq. A.2.1)
        for (int k = 0; k < cm->ncomp; ++k) {
            const fv_component& c = cm->comp[k];
            if (!(c.Tc > 0.0) || !(c.pc > 0.0) || !(c.M > 0.0) || !(c.cv > 0.0)) return "bad Peng-Robinson constants";
        }
        if (eos->sigma > 0.0 || eos->iles) return "CSF and the App. D switch need stiffened-gas / ideal-gas components";
    } else if (npr > 0) return "components must be all stiffened-gas / ideal-gas or all Peng-Robinson";
    double pis[FV_MAX_COMP];
    int npi = 0;
    for (int k = 0; k < cm->ncomp && npr == 0 && nbaro == 0; ++k) {
        const fv_component& c = cm->comp[k];
        if (c.kind != FV_SG) return "only stiffened-gas / ideal-gas components are supported";
        if (!(c.gamma > 1.0) || !(c.cv > 0.0) || !(c.pinf >= 0.0)) return "bad component constants";
        bool seen = false;
        for (int j = 0; j < npi; ++j) seen = seen || pis[j] == c.pinf;
        if (!seen) pis[npi++] = c.pinf;
    }
    if (npi > 2) return "at most two distinct pinf values";
    if (eos->lim_vel < 0 || eos->lim_vel > 6 || eos->lim_scalar < 0 || eos->lim_scalar > 6) return "bad limiter id";
    if (eos->precision != FV_FP64 && eos->precision != FV_MIXED) return "bad precision";
    if (eos->thinc && !(eos->beta > 0.0)) return "THINC beta must be positive";
    if (!(eos->sigma >= 0.0)) return "sigma must be >= 0";
    if (eos->curvature != 0 && eos->curvature != 1) return "curvature must be 0 or 1";
    if (eos->st_model != 0 && eos->st_model != 1) return "st_model must be 0 or 1";
    bool visc = false;
    for (int k = 0; k < cm->ncomp; ++k) {
        const fv_component& c = cm->comp[k];
        if (!(c.mu >= 0.0) || !(c.kc >= 0.0) || !std::isfinite(c.mu) || !std::isfinite(c.kc))
            return "viscosity and conductivity must be finite and >= 0";
        visc = visc || c.mu > 0.0 || c.kc > 0.0;
    }
    if (visc && npr > 0) return "viscous terms need stiffened-gas / ideal-gas components";
    if (visc && eos->st_model == 1 && eos->sigma > 0.0)
        return "the capillary jump model is not combined with viscous terms";
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(eos->gravity[d])) return "gravity must be finite";
    if (!std::isfinite(eos->sigma)) return "sigma must be finite";
    return nullptr;
}

static fv_status validate(int ncases, const fv_grid* g, const fv_components* cm, const fv_eos* eos,
                          std::string& why)
{
    const char* w = check_args(ncases, g, cm, eos);
    if (!w) return FV_OK;
    why = w;
    return FV_ERR_ARG;
}

static bool has_visc(const fv_components* cm)
{
    for (int k = 0; k < cm->ncomp; ++k)
        if (cm->comp[k].mu > 0.0 || cm->comp[k].kc > 0.0) return true;
    return false;
}

static bool is_baro(const fv_components* cm)
{
    return cm->ncomp > 0 && cm->comp[0].kind == FV_BARO;
}

static bool has_grav(const fv_eos* eos)
{
    return eos->gravity[0] != 0.0 || eos->gravity[1] != 0.0 || eos->gravity[2] != 0.0;
}

static void build_params(fv_ctx* x, const fv_components* cm, const fv_eos* eos)
{
    DevParams& P = x->P;
    memset(&P, 0, sizeof P);
    P.ndim = x->nd;
    P.ncomp = cm->ncomp;
    P.nv = x->nv;
    P.liquid = cm->liquid;
    P.iles = eos->iles ? 1 : 0;
    P.thinc = eos->thinc ? 1 : 0;
    P.lim_vel = eos->lim_vel;
    P.lim_scalar = eos->lim_scalar;
    P.capj = (eos->sigma > 0.0 && eos->st_model == 1) ? 1 : 0;
    P.csf = (eos->sigma > 0.0 && !P.capj) ? 1 : 0;
    P.hf = eos->curvature == 1 ? 1 : 0;
    P.visc = has_visc(cm) ? 1 : 0;
    P.grav = has_grav(eos) ? 1 : 0;
    P.baro = is_baro(cm) ? 1 : 0;
    P.aux_rc = (P.iles || P.grav || P.baro) ? 1 : 0;
    P.aux_al = (P.csf || P.iles || P.capj) ? 1 : 0;
    int np = x->nv;
    P.i_rho = P.i_c = P.i_al = P.i_mu = P.i_kc = P.i_av = P.i_kap = -1;
    if (P.aux_rc) { P.i_rho = np++; P.i_c = np++; }
    if (P.aux_al) P.i_al = np++;
    if (P.visc) { P.i_mu = np++; P.i_kc = np++; }
    if (P.baro) P.i_av = np++;
    if (P.capj) P.i_kap = np++;
    P.nprim = np;
    x->nprim = np;
    P.beta = eos->beta;
    P.thinc_eps = eos->thinc_eps;
    P.thinc_gamma = eos->thinc_gamma;
    P.tb = std::tanh(eos->beta);
    P.icb = 1.0 / std::cosh(eos->beta);
    P.itb = eos->beta > 0 ? 1.0 / std::tanh(eos->beta) : 0.0;
    P.thr_ducros = eos->thr_ducros;
    P.thr_gas = eos->thr_gas;
    P.eps_ducros = eos->eps_ducros;
    P.d3p_coef = eos->d3p_coef;
    P.sigma = eos->sigma;
    P.grad_eps = eos->grad_eps;
    P.p_ref = x->mixed ? eos->p_ref : 0.0;
    double piA = 0.0, piB = 1e300;
    for (int k = 0; k < cm->ncomp; ++k) {
        piA = std::max(piA, cm->comp[k].pinf);
        piB = std::min(piB, cm->comp[k].pinf);
    }
    P.single_class = piA == piB;
    for (int k = 0; k < cm->ncomp; ++k) {
        const fv_component& c = cm->comp[k];
        CompDev& d = P.c[k];
        d.gamma = c.gamma;
        d.pinf = c.pinf;
        d.cv = c.cv;
        d.q = c.q;
        d.gm1cv = (c.gamma - 1.0) * c.cv;
        d.gcv = c.gamma * c.cv;
        d.igamma = 1.0 / c.gamma;
        d.classA = (c.pinf == piA && !P.single_class) ? 1 : 0;
        d.pother = P.single_class ? 0.0 : (d.classA ? piB : piA);
        P.Pk[k] = P.p_ref + c.pinf;
    }
    // Peng-Robinson constants (Eq. A.2.1).  The components' critical volume
    // and compressibility are not given: Zc = 0.3074 (the PR value) and
    // vc = Zc R Tc / pc, so pc_aa = pc.
    int npr = 0;
    for (int k = 0; k < cm->ncomp; ++k) npr += cm->comp[k].kind == FV_PR;
    P.pr = npr == cm->ncomp;
    if (P.pr) {
        const double RU = 8.314462618, ZC = 0.3074;
        for (int i = 0; i < cm->ncomp; ++i) {
            const fv_component& ci = cm->comp[i];
            P.prc.b[i] = 0.077796 * RU * ci.Tc / ci.pc;
            P.prc.iM[i] = 1.0 / ci.M;
            P.prc.cv[i] = ci.cv;
            for (int j = 0; j < cm->ncomp; ++j) {
                const fv_component& cj = cm->comp[j];
                const double Tc = std::sqrt(ci.Tc * cj.Tc);
                const double vci = ZC * RU * ci.Tc / ci.pc, vcj = ZC * RU * cj.Tc / cj.pc;
                const double vc = std::pow(std::cbrt(vci) + std::cbrt(vcj), 3.0) / 8.0;
                const double pc = 0.5 * (ZC + ZC) * RU * Tc / vc;
                const double w = 0.5 * (ci.omega + cj.omega);
                P.prc.A[i][j] = 0.457236 * (RU * Tc) * (RU * Tc) / pc;
                P.prc.cc[i][j] = 0.37464 + 1.5422 * w - 0.26992 * w * w;
                P.prc.isqTc[i][j] = 1.0 / std::sqrt(Tc);
            }
        }
        for (int i = 0; i < MAXC; ++i) {
            P.prcf.b[i] = float(P.prc.b[i]);
            P.prcf.iM[i] = float(P.prc.iM[i]);
            P.prcf.cv[i] = float(P.prc.cv[i]);
            for (int j = 0; j < MAXC; ++j) {
                P.prcf.A[i][j] = float(P.prc.A[i][j]);
                P.prcf.cc[i][j] = float(P.prc.cc[i][j]);
                P.prcf.isqTc[i][j] = float(P.prc.isqTc[i][j]);
            }
        }
        P.single_class = 1;
    }
    // working-precision copies of the constants
    auto fill = [&](auto& Kt) {
        using T = std::remove_reference_t<decltype(Kt.p_ref)>;
        for (int k = 0; k < MAXC; ++k) {
            const CompDev& d = P.c[k];
            Kt.Pk[k] = T(P.Pk[k]);
            Kt.gm1cv[k] = T(d.gm1cv);
            Kt.igamma[k] = T(d.igamma);
            Kt.gcv[k] = T(d.gcv);
            Kt.cv[k] = T(d.cv);
            Kt.q[k] = T(d.q);
            Kt.pinf[k] = T(d.pinf);
            Kt.pother[k] = T(d.pother);
            // gamma - 1 and gamma pinf split into a float-float pair
            const double gm1 = d.gamma - 1.0, gpi = d.gamma * d.pinf + P.p_ref;
            Kt.Po[k] = T(d.pother + P.p_ref);
            Kt.gm1_hi[k] = T(gm1);
            Kt.gm1_lo[k] = T(gm1 - double(T(gm1)));
            Kt.gpi_hi[k] = T(gpi);
            Kt.gpi_lo[k] = T(gpi - double(T(gpi)));
        }
        Kt.p_ref = T(P.p_ref);
        Kt.beta = T(P.beta);
        Kt.thinc_eps = T(P.thinc_eps);
        Kt.thinc_gamma = T(P.thinc_gamma);
        Kt.tb = T(P.tb);
        Kt.icb = T(P.icb);
        Kt.itb = T(P.itb);
        Kt.thr_ducros = T(P.thr_ducros);
        Kt.thr_gas = T(P.thr_gas);
        Kt.eps_ducros = T(P.eps_ducros);
        Kt.d3p_coef = T(P.d3p_coef);
        Kt.sigma = T(P.sigma);
        Kt.grad_eps = T(P.grad_eps);
        double cvmin = cm->comp[0].cv;
        for (int k = 0; k < MAXC; ++k) {
            const bool on = k < cm->ncomp;
            Kt.mu[k] = T(on ? cm->comp[k].mu : 0.0);
            Kt.kc[k] = T(on ? cm->comp[k].kc : 0.0);
            if (on) cvmin = std::min(cvmin, cm->comp[k].cv);
        }
        Kt.icvmin = T(1.0 / cvmin);
        for (int d = 0; d < 3; ++d) Kt.grav[d] = T(eos->gravity[d]);
        if (P.baro) {
            const fv_component& lq = cm->comp[cm->liquid];
            for (int k = 0; k < MAXC; ++k) Kt.brt[k] = T(k < cm->ncomp && k != cm->liquid ? cm->comp[k].rt : 0.0);
            Kt.b_rsl = T(lq.rho_sl);
            Kt.b_rsv = T(lq.rho_sv);
            Kt.b_pso = T(lq.psat - P.p_ref);
            Kt.b_icl2 = T(1.0 / (lq.cl * lq.cl));
            Kt.b_icm2 = T(lq.rho_sl / lq.psat);   // 1/c_M^2, c_M^2 = p_sat / rho_sat,liq
            Kt.b_hcl2 = T(0.5 * lq.cl * lq.cl);
            Kt.b_irsl = T(1.0 / lq.rho_sl);
        }
        Kt.thr_vap = T(eos->thr_vap);
    };
    fill(P.kd);
    fill(P.kf);
}

static void plan(int ncases, const fv_grid* g, int nd, int nv, int nprim, int mixed, Layout& L,
                 std::vector<CaseDesc>* cases, std::vector<int4>* items_stage, std::vector<int4>* items_prim,
                 const SplitInfo* sp = nullptr)
{
    L = Layout{};
    long long qoff = 0, poff = 0, nin = sp ? 3 * sp->in_stride : 0;
    const int ts[3] = {tile_x(nd), tile_y(nd), tile_z(nd)};
    for (int c = 0; c < ncases; ++c) {
        CaseDesc C{};
        int gx[3];
        for (int d = 0; d < 3; ++d) {
            C.n[d] = g[c].n[d];
            C.g[d] = d < nd ? g[c].n[d] + 4 : 1;
            gx[d] = C.g[d];
            C.dx[d] = d < nd ? (sp ? sp->dx[d] : (g[c].hi[d] - g[c].lo[d]) / g[c].n[d]) : 1.0;
            C.idx[d] = 1.0 / C.dx[d];
            C.fdx[d] = float(C.dx[d]);
            C.fidx[d] = float(C.idx[d]);
            C.bc[d][0] = d < nd ? g[c].bc[d][0] : 0;
            C.bc[d][1] = d < nd ? g[c].bc[d][1] : 0;
        }
        C.gp = (C.g[0] + 3) & ~3;
        // a slab keeps two ghost planes of its split dimension on each side
        // next to its cells in the conserved registers
        const long long plane = sp ? (sp->last == 1 ? (long long)C.n[0] : (long long)C.n[0] * C.n[1]) : 0;
        qoff += 2 * plane;
        C.qoff = qoff;
        C.poff = poff;
        if (sp) C.org[sp->last] = sp->row0[c];
        C.inflow = g[c].bc[0][0] == FV_BC_INFLOW;
        // disc centre relative to the low corner (a slab keeps the whole grid's
        // corner and adds its origin to its cell indices)
        C.in_yc = g[c].in_yc - g[c].lo[1];
        C.in_zc = g[c].in_zc - g[c].lo[2];
        C.in_r2 = g[c].in_radius * g[c].in_radius;
        C.in_T = g[c].in_T;
        for (int d = 0; d < 3; ++d) C.in_u0[d] = g[c].in_u0[d];
        for (int k = 0; k < FV_MAX_COMP && k < MAXC; ++k) C.in_Y[k] = g[c].in_Y[k];
        C.in_uoff = -1;
        C.in_ustride = (long long)C.n[1] * C.n[2];
        if (sp && sp->in_stride && C.inflow) {
            // slabs index the grid's one inflow array from their origin
            // (the split dimension is the last one, so a slab's ny is the grid's)
            C.in_uoff = (long long)C.org[2] * C.n[1] + C.org[1];
            C.in_ustride = sp->in_stride;
        } else if (C.inflow && g[c].in_u) {
            C.in_uoff = nin;
            nin += 3LL * C.n[1] * C.n[2];
        }
        const long long ncell = (long long)C.n[0] * C.n[1] * C.n[2];
        qoff += ncell + 2 * plane;
        poff += (long long)C.gp * C.g[1] * C.g[2];
        L.max_cells = std::max(L.max_cells, ncell);
        if (cases) cases->push_back(C);
        long long nst = 0, npr = ntiles(gx, nd);
        for (int t = 0; t < NTILES; ++t) {
            const TileDef td = tile_def(nd, t);
            nst = std::max(nst, (long long)((C.n[0] + td.x - 1) / td.x) * ((C.n[1] + td.y - 1) / td.y) *
                                    ((C.n[2] + td.z - 1) / td.z));
        }
        L.n_items_stage += (int)nst;
        L.n_items_prim += (int)npr;
        if (nd == 2)
            L.n_items_march += ((C.n[0] + MARCH_COLS - 1) / MARCH_COLS) * ((C.n[1] + MARCH_CHUNK_MIN - 1) / MARCH_CHUNK_MIN);
        if (nd == 3)
            L.n_items_z += ((C.n[0] + ZM_TX - 1) / ZM_TX) * ((C.n[1] + ZM_TY - 1) / ZM_TY) *
                           ((C.n[2] + ZM_CHUNKS[0] - 1) / ZM_CHUNKS[0]);
        if (items_stage)
            for (int z = 0; z < C.n[2]; z += ts[2])
                for (int y = 0; y < C.n[1]; y += ts[1])
                    for (int x = 0; x < C.n[0]; x += ts[0]) items_stage->push_back(make_int4(c, x, y, z));
        if (items_prim)
            for (int z = 0; z < gx[2]; z += ts[2])
                for (int y = 0; y < gx[1]; y += ts[1])
                    for (int x = 0; x < gx[0]; x += ts[0]) items_prim->push_back(make_int4(c, x, y, z));
    }
    L.ntot_q = qoff;
    L.ntot_p = poff;
    L.n_in_u = nin;
    const size_t rsz = mixed ? sizeof(float) : sizeof(double);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o += align256(bytes); return at; };
    L.cases = take(sizeof(CaseDesc) * ncases);
    L.items_stage = take(sizeof(int4) * L.n_items_stage);
    L.items_prim = take(sizeof(int4) * L.n_items_prim);
    L.items_march = take(sizeof(int4) * std::max(1, L.n_items_march));
    L.q0 = take(sizeof(double) * nv * qoff);
    L.qa = take(sizeof(double) * nv * qoff);
    L.qb = take(sizeof(double) * nv * qoff);
    L.prim = take(rsz * nprim * poff);
    L.io = take(sizeof(double) * nv * L.max_cells);
    L.smax = take(sizeof(unsigned long long) * ncases);
    L.dt = take(sizeof(double) * ncases);
    L.t = take(sizeof(double) * ncases);
    L.err = take(sizeof(int));
    L.in_u = take(sizeof(double) * std::max(1LL, nin));
    L.partial = take(sizeof(double) * nv * 1024);
    L.tmaps = take(TMAP_BYTES * (size_t)ncases);
    L.items_z = take(sizeof(int4) * std::max(1, L.n_items_z));
    L.tmaps_z = take(TMAP_BYTES * (size_t)ncases);
    L.total = o;
}

static int count_nprim(const fv_components* cm, const fv_eos* eos, int nv)
{
    int np = nv;
    if (eos->iles || has_grav(eos) || is_baro(cm)) np += 2;
    if (eos->iles || eos->sigma > 0.0) np += 1;
    if (has_visc(cm)) np += 2;
    if (is_baro(cm)) np += 1;
    if (eos->sigma > 0.0 && eos->st_model == 1) np += 1;   // cell curvature of the jump model
    return np;
}

extern "C" fv_status fv_workspace_size(int ncases, const fv_grid* grids, const fv_components* comps,
                                       const fv_eos* eos, size_t* bytes)
{
    std::string why;
    fv_status s = validate(ncases, grids, comps, eos, why);
    if (s) return s;
    const int nd = grids[0].ndim, nv = nd + comps->ncomp + 1;
    Layout L;
    plan(ncases, grids, nd, nv, count_nprim(comps, eos, nv), eos->precision == FV_MIXED, L, nullptr, nullptr, nullptr);
    if (bytes) *bytes = L.total;
    return FV_OK;
}


// ------------------------------------------------------------------ TMA
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

static const void* stage_tmaps(const fv_ctx* x) { return x->tma ? x->d_tmaps : nullptr; }

// One 4D descriptor [x, y, z, field] of each case's primitive arrays with the
// halo box of `variant`'s tile; zero fill outside the ghosted box.  Every TMA
// alignment rule is checked here; if one fails (or FV_TMA=0 in the
// environment, or no encoder) the tiled kernel keeps its cp.async loads.
// Descriptors [x, y, z, field] of every case's primitive arrays with box
// `box` (zero fill outside the ghosted box) into `dst`.  Every TMA alignment
// rule is checked here (x0 = tile origins in x, multiples of `xalign` cells);
// false if one fails, if FV_TMA=0 is set or if there is no encoder.
static bool encode_maps(fv_ctx* x, const cuuint32_t* box, int xalign, unsigned char* dst)
{
    if (const char* f = getenv("FV_TMA"))
        if (atoi(f) == 0) return false;
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t es = x->mixed ? sizeof(float) : sizeof(double);
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    if ((xalign * es) % 16 || (box[0] * es) % 16 || box[0] > 256 || box[1] > 256 || box[2] > 256 || box[3] > 256)
        return false;
    std::vector<CUtensorMap> maps(x->ncases);
    for (int c = 0; c < x->ncases; ++c) {
        const CaseDesc& C = x->cases[c];
        unsigned char* base = static_cast<unsigned char*>(x->prim) + C.poff * es;
        const cuuint64_t dims[4] = {cuuint64_t(C.g[0]), cuuint64_t(C.g[1]), cuuint64_t(C.g[2]), cuuint64_t(x->nprim)};
        const cuuint64_t strides[3] = {C.gp * es, C.gp * es * C.g[1], cuuint64_t(x->L.ntot_p) * es};
        if (reinterpret_cast<uintptr_t>(base) % 16 || strides[0] % 16 || strides[1] % 16 || strides[2] % 16)
            return false;
        if (fn(&maps[c], es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, base, dims,
               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    static_assert(sizeof(CUtensorMap) == TMAP_BYTES, "descriptor size");
    return cudaMemcpy(dst, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice) == cudaSuccess;
}

// the tiled kernel's descriptors for `variant`'s halo box; without them it
// keeps its cp.async loads
static fv_status encode_tmaps(fv_ctx* x, int variant)
{
    const TileDef td = tile_def(x->nd, variant_tile(x->nd, variant));
    const cuuint32_t box[4] = {cuuint32_t(td.x + 4), cuuint32_t(td.y + 4), cuuint32_t(x->nd == 3 ? td.z + 4 : 1),
                               cuuint32_t(x->nprim)};
    x->tma = encode_maps(x, box, td.x, x->d_tmaps);
    return FV_OK;
}

// the z-marching kernel's viscous instantiations (Eq. 2-2 terms or gravity on)
static int zm_visc(const fv_ctx* x) { return (x->P.visc || x->P.grav) ? 1 : 0; }

// z-marching kernel with z-chunk `chunk` and variant `var` (needs TMA)
static fv_status apply_zmarch(fv_ctx* x, int chunk, int var)
{
    const bool t42 = x->P.lim_vel == FV_KOREN && x->P.lim_scalar == FV_MINMOD;
    if (!t42) var = 2;
    else if (zm_visc(x) || (!x->mixed && var != 4 && var != 5)) var = 1;
    const cuuint32_t box[4] = {cuuint32_t(ZM_TX + 4), cuuint32_t(ZM_TY + 4), 1, cuuint32_t(x->nprim)};
    if (!encode_maps(x, box, ZM_TX, x->d_tmaps_z)) return fail(x, FV_ERR_ARG, "z-marching kernel needs TMA%s");
    std::vector<int4> it;
    for (size_t c = 0; c < x->cases.size(); ++c) {
        const CaseDesc& C = x->cases[c];
        for (int z = 0; z < C.n[2]; z += chunk)
            for (int y = 0; y < C.n[1]; y += ZM_TY)
                for (int xx = 0; xx < C.n[0]; xx += ZM_TX) it.push_back(make_int4((int)c, xx, y, z));
    }
    if ((int)it.size() > x->L.n_items_z) return fail(x, FV_ERR_STATE, "z-march work list overflow%s");
    CK(x, cudaMemcpy(x->d_items_z, it.data(), sizeof(int4) * it.size(), cudaMemcpyHostToDevice));
    const size_t smem = zmarch_smem(x->nc, x->nprim, !x->mixed);
    if (smem > x->smem_max) return fail(x, FV_ERR_ARG, "z-marching kernel does not fit in shared memory%s");
    CK(x, zmarch_set_smem(x->nc, var, zm_visc(x), !x->mixed, smem));
    const int occ = zmarch_occupancy(x->nc, var, zm_visc(x), !x->mixed, smem);
    if (occ < 1) return fail(x, FV_ERR_CUDA, "z-marching kernel cannot be resident%s");
    x->zm = true;
    x->fused = false;
    x->zvar = var;
    x->zchunk = chunk;
    x->zm_smem = smem;
    x->n_items_z = (int)it.size();
    x->zm_grid = (int)std::min<long long>((long long)it.size(), (long long)x->nsm * occ);
    return FV_OK;
}

// work list of the stage kernel for one candidate tile
static void stage_items(const std::vector<CaseDesc>& cases, int nd, int tile, std::vector<int4>& out)
{
    const TileDef td = tile_def(nd, variant_tile(nd, tile));
    out.clear();
    for (size_t c = 0; c < cases.size(); ++c) {
        const CaseDesc& C = cases[c];
        for (int z = 0; z < C.n[2]; z += td.z)
            for (int y = 0; y < C.n[1]; y += td.y)
                for (int x = 0; x < C.n[0]; x += td.x) out.push_back(make_int4((int)c, x, y, z));
    }
}

// Stage-kernel variant for candidate tile `tile`: the autotuned tiles serve the
// stiffened/ideal-gas closure with the Table 4.2 limiter pair; Peng-Robinson
// and any other limiter pair run on tile 0.
static int kernel_variant(const DevParams& P, int tile)
{
    if (P.baro) return NTILES + 4;
    if (P.visc || P.grav) return NTILES + 3;
    if (P.capj) return NTILES + 1;   // the variant that carries the capillary jump model
    const bool t42 = P.lim_vel == FV_KOREN && P.lim_scalar == FV_MINMOD;
    if (t42 && !P.pr) return tile < NTILES ? tile : 0;
    if (t42) return NTILES;
    return P.pr ? NTILES + 2 : NTILES + 1;
}

static bool tunable(const DevParams& P) { return kernel_variant(P, 1) == 1; }

static fv_status apply_tile(fv_ctx* x, int tile)
{
    tile = kernel_variant(x->P, tile);
    std::vector<int4> it;
    stage_items(x->cases, x->nd, tile, it);
    if ((long long)it.size() > x->L.n_items_stage) return fail(x, FV_ERR_STATE, "work list overflow%s");
    CK(x, cudaMemcpy(x->d_items_stage, it.data(), sizeof(int4) * it.size(), cudaMemcpyHostToDevice));
    const size_t smem = stage_smem(x->nd, x->nc, x->mixed, tile, x->nprim, x->ff);
    if (smem > x->smem_max) return fail(x, FV_ERR_ARG, "stage kernel tile does not fit in shared memory%s");
    CK(x, stage_set_smem(x->nd, x->nc, x->mixed, tile, smem, x->ff));
    const int occ = stage_occupancy(x->nd, x->nc, x->mixed, tile, smem, x->ff);
    if (occ < 1) return fail(x, FV_ERR_CUDA, "stage kernel tile cannot be resident%s");
    x->tile = tile;
    x->fused = false;
    x->zm = false;
    x->smem = smem;
    {
        const fv_status st = encode_tmaps(x, tile);
        if (st) return st;
    }
    x->n_items_cur = (int)it.size();
    x->stage_grid = (int)std::min<long long>((long long)it.size(), (long long)x->nsm * occ);
    return FV_OK;
}

// scheme features of the fused kernel (App. D switch, CSF)
static int march_mode(const fv_ctx* x)
{
    return (x->P.iles ? MARCH_ILES : 0) | (x->P.csf ? MARCH_CSF : 0) | ((x->P.visc || x->P.grav) ? MARCH_VISC : 0) |
           (x->P.baro ? MARCH_BARO : 0);
}

// Fused kernel with row chunk `chunk` and variant `var`: work list of
// (case, strip column, first row, rows) items.
static fv_status apply_march(fv_ctx* x, int chunk, int var)
{
    const bool t42 = x->P.lim_vel == FV_KOREN && x->P.lim_scalar == FV_MINMOD;
    if (!t42) var = 2;
    std::vector<int4> it;
    for (size_t c = 0; c < x->cases.size(); ++c) {
        const CaseDesc& C = x->cases[c];
        for (int x0 = 0; x0 < C.n[0]; x0 += MARCH_COLS)
            for (int y0 = 0; y0 < C.n[1]; y0 += chunk) it.push_back(make_int4((int)c, x0, y0, chunk));
    }
    if ((int)it.size() > x->L.n_items_march) return fail(x, FV_ERR_STATE, "fused work list overflow%s");
    CK(x, cudaMemcpy(x->d_items_march, it.data(), sizeof(int4) * it.size(), cudaMemcpyHostToDevice));
    const int occ = march_occupancy(x->nc, x->mixed, march_mode(x), var);
    if (occ < 1) return fail(x, FV_ERR_CUDA, "fused stage kernel cannot be resident%s");
    x->fused = true;
    x->zm = false;
    x->mvar = var;
    x->chunk = chunk;
    x->n_items_march = (int)it.size();
    const long long warps = (long long)x->nsm * occ * MARCH_WARPS;
    x->march_grid = (int)((std::min<long long>(warps, it.size()) + MARCH_WARPS - 1) / MARCH_WARPS);
    return FV_OK;
}

// Tile autotuner: time every candidate tile of the stage kernel on this
// context's cases (current state, one primitive pass, 1 warm-up and 3 timed
// launches each, writing only the scratch register q^B) and keep the
// fastest.  Results are cached per workload class for the process; the
// environment variable FV_TILE=<index> forces a tile.
namespace {
std::mutex g_tune_mu;
std::map<std::string, int> g_tune_cache;
}

static std::string tune_key(const fv_ctx* x)
{
    long long cells = x->L.ntot_q;
    int lg = 0;
    while ((1LL << (lg + 1)) <= cells) ++lg;
    char buf[160];
    // every scheme switch that selects a different kernel instantiation
    snprintf(buf, sizeof buf, "%d/%d/%d/%d/%d/%d/%d%d/%d/%d/%d%d%d", x->nd, x->nc, x->mixed, x->P.iles, x->P.csf,
             x->P.pr, x->P.lim_vel, x->P.lim_scalar, x->ncases > 64 ? 2 : (x->ncases > 1 ? 1 : 0), lg,
             (x->P.visc || x->P.grav) ? 1 : 0, x->P.baro, x->P.hf);
    return buf;
}

static bool fused_cfl(const fv_ctx* x);

static fv_status tune(fv_ctx* x)
{
    if (x->tuned) return FV_OK;
    x->tuned = true;
    int want_fused = -1;   // -1: the tuner decides; FV_FUSED=0/1 in the environment forces it
    if (const char* f = getenv("FV_FUSED")) want_fused = atoi(f) ? 1 : 0;
    if (!x->fused_ok) want_fused = 0;
    if (const char* f = getenv("FV_TILE")) {
        const int t = atoi(f);
        if (t >= 0 && t < NTILES) return apply_tile(x, t);
    }
    int want_zm = -1;      // FV_ZMARCH=0/1 excludes or forces the z-marching kernel
    if (const char* f = getenv("FV_ZMARCH")) want_zm = atoi(f) ? 1 : 0;
    if (!x->zm_ok) want_zm = 0;
    int want_zvar = -1;    // FV_ZVAR=<v> keeps only the z-marching kernel's variant v
    if (const char* f = getenv("FV_ZVAR")) want_zvar = atoi(f);
    const bool tiles = tunable(x->P);
    if (!tiles && want_fused == 0 && want_zm == 0) return apply_tile(x, 0);   // a single candidate
    const std::string key = tune_key(x) + "/" + std::to_string(want_fused) + "/" + std::to_string(want_zm) + "/" +
                            std::to_string(want_zvar);
    auto apply = [&](int code) {
        if (code >= 200) return apply_zmarch(x, ZM_CHUNKS[(code - 200) / 10], (code - 200) % 10);
        return code < 100 ? apply_tile(x, code) : apply_march(x, MARCH_CHUNKS[(code - 100) / 10], (code - 100) % 10);
    };
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) return apply(it->second);
    }
    {
        fv_status e = exchange(x, x->Q0, x->stream);   // the candidates read q^0's ghost planes
        if (e) return e;
    }
    int err0 = 0;
    CK(x, cudaStreamSynchronize(x->stream));
    CK(x, cudaMemcpy(&err0, x->err, sizeof(int), cudaMemcpyDeviceToHost));
    cudaEvent_t e0, e1;
    CK(x, cudaEventCreate(&e0));
    CK(x, cudaEventCreate(&e1));
    // one warm-up and three timed launches; the minimum of the timed ones
    auto timed = [&](auto&& launch, float& tmin) -> fv_status {
        tmin = 1e30f;
        for (int r = 0; r < 4; ++r) {
            CK(x, cudaEventRecord(e0, x->stream));
            CK(x, launch());
            CK(x, cudaEventRecord(e1, x->stream));
            CK(x, cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(x, cudaEventElapsedTime(&ms, e0, e1));
            if (r > 0) tmin = std::min(tmin, ms);
        }
        return FV_OK;
    };
    // the primitive pass: input of the tiled kernel, and part of its cost
    // when the fused kernel (which needs none) competes
    PrimArgs pa{x->P, x->d_cases, x->d_items_prim, x->L.n_items_prim, x->Q0, x->prim, x->in_u, nullptr, x->err};
    float prim_ms = 0.f;
    fv_status st = timed([&] { return launch_prim(x->nd, x->nc, x->mixed, pa, x->prim_grid, x->stream, x->ff); },
                         prim_ms);
    if (st) return st;
    int best = -1;
    float best_ms = 1e30f;
    if (want_fused != 1 && want_zm != 1) {
        for (int t = 0; t < (tiles ? NTILES : 1); ++t) {
            if (apply_tile(x, t)) { x->msg.clear(); continue; }
            StageArgs sa{x->P, x->d_cases, x->d_items_stage, x->n_items_cur, x->prim, stage_tmaps(x), x->Q0, x->QB,
                         x->dt, 0.0,
                         x->err};
            float ms = 0.f;
            st = timed([&] { return launch_stage(x->nd, x->nc, x->mixed, x->tile, sa, x->stage_grid, x->smem,
                                                 x->stream, x->ff); }, ms);
            if (st) return st;
            x->tune_ms[t] = ms;
            const float cost = ms + (want_fused != 0 ? prim_ms : 0.f);
            if (cost < best_ms) { best_ms = cost; best = t; }
        }
    }
    if (want_fused != 0) {
        const bool t42 = x->P.lim_vel == FV_KOREN && x->P.lim_scalar == FV_MINMOD;
        float fbest = 1e30f;
        for (int ci = 0; ci < 3; ++ci)
            for (int var = (t42 ? 0 : 2); var < (t42 ? 1 : 3); ++var) {
                if (apply_march(x, MARCH_CHUNKS[ci], var)) { x->msg.clear(); continue; }
                MarchArgs ma{x->P, x->d_cases, x->d_items_march, x->n_items_march, x->Q0, x->Q0, x->QB, x->in_u,
                             x->dt, 0.0, x->err};
                float ms = 0.f;
                st = timed([&] { return launch_march(x->nc, x->mixed, march_mode(x), x->mvar, ma, x->march_grid,
                                                     x->stream); }, ms);
                if (st) return st;
                if (fused_cfl(x)) {
                    // a warm step's last stage also recovers q^{n+1} for the CFL
                    // speeds (in place of the tiled path's stage-1 primitive
                    // pass): charge the stage average (smax is cleared by the
                    // first, cold, step)
                    MarchArgs mc = ma;
                    mc.smax = x->smax;
                    float ms4 = 0.f;
                    st = timed([&] { return launch_march(x->nc, x->mixed, march_mode(x) | MARCH_CFL, x->mvar, mc,
                                                         x->march_grid, x->stream); }, ms4);
                    if (st) return st;
                    ms = (3.f * ms + ms4) / 4.f;
                }
                fbest = std::min(fbest, ms);
                if (ms < best_ms) { best_ms = ms; best = 100 + 10 * ci + var; }
            }
        x->march_ms = fbest;
    }
    if (want_zm != 0) {
        // after the primitive pass above, like the tiled kernel
        const bool t42 = x->P.lim_vel == FV_KOREN && x->P.lim_scalar == FV_MINMOD;
        float zbest = 1e30f;
        // the viscous instantiations: variant 1 (Table 4.2 pair) or 2 (run-time
        // pair); the FP64 ones 1, 4 or 5 (Table 4.2 pair), 2 (run-time pair)
        const int zvars_t42[5] = {0, 1, 3, 4, 5}, zvars_rt[1] = {2}, zvars_visc[1] = {1}, zvars_fp64[3] = {1, 4, 5};
        const int* const zv = !t42 ? zvars_rt : (zm_visc(x) ? zvars_visc : (x->mixed ? zvars_t42 : zvars_fp64));
        const int nzv = !t42 || zm_visc(x) ? 1 : (x->mixed ? 5 : 3);
        for (int ci = 0; ci < 3; ++ci)
            for (int vi = 0; vi < nzv; ++vi) {
                const int var = zv[vi];
                if (want_zvar >= 0 && var != want_zvar) continue;
                if (apply_zmarch(x, ZM_CHUNKS[ci], var)) { x->msg.clear(); continue; }
                ZArgs za{x->P, x->d_cases, x->d_items_z, x->n_items_z, x->zchunk, x->d_tmaps_z, x->Q0, x->QB,
                         x->dt, 0.0, x->err};
                float ms = 0.f;
                st = timed([&] {
                    return launch_zmarch(x->nc, x->zvar, zm_visc(x), !x->mixed, za, x->zm_grid, x->zm_smem, x->stream);
                }, ms);
                if (st) return st;
                zbest = std::min(zbest, ms);
                if (ms < best_ms) { best_ms = ms; best = 200 + 10 * ci + var; }
            }
        x->zm_ms = zbest;
    }
    x->prim_ms = prim_ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(x, cudaMemcpy(x->err, &err0, sizeof(int), cudaMemcpyHostToDevice));
    if (best < 0) return fail(x, FV_ERR_CUDA, "no stage kernel candidate can run%s");
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_cache[key] = best;
    }
    return apply(best);
}

static fv_status init_common(int ncases, const fv_grid* grids, const fv_components* comps, const fv_eos* eos,
                             void* ws, size_t ws_bytes, fv_ctx** out, const SplitInfo* sp = nullptr,
                             const double* sp_in_u = nullptr)
{
    if (!out) return FV_ERR_ARG;
    *out = nullptr;
    std::string why;
    // slab grids carry the internal BC_HALO kind; the whole grid was validated
    fv_status s = sp ? FV_OK : validate(ncases, grids, comps, eos, why);
    fv_ctx* x = new (std::nothrow) fv_ctx();
    if (!x) return FV_ERR_ALLOC;
    if (s) {
        x->msg = why;
        *out = x;   // returned so the caller can read fv_last_error, then fv_destroy
        return s;
    }
    x->ncases = ncases;
    x->nd = grids[0].ndim;
    x->nc = comps->ncomp;
    x->nv = x->nd + x->nc + 1;
    x->mixed = eos->precision == FV_MIXED;
    x->ff = x->mixed;
    x->grids.assign(grids, grids + ncases);
    build_params(x, comps, eos);
    if (sp) {
        x->split = true;
        x->sp = *sp;
    }
    std::vector<int4> ist, ipr;
    plan(ncases, grids, x->nd, x->nv, x->nprim, x->mixed, x->L, &x->cases, &ist, &ipr, sp);
    *out = x;
    const Layout& L = x->L;
    x->P.ntot_q = L.ntot_q;
    x->P.ntot_p = L.ntot_p;
    if (ws) {
        if (ws_bytes < L.total || (reinterpret_cast<uintptr_t>(ws) & 255))
            return fail(x, FV_ERR_ARG, "workspace too small or not 256-byte aligned%s");
        x->base = static_cast<unsigned char*>(ws);
    } else {
        cudaError_t e = cudaMalloc(&x->base, L.total);
        if (e != cudaSuccess) {
            x->base = nullptr;
            cudaGetLastError();
            return fail(x, FV_ERR_ALLOC, "cudaMalloc of the context workspace failed%s");
        }
        x->owns = true;
    }
    unsigned char* b = x->base;
    x->d_cases = reinterpret_cast<CaseDesc*>(b + L.cases);
    x->d_items_stage = reinterpret_cast<int4*>(b + L.items_stage);
    x->d_items_prim = reinterpret_cast<int4*>(b + L.items_prim);
    x->d_items_march = reinterpret_cast<int4*>(b + L.items_march);
    x->Q0 = reinterpret_cast<double*>(b + L.q0);
    x->QA = reinterpret_cast<double*>(b + L.qa);
    x->QB = reinterpret_cast<double*>(b + L.qb);
    x->prim = b + L.prim;
    x->io = reinterpret_cast<double*>(b + L.io);
    x->smax = reinterpret_cast<unsigned long long*>(b + L.smax);
    x->dt = reinterpret_cast<double*>(b + L.dt);
    x->t = reinterpret_cast<double*>(b + L.t);
    x->err = reinterpret_cast<int*>(b + L.err);
    x->in_u = reinterpret_cast<double*>(b + L.in_u);
    x->partial = reinterpret_cast<double*>(b + L.partial);
    x->d_tmaps = b + L.tmaps;
    x->d_items_z = reinterpret_cast<int4*>(b + L.items_z);
    x->d_tmaps_z = b + L.tmaps_z;
    CK(x, cudaStreamCreateWithFlags(&x->cap, cudaStreamNonBlocking));
    CK(x, cudaMemcpy(x->d_cases, x->cases.data(), sizeof(CaseDesc) * ncases, cudaMemcpyHostToDevice));
    CK(x, cudaMemcpy(x->d_items_prim, ipr.data(), sizeof(int4) * ipr.size(), cudaMemcpyHostToDevice));
    CK(x, cudaMemset(x->smax, 0, sizeof(unsigned long long) * ncases));
    CK(x, cudaMemset(x->dt, 0, sizeof(double) * ncases));
    CK(x, cudaMemset(x->t, 0, sizeof(double) * ncases));
    CK(x, cudaMemset(x->err, 0, sizeof(int)));
    CK(x, cudaMemset(x->Q0, 0, sizeof(double) * x->nv * L.ntot_q));
    CK(x, cudaMemset(x->prim, 0, (x->mixed ? sizeof(float) : sizeof(double)) * (size_t)x->nprim * L.ntot_p));
    if (sp && sp->in_stride && sp_in_u)
        CK(x, cudaMemcpy(x->in_u, sp_in_u, sizeof(double) * 3 * sp->in_stride, cudaMemcpyHostToDevice));
    for (int c = 0; c < ncases && !sp; ++c)
        if (x->cases[c].in_uoff >= 0)
            CK(x, cudaMemcpy(x->in_u + x->cases[c].in_uoff, grids[c].in_u,
                             sizeof(double) * 3 * grids[c].n[1] * grids[c].n[2], cudaMemcpyHostToDevice));
    // launch shapes: persistent grids of (resident blocks per SM) x (SMs)
    int dev = 0, nsm = 0;
    CK(x, cudaGetDevice(&dev));
    CK(x, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    x->nsm = nsm;
    int smax = 0;
    CK(x, cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    x->smem_max = (size_t)smax;
    if (const char* f = getenv("FV_FUSED_CFL")) x->cfl_fuse = atoi(f) != 0;
    const int occ_p = prim_occupancy(x->nd, x->nc, x->mixed);
    x->prim_grid = std::min(L.n_items_prim, std::max(1, nsm * occ_p));
    {
        // the first candidate tile that fits is the default until the tuner runs
        fv_status s = FV_ERR_ARG;
        for (int t = 0; t < NTILES && s; ++t) s = apply_tile(x, t);
        if (s) return s;
    }
    // the barotropic closure in the fused kernel: FP32-mixed form, plain mode
    x->fused_ok = x->nd == 2 && !x->P.pr && !x->P.hf && !x->P.capj &&
                  (!x->P.baro || (x->mixed && !x->P.iles && !x->P.csf && !x->P.visc && !x->P.grav));
    // FP32-mixed form, or the FP64 form without viscous terms and gravity
    x->zm_ok = x->nd == 3 && (x->mixed ? x->ff != 0 : !(x->P.visc || x->P.grav)) && !x->P.pr && !x->P.baro &&
               !x->P.hf &&
               !x->P.capj;
    CK(x, cudaDeviceSynchronize());
    return FV_OK;
}

extern "C" fv_status fv_init(int ncases, const fv_grid* grids, const fv_components* comps, const fv_eos* eos,
                             fv_ctx** out)
{
    return init_common(ncases, grids, comps, eos, nullptr, 0, out);
}

extern "C" fv_status fv_init_ws(int ncases, const fv_grid* grids, const fv_components* comps, const fv_eos* eos,
                                void* dev_workspace, size_t bytes, fv_ctx** out)
{
    if (!dev_workspace) return FV_ERR_ARG;
    return init_common(ncases, grids, comps, eos, dev_workspace, bytes, out);
}

// Slabs of a grid split along its last dimension: block grids (n of the
// split dimension = the slab's rows, sides towards neighbours BC_HALO, the
// whole grid's corner and cell sizes) and the neighbour table.
static const char* split_plan(const fv_grid* grid, int nblocks, const int* rows, std::vector<fv_grid>& blocks,
                              SplitInfo& sp)
{
    const int nd = grid->ndim, ld = nd - 1;
    const int n = grid->n[ld];
    if (nblocks < 1 || nblocks > n / 2) return "nblocks must be 1 .. n/2 of the split dimension";
    std::vector<int> r(nblocks);
    long long sum = 0;
    for (int b = 0; b < nblocks; ++b) {
        r[b] = rows ? rows[b] : n / nblocks + (b < n % nblocks ? 1 : 0);
        if (r[b] < 2) return "every slab needs at least two rows of the split dimension";
        sum += r[b];
    }
    if (sum != n) return "slab rows must add up to the grid's extent";
    const bool periodic = grid->bc[ld][0] == FV_BC_PERIODIC;
    sp = SplitInfo{};
    sp.last = ld;
    for (int d = 0; d < 3; ++d) sp.dx[d] = d < nd ? (grid->hi[d] - grid->lo[d]) / grid->n[d] : 1.0;
    sp.in_stride = (grid->bc[0][0] == FV_BC_INFLOW && grid->in_u) ? (long long)grid->n[1] * grid->n[2] : 0;
    blocks.assign(nblocks, *grid);
    int r0 = 0;
    for (int b = 0; b < nblocks; ++b) {
        fv_grid& g = blocks[b];
        g.n[ld] = r[b];
        g.in_u = nullptr;
        sp.row0.push_back(r0);
        const int lo = b > 0 ? b - 1 : (periodic ? nblocks - 1 : -1);
        const int hi = b < nblocks - 1 ? b + 1 : (periodic ? 0 : -1);
        sp.nbr_lo.push_back(lo);
        sp.nbr_hi.push_back(hi);
        if (lo >= 0) g.bc[ld][0] = BC_HALO;
        if (hi >= 0) g.bc[ld][1] = BC_HALO;
        r0 += r[b];
    }
    return nullptr;
}

extern "C" fv_status fv_split_workspace_size(const fv_grid* grid, int nblocks, const int* rows,
                                             const fv_components* comps, const fv_eos* eos, size_t* bytes)
{
    std::string why;
    fv_status s = validate(1, grid, comps, eos, why);
    if (s) return s;
    std::vector<fv_grid> blocks;
    SplitInfo sp;
    if (split_plan(grid, nblocks, rows, blocks, sp)) return FV_ERR_ARG;
    const int nd = grid->ndim, nv = nd + comps->ncomp + 1;
    Layout L;
    plan(nblocks, blocks.data(), nd, nv, count_nprim(comps, eos, nv), eos->precision == FV_MIXED, L, nullptr,
         nullptr, nullptr, &sp);
    if (bytes) *bytes = L.total;
    return FV_OK;
}

extern "C" fv_status fv_init_split(const fv_grid* grid, int nblocks, const int* rows, const fv_components* comps,
                                   const fv_eos* eos, void* dev_workspace, size_t bytes, fv_ctx** out)
{
    if (!out) return FV_ERR_ARG;
    *out = nullptr;
    std::string why;
    fv_status s = validate(1, grid, comps, eos, why);
    std::vector<fv_grid> blocks;
    SplitInfo sp;
    const char* w = s ? nullptr : split_plan(grid, nblocks, rows, blocks, sp);
    if (!s && !w && eos->st_model == 1 && eos->sigma > 0.0)
        w = "the capillary jump model's curvature pass needs more ghost layers than slabs exchange";
    if (s || w) {
        fv_ctx* x = new (std::nothrow) fv_ctx();
        if (!x) return FV_ERR_ALLOC;
        x->msg = s ? why : std::string(w);
        *out = x;
        return FV_ERR_ARG;
    }
    return init_common(nblocks, blocks.data(), comps, eos, dev_workspace, dev_workspace ? bytes : 0, out, &sp,
                       grid->in_u);
}

static void prof_clear(fv_ctx* x);

extern "C" void fv_destroy(fv_ctx* x)
{
    if (!x) return;
    for (auto& g : x->graphs) cudaGraphExecDestroy(g.second);
    prof_clear(x);
    if (x->cap) cudaStreamDestroy(x->cap);
    if (x->up_stream) cudaStreamSynchronize(x->up_stream);
    if (x->down_stream) cudaStreamSynchronize(x->down_stream);
    for (cudaEvent_t e : {x->ev_up_done[0], x->ev_up_free[0], x->ev_down_ready[0], x->ev_down_done[0],
                          x->ev_up_done[1], x->ev_up_free[1], x->ev_down_ready[1], x->ev_down_done[1]})
        if (e) cudaEventDestroy(e);
    if (x->up_stream) cudaStreamDestroy(x->up_stream);
    if (x->down_stream) cudaStreamDestroy(x->down_stream);
    for (int i = 0; i < 2; ++i) {
        cudaFree(x->stage_up[i]);
        cudaFree(x->stage_down[i]);
    }
    if (x->owns && x->base) cudaFree(x->base);
    delete x;
}

extern "C" fv_status fv_set_stream(fv_ctx* x, void* stream)
{
    if (!x) return FV_ERR_ARG;
    x->stream = static_cast<cudaStream_t>(stream);
    return FV_OK;
}

static fv_status case_ok(fv_ctx* x, int icase)
{
    if (!x) return FV_ERR_ARG;
    if (!x->base) return fail(x, FV_ERR_STATE, "context not initialised%s");
    if (icase < 0 || icase >= x->ncases) return fail(x, FV_ERR_ARG, "case index out of range%s");
    return FV_OK;
}

static long long case_cells(const fv_ctx* x, int c)
{
    return (long long)x->cases[c].n[0] * x->cases[c].n[1] * x->cases[c].n[2];
}

static fv_status read_err(fv_ctx* x)
{
    int e = 0;
    CK(x, cudaMemcpy(&e, x->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e & ERR_TIMEOUT) return fail(x, FV_ERR_CUDA, "a bounded wait in a kernel gave up%s");
    if (e & ERR_NONCONV) return fail(x, FV_ERR_EOS_NONCONV, "closure iteration did not converge%s");
    if (e & ERR_NONPHYS) return fail(x, FV_ERR_NONPHYSICAL, "non-physical state met in a kernel%s");
    return FV_OK;
}

// Device-accessible address of caller memory: the pointer itself for device
// memory, the mapped alias of page-locked host memory (the conversion kernels
// then read or write it over the host link, with no staging copy), or null
// for other host memory (staged through the context's I/O buffer).
static const void* device_alias(const void* p, cudaMemcpyKind mk)
{
    if (mk == cudaMemcpyDeviceToDevice) return p;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer) return a.devicePointer;
    return nullptr;
}

static fv_status set_state_impl(fv_ctx* x, int c, int kind, const double* src, cudaMemcpyKind mk, bool sync)
{
    fv_status s = case_ok(x, c);
    if (s) return s;
    x->smax_fresh = false;
    if (!src) return fail(x, FV_ERR_ARG, "null state pointer%s");
    const long long n = case_cells(x, c);
    const CaseDesc& C = x->cases[c];
    const double* in = static_cast<const double*>(device_alias(src, mk));
    if (!in) {
        CK(x, cudaMemcpyAsync(x->io, src, sizeof(double) * x->nv * n, mk, x->stream));
        in = x->io;
    }
    if (kind == FV_CONSERVED && !x->ff) {
        CK(x, launch_copy_fields(x->nv, in, n, x->Q0 + C.qoff, x->L.ntot_q, n, x->stream));
    } else if (kind == FV_CONSERVED) {
        CK(x, launch_split(x->nv, in, n, x->Q0, x->L.ntot_q, C.qoff, x->stream));
    } else if (kind == FV_PRIMITIVE) {
        IoArgs A{x->P, x->d_cases, c, n, in, x->Q0, x->err};
        CK(x, launch_prim_to_cons(x->nd, x->nc, A, x->stream, x->ff));
    } else {
        return fail(x, FV_ERR_ARG, "bad state kind%s");
    }
    x->launches++;
    CK(x, cudaMemsetAsync(x->t + c, 0, sizeof(double), x->stream));
    if (sync) {
        CK(x, cudaStreamSynchronize(x->stream));
        return read_err(x);
    }
    return FV_OK;
}

static fv_status get_state_impl(fv_ctx* x, int c, int kind, double* dst, cudaMemcpyKind mk, bool sync)
{
    fv_status s = case_ok(x, c);
    if (s) return s;
    if (!dst) return fail(x, FV_ERR_ARG, "null state pointer%s");
    const long long n = case_cells(x, c);
    const CaseDesc& C = x->cases[c];
    double* const direct = static_cast<double*>(const_cast<void*>(device_alias(dst, mk)));
    double* out = direct ? direct : x->io;
    if (kind == FV_CONSERVED && !x->ff) {
        CK(x, launch_copy_fields(x->nv, x->Q0 + C.qoff, x->L.ntot_q, out, n, n, x->stream));
    } else if (kind == FV_CONSERVED) {
        CK(x, launch_join(x->nv, x->Q0, x->L.ntot_q, C.qoff, n, out, x->stream));
    } else if (kind == FV_PRIMITIVE) {
        IoArgs A{x->P, x->d_cases, c, n, x->Q0, out, x->err};
        CK(x, launch_cons_to_prim(x->nd, x->nc, A, x->stream, x->ff));
    } else {
        return fail(x, FV_ERR_ARG, "bad state kind%s");
    }
    x->launches++;
    if (!direct) CK(x, cudaMemcpyAsync(dst, x->io, sizeof(double) * x->nv * n, mk, x->stream));
    if (sync) {
        CK(x, cudaStreamSynchronize(x->stream));
        return read_err(x);
    }
    return FV_OK;
}

extern "C" fv_status fv_set_state(fv_ctx* x, int icase, int kind, const double* host)
{
    if (x && x->base) CK(x, cudaMemsetAsync(x->err, 0, sizeof(int), x->stream));
    return set_state_impl(x, icase, kind, host, cudaMemcpyHostToDevice, true);
}

extern "C" fv_status fv_get_state(fv_ctx* x, int icase, int kind, double* host)
{
    return get_state_impl(x, icase, kind, host, cudaMemcpyDeviceToHost, true);
}

// All cases in one call (concatenated per-case blocks): conserved state in
// device or page-locked host memory takes one kernel over every case; any
// other case goes case by case, with one synchronisation at the end.
static fv_status state_all(fv_ctx* x, int kind, double* buf, bool set)
{
    fv_status s = case_ok(x, 0);
    if (s) return s;
    if (!buf) return fail(x, FV_ERR_ARG, "null state pointer%s");
    const cudaMemcpyKind mk = set ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    if (set) {
        CK(x, cudaMemsetAsync(x->err, 0, sizeof(int), x->stream));
        x->smax_fresh = false;
    }
    const double* direct = static_cast<const double*>(device_alias(buf, mk));
    if (direct && kind == FV_CONSERVED) {
        CK(x, launch_all_cases(x->nv, x->ncases, x->d_cases, x->L.max_cells, direct, x->Q0, x->L.ntot_q, x->ff,
                               set ? 1 : 0, x->stream));
        x->launches++;
        if (set) CK(x, cudaMemsetAsync(x->t, 0, sizeof(double) * x->ncases, x->stream));
    } else {
        long long off = 0;
        for (int c = 0; c < x->ncases; ++c) {
            s = set ? set_state_impl(x, c, kind, buf + off, mk, false) : get_state_impl(x, c, kind, buf + off, mk, false);
            if (s) return s;
            off += (long long)x->nv * case_cells(x, c);
        }
    }
    CK(x, cudaStreamSynchronize(x->stream));
    return read_err(x);
}

extern "C" fv_status fv_set_state_all(fv_ctx* x, int kind, const double* host)
{
    return state_all(x, kind, const_cast<double*>(host), true);
}

extern "C" fv_status fv_get_state_all(fv_ctx* x, int kind, double* host)
{
    return state_all(x, kind, host, false);
}

// ---------------------------------------------------------------- pipelined I/O
static long long state_doubles(const fv_ctx* x)
{
    long long n = 0;
    for (int c = 0; c < x->ncases; ++c) n += (long long)x->nv * case_cells(x, c);
    return n;
}

static fv_status io_setup(fv_ctx* x)
{
    if (x->stage_up[0]) return FV_OK;
    const size_t bytes = sizeof(double) * (size_t)state_doubles(x);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaMalloc(&x->stage_up[i], bytes);
        if (e == cudaSuccess) e = cudaMalloc(&x->stage_down[i], bytes);
    }
    if (e != cudaSuccess) {
        for (int i = 0; i < 2; ++i) {
            cudaFree(x->stage_up[i]);
            cudaFree(x->stage_down[i]);
            x->stage_up[i] = x->stage_down[i] = nullptr;
        }
        cudaGetLastError();
        return fail(x, FV_ERR_ALLOC, "cudaMalloc of the I/O staging buffers failed%s");
    }
    CK(x, cudaStreamCreateWithFlags(&x->up_stream, cudaStreamNonBlocking));
    CK(x, cudaStreamCreateWithFlags(&x->down_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
        for (cudaEvent_t* ev : {&x->ev_up_done[i], &x->ev_up_free[i], &x->ev_down_ready[i], &x->ev_down_done[i]})
            CK(x, cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
        // the staging slots start free
        CK(x, cudaEventRecord(x->ev_up_free[i], x->stream));
        CK(x, cudaEventRecord(x->ev_down_done[i], x->down_stream));
    }
    return FV_OK;
}

// staging buffer <-> conserved registers of every case, on the context's stream
static fv_status stage_convert(fv_ctx* x, bool to_reg, double* buf)
{
    if (x->ncases <= 8) {
        long long off = 0;
        for (int c = 0; c < x->ncases; ++c) {
            const CaseDesc& C = x->cases[c];
            const long long n = case_cells(x, c);
            if (x->ff) {
                if (to_reg) CK(x, launch_split(x->nv, buf + off, n, x->Q0, x->L.ntot_q, C.qoff, x->stream));
                else CK(x, launch_join(x->nv, x->Q0, x->L.ntot_q, C.qoff, n, buf + off, x->stream));
            } else {
                if (to_reg) CK(x, launch_copy_fields(x->nv, buf + off, n, x->Q0 + C.qoff, x->L.ntot_q, n, x->stream));
                else CK(x, launch_copy_fields(x->nv, x->Q0 + C.qoff, x->L.ntot_q, buf + off, n, n, x->stream));
            }
            x->launches++;
            off += (long long)x->nv * n;
        }
        return FV_OK;
    }
    CK(x, launch_all_cases(x->nv, x->ncases, x->d_cases, x->L.max_cells, buf, x->Q0, x->L.ntot_q, x->ff,
                           to_reg ? 1 : 0, x->stream));
    x->launches++;
    return FV_OK;
}

extern "C" fv_status fv_upload_async(fv_ctx* x, const double* host)
{
    fv_status s = case_ok(x, 0);
    if (s) return s;
    if (!host) return fail(x, FV_ERR_ARG, "null state pointer%s");
    if (x->up_pending) return fail(x, FV_ERR_STATE, "the previous upload has not been committed%s");
    s = io_setup(x);
    if (s) return s;
    // this slot is free once the commit that last used it (two uploads ago)
    // has converted it
    const int u = x->up_next;
    CK(x, cudaStreamWaitEvent(x->up_stream, x->ev_up_free[u], 0));
    CK(x, cudaMemcpyAsync(x->stage_up[u], host, sizeof(double) * (size_t)state_doubles(x), cudaMemcpyHostToDevice,
                          x->up_stream));
    CK(x, cudaEventRecord(x->ev_up_done[u], x->up_stream));
    x->up_pending = true;
    x->up_slot = u;
    x->up_next = u ^ 1;
    return FV_OK;
}

extern "C" fv_status fv_commit_upload(fv_ctx* x)
{
    fv_status s = case_ok(x, 0);
    if (s) return s;
    if (!x->up_pending) return fail(x, FV_ERR_STATE, "no upload to commit%s");
    x->smax_fresh = false;
    const int u = x->up_slot;
    CK(x, cudaStreamWaitEvent(x->stream, x->ev_up_done[u], 0));
    s = stage_convert(x, true, x->stage_up[u]);
    if (s) return s;
    CK(x, cudaEventRecord(x->ev_up_free[u], x->stream));
    CK(x, cudaMemsetAsync(x->t, 0, sizeof(double) * x->ncases, x->stream));
    x->up_pending = false;
    return FV_OK;
}

extern "C" fv_status fv_download_async(fv_ctx* x, double* host)
{
    fv_status s = case_ok(x, 0);
    if (s) return s;
    if (!host) return fail(x, FV_ERR_ARG, "null state pointer%s");
    s = io_setup(x);
    if (s) return s;
    // the download that last used this slot (two downloads ago) must have left it
    const int d = x->down_next;
    CK(x, cudaStreamWaitEvent(x->stream, x->ev_down_done[d], 0));
    s = stage_convert(x, false, x->stage_down[d]);
    if (s) return s;
    CK(x, cudaEventRecord(x->ev_down_ready[d], x->stream));
    CK(x, cudaStreamWaitEvent(x->down_stream, x->ev_down_ready[d], 0));
    CK(x, cudaMemcpyAsync(host, x->stage_down[d], sizeof(double) * (size_t)state_doubles(x), cudaMemcpyDeviceToHost,
                          x->down_stream));
    CK(x, cudaEventRecord(x->ev_down_done[d], x->down_stream));
    x->down_next = d ^ 1;
    return FV_OK;
}

extern "C" fv_status fv_io_wait(fv_ctx* x)
{
    fv_status s = case_ok(x, 0);
    if (s) return s;
    if (x->up_stream) CK(x, cudaStreamSynchronize(x->up_stream));
    if (x->down_stream) CK(x, cudaStreamSynchronize(x->down_stream));
    CK(x, cudaStreamSynchronize(x->stream));
    return read_err(x);
}

extern "C" fv_status fv_set_state_device(fv_ctx* x, int icase, int kind, const double* dev)
{
    return set_state_impl(x, icase, kind, dev, cudaMemcpyDeviceToDevice, false);
}

extern "C" fv_status fv_get_state_device(fv_ctx* x, int icase, int kind, double* dev)
{
    return get_state_impl(x, icase, kind, dev, cudaMemcpyDeviceToDevice, false);
}

// One stage on stream s: primitives (+ per-case CFL maximum and dt when
// cfl > 0 at stage 1), then the fused flux/update kernel.
// event pair around one launch when profiling (never inside a capture)
static fv_status prof_begin(fv_ctx* x, cudaStream_t s, cudaEvent_t* ev)
{
    ev[0] = ev[1] = nullptr;
    if (!x->profiling || s == x->cap) return FV_OK;
    CK(x, cudaEventCreate(&ev[0]));
    CK(x, cudaEventCreate(&ev[1]));
    CK(x, cudaEventRecord(ev[0], s));
    return FV_OK;
}

static fv_status prof_end(fv_ctx* x, cudaStream_t s, cudaEvent_t* ev, int kind)
{
    if (!ev[0]) return FV_OK;
    CK(x, cudaEventRecord(ev[1], s));
    x->prof.push_back({kind, {ev[0], ev[1]}});
    return FV_OK;
}

#define PROF(kind, launch_expr)                         \
    do {                                                \
        cudaEvent_t ev_[2];                             \
        fv_status ps_ = prof_begin(x, s, ev_);          \
        if (ps_) return ps_;                            \
        CK(x, (launch_expr));                           \
        ps_ = prof_end(x, s, ev_, kind);                \
        if (ps_) return ps_;                            \
    } while (0)

// Halo exchange of a split grid: the two planes of register `reg` next to
// each shared side, copied from the neighbouring slab into the slab's ghost
// planes (one strided device-to-device copy of all fields per side).  The
// primitives of those planes are then recovered by the same pointwise
// closure as the neighbour's own, so the slabs see exactly the unsplit
// grid's ghost values.
static fv_status exchange(fv_ctx* x, double* reg, cudaStream_t s)
{
    if (!x->split) return FV_OK;
    const size_t es = sizeof(double);   // FP64 values or float-float pairs: 8 bytes
    const size_t pitch = es * (size_t)x->L.ntot_q;
    const int ld = x->sp.last;
    for (int c = 0; c < x->ncases; ++c) {
        const CaseDesc& C = x->cases[c];
        const long long plane = ld == 1 ? (long long)C.n[0] : (long long)C.n[0] * C.n[1];
        for (int side = 0; side < 2; ++side) {
            const int nb = side ? x->sp.nbr_hi[c] : x->sp.nbr_lo[c];
            if (nb < 0) continue;
            const CaseDesc& N = x->cases[nb];
            double* dst = reg + C.qoff + (side ? C.n[ld] * plane : -2 * plane);
            const double* src = reg + N.qoff + (side ? 0 : (N.n[ld] - 2) * plane);
            CK(x, cudaMemcpy2DAsync(dst, pitch, src, pitch, es * 2 * plane, x->nv, cudaMemcpyDeviceToDevice, s));
        }
    }
    return FV_OK;
}

// the fused kernel's last stage accumulates the next step's CFL wave speeds
// (FP32 form, viscosity-free modes)
static bool fused_cfl(const fv_ctx* x)
{
    return x->cfl_fuse && x->fused && x->mixed && !(march_mode(x) & MARCH_VISC);
}

// cold = false: the CFL pass of stage 1 is left out (smax already holds the
// wave speeds of q^n, written by the previous step's last fused stage)
static fv_status enqueue_stage(fv_ctx* x, int k, double cfl, cudaStream_t s, bool cold = true)
{
    double* in = k == 1 ? x->Q0 : (k == 2 ? x->QA : (k == 3 ? x->QB : x->QA));
    double* out = k == 1 ? x->QA : (k == 2 ? x->QB : (k == 3 ? x->QA : x->Q0));
    {
        fv_status e = exchange(x, in, s);
        if (e) return e;
    }
    const bool cfl_here = (k == 1 && cfl > 0.0);
    if (x->fused) {
        // the CFL pass (primitive recovery without writing primitives), then
        // one fused pass that recovers the primitives it needs itself
        const bool fc = cfl > 0.0 && fused_cfl(x);
        if (cfl_here) {
            if (cold || !fc) {
                // smax may hold an older last stage's speeds
                if (fc) CK(x, cudaMemsetAsync(x->smax, 0, sizeof(unsigned long long) * x->ncases, s));
                PrimArgs pa{x->P, x->d_cases, x->d_items_prim, x->L.n_items_prim, in, nullptr, x->in_u, x->smax,
                            x->err};
                PROF(FV_KERNEL_PRIM, launch_prim(x->nd, x->nc, x->mixed, pa, x->prim_grid, s, x->ff));
                x->launches++;
            }
            PROF(FV_KERNEL_DT, launch_dt(x->ncases, x->smax, x->dt, x->t, cfl, x->err, s, x->split));
            x->launches++;
        }
        const bool last = k == 4 && fc;
        MarchArgs ma{x->P, x->d_cases, x->d_items_march, x->n_items_march, in, x->Q0, out, x->in_u, x->dt,
                     LSRK_A[k - 1], x->err, last ? x->smax : nullptr};
        PROF(FV_KERNEL_STAGE, launch_march(x->nc, x->mixed, march_mode(x) | (last ? MARCH_CFL : 0), x->mvar, ma,
                                           x->march_grid, s));
        x->launches++;
        return FV_OK;
    }
    PrimArgs pa{x->P, x->d_cases, x->d_items_prim, x->L.n_items_prim, in, x->prim, x->in_u,
                cfl_here ? x->smax : nullptr, x->err};
    PROF(FV_KERNEL_PRIM, launch_prim(x->nd, x->nc, x->mixed, pa, x->prim_grid, s, x->ff));
    x->launches++;
    if (x->P.capj) {
        // cell curvatures of the capillary jump model, from the primitives
        PROF(FV_KERNEL_PRIM, launch_kappa(x->nd, x->mixed, pa, x->prim_grid, s));
        x->launches++;
    }
    if (cfl_here) {
        PROF(FV_KERNEL_DT, launch_dt(x->ncases, x->smax, x->dt, x->t, cfl, x->err, s, x->split));
        x->launches++;
    }
    if (x->zm) {
        ZArgs za{x->P, x->d_cases, x->d_items_z, x->n_items_z, x->zchunk, x->d_tmaps_z, x->Q0, out, x->dt,
                 LSRK_A[k - 1], x->err};
        PROF(FV_KERNEL_STAGE, launch_zmarch(x->nc, x->zvar, zm_visc(x), !x->mixed, za, x->zm_grid, x->zm_smem, s));
        x->launches++;
        return FV_OK;
    }
    StageArgs sa{x->P, x->d_cases, x->d_items_stage, x->n_items_cur, x->prim, stage_tmaps(x), x->Q0, out, x->dt,
                 LSRK_A[k - 1], x->err};
    PROF(FV_KERNEL_STAGE, launch_stage(x->nd, x->nc, x->mixed, x->tile, sa, x->stage_grid, x->smem, s, x->ff));
    x->launches++;
    return FV_OK;
}

extern "C" fv_status fv_rk_stage(fv_ctx* x, int k, double dt)
{
    fv_status s = case_ok(x, 0);
    if (s) return s;
    if (k < 1 || k > 4) return fail(x, FV_ERR_ARG, "stage index must be 1..4%s");
    s = tune(x);
    if (s) return s;
    x->smax_fresh = false;
    if (k == 1) {
        if (!(dt > 0.0)) return fail(x, FV_ERR_ARG, "dt must be positive%s");
        CK(x, launch_fill(x->dt, x->ncases, dt, x->stream));
        x->launches++;
    }
    s = enqueue_stage(x, k, 0.0, x->stream);
    if (s) return s;
    if (k == 4) {
        // advance every case's clock by dt (same as fv_step does)
        std::vector<double> tt(x->ncases);
        CK(x, cudaMemcpyAsync(tt.data(), x->t, sizeof(double) * x->ncases, cudaMemcpyDeviceToHost, x->stream));
        CK(x, cudaStreamSynchronize(x->stream));
        for (auto& v : tt) v += dt;
        CK(x, cudaMemcpyAsync(x->t, tt.data(), sizeof(double) * x->ncases, cudaMemcpyHostToDevice, x->stream));
        CK(x, cudaStreamSynchronize(x->stream));
    }
    return FV_OK;
}

static fv_status step_graph(fv_ctx* x, double cfl, bool cold, cudaGraphExec_t* exec)
{
    for (auto& g : x->graphs)
        if (g.first.first == cfl && g.first.second == cold) { *exec = g.second; return FV_OK; }
    cudaGraph_t graph;
    const long long before = x->launches;
    CK(x, cudaStreamBeginCapture(x->cap, cudaStreamCaptureModeThreadLocal));
    fv_status s = FV_OK;
    for (int k = 1; k <= 4 && !s; ++k) s = enqueue_stage(x, k, cfl, x->cap, cold);
    cudaError_t e = cudaStreamEndCapture(x->cap, &graph);
    x->launches = before;
    if (s) return s;
    if (e != cudaSuccess) return cuda_fail(x, e, "cudaStreamEndCapture");
    cudaGraphExec_t ge;
    e = cudaGraphInstantiate(&ge, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(x, e, "cudaGraphInstantiate");
    x->graphs.emplace_back(std::make_pair(cfl, cold), ge);
    *exec = ge;
    return FV_OK;
}

// kernels per step: 4 prim + 1 dt + 4 stage, or with the fused kernel
// 1 CFL pass + 1 dt + 4 fused stages (a warm step: no CFL pass)
static int launches_per_step(const fv_ctx* x, bool cold = true)
{
    return x->fused ? (cold || !fused_cfl(x) ? 6 : 5) : 9;
}

extern "C" fv_status fv_step_async(fv_ctx* x, int nsteps, double cfl)
{
    fv_status s = case_ok(x, 0);
    if (s) return s;
    if (nsteps < 0 || !(cfl > 0.0)) return fail(x, FV_ERR_ARG, "need nsteps >= 0 and cfl > 0%s");
    s = tune(x);
    if (s) return s;
    const bool fc = fused_cfl(x);
    // the first step is cold unless the last fused stage of the previous
    // call left the wave speeds of the present state
    const bool cold0 = !(fc && x->smax_fresh);
    if (x->profiling) {
        for (int i = 0; i < nsteps; ++i)
            for (int k = 1; k <= 4; ++k) {
                s = enqueue_stage(x, k, cfl, x->stream, i == 0 ? cold0 : !fc);
                if (s) return s;
            }
    } else if (nsteps > 0) {
        cudaGraphExec_t first, rest = nullptr;
        s = step_graph(x, cfl, cold0, &first);
        if (s) return s;
        if (nsteps > 1) {
            s = step_graph(x, cfl, !fc, &rest);
            if (s) return s;
        }
        CK(x, cudaGraphLaunch(first, x->stream));
        for (int i = 1; i < nsteps; ++i) CK(x, cudaGraphLaunch(rest, x->stream));
        x->launches += launches_per_step(x, cold0) + (long long)launches_per_step(x, !fc) * (nsteps - 1);
    }
    if (nsteps > 0) x->smax_fresh = fc;
    return FV_OK;
}

extern "C" fv_status fv_step(fv_ctx* x, int nsteps, double cfl, double* t_out)
{
    fv_status s = fv_step_async(x, nsteps, cfl);
    if (s) return s;
    CK(x, cudaStreamSynchronize(x->stream));
    if (t_out) CK(x, cudaMemcpy(t_out, x->t, sizeof(double), cudaMemcpyDeviceToHost));
    return read_err(x);
}

extern "C" fv_status fv_get_diag(fv_ctx* x, int icase, int what, void* out)
{
    fv_status s = case_ok(x, icase);
    if (s) return s;
    if (!out) return fail(x, FV_ERR_ARG, "null output%s");
    if (what == FV_DIAG_TOTALS) {
        const int nblk = 1024;
        CK(x, launch_totals(x->nv, x->Q0, x->L.ntot_q, x->cases[icase].qoff, case_cells(x, icase), x->partial,
                            nblk, x->stream, x->ff));
        x->launches++;
        std::vector<double> part((size_t)x->nv * nblk);
        CK(x, cudaMemcpyAsync(part.data(), x->partial, sizeof(double) * part.size(), cudaMemcpyDeviceToHost,
                              x->stream));
        CK(x, cudaStreamSynchronize(x->stream));
        double* o = static_cast<double*>(out);
        for (int v = 0; v < x->nv; ++v) {
            double sum = 0.0, comp = 0.0;   // Neumaier
            for (int b = 0; b < nblk; ++b) {
                const double y = part[(size_t)v * nblk + b], t = sum + y;
                comp += std::fabs(sum) >= std::fabs(y) ? (sum - t) + y : (y - t) + sum;
                sum = t;
            }
            o[v] = sum + comp;
        }
        return FV_OK;
    }
    if (what == FV_DIAG_FLAGS) {
        // App. D sensor of the current state: a primitive pass, then the
        // stage kernel's sensor function per interior cell (scratch: the QB
        // register, free between steps)
        if (!x->P.iles) return fail(x, FV_ERR_ARG, "the sensor flags need the App. D switch%s");
        s = exchange(x, x->Q0, x->stream);
        if (s) return s;
        PrimArgs pa{x->P, x->d_cases, x->d_items_prim, x->L.n_items_prim, x->Q0, x->prim, x->in_u, nullptr, x->err};
        CK(x, launch_prim(x->nd, x->nc, x->mixed, pa, x->prim_grid, x->stream, x->ff));
        x->launches++;
        const long long nc = case_cells(x, icase);
        unsigned char* dflags = reinterpret_cast<unsigned char*>(x->QB);
        CK(x, launch_sensor_dump(x->nd, x->mixed, x->P, x->d_cases, icase, x->prim, nc, dflags, x->stream));
        x->launches++;
        CK(x, cudaMemcpyAsync(out, dflags, (size_t)nc, cudaMemcpyDeviceToHost, x->stream));
        CK(x, cudaStreamSynchronize(x->stream));
        return FV_OK;
    }
    if (what == FV_DIAG_DT || what == FV_DIAG_TIME) {
        CK(x, cudaStreamSynchronize(x->stream));
        CK(x, cudaMemcpy(out, (what == FV_DIAG_DT ? x->dt : x->t) + icase, sizeof(double), cudaMemcpyDeviceToHost));
        return FV_OK;
    }
    if (what == FV_DIAG_TILE) {
        s = tune(x);
        if (s) return s;
        const TileDef td = tile_def(x->nd, variant_tile(x->nd, x->tile));
        double* o = static_cast<double*>(out);
        if (x->fused) {
            o[0] = MARCH_COLS; o[1] = x->chunk; o[2] = 1; o[3] = 32 * MARCH_WARPS;
        } else if (x->zm) {
            o[0] = ZM_TX; o[1] = ZM_TY; o[2] = x->zchunk; o[3] = zmarch_threads(x->zvar);
        } else {
            o[0] = td.x; o[1] = td.y; o[2] = td.z; o[3] = td.nt;
        }
        for (int t = 0; t < NTILES; ++t) o[4 + t] = x->tune_ms[t];
        o[8] = x->fused ? 1.0 : (x->zm ? 2.0 : 0.0);
        o[9] = x->zm ? x->zm_ms : x->march_ms;
        o[10] = x->prim_ms;
        o[11] = x->fused ? x->mvar : (x->zm ? x->zvar : -1);
        return FV_OK;
    }
    if (what == FV_DIAG_ERROR) {
        CK(x, cudaStreamSynchronize(x->stream));
        CK(x, cudaMemcpy(out, x->err, sizeof(int), cudaMemcpyDeviceToHost));
        return FV_OK;
    }
    return fail(x, FV_ERR_ARG, "unknown diagnostic%s");
}

extern "C" long long fv_launch_count(const fv_ctx* x) { return x ? x->launches : 0; }

static void prof_clear(fv_ctx* x)
{
    for (auto& p : x->prof) {
        cudaEventDestroy(p.second.first);
        cudaEventDestroy(p.second.second);
    }
    x->prof.clear();
}

extern "C" fv_status fv_profile(fv_ctx* x, int enable)
{
    fv_status s = case_ok(x, 0);
    if (s) return s;
    CK(x, cudaStreamSynchronize(x->stream));
    prof_clear(x);
    x->profiling = enable != 0;
    return FV_OK;
}

extern "C" fv_status fv_profile_read(fv_ctx* x, double* out)
{
    fv_status s = case_ok(x, 0);
    if (s) return s;
    if (!out) return fail(x, FV_ERR_ARG, "null output%s");
    CK(x, cudaStreamSynchronize(x->stream));
    for (int k = 0; k < 2 * FV_KERNEL_KINDS; ++k) out[k] = 0.0;
    for (auto& p : x->prof) {
        float ms = 0.f;
        CK(x, cudaEventElapsedTime(&ms, p.second.first, p.second.second));
        out[2 * p.first] += ms;
        out[2 * p.first + 1] += 1.0;
    }
    return FV_OK;
}

extern "C" const char* fv_last_error(const fv_ctx* x) { return x ? x->msg.c_str() : "null context"; }

namespace {
__device__ int g_probe_err;   // error word of the wait self-test (not reentrant)

// Self-test of the bounded wait: one block waits on an mbarrier that nothing
// ever completes, with `polls` polls; the give-up path sets ERR_TIMEOUT in
// *err exactly as the stage kernels' waits do.
__global__ void wait_probe_kernel(int polls, int* err)
{
    __shared__ __align__(8) unsigned long long bar;
    const unsigned a = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(a, 1);
        mbar_init_fence();
    }
    __syncthreads();
    const bool ok = tma_wait(a, 0u, polls);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
}
}  // namespace

extern "C" fv_status fv_wait_selftest(int polls, int* err_word)
{
    if (polls < 1 || !err_word) return FV_ERR_ARG;
    int* d = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&d), g_probe_err) != cudaSuccess) return FV_ERR_CUDA;
    if (cudaMemset(d, 0, sizeof(int)) != cudaSuccess) return FV_ERR_CUDA;
    wait_probe_kernel<<<1, 64>>>(polls, d);
    if (cudaGetLastError() != cudaSuccess) return FV_ERR_CUDA;
    if (cudaMemcpy(err_word, d, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FV_ERR_CUDA;
    return FV_OK;
}

// FP64 arithmetic-rate probe: every thread runs eight independent chains of
// dependent fused multiply-adds (enough independent work per warp to keep the
// FP64 pipe fed); the result only reaches memory if it equals a value the
// chains never produce, so the work cannot be dropped.
namespace {
__device__ double g_fma_sink;
__global__ void fma64_probe_kernel(int iters, double b, double c)
{
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 1e-3 * (threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == -1.0) g_fma_sink = s;
}
}  // namespace

extern "C" fv_status fv_probe_fp64(int blocks, int threads, int iters, double* ms, double* flops)
{
    if (blocks < 1 || threads < 32 || threads > 1024 || iters < 1 || !ms || !flops) return FV_ERR_ARG;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FV_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return FV_ERR_CUDA; }
    fv_status st = FV_OK;
    fma64_probe_kernel<<<blocks, threads>>>(iters, 0.9999999, 1e-7);   // warm-up
    cudaEventRecord(e0);
    fma64_probe_kernel<<<blocks, threads>>>(iters, 0.9999999, 1e-7);
    cudaEventRecord(e1);
    float t = 0.0f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
        st = FV_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = t;
    *flops = 2.0 * 8.0 * (double)blocks * threads * iters;
    return st;
}

extern "C" const char* fv_status_string(int s)
{
    switch (s) {
    case FV_OK: return "FV_OK";
    case FV_ERR_ARG: return "FV_ERR_ARG";
    case FV_ERR_ALLOC: return "FV_ERR_ALLOC";
    case FV_ERR_CUDA: return "FV_ERR_CUDA";
    case FV_ERR_EOS_NONCONV: return "FV_ERR_EOS_NONCONV";
    case FV_ERR_NONPHYSICAL: return "FV_ERR_NONPHYSICAL";
    case FV_ERR_STATE: return "FV_ERR_STATE";
    default: return "unknown status";
    }
}

// --------------------------------------------------------------------------
// fv_rk_stage_noalloc: one stage of one grid for callers that cannot allocate
// device memory.  Its scratch (case descriptor, dt, error word, tile work
// lists, primitive fields) lives in the file-scope array below, which every
// GPU that loads the library keeps until the process exits.  Host code must
// not hand g_noalloc_scratch to a kernel directly: in host code that name is
// a host-side stand-in, so its device address is looked up per device with
// cudaGetSymbolAddress.
// --------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[FV_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;
void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

__global__ void noalloc_setup_kernel(CaseDesc C, CaseDesc* dcase, double* dt, double dtv, int* err, int4* ist,
                                     int n_st, int4* ipr, int n_pr, int tx, int ty, int tz, TileDef st)
{
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 == 0) {
        *dcase = C;
        *dt = dtv;
        *err = 0;
    }
    // tile origins in the same x-fastest order as the context work lists
    // (stage tile st, primitive-pass tile tx x ty x tz)
    const int sx = (C.n[0] + st.x - 1) / st.x, sy = (C.n[1] + st.y - 1) / st.y;
    for (int i = i0; i < n_st; i += gridDim.x * blockDim.x)
        ist[i] = make_int4(0, (i % sx) * st.x, ((i / sx) % sy) * st.y, (i / (sx * sy)) * st.z);
    const int px = (C.g[0] + tx - 1) / tx, py = (C.g[1] + ty - 1) / ty;
    for (int i = i0; i < n_pr; i += gridDim.x * blockDim.x)
        ipr[i] = make_int4(0, (i % px) * tx, ((i / px) % py) * ty, (i / (px * py)) * tz);
}

// argument checks of the no-alloc path: those of fv_init for one case
// (nothing allocated) plus what this path leaves out
bool noalloc_args_ok(const fv_grid* g, const fv_components* cm, const fv_eos* e)
{
    if (check_args(1, g, cm, e)) return false;
    if (g->in_u) return false;   // per-cell inflow velocities would need device memory
    if (e->st_model == 1 && e->sigma > 0.0) return false;   // the curvature pass is not part of this path
    for (int k = 0; k < cm->ncomp; ++k)
        if (cm->comp[k].kind == FV_PR) return false;   // Peng-Robinson variants are not instantiated here
    // barotropic closure: FP64 form only (the mixed no-alloc variants are
    // instantiated for the stiffened-gas closure)
    if (cm->comp[0].kind == FV_BARO && e->precision != FV_FP64) return false;
    return true;
}

}  // namespace

extern "C" fv_status fv_rk_stage_noalloc(const fv_grid* grid, const fv_components* comps, const fv_eos* eos,
                                         int k, double dt, const double* q0, const double* qprev, double* qout,
                                         void* stream)
{
    if (!noalloc_args_ok(grid, comps, eos) || k < 1 || k > 4 || !(dt > 0.0) || !std::isfinite(dt) || !q0 ||
        !qprev || !qout)
        return FV_ERR_ARG;
    // qout may be q0 itself (the update is pointwise) but may not overlap
    // qprev, whose halo cells other blocks still read, or part of q0
    {
        const size_t bytes = sizeof(double) * (size_t)(grid->ndim + comps->ncomp + 1) * (size_t)grid->n[0] *
                             (size_t)grid->n[1] * (size_t)grid->n[2];
        const uintptr_t o = reinterpret_cast<uintptr_t>(qout), pv = reinterpret_cast<uintptr_t>(qprev),
                        z = reinterpret_cast<uintptr_t>(q0);
        if (o < pv + bytes && pv < o + bytes) return FV_ERR_ARG;
        if (qout != q0 && o < z + bytes && z < o + bytes) return FV_ERR_ARG;
    }
    // per-device set-up: the device address of the scratch array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return FV_ERR_CUDA;
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FV_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    unsigned char* base = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    fv_ctx x;   // parameters only: nothing below allocates
    x.nd = grid->ndim;
    x.nc = comps->ncomp;
    x.nv = x.nd + x.nc + 1;
    x.mixed = eos->precision == FV_MIXED;
    build_params(&x, comps, eos);
    CaseDesc C{};
    for (int d = 0; d < 3; ++d) {
        C.n[d] = grid->n[d];
        C.g[d] = d < x.nd ? grid->n[d] + 4 : 1;
        C.dx[d] = d < x.nd ? (grid->hi[d] - grid->lo[d]) / grid->n[d] : 1.0;
        C.idx[d] = 1.0 / C.dx[d];
        C.fdx[d] = float(C.dx[d]);
        C.fidx[d] = float(C.idx[d]);
        C.bc[d][0] = d < x.nd ? grid->bc[d][0] : 0;
        C.bc[d][1] = d < x.nd ? grid->bc[d][1] : 0;
    }
    C.inflow = grid->bc[0][0] == FV_BC_INFLOW;
    C.in_yc = grid->in_yc - grid->lo[1];
    C.in_zc = grid->in_zc - grid->lo[2];
    C.in_r2 = grid->in_radius * grid->in_radius;
    C.in_T = grid->in_T;
    for (int d = 0; d < 3; ++d) C.in_u0[d] = grid->in_u0[d];
    for (int c = 0; c < FV_MAX_COMP && c < MAXC; ++c) C.in_Y[c] = grid->in_Y[c];
    C.in_uoff = -1;
    const long long ncell = (long long)C.n[0] * C.n[1] * C.n[2];
    C.gp = (C.g[0] + 3) & ~3;
    const long long nghost = (long long)C.gp * C.g[1] * C.g[2];
    x.P.ntot_q = ncell;
    x.P.ntot_p = nghost;
    const int tx = tile_x(x.nd), ty = tile_y(x.nd), tz = tile_z(x.nd);
    const int var = kernel_variant(x.P, 0);
    const TileDef stile = tile_def(x.nd, variant_tile(x.nd, var));
    const long long n_pr = ntiles(C.g, x.nd);
    const long long n_st = (long long)((C.n[0] + stile.x - 1) / stile.x) * ((C.n[1] + stile.y - 1) / stile.y) *
                           ((C.n[2] + stile.z - 1) / stile.z);
    // scratch layout
    const size_t o_case = 0, o_dt = align256(sizeof(CaseDesc)), o_err = o_dt + 256, o_ist = o_err + 256;
    const size_t o_ipr = o_ist + align256(sizeof(int4) * n_st);
    const size_t o_prim = o_ipr + align256(sizeof(int4) * n_pr);
    const size_t rsz = x.mixed ? sizeof(float) : sizeof(double);
    const size_t need = o_prim + rsz * (size_t)x.nprim * (size_t)nghost;
    if (need > (size_t)FV_NOALLOC_SCRATCH_BYTES) return FV_ERR_ARG;

    CaseDesc* dcase = reinterpret_cast<CaseDesc*>(base + o_case);
    double* ddt = reinterpret_cast<double*>(base + o_dt);
    int* derr = reinterpret_cast<int*>(base + o_err);
    int4* ist = reinterpret_cast<int4*>(base + o_ist);
    int4* ipr = reinterpret_cast<int4*>(base + o_ipr);
    void* prim = base + o_prim;

    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FV_ERR_CUDA;
    const size_t smem = stage_smem(x.nd, x.nc, x.mixed, var, x.nprim);
    if (stage_set_smem(x.nd, x.nc, x.mixed, var, smem) != cudaSuccess) return FV_ERR_CUDA;
    const int gs = (int)std::min<long long>(n_st, (long long)nsm * stage_occupancy(x.nd, x.nc, x.mixed, var, smem));
    const int gp = (int)std::min<long long>(n_pr, (long long)nsm * prim_occupancy(x.nd, x.nc, x.mixed));
    const int nsetup = (int)std::min<long long>(1024, (std::max(n_st, n_pr) + 255) / 256);

    noalloc_setup_kernel<<<std::max(1, nsetup), 256, 0, s>>>(C, dcase, ddt, dt, derr, ist, (int)n_st, ipr,
                                                            (int)n_pr, tx, ty, tz, stile);
    if (cudaGetLastError() != cudaSuccess) return FV_ERR_CUDA;
    PrimArgs pa{x.P, dcase, ipr, (int)n_pr, qprev, prim, nullptr, nullptr, derr};
    if (launch_prim(x.nd, x.nc, x.mixed, pa, gp, s) != cudaSuccess) return FV_ERR_CUDA;
    StageArgs sa{x.P, dcase, ist, (int)n_st, prim, nullptr, q0, qout, ddt, LSRK_A[k - 1], derr};
    if (launch_stage(x.nd, x.nc, x.mixed, var, sa, gs, smem, s) != cudaSuccess) return FV_ERR_CUDA;
    int e = 0;
    if (cudaMemcpyAsync(&e, derr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return FV_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FV_ERR_CUDA;
    if (e & ERR_TIMEOUT) return FV_ERR_CUDA;
    if (e & ERR_NONCONV) return FV_ERR_EOS_NONCONV;
    if (e & ERR_NONPHYS) return FV_ERR_NONPHYSICAL;
    return FV_OK;
}
