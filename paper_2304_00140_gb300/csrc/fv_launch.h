// fv_launch.h -- host-side launchers of the templated kernels (one
// translation unit per kernel family so the build compiles them in parallel).
#pragma once

#include <cuda_runtime.h>

#include "fv_kernels.cuh"

namespace tfv {

// prim kernel and stage kernel, dispatched on (ndim, ncomp, mixed)
// ff = 1: float-float (float2) registers of the mixed form; ff = 0: double registers
cudaError_t launch_prim(int nd, int nc, int mixed, const PrimArgs& A, int grid, cudaStream_t s, int ff = 0);
// `tile` is a stage-kernel variant (NVARIANTS): a candidate tile of TILES2 /
// TILES3, or one of the tile-0 variants for Peng-Robinson or a run-time limiter pair
cudaError_t launch_stage(int nd, int nc, int mixed, int tile, const StageArgs& A, int grid, size_t smem,
                         cudaStream_t s, int ff = 0);
size_t stage_smem(int nd, int nc, int mixed, int tile, int nprim, int ff = 0);
cudaError_t stage_set_smem(int nd, int nc, int mixed, int tile, size_t smem, int ff = 0);
int stage_occupancy(int nd, int nc, int mixed, int tile, size_t smem, int ff = 0);   // blocks per SM (0: cannot run)
int prim_occupancy(int nd, int nc, int mixed);
// curvature pass of the capillary jump model (after the primitive pass, on its work list)
cudaError_t launch_kappa(int nd, int mixed, const PrimArgs& A, int grid, cudaStream_t s);

// fused 2D stage kernel (fv_march.cuh), stiffened/ideal-gas closure.
// mode: MARCH_ILES | MARCH_CSF bits of the scheme.  var: 0 Table 4.2 limiter
// pair, 2 limiter pair read at run time.  mixed = 1: float-float registers.
struct MarchArgs;
constexpr int MARCH_WARPS = 4;
cudaError_t launch_march(int nc, int mixed, int mode, int var, const MarchArgs& A, int grid, cudaStream_t s);
int march_occupancy(int nc, int mixed, int mode, int var);   // blocks per SM

// z-marching 3D stage kernel (fv_zmarch.cuh), FP32-mixed, stiffened/ideal gas,
// TMA plane loads.  var: 0 / 1 / 3 Table 4.2 limiter pair with 320 / 256 /
// 352 threads, 2 limiter pair read at run time (320 threads).  visc = 1: with
// the Eq. 2-2 viscous, heat-flux and gravity terms (variants 1 and 2).
struct ZArgs;
// fp64 = 1: the FP64 form (variants 1 and 2, no viscous terms).
cudaError_t launch_zmarch(int nc, int var, int visc, int fp64, const ZArgs& A, int grid, size_t smem, cudaStream_t s);
cudaError_t zmarch_set_smem(int nc, int var, int visc, int fp64, size_t smem);
int zmarch_occupancy(int nc, int var, int visc, int fp64, size_t smem);   // blocks per SM (0: no such variant)
int zmarch_threads(int var);
size_t zmarch_smem(int nc, int nprim, int fp64);

// state I/O and diagnostics (FP64)
struct IoArgs {
    DevParams P;
    const CaseDesc* cases;
    int icase;
    long long ncell;            // interior cells of the case
    const void* in;             // [nv][ncell] doubles (case-local) or a register
    void* out;                  // a register or [nv][ncell] doubles (case-local)
    int* err;
};
cudaError_t launch_prim_to_cons(int nd, int nc, const IoArgs& A, cudaStream_t s, int ff);
cudaError_t launch_cons_to_prim(int nd, int nc, const IoArgs& A, cudaStream_t s, int ff);
// case-local conserved doubles <-> float-float registers; in / out may be
// device memory or mapped page-locked host memory
cudaError_t launch_split(int nv, const double* in, long long ncell, void* reg, long long ntot_q, long long off,
                         cudaStream_t s);
cudaError_t launch_join(int nv, const void* reg, long long ntot_q, long long off, long long ncell, double* out,
                        cudaStream_t s);
// every case's conserved doubles (concatenated [case][nv][ncell], device or
// mapped host memory) <-> the registers; to_reg = 1 writes the registers
cudaError_t launch_all_cases(int nv, int ncases, const CaseDesc* cases, long long max_cells, const double* host,
                             void* reg, long long ntot_q, int ff, int to_reg, cudaStream_t s);
// nv fields of ncell doubles between two field strides (FP64 registers)
cudaError_t launch_copy_fields(int nv, const double* in, long long in_stride, double* out, long long out_stride,
                               long long ncell, cudaStream_t s);
// per-block Kahan partial sums of each field of one case: partial[nv][nblk]
cudaError_t launch_totals(int nv, const void* q, long long ntot_q, long long off, long long ncell,
                          double* partial, int nblk, cudaStream_t s, int ff);
// dt[c] = cfl / smax[c]; t[c] += dt[c]; smax[c] = 0   (per case)
// grouped = true: every case takes the smallest dt of all (the slabs of one
// split grid: the min-reduction of dt)
cudaError_t launch_dt(int ncases, unsigned long long* smax, double* dt, double* t, double cfl, int* err,
                      cudaStream_t s, bool grouped = false);
cudaError_t launch_fill(double* x, int n, double v, cudaStream_t s);
// App. D flag (0/1) of every interior cell of case icase from the primitive
// arrays into out[ncell] (device)
cudaError_t launch_sensor_dump(int nd, int mixed, const DevParams& P, const CaseDesc* cases, int icase,
                               const void* prim, long long ncell, unsigned char* out, cudaStream_t s);

}  // namespace tfv
