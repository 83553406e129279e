// fv_march_fc.cu -- fused 2D stage kernel, FP32 arithmetic with float-float
// registers: the last-stage modes that also accumulate the next step's CFL
// wave speed (MARCH_CFL; a translation unit of their own so the build
// compiles them in parallel with fv_march_f.cu).
#define FV_MR float
#define FV_MQ float2
#define FV_MSUFFIX fc
#define FV_MCFL 1
#define FV_MBARO 1
#include "fv_march_inst.cuh"
