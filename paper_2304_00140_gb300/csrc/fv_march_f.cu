// fv_march_f.cu -- fused 2D stage kernel, FP32 arithmetic with float-float registers.
#define FV_MR float
#define FV_MQ float2
#define FV_MSUFFIX f
#define FV_MBARO 1
#include "fv_march_inst.cuh"
