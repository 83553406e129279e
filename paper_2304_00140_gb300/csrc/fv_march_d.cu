// fv_march_d.cu -- fused 2D stage kernel, FP64.
#define FV_MR double
#define FV_MQ double
#define FV_MSUFFIX d
#include "fv_march_inst.cuh"
