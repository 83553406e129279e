// fv_stage2f.cu -- 2D float instantiations of the stage kernel.
#define FV_ND 2
#define FV_REAL float
#define FV_IS_FLOAT 1
#define FV_SUFFIX 2f
#include "fv_stage_inst.cuh"
