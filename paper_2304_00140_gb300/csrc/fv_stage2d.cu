// fv_stage2d.cu -- 2D double instantiations of the stage kernel.
#define FV_ND 2
#define FV_REAL double
#define FV_IS_FLOAT 0
#define FV_SUFFIX 2d
#include "fv_stage_inst.cuh"
