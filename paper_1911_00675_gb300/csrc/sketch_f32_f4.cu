// Sketch kernel, FP32 candidate + FP64 recheck path, family 4.
#define PMH_F32 true
#define PMH_FAM 4
#include "sketch_inst.cuh"
