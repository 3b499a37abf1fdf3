// Sketch kernel, FP32 candidate + FP64 recheck path, family 2.
#define PMH_F32 true
#define PMH_FAM 2
#include "sketch_inst.cuh"
