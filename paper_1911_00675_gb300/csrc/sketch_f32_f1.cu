// Sketch kernel, FP32 candidate + FP64 recheck path, family 1.
#define PMH_F32 true
#define PMH_FAM 1
#include "sketch_inst.cuh"
