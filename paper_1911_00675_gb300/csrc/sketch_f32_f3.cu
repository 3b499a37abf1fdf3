// Sketch kernel, FP32 candidate + FP64 recheck path, family 3.
#define PMH_F32 true
#define PMH_FAM 3
#include "sketch_inst.cuh"
