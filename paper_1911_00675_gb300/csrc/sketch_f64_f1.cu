// Sketch kernel, plain FP64 path, family 1.
#define PMH_F32 false
#define PMH_FAM 1
#include "sketch_inst.cuh"
