// Sketch kernel, plain FP64 path, family 2.
#define PMH_F32 false
#define PMH_FAM 2
#include "sketch_inst.cuh"
