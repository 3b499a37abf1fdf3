// Sketch kernel, plain FP64 path, family 3.
#define PMH_F32 false
#define PMH_FAM 3
#include "sketch_inst.cuh"
