// Sketch kernel, plain FP64 path, family 4.
#define PMH_F32 false
#define PMH_FAM 4
#include "sketch_inst.cuh"
