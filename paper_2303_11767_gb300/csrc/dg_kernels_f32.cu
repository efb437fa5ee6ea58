// FP32 instantiation of the device code (tables applied in FP32, tables and
// mass sums built and reduced in FP64).
#define DG_REAL float
#define DG_REAL_IS_F32 1
#include "dg_kernels.cuh"
