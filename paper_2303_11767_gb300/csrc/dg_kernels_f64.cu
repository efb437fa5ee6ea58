// FP64 instantiation of the device code.
#define DG_REAL double
#include "dg_kernels.cuh"
