// FFT-correlator batch runner for N = 2^20 (one translation unit per size so that
// the sizes compile in parallel).
#include "polaris_kernels.cuh"
POLARIS_INSTANTIATE(20)
