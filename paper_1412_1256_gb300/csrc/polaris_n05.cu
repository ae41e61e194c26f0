// FFT-correlator batch runner for N = 2^5 (one translation unit per size so that
// the sizes compile in parallel).
#include "polaris_kernels.cuh"
POLARIS_INSTANTIATE(5)
