// pagd_k128_f32.cu -- kernel instantiation for fixed line length 128, FP32 iterations.
#include "kernels.cuh"
PAGD_INSTANTIATE(float, 128)
