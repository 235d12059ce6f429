// pagd_k256_f32.cu -- kernel instantiation for fixed line length 256, FP32 iterations.
#include "kernels.cuh"
PAGD_INSTANTIATE(float, 256)
