// pagd_k64_f32.cu -- kernel instantiation for fixed line length 64, FP32 iterations.
#include "kernels.cuh"
PAGD_INSTANTIATE(float, 64)
