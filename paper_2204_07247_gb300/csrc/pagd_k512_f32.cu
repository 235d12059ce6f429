// pagd_k512_f32.cu -- kernel instantiation for fixed line length 512, FP32 iterations.
#include "kernels.cuh"
PAGD_INSTANTIATE(float, 512)
