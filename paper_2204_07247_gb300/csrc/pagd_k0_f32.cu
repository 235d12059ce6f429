// pagd_k0_f32.cu -- kernel instantiation for runtime line lengths, FP32 iterations.
#include "kernels.cuh"
PAGD_INSTANTIATE(float, 0)
