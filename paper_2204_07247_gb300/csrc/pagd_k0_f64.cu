// pagd_k0_f64.cu -- kernel instantiation for runtime line lengths, FP64 iterations.
#include "kernels.cuh"
PAGD_INSTANTIATE(double, 0)
