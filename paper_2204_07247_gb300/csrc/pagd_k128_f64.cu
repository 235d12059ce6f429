// pagd_k128_f64.cu -- kernel instantiation for fixed line length 128, FP64 iterations.
#include "kernels.cuh"
PAGD_INSTANTIATE(double, 128)
