// pagd_k256_f64.cu -- kernel instantiation for fixed line length 256, FP64 iterations.
#include "kernels.cuh"
PAGD_INSTANTIATE(double, 256)
