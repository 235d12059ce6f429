// pagd_k64_f64.cu -- kernel instantiation for fixed line length 64, FP64 iterations.
#include "kernels.cuh"
PAGD_INSTANTIATE(double, 64)
