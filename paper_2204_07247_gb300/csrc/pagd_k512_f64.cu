// pagd_k512_f64.cu -- kernel instantiation for fixed line length 512, FP64 iterations.
#include "kernels.cuh"
PAGD_INSTANTIATE(double, 512)
