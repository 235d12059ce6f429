// pagd_k512.cu -- kernel instantiation for fixed line length 512.
#include "kernels.cuh"
PAGD_INSTANTIATE(512)
