// pagd_k64.cu -- kernel instantiation for fixed line length 64.
#include "kernels.cuh"
PAGD_INSTANTIATE(64)
