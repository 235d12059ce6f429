// pagd_k128.cu -- kernel instantiation for fixed line length 128.
#include "kernels.cuh"
PAGD_INSTANTIATE(128)
