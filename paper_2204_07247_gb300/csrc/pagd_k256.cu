// pagd_k256.cu -- kernel instantiation for fixed line length 256.
#include "kernels.cuh"
PAGD_INSTANTIATE(256)
