// pagd_k0.cu -- kernel instantiation for fixed line length 0 (0: runtime length).
#include "kernels.cuh"
PAGD_INSTANTIATE(0)
