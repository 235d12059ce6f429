// pagd_batch_f64.cu -- batched kernel instantiation, FP64 iterations.
#include "batch.cuh"
PAGD_INSTANTIATE_BATCH(double)
