// pagd_batch_f32.cu -- batched kernel instantiation, FP32 iterations.
#include "batch.cuh"
PAGD_INSTANTIATE_BATCH(float)
