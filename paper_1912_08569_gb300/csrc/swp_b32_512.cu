// The FP32 batched step kernel with 512-thread blocks (128 registers per thread).
#include "swp_internal.h"
#define SWP_BATCH_NS batched512
#define SWP_BATCH_THREADS 512
#define SWP_BATCH_MINB 1
#include "swp_batch_impl.cuh"
namespace swp {
SWP_BATCH_DEFINE(float)
}
