// Compiled launch shape 1 of the sloppy stencil (128 threads per block, 3 resident blocks
// per SM, next-direction prefetch off): its own translation unit so that the
// shapes compile in parallel.
#include "s16_kernels.cuh"

TMND_S16_DEFINE_SHAPE(1, 128, 3, false)
