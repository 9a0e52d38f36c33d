// Compiled launch shape 0 of the sloppy stencil (128 threads per block, 3 resident blocks
// per SM, next-direction prefetch on): its own translation unit so that the
// shapes compile in parallel.
#include "s16_kernels.cuh"

TMND_S16_DEFINE_SHAPE(0, 128, 3, true)
