// Compiled launch shape 2 of the sloppy stencil (64 threads per block, 6 resident blocks
// per SM, next-direction prefetch on): its own translation unit so that the
// shapes compile in parallel.
#include "s16_kernels.cuh"

TMND_S16_DEFINE_SHAPE(2, 64, 6, true)
