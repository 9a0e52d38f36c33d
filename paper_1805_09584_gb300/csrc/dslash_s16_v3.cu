// Compiled launch shape 3 of the sloppy stencil (256 threads per block, 1 resident blocks
// per SM, next-direction prefetch on): its own translation unit so that the
// shapes compile in parallel.
#include "s16_kernels.cuh"

TMND_S16_DEFINE_SHAPE(3, 256, 1, true)
