// Batched resampling kernels (filled in by the persistent batched path).
#include "common.cuh"
#include "internal.h"
