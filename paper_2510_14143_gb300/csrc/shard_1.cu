// Kernel instantiations, build shard 1 (lengths with index % 16 == 1).
#define CUBIC_SHARD 1
#include "kernels_shard.cuh"
