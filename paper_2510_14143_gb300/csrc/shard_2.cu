// Kernel instantiations, build shard 2 (lengths with index % 16 == 2).
#define CUBIC_SHARD 2
#include "kernels_shard.cuh"
