// Kernel instantiations, build shard 3 (lengths with index % 16 == 3).
#define CUBIC_SHARD 3
#include "kernels_shard.cuh"
