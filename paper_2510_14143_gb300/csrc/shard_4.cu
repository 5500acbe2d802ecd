// Kernel instantiations, build shard 4 (lengths with index % 16 == 4).
#define CUBIC_SHARD 4
#include "kernels_shard.cuh"
