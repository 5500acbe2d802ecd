// Kernel instantiations, build shard 10 (lengths with index % 16 == 10).
#define CUBIC_SHARD 10
#include "kernels_shard.cuh"
