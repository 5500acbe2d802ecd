// Kernel instantiations, build shard 8 (lengths with index % 16 == 8).
#define CUBIC_SHARD 8
#include "kernels_shard.cuh"
