// Kernel instantiations, build shard 11 (lengths with index % 16 == 11).
#define CUBIC_SHARD 11
#include "kernels_shard.cuh"
