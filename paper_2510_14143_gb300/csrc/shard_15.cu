// Kernel instantiations, build shard 15 (lengths with index % 16 == 15).
#define CUBIC_SHARD 15
#include "kernels_shard.cuh"
