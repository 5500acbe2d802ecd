// Kernel instantiations, build shard 7 (lengths with index % 16 == 7).
#define CUBIC_SHARD 7
#include "kernels_shard.cuh"
