// Kernel instantiations, build shard 0 (lengths with index % 16 == 0).
#define CUBIC_SHARD 0
#include "kernels_shard.cuh"
