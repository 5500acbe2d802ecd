// Kernel instantiations, build shard 5 (lengths with index % 16 == 5).
#define CUBIC_SHARD 5
#include "kernels_shard.cuh"
