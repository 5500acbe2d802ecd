// Kernel instantiations, build shard 6 (lengths with index % 16 == 6).
#define CUBIC_SHARD 6
#include "kernels_shard.cuh"
