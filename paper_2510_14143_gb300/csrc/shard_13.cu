// Kernel instantiations, build shard 13 (lengths with index % 16 == 13).
#define CUBIC_SHARD 13
#include "kernels_shard.cuh"
