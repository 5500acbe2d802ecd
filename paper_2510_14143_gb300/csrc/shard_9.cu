// Kernel instantiations, build shard 9 (lengths with index % 16 == 9).
#define CUBIC_SHARD 9
#include "kernels_shard.cuh"
