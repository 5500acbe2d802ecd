// Kernel instantiations, build shard 12 (lengths with index % 16 == 12).
#define CUBIC_SHARD 12
#include "kernels_shard.cuh"
