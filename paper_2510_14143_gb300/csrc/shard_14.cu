// Kernel instantiations, build shard 14 (lengths with index % 16 == 14).
#define CUBIC_SHARD 14
#include "kernels_shard.cuh"
