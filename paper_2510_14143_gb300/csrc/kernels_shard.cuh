// kernels_shard.cuh -- instantiates the kernels of one build shard.  Each
// shard_<k>.cu includes this with CUBIC_SHARD defined, so the lengths compile
// in parallel translation units.
#pragma once

#include "registry.cuh"

#ifndef CUBIC_SHARD
#error "define CUBIC_SHARD"
#endif

namespace cubic {

template <int I>
static void register_entry(AxisKernels *table)
{
    if constexpr (I < kNumLengths) {
        if constexpr (I % kShards == CUBIC_SHARD) table[I] = make_axis<kLengths[I]>();
        register_entry<I + 1>(table);
    }
}

template <>
void register_shard<CUBIC_SHARD>(AxisKernels *table)
{
    register_entry<0>(table);
}

}  // namespace cubic
