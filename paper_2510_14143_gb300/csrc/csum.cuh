// csum.cuh -- compensated float32 sums on the GPU.
//
// Reductions other than the flux sum and the twiddle factors run in float32 with
// an error term carried beside the sum, so a sum of n terms keeps about twice the
// float precision instead of losing log2(n) bits.
//
// CFloat: a register accumulator, value = s - c (Kahan; c is the negated low part).
// catomic_add: an atomic accumulator of two floats, value = hi + lo.  atomicAdd
// returns the value it added x to, so the adding thread can recover the exact
// rounding error of that add (Knuth's TwoSum) and add it into lo.
#pragma once

#include <cuda_runtime.h>

namespace cubic {

struct CFloat {
    float s, c;  // value = s - c (c: Kahan compensation, the negated lost low part)
};

__device__ __forceinline__ CFloat cf_add(CFloat a, float x)
{
    const float y = x - a.c;
    const float t = a.s + y;
    a.c = (t - a.s) - y;
    a.s = t;
    return a;
}

__device__ __forceinline__ CFloat cf_merge(CFloat a, CFloat b)
{
    // TwoSum of the leading parts (s + err == a.s + b.s exactly), then the tails:
    // value = s + err - a.c - b.c
    const float s = a.s + b.s;
    const float bb = s - a.s;
    const float err = (a.s - (s - bb)) + (b.s - bb);
    return CFloat{s, a.c + b.c - err};
}

// TwoSum: the exact error of fl(a + b), given s = fl(a + b).
__device__ __forceinline__ float two_sum_err(float a, float b, float s)
{
    const float bb = s - a;
    return (a - (s - bb)) + (b - bb);
}

// *hi + *lo += x, for global or shared memory.
__device__ __forceinline__ void catomic_add(float *hi, float *lo, float x)
{
    const float old = atomicAdd(hi, x);
    const float err = two_sum_err(old, x, old + x);
    if (err != 0.f) atomicAdd(lo, err);
}

}  // namespace cubic
