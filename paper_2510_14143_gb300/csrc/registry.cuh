// registry.cuh -- per-length kernel table: for every supported axis length n
// the X-pass variants, the Y pass and the Z pass compiled for that n, with the
// launch shape each uses.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "passes.cuh"

namespace cubic {

using XLaunch = cudaError_t (*)(const XArgs &, cudaStream_t);
using YLaunch = cudaError_t (*)(const YArgs &, cudaStream_t);
using ZLaunch = cudaError_t (*)(const ZArgs &, cudaStream_t);

struct AxisKernels {
    int n = 0;
    int x_threads = 0, x_lines = 0;  // X pass: threads per line, line pairs per CTA
    int yz_threads = 0, yz_cols = 0; // Y/Z passes: threads per line, columns per CTA
    XLaunch x[XM_COUNT] = {};
    YLaunch y = nullptr;
    ZLaunch z = nullptr;
};

// Table lookup; nullptr if n has no kernels.
const AxisKernels *find_axis(int64_t n);

// Every supported length, ascending (for enumeration by callers).
int supported_lengths(const int **out);

// ------------------------------------------------------------------ shapes

template <int N>
struct AxisShape {
    static constexpr int Emax = N >= 256 ? 32 : 40;
    static constexpr int P = (N == 1) ? 1 : choose_threads(N, Emax);
    static_assert(P > 0, "no thread split for this length");
    static constexpr int XL = (P >= 128) ? 1 : 128 / P;  // line pairs per X CTA
    static constexpr int B = 16;                           // columns per Y/Z CTA
};

inline cudaError_t set_smem(const void *fn, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int N, int MODE>
cudaError_t launch_x(const XArgs &a, cudaStream_t st)
{
    using S = AxisShape<N>;
    const int64_t pairs = (a.rows + 1) / 2;
    const int64_t grid = (pairs + S::XL - 1) / S::XL;
    const size_t smem = sizeof(float2) * S::XL * x_smem_line<N>();
    auto fn = k_xpass<N, S::P, S::XL, MODE>;
    static cudaError_t attr = set_smem((const void *)fn, smem);
    if (attr != cudaSuccess) return attr;
    if (grid == 0) return cudaSuccess;
    fn<<<(unsigned)grid, S::P * S::XL, smem, st>>>(a);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_y(const YArgs &a, cudaStream_t st)
{
    using S = AxisShape<N>;
    dim3 grid((unsigned)((a.xh + S::B - 1) / S::B), (unsigned)a.nz);
    const size_t smem = sizeof(float2) * S::B * N;
    auto fn = k_ypass<N, S::P, S::B>;
    static cudaError_t attr = set_smem((const void *)fn, smem);
    if (attr != cudaSuccess) return attr;
    fn<<<grid, S::P * S::B, smem, st>>>(a);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_z(const ZArgs &a, cudaStream_t st)
{
    using S = AxisShape<N>;
    dim3 grid((unsigned)((a.xh + S::B - 1) / S::B), (unsigned)a.ny);
    const size_t smem = sizeof(float2) * S::B * N;
    auto fn = k_zpass<N, S::P, S::B>;
    static cudaError_t attr = set_smem((const void *)fn, smem);
    if (attr != cudaSuccess) return attr;
    fn<<<grid, S::P * S::B, smem, st>>>(a);
    return cudaGetLastError();
}

template <int N>
AxisKernels make_axis()
{
    using S = AxisShape<N>;
    AxisKernels k;
    k.n = N;
    k.x_threads = S::P;
    k.x_lines = S::XL;
    k.yz_threads = S::P;
    k.yz_cols = S::B;
    k.x[XM_FWD] = launch_x<N, XM_FWD>;
    k.x[XM_INV] = launch_x<N, XM_INV>;
    k.x[XM_RATIO] = launch_x<N, XM_RATIO>;
    k.x[XM_UPDATE] = launch_x<N, XM_UPDATE>;
    k.x[XM_FINAL] = launch_x<N, XM_FINAL>;
    k.y = launch_y<N>;
    k.z = launch_z<N>;
    return k;
}

// The supported lengths; shard s of the build instantiates entries i with
// i % kShards == s.
constexpr int kLengths[] = {1,   2,   3,   4,   5,   6,   8,   9,   10,  12,  15,  16,  18,  20,  24,
                            25,  27,  30,  32,  36,  40,  45,  48,  50,  54,  60,  64,  72,  75,  80,
                            81,  90,  96,  100, 108, 120, 125, 128, 135, 144, 150, 160, 192, 256, 320,
                            384, 512, 640, 768, 1024};
constexpr int kNumLengths = sizeof(kLengths) / sizeof(kLengths[0]);
constexpr int kShards = 8;

// Fill table entries of shard S (defined in kernels_shard.cuh).
template <int S>
void register_shard(AxisKernels *table);

}  // namespace cubic
