// registry.cuh -- per-length kernel table.  For every supported axis length n
// there are one or more compiled launch-shape variants of each pass:
//   X pass: threads per line P and line pairs per CTA L (all five modes)
//   Y / Z pass: threads per line P and adjacent columns per CTA B
// Variant 0 is the default; the autotuner (tuner.cu) times the others on a
// plan's own buffers and picks per pass.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cudaTypedefs.h>

#include <mutex>
#include <utility>

#include "colpass_tma.cuh"
#include "passes.cuh"

namespace cubic {

using XLaunch = cudaError_t (*)(const XArgs &, cudaStream_t);
using YLaunch = cudaError_t (*)(const YArgs &, cudaStream_t);
using ZLaunch = cudaError_t (*)(const ZArgs &, cudaStream_t);
using XMultiLaunch = cudaError_t (*)(const MultiTable<XArgs> *, int64_t blocks, cudaStream_t);
using YMultiLaunch = cudaError_t (*)(const MultiTable<YArgs> *, int64_t blocks, int inverse, cudaStream_t);
using ZMultiLaunch = cudaError_t (*)(const MultiTable<ZArgs> *, int64_t blocks, int mode, cudaStream_t);

constexpr int kMaxVariants = 8;

struct XVariant {
    int P = 0, L = 0;
    XLaunch fn[XM_COUNT] = {};
    XMultiLaunch m[XM_COUNT] = {};  // the same kernels over a table of volumes
};

struct YZVariant {
    int P = 0, B = 0;
    bool tma = false;  // persistent TMA-pipelined kernel
    YLaunch y = nullptr;
    ZLaunch z = nullptr;
    // plain variants: the same kernels over a table of volumes (null for TMA variants,
    // whose tensor maps are per volume)
    YMultiLaunch ym = nullptr;
    ZMultiLaunch zm = nullptr;
};

struct AxisKernels {
    int n = 0;
    int nx = 0, nyz = 0;  // number of X and Y/Z variants
    XVariant xv[kMaxVariants];
    YZVariant yzv[kMaxVariants];
    // multi-volume launches (batched path): X with xv[0]'s shape, Y/Z with P0 x 16 columns
    XMultiLaunch xm[XM_COUNT] = {};
    YMultiLaunch ym = nullptr;
    ZMultiLaunch zm = nullptr;
    int xm_lines = 0;  // line pairs per X CTA
    int m_cols = 16;   // columns per Y/Z CTA
    // the adjoint X passes of the differentiable path (XM_ADJ_R, XM_ADJ_U), in one shape
    XLaunch adj[2] = {};
};

// Table lookup; nullptr if n has no kernels.
const AxisKernels *find_axis(int64_t n);

// ------------------------------------------------------------------ launchers

// Launch with programmatic stream serialization: the kernel may start while its
// predecessor in the stream is still running (its CTAs wait in pdl_wait before
// touching the predecessor's output), which hides launch latency and prologues.
template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*fn)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, std::forward<Args>(args)...);
}

inline cudaError_t set_smem(const void *fn, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int N, int P, int L, int MODE, bool PF = false>
cudaError_t launch_x(const XArgs &a, cudaStream_t st)
{
    const int64_t pairs = (a.rows + 1) / 2;
    const int64_t grid = (pairs + L - 1) / L;
    constexpr size_t smem = x_smem_bytes<N, P, L, MODE, PF>();
    auto fn = x_kernel<N, P, L, MODE, PF>();
    static cudaError_t attr = set_smem((const void *)fn, smem);
    if (attr != cudaSuccess) return attr;
    if (grid == 0) return cudaSuccess;
    return launch_pdl(fn, dim3((unsigned)grid), dim3(P * L), smem, st, a, (const MultiTable<XArgs> *)nullptr);
}

template <int N, int P, int B>
cudaError_t launch_y(const YArgs &a, cudaStream_t st)
{
    dim3 grid((unsigned)((a.col1 - a.col0 + B - 1) / B), (unsigned)a.nz);
    constexpr size_t smem = sizeof(float2) * (B * N + tw_table_size(N, N / P));
    auto fn = k_ypass<N, P, B>;
    static cudaError_t attr = set_smem((const void *)fn, smem);
    if (attr != cudaSuccess) return attr;
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    return launch_pdl(fn, grid, dim3(P * B), smem, st, a, (const MultiTable<YArgs> *)nullptr, a.inverse);
}

template <int N, int P, int B>
cudaError_t launch_z(const ZArgs &a, cudaStream_t st)
{
    dim3 grid((unsigned)((a.col1 - a.col0 + B - 1) / B), (unsigned)a.ny);
    constexpr size_t smem = sizeof(float2) * (B * N + tw_table_size(N, N / P));
    auto fn = k_zpass<N, P, B>;
    static cudaError_t attr = set_smem((const void *)fn, smem);
    if (attr != cudaSuccess) return attr;
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    return launch_pdl(fn, grid, dim3(P * B), smem, st, a, (const MultiTable<ZArgs> *)nullptr, a.mode);
}

// Default split: fewest radix stages with at most 32 (n >= 256) or 40 elements
// per thread.  Alternative: at most 16 elements per thread (more threads, more
// stages, fewer registers).
template <int N>
struct AxisShape {
    static constexpr int P0 = (N == 1) ? 1 : choose_threads(N, N >= 256 ? 32 : 40);
    static constexpr int P1 = (N == 1) ? 1 : choose_threads(N, 16);
    static_assert(P0 > 0, "no thread split for this length");
    static constexpr int lines(int P, int threads) { return P >= threads ? 1 : threads / P; }
    // lengths that get tuned variants (the large, bandwidth-critical ones)
    static constexpr bool kTuned = (N >= 64);
    static constexpr bool kAlt = kTuned && P1 > 0 && P1 != P0 && P1 * 16 <= 1024;
};

// ------------------------------------------------------------------ TMA column passes

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();  // defined in capi.cu

// Tensor map over a [nz][ny][xp] complex array viewed as float32 [nz][ny][2 xp].  The
// extents along y and z may stop short of the array (ny_ext <= ny, nz_ext <= nz): loads
// past them read zeros and stores past them are dropped.
inline cudaError_t encode_spectrum_map(CUtensorMap *tm, const void *base, int64_t nz, int64_t ny, int64_t xp,
                                       int box0, int box1, int box2, int64_t ny_ext = 0, int64_t nz_ext = 0)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * xp), (cuuint64_t)(ny_ext > 0 ? ny_ext : ny),
                                (cuuint64_t)(nz_ext > 0 ? nz_ext : nz)};
    const cuuint64_t strides[2] = {(cuuint64_t)(2 * xp * sizeof(float)), (cuuint64_t)(2 * xp * ny * sizeof(float))};
    const cuuint32_t box[3] = {(cuuint32_t)box0, (cuuint32_t)box1, (cuuint32_t)box2};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int N, int P, int B, int KIND, int NS, bool HREAL>
int col_grid_cap()
{
    static int cap = [] {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_colpass_tma<N, P, B, KIND, NS, HREAL>, P * B,
                                                      col_smem_bytes<N, P, B, KIND, NS, HREAL>());
        return (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
    }();
    return cap;
}

// nload / nstore: rows of each line loaded / stored (0: all N).  Y: rows along y of a
// spectrum array of nz planes of ny = N rows.  Z: planes of a spectrum array holding
// nload planes (loads and stores both stop there); H always has N planes.
template <int N, int P, int B, int KIND, int NS, bool HREAL = false>
cudaError_t launch_col(const float2 *spec, const float2 *H, const float *Hr, int64_t nz, int64_t ny, int64_t xp,
                       int64_t col0, int64_t col1, int64_t outer, const float2 *tw, int mode, float scale,
                       unsigned *err, cudaStream_t st, int64_t nload = 0, int64_t nstore = 0,
                       unsigned long long wait_ns = 0, int skip_first = 0)
{
    constexpr int R = box_rows(N);
    constexpr size_t smem = col_smem_bytes<N, P, B, KIND, NS, HREAL>();
    auto fn = k_colpass_tma<N, P, B, KIND, NS, HREAL>;
    static cudaError_t attr = set_smem((const void *)fn, smem);
    if (attr != cudaSuccess) return attr;
    if (col0 % B != 0) return cudaErrorInvalidValue;
    const int64_t nl = nload > 0 ? nload : N, ns = nstore > 0 ? nstore : N;
    if (nl > N || ns > N || (KIND == COL_Z && ns != nl)) return cudaErrorInvalidValue;
    CUtensorMap tm_spec, tm_h;
    // Z: the spectrum array itself holds nl planes
    cudaError_t e = (KIND == COL_Y) ? encode_spectrum_map(&tm_spec, spec, nz, ny, xp, 2 * B, R, 1, nl)
                                    : encode_spectrum_map(&tm_spec, spec, nl, ny, xp, 2 * B, 1, R);
    if (e != cudaSuccess) return e;
    if (KIND == COL_Z && mode == ZM_MUL_REAL && Hr) {
        // real H: float32 [nz][ny][xp], boxes of B floats
        PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
        if (!enc) return cudaErrorNotSupported;
        const cuuint64_t dims[3] = {(cuuint64_t)xp, (cuuint64_t)ny, (cuuint64_t)nz};
        const cuuint64_t strides[2] = {(cuuint64_t)(xp * sizeof(float)), (cuuint64_t)(xp * ny * sizeof(float))};
        const cuuint32_t box[3] = {(cuuint32_t)B, 1, (cuuint32_t)R};
        const cuuint32_t estr[3] = {1, 1, 1};
        if (enc(&tm_h, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(Hr), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    } else if (KIND == COL_Z && H) {
        e = encode_spectrum_map(&tm_h, H, nz, ny, xp, 2 * B, 1, R);
        if (e != cudaSuccess) return e;
    } else if (KIND == COL_Y && ns != nl) {
        e = encode_spectrum_map(&tm_h, spec, nz, ny, xp, 2 * B, R, 1, ns);  // the store map
        if (e != cudaSuccess) return e;
    } else {
        tm_h = tm_spec;
    }
    ColArgs c;
    c.tw = tw;
    c.ntiles_col = (col1 - col0 + B - 1) / B;
    c.ntiles = c.ntiles_col * outer;
    c.col_tile0 = col0 / B;
    c.mode = mode;
    c.scale = scale;
    c.err = err;
    c.nstore = (int)ns;
    c.wait_ns = wait_ns;
    c.skip_first = skip_first;
    if (c.ntiles == 0) return cudaSuccess;
    const int64_t cap = col_grid_cap<N, P, B, KIND, NS, HREAL>();
    const unsigned grid = (unsigned)(c.ntiles < cap ? c.ntiles : cap);
    return launch_pdl(fn, dim3(grid), dim3(P * B), smem, st, tm_spec, tm_h, c);
}

template <int N, int P, int B, int NS>
cudaError_t launch_y_tma(const YArgs &a, cudaStream_t st)
{
    return launch_col<N, P, B, COL_Y, NS>(a.spec, nullptr, nullptr, a.nz, N, a.xp, a.col0, a.col1, a.nz, a.tw, a.inverse, 1.f,
                                      a.err, st, a.nload, a.nstore, a.wait_ns, a.skip_first);
}

template <int N, int P, int B, int NS>
cudaError_t launch_z_tma(const ZArgs &a, cudaStream_t st)
{
    const bool needH = a.mode == ZM_CONV || a.mode == ZM_CORR;
    if (a.mode == ZM_MUL_REAL)
        return launch_col<N, P, B, COL_Z, NS, true>(a.spec, nullptr, a.Hr, N, a.ny, a.xp, a.col0, a.col1, a.ny,
                                                    a.tw, a.mode, a.scale, a.err, st, a.nload, a.nstore, a.wait_ns,
                                                    a.skip_first);
    return launch_col<N, P, B, COL_Z, NS>(a.spec, needH ? a.H : nullptr, a.Hr, N, a.ny, a.xp, a.col0, a.col1, a.ny, a.tw,
                                      a.mode, a.scale, a.err, st, a.nload, a.nstore, a.wait_ns, a.skip_first);
}

// Y and Z tile widths and stage counts may differ: the Z pass also stages H.
// widest plain (non-TMA) Y/Z column tile, 16, 8 or 4 columns, whose CTA fits: B * N
// complex elements plus the twiddle table in shared memory, and at most 512 threads
// (more would cap the long lines' transforms below their register needs)
template <int N, int P>
constexpr int plain_cols()
{
    constexpr size_t tw = (size_t)tw_table_size(N, N / P) * sizeof(float2);
    return (16 * N * sizeof(float2) + tw <= 220 * 1024 && P * 16 <= 512)  ? 16
           : (8 * N * sizeof(float2) + tw <= 220 * 1024 && P * 8 <= 512) ? 8
                                                                           : 4;
}

template <int N, int P, int BY, int NSY, int BZ, int NSZ>
YZVariant make_yzvariant_tma()
{
    YZVariant v;
    v.P = P;
    v.B = BY;
    v.tma = true;
    if constexpr (BY > 0)
        v.y = launch_y_tma<N, P, BY, NSY>;
    else
        v.y = launch_y<N, P, plain_cols<N, P>()>;
    if constexpr (BZ > 0)
        v.z = launch_z_tma<N, P, BZ, NSZ>;
    else
        v.z = launch_z<N, P, plain_cols<N, P>()>;
    return v;
}

constexpr size_t kTmaSmemBudget = 220 * 1024;

// A TMA tile of B columns fits when two stages fit the budget, the CTA has at most 1024
// threads and every box of the tile starts on a 128-byte boundary in shared memory
// (boxes of box_rows(N) rows sit at multiples of box_rows(N) * B * 8 bytes).
template <int N, int P, int B, int KIND>
constexpr bool tma_tile_fits()
{
    return col_smem_bytes<N, P, B, KIND, 2>() <= kTmaSmemBudget && P * B <= 1024 &&
           (N <= 256 || (box_rows(N) * B) % 16 == 0);
}

// widest column tile that fits: 16 or 8 columns, or 4 for lines longer than 1024;
// 0: no TMA variant
template <int N, int KIND>
constexpr int tma_cols()
{
    constexpr int P = AxisShape<N>::P0;
    return tma_tile_fits<N, P, 16, KIND>()                ? 16
           : tma_tile_fits<N, P, 8, KIND>()               ? 8
           : (N > 1024 && tma_tile_fits<N, P, 4, KIND>()) ? 4
                                                          : 0;
}

// most stages (2..4) that fit the budget at that width, for thread split P.
// CTAs of fewer than 256 threads keep two stages: they rely on several CTAs per
// SM for issue slots, which deep stages would crowd out.
template <int N, int P, int KIND>
constexpr int tma_stages()
{
    constexpr int B = tma_cols<N, KIND>();
    if constexpr (B == 0 || P * B < 256) {
        return 2;
    } else {
        return col_smem_bytes<N, P, B, KIND, 4>() <= kTmaSmemBudget   ? 4
               : col_smem_bytes<N, P, B, KIND, 3>() <= kTmaSmemBudget ? 3
                                                                       : 2;
    }
}

template <int N, int P, int L, int MODE, bool PF = false>
cudaError_t launch_x_multi(const MultiTable<XArgs> *tab, int64_t blocks, cudaStream_t st)
{
    constexpr size_t smem = x_smem_bytes<N, P, L, MODE, PF>();
    auto fn = x_kernel<N, P, L, MODE, PF>();
    static cudaError_t attr = set_smem((const void *)fn, smem);
    if (attr != cudaSuccess) return attr;
    if (blocks == 0) return cudaSuccess;
    return launch_pdl(fn, dim3((unsigned)blocks), dim3(P * L), smem, st, XArgs{}, tab);
}

template <int N, int P, int B>
cudaError_t launch_y_multi(const MultiTable<YArgs> *tab, int64_t blocks, int inverse, cudaStream_t st)
{
    constexpr size_t smem = sizeof(float2) * (B * N + tw_table_size(N, N / P));
    auto fn = k_ypass<N, P, B>;
    static cudaError_t attr = set_smem((const void *)fn, smem);
    if (attr != cudaSuccess) return attr;
    if (blocks == 0) return cudaSuccess;
    return launch_pdl(fn, dim3((unsigned)blocks), dim3(P * B), smem, st, YArgs{}, tab, inverse);
}

template <int N, int P, int B>
cudaError_t launch_z_multi(const MultiTable<ZArgs> *tab, int64_t blocks, int mode, cudaStream_t st)
{
    constexpr size_t smem = sizeof(float2) * (B * N + tw_table_size(N, N / P));
    auto fn = k_zpass<N, P, B>;
    static cudaError_t attr = set_smem((const void *)fn, smem);
    if (attr != cudaSuccess) return attr;
    if (blocks == 0) return cudaSuccess;
    return launch_pdl(fn, dim3((unsigned)blocks), dim3(P * B), smem, st, ZArgs{}, tab, mode);
}

// PR / PU: the ratio / update pass reads its operand rows through an L2 prefetch
// instead of staging them in shared memory
template <int N, int P, int L, bool PR = false, bool PU = false>
XVariant make_xvariant()
{
    XVariant v;
    v.P = P;
    v.L = L;
    v.fn[XM_FWD] = launch_x<N, P, L, XM_FWD>;
    v.fn[XM_INV] = launch_x<N, P, L, XM_INV>;
    v.fn[XM_RATIO] = launch_x<N, P, L, XM_RATIO, PR>;
    v.fn[XM_UPDATE] = launch_x<N, P, L, XM_UPDATE, PU>;
    v.fn[XM_FINAL] = launch_x<N, P, L, XM_FINAL>;
    v.m[XM_FWD] = launch_x_multi<N, P, L, XM_FWD>;
    v.m[XM_INV] = launch_x_multi<N, P, L, XM_INV>;
    v.m[XM_RATIO] = launch_x_multi<N, P, L, XM_RATIO, PR>;
    v.m[XM_UPDATE] = launch_x_multi<N, P, L, XM_UPDATE, PU>;
    v.m[XM_FINAL] = launch_x_multi<N, P, L, XM_FINAL>;
    return v;
}

template <int N, int P, int B>
YZVariant make_yzvariant()
{
    YZVariant v;
    v.P = P;
    v.B = B;
    v.y = launch_y<N, P, B>;
    v.z = launch_z<N, P, B>;
    v.ym = launch_y_multi<N, P, B>;
    v.zm = launch_z_multi<N, P, B>;
    return v;
}

// ------------------------------------------------------------------ shapes

inline void push_yz(AxisKernels &k, const YZVariant &v)
{
    if (k.nyz < kMaxVariants) k.yzv[k.nyz++] = v;
}

inline void push_x(AxisKernels &k, const XVariant &v)
{
    if (k.nx < kMaxVariants) k.xv[k.nx++] = v;
}

template <int N>
AxisKernels make_axis()
{
    using S = AxisShape<N>;
    AxisKernels k;
    k.n = N;
    constexpr int P0 = S::P0;
    // X default: for long lines the lighter split (<= 16 elements per thread, more
    // CTAs per SM) measured faster; the other split stays available to the tuner
    if constexpr (N >= 256 && S::kAlt) {
        k.xv[0] = make_xvariant<N, S::P1, S::lines(S::P1, 128)>();
        k.xv[1] = make_xvariant<N, P0, S::lines(P0, 128)>();
        k.nx = 2;
    } else {
        k.xv[0] = make_xvariant<N, P0, S::lines(P0, 128)>();
        k.nx = 1;
    }
    {
        // the split with at most 16 elements per thread where there is one: these passes
        // carry more operands than the forward ones, and the wider split keeps registers low
        constexpr int PA = (S::P1 > 0 && S::P1 * 16 <= 1024) ? S::P1 : P0;
        constexpr int LA = S::lines(PA, 128);
        k.adj[0] = launch_x<N, PA, LA, XM_ADJ_R>;
        k.adj[1] = launch_x<N, PA, LA, XM_ADJ_U>;
    }
    // lines longer than 1024: a split with up to 40 elements per thread may need fewer
    // stages (2560: 40 x 8 x 8 instead of 20 x 4 x 4 x 4 x 2)
    constexpr int PW = N > 1024 ? choose_threads(N, 40) : -1;
    if constexpr (PW > 0 && PW != P0 && PW != S::P1) {
        push_x(k, make_xvariant<N, PW, S::lines(PW, 128)>());
        // its operand rows through L2: no staged rows, one CTA more per SM
        if constexpr (N % 4 == 0) push_x(k, make_xvariant<N, PW, S::lines(PW, 128), true, true>());
    }
    // lines longer than 1024 hold one line pair per CTA in the default split (72 to 128
    // threads): two line pairs share one copy of the stage twiddle table
    if constexpr (N > 1024 && S::lines(P0, 128) == 1 && 2 * P0 <= 512) {
        push_x(k, make_xvariant<N, P0, 2>());
        if constexpr (N % 4 == 0) push_x(k, make_xvariant<N, P0, 2, true, true>());
    }
    // long lines: the default split with the ratio and/or the update reading their
    // operand rows through L2 (less shared memory per CTA, more CTAs per SM)
    if constexpr (N >= 256 && N % 4 == 0) {
        constexpr int PX = S::kAlt ? S::P1 : P0;
        constexpr int LX = S::lines(PX, 128);
        push_x(k, make_xvariant<N, PX, LX, true, true>());
        push_x(k, make_xvariant<N, PX, LX, true, false>());
        push_x(k, make_xvariant<N, PX, LX, false, true>());
        // the split with more elements per thread (fewer stages, fewer instructions) is held
        // to few CTAs per SM by its staged operand rows: both prefetched
        if constexpr (S::kAlt && N <= 1024) push_x(k, make_xvariant<N, P0, S::lines(P0, 128), true, true>());
    }
    constexpr int XL = S::lines(P0, 128);
    k.xm[XM_FWD] = launch_x_multi<N, P0, XL, XM_FWD>;
    k.xm[XM_INV] = launch_x_multi<N, P0, XL, XM_INV>;
    k.xm[XM_RATIO] = launch_x_multi<N, P0, XL, XM_RATIO>;
    k.xm[XM_UPDATE] = launch_x_multi<N, P0, XL, XM_UPDATE>;
    k.xm[XM_FINAL] = launch_x_multi<N, P0, XL, XM_FINAL>;
    k.xm_lines = XL;
    constexpr int B0 = plain_cols<N, P0>();
    // Short lines (one to four threads each): the plain shape with more threads per line
    // (at most 8 elements each) and wide tiles, so that small volumes still fill the GPU
    constexpr int PS = choose_threads(N, 8) > 0 ? choose_threads(N, 8) : P0;
    constexpr int BS = PS * 64 <= 512 ? 64 : PS * 32 <= 512 ? 32 : 16;
    constexpr bool kWide = P0 <= 4 && N >= 8 && PS * BS <= 512 &&
                           BS * N * sizeof(float2) + tw_table_size(N, N / PS) * sizeof(float2) <= 220 * 1024;
    // the batched path's multi-volume launches keep the default shape: the wide one
    // measured slower there (129.7 against 122.9 ms for the 64-volume batch)
    k.ym = launch_y_multi<N, P0, B0>;
    k.zm = launch_z_multi<N, P0, B0>;
    k.m_cols = B0;
    k.nyz = 0;
    constexpr int BY = tma_cols<N, COL_Y>(), BZ = tma_cols<N, COL_Z>();
    if constexpr (S::kTuned && (BY > 0 || BZ > 0)) {
        // TMA-pipelined variants first: they are the defaults where they exist
        // deepest pipeline that fits, then two stages (more CTAs per SM)
        constexpr int NY0 = tma_stages<N, P0, COL_Y>(), NZ0 = tma_stages<N, P0, COL_Z>();
        push_yz(k, make_yzvariant_tma<N, P0, BY, NY0, BZ, NZ0>());
        if constexpr (NY0 > 2 || NZ0 > 2) push_yz(k, make_yzvariant_tma<N, P0, BY, 2, BZ, 2>());
        if constexpr (S::P1 > 0 && S::P1 != P0 && S::P1 * (BY > BZ ? BY : BZ) <= 1024 && S::P1 * 16 <= 1024) {
            constexpr int P1 = S::P1;
            constexpr int NY1 = tma_stages<N, P1, COL_Y>(), NZ1 = tma_stages<N, P1, COL_Z>();
            push_yz(k, make_yzvariant_tma<N, P1, BY, NY1, BZ, NZ1>());
            if constexpr (NY1 > 2 || NZ1 > 2) push_yz(k, make_yzvariant_tma<N, P1, BY, 2, BZ, 2>());
            // Z-oriented shapes (their Y kernel is the one above): three stages, or
            // 32-column tiles
            if constexpr (BZ == 16 && col_smem_bytes<N, P1, 16, COL_Z, 3>() <= kTmaSmemBudget)
                push_yz(k, make_yzvariant_tma<N, P1, BY, NY1, 16, 3>());
            if constexpr (BZ == 16 && P1 * 32 <= 1024 && col_smem_bytes<N, P1, 32, COL_Z, 2>() <= kTmaSmemBudget)
                push_yz(k, make_yzvariant_tma<N, P1, BY, NY1, 32, 2>());
        }
    }
    push_yz(k, make_yzvariant<N, P0, B0>());
    // the wide plain shape as a tuning choice too (the reverse sweep's product passes run
    // on the widest plain variant)
    if constexpr (kWide) push_yz(k, make_yzvariant<N, PS, BS>());
    if constexpr (!S::kTuned && N >= 8 && BY > 0 && P0 * 64 <= 1024 && tma_tile_fits<N, P0, 64, COL_Z>()) {
        // short lines have one or two threads each: a TMA variant whose Z tile is 64
        // columns wide gives the CTA enough threads (thin stacks, e.g. 30 slices)
        push_yz(k, make_yzvariant_tma<N, P0, BY, 2, 64, 2>());
    }
    if constexpr (S::kTuned) {
        if constexpr (B0 == 16) push_yz(k, make_yzvariant<N, P0, 8>());
        if constexpr (S::kAlt) {
            constexpr int P1 = S::P1;
            if constexpr (N < 256) push_x(k, make_xvariant<N, P1, S::lines(P1, 128)>());
            constexpr int B1 = plain_cols<N, P1>() < 8 ? plain_cols<N, P1>() : 8;
            push_yz(k, make_yzvariant<N, P1, B1>());
        }
    }
    return k;
}

// The supported lengths; shard s of the build instantiates entries i with
// i % kShards == s.
constexpr int kLengths[] = {1,   2,   3,   4,   5,   6,   8,   9,   10,  12,  15,  16,  18,  20,  24,
                            25,  27,  30,  32,  36,  40,  45,  48,  50,  54,  60,  64,  72,  75,  80,
                            81,  90,  96,  100, 108, 120, 125, 128, 135, 144, 150, 160, 192, 256, 320,
                            384, 512, 640, 768, 1024, 2160, 2304, 2560, 2592};
constexpr int kNumLengths = sizeof(kLengths) / sizeof(kLengths[0]);
constexpr int kShards = 16;

// Fill table entries of shard S (defined in kernels_shard.cuh).
template <int S>
void register_shard(AxisKernels *table);

}  // namespace cubic
