// lens.cuh -- all-lengths passes of the batched path.
//
// A batch of volumes of many sizes would need one launch per pass and distinct axis
// length.  The kernels here take every volume whose axis length is in one length class
// in ONE launch per pass: each CTA finds its volume in a device table, then branches to
// that length's compiled transform.  All CTAs have kLensThreads threads; a length's
// shape (P threads per line, lines per CTA) is fixed at compile time by lens_threads(N),
// and the few threads past the CTA's whole lines idle through the transforms on a spare
// line of shared memory, so that every thread meets every barrier.
//
// The tables list the volumes in order of length, so CTAs that run at the same time on
// an SM mostly take the same branch.
//
// Y and Z tile a volume's lines in the order (plane, column): B = kLensThreads / P
// consecutive lines per CTA, so that no tile is cut short at the last column of a plane
// (the spectra of small volumes have few columns, nx / 2 + 1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "registry.cuh"

namespace cubic {

constexpr int kLensThreads = 128;

// threads per line: among the splits with at most 24 elements per thread, those with the
// fewest radix stages, and of them the one with the fewest elements per thread (fewer
// registers and less shared memory per thread, so more warps per SM); lengths divisible
// by 30 have none and take the default split of at most 40
constexpr int lens_threads(int N)
{
    int bestP = -1, bestS = 1 << 20;
    for (int P = N; P >= 1; --P) {
        if (N % P) continue;
        const int E = N / P;
        if (E > 24 || E % radical(N)) continue;
        const int st = plan_stages(N, E);
        if (st >= 0 && st < bestS) {
            bestS = st;
            bestP = P;
        }
    }
    return bestP > 0 ? bestP : choose_threads(N, 40);
}

// line pairs (X) or lines (Y, Z) per CTA
constexpr int lens_lines(int N) { return kLensThreads / lens_threads(N); }

template <int... Ns>
struct LenList {
    static constexpr bool has(int64_t len) { return ((len == Ns) || ...); }
    static constexpr int max_elems()
    {
        int m = 0;
        ((m = Ns / lens_threads(Ns) > m ? Ns / lens_threads(Ns) : m), ...);
        return m;
    }
};

// The lengths with all-lengths kernels, the 5-smooth lengths of small volumes, in three
// classes of one kernel each, by elements per thread, so that the registers a kernel is
// held to suit its lengths: up to 16, 18 to 24, and 30 (lengths divisible by 30 have no
// split between 16 and 30).
using LensLight = LenList<48, 50, 64, 72, 75, 81, 100, 125, 128, 135, 144>;
using LensMedium = LenList<54, 80, 96, 108, 160>;
using LensWide = LenList<60, 90, 120, 150>;
static_assert(LensLight::max_elems() <= 16 && LensMedium::max_elems() <= 24 && LensWide::max_elems() <= 30,
              "length classes");
constexpr int kLensClasses = 3;

// the class of an axis length (-1: none)
constexpr int lens_class(int64_t n)
{
    return LensLight::has(n) ? 0 : LensMedium::has(n) ? 1 : LensWide::has(n) ? 2 : -1;
}

// CTAs per SM a kernel is compiled for, which sets its register budget per thread.  The
// light class: 102 registers, at which none of its bodies spills.  The others: 128, at
// which the bodies of 24 and 30 elements per thread spill a little (up to 160 bytes a
// thread), for a third more warps per SM than at 168.
enum LensKind : int { LK_X = 0, LK_Y = 1, LK_Z = 2 };
template <class Lens, int KIND>
constexpr int lens_min_blocks()
{
    if constexpr (Lens::max_elems() <= 16)
        return 5;  // 102 registers
    else
        return 4;                     // 128
}

// One launch over several volumes: block b belongs to volume v with prefix[v] <= b <
// prefix[v+1]; len[v] is the volume's length along the pass's axis.
template <class Args>
struct LensTable {
    int nvol;
    int64_t prefix[kMaxBatch + 1];
    int len[kMaxBatch];
    Args args[kMaxBatch];
};

// calls f(std::integral_constant<int, N>{}) for the N of the list equal to n
template <int... Ns, class F>
__device__ __forceinline__ void lens_dispatch(LenList<Ns...>, int n, F &&f)
{
    (void)((n == Ns ? (f(std::integral_constant<int, Ns>{}), true) : false) || ...);
}

template <int MODE>
constexpr bool lens_x_pf()
{
    return MODE == XM_RATIO || MODE == XM_UPDATE;  // operand rows through an L2 prefetch
}

template <int N, int MODE>
constexpr size_t lens_x_smem_one()
{
    return x_smem_bytes<N, lens_threads(N), lens_lines(N), MODE, lens_x_pf<MODE>(), kLensThreads>();
}

template <int MODE, int... Ns>
constexpr size_t lens_x_smem(LenList<Ns...>)
{
    size_t m = 0;
    ((m = lens_x_smem_one<Ns, MODE>() > m ? lens_x_smem_one<Ns, MODE>() : m), ...);
    return m;
}

// shared memory of the Y / Z line tiles: B + 1 lines (the spare one last) and the stage
// twiddle table
template <int N>
constexpr size_t lens_col_smem_one()
{
    return sizeof(float2) * ((size_t)(lens_lines(N) + 1) * N + tw_table_size(N, N / lens_threads(N)));
}

template <int... Ns>
constexpr size_t lens_col_smem(LenList<Ns...>)
{
    size_t m = 0;
    ((m = lens_col_smem_one<Ns>() > m ? lens_col_smem_one<Ns>() : m), ...);
    return m;
}

// ------------------------------------------------------------------ Y: lines (z, column)

template <int N>
__device__ __forceinline__ void y_lines_body(const YArgs &a, const int64_t tile)
{
    constexpr int P = lens_threads(N), E = N / P, B = lens_lines(N), S = B + 1;
    using FFT = LineFFT<N, P, true>;
    extern __shared__ float2 smem_yl[];
    float2 *stw = smem_yl + S * N;
    const bool spare = threadIdx.x >= P * B;
    const int b = spare ? B : (int)threadIdx.x % B;
    const int t = spare ? (int)threadIdx.x - P * B : (int)threadIdx.x / B;
    // line j of the volume: plane j / xh, column j % xh (fewer than 2^31 lines)
    const unsigned xh = (unsigned)a.xh;
    const unsigned j = (unsigned)(tile * B) + (unsigned)b;
    const bool ok = !spare && j < (unsigned)a.nz * xh;
    const unsigned z = ok ? j / xh : 0u, c = ok ? j - z * xh : 0u;
    float2 *base = a.spec + (int64_t)z * N * a.xp + c;
    SmemStrided sm{smem_yl + b, S};
    auto sync = [] { __syncthreads(); };
    pdl_trigger();
    FFT::fill_twiddles(stw, a.tw, threadIdx.x, kLensThreads);
    __syncthreads();
    pdl_wait();
    float2 v[E];
    const float sgn = a.inverse ? -1.f : 1.f;
    static_for<0, E>([&](auto i_) {
        constexpr int i = CUBIC_CI(i_);
        const float2 x = ok ? base[(int64_t)(t + P * i) * a.xp] : make_float2(0.f, 0.f);
        v[i] = make_float2(x.x, sgn * x.y);
    });
    FFT::forward(v, sm, stw, t, sync);
    if (ok) {
        static_for<0, E>([&](auto i_) {
            constexpr int i = CUBIC_CI(i_);
            base[(int64_t)(t + P * i) * a.xp] = make_float2(v[i].x, sgn * v[i].y);
        });
    }
}

// ------------------------------------------------------------------ Z: lines (y, column)

// mode: ZM_CONV (times H), ZM_CORR (times conj H) or ZM_MUL_REAL (times the real H)
template <int N>
__device__ __forceinline__ void z_lines_body(const ZArgs &a, const int64_t tile, const int mode)
{
    constexpr int P = lens_threads(N), E = N / P, B = lens_lines(N), S = B + 1;
    using FFT = LineFFT<N, P, true>;
    extern __shared__ float2 smem_zl[];
    float2 *stw = smem_zl + S * N;
    const bool spare = threadIdx.x >= P * B;
    const int b = spare ? B : (int)threadIdx.x % B;
    const int t = spare ? (int)threadIdx.x - P * B : (int)threadIdx.x / B;
    // line j of the volume: row j / xh, column j % xh
    const unsigned xh = (unsigned)a.xh;
    const unsigned j = (unsigned)(tile * B) + (unsigned)b;
    const bool ok = !spare && j < (unsigned)a.ny * xh;
    const unsigned y = ok ? j / xh : 0u, c = ok ? j - y * xh : 0u;
    const int64_t zstride = a.ny * a.xp;
    const int64_t off = (int64_t)y * a.xp + c;
    float2 *base = a.spec + off;
    SmemStrided sm{smem_zl + b, S};
    auto sync = [] { __syncthreads(); };
    pdl_trigger();
    FFT::fill_twiddles(stw, a.tw, threadIdx.x, kLensThreads);
    __syncthreads();
    pdl_wait();
    float2 v[E];
    static_for<0, E>([&](auto i_) {
        constexpr int i = CUBIC_CI(i_);
        v[i] = ok ? base[(int64_t)(t + P * i) * zstride] : make_float2(0.f, 0.f);
    });
    FFT::forward(v, sm, stw, t, sync);
    if (mode == ZM_MUL_REAL) {
        const float *hb = a.Hr + off;
        static_for<0, E>([&](auto i_) {
            constexpr int i = CUBIC_CI(i_);
            const float h = ok ? __ldg(hb + (int64_t)(t + P * i) * zstride) : 0.f;
            v[i] = make_float2(v[i].x * h, -v[i].y * h);
        });
    } else {
        const bool corr = mode == ZM_CORR;
        const float2 *hb = a.H + off;
        // product with H or conj(H), then conjugate for the inverse transform
        static_for<0, E>([&](auto i_) {
            constexpr int i = CUBIC_CI(i_);
            const float2 h = ok ? __ldg(hb + (int64_t)(t + P * i) * zstride) : make_float2(0.f, 0.f);
            v[i] = cconj(corr ? cmulconj(v[i], h) : cmul(v[i], h));
        });
    }
    sync();  // the forward transform's last shared-memory reads are done
    // an opaque copy of the thread index: the second transform recomputes its exchange
    // addresses instead of keeping the first one's live through the product
    int tf = t;
    asm volatile("" : "+r"(tf));
    FFT::forward(v, sm, stw, tf, sync);
    if (ok) {
        static_for<0, E>([&](auto i_) {
            constexpr int i = CUBIC_CI(i_);
            base[(int64_t)(tf + P * i) * zstride] = cconj(v[i]);
        });
    }
}

// ------------------------------------------------------------------ kernels

template <class Args>
__device__ __forceinline__ int lens_volume(const LensTable<Args> *tab, int64_t *local)
{
    const int v = find_volume(tab->prefix, tab->nvol, blockIdx.x);
    *local = (int64_t)blockIdx.x - tab->prefix[v];
    return v;
}

// the batched path's X modes: XM_FWD, XM_RATIO, XM_UPDATE, XM_FINAL (no statistics)
template <class Lens, int MODE>
__global__ void __launch_bounds__(kLensThreads, lens_min_blocks<Lens, LK_X>()) k_xpass_lens(const LensTable<XArgs> *tab)
{
    int64_t block;
    const int v = lens_volume(tab, &block);
    const XArgs a = tab->args[v];
    lens_dispatch(Lens{}, tab->len[v], [&](auto n_) {
        constexpr int N = CUBIC_CI(n_);
        x_body<N, lens_threads(N), lens_lines(N), MODE, lens_x_pf<MODE>(), kLensThreads>(a, block);
    });
}

template <class Lens>
__global__ void __launch_bounds__(kLensThreads, lens_min_blocks<Lens, LK_Y>())
    k_ypass_lens(const LensTable<YArgs> *tab, int inverse)
{
    int64_t tile;
    const int v = lens_volume(tab, &tile);
    YArgs a = tab->args[v];
    a.inverse = inverse;
    lens_dispatch(Lens{}, tab->len[v], [&](auto n_) { y_lines_body<CUBIC_CI(n_)>(a, tile); });
}

// mode ZM_CONV or ZM_CORR; a volume with a real H multiplies by it for both
template <class Lens>
__global__ void __launch_bounds__(kLensThreads, lens_min_blocks<Lens, LK_Z>())
    k_zpass_lens(const LensTable<ZArgs> *tab, int mode)
{
    int64_t tile;
    const int v = lens_volume(tab, &tile);
    const ZArgs a = tab->args[v];
    const int m = a.Hr ? (int)ZM_MUL_REAL : mode;
    lens_dispatch(Lens{}, tab->len[v], [&](auto n_) { z_lines_body<CUBIC_CI(n_)>(a, tile, m); });
}

// ------------------------------------------------------------------ host side

// CTAs of one volume in a pass along an axis of length n: X over rows (nz * ny) in line
// pairs, Y and Z over lines (nz * xh or ny * xh)
inline int64_t lens_x_blocks(int n, int64_t rows)
{
    const int L = lens_lines(n);
    return ((rows + 1) / 2 + L - 1) / L;
}
inline int64_t lens_col_blocks(int n, int64_t lines)
{
    const int B = lens_lines(n);
    return (lines + B - 1) / B;
}

template <class... KArgs, class... Args>
inline cudaError_t lens_launch(void (*fn)(KArgs...), size_t smem, int64_t blocks, cudaStream_t st, Args &&...args)
{
    static_assert(sizeof...(KArgs) == sizeof...(Args), "kernel arguments");
    cudaError_t e = set_smem((const void *)fn, smem);
    if (e != cudaSuccess) return e;
    if (blocks == 0) return cudaSuccess;
    return launch_pdl(fn, dim3((unsigned)blocks), dim3(kLensThreads), smem, st, std::forward<Args>(args)...);
}

// calls f(the class's LenList{}) for class c
template <class F>
inline cudaError_t lens_for_class(int c, F &&f)
{
    switch (c) {
    case 0: return f(LensLight{});
    case 1: return f(LensMedium{});
    case 2: return f(LensWide{});
    default: return cudaErrorInvalidValue;
    }
}

// Launchers of class c; blocks = prefix[nvol] of the table.  X: one mode per translation
// unit (lens_x_*.cu); Y and Z in lens_y.cu and lens_z.cu.
template <int MODE>
cudaError_t launch_x_lens_mode(int c, const LensTable<XArgs> *tab, int64_t blocks, cudaStream_t st);

cudaError_t launch_x_lens(int c, int mode, const LensTable<XArgs> *tab, int64_t blocks, cudaStream_t st);
cudaError_t launch_y_lens(int c, const LensTable<YArgs> *tab, int64_t blocks, int inverse, cudaStream_t st);
cudaError_t launch_z_lens(int c, const LensTable<ZArgs> *tab, int64_t blocks, int mode, cudaStream_t st);

#define CUBIC_LENS_X_UNIT(MODE)                                                                              \
    template <>                                                                                              \
    cudaError_t launch_x_lens_mode<MODE>(int c, const LensTable<XArgs> *tab, int64_t blocks, cudaStream_t st) \
    {                                                                                                        \
        return lens_for_class(c, [&](auto lens) {                                                            \
            return lens_launch(k_xpass_lens<decltype(lens), MODE>, lens_x_smem<MODE>(lens), blocks, st, tab);  \
        });                                                                                                  \
    }

}  // namespace cubic
