// colpass_tma.cuh -- persistent, TMA-pipelined Y and Z passes.
//
// A tile is B adjacent spectrum columns x one full line (N elements) along y
// (Y pass, lines at stride xp) or along z (Z pass, lines at stride ny*xp).  A
// persistent CTA walks its tiles with two shared-memory stages: while tile i
// is being transformed, the TMA engine loads tile i+1 into the other stage and
// stores tile i-1 back to HBM.  Tiles move as 3D tensor boxes over the
// spectrum viewed as float32 [nz][ny][2*xp] (box {2B, rows, 1} for Y,
// {2B, 1, rows} for Z), so they land in shared memory as [line position][column],
// which is also the layout the line FFT exchanges through.
//
// The Z pass multiplies by H (forward convolution) or conj(H) (correlation
// with the PSF, i.e. convolution with the flipped PSF) between its forward and
// inverse transforms; the H tile rides on the same mbarrier as the data tile.
#pragma once

#include <cuda.h>

#include "passes.cuh"

namespace cubic {

enum ColKind : int { COL_Y = 0, COL_Z = 1 };

struct ColArgs {
    const float2 *tw;
    int64_t ntiles_col;  // column tiles per plane / row
    int64_t ntiles;      // total tiles
    int64_t col_tile0;   // first column tile of this launch
    int mode;            // Y: 0 forward, 1 inverse.  Z: a ZMode
    float scale;         // ZM_FWD_SCALE / ZM_INV_SCALE
    unsigned *err;
    int nstore;          // line rows stored (boxes starting at or past it are skipped); N: all
    unsigned long long wait_ns;  // limit of the tile waits (0: kWaitNs)
    // failure-path test: CTA 0 does not issue the copy of its first tile, so its first
    // wait runs out (nothing is left in flight: that copy never starts)
    int skip_first;
};

// largest divisor of n that is <= 256 (TMA box extent limit)
constexpr int box_rows(int n)
{
    for (int d = n < 256 ? n : 256; d > 1; --d)
        if (n % d == 0) return d;
    return 1;
}

__device__ __forceinline__ void tma_load_3d(void *smem_dst, const CUtensorMap *tm, int c0, int c1, int c2,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(smem_dst)),
        "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap *tm, int c0, int c1, int c2, const void *smem_src)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(tm),
                 "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(smem_src))
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void bulk_wait_read()  // at most K store groups still reading shared memory
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(K) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Exchange layout inside a stage: element pos of column b at base[(pos + pad(pos)) * S + b],
// pad(pos) = pos / R0 for an even first-stage radix R0 (one spare row every R0 rows, so
// the first stage's scattered writes j*R0 + r of the tile's different lines fall in
// different banks), 0 for an odd one.  Tiles arrive and leave unpadded; the exchanges
// only run after the tile's canonical reads and before its canonical writes.
template <int S, int R0>
struct SmemStridedT {
    float2 *base;
    __device__ __forceinline__ float2 &at(int pos) const { return base[(pos + ((R0 % 2 == 0) ? pos / R0 : 0)) * S]; }
};

template <int N, int P>
constexpr int col_pad_rows()
{
    constexpr int R0 = N == 1 ? 1 : plan_radix(N, N / P, 0);
    return (R0 % 2 == 0) ? N / R0 : 0;
}

// one stage holds a tile plus the exchange padding; rounded up to 1 KB so that every
// stage (and every box inside it, whose offsets are multiples of R*B*8 bytes) starts
// on the alignment tensor copies need
template <int N, int B, int P = N>
constexpr size_t col_stage_bytes()
{
    return ((size_t)(N + col_pad_rows<N, P>()) * B * sizeof(float2) + 1023) / 1024 * 1024;
}

template <int N, int B>
constexpr size_t col_tile_bytes()
{
    return (size_t)N * B * sizeof(float2);
}

// H stage of the Z pass: a complex tile, or half of it for a real H (HREAL)
template <int N, int B, int P, bool HREAL>
constexpr size_t col_hstage_bytes()
{
    return HREAL ? ((size_t)N * B * sizeof(float) + 1023) / 1024 * 1024 : col_stage_bytes<N, B, P>();
}

template <int N, int P, int B, int KIND, int NS = 2, bool HREAL = false>
constexpr size_t col_smem_bytes()
{
    // 1 KB for the barriers (keeps the stages 1 KB aligned), NS data stages,
    // NS H stages for the Z pass, then the stage twiddle table
    return 1024 + NS * (col_stage_bytes<N, B, P>() + (KIND == COL_Z ? col_hstage_bytes<N, B, P, HREAL>() : 0)) +
           (size_t)tw_table_size(N, N / P) * sizeof(float2);
}

// NS shared-memory stages; tiles are prefetched D = max(1, NS - 2) ahead, so up to
// NS - D - 1 tile stores may still be draining when a stage is refilled.
template <int N, int P, int B, int KIND, int NS = 2, bool HREAL = false>
__global__ void __launch_bounds__(P *B) k_colpass_tma(const __grid_constant__ CUtensorMap tm_spec,
                                                      const __grid_constant__ CUtensorMap tm_h, ColArgs a)
{
    static_assert(NS >= 2 && NS <= 8, "stages");
    constexpr int D = NS - 2 > 1 ? NS - 2 : 1;
    constexpr int KW = NS - D - 1;  // store groups allowed in flight at a refill
    constexpr int E = N / P;
    constexpr int R = box_rows(N);
    constexpr int NB = N / R;  // boxes per tile
    constexpr size_t SB = col_stage_bytes<N, B, P>();
    extern __shared__ __align__(1024) unsigned char smem_col[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_col);  // full[0 .. NS)
    constexpr size_t HB = col_hstage_bytes<N, B, P, HREAL>();
    auto stage = [&](int s) { return reinterpret_cast<float2 *>(smem_col + 1024 + (size_t)s * SB); };
    auto hstage = [&](int s) {
        return reinterpret_cast<float2 *>(smem_col + 1024 + (size_t)NS * SB + (size_t)s * HB);
    };
    // a real H needs the HREAL instantiation (its H stages are half size)
    const bool realH = HREAL && (KIND == COL_Z) && a.mode == ZM_MUL_REAL;
    const bool needH = (KIND == COL_Z) && (HREAL ? realH : (a.mode == ZM_CONV || a.mode == ZM_CORR));
    const unsigned tile_bytes = (unsigned)(col_tile_bytes<N, B>() * (needH ? (realH ? 3 : 4) : 2) / 2);
    using FFT = LineFFT<N, P, true>;
    float2 *stw = reinterpret_cast<float2 *>(smem_col + 1024 + (size_t)NS * (SB + (KIND == COL_Z ? HB : 0)));

    const int b = threadIdx.x % B;
    const int t = threadIdx.x / B;
    auto sync = [] { __syncthreads(); };
    pdl_trigger();
    FFT::fill_twiddles(stw, a.tw, threadIdx.x, P * B);  // plan constant: before the wait

    // tile -> tensor coordinates of its first box
    auto coords = [&](int64_t tile, int &cx, int &o) {
        const int64_t ct = a.col_tile0 + tile % a.ntiles_col;
        o = (int)(tile / a.ntiles_col);  // z for Y, y for Z
        cx = (int)(ct * B * 2);
    };
    auto issue = [&](int64_t tile, int s) {
        int cx, o;
        coords(tile, cx, o);
        mbar_arrive_expect_tx(&full[s], tile_bytes);
        for (int j = 0; j < NB; ++j) {
            float2 *dst = stage(s) + (size_t)j * R * B;
            if (KIND == COL_Y)
                tma_load_3d(dst, &tm_spec, cx, j * R, o, &full[s]);
            else
                tma_load_3d(dst, &tm_spec, cx, o, j * R, &full[s]);
            if (needH) {
                // real H: float boxes of B columns (x in floats = cx / 2), packed half-size
                if (realH)
                    tma_load_3d(reinterpret_cast<float *>(hstage(s)) + (size_t)j * R * B, &tm_h, cx / 2, o, j * R,
                                &full[s]);
                else
                    tma_load_3d(hstage(s) + (size_t)j * R * B, &tm_h, cx, o, j * R, &full[s]);
            }
        }
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    pdl_wait();  // the previous pass's output is complete from here on
    const int64_t first = blockIdx.x, step = gridDim.x;
    if (threadIdx.x == 0)
        for (int i = 0; i < D; ++i)
            if (first + i * step < a.ntiles && !(i == 0 && a.skip_first && blockIdx.x == 0))
                issue(first + i * step, i % NS);

    int it = 0;
    for (int64_t tile = first; tile < a.ntiles; tile += step, ++it) {
        const int s = it % NS;
        const unsigned phase = (unsigned)((it / NS) & 1);
        const int64_t ahead = tile + (int64_t)D * step;
        if (threadIdx.x == 0 && ahead < a.ntiles) {
            bulk_wait_read<KW>();  // the stage being refilled has left shared memory
            issue(ahead, (it + D) % NS);
        }
        const bool arrived = mbar_wait_bounded(&full[s], phase, a.err, a.wait_ns);
        if (!__syncthreads_and(arrived)) {
            // give already issued loads a bounded chance (the default limit, not the
            // launch's) to land before leaving
            if (threadIdx.x == 0)
                for (int i = 1; i <= D; ++i)
                    if (tile + (int64_t)i * step < a.ntiles)
                        mbar_wait_bounded(&full[(it + i) % NS], (unsigned)(((it + i) / NS) & 1), a.err);
            break;
        }

        float2 *buf = stage(s);
        SmemStridedT<B, (N == 1 ? 1 : plan_radix(N, N / P, 0))> sm{buf + b};
        float2 v[E];
        const bool conj_in = (KIND == COL_Y) ? a.mode == 1 : a.mode == ZM_INV_SCALE;
        static_for<0, E>([&](auto i_) {
            constexpr int i = CUBIC_CI(i_);
            const float2 x = buf[(t + P * i) * B + b];
            v[i] = conj_in ? cconj(x) : x;
        });
        __syncthreads();  // every canonical read is done before the exchanges reuse the stage
        FFT::forward(v, sm, stw, t, sync);
        if (KIND == COL_Z && needH) {
            if (realH) {
                const float *hb = reinterpret_cast<const float *>(hstage(s));
                static_for<0, E>([&](auto i_) {
                    constexpr int i = CUBIC_CI(i_);
                    const float h = hb[(t + P * i) * B + b];
                    v[i] = make_float2(v[i].x * h, -v[i].y * h);
                });
            } else {
                const float2 *hb = hstage(s);
                const bool corr = a.mode == ZM_CORR;
                static_for<0, E>([&](auto i_) {
                    constexpr int i = CUBIC_CI(i_);
                    const float2 h = hb[(t + P * i) * B + b];
                    v[i] = cconj(corr ? cmulconj(v[i], h) : cmul(v[i], h));
                });
            }
            FFT::forward(v, sm, stw, t, sync);
            static_for<0, E>([&](auto i_) { v[CUBIC_CI(i_)] = cconj(v[CUBIC_CI(i_)]); });
        } else if (KIND == COL_Z) {
            const float sc = a.scale, sy = conj_in ? -a.scale : a.scale;
            static_for<0, E>([&](auto i_) {
                constexpr int i = CUBIC_CI(i_);
                v[i] = make_float2(v[i].x * sc, v[i].y * sy);
            });
        } else if (conj_in) {
            static_for<0, E>([&](auto i_) { v[CUBIC_CI(i_)] = cconj(v[CUBIC_CI(i_)]); });
        }
        // canonical positions are owned by this thread: no barrier needed before writing
        static_for<0, E>([&](auto i_) {
            constexpr int i = CUBIC_CI(i_);
            buf[(t + P * i) * B + b] = v[i];
        });
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            int cx, o;
            coords(tile, cx, o);
            // the Y pass stores through its own map (tm_h, unused for H there), whose
            // extent can stop short of the loads'; boxes past it are not issued and the
            // tensor map clips the one that straddles it
            for (int j = 0; j < NB && j * R < a.nstore; ++j) {
                const float2 *src = buf + (size_t)j * R * B;
                if (KIND == COL_Y)
                    tma_store_3d(&tm_h, cx, j * R, o, src);
                else
                    tma_store_3d(&tm_spec, cx, o, j * R, src);
            }
            bulk_commit();
        }
    }
    if (threadIdx.x == 0) bulk_wait_all();
}

}  // namespace cubic
