// passes.cuh -- the three axis passes of the 3D real FFT convolution, with the
// Richardson-Lucy pointwise steps fused into them.
//
// Data layout in HBM (all C-order, x fastest):
//   real volumes   float  [nz][ny][nx]
//   spectrum       float2 [nz][ny][xp]   xp >= nx/2+1, columns >= nx/2+1 unused
//   PSF spectrum H float2 [nz][ny][xp]   same layout, already scaled by 1/V
//
// X pass  -- one CTA row-group owns complete x-lines.  Two real rows (2m, 2m+1)
//            are packed as one complex line z = row0 + i row1; one complex FFT
//            of length nx then gives both half spectra:
//              A[k] = (Z[k] + conj Z[N-k]) / 2,  B[k] = (Z[k] - conj Z[N-k]) / (2i).
//            The inverse packs Z[k] = A[k] + i B[k] (using A[N-k] = conj A[k]).
//            The pointwise Richardson-Lucy steps run between the inverse and
//            the forward transform of the same line (Section 4 of the paper:
//            ratio with the observed image, multiplicative update).
// Y pass  -- a CTA owns B adjacent spectrum columns x full y-lines (strided by xp).
// Z pass  -- a CTA owns B adjacent columns x full z-lines; forward z FFT,
//            pointwise product with H (forward convolution) or conj(H)
//            (correlation = convolution with the flipped PSF), inverse z FFT.
#pragma once

#include "csum.cuh"
#include "fft_core.cuh"
#include "tma.cuh"

namespace cubic {

enum XMode : int {
    XM_FWD = 0,     // real rows (src)            -> spectrum
    XM_INV = 1,     // spectrum                   -> real rows (dst)
    XM_RATIO = 2,   // spectrum -> b; r = d / max(b, eps)      -> spectrum of r
    XM_UPDATE = 3,  // spectrum -> q; u = u * q (stored)       -> spectrum of u
    XM_FINAL = 4,   // spectrum -> q; out = u * q
    XM_COUNT = 5,
    // the adjoint passes of the differentiable path (one launch shape per length)
    XM_ADJ_R = 5,   // spectrum -> rbar; dbar += rbar / c; bbar -> spectrum
    XM_ADJ_U = 6    // [spectrum -> t]; g = w + t; qbar = g u -> spectrum, w = g q (or w = g)
};

struct XArgs {
    const float2 *spec_in;
    float2 *spec_out;
    const float *src;  // XM_FWD input rows
    float *dst;        // XM_INV output rows, XM_FINAL output
    float *u;          // estimate (XM_UPDATE read/write, XM_FINAL read)
    const float *d;    // observed image (XM_RATIO)
    const float2 *tw;  // twiddles of length nx
    int64_t rows;      // nz * ny
    int64_t xp;        // spectrum pitch (complex elements)
    float eps;
    unsigned *err;     // device error word (bounded waits)
    unsigned long long wait_ns;  // limit of the bounded waits (0: kWaitNs)
    // optional copies of intermediates (null: not stored), used by the gradient's
    // recomputation: XM_RATIO stores b (keep_a) and r (keep_b); XM_UPDATE / XM_FINAL
    // store q (keep_a)
    float *keep_a;
    float *keep_b;
    // optional (XM_UPDATE / XM_FINAL): adds sum((u_new - u)^2) into the compensated
    // pair stats[4 s], stats[4 s + 1] (value = hi + lo) and sum(u^2) into stats[4 s + 2],
    // stats[4 s + 3]; s is one of 64 slots (spread to avoid contention)
    float *stats;
    // optional, accelerated RL (null: the plain pass):
    //  XM_FWD with acc_prev: the rows transformed are the prediction
    //    y = max(src + alpha (src - acc_prev), 0), alpha = *acc_alpha, also stored to acc_y;
    //  XM_FINAL with acc_g: g = out - u is stored to acc_g, and the CTA's compensated sums
    //    of g * acc_gprev (0 where acc_gprev is null) and of g * g go to acc_part[block]
    //    as (num.s, num.c, den.s, den.c), value = s - c.
    const float *acc_prev;
    const float *acc_alpha;
    float *acc_y;
    float *acc_g;
    const float *acc_gprev;
    float4 *acc_part;
    // optional (XM_RATIO): adds the Poisson negative log-likelihood sum(c - d ln c),
    // c = max(b, eps), into the compensated pair nll_stats[2 s], nll_stats[2 s + 1]
    // (value = hi + lo), s = one of 64 slots
    float *nll_stats;
    // linear-boundary plans (0: none): image row r = z * ny_img + y is spectrum row
    // z * ny_spec + y (the spectrum's planes have ny_spec >= ny_img rows)
    int64_t ny_img, ny_spec;
    // the adjoint passes (XM_ADJ_*): adj_b the blur b and adj_dbar the image gradient
    // (read-modify-write) of XM_ADJ_R; XM_ADJ_U: adj_w the running gradient of the iterate
    // (read-modify-write), adj_u and adj_q the iterate u and the correlation q of the
    // iteration whose qbar it transforms (null: it only stores g), spec_in null: no inverse
    // transform (t = 0)
    const float *adj_u, *adj_q, *adj_b;
    float *adj_w, *adj_dbar;
};

struct YArgs {
    float2 *spec;
    const float2 *tw;
    int64_t nz;
    int64_t xh;    // nx/2 + 1 valid columns
    int64_t xp;
    int inverse;
    int64_t col0;  // first column of this launch (multiple of the tile width)
    int64_t col1;  // one past the last column (<= xh)
    unsigned *err;
    // linear-boundary plans: rows of each line that are loaded (the rest reads as zero)
    // and stored; 0: all N
    int64_t nload, nstore;
    unsigned long long wait_ns;  // TMA variants: limit of the tile waits (0: kWaitNs)
    int skip_first;              // TMA variants: the failure-path test of ColArgs
};

// ZM_MUL_REAL: product with a real H (point-symmetric PSF), where convolution and
// correlation coincide
enum ZMode : int { ZM_FWD_SCALE = 0, ZM_CONV = 1, ZM_CORR = 2, ZM_INV_SCALE = 3, ZM_MUL_REAL = 4 };

struct ZArgs {
    float2 *spec;
    const float2 *H;
    const float2 *tw;
    int64_t ny;
    int64_t xh;
    int64_t xp;
    int mode;
    float scale;   // ZM_FWD_SCALE / ZM_INV_SCALE only
    int64_t col0;  // column range of this launch, as in YArgs
    int64_t col1;
    unsigned *err;
    int64_t nz;    // lines are this long (TMA path builds its tensor map from it)
    const float *Hr;  // real H, float [nz][ny][xp] (ZM_MUL_REAL)
    // linear-boundary plans: planes of the spectrum array that are loaded (the rest of each
    // line reads as zero) and stored; H keeps all N planes.  0: all N
    int64_t nload, nstore;
    // optional, the product modes of the plain Z kernel (the reverse sweep of the
    // differentiable path): save receives the z-transformed lines before the product with H;
    // gacc accumulates conj(V) gother (gconj != 0) or V conj(gother) (gconj = 0), V the
    // z-transformed lines, all in the spectrum array's layout
    float2 *save;
    float2 *gacc;
    const float2 *gother;
    int gconj;
    unsigned long long wait_ns;  // TMA variants: limit of the tile waits (0: kWaitNs)
    int skip_first;              // TMA variants: the failure-path test of ColArgs
};

// ------------------------------------------------------------------ X pass

// Element pos at base[pos + pos / R0] for an even first-stage radix R0 (its scattered
// writes j*R0 + r then spread over all banks), at base[pos] for an odd one (j*R0 + r is
// already conflict-free).
template <int R0>
struct SmemPadded {
    float2 *base;
    __device__ __forceinline__ float2 &at(int pos) const { return base[(R0 % 2 == 0) ? pos + pos / R0 : pos]; }
};

struct SmemStrided {  // element pos at base[pos * stride]
    float2 *base;
    int stride;
    __device__ __forceinline__ float2 &at(int pos) const { return base[pos * stride]; }
};

template <int N, int P>
constexpr int x_first_radix() { return N == 1 ? 1 : plan_radix(N, N / P, 0); }

// even number of complex elements >= nx/2+1: one spectrum row in a 16-byte multiple
template <int N>
constexpr int x_row_xb() { return ((N / 2 + 1) + 1) / 2 * 2; }

// float2 slots per line pair: the padded exchange line, which also receives the
// pair's two spectrum rows (2 * xb) at the start of the inverse passes
template <int N, int P>
constexpr int x_smem_line()
{
    constexpr int R0 = x_first_radix<N, P>();
    constexpr int ex = N + ((R0 % 2 == 0) ? N / R0 : 0) + 1;
    constexpr int sp = 2 * x_row_xb<N>();
    return ((ex > sp ? ex : sp) + 1) / 2 * 2;
}

// The pointwise operand rows (d for the ratio, u for the update) are staged
// into shared memory by one bulk TMA copy per CTA issued at kernel start, so
// their HBM latency hides behind the inverse transform.  Needs 16-byte rows.
// With PF (ratio and update only) they are instead prefetched into L2 at kernel
// start and read from global memory: 2 N floats less shared memory per line pair,
// so more CTAs fit on an SM.
template <int N, int MODE, bool PF = false>
constexpr bool x_prefetches()
{
    return PF && (MODE == XM_RATIO || MODE == XM_UPDATE) && (N % 4 == 0);
}

template <int N, int MODE, bool PF = false>
constexpr bool x_uses_tma()
{
    return (MODE == XM_RATIO || MODE == XM_UPDATE || MODE == XM_FINAL) && (N % 4 == 0) &&
           !x_prefetches<N, MODE, PF>();
}

// shared memory: [2 mbarriers | operand rows (TMA modes) | stage twiddles | line-pair regions]
// T: threads of the CTA.  Where T > P * L the threads past the L line pairs share one
// spare line-pair region (they transform garbage there and touch no global memory).
template <int N, int P, int L, int MODE, bool PF = false, int T = P * L>
constexpr size_t x_smem_bytes()
{
    return 16 + (x_uses_tma<N, MODE, PF>() ? (size_t)L * 2 * N * sizeof(float) : 0) +
           (size_t)((tw_table_size(N, N / P) + 1) / 2 * 2) * sizeof(float2) +
           (size_t)(L + (T > P * L ? 1 : 0)) * x_smem_line<N, P>() * sizeof(float2);
}

// Merges two compensated sums over the T threads of the CTA, in a fixed order
// (deterministic); thread 0 receives (a.s, a.c, b.s, b.c).  Every thread must call it.
template <int T>
__device__ __forceinline__ float4 block_merge2(CFloat a, CFloat b)
{
    __shared__ CFloat red[2][T % 32 == 0 ? T / 32 : T];
    if constexpr (T % 32 == 0) {
        // full warps: shuffle tree, then the warps' results in order
        for (int o = 16; o > 0; o >>= 1) {
            a = cf_merge(a, CFloat{__shfl_down_sync(0xffffffffu, a.s, o), __shfl_down_sync(0xffffffffu, a.c, o)});
            b = cf_merge(b, CFloat{__shfl_down_sync(0xffffffffu, b.s, o), __shfl_down_sync(0xffffffffu, b.c, o)});
        }
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = a;
            red[1][threadIdx.x >> 5] = b;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < T / 32; ++w) {
                a = cf_merge(a, red[0][w]);
                b = cf_merge(b, red[1][w]);
            }
        }
    } else {
        // other widths: pairwise tree in shared memory
        red[0][threadIdx.x] = a;
        red[1][threadIdx.x] = b;
        __syncthreads();
        for (int s = 1; s < T; s *= 2) {
            if (threadIdx.x % (2 * s) == 0 && threadIdx.x + s < T) {
                red[0][threadIdx.x] = cf_merge(red[0][threadIdx.x], red[0][threadIdx.x + s]);
                red[1][threadIdx.x] = cf_merge(red[1][threadIdx.x], red[1][threadIdx.x + s]);
            }
            __syncthreads();
        }
        a = red[0][0];
        b = red[1][0];
    }
    return make_float4(a.s, a.c, b.s, b.c);
}

// Adds each thread's compensated sum v into the pair (hi, lo) at pair[0], pair[1] of
// a slot: a shuffle reduction where the warp is full (T threads in the CTA), else one
// add per thread.
template <int T>
__device__ __forceinline__ void slot_add(float *pair, CFloat v)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if ((warp + 1) * 32 <= T) {
        for (int o = 16; o > 0; o >>= 1)
            v = cf_merge(v, CFloat{__shfl_down_sync(0xffffffffu, v.s, o), __shfl_down_sync(0xffffffffu, v.c, o)});
        if (lane != 0) return;
    }
    catomic_add(pair, pair + 1, v.s);
    catomic_add(pair, pair + 1, -v.c);
}

// T: threads of the CTA, P * L or more (the extra threads idle through the transforms on
// a spare line-pair region, so that every thread meets every barrier)
template <int N, int P, int L, int MODE, bool PF, int T = P * L>
__device__ __forceinline__ void x_body(const XArgs &a, const int64_t block)
{
    static_assert(T >= P * L && T < P * (L + 1), "a CTA of T threads holds L line pairs");
    constexpr int E = N / P;
    constexpr bool kTma = x_uses_tma<N, MODE, PF>();
    constexpr bool kPf = x_prefetches<N, MODE, PF>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using FFT = LineFFT<N, P, true>;
    constexpr int XB = x_row_xb<N>();
    constexpr bool kSpecIn = MODE != XM_FWD;  // the pair's spectrum rows arrive by TMA
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);  // [0] operand rows, [1] spectrum rows
    float *oprows = reinterpret_cast<float *>(smem_raw + 16);
    float2 *stw = reinterpret_cast<float2 *>(smem_raw + 16 + (kTma ? (size_t)L * 2 * N * sizeof(float) : 0));
    float2 *xch = stw + (FFT::kTwSize + 1) / 2 * 2;  // 16-byte aligned: bulk-copy destination

    const int t = threadIdx.x % P;
    const int l = threadIdx.x / P;
    const int64_t m = block * L + l;
    const int64_t r0 = 2 * m, r1 = 2 * m + 1;
    const bool live = T == P * L || l < L;
    const bool ok0 = live && r0 < a.rows, ok1 = live && r1 < a.rows;
    // image row -> spectrum row (row indices stay below 2^32: nz, ny <= 65535)
    auto srow = [&](int64_t r) -> int64_t {
        if (a.ny_img <= 0) return r;
        const unsigned q = (unsigned)r / (unsigned)a.ny_img;
        return (int64_t)q * a.ny_spec + ((unsigned)r - q * (unsigned)a.ny_img);
    };
    float2 *lpair = xch + l * x_smem_line<N, P>();
    SmemPadded<x_first_radix<N, P>()> sm{lpair};
    auto sync = [] { __syncthreads(); };

    pdl_trigger();
    if constexpr (kPf) {
        if (threadIdx.x == 0) {
            // a hint only, so it may run before the wait: the loads below come after it
            const int64_t row0 = block * L * 2;
            const int64_t left = a.rows - row0;
            const int64_t nrows = left < 2 * L ? left : 2 * L;
            bulk_prefetch_l2((MODE == XM_RATIO ? a.d : a.u) + row0 * N, (unsigned)(nrows * N * sizeof(float)));
        }
    }
    FFT::fill_twiddles(stw, a.tw, threadIdx.x, T);  // plan constant: before the wait
    if constexpr (kTma || kSpecIn) {
        if (threadIdx.x == 0) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            mbar_fence_init();
        }
    }
    __syncthreads();
    pdl_wait();  // the previous pass's output is complete from here on
    // XM_ADJ_U without a spectrum (the first adjoint step of a segment) has no inverse part
    const bool have_spec = MODE != XM_ADJ_U || a.spec_in != nullptr;
    if constexpr (kSpecIn) {
        if (threadIdx.x == 0 && have_spec) {
            // the CTA's spectrum rows, one bulk copy each, into the line-pair regions
            const int64_t row0 = block * L * 2;
            const int64_t left = a.rows - row0;
            const int nr = (int)(left < 2 * L ? left : 2 * L);
            mbar_arrive_expect_tx(&bar[1], (unsigned)(nr * XB * sizeof(float2)));
            for (int r = 0; r < nr; ++r)
                bulk_g2s(xch + (r >> 1) * x_smem_line<N, P>() + (r & 1) * XB, a.spec_in + srow(row0 + r) * a.xp,
                         (unsigned)(XB * sizeof(float2)), &bar[1]);
        }
    }
    if constexpr (kTma) {
        if (threadIdx.x == 0) {
            // this CTA's rows are contiguous: one copy
            const int64_t row0 = block * L * 2;
            const int64_t left = a.rows - row0;
            const int64_t nrows = left < 2 * L ? left : 2 * L;
            const float *src = (MODE == XM_RATIO ? a.d : a.u) + row0 * N;
            const unsigned bytes = (unsigned)(nrows * N * sizeof(float));
            mbar_arrive_expect_tx(&bar[0], bytes);
            bulk_g2s(oprows, src, bytes, &bar[0]);
        }
    }

    float2 v[E];
    if constexpr (MODE == XM_FWD) {
        const float *s0 = a.src + r0 * N, *s1 = a.src + r1 * N;
        if (a.acc_prev) {
            // accelerated RL: extrapolate along the last move, clamp at 0, keep y
            const float al = *a.acc_alpha;
            const float *p0 = a.acc_prev + r0 * N, *p1 = a.acc_prev + r1 * N;
            float *y0 = a.acc_y + r0 * N, *y1 = a.acc_y + r1 * N;
            // every load before the first store, so none waits behind a store it might alias
            static_for<0, E>([&](auto i_) {
                constexpr int i = CUBIC_CI(i_);
                const int n = t + P * i;
                const float x0 = ok0 ? __ldg(s0 + n) : 0.f, x1 = ok1 ? __ldg(s1 + n) : 0.f;
                const float q0 = ok0 ? __ldg(p0 + n) : 0.f, q1 = ok1 ? __ldg(p1 + n) : 0.f;
                v[i] = make_float2(fmaxf(fmaf(al, x0 - q0, x0), 0.f), fmaxf(fmaf(al, x1 - q1, x1), 0.f));
            });
            static_for<0, E>([&](auto i_) {
                constexpr int i = CUBIC_CI(i_);
                const int n = t + P * i;
                if (ok0) y0[n] = v[i].x;
                if (ok1) y1[n] = v[i].y;
            });
        } else {
            static_for<0, E>([&](auto i_) {
                constexpr int i = CUBIC_CI(i_);
                const int n = t + P * i;
                v[i] = make_float2(ok0 ? __ldg(s0 + n) : 0.f, ok1 ? __ldg(s1 + n) : 0.f);
            });
        }
    } else {
        if (!have_spec) {  // uniform over the launch
            static_for<0, E>([&](auto i_) { v[CUBIC_CI(i_)] = make_float2(0.f, 0.f); });
        } else {
            const bool landed = mbar_wait_bounded(&bar[1], 0, a.err, a.wait_ns);
            if (!__syncthreads_and(landed)) return;
            const float2 *q0 = lpair, *q1 = lpair + XB;
            static_for<0, E>([&](auto i_) {
                constexpr int i = CUBIC_CI(i_);
                const int k = t + P * i;
                const bool hi = 2 * k > N;
                const int kk = hi ? N - k : k;
                float2 A = ok0 ? q0[kk] : make_float2(0.f, 0.f);
                float2 B = ok1 ? q1[kk] : make_float2(0.f, 0.f);
                if (hi) {
                    A.y = -A.y;
                    B.y = -B.y;
                }
                if (k == 0 || 2 * k == N) {  // self-conjugate bins of a real line
                    A.y = 0.f;
                    B.y = 0.f;
                }
                v[i] = make_float2(A.x - B.y, A.y + B.x);  // A + i B
            });
            __syncthreads();  // the rows are read before the exchanges overwrite the region
            FFT::inverse(v, sm, stw, t, sync);
        }

        // operand rows: shared memory (TMA) or global
        const float *p0, *p1;
        if constexpr (kTma) {
            const bool arrived = mbar_wait_bounded(&bar[0], 0, a.err, a.wait_ns);
            if (!__syncthreads_and(arrived)) return;
            p0 = oprows + (2 * l) * N;
            p1 = oprows + (2 * l + 1) * N;
        } else {
            const float *g = (MODE == XM_RATIO) ? a.d : a.u;
            p0 = g + r0 * N;
            p1 = g + r1 * N;
        }

        // pointwise step on the real rows (v.x = row r0, v.y = row r1)
        if constexpr (MODE == XM_INV) {
            float *o0 = a.dst + r0 * N, *o1 = a.dst + r1 * N;
            static_for<0, E>([&](auto i_) {
                constexpr int i = CUBIC_CI(i_);
                const int n = t + P * i;
                if (ok0) o0[n] = v[i].x;
                if (ok1) o1[n] = v[i].y;
            });
        } else if constexpr (MODE == XM_ADJ_R) {
            // rbar = v: dbar += rbar / c and bbar = -rbar d / c^2 where b > eps (the clamp's
            // derivative is 0 below it), c = max(b, eps); bbar is transformed
            const float eps = a.eps;
            const float *bb0 = a.adj_b + r0 * N, *bb1 = a.adj_b + r1 * N;
            const float *d0 = a.d + r0 * N, *d1 = a.d + r1 * N;
            float *e0 = a.adj_dbar + r0 * N, *e1 = a.adj_dbar + r1 * N;
            static_for<0, E>([&](auto i_) {
                constexpr int i = CUBIC_CI(i_);
                const int n = t + P * i;
                const float b0v = ok0 ? __ldg(bb0 + n) : 0.f, b1v = ok1 ? __ldg(bb1 + n) : 0.f;
                const float c0 = fmaxf(b0v, eps), c1 = fmaxf(b1v, eps);
                const float r0v = v[i].x, r1v = v[i].y;
                if (ok0) e0[n] += r0v / c0;
                if (ok1) e1[n] += r1v / c1;
                v[i] = make_float2(b0v > eps ? -r0v * (ok0 ? __ldg(d0 + n) : 0.f) / (c0 * c0) : 0.f,
                                   b1v > eps ? -r1v * (ok1 ? __ldg(d1 + n) : 0.f) / (c1 * c1) : 0.f);
            });
        } else if constexpr (MODE == XM_ADJ_U) {
            // g = w + v, the gradient of the iterate (v = 0 without a spectrum); then either
            // qbar = g u (transformed) and w = g q, the running gradient of the iteration
            // before, or w = g.  One kernel serves every step of a segment, so that the
            // arithmetic does not depend on where the checkpoints fall.
            float *w0 = a.adj_w + r0 * N, *w1 = a.adj_w + r1 * N;
            if (a.adj_u) {  // uniform over the launch
                const float *u0 = a.adj_u + r0 * N, *u1 = a.adj_u + r1 * N;
                const float *q0 = a.adj_q + r0 * N, *q1 = a.adj_q + r1 * N;
                static_for<0, E>([&](auto i_) {
                    constexpr int i = CUBIC_CI(i_);
                    const int n = t + P * i;
                    const float x0 = v[i].x + (ok0 ? w0[n] : 0.f), x1 = v[i].y + (ok1 ? w1[n] : 0.f);
                    v[i] = make_float2(x0 * (ok0 ? __ldg(u0 + n) : 0.f), x1 * (ok1 ? __ldg(u1 + n) : 0.f));
                    if (ok0) w0[n] = x0 * __ldg(q0 + n);
                    if (ok1) w1[n] = x1 * __ldg(q1 + n);
                });
            } else {
                static_for<0, E>([&](auto i_) {
                    constexpr int i = CUBIC_CI(i_);
                    const int n = t + P * i;
                    if (ok0) w0[n] += v[i].x;
                    if (ok1) w1[n] += v[i].y;
                });
                return;  // uniform over the launch: no forward transform
            }
        } else if constexpr (MODE == XM_RATIO) {
            const float eps = a.eps;
            float *kb0 = a.keep_a + r0 * N, *kb1 = a.keep_a + r1 * N;
            float *kr0 = a.keep_b + r0 * N, *kr1 = a.keep_b + r1 * N;
            const bool keep = a.keep_a != nullptr;
            if (a.nll_stats) {
                // the likelihood of b, in a loop of its own so that the ratio loop below
                // keeps its schedule when it is off
                CFloat c_nll{0.f, 0.f};
                static_for<0, E>([&](auto i_) {
                    constexpr int i = CUBIC_CI(i_);
                    const int n = t + P * i;
                    const float c0 = fmaxf(v[i].x, eps), c1 = fmaxf(v[i].y, eps);
                    if (ok0) c_nll = cf_add(c_nll, c0 - p0[n] * logf(c0));
                    if (ok1) c_nll = cf_add(c_nll, c1 - p1[n] * logf(c1));
                });
                const int slot = (int)((block * ((T + 31) / 32) + (threadIdx.x >> 5)) & 63);
                slot_add<T>(a.nll_stats + 2 * slot, c_nll);
            }
            if (kPf && !keep) {
                // d from global memory: no store in this loop, so its loads issue together
                static_for<0, E>([&](auto i_) {
                    constexpr int i = CUBIC_CI(i_);
                    const int n = t + P * i;
                    const float x0 = ok0 ? __fdividef(__ldg(p0 + n), fmaxf(v[i].x, eps)) : 0.f;
                    const float x1 = ok1 ? __fdividef(__ldg(p1 + n), fmaxf(v[i].y, eps)) : 0.f;
                    v[i] = make_float2(x0, x1);
                });
            } else static_for<0, E>([&](auto i_) {
                constexpr int i = CUBIC_CI(i_);
                const int n = t + P * i;
                // fast division (max 2 ulp for denominators below 2^126; the
                // clamp keeps them >= eps)
                const float x0 = ok0 ? __fdividef(p0[n], fmaxf(v[i].x, eps)) : 0.f;
                const float x1 = ok1 ? __fdividef(p1[n], fmaxf(v[i].y, eps)) : 0.f;
                if (keep) {
                    if (ok0) { kb0[n] = v[i].x; kr0[n] = x0; }
                    if (ok1) { kb1[n] = v[i].y; kr1[n] = x1; }
                }
                v[i] = make_float2(x0, x1);
            });
        } else if constexpr (MODE == XM_UPDATE || MODE == XM_FINAL) {
            // the update writes to dst when given (out of place), else over u
            float *ob = (MODE == XM_FINAL || a.dst) ? a.dst : a.u;
            float *o0 = ob + r0 * N, *o1 = ob + r1 * N;
            float *kq0 = a.keep_a + r0 * N, *kq1 = a.keep_a + r1 * N;
            const bool keep = a.keep_a != nullptr;
            const bool stats = a.stats != nullptr;
            float s_num = 0.f, s_den = 0.f;
            // accelerated RL (XM_FINAL only): g = x - u and its two dot products
            const bool acc = MODE == XM_FINAL && a.acc_g != nullptr;
            const bool acc_prev = a.acc_gprev != nullptr;
            CFloat c_num{0.f, 0.f}, c_den{0.f, 0.f};
            // g_{k-1}, loaded ahead of the loop: its stores could alias it as far as the
            // compiler knows, which would serialise each load behind the previous store
            float gp0[MODE == XM_FINAL ? E : 1], gp1[MODE == XM_FINAL ? E : 1];
            if constexpr (MODE == XM_FINAL) {
                if (acc && acc_prev) {
                    const float *h0 = a.acc_gprev + r0 * N, *h1 = a.acc_gprev + r1 * N;
                    static_for<0, E>([&](auto i_) {
                        constexpr int i = CUBIC_CI(i_);
                        gp0[i] = ok0 ? __ldg(h0 + t + P * i) : 0.f;
                        gp1[i] = ok1 ? __ldg(h1 + t + P * i) : 0.f;
                    });
                }
            }
            if constexpr (kPf) {
                // u from global memory, usually updated in place: every load of the
                // loop below comes before the first store to u, so none waits behind one
                if (keep) {
                    static_for<0, E>([&](auto i_) {
                        constexpr int i = CUBIC_CI(i_);
                        const int n = t + P * i;
                        if (ok0) kq0[n] = v[i].x;
                        if (ok1) kq1[n] = v[i].y;
                    });
                }
                static_for<0, E>([&](auto i_) {
                    constexpr int i = CUBIC_CI(i_);
                    const int n = t + P * i;
                    const float u0v = ok0 ? p0[n] : 0.f, u1v = ok1 ? p1[n] : 0.f;
                    const float x0 = ok0 ? u0v * v[i].x : 0.f;
                    const float x1 = ok1 ? u1v * v[i].y : 0.f;
                    if (stats) {
                        s_num = fmaf(x0 - u0v, x0 - u0v, fmaf(x1 - u1v, x1 - u1v, s_num));
                        s_den = fmaf(u0v, u0v, fmaf(u1v, u1v, s_den));
                    }
                    v[i] = make_float2(x0, x1);
                });
                static_for<0, E>([&](auto i_) {
                    constexpr int i = CUBIC_CI(i_);
                    const int n = t + P * i;
                    if (ok0) o0[n] = v[i].x;
                    if (ok1) o1[n] = v[i].y;
                });
            } else static_for<0, E>([&](auto i_) {
                constexpr int i = CUBIC_CI(i_);
                const int n = t + P * i;
                const float u0v = ok0 ? p0[n] : 0.f, u1v = ok1 ? p1[n] : 0.f;
                const float x0 = ok0 ? u0v * v[i].x : 0.f;
                const float x1 = ok1 ? u1v * v[i].y : 0.f;
                if (keep) {
                    if (ok0) kq0[n] = v[i].x;
                    if (ok1) kq1[n] = v[i].y;
                }
                if constexpr (MODE == XM_FINAL) {
                    if (acc) {
                        const float g0 = x0 - u0v, g1 = x1 - u1v;  // 0 on rows past the end
                        if (ok0) a.acc_g[r0 * N + n] = g0;
                        if (ok1) a.acc_g[r1 * N + n] = g1;
                        if (acc_prev) c_num = cf_add(cf_add(c_num, g0 * gp0[i]), g1 * gp1[i]);
                        c_den = cf_add(cf_add(c_den, g0 * g0), g1 * g1);
                    }
                }
                if (stats) {
                    s_num = fmaf(x0 - u0v, x0 - u0v, fmaf(x1 - u1v, x1 - u1v, s_num));
                    s_den = fmaf(u0v, u0v, fmaf(u1v, u1v, s_den));
                }
                if (ok0) o0[n] = x0;
                if (ok1) o1[n] = x1;
                v[i] = make_float2(x0, x1);
            });
            if (stats) {
                // warp sums where the warp is full, else one add per thread
                const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
                const int slot = (int)((block * ((T + 31) / 32) + warp) & 63);
                float *st4 = a.stats + 4 * slot;
                if ((warp + 1) * 32 <= T) {
                    for (int o = 16; o > 0; o >>= 1) {
                        s_num += __shfl_down_sync(0xffffffffu, s_num, o);
                        s_den += __shfl_down_sync(0xffffffffu, s_den, o);
                    }
                    if (lane == 0) {
                        catomic_add(st4, st4 + 1, s_num);
                        catomic_add(st4 + 2, st4 + 3, s_den);
                    }
                } else {
                    catomic_add(st4, st4 + 1, s_num);
                    catomic_add(st4 + 2, st4 + 3, s_den);
                }
            }
            if constexpr (MODE == XM_FINAL) {
                if (acc) {  // uniform over the CTA
                    const float4 tot = block_merge2<T>(c_num, c_den);
                    if (threadIdx.x == 0) a.acc_part[block] = tot;
                }
            }
        }
    }

    if constexpr (MODE == XM_FWD || MODE == XM_RATIO || MODE == XM_UPDATE || MODE >= XM_ADJ_R) {
        // On lines longer than 1024 with more than 16 elements per thread, the passes that
        // run two transforms would keep every exchange address of the inverse transform
        // live across the pointwise step for reuse in the forward one (about 165 registers
        // at length 2560).  An opaque copy of the thread index makes the compiler recompute
        // them instead (96 registers).  Shorter lines do better without it.
        int tf = t;
        if constexpr (N > 1024 && E > 16 && MODE != XM_FWD) asm volatile("" : "+r"(tf));
        FFT::forward(v, sm, stw, tf, sync);
        // split the packed spectrum into the two rows' half spectra
        static_for<0, E>([&](auto i_) {
            constexpr int i = CUBIC_CI(i_);
            sm.at(tf + P * i) = v[i];
        });
        sync();
        float2 *q0 = a.spec_out + srow(r0) * a.xp, *q1 = a.spec_out + srow(r1) * a.xp;
        static_for<0, E>([&](auto i_) {
            constexpr int i = CUBIC_CI(i_);
            const int k = tf + P * i;
            if (2 * k <= N) {
                const float2 zk = v[i];
                const float2 zn = sm.at(k == 0 ? 0 : N - k);
                const float2 A = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
                const float2 B = make_float2(0.5f * (zk.y + zn.y), 0.5f * (zn.x - zk.x));
                if (ok0) q0[k] = A;
                if (ok1) q1[k] = B;
            }
        });
    }
}

// ------------------------------------------------------------------ multi-volume launches
// One launch covers several volumes of the same axis length (the batched path):
// block b belongs to the volume v with prefix[v] <= b < prefix[v+1].

constexpr int kMaxBatch = 256;

template <class Args>
struct MultiTable {
    int nvol;
    int64_t prefix[kMaxBatch + 1];
    Args args[kMaxBatch];
};

__device__ __forceinline__ int find_volume(const int64_t *prefix, int nvol, int64_t b)
{
    int lo = 0, hi = nvol - 1;
    while (lo < hi) {  // largest v with prefix[v] <= b
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// tab == nullptr: one volume, arguments by value.  Otherwise the volumes of tab.
template <int N, int P, int L, int MODE, bool PF>
__device__ __forceinline__ void x_entry(XArgs a, const MultiTable<XArgs> *tab)
{
    int64_t block = blockIdx.x;
    if (tab) {
        const int v = find_volume(tab->prefix, tab->nvol, blockIdx.x);
        a = tab->args[v];
        block -= tab->prefix[v];
    }
    x_body<N, P, L, MODE, PF>(a, block);
}

template <int N, int P, int L, int MODE>
__global__ void __launch_bounds__(P * L) k_xpass(XArgs a, const MultiTable<XArgs> *tab)
{
    x_entry<N, P, L, MODE, false>(a, tab);
}

// The prefetching ratio and update kernels exist to fit more CTAs on an SM: they are
// held to the register count of 28 resident warps (72 registers) for up to 16 elements
// per thread, of 16 warps (128 registers) up to 32, else of 12 warps (168 registers).
template <int N, int P, int L>
constexpr int x_pf_min_blocks()
{
    constexpr int threads = N / P <= 16 ? 896 : N / P <= 32 ? 512 : 384;
    return P * L <= threads / 2 ? threads / (P * L) : 1;
}

template <int N, int P, int L, int MODE>
__global__ void __launch_bounds__(P * L, (x_pf_min_blocks<N, P, L>()))
    k_xpass_pf(XArgs a, const MultiTable<XArgs> *tab)
{
    x_entry<N, P, L, MODE, true>(a, tab);
}

// the kernel of one X launch shape
template <int N, int P, int L, int MODE, bool PF>
constexpr auto x_kernel()
{
    if constexpr (x_prefetches<N, MODE, PF>())
        return k_xpass_pf<N, P, L, MODE>;
    else
        return k_xpass<N, P, L, MODE>;
}

// ------------------------------------------------------------------ Y pass

template <int N, int P, int B>
__device__ __forceinline__ void y_body(const YArgs &a, const int64_t bx, const int64_t by)
{
    constexpr int E = N / P;
    using FFT = LineFFT<N, P, true>;
    extern __shared__ float2 smem_y[];
    float2 *stw = smem_y + B * N;
    const int b = threadIdx.x % B;
    const int t = threadIdx.x / B;
    const int64_t col = a.col0 + bx * B + b;
    const bool ok = col < a.col1;
    float2 *base = a.spec + by * N * a.xp + col;
    SmemStrided sm{smem_y + b, B};
    auto sync = [] { __syncthreads(); };
    pdl_trigger();
    FFT::fill_twiddles(stw, a.tw, threadIdx.x, P * B);
    __syncthreads();
    pdl_wait();
    float2 v[E];
    const float sgn = a.inverse ? -1.f : 1.f;
    const int nl = a.nload > 0 ? (int)a.nload : N, ns = a.nstore > 0 ? (int)a.nstore : N;
    static_for<0, E>([&](auto i_) {
        constexpr int i = CUBIC_CI(i_);
        const int pos = t + P * i;
        float2 x = (ok && pos < nl) ? base[(int64_t)pos * a.xp] : make_float2(0.f, 0.f);
        v[i] = make_float2(x.x, sgn * x.y);
    });
    FFT::forward(v, sm, stw, t, sync);
    if (ok) {
        static_for<0, E>([&](auto i_) {
            constexpr int i = CUBIC_CI(i_);
            const int pos = t + P * i;
            if (pos < ns) base[(int64_t)pos * a.xp] = make_float2(v[i].x, sgn * v[i].y);
        });
    }
}

// tab == nullptr: one volume, grid (column tiles, nz).  Otherwise a 1D grid over the
// volumes of tab, volume v's blocks flattened as tile + ntiles * z; `inverse` then
// overrides the table's direction.
template <int N, int P, int B>
__global__ void __launch_bounds__(P * B) k_ypass(YArgs a, const MultiTable<YArgs> *tab, int inverse)
{
    int64_t bx = blockIdx.x, by = blockIdx.y;
    if (tab) {
        const int v = find_volume(tab->prefix, tab->nvol, blockIdx.x);
        a = tab->args[v];
        a.inverse = inverse;
        const int64_t local = (int64_t)blockIdx.x - tab->prefix[v];
        const int64_t nct = (a.col1 - a.col0 + B - 1) / B;
        bx = local % nct;
        by = local / nct;
    }
    y_body<N, P, B>(a, bx, by);
}

// ------------------------------------------------------------------ Z pass

template <int N, int P, int B>
__device__ __forceinline__ void z_body(const ZArgs &a, const int64_t bx, const int64_t by)
{
    constexpr int E = N / P;
    using FFT = LineFFT<N, P, true>;
    extern __shared__ float2 smem_z[];
    float2 *stw = smem_z + B * N;
    const int b = threadIdx.x % B;
    const int t = threadIdx.x / B;
    const int64_t col = a.col0 + bx * B + b;
    const bool ok = col < a.col1;
    const int64_t zstride = a.ny * a.xp;
    const int64_t off = by * a.xp + col;
    float2 *base = a.spec + off;
    SmemStrided sm{smem_z + b, B};
    auto sync = [] { __syncthreads(); };
    pdl_trigger();
    FFT::fill_twiddles(stw, a.tw, threadIdx.x, P * B);
    __syncthreads();
    pdl_wait();
    float2 v[E];
    const bool inv_only = a.mode == ZM_INV_SCALE;
    const int nl = a.nload > 0 ? (int)a.nload : N, ns = a.nstore > 0 ? (int)a.nstore : N;
    static_for<0, E>([&](auto i_) {
        constexpr int i = CUBIC_CI(i_);
        const int pos = t + P * i;
        const float2 x = (ok && pos < nl) ? base[(int64_t)pos * zstride] : make_float2(0.f, 0.f);
        v[i] = inv_only ? cconj(x) : x;
    });
    FFT::forward(v, sm, stw, t, sync);
    if (a.mode == ZM_FWD_SCALE || inv_only) {
        const float s = a.scale, sy = inv_only ? -a.scale : a.scale;
        if (ok) {
            static_for<0, E>([&](auto i_) {
                constexpr int i = CUBIC_CI(i_);
                const int pos = t + P * i;
                if (pos < ns) base[(int64_t)pos * zstride] = make_float2(v[i].x * s, v[i].y * sy);
            });
        }
        return;
    }
    const bool corr = a.mode == ZM_CORR;
    if (ok && a.save) {
        static_for<0, E>([&](auto i_) {
            constexpr int i = CUBIC_CI(i_);
            a.save[off + (int64_t)(t + P * i) * zstride] = v[i];
        });
    }
    if (ok && a.gacc) {
        static_for<0, E>([&](auto i_) {
            constexpr int i = CUBIC_CI(i_);
            const int64_t j = off + (int64_t)(t + P * i) * zstride;
            const float2 o = __ldg(a.gother + j);
            a.gacc[j] = cadd(a.gacc[j], a.gconj ? cmulconj(o, v[i]) : cmulconj(v[i], o));
        });
    }
    if (a.mode == ZM_MUL_REAL) {
        const float *hb = a.Hr + off;
        static_for<0, E>([&](auto i_) {
            constexpr int i = CUBIC_CI(i_);
            const float h = ok ? __ldg(hb + (int64_t)(t + P * i) * zstride) : 0.f;
            v[i] = make_float2(v[i].x * h, -v[i].y * h);
        });
    } else {
        const float2 *hb = a.H + off;
        // product with H or conj(H), then conjugate for the inverse transform
        static_for<0, E>([&](auto i_) {
            constexpr int i = CUBIC_CI(i_);
            const float2 h = ok ? __ldg(hb + (int64_t)(t + P * i) * zstride) : make_float2(0.f, 0.f);
            const float2 p = corr ? cmulconj(v[i], h) : cmul(v[i], h);
            v[i] = cconj(p);
        });
    }
    sync();  // the forward transform's last shared-memory reads are done
    FFT::forward(v, sm, stw, t, sync);
    if (ok) {
        static_for<0, E>([&](auto i_) {
            constexpr int i = CUBIC_CI(i_);
            const int pos = t + P * i;
            if (pos < ns) base[(int64_t)pos * zstride] = cconj(v[i]);
        });
    }
}

// as k_ypass: tab == nullptr for one volume (grid: column tiles, ny), else volume v's
// blocks flattened as tile + ntiles * y, with `mode` overriding the table's mode.
template <int N, int P, int B>
__global__ void __launch_bounds__(P * B) k_zpass(ZArgs a, const MultiTable<ZArgs> *tab, int mode)
{
    int64_t bx = blockIdx.x, by = blockIdx.y;
    if (tab) {
        const int v = find_volume(tab->prefix, tab->nvol, blockIdx.x);
        a = tab->args[v];
        // a volume with a real H multiplies by it for both convolution and correlation
        a.mode = (a.Hr && (mode == ZM_CONV || mode == ZM_CORR)) ? (int)ZM_MUL_REAL : mode;
        const int64_t local = (int64_t)blockIdx.x - tab->prefix[v];
        const int64_t nct = (a.col1 - a.col0 + B - 1) / B;
        bx = local % nct;
        by = local / nct;
    }
    z_body<N, P, B>(a, bx, by);
}

}  // namespace cubic
