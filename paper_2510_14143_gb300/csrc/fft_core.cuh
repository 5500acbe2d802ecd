// fft_core.cuh -- in-register mixed-radix DFTs and the line FFT used by every
// pass of the 3D transform (sm_103a).
//
// The paper's Richardson-Lucy iteration (Section 4, "Richardson-Lucy
// deconvolution") does its two convolutions per iteration with FFTs ("GPU-
// resident FFT operations for convolution steps").  This file is the FFT
// engine: a mixed-radix (2/3/4/5 and products) Stockham autosort transform of
// one line of length N, spread over P threads that each hold E = N/P elements
// in registers.
//
// Register layout ("canonical"): thread t, slot i holds element t + P*i.
// Stage s (radix R, span Ns = product of earlier radices) runs E/R butterflies
// per thread: butterfly j = t + P*g reads elements j + r*N/R, which are slots
// g + r*E/R of the same thread, twiddles them by W_{Ns R}^{(j mod Ns) r},
// does a radix-R DFT and writes its outputs to positions
// (j div Ns)*Ns*R + (j mod Ns) + r*Ns.  Between stages the outputs go through
// shared memory and come back in canonical order; after the last stage the
// outputs already sit in canonical order, so a transform costs (stages - 1)
// shared-memory exchanges and its first/last stage talk to global memory
// directly with coalesced accesses.
//
// The inverse transform is conj(F(conj(x))) (unnormalised).  Twiddles of the
// inter-stage kind come from a per-length table generated once in double
// precision (cospi/sinpi) and rounded to float; the fixed twiddles inside the
// in-register DFTs are compile-time constants computed below from their
// Taylor series in double precision.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace cubic {

// ------------------------------------------------------------ compile time

constexpr double kPi = 3.141592653589793238462643383279502884;

// Taylor series, valid to double precision for |x| <= pi/4.
constexpr double ct_sin_series(double x)
{
    double term = x, sum = x;
    for (int k = 1; k < 15; ++k) {
        term *= -x * x / double((2 * k) * (2 * k + 1));
        sum += term;
    }
    return sum;
}

constexpr double ct_cos_series(double x)
{
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 15; ++k) {
        term *= -x * x / double((2 * k - 1) * (2 * k));
        sum += term;
    }
    return sum;
}

struct CtCis {
    double c, s;
};

// cos and sin of 2*pi*m/n: reduce to the nearest quarter turn, evaluate the
// series on a residual of at most pi/4, rotate back exactly.
constexpr CtCis ct_cis(long m, long n)
{
    m %= n;
    if (m < 0) m += n;
    long q = (4 * m + n / 2) / n;  // nearest quarter, 0..4
    double th = 2.0 * kPi * double(4 * m - q * n) / double(4 * n);
    double c = ct_cos_series(th), s = ct_sin_series(th);
    switch (q & 3) {
    case 0: return {c, s};
    case 1: return {-s, c};
    case 2: return {-c, -s};
    default: return {s, -c};
    }
}

constexpr int smallest_radix(int r)
{
    return (r % 4 == 0 && r != 4) ? 4 : (r % 2 == 0) ? 2 : (r % 3 == 0) ? 3 : 5;
}

constexpr int gcd_ct(int a, int b) { return b == 0 ? a : gcd_ct(b, a % b); }

constexpr bool is_5smooth(int n)
{
    if (n < 1) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    while (n % 5 == 0) n /= 5;
    return n == 1;
}

constexpr int radical(int n)
{
    return (n % 2 == 0 ? 2 : 1) * (n % 3 == 0 ? 3 : 1) * (n % 5 == 0 ? 5 : 1);
}

// Greedy radix plan: each stage takes gcd(E, remaining).
constexpr int plan_stages(int N, int E)
{
    int M = N, s = 0;
    while (M > 1) {
        int R = gcd_ct(E, M);
        if (R == 1) return -1;
        M /= R;
        ++s;
    }
    return s;
}

constexpr int plan_radix(int N, int E, int stage)
{
    int M = N;
    for (int s = 0; s < stage; ++s) M /= gcd_ct(E, M);
    return gcd_ct(E, M);
}

constexpr int plan_span(int N, int E, int stage)
{
    int M = N, ns = 1;
    for (int s = 0; s < stage; ++s) {
        int R = gcd_ct(E, M);
        M /= R;
        ns *= R;
    }
    return ns;
}

// Stage twiddle tables: for stage s >= 1 (radix R, span Ns) the table holds
// W_{Ns R}^{k r} at [r - 1][k] (1 <= r < R, k < Ns; the r = 0 row is all ones and is
// not stored), so lanes with consecutive k read consecutive words.  Tables of all
// stages are stored back to back.
constexpr int tw_stage_offset(int N, int E, int stage)
{
    int off = 0;
    for (int s = 1; s < stage; ++s) off += (plan_radix(N, E, s) - 1) * plan_span(N, E, s);
    return off;
}

constexpr int tw_table_size(int N, int E)
{
    return (N == 1) ? 0 : tw_stage_offset(N, E, plan_stages(N, E));
}

// Threads per line: fewest stages with at most Emax elements per thread,
// ties broken towards E near 24.
constexpr int choose_threads(int N, int Emax)
{
    int bestP = -1, bestS = 1 << 20, bestD = 1 << 20;
    for (int P = 1; P <= N; ++P) {
        if (N % P) continue;
        int E = N / P;
        if (E > Emax || E % radical(N)) continue;
        int s = plan_stages(N, E);
        if (s < 0) continue;
        int d = E > 24 ? E - 24 : 24 - E;
        if (s < bestS || (s == bestS && d < bestD)) {
            bestS = s;
            bestD = d;
            bestP = P;
        }
    }
    return bestP;
}

template <int Begin, int End, class F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (Begin < End) {
        f(std::integral_constant<int, Begin>{});
        static_for<Begin + 1, End>(f);
    }
}

#define CUBIC_CI(v) decltype(v)::value

// ------------------------------------------------------------ complex ops

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulconj(float2 a, float2 b)  // a * conj(b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }  // * (-i)
__device__ __forceinline__ float2 mul_pi(float2 a) { return make_float2(-a.y, a.x); }  // * (+i)

// x * W_R^e with W_R = exp(-2 pi i / R), e and R compile-time.
template <int e_, int R>
__device__ __forceinline__ float2 mul_w(float2 x)
{
    constexpr int e = ((e_ % R) + R) % R;
    if constexpr (e == 0) {
        return x;
    } else if constexpr (4 * e == R) {
        return mul_mi(x);
    } else if constexpr (2 * e == R) {
        return make_float2(-x.x, -x.y);
    } else if constexpr (4 * e == 3 * R) {
        return mul_pi(x);
    } else if constexpr (8 * e == R) {  // (1 - i)/sqrt2
        constexpr float h = float(0.70710678118654752440);
        return make_float2((x.x + x.y) * h, (x.y - x.x) * h);
    } else if constexpr (8 * e == 3 * R) {  // (-1 - i)/sqrt2
        constexpr float h = float(0.70710678118654752440);
        return make_float2((x.y - x.x) * h, -(x.x + x.y) * h);
    } else {
        constexpr CtCis w = ct_cis(-e, R);
        constexpr float c = float(w.c), s = float(w.s);
        return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
    }
}

// ------------------------------------------------------------ register DFTs
// Forward DFT X[k] = sum_n x[n] W_R^{kn}, in place on v[0..R).

template <int R>
struct Dft;

template <>
struct Dft<1> {
    __device__ __forceinline__ static void run(float2 (&)[1]) {}
};

template <>
struct Dft<2> {
    __device__ __forceinline__ static void run(float2 (&v)[2])
    {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <>
struct Dft<3> {
    __device__ __forceinline__ static void run(float2 (&v)[3])
    {
        constexpr float s3 = float(0.86602540378443864676);  // sin(2 pi / 3)
        float2 a = v[0], t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
        float2 m = make_float2(fmaf(-0.5f, t1.x, a.x), fmaf(-0.5f, t1.y, a.y));
        float2 j = make_float2(s3 * t2.y, -s3 * t2.x);  // -i sin(2pi/3) (x1 - x2)
        v[0] = cadd(a, t1);
        v[1] = cadd(m, j);
        v[2] = csub(m, j);
    }
};

template <>
struct Dft<4> {
    __device__ __forceinline__ static void run(float2 (&v)[4])
    {
        float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        float2 s13 = cadd(v[1], v[3]), d13 = mul_mi(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    }
};

template <>
struct Dft<5> {
    __device__ __forceinline__ static void run(float2 (&v)[5])
    {
        constexpr CtCis w1 = ct_cis(1, 5), w2 = ct_cis(2, 5);
        constexpr float c1 = float(w1.c), s1 = float(w1.s), c2 = float(w2.c), s2 = float(w2.s);
        float2 a = v[0];
        float2 p1 = cadd(v[1], v[4]), m1 = csub(v[1], v[4]);
        float2 p2 = cadd(v[2], v[3]), m2 = csub(v[2], v[3]);
        float2 r1 = make_float2(a.x + c1 * p1.x + c2 * p2.x, a.y + c1 * p1.y + c2 * p2.y);
        float2 r2 = make_float2(a.x + c2 * p1.x + c1 * p2.x, a.y + c2 * p1.y + c1 * p2.y);
        // -i (s1 m1 + s2 m2) and -i (s2 m1 - s1 m2)
        float2 i1 = make_float2(s1 * m1.y + s2 * m2.y, -(s1 * m1.x + s2 * m2.x));
        float2 i2 = make_float2(s2 * m1.y - s1 * m2.y, -(s2 * m1.x - s1 * m2.x));
        v[0] = cadd(a, cadd(p1, p2));
        v[1] = cadd(r1, i1);
        v[4] = csub(r1, i1);
        v[2] = cadd(r2, i2);
        v[3] = csub(r2, i2);
    }
};

// Composite R = A*B: A-point DFTs over n1 for every n2 (input n = n2 + B*n1),
// twiddle W_R^{n2 k1}, then B-point DFTs over n2; output k = k1 + A*k2.
template <int R>
struct Dft {
    static constexpr int A = smallest_radix(R);
    static constexpr int B = R / A;
    static_assert(A * B == R && B > 1, "radix must be 5-smooth");
    __device__ __forceinline__ static void run(float2 (&v)[R])
    {
        float2 y[B][A];
        static_for<0, B>([&](auto n2_) {
            constexpr int n2 = CUBIC_CI(n2_);
            float2 s[A];
            static_for<0, A>([&](auto n1_) {
                constexpr int n1 = CUBIC_CI(n1_);
                s[n1] = v[n2 + B * n1];
            });
            Dft<A>::run(s);
            static_for<0, A>([&](auto k1_) {
                constexpr int k1 = CUBIC_CI(k1_);
                y[n2][k1] = mul_w<n2 * k1, R>(s[k1]);
            });
        });
        static_for<0, A>([&](auto k1_) {
            constexpr int k1 = CUBIC_CI(k1_);
            float2 t[B];
            static_for<0, B>([&](auto n2_) {
                constexpr int n2 = CUBIC_CI(n2_);
                t[n2] = y[n2][k1];
            });
            Dft<B>::run(t);
            static_for<0, B>([&](auto k2_) {
                constexpr int k2 = CUBIC_CI(k2_);
                v[k1 + A * k2] = t[k2];
            });
        });
    }
};

// ------------------------------------------------------------ line FFT

// kSmemTw: `tw` is the stage table in shared memory (fill_twiddles); otherwise it
// is the length-N table W_N^m in global memory.
template <int N, int P, bool kSmemTw = false>
struct LineFFT {
    static_assert(N % P == 0, "P must divide N");
    static constexpr int E = N / P;
    static constexpr int S = (N == 1) ? 0 : plan_stages(N, E);
    static_assert(S >= 0, "no radix plan for this (N, P)");
    static constexpr int kTwSize = tw_table_size(N, E);

    // Build the stage table in shared memory from the global W_N^m table
    // (threads tid = 0 .. nthreads-1 cooperate; the caller synchronises after).
    __device__ __forceinline__ static void fill_twiddles(float2 *smem_tw, const float2 *__restrict__ tw_global, int tid,
                                                         int nthreads)
    {
        static_for<1, (S > 1 ? S : 1)>([&](auto s_) {
            constexpr int s = CUBIC_CI(s_);
            constexpr int R = plan_radix(N, E, s);
            constexpr int Ns = plan_span(N, E, s);
            constexpr int TS = N / (Ns * R);
            float2 *dst = smem_tw + tw_stage_offset(N, E, s);
            for (int i = tid; i < (R - 1) * Ns; i += nthreads) {
                const int r = 1 + i / Ns, k = i % Ns;
                dst[i] = __ldg(tw_global + k * r * TS);
            }
        });
    }

    // Forward transform of the canonical register set v of thread t.  `sm` maps
    // a line position to its shared-memory slot (sm.at(pos)); `sync`
    // synchronises every thread sharing that buffer.
    template <class Sm, class Sync>
    __device__ __forceinline__ static void forward(float2 (&v)[E], const Sm &sm, const float2 *__restrict__ tw,
                                                   int t, Sync &&sync)
    {
        static_for<0, S>([&](auto s_) {
            constexpr int s = CUBIC_CI(s_);
            constexpr int R = plan_radix(N, E, s);
            constexpr int Ns = plan_span(N, E, s);
            constexpr int G = E / R;
            constexpr int TS = N / (Ns * R);  // twiddle table stride
            constexpr bool last = (s == S - 1);
            static_for<0, G>([&](auto g_) {
                constexpr int g = CUBIC_CI(g_);
                float2 x[R];
                static_for<0, R>([&](auto r_) {
                    constexpr int r = CUBIC_CI(r_);
                    x[r] = v[g + r * G];
                });
                const int j = t + P * g;
                const int k = j % Ns;
                if constexpr (s > 0) {
                    if constexpr (kSmemTw) {
                        const float2 *ts = tw + tw_stage_offset(N, E, s) + k;
                        static_for<1, R>([&](auto r_) {
                            constexpr int r = CUBIC_CI(r_);
                            x[r] = cmul(x[r], ts[(r - 1) * Ns]);
                        });
                    } else {
                        static_for<1, R>([&](auto r_) {
                            constexpr int r = CUBIC_CI(r_);
                            x[r] = cmul(x[r], __ldg(tw + k * r * TS));
                        });
                    }
                }
                Dft<R>::run(x);
                if constexpr (last) {
                    static_for<0, R>([&](auto r_) {
                        constexpr int r = CUBIC_CI(r_);
                        v[g + r * G] = x[r];
                    });
                } else {
                    const int base = (j / Ns) * Ns * R + k;
                    static_for<0, R>([&](auto r_) {
                        constexpr int r = CUBIC_CI(r_);
                        sm.at(base + r * Ns) = x[r];
                    });
                }
            });
            if constexpr (!last) {
                sync();
                static_for<0, E>([&](auto i_) {
                    constexpr int i = CUBIC_CI(i_);
                    v[i] = sm.at(t + P * i);
                });
                sync();
            }
        });
    }

    template <class Sm, class Sync>
    __device__ __forceinline__ static void inverse(float2 (&v)[E], const Sm &sm, const float2 *__restrict__ tw,
                                                   int t, Sync &&sync)
    {
        static_for<0, E>([&](auto i_) { v[CUBIC_CI(i_)].y = -v[CUBIC_CI(i_)].y; });
        forward(v, sm, tw, t, sync);
        static_for<0, E>([&](auto i_) { v[CUBIC_CI(i_)].y = -v[CUBIC_CI(i_)].y; });
    }
};

}  // namespace cubic
