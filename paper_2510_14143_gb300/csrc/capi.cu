// capi.cu -- the extern "C" boundary (include/cubic_rl.h) and the host-side
// plan: argument validation, device buffers, and the enqueueing of the pass
// kernels that make up each Richardson-Lucy iteration.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <stdlib.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/cubic_rl.h"
#include "lens.cuh"
#include "registry.cuh"

using namespace cubic;

// ------------------------------------------------------------------ errors

static thread_local char g_last_error[512];

static cubic_status_t fail(cubic_status_t s, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
static cubic_status_t fail(cubic_status_t s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return s;
}

#define CUBIC_CUDA(call)                                                                         \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(e_ == cudaErrorMemoryAllocation ? CUBIC_ERR_OUT_OF_MEMORY : CUBIC_ERR_CUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);    \
    } while (0)

extern "C" const char *cubic_status_string(cubic_status_t s)
{
    switch (s) {
    case CUBIC_OK: return "ok";
    case CUBIC_ERR_INVALID_ARG: return "invalid argument";
    case CUBIC_ERR_UNSUPPORTED_SIZE: return "unsupported size";
    case CUBIC_ERR_ALIGNMENT: return "misaligned pointer";
    case CUBIC_ERR_OUT_OF_MEMORY: return "out of device memory";
    case CUBIC_ERR_CUDA: return "CUDA error";
    case CUBIC_ERR_TIMEOUT: return "device wait timed out";
    case CUBIC_ERR_NOT_READY: return "not ready";
    }
    return "unknown status";
}

extern "C" const char *cubic_last_error(void) { return g_last_error; }

// ------------------------------------------------------------------ registry

namespace cubic {
template <int S>
void register_shard(AxisKernels *table);
}

static AxisKernels g_table[kNumLengths];
static std::once_flag g_table_once;

template <int S>
static void register_all()
{
    if constexpr (S < kShards) {
        register_shard<S>(g_table);
        register_all<S + 1>();
    }
}

static void init_table() { register_all<0>(); }

const AxisKernels *cubic::find_axis(int64_t n)
{
    std::call_once(g_table_once, init_table);
    for (int i = 0; i < kNumLengths; ++i)
        if (kLengths[i] == n) return g_table[i].n == n ? &g_table[i] : nullptr;
    return nullptr;
}

extern "C" int cubic_rl_supported_length(int64_t n) { return find_axis(n) != nullptr; }

PFN_cuTensorMapEncodeTiled_v12000 cubic::tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
        return (PFN_cuTensorMapEncodeTiled_v12000)p;
    }();
    return fn;
}

// ------------------------------------------------------------------ small kernels

// Twiddles W_n^m = exp(-2 pi i m / n), m < n: evaluated in double, rounded to float.
__global__ void k_twiddles(float2 *tw, int n)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double s, c;
    sincospi(2.0 * (double)m / (double)n, &s, &c);
    tw[m] = make_float2((float)c, (float)(-s));
}

// h0(z,y,x) = psf((z+nz/2) mod nz, (y+ny/2) mod ny, (x+nx/2) mod nx): PSF peak to the origin.
__global__ void k_center_to_origin(const float *__restrict__ psf, float *__restrict__ h0, int64_t nz, int64_t ny,
                                   int64_t nx)
{
    const int64_t V = nz * ny * nx;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
        int64_t xs = x + nx / 2, ys = y + ny / 2, zs = z + nz / 2;
        if (xs >= nx) xs -= nx;
        if (ys >= ny) ys -= ny;
        if (zs >= nz) zs -= nz;
        h0[i] = psf[(zs * ny + ys) * nx + xs];
    }
}

// Flux sum: each thread reads 16-byte vectors and keeps two compensated float32 sums
// (about twice float precision over its few hundred terms); the threads' sums merge in
// double per warp and per block, and one block folds the block partials in double.
constexpr int kReduceThreads = 256;
constexpr int kReduceBlocks = 1024;

__global__ void __launch_bounds__(kReduceThreads) k_sum_partial(const float *__restrict__ x, int64_t n,
                                                                double *__restrict__ partial)
{
    __shared__ double sh[kReduceThreads / 32];
    CFloat a{0.f, 0.f}, b{0.f, 0.f};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // 16-byte vectors where x is 16-byte aligned, then the scalar tail
    const int64_t n4 = ((uintptr_t)x & 15u) == 0 ? n / 4 : 0;
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    for (int64_t i = first; i < n4; i += stride) {
        const float4 v = __ldg(x4 + i);
        a = cf_add(cf_add(a, v.x), v.y);
        b = cf_add(cf_add(b, v.z), v.w);
    }
    for (int64_t i = 4 * n4 + first; i < n; i += stride) a = cf_add(a, __ldg(x + i));
    double s = ((double)a.s - (double)a.c) + ((double)b.s - (double)b.c);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < kReduceThreads / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) partial[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kReduceThreads) k_sum_final(const double *__restrict__ partial, int n,
                                                              double *__restrict__ out)
{
    __shared__ double sh[kReduceThreads / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < kReduceThreads / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) out[0] = s;
    }
}

// max(sum / V, eps), once per CTA: the double division is slow on this GPU's FP64 units,
// and small volumes launch one thread per voxel
__device__ __forceinline__ float initial_value_block(const double *__restrict__ sum, int64_t V, float eps)
{
    __shared__ float v_sh;
    if (threadIdx.x == 0) {
        const double m = sum[0] / (double)V;
        v_sh = m > (double)eps ? (float)m : eps;
    }
    __syncthreads();
    return v_sh;
}

// u0 = max(sum / V, eps) everywhere.
__global__ void k_fill_initial(float *__restrict__ u, int64_t V, const double *__restrict__ sum, float eps)
{
    const float v = initial_value_block(sum, V, eps);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x)
        u[i] = v;
}

static unsigned grid_for(int64_t n, int threads, int64_t cap = 152 * 32)
{
    int64_t g = (n + threads - 1) / threads;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

// ------------------------------------------------------------------ kernel kinds

enum KernelKind : int {
    KK_SUM = 0, KK_FILL, KK_SHIFT, KK_X_FWD, KK_X_INV, KK_X_RATIO, KK_X_UPDATE, KK_X_FINAL,
    KK_Y_FWD, KK_Y_INV, KK_Z_FWD, KK_Z_INV, KK_Z_CONV, KK_Z_CORR,
    KK_X_ACC_UPDATE, KK_X_ACC_PREDICT, KK_ACC_ALPHA, KK_X_ADJOINT, KK_COUNT
};

static const char *const kKindNames[KK_COUNT] = {
    "sum", "fill_initial", "center_to_origin", "x_fwd", "x_inv", "x_ratio", "x_update", "x_final",
    "y_fwd", "y_inv", "z_fwd", "z_inv", "z_conv", "z_corr", "x_acc_update", "x_acc_predict", "acc_alpha",
    "x_adjoint"};

// ------------------------------------------------------------------ plan

struct cubic_rl_plan_s {
    int device = 0;
    int64_t nz = 0, ny = 0, nx = 0, V = 0, rows = 0, xh = 0, xp = 0;
    const AxisKernels *kx = nullptr, *ky = nullptr, *kz = nullptr;
    int vx = 0, vy = 0, vz = 0; // launch-shape variant of each pass
    int64_t chunk = 0;          // spectrum columns per Y/Z chunk (0: all at once)
    unsigned *err = nullptr;    // device error word (bounded waits), owned
    unsigned long long wait_ns = 0;  // limit of every bounded device wait (0: 2 s)
    float2 *H = nullptr;        // [nz][ny][xp], owned
    float2 *tw = nullptr;       // twiddles: x | y | z, owned
    float2 *tw_x = nullptr, *tw_y = nullptr, *tw_z = nullptr;
    double *partial = nullptr;  // kReduceBlocks + 1 doubles, owned
    float2 *ws = nullptr;       // spectrum work array
    bool own_ws = false;
    float *stage_in = nullptr, *stage_out = nullptr;  // device copies for host-buffer calls, owned
    unsigned char *bwd = nullptr;                      // gradient scratch, owned
    size_t bwd_bytes = 0;
    // point-symmetric PSF: H is real and the Z passes read it as float (half the bytes)
    float2 *ws2 = nullptr;         // second spectrum (FSC), owned
    float *fsc_sums = nullptr;     // [2][3][n_shells] compensated pairs, owned
    int fsc_cap = 0;
    float *auto_stats = nullptr;  // automatic stopping: [iteration][64 slots][2 sums][hi, lo], owned
    float *auto_delta = nullptr;  // [iteration]
    int auto_cap = 0;
    // accelerated RL: x (two), y, g (two) volumes, the update pass's per-CTA partial
    // sums and the state (den_{k-1}, alpha_{k+1}); allocated on first use, owned
    float *acc = nullptr;
    float4 *acc_part = nullptr;
    float *acc_state = nullptr;
    // metric-guided stopping: per-iteration slots and records, owned
    float *mon = nullptr;
    int mon_cap = 0;
    bool allow_real_h = false;  // set by cubic_rl_plan (may allocate Hr)
    bool use_real_h = false;
    float *Hr = nullptr;        // [nz][ny][xp], owned
    // linear ("same"-mode) boundaries: nz, ny, nx are then the transform's dims, the image is
    // iz x iy x ix (V, rows count its voxels and rows), the plan keeps the image and the
    // estimate in rows zero-padded to nx (lin: [2][iz][iy][nx]) and the spectrum work array
    // holds iz planes
    bool linear = false;
    int64_t iz = 0, iy = 0, ix = 0;
    int64_t pdims[3] = {0, 0, 0};  // the PSF box of a linear plan
    float *lin = nullptr;
    // launch accounting and optional per-kernel CUDA-event timing
    int64_t launches[KK_COUNT] = {};
    double bytes[KK_COUNT] = {};
    bool prof = false;
    std::vector<cudaEvent_t> ev;       // pairs (begin, end)
    std::vector<int> ev_kind;
    size_t ev_used = 0;
};

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// planes and rows per plane of the work arrays (the image's for a linear plan)
static int64_t work_planes(const cubic_rl_plan_s *p) { return p->linear ? p->iz : p->nz; }
static int64_t work_ny(const cubic_rl_plan_s *p) { return p->linear ? p->iy : p->ny; }
// the spectrum work array, and H (all nz planes of the transform)
static size_t spec_elems(const cubic_rl_plan_s *p) { return (size_t)work_planes(p) * p->ny * p->xp; }
static size_t h_elems(const cubic_rl_plan_s *p) { return (size_t)p->nz * p->ny * p->xp; }
// elements of one padded real work array of a linear plan
static size_t lin_elems(const cubic_rl_plan_s *p) { return (size_t)p->iz * p->iy * p->nx; }

static cubic_status_t ensure_workspace(cubic_rl_plan_s *p)
{
    if (p->ws) return CUBIC_OK;
    void *w = nullptr;
    CUBIC_CUDA(cudaMalloc(&w, spec_elems(p) * sizeof(float2)));
    p->ws = (float2 *)w;
    p->own_ws = true;
    return CUBIC_OK;
}

// Algorithmic HBM bytes of one launch of each pass kind: every array the pass
// must read or write, once (complex half spectrum = rows * xh * 8 bytes).
static double kind_bytes(const cubic_rl_plan_s *p, int kind)
{
    const double spec = (double)p->rows * p->xh * 8.0, real = (double)p->V * 4.0;
    switch (kind) {
    case KK_SUM: return real;
    case KK_FILL: return real;
    case KK_SHIFT: return 2 * real;
    case KK_X_FWD: return real + spec;
    case KK_X_INV: return spec + real;
    case KK_X_RATIO: return spec + real + spec;
    case KK_X_UPDATE: return spec + 2 * real + spec;
    case KK_X_FINAL: return spec + 2 * real;
    case KK_Y_FWD: case KK_Y_INV: case KK_Z_FWD: case KK_Z_INV: return 2 * spec;
    case KK_Z_CONV: case KK_Z_CORR: return 3 * spec;
    case KK_X_ACC_UPDATE: return spec + 4 * real;
    case KK_X_ACC_PREDICT: return 3 * real + spec;
    case KK_ACC_ALPHA: return 0.0;
    case KK_X_ADJOINT: return spec + 3 * real;  // each adjoint pass gives its own count
    }
    return 0.0;
}

static void prof_mark(cubic_rl_plan_s *p, int kind, cudaStream_t st)
{
    if (!p->prof || p->ev_used >= p->ev.size()) return;
    if (cudaEventRecord(p->ev[p->ev_used], st) == cudaSuccess) {
        p->ev_kind[p->ev_used] = kind;
        ++p->ev_used;
    }
}

// Run one launch of `kind`, counting it and (when profiling) bracketing it by events.
template <class F>
static cudaError_t counted(cubic_rl_plan_s *p, int kind, cudaStream_t st, F &&launch, double bytes = -1.0)
{
    const bool pair = p->prof && p->ev_used + 2 <= p->ev.size();
    if (pair) prof_mark(p, kind, st);
    cudaError_t e = launch();
    if (pair) prof_mark(p, kind, st);
    p->launches[kind] += 1;
    p->bytes[kind] += bytes >= 0.0 ? bytes : kind_bytes(p, kind);
    return e;
}

static const int kXKind[XM_COUNT] = {KK_X_FWD, KK_X_INV, KK_X_RATIO, KK_X_UPDATE, KK_X_FINAL};

static cudaError_t run_x(cubic_rl_plan_s *p, int mode, const XArgs &a, cudaStream_t st)
{
    return counted(p, kXKind[mode], st, [&] { return p->kx->xv[p->vx].fn[mode](a, st); });
}

// an X pass counted under another kind (the accelerated-RL forms of XM_FWD / XM_FINAL)
static cudaError_t run_x_as(cubic_rl_plan_s *p, int mode, int kind, const XArgs &a, double bytes, cudaStream_t st)
{
    return counted(p, kind, st, [&] { return p->kx->xv[p->vx].fn[mode](a, st); }, bytes);
}

// Failure-path test (cubic_test_skip_next_tile_copy): armed with a wait limit, the next
// Y launch of a TMA-pipelined variant takes it and has its CTA 0 skip its first tile copy.
static std::atomic<unsigned long long> g_skip_copy_ns{0};

static cudaError_t run_y(cubic_rl_plan_s *p, const YArgs &a, cudaStream_t st)
{
    const double bytes = 2.0 * 8.0 * (double)p->rows * (double)(a.col1 - a.col0);
    YArgs b = a;
    const YZVariant &yv = p->ky->yzv[p->vy];
    if (yv.tma && yv.B > 0 && g_skip_copy_ns.load(std::memory_order_relaxed)) {
        const unsigned long long ns = g_skip_copy_ns.exchange(0);
        if (ns) {
            b.wait_ns = ns;
            b.skip_first = 1;
        }
    }
    return counted(p, a.inverse ? KK_Y_INV : KK_Y_FWD, st, [&] { return p->ky->yzv[p->vy].y(b, st); }, bytes);
}

static cudaError_t run_z(cubic_rl_plan_s *p, const ZArgs &a, cudaStream_t st)
{
    static const int kind[5] = {KK_Z_FWD, KK_Z_CONV, KK_Z_CORR, KK_Z_INV, KK_Z_CONV};
    const double arrays = (a.mode == ZM_CONV || a.mode == ZM_CORR) ? 3.0 : a.mode == ZM_MUL_REAL ? 2.5 : 2.0;
    const double bytes = arrays * 8.0 * (double)p->rows * (double)(a.col1 - a.col0);
    return counted(p, kind[a.mode], st, [&] { return p->kz->yzv[p->vz].z(a, st); }, bytes);
}

// full: the whole transform box (H); otherwise the work geometry, where a linear plan's Y
// lines load their first iy rows (forward; the rest is zero padding) or store them (inverse)
static YArgs y_args(const cubic_rl_plan_s *p, float2 *spec, int inverse, int64_t c0, int64_t c1, bool full = false)
{
    YArgs a{spec, p->tw_y, full ? p->nz : work_planes(p), p->xh, p->xp, inverse, c0, c1, p->err};
    if (!full && p->linear && p->iy < p->ny) (inverse ? a.nstore : a.nload) = p->iy;
    a.wait_ns = p->wait_ns;
    return a;
}

// the spectral product of a convolution (ZM_CONV) or correlation (ZM_CORR); with a real
// H both are the same product
static int conv_mode(const cubic_rl_plan_s *p, int zmode)
{
    return (p->use_real_h && (zmode == ZM_CONV || zmode == ZM_CORR)) ? (int)ZM_MUL_REAL : zmode;
}

// a linear plan's Z lines have iz planes of data; the rest reads as zero and is not stored
static ZArgs z_args(const cubic_rl_plan_s *p, float2 *spec, int mode, float scale, int64_t c0, int64_t c1,
                    bool full = false)
{
    ZArgs a{spec, p->H, p->tw_z, p->ny, p->xh, p->xp, conv_mode(p, mode), scale, c0, c1, p->err, p->nz,
            p->use_real_h ? p->Hr : nullptr};
    if (!full && p->linear && p->iz < p->nz) a.nload = a.nstore = p->iz;
    a.wait_ns = p->wait_ns;
    return a;
}

// a linear plan's X rows are the image's (zero-padded to nx), mapped onto its spectrum rows
static XArgs x_args(const cubic_rl_plan_s *p, bool full = false)
{
    XArgs a{};
    a.tw = p->tw_x;
    a.rows = full ? p->nz * p->ny : work_planes(p) * work_ny(p);
    a.xp = p->xp;
    a.err = p->err;
    a.wait_ns = p->wait_ns;
    if (!full && p->linear && p->iy < p->ny) {
        a.ny_img = p->iy;
        a.ny_spec = p->ny;
    }
    return a;
}

// Forward 3D real-to-half-complex transform of `real` into `spec`, optionally
// scaled (scale applies in the Z pass).
static cubic_status_t enqueue_forward3(cubic_rl_plan_s *p, const float *real, float2 *spec, float scale,
                                       cudaStream_t st, bool full = false)
{
    XArgs xa = x_args(p, full);
    xa.spec_out = spec;
    xa.src = real;
    CUBIC_CUDA(run_x(p, XM_FWD, xa, st));
    CUBIC_CUDA(run_y(p, y_args(p, spec, 0, 0, p->xh, full), st));
    CUBIC_CUDA(run_z(p, z_args(p, spec, ZM_FWD_SCALE, scale, 0, p->xh, full), st));
    return CUBIC_OK;
}

// Y forward, Z (product with H or conj H), Y inverse on the plan's spectrum.
// With p->chunk > 0 the three passes run chunk by chunk over groups of
// p->chunk spectrum columns, so that a chunk written by one pass is still in
// L2 when the next pass reads it: per voxel, HBM then sees one read and one
// write of the spectrum (plus H) instead of three of each.
static cubic_status_t enqueue_yzy(cubic_rl_plan_s *p, float2 *spec, int zmode, cudaStream_t st)
{
    const int64_t step = p->chunk > 0 ? p->chunk : p->xh;
    for (int64_t c0 = 0; c0 < p->xh; c0 += step) {
        const int64_t c1 = c0 + step < p->xh ? c0 + step : p->xh;
        CUBIC_CUDA(run_y(p, y_args(p, spec, 0, c0, c1), st));
        CUBIC_CUDA(run_z(p, z_args(p, spec, zmode, 1.f, c0, c1), st));
        CUBIC_CUDA(run_y(p, y_args(p, spec, 1, c0, c1), st));
    }
    return CUBIC_OK;
}

// flag |= 1 unless h0(x) == h0(-x) for every x (bitwise): a point-symmetric PSF about
// its centre, whose spectrum is real
__global__ void k_check_even(const float *__restrict__ h0, int64_t nz, int64_t ny, int64_t nx, unsigned *flag)
{
    const int64_t V = nz * ny * nx;
    bool odd = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
        const int64_t j = (((nz - z) % nz) * ny + (ny - y) % ny) * nx + (nx - x) % nx;
        odd |= h0[i] != h0[j];
    }
    if (__syncthreads_or(odd) && threadIdx.x == 0) atomicOr(flag, 1u);
}

// Hr = Re H and Im H = 0 (the spectrum of an even PSF, with the rounding noise of
// the transform removed)
__global__ void k_real_h(float2 *__restrict__ H, float *__restrict__ Hr, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 h = H[i];
        Hr[i] = h.x;
        H[i] = make_float2(h.x, 0.f);
    }
}

// Places the PSF box (kz, ky, kx; peak at floor(k/2)) into the zeroed transform box h0
// (nz, ny, nx) with its peak at the origin, wrapping negative offsets: the same-mode
// convolution's kernel on the padded box.
__global__ void k_place_psf(const float *__restrict__ psf, int64_t kz, int64_t ky, int64_t kx,
                            float *__restrict__ h0, int64_t nz, int64_t ny, int64_t nx)
{
    const int64_t K = kz * ky * kx;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = i % kx, y = (i / kx) % ky, z = i / (kx * ky);
        const int64_t zz = ((z - kz / 2) % nz + nz) % nz, yy = ((y - ky / 2) % ny + ny) % ny,
                      xx = ((x - kx / 2) % nx + nx) % nx;
        h0[(zz * ny + yy) * nx + xx] = psf[i];
    }
}

static cubic_status_t load_psf(cubic_rl_plan_s *p, const float *psf, cudaStream_t st)
{
    cubic_status_t s = ensure_workspace(p);
    if (s != CUBIC_OK) return s;
    const int64_t Vt = p->nz * p->ny * p->nx;  // the transform box
    float *h0 = (float *)p->ws;
    if (p->linear) {
        // the work spectrum holds only the image's planes: a scratch box for h0
        void *m = nullptr;
        CUBIC_CUDA(cudaMallocAsync(&m, (size_t)Vt * sizeof(float), st));
        h0 = (float *)m;
        CUBIC_CUDA(cudaMemsetAsync(h0, 0, (size_t)Vt * sizeof(float), st));
        CUBIC_CUDA(counted(p, KK_SHIFT, st, [&] {
            k_place_psf<<<grid_for(p->pdims[0] * p->pdims[1] * p->pdims[2], 256), 256, 0, st>>>(
                psf, p->pdims[0], p->pdims[1], p->pdims[2], h0, p->nz, p->ny, p->nx);
            return cudaGetLastError();
        }));
    } else {
        // the shifted real PSF fits in the workspace (xp >= nx/2+1 complex >= nx floats)
        CUBIC_CUDA(counted(p, KK_SHIFT, st, [&] {
            k_center_to_origin<<<grid_for(p->V, 256), 256, 0, st>>>(psf, h0, p->nz, p->ny, p->nx);
            return cudaGetLastError();
        }));
    }
    bool even = false;
    if (p->allow_real_h) {
        // the reduction slot after the partial sums holds the flag for a moment
        unsigned *flag = (unsigned *)(p->partial + kReduceBlocks);
        CUBIC_CUDA(cudaMemsetAsync(flag, 0, sizeof(unsigned), st));
        k_check_even<<<grid_for(Vt, 256), 256, 0, st>>>(h0, p->nz, p->ny, p->nx, flag);
        unsigned host = 1;
        CUBIC_CUDA(cudaMemcpyAsync(&host, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        CUBIC_CUDA(cudaStreamSynchronize(st));
        even = host == 0;
    }
    p->use_real_h = false;  // H itself is complex while it is computed
    s = enqueue_forward3(p, h0, p->H, (float)(1.0 / (double)Vt), st, true);
    if (p->linear) CUBIC_CUDA(cudaFreeAsync(h0, st));
    if (s != CUBIC_OK || !even) return s;
    if (!p->Hr) {
        void *m = nullptr;
        CUBIC_CUDA(cudaMalloc(&m, h_elems(p) * sizeof(float)));
        p->Hr = (float *)m;
    }
    k_real_h<<<grid_for((int64_t)h_elems(p), 256), 256, 0, st>>>(p->H, p->Hr, (int64_t)h_elems(p));
    CUBIC_CUDA(cudaGetLastError());
    p->use_real_h = true;
    return CUBIC_OK;
}

// ------------------------------------------------------------------ tuning cache
// Chosen variants per volume shape, shared by every plan of this process and,
// when CUBIC_TUNE_CACHE names a file, persisted there as lines "nz ny nx vx vy vz".

struct TuneEntry {
    int64_t nz, ny, nx;
    int vx, vy, vz;
};
static std::mutex g_tune_mu;
static std::vector<TuneEntry> g_tune;
static bool g_tune_loaded = false;

static void tune_load_locked()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("CUBIC_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    TuneEntry e;
    long long a, b, c;
    while (fscanf(f, "%lld %lld %lld %d %d %d", &a, &b, &c, &e.vx, &e.vy, &e.vz) == 6) {
        e.nz = a;
        e.ny = b;
        e.nx = c;
        g_tune.push_back(e);
    }
    fclose(f);
}

static void tuned_variants(cubic_rl_plan_s *p)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    for (const TuneEntry &e : g_tune)
        if (e.nz == p->nz && e.ny == p->ny && e.nx == p->nx && e.vx < p->kx->nx && e.vy < p->ky->nyz &&
            e.vz < p->kz->nyz) {
            p->vx = e.vx;
            p->vy = e.vy;
            p->vz = e.vz;
        }
}

static void tune_store(const cubic_rl_plan_s *p)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    g_tune.push_back({p->nz, p->ny, p->nx, p->vx, p->vy, p->vz});
    const char *path = getenv("CUBIC_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%lld %lld %lld %d %d %d\n", (long long)p->nz, (long long)p->ny, (long long)p->nx, p->vx, p->vy,
            p->vz);
    fclose(f);
}

// Allocations, twiddles and H of a plan whose dims (and, for a linear plan, image dims and
// PSF box) are set; destroys it on failure.
static cubic_status_t plan_build(cubic_rl_plan_s *p, const float *psf, cudaStream_t st, cubic_rl_plan_t *plan)
{
    p->xh = p->nx / 2 + 1;
    p->xp = (p->xh + 15) / 16 * 16;
    p->kx = find_axis(p->nx);
    p->ky = find_axis(p->ny);
    p->kz = find_axis(p->nz);
    p->allow_real_h = true;

    cubic_status_t s = CUBIC_OK;
    auto bail = [&](cubic_status_t st_) {
        cubic_rl_plan_destroy(p);
        return st_;
    };
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) return bail(fail(CUBIC_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e)));
    void *mem = nullptr;
    e = cudaMalloc(&mem, h_elems(p) * sizeof(float2));
    if (e != cudaSuccess) return bail(fail(CUBIC_ERR_OUT_OF_MEMORY, "H: %s", cudaGetErrorString(e)));
    p->H = (float2 *)mem;
    const int64_t ntw = p->nx + p->ny + p->nz;
    e = cudaMalloc(&mem, ntw * sizeof(float2));
    if (e != cudaSuccess) return bail(fail(CUBIC_ERR_OUT_OF_MEMORY, "twiddles: %s", cudaGetErrorString(e)));
    p->tw = (float2 *)mem;
    p->tw_x = p->tw;
    p->tw_y = p->tw + p->nx;
    p->tw_z = p->tw + p->nx + p->ny;
    e = cudaMalloc(&mem, (kReduceBlocks + 1) * sizeof(double));
    if (e != cudaSuccess) return bail(fail(CUBIC_ERR_OUT_OF_MEMORY, "reduction: %s", cudaGetErrorString(e)));
    p->partial = (double *)mem;
    e = cudaMalloc(&mem, sizeof(unsigned));
    if (e != cudaSuccess) return bail(fail(CUBIC_ERR_OUT_OF_MEMORY, "error word: %s", cudaGetErrorString(e)));
    p->err = (unsigned *)mem;
    e = cudaMemsetAsync(p->err, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return bail(fail(CUBIC_ERR_CUDA, "error word: %s", cudaGetErrorString(e)));
    if (p->linear) {
        e = cudaMalloc(&mem, 2 * lin_elems(p) * sizeof(float));
        if (e != cudaSuccess) return bail(fail(CUBIC_ERR_OUT_OF_MEMORY, "padded arrays: %s", cudaGetErrorString(e)));
        p->lin = (float *)mem;
    }
    tuned_variants(p);

    k_twiddles<<<grid_for(p->nx, 128, 1 << 20), 128, 0, st>>>(p->tw_x, (int)p->nx);
    k_twiddles<<<grid_for(p->ny, 128, 1 << 20), 128, 0, st>>>(p->tw_y, (int)p->ny);
    k_twiddles<<<grid_for(p->nz, 128, 1 << 20), 128, 0, st>>>(p->tw_z, (int)p->nz);
    e = cudaGetLastError();
    if (e != cudaSuccess) return bail(fail(CUBIC_ERR_CUDA, "twiddles: %s", cudaGetErrorString(e)));
    s = load_psf(p, psf, st);
    if (s != CUBIC_OK) return bail(s);
    *plan = p;
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_plan(cubic_rl_plan_t *plan, const int64_t dims[3], const float *psf,
                                        unsigned flags, void *stream)
{
    if (!plan || !dims || !psf) return fail(CUBIC_ERR_INVALID_ARG, "plan, dims and psf must be non-null");
    *plan = nullptr;
    if (flags != 0) return fail(CUBIC_ERR_INVALID_ARG, "flags must be 0");
    for (int i = 0; i < 3; ++i)
        if (dims[i] < 1 || !find_axis(dims[i]))
            return fail(CUBIC_ERR_UNSUPPORTED_SIZE, "axis %d has unsupported length %lld", i, (long long)dims[i]);
    if (!aligned16(psf)) return fail(CUBIC_ERR_ALIGNMENT, "psf must be 16-byte aligned");
    if (dims[0] > 65535 || dims[1] > 65535)
        return fail(CUBIC_ERR_UNSUPPORTED_SIZE, "nz and ny must be <= 65535");

    cubic_rl_plan_s *p = new (std::nothrow) cubic_rl_plan_s();
    if (!p) return fail(CUBIC_ERR_OUT_OF_MEMORY, "host allocation failed");
    p->nz = dims[0];
    p->ny = dims[1];
    p->nx = dims[2];
    p->V = p->nz * p->ny * p->nx;
    p->rows = p->nz * p->ny;
    return plan_build(p, psf, (cudaStream_t)stream, plan);
}

// smallest supported transform length >= n (0: none)
static int64_t supported_at_least(int64_t n)
{
    for (int i = 0; i < kNumLengths; ++i)
        if (kLengths[i] >= n) return kLengths[i];
    return 0;
}

extern "C" cubic_status_t cubic_rl_plan_linear(cubic_rl_plan_t *plan, const int64_t dims[3],
                                               const int64_t psf_dims[3], const float *psf, unsigned flags,
                                               void *stream)
{
    if (!plan || !dims || !psf_dims || !psf) return fail(CUBIC_ERR_INVALID_ARG, "plan, dims, psf_dims, psf must be non-null");
    *plan = nullptr;
    if (flags != 0) return fail(CUBIC_ERR_INVALID_ARG, "flags must be 0");
    if (!aligned16(psf)) return fail(CUBIC_ERR_ALIGNMENT, "psf must be 16-byte aligned");
    int64_t m[3];
    for (int i = 0; i < 3; ++i) {
        if (dims[i] < 1 || psf_dims[i] < 1) return fail(CUBIC_ERR_INVALID_ARG, "dims and psf_dims must be >= 1");
        // "same" output reaches floor(k/2) past each edge; a box at least as long as the
        // PSF keeps its offsets from wrapping onto each other
        const int64_t need = std::max(dims[i] + psf_dims[i] / 2, psf_dims[i]);
        m[i] = supported_at_least(need);
        if (m[i] == 0)
            return fail(CUBIC_ERR_UNSUPPORTED_SIZE, "axis %d: no supported transform length >= %lld", i, (long long)need);
    }
    if (m[0] > 65535 || m[1] > 65535) return fail(CUBIC_ERR_UNSUPPORTED_SIZE, "nz and ny must be <= 65535");
    cubic_rl_plan_s *p = new (std::nothrow) cubic_rl_plan_s();
    if (!p) return fail(CUBIC_ERR_OUT_OF_MEMORY, "host allocation failed");
    p->linear = true;
    p->iz = dims[0];
    p->iy = dims[1];
    p->ix = dims[2];
    for (int i = 0; i < 3; ++i) p->pdims[i] = psf_dims[i];
    p->nz = m[0];
    p->ny = m[1];
    p->nx = m[2];
    p->V = p->iz * p->iy * p->ix;
    p->rows = p->iz * p->iy;
    return plan_build(p, psf, (cudaStream_t)stream, plan);
}

extern "C" cubic_status_t cubic_rl_plan_dims(cubic_rl_plan_t plan, int64_t image[3], int64_t transform[3])
{
    if (!plan) return fail(CUBIC_ERR_INVALID_ARG, "plan must be non-null");
    const int64_t im[3] = {plan->linear ? plan->iz : plan->nz, plan->linear ? plan->iy : plan->ny,
                           plan->linear ? plan->ix : plan->nx};
    for (int i = 0; i < 3; ++i) {
        if (image) image[i] = im[i];
        if (transform) transform[i] = i == 0 ? plan->nz : i == 1 ? plan->ny : plan->nx;
    }
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_plan_update_psf(cubic_rl_plan_t plan, const float *psf, void *stream)
{
    if (!plan || !psf) return fail(CUBIC_ERR_INVALID_ARG, "plan and psf must be non-null");
    if (!aligned16(psf)) return fail(CUBIC_ERR_ALIGNMENT, "psf must be 16-byte aligned");
    return load_psf(plan, psf, (cudaStream_t)stream);
}

extern "C" cubic_status_t cubic_rl_plan_destroy(cubic_rl_plan_t plan)
{
    if (!plan) return CUBIC_OK;
    cudaDeviceSynchronize();
    cudaFree(plan->H);
    cudaFree(plan->tw);
    cudaFree(plan->partial);
    cudaFree(plan->err);
    if (plan->own_ws) cudaFree(plan->ws);
    cudaFree(plan->stage_in);
    cudaFree(plan->stage_out);
    cudaFree(plan->bwd);
    cudaFree(plan->Hr);
    cudaFree(plan->ws2);
    cudaFree(plan->fsc_sums);
    cudaFree(plan->auto_stats);
    cudaFree(plan->auto_delta);
    cudaFree(plan->acc);
    cudaFree(plan->mon);
    cudaFree(plan->lin);
    for (cudaEvent_t e : plan->ev) cudaEventDestroy(e);
    delete plan;
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_workspace_bytes(cubic_rl_plan_t plan, size_t *bytes)
{
    if (!plan || !bytes) return fail(CUBIC_ERR_INVALID_ARG, "plan and bytes must be non-null");
    *bytes = spec_elems(plan) * sizeof(float2);
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_set_workspace(cubic_rl_plan_t plan, void *dev_ptr, size_t bytes)
{
    if (!plan || !dev_ptr) return fail(CUBIC_ERR_INVALID_ARG, "plan and dev_ptr must be non-null");
    if (((uintptr_t)dev_ptr & 255u) != 0) return fail(CUBIC_ERR_ALIGNMENT, "workspace must be 256-byte aligned");
    if (bytes < spec_elems(plan) * sizeof(float2))
        return fail(CUBIC_ERR_INVALID_ARG, "workspace too small: %zu < %zu", bytes, spec_elems(plan) * sizeof(float2));
    if (plan->own_ws) {
        cudaDeviceSynchronize();
        cudaFree(plan->ws);
    }
    plan->ws = (float2 *)dev_ptr;
    plan->own_ws = false;
    return CUBIC_OK;
}

static bool overlaps(const void *a, const void *b, size_t n)
{
    const char *x = (const char *)a, *y = (const char *)b;
    return x < y + n && y < x + n;
}

// [a, a + na) and [b, b + nb) share a byte
static bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const char *x = (const char *)a, *y = (const char *)b;
    return x < y + nb && y < x + na;
}

// u0 = max(mean(image), eps) into out.
static cubic_status_t enqueue_init(cubic_rl_plan_s *p, const float *image, float eps, float *out, cudaStream_t st)
{
    CUBIC_CUDA(counted(p, KK_SUM, st, [&] {
        k_sum_partial<<<kReduceBlocks, kReduceThreads, 0, st>>>(image, p->V, p->partial);
        k_sum_final<<<1, kReduceThreads, 0, st>>>(p->partial, kReduceBlocks, p->partial + kReduceBlocks);
        return cudaGetLastError();
    }));
    p->launches[KK_SUM] += 1;  // two kernels
    CUBIC_CUDA(counted(p, KK_FILL, st, [&] {
        k_fill_initial<<<grid_for(p->V, 256), 256, 0, st>>>(out, p->V, p->partial + kReduceBlocks, eps);
        return cudaGetLastError();
    }));
    return CUBIC_OK;
}

// ------------------------------------------------------------------ linear boundaries
// A linear plan runs the same passes on rows zero-padded to the transform length: the
// padded image has d = 0 there, so r = 0 there, and the estimate starts and stays at 0
// there (u q with u = 0), which is exactly "same"-mode convolution with zero padding.

// rows of nin values -> rows of nout >= nin values, zero past nin
__global__ void k_pad_rows(const float *__restrict__ in, float *__restrict__ out, int64_t rows, int64_t nin,
                           int64_t nout)
{
    const int64_t n = rows * nout;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / nout, x = i - r * nout;
        out[i] = x < nin ? in[r * nin + x] : 0.f;
    }
}

// rows of nin values -> their first nout values
__global__ void k_crop_rows(const float *__restrict__ in, float *__restrict__ out, int64_t rows, int64_t nin,
                            int64_t nout)
{
    const int64_t n = rows * nout;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / nout, x = i - r * nout;
        out[i] = in[r * nin + x];
    }
}

// x_0 = max(sum / V, eps) on the first nvalid values of each padded row, 0 past them
__global__ void k_fill_padded(float *__restrict__ u, int64_t rows, int64_t nvalid, int64_t n,
                              const double *__restrict__ sum, int64_t V, float eps)
{
    const float v = initial_value_block(sum, V, eps);
    const int64_t total = rows * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        u[i] = (i % n) < nvalid ? v : 0.f;
}

static cubic_status_t lin_pad(cubic_rl_plan_s *p, const float *in, float *out_padded, cudaStream_t st)
{
    const int64_t R = p->iz * p->iy, E = (int64_t)lin_elems(p);
    CUBIC_CUDA(counted(p, KK_SHIFT, st, [&] {
        k_pad_rows<<<grid_for(E, 256), 256, 0, st>>>(in, out_padded, R, p->ix, p->nx);
        return cudaGetLastError();
    }, 4.0 * (double)(p->V + E)));
    return CUBIC_OK;
}

static cubic_status_t lin_crop(cubic_rl_plan_s *p, const float *padded, float *out, cudaStream_t st)
{
    const int64_t R = p->iz * p->iy;
    CUBIC_CUDA(counted(p, KK_SHIFT, st, [&] {
        k_crop_rows<<<grid_for(p->V, 256), 256, 0, st>>>(padded, out, R, p->nx, p->ix);
        return cudaGetLastError();
    }, 8.0 * (double)p->V));
    return CUBIC_OK;
}

static cubic_status_t enqueue_yzy(cubic_rl_plan_s *p, float2 *spec, int zmode, cudaStream_t st);

// A linear plan's start: the image padded into dp, and the estimate x_0 = max(mean, eps)
// on its box (zero padding elsewhere) in up; the mean is over the image's voxels, to which
// the padding adds nothing.
static cubic_status_t lin_init(cubic_rl_plan_s *p, const float *image, float eps, float *dp, float *up,
                               cudaStream_t st)
{
    const int64_t R = p->iz * p->iy, E = (int64_t)lin_elems(p);
    cubic_status_t s = lin_pad(p, image, dp, st);
    if (s != CUBIC_OK) return s;
    CUBIC_CUDA(counted(p, KK_SUM, st, [&] {
        k_sum_partial<<<kReduceBlocks, kReduceThreads, 0, st>>>(dp, E, p->partial);
        k_sum_final<<<1, kReduceThreads, 0, st>>>(p->partial, kReduceBlocks, p->partial + kReduceBlocks);
        return cudaGetLastError();
    }));
    CUBIC_CUDA(counted(p, KK_FILL, st, [&] {
        k_fill_padded<<<grid_for(E, 256), 256, 0, st>>>(up, R, p->ix, p->nx, p->partial + kReduceBlocks, p->V, eps);
        return cudaGetLastError();
    }));
    return CUBIC_OK;
}

// RL of a linear plan: the image and the estimate live in the plan's padded arrays
static cubic_status_t enqueue_rl_linear(cubic_rl_plan_s *p, const float *image, int n_iter, float eps, float *out,
                                       float2 *spec, cudaStream_t st)
{
    float *dp = p->lin, *up = p->lin + lin_elems(p);
    cubic_status_t s = lin_init(p, image, eps, dp, up, st);
    if (s != CUBIC_OK) return s;
    if (n_iter > 0) {
        XArgs xa = x_args(p);
        xa.spec_in = spec;
        xa.spec_out = spec;
        xa.src = up;
        xa.u = up;
        xa.dst = up;
        xa.d = dp;
        xa.eps = eps;
        CUBIC_CUDA(run_x(p, XM_FWD, xa, st));
        for (int k = 0; k < n_iter; ++k) {
            if ((s = enqueue_yzy(p, spec, ZM_CONV, st)) != CUBIC_OK) return s;
            CUBIC_CUDA(run_x(p, XM_RATIO, xa, st));
            if ((s = enqueue_yzy(p, spec, ZM_CORR, st)) != CUBIC_OK) return s;
            CUBIC_CUDA(run_x(p, k + 1 < n_iter ? XM_UPDATE : XM_FINAL, xa, st));
        }
    }
    return lin_crop(p, up, out, st);
}

static cubic_status_t no_linear(const cubic_rl_plan_s *p, const char *what)
{
    return p->linear ? fail(CUBIC_ERR_INVALID_ARG, "%s is not available for linear-boundary plans", what)
                     : CUBIC_OK;
}

// The n_iter-iteration sequence, enqueued on `st`.
static cubic_status_t enqueue_rl(cubic_rl_plan_s *p, const float *image, int n_iter, float eps, float *out,
                                 float2 *spec, cudaStream_t st)
{
    if (p->linear) return enqueue_rl_linear(p, image, n_iter, eps, out, spec, st);
    cubic_status_t s0 = enqueue_init(p, image, eps, out, st);
    if (s0 != CUBIC_OK) return s0;
    if (n_iter == 0) return CUBIC_OK;

    XArgs xa = x_args(p);
    xa.spec_in = spec;
    xa.spec_out = spec;
    xa.src = out;
    xa.u = out;
    xa.dst = out;
    xa.d = image;
    xa.eps = eps;
    CUBIC_CUDA(run_x(p, XM_FWD, xa, st));  // spectrum of u0
    cubic_status_t s;
    for (int k = 0; k < n_iter; ++k) {
        if ((s = enqueue_yzy(p, spec, ZM_CONV, st)) != CUBIC_OK) return s;   // b = h * u
        CUBIC_CUDA(run_x(p, XM_RATIO, xa, st));                              // r = d / max(b, eps)
        if ((s = enqueue_yzy(p, spec, ZM_CORR, st)) != CUBIC_OK) return s;   // q = h (flipped) * r
        CUBIC_CUDA(run_x(p, k + 1 < n_iter ? XM_UPDATE : XM_FINAL, xa, st)); // u = u * q
    }
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_deconvolve(cubic_rl_plan_t plan, const float *image, int n_iter, float eps,
                                              float *out, void *stream)
{
    if (!plan || !image || !out) return fail(CUBIC_ERR_INVALID_ARG, "plan, image and out must be non-null");
    if (n_iter < 0) return fail(CUBIC_ERR_INVALID_ARG, "n_iter must be >= 0");
    if (!(eps > 0.f) || !(eps < INFINITY)) return fail(CUBIC_ERR_INVALID_ARG, "eps must be finite and > 0");
    if (!aligned16(image) || !aligned16(out)) return fail(CUBIC_ERR_ALIGNMENT, "image and out must be 16-byte aligned");
    if (overlaps(image, out, (size_t)plan->V * sizeof(float)))
        return fail(CUBIC_ERR_INVALID_ARG, "out must not overlap image");
    cubic_status_t s = ensure_workspace(plan);
    if (s != CUBIC_OK) return s;
    return enqueue_rl(plan, image, n_iter, eps, out, plan->ws, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ building blocks

extern "C" cubic_status_t cubic_rl_convolve(cubic_rl_plan_t plan, const float *in, int flipped, float *out,
                                            void *stream)
{
    if (!plan || !in || !out) return fail(CUBIC_ERR_INVALID_ARG, "plan, in and out must be non-null");
    if (!aligned16(in) || !aligned16(out)) return fail(CUBIC_ERR_ALIGNMENT, "in and out must be 16-byte aligned");
    cubic_status_t s = ensure_workspace(plan);
    if (s != CUBIC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    XArgs xa = x_args(plan);
    xa.spec_in = plan->ws;
    xa.spec_out = plan->ws;
    xa.src = in;
    xa.dst = out;
    if (plan->linear) {  // through the padded arrays
        if ((s = lin_pad(plan, in, plan->lin, st)) != CUBIC_OK) return s;
        xa.src = plan->lin;
        xa.dst = plan->lin + lin_elems(plan);
    }
    CUBIC_CUDA(run_x(plan, XM_FWD, xa, st));
    if ((s = enqueue_yzy(plan, plan->ws, flipped ? ZM_CORR : ZM_CONV, st)) != CUBIC_OK) return s;
    CUBIC_CUDA(run_x(plan, XM_INV, xa, st));
    if (plan->linear) return lin_crop(plan, plan->lin + lin_elems(plan), out, st);
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_spectrum_layout(cubic_rl_plan_t plan, int64_t *xh, int64_t *xp)
{
    if (!plan) return fail(CUBIC_ERR_INVALID_ARG, "plan must be non-null");
    if (xh) *xh = plan->xh;
    if (xp) *xp = plan->xp;
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_fft3_forward(cubic_rl_plan_t plan, const float *in, void *spec, void *stream)
{
    if (!plan || !in || !spec) return fail(CUBIC_ERR_INVALID_ARG, "plan, in and spec must be non-null");
    if (cubic_status_t g = no_linear(plan, "the spectrum entry point")) return g;
    if (!aligned16(in) || !aligned16(spec)) return fail(CUBIC_ERR_ALIGNMENT, "in and spec must be 16-byte aligned");
    return enqueue_forward3(plan, in, (float2 *)spec, 1.f, (cudaStream_t)stream);
}

extern "C" cubic_status_t cubic_rl_fft3_inverse(cubic_rl_plan_t plan, void *spec, float *out, void *stream)
{
    if (!plan || !out || !spec) return fail(CUBIC_ERR_INVALID_ARG, "plan, spec and out must be non-null");
    if (cubic_status_t g = no_linear(plan, "the spectrum entry point")) return g;
    if (!aligned16(out) || !aligned16(spec)) return fail(CUBIC_ERR_ALIGNMENT, "out and spec must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    float2 *sp = (float2 *)spec;
    CUBIC_CUDA(run_z(plan, z_args(plan, sp, ZM_INV_SCALE, (float)(1.0 / (double)plan->V), 0, plan->xh), st));
    CUBIC_CUDA(run_y(plan, y_args(plan, sp, 1, 0, plan->xh), st));
    XArgs xa = x_args(plan);
    xa.spec_in = sp;
    xa.dst = out;
    CUBIC_CUDA(run_x(plan, XM_INV, xa, st));
    return CUBIC_OK;
}

// ------------------------------------------------------------------ host buffers

extern "C" cubic_status_t cubic_rl_deconvolve_host(cubic_rl_plan_t plan, const float *image, int n_iter, float eps,
                                                   float *out, void *stream)
{
    if (!plan || !image || !out) return fail(CUBIC_ERR_INVALID_ARG, "plan, image and out must be non-null");
    if (n_iter < 0) return fail(CUBIC_ERR_INVALID_ARG, "n_iter must be >= 0");
    if (!(eps > 0.f) || !(eps < INFINITY)) return fail(CUBIC_ERR_INVALID_ARG, "eps must be finite and > 0");
    const size_t nbytes = (size_t)plan->V * sizeof(float);
    if (overlaps(image, out, nbytes)) return fail(CUBIC_ERR_INVALID_ARG, "out must not overlap image");
    cubic_status_t s = ensure_workspace(plan);
    if (s != CUBIC_OK) return s;
    if (!plan->stage_in) {
        void *a = nullptr, *b = nullptr;
        CUBIC_CUDA(cudaMalloc(&a, nbytes));
        cudaError_t e = cudaMalloc(&b, nbytes);
        if (e != cudaSuccess) {
            cudaFree(a);
            return fail(CUBIC_ERR_OUT_OF_MEMORY, "staging: %s", cudaGetErrorString(e));
        }
        plan->stage_in = (float *)a;
        plan->stage_out = (float *)b;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CUBIC_CUDA(cudaMemcpyAsync(plan->stage_in, image, nbytes, cudaMemcpyHostToDevice, st));
    s = enqueue_rl(plan, plan->stage_in, n_iter, eps, plan->stage_out, plan->ws, st);
    if (s != CUBIC_OK) return s;
    CUBIC_CUDA(cudaMemcpyAsync(out, plan->stage_out, nbytes, cudaMemcpyDeviceToHost, st));
    return CUBIC_OK;
}

// ------------------------------------------------------------------ profiling

extern "C" int cubic_rl_kernel_kinds(void) { return KK_COUNT; }

extern "C" const char *cubic_rl_kernel_name(int kind)
{
    return (kind >= 0 && kind < KK_COUNT) ? kKindNames[kind] : "";
}

extern "C" cubic_status_t cubic_rl_profile(cubic_rl_plan_t plan, int enable, int max_events)
{
    if (!plan) return fail(CUBIC_ERR_INVALID_ARG, "plan must be non-null");
    for (int k = 0; k < KK_COUNT; ++k) {
        plan->launches[k] = 0;
        plan->bytes[k] = 0.0;
    }
    plan->ev_used = 0;
    plan->prof = enable != 0;
    if (enable) {
        if (max_events < 2) max_events = 2;
        while ((int)plan->ev.size() < max_events) {
            cudaEvent_t e;
            CUBIC_CUDA(cudaEventCreate(&e));
            plan->ev.push_back(e);
        }
        plan->ev_kind.assign(plan->ev.size(), 0);
    }
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_profile_read(cubic_rl_plan_t plan, int n_kinds, double *total_ms,
                                                int64_t *timed_launches, int64_t *launches, double *bytes)
{
    if (!plan || n_kinds < 0) return fail(CUBIC_ERR_INVALID_ARG, "bad arguments");
    const int nk = n_kinds < KK_COUNT ? n_kinds : KK_COUNT;
    for (int k = 0; k < nk; ++k) {
        if (total_ms) total_ms[k] = 0.0;
        if (timed_launches) timed_launches[k] = 0;
        if (launches) launches[k] = plan->launches[k];
        if (bytes) bytes[k] = plan->bytes[k];
    }
    if (plan->ev_used >= 2) CUBIC_CUDA(cudaEventSynchronize(plan->ev[plan->ev_used - 1]));
    for (size_t i = 0; i + 1 < plan->ev_used; i += 2) {
        float ms = 0.f;
        CUBIC_CUDA(cudaEventElapsedTime(&ms, plan->ev[i], plan->ev[i + 1]));
        const int k = plan->ev_kind[i];
        if (k < nk) {
            if (total_ms) total_ms[k] += ms;
            if (timed_launches) timed_launches[k] += 1;
        }
    }
    return CUBIC_OK;
}

// ------------------------------------------------------------------ Gaussian PSF

// g = exp(-(dx^2+dy^2) a_xy - dz^2 a_z), (dx,dy,dz) = index - floor(n/2); block partial
// sums of g in double (the PSF's flux) for the normalisation.
__global__ void __launch_bounds__(kReduceThreads) k_psf_gauss(float *__restrict__ psf, int64_t nz, int64_t ny,
                                                              int64_t nx, float a_xy, float a_z,
                                                              double *__restrict__ partial)
{
    __shared__ double sh[kReduceThreads / 32];
    const int64_t V = nz * ny * nx;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
        const float dx = (float)(i % nx - nx / 2);
        const float dy = (float)((i / nx) % ny - ny / 2);
        const float dz = (float)(i / (nx * ny) - nz / 2);
        const float g = expf(-(dx * dx + dy * dy) * a_xy - dz * dz * a_z);
        psf[i] = g;
        s += (double)g;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < kReduceThreads / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) partial[blockIdx.x] = s;
    }
}

__global__ void k_scale_by_sum(float *__restrict__ x, int64_t n, const double *__restrict__ sum, double amp)
{
    const float f = (float)(amp / sum[0]);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] *= f;
}

extern "C" cubic_status_t cubic_psf_gaussian(const int64_t dims[3], float sigma_xy, float sigma_z, float amp,
                                             float *psf, void *stream)
{
    if (!dims || !psf) return fail(CUBIC_ERR_INVALID_ARG, "dims and psf must be non-null");
    for (int i = 0; i < 3; ++i)
        if (dims[i] < 1) return fail(CUBIC_ERR_INVALID_ARG, "dims must be >= 1");
    if (!(sigma_xy > 0.f) || !(sigma_z > 0.f) || !(sigma_xy < INFINITY) || !(sigma_z < INFINITY) ||
        !(fabsf(amp) < INFINITY))
        return fail(CUBIC_ERR_INVALID_ARG, "sigmas must be finite and > 0, amp finite");
    if (!aligned16(psf)) return fail(CUBIC_ERR_ALIGNMENT, "psf must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t V = dims[0] * dims[1] * dims[2];
    void *scratch = nullptr;
    CUBIC_CUDA(cudaMallocAsync(&scratch, (kReduceBlocks + 1) * sizeof(double), st));
    double *partial = (double *)scratch;
    const float a_xy = (float)(0.5 / ((double)sigma_xy * sigma_xy));
    const float a_z = (float)(0.5 / ((double)sigma_z * sigma_z));
    k_psf_gauss<<<kReduceBlocks, kReduceThreads, 0, st>>>(psf, dims[0], dims[1], dims[2], a_xy, a_z, partial);
    k_sum_final<<<1, kReduceThreads, 0, st>>>(partial, kReduceBlocks, partial + kReduceBlocks);
    k_scale_by_sum<<<grid_for(V, 256), 256, 0, st>>>(psf, V, partial + kReduceBlocks, (double)amp);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return fail(CUBIC_ERR_CUDA, "psf kernels: %s", cudaGetErrorString(e));
    return CUBIC_OK;
}

// ------------------------------------------------------------------ variants and tuning

extern "C" cubic_status_t cubic_rl_plan_variants(cubic_rl_plan_t plan, int counts[3], int chosen[3])
{
    if (!plan) return fail(CUBIC_ERR_INVALID_ARG, "plan must be non-null");
    if (counts) {
        counts[0] = plan->kx->nx;
        counts[1] = plan->ky->nyz;
        counts[2] = plan->kz->nyz;
    }
    if (chosen) {
        chosen[0] = plan->vx;
        chosen[1] = plan->vy;
        chosen[2] = plan->vz;
    }
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_plan_set_variants(cubic_rl_plan_t plan, int vx, int vy, int vz)
{
    if (!plan) return fail(CUBIC_ERR_INVALID_ARG, "plan must be non-null");
    if (vx < 0 || vx >= plan->kx->nx || vy < 0 || vy >= plan->ky->nyz || vz < 0 || vz >= plan->kz->nyz)
        return fail(CUBIC_ERR_INVALID_ARG, "variant index out of range");
    plan->vx = vx;
    plan->vy = vy;
    plan->vz = vz;
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_plan_set_chunk(cubic_rl_plan_t plan, int64_t columns)
{
    if (!plan) return fail(CUBIC_ERR_INVALID_ARG, "plan must be non-null");
    if (columns < 0 || columns % 16 != 0) return fail(CUBIC_ERR_INVALID_ARG, "chunk must be a multiple of 16 (0: off)");
    plan->chunk = columns;
    return CUBIC_OK;
}

extern "C" int64_t cubic_rl_plan_chunk(cubic_rl_plan_t plan) { return plan ? plan->chunk : -1; }

// Best-of-3 device time of `body` (after one untimed run); `prepare` runs,
// untimed, before every run.
template <class G, class F>
static cubic_status_t time_best(cudaStream_t st, G &&prepare, F &&body, float *best_ms)
{
    cudaEvent_t e0, e1;
    CUBIC_CUDA(cudaEventCreate(&e0));
    CUBIC_CUDA(cudaEventCreate(&e1));
    cubic_status_t s = prepare();
    if (s == CUBIC_OK) s = body();
    float best = 1e30f;
    for (int r = 0; r < 5 && s == CUBIC_OK; ++r) {
        s = prepare();
        if (s != CUBIC_OK) break;
        cudaEventRecord(e0, st);
        s = body();
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) s = fail(CUBIC_ERR_CUDA, "tuning sync failed");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *best_ms = best;
    return s;
}

extern "C" cubic_status_t cubic_rl_autotune(cubic_rl_plan_t plan, const float *image, float *out, void *stream)
{
    if (!plan || !image || !out) return fail(CUBIC_ERR_INVALID_ARG, "plan, image and out must be non-null");
    if (!aligned16(image) || !aligned16(out)) return fail(CUBIC_ERR_ALIGNMENT, "image and out must be 16-byte aligned");
    if (overlaps(image, out, (size_t)plan->V * sizeof(float)))
        return fail(CUBIC_ERR_INVALID_ARG, "out must not overlap image");
    cubic_status_t s = ensure_workspace(plan);
    if (s != CUBIC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const bool prof = plan->prof;
    plan->prof = false;
    float2 *ws = plan->ws;
    // a linear plan tunes on its padded arrays
    const float *img_w = plan->linear ? plan->lin : image;
    float *out_w = plan->linear ? plan->lin + lin_elems(plan) : out;
    const size_t nw = plan->linear ? lin_elems(plan) : (size_t)plan->V;
    // every timed run starts from the spectrum of the image and a copy of it as estimate
    auto prepare = [&]() -> cubic_status_t {
        if (plan->linear) {
            cubic_status_t sp = lin_pad(plan, image, plan->lin, st);
            if (sp != CUBIC_OK) return sp;
        }
        CUBIC_CUDA(cudaMemcpyAsync(out_w, img_w, nw * sizeof(float), cudaMemcpyDeviceToDevice, st));
        return enqueue_forward3(plan, img_w, ws, 1.f / (float)plan->V, st);
    };
    auto nothing = []() -> cubic_status_t { return CUBIC_OK; };
    float best, ms;
    // X pass: one ratio and one update launch
    int bx = plan->vx;
    best = 1e30f;
    for (int v = 0; v < plan->kx->nx && s == CUBIC_OK; ++v) {
        plan->vx = v;
        XArgs xa = x_args(plan);
        xa.spec_in = ws;
        xa.spec_out = ws;
        xa.u = out_w;
        xa.d = img_w;
        xa.eps = 1.f;
        s = time_best(st, prepare, [&]() -> cubic_status_t {
            CUBIC_CUDA(run_x(plan, XM_RATIO, xa, st));
            CUBIC_CUDA(run_x(plan, XM_UPDATE, xa, st));
            return CUBIC_OK;
        }, &ms);
        if (ms < best) { best = ms; bx = v; }
    }
    plan->vx = bx;
    // Y pass: forward + inverse
    int by = plan->vy;
    best = 1e30f;
    for (int v = 0; v < plan->ky->nyz && s == CUBIC_OK; ++v) {
        plan->vy = v;
        YArgs ya = y_args(plan, ws, 0, 0, plan->xh);
        s = time_best(st, nothing, [&]() -> cubic_status_t {
            ya.inverse = 0;
            CUBIC_CUDA(run_y(plan, ya, st));
            ya.inverse = 1;
            CUBIC_CUDA(run_y(plan, ya, st));
            return CUBIC_OK;
        }, &ms);
        if (ms < best) { best = ms; by = v; }
    }
    plan->vy = by;
    // Z pass: spectral product with H
    int bz = plan->vz;
    best = 1e30f;
    for (int v = 0; v < plan->kz->nyz && s == CUBIC_OK; ++v) {
        plan->vz = v;
        ZArgs za = z_args(plan, ws, ZM_CONV, 1.f, 0, plan->xh);
        s = time_best(st, nothing, [&]() -> cubic_status_t {
            CUBIC_CUDA(run_z(plan, za, st));
            return CUBIC_OK;
        }, &ms);
        if (ms < best) { best = ms; bz = v; }
    }
    plan->vz = bz;
    plan->prof = prof;
    if (s == CUBIC_OK) s = prepare();  // leave finite data behind
    if (s == CUBIC_OK && plan->linear) s = lin_crop(plan, out_w, out, st);
    if (s != CUBIC_OK) return s;
    tune_store(plan);
    return CUBIC_OK;
}

// ------------------------------------------------------------------ device status

extern "C" cubic_status_t cubic_rl_stream_status(cubic_rl_plan_t plan, void *stream)
{
    if (!plan) return fail(CUBIC_ERR_INVALID_ARG, "plan must be non-null");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned word = 0;
    CUBIC_CUDA(cudaMemcpyAsync(&word, plan->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CUBIC_CUDA(cudaStreamSynchronize(st));
    if (word) {
        CUBIC_CUDA(cudaMemsetAsync(plan->err, 0, sizeof(unsigned), st));
        return fail(CUBIC_ERR_TIMEOUT, "a device wait timed out (error word 0x%x)", word);
    }
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_plan_set_wait_limit(cubic_rl_plan_t plan, uint64_t limit_ns)
{
    if (!plan) return fail(CUBIC_ERR_INVALID_ARG, "plan must be non-null");
    plan->wait_ns = limit_ns;
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_test_skip_next_tile_copy(uint64_t wait_ns)
{
    g_skip_copy_ns.store(wait_ns);  // 0 disarms
    return CUBIC_OK;
}

// ------------------------------------------------------------------ differentiation
//
// Reverse mode through n_iter Richardson-Lucy iterations.  One iteration,
//   b = h * u,  c = max(b, eps),  r = d / c,  q = h (x) r,  u' = u q,
// has the adjoint (g = dL/du'):
//   qbar = g u;  ubar = g q + h (x) bbar;  rbar = h * qbar;
//   dbar += rbar / c;  bbar = -rbar d / c^2 [b > eps];
//   dL/dh0 += bbar (x) u + r (x) qbar  ->  spectrum  G += Bbar conj(U) + conj(Qbar) R,
// where * is the circular convolution and (x) the correlation (convolution with the
// flipped PSF).  The forward stores u every `ckpt_every` iterations; the backward
// recomputes each segment from its checkpoint, keeping u, b, r and q of every
// iteration of the segment, then walks the segment backwards.

// Compensated float32 sum of x over V elements: block partials (CFloat) ...
__global__ void __launch_bounds__(kReduceThreads) k_csum_partial(const float *__restrict__ x, int64_t V,
                                                                 CFloat *__restrict__ partial)
{
    __shared__ CFloat sh[kReduceThreads / 32];
    CFloat s{0.f, 0.f};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x)
        s = cf_add(s, x[i]);
    for (int o = 16; o > 0; o >>= 1)
        s = cf_merge(s, CFloat{__shfl_down_sync(0xffffffffu, s.s, o), __shfl_down_sync(0xffffffffu, s.c, o)});
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        CFloat t{0.f, 0.f};
        for (int w = 0; w < kReduceThreads / 32; ++w) t = cf_merge(t, sh[w]);
        partial[blockIdx.x] = t;
    }
}

// ... merged in a fixed order into *out
__global__ void k_csum_final(const CFloat *__restrict__ partial, int n, float *__restrict__ out)
{
    if (threadIdx.x != 0) return;
    CFloat t{0.f, 0.f};
    for (int i = 0; i < n; ++i) t = cf_merge(t, partial[i]);
    out[0] = t.s - t.c;
}

// dbar += sum(g) / V where mean(d) > eps (u0 = max(mean(d), eps)); sum_d is the
// FP64 flux sum of the image, sum_g a compensated float32 sum
__global__ void k_add_mean_grad(float *__restrict__ dbar, const float *__restrict__ sum_g,
                                const double *__restrict__ sum_d, int64_t V, float eps)
{
    const bool pass = sum_d[0] / (double)V > (double)eps;
    const float add = pass ? sum_g[0] / (float)V : 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x)
        dbar[i] += add;
}

// p(x) = h0(x - floor(n/2)) (+= p when accumulate): PSF gradient back to centred indexing
__global__ void k_origin_to_center(const float *__restrict__ h0, float *__restrict__ p, int64_t nz, int64_t ny,
                                   int64_t nx, int accumulate)
{
    const int64_t V = nz * ny * nx;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
        int64_t xs = x + nx / 2, ys = y + ny / 2, zs = z + nz / 2;
        if (xs >= nx) xs -= nx;
        if (ys >= ny) ys -= ny;
        if (zs >= nz) zs -= nz;
        const int64_t j = (zs * ny + ys) * nx + xs;
        p[j] = accumulate ? p[j] + h0[i] : h0[i];
    }
}

// Unnormalised (scale = 1) or normalised (scale = 1/V) inverse 3D transform of a half spectrum.
static cubic_status_t enqueue_inverse3(cubic_rl_plan_s *p, float2 *spec, float *out, float scale, cudaStream_t st)
{
    CUBIC_CUDA(run_z(p, z_args(p, spec, ZM_INV_SCALE, scale, 0, p->xh), st));
    CUBIC_CUDA(run_y(p, y_args(p, spec, 1, 0, p->xh), st));
    XArgs xa = x_args(p);
    xa.spec_in = spec;
    xa.dst = out;
    CUBIC_CUDA(run_x(p, XM_INV, xa, st));
    return CUBIC_OK;
}

// Recompute iterations k0 .. k0+cnt-1 from u_k0 = seg_u[0], keeping u, b, r, q per iteration.
// The plain (non-TMA) Z launch shape of the plan's z length: the reverse sweep's extras
// (saved spectra, PSF-gradient accumulation) exist only there.
// The widest plain variant (most threads per CTA) is taken.
static cudaError_t run_z_plain(cubic_rl_plan_s *p, const ZArgs &a, cudaStream_t st)
{
    static const int kind[5] = {KK_Z_FWD, KK_Z_CONV, KK_Z_CORR, KK_Z_INV, KK_Z_CONV};
    int best = -1;
    for (int v = 0; v < p->kz->nyz; ++v) {
        const YZVariant &y = p->kz->yzv[v];
        if (!y.tma && (best < 0 || y.P * y.B > p->kz->yzv[best].P * p->kz->yzv[best].B)) best = v;
    }
    if (best < 0) return cudaErrorNotSupported;
    return counted(p, kind[a.mode], st, [&] { return p->kz->yzv[best].z(a, st); });
}

// Y forward, the plain Z product (saving its z-transformed input to `save`, and adding
// conj(V) other or V conj(other) into `gacc`), Y inverse
static cubic_status_t enqueue_yzy_grad(cubic_rl_plan_s *p, float2 *spec, int zmode, float2 *save, float2 *gacc,
                                       const float2 *other, int gconj, cudaStream_t st)
{
    CUBIC_CUDA(run_y(p, y_args(p, spec, 0, 0, p->xh), st));
    ZArgs za = z_args(p, spec, zmode, 1.f, 0, p->xh);
    za.save = save;
    za.gacc = gacc;
    za.gother = other;
    za.gconj = gconj;
    CUBIC_CUDA(run_z_plain(p, za, st));
    CUBIC_CUDA(run_y(p, y_args(p, spec, 1, 0, p->xh), st));
    return CUBIC_OK;
}

// Recomputes cnt iterations from seg_u[0], keeping u, b, r, q of each and, when seg_U /
// seg_R are given, the spectra U = DFT(u) and R = DFT(r) that the convolutions form anyway.
static cubic_status_t enqueue_segment(cubic_rl_plan_s *p, const float *image, float eps, int cnt, float *const *seg_u,
                                      float *const *seg_b, float *const *seg_r, float *const *seg_q, float2 *spec,
                                      cudaStream_t st, float2 *const *seg_U = nullptr, float2 *const *seg_R = nullptr)
{
    XArgs xa = x_args(p);
    xa.spec_in = spec;
    xa.spec_out = spec;
    xa.src = seg_u[0];
    xa.d = image;
    xa.eps = eps;
    CUBIC_CUDA(run_x(p, XM_FWD, xa, st));
    cubic_status_t s;
    for (int j = 0; j < cnt; ++j) {
        s = seg_U ? enqueue_yzy_grad(p, spec, ZM_CONV, seg_U[j], nullptr, nullptr, 0, st)
                  : enqueue_yzy(p, spec, ZM_CONV, st);
        if (s != CUBIC_OK) return s;
        xa.keep_a = seg_b[j];
        xa.keep_b = seg_r[j];
        CUBIC_CUDA(run_x(p, XM_RATIO, xa, st));
        s = seg_R ? enqueue_yzy_grad(p, spec, ZM_CORR, seg_R[j], nullptr, nullptr, 0, st)
                  : enqueue_yzy(p, spec, ZM_CORR, st);
        if (s != CUBIC_OK) return s;
        xa.keep_a = seg_q[j];
        xa.keep_b = nullptr;
        xa.u = seg_u[j];
        xa.dst = seg_u[j + 1];
        CUBIC_CUDA(run_x(p, j + 1 < cnt ? XM_UPDATE : XM_FINAL, xa, st));
        xa.keep_a = nullptr;
    }
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_deconvolve_ckpt(cubic_rl_plan_t plan, const float *image, int n_iter, float eps,
                                                   int ckpt_every, float *ckpts, float *out, void *stream)
{
    if (!plan || !image || !out || !ckpts) return fail(CUBIC_ERR_INVALID_ARG, "null pointer");
    if (cubic_status_t g = no_linear(plan, "the differentiable path")) return g;
    if (n_iter < 1 || ckpt_every < 1) return fail(CUBIC_ERR_INVALID_ARG, "n_iter and ckpt_every must be >= 1");
    if (!(eps > 0.f) || !(eps < INFINITY)) return fail(CUBIC_ERR_INVALID_ARG, "eps must be finite and > 0");
    if (!aligned16(image) || !aligned16(out) || !aligned16(ckpts))
        return fail(CUBIC_ERR_ALIGNMENT, "image, out and ckpts must be 16-byte aligned");
    const size_t vb = (size_t)plan->V * sizeof(float);
    const int nck = (n_iter + ckpt_every - 1) / ckpt_every;
    if (overlaps(image, out, vb) || ranges_overlap(image, vb, ckpts, vb * nck) || ranges_overlap(out, vb, ckpts, vb * nck))
        return fail(CUBIC_ERR_INVALID_ARG, "image, out and ckpts must not overlap");
    cubic_status_t s = ensure_workspace(plan);
    if (s != CUBIC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    cubic_rl_plan_s *p = plan;
    if ((s = enqueue_init(p, image, eps, out, st)) != CUBIC_OK) return s;
    XArgs xa = x_args(p);
    xa.spec_in = p->ws;
    xa.spec_out = p->ws;
    xa.src = out;
    xa.u = out;
    xa.dst = out;
    xa.d = image;
    xa.eps = eps;
    CUBIC_CUDA(run_x(p, XM_FWD, xa, st));
    for (int k = 0; k < n_iter; ++k) {
        if (k % ckpt_every == 0)
            CUBIC_CUDA(cudaMemcpyAsync(ckpts + (size_t)(k / ckpt_every) * p->V, out, vb, cudaMemcpyDeviceToDevice, st));
        if ((s = enqueue_yzy(p, p->ws, ZM_CONV, st)) != CUBIC_OK) return s;
        CUBIC_CUDA(run_x(p, XM_RATIO, xa, st));
        if ((s = enqueue_yzy(p, p->ws, ZM_CORR, st)) != CUBIC_OK) return s;
        CUBIC_CUDA(run_x(p, k + 1 < n_iter ? XM_UPDATE : XM_FINAL, xa, st));
    }
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_backward_workspace_bytes(cubic_rl_plan_t plan, int ckpt_every, size_t *bytes)
{
    if (!plan || !bytes || ckpt_every < 1) return fail(CUBIC_ERR_INVALID_ARG, "bad arguments");
    const size_t vb = ((size_t)plan->V * sizeof(float) + 255) / 256 * 256;
    const size_t sb = (spec_elems(plan) * sizeof(float2) + 255) / 256 * 256;
    const size_t rb = ((kReduceBlocks + 1) * sizeof(double) + 255) / 256 * 256;
    // u (c + 1), b, r, q (c each), g, tmp, dbar; spectra U, R (c each) and G
    *bytes = vb * (4 * (size_t)ckpt_every + 1 + 3) + (2 * (size_t)ckpt_every + 1) * sb + rb;
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_backward(cubic_rl_plan_t plan, const float *image, int n_iter, float eps,
                                            int ckpt_every, const float *ckpts, const float *grad_out,
                                            float *grad_image, float *grad_psf, int accumulate_psf, void *stream)
{
    if (!plan || !image || !ckpts || !grad_out) return fail(CUBIC_ERR_INVALID_ARG, "null pointer");
    if (cubic_status_t g = no_linear(plan, "the differentiable path")) return g;
    if (n_iter < 1 || ckpt_every < 1) return fail(CUBIC_ERR_INVALID_ARG, "n_iter and ckpt_every must be >= 1");
    if (!(eps > 0.f) || !(eps < INFINITY)) return fail(CUBIC_ERR_INVALID_ARG, "eps must be finite and > 0");
    if (!aligned16(image) || !aligned16(ckpts) || !aligned16(grad_out) || (grad_image && !aligned16(grad_image)) ||
        (grad_psf && !aligned16(grad_psf)))
        return fail(CUBIC_ERR_ALIGNMENT, "pointers must be 16-byte aligned");
    cubic_rl_plan_s *p = plan;
    cubic_status_t s = ensure_workspace(p);
    if (s != CUBIC_OK) return s;
    size_t need = 0;
    cubic_rl_backward_workspace_bytes(p, ckpt_every, &need);
    if (p->bwd_bytes < need) {
        cudaDeviceSynchronize();
        cudaFree(p->bwd);
        p->bwd = nullptr;
        p->bwd_bytes = 0;
        void *m = nullptr;
        CUBIC_CUDA(cudaMalloc(&m, need));
        p->bwd = (unsigned char *)m;
        p->bwd_bytes = need;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t V = p->V;
    const size_t vb = ((size_t)V * sizeof(float) + 255) / 256 * 256;
    const size_t sb = (spec_elems(p) * sizeof(float2) + 255) / 256 * 256;
    unsigned char *m = p->bwd;
    const int c = ckpt_every;
    std::vector<float *> seg_u(c + 1), seg_b(c), seg_r(c), seg_q(c);
    for (int j = 0; j <= c; ++j) seg_u[j] = (float *)(m + vb * j);
    for (int j = 0; j < c; ++j) {
        seg_b[j] = (float *)(m + vb * (c + 1 + j));
        seg_r[j] = (float *)(m + vb * (2 * c + 1 + j));  // written by the ratio pass with b
        seg_q[j] = (float *)(m + vb * (3 * c + 1 + j));
    }
    float *g = (float *)(m + vb * (4 * c + 1));     // the running gradient of the iterate
    float *tmp = (float *)(m + vb * (4 * c + 2));   // the PSF gradient, back in real space
    float *dbar = (float *)(m + vb * (4 * c + 3));
    std::vector<float2 *> seg_U(c), seg_R(c);
    unsigned char *specs = m + vb * (4 * c + 4);
    for (int j = 0; j < c; ++j) {
        seg_U[j] = (float2 *)(specs + sb * j);
        seg_R[j] = (float2 *)(specs + sb * (c + j));
    }
    float2 *G = (float2 *)(specs + sb * 2 * c);
    double *red = (double *)((unsigned char *)G + sb);  // kReduceBlocks + 1 doubles
    float2 *spec = p->ws;
    const unsigned gr = grid_for(V, 256);

    CUBIC_CUDA(cudaMemcpyAsync(g, grad_out, (size_t)V * sizeof(float), cudaMemcpyDeviceToDevice, st));
    CUBIC_CUDA(cudaMemsetAsync(dbar, 0, (size_t)V * sizeof(float), st));
    CUBIC_CUDA(cudaMemsetAsync(G, 0, sb, st));
    const int nseg = (n_iter + c - 1) / c;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int k0 = sg * c;
        const int cnt = std::min(c, n_iter - k0);
        CUBIC_CUDA(cudaMemcpyAsync(seg_u[0], ckpts + (size_t)sg * V, (size_t)V * sizeof(float),
                                   cudaMemcpyDeviceToDevice, st));
        if ((s = enqueue_segment(p, image, eps, cnt, seg_u.data(), seg_b.data(), seg_r.data(), seg_q.data(), spec,
                                 st, seg_U.data(), seg_R.data())) != CUBIC_OK)
            return s;
        // The adjoint iterations as fused pass chains: every pointwise step rides in an X
        // pass (XM_ADJ_*), so an iteration is 8 passes, like a forward one.  One buffer, g,
        // carries the running gradient of the iterate through the segment.
        XArgs xa = x_args(p);
        xa.spec_out = spec;
        xa.d = image;
        xa.eps = eps;
        const double real = (double)V * 4.0, cplx = (double)p->rows * p->xh * 8.0;
        auto adj = [&](int mode, const XArgs &a, double bytes) {
            return counted(p, KK_X_ADJOINT, st, [&] { return p->kx->adj[mode - XM_ADJ_R](a, st); }, bytes);
        };
        XArgs au = xa;
        au.adj_w = g;
        {
            // the segment's last iteration: qbar = g u (its spectrum), g = g q
            XArgs a0 = au;
            a0.adj_u = seg_u[cnt - 1];
            a0.adj_q = seg_q[cnt - 1];
            CUBIC_CUDA(adj(XM_ADJ_U, a0, 4 * real + cplx));
        }
        for (int j = cnt - 1; j >= 0; --j) {
            // rbar = h * qbar, with G += conj(Qbar) R in its z pass
            if ((s = enqueue_yzy_grad(p, spec, ZM_CONV, nullptr, G, seg_R[j], 1, st)) != CUBIC_OK) return s;
            // dbar += rbar / c; the spectrum of bbar
            XArgs ar = xa;
            ar.spec_in = spec;
            ar.adj_b = seg_b[j];
            ar.adj_dbar = dbar;
            CUBIC_CUDA(adj(XM_ADJ_R, ar, 4 * real + 2 * cplx));
            // h (x) bbar, with G += Bbar conj(U) in its z pass
            if ((s = enqueue_yzy_grad(p, spec, ZM_CORR, nullptr, G, seg_U[j], 0, st)) != CUBIC_OK) return s;
            // g += h (x) bbar: dL/du_j; then the previous iteration's qbar and g q
            XArgs a1 = au;
            a1.spec_in = spec;
            if (j > 0) {
                a1.adj_u = seg_u[j - 1];
                a1.adj_q = seg_q[j - 1];
            }
            CUBIC_CUDA(adj(XM_ADJ_U, a1, (j > 0 ? 4 * real : 2 * real) + (j > 0 ? 2 : 1) * cplx));
        }
        CUBIC_CUDA(cudaGetLastError());
    }
    // the initial estimate u0 = max(mean(d), eps) depends on d
    if (grad_image) {
        // the plan's reduction scratch holds kReduceBlocks + 1 doubles: as CFloat partials
        // (8 bytes each) plus one float result
        CFloat *gpart = reinterpret_cast<CFloat *>(p->partial);
        float *gsum = reinterpret_cast<float *>(gpart + kReduceBlocks);
        k_csum_partial<<<kReduceBlocks, kReduceThreads, 0, st>>>(g, V, gpart);
        k_csum_final<<<1, 32, 0, st>>>(gpart, kReduceBlocks, gsum);
        k_sum_partial<<<kReduceBlocks, kReduceThreads, 0, st>>>(image, V, red);
        k_sum_final<<<1, kReduceThreads, 0, st>>>(red, kReduceBlocks, red + kReduceBlocks);
        k_add_mean_grad<<<gr, 256, 0, st>>>(dbar, gsum, red + kReduceBlocks, V, eps);
        CUBIC_CUDA(cudaMemcpyAsync(grad_image, dbar, (size_t)V * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    if (grad_psf) {
        if ((s = enqueue_inverse3(p, G, tmp, (float)(1.0 / (double)V), st)) != CUBIC_OK) return s;
        k_origin_to_center<<<gr, 256, 0, st>>>(tmp, grad_psf, p->nz, p->ny, p->nx, accumulate_psf);
    }
    CUBIC_CUDA(cudaGetLastError());
    return CUBIC_OK;
}

// ---- Gaussian PSF parameter gradient
//
// psf = A g / S, S = sum g, g = exp(-(dx^2+dy^2) a - dz^2 c), a = 1/(2 sxy^2), c = 1/(2 sz^2):
//   dL/dA   = P / S,                          P = sum(pbar g)
//   dL/dsxy = A/S (Pxy - P Sxy / S),          Pxy = sum(pbar g rxy/sxy^3), Sxy = sum(g rxy/sxy^3)
//   dL/dsz  = A/S (Pz - P Sz / S)             (same with dz^2 / sz^3)
// Six sums: S (the PSF's flux) in double; the five others in compensated float
// (a Kahan running sum per thread, error-free TwoSum merges across threads).

__global__ void __launch_bounds__(kReduceThreads) k_psf_gauss_grad(const float *__restrict__ gp, int64_t nz,
                                                                   int64_t ny, int64_t nx, float a_xy, float a_z,
                                                                   float inv_sxy3, float inv_sz3,
                                                                   double *__restrict__ part_S,
                                                                   float *__restrict__ part5)
{
    __shared__ double shS[kReduceThreads];
    __shared__ CFloat sh[5][kReduceThreads];
    const int64_t V = nz * ny * nx;
    double S = 0.0;
    CFloat acc[5] = {};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
        const float dx = (float)(i % nx - nx / 2);
        const float dy = (float)((i / nx) % ny - ny / 2);
        const float dz = (float)(i / (nx * ny) - nz / 2);
        const float rxy = dx * dx + dy * dy, rz = dz * dz;
        const float g = expf(-rxy * a_xy - rz * a_z);
        const float gxy = g * rxy * inv_sxy3, gz = g * rz * inv_sz3;
        const float pb = gp[i];
        S += (double)g;
        acc[0] = cf_add(acc[0], gxy);
        acc[1] = cf_add(acc[1], gz);
        acc[2] = cf_add(acc[2], pb * g);
        acc[3] = cf_add(acc[3], pb * gxy);
        acc[4] = cf_add(acc[4], pb * gz);
    }
    shS[threadIdx.x] = S;
    for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = kReduceThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            shS[threadIdx.x] += shS[threadIdx.x + w];
            for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = cf_merge(sh[k][threadIdx.x], sh[k][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part_S[blockIdx.x] = shS[0];
        for (int k = 0; k < 5; ++k) {
            part5[(blockIdx.x * 5 + k) * 2] = sh[k][0].s;
            part5[(blockIdx.x * 5 + k) * 2 + 1] = sh[k][0].c;
        }
    }
}

__global__ void __launch_bounds__(kReduceThreads) k_psf_gauss_grad_final(const double *__restrict__ part_S,
                                                                         const float *__restrict__ part5, int nblk,
                                                                         float amp, float *__restrict__ out3)
{
    __shared__ double shS[kReduceThreads];
    __shared__ CFloat sh[5][kReduceThreads];
    double S = 0.0;
    CFloat acc[5] = {};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        S += part_S[b];
        for (int k = 0; k < 5; ++k)
            acc[k] = cf_merge(acc[k], CFloat{part5[(b * 5 + k) * 2], part5[(b * 5 + k) * 2 + 1]});
    }
    shS[threadIdx.x] = S;
    for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = kReduceThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            shS[threadIdx.x] += shS[threadIdx.x + w];
            for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = cf_merge(sh[k][threadIdx.x], sh[k][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float Sf = (float)shS[0];
        const float Sxy = sh[0][0].s - sh[0][0].c, Sz = sh[1][0].s - sh[1][0].c;
        const float P = sh[2][0].s - sh[2][0].c, Pxy = sh[3][0].s - sh[3][0].c, Pz = sh[4][0].s - sh[4][0].c;
        out3[0] = amp / Sf * (Pxy - P * Sxy / Sf);
        out3[1] = amp / Sf * (Pz - P * Sz / Sf);
        out3[2] = P / Sf;
    }
}

extern "C" cubic_status_t cubic_psf_gaussian_backward(const int64_t dims[3], float sigma_xy, float sigma_z, float amp,
                                                      const float *grad_psf, float *grad_params_dev, void *stream)
{
    if (!dims || !grad_psf || !grad_params_dev) return fail(CUBIC_ERR_INVALID_ARG, "null pointer");
    for (int i = 0; i < 3; ++i)
        if (dims[i] < 1) return fail(CUBIC_ERR_INVALID_ARG, "dims must be >= 1");
    if (!(sigma_xy > 0.f) || !(sigma_z > 0.f) || !(sigma_xy < INFINITY) || !(sigma_z < INFINITY) ||
        !(fabsf(amp) < INFINITY))
        return fail(CUBIC_ERR_INVALID_ARG, "sigmas must be finite and > 0, amp finite");
    if (!aligned16(grad_psf)) return fail(CUBIC_ERR_ALIGNMENT, "grad_psf must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    void *scratch = nullptr;
    const size_t bytes = kReduceBlocks * sizeof(double) + kReduceBlocks * 10 * sizeof(float);
    CUBIC_CUDA(cudaMallocAsync(&scratch, bytes, st));
    double *part_S = (double *)scratch;
    float *part5 = (float *)(part_S + kReduceBlocks);
    const double sxy = sigma_xy, sz = sigma_z;
    k_psf_gauss_grad<<<kReduceBlocks, kReduceThreads, 0, st>>>(grad_psf, dims[0], dims[1], dims[2],
                                                               (float)(0.5 / (sxy * sxy)), (float)(0.5 / (sz * sz)),
                                                               (float)(1.0 / (sxy * sxy * sxy)),
                                                               (float)(1.0 / (sz * sz * sz)), part_S, part5);
    k_psf_gauss_grad_final<<<1, kReduceThreads, 0, st>>>(part_S, part5, kReduceBlocks, amp, grad_params_dev);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return fail(CUBIC_ERR_CUDA, "psf gradient kernels: %s", cudaGetErrorString(e));
    return CUBIC_OK;
}

// ------------------------------------------------------------------ automatic stopping
//
// The paper (Section 4) stops Richardson-Lucy automatically when the improvement
// between consecutive iterations falls under a threshold.  Here the improvement of
// iteration k is the relative change of the estimate,
//   delta_k = ||u_{k+1} - u_k||_2 / ||u_k||_2,
// whose two sums the update pass accumulates, in compensated float32, as it writes
// u_{k+1}.  Every check_every iterations (and after the last) the host reads delta and
// stops below the threshold.

// merges the 64 compensated slots of one iteration in a fixed order
__global__ void k_delta(const float *__restrict__ slots, float *__restrict__ delta)
{
    if (threadIdx.x != 0) return;
    CFloat num{0.f, 0.f}, den{0.f, 0.f};
    for (int i = 0; i < 64; ++i) {
        num = cf_merge(num, CFloat{slots[4 * i], -slots[4 * i + 1]});
        den = cf_merge(den, CFloat{slots[4 * i + 2], -slots[4 * i + 3]});
    }
    const float n = num.s - num.c, d = den.s - den.c;
    delta[0] = d > 0.f ? sqrtf(n / d) : 0.f;
}

extern "C" cubic_status_t cubic_rl_deconvolve_auto(cubic_rl_plan_t plan, const float *image, int max_iter, float eps,
                                                   float tol, int check_every, float *out, int *n_done,
                                                   double *history, void *stream)
{
    if (!plan || !image || !out || !n_done) return fail(CUBIC_ERR_INVALID_ARG, "plan, image, out, n_done must be non-null");
    if (max_iter < 1 || check_every < 1) return fail(CUBIC_ERR_INVALID_ARG, "max_iter and check_every must be >= 1");
    if (!(eps > 0.f) || !(eps < INFINITY)) return fail(CUBIC_ERR_INVALID_ARG, "eps must be finite and > 0");
    if (!(tol >= 0.f) || !(tol < INFINITY)) return fail(CUBIC_ERR_INVALID_ARG, "tol must be finite and >= 0");
    if (!aligned16(image) || !aligned16(out)) return fail(CUBIC_ERR_ALIGNMENT, "image and out must be 16-byte aligned");
    if (overlaps(image, out, (size_t)plan->V * sizeof(float))) return fail(CUBIC_ERR_INVALID_ARG, "out must not overlap image");
    cubic_rl_plan_s *p = plan;
    cubic_status_t s = ensure_workspace(p);
    if (s != CUBIC_OK) return s;
    if (p->auto_cap < max_iter) {
        cudaDeviceSynchronize();
        cudaFree(p->auto_stats);
        cudaFree(p->auto_delta);
        p->auto_stats = nullptr;
        p->auto_delta = nullptr;
        p->auto_cap = 0;
        void *a = nullptr, *b = nullptr;
        CUBIC_CUDA(cudaMalloc(&a, (size_t)max_iter * 256 * sizeof(float)));
        p->auto_stats = (float *)a;
        CUBIC_CUDA(cudaMalloc(&b, (size_t)max_iter * sizeof(float)));
        p->auto_delta = (float *)b;
        p->auto_cap = max_iter;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CUBIC_CUDA(cudaMemsetAsync(p->auto_stats, 0, (size_t)max_iter * 256 * sizeof(float), st));
    // a linear plan iterates on its padded arrays (the padding contributes zeros to the sums)
    float *uw = p->linear ? p->lin + lin_elems(p) : out;
    const float *dw = p->linear ? p->lin : image;
    s = p->linear ? lin_init(p, image, eps, p->lin, uw, st) : enqueue_init(p, image, eps, out, st);
    if (s != CUBIC_OK) return s;
    XArgs xa = x_args(p);
    xa.spec_in = p->ws;
    xa.spec_out = p->ws;
    xa.src = uw;
    xa.u = uw;
    xa.dst = uw;
    xa.d = dw;
    xa.eps = eps;
    CUBIC_CUDA(run_x(p, XM_FWD, xa, st));
    int k = 0;
    while (k < max_iter) {
        if ((s = enqueue_yzy(p, p->ws, ZM_CONV, st)) != CUBIC_OK) return s;
        CUBIC_CUDA(run_x(p, XM_RATIO, xa, st));
        if ((s = enqueue_yzy(p, p->ws, ZM_CORR, st)) != CUBIC_OK) return s;
        XArgs xs = xa;
        xs.stats = p->auto_stats + (size_t)k * 256;
        CUBIC_CUDA(run_x(p, k + 1 < max_iter ? XM_UPDATE : XM_FINAL, xs, st));
        k_delta<<<1, 64, 0, st>>>(xs.stats, p->auto_delta + k);
        CUBIC_CUDA(cudaGetLastError());
        ++k;
        if (k % check_every == 0 || k == max_iter) {
            float delta = 0.f;
            CUBIC_CUDA(cudaMemcpyAsync(&delta, p->auto_delta + k - 1, sizeof(float), cudaMemcpyDeviceToHost, st));
            CUBIC_CUDA(cudaStreamSynchronize(st));
            if (delta < tol) break;  // the estimate already holds u_k (the update wrote it)
        }
    }
    if (p->linear && (s = lin_crop(p, uw, out, st)) != CUBIC_OK) return s;
    *n_done = k;
    if (history) {
        std::vector<float> h((size_t)k);
        CUBIC_CUDA(cudaMemcpyAsync(h.data(), p->auto_delta, (size_t)k * sizeof(float), cudaMemcpyDeviceToHost, st));
        CUBIC_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < k; ++i) history[i] = (double)h[(size_t)i];
    }
    return CUBIC_OK;
}

// ------------------------------------------------------------------ accelerated RL
//
// Biggs-Andrews first-order vector extrapolation (the acceleration the paper cites for
// Richardson-Lucy): every RL step starts from a prediction along the last move,
//   y_k = max(x_k + alpha_k (x_k - x_{k-1}), 0),   x_{k+1} = RL step from y_k,
//   g_k = x_{k+1} - y_k,   alpha_{k+1} = <g_k, g_{k-1}> / <g_{k-1}, g_{k-1}> clamped to [0, 1],
// alpha_0 = alpha_1 = 0, and alpha = 0 for a zero denominator.  Per iteration:
//   the usual passes up to the back-correlation's spectrum; then
//   XM_FINAL (accelerated): x_{k+1} = y_k q, g_k, per-CTA partial sums of the two products;
//   k_acc_alpha: the partials merged in a fixed order, alpha_{k+1} on the device;
//   XM_FWD (accelerated): y_{k+1} from x_{k+1}, x_k, alpha, stored and transformed.
// No host synchronisation: alpha stays on the device.

// state[0] = <g_{k-1}, g_{k-1}> (from the previous call), state[1] = alpha_{k+1}
__global__ void __launch_bounds__(1024) k_acc_alpha(const float4 *__restrict__ part, int64_t nblocks, int k,
                                                    float *__restrict__ state, float *__restrict__ alpha_hist,
                                                    int n_iter)
{
    __shared__ CFloat sn[1024], sd[1024];
    CFloat num{0.f, 0.f}, den{0.f, 0.f};
    constexpr int U = 8;  // loads in flight per thread
    for (int64_t i0 = threadIdx.x; i0 < nblocks; i0 += (int64_t)U * blockDim.x) {
        float4 q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x;
            q[u] = i < nblocks ? part[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            num = cf_merge(num, CFloat{q[u].x, q[u].y});
            den = cf_merge(den, CFloat{q[u].z, q[u].w});
        }
    }
    sn[threadIdx.x] = num;
    sd[threadIdx.x] = den;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sn[threadIdx.x] = cf_merge(sn[threadIdx.x], sn[threadIdx.x + w]);
            sd[threadIdx.x] = cf_merge(sd[threadIdx.x], sd[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float nk = sn[0].s - sn[0].c, dk = sd[0].s - sd[0].c;
        const float dprev = state[0];
        float al = 0.f;
        if (k >= 1 && dprev > 0.f) {
            const float r = nk / dprev;
            al = r > 0.f ? (r < 1.f ? r : 1.f) : 0.f;  // also maps NaN to 0
        }
        state[0] = dk;
        state[1] = al;
        if (alpha_hist && k + 1 < n_iter) alpha_hist[k + 1] = al;
    }
}

// the padded arrays' size for a linear plan
static size_t acc_vol_bytes(const cubic_rl_plan_s *p)
{
    return ((p->linear ? lin_elems(p) : (size_t)p->V) * sizeof(float) + 255) / 256 * 256;
}

static cubic_status_t ensure_accel(cubic_rl_plan_s *p)
{
    if (p->acc) return CUBIC_OK;
    const size_t vol = acc_vol_bytes(p);
    const size_t nb = (size_t)((p->rows + 1) / 2);  // most X blocks: one line pair each
    const size_t part = (nb * sizeof(float4) + 255) / 256 * 256;
    void *m = nullptr;
    if (cudaMalloc(&m, 5 * vol + part + 256) != cudaSuccess) {
        cudaGetLastError();
        return fail(CUBIC_ERR_OUT_OF_MEMORY, "accelerated RL buffers (%zu bytes)", 5 * vol + part + 256);
    }
    p->acc = (float *)m;
    p->acc_part = (float4 *)((unsigned char *)m + 5 * vol);
    p->acc_state = (float *)((unsigned char *)m + 5 * vol + part);
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_deconvolve_accel(cubic_rl_plan_t plan, const float *image, int n_iter, float eps,
                                                    float *out, float *alpha, void *stream)
{
    if (!plan || !image || !out) return fail(CUBIC_ERR_INVALID_ARG, "plan, image and out must be non-null");
    if (n_iter < 0) return fail(CUBIC_ERR_INVALID_ARG, "n_iter must be >= 0");
    if (!(eps > 0.f) || !(eps < INFINITY)) return fail(CUBIC_ERR_INVALID_ARG, "eps must be finite and > 0");
    if (!aligned16(image) || !aligned16(out)) return fail(CUBIC_ERR_ALIGNMENT, "image and out must be 16-byte aligned");
    if (overlaps(image, out, (size_t)plan->V * sizeof(float)))
        return fail(CUBIC_ERR_INVALID_ARG, "out must not overlap image");
    if (alpha && ((uintptr_t)alpha % sizeof(float)) != 0) return fail(CUBIC_ERR_ALIGNMENT, "alpha must be 4-byte aligned");
    cubic_rl_plan_s *p = plan;
    cubic_status_t s = ensure_workspace(p);
    if (s != CUBIC_OK) return s;
    if ((s = ensure_accel(p)) != CUBIC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t vol = acc_vol_bytes(p) / sizeof(float);
    float *xc = p->acc, *xn = p->acc + vol, *y = p->acc + 2 * vol, *gc = p->acc + 3 * vol, *gn = p->acc + 4 * vol;
    // a linear plan iterates on zero-padded rows: the padding stays 0 under the update and
    // the prediction, and adds 0 to the dot products
    const size_t nw = p->linear ? lin_elems(p) : (size_t)p->V;
    const float *dw = p->linear ? p->lin : image;
    auto finish = [&](const float *x) -> cubic_status_t {
        if (p->linear) return lin_crop(p, x, out, st);
        CUBIC_CUDA(cudaMemcpyAsync(out, x, nw * sizeof(float), cudaMemcpyDeviceToDevice, st));
        return CUBIC_OK;
    };

    s = p->linear ? lin_init(p, image, eps, p->lin, xc, st) : enqueue_init(p, image, eps, xc, st);  // x_0
    if (s != CUBIC_OK) return s;
    if (n_iter == 0) return finish(xc);
    CUBIC_CUDA(cudaMemcpyAsync(y, xc, nw * sizeof(float), cudaMemcpyDeviceToDevice, st));  // y_0 = x_0
    CUBIC_CUDA(cudaMemsetAsync(p->acc_state, 0, 2 * sizeof(float), st));
    if (alpha) CUBIC_CUDA(cudaMemsetAsync(alpha, 0, (size_t)n_iter * sizeof(float), st));

    const double spec = (double)p->rows * p->xh * 8.0, real = (double)p->V * 4.0;
    const int64_t L = p->kx->xv[p->vx].L;
    const int64_t nblocks = (p->rows + 2 * L - 1) / (2 * L);
    XArgs xa = x_args(p);
    xa.spec_in = p->ws;
    xa.spec_out = p->ws;
    xa.d = dw;
    xa.eps = eps;
    xa.src = y;
    CUBIC_CUDA(run_x(p, XM_FWD, xa, st));  // spectrum of y_0
    for (int k = 0; k < n_iter; ++k) {
        if ((s = enqueue_yzy(p, p->ws, ZM_CONV, st)) != CUBIC_OK) return s;  // b = h * y_k
        CUBIC_CUDA(run_x(p, XM_RATIO, xa, st));                             // r = d / max(b, eps)
        if ((s = enqueue_yzy(p, p->ws, ZM_CORR, st)) != CUBIC_OK) return s;  // q = h (flipped) * r
        const bool last = k + 1 == n_iter;
        XArgs xu = xa;                                                       // x_{k+1} = y_k q, g_k
        xu.u = y;
        xu.dst = (last && !p->linear) ? out : xn;
        xu.acc_g = gn;
        xu.acc_gprev = k >= 1 ? gc : nullptr;
        xu.acc_part = p->acc_part;
        CUBIC_CUDA(run_x_as(p, XM_FINAL, KK_X_ACC_UPDATE, xu, spec + (k >= 1 ? 4 : 3) * real, st));
        if (last) return p->linear ? lin_crop(p, xn, out, st) : CUBIC_OK;
        CUBIC_CUDA(counted(p, KK_ACC_ALPHA, st, [&] {
            k_acc_alpha<<<1, 1024, 0, st>>>(p->acc_part, nblocks, k, p->acc_state, alpha, n_iter);
            return cudaGetLastError();
        }));
        XArgs xq = xa;                                                       // y_{k+1}, its spectrum
        xq.src = xn;
        xq.acc_prev = xc;
        xq.acc_alpha = p->acc_state + 1;
        xq.acc_y = y;
        CUBIC_CUDA(run_x_as(p, XM_FWD, KK_X_ACC_PREDICT, xq, 3 * real + spec, st));
        std::swap(xc, xn);
        std::swap(gc, gn);
    }
    return CUBIC_OK;
}

// ------------------------------------------------------------------ metric-guided stopping
//
// Three measures per iteration k (the one that made u_{k+1}), each in compensated float32
// sums on the GPU:
//   delta_k = ||u_{k+1} - u_k|| / ||u_k||          (update pass, as in automatic stopping)
//   NLL(u_k) = sum (c - d ln c), c = max(h * u_k, eps)   (ratio pass)
//   PSNR_si(u_{k+1}, y) against a reference y: sums of x, x^2, x y (k_ref_sums) and the
//     reference's sum, sum of squares and range (k_ref_moments, once); the least-squares
//     affine fit and the logarithm are finished on the host in double precision.
// At each check the host applies the stopping rule of the chosen measure.

constexpr int kMonBlocks = 608;  // reduction blocks: four per SM
constexpr int kMonRec = 12;      // floats per iteration record

// merges a CTA's compensated sums (NS of them, in order) into thread 0's registers
template <int NS>
__device__ __forceinline__ void block_merge_n(CFloat (&v)[NS])
{
    __shared__ CFloat red[NS][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = 0; j < NS; ++j)
        for (int o = 16; o > 0; o >>= 1)
            v[j] = cf_merge(v[j], CFloat{__shfl_down_sync(0xffffffffu, v[j].s, o),
                                         __shfl_down_sync(0xffffffffu, v[j].c, o)});
    if (lane == 0)
        for (int j = 0; j < NS; ++j) red[j][warp] = v[j];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int j = 0; j < NS; ++j) {
            v[j] = red[j][0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v[j] = cf_merge(v[j], red[j][w]);
        }
}

// per-block (sum x, sum x^2, sum x y) as three (s, c) pairs
__global__ void __launch_bounds__(256) k_ref_sums(const float *__restrict__ x, const float *__restrict__ y, int64_t V,
                                                  float *__restrict__ part)
{
    CFloat v[3] = {};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
        const float xv = x[i], yv = y[i];
        v[0] = cf_add(v[0], xv);
        v[1] = cf_add(v[1], xv * xv);
        v[2] = cf_add(v[2], xv * yv);
    }
    block_merge_n<3>(v);
    if (threadIdx.x == 0)
        for (int j = 0; j < 3; ++j) {
            part[6 * blockIdx.x + 2 * j] = v[j].s;
            part[6 * blockIdx.x + 2 * j + 1] = v[j].c;
        }
}

// Poisson likelihood sum (c - d ln c), c = max(b, eps), over the image columns of a
// linear plan's padded rows (past them d = 0 and the term would count the blur that
// spills into the padding); compensated, into the 64 (hi, lo) slots the ratio pass fills
// for a circular plan.
__global__ void __launch_bounds__(256) k_nll_image(const float *__restrict__ b, const float *__restrict__ d,
                                                   int64_t rows, int64_t pitch, int64_t cols, float eps,
                                                   float *__restrict__ slots)
{
    CFloat v{0.f, 0.f};
    const int64_t n = rows * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / cols, x = i - r * cols;
        const float c = fmaxf(b[r * pitch + x], eps);
        v = cf_add(v, c - d[r * pitch + x] * logf(c));
    }
    const int slot = (int)((blockIdx.x * 8 + (threadIdx.x >> 5)) & 63);
    slot_add<256>(slots + 2 * slot, v);
}

// per-block (sum y, sum y^2) as (s, c) pairs, then min y and max y
__global__ void __launch_bounds__(256) k_ref_moments(const float *__restrict__ y, int64_t V, float *__restrict__ part)
{
    CFloat v[2] = {};
    float mn = INFINITY, mx = -INFINITY;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
        const float yv = y[i];
        v[0] = cf_add(v[0], yv);
        v[1] = cf_add(v[1], yv * yv);
        mn = fminf(mn, yv);
        mx = fmaxf(mx, yv);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    __shared__ float smn[32], smx[32];
    if ((threadIdx.x & 31) == 0) {
        smn[threadIdx.x >> 5] = mn;
        smx[threadIdx.x >> 5] = mx;
    }
    block_merge_n<2>(v);  // synchronises: smn / smx are complete after it
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            mn = fminf(mn, smn[w]);
            mx = fmaxf(mx, smx[w]);
        }
        part[6 * blockIdx.x + 0] = v[0].s;
        part[6 * blockIdx.x + 1] = v[0].c;
        part[6 * blockIdx.x + 2] = v[1].s;
        part[6 * blockIdx.x + 3] = v[1].c;
        part[6 * blockIdx.x + 4] = mn;
        part[6 * blockIdx.x + 5] = mx;
    }
}

// One iteration's record, merged in a fixed order: rec = (delta, nll s, nll c,
// sx s, sx c, sxx s, sxx c, sxy s, sxy c) (value = s - c); ref_part may be null.
__global__ void k_metrics(const float *__restrict__ dslots, const float *__restrict__ nslots,
                          const float *__restrict__ ref_part, int nblk, float *__restrict__ rec)
{
    if (threadIdx.x != 0) return;
    CFloat num{0.f, 0.f}, den{0.f, 0.f}, nll{0.f, 0.f};
    for (int i = 0; i < 64; ++i) {
        num = cf_merge(num, CFloat{dslots[4 * i], -dslots[4 * i + 1]});
        den = cf_merge(den, CFloat{dslots[4 * i + 2], -dslots[4 * i + 3]});
        nll = cf_merge(nll, CFloat{nslots[2 * i], -nslots[2 * i + 1]});
    }
    const float n = num.s - num.c, d = den.s - den.c;
    rec[0] = d > 0.f ? sqrtf(n / d) : 0.f;
    rec[1] = nll.s;
    rec[2] = nll.c;
    CFloat r[3] = {};
    if (ref_part)
        for (int b = 0; b < nblk; ++b)
            for (int j = 0; j < 3; ++j) r[j] = cf_merge(r[j], CFloat{ref_part[6 * b + 2 * j], ref_part[6 * b + 2 * j + 1]});
    for (int j = 0; j < 3; ++j) {
        rec[3 + 2 * j] = r[j].s;
        rec[4 + 2 * j] = r[j].c;
    }
}

extern "C" cubic_status_t cubic_rl_deconvolve_monitor(cubic_rl_plan_t plan, const float *image, const float *reference,
                                                      int max_iter, float eps, int metric, double tol, int check_every,
                                                      float *out, int *n_done, double *history, void *stream)
{
    if (!plan || !image || !out || !n_done) return fail(CUBIC_ERR_INVALID_ARG, "plan, image, out, n_done must be non-null");
    if (max_iter < 1 || check_every < 1) return fail(CUBIC_ERR_INVALID_ARG, "max_iter and check_every must be >= 1");
    if (!(eps > 0.f) || !(eps < INFINITY)) return fail(CUBIC_ERR_INVALID_ARG, "eps must be finite and > 0");
    if (!(tol >= -INFINITY) || tol != tol) return fail(CUBIC_ERR_INVALID_ARG, "tol must not be NaN");
    if (metric < CUBIC_METRIC_REL_CHANGE || metric > CUBIC_METRIC_PSNR)
        return fail(CUBIC_ERR_INVALID_ARG, "unknown metric %d", metric);
    if (metric == CUBIC_METRIC_PSNR && !reference) return fail(CUBIC_ERR_INVALID_ARG, "the PSNR measure needs a reference");
    if (!aligned16(image) || !aligned16(out) || (reference && !aligned16(reference)))
        return fail(CUBIC_ERR_ALIGNMENT, "image, out and reference must be 16-byte aligned");
    const size_t vb = (size_t)plan->V * sizeof(float);
    if (overlaps(image, out, vb) || (reference && overlaps(reference, out, vb)))
        return fail(CUBIC_ERR_INVALID_ARG, "out must not overlap image or reference");
    cubic_rl_plan_s *p = plan;
    cubic_status_t s = ensure_workspace(p);
    if (s != CUBIC_OK) return s;
    // [dslots: max_iter x 256][nslots: max_iter x 128][ref part: blocks x 6][ref moments: blocks x 6][rec: max_iter x 12]
    const size_t f_d = (size_t)max_iter * 256, f_n = (size_t)max_iter * 128, f_r = (size_t)kMonBlocks * 6;
    // a linear plan also keeps the ratio pass's b and r (padded rows) for the likelihood
    const size_t f_lin = p->linear ? 2 * lin_elems(p) : 0;
    const size_t f_rec = (size_t)max_iter * kMonRec, total = f_d + f_n + 2 * f_r + f_rec + f_lin;
    if (p->mon_cap < max_iter) {
        cudaDeviceSynchronize();
        cudaFree(p->mon);
        p->mon = nullptr;
        p->mon_cap = 0;
        void *m = nullptr;
        CUBIC_CUDA(cudaMalloc(&m, total * sizeof(float)));
        p->mon = (float *)m;
        p->mon_cap = max_iter;
    }
    float *dslots = p->mon, *nslots = dslots + f_d, *rpart = nslots + f_n, *mpart = rpart + f_r, *rec = mpart + f_r;
    float *kept_b = rec + f_rec, *kept_r = kept_b + f_lin / 2;
    cudaStream_t st = (cudaStream_t)stream;
    CUBIC_CUDA(cudaMemsetAsync(p->mon, 0, (f_d + f_n) * sizeof(float), st));

    // the reference's moments, once: sum y, sum y^2 (double on the host), range
    double sy = 0.0, syy = 0.0, range = 0.0;
    if (reference) {
        k_ref_moments<<<kMonBlocks, 256, 0, st>>>(reference, p->V, mpart);
        CUBIC_CUDA(cudaGetLastError());
        std::vector<float> h((size_t)kMonBlocks * 6);
        CUBIC_CUDA(cudaMemcpyAsync(h.data(), mpart, h.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
        CUBIC_CUDA(cudaStreamSynchronize(st));
        float mn = INFINITY, mx = -INFINITY;
        for (int b = 0; b < kMonBlocks; ++b) {
            sy += (double)h[6 * b] - (double)h[6 * b + 1];
            syy += (double)h[6 * b + 2] - (double)h[6 * b + 3];
            mn = std::min(mn, h[6 * b + 4]);
            mx = std::max(mx, h[6 * b + 5]);
        }
        range = (double)mx - (double)mn;
    }
    const double nV = (double)p->V;
    auto psnr = [&](const float *r) -> double {
        const double sx = (double)r[3] - (double)r[4], sxx = (double)r[5] - (double)r[6];
        const double sxy = (double)r[7] - (double)r[8];
        const double vx = sxx / nV - (sx / nV) * (sx / nV), vy = syy / nV - (sy / nV) * (sy / nV);
        const double cxy = sxy / nV - (sx / nV) * (sy / nV);
        double mse = vx > 0.0 ? vy - cxy * cxy / vx : vy;
        if (mse < 0.0) mse = 0.0;
        return 20.0 * log10(range / sqrt(mse));
    };

    // a linear plan iterates on its padded arrays: the padding adds zeros to the update's
    // sums, the likelihood is summed over the image's columns by k_nll_image, and the PSNR
    // is taken on the estimate cropped into out
    float *uw = p->linear ? p->lin + lin_elems(p) : out;
    const float *dw = p->linear ? p->lin : image;
    s = p->linear ? lin_init(p, image, eps, p->lin, uw, st) : enqueue_init(p, image, eps, out, st);
    if (s != CUBIC_OK) return s;
    XArgs xa = x_args(p);
    xa.spec_in = p->ws;
    xa.spec_out = p->ws;
    xa.src = uw;
    xa.u = uw;
    xa.dst = uw;
    xa.d = dw;
    xa.eps = eps;
    CUBIC_CUDA(run_x(p, XM_FWD, xa, st));
    std::vector<float> hrec;
    std::vector<double> hist;  // [k][3]
    int k = 0;
    while (k < max_iter) {
        if ((s = enqueue_yzy(p, p->ws, ZM_CONV, st)) != CUBIC_OK) return s;
        XArgs xr = xa;
        if (p->linear) {
            xr.keep_a = kept_b;
            xr.keep_b = kept_r;
        } else {
            xr.nll_stats = nslots + (size_t)k * 128;
        }
        CUBIC_CUDA(run_x(p, XM_RATIO, xr, st));
        if (p->linear) {
            k_nll_image<<<kMonBlocks, 256, 0, st>>>(kept_b, dw, p->iz * p->iy, p->nx, p->ix, eps,
                                                     nslots + (size_t)k * 128);
            CUBIC_CUDA(cudaGetLastError());
        }
        if ((s = enqueue_yzy(p, p->ws, ZM_CORR, st)) != CUBIC_OK) return s;
        XArgs xu = xa;
        xu.stats = dslots + (size_t)k * 256;
        CUBIC_CUDA(run_x(p, k + 1 < max_iter ? XM_UPDATE : XM_FINAL, xu, st));
        if (p->linear && (reference || k + 1 == max_iter) && (s = lin_crop(p, uw, out, st)) != CUBIC_OK) return s;
        if (reference) k_ref_sums<<<kMonBlocks, 256, 0, st>>>(out, reference, p->V, rpart);
        k_metrics<<<1, 32, 0, st>>>(dslots + (size_t)k * 256, nslots + (size_t)k * 128, reference ? rpart : nullptr,
                                    kMonBlocks, rec + (size_t)k * kMonRec);
        CUBIC_CUDA(cudaGetLastError());
        ++k;
        if (k % check_every == 0 || k == max_iter) {
            const int from = (int)hist.size() / 3;
            hrec.resize((size_t)k * kMonRec);
            CUBIC_CUDA(cudaMemcpyAsync(hrec.data() + (size_t)from * kMonRec, rec + (size_t)from * kMonRec,
                                       (size_t)(k - from) * kMonRec * sizeof(float), cudaMemcpyDeviceToHost, st));
            CUBIC_CUDA(cudaStreamSynchronize(st));
            for (int j = from; j < k; ++j) {
                const float *r = hrec.data() + (size_t)j * kMonRec;
                hist.push_back((double)r[0]);
                hist.push_back((double)r[1] - (double)r[2]);
                hist.push_back(reference ? psnr(r) : NAN);
            }
            const double *h = hist.data() + 3 * (size_t)(k - 1);
            bool stop = false;
            if (metric == CUBIC_METRIC_REL_CHANGE) stop = h[0] < tol;
            else if (k >= 2 && metric == CUBIC_METRIC_NLL) stop = (h[-2] - h[1]) / fabs(h[1]) < tol;
            else if (k >= 2 && metric == CUBIC_METRIC_PSNR) stop = h[2] - h[-1] < tol;
            if (stop) break;  // the estimate holds u_k (the update wrote it)
        }
    }
    // a linear plan without a reference crops only after the last iteration it ran
    if (p->linear && !reference && k < max_iter && (s = lin_crop(p, uw, out, st)) != CUBIC_OK) return s;
    *n_done = k;
    if (history) std::copy(hist.begin(), hist.begin() + 3 * (size_t)k, history);
    return CUBIC_OK;
}

// ------------------------------------------------------------------ Fourier Shell Correlation
//
// FSC(s) = Re sum A conj B / sqrt(sum |A|^2 sum |B|^2) over the frequencies of shell s,
// the paper's resolution metric (FRC/FSC, Sections 3 and 4).  Shells are uniform in the
// normalised radius rho = |(kz/nz, ky/ny, kx/nx)| (signed frequencies) up to Nyquist:
// s = floor(2 S rho), rho >= 1/2 left out.  rho^2 = rn / den is rational, so the shell is
// decided exactly in integers.  The half spectrum stands for the full one: columns
// 0 < kx < nx/2 count twice (their mirror -kx has the same shell and conjugate values).

constexpr int kFscMaxShells = 1024;

// Shell sums in compensated float32: per block in shared memory, then into the
// global pairs (value = hi + lo) -- sums[0..3S) high words, sums[3S..6S) low words.
__global__ void __launch_bounds__(256) k_fsc_bins(const float2 *__restrict__ A, const float2 *__restrict__ B,
                                                  int64_t nz, int64_t ny, int64_t nx, int64_t xh, int64_t xp,
                                                  int S, float *__restrict__ sums)
{
    extern __shared__ float sh_fsc[];  // [2][3][S]: high words, then low words
    for (int i = threadIdx.x; i < 6 * S; i += blockDim.x) sh_fsc[i] = 0.f;
    __syncthreads();
    float *lo = sh_fsc + 3 * S;
    const int64_t cA = ny * ny * nx * nx, cB = nz * nz * nx * nx, cC = nz * nz * ny * ny;
    const __int128 den = (__int128)cA * nz * nz;
    const __int128 S4 = (__int128)4 * S * S;
    const int64_t n = nz * ny * xh;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t kx = i % xh, row = i / xh, y = row % ny, z = row / ny;
        const int64_t kz = 2 * z > nz ? z - nz : z, ky = 2 * y > ny ? y - ny : y;
        const int64_t rn = kz * kz * cA + ky * ky * cB + kx * kx * cC;
        const __int128 t = S4 * rn;  // shell s iff s^2 den <= t < (s+1)^2 den
        if (t >= den * S * S) continue;  // rho >= 1/2
        int sh = (int)(2.f * (float)S * sqrtf((float)rn / (float)den));  // estimate, corrected below
        if (sh > S - 1) sh = S - 1;
        while (sh > 0 && (__int128)sh * sh * den > t) --sh;
        while (sh + 1 < S && (__int128)(sh + 1) * (sh + 1) * den <= t) ++sh;
        const float w = (kx == 0 || 2 * kx == nx) ? 1.f : 2.f;
        const float2 a = A[row * xp + kx], b = B[row * xp + kx];
        catomic_add(&sh_fsc[sh], &lo[sh], w * (a.x * b.x + a.y * b.y));
        catomic_add(&sh_fsc[S + sh], &lo[S + sh], w * (a.x * a.x + a.y * a.y));
        catomic_add(&sh_fsc[2 * S + sh], &lo[2 * S + sh], w * (b.x * b.x + b.y * b.y));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * S; i += blockDim.x) {
        if (sh_fsc[i] != 0.f) catomic_add(&sums[i], &sums[3 * S + i], sh_fsc[i]);
        if (lo[i] != 0.f) catomic_add(&sums[i], &sums[3 * S + i], lo[i]);
    }
}

__global__ void k_fsc_final(const float *__restrict__ sums, int S, float *__restrict__ fsc)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
        const float num = sums[s] + sums[3 * S + s];
        const float aa = sums[S + s] + sums[4 * S + s], bb = sums[2 * S + s] + sums[5 * S + s];
        const float d = sqrtf(aa) * sqrtf(bb);  // two roots: the product of the sums may overflow
        fsc[s] = d > 0.f ? num / d : 0.f;
    }
}

// The FSC's scratch: a second spectrum and the shell sums
static cubic_status_t ensure_fsc(cubic_rl_plan_s *p)
{
    cubic_status_t s = ensure_workspace(p);
    if (s != CUBIC_OK) return s;
    if (!p->ws2) {
        void *m = nullptr;
        CUBIC_CUDA(cudaMalloc(&m, spec_elems(p) * sizeof(float2)));
        p->ws2 = (float2 *)m;
    }
    if (p->fsc_cap < kFscMaxShells) {
        cudaDeviceSynchronize();
        cudaFree(p->fsc_sums);
        p->fsc_sums = nullptr;
        p->fsc_cap = 0;
        void *m = nullptr;
        CUBIC_CUDA(cudaMalloc(&m, 6 * (size_t)kFscMaxShells * sizeof(float)));
        p->fsc_sums = (float *)m;
        p->fsc_cap = kFscMaxShells;
    }
    return CUBIC_OK;
}

static cubic_status_t enqueue_fsc(cubic_rl_plan_s *p, const float *a, const float *b, int n_shells, float *fsc,
                                  cudaStream_t st)
{
    cubic_status_t s;
    if ((s = enqueue_forward3(p, a, p->ws, 1.f, st)) != CUBIC_OK) return s;
    if ((s = enqueue_forward3(p, b, p->ws2, 1.f, st)) != CUBIC_OK) return s;
    CUBIC_CUDA(cudaMemsetAsync(p->fsc_sums, 0, 6 * (size_t)n_shells * sizeof(float), st));
    k_fsc_bins<<<grid_for(p->rows * p->xh, 256, 152 * 8), 256, 6 * n_shells * sizeof(float), st>>>(
        p->ws, p->ws2, p->nz, p->ny, p->nx, p->xh, p->xp, n_shells, p->fsc_sums);
    k_fsc_final<<<(n_shells + 255) / 256, 256, 0, st>>>(p->fsc_sums, n_shells, fsc);
    CUBIC_CUDA(cudaGetLastError());
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_fsc(cubic_rl_plan_t plan, const float *a, const float *b, int n_shells, float *fsc,
                                    void *stream)
{
    if (!plan || !a || !b || !fsc) return fail(CUBIC_ERR_INVALID_ARG, "plan, a, b and fsc must be non-null");
    if (cubic_status_t g = no_linear(plan, "FSC")) return g;
    if (n_shells < 1 || n_shells > kFscMaxShells)
        return fail(CUBIC_ERR_INVALID_ARG, "n_shells must be in [1, %d]", kFscMaxShells);
    if (!aligned16(a) || !aligned16(b)) return fail(CUBIC_ERR_ALIGNMENT, "a and b must be 16-byte aligned");
    cubic_status_t s = ensure_fsc(plan);
    if (s != CUBIC_OK) return s;
    return enqueue_fsc(plan, a, b, n_shells, fsc, (cudaStream_t)stream);
}

// Single-image FSC: the sub-volumes of opposite parity, pair `pair` (z-parity 0 and
// (y, x) parities from its bits against the complementary parities), of a volume of
// dims 2h into a and b of dims h
__global__ void k_split_pair(const float *__restrict__ d, float *__restrict__ a, float *__restrict__ b, int64_t hz,
                             int64_t hy, int64_t hx, int pair)
{
    const int py = (pair >> 1) & 1, px = pair & 1;
    const int64_t ny = 2 * hy, nx = 2 * hx, H = hz * hy * hx;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < H; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = i % hx, y = (i / hx) % hy, z = i / (hx * hy);
        a[i] = d[((2 * z) * ny + 2 * y + py) * nx + 2 * x + px];
        b[i] = d[((2 * z + 1) * ny + 2 * y + 1 - py) * nx + 2 * x + 1 - px];
    }
}

// fsc[s] = the mean of the four curves in curves[4][S]
__global__ void k_mean4(const float *__restrict__ curves, int S, float *__restrict__ fsc)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x)
        fsc[s] = 0.25f * (curves[s] + curves[S + s] + curves[2 * S + s] + curves[3 * S + s]);
}

extern "C" cubic_status_t cubic_fsc_split(cubic_rl_plan_t half_plan, const float *image, int n_shells, float *fsc,
                                          void *stream)
{
    if (!half_plan || !image || !fsc) return fail(CUBIC_ERR_INVALID_ARG, "plan, image and fsc must be non-null");
    if (cubic_status_t g = no_linear(half_plan, "FSC")) return g;
    if (n_shells < 1 || n_shells > kFscMaxShells)
        return fail(CUBIC_ERR_INVALID_ARG, "n_shells must be in [1, %d]", kFscMaxShells);
    if (!aligned16(image)) return fail(CUBIC_ERR_ALIGNMENT, "image must be 16-byte aligned");
    cubic_rl_plan_s *p = half_plan;
    cubic_status_t s = ensure_fsc(p);
    if (s != CUBIC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t hb = ((size_t)p->V * sizeof(float) + 255) / 256 * 256;
    const size_t cb = (4 * (size_t)n_shells * sizeof(float) + 255) / 256 * 256;
    void *m = nullptr;
    CUBIC_CUDA(cudaMallocAsync(&m, 2 * hb + cb, st));
    float *a = (float *)m, *b = (float *)((unsigned char *)m + hb), *curves = (float *)((unsigned char *)m + 2 * hb);
    for (int pair = 0; pair < 4 && s == CUBIC_OK; ++pair) {
        k_split_pair<<<grid_for(p->V, 256), 256, 0, st>>>(image, a, b, p->nz, p->ny, p->nx, pair);
        s = enqueue_fsc(p, a, b, n_shells, curves + (size_t)pair * n_shells, st);
    }
    if (s == CUBIC_OK) k_mean4<<<(n_shells + 255) / 256, 256, 0, st>>>(curves, n_shells, fsc);
    cudaFreeAsync(m, st);
    if (s == CUBIC_OK) CUBIC_CUDA(cudaGetLastError());
    return s;
}

// ------------------------------------------------------------------ batched deconvolution
//
// Many volumes of different sizes in one CUDA graph.  For every pass, the volumes whose
// axis along that pass has a length of one of the all-lengths classes (lens.cuh) share
// one launch per class, whatever their lengths; the volumes of other lengths share one
// launch per length (k_*pass with a MultiTable).  A launch's blocks are the
// concatenation of every member volume's blocks, and each block finds its volume in a
// device-side table.  The whole n_iter sequence is captured once into a graph and
// replayed on later calls with the same arguments.

namespace {

// One multi-volume launch: the volumes whose axis has the same length, launched with
// launch shape `shape` (an index into k->xv for X, into k->yzv for Y and Z)
struct XGroup {
    const AxisKernels *k;
    MultiTable<XArgs> *tab;
    int64_t blocks;
    int shape;
};
struct YGroup {
    const AxisKernels *k;
    MultiTable<YArgs> *tab;
    int64_t blocks;
    int shape;
};
struct ZGroup {
    const AxisKernels *k;
    MultiTable<ZArgs> *tab;
    int64_t blocks;
    int shape;
};

// One all-lengths launch: the volumes of one length class
template <class Args>
struct LensGroup {
    int cls;
    LensTable<Args> *tab;
    int64_t blocks;
};

struct BatchState {
    std::vector<cubic_rl_plan_s *> plans;
    std::vector<const float *> images;
    std::vector<float *> outs;
    int n_iter = 0;
    float eps = 0.f;
    std::vector<XGroup> gx;
    std::vector<YGroup> gy;
    std::vector<ZGroup> gz;
    std::vector<LensGroup<XArgs>> lx;
    std::vector<LensGroup<YArgs>> ly;
    std::vector<LensGroup<ZArgs>> lz;
    void *dmem = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t kernel_nodes = 0;
    ~BatchState()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (dmem) cudaFree(dmem);
    }
};

std::mutex g_batch_mu;
std::vector<BatchState *> g_batches;  // most recent last; a few kept
int64_t g_batch_last_nodes = 0;

}  // namespace

static cubic_status_t enqueue_batched(BatchState &b, cudaStream_t st)
{
    for (size_t v = 0; v < b.plans.size(); ++v) {
        cubic_status_t s = enqueue_init(b.plans[v], b.images[v], b.eps, b.outs[v], st);
        if (s != CUBIC_OK) return s;
    }
    if (b.n_iter == 0) return CUBIC_OK;
    auto xstage = [&](int mode) -> cubic_status_t {
        for (const auto &g : b.lx) CUBIC_CUDA(launch_x_lens(g.cls, mode, g.tab, g.blocks, st));
        for (const XGroup &g : b.gx) CUBIC_CUDA(g.k->xv[g.shape].m[mode](g.tab, g.blocks, st));
        return CUBIC_OK;
    };
    auto ystage = [&](int inverse) -> cubic_status_t {
        for (const auto &g : b.ly) CUBIC_CUDA(launch_y_lens(g.cls, g.tab, g.blocks, inverse, st));
        for (const YGroup &g : b.gy) CUBIC_CUDA(g.k->yzv[g.shape].ym(g.tab, g.blocks, inverse, st));
        return CUBIC_OK;
    };
    auto yzy = [&](int zmode) -> cubic_status_t {
        if (cubic_status_t e = ystage(0)) return e;
        for (const auto &g : b.lz) CUBIC_CUDA(launch_z_lens(g.cls, g.tab, g.blocks, zmode, st));
        for (const ZGroup &g : b.gz) CUBIC_CUDA(g.k->yzv[g.shape].zm(g.tab, g.blocks, zmode, st));
        return ystage(1);
    };
    cubic_status_t s = xstage(XM_FWD);
    for (int k = 0; k < b.n_iter && s == CUBIC_OK; ++k) {
        if ((s = yzy(ZM_CONV)) != CUBIC_OK) break;
        if ((s = xstage(XM_RATIO)) != CUBIC_OK) break;
        if ((s = yzy(ZM_CORR)) != CUBIC_OK) break;
        s = xstage(k + 1 < b.n_iter ? XM_UPDATE : XM_FINAL);
    }
    return s;
}

// ---- launch shapes of the batched path
// For every axis length and pass (X, Y, Z) the shape comes from this table, filled by
// timing the candidates on the first batch that has the length (batch_tune); until then,
// and where tuning fails, the default shape serves.
static std::mutex g_bshape_mu;
static std::map<std::pair<int64_t, int>, int> g_bshape;  // (length, pass 0/1/2) -> variant index

// the default shapes: X with the multi launcher's line count, Y/Z the P0 x m_cols plain one
static int default_xshape(const AxisKernels *k)
{
    for (int v = 0; v < k->nx; ++v)
        if (k->xv[v].L == k->xm_lines && k->xv[v].m[XM_FWD]) return v;
    return 0;
}
static int default_yzshape(const AxisKernels *k)
{
    int first = -1;
    for (int v = 0; v < k->nyz; ++v) {
        if (!k->yzv[v].ym) continue;
        if (k->yzv[v].B == k->m_cols) return v;  // the first plain variant: P0 x m_cols
        if (first < 0) first = v;
    }
    return first < 0 ? 0 : first;
}

static int chosen_shape(int64_t len, int pass, int fallback)
{
    std::lock_guard<std::mutex> lk(g_bshape_mu);
    auto it = g_bshape.find({len, pass});
    return it == g_bshape.end() ? fallback : it->second;
}

// Host table of one group for one launch shape; returns its block count.
static int64_t fill_xtable(const BatchState &b, const std::vector<int> &vols, const AxisKernels *k, int shape,
                    MultiTable<XArgs> *t)
{
    t->nvol = (int)vols.size();
    int64_t blocks = 0;
    const int L = k->xv[shape].L;
    for (int i = 0; i < t->nvol; ++i) {
        cubic_rl_plan_s *p = b.plans[vols[i]];
        XArgs a = x_args(p);
        a.spec_in = p->ws;
        a.spec_out = p->ws;
        a.src = b.outs[vols[i]];
        a.u = b.outs[vols[i]];
        a.dst = b.outs[vols[i]];
        a.d = b.images[vols[i]];
        a.eps = b.eps;
        t->args[i] = a;
        t->prefix[i] = blocks;
        blocks += ((p->rows + 1) / 2 + L - 1) / L;
    }
    t->prefix[t->nvol] = blocks;
    return blocks;
}

static int64_t fill_ytable(const BatchState &b, const std::vector<int> &vols, const AxisKernels *k, int shape,
                    MultiTable<YArgs> *t)
{
    t->nvol = (int)vols.size();
    int64_t blocks = 0;
    const int B = k->yzv[shape].B;
    for (int i = 0; i < t->nvol; ++i) {
        cubic_rl_plan_s *p = b.plans[vols[i]];
        t->args[i] = y_args(p, p->ws, 0, 0, p->xh);
        t->prefix[i] = blocks;
        blocks += (p->xh + B - 1) / B * p->nz;
    }
    t->prefix[t->nvol] = blocks;
    return blocks;
}

static int64_t fill_ztable(const BatchState &b, const std::vector<int> &vols, const AxisKernels *k, int shape,
                    MultiTable<ZArgs> *t)
{
    t->nvol = (int)vols.size();
    int64_t blocks = 0;
    const int B = k->yzv[shape].B;
    for (int i = 0; i < t->nvol; ++i) {
        cubic_rl_plan_s *p = b.plans[vols[i]];
        t->args[i] = z_args(p, p->ws, ZM_CONV, 1.f, 0, p->xh);
        t->prefix[i] = blocks;
        blocks += (p->xh + B - 1) / B * p->ny;
    }
    t->prefix[t->nvol] = blocks;
    return blocks;
}

using LenGroups = std::map<int64_t, std::vector<int>>;

// Host tables of the all-lengths launches of one class (volumes in order of length);
// each returns the launch's block count.
static int64_t fill_lens_x(const BatchState &b, const std::vector<int> &vols, LensTable<XArgs> *t)
{
    t->nvol = (int)vols.size();
    int64_t blocks = 0;
    for (int i = 0; i < t->nvol; ++i) {
        cubic_rl_plan_s *p = b.plans[vols[i]];
        XArgs a = x_args(p);
        a.spec_in = p->ws;
        a.spec_out = p->ws;
        a.src = b.outs[vols[i]];
        a.u = b.outs[vols[i]];
        a.dst = b.outs[vols[i]];
        a.d = b.images[vols[i]];
        a.eps = b.eps;
        t->args[i] = a;
        t->len[i] = (int)p->nx;
        t->prefix[i] = blocks;
        blocks += lens_x_blocks((int)p->nx, p->rows);
    }
    t->prefix[t->nvol] = blocks;
    return blocks;
}

static int64_t fill_lens_y(const BatchState &b, const std::vector<int> &vols, LensTable<YArgs> *t)
{
    t->nvol = (int)vols.size();
    int64_t blocks = 0;
    for (int i = 0; i < t->nvol; ++i) {
        cubic_rl_plan_s *p = b.plans[vols[i]];
        t->args[i] = y_args(p, p->ws, 0, 0, p->xh);
        t->len[i] = (int)p->ny;
        t->prefix[i] = blocks;
        blocks += lens_col_blocks((int)p->ny, p->nz * p->xh);
    }
    t->prefix[t->nvol] = blocks;
    return blocks;
}

static int64_t fill_lens_z(const BatchState &b, const std::vector<int> &vols, LensTable<ZArgs> *t)
{
    t->nvol = (int)vols.size();
    int64_t blocks = 0;
    for (int i = 0; i < t->nvol; ++i) {
        cubic_rl_plan_s *p = b.plans[vols[i]];
        t->args[i] = z_args(p, p->ws, ZM_CONV, 1.f, 0, p->xh);
        t->len[i] = (int)p->nz;
        t->prefix[i] = blocks;
        blocks += lens_col_blocks((int)p->nz, p->ny * p->xh);
    }
    t->prefix[t->nvol] = blocks;
    return blocks;
}

// Times every candidate shape of every group whose length has no chosen shape yet, on
// the batch's own buffers, and records the fastest: X by a ratio and an update launch, Y
// by a forward and an inverse, Z by one product.  The buffers are left with arbitrary
// finite contents; the batched run starts from its images anyway.
static cubic_status_t batch_tune(BatchState &b, const LenGroups &byx, const LenGroups &byy, const LenGroups &byz,
                          cudaStream_t st)
{
    auto known = [&](int64_t len, int pass) {
        std::lock_guard<std::mutex> lk(g_bshape_mu);
        return g_bshape.count({len, pass}) > 0;
    };
    bool any = false;
    for (auto &kv : byx) any |= !known(kv.first, 0);
    for (auto &kv : byy) any |= !known(kv.first, 1);
    for (auto &kv : byz) any |= !known(kv.first, 2);
    if (!any) return CUBIC_OK;
    // finite data everywhere: each volume's start and the spectrum of it
    for (size_t v = 0; v < b.plans.size(); ++v) {
        cubic_rl_plan_s *p = b.plans[v];
        cubic_status_t s = enqueue_init(p, b.images[v], b.eps, b.outs[v], st);
        if (s != CUBIC_OK) return s;
        if ((s = enqueue_forward3(p, b.outs[v], p->ws, 1.f / (float)p->V, st)) != CUBIC_OK) return s;
    }
    const size_t tsz = std::max({sizeof(MultiTable<XArgs>), sizeof(MultiTable<YArgs>), sizeof(MultiTable<ZArgs>)});
    std::vector<unsigned char> host(tsz, 0);
    void *dtab = nullptr;
    CUBIC_CUDA(cudaMalloc(&dtab, tsz));
    auto nothing = []() -> cubic_status_t { return CUBIC_OK; };
    cubic_status_t s = CUBIC_OK;
    auto upload = [&]() -> cubic_status_t {
        CUBIC_CUDA(cudaMemcpyAsync(dtab, host.data(), tsz, cudaMemcpyHostToDevice, st));
        return CUBIC_OK;
    };
    auto record = [&](int64_t len, int pass, int v) {
        std::lock_guard<std::mutex> lk(g_bshape_mu);
        g_bshape[{len, pass}] = v;
    };
    for (auto &kv : byx) {
        if (s != CUBIC_OK || known(kv.first, 0)) continue;
        const AxisKernels *k = find_axis(kv.first);
        int best = default_xshape(k);
        float best_ms = 1e30f;
        for (int v = 0; v < k->nx && s == CUBIC_OK; ++v) {
            auto *t = reinterpret_cast<MultiTable<XArgs> *>(host.data());
            const int64_t blocks = fill_xtable(b, kv.second, k, v, t);
            if ((s = upload()) != CUBIC_OK) break;
            auto *tab = reinterpret_cast<const MultiTable<XArgs> *>(dtab);
            float ms = 0.f;
            s = time_best(st, nothing, [&]() -> cubic_status_t {
                CUBIC_CUDA(k->xv[v].m[XM_RATIO](tab, blocks, st));
                CUBIC_CUDA(k->xv[v].m[XM_UPDATE](tab, blocks, st));
                return CUBIC_OK;
            }, &ms);
            if (ms < best_ms) { best_ms = ms; best = v; }
        }
        if (s == CUBIC_OK) record(kv.first, 0, best);
    }
    for (int pass = 1; pass <= 2 && s == CUBIC_OK; ++pass) {
        for (auto &kv : (pass == 1 ? byy : byz)) {
            if (s != CUBIC_OK || known(kv.first, pass)) continue;
            const AxisKernels *k = find_axis(kv.first);
            int best = default_yzshape(k);
            float best_ms = 1e30f;
            for (int v = 0; v < k->nyz && s == CUBIC_OK; ++v) {
                if (!k->yzv[v].ym) continue;  // TMA variants have no multi-volume form
                int64_t blocks;
                if (pass == 1) blocks = fill_ytable(b, kv.second, k, v, reinterpret_cast<MultiTable<YArgs> *>(host.data()));
                else blocks = fill_ztable(b, kv.second, k, v, reinterpret_cast<MultiTable<ZArgs> *>(host.data()));
                if ((s = upload()) != CUBIC_OK) break;
                float ms = 0.f;
                s = time_best(st, nothing, [&]() -> cubic_status_t {
                    if (pass == 1) {
                        auto *tab = reinterpret_cast<const MultiTable<YArgs> *>(dtab);
                        CUBIC_CUDA(k->yzv[v].ym(tab, blocks, 0, st));
                        CUBIC_CUDA(k->yzv[v].ym(tab, blocks, 1, st));
                    } else {
                        auto *tab = reinterpret_cast<const MultiTable<ZArgs> *>(dtab);
                        CUBIC_CUDA(k->yzv[v].zm(tab, blocks, ZM_CONV, st));
                    }
                    return CUBIC_OK;
                }, &ms);
                if (ms < best_ms) { best_ms = ms; best = v; }
            }
            if (s == CUBIC_OK) record(kv.first, pass, best);
        }
    }
    cudaStreamSynchronize(st);
    cudaFree(dtab);
    return s;
}

// Group volumes by axis length, tune the launch shapes of new lengths, and build the
// device tables.
static cubic_status_t build_batch(BatchState &b, cudaStream_t st)
{
    const int n = (int)b.plans.size();
    // all-lengths classes where the axis length has one (their line indices are 32-bit),
    // else a launch per length
    LenGroups byx, byy, byz;
    LenGroups lensx[kLensClasses], lensy[kLensClasses], lensz[kLensClasses];  // class -> length -> volumes
    const int64_t kLines32 = (int64_t)1 << 31;
    for (int v = 0; v < n; ++v) {
        const cubic_rl_plan_s *p = b.plans[v];
        const int cx = lens_class(p->nx), cy = lens_class(p->ny), cz = lens_class(p->nz);
        if (cx >= 0) lensx[cx][p->nx].push_back(v);
        else byx[p->nx].push_back(v);
        if (cy >= 0 && p->nz * p->xh < kLines32) lensy[cy][p->ny].push_back(v);
        else byy[p->ny].push_back(v);
        if (cz >= 0 && p->ny * p->xh < kLines32) lensz[cz][p->nz].push_back(v);
        else byz[p->nz].push_back(v);
    }
    cubic_status_t s = batch_tune(b, byx, byy, byz, st);
    if (s != CUBIC_OK) return s;
    auto flat = [](const LenGroups &g) {
        std::vector<int> vols;
        for (auto &kv : g) vols.insert(vols.end(), kv.second.begin(), kv.second.end());
        return vols;
    };
    size_t nlens = 0;
    for (int c = 0; c < kLensClasses; ++c) nlens += !lensx[c].empty() + !lensy[c].empty() + !lensz[c].empty();
    const size_t ntab = byx.size() + byy.size() + byz.size() + nlens;
    const size_t tsz = std::max({sizeof(MultiTable<XArgs>), sizeof(MultiTable<YArgs>), sizeof(MultiTable<ZArgs>),
                                 sizeof(LensTable<XArgs>), sizeof(LensTable<YArgs>), sizeof(LensTable<ZArgs>)});
    const size_t stride = (tsz + 255) / 256 * 256;
    std::vector<unsigned char> host(stride * ntab, 0);
    CUBIC_CUDA(cudaMalloc(&b.dmem, host.size()));
    unsigned char *dbase = (unsigned char *)b.dmem;
    size_t slot = 0;
    for (auto &kv : byx) {
        const AxisKernels *k = find_axis(kv.first);
        const int shape = chosen_shape(kv.first, 0, default_xshape(k));
        const int64_t blocks =
            fill_xtable(b, kv.second, k, shape, reinterpret_cast<MultiTable<XArgs> *>(host.data() + slot * stride));
        b.gx.push_back({k, reinterpret_cast<MultiTable<XArgs> *>(dbase + slot * stride), blocks, shape});
        ++slot;
    }
    for (auto &kv : byy) {
        const AxisKernels *k = find_axis(kv.first);
        const int shape = chosen_shape(kv.first, 1, default_yzshape(k));
        const int64_t blocks =
            fill_ytable(b, kv.second, k, shape, reinterpret_cast<MultiTable<YArgs> *>(host.data() + slot * stride));
        b.gy.push_back({k, reinterpret_cast<MultiTable<YArgs> *>(dbase + slot * stride), blocks, shape});
        ++slot;
    }
    for (auto &kv : byz) {
        const AxisKernels *k = find_axis(kv.first);
        const int shape = chosen_shape(kv.first, 2, default_yzshape(k));
        const int64_t blocks =
            fill_ztable(b, kv.second, k, shape, reinterpret_cast<MultiTable<ZArgs> *>(host.data() + slot * stride));
        b.gz.push_back({k, reinterpret_cast<MultiTable<ZArgs> *>(dbase + slot * stride), blocks, shape});
        ++slot;
    }
    for (int c = 0; c < kLensClasses; ++c) {
        if (!lensx[c].empty()) {
            const int64_t blocks =
                fill_lens_x(b, flat(lensx[c]), reinterpret_cast<LensTable<XArgs> *>(host.data() + slot * stride));
            b.lx.push_back({c, reinterpret_cast<LensTable<XArgs> *>(dbase + slot * stride), blocks});
            ++slot;
        }
        if (!lensy[c].empty()) {
            const int64_t blocks =
                fill_lens_y(b, flat(lensy[c]), reinterpret_cast<LensTable<YArgs> *>(host.data() + slot * stride));
            b.ly.push_back({c, reinterpret_cast<LensTable<YArgs> *>(dbase + slot * stride), blocks});
            ++slot;
        }
        if (!lensz[c].empty()) {
            const int64_t blocks =
                fill_lens_z(b, flat(lensz[c]), reinterpret_cast<LensTable<ZArgs> *>(host.data() + slot * stride));
            b.lz.push_back({c, reinterpret_cast<LensTable<ZArgs> *>(dbase + slot * stride), blocks});
            ++slot;
        }
    }
    auto too_many = [](int64_t blocks) { return blocks > 0x7fffffff; };
    for (const auto &g : b.lx) if (too_many(g.blocks)) return fail(CUBIC_ERR_INVALID_ARG, "batch too large for one launch");
    for (const auto &g : b.ly) if (too_many(g.blocks)) return fail(CUBIC_ERR_INVALID_ARG, "batch too large for one launch");
    for (const auto &g : b.lz) if (too_many(g.blocks)) return fail(CUBIC_ERR_INVALID_ARG, "batch too large for one launch");
    CUBIC_CUDA(cudaMemcpy(b.dmem, host.data(), host.size(), cudaMemcpyHostToDevice));
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_deconvolve_batched(const cubic_rl_plan_t *plans, int n, const float *const *images,
                                                      int n_iter, float eps, float *const *outs, void *stream)
{
    if (!plans || !images || !outs || n < 1 || n > kMaxBatch)
        return fail(CUBIC_ERR_INVALID_ARG, "plans, images, outs must be non-null and 1 <= n <= %d", kMaxBatch);
    if (n_iter < 0) return fail(CUBIC_ERR_INVALID_ARG, "n_iter must be >= 0");
    if (!(eps > 0.f) || !(eps < INFINITY)) return fail(CUBIC_ERR_INVALID_ARG, "eps must be finite and > 0");
    for (int v = 0; v < n; ++v) {
        if (!plans[v] || !images[v] || !outs[v]) return fail(CUBIC_ERR_INVALID_ARG, "volume %d: null pointer", v);
        if (cubic_status_t g = no_linear(plans[v], "batched deconvolution")) return g;
        if (!aligned16(images[v]) || !aligned16(outs[v]))
            return fail(CUBIC_ERR_ALIGNMENT, "volume %d: image and out must be 16-byte aligned", v);
        if (overlaps(images[v], outs[v], (size_t)plans[v]->V * sizeof(float)))
            return fail(CUBIC_ERR_INVALID_ARG, "volume %d: out must not overlap image", v);
        for (int w = 0; w < v; ++w) {
            if (plans[w] == plans[v]) return fail(CUBIC_ERR_INVALID_ARG, "volumes %d and %d share a plan", w, v);
            if (overlaps(outs[w], outs[v], std::min(plans[w]->V, plans[v]->V) * sizeof(float)))
                return fail(CUBIC_ERR_INVALID_ARG, "volumes %d and %d have overlapping outputs", w, v);
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    BatchState *hit = nullptr;
    for (BatchState *b : g_batches) {
        if ((int)b->plans.size() != n || b->n_iter != n_iter || b->eps != eps) continue;
        bool same = true;
        for (int v = 0; v < n && same; ++v)
            same = b->plans[v] == plans[v] && b->images[v] == images[v] && b->outs[v] == outs[v];
        if (same) hit = b;
    }
    if (!hit) {
        for (int v = 0; v < n; ++v) {
            cubic_status_t s = ensure_workspace(plans[v]);
            if (s != CUBIC_OK) return s;
        }
        BatchState *b = new (std::nothrow) BatchState();
        if (!b) return fail(CUBIC_ERR_OUT_OF_MEMORY, "host allocation failed");
        b->plans.assign(plans, plans + n);
        b->images.assign(images, images + n);
        b->outs.assign(outs, outs + n);
        b->n_iter = n_iter;
        b->eps = eps;
        cubic_status_t s = build_batch(*b, st);
        // capture the sequence on a private stream, then keep the instantiated graph
        cudaStream_t cap = nullptr;
        if (s == CUBIC_OK && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
            s = fail(CUBIC_ERR_CUDA, "stream creation failed");
        if (s == CUBIC_OK) {
            if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                s = fail(CUBIC_ERR_CUDA, "graph capture failed to start");
            else {
                cubic_status_t se = enqueue_batched(*b, cap);
                cudaError_t ee = cudaStreamEndCapture(cap, &b->graph);
                if (se != CUBIC_OK) s = se;
                else if (ee != cudaSuccess) s = fail(CUBIC_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ee));
            }
        }
        if (s == CUBIC_OK && cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
            s = fail(CUBIC_ERR_CUDA, "graph instantiation failed");
        if (s == CUBIC_OK) cudaGraphGetNodes(b->graph, nullptr, &b->kernel_nodes);
        if (cap) cudaStreamDestroy(cap);
        if (s != CUBIC_OK) {
            delete b;
            return s;
        }
        if (g_batches.size() >= 4) {
            cudaDeviceSynchronize();
            delete g_batches.front();
            g_batches.erase(g_batches.begin());
        }
        g_batches.push_back(b);
        hit = b;
    }
    g_batch_last_nodes = (int64_t)hit->kernel_nodes;
    CUBIC_CUDA(cudaGraphLaunch(hit->exec, st));
    return CUBIC_OK;
}

extern "C" int64_t cubic_rl_batched_graph_nodes(void)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    return g_batch_last_nodes;
}

// ------------------------------------------------------------------ allocation-free entry point
//
// For callers that cannot call cudaMalloc: frameworks whose device memory is entirely
// reserved by their own pool allocator, plug-in code that its host application does not
// let allocate, and latency-critical loops that cannot take cudaMalloc's implicit
// device-wide synchronisation.  Everything a deconvolution needs beyond its inputs and
// outputs (PSF spectrum, work spectrum, twiddles, reduction partials, error word) lives
// in one fixed file-scope device array.
//
// Layout of the array: the device error word alone in the first 256 bytes, at the same
// place for every volume shape (so a timeout stays there until it is read), then H, the
// work spectrum, the twiddles and the reduction partials of the current call.

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_ptr[64];  // device address of the array, per device ordinal

static size_t align256(size_t n) { return (n + 255) / 256 * 256; }

// The array's device address on the current device, looked up once per device (with that
// device current) and kept for the life of the process.
static cubic_status_t noalloc_base(unsigned char **base, int *device)
{
    int dev = 0;
    CUBIC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CUBIC_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *addr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
        if (e != cudaSuccess || !addr) return fail(CUBIC_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = (unsigned char *)addr;
    }
    *base = g_noalloc_ptr[dev];
    *device = dev;
    return CUBIC_OK;
}

extern "C" cubic_status_t cubic_rl_deconvolve_noalloc(const int64_t dims[3], const float *psf, const float *image,
                                                      int n_iter, float eps, float *out, void *stream)
{
    if (!dims || !psf || !image || !out) return fail(CUBIC_ERR_INVALID_ARG, "dims, psf, image and out must be non-null");
    for (int i = 0; i < 3; ++i)
        if (dims[i] < 1 || !find_axis(dims[i]))
            return fail(CUBIC_ERR_UNSUPPORTED_SIZE, "axis %d has unsupported length %lld", i, (long long)dims[i]);
    if (dims[0] > 65535 || dims[1] > 65535) return fail(CUBIC_ERR_UNSUPPORTED_SIZE, "nz and ny must be <= 65535");
    if (n_iter < 0) return fail(CUBIC_ERR_INVALID_ARG, "n_iter must be >= 0");
    if (!(eps > 0.f) || !(eps < INFINITY)) return fail(CUBIC_ERR_INVALID_ARG, "eps must be finite and > 0");
    if (!aligned16(psf) || !aligned16(image) || !aligned16(out))
        return fail(CUBIC_ERR_ALIGNMENT, "psf, image and out must be 16-byte aligned");

    // a plan that lives on this stack frame; its device buffers are carved out of the array.
    // It never takes the real-spectrum Z passes: deciding that the PSF is point-symmetric
    // takes a host synchronisation, so H stays complex (same result to float rounding)
    cubic_rl_plan_s p;
    p.nz = dims[0];
    p.ny = dims[1];
    p.nx = dims[2];
    p.V = p.nz * p.ny * p.nx;
    p.rows = p.nz * p.ny;
    p.xh = p.nx / 2 + 1;
    p.xp = (p.xh + 15) / 16 * 16;
    p.kx = find_axis(p.nx);
    p.ky = find_axis(p.ny);
    p.kz = find_axis(p.nz);
    if (overlaps(image, out, (size_t)p.V * sizeof(float)))
        return fail(CUBIC_ERR_INVALID_ARG, "out must not overlap image");
    const size_t err_bytes = 256;
    const size_t spec_bytes = align256(spec_elems(&p) * sizeof(float2));
    const size_t tw_bytes = align256((size_t)(p.nx + p.ny + p.nz) * sizeof(float2));
    const size_t red_bytes = align256((kReduceBlocks + 1) * sizeof(double));
    const size_t need = err_bytes + 2 * spec_bytes + tw_bytes + red_bytes;
    if (need > kNoAllocScratchBytes)
        return fail(CUBIC_ERR_UNSUPPORTED_SIZE,
                    "volume needs %zu bytes of scratch; the allocation-free entry point has %zu "
                    "(nz*ny*(nx/2+1 rounded up to 16) must stay below about 2^19)",
                    need, kNoAllocScratchBytes);

    unsigned char *base = nullptr;
    cubic_status_t s = noalloc_base(&base, &p.device);
    if (s != CUBIC_OK) return s;
    p.err = (unsigned *)base;
    p.H = (float2 *)(base + err_bytes);
    p.ws = (float2 *)(base + err_bytes + spec_bytes);
    p.own_ws = false;
    p.tw = (float2 *)(base + err_bytes + 2 * spec_bytes);
    p.tw_x = p.tw;
    p.tw_y = p.tw + p.nx;
    p.tw_z = p.tw + p.nx + p.ny;
    p.partial = (double *)(base + err_bytes + 2 * spec_bytes + tw_bytes);
    tuned_variants(&p);

    // The array keeps the previous call's contents.  Everything but the error word is
    // rewritten below before it is read; the error word starts at zero (static
    // initialisation) and only cubic_rl_noalloc_status clears it.
    cudaStream_t st = (cudaStream_t)stream;
    k_twiddles<<<grid_for(p.nx, 128, 1 << 20), 128, 0, st>>>(p.tw_x, (int)p.nx);
    k_twiddles<<<grid_for(p.ny, 128, 1 << 20), 128, 0, st>>>(p.tw_y, (int)p.ny);
    k_twiddles<<<grid_for(p.nz, 128, 1 << 20), 128, 0, st>>>(p.tw_z, (int)p.nz);
    CUBIC_CUDA(cudaGetLastError());
    s = load_psf(&p, psf, st);
    if (s != CUBIC_OK) return s;
    return enqueue_rl(&p, image, n_iter, eps, out, p.ws, st);
}

extern "C" cubic_status_t cubic_rl_noalloc_status(void *stream)
{
    unsigned char *base = nullptr;
    int dev = 0;
    cubic_status_t s = noalloc_base(&base, &dev);
    if (s != CUBIC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned word = 0;
    CUBIC_CUDA(cudaMemcpyAsync(&word, base, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CUBIC_CUDA(cudaStreamSynchronize(st));
    if (word) {
        CUBIC_CUDA(cudaMemsetAsync(base, 0, sizeof(unsigned), st));
        CUBIC_CUDA(cudaStreamSynchronize(st));
        return fail(CUBIC_ERR_TIMEOUT, "a device wait of an allocation-free call timed out (error word 0x%x)", word);
    }
    return CUBIC_OK;
}
