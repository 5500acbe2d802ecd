// capi.cu -- the extern "C" boundary (include/cubic_rl.h) and the host-side
// plan: argument validation, device buffers, and the enqueueing of the pass
// kernels that make up each Richardson-Lucy iteration.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>

#include "../../include/cubic_rl.h"
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

static void init_table()
{
    register_shard<0>(g_table);
    register_shard<1>(g_table);
    register_shard<2>(g_table);
    register_shard<3>(g_table);
    register_shard<4>(g_table);
    register_shard<5>(g_table);
    register_shard<6>(g_table);
    register_shard<7>(g_table);
}

const AxisKernels *cubic::find_axis(int64_t n)
{
    std::call_once(g_table_once, init_table);
    for (int i = 0; i < kNumLengths; ++i)
        if (kLengths[i] == n) return g_table[i].n == n ? &g_table[i] : nullptr;
    return nullptr;
}

int cubic::supported_lengths(const int **out)
{
    if (out) *out = kLengths;
    return kNumLengths;
}

extern "C" int cubic_rl_supported_length(int64_t n) { return find_axis(n) != nullptr; }

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

// Flux sum in double: per-block partial sums, then one block folds them.
constexpr int kReduceThreads = 256;
constexpr int kReduceBlocks = 1024;

__global__ void __launch_bounds__(kReduceThreads) k_sum_partial(const float *__restrict__ x, int64_t n,
                                                                double *__restrict__ partial)
{
    __shared__ double sh[kReduceThreads / 32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += (double)x[i];
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

// u0 = max(sum / V, eps) everywhere.
__global__ void k_fill_initial(float *__restrict__ u, int64_t V, const double *__restrict__ sum, float eps)
{
    const double m = sum[0] / (double)V;
    const float v = m > (double)eps ? (float)m : eps;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x)
        u[i] = v;
}

static unsigned grid_for(int64_t n, int threads, int64_t cap = 152 * 32)
{
    int64_t g = (n + threads - 1) / threads;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

// ------------------------------------------------------------------ plan

struct cubic_rl_plan_s {
    int device = 0;
    int64_t nz = 0, ny = 0, nx = 0, V = 0, rows = 0, xh = 0, xp = 0;
    const AxisKernels *kx = nullptr, *ky = nullptr, *kz = nullptr;
    float2 *H = nullptr;        // [nz][ny][xp], owned
    float2 *tw = nullptr;       // twiddles: x | y | z, owned
    float2 *tw_x = nullptr, *tw_y = nullptr, *tw_z = nullptr;
    double *partial = nullptr;  // kReduceBlocks + 1 doubles, owned
    float2 *ws = nullptr;       // spectrum work array
    bool own_ws = false;
};

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static size_t spec_elems(const cubic_rl_plan_s *p) { return (size_t)p->nz * p->ny * p->xp; }

static cubic_status_t ensure_workspace(cubic_rl_plan_s *p)
{
    if (p->ws) return CUBIC_OK;
    void *w = nullptr;
    CUBIC_CUDA(cudaMalloc(&w, spec_elems(p) * sizeof(float2)));
    p->ws = (float2 *)w;
    p->own_ws = true;
    return CUBIC_OK;
}

// Forward 3D real-to-half-complex transform of `real` into `spec`, optionally
// scaled (scale applies in the Z pass).
static cubic_status_t enqueue_forward3(cubic_rl_plan_s *p, const float *real, float2 *spec, float scale,
                                       cudaStream_t st)
{
    XArgs xa{};
    xa.spec_out = spec;
    xa.src = real;
    xa.tw = p->tw_x;
    xa.rows = p->rows;
    xa.xp = p->xp;
    CUBIC_CUDA(p->kx->x[XM_FWD](xa, st));
    YArgs ya{spec, p->tw_y, p->nz, p->xh, p->xp, 0};
    CUBIC_CUDA(p->ky->y(ya, st));
    ZArgs za{spec, nullptr, p->tw_z, p->ny, p->xh, p->xp, ZM_FWD_SCALE, scale};
    CUBIC_CUDA(p->kz->z(za, st));
    return CUBIC_OK;
}

// Y forward, Z (product with H or conj H), Y inverse on the plan's spectrum.
static cubic_status_t enqueue_yzy(cubic_rl_plan_s *p, float2 *spec, int zmode, cudaStream_t st)
{
    YArgs ya{spec, p->tw_y, p->nz, p->xh, p->xp, 0};
    CUBIC_CUDA(p->ky->y(ya, st));
    ZArgs za{spec, p->H, p->tw_z, p->ny, p->xh, p->xp, zmode, 1.f};
    CUBIC_CUDA(p->kz->z(za, st));
    ya.inverse = 1;
    CUBIC_CUDA(p->ky->y(ya, st));
    return CUBIC_OK;
}

static cubic_status_t load_psf(cubic_rl_plan_s *p, const float *psf, cudaStream_t st)
{
    cubic_status_t s = ensure_workspace(p);
    if (s != CUBIC_OK) return s;
    // the shifted real PSF fits in the workspace (xp >= nx/2+1 complex >= nx floats)
    float *h0 = (float *)p->ws;
    k_center_to_origin<<<grid_for(p->V, 256), 256, 0, st>>>(psf, h0, p->nz, p->ny, p->nx);
    CUBIC_CUDA(cudaGetLastError());
    return enqueue_forward3(p, h0, p->H, (float)(1.0 / (double)p->V), st);
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
    cudaStream_t st = (cudaStream_t)stream;
    p->nz = dims[0];
    p->ny = dims[1];
    p->nx = dims[2];
    p->V = p->nz * p->ny * p->nx;
    p->rows = p->nz * p->ny;
    p->xh = p->nx / 2 + 1;
    p->xp = (p->xh + 15) / 16 * 16;
    p->kx = find_axis(p->nx);
    p->ky = find_axis(p->ny);
    p->kz = find_axis(p->nz);

    cubic_status_t s = CUBIC_OK;
    auto bail = [&](cubic_status_t st_) {
        cubic_rl_plan_destroy(p);
        return st_;
    };
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) return bail(fail(CUBIC_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e)));
    void *mem = nullptr;
    e = cudaMalloc(&mem, spec_elems(p) * sizeof(float2));
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
    if (plan->own_ws) cudaFree(plan->ws);
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

// The n_iter-iteration sequence, enqueued on `st`.
static cubic_status_t enqueue_rl(cubic_rl_plan_s *p, const float *image, int n_iter, float eps, float *out,
                                 float2 *spec, cudaStream_t st)
{
    // u0 = max(mean(image), eps)
    k_sum_partial<<<kReduceBlocks, kReduceThreads, 0, st>>>(image, p->V, p->partial);
    k_sum_final<<<1, kReduceThreads, 0, st>>>(p->partial, kReduceBlocks, p->partial + kReduceBlocks);
    k_fill_initial<<<grid_for(p->V, 256), 256, 0, st>>>(out, p->V, p->partial + kReduceBlocks, eps);
    CUBIC_CUDA(cudaGetLastError());
    if (n_iter == 0) return CUBIC_OK;

    XArgs xa{};
    xa.spec_in = spec;
    xa.spec_out = spec;
    xa.src = out;
    xa.u = out;
    xa.dst = out;
    xa.d = image;
    xa.tw = p->tw_x;
    xa.rows = p->rows;
    xa.xp = p->xp;
    xa.eps = eps;
    CUBIC_CUDA(p->kx->x[XM_FWD](xa, st));  // spectrum of u0
    cubic_status_t s;
    for (int k = 0; k < n_iter; ++k) {
        if ((s = enqueue_yzy(p, spec, ZM_CONV, st)) != CUBIC_OK) return s;   // b = h * u
        CUBIC_CUDA(p->kx->x[XM_RATIO](xa, st));                              // r = d / max(b, eps)
        if ((s = enqueue_yzy(p, spec, ZM_CORR, st)) != CUBIC_OK) return s;   // q = h (flipped) * r
        CUBIC_CUDA(p->kx->x[k + 1 < n_iter ? XM_UPDATE : XM_FINAL](xa, st)); // u = u * q
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
    XArgs xa{};
    xa.spec_in = plan->ws;
    xa.spec_out = plan->ws;
    xa.src = in;
    xa.dst = out;
    xa.tw = plan->tw_x;
    xa.rows = plan->rows;
    xa.xp = plan->xp;
    CUBIC_CUDA(plan->kx->x[XM_FWD](xa, st));
    if ((s = enqueue_yzy(plan, plan->ws, flipped ? ZM_CORR : ZM_CONV, st)) != CUBIC_OK) return s;
    CUBIC_CUDA(plan->kx->x[XM_INV](xa, st));
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
    if (!aligned16(in) || !aligned16(spec)) return fail(CUBIC_ERR_ALIGNMENT, "in and spec must be 16-byte aligned");
    return enqueue_forward3(plan, in, (float2 *)spec, 1.f, (cudaStream_t)stream);
}

extern "C" cubic_status_t cubic_rl_fft3_inverse(cubic_rl_plan_t plan, void *spec, float *out, void *stream)
{
    if (!plan || !out || !spec) return fail(CUBIC_ERR_INVALID_ARG, "plan, spec and out must be non-null");
    if (!aligned16(out) || !aligned16(spec)) return fail(CUBIC_ERR_ALIGNMENT, "out and spec must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    float2 *sp = (float2 *)spec;
    ZArgs za{sp, nullptr, plan->tw_z, plan->ny, plan->xh, plan->xp, ZM_INV_SCALE, (float)(1.0 / (double)plan->V)};
    CUBIC_CUDA(plan->kz->z(za, st));
    YArgs ya{sp, plan->tw_y, plan->nz, plan->xh, plan->xp, 1};
    CUBIC_CUDA(plan->ky->y(ya, st));
    XArgs xa{};
    xa.spec_in = sp;
    xa.dst = out;
    xa.tw = plan->tw_x;
    xa.rows = plan->rows;
    xa.xp = plan->xp;
    CUBIC_CUDA(plan->kx->x[XM_INV](xa, st));
    return CUBIC_OK;
}
