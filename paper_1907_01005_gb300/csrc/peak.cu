// FMA throughput probe: the FP32 / FP64 ALU peaks that the roofline of the
// cell kernels and of the FP64 Gram is reported against.  Each thread runs
// eight independent FMA chains so that latency is hidden; the grid covers
// every SM several times.
#include <cmath>
#include <cstring>
#include <mutex>

#include "fe_internal.h"

namespace femf {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T* out, int64_t iters, T a, T b) {
    T x0 = T(threadIdx.x), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
    T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    // thread 0 records its sum in the CTA's slot (every CTA runs the same
    // chains, so every slot gets the same value, which the host checks);
    // the compare keeps the other threads' chains alive
    if (threadIdx.x == 0 || s == T(-1.2345)) out[blockIdx.x] = s;
}

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2,%3};\n mov.b64 rb, {%4,%5};\n"
        " mov.b64 rc, {%6,%7};\n fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0,%1}, rd;\n}\n"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// packed FP32x2 chains: 8 chains of two lanes each
__global__ void __launch_bounds__(256) fma2_chains(float* out, int64_t iters, float a, float b) {
    const float2 A = make_float2(a, a), B = make_float2(b, b);
    float2 x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = make_float2(float(threadIdx.x + c), float(threadIdx.x - c));
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < 8; ++c) x[c] = fma2(x[c], A, B);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c].x + x[c].y;
    if (threadIdx.x == 0 || s == -1.2345f) out[blockIdx.x] = s;
}

}  // namespace

// Thread 0's chain sum, computed on the host with the same IEEE fused
// multiply-adds and the same order of additions as the kernels (FE_F64,
// FE_F32, or 3 for the packed FP32x2 chains, whose two halves start at c and
// at the unsigned difference 0 - c, i.e. 2^32 - c rounded to FP32).  Used to
// check what the kernels stored in the sink.
static double chain_sum_thread0(int dtype, int64_t iters) {
    if (dtype == FE_F64) {
        double x[8];
        for (int c = 0; c < 8; ++c) x[c] = double(c);
        for (int64_t i = 0; i < iters * 16; ++i)
            for (int c = 0; c < 8; ++c) x[c] = std::fma(x[c], 0.999999, 1e-7);
        return ((x[0] + x[1]) + (x[2] + x[3])) + ((x[4] + x[5]) + (x[6] + x[7]));
    }
    if (dtype == 3) {
        float a[8], b[8];
        for (int c = 0; c < 8; ++c) { a[c] = float(c); b[c] = float(0u - (unsigned)c); }
        for (int64_t i = 0; i < iters * 8; ++i)
            for (int c = 0; c < 8; ++c) {
                a[c] = std::fma(a[c], 0.999999f, 1e-7f);
                b[c] = std::fma(b[c], 0.999999f, 1e-7f);
            }
        float s = 0.f;
        for (int c = 0; c < 8; ++c) s += a[c] + b[c];
        return s;
    }
    float x[8];
    for (int c = 0; c < 8; ++c) x[c] = float(c);
    for (int64_t i = 0; i < iters * 16; ++i)
        for (int c = 0; c < 8; ++c) x[c] = std::fma(x[c], 0.999999f, 1e-7f);
    return ((x[0] + x[1]) + (x[2] + x[3])) + ((x[4] + x[5]) + (x[6] + x[7]));
}

// Reads slot `slot` of the sink (FP64 slots for FE_F64, FP32 otherwise) into
// *v: through the pointer, or, when `sym` is set, through the symbol of the
// static sink (so that a wrong device address of the array would show).
static cudaError_t read_slot(int dtype, const void* out, bool sym, int slot, double* v, cudaStream_t s);

// Timed launches of the chains into the per-CTA sink `out` (blocks slots),
// then a check of the first and last slot against the host's chain sum.
static cudaError_t run_probe(int dtype, int64_t iters, int blocks, void* out, bool sym, double* flops_per_s,
                             cudaStream_t s, bool* sink_ok) {
    const int threads = 256;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e != cudaSuccess) {
        if (t0) cudaEventDestroy(t0);
        return e;
    }
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // first pass warms up the clocks
        e = cudaEventRecord(t0, s);
        if (e != cudaSuccess) break;
        if (dtype == FE_F64)
            fma_chains<double><<<blocks, threads, 0, s>>>((double*)out, iters, 0.999999, 1e-7);
        else if (dtype == 3)
            fma2_chains<<<blocks, threads, 0, s>>>((float*)out, iters, 0.999999f, 1e-7f);
        else
            fma_chains<float><<<blocks, threads, 0, s>>>((float*)out, iters, 0.999999f, 1e-7f);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(t1, s);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
    *flops_per_s = flops / (ms * 1e-3);
    // the sink: first and last CTA slot hold thread 0's chain sum
    double first = 0.0, last = 0.0;
    e = read_slot(dtype, out, sym, 0, &first, s);
    if (e == cudaSuccess) e = read_slot(dtype, out, sym, blocks - 1, &last, s);
    if (e != cudaSuccess) return e;
    const double want = chain_sum_thread0(dtype, iters);
    *sink_ok = first == want && last == want;
    return cudaSuccess;
}

static cudaError_t probe_blocks(int& blocks) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    blocks = sms * 8;
    return cudaSuccess;
}

cudaError_t probe_fma(int dtype, int64_t iters, double* flops_per_s, cudaStream_t s, bool* sink_ok) {
    int blocks = 0;
    cudaError_t e = probe_blocks(blocks);
    if (e != cudaSuccess) return e;
    void* out = nullptr;
    e = cudaMallocAsync(&out, sizeof(double) * blocks, s);
    if (e != cudaSuccess) return e;
    *sink_ok = false;
    e = run_probe(dtype, iters, blocks, out, false, flops_per_s, s, sink_ok);
    const cudaError_t ef = cudaFreeAsync(out, s);
    return e != cudaSuccess ? e : ef;
}

// ---------------------------------------------------------------------------
// Allocation-free variant: the per-CTA sink lives in a file-scope device
// array instead of a stream-ordered allocation.  It serves callers that must
// not allocate device memory at all, e.g. a serving process that has already
// admitted work up to its HBM budget: an allocation there can fail or take
// memory the admitted requests were promised, and a peak measurement must not
// disturb them.  The sink holds one slot per CTA (8 CTAs per SM); nothing in
// it has to start at zero, because a CTA only ever writes its own slot.  All
// calls share the array and it keeps the last contents; calls that overlap
// in time (other streams, other host threads) write the same slots, which is
// harmless for the probe's result but is a race on the array's contents.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_probe_sink[kProbeSinkSlots];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_sink_mu;
void* g_sink_ptr[kMaxDevices] = {};
}  // namespace

cudaError_t probe_fma_static(int dtype, int64_t iters, double* flops_per_s, cudaStream_t s, int* too_many) {
    *too_many = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) {
        *too_many = -1;
        return cudaSuccess;
    }
    int blocks = 0;
    e = probe_blocks(blocks);
    if (e != cudaSuccess) return e;
    if (blocks > kProbeSinkSlots) {
        *too_many = blocks;
        return cudaSuccess;
    }
    void* out = nullptr;
    {
        // set-up once per device, with that device current: resolve the
        // device address of the array (this is the call to make before any
        // stream capture)
        std::lock_guard<std::mutex> lock(g_sink_mu);
        if (!g_sink_ptr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_probe_sink);
            if (e != cudaSuccess) return e;
            g_sink_ptr[dev] = ptr;
        }
        out = g_sink_ptr[dev];
    }
    bool ok = false;
    e = run_probe(dtype, iters, blocks, out, true, flops_per_s, s, &ok);
    if (e == cudaSuccess && !ok) *too_many = -2;
    return e;
}

static cudaError_t read_slot(int dtype, const void* out, bool sym, int slot, double* v, cudaStream_t s) {
    const size_t elem = dtype == FE_F64 ? sizeof(double) : sizeof(float);
    unsigned char buf[8] = {0};
    cudaError_t e = sym ? cudaMemcpyFromSymbolAsync(buf, g_probe_sink, elem, elem * (size_t)slot,
                                                     cudaMemcpyDeviceToHost, s)
                        : cudaMemcpyAsync(buf, static_cast<const unsigned char*>(out) + elem * (size_t)slot, elem,
                                          cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (elem == sizeof(double)) {
        std::memcpy(v, buf, sizeof(double));
    } else {
        float f;
        std::memcpy(&f, buf, sizeof(float));
        *v = f;
    }
    return cudaSuccess;
}

}  // namespace femf
