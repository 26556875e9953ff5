// Measured rates of the device resources the photon walk draws on (diagnostics).
//
// The walk is an issue-bound kernel (a few hundred thread-instructions per segment) that
// also leans on the special-function unit (one lg2 per hop, one ex2 per segment, a
// reciprocal, square roots and the azimuth's sine and cosine per scattering event) and on
// L2 atomics (one fluence atomic per (gate, voxel) run).  Its roofline is the slower of
// these resources' rates, each divided by the walk's per-photon demand on it.  The kernels
// below measure the rates on the device at hand instead of taking them from data sheets:
//   * issue: eight independent dependency chains per thread of one FP32 FMA each (the FMA
//     pipe), or of one three-input logic op each (the ALU pipe);
//   * special-function unit: eight independent chains of lg2 / ex2 / rsqrt / sin;
//   * atomics: fire-and-forget adds (RED) of FP32 or FP64 to addresses spread over a map of
//     a given size (L2-resident or HBM-resident), or to 32 hot words per warp.
// Every kernel runs a fixed number of iterations and ends; the call times the second of two
// launches with CUDA events.
#include <cstdint>
#include <string>

#include "mcx_internal.h"

namespace mcxg {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) probe_ffma(int iters, float x, float y, float *sink)
{
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[c]) : "f"(x), "f"(y));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.f) sink[0] = s;                  // keeps the chains alive
}

__global__ void __launch_bounds__(kProbeThreads) probe_lop3(int iters, unsigned b, unsigned c, unsigned *sink)
{
    unsigned a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 2654435761u + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k)           // a = (a ^ b) & c | ~a & b  (one LOP3)
            asm volatile("lop3.b32 %0, %0, %1, %2, 0x6C;" : "+r"(a[k]) : "r"(b), "r"(c));
    }
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s ^= a[k];
    if (s == 0x12345u) sink[0] = s;
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) probe_xu(int iters, float *sink)
{
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 1.25f + 0.01f * (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (OP == 0) asm volatile("lg2.approx.ftz.f32 %0, %0;" : "+f"(a[c]));
            if (OP == 1) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(a[c]));
            if (OP == 2) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(a[c]));
            if (OP == 3) asm volatile("sin.approx.ftz.f32 %0, %0;" : "+f"(a[c]));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.f) sink[0] = s;
}

// Adds to word h(thread, i) of a map of n_words (n_words a power of two): a multiplicative
// hash spreads a warp's 32 adds over 32 different lines; `hot` sends every warp's lanes to
// the same 32 words.
template <typename T>
__global__ void __launch_bounds__(kProbeThreads) probe_red(int iters, T *map, unsigned long long mask, int hot)
{
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    unsigned long long h = tid * 0x9E3779B97F4A7C15ull;
    for (int i = 0; i < iters; ++i) {
        h = h * 6364136223846793005ull + 1442695040888963407ull;
        const unsigned long long w = hot ? (threadIdx.x & 31u) : ((h >> 20) & mask);
        atomicAdd(map + w, T(1));
    }
}

}  // namespace
}  // namespace mcxg

using namespace mcxg;

extern "C" mcx_status mcx_probe_rate(int32_t kind, uint64_t map_bytes, double *rate)
{
    if (!rate || kind < 0 || kind > 9) {
        set_global_error("mcx_probe_rate: kind is 0..9 and rate must not be NULL");
        return MCX_E_ARG;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_global_error("mcx_probe_rate: no usable CUDA device");
        return MCX_E_CUDA;
    }
    const bool red = kind >= 6;
    const size_t elem = (kind == 7 || kind == 9) ? 8 : 4;
    const bool hot = kind >= 8;
    unsigned long long n_words = 32;
    if (red && !hot) {
        if (map_bytes < 4096 || map_bytes > (64ull << 30)) {
            set_global_error("mcx_probe_rate: map_bytes must be 4 KiB .. 64 GiB for kinds 6 and 7");
            return MCX_E_ARG;
        }
        n_words = 1;
        while (n_words * 2 * elem <= map_bytes) n_words *= 2;     // a power of two words
    }
    void *buf = nullptr;
    const size_t bytes = red ? (size_t)(n_words * elem) : 64;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        set_global_error("mcx_probe_rate: cannot allocate the probe buffer");
        return MCX_E_OOM;
    }
    cudaMemset(buf, 0, bytes);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // 8 resident blocks of 256 threads per SM; iteration counts give launches of 5-50 ms
    const int grid = sms * 8;
    const int iters = red ? (hot ? 256 : 1024) : (kind <= 1 ? 1 << 16 : 1 << 13);
    const double threads = (double)grid * kProbeThreads;
    const double ops = red ? threads * iters : threads * iters * kChains;
    float ms = 0.f;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {
        cudaEventRecord(e0);
        switch (kind) {
        case 0: probe_ffma<<<grid, kProbeThreads>>>(iters, 0.999f, 0.001f, (float *)buf); break;
        case 1: probe_lop3<<<grid, kProbeThreads>>>(iters, 0x5bd1e995u, 0x1b873593u, (unsigned *)buf); break;
        case 2: probe_xu<0><<<grid, kProbeThreads>>>(iters, (float *)buf); break;
        case 3: probe_xu<1><<<grid, kProbeThreads>>>(iters, (float *)buf); break;
        case 4: probe_xu<2><<<grid, kProbeThreads>>>(iters, (float *)buf); break;
        case 5: probe_xu<3><<<grid, kProbeThreads>>>(iters, (float *)buf); break;
        case 6: case 8:
            probe_red<float><<<grid, kProbeThreads>>>(iters, (float *)buf, n_words - 1, hot); break;
        default:
            probe_red<double><<<grid, kProbeThreads>>>(iters, (double *)buf, n_words - 1, hot); break;
        }
        cudaEventRecord(e1);
        err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (err != cudaSuccess) {
        set_global_error(std::string("mcx_probe_rate: ") + cudaGetErrorString(err));
        return MCX_E_CUDA;
    }
    *rate = ops / (ms * 1e-3);
    return MCX_OK;
}
