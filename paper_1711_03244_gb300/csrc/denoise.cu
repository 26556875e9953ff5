// Learned 3-D denoiser for low-photon fluence maps: a small U-Net (3 levels, 16/32/64
// channels, 3x3x3 convolutions) with BF16 weights and activations and FP32 accumulation,
// trained and run by hand-written tensor-core kernels (warp-level mma.sync m16n8k16).
// The network stands in for photons: it maps the log-fluence of a low-photon run to the
// log-fluence a high-photon run would give, and a plain high-photon run stays the
// fallback.  (This extends the method; the paper has no counterpart.)
//
// Layout: activations are BF16, [batch][z][y][x][channels] (channels innermost);
// convolution weights are BF16 [27 taps][Cout][Cin] for the forward pass and
// [27 taps][Cin][Cout] with flipped taps for the input gradient; FP32 master weights,
// gradients and Adam moments live beside them.
//
// Network (residual: output = input + head):
//   e1: conv(1->16), conv(16->16)      at D        skip s1
//   pool 2x2x2 (average)
//   e2: conv(16->32), conv(32->32)     at D/2      skip s2
//   pool
//   b:  conv(32->64), conv(64->64)     at D/4
//   upsample x2 (nearest), concat s2 -> 96 channels
//   d2: conv(96->32), conv(32->32)     at D/2
//   upsample, concat s1 -> 48 channels
//   d1: conv(48->16), conv(16->16)     at D
//   head: 1x1x1 conv 16->1 (FP32), added to the input
// Every 3x3x3 convolution has a bias and ReLU; the input layer sees the single input
// channel padded to 16 with zeros.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "mcx_internal.h"

using namespace mcxg;

namespace {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned *>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

struct Vol {
    int n, d, h, w;               // batch, depth (z), height (y), width (x)
    __host__ __device__ long long pos() const { return (long long)n * d * h * w; }
};

// ------------------------------------------------------------------------ convolution
// Y[p][co] = act(bias[co] + sum_tap sum_ci X[p + off(tap)][ci] * W[tap][co][ci]) (zero
// outside the volume) as an implicit GEMM on the 5th-generation tensor cores: one CTA
// (4 warps) computes 128 consecutive output positions x COUT channels as
// D[128][COUT] += A_tap[128][cin] * W_tap[cin][COUT] over the 27 taps, with D in tensor
// memory (FP32, one TMEM lane per position).  Each tap's operands are staged into shared memory by cp.async (zero-filled
// where the tap reads outside the volume) through a 3-buffer ring; one thread issues the
// tcgen05.mma instructions (K = 16 each) and tcgen05.commit signals an mbarrier when a
// buffer may be refilled.  Operand layout (K-major, no swizzle, 16-byte core-matrix rows):
// for each 16-channel slice kk, 8-row groups of two 8-channel core matrices:
//   byte(row r, 8-channel chunk c) = (c / 2) * (rows * 32) + (r / 8) * 256 + (c % 2) * 128 + (r % 8) * 16
// so an instruction's operand starts at slice kk with leading-dimension (K) offset 128 B and
// stride-dimension (M/N) offset 256 B.  Every wait is bounded: on a timeout the CTA records
// an error, still waits (bounded) for its own MMAs, frees its tensor memory and returns.
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

// shared-memory matrix descriptor: start, leading- and stride-dimension byte offsets,
// descriptor version 1 (bits 46-47), no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12
// = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                   "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int kTcRows = 128, kTcStages = 3, kTcHeader = 128, kTcSlack = 8192;

__host__ __device__ constexpr int tc_stage_bytes(int cin, int cout) { return (kTcRows + cout) * cin * 2; }

__host__ __device__ constexpr int tc_smem_bytes(int cin, int cout)
{
    return kTcHeader + kTcStages * tc_stage_bytes(cin, cout) + kTcSlack;
}

template <int COUT>
__global__ void __launch_bounds__(128)
conv3d_fwd_tc(const bf16 *__restrict__ X, int cin, const bf16 *__restrict__ Wt,
              const float *__restrict__ bias, Vol v, int relu, bf16 *__restrict__ Y, unsigned *err)
{
    constexpr int NCOL = COUT <= 32 ? 32 : (COUT <= 64 ? 64 : 128);   // TMEM columns
    constexpr uint32_t IDESC = idesc_bf16_f32(kTcRows, COUT);
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t bar0 = smem_u32(smem);                     // 3 mbarriers, 8 B each
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + 64);
    unsigned char *ring = smem + kTcHeader;
    const int a_bytes = kTcRows * cin * 2, st_bytes = tc_stage_bytes(cin, COUT);
    const int tid = threadIdx.x, warp = tid >> 5;

    const long long P = v.pos();
    const long long p = (long long)blockIdx.x * kTcRows + tid;  // this thread's row
    const bool valid = p < P;
    int x = 0, y = 0, z = 0, b = 0;
    if (valid) {
        long long r = p;
        x = (int)(r % v.w); r /= v.w;
        y = (int)(r % v.h); r /= v.h;
        z = (int)(r % v.d);
        b = (int)(r / v.d);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(smem_u32(tslot)), "r"(NCOL) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0 + 8 * s) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    // stage tap `tap` into ring buffer s
    auto stage = [&](int tap, int s) {
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        const uint32_t A = smem_u32(ring + s * st_bytes), B = A + a_bytes;
        const int xs = x + dx, ys = y + dy, zs = z + dz;
        const bool in = valid && xs >= 0 && xs < v.w && ys >= 0 && ys < v.h && zs >= 0 && zs < v.d;
        const bf16 *src = in ? X + ((((long long)b * v.d + zs) * v.h + ys) * v.w + xs) * cin : X;
        const uint32_t arow = A + (tid >> 3) * 256 + (tid & 7) * 16;
        for (int c = 0; c < cin / 8; ++c)
            cp_async16(arow + (c >> 1) * (kTcRows * 32) + (c & 1) * 128, src + (in ? 8 * c : 0), in ? 16u : 0u);
        const bf16 *wt = Wt + (size_t)tap * COUT * cin;
        for (int i = tid; i < COUT * (cin / 8); i += 128) {
            const int co = i % COUT, c = i / COUT;
            cp_async16(B + (c >> 1) * (COUT * 32) + (co >> 3) * 256 + (c & 1) * 128 + (co & 7) * 16,
                       wt + (size_t)co * cin + 8 * c, 16u);
        }
    };

    bool ok = true;
    stage(0, 0);
    cp_async_commit();
    stage(1, 1);
    cp_async_commit();
    for (int t = 0; t < 27; ++t) {
        cp_async_wait<1>();                    // this thread's copies of tap t have landed
        fence_proxy_async_smem();              // make them visible to the tensor cores
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const int s = t % kTcStages;
            const uint32_t A = smem_u32(ring + s * st_bytes), B = A + a_bytes;
            for (int kk = 0; kk < cin / 16; ++kk) {
                const uint64_t ad = umma_desc(A + kk * (kTcRows * 32), 128, 256);
                const uint64_t bd = umma_desc(B + kk * (COUT * 32), 128, 256);
                const uint32_t acc = (t | kk) ? 1u : 0u;
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             ::"r"(tmem), "l"(ad), "l"(bd), "r"(IDESC), "r"(acc) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                         ::"r"(bar0 + 8 * s) : "memory");
        }
        // refill the buffer of tap t - 1 with tap t + 2 once its MMAs have completed
        const int nt = t + kTcStages - 1;
        if (nt < 27) {
            const int s = nt % kTcStages;
            if (nt >= kTcStages) ok &= mbar_wait(bar0 + 8 * s, (uint32_t)((nt / kTcStages - 1) & 1));
            stage(nt, s);
        }
        cp_async_commit();
    }
    // the last commit (tap 26) covers every MMA of this CTA
    ok &= mbar_wait(bar0 + 8 * (26 % kTcStages), (uint32_t)((26 / kTcStages) & 1));
    ok = __syncthreads_and(ok);                // the warp-collective reads below need one answer
    tc_fence_after();
    if (ok) {
        float acc[COUT];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < COUT; c0 += 16) tmem_ld16(taddr + c0, acc + c0);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (valid) {
            bf16 *yr = Y + p * COUT;
#pragma unroll
            for (int c = 0; c < COUT; c += 8) {
                float o[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    o[i] = acc[c + i] + (bias ? bias[c + i] : 0.f);
                    if (relu) o[i] = fmaxf(o[i], 0.f);
                }
                uint4 pk;
                pk.x = pack_bf16(o[0], o[1]);
                pk.y = pack_bf16(o[2], o[3]);
                pk.z = pack_bf16(o[4], o[5]);
                pk.w = pack_bf16(o[6], o[7]);
                *reinterpret_cast<uint4 *>(yr + c) = pk;
            }
        }
    } else if (tid == 0) {
        atomicOr(err, 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NCOL) : "memory");
    }
}

// Weight gradient of one tap: dW[tap][co][ci] += sum_p dY[p][co] * X[p + off(tap)][ci],
// a GEMM with M = Cout (16 per warp), N = Cin (8 per mma), K = positions (16 per mma),
// over one chunk of positions; chunks are summed with FP32 atomics.
template <int CIN>
__global__ void __launch_bounds__(128)
conv3d_bwd_w(const bf16 *__restrict__ X, const bf16 *__restrict__ dY, int cout, Vol v,
             long long chunk, float *__restrict__ dW)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int tap = blockIdx.y;
    const int mt = warp;                                   // rows co = 16 mt .. 16 mt + 15
    if (mt * 16 >= cout) return;
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const long long P = v.pos();
    const long long pbeg = blockIdx.x * chunk, pend = min(P, pbeg + chunk);
    float acc[CIN / 8][4];
#pragma unroll
    for (int j = 0; j < CIN / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const int co_a = mt * 16 + g, co_b = co_a + 8;
    for (long long k0 = pbeg; k0 < pend; k0 += 16) {
        // four positions per thread: k0 + 2t, +1, +8, +9
        long long pk[4] = {k0 + 2 * t, k0 + 2 * t + 1, k0 + 2 * t + 8, k0 + 2 * t + 9};
        float ya[4], yb[4];
        long long src[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const long long p = pk[i];
            bool ok = p < pend;
            long long s = -1;
            if (ok) {
                const int x = (int)(p % v.w);
                long long r = p / v.w;
                const int yy = (int)(r % v.h);
                r /= v.h;
                const int zz = (int)(r % v.d);
                const int bb = (int)(r / v.d);
                const int xs = x + dx, ys = yy + dy, zs = zz + dz;
                if (xs >= 0 && xs < v.w && ys >= 0 && ys < v.h && zs >= 0 && zs < v.d)
                    s = (((long long)bb * v.d + zs) * v.h + ys) * v.w + xs;
            }
            src[i] = s;
            ya[i] = ok ? __bfloat162float(dY[p * cout + co_a]) : 0.f;
            yb[i] = ok ? __bfloat162float(dY[p * cout + co_b]) : 0.f;
        }
        const unsigned a0 = pack_bf16(ya[0], ya[1]), a1 = pack_bf16(yb[0], yb[1]);
        const unsigned a2 = pack_bf16(ya[2], ya[3]), a3 = pack_bf16(yb[2], yb[3]);
#pragma unroll
        for (int j = 0; j < CIN / 8; ++j) {
            const int ci = j * 8 + g;
            float xv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) xv[i] = src[i] >= 0 ? __bfloat162float(X[src[i] * CIN + ci]) : 0.f;
            mma_bf16(acc[j], a0, a1, a2, a3, pack_bf16(xv[0], xv[1]), pack_bf16(xv[2], xv[3]));
        }
    }
    float *dWt = dW + (size_t)tap * cout * CIN;
#pragma unroll
    for (int j = 0; j < CIN / 8; ++j) {
        const int ci = j * 8 + 2 * t;
        atomicAdd(dWt + (size_t)co_a * CIN + ci, acc[j][0]);
        atomicAdd(dWt + (size_t)co_a * CIN + ci + 1, acc[j][1]);
        atomicAdd(dWt + (size_t)co_b * CIN + ci, acc[j][2]);
        atomicAdd(dWt + (size_t)co_b * CIN + ci + 1, acc[j][3]);
    }
}

// ------------------------------------------------------------------------ elementwise
__global__ void relu_mask(bf16 *dY, const bf16 *Y, long long n)
{
    const long long s = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += s)
        if (__bfloat162float(Y[i]) <= 0.f) dY[i] = __float2bfloat16(0.f);
}

__global__ void bias_grad(const bf16 *dY, long long npos, int c, float *db)
{
    // one thread per (channel, slice of positions)
    const int ch = blockIdx.y;
    float s = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npos; p += stride)
        s += __bfloat162float(dY[p * c + ch]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(db + ch, s);
}

// input layer: the FP32 input as channel 0 of a 16-channel BF16 volume
__global__ void pad_input(const float *x, long long npos, bf16 *X16)
{
    const long long s = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npos * 16; i += s)
        X16[i] = __float2bfloat16((i & 15) == 0 ? x[i >> 4] : 0.f);
}

__global__ void avgpool_fwd(const bf16 *X, Vol vo, int c, bf16 *Y)   // vo: output volume
{
    const long long n = vo.pos() * c, s = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += s) {
        const int ch = (int)(i % c);
        long long p = i / c;
        const int x = (int)(p % vo.w); p /= vo.w;
        const int y = (int)(p % vo.h); p /= vo.h;
        const int z = (int)(p % vo.d);
        const int b = (int)(p / vo.d);
        const int W = 2 * vo.w, H = 2 * vo.h, D = 2 * vo.d;
        float acc = 0.f;
        for (int k = 0; k < 8; ++k) {
            const long long q = (((long long)b * D + 2 * z + (k >> 2)) * H + 2 * y + ((k >> 1) & 1)) * W + 2 * x + (k & 1);
            acc += __bfloat162float(X[q * c + ch]);
        }
        Y[i] = __float2bfloat16(acc * 0.125f);
    }
}

__global__ void avgpool_bwd(const bf16 *dY, Vol vi, int c, bf16 *dX)  // vi: input (fine) volume
{
    const long long n = vi.pos() * c, s = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += s) {
        const int ch = (int)(i % c);
        long long p = i / c;
        const int x = (int)(p % vi.w); p /= vi.w;
        const int y = (int)(p % vi.h); p /= vi.h;
        const int z = (int)(p % vi.d);
        const int b = (int)(p / vi.d);
        const long long q = (((long long)b * (vi.d / 2) + z / 2) * (vi.h / 2) + y / 2) * (vi.w / 2) + x / 2;
        dX[i] = __float2bfloat16(__bfloat162float(dY[q * c + ch]) * 0.125f);
    }
}

// nearest x2 upsampling of X (coarse, cx channels) into channels [0, cx) of a cdst-channel
// fine volume, and the skip S (cs channels) into channels [cx, cx + cs)
__global__ void upcat_fwd(const bf16 *X, int cx, const bf16 *S, int cs, Vol vf, bf16 *Y)
{
    const int c = cx + cs;
    const long long n = vf.pos() * c, st = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += st) {
        const int ch = (int)(i % c);
        const long long p = i / c;
        if (ch >= cx) {
            Y[i] = S[p * cs + (ch - cx)];
        } else {
            long long q = p;
            const int x = (int)(q % vf.w); q /= vf.w;
            const int y = (int)(q % vf.h); q /= vf.h;
            const int z = (int)(q % vf.d);
            const int b = (int)(q / vf.d);
            const long long pc = (((long long)b * (vf.d / 2) + z / 2) * (vf.h / 2) + y / 2) * (vf.w / 2) + x / 2;
            Y[i] = X[pc * cx + ch];
        }
    }
}

// gradient of upcat: the coarse part sums its 8 children; the skip part is copied
__global__ void upcat_bwd_coarse(const bf16 *dY, int cx, int cs, Vol vc, bf16 *dX)
{
    const int c = cx + cs;
    const long long n = vc.pos() * cx, st = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += st) {
        const int ch = (int)(i % cx);
        long long p = i / cx;
        const int x = (int)(p % vc.w); p /= vc.w;
        const int y = (int)(p % vc.h); p /= vc.h;
        const int z = (int)(p % vc.d);
        const int b = (int)(p / vc.d);
        const int W = 2 * vc.w, H = 2 * vc.h, D = 2 * vc.d;
        float acc = 0.f;
        for (int k = 0; k < 8; ++k) {
            const long long q = (((long long)b * D + 2 * z + (k >> 2)) * H + 2 * y + ((k >> 1) & 1)) * W + 2 * x + (k & 1);
            acc += __bfloat162float(dY[q * c + ch]);
        }
        dX[i] = __float2bfloat16(acc);
    }
}

__global__ void upcat_bwd_skip_add(const bf16 *dY, int cx, int cs, long long npos, bf16 *dS)
{
    const int c = cx + cs;
    const long long n = npos * cs, st = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += st) {
        const long long p = i / cs;
        const int ch = (int)(i % cs);
        dS[i] = __float2bfloat16(__bfloat162float(dS[i]) + __bfloat162float(dY[p * c + cx + ch]));
    }
}

// head: out[p] = x[p] + hb + sum_c hw[c] Y[p][c]
__global__ void head_fwd(const bf16 *Y, const float *x, const float *hw, const float *hb,
                         long long npos, float *out)
{
    const long long st = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npos; p += st) {
        float s = hb[0];
        for (int c = 0; c < 16; ++c) s += hw[c] * __bfloat162float(Y[p * 16 + c]);
        out[p] = x[p] + s;
    }
}

// loss L = mean (out - target)^2, dout = 2 (out - target) / n; dY = dout hw; head grads
__global__ void head_bwd(const bf16 *Y, const float *out, const float *target, const float *hw,
                         long long npos, bf16 *dY, float *dhw, float *dhb, float *loss)
{
    float gw[16] = {0}, gb = 0.f, l = 0.f;
    const float inv_n = 1.f / (float)npos;
    const long long st = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npos; p += st) {
        const float e = out[p] - target[p];
        l += e * e * inv_n;
        const float d = 2.f * e * inv_n;
        gb += d;
        for (int c = 0; c < 16; ++c) {
            gw[c] += d * __bfloat162float(Y[p * 16 + c]);
            dY[p * 16 + c] = __float2bfloat16(d * hw[c]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        l += __shfl_down_sync(0xffffffffu, l, o);
        gb += __shfl_down_sync(0xffffffffu, gb, o);
        for (int c = 0; c < 16; ++c) gw[c] += __shfl_down_sync(0xffffffffu, gw[c], o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(loss, l);
        atomicAdd(dhb, gb);
        for (int c = 0; c < 16; ++c) atomicAdd(dhw + c, gw[c]);
    }
}

// Adam on the FP32 master weights; refreshes the BF16 forward copy [tap][co][ci] and the
// input-gradient copy [26 - tap][ci][co] of convolution weights
__global__ void adam_step(float *w, const float *gr, float *m, float *v, long long n, float lr,
                          float b1, float b2, float c1, float c2, float eps)
{
    const long long st = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += st) {
        const float g = gr[i];
        const float mm = b1 * m[i] + (1.f - b1) * g;
        const float vv = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mm;
        v[i] = vv;
        w[i] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
    }
}

__global__ void refresh_conv_bf16(const float *w, int cin, int cout, bf16 *wf, bf16 *wb)
{
    const long long n = 27LL * cin * cout, st = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += st) {
        const int ci = (int)(i % cin);
        const int co = (int)((i / cin) % cout);
        const int tap = (int)(i / ((long long)cin * cout));
        const bf16 b = __float2bfloat16(w[i]);
        wf[i] = b;
        wb[((size_t)(26 - tap) * cin + ci) * cout + co] = b;
    }
}

// fluence <-> network domain: x = (log10(phi + floor) - mu) / sigma and its inverse
__global__ void encode_kernel(const float *phi, long long n, float floor_, float mu, float inv_sigma, float *x)
{
    const long long st = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += st)
        x[i] = (log10f(fmaxf(phi[i], 0.f) + floor_) - mu) * inv_sigma;
}

__global__ void decode_kernel(const float *x, long long n, float floor_, float mu, float sigma, float *phi)
{
    const long long st = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += st)
        phi[i] = fmaxf(exp10f(fmaf(x[i], sigma, mu)) - floor_, 0.f);
}

// training batches: sample s of dst is volume idx[s] of a stored set, mirrored in x
// (flags bit 0) and y (bit 1) and then transposed in x/y (bit 2) -- symmetries of a
// pencil beam entering through the z = 0 face
constexpr int kMaxGather = 64;
struct GatherList {
    unsigned long long idx[kMaxGather];
    unsigned flags[kMaxGather];
};

__global__ void gather_kernel(const float *set, GatherList L, int n, int D, int H, int W, float *dst)
{
    const long long vol = (long long)D * H * W, total = vol * n;
    const long long st = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += st) {
        const int s = (int)(i / vol);
        long long r = i % vol;
        const int x = (int)(r % W);
        r /= W;
        const int y = (int)(r % H);
        const int z = (int)(r / H);
        const unsigned f = L.flags[s];
        int xs = x, ys = y;
        if (f & 4u) { xs = y; ys = x; }
        if (f & 1u) xs = W - 1 - xs;
        if (f & 2u) ys = H - 1 - ys;
        dst[i] = set[(long long)L.idx[s] * vol + ((long long)z * H + ys) * W + xs];
    }
}

unsigned grid1(long long n)
{
    return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 32));
}

template <int COUT>
cudaError_t launch_tc_t(const bf16 *X, int cin, const bf16 *W, const float *bias, Vol v, int relu,
                        bf16 *Y, unsigned *err, cudaStream_t st)
{
    const int smem = tc_smem_bytes(cin, COUT);
    cudaError_t e = cudaFuncSetAttribute(conv3d_fwd_tc<COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((v.pos() + kTcRows - 1) / kTcRows);
    conv3d_fwd_tc<COUT><<<blocks, 128, smem, st>>>(X, cin, W, bias, v, relu, Y, err);
    return cudaGetLastError();
}

cudaError_t launch_fwd_tc(const bf16 *X, int cin, const bf16 *W, const float *bias, Vol v, int cout,
                          int relu, bf16 *Y, unsigned *err, cudaStream_t st)
{
    if (cin % 16 || cin < 16 || cin > 96) return cudaErrorInvalidValue;
    switch (cout) {
    case 16: return launch_tc_t<16>(X, cin, W, bias, v, relu, Y, err, st);
    case 32: return launch_tc_t<32>(X, cin, W, bias, v, relu, Y, err, st);
    case 48: return launch_tc_t<48>(X, cin, W, bias, v, relu, Y, err, st);
    case 64: return launch_tc_t<64>(X, cin, W, bias, v, relu, Y, err, st);
    case 96: return launch_tc_t<96>(X, cin, W, bias, v, relu, Y, err, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_bwd_w(const bf16 *X, int cin, const bf16 *dY, int cout, Vol v, float *dW,
                         cudaStream_t st)
{
    // about 48 position chunks per tap: enough blocks to fill the GPU, few FP32 atomics
    const long long chunk = std::max<long long>(2048, ((v.pos() / 48 + 15) / 16) * 16);
    const dim3 grid((unsigned)((v.pos() + chunk - 1) / chunk), 27);
    const int warps = (cout + 15) / 16;
    switch (cin) {
    case 16: conv3d_bwd_w<16><<<grid, 32 * warps, 0, st>>>(X, dY, cout, v, chunk, dW); break;
    case 32: conv3d_bwd_w<32><<<grid, 32 * warps, 0, st>>>(X, dY, cout, v, chunk, dW); break;
    case 48: conv3d_bwd_w<48><<<grid, 32 * warps, 0, st>>>(X, dY, cout, v, chunk, dW); break;
    case 64: conv3d_bwd_w<64><<<grid, 32 * warps, 0, st>>>(X, dY, cout, v, chunk, dW); break;
    case 96: conv3d_bwd_w<96><<<grid, 32 * warps, 0, st>>>(X, dY, cout, v, chunk, dW); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t alloc(size_t b)
    {
        bytes = b;
        return b ? cudaMalloc(&p, b) : cudaSuccess;
    }
    ~DBuf() { if (p) cudaFree(p); }
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

// the ten 3x3x3 convolutions: (cin, cout, level)
struct LayerSpec { int cin, cout, level; };
const LayerSpec kLayers[10] = {{16, 16, 0}, {16, 16, 0}, {16, 32, 1}, {32, 32, 1}, {32, 64, 2},
                               {64, 64, 2}, {96, 32, 1}, {32, 32, 1}, {48, 16, 0}, {16, 16, 0}};

thread_local std::string g_dn_err;

}  // namespace

struct mcx_denoiser {
    int D, H, W, maxb;
    size_t nparam = 0;
    std::vector<size_t> w_off, b_off;   // offsets of each layer's weights / bias in params
    size_t hw_off = 0, hb_off = 0;
    DBuf params, grads, m1, m2;         // FP32 master weights, gradients, Adam moments
    DBuf wf[10], wb[10];                // BF16 forward / input-gradient weights
    // activations (BF16, max batch) and their gradients
    DBuf x16, a[10], p1, p2, u2, u1, out, loss;
    DBuf g_x16, ga[10], gp1, gp2, gu2, gu1, gtmp;
    DBuf xin;                           // encoded input of apply()
    DBuf status;                        // set when a tensor-core wait timed out
    float floor_ = 1e-8f, mu = -4.f, sigma = 2.f;
    long long step = 0;
    std::string err;
};

static mcx_status dn_fail(mcx_denoiser *d, mcx_status st, const std::string &m)
{
    if (d) d->err = m;
    set_global_error(m);
    return st;
}

#define DNC(d, call, what)                                                                     \
    do {                                                                                       \
        const cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                                 \
            return dn_fail((d), e_ == cudaErrorMemoryAllocation ? MCX_E_OOM : MCX_E_CUDA,      \
                           std::string(what) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

// after the device has been synchronised: reports (and clears) a tensor-core wait timeout
static mcx_status check_status(mcx_denoiser *d)
{
    unsigned h = 0;
    DNC(d, cudaMemcpy(&h, d->status.p, 4, cudaMemcpyDeviceToHost), "reading the status");
    if (h) {
        DNC(d, cudaMemset(d->status.p, 0, 4), "clearing the status");
        return dn_fail(d, MCX_E_TIMEOUT, "a tensor-core pipeline wait timed out; results are invalid");
    }
    return MCX_OK;
}

static Vol level_vol(const mcx_denoiser *d, int level, int n)
{
    return Vol{n, d->D >> level, d->H >> level, d->W >> level};
}

static mcx_status refresh_weights(mcx_denoiser *d, cudaStream_t st)
{
    for (int l = 0; l < 10; ++l) {
        const LayerSpec &L = kLayers[l];
        refresh_conv_bf16<<<grid1(27LL * L.cin * L.cout), 256, 0, st>>>(
            d->params.as<float>() + d->w_off[l], L.cin, L.cout, d->wf[l].as<bf16>(), d->wb[l].as<bf16>());
    }
    DNC(d, cudaGetLastError(), "refreshing BF16 weights");
    return MCX_OK;
}

// forward pass for n volumes; activations stay for the backward pass
static mcx_status forward(mcx_denoiser *d, const float *x, int n, float *out, cudaStream_t st)
{
    const Vol v0 = level_vol(d, 0, n), v1 = level_vol(d, 1, n), v2 = level_vol(d, 2, n);
    const float *P = d->params.as<float>();
    pad_input<<<grid1(v0.pos() * 16), 256, 0, st>>>(x, v0.pos(), d->x16.as<bf16>());
    auto conv = [&](int l, const bf16 *in, Vol v) {
        return launch_fwd_tc(in, kLayers[l].cin, d->wf[l].as<bf16>(), P + d->b_off[l], v,
                             kLayers[l].cout, 1, d->a[l].as<bf16>(), d->status.as<unsigned>(), st);
    };
    DNC(d, conv(0, d->x16.as<bf16>(), v0), "conv e1a");
    DNC(d, conv(1, d->a[0].as<bf16>(), v0), "conv e1b");
    avgpool_fwd<<<grid1(v1.pos() * 16), 256, 0, st>>>(d->a[1].as<bf16>(), v1, 16, d->p1.as<bf16>());
    DNC(d, conv(2, d->p1.as<bf16>(), v1), "conv e2a");
    DNC(d, conv(3, d->a[2].as<bf16>(), v1), "conv e2b");
    avgpool_fwd<<<grid1(v2.pos() * 32), 256, 0, st>>>(d->a[3].as<bf16>(), v2, 32, d->p2.as<bf16>());
    DNC(d, conv(4, d->p2.as<bf16>(), v2), "conv ba");
    DNC(d, conv(5, d->a[4].as<bf16>(), v2), "conv bb");
    upcat_fwd<<<grid1(v1.pos() * 96), 256, 0, st>>>(d->a[5].as<bf16>(), 64, d->a[3].as<bf16>(), 32, v1, d->u2.as<bf16>());
    DNC(d, conv(6, d->u2.as<bf16>(), v1), "conv d2a");
    DNC(d, conv(7, d->a[6].as<bf16>(), v1), "conv d2b");
    upcat_fwd<<<grid1(v0.pos() * 48), 256, 0, st>>>(d->a[7].as<bf16>(), 32, d->a[1].as<bf16>(), 16, v0, d->u1.as<bf16>());
    DNC(d, conv(8, d->u1.as<bf16>(), v0), "conv d1a");
    DNC(d, conv(9, d->a[8].as<bf16>(), v0), "conv d1b");
    head_fwd<<<grid1(v0.pos()), 256, 0, st>>>(d->a[9].as<bf16>(), x, P + d->hw_off, P + d->hb_off,
                                             v0.pos(), out);
    DNC(d, cudaGetLastError(), "forward");
    return MCX_OK;
}

// backward of a conv layer l with input `in`: dA (gradient of its ReLU output, in place in
// ga[l]) -> weight and bias gradients, and (if dIn) the input gradient
static mcx_status conv_bwd(mcx_denoiser *d, int l, const bf16 *in, Vol v, bf16 *dIn, cudaStream_t st)
{
    const LayerSpec &L = kLayers[l];
    float *G = d->grads.as<float>();
    bf16 *dA = d->ga[l].as<bf16>();
    relu_mask<<<grid1(v.pos() * L.cout), 256, 0, st>>>(dA, d->a[l].as<bf16>(), v.pos() * L.cout);
    bias_grad<<<dim3(64, L.cout), 256, 0, st>>>(dA, v.pos(), L.cout, G + d->b_off[l]);
    DNC(d, launch_bwd_w(in, L.cin, dA, L.cout, v, G + d->w_off[l], st), "weight gradient");
    if (dIn)
        DNC(d, launch_fwd_tc(dA, L.cout, d->wb[l].as<bf16>(), nullptr, v, L.cin, 0, dIn, d->status.as<unsigned>(), st),
            "input gradient");
    return MCX_OK;
}

static mcx_status backward(mcx_denoiser *d, const float *x, const float *target, int n, cudaStream_t st)
{
    const Vol v0 = level_vol(d, 0, n), v1 = level_vol(d, 1, n), v2 = level_vol(d, 2, n);
    float *G = d->grads.as<float>();
    const float *P = d->params.as<float>();
    DNC(d, cudaMemsetAsync(d->grads.p, 0, d->nparam * sizeof(float), st), "clearing gradients");
    DNC(d, cudaMemsetAsync(d->loss.p, 0, sizeof(float), st), "clearing the loss");
    head_bwd<<<grid1(v0.pos()), 256, 0, st>>>(d->a[9].as<bf16>(), d->out.as<float>(), target,
                                             P + d->hw_off, v0.pos(), d->ga[9].as<bf16>(),
                                             G + d->hw_off, G + d->hb_off, d->loss.as<float>());
    mcx_status s;
    if ((s = conv_bwd(d, 9, d->a[8].as<bf16>(), v0, d->ga[8].as<bf16>(), st)) != MCX_OK) return s;
    if ((s = conv_bwd(d, 8, d->u1.as<bf16>(), v0, d->gu1.as<bf16>(), st)) != MCX_OK) return s;
    // upcat 1: coarse part -> d2b output gradient, skip part -> e1b output gradient (later)
    upcat_bwd_coarse<<<grid1(v1.pos() * 32), 256, 0, st>>>(d->gu1.as<bf16>(), 32, 16, v1, d->ga[7].as<bf16>());
    if ((s = conv_bwd(d, 7, d->a[6].as<bf16>(), v1, d->ga[6].as<bf16>(), st)) != MCX_OK) return s;
    if ((s = conv_bwd(d, 6, d->u2.as<bf16>(), v1, d->gu2.as<bf16>(), st)) != MCX_OK) return s;
    upcat_bwd_coarse<<<grid1(v2.pos() * 64), 256, 0, st>>>(d->gu2.as<bf16>(), 64, 32, v2, d->ga[5].as<bf16>());
    if ((s = conv_bwd(d, 5, d->a[4].as<bf16>(), v2, d->ga[4].as<bf16>(), st)) != MCX_OK) return s;
    if ((s = conv_bwd(d, 4, d->p2.as<bf16>(), v2, d->gp2.as<bf16>(), st)) != MCX_OK) return s;
    // e2b output gradient = pool backward + the skip part of upcat 2
    avgpool_bwd<<<grid1(v1.pos() * 32), 256, 0, st>>>(d->gp2.as<bf16>(), v1, 32, d->ga[3].as<bf16>());
    upcat_bwd_skip_add<<<grid1(v1.pos() * 32), 256, 0, st>>>(d->gu2.as<bf16>(), 64, 32, v1.pos(), d->ga[3].as<bf16>());
    if ((s = conv_bwd(d, 3, d->a[2].as<bf16>(), v1, d->ga[2].as<bf16>(), st)) != MCX_OK) return s;
    if ((s = conv_bwd(d, 2, d->p1.as<bf16>(), v1, d->gp1.as<bf16>(), st)) != MCX_OK) return s;
    avgpool_bwd<<<grid1(v0.pos() * 16), 256, 0, st>>>(d->gp1.as<bf16>(), v0, 16, d->ga[1].as<bf16>());
    upcat_bwd_skip_add<<<grid1(v0.pos() * 16), 256, 0, st>>>(d->gu1.as<bf16>(), 32, 16, v0.pos(), d->ga[1].as<bf16>());
    if ((s = conv_bwd(d, 1, d->a[0].as<bf16>(), v0, d->ga[0].as<bf16>(), st)) != MCX_OK) return s;
    if ((s = conv_bwd(d, 0, d->x16.as<bf16>(), v0, nullptr, st)) != MCX_OK) return s;
    DNC(d, cudaGetLastError(), "backward");
    return MCX_OK;
}

extern "C" {

mcx_status mcx_denoiser_create(mcx_denoiser **out, uint32_t nx, uint32_t ny, uint32_t nz,
                               uint32_t max_batch, uint64_t seed)
{
    if (!out) return dn_fail(nullptr, MCX_E_ARG, "out is NULL");
    *out = nullptr;
    if (nx % 64 || nx < 64 || ny % 4 || nz % 4 || ny < 4 || nz < 4 || max_batch < 1)
        return dn_fail(nullptr, MCX_E_ARG, "need nx a multiple of 64, ny and nz multiples of 4, max_batch >= 1");
    mcx_denoiser *d = new (std::nothrow) mcx_denoiser();
    if (!d) return dn_fail(nullptr, MCX_E_OOM, "host allocation failed");
    d->D = (int)nz; d->H = (int)ny; d->W = (int)nx; d->maxb = (int)max_batch;
    size_t off = 0;
    for (int l = 0; l < 10; ++l) {
        d->w_off.push_back(off);
        off += 27ull * kLayers[l].cin * kLayers[l].cout;
        d->b_off.push_back(off);
        off += kLayers[l].cout;
    }
    d->hw_off = off; off += 16;
    d->hb_off = off; off += 1;
    d->nparam = off;
    // He-normal initial weights (fan-in 27 cin; the padded input layer's fan-in is 27)
    std::vector<float> init(d->nparam, 0.f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < 10; ++l) {
        const int fan = 27 * (l == 0 ? 1 : kLayers[l].cin);
        std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / fan));
        for (size_t i = 0; i < 27ull * kLayers[l].cin * kLayers[l].cout; ++i) {
            const int ci = (int)(i % kLayers[l].cin);
            init[d->w_off[l] + i] = (l == 0 && ci > 0) ? 0.f : (float)nd(rng);
        }
    }
    // the head starts at zero: the untrained network returns its input
    const Vol v0 = {d->maxb, d->D, d->H, d->W};
    const long long p0 = v0.pos(), p1 = p0 / 8, p2 = p0 / 64;
    const size_t B2 = sizeof(bf16);
    cudaError_t e = cudaSuccess;
    auto A = [&](DBuf &b, size_t bytes) { if (e == cudaSuccess) e = b.alloc(bytes); };
    A(d->params, d->nparam * 4); A(d->grads, d->nparam * 4); A(d->m1, d->nparam * 4); A(d->m2, d->nparam * 4);
    for (int l = 0; l < 10; ++l) {
        const size_t nw = 27ull * kLayers[l].cin * kLayers[l].cout * B2;
        A(d->wf[l], nw); A(d->wb[l], nw);
        const long long np = kLayers[l].level == 0 ? p0 : (kLayers[l].level == 1 ? p1 : p2);
        A(d->a[l], np * kLayers[l].cout * B2);
        A(d->ga[l], np * kLayers[l].cout * B2);
    }
    A(d->x16, p0 * 16 * B2); A(d->p1, p1 * 16 * B2); A(d->p2, p2 * 32 * B2);
    A(d->u2, p1 * 96 * B2); A(d->u1, p0 * 48 * B2); A(d->out, p0 * 4); A(d->loss, 4);
    A(d->xin, p0 * 4);
    A(d->status, 4);
    A(d->gp1, p1 * 16 * B2); A(d->gp2, p2 * 32 * B2); A(d->gu2, p1 * 96 * B2); A(d->gu1, p0 * 48 * B2);
    if (e == cudaSuccess) e = cudaMemcpy(d->params.p, init.data(), d->nparam * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d->status.p, 0, 4);
    if (e == cudaSuccess) e = cudaMemset(d->m1.p, 0, d->nparam * 4);
    if (e == cudaSuccess) e = cudaMemset(d->m2.p, 0, d->nparam * 4);
    if (e != cudaSuccess) {
        delete d;
        return dn_fail(nullptr, e == cudaErrorMemoryAllocation ? MCX_E_OOM : MCX_E_CUDA,
                       std::string("creating the denoiser: ") + cudaGetErrorString(e));
    }
    mcx_status s = refresh_weights(d, nullptr);
    if (s == MCX_OK && cudaDeviceSynchronize() != cudaSuccess) s = MCX_E_CUDA;
    if (s != MCX_OK) { delete d; return s; }
    *out = d;
    return MCX_OK;
}

mcx_status mcx_denoiser_param_count(const mcx_denoiser *d, uint64_t *n)
{
    if (!d || !n) return dn_fail(nullptr, MCX_E_ARG, "NULL argument");
    *n = d->nparam;
    return MCX_OK;
}

mcx_status mcx_denoiser_get_params(mcx_denoiser *d, float *host, uint64_t n, int32_t which)
{
    if (!d || !host) return dn_fail(d, MCX_E_ARG, "NULL argument");
    if (n != d->nparam) return dn_fail(d, MCX_E_ARG, "n must equal the parameter count");
    DNC(d, cudaDeviceSynchronize(), "waiting");
    if (mcx_status s = check_status(d)) return s;
    const DBuf &src = which == 1 ? d->grads : d->params;
    DNC(d, cudaMemcpy(host, src.p, n * 4, cudaMemcpyDeviceToHost), "reading parameters");
    return MCX_OK;
}

mcx_status mcx_denoiser_set_params(mcx_denoiser *d, const float *host, uint64_t n)
{
    if (!d || !host) return dn_fail(d, MCX_E_ARG, "NULL argument");
    if (n != d->nparam) return dn_fail(d, MCX_E_ARG, "n must equal the parameter count");
    DNC(d, cudaMemcpy(d->params.p, host, n * 4, cudaMemcpyHostToDevice), "writing parameters");
    d->step = 0;
    DNC(d, cudaMemset(d->m1.p, 0, d->nparam * 4), "resetting Adam");
    DNC(d, cudaMemset(d->m2.p, 0, d->nparam * 4), "resetting Adam");
    mcx_status s = refresh_weights(d, nullptr);
    if (s != MCX_OK) return s;
    DNC(d, cudaDeviceSynchronize(), "refreshing weights");
    return MCX_OK;
}

mcx_status mcx_denoiser_forward(mcx_denoiser *d, const float *x_dev, float *y_dev, uint32_t n,
                                void *stream)
{
    if (!d || !x_dev || !y_dev) return dn_fail(d, MCX_E_ARG, "NULL argument");
    if (n < 1 || (int)n > d->maxb) return dn_fail(d, MCX_E_ARG, "n must be 1..max_batch");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mcx_status s = forward(d, x_dev, (int)n, d->out.as<float>(), st);
    if (s != MCX_OK) return s;
    DNC(d, cudaMemcpyAsync(y_dev, d->out.p, (size_t)level_vol(d, 0, n).pos() * 4, cudaMemcpyDeviceToDevice, st),
        "copying the output");
    return MCX_OK;
}

mcx_status mcx_denoiser_train_step(mcx_denoiser *d, const float *x_dev, const float *t_dev,
                                   uint32_t n, float lr, float *loss_host, void *stream)
{
    if (!d || !x_dev || !t_dev) return dn_fail(d, MCX_E_ARG, "NULL argument");
    if (n < 1 || (int)n > d->maxb) return dn_fail(d, MCX_E_ARG, "n must be 1..max_batch");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mcx_status s = forward(d, x_dev, (int)n, d->out.as<float>(), st);
    if (s != MCX_OK) return s;
    if ((s = backward(d, x_dev, t_dev, (int)n, st)) != MCX_OK) return s;
    if (lr > 0.f) {
        d->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f / (1.f - std::pow(b1, (float)d->step));
        const float c2 = 1.f / (1.f - std::pow(b2, (float)d->step));
        adam_step<<<grid1((long long)d->nparam), 256, 0, st>>>(d->params.as<float>(), d->grads.as<float>(),
                                                               d->m1.as<float>(), d->m2.as<float>(),
                                                               (long long)d->nparam, lr, b1, b2, c1, c2, 1e-8f);
        DNC(d, cudaGetLastError(), "optimizer step");
        if ((s = refresh_weights(d, st)) != MCX_OK) return s;
    }
    if (loss_host) {
        DNC(d, cudaMemcpyAsync(loss_host, d->loss.p, 4, cudaMemcpyDeviceToHost, st), "reading the loss");
        DNC(d, cudaStreamSynchronize(st), "waiting for the step");
        return check_status(d);
    }
    return MCX_OK;
}

mcx_status mcx_denoiser_set_encoding(mcx_denoiser *d, float floor_, float mu, float sigma)
{
    if (!d) return dn_fail(nullptr, MCX_E_ARG, "NULL denoiser");
    if (!(floor_ > 0.f) || !(sigma > 0.f) || !std::isfinite(mu) || !std::isfinite(floor_) || !std::isfinite(sigma))
        return dn_fail(d, MCX_E_ARG, "need floor > 0, sigma > 0, finite mu");
    d->floor_ = floor_; d->mu = mu; d->sigma = sigma;
    return MCX_OK;
}

mcx_status mcx_denoiser_encode(mcx_denoiser *d, const float *phi_dev, float *x_dev, uint64_t count, void *stream)
{
    if (!d || (count && (!phi_dev || !x_dev))) return dn_fail(d, MCX_E_ARG, "NULL argument");
    if (!count) return MCX_OK;
    encode_kernel<<<grid1((long long)count), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        phi_dev, (long long)count, d->floor_, d->mu, 1.f / d->sigma, x_dev);
    DNC(d, cudaGetLastError(), "encode");
    return MCX_OK;
}

mcx_status mcx_denoiser_decode(mcx_denoiser *d, const float *x_dev, float *phi_dev, uint64_t count, void *stream)
{
    if (!d || (count && (!phi_dev || !x_dev))) return dn_fail(d, MCX_E_ARG, "NULL argument");
    if (!count) return MCX_OK;
    decode_kernel<<<grid1((long long)count), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        x_dev, (long long)count, d->floor_, d->mu, d->sigma, phi_dev);
    DNC(d, cudaGetLastError(), "decode");
    return MCX_OK;
}

mcx_status mcx_denoiser_apply(mcx_denoiser *d, const float *phi_in_dev, float *phi_out_dev, uint32_t n,
                              void *stream)
{
    if (!d || !phi_in_dev || !phi_out_dev) return dn_fail(d, MCX_E_ARG, "NULL argument");
    if (n < 1 || (int)n > d->maxb) return dn_fail(d, MCX_E_ARG, "n must be 1..max_batch");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long cnt = level_vol(d, 0, (int)n).pos();
    encode_kernel<<<grid1(cnt), 256, 0, st>>>(phi_in_dev, cnt, d->floor_, d->mu, 1.f / d->sigma, d->xin.as<float>());
    DNC(d, cudaGetLastError(), "encode");
    mcx_status s = forward(d, d->xin.as<float>(), (int)n, d->out.as<float>(), st);
    if (s != MCX_OK) return s;
    decode_kernel<<<grid1(cnt), 256, 0, st>>>(d->out.as<float>(), cnt, d->floor_, d->mu, d->sigma, phi_out_dev);
    DNC(d, cudaGetLastError(), "decode");
    return MCX_OK;
}

mcx_status mcx_denoiser_gather(mcx_denoiser *d, const float *set_dev, uint64_t set_count,
                               const uint64_t *idx, const uint32_t *flags, uint32_t n,
                               float *dst_dev, void *stream)
{
    if (!d || !set_dev || !idx || !flags || !dst_dev) return dn_fail(d, MCX_E_ARG, "NULL argument");
    if (n < 1 || (int)n > kMaxGather) return dn_fail(d, MCX_E_ARG, "n must be 1..64");
    GatherList L;
    for (uint32_t s = 0; s < n; ++s) {
        if (idx[s] >= set_count) return dn_fail(d, MCX_E_ARG, "index beyond the set");
        if (flags[s] > 7u || ((flags[s] & 4u) && d->H != d->W))
            return dn_fail(d, MCX_E_ARG, "flags must be 0..7 (bit 2 needs ny == nx)");
        L.idx[s] = idx[s];
        L.flags[s] = flags[s];
    }
    const long long total = level_vol(d, 0, (int)n).pos();
    gather_kernel<<<grid1(total), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        set_dev, L, (int)n, d->D, d->H, d->W, dst_dev);
    DNC(d, cudaGetLastError(), "gather");
    return MCX_OK;
}

mcx_status mcx_denoiser_sync(mcx_denoiser *d)
{
    if (!d) return dn_fail(nullptr, MCX_E_ARG, "NULL denoiser");
    DNC(d, cudaDeviceSynchronize(), "waiting");
    return check_status(d);
}

void mcx_denoiser_destroy(mcx_denoiser *d)
{
    if (!d) return;
    cudaDeviceSynchronize();
    delete d;
}

// One convolution on host arrays (parity diagnostic): kind 0 = forward with bias and ReLU
// (x [n][d][h][w][cin] -> y [..][cout]); kind 1 = weight gradient (x, dy -> dW [27][cout][cin]).
// Arrays are FP32 on the host and rounded to BF16 on the way in.
mcx_status mcx_debug_conv3d(int32_t kind, int32_t n, int32_t dd, int32_t hh, int32_t ww, int32_t cin,
                            int32_t cout, const float *x, const float *w, const float *bias,
                            const float *dy, float *out)
{
    if (!x || !out || kind < 0 || kind > 1 || (kind == 0 && !w) || (kind == 1 && !dy) || ww % 16 || n < 1)
        return dn_fail(nullptr, MCX_E_ARG, "bad arguments");
    const Vol v{n, dd, hh, ww};
    const long long P = v.pos();
    std::vector<bf16> hx(P * cin), hw, hdy;
    for (long long i = 0; i < P * cin; ++i) hx[i] = __float2bfloat16(x[i]);
    DBuf bx, bw, bb, bdy, by, bdw;
    cudaError_t e = bx.alloc(hx.size() * 2);
    if (e == cudaSuccess) e = cudaMemcpy(bx.p, hx.data(), hx.size() * 2, cudaMemcpyHostToDevice);
    if (kind == 0) {
        hw.resize(27ull * cin * cout);
        for (size_t i = 0; i < hw.size(); ++i) hw[i] = __float2bfloat16(w[i]);
        if (e == cudaSuccess) e = bw.alloc(hw.size() * 2);
        if (e == cudaSuccess) e = cudaMemcpy(bw.p, hw.data(), hw.size() * 2, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && bias) e = bb.alloc(cout * 4);
        if (e == cudaSuccess && bias) e = cudaMemcpy(bb.p, bias, cout * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = by.alloc(P * cout * 2);
        DBuf berr;
        if (e == cudaSuccess) e = berr.alloc(4);
        if (e == cudaSuccess) e = cudaMemset(berr.p, 0, 4);
        if (e == cudaSuccess)
            e = launch_fwd_tc(bx.as<bf16>(), cin, bw.as<bf16>(), bias ? bb.as<float>() : nullptr, v, cout, 1,
                              by.as<bf16>(), berr.as<unsigned>(), nullptr);
        unsigned herr = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&herr, berr.p, 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && herr) return dn_fail(nullptr, MCX_E_TIMEOUT, "tensor-core wait timed out");
        std::vector<bf16> hy(P * cout);
        if (e == cudaSuccess) e = cudaMemcpy(hy.data(), by.p, hy.size() * 2, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) for (size_t i = 0; i < hy.size(); ++i) out[i] = __bfloat162float(hy[i]);
    } else {
        hdy.resize(P * cout);
        for (size_t i = 0; i < hdy.size(); ++i) hdy[i] = __float2bfloat16(dy[i]);
        if (e == cudaSuccess) e = bdy.alloc(hdy.size() * 2);
        if (e == cudaSuccess) e = cudaMemcpy(bdy.p, hdy.data(), hdy.size() * 2, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = bdw.alloc(27ull * cin * cout * 4);
        if (e == cudaSuccess) e = cudaMemset(bdw.p, 0, 27ull * cin * cout * 4);
        if (e == cudaSuccess) e = launch_bwd_w(bx.as<bf16>(), cin, bdy.as<bf16>(), cout, v, bdw.as<float>(), nullptr);
        if (e == cudaSuccess) e = cudaMemcpy(out, bdw.p, 27ull * cin * cout * 4, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return dn_fail(nullptr, MCX_E_CUDA, std::string("debug conv: ") + cudaGetErrorString(e));
    return MCX_OK;
}

}  // extern "C"
