// Learned 3-D denoiser for low-photon fluence maps: a small U-Net (3 levels, 16/32/64
// channels, 3x3x3 convolutions) with BF16 weights and activations and FP32 accumulation,
// trained and run by hand-written tensor-core kernels: the convolutions, their input
// gradients and their weight gradients on tcgen05 (TMA-fed shared-memory operands,
// accumulators in tensor memory).
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
#include <cuda.h>
#include <cudaTypedefs.h>
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

struct Vol {
    int n, d, h, w;               // batch, depth (z), height (y), width (x)
    __host__ __device__ long long pos() const { return (long long)n * d * h * w; }
};

// ------------------------------------------------------------------------ convolution
// Y[p][co] = act(bias[co] + sum_tap sum_ci X[p + off(tap)][ci] * W[tap][co][ci]) (zero
// outside the volume) as an implicit GEMM on the 5th-generation tensor cores.
//
// Tiles.  Within one z-plane, positions are numbered along padded lines of pitch
// PW = W + 2: q = y * PW + (x + 1), so x = -1 and x = W are pad columns.  A tile is 128
// consecutive q (GEMM rows M = 128); rows that land on pad columns or past the last line
// are computed and discarded.  In this numbering the tap (dz, dy, dx) reads row
// q + dy * PW + dx of plane z + dz, so for a fixed dz all nine (dy, dx) taps read one
// window of consecutive rows at offsets dy * PW + dx.  In conv3d_fwd_tc the window is one
// TMA box of [16 channels][PW columns from x = -1][L lines][1 plane][1 volume] per
// 16-channel group: the tensor map's out-of-bounds fill supplies the zero padding
// (x = -1, x = W, lines and planes outside the volume), and the box lands in shared
// memory as consecutive 32-byte rows in q order, swizzled by the TMA unit in the 32-byte
// pattern -- the K-major SWIZZLE_32B operand layout (one row holds one MMA's K = 16;
// 8-row groups 256 B apart), so a one-row shift of the operand is a 32-byte shift of its
// start address (the swizzle follows absolute shared addresses).  Two 16-channel groups
// per 32-byte row halve the TMA rows of the earlier 8-channel boxes.  conv3d_fwd_ws stages
// 8-channel boxes of 16-byte rows in the no-swizzle layout
// (8-row core matrices 128 B apart; chunks one leading-dimension offset apart).  A tile
// takes 3 windows (one per plane); each feeds 9 taps x cin/16 tcgen05.mma instructions
// (K = 16, N = COUT).
//
// Warp roles (6 warps, persistent over tiles): warp 0 lane 0 issues the TMA loads into a
// ring of stages (mbarrier "full" with transaction bytes); warp 1 lane 0 issues the MMAs
// and commits to "empty" (the stage may be refilled) and, after a tile's last window, to
// "acc full"; warps 2-5 read the accumulator out (tcgen05.ld; warp w reads TMEM lanes
// 32 (w mod 4) ...), arrive on "acc empty", and store bias + ReLU in BF16 for the valid
// rows.  Several TMEM accumulators let a tile's read-out overlap the next tiles' MMAs.
// The layer's weights stay resident in shared memory when they fit (one TMA load each).
// With cout = 16 the three tiles a window feeds sit in consecutive accumulators and take
// one MMA of N = 48 per (dy, dx) tap and K step (two where the accumulator ring wraps), so
// the window's A rows are read from shared memory once instead of three times.
//
// Every wait is bounded: on a timeout the role records an error and stops; the CTA still
// waits (bounded) for its TMA loads and for the MMAs it issued, then frees its tensor
// memory.
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

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

constexpr int kTcRows = 128, kTcThreads = 192, kTcFwdHeader = 384;
constexpr int kTcWallMax = 64 * 1024;       // weights up to this size stay resident
constexpr int kTcSmemBudget = 112 * 1024;   // preferred shared memory per CTA
constexpr int kTcSmemMax = 227 * 1024;      // shared memory one CTA may use
constexpr int kTcMaxStages = 8;

__host__ __device__ constexpr bool tc_wall(int cin, int cout) { return 27 * cin * cout * 2 <= kTcWallMax; }
// resident weights and cout 16: one window's products for its (up to) three tiles go out
// as one MMA with N = tiles x cout (weights stored dz-interleaved per (dy, dx) tap).  With
// cout 32 the same scheme measured slower (four accumulators: the MMA thread waits for
// read-outs, since a tile completes only with the whole window's MMAs)
__host__ __device__ constexpr bool tc_merge(int cin, int cout) { return tc_wall(cin, cout) && cout == 16; }
// TMEM columns per accumulator and accumulators per CTA (the launch counts their product
// against an SM's 512 columns when it sizes the grid)
__host__ __device__ constexpr int tc_ncol(int cin, int cout)
{
    return tc_merge(cin, cout) ? cout : (cout <= 32 ? 32 : (cout <= 64 ? 64 : 128));
}
__host__ __device__ constexpr int tc_nslot(int cin, int cout)
{
    return tc_merge(cin, cout) ? 8 : (tc_wall(cin, cout) ? 4 : 2);
}
// lines of a window: the tile's rows q0 - 1 - PW .. q0 + 128 + PW
__host__ __device__ constexpr int tc_lines(int w) { return (kTcRows + 2 + w + 1) / (w + 2) + 3; }
// one 8-channel chunk of a window: L lines x PW rows of 16 B, padded to 128 B
__host__ __device__ constexpr int tc_lbo_a(int w) { return ((tc_lines(w) * (w + 2) * 16 + 127) / 128) * 128; }
// one 16-channel group of a window: L lines x PW rows of 32 B, swizzled in 256-byte atoms
// (SWIZZLE_32B), padded to 1 KiB so that every group starts on a swizzle-atom boundary
__host__ __device__ constexpr int tc_gbytes(int w) { return ((tc_lines(w) * (w + 2) * 32 + 1023) / 1024) * 1024; }
__host__ __device__ constexpr int tc_stage_bytes(int cin, int cout, int w)
{
    return (cin / 16) * tc_gbytes(w) + (tc_wall(cin, cout) ? 0 : ((9 * cout * cin * 2 + 1023) / 1024) * 1024);
}
__host__ __device__ constexpr int tc_smem_bytes(int cin, int cout, int w, int ns)
{
    return 1024 + kTcFwdHeader + (tc_wall(cin, cout) ? 27 * cout * cin * 2 : 0) + 1024 + ns * tc_stage_bytes(cin, cout, w);
}
// shared-memory descriptor of a K-major operand in the 32-byte swizzle (layout type 6):
// rows of 32 B (K = 16 BF16, one MMA's K), 8-row groups 256 B apart (SBO); the leading
// offset is unused at this K.  The hardware applies the swizzle on the absolute shared
// address, so a start address shifted by any whole number of rows (the taps' row offsets)
// needs no base offset (measured: base offset 0 reproduces the oracle, the start address's
// bits 7..9 as base offset do not)
__device__ __forceinline__ uint64_t sw32_desc(uint32_t saddr)
{
    const uint64_t bo = 0ull;
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(256 >> 4) << 32) | (1ull << 46) |
           (bo << 49) | (6ull << 61);
}
// ring depth: each CTA has one MMA-issuing thread, so more resident CTAs issue more
// MMAs; prefer 3-8 stages within a quarter of the SM's shared memory (4 CTAs), then 2-8
// within half (2 CTAs), then 2-4 within all of it; 0 when not even 2 fit
__host__ __device__ constexpr int tc_stages(int cin, int cout, int w)
{
    for (int ns = kTcMaxStages; ns >= 3; --ns)
        if (tc_smem_bytes(cin, cout, w, ns) <= kTcSmemBudget / 2) return ns;
    for (int ns = kTcMaxStages; ns >= 2; --ns)
        if (tc_smem_bytes(cin, cout, w, ns) <= kTcSmemBudget) return ns;
    for (int ns = 4; ns >= 2; --ns)
        if (tc_smem_bytes(cin, cout, w, ns) <= kTcSmemMax) return ns;
    return 0;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit = 1 << 22)
{
    for (int it = 0; it < limit; ++it) {            // 1 << 22: about a second of polling
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n"
                 ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
                   "r"(bar) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];\n"
                 ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar) : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(kTcThreads)
conv3d_fwd_tc(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmw,
              const float *__restrict__ bias, Vol v, int relu, bf16 *__restrict__ Y, unsigned *err, int ns,
              int zc)
{
    constexpr int cin = CIN;
    constexpr bool WALL = tc_wall(CIN, COUT);
    constexpr bool MERGE = tc_merge(CIN, COUT);
    constexpr int NCOL = tc_ncol(CIN, COUT);                           // TMEM columns per accumulator
    constexpr int NSLOT = tc_nslot(CIN, COUT);                         // accumulators per CTA
    constexpr uint32_t IDESC = idesc_bf16_f32(kTcRows, COUT);
    extern __shared__ unsigned char smem_raw[];
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;      // 1 KiB aligned
    // header: full[ns] at 0, empty[ns] at 64, acc full[NSLOT] at 128, acc empty[NSLOT] at
    // 192, weights barrier at 256, MMA drain barrier at 264, TMEM address at 320
    const uint32_t full0 = base, empty0 = base + 64, accf0 = base + 128, acce0 = base + 192, wbar = base + 256;
    const uint32_t drain = base + 264;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem_raw + (base + 320 - smem_u32(smem_raw)));
    const int wtap = COUT * cin * 2, lbo_b = COUT * 16;
    const int PW = v.w + 2, L = tc_lines(v.w), lbo_a = tc_gbytes(v.w);
    const int a_bytes = (cin / 16) * lbo_a;
    const uint32_t wres = base + kTcFwdHeader;
    const uint32_t ring = (wres + (WALL ? 27 * wtap : 0) + 1023u) & ~1023u;
    const int stage_bytes = tc_stage_bytes(CIN, COUT, v.w);
    // merged weights: per (dy, dx) tap tt and 8-channel chunk c, the rows of dz = +1, 0, -1
    // (cout each, 16 B per row) one after another, so the tiles w - 1, w, w + 1 that a
    // window of plane w feeds are consecutive N rows; chunks LBOM bytes apart
    constexpr int LBOM = 3 * COUT * 16;
    const int tid = threadIdx.x, warp = tid >> 5;
    // work units: columns of up to zc tiles at the same q0 in consecutive planes
    const int tiles_plane = (v.h * PW + kTcRows - 1) / kTcRows;
    const int cols_z = (v.d + zc - 1) / zc;
    const int n_units = v.n * cols_z * tiles_plane;
    const int my_units = n_units > (int)blockIdx.x ? (n_units - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    struct Unit { int b, z0, nz, q0; };
    auto unit_of = [&](int j) {
        const int u = (int)blockIdx.x + j * (int)gridDim.x;
        const int k = u % tiles_plane, r = u / tiles_plane;
        const int z0 = (r % cols_z) * zc;
        return Unit{r / cols_z, z0, min(zc, v.d - z0), k * kTcRows};
    };
    // first window line: one above the line of q0 - 1
    auto first_line = [&](int q0) { return (q0 >= 1 ? (q0 - 1) / PW : -1) - 1; };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(smem_u32(tslot)), "r"(NSLOT * NCOL) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < ns; ++b) {
            mbar_init(full0 + 8 * b, 1);
            mbar_init(empty0 + 8 * b, 1);
        }
        for (int a = 0; a < NSLOT; ++a) {
            mbar_init(accf0 + 8 * a, 1);
            mbar_init(acce0 + 8 * a, 4 * 32);
        }
        mbar_init(wbar, 1);
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok = true;

    if (tid == 0) {
        // ------------------------------------------------------------ producer (TMA)
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmx)) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmw)) : "memory");
        if (WALL && my_units) {
            mbar_expect_tx(wbar, 27 * wtap);
            for (int tap = 0; tap < 27; ++tap)
                for (int c = 0; c < cin / 8; ++c) {
                    const int tt = tap % 9, dzi = 2 - tap / 9;    // dzi = 1 - dz
                    const uint32_t dst = MERGE ? wres + tt * 3 * wtap + c * LBOM + dzi * COUT * 16
                                               : wres + tap * wtap + c * lbo_b;
                    tma_load_2d(dst, &tmw, 8 * c, tap * COUT, wbar);
                }
        }
        const uint32_t tx = (cin / 16) * (L * PW * 32) + (WALL ? 0 : 9 * wtap);
        int b = 0, use = 0;
        for (int uj = 0; uj < my_units && ok; ++uj) {
            const Unit U = unit_of(uj);
            const int fl = first_line(U.q0);
            for (int j = 0; j < U.nz + 2 && ok; ++j) {        // window of plane z0 - 1 + j
                if (use > 0) ok &= mbar_wait(empty0 + 8 * b, (uint32_t)((use - 1) & 1));
                if (!ok) break;
                const uint32_t st = ring + b * stage_bytes, fb = full0 + 8 * b;
                mbar_expect_tx(fb, tx);
                for (int c = 0; c < cin / 16; ++c)
                    tma_load_5d(st + c * lbo_a, &tmx, 16 * c, -1, fl, U.z0 - 1 + j, U.b, fb);
                if (!WALL)                                       // one tile per unit: dz = j - 1
                    for (int tt = 0; tt < 9; ++tt)
                        for (int c = 0; c < cin / 8; ++c)
                            tma_load_2d(st + a_bytes + tt * wtap + c * lbo_b, &tmw, 8 * c, (9 * j + tt) * COUT, fb);
                if (++b == ns) { b = 0; ++use; }
            }
        }
        // every load issued has landed before the CTA may exit
        for (int bb = 0; bb < ns; ++bb) {
            const int issued = use + (bb < b ? 1 : 0);       // fills of buffer bb
            if (issued > 0) ok &= mbar_wait(full0 + 8 * bb, (uint32_t)((issued - 1) & 1));
        }
        if (WALL && my_units) ok &= mbar_wait(wbar, 0);
    } else if (tid == 32) {
        // ------------------------------------------------------------ MMA issuer
        if (WALL && my_units) ok &= mbar_wait(wbar, 0);
        const uint64_t bdesc0 = umma_desc(WALL ? wres : ring + a_bytes, lbo_b, 128);
        int toff[9];                                            // row offset of each (dy, dx) tap
#pragma unroll
        for (int tt = 0; tt < 9; ++tt) toff[tt] = (tt / 3 - 1) * PW + (tt % 3 - 1);
        int b = 0, use = 0, T0 = 0;                             // T0: tiles of earlier units
        for (int uj = 0; uj < my_units && ok; ++uj) {
            const Unit U = unit_of(uj);
            const int off = U.q0 - first_line(U.q0) * PW;      // window row of q0
            for (int j = 0; j < U.nz + 2 && ok; ++j) {
                ok &= mbar_wait(full0 + 8 * b, (uint32_t)(use & 1));
                if (!ok) break;
                tc_fence_after();
                // descriptors differ only in the start-address field (address / 16, 14 bits;
                // every address here is below 256 KiB): base descriptor plus an offset
                const uint32_t abase = ring + (uint32_t)(b * stage_bytes + off * 32);
                if constexpr (MERGE) {
                    // tiles ilo .. ihi read this plane (tile i with dz = j - 1 - i, weight block
                    // dzi = i - j + 2); tile j starts here, tile j - 2 finishes here
                    const int ilo = max(0, j - 2), ihi = min(U.nz - 1, j);
                    const bool starts = ihi == j;
                    if (starts && T0 + j >= NSLOT) {            // the slot's previous tile is read out
                        ok &= mbar_wait(acce0 + 8 * ((T0 + j) & (NSLOT - 1)), (uint32_t)(((T0 + j) / NSLOT - 1) & 1));
                        tc_fence_after();
                    }
                    if (!ok) break;
                    const uint64_t bdm = umma_desc(wres, LBOM, 128);
                    // one MMA for tiles a .. e (consecutive accumulators, no wrap of the ring)
                    auto mma_run = [&](uint64_t ad, uint64_t bk, int a, int e, uint32_t accum) {
                        const uint32_t d = tmem + (uint32_t)(((T0 + a) & (NSLOT - 1)) * NCOL);
                        const uint64_t bd = bk + (uint64_t)(((a - j + 2) * COUT * 16) >> 4);
                        const uint32_t idesc = idesc_bf16_f32(kTcRows, (e - a + 1) * COUT);
                        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                                     ::"r"(d), "l"(ad), "l"(bd), "r"(idesc), "r"(accum) : "memory");
                    };
#pragma unroll
                    for (int tt = 0; tt < 9; ++tt)
#pragma unroll
                        for (int kk = 0; kk < CIN / 16; ++kk) {
                            const uint64_t ad = sw32_desc(abase + (uint32_t)(toff[tt] * 32 + kk * lbo_a));
                            const uint64_t bk = bdm + (uint64_t)((tt * 3 * wtap + 2 * kk * LBOM) >> 4);
                            // the starting tile's first product overwrites its accumulator
                            const bool fresh = starts && tt == 0 && kk == 0;
                            const int last = fresh ? j - 1 : ihi;
                            for (int a = ilo; a <= last;) {
                                const int e = min(last, a + (NSLOT - 1) - ((T0 + a) & (NSLOT - 1)));
                                mma_run(ad, bk, a, e, 1u);
                                a = e + 1;
                            }
                            if (fresh) mma_run(ad, bk, j, j, 0u);
                        }
                    if (j >= 2) tc_commit(accf0 + 8 * ((T0 + j - 2) & (NSLOT - 1)));   // tile j - 2 is complete
                    tc_commit(empty0 + 8 * b);
                    if (++b == ns) { b = 0; ++use; }
                } else {
                    // tiles i of the unit reading this plane, the finishing one first: dz = j - 1 - i
                    for (int i = j - 2; i <= j; ++i) {
                        if (i < 0 || i >= U.nz) continue;
                        const int dz = j - 1 - i, T = T0 + i, slot = T & (NSLOT - 1);
                        if (dz == -1 && T >= NSLOT)                 // the slot's previous tile is read out
                            ok &= mbar_wait(acce0 + 8 * slot, (uint32_t)((T / NSLOT - 1) & 1));
                        if (!ok) break;
                        const uint64_t bbase = WALL ? bdesc0 + (uint64_t)((9 * (dz + 1) * wtap) >> 4)
                                                    : bdesc0 + (uint64_t)((b * stage_bytes) >> 4);
                        const uint32_t d = tmem + slot * NCOL;
#pragma unroll
                        for (int tt = 0; tt < 9; ++tt)              // tt = 3 (dy + 1) + (dx + 1)
#pragma unroll
                            for (int kk = 0; kk < CIN / 16; ++kk) {
                                const uint64_t ad = sw32_desc(abase + (uint32_t)(toff[tt] * 32 + kk * lbo_a));
                                const uint64_t bd = bbase + (uint64_t)((tt * wtap + 2 * kk * lbo_b) >> 4);
                                const uint32_t accum = (dz == -1 && tt == 0 && kk == 0) ? 0u : 1u;
                                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                                             ::"r"(d), "l"(ad), "l"(bd), "r"(IDESC), "r"(accum) : "memory");
                            }
                        if (dz == 1) tc_commit(accf0 + 8 * slot);    // tile i is complete
                    }
                    tc_commit(empty0 + 8 * b);
                    if (++b == ns) { b = 0; ++use; }
                }
            }
            T0 += U.nz;
        }
        // every MMA issued has completed before the CTA may free tensor memory, also when
        // a wait above gave up (the epilogue then no longer waits for the accumulators)
        tc_commit(drain);
        ok &= mbar_wait(drain, 0);
    } else if (warp >= 2) {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp & 3, r = quarter * 32 + (tid & 31);
        int T = 0;
        for (int uj = 0; uj < my_units && ok; ++uj) {
            const Unit U = unit_of(uj);
            const int q = U.q0 + r, y = q / PW, x = q - y * PW - 1;
            const bool valid = y < v.h && x >= 0 && x < v.w;
            for (int i = 0; i < U.nz && ok; ++i, ++T) {
                const int slot = T & (NSLOT - 1);
                ok &= mbar_wait(accf0 + 8 * slot, (uint32_t)((T / NSLOT) & 1));
                ok = __all_sync(0xffffffffu, ok);               // the collective reads below
                if (!ok) break;
                tc_fence_after();
                float a[COUT];
                const uint32_t taddr = tmem + slot * NCOL + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
                for (int c0 = 0; c0 < COUT; c0 += 16) tmem_ld16(taddr + c0, a + c0);
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                tc_fence_before();
                mbar_arrive(acce0 + 8 * slot);
                if (valid) {
                    bf16 *yr = Y + ((((long long)U.b * v.d + U.z0 + i) * v.h + y) * v.w + x) * COUT;
#pragma unroll
                    for (int c = 0; c < COUT; c += 8) {
                        float o[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            o[e] = a[c + e] + (bias ? __ldg(bias + c + e) : 0.f);
                            if (relu) o[e] = fmaxf(o[e], 0.f);
                        }
                        uint4 pk;
                        pk.x = pack_bf16(o[0], o[1]);
                        pk.y = pack_bf16(o[2], o[3]);
                        pk.z = pack_bf16(o[4], o[5]);
                        pk.w = pack_bf16(o[6], o[7]);
                        *reinterpret_cast<uint4 *>(yr + c) = pk;
                    }
                }
            }
        }
    }
    if (!__syncthreads_and(ok) && tid == 0) atomicOr(err, 1u);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NSLOT * NCOL) : "memory");
    }
}

// Layers whose weights do not fit in shared memory (more than 64 KiB: cin x cout of 96 x 32,
// 64 x 64, ...) run weights-stationary: a work unit is TU consecutive tiles with one
// accumulator each (two units' worth of tensor memory, so one unit's read-out overlaps the
// next unit's MMAs), and the unit goes through the planes dz = -1, 0, +1 in turn: the
// plane's 9 taps of weights are loaded once (one buffer, refilled when the previous
// plane's MMAs have completed), then each tile's window of that plane streams through
// the ring.  Weights then cross L2 once per unit and plane instead of once per tile and
// plane.  Tiles, windows, operand layouts and the bounded waits are those of
// conv3d_fwd_tc.
constexpr int kWsHeader = 512;

__host__ __device__ constexpr int ws_tiles_per_unit(int cout)
{
    return cout <= 32 ? 8 : (cout <= 64 ? 4 : 2);          // 2 x TU x columns = 512
}
__host__ __device__ constexpr int ws_smem_bytes(int cin, int cout, int w, int ns)
{
    return 1024 + kWsHeader + 9 * cout * cin * 2 + ns * (cin / 8) * tc_lbo_a(w);
}
__host__ __device__ constexpr int ws_stages(int cin, int cout, int w)
{
    for (int ns = 6; ns >= 2; --ns)
        if (ws_smem_bytes(cin, cout, w, ns) <= kTcSmemMax) return ns;
    return 0;
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(kTcThreads)
conv3d_fwd_ws(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmw,
              const float *__restrict__ bias, Vol v, int relu, bf16 *__restrict__ Y, unsigned *err, int ns)
{
    constexpr int NCOL = COUT <= 32 ? 32 : (COUT <= 64 ? 64 : 128);   // TMEM columns per accumulator
    constexpr int TU = ws_tiles_per_unit(COUT);
    constexpr uint32_t IDESC = idesc_bf16_f32(kTcRows, COUT);
    extern __shared__ unsigned char smem_raw[];
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;      // 1 KiB aligned
    // header: full[ns] at 0, empty[ns] at 64, acc full[2 TU] at 128, acc empty[2 TU] at 256,
    // weights full at 384, weights empty at 392, MMA drain at 400, TMEM address at 448
    const uint32_t full0 = base, empty0 = base + 64, accf0 = base + 128, acce0 = base + 256;
    const uint32_t wfull = base + 384, wempty = base + 392, drain = base + 400;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem_raw + (base + 448 - smem_u32(smem_raw)));
    const int wtap = COUT * CIN * 2, lbo_b = COUT * 16;
    const int PW = v.w + 2, L = tc_lines(v.w), lbo_a = tc_lbo_a(v.w);
    const int a_bytes = (CIN / 8) * lbo_a;
    const uint32_t wbuf = base + kWsHeader;                // one plane's 9 taps
    const uint32_t ring = wbuf + 9 * wtap;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tiles_plane = (v.h * PW + kTcRows - 1) / kTcRows;
    const int n_tiles = v.n * v.d * tiles_plane;
    const int n_units = (n_tiles + TU - 1) / TU;
    const int my_units = n_units > (int)blockIdx.x ? (n_units - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    struct Tl { int b, z, q0; };
    auto tile_at = [&](int tile) {
        const int plane = tile / tiles_plane;
        return Tl{plane / v.d, plane % v.d, (tile % tiles_plane) * kTcRows};
    };
    auto unit_tiles = [&](int uj, int &t0, int &nt) {
        const int u = (int)blockIdx.x + uj * (int)gridDim.x;
        t0 = u * TU;
        nt = min(TU, n_tiles - t0);
    };
    auto first_line = [&](int q0) { return (q0 >= 1 ? (q0 - 1) / PW : -1) - 1; };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(smem_u32(tslot)), "r"(2 * TU * NCOL) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < ns; ++b) {
            mbar_init(full0 + 8 * b, 1);
            mbar_init(empty0 + 8 * b, 1);
        }
        for (int a = 0; a < 2 * TU; ++a) {
            mbar_init(accf0 + 8 * a, 1);
            mbar_init(acce0 + 8 * a, 4 * 32);
        }
        mbar_init(wfull, 1);
        mbar_init(wempty, 1);
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok = true;

    if (tid == 0) {
        // ------------------------------------------------------------ producer (TMA)
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmx)) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmw)) : "memory");
        const uint32_t tx = (CIN / 8) * (L * PW * 16);
        int b = 0, use = 0, wpass = 0;
        for (int uj = 0; uj < my_units && ok; ++uj) {
            int t0, nt;
            unit_tiles(uj, t0, nt);
            for (int g = 0; g < 3 && ok; ++g) {               // plane z + g - 1
                if (wpass > 0) ok &= mbar_wait(wempty, (uint32_t)((wpass - 1) & 1));
                if (!ok) break;
                mbar_expect_tx(wfull, 9 * wtap);
                for (int tt = 0; tt < 9; ++tt)
                    for (int c = 0; c < CIN / 8; ++c)
                        tma_load_2d(wbuf + tt * wtap + c * lbo_b, &tmw, 8 * c, (9 * g + tt) * COUT, wfull);
                ++wpass;
                for (int t = 0; t < nt && ok; ++t) {
                    if (use > 0) ok &= mbar_wait(empty0 + 8 * b, (uint32_t)((use - 1) & 1));
                    if (!ok) break;
                    const Tl T = tile_at(t0 + t);
                    const uint32_t st = ring + b * a_bytes, fb = full0 + 8 * b;
                    mbar_expect_tx(fb, tx);
                    for (int c = 0; c < CIN / 8; ++c)
                        tma_load_5d(st + c * lbo_a, &tmx, 8 * c, -1, first_line(T.q0), T.z + g - 1, T.b, fb);
                    if (++b == ns) { b = 0; ++use; }
                }
            }
        }
        for (int bb = 0; bb < ns; ++bb) {                     // every load has landed
            const int issued = use + (bb < b ? 1 : 0);
            if (issued > 0) ok &= mbar_wait(full0 + 8 * bb, (uint32_t)((issued - 1) & 1));
        }
        if (wpass > 0) ok &= mbar_wait(wfull, (uint32_t)((wpass - 1) & 1));
    } else if (tid == 32) {
        // ------------------------------------------------------------ MMA issuer
        const uint64_t adesc0 = umma_desc(ring, lbo_a, 128);
        const uint64_t bdesc0 = umma_desc(wbuf, lbo_b, 128);
        int toff[9];
#pragma unroll
        for (int tt = 0; tt < 9; ++tt) toff[tt] = (tt / 3 - 1) * PW + (tt % 3 - 1);
        int b = 0, use = 0, wpass = 0;
        for (int uj = 0; uj < my_units && ok; ++uj) {
            int t0, nt;
            unit_tiles(uj, t0, nt);
            const int set = uj & 1;
            for (int g = 0; g < 3 && ok; ++g) {
                ok &= mbar_wait(wfull, (uint32_t)(wpass & 1));
                if (!ok) break;
                for (int t = 0; t < nt && ok; ++t) {
                    const int slot = set * TU + t;
                    if (g == 0 && uj >= 2)                      // the slot's previous tile is read out
                        ok &= mbar_wait(acce0 + 8 * slot, (uint32_t)(((uj >> 1) - 1) & 1));
                    ok &= mbar_wait(full0 + 8 * b, (uint32_t)(use & 1));
                    if (!ok) break;
                    tc_fence_after();
                    const Tl T = tile_at(t0 + t);
                    const int off = T.q0 - first_line(T.q0) * PW;
                    const uint64_t abase = adesc0 + (uint64_t)((b * a_bytes + off * 16) >> 4);
                    const uint32_t d = tmem + slot * NCOL;
#pragma unroll
                    for (int tt = 0; tt < 9; ++tt)
#pragma unroll
                        for (int kk = 0; kk < CIN / 16; ++kk) {
                            const uint64_t ad = abase + (uint64_t)(int64_t)((toff[tt] * 16 + 2 * kk * lbo_a) >> 4);
                            const uint64_t bd = bdesc0 + (uint64_t)((tt * wtap + 2 * kk * lbo_b) >> 4);
                            const uint32_t accum = (g == 0 && tt == 0 && kk == 0) ? 0u : 1u;
                            asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                         " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                                         ::"r"(d), "l"(ad), "l"(bd), "r"(IDESC), "r"(accum) : "memory");
                        }
                    tc_commit(empty0 + 8 * b);
                    if (g == 2) tc_commit(accf0 + 8 * slot);    // tile t of the unit is complete
                    if (++b == ns) { b = 0; ++use; }
                }
                tc_commit(wempty);                              // this plane's weights are free
                ++wpass;
            }
        }
        // every MMA issued has completed before the CTA may free tensor memory, also when
        // a wait above gave up (the epilogue then no longer waits for the accumulators)
        tc_commit(drain);
        ok &= mbar_wait(drain, 0);
    } else if (warp >= 2) {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp & 3, r = quarter * 32 + (tid & 31);
        for (int uj = 0; uj < my_units && ok; ++uj) {
            int t0, nt;
            unit_tiles(uj, t0, nt);
            for (int t = 0; t < nt && ok; ++t) {
                const int slot = (uj & 1) * TU + t;
                ok &= mbar_wait(accf0 + 8 * slot, (uint32_t)((uj >> 1) & 1));
                ok = __all_sync(0xffffffffu, ok);               // the collective reads below
                if (!ok) break;
                tc_fence_after();
                float a[COUT];
                const uint32_t taddr = tmem + slot * NCOL + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
                for (int c0 = 0; c0 < COUT; c0 += 16) tmem_ld16(taddr + c0, a + c0);
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                tc_fence_before();
                mbar_arrive(acce0 + 8 * slot);
                const Tl T = tile_at(t0 + t);
                const int q = T.q0 + r, y = q / PW, x = q - y * PW - 1;
                if (y < v.h && x >= 0 && x < v.w) {
                    bf16 *yr = Y + ((((long long)T.b * v.d + T.z) * v.h + y) * v.w + x) * COUT;
#pragma unroll
                    for (int c = 0; c < COUT; c += 8) {
                        float o[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            o[e] = a[c + e] + (bias ? __ldg(bias + c + e) : 0.f);
                            if (relu) o[e] = fmaxf(o[e], 0.f);
                        }
                        uint4 pk;
                        pk.x = pack_bf16(o[0], o[1]);
                        pk.y = pack_bf16(o[2], o[3]);
                        pk.z = pack_bf16(o[4], o[5]);
                        pk.w = pack_bf16(o[6], o[7]);
                        *reinterpret_cast<uint4 *>(yr + c) = pk;
                    }
                }
            }
        }
    }
    if (!__syncthreads_and(ok) && tid == 0) atomicOr(err, 1u);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * TU * NCOL) : "memory");
    }
}

// ------------------------------------------------------ weight gradient on tcgen05
// dW[tap][co][ci] = sum_p dY[p][co] X[p + off(tap)][ci] as tcgen05 GEMMs whose reduction
// (K) runs over positions q, numbered along padded lines as in the forward kernel.  The
// taps are stacked into the MMA's two free dimensions by shifted reads of staged windows,
// both read MN-major (channels contiguous) in the 32-byte swizzle:
//   M = (a, ci), a = dx + 1: the X window, one 16-channel atom per a, atoms one 32-byte
//       row apart, so atom a reads the row a positions further on (a = 0..3, M = 64; the
//       products of a = 3 are computed and discarded);
//   N = (j, co), j = 1 - dy: the dY window, atoms one padded line (PW rows) apart.
// For K index b, atom pair (a, j) multiplies X[b - PW - 1 + a] with dY[b + (j - 2) PW]:
// the tap (dy, dx) = (1 - j, a - 1) at dY position p = b + (j - 2) PW.  A plane's K range
// runs over (h + 2) padded lines, so every shift j covers each position of the plane
// exactly once; rows outside the volume come in as zeros from the tensor maps'
// out-of-bounds fill (pad columns, lines and planes outside) and add nothing.  One MMA of
// M = 64, N = 48, K = 16 thus forms 9 taps x 16 x 16 products, 3/4 of its rows useful.
//
// Work units are columns of up to zc planes at one q0, as in the forward kernel.  A stage
// holds the X and dY windows of one plane w = z0 - 1 .. z0 + nz (dY only for the unit's
// own planes); the MMAs of stage w form the dz = 0 product X_w dY_w and, with the
// previous stage's windows, the dz = +1 product X_w dY_(w-1) and the dz = -1 product
// X_(w-1) dY_w.  A stage is released once the next one's MMAs are issued, so each plane's
// windows are loaded once per unit.  A CTA handles one pair of 16-channel groups (cin
// group, cout group) and sums the three dz products over all its units in tensor memory
// (3 x 48 of 256 allocated columns); after its last MMA the four warps read them out and
// add them to dW with FP32 atomics.  Warp 0 lane 0 issues the TMA loads, warp 1 lane 0
// the MMAs; every wait is bounded.
constexpr int kWtThreads = 128, kWtM = 64, kWtN = 48, kWtCols = 256, kWtHeader = 1024;

// lines of a window: X rows from q0 - PW - 1 through q0 - PW + 129, dY rows from
// q0 - 2 PW through q0 + 127
__host__ __device__ constexpr int wt_xlines(int w) { return 130 / (w + 2) + 2; }
__host__ __device__ constexpr int wt_ylines(int w) { return 127 / (w + 2) + 4; }
// a window in shared memory: its lines of PW 32-byte rows plus 2 KiB that no load writes
// (a bound on any read past the window), rounded to 1 KiB (swizzle atoms stay aligned)
__host__ __device__ constexpr int wt_win_bytes(int lines, int w) { return ((lines * (w + 2) * 32 + 2048 + 1023) / 1024) * 1024; }
__host__ __device__ constexpr int wt_stage_bytes(int w) { return wt_win_bytes(wt_xlines(w), w) + wt_win_bytes(wt_ylines(w), w); }
__host__ __device__ constexpr int wt_smem_bytes(int w, int ns) { return 1024 + kWtHeader + ns * wt_stage_bytes(w); }
// ring depth: 3-6 stages within the budget for two CTAs per SM, else 2-4 within one SM
__host__ __device__ constexpr int wt_stages(int w)
{
    for (int ns = 6; ns >= 3; --ns)
        if (wt_smem_bytes(w, ns) <= kTcSmemBudget) return ns;
    for (int ns = 4; ns >= 2; --ns)
        if (wt_smem_bytes(w, ns) <= kTcSmemMax) return ns;
    return 0;
}

// shared-memory descriptor of an MN-major operand in the 32-byte swizzle (layout type 6):
// atoms of 16 MN elements x 8 K rows (rows of 32 B); lbo = byte stride between atoms along
// MN, sbo = byte stride between 8-row groups along K
__device__ __forceinline__ uint64_t sw32_mn_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (6ull << 61);
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(kWtThreads)
conv3d_wgrad_tc(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmdy, Vol v, int ns,
                int zc, float *__restrict__ dW, unsigned *err)
{
    constexpr int NG = COUT / 16;
    // kind::f16, M = 64, N = 48, A and B both MN-major (bits 15 and 16)
    constexpr uint32_t IDESC = idesc_bf16_f32(kWtM, kWtN) | (1u << 15) | (1u << 16);
    extern __shared__ unsigned char smem_raw[];
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;      // 1 KiB aligned
    // header: full[ns] at 0, empty[ns] at 64, MMA drain barrier at 128, TMEM address at 192
    const uint32_t full0 = base, empty0 = base + 64, drain = base + 128;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem_raw + (base + 192 - smem_u32(smem_raw)));
    const int cig = (int)blockIdx.y / NG, cog = (int)blockIdx.y % NG;
    const int PW = v.w + 2, Lx = wt_xlines(v.w), Ly = wt_ylines(v.w);
    const int xbytes = wt_win_bytes(Lx, v.w), stage_bytes = wt_stage_bytes(v.w);
    const uint32_t ring = base + kWtHeader;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // work units: columns of up to zc planes at one q0 over the extended plane
    const int tiles_plane = ((v.h + 2) * PW + kTcRows - 1) / kTcRows;
    const int cols_z = (v.d + zc - 1) / zc;
    const int n_units = v.n * cols_z * tiles_plane;
    const int my_units = n_units > (int)blockIdx.x ? (n_units - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    struct Unit { int b, z0, nz, q0; };
    auto unit_of = [&](int j) {
        const int u = (int)blockIdx.x + j * (int)gridDim.x;
        const int k = u % tiles_plane, r = u / tiles_plane;
        const int z0 = (r % cols_z) * zc;
        return Unit{r / cols_z, z0, min(zc, v.d - z0), k * kTcRows};
    };
    // first window lines (floor division): X from row q0 - PW - 1, dY from row q0 - 2 PW
    auto x_line = [&](int q0) { const int r = q0 - PW - 1; return r >= 0 ? r / PW : -((PW - 1 - r) / PW); };
    auto y_line = [&](int q0) { return q0 / PW - 2; };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(smem_u32(tslot)), "r"(kWtCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < ns; ++b) {
            mbar_init(full0 + 8 * b, 1);
            mbar_init(empty0 + 8 * b, 1);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            // -------------------------------------------------------- producer (TMA)
            asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmx)) : "memory");
            asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmdy)) : "memory");
            const uint32_t txx = (uint32_t)(Lx * PW * 32), txy = (uint32_t)(Ly * PW * 32);
            int b = 0, use = 0;
            for (int uj = 0; uj < my_units && ok; ++uj) {
                const Unit U = unit_of(uj);
                const int xl = x_line(U.q0), yl = y_line(U.q0);
                for (int j = 0; j < U.nz + 2 && ok; ++j) {     // plane z0 - 1 + j
                    const bool hasy = j >= 1 && j <= U.nz;
                    if (use > 0) ok &= mbar_wait(empty0 + 8 * b, (uint32_t)((use - 1) & 1));
                    if (!ok) break;
                    const uint32_t st = ring + b * stage_bytes, fb = full0 + 8 * b;
                    mbar_expect_tx(fb, txx + (hasy ? txy : 0u));
                    tma_load_5d(st, &tmx, 16 * cig, -1, xl, U.z0 - 1 + j, U.b, fb);
                    if (hasy) tma_load_5d(st + xbytes, &tmdy, 16 * cog, -1, yl, U.z0 - 1 + j, U.b, fb);
                    if (++b == ns) { b = 0; ++use; }
                }
            }
            // every load issued has landed before the CTA may exit
            for (int bb = 0; bb < ns; ++bb) {
                const int issued = use + (bb < b ? 1 : 0);
                if (issued > 0) ok &= mbar_wait(full0 + 8 * bb, (uint32_t)((issued - 1) & 1));
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // -------------------------------------------------------- MMA issuer
            int started = 0;                                    // bit dz + 1: accumulator written
            auto mma = [&](int dzi, uint64_t ad, uint64_t bd) {
                const uint32_t accum = (uint32_t)((started >> dzi) & 1);
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             ::"r"(tmem + (uint32_t)(dzi * kWtN)), "l"(ad), "l"(bd), "r"(IDESC), "r"(accum)
                             : "memory");
                started |= 1 << dzi;
            };
            const uint32_t xlbo = 32, ylbo = (uint32_t)(PW * 32), sbo = 256;
            int b = 0, use = 0, bp = 0;
            for (int uj = 0; uj < my_units && ok; ++uj) {
                const Unit U = unit_of(uj);
                // window rows of K index q0
                const uint32_t rx = (uint32_t)(U.q0 - PW - 1 - x_line(U.q0) * PW) * 32;
                const uint32_t ry = (uint32_t)(U.q0 % PW) * 32;
                for (int j = 0; j < U.nz + 2 && ok; ++j) {
                    ok &= mbar_wait(full0 + 8 * b, (uint32_t)(use & 1));
                    if (!ok) break;
                    tc_fence_after();
                    const bool hasy = j >= 1 && j <= U.nz, prevy = j >= 2;
                    const uint32_t xs = ring + b * stage_bytes, xp = ring + bp * stage_bytes;
                    const uint32_t ys = xs + xbytes, yp = xp + xbytes;
#pragma unroll 1
                    for (int kk = 0; kk < kTcRows / 16; ++kk) {
                        const uint32_t ko = (uint32_t)(kk * 16 * 32);
                        const uint64_t ax = sw32_mn_desc(xs + rx + ko, xlbo, sbo);
                        if (hasy) {
                            const uint64_t ay = sw32_mn_desc(ys + ry + ko, ylbo, sbo);
                            mma(1, ax, ay);                                          // dz = 0
                            mma(0, sw32_mn_desc(xp + rx + ko, xlbo, sbo), ay);         // dz = -1
                        }
                        if (prevy) mma(2, ax, sw32_mn_desc(yp + ry + ko, ylbo, sbo));  // dz = +1
                    }
                    if (j >= 1) tc_commit(empty0 + 8 * bp);             // the previous plane is done
                    if (j == U.nz + 1) tc_commit(empty0 + 8 * b);       // and so is the unit's last
                    bp = b;
                    if (++b == ns) { b = 0; ++use; }
                }
            }
            // every MMA issued has completed before the read-out or the release of tensor
            // memory, also when a wait above gave up
            tc_commit(drain);
            ok &= mbar_wait(drain, 0);
        }
        __syncwarp();
    }
    const bool all_ok = __syncthreads_and(ok);
    if (all_ok && my_units > 0) {
        // ------------------------------------------------------------ read-out
        tc_fence_after();
        // accumulator row r = 16 a + ci (M = 64) sits in TMEM lane 32 (r / 16) + r % 16
        const int a = warp, ci = lane;
        const bool row = lane < 16 && warp < 3;
#pragma unroll 1
        for (int dzi = 0; dzi < 3; ++dzi)
#pragma unroll 1
            for (int jn = 0; jn < 3; ++jn) {
                float acc[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(dzi * kWtN + jn * 16), acc);
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                if (row) {
                    const int tap = 9 * dzi + 3 * (2 - jn) + a;          // (dz, dy, dx) + 1
                    float *w = dW + ((size_t)tap * COUT + 16 * cog) * CIN + 16 * cig + ci;
#pragma unroll
                    for (int co = 0; co < 16; ++co) atomicAdd(w + (size_t)co * CIN, acc[co]);
                }
            }
    }
    if (!all_ok && tid == 0) atomicOr(err, 1u);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kWtCols) : "memory");
    }
}

// ------------------------------------------------------------------------ elementwise
// Elementwise layer kernels on 8-channel (16-byte) chunks; every count and index fits in
// 32 bits (mcx_denoiser_create bounds max_batch * nx * ny * nz * 96).
struct Bf8 {
    uint4 u;
    __device__ void to(float *f) const
    {
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 t = __bfloat1622float2(h[i]);
            f[2 * i] = t.x;
            f[2 * i + 1] = t.y;
        }
    }
    __device__ static Bf8 from(const float *f)
    {
        Bf8 r;
        r.u.x = pack_bf16(f[0], f[1]);
        r.u.y = pack_bf16(f[2], f[3]);
        r.u.z = pack_bf16(f[4], f[5]);
        r.u.w = pack_bf16(f[6], f[7]);
        return r;
    }
};

__device__ __forceinline__ uint4 ld16(const bf16 *p) { return *reinterpret_cast<const uint4 *>(p); }
__device__ __forceinline__ void st16(bf16 *p, uint4 v) { *reinterpret_cast<uint4 *>(p) = v; }

// position p of volume v -> its coarse parent (v's dimensions halved)
__device__ __forceinline__ int parent_of(int p, const Vol &v)
{
    const int x = p % v.w;
    int r = p / v.w;
    const int y = r % v.h;
    r /= v.h;
    const int z = r % v.d, b = r / v.d;
    return ((b * (v.d >> 1) + (z >> 1)) * (v.h >> 1) + (y >> 1)) * (v.w >> 1) + (x >> 1);
}

// the 8 children of coarse position pc (fine volume vf) as fine indices
__device__ __forceinline__ void children_of(int pc, const Vol &vf, int *ch)
{
    const int wc = vf.w >> 1, hc = vf.h >> 1, dc = vf.d >> 1;
    const int x = pc % wc;
    int r = pc / wc;
    const int y = r % hc;
    r /= hc;
    const int z = r % dc, b = r / dc;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        ch[k] = ((b * vf.d + 2 * z + (k >> 2)) * vf.h + 2 * y + ((k >> 1) & 1)) * vf.w + 2 * x + (k & 1);
}

#define GRID_LOOP(i, n) \
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)

// ReLU backward fused with the bias gradient: zero dY where the stored output is not
// positive and add what survives into db[channel].  Chunk i holds channels
// 8 (i mod C/8) .. +7 of position i / (C/8); the grid stride is a multiple of 256 chunks,
// so each thread keeps one 8-channel group and sums it in registers, then lanes of the
// same group, then the block's warps, with one atomic per channel per block.
template <int C>
__global__ void __launch_bounds__(256) relu_bias_grad(bf16 *dY, const bf16 *Y, int n8, float *db)
{
    static_assert(C % 8 == 0 && 32 % (C / 8) == 0, "8-channel groups must tile a warp");
    constexpr int G = C / 8;
    __shared__ float red[8][C];
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    GRID_LOOP(i, n8) {
        float y[8], g[8];
        Bf8{ld16(Y + 8 * (size_t)i)}.to(y);
        Bf8{ld16(dY + 8 * (size_t)i)}.to(g);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (y[k] <= 0.f) g[k] = 0.f;
            acc[k] += g[k];
        }
        st16(dY + 8 * (size_t)i, Bf8::from(g).u);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= G; o >>= 1)
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if (lane < G)
#pragma unroll
        for (int k = 0; k < 8; ++k) red[warp][8 * lane + k] = acc[k];
    __syncthreads();
    if (threadIdx.x < C) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
        atomicAdd(db + threadIdx.x, s);
    }
}

// input layer: the FP32 input as channel 0 of a 16-channel BF16 volume, the n_aux medium
// features (aux [volume][feature][position]) as channels 1 .. n_aux, zeros above
__global__ void pad_input(const float *x, const float *aux, int n_aux, int vol, int npos, bf16 *X16)
{
    GRID_LOOP(p, npos) {
        float f[8] = {x[p], 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const int b = p / vol, q = p - b * vol;
        for (int c = 0; c < n_aux; ++c) f[1 + c] = aux[((size_t)b * n_aux + c) * vol + q];
        st16(X16 + 16 * (size_t)p, Bf8::from(f).u);
        st16(X16 + 16 * (size_t)p + 8, make_uint4(0u, 0u, 0u, 0u));
    }
}

// input layer without medium features (one input channel): Y[p][co] = ReLU(b[co] +
// sum_tap W[tap][co][0] x[p + off(tap)]), zero outside the volume.  The 16-channel
// tensor-core path would multiply 15 zero input channels; here each thread forms the 16
// outputs of 4 consecutive positions of a line (the width is a multiple of 16) from the
// FP32 input, rounded to BF16 as the padded path stores it, with FP32 sums on the CUDA
// cores: each input line segment is loaded once per (dz, dy) and each 4-channel weight
// vector (shared memory) serves 16 products
constexpr int kInThreads = 256;
__global__ void __launch_bounds__(kInThreads, 2)
conv_in_fwd(const float *__restrict__ x, const bf16 *__restrict__ W, const float *__restrict__ bias, Vol v,
            bf16 *__restrict__ Y)
{
    __shared__ float4 sw[27][4];                  // W[tap][co][ci = 0], 4 channels per float4
    __shared__ float sb[16];
    for (int i = threadIdx.x; i < 27 * 16; i += blockDim.x)
        reinterpret_cast<float *>(sw)[i] = __bfloat162float(W[(size_t)i * 16]);   // [27][16][16]
    if (threadIdx.x < 16) sb[threadIdx.x] = bias ? bias[threadIdx.x] : 0.f;
    __syncthreads();
    const int nquad = (int)(v.pos() / 4), wq = v.w / 4;
    auto rnd = [](float f) { return __bfloat162float(__float2bfloat16(f)); };
    GRID_LOOP(qd, nquad) {
        const int x0 = 4 * (qd % wq), r1 = qd / wq, yy = r1 % v.h, r2 = r1 / v.h, zz = r2 % v.d, b = r2 / v.d;
        float acc[4][16];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int co = 0; co < 16; ++co) acc[i][co] = sb[co];
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            const int z2 = zz + dz;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const int y2 = yy + dy;
                // the line's inputs at x0 - 1 .. x0 + 4 (zero outside the volume)
                float xs[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if ((unsigned)z2 < (unsigned)v.d && (unsigned)y2 < (unsigned)v.h) {
                    const float *line = x + ((size_t)(b * v.d + z2) * v.h + y2) * v.w;
                    const float4 m = __ldg(reinterpret_cast<const float4 *>(line + x0));   // 16-B aligned
                    xs[1] = rnd(m.x); xs[2] = rnd(m.y); xs[3] = rnd(m.z); xs[4] = rnd(m.w);
                    if (x0 > 0) xs[0] = rnd(__ldg(line + x0 - 1));
                    if (x0 + 4 < v.w) xs[5] = rnd(__ldg(line + x0 + 4));
                }
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const int t = 9 * (dz + 1) + 3 * (dy + 1) + dx;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 wv = sw[t][q];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float xv = xs[i + dx];
                            acc[i][4 * q] = fmaf(xv, wv.x, acc[i][4 * q]);
                            acc[i][4 * q + 1] = fmaf(xv, wv.y, acc[i][4 * q + 1]);
                            acc[i][4 * q + 2] = fmaf(xv, wv.z, acc[i][4 * q + 2]);
                            acc[i][4 * q + 3] = fmaf(xv, wv.w, acc[i][4 * q + 3]);
                        }
                    }
                }
            }
        }
        bf16 *yo = Y + 16 * ((size_t)qd * 4);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int co = 0; co < 16; ++co) acc[i][co] = fmaxf(acc[i][co], 0.f);
            st16(yo + 16 * i, Bf8::from(acc[i]).u);
            st16(yo + 16 * i + 8, Bf8::from(acc[i] + 8).u);
        }
    }
}

// medium features of a label volume: log10(max(mua, 1e-4)) + 2 and
// log10(max(mus (1 - g), 1e-3)), per voxel from a per-label table
__global__ void features_kernel(const uint8_t *labels, int nvox, const float2 *tab, int n_media, float *out)
{
    GRID_LOOP(i, nvox) {
        const int l = labels[i];
        const float2 f = l < n_media ? tab[l] : make_float2(-2.f, -3.f);
        out[i] = f.x;
        out[(size_t)nvox + i] = f.y;
    }
}

// 2x2x2 average pooling; vo is the output (coarse) volume
__global__ void avgpool_fwd(const bf16 *X, Vol vo, int c, bf16 *Y)
{
    const int c8 = c / 8, n = vo.n * vo.d * vo.h * vo.w * c8;
    const Vol vf{vo.n, 2 * vo.d, 2 * vo.h, 2 * vo.w};
    GRID_LOOP(i, n) {
        const int pc = i / c8, j = i - pc * c8;
        int ch[8];
        children_of(pc, vf, ch);
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float f[8];
            Bf8{ld16(X + (size_t)ch[k] * c + 8 * j)}.to(f);
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[e] += f[e];
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[e] *= 0.125f;
        st16(Y + (size_t)pc * c + 8 * j, Bf8::from(acc).u);
    }
}

// gradient of the pooling: each fine position gets its parent's gradient / 8
__global__ void avgpool_bwd(const bf16 *dY, Vol vi, int c, bf16 *dX)
{
    const int c8 = c / 8, n = vi.n * vi.d * vi.h * vi.w * c8;
    GRID_LOOP(i, n) {
        const int p = i / c8, j = i - p * c8;
        float f[8];
        Bf8{ld16(dY + (size_t)parent_of(p, vi) * c + 8 * j)}.to(f);
#pragma unroll
        for (int e = 0; e < 8; ++e) f[e] *= 0.125f;
        st16(dX + (size_t)p * c + 8 * j, Bf8::from(f).u);
    }
}

// nearest x2 upsampling of X (coarse, cx channels) into channels [0, cx) of the fine
// volume vf, and the skip S (cs channels) into channels [cx, cx + cs)
__global__ void upcat_fwd(const bf16 *X, int cx, const bf16 *S, int cs, Vol vf, bf16 *Y)
{
    const int c8 = (cx + cs) / 8, x8 = cx / 8, n = vf.n * vf.d * vf.h * vf.w * c8;
    GRID_LOOP(i, n) {
        const int p = i / c8, j = i - p * c8;
        const uint4 v = j < x8 ? ld16(X + (size_t)parent_of(p, vf) * cx + 8 * j)
                               : ld16(S + (size_t)p * cs + 8 * (j - x8));
        st16(Y + (size_t)p * (cx + cs) + 8 * j, v);
    }
}

// gradient of upcat, coarse part: each coarse position sums its 8 children
__global__ void upcat_bwd_coarse(const bf16 *dY, int cx, int cs, Vol vc, bf16 *dX)
{
    const int c = cx + cs, x8 = cx / 8, n = vc.n * vc.d * vc.h * vc.w * x8;
    const Vol vf{vc.n, 2 * vc.d, 2 * vc.h, 2 * vc.w};
    GRID_LOOP(i, n) {
        const int pc = i / x8, j = i - pc * x8;
        int ch[8];
        children_of(pc, vf, ch);
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float f[8];
            Bf8{ld16(dY + (size_t)ch[k] * c + 8 * j)}.to(f);
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[e] += f[e];
        }
        st16(dX + (size_t)pc * cx + 8 * j, Bf8::from(acc).u);
    }
}

// gradient of upcat, skip part, added to dS
__global__ void upcat_bwd_skip_add(const bf16 *dY, int cx, int cs, int npos, bf16 *dS)
{
    const int c = cx + cs, s8 = cs / 8, n = npos * s8;
    GRID_LOOP(i, n) {
        const int p = i / s8, j = i - p * s8;
        float a[8], b[8];
        Bf8{ld16(dS + (size_t)p * cs + 8 * j)}.to(a);
        Bf8{ld16(dY + (size_t)p * c + cx + 8 * j)}.to(b);
#pragma unroll
        for (int e = 0; e < 8; ++e) a[e] += b[e];
        st16(dS + (size_t)p * cs + 8 * j, Bf8::from(a).u);
    }
}

// head: out[p] = x[p] + hb + sum_c hw[c] Y[p][c]
__global__ void head_fwd(const bf16 *Y, const float *x, const float *hw, const float *hb, int npos, float *out)
{
    GRID_LOOP(p, npos) {
        float y[16];
        Bf8{ld16(Y + 16 * (size_t)p)}.to(y);
        Bf8{ld16(Y + 16 * (size_t)p + 8)}.to(y + 8);
        float s = hb[0];
#pragma unroll
        for (int c = 0; c < 16; ++c) s += hw[c] * y[c];
        out[p] = x[p] + s;
    }
}

// loss L = mean (out - target)^2, dout = 2 (out - target) / n; dY = dout hw; head grads
__global__ void head_bwd(const bf16 *Y, const float *out, const float *target, const float *hw, int npos,
                         bf16 *dY, float *dhw, float *dhb, float *loss)
{
    float gw[16] = {0}, gb = 0.f, l = 0.f;
    const float inv_n = 1.f / (float)npos;
    GRID_LOOP(p, npos) {
        const float e = out[p] - target[p];
        l += e * e * inv_n;
        const float d = 2.f * e * inv_n;
        gb += d;
        float y[16], g[16];
        Bf8{ld16(Y + 16 * (size_t)p)}.to(y);
        Bf8{ld16(Y + 16 * (size_t)p + 8)}.to(y + 8);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            gw[c] += d * y[c];
            g[c] = d * hw[c];
        }
        st16(dY + 16 * (size_t)p, Bf8::from(g).u);
        st16(dY + 16 * (size_t)p + 8, Bf8::from(g + 8).u);
    }
    // warp sums, then block sums in shared memory: 18 atomics per block
    __shared__ float red[8][18];
    for (int o = 16; o > 0; o >>= 1) {
        l += __shfl_down_sync(0xffffffffu, l, o);
        gb += __shfl_down_sync(0xffffffffu, gb, o);
#pragma unroll
        for (int c = 0; c < 16; ++c) gw[c] += __shfl_down_sync(0xffffffffu, gw[c], o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[w][0] = l;
        red[w][1] = gb;
        for (int c = 0; c < 16; ++c) red[w][2 + c] = gw[c];
    }
    __syncthreads();
    if (threadIdx.x < 18) {
        float t = 0.f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k][threadIdx.x];
        atomicAdd(threadIdx.x == 0 ? loss : threadIdx.x == 1 ? dhb : dhw + (threadIdx.x - 2), t);
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

// the bounded wait on an mbarrier that nothing arrives on (arrive = 0) or that one arrival
// completes first (arrive = 1): out[0] = 1 when the wait gave up
__global__ void wait_probe_kernel(int arrive, int limit, unsigned *out)
{
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    if (arrive) mbar_arrive(b);
    out[0] = mbar_wait(b, 0u, limit) ? 0u : 1u;
}

unsigned grid1(long long n)
{
    return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 32));
}

// persistent grid of the direct input layer: the two resident blocks per SM that its
// registers allow, so that each block's weight staging is paid once
inline unsigned grid_in(long long positions) { return std::min(grid1(positions / 4), 152u * 2u); }

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

template <int CIN, int COUT>
cudaError_t launch_tc_t(const bf16 *X, const bf16 *W, const float *bias, Vol v, int relu, bf16 *Y,
                        unsigned *err, cudaStream_t st)
{
    constexpr int cin = CIN;
    if (v.w + 2 > 256 || tc_lines(v.w) > 256) return cudaErrorInvalidValue;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    // activations [n][d][h][w][cin] as a 5-D tensor, innermost first
    CUtensorMap mx, mw;
    const cuuint64_t xdim[5] = {(cuuint64_t)cin, (cuuint64_t)v.w, (cuuint64_t)v.h, (cuuint64_t)v.d, (cuuint64_t)v.n};
    const cuuint64_t xstr[4] = {(cuuint64_t)cin * 2, (cuuint64_t)v.w * cin * 2, (cuuint64_t)v.h * v.w * cin * 2,
                                (cuuint64_t)v.d * v.h * v.w * cin * 2};
    const cuuint32_t xbox[5] = {8, (cuuint32_t)(v.w + 2), (cuuint32_t)tc_lines(v.w), 1, 1};
    const cuuint32_t one[5] = {1, 1, 1, 1, 1};
    if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16 *>(X), xdim, xstr, xbox, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    // weights [27 * cout][cin]
    const cuuint64_t wdim[2] = {(cuuint64_t)cin, (cuuint64_t)27 * COUT};
    const cuuint64_t wstr[1] = {(cuuint64_t)cin * 2};
    const cuuint32_t wbox[2] = {8, (cuuint32_t)COUT};
    if (enc(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(W), wdim, wstr, wbox, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    if constexpr (!tc_wall(CIN, COUT)) {
        // weights too large to keep: the weights-stationary kernel, one CTA per SM (its
        // two units of accumulators take the SM's 512 tensor-memory columns)
        const int wns = ws_stages(CIN, COUT, v.w);
        if (wns < 2) return cudaErrorInvalidValue;
        const int wsmem = ws_smem_bytes(CIN, COUT, v.w, wns);
        cudaError_t we = cudaFuncSetAttribute(conv3d_fwd_ws<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, wsmem);
        if (we != cudaSuccess) return we;
        int wdev = 0, wsms = 0;
        if ((we = cudaGetDevice(&wdev)) != cudaSuccess) return we;
        if ((we = cudaDeviceGetAttribute(&wsms, cudaDevAttrMultiProcessorCount, wdev)) != cudaSuccess) return we;
        const long long wtiles = (long long)v.n * v.d * ((v.h * (v.w + 2) + kTcRows - 1) / kTcRows);
        if (wtiles * 3 >= (1LL << 31)) return cudaErrorInvalidValue;
        const long long wunits = (wtiles + ws_tiles_per_unit(COUT) - 1) / ws_tiles_per_unit(COUT);
        const unsigned wblocks = (unsigned)std::max<long long>(1, std::min<long long>(wunits, wsms));
        conv3d_fwd_ws<CIN, COUT><<<wblocks, kTcThreads, wsmem, st>>>(mx, mw, bias, v, relu, Y, err, wns);
        return cudaGetLastError();
    }
    const cuuint32_t xbox32[5] = {16, (cuuint32_t)(v.w + 2), (cuuint32_t)tc_lines(v.w), 1, 1};
    if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16 *>(X), xdim, xstr, xbox32, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const int ns = tc_stages(cin, COUT, v.w);
    if (ns < 2) return cudaErrorInvalidValue;                   // the volume is too wide
    const int smem = tc_smem_bytes(cin, COUT, v.w, ns);
    cudaError_t e = cudaFuncSetAttribute(conv3d_fwd_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    // resident CTAs per SM: shared memory (1 KiB per CTA reserved by the system), tensor
    // memory (512 columns, NSLOT accumulators per CTA), threads
    int dev = 0, sms = 0, smem_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
        return e;
    const int per_sm = std::max(1, std::min({smem_sm / (smem + 1024), 512 / (tc_nslot(CIN, COUT) * tc_ncol(CIN, COUT)),
                                             2048 / kTcThreads}));
    const long long tiles_plane = (v.h * (v.w + 2) + kTcRows - 1) / kTcRows;
    if ((long long)v.n * v.d * tiles_plane * 3 >= (1LL << 31)) return cudaErrorInvalidValue;
    // column depth: the deepest of 16, 8, 4, 2 that still leaves 3 units per resident CTA
    // (a window then serves up to 3 tiles); on volumes too small for that, min(16, d);
    // 1 without resident weights
    int zc = 1;
    if (tc_wall(CIN, COUT)) {
        zc = std::min(16, v.d);
        for (int z = 16; z >= 2; z /= 2)
            if ((long long)v.n * ((v.d + z - 1) / z) * tiles_plane >= 3LL * sms * per_sm) { zc = z; break; }
    }
    const long long units = (long long)v.n * ((v.d + zc - 1) / zc) * tiles_plane;
    const unsigned blocks = (unsigned)std::max<long long>(1, std::min<long long>(units, (long long)sms * per_sm));
    conv3d_fwd_tc<CIN, COUT><<<blocks, kTcThreads, smem, st>>>(mx, mw, bias, v, relu, Y, err, ns, zc);
    return cudaGetLastError();
}

cudaError_t launch_fwd_tc(const bf16 *X, int cin, const bf16 *W, const float *bias, Vol v, int cout,
                          int relu, bf16 *Y, unsigned *err, cudaStream_t st)
{
    // the (cin, cout) pairs of the network's convolutions and of their input gradients
#define MCX_TC(ci, co) \
    if (cin == ci && cout == co) return launch_tc_t<ci, co>(X, W, bias, v, relu, Y, err, st);
    MCX_TC(16, 16) MCX_TC(16, 32) MCX_TC(16, 48) MCX_TC(32, 16) MCX_TC(32, 32) MCX_TC(32, 64)
    MCX_TC(32, 96) MCX_TC(48, 16) MCX_TC(64, 32) MCX_TC(64, 64) MCX_TC(96, 32)
#undef MCX_TC
    return cudaErrorInvalidValue;
}

template <int CIN, int COUT>
cudaError_t launch_wt_t(const bf16 *X, const bf16 *dY, Vol v, float *dW, unsigned *err, cudaStream_t st)
{
    if (v.w + 2 > 256 || wt_ylines(v.w) > 256) return cudaErrorInvalidValue;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    // 16-channel boxes of whole padded lines (from x = -1), 32-byte swizzle
    CUtensorMap mx, my;
    const cuuint32_t one[5] = {1, 1, 1, 1, 1};
    auto map5 = [&](CUtensorMap *m, const bf16 *ptr, int c, int lines) {
        const cuuint64_t dim[5] = {(cuuint64_t)c, (cuuint64_t)v.w, (cuuint64_t)v.h, (cuuint64_t)v.d, (cuuint64_t)v.n};
        const cuuint64_t str[4] = {(cuuint64_t)c * 2, (cuuint64_t)v.w * c * 2, (cuuint64_t)v.h * v.w * c * 2,
                                   (cuuint64_t)v.d * v.h * v.w * c * 2};
        const cuuint32_t box[5] = {16, (cuuint32_t)(v.w + 2), (cuuint32_t)lines, 1, 1};
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16 *>(ptr), dim, str, box, one,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    if (!map5(&mx, X, CIN, wt_xlines(v.w)) || !map5(&my, dY, COUT, wt_ylines(v.w))) return cudaErrorInvalidValue;
    const int ns = wt_stages(v.w);
    if (ns < 2) return cudaErrorInvalidValue;
    const int smem = wt_smem_bytes(v.w, ns);
    cudaError_t e = cudaFuncSetAttribute(conv3d_wgrad_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, smem_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
        return e;
    // resident CTAs per SM: shared memory (1 KiB per CTA reserved by the system), tensor
    // memory (512 columns), threads
    const int per_sm = std::max(1, std::min({smem_sm / (smem + 1024), 512 / kWtCols, 2048 / kWtThreads}));
    const long long tiles_plane = ((long long)(v.h + 2) * (v.w + 2) + kTcRows - 1) / kTcRows;
    if ((long long)v.n * v.d * tiles_plane * 3 >= (1LL << 31)) return cudaErrorInvalidValue;
    constexpr int pairs = (CIN / 16) * (COUT / 16);
    const long long slots = (long long)sms * per_sm;
    // column depth: the deepest of 16, 8, 4, 2 that leaves 2 units per resident CTA, else 1
    int zc = 1;
    for (int z = 16; z >= 2; z /= 2)
        if ((long long)v.n * ((v.d + z - 1) / z) * tiles_plane * pairs >= 2 * slots) { zc = z; break; }
    zc = std::min(zc, v.d);
    const long long units = (long long)v.n * ((v.d + zc - 1) / zc) * tiles_plane;
    const long long per_pair = std::max<long long>(1, std::min<long long>(units, std::max<long long>(1, slots / pairs)));
    const dim3 grid((unsigned)per_pair, (unsigned)pairs);
    conv3d_wgrad_tc<CIN, COUT><<<grid, kWtThreads, smem, st>>>(mx, my, v, ns, zc, dW, err);
    return cudaGetLastError();
}

// dW (FP32, [27][cout][cin]) += the weight gradient of a convolution with input X and
// output gradient dY; (cin, cout) one of the network's layer pairs
cudaError_t launch_bwd_w(const bf16 *X, int cin, const bf16 *dY, int cout, Vol v, float *dW, unsigned *err,
                         cudaStream_t st)
{
#define MCX_WG(ci, co) \
    if (cin == ci && cout == co) return launch_wt_t<ci, co>(X, dY, v, dW, err, st);
    MCX_WG(16, 16) MCX_WG(16, 32) MCX_WG(32, 32) MCX_WG(32, 64) MCX_WG(64, 64) MCX_WG(96, 32) MCX_WG(48, 16)
#undef MCX_WG
    return cudaErrorInvalidValue;
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
    int D, H, W, maxb, n_aux;
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
static mcx_status forward(mcx_denoiser *d, const float *x, const float *aux, int n, float *out, cudaStream_t st)
{
    const Vol v0 = level_vol(d, 0, n), v1 = level_vol(d, 1, n), v2 = level_vol(d, 2, n);
    const float *P = d->params.as<float>();
    auto conv = [&](int l, const bf16 *in, Vol v) {
        return launch_fwd_tc(in, kLayers[l].cin, d->wf[l].as<bf16>(), P + d->b_off[l], v,
                             kLayers[l].cout, 1, d->a[l].as<bf16>(), d->status.as<unsigned>(), st);
    };
    if (d->n_aux == 0 && (reinterpret_cast<uintptr_t>(x) & 15u) == 0) {
        // one input channel: the direct input layer, which reads the input in 16-byte
        // vectors (the padded copy is made by the backward pass, which needs it for the
        // layer's weight gradient)
        conv_in_fwd<<<grid_in(v0.pos()), kInThreads, 0, st>>>(x, d->wf[0].as<bf16>(), P + d->b_off[0], v0,
                                                          d->a[0].as<bf16>());
        DNC(d, cudaGetLastError(), "conv e1a");
    } else {
        pad_input<<<grid1(v0.pos()), 256, 0, st>>>(x, aux, d->n_aux, d->D * d->H * d->W, (int)v0.pos(),
                                                  d->x16.as<bf16>());
        DNC(d, conv(0, d->x16.as<bf16>(), v0), "conv e1a");
    }
    DNC(d, conv(1, d->a[0].as<bf16>(), v0), "conv e1b");
    avgpool_fwd<<<grid1(v1.pos() * 2), 256, 0, st>>>(d->a[1].as<bf16>(), v1, 16, d->p1.as<bf16>());
    DNC(d, conv(2, d->p1.as<bf16>(), v1), "conv e2a");
    DNC(d, conv(3, d->a[2].as<bf16>(), v1), "conv e2b");
    avgpool_fwd<<<grid1(v2.pos() * 4), 256, 0, st>>>(d->a[3].as<bf16>(), v2, 32, d->p2.as<bf16>());
    DNC(d, conv(4, d->p2.as<bf16>(), v2), "conv ba");
    DNC(d, conv(5, d->a[4].as<bf16>(), v2), "conv bb");
    upcat_fwd<<<grid1(v1.pos() * 12), 256, 0, st>>>(d->a[5].as<bf16>(), 64, d->a[3].as<bf16>(), 32, v1, d->u2.as<bf16>());
    DNC(d, conv(6, d->u2.as<bf16>(), v1), "conv d2a");
    DNC(d, conv(7, d->a[6].as<bf16>(), v1), "conv d2b");
    upcat_fwd<<<grid1(v0.pos() * 6), 256, 0, st>>>(d->a[7].as<bf16>(), 32, d->a[1].as<bf16>(), 16, v0, d->u1.as<bf16>());
    DNC(d, conv(8, d->u1.as<bf16>(), v0), "conv d1a");
    DNC(d, conv(9, d->a[8].as<bf16>(), v0), "conv d1b");
    head_fwd<<<grid1(v0.pos()), 256, 0, st>>>(d->a[9].as<bf16>(), x, P + d->hw_off, P + d->hb_off,
                                             (int)v0.pos(), out);
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
    const int n8 = (int)(v.pos() * L.cout / 8);
    const unsigned rb = std::min(grid1(n8), 152u * 4u);
    const bf16 *A = d->a[l].as<bf16>();
    float *db = G + d->b_off[l];
    switch (L.cout) {
    case 16: relu_bias_grad<16><<<rb, 256, 0, st>>>(dA, A, n8, db); break;
    case 32: relu_bias_grad<32><<<rb, 256, 0, st>>>(dA, A, n8, db); break;
    case 64: relu_bias_grad<64><<<rb, 256, 0, st>>>(dA, A, n8, db); break;
    default: return dn_fail(d, MCX_E_STATE, "no ReLU/bias-gradient kernel for this channel count");
    }
    DNC(d, launch_bwd_w(in, L.cin, dA, L.cout, v, G + d->w_off[l], d->status.as<unsigned>(), st), "weight gradient");
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
    head_bwd<<<std::min(grid1(v0.pos()), 152u * 8u), 256, 0, st>>>(d->a[9].as<bf16>(), d->out.as<float>(), target,
                                             P + d->hw_off, (int)v0.pos(), d->ga[9].as<bf16>(),
                                             G + d->hw_off, G + d->hb_off, d->loss.as<float>());
    mcx_status s;
    if ((s = conv_bwd(d, 9, d->a[8].as<bf16>(), v0, d->ga[8].as<bf16>(), st)) != MCX_OK) return s;
    if ((s = conv_bwd(d, 8, d->u1.as<bf16>(), v0, d->gu1.as<bf16>(), st)) != MCX_OK) return s;
    // upcat 1: coarse part -> d2b output gradient, skip part -> e1b output gradient (later)
    upcat_bwd_coarse<<<grid1(v1.pos() * 4), 256, 0, st>>>(d->gu1.as<bf16>(), 32, 16, v1, d->ga[7].as<bf16>());
    if ((s = conv_bwd(d, 7, d->a[6].as<bf16>(), v1, d->ga[6].as<bf16>(), st)) != MCX_OK) return s;
    if ((s = conv_bwd(d, 6, d->u2.as<bf16>(), v1, d->gu2.as<bf16>(), st)) != MCX_OK) return s;
    upcat_bwd_coarse<<<grid1(v2.pos() * 8), 256, 0, st>>>(d->gu2.as<bf16>(), 64, 32, v2, d->ga[5].as<bf16>());
    if ((s = conv_bwd(d, 5, d->a[4].as<bf16>(), v2, d->ga[4].as<bf16>(), st)) != MCX_OK) return s;
    if ((s = conv_bwd(d, 4, d->p2.as<bf16>(), v2, d->gp2.as<bf16>(), st)) != MCX_OK) return s;
    // e2b output gradient = pool backward + the skip part of upcat 2
    avgpool_bwd<<<grid1(v1.pos() * 4), 256, 0, st>>>(d->gp2.as<bf16>(), v1, 32, d->ga[3].as<bf16>());
    upcat_bwd_skip_add<<<grid1(v1.pos() * 4), 256, 0, st>>>(d->gu2.as<bf16>(), 64, 32, (int)v1.pos(), d->ga[3].as<bf16>());
    if ((s = conv_bwd(d, 3, d->a[2].as<bf16>(), v1, d->ga[2].as<bf16>(), st)) != MCX_OK) return s;
    if ((s = conv_bwd(d, 2, d->p1.as<bf16>(), v1, d->gp1.as<bf16>(), st)) != MCX_OK) return s;
    avgpool_bwd<<<grid1(v0.pos() * 2), 256, 0, st>>>(d->gp1.as<bf16>(), v0, 16, d->ga[1].as<bf16>());
    upcat_bwd_skip_add<<<grid1(v0.pos() * 2), 256, 0, st>>>(d->gu1.as<bf16>(), 32, 16, (int)v0.pos(), d->ga[1].as<bf16>());
    if ((s = conv_bwd(d, 1, d->a[0].as<bf16>(), v0, d->ga[0].as<bf16>(), st)) != MCX_OK) return s;
    if (d->n_aux == 0)                  // the forward pass used the direct input layer
        pad_input<<<grid1(v0.pos()), 256, 0, st>>>(x, nullptr, 0, d->D * d->H * d->W, (int)v0.pos(),
                                                  d->x16.as<bf16>());
    if ((s = conv_bwd(d, 0, d->x16.as<bf16>(), v0, nullptr, st)) != MCX_OK) return s;
    DNC(d, cudaGetLastError(), "backward");
    return MCX_OK;
}

extern "C" {

mcx_status mcx_denoiser_create(mcx_denoiser **out, uint32_t nx, uint32_t ny, uint32_t nz,
                               uint32_t max_batch, uint32_t n_aux, uint64_t seed)
{
    if (!out) return dn_fail(nullptr, MCX_E_ARG, "out is NULL");
    *out = nullptr;
    if (nx % 64 || nx < 64 || nx > 252 || ny % 4 || nz % 4 || ny < 4 || nz < 4 || max_batch < 1)
        return dn_fail(nullptr, MCX_E_ARG,
                       "need nx a multiple of 64 up to 252, ny and nz multiples of 4, max_batch >= 1");
    if (n_aux > 7) return dn_fail(nullptr, MCX_E_ARG, "n_aux must be 0..7");
    if ((unsigned long long)max_batch * nx * ny * nz * 96ull >= (1ull << 31))
        return dn_fail(nullptr, MCX_E_ARG, "max_batch * nx * ny * nz * 96 must stay below 2^31");
    mcx_denoiser *d = new (std::nothrow) mcx_denoiser();
    if (!d) return dn_fail(nullptr, MCX_E_OOM, "host allocation failed");
    d->D = (int)nz; d->H = (int)ny; d->W = (int)nx; d->maxb = (int)max_batch; d->n_aux = (int)n_aux;
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
    // He-normal initial weights (fan-in 27 cin; the input layer's fan-in is 27 (1 + n_aux))
    std::vector<float> init(d->nparam, 0.f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < 10; ++l) {
        const int fan = 27 * (l == 0 ? 1 + d->n_aux : kLayers[l].cin);
        std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / fan));
        for (size_t i = 0; i < 27ull * kLayers[l].cin * kLayers[l].cout; ++i) {
            const int ci = (int)(i % kLayers[l].cin);
            init[d->w_off[l] + i] = (l == 0 && ci > d->n_aux) ? 0.f : (float)nd(rng);
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

mcx_status mcx_denoiser_forward(mcx_denoiser *d, const float *x_dev, const float *aux_dev, float *y_dev,
                                uint32_t n, void *stream)
{
    if (!d || !x_dev || !y_dev || (d->n_aux && !aux_dev)) return dn_fail(d, MCX_E_ARG, "NULL argument");
    if (n < 1 || (int)n > d->maxb) return dn_fail(d, MCX_E_ARG, "n must be 1..max_batch");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mcx_status s = forward(d, x_dev, aux_dev, (int)n, d->out.as<float>(), st);
    if (s != MCX_OK) return s;
    DNC(d, cudaMemcpyAsync(y_dev, d->out.p, (size_t)level_vol(d, 0, n).pos() * 4, cudaMemcpyDeviceToDevice, st),
        "copying the output");
    return MCX_OK;
}

mcx_status mcx_denoiser_train_step(mcx_denoiser *d, const float *x_dev, const float *aux_dev,
                                   const float *t_dev, uint32_t n, float lr, float *loss_host, void *stream)
{
    if (!d || !x_dev || !t_dev || (d->n_aux && !aux_dev)) return dn_fail(d, MCX_E_ARG, "NULL argument");
    if (n < 1 || (int)n > d->maxb) return dn_fail(d, MCX_E_ARG, "n must be 1..max_batch");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mcx_status s = forward(d, x_dev, aux_dev, (int)n, d->out.as<float>(), st);
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

mcx_status mcx_denoiser_apply(mcx_denoiser *d, const float *phi_in_dev, const float *aux_dev,
                              float *phi_out_dev, uint32_t n, void *stream)
{
    if (!d || !phi_in_dev || !phi_out_dev || (d->n_aux && !aux_dev))
        return dn_fail(d, MCX_E_ARG, "NULL argument");
    if (n < 1 || (int)n > d->maxb) return dn_fail(d, MCX_E_ARG, "n must be 1..max_batch");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long cnt = level_vol(d, 0, (int)n).pos();
    encode_kernel<<<grid1(cnt), 256, 0, st>>>(phi_in_dev, cnt, d->floor_, d->mu, 1.f / d->sigma, d->xin.as<float>());
    DNC(d, cudaGetLastError(), "encode");
    mcx_status s = forward(d, d->xin.as<float>(), aux_dev, (int)n, d->out.as<float>(), st);
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

mcx_status mcx_denoiser_features(const uint8_t *labels_dev, uint64_t nvox, uint32_t n_media,
                                 const float *props, float *out_dev, void *stream)
{
    if (!labels_dev || !props || !out_dev || n_media < 1 || n_media > 256 || nvox >= (1ull << 30))
        return dn_fail(nullptr, MCX_E_ARG, "bad arguments");
    float2 tab[256];
    for (uint32_t l = 0; l < n_media; ++l) {
        const float mua = props[4 * l], mus = props[4 * l + 1], g = props[4 * l + 2];
        tab[l] = make_float2(std::log10(std::max(mua, 1e-4f)) + 2.f, std::log10(std::max(mus * (1.f - g), 1e-3f)));
    }
    DBuf dt;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DNC(nullptr, dt.alloc(n_media * sizeof(float2)), "allocating the feature table");
    DNC(nullptr, cudaMemcpyAsync(dt.p, tab, n_media * sizeof(float2), cudaMemcpyHostToDevice, st), "copying the table");
    if (nvox) {
        features_kernel<<<grid1((long long)nvox), 256, 0, st>>>(labels_dev, (int)nvox, dt.as<float2>(), (int)n_media, out_dev);
        DNC(nullptr, cudaGetLastError(), "features");
    }
    DNC(nullptr, cudaStreamSynchronize(st), "waiting for the features");
    return MCX_OK;
}

mcx_status mcx_debug_wait_timeout(int32_t arrive, int32_t limit_log2, int32_t *timed_out)
{
    if (!timed_out || limit_log2 < 0 || limit_log2 > 22) return dn_fail(nullptr, MCX_E_ARG, "bad arguments");
    DBuf o;
    DNC(nullptr, o.alloc(4), "allocating");
    wait_probe_kernel<<<1, 1>>>(arrive ? 1 : 0, 1 << limit_log2, o.as<unsigned>());
    DNC(nullptr, cudaGetLastError(), "launching the wait probe");
    unsigned h = 0;
    DNC(nullptr, cudaMemcpy(&h, o.p, 4, cudaMemcpyDeviceToHost), "reading the wait probe");
    *timed_out = (int32_t)h;
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
    if (kind == 0 && cin == 1) {
        // the direct input layer: FP32 input, weights [27][16][1] placed at ci = 0 of the
        // network's [27][16][16] layout
        if (cout != 16 || P * 96 >= (1LL << 31)) return dn_fail(nullptr, MCX_E_ARG, "bad arguments");
        std::vector<bf16> hw16(27 * 16 * 16, __float2bfloat16(0.f));
        for (int i = 0; i < 27 * 16; ++i) hw16[(size_t)i * 16] = __float2bfloat16(w[i]);
        DBuf bx, bw, bb, by;
        cudaError_t e = bx.alloc(P * 4);
        if (e == cudaSuccess) e = cudaMemcpy(bx.p, x, P * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = bw.alloc(hw16.size() * 2);
        if (e == cudaSuccess) e = cudaMemcpy(bw.p, hw16.data(), hw16.size() * 2, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && bias) e = bb.alloc(16 * 4);
        if (e == cudaSuccess && bias) e = cudaMemcpy(bb.p, bias, 16 * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = by.alloc(P * 16 * 2);
        if (e == cudaSuccess) {
            conv_in_fwd<<<grid_in(P), kInThreads>>>(bx.as<float>(), bw.as<bf16>(), bias ? bb.as<float>() : nullptr, v,
                                                  by.as<bf16>());
            e = cudaGetLastError();
        }
        std::vector<bf16> hy(P * 16);
        if (e == cudaSuccess) e = cudaMemcpy(hy.data(), by.p, hy.size() * 2, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) for (size_t i = 0; i < hy.size(); ++i) out[i] = __bfloat162float(hy[i]);
        if (e != cudaSuccess) return dn_fail(nullptr, MCX_E_CUDA, std::string("debug conv: ") + cudaGetErrorString(e));
        return MCX_OK;
    }
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
        DBuf berr;
        if (e == cudaSuccess) e = berr.alloc(4);
        if (e == cudaSuccess) e = cudaMemset(berr.p, 0, 4);
        if (e == cudaSuccess)
            e = launch_bwd_w(bx.as<bf16>(), cin, bdy.as<bf16>(), cout, v, bdw.as<float>(), berr.as<unsigned>(), nullptr);
        unsigned herr = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&herr, berr.p, 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && herr) return dn_fail(nullptr, MCX_E_TIMEOUT, "weight-gradient wait timed out");
        if (e == cudaSuccess) e = cudaMemcpy(out, bdw.p, 27ull * cin * cout * 4, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return dn_fail(nullptr, MCX_E_CUDA, std::string("debug conv: ") + cudaGetErrorString(e));
    return MCX_OK;
}

}  // extern "C"
