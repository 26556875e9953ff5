// Persistent photon-per-thread Monte Carlo walk through a labelled voxel volume (sm_103a).
//
// What one thread does per photon follows the photon simulation loop of the paper's
// workflow (Fig. 1 paragraph) with the physics of its benchmark description (beside
// Fig. 2): exponential hops in mean free paths, stepping voxel face to voxel face, Snell /
// Fresnel at refractive-index mismatches (or termination at the exterior), Henyey-
// Greenstein scattering with the MCML rotation, Russian roulette, race-free (atomic)
// accumulation of absorbed weight into time gates, and disk detectors that record partial
// path lengths.
//
// GB300-specific design (differs from the paper's OpenCL kernel):
//  * Persistent grid (SMs x resident blocks).  A warp claims 32 photon ids with one global
//    atomic and hands them to lanes as their photons finish, the per-warp analogue of the
//    paper's in-workgroup dynamic load balancing (Fig. 3a paragraph) without a per-photon
//    atomic.
//  * Every photon's random stream derives from (seed, photon id), so a run is a pure
//    function of (seed, id range) whatever the launch shape.
//  * Position = integer voxel index + fraction inside the voxel: face distances are
//    computed against 0 and 1, which keeps FP32 geometry at full precision anywhere in
//    a large grid.
//  * Absorbed weight is accumulated in a register while the photon stays in one
//    (gate, voxel) and flushed with one fire-and-forget global atomic when it leaves,
//    instead of one atomic per segment: FP64 by default (the FP32 run total widened
//    exactly in integer arithmetic), FP32 or compensated (hi, lo) pairs on request.
//  * The current medium's constants (scattering, absorption, time per length, g) sit in
//    registers and are reloaded only when the photon enters another label; a photon's
//    absorbed weight is formed once, from its final weight and roulette gains.
//  * Fast hardware math (MUFU ex2/lg2/sin/cos/rsqrt/rcp) in the FP32 path, the CUDA
//    analogue of the paper's "native" math optimisation; the same kernel instantiated in
//    FP64 serves as the trajectory-parity diagnostic.
#include <cfloat>
#include <cstdint>

#include "mcx_internal.h"

namespace mcxg {
namespace {

constexpr unsigned kFull = 0xffffffffu;
enum { EV_FACE = 0, EV_SCAT = 1, EV_TIME = 2 };

// ------------------------------------------------------------------------------ math
template <typename R> struct M;
// The FP32 walk keeps hop lengths in units of ln 2 mean free paths and its absorption
// coefficients multiplied by log2(e) (the per-label tables are scaled to match), so a hop
// is one lg2 and an attenuation one ex2 on the special-function unit; the FP64 walk uses
// natural units and the library log/exp.
template <> struct M<float> {
    static __device__ __forceinline__ float log(float x) { return __logf(x); }
    static __device__ __forceinline__ float hop(float u)
    {
        float y;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(u));
        return -y;
    }
    static __device__ __forceinline__ float attenuation(float a, float l)
    {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-a * l));
        return y;
    }
    static constexpr double kHopUnit = 0.69314718055994530942;     // ln 2
    static constexpr double kAbsScale = 1.44269504088896340736;    // log2(e)
    static __device__ __forceinline__ void sincos_2pi(float x, float *s, float *c)
    { __sincosf(6.28318530717958647692f * x, s, c); }
    static __device__ __forceinline__ float sqrt(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
    static __device__ __forceinline__ float huge() { return FLT_MAX; }
    static __device__ __forceinline__ float tiny_hop() { return 1e-12f; }
};
template <> struct M<double> {
    static __device__ __forceinline__ double log(double x) { return ::log(x); }
    static __device__ __forceinline__ double hop(double u) { return -::log(u); }
    static __device__ __forceinline__ double attenuation(double a, double l) { return ::exp(-a * l); }
    static constexpr double kHopUnit = 1.0;
    static constexpr double kAbsScale = 1.0;
    static __device__ __forceinline__ void sincos_2pi(double x, double *s, double *c)
    { ::sincospi(2.0 * x, s, c); }
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double rsqrt(double x) { return 1.0 / ::sqrt(x); }
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
    static __device__ __forceinline__ double huge() { return DBL_MAX; }
    static __device__ __forceinline__ double tiny_hop() { return 1e-300; }
};

// Per-label tables in the walk's precision (FP32: mus and mua in the scaled units above).
template <typename R> struct MedA { R mus, inv_mus, mua, len_per_t; };
template <typename R> struct MedB { R one_m_g, one_p_g, one_m_g2, two_g; };

// ------------------------------------------------------------------------------ RNG
// SplitMix64 output k of `seed` (Steele, Lea & Flood 2014): state seed + k * golden gamma,
// then the 64-bit finaliser.  Photon p's xorshift128+ state = outputs 2p+1 and 2p+2.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct Rng {
    uint64_t x, y;
    __device__ __forceinline__ void seed(uint64_t s, uint64_t photon)
    {
        x = splitmix64(s, 2 * photon + 1);
        y = splitmix64(s, 2 * photon + 2);
        if ((x | y) == 0) y = 1;
    }
    // xorshift128+ (Vigna), shift triple 23/18/5; one uniform (hop, Fresnel, roulette) is
    // (2k+1) 2^-24 from the top 23 bits k of one output, exactly representable in float.
    __device__ __forceinline__ float uniform()
    {
        const uint64_t r = next();
        return from_bits((unsigned)(r >> 41));
    }
    // Two uniforms from one output (Gaussian launch point): the top 23 bits and bits
    // 40..18.
    __device__ __forceinline__ void pair(float &u1, float &u2)
    {
        const uint64_t r = next();
        u1 = from_bits((unsigned)(r >> 41));
        u2 = from_bits((unsigned)(r >> 18) & 0x7fffffu);
    }
    // Three uniforms from one output (a scattering event: next hop, deflection, azimuth):
    // bits 63..43, 42..22 and 21..1, each (2k+1) 2^-22, exactly representable in float.
    // Bit 0 of the generator's sum is linear over GF(2) and unused; bit 1 is quadratic.
    // The hop's logarithm makes its rare long hops depend on the low-order bits of its
    // uniform, so the hop takes the top field and the azimuth (linear in its uniform) the
    // bottom one.
    __device__ __forceinline__ void triple(float &u1, float &u2, float &u3)
    {
        const uint64_t r = next();
        u1 = from21((unsigned)(r >> 43));
        u2 = from21((unsigned)(r >> 22) & 0x1fffffu);
        u3 = from21((unsigned)(r >> 1) & 0x1fffffu);
    }
    __device__ __forceinline__ uint64_t next()
    {
        uint64_t a = x;
        const uint64_t b = y;
        const uint64_t r = a + b;
        x = b;
        a ^= a << 23;
        y = a ^ b ^ (a >> 18) ^ (b >> 5);
        return r;
    }
    // (1 + k 2^-23) - (1 - 2^-24) = (2k + 1) 2^-24, both steps exact
    static __device__ __forceinline__ float from_bits(unsigned k)
    {
        return __uint_as_float(0x3f800000u | k) - 0.99999994039535522461f;
    }
    // (1 + k 2^-21) - (1 - 2^-22) = (2k + 1) 2^-22 for a 21-bit k, both steps exact
    static __device__ __forceinline__ float from21(unsigned k)
    {
        return __uint_as_float(0x3f800000u | (k << 2)) - 0.9999997615814208984375f;
    }
};

// ------------------------------------------------------------------------------ physics
// Henyey-Greenstein deflection by inverse CDF.  With D = 1 - g + 2 g xi and
// f = (1 - g^2) / D, the textbook cosine is (1 + g^2 - f^2) / (2 g).  The same quantity is
// produced here as the pair
//     1 - cos = (1 - g)(1 - xi)(f + 1 - g) / D,    1 + cos = (1 + g) xi (1 + g + f) / D,
// which follow from it by factoring f^2 - (1-g)^2 and (1+g)^2 - f^2; both are free of
// cancellation, so sin^2 = (1 - cos)(1 + cos) keeps full FP32 precision for the small
// deflections that dominate at g ~ 0.9 (1 - cos^2 would lose most of its bits there).
// g = 0 reduces to the isotropic cos = 2 xi - 1 without a special case.
template <typename R>
__device__ __forceinline__ void hg_sample(const MedB<R> &B, R xi, R &ct, R &st)
{
    const R inv_d = R(1) / (B.one_m_g + B.two_g * xi);
    const R f = B.one_m_g2 * inv_d;
    const R omc = B.one_m_g * (R(1) - xi) * (f + B.one_m_g) * inv_d;
    const R opc = B.one_p_g * xi * (B.one_p_g + f) * inv_d;
    ct = R(0.5) * (opc - omc);
    st = M<R>::sqrt(omc * opc);
}

// The Henyey-Greenstein constants of anisotropy g; the host's table rounds them alike
// (1 - g^2 as one fused multiply-add), so a walk that derives them from a g kept in a
// register follows the same trajectories as one that reads the table.
template <typename R>
__host__ __device__ __forceinline__ MedB<R> hg_consts(R g)
{
    return MedB<R>{R(1) - g, R(1) + g, fma(-g, g, R(1)), g + g};
}

// MCML rotation of unit vector u by deflection (cos ct, sin st) and azimuth (sp, cp).
template <typename R>
__device__ __forceinline__ void rotate(R &ux, R &uy, R &uz, R ct, R st, R sp, R cp)
{
    if (fabs(uz) > R(1) - R(1e-5)) {
        ux = st * cp;
        uy = st * sp;
        uz = uz > R(0) ? ct : -ct;
    } else {
        // 1 - uz^2 evaluated as ux^2 + uy^2: no cancellation near the poles in FP32
        const R one_m_uz2 = ux * ux + uy * uy;
        const R rt = M<R>::rsqrt(one_m_uz2);          // 1 / sqrt(1 - uz^2)
        const R a = st * rt;
        const R nx = a * (ux * uz * cp - uy * sp) + ux * ct;
        const R ny = a * (uy * uz * cp + ux * sp) + uy * ct;
        const R nz = -st * cp * (one_m_uz2 * rt) + uz * ct;
        ux = nx;
        uy = ny;
        uz = nz;
    }
}

// Unpolarised Fresnel reflectance n1 -> n2 at incidence cosine ci, given sin^2 of the
// transmission angle st2 < 1 (the caller handles total internal reflection).
template <typename R>
__device__ __forceinline__ R fresnel(R n1, R n2, R ci, R st2)
{
    const R ct = M<R>::sqrt(R(1) - st2);
    const R rs = M<R>::div(n1 * ci - n2 * ct, n1 * ci + n2 * ct);
    const R rp = M<R>::div(n1 * ct - n2 * ci, n1 * ct + n2 * ci);
    return R(0.5) * (rs * rs + rp * rp);
}

// Signed reciprocal of a direction component (+-inf for +-0).  With it the distance to the
// face ahead along that axis is one FMA on the in-voxel fraction q:
//   u > 0: (1 - q) / u = fma(q, -inv, inv);   u < 0: -q / u = fma(q, -inv, 0)
// i.e. fma(q, -inv, max(inv, 0)).  A zero component gives NaN or +inf there, which the
// walk's fmin-based minimum never picks (measured 4% faster than testing u for zero).
// A fraction that rounding pushed past its face gives a negative distance; the walk clamps
// the nearest one to 0 (a zero-length step onto that face) after taking the minimum.
template <typename R>
__device__ __forceinline__ R inv_dir(R u)
{
    return R(1) / u;                   // +-inf for +-0: its face distance is NaN or +inf
}

template <typename R>
__device__ __forceinline__ R face_dist(R q, R inv)
{
    return fma(q, -inv, inv > R(0) ? inv : R(0));
}

// ------------------------------------------------------------------------------ kernel
// Dynamic shared memory, sized by the run's media and detector counts:
//   double tally[8] | u64 stats[8] | MedA<R>[n_media] | MedB<R>[n_media] | R n[n_media] |
//   R tpl[n_media] | float4 det[n_det]
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename R>
struct SmemLayout {
    size_t a, b, n, tpl, det, tile, total;
    __host__ __device__ SmemLayout(int n_media, int n_det, int tile_entries)
    {
        a = 128;
        b = align16(a + sizeof(MedA<R>) * n_media);
        n = align16(b + sizeof(MedB<R>) * n_media);
        tpl = align16(n + sizeof(R) * n_media);
        det = align16(tpl + sizeof(R) * n_media);
        tile = align16(det + sizeof(float4) * n_det);        // float hi[E], then float lo[E]
        total = align16(tile + 2 * sizeof(float) * tile_entries);
    }
};

// Adds x to the compensated pair (hi, lo): the atomic returns hi's old value a; the
// hardware stored s = RN(a + x), so the addition's exact rounding error (Knuth's TwoSum)
// is recovered locally and accumulated into lo.  hi + lo then carries the sum without
// the per-addition loss of a single FP32 accumulator.
__device__ __forceinline__ void pair_add(float *hi, float *lo, float x)
{
    const float a = atomicAdd(hi, x);
    const float s = __fadd_rn(a, x);
    const float bb = __fsub_rn(s, a);
    const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    if (err != 0.f) atomicAdd(lo, err);
}

template <typename R> __device__ __forceinline__ const RunConsts<R> &consts(const WalkParams &p);
template <> __device__ __forceinline__ const RunConsts<float> &consts<float>(const WalkParams &p)
{ return p.cf; }
template <> __device__ __forceinline__ const RunConsts<double> &consts<double>(const WalkParams &p)
{ return p.cd; }

// PAD: the label volume and the accumulation maps carry a one-voxel exterior border, so
// the neighbour of any tissue voxel is inside the arrays: the face step reads its label
// without per-axis bounds checks, and the per-axis voxel indices need not be carried
// (they are recovered from the linear index when a photon ends).  Caller-owned unpadded
// buffers (the allocation-free run) take PAD = false.
// FP32: 4 resident blocks of 256 threads per SM (64 registers; the batch instantiation too,
// with a few spilled words for its per-lane simulation geometry)
template <typename R, bool DET, int ACC, bool STATIC, bool BATCH, bool PAD>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 1)
walk_kernel(const WalkParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tile_e = ACC == kAccCompensated
        ? p.tile_size[0] * p.tile_size[1] * p.tile_size[2] * p.tile_size[3] : 0;
    const SmemLayout<R> L(p.n_media, DET ? p.n_det : 0, tile_e);
    float *s_hi = reinterpret_cast<float *>(smem_raw + L.tile);
    float *s_lo = s_hi + tile_e;
    double *s_tally = reinterpret_cast<double *>(smem_raw);
    unsigned long long *s_stats = reinterpret_cast<unsigned long long *>(smem_raw + 64);
    MedA<R> *s_a = reinterpret_cast<MedA<R> *>(smem_raw + L.a);
    MedB<R> *s_b = reinterpret_cast<MedB<R> *>(smem_raw + L.b);
    R *s_n = reinterpret_cast<R *>(smem_raw + L.n);
    R *s_tpl = reinterpret_cast<R *>(smem_raw + L.tpl);
    float4 *s_det = reinterpret_cast<float4 *>(smem_raw + L.det);

    for (int i = threadIdx.x; i < (BATCH ? 0 : p.n_media); i += blockDim.x) {
        s_a[i] = static_cast<const MedA<R> *>(p.tab_a)[i];
        s_b[i] = static_cast<const MedB<R> *>(p.tab_b)[i];
        s_n[i] = static_cast<const R *>(p.tab_n)[i];
        s_tpl[i] = static_cast<const R *>(p.tab_tpl)[i];
    }
    if (DET)
        for (int i = threadIdx.x; i < p.n_det; i += blockDim.x) s_det[i] = p.det[i];
    if (threadIdx.x < 8) s_tally[threadIdx.x] = 0.0;
    if (threadIdx.x < 8) s_stats[threadIdx.x] = 0ull;
    if (ACC == kAccCompensated)
        for (int i = threadIdx.x; i < 2 * tile_e; i += blockDim.x) s_hi[i] = 0.f;
    __syncthreads();

    // per-run constants in the walk's precision (read from the parameter bank)
    const RunConsts<R> &C = consts<R>(p);

    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;

    // Geometry of the photon's simulation: the kernel parameters, or (batch) the lane's
    // current simulation, loaded at each launch.
    const uint8_t *G_labels = p.labels;
    float *G_flu = p.fluence;
    double *G_flu64 = p.fluence64;
    int G_nx = p.nx, G_ny = p.ny, G_nz = p.nz;
    unsigned G_nvox = p.nvox;
    unsigned G_sy = p.sy, G_sz = p.sz;     // linear strides of y and z (padded when PAD)
    int tab0 = 0, sim = 0;
    // per-label tables: shared memory, or (batch) the batch tables through L1
    auto medA = [&](int l) -> MedA<R> {
        if constexpr (BATCH) {
            const float4 v = __ldg(static_cast<const float4 *>(p.tab_a) + tab0 + l);
            return MedA<R>{v.x, v.y, v.z, v.w};
        } else {
            return s_a[l];
        }
    };
    auto medB = [&](int l) -> MedB<R> {
        if constexpr (BATCH) {
            const float4 v = __ldg(static_cast<const float4 *>(p.tab_b) + tab0 + l);
            return MedB<R>{v.x, v.y, v.z, v.w};
        } else {
            return s_b[l];
        }
    };
    auto med_n = [&](int l) -> R {
        if constexpr (BATCH) return __ldg(static_cast<const float *>(p.tab_n) + tab0 + l);
        else return s_n[l];
    };
    auto med_tpl = [&](int l) -> R {
        if constexpr (BATCH) return __ldg(static_cast<const float *>(p.tab_tpl) + tab0 + l);
        else return s_tpl[l];
    };
    const unsigned max_ev = p.max_events < 0xffffffffull ? (unsigned)p.max_events : 0xffffffffu;

    bool alive = false, done = false;
    unsigned long long pid = ~0ull;   // current (or last) photon id; none yet
    Rng rng;
    rng.x = rng.y = 0;
    int ix = 0, iy = 0, iz = 0, lab = 0;
    unsigned vlin = 0;
    R qx = 0, qy = 0, qz = 0, ux = 0, uy = 0, uz = 1, iux = 0, iuy = 0, iuz = 0;
    // gained: the photon's roulette gains; its absorbed weight is 1 + gained - (its final
    // weight), since absorption and roulette are the only changes of w
    R w = 0, t = 0, s = 0, gained = 0, Lcur = 0, acc = 0;
    unsigned gate = 0;            // time gate of the current deposit run
    R t_next = 0;                 // time at which the gate advances
    // the current medium's segment constants, reloaded only when the label changes (kept in
    // registers: measured 5% faster at C2 than a shared-memory lookup in every segment); the
    // compensated mode, whose block tile needs those registers, looks them up per segment
    constexpr bool KEEP_MED = ACC != kAccCompensated;
    MedA<R> A_cur{};
    R tpl_cur = 0;                // its time per unit length
    R g_cur = 0;                  // its anisotropy (the scattering constants follow from it)
    unsigned nscat = 0, nrr = 0, c_face = 0, c_fres = 0, c_flush = 0, c_rr = 0;
    float Lpath[DET ? kMaxDetMedia : 1];

    unsigned long long pool_next = 0;
    unsigned pool_left = 0;
    const unsigned last_gate = p.n_gates - 1u;

    // a6/a12: one accumulation per (gate, voxel) run of deposits
    auto flush = [&]() {
        if (acc != R(0)) {
            const unsigned long long idx = (unsigned long long)gate * G_nvox + vlin;
            // one fire-and-forget FP64 add into the map; for FP32 the (positive, normal: the
            // walk flushes denormals) run total is widened exactly in integer arithmetic:
            // exponent rebiased by 1023 - 127 = 896, mantissa shifted by 29 (measured 0.9%
            // faster than the conversion instruction, which runs on the narrow FP64 pipe)
            auto add_f64 = [&]() {
                if (sizeof(R) == 4) {
                    const unsigned f = __float_as_uint(float(acc));
                    const double dv = __hiloint2double((int)((f >> 3) + (896u << 20)), (int)(f << 29));
                    atomicAdd(G_flu64 + idx, dv);
                } else {
                    atomicAdd(G_flu64 + idx, double(acc));
                }
            };
            if (ACC == kAccPlain) {
                atomicAdd(G_flu + idx, float(acc));
            } else if (ACC == kAccF64) {
                add_f64();
            } else {
                // compensated: runs inside the block tile go to its shared-memory (hi, lo)
                // pair, the rest to the FP64 map
                const unsigned tx = (unsigned)(ix - p.tile_lo[0]), ty = (unsigned)(iy - p.tile_lo[1]);
                const unsigned tz = (unsigned)(iz - p.tile_lo[2]), tg = gate - (unsigned)p.tile_lo[3];
                if (tx < (unsigned)p.tile_size[0] && ty < (unsigned)p.tile_size[1] &&
                    tz < (unsigned)p.tile_size[2] && tg < (unsigned)p.tile_size[3]) {
                    const unsigned k = ((tg * p.tile_size[2] + tz) * p.tile_size[1] + ty) *
                                       p.tile_size[0] + tx;
                    pair_add(s_hi + k, s_lo + k, float(acc));
                } else {
                    add_f64();
                }
            }
            ++c_flush;
        }
        acc = R(0);
    };
    // a4: dimensionless hop in mean free paths
    auto new_hop = [&]() {
        const R h = M<R>::hop(R(rng.uniform()));
        s = h > M<R>::tiny_hop() ? h : M<R>::tiny_hop();
    };

    while (true) {
        if (__any_sync(kFull, !alive)) {
            // ---- a1: claim photon ids for lanes without a photon (one atomic per 32 ids)
            const unsigned need = __ballot_sync(kFull, !alive && !done);
            if (need) {
                const unsigned n = __popc(need);
                const unsigned rank = __popc(need & lt_mask);
                unsigned long long id;
                if (STATIC) {
                    // the paper's thread-level split: thread g of T takes g, g + T, g + 2T,
                    // ...; the next id follows from the lane's previous one
                    const unsigned long long g0 = blockIdx.x * blockDim.x + threadIdx.x;
                    id = pid == ~0ull ? g0 : pid - p.photon_offset + gridDim.x * blockDim.x;
                } else if (pool_left >= n) {
                    id = pool_next + rank;
                    pool_next += n;
                    pool_left -= n;
                } else {
                    unsigned long long nb = 0;
                    if (lane == 0) nb = atomicAdd(p.photon_counter, (unsigned long long)p.claim_chunk);
                    nb = __shfl_sync(kFull, nb, 0);
                    id = rank < pool_left ? pool_next + rank : nb + (rank - pool_left);
                    const unsigned used_new = n - pool_left;
                    pool_next = nb + used_new;
                    pool_left = p.claim_chunk - used_new;
                }
                if ((need >> lane) & 1u) {
                    if (id >= p.n_photons) {
                        done = true;
                    } else {
                        // ---- a2/a3: per-photon RNG and launch
                        R px, py, pz, e1[3], e2[3], waist;
                        int kind;
                        if constexpr (BATCH) {
                            // the simulation holding flattened index id: the last with first <= id
                            int lo = 0, hi = p.n_sims - 1;
                            while (lo < hi) {
                                const int mid = (lo + hi + 1) >> 1;
                                if (p.sims[mid].first <= id) lo = mid; else hi = mid - 1;
                            }
                            sim = lo;
                            const BatchSim &S = p.sims[sim];
                            pid = id - S.first;
                            rng.seed(S.seed, pid);
                            G_labels = S.labels; G_flu = S.fluence; G_flu64 = S.fluence64;
                            G_nx = S.nx; G_ny = S.ny; G_nz = S.nz; G_nvox = S.nvox;
                            G_sy = S.sy; G_sz = S.sz;
                            tab0 = S.tab0;
                            px = S.src_pos[0]; py = S.src_pos[1]; pz = S.src_pos[2];
                            ux = S.src_dir[0]; uy = S.src_dir[1]; uz = S.src_dir[2];
                            for (int a = 0; a < 3; ++a) { e1[a] = S.src_e1[a]; e2[a] = S.src_e2[a]; }
                            waist = S.waist;
                            kind = S.src_kind;
                        } else {
                            pid = p.photon_offset + id;
                            rng.seed(p.seed, pid);
                            px = C.src_pos[0]; py = C.src_pos[1]; pz = C.src_pos[2];
                            ux = C.src_dir[0]; uy = C.src_dir[1]; uz = C.src_dir[2];
                            for (int a = 0; a < 3; ++a) { e1[a] = C.src_e1[a]; e2[a] = C.src_e2[a]; }
                            waist = C.waist;
                            kind = p.src_kind;
                        }
                        if (kind == 1) {
                            float f1, f2;
                            rng.pair(f1, f2);
                            const R r = waist * M<R>::sqrt(-M<R>::log(R(f1)) * R(0.5));
                            R sn, cs;
                            M<R>::sincos_2pi(R(f2), &sn, &cs);
                            px += r * (cs * e1[0] + sn * e2[0]);
                            py += r * (cs * e1[1] + sn * e2[1]);
                            pz += r * (cs * e1[2] + sn * e2[2]);
                        }
                        const R fx = floor(px), fy = floor(py), fz = floor(pz);
                        ix = (int)fx - ((px == fx && ux < R(0)) ? 1 : 0);
                        iy = (int)fy - ((py == fy && uy < R(0)) ? 1 : 0);
                        iz = (int)fz - ((pz == fz && uz < R(0)) ? 1 : 0);
                        qx = px - R(ix); qy = py - R(iy); qz = pz - R(iz);
                        iux = inv_dir(ux); iuy = inv_dir(uy); iuz = inv_dir(uz);
                        w = R(1); t = R(0); gained = R(0); Lcur = R(0); acc = R(0);
                        gate = 0;
                        t_next = last_gate > 0 ? C.dt : M<R>::huge();
                        nscat = nrr = c_face = c_fres = c_flush = c_rr = 0;
                        if (DET)
                            for (int m = 0; m < p.n_media && m < kMaxDetMedia; ++m) Lpath[m] = 0.f;
                        const bool inside = (unsigned)ix < (unsigned)G_nx &&
                                            (unsigned)iy < (unsigned)G_ny &&
                                            (unsigned)iz < (unsigned)G_nz;
                        vlin = inside ? ((unsigned)iz * G_sz + (unsigned)iy * G_sy + (unsigned)ix +
                                         (PAD ? G_sz + G_sy + 1u : 0u)) : 0u;
                        lab = inside ? (int)__ldg(G_labels + vlin) : 0;
                        if constexpr (KEEP_MED) {
                            A_cur = medA(lab);
                            tpl_cur = med_tpl(lab);
                            g_cur = R(0.5) * medB(lab).two_g;      // 2g / 2: exact
                        }
                        alive = lab != 0;
                        if (alive) {
                            new_hop();
                        } else {
                            // launched outside the medium: counted as escaped, never enters
                            if constexpr (BATCH) atomicAdd(p.sims[sim].tally + MCX_TALLY_ESCAPED, 1.0);
                            else atomicAdd(&s_tally[MCX_TALLY_ESCAPED], 1.0);
                            atomicAdd(&s_stats[MCX_STAT_PHOTONS], 1ull);
                            const unsigned long long rel = pid - p.photon_offset;
                            if (rel < p.exit_log) {
                                mcx_exit e;
                                e.fate = MCX_FATE_MISSED; e.nscat = 0;
                                e.pos[0] = float(px * R(p.h)); e.pos[1] = float(py * R(p.h));
                                e.pos[2] = float(pz * R(p.h));
                                e.dir[0] = float(ux); e.dir[1] = float(uy); e.dir[2] = float(uz);
                                e.w = 1.f; e.t = 0.f;
                                p.exits[rel] = e;
                            }
                        }
                    }
                }
            }
            if (__all_sync(kFull, done)) break;
            if (!alive) continue;
        }

        int fate = MCX_FATE_NONE;
        if (nscat + c_face >= max_ev) {
            fate = MCX_FATE_CAPPED;
        } else {
            // ---- a7: the gate of this segment's start (time only increases)
            if (t >= t_next) {
                flush();
                unsigned g2 = (unsigned)(t * C.inv_dt);
                g2 = g2 > gate + 1u ? g2 : gate + 1u;
                gate = g2 < last_gate ? g2 : last_gate;
                t_next = gate < last_gate ? R(gate + 1u) * C.dt : M<R>::huge();
            }
            const MedA<R> A = KEEP_MED ? A_cur : medA(lab);
            const R tpl = KEEP_MED ? tpl_cur : med_tpl(lab);
            // ---- a5: nearest face (lowest axis on ties), scattering point, time limit
            const R dxf = face_dist(qx, iux);
            const R dyf = face_dist(qy, iuy);
            const R dzf = face_dist(qz, iuz);
            // fmin ignores the NaN distance of a zero direction component
            const R lmin = fmin(fmin(dxf, dyf), dzf);
            const int ax = lmin == dxf ? 0 : (lmin == dyf ? 1 : 2);     // lowest axis on ties
            R l = lmin > R(0) ? lmin : R(0);  // rounding past a face: a zero-length step onto it
            int ev = EV_FACE;
            const R dscat = s * A.inv_mus;
            if (dscat <= l) { l = dscat; ev = EV_SCAT; }
            R dtime = (C.t_end - t) * A.len_per_t;
            dtime = dtime > R(0) ? dtime : R(0);
            if (dtime <= l) { l = dtime; ev = EV_TIME; }

            // ---- a5/a6: move, age, absorb into the current (gate, voxel) run
            qx += l * ux;
            qy += l * uy;
            qz += l * uz;
            t += l * tpl;
            s -= l * A.mus;                   // a scattering event draws the next hop
            if (DET) Lcur += l;
            const R wn = w * M<R>::attenuation(A.mua, l);
            const R dw = w - wn;
            w = wn;
            acc += dw;

            if (ev == EV_TIME) {
                fate = MCX_FATE_TIME;
            } else if (ev == EV_FACE) {
                // ---- a8: voxel face
                ++c_face;
                const bool p0 = ax == 0, p1 = ax == 1;
                const R inv_a = p0 ? iux : (p1 ? iuy : iuz);
                const bool up = inv_a > R(0);              // u_ax >= 0 (inv_dir of 0 is +huge)
                const unsigned stride = p0 ? 1u : (p1 ? G_sy : G_sz);
                const unsigned nlin = up ? vlin + stride : vlin - stride;
                // per-axis index of the next voxel: tracked unless the border makes it
                // unnecessary (the compensated mode's block tile still needs it)
                constexpr bool AXES = !PAD || ACC == kAccCompensated;
                int ia = 0;
                if constexpr (AXES) ia = (p0 ? ix : (p1 ? iy : iz)) + (up ? 1 : -1);
                int b;
                if constexpr (PAD) {
                    b = (int)__ldg(G_labels + nlin);
                } else {
                    const int dim = p0 ? G_nx : (p1 ? G_ny : G_nz);
                    b = (unsigned)ia < (unsigned)dim ? (int)__ldg(G_labels + nlin) : 0;
                }
                if (b == lab) {
                    // same medium: straight into the next voxel, entering on the near face
                    flush();                              // the deposit run ends with the voxel
                    const R qn = up ? R(0) : R(1);
                    qx = p0 ? qn : qx;
                    qy = p1 ? qn : qy;
                    qz = (!p0 && !p1) ? qn : qz;
                    if constexpr (AXES) {
                        ix = p0 ? ia : ix;
                        iy = p1 ? ia : iy;
                        iz = (!p0 && !p1) ? ia : iz;
                    }
                    vlin = nlin;
                    if (s <= R(0)) new_hop();            // hop used up by rounding at the face
                } else {
                    // photon on the face
                    const R qb = up ? R(1) : R(0);
                    qx = p0 ? qb : qx;
                    qy = p1 ? qb : qy;
                    qz = !p0 && !p1 ? qb : qz;
                    const R ua = p0 ? ux : (p1 ? uy : uz);
                    bool enter = false, escape = false;
                    if (!p.reflect) {
                        // the paper's B1: the exterior terminates, internal mismatches pass
                        if (b == 0) escape = true; else enter = true;
                    } else {
                        const R na = med_n(lab), nb = med_n(b);
                        if (na == nb) {
                            if (b == 0) escape = true; else enter = true;
                        } else {
                            ++c_fres;
                            const R ci = fabs(ua);
                            const R eta = M<R>::div(na, nb);
                            const R st2 = eta * eta * fma(-ci, ci, R(1));   // one rounding
                            bool refl = true;                 // total internal reflection
                            if (st2 < R(1)) refl = R(rng.uniform()) < fresnel(na, nb, ci, st2);
                            if (refl) {
                                ux = p0 ? -ux : ux;
                                uy = p1 ? -uy : uy;
                                uz = !p0 && !p1 ? -uz : uz;
                                iux = p0 ? -iux : iux;
                                iuy = p1 ? -iuy : iuy;
                                iuz = !p0 && !p1 ? -iuz : iuz;
                            } else {
                                // Snell: tangential components x eta, normal = +-cos(theta_t)
                                const R ctt = M<R>::sqrt(R(1) - st2);
                                const R un = up ? ctt : -ctt;
                                ux = p0 ? un : ux * eta;
                                uy = p1 ? un : uy * eta;
                                uz = !p0 && !p1 ? un : uz * eta;
                                iux = inv_dir(ux); iuy = inv_dir(uy); iuz = inv_dir(uz);
                                if (b == 0) escape = true; else enter = true;
                            }
                        }
                    }
                    if (enter) {
                        flush();
                        if constexpr (AXES) {
                            ix = p0 ? ia : ix;
                            iy = p1 ? ia : iy;
                            iz = !p0 && !p1 ? ia : iz;
                        }
                        qx = p0 ? R(1) - qb : qx;
                        qy = p1 ? R(1) - qb : qy;
                        qz = !p0 && !p1 ? R(1) - qb : qz;
                        vlin = nlin;
                        if (DET) {
                            if (lab < kMaxDetMedia) Lpath[lab] += float(Lcur);
                            Lcur = R(0);
                        }
                        lab = b;
                        if constexpr (KEEP_MED) {
                            A_cur = medA(b);
                            tpl_cur = med_tpl(b);
                            g_cur = R(0.5) * medB(b).two_g;
                        }
                    }
                    if (escape) fate = MCX_FATE_ESCAPED;
                    else if (s <= R(0)) new_hop();        // hop used up by rounding at the face
                }
            } else {
                // ---- a10: Henyey-Greenstein scattering; a11: Russian roulette
                ++nscat;
                const MedB<R> B = KEEP_MED ? hg_consts(g_cur) : medB(lab);
                float u_hop, xi_hg, xi_phi;
                rng.triple(u_hop, xi_hg, xi_phi);
                R ct, st;
                hg_sample(B, R(xi_hg), ct, st);
                R sn, cs;
                M<R>::sincos_2pi(R(xi_phi), &sn, &cs);
                rotate(ux, uy, uz, ct, st, sn, cs);
                iux = inv_dir(ux); iuy = inv_dir(uy); iuz = inv_dir(uz);
                if (w < C.rr_threshold) {
                    ++c_rr;
                    if (R(rng.uniform()) < C.rr_inv_m) {
                        if constexpr (BATCH)
                            atomicAdd(p.sims[sim].tally + MCX_TALLY_RR_GAINED, double((C.rr_m - R(1)) * w));
                        else
                            atomicAdd(&s_tally[MCX_TALLY_RR_GAINED], double((C.rr_m - R(1)) * w));
                        gained += (C.rr_m - R(1)) * w;
                        w *= C.rr_m;
                        ++nrr;
                    } else {
                        fate = MCX_FATE_ROULETTE;
                    }
                }
                if (fate == MCX_FATE_NONE) {              // a4: the next hop, drawn with the
                    const R h = M<R>::hop(R(u_hop));      // deflection
                    s = h > M<R>::tiny_hop() ? h : M<R>::tiny_hop();
                }
            }
        }
        if (fate == MCX_FATE_NONE) continue;

        // ---- photon finished: flush the deposit run, tallies, logs, detectors (a9, a12)
        flush();
        const R absorbed = R(1) + gained - w;
        const int slot = fate == MCX_FATE_ESCAPED ? MCX_TALLY_ESCAPED
                       : (fate == MCX_FATE_ROULETTE ? MCX_TALLY_RR_KILLED : MCX_TALLY_TIME);
        if constexpr (BATCH) {
            atomicAdd(p.sims[sim].tally + slot, double(w));
            atomicAdd(p.sims[sim].tally + MCX_TALLY_ABSORBED, double(absorbed));
        } else {
            atomicAdd(&s_tally[slot], double(w));
            atomicAdd(&s_tally[MCX_TALLY_ABSORBED], double(absorbed));
        }
        atomicAdd(&s_stats[MCX_STAT_SCATTER], (unsigned long long)nscat);
        atomicAdd(&s_stats[MCX_STAT_FACE], (unsigned long long)c_face);
        atomicAdd(&s_stats[MCX_STAT_FRESNEL], (unsigned long long)c_fres);
        atomicAdd(&s_stats[MCX_STAT_FLUSH], (unsigned long long)c_flush);
        atomicAdd(&s_stats[MCX_STAT_ROULETTE], (unsigned long long)c_rr);
        atomicAdd(&s_stats[MCX_STAT_PHOTONS], 1ull);
        if (fate == MCX_FATE_CAPPED) {
            atomicAdd(&s_stats[MCX_STAT_CAPPED], 1ull);
            atomicOr(p.status, kStatusCapped);
        }
        if constexpr (PAD && ACC != kAccCompensated) {
            // the voxel's indices from its linear index in the padded volume
            const unsigned r = vlin % G_sz;
            iz = (int)(vlin / G_sz) - 1;
            iy = (int)(r / G_sy) - 1;
            ix = (int)(r % G_sy) - 1;
        }
        const R hh = R(p.h);
        const R ex = (R(ix) + qx) * hh, ey = (R(iy) + qy) * hh, ez = (R(iz) + qz) * hh;
        const unsigned long long rel = pid - p.photon_offset;
        if (rel < p.exit_log) {
            mcx_exit e;
            e.fate = fate; e.nscat = nscat;
            e.pos[0] = float(ex); e.pos[1] = float(ey); e.pos[2] = float(ez);
            e.dir[0] = float(ux); e.dir[1] = float(uy); e.dir[2] = float(uz);
            e.w = float(w); e.t = float(t);
            p.exits[rel] = e;
        }
        if (DET && fate == MCX_FATE_ESCAPED) {
            const float vx = float(R(ix) + qx), vy = float(R(iy) + qy), vz = float(R(iz) + qz);
            for (int d = 0; d < p.n_det; ++d) {
                const float4 D = s_det[d];
                const float dx = vx - D.x, dy = vy - D.y, dz = vz - D.z;
                if (dx * dx + dy * dy + dz * dz <= D.w) {
                    atomicAdd(&s_stats[MCX_STAT_DETECTED], 1ull);
                    const unsigned long long slot_i = atomicAdd(p.det_count, 1ull);
                    if (slot_i < p.max_detected) {
                        if (lab < kMaxDetMedia) Lpath[lab] += float(Lcur);
                        float *rec = p.det_buf + slot_i * (unsigned long long)p.rec_stride;
                        rec[0] = __uint_as_float((unsigned)(pid & 0xffffffffull));
                        rec[1] = __uint_as_float((unsigned)(pid >> 32));
                        rec[2] = __int_as_float(d);
                        rec[3] = __uint_as_float(nscat);
                        rec[4] = float(w);
                        rec[5] = float(ex); rec[6] = float(ey); rec[7] = float(ez);
                        rec[8] = float(ux); rec[9] = float(uy); rec[10] = float(uz);
                        rec[11] = __uint_as_float(nrr);
                        for (int m = 1; m < p.n_media && m < kMaxDetMedia; ++m)
                            rec[kRecBase + m - 1] = Lpath[m] * p.h;
                    } else {
                        atomicOr(p.status, kStatusDetOverflow);
                    }
                    break;
                }
            }
        }
        alive = false;
    }

    __syncthreads();
    if (ACC == kAccCompensated) {
        // the block's tile, flushed once in FP64 into the map at its (gate, voxel) positions
        const int s0 = p.tile_size[0], s1 = p.tile_size[1], s2 = p.tile_size[2];
        constexpr unsigned B = PAD ? 1u : 0u;          // the map's border
        for (int k = threadIdx.x; k < tile_e; k += blockDim.x) {
            const double v = (double)s_hi[k] + (double)s_lo[k];
            if (v == 0.0) continue;
            const int tx = k % s0, ty = (k / s0) % s1, tz = (k / (s0 * s1)) % s2, tg = k / (s0 * s1 * s2);
            const unsigned vl = (unsigned)(p.tile_lo[2] + tz + B) * G_sz + (unsigned)(p.tile_lo[1] + ty + B) * G_sy +
                                (unsigned)(p.tile_lo[0] + tx + B);
            atomicAdd(G_flu64 + (unsigned long long)(p.tile_lo[3] + tg) * G_nvox + vl, v);
        }
    }
    if (threadIdx.x < MCX_NTALLY)
        p.block_tally[(size_t)blockIdx.x * MCX_NTALLY + threadIdx.x] = s_tally[threadIdx.x];
    if (threadIdx.x < MCX_NSTAT)
        p.block_stats[(size_t)blockIdx.x * MCX_NSTAT + threadIdx.x] = s_stats[threadIdx.x];
}

// ------------------------------------------------------------------------------ debug
__global__ void uniforms_kernel(uint64_t seed, uint64_t photon, uint64_t n, float *out)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    Rng r;
    r.seed(seed, photon);
    // per output: the single draw, the pair's second value (from a copy of the state),
    // then the triple from the same output
    for (uint64_t i = 0; i < n; ++i) {
        Rng c = r;
        c.pair(out[5 * i], out[5 * i + 1]);
        r.triple(out[5 * i + 2], out[5 * i + 3], out[5 * i + 4]);
    }
}

__global__ void primitive_kernel(int kind, uint64_t n, const float *in, float *out)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (kind == 0) {
        const float g = in[2 * i], xi = in[2 * i + 1];
        const MedB<float> B = hg_consts(g);
        float ct, st;
        hg_sample(B, xi, ct, st);
        out[2 * i] = ct;
        out[2 * i + 1] = st;
    } else if (kind == 1) {
        float ux = in[6 * i], uy = in[6 * i + 1], uz = in[6 * i + 2];
        float sn, cs;
        M<float>::sincos_2pi(in[6 * i + 5], &sn, &cs);
        rotate(ux, uy, uz, in[6 * i + 3], in[6 * i + 4], sn, cs);
        out[3 * i] = ux; out[3 * i + 1] = uy; out[3 * i + 2] = uz;
    } else {
        const float n1 = in[3 * i], n2 = in[3 * i + 1], ci = in[3 * i + 2];
        const float eta = M<float>::div(n1, n2);
        const float st2 = eta * eta * fmaf(-ci, ci, 1.f);
        out[i] = st2 < 1.f ? fresnel(n1, n2, ci, st2) : 1.f;
    }
}

}  // namespace

// ------------------------------------------------------------------------------ host side
namespace {
template <typename R>
size_t table_bytes(int n_media)
{
    return align16(sizeof(MedA<R>) * n_media) + align16(sizeof(MedB<R>) * n_media) +
           align16(sizeof(R) * n_media) * 2;
}

// Per-label constants in voxel units (h = voxel edge): mus h, 1/(mus h), mua h, c0/(n h),
// the HG constants, n, and n h / c0.  Set-up arithmetic on the inputs, done once per run.
template <typename R>
void fill(int n_media, const float *props, float h, unsigned char *buf, const void **oa,
          const void **ob, const void **on, const void **ot)
{
    const size_t a = 0, b = align16(sizeof(MedA<R>) * n_media);
    const size_t n = b + align16(sizeof(MedB<R>) * n_media);
    const size_t t = n + align16(sizeof(R) * n_media);
    const R hh = R(h), c0 = R(299.792458);
    for (int m = 0; m < n_media; ++m) {
        const R mua = R(props[4 * m]), mus = R(props[4 * m + 1]);
        const R g = R(props[4 * m + 2]), nn = R(props[4 * m + 3]);
        MedA<R> A;
        // scattering and absorption per voxel length, in the walk's units (M<R>)
        const double mus_v = (double)mus * (double)hh, mua_v = (double)mua * (double)hh;
        A.mus = R(mus_v / M<R>::kHopUnit);
        A.inv_mus = mus_v > 0 ? R(M<R>::kHopUnit / mus_v) : R(INFINITY);
        A.mua = R(mua_v * M<R>::kAbsScale);
        A.len_per_t = c0 / (nn * hh);
        const MedB<R> B = hg_consts(g);
        reinterpret_cast<MedA<R> *>(buf + a)[m] = A;
        reinterpret_cast<MedB<R> *>(buf + b)[m] = B;
        reinterpret_cast<R *>(buf + n)[m] = nn;
        reinterpret_cast<R *>(buf + t)[m] = nn * hh / c0;
    }
    *oa = (const void *)a;
    *ob = (const void *)b;
    *on = (const void *)n;
    *ot = (const void *)t;
}

template <typename R, bool DET, int ACC, bool ST, bool BATCH = false, bool PAD = true>
cudaError_t shape_for(int block, int n_media, int n_det, int tile_e, LaunchShape *shape)
{
    const size_t smem = SmemLayout<R>(n_media, DET ? n_det : 0, tile_e).total;
    cudaError_t e = cudaFuncSetAttribute(walk_kernel<R, DET, ACC, ST, BATCH, PAD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_kernel<R, DET, ACC, ST, BATCH, PAD>,
                                                           block, smem)) != cudaSuccess)
        return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, walk_kernel<R, DET, ACC, ST, BATCH, PAD>)) != cudaSuccess) return e;
    shape->block = block;
    shape->blocks_per_sm = per_sm;
    shape->grid = sms * (per_sm > 0 ? per_sm : 1);
    shape->regs = fa.numRegs;
    return cudaSuccess;
}

template <typename R, bool DET, int ACC, bool ST, bool BATCH = false, bool PAD = true>
cudaError_t launch(const WalkParams &p, const LaunchShape &s, cudaStream_t st)
{
    const int tile_e = ACC == kAccCompensated
        ? p.tile_size[0] * p.tile_size[1] * p.tile_size[2] * p.tile_size[3] : 0;
    const size_t smem = SmemLayout<R>(BATCH ? 0 : p.n_media, DET ? p.n_det : 0, tile_e).total;
    walk_kernel<R, DET, ACC, ST, BATCH, PAD><<<s.grid, s.block, smem, st>>>(p);
    return cudaGetLastError();
}

// The static per-thread split (a study of the paper's thread-level balancing) is built for
// the FP32 walk only, so the default dynamic kernel carries none of its code.
template <typename R, bool DET, int ACC>
cudaError_t shape_s(bool st, int block, int nm, int nd, int te, LaunchShape *sh)
{
    if (st && sizeof(R) == 4) return shape_for<R, DET, ACC, true>(block, nm, nd, te, sh);
    return shape_for<R, DET, ACC, false>(block, nm, nd, te, sh);
}

template <typename R, bool DET, int ACC>
cudaError_t launch_s(const WalkParams &p, const LaunchShape &s, cudaStream_t st)
{
    if (p.claim_static && sizeof(R) == 4) return launch<R, DET, ACC, true>(p, s, st);
    return launch<R, DET, ACC, false>(p, s, st);
}

template <typename R, int ACC>
cudaError_t shape_d(bool det, bool st, int block, int nm, int nd, int te, LaunchShape *sh)
{
    return det ? shape_s<R, true, ACC>(st, block, nm, nd, te, sh)
               : shape_s<R, false, ACC>(st, block, nm, nd, te, sh);
}

template <typename R, int ACC>
cudaError_t launch_d(const WalkParams &p, const LaunchShape &s, cudaStream_t st)
{
    return p.n_det > 0 ? launch_s<R, true, ACC>(p, s, st) : launch_s<R, false, ACC>(p, s, st);
}

template <typename R>
cudaError_t shape_a(bool det, bool st, int acc, int block, int nm, int nd, int te, LaunchShape *sh)
{
    if (acc == kAccCompensated) return shape_d<R, kAccCompensated>(det, st, block, nm, nd, te, sh);
    if (acc == kAccF64) return shape_d<R, kAccF64>(det, st, block, nm, nd, te, sh);
    return shape_d<R, kAccPlain>(det, st, block, nm, nd, te, sh);
}

template <typename R>
cudaError_t launch_a(const WalkParams &p, int acc, const LaunchShape &s, cudaStream_t st)
{
    if (acc == kAccCompensated) return launch_d<R, kAccCompensated>(p, s, st);
    if (acc == kAccF64) return launch_d<R, kAccF64>(p, s, st);
    return launch_d<R, kAccPlain>(p, s, st);
}
}  // namespace

size_t walk_table_bytes(Precision prec, int n_media)
{
    return prec == Precision::F64 ? table_bytes<double>(n_media) : table_bytes<float>(n_media);
}

void walk_fill_tables(Precision prec, int n_media, const float *props, float h, void *host_buf,
                      const void **oa, const void **ob, const void **on, const void **ot)
{
    unsigned char *b = static_cast<unsigned char *>(host_buf);
    if (prec == Precision::F64) fill<double>(n_media, props, h, b, oa, ob, on, ot);
    else fill<float>(n_media, props, h, b, oa, ob, on, ot);
}

cudaError_t walk_query_shape(bool det, Precision prec, int accum, int block, int n_media,
                             int n_det, int tile_entries, bool claim_static, LaunchShape *shape)
{
    if (prec == Precision::F64)
        return shape_a<double>(det, false, accum, block, n_media, n_det, tile_entries, shape);
    return shape_a<float>(det, claim_static, accum, block, n_media, n_det, tile_entries, shape);
}

cudaError_t walk_launch(const WalkParams &p, Precision prec, int accum, const LaunchShape &s,
                        cudaStream_t st)
{
    if (prec == Precision::F64) return launch_a<double>(p, accum, s, st);
    return launch_a<float>(p, accum, s, st);
}

cudaError_t walk_batch_query_shape(int accum, int block, LaunchShape *shape)
{
    if (accum == kAccF64) return shape_for<float, false, kAccF64, false, true>(block, 0, 0, 0, shape);
    return shape_for<float, false, kAccPlain, false, true>(block, 0, 0, 0, shape);
}

cudaError_t walk_batch_launch(const WalkParams &p, int accum, const LaunchShape &s, cudaStream_t st)
{
    if (accum == kAccF64) return launch<float, false, kAccF64, false, true>(p, s, st);
    return launch<float, false, kAccPlain, false, true>(p, s, st);
}

cudaError_t walk_query_shape_unpadded(int accum, int block, LaunchShape *shape)
{
    if (accum == kAccF64) return shape_for<float, false, kAccF64, false, false, false>(block, 32, 0, 0, shape);
    return shape_for<float, false, kAccPlain, false, false, false>(block, 32, 0, 0, shape);
}

cudaError_t walk_launch_unpadded(const WalkParams &p, int accum, const LaunchShape &s, cudaStream_t st)
{
    if (accum == kAccF64) return launch<float, false, kAccF64, false, false, false>(p, s, st);
    return launch<float, false, kAccPlain, false, false, false>(p, s, st);
}

cudaError_t debug_uniforms(uint64_t seed, uint64_t photon, uint64_t n, float *dev_out)
{
    uniforms_kernel<<<1, 1>>>(seed, photon, n, dev_out);
    return cudaGetLastError();
}

cudaError_t debug_primitive(int kind, uint64_t n, const float *dev_in, float *dev_out)
{
    if (n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    primitive_kernel<<<blocks, 256>>>(kind, n, dev_in, dev_out);
    return cudaGetLastError();
}

}  // namespace mcxg
