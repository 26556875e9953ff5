// C ABI of the photon-transport library (include/mcx.h): host-side set-up, buffer
// ownership, run orchestration on a caller-chosen stream, and the post-processing kernels
// (tally reduction, fluence normalisation, detected-record ordering).
//
// Mirrors the host side of the paper's workflow (Fig. 1 paragraph): inputs are processed
// and copied to the device, the device runs the photon loop, the host waits and reads back
// the fluence maps and detected-photon data, and post-processing yields the final
// (normalised) solution.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "mcx_internal.h"

using namespace mcxg;

namespace {

thread_local std::string g_err;   // errors raised before a handle exists

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t want)
    {
        if (want <= bytes && p) return cudaSuccess;
        release();
        if (want == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) { p = nullptr; bytes = 0; return e; }
        bytes = want;
        return cudaSuccess;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// ---------------------------------------------------------------------------- kernels
__global__ void zero_words(uint32_t *p, size_t n)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const size_t n4 = n / 4;
    uint4 *p4 = reinterpret_cast<uint4 *>(p);
    for (size_t k = i; k < n4; k += stride) p4[k] = make_uint4(0, 0, 0, 0);
    for (size_t k = n4 * 4 + i; k < n; k += stride) p[k] = 0u;
}

// Sums the per-block FP64 tallies and counters in a fixed order (strided partial sums,
// then a tree), so the result depends only on the per-block partials.
__global__ void finalize_kernel(const double *bt, const unsigned long long *bs, int nblocks,
                                double n_launched, double *out_t, unsigned long long *out_s)
{
    __shared__ double st[256][MCX_NTALLY];
    __shared__ unsigned long long ss[256][MCX_NSTAT];
    const int tid = threadIdx.x;
    double t[MCX_NTALLY] = {0};
    unsigned long long c[MCX_NSTAT] = {0};
    for (int b = tid; b < nblocks; b += blockDim.x) {
        for (int k = 0; k < MCX_NTALLY; ++k) t[k] += bt[(size_t)b * MCX_NTALLY + k];
        for (int k = 0; k < MCX_NSTAT; ++k) c[k] += bs[(size_t)b * MCX_NSTAT + k];
    }
    for (int k = 0; k < MCX_NTALLY; ++k) st[tid][k] = t[k];
    for (int k = 0; k < MCX_NSTAT; ++k) ss[tid][k] = c[k];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (tid < h) {
            for (int k = 0; k < MCX_NTALLY; ++k) st[tid][k] += st[tid + h][k];
            for (int k = 0; k < MCX_NSTAT; ++k) ss[tid][k] += ss[tid + h][k];
        }
        __syncthreads();
    }
    if (tid == 0) {
        for (int k = 0; k < MCX_NTALLY; ++k) out_t[k] = st[0][k];
        out_t[MCX_TALLY_LAUNCHED] = n_launched;
        for (int k = 0; k < MCX_NSTAT; ++k) out_s[k] = ss[0][k];
    }
}

// The fluence map as accumulated, in the caller's type, optionally normalised to fluence
// rate per launched photon (x inv_norm[label], inv_norm = 1 / (mua h^3 N dt)):
//   accum 0: the FP32 map;  accum 1 and 2: the FP64 map (accum 1 adds its block tiles
//   into it when the walk ends).

// The maps and labels carry the walk's one-voxel border ([g][nz+2][ny+2][nx+2]); the
// output is unpadded [g][nz][ny][nx].
template <typename T>
__global__ void resolve_kernel(int mode, const float *hi, const double *f64,
                               unsigned nx, unsigned ny, unsigned nvox, unsigned pnvox,
                               unsigned n_gates, const uint8_t *labels, const float *inv_norm,
                               T *out)
{
    const size_t total = (size_t)nvox * n_gates;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += stride) {
        const unsigned v = (unsigned)(i % nvox);
        const unsigned g = (unsigned)(i / nvox);
        const unsigned x = v % nx, y = (v / nx) % ny, z = v / (nx * ny);
        const unsigned pv = (unsigned)padded_index(x, y, z, nx, ny);
        const size_t pi = (size_t)g * pnvox + pv;
        if (mode == 0) {
            float f = hi[pi];
            if (inv_norm) f *= inv_norm[labels[pv]];
            out[i] = (T)f;
            continue;
        }
        double d = f64[pi];
        if (inv_norm) d *= (double)inv_norm[labels[pv]];
        out[i] = (T)d;
    }
}

// Copies an unpadded label volume into the interior of its bordered copy (border zeroed
// beforehand).
__global__ void pad_labels_kernel(const uint8_t *src, unsigned nx, unsigned ny, unsigned nz, uint8_t *dst)
{
    const size_t n = (size_t)nx * ny * nz;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned x = (unsigned)(i % nx), y = (unsigned)((i / nx) % ny), z = (unsigned)(i / ((size_t)nx * ny));
        dst[padded_index(x, y, z, nx, ny)] = src[i];
    }
}

__global__ void label_max_kernel(const uint8_t *labels, size_t n, unsigned *out)
{
    unsigned m = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride)
        m = max(m, (unsigned)labels[i]);
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// detected-record ordering: key = photon id (padding keys = max), value = record slot
__global__ void det_keys_kernel(const float *rec, int stride, unsigned long long n,
                                unsigned long long npow2, unsigned long long *keys,
                                unsigned *vals)
{
    const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (i >= npow2) return;
    if (i < n) {
        const float *r = rec + i * (unsigned long long)stride;
        keys[i] = (unsigned long long)__float_as_uint(r[0]) |
                  ((unsigned long long)__float_as_uint(r[1]) << 32);
    } else {
        keys[i] = ~0ull;
    }
    vals[i] = (unsigned)i;
}

__global__ void bitonic_step(unsigned long long *keys, unsigned *vals, unsigned long long j,
                             unsigned long long k, unsigned long long n)
{
    const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long l = i ^ j;
    if (l <= i) return;
    const bool asc = (i & k) == 0;
    const unsigned long long a = keys[i], b = keys[l];
    if ((a > b) == asc) {
        keys[i] = b; keys[l] = a;
        const unsigned t = vals[i]; vals[i] = vals[l]; vals[l] = t;
    }
}

__global__ void det_gather_kernel(const float *rec, const unsigned *vals, int stride,
                                  unsigned long long n, float *out)
{
    const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (i >= n * (unsigned long long)stride) return;
    const unsigned long long r = i / stride, w = i % stride;
    out[i] = rec[(unsigned long long)vals[r] * stride + w];
}

unsigned grid_for(size_t n, int block = 256, unsigned cap = 152u * 16u)
{
    size_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    return (unsigned)std::min<size_t>(g, cap);
}

}  // namespace

// ---------------------------------------------------------------------------- handle
struct mcx_sim {
    int device = 0;
    uint32_t nx = 0, ny = 0, nz = 0;
    float h = 1.f;
    unsigned label_max = 0;
    std::vector<float> props;           // [n_media][4]
    uint32_t n_media = 0;
    int src_kind = 0;
    double src_pos[3] = {0, 0, 0}, src_dir[3] = {0, 0, 1}, src_waist = 0;
    bool source_set = false;
    std::vector<float> det;             // [n_det][4] cx, cy, cz, r (mm)

    DevBuf labels, fluence, fluence64, tables, detb, det_buf, exits, block_tally,
        block_stats, ctrl, out, staging, inv_norm, sort_keys, sort_vals;
    std::vector<unsigned char> host_tables;

    // last run
    bool ran = false;
    mcx_run_cfg cfg{};
    LaunchShape shape{};
    int rec_stride = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr, ev_done = nullptr;
    std::map<std::tuple<int, int, int, int, int, int, int>, LaunchShape> shape_cache;

    std::string err;
};

void mcxg::set_global_error(const std::string &msg) { g_err = msg; }

static mcx_status fail(mcx_sim *s, mcx_status st, const std::string &msg)
{
    if (s) s->err = msg; else g_err = msg;
    return st;
}

static mcx_status cuda_fail(mcx_sim *s, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(s, e == cudaErrorMemoryAllocation ? MCX_E_OOM : MCX_E_CUDA, m);
}

#define MCX_CUDA(s, call, what)                                   \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail((s), e_, (what)); \
    } while (0)

extern "C" {

int32_t mcx_abi_version(void) { return MCX_ABI_VERSION; }

const char *mcx_status_string(int32_t st)
{
    switch (st) {
    case MCX_OK: return "ok";
    case MCX_E_ARG: return "invalid argument";
    case MCX_E_STATE: return "call out of order";
    case MCX_E_CUDA: return "CUDA error";
    case MCX_E_OOM: return "device out of memory";
    case MCX_E_CAP: return "capacity reached (outputs valid)";
    case MCX_E_TIMEOUT: return "timed out waiting for the run";
    default: return "unknown status";
    }
}

void mcx_run_cfg_default(mcx_run_cfg *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->struct_size = sizeof(mcx_run_cfg);
    c->n_gates = 1;
    c->n_photons = 0;
    c->seed = 1;
    c->dt_ns = 5.f;
    c->reflect = 1;
    c->rr_threshold = 1e-4f;
    c->rr_m = 10.f;
    c->max_detected = 0;
    c->exit_log = 0;
    c->max_events_per_photon = 0;
    c->accum_mode = 2;      // FP64 atomics: exact, and as fast as FP32 atomics on GB300
    c->block_size = 0;
    c->grid_size = 0;
    c->precision = 0;
    c->cuda_stream = nullptr;
}

// The device copy of the labels carries a one-voxel border of label 0 (the exterior) on
// every side, which lets the walk step into a neighbour voxel without bounds checks.
static mcx_status upload_labels(mcx_sim *s, const uint8_t *labels, int on_device)
{
    const size_t n = (size_t)s->nx * s->ny * s->nz;
    const size_t np = (size_t)(s->nx + 2) * (s->ny + 2) * (s->nz + 2);
    MCX_CUDA(s, s->labels.ensure(np), "allocating the label volume");
    if (on_device) {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, labels) != cudaSuccess || pa.type != cudaMemoryTypeDevice)
            return fail(s, MCX_E_ARG, "labels_on_device = 1 but labels is not device memory");
        MCX_CUDA(s, cudaMemset(s->labels.p, 0, np), "clearing the label volume");
        pad_labels_kernel<<<grid_for(n), 256>>>(labels, s->nx, s->ny, s->nz, s->labels.as<uint8_t>());
        unsigned *d_max = nullptr;
        MCX_CUDA(s, cudaMalloc(&d_max, sizeof(unsigned)), "allocating");
        cudaMemset(d_max, 0, sizeof(unsigned));
        label_max_kernel<<<grid_for(np), 256>>>(s->labels.as<uint8_t>(), np, d_max);
        cudaError_t e = cudaMemcpy(&s->label_max, d_max, sizeof(unsigned), cudaMemcpyDeviceToHost);
        cudaFree(d_max);
        if (e != cudaSuccess) return cuda_fail(s, e, "label scan");
    } else {
        unsigned m = 0;
        for (size_t i = 0; i < n; ++i) m = std::max<unsigned>(m, labels[i]);
        s->label_max = m;
        std::vector<uint8_t> padded(np, 0);
        for (uint32_t z = 0; z < s->nz; ++z)
            for (uint32_t y = 0; y < s->ny; ++y)
                std::memcpy(padded.data() + padded_index(0, y, z, s->nx, s->ny),
                            labels + ((size_t)z * s->ny + y) * s->nx, s->nx);
        MCX_CUDA(s, cudaMemcpy(s->labels.p, padded.data(), np, cudaMemcpyHostToDevice), "copying labels");
    }
    s->ran = false;
    return MCX_OK;
}

mcx_status mcx_create_volume(mcx_sim **out, uint32_t nx, uint32_t ny, uint32_t nz,
                             float voxel_mm, const uint8_t *labels, int32_t labels_on_device)
{
    if (!out) return fail(nullptr, MCX_E_ARG, "out is NULL");
    *out = nullptr;
    if (!labels) return fail(nullptr, MCX_E_ARG, "labels is NULL");
    if (nx == 0 || ny == 0 || nz == 0) return fail(nullptr, MCX_E_ARG, "empty volume");
    if ((uint64_t)(nx + 2ull) * (ny + 2ull) * (nz + 2ull) >= (1ull << 32))
        return fail(nullptr, MCX_E_ARG, "volume must have (nx+2)(ny+2)(nz+2) < 2^32 voxels");
    if (!(voxel_mm > 0.f) || !std::isfinite(voxel_mm))
        return fail(nullptr, MCX_E_ARG, "voxel_mm must be positive and finite");
    mcx_sim *s = new (std::nothrow) mcx_sim();
    if (!s) return fail(nullptr, MCX_E_OOM, "host allocation failed");
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return fail(nullptr, MCX_E_CUDA, "no CUDA device");
    }
    s->nx = nx; s->ny = ny; s->nz = nz; s->h = voxel_mm;
    mcx_status st = upload_labels(s, labels, labels_on_device);
    if (st != MCX_OK) {
        g_err = s->err;
        mcx_destroy(s);
        return st;
    }
    if (cudaEventCreate(&s->ev_start) != cudaSuccess || cudaEventCreate(&s->ev_stop) != cudaSuccess ||
        cudaEventCreate(&s->ev_done) != cudaSuccess) {
        mcx_destroy(s);
        return fail(nullptr, MCX_E_CUDA, "event creation failed");
    }
    *out = s;
    return MCX_OK;
}

mcx_status mcx_update_labels(mcx_sim *s, const uint8_t *labels, int32_t on_device)
{
    if (!s) return fail(nullptr, MCX_E_ARG, "sim is NULL");
    if (!labels) return fail(s, MCX_E_ARG, "labels is NULL");
    DeviceGuard g(s->device);
    if (s->ran) cudaEventSynchronize(s->ev_done);
    return upload_labels(s, labels, on_device);
}

mcx_status mcx_set_media(mcx_sim *s, uint32_t n_media, const float *props)
{
    if (!s) return fail(nullptr, MCX_E_ARG, "sim is NULL");
    if (!props || n_media < 1 || n_media > (uint32_t)kMaxMedia)
        return fail(s, MCX_E_ARG, "need 1..256 media rows");
    for (uint32_t m = 0; m < n_media; ++m) {
        const float mua = props[4 * m], mus = props[4 * m + 1], g = props[4 * m + 2],
                    n = props[4 * m + 3];
        if (m == 0) {                       // the exterior: only n is used
            if (!(n > 0.f) || !std::isfinite(n))
                return fail(s, MCX_E_ARG, "media row 0 (exterior): need n > 0");
            continue;
        }
        if (!std::isfinite(mua) || !std::isfinite(mus) || !std::isfinite(g) || !std::isfinite(n) ||
            mua < 0.f || mus < 0.f || !(std::fabs(g) < 1.f) || !(n > 0.f))
            return fail(s, MCX_E_ARG, "media row " + std::to_string(m) +
                                          ": need mua >= 0, mus >= 0, |g| < 1, n > 0");
    }
    s->props.assign(props, props + 4 * n_media);
    s->n_media = n_media;
    s->ran = false;
    return MCX_OK;
}

mcx_status mcx_set_source(mcx_sim *s, int32_t kind, const float pos[3], const float dir[3],
                          float waist)
{
    if (!s) return fail(nullptr, MCX_E_ARG, "sim is NULL");
    if (!pos || !dir || (kind != 0 && kind != 1)) return fail(s, MCX_E_ARG, "bad source");
    const double n = std::sqrt((double)dir[0] * dir[0] + (double)dir[1] * dir[1] +
                               (double)dir[2] * dir[2]);
    if (!(n > 0.0) || !std::isfinite(n)) return fail(s, MCX_E_ARG, "source direction is zero");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(pos[a])) return fail(s, MCX_E_ARG, "source position not finite");
    if (kind == 1 && !(waist > 0.f)) return fail(s, MCX_E_ARG, "Gaussian waist must be > 0");
    s->src_kind = kind;
    for (int a = 0; a < 3; ++a) {
        s->src_pos[a] = pos[a];
        s->src_dir[a] = dir[a] / n;
    }
    s->src_waist = waist;
    s->source_set = true;
    s->ran = false;
    return MCX_OK;
}

mcx_status mcx_add_detector(mcx_sim *s, const float c[3], float r, int32_t *out_id)
{
    if (!s) return fail(nullptr, MCX_E_ARG, "sim is NULL");
    if (!c || !(r > 0.f) || !std::isfinite(r)) return fail(s, MCX_E_ARG, "bad detector");
    if (s->det.size() / 4 >= (size_t)kMaxDet) return fail(s, MCX_E_ARG, "at most 64 detectors");
    s->det.insert(s->det.end(), {c[0], c[1], c[2], r});
    if (out_id) *out_id = (int32_t)(s->det.size() / 4 - 1);
    s->ran = false;
    return MCX_OK;
}

mcx_status mcx_clear_detectors(mcx_sim *s)
{
    if (!s) return fail(nullptr, MCX_E_ARG, "sim is NULL");
    s->det.clear();
    s->ran = false;
    return MCX_OK;
}

mcx_status mcx_run(mcx_sim *s, const mcx_run_cfg *cfg)
{
    if (!s) return fail(nullptr, MCX_E_ARG, "sim is NULL");
    if (!cfg || cfg->struct_size != sizeof(mcx_run_cfg))
        return fail(s, MCX_E_ARG, "cfg is NULL or struct_size does not match this library");
    if (s->n_media == 0) return fail(s, MCX_E_STATE, "mcx_set_media has not been called");
    if (!s->source_set) return fail(s, MCX_E_STATE, "mcx_set_source has not been called");
    if (s->label_max >= s->n_media)
        return fail(s, MCX_E_STATE, "the volume has label " + std::to_string(s->label_max) +
                                        " but only " + std::to_string(s->n_media) + " media rows");
    const int n_det = (int)(s->det.size() / 4);
    if (n_det > 0 && s->n_media > (uint32_t)kMaxDetMedia)
        return fail(s, MCX_E_ARG, "with detectors, at most 33 media rows");
    if (cfg->n_gates < 1 || !(cfg->dt_ns > 0.f) || !std::isfinite(cfg->dt_ns))
        return fail(s, MCX_E_ARG, "need n_gates >= 1 and dt_ns > 0");
    if (!(cfg->rr_threshold >= 0.f) || (cfg->rr_threshold > 0.f && !(cfg->rr_m > 1.f)))
        return fail(s, MCX_E_ARG, "need rr_threshold >= 0 and rr_m > 1");
    if (cfg->photon_offset + cfg->n_photons < cfg->photon_offset)
        return fail(s, MCX_E_ARG, "photon id range overflows");
    if (cfg->precision != 0 && cfg->precision != 1) return fail(s, MCX_E_ARG, "precision is 0 or 1");
    if (cfg->accum_mode < 0 || cfg->accum_mode > 2) return fail(s, MCX_E_ARG, "accum_mode is 0, 1 or 2");
    const int block = cfg->block_size ? cfg->block_size : 256;
    if (block < 32 || block > 256 || block % 32) return fail(s, MCX_E_ARG, "block_size: 32..256, multiple of 32");
    if (cfg->grid_size < 0) return fail(s, MCX_E_ARG, "grid_size < 0");
    if (cfg->claim_mode != 0 && cfg->claim_mode != 1) return fail(s, MCX_E_ARG, "claim_mode is 0 or 1");

    DeviceGuard guard(s->device);
    if (!guard.ok) return fail(s, MCX_E_CUDA, "cannot select the handle's device");
    if (s->ran) MCX_CUDA(s, cudaEventSynchronize(s->ev_done), "waiting for the previous run");

    const Precision prec = cfg->precision ? Precision::F64 : Precision::F32;
    const int accum = cfg->accum_mode;
    // block tile of the compensated mode: given, or 16 x 16 x 24 voxels of gate 0 from the
    // source voxel down, clipped to the grid
    int tlo[4] = {0, 0, 0, 0}, tsz[4] = {0, 0, 0, 0};
    if (accum == kAccCompensated) {
        const bool automatic = !(cfg->tile_size[0] | cfg->tile_size[1] | cfg->tile_size[2] |
                                 cfg->tile_size[3]);
        const int dims[4] = {(int)s->nx, (int)s->ny, (int)s->nz, (int)cfg->n_gates};
        if (automatic) {
            const int want[4] = {16, 16, 24, 1};
            for (int a = 0; a < 4; ++a) {
                int c = a < 3 ? (int)std::floor(s->src_pos[a] / s->h) : 0;
                c = std::min(std::max(c, 0), dims[a] - 1);
                int lo = a < 2 ? c - want[a] / 2 : c;
                lo = std::min(std::max(lo, 0), std::max(dims[a] - want[a], 0));
                tlo[a] = lo;
                tsz[a] = std::min(want[a], dims[a] - lo);
            }
        } else {
            long long e = 1;
            for (int a = 0; a < 4; ++a) {
                tlo[a] = cfg->tile_lo[a];
                tsz[a] = cfg->tile_size[a];
                if (tsz[a] < 1 || tlo[a] < 0 || tlo[a] + tsz[a] > dims[a])
                    return fail(s, MCX_E_ARG, "tile outside the grid or empty");
                e *= tsz[a];
            }
            if (e > kTileMaxEntries)
                return fail(s, MCX_E_ARG, "tile larger than 6144 (gate, voxel) entries");
        }
    }
    const int tile_e = tsz[0] * tsz[1] * tsz[2] * tsz[3];
    const bool claim_static = cfg->claim_mode == 1;
    if (claim_static && prec == Precision::F64)
        return fail(s, MCX_E_ARG, "claim_mode 1 needs precision 0");
    const auto key = std::make_tuple((int)(n_det > 0) + 2 * (int)claim_static, (int)prec, block,
                                     (int)s->n_media, n_det, accum, tile_e);
    LaunchShape shape;
    auto it = s->shape_cache.find(key);
    if (it == s->shape_cache.end()) {
        MCX_CUDA(s, walk_query_shape(n_det > 0, prec, accum, block, (int)s->n_media, n_det,
                                     tile_e, claim_static, &shape),
                 "querying the walk kernel");
        if (shape.blocks_per_sm < 1) return fail(s, MCX_E_ARG, "block_size does not fit on an SM");
        s->shape_cache[key] = shape;
    } else {
        shape = it->second;
    }
    if (cfg->grid_size > 0) shape.grid = cfg->grid_size;

    // maps with the walk's one-voxel border, as the label volume
    const uint64_t nvox = (uint64_t)(s->nx + 2) * (s->ny + 2) * (s->nz + 2);
    const uint64_t nflu = nvox * cfg->n_gates;
    const int stride = kRecBase + (int)s->n_media - 1;
    // accum 0 accumulates into the FP32 map, accum 1 and 2 into the FP64 one
    const uint64_t nflu32 = accum == kAccPlain ? nflu : 1;
    MCX_CUDA(s, s->fluence.ensure(nflu32 * sizeof(float)), "allocating the fluence map");
    if (accum != kAccPlain)
        MCX_CUDA(s, s->fluence64.ensure(nflu * sizeof(double)), "allocating the FP64 fluence map");
    MCX_CUDA(s, s->block_tally.ensure((size_t)shape.grid * MCX_NTALLY * sizeof(double)), "allocating");
    MCX_CUDA(s, s->block_stats.ensure((size_t)shape.grid * MCX_NSTAT * 8), "allocating");
    MCX_CUDA(s, s->ctrl.ensure(64), "allocating");
    MCX_CUDA(s, s->out.ensure(MCX_NTALLY * sizeof(double) + MCX_NSTAT * 8), "allocating");
    if (n_det > 0 && cfg->max_detected > 0)
        MCX_CUDA(s, s->det_buf.ensure(cfg->max_detected * stride * sizeof(float)),
                 "allocating the detected-photon buffer");
    if (cfg->exit_log > 0) MCX_CUDA(s, s->exits.ensure(cfg->exit_log * sizeof(mcx_exit)), "allocating the exit log");

    // per-label tables (voxel units) and detectors, copied on the run's stream
    const size_t tb = walk_table_bytes(prec, (int)s->n_media);
    s->host_tables.assign(tb + 16 * kMaxDet, 0);
    const void *oa, *ob, *on, *ot;
    walk_fill_tables(prec, (int)s->n_media, s->props.data(), s->h, s->host_tables.data(), &oa, &ob,
                     &on, &ot);
    float4 *hdet = reinterpret_cast<float4 *>(s->host_tables.data() + tb);
    for (int d = 0; d < n_det; ++d) {
        const float r = s->det[4 * d + 3] / s->h;
        hdet[d] = make_float4(s->det[4 * d] / s->h, s->det[4 * d + 1] / s->h,
                              s->det[4 * d + 2] / s->h, r * r);
    }
    MCX_CUDA(s, s->tables.ensure(s->host_tables.size()), "allocating the media tables");
    cudaStream_t st = static_cast<cudaStream_t>(cfg->cuda_stream);
    MCX_CUDA(s, cudaMemcpyAsync(s->tables.p, s->host_tables.data(), s->host_tables.size(),
                                cudaMemcpyHostToDevice, st), "uploading the media tables");

    WalkParams p{};
    unsigned char *tbase = s->tables.as<unsigned char>();
    p.labels = s->labels.as<uint8_t>();
    p.fluence = s->fluence.as<float>();
    p.fluence64 = s->fluence64.as<double>();
    for (int a = 0; a < 4; ++a) {
        p.tile_lo[a] = tlo[a];
        p.tile_size[a] = tsz[a];
    }
    p.tab_a = tbase + (size_t)oa;
    p.tab_b = tbase + (size_t)ob;
    p.tab_n = tbase + (size_t)on;
    p.tab_tpl = tbase + (size_t)ot;
    p.det = reinterpret_cast<const float4 *>(tbase + tb);
    p.det_buf = s->det_buf.as<float>();
    unsigned long long *ctrl = s->ctrl.as<unsigned long long>();
    p.photon_counter = ctrl;
    p.det_count = ctrl + 1;
    p.status = reinterpret_cast<unsigned *>(ctrl + 2);
    p.exits = s->exits.as<mcx_exit>();
    p.block_tally = s->block_tally.as<double>();
    p.block_stats = s->block_stats.as<unsigned long long>();
    p.nx = (int)s->nx; p.ny = (int)s->ny; p.nz = (int)s->nz;
    p.nvox = (unsigned)nvox;
    p.sy = s->nx + 2;
    p.sz = (s->nx + 2) * (s->ny + 2);
    p.n_media = (int)s->n_media;
    p.n_det = n_det;
    p.rec_stride = stride;
    p.n_gates = cfg->n_gates;
    p.h = s->h;
    {
        RunConsts<double> &d = p.cd;
        d.dt = (double)cfg->dt_ns;
        d.inv_dt = 1.0 / (double)cfg->dt_ns;
        d.t_end = (double)cfg->dt_ns * cfg->n_gates;
        for (int a = 0; a < 3; ++a) {
            d.src_pos[a] = s->src_pos[a] / s->h;
            d.src_dir[a] = s->src_dir[a];
        }
        launch_plane(s->src_dir, d.src_e1, d.src_e2);
        d.waist = s->src_waist / s->h;
        d.rr_threshold = cfg->rr_threshold;
        d.rr_m = cfg->rr_m;
        d.rr_inv_m = cfg->rr_threshold > 0.f ? 1.0 / (double)cfg->rr_m : 0.0;
        RunConsts<float> &f = p.cf;
        f.dt = cfg->dt_ns;
        f.inv_dt = (float)d.inv_dt;
        f.t_end = (float)d.t_end;
        for (int a = 0; a < 3; ++a) {
            f.src_pos[a] = (float)d.src_pos[a];
            f.src_dir[a] = (float)d.src_dir[a];
            f.src_e1[a] = (float)d.src_e1[a];
            f.src_e2[a] = (float)d.src_e2[a];
        }
        f.waist = (float)d.waist;
        f.rr_threshold = (float)d.rr_threshold;
        f.rr_m = (float)d.rr_m;
        f.rr_inv_m = (float)d.rr_inv_m;
    }
    p.src_kind = s->src_kind;
    p.n_photons = cfg->n_photons;
    p.photon_offset = cfg->photon_offset;
    p.seed = cfg->seed;
    p.max_detected = n_det > 0 ? cfg->max_detected : 0;
    p.exit_log = cfg->exit_log;
    p.max_events = cfg->max_events_per_photon ? cfg->max_events_per_photon : 100000000ull;
    p.reflect = cfg->reflect;
    p.claim_static = cfg->claim_mode == 1;
    p.claim_chunk = kClaimChunk;

    // zero the outputs, walk, reduce
    if (accum == kAccPlain)
        zero_words<<<grid_for(nflu32 / 4 + 1), 256, 0, st>>>(s->fluence.as<uint32_t>(), (size_t)nflu32);
    else
        zero_words<<<grid_for(nflu / 2 + 1), 256, 0, st>>>(s->fluence64.as<uint32_t>(), (size_t)nflu * 2);
    zero_words<<<1, 32, 0, st>>>(s->ctrl.as<uint32_t>(), 16);
    if (cfg->exit_log > 0)
        zero_words<<<grid_for(cfg->exit_log * 10 / 4 + 1), 256, 0, st>>>(
            s->exits.as<uint32_t>(), (size_t)cfg->exit_log * sizeof(mcx_exit) / 4);
    MCX_CUDA(s, cudaGetLastError(), "launching the zeroing kernel");
    MCX_CUDA(s, cudaEventRecord(s->ev_start, st), "recording an event");
    MCX_CUDA(s, walk_launch(p, prec, accum, shape, st), "launching the walk kernel");
    MCX_CUDA(s, cudaEventRecord(s->ev_stop, st), "recording an event");
    double *out_t = s->out.as<double>();
    finalize_kernel<<<1, 256, 0, st>>>(p.block_tally, p.block_stats, shape.grid,
                                       (double)cfg->n_photons, out_t,
                                       reinterpret_cast<unsigned long long *>(out_t + MCX_NTALLY));
    MCX_CUDA(s, cudaGetLastError(), "launching the tally reduction");
    MCX_CUDA(s, cudaEventRecord(s->ev_done, st), "recording an event");

    s->cfg = *cfg;
    s->shape = shape;
    s->rec_stride = stride;
    s->stream = st;
    s->ran = true;
    return MCX_OK;
}

static mcx_status wait_done(mcx_sim *s)
{
    if (!s->ran) return fail(s, MCX_E_STATE, "no completed run");
    MCX_CUDA(s, cudaEventSynchronize(s->ev_done), "waiting for the run");
    return MCX_OK;
}

mcx_status mcx_sync(mcx_sim *s, double timeout_s)
{
    if (!s) return fail(nullptr, MCX_E_ARG, "sim is NULL");
    if (!s->ran) return fail(s, MCX_E_STATE, "no run to wait for");
    DeviceGuard g(s->device);
    const auto t0 = std::chrono::steady_clock::now();
    while (true) {
        const cudaError_t e = cudaEventQuery(s->ev_done);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(s, e, "run failed");
        if (timeout_s >= 0) {
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (el > timeout_s) return fail(s, MCX_E_TIMEOUT, "run still in flight after the timeout");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    unsigned long long ctrl[3];
    MCX_CUDA(s, cudaMemcpy(ctrl, s->ctrl.p, sizeof(ctrl), cudaMemcpyDeviceToHost), "reading status");
    const unsigned status = (unsigned)ctrl[2];
    if (status & kStatusCapped)
        return fail(s, MCX_E_CAP, "a photon reached max_events_per_photon; it was stopped and its weight counted as time-exceeded");
    if (status & kStatusDetOverflow)
        return fail(s, MCX_E_CAP, "detected-photon buffer overflowed (" + std::to_string(ctrl[1]) +
                                      " detected, capacity " + std::to_string(s->cfg.max_detected) + ")");
    return MCX_OK;
}

mcx_status mcx_last_kernel_ms(mcx_sim *s, float *ms)
{
    if (!s || !ms) return fail(s, MCX_E_ARG, "NULL argument");
    DeviceGuard g(s->device);
    mcx_status st = wait_done(s);
    if (st != MCX_OK) return st;
    MCX_CUDA(s, cudaEventElapsedTime(ms, s->ev_start, s->ev_stop), "reading the kernel time");
    return MCX_OK;
}

}  // extern "C"

template <typename T>
static mcx_status read_fluence_t(mcx_sim *s, T *dst, uint64_t n_elems, int32_t normalized,
                                 int32_t dst_on_device)
{
    if (!s) return fail(nullptr, MCX_E_ARG, "sim is NULL");
    if (!dst) return fail(s, MCX_E_ARG, "dst is NULL");
    if (!s->ran) return fail(s, MCX_E_STATE, "no run");
    DeviceGuard g(s->device);
    const uint64_t nvox = (uint64_t)s->nx * s->ny * s->nz;
    const uint64_t pnvox = (uint64_t)(s->nx + 2) * (s->ny + 2) * (s->nz + 2);
    const uint64_t n = nvox * s->cfg.n_gates;
    if (n_elems != n) return fail(s, MCX_E_ARG, "n_elems must be n_gates*nx*ny*nz = " + std::to_string(n));
    cudaStream_t st = s->stream;
    const int mode = s->cfg.accum_mode;
    const float *inv_dev = nullptr;
    if (normalized) {
        // inv_norm[label] = 1 / (mua h^3 N dt), 0 where mua = 0 or N = 0
        std::vector<float> inv(kMaxMedia, 0.f);
        const double N = (double)s->cfg.n_photons;
        const double v = (double)s->h * s->h * s->h;
        for (uint32_t m = 1; m < s->n_media; ++m) {
            const double mua = s->props[4 * m];
            if (mua > 0 && N > 0) inv[m] = (float)(1.0 / (mua * v * N * (double)s->cfg.dt_ns));
        }
        MCX_CUDA(s, s->inv_norm.ensure(kMaxMedia * sizeof(float)), "allocating");
        MCX_CUDA(s, cudaMemcpyAsync(s->inv_norm.p, inv.data(), kMaxMedia * sizeof(float),
                                    cudaMemcpyHostToDevice, st), "uploading normalisation");
        MCX_CUDA(s, cudaStreamSynchronize(st), "uploading normalisation");
        inv_dev = s->inv_norm.as<float>();
    }
    T *out = dst;
    if (!dst_on_device) {
        MCX_CUDA(s, s->staging.ensure(n * sizeof(T)), "allocating the staging buffer");
        out = static_cast<T *>(s->staging.p);
    }
    resolve_kernel<T><<<grid_for(n), 256, 0, st>>>(mode, s->fluence.as<float>(),
                                                   s->fluence64.as<double>(), s->nx, s->ny,
                                                   (unsigned)nvox, (unsigned)pnvox, s->cfg.n_gates,
                                                   s->labels.as<uint8_t>(), inv_dev, out);
    MCX_CUDA(s, cudaGetLastError(), "launching the fluence read-out");
    if (dst_on_device) return MCX_OK;
    MCX_CUDA(s, cudaMemcpyAsync(dst, out, n * sizeof(T), cudaMemcpyDeviceToHost, st),
             "copying the fluence");
    MCX_CUDA(s, cudaStreamSynchronize(st), "waiting for the copy");
    return MCX_OK;
}

extern "C" {

mcx_status mcx_read_fluence(mcx_sim *s, float *dst, uint64_t n_elems, int32_t normalized,
                            int32_t dst_on_device)
{
    return read_fluence_t<float>(s, dst, n_elems, normalized, dst_on_device);
}

mcx_status mcx_read_fluence64(mcx_sim *s, double *dst, uint64_t n_elems, int32_t normalized,
                              int32_t dst_on_device)
{
    return read_fluence_t<double>(s, dst, n_elems, normalized, dst_on_device);
}

int32_t mcx_detected_stride(const mcx_sim *s)
{
    if (!s) return 0;
    return kRecBase + (int)(s->n_media > 0 ? s->n_media : 1) - 1;
}

mcx_status mcx_read_detected(mcx_sim *s, void *dst, uint64_t cap, uint64_t *n_written,
                             uint64_t *n_total)
{
    if (!s) return fail(nullptr, MCX_E_ARG, "sim is NULL");
    if (!dst && cap > 0) return fail(s, MCX_E_ARG, "dst is NULL");
    DeviceGuard g(s->device);
    mcx_status st0 = wait_done(s);
    if (st0 != MCX_OK) return st0;
    unsigned long long ctrl[2];
    MCX_CUDA(s, cudaMemcpy(ctrl, s->ctrl.p, sizeof(ctrl), cudaMemcpyDeviceToHost), "reading the count");
    const bool has_det = !s->det.empty();
    const uint64_t total = has_det ? ctrl[1] : 0;
    const uint64_t stored = std::min<uint64_t>(total, has_det ? s->cfg.max_detected : 0);
    const uint64_t nw = std::min<uint64_t>(stored, cap);
    if (n_total) *n_total = total;
    if (n_written) *n_written = nw;
    if (nw == 0) return MCX_OK;
    const int stride = s->rec_stride;
    uint64_t np2 = 1;
    while (np2 < stored) np2 <<= 1;
    MCX_CUDA(s, s->sort_keys.ensure(np2 * 8), "allocating sort keys");
    MCX_CUDA(s, s->sort_vals.ensure(np2 * 4), "allocating sort values");
    MCX_CUDA(s, s->staging.ensure(stored * stride * sizeof(float)), "allocating staging");
    unsigned long long *keys = s->sort_keys.as<unsigned long long>();
    unsigned *vals = s->sort_vals.as<unsigned>();
    const unsigned gb = (unsigned)((np2 + 255) / 256);
    det_keys_kernel<<<gb, 256>>>(s->det_buf.as<float>(), stride, stored, np2, keys, vals);
    for (uint64_t k = 2; k <= np2; k <<= 1)
        for (uint64_t j = k >> 1; j > 0; j >>= 1) bitonic_step<<<gb, 256>>>(keys, vals, j, k, np2);
    const uint64_t words = nw * stride;
    det_gather_kernel<<<(unsigned)((words + 255) / 256), 256>>>(s->det_buf.as<float>(), vals, stride,
                                                                 nw, s->staging.as<float>());
    MCX_CUDA(s, cudaGetLastError(), "ordering detected records");
    MCX_CUDA(s, cudaMemcpy(dst, s->staging.p, words * sizeof(float), cudaMemcpyDeviceToHost),
             "copying detected records");
    return MCX_OK;
}

mcx_status mcx_read_tally(mcx_sim *s, double out[MCX_NTALLY])
{
    if (!s || !out) return fail(s, MCX_E_ARG, "NULL argument");
    DeviceGuard g(s->device);
    mcx_status st = wait_done(s);
    if (st != MCX_OK) return st;
    MCX_CUDA(s, cudaMemcpy(out, s->out.p, MCX_NTALLY * sizeof(double), cudaMemcpyDeviceToHost),
             "reading tallies");
    return MCX_OK;
}

mcx_status mcx_read_stats(mcx_sim *s, uint64_t out[MCX_NSTAT])
{
    if (!s || !out) return fail(s, MCX_E_ARG, "NULL argument");
    DeviceGuard g(s->device);
    mcx_status st = wait_done(s);
    if (st != MCX_OK) return st;
    MCX_CUDA(s, cudaMemcpy(out, s->out.as<double>() + MCX_NTALLY, MCX_NSTAT * 8,
                           cudaMemcpyDeviceToHost), "reading counters");
    return MCX_OK;
}

mcx_status mcx_read_exits(mcx_sim *s, mcx_exit *dst, uint64_t cap, uint64_t *n_written)
{
    if (!s) return fail(nullptr, MCX_E_ARG, "sim is NULL");
    if (!dst && cap > 0) return fail(s, MCX_E_ARG, "dst is NULL");
    DeviceGuard g(s->device);
    mcx_status st = wait_done(s);
    if (st != MCX_OK) return st;
    const uint64_t n = std::min<uint64_t>(cap, s->cfg.exit_log);
    if (n_written) *n_written = n;
    if (n) MCX_CUDA(s, cudaMemcpy(dst, s->exits.p, n * sizeof(mcx_exit), cudaMemcpyDeviceToHost),
                    "reading the exit log");
    return MCX_OK;
}

mcx_status mcx_launch_info(mcx_sim *s, int32_t out[4])
{
    if (!s || !out) return fail(s, MCX_E_ARG, "NULL argument");
    if (!s->ran) return fail(s, MCX_E_STATE, "no run");
    out[0] = s->shape.grid;
    out[1] = s->shape.block;
    out[2] = s->shape.blocks_per_sm;
    out[3] = s->shape.regs;
    return MCX_OK;
}

const char *mcx_last_error(const mcx_sim *s) { return s ? s->err.c_str() : g_err.c_str(); }

void mcx_destroy(mcx_sim *s)
{
    if (!s) return;
    DeviceGuard g(s->device);
    if (s->ran) cudaEventSynchronize(s->ev_done);
    for (DevBuf *b : {&s->labels, &s->fluence, &s->fluence64, &s->tables,
                      &s->detb, &s->det_buf, &s->exits,
                      &s->block_tally, &s->block_stats, &s->ctrl, &s->out, &s->staging,
                      &s->inv_norm, &s->sort_keys, &s->sort_vals})
        b->release();
    if (s->ev_start) cudaEventDestroy(s->ev_start);
    if (s->ev_stop) cudaEventDestroy(s->ev_stop);
    if (s->ev_done) cudaEventDestroy(s->ev_done);
    delete s;
}

mcx_status mcx_debug_uniforms(uint64_t seed, uint64_t photon, uint64_t n, float *out_host)
{
    if (!out_host && n) return fail(nullptr, MCX_E_ARG, "out is NULL");
    if (n == 0) return MCX_OK;
    float *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 5 * n * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "allocating");
    e = debug_uniforms(seed, photon, n, d);
    if (e == cudaSuccess) e = cudaMemcpy(out_host, d, 5 * n * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? MCX_OK : cuda_fail(nullptr, e, "debug uniforms");
}

mcx_status mcx_debug_primitive(int32_t kind, uint64_t n, const float *in, float *out)
{
    if (kind < 0 || kind > 2) return fail(nullptr, MCX_E_ARG, "kind is 0, 1 or 2");
    if (n == 0) return MCX_OK;
    if (!in || !out) return fail(nullptr, MCX_E_ARG, "NULL argument");
    const int nin = kind == 0 ? 2 : (kind == 1 ? 6 : 3);
    const int nout = kind == 1 ? 3 : (kind == 0 ? 2 : 1);
    float *din = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&din, n * nin * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dout, n * nout * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(din, in, n * nin * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = debug_primitive(kind, n, din, dout);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, n * nout * sizeof(float), cudaMemcpyDeviceToHost);
    if (din) cudaFree(din);
    if (dout) cudaFree(dout);
    return e == cudaSuccess ? MCX_OK : cuda_fail(nullptr, e, "debug primitive");
}

}  // extern "C"
