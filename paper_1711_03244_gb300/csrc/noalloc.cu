// mcx_run_noalloc: one simulation that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: applications that hand all device
// memory to their own pool or caching allocator (memory the library grabs behind the
// pool's back is invisible to it and fragments it), and latency-sensitive loops that
// cannot afford the device-wide synchronisation cudaFree may cause.  This entry point
// runs the same walk kernel as mcx_run on the caller's device buffers (labels in,
// fluence and tallies out) and keeps its own working memory (photon-claim counter,
// status word, per-label tables, per-block tally and event-count partials) in the fixed
// array below.
//
// The array lives in every GPU that loads this library, for the life of the process.
// Its device address is looked up once per device, on that device's first call.  Every
// call reuses it and re-initialises what must start at zero, so two calls whose work
// overlaps on the GPU (different streams, or different host threads, same device) race
// on it and corrupt each other's results: serialise calls per device.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "mcx_internal.h"

namespace mcxg {
namespace {

// Limits of the fixed working memory.
constexpr int kNaMaxMedia = 32;          // media rows (label values 0..31)
constexpr int kNaMaxBlocks = 2048;       // persistent blocks per run
constexpr size_t kNaCtrl = 0;            // photon counter, det count, status, label flag
constexpr size_t kNaTables = 256;        // per-label tables (FP32 layout)
constexpr size_t kNaTableBytes = 2048;
constexpr size_t kNaTally = kNaTables + kNaTableBytes;
constexpr size_t kNaStats = kNaTally + sizeof(double) * MCX_NTALLY * kNaMaxBlocks;
constexpr size_t kNaBytes = kNaStats + sizeof(unsigned long long) * MCX_NSTAT * kNaMaxBlocks;

static __device__ __align__(256) unsigned char g_scratch[kNaBytes];

struct TableImage {                      // the tables, passed by value to the set-up kernel
    unsigned char bytes[kNaTableBytes];
};

// Copies the per-label tables into the working memory and clears the counters.
__global__ void na_setup(unsigned char *scratch, const TableImage img, unsigned table_bytes)
{
    for (unsigned i = threadIdx.x; i < table_bytes; i += blockDim.x)
        scratch[kNaTables + i] = img.bytes[i];
    if (threadIdx.x < 8) reinterpret_cast<unsigned long long *>(scratch + kNaCtrl)[threadIdx.x] = 0ull;
}

// Flags any label without a media row.
__global__ void na_check_labels(const uint8_t *labels, size_t n, unsigned n_media, unsigned *flag)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    unsigned bad = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride)
        bad |= labels[i] >= n_media;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

template <typename T>
__global__ void na_zero(T *p, size_t n)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) p[i] = T(0);
}

// Sums the block partials (fixed order) into the caller's tally output, and the blocks'
// counts of photons stopped by the per-photon event cap into its last word.
__global__ void na_finalize(const double *bt, const unsigned long long *bs, int nblocks,
                            double n_launched, double *out)
{
    __shared__ double st[256][MCX_NTALLY + 1];
    const int tid = threadIdx.x;
    double t[MCX_NTALLY + 1] = {0};
    for (int b = tid; b < nblocks; b += blockDim.x) {
        for (int k = 0; k < MCX_NTALLY; ++k) t[k] += bt[(size_t)b * MCX_NTALLY + k];
        t[MCX_NTALLY] += (double)bs[(size_t)b * MCX_NSTAT + MCX_STAT_CAPPED];
    }
    for (int k = 0; k <= MCX_NTALLY; ++k) st[tid][k] = t[k];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (tid < h)
            for (int k = 0; k <= MCX_NTALLY; ++k) st[tid][k] += st[tid + h][k];
        __syncthreads();
    }
    if (tid == 0) {
        for (int k = 0; k <= MCX_NTALLY; ++k) out[k] = st[0][k];
        out[MCX_TALLY_LAUNCHED] = n_launched;
    }
}

// Per-device device address of g_scratch and walk launch shape, set up once.
struct DeviceState {
    bool ready = false;
    unsigned char *scratch = nullptr;
    LaunchShape shape{};
    int shape_block = 0;
    int shape_accum = -1;
};
constexpr int kMaxDevices = 64;
DeviceState g_dev[kMaxDevices];
std::mutex g_mu;

mcx_status na_fail(mcx_status st, const std::string &m)
{
    set_global_error(m);          // readable with mcx_last_error(NULL)
    return st;
}

// True when p is device (or managed) memory that the current device `dev` can use.
bool device_pointer(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();         // the failed query leaves its error behind; clear it
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) &&
           (a.type == cudaMemoryTypeManaged || a.device == dev);
}

}  // namespace
}  // namespace mcxg

using namespace mcxg;

extern "C" mcx_status mcx_run_noalloc(const uint8_t *labels_dev, uint32_t nx, uint32_t ny,
                                      uint32_t nz, float voxel_mm, uint32_t n_media,
                                      const float *props, int32_t src_kind, const float pos_mm[3],
                                      const float dir[3], float waist_mm, const mcx_run_cfg *cfg,
                                      void *fluence_dev, double *tally_dev)
{
    // ---- arguments and limits (nothing is touched on an error)
    if (!labels_dev || !props || !pos_mm || !dir || !cfg || !fluence_dev || !tally_dev)
        return na_fail(MCX_E_ARG, "mcx_run_noalloc: NULL argument");
    if (cfg->struct_size != sizeof(mcx_run_cfg))
        return na_fail(MCX_E_ARG, "mcx_run_noalloc: cfg->struct_size does not match this library");
    if (nx == 0 || ny == 0 || nz == 0 || (uint64_t)nx * ny * nz >= (1ull << 32))
        return na_fail(MCX_E_ARG, "mcx_run_noalloc: need 0 < nx*ny*nz < 2^32");
    if (!(voxel_mm > 0.f) || !std::isfinite(voxel_mm))
        return na_fail(MCX_E_ARG, "mcx_run_noalloc: voxel_mm must be positive");
    if (n_media < 1 || n_media > (uint32_t)kNaMaxMedia)
        return na_fail(MCX_E_ARG, "mcx_run_noalloc: n_media must be 1.." +
                                      std::to_string(kNaMaxMedia) + " (fixed working memory)");
    for (uint32_t m = 0; m < n_media; ++m) {
        const float *r = props + 4 * m;
        const bool ok = m == 0 ? (r[3] > 0.f && std::isfinite(r[3]))
                               : (r[0] >= 0.f && r[1] >= 0.f && std::fabs(r[2]) < 1.f && r[3] > 0.f &&
                                  std::isfinite(r[0]) && std::isfinite(r[1]) && std::isfinite(r[3]));
        if (!ok) return na_fail(MCX_E_ARG, "mcx_run_noalloc: bad media row " + std::to_string(m));
    }
    const double dn = std::sqrt((double)dir[0] * dir[0] + (double)dir[1] * dir[1] + (double)dir[2] * dir[2]);
    if ((src_kind != 0 && src_kind != 1) || !(dn > 0.0) || (src_kind == 1 && !(waist_mm > 0.f)))
        return na_fail(MCX_E_ARG, "mcx_run_noalloc: bad source");
    if (cfg->n_gates < 1 || !(cfg->dt_ns > 0.f) || !std::isfinite(cfg->dt_ns) ||
        !std::isfinite((float)((double)cfg->dt_ns * cfg->n_gates)))
        return na_fail(MCX_E_ARG, "mcx_run_noalloc: need n_gates >= 1 and a finite dt_ns > 0");
    if (!(cfg->rr_threshold >= 0.f) || (cfg->rr_threshold > 0.f && !(cfg->rr_m > 1.f)))
        return na_fail(MCX_E_ARG, "mcx_run_noalloc: need rr_threshold >= 0 and rr_m > 1");
    if (cfg->photon_offset + cfg->n_photons < cfg->photon_offset)
        return na_fail(MCX_E_ARG, "mcx_run_noalloc: photon id range overflows");
    if (cfg->precision != 0 || (cfg->accum_mode != 0 && cfg->accum_mode != 2) ||
        cfg->exit_log != 0 || cfg->max_detected != 0)
        return na_fail(MCX_E_ARG, "mcx_run_noalloc: need precision 0, accum_mode 0 or 2, "
                                  "exit_log 0, max_detected 0");
    const int block = cfg->block_size ? cfg->block_size : 256;
    if (block < 32 || block > 256 || block % 32)
        return na_fail(MCX_E_ARG, "mcx_run_noalloc: block_size 32..256, multiple of 32");
    if (cfg->grid_size < 0 || cfg->grid_size > kNaMaxBlocks)
        return na_fail(MCX_E_ARG, "mcx_run_noalloc: grid_size above the fixed limit of " +
                                      std::to_string(kNaMaxBlocks) + " blocks");
    if (walk_table_bytes(Precision::F32, (int)n_media) > kNaTableBytes)
        return na_fail(MCX_E_ARG, "mcx_run_noalloc: media tables exceed the fixed working memory");

    // ---- once per device: device address of the working memory and the launch shape
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return na_fail(MCX_E_CUDA, "mcx_run_noalloc: no usable CUDA device");
    cudaStream_t stream = static_cast<cudaStream_t>(cfg->cuda_stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        (void)cudaGetLastError();
        return na_fail(MCX_E_STATE, "mcx_run_noalloc: cannot run inside stream capture (the label "
                                    "check waits for the stream)");
    }
    if (!device_pointer(labels_dev, dev) || !device_pointer(fluence_dev, dev) ||
        !device_pointer(tally_dev, dev))
        return na_fail(MCX_E_ARG, "mcx_run_noalloc: labels_dev, fluence_dev and tally_dev must "
                                  "be device memory of the current device");
    const int accum = cfg->accum_mode == 2 ? kAccF64 : kAccPlain;
    DeviceState st;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        DeviceState &d = g_dev[dev];
        if (!d.ready) {
            void *ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess)
                return na_fail(MCX_E_CUDA, std::string("mcx_run_noalloc: cudaGetSymbolAddress: ") +
                                               cudaGetErrorString(e));
            d.scratch = static_cast<unsigned char *>(ptr);
            d.ready = true;
        }
        if (d.shape_block != block || d.shape_accum != accum) {
            const cudaError_t e = walk_query_shape_unpadded(accum, block, &d.shape);
            if (e != cudaSuccess)
                return na_fail(MCX_E_CUDA, std::string("mcx_run_noalloc: ") + cudaGetErrorString(e));
            d.shape_block = block;
            d.shape_accum = accum;
        }
        st = d;
    }
    LaunchShape shape = st.shape;
    if (cfg->grid_size > 0) shape.grid = cfg->grid_size;
    if (shape.grid > kNaMaxBlocks) shape.grid = kNaMaxBlocks;
    unsigned char *scratch = st.scratch;

    // ---- tables (host set-up arithmetic), then the labels check
    TableImage img;
    std::memset(img.bytes, 0, sizeof(img.bytes));
    const void *oa, *ob, *on, *ot;
    walk_fill_tables(Precision::F32, (int)n_media, props, voxel_mm, img.bytes, &oa, &ob, &on, &ot);
    const unsigned tb = (unsigned)walk_table_bytes(Precision::F32, (int)n_media);
    na_setup<<<1, 256, 0, stream>>>(scratch, img, tb);
    unsigned *ctrl32 = reinterpret_cast<unsigned *>(scratch + kNaCtrl);
    const size_t nvox = (size_t)nx * ny * nz;
    na_check_labels<<<(unsigned)std::min<size_t>((nvox + 255) / 256, 1024), 256, 0, stream>>>(
        labels_dev, nvox, n_media, ctrl32 + 6);
    unsigned flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, ctrl32 + 6, sizeof(unsigned), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess)
        return na_fail(MCX_E_CUDA, std::string("mcx_run_noalloc: ") + cudaGetErrorString(e));
    if (flag) return na_fail(MCX_E_STATE, "mcx_run_noalloc: the volume has a label >= n_media");

    // ---- zero the caller's fluence, walk, reduce the tallies into the caller's output
    const size_t nflu = nvox * cfg->n_gates;
    const unsigned zblocks = (unsigned)std::min<size_t>((nflu + 255) / 256, 152u * 16u);
    if (accum == kAccF64)
        na_zero<<<zblocks, 256, 0, stream>>>(static_cast<double *>(fluence_dev), nflu);
    else
        na_zero<<<zblocks, 256, 0, stream>>>(static_cast<float *>(fluence_dev), nflu);

    WalkParams p{};
    p.labels = labels_dev;
    if (accum == kAccF64) p.fluence64 = static_cast<double *>(fluence_dev);
    else p.fluence = static_cast<float *>(fluence_dev);
    p.tab_a = scratch + kNaTables + (size_t)oa;
    p.tab_b = scratch + kNaTables + (size_t)ob;
    p.tab_n = scratch + kNaTables + (size_t)on;
    p.tab_tpl = scratch + kNaTables + (size_t)ot;
    unsigned long long *ctrl = reinterpret_cast<unsigned long long *>(scratch + kNaCtrl);
    p.photon_counter = ctrl;
    p.det_count = ctrl + 1;
    p.status = reinterpret_cast<unsigned *>(ctrl + 2);
    p.block_tally = reinterpret_cast<double *>(scratch + kNaTally);
    p.block_stats = reinterpret_cast<unsigned long long *>(scratch + kNaStats);
    p.nx = (int)nx; p.ny = (int)ny; p.nz = (int)nz;
    p.nvox = (unsigned)nvox;                       // the caller's unpadded layout
    p.sy = nx;
    p.sz = nx * ny;
    p.n_media = (int)n_media;
    p.n_det = 0;
    p.rec_stride = kRecBase + (int)n_media - 1;
    p.n_gates = cfg->n_gates;
    p.h = voxel_mm;
    RunConsts<float> &c = p.cf;
    c.dt = cfg->dt_ns;
    c.inv_dt = (float)(1.0 / (double)cfg->dt_ns);
    c.t_end = (float)((double)cfg->dt_ns * cfg->n_gates);
    const double d[3] = {dir[0] / dn, dir[1] / dn, dir[2] / dn};
    double e1[3], e2[3];
    launch_plane(d, e1, e2);
    for (int a = 0; a < 3; ++a) {
        c.src_pos[a] = (float)((double)pos_mm[a] / voxel_mm);
        c.src_dir[a] = (float)d[a];
        c.src_e1[a] = (float)e1[a];
        c.src_e2[a] = (float)e2[a];
    }
    c.waist = (float)((double)waist_mm / voxel_mm);
    c.rr_threshold = cfg->rr_threshold;
    c.rr_m = cfg->rr_m;
    c.rr_inv_m = cfg->rr_threshold > 0.f ? (float)(1.0 / (double)cfg->rr_m) : 0.f;
    p.src_kind = src_kind;
    p.n_photons = cfg->n_photons;
    p.photon_offset = cfg->photon_offset;
    p.seed = cfg->seed;
    p.max_events = cfg->max_events_per_photon ? cfg->max_events_per_photon : 100000000ull;
    p.reflect = cfg->reflect;
    p.claim_chunk = kClaimChunk;

    e = walk_launch_unpadded(p, accum, shape, stream);
    if (e != cudaSuccess)
        return na_fail(MCX_E_CUDA, std::string("mcx_run_noalloc: walk launch: ") + cudaGetErrorString(e));
    na_finalize<<<1, 256, 0, stream>>>(p.block_tally, p.block_stats, shape.grid,
                                        (double)cfg->n_photons, tally_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return na_fail(MCX_E_CUDA, std::string("mcx_run_noalloc: ") + cudaGetErrorString(e));
    return MCX_OK;
}
