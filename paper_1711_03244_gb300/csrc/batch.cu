// Batched simulations (include/mcx.h, mcx_batch_*): many independent problems in one
// persistent launch of the walk kernel, with their photons in one queue, optionally
// recorded once as a CUDA graph and replayed, and an autotuner for the launch shape.
//
// The paper balances photons across the threads of a workgroup and across devices
// (Fig. 3 and the paragraphs on load balancing); a batch carries that balancing across
// problems: a warp that finishes its simulation's last photons claims the next
// simulation's first ones, so many small problems fill the GPU the way one large one does.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <tuple>
#include <vector>

#include "mcx_internal.h"

using namespace mcxg;

namespace {

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t want)
    {
        if (want <= bytes && p) return cudaSuccess;
        release();
        if (want == 0) return cudaSuccess;
        const cudaError_t e = cudaMalloc(&p, want);
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

__global__ void batch_zero(uint32_t *p, size_t n)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) p[i] = 0u;
}

// sums the per-block event counters of the batch run (fixed order)
__global__ void batch_stats(const unsigned long long *bs, int nblocks, unsigned long long *out)
{
    __shared__ unsigned long long ss[256][MCX_NSTAT];
    const int tid = threadIdx.x;
    unsigned long long c[MCX_NSTAT] = {0};
    for (int b = tid; b < nblocks; b += blockDim.x)
        for (int k = 0; k < MCX_NSTAT; ++k) c[k] += bs[(size_t)b * MCX_NSTAT + k];
    for (int k = 0; k < MCX_NSTAT; ++k) ss[tid][k] = c[k];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (tid < h)
            for (int k = 0; k < MCX_NSTAT; ++k) ss[tid][k] += ss[tid + h][k];
        __syncthreads();
    }
    if (tid == 0)
        for (int k = 0; k < MCX_NSTAT; ++k) out[k] = ss[0][k];
}

// one simulation's map as float [g][nz][ny][nx], optionally normalised per launched
// photon; the map and the labels carry the walk's one-voxel border
__global__ void batch_resolve(const float *f32, const double *f64, const uint8_t *labels,
                              const float *inv_norm, unsigned nx, unsigned ny, unsigned nvox,
                              unsigned pnvox, size_t n, float *out)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned v = (unsigned)(i % nvox), g = (unsigned)(i / nvox);
        const unsigned pv = (unsigned)padded_index(v % nx, (v / nx) % ny, v / (nx * ny), nx, ny);
        const size_t pi = (size_t)g * pnvox + pv;
        double x = f64 ? f64[pi] : (double)f32[pi];
        if (inv_norm) x *= (double)inv_norm[labels[pv]];
        out[i] = (float)x;
    }
}

unsigned grid_of(size_t n)
{
    size_t g = (n + 255) / 256;
    return (unsigned)std::max<size_t>(1, std::min<size_t>(g, 152u * 16u));
}

struct SimHost {
    uint32_t nx, ny, nz;
    float h;
    uint32_t n_media;
    std::vector<float> props;
    int kind;
    double pos[3], dir[3], waist;
    uint64_t n_photons, seed;
    std::vector<double> frac;     // volume fraction of each label
    Buf labels;
};

// Expected work of the longest photon histories of a simulation, for ordering the queue
// (a scheduling heuristic, not part of the method).  Per label: photons are lost at the
// rate mua + pi^2 / (L^2 mus') per unit path (absorption, and escape by diffusion from a
// cube of the grid's mean side L: the slowest mode's loss rate, mus' = mus (1 - g)), so the
// longest of N photons travels about ln(N) / rate, or up to the time window; times the
// events per unit path (scatterings mus and voxel crossings 1 / h), weighted by the label's
// volume fraction.  Starting these photons first keeps them out of the launch's tail.
double photon_cost(const SimHost *s, uint32_t n_gates, float dt_ns)
{
    const double L = s->h * (s->nx + s->ny + s->nz) / 3.0;
    const double ln_n = std::log(std::max<double>((double)s->n_photons, 2.0));
    double c = 0.0;
    for (uint32_t l = 1; l < s->n_media && l < s->frac.size(); ++l) {
        if (s->frac[l] <= 0.0) continue;
        const double mua = s->props[4 * l], mus = s->props[4 * l + 1], g = s->props[4 * l + 2];
        const double n = s->props[4 * l + 3], musp = std::max(mus * (1.0 - g), 1e-6);
        const double rate = mua + 9.8696044 / (L * L * musp);
        const double path = std::min(ln_n / std::max(rate, 1e-9), 299.792458 / n * n_gates * dt_ns);
        c += s->frac[l] * path * (mus + 1.0 / s->h);
    }
    return c;
}

}  // namespace

struct mcx_batch {
    int device = 0;
    std::vector<SimHost *> sims;
    Buf fluence, descs, descs_tune, tab_a, tab_b, tab_n, tab_tpl, tallies, ctrl, block_tally,
        block_stats, out_stats, staging, inv_norm;
    std::vector<BatchSim> host_descs;
    std::vector<uint64_t> flu_off;          // element offset of each simulation's map
    bool dirty = true;
    // last run
    bool ran = false;
    mcx_batch_cfg cfg{};
    LaunchShape shape{};
    cudaStream_t stream = nullptr, own_stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // recorded run
    cudaGraphExec_t graph = nullptr;
    std::tuple<int, int, int, int, uint32_t, float, int, float, float, uint64_t, void *> graph_key;
    std::string err;
};

static mcx_status bfail(mcx_batch *b, mcx_status st, const std::string &m)
{
    if (b) b->err = m; else set_global_error(m);
    return st;
}

#define BCUDA(b, call, what)                                                                  \
    do {                                                                                      \
        const cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                                \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? MCX_E_OOM : MCX_E_CUDA,       \
                         std::string(what) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

static void drop_graph(mcx_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

extern "C" {

void mcx_batch_cfg_default(mcx_batch_cfg *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->struct_size = sizeof(mcx_batch_cfg);
    c->n_gates = 1;
    c->dt_ns = 5.f;
    c->reflect = 1;
    c->rr_threshold = 1e-4f;
    c->rr_m = 10.f;
    c->accum_mode = 2;
    c->order = 1;
}

mcx_status mcx_batch_create(mcx_batch **out)
{
    if (!out) return bfail(nullptr, MCX_E_ARG, "out is NULL");
    *out = nullptr;
    mcx_batch *b = new (std::nothrow) mcx_batch();
    if (!b) return bfail(nullptr, MCX_E_OOM, "host allocation failed");
    if (cudaGetDevice(&b->device) != cudaSuccess || cudaEventCreate(&b->ev0) != cudaSuccess ||
        cudaEventCreate(&b->ev1) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        mcx_batch_destroy(b);
        return bfail(nullptr, MCX_E_CUDA, "no usable CUDA device");
    }
    *out = b;
    return MCX_OK;
}

int32_t mcx_batch_size(const mcx_batch *b) { return b ? (int32_t)b->sims.size() : 0; }

const char *mcx_batch_last_error(const mcx_batch *b) { return b ? b->err.c_str() : ""; }

mcx_status mcx_batch_add(mcx_batch *b, uint32_t nx, uint32_t ny, uint32_t nz, float voxel_mm,
                         const uint8_t *labels, int32_t on_device, uint32_t n_media,
                         const float *props, int32_t kind, const float pos[3], const float dir[3],
                         float waist, uint64_t n_photons, uint64_t seed, int32_t *out_id)
{
    if (!b) return bfail(nullptr, MCX_E_ARG, "batch is NULL");
    if (!labels || !props || !pos || !dir) return bfail(b, MCX_E_ARG, "NULL argument");
    if (nx == 0 || ny == 0 || nz == 0 || (uint64_t)(nx + 2ull) * (ny + 2ull) * (nz + 2ull) >= (1ull << 32))
        return bfail(b, MCX_E_ARG, "need nx, ny, nz > 0 and (nx+2)(ny+2)(nz+2) < 2^32");
    if (!(voxel_mm > 0.f) || n_media < 1 || n_media > (uint32_t)kMaxMedia)
        return bfail(b, MCX_E_ARG, "bad voxel size or media count");
    for (uint32_t m = 0; m < n_media; ++m) {
        const float *r = props + 4 * m;
        const bool ok = m == 0 ? r[3] > 0.f
                               : (r[0] >= 0.f && r[1] >= 0.f && std::fabs(r[2]) < 1.f && r[3] > 0.f);
        if (!ok) return bfail(b, MCX_E_ARG, "bad media row " + std::to_string(m));
    }
    const double dn = std::sqrt((double)dir[0] * dir[0] + (double)dir[1] * dir[1] + (double)dir[2] * dir[2]);
    if ((kind != 0 && kind != 1) || !(dn > 0.0) || (kind == 1 && !(waist > 0.f)))
        return bfail(b, MCX_E_ARG, "bad source");
    SimHost *s = new (std::nothrow) SimHost();
    if (!s) return bfail(b, MCX_E_OOM, "host allocation failed");
    s->nx = nx; s->ny = ny; s->nz = nz; s->h = voxel_mm; s->n_media = n_media;
    s->props.assign(props, props + 4 * n_media);
    s->kind = kind;
    for (int a = 0; a < 3; ++a) { s->pos[a] = pos[a]; s->dir[a] = dir[a] / dn; }
    s->waist = waist;
    s->n_photons = n_photons;
    s->seed = seed;
    const size_t nv = (size_t)nx * ny * nz;
    // every label must have a media row
    std::vector<uint8_t> host(nv);
    if (on_device) {
        if (cudaMemcpy(host.data(), labels, nv, cudaMemcpyDeviceToHost) != cudaSuccess) {
            delete s;
            return bfail(b, MCX_E_ARG, "labels_on_device = 1 but labels is not device memory");
        }
    } else {
        std::memcpy(host.data(), labels, nv);
    }
    const uint8_t mx = *std::max_element(host.begin(), host.end());
    if (mx >= n_media) {
        delete s;
        return bfail(b, MCX_E_STATE, "the volume has a label without a media row");
    }
    s->frac.assign(n_media, 0.0);
    for (const uint8_t l : host) s->frac[l] += 1.0;
    for (double &f : s->frac) f /= (double)nv;
    // the device copy carries a one-voxel exterior border (label 0) on every side
    const size_t np = (size_t)(nx + 2) * (ny + 2) * (nz + 2);
    std::vector<uint8_t> padded(np, 0);
    for (uint32_t z = 0; z < nz; ++z)
        for (uint32_t y = 0; y < ny; ++y)
            std::memcpy(padded.data() + padded_index(0, y, z, nx, ny), host.data() + ((size_t)z * ny + y) * nx, nx);
    if (s->labels.ensure(np) != cudaSuccess ||
        cudaMemcpy(s->labels.p, padded.data(), np, cudaMemcpyHostToDevice) != cudaSuccess) {
        delete s;
        return bfail(b, MCX_E_OOM, "allocating the label volume");
    }
    b->sims.push_back(s);
    b->dirty = true;
    b->ran = false;
    drop_graph(b);
    if (out_id) *out_id = (int32_t)b->sims.size() - 1;
    return MCX_OK;
}

}  // extern "C"

// Lays out the batch on the device for `cfg` (maps, tables, descriptors); photon counts
// scaled by `fraction` go to `dst` (the run's descriptors or the autotuner's).
static mcx_status layout(mcx_batch *b, const mcx_batch_cfg *cfg, double fraction, Buf &dst,
                         uint64_t *total_out)
{
    const size_t n = b->sims.size();
    const size_t elt = cfg->accum_mode == kAccF64 ? sizeof(double) : sizeof(float);
    uint64_t vox_total = 0;
    b->flu_off.assign(n, 0);
    int rows = 0;
    for (size_t i = 0; i < n; ++i) {
        b->flu_off[i] = vox_total * cfg->n_gates;
        vox_total += (uint64_t)(b->sims[i]->nx + 2) * (b->sims[i]->ny + 2) * (b->sims[i]->nz + 2);
        rows += (int)b->sims[i]->n_media;
    }
    BCUDA(b, b->fluence.ensure(vox_total * cfg->n_gates * elt), "allocating the batch fluence maps");
    BCUDA(b, b->tallies.ensure(std::max<size_t>(n, 1) * MCX_NTALLY * sizeof(double)), "allocating");
    // tables: every simulation's rows, concatenated table by table
    std::vector<unsigned char> A(16 * (size_t)rows), B(16 * (size_t)rows), N(4 * (size_t)rows),
        T(4 * (size_t)rows);
    std::vector<unsigned char> tmp;
    // queue order: as added, or the longest expected photon histories first (their
    // photons then start early instead of forming the tail of the launch)
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; ++i) order[i] = i;
    if (cfg->order == 1) {
        std::vector<double> cost(n);
        for (size_t i = 0; i < n; ++i) cost[i] = photon_cost(b->sims[i], cfg->n_gates, cfg->dt_ns);
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t c) { return cost[a] > cost[c]; });
    }
    std::vector<size_t> slot(n);
    for (size_t k = 0; k < n; ++k) slot[order[k]] = k;
    std::vector<BatchSim> d(n);
    int row = 0;
    for (size_t i = 0; i < n; ++i) {
        const SimHost *s = b->sims[i];
        tmp.assign(walk_table_bytes(Precision::F32, (int)s->n_media), 0);
        const void *oa, *ob, *on, *ot;
        walk_fill_tables(Precision::F32, (int)s->n_media, s->props.data(), s->h, tmp.data(), &oa,
                         &ob, &on, &ot);
        std::memcpy(&A[16 * (size_t)row], tmp.data() + (size_t)oa, 16 * s->n_media);
        std::memcpy(&B[16 * (size_t)row], tmp.data() + (size_t)ob, 16 * s->n_media);
        std::memcpy(&N[4 * (size_t)row], tmp.data() + (size_t)on, 4 * s->n_media);
        std::memcpy(&T[4 * (size_t)row], tmp.data() + (size_t)ot, 4 * s->n_media);
        BatchSim &D = d[slot[i]];
        D.labels = s->labels.as<uint8_t>();
        D.fluence = elt == sizeof(float) ? b->fluence.as<float>() + b->flu_off[i] : nullptr;
        D.fluence64 = elt == sizeof(double) ? b->fluence.as<double>() + b->flu_off[i] : nullptr;
        D.tally = b->tallies.as<double>() + i * MCX_NTALLY;
        D.n_photons = fraction >= 1.0 ? s->n_photons
                                      : (uint64_t)std::max(1.0, std::round((double)s->n_photons * fraction));
        if (s->n_photons == 0) D.n_photons = 0;
        D.seed = s->seed;
        D.nx = (int)s->nx; D.ny = (int)s->ny; D.nz = (int)s->nz;
        D.nvox = (s->nx + 2) * (s->ny + 2) * (s->nz + 2);
        D.sy = s->nx + 2;
        D.sz = (s->nx + 2) * (s->ny + 2);
        D.tab0 = row;
        D.src_kind = s->kind;
        double e1[3], e2[3];
        launch_plane(s->dir, e1, e2);
        for (int a = 0; a < 3; ++a) {
            D.src_pos[a] = (float)(s->pos[a] / s->h);
            D.src_dir[a] = (float)s->dir[a];
            D.src_e1[a] = (float)e1[a];
            D.src_e2[a] = (float)e2[a];
        }
        D.waist = (float)(s->waist / s->h);
        row += (int)s->n_media;
    }
    uint64_t first = 0;                       // flattened photon ids, in queue order
    for (size_t k = 0; k < n; ++k) {
        d[k].first = first;
        first += d[k].n_photons;
    }
    BCUDA(b, b->tab_a.ensure(A.size()), "allocating tables");
    BCUDA(b, b->tab_b.ensure(B.size()), "allocating tables");
    BCUDA(b, b->tab_n.ensure(N.size()), "allocating tables");
    BCUDA(b, b->tab_tpl.ensure(T.size()), "allocating tables");
    BCUDA(b, cudaMemcpy(b->tab_a.p, A.data(), A.size(), cudaMemcpyHostToDevice), "uploading tables");
    BCUDA(b, cudaMemcpy(b->tab_b.p, B.data(), B.size(), cudaMemcpyHostToDevice), "uploading tables");
    BCUDA(b, cudaMemcpy(b->tab_n.p, N.data(), N.size(), cudaMemcpyHostToDevice), "uploading tables");
    BCUDA(b, cudaMemcpy(b->tab_tpl.p, T.data(), T.size(), cudaMemcpyHostToDevice), "uploading tables");
    BCUDA(b, dst.ensure(std::max<size_t>(n, 1) * sizeof(BatchSim)), "allocating descriptors");
    BCUDA(b, cudaMemcpy(dst.p, d.data(), n * sizeof(BatchSim), cudaMemcpyHostToDevice),
          "uploading descriptors");
    if (&dst == &b->descs) b->host_descs = d;
    *total_out = first;
    return MCX_OK;
}

// Enqueues zeroing, the batch walk and the counter reduction on `st`.
static mcx_status enqueue(mcx_batch *b, const mcx_batch_cfg *cfg, const BatchSim *descs,
                          uint64_t total, const LaunchShape &shape, cudaStream_t st)
{
    const size_t n = b->sims.size();
    const size_t words = b->fluence.bytes / 4;
    batch_zero<<<grid_of(words), 256, 0, st>>>(b->fluence.as<uint32_t>(), words);
    batch_zero<<<grid_of(n * MCX_NTALLY * 2), 256, 0, st>>>(b->tallies.as<uint32_t>(), n * MCX_NTALLY * 2);
    batch_zero<<<1, 32, 0, st>>>(b->ctrl.as<uint32_t>(), 16);
    BCUDA(b, cudaGetLastError(), "launching the zeroing");
    WalkParams p{};
    p.tab_a = b->tab_a.p;
    p.tab_b = b->tab_b.p;
    p.tab_n = b->tab_n.p;
    p.tab_tpl = b->tab_tpl.p;
    unsigned long long *ctrl = b->ctrl.as<unsigned long long>();
    p.photon_counter = ctrl;
    p.det_count = ctrl + 1;
    p.status = reinterpret_cast<unsigned *>(ctrl + 2);
    p.block_tally = b->block_tally.as<double>();
    p.block_stats = b->block_stats.as<unsigned long long>();
    p.n_media = 0;
    p.n_det = 0;
    p.n_gates = cfg->n_gates;
    p.h = 1.f;
    RunConsts<float> &c = p.cf;
    c.dt = cfg->dt_ns;
    c.inv_dt = (float)(1.0 / (double)cfg->dt_ns);
    c.t_end = (float)((double)cfg->dt_ns * cfg->n_gates);
    c.rr_threshold = cfg->rr_threshold;
    c.rr_m = cfg->rr_m;
    c.rr_inv_m = cfg->rr_threshold > 0.f ? (float)(1.0 / (double)cfg->rr_m) : 0.f;
    p.n_photons = total;
    p.max_events = cfg->max_events_per_photon ? cfg->max_events_per_photon : 100000000ull;
    p.reflect = cfg->reflect;
    p.claim_chunk = cfg->claim_chunk ? (unsigned)cfg->claim_chunk : (unsigned)kClaimChunk;
    p.sims = descs;
    p.n_sims = (int)n;
    BCUDA(b, walk_batch_launch(p, cfg->accum_mode, shape, st), "launching the batch walk");
    batch_stats<<<1, 256, 0, st>>>(p.block_stats, shape.grid, b->out_stats.as<unsigned long long>());
    BCUDA(b, cudaGetLastError(), "launching the counter reduction");
    return MCX_OK;
}

static mcx_status check_cfg(mcx_batch *b, const mcx_batch_cfg *cfg)
{
    if (!cfg || cfg->struct_size != sizeof(mcx_batch_cfg))
        return bfail(b, MCX_E_ARG, "cfg is NULL or struct_size does not match this library");
    if (b->sims.empty()) return bfail(b, MCX_E_STATE, "the batch is empty");
    if (cfg->n_gates < 1 || !(cfg->dt_ns > 0.f)) return bfail(b, MCX_E_ARG, "need n_gates >= 1, dt_ns > 0");
    if (!(cfg->rr_threshold >= 0.f) || (cfg->rr_threshold > 0.f && !(cfg->rr_m > 1.f)))
        return bfail(b, MCX_E_ARG, "need rr_threshold >= 0 and rr_m > 1");
    if (cfg->accum_mode != 0 && cfg->accum_mode != 2) return bfail(b, MCX_E_ARG, "accum_mode is 0 or 2");
    const int block = cfg->block_size ? cfg->block_size : 256;
    if (block < 32 || block > 256 || block % 32) return bfail(b, MCX_E_ARG, "block_size 32..256, multiple of 32");
    if (cfg->claim_chunk && (cfg->claim_chunk < 32 || cfg->claim_chunk > 4096))
        return bfail(b, MCX_E_ARG, "claim_chunk 32..4096");
    if (cfg->grid_size < 0) return bfail(b, MCX_E_ARG, "grid_size < 0");
    if (cfg->order != 0 && cfg->order != 1) return bfail(b, MCX_E_ARG, "order is 0 or 1");
    return MCX_OK;
}

static mcx_status prepare(mcx_batch *b, const mcx_batch_cfg *cfg, LaunchShape *shape)
{
    const int block = cfg->block_size ? cfg->block_size : 256;
    BCUDA(b, walk_batch_query_shape(cfg->accum_mode, block, shape), "querying the batch walk");
    if (shape->blocks_per_sm < 1) return bfail(b, MCX_E_ARG, "block_size does not fit on an SM");
    if (cfg->grid_size > 0) shape->grid = cfg->grid_size;
    BCUDA(b, b->ctrl.ensure(64), "allocating");
    BCUDA(b, b->block_tally.ensure((size_t)shape->grid * MCX_NTALLY * sizeof(double)), "allocating");
    BCUDA(b, b->block_stats.ensure((size_t)shape->grid * MCX_NSTAT * 8), "allocating");
    BCUDA(b, b->out_stats.ensure(MCX_NSTAT * 8), "allocating");
    return MCX_OK;
}

extern "C" {

mcx_status mcx_batch_run(mcx_batch *b, const mcx_batch_cfg *cfg)
{
    if (!b) return bfail(nullptr, MCX_E_ARG, "batch is NULL");
    mcx_status st = check_cfg(b, cfg);
    if (st != MCX_OK) return st;
    if (b->ran) BCUDA(b, cudaEventSynchronize(b->ev1), "waiting for the previous run");
    cudaStream_t stream = static_cast<cudaStream_t>(cfg->cuda_stream);
    if (cfg->use_graph && !stream) stream = b->own_stream;
    const auto key = std::make_tuple(cfg->accum_mode, cfg->block_size, cfg->claim_chunk, cfg->grid_size,
                                     cfg->n_gates, cfg->dt_ns, cfg->reflect, cfg->rr_threshold,
                                     cfg->rr_m, cfg->max_events_per_photon, (void *)stream);
    if (b->dirty || !b->ran || key != b->graph_key || cfg->accum_mode != b->cfg.accum_mode ||
        cfg->n_gates != b->cfg.n_gates || cfg->order != b->cfg.order)
        drop_graph(b);
    LaunchShape shape;
    st = prepare(b, cfg, &shape);
    if (st != MCX_OK) return st;
    uint64_t total = 0;
    if (!b->graph) {
        st = layout(b, cfg, 1.0, b->descs, &total);
        if (st != MCX_OK) return st;
        b->dirty = false;
    }
    BCUDA(b, cudaEventRecord(b->ev0, stream), "recording an event");
    if (cfg->use_graph) {
        if (!b->graph) {
            cudaGraph_t g = nullptr;
            BCUDA(b, cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal), "starting the graph capture");
            st = enqueue(b, cfg, b->descs.as<BatchSim>(), total, shape, stream);
            const cudaError_t ce = cudaStreamEndCapture(stream, &g);
            if (st != MCX_OK) { if (g) cudaGraphDestroy(g); return st; }
            if (ce != cudaSuccess) return bfail(b, MCX_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
            const cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) { b->graph = nullptr; return bfail(b, MCX_E_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(ie)); }
            b->graph_key = key;
        }
        BCUDA(b, cudaGraphLaunch(b->graph, stream), "launching the graph");
    } else {
        st = enqueue(b, cfg, b->descs.as<BatchSim>(), total, shape, stream);
        if (st != MCX_OK) return st;
    }
    BCUDA(b, cudaEventRecord(b->ev1, stream), "recording an event");
    b->cfg = *cfg;
    b->shape = shape;
    b->stream = stream;
    b->ran = true;
    return MCX_OK;
}

mcx_status mcx_batch_sync(mcx_batch *b)
{
    if (!b) return bfail(nullptr, MCX_E_ARG, "batch is NULL");
    if (!b->ran) return bfail(b, MCX_E_STATE, "no run");
    BCUDA(b, cudaEventSynchronize(b->ev1), "waiting for the run");
    return MCX_OK;
}

mcx_status mcx_batch_last_ms(mcx_batch *b, float *ms)
{
    if (!b || !ms) return bfail(b, MCX_E_ARG, "NULL argument");
    mcx_status st = mcx_batch_sync(b);
    if (st != MCX_OK) return st;
    BCUDA(b, cudaEventElapsedTime(ms, b->ev0, b->ev1), "reading the run time");
    return MCX_OK;
}

mcx_status mcx_batch_read_fluence(mcx_batch *b, int32_t id, float *dst, uint64_t n_elems,
                                  int32_t normalized, int32_t dst_on_device)
{
    if (!b || !dst) return bfail(b, MCX_E_ARG, "NULL argument");
    if (id < 0 || (size_t)id >= b->sims.size()) return bfail(b, MCX_E_ARG, "no such simulation");
    mcx_status st = mcx_batch_sync(b);
    if (st != MCX_OK) return st;
    const SimHost *s = b->sims[id];
    const uint64_t nvox = (uint64_t)s->nx * s->ny * s->nz, n = nvox * b->cfg.n_gates;
    if (n_elems != n) return bfail(b, MCX_E_ARG, "n_elems must be n_gates*nx*ny*nz = " + std::to_string(n));
    const float *inv = nullptr;
    if (normalized) {
        std::vector<float> iv(kMaxMedia, 0.f);
        const double N = (double)s->n_photons, v = (double)s->h * s->h * s->h;
        for (uint32_t m = 1; m < s->n_media; ++m)
            if (s->props[4 * m] > 0 && N > 0) iv[m] = (float)(1.0 / (s->props[4 * m] * v * N * b->cfg.dt_ns));
        BCUDA(b, b->inv_norm.ensure(kMaxMedia * sizeof(float)), "allocating");
        BCUDA(b, cudaMemcpy(b->inv_norm.p, iv.data(), kMaxMedia * sizeof(float), cudaMemcpyHostToDevice),
              "uploading normalisation");
        inv = b->inv_norm.as<float>();
    }
    float *out = dst;
    if (!dst_on_device) {
        BCUDA(b, b->staging.ensure(n * sizeof(float)), "allocating");
        out = b->staging.as<float>();
    }
    const bool f64 = b->cfg.accum_mode == kAccF64;
    batch_resolve<<<grid_of(n), 256, 0, b->stream>>>(
        f64 ? nullptr : b->fluence.as<float>() + b->flu_off[id],
        f64 ? b->fluence.as<double>() + b->flu_off[id] : nullptr, s->labels.as<uint8_t>(), inv,
        s->nx, s->ny, (unsigned)nvox, (s->nx + 2) * (s->ny + 2) * (s->nz + 2), n, out);
    BCUDA(b, cudaGetLastError(), "launching the read-out");
    if (!dst_on_device) {
        BCUDA(b, cudaMemcpyAsync(dst, out, n * sizeof(float), cudaMemcpyDeviceToHost, b->stream), "copying");
    }
    BCUDA(b, cudaStreamSynchronize(b->stream), "waiting for the read-out");
    return MCX_OK;
}

mcx_status mcx_batch_read_tally(mcx_batch *b, int32_t id, double out[MCX_NTALLY])
{
    if (!b || !out) return bfail(b, MCX_E_ARG, "NULL argument");
    if (id < 0 || (size_t)id >= b->sims.size()) return bfail(b, MCX_E_ARG, "no such simulation");
    mcx_status st = mcx_batch_sync(b);
    if (st != MCX_OK) return st;
    BCUDA(b, cudaMemcpy(out, b->tallies.as<double>() + (size_t)id * MCX_NTALLY,
                        MCX_NTALLY * sizeof(double), cudaMemcpyDeviceToHost), "reading tallies");
    out[MCX_TALLY_LAUNCHED] = (double)b->sims[id]->n_photons;
    return MCX_OK;
}

mcx_status mcx_batch_read_stats(mcx_batch *b, uint64_t out[MCX_NSTAT])
{
    if (!b || !out) return bfail(b, MCX_E_ARG, "NULL argument");
    mcx_status st = mcx_batch_sync(b);
    if (st != MCX_OK) return st;
    BCUDA(b, cudaMemcpy(out, b->out_stats.p, MCX_NSTAT * 8, cudaMemcpyDeviceToHost), "reading counters");
    return MCX_OK;
}

mcx_status mcx_batch_autotune(mcx_batch *b, mcx_batch_cfg *cfg, double fraction, float *best_ms)
{
    if (!b) return bfail(nullptr, MCX_E_ARG, "batch is NULL");
    mcx_status st = check_cfg(b, cfg);
    if (st != MCX_OK) return st;
    if (!(fraction > 0.0) || fraction > 1.0) return bfail(b, MCX_E_ARG, "fraction in (0, 1]");
    if (b->ran) BCUDA(b, cudaEventSynchronize(b->ev1), "waiting for the previous run");
    cudaStream_t stream = static_cast<cudaStream_t>(cfg->cuda_stream);
    const int blocks[] = {128, 256};
    const int chunks[] = {32, 64, 128, 256};
    float best = -1.f;
    int best_block = 256, best_chunk = 32;
    for (int bl : blocks) {
        for (int ch : chunks) {
            mcx_batch_cfg c = *cfg;
            c.block_size = bl;
            c.claim_chunk = ch;
            c.grid_size = 0;
            LaunchShape shape;
            st = prepare(b, &c, &shape);
            if (st != MCX_OK) return st;
            uint64_t total = 0;
            st = layout(b, &c, fraction, b->descs_tune, &total);
            if (st != MCX_OK) return st;
            for (int rep = 0; rep < 2; ++rep) {       // the first pass warms the shape
                BCUDA(b, cudaEventRecord(b->ev0, stream), "recording an event");
                st = enqueue(b, &c, b->descs_tune.as<BatchSim>(), total, shape, stream);
                if (st != MCX_OK) return st;
                BCUDA(b, cudaEventRecord(b->ev1, stream), "recording an event");
            }
            BCUDA(b, cudaEventSynchronize(b->ev1), "waiting for a trial");
            float ms = 0.f;
            BCUDA(b, cudaEventElapsedTime(&ms, b->ev0, b->ev1), "timing a trial");
            if (best < 0.f || ms < best) { best = ms; best_block = bl; best_chunk = ch; }
        }
    }
    cfg->block_size = best_block;
    cfg->claim_chunk = best_chunk;
    if (best_ms) *best_ms = best;
    b->dirty = true;                                  // the next run lays out the full batch
    b->ran = false;
    drop_graph(b);
    return MCX_OK;
}

void mcx_batch_destroy(mcx_batch *b)
{
    if (!b) return;
    if (b->ran) cudaEventSynchronize(b->ev1);
    drop_graph(b);
    for (SimHost *s : b->sims) {
        s->labels.release();
        delete s;
    }
    for (Buf *x : {&b->fluence, &b->descs, &b->descs_tune, &b->tab_a, &b->tab_b, &b->tab_n,
                   &b->tab_tpl, &b->tallies, &b->ctrl, &b->block_tally, &b->block_stats,
                   &b->out_stats, &b->staging, &b->inv_norm})
        x->release();
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
    delete b;
}

}  // extern "C"
