/*
 * mcx.h - C ABI of the GB300 voxel Monte Carlo photon-transport library.
 *
 * The operation is the paper's photon simulation workflow (Fig. 1 and the paragraph that
 * describes it): the host processes the user's inputs (domain, optical properties, source,
 * photon count), the device runs the photon simulation loop in every thread with
 * independent random streams, and the host reads back the 3-D fluence maps and the
 * detected-photon data, then post-processes them.  The photon loop's physics is the one
 * the paper's benchmark description (beside Fig. 2) relies on: exponential hops through a
 * labelled voxel domain, Snell/Fresnel at refractive-index mismatches (or termination at
 * the boundary), Henyey-Greenstein scattering, Russian roulette, atomic (race-free)
 * fluence accumulation into time gates, and disk detectors recording partial path lengths.
 *
 * Conventions for every entry point:
 *   - Every call returns an mcx_status; no call aborts or throws across the ABI.  On an
 *     error, mcx_last_error(sim) describes it (mcx_last_error(NULL) for errors raised
 *     before a handle exists).
 *   - Inputs passed as host pointers are copied before the call returns; the caller keeps
 *     ownership.  Outputs are written to caller-owned buffers.
 *   - Positions and lengths are in mm, times in ns, coefficients in 1/mm.
 *   - Label volumes are uint8 arrays [nz][ny][nx] (x fastest).  Label 0, and everything
 *     outside the grid, is the exterior medium.
 *   - A handle is not thread-safe; use one handle per host thread.
 *   - Needs a CUDA device of compute capability 10.3 (GB300); the library is built for
 *     sm_103a only.
 */
#ifndef MCX_H
#define MCX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MCX_ABI_VERSION 2

typedef struct mcx_sim mcx_sim;   /* opaque; owns all device buffers of one simulation */

typedef enum mcx_status {
    MCX_OK = 0,
    MCX_E_ARG = -1,      /* invalid argument; nothing was changed */
    MCX_E_STATE = -2,    /* call out of order (e.g. run before media are set) */
    MCX_E_CUDA = -3,     /* a CUDA call failed; see mcx_last_error */
    MCX_E_OOM = -4,      /* device allocation failed */
    MCX_E_CAP = -5,      /* outputs are valid, but a capacity was hit: the detected-photon
                            buffer overflowed or a photon reached the per-photon event cap */
    MCX_E_TIMEOUT = -6   /* mcx_sync gave up waiting; the run is still in flight */
} mcx_status;

/* photon fates (mcx_exit.fate) */
enum { MCX_FATE_NONE = 0, MCX_FATE_ESCAPED = 1, MCX_FATE_ROULETTE = 2, MCX_FATE_TIME = 3,
       MCX_FATE_MISSED = 4, MCX_FATE_CAPPED = 5 };

/* energy tallies (mcx_read_tally); launched = absorbed + escaped + time_exceeded
   + roulette_killed - roulette_gained holds up to rounding */
enum { MCX_TALLY_LAUNCHED = 0, MCX_TALLY_ABSORBED = 1, MCX_TALLY_ESCAPED = 2,
       MCX_TALLY_TIME = 3, MCX_TALLY_RR_KILLED = 4, MCX_TALLY_RR_GAINED = 5, MCX_NTALLY = 6 };

/* event counters (mcx_read_stats): scattering events, voxel-face crossings, Fresnel
   evaluations (including total internal reflection), fluence atomics issued, roulette
   draws, photons finished (all fates), photons detected, photons stopped by the cap */
enum { MCX_STAT_SCATTER = 0, MCX_STAT_FACE = 1, MCX_STAT_FRESNEL = 2, MCX_STAT_FLUSH = 3,
       MCX_STAT_ROULETTE = 4, MCX_STAT_PHOTONS = 5, MCX_STAT_DETECTED = 6, MCX_STAT_CAPPED = 7,
       MCX_NSTAT = 8 };

/* Per-run settings.  Fill with mcx_run_cfg_default() and then override fields; the
   defaults are n_gates 1, dt_ns 5, reflect 1, rr_threshold 1e-4, rr_m 10, accum_mode 2,
   precision 0, automatic launch shape. */
typedef struct mcx_run_cfg {
    uint32_t struct_size;          /* sizeof(mcx_run_cfg); checked by mcx_run */
    uint32_t n_gates;              /* time gates [g dt, (g+1) dt), g < n_gates; >= 1 */
    uint64_t n_photons;            /* photons launched by this run (may be 0) */
    uint64_t photon_offset;        /* id of the first photon; a run over ids [a, a+n) is a
                                      pure function of (seed, a, n), so ranges compose */
    uint64_t seed;                 /* run seed; photon p's stream derives from (seed, p) */
    float dt_ns;                   /* gate width, > 0; photons stop at n_gates * dt_ns */
    int32_t reflect;               /* 1: Fresnel/Snell at index mismatches; 0: photons are
                                      terminated on reaching the exterior and pass internal
                                      mismatches unchanged (the paper's benchmark B1) */
    float rr_threshold;            /* Russian roulette below this weight (0 disables) */
    float rr_m;                    /* roulette: survive with probability 1/rr_m, weight x rr_m */
    uint64_t max_detected;         /* capacity of the detected-photon buffer (records) */
    uint64_t exit_log;             /* log fate/exit of photons offset .. offset+exit_log-1 */
    uint64_t max_events_per_photon;/* segment cap per photon (0 = library default 1e8) */
    int32_t accum_mode;            /* fluence accumulation; every mode first sums a photon's
                                      deposits in a register while it stays in one (gate, voxel):
                                      0: one FP32 atomic add per run into the map (fastest);
                                      1: compensated FP32 pairs in block tiles: runs inside the
                                         block tile (below) go to a block-private shared-memory
                                         (hi, lo) pair, the rounding error of each hi addition
                                         recovered exactly (TwoSum on the atomic's old value)
                                         into lo; each block flushes its tile once, in FP64,
                                         into the FP64 map; runs outside the tile go to that map
                                         as in mode 2;
                                      2: FP64 global atomics (the default: exact to FP64
                                         rounding, and measured as fast as mode 0 on GB300,
                                         whose L2 adds FP64 at the FP32 rate; at 1e8 photons
                                         mode 0 loses up to tens of percent in the hottest
                                         voxels, where additions fall below half an ulp) */
    int32_t block_size;            /* threads per block, multiple of 32 (0 = 256) */
    int32_t grid_size;             /* persistent blocks (0 = SMs x resident blocks/SM) */
    int32_t precision;             /* 0: FP32 photon state (the product path); 1: the same walk
                                      in FP64, a trajectory-parity diagnostic that runs at the
                                      part's much lower FP64 rate */
    void *cuda_stream;             /* cudaStream_t to enqueue on (NULL = legacy default) */
    int32_t tile_lo[4];            /* accum_mode 1: block tile origin (voxel x, y, z, gate) */
    int32_t tile_size[4];          /* and extent; all zero = automatic: 16 x 16 x 24 voxels of
                                      gate 0 from the source voxel down, clipped to the grid;
                                      at most 6144 (gate, voxel) entries (48 KiB per block) */
    int32_t claim_mode;            /* photon distribution: 0 = dynamic (a warp claims 32 ids
                                      at a time from a global counter as its lanes finish);
                                      1 = static per-thread split (thread k of T simulates
                                      ids k, k+T, k+2T, ...), the paper's thread-level
                                      baseline in its load-balancing comparison (Fig. 3a);
                                      FP32 walk only */
    int32_t reserved1;
} mcx_run_cfg;

/* Fate and end state of one logged photon (fixed-seed parity log). */
typedef struct mcx_exit {
    int32_t fate;                  /* MCX_FATE_* */
    uint32_t nscat;                /* scattering events */
    float pos[3];                  /* mm: exit point for escaped photons, else end point */
    float dir[3];                  /* direction at the end (refracted on escape) */
    float w;                       /* weight at the end */
    float t;                       /* ns */
} mcx_exit;

/* ABI version of the loaded library (MCX_ABI_VERSION it was built with). */
int32_t mcx_abi_version(void);
const char *mcx_status_string(int32_t status);
void mcx_run_cfg_default(mcx_run_cfg *cfg);

/* The paper's input "domain" (workflow beside Fig. 1; the benchmark volumes beside Fig. 2
   are such labelled voxel grids).
   Creates a simulation over an nx x ny x nz label volume of cubic voxels voxel_mm wide.
   labels: uint8 [nz][ny][nx]; a host pointer (labels_on_device = 0) or a device pointer on
   the current device (labels_on_device = 1); copied into the handle's device memory.
   The handle binds to the CUDA device current at this call.  (nx+2)(ny+2)(nz+2) < 2^32: the
   device copy carries a one-voxel exterior border on every side. */
mcx_status mcx_create_volume(mcx_sim **out, uint32_t nx, uint32_t ny, uint32_t nz,
                             float voxel_mm, const uint8_t *labels, int32_t labels_on_device);

/* Replaces the label volume (same dimensions; the workflow's domain input, Fig. 1);
   invalidates previous outputs. */
mcx_status mcx_update_labels(mcx_sim *sim, const uint8_t *labels, int32_t labels_on_device);

/* The workflow's "optical properties" input (Fig. 1); the benchmark description beside
   Fig. 2 gives them per medium as absorption, scattering, anisotropy and index.
   Optical properties, host array props[n_media][4] = (mua /mm, mus /mm, g, n); row m
   applies to label m; row 0 is the exterior (only its n is used).  1 <= n_media <= 256;
   every label present in the volume must have a row.  mua, mus >= 0, |g| < 1, n > 0. */
mcx_status mcx_set_media(mcx_sim *sim, uint32_t n_media, const float *props);

/* The workflow's source input (Fig. 1); the benchmarks beside Fig. 2 use a pencil beam.
   Source: kind 0 = pencil beam at pos along dir; kind 1 = Gaussian beam whose launch
   points are spread over the plane normal to dir with I(r) ~ exp(-2 r^2 / waist^2).
   dir is normalised by the library.  A photon whose launch point is outside the grid or
   in a label-0 voxel is counted as escaped with fate MCX_FATE_MISSED. */
mcx_status mcx_set_source(mcx_sim *sim, int32_t kind, const float pos_mm[3],
                          const float dir[3], float waist_mm);

/* Detectors produce the workflow's "detected photon data" output (Fig. 1 paragraph).
   Adds a detector: a photon escaping at a point within radius_mm of center_mm is recorded
   (lowest detector id on overlap).  Up to 64 detectors; with detectors present the number
   of media is limited to 33 (32 tissue labels, for the partial-path record). */
mcx_status mcx_add_detector(mcx_sim *sim, const float center_mm[3], float radius_mm,
                            int32_t *out_id);
mcx_status mcx_clear_detectors(mcx_sim *sim);

/* The device side of the workflow (Fig. 1): every thread runs the photon simulation loop
   with its own random stream; photon counts and per-thread balancing follow the
   load-balancing discussion (Fig. 3a), as a dynamic per-warp claim by default.
   Enqueues one simulation on cfg->cuda_stream and returns without waiting.  Zeroes the
   outputs, runs the persistent photon-walk kernel, then reduces the energy tallies.
   Output buffers are (re)allocated here when the gate count or capacities change. */
mcx_status mcx_run(mcx_sim *sim, const mcx_run_cfg *cfg);

/* The host's wait for the device in the workflow (Fig. 1), bounded.
   Waits for the last run, polling for at most timeout_s seconds (< 0: no limit).
   MCX_E_TIMEOUT leaves the run in flight.  MCX_E_CAP: finished, but a capacity was hit. */
mcx_status mcx_sync(mcx_sim *sim, double timeout_s);

/* The simulation time the paper's speed figures are built from (photons per ms, Fig. 2).
   Device time of the last run's walk kernel (CUDA events on the run's stream), in ms.
   Waits for the run. */
mcx_status mcx_last_kernel_ms(mcx_sim *sim, float *ms);

/* The workflow's "3-D fluence maps" output and its post-processing (Fig. 1 paragraph).
   Fluence of the last run, float [n_gates][nz][ny][nx].  normalized = 0: absorbed weight
   per voxel and gate (sum of deposited photon weight).  normalized = 1: fluence rate per
   launched photon, E / (mua h^3 N dt) in 1/(mm^2 ns), 0 where mua = 0.  dst is host memory
   (dst_on_device = 0; the call waits) or device memory on the handle's device
   (dst_on_device = 1; the copy is enqueued on the run's stream).  n_elems must equal
   n_gates*nx*ny*nz. */
mcx_status mcx_read_fluence(mcx_sim *sim, float *dst, uint64_t n_elems, int32_t normalized,
                            int32_t dst_on_device);

/* As mcx_read_fluence, in FP64: the map as accumulated (accum_mode 1 and 2: the FP64 map,
   with accum_mode 1's block tiles added into it; accum_mode 0: the FP32 map widened). */
mcx_status mcx_read_fluence64(mcx_sim *sim, double *dst, uint64_t n_elems, int32_t normalized,
                              int32_t dst_on_device);

/* Words (4 bytes each) per detected-photon record: 12 + (n_media - 1). */
int32_t mcx_detected_stride(const mcx_sim *sim);

/* The workflow's "detected photon data" output (Fig. 1 paragraph).
   Detected-photon records of the last run, in photon-id order, into host memory dst
   (cap_records * stride words).  Record layout, 32-bit words:
     [0] photon id low 32 bits, [1] high 32 bits (uint32 bit patterns)
     [2] detector id (int32)   [3] scattering events (uint32)
     [4] exit weight (float)   [5..7] exit point (mm)   [8..10] exit direction
     [11] roulette survivals (uint32)   [12 + m - 1] path length in label m (mm), m >= 1
   n_written: records copied; n_total: photons detected (more than the buffer held when the
   buffer overflowed).  Waits for the run. */
mcx_status mcx_read_detected(mcx_sim *sim, void *dst, uint64_t cap_records,
                             uint64_t *n_written, uint64_t *n_total);

/* Energy bookkeeping of the photon loop (absorbed, escaped, time-limited, roulette; the
   physics the benchmarks beside Fig. 2 rely on), FP64, into host memory.  Waits. */
mcx_status mcx_read_tally(mcx_sim *sim, double out[MCX_NTALLY]);

/* Event counts of the photon loop (the work behind the paper's kernel profile, which
   counts it in compute and memory instructions in its profiling observations) of the
   last run, into host memory.  Waits. */
mcx_status mcx_read_stats(mcx_sim *sim, uint64_t out[MCX_NSTAT]);

/* Per-photon end states for fixed-seed comparison (the paper's per-thread independent
   seeds, Fig. 1 paragraph, made per photon id).  Exit log of the last run (photons
   offset .. offset + exit_log - 1, by photon id) into host memory.  Waits. */
mcx_status mcx_read_exits(mcx_sim *sim, mcx_exit *dst, uint64_t cap, uint64_t *n_written);

/* The thread configuration the paper tunes per device (its Opt2, Fig. 2): the shape the
   last run used (blocks, threads per block, resident blocks per SM, registers per
   thread). */
mcx_status mcx_launch_info(mcx_sim *sim, int32_t out[4]);

const char *mcx_last_error(const mcx_sim *sim);
void mcx_destroy(mcx_sim *sim);

/* ---- batched simulations --------------------------------------------------------------
   Many independent simulations of different volumes, optical properties, sources and
   photon counts run in ONE persistent launch of the walk: photons of all simulations form
   one queue, so small simulations do not leave the GPU idle (the paper balances photons
   within a workgroup and across devices, Fig. 3; this extends the idea across problems).
   Every simulation's photon p uses the stream of (its seed, p): a batched simulation gives
   the same per-photon trajectories as the same simulation run alone with mcx_run.
   All simulations share the time gates, the roulette and reflection settings and the
   accumulation mode; the walk runs with FP32 photon state; no detectors or exit log. */
typedef struct mcx_batch mcx_batch;

typedef struct mcx_batch_cfg {
    uint32_t struct_size;          /* sizeof(mcx_batch_cfg) */
    uint32_t n_gates;              /* shared time gates [g dt, (g+1) dt) */
    float dt_ns;
    int32_t reflect;
    float rr_threshold;
    float rr_m;
    int32_t accum_mode;            /* 0 (FP32 atomics) or 2 (FP64 atomics, default) */
    int32_t block_size;            /* 0 = 256 (multiple of 32, <= 256) */
    int32_t claim_chunk;           /* photon ids per warp claim: 0 = 32; 32..4096 */
    int32_t grid_size;             /* 0 = SMs x resident blocks per SM */
    uint64_t max_events_per_photon;/* 0 = 1e8 */
    int32_t use_graph;             /* 1: record the run (zeroing, walk, reductions) as a CUDA
                                      graph on first use and replay it while the batch and the
                                      settings stay the same */
    int32_t order;                 /* photon queue order: 0 = the simulations as added, 1 =
                                      (default) the longest expected photon histories first, a
                                      scheduling heuristic from the optical properties that
                                      shortens the launch's tail; results do not depend on it
                                      (each simulation keeps its own photon streams) */
    void *cuda_stream;             /* cudaStream_t (NULL = legacy default; with use_graph the
                                      library then uses a stream of its own) */
} mcx_batch_cfg;

void mcx_batch_cfg_default(mcx_batch_cfg *cfg);
mcx_status mcx_batch_create(mcx_batch **out);
/* Adds one simulation (arguments as in mcx_create_volume, mcx_set_media, mcx_set_source);
   inputs are copied; out_id receives its index in the batch.  Invalidates earlier runs. */
mcx_status mcx_batch_add(mcx_batch *b, uint32_t nx, uint32_t ny, uint32_t nz, float voxel_mm,
                         const uint8_t *labels, int32_t labels_on_device, uint32_t n_media,
                         const float *props, int32_t src_kind, const float pos_mm[3],
                         const float dir[3], float waist_mm, uint64_t n_photons, uint64_t seed,
                         int32_t *out_id);
/* Enqueues one run of every simulation in the batch; returns without waiting. */
mcx_status mcx_batch_run(mcx_batch *b, const mcx_batch_cfg *cfg);
mcx_status mcx_batch_sync(mcx_batch *b);
/* Device time of the last run: the whole enqueued sequence (ms). */
mcx_status mcx_batch_last_ms(mcx_batch *b, float *ms);
/* Fluence of simulation `id` (float [n_gates][nz][ny][nx]; normalized as in
   mcx_read_fluence), host or device destination; waits for the run. */
mcx_status mcx_batch_read_fluence(mcx_batch *b, int32_t id, float *dst, uint64_t n_elems,
                                  int32_t normalized, int32_t dst_on_device);
mcx_status mcx_batch_read_tally(mcx_batch *b, int32_t id, double out[MCX_NTALLY]);
/* Event counters of the whole batch (MCX_STAT_*). */
mcx_status mcx_batch_read_stats(mcx_batch *b, uint64_t out[MCX_NSTAT]);
/* Times the batch with every simulation's photon count scaled by `fraction` (0 < f <= 1)
   for block sizes {128, 256} x claim chunks {32, 64, 128, 256}, and writes the fastest
   into cfg (block_size, claim_chunk); best_ms receives its time.  Runs on cfg's stream. */
mcx_status mcx_batch_autotune(mcx_batch *b, mcx_batch_cfg *cfg, double fraction, float *best_ms);
int32_t mcx_batch_size(const mcx_batch *b);
const char *mcx_batch_last_error(const mcx_batch *b);
void mcx_batch_destroy(mcx_batch *b);

/* ---- allocation-free run --------------------------------------------------------------
   The paper has no counterpart to this entry point; it exists for callers that cannot let
   a library allocate device memory: applications whose own pool or caching allocator owns
   the whole device memory (memory taken behind its back is invisible to it and fragments
   it), and latency-sensitive loops that cannot afford the device-wide synchronisation a
   cudaFree may cause.

   Runs one simulation like mcx_create_volume + set_media + set_source + mcx_run, on the
   caller's buffers, and calls no cudaMalloc, cudaFree or other allocating routine.
     labels_dev   uint8 [nz][ny][nx] on the current device (read only)
     props        host float [n_media][4] as in mcx_set_media; 1 <= n_media <= 32
     src_kind, pos_mm, dir, waist_mm   as in mcx_set_source
     cfg          as for mcx_run (cuda_stream honoured); needs precision = 0, exit_log = 0,
                  max_detected = 0 (no detectors), grid_size <= 2048, and accum_mode
                  0 (FP32 atomics: additions into a voxel that already holds more than about
                  1e7 times their weight are lost, so a hot voxel's sum falls short by tens of
                  percent at 1e8 photons) or 2 (FP64 atomics, exact to FP64 rounding)
     fluence_dev  device memory of the current device holding n_gates*nz*ny*nx elements,
                  float [n_gates][nz][ny][nx] for accum_mode 0, double for accum_mode 2;
                  zeroed, then filled with absorbed weight (as mcx_read_fluence with
                  normalized = 0).  The library cannot check its size: a smaller buffer is
                  written past its end.
     tally_dev    double [MCX_NOALLOC_NOUT] on the current device: the energy tallies
                  (MCX_TALLY_*), then in word MCX_NTALLY the number of photons stopped by the
                  per-photon event cap (their weight counted as time-exceeded).  A nonzero
                  count is the condition mcx_sync reports as MCX_E_CAP for mcx_run: this
                  call returns before the walk ends, so the caller reads it after
                  synchronising the stream.
   Its working memory (photon counter, status, per-label tables, per-block partials) is a
   fixed 226 KiB array in the library, held by every GPU that loads it until the process
   exits; sizes beyond its limits are rejected with MCX_E_ARG, as are pointers that are not
   device memory of the current device.  The first call on a device looks up that array's
   device address.  The call checks the labels (a 4-byte read-back that waits for the
   stream), then enqueues the rest on cfg->cuda_stream and returns; because of that wait it
   cannot be made while its stream is being captured into a CUDA graph (MCX_E_STATE).
   Every call reuses the same array: calls whose work overlaps on one GPU (other streams or
   host threads) race on it; serialise them.  Errors: MCX_E_ARG / MCX_E_STATE (a label >=
   n_media, or stream capture) / MCX_E_CUDA, described by mcx_last_error(NULL). */
#define MCX_NOALLOC_NOUT (MCX_NTALLY + 1)
mcx_status mcx_run_noalloc(const uint8_t *labels_dev, uint32_t nx, uint32_t ny, uint32_t nz,
                           float voxel_mm, uint32_t n_media, const float *props,
                           int32_t src_kind, const float pos_mm[3], const float dir[3],
                           float waist_mm, const mcx_run_cfg *cfg, void *fluence_dev,
                           double *tally_dev);

/* ---- learned denoiser -----------------------------------------------------------------
   The paper has no counterpart: this extends the method with a small 3-D convolutional
   network that maps the fluence of a low-photon run to an estimate of a high-photon run's,
   so that fewer photons reach a given voxel-wise error.  A plain run with more photons
   stays the fallback: the denoiser never replaces the walk, it post-processes its map.

   Network (a U-Net; all 3x3x3 convolutions have a bias and ReLU, "same" zero padding):
     level 0 (nz,ny,nx):   e1a 16->16 (input channel 0: the encoded fluence; channels
                           1..n_aux: medium features; the rest zero), e1b 16->16
     2x2x2 average pool;   level 1: e2a 16->32, e2b 32->32
     2x2x2 average pool;   level 2: ba 32->64, bb 64->64
     nearest x2 upsample, concatenated with e2b's output (upsampled channels first):
                           level 1: d2a 96->32, d2b 32->32
     nearest x2 upsample, concatenated with e1b's output: level 0: d1a 48->16, d1b 16->16
     head: y = x + hb + sum_c hw[c] * d1b[c]   (1x1x1, FP32)
   Weights and activations are BF16, every convolution accumulates in FP32 on tensor
   cores; master weights, gradients and the Adam state are FP32.

   Parameters are one FP32 vector, layer by layer in the order above: for each of the ten
   convolutions its weights [27 taps][cout][cin] (tap = 9 (dz+1) + 3 (dy+1) + (dx+1), the
   input read at (z+dz, y+dy, x+dx)) then its bias [cout]; then hw[16], then hb.
   The network domain: x = (log10(max(phi, 0) + floor) - mu) / sigma, with the inverse
   phi = max(10^(x sigma + mu) - floor, 0); defaults floor 1e-8, mu -4, sigma 2.

   Volumes are FP32 [n][nz][ny][nx] device arrays on the denoiser's device, n <= max_batch;
   medium features (when n_aux > 0) are FP32 [n][n_aux][nz][ny][nx] (mcx_denoiser_features
   computes the two this library defines from a label volume).
   Sizes: nx a multiple of 64 up to 252 (so nx = 64 or 128), ny and nz multiples of 4,
   max_batch * nx * ny * nz * 96 < 2^31.  The object owns every buffer it
   needs (activations for max_batch volumes); calls on one object must not overlap.
   Errors: MCX_E_ARG (bad sizes or NULL), MCX_E_OOM, MCX_E_CUDA, MCX_E_TIMEOUT (see
   mcx_denoiser_sync), described by mcx_last_error(NULL). */
typedef struct mcx_denoiser mcx_denoiser;

/* n_aux = 0..7 medium-feature input channels.  He-normal weights drawn from `seed`, zero
   biases and a zero head (the untrained network returns its input). */
mcx_status mcx_denoiser_create(mcx_denoiser **out, uint32_t nx, uint32_t ny, uint32_t nz,
                               uint32_t max_batch, uint32_t n_aux, uint64_t seed);
mcx_status mcx_denoiser_param_count(const mcx_denoiser *d, uint64_t *n);
/* which = 0: the FP32 master weights; which = 1: the gradients of the last train step.
   Waits for the device. */
mcx_status mcx_denoiser_get_params(mcx_denoiser *d, float *host, uint64_t n, int32_t which);
/* Replaces the weights (and resets the optimizer state). Waits for the device. */
mcx_status mcx_denoiser_set_params(mcx_denoiser *d, const float *host, uint64_t n);
mcx_status mcx_denoiser_set_encoding(mcx_denoiser *d, float floor_, float mu, float sigma);
/* Network domain in and out: y_dev = net(x_dev, aux_dev) for n volumes, enqueued on
   `stream`; aux_dev may be NULL when n_aux = 0. */
mcx_status mcx_denoiser_forward(mcx_denoiser *d, const float *x_dev, const float *aux_dev,
                                float *y_dev, uint32_t n, void *stream);
/* One training step on n (input, target) pairs in the network domain: loss = mean over all
   voxels of (net(x) - t)^2, gradients of every parameter, then (if lr > 0) one Adam step
   (beta 0.9 / 0.999, eps 1e-8).  With loss_host non-NULL the call waits and returns the
   loss there. */
mcx_status mcx_denoiser_train_step(mcx_denoiser *d, const float *x_dev, const float *aux_dev,
                                   const float *t_dev, uint32_t n, float lr, float *loss_host,
                                   void *stream);
/* Elementwise maps between fluence and the network domain (count values). */
mcx_status mcx_denoiser_encode(mcx_denoiser *d, const float *phi_dev, float *x_dev,
                               uint64_t count, void *stream);
mcx_status mcx_denoiser_decode(mcx_denoiser *d, const float *x_dev, float *phi_dev,
                               uint64_t count, void *stream);
/* Denoises n fluence maps: encode, forward, decode, enqueued on `stream`. */
mcx_status mcx_denoiser_apply(mcx_denoiser *d, const float *phi_in_dev, const float *aux_dev,
                              float *phi_out_dev, uint32_t n, void *stream);
/* The two medium features of a label volume (uint8 [nvox] on the device; props as in
   mcx_set_media, label l -> row l, labels >= n_media count as exterior):
   out_dev[0][v] = log10(max(mua, 1e-4)) + 2, out_dev[1][v] = log10(max(mus (1 - g), 1e-3))
   (FP32 [2][nvox]).  Waits for `stream`. */
mcx_status mcx_denoiser_features(const uint8_t *labels_dev, uint64_t nvox, uint32_t n_media,
                                 const float *props, float *out_dev, void *stream);
/* Builds a training batch: volume s of dst_dev (n volumes) is volume idx[s] of set_dev
   (set_count volumes of the denoiser's shape), mirrored in x (flags[s] bit 0) and in y
   (bit 1), then transposed in x/y (bit 2; needs ny == nx).  idx and flags are host arrays
   of n <= 64 entries, read before the call returns. */
mcx_status mcx_denoiser_gather(mcx_denoiser *d, const float *set_dev, uint64_t set_count,
                               const uint64_t *idx, const uint32_t *flags, uint32_t n,
                               float *dst_dev, void *stream);
/* Waits for the device; MCX_E_TIMEOUT if a tensor-core pipeline wait of an earlier call
   gave up (its results are invalid; the object stays usable).  train_step with a loss
   pointer and get_params make the same check. */
mcx_status mcx_denoiser_sync(mcx_denoiser *d);
void mcx_denoiser_destroy(mcx_denoiser *d);

/* ---- diagnostics: run the library's device primitives on small host arrays ---------- */

/* Photon `photon`'s stream for `seed`, as the walk kernel draws it: for each of the first
   n generator outputs, out_host[5i] is the single-uniform draw (top 23 bits, also the
   first of a pair), out_host[5i+1] the second uniform of a pair draw (bits 40..18), and
   out_host[5i+2..5i+4] the triple draw of a scattering event (bits 63..43: the next hop,
   42..22: the deflection, 21..1: the azimuth); 5n floats. */
mcx_status mcx_debug_uniforms(uint64_t seed, uint64_t photon, uint64_t n, float *out_host);

/* Measured rate of one device resource the walk draws on, for its roofline (the walk is
   bound by the slowest of issue, special-function unit and L2 atomics, each rate divided by
   the walk's per-photon demand on it; the paper reports the walk compute-bound, with 91 M
   compute against 0.5 M memory instructions in its kernel profile).  Times the second of
   two launches of a microbenchmark on the current device (8 blocks of 256 threads per SM):
     kind 0: FP32 FMA issue (8 independent chains per thread), thread-ops/s
     kind 1: three-input logic issue (LOP3, 8 chains), thread-ops/s
     kind 2..5: special-function unit lg2 / ex2 / rsqrt / sin (approx), ops/s
     kind 6 / 7: fire-and-forget FP32 / FP64 atomic adds to addresses hashed over a map of
                 map_bytes (rounded down to a power of two; 4 KiB .. 64 GiB), ops/s
     kind 8 / 9: FP32 / FP64 atomic adds, every warp's lanes to the same 32 words, ops/s
   Allocates (and frees) its buffer; waits for the device.  MCX_E_ARG / MCX_E_OOM /
   MCX_E_CUDA described by mcx_last_error(NULL). */
mcx_status mcx_probe_rate(int32_t kind, uint64_t map_bytes, double *rate);

/* Evaluates one device primitive on n input tuples (host arrays, row-major):
     kind 0: Henyey-Greenstein sample,  in (g, xi)                             -> out (cos, sin)
     kind 1: direction rotation,        in (ux, uy, uz, cos_t, sin_t, phi/2pi) -> out (ux, uy, uz)
     kind 2: Fresnel reflectance,       in (n1, n2, cos_i)                     -> out (R; 1 on TIR) */
mcx_status mcx_debug_primitive(int32_t kind, uint64_t n, const float *in_host,
                               float *out_host);

/* The bounded mbarrier wait the denoiser's pipelines use, on a barrier that nothing
   arrives on (arrive = 0: the wait must give up after 2^limit_log2 polls, limit_log2 <= 22)
   or that one arrival completes first (arrive = 1).  *timed_out = 1 when it gave up.  No
   device state is left behind either way. */
mcx_status mcx_debug_wait_timeout(int32_t arrive, int32_t limit_log2, int32_t *timed_out);

/* One 3x3x3 convolution of the denoiser on host arrays, run by the denoiser's own
   kernels (tcgen05 for kind 0 and kind 1; the direct input layer for kind 0 with cin 1);
   values are rounded to BF16 on the way in; n volumes of nz x ny x nx, nx a multiple of 16
   up to 254:
     kind 0: forward,  x [n][nz][ny][nx][cin], w [27][cout][cin], bias [cout] or NULL
             -> out = ReLU(conv + bias) [n][nz][ny][nx][cout], rounded to BF16
     kind 1: weight gradient, x as above, dy [n][nz][ny][nx][cout]
             -> out [27][cout][cin] = sum over positions of dy * x(shifted by the tap), FP32
   (cin, cout) one of the network's pairs: (16,16) (16,32) (16,48) (32,16) (32,32) (32,64)
   (32,96) (48,16) (64,32) (64,64) (96,32); for kind 0 also (1,16), the network's input
   layer without medium features. */
mcx_status mcx_debug_conv3d(int32_t kind, int32_t n, int32_t nz, int32_t ny, int32_t nx,
                            int32_t cin, int32_t cout, const float *x, const float *w,
                            const float *bias, const float *dy, float *out);

#ifdef __cplusplus
}
#endif
#endif /* MCX_H */
