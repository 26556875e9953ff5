// Internal interface between the C-ABI layer (api.cu) and the photon-walk kernels
// (walk.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "../../include/mcx.h"

namespace mcxg {

constexpr int kMaxMedia = 256;       // label values 0..255
constexpr int kMaxDetMedia = 33;     // media rows allowed when detectors are present
constexpr int kMaxDet = 64;
constexpr int kRecBase = 12;         // detected-record words before the partial paths
constexpr int kClaimChunk = 32;      // default photon ids a warp claims per global atomic
constexpr float kC0 = 299.792458f;   // mm/ns

// device status word bits
constexpr unsigned kStatusCapped = 1u;
constexpr unsigned kStatusDetOverflow = 2u;

// Per-run constants in the walk's precision R.
template <typename R>
struct RunConsts {
    R dt;                             // gate width, ns
    R inv_dt;                         // 1 / gate width
    R t_end;                          // n_gates * gate width, ns
    R src_pos[3];                     // voxel units
    R src_dir[3];                     // unit vector
    R src_e1[3], src_e2[3];           // Gaussian launch-plane basis
    R waist;                          // voxel units
    R rr_threshold;
    R rr_m;
    R rr_inv_m;
};

// One simulation of a batch (all lengths in its own voxel units).
struct BatchSim {
    const uint8_t *labels;            // [nz][ny][nx]
    float *fluence;                   // accum 0: [n_gates][nvox]
    double *fluence64;                // accum 2: [n_gates][nvox]
    double *tally;                    // [MCX_NTALLY], FP64 atomics
    unsigned long long first;         // first flattened photon index of this simulation
    unsigned long long n_photons;
    unsigned long long seed;
    int nx, ny, nz;
    unsigned nvox;                    // voxels of the padded volume (nx+2)(ny+2)(nz+2)
    unsigned sy, sz;                  // padded strides: nx + 2, (nx + 2)(ny + 2)
    int tab0;                         // first row of this simulation in the batch tables
    int src_kind;
    float src_pos[3], src_dir[3], src_e1[3], src_e2[3], waist;
};

struct WalkParams {
    // Volumes (labels and the accumulation maps) carry a one-voxel exterior border on every
    // side ([nz+2][ny+2][nx+2]) except in the allocation-free run, whose caller-owned
    // buffers are unpadded; nvox, sy and sz describe the layout actually used.
    const uint8_t *labels;            // [nz][ny][nx] (+ border)
    float *fluence;                   // [n_gates][nvox] absorbed weight; accum 1: [n_gates][nvox][2]
                                      // compensated (hi, lo) pairs, the two words adjacent
    double *fluence64;                // accum 2: [n_gates][nvox]; accum 1: the tile's FP64 map
    int tile_lo[4];                   // accum 1: tile origin (x, y, z, gate)
    int tile_size[4];                 // accum 1: tile extent; entries = product
    const void *tab_a;                // [n_media] MedA<R>: mus, 1/mus, mua (voxel units), c0/(n h)
    const void *tab_b;                // [n_media] MedB<R>: g, 1-g^2, 1+g^2, 1/(2g)
    const void *tab_n;                // [n_media] R: refractive index
    const void *tab_tpl;              // [n_media] R: ns per voxel length, n h / c0
    const float4 *det;                // [n_det] cx, cy, cz, r^2 in voxel units
    float *det_buf;                   // [max_detected][rec_stride] words
    unsigned long long *det_count;
    unsigned long long *photon_counter;
    mcx_exit *exits;                  // [exit_log]
    double *block_tally;              // [grid][MCX_NTALLY]
    unsigned long long *block_stats;  // [grid][MCX_NSTAT]
    unsigned *status;

    int nx, ny, nz;                   // the volume's voxels (without border)
    unsigned nvox;                    // voxels per gate of the maps (with border, if any)
    unsigned sy, sz;                  // linear strides of y and z in the labels and maps
    int src_kind;
    int n_media;
    int n_det;
    int rec_stride;
    unsigned n_gates;
    float h;                          // voxel edge, mm

    // per-run constants, given in both precisions so the walk never converts in its loop
    RunConsts<float> cf;
    RunConsts<double> cd;

    unsigned long long n_photons;
    unsigned long long photon_offset;
    unsigned long long seed;
    unsigned long long max_detected;
    unsigned long long exit_log;
    unsigned long long max_events;
    int reflect;
    int claim_static;                 // 1: static per-thread photon split
    unsigned claim_chunk;             // photon ids a warp claims per global atomic (>= 32)
    const BatchSim *sims;             // batch: [n_sims], ordered by `first`
    int n_sims;
};

struct LaunchShape {
    int grid, block, blocks_per_sm, regs;
};

// Walk precision: the FP32 product path, or the same kernel in FP64 (trajectory-parity
// diagnostic; FP64 runs at a small fraction of the FP32 rate on this part).
enum class Precision { F32 = 0, F64 = 1 };

// walk.cu
size_t walk_table_bytes(Precision prec, int n_media);   // bytes of the 4 tables together
void walk_fill_tables(Precision prec, int n_media, const float *props, float h, void *host_buf,
                      const void **tab_a_off, const void **tab_b_off, const void **tab_n_off,
                      const void **tab_tpl_off);        // offsets into the buffer
// accumulation modes (mcx_run_cfg.accum_mode)
enum { kAccPlain = 0, kAccCompensated = 1, kAccF64 = 2 };
constexpr int kTileMaxEntries = 6144;  // (gate, voxel) pairs per block tile, 48 KiB

cudaError_t walk_query_shape(bool detectors, Precision prec, int accum, int block, int n_media,
                             int n_det, int tile_entries, bool claim_static, LaunchShape *shape);
cudaError_t walk_launch(const WalkParams &p, Precision prec, int accum, const LaunchShape &shape,
                        cudaStream_t stream);
// batch walk: FP32 photon state, accumulation 0 or 2, no detectors or exit log
cudaError_t walk_batch_query_shape(int accum, int block, LaunchShape *shape);
// unpadded caller-owned volume and map (allocation-free run): FP32 walk, no detectors,
// accumulation 0 or 2
cudaError_t walk_query_shape_unpadded(int accum, int block, LaunchShape *shape);
cudaError_t walk_launch_unpadded(const WalkParams &p, int accum, const LaunchShape &shape,
                                 cudaStream_t stream);
cudaError_t walk_batch_launch(const WalkParams &p, int accum, const LaunchShape &shape,
                              cudaStream_t stream);
// Gaussian launch plane of a beam along unit vector d: e1 = normalise(d x z) (x when the
// beam is along z), e2 = d x e1.
inline void launch_plane(const double d[3], double e1[3], double e2[3])
{
    if (d[2] > 0.999999 || d[2] < -0.999999) {
        e1[0] = 1; e1[1] = 0; e1[2] = 0;
    } else {
        double n1 = d[0] * d[0] + d[1] * d[1];
        n1 = n1 > 0 ? 1.0 / __builtin_sqrt(n1) : 0.0;
        e1[0] = d[1] * n1; e1[1] = -d[0] * n1; e1[2] = 0;
    }
    e2[0] = d[1] * e1[2] - d[2] * e1[1];
    e2[1] = d[2] * e1[0] - d[0] * e1[2];
    e2[2] = d[0] * e1[1] - d[1] * e1[0];
}

// api.cu: the error text mcx_last_error(NULL) returns (per host thread)
void set_global_error(const std::string &msg);

cudaError_t debug_uniforms(uint64_t seed, uint64_t photon, uint64_t n, float *dev_out);
cudaError_t debug_primitive(int kind, uint64_t n, const float *dev_in, float *dev_out);

// Padded volume layout: index of voxel (x, y, z) of an nx x ny volume in its bordered copy.
__host__ __device__ inline unsigned long long padded_index(unsigned x, unsigned y, unsigned z,
                                                        unsigned nx, unsigned ny)
{
    return ((unsigned long long)(z + 1) * (ny + 2) + (y + 1)) * (nx + 2) + (x + 1);
}

}  // namespace mcxg
