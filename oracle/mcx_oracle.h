/*
 * FP64 CPU oracle for the voxel Monte Carlo photon walk.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that the CUDA
 * path is checked against.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the product path never does.  It shares no code, header,
 * constant table or helper with the CUDA library.
 *
 * What it computes follows the paper's workflow (Fig. 1 and the paragraph describing it):
 * the host sets up the domain, the optical properties and independent per-photon random
 * streams; each photon runs the photon simulation loop; the results are the 3-D
 * (time-gated) absorbed-energy map, the detected-photon records and, here, the energy
 * tallies.  The loop's physics is the standard voxel MC formulation named in the paper's
 * benchmark description (exponential hops, voxel-face crossing, Snell/Fresnel at index
 * mismatches, Henyey-Greenstein scattering, Russian roulette), written from MCML
 * (Wang, Jacques & Zheng 1995), Henyey & Greenstein (1941) and the Fresnel equations.
 */
#ifndef MCX_ORACLE_H
#define MCX_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* photon fates */
enum { ORC_FATE_NONE = 0, ORC_FATE_ESCAPED = 1, ORC_FATE_ROULETTE = 2,
       ORC_FATE_TIME = 3, ORC_FATE_MISSED = 4, ORC_FATE_CAPPED = 5 };

/* tally slots */
enum { ORC_T_LAUNCHED = 0, ORC_T_ABSORBED = 1, ORC_T_ESCAPED = 2, ORC_T_TIME = 3,
       ORC_T_RR_KILLED = 4, ORC_T_RR_GAINED = 5, ORC_NTALLY = 6 };

/* event counters */
enum { ORC_C_SCATTER = 0, ORC_C_FACE = 1, ORC_C_FRESNEL = 2, ORC_C_RUNS = 3,
       ORC_C_ROULETTE = 4, ORC_C_HOPS = 5, ORC_C_SEGMENTS = 6, ORC_C_DETECTED = 7,
       ORC_NCOUNT = 8 };

typedef struct {
    /* volume: labels[z][y][x], x fastest; label 0 = exterior */
    uint32_t nx, ny, nz;
    double h;                     /* voxel edge, mm */
    const uint8_t *labels;
    /* media: props[m*4 + {0,1,2,3}] = mua /mm, mus /mm, g, n; row 0 = exterior */
    uint32_t n_media;
    const double *props;
    /* source */
    int32_t src_kind;             /* 0 pencil, 1 gaussian (1/e^2 waist) */
    double src_pos[3];            /* mm */
    double src_dir[3];            /* normalised by the oracle */
    double waist;                 /* mm */
    /* disk detectors: det[d*4 + {0,1,2,3}] = cx, cy, cz, r (mm) */
    uint32_t n_det;
    const double *det;
    /* run */
    uint64_t n_photons;
    uint64_t photon_offset;       /* first photon id */
    uint64_t seed;
    double dt;                    /* gate width, ns; gates start at t = 0 */
    uint32_t n_gates;
    int32_t reflect;              /* 1 = Fresnel/Snell at mismatches, 0 = terminate at exterior */
    double rr_threshold;          /* roulette weight threshold (0 disables roulette) */
    double rr_m;                  /* roulette survival factor m (survive with p = 1/m) */
    uint64_t max_events;          /* per-photon segment cap (0 = none) */
    int32_t n_threads;            /* 0 = OpenMP default */
} orc_problem;

typedef struct {
    int32_t fate;
    uint32_t nscat;
    double pos[3];                /* mm, where the photon ended */
    double dir[3];                /* direction at the end (refracted on escape) */
    double w;                     /* weight at the end */
    double t;                     /* ns */
} orc_exit;

typedef struct {
    double *energy;               /* [n_gates][nz][ny][nx] absorbed weight, or NULL */
    double tally[ORC_NTALLY];
    uint64_t count[ORC_NCOUNT];
    orc_exit *exits;              /* exits[i] for photon id photon_offset + i < exit_cap */
    uint64_t exit_cap;
    /* detected records, photon-id order: rec_stride = 11 + (n_media - 1) doubles:
       id, det, nscat, w, px, py, pz, ux, uy, uz, n_roulette_survived, L[1..n_media-1] */
    double *det_rec;
    uint64_t det_cap;
    uint64_t det_n;               /* records found (may exceed det_cap) */
} orc_result;

/* Runs the photons [photon_offset, photon_offset + n_photons).  Returns 0 on success,
   negative on invalid input. */
int orc_run(const orc_problem *p, orc_result *r);

/* Primitives, exported so tests can pin each against closed forms. */
uint64_t orc_splitmix64_output(uint64_t seed, uint64_t k);      /* k-th output, k >= 1 */
void orc_uniforms(uint64_t seed, uint64_t photon, uint64_t n, double *out);
void orc_uniform_pairs(uint64_t seed, uint64_t photon, uint64_t n, double *out);  /* 2n values */
void orc_uniform_triples(uint64_t seed, uint64_t photon, uint64_t n, double *out);  /* 3n values */
/* one xorshift128+ state transition of state[0..1] in place (the output is not formed) */
void orc_xorshift_step(uint64_t state[2]);
double orc_hg_cos(double g, double xi);
void orc_rotate(const double u[3], double cos_t, double phi, double out[3]);
double orc_fresnel_R(double n1, double n2, double cos_i);       /* returns 1 on TIR */
int orc_rec_stride(uint32_t n_media);

#ifdef __cplusplus
}
#endif
#endif
