/*
 * FP64 CPU oracle for the voxel Monte Carlo photon walk.  TEST INFRASTRUCTURE ONLY:
 * see mcx_oracle.h.  Plain, slow and written step by step in the order the method
 * takes them; one photon at a time, every segment deposited straight into the map.
 *
 * Photon loop (paper: "a photon simulation loop is carried out within each computing
 * thread", workflow paragraph beside Fig. 1; physics per the benchmark description beside
 * Fig. 2 and the MCML formulation):
 *   launch -> repeat { draw a hop if none is pending (the first one, or one that rounding
 *   used up at a face); move to the nearest of (voxel face, scattering point, end of the
 *   time window); deposit the absorbed weight w(1 - exp(-mua l)) in the (gate, voxel) of
 *   the segment start; then handle the event: time-out, face (pass / Fresnel reflect /
 *   refract / escape + detector), or scatter (Henyey-Greenstein + rotation with the next
 *   hop drawn alongside, then Russian roulette) }.
 *
 * The paper defers the photon physics to the MCX/MCML formulation, so where it is silent
 * this file takes these readings (each is repeated where it applies): voxel (i,j,k) covers
 * [i h, (i+1) h) on each axis and label 0 or anything outside the grid is the exterior;
 * the photon starts inside the medium with weight 1 and no specular loss; hops are in
 * mean free paths, and the nearest of face, scattering point and time limit ends a
 * segment (faces tie to the lowest axis, the time limit wins every tie); the deposit goes
 * to the gate of the segment's start; unpolarised Fresnel reflectance with Snell
 * refraction and total internal reflection; Russian roulette after each scattering event
 * below w_min = 1e-4 with survival 1/m, m = 10; a detector takes an escaping photon whose
 * exit point lies within its radius, the lowest id winning.
 */
#include "mcx_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_C0 299.792458          /* mm / ns */
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------------------
 * Random numbers.  Each photon has its own xorshift128+ stream (Vigna, "Further
 * scramblings of Marsaglia's xorshift generators", shifts 23/18/5), seeded from the
 * SplitMix64 sequence of the run seed (Steele, Lea & Flood 2014): photon p takes outputs
 * number 2p+1 and 2p+2.  Events that need one uniform (the first hop, Fresnel, roulette)
 * take the top 23 bits of one output; the Gaussian launch point takes two, the top 23
 * bits and bits 40..18; a scattering event takes three from one output, bits 63..43 for
 * the next hop, 42..22 for the deflection and 21..1 for the azimuth.  Bit 0 of a sum of
 * the two state words is linear over GF(2) (linear complexity 128) and is never used;
 * bit 1 is quadratic (linear complexity 8256); higher bits are of higher degree.  The hop
 * goes through a logarithm, so its rare long hops are decided by its uniform's low-order
 * bits: it takes the top field, and the azimuth, linear in its uniform, the bottom one.
 * This is the per-thread independent seeding of the paper's workflow, made per photon so
 * a run is a pure function of (seed, photon ids).
 *
 * Compiled with -DORC_FULL_RES_DRAWS (a test-only build) every uniform instead takes its
 * own generator output at 53 bits, so tests can measure what the 21- and 23-bit draws do
 * to the results.
 * ---------------------------------------------------------------------------------- */
static uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64_output(uint64_t seed, uint64_t k)
{
    /* the generator's state advances by the golden-ratio increment before each output */
    return sm64_mix(seed + k * 0x9E3779B97F4A7C15ULL);
}

typedef struct { uint64_t s0, s1; } orc_rng;

static void rng_init(orc_rng *g, uint64_t seed, uint64_t photon)
{
    g->s0 = orc_splitmix64_output(seed, 2 * photon + 1);
    g->s1 = orc_splitmix64_output(seed, 2 * photon + 2);
    if (g->s0 == 0 && g->s1 == 0) g->s1 = 1;   /* the all-zero state is not allowed */
}

static uint64_t rng_next(orc_rng *g)
{
    uint64_t a = g->s0;
    const uint64_t b = g->s1;
    const uint64_t result = a + b;
    g->s0 = b;
    a ^= a << 23;
    g->s1 = a ^ b ^ (a >> 18) ^ (b >> 5);
    return result;
}

#ifdef ORC_FULL_RES_DRAWS
/* uniform in (0,1) from the top 53 bits k of one output: (k + 1/2) 2^-53 */
static double rng_u53(orc_rng *g)
{
    return ((double)(rng_next(g) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}
#endif

/* uniform in (0,1): the top 23 bits k give (2k+1) * 2^-24, exact in float and double */
static double rng_uniform(orc_rng *g)
{
#ifdef ORC_FULL_RES_DRAWS
    return rng_u53(g);
#endif
    const uint64_t k = rng_next(g) >> 41;
    return (double)(2 * k + 1) * (1.0 / 16777216.0);
}

/* two uniforms from one output, for events that need two (Gaussian launch point,
   scattering): the top 23 bits give the first and bits 40..18 the second, each as
   (2k+1) 2^-24 */
static void rng_uniform_pair(orc_rng *g, double *u1, double *u2)
{
#ifdef ORC_FULL_RES_DRAWS
    *u1 = rng_u53(g);
    *u2 = rng_u53(g);
    return;
#endif
    const uint64_t r = rng_next(g);
    *u1 = (double)(2 * (r >> 41) + 1) * (1.0 / 16777216.0);
    *u2 = (double)(2 * ((r >> 18) & 0x7FFFFFULL) + 1) * (1.0 / 16777216.0);
}

/* three uniforms from one output, for a scattering event (next hop, deflection,
   azimuth): bits 63..43, 42..22 and 21..1, each as (2k+1) 2^-22 */
static void rng_uniform_triple(orc_rng *g, double *u1, double *u2, double *u3)
{
#ifdef ORC_FULL_RES_DRAWS
    *u1 = rng_u53(g);
    *u2 = rng_u53(g);
    *u3 = rng_u53(g);
    return;
#endif
    const uint64_t r = rng_next(g);
    *u1 = (double)(2 * (r >> 43) + 1) * (1.0 / 4194304.0);
    *u2 = (double)(2 * ((r >> 22) & 0x1FFFFFULL) + 1) * (1.0 / 4194304.0);
    *u3 = (double)(2 * ((r >> 1) & 0x1FFFFFULL) + 1) * (1.0 / 4194304.0);
}

void orc_uniforms(uint64_t seed, uint64_t photon, uint64_t n, double *out)
{
    orc_rng g;
    rng_init(&g, seed, photon);
    for (uint64_t i = 0; i < n; ++i) out[i] = rng_uniform(&g);
}

void orc_uniform_pairs(uint64_t seed, uint64_t photon, uint64_t n, double *out)
{
    orc_rng g;
    rng_init(&g, seed, photon);
    for (uint64_t i = 0; i < n; ++i) rng_uniform_pair(&g, &out[2 * i], &out[2 * i + 1]);
}

void orc_uniform_triples(uint64_t seed, uint64_t photon, uint64_t n, double *out)
{
    orc_rng g;
    rng_init(&g, seed, photon);
    for (uint64_t i = 0; i < n; ++i) rng_uniform_triple(&g, &out[3 * i], &out[3 * i + 1], &out[3 * i + 2]);
}

void orc_xorshift_step(uint64_t state[2])
{
    orc_rng g;
    g.s0 = state[0];
    g.s1 = state[1];
    (void)rng_next(&g);
    state[0] = g.s0;
    state[1] = g.s1;
}

/* ------------------------------------------------------------------------------------
 * Henyey-Greenstein: inverse-CDF sample of the deflection cosine (Henyey & Greenstein
 * 1941; the closed-form inverse as used by MCML).  g = 0 is isotropic.
 * ---------------------------------------------------------------------------------- */
double orc_hg_cos(double g, double xi)
{
    double c;
    if (g != 0.0) {
        const double f = (1.0 - g * g) / (1.0 - g + 2.0 * g * xi);
        c = (1.0 + g * g - f * f) / (2.0 * g);
    } else {
        c = 2.0 * xi - 1.0;
    }
    if (c < -1.0) c = -1.0;
    if (c > 1.0) c = 1.0;
    return c;
}

/* New direction after deflection (cos_t, azimuth phi) of unit vector u: the MCML
   rotation, with the near-vertical case (|uz| > 1 - 1e-5) handled on the z axis. */
void orc_rotate(const double u[3], double cos_t, double phi, double out[3])
{
    const double sin_t = sqrt(1.0 - cos_t * cos_t);
    const double cp = cos(phi), sp = sin(phi);
    if (fabs(u[2]) > 1.0 - 1e-5) {
        out[0] = sin_t * cp;
        out[1] = sin_t * sp;
        out[2] = (u[2] > 0.0 ? 1.0 : -1.0) * cos_t;
    } else {
        const double tmp = sqrt(1.0 - u[2] * u[2]);
        out[0] = sin_t * (u[0] * u[2] * cp - u[1] * sp) / tmp + u[0] * cos_t;
        out[1] = sin_t * (u[1] * u[2] * cp + u[0] * sp) / tmp + u[1] * cos_t;
        out[2] = -sin_t * cp * tmp + u[2] * cos_t;
    }
}

/* Unpolarised Fresnel reflectance from medium n1 into n2 at incidence cosine cos_i;
   1 for total internal reflection. */
double orc_fresnel_R(double n1, double n2, double cos_i)
{
    const double sin_t2 = (n1 / n2) * (n1 / n2) * (1.0 - cos_i * cos_i);
    if (sin_t2 >= 1.0) return 1.0;
    const double cos_t = sqrt(1.0 - sin_t2);
    const double rs = (n1 * cos_i - n2 * cos_t) / (n1 * cos_i + n2 * cos_t);
    const double rp = (n1 * cos_t - n2 * cos_i) / (n1 * cos_t + n2 * cos_i);
    return 0.5 * (rs * rs + rp * rp);
}

int orc_rec_stride(uint32_t n_media)
{
    return 11 + (int)(n_media > 0 ? n_media - 1 : 0);
}

/* ------------------------------------------------------------------------------------
 * One photon.
 * ---------------------------------------------------------------------------------- */
typedef struct {
    double *energy;               /* this thread's map (or the shared one) */
    int shared_energy;            /* 1: add atomically */
    double tally[ORC_NTALLY];
    uint64_t count[ORC_NCOUNT];
    double *rec;                  /* this thread's detected records */
    uint64_t rec_n, rec_cap;
} orc_ctx;

static void deposit(orc_ctx *c, uint64_t idx, double dw)
{
    if (c->shared_energy) {
#ifdef _OPENMP
#pragma omp atomic
#endif
        c->energy[idx] += dw;
    } else {
        c->energy[idx] += dw;
    }
}

static uint8_t label_at(const orc_problem *P, const int64_t v[3])
{
    if (v[0] < 0 || v[1] < 0 || v[2] < 0 ||
        v[0] >= (int64_t)P->nx || v[1] >= (int64_t)P->ny || v[2] >= (int64_t)P->nz)
        return 0;
    return P->labels[((uint64_t)v[2] * P->ny + (uint64_t)v[1]) * P->nx + (uint64_t)v[0]];
}

static void add_record(orc_ctx *c, const orc_problem *P, uint64_t id, int det, uint32_t nscat,
                       double w, const double pos[3], const double dir[3], uint32_t n_rr,
                       const double *L)
{
    const int stride = orc_rec_stride(P->n_media);
    if (c->rec_n >= c->rec_cap) {
        uint64_t cap = c->rec_cap ? 2 * c->rec_cap : 1024;
        double *nr = (double *)realloc(c->rec, cap * (uint64_t)stride * sizeof(double));
        if (!nr) { c->rec_n++; return; }
        c->rec = nr;
        c->rec_cap = cap;
    }
    double *r = c->rec + c->rec_n * (uint64_t)stride;
    r[0] = (double)id; r[1] = det; r[2] = nscat; r[3] = w;
    r[4] = pos[0]; r[5] = pos[1]; r[6] = pos[2];
    r[7] = dir[0]; r[8] = dir[1]; r[9] = dir[2];
    r[10] = n_rr;
    for (uint32_t m = 1; m < P->n_media; ++m) r[10 + m] = L[m];
    c->rec_n++;
}

static void run_photon(const orc_problem *P, uint64_t id, orc_ctx *C, orc_exit *ex)
{
    enum { EV_TIME, EV_SCATTER, EV_FACE };
    const double h = P->h;
    const double t_end = P->dt * (double)P->n_gates;
    const uint64_t nvox = (uint64_t)P->nx * P->ny * P->nz;
    double L[256];
    memset(L, 0, sizeof(double) * P->n_media);

    orc_rng rng;
    rng_init(&rng, P->seed, id);

    /* launch: weight 1 at t = 0; pencil at src_pos, Gaussian offset by r, phi */
    double pos[3] = { P->src_pos[0], P->src_pos[1], P->src_pos[2] };
    double dir[3];
    {
        const double nrm = sqrt(P->src_dir[0] * P->src_dir[0] + P->src_dir[1] * P->src_dir[1] +
                                P->src_dir[2] * P->src_dir[2]);
        for (int a = 0; a < 3; ++a) dir[a] = P->src_dir[a] / nrm;
    }
    if (P->src_kind == 1) {
        /* I(r) ~ exp(-2 r^2 / w^2): r = w sqrt(-ln xi1 / 2), phi = 2 pi xi2, in the plane
           normal to the beam spanned by e1 = normalise(dir x z) (x when the beam is along
           z) and e2 = dir x e1. */
        double xi1, xi2;
        rng_uniform_pair(&rng, &xi1, &xi2);
        const double r = P->waist * sqrt(-log(xi1) / 2.0), ph = 2.0 * ORC_PI * xi2;
        double e1[3], e2[3];
        if (fabs(dir[2]) > 0.999999) { e1[0] = 1; e1[1] = 0; e1[2] = 0; }
        else {
            const double n1 = sqrt(dir[0] * dir[0] + dir[1] * dir[1]);
            e1[0] = dir[1] / n1; e1[1] = -dir[0] / n1; e1[2] = 0;
        }
        e2[0] = dir[1] * e1[2] - dir[2] * e1[1];
        e2[1] = dir[2] * e1[0] - dir[0] * e1[2];
        e2[2] = dir[0] * e1[1] - dir[1] * e1[0];
        for (int a = 0; a < 3; ++a) pos[a] += r * (cos(ph) * e1[a] + sin(ph) * e2[a]);
    }
    double w = 1.0, t = 0.0, s = 0.0;
    uint32_t nscat = 0, n_rr = 0;
    int64_t v[3];
    for (int a = 0; a < 3; ++a) {
        const double c = pos[a] / h;
        v[a] = (int64_t)floor(c);
        if (c == (double)v[a] && dir[a] < 0.0) v[a] -= 1;   /* on a face: the voxel ahead */
    }
    C->tally[ORC_T_LAUNCHED] += 1.0;
    int fate = ORC_FATE_NONE;
    uint8_t lab = label_at(P, v);
    if (lab == 0) {
        /* reading: a photon launched outside the labelled medium never enters it */
        C->tally[ORC_T_ESCAPED] += w;
        fate = ORC_FATE_MISSED;
    }
    uint64_t last_idx = UINT64_MAX;
    uint64_t nseg = 0;

    while (fate == ORC_FATE_NONE) {
        if (P->max_events && nseg >= P->max_events) {
            C->tally[ORC_T_TIME] += w;
            fate = ORC_FATE_CAPPED;
            break;
        }
        ++nseg;
        if (s <= 0.0) {                      /* new dimensionless hop, in mean free paths */
            s = -log(rng_uniform(&rng));
            C->count[ORC_C_HOPS]++;
        }
        const double *pr = P->props + 4 * (uint32_t)lab;
        const double mua = pr[0], mus = pr[1], g = pr[2], n = pr[3];

        /* distances to the scattering point, the nearest face (lowest axis on ties) and
           the end of the time window */
        const double d_scat = mus > 0.0 ? s / mus : INFINITY;
        double d_face = INFINITY, bound = 0.0;
        int axis = -1;
        for (int a = 0; a < 3; ++a) {
            if (dir[a] == 0.0) continue;
            const double b = (dir[a] > 0.0 ? (double)(v[a] + 1) : (double)v[a]) * h;
            double d = (b - pos[a]) / dir[a];
            if (d < 0.0) d = 0.0;
            if (d < d_face) { d_face = d; axis = a; bound = b; }
        }
        const double d_time = (t_end - t) * ORC_C0 / n;
        int ev;
        double l;
        if (d_time <= d_face && d_time <= d_scat) { ev = EV_TIME; l = d_time; }
        else if (d_scat <= d_face) { ev = EV_SCATTER; l = d_scat; }
        else { ev = EV_FACE; l = d_face; }

        /* move, age, and deposit into the (gate, voxel) of the segment start */
        int64_t gate = (int64_t)floor(t / P->dt);
        if (gate >= (int64_t)P->n_gates) gate = P->n_gates - 1;
        if (gate < 0) gate = 0;
        for (int a = 0; a < 3; ++a) pos[a] += l * dir[a];
        t += l * n / ORC_C0;
        s = (ev == EV_SCATTER) ? 0.0 : s - l * mus;
        L[lab] += l;
        const double dw = w * (1.0 - exp(-mua * l));
        w -= dw;
        if (P->n_gates > 0) {
            const uint64_t idx = (uint64_t)gate * nvox +
                ((uint64_t)v[2] * P->ny + (uint64_t)v[1]) * P->nx + (uint64_t)v[0];
            if (C->energy) deposit(C, idx, dw);
            if (dw > 0.0 && idx != last_idx) { C->count[ORC_C_RUNS]++; last_idx = idx; }
        }
        C->tally[ORC_T_ABSORBED] += dw;

        if (ev == EV_TIME) {
            C->tally[ORC_T_TIME] += w;
            fate = ORC_FATE_TIME;
        } else if (ev == EV_FACE) {
            C->count[ORC_C_FACE]++;
            pos[axis] = bound;               /* exactly on the face */
            int64_t nv[3] = { v[0], v[1], v[2] };
            nv[axis] += dir[axis] > 0.0 ? 1 : -1;
            const uint8_t b = label_at(P, nv);
            int escape = 0;
            if (b == lab) {
                v[axis] = nv[axis];          /* same medium: straight through */
            } else if (!P->reflect) {
                if (b == 0) escape = 1;      /* B1: the exterior terminates the photon */
                else { v[axis] = nv[axis]; lab = b; }
            } else {
                const double na = n, nb = P->props[4 * (uint32_t)b + 3];
                if (na == nb) {
                    if (b == 0) escape = 1;
                    else { v[axis] = nv[axis]; lab = b; }
                } else {
                    C->count[ORC_C_FRESNEL]++;
                    const double cos_i = fabs(dir[axis]);
                    const double eta = na / nb;
                    const double sin_t2 = eta * eta * (1.0 - cos_i * cos_i);
                    int refl;
                    if (sin_t2 >= 1.0) refl = 1;                 /* total internal reflection */
                    else refl = rng_uniform(&rng) < orc_fresnel_R(na, nb, cos_i);
                    if (refl) {
                        dir[axis] = -dir[axis];
                    } else {                 /* Snell: tangential x eta, normal = +-cos_t */
                        const double cos_t = sqrt(1.0 - sin_t2);
                        for (int a = 0; a < 3; ++a) if (a != axis) dir[a] *= eta;
                        dir[axis] = dir[axis] > 0.0 ? cos_t : -cos_t;
                        if (b == 0) escape = 1;
                        else { v[axis] = nv[axis]; lab = b; }
                    }
                }
            }
            if (escape) {
                C->tally[ORC_T_ESCAPED] += w;
                fate = ORC_FATE_ESCAPED;
                for (uint32_t d = 0; d < P->n_det; ++d) {
                    const double *dd = P->det + 4 * d;
                    const double dx = pos[0] - dd[0], dy = pos[1] - dd[1], dz = pos[2] - dd[2];
                    if (dx * dx + dy * dy + dz * dz <= dd[3] * dd[3]) {
                        C->count[ORC_C_DETECTED]++;
                        add_record(C, P, id, (int)d, nscat, w, pos, dir, n_rr, L);
                        break;               /* the lowest detector id wins */
                    }
                }
            }
        } else {                             /* scattering event */
            C->count[ORC_C_SCATTER]++;
            ++nscat;
            double u_hop, xi_hg, xi_phi;
            rng_uniform_triple(&rng, &u_hop, &xi_hg, &xi_phi);
            const double ct = orc_hg_cos(g, xi_hg);
            const double ph = 2.0 * ORC_PI * xi_phi;
            double nd[3];
            orc_rotate(dir, ct, ph, nd);
            dir[0] = nd[0]; dir[1] = nd[1]; dir[2] = nd[2];
            if (w < P->rr_threshold) {       /* Russian roulette after each scatter */
                C->count[ORC_C_ROULETTE]++;
                if (rng_uniform(&rng) < 1.0 / P->rr_m) {
                    C->tally[ORC_T_RR_GAINED] += (P->rr_m - 1.0) * w;
                    w *= P->rr_m;
                    ++n_rr;
                } else {
                    C->tally[ORC_T_RR_KILLED] += w;
                    fate = ORC_FATE_ROULETTE;
                }
            }
            if (fate == ORC_FATE_NONE) {     /* the next hop, drawn with the deflection */
                s = -log(u_hop);
                C->count[ORC_C_HOPS]++;
            }
        }
    }
    C->count[ORC_C_SEGMENTS] += nseg;
    if (ex) {
        ex->fate = fate;
        ex->nscat = nscat;
        for (int a = 0; a < 3; ++a) { ex->pos[a] = pos[a]; ex->dir[a] = dir[a]; }
        ex->w = w;
        ex->t = t;
    }
}

/* ------------------------------------------------------------------------------------
 * Run: contiguous photon-id ranges per thread; private maps summed in thread order when
 * they fit in memory, one shared map with atomic adds otherwise.
 * ---------------------------------------------------------------------------------- */
int orc_run(const orc_problem *P, orc_result *R)
{
    if (!P || !R || !P->labels || !P->props || P->n_media < 1 || P->n_media > 256 ||
        P->nx == 0 || P->ny == 0 || P->nz == 0 || !(P->h > 0.0) || !(P->dt > 0.0) ||
        P->n_gates == 0 || (P->n_det && !P->det) || (P->src_kind != 0 && P->src_kind != 1) ||
        (P->rr_threshold > 0.0 && !(P->rr_m > 1.0)))
        return -1;
    const uint64_t nvox = (uint64_t)P->nx * P->ny * P->nz;
    const uint64_t nen = nvox * P->n_gates;
    memset(R->tally, 0, sizeof(R->tally));
    memset(R->count, 0, sizeof(R->count));
    R->det_n = 0;
    if (R->energy) memset(R->energy, 0, nen * sizeof(double));
    if (R->exits) memset(R->exits, 0, R->exit_cap * sizeof(orc_exit));

    int nt = 1;
#ifdef _OPENMP
    nt = P->n_threads > 0 ? P->n_threads : omp_get_max_threads();
#endif
    if ((uint64_t)nt > P->n_photons && P->n_photons > 0) nt = (int)P->n_photons;
    if (nt < 1) nt = 1;
    /* private maps only while they stay under 8 GiB in total */
    const int private_maps = R->energy && nt > 1 &&
        (double)nen * 8.0 * nt < 8.0 * 1024 * 1024 * 1024;
    orc_ctx *ctx = (orc_ctx *)calloc((size_t)nt, sizeof(orc_ctx));
    if (!ctx) return -2;
    int fail = 0;
    for (int k = 0; k < nt; ++k) {
        if (private_maps) {
            ctx[k].energy = (double *)calloc(nen, sizeof(double));
            if (!ctx[k].energy) fail = 1;
        } else {
            ctx[k].energy = R->energy;
            ctx[k].shared_energy = nt > 1;
        }
    }
    if (!fail) {
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
        {
            int k = 0;
#ifdef _OPENMP
            k = omp_get_thread_num();
#endif
            const uint64_t lo = P->n_photons * (uint64_t)k / (uint64_t)nt;
            const uint64_t hi = P->n_photons * (uint64_t)(k + 1) / (uint64_t)nt;
            for (uint64_t i = lo; i < hi; ++i) {
                orc_exit *ex = (R->exits && i < R->exit_cap) ? &R->exits[i] : NULL;
                run_photon(P, P->photon_offset + i, &ctx[k], ex);
            }
        }
    }
    for (int k = 0; k < nt; ++k) {
        for (int j = 0; j < ORC_NTALLY; ++j) R->tally[j] += ctx[k].tally[j];
        for (int j = 0; j < ORC_NCOUNT; ++j) R->count[j] += ctx[k].count[j];
        if (private_maps && ctx[k].energy) {
            for (uint64_t i = 0; i < nen; ++i) R->energy[i] += ctx[k].energy[i];
            free(ctx[k].energy);
        }
        const int stride = orc_rec_stride(P->n_media);
        for (uint64_t i = 0; i < ctx[k].rec_n; ++i) {
            if (R->det_rec && R->det_n < R->det_cap && i < ctx[k].rec_cap)
                memcpy(R->det_rec + R->det_n * (uint64_t)stride,
                       ctx[k].rec + i * (uint64_t)stride, sizeof(double) * (size_t)stride);
            R->det_n++;
        }
        free(ctx[k].rec);
    }
    free(ctx);
    return fail ? -2 : 0;
}
