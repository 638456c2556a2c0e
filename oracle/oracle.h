/*
 * oracle.h -- CPU oracle for the quantized MLS-MPM time step of
 * "Automatic Quantization for Physics-Based Simulation" (Liu et al., SIGGRAPH 2022).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded FP64 restatement
 * of what the hot path computes, used to check the CUDA library.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or helper with the CUDA library, and it never calls into it.
 *
 * Conventions
 *   - Particle state is an AoS array of doubles, n_comp values per particle, in the
 *     canonical component order  x[d], v[d], C[d*d] (row major), then F[d*d] (row major,
 *     elastic materials) or J (fluid).
 *   - Grid nodes: n = 2^grid_log2 nodes per axis, dx = 1/n, node (i,j[,k]) sits at
 *     (i,j[,k])*dx.  The oracle's grid is a dense row-major array of (1+d) doubles per
 *     node: mass, then momentum (after P2G) or velocity (after the grid update).
 *   - Packed words: AoS, n_words 32-bit words per particle; record bit b is bit (b & 31)
 *     of word (b >> 5); a component occupies bits [bitpos, bitpos + bits).
 *
 * Parity status of each function is listed in its comment; every function here is
 * pinned by a "not gpu" test against facts fixed by the paper or by mathematics.
 */
#ifndef QMPM_ORACLE_H
#define QMPM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_COMP 24

enum { OR_NEOHOOKEAN = 0, OR_COROTATED = 1, OR_FLUID = 2 };
enum { OR_FIELD_X = 0, OR_FIELD_V = 1, OR_FIELD_C = 2, OR_FIELD_F = 3 };

typedef struct {
    int dim;            /* 2 or 3 */
    int material;       /* OR_NEOHOOKEAN, OR_COROTATED, OR_FLUID */
    int grid_log2;      /* n = 2^grid_log2 */
    int bound;          /* sticky-wall width in nodes */
    double dt;
    double E, nu;       /* Young's modulus, Poisson ratio (elastic) */
    double bulk;        /* bulk modulus K (fluid) */
    double p_vol, p_mass;
    double gravity[3];
} or_phys_t;

typedef struct {
    int n_comp;
    int n_words;
    int bits[OR_MAX_COMP];
    int frac[OR_MAX_COMP];          /* resolution 2^-frac */
    int64_t offset[OR_MAX_COMP];    /* value = (u + offset) * 2^-frac */
    int bitpos[OR_MAX_COMP];
    int field[OR_MAX_COMP];         /* 0..3: x, v, C, F/J */
    uint64_t seed;                  /* dither hash key */
    int dither;                     /* 1: dithered store (Sec. 5), 0: round to nearest */
} or_codec_t;

/* stats: per field h (0..3): saturations, round-ups, round-downs; then out-of-grid count */
#define OR_STAT_SAT(h)  (h)
#define OR_STAT_UP(h)   (4 + (h))
#define OR_STAT_DOWN(h) (8 + (h))
#define OR_STAT_OOG     12
#define OR_N_STATS      13

/* ---- counter-based generator (Philox4x32, Salmon et al. SC'11; 10 rounds, the dither 7) ---- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Philox4x32 with `rounds` rounds; the dither draws take OR_DITHER_ROUNDS */
void or_philox4x32(const uint32_t ctr[4], const uint32_t key[2], int rounds, uint32_t out[4]);
#define OR_DITHER_ROUNDS 7
/* dither draw for (slot, step, comp): Philox(ctr={slot, step, comp/4, 0}, key=seed)[comp%4] */
uint32_t or_dither_draw(uint64_t seed, uint32_t slot, uint32_t step, int comp);

/* ---- fixed-point codec (Sec. 3.1 Eq. 3, Sec. 5 Eq. 11) ---- */
uint32_t or_encode(double v, int bits, int frac, int64_t offset, int dither, uint32_t r, int *flags);
double or_decode(uint32_t u, int frac, int64_t offset);
#define OR_FLAG_SAT  1
#define OR_FLAG_UP   2
#define OR_FLAG_DOWN 4

/* ---- bit pack / bit struct placement (Sec. 7) ---- */
int or_n_comp(int dim, int material);
int or_comp_field(int dim, int material, int comp);
/* container[h]: 0 = bit pack stream, 32 or 64 = bit struct containers.  Returns 0 or -1. */
int or_layout(int dim, int material, const int *bits, const int container[4],
              int *bitpos, int *n_words);
void or_pack(int n_comp, const int *bits, const int *bitpos, int n_words,
             const uint32_t *u, uint32_t *words);
void or_unpack(int n_comp, const int *bits, const int *bitpos, const uint32_t *words,
               uint32_t *u);

/* ---- MLS-MPM pieces ---- */
void or_lame(double E, double nu, double *mu, double *lambda);
void or_polar2(const double F[4], double R[4]);
void or_polar3(const double F[9], double R[9]);
/* Kirchhoff stress tau (d*d, row major) of one particle's F (or J for the fluid) */
void or_kirchhoff(const or_phys_t *ph, const double *FJ, double *tau);
int or_n_nodes(const or_phys_t *ph);
int64_t or_p2g(const or_phys_t *ph, int64_t N, const double *s, double *grid);
void or_grid_update(const or_phys_t *ph, double *grid);
int64_t or_g2p(const or_phys_t *ph, int64_t N, const double *grid, double *s);
int64_t or_step_fp64(const or_phys_t *ph, int64_t N, double *s, double *grid_scratch);
/* s += sign * sigma[field] * xi at every component: the store error of the noise-injection
 * estimate of the second-order term (xi uniform, unit variance, Philox counter (p, step,
 * c / 4, 0xA5), key seed). */
void or_add_noise(int dim, int material, int64_t N, double *s, uint32_t step, uint64_t seed,
                  const double sigma[4], double sign);
/* the same; matched != 0: sigma[h] = Delta_h, each store's variance Delta_h^2 Y (1 - Y) */
void or_add_noise_matched(int dim, int material, int64_t N, double *s, uint32_t step, uint64_t seed,
                          const double sigma[4], double sign, int matched);

/* ---- quantized state ---- */
void or_encode_state(const or_codec_t *cd, int64_t N, const double *s, uint32_t step,
                     uint32_t *words, int64_t *stats);
void or_decode_state(const or_codec_t *cd, int64_t N, const uint32_t *words, double *s);
/* one quantized step: decode -> FP64 step -> dithered encode with step index `step` */
void or_step_quant(const or_phys_t *ph, const or_codec_t *cd, int64_t N, uint32_t *words,
                   uint32_t step, double *s_scratch, double *grid_scratch, int64_t *stats);

/* ---- particle ordering ---- */
/* tile key of each particle: origin block of the 2^d-block tile that holds its stencil */
void or_tile_keys(const or_phys_t *ph, int64_t N, const double *s, int64_t *keys);
/* stable counting sort: perm[i] = old slot of the particle placed at new slot i */
void or_stable_sort(int64_t N, const int64_t *keys, int64_t n_keys, int64_t *perm);
int64_t or_n_keys(const or_phys_t *ph);

/* ---- measurement ---- */
double or_mean_sq_pos(int dim, int n_comp, int64_t N, const double *s);

/* ---- reverse mode (Sec. 6, Eq. 12-13) ---- */
/* sb = adjoint of s_t given sbn = adjoint of s_{t+1} = F(s_t) (FP64 step of or_step_fp64) */
void or_adjoint_step(const or_phys_t *ph, int64_t N, const double *s, const double *sbn, double *sb);

/* ---- scheme solve (Sec. 4.2 Eq. 8-10, Algorithm 1) ---- */
typedef struct {
    int H;
    double P[8];        /* number of variables of type h */
    double g[8];        /* accumulated squared gradients, Eq. 8 */
    double lo[8], hi[8];/* recorded ranges */
    double kappa;       /* range factor (Sec. 3.1) */
    double z;           /* reference evaluation value */
    double eps;         /* eps_err or eps_mem */
    int mode;           /* 0 = error bound (Eq. 6), 1 = memory bound (Eq. 7) */
    int rounding;       /* 0 = paper ceil (Alg. 1), 1 = exact integer */
} or_solve_in_t;

typedef struct {
    double delta_cont[8];   /* continuous optimum Delta_h */
    int bits_paper[8];      /* b_h = ceil(-log2(Delta_h / R_h)) */
    int bits[8];            /* power-of-two scheme: total bits n_h */
    int frac[8];            /* Delta_h = 2^-frac */
    int64_t offset[8];
    double pred_err;        /* (1/12) sum Delta_h^2 g_h for the final scheme */
    double total_bits;      /* sum P_h n_h */
    double pred_bias;       /* sum beta_h Delta_h^2 / 6 (or_scheme_options) */
    double pred_var_dither; /* sum g_h Delta_h^2 / 6 */
    int capped;             /* bit h: type h held at max_bits */
    int refined;            /* fraction bits added by the refinement */
} or_solve_out_t;

/* Options applied to a solved scheme, in this order: (1) max_bits > 0 holds each type at
 * max_bits bits over the same window, one power of two coarser per bit dropped; (2) refine
 * (error mode): while (sum beta Delta^2/6)^2 + sum g Delta^2/6 > (eps z)^2, one more
 * fraction bit (code range doubled, window kept) to the type with the largest decrease of
 * that sum per P_h (to every type when no single bit decreases it: biases of opposite
 * signs), bits never above max_bits (24 when 0); (3) margin_gain[h] > 0: type
 * h's window widened by margin_gain[h] * Delta_(margin_src[h]) on each side at h's
 * resolution, coarser while it needs more than max_bits bits. */
typedef struct {
    int max_bits;
    int refine;
    double beta[8];
    double margin_gain[8];
    int margin_src[8];
} or_solve_opt_t;

int or_scheme_options(const or_solve_in_t *in, const or_solve_opt_t *opt, or_solve_out_t *out);

int or_scheme_solve(const or_solve_in_t *in, or_solve_out_t *out);
/* brute force over integer frac_h in [lo, hi] for error mode (min bits s.t. error) or
 * memory mode (min error s.t. bits); returns the optimum's frac_h / bits */
int or_scheme_bruteforce(const or_solve_in_t *in, int frac_lo, int frac_hi, or_solve_out_t *out);

/* ---- 2D Eulerian smoke (Sec. 8.1: advection-reflection, quantized pressure and velocity) ---- */
typedef struct {
    int n;             /* n x n cells, h = 1/n */
    int jacobi;        /* Jacobi sweeps per projection */
    double dt;
    double buoyancy;   /* v += dt * buoyancy * density */
    double v_in;       /* inflow velocity inside the source box */
    double src[4];     /* source box x0, y0, x1, y1 */
    uint64_t seed;
    int dither;
} or_smoke_t;

typedef struct {       /* type 0: velocity (u and v), type 1: pressure q */
    int bits[2];
    int frac[2];
    int64_t offset[2];
} or_smoke_scheme_t;

/* One step in place; sch NULL for the unquantized step.  q receives the final pressure.
 * Returns the number of saturated stores. */
int64_t or_smoke_step(const or_smoke_t *sm, const or_smoke_scheme_t *sch, uint32_t step, double *u, double *v,
                      double *d, double *q);
double or_smoke_measure(const or_smoke_t *sm, const double *d);
/* one stage of the step from given stored inputs (see or_smoke.c) */
#define OR_SMOKE_ADVECT1 0
#define OR_SMOKE_JACOBI 1
#define OR_SMOKE_GRADSUB2 2
#define OR_SMOKE_ADVECT4 3
#define OR_SMOKE_GRADSUB5 4
int or_smoke_stage(const or_smoke_t *sm, const or_smoke_scheme_t *sch, int stage, int arg, uint32_t step,
                   const double *a_u, const double *a_v, const double *b_u, const double *b_v, const double *q,
                   const double *div, double *out_u, double *out_v, double *out2_u, double *out2_v, double *out_q);
/* inject delta at the store (field 0 u, 1 v, 2 q; sample index; store counter) while active */
void or_smoke_inject(int active, int field, uint32_t idx, uint32_t counter, double delta);
/* +-sigma_h noise at every store of type h but the reflection and the wall faces (signs
 * from Philox with key seed), times sign; active 0 turns it off */
void or_smoke_noise(int active, double sigma_v, double sigma_p, uint64_t seed, double sign);
/* record the oracle's own code of every store in order (buf NULL: off) */
void or_smoke_record(uint32_t *buf, int64_t n);
/* the same, also recording the value each store was offered (FP64, before the codec) */
void or_smoke_record_values(uint32_t *buf, double *xs, int64_t n);
int64_t or_smoke_recorded(void);

#ifdef __cplusplus
}
#endif
#endif
