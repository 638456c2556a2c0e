/*
 * qmpm.h -- C ABI of libqmpm: the quantized MLS-MPM time step of
 * "Automatic Quantization for Physics-Based Simulation" (Liu et al., SIGGRAPH 2022)
 * on bit-packed fixed-point particle state, for NVIDIA B300 (sm_103a).
 *
 * Conventions for every entry point
 *   - Return value: QMPM_OK (0) or a negative QMPM_ERR_* code; the message of the last
 *     failure on the calling thread is available from qmpm_last_error().
 *   - Pointers named h_* are host memory, d_* are device memory.  Caller-owned buffers
 *     are only read or written during the call (or, for the *_async calls, until the
 *     handle's stream reaches the enqueued work); the library keeps no reference.
 *   - A qmpm_handle owns every device allocation it makes; qmpm_destroy frees them.
 *     A handle is not thread-safe; separate handles may run on separate streams.
 *   - Particle state on the host is an array of doubles, n_comp values per particle,
 *     in the canonical component order x[d], v[d], C[d*d] (row major), then F[d*d]
 *     (row major, elastic materials) or J (fluid); n_comp = 2d + d^2 + (d^2 or 1).
 *   - Packed words use word planes: word j of particle slot p lives at
 *     words[j * ld + p].  Record bit b of a particle is bit (b & 31) of its word
 *     (b >> 5); a component occupies bits [bitpos, bitpos + bits).
 */
#ifndef QMPM_H
#define QMPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QMPM_OK 0
#define QMPM_ERR_INVALID_ARG (-1)
#define QMPM_ERR_OOM (-2)
#define QMPM_ERR_SCHEME (-3)   /* field wider than 24 bits, |offset| >= 2^24, bad layout */
#define QMPM_ERR_CUDA (-4)
#define QMPM_ERR_TIMEOUT (-5)  /* a bounded device wait expired */
#define QMPM_ERR_OVERFLOW (-6) /* strict mode: a store saturated */

#define QMPM_MAX_COMP 24
#define QMPM_MAX_FIELD_BITS 24

enum { QMPM_NEOHOOKEAN = 0, QMPM_COROTATED = 1, QMPM_FLUID = 2 };
enum { QMPM_FIELD_X = 0, QMPM_FIELD_V = 1, QMPM_FIELD_C = 2, QMPM_FIELD_F = 3 };

#define QMPM_FLAG_STATS 1  /* count saturations and round-ups/-downs per field */
#define QMPM_FLAG_STRICT 2 /* qmpm_readback fails with QMPM_ERR_OVERFLOW after a saturation */
#define QMPM_FLAG_PROFILE 4 /* record CUDA events around each launch group (qmpm_profile) */

/* Scene: one MLS-MPM simulation (the simulator quantized in Sec. 8.1).
 * Grid: n = 2^grid_log2 nodes per axis (n >= 16), dx = 1/n; sticky walls zero the grid
 * velocity within `bound` nodes of each face.  Particles keep a tile order: they are
 * stably re-sorted by (tile, cell) at initialisation and after every `resort_every`-th
 * step (0 disables later re-sorts), where the tile is the 2^d-block group of 4^d-node
 * grid blocks that holds the particle's stencil and the cell is its stencil base inside
 * the tile.  The dither counter of a store is the particle's slot in this order. */
typedef struct {
    int32_t dim;          /* 2 or 3 */
    int32_t material;     /* QMPM_NEOHOOKEAN, QMPM_COROTATED, QMPM_FLUID */
    int32_t grid_log2;    /* 4 .. 11 (2D), 4 .. 10 (3D) */
    int32_t bound;        /* >= 2 */
    int64_t n_particles;
    double dt;
    double E, nu;         /* elastic materials */
    double bulk;          /* fluid bulk modulus K */
    double p_vol, p_mass; /* per-particle volume and mass */
    double gravity[3];
    uint64_t seed;        /* key of the dither hash */
    int32_t dither;       /* 1: dithered stores (Sec. 5), 0: round to nearest */
    int32_t resort_every;
    int32_t chunk;        /* particles per CTA work item, 0 = default (256) */
    int32_t flags;        /* QMPM_FLAG_* */
} qmpm_scene_t;

/* One quantized type h (Sec. 3.1): values (u + offset) * 2^-frac, u in [0, 2^bits). */
typedef struct {
    int32_t bits;         /* 1 .. 24 */
    int32_t frac;         /* resolution Delta = 2^-frac */
    int64_t offset;       /* |offset| < 2^24 */
    int32_t container;    /* 0: bit pack (Sec. 7); 32 or 64: bit struct containers */
} qmpm_field_t;

/* Quantization scheme: one type per field x, v, C, F (or J), shared by the field's
 * components.  n_words and bitpos are outputs of qmpm_scheme_layout. */
typedef struct {
    int32_t quantized;    /* 0: plain FP32 state (the comparator), 1: fixed point */
    qmpm_field_t field[4];
    int32_t n_words;
    int32_t bitpos[QMPM_MAX_COMP];
} qmpm_scheme_t;

typedef struct {
    int64_t saturations[4];
    int64_t round_ups[4];
    int64_t round_downs[4];
    int64_t out_of_grid;  /* particle-steps whose stencil base left [0, n-3] */
    int64_t out_of_tile;  /* particle-steps that left their tile (slow path) */
    int64_t steps;        /* steps taken since qmpm_init */
    int64_t active_blocks;/* grid blocks (4^d nodes) holding mass for the current state */
    int32_t error_word;   /* 0, or a QMPM_ERR_* code raised on the device */
    int32_t n_words;
} qmpm_stats_t;

/* Device time per launch group, from CUDA events recorded on the handle's stream around
 * each group while QMPM_FLAG_PROFILE is set. */
typedef struct {
    double step_ms;          /* fused G2P -> store -> P2G kernel */
    int64_t step_launches;
    double clear_ms;         /* grid-buffer clear kernel */
    int64_t clear_launches;
    double sort_ms;          /* a whole re-sort: keys, radix passes, gather, chunk list */
    int64_t sort_calls;
    double p2g_ms;           /* stand-alone P2G (initialisation, after an upload) */
    int64_t p2g_launches;
    int64_t kernel_launches; /* every kernel the library launched since the last reset */
} qmpm_profile_t;

typedef struct qmpm_ctx *qmpm_handle;

/* ---- scheme (host only) --------------------------------------------------------- */

/* Place the scheme's fields in the particle record (Sec. 7, Fig. 6/7).  Fields go in
 * the order x, v, C, F/J.  container 0 (bit pack): components follow bit by bit and may
 * straddle a 32-bit word; consecutive bit-pack fields form one stream.  container 32/64
 * (bit struct): the field starts a new container on a 32-bit boundary, components never
 * cross a container, a component that does not fit opens the next one, and the field's
 * last container is used in full.  Fills scheme->n_words and scheme->bitpos.
 * Errors: QMPM_ERR_INVALID_ARG (dim/material), QMPM_ERR_SCHEME (bits outside 1..24,
 * |offset| >= 2^24, unknown container). */
int qmpm_scheme_layout(int32_t dim, int32_t material, qmpm_scheme_t *scheme);

/* Input of the bit-allocation solve (Sec. 4, Eq. 6-10, Algorithm 1).  For each type h:
 * P_h variables, accumulated squared sensitivity g_h (Eq. 8), recorded range [lo_h, hi_h]
 * (widened by kappa about its midpoint, Sec. 3.1). */
typedef struct {
    int32_t H;            /* 1 .. 8 */
    double P[8], g[8], lo[8], hi[8];
    double kappa;         /* range factor, e.g. 2 */
    double z;             /* reference evaluation value */
    double eps;           /* eps_err (error mode) or eps_mem (memory mode) */
    int32_t mode;         /* 0: error bound (Eq. 6), 1: memory bound (Eq. 7) */
    int32_t rounding;     /* 0: Algorithm 1's ceil (memory mode: floor then greedy),
                             1: exact integer search around it */
} qmpm_solve_in_t;

typedef struct {
    double delta_cont[8]; /* continuous optimum Delta_h (Eq. 10, or its memory form) */
    int32_t bits_paper[8];/* ceil(-log2(Delta_h / R_h)) as in Algorithm 1 */
    int32_t bits[8];      /* power-of-two scheme */
    int32_t frac[8];
    int64_t offset[8];
    double pred_err;      /* (1/12) sum Delta_h^2 g_h (Eq. 8) of the scheme */
    double total_bits;    /* sum P_h bits_h */
} qmpm_solve_out_t;

/* Solve for a scheme.  Error mode: Delta_h of Eq. 10, b_h = ceil(-log2(Delta_h/R_h)),
 * then Delta_h rounded down to a power of two (frac_h = ceil(-log2 Delta_h)) and the
 * bits that cover the widened range at that resolution.  Memory mode (budget
 * eps * 32 * sum P_h bits): Delta_h^2 g_h = c P_h with c fixed by the budget, bits
 * floored and then raised greedily by error reduction per bit while within budget.
 * Pure host, deterministic.  Errors: QMPM_ERR_INVALID_ARG, QMPM_ERR_SCHEME (no feasible
 * scheme in the search window). */
int qmpm_scheme_solve(const qmpm_solve_in_t *in, qmpm_solve_out_t *out);

/* ---- simulation --------------------------------------------------------------- */

/* Create a scene on the current CUDA device.  h_state: the initial state (host, see the
 * conventions above), encoded on the device with the dithered store of step 0 and then
 * sorted into tile order.  scheme NULL (or quantized == 0) keeps FP32 state.  stream:
 * a cudaStream_t (NULL = legacy default stream); every later call on the handle is
 * ordered on it.  Errors: QMPM_ERR_INVALID_ARG, QMPM_ERR_SCHEME, QMPM_ERR_OOM,
 * QMPM_ERR_CUDA. */
int qmpm_init(const qmpm_scene_t *scene, const qmpm_scheme_t *scheme, const double *h_state,
              void *stream, qmpm_handle *out);

/* Enqueue nsteps MLS-MPM steps (P2G, grid update, G2P, dithered store, Eq. 1) on the
 * handle's stream; returns without waiting.  Errors: QMPM_ERR_INVALID_ARG,
 * QMPM_ERR_CUDA (launch failure). */
int qmpm_step(qmpm_handle h, int32_t nsteps);

/* Copy the state out (synchronises the stream).  Any pointer may be NULL.
 * h_state: decoded values in FP64, slot order, [n_particles][n_comp];
 * h_words: packed words, [n_words][n_particles] (plane layout, ld = n_particles);
 * h_ids:   original particle index of each slot.
 * Errors: QMPM_ERR_CUDA, QMPM_ERR_OVERFLOW (strict mode), QMPM_ERR_TIMEOUT. */
int qmpm_readback(qmpm_handle h, double *h_state, uint32_t *h_words, int64_t *h_ids,
                  qmpm_stats_t *stats);

/* Position measurement z = (1/N) sum_p |x_p|^2 of the current state (a form of the
 * evaluation function Z of Eq. 2), reduced on the device in FP64.  Synchronises. */
int qmpm_measure(qmpm_handle h, double *z);

/* End-to-end step with host buffers: enqueue the copy of h_words_in (pinned host,
 * plane layout, ld = n_particles) into the device state, nsteps steps, and the copy of
 * the state back into h_words_out, then wait for the stream.  Either pointer may be
 * NULL to skip that copy. */
int qmpm_step_host(qmpm_handle h, int32_t nsteps, const uint32_t *h_words_in,
                   uint32_t *h_words_out);

/* Collect the device times recorded since the last reset (synchronises the stream).
 * reset != 0 clears the totals afterwards.  Kernel launches are counted whether or not
 * QMPM_FLAG_PROFILE is set. */
int qmpm_profile(qmpm_handle h, qmpm_profile_t *out, int32_t reset);

/* Device pointers of the resident packed state (word planes, leading dimension *ld)
 * and of the slot ids; valid until the next step or destroy. */
int qmpm_state_device(qmpm_handle h, uint32_t **d_words, int64_t *ld, int64_t **d_ids);

int qmpm_destroy(qmpm_handle h);

/* Message of the last failure on the calling thread ("" if none). */
const char *qmpm_last_error(void);

/* ---- reverse mode (Sec. 6, Eq. 12-13) and the sensitivities of Eq. 8 ------------ */

#define QMPM_MEASURE_MEAN_SQ_POS 0 /* z = (1/N) sum |x_T|^2, seed 2 x_T / N */
#define QMPM_MEASURE_USER 1        /* seed dz/ds_T supplied by the caller (z reported as
                                      the mean square position) */
#define QMPM_MEASURE_KINETIC_ENERGY 2 /* z = (1/2) m sum |v_T|^2, seed m v_T (Sec. 8.1) */

typedef struct {
    double z;          /* the measurement of s_T (kinetic energy for that measure, else the
                          mean square position) */
    double g[4];       /* Eq. 8: sum over t = 0..T and over the field's variables of (dz/ds_t)^2 */
    double lo[4];      /* smallest value of each field over the states t = 0..T */
    double hi[4];      /* largest value (Algorithm 1's range update) */
    int64_t P[4];      /* variables per field: N times the field's components */
} qmpm_adjoint_out_t;

/* Reverse mode over T steps from the handle's current state, in FP32 (the state is decoded
 * first if the handle is quantized; gradients are taken in full precision as in the
 * paper's workflow).  The call runs its own forward (particle order fixed, no re-sort),
 * keeps a checkpoint every ckpt_every steps and recomputes each segment from its
 * checkpoint while reversing it (adjoint kernel G of Eq. 13), and accumulates the squared
 * sensitivities g_h of Eq. 8, which qmpm_scheme_solve takes.  The handle's own state is
 * not advanced.
 *   measure:  QMPM_MEASURE_MEAN_SQ_POS, QMPM_MEASURE_KINETIC_ENERGY or QMPM_MEASURE_USER
 *             (then d_seed = dz/ds_T, device, [N][n_comp] in the handle's slot order);
 *   d_grad0:  optional output dz/ds_0, device, [N][n_comp], slot order.
 * Allocates O((T/ckpt_every + ckpt_every) N n_comp) floats of device memory for the call.
 * Errors: QMPM_ERR_INVALID_ARG, QMPM_ERR_OOM, QMPM_ERR_CUDA. */
int qmpm_adjoint(qmpm_handle h, int32_t T, int32_t ckpt_every, int32_t measure, const float *d_seed,
                 float *d_grad0, qmpm_adjoint_out_t *out);

/* ---- codec on device buffers (Sec. 3.1 Eq. 3, Sec. 5 Eq. 11, Sec. 7) ------------ */

/* Encode N particles of FP32 values d_vals ([N][n_comp], device) into d_words
 * (word planes, leading dimension ld >= N, device) with the dithered store of
 * `step`, slot p = particle index.  stats may be NULL.  Asynchronous on `stream`
 * except when stats != NULL (then it waits). */
int qmpm_pack_f32(int32_t dim, int32_t material, const qmpm_scheme_t *scheme, uint64_t seed,
                  int32_t dither, uint32_t step, const float *d_vals, int64_t N, uint32_t *d_words,
                  int64_t ld, qmpm_stats_t *stats, void *stream);

/* Decode word planes into FP32 values [N][n_comp] (device).  Asynchronous. */
int qmpm_unpack_f32(int32_t dim, int32_t material, const qmpm_scheme_t *scheme,
                    const uint32_t *d_words, int64_t N, int64_t ld, float *d_vals, void *stream);

/* ---- ordering without device allocation ----------------------------------------- */

/* Largest N accepted by qmpm_tile_order_static. */
#define QMPM_STATIC_SORT_MAX 262144

/* The stable (tile, cell) order of N packed records -- the order qmpm_init puts particles
 * in -- computed without allocating anything.  It exists for callers that cannot call
 * cudaMalloc or cudaFree: code that runs inside another runtime's memory pool or
 * allocator, or a host thread that must not take the device-wide synchronisation an
 * allocation or a free can cause.  The paper has no counterpart; it is a service of this
 * library.
 *   d_words: N records as word planes (leading dimension ld >= N), device, in the layout
 *            of `scheme` (NULL or quantized == 0: FP32 state, one word per component);
 *   d_order: output, device, N slots: d_order[i] is the input index of the record that
 *            goes to slot i (equal keys keep their input order).
 * Scratch: one file-scope device array of about 4.3 MB (four key/value buffers of
 * QMPM_STATIC_SORT_MAX entries plus the radix digit counts), which every GPU that loads
 * the library holds until the process exits.  All calls share it and it keeps the last
 * call's contents; every word a call reads is written earlier in the same call, so
 * nothing has to be cleared.  Calls whose work overlaps on the GPU (other streams or
 * threads) race on the array: order them.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  Asynchronous on `stream` after the lookup.
 * Errors: QMPM_ERR_INVALID_ARG (N > QMPM_STATIC_SORT_MAX, bad dim/material/grid/buffers),
 * QMPM_ERR_SCHEME, QMPM_ERR_CUDA. */
int qmpm_tile_order_static(int32_t dim, int32_t material, int32_t grid_log2, const qmpm_scheme_t *scheme,
                           const uint32_t *d_words, int64_t N, int64_t ld, uint32_t *d_order, void *stream);

#ifdef __cplusplus
}
#endif
#endif
