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

#ifdef __CUDACC_RTC__
/* compiled at run time (the scheme-specialised step kernel): no C library headers */
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
#else
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define QMPM_OK 0
#define QMPM_ERR_INVALID_ARG (-1)
#define QMPM_ERR_OOM (-2)
#define QMPM_ERR_SCHEME (-3)   /* field wider than 24 bits, |offset| >= 2^24, bad layout */
#define QMPM_ERR_CUDA (-4)
#define QMPM_ERR_TIMEOUT (-5)  /* a bounded wait expired (qmpm_engine_wait) */
#define QMPM_ERR_OVERFLOW (-6) /* strict mode: a store saturated */
#define QMPM_ERR_QUEUE_FULL (-7) /* the serving queue holds max_queued requests */

#define QMPM_MAX_COMP 24
#define QMPM_MAX_FIELD_BITS 24

enum { QMPM_NEOHOOKEAN = 0, QMPM_COROTATED = 1, QMPM_FLUID = 2 };
enum { QMPM_FIELD_X = 0, QMPM_FIELD_V = 1, QMPM_FIELD_C = 2, QMPM_FIELD_F = 3 };

#define QMPM_FLAG_STATS 1  /* count saturations and round-ups/-downs per field */
#define QMPM_FLAG_STRICT 2 /* qmpm_readback fails with QMPM_ERR_OVERFLOW after a saturation */
#define QMPM_FLAG_PROFILE 4 /* record CUDA events around each launch group (qmpm_profile) */
#define QMPM_FLAG_SPECIALIZE 8 /* step with a kernel compiled at qmpm_init for this scheme (FP32
                                  state: for its word count; see qmpm_specialize_compile) */

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
    uint64_t seed;        /* key of the dither hash (Philox4x32-7, counter (slot, step, comp / 8, 0)) */
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
    /* Options, applied in this order after the solve; all zero gives the plain solve. */
    int32_t max_bits;     /* > 0: a type given more bits keeps its window at max_bits bits and
                             a resolution one power of two coarser per bit dropped (FP32
                             compute decodes exactly up to 24 bits) */
    int32_t refine;       /* 1 (error mode): the second-order refinement.  Eq. 6 bounds the
                             second moment of the error of z; Eq. 8 keeps its linear part.
                             With dithered stores (error variance Delta_h^2 / 6 averaged
                             over the fraction) the moments are bias = sum beta_h Delta_h^2
                             / 6 and var = sum g_h Delta_h^2 / 6; while bias^2 + var >
                             (eps z)^2, one fraction bit goes to the type with the largest
                             drop of bias^2 + var per stored bit (P_h; to every type when
                             no single bit lowers it, as when biases of opposite signs
                             cancel), never past max_bits (24 if 0), the window kept (its
                             code range doubles) */
    double beta[8];       /* second-order coefficients of z (qmpm_noise_moments' shift per
                             sigma_h^2), for refine */
    double margin_gain[8];/* > 0: type h's window is widened on each side by margin_gain[h]
                             times the solved resolution of type margin_src[h] (a field that
                             picks up another's store noise, e.g. the affine velocity C
                             takes about 6 n Delta_v from the dithered velocities), h keeping
                             its resolution (max_bits applies) */
    int32_t margin_src[8];
} qmpm_solve_in_t;

typedef struct {
    double delta_cont[8]; /* continuous optimum Delta_h (Eq. 10, or its memory form) */
    int32_t bits_paper[8];/* ceil(-log2(Delta_h / R_h)) as in Algorithm 1 */
    int32_t bits[8];      /* power-of-two scheme */
    int32_t frac[8];
    int64_t offset[8];
    double pred_err;      /* (1/12) sum Delta_h^2 g_h (Eq. 8) of the scheme */
    double total_bits;    /* sum P_h bits_h */
    double pred_bias;     /* sum beta_h Delta_h^2 / 6 (dithered stores) */
    double pred_var_dither; /* sum g_h Delta_h^2 / 6 */
    int32_t capped;       /* bit h set: type h was held at max_bits */
    int32_t refined;      /* fraction bits the refinement added */
} qmpm_solve_out_t;

/* Solve for a scheme.  Error mode: Delta_h of Eq. 10, b_h = ceil(-log2(Delta_h/R_h)),
 * then Delta_h rounded down to a power of two (frac_h = ceil(-log2 Delta_h)) and the
 * bits that cover the widened range at that resolution.  Memory mode (budget
 * eps * 32 * sum P_h bits): Delta_h^2 g_h = c P_h with c fixed by the budget, bits
 * floored and then raised greedily by error reduction per bit while within budget.
 * Pure host, deterministic.  Errors: QMPM_ERR_INVALID_ARG, QMPM_ERR_SCHEME (no feasible
 * scheme in the search window). */
int qmpm_scheme_solve(const qmpm_solve_in_t *in, qmpm_solve_out_t *out);

/* Edits of one type h (0 x, 1 v, 2 C, 3 F or J) of a quantized scheme, in place; the other
 * types are kept.  They serve the second-order refinement of a solved scheme and its
 * acceptance check (Sec. 4): a type's fixed point is its resolution 2^-frac and its window
 * [offset 2^-frac, (offset + 2^bits - 1) 2^-frac] (Sec. 3.1).  Each fails without touching
 * the scheme when the edited type would leave 1..24 bits or |offset| < 2^24
 * (QMPM_ERR_SCHEME), or on a NULL or unquantized scheme or h out of 0..3
 * (QMPM_ERR_INVALID_ARG).
 *
 * qmpm_scheme_shift: k fraction bits finer (k < 0: coarser) over the same window: bits and
 *   frac + k, offset 2^k (rounded down).
 * qmpm_scheme_widen: the window doubled about its middle at the same resolution: bits + 1,
 *   offset - 2^(bits - 1).
 * qmpm_scheme_window: the window set, at the type's resolution, to qmpm_scheme_solve's
 *   window of the recorded range [lo, hi] (kappa times its width about its middle), widened
 *   by gain 2^-frac[src] on each side (src < 0: no margin; the solve's window-margin
 *   option); grow != 0 keeps the union with the current window.  offset = floor(lo'
 *   2^frac), and the fewest bits that reach ceil(hi' 2^frac).  Also QMPM_ERR_INVALID_ARG
 *   unless lo <= hi, kappa > 0, gain >= 0.
 * qmpm_scheme_fill_words: the free bits of the last packed word (Sec. 7 bit pack) spent on
 *   wider windows: each type in type_mask (bit h) in turn has its window doubled while the
 *   layout for (dim, material) keeps its word count and the type stays within 24 bits,
 *   until none fits; *widened (may be NULL) receives the number of doublings.  Layout
 *   errors as qmpm_scheme_layout. */
int qmpm_scheme_shift(qmpm_scheme_t *scheme, int32_t h, int32_t k);
int qmpm_scheme_widen(qmpm_scheme_t *scheme, int32_t h);
int qmpm_scheme_window(qmpm_scheme_t *scheme, int32_t h, double lo, double hi, double kappa, int32_t src,
                       double gain, int32_t grow);
int qmpm_scheme_fill_words(int32_t dim, int32_t material, qmpm_scheme_t *scheme, int32_t type_mask,
                           int32_t *widened);

/* ---- simulation --------------------------------------------------------------- */

/* Create a scene on the current CUDA device.  h_state: the initial state (host, see the
 * conventions above), encoded on the device with the dithered store of step 0 and then
 * sorted into tile order.  scheme NULL (or quantized == 0) keeps FP32 state.  stream:
 * a cudaStream_t (NULL = legacy default stream); every later call on the handle is
 * ordered on it.  Errors: QMPM_ERR_INVALID_ARG, QMPM_ERR_SCHEME, QMPM_ERR_OOM,
 * QMPM_ERR_CUDA. */
int qmpm_init(const qmpm_scene_t *scene, const qmpm_scheme_t *scheme, const double *h_state,
              void *stream, qmpm_handle *out);

/* Device memory a handle of this scene and scheme holds (resident_bytes), and the most it
 * holds while qmpm_init runs (init_peak_bytes: plus the FP64 initial state).  Host only;
 * either pointer may be NULL.  Errors: QMPM_ERR_INVALID_ARG, QMPM_ERR_SCHEME. */
int qmpm_footprint(const qmpm_scene_t *scene, const qmpm_scheme_t *scheme, int64_t *resident_bytes,
                   int64_t *init_peak_bytes);

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

/* End-to-end rollout through host memory, pipelined: nsteps steps, each of which takes
 * its input state from h_words (pinned host, plane layout as qmpm_step_host, ld =
 * n_particles) and writes its result back into h_words.  Every step uploads the words,
 * clears the grid and redoes the P2G of the uploaded state (as qmpm_step_host), steps, and
 * downloads the result.  The copies are split into `chunks` particle ranges: downloads run
 * on a second stream owned by the handle, and the next step's upload of range j waits only
 * for the download of range j, so the two directions of the host link overlap.  On return
 * (the handle's stream and the copy stream synchronised) h_words holds the state after
 * nsteps steps.  chunks in [0, 64]; 0 picks one range per 16 MiB of packed state, between
 * 1 and 8.
 * Errors: QMPM_ERR_INVALID_ARG (bad handle, nsteps < 0, chunks out of range, NULL
 * h_words with work to do), QMPM_ERR_CUDA. */
int qmpm_step_host_stream(qmpm_handle h, int32_t nsteps, uint32_t *h_words, int32_t chunks);

/* The scheme-specialised step kernel (Sec. 3.1 Eq. 3 codec, Sec. 7 bit pack).  The step
 * kernel compiled with the library reads each component's codec (word, shift, straddle,
 * scale, offset) from its parameters; with QMPM_FLAG_SPECIALIZE, qmpm_init compiles the same
 * kernel source once more at run time (NVRTC, sm_103a) with the scene's codec table as
 * compile-time constants (FP32 state: its word count), and qmpm_step launches that kernel
 * for the G2P -> store -> P2G step (the priming P2G, batches and the adjoint keep the
 * library's kernels).  The results are those of the library's kernel: the arithmetic is
 * the same.  Compiled kernels are kept for the life of the process, one per (dim,
 * material, state, statistics and dither flags, codec table); a first compile takes about
 * a second.  The loaded kernels do not survive a device reset (cudaDeviceReset): a process
 * that resets the device must not ask for specialised kernels afterwards.  The kernel sources are read from the csrc/
 * directory beside the library file.
 *
 * qmpm_specialize_compile compiles (or finds) the kernel of a scheme without a device, for
 * warming the cache and for checking that the runtime compiler works: *seconds receives
 * the compile time of the first build, *cubin_bytes the size of the code (either may be
 * NULL).  stats != 0 takes the variant with saturation counters, dither != 0 the one with
 * dithered stores (the scene's dither flag is a compile-time constant of the kernel, as are
 * the record's word count and the codec table).
 * scheme NULL (or not quantized) compiles the FP32-state kernel, whose record word count is
 * the constant.
 * Errors: QMPM_ERR_INVALID_ARG (bad dim or material), QMPM_ERR_SCHEME (layout),
 * QMPM_ERR_CUDA (the runtime compiler failed: its log is in qmpm_last_error()). */
int qmpm_specialize_compile(int32_t dim, int32_t material, const qmpm_scheme_t *scheme, int32_t stats,
                            int32_t dither, double *seconds, int64_t *cubin_bytes);

/* Which step kernel the handle launches: *specialized = 1 for the scheme-specialised one
 * (QMPM_FLAG_SPECIALIZE), else 0; *compile_seconds = its compile time (0 if none).  Either
 * pointer may be NULL.  Errors: QMPM_ERR_INVALID_ARG (bad handle). */
int qmpm_step_kernel_info(qmpm_handle h, int32_t *specialized, double *compile_seconds);

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
#define QMPM_MEASURE_POSITIONS 3   /* the vector of final positions x_T (qmpm_noise_moments) */
#define QMPM_NOISE_MATCHED 0x200   /* qmpm_noise_moments: sigma[h] is Delta_h and each store gets its
                                      dithered store's variance Delta_h^2 Y (1 - Y) */
/* OR'ed into `measure`: the adjoint's forward follows the quantized trajectory of the
 * handle's scheme (each step's state goes through the dithered store, Eq. 1), so the
 * gradients and ranges are taken at the quantized solution -- one round of the iterative
 * re-linearisation of Sec. 4.  Requires a quantized handle. */
#define QMPM_ADJ_QUANTIZED_FORWARD 0x100

typedef struct {
    double z;          /* the measurement of s_T (kinetic energy for that measure, else the
                          mean square position) */
    double g[4];       /* Eq. 8: sum over t = 0..T and over the field's variables of (dz/ds_t)^2 */
    double lo[4];      /* smallest value of each field over the states t = 0..T */
    double hi[4];      /* largest value (Algorithm 1's range update) */
    int64_t P[4];      /* variables per field: N times the field's components */
    int64_t forward_steps; /* forward steps run, the first pass and the recomputation */
    int32_t state_buffers; /* FP32 states held at once (checkpoints and recomputed ones) */
    int32_t pad;
} qmpm_adjoint_out_t;

#define QMPM_CKPT_BISECTION 0 /* ckpt_every value: bisection checkpoints (Sec. 6) */

/* The bisection schedule of qmpm_adjoint over T steps (Sec. 6, Fig. 7): the states
 * s_0..s_T are the leaves of a binary tree whose inner nodes are checkpoints at the first
 * leaf of their subtree; reversing step t needs s_t, recomputed from the nearest checkpoint
 * on the path from the root, which places new checkpoints halfway on the way.  Op kinds:
 *   QMPM_OP_ADVANCE: slot `to` := F^(t1 - t0)(state in slot `from`, which holds s_t0);
 *   QMPM_OP_REVERSE: dz/ds_t0 = G(state s_t0 in slot `from`, dz/ds_(t0 + 1)).
 * Writes up to max_ops ops to ops (may be NULL to count), the op count to *n_ops, and the
 * number of state slots used to *n_slots (floor(log2 T) + 1 for T >= 1).  Host only.
 * Errors: QMPM_ERR_INVALID_ARG (T < 0, or more ops than max_ops). */
enum { QMPM_OP_ADVANCE = 0, QMPM_OP_REVERSE = 1 };
typedef struct {
    int32_t kind;
    int32_t from, to;
    int32_t t0, t1;
} qmpm_rev_op_t;
int qmpm_bisection_schedule(int32_t T, qmpm_rev_op_t *ops, int64_t max_ops, int64_t *n_ops, int32_t *n_slots);

/* Reverse mode over T steps from the handle's current state, in FP32 (the state is decoded
 * first if the handle is quantized; gradients are taken in full precision as in the
 * paper's workflow).  The call runs its own forward (particle order fixed, no re-sort),
 * keeps a checkpoint every ckpt_every steps and recomputes each segment from its
 * checkpoint while reversing it (adjoint kernel G of Eq. 13), and accumulates the squared
 * sensitivities g_h of Eq. 8, which qmpm_scheme_solve takes.  ckpt_every =
 * QMPM_CKPT_BISECTION follows qmpm_bisection_schedule instead: O(log T) states held,
 * about (T/2) log2 T forward steps recomputed.  The handle's own state is not advanced.
 *   measure:  QMPM_MEASURE_MEAN_SQ_POS, QMPM_MEASURE_KINETIC_ENERGY or QMPM_MEASURE_USER
 *             (then d_seed = dz/ds_T, device, [N][n_comp] in the handle's slot order);
 *   d_grad0:  optional output dz/ds_0, device, [N][n_comp], slot order.
 * Allocates O((T/ckpt_every + ckpt_every) N n_comp) floats (bisection: O(log T N n_comp))
 * of device memory for the call.
 * Errors: QMPM_ERR_INVALID_ARG, QMPM_ERR_OOM, QMPM_ERR_CUDA. */
int qmpm_adjoint(qmpm_handle h, int32_t T, int32_t ckpt_every, int32_t measure, const float *d_seed,
                 float *d_grad0, qmpm_adjoint_out_t *out);

typedef struct {
    double z0;         /* the noise-free FP32 run's measurement */
    double shift;      /* mean over pairs of (z+ + z-) / 2 - z0: the second-order shift */
    double shift_se;   /* its standard error */
    double spread;     /* mean over pairs of ((z+ - z-) / 2)^2: the first-order variance */
    double spread_se;
    int32_t pairs;
    int32_t pad;
} qmpm_noise_out_t;

/* The moments of z under an explicit error injected at every store, by antithetic pairs
 * of FP32 runs (the forward of qmpm_adjoint: the same MLS-MPM step, from the handle's
 * current state, fixed particle order).  Eq. 6 bounds the second moment of the error of z;
 * Eq. 8 keeps its linear part only, so zero-mean store errors also shift the mean of z at
 * second order (half the Hessian against their covariance).  Run k (k < n_pairs) adds to
 * component c of particle p after step t (t = 1..T) the error sign * sigma[h(c)] * xi,
 * xi uniform on [-sqrt 3, sqrt 3) (unit variance) from Philox4x32-10 with counter
 * (p, t, c / 4, 0xA5) and key seed0 + k, once with sign +1 and once with -1; then
 *   shift  = mean_k ((z+ + z-) / 2 - z0)   ~ sum_h beta_h sigma_h^2  (second order),
 *   spread = mean_k ((z+ - z-) / 2)^2      ~ sum_h g_h sigma_h^2     (Eq. 8's linear term).
 * With sigma_h = Delta_h / sqrt 6 (the variance of a dithered store, averaged over the
 * fraction) the shift estimates the mean error of the quantized runs; with measure |
 * QMPM_NOISE_MATCHED and sigma_h = Delta_h (a power of two) each store gets the variance
 * its dithered store has, Delta_h^2 Y (1 - Y) with Y the fraction of x / Delta_h (a value
 * on the lattice is stored without error), which the second-order term depends on.  measure:
 * QMPM_MEASURE_MEAN_SQ_POS or QMPM_MEASURE_KINETIC_ENERGY (z a scalar), or
 * QMPM_MEASURE_POSITIONS (the evaluation is the vector of final positions): then with
 * m_k = (x+ + x-)/2 - x0 per particle, shift = |b|^2, the squared norm of the bias vector
 * b = E[m], estimated without the noise of the mean as (K |mean_k m_k|^2 - mean_k |m_k|^2)
 * / (K - 1), and spread = mean_k sum_p |(x+ - x-)/2|^2; z0 = mean |x_T|^2.  Synchronous;
 * allocates up to five FP32 states and a dense grid for the call.  Errors:
 * QMPM_ERR_INVALID_ARG (n_pairs < 2, negative sigma), QMPM_ERR_OOM, QMPM_ERR_CUDA. */
int qmpm_noise_moments(qmpm_handle h, int32_t T, int32_t measure, const double *sigma, uint64_t seed0,
                       int32_t n_pairs, qmpm_noise_out_t *out);

/* ---- several scenes in one launch ------------------------------------------------- */

typedef struct qmpm_batch *qmpm_batch_handle;

#define QMPM_BATCH_GRAPHS 1 /* replay each half period (resort_every steps) as a CUDA graph */

typedef struct {
    int32_t n_members;
    int32_t n_classes;        /* multi-scene launches: (dim, material, quantized, stats) classes */
    int32_t resort_every;
    int32_t n_solo;           /* members with a launch of their own (at least 1024 chunks) */
    int64_t particles;        /* over all members */
    int64_t steps;            /* batch steps run */
    int64_t kernel_launches;  /* kernels launched directly or captured, since creation */
    int64_t graph_launches;   /* graph replays */
} qmpm_batch_info_t;

/* A batch steps several scenes together: every step runs one persistent step launch per
 * launch class over the concatenated chunk lists of its members (a work queue of
 * (scene, chunk) items with per-scene parameters: grid, scheme, physics, buffers,
 * dither step index), one clear launch for all consumed grid buffers, and each member's
 * re-sort when it falls due.  A member with at least 1024 chunks (about 260,000
 * particles), which fills the GPU alone, gets a persistent launch of its own instead.  Members keep their own state, results and step count: a
 * scene stepped in a batch goes through the same sequence of stores and re-sorts as one
 * stepped alone with the same resort_every (only the order of floating-point atomic
 * additions differs).
 *   stream: the batch's stream (NULL: the batch creates one); members' work is ordered on
 *           it while they belong to the batch (qmpm_batch_add makes it wait for the
 *           scene's stream, qmpm_batch_remove makes the scene's stream wait for it);
 *   resort_every: the members' re-sort interval while in the batch (0: never);
 *   flags: QMPM_BATCH_GRAPHS.
 * Errors: QMPM_ERR_INVALID_ARG, QMPM_ERR_CUDA. */
int qmpm_batch_create(void *stream, int32_t resort_every, int32_t flags, qmpm_batch_handle *out);

/* Add a scene (not in another batch; at most 256 members).  Membership changes rebuild the
 * batch's tables (and graphs) at the next qmpm_batch_step. */
int qmpm_batch_add(qmpm_batch_handle b, qmpm_handle h);
int qmpm_batch_remove(qmpm_batch_handle b, qmpm_handle h);

/* Enqueue nsteps steps of every member on the batch's stream (asynchronous).  With
 * QMPM_BATCH_GRAPHS, runs of resort_every steps that start on a half-period boundary are
 * graph replays.  A member may still be stepped or read alone between calls. */
int qmpm_batch_step(qmpm_batch_handle b, int32_t nsteps);

int qmpm_batch_info(qmpm_batch_handle b, qmpm_batch_info_t *out);

/* Remove every member (their streams and re-sort intervals are restored) and free the
 * batch. */
int qmpm_batch_destroy(qmpm_batch_handle b);

/* ---- autotuning ------------------------------------------------------------------ */

typedef struct {
    int32_t chunk;             /* best particles per work item (qmpm_scene_t.chunk) */
    int32_t resort_every;      /* best re-sort interval */
    double best_ms_per_step;
    int32_t n_candidates;
    int32_t from_cache;        /* 1: answered from this process's cache, nothing was timed */
    int32_t chunk_cand[16], resort_cand[16];
    double ms_per_step[16];    /* device time per step of each candidate, re-sorts included */
} qmpm_tune_t;

/* Time the step of this scene for every candidate chunk in {64, 128, 192, 256} and
 * re-sort interval in {4, 8, 16, 32} (scratch scenes created from h_state on a private
 * stream, each stepped 2 + trial_steps steps rounded up to whole re-sort periods) and
 * return the fastest.  The result is cached per (dim, material, quantized, words per
 * particle, grid, round(log2 N)) for the process; use_cache != 0 answers from the cache
 * when it can.  The caller applies the result (qmpm_scene_t.chunk, .resort_every); it
 * changes the particle order and so the dither draws, not the method.  Errors:
 * QMPM_ERR_INVALID_ARG, QMPM_ERR_SCHEME, QMPM_ERR_OOM, QMPM_ERR_CUDA. */
int qmpm_autotune(const qmpm_scene_t *scene, const qmpm_scheme_t *scheme, const double *h_state,
                  int32_t trial_steps, int32_t use_cache, qmpm_tune_t *out);

/* ---- serving: continuous batching of arriving scenes ------------------------------ */

typedef struct qmpm_engine *qmpm_engine_handle;

enum { QMPM_REQ_QUEUED = 0, QMPM_REQ_RUNNING = 1, QMPM_REQ_DONE = 2, QMPM_REQ_FAILED = 3 };

typedef struct {
    int64_t budget_bytes;  /* device memory the admitted scenes may hold (qmpm_footprint) */
    int32_t resort_every;  /* the batch's re-sort interval; also the longest iteration */
    int32_t max_active;    /* scenes stepping at once, 1 .. 256 */
    int32_t flags;         /* QMPM_BATCH_GRAPHS */
    int32_t max_queued;    /* requests waiting for admission at most (0: no limit) */
} qmpm_engine_config_t;

typedef struct {
    int64_t id;
    int32_t status;        /* QMPM_REQ_DONE or QMPM_REQ_FAILED */
    int32_t error;         /* QMPM_ERR_* of a failed request */
    int32_t steps;
    int32_t pad;
    int64_t particles;
    int64_t resident_bytes;
    double t_submit, t_admit, t_done; /* seconds since the engine was created (host clock) */
    double z;              /* mean square position of the final state (qmpm_measure) */
} qmpm_request_t;

typedef struct {
    int64_t queued, active, finished;
    int64_t bytes_in_use;
    int64_t particle_steps;  /* stepped so far, all requests */
    int64_t iterations;
    int64_t kernel_launches, graph_launches;
    double elapsed;          /* seconds since creation */
} qmpm_engine_stats_t;

/* A serving engine on the current device.  Requests (scene, scheme, initial state, step
 * count) wait in a FIFO queue and are admitted, in order, while the next one's peak
 * footprint fits under budget_bytes and fewer than max_active scenes run.  Admitted scenes
 * step together in one batch (see qmpm_batch_*); each iteration runs up to resort_every
 * steps, and scenes join and leave between iterations while the others keep running.  A
 * new scene's upload, encode and sort run on a second stream, overlapping the batch.
 * Finished scenes are measured, optionally read back, and freed.  Creation is host only;
 * the engine's streams, events and batch are made by the first iteration (an iteration on
 * a host without a usable device fails with QMPM_ERR_CUDA after admission has run).
 * Errors: QMPM_ERR_INVALID_ARG. */
int qmpm_engine_create(const qmpm_engine_config_t *cfg, qmpm_engine_handle *out);

#define QMPM_SUBMIT_KEEP_STATE 1 /* keep the final state for qmpm_engine_result */
#define QMPM_SUBMIT_BORROW 2     /* read h_state at admission instead of copying it now: the
                                    caller keeps it unchanged until the request is polled */

/* Queue a request; the engine copies h_state (host, as for qmpm_init) unless flags has
 * QMPM_SUBMIT_BORROW.  The request is checked before it is queued: the scene (as
 * qmpm_init), the scheme (as qmpm_scheme_layout), steps >= 0 and every initial value
 * finite (a corrupted request is refused, not simulated).  Thread-safe.  Errors:
 * QMPM_ERR_INVALID_ARG, QMPM_ERR_SCHEME, QMPM_ERR_QUEUE_FULL (max_queued requests wait
 * already), QMPM_ERR_OOM (host allocation).  A request larger than the budget fails with
 * QMPM_ERR_OOM when it reaches the head of the queue. */
int qmpm_engine_submit(qmpm_engine_handle e, const qmpm_scene_t *scene, const qmpm_scheme_t *scheme,
                       const double *h_state, int32_t steps, int32_t flags, int64_t *id);

/* Run the loop on a background thread until qmpm_engine_stop (drain != 0: after every
 * submitted request has finished). */
int qmpm_engine_start(qmpm_engine_handle e);
int qmpm_engine_stop(qmpm_engine_handle e, int32_t drain);

/* Or run `iterations` iterations in the calling thread (not while the thread runs);
 * *busy = 0 once nothing is queued, running or finishing.  Errors: QMPM_ERR_INVALID_ARG,
 * QMPM_ERR_CUDA (the engine's device setup failed). */
int qmpm_engine_run(qmpm_engine_handle e, int32_t iterations, int32_t *busy);

/* Wait at most timeout_s seconds (host clock) for the engine to become idle: nothing
 * queued, admitted, running or finishing.  The waiting is done by the engine's thread
 * (qmpm_engine_start); without it the queue does not move and the wait expires unless the
 * engine is idle already.  *busy (may be NULL) = 1 if work remains.  Errors:
 * QMPM_ERR_INVALID_ARG, QMPM_ERR_TIMEOUT (the deadline passed with work remaining). */
int qmpm_engine_wait(qmpm_engine_handle e, double timeout_s, int32_t *busy);

/* Take up to max finished requests (oldest first).  Thread-safe. */
int qmpm_engine_poll(qmpm_engine_handle e, qmpm_request_t *out, int32_t max, int32_t *n_out);

/* Final state of a polled request submitted with keep_state (decoded FP64, slot order, as
 * qmpm_readback), kept until qmpm_engine_release.  Either pointer may be NULL. */
int qmpm_engine_result(qmpm_engine_handle e, int64_t id, double *h_state, int64_t *h_ids);
int qmpm_engine_release(qmpm_engine_handle e, int64_t id);

int qmpm_engine_stats(qmpm_engine_handle e, qmpm_engine_stats_t *out);

/* Stop the thread (without draining), free every scene and the engine. */
int qmpm_engine_destroy(qmpm_engine_handle e);

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

/* ---- host-side fault injection ------------------------------------------------- */

/* Kinds of injected faults.  None touches a GPU: the library reports the failure where the
 * real one would be detected, so that callers' recovery paths can be tested. */
#define QMPM_FAULT_DEVICE_ALLOC 0 /* a device allocation of qmpm_init fails: QMPM_ERR_OOM */
#define QMPM_FAULT_HOST_ALLOC 1   /* the host allocation of a request in qmpm_engine_submit
                                     fails: QMPM_ERR_OOM */
#define QMPM_FAULT_WAIT 2         /* qmpm_engine_wait expires at once: QMPM_ERR_TIMEOUT */
#define QMPM_FAULT_KINDS 3

/* Arm `kind`: the next `after` occurrences pass, the `count` after them fail (count 0
 * disarms).  Process-wide and thread-safe.  Errors: QMPM_ERR_INVALID_ARG. */
int qmpm_fault_inject(int32_t kind, int64_t after, int64_t count);
/* How many faults of `kind` were injected since the last qmpm_fault_clear. */
int qmpm_fault_hits(int32_t kind, int64_t *hits);
/* Disarm every kind and reset the counts. */
int qmpm_fault_clear(void);

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
 * array's device address (cudaGetSymbolAddress) with that device current; with lazy module
 * loading (the CUDA default) that lookup may load the library's device code, which can
 * synchronise the device, so make that first call early: before any stream capture and
 * outside the code that must not allocate.  The address is kept for the life of the
 * process; a cudaDeviceReset between calls is not supported.  Asynchronous on `stream`
 * after the lookup.
 * Errors: QMPM_ERR_INVALID_ARG (N > QMPM_STATIC_SORT_MAX, bad dim/material/grid/buffers),
 * QMPM_ERR_SCHEME, QMPM_ERR_CUDA. */
int qmpm_tile_order_static(int32_t dim, int32_t material, int32_t grid_log2, const qmpm_scheme_t *scheme,
                           const uint32_t *d_words, int64_t N, int64_t ld, uint32_t *d_order, void *stream);

#ifdef __cplusplus
}
#endif
#endif
