/*
 * qmpm_smoke.h -- C ABI of the quantized 2D Eulerian smoke of libqmpm: the
 * advection-reflection solver of the paper's second error-bounded experiment (Sec. 8.1:
 * semi-Lagrangian advection with RK-3 paths, 64 Jacobi sweeps for the pressure Poisson
 * equation, evaluation z = sum of squared density, pressure and velocity quantized), run
 * for a batch of independent scenes on one B300 (sm_103a).
 *
 * The conventions of qmpm.h hold (QMPM_OK / QMPM_ERR_* returns, qmpm_last_error(),
 * h_* host and d_* device pointers, the library keeps no reference to caller buffers).
 *
 * Grid and step.  n x n cells of size h = 1/n on [0,1]^2 (n a multiple of 32), MAC layout
 * with walls on all four sides:
 *   u  x-faces, n rows of n+1:  u[j][i] at (i h, (j+1/2) h)
 *   v  y-faces, n+1 rows of n:  v[j][i] at ((i+1/2) h, j h)
 *   d, q  cells, n rows of n:   at ((i+1/2) h, (j+1/2) h)
 * One step: forces (density 1 and v = v_in inside the source box, buoyancy
 * v += dt b (average of the two adjacent cells' density)); u~ = A(u; u, dt/2);
 * u' = P(u~); u^ = 2u' - u~; u~2 = A(u^; u', dt/2); u'' = P(u~2); d = A(d; u', dt).
 * A(f; w, s) traces each sample point back along w with Ralston's RK-3 and interpolates f
 * bilinearly (sample point clamped into f's lattice); P(w) runs `jacobi` sweeps from q = 0
 * of lap q = div w with zero normal derivative (a cell divides by its number of interior
 * neighbours) and subtracts grad q on the interior faces; boundary faces are zero.
 *
 * Quantized stores (Sec. 3.1, Sec. 5).  Every store of a velocity value (u~, u', u^, u~2,
 * u'': stores 1-5 of a step) and of every Jacobi iterate of q goes through the fixed-point
 * codec of its type (0 velocity, 1 pressure) and is kept in HBM as a bit stream of
 * `bits` per value; density stays FP32.  The store counter of the k-th store of step t
 * (t = 1, 2, ...) is 1024 t + k.  With dither on, the threshold of the store of sample i of
 * field f (0 u, 1 v, 2 q; i the row-major index in the layout above) is the 16-bit draw of
 * Philox4x32-7 (the dither generator) with key = the scene's seed, counter (i / 8, counter, f, 0), lane i % 8
 * (the same rule as the particle codec's component lanes).
 */
#ifndef QMPM_SMOKE_H
#define QMPM_SMOKE_H

#include <stdint.h>

#include "qmpm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t n;          /* cells per side: a multiple of 32, 32 .. 4096 */
    int32_t jacobi;     /* sweeps per projection, 0 .. 500 (Sec. 8.1 uses 64) */
    float dt;
    float buoyancy;     /* v += dt * buoyancy * density */
    float v_in;         /* inflow velocity inside the source box */
    double src[4];      /* source box x0, y0, x1, y1 in [0,1]; a sample is inside when its
                           position ((i + 1/2) h for cells, j h for y-faces) lies in the box,
                           compared in FP64 */
    int32_t dither;     /* 1: dithered stores (Sec. 5), 0: round to nearest */
    int32_t flags;      /* QMPM_SMOKE_RANGES: record the range of every type's stored values;
                           QMPM_SMOKE_PROFILE: time the Jacobi sweeps (qmpm_smoke_profile) */
} qmpm_smoke_config_t;

#define QMPM_SMOKE_RANGES 1
#define QMPM_SMOKE_PROFILE 2  /* plain launches with CUDA events around the Jacobi sweeps */

/* Type 0: velocity (u and v), type 1: pressure q.  value = (code + offset) * 2^-frac,
 * code in [0, 2^bits); bits 1 .. 24, |offset| < 2^24. */
typedef struct {
    int32_t bits[2];
    int32_t frac[2];
    int64_t offset[2];
} qmpm_smoke_scheme_t;

typedef struct qmpm_smoke *qmpm_smoke_handle;

typedef struct {
    int32_t n, jacobi, n_scenes, quantized;
    int64_t steps;              /* steps run */
    int64_t state_bytes;        /* u, v, d of one scene as stored (packed velocity) */
    int64_t state_bytes_fp32;   /* the same in FP32 */
    int64_t device_bytes;       /* everything the handle holds */
    int64_t kernel_launches;    /* launched directly or captured, since creation */
    int64_t graph_launches;
    int32_t launches_per_step;
    int32_t pad;
} qmpm_smoke_info_t;

/* Create a batch of n_scenes scenes (1 .. 4096) sharing config and scheme, all at rest
 * (u = v = d = 0).  scheme NULL: FP32 stores.  h_seeds: n_scenes dither seeds (host; NULL
 * = scene index).  stream: a cudaStream_t (NULL: the handle creates its own, since a CUDA
 * graph cannot capture the legacy stream).
 * Errors: QMPM_ERR_INVALID_ARG, QMPM_ERR_SCHEME, QMPM_ERR_OOM, QMPM_ERR_CUDA. */
int qmpm_smoke_create(const qmpm_smoke_config_t *cfg, const qmpm_smoke_scheme_t *scheme, int32_t n_scenes,
                      const uint64_t *h_seeds, void *stream, qmpm_smoke_handle *out);

/* Set the state of one scene (scene >= 0) or of every scene (-1) from host FP32 arrays in
 * the layout above (any may be NULL = zero).  Quantized velocities are rounded to the
 * nearest code (no dither); boundary faces are set to zero.  Synchronises the stream.
 * Errors: QMPM_ERR_INVALID_ARG, QMPM_ERR_CUDA. */
int qmpm_smoke_set_state(qmpm_smoke_handle h, int32_t scene, const float *h_u, const float *h_v,
                         const float *h_d);

/* Every scene's state at once: host FP32 arrays of n_scenes consecutive scenes in the
 * layout above (u [n_scenes][n][n+1], v [n_scenes][n+1][n], d [n_scenes][n][n]; any may be
 * NULL = zero), set as qmpm_smoke_set_state sets one (get: decoded, NULL = not copied).
 * One copy each way and one kernel over the batch; pinned host arrays copy fastest.  The
 * first call allocates device staging for the whole batch (4 (2 n (n+1) + 2 n^2) bytes per
 * scene), held until qmpm_smoke_destroy.  Synchronise the stream.
 * Errors: QMPM_ERR_INVALID_ARG, QMPM_ERR_OOM, QMPM_ERR_CUDA. */
int qmpm_smoke_set_states(qmpm_smoke_handle h, const float *h_u, const float *h_v, const float *h_d);
int qmpm_smoke_get_states(qmpm_smoke_handle h, float *h_u, float *h_v, float *h_d);

/* Noise injection for sensitivity estimates (FP32 handles only): every velocity store
 * except the reflection u^ and every pressure store gets sign_s * sigma_h * r added, r = +-1
 * from Philox4x32-7 with key = h_noise_seeds[s] and the store's dither counter (the top bit
 * of lane i % 8); wall faces (an exact zero) get none.  sigma = {0, 0} turns it off.
 * Scenes 2k and 2k+1 given one noise seed and signs +1, -1 form antithetic pairs:
 * E[((z+ - z-) / 2)^2] = sigma_h^2 sum over stores of type h of (dz/dstore)^2 (Eq. 8's g_h).
 * Errors: QMPM_ERR_INVALID_ARG (quantized handle, NULL arrays), QMPM_ERR_CUDA. */
int qmpm_smoke_set_noise(qmpm_smoke_handle h, const float sigma[2], const uint64_t *h_noise_seeds,
                         const float *h_signs);

/* Enqueue `steps` steps of every scene on the handle's stream.  d_trace NULL: replay a
 * CUDA graph of one step.  d_trace non-NULL (quantized handles, parity tests): plain
 * launches, and the code of every store of scene 0 is written to d_trace (device, uint32)
 * in store order: per step u~ v~, jacobi x q, u' v', u^ v^, u~2 v~2, jacobi x q, u'' v''
 * (velocity stores u then v, each in the layout above); trace_len must hold
 * steps * (10 n (n+1) + 2 jacobi n^2) codes.
 * Errors: QMPM_ERR_INVALID_ARG, QMPM_ERR_CUDA. */
int qmpm_smoke_step(qmpm_smoke_handle h, int32_t steps, uint32_t *d_trace, int64_t trace_len);

/* z_s = sum over cells of d^2 (FP64 accumulation) for every scene into h_z[n_scenes];
 * synchronises.  Errors: QMPM_ERR_INVALID_ARG, QMPM_ERR_CUDA. */
int qmpm_smoke_measure(qmpm_smoke_handle h, double *h_z);

/* Copy one scene's decoded state to host FP32 arrays (any may be NULL); q is the last
 * projection's final pressure iterate.  Synchronises.  Errors: QMPM_ERR_INVALID_ARG,
 * QMPM_ERR_CUDA. */
int qmpm_smoke_readback(qmpm_smoke_handle h, int32_t scene, float *h_u, float *h_v, float *h_d, float *h_q);

/* Per scene and type, the smallest and largest value offered to a store so far (handles
 * created with QMPM_SMOKE_RANGES; zeros otherwise) and the number of saturated stores:
 * h_lo, h_hi [n_scenes][2], h_sat [n_scenes][2] (any may be NULL).  Synchronises.
 * Errors: QMPM_ERR_INVALID_ARG, QMPM_ERR_CUDA. */
int qmpm_smoke_ranges(qmpm_smoke_handle h, float *h_lo, float *h_hi, int64_t *h_sat);

int qmpm_smoke_info(qmpm_smoke_handle h, qmpm_smoke_info_t *out);

/* Handles created with QMPM_SMOKE_PROFILE: device time of the steps run since the last
 * call (h_step_ms), of their Jacobi sweep launches (h_jacobi_ms) and the number of those
 * launches; resets.  Synchronises.  Errors: QMPM_ERR_INVALID_ARG (no profile flag),
 * QMPM_ERR_CUDA. */
int qmpm_smoke_profile(qmpm_smoke_handle h, double *h_step_ms, double *h_jacobi_ms, int64_t *h_jacobi_launches);

/* One stage of a quantized step, run by its own kernel launch on scene 0 from inputs the
 * caller gives (the stage-by-stage parity check of the advection-reflection step, Sec. 8.1:
 * every stage's stores compared with the FP64 oracle's from identical stored inputs).
 * Inputs in the layouts of qmpm_smoke_set_state (u: n rows of n + 1 faces, v: n + 1 rows
 * of n faces, cells n x n; FP32, host); stored inputs are encoded with nearest rounding, so values on
 * the type's lattice are stored exactly.  step >= 1 is the step index of the stores (store
 * counter 1024 step + k, as in qmpm_smoke_step).
 *   QMPM_SMOKE_ADVECT1   a = (u, v after the forces; v stays FP32): out = store 1 of
 *                        A(a; a, dt/2)
 *   QMPM_SMOKE_JACOBI    sweep `arg` (1..jacobi) of the first projection from the stored
 *                        iterate q (unused for arg 1) and the FP32 divergence div: store 1 + arg
 *   QMPM_SMOKE_GRADSUB2  a = u~ (stored), q: out = store J + 2 of a - grad q, then store
 *                        J + 3 of the reflection 2 out - a
 *   QMPM_SMOKE_ADVECT4   a = u^ (stored), b = u' (stored): out = store J + 4 of A(a; b, dt/2)
 *   QMPM_SMOKE_GRADSUB5  a = u~2 (stored), q: out = store 2 J + 5 of a - grad q
 * h_codes (host) receives the stage's codes in store order: the u codes (k = row (n+1) +
 * column) then the v codes (k = row n + column), or the n^2 pressure codes; GRADSUB2 writes
 * both of its stores, 4 n (n+1) codes.  The call overwrites the scene's stored fields and
 * leaves its step count as it was.  Synchronous.  Errors: QMPM_ERR_INVALID_ARG (FP32
 * handle, unknown stage, missing input), QMPM_ERR_OOM, QMPM_ERR_CUDA. */
#define QMPM_SMOKE_ADVECT1 0
#define QMPM_SMOKE_JACOBI 1
#define QMPM_SMOKE_GRADSUB2 2
#define QMPM_SMOKE_ADVECT4 3
#define QMPM_SMOKE_GRADSUB5 4
int qmpm_smoke_stage(qmpm_smoke_handle h, int32_t stage, int32_t arg, uint32_t step, const float *h_a_u,
                     const float *h_a_v, const float *h_b_u, const float *h_b_v, const float *h_q,
                     const float *h_div, uint32_t *h_codes);

/* Free everything the handle holds (synchronises its stream).  NULL is a no-op. */
int qmpm_smoke_destroy(qmpm_smoke_handle h);

#ifdef __cplusplus
}
#endif
#endif
