/*
 * sp2.h -- C ABI of the GB300 (sm_103a) SP2 density-matrix library.
 *
 * Method: mixed-precision Deep-NN SP2 recursive Fermi-operator expansion of
 * Finkelstein et al., "Mixed Precision Fermi-Operator Expansion on Tensor
 * Cores From a Machine Learning Perspective" (arXiv:2101.06385):
 *   Alg. 1  (layer loop, branch choice, parameter-free convergence),
 *   Alg. 2 / Eqs. 12-14 (split FP16 squaring with FP32 accumulation; the
 *            pair is stored as hp = 2^s hi and lo' = 2^s lo),
 *   Eq. 15  (refinement layer f_final),
 *   Eq. 16  (generalised second-order layer, used by the network entry points),
 *   Sec. "Accelerated Deep-NN SP2" (bound-driven layers from HOMO/LUMO estimates),
 *   Sec. "Optimized SP2 Finite Temperature Fermi-Operator Expansion"
 *            (generalised layers with a readout).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are dense, real, symmetric, row-major float32 with leading
 *   dimension N (no padding).  Symmetry is assumed, not checked.
 * - Unless stated otherwise every matrix pointer is a DEVICE pointer on the
 *   device selected in sp2_init, owned by the caller; the library neither
 *   frees nor retains it after the call returns.  Host pointers are marked.
 * - All device work is enqueued on the library stream (sp2_config.stream, or
 *   the one set with sp2_set_stream).  A call with a non-NULL stats pointer
 *   synchronises that stream before returning; with stats == NULL the call
 *   only enqueues.
 * - Return value: SP2_OK (0), SP2_NOT_CONVERGED (> 0, outputs still written)
 *   or a negative error.  On SP2_ERR_INVALID_ARG nothing is enqueued and the
 *   outputs are untouched.  Errors found on the device (non-finite or
 *   degenerate spectral bounds, device wait time-outs) are reported through
 *   the status of a synchronising call; outputs are then unspecified.
 * - No C++ exception crosses this interface.  sp2_last_error() returns a
 *   thread-local description of the last failure.
 * - Not re-entrant: one thread at a time per process (the workspace is
 *   shared).
 */
#ifndef SP2_H
#define SP2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SP2_MAX_LAYERS 128 /* max_iter <= SP2_MAX_LAYERS - 3 */

typedef enum {
  SP2_OK = 0,
  SP2_NOT_CONVERGED = 1,
  SP2_ERR_INVALID_ARG = -1,
  SP2_ERR_NOT_INITIALIZED = -2,
  SP2_ERR_DEGENERATE_SPECTRUM = -3, /* e_max - e_min <= 0 with 0 < N_occ < N */
  SP2_ERR_NONFINITE = -4,           /* non-finite spectral bounds (NaN/Inf in H) */
  SP2_ERR_CUDA = -5,
  SP2_ERR_OOM = -6,
  SP2_ERR_DEVICE_TIMEOUT = -7,      /* a bounded device wait ran out */
  SP2_ERR_UNSUPPORTED = -8,
  SP2_ERR_BAD_ESTIMATE = -9         /* accelerated solve: the HOMO/LUMO estimates were not safe
                                       (Tr D differs from N_occ by more than 1/2) */
} sp2_status;

typedef enum {
  SP2_PREC_SPLIT_FP16 = 0, /* Alg. 2: X ~ hi + lo, X^2 ~ hi hi + hi lo + lo hi, FP32 accumulate (tcgen05) */
  SP2_PREC_FP16 = 1,       /* single FP16 product hi hi, FP32 accumulate (tcgen05) */
  SP2_PREC_FP32 = 2        /* FP32 FFMA on the CUDA cores: the paper's "GPU-only" comparator */
} sp2_precision;

typedef enum {
  SP2_STOP_NONE = 0,
  SP2_STOP_TOL = 1,      /* IdErr_n <= tol */
  SP2_STOP_IDERR = 2,    /* IdErr_n <= 0 (Alg. 1) */
  SP2_STOP_RULE45 = 3,   /* IdErr_n > 4.5 IdErr_{n-2}^2 after a sign change (Alg. 1, appendix) */
  SP2_STOP_MAXITER = 4,  /* n == max_iter: returns SP2_NOT_CONVERGED */
  SP2_STOP_BOUNDS = 5    /* accelerated solve: eigenvalue bounds within tol of 0 and 1 */
} sp2_stop_reason;

typedef struct {
  int device;             /* CUDA device ordinal */
  void* stream;           /* cudaStream_t; NULL selects the legacy default stream */
  int precision;          /* sp2_precision */
  int lo_scale_exp;       /* s: the low FP16 part stores 2^s (X - hi); default 11, range 0..14 */
  int shift_identity;     /* 1 (default): iterate S = alpha I + Y with FP64 alpha, square only Y */
  double eps_bias;        /* epsilon of the branch rule (Alg. 1); default 0 */
} sp2_config;

typedef struct {
  int iterations;                 /* n: squaring layers of the loop (refinement not counted;
                                     the accelerated solves count all their layers) */
  int converged_by;               /* sp2_stop_reason */
  int status_device;              /* sp2_status recorded on the device */
  int n_occ;
  double e_min, e_max;            /* Gershgorin bounds used for the input layer */
  double idemp_err;               /* IdErr_n of the last loop layer (Tr[S - S^2]) */
  double trace;                   /* tr D after refinement */
  double alpha;                   /* identity shift of the last iterate (0 without shift) */
  double time_ms;                 /* device time of the whole call (CUDA events) */
  double flops_alg;               /* algorithmic FLOPs: layers x 3N^3 (split), N^3 (fp16/fp32) */
  double prologue_ms;             /* device time of the bounds, input layer and first row-norm
                                     kernels */
  int launches;                   /* squaring launches enqueued (max_iter + 2; max_iter for the
                                     accelerated solves); launches past the last layer find the
                                     solve finished and return at once */
  int8_t sigma[SP2_MAX_LAYERS];   /* sigma[k] = sigma_{k+1} in {+1,-1}; 0 past the end */
  double iderr[SP2_MAX_LAYERS];   /* iderr[k] = IdErr_{k+1} */
  float layer_ms[SP2_MAX_LAYERS]; /* device time of layer k (k < launches): the loop layers, then
                                     the two refinement layers of Eq. 15 (one squaring launch per
                                     layer on the tensor-core path; launch plus row-norm pass on
                                     the FFMA path) */
  float square_ms[SP2_MAX_LAYERS];/* device time of squaring launch k alone */
  double energy;                  /* Tr[D H] (Alg. 1, last line), accumulated by the launch that
                                     writes D (tensor-core path; 0 on the FFMA path) */
} sp2_stats;

/* Library set-up.  cfg == NULL selects the defaults {device 0, NULL stream,
 * SPLIT_FP16, s = 11, shift on, eps 0}.  Calling again re-applies a config
 * (the workspace is kept).  Errors: INVALID_ARG (bad field), CUDA.
 * Schedule switches read here from the environment (none changes a result
 * except where stated): SP2_SQUARE_KERNEL=single (single CTAs instead of CTA
 * pairs), SP2_BATCHED_KERNEL=single|pairs (fix the batched schedule instead
 * of timing both on the first call of a batch signature), SP2_GRAPHS=0
 * (enqueue the batched launches directly instead of replaying a CUDA graph),
 * SP2_WAVE_SYNC=<K stages> (epoch of the pairs' soft synchronisation in the
 * single solve, 16; 0 off), SP2_TILE_GROUP=<n> (side of the square tile
 * groups, 8), SP2_WIDE=0|1 (two super tiles of a row per pair pass in the
 * single solve; default: where it takes no more waves, i.e. N = 16384),
 * SP2_SNAKE=1 (alternate waves walk K backwards: changes the accumulation
 * order), SP2_FAULT=<spec> (test-only fault injection, sp2_set_fault). */
sp2_status sp2_init(const sp2_config* cfg);

/* Frees the workspace.  Safe to call when not initialised. */
sp2_status sp2_finalize(void);

/* Selects the stream for subsequent calls (cudaStream_t, NULL = default). */
sp2_status sp2_set_stream(void* stream);

/* Selects the precision for subsequent calls (sp2_precision). */
sp2_status sp2_set_precision(int precision);

/* Thread-local text of the last error ("" if none).  Never NULL. */
const char* sp2_last_error(void);

/*
 * Fault injection for tests of the error paths (failure detection; the
 * paper has no counterpart).  spec is a comma-separated list; NULL, "" or
 * "none" clears every fault.  Items:
 *   alloc_fail  the library's next workspace request fails as if cudaMalloc
 *               had run out of memory: the call returns SP2_ERR_OOM before it
 *               enqueues any work (D_out untouched)
 *   nan_input   the next sp2_density_matrix / _accelerated reads row 0 of H
 *               as holding a NaN: SP2_ERR_NONFINITE, no layer runs
 *   timeout     in the next single-matrix solve's first squaring launch the
 *               MMA issuer waits on a barrier that nothing arrives on; the
 *               wait runs out, every CTA stops issuing, drains its copies and
 *               MMAs, frees its tensor memory and returns; the call returns
 *               SP2_ERR_DEVICE_TIMEOUT (D_out holds no meaningful values)
 *   wait_ms=<n> bound of every device wait of the tensor-core squaring
 *               kernels, 1..60000 ms (default 4000); stays in force
 * alloc_fail, nan_input and timeout each fire once.  The environment variable
 * SP2_FAULT, when set, is applied by sp2_init.  Needs neither a GPU nor
 * sp2_init.  Returns SP2_ERR_INVALID_ARG (and changes nothing) for an unknown
 * or malformed item.  Nothing here faults, traps or hangs a GPU.
 */
sp2_status sp2_set_fault(const char* spec);

/*
 * Zero-temperature density matrix D = theta(mu I - H) with Tr D = N_occ by
 * Deep-NN SP2 (Alg. 1) with the refinement layer f_final (Eq. 15).
 *
 *   H        [N, N] device, input Hamiltonian (orthonormal basis, Sec. 2).
 *   N        matrix size, 1 <= N <= 65536.
 *   N_occ    number of occupied states, 0 <= N_occ <= N.
 *   tol      stop once IdErr_n <= tol (0: only the paper's parameter-free rule).
 *   max_iter 1 <= max_iter <= SP2_MAX_LAYERS - 3.
 *   D_out    [N, N] device output; also used as the iterate's storage during
 *            the call.  Must not alias H.
 *   stats    host pointer or NULL (see conventions).
 * Spectral bounds: Gershgorin discs (Alg. 1 "spectral bound estimates").
 */
sp2_status sp2_density_matrix(const float* H, int N, int N_occ, double tol, int max_iter,
                              float* D_out, sp2_stats* stats);

/*
 * Accelerated Deep-NN SP2 (Sec. "Accelerated Deep-NN SP2"): each layer is a
 * generalised layer X' = a X^2 + b X + c I chosen from bounds on the scaled
 * spectrum instead of the trace rule.  With the unoccupied eigenvalues of
 * the scaled iterate in [0, l] and the occupied ones in [h, 1]: if
 * 1 - h <= l the layer is x -> ((x - l/2)/(1 - l/2))^2, else
 * x -> 1 - ((1 - x - t)/(1 - t))^2 with t = (1 - h)/2; both fix 0 and 1,
 * keep the two sets apart, and give the next bounds in closed form.  The
 * solve stops once max(l, 1 - h) <= tol; D_out is the last layer (no Eq. 15
 * refinement).
 *
 *   homo, lumo  estimates of the highest occupied and lowest unoccupied
 *               eigenvalues of H (e.g. from a previous step of a dynamics
 *               run).  Safe when homo >= true HOMO and lumo <= true LUMO
 *               (a narrower gap); homo < lumo required.  The initial bounds
 *               are l = (e_max - lumo)/(e_max - e_min), h = (e_max - homo)/
 *               (e_max - e_min) with the Gershgorin e_min, e_max, clamped to
 *               [0, 1]; the device reports SP2_ERR_INVALID_ARG when l >= h.
 *   tol         bound tolerance, 0 selects 1e-9.
 *   max_iter    layer limit as for sp2_density_matrix (SP2_NOT_CONVERGED
 *               when it is reached first).
 *   other arguments and ownership as for sp2_density_matrix.
 * Errors: as sp2_density_matrix, plus INVALID_ARG for non-finite or
 * gapless estimates and BAD_ESTIMATE when Tr D misses N_occ by more than
 * 1/2 (D_out then holds the wrong projection).
 */
sp2_status sp2_density_matrix_accelerated(const float* H, int N, int N_occ, double homo, double lumo, double tol,
                                          int max_iter, float* D_out, sp2_stats* stats);

/*
 * Many independent SP2 problems of uneven size in grouped launches (the
 * batching remark of Sec. 4).  H, N, N_occ, D_out are HOST arrays of length
 * batch; H[i] and D_out[i] are device pointers to [N[i], N[i]] matrices.
 * Each instance follows its own branch sequence and convergence.  Sizes
 * 1 <= N[i] <= 4096, batch <= 4096.  stats: host array [batch] or NULL.
 * Returns SP2_NOT_CONVERGED if any instance hit max_iter.
 */
sp2_status sp2_density_matrix_batched(const float* const* H, const int* N, const int* N_occ, int batch,
                                      double tol, int max_iter, float* const* D_out, sp2_stats* stats);

/*
 * Batched form of sp2_density_matrix_accelerated: instance b uses the HOMO /
 * LUMO estimates homo[b] < lumo[b] (HOST arrays of batch doubles); other
 * arguments, statuses and conventions as sp2_density_matrix_batched, plus
 * BAD_ESTIMATE for an instance whose Tr D misses N_occ by more than 1/2
 * (checked when stats is non-NULL).
 */
sp2_status sp2_density_matrix_batched_accelerated(const float* const* H, const int* N, const int* N_occ,
                                                  const double* homo, const double* lumo, int batch, double tol,
                                                  int max_iter, float* const* D_out, sp2_stats* stats);

/*
 * Differentiable network (Eq. 16 in matrix form), batched over B instances:
 *   X_0 = (e_max I - H)/(e_max - e_min)    (Gershgorin bounds per instance, Alg. 1 input layer)
 *   X_{n+1} = a_n X_n^2 + b_n X_n + c_n I,  n = 0 .. L-1,
 * with X^2 computed by the split-FP16 tensor-core squaring.
 *   H      [B, N, N] device.        coef  [L, 3] HOST float (a_n, b_n, c_n).
 *   X_out  [B, N, N] device, X_L.
 *   ckpt   [(L / ckpt_every) + 1, B, N, N] device or NULL: X_{k ckpt_every}
 *          for k = 0 .. L / ckpt_every, in that order.
 *   bounds [B, 2] device double or NULL: receives (e_min, e_max) per instance.
 * 1 <= L <= 256, 1 <= ckpt_every <= L, B * N * N < 2^31, N <= 8192.
 */
sp2_status sp2_network_forward(const float* H, int B, int N, int L, const float* coef, int ckpt_every,
                               float* X_out, float* ckpt, double* bounds);

/*
 * Adjoint of sp2_network_forward (reverse mode, layer checkpointing).
 *   ckpt   the checkpoints written by sp2_network_forward with the same
 *          H, B, N, L, coef, ckpt_every.
 *   G_out  [B, N, N] device, dLoss/dX_L (symmetric).
 *   dcoef  [L, 3] HOST double output: (dL/da_n, dL/db_n, dL/dc_n) summed over the batch.
 *   G_in   [B, N, N] device output dLoss/dX_0, or NULL.
 * Per layer, with G = G_{n+1}:  G_n = a_n (X_n G + G X_n) + b_n G,
 *   dL/da_n = <G, X_n^2>, dL/db_n = <G, X_n>, dL/dc_n = tr G.
 * Workspace: the ckpt_every iterates of one checkpoint segment are
 * recomputed and kept in FP32 together with their FP16 operand planes
 * (about ckpt_every * B * N^2 * 8 bytes on the split path, * 6 on plain FP16),
 * plus the FP32 adjoint and its planes.  Errors: INVALID_ARG, UNSUPPORTED
 * (FP32 precision), CUDA / OOM, DEVICE_TIMEOUT.
 */
sp2_status sp2_network_backward(const float* H, int B, int N, int L, const float* coef, int ckpt_every,
                                const float* ckpt, const float* G_out, double* dcoef, float* G_in);

/*
 * Finite-temperature Fermi-operator expansion (Sec. "Optimized SP2 Finite
 * Temperature Fermi-Operator Expansion"): the generalised SP2 layers with a
 * readout,
 *   X_0 = (H - e_lo I)/(e_hi - e_lo),
 *   X_n = theta[n-1][0] X_{n-1}^2 + theta[n-1][1] X_{n-1} + theta[n-1][2] I,
 *   D   = I - sum_{i=0}^{L} c_i X_i,
 * the matrix form of F~(eps) = 1 - sum_i c_i eps_i on the scaled energy
 * eps = (E - e_lo)/(e_hi - e_lo) (fit theta and c so that F~ approximates the
 * Fermi function, e.g. 1/(exp(beta (eps - 1/2)) + 1)).
 *
 *   H       [B, N, N] device, B instances (1 <= N <= 8192, B N^2 < 2^31).
 *   L       layers, 1 <= L <= SP2_MAX_LAYERS.
 *   theta   [L, 3] HOST, c [L + 1] HOST, FP64.
 *   e_lo, e_hi  the energy window mapped to [0, 1]; both 0 selects each
 *           instance's Gershgorin bounds.
 *   D_out   [B, N, N] device output (also the iterate's storage).
 *   bounds  [B, 2] device (e_lo, e_hi used per instance) or NULL.
 * Tensor-core precisions only (split or fp16; UNSUPPORTED otherwise).
 * Stream-ordered; synchronises only to read Gershgorin bounds back.
 * Errors: INVALID_ARG, NONFINITE / DEGENERATE_SPECTRUM (Gershgorin mode),
 * UNSUPPORTED, CUDA, OOM.
 */
sp2_status sp2_fermi_expansion(const float* H, int B, int N, int L, const double* theta, const double* c,
                               double e_lo, double e_hi, float* D_out, double* bounds);

/* ---- single steps of the path, exposed for testing and composition ---- */

/* Gershgorin spectral bounds (Alg. 1 inputs): bounds_out (HOST double[2]) =
 * { min_i H_ii - R_i, max_i H_ii + R_i }, R_i = sum_{j != i} |H_ij|,
 * accumulated in FP64.  Synchronises.  1 <= N <= 65536. */
sp2_status sp2_gershgorin(const float* H, int N, double* bounds_out);

/* Split of an FP32 matrix into FP16 parts (Eq. 12), round-to-nearest-even:
 * hi = FP16[X], lo = FP16[2^s (X - hi)].  X [N, N] device float; hi, lo
 * [N, N] device uint16 (IEEE binary16 bit patterns).  0 <= s <= 14. */
sp2_status sp2_split(const float* X, int N, int lo_scale_exp, uint16_t* hi, uint16_t* lo);

/* One generalised layer (Eq. 16) through the selected precision's squaring
 * kernel: X_out = a X^2 + b X + c I for a batch of B matrices [B, N, N].
 * traces_out: HOST double[2 B] or NULL -> (tr X_out, ||X_out||_F^2) per
 * matrix (synchronises when non-NULL).  X_out must not alias X. */
sp2_status sp2_layer(const float* X, int B, int N, float a, float b, float c, float* X_out,
                     double* traces_out);

/* Observable alpha = Tr[D A] (Alg. 1, last line; A = H gives the band
 * energy).  D, A [N, N] device; out: HOST double.  Synchronises. */
sp2_status sp2_observable(const float* D, const float* A, int N, double* out);

/* ---- allocation-free variant (no counterpart in the paper) ---- */

#define SP2_NOALLOC_MAX_N 1024
#define SP2_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u + 65536u)

/*
 * sp2_density_matrix for callers that cannot allocate device memory when they
 * need D: engines that pre-size every buffer at start-up and must not grow the
 * process footprint mid-run, real-time loops in which an allocation (which can
 * synchronise the device) would stall a step, and hosts that hand the library
 * only memory they manage themselves.
 * It calls no cudaMalloc, cudaFree or other allocating routine: its scratch is
 * one file-scope device array of SP2_NOALLOC_SCRATCH_BYTES (about 8 MiB),
 * which every GPU that loads the library holds until the process exits.
 *
 *   H, N, N_occ, tol, max_iter, D_out, stats: as sp2_density_matrix, with
 *            N <= SP2_NOALLOC_MAX_N; larger N returns SP2_ERR_INVALID_ARG
 *            ("N exceeds SP2_NOALLOC_MAX_N" in sp2_last_error()).
 *   stream   cudaStream_t to enqueue on (NULL = legacy default stream).
 * Split-FP16 precision with the sp2_init defaults (shift on, epsilon 0,
 * low-part scale 2^11); needs no sp2_init.  stats->time_ms, layer_ms,
 * square_ms, prologue_ms and energy are not measured (0).  With stats ==
 * NULL the call returns once the work is enqueued and its status reflects
 * the argument checks only: a device-side failure (non-finite H, degenerate
 * spectrum, a timed-out wait) is reported only through a call with stats,
 * whose read-back synchronises the stream (refused with SP2_ERR_INVALID_ARG
 * on a stream that is being captured).  The first call on a device, with that device current,
 * looks up the array's device address (cudaGetSymbolAddress); make that first
 * call before any stream capture.  All calls share the array and leave their
 * contents in it (the zero-start counters are cleared at the start of each
 * call); calls whose GPU work overlaps (other streams or host threads) race.
 */
sp2_status sp2_density_matrix_noalloc(const float* H, int N, int N_occ, double tol, int max_iter,
                                      float* D_out, sp2_stats* stats, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SP2_H */
