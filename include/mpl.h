/*
 * mpl.h -- C ABI of the GB300 batch-mode Matching Pursuit LASSO library.
 *
 * The library solves, for every column b_i of B independently,
 *
 *     x_i = argmin_x  lambda_i * ||x||_1 + 0.5 * ||b_i - A x||^2
 *
 * which is the LASSO of eq. 2 per signal and the batch problem of eq. 3 with
 * the 1/2 factor of eq. 2 (eq. 3 as printed omits it; it is the same problem
 * with lambda halved).  It runs the MPL outer loop of Algorithm 1 for all
 * signals at once (the batch mode of Sec. 3): the correlation A^T R of the
 * worst-case analysis for every signal as one GEMM, the rho largest
 * violators per signal, growth of each active set, the master problem
 * (eq. "primal_MPL") by accelerated proximal gradient on the Gram block
 * A_S^T A_S, and the residual R = B - A_S X_S, until every signal meets the
 * stopping condition ||xi^T A||_inf <= lambda of Sec. 2.3 to a relative
 * tolerance, certified in FP64.
 *
 * Conventions
 *   - All matrices are column-major with the leading dimension equal to the
 *     number of rows: A is n x m (each atom a_j is n contiguous floats),
 *     B is n x p (each signal contiguous), X is m x p (each code contiguous).
 *   - Pointers may be device memory or host memory (the library tells them
 *     apart; host buffers are staged through device memory inside the call).
 *   - Every entry point returns an mpl_status_t; no entry point aborts the
 *     process.  MPL_ERR_ARG is returned synchronously for bad arguments.
 *   - A handle is not thread-safe: use one handle per host thread/stream.
 */
#ifndef MPL_H
#define MPL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpl_ctx* mpl_handle_t;

typedef enum {
    MPL_OK = 0,
    MPL_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, lambda <= 0 ...) */
    MPL_ERR_CUDA = 2,           /* a CUDA runtime call failed; the handle may be unusable */
    MPL_ERR_OOM = 3,            /* device allocation failed */
    MPL_ERR_TIMEOUT = 4,        /* a bounded device-side wait gave up */
    MPL_ERR_NOT_CONVERGED = 5,  /* solve finished, but some signal is not certified (see stats) */
    MPL_ERR_UNSUPPORTED = 6     /* option or size outside what this build supports */
} mpl_status_t;

/* Keys for mpl_set_option / mpl_get_option. */
typedef enum {
    MPL_OPT_RHO = 0,        /* atoms added per outer iteration (varrho, Sec. 2.1). default 1 */
    MPL_OPT_PRECISION = 1,  /* 0: correlation A^T R in FP32 (plain);
                               1: BF16 operands on tensor cores, FP32 accumulation, with
                                  near-ties re-scored in FP32 (mixed).  default 0 */
    MPL_OPT_MAX_OUTER = 2,  /* cap on outer iterations.  default 200 */
    MPL_OPT_SMAX = 3,       /* capacity of each active set.  default min(n, m, 256) */
    MPL_OPT_EPS_IN = 4,     /* relative-decrease tolerance of eq. (inner) for the FP32
                               master problem.  default 1e-4 */
    MPL_OPT_INNER_MAX = 5,  /* s_max, PG iterations per master problem.  default 400 */
    MPL_OPT_WARM_START = 6, /* 0: x^0 = 0 (Alg. 1);
                               2: proposal network seeds the active sets.  default 0 */
    MPL_OPT_SYNC_EVERY = 7, /* outer iterations launched per host/device handshake. default 2 */
    MPL_OPT_PROFILE = 8,    /* 1: record per-phase device times (mpl_get_phase_times) with
                               timing events, inside the captured graphs too. default 0 */
    MPL_OPT_GRAPH = 9,      /* 1: each outer iteration is replayed from a captured CUDA graph
                               (captured on first use per batch size and iteration). default 1 */
    MPL_OPT_WARM_CANDIDATES = 10, /* W: atoms per signal scored by the proposal network (the W
                                     largest |a_j^T b| of the first correlation; the rho largest
                                     violators join S anyway, the network picks among the
                                     rest, so the warm start only acts when W > rho * omega).
                                     1..64, default 64 */
    MPL_OPT_WARM_MAX = 11,        /* most atoms a proposal adds to a signal's set. default 3 rho */
    MPL_OPT_WARM_THRESHOLD = 12,  /* accept a candidate when its logit exceeds this. default -1 */
    MPL_OPT_QROUTE = 13,          /* identity route of the worst-case analysis (Sec. 3, eq.
                                     "batchQ"): g_i = beta_i - Q_S x_S with Q = A^T A (m x m
                                     FP32, built on first use, 4 m^2 bytes held by the handle)
                                     and beta_i = A^T b_i (kept from the first iteration, which
                                     then runs the FP32 GEMM).  Taken at outer iterations whose
                                     bound on |S| (t rho plus warm-start additions) is at most
                                     this value; 0 = never (default).  The selection widens its
                                     re-score band to the route's error bound, so the atoms
                                     chosen, and the solution, are the same on either route. */
    MPL_OPT_OMEGA = 14,           /* subspace exploratory matching (Algorithm 2, SMPL): each
                                     outer iteration takes the omega*rho largest violators, solves
                                     the master problem with all of them, and keeps the rho with
                                     the largest |u| (ties to the larger correlation); the others
                                     leave S and may return later.  1 = Algorithm 1 (default),
                                     at most 16. */
    MPL_OPT_STOP_RINF = 15,       /* early stopping, eq. (stop1) of Sec. 2.5: a signal stops at
                                     the worst-case analysis once the certified bound on
                                     |a_j^T xi| over the atoms outside S is <= this value.
                                     Negative = off (default) */
    MPL_OPT_STOP_R2 = 16,         /* eq. (stop1): stop once ||xi|| <= this value.  Negative =
                                     off (default) */
    MPL_OPT_STOP_EPS = 17,        /* eq. (stop_con): stop after a master problem whose decrease
                                     of the objective, f(x^{t-1}) - f(x^t), is <= this value
                                     times |rho f(x^0)|, f(x^0) = ||b||^2 / 2.  Negative = off
                                     (default).  A stopped signal gets the exact restricted
                                     solution on its S and status MPL_SIG_EARLY_STOP; lambda = 0
                                     (least squares, the OMP reduction of Sec. 2.5 with rho = 1)
                                     needs one of these rules or MPL_OPT_MAX_OUTER to end. */
    MPL_OPT_QGRAM = 18,           /* 1: the Gram growth reads the new entries of A_S^T A_S from
                                     Q = A^T A (Sec. 3: Q is precomputed off-line for the batch,
                                     and the master problem's Gram block Q_SS is a sub-block of
                                     it) instead of multiplying the atoms' columns; the entries
                                     of A_S^T b for the new atoms are one FP32 FMA chain each.
                                     Q (4 m^2 bytes) is built on first use, as for
                                     MPL_OPT_QROUTE, by one FMA chain per entry in the order
                                     the computed Gram block uses, so the solution is
                                     bit-identical either way.  0 = compute (default). */
    MPL_OPT_GEMM_TILE = 19,       /* signals per output tile of the BF16 tensor-core GEMM
                                     (MPL_OPT_PRECISION = 1): 64, 128 (default) or 256; every
                                     score is accumulated in the same order whatever the
                                     tile, so the solution does not depend on it. */
    MPL_OPT_REENTRY = 20          /* when a signal whose exact finish certified its active set
                                     rejoins the loop for the worst-case analysis of eq. (8):
                                     0 (default): at the first outer iteration that starts after
                                     its finish is done (an iteration waits only for the finish
                                     of four iterations back).  The outer iteration a signal's
                                     next finish falls in, and so that finish's launch shape,
                                     then depends on timing, and the certified solution may
                                     differ between runs in its last bits.  1: exactly two
                                     outer iterations later (each iteration waits for the
                                     finish of two iterations back): the same bits on every
                                     run, whatever the timing.  Both certify every signal. */
} mpl_option_t;

/* Per-signal outcome (host struct filled by mpl_get_stats). */
typedef enum {
    MPL_SIG_CERTIFIED = 0,      /* KKT certified to tol in FP64 */
    MPL_SIG_MAX_OUTER = 1,      /* stopped by MPL_OPT_MAX_OUTER */
    MPL_SIG_CAPACITY = 2,       /* active set reached MPL_OPT_SMAX */
    MPL_SIG_UNCERTIFIED = 3,    /* exact finish failed repeatedly */
    MPL_SIG_NONFINITE = 4,      /* NaN/Inf met in the data or iterates */
    MPL_SIG_EARLY_STOP = 5      /* stopped by an early-stopping rule (MPL_OPT_STOP_*); x is the
                                   exact minimiser of eq. 2 restricted to the final S, the
                                   atoms outside S are not certified */
} mpl_signal_status_t;

typedef struct {
    int32_t outer_iters;  /* evaluations of the correlation (FMVPs, Sec. 4.2) */
    int32_t inner_iters;  /* PG iterations over all master problems (PMVP pairs) */
    int32_t active_size;  /* |S| at exit */
    int32_t nnz;          /* nonzeros of x */
    int32_t status;       /* mpl_signal_status_t */
    int32_t finishes;     /* active-set steps of the exact finish (all attempts) */
    double objective;     /* lambda*||x||_1 + 0.5*||b - A x||^2, FP64 */
    double kkt;           /* certified upper bound on the max KKT violation / lambda */
    double gap;           /* relative duality gap with the scaled dual point of eq. 5 */
} mpl_signal_stats_t;

/*
 * mpl_create -- load a dictionary.
 *   A   n x m column-major FP32 (atom j at A + j*n), device or host memory.
 *       Copied: the caller may free A after the call returns.
 *   n   signal length, 1 <= n <= 65536.  m  number of atoms, 1 <= m <= 2^26.
 *   out receives the handle.
 * The library keeps an FP32 and (on first mixed solve) a BF16 copy of A and
 * the column norms.  The one-time layout work corresponds to the paper's
 * offline precomputation for BMPL (Sec. 3, remark on Q).
 * Errors: MPL_ERR_ARG, MPL_ERR_OOM, MPL_ERR_CUDA.
 */
mpl_status_t mpl_create(const float* A, int n, int m, mpl_handle_t* out);

/*
 * bmpl_solve -- solve p LASSO problems sharing the dictionary (eq. 3).
 *   B       n x p column-major FP32 signals (device or host).
 *   p       number of signals, p >= 0 (p = 0 returns MPL_OK at once).
 *   lambda  p FP32 values, each > 0 and finite (device or host).
 *   X       m x p column-major FP32 output, overwritten with the solutions
 *           (device or host).
 *   tol     relative KKT tolerance (e.g. 1e-6): a signal is certified when,
 *           in FP64 or by a rigorous FP32 error bound, |a_j^T r - lambda*s_j|
 *           <= tol*lambda on the support and |a_j^T r| <= (1+tol)*lambda off it.
 *   stream  a cudaStream_t (NULL = legacy default stream).
 * Device buffers are read and written in stream order; the call returns after
 * the solve has completed on the stream (the outer loop is host-driven), so X
 * and the statistics are ready on return.
 * Returns MPL_OK when every signal is certified, MPL_ERR_NOT_CONVERGED when
 * some signal is not (its best iterate is still written to X), or an error.
 */
mpl_status_t bmpl_solve(mpl_handle_t h, const float* B, int p, const float* lambda, float* X,
                        double tol, void* stream);

/*
 * mpl_correlate -- the worst-case analysis product of Algorithm 1,
 * g_i = A^T r_i for p given vectors (a full matrix-vector product, FMVP,
 * Sec. 2.4), computed by the handle's current correlation path
 * (MPL_OPT_PRECISION).
 *   R  n x p column-major FP32 (device or host).
 *   C  m x p column-major FP32 output, C[i*m + j] = a_j^T r_i (device or host).
 * Synchronous with respect to the stream.  Errors: MPL_ERR_ARG, MPL_ERR_CUDA,
 * MPL_ERR_TIMEOUT (a bounded tensor-core pipeline wait expired).
 */
mpl_status_t mpl_correlate(mpl_handle_t h, const float* R, int p, float* C, void* stream);

/*
 * mpl_correlate_noalloc -- the same FP32 correlation as mpl_correlate with
 * MPL_OPT_PRECISION = 0, for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a library-usage entry point.
 *
 * Who it is for: programs whose device memory is owned up front by their own
 * pool allocator (a framework's caching allocator, a serving runtime with a
 * fixed budget).  A cudaMalloc issued behind their back can fail once the pool
 * has reserved the memory, and it synchronises the device mid-pipeline.  This
 * call needs no handle and allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library routine.
 *
 *   A  n x m column-major FP32 dictionary, device memory.
 *   R  n x p column-major FP32 vectors, device memory.
 *   C  m x p column-major FP32 output, C[i*m + j] = a_j^T r_i, device memory.
 *   stream  cudaStream_t (NULL = legacy default stream); the call is
 *           asynchronous and stream-ordered.
 * A, R and C must be device (or managed) memory that the current device owns,
 * each 16-byte aligned (a view that starts inside an allocation at an offset
 * that is not a multiple of 4 floats is refused); anything else returns
 * MPL_ERR_ARG before any launch.
 * Limits: 1 <= n <= 65536, 1 <= m <= 2^26, 0 <= p <= MPL_NOALLOC_MAX_SIGNALS;
 * a larger p returns MPL_ERR_UNSUPPORTED, a bad n or m MPL_ERR_ARG.
 * Scratch: a fixed MPL_NOALLOC_SCRATCH_BYTES device array inside the library,
 * held by every GPU that loads it until the process exits.  The first call on
 * a device looks up that array's address (cudaGetSymbolAddress) with the
 * device current and caches it with the current CUDA context; a later call
 * that finds another context current (after cudaDeviceReset, say) looks it up
 * again.  Make the first call on a device, and the first after such a reset,
 * before any stream capture.  Every call rewrites the scratch it reads, and
 * all calls share it, so calls whose GPU work overlaps (different streams, no
 * ordering between them) race.
 */
#define MPL_NOALLOC_SCRATCH_BYTES (1u << 20)
#define MPL_NOALLOC_MAX_SIGNALS ((int)((MPL_NOALLOC_SCRATCH_BYTES - 256u) / 4u))
mpl_status_t mpl_correlate_noalloc(const float* A, int n, int m, const float* R, int p, float* C, void* stream);

/*
 * Learned warm start (MPL_OPT_WARM_START = 2).  A per-atom network scores the
 * W candidates of each signal from the first correlation c = A^T b:
 *   features (|c_j|/lambda, log(||b||/lambda), ||A^T a_j|| / sqrt(1 + m/n)),
 *   standardised, then 64 ReLU -> 64 ReLU -> 1 logit; BF16 weights, FP32 arithmetic.
 * The first outer iteration then adds MPL's own rho largest violators (the
 * worst-case analysis of Alg. 1) plus every candidate whose logit exceeds MPL_OPT_WARM_THRESHOLD; the
 * loop continues unchanged to the KKT tolerance, so solutions do not depend on
 * the proposal (atoms are never deleted, Sec. 2.2).
 * Parameter vector (MPL_PROPOSAL_NPARAM floats): mean[3], std[3], W1[64][3],
 * b1[64], W2[64][64], b2[64], w3[64], b3.
 */
#define MPL_PROPOSAL_NPARAM 4487
mpl_status_t mpl_proposal_set_weights(mpl_handle_t h, const float* w, int count);
mpl_status_t mpl_proposal_get_weights(mpl_handle_t h, float* w, int count);
/* Train the network on p signals with reference solutions Xref (m x p column-major,
 * labels = nonzeros), on the device with hand-written kernels: minibatch Adam on the
 * binary cross-entropy, features standardised with the training set's mean and
 * deviation.  B, lambda, Xref: device or host.  loss_out: host, epochs values (mean
 * loss per epoch) or NULL.  Initialisation and shuffling are seeded. */
mpl_status_t mpl_proposal_train(mpl_handle_t h, const float* B, int p, const float* lambda, const float* Xref,
                                int epochs, double lr, int batch, uint64_t seed, float* loss_out);
/* Mean loss and its gradient (host, MPL_PROPOSAL_NPARAM floats; zero for the
 * normalisation constants) over the examples of (B, lambda, Xref) with the current
 * FP32 weights; for gradient checks. */
mpl_status_t mpl_proposal_loss_grad(mpl_handle_t h, const float* B, int p, const float* lambda, const float* Xref,
                                    double* loss, float* grad);

/* Release the handle and all its device memory.  NULL-safe. */
void mpl_destroy(mpl_handle_t h);

/* Set / read an option (mpl_option_t).  Errors: MPL_ERR_ARG for unknown keys or
 * out-of-range values, MPL_ERR_UNSUPPORTED for modes this build lacks. */
mpl_status_t mpl_set_option(mpl_handle_t h, int key, double value);
mpl_status_t mpl_get_option(mpl_handle_t h, int key, double* value);

/* Copy per-signal statistics of the last bmpl_solve to host memory
 * (p entries; p must equal the last solve's p). */
mpl_status_t mpl_get_stats(mpl_handle_t h, int p, mpl_signal_stats_t* host_out);

/* Copy the last solve's FP64 solutions (the certified iterates, before the
 * FP32 rounding of X) as a dense m x p column-major array (device or host). */
mpl_status_t mpl_get_solution_f64(mpl_handle_t h, int p, double* X64);

/* Phase data of the last solve.  Entries 0..6 are device milliseconds,
 * filled when MPL_OPT_PROFILE is 1: total, correlation, selection, Gram
 * growth, exact finish, master problem, residual (with captured graphs only
 * the correlation and the exact finish are timed).  Entry 7 is the number of
 * signal columns the correlation processed, summed over outer iterations;
 * entry 8 the algorithmic FLOPs of the exact finish (factorisations, solves,
 * residual and correlation sums); entry 9 how many of the entry-7 columns the
 * identity route (MPL_OPT_QROUTE) scored instead of the GEMM; 7..9 always
 * filled.  Entry 10: device milliseconds of the identity-route scoring (entry
 * 1 then holds the GEMM alone).  Entries 11..14, always filled, count the
 * algorithmic work of the memory-bound kernels over the whole solve: 11 the
 * Gram-block entries read by the master problems' products, 12 how many of
 * them came from global memory (blocks too large for shared memory), 13 the
 * bytes the residual update reads and writes, 14 the bytes the Gram growth
 * reads and writes, 15 the bytes the exact finish streams (Gram rows of its
 * solves, the support's atom columns of its exact residuals and correlations).
 * Returns the number of values written (<= cap, <= 16). */
int mpl_get_phase_times(mpl_handle_t h, double* ms_out, int cap);

/* Autotuner of the batched solve (no counterpart in the paper, which has no
 * batching layer to tune).  Times complete solves of the caller's batch
 * (B, p, lambda, tol as for bmpl_solve; device or host memory) under each
 * candidate setting -- the identity route for the first k = 0, 1, 2, 4 outer
 * iterations after the first (MPL_OPT_QROUTE = k rho plus the warm-start
 * additions; k > 0 only when Q = A^T A fits in a quarter of the free device
 * memory) and MPL_OPT_SYNC_EVERY in {1, 2, 4}; then, where Q fits, the best
 * of those with MPL_OPT_QGRAM = 1 at each MPL_OPT_SYNC_EVERY; then, for the
 * BF16 path, the other GEMM tile widths (MPL_OPT_GEMM_TILE 64, 128, 256) with
 * the best of those -- and keeps the fastest on the handle.  Every candidate computes the same solution, so only time is
 * compared.  Each candidate runs once untimed (graph capture, Q build) and
 * three times timed with events on `stream`; the median counts.  The solutions
 * go to a scratch buffer the call allocates and frees; the handle's last-solve
 * statistics are those of the final timed run.  `out` (may be NULL) receives
 * the choice.  Synchronises `stream`.  Errors: those of bmpl_solve (the first
 * candidate's), MPL_ERR_OOM for the scratch buffer. */
typedef struct {
    int qroute;          /* chosen MPL_OPT_QROUTE */
    int sync_every;      /* chosen MPL_OPT_SYNC_EVERY */
    double ms;           /* median solve time of the choice */
    double ms_default;   /* median solve time with qroute 0, sync_every 2, qgram 0 */
    int candidates;      /* settings timed */
    int qgram;           /* chosen MPL_OPT_QGRAM */
    int gemm_tile;       /* chosen MPL_OPT_GEMM_TILE (timed last, BF16 path only) */
} mpl_tune_result_t;
mpl_status_t mpl_autotune(mpl_handle_t h, const float* B, int p, const float* lambda, double tol,
                          void* stream, mpl_tune_result_t* out);

/* Number of CUDA kernel launches issued by the last bmpl_solve. */
int64_t mpl_get_launch_count(mpl_handle_t h);

/* Human-readable text for a status code (static storage). */
const char* mpl_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* MPL_H */
