// Internal declarations shared by the CUDA translation units of the BMPL library.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mpl.h"

namespace mpl {

// Programmatic dependent launch for the kernels of the outer-iteration chain: each is
// launched with the programmatic-serialisation attribute, so that its launch is set up
// while its predecessor on the stream drains (the predecessor's CTAs trigger it as they
// exit), and it waits (griddepcontrol.wait: the predecessor grid complete, its writes
// visible) before touching anything.  Launched without the attribute (or after a
// non-kernel node) the wait returns at once.
// (MPL_NO_PDL builds the chain without the attribute, for measuring what it saves.)
__device__ __forceinline__ void pdl_enter() {
#if !defined(MPL_NO_PDL)
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

template <typename... P, typename... A>
inline cudaError_t launch_chain(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args) {
    cudaLaunchConfig_t c{};
    c.gridDim = grid;
    c.blockDim = block;
    c.dynamicSmemBytes = smem;
    c.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
#if defined(MPL_NO_PDL)
    at[0].val.programmaticStreamSerializationAllowed = 0;
#else
    at[0].val.programmaticStreamSerializationAllowed = 1;
#endif
    c.attrs = at;
    c.numAttrs = 1;
    return cudaLaunchKernelEx(&c, k, static_cast<P>(args)...);
}

// Per-signal phase decided by the selection kernel each outer iteration.
enum SigState : int {
    ST_GROW = 1,      // new atoms were appended: Gram growth, master problem, residual
    ST_FINALIZE = 2,  // no violator left: FP64 exact finish and certificate
    ST_DONE = 3,      // certified (or given up); leaves the active list
    ST_REFINE = 4,    // the exact finish failed: one more master-problem pass next iteration
};

// The exact finishes of outer iteration t use list slot t % FIN_SLOTS: a finish runs beside
// the following iterations, and an iteration waits only for the finish whose slot it reuses.
constexpr int FIN_SLOTS = 4;

// Device-side counters and work-list lengths (one instance per solve).
struct Counters {
    int act_n[2];    // active-list lengths (double-buffered by outer-iteration parity)
    int grow_n;      // signals that took new atoms
    int fin_n;       // signals sent to the exact finish (this iteration)
    int fin_par[FIN_SLOTS];  // ... by list slot (a finish runs while the next iterations do)
    int reent_n[FIN_SLOTS];  // finished signals waiting to re-enter the active list, by the
                             // slot of the finish they left
    int fslot;       // the slot this iteration's selection fills (t % FIN_SLOTS, kept by the merge)
    int mslots;      // bit s: the finish of slot s is done, merge its signals this iteration
                     // (set by the host through k_set_merge, cleared by the merge)
    int apg_n;       // signals in the master-problem list (grow + failed finishes)
    int apg_head;    // work-queue head of the persistent master-problem kernel
    int apg_head2;   // head of its second queue (blocks streamed from global memory)
    int err;         // first device-side error code (0 = none)
    int sel_fallback;// candidate-buffer overflows in the selection
    unsigned long long cols;  // signal columns processed by the correlation (all iterations)
    unsigned long long fin_flops;  // algorithmic FLOPs of the exact finish (factor, solves, residual sums)
    unsigned long long qcols;  // signal columns scored by the identity route beta - Q_S x_S
    int sel_done;    // selection CTAs finished (the last one compacts the lists)
    int bounds_site; // diagnostic builds: the first failed bounds check
    // algorithmic work of the memory-bound kernels (roofline accounting, all iterations)
    unsigned long long apg_elems;     // Gram-block entries read by the master problems' products
    unsigned long long apg_gl_elems;  // of those, read from global memory (blocks outside shared memory)
    unsigned long long res_bytes;     // bytes the residual update reads (atoms, b) and writes (R)
    unsigned long long gram_bytes;    // bytes the Gram growth reads (Q or atoms, b) and writes (G, h)
    unsigned long long fin_bytes;     // bytes the exact finish streams (Gram rows, atom columns, b)
    __host__ __device__ int act_n_of(int c) const { return act_n[c]; }
};

// Everything a kernel may touch, passed by value.
struct Dev {
    int n, m, p, smax, rho, mw;  // mw = words of the per-signal membership bitmap
    int precision;               // 0 plain FP32, 1 mixed BF16
    int omega;                   // subspace search length of Algorithm 2 (1 = Algorithm 1)
    float stop_rinf, stop_r2, stop_eps;  // early-stopping thresholds of Sec. 2.5 (< 0: off)
    int inner_max;
    float eps_in;
    double tol;
    float colmax;                // max_j ||a_j|| (rounded up)
    float bound_c;               // |score_gemm - a_j^T r| <= bound_c * colmax * ||r||
    // BF16 GEMM, measured rounding: |score - a_j^T r| <= bf_ea ||r|| + bf_ta (||r - bf(r)|| +
    // bf_acc ||bf(r)||) + bound_c32 colmax ||r||, with bf_ea >= max_j ||a_j - bf(a_j)|| and
    // bf_ta >= max_j ||bf(a_j)|| (per dictionary), the residual terms per signal (r16e, r16t)
    float bf_ea, bf_ta, bf_acc;
    float* r16e;                 // p ||r - bf(r)|| upper bound (mixed)
    float* r16t;                 // p ||bf(r)|| upper bound (mixed)
    float bound_c32;             // same for the fixed-order FP32 re-score
    float bound_f32;             // FP32 correlation GEMM (either precision)
    float bound_q;               // identity route: |score - a_j^T r| <= bound_q*colmax*(||b|| + colmax*||x||_1)
    const float* Q;              // m x m Gram matrix A^T A (row k = A^T a_k), identity route only
    float* beta;                 // p x m beta = A^T b (FP32), identity route only
    float* bnorm;                // p ||b|| upper bound
    float* xl1;                  // p ||x_S||_1 upper bound of the FP32 iterate
    const float* A32;            // m x n atom-major
    const __nv_bfloat16* A16;    // m x n atom-major (mixed)
    const float* B;              // p x n signals (device)
    const float* lam;            // p
    float* R32;                  // p x n residual (FP32; high part after an exact finish)
    float* R32lo;                // p x n low part of the exact-finish residual
    double* R64;                 // p x n residual of the exact finish (FP64)
    __nv_bfloat16* R16;          // p x n residual (BF16, mixed)
    __nv_bfloat16* R16c;         // act_n x n compacted BF16 residual for the GEMM
    int* pos;                    // p row of each signal in R16c (its place in the next active list)
    float* Cs;                   // act_n x m correlation scores (row k <-> act[k])
    uint32_t* mask;              // p x mw membership bitmap of S_i
    int* S;                      // p x smax active-set atom indices (append order)
    float* xS;                   // p x smax FP32 master-problem iterate
    double* xS64;                // p x smax FP64 finished solution
    float* G;                    // p x smax x smax Gram blocks A_S^T A_S (ld = smax)
    float* h;                    // p x smax A_S^T b (an entry per atom, from the selection's re-score)
    float* ritz;                 // p x smax power-iteration vector (warm start of L)
    double* chol;                // p x smax x smax FP64 workspace (large supports)
    double* fin_pool;            // FIN_SLOTS x fin_slots more such workspaces: one per CTA of a
    int fin_slots;               // clustered finish, a part per finish list slot
    unsigned* sel_tmax;          // P x ceil(m / SEL_CHUNK) chunk maxima of the score rows (m above the row cache)
    int* sel_nf;                 // P flags: a non-finite score in the row
    int* state;                  // p SigState
    int* ssize;                  // p |S_i|
    int* snew;                   // p atoms appended this iteration
    int* finalized;              // p 1 when R holds the residual of the exact finish
    int* outer;                  // p outer iterations
    int* inner;                  // p PG iterations
    int* finishes;               // p exact-finish attempts
    int* fails;                  // p consecutive failed finishes
    int* sstatus;                // p mpl_signal_status_t
    int* explore;                // p atoms explored this iteration (Algorithm 2), 0 = keep all
    int* early;                  // p 1 once an early-stopping rule fired
    float* f0;                   // p f(x^0) = ||b||^2 / 2
    int* nnz;                    // p
    float* rnorm;                // p ||r|| upper bound
    float* res_part;             // p x RES_BLOCKS(n) x 3 partial sums of the residual's row blocks
    int* res_tick;               // p row blocks of the residual update done (reset by the last one)
    float* eps;                  // p current eq. (inner) tolerance
    double* obj;                 // p FP64 objective
    double* kkt_in;              // p KKT violation / lambda on S (from the finish)
    double* kkt_out;             // p certified bound off S / lambda (from selection)
    double* ginf;                // p certified bound on ||A^T r||_inf
    double* rr;                  // p ||r||^2
    double* rb;                  // p r^T b
    int* act[2];                 // active lists (signal ids), by outer-iteration parity
    int* ovf_list;               // signals whose candidate band overflowed (second pass), or null
    Counters* ovf_cnt;           // its length in act_n[parity]
    int* list_grow;              // signals with new atoms
    int* list_fin[FIN_SLOTS];    // signals sent to the exact finish, by list slot
    int* reent[FIN_SLOTS];       // finished signals to merge back into the active list, by slot
    int* list_apg;               // master-problem work list
    Counters* cnt;
    __device__ const int* act_of(int c) const { return act[c]; }
};

// ---------------------------------------------------------------- proposal network
// Per-atom warm-start proposal: features (|c_j|/lambda, log(||r||/lambda), ||A^T a_j|| /
// sqrt(1 + m/n)) -> standardised -> 64 ReLU -> 64 ReLU -> 1 logit.  Parameter vector
// layout (FP32 master copy; inference reads the BF16-rounded values):
constexpr int PROP_H = 64;
constexpr int P_MEAN = 0, P_STD = 3, P_W1 = 6, P_B1 = P_W1 + PROP_H * 3, P_W2 = P_B1 + PROP_H,
              P_B2 = P_W2 + PROP_H * PROP_H, P_W3 = P_B2 + PROP_H, P_B3 = P_W3 + PROP_H,
              PROP_NPARAM = P_B3 + 1;  // 4487
constexpr int PROP_FIRST_TRAINABLE = P_W1;

enum SelMode : int { SEL_NORMAL = 0, SEL_PROPOSE = 1, SEL_EXAMPLES = 2 };
struct PropArgs {
    int mode;          // SelMode
    int W;             // candidates per signal (top-W by the re-scored |c_j|)
    int cap;           // most atoms a proposal may add
    float thr;         // accept when logit > thr
    const float* w;    // parameters (PROP_NPARAM), BF16-rounded for inference
    const float* rn;   // ||A^T a_j|| (m)
    float* ex;         // examples out: p x W x 4 (features, label; label -1 = empty slot)
    const float* xref; // reference solutions (p x m), labels = nonzeros
};

// ---------------------------------------------------------------- launchers
// Each returns the CUDA error of its launch and adds its launches to *nl.
cudaError_t launch_corr_f32(const Dev& d, int cur, int act_n_ub, cudaStream_t s, int64_t* nl);
// Matrix-vector correlations for at most GEMV_P active signals (n >= GEMV_MIN_N): the FP32
// and BF16 launchers take this route themselves when gemv_route holds.
constexpr int GEMV_P = 8;
constexpr int GEMV_MIN_N = 256;
bool gemv_route(const Dev& d, int act_n_ub);
cudaError_t launch_corr_gemv(const Dev& d, int cur, int act_n_ub, bool bf16, cudaStream_t s, int64_t* nl);
// BF16 tensor-core correlation (tcgen05 + TMA).  prepare() encodes the TMA
// descriptors for A16 (m x n) and R16c (pmax x n, one per tile width) into tmap
// (TC_TMAP_BYTES).  bn: signals per output tile, 64, 128 or 256.
constexpr int TC_TMAP_BYTES = 4 * 128;
cudaError_t corr_bf16_prepare(int n, int m, int pmax, const __nv_bfloat16* A16,
                              const __nv_bfloat16* R16c, void* tmap);
cudaError_t launch_corr_bf16(const Dev& d, int cur, const void* tmap, int act_n_ub, int sms,
                             cudaStream_t s, int64_t* nl, int bn = 128);
cudaError_t launch_gather_r16(const Dev& d, int cur, int act_n_ub, cudaStream_t s, int64_t* nl);
// Correlation routes of one outer iteration (selects the selection kernel's error band).
enum CorrRoute : int { ROUTE_GEMM = 0, ROUTE_GEMM_F32 = 1, ROUTE_Q = 2 };
// fuse_compact: the selection's last CTA also builds the work lists (k_compact not needed).
// chunked: for at most GEMV_P signals on rows above the row cache, a first kernel writes
// the rows' SEL_CHUNK-atom maxima and the selection starts from them (sel_chunked).
constexpr int SEL_CHUNK = 32;
// rows of the residual update per CTA (256 threads x float4): a signal's residual is split
// into ceil(n / RES_ROWS) row blocks, one CTA each
constexpr int RES_ROWS = 1024;
inline int res_blocks(int n) { return (n + RES_ROWS - 1) / RES_ROWS; }
bool sel_chunked(const Dev& d, int act_n_ub);
cudaError_t launch_select(const Dev& d, int cur, int no_grow, int act_n_ub, cudaStream_t s, int64_t* nl,
                          const PropArgs* pa = nullptr, int route = ROUTE_GEMM, int fuse_compact = 0,
                          int chunked = 0);
// Identity route (eq. batchQ): scores beta_i - Q_S x_S into the compacted score rows.
cudaError_t launch_corr_q(const Dev& d, int cur, int act_n_ub, cudaStream_t s, int64_t* nl);
// beta_i = score row of signal i (after an FP32 correlation of the residual b_i).
cudaError_t launch_save_beta(const Dev& d, int cur, int act_n_ub, cudaStream_t s, int64_t* nl);
cudaError_t build_gram_q(const float* A32, int n, int m, float* Q, int* act, Counters* cnt, cudaStream_t s,
                         int64_t* nl);
cudaError_t launch_compact(const Dev& d, int cur, cudaStream_t s, int64_t* nl);
// The new rows and columns of each growing signal's Gram block (h of the new atoms was
// written by the selection that appended them).
// qmax: most atoms a signal can take this iteration (picks the tile width).
cudaError_t launch_gram(const Dev& d, int ub, int qmax, cudaStream_t s, int64_t* nl);
// Gram growth gathered from Q (MPL_OPT_QGRAM): same outputs, bit for bit, as launch_gram.
cudaError_t launch_gram_gather(const Dev& d, int ub, cudaStream_t s, int64_t* nl);
// The exact finish of the signals the selection of an iteration sent to list slot `slot`
// (list_fin[slot]); each finished signal that is not done joins reent[slot].  ub bounds the
// number of finishing signals, est estimates it; when est is small against the sms SMs a
// signal's finish runs on a cluster of up to FIN_CLUSTER_MAX CTAs.
constexpr int FIN_CLUSTER_MAX = 8;
constexpr int FIN_CLUSTER_MIN_N = 2048;
cudaError_t launch_finish(const Dev& d, int slot, int ub, int est, int scap, cudaStream_t s, int64_t* nl, int sms);
// Set the device counter mslots (the finished slots the next merge takes back).
cudaError_t launch_set_merge(const Dev& d, int mask, cudaStream_t s, int64_t* nl);
// Append reent[s] of every slot s in the device counter mslots to the active list of an
// iteration with parity cur (rows for the GEMM included); the finishes that filled those
// slots must be complete.  Advances the finish list slot to the one of this iteration.
cudaError_t launch_merge(const Dev& d, int cur, int ub, cudaStream_t s, int64_t* nl);
// Master-problem launches: every signal of the work list, or only those whose Gram block fits
// shared memory, or only those streamed from global memory.
enum ApgClass : int { APG_ALL = 0, APG_SMEM = 1, APG_GLOBAL = 2 };
cudaError_t launch_apg(const Dev& d, int ub, int sms, int vcap, cudaStream_t s, int64_t* nl, int cls = APG_ALL);
// True when blocks up to the bound vcap may outgrow shared memory: the caller then runs an
// APG_SMEM and an APG_GLOBAL launch (concurrently) instead of one APG_ALL launch.
bool apg_split(const Dev& d, int vcap);
cudaError_t launch_residual(const Dev& d, int ub, cudaStream_t s, int64_t* nl);
// Algorithm 2: keep the rho explored atoms with the largest |u| (compacts S, x_S, h, G).
cudaError_t launch_smpl_prune(const Dev& d, int ub, cudaStream_t s, int64_t* nl);
cudaError_t launch_init(const Dev& d, cudaStream_t s, int64_t* nl);
cudaError_t launch_prep_correlate(const Dev& d, const float* R, cudaStream_t s, int64_t* nl);
cudaError_t launch_scatter(const Dev& d, float* X, double* X64, cudaStream_t s, int64_t* nl);
cudaError_t launch_pack_stats(const Dev& d, mpl_signal_stats_t* out, cudaStream_t s, int64_t* nl);
// err2 (2m floats, may be null): ||a_j - bf(a_j)|| and ||bf(a_j)||, rounded up.
cudaError_t launch_colnorm(const float* A32, int n, int m, float* colnorm, __nv_bfloat16* A16,
                           cudaStream_t s, int64_t* nl, float* err2 = nullptr);
cudaError_t launch_max_reduce(const float* v, int len, float* out, cudaStream_t s, int64_t* nl);

// Proposal network support (proposal.cu).
cudaError_t launch_sketch_rownorm(const float* A32, int n, int m, int T, float* Z, cudaStream_t s, int64_t* nl);
cudaError_t launch_rownorm(const float* C, int m, int T, float* rn, cudaStream_t s, int64_t* nl);
cudaError_t launch_train_step(const float* w, const float* ex, const int* perm, int off, int count, float inv_batch,
                              float* grad, float* loss_acc, int* n_acc, cudaStream_t s, int64_t* nl);
cudaError_t launch_adam(float* w, float* grad, float* m1, float* m2, float lr, int step, cudaStream_t s, int64_t* nl);
cudaError_t launch_round_bf16(const float* w, float* wb, cudaStream_t s, int64_t* nl);

// One-time kernel attribute set-up (call before any stream capture).
cudaError_t prepare_select();
cudaError_t prepare_apg();
cudaError_t prepare_gram();
cudaError_t prepare_finish();
cudaError_t prepare_corr_bf16();

// Device-side error codes written to Counters::err.
enum DevErr : int { DERR_NONE = 0, DERR_TIMEOUT = 1, DERR_NONFINITE = 2, DERR_SHAPE = 3, DERR_BOUNDS = 4 };

// Bounds checks of the diagnostic build (-DMPL_BOUNDS): a failed check records DERR_BOUNDS
// and its site in the counters (first one wins) and the caller skips the access.  Compiled
// out otherwise.
#ifdef MPL_BOUNDS
__device__ __forceinline__ bool mpl_bad(Counters* c, bool bad, int site) {
    if (bad) {
        atomicCAS(&c->err, 0, (int)DERR_BOUNDS);
        atomicCAS(&c->bounds_site, 0, site);
    }
    return bad;
}
#define MPL_OOB(cond, site) mpl_bad(d.cnt, (cond), (site))
#else
#define MPL_OOB(cond, site) false
#endif

// Candidate capacity of the selection kernel (per signal, in shared memory).
constexpr int SEL_KCAP = 2048;
constexpr int SEL_THREADS = 512;
// Largest W of the learned warm start (candidates scored per signal).  Larger values
// (W = 400 at the 4096 x 65536 workload) faulted on the GPU with a cause not found by
// reading, so the option stops here, at the value the GPU tests exercise.
constexpr int WARM_W_MAX = 64;
constexpr int SEL_ROWCACHE_ATOMS = 8192;  // score rows up to this length are cached in shared memory
// Master problem: Gram block kept in shared memory up to this size.
constexpr int APG_SMEM_S = 200;
constexpr int APG_THREADS = 256;
// Exact finish: FP32 factor in shared memory up to this support size (global beyond).
constexpr size_t FIN_SMEM_TWO_CTAS = 110 * 1024;  // dynamic shared memory that keeps 2 finish CTAs per SM
constexpr size_t FIN_SMEM_MAX = 225 * 1024;       // the most one finish CTA takes
constexpr int FIN_THREADS = 256;
constexpr int FIN_THREADS_WIDE = 512;  // one finish CTA per SM (large active sets)
constexpr int FIN_MAX_PIVOTS = 16;
constexpr int FIN_CG_MAXIT = 60;  // CG iterations per solve before the finish falls back to a factor
constexpr int FIN_CG_MIN_S = 128; // active sets above this size (with a factor outside shared memory) use CG
constexpr int FIN_MAX_FAILS = 6;

}  // namespace mpl
