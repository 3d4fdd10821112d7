// Exact finish and certificate of a master problem (eq. "primal_MPL").
//
// When a signal has no violator left, its FP32 proximal-gradient iterate u is
// driven to the exact restricted minimiser by an active-set method on the
// Gram block (the optimality conditions of the dual eq. 5 restricted to S):
//
//   P = supp(x), s = sign(x_P); solve G_PP z = h_P - lambda*s_P (Cholesky of G_PP);
//   if sign(z) = s:  x <- z, else step from x towards z up to the first sign
//                    crossing and drop that atom (the objective decreases
//                    along the segment, which stays inside the orthant of s);
//   if a zero entry j of S has |h_j - G_jP x_P| > lambda: add the largest one
//                    with the sign of its correlation;
//   repeat until consistent.
//
// The Gram block is only FP32-accurate, so the consistent point is then
// verified and refined with exact residuals r = b - A_P x and correlations
// A^T r: these O(n|P|) sums run in double-FP32 arithmetic (error-free
// products and sums via FMA, ~2^-44 relative) on the FP32 pipe, since GB300's
// FP64 rate is a small fraction of its FP32 rate.  The factor is FP32 (the
// refinement with exact residuals restores full accuracy), updated in place when
// an atom leaves or joins P; an FP64 factor, and then an exactly recomputed Gram
// block, take over when the refinement stops contracting.  The certified KKT
// violation on S and the exact residual (FP32 hi/lo pair and FP64) are stored;
// the next worst-case analysis certifies the atoms outside S (eq. 8).
//
// One CTA per signal (256 threads, two CTAs per SM; 512 when the shared-memory
// layout allows only one).  Shared memory is sized by the host from its bound on
// |S|; the FP32 factor lives in shared memory when the bound fits there at two
// CTAs per SM (panel Cholesky), else in the signal's global workspace (tiled
// Cholesky staged through shared memory); the FP64 factor always uses the
// workspace.
#include "mpl_internal.cuh"

namespace mpl {

#ifdef MPL_FIN_TRACE
// Per-signal phase cycle counters of the exact finish (diagnostic builds only):
// [factor, solve, crossing, gram-zero-check, verify, exact-zero-check, steps, refinements,
//  of the factor: support + right-hand side, Gram gather, evaluation cycles, evaluations,
//  refinement-solve cycles, FP64 refactors, their cycles, exact Gram rebuilds, CG iterations
//  of the steps' solves, CG solves of the steps, CG iterations of the refinements, finishes]
__device__ long long g_fin_trace[8192][20];
#define FT_BEGIN long long ft0_ = clock64(), fx_ = 0;
#define FT_SPLIT(slot) do { if (threadIdx.x == 0 && rank == 0 && i < 8192) g_fin_trace[i][slot] += clock64() - ft0_; } while (0)
#define FT_ADD(slot) do { if (threadIdx.x == 0 && rank == 0 && i < 8192) g_fin_trace[i][slot] += clock64() - ft0_; ft0_ = clock64(); } while (0)
#define FT_CNT(slot) do { if (threadIdx.x == 0 && rank == 0 && i < 8192) g_fin_trace[i][slot] += 1; } while (0)
#define FT_VAL(slot, v) do { if (threadIdx.x == 0 && rank == 0 && i < 8192) g_fin_trace[i][slot] += (v); } while (0)
#define FX_BEGIN fx_ = clock64();
#define FX_END(slot) do { if (threadIdx.x == 0 && rank == 0 && i < 8192) g_fin_trace[i][slot] += clock64() - fx_; } while (0)
#else
#define FX_BEGIN
#define FX_END(slot) do {} while (0)
#define FT_BEGIN
#define FT_ADD(slot) do {} while (0)
#define FT_CNT(slot) do {} while (0)
#define FT_VAL(slot, v) do {} while (0)
#define FT_SPLIT(slot) do {} while (0)
#endif

namespace {

// ---------------------------------------------------------------- double-FP32
struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_add(df x, df y) {
    const df s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

// acc + a*z with a an FP32 value (exact) and z a double-FP32 value.
__device__ __forceinline__ df df_fma(df acc, float a, df z) {
    const float p = __fmul_rn(a, z.hi);
    const float pe = fmaf(a, z.hi, -p);  // exact remainder of a*z.hi
    const float q = fmaf(a, z.lo, pe);
    const df s = two_sum(acc.hi, p);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(acc.lo, q)));
}

__device__ __forceinline__ df to_df(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

__device__ __forceinline__ double to_d(df v) { return (double)v.hi + (double)v.lo; }

__device__ __forceinline__ df warp_df_sum(df v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        df w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = df_add(v, w);
    }
    return v;
}

// ---------------------------------------------------------------- block helpers
__device__ __forceinline__ double bsum(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    return t;
}



// Blocked right-looking Cholesky by the whole CTA, panels of W columns: one
// thread factors the W x W diagonal block, the threads take the panel's rows
// below it, then the trailing lower triangle gets the rank-W update with its
// elements spread evenly over the CTA.  Three CTA barriers per panel.  With the
// factor in global memory (stage != null) the panel is kept in shared memory
// and wide panels (fewer passes over the trailing triangle) pay off.
// Returns 0 or -1 (non-positive pivot); flag likewise.
template <typename T, int W>
__device__ __noinline__ int chol_panel(T* M, int ld, int np, T* rdiag, int* flag, T* stage = nullptr) {
    const int tid = threadIdx.x, nt = blockDim.x;
    // (r', c') of this thread's first TPOS elements of any trailing triangle (the
    // row-major enumeration does not depend on the triangle's size)
    constexpr int TPOS = 6;
    int rpos[TPOS], cpos[TPOS];
#pragma unroll
    for (int k = 0; k < TPOS; ++k) {
        const int e = tid + k * nt;
        int rr = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
        while ((rr + 1) * (rr + 2) / 2 <= e) ++rr;
        while (rr * (rr + 1) / 2 > e) --rr;
        rpos[k] = rr;
        cpos[k] = e - rr * (rr + 1) / 2;
    }
    for (int j = 0; j < np; j += W) {
        const int w = min(W, np - j);
        if (tid == 0) {
            int bad = 0;
            for (int k = 0; k < w && !bad; ++k) {
                T* Rk = M + (size_t)(j + k) * ld + j;
                T dkk = Rk[k];
                for (int q = 0; q < k; ++q) dkk -= Rk[q] * Rk[q];
                if (!(dkk > T(0))) { bad = 1; break; }
                const T dg = sqrt(dkk), inv = T(1) / dg;
                Rk[k] = dg;
                rdiag[j + k] = inv;
                for (int r = k + 1; r < w; ++r) {
                    T* Rr = M + (size_t)(j + r) * ld + j;
                    T v = Rr[k];
                    for (int q = 0; q < k; ++q) v -= Rr[q] * Rk[q];
                    Rr[k] = v * inv;
                }
            }
            *flag = bad;
        }
        __syncthreads();
        if (*flag) return -1;
        // panel rows below the diagonal block
        for (int r = j + w + tid; r < np; r += nt) {
            T* Rr = M + (size_t)r * ld + j;
            T l[W];
#pragma unroll
            for (int k = 0; k < W; ++k) {
                if (k < w) {
                    const T* Rk = M + (size_t)(j + k) * ld + j;
                    T v = Rr[k];
#pragma unroll
                    for (int q = 0; q < k; ++q) v -= l[q] * Rk[q];
                    l[k] = v * rdiag[j + k];
                    Rr[k] = l[k];
                    if (stage) stage[(size_t)r * W + k] = l[k];
                }
            }
        }
        __syncthreads();
        // trailing triangle: rows r >= c >= j + w, element e <-> (r', c') in row-major order;
        // the first elements of a thread reuse the positions worked out before the loop
        const int b0 = j + w, nr = np - b0;
        const int tot = nr * (nr + 1) / 2;
        if (stage) {
            // factor in global memory: the panel comes from shared memory and each
            // thread keeps four element loads in flight before its stores
            for (int e0 = tid; e0 < tot; e0 += 4 * nt) {
                int rr4[4], cc4[4];
                T a4[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = e0 + u * nt;
                    rr4[u] = -1;
                    if (e < tot) {
                        int rr = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
                        while ((rr + 1) * (rr + 2) / 2 <= e) ++rr;
                        while (rr * (rr + 1) / 2 > e) --rr;
                        rr4[u] = b0 + rr;
                        cc4[u] = b0 + (e - rr * (rr + 1) / 2);
                        a4[u] = M[(size_t)rr4[u] * ld + cc4[u]];
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (rr4[u] < 0) continue;
                    const T* Lr = stage + (size_t)rr4[u] * W;
                    const T* Lc = stage + (size_t)cc4[u] * W;
                    T acc = a4[u];
#pragma unroll
                    for (int k = 0; k < W; ++k)
                        if (k < w) acc -= Lr[k] * Lc[k];
                    M[(size_t)rr4[u] * ld + cc4[u]] = acc;
                }
            }
            __syncthreads();
            continue;
        }
        for (int e = tid, k8 = 0; e < tot; e += nt, ++k8) {
            int rr, cc;
            if (k8 < TPOS) {
                rr = rpos[k8];
                cc = cpos[k8];
            } else {
                rr = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
                while ((rr + 1) * (rr + 2) / 2 <= e) ++rr;
                while (rr * (rr + 1) / 2 > e) --rr;
                cc = e - rr * (rr + 1) / 2;
            }
            const int r = b0 + rr, c = b0 + cc;
            const T* Lr = M + (size_t)r * ld + j;
            const T* Lc = M + (size_t)c * ld + j;
            T acc = M[(size_t)r * ld + c];
#pragma unroll
            for (int k = 0; k < W; ++k)
                if (k < w) acc -= Lr[k] * Lc[k];
            M[(size_t)r * ld + c] = acc;
        }
        __syncthreads();
    }
    if (tid == 0) *flag = 0;
    return 0;
}

// (L L^T) v = v by one warp, dot-product form (lanes split each sum).
template <typename T>
__device__ void solve_warp(const T* M, int ld, int np, const T* rdiag, T* v) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < np; ++j) {  // forward: L y = v
        const T* Lj = M + (size_t)j * ld;
        T acc = T(0);
        for (int q = lane; q < j; q += 32) acc += Lj[q] * v[q];
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) v[j] = (v[j] - acc) * rdiag[j];
        __syncwarp();
    }
    for (int j = np - 1; j >= 0; --j) {  // backward: L^T x = y
        T acc = T(0);
        for (int q = j + 1 + lane; q < np; q += 32) acc += M[(size_t)q * ld + j] * v[q];
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) v[j] = (v[j] - acc) * rdiag[j];
        __syncwarp();
    }
}

// (L L^T) v = v by one warp for np <= 64, column sweeps with the right-hand
// side in registers (lane owns rows lane and lane + 32).
template <typename T>
__device__ void solve_warp_reg(const T* M, int ld, int np, const T* rdiag, T* v) {
    const int lane = threadIdx.x & 31;
    const int r0 = lane, r1 = lane + 32;
    T y0 = r0 < np ? v[r0] : T(0), y1 = r1 < np ? v[r1] : T(0);
    for (int j = 0; j < np; ++j) {  // forward
        const int owner = j & 31;
        const T mine = (j < 32) ? y0 : y1;
        const T yj = __shfl_sync(0xffffffffu, mine, owner) * rdiag[j];
        if (lane == owner) { if (j < 32) y0 = yj; else y1 = yj; }
        if (r0 > j && r0 < np) y0 -= M[(size_t)r0 * ld + j] * yj;
        if (r1 > j && r1 < np) y1 -= M[(size_t)r1 * ld + j] * yj;
    }
    for (int j = np - 1; j >= 0; --j) {  // backward with L^T: row j of L
        const int owner = j & 31;
        const T mine = (j < 32) ? y0 : y1;
        const T xj = __shfl_sync(0xffffffffu, mine, owner) * rdiag[j];
        if (lane == owner) { if (j < 32) y0 = xj; else y1 = xj; }
        if (r0 < j) y0 -= M[(size_t)j * ld + r0] * xj;
        if (r1 < j) y1 -= M[(size_t)j * ld + r1] * xj;
    }
    if (r0 < np) v[r0] = y0;
    if (r1 < np) v[r1] = y1;
    __syncwarp();
}

// (L L^T) v = v by the CTA in blocks of 32 unknowns: warp 0 solves each diagonal
// block with the right-hand side in registers, then all threads apply the block to
// the remaining unknowns (rows of L below it going forward, its columns going back).
template <typename T>
__device__ void fwd_cta(const T* M, int ld, int np, const T* rdiag, T* v, T* scr = nullptr) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    for (int b0 = 0; b0 < np; b0 += 32) {  // forward: L y = v
        const int bw = min(32, np - b0);
        // the diagonal block: from M, or (a factor in global memory) from a shared-memory
        // copy, so that warp 0's dependent chain waits on shared memory, not on L2
        const T* D = M + (size_t)b0 * ld + b0;
        int dld = ld;
        if (scr) {
            for (int e = tid; e < bw * bw; e += nt) {
                const int r = e / bw, c = e - r * bw;
                if (c < r) scr[r * 33 + c] = D[(size_t)r * ld + c];
            }
            __syncthreads();
            D = scr;
            dld = 33;
        }
        if (tid < 32) {
            T y = lane < bw ? v[b0 + lane] : T(0);
            for (int j = 0; j < bw; ++j) {
                const T yj = __shfl_sync(0xffffffffu, y, j) * rdiag[b0 + j];
                if (lane == j) y = yj;
                if (lane > j && lane < bw) y -= D[(size_t)lane * dld + j] * yj;
            }
            if (lane < bw) v[b0 + lane] = y;
        }
        __syncthreads();
        for (int r = b0 + bw + tid; r < np; r += nt) {
            const T* Lr = M + (size_t)r * ld + b0;
            T acc = T(0);
#pragma unroll 8
            for (int c = 0; c < bw; ++c) acc += Lr[c] * v[b0 + c];
            v[r] -= acc;
        }
        __syncthreads();
    }
}

// scr: null, or 32 x 33 elements of shared memory for the diagonal blocks (worth it
// when M is in global memory).
template <typename T>
__device__ void solve_cta(const T* M, int ld, int np, const T* rdiag, T* v, T* scr = nullptr) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    fwd_cta(M, ld, np, rdiag, v, scr);
    for (int b1 = np; b1 > 0; b1 -= 32) {  // backward: L^T x = y
        const int b0 = max(0, b1 - 32), bw = b1 - b0;
        const T* D = M + (size_t)b0 * ld + b0;
        int dld = ld;
        if (scr) {
            for (int e = tid; e < bw * bw; e += nt) {
                const int r = e / bw, c = e - r * bw;
                if (c < r) scr[r * 33 + c] = D[(size_t)r * ld + c];
            }
            __syncthreads();
            D = scr;
            dld = 33;
        }
        if (tid < 32) {
            T y = lane < bw ? v[b0 + lane] : T(0);
            for (int j = bw - 1; j >= 0; --j) {
                const T xj = __shfl_sync(0xffffffffu, y, j) * rdiag[b0 + j];
                if (lane == j) y = xj;
                if (lane < j) y -= D[(size_t)j * dld + lane] * xj;
            }
            if (lane < bw) v[b0 + lane] = y;
        }
        __syncthreads();
        for (int r = tid; r < b0; r += nt) {
            T acc = T(0);
#pragma unroll 8
            for (int c = 0; c < bw; ++c) acc += M[(size_t)(b0 + c) * ld + r] * v[b0 + c];
            v[r] -= acc;
        }
        __syncthreads();
    }
}

// Block version: warp 0 runs the sweeps (each sum is split over its lanes).
template <typename T>
__device__ void solve_block(const T* M, int ld, int np, const T* rdiag, T* v) {
    if (np > 64) {
        solve_cta(M, ld, np, rdiag, v);
        return;
    }
    if (threadIdx.x < 32) solve_warp_reg(M, ld, np, rdiag, v);
    __syncthreads();
}

// Factor of G_PP: FP32 in shared memory (the Gram block itself is only
// FP32-accurate; refinement with exact residuals recovers full accuracy), or
// FP64 in the global workspace when FP32 refinement stagnates.  Every thread
// of the CTA returns the same result.
constexpr int FAC_TILE_W = 16;  // panel width of the tiled factorisation (factor in global memory)

// Floats of shared-memory staging for a global-memory factor of up to scap rows: the
// panel (FAC_TILE_W x scap rounded up to the 64-row tiles), its diagonal block, slack.
__host__ __device__ inline int fac_stage_floats(int scap) {
    return FAC_TILE_W * ((scap + 63) / 64) * 64 + FAC_TILE_W * (FAC_TILE_W + 1) + 16;
}

// Blocked right-looking Cholesky of a factor in global memory, by the CTA, panels of
// W = FAC_TILE_W columns.  Per panel: the W x W diagonal block is factored by warp 0
// in shared memory; each thread takes panel rows below it (forward substitution
// against the block, W values in registers) and writes them to M and, k-major, to the
// shared staging area; then the trailing lower triangle gets the rank-W update in
// 64 x 64 tiles, each thread a 4 x 4 register block fed by float4 reads of the staged
// panel, with the tile's 16 global values loaded before the products.  Per element the
// trailing triangle is read and written once per W columns (np^3 / (3W) touches in
// all) instead of once per 4 or 8.  stage: fac_stage_floats(rows) floats, 16-byte
// aligned.  Returns 0 or -1 (non-positive pivot); flag likewise.
// (blockDim.x a multiple of 256: each 256 threads take one 64 x 64 tile at a time as
// 16 x 16 blocks of 4 x 4)
__device__ __noinline__ int chol_tiled(float* M, int ld, int np, float* rdiag, int* flag, float* stage) {
    constexpr int W = FAC_TILE_W, DS = W + 1;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    float* D = stage;                 // W x W diagonal block, stride DS
    // k-major panel PT[k * PS + (r - j1)], 16-byte aligned for the float4 reads
    float* PT = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(stage + W * DS) + 15) & ~(uintptr_t)15);
    const int ty = (tid & 255) >> 4, tx = tid & 15;  // 16 x 16 threads of 4 x 4 blocks per tile
    const int sub = tid >> 8, nsub = nt >> 8;        // tiles in flight at once
    for (int j0 = 0; j0 < np; j0 += W) {
        const int w = min(W, np - j0), j1 = j0 + w, nr = np - j1;
        const int PS = ((nr + 63) / 64) * 64;
        for (int e = tid; e < w * w; e += nt) {
            const int r = e / w, c = e - r * w;
            if (c <= r) D[r * DS + c] = M[(size_t)(j0 + r) * ld + j0 + c];
        }
        __syncthreads();
        if (warp == 0) {
            int bad = 0;
            for (int k = 0; k < w; ++k) {
                const float dkk = D[k * DS + k];
                if (!(dkk > 0.f)) { bad = 1; break; }  // the same value on every lane
                const float dg = sqrtf(dkk), inv = 1.f / dg;
                __syncwarp();
                if (lane == k) { D[k * DS + k] = dg; rdiag[j0 + k] = inv; }
                if (lane > k && lane < w) D[lane * DS + k] *= inv;
                __syncwarp();
                if (lane > k && lane < w) {
                    const float lk = D[lane * DS + k];
                    for (int c = k + 1; c <= lane; ++c) D[lane * DS + c] -= lk * D[c * DS + k];
                }
                __syncwarp();
            }
            if (lane == 0) *flag = bad;
        }
        __syncthreads();
        if (*flag) return -1;
        for (int e = tid; e < w * w; e += nt) {
            const int r = e / w, c = e - r * w;
            if (c <= r) M[(size_t)(j0 + r) * ld + j0 + c] = D[r * DS + c];
        }
        // panel rows below the block
        for (int r = j1 + tid; r < np; r += nt) {
            float* Rr = M + (size_t)r * ld + j0;
            float l[W];
#pragma unroll
            for (int k = 0; k < W; ++k) l[k] = k < w ? Rr[k] : 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                if (k < w) {
                    float v = l[k];
#pragma unroll
                    for (int q = 0; q < k; ++q) v -= l[q] * D[k * DS + q];
                    l[k] = v * rdiag[j0 + k];
                }
            }
#pragma unroll
            for (int k = 0; k < W; ++k) {
                if (k < w) {
                    Rr[k] = l[k];
                    PT[k * PS + (r - j1)] = l[k];
                }
            }
        }
        __syncthreads();
        // trailing triangle: 64 x 64 tiles (ti >= tj), element (r, c) with c <= r
        const int T = (nr + 63) / 64;
        for (int t = sub; t < T * (T + 1) / 2; t += nsub) {
            int ti = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
            while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
            while (ti * (ti + 1) / 2 > t) --ti;
            const int tj = t - ti * (ti + 1) / 2;
            const int rr0 = ti * 64 + ty * 4, cc0 = tj * 64 + tx * 4;  // offsets from j1
            float a[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int r = rr0 + u, c = cc0 + v;
                    a[u][v] = (r < nr && c <= r) ? M[(size_t)(j1 + r) * ld + j1 + c] : 0.f;
                }
            float acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
            for (int k = 0; k < w; ++k) {
                const float4 x = *reinterpret_cast<const float4*>(PT + k * PS + rr0);
                const float4 y = *reinterpret_cast<const float4*>(PT + k * PS + cc0);
                const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(xs[u], ys[v], acc[u][v]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int r = rr0 + u, c = cc0 + v;
                    if (r < nr && c <= r) M[(size_t)(j1 + r) * ld + j1 + c] = a[u][v] - acc[u][v];
                }
        }
        __syncthreads();
    }
    return 0;
}


struct Factor {
    float* Mf;       // FP32 factor, leading dimension ldf
    float* rdf;
    double* Md;      // FP64 factor (global workspace), leading dimension ldd
    double* rdd;     // reciprocal diagonal for the FP64 factor
    float* vf;       // FP32 right-hand side scratch
    float* stage;    // staging (fac_stage_floats) for an FP32 factor in global memory, else null
    int stage_n;     // floats at stage
    int ldf, ldd;
    int fp64;        // which factor is current
};

__device__ int factor(Factor& F, int np, int* flag) {
    if (!F.fp64) {
        if (F.stage) return chol_tiled(F.Mf, F.ldf, np, F.rdf, flag, F.stage);
        return chol_panel<float, 4>(F.Mf, F.ldf, np, F.rdf, flag);
    }
    return chol_panel<double, 4>(F.Md, F.ldd, np, F.rdd, flag);
}

// v <- G_PP^{-1} v with the current factor (FP32 factor: solved in FP32).
__device__ void fsolve(const Factor& F, int np, double* v) {
    if (!F.fp64) {
        for (int a = threadIdx.x; a < np; a += blockDim.x) F.vf[a] = (float)v[a];
        __syncthreads();
        if (np > 64) {
            // the staging area is free outside factorisations: the diagonal blocks go there
            solve_cta(F.Mf, F.ldf, np, F.rdf, F.vf, F.stage_n >= 32 * 33 ? F.stage : nullptr);
        } else {
            if (threadIdx.x < 32) solve_warp_reg(F.Mf, F.ldf, np, F.rdf, F.vf);
            __syncthreads();
        }
        for (int a = threadIdx.x; a < np; a += blockDim.x) v[a] = (double)F.vf[a];
        __syncthreads();
        return;
    }
    solve_block(F.Md, F.ldd, np, F.rdd, v);
}

struct FinShared {
    Factor F;
    double* x;   // current point on S (position-indexed)
    double* z;   // solve result on P
    double* w;   // scratch on P / S
    int* P;      // support positions
    int* sg;     // sign per position of S
    int* Pi;     // atom index of each support position
    int* adds;   // times each position entered the support in this finish
    float* rh;   // exact residual, high part
    float* rl;   // exact residual, low part
    double red[32];
    int ival[4];
    double dval[4];
    int fac_np;  // rows of the FP32 factor that match P in its order (-1: rebuild next step)
    float cs[2]; // rotation of the factor update
    float rot[2][2];  // rotations of the CTA-wide update, alternating slots
    int cg;      // 1: solves by conjugate gradients on the Gram block (no factor)
    uint64_t cbar[2];  // cluster barriers of a clustered finish (C arrivals per phase; phases alternate)
};

// Ordered support of the sign pattern (one warp writes sh.P, count in ival[1]).
__device__ int build_support(int s, FinShared& sh) {
    if (threadIdx.x < 32) {
        int base = 0;
        for (int a0 = 0; a0 < s; a0 += 32) {
            const int a = a0 + threadIdx.x;
            const bool on = a < s && sh.sg[a] != 0;
            const unsigned b = __ballot_sync(0xffffffffu, on);
            if (on) sh.P[base + __popc(b & ((1u << threadIdx.x) - 1u))] = a;
            base += __popc(b);
        }
        if (threadIdx.x == 0) sh.ival[1] = base;
    }
    __syncthreads();
    return sh.ival[1];
}

// Incremental changes of the FP32 factor of G_PP when the support loses or
// gains one atom, instead of refactoring: by warp 0 up to FAC_INC_MAX atoms, by the
// whole CTA above that.
constexpr int FAC_INC_MAX = 64;

// Drop factor row/column k: the trailing factor absorbs the dropped column by a
// rank-one update (L33' L33'^T = L33 L33^T + l l^T, rotations by warp 0), then
// rows and columns after k move up by one; P and the reciprocal diagonal follow.
__device__ __noinline__ void fac_remove(FinShared& sh, int k, int np) {
    float* M = sh.F.Mf;
    const int ld = sh.F.ldf;
    const int m = np - k - 1;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
        // lane owns entries lane and lane + 32 of the dropped column below the diagonal
        float x0 = lane < m ? M[(size_t)(k + 1 + lane) * ld + k] : 0.f;
        float x1 = lane + 32 < m ? M[(size_t)(k + 33 + lane) * ld + k] : 0.f;
        for (int j = 0; j < m; ++j) {
            const int J = k + 1 + j;
            const float xj = __shfl_sync(0xffffffffu, j < 32 ? x0 : x1, j & 31);
            const float ljj = M[(size_t)J * ld + J];
            const float r = sqrtf(ljj * ljj + xj * xj);
            const float c = r / ljj, sn = xj / ljj;
            __syncwarp();
            if (lane == 0) { M[(size_t)J * ld + J] = r; sh.F.rdf[J] = 1.f / r; }
            if (lane > j && lane < m) {
                float* L = M + (size_t)(k + 1 + lane) * ld + J;
                const float ln = (*L + sn * x0) / c;
                *L = ln;
                x0 = c * x0 - sn * ln;
            }
            if (lane + 32 > j && lane + 32 < m) {
                float* L = M + (size_t)(k + 33 + lane) * ld + J;
                const float ln = (*L + sn * x1) / c;
                *L = ln;
                x1 = c * x1 - sn * ln;
            }
            __syncwarp();
        }
    }
    __syncthreads();
    // move rows/columns after k by one (each thread stages up to 16 entries of one row)
    const int r = tid >> 2, cq = tid & 3;
    float v[16];
    const bool live = r < np - 1;
    const int rs = r < k ? r : r + 1;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int c = cq + 4 * u;
        v[u] = (live && c <= r) ? M[(size_t)rs * ld + (c < k ? c : c + 1)] : 0.f;
    }
    float rd = 0.f;
    int pr = 0;
    if (tid < np - 1) { rd = sh.F.rdf[tid < k ? tid : tid + 1]; pr = sh.P[tid < k ? tid : tid + 1]; }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int c = cq + 4 * u;
        if (live && c <= r) M[(size_t)r * ld + c] = v[u];
    }
    if (tid < np - 1) { sh.F.rdf[tid] = rd; sh.P[tid] = pr; }
    __syncthreads();
}

// Append the support atom at position a as the factor's last row: forward
// substitution L l = G_Pa by warp 0, l_nn = sqrt(G_aa - l^T l).  Returns 0, or
// -1 when the new pivot is not positive (the caller refactors).
__device__ __noinline__ int fac_append(FinShared& sh, const float* Gi, int smax, int a, int np) {
    float* M = sh.F.Mf;
    const int ld = sh.F.ldf;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
        const int r0 = lane, r1 = lane + 32;
        float y0 = r0 < np ? Gi[(size_t)sh.P[r0] * smax + a] : 0.f;
        float y1 = r1 < np ? Gi[(size_t)sh.P[r1] * smax + a] : 0.f;
        for (int j = 0; j < np; ++j) {
            const float yj = __shfl_sync(0xffffffffu, j < 32 ? y0 : y1, j & 31) * sh.F.rdf[j];
            if (lane == (j & 31)) { if (j < 32) y0 = yj; else y1 = yj; }
            if (r0 > j && r0 < np) y0 -= M[(size_t)r0 * ld + j] * yj;
            if (r1 > j && r1 < np) y1 -= M[(size_t)r1 * ld + j] * yj;
        }
        float ss = (r0 < np ? y0 * y0 : 0.f) + (r1 < np ? y1 * y1 : 0.f);
#pragma unroll
        for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        const float dnn = Gi[(size_t)a * smax + a] - ss;
        if (r0 < np) M[(size_t)np * ld + r0] = y0;
        if (r1 < np) M[(size_t)np * ld + r1] = y1;
        if (lane == 0) {
            const bool ok = dnn > 0.f;
            sh.ival[0] = ok ? 0 : 1;
            if (ok) {
                const float dg = sqrtf(dnn);
                M[(size_t)np * ld + np] = dg;
                sh.F.rdf[np] = 1.f / dg;
                sh.P[np] = a;
            }
        }
    }
    __syncthreads();
    return sh.ival[0] ? -1 : 0;
}

// Drop factor row/column k of a factor of any size (np <= 4 blockDim.x + 1), by the
// CTA.  The trailing factor absorbs the dropped column by the same rank-one update as
// fac_remove: thread t owns trailing rows k + 1 + t + q nt (q < 4) and keeps their
// entries of the dropped column in registers.  Rotation j (row J = k + 1 + j) is
// worked out by the owner of row J from its own entries, so one barrier per rotation
// suffices (two slots alternate); the entries of column J + 1, which rotation j does
// not touch, are loaded while it runs.  Then rows below k move up by one row and,
// right of column k, one column left, a few rows at a time (every source read before
// the barrier that precedes the writes of its chunk, and a destination is never a
// source of a later chunk); P and the reciprocal diagonal follow.
__device__ __noinline__ void fac_remove_cta(FinShared& sh, int k, int np) {
    constexpr int RQ = 4;
    float* M = sh.F.Mf;
    const int ld = sh.F.ldf;
    const int m = np - k - 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    float x[RQ], nx[RQ];
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
        const int i = tid + q * nt;
        x[q] = i < m ? M[(size_t)(k + 1 + i) * ld + k] : 0.f;
        nx[q] = i < m ? M[(size_t)(k + 1 + i) * ld + k + 1] : 0.f;  // column J of rotation 0
    }
    for (int j = 0; j < m; ++j) {
        const int J = k + 1 + j;
        float cur[RQ];
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
            cur[q] = nx[q];
            const int i = tid + q * nt;
            nx[q] = (i > j && i < m) ? M[(size_t)(k + 1 + i) * ld + J + 1] : 0.f;  // i > j: j + 1 < m
        }
        if (tid == j % nt) {
            const int qo = j / nt;
            float ljj = 0.f, xj = 0.f;
#pragma unroll
            for (int q = 0; q < RQ; ++q)
                if (q == qo) { ljj = cur[q]; xj = x[q]; }
            const float r = sqrtf(ljj * ljj + xj * xj);
            sh.rot[j & 1][0] = r / ljj;
            sh.rot[j & 1][1] = xj / ljj;
            M[(size_t)J * ld + J] = r;
            sh.F.rdf[J] = 1.f / r;
        }
        __syncthreads();
        const float c = sh.rot[j & 1][0], sn = sh.rot[j & 1][1];
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
            const int i = tid + q * nt;
            if (i > j && i < m) {
                const float ln = (cur[q] + sn * x[q]) / c;
                M[(size_t)(k + 1 + i) * ld + J] = ln;
                x[q] = c * x[q] - sn * ln;
            }
        }
    }
    __syncthreads();
    // rows k + 1 .. np - 1 up by one; their columns right of k left by one
    const int rows = max(1, (8 * nt) / np);
    for (int r0 = k + 1; r0 < np; r0 += rows) {
        const int r1 = min(np, r0 + rows);
        const int tot = (r1 - r0) * np;
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = tid + u * nt;
            v[u] = 0.f;
            if (e < tot) {
                const int r = r0 + e / np, c = e % np;  // destination column c of row r - 1
                if (c < r) v[u] = M[(size_t)r * ld + (c < k ? c : c + 1)];
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = tid + u * nt;
            if (e < tot) {
                const int r = r0 + e / np, c = e % np;
                if (c < r) M[(size_t)(r - 1) * ld + c] = v[u];
            }
        }
        __syncthreads();
    }
    float rd[RQ];
    int pr[RQ];
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
        const int i = k + tid + q * nt;
        if (i < np - 1) { rd[q] = sh.F.rdf[i + 1]; pr[q] = sh.P[i + 1]; }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
        const int i = k + tid + q * nt;
        if (i < np - 1) { sh.F.rdf[i] = rd[q]; sh.P[i] = pr[q]; }
    }
    __syncthreads();
}

// Append the support atom at position a as row np of a factor of any size, by the
// CTA: the forward sweep L y = G_Pa in the FP32 scratch vector, l_nn = sqrt(G_aa -
// y^T y).  Returns 0, or -1 when the new pivot is not positive (the caller refactors).
__device__ __noinline__ int fac_append_cta(FinShared& sh, const float* Gi, int smax, int a, int np) {
    float* M = sh.F.Mf;
    const int ld = sh.F.ldf;
    float* v = sh.F.vf;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    for (int r = tid; r < np; r += nt) v[r] = Gi[(size_t)sh.P[r] * smax + a];
    __syncthreads();
    fwd_cta(M, ld, np, sh.F.rdf, v, sh.F.stage_n >= 32 * 33 ? sh.F.stage : nullptr);
    double ss = 0.0;
    for (int r = tid; r < np; r += nt) ss += (double)v[r] * (double)v[r];
#pragma unroll
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) sh.red[warp] = ss;
    __syncthreads();
    double tot = 0.0;
    for (int q = 0; q < nw; ++q) tot += sh.red[q];
    const float dnn = (float)((double)Gi[(size_t)a * smax + a] - tot);
    const bool ok = dnn > 0.f;
    if (ok) {
        for (int r = tid; r < np; r += nt) M[(size_t)np * ld + r] = v[r];
        if (tid == 0) {
            const float dg = sqrtf(dnn);
            M[(size_t)np * ld + np] = dg;
            sh.F.rdf[np] = 1.f / dg;
            sh.P[np] = a;
        }
    }
    __syncthreads();
    return ok ? 0 : -1;
}

// After atoms of P were zeroed (sign 0): drop them from the FP32 factor, last
// first, or leave the factor to be rebuilt.
__device__ void drop_zeroed(FinShared& sh, int np) {
    if (sh.fac_np < 0 || sh.F.fp64) {
        __syncthreads();
        if (threadIdx.x == 0) sh.fac_np = -1;
        __syncthreads();
        return;
    }
    int cur = np;
    for (int a = np - 1; a >= 0; --a) {
        if (sh.sg[sh.P[a]] != 0) continue;
        if (cur <= FAC_INC_MAX) fac_remove(sh, a, cur);
        else fac_remove_cta(sh, a, cur);
        --cur;
    }
    __syncthreads();
    if (threadIdx.x == 0) sh.fac_np = cur;
    __syncthreads();
}

// The atom at position a joins P: append it to the FP32 factor, or leave the
// factor to be rebuilt.
__device__ void join_support(FinShared& sh, const float* Gi, int smax, int a, int np) {
    const bool ok = sh.fac_np >= 0 && !sh.F.fp64;
    __syncthreads();
    const int res = !ok ? -1 : (np < FAC_INC_MAX ? fac_append(sh, Gi, smax, a, np) : fac_append_cta(sh, Gi, smax, a, np));
    if (threadIdx.x == 0) sh.fac_np = res == 0 ? np + 1 : -1;
    __syncthreads();
}

// r = b - A_P x in double-FP32.  Each thread keeps 8 independent chains (8
// entries of r), so the loads of one atom column overlap the arithmetic.
__device__ void residual_df(const float* __restrict__ A, int n, const int* Pi, const df* xd, int np,
                            const float* __restrict__ b, float* rh, float* rl) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int k0 = 0; k0 < n; k0 += 8 * nt) {
        const int live = min(8, (n - k0 + nt - 1) / nt);  // slots with any entry in range
        df acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + tid + u * nt;
            acc[u] = df{k < n ? b[k] : 0.f, 0.f};
        }
        // four atom columns per pass, all loads issued before the arithmetic
        int a = 0;
        for (; a + 3 < np; a += 4) {
            const float* c0 = A + (size_t)Pi[a] * n;
            const float* c1 = A + (size_t)Pi[a + 1] * n;
            const float* c2 = A + (size_t)Pi[a + 2] * n;
            const float* c3 = A + (size_t)Pi[a + 3] * n;
            float v0[8], v1[8], v2[8], v3[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + tid + u * nt;
                const bool ok = u < live && k < n;
                v0[u] = ok ? __ldg(c0 + k) : 0.f;
                v1[u] = ok ? __ldg(c1 + k) : 0.f;
                v2[u] = ok ? __ldg(c2 + k) : 0.f;
                v3[u] = ok ? __ldg(c3 + k) : 0.f;
            }
            const df x0 = xd[a], x1 = xd[a + 1], x2 = xd[a + 2], x3 = xd[a + 3];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (u < live) {
                    acc[u] = df_fma(acc[u], -v0[u], x0);
                    acc[u] = df_fma(acc[u], -v1[u], x1);
                    acc[u] = df_fma(acc[u], -v2[u], x2);
                    acc[u] = df_fma(acc[u], -v3[u], x3);
                }
            }
        }
        for (; a < np; ++a) {
            const float* col = A + (size_t)Pi[a] * n;
            const df xa = xd[a];
            float av[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + tid + u * nt;
                av[u] = (u < live && k < n) ? __ldg(col + k) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (u < live) acc[u] = df_fma(acc[u], -av[u], xa);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + tid + u * nt;
            if (k < n) { rh[k] = acc[u].hi; rl[k] = acc[u].lo; }
        }
    }
}

// a^T r in double-FP32 by one warp (4 independent chains per lane); every lane
// returns the same value.
__device__ double dot_df(const float* __restrict__ a, const float* rh, const float* rl, int n) {
    const int lane = threadIdx.x & 31;
    df c0 = {0.f, 0.f}, c1 = c0, c2 = c0, c3 = c0;
    int k = lane;
    for (; k + 224 < n; k += 256) {  // 8 loads of the atom in flight per lane
        float av[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) av[u] = __ldg(a + k + 32 * u);
        c0 = df_fma(c0, av[0], df{rh[k], rl[k]});
        c1 = df_fma(c1, av[1], df{rh[k + 32], rl[k + 32]});
        c2 = df_fma(c2, av[2], df{rh[k + 64], rl[k + 64]});
        c3 = df_fma(c3, av[3], df{rh[k + 96], rl[k + 96]});
        c0 = df_fma(c0, av[4], df{rh[k + 128], rl[k + 128]});
        c1 = df_fma(c1, av[5], df{rh[k + 160], rl[k + 160]});
        c2 = df_fma(c2, av[6], df{rh[k + 192], rl[k + 192]});
        c3 = df_fma(c3, av[7], df{rh[k + 224], rl[k + 224]});
    }
    for (; k + 96 < n; k += 128) {
        const float a0 = __ldg(a + k), a1 = __ldg(a + k + 32), a2 = __ldg(a + k + 64), a3 = __ldg(a + k + 96);
        c0 = df_fma(c0, a0, df{rh[k], rl[k]});
        c1 = df_fma(c1, a1, df{rh[k + 32], rl[k + 32]});
        c2 = df_fma(c2, a2, df{rh[k + 64], rl[k + 64]});
        c3 = df_fma(c3, a3, df{rh[k + 96], rl[k + 96]});
    }
    for (; k < n; k += 32) c0 = df_fma(c0, __ldg(a + k), df{rh[k], rl[k]});
    df acc = df_add(df_add(c0, c1), df_add(c2, c3));
    acc = warp_df_sum(acc);
    return to_d(acc);
}

// a^T b of two FP32 atoms in double-FP32 (products are exact) by one warp.
__device__ double dot_ff(const float* __restrict__ a, const float* __restrict__ b, int n) {
    const int lane = threadIdx.x & 31;
    df c0 = {0.f, 0.f}, c1 = c0;
    int k = lane;
    for (; k + 32 < n; k += 64) {
        const float a0 = __ldg(a + k), b0 = __ldg(b + k), a1 = __ldg(a + k + 32), b1 = __ldg(b + k + 32);
        c0 = df_fma(c0, a0, df{b0, 0.f});
        c1 = df_fma(c1, a1, df{b1, 0.f});
    }
    for (; k < n; k += 32) c0 = df_fma(c0, __ldg(a + k), df{__ldg(b + k), 0.f});
    return to_d(warp_df_sum(df_add(c0, c1)));
}

// r = b - A_P x in double-FP32 for n % 4 == 0: thread t owns the four entries
// 4t + 4 nt c; the atom columns are read as float4, eight atoms per round so
// that eight loads are in flight.  Each entry sums the atoms in order of P, as
// residual_df does.
__device__ void residual_df4_range(const float* __restrict__ A, int n, const int* Pi, const df* xd, int np,
                                   const float* __restrict__ b, float* rh, float* rl, int k_lo, int k_hi) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int k = k_lo + tid * 4; k < k_hi; k += nt * 4) {
        const float4 bv = __ldg(reinterpret_cast<const float4*>(b + k));
        df c0{bv.x, 0.f}, c1{bv.y, 0.f}, c2{bv.z, 0.f}, c3{bv.w, 0.f};
        int a = 0;
        for (; a + 7 < np; a += 8) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldg(reinterpret_cast<const float4*>(A + (size_t)Pi[a + u] * n + k));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const df x = xd[a + u];
                c0 = df_fma(c0, -v[u].x, x);
                c1 = df_fma(c1, -v[u].y, x);
                c2 = df_fma(c2, -v[u].z, x);
                c3 = df_fma(c3, -v[u].w, x);
            }
        }
        for (; a < np; ++a) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(A + (size_t)Pi[a] * n + k));
            const df x = xd[a];
            c0 = df_fma(c0, -v.x, x);
            c1 = df_fma(c1, -v.y, x);
            c2 = df_fma(c2, -v.z, x);
            c3 = df_fma(c3, -v.w, x);
        }
        *reinterpret_cast<float4*>(rh + k) = make_float4(c0.hi, c1.hi, c2.hi, c3.hi);
        *reinterpret_cast<float4*>(rl + k) = make_float4(c0.lo, c1.lo, c2.lo, c3.lo);
    }
}

__device__ __forceinline__ void residual_df4(const float* __restrict__ A, int n, const int* Pi, const df* xd, int np,
                                             const float* __restrict__ b, float* rh, float* rl) {
    residual_df4_range(A, n, Pi, xd, np, b, rh, rl, 0, n);
}

// The same rows [k_lo, k_hi) when they are fewer than the CTA's threads (a cluster's block
// of a short residual): thread g nv + v takes float4 slot v and the atoms g, g + G, ... of P
// (G groups), group 0 starting from b; the groups' double-FP32 partial sums meet in scratch
// (blockDim.x x 8 floats) and are added in group order.  Ends with the CTA synchronised.
__device__ void residual_df4_groups(const float* __restrict__ A, int n, const int* Pi, const df* xd, int np,
                                    const float* __restrict__ b, float* rh, float* rl, int k_lo, int k_hi, int G,
                                    float* scratch) {
    const int tid = threadIdx.x;
    const int nv = (k_hi - k_lo) >> 2;
    const int g = tid / nv, v = tid - g * nv;
    if (g < G) {
        const int k = k_lo + 4 * v;
        df c0{0.f, 0.f}, c1 = c0, c2 = c0, c3 = c0;
        if (g == 0) {
            const float4 bv = __ldg(reinterpret_cast<const float4*>(b + k));
            c0.hi = bv.x; c1.hi = bv.y; c2.hi = bv.z; c3.hi = bv.w;
        }
        int a = g;
        for (; a + 7 * G < np; a += 8 * G) {
            float4 w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                w[u] = __ldg(reinterpret_cast<const float4*>(A + (size_t)Pi[a + u * G] * n + k));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const df x = xd[a + u * G];
                c0 = df_fma(c0, -w[u].x, x);
                c1 = df_fma(c1, -w[u].y, x);
                c2 = df_fma(c2, -w[u].z, x);
                c3 = df_fma(c3, -w[u].w, x);
            }
        }
        for (; a < np; a += G) {
            const float4 w = __ldg(reinterpret_cast<const float4*>(A + (size_t)Pi[a] * n + k));
            const df x = xd[a];
            c0 = df_fma(c0, -w.x, x);
            c1 = df_fma(c1, -w.y, x);
            c2 = df_fma(c2, -w.z, x);
            c3 = df_fma(c3, -w.w, x);
        }
        float4* sp = reinterpret_cast<float4*>(scratch + (size_t)tid * 8);
        sp[0] = make_float4(c0.hi, c0.lo, c1.hi, c1.lo);
        sp[1] = make_float4(c2.hi, c2.lo, c3.hi, c3.lo);
    }
    __syncthreads();
    if (tid < nv) {
        const float4* s0 = reinterpret_cast<const float4*>(scratch + (size_t)tid * 8);
        df c0{s0[0].x, s0[0].y}, c1{s0[0].z, s0[0].w}, c2{s0[1].x, s0[1].y}, c3{s0[1].z, s0[1].w};
        for (int q = 1; q < G; ++q) {
            const float4* sq = reinterpret_cast<const float4*>(scratch + (size_t)(q * nv + tid) * 8);
            c0 = df_add(c0, df{sq[0].x, sq[0].y});
            c1 = df_add(c1, df{sq[0].z, sq[0].w});
            c2 = df_add(c2, df{sq[1].x, sq[1].y});
            c3 = df_add(c3, df{sq[1].z, sq[1].w});
        }
        const int k = k_lo + 4 * tid;
        *reinterpret_cast<float4*>(rh + k) = make_float4(c0.hi, c1.hi, c2.hi, c3.hi);
        *reinterpret_cast<float4*>(rl + k) = make_float4(c0.lo, c1.lo, c2.lo, c3.lo);
    }
    __syncthreads();
}

// out[a] = a_{idx[a]}^T r for a < cnt, in double-FP32, two atoms per warp at a
// time (n % 4 == 0): lane l takes the float4 slices k = 4l + 128q, up to eight
// slices of both atoms in flight per round, the residual pair from shared
// memory; one butterfly per pair (the first level splits the two atoms over the
// half-warps).  Fixed summation order.
__device__ void dots_df_warp(const float* __restrict__ A, int n, const int* idx, int cnt, const float* rh,
                             const float* rl, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int a0 = 2 * warp; a0 < cnt; a0 += 2 * nw) {
        const bool two = a0 + 1 < cnt;
        const float* pa = A + (size_t)idx[a0] * n;
        const float* pb = A + (size_t)idx[two ? a0 + 1 : a0] * n;
        df sa0{0.f, 0.f}, sa1{0.f, 0.f}, sb0{0.f, 0.f}, sb1{0.f, 0.f};
        for (int k0 = lane * 4; k0 < n; k0 += 128 * 8) {
            float4 va[8], vb[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = k0 + 128 * q;
                va[q] = k < n ? __ldg(reinterpret_cast<const float4*>(pa + k)) : make_float4(0.f, 0.f, 0.f, 0.f);
                vb[q] = (two && k < n) ? __ldg(reinterpret_cast<const float4*>(pb + k)) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = k0 + 128 * q;
                if (k < n) {
                    const float4 h4 = *reinterpret_cast<const float4*>(rh + k);
                    const float4 l4 = *reinterpret_cast<const float4*>(rl + k);
                    sa0 = df_fma(sa0, va[q].x, df{h4.x, l4.x});
                    sa1 = df_fma(sa1, va[q].y, df{h4.y, l4.y});
                    sa0 = df_fma(sa0, va[q].z, df{h4.z, l4.z});
                    sa1 = df_fma(sa1, va[q].w, df{h4.w, l4.w});
                    sb0 = df_fma(sb0, vb[q].x, df{h4.x, l4.x});
                    sb1 = df_fma(sb1, vb[q].y, df{h4.y, l4.y});
                    sb0 = df_fma(sb0, vb[q].z, df{h4.z, l4.z});
                    sb1 = df_fma(sb1, vb[q].w, df{h4.w, l4.w});
                }
            }
        }
        df sa = df_add(sa0, sa1), sb = df_add(sb0, sb1);
        // level 16: the lower half-warp keeps atom a, the upper atom b
        const bool up = lane >= 16;
        df send = up ? sa : sb, keep = up ? sb : sa;
        df recv;
        recv.hi = __shfl_xor_sync(0xffffffffu, send.hi, 16);
        recv.lo = __shfl_xor_sync(0xffffffffu, send.lo, 16);
        keep = up ? df_add(recv, keep) : df_add(keep, recv);  // partner order: lower lane first
#pragma unroll
        for (int o = 8; o; o >>= 1) {
            df w;
            w.hi = __shfl_xor_sync(0xffffffffu, keep.hi, o);
            w.lo = __shfl_xor_sync(0xffffffffu, keep.lo, o);
            keep = df_add(keep, w);
        }
        if (lane == 0) out[a0] = to_d(keep);
        if (lane == 16 && two) out[a0 + 1] = to_d(keep);
    }
}

// Last resort for ill-conditioned blocks: G_PP recomputed from the atoms in
// double-FP32 into the FP64 factor storage, then factored in FP64.
__device__ int exact_factor(FinShared& sh, const float* A, int n, int np) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int e = warp; e < np * (np + 1) / 2; e += nw) {
        int r = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
        while ((r + 1) * (r + 2) / 2 <= e) ++r;
        while (r * (r + 1) / 2 > e) --r;
        const int c = e - r * (r + 1) / 2;
        const double v = dot_ff(A + (size_t)sh.Pi[r] * n, A + (size_t)sh.Pi[c] * n, n);
        if (lane == 0) sh.F.Md[(size_t)r * sh.F.ldd + c] = v;
    }
    __syncthreads();
    return factor(sh.F, np, &sh.ival[0]);
}

// Copy the lower triangle of G_PP into the current factor storage and factor it.
__device__ void gather_gram(FinShared& sh, const float* Gi, int smax, int np) {
    // the np x np lower triangle as one flat range of independent loads (row r holds
    // entries r(r+1)/2 .. r(r+1)/2 + r)
    const int tot = np * (np + 1) / 2;
    for (int e0 = threadIdx.x; e0 < tot; e0 += 4 * blockDim.x) {
        // four loads in flight before the stores (the stores could alias them)
        float v[4];
        int rr[4], cc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * blockDim.x;
            rr[u] = -1;
            if (e < tot) {
                int r = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
                while ((r + 1) * (r + 2) / 2 <= e) ++r;
                while (r * (r + 1) / 2 > e) --r;
                rr[u] = r;
                cc[u] = e - r * (r + 1) / 2;
                v[u] = __ldg(Gi + (size_t)sh.P[r] * smax + sh.P[cc[u]]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (rr[u] < 0) continue;
            if (sh.F.fp64) sh.F.Md[(size_t)rr[u] * sh.F.ldd + cc[u]] = (double)v[u];
            else sh.F.Mf[(size_t)rr[u] * sh.F.ldf + cc[u]] = v[u];
        }
    }
    __syncthreads();
}

__device__ int load_factor(FinShared& sh, const float* Gi, int smax, int np) {
    gather_gram(sh, Gi, smax, np);
    return factor(sh.F, np, &sh.ival[0]);
}

// ---------------------------------------------------------------- conjugate gradients
// FP32 block sum in a fixed order (warp butterfly, then the warps' totals in order); every
// thread returns the total.
__device__ __forceinline__ float bsumf(float v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = (double)v;
    __syncthreads();
    float t = 0.f;
    for (int w = 0; w < nw; ++w) t += (float)red[w];
    return t;
}

// ---------------------------------------------------------------- cluster finish
// When few signals finish at once (the last outer iterations, where each finish sits on the
// critical path), a signal's finish runs on a cluster of C CTAs (C SMs).  Every CTA runs the
// whole finish on identical data, so their control flow is identical; only the column sweeps
// are divided: the exact residual by row blocks of n / C entries, the correlations by blocks
// of the atom list, after which every CTA reads the other blocks from its peers' shared
// memory (distributed shared memory).  Before such reads, and before a CTA overwrites what
// its peers may still read, the cluster meets at a barrier built on two mbarriers per CTA used
// in turn (C arrivals, one remote arrive from each CTA), waited on with a bound: on expiry the
// CTA records DERR_TIMEOUT and the finish returns without its result.
constexpr uint64_t FIN_CLUSTER_WAIT_NS = 4000000000ull;

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Generic address of the same shared-memory object in CTA `rank` of the cluster.
template <typename T>
__device__ __forceinline__ T* peer_ptr(T* p, unsigned rank) {
    uint64_t out;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(reinterpret_cast<uint64_t>(p)), "r"(rank));
    return reinterpret_cast<T*>(out);
}

struct ClusterSync {
    uint64_t* bar;  // this CTA's two barriers (count C each)
    int C;
    unsigned phase;
};

// All threads of all C CTAs: returns false (uniformly within the CTA) when the wait expired.
// Each CTA arrives once on the barrier of every CTA of the cluster and waits on its own.
// Consecutive phases use the two barriers in turn: an arrival for phase k + 1 cannot land on
// a barrier that is still in phase k (with one barrier, a CTA that has passed phase k could
// complete a slower CTA's phase k before a third CTA's arrival for k), and an arrival for
// phase k + 2 comes only after every CTA has passed phase k + 1, so after the barrier of
// phase k has completed it.  The n-th phase of barrier b has parity n & 1.
__device__ bool csync(const Dev& d, ClusterSync& cs) {
    __syncthreads();
    uint64_t* bar = cs.bar + (cs.phase & 1u);
    if (threadIdx.x == 0) {
        asm volatile("fence.acq_rel.cluster;" ::: "memory");
        const uint32_t local = static_cast<uint32_t>(__cvta_generic_to_shared(bar));
        for (int r = 0; r < cs.C; ++r) {
            uint32_t remote;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(r));
            asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
        }
    }
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(bar));
    const uint32_t parity = (cs.phase >> 1) & 1u;
    bool ok = false;
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) { ok = true; break; }
        if ((it & 255u) == 0u) {
            uint64_t now;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
            if (it == 0) t0 = now;
            else if (now - t0 > FIN_CLUSTER_WAIT_NS) break;
        }
    }
    ++cs.phase;
    ok = __syncthreads_and(ok) != 0;
    if (!ok && threadIdx.x == 0) atomicCAS(&d.cnt->err, 0, (int)DERR_TIMEOUT);
#ifdef MPL_BOUNDS
    if (!ok && threadIdx.x == 0) atomicCAS(&d.cnt->bounds_site, 0, 706);
#endif
    return ok;
}

// Block b of [0, len) split into C parts (multiples of `align`).
__device__ __forceinline__ void part_of(int len, int C, int b, int align, int* lo, int* hi) {
    const int per = (((len + C - 1) / C) + align - 1) / align * align;
    *lo = min(len, b * per);
    *hi = min(len, *lo + per);
}

// r = b - A_P x: this CTA's row block (with the atoms spread over thread groups when the block
// has fewer float4 slots than the CTA has threads, given scratch of blockDim.x x 8 floats),
// then the other blocks from the peers.
__device__ bool residual_cluster(const Dev& d, ClusterSync& cs, unsigned rank, const float* A, int n,
                                 const int* Pi, const df* xd, int np, const float* b, float* rh, float* rl,
                                 float* scratch, int scratch_n) {
    int lo, hi;
    part_of(n, cs.C, (int)rank, 4, &lo, &hi);
#ifdef MPL_BOUNDS
    for (int a = threadIdx.x; a < np; a += blockDim.x)
        MPL_OOB(Pi[a] < 0 || Pi[a] >= d.m, 702);
    MPL_OOB(lo < 0 || hi > n || (lo & 3) || (hi & 3), 703);
#endif
    const int nv = (hi - lo) >> 2, nt = (int)blockDim.x;
    const int G = nv > 0 ? min(8, nt / nv) : 1;
    if (G >= 2 && scratch && scratch_n >= nt * 8)
        residual_df4_groups(A, n, Pi, xd, np, b, rh, rl, lo, hi, G, scratch);
    else
        residual_df4_range(A, n, Pi, xd, np, b, rh, rl, lo, hi);
    if (!csync(d, cs)) return false;
    for (int q = 1; q < cs.C; ++q) {
        const unsigned pr = (rank + q) % cs.C;
        int plo, phi;
        part_of(n, cs.C, (int)pr, 4, &plo, &phi);
        const float4* sh4 = reinterpret_cast<const float4*>(peer_ptr(rh, pr));
        const float4* sl4 = reinterpret_cast<const float4*>(peer_ptr(rl, pr));
        for (int k = plo + 4 * (int)threadIdx.x; k < phi; k += 4 * (int)blockDim.x) {
            reinterpret_cast<float4*>(rh)[k >> 2] = sh4[k >> 2];
            reinterpret_cast<float4*>(rl)[k >> 2] = sl4[k >> 2];
        }
    }
    return csync(d, cs);  // no peer overwrites its block before every CTA has read it
}

// out[a] = a_{idx[a]}^T r for a < cnt: this CTA's block of atoms, then the others' results.
__device__ bool dots_cluster(const Dev& d, ClusterSync& cs, unsigned rank, const float* A, int n, const int* idx,
                             int cnt, const float* rh, const float* rl, double* out) {
    int lo, hi;
    part_of(cnt, cs.C, (int)rank, 2, &lo, &hi);
#ifdef MPL_BOUNDS
    for (int a = threadIdx.x; a < cnt; a += blockDim.x)
        MPL_OOB(idx[a] < 0 || idx[a] >= d.m, 704);
#endif
    if (hi > lo) dots_df_warp(A, n, idx + lo, hi - lo, rh, rl, out + lo);
    if (!csync(d, cs)) return false;
    for (int q = 1; q < cs.C; ++q) {
        const unsigned pr = (rank + q) % cs.C;
        int plo, phi;
        part_of(cnt, cs.C, (int)pr, 2, &plo, &phi);
        const double* po = peer_ptr(out, pr);
        for (int a = plo + (int)threadIdx.x; a < phi; a += (int)blockDim.x) out[a] = po[a];
    }
    return csync(d, cs);
}

// q_a = (G_SS v)_a for the support positions a = P[k] (v is zero outside P, so this is
// G_PP v_P): a warp per pair of rows, the row's first s entries as float4 slices when the
// block's leading dimension allows (else scalar), fixed butterfly per row.
__device__ __noinline__ void gram_rows_mv(const float* __restrict__ Gi, int smax, int s, const int* P, int np,
                             const float* v, float* q) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool vec = (smax & 3) == 0;
    for (int k = 2 * warp; k < np; k += 2 * nw) {
        const int ra = P[k], rb = k + 1 < np ? P[k + 1] : P[k];
        const float* ga = Gi + (size_t)ra * smax;
        const float* gb = Gi + (size_t)rb * smax;
        float sa = 0.f, sb = 0.f;
        for (int c0 = 4 * lane; c0 < s; c0 += 512) {
            float4 a4[4], b4[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = c0 + 128 * u;
                if (c < s) {
                    if (vec) {
                        a4[u] = __ldg(reinterpret_cast<const float4*>(ga + c));
                        b4[u] = __ldg(reinterpret_cast<const float4*>(gb + c));
                    } else {
                        a4[u] = make_float4(__ldg(ga + c), c + 1 < s ? __ldg(ga + c + 1) : 0.f,
                                            c + 2 < s ? __ldg(ga + c + 2) : 0.f, c + 3 < s ? __ldg(ga + c + 3) : 0.f);
                        b4[u] = make_float4(__ldg(gb + c), c + 1 < s ? __ldg(gb + c + 1) : 0.f,
                                            c + 2 < s ? __ldg(gb + c + 2) : 0.f, c + 3 < s ? __ldg(gb + c + 3) : 0.f);
                    }
                } else {
                    a4[u] = b4[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = c0 + 128 * u;
                if (c < s) {
                    // v has zeros from s up to the next multiple of 4 (and outside P)
                    const float4 x = *reinterpret_cast<const float4*>(v + c);
                    sa = fmaf(a4[u].x, x.x, sa); sa = fmaf(a4[u].y, x.y, sa);
                    sa = fmaf(a4[u].z, x.z, sa); sa = fmaf(a4[u].w, x.w, sa);
                    sb = fmaf(b4[u].x, x.x, sb); sb = fmaf(b4[u].y, x.y, sb);
                    sb = fmaf(b4[u].z, x.z, sb); sb = fmaf(b4[u].w, x.w, sb);
                }
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
            sb += __shfl_xor_sync(0xffffffffu, sb, o);
        }
        if (lane == 0) {
            q[ra] = sa;
            if (k + 1 < np) q[rb] = sb;
        }
    }
}

// Conjugate gradients for G_PP z = rhs in FP32 (supports whose FP32 factor would not fit
// shared memory; the Gram blocks of these workloads are well conditioned).  io holds the
// right-hand side on entry and the solution on exit, both indexed by support slot k < np;
// x0 (indexed by S position, may be null) is the warm start on P.  The four vectors are
// kept by S position in `vec` (4 x ld floats, 16-byte aligned, ld >= s rounded up to 4):
// z, r, p (zero outside P, the product's operand) and q = G p.  Stops when the recurred
// residual is at most rtol ||rhs||; returns the iterations taken, or -1 when maxit is
// reached or the curvature p^T G p is not positive (the caller falls back to a factor).
// G_PP v for the CG: the whole block by this CTA, or in a clustered finish this CTA's block
// of rows followed by the other rows' products from the peers (each row by one CTA, with
// the same arithmetic, so the product does not depend on the cluster size).  false: a
// cluster barrier timed out.
__device__ bool cg_product(const Dev& d, ClusterSync* cs, unsigned rank, const float* Gi, int smax, int s,
                           const int* P, int np, const float* v, float* q) {
    if (!cs || cs->C <= 1) {
        gram_rows_mv(Gi, smax, s, P, np, v, q);
        return true;
    }
    int lo, hi;
    part_of(np, cs->C, (int)rank, 2, &lo, &hi);
#ifdef MPL_BOUNDS
    for (int k = threadIdx.x; k < np; k += blockDim.x)
        MPL_OOB(P[k] < 0 || P[k] >= s, 705);
#endif
    if (hi > lo) gram_rows_mv(Gi, smax, s, P + lo, hi - lo, v, q);
    if (!csync(d, *cs)) return false;
    for (int r = 1; r < cs->C; ++r) {
        const unsigned pr = (rank + r) % cs->C;
        int plo, phi;
        part_of(np, cs->C, (int)pr, 2, &plo, &phi);
        const float* pq = peer_ptr(q, pr);
        for (int k = plo + (int)threadIdx.x; k < phi; k += (int)blockDim.x) q[P[k]] = pq[P[k]];
    }
    return csync(d, *cs);
}

// Returns the iterations taken, -1 when it does not converge, -2 when a cluster barrier
// timed out (the finish must return).
__device__ __noinline__ int cg_solve(FinShared& sh, const float* Gi, int smax, int s, int np, double* io, const double* x0,
                        float rtol, int maxit, float* vec, int ld, const Dev& d, ClusterSync* cs, unsigned rank) {
    const int tid = threadIdx.x, nt = blockDim.x;
    float* z = vec;
    float* r = vec + ld;
    float* p = vec + 2 * ld;
    float* q = vec + 3 * ld;
    const int sp = (s + 3) & ~3;
    for (int a = tid; a < sp; a += nt) { p[a] = 0.f; z[a] = 0.f; }
    __syncthreads();
    float bb = 0.f;
    for (int k = tid; k < np; k += nt) {
        const int a = sh.P[k];
        const float rhs = (float)io[k];
        bb = fmaf(rhs, rhs, bb);
        r[a] = rhs;
        if (x0) { z[a] = (float)x0[a]; p[a] = z[a]; }
    }
    bb = bsumf(bb, sh.red);
    if (x0) {  // r = rhs - G z0
        if (!cg_product(d, cs, rank, Gi, smax, s, sh.P, np, p, q)) return -2;
        __syncthreads();
        for (int k = tid; k < np; k += nt) { const int a = sh.P[k]; r[a] -= q[a]; }
        __syncthreads();
    }
    float rr = 0.f;
    for (int k = tid; k < np; k += nt) { const int a = sh.P[k]; rr = fmaf(r[a], r[a], rr); p[a] = r[a]; }
    rr = bsumf(rr, sh.red);
    const float stop2 = rtol * rtol * bb;
    int it = 0;
    int ok = 0;
    for (;;) {
        if (rr <= stop2) { ok = 1; break; }
        if (it >= maxit) break;
        if (!cg_product(d, cs, rank, Gi, smax, s, sh.P, np, p, q)) return -2;
        __syncthreads();
        float pq = 0.f;
        for (int k = tid; k < np; k += nt) { const int a = sh.P[k]; pq = fmaf(p[a], q[a], pq); }
        pq = bsumf(pq, sh.red);
        if (!(pq > 0.f)) break;
        const float alpha = rr / pq;
        float rn = 0.f;
        for (int k = tid; k < np; k += nt) {
            const int a = sh.P[k];
            z[a] = fmaf(alpha, p[a], z[a]);
            const float ra = fmaf(-alpha, q[a], r[a]);
            r[a] = ra;
            rn = fmaf(ra, ra, rn);
        }
        rn = bsumf(rn, sh.red);
        const float beta = rn / rr;
        rr = rn;
        for (int k = tid; k < np; k += nt) { const int a = sh.P[k]; p[a] = fmaf(beta, p[a], r[a]); }
        __syncthreads();
        ++it;
    }
    for (int k = tid; k < np; k += nt) io[k] = (double)z[sh.P[k]];
    __syncthreads();
    return ok ? it : -1;
}

// NT = FIN_THREADS (two CTAs per SM) or FIN_THREADS_WIDE (one CTA per SM, taken when the
// shared-memory layout allows only one anyway: the wider CTA shortens the latency-bound
// sweeps over the support's columns).
// C > 1: a cluster of C CTAs per signal (C consecutive blocks), see csync.
template <int NT>
__global__ void __launch_bounds__(NT, 2 * FIN_THREADS / NT) k_finish(Dev d, int cur, int scap, int msm, int rsm,
                                                                      int C) {
    const int g = blockIdx.x / C;
    if (g >= d.cnt->fin_par[cur]) return;
    const int i = d.list_fin[cur][g];
    extern __shared__ __align__(16) double fsm[];
    __shared__ FinShared sh;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int n = d.n, smax = d.smax, s = d.ssize[i];
    if (s > scap) {
        if (tid == 0) atomicCAS(&d.cnt->err, 0, (int)DERR_SHAPE);
        return;
    }
    if (tid == 0) {
        double* p = fsm;
        sh.x = p; p += scap;
        sh.z = p; p += scap;
        sh.w = p; p += scap;
        sh.F.rdd = p; p += scap;
        float* q = reinterpret_cast<float*>(p);
        sh.F.rdf = q; q += scap;
        sh.F.vf = q; q += scap;
        // the FP32 factor sits in shared memory when the signal's whole active set fits
        // the msm x msm area the launch reserved, else in the signal's global workspace;
        // an odd stride spreads a column over the banks
        const bool fsm = s <= msm;
        sh.F.ldf = fsm ? ((msm + 1) | 1) : ((scap + 1) | 1);
        // the factor workspace: the signal's own, or in a clustered finish this CTA's slot of
        // the pool (the CTAs of a cluster factor the same block side by side); the finishes of
        // the FIN_SLOTS list slots run concurrently, so each slot has its own part
        double* wk = C > 1 ? d.fin_pool + ((size_t)cur * d.fin_slots + blockIdx.x) * smax * smax
                           : d.chol + (size_t)i * smax * smax;
        sh.F.Mf = fsm ? q : reinterpret_cast<float*>(wk);
        if (msm) q += (size_t)msm * ((msm + 1) | 1);
        sh.F.stage = msm ? nullptr : q;  // panel staging for a factor in global memory
        sh.F.stage_n = msm ? 0 : fac_stage_floats(scap);
        if (!msm) q += (size_t)fac_stage_floats(scap);
        sh.P = reinterpret_cast<int*>(q);
        sh.sg = sh.P + scap;
        sh.Pi = sh.sg + scap;
        sh.adds = sh.Pi + scap;
        // residual pair in shared memory when it fits (rsm), else in the global R32 / R32lo rows
        // (16-byte aligned: the residual rows are read and written as float4)
        float* rbase = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(sh.adds + scap) + 15) & ~(uintptr_t)15);
        sh.rh = rsm ? rbase : d.R32 + (size_t)i * d.n;
        sh.rl = rsm ? rbase + d.n : d.R32lo + (size_t)i * d.n;
        sh.F.Md = wk;  // shares the workspace with a global FP32 factor
        sh.F.ldd = smax;
        sh.F.fp64 = 0;
        // supports too large for a shared-memory factor are solved by conjugate gradients on
        // the Gram block (their vectors in the staging area); a factor in global memory is the
        // fallback when CG does not converge
        sh.cg = (msm == 0 && s > FIN_CG_MIN_S) ? 1 : 0;
        if (C > 1) {
            for (int q = 0; q < 2; ++q)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(
                                 static_cast<uint32_t>(__cvta_generic_to_shared(&sh.cbar[q]))),
                             "r"(C)
                             : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    __syncthreads();
    // every CTA's barrier is initialised before any remote arrive (reached by all CTAs of the
    // cluster: the returns above depend only on the signal, which they share)
    if (C > 1) {
        asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
    const unsigned rank = C > 1 ? cluster_rank() : 0u;
    ClusterSync cs{sh.cbar, C, 0u};
    // (the cluster's last block bounds every block's workspace slot: a uniform check)
    if (MPL_OOB(C > 1 && ((int)(blockIdx.x / C) * C + C > d.fin_slots || (int)rank >= C), 701)) return;
    float* cgv = msm ? nullptr
                     : reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(sh.F.stage) + 15) & ~(uintptr_t)15);
    const double lam = (double)d.lam[i];
    const double tol = d.tol;
    const bool vec4 = (n & 3) == 0;  // float4 rows: block-cooperative residual and correlations
    const bool lam0 = !(lam > 0.0);
    // scale of the optimality conditions on S: lambda, or a bound on |a_j^T b| when lambda = 0
    const double lsc = lam0 ? fmax((double)d.colmax * (double)d.bnorm[i], 1e-300) : lam;
    const int* Si = d.S + (size_t)i * smax;
    const float* Gi = d.G + (size_t)i * smax * smax;
    const float* hi = d.h + (size_t)i * smax;
    float* xS = d.xS + (size_t)i * smax;
    const float* b = d.B + (size_t)i * n;
    float* rh = sh.rh;
    float* rl = sh.rl;

    if (MPL_OOB(s > smax || i < 0 || i >= d.p, 601)) return;
    for (int a = tid; a < s; a += nt) {
        const float v = xS[a];
        sh.x[a] = (double)v;
        // lambda = 0 (least squares): every atom of S stays, signs play no part
        sh.sg[a] = lam0 ? 1 : (v > 0.f ? 1 : (v < 0.f ? -1 : 0));
    }
    __syncthreads();
    // every CTA of a cluster has read the signal's point before the first one can write it back
    if (C > 1 && !csync(d, cs)) return;

    FT_BEGIN
    FT_CNT(19);
    bool ok = false;
    double kkt_on = 0.0, cmax_s = 0.0;
    int np = 0;
    const int max_steps = s + 32;
    if (tid == 0) { sh.ival[3] = 0; sh.fac_np = -1; }  // ival[3] = 1: the last step added an atom from the exact check
    for (int a = tid; a < s; a += nt) sh.adds[a] = 0;
    __syncthreads();
    int steps = 0;
    unsigned long long flops = 0;  // algorithmic work (thread 0 keeps the tally)
    unsigned long long bytes = 0;  // algorithmic bytes streamed: Gram rows, atom columns, b
    for (int step = 0; step < max_steps; ++step, ++steps) {
        // the FP32 factor of the previous step, updated for the atoms that left or joined P,
        // or a new support list and factor
        const bool inc = sh.fac_np >= 0 && !sh.F.fp64;
        np = inc ? sh.fac_np : build_support(s, sh);
        // ---- solve on P
        if (np > 0) {
            for (int a = tid; a < np; a += nt) sh.z[a] = (double)hi[sh.P[a]] - lam * (double)sh.sg[sh.P[a]];
            FT_CNT(6);
            if (sh.cg) {
                // the sign-fixed system from the current point (the master problem's solution)
                const int it = cg_solve(sh, Gi, smax, s, np, sh.z, sh.x, 1e-6f, FIN_CG_MAXIT, cgv, (scap + 3) & ~3,
                                        d, &cs, rank);
                FT_ADD(1);
                FT_VAL(16, it);
                FT_CNT(17);
                if (it == -2) return;
                if (it < 0) {  // not converging: factor this signal's blocks from now on
                    __syncthreads();
                    if (tid == 0) sh.cg = 0;
                    __syncthreads();
                    --step;
                    continue;
                }
                flops += (unsigned long long)(it + 1) * 2ull * np * np;
                bytes += (unsigned long long)(it + 1) * 4ull * np * s;  // rows of G_PS per product
            } else {
                if (!inc) {
                    flops += (unsigned long long)np * np * np / 3 + 2ull * np * np;
                    bytes += 2ull * np * (np + 1);  // the lower triangle of G_PP gathered
                    FT_SPLIT(8);
                    gather_gram(sh, Gi, smax, np);
                    FT_SPLIT(9);
                    const int fres = factor(sh.F, np, &sh.ival[0]);
                    FT_ADD(0);
                    if (fres != 0) {
                        if (sh.F.fp64) break;
                        __syncthreads();
                        if (tid == 0) sh.F.fp64 = 1;  // FP32 pivot breakdown: retry this step in FP64
                        __syncthreads();
                        --step;
                        continue;
                    }
                } else {
                    flops += 2ull * np * np;
                }
                fsolve(sh.F, np, sh.z);
                FT_ADD(1);
            }
        }
        if (tid == 0) sh.fac_np = (!sh.F.fp64 && !sh.cg) ? np : -1;
        __syncthreads();
        // ---- first sign crossing on the segment x -> z.  Skipped right after the
        // exact check admitted an atom: its coefficient may be below the FP32
        // Gram block's resolution, so it goes straight to exact refinement.
        const bool exact_entry = sh.ival[3] != 0;
        __syncthreads();
        if (tid == 0) { sh.dval[1] = 2.0; sh.ival[2] = -1; sh.ival[3] = 0; }
        __syncthreads();
        if (!exact_entry && !lam0) {
          for (int a = tid; a < np; a += nt) {
            const int pa = sh.P[a];
            const double xa = sh.x[pa], za = sh.z[a];
            if (!(za * (double)sh.sg[pa] > 0.0)) {
                const double t = xa / (xa - za);  // in [0, 1]: xa has the sign, za not
                // smallest crossing; ties to the lowest position (deterministic)
                unsigned long long key = ((unsigned long long)__double_as_longlong(fmax(t, 0.0)) & ~0xFFFull) |
                                         (unsigned long long)pa;
                atomicMin(reinterpret_cast<unsigned long long*>(&sh.dval[1]), key);
                sh.ival[2] = 1;
            }
          }
        }
        __syncthreads();
        FT_ADD(2);
        if (sh.ival[2] > 0) {
            const unsigned long long key = (unsigned long long)__double_as_longlong(sh.dval[1]);
            const int pstar = (int)(key & 0xFFFull);
            double t = __longlong_as_double((long long)(key & ~0xFFFull));
            t = fmin(fmax(t, 0.0), 1.0);
            for (int a = tid; a < np; a += nt) {
                const int pa = sh.P[a];
                double v = sh.x[pa] + t * (sh.z[a] - sh.x[pa]);
                if (pa == pstar || !(v * (double)sh.sg[pa] > 0.0)) v = 0.0;
                sh.x[pa] = v;
            }
            __syncthreads();
            for (int a = tid; a < np; a += nt) {
                const int pa = sh.P[a];
                if (sh.x[pa] == 0.0) sh.sg[pa] = 0;
            }
            __syncthreads();
            drop_zeroed(sh, np);
            continue;
        }
        // consistent: x <- z on P (zero elsewhere)
        for (int a = tid; a < s; a += nt) if (sh.sg[a] == 0) sh.x[a] = 0.0;
        __syncthreads();
        for (int a = tid; a < np; a += nt) sh.x[sh.P[a]] = sh.z[a];
        __syncthreads();
        // ---- zero entries of S through the Gram block: add the largest violator
        if (tid == 0) sh.dval[2] = 0.0;
        __syncthreads();
        for (int a = warp; a < s; a += nw) {
            if (sh.sg[a] != 0) continue;
            double acc = 0.0;
            for (int c = lane; c < np; c += 32)
                acc += (double)Gi[(size_t)a * smax + sh.P[c]] * sh.x[sh.P[c]];
#pragma unroll
            for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            const double ca = (double)hi[a] - acc;
            if (lane == 0 && fabs(ca) > lam * (1.0 + 1e-3)) {  // well beyond the Gram block's resolution
                // largest |c|, ties to the lowest position
                unsigned long long key = ((unsigned long long)__double_as_longlong(fabs(ca)) & ~0xFFFull) |
                                         (unsigned long long)(0xFFF - a);
                atomicMax(reinterpret_cast<unsigned long long*>(&sh.dval[2]), key);
            }
        }
        __syncthreads();
        FT_ADD(3);
        if (sh.dval[2] != 0.0) {
            const unsigned long long key = (unsigned long long)__double_as_longlong(sh.dval[2]);
            const int a = 0xFFF - (int)(key & 0xFFFull);
            if (tid == 0) {
                double acc = 0.0;
                for (int c = 0; c < np; ++c) acc += (double)Gi[(size_t)a * smax + sh.P[c]] * sh.x[sh.P[c]];
                sh.sg[a] = ((double)hi[a] - acc) > 0.0 ? 1 : -1;
                sh.ival[0] = ++sh.adds[a] > 3;  // an atom that keeps re-entering: give up
            }
            __syncthreads();
            if (sh.ival[0]) break;
            join_support(sh, Gi, smax, a, np);
            continue;
        }
        // ---- exact verification: r = b - A_P x, c = A^T r (double-FP32), Newton refinement on P
        double dmax = 0.0, dprev = 0.0;
        bool broke = false, exact_g = false;
        df* xd = reinterpret_cast<df*>(sh.z);  // z is free now: x_P split into FP32 pairs
        for (int a = tid; a < np; a += nt) sh.Pi[a] = Si[sh.P[a]];
        for (int ref = 0; ref < 24; ++ref) {
            for (int a = tid; a < np; a += nt) xd[a] = to_df(sh.x[sh.P[a]]);
            __syncthreads();
            FX_BEGIN
            FT_CNT(11);
            if (vec4) {
                if (C > 1) {
                    if (!residual_cluster(d, cs, rank, d.A32, n, sh.Pi, xd, np, b, rh, rl, cgv,
                                          msm ? 0 : sh.F.stage_n - 4))
                        return;
                } else {
                    residual_df4(d.A32, n, sh.Pi, xd, np, b, rh, rl);
                }
            } else {
                residual_df(d.A32, n, sh.Pi, xd, np, b, rh, rl);
            }
            __syncthreads();
            flops += 4ull * n * np;  // residual and on-support correlations
            bytes += 8ull * n * np + 4ull * n;  // the support's columns twice, and b
            double lmax = 0.0;
            if (vec4) {
                if (C > 1) {
                    if (!dots_cluster(d, cs, rank, d.A32, n, sh.Pi, np, rh, rl, sh.w)) return;
                } else {
                    dots_df_warp(d.A32, n, sh.Pi, np, rh, rl, sh.w);
                }
                __syncthreads();
                for (int a = tid; a < np; a += nt) {
                    const double dv = sh.w[a] - lam * (double)sh.sg[sh.P[a]];
                    sh.w[a] = dv;
                    lmax = fmax(lmax, fabs(dv));
                }
            } else {
                for (int a = warp; a < np; a += nw) {
                    const double dv = dot_df(d.A32 + (size_t)sh.Pi[a] * n, rh, rl, n) - lam * (double)sh.sg[sh.P[a]];
                    if (lane == 0) sh.w[a] = dv;
                    lmax = fmax(lmax, fabs(dv));
                }
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
            __syncthreads();
            FX_END(10);
            if (lane == 0) sh.red[warp] = lmax;
            __syncthreads();
            dmax = 0.0;
            for (int q = 0; q < nw; ++q) dmax = fmax(dmax, sh.red[q]);
            if (np == 0 || dmax <= 0.1 * tol * lsc) break;
            if (ref > 0 && dmax > 0.25 * dprev) {
                // slow contraction: CG's FP32 block limits it (factor it), or the FP32 factor
                // does (refactor once in FP64)
                if (sh.cg) {
                    __syncthreads();
                    if (tid == 0) sh.cg = 0;
                    __syncthreads();
                    if (load_factor(sh, Gi, smax, np) != 0) { broke = true; break; }
                } else if (!sh.F.fp64) {
                    __syncthreads();
                    if (tid == 0) sh.F.fp64 = 1;
                    __syncthreads();
                    FX_BEGIN
                    FT_CNT(13);
                    if (load_factor(sh, Gi, smax, np) != 0) { broke = true; break; }
                    FX_END(14);
                } else if (dmax >= dprev) {
                    if (exact_g) break;  // no further progress possible
                    exact_g = true;      // the FP32 Gram block limits it: rebuild it exactly
                    FT_CNT(15);
                    if (exact_factor(sh, d.A32, n, np) != 0) { broke = true; break; }
                }
            }
            dprev = dmax;
            FT_CNT(7);
            FX_BEGIN
            if (sh.cg) {
                const int it = cg_solve(sh, Gi, smax, s, np, sh.w, nullptr, 1e-4f, FIN_CG_MAXIT, cgv, (scap + 3) & ~3,
                                        d, &cs, rank);
                FT_VAL(18, it);
                if (it == -2) return;
                if (it < 0) {
                    // not converging: factor the block and evaluate the correction again
                    __syncthreads();
                    if (tid == 0) sh.cg = 0;
                    __syncthreads();
                    if (load_factor(sh, Gi, smax, np) != 0) { broke = true; break; }
                    continue;
                }
                flops += (unsigned long long)(it + 1) * 2ull * np * np;
                bytes += (unsigned long long)(it + 1) * 4ull * np * s;
            } else {
                flops += 2ull * np * np;
                fsolve(sh.F, np, sh.w);
            }
            FX_END(12);
            for (int a = tid; a < np; a += nt) sh.x[sh.P[a]] += sh.w[a];
            __syncthreads();
        }
        FT_ADD(4);
        if (broke) break;
        // on exit w holds c_P - lambda*s_P of the last evaluated residual
        // sign consistency after refinement
        if (tid == 0) sh.ival[0] = 0;
        __syncthreads();
        for (int a = tid; a < np; a += nt) {
            const int pa = sh.P[a];
            if (!lam0 && !(sh.x[pa] * (double)sh.sg[pa] > 0.0)) { sh.sg[pa] = 0; sh.x[pa] = 0.0; sh.ival[0] = 1; }
        }
        __syncthreads();
        if (sh.ival[0]) {
            drop_zeroed(sh, np);
            continue;
        }
        flops += 2ull * n * (unsigned long long)(s - np);
        bytes += 4ull * n * (unsigned long long)(s - np);  // the zero entries' columns
        // exact check of the zero entries of S
        double cmax = 0.0;
        int worst = -1;
        if (vec4) {
            // zero entries of S: atom indices after those of P in Pi, positions in z (free now)
            int* zpos = reinterpret_cast<int*>(sh.z);
            if (warp == 0) {
                int base = 0;
                for (int a0 = 0; a0 < s; a0 += 32) {
                    const int a = a0 + lane;
                    const bool z0 = a < s && sh.sg[a] == 0;
                    const unsigned bal = __ballot_sync(0xffffffffu, z0);
                    if (z0) {
                        const int k = base + __popc(bal & ((1u << lane) - 1u));
                        zpos[k] = a;
                        sh.Pi[np + k] = Si[a];
                    }
                    base += __popc(bal);
                }
                if (lane == 0) sh.ival[2] = base;
            }
            __syncthreads();
            const int nz = sh.ival[2];
            if (C > 1) {
                if (!dots_cluster(d, cs, rank, d.A32, n, sh.Pi + np, nz, rh, rl, sh.w + np)) return;
            } else {
                dots_df_warp(d.A32, n, sh.Pi + np, nz, rh, rl, sh.w + np);
            }
            __syncthreads();
            for (int k = tid; k < nz; k += nt) {
                const double ca = sh.w[np + k];
                if (fabs(ca) > cmax) { cmax = fabs(ca); worst = zpos[k]; }
            }
        } else {
            for (int a = warp; a < s; a += nw) {
                if (sh.sg[a] != 0) continue;
                const double ca = dot_df(d.A32 + (size_t)Si[a] * n, rh, rl, n);
                if (fabs(ca) > cmax) { cmax = fabs(ca); worst = a; }
            }
        }
        if (tid == 0) sh.dval[3] = 0.0;
        __syncthreads();
        if ((vec4 || lane == 0) && worst >= 0 && cmax > lam * (1.0 + tol)) {
            unsigned long long key = ((unsigned long long)__double_as_longlong(cmax) & ~0xFFFull) |
                                     (unsigned long long)(0xFFF - worst);
            atomicMax(reinterpret_cast<unsigned long long*>(&sh.dval[3]), key);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
        __syncthreads();
        if (lane == 0) sh.red[warp] = cmax;
        __syncthreads();
        cmax_s = 0.0;
        for (int q = 0; q < nw; ++q) cmax_s = fmax(cmax_s, sh.red[q]);
        FT_ADD(5);
        if (sh.dval[3] != 0.0) {
            const unsigned long long key = (unsigned long long)__double_as_longlong(sh.dval[3]);
            const int a = 0xFFF - (int)(key & 0xFFFull);
            // sign of the exact correlation of the entering atom
            if (warp == 0) {
                const double ca = dot_df(d.A32 + (size_t)Si[a] * n, rh, rl, n);
                if (lane == 0) {
                    sh.sg[a] = ca > 0.0 ? 1 : -1;
                    sh.ival[3] = 1;  // enters through exact refinement
                    sh.ival[0] = ++sh.adds[a] > 3;
                }
            }
            __syncthreads();
            if (sh.ival[0]) break;
            join_support(sh, Gi, smax, a, np);
            continue;
        }
        kkt_on = fmax(dmax / lsc, fmax(cmax_s - lam, 0.0) / lsc);
        ok = kkt_on <= tol;
        break;
    }

    // (the CTAs of a cluster hold the same result: the first one writes it)
    if (tid == 0 && rank == 0) {
        atomicAdd(&d.cnt->fin_flops, flops);
        atomicAdd(&d.cnt->fin_bytes, bytes);
    }
    if (rank != 0) {
        csync(d, cs);  // the peers' reads of this CTA's shared memory are over
        return;
    }
    if (ok) {
        double* x64 = d.xS64 + (size_t)i * smax;
        double l1 = 0.0, cm = 0.0;
        for (int a = tid; a < s; a += nt) {
            const double v = sh.x[a];
            x64[a] = v;
            xS[a] = (float)v;
            l1 += fabs(v);
        }
        for (int a = tid; a < np; a += nt) cm = fmax(cm, fabs(sh.w[a] + lam * (double)sh.sg[sh.P[a]]));
        double* r64 = d.R64 + (size_t)i * n;
        double rr = 0.0, rb = 0.0, rs = 0.0, es = 0.0, ts = 0.0;
        for (int k = tid; k < n; k += nt) {
            const double v = (double)rh[k] + (double)rl[k];
            r64[k] = v;
            if (rsm) { d.R32[(size_t)i * n + k] = rh[k]; d.R32lo[(size_t)i * n + k] = rl[k]; }
            const __nv_bfloat16 q = __float2bfloat16_rn(rh[k]);
            if (d.R16) d.R16[(size_t)i * n + k] = q;  // (copied into the GEMM's rows on re-entry)
            rr += v * v;
            rb += v * (double)b[k];
            rs += (double)rh[k] * (double)rh[k];
            const double fq = (double)__bfloat162float(q), e = (double)rh[k] - fq;
            es += e * e;
            ts += fq * fq;
        }
        const double L1 = bsum(l1, sh.red);
        const double RR = bsum(rr, sh.red);
        const double RB = bsum(rb, sh.red);
        const double RS = bsum(rs, sh.red);
        const double ES = bsum(es, sh.red);
        const double TS = bsum(ts, sh.red);
#pragma unroll
        for (int o = 16; o; o >>= 1) cm = fmax(cm, __shfl_xor_sync(0xffffffffu, cm, o));
        __syncthreads();
        if (lane == 0) sh.red[warp] = cm;
        __syncthreads();
        if (tid == 0) {
            double CM = 0.0;
            for (int q = 0; q < nw; ++q) CM = fmax(CM, sh.red[q]);
            d.obj[i] = lam * L1 + 0.5 * RR;
            d.rr[i] = RR;
            d.rb[i] = RB;
            d.rnorm[i] = (float)(sqrt(RS) * (1.0 + 1e-5));
            d.r16e[i] = (float)(sqrt(ES) * (1.0 + 1e-5));
            d.r16t[i] = (float)(sqrt(TS) * (1.0 + 1e-5));
            if (d.xl1) d.xl1[i] = __double2float_ru(L1 * (1.0 + 1e-6));
            d.kkt_in[i] = kkt_on;
            d.ginf[i] = fmax(CM, cmax_s);
            d.nnz[i] = np;
            d.finalized[i] = 1;
            d.fails[i] = 0;
            d.finishes[i] += steps + 1;
            if (d.early && d.early[i]) {  // an early-stopping rule ended this signal
                d.state[i] = ST_DONE;
                d.sstatus[i] = MPL_SIG_EARLY_STOP;
            } else {
                // back into the active list once this finish is done: the worst-case
                // analysis of its exact residual certifies the atoms outside S (eq. 8)
                d.reent[cur][atomicAdd(&d.cnt->reent_n[cur], 1)] = i;
            }
        }
    } else {
        // keep the (monotonically improved) point as the next warm start
        for (int a = tid; a < s; a += nt) xS[a] = (float)sh.x[a];
        __syncthreads();
        if (tid == 0) {
            d.finalized[i] = 0;
            d.finishes[i] += steps;
            const int f = ++d.fails[i];
            if (f >= FIN_MAX_FAILS) {
                d.state[i] = ST_DONE;
                d.sstatus[i] = MPL_SIG_UNCERTIFIED;
            } else {
                d.eps[i] = fmaxf(d.eps[i] * 1e-2f, 1e-7f);
                d.state[i] = ST_REFINE;  // one more master problem after its re-entry
                d.reent[cur][atomicAdd(&d.cnt->reent_n[cur], 1)] = i;
            }
        }
    }
    if (C > 1) csync(d, cs);
}

}  // namespace

cudaError_t prepare_finish() {
    static bool attr = false;
    if (attr) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_finish<FIN_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)FIN_SMEM_MAX);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_finish<FIN_THREADS_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)FIN_SMEM_MAX);
    if (e == cudaSuccess) attr = true;
    return e;
}

cudaError_t launch_finish(const Dev& d, int cur, int ub, int est, int scap, cudaStream_t s, int64_t* nl, int sms) {
    if (ub <= 0) return cudaSuccess;
    scap = ((scap + 31) / 32) * 32;
    if (scap > d.smax) scap = d.smax;
    // shared-memory factor area: the whole bound while two CTAs still fit on an SM
    auto dyn_of = [&](int mf, int rs) {
        return 4 * (size_t)scap * sizeof(double) +
               (2 * (size_t)scap + (mf ? (size_t)mf * ((mf + 1) | 1) : (size_t)fac_stage_floats(scap))) * sizeof(float) +
               4 * (size_t)scap * sizeof(int) + (rs ? 2 * (size_t)d.n * sizeof(float) + 16 : 0);
    };
    const int rsm = d.n <= 4096 ? 1 : 0;
    // (one CTA per SM with a larger area loses more to the halved concurrency than the
    // shared-memory factor gains, so the area is the bound or nothing)
    const int msm = dyn_of(scap, rsm) <= FIN_SMEM_TWO_CTAS ? scap : 0;
    const size_t dyn = dyn_of(msm, rsm);
    cudaError_t ep = prepare_finish();
    if (ep != cudaSuccess) return ep;
    // a cluster per signal when the finishing signals leave most SMs idle: about est of them
    // (at most ub), clusters of C so that C est stays within two CTAs per SM (four per SM
    // measured slower: the clusters then crowd out the concurrent iteration) and every CTA of
    // the grid has a workspace slot; the row-block exchange needs the residual pair in shared
    // memory and float4 rows, and signals of at least FIN_CLUSTER_MIN_N entries (shorter
    // sweeps gain less than the cluster barriers cost).  (The solve passes the exact count
    // as both.)  Builds with -DMPL_NO_FIN_CLUSTER keep one CTA per signal.
    int C = 1;
#if !defined(MPL_NO_FIN_CLUSTER)
    if (rsm && (d.n & 3) == 0 && d.n >= FIN_CLUSTER_MIN_N && sms > 0 && d.fin_pool)
        while (C < FIN_CLUSTER_MAX && 2 * C * est <= 2 * sms && 2 * C * ub <= d.fin_slots) C *= 2;
#endif
    const bool wide = dyn > FIN_SMEM_TWO_CTAS;
    cudaLaunchConfig_t c{};
    c.gridDim = dim3((unsigned)(ub * C));
    c.blockDim = dim3(wide ? FIN_THREADS_WIDE : FIN_THREADS);
    c.dynamicSmemBytes = dyn;
    c.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    c.attrs = at;
    c.numAttrs = C > 1 ? 1 : 0;
    const cudaError_t e = wide ? cudaLaunchKernelEx(&c, k_finish<FIN_THREADS_WIDE>, d, cur, scap, msm, rsm, C)
                               : cudaLaunchKernelEx(&c, k_finish<FIN_THREADS>, d, cur, scap, msm, rsm, C);
    if (e != cudaSuccess) return e;
    ++*nl;
    return cudaGetLastError();
}

}  // namespace mpl

#ifdef MPL_FIN_TRACE
extern "C" int mpl_debug_fin_trace(long long* out, int count, int reset) {
    if (count > 8192) count = 8192;
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    if (cudaMemcpyFromSymbol(out, mpl::g_fin_trace, sizeof(long long) * 20 * (size_t)count) != cudaSuccess) return -1;
    if (reset) {
        static long long zero[8192][20];
        if (cudaMemcpyToSymbol(mpl::g_fin_trace, zero, sizeof(zero)) != cudaSuccess) return -1;
    }
    return count;
}
#endif
