// Master problem (eq. "primal_MPL") and residual update of Algorithm 1,
// batched over signals, plus solve set-up and output.
//
//   k_init      x^0 = 0, xi^0 = b, I_0 = {} (the initialisation of Alg. 1)
//   k_gram      new rows of the Gram block G_S = A_S^T A_S and h_S = A_S^T b
//               for the atoms appended this iteration (the explicit copies of
//               A_I that Sec. 2.4 recommends become Gram rows here)
//   k_apg       accelerated proximal gradient on
//                   min_u lambda*||u||_1 + 0.5 u^T G u - h^T u
//               warm started from x_S (Alg. 1), stopped by eq. (inner)
//               or s_max; persistent CTAs pull signals from a device queue
//   k_residual  xi = b - A_S x_S (the residual update of Alg. 1), FP32 (+ BF16 copy)
//   k_scatter   dense X from the active sets
//   k_smpl_prune  Algorithm 2's pruning of the explored atoms back to rho
// (the Gram growth read out of Q instead of k_gram is in corr_q.cu.)  The chain's
// kernels start with pdl_enter (programmatic dependent launch).
#include "mpl_internal.cuh"

namespace mpl {

#ifdef MPL_APG_TRACE
// Per-signal phase cycle counters of the master problem (diagnostic builds only):
// [Gram block + vectors, power iteration, FISTA, write-back, master problems, FISTA iterations]
__device__ long long g_apg_trace[8192][8];
#define AT_BEGIN long long at0_ = clock64();
#define AT_ADD(slot) do { if (threadIdx.x == 0 && i < 8192) g_apg_trace[i][slot] += clock64() - at0_; at0_ = clock64(); } while (0)
#define AT_CNT(slot, v) do { if (threadIdx.x == 0 && i < 8192) g_apg_trace[i][slot] += (v); } while (0)
#else
#define AT_BEGIN
#define AT_ADD(slot) do {} while (0)
#define AT_CNT(slot, v) do {} while (0)
#endif

namespace {

__device__ __forceinline__ float block_sum(float v, float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float t = 0.f;
    for (int w = 0; w < nw; ++w) t += red[w];  // same order in every thread
    return t;
}

// block_sum without its leading barrier, for callers where a barrier already separates
// the previous readers of red from these writes.
__device__ __forceinline__ float block_sum_after_barrier(float v, float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float t = 0.f;
    for (int w = 0; w < nw; ++w) t += red[w];  // same order in every thread
    return t;
}

__device__ __forceinline__ double block_sum_d(double v, double* red) {
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

__device__ __forceinline__ float softf(float v, float t) {
    return v > t ? v - t : (v < -t ? v + t : 0.f);
}

// ------------------------------------------------------------------ init
__global__ void __launch_bounds__(256) k_init(Dev d) {
    pdl_enter();
    const int i = blockIdx.x;
    if (i >= d.p) return;
    __shared__ double red[32];
    const int n = d.n;
    const float* b = d.B + (size_t)i * n;
    float* r32 = d.R32 + (size_t)i * n;
    double* r64 = d.R64 + (size_t)i * n;
    double ss = 0.0, es = 0.0, ts = 0.0;
    int nf = 0;
    // entries k = tid + j nt in order of j; four loads in flight before their stores
    for (int k0 = threadIdx.x; k0 < n; k0 += 4 * blockDim.x) {
        float bv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = k0 + u * blockDim.x;
            bv[u] = k < n ? b[k] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = k0 + u * blockDim.x;
            if (k >= n) break;
            const float v = bv[u];
            if (!isfinite(v)) nf = 1;
            r32[k] = v;
            d.R32lo[(size_t)i * n + k] = 0.f;
            r64[k] = (double)v;
            const __nv_bfloat16 q = __float2bfloat16_rn(v);
            if (d.R16) d.R16[(size_t)i * n + k] = q;
            if (d.pos) d.R16c[(size_t)i * n + k] = q;  // active list = identity
            ss += (double)v * (double)v;
            const double fq = (double)__bfloat162float(q), e = (double)v - fq;
            es += e * e;
            ts += fq * fq;
        }
    }
    uint32_t* mw = d.mask + (size_t)i * d.mw;
    for (int w = threadIdx.x; w < d.mw; w += blockDim.x) mw[w] = 0u;
    nf = __syncthreads_or(nf);
    const double bb = block_sum_d(ss, red);
    const double ee = block_sum_d(es, red);
    const double tt = block_sum_d(ts, red);
    if (threadIdx.x == 0) {
        d.r16e[i] = __double2float_ru(sqrt(ee) * (1.0 + 1e-6));
        d.r16t[i] = __double2float_ru(sqrt(tt) * (1.0 + 1e-6));
    }
    if (threadIdx.x == 0) {
        const float lam = d.lam[i];
        const bool bad = nf || !(lam >= 0.f) || !isfinite(lam);  // lambda = 0: least squares
        d.state[i] = bad ? ST_DONE : ST_GROW;
        d.sstatus[i] = bad ? MPL_SIG_NONFINITE : MPL_SIG_MAX_OUTER;
        d.ssize[i] = 0;
        d.snew[i] = 0;
        d.finalized[i] = 1;  // x = 0 and xi = b are exact
        d.outer[i] = 0;
        d.inner[i] = 0;
        d.finishes[i] = 0;
        d.fails[i] = 0;
        d.nnz[i] = 0;
        d.res_tick[i] = 0;  // (a solve that stopped on an error may have left a count)
        d.rnorm[i] = __double2float_ru(sqrt(bb)) * (1.f + 1e-6f);
        if (d.pos) d.pos[i] = i;
        if (d.bnorm) { d.bnorm[i] = d.rnorm[i]; d.xl1[i] = 0.f; }
        if (d.explore) d.explore[i] = 0;
        if (i == 0 && d.ovf_cnt) { d.ovf_cnt->act_n[0] = 0; d.ovf_cnt->act_n[1] = 0; }
        if (d.early) { d.early[i] = 0; d.f0[i] = (float)(0.5 * bb); }
        d.eps[i] = d.eps_in;
        d.obj[i] = 0.5 * bb;
        d.rr[i] = bb;
        d.rb[i] = bb;
        d.kkt_in[i] = 0.0;
        d.kkt_out[i] = 0.0;
        d.ginf[i] = 0.0;
        d.act[0][i] = i;
        if (i == 0) {
            d.cnt->act_n[0] = d.p;
            d.cnt->act_n[1] = 0;
            d.cnt->grow_n = d.cnt->fin_n = d.cnt->apg_n = d.cnt->apg_head = d.cnt->apg_head2 = 0;
            d.cnt->err = 0;
            d.cnt->sel_fallback = 0;
            d.cnt->cols = 0ull;
            d.cnt->fin_flops = 0ull;
            d.cnt->qcols = 0ull;
            d.cnt->sel_done = 0;
            d.cnt->bounds_site = 0;
            d.cnt->apg_elems = d.cnt->apg_gl_elems = 0ull;
            for (int q = 0; q < FIN_SLOTS; ++q) d.cnt->fin_par[q] = d.cnt->reent_n[q] = 0;
            d.cnt->fslot = 0;
            d.cnt->mslots = 0;
            d.cnt->res_bytes = d.cnt->gram_bytes = d.cnt->fin_bytes = 0ull;
        }
    }
}

// ------------------------------------------------------------------ gram
// G[a][b] for a in [0, s), b in [s0, s) (mirrored), tile 64 (a) x 32 (b).
constexpr int GBM = 64, GBN = 32, GBK = 32;

template <bool VEC>
__device__ __forceinline__ float4 gram_load(const float* row, int k, int n) {
    if (row == nullptr || k >= n) return make_float4(0.f, 0.f, 0.f, 0.f);
    if (VEC) return __ldg(reinterpret_cast<const float4*>(row + k));
    float t[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) t[e] = (k + e < n) ? __ldg(row + k + e) : 0.f;
    return make_float4(t[0], t[1], t[2], t[3]);
}

template <bool VEC>
__global__ void __launch_bounds__(256) k_gram(Dev d) {
    pdl_enter();
    const int g = blockIdx.x;
    if (g >= d.cnt->grow_n) return;
    const int i = d.list_grow[g];
    const int s = d.ssize[i], q = d.snew[i], s0 = s - q;
    const int a0 = blockIdx.y * GBM;
    if (a0 >= s || q == 0) return;  // q == 0: a refine pass, the block is complete
    const int n = d.n, smax = d.smax;
    const int* Si = d.S + (size_t)i * smax;
    float* Gi = d.G + (size_t)i * smax * smax;
    // two K-slices: the next slice's loads are in flight while this one is used
    __shared__ __align__(16) float As[2][GBK][GBM + 4];
    __shared__ __align__(16) float Bs[2][GBK][GBN + 4];
    const int tid = threadIdx.x;
    const int ty = tid >> 3, tx = tid & 7;
    const int lr = tid >> 3, lk = (tid & 7) * 4;

    // columns 0..q-1 are the new atoms (their h = a^T b comes with the selection's re-score)
    for (int b0 = 0; b0 < q; b0 += GBN) {
        float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        const int ra0 = a0 + lr, ra1 = a0 + lr + 32;
        const float* pa0 = (ra0 < s) ? d.A32 + (size_t)Si[ra0] * n : nullptr;
        const float* pa1 = (ra1 < s) ? d.A32 + (size_t)Si[ra1] * n : nullptr;
        const int rb = b0 + lr;
        const float* pb = (rb < q) ? d.A32 + (size_t)Si[s0 + rb] * n : nullptr;
        float4 v0 = gram_load<VEC>(pa0, lk, n), v1 = gram_load<VEC>(pa1, lk, n), vb = gram_load<VEC>(pb, lk, n);
        const int nsl = (n + GBK - 1) / GBK;
        for (int sl = 0; sl < nsl; ++sl) {
            const int buf = sl & 1;
            As[buf][lk + 0][lr] = v0.x; As[buf][lk + 1][lr] = v0.y; As[buf][lk + 2][lr] = v0.z; As[buf][lk + 3][lr] = v0.w;
            As[buf][lk + 0][lr + 32] = v1.x; As[buf][lk + 1][lr + 32] = v1.y;
            As[buf][lk + 2][lr + 32] = v1.z; As[buf][lk + 3][lr + 32] = v1.w;
            Bs[buf][lk + 0][lr] = vb.x; Bs[buf][lk + 1][lr] = vb.y; Bs[buf][lk + 2][lr] = vb.z; Bs[buf][lk + 3][lr] = vb.w;
            __syncthreads();
            if (sl + 1 < nsl) {
                const int kk = (sl + 1) * GBK + lk;
                v0 = gram_load<VEC>(pa0, kk, n);
                v1 = gram_load<VEC>(pa1, kk, n);
                vb = gram_load<VEC>(pb, kk, n);
            }
#pragma unroll 8
            for (int k = 0; k < GBK; ++k) {
                const float x0 = As[buf][k][ty * 2], x1 = As[buf][k][ty * 2 + 1];
                const float4 y = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
                acc[0][0] = fmaf(x0, y.x, acc[0][0]); acc[0][1] = fmaf(x0, y.y, acc[0][1]);
                acc[0][2] = fmaf(x0, y.z, acc[0][2]); acc[0][3] = fmaf(x0, y.w, acc[0][3]);
                acc[1][0] = fmaf(x1, y.x, acc[1][0]); acc[1][1] = fmaf(x1, y.y, acc[1][1]);
                acc[1][2] = fmaf(x1, y.z, acc[1][2]); acc[1][3] = fmaf(x1, y.w, acc[1][3]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int a = a0 + ty * 2 + u;
            if (a >= s) continue;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int bb = b0 + tx * 4 + v;
                if (bb >= q) continue;
                const int col = s0 + bb;
                Gi[(size_t)a * smax + col] = acc[u][v];
                Gi[(size_t)col * smax + a] = acc[u][v];
            }
        }
    }
}

// Same per-output summation order (k ascending, one FMA chain) as k_gram, with
// the K slices staged by cp.async in a GS-deep ring so that GS - 1 slices are in
// flight while one is consumed.  Tile BM rows (atoms of S) x BN columns (new
// atoms); each thread computes TR rows x TC columns.  The host takes the
// narrow 32 x 16 tile when at most 16 atoms arrive per signal (the columns of a
// wider tile would mostly be empty).  Needs n % 4 == 0 (16-byte rows).
constexpr int GS = 4, GPAD = GBK + 4;

__device__ __forceinline__ void cp_async16(float* dst, const float* src, int bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int BM, int BN, int TR, int TC>
__global__ void __launch_bounds__(256) k_gram_async(Dev d) {
    pdl_enter();
    static_assert((BM / TR) * (BN / TC) == 256, "one output block per thread");
    constexpr int NX = BN / TC;                  // threads along the columns
    constexpr int CHUNKS = (BM + BN) * (GBK / 4);  // 16-byte chunks per slice
    const int g = blockIdx.x;
    if (g >= d.cnt->grow_n) return;
    const int i = d.list_grow[g];
    const int s = d.ssize[i], q = d.snew[i], s0 = s - q;
    const int a0 = blockIdx.y * BM;
    if (a0 >= s || q == 0) return;
    const int n = d.n, smax = d.smax;
    if (blockIdx.y == 0 && threadIdx.x == 0)  // s atom columns read, 2 s q of G written
        atomicAdd(&d.cnt->gram_bytes, 4ull * n * s + 8ull * s * q);
    const int* Si = d.S + (size_t)i * smax;
    float* Gi = d.G + (size_t)i * smax * smax;
    extern __shared__ __align__(16) float gsm[];
    float* As = gsm;                            // [GS][BM][GPAD]
    float* Bs = gsm + (size_t)GS * BM * GPAD;   // [GS][BN][GPAD]
    const int tid = threadIdx.x;
    const int ty = tid / NX, tx = tid % NX;
    const int nsl = (n + GBK - 1) / GBK;
    for (int b0 = 0; b0 < q; b0 += BN) {
        // source rows of this thread's chunks (c = tid + 256 e), fixed for the column chunk
        constexpr int PER = (CHUNKS + 255) / 256;
        const float* src[PER];
        float* dst0[PER];
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const int c = tid + 256 * e;
            const int rr = c / (GBK / 4), kc = (c % (GBK / 4)) * 4;
            const float* p = nullptr;
            if (c < CHUNKS) {
                if (rr < BM) {
                    const int ra = a0 + rr;
                    p = ra < s ? d.A32 + (size_t)Si[ra] * n : nullptr;
                } else {
                    const int rb = b0 + rr - BM;
                    p = rb < q ? d.A32 + (size_t)Si[s0 + rb] * n : nullptr;
                }
            }
            src[e] = p;
            dst0[e] = c >= CHUNKS ? nullptr : (rr < BM ? As + (size_t)rr * GPAD + kc : Bs + (size_t)(rr - BM) * GPAD + kc);
        }
        auto issue = [&](int sl) {
            const int st = sl % GS;
#pragma unroll
            for (int e = 0; e < PER; ++e) {
                if (dst0[e] == nullptr) continue;
                const int c = tid + 256 * e;
                const int rr = c / (GBK / 4), kc = (c % (GBK / 4)) * 4, k = sl * GBK + kc;
                float* dst = dst0[e] + (size_t)st * (rr < BM ? BM : BN) * GPAD;
                const bool ok = src[e] != nullptr && k < n;
                cp_async16(dst, ok ? src[e] + k : d.A32, ok ? 16 : 0);
            }
        };
#pragma unroll
        for (int sl = 0; sl < GS - 1; ++sl) {
            if (sl < nsl) issue(sl);
            cp_async_commit();
        }
        float acc[TR][TC];
#pragma unroll
        for (int u = 0; u < TR; ++u)
#pragma unroll
            for (int v = 0; v < TC; ++v) acc[u][v] = 0.f;
        for (int sl = 0; sl < nsl; ++sl) {
            cp_async_wait<GS - 2>();
            __syncthreads();
            if (sl + GS - 1 < nsl) issue(sl + GS - 1);
            cp_async_commit();
            const int st = sl % GS;
            const float* Ar = As + ((size_t)st * BM + ty * TR) * GPAD;
            const float* Bt = Bs + ((size_t)st * BN + tx) * GPAD;
#pragma unroll
            for (int k = 0; k < GBK; k += 4) {
                float4 x[TR];
#pragma unroll
                for (int u = 0; u < TR; ++u) x[u] = *reinterpret_cast<const float4*>(Ar + (size_t)u * GPAD + k);
#pragma unroll
                for (int v = 0; v < TC; ++v) {
                    const float4 y = *reinterpret_cast<const float4*>(Bt + (size_t)v * NX * GPAD + k);
#pragma unroll
                    for (int u = 0; u < TR; ++u) {
                        acc[u][v] = fmaf(x[u].x, y.x, acc[u][v]);
                        acc[u][v] = fmaf(x[u].y, y.y, acc[u][v]);
                        acc[u][v] = fmaf(x[u].z, y.z, acc[u][v]);
                        acc[u][v] = fmaf(x[u].w, y.w, acc[u][v]);
                    }
                }
            }
        }
        cp_async_wait<0>();
        __syncthreads();  // the ring is reused by the next column chunk
#pragma unroll
        for (int u = 0; u < TR; ++u) {
            const int a = a0 + ty * TR + u;
            if (a >= s) continue;
#pragma unroll
            for (int v = 0; v < TC; ++v) {
                const int bb = b0 + tx + NX * v;
                if (bb >= q) continue;
                const int col = s0 + bb;
                Gi[(size_t)a * smax + col] = acc[u][v];
                Gi[(size_t)col * smax + a] = acc[u][v];
            }
        }
    }
}

template <int BM, int BN>
constexpr size_t gram_smem() { return (size_t)GS * (BM + BN) * GPAD * sizeof(float); }

// ------------------------------------------------------------------ APG
// Gram block in shared memory when s <= gcap (<= APG_SMEM_S), else read from
// global memory (L2).  Dynamic shared memory: [G gcap^2 | 6 vectors of vcap].
// y = G x with TPR threads per row (s <= 256 / TPR): lane = row slot + (256 / TPR / 8)
// ... the TPR threads of a row sit 32 / TPR lanes apart and take every TPR-th
// column; their partial sums meet in a fixed butterfly.  With the packed leading
// dimension ld = 32 / TPR (mod 32) the TPR column phases fall in disjoint banks.
// With h != nullptr the thread that writes y_r also returns its share of the
// restricted objective, lambda |x_r| + x_r (y_r / 2 - h_r) (summed over its rows).
template <int TPR>
__device__ __forceinline__ float gram_mv_split(const float* __restrict__ G, int ld, int s, const float* __restrict__ x,
                                               float* __restrict__ y, const float* h = nullptr, float lam = 0.f) {
    constexpr int RW = 32 / TPR;  // rows per warp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = lane / RW, r = warp * RW + (lane % RW);
    float a = 0.f;
    if (r < s)
        for (int c = p; c < s; c += TPR) a = fmaf(G[(size_t)c * ld + r], x[c], a);
#pragma unroll
    for (int o = RW; o < 32; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    float part = 0.f;
    if (p == 0 && r < s) {
        y[r] = a;
        if (h) part = lam * fabsf(x[r]) + x[r] * (0.5f * a - h[r]);
    }
    return part;
}

// Packed leading dimension of an s x s block for gram_mv_split (see above).
__host__ __device__ __forceinline__ int apg_ld(int s) {
    if (s <= 64) return s + ((8 - s) & 31);    // = 8 (mod 32), TPR 4
    if (s <= 128) return s + ((16 - s) & 31);  // = 16 (mod 32), TPR 2
    return s;
}

// Floats reserved for a packed block of up to gcap atoms (padded rows included).
__host__ __device__ __forceinline__ size_t apg_area(int gcap) {
    const size_t g = (size_t)gcap, h = (size_t)(gcap < 128 ? gcap : 128);
    return g * g > h * (h + 32) ? g * g : h * (h + 32);
}

__device__ __forceinline__ float gram_mv(const float* __restrict__ G, int ld, int s, const float* __restrict__ x,
                                         float* __restrict__ y, const float* h = nullptr, float lam = 0.f) {
    float part = 0.f;
    // y = G x, one row per thread; G symmetric so column r is read with unit
    // stride across threads (conflict-free in shared memory, coalesced in global)
    for (int r = threadIdx.x; r < s; r += blockDim.x) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int c = 0;
        for (; c + 3 < s; c += 4) {
            a0 = fmaf(G[(size_t)(c + 0) * ld + r], x[c + 0], a0);
            a1 = fmaf(G[(size_t)(c + 1) * ld + r], x[c + 1], a1);
            a2 = fmaf(G[(size_t)(c + 2) * ld + r], x[c + 2], a2);
            a3 = fmaf(G[(size_t)(c + 3) * ld + r], x[c + 3], a3);
        }
        for (; c < s; ++c) a0 = fmaf(G[(size_t)c * ld + r], x[c], a0);
        const float yr = (a0 + a1) + (a2 + a3);
        y[r] = yr;
        if (h) part += lam * fabsf(x[r]) + x[r] * (0.5f * yr - h[r]);
    }
    return part;
}

// y = G x for a block in global memory (leading dimension ld, row r = column r by
// symmetry).  Lane l of a warp owns the float4 slices c = 4 l + 128 u (u < U = ceil(s / 128))
// of a row and sums them in order of u, then a fixed butterfly combines the lanes; a warp
// takes RW rows per round and issues all RW x U slice loads before the first product (up to
// 16 per lane in flight: the streamed products are latency-bound).  x is zero from s up to
// the next multiple of 4.  With h != nullptr lane 0 also returns its rows' share of the
// restricted objective, lambda |x_r| + x_r (y_r / 2 - h_r).
template <int U, int RW>
__device__ __forceinline__ float gram_mv_stream_vec(const float* __restrict__ G, int ld, int s,
                                                    const float* __restrict__ x, float* __restrict__ y,
                                                    const float* h, float lam) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float part = 0.f;
    for (int r = RW * warp; r < s; r += RW * nw) {
        float4 g[RW][U];
#pragma unroll
        for (int w = 0; w < RW; ++w) {
            const float* gr = G + (size_t)min(r + w, s - 1) * ld;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int c = 4 * lane + 128 * u;
                g[w][u] = c < s ? __ldg(reinterpret_cast<const float4*>(gr + c)) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        float acc[RW];
#pragma unroll
        for (int w = 0; w < RW; ++w) acc[w] = 0.f;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = 4 * lane + 128 * u;
            if (c < s) {
                const float4 xv = *reinterpret_cast<const float4*>(x + c);
#pragma unroll
                for (int w = 0; w < RW; ++w) {
                    acc[w] = fmaf(g[w][u].x, xv.x, acc[w]); acc[w] = fmaf(g[w][u].y, xv.y, acc[w]);
                    acc[w] = fmaf(g[w][u].z, xv.z, acc[w]); acc[w] = fmaf(g[w][u].w, xv.w, acc[w]);
                }
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
#pragma unroll
            for (int w = 0; w < RW; ++w) acc[w] += __shfl_xor_sync(0xffffffffu, acc[w], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int w = 0; w < RW; ++w) {
                if (r + w < s) {
                    y[r + w] = acc[w];
                    if (h) part += lam * fabsf(x[r + w]) + x[r + w] * (0.5f * acc[w] - h[r + w]);
                }
            }
        }
    }
    return part;
}

// The same product with scalar loads (ld not a multiple of 4): a warp per pair of rows.
__device__ __forceinline__ float gram_mv_stream_scalar(const float* __restrict__ G, int ld, int s,
                                                       const float* __restrict__ x, float* __restrict__ y,
                                                       const float* h, float lam) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float part = 0.f;
    for (int r = 2 * warp; r < s; r += 2 * nw) {
        const int rb = r + 1 < s ? r + 1 : r;
        const float* ga = G + (size_t)r * ld;
        const float* gb = G + (size_t)rb * ld;
        float sa = 0.f, sb = 0.f;
        for (int c0 = 4 * lane; c0 < s; c0 += 512) {
            float4 a4[4], b4[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = c0 + 128 * u;
                if (c < s) {
                    a4[u] = make_float4(__ldg(ga + c), c + 1 < s ? __ldg(ga + c + 1) : 0.f,
                                        c + 2 < s ? __ldg(ga + c + 2) : 0.f, c + 3 < s ? __ldg(ga + c + 3) : 0.f);
                    b4[u] = make_float4(__ldg(gb + c), c + 1 < s ? __ldg(gb + c + 1) : 0.f,
                                        c + 2 < s ? __ldg(gb + c + 2) : 0.f, c + 3 < s ? __ldg(gb + c + 3) : 0.f);
                } else {
                    a4[u] = b4[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = c0 + 128 * u;
                if (c < s) {
                    const float4 xv = *reinterpret_cast<const float4*>(x + c);
                    sa = fmaf(a4[u].x, xv.x, sa); sa = fmaf(a4[u].y, xv.y, sa);
                    sa = fmaf(a4[u].z, xv.z, sa); sa = fmaf(a4[u].w, xv.w, sa);
                    sb = fmaf(b4[u].x, xv.x, sb); sb = fmaf(b4[u].y, xv.y, sb);
                    sb = fmaf(b4[u].z, xv.z, sb); sb = fmaf(b4[u].w, xv.w, sb);
                }
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
            sb += __shfl_xor_sync(0xffffffffu, sb, o);
        }
        if (lane == 0) {
            y[r] = sa;
            if (h) part += lam * fabsf(x[r]) + x[r] * (0.5f * sa - h[r]);
            if (r + 1 < s) {
                y[r + 1] = sb;
                if (h) part += lam * fabsf(x[r + 1]) + x[r + 1] * (0.5f * sb - h[r + 1]);
            }
        }
    }
    return part;
}

__device__ __noinline__ float gram_mv_stream(const float* __restrict__ G, int ld, int s, const float* __restrict__ x,
                                             float* __restrict__ y, const float* h = nullptr, float lam = 0.f) {
    if ((ld & 3) != 0) return gram_mv_stream_scalar(G, ld, s, x, y, h, lam);
    switch ((s + 127) >> 7) {
        case 0:
        case 1: return gram_mv_stream_vec<1, 8>(G, ld, s, x, y, h, lam);
        case 2: return gram_mv_stream_vec<2, 8>(G, ld, s, x, y, h, lam);
        case 3: return gram_mv_stream_vec<3, 4>(G, ld, s, x, y, h, lam);
        case 4: return gram_mv_stream_vec<4, 4>(G, ld, s, x, y, h, lam);
        case 5: return gram_mv_stream_vec<5, 2>(G, ld, s, x, y, h, lam);
        case 6: return gram_mv_stream_vec<6, 2>(G, ld, s, x, y, h, lam);
        case 7: return gram_mv_stream_vec<7, 2>(G, ld, s, x, y, h, lam);
        default: return gram_mv_stream_vec<8, 2>(G, ld, s, x, y, h, lam);
    }
}

struct ApgVec {
    float *u, *up, *Gu, *Gup, *h, *v;
    float red[96];
    int item;
};

// Three block sums in one pass (two barriers); every thread gets the totals.
__device__ __forceinline__ void block_sum3(float& a, float& b, float& c, float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    __syncthreads();
    if (lane == 0) { red[warp] = a; red[32 + warp] = b; red[64 + warp] = c; }
    __syncthreads();
    a = b = c = 0.f;
    for (int w = 0; w < nw; ++w) { a += red[w]; b += red[32 + w]; c += red[64 + w]; }
}

// STREAM: the APG_GLOBAL launch (every block streamed from global memory by warp rows);
// otherwise blocks in shared memory (or, past gcap, read by the thread-per-row product).
template <bool STREAM>
__global__ void __launch_bounds__(APG_THREADS) k_apg(Dev d, int vcap, int gcap, int cls) {
    pdl_enter();
    extern __shared__ __align__(16) float gsm[];
    __shared__ ApgVec sh;
    const int tid = threadIdx.x;
    const int smax = d.smax;
    if (tid == 0) {
        float* base = gsm + apg_area(gcap);
        sh.u = base; sh.up = base + vcap; sh.Gu = base + 2 * vcap;
        sh.Gup = base + 3 * vcap; sh.h = base + 4 * vcap; sh.v = base + 5 * vcap;
    }
    int* head = cls == APG_GLOBAL ? &d.cnt->apg_head2 : &d.cnt->apg_head;
    for (;;) {
        if (tid == 0) sh.item = atomicAdd(head, 1);
        __syncthreads();
        const int it = sh.item;
        if (it >= d.cnt->apg_n) break;
        const int i = d.list_apg[it];
        const int s = d.ssize[i];
        // a class launch takes only its own signals (the other launch takes the rest)
        if ((cls == APG_SMEM && s > gcap) || (cls == APG_GLOBAL && s <= APG_SMEM_S)) {
            __syncthreads();  // every thread has read sh.item before thread 0 takes the next
            continue;
        }
        AT_BEGIN
        const float lam = d.lam[i];
        const float eps = d.eps[i];
        const float* Gg = d.G + (size_t)i * smax * smax;
        if (s > vcap) {  // cannot happen with a correct bound; refuse rather than overrun
            if (tid == 0) atomicCAS(&d.cnt->err, 0, (int)DERR_SHAPE);
            __syncthreads();
            continue;
        }
        const bool insm = s <= gcap;
        const float* G = insm ? gsm : Gg;
        const int ld = insm ? apg_ld(s) : smax;
        if (insm) {
            // eight loads in flight per thread before their stores
            for (int e0 = tid; e0 < s * s; e0 += 8 * blockDim.x) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = e0 + u * blockDim.x;
                    if (e < s * s) {
                        const int r = e / s, c = e - r * s;
                        v[u] = __ldg(Gg + (size_t)r * smax + c);
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = e0 + u * blockDim.x;
                    if (e < s * s) {
                        const int r = e / s, c = e - r * s;
                        gsm[(size_t)r * ld + c] = v[u];
                    }
                }
            }
        }
        // the block's matrix-vector product: split rows while the block is small, warp rows
        // streamed as float4 slices from global memory when it is not in shared memory
        auto mv = [&](const float* x, float* y) {
            if constexpr (STREAM) {
                gram_mv_stream(G, ld, s, x, y);
            } else {
                if (insm && s <= 64) gram_mv_split<4>(G, ld, s, x, y);
                else if (insm && s <= 128) gram_mv_split<2>(G, ld, s, x, y);
                else gram_mv(G, ld, s, x, y);
            }
        };
        // y = G x and this thread's share of the restricted objective at x
        auto mvF = [&](const float* x, float* y) -> float {
            if constexpr (STREAM) {
                return gram_mv_stream(G, ld, s, x, y, sh.h, lam);
            } else {
                if (insm && s <= 64) return gram_mv_split<4>(G, ld, s, x, y, sh.h, lam);
                if (insm && s <= 128) return gram_mv_split<2>(G, ld, s, x, y, sh.h, lam);
                return gram_mv(G, ld, s, x, y, sh.h, lam);
            }
        };
        float* xi = d.xS + (size_t)i * smax;
        float* ritz = d.ritz + (size_t)i * smax;
        const int prev = s - d.snew[i];  // ritz vector valid for the first `prev` entries
        // (entries from s up to the next multiple of 4 are zero: the streamed product reads
        // its operand as float4 slices)
        const int s4 = (s + 3) & ~3;
        if (MPL_OOB(s4 > vcap || s > smax, 201)) { __syncthreads(); continue; }
        for (int r = tid; r < s4; r += blockDim.x) {
            const bool in = r < s;
            sh.u[r] = in ? xi[r] : 0.f;
            sh.h[r] = in ? d.h[(size_t)i * smax + r] : 0.f;
            sh.v[r] = !in ? 0.f : ((r < prev && d.outer[i] > 1) ? ritz[r] : 1.f);
            sh.up[r] = 0.f;
            sh.Gu[r] = 0.f;
            sh.Gup[r] = 0.f;
        }
        __syncthreads();
        AT_ADD(0);
        // Step size: power iteration for lambda_max(G) (warm started), L = 1.05 theta.  The
        // iterate ping-pongs between two vectors and is normalised every fourth step (and
        // at the last, where the Rayleigh quotient is taken): growth over four steps stays
        // far inside FP32 range for |S| <= 1024.
        float theta = 1.f;
        const int npow = !(lam > 0.f) ? 0 : ((prev > 0 && d.outer[i] > 1) ? 3 : 8);  // CG needs no step size
        float* pv = sh.v;
        float* pw = sh.Gu;
        for (int pi = 0; pi < npow; ++pi) {
            mv(pv, pw);
            __syncthreads();
            if ((pi & 3) == 3 || pi == npow - 1) {
                float vv = 0.f, vg = 0.f, gg = 0.f;
                for (int r = tid; r < s; r += blockDim.x) {
                    vv += pv[r] * pv[r];
                    vg += pv[r] * pw[r];
                    gg += pw[r] * pw[r];
                }
                block_sum3(vv, vg, gg, sh.red);
                theta = vv > 0.f ? vg / vv : 1.f;
                const float inv = gg > 0.f ? rsqrtf(gg) : 0.f;
                for (int r = tid; r < s; r += blockDim.x) pv[r] = pw[r] * inv;
                __syncthreads();
            } else {
                float* t = pv;
                pv = pw;
                pw = t;
            }
        }
        for (int r = tid; r < s; r += blockDim.x) ritz[r] = pv[r];
        __syncthreads();  // pv may be the Gu buffer, which the next product overwrites
        AT_ADD(1);
        float L = fmaxf(1.05f * theta, 1e-30f);

        // F(u) and G u at the warm start
        mv(sh.u, sh.Gu);
        __syncthreads();
        float part = 0.f;
        for (int r = tid; r < s; r += blockDim.x) {
            sh.up[r] = sh.u[r];
            sh.Gup[r] = sh.Gu[r];
            part += lam * fabsf(sh.u[r]) + sh.u[r] * (0.5f * sh.Gu[r] - sh.h[r]);
        }
        float F = block_sum(part, sh.red);
        const float F0 = F;
        float t = 1.f, beta = 0.f;
        int iters = 0, restarts_in_row = 0;
        if (!(lam > 0.f)) {
            // lambda = 0: the restricted problem is least squares G u = h, solved by
            // conjugate gradients (the paper's CGD rule for lambda = 0) from the warm start;
            // r in up, the direction in Gup, G times the direction in v
            float rr = 0.f, hh = 0.f;
            for (int r = tid; r < s; r += blockDim.x) {
                const float res = sh.h[r] - sh.Gu[r];
                sh.up[r] = res;
                sh.Gup[r] = res;
                rr += res * res;
                hh += sh.h[r] * sh.h[r];
            }
            float z0 = 0.f;
            block_sum3(rr, hh, z0, sh.red);
            const float stop2 = eps * eps * hh;
            const int cg_max = min(d.inner_max, 4 * s + 20);
            for (int k = 0; k < cg_max && rr > stop2; ++k) {
                mv(sh.Gup, sh.v);
                __syncthreads();
                float pgp = 0.f;
                for (int r = tid; r < s; r += blockDim.x) pgp += sh.Gup[r] * sh.v[r];
                pgp = block_sum(pgp, sh.red);
                if (!(pgp > 0.f)) break;
                const float alpha = rr / pgp;
                float rn = 0.f;
                for (int r = tid; r < s; r += blockDim.x) {
                    sh.u[r] += alpha * sh.Gup[r];
                    sh.Gu[r] += alpha * sh.v[r];
                    const float res = sh.up[r] - alpha * sh.v[r];
                    sh.up[r] = res;
                    rn += res * res;
                }
                rn = block_sum(rn, sh.red);
                const float bcg = rn / rr;
                rr = rn;
                for (int r = tid; r < s; r += blockDim.x) sh.Gup[r] = sh.up[r] + bcg * sh.Gup[r];
                __syncthreads();
                ++iters;
            }
            part = 0.f;
            for (int r = tid; r < s; r += blockDim.x) part += sh.u[r] * (0.5f * sh.Gu[r] - sh.h[r]);
            F = block_sum(part, sh.red);
        }
        for (int k = 0; lam > 0.f && k < d.inner_max; ++k) {
            // extrapolate, prox-gradient step (the one matvec is G u of the new point)
            const float invL = 1.f / L, thr = lam * invL;
            for (int r = tid; r < s; r += blockDim.x) {
                const float y = sh.u[r] + beta * (sh.u[r] - sh.up[r]);
                const float gy = sh.Gu[r] + beta * (sh.Gu[r] - sh.Gup[r]) - sh.h[r];
                const float z = softf(y - gy * invL, thr);
                sh.up[r] = sh.u[r];
                sh.Gup[r] = sh.Gu[r];
                sh.u[r] = z;
            }
            __syncthreads();
            part = mvF(sh.u, sh.Gu);  // the block sum's barrier also publishes Gu
            // (the barrier above already follows every read of red by the last block sum)
            const float Fn = block_sum_after_barrier(part, sh.red);
            ++iters;
            if (Fn > F) {
                // function-value restart: back to the previous point, momentum off;
                // a plain step that still increases F means L was too small
                const bool genuine = (Fn - F) > 1e-4f * fmaxf(F0 - F, 1e-30f);
                if (beta == 0.f && genuine) L *= 2.f;
                for (int r = tid; r < s; r += blockDim.x) { sh.u[r] = sh.up[r]; sh.Gu[r] = sh.Gup[r]; }
                __syncthreads();
                beta = 0.f;
                t = 1.f;
                if (++restarts_in_row >= 3) break;  // stalled at FP32 resolution
                continue;
            }
            restarts_in_row = 0;
            const float dec = F - Fn, tot = F0 - Fn;
            F = Fn;
            // relative-decrease stop of eq. (inner)
            if (tot <= 0.f ? dec <= 0.f : dec <= eps * tot) break;
            const float tn = 0.5f * (1.f + sqrtf(1.f + 4.f * t * t));
            beta = (t - 1.f) / tn;
            t = tn;
        }
        AT_ADD(2);
        for (int r = tid; r < s; r += blockDim.x) xi[r] = sh.u[r];
        AT_ADD(3);
        AT_CNT(4, 1);
        AT_CNT(5, iters);
        if (tid == 0) {
            d.inner[i] += iters;
            // products with the block: the power steps, G u at the warm start, one per iteration
            const unsigned long long ss = (unsigned long long)s * (unsigned long long)s;
            const unsigned long long nmv = (unsigned long long)(npow + 1 + iters);
            atomicAdd(&d.cnt->apg_elems, ss * nmv);
            atomicAdd(&d.cnt->apg_gl_elems, insm ? ss : ss * nmv);
            // early stopping, eq. (stop_con): decrease of f over this outer iteration's
            // master problem (F0 is f at x^{t-1}, new entries at zero)
            if (d.early && d.stop_eps >= 0.f && d.snew[i] > 0 &&
                F0 - F <= d.stop_eps * fabsf((float)d.rho * d.f0[i]))
                d.early[i] = 1;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ residual
// Row block y = blockIdx.y of signal position blockIdx.x: rows [RES_ROWS y, RES_ROWS (y + 1)).
// Each entry sums the atoms in order of the support, whatever the split.  The three norms
// are block sums per row block, combined in order of y by the block that finishes last (a
// ticket per signal, no waiting), so they do not depend on the order the blocks run in.
__global__ void __launch_bounds__(256) k_residual(Dev d) {
    pdl_enter();
    const int g = blockIdx.x;
    if (g >= d.cnt->apg_n) return;
    const int i = d.list_apg[g];
    const int yb = blockIdx.y, nb = gridDim.y;
    const int n = d.n, smax = d.smax, s = d.ssize[i];
    __shared__ int nzi[1024];
    __shared__ float nzv[1024];
    __shared__ int cntnz;
    __shared__ float red[96];
    if (threadIdx.x == 0) cntnz = 0;
    __syncthreads();
    const float* xi = d.xS + (size_t)i * smax;
    const int* Si = d.S + (size_t)i * smax;
    // nonzeros of x_S in append order (ordered compaction by one warp)
    if (threadIdx.x < 32) {
        int base = 0;
        for (int a0 = 0; a0 < s; a0 += 32) {
            const int a = a0 + threadIdx.x;
            const float v = a < s ? xi[a] : 0.f;
            const unsigned b = __ballot_sync(0xffffffffu, v != 0.f);
            const int off = base + __popc(b & ((1u << threadIdx.x) - 1u));
            if (v != 0.f) { nzi[off] = Si[a]; nzv[off] = v; }
            base += __popc(b);
        }
        if (threadIdx.x == 0) cntnz = base;
    }
    __syncthreads();
    const int nz = cntnz;
    if (MPL_OOB(s > 1024 || nz > 1024, 301)) return;
    if (d.Q && yb == 0) {  // ||x_S||_1 for the identity route's error band (FP32 sum, rounded up by gamma_1024)
        float l1 = 0.f;
        for (int a = threadIdx.x; a < nz; a += blockDim.x) l1 += fabsf(nzv[a]);
        const float t1 = block_sum(l1, red);
        if (threadIdx.x == 0) d.xl1[i] = t1 * (1.f + 2e-4f);
        __syncthreads();
    }
    const float* b = d.B + (size_t)i * n;
    float* r32 = d.R32 + (size_t)i * n;
    float ss = 0.f, es = 0.f, ts = 0.f;  // ||r||^2, ||r - bf(r)||^2, ||bf(r)||^2
    const bool r16 = d.R16 || d.pos;
    auto bf_terms = [&](float v) {
        const float fq = __bfloat162float(__float2bfloat16_rn(v));
        const float e = v - fq;  // exact (Sterbenz)
        es = fmaf(e, e, es);
        ts = fmaf(fq, fq, ts);
    };
    const int k_lo = yb * RES_ROWS, k_hi = min(n, k_lo + RES_ROWS);
    if ((n & 3) == 0) {
        // float4 columns, four atoms per pass with their loads issued first
        for (int k = k_lo + threadIdx.x * 4; k < k_hi; k += blockDim.x * 4) {
            float4 acc = *reinterpret_cast<const float4*>(b + k);
            int a = 0;
            for (; a + 7 < nz; a += 8) {  // eight atom columns' loads in flight, then in order
                float4 cv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    cv[u] = __ldg(reinterpret_cast<const float4*>(d.A32 + (size_t)nzi[a + u] * n + k));
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float vu = nzv[a + u];
                    acc.x = fmaf(-vu, cv[u].x, acc.x); acc.y = fmaf(-vu, cv[u].y, acc.y);
                    acc.z = fmaf(-vu, cv[u].z, acc.z); acc.w = fmaf(-vu, cv[u].w, acc.w);
                }
            }
            for (; a + 3 < nz; a += 4) {
                const float4 c0 = __ldg(reinterpret_cast<const float4*>(d.A32 + (size_t)nzi[a] * n + k));
                const float4 c1 = __ldg(reinterpret_cast<const float4*>(d.A32 + (size_t)nzi[a + 1] * n + k));
                const float4 c2 = __ldg(reinterpret_cast<const float4*>(d.A32 + (size_t)nzi[a + 2] * n + k));
                const float4 c3 = __ldg(reinterpret_cast<const float4*>(d.A32 + (size_t)nzi[a + 3] * n + k));
                const float v0 = nzv[a], v1 = nzv[a + 1], v2 = nzv[a + 2], v3 = nzv[a + 3];
                acc.x = fmaf(-v0, c0.x, acc.x); acc.y = fmaf(-v0, c0.y, acc.y);
                acc.z = fmaf(-v0, c0.z, acc.z); acc.w = fmaf(-v0, c0.w, acc.w);
                acc.x = fmaf(-v1, c1.x, acc.x); acc.y = fmaf(-v1, c1.y, acc.y);
                acc.z = fmaf(-v1, c1.z, acc.z); acc.w = fmaf(-v1, c1.w, acc.w);
                acc.x = fmaf(-v2, c2.x, acc.x); acc.y = fmaf(-v2, c2.y, acc.y);
                acc.z = fmaf(-v2, c2.z, acc.z); acc.w = fmaf(-v2, c2.w, acc.w);
                acc.x = fmaf(-v3, c3.x, acc.x); acc.y = fmaf(-v3, c3.y, acc.y);
                acc.z = fmaf(-v3, c3.z, acc.z); acc.w = fmaf(-v3, c3.w, acc.w);
            }
            for (; a < nz; ++a) {
                const float4 c0 = __ldg(reinterpret_cast<const float4*>(d.A32 + (size_t)nzi[a] * n + k));
                const float v0 = nzv[a];
                acc.x = fmaf(-v0, c0.x, acc.x); acc.y = fmaf(-v0, c0.y, acc.y);
                acc.z = fmaf(-v0, c0.z, acc.z); acc.w = fmaf(-v0, c0.w, acc.w);
            }
            *reinterpret_cast<float4*>(r32 + k) = acc;
            if (d.R16) {
                __nv_bfloat16* o = d.R16 + (size_t)i * n + k;
                o[0] = __float2bfloat16_rn(acc.x); o[1] = __float2bfloat16_rn(acc.y);
                o[2] = __float2bfloat16_rn(acc.z); o[3] = __float2bfloat16_rn(acc.w);
            }
            if (d.pos) {  // straight into the GEMM's compacted rows for the next iteration
                __nv_bfloat16* o = d.R16c + (size_t)d.pos[i] * n + k;
                o[0] = __float2bfloat16_rn(acc.x); o[1] = __float2bfloat16_rn(acc.y);
                o[2] = __float2bfloat16_rn(acc.z); o[3] = __float2bfloat16_rn(acc.w);
            }
            ss = fmaf(acc.x, acc.x, ss); ss = fmaf(acc.y, acc.y, ss);
            ss = fmaf(acc.z, acc.z, ss); ss = fmaf(acc.w, acc.w, ss);
            if (r16) { bf_terms(acc.x); bf_terms(acc.y); bf_terms(acc.z); bf_terms(acc.w); }
        }
    } else {
        for (int k = k_lo + threadIdx.x; k < k_hi; k += blockDim.x) {
            float acc = b[k];
            for (int a = 0; a < nz; ++a) acc = fmaf(-nzv[a], __ldg(d.A32 + (size_t)nzi[a] * n + k), acc);
            r32[k] = acc;
            if (d.R16) d.R16[(size_t)i * n + k] = __float2bfloat16_rn(acc);
            if (d.pos) d.R16c[(size_t)d.pos[i] * n + k] = __float2bfloat16_rn(acc);
            ss = fmaf(acc, acc, ss);
            if (r16) bf_terms(acc);
        }
    }
    // FP32 sums: a few roundings per term, a 256-way tree and at most 64 row blocks, far
    // inside the 1e-5 margin
    block_sum3(ss, es, ts, red);
    if (threadIdx.x == 0) {
        if (yb == 0) {
            d.nnz[i] = nz;
            // atom columns and b read, the FP32 residual (and its BF16 copies) written
            atomicAdd(&d.cnt->res_bytes, (unsigned long long)n * (4ull * (nz + 2) + (d.R16 ? 2ull : 0ull) +
                                                                  (d.pos ? 2ull : 0ull)));
        }
        bool last = nb == 1;
        if (!last) {
            float* part = d.res_part + ((size_t)i * nb + yb) * 3;
            part[0] = ss; part[1] = es; part[2] = ts;
            __threadfence();
            last = atomicAdd(&d.res_tick[i], 1) == nb - 1;
            if (last) {
                __threadfence();
                const volatile float* all = d.res_part + (size_t)i * nb * 3;
                ss = es = ts = 0.f;
                for (int y = 0; y < nb; ++y) { ss += all[3 * y]; es += all[3 * y + 1]; ts += all[3 * y + 2]; }
                d.res_tick[i] = 0;
            }
        }
        if (last) {
            d.rnorm[i] = sqrtf(ss) * (1.f + 1e-5f);
            d.r16e[i] = sqrtf(es) * (1.f + 1e-5f);
            d.r16t[i] = sqrtf(ts) * (1.f + 1e-5f);
        }
    }
}

// ------------------------------------------------------------------ Algorithm 2
// Subspace exploratory matching: of the q explored atoms (positions s0..s-1,
// appended by this iteration's selection) keep the rho with the largest
// |u| after the master problem, ties to the earlier position; the others
// leave S with their entries.  S, x_S, h, the power-iteration vector and the
// Gram block are compacted with the order of the remaining entries kept; the
// signal's FP64 factor workspace (idle while it grows) stages the Gram block.
__global__ void __launch_bounds__(256) k_smpl_prune(Dev d) {
    pdl_enter();
    const int g = blockIdx.x;
    if (g >= d.cnt->grow_n) return;
    const int i = d.list_grow[g];
    const int q = d.explore[i];
    if (q == 0) return;
    const int smax = d.smax, s = d.ssize[i], s0 = s - q, keep = d.rho;
    __shared__ int from[1024];
    __shared__ int ns_sh;
    int* Si = d.S + (size_t)i * smax;
    float* xi = d.xS + (size_t)i * smax;
    float* hi = d.h + (size_t)i * smax;
    float* ri = d.ritz + (size_t)i * smax;
    float* Gi = d.G + (size_t)i * smax * smax;
    uint32_t* mw = d.mask + (size_t)i * d.mw;
    // rank of each explored atom by |u| (descending, ties to the lower position)
    for (int a = threadIdx.x; a < q; a += blockDim.x) {
        const float ua = fabsf(xi[s0 + a]);
        int rank = 0;
        for (int b = 0; b < q; ++b) {
            const float ub = fabsf(xi[s0 + b]);
            rank += (ub > ua || (ub == ua && b < a)) ? 1 : 0;
        }
        from[s0 + a] = rank < keep ? 1 : 0;  // flag for now
    }
    __syncthreads();
    // ordered list of the surviving positions (one warp)
    if (threadIdx.x < 32) {
        int base = s0;
        for (int a0 = 0; a0 < q; a0 += 32) {
            const int a = a0 + threadIdx.x;
            const bool on = a < q && from[s0 + a] == 1;
            const unsigned bal = __ballot_sync(0xffffffffu, on);
            const int pos = base + __popc(bal & ((1u << threadIdx.x) - 1u));
            __syncwarp();
            if (on) from[pos] = s0 + a;
            base += __popc(bal);
        }
        if (threadIdx.x == 0) ns_sh = base;
    }
    __syncthreads();
    const int ns = ns_sh;
    for (int a = threadIdx.x; a < s0; a += blockDim.x) from[a] = a;
    __syncthreads();
    // removed atoms leave the membership bitmap (positions not in from[s0..ns))
    for (int a = threadIdx.x; a < q; a += blockDim.x) {
        bool kept = false;
        for (int b = s0; b < ns; ++b) kept |= from[b] == s0 + a;
        if (!kept) {
            const int j = Si[s0 + a];
            atomicAnd(&mw[j >> 5], ~(1u << (j & 31)));
        }
    }
    // stage everything that moves, then write it back
    float* stage = reinterpret_cast<float*>(d.chol + (size_t)i * smax * smax);
    const int nk = ns - s0;  // kept explored atoms
    int Sk[4];
    float xk[4], hk[4], rk[4];
    for (int u = 0; u < 4; ++u) {
        const int a = s0 + threadIdx.x + u * blockDim.x;
        if (a < ns) { Sk[u] = Si[from[a]]; xk[u] = xi[from[a]]; hk[u] = hi[from[a]]; rk[u] = ri[from[a]]; }
    }
    // rows a >= s0 (all columns) and columns c >= s0 of rows a < s0
    const int moved = nk * ns + s0 * nk;
    for (int e = threadIdx.x; e < moved; e += blockDim.x) {
        int a, c;
        if (e < nk * ns) { a = s0 + e / ns; c = e % ns; }
        else { const int f = e - nk * ns; a = f / nk; c = s0 + f % nk; }
        stage[e] = Gi[(size_t)from[a] * smax + from[c]];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < moved; e += blockDim.x) {
        int a, c;
        if (e < nk * ns) { a = s0 + e / ns; c = e % ns; }
        else { const int f = e - nk * ns; a = f / nk; c = s0 + f % nk; }
        Gi[(size_t)a * smax + c] = stage[e];
    }
    for (int u = 0; u < 4; ++u) {
        const int a = s0 + threadIdx.x + u * blockDim.x;
        if (a < ns) { Si[a] = Sk[u]; xi[a] = xk[u]; hi[a] = hk[u]; ri[a] = rk[u]; }
    }
    for (int a = ns + threadIdx.x; a < s; a += blockDim.x) xi[a] = 0.f;
    if (threadIdx.x == 0) {
        d.ssize[i] = ns;
        d.snew[i] = nk;
        d.explore[i] = 0;
    }
}

// ------------------------------------------------------------------ output
__global__ void k_scatter(Dev d, float* X, double* X64) {
    pdl_enter();
    const int i = blockIdx.x;
    if (i >= d.p) return;
    const int s = d.ssize[i];
    const bool fin = d.finalized[i] != 0;
    for (int a = threadIdx.x; a < s; a += blockDim.x) {
        const int j = d.S[(size_t)i * d.smax + a];
        const double v = fin ? d.xS64[(size_t)i * d.smax + a] : (double)d.xS[(size_t)i * d.smax + a];
        if (X) X[(size_t)i * d.m + j] = (float)v;
        if (X64) X64[(size_t)i * d.m + j] = v;
    }
}

// ------------------------------------------------------------------ dictionary prep
__global__ void k_colnorm(const float* A32, int n, int m, float* colnorm, __nv_bfloat16* A16, float* err2) {
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= m) return;
    const float* a = A32 + (size_t)j * n;
    double ss = 0.0, es = 0.0, ts = 0.0;
    for (int k = lane; k < n; k += 32) {
        const float v = a[k];
        ss += (double)v * (double)v;
        if (A16) {
            const __nv_bfloat16 q = __float2bfloat16_rn(v);
            A16[(size_t)j * n + k] = q;
            const double fq = (double)__bfloat162float(q), e = (double)v - fq;  // both exact in FP64
            es += e * e;
            ts += fq * fq;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        es += __shfl_xor_sync(0xffffffffu, es, o);
        ts += __shfl_xor_sync(0xffffffffu, ts, o);
    }
    if (lane == 0) {
        colnorm[j] = __double2float_ru(sqrt(ss));
        // FP64 sums of at most n squares: relative error far below the 1e-6 margin
        if (err2) {
            err2[j] = __double2float_ru(sqrt(es) * (1.0 + 1e-6));
            err2[m + j] = __double2float_ru(sqrt(ts) * (1.0 + 1e-6));
        }
    }
}

__global__ void k_max_reduce(const float* v, int len, float* out) {
    float mx = 0.f;
    for (int t = threadIdx.x; t < len; t += blockDim.x) mx = fmaxf(mx, v[t]);
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
        *out = t;
    }
}

__global__ void k_gather_r16(Dev d, int cur) {
    pdl_enter();
    const int k = blockIdx.x;
    if (k >= d.cnt->act_n[cur]) return;
    const int i = d.act[cur][k];
    const int n = d.n;
    const uint4* src = reinterpret_cast<const uint4*>(d.R16 + (size_t)i * n);
    uint4* dst = reinterpret_cast<uint4*>(d.R16c + (size_t)k * n);
    for (int t = threadIdx.x; t < n / 8; t += blockDim.x) dst[t] = src[t];
}

// Load caller residuals for a stand-alone correlation: R32 (and R16), identity active list.
__global__ void k_prep_correlate(Dev d, const float* R) {
    const int i = blockIdx.x;
    if (i >= d.p) return;
    const int n = d.n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const float v = R[(size_t)i * n + k];
        d.R32[(size_t)i * n + k] = v;
        if (d.R16) d.R16[(size_t)i * n + k] = __float2bfloat16_rn(v);
    }
    if (threadIdx.x == 0) {
        d.act[0][i] = i;
        if (i == 0) { d.cnt->act_n[0] = d.p; d.cnt->err = 0; }
    }
}

}  // namespace

cudaError_t launch_prep_correlate(const Dev& d, const float* R, cudaStream_t s, int64_t* nl) {
    if (d.p <= 0) return cudaSuccess;
    k_prep_correlate<<<d.p, 256, 0, s>>>(d, R);
    ++*nl;
    return cudaGetLastError();
}

cudaError_t launch_init(const Dev& d, cudaStream_t s, int64_t* nl) {
    if (d.p <= 0) return cudaSuccess;
    const cudaError_t e = launch_chain(k_init, dim3(d.p), dim3(256), 0, s, d);
    if (e != cudaSuccess) return e;
    ++*nl;
    return cudaGetLastError();
}

cudaError_t prepare_gram() {
    static bool attr = false;
    if (attr) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_gram_async<64, 32, 2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gram_smem<64, 32>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gram_async<64, 64, 4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gram_smem<64, 64>());
    if (e == cudaSuccess) attr = true;
    return e;
}

cudaError_t launch_gram(const Dev& d, int ub, int qmax, cudaStream_t s, int64_t* nl) {
    if (ub <= 0) return cudaSuccess;
    if ((d.n & 3) == 0) {
        cudaError_t ep = prepare_gram();
        if (ep != cudaSuccess) return ep;
        if (qmax <= 16) {  // the new atoms fit one 16-column tile
            dim3 grid(ub, (d.smax + 31) / 32);
            ep = launch_chain(k_gram_async<32, 16, 1, 2>, grid, dim3(256), gram_smem<32, 16>(), s, d);
        } else if (qmax <= 64) {  // one 64-column pass (e.g. a warm start's first iteration)
            dim3 grid(ub, (d.smax + 63) / 64);
            ep = launch_chain(k_gram_async<64, 64, 4, 4>, grid, dim3(256), gram_smem<64, 64>(), s, d);
        } else {
            dim3 grid(ub, (d.smax + 63) / 64);
            ep = launch_chain(k_gram_async<64, 32, 2, 4>, grid, dim3(256), gram_smem<64, 32>(), s, d);
        }
        if (ep != cudaSuccess) return ep;
    } else {
        dim3 grid(ub, (d.smax + GBM - 1) / GBM);
        const cudaError_t eg = launch_chain(k_gram<false>, grid, dim3(256), 0, s, d);
        if (eg != cudaSuccess) return eg;
    }
    ++*nl;
    return cudaGetLastError();
}

#ifdef MPL_APG_TRACE
extern "C" int mpl_debug_apg_trace(long long* out, int count, int reset) {
    if (count > 8192) count = 8192;
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    if (cudaMemcpyFromSymbol(out, g_apg_trace, sizeof(long long) * 8 * (size_t)count) != cudaSuccess) return -1;
    if (reset) {
        static long long zero[8192][8];
        if (cudaMemcpyToSymbol(g_apg_trace, zero, sizeof(zero)) != cudaSuccess) return -1;
    }
    return count;
}
#endif

cudaError_t prepare_apg() {
    static bool attr = false;
    if (attr) return cudaSuccess;
    const int mx = (int)((apg_area(APG_SMEM_S) + 6 * 1024) * sizeof(float));
    cudaError_t e = cudaFuncSetAttribute(k_apg<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apg<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) attr = true;
    return e;
}

// Vector stride of the master problem for a bound vcap on |S|: a multiple of 32 (and so of
// 4, the streamed product's float4 slices), at least the bound, at most the capacity rounded
// up to 4.
static int apg_vcap(const Dev& d, int vcap) {
    vcap = ((vcap + 31) / 32) * 32;
    const int cap4 = (d.smax + 3) & ~3;
    return vcap < cap4 ? vcap : cap4;
}

bool apg_split(const Dev& d, int vcap) { return apg_vcap(d, vcap) > APG_SMEM_S; }

cudaError_t launch_apg(const Dev& d, int ub, int sms, int vcap, cudaStream_t s, int64_t* nl, int cls) {
    if (ub <= 0) return cudaSuccess;
    vcap = apg_vcap(d, vcap);
    cudaError_t ep = prepare_apg();
    if (ep != cudaSuccess) return ep;
    // APG_ALL: one launch, blocks up to the bound (at most APG_SMEM_S) in shared memory;
    // APG_SMEM: the blocks that fit shared memory; APG_GLOBAL: the others, without the block
    // area, so that several CTAs per SM stream their blocks from L2/HBM
    const int gcap = cls == APG_GLOBAL ? 0 : (vcap < APG_SMEM_S ? vcap : APG_SMEM_S);
    const size_t dyn = (apg_area(gcap) + 6 * (size_t)vcap) * sizeof(float);
    int per_sm = 0;
    const bool stream = cls == APG_GLOBAL;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream ? k_apg<true> : k_apg<false>,
                                                                  APG_THREADS, dyn);
    if (e != cudaSuccess) return e;
    int grid = sms * (per_sm > 0 ? per_sm : 1);
    if (grid > ub) grid = ub;
    e = stream ? launch_chain(k_apg<true>, dim3(grid), dim3(APG_THREADS), dyn, s, d, vcap, gcap, cls)
               : launch_chain(k_apg<false>, dim3(grid), dim3(APG_THREADS), dyn, s, d, vcap, gcap, cls);
    if (e != cudaSuccess) return e;
    ++*nl;
    return cudaGetLastError();
}

cudaError_t launch_residual(const Dev& d, int ub, cudaStream_t s, int64_t* nl) {
    if (ub <= 0) return cudaSuccess;
    const cudaError_t e = launch_chain(k_residual, dim3(ub, res_blocks(d.n)), dim3(256), 0, s, d);
    if (e != cudaSuccess) return e;
    ++*nl;
    return cudaGetLastError();
}

// Per-signal statistics packed on the device into the host struct layout (one copy back).
// ------------------------------------------------------------------ re-entry
// Finished signals (reent[s] of the slots s in mslots, in slot order) go back to the end of
// the active list of this iteration, with their rows in the GEMM's compacted BF16 residual
// (the finish wrote the per-signal copy); the counters are updated by k_merge_count once
// every row is in place.
__global__ void __launch_bounds__(256) k_merge(Dev d, int cur) {
    pdl_enter();
    const int mask = d.cnt->mslots, n = d.n;
    int base = d.cnt->act_n[cur];
    for (int q = 0; q < FIN_SLOTS; ++q) {
        if (!((mask >> q) & 1)) continue;
        const int cnt = d.cnt->reent_n[q];
        for (int b = blockIdx.x; b < cnt; b += gridDim.x) {
            const int i = d.reent[q][b];
            const int row = base + b;
            if (MPL_OOB(row >= d.p || i < 0 || i >= d.p, 101)) continue;
            if (threadIdx.x == 0) {
                d.act[cur][row] = i;
                if (d.pos) d.pos[i] = row;
            }
            if (d.pos) {
                const __nv_bfloat16* src = d.R16 + (size_t)i * n;
                __nv_bfloat16* dst = d.R16c + (size_t)row * n;
                for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
            }
        }
        base += cnt;
    }
}

// Also advances the finish list slot of the selection that follows (t % FIN_SLOTS for outer
// iteration t; k_init starts it at 0) and clears the merge mask the host set.
__global__ void k_merge_count(Dev d, int cur) {
    pdl_enter();
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int mask = d.cnt->mslots;
        for (int q = 0; q < FIN_SLOTS; ++q) {
            if (!((mask >> q) & 1)) continue;
            d.cnt->act_n[cur] += d.cnt->reent_n[q];
            d.cnt->reent_n[q] = 0;
        }
        d.cnt->mslots = 0;
        d.cnt->fslot = (d.cnt->fslot + 1) % FIN_SLOTS;
    }
}

// The finishes whose signals the next merge takes back (bit s: list slot s), from the host.
__global__ void k_set_merge(Dev d, int mask) {
    pdl_enter();
    if (threadIdx.x == 0 && blockIdx.x == 0) d.cnt->mslots = mask;
}

cudaError_t launch_set_merge(const Dev& d, int mask, cudaStream_t s, int64_t* nl) {
    const cudaError_t e = launch_chain(k_set_merge, dim3(1), dim3(32), 0, s, d, mask);
    if (e != cudaSuccess) return e;
    ++*nl;
    return cudaGetLastError();
}

cudaError_t launch_merge(const Dev& d, int cur, int ub, cudaStream_t s, int64_t* nl) {
    if (ub <= 0) return cudaSuccess;
    const int grid = ub < 608 ? ub : 608;
    cudaError_t e = launch_chain(k_merge, dim3(grid), dim3(256), 0, s, d, cur);
    if (e != cudaSuccess) return e;
    e = launch_chain(k_merge_count, dim3(1), dim3(32), 0, s, d, cur);
    if (e != cudaSuccess) return e;
    *nl += 2;
    return cudaGetLastError();
}

__global__ void k_pack_stats(Dev d, mpl_signal_stats_t* out) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.p) return;
    mpl_signal_stats_t s;
    s.outer_iters = d.outer[i];
    s.inner_iters = d.inner[i];
    s.active_size = d.ssize[i];
    s.nnz = d.nnz[i];
    s.status = d.sstatus[i];
    s.finishes = d.finishes[i];
    const double obj = d.obj[i];
    s.objective = obj;
    s.kkt = fmax(d.kkt_in[i], d.kkt_out[i]);
    // relative duality gap with the dual point xi * min(1, lambda / ||A^T xi||_inf) of eq. 5
    const double ginf = d.ginf[i], rr = d.rr[i], rb = d.rb[i], lam = (double)d.lam[i];
    const double sc = (ginf > lam && ginf > 0.0) ? lam / ginf : 1.0;
    const double D = -0.5 * sc * sc * rr + sc * rb;
    s.gap = obj > 0.0 ? (obj - D) / obj : 0.0;
    out[i] = s;
}

cudaError_t launch_pack_stats(const Dev& d, mpl_signal_stats_t* out, cudaStream_t s, int64_t* nl) {
    if (d.p <= 0) return cudaSuccess;
    const cudaError_t e = launch_chain(k_pack_stats, dim3((d.p + 127) / 128), dim3(128), 0, s, d, out);
    if (e != cudaSuccess) return e;
    ++*nl;
    return cudaGetLastError();
}

cudaError_t launch_smpl_prune(const Dev& d, int ub, cudaStream_t s, int64_t* nl) {
    if (ub <= 0) return cudaSuccess;
    const cudaError_t e = launch_chain(k_smpl_prune, dim3(ub), dim3(256), 0, s, d);
    if (e != cudaSuccess) return e;
    ++*nl;
    return cudaGetLastError();
}

cudaError_t launch_scatter(const Dev& d, float* X, double* X64, cudaStream_t s, int64_t* nl) {
    if (d.p <= 0) return cudaSuccess;
    const cudaError_t e = launch_chain(k_scatter, dim3(d.p), dim3(128), 0, s, d, X, X64);
    if (e != cudaSuccess) return e;
    ++*nl;
    return cudaGetLastError();
}

cudaError_t launch_colnorm(const float* A32, int n, int m, float* colnorm, __nv_bfloat16* A16,
                           cudaStream_t s, int64_t* nl, float* err2) {
    const int per = 8;  // warps per block
    k_colnorm<<<(m + per - 1) / per, per * 32, 0, s>>>(A32, n, m, colnorm, A16, err2);
    ++*nl;
    return cudaGetLastError();
}

cudaError_t launch_max_reduce(const float* v, int len, float* out, cudaStream_t s, int64_t* nl) {
    k_max_reduce<<<1, 1024, 0, s>>>(v, len, out);
    ++*nl;
    return cudaGetLastError();
}

cudaError_t launch_gather_r16(const Dev& d, int cur, int act_n_ub, cudaStream_t s, int64_t* nl) {
    if (act_n_ub <= 0) return cudaSuccess;
    const cudaError_t e = launch_chain(k_gather_r16, dim3(act_n_ub), dim3(128), 0, s, d, cur);
    if (e != cudaSuccess) return e;
    ++*nl;
    return cudaGetLastError();
}

}  // namespace mpl
