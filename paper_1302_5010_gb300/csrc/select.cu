// Worst-case analysis of Algorithm 1, second half: per signal, the rho
// atoms outside the active set with the largest |a_j^T r| above lambda, and
// the stopping test ||r^T A||_inf <= lambda of Sec. 2.3.
//
// One CTA per active signal.  The correlation scores come from a GEMM whose
// error against the exact a_j^T r is bounded by delta = bound_c*colmax*||r||
// (FP32: gamma_n; BF16 operands: 2^-7 plus the accumulation term), or for the
// BF16 GEMM by the measured form ||a_j - bf(a_j)|| ||r|| + ||bf(a_j)|| ||r - bf(r)||
// plus the accumulation term (maxima over j kept per dictionary, the residual
// terms per signal), whichever is smaller.  The atoms
// whose GEMM score can still matter,
//     K = { j not in S : s_j >= max(s_(rho) - 2D, lambda(1+tol) - D) },
// with s_(rho) the rho-th largest GEMM score and D the bound between a GEMM
// score and the fixed-order FP32 re-score, are collected and re-scored with
// one warp-level dot product of fixed summation order.  Selection ranks by the
// re-score (ties to the lower atom index), so the plain FP32 and the mixed BF16
// paths select identically by construction.  For a signal whose residual is
// the FP64 residual of an exact finish, candidates whose re-score is within its
// own bound of lambda(1+tol) are scored once more in FP64: this certifies the
// off-support half of the KKT conditions (eq. 8).
//
// The re-score also forms a_j^T b for every candidate, with the same loads and in the same
// summation order; an atom that joins S takes it as its entry of h = A_S^T b, the linear term
// of the master problem, so the Gram growth that follows reads no atom column for h.
#include "mpl_internal.cuh"

namespace mpl {

#ifdef MPL_SEL_TRACE
// Per-signal phase cycle counters of the selection (diagnostic builds only):
// [row cache, k-th key, collect, re-score, sort + state, calls, band size, list-path
//  k-th keys, list size, -, the last call's row cache, k-th key, collect, re-score,
//  sort + state, band size, and of its chunk route: the check that failed (0: none), the
//  keys >= T, the keys in [TL, T), the chunks that qualified]
__device__ long long g_sel_trace[8192][20];
#define ST_BEGIN long long st0_ = clock64();
#define ST_ADD(slot) do { if (threadIdx.x == 0 && i < 8192) { const long long dt_ = clock64() - st0_; g_sel_trace[i][slot] += dt_; g_sel_trace[i][10 + (slot)] = dt_; } st0_ = clock64(); } while (0)
#define ST_CNT(slot) do { if (threadIdx.x == 0 && i < 8192) g_sel_trace[i][slot] += 1; } while (0)
#define ST_VAL(slot, v) do { if (threadIdx.x == 0 && i < 8192) g_sel_trace[i][slot] += (v); } while (0)
#else
#define ST_BEGIN
#define ST_ADD(slot) do {} while (0)
#define ST_CNT(slot) do {} while (0)
#define ST_VAL(slot, v) do {} while (0)
#endif

namespace {

__device__ __forceinline__ bool in_set(const uint32_t* msk, int j) {
    return (msk[j >> 5] >> (j & 31)) & 1u;
}

// Fixed-order FP32 dot of atom a with residual r by one warp; every lane
// returns the same value.  Lane l sums its float4 chunks k = 4l + 128q in
// order of q, then a fixed butterfly combines the lanes.
__device__ __forceinline__ float warp_dot_f32(const float* __restrict__ a, const float* __restrict__ r,
                                              int n, int lane) {
    float acc = 0.f;
    if ((n & 3) == 0) {
#pragma unroll 8
        for (int k = lane * 4; k < n; k += 128) {
            const float4 av = __ldg(reinterpret_cast<const float4*>(a + k));
            const float4 rv = __ldg(reinterpret_cast<const float4*>(r + k));
            acc = fmaf(av.x, rv.x, acc);
            acc = fmaf(av.y, rv.y, acc);
            acc = fmaf(av.z, rv.z, acc);
            acc = fmaf(av.w, rv.w, acc);
        }
    } else {
        for (int k = lane; k < n; k += 32) acc = fmaf(__ldg(a + k), __ldg(r + k), acc);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// The re-score of two candidates: for each atom a, a^T r and a^T b as warp_dot_f32 computes
// them (the same products summed in the same order), sharing the atoms' loads; r and b come
// from shared memory when staged there.  Each step issues RS_U loads of both columns before
// its products.  n % 4 == 0.
constexpr int RS_U = 4;
__device__ __forceinline__ void warp_dot2h_f32(const float* __restrict__ a0, const float* __restrict__ a1,
                                               const float* r, const float* b, int n, int lane, float* c0,
                                               float* c1, float* h0, float* h1) {
    float s0 = 0.f, s1 = 0.f, t0 = 0.f, t1 = 0.f;
    for (int kb = lane * 4; kb < n; kb += 128 * RS_U) {
        float4 u[RS_U], v[RS_U];
#pragma unroll
        for (int e = 0; e < RS_U; ++e) {
            const int k = kb + 128 * e;
            u[e] = k < n ? __ldg(reinterpret_cast<const float4*>(a0 + k)) : make_float4(0.f, 0.f, 0.f, 0.f);
            v[e] = k < n ? __ldg(reinterpret_cast<const float4*>(a1 + k)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int e = 0; e < RS_U; ++e) {
            const int k = kb + 128 * e;
            if (k < n) {
                const float4 rv = *reinterpret_cast<const float4*>(r + k);
                const float4 bv = *reinterpret_cast<const float4*>(b + k);
                s0 = fmaf(u[e].x, rv.x, s0); s0 = fmaf(u[e].y, rv.y, s0);
                s0 = fmaf(u[e].z, rv.z, s0); s0 = fmaf(u[e].w, rv.w, s0);
                s1 = fmaf(v[e].x, rv.x, s1); s1 = fmaf(v[e].y, rv.y, s1);
                s1 = fmaf(v[e].z, rv.z, s1); s1 = fmaf(v[e].w, rv.w, s1);
                t0 = fmaf(u[e].x, bv.x, t0); t0 = fmaf(u[e].y, bv.y, t0);
                t0 = fmaf(u[e].z, bv.z, t0); t0 = fmaf(u[e].w, bv.w, t0);
                t1 = fmaf(v[e].x, bv.x, t1); t1 = fmaf(v[e].y, bv.y, t1);
                t1 = fmaf(v[e].z, bv.z, t1); t1 = fmaf(v[e].w, bv.w, t1);
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        t0 += __shfl_xor_sync(0xffffffffu, t0, o);
        t1 += __shfl_xor_sync(0xffffffffu, t1, o);
    }
    *c0 = s0;
    *c1 = s1;
    *h0 = t0;
    *h1 = t1;
}

// One candidate: a^T r and a^T b, each in the order of warp_dot_f32.
__device__ __forceinline__ void warp_doth_f32(const float* __restrict__ a, const float* r, const float* b, int n,
                                              int lane, float* c, float* h) {
    float s = 0.f, t = 0.f;
    if ((n & 3) == 0) {
#pragma unroll 4
        for (int k = lane * 4; k < n; k += 128) {
            const float4 av = __ldg(reinterpret_cast<const float4*>(a + k));
            const float4 rv = *reinterpret_cast<const float4*>(r + k);
            const float4 bv = *reinterpret_cast<const float4*>(b + k);
            s = fmaf(av.x, rv.x, s); s = fmaf(av.y, rv.y, s); s = fmaf(av.z, rv.z, s); s = fmaf(av.w, rv.w, s);
            t = fmaf(av.x, bv.x, t); t = fmaf(av.y, bv.y, t); t = fmaf(av.z, bv.z, t); t = fmaf(av.w, bv.w, t);
        }
    } else {
        for (int k = lane; k < n; k += 32) {
            const float av = __ldg(a + k);
            s = fmaf(av, r[k], s);
            t = fmaf(av, b[k], t);
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    *c = s;
    *h = t;
}

__device__ __forceinline__ double warp_dot_f64(const float* __restrict__ a, const double* __restrict__ r,
                                               int n, int lane) {
    double acc = 0.0;
    for (int k = lane; k < n; k += 32) acc = fma((double)__ldg(a + k), r[k], acc);
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

constexpr int SEL_ROWCACHE = SEL_ROWCACHE_ATOMS;

struct SelSmem {
    unsigned hist[2048];
    unsigned long long key[SEL_KCAP];  // sort keys of the violators
    int idx[SEL_KCAP];                 // candidate atoms
    float sc[SEL_KCAP];                // their re-scores, negated for non-violators
    float hb[SEL_KCAP];                // their a^T b (the master problem's h when they join S)
    float row[SEL_ROWCACHE];           // selection keys of the signal's scores (when m fits): the
                                       // bits of |c_j|, 0 for members of S and non-finite scores
    unsigned wsum[32];                 // per-warp partial sums of the histogram scan
    unsigned kc;                       // candidates collected
    unsigned vc;                       // violators
    unsigned bin, need;
    unsigned lcnt;                     // keys in the chosen bin / gathered into the list
    unsigned outmax;                   // largest key outside K
    float offmax;                      // largest certified bound inside K
    int nonfinite;
    int qsel;                          // atoms appended to S by this selection
};

// Key of atom j: the IEEE bits of |score| (monotone for non-negative floats);
// members of S and non-finite scores key to 0 (non-finite is flagged).
__device__ __forceinline__ unsigned key_of(const float* v, const uint32_t* msk, int j, int u, int* nf) {
    if (in_set(msk, j)) return 0u;
    const unsigned b = __float_as_uint(fabsf(v[u]));
    if (b >= 0x7f800000u) { *nf = 1; return 0u; }
    return b;
}

__device__ __forceinline__ unsigned key_of(const float* row, const uint32_t* msk, int j, int* nf) {
    if (in_set(msk, j)) return 0u;
    const float v = fabsf(row[j]);
    const unsigned u = __float_as_uint(v);
    if (u >= 0x7f800000u) { *nf = 1; return 0u; }
    return u;
}

// Copy the score row and the membership bitmap into shared memory.  Thread t
// owns atoms j = 4 (t + u nt) + e (u, e < 4): four float4 loads (scalar loads
// when rows are not 16-byte aligned), all in flight together and issued before
// the bitmap is staged, so both round trips overlap.  Returns the largest key
// this thread wrote.
__device__ __forceinline__ int own_atom(int tid, int nt, int u, int e) { return 4 * (tid + u * nt) + e; }

__device__ unsigned fill_cache(const float* row, const uint32_t* msk_g, int m, SelSmem& sh) {
    static_assert(SEL_ROWCACHE <= 16 * SEL_THREADS, "one pass covers the cached row");
    const int tid = threadIdx.x, nt = blockDim.x;
    unsigned* keys = reinterpret_cast<unsigned*>(sh.row);
    // the membership bitmap (m / 32 <= 256 words) staged in the histogram, free until the radix passes
    uint32_t* msk = sh.hist;
    float4 v[4];
    if ((m & 3) == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = own_atom(tid, nt, u, 0);
            v[u] = j < m ? __ldcg(reinterpret_cast<const float4*>(row + j)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = own_atom(tid, nt, u, 0);
            v[u].x = j + 0 < m ? row[j + 0] : 0.f;
            v[u].y = j + 1 < m ? row[j + 1] : 0.f;
            v[u].z = j + 2 < m ? row[j + 2] : 0.f;
            v[u].w = j + 3 < m ? row[j + 3] : 0.f;
        }
    }
    for (int w = tid; w < (m + 31) / 32; w += nt) msk[w] = msk_g[w];
    __syncthreads();
    int nf = 0;
    unsigned tmax = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int j = own_atom(tid, nt, u, 0);
        if (j >= m) continue;
        const float f[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
        unsigned k4[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            k4[e] = j + e < m ? key_of(f, msk, j + e, e, &nf) : 0u;
            tmax = max(tmax, k4[e]);
        }
        if (j + 3 < m) {
            *reinterpret_cast<uint4*>(keys + j) = make_uint4(k4[0], k4[1], k4[2], k4[3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (j + e < m) keys[j + e] = k4[e];
        }
    }
    if (nf) sh.nonfinite = 1;
    __syncthreads();
    return tmax;
}

// Keys read from the cache (S members and non-finite scores already 0) or
// computed from the score row in global memory.
struct CachedKeys {
    const unsigned* k;
    __device__ __forceinline__ unsigned operator()(int j, int*) const { return k[j]; }
};
struct RowKeys {
    const float* row;
    const uint32_t* msk;
    __device__ __forceinline__ unsigned operator()(int j, int* nf) const { return key_of(row, msk, j, nf); }
};
// Keys already computed (the chunk maxima of k_sel_maxima).
struct PlainKeys {
    const unsigned* k;
    __device__ __forceinline__ unsigned operator()(int j, int*) const { return k[j]; }
};

// Key of the kth largest score (1-based) among the m keys, by 3 radix passes
// over 11/11/10 bits.  Returns 0 when fewer than kth keys exceed 0.  The bin
// holding the kth key is found by a block-wide suffix sum over the histogram
// (each thread owns nb / blockDim.x consecutive bins).
// The histogram scan shared by the passes: the bin that holds the need-th
// largest key (at most one thread finds it) and what is still needed inside it.
__device__ void radix_pick(int nb, unsigned need, SelSmem& sh) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int per = nb / nt;  // 4 or 2 consecutive bins per thread
    unsigned own = 0;
    for (int b = 0; b < per; ++b) own += sh.hist[tid * per + b];
    // inclusive suffix sum over the block (higher threads hold larger keys)
    unsigned suf = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_down_sync(0xffffffffu, suf, o);
        if (lane + o < 32) suf += v;
    }
    if (lane == 0) sh.wsum[warp] = suf;  // the warp's total
    __syncthreads();
    for (int w = warp + 1; w < nw; ++w) suf += sh.wsum[w];
    const unsigned above = suf - own;  // keys in bins above this thread's
    if (tid == 0) { sh.bin = 0; sh.need = need; }
    __syncthreads();
    if (above < need && suf >= need) {
        unsigned cum = above;
        int b = per - 1;
        for (; b > 0; --b) {
            const unsigned c = sh.hist[tid * per + b];
            if (cum + c >= need) break;
            cum += c;
        }
        sh.bin = (unsigned)(tid * per + b);
        sh.need = need - cum;
        sh.lcnt = sh.hist[tid * per + b];  // keys in the chosen bin
    }
    __syncthreads();
}

// Key of the kth largest score (1-based) among the m keys, by 3 radix passes
// over 11/11/10 bits.  Returns 0 when fewer than kth keys exceed 0.  After the
// first pass the keys of the chosen top bin (all the later passes look at) are
// gathered into a list in shared memory when they fit, so the second and third
// passes scan that list instead of all m keys.
template <typename K>
__device__ unsigned radix_kth(K key, int m, int kth, SelSmem& sh) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    unsigned* lst = reinterpret_cast<unsigned*>(sh.key);  // free until the violators are sorted
    constexpr unsigned LCAP = sizeof(sh.key) / sizeof(unsigned);
    unsigned prefix = 0, pmask = 0;
    unsigned need = (unsigned)kth;
    bool listed = false;
    unsigned lcount = 0;
    for (int pass = 0; pass < 3; ++pass) {
        const int nb = pass < 2 ? 2048 : 1024;          // 11, 11, 10 bits
        const int sh_ = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
        for (int b = tid; b < nb; b += nt) sh.hist[b] = 0;
        if (tid == 0) sh.lcnt = 0;
        __syncthreads();
        if (listed) {
            for (unsigned e = tid; e < lcount; e += nt) {
                const unsigned kj = lst[e];
                if ((kj & pmask) == prefix) atomicAdd(&sh.hist[(kj >> sh_) & (nb - 1)], 1u);
            }
        } else {
            int nf = 0;
#pragma unroll 4
            for (int j = tid; j < m; j += nt) {
                const unsigned kj = key(j, &nf);
                if ((kj & pmask) == prefix) atomicAdd(&sh.hist[(kj >> sh_) & (nb - 1)], 1u);
            }
            if (nf) sh.nonfinite = 1;
        }
        __syncthreads();
        radix_pick(nb, need, sh);
        prefix |= sh.bin << sh_;
        pmask |= (unsigned)(nb - 1) << sh_;
        need = sh.need;
        const unsigned inbin = sh.lcnt;
        __syncthreads();
        if (pass == 0 && inbin <= LCAP && inbin > 0) {
            // gather the keys of the chosen top bin (warp-aggregated slots)
            if (tid == 0) sh.lcnt = 0;
            __syncthreads();
            int nf = 0;
            for (int jb = tid - lane; jb < m; jb += nt) {
                const int j = jb + lane;
                const unsigned kj = j < m ? key(j, &nf) : 0u;
                const bool take = j < m && (kj & pmask) == prefix;
                const unsigned bal = __ballot_sync(0xffffffffu, take);
                unsigned base = 0;
                if (lane == 0 && bal) base = atomicAdd(&sh.lcnt, (unsigned)__popc(bal));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (take) lst[base + __popc(bal & ((1u << lane) - 1u))] = kj;
            }
            __syncthreads();
            lcount = sh.lcnt;
            listed = true;
            __syncthreads();
        }
    }
    return prefix;
}

// Key of the kth largest cached key without a histogram, for kth <= 512 (one
// thread per key of the short list below).  Each thread's largest key is known
// from fill_cache.  Let jw = ceil(kth / warps); every warp has jw threads whose
// largest key is at least the warp's jw-th largest thread maximum, so at least
// kth distinct keys are >= T = the minimum of those over the warps: T is a lower
// bound on the kth largest key.  The keys >= T (with their atoms) go to a list
// in sh.key as (key << 32 | j); the kth largest is the entry with exactly
// kth - 1 entries above it.  Returns false (the caller takes the radix passes)
// when T is 0 or the list has more than blockDim.x entries.  On success *tlo = T
// and *below = the largest key < T (for the bound on the atoms left out).
__device__ bool fast_kth(const unsigned* keys, int m, int kth, unsigned tmax, SelSmem& sh, unsigned* kkey,
                         unsigned* tlo, unsigned* below) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int jw = (kth + nw - 1) / nw;
    if (jw > 32) return false;
    unsigned v = tmax;
    if (jw == 1) {
#pragma unroll
        for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    } else {
        // bitonic sort of the warp's 32 thread maxima, descending from lane 0
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const unsigned o = __shfl_xor_sync(0xffffffffu, v, j);
                const bool desc = (lane & k) == 0, lower = (lane & j) == 0;
                v = (desc == lower) ? max(v, o) : min(v, o);
            }
        }
        v = __shfl_sync(0xffffffffu, v, jw - 1);
    }
    if (tid == 0) { sh.lcnt = 0; sh.outmax = 0; }
    if (lane == 0) sh.wsum[warp] = v;
    __syncthreads();
    unsigned T = lane < nw ? sh.wsum[lane] : 0xffffffffu;
#pragma unroll
    for (int o = 16; o; o >>= 1) T = min(T, __shfl_xor_sync(0xffffffffu, T, o));
    if (T == 0u) return false;  // uniform: every warp reduced the same values
    // the list: keys >= T.  A thread whose largest key is below T has nothing to add,
    // and that key is its largest below T; the few others scan their keys.
    unsigned omax = tmax;
    if (tmax >= T) {
        omax = 0;
        for (int q = 0; q < 16; ++q) {
            const int j = own_atom(tid, nt, q >> 2, q & 3);
            if (j >= m) break;
            const unsigned kj = keys[j];
            if (kj >= T) {
                const unsigned pos = atomicAdd(&sh.lcnt, 1u);
                if (pos < (unsigned)nt) sh.key[pos] = ((unsigned long long)kj << 32) | (unsigned)j;
            } else {
                omax = max(omax, kj);
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) omax = max(omax, __shfl_xor_sync(0xffffffffu, omax, o));
    if (lane == 0 && omax) atomicMax(&sh.outmax, omax);
    __syncthreads();
    const unsigned c = sh.lcnt;
    if (c > (unsigned)nt) return false;  // uniform
    if (tid < (int)c) {
        const unsigned long long e = sh.key[tid];
        unsigned above = 0;
#pragma unroll 8
        for (unsigned u = 0; u < c; ++u) above += sh.key[u] > e ? 1u : 0u;
        if (above == (unsigned)kth - 1u) sh.bin = (unsigned)(e >> 32);
    }
    __syncthreads();
    *kkey = sh.bin;
    *tlo = T;
    *below = sh.outmax;
    return true;
}

// fast_kth for a score row in global memory (m above the row cache): thread t owns atoms
// 4 (t + u nt) + e (e < 4, u = 0, 1, ...), the cached layout extended to any m.  One scan
// (float4 loads when the row is 16-byte aligned) gives each thread's largest key; the rest
// is fast_kth's bound T, list and rank, with the list's owners reading their atoms again.
// Returns false (radix passes) in the same cases.
template <typename K>
__device__ bool fast_kth_row(K key, const float* row, const uint32_t* msk, int m, int kth, SelSmem& sh,
                             unsigned* kkey, unsigned* tlo, unsigned* below) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int jw = (kth + nw - 1) / nw;
    if (jw > 32) return false;
    unsigned tmax = 0;
    int nf = 0;
    if ((m & 3) == 0) {
        for (int j0 = 4 * tid; j0 < m; j0 += 16 * nt) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j0 + 4 * u * nt;
                v[u] = j < m ? __ldcg(reinterpret_cast<const float4*>(row + j)) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j0 + 4 * u * nt;
                if (j < m) {
                    const float f[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) tmax = max(tmax, key_of(f, msk, j + e, e, &nf));
                }
            }
        }
    } else {
        for (int j0 = 4 * tid; j0 < m; j0 += 4 * nt)
            for (int e = 0; e < 4 && j0 + e < m; ++e) tmax = max(tmax, key(j0 + e, &nf));
    }
    if (nf) sh.nonfinite = 1;
    unsigned v = tmax;
    if (jw == 1) {
#pragma unroll
        for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    } else {
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const unsigned o = __shfl_xor_sync(0xffffffffu, v, j);
                const bool desc = (lane & k) == 0, lower = (lane & j) == 0;
                v = (desc == lower) ? max(v, o) : min(v, o);
            }
        }
        v = __shfl_sync(0xffffffffu, v, jw - 1);
    }
    if (tid == 0) { sh.lcnt = 0; sh.outmax = 0; }
    if (lane == 0) sh.wsum[warp] = v;
    __syncthreads();
    unsigned T = lane < nw ? sh.wsum[lane] : 0xffffffffu;
#pragma unroll
    for (int o = 16; o; o >>= 1) T = min(T, __shfl_xor_sync(0xffffffffu, T, o));
    if (T == 0u) return false;
    unsigned omax = tmax;
    if (tmax >= T) {
        omax = 0;
        for (int j0 = 4 * tid; j0 < m; j0 += 4 * nt)
            for (int e = 0; e < 4 && j0 + e < m; ++e) {
                const int j = j0 + e;
                const unsigned kj = key(j, &nf);
                if (kj >= T) {
                    const unsigned pos = atomicAdd(&sh.lcnt, 1u);
                    if (pos < (unsigned)nt) sh.key[pos] = ((unsigned long long)kj << 32) | (unsigned)j;
                } else {
                    omax = max(omax, kj);
                }
            }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) omax = max(omax, __shfl_xor_sync(0xffffffffu, omax, o));
    if (lane == 0 && omax) atomicMax(&sh.outmax, omax);
    __syncthreads();
    const unsigned c = sh.lcnt;
    if (c > (unsigned)nt) return false;
    if (tid < (int)c) {
        const unsigned long long e = sh.key[tid];
        unsigned above = 0;
#pragma unroll 8
        for (unsigned u = 0; u < c; ++u) above += sh.key[u] > e ? 1u : 0u;
        if (above == (unsigned)kth - 1u) sh.bin = (unsigned)(e >> 32);
    }
    __syncthreads();
    *kkey = sh.bin;
    *tlo = T;
    *below = sh.outmax;
    return true;
}

// Score rows above the shared-memory row cache: the maxima of the row's SEL_CHUNK-atom chunks
// come from k_sel_maxima (many CTAs per signal), so the signal's CTA works on m / SEL_CHUNK
// maxima instead of m scores.  T = the kth largest chunk maximum is a lower bound on the kth
// largest key (the maxima are keys of distinct atoms); the caller's band starts at or above
// both value(T) - band and lo (a lower bound it knows in advance: the threshold side of the
// band), so only chunks whose maximum reaches TL = key(max(value(T) - band, lo)), at most T,
// can hold a key the band takes, and those chunks' keys at or above TL form the list: the
// keys >= T at the front of sh.key (their rank gives the kth largest), those in [TL, T)
// behind them.
// Returns false (the row path) when more than SEL_KCAP chunks qualify, more than blockDim.x
// keys are >= T, or the list overflows.  On success as fast_kth_row.
#ifdef MPL_SEL_TRACE
#define CK_TRACE(sig, w, a, b, c) do { if (threadIdx.x == 0 && (sig) < 8192) { g_sel_trace[sig][16] = (w); g_sel_trace[sig][17] = (a); g_sel_trace[sig][18] = (b); g_sel_trace[sig][19] = (c); } } while (0)
#else
#define CK_TRACE(sig, w, a, b, c) do {} while (0)
#endif
__device__ bool fast_kth_chunks(const float* row, const uint32_t* msk, int m, const unsigned* tm, int nch, int kth,
                                float band, float lo, SelSmem& sh, unsigned* kkey, unsigned* tlo, unsigned* below,
                                int sig) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    if (kth > nch) { CK_TRACE(sig, 1, 0, 0, 0); return false; }
    const unsigned T = radix_kth(PlainKeys{tm}, nch, kth, sh);
    if (T == 0u) { CK_TRACE(sig, 2, 0, 0, 0); return false; }
    const float tv = fmaxf((__uint_as_float(T) - band) * (1.f - 2e-6f), lo);
    const unsigned TL = tv > 0.f ? min(__float_as_uint(tv), T) : 1u;
    // the chunks whose maximum reaches TL (warp-aggregated slots in sh.idx)
    if (tid == 0) { sh.kc = 0; sh.outmax = 0; }
    __syncthreads();
    unsigned omax = 0;
    for (int cb = tid - lane; cb < nch; cb += nt) {
        const int c = cb + lane;
        const unsigned mx = c < nch ? tm[c] : 0u;
        const bool take = c < nch && mx >= TL;
        const unsigned bal = __ballot_sync(0xffffffffu, take);
        unsigned base = 0;
        if (lane == 0 && bal) base = atomicAdd(&sh.kc, (unsigned)__popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (take) {
            const unsigned pos = base + __popc(bal & ((1u << lane) - 1u));
            if (pos < (unsigned)SEL_KCAP) sh.idx[pos] = c;
        } else if (mx > omax) {
            omax = mx;
        }
    }
    if (tid == 0) { sh.lcnt = 0; sh.vc = 0; }
    __syncthreads();
    const unsigned cc = sh.kc;
    if (cc > (unsigned)SEL_KCAP) { CK_TRACE(sig, 3, 0, 0, cc); return false; }  // uniform
    // their keys: one warp per chunk, lane l on atom l of the chunk (the front holds at most
    // nt entries, the back the other SEL_KCAP - nt)
    for (unsigned q = warp; q < cc; q += nw) {
        const int j0 = sh.idx[q] * SEL_CHUNK;
        for (int u = 0; u < SEL_CHUNK; u += 32) {
            const int j = j0 + u + lane;
            int nf = 0;
            const unsigned kj = j < m ? key_of(row, msk, j, &nf) : 0u;
            const bool hiw = j < m && kj >= T;
            const bool low = j < m && kj >= TL && kj < T;
            const unsigned bh = __ballot_sync(0xffffffffu, hiw), bl = __ballot_sync(0xffffffffu, low);
            unsigned baseh = 0, basel = 0;
            if (lane == 0 && bh) baseh = atomicAdd(&sh.lcnt, (unsigned)__popc(bh));
            if (lane == 0 && bl) basel = atomicAdd(&sh.vc, (unsigned)__popc(bl));
            baseh = __shfl_sync(0xffffffffu, baseh, 0);
            basel = __shfl_sync(0xffffffffu, basel, 0);
            const unsigned long long e = ((unsigned long long)kj << 32) | (unsigned)j;
            if (hiw) {
                const unsigned pos = baseh + __popc(bh & ((1u << lane) - 1u));
                if (pos < (unsigned)nt) sh.key[pos] = e;
            } else if (low) {
                const unsigned pos = basel + __popc(bl & ((1u << lane) - 1u));
                if (pos < (unsigned)(SEL_KCAP - nt)) sh.key[SEL_KCAP - 1 - pos] = e;
            } else if (kj > omax) {
                omax = kj;
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) omax = max(omax, __shfl_xor_sync(0xffffffffu, omax, o));
    if (lane == 0 && omax) atomicMax(&sh.outmax, omax);
    __syncthreads();
    const unsigned c = sh.lcnt, cl = sh.vc;
    if (c > (unsigned)nt || cl > (unsigned)(SEL_KCAP - nt)) { CK_TRACE(sig, 4, c, cl, cc); return false; }  // uniform
    CK_TRACE(sig, 0, c, cl, cc);
    if (tid < (int)c) {
        const unsigned long long e = sh.key[tid];
        unsigned above = 0;
#pragma unroll 8
        for (unsigned u = 0; u < c; ++u) above += sh.key[u] > e ? 1u : 0u;
        if (above == (unsigned)kth - 1u) sh.bin = (unsigned)(e >> 32);
    }
    // the back part behind the front one (through registers: the ranges may overlap)
    unsigned long long mv[SEL_KCAP / SEL_THREADS];
#pragma unroll
    for (int q = 0; q < SEL_KCAP / SEL_THREADS; ++q) {
        const unsigned t = tid + q * nt;
        mv[q] = t < cl ? sh.key[SEL_KCAP - 1 - t] : 0ull;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < SEL_KCAP / SEL_THREADS; ++q) {
        const unsigned t = tid + q * nt;
        if (t < cl) sh.key[c + t] = mv[q];
    }
    if (tid == 0) { sh.lcnt = c + cl; sh.vc = 0; }
    __syncthreads();
    *kkey = sh.bin;
    *tlo = TL;
    *below = sh.outmax;
    return true;
}

// The band { j : key >= tkey } from the list of fast_kth (tkey >= its T): into
// sh.idx, with the largest key left outside (list keys below tkey, or below T).
__device__ unsigned collect_list(unsigned tkey, unsigned below, SelSmem& sh) {
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned c = sh.lcnt;
    if (tid == 0) { sh.kc = 0; sh.outmax = below; }
    __syncthreads();
    unsigned omax = 0;
    for (unsigned t0 = tid - lane; t0 < c; t0 += blockDim.x) {
        const unsigned t = t0 + lane;
        const unsigned long long e = t < c ? sh.key[t] : 0ull;
        const unsigned kj = (unsigned)(e >> 32);
        const bool take = t < c && kj >= tkey;
        const unsigned bal = __ballot_sync(0xffffffffu, take);
        unsigned base = 0;
        if (lane == 0 && bal) base = atomicAdd(&sh.kc, (unsigned)__popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (take) sh.idx[base + __popc(bal & ((1u << lane) - 1u))] = (int)(unsigned)(e & 0xffffffffull);
        else if (t < c) omax = max(omax, kj);
    }
    if (omax) atomicMax(&sh.outmax, omax);
    __syncthreads();
    return sh.kc;
}

// Collect { j not in S : key >= tkey } into sh.idx (capacity SEL_KCAP) and the
// largest key left outside.  Returns the number found (may exceed the capacity).
template <typename K>
__device__ unsigned collect(K key, int m, unsigned tkey, SelSmem& sh) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) { sh.kc = 0; sh.outmax = 0; }
    __syncthreads();
    int nf = 0;
    unsigned omax = 0;
    const int lane = tid & 31;
    for (int jb = tid - lane; jb < m; jb += nt) {  // warp-aggregated slots
        const int j = jb + lane;
        unsigned kj = 0u;
        if (j < m) kj = key(j, &nf);
        const bool take = j < m && kj >= tkey && kj > 0u;
        const unsigned bal = __ballot_sync(0xffffffffu, take);
        unsigned base = 0;
        if (lane == 0 && bal) base = atomicAdd(&sh.kc, (unsigned)__popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (take) {
            const unsigned pos = base + __popc(bal & ((1u << lane) - 1u));
            if (pos < (unsigned)SEL_KCAP) sh.idx[pos] = j;
        } else if (kj > omax) {
            omax = kj;
        }
    }
    if (omax) atomicMax(&sh.outmax, omax);
    __syncthreads();
    return sh.kc;
}

// Bitonic sort of sh.key[0..len) descending; len a power of two.
__device__ void sort_desc(SelSmem& sh, int len) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int k = 2; k <= len; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = tid; t < len; t += nt) {
                const int ixj = t ^ j;
                if (ixj > t) {
                    const unsigned long long a = sh.key[t], b = sh.key[ixj];
                    const bool desc = ((t & k) == 0);
                    if (desc ? (a < b) : (a > b)) { sh.key[t] = b; sh.key[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
}

// sh.key[0..cnt) (distinct keys) in descending order.  Up to one key per
// thread: each key's rank is the number of keys above it, and it is written
// there (two barriers); otherwise the bitonic network over len (a power of two
// >= cnt, keys [cnt, len) zero).  The row cache is free by then and holds the
// ranked copy.
__device__ void sort_keys_desc(SelSmem& sh, int cnt, int len) {
    if (cnt <= 1) return;
    if (cnt > (int)blockDim.x) {
        sort_desc(sh, len);
        return;
    }
    unsigned long long* tmp = reinterpret_cast<unsigned long long*>(sh.row);
    const int t = threadIdx.x;
    if (t < cnt) {
        const unsigned long long e = sh.key[t];
        int r = 0;
#pragma unroll 8
        for (int u = 0; u < cnt; ++u) r += sh.key[u] > e ? 1 : 0;
        tmp[r] = e;
    }
    __syncthreads();
    if (t < cnt) sh.key[t] = tmp[t];
    __syncthreads();
}

// Proposal network forward pass for one candidate by one warp (weights in
// shared memory, W2 stored transposed so that lane o reads W2[o][q] without
// bank conflicts).  Lane l holds hidden units l and l + 32; every lane returns
// the logit, summed in the unit order 0..63.
__device__ float prop_logit_warp(const float* w, float f0, float f1, float f2, int lane) {
    const float x0 = (f0 - w[P_MEAN + 0]) / w[P_STD + 0];
    const float x1 = (f1 - w[P_MEAN + 1]) / w[P_STD + 1];
    const float x2 = (f2 - w[P_MEAN + 2]) / w[P_STD + 2];
    float h1[2], a2[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int o = lane + 32 * u;
        const float* r = w + P_W1 + o * 3;
        h1[u] = fmaxf(w[P_B1 + o] + r[0] * x0 + r[1] * x1 + r[2] * x2, 0.f);
        a2[u] = w[P_B2 + o];
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
#pragma unroll 8
        for (int l = 0; l < 32; ++l) {
            const int q = 32 * u + l;
            const float hq = __shfl_sync(0xffffffffu, h1[u], l);
            a2[0] = fmaf(w[P_W2 + q * PROP_H + lane], hq, a2[0]);
            a2[1] = fmaf(w[P_W2 + q * PROP_H + lane + 32], hq, a2[1]);
        }
    }
    float z = w[P_B3];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        for (int l = 0; l < 32; ++l) {
            const float ao = __shfl_sync(0xffffffffu, a2[u], l);
            z = fmaf(w[P_W3 + 32 * u + l], fmaxf(ao, 0.f), z);
        }
    }
    return z;
}

__device__ __forceinline__ unsigned ordered_bits(float x) {
    const unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

template <bool CHUNKED>
__device__ __forceinline__ void select_body(const Dev& d, int cur, int no_grow, const PropArgs& pa, int route) {
    const int kblk = blockIdx.x;
    if (kblk >= d.cnt->act_n[cur]) return;
    // the chunk maxima's non-finite flag of this position, read and cleared before any
    // return, so that it cannot reach the signal the position holds next iteration
    int nf_flag = 0;
    if (CHUNKED && threadIdx.x == 0) {
        nf_flag = d.sel_nf[kblk];
        if (nf_flag) d.sel_nf[kblk] = 0;
    }
    const int i = d.act[cur][kblk];
    const int st0 = d.state[i];
    if (st0 == ST_DONE || st0 == ST_REFINE) return;  // no worst-case analysis this iteration
    if (d.early && d.early[i] && pa.mode == SEL_NORMAL) {
        // an early-stopping rule fired after the last master problem: finish on S
        if (threadIdx.x == 0) { d.snew[i] = 0; d.state[i] = ST_FINALIZE; }
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SelSmem& sh = *reinterpret_cast<SelSmem*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int n = d.n, m = d.m;
    float* row = d.Cs + (size_t)kblk * m;
    const uint32_t* msk = d.mask + (size_t)i * d.mw;
    const float* r32 = d.R32 + (size_t)i * n;
    const float* b32 = d.B + (size_t)i * n;
    const double* r64 = d.R64 + (size_t)i * n;
    const int fin = d.finalized[i];
    const float lam = d.lam[i];
    const double lam_hi = (double)lam * (1.0 + d.tol);  // certification threshold
    const float lam_sel = (float)lam_hi;                // selection threshold
    const float rn = d.rnorm[i];
    const float delta32 = d.bound_c32 * d.colmax * rn;  // |rescore - a^T r|
    // |score - a^T r| for the route that produced this iteration's scores
    float delta = route == ROUTE_Q ? d.bound_q * d.colmax * (d.bnorm[i] + d.colmax * d.xl1[i])
                                   : (route == ROUTE_GEMM_F32 ? d.bound_f32 : d.bound_c) * d.colmax * rn;
    if (route == ROUTE_GEMM && d.precision == 1 && d.bf_ta > 0.f) {
        // the BF16 GEMM's bound from the measured rounding of this dictionary and this
        // residual (both bounds hold; the measured one is the tighter in practice)
        const float meas = (d.bf_ea * rn + d.bf_ta * (d.r16e[i] + d.bf_acc * d.r16t[i])) * 1.001f +
                           d.bound_c32 * d.colmax * rn;
        delta = fminf(delta, meas);
    }
    if (tid == 0) sh.nonfinite = 0;
    __syncthreads();

    const int ss = d.ssize[i];
    const bool prop = pa.mode != SEL_NORMAL;
    // Algorithm 1 takes rho atoms; Algorithm 2 (subspace exploratory matching)
    // takes omega*rho, of which the master problem's largest |u| stay
    const int want = d.rho * d.omega;
    const int kth = prop ? min(pa.W, m) : min(want, m);
    bool exact_scores = false;  // row holds re-scores themselves (overflow fallback)
    float kth_floor = 0.f;      // lower bound on the kth largest re-score (s_(kth) - D)
    ST_BEGIN
    unsigned kc = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        const float D = exact_scores ? 0.f : delta + delta32;
        const bool cache = m <= SEL_ROWCACHE;
        const unsigned tmax = cache ? fill_cache(row, msk, m, sh) : 0u;
        ST_ADD(0);
        const CachedKeys ck{reinterpret_cast<const unsigned*>(sh.row)};
        const RowKeys rk{row, msk};
        unsigned kkey = 0, tlo = 0, below = 0;
        // (chunked: the row's chunk maxima are in d.sel_tmax; they describe the first attempt's scores)
        const int nch = (m + SEL_CHUNK - 1) / SEL_CHUNK;
        if (CHUNKED && attempt == 0 && !cache && tid == 0 && nf_flag) sh.nonfinite = 1;
        bool listed = false;
        if (cache) {
            listed = fast_kth(ck.k, m, kth, tmax, sh, &kkey, &tlo, &below);
        } else {
            if (CHUNKED && attempt == 0) {
                // (the band below starts at or above lam_sel - D outside the warm start's pass;
                // the list's floor sits a little lower, below any rounding of that bound)
                const float lo = prop ? 0.f : (lam_sel - D) * (1.f - 2e-6f);
                listed = fast_kth_chunks(row, msk, m, d.sel_tmax + (size_t)kblk * nch, nch, kth, 2.f * D, lo, sh,
                                         &kkey, &tlo, &below, i);
                __syncthreads();  // (a failed chunk route's shared state is read before it is reused)
            }
            if (!listed) listed = fast_kth_row(rk, row, msk, m, kth, sh, &kkey, &tlo, &below);
        }
        if (!listed) kkey = cache ? radix_kth(ck, m, kth, sh) : radix_kth(rk, m, kth, sh);
        ST_VAL(7, listed ? 1 : 0);
        ST_VAL(8, listed ? sh.lcnt : 0);
        ST_ADD(1);
        const float s_rho = __uint_as_float(kkey);
        kth_floor = (s_rho - D) * (1.f - 1e-6f);
        float tau = prop ? s_rho - 2.f * D : fmaxf(s_rho - 2.f * D, lam_sel - (exact_scores ? delta32 : D));
        tau = tau * (1.f - 1e-6f);  // keep the band closed under rounding of the bound itself
        const unsigned tkey = tau > 0.f ? __float_as_uint(tau) : 1u;
        if (listed && tkey >= tlo) kc = collect_list(tkey, below, sh);
        else kc = cache ? collect(ck, m, tkey, sh) : collect(rk, m, tkey, sh);
        ST_ADD(2);
        if (kc <= (unsigned)SEL_KCAP || exact_scores) break;
        if (d.ovf_list) {
            // the band of this route is too wide: this signal is selected again from FP32
            // correlations (second pass of the iteration, narrower band)
            if (tid == 0) d.ovf_list[atomicAdd(&d.ovf_cnt->act_n[cur], 1)] = i;
            return;
        }
        // Too many candidates in the band: re-score every atom outside S in place
        // (this row is private to the signal) and select on the re-scores.
        for (int j = warp; j < m; j += nwarps) {
            float v = 0.f;
            if (!in_set(msk, j)) v = warp_dot_f32(d.A32 + (size_t)j * n, r32, n, lane);
            if (lane == 0) row[j] = v;
        }
        __syncthreads();
        if (tid == 0) atomicAdd(&d.cnt->sel_fallback, 1);
        exact_scores = true;
        delta = delta32;
    }
    kc = min(kc, (unsigned)SEL_KCAP);
    ST_VAL(6, kc);
#ifdef MPL_SEL_TRACE
    if (threadIdx.x == 0 && i < 8192) g_sel_trace[i][15] = kc;
#endif

    // Re-score the candidates (one warp each) and mark the violators.  The residual is staged
    // in the row cache's space (free once the band is collected) when it fits.
    const bool rstage = (n & 3) == 0 && n <= SEL_ROWCACHE && kc > 0;
    const bool bstage = rstage && 2 * n <= SEL_ROWCACHE;
    const float* rsm = rstage ? reinterpret_cast<const float*>(sh.row) : r32;
    const float* bsm = bstage ? reinterpret_cast<const float*>(sh.row) + n : b32;
    if (rstage) {
        float* rw = reinterpret_cast<float*>(sh.row);
        for (int k = tid * 4; k < n; k += 4 * (int)blockDim.x) {
            *reinterpret_cast<float4*>(rw + k) = __ldg(reinterpret_cast<const float4*>(r32 + k));
            if (bstage) *reinterpret_cast<float4*>(rw + n + k) = __ldg(reinterpret_cast<const float4*>(b32 + k));
        }
    }
    if (tid == 0) { sh.vc = 0; sh.offmax = 0.f; }
    __syncthreads();
    float offmax = 0.f;
    const bool pair = (n & 3) == 0;  // two candidates per warp, sharing the residual loads
    const unsigned cstep = pair ? 2u * nwarps : (unsigned)nwarps;
    for (unsigned c0 = pair ? 2u * warp : (unsigned)warp; c0 < kc; c0 += cstep) {
      float dots[2], hs[2];
      if (pair && c0 + 1 < kc) {
          warp_dot2h_f32(d.A32 + (size_t)sh.idx[c0] * n, d.A32 + (size_t)sh.idx[c0 + 1] * n, rsm, bsm, n, lane,
                         &dots[0], &dots[1], &hs[0], &hs[1]);
      } else {
          warp_doth_f32(d.A32 + (size_t)sh.idx[c0] * n, rsm, bsm, n, lane, &dots[0], &hs[0]);
          dots[1] = hs[1] = 0.f;
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const unsigned c = c0 + e;
        if (c >= kc || (e == 1 && !pair)) break;
        const int j = sh.idx[c];
        const float* aj = d.A32 + (size_t)j * n;
        const float c32 = fabsf(dots[e]);
        float score = c32;
        int viol = c32 > lam_sel;
        float certb = c32 + delta32;
        if (fin && !viol && (double)c32 + (double)delta32 > lam_hi) {
            const double c64 = fabs(warp_dot_f64(aj, r64, n, lane));
            score = (float)c64;
            viol = c64 > lam_hi;
            certb = (float)(c64 * (1.0 + 1e-12));
        }
        if (lane == 0) {
            sh.sc[c] = viol ? score : -score;
            sh.hb[c] = hs[e];
        }
        offmax = fmaxf(offmax, certb);
      }
    }
    if (lane == 0 && offmax > 0.f) atomicMax(reinterpret_cast<unsigned*>(&sh.offmax), __float_as_uint(offmax));
    __syncthreads();
    ST_ADD(3);
    if (prop) {
        // --- warm-start proposal / training examples: the top-W candidates by re-score
        float* wsm = reinterpret_cast<float*>(smem_raw + sizeof(SelSmem));
        for (int t = tid; t < PROP_NPARAM; t += blockDim.x) {
            int dst = t;
            if (t >= P_W2 && t < P_W2 + PROP_H * PROP_H) {  // W2 transposed
                const int o = (t - P_W2) / PROP_H, q = (t - P_W2) % PROP_H;
                dst = P_W2 + q * PROP_H + o;
            }
            wsm[dst] = pa.w ? pa.w[t] : 0.f;
        }
        // only candidates that can be among the W largest re-scores are sorted: the W-th
        // largest re-score is at least s_(W) - D
        if (tid == 0) sh.vc = 0;
        __syncthreads();
        for (unsigned c = tid; c < kc; c += blockDim.x) {
            const float a = fabsf(sh.sc[c]);
            if (a >= kth_floor) {
                const unsigned pos = atomicAdd(&sh.vc, 1u);
                sh.key[pos] = ((unsigned long long)__float_as_uint(a) << 32) |
                              (unsigned long long)(0xffffffffu - (unsigned)sh.idx[c]);
            }
        }
        __syncthreads();
        const unsigned kw = sh.vc;
        int len2 = 1;
        while (len2 < (int)kw) len2 <<= 1;
        for (int t = kw + tid; t < len2; t += blockDim.x) sh.key[t] = 0ull;
        __syncthreads();
        sort_keys_desc(sh, (int)kw, len2);
        const int W = min((int)kw, pa.W);
        const float f1 = logf(fmaxf(rn, 1e-30f) / lam);
        const float gscale = rsqrtf(1.f + (float)m / (float)n);
        // logits (or examples) for the W candidates, in score order
        if (pa.mode == SEL_EXAMPLES) {
            for (int r = tid; r < W; r += blockDim.x) {
                const unsigned long long k = sh.key[r];
                const int j = (int)(0xffffffffu - (unsigned)(k & 0xffffffffull));
                const float c32 = __uint_as_float((unsigned)(k >> 32));
                float* e = pa.ex + ((size_t)i * pa.W + r) * 4;
                e[0] = c32 / lam; e[1] = f1; e[2] = (pa.rn ? pa.rn[j] : 1.f) * gscale;
                e[3] = pa.xref[(size_t)i * m + j] != 0.f ? 1.f : 0.f;
            }
        } else {
            for (int r = warp; r < W; r += nwarps) {
                const unsigned long long k = sh.key[r];
                const int j = (int)(0xffffffffu - (unsigned)(k & 0xffffffffull));
                const float c32 = __uint_as_float((unsigned)(k >> 32));
                const float z = prop_logit_warp(wsm, c32 / lam, f1, (pa.rn ? pa.rn[j] : 1.f) * gscale, lane);
                if (lane == 0) { sh.sc[r] = z; sh.idx[r] = j; }
            }
        }
        if (pa.mode == SEL_EXAMPLES) {
            for (int r = W + tid; r < pa.W; r += blockDim.x) pa.ex[((size_t)i * pa.W + r) * 4 + 3] = -1.f;
            return;
        }
        __syncthreads();
        // tier 1: MPL's own rho largest violators (the first candidates with c > lambda);
        // tier 2: the others the network accepts, by logit
        int nv = 0;
        for (int r = 0; r < W && nv < d.rho; ++r)
            if (__uint_as_float((unsigned)(sh.key[r] >> 32)) > lam_sel) ++nv; else break;
        __syncthreads();
        if (tid == 0) sh.vc = 0;
        __syncthreads();
        for (int r = nv + tid; r < W; r += blockDim.x) {
            if (sh.sc[r] > pa.thr) {
                const unsigned pos = atomicAdd(&sh.vc, 1u);
                if (MPL_OOB(SEL_KCAP / 2 + pos >= SEL_KCAP, 501)) continue;
                sh.key[SEL_KCAP / 2 + pos] = ((unsigned long long)ordered_bits(sh.sc[r]) << 32) |
                                             (unsigned long long)(0xffffffffu - (unsigned)sh.idx[r]);
            }
        }
        __syncthreads();
        // tier-1 atoms into the front of key[] (score order), tier 2 sorted by logit
        const int n2 = (int)sh.vc;
        int len3 = 1;
        while (len3 < n2) len3 <<= 1;
        // move tier 2 into key[0..] for sorting, tier-1 indices saved in idx[] copies
        for (int t = tid; t < nv; t += blockDim.x) sh.sc[SEL_KCAP / 2 + t] = __int_as_float(sh.idx[t]);
        __syncthreads();
        for (int t = tid; t < len3; t += blockDim.x) sh.key[t] = t < n2 ? sh.key[SEL_KCAP / 2 + t] : 0ull;
        __syncthreads();
        sort_keys_desc(sh, n2, len3);
        if (tid == 0) {
            d.outer[i] += 1;
            int q = 0;
            const int room = min(d.smax - ss, pa.cap);
            int* Si = d.S + (size_t)i * d.smax;
            float* xi = d.xS + (size_t)i * d.smax;
            uint32_t* mw = d.mask + (size_t)i * d.mw;
            for (int t = 0; t < nv + n2 && q < room; ++t) {
                const int j = t < nv ? __float_as_int(sh.sc[SEL_KCAP / 2 + t])
                                     : (int)(0xffffffffu - (unsigned)(sh.key[t - nv] & 0xffffffffull));
                if (MPL_OOB(j < 0 || j >= m || ss + q >= d.smax, 502)) break;
                Si[ss + q] = j;
                xi[ss + q] = 0.f;
                mw[j >> 5] |= 1u << (j & 31);
                ++q;
            }
            d.ssize[i] = ss + q;
            d.snew[i] = q;
            if (d.explore) d.explore[i] = 0;
            d.state[i] = q > 0 ? ST_GROW : ST_FINALIZE;
            if (q > 0) d.finalized[i] = 0;
            sh.qsel = q;
        }
        __syncthreads();
        // h of the appended atoms (the order of the proposal's list is not the candidates')
        const int qp = sh.qsel;
        const int* Sp = d.S + (size_t)i * d.smax;
        for (int a = warp; a < qp; a += nwarps) {
            float c, h;
            warp_doth_f32(d.A32 + (size_t)Sp[ss + a] * n, r32, b32, n, lane, &c, &h);
            if (lane == 0) d.h[(size_t)i * d.smax + ss + a] = h;
        }
        return;
    }
    // Sort keys: (re-score bits, inverted index) so that larger scores come
    // first and the lower index wins ties.
    for (unsigned c = tid; c < kc; c += blockDim.x) {
        if (sh.sc[c] > 0.f) {
            const unsigned pos = atomicAdd(&sh.vc, 1u);
            sh.key[pos] = ((unsigned long long)__float_as_uint(sh.sc[c]) << 32) |
                          (unsigned long long)(0xffffffffu - (unsigned)sh.idx[c]);
        }
    }
    __syncthreads();
    const int vc = (int)sh.vc;
    int len = 1;
    while (len < vc) len <<= 1;
    for (int t = vc + tid; t < len; t += blockDim.x) sh.key[t] = 0ull;
    __syncthreads();
    sort_keys_desc(sh, vc, len);

    // State transition (one thread).
    ST_ADD(4);
    ST_CNT(5);
    if (tid == 0) {
        d.outer[i] += 1;
        sh.qsel = 0;
        if (sh.nonfinite) {
            d.sstatus[i] = MPL_SIG_NONFINITE;
            d.state[i] = ST_DONE;
        } else {
            // certified bound on |a_j^T r| over atoms outside S
            const float outside = (sh.outmax ? __uint_as_float(sh.outmax) : 0.f) + delta;
            const double offb = fmax((double)outside, (double)sh.offmax);
            int q = min(vc, want);
            if (q > d.smax - ss) q = d.smax - ss;
            if (no_grow) q = 0;
            // early stopping, eq. (stop1): the residual norm, or the certified bound on the
            // correlations outside S
            // (only while violators remain: without them the stopping condition of eq. 8 holds)
            const bool stop1 = d.early && vc > 0 &&
                               ((d.stop_r2 >= 0.f && rn <= d.stop_r2) ||
                                (d.stop_rinf >= 0.f && offb <= (double)d.stop_rinf));
            if (stop1) {
                d.early[i] = 1;
                q = 0;
            }
            if (d.explore) d.explore[i] = q > d.rho ? q : 0;  // prune to rho after the master problem
            if (q > 0) {
                int* Si = d.S + (size_t)i * d.smax;
                float* xi = d.xS + (size_t)i * d.smax;
                uint32_t* mw = d.mask + (size_t)i * d.mw;
                for (int a = 0; a < q; ++a) {
                    const int j = (int)(0xffffffffu - (unsigned)(sh.key[a] & 0xffffffffull));
                    if (MPL_OOB(j < 0 || j >= m || ss + a >= d.smax, 503)) break;
                    Si[ss + a] = j;
                    xi[ss + a] = 0.f;  // warm start: new entries at zero (Alg. 1)
                    mw[j >> 5] |= 1u << (j & 31);
                }
                d.ssize[i] = ss + q;
                d.snew[i] = q;
                d.finalized[i] = 0;
                d.state[i] = ST_GROW;
                sh.qsel = q;
            } else if (fin && stop1) {
                // the current point is already the exact restricted solution
                d.ginf[i] = fmax(d.ginf[i], offb);
                d.state[i] = ST_DONE;
                d.sstatus[i] = MPL_SIG_EARLY_STOP;
            } else if (fin) {
                d.kkt_out[i] = lam > 0.f ? fmax(offb - (double)lam, 0.0) / (double)lam : offb;
                d.ginf[i] = fmax(d.ginf[i], offb);
                d.state[i] = ST_DONE;
                if (vc == 0) d.sstatus[i] = MPL_SIG_CERTIFIED;
                else d.sstatus[i] = no_grow ? MPL_SIG_MAX_OUTER : MPL_SIG_CAPACITY;
            } else {
                d.snew[i] = 0;
                d.state[i] = ST_FINALIZE;
            }
        }
    }
    __syncthreads();
    // h of the appended atoms: a violator's rank among the sorted keys is its position after ss
    const int qs = sh.qsel;
    if (qs > 0) {
        for (unsigned c = tid; c < kc; c += blockDim.x) {
            if (!(sh.sc[c] > 0.f)) continue;
            const unsigned long long kcand = ((unsigned long long)__float_as_uint(sh.sc[c]) << 32) |
                                             (unsigned long long)(0xffffffffu - (unsigned)sh.idx[c]);
            int lo = 0, hi = vc;  // keys descending: the first position whose key is <= kcand
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (sh.key[mid] > kcand) lo = mid + 1; else hi = mid;
            }
            if (lo < qs && !MPL_OOB(ss + lo >= d.smax, 504))
                d.h[(size_t)i * d.smax + ss + lo] = sh.hb[c];
        }
    }
}

// Stable compaction of the active list into the work lists of this outer
// iteration (one CTA): grow, finish, master problem, and the next active list.
// The states were written by other CTAs of the same launch when the compaction
// runs at the end of the selection, so they are read past L1.
__device__ void compact_body(const Dev& d, int cur) {
    const int nact = d.cnt->act_n[cur];
    const int* act = d.act[cur];
    int* nxt = d.act[cur ^ 1];
    __shared__ int wsum[3][32];
    __shared__ int base[3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x, nw = nt >> 5;
    if (tid < 3) base[tid] = 0;
    if (tid < 96) wsum[tid / 32][tid % 32] = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nact; c0 += nt) {
        const int k = c0 + tid;
        int sig = -1, st = ST_DONE;
        if (k < nact) { sig = __ldcg(act + k); st = __ldcg(d.state + sig); }
        // the next active list: signals with a master problem to solve; the ones sent to the
        // exact finish leave it and come back through reent[] once their finish is done
        const int f[3] = {st == ST_GROW || st == ST_REFINE, st == ST_FINALIZE, st == ST_GROW || st == ST_REFINE};
        if (st == ST_REFINE) d.state[sig] = ST_GROW;  // master problem again, no new atoms
        int pre[3];
        const unsigned lt = (1u << lane) - 1u;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const unsigned b = __ballot_sync(0xffffffffu, f[q]);
            pre[q] = __popc(b & lt);
            if (lane == 0) wsum[q][warp] = __popc(b);
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                int v = lane < nw ? wsum[q][lane] : 0;
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v += u;
                }
                wsum[q][lane] = v;  // inclusive
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int off = base[q] + (warp ? wsum[q][warp - 1] : 0) + pre[q];
            if (f[q]) {
                if (MPL_OOB(off < 0 || off >= d.p || sig < 0 || sig >= d.p, 504)) continue;
                if (q == 0) { d.list_grow[off] = sig; d.list_apg[off] = sig; }
                else if (q == 1) d.list_fin[d.cnt->fslot][off] = sig;
                else {
                    nxt[off] = sig;
                    if (d.pos) d.pos[sig] = off;  // its GEMM row next iteration
                }
            }
        }
        __syncthreads();
        if (tid < 3) base[tid] += wsum[tid][31];
        __syncthreads();
    }
    if (tid == 0) {
        if (d.ovf_cnt) d.ovf_cnt->act_n[cur ^ 1] = 0;  // next iteration's second-pass list
        d.cnt->cols += (unsigned long long)nact;
        d.cnt->grow_n = base[0];
        d.cnt->apg_n = base[0];
        d.cnt->fin_n = base[1];
        d.cnt->fin_par[d.cnt->fslot] = base[1];
        d.cnt->act_n[cur ^ 1] = base[2];
        d.cnt->apg_head = 0;
        d.cnt->apg_head2 = 0;
    }
}

__global__ void __launch_bounds__(1024) k_compact(Dev d, int cur) {
    pdl_enter();
    compact_body(d, cur);
}

// The selection of one outer iteration; with fuse set, the last CTA to finish
// (counted with a fenced atomic) also runs the compaction, saving a launch.
template <bool CHUNKED>
__global__ void __launch_bounds__(SEL_THREADS, 2) k_select(Dev d, int cur, int no_grow, PropArgs pa, int route,
                                                           int fuse) {
    pdl_enter();
    select_body<CHUNKED>(d, cur, no_grow, pa, route);
    if (!fuse) return;
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&d.cnt->sel_done, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    compact_body(d, cur);
    if (threadIdx.x == 0) d.cnt->sel_done = 0;
}

// Chunk maxima of the score rows (see fast_kth_chunks): warp w of signal position blockIdx.x
// takes the 32 chunks [32 w', 32 w' + 32) (w' = 8 blockIdx.y + w), i.e. 1024 consecutive atoms.  Each of
// its eight float4 loads covers four chunks (eight lanes per chunk, coalesced across the warp);
// the eight lanes of a chunk combine by shuffles.  Ragged ends (a partial last warp, or
// m % 4 != 0) take one chunk per lane with scalar loads.  Writes the largest key of each chunk
// (0 for members of S and non-finite scores) and flags non-finite scores per signal position
// (cleared by the selection that reads the flag).
__global__ void __launch_bounds__(256) k_sel_maxima(Dev d, int cur) {
    static_assert(SEL_CHUNK == 32, "k_sel_maxima: a warp covers 32 chunks of 32 atoms");
    pdl_enter();
    const int kblk = blockIdx.x;
    if (kblk >= d.cnt->act_n[cur]) return;
    const int i = d.act[cur][kblk];
    const int m = d.m, nch = (m + SEL_CHUNK - 1) / SEL_CHUNK;
    const int lane = threadIdx.x & 31;
    const int cw = (blockIdx.y * 8 + (threadIdx.x >> 5)) * 32;  // first chunk of this warp
    if (cw >= nch) return;
    const float* row = d.Cs + (size_t)kblk * m;
    const uint32_t* msk = d.mask + (size_t)i * d.mw;
    unsigned* tm = d.sel_tmax + (size_t)kblk * nch;
    const int j0 = cw * SEL_CHUNK;
    int nf = 0;
    if ((m & 3) == 0 && j0 + 32 * SEL_CHUNK <= m) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcs(reinterpret_cast<const float4*>(row + j0 + 128 * u + 4 * lane));
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float f[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
            const int j = j0 + 128 * u + 4 * lane;
            unsigned mx = 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) mx = max(mx, key_of(f, msk, j + e, e, &nf));
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 4));
            if ((lane & 7) == 0) tm[cw + 4 * u + (lane >> 3)] = mx;
        }
    } else {
        const int c = cw + lane;
        if (c < nch) {
            unsigned mx = 0;
            for (int j = c * SEL_CHUNK; j < (c + 1) * SEL_CHUNK && j < m; ++j) mx = max(mx, key_of(row, msk, j, &nf));
            tm[c] = mx;
        }
    }
    if (nf) atomicExch(&d.sel_nf[kblk], 1);
}

}  // namespace

#ifdef MPL_SEL_TRACE
extern "C" int mpl_debug_sel_trace(long long* out, int count, int reset) {
    if (count > 8192) count = 8192;
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    if (cudaMemcpyFromSymbol(out, g_sel_trace, sizeof(long long) * 20 * (size_t)count) != cudaSuccess) return -1;
    if (reset) {
        static long long zero[8192][20];
        if (cudaMemcpyToSymbol(g_sel_trace, zero, sizeof(zero)) != cudaSuccess) return -1;
    }
    return count;
}
#endif

bool sel_chunked(const Dev& d, int act_n_ub) {
    return d.sel_tmax && d.sel_nf && act_n_ub > 0 && d.m > SEL_ROWCACHE_ATOMS;
}

cudaError_t prepare_select() {
    static bool attr = false;
    if (attr) return cudaSuccess;
    const int mx = (int)(sizeof(SelSmem) + PROP_NPARAM * sizeof(float));
    cudaError_t e = cudaFuncSetAttribute(k_select<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_select<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) attr = true;
    return e;
}

cudaError_t launch_select(const Dev& d, int cur, int no_grow, int act_n_ub, cudaStream_t s, int64_t* nl,
                          const PropArgs* pa, int route, int fuse_compact, int chunked) {
    if (act_n_ub <= 0) return cudaSuccess;
    PropArgs a{};
    if (pa) a = *pa;
    const size_t sm = sizeof(SelSmem) + (a.mode != SEL_NORMAL ? PROP_NPARAM * sizeof(float) : 0);
    cudaError_t e = prepare_select();
    if (e != cudaSuccess) return e;
    chunked = chunked && sel_chunked(d, act_n_ub) ? 1 : 0;
    if (chunked) {
        const int nch = (d.m + SEL_CHUNK - 1) / SEL_CHUNK;
        e = launch_chain(k_sel_maxima, dim3(act_n_ub, (nch + 255) / 256), dim3(256), 0, s, d, cur);
        if (e != cudaSuccess) return e;
        ++*nl;
    }
    e = chunked ? launch_chain(k_select<true>, dim3(act_n_ub), dim3(SEL_THREADS), sm, s, d, cur, no_grow, a, route,
                               fuse_compact)
                : launch_chain(k_select<false>, dim3(act_n_ub), dim3(SEL_THREADS), sm, s, d, cur, no_grow, a, route,
                               fuse_compact);
    if (e != cudaSuccess) return e;
    ++*nl;
    return cudaGetLastError();
}

cudaError_t launch_compact(const Dev& d, int cur, cudaStream_t s, int64_t* nl) {
    const cudaError_t e = launch_chain(k_compact, dim3(1), dim3(1024), 0, s, d, cur);
    if (e != cudaSuccess) return e;
    ++*nl;
    return cudaGetLastError();
}

}  // namespace mpl
