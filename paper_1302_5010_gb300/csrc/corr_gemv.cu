// Worst-case analysis of Algorithm 1 for a handful of signals (at most GEMV_P active):
// C = A^T R as matrix-vector products.  With one to eight residuals the GEMM tiles would
// be almost empty (a 128-signal tile for one signal does 128 times the work), while the
// products are bound by reading the dictionary once: m n FP32 (or BF16) values from HBM
// per call, e.g. 16 GiB (8 GiB) for the 4096 x 2^20 dictionary of the paper's Sec. 4.6.
//
// One warp per atom (grid-stride): the atom row (n-contiguous) is read with 16-byte loads,
// four in flight per lane, and dotted with each residual (small, L1/L2 resident).  Lane l
// sums the k = 4l + 128u (FP32) or 8l + 256u (BF16) entries in order, then a butterfly adds
// the 32 lane sums, so each score is a sum of n products in a fixed order whose rounding
// error is at most gamma_n sum_k |a_jk r_k| for n >= GEMV_MIN_N (every partial sum takes at
// most n/32 + 5 roundings): the FP32 route's bound.  The BF16 products bf(a) bf(r) are exact
// in FP32 and the FP32 sums stay inside the BF16 route's accumulation term
// (1.25 n 2^-22 > n 2^-24), so the selection keeps the error band of the route it takes.
//
// C row k (k < act_n) holds the scores of signal act[k], as the GEMMs write it; the BF16
// residual of list position k is row k of the compacted R16c (the GEMM's operand).
#include "mpl_internal.cuh"

namespace mpl {

namespace {

constexpr int GEMV_THREADS = 256;
constexpr int GEMV_U = 4;  // 16-byte atom loads in flight per lane

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// streamed once per call: no L1 allocation for the dictionary
__device__ __forceinline__ float4 ld_stream4(const float* p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}
__device__ __forceinline__ uint4 ld_stream4u(const void* p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

template <int NP>
__global__ void __launch_bounds__(GEMV_THREADS) k_corr_gemv_f32(Dev d, int cur) {
    pdl_enter();
    const int act_n = min(d.cnt->act_n_of(cur), NP);
    if (act_n <= 0) return;
    const int n = d.n, m = d.m;
    const int* act = d.act_of(cur);
    const int lane = threadIdx.x & 31;
    const float* r[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) r[q] = d.R32 + (size_t)act[q < act_n ? q : 0] * n;
    const int nwarp = (gridDim.x * GEMV_THREADS) >> 5;
    const bool vec = (n & 3) == 0;
    for (int j = (int)((blockIdx.x * GEMV_THREADS + threadIdx.x) >> 5); j < m; j += nwarp) {
        const float* a = d.A32 + (size_t)j * n;
        float acc[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) acc[q] = 0.f;
        if (vec) {
            for (int k0 = 4 * lane; k0 < n; k0 += 128 * GEMV_U) {
                float4 av[GEMV_U];
#pragma unroll
                for (int u = 0; u < GEMV_U; ++u) {
                    const int k = k0 + 128 * u;
                    av[u] = k < n ? ld_stream4(a + k) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < GEMV_U; ++u) {
                    const int k = k0 + 128 * u;
                    if (k < n) {
#pragma unroll
                        for (int q = 0; q < NP; ++q) {
                            if (q < act_n) {
                                const float4 rv = __ldg(reinterpret_cast<const float4*>(r[q] + k));
                                acc[q] = fmaf(av[u].x, rv.x, acc[q]);
                                acc[q] = fmaf(av[u].y, rv.y, acc[q]);
                                acc[q] = fmaf(av[u].z, rv.z, acc[q]);
                                acc[q] = fmaf(av[u].w, rv.w, acc[q]);
                            }
                        }
                    }
                }
            }
        } else {
            for (int k = lane; k < n; k += 32) {
                const float av = __ldg(a + k);
#pragma unroll
                for (int q = 0; q < NP; ++q)
                    if (q < act_n) acc[q] = fmaf(av, __ldg(r[q] + k), acc[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const float v = warp_sum(acc[q]);
            if (lane == 0 && q < act_n) d.Cs[(size_t)q * m + j] = v;
        }
    }
}

// BF16 operands (n % 8 == 0): the atom's row of A16 and the compacted BF16 residual rows.
template <int NP>
__global__ void __launch_bounds__(GEMV_THREADS) k_corr_gemv_bf16(Dev d, int cur) {
    pdl_enter();
    const int act_n = min(d.cnt->act_n_of(cur), NP);
    if (act_n <= 0) return;
    const int n = d.n, m = d.m;
    const int lane = threadIdx.x & 31;
    const int nwarp = (gridDim.x * GEMV_THREADS) >> 5;
    for (int j = (int)((blockIdx.x * GEMV_THREADS + threadIdx.x) >> 5); j < m; j += nwarp) {
        const __nv_bfloat16* a = d.A16 + (size_t)j * n;
        float acc[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) acc[q] = 0.f;
        for (int k0 = 8 * lane; k0 < n; k0 += 256 * GEMV_U) {
            uint4 av[GEMV_U];
#pragma unroll
            for (int u = 0; u < GEMV_U; ++u) {
                const int k = k0 + 256 * u;
                av[u] = k < n ? ld_stream4u(a + k) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < GEMV_U; ++u) {
                const int k = k0 + 256 * u;
                if (k >= n) continue;
                const __nv_bfloat162* ap = reinterpret_cast<const __nv_bfloat162*>(&av[u]);
                float2 af[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) af[e] = __bfloat1622float2(ap[e]);
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    if (q < act_n) {
                        const uint4 rv = __ldg(reinterpret_cast<const uint4*>(d.R16c + (size_t)q * n + k));
                        const __nv_bfloat162* rp = reinterpret_cast<const __nv_bfloat162*>(&rv);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float2 rf = __bfloat1622float2(rp[e]);
                            acc[q] = fmaf(af[e].x, rf.x, acc[q]);
                            acc[q] = fmaf(af[e].y, rf.y, acc[q]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const float v = warp_sum(acc[q]);
            if (lane == 0 && q < act_n) d.Cs[(size_t)q * m + j] = v;
        }
    }
}

// Eight blocks per SM (up to 64 warps, each with four 512-byte atom loads in flight), but
// no more warps than atoms.
int gemv_blocks(const Dev& d) {
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (long long)sms * 8;
    const long long atoms_per_block = GEMV_THREADS / 32;
    const long long cap = ((long long)d.m + atoms_per_block - 1) / atoms_per_block;
    return (int)(want < cap ? want : cap);
}

}  // namespace

bool gemv_route(const Dev& d, int act_n_ub) { return act_n_ub > 0 && act_n_ub <= GEMV_P && d.n >= GEMV_MIN_N; }

cudaError_t launch_corr_gemv(const Dev& d, int cur, int act_n_ub, bool bf16, cudaStream_t s, int64_t* nl) {
    const dim3 grid(gemv_blocks(d)), block(GEMV_THREADS);
    cudaError_t e;
    const int np = act_n_ub <= 1 ? 1 : act_n_ub <= 2 ? 2 : act_n_ub <= 4 ? 4 : 8;
    if (bf16) {
        e = np == 1   ? launch_chain(k_corr_gemv_bf16<1>, grid, block, 0, s, d, cur)
            : np == 2 ? launch_chain(k_corr_gemv_bf16<2>, grid, block, 0, s, d, cur)
            : np == 4 ? launch_chain(k_corr_gemv_bf16<4>, grid, block, 0, s, d, cur)
                      : launch_chain(k_corr_gemv_bf16<8>, grid, block, 0, s, d, cur);
    } else {
        e = np == 1   ? launch_chain(k_corr_gemv_f32<1>, grid, block, 0, s, d, cur)
            : np == 2 ? launch_chain(k_corr_gemv_f32<2>, grid, block, 0, s, d, cur)
            : np == 4 ? launch_chain(k_corr_gemv_f32<4>, grid, block, 0, s, d, cur)
                      : launch_chain(k_corr_gemv_f32<8>, grid, block, 0, s, d, cur);
    }
    if (e != cudaSuccess) return e;
    ++*nl;
    return cudaGetLastError();
}

}  // namespace mpl
