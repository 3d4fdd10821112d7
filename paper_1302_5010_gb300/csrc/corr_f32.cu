// Worst-case analysis of Algorithm 1 for all active signals at once:
// the correlation scores C = A^T R, computed in plain FP32 on the SIMT cores.
//
// C row k holds the m scores of signal act[k]: C[k*m + j] = a_j^T r_{act[k]}.
// Both operands are K-major in HBM (atoms and residuals are n-contiguous), so a
// 128 x 128 output tile streams 128 atoms and 128 residuals through shared
// memory in K-slices of 8, transposed on the way in, with register
// double-buffering of the next slice.  Each thread owns an 8 x 8 sub-tile.
// Each score is accumulated sequentially over k with FMA, so its rounding error
// is at most gamma_n * sum_k |a_jk r_k| (used by the selection's error bound).
#include "mpl_internal.cuh"

namespace mpl {

namespace {

constexpr int BM = 128;  // atoms per tile
constexpr int BN = 128;  // signals per tile
constexpr int BK = 8;
constexpr int PAD = 4;

template <bool VEC>
__device__ __forceinline__ float4 load4(const float* row, int k, int n) {
    if (row == nullptr) return make_float4(0.f, 0.f, 0.f, 0.f);
    if (VEC) {
        if (k < n) return __ldg(reinterpret_cast<const float4*>(row + k));
        return make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float4 v;
    v.x = (k + 0 < n) ? __ldg(row + k + 0) : 0.f;
    v.y = (k + 1 < n) ? __ldg(row + k + 1) : 0.f;
    v.z = (k + 2 < n) ? __ldg(row + k + 2) : 0.f;
    v.w = (k + 3 < n) ? __ldg(row + k + 3) : 0.f;
    return v;
}

// jtile0: first atom tile of this launch (grids cover at most 65535 atom tiles; larger
// dictionaries take several launches).
template <bool VEC>
__global__ void __launch_bounds__(256) k_corr_f32(Dev d, int cur, int jtile0) {
    pdl_enter();
    const int act_n = d.cnt->act_n_of(cur);
    // signal tiles vary fastest, so the blocks in flight share their atom tile in L2
    // (the dictionary streams from HBM once per launch)
    const int k0 = blockIdx.x * BN;
    if (k0 >= act_n) return;
    const int j0 = (jtile0 + (int)blockIdx.y) * BM;
    const int n = d.n, m = d.m;
    const int* act = d.act_of(cur);

    __shared__ __align__(16) float As[2][BK][BM + PAD];
    __shared__ __align__(16) float Bs[2][BK][BN + PAD];

    const int tid = threadIdx.x;
    const int lrow = tid >> 1;       // 0..127: row of the tile this thread loads
    const int lk = (tid & 1) * 4;    // 0 or 4: k offset within the slice
    const int ja = j0 + lrow;
    const float* arow = (ja < m) ? d.A32 + (size_t)ja * n : nullptr;
    const int kb = k0 + lrow;
    const float* brow = (kb < act_n) ? d.R32 + (size_t)act[kb] * n : nullptr;

    const int tx = tid & 15;  // signal group
    const int ty = tid >> 4;  // atom group

    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

    float4 ra = load4<VEC>(arow, lk, n);
    float4 rb = load4<VEC>(brow, lk, n);
    As[0][lk + 0][lrow] = ra.x; As[0][lk + 1][lrow] = ra.y;
    As[0][lk + 2][lrow] = ra.z; As[0][lk + 3][lrow] = ra.w;
    Bs[0][lk + 0][lrow] = rb.x; Bs[0][lk + 1][lrow] = rb.y;
    Bs[0][lk + 2][lrow] = rb.z; Bs[0][lk + 3][lrow] = rb.w;
    __syncthreads();

    const int nslices = (n + BK - 1) / BK;
    for (int sl = 0; sl < nslices; ++sl) {
        const int buf = sl & 1;
        const bool more = (sl + 1) < nslices;
        if (more) {
            ra = load4<VEC>(arow, (sl + 1) * BK + lk, n);
            rb = load4<VEC>(brow, (sl + 1) * BK + lk, n);
        }
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float av[8], bv[8];
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
            av[0] = a0.x; av[1] = a0.y; av[2] = a0.z; av[3] = a0.w;
            av[4] = a1.x; av[5] = a1.y; av[6] = a1.z; av[7] = a1.w;
            bv[0] = b0.x; bv[1] = b0.y; bv[2] = b0.z; bv[3] = b0.w;
            bv[4] = b1.x; bv[5] = b1.y; bv[6] = b1.z; bv[7] = b1.w;
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
        }
        if (more) {
            const int nb = buf ^ 1;
            As[nb][lk + 0][lrow] = ra.x; As[nb][lk + 1][lrow] = ra.y;
            As[nb][lk + 2][lrow] = ra.z; As[nb][lk + 3][lrow] = ra.w;
            Bs[nb][lk + 0][lrow] = rb.x; Bs[nb][lk + 1][lrow] = rb.y;
            Bs[nb][lk + 2][lrow] = rb.z; Bs[nb][lk + 3][lrow] = rb.w;
        }
        __syncthreads();
    }

    // epilogue: row k of C is signal act[k]; atoms are contiguous within a row
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int kk = k0 + (b < 4 ? tx * 4 + b : 64 + tx * 4 + (b - 4));
        if (kk >= act_n) continue;
        float* crow = d.Cs + (size_t)kk * m;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int jb = j0 + h * 64 + ty * 4;
            if (jb + 3 < m && (m & 3) == 0) {
                *reinterpret_cast<float4*>(crow + jb) =
                    make_float4(acc[h * 4 + 0][b], acc[h * 4 + 1][b], acc[h * 4 + 2][b], acc[h * 4 + 3][b]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (jb + e < m) crow[jb + e] = acc[h * 4 + e][b];
            }
        }
    }
}

}  // namespace

cudaError_t launch_corr_f32(const Dev& d, int cur, int act_n_ub, cudaStream_t s, int64_t* nl) {
    if (act_n_ub <= 0) return cudaSuccess;
    if (gemv_route(d, act_n_ub)) return launch_corr_gemv(d, cur, act_n_ub, false, s, nl);
    const int tiles_m = (d.m + BM - 1) / BM;
    const bool vec = (d.n % 4) == 0;
    for (int t0 = 0; t0 < tiles_m; t0 += 65535) {  // grid.y is at most 65535
        dim3 grid((act_n_ub + BN - 1) / BN, tiles_m - t0 < 65535 ? tiles_m - t0 : 65535);
        const cudaError_t e = vec ? launch_chain(k_corr_f32<true>, grid, dim3(256), 0, s, d, cur, t0)
                                  : launch_chain(k_corr_f32<false>, grid, dim3(256), 0, s, d, cur, t0);
        if (e != cudaSuccess) return e;
        ++*nl;
    }
    return cudaGetLastError();
}

}  // namespace mpl
