// Worst-case analysis by the BMPL identity (eq. "batchQ", Sec. 3):
//
//     g_i = A^T (b_i - A_S x_S) = beta_i - Q_S x_S,   beta_i = A^T b_i,  Q = A^T A,
//
// with Q and beta computed once (Q per dictionary, beta at the first outer
// iteration, where x = 0 and the ordinary correlation of the residual b_i is
// beta_i itself).  Per signal the route reads |supp(x)| rows of Q (m floats
// each) instead of the whole dictionary, so it is HBM-bound at
// 4 m |supp(x)| bytes per signal against 2 n m FLOPs for the GEMM; the host
// takes it only for iterations where its bound on |S| makes it the cheaper one.
//
// Scores: c_j = beta_j - sum_a Q[S_a][j] x_a in FP32, nonzeros of x_S in append
// order, one FMA chain per j.  Error against a_j^T r: at most
// bound_q * colmax * (||b|| + colmax ||x||_1) (FP32 beta and Q entries from
// the FP32 GEMM, the FP32 sum, and the FP32 residual the re-score uses), which
// the selection kernel takes as this route's band.
//
// Q also serves the Gram growth (MPL_OPT_QGRAM): the master problem's Gram block
// G_SS is Q's S x S sub-block, so its new columns are read out of Q (k_gram_gather).
#include "mpl_internal.cuh"

namespace mpl {

namespace {

constexpr int QT = 256;  // threads per block; each thread scores 4 consecutive atoms

__global__ void __launch_bounds__(QT) k_corr_q(Dev d, int cur) {
    pdl_enter();
    const int kblk = blockIdx.x;
    if (kblk >= d.cnt->act_n[cur]) return;
    const int i = d.act[cur][kblk];
    const int m = d.m, smax = d.smax, s = d.ssize[i];
    __shared__ int nzi[1024];
    __shared__ float nzv[1024];
    __shared__ int cntnz;
    const float* xi = d.xS + (size_t)i * smax;
    const int* Si = d.S + (size_t)i * smax;
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
    if (blockIdx.y == 0 && threadIdx.x == 0) atomicAdd(&d.cnt->qcols, 1ull);
    const int nz = cntnz;
    const int j0 = (blockIdx.y * QT + threadIdx.x) * 4;
    if (j0 >= m) return;
    const float* beta = d.beta + (size_t)i * m;
    float* out = d.Cs + (size_t)kblk * m;
    if ((m & 3) == 0) {
        float4 acc = *reinterpret_cast<const float4*>(beta + j0);
        int a = 0;
        for (; a + 3 < nz; a += 4) {
            const float4 q0 = __ldg(reinterpret_cast<const float4*>(d.Q + (size_t)nzi[a] * m + j0));
            const float4 q1 = __ldg(reinterpret_cast<const float4*>(d.Q + (size_t)nzi[a + 1] * m + j0));
            const float4 q2 = __ldg(reinterpret_cast<const float4*>(d.Q + (size_t)nzi[a + 2] * m + j0));
            const float4 q3 = __ldg(reinterpret_cast<const float4*>(d.Q + (size_t)nzi[a + 3] * m + j0));
            const float v0 = nzv[a], v1 = nzv[a + 1], v2 = nzv[a + 2], v3 = nzv[a + 3];
            acc.x = fmaf(-v0, q0.x, acc.x); acc.y = fmaf(-v0, q0.y, acc.y);
            acc.z = fmaf(-v0, q0.z, acc.z); acc.w = fmaf(-v0, q0.w, acc.w);
            acc.x = fmaf(-v1, q1.x, acc.x); acc.y = fmaf(-v1, q1.y, acc.y);
            acc.z = fmaf(-v1, q1.z, acc.z); acc.w = fmaf(-v1, q1.w, acc.w);
            acc.x = fmaf(-v2, q2.x, acc.x); acc.y = fmaf(-v2, q2.y, acc.y);
            acc.z = fmaf(-v2, q2.z, acc.z); acc.w = fmaf(-v2, q2.w, acc.w);
            acc.x = fmaf(-v3, q3.x, acc.x); acc.y = fmaf(-v3, q3.y, acc.y);
            acc.z = fmaf(-v3, q3.z, acc.z); acc.w = fmaf(-v3, q3.w, acc.w);
        }
        for (; a < nz; ++a) {
            const float4 q0 = __ldg(reinterpret_cast<const float4*>(d.Q + (size_t)nzi[a] * m + j0));
            const float v0 = nzv[a];
            acc.x = fmaf(-v0, q0.x, acc.x); acc.y = fmaf(-v0, q0.y, acc.y);
            acc.z = fmaf(-v0, q0.z, acc.z); acc.w = fmaf(-v0, q0.w, acc.w);
        }
        *reinterpret_cast<float4*>(out + j0) = acc;
    } else {
        for (int e = 0; e < 4 && j0 + e < m; ++e) {
            const int j = j0 + e;
            float acc = beta[j];
            for (int a = 0; a < nz; ++a) acc = fmaf(-nzv[a], __ldg(d.Q + (size_t)nzi[a] * m + j), acc);
            out[j] = acc;
        }
    }
}

// beta_i <- score row of signal i (the iteration's residual is b_i).
__global__ void k_save_beta(Dev d, int cur) {
    pdl_enter();
    const int kblk = blockIdx.x;
    if (kblk >= d.cnt->act_n[cur]) return;
    const int i = d.act[cur][kblk];
    const float* src = d.Cs + (size_t)kblk * d.m;
    float* dst = d.beta + (size_t)i * d.m;
    // eight loads per thread in flight before their stores (float4 rows when m % 4 == 0)
    if ((d.m & 3) == 0) {
        const int m4 = d.m >> 2;
        for (int j0 = threadIdx.x; j0 < m4; j0 += 8 * blockDim.x) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + u * blockDim.x;
                if (j < m4) v[u] = reinterpret_cast<const float4*>(src)[j];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + u * blockDim.x;
                if (j < m4) reinterpret_cast<float4*>(dst)[j] = v[u];
            }
        }
    } else {
        for (int j0 = threadIdx.x; j0 < d.m; j0 += 8 * blockDim.x) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + u * blockDim.x;
                if (j < d.m) v[u] = src[j];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + u * blockDim.x;
                if (j < d.m) dst[j] = v[u];
            }
        }
    }
}

// Identity column list and counters for the Gram build (the FP32 correlation
// kernel treats the atoms as m signals).
__global__ void k_gram_q_prep(Counters* cnt, int* act, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) act[i] = i;
    if (i == 0) {
        cnt->act_n[0] = m;
        cnt->act_n[1] = 0;
        cnt->err = 0;
    }
}

// Gram growth from Q (Sec. 3: Q = A^T A is precomputed off-line, and the master
// problem's Gram block G_SS is its S x S sub-block).  For each growing signal
// the new columns of G_SS are copied out of Q (the new entries of h = A_S^T b
// come with the selection's re-score).  Q was built by the FP32 GEMM with one
// FMA chain per entry over k ascending, the order of the computed Gram block, so
// G is the same bits as launch_gram's.

__global__ void __launch_bounds__(256) k_gram_gather(Dev d) {
    pdl_enter();
    const int g = blockIdx.x;
    if (g >= d.cnt->grow_n) return;
    const int i = d.list_grow[g];
    const int s = d.ssize[i], q = d.snew[i], s0 = s - q;
    if (q == 0) return;  // a refine pass: the block is complete
    const int m = d.m, smax = d.smax;
    const int* Si = d.S + (size_t)i * smax;
    float* Gi = d.G + (size_t)i * smax * smax;
    __shared__ int sidx[1024];  // smax <= 1024
    constexpr int GT_A = 32, GT_C = 64;
    __shared__ float gt[GT_C][GT_A + 1];
    if (threadIdx.x == 0)  // s q entries of Q read, 2 s q of G written
        atomicAdd(&d.cnt->gram_bytes, 12ull * s * q);
    if (MPL_OOB(s > smax || s > 1024 || q > s, 401)) return;
    for (int a = threadIdx.x; a < s; a += blockDim.x) sidx[a] = Si[a];
    __syncthreads();
    // new columns (and, by symmetry, rows) of G_SS in tiles of GT_A positions of S by GT_C new
    // atoms: eight independent Q reads per thread in flight (scattered either way), the new
    // rows G[s0 + c][a] written along a, then through a shared-memory tile the new columns
    // G[a][s0 + c] written along c, so that both halves are stored in whole sectors
    const int ta = threadIdx.x & (GT_A - 1), tc = threadIdx.x >> 5;  // 256 threads: tc < 8
    for (int a0 = 0; a0 < s; a0 += GT_A) {
        for (int c0 = 0; c0 < q; c0 += GT_C) {
            const int a = a0 + ta;
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = c0 + tc + 8 * u;
                v[u] = (a < s && c < q) ? __ldg(d.Q + (size_t)sidx[a] * m + sidx[s0 + c]) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = c0 + tc + 8 * u;
                if (a < s && c < q) Gi[(size_t)(s0 + c) * smax + a] = v[u];
                gt[tc + 8 * u][ta] = v[u];
            }
            __syncthreads();
            // the transposed tile: thread (row, lane) writes G[a0 + row][s0 + c0 + lane (+ 32)]
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int ar = tc + 8 * u;  // 0..31
                const int at = a0 + ar;
#pragma unroll
                for (int h2 = 0; h2 < GT_C; h2 += 32) {
                    const int c = c0 + h2 + ta;
                    if (at < s && c < q) Gi[(size_t)at * smax + s0 + c] = gt[h2 + ta][ar];
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace

cudaError_t launch_gram_gather(const Dev& d, int ub, cudaStream_t s, int64_t* nl) {
    if (ub <= 0) return cudaSuccess;
    const cudaError_t e = launch_chain(k_gram_gather, dim3(ub), dim3(256), 0, s, d);
    if (e != cudaSuccess) return e;
    ++*nl;
    return cudaGetLastError();
}

cudaError_t launch_corr_q(const Dev& d, int cur, int act_n_ub, cudaStream_t s, int64_t* nl) {
    if (act_n_ub <= 0) return cudaSuccess;
    dim3 grid(act_n_ub, (d.m + 4 * QT - 1) / (4 * QT));
    const cudaError_t e = launch_chain(k_corr_q, grid, dim3(QT), 0, s, d, cur);
    if (e != cudaSuccess) return e;
    ++*nl;
    return cudaGetLastError();
}

cudaError_t launch_save_beta(const Dev& d, int cur, int act_n_ub, cudaStream_t s, int64_t* nl) {
    if (act_n_ub <= 0) return cudaSuccess;
    const cudaError_t e = launch_chain(k_save_beta, dim3(act_n_ub), dim3(256), 0, s, d, cur);
    if (e != cudaSuccess) return e;
    ++*nl;
    return cudaGetLastError();
}

// Q = A^T A (m x m, row k = A^T a_k) by the FP32 correlation kernel with the
// atoms as its residuals.  act (m ints) and cnt are scratch.
cudaError_t build_gram_q(const float* A32, int n, int m, float* Q, int* act, Counters* cnt, cudaStream_t s,
                         int64_t* nl) {
    k_gram_q_prep<<<(m + 255) / 256, 256, 0, s>>>(cnt, act, m);
    ++*nl;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    Dev d{};
    d.n = n;
    d.m = m;
    d.p = m;
    d.A32 = A32;
    d.R32 = const_cast<float*>(A32);  // read only
    d.Cs = Q;
    d.act[0] = act;
    d.cnt = cnt;
    return launch_corr_f32(d, 0, m, s, nl);
}

}  // namespace mpl
