// Exact finish and FP64 certificate of a master problem (eq. "primal_MPL").
//
// When a signal has no violator left, its FP32 proximal-gradient iterate u
// fixes a sign pattern s on P = supp(u).  The optimality conditions of the
// restricted LASSO (the dual eq. 5 restricted to S) then read
//     A_P^T (b - A_P z) = lambda * s_P,        |a_j^T (b - A_P z)| <= lambda, j in S \ P,
// and sign(z) = s_P.  The kernel solves G_PP z = h_P - lambda*s_P with an FP64
// Cholesky factor of the Gram block, refines z with FP64 residuals
// r = b - A_P z (the Gram block itself is only FP32-accurate, the residuals
// are exact to FP64 rounding), and pivots: entries whose sign disagrees leave
// P, zero entries of S that violate their bound join it.  On success the
// on-support KKT violation (in FP64) and the FP64 residual are stored; the next
// worst-case analysis then certifies the atoms outside S (eq. 8).
//
// One CTA per signal; the factor lives in shared memory up to FIN_SMEM_P
// atoms and in a global FP64 workspace beyond.
#include "mpl_internal.cuh"

namespace mpl {

namespace {

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

__device__ __forceinline__ double bmax(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t = fmax(t, red[w]);
    return t;
}

struct FinSmem {
    double M[FIN_SMEM_P * FIN_SMEM_P];
    double z[1024];
    double w[1024];
    double c[1024];
    int P[1024];      // positions (in S) of the support
    int sg[1024];     // sign pattern per position in S (-1, 0, +1)
    double red[32];
    int flag;
    int np;
};

// In-place Cholesky (lower) of the np x np block M (row-major, ld).  Returns 0
// or -1 on a non-positive pivot.
__device__ int chol(double* M, int ld, int np, FinSmem& sh) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = 0; j < np; ++j) {
        if (tid == 0) {
            const double dj = M[(size_t)j * ld + j];
            sh.flag = (dj > 0.0) ? 0 : 1;
            M[(size_t)j * ld + j] = dj > 0.0 ? sqrt(dj) : 1.0;
        }
        __syncthreads();
        if (sh.flag) return -1;
        const double dj = M[(size_t)j * ld + j];
        for (int r = j + 1 + tid; r < np; r += nt) M[(size_t)r * ld + j] /= dj;
        __syncthreads();
        const int rem = np - j - 1;
        for (int e = tid; e < rem * rem; e += nt) {
            const int r = j + 1 + e / rem, c = j + 1 + e % rem;
            if (c <= r) M[(size_t)r * ld + c] -= M[(size_t)r * ld + j] * M[(size_t)c * ld + j];
        }
        __syncthreads();
    }
    return 0;
}

// Solve (L L^T) x = x in place (x in shared memory).
__device__ void chol_solve(const double* M, int ld, int np, double* x) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = 0; j < np; ++j) {  // forward, column-oriented
        if (tid == 0) x[j] /= M[(size_t)j * ld + j];
        __syncthreads();
        const double xj = x[j];
        for (int r = j + 1 + tid; r < np; r += nt) x[r] -= M[(size_t)r * ld + j] * xj;
        __syncthreads();
    }
    for (int j = np - 1; j >= 0; --j) {  // backward with L^T
        if (tid == 0) x[j] /= M[(size_t)j * ld + j];
        __syncthreads();
        const double xj = x[j];
        for (int r = tid; r < j; r += nt) x[r] -= M[(size_t)j * ld + r] * xj;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(FIN_THREADS) k_finish(Dev d) {
    const int g = blockIdx.x;
    if (g >= d.cnt->fin_n) return;
    const int i = d.list_fin[g];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FinSmem& sh = *reinterpret_cast<FinSmem*>(smem_raw);
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int n = d.n, smax = d.smax, s = d.ssize[i];
    const double lam = (double)d.lam[i];
    const double tol = d.tol;
    const int* Si = d.S + (size_t)i * smax;
    const float* Gi = d.G + (size_t)i * smax * smax;
    const float* hi = d.h + (size_t)i * smax;
    const float* xi = d.xS + (size_t)i * smax;
    const float* b = d.B + (size_t)i * n;
    double* r64 = d.R64 + (size_t)i * n;

    for (int a = tid; a < s; a += nt) {
        const float v = xi[a];
        sh.sg[a] = v > 0.f ? 1 : (v < 0.f ? -1 : 0);
    }
    __syncthreads();

    bool ok = false;
    double kkt_on = 0.0, zmax_c = 0.0;
    int np = 0;
    for (int piv = 0; piv < FIN_MAX_PIVOTS; ++piv) {
        // support positions in S order
        if (tid == 0) {
            int c = 0;
            for (int a = 0; a < s; ++a)
                if (sh.sg[a] != 0) sh.P[c++] = a;
            sh.np = c;
        }
        __syncthreads();
        np = sh.np;
        double* M = (np <= FIN_SMEM_P) ? sh.M : d.chol + (size_t)i * smax * smax;
        const int ld = (np <= FIN_SMEM_P) ? FIN_SMEM_P : smax;
        for (int e = tid; e < np * np; e += nt) {
            const int r = e / np, c = e - r * np;
            M[(size_t)r * ld + c] = (double)Gi[(size_t)sh.P[r] * smax + sh.P[c]];
        }
        for (int a = tid; a < np; a += nt) sh.z[a] = (double)hi[sh.P[a]] - lam * (double)sh.sg[sh.P[a]];
        __syncthreads();
        if (np > 0 && chol(M, ld, np, sh) != 0) break;
        if (np > 0) chol_solve(M, ld, np, sh.z);
        // FP64 residual refinement: z += G^{-1} (A_P^T r - lambda s_P)
        double dmax = 0.0;
        for (int ref = 0; ref < 4; ++ref) {
            for (int k = tid; k < n; k += nt) {
                double acc = (double)b[k];
                for (int a = 0; a < np; ++a)
                    acc = fma(-(double)__ldg(d.A32 + (size_t)Si[sh.P[a]] * n + k), sh.z[a], acc);
                r64[k] = acc;
            }
            __syncthreads();
            double lmax = 0.0;
            for (int a = warp; a < np; a += nw) {
                const float* aj = d.A32 + (size_t)Si[sh.P[a]] * n;
                double acc = 0.0;
                for (int k = lane; k < n; k += 32) acc = fma((double)__ldg(aj + k), r64[k], acc);
#pragma unroll
                for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                const double dv = acc - lam * (double)sh.sg[sh.P[a]];
                if (lane == 0) { sh.w[a] = dv; sh.c[a] = acc; }
                lmax = fmax(lmax, fabs(dv));
            }
            dmax = bmax(lmax, sh.red);
            if (np == 0 || dmax <= 1e-3 * tol * lam || ref == 3) break;
            chol_solve(M, ld, np, sh.w);
            for (int a = tid; a < np; a += nt) sh.z[a] += sh.w[a];
            __syncthreads();
        }
        // sign consistency: entries that disagree with their pattern leave P
        if (tid == 0) sh.flag = 0;
        __syncthreads();
        for (int a = tid; a < np; a += nt) {
            if (!(sh.z[a] * (double)sh.sg[sh.P[a]] > 0.0)) {
                sh.sg[sh.P[a]] = 0;
                sh.flag = 1;
            }
        }
        __syncthreads();
        if (sh.flag) continue;
        // zero entries of S: |a_j^T r| <= lambda(1+tol), else they join P
        double cmax = 0.0;
        for (int a = warp; a < s; a += nw) {
            if (sh.sg[a] != 0) continue;
            const float* aj = d.A32 + (size_t)Si[a] * n;
            double acc = 0.0;
            for (int k = lane; k < n; k += 32) acc = fma((double)__ldg(aj + k), r64[k], acc);
#pragma unroll
            for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            cmax = fmax(cmax, fabs(acc));
            if (lane == 0 && fabs(acc) > lam * (1.0 + tol)) {
                sh.sg[a] = acc > 0.0 ? 2 : -2;  // marked, turned into +-1 below
            }
        }
        zmax_c = bmax(cmax, sh.red);
        if (tid == 0) {
            int added = 0;
            for (int a = 0; a < s; ++a)
                if (sh.sg[a] == 2 || sh.sg[a] == -2) { sh.sg[a] /= 2; ++added; }
            sh.flag = added;
        }
        __syncthreads();
        if (sh.flag) continue;
        kkt_on = fmax(dmax / lam, fmax(zmax_c - lam, 0.0) / lam);
        ok = kkt_on <= tol;
        break;
    }

    // outcome
    if (ok) {
        double* x64 = d.xS64 + (size_t)i * smax;
        float* xf = d.xS + (size_t)i * smax;
        for (int a = tid; a < s; a += nt) { x64[a] = 0.0; xf[a] = 0.f; }
        __syncthreads();
        double l1 = 0.0, cm = 0.0;
        for (int a = tid; a < np; a += nt) {
            const double v = sh.z[a];
            x64[sh.P[a]] = v;
            xf[sh.P[a]] = (float)v;
            l1 += fabs(v);
            cm = fmax(cm, fabs(sh.c[a]));
        }
        float* r32 = d.R32 + (size_t)i * n;
        double rr = 0.0, rb = 0.0;
        float rs = 0.f;
        for (int k = tid; k < n; k += nt) {
            const double v = r64[k];
            const float vf = (float)v;
            r32[k] = vf;
            if (d.R16) d.R16[(size_t)i * n + k] = __float2bfloat16_rn(vf);
            rr += v * v;
            rb += v * (double)b[k];
            rs = fmaf(vf, vf, rs);
        }
        const double L1 = bsum(l1, sh.red);
        const double RR = bsum(rr, sh.red);
        const double RB = bsum(rb, sh.red);
        const double RS = bsum((double)rs, sh.red);
        const double CM = bmax(cm, sh.red);
        if (tid == 0) {
            d.obj[i] = lam * L1 + 0.5 * RR;
            d.rr[i] = RR;
            d.rb[i] = RB;
            d.rnorm[i] = (float)(sqrt(RS) * (1.0 + 1e-5));
            d.kkt_in[i] = kkt_on;
            d.ginf[i] = fmax(CM, zmax_c);
            d.nnz[i] = np;
            d.finalized[i] = 1;
            d.fails[i] = 0;
            d.finishes[i] += 1;
        }
    } else if (tid == 0) {
        d.finalized[i] = 0;
        d.finishes[i] += 1;
        const int f = ++d.fails[i];
        if (f >= FIN_MAX_FAILS) {
            d.state[i] = ST_DONE;
            d.sstatus[i] = MPL_SIG_UNCERTIFIED;
        } else {
            // more proximal-gradient work on the same set, with a tighter eq. (inner)
            d.eps[i] = fmaxf(d.eps[i] * 1e-2f, 1e-7f);
            const int pos = atomicAdd(&d.cnt->apg_n, 1);
            d.list_apg[pos] = i;
        }
    }
}

}  // namespace

cudaError_t launch_finish(const Dev& d, int ub, cudaStream_t s, int64_t* nl) {
    if (ub <= 0) return cudaSuccess;
    const size_t sm = sizeof(FinSmem);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_finish<<<ub, FIN_THREADS, sm, s>>>(d);
    ++*nl;
    return cudaGetLastError();
}

}  // namespace mpl
