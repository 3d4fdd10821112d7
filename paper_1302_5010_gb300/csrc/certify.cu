// Exact finish and certificate of a master problem (eq. "primal_MPL").
//
// When a signal has no violator left, its FP32 proximal-gradient iterate u is
// driven to the exact restricted minimiser by an active-set method on the
// Gram block (the optimality conditions of the dual eq. 5 restricted to S):
//
//   P = supp(x), s = sign(x_P); solve G_PP z = h_P - lambda*s_P (FP64 Cholesky);
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
// FP64 rate is a small fraction of its FP32 rate; the factorisation and the
// small triangular solves stay in FP64.  The certified KKT violation on S and
// the exact residual (FP32 hi/lo pair and FP64) are stored; the next
// worst-case analysis certifies the atoms outside S (eq. 8).
//
// One CTA per signal.  Shared memory is sized by the host from its bound on
// |S|; the FP64 factor lives in shared memory up to FIN_SMEM_P atoms and in a
// global FP64 workspace beyond.
#include "mpl_internal.cuh"

namespace mpl {

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

struct FinShared {
    double* M;   // factor (shared or global), ld
    double* x;   // current point on S (position-indexed)
    double* z;   // solve result on P
    double* w;   // scratch on P / S
    int* P;      // support positions
    int* sg;     // sign per position of S
    int* Pi;     // atom index of each support position
    double red[32];
    int ival[4];
    double dval[4];
};

// In-place FP64 Cholesky (lower) of the np x np block M.  0 or -1 on a
// non-positive pivot.
__device__ int chol(double* M, int ld, int np, FinShared& sh) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = 0; j < np; ++j) {
        if (tid == 0) {
            const double dj = M[(size_t)j * ld + j];
            sh.ival[0] = (dj > 0.0) ? 0 : 1;
            M[(size_t)j * ld + j] = dj > 0.0 ? sqrt(dj) : 1.0;
        }
        __syncthreads();
        if (sh.ival[0]) return -1;
        const double inv = 1.0 / M[(size_t)j * ld + j];
        for (int r = j + 1 + tid; r < np; r += nt) M[(size_t)r * ld + j] *= inv;
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

// Solve (L L^T) v = v in place.
__device__ void chol_solve(const double* M, int ld, int np, double* v) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = 0; j < np; ++j) {
        if (tid == 0) v[j] /= M[(size_t)j * ld + j];
        __syncthreads();
        const double vj = v[j];
        for (int r = j + 1 + tid; r < np; r += nt) v[r] -= M[(size_t)r * ld + j] * vj;
        __syncthreads();
    }
    for (int j = np - 1; j >= 0; --j) {
        if (tid == 0) v[j] /= M[(size_t)j * ld + j];
        __syncthreads();
        const double vj = v[j];
        for (int r = tid; r < j; r += nt) v[r] -= M[(size_t)j * ld + r] * vj;
        __syncthreads();
    }
}

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

__global__ void __launch_bounds__(FIN_THREADS) k_finish(Dev d, int scap, int msm) {
    const int g = blockIdx.x;
    if (g >= d.cnt->fin_n) return;
    const int i = d.list_fin[g];
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
        sh.M = msm ? p : d.chol + (size_t)i * smax * smax;
        if (msm) p += (size_t)scap * scap;
        sh.x = p; p += scap;
        sh.z = p; p += scap;
        sh.w = p; p += scap;
        sh.P = reinterpret_cast<int*>(p);
        sh.sg = sh.P + scap;
        sh.Pi = sh.sg + scap;
    }
    __syncthreads();
    const int ld = msm ? scap : smax;
    const double lam = (double)d.lam[i];
    const double tol = d.tol;
    const int* Si = d.S + (size_t)i * smax;
    const float* Gi = d.G + (size_t)i * smax * smax;
    const float* hi = d.h + (size_t)i * smax;
    float* xS = d.xS + (size_t)i * smax;
    const float* b = d.B + (size_t)i * n;
    float* rh = d.R32 + (size_t)i * n;   // residual, high part
    float* rl = d.R32lo + (size_t)i * n; // residual, low part

    for (int a = tid; a < s; a += nt) {
        const float v = xS[a];
        sh.x[a] = (double)v;
        sh.sg[a] = v > 0.f ? 1 : (v < 0.f ? -1 : 0);
    }
    __syncthreads();

    bool ok = false;
    double kkt_on = 0.0, cmax_s = 0.0;
    int np = 0;
    const int max_steps = 4 * s + 16;
    for (int step = 0; step < max_steps; ++step) {
        np = build_support(s, sh);
        // ---- solve on P
        if (np > 0) {
            for (int e = tid; e < np * np; e += nt) {
                const int r = e / np, c = e - r * np;
                sh.M[(size_t)r * ld + c] = (double)Gi[(size_t)sh.P[r] * smax + sh.P[c]];
            }
            for (int a = tid; a < np; a += nt) sh.z[a] = (double)hi[sh.P[a]] - lam * (double)sh.sg[sh.P[a]];
            __syncthreads();
            if (chol(sh.M, ld, np, sh) != 0) break;
            chol_solve(sh.M, ld, np, sh.z);
        }
        // ---- first sign crossing on the segment x -> z
        if (tid == 0) { sh.dval[1] = 2.0; sh.ival[2] = -1; }
        __syncthreads();
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
        __syncthreads();
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
            continue;
        }
        // consistent: x <- z on P (zero elsewhere)
        for (int a = tid; a < s; a += nt) if (sh.sg[a] == 0) sh.x[a] = 0.0;
        __syncthreads();
        for (int a = tid; a < np; a += nt) sh.x[sh.P[a]] = sh.z[a];
        __syncthreads();
        // ---- zero entries of S through the Gram block: add the largest violator
        if (tid == 0) { sh.dval[2] = 0.0; sh.ival[3] = -1; }
        __syncthreads();
        for (int a = warp; a < s; a += nw) {
            if (sh.sg[a] != 0) continue;
            double acc = 0.0;
            for (int c = lane; c < np; c += 32)
                acc += (double)Gi[(size_t)a * smax + sh.P[c]] * sh.x[sh.P[c]];
#pragma unroll
            for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            const double ca = (double)hi[a] - acc;
            if (lane == 0 && fabs(ca) > lam * (1.0 + 0.5 * tol)) {
                // largest |c|, ties to the lowest position
                unsigned long long key = ((unsigned long long)__double_as_longlong(fabs(ca)) & ~0xFFFull) |
                                         (unsigned long long)(0xFFF - a);
                atomicMax(reinterpret_cast<unsigned long long*>(&sh.dval[2]), key);
            }
        }
        __syncthreads();
        if (sh.dval[2] != 0.0) {
            const unsigned long long key = (unsigned long long)__double_as_longlong(sh.dval[2]);
            const int a = 0xFFF - (int)(key & 0xFFFull);
            if (tid == 0) {
                double acc = 0.0;
                for (int c = 0; c < np; ++c) acc += (double)Gi[(size_t)a * smax + sh.P[c]] * sh.x[sh.P[c]];
                sh.sg[a] = ((double)hi[a] - acc) > 0.0 ? 1 : -1;
            }
            __syncthreads();
            continue;
        }
        // ---- exact verification: r = b - A_P x, c = A^T r (double-FP32), Newton refinement on P
        double dmax = 0.0;
        df* xd = reinterpret_cast<df*>(sh.z);  // z is free now: x_P split into FP32 pairs
        for (int a = tid; a < np; a += nt) sh.Pi[a] = Si[sh.P[a]];
        for (int ref = 0; ref < 5; ++ref) {
            for (int a = tid; a < np; a += nt) xd[a] = to_df(sh.x[sh.P[a]]);
            __syncthreads();
            for (int k = tid; k < n; k += nt) {
                df acc = {b[k], 0.f};
                for (int a = 0; a < np; ++a)
                    acc = df_fma(acc, -__ldg(d.A32 + (size_t)sh.Pi[a] * n + k), xd[a]);
                rh[k] = acc.hi;
                rl[k] = acc.lo;
            }
            __syncthreads();
            double lmax = 0.0;
            for (int a = warp; a < np; a += nw) {
                const float* aj = d.A32 + (size_t)sh.Pi[a] * n;
                df acc = {0.f, 0.f};
                for (int k = lane; k < n; k += 32) {
                    const float av = __ldg(aj + k);
                    acc = df_fma(acc, av, df{rh[k], rl[k]});
                }
                acc = warp_df_sum(acc);
                const double dv = to_d(acc) - lam * (double)sh.sg[sh.P[a]];
                if (lane == 0) sh.w[a] = dv;
                lmax = fmax(lmax, fabs(dv));
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
            __syncthreads();
            if (lane == 0) sh.red[warp] = lmax;
            __syncthreads();
            dmax = 0.0;
            for (int q = 0; q < nw; ++q) dmax = fmax(dmax, sh.red[q]);
            if (np == 0 || dmax <= 1e-3 * tol * lam || ref == 4) break;
            chol_solve(sh.M, ld, np, sh.w);
            for (int a = tid; a < np; a += nt) sh.x[sh.P[a]] += sh.w[a];
            __syncthreads();
        }
        // on exit w holds c_P - lambda*s_P of the last evaluated residual
        // sign consistency after refinement
        if (tid == 0) sh.ival[0] = 0;
        __syncthreads();
        for (int a = tid; a < np; a += nt) {
            const int pa = sh.P[a];
            if (!(sh.x[pa] * (double)sh.sg[pa] > 0.0)) { sh.sg[pa] = 0; sh.x[pa] = 0.0; sh.ival[0] = 1; }
        }
        __syncthreads();
        if (sh.ival[0]) continue;
        // exact check of the zero entries of S
        double cmax = 0.0;
        int worst = -1;
        double worst_c = 0.0;
        for (int a = warp; a < s; a += nw) {
            if (sh.sg[a] != 0) continue;
            const float* aj = d.A32 + (size_t)Si[a] * n;
            df acc = {0.f, 0.f};
            for (int k = lane; k < n; k += 32) acc = df_fma(acc, __ldg(aj + k), df{rh[k], rl[k]});
            acc = warp_df_sum(acc);
            const double ca = to_d(acc);
            if (fabs(ca) > cmax) { cmax = fabs(ca); worst = a; worst_c = ca; }
        }
        if (tid == 0) { sh.dval[3] = 0.0; sh.ival[3] = -1; }
        __syncthreads();
        if (lane == 0 && worst >= 0 && cmax > lam * (1.0 + tol)) {
            unsigned long long key = ((unsigned long long)__double_as_longlong(cmax) & ~0xFFFull) |
                                     (unsigned long long)(0xFFF - worst);
            atomicMax(reinterpret_cast<unsigned long long*>(&sh.dval[3]), key);
            (void)worst_c;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
        __syncthreads();
        if (lane == 0) sh.red[warp] = cmax;
        __syncthreads();
        cmax_s = 0.0;
        for (int q = 0; q < nw; ++q) cmax_s = fmax(cmax_s, sh.red[q]);
        if (sh.dval[3] != 0.0) {
            const unsigned long long key = (unsigned long long)__double_as_longlong(sh.dval[3]);
            const int a = 0xFFF - (int)(key & 0xFFFull);
            // sign of the exact correlation of the entering atom
            if (warp == 0) {
                const float* aj = d.A32 + (size_t)Si[a] * n;
                df acc = {0.f, 0.f};
                for (int k = lane; k < n; k += 32) acc = df_fma(acc, __ldg(aj + k), df{rh[k], rl[k]});
                acc = warp_df_sum(acc);
                if (lane == 0) sh.sg[a] = to_d(acc) > 0.0 ? 1 : -1;
            }
            __syncthreads();
            continue;
        }
        kkt_on = fmax(dmax / lam, fmax(cmax_s - lam, 0.0) / lam);
        ok = kkt_on <= tol;
        break;
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
        double rr = 0.0, rb = 0.0, rs = 0.0;
        for (int k = tid; k < n; k += nt) {
            const double v = (double)rh[k] + (double)rl[k];
            r64[k] = v;
            if (d.R16) d.R16[(size_t)i * n + k] = __float2bfloat16_rn(rh[k]);
            rr += v * v;
            rb += v * (double)b[k];
            rs += (double)rh[k] * (double)rh[k];
        }
        const double L1 = bsum(l1, sh.red);
        const double RR = bsum(rr, sh.red);
        const double RB = bsum(rb, sh.red);
        const double RS = bsum(rs, sh.red);
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
            d.kkt_in[i] = kkt_on;
            d.ginf[i] = fmax(CM, cmax_s);
            d.nnz[i] = np;
            d.finalized[i] = 1;
            d.fails[i] = 0;
            d.finishes[i] += 1;
        }
    } else {
        // keep the (monotonically improved) point as the next warm start
        for (int a = tid; a < s; a += nt) xS[a] = (float)sh.x[a];
        __syncthreads();
        if (tid == 0) {
            d.finalized[i] = 0;
            d.finishes[i] += 1;
            const int f = ++d.fails[i];
            if (f >= FIN_MAX_FAILS) {
                d.state[i] = ST_DONE;
                d.sstatus[i] = MPL_SIG_UNCERTIFIED;
            } else {
                d.eps[i] = fmaxf(d.eps[i] * 1e-2f, 1e-7f);
                const int pos = atomicAdd(&d.cnt->apg_n, 1);
                d.list_apg[pos] = i;
            }
        }
    }
}

}  // namespace

cudaError_t launch_finish(const Dev& d, int ub, int scap, cudaStream_t s, int64_t* nl) {
    if (ub <= 0) return cudaSuccess;
    scap = ((scap + 31) / 32) * 32;
    if (scap > d.smax) scap = d.smax;
    const int msm = scap <= FIN_SMEM_P ? 1 : 0;
    const size_t dyn = ((msm ? (size_t)scap * scap : 0) + 3 * (size_t)scap) * sizeof(double) +
                       3 * (size_t)scap * sizeof(int);
    static bool attr = false;
    if (!attr) {
        const int mx = (int)(((size_t)FIN_SMEM_P * FIN_SMEM_P + 3 * 1024) * sizeof(double) + 3 * 1024 * sizeof(int));
        cudaError_t e = cudaFuncSetAttribute(k_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_finish<<<ub, FIN_THREADS, dyn, s>>>(d, scap, msm);
    ++*nl;
    return cudaGetLastError();
}

}  // namespace mpl
