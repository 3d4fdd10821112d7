// Worst-case analysis of Algorithm 1 on the 5th-generation tensor
// cores: C = A^T R with BF16 operands and FP32 accumulation.
//
// Both operands are K-major rows in HBM: atoms A16 (m x n) and the compacted
// residuals R16c (act_n x n).  A persistent CTA walks output tiles of
// 128 atoms x BN signals.  Warp roles:
//   warp 0  TMA producer: 128B-swizzled K-slices of 64 elements of both
//           operands into a STAGES-deep shared-memory ring (mbarrier
//           expect-tx / complete-tx);
//   warp 1  allocates TMEM, one elected thread issues tcgen05.mma
//           (M = 128, N = BN, K = 16) into one of two TMEM accumulators and
//           commits to the ring's empty barriers and the accumulator's full
//           barrier;
//   warps 2-5  epilogue: tcgen05.ld of the accumulator (each warp its 32-lane
//           quarter = 32 atoms), coalesced FP32 stores of the score rows
//           C[k*m + j], then release the accumulator.
// Every mbarrier wait is bounded; on expiry the CTA records DERR_TIMEOUT and
// drains before it frees its TMEM: the producer waits (bounded) for every
// stage whose TMA loads it issued, the MMA thread commits to a drain barrier
// and waits (bounded) for the MMAs it issued, then the CTA deallocates and
// exits.  No cluster multicast is used.
#include <cuda.h>

#include "mpl_internal.cuh"

namespace mpl {

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;  // bf16 elements per K-slice = one 128-byte swizzle row
constexpr int TC_THREADS = 192;
constexpr uint64_t WAIT_LIMIT_NS = 4000000000ull;  // a wait gives up after 4 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

constexpr uint64_t DRAIN_LIMIT_NS = 1000000000ull;  // a drain wait gives up after 1 s

// Bounded wait for the phase with the given parity to complete.  Returns false
// on expiry (WAIT_LIMIT_NS) or when another role of the CTA has given up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const volatile int* abort_flag) {
    const uint32_t a = smem_u32(bar);
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255u) == 0u) {
            const uint64_t now = globaltimer_ns();
            if (it == 0) t0 = now;
            else if (now - t0 > WAIT_LIMIT_NS || *abort_flag) return false;
        }
    }
}

// Drain wait after a give-up: bounded by time only (the abort flag is already set).
__device__ __forceinline__ bool mbar_wait_drain(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255u) == 0u) {
            const uint64_t now = globaltimer_ns();
            if (it == 0) t0 = now;
            else if (now - t0 > DRAIN_LIMIT_NS) return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms
// 1024 bytes apart (SBO), version 1.
__device__ __forceinline__ uint64_t sdesc_sw128(const void* p) {
    const uint64_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (addr & 0x3FFFFull) >> 4;          // start address
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D f32, A/B bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int BN, int STAGES>
struct TcSmem {
    static constexpr int A_BYTES = TC_BM * TC_BK * 2;
    static constexpr int B_BYTES = BN * TC_BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int TOTAL = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
    static_assert((2 * STAGES + 5) * 8 + 8 <= 256, "barriers, TMEM slot and abort flag fit their area");
};

template <int BN, int STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_corr_bf16(Dev d, int cur, const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmR) {
    pdl_enter();
    using L = TcSmem<BN, STAGES>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * L::STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;  // the MMA thread's completion barrier after a give-up
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int act_n = d.cnt->act_n[cur];
    const int m = d.m, n = d.n;
    const int tiles_m = (m + TC_BM - 1) / TC_BM;
    const int tiles_n = (act_n + BN - 1) / BN;
    const int ntiles = tiles_m * tiles_n;
    const int nk = (n + TC_BK - 1) / TC_BK;
    constexpr int TMEM_COLS = 2 * BN;  // two accumulators

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int a = 0; a < 2; ++a) { mbar_init(&tfull[a], 1); mbar_init(&tempty[a], 4); }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    auto give_up = [&]() {
        *abort_flag = 1;
        atomicCAS(&d.cnt->err, 0, (int)DERR_TIMEOUT);
    };

    if (warp == 0) {
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmR)) : "memory");
            int stage = 0;
            uint32_t ph = 0;
            uint32_t armed = 0, armed_par = 0;  // stages with loads issued, and the phase they complete
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                const int tm = t / tiles_n, tn = t - tm * tiles_n;
                for (int kb = 0; kb < nk; ++kb) {
                    if (!mbar_wait(&empty[stage], ph ^ 1u, abort_flag)) { give_up(); break; }
                    uint8_t* sa = base + stage * L::STAGE_BYTES;
                    uint8_t* sb = sa + L::A_BYTES;
                    mbar_expect_tx(&full[stage], L::STAGE_BYTES);
                    tma_load_2d(sa, &tmA, &full[stage], kb * TC_BK, tm * TC_BM);
                    tma_load_2d(sb, &tmR, &full[stage], kb * TC_BK, tn * BN);
                    armed |= 1u << stage;
                    armed_par = (armed_par & ~(1u << stage)) | (ph << stage);
                    if (++stage == STAGES) { stage = 0; ph ^= 1u; }
                }
            }
            if (*abort_flag) {
                // no copy may still target this CTA's shared memory when it exits: wait for the
                // last phase armed on each stage (a consumed one returns at once)
                for (int st = 0; st < STAGES; ++st)
                    if (armed & (1u << st)) mbar_wait_drain(&full[st], (armed_par >> st) & 1u);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(TC_BM, BN);
            int stage = 0, it = 0;
            uint32_t ph = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++it) {
                const int acc = it & 1;
                const uint32_t aph = (uint32_t)((it >> 1) & 1);
                if (!mbar_wait(&tempty[acc], aph ^ 1u, abort_flag)) { give_up(); break; }
                fence_after();
                const uint32_t dt = tmem + (uint32_t)(acc * BN);
                bool ok = true;
                for (int kb = 0; kb < nk; ++kb) {
                    if (!mbar_wait(&full[stage], ph, abort_flag)) { give_up(); ok = false; break; }
                    fence_after();
                    uint8_t* sa = base + stage * L::STAGE_BYTES;
                    uint8_t* sb = sa + L::A_BYTES;
                    const uint64_t da = sdesc_sw128(sa), db = sdesc_sw128(sb);
#pragma unroll
                    for (int k = 0; k < TC_BK / 16; ++k) {
                        // advance 16 elements (32 bytes) along K inside the swizzle row
                        const uint64_t off = (uint64_t)((k * 32) >> 4);
                        mma_bf16(dt, da + off, db + off, idesc, (kb | k) ? 1u : 0u);
                    }
                    mma_commit(&empty[stage]);
                    if (++stage == STAGES) { stage = 0; ph ^= 1u; }
                }
                if (!ok) break;
                mma_commit(&tfull[acc]);
            }
            if (*abort_flag) {
                // every MMA this thread issued completes before the accumulators are freed
                mma_commit(drain);
                mbar_wait_drain(drain, 0);
            }
        }
    } else {
        // epilogue warps 2..5: TMEM lane quarter = warp % 4
        const int q = warp & 3;
        int it = 0;
        for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++it) {
            const int tm = t / tiles_n, tn = t - tm * tiles_n;
            const int acc = it & 1;
            const uint32_t aph = (uint32_t)((it >> 1) & 1);
            bool ok = true;
            if (lane == 0) ok = mbar_wait(&tfull[acc], aph, abort_flag);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) { if (lane == 0) give_up(); break; }
            fence_after();
            const int atom = tm * TC_BM + q * 32 + lane;
            const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN);
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float v[16];
                tmem_ld16(tbase + (uint32_t)c0, v);
                const int sig0 = tn * BN + c0;
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int k = sig0 + e;
                    if (k < act_n && atom < m) d.Cs[(size_t)k * m + atom] = v[e];
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
    static EncodeFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    }
    return fn;
}

cudaError_t encode_rows(CUtensorMap* map, const void* ptr, int rows, int n, int box_rows) {
    EncodeFn enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)n * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tile widths (signals per output tile) with their ring depths: the operand ring takes
// ~190 KB of shared memory in each, so one CTA per SM; the two accumulators take 2 BN of
// the 512 TMEM columns.
constexpr int TC_BN_LIST[3] = {64, 128, 256};
template <int BN> struct TcStages;
template <> struct TcStages<64> { static constexpr int v = 8; };
template <> struct TcStages<128> { static constexpr int v = 6; };
template <> struct TcStages<256> { static constexpr int v = 4; };

int bn_slot(int bn) { return bn == 64 ? 0 : (bn == 256 ? 2 : 1); }

template <int BN>
cudaError_t set_attr() {
    using L = TcSmem<BN, TcStages<BN>::v>;
    return cudaFuncSetAttribute(k_corr_bf16<BN, TcStages<BN>::v>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                L::TOTAL);
}

template <int BN>
cudaError_t launch_bn(const Dev& d, int cur, const CUtensorMap* maps, int act_n_ub, int sms, cudaStream_t s) {
    using L = TcSmem<BN, TcStages<BN>::v>;
    const int tiles = ((d.m + TC_BM - 1) / TC_BM) * ((act_n_ub + BN - 1) / BN);
    const int grid = tiles < sms ? tiles : sms;
    return launch_chain(k_corr_bf16<BN, TcStages<BN>::v>, dim3(grid), dim3(TC_THREADS), (size_t)L::TOTAL, s, d, cur,
                        maps[0], maps[1 + bn_slot(BN)]);
}

}  // namespace

cudaError_t corr_bf16_prepare(int n, int m, int pmax, const __nv_bfloat16* A16, const __nv_bfloat16* R16c,
                              void* tmap) {
    if ((n % 8) != 0 || !A16 || !R16c) return cudaErrorNotSupported;
    CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(tmap);
    cudaError_t e = encode_rows(&maps[0], A16, m, n, TC_BM);
    // one residual map per tile width (the box is the tile's rows)
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = encode_rows(&maps[1 + k], R16c, pmax, n, TC_BN_LIST[k]);
    return e;
}

cudaError_t prepare_corr_bf16() {
    static bool attr = false;
    if (attr) return cudaSuccess;
    cudaError_t e = set_attr<64>();
    if (e == cudaSuccess) e = set_attr<128>();
    if (e == cudaSuccess) e = set_attr<256>();
    if (e == cudaSuccess) attr = true;
    return e;
}

cudaError_t launch_corr_bf16(const Dev& d, int cur, const void* tmap, int act_n_ub, int sms, cudaStream_t s,
                             int64_t* nl, int bn) {
    if (act_n_ub <= 0) return cudaSuccess;
    if (gemv_route(d, act_n_ub)) return launch_corr_gemv(d, cur, act_n_ub, true, s, nl);
    cudaError_t ep = prepare_corr_bf16();
    if (ep != cudaSuccess) return ep;
    const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(tmap);
    const cudaError_t e = bn == 64    ? launch_bn<64>(d, cur, maps, act_n_ub, sms, s)
                          : bn == 256 ? launch_bn<256>(d, cur, maps, act_n_ub, sms, s)
                                      : launch_bn<128>(d, cur, maps, act_n_ub, sms, s);
    if (e != cudaSuccess) return e;
    ++*nl;
    return cudaGetLastError();
}

}  // namespace mpl
