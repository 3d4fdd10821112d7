// mpl_correlate_noalloc: the FP32 correlation g_i = A^T r_i for callers that
// cannot allocate device memory.
//
// Who needs it: applications whose device memory is owned up front by their
// own pool allocator (a framework's caching allocator, a serving runtime with a
// fixed memory budget).  For them a library that calls cudaMalloc on its own
// is a problem: the call can fail once the pool has reserved the memory, and it
// synchronises the device in the middle of their pipeline.  This entry point
// takes every input and output from the caller and keeps its small scratch
// (the list of signal columns and the work counters read by the correlation
// kernel) in a file-scope device array, so it never allocates.
//
// The array lives in every GPU that loads the library until the process
// exits.  Host code cannot use the array's name as a device address: on the
// first call on each device (with that device current) the address is fetched
// with cudaGetSymbolAddress and cached together with the CUDA context it
// belongs to; a call that finds another context current (the old one was torn
// down by cudaDeviceReset, or the caller switched contexts) fetches it again.
// The first call on a device, and the first after such a change, should come
// before any stream capture.  All calls share the one array, so two calls whose
// work overlaps on the GPU race on it; issue them on one stream, or wait for
// one to finish before starting the next.
//
// The caller's pointers must be device memory of the current device, 16-byte
// aligned (the kernel reads A and R, and writes C, as float4 rows when n, m
// are multiples of 4); anything else is refused with MPL_ERR_ARG before a
// launch.
#include <cuda.h>

#include <cstdint>
#include <mutex>

#include "mpl_internal.cuh"

namespace mpl {

namespace {

constexpr size_t NOALLOC_HEADER = 256;  // Counters, padded
static_assert(sizeof(Counters) <= NOALLOC_HEADER, "counters must fit the scratch header");
static_assert(NOALLOC_HEADER + 4ull * MPL_NOALLOC_MAX_SIGNALS <= MPL_NOALLOC_SCRATCH_BYTES, "scratch too small");
static __device__ __align__(256) unsigned char g_noalloc_scratch[MPL_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[MAX_DEVICES] = {nullptr};
CUcontext g_noalloc_ctx[MAX_DEVICES] = {nullptr};  // context the cached address belongs to

// The current driver context, through the runtime's driver entry point (no libcuda link).
CUcontext current_context() {
    using GetCtx = CUresult (*)(CUcontext*);
    static GetCtx fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        fn = reinterpret_cast<GetCtx>(p);
    }
    CUcontext c = nullptr;
    return fn(&c) == CUDA_SUCCESS ? c : nullptr;
}

// Identity column list and fresh counters for one call (everything the
// correlation kernel reads from scratch is rewritten here).
__global__ void k_noalloc_prep(Counters* cnt, int* act, int p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < p) act[i] = i;
    if (i == 0) {
        cnt->act_n[0] = p;
        cnt->act_n[1] = 0;
        cnt->grow_n = cnt->fin_n = cnt->apg_n = cnt->apg_head = cnt->apg_head2 = 0;
        cnt->err = 0;
        cnt->sel_fallback = 0;
    }
}

// Device (or managed) memory that the current device can address directly: memory of
// another GPU would need peer access, which this call does not set up.
bool device_accessible(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

}  // namespace mpl

using namespace mpl;

extern "C" mpl_status_t mpl_correlate_noalloc(const float* A, int n, int m, const float* R, int p, float* C,
                                              void* stream) {
    if (n < 1 || n > 65536 || m < 1 || m > (1 << 26) || p < 0) return MPL_ERR_ARG;
    if (p > MPL_NOALLOC_MAX_SIGNALS) return MPL_ERR_UNSUPPORTED;
    if (p == 0) return MPL_OK;
    if (!A || !R || !C) return MPL_ERR_ARG;
    if (!aligned16(A) || !aligned16(R) || !aligned16(C)) return MPL_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return MPL_ERR_CUDA;
    if (!device_accessible(A, dev) || !device_accessible(R, dev) || !device_accessible(C, dev)) return MPL_ERR_ARG;
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        const CUcontext ctx = current_context();
        if (!g_noalloc_addr[dev] || ctx != g_noalloc_ctx[dev]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return MPL_ERR_CUDA;
            }
            g_noalloc_addr[dev] = ptr;
            g_noalloc_ctx[dev] = current_context();
        }
        base = g_noalloc_addr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Counters* cnt = static_cast<Counters*>(base);
    int* act = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + NOALLOC_HEADER);
    k_noalloc_prep<<<(p + 255) / 256, 256, 0, st>>>(cnt, act, p);
    if (cudaGetLastError() != cudaSuccess) return MPL_ERR_CUDA;
    Dev d{};
    d.n = n;
    d.m = m;
    d.p = p;
    d.A32 = A;
    d.R32 = const_cast<float*>(R);  // read only
    d.Cs = C;
    d.act[0] = act;
    d.cnt = cnt;
    int64_t nl = 0;
    if (launch_corr_f32(d, 0, p, st, &nl) != cudaSuccess) return MPL_ERR_CUDA;
    return MPL_OK;
}
