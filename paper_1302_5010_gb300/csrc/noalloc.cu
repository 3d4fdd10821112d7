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
// with cudaGetSymbolAddress and cached.  That first call should therefore come
// before any stream capture.  All calls share the one array, so two calls whose
// work overlaps on the GPU race on it; issue them on one stream, or wait for
// one to finish before starting the next.
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

// Identity column list and fresh counters for one call (everything the
// correlation kernel reads from scratch is rewritten here).
__global__ void k_noalloc_prep(Counters* cnt, int* act, int p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < p) act[i] = i;
    if (i == 0) {
        cnt->act_n[0] = p;
        cnt->act_n[1] = 0;
        cnt->grow_n = cnt->fin_n = cnt->apg_n = cnt->apg_head = 0;
        cnt->err = 0;
        cnt->sel_fallback = 0;
    }
}

bool device_accessible(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace mpl

using namespace mpl;

extern "C" mpl_status_t mpl_correlate_noalloc(const float* A, int n, int m, const float* R, int p, float* C,
                                              void* stream) {
    if (n < 1 || n > 65536 || m < 1 || p < 0) return MPL_ERR_ARG;
    if (p > MPL_NOALLOC_MAX_SIGNALS) return MPL_ERR_UNSUPPORTED;
    if (p == 0) return MPL_OK;
    if (!A || !R || !C) return MPL_ERR_ARG;
    if (!device_accessible(A) || !device_accessible(R) || !device_accessible(C)) return MPL_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return MPL_ERR_CUDA;
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return MPL_ERR_CUDA;
            }
            g_noalloc_addr[dev] = ptr;
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
