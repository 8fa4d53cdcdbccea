// pic_sort_keys_noalloc: the library's counting sort (histogram, single-pass
// scan, scatter) on caller arrays, for callers that cannot allocate device
// memory.  Its scratch (per-bin counts, the scan's look-back words and an
// error word) lives in one file-scope static __device__ array; the call
// allocates nothing.  The histogram and scan kernels are the ones pic_step
// runs (pic_sort.cu, constants in pic_sort.cuh); only the scatter of a
// permutation is specific to this entry point.
#include <cuda.h>  // CUcontext (the type only: cuCtxGetCurrent is reached through the runtime)
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "pic_ctx.h"
#include "pic_device.cuh"
#include "pic_sort.cuh"

namespace pic {

// message reported by pic_last_error() (pic_api.cu)
void set_last_error(const std::string& msg);

namespace {

constexpr int kBlockNA = kSortBlock;
constexpr int64_t kMaxBins = int64_t(1) << 22;
constexpr int64_t kMaxChunks = kMaxBins / kScanChunk;
static_assert(kMaxBins % kScanChunk == 0, "the bin limit is a whole number of scan chunks");

// layout: [error words: 4 x u32 = 16 B][pad to 256 B]
//         [look-back words + ticket: (kMaxChunks + 1) x u64]
//         [counts: kMaxBins x i32]
constexpr size_t kErrBytes = 256;
constexpr size_t kStatusBytes = size_t(kMaxChunks + 1) * sizeof(unsigned long long);
constexpr size_t kStatusPadded = (kStatusBytes + 255) / 256 * 256;
constexpr size_t kScratchBytes = kErrBytes + kStatusPadded + size_t(kMaxBins) * sizeof(int);

// Every GPU that loads the library holds this array (about 16 MiB) until
// the process exits.  Host code must not use its name as an address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
CUcontext g_scratch_ctx[kMaxDevices] = {nullptr};  // the context each address belongs to

__device__ __forceinline__ unsigned lanemask_lt_na() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// perm[dest] = p for every key, dest in its bin's range [offsets[k], offsets[k+1]);
// count[k] is decremented back to zero.
__global__ void __launch_bounds__(kBlockNA) k_perm_scatter(const int* __restrict__ key, int64_t n,
                                                           const int* __restrict__ offsets, int* count, int64_t nbins,
                                                           int* perm) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int k = -1;
    if (p < n) {
        k = key[p];
        if (k < 0 || k >= nbins) k = -1;
    }
    const unsigned mask = __match_any_sync(0xffffffffu, k);
    if (k < 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    const int ng = __popc(mask);
    int old = 0;
    if (lane == leader) old = atomicSub(count + k, ng);
    old = __shfl_sync(mask, old, leader);
    const int dest = offsets[k] + (old - ng) + __popc(mask & lanemask_lt_na());
    if (dest >= 0 && dest < n) perm[dest] = int(p);
}

// The calling thread's current CUDA context (null if the driver entry point is
// unavailable): a device reset or a new primary context loads the module again
// and can move the scratch array, so its address is looked up again whenever
// the context differs from the one it was taken in.
CUcontext current_context() {
    using Fn = CUresult (*)(CUcontext*);
    static Fn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<Fn>(p);
    }();
    CUcontext ctx = nullptr;
    if (!fn || fn(&ctx) != CUDA_SUCCESS) return nullptr;
    return ctx;
}

// Device address of the scratch array for the current device: looked up with
// cudaGetSymbolAddress on the first call per device (that device current), and
// again after the device's context has changed.
cudaError_t scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    const CUcontext ctx = current_context();
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev] || (ctx && ctx != g_scratch_ctx[dev])) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = ptr;
        g_scratch_ctx[dev] = current_context();  // the lookup may have created the primary context
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return cudaSuccess;
}

pic_status na_fail(pic_status s, const std::string& msg) {
    set_last_error(msg);
    return s;
}

}  // namespace
}  // namespace pic

extern "C" pic_status pic_sort_keys_noalloc(const int32_t* keys, int64_t n, int32_t nbins, int32_t* offsets,
                                            int32_t* perm, void* cuda_stream) {
    using namespace pic;
    if (n < 0 || n >= (int64_t(1) << 31)) return na_fail(PIC_ERR_ARG, "n must be in [0, 2^31)");
    // an error left by the caller's earlier work stays where it is (not
    // cleared): the launches below could not be told apart from it
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess)
        return na_fail(PIC_ERR_CUDA, std::string("a CUDA error is pending from earlier work: ") +
                                         cudaGetErrorString(pending));
    if (nbins < 1 || nbins > kMaxBins)
        return na_fail(PIC_ERR_ARG, "nbins must be in [1, 4194304], the no-allocation scratch limit");
    if (!offsets || (n > 0 && (!keys || !perm))) return na_fail(PIC_ERR_ARG, "NULL array");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned char* base = nullptr;
    cudaError_t e = scratch_for_current_device(&base);
    if (e != cudaSuccess) return na_fail(PIC_ERR_CUDA, std::string("scratch address: ") + cudaGetErrorString(e));
    unsigned* err = reinterpret_cast<unsigned*>(base);
    unsigned long long* status = reinterpret_cast<unsigned long long*>(base + kErrBytes);
    int* count = reinterpret_cast<int*>(base + kErrBytes + kStatusPadded);
    const int nchunks = int((int64_t(nbins) + kScanChunk - 1) / kScanChunk);
    // the scratch keeps the previous call's contents: clear the error words,
    // the look-back words and ticket, and this call's counts
    e = cudaMemsetAsync(err, 0, kErrBytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, (size_t(nchunks) + 1) * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, size_t(nbins) * sizeof(int), s);
    if (e != cudaSuccess) return na_fail(PIC_ERR_CUDA, std::string("scratch clear: ") + cudaGetErrorString(e));
    if (n > 0) {
        const unsigned nb = unsigned((n + kBlockNA - 1) / kBlockNA);
        k_hist<<<nb, kBlockNA, 0, s>>>(keys, n, count, nbins, err);
    }
    k_scan<<<unsigned(nchunks), kBlockNA, 0, s>>>(count, offsets, nbins, status, nchunks, err);
    if (n > 0) {
        const unsigned nb = unsigned((n + kBlockNA - 1) / kBlockNA);
        k_perm_scatter<<<nb, kBlockNA, 0, s>>>(keys, n, offsets, count, nbins, perm);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(PIC_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    unsigned h = 0;
    e = cudaMemcpyAsync(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return na_fail(PIC_ERR_CUDA, std::string("sort: ") + cudaGetErrorString(e));
    if (h & ERRBIT_TIMEOUT) return na_fail(PIC_ERR_TIMEOUT, "a bounded device-side wait ran out");
    if (h & ERRBIT_RANGE) return na_fail(PIC_ERR_ARG, "a key is outside [0, nbins)");
    return PIC_OK;
}
