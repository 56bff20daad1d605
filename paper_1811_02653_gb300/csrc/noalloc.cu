// Left sketch for callers that cannot allocate device memory.
//
// oversketch_sketch_left needs a packing workspace that its caller allocates.
// Some callers cannot allocate at the point where they sketch: code that runs
// while a stream is being captured into a CUDA graph (cudaMalloc is not allowed
// there), code whose device memory is owned by another allocator or a fixed
// budget, and latency-critical loops that must not call cudaMalloc (it can
// synchronise the device).  This entry point takes its workspace from a
// fixed-size scratch array in device memory that exists for as long as the
// library is loaded, so a call allocates nothing.
#include <mutex>

#include "common.cuh"

namespace osk {

os_status sketch_left_impl(const Plan *p, const void *A, os_dtype a_t, int64_t m, int64_t lda,
                           void *At, os_dtype out_t, int64_t ldat, float *scales,
                           const float *col_scale, uint64_t block_mask, void *ws, size_t ws_bytes,
                           cudaStream_t st);
size_t sketch_workspace_bytes(const Plan *p, int64_t F, os_dtype in_t);

namespace {

// 32 MiB, held on every GPU that loads the library until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// g_noalloc_scratch names a host-side stand-in, not device memory, so the
// address is looked up once per device with that device current.
os_status scratch_address(void **out) {
    int dev = 0;
    OSK_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return OS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        OSK_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return OS_OK;
}

}  // namespace

}  // namespace osk

using namespace osk;

extern "C" os_status oversketch_sketch_left_noalloc(oversketch_plan_t plan, const void *A, os_dtype a_t,
                                                    int64_t m, int64_t lda, void *At, os_dtype out_t,
                                                    int64_t ldat, float *scales, const float *col_scale,
                                                    uint64_t block_mask, void *stream) {
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p || m < 0) return OS_ERR_INVALID_ARG;
    if (a_t != OS_F32 && a_t != OS_BF16) return OS_ERR_DTYPE;
    // the packed operand must fit the fixed scratch array
    if (sketch_workspace_bytes(p, m, a_t) > kNoAllocScratchBytes) return OS_ERR_WORKSPACE;
    void *ws = nullptr;
    OSK_TRY(scratch_address(&ws));
    return sketch_left_impl(p, A, a_t, m, lda, At, out_t, ldat, scales, col_scale, block_mask, ws,
                            kNoAllocScratchBytes, as_stream(stream));
}
