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
#include <cuda.h>

#include <mutex>

#include "common.cuh"

namespace osk {

os_status sketch_left_impl(const Plan *p, const void *A, os_dtype a_t, int64_t m, int64_t lda,
                           void *At, os_dtype out_t, int64_t ldat, float *scales,
                           const float *col_scale, uint64_t block_mask, void *ws, size_t ws_bytes,
                           cudaStream_t st, const uint64_t *dmask = nullptr);
size_t sketch_workspace_bytes(const Plan *p, int64_t F, os_dtype in_t);
os_status sketch_left_check(const Plan *p, const void *A, os_dtype a_t, int64_t m, int64_t lda, void *At,
                            os_dtype out_t, int64_t ldat, float *scales, uint64_t block_mask);

namespace {

// 32 MiB, held on every GPU that loads the library until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// Unique id of the current CUDA context (driver entry points fetched through the
// runtime, so the library does not link the driver); 0 when none is current or
// the driver lacks cuCtxGetId.
typedef CUresult (*PFN_ctxGetCurrent)(CUcontext *);
typedef CUresult (*PFN_ctxGetId)(CUcontext, unsigned long long *);

unsigned long long current_context_id() {
    static PFN_ctxGetCurrent get_current = nullptr;
    static PFN_ctxGetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_ctxGetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_ctxGetId>(f);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the scratch array in the current context.  In host code
// g_noalloc_scratch names a host-side stand-in, not device memory, so the
// address is looked up with the device current, once per context: a context
// created after cudaDeviceReset loads the module again, possibly elsewhere, and
// gets its own lookup.  Without a context id the address is looked up on every
// call.
os_status scratch_address(void **out) {
    int dev = 0;
    OSK_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return OS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_ptr[dev] || ctx == 0 || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        OSK_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_ptr[dev] = p;
        g_scratch_ctx[dev] = current_context_id();   // the lookup creates the context if needed
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
    // the same argument checks as oversketch_sketch_left, and nothing to do for an
    // empty output, before the scratch array is looked up
    OSK_TRY(sketch_left_check(p, A, a_t, m, lda, At, out_t, ldat, scales, block_mask));
    if (m == 0) return OS_OK;
    // the packed operand must fit the fixed scratch array
    if (sketch_workspace_bytes(p, m, a_t) > kNoAllocScratchBytes) return OS_ERR_WORKSPACE;
    void *ws = nullptr;
    OSK_TRY(scratch_address(&ws));
    return sketch_left_impl(p, A, a_t, m, lda, At, out_t, ldat, scales, col_scale, block_mask, ws,
                            kNoAllocScratchBytes, as_stream(stream));
}
