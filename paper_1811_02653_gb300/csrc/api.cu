// C ABI glue: status strings, mask handling, the masked-GEMM dispatcher, the
// whole-product entry point and the FP64 error reductions.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace osk {

// implemented in sketch.cu / sketch_sparse.cu / gemm_simt.cu / gemm_tc.cu
size_t sketch_workspace_bytes(const Plan *p, int64_t F, os_dtype in_t);
size_t fp8_staging_bytes(const Plan *p, int64_t F);
os_status sketch_left_impl(const Plan *p, const void *A, os_dtype a_t, int64_t m, int64_t lda,
                           void *At, os_dtype out_t, int64_t ldat, float *scales,
                           const float *col_scale, uint64_t block_mask, void *ws, size_t ws_bytes,
                           cudaStream_t st, const uint64_t *dmask = nullptr);
os_status sketch_right_impl(const Plan *p, const void *B, os_dtype b_t, int64_t l, int64_t ldb,
                            void *BtT, os_dtype out_t, int64_t ldbt, float *scales, uint64_t block_mask,
                            void *ws, size_t ws_bytes, cudaStream_t st, const float *row_scale = nullptr,
                            const uint64_t *dmask = nullptr);
bool sketch_left_sparse_fits(const Plan *p, uint64_t block_mask);
os_status sketch_left_sparse_impl(const Plan *p, const void *A, os_dtype a_t, int64_t m, int64_t lda, void *At,
                                  os_dtype out_t, int64_t ldat, float *scales, const float *col_scale,
                                  uint64_t block_mask, cudaStream_t st);
os_status gemm_masked_f32(const Plan *p, const float *At, int64_t ldat, const float *BtT,
                          int64_t ldbt, int64_t m, int64_t l, uint64_t mask, float alpha, float beta,
                          float *C, int64_t ldc, cudaStream_t st);
os_status gemm_bf16_mn(const void *A, int64_t lda, bool a_mn, const void *B, int64_t ldb, bool b_mn, int64_t m,
                       int64_t l, int64_t K, float alpha, float *C, int64_t ldc, int32_t mn_b, int32_t remap,
                       uint64_t mask, int32_t P, cudaStream_t st);
os_status gemm_masked_tc(const Plan *p, const void *At, int64_t ldat, const float *a_scales,
                         const void *BtT, int64_t ldbt, const float *b_scales, os_dtype dt, int64_t m,
                         int64_t l, uint64_t mask, float alpha, float beta, float *C, int64_t ldc,
                         cudaStream_t st);

namespace {
thread_local char g_last_cuda_error[256] = "no error";
}

os_status set_cuda_error(cudaError_t err) {
    std::snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s", cudaGetErrorName(err),
                  cudaGetErrorString(err));
    return OS_ERR_CUDA;
}

os_status check_launch() {
    const cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? OS_OK : set_cuda_error(err);
}

os_status check_mask(uint64_t mask, int P) {
    if (mask == 0) return OS_ERR_MASK;
    if (P < 64 && (mask >> P) != 0) return OS_ERR_MASK;
    return OS_OK;
}

BlockList mask_to_list(uint64_t mask, int P) {
    BlockList L;
    L.count = 0;
    for (int j = 0; j < P && j < 64; ++j)
        if ((mask >> j) & 1ull) L.idx[L.count++] = j;
    for (int t = L.count; t < 64; ++t) L.idx[t] = 0;
    return L;
}

namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct MatmulLayout {
    int64_t z, ldat, ldbt, nsl;
    size_t at_bytes, bt_bytes, as_bytes, bs_bytes, left_ws;
};

// dtype of the sketched operands for a GEMM dtype: FP32 products run on the
// tensor cores as 3xTF32 (operands split into hi/lo planes by the sketch) when
// the block width fits the 32-element K tile, else on the FFMA kernel.
os_dtype sketch_dtype(const Plan *p, os_dtype g) {
    return (g == OS_F32 && p->b % 32 == 0) ? OS_TF32X2 : g;
}

MatmulLayout layout(const Plan *p, int64_t m, int64_t l, os_dtype a_t, os_dtype b_t, const os_opts *o) {
    MatmulLayout L;
    const os_dtype g = sketch_dtype(p, o ? o->gemm_dtype : OS_F32);
    const size_t es = dtype_size(g);
    const size_t planes = g == OS_TF32X2 ? 2 : 1;
    L.z = (int64_t)p->P * p->b;
    const int64_t align_el = 16 / (int64_t)es;
    L.ldat = (L.z + align_el - 1) / align_el * align_el;
    L.ldbt = L.ldat;
    L.nsl = (L.z + 127) / 128;
    L.at_bytes = align256((size_t)m * L.ldat * es * planes);
    const bool sym = o && o->symmetric;
    L.bt_bytes = sym ? 0 : align256((size_t)l * L.ldbt * es * planes);
    L.as_bytes = g == OS_FP8E4M3 ? align256((size_t)fp8_scale_ld(m) * L.nsl * 4) : 0;
    L.bs_bytes = (g == OS_FP8E4M3 && !sym) ? align256((size_t)fp8_scale_ld(l) * L.nsl * 4) : 0;
    // the packed-strip buffer is reused by the left and then the right sketch; FP8
    // sketches stage their FP32 sums after it and quantise them in a second pass
    size_t wl = sketch_workspace_bytes(p, m, a_t);
    size_t wr = sym ? 0 : sketch_workspace_bytes(p, l, b_t);
    if (g == OS_FP8E4M3) {
        wl = align256(wl) + fp8_staging_bytes(p, m);
        if (!sym) wr = align256(wr) + fp8_staging_bytes(p, l);
    }
    L.left_ws = align256(wl > wr ? wl : wr);
    return L;
}

// Deterministic FP64 partial sums: fixed grid, fixed per-thread order, fixed tree.
constexpr int kFrobBlocks = 512;

__global__ void __launch_bounds__(256) frob_partial_kernel(const float *__restrict__ X, int64_t ldx,
                                                           const float *__restrict__ Y, int64_t ldy,
                                                           int64_t rows, int64_t cols,
                                                           double *__restrict__ part) {
    __shared__ double red[3][256];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    const int64_t total = rows * cols;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / cols, c = t - r * cols;
        const double x = X[r * ldx + c];
        if (Y) {
            const double y = Y[r * ldy + c];
            s0 += (x - y) * (x - y);
            s1 += y * y;
            s2 += x * y;
        } else {
            s0 += x * x;
        }
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    red[2][threadIdx.x] = s2;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 3) part[blockIdx.x * 3 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void frob_final_kernel(const double *__restrict__ part, int nblocks, double *__restrict__ out) {
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int bidx = 0; bidx < nblocks; ++bidx) s += part[bidx * 3 + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

}  // namespace

}  // namespace osk

using namespace osk;

extern "C" const char *oversketch_status_string(os_status s) {
    switch (s) {
        case OS_OK: return "OS_OK";
        case OS_ERR_INVALID_ARG: return "OS_ERR_INVALID_ARG";
        case OS_ERR_MASK: return "OS_ERR_MASK";
        case OS_ERR_DTYPE: return "OS_ERR_DTYPE";
        case OS_ERR_OOM: return "OS_ERR_OOM";
        case OS_ERR_CUDA: return "OS_ERR_CUDA";
        case OS_ERR_TIMEOUT: return "OS_ERR_TIMEOUT";
        case OS_ERR_UNSUPPORTED: return "OS_ERR_UNSUPPORTED";
        case OS_ERR_WORKSPACE: return "OS_ERR_WORKSPACE";
    }
    return "OS_ERR_UNKNOWN";
}

extern "C" const char *oversketch_last_cuda_error(void) { return g_last_cuda_error; }

extern "C" os_status oversketch_gemm_masked(oversketch_plan_t plan, const void *At, int64_t ldat,
                                            const float *a_scales, const void *BtT, int64_t ldbt,
                                            const float *b_scales, os_dtype dt, int64_t m, int64_t l,
                                            uint64_t mask, float alpha, float beta, float *C,
                                            int64_t ldc, void *stream) {
    OSK_NVTX("gemm_masked");
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p || m < 0 || l < 0 || ldc < l) return OS_ERR_INVALID_ARG;
    OSK_TRY(check_mask(mask, p->P));
    if (m == 0 || l == 0) return OS_OK;   // an empty C: nothing to read or write
    if (!At || !BtT || !C) return OS_ERR_INVALID_ARG;
    const int64_t z = (int64_t)p->P * p->b;
    if (ldat < z || ldbt < z) return OS_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    // the 1/k of (*) (Eq. 3's 1/sqrt(N) on both sides, k = N under Alg. 3's rule)
    const float scale = alpha / (float)__builtin_popcountll(mask);
    switch (dt) {
        case OS_F32:
            return gemm_masked_f32(p, (const float *)At, ldat, (const float *)BtT, ldbt, m, l, mask,
                                   scale, beta, C, ldc, st);
        case OS_BF16:
        case OS_FP8E4M3:
        case OS_TF32X2:
            return gemm_masked_tc(p, At, ldat, a_scales, BtT, ldbt, b_scales, dt, m, l, mask, scale,
                                  beta, C, ldc, st);
    }
    return OS_ERR_DTYPE;
}

extern "C" os_status oversketch_workspace_size(oversketch_plan_t plan, int64_t m, int64_t l,
                                               os_dtype a_t, os_dtype b_t, const os_opts *opts,
                                               size_t *bytes) {
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p || !bytes || m < 0 || l < 0) return OS_ERR_INVALID_ARG;
    const MatmulLayout L = layout(p, m, l, a_t, b_t, opts);
    *bytes = L.at_bytes + L.bt_bytes + L.as_bytes + L.bs_bytes + L.left_ws + 256;
    return OS_OK;
}

extern "C" os_status oversketch_matmul(oversketch_plan_t plan, const void *A, os_dtype a_t,
                                       int64_t lda, const void *B, os_dtype b_t, int64_t ldb,
                                       float *C, int64_t ldc, int64_t m, int64_t n, int64_t l,
                                       uint64_t mask, const os_opts *opts, void *workspace,
                                       size_t ws_bytes, void *stream) {
    OSK_NVTX("matmul");
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p) return OS_ERR_INVALID_ARG;
    const bool sym = opts && opts->symmetric;
    if (sym) l = m;
    if (n != p->n || m < 0 || l < 0 || ldc < l) return OS_ERR_INVALID_ARG;
    OSK_TRY(check_mask(mask, p->P));
    const os_dtype g0 = opts ? opts->gemm_dtype : OS_F32;
    if (g0 != OS_F32 && g0 != OS_BF16 && g0 != OS_FP8E4M3 && g0 != OS_TF32X2) return OS_ERR_DTYPE;
    if (m == 0 || l == 0) return OS_OK;   // an empty C: nothing to read or write
    if (!A || !C || (!sym && !B)) return OS_ERR_INVALID_ARG;
    const os_dtype g = sketch_dtype(p, g0);
    const MatmulLayout L = layout(p, m, l, a_t, b_t, opts);
    const size_t need = L.at_bytes + L.bt_bytes + L.as_bytes + L.bs_bytes + L.left_ws + 256;
    if (!workspace || ws_bytes < need) return OS_ERR_WORKSPACE;
    cudaStream_t st = as_stream(stream);
    char *base = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(workspace) + 255) & ~uintptr_t(255));
    void *At = base;
    void *BtT = sym ? At : base + L.at_bytes;
    float *as = g == OS_FP8E4M3 ? reinterpret_cast<float *>(base + L.at_bytes + L.bt_bytes) : nullptr;
    float *bs = g == OS_FP8E4M3 ? (sym ? as : reinterpret_cast<float *>(base + L.at_bytes + L.bt_bytes + L.as_bytes))
                                : nullptr;
    void *lws = base + L.at_bytes + L.bt_bytes + L.as_bytes + L.bs_bytes;
    const float *cs = opts ? opts->col_scale : nullptr;
    // Only the kept blocks are sketched: the dropped blocks' columns of A~ and
    // B~ would never be read by the masked GEMM.
    if (opts && (opts->flags & OS_OPT_SPARSE_A) && sketch_left_sparse_fits(p, mask))
        OSK_TRY(sketch_left_sparse_impl(p, A, a_t, m, lda, At, g, L.ldat, as, cs, mask, st));
    else
        OSK_TRY(sketch_left_impl(p, A, a_t, m, lda, At, g, L.ldat, as, cs, mask, lws, L.left_ws, st));
    if (!sym) OSK_TRY(sketch_right_impl(p, B, b_t, l, ldb, BtT, g, L.ldbt, bs, mask, lws, L.left_ws, st));
    return oversketch_gemm_masked(plan, At, L.ldat, as, BtT, L.ldbt, bs, g, m, l, mask, 1.0f, 0.0f, C, ldc,
                                  stream);
}

extern "C" os_status oversketch_frob(const float *X, int64_t ldx, const float *Y, int64_t ldy,
                                     int64_t rows, int64_t cols, double *out, void *workspace,
                                     size_t ws_bytes, void *stream) {
    if (!X || !out || rows < 0 || cols < 0 || ldx < cols || (Y && ldy < cols))
        return OS_ERR_INVALID_ARG;
    if (!workspace || ws_bytes < sizeof(double) * 3 * kFrobBlocks) return OS_ERR_WORKSPACE;
    cudaStream_t st = as_stream(stream);
    double *part = reinterpret_cast<double *>(workspace);
    frob_partial_kernel<<<kFrobBlocks, 256, 0, st>>>(X, ldx, Y, ldy, rows, cols, part);
    OSK_TRY(check_launch());
    frob_final_kernel<<<1, 32, 0, st>>>(part, kFrobBlocks, out);
    return check_launch();
}

// ---------------------------------------------------------------------------
// The whole product from and to HOST memory, with the transfers overlapped.
//
// Order on two streams (the caller's compute stream and an internal copy stream
// of the device, ordered after the caller's earlier work):
//   copy:    B (whole) | A chunk 0 | A chunk 1 | ...            | C panel 0 | C panel 1 ...
//   compute:           | right sketch | left sketch chunk 0 | ... | GEMM panel 0 | panel 1 ...
// The right sketch of B runs while A streams in; each chunk of A rows (a
// multiple of 128 rows) is sketched as soon as it lands; the masked GEMM runs
// in row panels and every panel of C goes back while the next one is computed.
// The device copies use 16-byte aligned row pitches, so the right sketch always
// gathers B in place.  FP8 and FP32 products (whose sketches carry scale rows or
// TF32 planes sized by the full row count) sketch A in one piece.
namespace osk {
namespace {

struct HostPlan {
    int64_t lda_d, ldb_d, ldc_d;     // device row pitches (elements)
    size_t a_bytes, b_bytes, c_bytes, mm_bytes;
    int64_t a_rows, c_rows;           // rows per A chunk / per C panel
};

int64_t round_up(int64_t x, int64_t q) { return (x + q - 1) / q * q; }

HostPlan host_plan(const Plan *p, int64_t m, int64_t l, os_dtype a_t, os_dtype b_t, const os_opts *o) {
    HostPlan h;
    const bool sym = o && o->symmetric;
    const size_t ea = dtype_size(a_t), eb = dtype_size(b_t);
    h.lda_d = round_up(p->n, (int64_t)(16 / ea));
    // FP32 B keeps the pitch of a contiguous device tensor (l), so its right sketch
    // takes the same in-place path as the device entry point on that tensor
    h.ldb_d = b_t == OS_F32 ? l : round_up(l, (int64_t)(16 / eb));
    h.ldc_d = round_up(l, 4);
    h.a_bytes = align256((size_t)m * h.lda_d * ea);
    h.b_bytes = sym ? 0 : align256((size_t)p->n * h.ldb_d * eb);
    h.c_bytes = align256((size_t)m * h.ldc_d * 4);
    const os_dtype g = sketch_dtype(p, o ? o->gemm_dtype : OS_F32);
    const bool chunked = g == OS_BF16;
    h.a_rows = chunked ? (m + 7) / 8 : m;
    h.a_rows = round_up(h.a_rows < 1 ? 1 : h.a_rows, 128);
    h.c_rows = chunked ? round_up((m + 3) / 4, 128) : m;
    if (h.c_rows < 1) h.c_rows = 1;
    // oversketch_matmul's sketched operands, with the packing buffer sized for one
    // A chunk and for the right sketch's ragged remainder (B is gathered in place)
    const MatmulLayout L = layout(p, m, l, a_t, b_t, o);
    const size_t wl = sketch_workspace_bytes(p, h.a_rows < m ? h.a_rows : m, a_t);
    const size_t wr = sym ? 0 : sketch_workspace_bytes(p, b_t == OS_F32 ? 128 : l, b_t);
    h.mm_bytes = L.at_bytes + L.bt_bytes + L.as_bytes + L.bs_bytes + align256(wl > wr ? wl : wr) + 256;
    return h;
}

// 2-D copy that degenerates to one contiguous copy when the rows are packed.
cudaError_t copy2d(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width, size_t height,
                   cudaMemcpyKind kind, cudaStream_t st) {
    if (dpitch == width && spitch == width) return cudaMemcpyAsync(dst, src, width * height, kind, st);
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, height, kind, st);
}

cudaStream_t copy_stream(int dev) {
    static cudaStream_t streams[64] = {nullptr};
    if (dev < 0 || dev >= 64) return nullptr;
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        streams[dev] = nullptr;
    }
    return streams[dev];
}

}  // namespace
}  // namespace osk

extern "C" os_status oversketch_matmul_host_workspace_size(oversketch_plan_t plan, int64_t m, int64_t l,
                                                           os_dtype a_t, os_dtype b_t, const os_opts *opts,
                                                           size_t *bytes) {
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p || !bytes || m < 0 || l < 0) return OS_ERR_INVALID_ARG;
    if ((a_t != OS_F32 && a_t != OS_BF16) || (b_t != OS_F32 && b_t != OS_BF16)) return OS_ERR_DTYPE;
    if (opts && opts->symmetric) l = m;
    const HostPlan h = host_plan(p, m, l, a_t, b_t, opts);
    *bytes = h.a_bytes + h.b_bytes + h.c_bytes + h.mm_bytes + 256;
    return OS_OK;
}

extern "C" os_status oversketch_matmul_host(oversketch_plan_t plan, const void *A, os_dtype a_t, int64_t lda,
                                            const void *B, os_dtype b_t, int64_t ldb, float *C, int64_t ldc,
                                            int64_t m, int64_t n, int64_t l, uint64_t mask, const os_opts *opts,
                                            void *workspace, size_t ws_bytes, void *stream) {
    OSK_NVTX("matmul_host");
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p) return OS_ERR_INVALID_ARG;
    const bool sym = opts && opts->symmetric;
    if (sym) l = m;
    if (n != p->n || m < 0 || l < 0 || lda < n || ldc < l || (!sym && ldb < l)) return OS_ERR_INVALID_ARG;
    if ((a_t != OS_F32 && a_t != OS_BF16) || (!sym && b_t != OS_F32 && b_t != OS_BF16)) return OS_ERR_DTYPE;
    if (sym) b_t = a_t;
    OSK_TRY(check_mask(mask, p->P));
    const os_dtype g0 = opts ? opts->gemm_dtype : OS_F32;
    if (g0 != OS_F32 && g0 != OS_BF16 && g0 != OS_FP8E4M3) return OS_ERR_DTYPE;
    if (m == 0 || l == 0) return OS_OK;   // an empty C: nothing to copy or compute
    if (!A || !C || (!sym && !B)) return OS_ERR_INVALID_ARG;
    const os_dtype g = sketch_dtype(p, g0);
    const HostPlan h = host_plan(p, m, l, a_t, b_t, opts);
    if (!workspace || ws_bytes < h.a_bytes + h.b_bytes + h.c_bytes + h.mm_bytes + 256) return OS_ERR_WORKSPACE;
    int dev = 0;
    OSK_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != p->device) return OS_ERR_INVALID_ARG;
    cudaStream_t cs = as_stream(stream);
    cudaStream_t xs = copy_stream(dev);
    if (!xs) return OS_ERR_CUDA;
    const size_t ea = dtype_size(a_t), eb = dtype_size(b_t);
    char *base = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(workspace) + 255) & ~uintptr_t(255));
    char *Ad = base;
    char *Bd = base + h.a_bytes;
    float *Cd = reinterpret_cast<float *>(base + h.a_bytes + h.b_bytes);
    char *mm = base + h.a_bytes + h.b_bytes + h.c_bytes;
    const MatmulLayout L = layout(p, m, l, a_t, b_t, opts);
    void *At = mm;
    void *BtT = sym ? At : mm + L.at_bytes;
    float *as = g == OS_FP8E4M3 ? reinterpret_cast<float *>(mm + L.at_bytes + L.bt_bytes) : nullptr;
    float *bs = g == OS_FP8E4M3 ? (sym ? as : reinterpret_cast<float *>(mm + L.at_bytes + L.bt_bytes + L.as_bytes))
                                : nullptr;
    void *pack = mm + L.at_bytes + L.bt_bytes + L.as_bytes + L.bs_bytes;
    const size_t pack_bytes = h.mm_bytes - 256 - (L.at_bytes + L.bt_bytes + L.as_bytes + L.bs_bytes);
    const float *cs_scale = opts ? opts->col_scale : nullptr;
    const bool sparse = opts && (opts->flags & OS_OPT_SPARSE_A) && sketch_left_sparse_fits(p, mask);
    const int64_t nchunks = (m + h.a_rows - 1) / h.a_rows;
    const int64_t npanels = (m + h.c_rows - 1) / h.c_rows;

    std::vector<cudaEvent_t> ev;
    auto event = [&](cudaEvent_t *e) -> os_status {
        if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return set_cuda_error(cudaGetLastError());
        ev.push_back(*e);
        return OS_OK;
    };
    os_status st = OS_OK;
    do {
        // the copy stream starts after the caller's earlier work on `stream`
        cudaEvent_t e0;
        if ((st = event(&e0)) != OS_OK) break;
        if (cudaEventRecord(e0, cs) != cudaSuccess || cudaStreamWaitEvent(xs, e0, 0) != cudaSuccess) {
            st = set_cuda_error(cudaGetLastError());
            break;
        }
        // B, then the right sketch while A arrives
        if (!sym) {
            cudaEvent_t eb_done;
            if ((st = event(&eb_done)) != OS_OK) break;
            if (copy2d(Bd, h.ldb_d * eb, B, ldb * eb, l * eb, n, cudaMemcpyHostToDevice, xs) != cudaSuccess ||
                cudaEventRecord(eb_done, xs) != cudaSuccess || cudaStreamWaitEvent(cs, eb_done, 0) != cudaSuccess) {
                st = set_cuda_error(cudaGetLastError());
                break;
            }
            if ((st = sketch_right_impl(p, Bd, b_t, l, h.ldb_d, BtT, g, L.ldbt, bs, mask, pack, pack_bytes, cs)) != OS_OK)
                break;
        }
        // A in chunks of rows, each sketched as it lands
        for (int64_t c = 0; st == OS_OK && c < nchunks; ++c) {
            const int64_t r0 = c * h.a_rows, rows = (m - r0 < h.a_rows) ? m - r0 : h.a_rows;
            cudaEvent_t ea_done;
            if ((st = event(&ea_done)) != OS_OK) break;
            if (copy2d(Ad + (size_t)r0 * h.lda_d * ea, h.lda_d * ea, (const char *)A + (size_t)r0 * lda * ea, lda * ea,
                       n * ea, rows, cudaMemcpyHostToDevice, xs) != cudaSuccess ||
                cudaEventRecord(ea_done, xs) != cudaSuccess || cudaStreamWaitEvent(cs, ea_done, 0) != cudaSuccess) {
                st = set_cuda_error(cudaGetLastError());
                break;
            }
            void *at_c = (char *)At + (size_t)r0 * L.ldat * dtype_size(g);
            const void *a_c = Ad + (size_t)r0 * h.lda_d * ea;
            if (sparse)
                st = sketch_left_sparse_impl(p, a_c, a_t, rows, h.lda_d, at_c, g, L.ldat, as, cs_scale, mask, cs);
            else
                st = sketch_left_impl(p, a_c, a_t, rows, h.lda_d, at_c, g, L.ldat, as, cs_scale, mask, pack, pack_bytes,
                                      cs);
        }
        if (st != OS_OK) break;
        // the GEMM in row panels; each panel of C goes back while the next is computed
        for (int64_t q = 0; q < npanels; ++q) {
            const int64_t r0 = q * h.c_rows, rows = (m - r0 < h.c_rows) ? m - r0 : h.c_rows;
            const void *at_q = (const char *)At + (size_t)r0 * L.ldat * dtype_size(g);
            const float *as_q = as ? as + r0 : nullptr;   // slice-major scales: the panel's rows start at r0
            if ((st = oversketch_gemm_masked(plan, at_q, L.ldat, as_q, BtT, L.ldbt, bs, g, rows, l, mask, 1.0f,
                                             0.0f, Cd + r0 * h.ldc_d, h.ldc_d, cs)) != OS_OK)
                break;
            cudaEvent_t ec;
            if ((st = event(&ec)) != OS_OK) break;
            if (cudaEventRecord(ec, cs) != cudaSuccess || cudaStreamWaitEvent(xs, ec, 0) != cudaSuccess ||
                copy2d(C + r0 * ldc, ldc * 4, Cd + r0 * h.ldc_d, h.ldc_d * 4, l * 4, rows, cudaMemcpyDeviceToHost,
                       xs) != cudaSuccess) {
                st = set_cuda_error(cudaGetLastError());
                break;
            }
        }
        if (st != OS_OK) break;
        // the call is complete on `stream` once the last panel is in C
        cudaEvent_t e_end;
        if ((st = event(&e_end)) != OS_OK) break;
        if (cudaEventRecord(e_end, xs) != cudaSuccess || cudaStreamWaitEvent(cs, e_end, 0) != cudaSuccess)
            st = set_cuda_error(cudaGetLastError());
    } while (0);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);   // released once their work completes
    return st;
}

// ---------------------------------------------------------------------------
// Backward pass of (*) as a function of both operands (the adjoint of Eq. 3's
// linear map S restricted to the kept blocks):
//   dX = (1/k) (dC . B~_sel^T) . S_sel^T      dG = (1/k) S_sel . (A~_sel^T . dC)
// Each side is a BF16 tensor-core GEMM with FP32 accumulation (the 1/k applied in
// its epilogue) followed by an unsketch gather; the operand layouts the GEMMs need
// (dC in BF16, the kept blocks of B~^T and A~ transposed, dC^T) are written into
// the workspace first.
namespace osk {
namespace {

// Workspace of the backward pass: dC in BF16 (both products use it), then T (and
// the compacted kept blocks of B~, laid out K-major) for dX, then U (and A~'s kept
// blocks and dC^T, K-major) for dG.  With b a multiple of 128 and m, l multiples of
// 8 the tensor cores read B~^T, A~ and dC MN-major as they are stored (dC's rows
// padded to a multiple of 64), and the K-major copies are not made.
struct BackwardLayout {
    bool mn;                         // operands read MN-major (no transposed copies)
    int64_t kb, ld_l, ld_m, ld_kb;   // padded row pitches (elements) of the BF16 / FP32 buffers
    size_t dc16, bsel, t, asel, dct16, u;
};

BackwardLayout backward_layout(const Plan *p, int64_t m, int64_t l, uint64_t mask) {
    BackwardLayout L;
    L.mn = p->b % 128 == 0 && m % 8 == 0 && l % 8 == 0;
    L.kb = (int64_t)__builtin_popcountll(mask) * p->b;
    L.ld_l = L.mn ? (l + 63) / 64 * 64 : (l + 7) / 8 * 8;   // BF16 rows of l elements
    L.ld_m = (m + 7) / 8 * 8;      // BF16 rows of m elements
    L.ld_kb = (L.kb + 3) / 4 * 4;  // FP32 rows of k*b elements
    L.dc16 = align256((size_t)m * L.ld_l * 2);
    L.bsel = L.mn ? 0 : align256((size_t)L.kb * L.ld_l * 2);
    L.t = align256((size_t)m * L.ld_kb * 4);
    L.asel = L.mn ? 0 : align256((size_t)L.kb * L.ld_m * 2);
    L.dct16 = L.mn ? 0 : align256((size_t)l * L.ld_m * 2);
    L.u = align256((size_t)L.kb * ((l + 3) / 4 * 4) * 4);
    return L;
}

size_t backward_bytes(const BackwardLayout &L, bool need_dx, bool need_dg) {
    return L.dc16 + (need_dx ? L.bsel + L.t : 0) + (need_dg ? L.asel + L.dct16 + L.u : 0) + 256;
}

}  // namespace
}  // namespace osk

extern "C" os_status oversketch_matmul_backward_workspace_size(oversketch_plan_t plan, int64_t m, int64_t l,
                                                                uint64_t mask, int32_t need_dx, int32_t need_dg,
                                                                size_t *bytes) {
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p || !bytes || m < 0 || l < 0) return OS_ERR_INVALID_ARG;
    OSK_TRY(check_mask(mask, p->P));
    *bytes = backward_bytes(backward_layout(p, m, l, mask), need_dx != 0, need_dg != 0);
    return OS_OK;
}

extern "C" os_status oversketch_matmul_backward(oversketch_plan_t plan, const void *At, int64_t ldat,
                                                const void *BtT, int64_t ldbt, const float *dC, int64_t lddc,
                                                int64_t m, int64_t l, uint64_t mask, void *dX, os_dtype x_t,
                                                int64_t ldx, void *dG, os_dtype g_t, int64_t ldg, void *workspace,
                                                size_t ws_bytes, void *stream) {
    OSK_NVTX("matmul_backward");
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p || m < 0 || l < 0 || lddc < l) return OS_ERR_INVALID_ARG;
    OSK_TRY(check_mask(mask, p->P));
    const int64_t z = (int64_t)p->P * p->b;
    if ((dX && (x_t != OS_F32 && x_t != OS_BF16)) || (dG && (g_t != OS_F32 && g_t != OS_BF16))) return OS_ERR_DTYPE;
    if ((dX && (ldbt < z || ldx < p->n)) || (dG && (ldat < z || ldg < l))) return OS_ERR_INVALID_ARG;
    const bool need_dx = dX != nullptr && m > 0, need_dg = dG != nullptr && l > 0;
    if (!need_dx && !need_dg) return OS_OK;
    const BackwardLayout L = backward_layout(p, m, l, mask);
    if (!workspace || ws_bytes < backward_bytes(L, need_dx, need_dg)) return OS_ERR_WORKSPACE;
    if (!dC && m > 0 && l > 0) return OS_ERR_INVALID_ARG;
    const float inv_k = 1.0f / (float)__builtin_popcountll(mask);
    char *base = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(workspace) + 255) & ~uintptr_t(255));
    cudaStream_t st = as_stream(stream);
    void *dc16 = base;
    base += L.dc16;
    if (m > 0 && l > 0 && (need_dx || L.mn)) OSK_TRY(oversketch_cast(dC, OS_F32, m, l, lddc, dc16, OS_BF16, L.ld_l, stream));
    if (need_dx) {
        if (l > 0 && !BtT) return OS_ERR_INVALID_ARG;
        void *bsel = base;
        float *T = reinterpret_cast<float *>(base + L.bsel);
        base += L.bsel + L.t;
        if (l > 0 && L.mn) {
            // T = dC B~_sel^T: B~^T (l x z) read MN-major, kept blocks picked by column
            OSK_TRY(gemm_bf16_mn(dc16, L.ld_l, false, BtT, ldbt, true, m, L.kb, l, inv_k, T, L.ld_kb, p->b, 2, mask,
                                 p->P, st));
        } else if (l > 0) {
            OSK_TRY(oversketch_select_transpose(BtT, OS_BF16, l, z, ldbt, mask, p->b, bsel, OS_BF16, L.ld_l, stream));
            OSK_TRY(oversketch_gemm_bf16(dc16, L.ld_l, bsel, L.ld_l, m, L.kb, l, inv_k, 0.0f, T, L.ld_kb, stream));
        } else {
            OSK_CUDA_TRY(cudaMemsetAsync(T, 0, (size_t)m * L.ld_kb * 4, st));
        }
        OSK_TRY(oversketch_unsketch_cols(plan, T, m, L.ld_kb, mask, 1.0f, dX, x_t, ldx, stream));
    }
    if (need_dg) {
        if (m > 0 && !At) return OS_ERR_INVALID_ARG;
        void *asel = base;
        void *dct16 = base + L.asel;
        float *U = reinterpret_cast<float *>(base + L.asel + L.dct16);
        const int64_t ldu = (l + 3) / 4 * 4;
        if (m > 0 && L.mn) {
            // U = A~_sel^T dC: A~ (m x z, kept blocks picked by column) and dC read MN-major
            OSK_TRY(gemm_bf16_mn(At, ldat, true, dc16, L.ld_l, true, L.kb, l, m, inv_k, U, ldu, p->b, 1, mask, p->P,
                                 st));
        } else if (m > 0) {
            OSK_TRY(oversketch_select_transpose(At, OS_BF16, m, z, ldat, mask, p->b, asel, OS_BF16, L.ld_m, stream));
            OSK_TRY(oversketch_select_transpose(dC, OS_F32, m, l, lddc, 0, 0, dct16, OS_BF16, L.ld_m, stream));
            OSK_TRY(oversketch_gemm_bf16(asel, L.ld_m, dct16, L.ld_m, L.kb, l, m, inv_k, 0.0f, U, ldu, stream));
        } else {
            OSK_CUDA_TRY(cudaMemsetAsync(U, 0, (size_t)L.kb * ldu * 4, st));
        }
        OSK_TRY(oversketch_unsketch_rows(plan, U, l, ldu, mask, 1.0f, dG, g_t, ldg, stream));
    }
    return OS_OK;
}

// Sketch size for a target accuracy (Thm. 4.1): d = 2/(eps*theta) columns make
// (A S)(S^T B) (eps, theta)-accurate, i.e. ||AB - A S S^T B||_F^2 <= eps ||A||_F^2 ||B||_F^2
// with probability at least 1 - theta; with blocks of width b that is N = ceil(r d / b)
// blocks (r >= 1 multiplies the dimension as in the spectral-norm remark after the
// theorem), and e extra blocks absorb the stragglers: the smallest e with
// e >= p (N + e) for a straggler fraction p, so that dropping a fraction p of the
// N + e blocks still leaves N.  Host-only; no device is touched.
extern "C" os_status oversketch_sketch_size(double eps, double theta, int32_t b, double straggler_fraction,
                                            int32_t r, int32_t *N, int32_t *e) {
    if (!N || !e || !(eps > 0.0) || !(theta > 0.0) || theta >= 1.0 || b < 1 || r < 1) return OS_ERR_INVALID_ARG;
    if (!(straggler_fraction >= 0.0) || straggler_fraction >= 1.0) return OS_ERR_INVALID_ARG;
    const double d = 2.0 / (eps * theta);
    const double nb = std::ceil((double)r * d / (double)b - 1e-9);
    if (nb > 64.0) return OS_ERR_UNSUPPORTED;
    const int32_t n_blocks = nb < 1.0 ? 1 : (int32_t)nb;
    const double p = straggler_fraction;
    const double ex = std::ceil(p * (double)n_blocks / (1.0 - p) - 1e-9);
    const int32_t extra = ex < 0.0 ? 0 : (int32_t)ex;
    if (n_blocks + extra > 64) return OS_ERR_UNSUPPORTED;
    *N = n_blocks;
    *e = extra;
    return OS_OK;
}
