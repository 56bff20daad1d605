// Layout utilities of the backward pass: transposes that also select the kept
// sketch blocks and convert between FP32 and BF16.  They move data only.
#include "common.cuh"

namespace osk {

namespace {

template <typename T>
__device__ __forceinline__ float to_f(T x);
template <>
__device__ __forceinline__ float to_f<float>(float x) { return x; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <typename T>
__device__ __forceinline__ T from_f(float x);
template <>
__device__ __forceinline__ float from_f<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

// Y[c', r] = X[r, col(c')] with col(c') = kept[c' / b] * b + c' mod b (all columns
// when the block list is empty); 64 x 64 tiles through shared memory.
template <typename TI, typename TO>
__global__ void __launch_bounds__(256) select_transpose_kernel(const TI *__restrict__ X, int64_t ldx, int64_t rows,
                                                               int64_t ocols, int32_t b, BlockList kept,
                                                               TO *__restrict__ Y, int64_t ldy) {
    __shared__ float tile[64][65];
    const int64_t r0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    for (int k = ty; k < 64; k += 4) {
        const int64_t r = r0 + k, c = c0 + tx;
        if (r < rows && c < ocols) {
            const int64_t col = kept.count ? (int64_t)kept.idx[c / b] * b + (c % b) : c;
            tile[k][tx] = to_f(X[r * ldx + col]);
        }
    }
    __syncthreads();
    for (int k = ty; k < 64; k += 4) {
        const int64_t c = c0 + k, r = r0 + tx;
        if (r < rows && c < ocols) Y[c * ldy + r] = from_f<TO>(tile[tx][k]);
    }
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(256) cast_kernel(const TI *__restrict__ X, int64_t ldx, int64_t rows, int64_t cols,
                                                   TO *__restrict__ Y, int64_t ldy) {
    const int64_t total = rows * cols;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / cols, c = t - r * cols;
        Y[r * ldy + c] = from_f<TO>(to_f(X[r * ldx + c]));
    }
}

template <typename TI, typename TO>
os_status launch_st(const void *X, int64_t ldx, int64_t rows, int64_t ocols, int32_t b, const BlockList &kept,
                    void *Y, int64_t ldy, cudaStream_t st) {
    dim3 grid((unsigned)((ocols + 63) / 64), (unsigned)((rows + 63) / 64));
    if (grid.y > 65535u) return OS_ERR_UNSUPPORTED;
    select_transpose_kernel<TI, TO><<<grid, 256, 0, st>>>((const TI *)X, ldx, rows, ocols, b, kept, (TO *)Y, ldy);
    return check_launch();
}

template <typename TI, typename TO>
os_status launch_cast(const void *X, int64_t ldx, int64_t rows, int64_t cols, void *Y, int64_t ldy, cudaStream_t st) {
    const int64_t total = rows * cols;
    const int64_t blocks = (total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32;
    cast_kernel<TI, TO><<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, st>>>((const TI *)X, ldx, rows, cols, (TO *)Y,
                                                                            ldy);
    return check_launch();
}

bool float_type(os_dtype t) { return t == OS_F32 || t == OS_BF16; }

}  // namespace

}  // namespace osk

using namespace osk;

extern "C" os_status oversketch_select_transpose(const void *X, os_dtype x_t, int64_t rows, int64_t cols, int64_t ldx,
                                                 uint64_t block_mask, int32_t b, void *Y, os_dtype y_t, int64_t ldy,
                                                 void *stream) {
    if (rows < 0 || cols < 0 || ldx < cols) return OS_ERR_INVALID_ARG;
    if (!float_type(x_t) || !float_type(y_t)) return OS_ERR_DTYPE;
    BlockList kept;
    kept.count = 0;
    for (int t = 0; t < 64; ++t) kept.idx[t] = 0;
    int64_t ocols = cols;
    if (block_mask) {
        if (b < 1 || cols % b != 0) return OS_ERR_INVALID_ARG;
        const int P = (int)(cols / b);
        if (P > 64) return OS_ERR_UNSUPPORTED;
        OSK_TRY(check_mask(block_mask, P));
        kept = mask_to_list(block_mask, P);
        ocols = (int64_t)kept.count * b;
    }
    if (ldy < rows) return OS_ERR_INVALID_ARG;
    if (rows == 0 || ocols == 0) return OS_OK;   // an empty Y
    if (!X || !Y) return OS_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    if (x_t == OS_F32 && y_t == OS_F32) return launch_st<float, float>(X, ldx, rows, ocols, b, kept, Y, ldy, st);
    if (x_t == OS_F32 && y_t == OS_BF16) return launch_st<float, __nv_bfloat16>(X, ldx, rows, ocols, b, kept, Y, ldy, st);
    if (x_t == OS_BF16 && y_t == OS_F32) return launch_st<__nv_bfloat16, float>(X, ldx, rows, ocols, b, kept, Y, ldy, st);
    return launch_st<__nv_bfloat16, __nv_bfloat16>(X, ldx, rows, ocols, b, kept, Y, ldy, st);
}

extern "C" os_status oversketch_cast(const void *X, os_dtype x_t, int64_t rows, int64_t cols, int64_t ldx, void *Y,
                                     os_dtype y_t, int64_t ldy, void *stream) {
    if (rows < 0 || cols < 0 || ldx < cols || ldy < cols) return OS_ERR_INVALID_ARG;
    if (!float_type(x_t) || !float_type(y_t)) return OS_ERR_DTYPE;
    if (rows == 0 || cols == 0) return OS_OK;   // an empty Y
    if (!X || !Y) return OS_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    if (x_t == OS_F32 && y_t == OS_F32) return launch_cast<float, float>(X, ldx, rows, cols, Y, ldy, st);
    if (x_t == OS_F32 && y_t == OS_BF16) return launch_cast<float, __nv_bfloat16>(X, ldx, rows, cols, Y, ldy, st);
    if (x_t == OS_BF16 && y_t == OS_F32) return launch_cast<__nv_bfloat16, float>(X, ldx, rows, cols, Y, ldy, st);
    return launch_cast<__nv_bfloat16, __nv_bfloat16>(X, ldx, rows, cols, Y, ldy, st);
}
