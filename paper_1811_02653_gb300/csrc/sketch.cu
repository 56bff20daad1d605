// Sketch kernels: A~ = A S and B~ = S^T B (Alg. 5, Alg. 4 step 3), plus the
// adjoint gathers used by the backward pass.
//
// One gather kernel serves both sides.  It reads a matrix X whose rows are
// indexed by the sketched dimension i (n rows) and whose "free" dimension f
// is contiguous in memory, and writes Y^T[f, q] for q = j*b + c:
//
//     Y^T[f, j*b + c] = sum_{i in bucket c of block j} sigma_j(i) * s_i * X[i, f]
//
// Right sketch: X = B (n x l), Y^T = B~^T (l x z).  Left sketch: X = A^T, staged
// by a tiled transpose into the workspace, Y^T = A~ (m x z).
//
// A CTA owns 128 consecutive sketched columns q (whole buckets) and a strip of
// 128 free indices.  Each warp walks the bucket-CSR of its buckets (indices
// ascending inside a bucket, the same order in every run: no atomics, bitwise
// reproducible) and gathers whole 128-wide row segments of X with 16-byte
// loads, accumulating in FP32.  The 128 x 128 tile is transposed through
// shared memory so that Y^T rows are written contiguously, and, for FP8, the
// per-(row, 128-q) power-of-two scale is taken over exactly that row of the
// tile.  CTAs of one strip are adjacent in launch order so the strip stays
// in L2 while all of its buckets are gathered.
#include <cstdint>
#include <cstdlib>
#include <type_traits>

#include "common.cuh"

namespace osk {

namespace {

constexpr int kTileQ = 128;
constexpr int kWarps = 8;
constexpr int kUnroll = 8;

// VW consecutive elements of the free dimension per lane (strip = 32*VW).
template <typename InT, int VW, bool kAligned>
struct Loader {
    __device__ __forceinline__ static void load(const InT *p, float (&v)[VW]) {
        if constexpr (kAligned && std::is_same<InT, float>::value && VW == 4) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
            v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        } else if constexpr (kAligned && std::is_same<InT, float>::value && VW == 2) {
            const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
            v[0] = t.x; v[1] = t.y;
        } else if constexpr (kAligned && std::is_same<InT, __nv_bfloat16>::value && VW == 4) {
            const uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
            const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
            const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
            v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
        } else if constexpr (kAligned && std::is_same<InT, __nv_bfloat16>::value && VW == 2) {
            const unsigned u = __ldg(reinterpret_cast<const unsigned *>(p));
            const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
            v[0] = a.x; v[1] = a.y;
        } else {
#pragma unroll
            for (int k = 0; k < VW; ++k) v[k] = to_f32(p[k]);
        }
    }
    __device__ __forceinline__ static float to_f32(float x) { return x; }
    __device__ __forceinline__ static float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }
    __device__ __forceinline__ static float load1(const InT *p) { return to_f32(p[0]); }
};

// Smallest e with amax <= 448 * 2^e (exact), clamped to the UE8M0 range.
__device__ __forceinline__ int fp8_scale_exponent(float amax) {
    if (!(amax > 0.f)) return 0;
    int E;
    const float m = frexpf(amax, &E);   // amax = m * 2^E, m in [0.5, 1)
    int e = (m <= 0.875f) ? E - 9 : E - 8;
    return e < -127 ? -127 : (e > 127 ? 127 : e);
}

// Lane layout: lane = slot * 8 + sub.  The 4 slots of a warp gather 4
// different members of the current bucket at once, each 8-lane group reading
// a 32-element row segment (128 B for FP32) of X; lane `sub` holds elements
// 4*sub .. 4*sub+3 of the strip.  Slot s accumulates members s, s+4, s+8, ...
// in ascending order and the four partial sums are combined as
// (p0 + p1) + (p2 + p3): a fixed order, so results are bitwise reproducible.
template <typename InT, typename OutT, bool kAligned>
__global__ void __launch_bounds__(kWarps * 32)
sketch_gather_kernel(const InT *__restrict__ X, int64_t ldx, int64_t F,
                     const uint32_t *__restrict__ perm, const uint32_t *__restrict__ offs,
                     int64_t n, int32_t b, int32_t z, const float *__restrict__ col_scale,
                     OutT *__restrict__ Yt, int64_t ldy, float *__restrict__ scales,
                     int64_t lds) {
    constexpr int TF = 32;               // free indices per CTA
    constexpr int PITCH = TF + 1;        // odd pitch: conflict-free column reads
    constexpr int UNR = 4;               // groups of 4 members in flight per lane
    __shared__ float tile[kTileQ * PITCH];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = lane >> 3, sub = lane & 7;
    const int q0 = blockIdx.x * kTileQ;
    const int64_t f0 = (int64_t)blockIdx.y * TF;
    const int64_t f = f0 + 4 * sub;
    const bool full = kAligned && (f + 3 < F);
    using L = Loader<InT, 4, true>;

    for (int t = 0; t < kTileQ / kWarps; ++t) {
        const int qq = warp * (kTileQ / kWarps) + t;
        const int q = q0 + qq;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        if (q < z) {
            const int j = q / b, c = q - j * b;
            const uint32_t *prow = perm + (int64_t)j * n;
            const uint32_t beg = __ldg(offs + (int64_t)j * (b + 1) + c);
            const uint32_t end = __ldg(offs + (int64_t)j * (b + 1) + c + 1);
            for (uint32_t base = beg; base < end; base += 32) {
                const int cnt = (int)min(32u, end - base);
                const uint32_t my = lane < cnt ? __ldg(prow + base + lane) : 0u;
                const float mysc = (col_scale && lane < cnt) ? __ldg(col_scale + (my & kIndexMask)) : 1.f;
                for (int u = 0; u < cnt; u += 4 * UNR) {
                    float v[UNR][4];
                    float sg[UNR];
#pragma unroll
                    for (int g = 0; g < UNR; ++g) {
                        const int src = u + 4 * g + slot;
                        const uint32_t ent = __shfl_sync(0xffffffffu, my, src & 31);
                        const float sc = __shfl_sync(0xffffffffu, mysc, src & 31);
                        const bool valid = src < cnt;
                        sg[g] = valid ? ((ent & kSignBit) ? -sc : sc) : 0.f;
                        const InT *ptr = X + (int64_t)(ent & kIndexMask) * ldx + f;
                        if (valid && full) {
                            L::load(ptr, v[g]);
                        } else {
#pragma unroll
                            for (int w = 0; w < 4; ++w)
                                v[g][w] = (valid && f + w < F) ? L::load1(ptr + w) : 0.f;
                        }
                    }
#pragma unroll
                    for (int g = 0; g < UNR; ++g)
#pragma unroll
                        for (int w = 0; w < 4; ++w) acc[w] = fmaf(sg[g], v[g][w], acc[w]);
                }
            }
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            acc[w] += __shfl_xor_sync(0xffffffffu, acc[w], 8);
            acc[w] += __shfl_xor_sync(0xffffffffu, acc[w], 16);
        }
        if (slot == 0) {
#pragma unroll
            for (int w = 0; w < 4; ++w) tile[qq * PITCH + 4 * sub + w] = acc[w];
        }
    }
    __syncthreads();

    // Transposed write-out: warp w writes rows f0 + 4w .. 4w+3 of Y^T.
    for (int t = 0; t < TF / kWarps; ++t) {
        const int ff = warp * (TF / kWarps) + t;
        const int64_t frow = f0 + ff;
        if (frow >= F) break;
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = tile[(lane + 32 * k) * PITCH + ff];
        OutT *dst = Yt + frow * ldy + q0;
        if constexpr (sizeof(OutT) == 1) {
            float amax = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (q0 + lane + 32 * k < z) amax = fmaxf(amax, fabsf(v[k]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
            const int e = fp8_scale_exponent(amax);
            const float inv = ldexpf(1.f, -e);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int q = q0 + lane + 32 * k;
                if (q < z) {
                    __nv_fp8_e4m3 r(v[k] * inv);   // RNE, saturating to +-448
                    dst[lane + 32 * k] = r;
                }
            }
            if (lane == 0) scales[frow * lds + q0 / kTileQ] = ldexpf(1.f, e);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int q = q0 + lane + 32 * k;
                if (q < z) {
                    if constexpr (sizeof(OutT) == 4)
                        dst[lane + 32 * k] = v[k];
                    else
                        dst[lane + 32 * k] = __float2bfloat16_rn(v[k]);
                }
            }
        }
    }
}

// Tiled transpose: Xt[c, r] = X[r, c] (X rows x cols, ld ldx; Xt ld ldt).
template <typename T>
__global__ void __launch_bounds__(256) transpose_kernel(const T *__restrict__ X, int64_t ldx,
                                                        int64_t rows, int64_t cols,
                                                        T *__restrict__ Xt, int64_t ldt) {
    __shared__ T tile[64][65];
    const int64_t r0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;   // 64 x 4
    for (int k = ty; k < 64; k += 4) {
        const int64_t r = r0 + k, c = c0 + tx;
        if (r < rows && c < cols) tile[k][tx] = X[r * ldx + c];
    }
    __syncthreads();
    for (int k = ty; k < 64; k += 4) {
        const int64_t c = c0 + k, r = r0 + tx;
        if (r < rows && c < cols) Xt[c * ldt + r] = tile[tx][k];
    }
}

// dX[r, i] = scale * sum_{j kept} sigma_j(i) T[r, j*b + h_j(i)]
template <typename OutT>
__global__ void __launch_bounds__(256) unsketch_cols_kernel(
    const float *__restrict__ T, int64_t m, int64_t ldt, const uint32_t *__restrict__ hs, int64_t n,
    int32_t b, BlockList kept, float scale, OutT *__restrict__ dX, int64_t ldx) {
    const int64_t r = blockIdx.y;
    const float *trow = T + r * ldt;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int t = 0; t < kept.count; ++t) {
            const int j = kept.idx[t];
            const uint32_t v = __ldg(hs + (int64_t)j * n + i);
            const float x = __ldg(trow + (int64_t)j * b + (v & kIndexMask));
            acc += (v & kSignBit) ? -x : x;
        }
        acc *= scale;
        if constexpr (sizeof(OutT) == 4)
            dX[r * ldx + i] = acc;
        else
            dX[r * ldx + i] = __float2bfloat16_rn(acc);
    }
}

// dG[i, c] = scale * sum_{j kept} sigma_j(i) U[j*b + h_j(i), c]; one warp per
// row i, whole-row gathers of U.
template <typename OutT>
__global__ void __launch_bounds__(256) unsketch_rows_kernel(
    const float *__restrict__ U, int64_t l, int64_t ldu, const uint32_t *__restrict__ hs, int64_t n,
    int32_t b, BlockList kept, float scale, OutT *__restrict__ dG, int64_t ldg) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + warp;
    if (i >= n) return;
    const int64_t c0 = (int64_t)blockIdx.y * 1024;
    int64_t rows[64];
    float sg[64];
    for (int t = 0; t < kept.count; ++t) {
        const int j = kept.idx[t];
        const uint32_t v = __ldg(hs + (int64_t)j * n + i);
        rows[t] = (int64_t)j * b + (v & kIndexMask);
        sg[t] = (v & kSignBit) ? -scale : scale;
    }
    for (int64_t c = c0 + lane; c < min(l, c0 + 1024); c += 32) {
        float acc = 0.f;
        for (int t = 0; t < kept.count; ++t) acc = fmaf(sg[t], __ldg(U + rows[t] * ldu + c), acc);
        if constexpr (sizeof(OutT) == 4)
            dG[i * ldg + c] = acc;
        else
            dG[i * ldg + c] = __float2bfloat16_rn(acc);
    }
}

template <typename InT, typename OutT, bool kAligned>
os_status launch_gather_t(const Plan *p, const InT *X, int64_t ldx, int64_t F, const float *col_scale,
                          void *Yt, int64_t ldy, float *scales, cudaStream_t st) {
    const int z = p->P * p->b;
    dim3 grid((unsigned)((z + kTileQ - 1) / kTileQ), (unsigned)((F + 31) / 32));
    if (grid.y > 65535u) return OS_ERR_UNSUPPORTED;
    sketch_gather_kernel<InT, OutT, kAligned><<<grid, kWarps * 32, 0, st>>>(
        X, ldx, F, p->perm, p->offs, p->n, p->b, z, col_scale, (OutT *)Yt, ldy, scales, z / kTileQ);
    return check_launch();
}

template <typename InT, typename OutT>
os_status launch_gather_o(const Plan *p, const InT *X, int64_t ldx, int64_t F, const float *col_scale,
                          void *Yt, int64_t ldy, float *scales, cudaStream_t st) {
    const bool aligned = aligned16(X) && (ldx * (int64_t)sizeof(InT)) % 16 == 0;
    if (!aligned) return launch_gather_t<InT, OutT, false>(p, X, ldx, F, col_scale, Yt, ldy, scales, st);
    return launch_gather_t<InT, OutT, true>(p, X, ldx, F, col_scale, Yt, ldy, scales, st);
}

template <typename InT>
os_status launch_gather(const Plan *p, const InT *X, int64_t ldx, int64_t F, const float *col_scale,
                        void *Yt, os_dtype out_t, int64_t ldy, float *scales, cudaStream_t st) {
    switch (out_t) {
        case OS_F32:
            return launch_gather_o<InT, float>(p, X, ldx, F, col_scale, Yt, ldy, scales, st);
        case OS_BF16:
            return launch_gather_o<InT, __nv_bfloat16>(p, X, ldx, F, col_scale, Yt, ldy, scales, st);
        case OS_FP8E4M3:
            return launch_gather_o<InT, __nv_fp8_e4m3>(p, X, ldx, F, col_scale, Yt, ldy, scales, st);
    }
    return OS_ERR_DTYPE;
}

os_status check_out(const Plan *p, int64_t rows, void *Yt, os_dtype out_t, int64_t ldy,
                    float *scales) {
    const int64_t z = (int64_t)p->P * p->b;
    if (!Yt || rows < 0) return OS_ERR_INVALID_ARG;
    if (out_t != OS_F32 && out_t != OS_BF16 && out_t != OS_FP8E4M3) return OS_ERR_DTYPE;
    if (ldy < z) return OS_ERR_INVALID_ARG;
    if (!aligned16(Yt) || (ldy * (int64_t)dtype_size(out_t)) % 16 != 0) return OS_ERR_INVALID_ARG;
    if (out_t == OS_FP8E4M3) {
        if (!scales) return OS_ERR_INVALID_ARG;
        if (p->b % 128 != 0) return OS_ERR_UNSUPPORTED;
    }
    return OS_OK;
}

}  // namespace

size_t left_workspace_bytes(const Plan *p, int64_t m, os_dtype a_t) {
    const int64_t ldt = (m + 7) / 8 * 8;
    return (size_t)p->n * ldt * dtype_size(a_t) + 256;
}

os_status sketch_left_impl(const Plan *p, const void *A, os_dtype a_t, int64_t m, int64_t lda,
                           void *At, os_dtype out_t, int64_t ldat, float *scales,
                           const float *col_scale, void *ws, size_t ws_bytes, cudaStream_t st) {
    if (!p || !A || m < 0) return OS_ERR_INVALID_ARG;
    if (a_t != OS_F32 && a_t != OS_BF16) return OS_ERR_DTYPE;
    if (lda < p->n) return OS_ERR_INVALID_ARG;
    OSK_TRY(check_out(p, m, At, out_t, ldat, scales));
    if (m == 0) return OS_OK;
    const size_t need = left_workspace_bytes(p, m, a_t);
    if (!ws || ws_bytes < need) return OS_ERR_WORKSPACE;
    const int64_t ldt = (m + 7) / 8 * 8;
    void *Xt = reinterpret_cast<void *>((reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255));
    dim3 tg((unsigned)((p->n + 63) / 64), (unsigned)((m + 63) / 64));
    if (tg.y > 65535u) return OS_ERR_UNSUPPORTED;
    if (a_t == OS_F32) {
        transpose_kernel<float><<<tg, 256, 0, st>>>((const float *)A, lda, m, p->n, (float *)Xt, ldt);
        OSK_TRY(check_launch());
        return launch_gather<float>(p, (const float *)Xt, ldt, m, col_scale, At, out_t, ldat, scales, st);
    }
    transpose_kernel<__nv_bfloat16><<<tg, 256, 0, st>>>((const __nv_bfloat16 *)A, lda, m, p->n,
                                                       (__nv_bfloat16 *)Xt, ldt);
    OSK_TRY(check_launch());
    return launch_gather<__nv_bfloat16>(p, (const __nv_bfloat16 *)Xt, ldt, m, col_scale, At, out_t,
                                        ldat, scales, st);
}

os_status sketch_right_impl(const Plan *p, const void *B, os_dtype b_t, int64_t l, int64_t ldb,
                            void *BtT, os_dtype out_t, int64_t ldbt, float *scales, cudaStream_t st) {
    if (!p || !B || l < 0) return OS_ERR_INVALID_ARG;
    if (b_t != OS_F32 && b_t != OS_BF16) return OS_ERR_DTYPE;
    if (ldb < l) return OS_ERR_INVALID_ARG;
    OSK_TRY(check_out(p, l, BtT, out_t, ldbt, scales));
    if (l == 0) return OS_OK;
    if (b_t == OS_F32)
        return launch_gather<float>(p, (const float *)B, ldb, l, nullptr, BtT, out_t, ldbt, scales, st);
    return launch_gather<__nv_bfloat16>(p, (const __nv_bfloat16 *)B, ldb, l, nullptr, BtT, out_t, ldbt,
                                        scales, st);
}

os_status unsketch_cols_impl(const Plan *p, const float *T, int64_t m, int64_t ldt, uint64_t mask,
                             float scale, void *dX, os_dtype x_t, int64_t ldx, cudaStream_t st) {
    if (!p || !T || !dX || m < 0) return OS_ERR_INVALID_ARG;
    OSK_TRY(check_mask(mask, p->P));
    if (ldt < (int64_t)p->P * p->b || ldx < p->n) return OS_ERR_INVALID_ARG;
    if (x_t != OS_F32 && x_t != OS_BF16) return OS_ERR_DTYPE;
    if (m == 0) return OS_OK;
    if (m > 65535) return OS_ERR_UNSUPPORTED;
    const BlockList kept = mask_to_list(mask, p->P);
    const int64_t gx = (p->n + 255) / 256 < 1024 ? (p->n + 255) / 256 : 1024;
    dim3 grid((unsigned)gx, (unsigned)m);
    if (x_t == OS_F32)
        unsketch_cols_kernel<float><<<grid, 256, 0, st>>>(T, m, ldt, p->hs, p->n, p->b, kept, scale,
                                                          (float *)dX, ldx);
    else
        unsketch_cols_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(T, m, ldt, p->hs, p->n, p->b, kept,
                                                                  scale, (__nv_bfloat16 *)dX, ldx);
    return check_launch();
}

os_status unsketch_rows_impl(const Plan *p, const float *U, int64_t l, int64_t ldu, uint64_t mask,
                             float scale, void *dG, os_dtype g_t, int64_t ldg, cudaStream_t st) {
    if (!p || !U || !dG || l < 0) return OS_ERR_INVALID_ARG;
    OSK_TRY(check_mask(mask, p->P));
    if (ldu < l || ldg < l) return OS_ERR_INVALID_ARG;
    if (g_t != OS_F32 && g_t != OS_BF16) return OS_ERR_DTYPE;
    if (l == 0) return OS_OK;
    const BlockList kept = mask_to_list(mask, p->P);
    dim3 grid((unsigned)((p->n + 7) / 8), (unsigned)((l + 1023) / 1024));
    if (grid.y > 65535u) return OS_ERR_UNSUPPORTED;
    if (g_t == OS_F32)
        unsketch_rows_kernel<float><<<grid, 256, 0, st>>>(U, l, ldu, p->hs, p->n, p->b, kept, scale,
                                                          (float *)dG, ldg);
    else
        unsketch_rows_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(U, l, ldu, p->hs, p->n, p->b, kept,
                                                                  scale, (__nv_bfloat16 *)dG, ldg);
    return check_launch();
}

}  // namespace osk

using namespace osk;

extern "C" os_status oversketch_sketch_left_workspace(oversketch_plan_t plan, int64_t m,
                                                      os_dtype a_t, size_t *bytes) {
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p || !bytes || m < 0) return OS_ERR_INVALID_ARG;
    if (a_t != OS_F32 && a_t != OS_BF16) return OS_ERR_DTYPE;
    *bytes = left_workspace_bytes(p, m, a_t);
    return OS_OK;
}

extern "C" os_status oversketch_sketch_left(oversketch_plan_t plan, const void *A, os_dtype a_t,
                                            int64_t m, int64_t lda, void *At, os_dtype out_t,
                                            int64_t ldat, float *scales, const float *col_scale,
                                            void *workspace, size_t ws_bytes, void *stream) {
    return sketch_left_impl(reinterpret_cast<const Plan *>(plan), A, a_t, m, lda, At, out_t, ldat,
                            scales, col_scale, workspace, ws_bytes, as_stream(stream));
}

extern "C" os_status oversketch_sketch_right(oversketch_plan_t plan, const void *B, os_dtype b_t,
                                             int64_t l, int64_t ldb, void *BtT, os_dtype out_t,
                                             int64_t ldbt, float *scales, void *stream) {
    return sketch_right_impl(reinterpret_cast<const Plan *>(plan), B, b_t, l, ldb, BtT, out_t, ldbt,
                             scales, as_stream(stream));
}

extern "C" os_status oversketch_unsketch_cols(oversketch_plan_t plan, const float *T, int64_t m,
                                              int64_t ldt, uint64_t mask, float scale, void *dX,
                                              os_dtype x_t, int64_t ldx, void *stream) {
    return unsketch_cols_impl(reinterpret_cast<const Plan *>(plan), T, m, ldt, mask, scale, dX, x_t,
                              ldx, as_stream(stream));
}

extern "C" os_status oversketch_unsketch_rows(oversketch_plan_t plan, const float *U, int64_t l,
                                              int64_t ldu, uint64_t mask, float scale, void *dG,
                                              os_dtype g_t, int64_t ldg, void *stream) {
    return unsketch_rows_impl(reinterpret_cast<const Plan *>(plan), U, l, ldu, mask, scale, dG, g_t,
                              ldg, as_stream(stream));
}
