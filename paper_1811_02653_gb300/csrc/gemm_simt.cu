// FP32 masked block-sum GEMM on the CUDA cores (FFMA), the FP32-accuracy
// path of Alg. 3's computation and reduction phases:
//
//   C[r, c] = alpha * sum_{j kept} sum_{q < b} At[r, j*b + q] * BtT[c, j*b + q] + beta * C[r, c]
//
// Both operands are K-major (the sketched dimension is contiguous).  The K
// loop runs over the concatenation of the kept blocks; a 16-wide K tile never
// straddles two blocks because b % 16 == 0, so tile t starts at column
// kept[t*16 / b]*b + (t*16 mod b).  128 x 128 output tile per CTA, 8 x 8 per
// thread, register-staged double buffering of the shared tiles.
#include "common.cuh"

namespace osk {

namespace {

constexpr int BM = 128, BN = 128, BK = 16, PAD = 4;

__global__ void __launch_bounds__(256)
gemm_masked_f32_kernel(const float *__restrict__ A, int64_t lda, const float *__restrict__ B,
                       int64_t ldb, int64_t m, int64_t l, int32_t b, BlockList kept, float alpha,
                       float beta, float *__restrict__ C, int64_t ldc) {
    __shared__ __align__(16) float As[2][BK][BM + PAD];
    __shared__ __align__(16) float Bs[2][BK][BN + PAD];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t r0 = (int64_t)blockIdx.y * BM, c0 = (int64_t)blockIdx.x * BN;
    const int K = kept.count * b;
    const int ktiles = K / BK;

    // loader mapping: 128 rows x 16 k = 512 float4; thread loads 2 float4
    const int lr = tid >> 1;            // 0..127
    const int lk = (tid & 1) * 8;       // 0 or 8
    float4 ra[2], rb[2];

    auto kbase = [&](int t) -> int64_t {
        const int kk = t * BK;
        const int blk = kk / b;
        return (int64_t)kept.idx[blk] * b + (kk - blk * b);
    };
    auto load = [&](int t) {
        const int64_t kb = kbase(t) + lk;
        const int64_t ar = r0 + lr, bc = c0 + lr;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            ra[u] = ar < m ? __ldg(reinterpret_cast<const float4 *>(A + ar * lda + kb + 4 * u))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
            rb[u] = bc < l ? __ldg(reinterpret_cast<const float4 *>(B + bc * ldb + kb + 4 * u))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            As[buf][lk + 4 * u + 0][lr] = ra[u].x;
            As[buf][lk + 4 * u + 1][lr] = ra[u].y;
            As[buf][lk + 4 * u + 2][lr] = ra[u].z;
            As[buf][lk + 4 * u + 3][lr] = ra[u].w;
            Bs[buf][lk + 4 * u + 0][lr] = rb[u].x;
            Bs[buf][lk + 4 * u + 1][lr] = rb[u].y;
            Bs[buf][lk + 4 * u + 2][lr] = rb[u].z;
            Bs[buf][lk + 4 * u + 3][lr] = rb[u].w;
        }
    };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    if (ktiles > 0) {
        load(0);
        store(0);
    }
    __syncthreads();
    for (int t = 0; t < ktiles; ++t) {
        const int buf = t & 1;
        if (t + 1 < ktiles) load(t + 1);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][k][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (t + 1 < ktiles) store(buf ^ 1);
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = r0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t c = c0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            if (c >= l) continue;
            float v = alpha * acc[i][j];
            if (beta != 0.f) v = fmaf(beta, C[r * ldc + c], v);
            C[r * ldc + c] = v;
        }
    }
}

}  // namespace

os_status gemm_masked_f32(const Plan *p, const float *At, int64_t ldat, const float *BtT,
                          int64_t ldbt, int64_t m, int64_t l, uint64_t mask, float alpha, float beta,
                          float *C, int64_t ldc, cudaStream_t st) {
    if (p->b % BK != 0) return OS_ERR_UNSUPPORTED;
    if (!aligned16(At) || !aligned16(BtT) || ldat % 4 != 0 || ldbt % 4 != 0)
        return OS_ERR_INVALID_ARG;
    const BlockList kept = mask_to_list(mask, p->P);
    dim3 grid((unsigned)((l + BN - 1) / BN), (unsigned)((m + BM - 1) / BM));
    if (grid.y > 65535u) return OS_ERR_UNSUPPORTED;
    gemm_masked_f32_kernel<<<grid, 256, 0, st>>>(At, ldat, BtT, ldbt, m, l, p->b, kept, alpha, beta,
                                                 C, ldc);
    return check_launch();
}

}  // namespace osk
