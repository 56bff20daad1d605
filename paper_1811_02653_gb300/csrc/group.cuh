// Descriptors of a grouped (many-product) masked GEMM launch: shared by the
// GEMM translation unit and the batched-product driver.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace osk {

// Products per grouped launch (the tile-start table is staged in shared memory).
constexpr int kMaxGroup = 1024;

// One product C_p = alpha_p * sum over its kept blocks of A_blk B_blk^T (+ beta_p C_p),
// in device memory (CUtensorMap members keep the tensor maps on the
// boundaries TMA requires).
struct GroupProblem {
    CUtensorMap ta;            // A: m x zK, K-major
    CUtensorMap tb;            // B: l x zK, K-major, box of the launch's tile width
    float *C;
    int64_t m, l, ldc;
    float alpha, beta;         // with dmask: alpha is multiplied by 1/popcount(*dmask) in the kernel
    int32_t b, kb_per_blk;
    int32_t P;                 // sketch blocks of the product's plan
    int32_t tiles_m, tiles_n;
    int32_t tile_begin;        // first global tile index of this product
    uint64_t mask;             // kept sketch blocks (when dmask is null)
    const uint64_t *dmask;     // device word holding the kept blocks, read at run time, or null
};

// Kept blocks of a product as the kernel sees them: the device word when given
// (bits >= P ignored), else the mask fixed at creation.
__device__ __forceinline__ uint64_t group_mask(const GroupProblem *gp) {
    const uint64_t pm = gp->P >= 64 ? ~0ull : ((1ull << gp->P) - 1ull);
    return gp->dmask ? (*gp->dmask & pm) : gp->mask;
}

// Tile widths a grouped BF16 launch can use (picked per batch by timing).
enum GroupTile { kGroupBN256 = 0, kGroupBN128 = 1 };

// Fill one descriptor (host side; builds the tensor maps).  A, B: BF16, K-major.
os_status group_problem_bf16(GroupProblem *gp, GroupTile tile, const void *A, int64_t lda, const void *B,
                             int64_t ldb, int64_t m, int64_t l, int64_t zK, int32_t blk, int32_t P, uint64_t mask,
                             const uint64_t *dmask, float alpha, float beta, float *C, int64_t ldc);

// Kernel attributes of the grouped launches; call once before any stream
// capture that records gemm_grouped_bf16.
os_status gemm_grouped_prepare();

// One persistent launch over all tiles of `count` products (descriptors in
// device memory, tile_begin ascending from 0, total_tiles in all).
os_status gemm_grouped_bf16(const GroupProblem *probs, int32_t count, int32_t total_tiles, GroupTile tile,
                            cudaStream_t st);

}  // namespace osk
