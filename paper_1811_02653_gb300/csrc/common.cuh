// Shared definitions of the sm_103a OverSketch library (device + host).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/oversketch.h"

namespace osk {

// Plan: the sketch S of Eq. 3 as device tables.
//   hs[j*n + i]   = h_j(i) | (sigma_j(i) < 0) << 31      (per-index lookup)
//   perm[j*n + p] = i | (sigma_j(i) < 0) << 31           (bucket-sorted, i ascending in a bucket)
//   offs[j*(b+1) + c] = start of bucket c of block j in perm[j*n ...]; offs[.. + b] = n
//   pperm/poffs: the same lists with every bucket padded to a multiple of 4
//   entries by kPadEntry (zero weight), so that the gather kernels can take
//   members four at a time from one bucket; block j's list starts at
//   pperm + j*pstride.
struct Plan {
    int64_t n;
    int32_t b, N, e, P;
    uint64_t seed;
    uint32_t *hs;
    uint32_t *perm;
    uint32_t *offs;
    uint32_t *pperm;
    uint32_t *poffs;
    int64_t pstride;
    int32_t hashed;   // 1: hs is the seeded hash below (oversketch_plan); 0: tables given by the caller
    int device;
};

constexpr uint32_t kSignBit = 0x80000000u;
constexpr uint32_t kIndexMask = 0x7fffffffu;
constexpr uint32_t kPadEntry = 0x7fffffffu;   // padding entry: no index (n < 2^31 - 1)

// Kept blocks of a mask as a list (launch parameter, passed by value).
struct BlockList {
    int32_t count;
    int32_t idx[64];
};

os_status set_cuda_error(cudaError_t err);
os_status check_launch();
BlockList mask_to_list(uint64_t mask, int P);
os_status check_mask(uint64_t mask, int P);

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// NVTX range over a host call (plan, sketches, GEMM, product): shows the path's
// phases on a profiler timeline; a no-op when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define OSK_NVTX(name) ::osk::NvtxRange osk_nvtx_range_(name)

inline size_t dtype_size(os_dtype t) {   // bytes per element of one plane
    return (t == OS_F32 || t == OS_TF32X2) ? 4 : (t == OS_BF16 ? 2 : 1);
}

// Output tag of the sketch kernels for OS_TF32X2 (two FP32 planes hi, lo).
struct Tf32Pair {
    float v;
};

#ifdef __CUDACC__
// The plan's hash (Alg. 4 steps 1-2 made concrete): splitmix64's finaliser used
// as a counter-based generator.  key_j = mix(seed + (j+1) gamma) per block,
// w = mix(key_j + (i+1) gamma) per index, h_j(i) = ((w >> 32) * b) >> 32,
// sigma_j(i) = -1 when w is odd.  Returned as h | sign << 31, the layout of hs.
constexpr uint64_t kSplitmixGamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

__device__ __forceinline__ uint64_t block_key(uint64_t seed, int j) {
    return splitmix_mix(seed + (uint64_t)(j + 1) * kSplitmixGamma);
}

__device__ __forceinline__ uint32_t hash_code(uint64_t key, int64_t i, int32_t b) {
    const uint64_t w = splitmix_mix(key + (uint64_t)(i + 1) * kSplitmixGamma);
    const uint32_t h = (uint32_t)(((w >> 32) * (uint64_t)(uint32_t)b) >> 32);
    return h | ((w & 1ull) ? kSignBit : 0u);
}

// FP8 block scale of the sketch outputs: the smallest e with amax <= 448 * 2^e
// (exact), clamped to the UE8M0 range; 0 for an all-zero slice.
__device__ __forceinline__ int fp8_scale_exponent(float amax) {
    if (!(amax > 0.f)) return 0;
    int E;
    const float m = frexpf(amax, &E);   // amax = m * 2^E, m in [0.5, 1)
    int e = (m <= 0.875f) ? E - 9 : E - 8;
    return e < -127 ? -127 : (e > 127 ? 127 : e);
}
#endif

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// FP8 scales are stored slice-major: entry [t, r] (slice t of z/128, row r) at
// t * fp8_scale_ld(rows) + r, rows padded to a multiple of 4 so that every
// slice starts on a 16-byte boundary.
inline int64_t fp8_scale_ld(int64_t rows) { return (rows + 3) / 4 * 4; }

}  // namespace osk

#define OSK_CUDA_TRY(expr)                                      \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) return ::osk::set_cuda_error(_e); \
    } while (0)

#define OSK_TRY(expr)                        \
    do {                                     \
        os_status _s = (expr);               \
        if (_s != OS_OK) return _s;          \
    } while (0)
