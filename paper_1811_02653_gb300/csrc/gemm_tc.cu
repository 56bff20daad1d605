// Masked block-sum GEMM on the 5th-generation tensor cores (sm_103a).
//
// Alg. 3's computation phase multiplies b x b blocks of A~ and B~, its
// termination rule keeps any k of the N+e blocks of the inner dimension, and
// Alg. 2's reduction phase adds the kept partial products.  On one GPU this
// is a single GEMM whose K loop walks the concatenation of the kept blocks:
//
//   C[r, c] = alpha * sum_{j kept} sum_{q < b} At[r, j*b + q] * BtT[c, j*b + q]  (+ beta * C)
//
// K block kb of the loop (one 128-byte row of K per operand row: 64 BF16, 32
// TF32 or 128 FP8 values) is read by TMA at sketched column
// kept[kb / (b/BK)] * b + (kb mod (b/BK)) * BK, so dropped blocks are never
// loaded.  Operands are K-major in the 128-byte swizzled layout.
//
// Kernel organisation (one persistent CTA per SM):
//   warp 0      TMA producer: ring of {A 128 x BK, B BN x BK} stages (FP8 stages
//               also carry the A and B scale rows of their 128-wide K slice)
//   warp 1      TMEM owner + MMA issuer: tcgen05.mma 128 x BN per K step, FP32
//               accumulators in TMEM, double-buffered
//   warps 2..5  epilogue: tcgen05.ld of the accumulator, alpha / beta, FP32
//               stores; overlaps the next tile's MMAs
//   warp 6      (FP8) converts each stage's FP32 scales to UE8M0 bytes in the
//               layout tcgen05.cp copies to TMEM for the block-scaled MMA
// Every mbarrier wait is bounded (1 s); on expiry the kernel records
// OS_ERR_TIMEOUT in the device status word, drains its own copies and MMAs,
// frees TMEM and returns.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "group.cuh"
#include "tc_common.cuh"

namespace osk {

namespace {

using namespace tc;

constexpr int BM = 128;
constexpr int ROWB = 128;                     // bytes per tile row: one 128-byte swizzle row

// Operand kinds.  Bf16: BF16 operands, 64 K-elements per 128-byte stage row,
// tcgen05 kind::f16.  Tf32x3: FP32 operands given as two TF32-exact planes
// hi/lo (32 K-elements per stage row, kind::tf32, three products hi.hi +
// hi.lo + lo.hi per K step: FP32-level accuracy on the tensor cores).  Fp8:
// E4M3 operands with one power-of-two scale per (row, 128-element K slice),
// 128 K-elements per stage row, kind::mxf8f6f4 with UE8M0 block scaling.
enum class Kind { Bf16, Tf32x3, Fp8 };

template <int kBN, int kStages, Kind kKind>
struct Cfg {
    static constexpr int BN = kBN;
    static constexpr int STAGES = kStages;
    static constexpr bool FP8 = kKind == Kind::Fp8;
    static constexpr int PLANES = kKind == Kind::Tf32x3 ? 2 : 1;
    static constexpr int ELEM = kKind == Kind::Bf16 ? 2 : (kKind == Kind::Tf32x3 ? 4 : 1);   // bytes
    static constexpr int BKE = ROWB / ELEM;                    // K elements per stage
    static constexpr int A_BYTES = BM * ROWB;                  // one plane of A
    static constexpr int B_BYTES = BN * ROWB;                  // one plane of B
    static constexpr int TILE_BYTES = PLANES * (A_BYTES + B_BYTES);
    // FP8 only: the stage's FP32 scale rows (loaded by TMA) and their UE8M0
    // copies in the 32 x 16-byte chunk layout that tcgen05.cp moves to TMEM
    // (chunk c holds rows 128c .. 128c+127: row r at byte 16 (r % 32) + 4 (r / 32)).
    static constexpr int SA_BYTES = FP8 ? BM * 4 : 0;
    static constexpr int SB_BYTES = FP8 ? BN * 4 : 0;
    static constexpr int SFB_CHUNKS = (BN + 127) / 128;
    static constexpr int CHUNK_BYTES = FP8 ? 512 * (1 + SFB_CHUNKS) : 0;
    static constexpr int TX_BYTES = TILE_BYTES + SA_BYTES + SB_BYTES;
    static constexpr int STAGE_BYTES = (TX_BYTES + CHUNK_BYTES + 1023) / 1024 * 1024;
    // TMEM: two accumulators of BN columns.  FP8 places them 256 columns apart
    // and keeps one 16-column scale slot per stage in the gaps behind them.
    static constexpr int ACC_STRIDE = FP8 ? 256 : BN;
    static constexpr int TMEM_COLS = FP8 ? 512 : 2 * BN;
    static constexpr int SF_GAP_SLOTS = (256 - BN) / 16;
    static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE_BYTES + 256;
    // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue; FP8 adds warp 6, which turns
    // each stage's FP32 scales into UE8M0 chunks ahead of the MMA warp
    static constexpr int THREADS = FP8 ? 224 : 192;
    static constexpr uint32_t IDESC = kKind == Kind::Bf16     ? idesc_bf16_f32(BM, BN)
                                      : kKind == Kind::Tf32x3 ? idesc_tf32_f32(BM, BN)
                                                              : idesc_mxf8_f32(BM, BN);
    // 3xTF32: the tensor core accumulates each chunk of CHUNK_KB K blocks (K = 256)
    // in TMEM and the epilogue adds the chunks in FP32 registers, so the
    // accumulation error does not grow with K.  Otherwise one chunk per tile.
    static constexpr int CHUNK_KB = kKind == Kind::Tf32x3 ? 8 : (1 << 30);
    static_assert(!FP8 || (BN <= 240 && 2 * SF_GAP_SLOTS >= STAGES), "FP8 scale slots do not fit in TMEM");
    static_assert(BN % 32 == 0 && BN <= 256, "tile width");
    static_assert(SMEM <= 232448, "shared memory");

    // TMEM column of stage s's scale slot (A scales at +0..3, B scales at +4..)
    __host__ __device__ static constexpr uint32_t sf_slot(int s) {
        return s < SF_GAP_SLOTS ? (uint32_t)(BN + 16 * s) : (uint32_t)(256 + BN + 16 * (s - SF_GAP_SLOTS));
    }
};

using CfgBf16 = Cfg<256, 4, Kind::Bf16>;        // grouped launches (single products run on CTA pairs)
using CfgBf16N128 = Cfg<128, 6, Kind::Bf16>;   // narrower tiles for grouped launches of small products
using CfgTf32x3 = Cfg<128, 3, Kind::Tf32x3>;
using CfgFp8 = Cfg<224, 4, Kind::Fp8>;

// UE8M0 code of a power-of-two FP32 scale in [2^-127, 2^127] (its biased
// exponent field; 2^-127 is the subnormal with exponent field 0), in all four bytes.
__device__ __forceinline__ uint32_t ue8m0_x4(float s) {
    return ((__float_as_uint(s) >> 23) & 0xffu) * 0x01010101u;
}

struct GemmArgs {
    const GroupProblem *group;   // grouped launch: product descriptors (else null)
    int32_t group_count;
    int64_t m, l;
    int32_t b;            // block width (multiple of the stage's K elements)
    int32_t kb_per_blk;   // b / BKE
    int32_t num_kb;       // k * b / BKE
    int32_t tiles_m, tiles_n, num_tiles;
    float alpha, beta;
    float *C;
    int64_t ldc;
    BlockList kept;
    // per-block masks (CTA-pair kernel): block (i, j) of C is bm x bn, its kept set
    // block_masks[i * nbc + j] (bits >= P ignored); null: `kept` for every tile
    const uint64_t *block_masks;
    int64_t bm, bn;
    int32_t nbc, P;
    // CTA-pair kernel, C = A A^T (B is A): only the tile pairs on and below the
    // diagonal are computed; each off-diagonal one is also stored transposed
    int32_t sym;
    // CTA-pair kernel with MN-major operands: for the operands flagged in mn_remap
    // (1: A, 2: B) row/column q of C comes from column mn_kept[q / mn_b] * mn_b +
    // q % mn_b of the operand (its listed blocks of width mn_b, P of them stored)
    int32_t mn_b, mn_remap;
    BlockList mn_kept;
};

// Tile pair t of the lower triangle (row-major: pair row pm, tile column tn <= pm).
__device__ __forceinline__ void tri_coords(int t, int &pm, int &tn) {
    int r = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    pm = r;
    tn = t - r * (r + 1) / 2;
}

__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int &tm, int &tn) {
    // Groups of 16 m-tiles: consecutive tiles share A panels and nearby B panels.
    constexpr int G = 16;
    const int group = t / (G * tiles_n);
    const int first_m = group * G;
    const int gm = min(G, tiles_m - first_m);
    const int in = t - group * G * tiles_n;
    tm = first_m + in % gm;
    tn = in / gm;
}

// Product owning global tile t of a grouped launch: the last p with begin[p] <= t.
__device__ __forceinline__ int find_problem(const int32_t *begin, int count, int t) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Everything one role needs to know about a tile.
struct TileJob {
    const CUtensorMap *ta, *tb;
    uint64_t mask;                // grouped launches: kept sketch blocks (bit j = block j)
    int tm, tn;
    int num_kb, kb_per_blk, b;
    float *C;
    int64_t m, l, ldc;
    float alpha, beta;
};

// tmap_a0/b0: BF16 or E4M3 operands, or the TF32 hi planes.  tmap_a1/b1: the
// TF32 lo planes, or for FP8 the slice-major FP32 scale arrays.  GROUPED: the
// tiles of g.group_count products (descriptors g.group, tile_begin ascending)
// share one persistent launch; the tensor maps come from the descriptors.
template <class C, bool GROUPED>
__global__ void __launch_bounds__(C::THREADS, 1)
gemm_masked_tc_kernel(const __grid_constant__ CUtensorMap tmap_a0, const __grid_constant__ CUtensorMap tmap_b0,
                      const __grid_constant__ CUtensorMap tmap_a1, const __grid_constant__ CUtensorMap tmap_b1,
                      const GemmArgs g) {
    constexpr int STAGES = C::STAGES, BN = C::BN, BKE = C::BKE;
    static_assert(!GROUPED || C::PLANES == 1 && !C::FP8, "grouped launches take BF16 operands");
    extern __shared__ uint8_t smem_raw[];
    __shared__ int32_t s_begin[GROUPED ? kMaxGroup : 1];   // first tile of each product
    // 1024-byte alignment for the swizzled tiles
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    // stage s: [A plane 0][A plane 1][B plane 0][B plane 1] | FP8: [A scales][B scales][UE8M0 chunks]
    uint8_t *tiles = smem;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * C::STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *tmem_full = empty + STAGES;
    uint64_t *tmem_empty = tmem_full + 2;
    uint64_t *drain = tmem_empty + 2;
    uint64_t *sf_ready = drain + 1;    // FP8: stage's scale chunks written (STAGES barriers)
    uint32_t *tmem_base_slot = reinterpret_cast<uint32_t *>(sf_ready + STAGES);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_base_slot + 1);
    // test hook (first CTA only): a K step of the first tile left unloaded, and this
    // CTA's wait limit
    __shared__ int s_skip_kb;
    __shared__ unsigned long long s_wait_ns;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if constexpr (GROUPED)
        for (int i = threadIdx.x; i < g.group_count; i += blockDim.x) s_begin[i] = g.group[i].tile_begin;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tmem_full[a], 1);
            mbar_init(&tmem_empty[a], 128);
        }
        mbar_init(drain, 1);
        for (int s = 0; s < STAGES; ++s) mbar_init(&sf_ready[s], 1);
        *abort = 0;
        s_skip_kb = -1;
        s_wait_ns = kWaitLimitNs;
        if (blockIdx.x == 0 && *(volatile int *)&g_test_skip_kb >= 0) {
            s_skip_kb = atomicExch(&g_test_skip_kb, -1);   // one-shot
            s_wait_ns = *(volatile unsigned long long *)&g_test_wait_ns;
        }
        fence_barrier_init();
        if constexpr (!GROUPED) {
            prefetch_tmap(&tmap_a0);
            prefetch_tmap(&tmap_b0);
            if (C::PLANES == 2 || C::FP8) {
                prefetch_tmap(&tmap_a1);
                prefetch_tmap(&tmap_b1);
            }
        }
    }
    if (warp == 1) tmem_alloc(tmem_base_slot, C::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_base_slot;
    const int skip_kb = s_skip_kb;
    const unsigned long long wait_ns = s_wait_ns;

    // The tile's product, coordinates and epilogue parameters.
    auto job = [&](int t) {
        TileJob j;
        if constexpr (GROUPED) {
            const int p = find_problem(s_begin, g.group_count, t);
            const GroupProblem *P = g.group + p;
            tile_coords(t - s_begin[p], P->tiles_m, P->tiles_n, j.tm, j.tn);
            j.ta = &P->ta;
            j.tb = &P->tb;
            j.mask = group_mask(P);
            const int k = __popcll(j.mask);
            j.num_kb = k * P->kb_per_blk;
            j.kb_per_blk = P->kb_per_blk;
            j.b = P->b;
            j.C = P->C;
            j.m = P->m;
            j.l = P->l;
            j.ldc = P->ldc;
            // a run-time mask brings its own 1/k; an empty one gives a zero product
            j.alpha = P->dmask ? (k ? P->alpha / (float)k : 0.f) : P->alpha;
            j.beta = P->beta;
        } else {
            tile_coords(t, g.tiles_m, g.tiles_n, j.tm, j.tn);
            j.ta = &tmap_a0;
            j.tb = &tmap_b0;
            j.mask = 0;                   // read g.kept directly (no copy of the parameter)
            j.num_kb = g.num_kb;
            j.kb_per_blk = g.kb_per_blk;
            j.b = g.b;
            j.C = g.C;
            j.m = g.m;
            j.l = g.l;
            j.ldc = g.ldc;
            j.alpha = g.alpha;
            j.beta = g.beta;
        }
        return j;
    };
    auto num_kb_of = [&](int t) -> int {
        if constexpr (GROUPED) {
            const GroupProblem *P = g.group + find_problem(s_begin, g.group_count, t);
            return __popcll(group_mask(P)) * P->kb_per_blk;
        } else {
            return g.num_kb;
        }
    };

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued_phase[STAGES];
            bool issued[STAGES];
            for (int s = 0; s < STAGES; ++s) issued[s] = false, issued_phase[s] = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < g.num_tiles; t += gridDim.x) {
                const TileJob j = job(t);
                uint64_t rest = j.mask;          // grouped: kept blocks not yet started
                int kidx = 0;
                if constexpr (GROUPED) {
                    // the descriptors' tensor maps may have been written by a kernel
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(j.ta) : "memory");
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(j.tb) : "memory");
                }
                for (int kb = 0; kb < j.num_kb; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, abort, wait_ns)) { ok = false; break; }
                    const int blk = kb / j.kb_per_blk;
                    const int kin = kb - blk * j.kb_per_blk;
                    if constexpr (GROUPED) {
                        if (kin == 0) {
                            kidx = __ffsll((long long)rest) - 1;
                            rest &= rest - 1;
                        }
                    } else {
                        kidx = g.kept.idx[blk];
                    }
                    if (t == blockIdx.x && kb == skip_kb) {
                        // test hook: this stage is never loaded nor armed, so the
                        // MMA warp's wait for it runs out
                        if (++stage == STAGES) stage = 0, phase ^= 1u;
                        continue;
                    }
                    const int kz = kidx * j.b + kin * BKE;
                    uint8_t *st = tiles + stage * C::STAGE_BYTES;
                    mbar_expect_tx(&full[stage], C::TX_BYTES);
                    tma_load_2d(j.ta, &full[stage], st, kz, j.tm * BM);
                    if (C::PLANES == 2) tma_load_2d(&tmap_a1, &full[stage], st + C::A_BYTES, kz, j.tm * BM);
                    uint8_t *sb = st + C::PLANES * C::A_BYTES;
                    tma_load_2d(j.tb, &full[stage], sb, kz, j.tn * BN);
                    if (C::PLANES == 2) tma_load_2d(&tmap_b1, &full[stage], sb + C::B_BYTES, kz, j.tn * BN);
                    if (C::FP8) {
                        // scale rows of K slice kz / 128 (one stage = one slice)
                        tma_load_2d(&tmap_a1, &full[stage], st + C::TILE_BYTES, j.tm * BM, kz / 128);
                        tma_load_2d(&tmap_b1, &full[stage], st + C::TILE_BYTES + C::SA_BYTES, j.tn * BN, kz / 128);
                    }
                    issued[stage] = true;
                    issued_phase[stage] = phase;
                    if (++stage == STAGES) stage = 0, phase ^= 1u;
                }
            }
            // Drain: every copy this thread issued must have landed before exit.
            for (int s = 0; s < STAGES; ++s)
                if (issued[s]) mbar_wait_drain(&full[s], issued_phase[s]);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (lane 0 issues; the warp waits together) ----------------
        int stage = 0;
        uint32_t phase = 0;
        int iter = 0;
        bool ok = true;
        bool any = false;
        for (int t = blockIdx.x; ok && t < g.num_tiles; t += gridDim.x) {
          const int num_kb = num_kb_of(t);
          if (GROUPED && num_kb == 0) {
              // a product whose run-time mask keeps no block: hand the epilogue an
              // accumulator (no MMA issued; it writes zeros)
              const int a = iter & 1;
              const uint32_t aphase = (uint32_t)(iter >> 1) & 1u;
              ++iter;
              if (!__all_sync(0xffffffffu, mbar_wait(&tmem_empty[a], aphase ^ 1u, abort, wait_ns))) { ok = false; break; }
              tc_fence_after();
              if (lane == 0) umma_commit(&tmem_full[a]);
              __syncwarp();
              continue;
          }
          for (int kc = 0; ok && kc < num_kb; kc += C::CHUNK_KB, ++iter) {
            const int kc_end = min(num_kb, kc + C::CHUNK_KB);
            const int a = iter & 1;
            const uint32_t aphase = (uint32_t)(iter >> 1) & 1u;
            if (!__all_sync(0xffffffffu, mbar_wait(&tmem_empty[a], aphase ^ 1u, abort, wait_ns))) { ok = false; break; }
            tc_fence_after();
            const uint32_t d = tmem_base + (uint32_t)(a * C::ACC_STRIDE);
            for (int kb = kc; kb < kc_end; ++kb) {
                // FP8: the converter warp signals sf_ready once the stage's tiles have
                // landed and its scale chunks are written
                uint64_t *ready = C::FP8 ? &sf_ready[stage] : &full[stage];
                if (!__all_sync(0xffffffffu, mbar_wait(ready, phase, abort, wait_ns))) { ok = false; break; }
                tc_fence_after();
                uint8_t *st = tiles + stage * C::STAGE_BYTES;
                const uint32_t sa0 = smem_u32(st);
                const uint32_t sb0 = sa0 + C::PLANES * C::A_BYTES;
                uint32_t sfa = 0, sfb = 0;
                if constexpr (C::FP8) {
                    sfa = tmem_base + C::sf_slot(stage);
                    sfb = sfa + 4;
                    if (lane == 0) {
                        uint8_t *ch = st + C::TX_BYTES;
                        tmem_cp_32x128b_x4(sfa, sdesc_rows16(smem_u32(ch)));
#pragma unroll
                        for (int c = 0; c < C::SFB_CHUNKS; ++c)
                            tmem_cp_32x128b_x4(sfb + 4 * c, sdesc_rows16(smem_u32(ch + 512 * (1 + c))));
                    }
                }
                if (lane == 0) {
#pragma unroll
                    for (int kk = 0; kk < ROWB / 32; ++kk) {
                        const uint32_t acc0 = (kb > kc || kk > 0) ? 1u : 0u;
                        const uint64_t ad = sdesc_kmajor_sw128(sa0 + kk * 32);
                        const uint64_t bd = sdesc_kmajor_sw128(sb0 + kk * 32);
                        if constexpr (C::FP8) {
                            umma_mxf8(d, ad, bd, C::IDESC, sfa, sfb, acc0);
                        } else if constexpr (C::PLANES == 1) {
                            umma_f16(d, ad, bd, C::IDESC, acc0);
                        } else {
                            const uint64_t adl = sdesc_kmajor_sw128(sa0 + C::A_BYTES + kk * 32);
                            const uint64_t bdl = sdesc_kmajor_sw128(sb0 + C::B_BYTES + kk * 32);
                            umma_tf32(d, ad, bd, C::IDESC, acc0);     // hi . hi
                            umma_tf32(d, ad, bdl, C::IDESC, 1u);      // hi . lo
                            umma_tf32(d, adl, bd, C::IDESC, 1u);      // lo . hi
                        }
                    }
                    umma_commit(&empty[stage]);
                }
                __syncwarp();
                any = true;
                if (++stage == STAGES) stage = 0, phase ^= 1u;
            }
            if (!ok) break;
            if (lane == 0) umma_commit(&tmem_full[a]);
          }
        }
        if (!ok && any && lane == 0) {
            // Drain: wait for the MMAs already issued before freeing TMEM.
            umma_commit(drain);
            mbar_wait_drain(drain, 0);
        }
    } else if (warp == 6) {
        // ---------------- FP8 scale converter ----------------
        // FP32 scales -> UE8M0 bytes in the chunk layout; lane i owns chunk row i
        if constexpr (C::FP8) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < g.num_tiles; t += gridDim.x) {
                const int num_kb = num_kb_of(t);
                for (int kb = 0; kb < num_kb; ++kb) {
                    if (!__all_sync(0xffffffffu, mbar_wait(&full[stage], phase, abort, wait_ns))) { ok = false; break; }
                    uint8_t *st = tiles + stage * C::STAGE_BYTES;
                    const float *fa = reinterpret_cast<const float *>(st + C::TILE_BYTES);
                    const float *fb = fa + BM;
                    uint8_t *ch = st + C::TX_BYTES;
                    *reinterpret_cast<uint4 *>(ch + 16 * lane) =
                        make_uint4(ue8m0_x4(fa[lane]), ue8m0_x4(fa[lane + 32]), ue8m0_x4(fa[lane + 64]),
                                   ue8m0_x4(fa[lane + 96]));
#pragma unroll
                    for (int c = 0; c < C::SFB_CHUNKS; ++c) {
                        uint32_t w[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int row = 128 * c + 32 * q + lane;
                            w[q] = row < BN ? ue8m0_x4(fb[row]) : 0x7f7f7f7fu;
                        }
                        *reinterpret_cast<uint4 *>(ch + 512 * (1 + c) + 16 * lane) = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                    fence_proxy_async_smem();   // generic-proxy writes -> tcgen05.cp reads
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sf_ready[stage]);
                    if (++stage == STAGES) stage = 0, phase ^= 1u;
                }
            }
        }
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        const int quarter = warp & 3;                 // TMEM lanes 32*quarter .. +31
        const int row_in_tile = quarter * 32 + lane;
        int iter = 0;
        // FP32 store of 32 consecutive values of row r starting at column cbase
        auto store32 = [&](const TileJob &j, bool vec_ok, int64_t r, int64_t cbase, const float *val) {
            if (r >= j.m) return;
            float *dst = j.C + r * j.ldc + cbase;
            if (vec_ok && cbase + 32 <= j.l) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    float4 o = make_float4(j.alpha * val[4 * u + 0], j.alpha * val[4 * u + 1],
                                           j.alpha * val[4 * u + 2], j.alpha * val[4 * u + 3]);
                    if (j.beta != 0.f) {
                        const float4 old = *reinterpret_cast<const float4 *>(dst + 4 * u);
                        o.x = fmaf(j.beta, old.x, o.x);
                        o.y = fmaf(j.beta, old.y, o.y);
                        o.z = fmaf(j.beta, old.z, o.z);
                        o.w = fmaf(j.beta, old.w, o.w);
                    }
                    *reinterpret_cast<float4 *>(dst + 4 * u) = o;
                }
            } else {
#pragma unroll
                for (int u = 0; u < 32; ++u) {
                    if (cbase + u < j.l) {
                        float o = j.alpha * val[u];
                        if (j.beta != 0.f) o = fmaf(j.beta, dst[u], o);
                        dst[u] = o;
                    }
                }
            }
        };
        bool ok = true;
        for (int t = blockIdx.x; ok && t < g.num_tiles; t += gridDim.x) {
            const TileJob j = job(t);
            const bool vec_ok = ((reinterpret_cast<uintptr_t>(j.C) & 15u) == 0) && (j.ldc % 4 == 0);
            const int64_t r = (int64_t)j.tm * BM + row_in_tile;
            const int64_t c0 = (int64_t)j.tn * BN;
            if constexpr (C::CHUNK_KB < (1 << 30)) {
                // chunked accumulation: running FP32 sum of the tile row in registers
                float total[BN];
#pragma unroll
                for (int u = 0; u < BN; ++u) total[u] = 0.f;
                for (int kc = 0; kc < j.num_kb; kc += C::CHUNK_KB, ++iter) {
                    const int a = iter & 1;
                    const uint32_t aphase = (uint32_t)(iter >> 1) & 1u;
                    // warp-uniform decision: tcgen05.ld below is a .sync.aligned instruction
                    if (!__all_sync(0xffffffffu, mbar_wait(&tmem_full[a], aphase, abort, wait_ns))) { ok = false; break; }
                    tc_fence_after();
#pragma unroll
                    for (int ch = 0; ch < BN / 32; ++ch) {
                        uint32_t v[32];
                        tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) +
                                               (uint32_t)(a * C::ACC_STRIDE + ch * 32), v);
#pragma unroll
                        for (int u = 0; u < 32; ++u) total[ch * 32 + u] += __uint_as_float(v[u]);
                    }
                    tc_fence_before();
                    mbar_arrive(&tmem_empty[a]);
                }
                if (!ok) break;
#pragma unroll
                for (int ch = 0; ch < BN / 32; ++ch) store32(j, vec_ok, r, c0 + ch * 32, total + ch * 32);
            } else {
                const int a = iter & 1;
                const uint32_t aphase = (uint32_t)(iter >> 1) & 1u;
                ++iter;
                if (!__all_sync(0xffffffffu, mbar_wait(&tmem_full[a], aphase, abort, wait_ns))) break;
                tc_fence_after();
                for (int ch = 0; ch < BN / 32; ++ch) {
                    uint32_t v[32];
                    if (j.num_kb > 0) {
                        tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) +
                                               (uint32_t)(a * C::ACC_STRIDE + ch * 32), v);
                    } else {
#pragma unroll
                        for (int u = 0; u < 32; ++u) v[u] = 0u;   // no kept block: a zero product
                    }
                    store32(j, vec_ok, r, c0 + ch * 32, reinterpret_cast<const float *>(v));
                }
                tc_fence_before();
                mbar_arrive(&tmem_empty[a]);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, C::TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------
// BF16 masked GEMM on CTA pairs (cta_group::2).  A pair of CTAs on two SMs
// computes a 256 x 256 tile: CTA r stages rows 128r .. 128r+127 of the tile's A
// panel and rows 128r .. 128r+127 of its B panel; the even CTA (the leader)
// issues one 256 x 256 x 16 MMA per K slice that reads both CTAs' shared memory
// and accumulates into both CTAs' TMEM (each holds its 128 rows x 256 columns).
// A K step thus writes and reads 32 KB of each SM's shared memory per 512
// tensor clocks instead of 48 KB, which is what bounds the one-CTA kernel.
//   warp 0      TMA producer of this CTA's half (completion on the leader's barrier)
//   warp 1      TMEM (both CTAs, jointly); MMA issue and commits (leader)
//   warps 2..5  epilogue of this CTA's 128 rows; release the accumulator on the leader
// Waits are bounded as in gemm_masked_tc_kernel.
struct CfgPair {
    static constexpr int BN = 256;                    // tile columns (the pair's N)
    static constexpr int STAGES = 6;
    static constexpr int BKE = ROWB / 2;              // 64 BF16 per K step
    static constexpr int A_BYTES = BM * ROWB;         // this CTA's 128 rows of A
    static constexpr int B_BYTES = (BN / 2) * ROWB;   // this CTA's 128 rows of B
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr uint32_t PAIR_TX = 2u * STAGE_BYTES;   // both CTAs' loads land on the leader's barrier
    static constexpr int TMEM_COLS = 512;             // two 256-column accumulators
    static constexpr int THREADS = 192;
    static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE_BYTES + 256;
    static constexpr uint32_t IDESC = idesc_bf16_f32(2 * BM, BN);
    static_assert(SMEM <= 232448, "shared memory");
};

// kAMN / kBMN: A (M x K) or B (N x K) is read MN-major: stored K rows by MN
// columns (MN contiguous).  One 4-D copy per operand and stage brings the CTA's
// 128 of MN (two 64-element chunks, adjacent in memory) for the stage's 64 of K
// as groups of 8 K rows, each group the two chunks' 1 KB atoms side by side;
// the MN coordinate goes through g.mn_kept for the operands flagged in g.mn_remap.
template <bool kAMN, bool kBMN>
__global__ void __launch_bounds__(CfgPair::THREADS, 1)
gemm_pair_bf16_kernel(const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_b,
                      const GemmArgs g) {
    using C = CfgPair;
    constexpr int STAGES = C::STAGES, BN = C::BN, BKE = C::BKE;
    constexpr uint32_t kKGroup = 2 * 1024;   // MN-major stage: 8 K rows of both MN chunks
    constexpr uint32_t kIdesc = C::IDESC | (kAMN ? 1u << 15 : 0u) | (kBMN ? 1u << 16 : 0u);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *tiles = smem;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * C::STAGE_BYTES);   // leader's are used
    uint64_t *empty = full + STAGES;
    uint64_t *tmem_full = empty + STAGES;
    uint64_t *tmem_empty = tmem_full + 2;                                          // leader's are used
    uint64_t *drain = tmem_empty + 2;
    uint32_t *tmem_base_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_base_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rank = (int)cluster_ctarank();
    const bool leader = rank == 0;
    const int t_first = blockIdx.x / 2, t_step = gridDim.x / 2;
    const int tiles_mp = (g.tiles_m + 1) / 2;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tmem_full[a], 1);
            mbar_init(&tmem_empty[a], 2 * 128);   // the epilogue threads of both CTAs
        }
        mbar_init(drain, 1);
        *abort = 0;
        fence_barrier_init();
        prefetch_tmap(&tmap_a);
        prefetch_tmap(&tmap_b);
    }
    if (warp == 1) tmem_alloc_pair(tmem_base_slot, C::TMEM_COLS);
    tc_fence_before();
    cluster_sync_all();   // both CTAs' barriers exist before any remote arrival
    tc_fence_after();
    const uint32_t tmem_base = *tmem_base_slot;

    auto coords = [&](int t, int &tm, int &tn) {
        int pm = 0;
        if (g.sym) tri_coords(t, pm, tn);
        else tile_coords(t, tiles_mp, g.tiles_n, pm, tn);
        tm = 2 * pm + rank;   // past the last tile (odd count): zero rows, no stores
    };
    // kept sketch blocks of the block of C holding tile pair (tm / 2, tn) (the pair's
    // 256 rows and 256 columns lie in one block: bm and bn are multiples of 256)
    const uint64_t pmask = g.P >= 64 ? ~0ull : ((1ull << g.P) - 1ull);
    auto tile_mask = [&](int tm, int tn) -> uint64_t {
        if (!g.block_masks) return 0ull;
        const int64_t bi = (int64_t)(tm >> 1) * (2 * BM) / g.bm, bj = (int64_t)tn * BN / g.bn;
        return __ldg(g.block_masks + bi * g.nbc + bj) & pmask;
    };
    auto tile_num_kb = [&](uint64_t msk) -> int {
        return g.block_masks ? __popcll(msk) * g.kb_per_blk : g.num_kb;
    };
    // MN coordinate of row/column q of C (extent `ext`) in an MN-major operand;
    // `remap`: through the listed blocks, and rows past the extent at column
    // P * mn_b, past the stored blocks (the load fills zeros there as it does
    // past the extent of an operand that is not remapped)
    auto mn_coord = [&](int64_t q, int64_t ext, bool remap) -> int {
        if (!remap) return (int)q;
        if (q >= ext) return (int)((int64_t)g.P * g.mn_b);
        const int64_t blk = q / g.mn_b;
        return (int)((int64_t)g.mn_kept.idx[blk] * g.mn_b + (q - blk * g.mn_b));
    };

    if (warp == 0) {
        // ---------------- TMA producer (this CTA's half of every stage) ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued_phase[STAGES];
            bool issued[STAGES];
            for (int s = 0; s < STAGES; ++s) issued[s] = false, issued_phase[s] = 0;
            bool ok = true;
            for (int t = t_first; ok && t < g.num_tiles; t += t_step) {
                int tm, tn;
                coords(t, tm, tn);
                const uint64_t msk = tile_mask(tm, tn);
                const int nkb = tile_num_kb(msk);
                uint64_t rest = msk;
                int kidx = 0;
                for (int kb = 0, kin = 0; kb < nkb; ++kb) {
                    if (!mbar_wait_cluster(&empty[stage], phase ^ 1u, abort)) { ok = false; break; }
                    if (kin == 0) {
                        // the next kept sketch block of this tile
                        if (g.block_masks) {
                            kidx = __ffsll((long long)rest) - 1;
                            rest &= rest - 1;
                        } else {
                            kidx = g.kept.idx[kb / g.kb_per_blk];
                        }
                    }
                    const int kz = kidx * g.b + kin * BKE;
                    if (++kin == g.kb_per_blk) kin = 0;
                    uint8_t *st = tiles + stage * C::STAGE_BYTES;
                    const uint32_t fb = cluster_addr(&full[stage], 0);
                    if (leader) mbar_expect_tx(&full[stage], C::PAIR_TX);
                    if constexpr (kAMN) {
                        const int x = mn_coord((int64_t)tm * BM, g.m, g.mn_remap & 1);
                        tma_load_4d_pair(&tmap_a, fb, st, 0, 0, x / 64, kz / 8);
                    } else {
                        tma_load_2d_pair(&tmap_a, fb, st, kz, tm * BM);
                    }
                    if constexpr (kBMN) {
                        const int x = mn_coord((int64_t)tn * BN + rank * (BN / 2), g.l, g.mn_remap & 2);
                        tma_load_4d_pair(&tmap_b, fb, st + C::A_BYTES, 0, 0, x / 64, kz / 8);
                    } else {
                        tma_load_2d_pair(&tmap_b, fb, st + C::A_BYTES, kz, tn * BN + rank * (BN / 2));
                    }
                    issued[stage] = true;
                    issued_phase[stage] = phase;
                    if (++stage == STAGES) stage = 0, phase ^= 1u;
                }
            }
            // every stage this CTA loaded has been consumed by the pair's MMAs (so its
            // copies have landed and no commit is still on its way here)
            for (int s = 0; ok && s < STAGES; ++s)
                if (issued[s] && !mbar_wait_cluster(&empty[s], issued_phase[s], abort)) ok = false;
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (leader; lane 0 issues, the warp waits together) ----------------
        if (leader) {
            int stage = 0;
            uint32_t phase = 0;
            int iter = 0;
            bool ok = true;
            bool any = false;
            for (int t = t_first; ok && t < g.num_tiles; t += t_step, ++iter) {
                const int a = iter & 1;
                const uint32_t aphase = (uint32_t)(iter >> 1) & 1u;
                int tm, tn;
                coords(t, tm, tn);
                const int nkb = tile_num_kb(tile_mask(tm, tn));
                if (!__all_sync(0xffffffffu, mbar_wait_cluster(&tmem_empty[a], aphase ^ 1u, abort))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(a * BN);
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!__all_sync(0xffffffffu, mbar_wait_cluster(&full[stage], phase, abort))) { ok = false; break; }
                    tc_fence_after();
                    if (lane == 0) {
                        const uint32_t sa0 = smem_u32(tiles + stage * C::STAGE_BYTES);
                        const uint32_t sb0 = sa0 + C::A_BYTES;
#pragma unroll
                        for (int kk = 0; kk < ROWB / 32; ++kk) {
                            // a K slice of 16: 32 bytes into each K-major row, or 16 rows
                            // of an MN-major chunk
                            const uint64_t da = kAMN ? sdesc_mnmajor_sw128(sa0 + kk * 2 * kKGroup, 1024, kKGroup)
                                                     : sdesc_kmajor_sw128(sa0 + kk * 32);
                            const uint64_t db = kBMN ? sdesc_mnmajor_sw128(sb0 + kk * 2 * kKGroup, 1024, kKGroup)
                                                     : sdesc_kmajor_sw128(sb0 + kk * 32);
                            umma_f16_pair(d, da, db, kIdesc, (kb > 0 || kk > 0) ? 1u : 0u);
                        }
                        umma_commit_pair(&empty[stage], 0x3);   // the stage is free in both CTAs
                    }
                    __syncwarp();
                    any = true;
                    if (++stage == STAGES) stage = 0, phase ^= 1u;
                }
                if (!ok) break;
                if (lane == 0) umma_commit_pair(&tmem_full[a], 0x3);   // both halves of the accumulator
            }
            if (!ok && any && lane == 0) {
                // drain: wait for the MMAs already issued before TMEM is freed
                umma_commit_pair(drain, 0x1);
                mbar_wait_drain(drain, 0);
            }
        }
    } else {
        // ---------------- epilogue (warps 2..5): this CTA's 128 rows ----------------
        const int quarter = warp & 3;
        const int row_in_tile = quarter * 32 + lane;
        const uint32_t empty_cl0 = cluster_addr(&tmem_empty[0], 0);
        const uint32_t empty_cl1 = cluster_addr(&tmem_empty[1], 0);
        int iter = 0;
        for (int t = t_first; t < g.num_tiles; t += t_step, ++iter) {
            int tm, tn;
            coords(t, tm, tn);
            const int a = iter & 1;
            const uint32_t aphase = (uint32_t)(iter >> 1) & 1u;
            if (!__all_sync(0xffffffffu, mbar_wait_cluster(&tmem_full[a], aphase, abort))) break;
            tc_fence_after();
            const int64_t r = (int64_t)tm * BM + row_in_tile;
            const int64_t c0 = (int64_t)tn * BN;
            const bool vec_ok = ((reinterpret_cast<uintptr_t>(g.C) & 15u) == 0) && (g.ldc % 4 == 0);
            // per-block masks: 1/k of this tile's block; an empty kept set gives zeros
            const uint64_t msk = tile_mask(tm, tn);
            const bool none = g.block_masks && msk == 0;
            const float alpha = g.block_masks ? (none ? 0.f : 1.f / (float)__popcll(msk)) : g.alpha;
            for (int ch = 0; ch < BN / 32; ++ch) {
                uint32_t v[32];
                tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * BN + ch * 32), v);
                if (none) {
#pragma unroll
                    for (int u = 0; u < 32; ++u) v[u] = 0u;
                }
                if (r < g.m) {
                    float *dst = g.C + r * g.ldc + c0 + ch * 32;
                    const int64_t cb = c0 + ch * 32;
                    if (vec_ok && cb + 32 <= g.l) {
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            float4 o = make_float4(alpha * __uint_as_float(v[4 * u]),
                                                   alpha * __uint_as_float(v[4 * u + 1]),
                                                   alpha * __uint_as_float(v[4 * u + 2]),
                                                   alpha * __uint_as_float(v[4 * u + 3]));
                            if (g.beta != 0.f) {
                                const float4 old = *reinterpret_cast<const float4 *>(dst + 4 * u);
                                o.x = fmaf(g.beta, old.x, o.x);
                                o.y = fmaf(g.beta, old.y, o.y);
                                o.z = fmaf(g.beta, old.z, o.z);
                                o.w = fmaf(g.beta, old.w, o.w);
                            }
                            *reinterpret_cast<float4 *>(dst + 4 * u) = o;
                        }
                    } else {
#pragma unroll
                        for (int u = 0; u < 32; ++u) {
                            if (cb + u < g.l) {
                                float o = alpha * __uint_as_float(v[u]);
                                if (g.beta != 0.f) o = fmaf(g.beta, dst[u], o);
                                dst[u] = o;
                            }
                        }
                    }
                    if (g.sym && (tm >> 1) != tn) {
                        // the mirror tile: value (r, cb + u) also at (cb + u, r); the
                        // warp's 32 rows make each of these stores one 128-byte line
#pragma unroll
                        for (int u = 0; u < 32; ++u) {
                            if (cb + u < g.l) {
                                float *dt = g.C + (cb + u) * g.ldc + r;
                                float o = alpha * __uint_as_float(v[u]);
                                if (g.beta != 0.f) o = fmaf(g.beta, *dt, o);
                                *dt = o;
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive_cluster(a == 0 ? empty_cl0 : empty_cl1);
        }
    }

    tc_fence_before();
    __syncthreads();
    cluster_sync_all();   // both CTAs are done with the shared TMEM and with each other's barriers
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, C::TMEM_COLS);
    }
}

// ---------------------------------------------------------------- host ----

typedef CUresult (*PFN_encodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                    const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                    const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

PFN_encodeTiled get_encode() {
    static PFN_encodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_encodeTiled>(p);
    });
    return fn;
}

// 2-D K-major tensor map: rows x cols (cols contiguous), box box_rows x box_cols.
os_status make_tmap(CUtensorMap *map, const void *base, CUtensorMapDataType dt, int elem_bytes, int64_t rows,
                    int64_t cols, int64_t ld, int box_rows, int box_cols,
                    CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_128B) {
    PFN_encodeTiled enc = get_encode();
    if (!enc) return OS_ERR_CUDA;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * elem_bytes)};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, dt, 2, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? OS_OK : OS_ERR_INVALID_ARG;
}

// 4-D view of a matrix stored K rows by MN columns (pitch ld elements) for
// MN-major loads: {64 of MN, 8 rows of K, MN / 64 chunks, K / 8 groups}, box
// {64, 8, 2, 8}: two adjacent 64-element chunks for 64 rows of K, stored as 8 groups
// of 8 rows, each group the two chunks' 1 KB atoms side by side (128-byte swizzle).
// K % 8 == 0 and mn_ext % 64 == 0 keep every box inside the rows and columns it
// names (past the last group or chunk the load fills zeros).
os_status make_tmap_mn4(CUtensorMap *map, const void *base, int64_t K, int64_t mn_ext, int64_t ld) {
    PFN_encodeTiled enc = get_encode();
    if (!enc) return OS_ERR_CUDA;
    if (K % 8 != 0 || mn_ext % 64 != 0 || ld < mn_ext) return OS_ERR_INVALID_ARG;
    cuuint64_t dims[4] = {64, 8, (cuuint64_t)(mn_ext / 64), (cuuint64_t)(K / 8)};
    cuuint64_t strides[3] = {(cuuint64_t)(ld * 2), 128, (cuuint64_t)(8 * ld * 2)};
    cuuint32_t box[4] = {64, 8, 2, 8};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? OS_OK : OS_ERR_INVALID_ARG;
}

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

}  // namespace

namespace {

// C = alpha * sum over the listed K blocks of A_blk . B_blk^T (+ beta C).  A is
// rows x zK, B cols x zK, K-major; for the TF32 configuration A1/B1 are the lo
// planes (A0/B0 the hi planes); for FP8 they are the FP32 scale arrays
// (slice-major, fp8_scale_ld(rows) entries per 128-wide K slice).
template <class C>
os_status launch_tc(const void *A0, const void *A1, int64_t lda, const void *B0, const void *B1, int64_t ldb,
                    int64_t m, int64_t l, int64_t zK, int32_t blk, const BlockList &kept, float alpha, float beta,
                    float *Cout, int64_t ldc, cudaStream_t st) {
    if (blk % C::BKE != 0) return OS_ERR_UNSUPPORTED;
    if (!aligned16(A0) || !aligned16(B0) || (lda * C::ELEM) % 16 != 0 || (ldb * C::ELEM) % 16 != 0)
        return OS_ERR_INVALID_ARG;
    if ((C::PLANES == 2 || C::FP8) && (!aligned16(A1) || !aligned16(B1))) return OS_ERR_INVALID_ARG;
    if (zK >= (int64_t(1) << 31)) return OS_ERR_UNSUPPORTED;
    GemmArgs g;
    g.group = nullptr;
    g.group_count = 0;
    g.m = m;
    g.l = l;
    g.b = blk;
    g.kb_per_blk = blk / C::BKE;
    g.kept = kept;
    g.num_kb = kept.count * g.kb_per_blk;
    g.tiles_m = (int)((m + BM - 1) / BM);
    g.tiles_n = (int)((l + C::BN - 1) / C::BN);
    g.num_tiles = g.tiles_m * g.tiles_n;
    g.alpha = alpha;
    g.beta = beta;
    g.C = Cout;
    g.ldc = ldc;
    const CUtensorMapDataType dt = C::FP8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                   : C::PLANES == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                    : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUtensorMap ta0, tb0, ta1, tb1;
    OSK_TRY(make_tmap(&ta0, A0, dt, C::ELEM, m, zK, lda, BM, C::BKE));
    OSK_TRY(make_tmap(&tb0, B0, dt, C::ELEM, l, zK, ldb, C::BN, C::BKE));
    if (C::FP8) {
        // one row of 128 (A) or BN (B) FP32 scales per stage; rows past m / l read as 0
        const int64_t nsl = zK / 128;
        OSK_TRY(make_tmap(&ta1, A1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, nsl, m, fp8_scale_ld(m), 1, BM,
                          CU_TENSOR_MAP_SWIZZLE_NONE));
        OSK_TRY(make_tmap(&tb1, B1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, nsl, l, fp8_scale_ld(l), 1, C::BN,
                          CU_TENSOR_MAP_SWIZZLE_NONE));
    } else if (C::PLANES == 2) {
        OSK_TRY(make_tmap(&ta1, A1, dt, C::ELEM, m, zK, lda, BM, C::BKE));
        OSK_TRY(make_tmap(&tb1, B1, dt, C::ELEM, l, zK, ldb, C::BN, C::BKE));
    } else {
        ta1 = ta0;
        tb1 = tb0;
    }
    static bool attr_set = false;
    if (!attr_set) {
        OSK_CUDA_TRY(cudaFuncSetAttribute(gemm_masked_tc_kernel<C, false>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
        attr_set = true;
    }
    const int grid = g.num_tiles < num_sms() ? g.num_tiles : num_sms();
    gemm_masked_tc_kernel<C, false><<<grid, C::THREADS, C::SMEM, st>>>(ta0, tb0, ta1, tb1, g);
    return check_launch();
}

template <bool kAMN, bool kBMN>
os_status launch_pair_args(const CUtensorMap &ta, const CUtensorMap &tb, const GemmArgs &g, cudaStream_t st);

// BF16 on CTA pairs (gemm_pair_bf16_kernel): 256 x 256 tiles, two SMs each.
// C = A A^T (B the same matrix as A) is symmetric: only the lower triangle of
// tile pairs is computed and mirrored.
os_status launch_pair_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, int64_t m, int64_t l, int64_t zK,
                           int32_t blk, const BlockList &kept, float alpha, float beta, float *Cout, int64_t ldc,
                           cudaStream_t st, const uint64_t *block_masks = nullptr, int64_t bm = 0,
                           int64_t bn = 0, int32_t P = 0) {
    using C = CfgPair;
    if (blk % C::BKE != 0) return OS_ERR_UNSUPPORTED;
    if (!aligned16(A) || !aligned16(B) || (lda * 2) % 16 != 0 || (ldb * 2) % 16 != 0) return OS_ERR_INVALID_ARG;
    if (zK >= (int64_t(1) << 31)) return OS_ERR_UNSUPPORTED;
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.m = m;
    g.l = l;
    g.b = blk;
    g.kb_per_blk = blk / C::BKE;
    g.kept = kept;
    g.num_kb = kept.count * g.kb_per_blk;
    g.tiles_m = (int)((m + BM - 1) / BM);
    g.tiles_n = (int)((l + C::BN - 1) / C::BN);
    g.num_tiles = (g.tiles_m + 1) / 2 * g.tiles_n;   // tile pairs
    g.sym = A == B && lda == ldb && m == l && !block_masks;
    if (g.sym) g.num_tiles = g.tiles_n * (g.tiles_n + 1) / 2;   // tiles_n = (tiles_m + 1) / 2
    g.alpha = alpha;
    g.beta = beta;
    g.C = Cout;
    g.ldc = ldc;
    g.block_masks = block_masks;
    g.bm = bm;
    g.bn = bn;
    g.nbc = bn > 0 ? (int32_t)((l + bn - 1) / bn) : 0;
    g.P = P;
    CUtensorMap ta, tb;
    OSK_TRY(make_tmap(&ta, A, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, m, zK, lda, BM, C::BKE));
    OSK_TRY(make_tmap(&tb, B, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, l, zK, ldb, C::BN / 2, C::BKE));
    return launch_pair_args<false, false>(ta, tb, g, st);
}

// The pair kernel with prepared arguments: one CTA pair per two SMs, persistent.
template <bool kAMN, bool kBMN>
os_status launch_pair_args(const CUtensorMap &ta, const CUtensorMap &tb, const GemmArgs &g, cudaStream_t st) {
    using C = CfgPair;
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(gemm_pair_bf16_kernel<kAMN, kBMN>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    });
    OSK_CUDA_TRY(attr_err);
    const int pairs = num_sms() / 2;
    const int grid = 2 * (g.num_tiles < pairs ? g.num_tiles : pairs);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(C::THREADS);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    OSK_CUDA_TRY(cudaLaunchKernelEx(&cfg, gemm_pair_bf16_kernel<kAMN, kBMN>, ta, tb, g));
    return check_launch();
}

// C (m x l) = alpha A B^T + beta C in BF16 on CTA pairs, contraction length K,
// with A and/or B read MN-major (stored K rows by MN columns, row pitch lda/ldb),
// so that neither needs a transpose.  For the operands flagged in remap (1: A,
// 2: B) row/column q of C is column kept[q / mn_b] * mn_b + q % mn_b of the
// stored operand, whose MN extent is P * mn_b.  MN-major operands need K % 8 == 0,
// a stored MN extent (and pitch) that is a multiple of 64, and mn_b % 128 == 0.
os_status launch_pair_bf16_mn(const void *A, int64_t lda, bool a_mn, const void *B, int64_t ldb, bool b_mn,
                              int64_t m, int64_t l, int64_t K, float alpha, float beta, float *Cout, int64_t ldc,
                              int32_t mn_b, int32_t remap, const BlockList &kept, int32_t P, cudaStream_t st) {
    using C = CfgPair;
    if (!aligned16(A) || !aligned16(B) || (lda * 2) % 16 != 0 || (ldb * 2) % 16 != 0) return OS_ERR_INVALID_ARG;
    if (remap && (mn_b <= 0 || mn_b % 128 != 0 || P < 1)) return OS_ERR_INVALID_ARG;
    if (K <= 0 || K >= (int64_t(1) << 31) || m >= (int64_t(1) << 30) || l >= (int64_t(1) << 30))
        return OS_ERR_UNSUPPORTED;
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    const int64_t kpad = (K + C::BKE - 1) / C::BKE * C::BKE;
    g.m = m;
    g.l = l;
    g.b = (int32_t)kpad;
    g.kb_per_blk = (int32_t)(kpad / C::BKE);
    g.kept.count = 1;   // one K block, [0, kpad): the loads fill zeros past K
    g.num_kb = g.kb_per_blk;
    g.tiles_m = (int)((m + BM - 1) / BM);
    g.tiles_n = (int)((l + C::BN - 1) / C::BN);
    g.num_tiles = (g.tiles_m + 1) / 2 * g.tiles_n;
    g.alpha = alpha;
    g.beta = beta;
    g.C = Cout;
    g.ldc = ldc;
    g.P = P;
    g.mn_b = mn_b;
    g.mn_remap = remap;
    g.mn_kept = kept;
    // stored MN extents (an operand that is not remapped: its pitch must reach the
    // next multiple of 64; those columns only feed rows/columns of C past m or l)
    const int64_t a_ext = (remap & 1) ? (int64_t)P * mn_b : (m + 63) / 64 * 64;
    const int64_t b_ext = (remap & 2) ? (int64_t)P * mn_b : (l + 63) / 64 * 64;
    CUtensorMap ta, tb;
    if (a_mn) OSK_TRY(make_tmap_mn4(&ta, A, K, a_ext, lda));
    else OSK_TRY(make_tmap(&ta, A, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, m, K, lda, BM, C::BKE));
    if (b_mn) OSK_TRY(make_tmap_mn4(&tb, B, K, b_ext, ldb));
    else OSK_TRY(make_tmap(&tb, B, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, l, K, ldb, C::BN / 2, C::BKE));
    if (a_mn && b_mn) return launch_pair_args<true, true>(ta, tb, g, st);
    if (a_mn) return launch_pair_args<true, false>(ta, tb, g, st);
    if (b_mn) return launch_pair_args<false, true>(ta, tb, g, st);
    return launch_pair_args<false, false>(ta, tb, g, st);
}

os_status launch_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, int64_t m, int64_t l, int64_t zK,
                      int32_t blk, const BlockList &kept, float alpha, float beta, float *C, int64_t ldc,
                      cudaStream_t st) {
    return launch_pair_bf16(A, lda, B, ldb, m, l, zK, blk, kept, alpha, beta, C, ldc, st);
}

}  // namespace

// The backward pass's products straight from the sketched operands: T = dC
// B~_sel^T (B~^T read MN-major, its kept blocks picked by column) and U =
// A~_sel^T dC (A~ and dC read MN-major).  See launch_pair_bf16_mn.
os_status gemm_bf16_mn(const void *A, int64_t lda, bool a_mn, const void *B, int64_t ldb, bool b_mn, int64_t m,
                       int64_t l, int64_t K, float alpha, float *C, int64_t ldc, int32_t mn_b, int32_t remap,
                       uint64_t mask, int32_t P, cudaStream_t st) {
    const BlockList kept = mask_to_list(mask ? mask : ~0ull, P);
    return launch_pair_bf16_mn(A, lda, a_mn, B, ldb, b_mn, m, l, K, alpha, 0.0f, C, ldc, mn_b, remap, kept, P, st);
}

os_status gemm_masked_tc(const Plan *p, const void *At, int64_t ldat, const float *a_scales,
                         const void *BtT, int64_t ldbt, const float *b_scales, os_dtype dt, int64_t m,
                         int64_t l, uint64_t mask, float alpha, float beta, float *C, int64_t ldc,
                         cudaStream_t st) {
    const int64_t z = (int64_t)p->P * p->b;
    const BlockList kept = mask_to_list(mask, p->P);
    if (dt == OS_BF16) return launch_bf16(At, ldat, BtT, ldbt, m, l, z, p->b, kept, alpha, beta, C, ldc, st);
    if (dt == OS_TF32X2) {
        // two planes per operand: hi at the pointer, lo one plane (rows * ld elements) later
        const float *a0 = (const float *)At, *b0 = (const float *)BtT;
        return launch_tc<CfgTf32x3>(a0, a0 + m * ldat, ldat, b0, b0 + l * ldbt, ldbt, m, l, z, p->b, kept, alpha,
                                    beta, C, ldc, st);
    }
    if (dt == OS_FP8E4M3) {
        if (!a_scales || !b_scales) return OS_ERR_INVALID_ARG;
        return launch_tc<CfgFp8>(At, a_scales, ldat, BtT, b_scales, ldbt, m, l, z, p->b, kept, alpha, beta, C, ldc,
                                 st);
    }
    return OS_ERR_UNSUPPORTED;
}

os_status group_problem_bf16(GroupProblem *gp, GroupTile tile, const void *A, int64_t lda, const void *B,
                             int64_t ldb, int64_t m, int64_t l, int64_t zK, int32_t blk, int32_t P, uint64_t mask,
                             const uint64_t *dmask, float alpha, float beta, float *C, int64_t ldc) {
    const int BN = tile == kGroupBN256 ? CfgBf16::BN : CfgBf16N128::BN;
    constexpr int BKE = CfgBf16::BKE;
    if (m <= 0 || l <= 0 || P < 1 || P > 64 || (!dmask && mask == 0)) return OS_ERR_INVALID_ARG;
    if (blk % BKE != 0) return OS_ERR_UNSUPPORTED;
    if (!aligned16(A) || !aligned16(B) || (lda * 2) % 16 != 0 || (ldb * 2) % 16 != 0) return OS_ERR_INVALID_ARG;
    if (zK >= (int64_t(1) << 31)) return OS_ERR_UNSUPPORTED;
    std::memset(gp, 0, sizeof(*gp));
    OSK_TRY(make_tmap(&gp->ta, A, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, m, zK, lda, BM, BKE));
    OSK_TRY(make_tmap(&gp->tb, B, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, l, zK, ldb, BN, BKE));
    gp->C = C;
    gp->m = m;
    gp->l = l;
    gp->ldc = ldc;
    gp->alpha = alpha;
    gp->beta = beta;
    gp->b = blk;
    gp->kb_per_blk = blk / BKE;
    gp->P = P;
    gp->tiles_m = (int32_t)((m + BM - 1) / BM);
    gp->tiles_n = (int32_t)((l + BN - 1) / BN);
    gp->tile_begin = 0;
    gp->mask = mask;
    gp->dmask = dmask;
    return OS_OK;
}

namespace {
template <class C>
os_status prepare_grouped() {
    OSK_CUDA_TRY(cudaFuncSetAttribute(gemm_masked_tc_kernel<C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)C::SMEM));
    return OS_OK;
}

template <class C>
os_status launch_grouped(const GroupProblem *probs, int32_t count, int32_t total_tiles, cudaStream_t st) {
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.group = probs;
    g.group_count = count;
    g.num_tiles = total_tiles;
    // the per-product tensor maps are read from global memory; these are placeholders
    CUtensorMap dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    const int grid = total_tiles < num_sms() ? total_tiles : num_sms();
    gemm_masked_tc_kernel<C, true><<<grid, C::THREADS, C::SMEM, st>>>(dummy, dummy, dummy, dummy, g);
    return check_launch();
}
}  // namespace

os_status gemm_grouped_prepare() {
    static std::mutex mu;
    static bool done = false;
    std::lock_guard<std::mutex> lock(mu);
    if (done) return OS_OK;
    OSK_TRY(prepare_grouped<CfgBf16>());
    OSK_TRY(prepare_grouped<CfgBf16N128>());
    done = true;
    return OS_OK;
}

os_status gemm_grouped_bf16(const GroupProblem *probs, int32_t count, int32_t total_tiles, GroupTile tile,
                            cudaStream_t st) {
    if (!probs || count <= 0 || count > kMaxGroup || total_tiles <= 0) return OS_ERR_INVALID_ARG;
    if (tile == kGroupBN256) return launch_grouped<CfgBf16>(probs, count, total_tiles, st);
    return launch_grouped<CfgBf16N128>(probs, count, total_tiles, st);
}

}  // namespace osk

using namespace osk;

extern "C" os_status oversketch_device_status(void *stream, int32_t *status, int32_t reset) {
    if (!status) return OS_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    unsigned int v = 0;
    OSK_CUDA_TRY(cudaMemcpyFromSymbolAsync(&v, tc::g_device_status, sizeof(v), 0, cudaMemcpyDeviceToHost, st));
    OSK_CUDA_TRY(cudaStreamSynchronize(st));
    *status = (v & 1u) ? OS_ERR_TIMEOUT : OS_OK;
    if (reset && v) {
        const unsigned int zero = 0;
        OSK_CUDA_TRY(cudaMemcpyToSymbolAsync(tc::g_device_status, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st));
        OSK_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return OS_OK;
}

extern "C" os_status oversketch_test_wait_timeout(uint64_t limit_ns, int32_t skip_kb) {
    if (skip_kb >= 0 && limit_ns == 0) return OS_ERR_INVALID_ARG;
    const unsigned long long lim = skip_kb >= 0 ? (unsigned long long)limit_ns : tc::kWaitLimitNs;
    const int skip = skip_kb >= 0 ? skip_kb : -1;
    OSK_CUDA_TRY(cudaMemcpyToSymbol(tc::g_test_wait_ns, &lim, sizeof(lim)));
    OSK_CUDA_TRY(cudaMemcpyToSymbol(tc::g_test_skip_kb, &skip, sizeof(skip)));
    return OS_OK;
}

extern "C" os_status oversketch_gemm_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, int64_t m,
                                          int64_t n, int64_t K, float alpha, float beta, float *C, int64_t ldc,
                                          void *stream) {
    OSK_NVTX("gemm_bf16");
    if (m < 0 || n < 0 || K < 0 || ldc < n || lda < K || ldb < K) return OS_ERR_INVALID_ARG;
    if (m == 0 || n == 0) return OS_OK;   // an empty C
    if (!A || !B || !C) return OS_ERR_INVALID_ARG;
    if (K == 0) return OS_ERR_UNSUPPORTED;
    // one K block rounded up to the 64-wide K tile; TMA fills the columns past K with zeros
    BlockList one;
    one.count = 1;
    for (int t = 0; t < 64; ++t) one.idx[t] = 0;
    const int64_t kpad = (K + 63) / 64 * 64;
    return launch_bf16(A, lda, B, ldb, m, n, K, (int32_t)kpad, one, alpha, beta, C, ldc, as_stream(stream));
}

extern "C" os_status oversketch_gemm_masked_blocks(oversketch_plan_t plan, const void *At, int64_t ldat,
                                                   const void *BtT, int64_t ldbt, int64_t m, int64_t l,
                                                   const uint64_t *block_masks, int64_t bm, int64_t bn,
                                                   float beta, float *C, int64_t ldc, void *stream) {
    OSK_NVTX("gemm_masked_blocks");
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p || m < 0 || l < 0 || ldc < l) return OS_ERR_INVALID_ARG;
    if (bm < 256 || bn < 256 || bm % 256 != 0 || bn % 256 != 0) return OS_ERR_UNSUPPORTED;
    if (m == 0 || l == 0) return OS_OK;   // an empty C: nothing to read or write
    if (!At || !BtT || !C || !block_masks) return OS_ERR_INVALID_ARG;
    const int64_t z = (int64_t)p->P * p->b;
    if (ldat < z || ldbt < z) return OS_ERR_INVALID_ARG;
    const BlockList all = mask_to_list(~0ull, p->P);
    return launch_pair_bf16(At, ldat, BtT, ldbt, m, l, z, p->b, all, 1.f, beta, C, ldc, as_stream(stream),
                            block_masks, bm, bn, p->P);
}
