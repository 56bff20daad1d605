// Sketch kernels: A~ = A S and B~ = S^T B (Alg. 5, Alg. 4 step 3), plus the
// adjoint gathers used by the backward pass.
//
// One gather kernel serves both sides.  It reads a matrix X whose rows are
// indexed by the sketched dimension i (n rows) and whose "free" dimension f
// runs along the other axis, and writes Y^T[f, q] for q = j*b + c:
//
//     Y^T[f, j*b + c] = sum_{i in bucket c of block j} sigma_j(i) * s_i * X[i, f]
//
// Right sketch: X = B (n x l), Y^T = B~^T (l x z).  Left sketch: X = A^T,
// Y^T = A~ (m x z).
//
// The gather reads X in strips of W free indices (W = 128 for FP32, 256 for
// BF16): strip s holds X[0..n-1, Ws .. Ws+W-1], and a random row of it is one
// 512-byte piece, 16 bytes per lane of a warp.  The left operand (and a BF16
// right operand) is first packed strip-major into the workspace, n contiguous
// rows of 128 elements per strip, zero-padded past the free extent; packing
// the left operand is the transpose it needs anyway.  An FP32 right operand
// is gathered in place: in 128-wide strips when its rows are 16-byte aligned,
// else in 124-wide strips whose row pieces start d = 0..3 elements into a
// 16-byte granule (lane c loads granule c; the sums are kept per class d and
// realigned with one shuffle per bucket), or packed when that costs less
// (more than 6 blocks gathered).  Whole 512-byte pieces keep the address
// translations of the random row accesses cheap; 128-byte pieces spread over
// a 4 GB matrix ran at a quarter to a half of the L2 gather rate on GB300.
//
// A gather CTA owns 16 consecutive sketched columns q (32 for FP8 output;
// whole buckets of one block) and one strip.  Each warp walks the bucket-CSR of its buckets
// (indices ascending inside a bucket, the same order in every run: no
// atomics, bitwise reproducible) and gathers row pieces with 16-byte loads,
// accumulating in FP32.  The (16 or 32)-column x 128-row tile is transposed through
// shared memory so that Y^T rows are written contiguously.  CTAs of one strip
// are adjacent in launch order, so a strip stays in L2 while all of its
// buckets are gathered.  For FP8 output the four CTAs that own the quarters of
// one 128-column scale slice form a thread-block cluster and combine their
// per-row maxima through distributed shared memory.
#include <cooperative_groups.h>
#include <cstdint>
#include <cstdlib>
#include <type_traits>

#include "common.cuh"

namespace osk {

namespace {

constexpr int kTileQ = 128;
constexpr int kWarps = 8;
constexpr int kStrip = 128;   // free indices per FP32 strip (the in-place right sketch)

// Free indices per packed strip of an element type: 16 bytes per lane of a warp
// (128 FP32, 256 BF16), so every gathered row piece is 512 bytes.
template <typename T>
__host__ __device__ constexpr int strip_of() {
    return 32 * (16 / (int)sizeof(T));
}
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
    // 16 raw bytes (VW = 16 / sizeof(InT)) now, converted when they are summed
    using Raw = uint4;
    __device__ __forceinline__ static Raw load_raw(const InT *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }
    __device__ __forceinline__ static void unpack(const Raw &u, float (&v)[VW]) {
        if constexpr (std::is_same<InT, float>::value) {
            static_assert(VW == 4, "four FP32 per 16 bytes");
            v[0] = __uint_as_float(u.x); v[1] = __uint_as_float(u.y);
            v[2] = __uint_as_float(u.z); v[3] = __uint_as_float(u.w);
        } else {
            static_assert(VW == 8, "eight BF16 per 16 bytes");
            const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w[q]));
                v[2 * q] = f.x;
                v[2 * q + 1] = f.y;
            }
        }
    }
    __device__ __forceinline__ static float to_f32(float x) { return x; }
    __device__ __forceinline__ static float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }
    __device__ __forceinline__ static float load1(const InT *p) { return to_f32(p[0]); }
};

// Sixteen bytes of zeros: the row segment that padding entries of the bucket
// lists point at, so the gather loop needs no predication.
__device__ __align__(16) float g_zero_row[8];

// Lane layout: lane = slot * SUBS + sub (SUBS = 32 / SLOTS lanes per member;
// the launches use SLOTS = 1, one member per warp load).  With SLOTS > 1 the
// slots of a warp gather different members of one bucket at once (bucket lists
// are padded to a multiple of 4).  Lane `sub` holds the 16 bytes at elements
// VW*sub .. VW*sub+VW-1 of the strip (VW = 4 FP32 or 8 BF16).
// A warp owns QT/8 consecutive buckets and streams their (contiguous) padded
// member list 32 entries at a time, keeping 8 independent 16-byte loads per
// lane in flight and prefetching the next 32 entries.  Slot s accumulates
// members s, s+SLOTS, ... of a bucket in ascending order and the partial sums
// are combined by a fixed butterfly (one chain when SLOTS = 1): a fixed order,
// so the results are bitwise reproducible.
template <typename InT, typename OutT, int QT, bool kScale, int SLOTS, bool kMis>
__global__ void __launch_bounds__(kWarps * 32, kMis ? 3 : 4)
sketch_gather_kernel(const InT *__restrict__ X, int64_t strip_stride, int64_t ldx, int64_t F,
                     const uint32_t *__restrict__ pperm, const uint32_t *__restrict__ poffs,
                     int64_t pstride, int32_t b, int32_t z, const float *__restrict__ wts,
                     OutT *__restrict__ Yt, int64_t ldy, float *__restrict__ scales,
                     int64_t lds, BlockList blocks, int32_t tiles_per_block, int64_t plane_elems,
                     const uint64_t *__restrict__ dmask) {
    constexpr int SUBS = 32 / SLOTS;     // lanes per member
    constexpr int VW = 16 / (int)sizeof(InT);   // free indices per lane: 16 bytes
    constexpr int TF = VW * SUBS;        // free indices per tile row (one strip)
    constexpr int TFO = kMis ? TF - 4 : TF;   // free indices written per CTA
    constexpr int PITCH = TF + 1;        // odd pitch: conflict-free column reads
    constexpr int NC = kMis ? 4 : 1;     // accumulator sets: one per misalignment class
    static_assert(!kMis || (std::is_same<InT, float>::value && SLOTS == 1), "misaligned rows: FP32, one member per load");
    constexpr int G = 2 * SLOTS;         // groups of 4 members per batch: 8 loads per lane in flight
    constexpr int QPW = QT / kWarps;     // buckets per warp
    static_assert(QT == 8 || QT == 16 || QT == 32 || QT == 128, "tile of 8, 16, 32 or 128 sketched columns");
    static_assert(SLOTS == 1 || SLOTS == 2 || SLOTS == 4, "1, 2 or 4 members per warp load");
    extern __shared__ float4 smem_tile[];
    float *tile = reinterpret_cast<float *>(smem_tile);   // [QT][PITCH]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = lane / SUBS, sub = lane % SUBS;
    // q0: first sketched column of this CTA, inside one of the listed blocks
    const int bt = blockIdx.x / tiles_per_block;
    const int jblk = blocks.idx[bt];
    const int q0 = jblk * b + (blockIdx.x - bt * tiles_per_block) * QT;
    const int qend = min(z, jblk * b + b);
    const int64_t f0 = (int64_t)blockIdx.y * TFO;
    // a block mask read at run time: CTAs of blocks it does not keep have nothing to do
    if (dmask && !((__ldg(dmask) >> jblk) & 1ull)) return;
    using L = Loader<InT, VW, true>;

    const int nb = min(QPW, qend - q0 - warp * QPW);   // buckets owned by this warp
    if (nb > 0) {
        const int cb = q0 - jblk * b + warp * QPW;        // first bucket (within the block)
        const uint32_t *pl = pperm + (int64_t)jblk * pstride;
        const float *wl = kScale ? wts + (int64_t)jblk * pstride : nullptr;
        // group boundaries of the warp's buckets: lane t holds poffs[cb + t] / 4
        const uint32_t gbl = lane <= nb ? __ldg(poffs + (int64_t)jblk * (b + 1) + cb + lane) >> 2 : 0u;
        const uint32_t gend = __shfl_sync(0xffffffffu, gbl, nb);
        // row i of the strip at xbase + i * row_bytes: one wide multiply-add per member
        const uint64_t xbase = reinterpret_cast<uint64_t>(X + blockIdx.y * strip_stride + VW * sub);
        const uint32_t row_bytes = (uint32_t)(ldx * (int64_t)sizeof(InT));
        const uint64_t zrow = reinterpret_cast<uint64_t>(g_zero_row);

        // 32 entries starting at group g (past the warp's last group: padding)
        auto load_entries = [&](uint32_t g) -> uint32_t {
            const uint32_t pos = 4 * g + lane;
            return pos < 4 * gend ? __ldg(pl + pos) : kPadEntry;
        };
        // the signed scales sigma_j(i) s_i of the same 32 entries (scaled sketches)
        auto load_weights = [&](uint32_t g) -> float {
            if constexpr (!kScale) return 1.f;
            const uint32_t pos = 4 * g + lane;
            return pos < 4 * gend ? __ldg(wl + pos) : 0.f;
        };
        // GG groups (4*GG members) of the current bucket, entries in lanes 0 .. 4*GG-1
        // of e, their signed scales in the same lanes of w
        auto batch = [&](auto gg, uint32_t e, float w, float *acc) {
            constexpr int GG = decltype(gg)::value;
            constexpr int KS = 4 * GG / SLOTS;            // member loads per lane
            uint4 v[KS];
            float wgt[KS];
            uint32_t cls = 0;                             // 4 x misalignment class of member k: bits 2k+2, 2k+3
#pragma unroll
            for (int k = 0; k < KS; ++k) {
                const uint32_t ent = __shfl_sync(0xffffffffu, e, k * SLOTS + slot);
                // +-1 from the sign bit (or the signed scale); padding reads the zero row
                if constexpr (kScale) {
                    wgt[k] = __shfl_sync(0xffffffffu, w, k * SLOTS + slot);
                } else {
                    wgt[k] = __uint_as_float(0x3f800000u | (ent & kSignBit));
                }
                uint64_t addr = (uint64_t)(ent & kIndexMask) * row_bytes + xbase;
                if constexpr (kMis) {
                    // The row piece starts d = 0..3 elements into a 16-byte granule
                    // (the same d on every lane); lane c loads granule c from there:
                    // the 32 granules cover the strip's 124 elements and end inside
                    // the row (the launch keeps 128 elements of every strip in it).
                    cls |= ((uint32_t)addr & 12u) << (2 * k);
                    addr &= ~uint64_t(15);
                }
                v[k] = L::load_raw(reinterpret_cast<const InT *>(ent != kPadEntry ? addr : zrow));
            }
#pragma unroll
            for (int k = 0; k < KS; ++k) {
                float x[VW];
                L::unpack(v[k], x);
                if constexpr (kMis) {
                    // one accumulator set per class (a warp-uniform branch)
                    const uint32_t d = (cls >> (2 * k)) & 12u;
                    if (d == 0u) {
#pragma unroll
                        for (int w = 0; w < VW; ++w) acc[w] = fmaf(wgt[k], x[w], acc[w]);
                    } else if (d == 4u) {
#pragma unroll
                        for (int w = 0; w < VW; ++w) acc[VW + w] = fmaf(wgt[k], x[w], acc[VW + w]);
                    } else if (d == 8u) {
#pragma unroll
                        for (int w = 0; w < VW; ++w) acc[2 * VW + w] = fmaf(wgt[k], x[w], acc[2 * VW + w]);
                    } else {
#pragma unroll
                        for (int w = 0; w < VW; ++w) acc[3 * VW + w] = fmaf(wgt[k], x[w], acc[3 * VW + w]);
                    }
                } else {
#pragma unroll
                    for (int w = 0; w < VW; ++w) acc[w] = fmaf(wgt[k], x[w], acc[w]);
                }
            }
        };
        auto flush = [&](int t, float *acc) {
            float out[VW];
            if constexpr (kMis) {
                // class d holds element 4*sub + w - d of the strip in lane sub, slot w:
                // free index 4*sub + w is slot w + d of this lane, or slot w + d - 4
                // of the next lane; the classes are added in the order 0, 1, 2, 3
                float nx[NC * VW];
#pragma unroll
                for (int d = 1; d < NC; ++d)
#pragma unroll
                    for (int w = 0; w < d; ++w) nx[d * VW + w] = __shfl_down_sync(0xffffffffu, acc[d * VW + w], 1);
#pragma unroll
                for (int w = 0; w < VW; ++w) {
                    float o = acc[w];
#pragma unroll
                    for (int d = 1; d < NC; ++d)
                        o += (w + d < VW) ? acc[d * VW + (w + d) % VW] : nx[d * VW + (w + d) % VW];
                    out[w] = o;
                }
            } else {
#pragma unroll
                for (int w = 0; w < VW; ++w) {
                    out[w] = acc[w];
                    if constexpr (SLOTS == 4) out[w] += __shfl_xor_sync(0xffffffffu, out[w], 8);
                    if constexpr (SLOTS >= 2) out[w] += __shfl_xor_sync(0xffffffffu, out[w], 16);
                }
            }
            if (slot == 0) {
#pragma unroll
                for (int w = 0; w < VW; ++w) tile[(warp * QPW + t) * PITCH + VW * sub + w] = out[w];
            }
        };

        // The warp's buckets are contiguous in the list: stream it in batches that
        // never cross a bucket end (full batches of G groups, then the tail as
        // G/2, G/4, ..., 1 groups), prefetching the next 32 entries each time.
        uint32_t g = __shfl_sync(0xffffffffu, gbl, 0);
        uint32_t e_cur = load_entries(g);
        float w_cur = load_weights(g);
        auto step = [&](auto gg, float *acc) {
            constexpr int GG = decltype(gg)::value;
            const uint32_t e_nxt = load_entries(g + GG);
            const float w_nxt = load_weights(g + GG);
            batch(gg, GG * 4 >= 32 ? e_cur : (lane < 4 * GG ? e_cur : kPadEntry), w_cur, acc);
            g += GG;
            e_cur = e_nxt;
            w_cur = w_nxt;
        };
        for (int t = 0; t < nb; ++t) {
            const uint32_t gE = __shfl_sync(0xffffffffu, gbl, t + 1);
            float acc[NC * VW];
#pragma unroll
            for (int w = 0; w < NC * VW; ++w) acc[w] = 0.f;
            while (gE - g >= (uint32_t)G) step(std::integral_constant<int, G>(), acc);
            const uint32_t r = gE - g;   // < G
            if constexpr (G >= 8) if (r & 4u) step(std::integral_constant<int, 4>(), acc);
            if constexpr (G >= 4) if (r & 2u) step(std::integral_constant<int, 2>(), acc);
            if (r & 1u) step(std::integral_constant<int, 1>(), acc);
            flush(t, acc);
        }
    }
    __syncthreads();

    if constexpr (sizeof(OutT) == 1) {
        // FP8: cluster rank r holds columns 32r .. 32r+31 of the slice.  Per row:
        // partial max over 32 columns here, the slice max from all four ranks.
        static_assert(QT == 32, "FP8 tiles are the quarters of a 128-column scale slice");
        namespace cg = cooperative_groups;
        __shared__ float amax_part[TF];
        cg::cluster_group cl = cg::this_cluster();
        for (int t = 0; t < TF / kWarps; ++t) {
            const int ff = warp * (TF / kWarps) + t;
            float a = fabsf(tile[lane * PITCH + ff]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
            if (lane == 0) amax_part[ff] = a;
        }
        cl.sync();
        const bool scale_writer = cl.block_rank() == 0 && lane == 0;
        for (int t = 0; t < TF / kWarps; ++t) {
            const int ff = warp * (TF / kWarps) + t;
            const int64_t frow = f0 + ff;
            float a = lane < 4 ? *cl.map_shared_rank(amax_part + ff, (unsigned)lane) : 0.f;
            a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, 1));
            a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, 2));
            a = __shfl_sync(0xffffffffu, a, 0);
            if (ff < TFO && frow < F) {
                const int e = fp8_scale_exponent(a);
                const float inv = ldexpf(1.f, -e);
                Yt[frow * ldy + q0 + lane] = __nv_fp8_e4m3(tile[lane * PITCH + ff] * inv);   // RNE, saturating
                if (scale_writer) scales[(q0 / 128) * lds + frow] = ldexpf(1.f, e);           // slice-major
            }
        }
        cl.sync();   // the partial maxima stay readable until every rank is done
    } else {
        // Transposed write-out: warp w writes rows f0 + 16w .. 16w+15 of Y^T.
        if constexpr (QT < 32) {
            // 32 / QT rows per warp pass, QT lanes per row
            constexpr int RPI = 32 / QT;
            const int qq = lane % QT, rr = lane / QT;
            for (int t = 0; t < TF / kWarps; t += RPI) {
                const int ff = warp * (TF / kWarps) + t + rr;
                const int64_t frow = f0 + ff;
                const int q = q0 + qq;
                if (ff < TFO && frow < F && q < qend) {
                    const float v = tile[qq * PITCH + ff];
                    OutT *dst = Yt + frow * ldy + q;
                    if constexpr (std::is_same<OutT, Tf32Pair>::value) {
                        float *d0 = reinterpret_cast<float *>(dst);
                        const float hi = __uint_as_float(__float_as_uint(v) & 0xffffe000u);
                        d0[0] = hi;
                        d0[plane_elems] = v - hi;
                    } else if constexpr (sizeof(OutT) == 4) {
                        *dst = v;
                    } else {
                        *dst = __float2bfloat16_rn(v);
                    }
                }
            }
            return;
        }
        constexpr int VPL = QT >= 32 ? QT / 32 : 1;   // values per lane per row
        for (int t = 0; t < TF / kWarps; ++t) {
            const int ff = warp * (TF / kWarps) + t;
            const int64_t frow = f0 + ff;
            if (ff >= TFO || frow >= F) break;
            float v[VPL];
#pragma unroll
            for (int k = 0; k < VPL; ++k) v[k] = tile[(lane + 32 * k) * PITCH + ff];
            OutT *dst = Yt + frow * ldy + q0;
            if constexpr (std::is_same<OutT, Tf32Pair>::value) {
                // FP32 as hi + lo: hi keeps 10 mantissa bits (exact in TF32), lo = x - hi (exact)
                float *d0 = reinterpret_cast<float *>(dst);
#pragma unroll
                for (int k = 0; k < VPL; ++k) {
                    const int q = q0 + lane + 32 * k;
                    if (q < qend) {
                        const float hi = __uint_as_float(__float_as_uint(v[k]) & 0xffffe000u);
                        d0[lane + 32 * k] = hi;
                        d0[plane_elems + lane + 32 * k] = v[k] - hi;
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < VPL; ++k) {
                    const int q = q0 + lane + 32 * k;
                    if (q < qend) {
                        if constexpr (sizeof(OutT) == 4)
                            dst[lane + 32 * k] = v[k];
                        else
                            dst[lane + 32 * k] = __float2bfloat16_rn(v[k]);
                    }
                }
            }
        }
    }
}

// Strip-major packing of the right operand: Xs[s][i][t] = X[i, 128s + t]
// (zero past the free extent F).  One thread moves 16 bytes; consecutive
// threads read consecutive pieces of a row and write consecutive pieces of a
// strip row.
template <typename T, bool kVec>
__global__ void __launch_bounds__(256) pack_rows_kernel(const T *__restrict__ X, int64_t ldx, int64_t n,
                                                        int64_t F, int64_t nstrips, T *__restrict__ Xs) {
    constexpr int V = 16 / sizeof(T);                // elements per 16-byte piece
    constexpr int SW = strip_of<T>();                // strip width
    constexpr int PPS = SW / V;                      // pieces per strip row
    const int64_t pieces_per_row = nstrips * PPS;
    const int64_t total = n * pieces_per_row;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / pieces_per_row;
        const int64_t pr = t - i * pieces_per_row;
        const int64_t s = pr / PPS, pc = pr - s * PPS;
        const int64_t c0 = s * SW + pc * V;
        uint4 u = make_uint4(0u, 0u, 0u, 0u);
        if (kVec && c0 + V <= F) {
            u = __ldg(reinterpret_cast<const uint4 *>(X + i * ldx + c0));
        } else {
            T *e = reinterpret_cast<T *>(&u);
#pragma unroll
            for (int k = 0; k < V; ++k) e[k] = c0 + k < F ? X[i * ldx + c0 + k] : T(0.f);
        }
        *reinterpret_cast<uint4 *>(Xs + (s * n + i) * SW + pc * V) = u;
    }
}

// Strip-major packing of the left operand (a transpose): Xs[s][i][t] =
// A[128s + t, i] (zero for rows past m).  A CTA moves a 32-row x 256-column
// tile of A (a quarter of a strip's width) through shared memory with 16-byte
// loads and stores; every strip row receives one contiguous 32-element piece.
template <typename T, bool kVec>
__global__ void __launch_bounds__(256) pack_cols_kernel(const T *__restrict__ A, int64_t lda, int64_t m,
                                                        int64_t n, T *__restrict__ Xs) {
    constexpr int W = 256;                          // columns of A per tile
    constexpr int V = 16 / sizeof(T);               // elements per 16-byte vector
    __shared__ T tile[32][W + 1];
    const int64_t rb = blockIdx.y;                  // 32-row block of A
    constexpr int SW = strip_of<T>();               // strip width: SW / 32 row blocks per strip
    const int64_t s = rb / (SW / 32), quarter = rb % (SW / 32);
    const int64_t i0 = (int64_t)blockIdx.x * W;
    const int tid = threadIdx.x;
    const bool whole = kVec && rb * 32 + 32 <= m && i0 + W <= n;
    if (whole) {
        for (int idx = tid; idx < 32 * W / V; idx += 256) {
            const int r = idx / (W / V), cv = idx - r * (W / V);
            const uint4 u = __ldg(reinterpret_cast<const uint4 *>(A + (rb * 32 + r) * lda + i0 + cv * V));
            const T *e = reinterpret_cast<const T *>(&u);
#pragma unroll
            for (int k = 0; k < V; ++k) tile[r][cv * V + k] = e[k];
        }
    } else {
        for (int idx = tid; idx < 32 * W; idx += 256) {
            const int r = idx / W, c = idx - r * W;
            const int64_t row = rb * 32 + r, col = i0 + c;
            tile[r][c] = (row < m && col < n) ? A[row * lda + col] : T(0.f);
        }
    }
    __syncthreads();
    // output: W strip rows, each receiving 32 elements (elements 32*quarter ..)
    for (int idx = tid; idx < W * 32 / V; idx += 256) {
        const int c = idx / (32 / V), rq = idx - c * (32 / V);
        const int64_t col = i0 + c;
        if (col >= n) continue;
        uint4 u;
        T *e = reinterpret_cast<T *>(&u);
#pragma unroll
        for (int k = 0; k < V; ++k) e[k] = tile[rq * V + k][c];
        *reinterpret_cast<uint4 *>(Xs + (s * n + col) * SW + quarter * 32 + rq * V) = u;
    }
}

// dX[r, i] = scale * sum_{t < k} sigma_j(i) T[r, t*b + h_j(i)], j = kept[t]  (T holds the kept blocks only)
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
            const float x = __ldg(trow + (int64_t)t * b + (v & kIndexMask));   // kept blocks compacted
            acc += (v & kSignBit) ? -x : x;
        }
        acc *= scale;
        if constexpr (sizeof(OutT) == 4)
            dX[r * ldx + i] = acc;
        else
            dX[r * ldx + i] = __float2bfloat16_rn(acc);
    }
}

// The same sums with the CTA's R rows of T staged in shared memory: a CTA owns
// rows r0 .. r0+R-1 of dX and sweeps all n columns, so each table entry h_j(i)
// is read once for R rows and the k random reads per output hit shared memory
// instead of a 32-byte L2 sector each.  The R rows are interleaved (column c of
// the R rows at ts[c*R .. c*R+R-1]): one 4R-byte shared load serves all R
// rows.  Same order of operations as above, so the results are bitwise equal.
template <int R> struct RowVec;
template <> struct RowVec<1> { using T = float; };
template <> struct RowVec<2> { using T = float2; };
template <> struct RowVec<4> { using T = float4; };
template <int R>
__device__ __forceinline__ float row_of(const typename RowVec<R>::T &v, int r) {
    if constexpr (R == 1) return v;
    else if constexpr (R == 2) return r == 0 ? v.x : v.y;
    else return r == 0 ? v.x : r == 1 ? v.y : r == 2 ? v.z : v.w;
}

template <typename OutT, int R>
__global__ void __launch_bounds__(1024) unsketch_cols_smem_kernel(
    const float *__restrict__ T, int64_t m, int64_t ldt, int64_t kb, const uint32_t *__restrict__ hs, int64_t n,
    int32_t b, BlockList kept, float scale, OutT *__restrict__ dX, int64_t ldx) {
    using V = typename RowVec<R>::T;
    extern __shared__ float4 ts4[];
    V *ts = reinterpret_cast<V *>(ts4);     // [kb] columns of R interleaved rows
    const int64_t r0 = (int64_t)blockIdx.x * R;
    const int rows = (int)(m - r0 < R ? m - r0 : R);
    for (int64_t c = threadIdx.x; c < kb; c += blockDim.x) {
        float x[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (r < rows) x[r] = __ldg(T + (r0 + r) * ldt + c);
        if constexpr (R == 1) ts[c] = x[0];
        else if constexpr (R == 2) ts[c] = make_float2(x[0], x[1]);
        else ts[c] = make_float4(x[0], x[1], x[2], x[3]);
    }
    __syncthreads();
    // four columns per thread and pass, so that four table loads per kept block
    // are in flight at once
    constexpr int NI = 4;
    for (int64_t i0 = threadIdx.x; i0 < n; i0 += NI * (int64_t)blockDim.x) {
        float acc[NI][R];
#pragma unroll
        for (int u = 0; u < NI; ++u)
#pragma unroll
            for (int r = 0; r < R; ++r) acc[u][r] = 0.f;
        // the table entries of four kept blocks at a time: 16 loads in flight
        constexpr int TB = 4;
        for (int t0 = 0; t0 < kept.count; t0 += TB) {
            uint32_t v[TB][NI];
#pragma unroll
            for (int tt = 0; tt < TB; ++tt) {
                const uint32_t *hrow = hs + (int64_t)kept.idx[t0 + tt < kept.count ? t0 + tt : t0] * n;
#pragma unroll
                for (int u = 0; u < NI; ++u) {
                    const int64_t i = i0 + (int64_t)u * blockDim.x;
                    v[tt][u] = i < n && t0 + tt < kept.count ? __ldg(hrow + i) : 0u;
                }
            }
#pragma unroll
            for (int tt = 0; tt < TB; ++tt) {
                if (t0 + tt >= kept.count) break;
#pragma unroll
                for (int u = 0; u < NI; ++u) {
                    const int64_t c = (int64_t)(t0 + tt) * b + (v[tt][u] & kIndexMask);   // kept blocks compacted
                    const bool neg = (v[tt][u] & kSignBit) != 0u;
                    const V xv = ts[c];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const float x = row_of<R>(xv, r);
                        acc[u][r] += neg ? -x : x;
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < NI; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x;
            if (i >= n) continue;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r < rows) {
                    const float y = acc[u][r] * scale;
                    if constexpr (sizeof(OutT) == 4)
                        dX[(r0 + r) * ldx + i] = y;
                    else
                        dX[(r0 + r) * ldx + i] = __float2bfloat16_rn(y);
                }
            }
        }
    }
}

template <typename OutT>
__global__ void __launch_bounds__(256) unsketch_rows_kernel(
    const float *__restrict__ U, int64_t l, int64_t ldu, const uint32_t *__restrict__ hs, int64_t n,
    int32_t b, BlockList kept, float scale, OutT *__restrict__ dG, int64_t ldg) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + warp;
    if (i >= n) return;
    const int64_t c0 = (int64_t)blockIdx.y * 1024 + lane;
    float acc[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) acc[q] = 0.f;
    // the k table entries of row i, loaded at once: lane t holds kept blocks t and t + 32
    const uint32_t v_lo = lane < kept.count ? __ldg(hs + (int64_t)kept.idx[lane] * n + i) : 0u;
    const uint32_t v_hi = lane + 32 < kept.count ? __ldg(hs + (int64_t)kept.idx[lane + 32] * n + i) : 0u;
    for (int t = 0; t < kept.count; ++t) {
        const uint32_t v = __shfl_sync(0xffffffffu, t < 32 ? v_lo : v_hi, t & 31);
        const float sg = (v & kSignBit) ? -scale : scale;
        const float *urow = U + ((int64_t)t * b + (v & kIndexMask)) * ldu;   // kept blocks compacted
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int64_t c = c0 + 32 * q;
            if (c < l) acc[q] = fmaf(sg, __ldg(urow + c), acc[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const int64_t c = c0 + 32 * q;
        if (c < l) {
            if constexpr (sizeof(OutT) == 4)
                dG[i * ldg + c] = acc[q];
            else
                dG[i * ldg + c] = __float2bfloat16_rn(acc[q]);
        }
    }
}

// The same sums with 16-byte accesses (l, ldu and ldg multiples of 4, U and dG
// 16-byte aligned): lane t covers columns 4t .. 4t+3 of every 128-column group,
// a quarter of the load instructions for the same bytes.  Same order of
// operations, so the results are bitwise equal.
template <typename OutT>
__global__ void __launch_bounds__(256) unsketch_rows_vec_kernel(
    const float *__restrict__ U, int64_t l, int64_t ldu, const uint32_t *__restrict__ hs, int64_t n,
    int32_t b, BlockList kept, float scale, OutT *__restrict__ dG, int64_t ldg) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + warp;
    if (i >= n) return;
    const int64_t c0 = (int64_t)blockIdx.y * 1024 + 4 * lane;
    float4 acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t v_lo = lane < kept.count ? __ldg(hs + (int64_t)kept.idx[lane] * n + i) : 0u;
    const uint32_t v_hi = lane + 32 < kept.count ? __ldg(hs + (int64_t)kept.idx[lane + 32] * n + i) : 0u;
    for (int t = 0; t < kept.count; ++t) {
        const uint32_t v = __shfl_sync(0xffffffffu, t < 32 ? v_lo : v_hi, t & 31);
        const float sg = (v & kSignBit) ? -scale : scale;
        const float *urow = U + ((int64_t)t * b + (v & kIndexMask)) * ldu;   // kept blocks compacted
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t c = c0 + 128 * q;
            if (c < l) {
                const float4 u = __ldg(reinterpret_cast<const float4 *>(urow + c));
                acc[q].x = fmaf(sg, u.x, acc[q].x);
                acc[q].y = fmaf(sg, u.y, acc[q].y);
                acc[q].z = fmaf(sg, u.z, acc[q].z);
                acc[q].w = fmaf(sg, u.w, acc[q].w);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int64_t c = c0 + 128 * q;
        if (c < l) {
            if constexpr (sizeof(OutT) == 4) {
                *reinterpret_cast<float4 *>(dG + i * ldg + c) = acc[q];
            } else {
                __nv_bfloat162 h[2] = {__floats2bfloat162_rn(acc[q].x, acc[q].y),
                                       __floats2bfloat162_rn(acc[q].z, acc[q].w)};
                *reinterpret_cast<uint2 *>(dG + i * ldg + c) = *reinterpret_cast<uint2 *>(h);
            }
        }
    }
}

// The signed scale of every entry of the listed blocks' padded bucket lists,
// in list order: w[j][pos] = sigma_j(i) * s_i for the entry (i, sigma) at pos
// (0 for padding), so the gather loads the weights of 32 entries with one
// coalesced load instead of 32 scattered loads of s.
__global__ void __launch_bounds__(256) entry_weights_kernel(const uint32_t *__restrict__ pperm,
                                                            const uint32_t *__restrict__ poffs, int64_t pstride,
                                                            int32_t b, const float *__restrict__ s,
                                                            BlockList blocks, float *__restrict__ w) {
    const int j = blocks.idx[blockIdx.y];
    const int64_t len = __ldg(poffs + (int64_t)j * (b + 1) + b);     // padded list length
    const uint32_t *pl = pperm + (int64_t)j * pstride;
    float *wl = w + (int64_t)j * pstride;
    for (int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pos < len;
         pos += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t ent = __ldg(pl + pos);
        wl[pos] = ent == kPadEntry ? 0.f
                                   : __uint_as_float(__float_as_uint(__ldg(s + (ent & kIndexMask))) ^ (ent & kSignBit));
    }
}

os_status launch_entry_weights(const Plan *p, const float *s, uint64_t block_mask, float *w, cudaStream_t st) {
    const BlockList blocks = mask_to_list(block_mask ? block_mask : ~0ull, p->P);
    const int64_t per = (p->pstride + 255) / 256;
    dim3 grid((unsigned)(per < 1024 ? per : 1024), (unsigned)blocks.count);
    entry_weights_kernel<<<grid, 256, 0, st>>>(p->pperm, p->poffs, p->pstride, p->b, s, blocks, w);
    return check_launch();
}

// FP8 codes and UE8M0 scales from FP32 sums staged in global memory: one warp per
// (row, 128-column slice of a listed block); the same rule as the gather's fused
// FP8 epilogue (smallest e with amax <= 448 * 2^e, codes = RNE(x / 2^e)), so the
// codes and scales are the same bits.
__global__ void __launch_bounds__(256) quantize_fp8_kernel(const float *__restrict__ Y, int64_t ldy, int64_t rows,
                                                           int32_t b, BlockList blocks,
                                                           __nv_fp8_e4m3 *__restrict__ Q, int64_t ldq,
                                                           float *__restrict__ scales, int64_t lds) {
    const int lane = threadIdx.x & 31;
    const int64_t per_row = (int64_t)blocks.count * (b / 128);
    const int64_t total = rows * per_row;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total;
         w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t r = w / per_row;
        const int s = (int)(w - r * per_row);
        const int bt = s / (b / 128);
        const int64_t q0 = (int64_t)blocks.idx[bt] * b + (int64_t)(s - bt * (b / 128)) * 128;
        const float4 v = __ldg(reinterpret_cast<const float4 *>(Y + r * ldy + q0) + lane);
        float a = fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
        const int e = fp8_scale_exponent(a);
        const float inv = ldexpf(1.f, -e);
        __nv_fp8_e4m3 c[4] = {__nv_fp8_e4m3(v.x * inv), __nv_fp8_e4m3(v.y * inv), __nv_fp8_e4m3(v.z * inv),
                              __nv_fp8_e4m3(v.w * inv)};
        *reinterpret_cast<uint32_t *>(Q + r * ldq + q0 + 4 * lane) = *reinterpret_cast<const uint32_t *>(c);
        if (lane == 0) scales[(q0 / 128) * lds + r] = ldexpf(1.f, e);   // slice-major
    }
}

os_status launch_quantize_fp8(const Plan *p, const float *Y, int64_t ldy, int64_t rows, uint64_t block_mask,
                              void *Q, int64_t ldq, float *scales, int64_t lds, cudaStream_t st) {
    const BlockList blocks = mask_to_list(block_mask ? block_mask : ~0ull, p->P);
    const int64_t warps = rows * blocks.count * (p->b / 128);
    const int64_t ctas = (warps + 7) / 8;
    quantize_fp8_kernel<<<(unsigned)(ctas < 152 * 16 ? ctas : 152 * 16), 256, 0, st>>>(
        Y, ldy, rows, p->b, blocks, (__nv_fp8_e4m3 *)Q, ldq, scales, lds);
    return check_launch();
}

template <typename InT, typename OutT, int QT, int SLOTS, bool kMis = false>
os_status launch_gather_t(const Plan *p, const InT *X, int64_t strip_stride, int64_t ldx, int64_t F,
                          const float *wts, void *Yt, int64_t ldy, float *scales, int64_t scale_ld,
                          const BlockList &blocks, cudaStream_t st, int64_t plane_elems = 0,
                          const uint64_t *dmask = nullptr) {
    const int z = p->P * p->b;
    const int tpb = (p->b + QT - 1) / QT;
    constexpr int TF = strip_of<InT>() / SLOTS;
    constexpr int TFO = kMis ? TF - 4 : TF;   // free indices written per CTA
    dim3 grid((unsigned)(tpb * blocks.count), (unsigned)((F + TFO - 1) / TFO));
    if (grid.y > 65535u) return OS_ERR_UNSUPPORTED;
    const size_t smem = sizeof(float) * QT * (TF + 1);
    auto k = wts ? sketch_gather_kernel<InT, OutT, QT, true, SLOTS, kMis>
                       : sketch_gather_kernel<InT, OutT, QT, false, SLOTS, kMis>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if constexpr (sizeof(OutT) == 1) {
        // clusters of the 4 CTAs of a 128-column scale slice (b % 128 == 0, so
        // grid.x is a multiple of 4 and no cluster straddles two blocks)
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = dim3(kWarps * 32);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 4;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        OSK_CUDA_TRY(cudaLaunchKernelEx(&cfg, k, X, strip_stride, ldx, F, (const uint32_t *)p->pperm,
                                        (const uint32_t *)p->poffs, p->pstride, p->b, z, wts, (OutT *)Yt, ldy,
                                        scales, scale_ld, blocks, tpb, plane_elems, dmask));
    } else {
        k<<<grid, kWarps * 32, smem, st>>>(X, strip_stride, ldx, F, p->pperm, p->poffs, p->pstride, p->b, z,
                                          wts, (OutT *)Yt, ldy, scales, scale_ld, blocks, tpb, plane_elems, dmask);
    }
    return check_launch();
}

// Gather from an operand packed in 128-wide strips (n rows each) in tiles of
// 32 sketched columns, which keeps the CTAs that run together on few strips.
// Sketched columns per gather CTA (FP8 outputs: 32, the quarter of a scale slice).
// 16 puts 512 CTAs on each strip of the square workload (b = 1024, 8 kept
// blocks), so fewer strips are in flight at once than with 32 and more of the
// gathered rows hit L2 (right sketch 1.89 -> 1.74 ms on GB300).
constexpr int kGatherQT = 16;

// ss, W: the distance between strips and between rows of a strip (elements);
// the defaults are the packed workspace layout.
template <typename InT>
os_status launch_gather(const Plan *p, const InT *Xs, int64_t F, const float *wts, void *Yt,
                        os_dtype out_t, int64_t ldy, float *scales, int64_t scale_ld, uint64_t block_mask,
                        cudaStream_t st, int64_t plane_rows = 0, const uint64_t *dmask = nullptr,
                        int64_t ss = -1, int64_t W = strip_of<InT>()) {
    const BlockList blocks = mask_to_list(block_mask ? block_mask : ~0ull, p->P);
    if (ss < 0) ss = p->n * W;
    switch (out_t) {
        case OS_F32:
            return launch_gather_t<InT, float, kGatherQT, 1>(p, Xs, ss, W, F, wts, Yt, ldy, scales, scale_ld, blocks, st, 0, dmask);
        case OS_BF16:
            return launch_gather_t<InT, __nv_bfloat16, kGatherQT, 1>(p, Xs, ss, W, F, wts, Yt, ldy, scales, scale_ld,
                                                              blocks, st, 0, dmask);
        case OS_FP8E4M3:
            return launch_gather_t<InT, __nv_fp8_e4m3, 32, 1>(p, Xs, ss, W, F, wts, Yt, ldy, scales, scale_ld,
                                                               blocks, st, 0, dmask);
        case OS_TF32X2:
            return launch_gather_t<InT, Tf32Pair, kGatherQT, 1>(p, Xs, ss, W, F, wts, Yt, ldy, scales, scale_ld, blocks,
                                                         st, plane_rows * ldy, dmask);
    }
    return OS_ERR_DTYPE;
}

// Gather straight from a row-major FP32 operand in 128-wide strips (512-byte row
// pieces: one address translation per 512 bytes is cheap enough that no
// packing pass is needed).  F must be a multiple of 128.  With kMis the rows
// need only 4-byte alignment: strips are 124 wide, each lane loads the 16-byte
// granule holding its first element, and the sums are kept per misalignment
// class and realigned once per bucket (F a multiple of 124).
template <bool kMis>
os_status launch_gather_direct(const Plan *p, const float *X, int64_t ldx, int64_t F, const float *wts,
                               void *Yt, os_dtype out_t, int64_t ldy, float *scales, int64_t scale_ld,
                               uint64_t block_mask, cudaStream_t st, int64_t plane_rows = 0,
                               const uint64_t *dmask = nullptr) {
    const BlockList blocks = mask_to_list(block_mask ? block_mask : ~0ull, p->P);
    constexpr int64_t ss = kMis ? kStrip - 4 : kStrip;
    switch (out_t) {
        case OS_F32:
            return launch_gather_t<float, float, kGatherQT, 1, kMis>(p, X, ss, ldx, F, wts, Yt, ldy, nullptr,
                                                                    scale_ld, blocks, st, 0, dmask);
        case OS_BF16:
            return launch_gather_t<float, __nv_bfloat16, kGatherQT, 1, kMis>(p, X, ss, ldx, F, wts, Yt, ldy, nullptr,
                                                                            scale_ld, blocks, st, 0, dmask);
        case OS_FP8E4M3:
            return launch_gather_t<float, __nv_fp8_e4m3, 32, 1, kMis>(p, X, ss, ldx, F, wts, Yt, ldy, scales,
                                                                     scale_ld, blocks, st, 0, dmask);
        case OS_TF32X2:
            return launch_gather_t<float, Tf32Pair, kGatherQT, 1, kMis>(p, X, ss, ldx, F, wts, Yt, ldy, nullptr,
                                                                       scale_ld, blocks, st, plane_rows * ldy, dmask);
    }
    return OS_ERR_DTYPE;
}

template <typename T>
os_status launch_pack_rows(const T *X, int64_t ldx, int64_t n, int64_t F, T *Xs, cudaStream_t st) {
    constexpr int64_t SW = strip_of<T>();
    const int64_t nstrips = (F + SW - 1) / SW;
    const int64_t total = n * nstrips * (SW / (16 / (int64_t)sizeof(T)));
    const int64_t blocks = (total + 255) / 256 < 152 * 64 ? (total + 255) / 256 : 152 * 64;
    const bool vec = aligned16(X) && (ldx * (int64_t)sizeof(T)) % 16 == 0;
    if (vec)
        pack_rows_kernel<T, true><<<(unsigned)blocks, 256, 0, st>>>(X, ldx, n, F, nstrips, Xs);
    else
        pack_rows_kernel<T, false><<<(unsigned)blocks, 256, 0, st>>>(X, ldx, n, F, nstrips, Xs);
    return check_launch();
}

template <typename T>
os_status launch_pack_cols(const T *A, int64_t lda, int64_t m, int64_t n, T *Xs, cudaStream_t st) {
    // 32-row blocks of the (zero-padded) strips
    constexpr int64_t SW = strip_of<T>();
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)((m + SW - 1) / SW * (SW / 32)));
    if (grid.y > 65535u) return OS_ERR_UNSUPPORTED;
    if (aligned16(A) && (lda * (int64_t)sizeof(T)) % 16 == 0)
        pack_cols_kernel<T, true><<<grid, 256, 0, st>>>(A, lda, m, n, Xs);
    else
        pack_cols_kernel<T, false><<<grid, 256, 0, st>>>(A, lda, m, n, Xs);
    return check_launch();
}

os_status check_out(const Plan *p, int64_t rows, void *Yt, os_dtype out_t, int64_t ldy,
                    float *scales) {
    const int64_t z = (int64_t)p->P * p->b;
    if (rows < 0) return OS_ERR_INVALID_ARG;
    if (out_t != OS_F32 && out_t != OS_BF16 && out_t != OS_FP8E4M3 && out_t != OS_TF32X2) return OS_ERR_DTYPE;
    if (ldy < z || (ldy * (int64_t)dtype_size(out_t)) % 16 != 0) return OS_ERR_INVALID_ARG;
    if (out_t == OS_FP8E4M3 && p->b % 128 != 0) return OS_ERR_UNSUPPORTED;
    if (rows == 0) return OS_OK;   // an empty output: nothing is written
    if (!Yt || !aligned16(Yt)) return OS_ERR_INVALID_ARG;
    if (out_t == OS_FP8E4M3 && !scales) return OS_ERR_INVALID_ARG;
    return OS_OK;
}

}  // namespace

namespace {
size_t ws_align(size_t x) { return (x + 255) / 256 * 256; }
// ceil(F/128) packed strips of n x 128 elements
size_t strip_bytes(const Plan *p, int64_t F, os_dtype in_t) {
    const int64_t sw = 32 * (16 / (int64_t)dtype_size(in_t));   // strip_of<> of the element type
    return (size_t)((F + sw - 1) / sw) * sw * (size_t)p->n * dtype_size(in_t);
}
}  // namespace

// Sketch workspace for F free indices: the packed strips, then the signed
// scale of every bucket-list entry (P x pstride FP32, used by scaled sketches).
size_t sketch_workspace_bytes(const Plan *p, int64_t F, os_dtype in_t) {
    return ws_align(strip_bytes(p, F, in_t)) + (size_t)p->P * p->pstride * sizeof(float) + 256;
}

// FP8 output staged in FP32: a workspace this much larger (F x z FP32 sums after the
// regular workspace) lets the sketch gather FP32 sums without clusters and quantise
// them in a second pass (same codes and scales as the fused FP8 epilogue).
size_t fp8_staging_bytes(const Plan *p, int64_t F) { return (size_t)F * (size_t)p->P * p->b * sizeof(float) + 256; }

namespace {
float *fp8_staging(const Plan *p, void *ws, size_t ws_bytes, int64_t F, os_dtype in_t) {
    const size_t off = ws_align(sketch_workspace_bytes(p, F, in_t));
    if (!ws || ws_bytes < off + fp8_staging_bytes(p, F)) return nullptr;
    const uintptr_t a = (reinterpret_cast<uintptr_t>(ws) + off + 255) & ~uintptr_t(255);
    return reinterpret_cast<float *>(a);
}
}  // namespace

namespace {
void *ws_base(void *ws) {
    return reinterpret_cast<void *>((reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255));
}
// the entry weights of a workspace whose strips hold F free indices
float *ws_weights(const Plan *p, void *ws, int64_t F, os_dtype in_t) {
    return reinterpret_cast<float *>(reinterpret_cast<char *>(ws_base(ws)) + ws_align(strip_bytes(p, F, in_t)));
}
// the entry weights for scale s (NULL without a scale)
os_status make_weights(const Plan *p, const float *s, uint64_t block_mask, float *w, const float **out,
                       cudaStream_t st) {
    *out = nullptr;
    if (!s) return OS_OK;
    OSK_TRY(launch_entry_weights(p, s, block_mask, w, st));
    *out = w;
    return OS_OK;
}
}  // namespace

// The argument checks of the left sketch that need no workspace (OS_OK for a
// valid call, including an empty output m == 0).
os_status sketch_left_check(const Plan *p, const void *A, os_dtype a_t, int64_t m, int64_t lda, void *At,
                            os_dtype out_t, int64_t ldat, float *scales, uint64_t block_mask) {
    if (!p || m < 0) return OS_ERR_INVALID_ARG;
    if (block_mask) OSK_TRY(check_mask(block_mask, p->P));
    if (a_t != OS_F32 && a_t != OS_BF16) return OS_ERR_DTYPE;
    if (lda < p->n) return OS_ERR_INVALID_ARG;
    OSK_TRY(check_out(p, m, At, out_t, ldat, scales));
    if (m == 0) return OS_OK;
    if (!A) return OS_ERR_INVALID_ARG;
    return OS_OK;
}

os_status sketch_left_impl(const Plan *p, const void *A, os_dtype a_t, int64_t m, int64_t lda,
                           void *At, os_dtype out_t, int64_t ldat, float *scales,
                           const float *col_scale, uint64_t block_mask, void *ws, size_t ws_bytes,
                           cudaStream_t st, const uint64_t *dmask = nullptr) {
    OSK_NVTX("sketch_left");
    OSK_TRY(sketch_left_check(p, A, a_t, m, lda, At, out_t, ldat, scales, block_mask));
    if (m == 0) return OS_OK;
    if (!ws || ws_bytes < sketch_workspace_bytes(p, m, a_t)) return OS_ERR_WORKSPACE;
    if (out_t == OS_FP8E4M3 && !dmask) {
        if (float *stg = fp8_staging(p, ws, ws_bytes, m, a_t)) {
            const int64_t z = (int64_t)p->P * p->b;
            OSK_TRY(sketch_left_impl(p, A, a_t, m, lda, stg, OS_F32, z, nullptr, col_scale, block_mask, ws, ws_bytes,
                                     st, dmask));
            return launch_quantize_fp8(p, stg, z, m, block_mask, At, ldat, scales, fp8_scale_ld(m), st);
        }
    }
    void *Xs = ws_base(ws);
    const float *wts = nullptr;
    OSK_TRY(make_weights(p, col_scale, block_mask, ws_weights(p, ws, m, a_t), &wts, st));
    if (a_t == OS_F32) {
        OSK_TRY(launch_pack_cols<float>((const float *)A, lda, m, p->n, (float *)Xs, st));
        return launch_gather<float>(p, (const float *)Xs, m, wts, At, out_t, ldat, scales, fp8_scale_ld(m),
                                    block_mask, st, m, dmask);
    }
    OSK_TRY(launch_pack_cols<__nv_bfloat16>((const __nv_bfloat16 *)A, lda, m, p->n, (__nv_bfloat16 *)Xs, st));
    return launch_gather<__nv_bfloat16>(p, (const __nv_bfloat16 *)Xs, m, wts, At, out_t, ldat, scales,
                                        fp8_scale_ld(m), block_mask, st, m, dmask);
}

os_status sketch_right_impl(const Plan *p, const void *B, os_dtype b_t, int64_t l, int64_t ldb,
                            void *BtT, os_dtype out_t, int64_t ldbt, float *scales, uint64_t block_mask,
                            void *ws, size_t ws_bytes, cudaStream_t st, const float *row_scale = nullptr,
                            const uint64_t *dmask = nullptr) {
    OSK_NVTX("sketch_right");
    if (!p || l < 0) return OS_ERR_INVALID_ARG;
    if (block_mask) OSK_TRY(check_mask(block_mask, p->P));
    if (b_t != OS_F32 && b_t != OS_BF16) return OS_ERR_DTYPE;
    if (ldb < l) return OS_ERR_INVALID_ARG;
    OSK_TRY(check_out(p, l, BtT, out_t, ldbt, scales));
    if (l == 0) return OS_OK;
    if (!B) return OS_ERR_INVALID_ARG;
    if (out_t == OS_FP8E4M3 && !dmask) {
        if (float *stg = fp8_staging(p, ws, ws_bytes, l, b_t)) {
            const int64_t z = (int64_t)p->P * p->b;
            OSK_TRY(sketch_right_impl(p, B, b_t, l, ldb, stg, OS_F32, z, nullptr, block_mask, ws, ws_bytes, st,
                                      row_scale, dmask));
            return launch_quantize_fp8(p, stg, z, l, block_mask, BtT, ldbt, scales, fp8_scale_ld(l), st);
        }
    }
    // FP32 input: gather whole strips in place, and pack only a ragged remainder
    // narrower than a strip.  Strips are 128 wide for 16-byte aligned rows; other
    // rows are gathered in 124-wide strips (about twice the instructions per row
    // piece: on GB300 that beats packing B first while at most 6 blocks are
    // gathered, 1.82 vs 2.35 ms for 4 blocks of 65536 x 16383, and loses above,
    // 3.28 vs 3.01 ms for 8 blocks).
    const bool aligned = aligned16(B) && ldb % 4 == 0;
    const uint64_t listed = (block_mask ? block_mask : ~0ull) & (p->P >= 64 ? ~0ull : (1ull << p->P) - 1);
    const bool mis_pays = __builtin_popcountll(listed) <= 6;
    const int64_t sw = aligned ? kStrip : kStrip - 4;
    // (a misaligned strip reads up to 4 elements past its end: keep them in the row)
    const int64_t lf = aligned ? l / sw * sw : (l >= 4 ? (l - 4) / sw * sw : 0);
    const bool direct = b_t == OS_F32 && (reinterpret_cast<uintptr_t>(B) & 3u) == 0 &&
                        ldb * 4 < (int64_t(1) << 32) && lf > 0 && (aligned || mis_pays);
    if (direct) {
        // the workspace holds the remainder's strips (if any) and the entry weights
        if ((lf < l || row_scale) && (!ws || ws_bytes < sketch_workspace_bytes(p, l - lf, b_t)))
            return OS_ERR_WORKSPACE;
        const float *wts = nullptr;
        if (row_scale) OSK_TRY(make_weights(p, row_scale, block_mask, ws_weights(p, ws, l - lf, b_t), &wts, st));
        if (aligned)
            OSK_TRY(launch_gather_direct<false>(p, (const float *)B, ldb, lf, wts, BtT, out_t, ldbt, scales,
                                                fp8_scale_ld(l), block_mask, st, l, dmask));
        else
            OSK_TRY(launch_gather_direct<true>(p, (const float *)B, ldb, lf, wts, BtT, out_t, ldbt, scales,
                                               fp8_scale_ld(l), block_mask, st, l, dmask));
        if (lf == l) return OS_OK;
        float *Xs = (float *)ws_base(ws);
        OSK_TRY(launch_pack_rows<float>((const float *)B + lf, ldb, p->n, l - lf, Xs, st));
        char *yt = (char *)BtT + (size_t)lf * ldbt * dtype_size(out_t);
        float *sc = scales ? scales + lf : nullptr;   // slice-major: the remainder's rows start at lf
        return launch_gather<float>(p, Xs, l - lf, wts, yt, out_t, ldbt, sc, fp8_scale_ld(l), block_mask, st, l, dmask);
    }
    // BF16 input with 16-byte aligned rows: 256-wide strips gathered in place (the
    // same 512-byte row pieces as a packed strip), a ragged remainder packed
    constexpr int64_t sw16 = strip_of<__nv_bfloat16>();
    const int64_t lf16 = l / sw16 * sw16;
    if (b_t == OS_BF16 && aligned16(B) && ldb % 8 == 0 && ldb * 2 < (int64_t(1) << 32) && lf16 > 0) {
        if ((lf16 < l || row_scale) && (!ws || ws_bytes < sketch_workspace_bytes(p, l - lf16, b_t)))
            return OS_ERR_WORKSPACE;
        const float *wts = nullptr;
        if (row_scale) OSK_TRY(make_weights(p, row_scale, block_mask, ws_weights(p, ws, l - lf16, b_t), &wts, st));
        const __nv_bfloat16 *Bh = (const __nv_bfloat16 *)B;
        OSK_TRY(launch_gather<__nv_bfloat16>(p, Bh, lf16, wts, BtT, out_t, ldbt, scales, fp8_scale_ld(l), block_mask,
                                             st, l, dmask, sw16, ldb));
        if (lf16 == l) return OS_OK;
        __nv_bfloat16 *Xs = (__nv_bfloat16 *)ws_base(ws);
        OSK_TRY(launch_pack_rows<__nv_bfloat16>(Bh + lf16, ldb, p->n, l - lf16, Xs, st));
        char *yt = (char *)BtT + (size_t)lf16 * ldbt * dtype_size(out_t);
        float *sc = scales ? scales + lf16 : nullptr;
        return launch_gather<__nv_bfloat16>(p, Xs, l - lf16, wts, yt, out_t, ldbt, sc, fp8_scale_ld(l), block_mask,
                                            st, l, dmask);
    }
    if (!ws || ws_bytes < sketch_workspace_bytes(p, l, b_t)) return OS_ERR_WORKSPACE;
    void *Xs = ws_base(ws);
    const float *wts = nullptr;
    OSK_TRY(make_weights(p, row_scale, block_mask, ws_weights(p, ws, l, b_t), &wts, st));
    if (b_t == OS_F32) {
        OSK_TRY(launch_pack_rows<float>((const float *)B, ldb, p->n, l, (float *)Xs, st));
        return launch_gather<float>(p, (const float *)Xs, l, wts, BtT, out_t, ldbt, scales, fp8_scale_ld(l),
                                    block_mask, st, l, dmask);
    }
    OSK_TRY(launch_pack_rows<__nv_bfloat16>((const __nv_bfloat16 *)B, ldb, p->n, l, (__nv_bfloat16 *)Xs, st));
    return launch_gather<__nv_bfloat16>(p, (const __nv_bfloat16 *)Xs, l, wts, BtT, out_t, ldbt, scales,
                                        fp8_scale_ld(l), block_mask, st, l, dmask);
}

os_status unsketch_cols_impl(const Plan *p, const float *T, int64_t m, int64_t ldt, uint64_t mask,
                             float scale, void *dX, os_dtype x_t, int64_t ldx, cudaStream_t st) {
    if (!p || m < 0) return OS_ERR_INVALID_ARG;
    OSK_TRY(check_mask(mask, p->P));
    const int kcnt = __builtin_popcountll(mask);
    if (ldt < (int64_t)kcnt * p->b || ldx < p->n) return OS_ERR_INVALID_ARG;
    if (x_t != OS_F32 && x_t != OS_BF16) return OS_ERR_DTYPE;
    if (m == 0) return OS_OK;   // an empty dX
    if (!T || !dX) return OS_ERR_INVALID_ARG;
    const BlockList kept = mask_to_list(mask, p->P);
    // rows of T staged per CTA (1024 threads): 4, 2 or 1, the most that fit in
    // 200 KB, else the unstaged kernel
    const int64_t kb = (int64_t)kcnt * p->b;
    const size_t row_bytes = (size_t)kb * sizeof(float);
    const int R = row_bytes * 4 <= 200 * 1024 ? 4 : row_bytes * 2 <= 200 * 1024 ? 2 : row_bytes <= 200 * 1024 ? 1 : 0;
    if (R > 0) {
        const size_t smem = row_bytes * R;
        const unsigned gxs = (unsigned)((m + R - 1) / R);
        auto launch = [&](auto kern, auto *out) -> os_status {
            if (smem > 48 * 1024)
                OSK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<gxs, 1024, smem, st>>>(T, m, ldt, kb, p->hs, p->n, p->b, kept, scale, out, ldx);
            return check_launch();
        };
        if (x_t == OS_F32) {
            float *o = (float *)dX;
            if (R == 4) return launch(unsketch_cols_smem_kernel<float, 4>, o);
            if (R == 2) return launch(unsketch_cols_smem_kernel<float, 2>, o);
            return launch(unsketch_cols_smem_kernel<float, 1>, o);
        }
        __nv_bfloat16 *o = (__nv_bfloat16 *)dX;
        if (R == 4) return launch(unsketch_cols_smem_kernel<__nv_bfloat16, 4>, o);
        if (R == 2) return launch(unsketch_cols_smem_kernel<__nv_bfloat16, 2>, o);
        return launch(unsketch_cols_smem_kernel<__nv_bfloat16, 1>, o);
    }
    if (m > 65535) return OS_ERR_UNSUPPORTED;
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
    if (!p || l < 0) return OS_ERR_INVALID_ARG;
    OSK_TRY(check_mask(mask, p->P));
    if (ldu < l || ldg < l) return OS_ERR_INVALID_ARG;
    if (g_t != OS_F32 && g_t != OS_BF16) return OS_ERR_DTYPE;
    if (l == 0) return OS_OK;   // an empty dG
    if (!U || !dG) return OS_ERR_INVALID_ARG;
    const BlockList kept = mask_to_list(mask, p->P);
    dim3 grid((unsigned)((p->n + 7) / 8), (unsigned)((l + 1023) / 1024));
    if (grid.y > 65535u) return OS_ERR_UNSUPPORTED;
    const bool vec = l % 4 == 0 && ldu % 4 == 0 && ldg % 4 == 0 && aligned16(U) && aligned16(dG);
    if (g_t == OS_F32) {
        if (vec)
            unsketch_rows_vec_kernel<float><<<grid, 256, 0, st>>>(U, l, ldu, p->hs, p->n, p->b, kept, scale,
                                                                  (float *)dG, ldg);
        else
            unsketch_rows_kernel<float><<<grid, 256, 0, st>>>(U, l, ldu, p->hs, p->n, p->b, kept, scale,
                                                              (float *)dG, ldg);
    } else {
        if (vec)
            unsketch_rows_vec_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(U, l, ldu, p->hs, p->n, p->b, kept,
                                                                          scale, (__nv_bfloat16 *)dG, ldg);
        else
            unsketch_rows_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(U, l, ldu, p->hs, p->n, p->b, kept,
                                                                      scale, (__nv_bfloat16 *)dG, ldg);
    }
    return check_launch();
}

}  // namespace osk

using namespace osk;

extern "C" os_status oversketch_sketch_workspace(oversketch_plan_t plan, int64_t free_extent,
                                                 os_dtype in_t, size_t *bytes) {
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p || !bytes || free_extent < 0) return OS_ERR_INVALID_ARG;
    if (in_t != OS_F32 && in_t != OS_BF16) return OS_ERR_DTYPE;
    *bytes = sketch_workspace_bytes(p, free_extent, in_t);
    return OS_OK;
}

extern "C" os_status oversketch_sketch_left(oversketch_plan_t plan, const void *A, os_dtype a_t,
                                            int64_t m, int64_t lda, void *At, os_dtype out_t,
                                            int64_t ldat, float *scales, const float *col_scale,
                                            uint64_t block_mask, void *workspace, size_t ws_bytes,
                                            void *stream) {
    return sketch_left_impl(reinterpret_cast<const Plan *>(plan), A, a_t, m, lda, At, out_t, ldat,
                            scales, col_scale, block_mask, workspace, ws_bytes, as_stream(stream));
}

extern "C" os_status oversketch_sketch_right(oversketch_plan_t plan, const void *B, os_dtype b_t,
                                             int64_t l, int64_t ldb, void *BtT, os_dtype out_t,
                                             int64_t ldbt, float *scales, const float *row_scale,
                                             uint64_t block_mask, void *workspace, size_t ws_bytes,
                                             void *stream) {
    return sketch_right_impl(reinterpret_cast<const Plan *>(plan), B, b_t, l, ldb, BtT, out_t, ldbt,
                             scales, block_mask, workspace, ws_bytes, as_stream(stream), row_scale);
}

extern "C" os_status oversketch_unsketch_cols(oversketch_plan_t plan, const float *T, int64_t m,
                                              int64_t ldt, uint64_t mask, float scale, void *dX,
                                              os_dtype x_t, int64_t ldx, void *stream) {
    OSK_NVTX("unsketch_cols");
    return unsketch_cols_impl(reinterpret_cast<const Plan *>(plan), T, m, ldt, mask, scale, dX, x_t,
                              ldx, as_stream(stream));
}

extern "C" os_status oversketch_unsketch_rows(oversketch_plan_t plan, const float *U, int64_t l,
                                              int64_t ldu, uint64_t mask, float scale, void *dG,
                                              os_dtype g_t, int64_t ldg, void *stream) {
    OSK_NVTX("unsketch_rows");
    return unsketch_rows_impl(reinterpret_cast<const Plan *>(plan), U, l, ldu, mask, scale, dG, g_t,
                              ldg, as_stream(stream));
}
