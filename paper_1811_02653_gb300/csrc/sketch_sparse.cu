// Left sketch of a sparse operand stored dense (Alg. 4 step 3 / Alg. 5 over the
// nonzeros only: the paper prices sketching at O(nnz(A) (N+e)), Sec. 4).
//
//   At[r, j*b + c] = sum_{i : A[r,i] != 0, h_j(i) = c} sigma_j(i) * s_i * A[r, i]
//
// The dense gather path reads every element k times from L2 (once per kept
// block) and, when a 128-wide strip of the sketched dimension no longer fits in
// L2 (n = 2^20: 512 MB per strip), from DRAM.  Here one CTA per row reads the
// row once, coalesced, and routes only its nonzeros.  Two kernels, one after
// the other:
//
// One-pass kernel (b <= 4096): the whole row's nonzeros are held in shared
// memory, then routed one kept block at a time (sp_row_onepass):
//   1. compaction: warp w streams the w-th 32nd of the row (16 elements per
//      lane per step, the next step's loads issued before this one is
//      processed, an L2 prefetch two steps ahead) and appends its nonzeros
//      (index, value) to its own region in ascending index order: warp scans
//      only, no block barrier;
//   2. per kept block: bucket codes h_j(i), sigma_j(i) of every entry and the
//      bucket counts (integer shared-memory atomics), a scan into bucket
//      starts, a scatter of entry numbers into their buckets, then each thread
//      sorts the entry numbers of its 4 buckets and adds the members in that
//      order (= ascending index) and writes the sums out in the output dtype
//      (BF16 RNE, FP8 with the per-128-column UE8M0 scale, FP32, or TF32
//      hi/lo planes).  No float atomics: bitwise reproducible.
//   A row with more nonzeros in some 32nd than a region holds is left to the
//   flushing kernel: its first kept output gets a marker value.
//
// Flushing kernel (any density; all rows when b > 4096, else the marked ones):
//   1. compaction: the row streams through registers in chunks of 16 elements
//      per thread (an L2 prefetch runs a few chunks ahead); a block-wide scan
//      appends the nonzeros in ascending index order to an entry buffer;
//   2. flush (buffer full or row done): values take their scale s_i; then for
//      every kept block the entries are counted per bucket, scanned into
//      bucket offsets, scattered into their buckets, and each thread adds the
//      members of its own buckets to their accumulators in ascending index
//      order (the same order as the one-pass kernel: the same bits);
//   3. the row's k*b accumulators are written out in the output dtype.
//   Shared memory holds the k*b accumulators and two b-entry bucket tables:
//   4*k*b + 8*b bytes plus an entry buffer of at least 1024 entries must fit
//   (k*b <= kSparseMaxBuckets).
#include <cstdint>
#include <type_traits>

#include "common.cuh"

namespace osk {

namespace {

constexpr int kSpThreads = 1024;
constexpr int kSpWarps = kSpThreads / 32;
constexpr int kSpElems = 16;                         // elements per thread per chunk
constexpr int kSpChunk = kSpThreads * kSpElems;      // elements per chunk
constexpr int kSpPrefetchChunks = 4;                 // L2 prefetch distance
constexpr int kSmemLimit = 232448;                   // usable shared memory per CTA (227 KB)
constexpr int kEntryBytes = 20;                      // index, value, code, sorted entry, sorted value
constexpr int kMinEntries = 1024;

}  // namespace

// Largest number of kept buckets (k*b) whose accumulators fit beside a useful entry buffer.
constexpr int kSparseMaxBuckets = 32768;

namespace {

// 16 consecutive elements of a row as FP32 (vector loads when aligned, bounds-checked otherwise).
template <typename InT, bool kVec>
__device__ __forceinline__ void load16(const InT *__restrict__ p, int64_t i0, int64_t n, float (&v)[16]) {
    if (kVec && i0 + 16 <= n) {
        if constexpr (std::is_same<InT, float>::value) {
            const float4 *q = reinterpret_cast<const float4 *>(p + i0);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 t = __ldcs(q + u);   // streamed: no reuse
                v[4 * u] = t.x; v[4 * u + 1] = t.y; v[4 * u + 2] = t.z; v[4 * u + 3] = t.w;
            }
        } else {
            const uint4 *q = reinterpret_cast<const uint4 *>(p + i0);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const uint4 t = __ldcs(q + u);
                const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w[h]));
                    v[8 * u + 2 * h] = f.x;
                    v[8 * u + 2 * h + 1] = f.y;
                }
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            if (i0 + q < n) {
                if constexpr (std::is_same<InT, float>::value) v[q] = p[i0 + q];
                else v[q] = __bfloat162float(p[i0 + q]);
            } else {
                v[q] = 0.f;
            }
        }
    }
}

// Exclusive block-wide scan of one int per thread (1024 threads); returns the
// thread's offset and writes the total to *total.  Two barriers.
__device__ __forceinline__ int block_scan(int x, int *warp_tot, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int t = warp_tot[lane];
        int ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        warp_tot[32 + lane] = ti - t;            // exclusive warp offsets
        if (lane == 31) warp_tot[64] = ti;
    }
    __syncthreads();
    *total = warp_tot[64];
    return warp_tot[32 + warp] + inc - x;
}

struct SpSmem {
    float *state;        // [k*b] the row's accumulators, block t at t*b
    uint32_t *ent_i;     // [emax] entry index i
    float *ent_v;        // [emax] entry value (scaled by s_i at flush time)
    uint32_t *codes;     // [emax] hs entry of the current block (bucket | sign)
    uint32_t *srt_c;     // [emax] entry numbers grouped by bucket
    float *srt_v;        // [emax] signed values grouped by bucket
    int *bcnt;           // [b] entries per bucket, then the scatter cursor
    int *bstart;         // [b+1] first entry of each bucket in srt_*
    int *warp_tot;       // [72] block-scan scratch
};

// shared memory beyond the accumulators and the entry arrays
__host__ __device__ constexpr size_t sp_fixed_bytes(int b) { return sizeof(int) * ((size_t)2 * b + 1 + 72 + 7); }

__device__ __forceinline__ SpSmem sp_layout(void *base, int kb, int b, int emax) {
    SpSmem s;
    s.state = reinterpret_cast<float *>(base);
    s.ent_i = reinterpret_cast<uint32_t *>(s.state + kb);
    s.ent_v = reinterpret_cast<float *>(s.ent_i + emax);
    s.codes = reinterpret_cast<uint32_t *>(s.ent_v + emax);
    s.srt_c = s.codes + emax;
    s.srt_v = reinterpret_cast<float *>(s.srt_c + emax);
    s.bcnt = reinterpret_cast<int *>(s.srt_v + emax);
    s.bstart = s.bcnt + b;
    s.warp_tot = s.bstart + b + 1;
    return s;
}

constexpr int kSpPerThread = 8;   // entries per thread in a flush (emax <= kSpThreads * kSpPerThread)

// Route the nent buffered entries into the accumulators of every kept block.
// Called by all threads; starts and ends with the buffer stable (barriers).
// Per block: count the entries of every bucket (integer shared-memory atomics),
// scan the counts into bucket offsets, scatter the entry numbers into their
// buckets (in whatever order the atomics give), then every thread adds the
// members of its own buckets in ascending entry order (= ascending index i),
// picking them from the short unordered lists: a fixed order, no float atomics.
template <bool kScale>
__device__ void sp_flush(const SpSmem &s, int nent, const uint32_t *__restrict__ hs, int64_t n, int32_t b,
                         const BlockList &blocks, const float *__restrict__ col_scale, uint64_t seed,
                         bool hashed) {
    const int tid = threadIdx.x;
    if constexpr (kScale) {
        // all of a thread's scale loads in flight at once
        float sc[kSpPerThread];
#pragma unroll
        for (int u = 0; u < kSpPerThread; ++u) {
            const int e = tid + u * kSpThreads;
            sc[u] = e < nent ? __ldg(col_scale + s.ent_i[e]) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kSpPerThread; ++u) {
            const int e = tid + u * kSpThreads;
            if (e < nent) s.ent_v[e] *= sc[u];
        }
    }
    // bucket codes of the next block, one block ahead: recomputed from the seed for
    // hashed plans (random reads of the table would miss L2 while the operand
    // streams through it), else loaded (the latency hides behind the current block)
    uint32_t nxt[kSpPerThread];
    auto load_codes = [&](int t) {
        if (hashed) {
            const uint64_t key = block_key(seed, blocks.idx[t]);
#pragma unroll
            for (int u = 0; u < kSpPerThread; ++u) {
                const int e = tid + u * kSpThreads;
                nxt[u] = e < nent ? hash_code(key, (int64_t)s.ent_i[e], b) : 0u;
            }
        } else {
            const uint32_t *hj = hs + (int64_t)blocks.idx[t] * n;
#pragma unroll
            for (int u = 0; u < kSpPerThread; ++u) {
                const int e = tid + u * kSpThreads;
                nxt[u] = e < nent ? __ldg(hj + s.ent_i[e]) : 0u;
            }
        }
    };
    load_codes(0);
    for (int t = 0; t < blocks.count; ++t) {
        for (int c = tid; c < b; c += kSpThreads) s.bcnt[c] = 0;
#pragma unroll
        for (int u = 0; u < kSpPerThread; ++u) {
            const int e = tid + u * kSpThreads;
            if (e < nent) s.codes[e] = nxt[u];
        }
        __syncthreads();
        if (t + 1 < blocks.count) load_codes(t + 1);
        // counts (the thread's codes stay in registers for the scatter)
        uint32_t code[kSpPerThread];
        float val[kSpPerThread];
#pragma unroll
        for (int u = 0; u < kSpPerThread; ++u) {
            const int e = tid + u * kSpThreads;
            code[u] = e < nent ? s.codes[e] : 0u;
            val[u] = e < nent ? s.ent_v[e] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kSpPerThread; ++u)
            if (tid + u * kSpThreads < nent) atomicAdd(&s.bcnt[code[u] & kIndexMask], 1);
        __syncthreads();
        // exclusive scan of the b counts: thread t owns a contiguous run of buckets
        const int per = (b + kSpThreads - 1) / kSpThreads;
        const int c0 = min(b, tid * per), c1 = min(b, c0 + per);
        int run = 0;
        for (int c = c0; c < c1; ++c) run += s.bcnt[c];
        int total = 0;
        int off = block_scan(run, s.warp_tot, &total);
        for (int c = c0; c < c1; ++c) {
            const int k = s.bcnt[c];
            s.bstart[c] = off;
            s.bcnt[c] = off;          // cursor for the scatter
            off += k;
        }
        if (tid == 0) s.bstart[b] = total;
        __syncthreads();
        // scatter entry numbers and signed values into their buckets
        int pos[kSpPerThread];
#pragma unroll
        for (int u = 0; u < kSpPerThread; ++u)
            pos[u] = tid + u * kSpThreads < nent ? atomicAdd(&s.bcnt[code[u] & kIndexMask], 1) : 0;
#pragma unroll
        for (int u = 0; u < kSpPerThread; ++u) {
            const int e = tid + u * kSpThreads;
            if (e < nent) {
                s.srt_c[pos[u]] = (uint32_t)e;
                s.srt_v[pos[u]] = (code[u] & kSignBit) ? -val[u] : val[u];
            }
        }
        __syncthreads();
        // each bucket's members in ascending entry order, one FP32 chain per bucket
        float *acc = s.state + t * b;
        for (int c = tid; c < b; c += kSpThreads) {
            const int p0 = s.bstart[c], p1 = s.bstart[c + 1];
            if (p0 == p1) continue;
            float a = acc[c];
            if (p1 - p0 == 1) {
                a += s.srt_v[p0];
            } else if (p1 - p0 == 2) {
                const bool swap = s.srt_c[p0] > s.srt_c[p0 + 1];
                const float x0 = s.srt_v[p0], x1 = s.srt_v[p0 + 1];
                a += swap ? x1 : x0;
                a += swap ? x0 : x1;
            } else {
                // longer lists: the members in ascending entry order by repeated minimum
                int last = -1;
                for (int k = p0; k < p1; ++k) {
                    int best = 0x7fffffff, bp = p0;
                    for (int q = p0; q < p1; ++q) {
                        const int eq = (int)s.srt_c[q];
                        if (eq > last && eq < best) best = eq, bp = q;
                    }
                    a += s.srt_v[bp];
                    last = best;
                }
            }
            acc[c] = a;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void l2_prefetch(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<uint64_t>(p)), "r"(bytes)
                 : "memory");
}

template <typename OutT>
__device__ __forceinline__ void sp_store(OutT *dst, int64_t plane_elems, float v) {
    if constexpr (std::is_same<OutT, Tf32Pair>::value) {
        // FP32 as hi + lo: hi keeps 10 mantissa bits (exact in TF32), lo = x - hi (exact)
        float *d = reinterpret_cast<float *>(dst);
        const float hi = __uint_as_float(__float_as_uint(v) & 0xffffe000u);
        d[0] = hi;
        d[plane_elems] = v - hi;
    } else if constexpr (std::is_same<OutT, float>::value) {
        *dst = v;
    } else {
        *dst = __float2bfloat16_rn(v);
    }
}

// The row in flushes (any density): the nonzeros are appended to an entry buffer
// in ascending index order and routed into the k*b accumulators whenever it
// fills; see the file comment.  Starts and ends with all threads in step.
template <typename InT, typename OutT, bool kScale>
__device__ __forceinline__ void sp_row_flushing(const InT *__restrict__ row, int64_t r, int64_t n, bool vec,
                                const uint32_t *__restrict__ hs, uint64_t seed, bool hashed, int32_t b,
                                const BlockList &blocks, int emax, const float *__restrict__ col_scale,
                                OutT *__restrict__ At, int64_t ldat, float *__restrict__ scales, int64_t lds,
                                int64_t plane_elems, void *smem) {
    const int kb = blocks.count * b;
    const SpSmem s = sp_layout(smem, kb, b, emax);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t chunk_bytes = (int64_t)kSpChunk * sizeof(InT);
    for (int q = tid; q < kb; q += kSpThreads) s.state[q] = 0.f;
    int nent = 0;
    for (int64_t base = 0; base < n; base += kSpChunk) {
        if (vec && tid == 0) {
            const int64_t pf = base + (int64_t)kSpPrefetchChunks * kSpChunk;
            if (pf < n) {
                const int64_t bytes = ((n - pf) * (int64_t)sizeof(InT) < chunk_bytes
                                           ? (n - pf) * (int64_t)sizeof(InT) : chunk_bytes) & ~int64_t(15);
                if (bytes > 0) l2_prefetch(row + pf, (uint32_t)bytes);
            }
        }
        float v[kSpElems];
        const int64_t i0 = base + (int64_t)tid * kSpElems;
        if (vec) load16<InT, true>(row, i0, n, v);
        else load16<InT, false>(row, i0, n, v);
        int cnt = 0;
#pragma unroll
        for (int q = 0; q < kSpElems; ++q) cnt += v[q] != 0.f;
        int total = 0;
        const int off = block_scan(cnt, s.warp_tot, &total);
        // append in index order; a chunk with more nonzeros than the buffer holds
        // is appended in pieces, flushing in between
        int done = 0;
        while (done < total) {
            if (nent == emax) {
                sp_flush<kScale>(s, nent, hs, n, b, blocks, col_scale, seed, hashed);
                nent = 0;
            }
            const int take = min(total - done, emax - nent);
            int rank = off;
#pragma unroll
            for (int q = 0; q < kSpElems; ++q) {
                if (v[q] != 0.f) {
                    if (rank >= done && rank < done + take) {
                        s.ent_i[nent + rank - done] = (uint32_t)(i0 + q);
                        s.ent_v[nent + rank - done] = v[q];
                    }
                    ++rank;
                }
            }
            nent += take;
            done += take;
            if (done < total) __syncthreads();   // the pieces so far are visible to the flush
        }
    }
    __syncthreads();
    if (nent > 0) sp_flush<kScale>(s, nent, hs, n, b, blocks, col_scale, seed, hashed);

    // write the row's sums of every listed block
    for (int t = 0; t < blocks.count; ++t) {
        const int64_t col0 = (int64_t)blocks.idx[t] * b;
        const float *acc = s.state + t * b;
        OutT *dst = At + r * ldat + col0;
        if constexpr (sizeof(OutT) == 1) {
            // FP8: warp per 128-column slice; lane holds 4 consecutive sums
            for (int sl = warp; sl < b / 128; sl += kSpWarps) {
                const float4 x = *reinterpret_cast<const float4 *>(acc + 128 * sl + 4 * lane);
                float a = fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w)));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
                const int e = fp8_scale_exponent(a);
                const float inv = ldexpf(1.f, -e);
                __nv_fp8_e4m3 q[4] = {__nv_fp8_e4m3(x.x * inv), __nv_fp8_e4m3(x.y * inv),
                                      __nv_fp8_e4m3(x.z * inv), __nv_fp8_e4m3(x.w * inv)};
                *reinterpret_cast<uint32_t *>(dst + 128 * sl + 4 * lane) = *reinterpret_cast<uint32_t *>(q);
                if (lane == 0) scales[(col0 / 128 + sl) * lds + r] = ldexpf(1.f, e);
            }
        } else {
            for (int c = tid; c < b; c += kSpThreads) sp_store(dst + c, plane_elems, acc[c]);
        }
    }
    __syncthreads();   // the shared memory is free for the next row
}

// Shared memory of the one-pass row (b <= 4096): the bucket counts and starts,
// then per warp a region of cw entries (index, value), and per entry its bucket
// code in the current block and its place in the bucket order.
constexpr int kOpElems = 16;   // one-pass compaction: elements per lane per step
constexpr int kOpAhead = 2;    // L2 prefetch distance of a warp, in steps

struct Sp1Smem {
    int *cnt;            // [b] entries per bucket, then the scatter cursor
    int *bstart;         // [b+1] first entry of each bucket in srt
    int *warp_tot;       // [72] block-scan scratch
    uint32_t *idx;       // [32*cw] column index of each entry
    float *val;          // [32*cw] its value (times s_i)
    uint16_t *code;      // [32*cw] bucket | 0x8000 for sign -1, current block
    uint16_t *srt;       // [32*cw] entry numbers grouped by bucket
};

__host__ __device__ constexpr size_t sp1_fixed_bytes(int b) { return sizeof(int) * ((size_t)2 * b + 1 + 72 + 7); }
constexpr int kSp1EntryBytes = 12;

__device__ __forceinline__ Sp1Smem sp1_layout(void *base, int b, int cw) {
    Sp1Smem s;
    s.cnt = reinterpret_cast<int *>(base);
    s.bstart = s.cnt + b;
    s.warp_tot = s.bstart + b + 1;
    s.idx = reinterpret_cast<uint32_t *>(s.warp_tot + 72 + 7);
    s.val = reinterpret_cast<float *>(s.idx + 32 * cw);
    s.code = reinterpret_cast<uint16_t *>(s.val + 32 * cw);
    s.srt = s.code + 32 * cw;
    return s;
}

// The row in one pass (b <= 4096, at most cw nonzeros in each 32nd of the row):
//   1. warp w compacts the w-th 32nd of the row into its own region (a warp
//      scan of each lane's nonzero count, no block barrier), entries in
//      ascending index order; each step's loads are issued before the previous
//      step is processed, an L2 prefetch runs two steps ahead, and the start of
//      the next row is prefetched before the routing;
//   2. per kept block: codes and bucket counts (integer atomics), a scan into
//      bucket starts, a scatter of entry numbers into their buckets, then each
//      thread sums the members of its 4 buckets in ascending entry order (the
//      order of the flushing path: both give the same bits) and writes them
//      out directly, so no accumulators outlive the block.
// Returns false, with nothing written, when a region overflows.
template <typename InT, typename OutT, bool kScale>
__device__ bool sp_row_onepass(const InT *__restrict__ row, const InT *__restrict__ next_row, int64_t r,
                               int64_t n, bool vec, const uint32_t *__restrict__ hs, uint64_t seed, bool hashed,
                               int32_t b, const BlockList &blocks, int cw, const float *__restrict__ col_scale,
                               OutT *__restrict__ At, int64_t ldat, float *__restrict__ scales, int64_t lds,
                               int64_t plane_elems, void *smem) {
    const Sp1Smem s = sp1_layout(smem, b, cw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kOp = kOpElems;                             // elements per lane per step
    constexpr int64_t kStep = 32 * kOp;                       // elements per warp step
    const int64_t seg = ((n + 31) / 32 + kOp - 1) / kOp * kOp;
    const int64_t s0 = min(n, (int64_t)warp * seg), s1 = min(n, s0 + seg);
    uint32_t *ridx = s.idx + warp * cw;
    float *rval = s.val + warp * cw;
    int have = 0;          // entries in this warp's region
    bool over = false;
    // one step of kOp elements per lane: its loads are issued a step ahead
    auto load_step = [&](int64_t i0, float (&v)[kOp]) {
        const int64_t il = i0 + (int64_t)kOp * lane;
        if (i0 < s1 && il < s1) {
#pragma unroll
            for (int h = 0; h < kOp / 16; ++h) {
                float(&vh)[16] = *reinterpret_cast<float(*)[16]>(v + 16 * h);
                if (vec) load16<InT, true>(row, il + 16 * h, n, vh);
                else load16<InT, false>(row, il + 16 * h, n, vh);
            }
        } else {
#pragma unroll
            for (int q = 0; q < kOp; ++q) v[q] = 0.f;
        }
    };
    // append the nonzeros of one step (false: the region is full, nothing appended)
    auto process = [&](const float (&v)[kOp], int64_t i0) -> bool {
        if (vec && lane == 0) {
            const int64_t pf = i0 + kOpAhead * kStep;
            if (pf < s1) {
                const int64_t bytes = (min(kStep, s1 - pf) * (int64_t)sizeof(InT)) & ~int64_t(15);
                if (bytes > 0) l2_prefetch(row + pf, (uint32_t)bytes);
            }
        }
        const int64_t il = i0 + (int64_t)kOp * lane;
        uint32_t nz = 0;
#pragma unroll
        for (int q = 0; q < kOp; ++q) nz |= (v[q] != 0.f ? 1u : 0u) << q;
        const int c = __popc(nz);
        int inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const int total = __shfl_sync(0xffffffffu, inc, 31);
        if (have + total > cw) return false;   // warp-uniform
        int pos = have + inc - c;
#pragma unroll
        for (int q = 0; q < kOp; ++q) {
            if ((nz >> q) & 1u) {
                ridx[pos] = (uint32_t)(il + q);
                rval[pos] = v[q];
                ++pos;
            }
        }
        have += total;
        return true;
    };
    // two steps per pass, each one's loads issued before the other is processed
    float va[kOp], vb[kOp];
    load_step(s0, va);
    for (int64_t i0 = s0; i0 < s1; i0 += 2 * kStep) {
        load_step(i0 + kStep, vb);
        if (!process(va, i0)) {
            over = true;
            break;
        }
        if (i0 + kStep >= s1) break;
        load_step(i0 + 2 * kStep, va);
        if (!process(vb, i0 + kStep)) {
            over = true;
            break;
        }
    }
    if (vec && next_row && lane == 0 && s0 < s1) {
        const int64_t bytes = (min(kOpAhead * kStep, s1 - s0) * (int64_t)sizeof(InT)) & ~int64_t(15);
        if (bytes > 0) l2_prefetch(next_row + s0, (uint32_t)bytes);
    }
    if (!__syncthreads_and(!over)) return false;

    if constexpr (kScale) {
#pragma unroll 4
        for (int k = lane; k < have; k += 32) rval[k] *= __ldg(col_scale + ridx[k]);
    }
    for (int c = tid; c < b; c += kSpThreads) s.cnt[c] = 0;
    __syncthreads();

    for (int t = 0; t < blocks.count; ++t) {
        const int jb = blocks.idx[t];
        const uint64_t key = hashed ? block_key(seed, jb) : 0ull;
        const uint32_t *hj = hs + (int64_t)jb * n;
        // codes and counts of the warp's own entries
        for (int k = lane; k < have; k += 32) {
            const uint32_t i = ridx[k];
            const uint32_t cd = hashed ? hash_code(key, (int64_t)i, b) : __ldg(hj + i);
            const uint32_t bk = cd & kIndexMask;
            s.code[warp * cw + k] = (uint16_t)(bk | ((cd & kSignBit) ? 0x8000u : 0u));
            atomicAdd(&s.cnt[bk], 1);
        }
        __syncthreads();
        // bucket starts: thread t owns buckets 4t .. 4t+3
        const int c0 = min(b, 4 * tid), c1 = min(b, 4 * tid + 4);
        int run = 0;
        for (int c = c0; c < c1; ++c) run += s.cnt[c];
        int all = 0;
        int off = block_scan(run, s.warp_tot, &all);
        for (int c = c0; c < c1; ++c) {
            const int k = s.cnt[c];
            s.bstart[c] = off;
            s.cnt[c] = off;
            off += k;
        }
        if (tid == 0) s.bstart[b] = all;
        __syncthreads();
        // entry numbers into their buckets
        for (int k = lane; k < have; k += 32) {
            const int e = warp * cw + k;
            const int p = atomicAdd(&s.cnt[s.code[e] & 0x7fff], 1);
            s.srt[p] = (uint16_t)e;
        }
        __syncthreads();
        // each bucket's members in ascending entry order (= ascending index)
        float a[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = 4 * tid + q;
            a[q] = 0.f;
            if (c < b) {
                const int p0 = s.bstart[c], p1 = s.bstart[c + 1];
                auto add = [&](int e) {
                    const float x = s.val[e];
                    a[q] += (s.code[e] & 0x8000u) ? -x : x;
                };
                if (p1 - p0 == 1) {
                    add(s.srt[p0]);
                } else if (p1 - p0 == 2) {
                    const int e0 = s.srt[p0], e1 = s.srt[p0 + 1];
                    add(min(e0, e1));
                    add(max(e0, e1));
                } else if (p1 > p0) {
                    // longer lists: insertion sort of the bucket's own slice of srt
                    for (int k = p0 + 1; k < p1; ++k) {
                        const uint16_t x = s.srt[k];
                        int j = k - 1;
                        for (; j >= p0 && s.srt[j] > x; --j) s.srt[j + 1] = s.srt[j];
                        s.srt[j + 1] = x;
                    }
                    for (int k = p0; k < p1; ++k) add(s.srt[k]);
                }
                s.cnt[c] = 0;
            }
        }
        const int64_t col0 = (int64_t)jb * b;
        OutT *dst = At + r * ldat + col0;
        if constexpr (sizeof(OutT) == 1) {
            // FP8: warp w holds the 128-column slice w of the block
            if (128 * warp < b) {
                float am = fmaxf(fmaxf(fabsf(a[0]), fabsf(a[1])), fmaxf(fabsf(a[2]), fabsf(a[3])));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
                const int e = fp8_scale_exponent(am);
                const float inv = ldexpf(1.f, -e);
                __nv_fp8_e4m3 qv[4] = {__nv_fp8_e4m3(a[0] * inv), __nv_fp8_e4m3(a[1] * inv),
                                       __nv_fp8_e4m3(a[2] * inv), __nv_fp8_e4m3(a[3] * inv)};
                *reinterpret_cast<uint32_t *>(dst + 4 * tid) = *reinterpret_cast<uint32_t *>(qv);
                if (lane == 0) scales[(col0 / 128 + warp) * lds + r] = ldexpf(1.f, e);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (4 * tid + q < b) sp_store(dst + 4 * tid + q, plane_elems, a[q]);
        }
        __syncthreads();   // counts cleared, codes and bucket lists free for the next block
    }
    return true;
}

// Bits that mark a row the one-pass kernel left to the flushing kernel, stored
// in the row's first kept output: a quiet NaN with a payload (FP32, BF16, and
// the hi plane of TF32 pairs) or the E4M3 NaN code.  A genuine output with the
// same bits only makes the flushing kernel recompute that row.
template <typename OutT>
struct RowMark;
template <> struct RowMark<float> { using U = uint32_t; static constexpr U bits = 0x7fd1c0deu; };
template <> struct RowMark<Tf32Pair> { using U = uint32_t; static constexpr U bits = 0x7fd1c0deu; };
template <> struct RowMark<__nv_bfloat16> { using U = uint16_t; static constexpr U bits = 0x7fd1u; };
template <> struct RowMark<__nv_fp8_e4m3> { using U = uint8_t; static constexpr U bits = 0x7fu; };

template <typename OutT>
__device__ __forceinline__ typename RowMark<OutT>::U *row_mark(OutT *At, int64_t r, int64_t ldat, int64_t col) {
    return reinterpret_cast<typename RowMark<OutT>::U *>(At + r * ldat + col);
}

// The one-pass kernel: one CTA per row (persistent over rows); a row whose
// nonzeros overflow a warp's region is marked for the flushing kernel.
template <typename InT, typename OutT, bool kScale>
__global__ void __launch_bounds__(kSpThreads, 1)
sketch_left_onepass_kernel(const InT *__restrict__ A, int64_t lda, int64_t m, int64_t n, bool vec,
                           const uint32_t *__restrict__ hs, uint64_t seed, bool hashed, int32_t b,
                           BlockList blocks, int cw,
                           const float *__restrict__ col_scale, OutT *__restrict__ At, int64_t ldat,
                           float *__restrict__ scales, int64_t lds, int64_t plane_elems) {
    extern __shared__ float4 sp_smem[];
    for (int64_t r = blockIdx.x; r < m; r += gridDim.x) {
        const InT *row = A + r * lda;
        const InT *next = r + gridDim.x < m ? row + (int64_t)gridDim.x * lda : nullptr;
        if (!sp_row_onepass<InT, OutT, kScale>(row, next, r, n, vec, hs, seed, hashed, b, blocks, cw, col_scale,
                                               At, ldat, scales, lds, plane_elems, sp_smem) &&
            threadIdx.x == 0)
            *row_mark(At, r, ldat, (int64_t)blocks.idx[0] * b) = RowMark<OutT>::bits;
    }
}

// The flushing kernel: one CTA per row (persistent over rows); with kMarked,
// only the rows the one-pass kernel marked.
template <typename InT, typename OutT, bool kScale, bool kMarked>
__global__ void __launch_bounds__(kSpThreads, 1)
sketch_left_sparse_kernel(const InT *__restrict__ A, int64_t lda, int64_t m, int64_t n, bool vec,
                          const uint32_t *__restrict__ hs, uint64_t seed, bool hashed, int32_t b,
                          BlockList blocks, int emax,
                          const float *__restrict__ col_scale, OutT *__restrict__ At, int64_t ldat,
                          float *__restrict__ scales, int64_t lds, int64_t plane_elems) {
    extern __shared__ float4 sp_smem[];
    if constexpr (kMarked) {
        // 32 of the CTA's rows at a time: every warp reads their marks (the same
        // ballot in every warp), then the CTA runs the marked ones
        const int lane = threadIdx.x & 31;
        for (int64_t base = blockIdx.x; base < m; base += (int64_t)gridDim.x * 32) {
            const int64_t rl = base + (int64_t)lane * gridDim.x;
            const bool take = rl < m && *row_mark(At, rl, ldat, (int64_t)blocks.idx[0] * b) == RowMark<OutT>::bits;
            uint32_t todo = __ballot_sync(0xffffffffu, take);
            while (todo) {
                const int t = __ffs(todo) - 1;
                todo &= todo - 1;
                const int64_t r = base + (int64_t)t * gridDim.x;
                sp_row_flushing<InT, OutT, kScale>(A + r * lda, r, n, vec, hs, seed, hashed, b, blocks, emax,
                                                   col_scale, At, ldat, scales, lds, plane_elems, sp_smem);
            }
        }
    } else {
        for (int64_t r = blockIdx.x; r < m; r += gridDim.x)
            sp_row_flushing<InT, OutT, kScale>(A + r * lda, r, n, vec, hs, seed, hashed, b, blocks, emax,
                                               col_scale, At, ldat, scales, lds, plane_elems, sp_smem);
    }
}

// Entries the buffer holds beside kb accumulators and the bucket tables (multiple of 32).
int sparse_entry_capacity(int64_t kb, int64_t b) {
    const int64_t avail = (int64_t)kSmemLimit - 4 * kb - (int64_t)sp_fixed_bytes((int)b) - 64;
    if (avail <= 0) return 0;
    const int64_t e = avail / kEntryBytes / 32 * 32;
    return (int)(e < kSpThreads * kSpPerThread ? e : kSpThreads * kSpPerThread);
}

int sp_num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

template <typename InT, typename OutT>
os_status launch_sparse_t(const InT *A, int64_t lda, int64_t m, int64_t n, const Plan *p, const BlockList &blocks,
                          const float *col_scale, void *At, int64_t ldat, float *scales, int64_t lds,
                          int64_t plane_elems, cudaStream_t st) {
    const int kb = blocks.count * p->b;
    const int emax = sparse_entry_capacity(kb, p->b);
    if (emax < kMinEntries) return OS_ERR_UNSUPPORTED;
    const size_t smem0 = sizeof(float) * (size_t)kb + (size_t)kEntryBytes * emax + sp_fixed_bytes(p->b);
    const bool vec = aligned16(A) && (lda * (int64_t)sizeof(InT)) % 16 == 0;
    const int64_t grid = m < sp_num_sms() ? m : sp_num_sms();
    // one-pass rows: per warp a region of cw entries (entry numbers fit 16 bits)
    int cw = 0;
    if (p->b <= 4 * kSpThreads) {
        const int64_t avail = (int64_t)kSmemLimit - (int64_t)sp1_fixed_bytes(p->b) - 64;
        const int64_t c = avail / (32 * kSp1EntryBytes);
        cw = (int)(c < 2047 ? c : 2047);
        if (cw < 32) cw = 0;
    }
    if (cw > 0) {
        const size_t smem1 = sp1_fixed_bytes(p->b) + (size_t)kSp1EntryBytes * 32 * cw + 64;
        auto k1 = col_scale ? sketch_left_onepass_kernel<InT, OutT, true>
                            : sketch_left_onepass_kernel<InT, OutT, false>;
        OSK_CUDA_TRY(cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1));
        k1<<<(unsigned)grid, kSpThreads, smem1, st>>>(A, lda, m, n, vec, p->hs, p->seed, p->hashed != 0, p->b,
                                                      blocks, cw, col_scale, (OutT *)At, ldat, scales, lds,
                                                      plane_elems);
        OSK_TRY(check_launch());
    }
    auto k = cw > 0 ? (col_scale ? sketch_left_sparse_kernel<InT, OutT, true, true>
                                 : sketch_left_sparse_kernel<InT, OutT, false, true>)
                    : (col_scale ? sketch_left_sparse_kernel<InT, OutT, true, false>
                                 : sketch_left_sparse_kernel<InT, OutT, false, false>);
    OSK_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem0));
    k<<<(unsigned)grid, kSpThreads, smem0, st>>>(A, lda, m, n, vec, p->hs, p->seed, p->hashed != 0, p->b, blocks,
                                                 emax, col_scale, (OutT *)At, ldat, scales, lds, plane_elems);
    return check_launch();
}

template <typename InT>
os_status launch_sparse(const InT *A, int64_t lda, int64_t m, const Plan *p, const BlockList &blocks,
                        const float *col_scale, void *At, os_dtype out_t, int64_t ldat, float *scales,
                        cudaStream_t st) {
    const int64_t lds = fp8_scale_ld(m);
    switch (out_t) {
        case OS_F32:
            return launch_sparse_t<InT, float>(A, lda, m, p->n, p, blocks, col_scale, At, ldat, nullptr, lds, 0, st);
        case OS_BF16:
            return launch_sparse_t<InT, __nv_bfloat16>(A, lda, m, p->n, p, blocks, col_scale, At, ldat, nullptr, lds,
                                                       0, st);
        case OS_FP8E4M3:
            return launch_sparse_t<InT, __nv_fp8_e4m3>(A, lda, m, p->n, p, blocks, col_scale, At, ldat, scales, lds,
                                                       0, st);
        case OS_TF32X2:
            return launch_sparse_t<InT, Tf32Pair>(A, lda, m, p->n, p, blocks, col_scale, At, ldat, nullptr, lds,
                                                  m * ldat, st);
    }
    return OS_ERR_DTYPE;
}

}  // namespace

// Whether the sparse-row left sketch can hold the accumulators of these blocks.
bool sketch_left_sparse_fits(const Plan *p, uint64_t block_mask) {
    const BlockList blocks = mask_to_list(block_mask ? block_mask : ~0ull, p->P);
    const int64_t kb = (int64_t)blocks.count * p->b;
    return kb <= kSparseMaxBuckets && p->b <= kSparseMaxBuckets &&
           sparse_entry_capacity(kb, p->b) >= kMinEntries;
}

os_status sketch_left_sparse_impl(const Plan *p, const void *A, os_dtype a_t, int64_t m, int64_t lda, void *At,
                                  os_dtype out_t, int64_t ldat, float *scales, const float *col_scale,
                                  uint64_t block_mask, cudaStream_t st) {
    if (!p || m < 0) return OS_ERR_INVALID_ARG;
    if (block_mask) OSK_TRY(check_mask(block_mask, p->P));
    if (a_t != OS_F32 && a_t != OS_BF16) return OS_ERR_DTYPE;
    if (out_t != OS_F32 && out_t != OS_BF16 && out_t != OS_FP8E4M3 && out_t != OS_TF32X2) return OS_ERR_DTYPE;
    const int64_t z = (int64_t)p->P * p->b;
    if (lda < p->n || ldat < z || (ldat * (int64_t)dtype_size(out_t)) % 16 != 0) return OS_ERR_INVALID_ARG;
    if (out_t == OS_FP8E4M3 && p->b % 128 != 0) return OS_ERR_UNSUPPORTED;
    if (!sketch_left_sparse_fits(p, block_mask)) return OS_ERR_UNSUPPORTED;
    if (m == 0) return OS_OK;   // an empty output
    if (!A || !At || !aligned16(At)) return OS_ERR_INVALID_ARG;
    if (out_t == OS_FP8E4M3 && !scales) return OS_ERR_INVALID_ARG;
    const BlockList blocks = mask_to_list(block_mask ? block_mask : ~0ull, p->P);
    if (a_t == OS_F32)
        return launch_sparse<float>((const float *)A, lda, m, p, blocks, col_scale, At, out_t, ldat, scales, st);
    return launch_sparse<__nv_bfloat16>((const __nv_bfloat16 *)A, lda, m, p, blocks, col_scale, At, out_t, ldat,
                                        scales, st);
}

}  // namespace osk

using namespace osk;

extern "C" os_status oversketch_sketch_left_sparse(oversketch_plan_t plan, const void *A, os_dtype a_t, int64_t m,
                                                   int64_t lda, void *At, os_dtype out_t, int64_t ldat,
                                                   float *scales, const float *col_scale, uint64_t block_mask,
                                                   void *stream) {
    OSK_NVTX("sketch_left_sparse");
    return sketch_left_sparse_impl(reinterpret_cast<const Plan *>(plan), A, a_t, m, lda, At, out_t, ldat, scales,
                                   col_scale, block_mask, as_stream(stream));
}
