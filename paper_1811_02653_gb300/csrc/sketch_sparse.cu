// Left sketch of a sparse operand stored dense (Alg. 4 step 3 / Alg. 5 over the
// nonzeros only: the paper prices sketching at O(nnz(A) (N+e)), Sec. 4).
//
//   At[r, j*b + c] = sum_{i : A[r,i] != 0, h_j(i) = c} sigma_j(i) * s_i * A[r, i]
//
// The dense gather path reads every element k times from L2 (once per kept
// block) and, when a 128-wide strip of the sketched dimension no longer fits in
// L2 (n = 2^20: 512 MB per strip), from DRAM.  For a row with few nonzeros the
// whole row's accumulators (k*b FP32 values) fit in shared memory instead, so
// one CTA per row reads the row once, coalesced, and routes only its nonzeros:
//
//   1. compaction: the row streams through registers in chunks of 16 elements
//      per thread (an L2 prefetch runs a few chunks ahead); a block-wide scan
//      appends the nonzeros (index, value) in ascending index order to an
//      entry buffer in shared memory;
//   2. flush (buffer full or row done): values take their scale s_i; then for
//      every kept block j the entries are counted per bucket h_j(i) (integer
//      shared-memory atomics), the counts are scanned into bucket offsets, the
//      entries are scattered into their buckets, and each thread adds the
//      members of its own buckets to their accumulators in ascending index
//      order.  No float atomics; every bucket sums its members in a fixed
//      order (ascending index), so results are bitwise reproducible;
//   3. the row's accumulators are written out in the output dtype (BF16 RNE,
//      FP8 with the per-128-column UE8M0 scale, FP32, or TF32 hi/lo planes).
//
// Any density is handled (a dense row just flushes often, slowly); the caller
// picks this path for sparse operands.  Shared memory holds the k*b
// accumulators and two b-entry bucket tables: 4*k*b + 8*b bytes plus an
// entry buffer of at least 1024 entries must fit (k*b <= kSparseMaxBuckets).
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

// One CTA per row (persistent over rows); see the file comment.
template <typename InT, typename OutT, bool kScale>
__global__ void __launch_bounds__(kSpThreads, 1)
sketch_left_sparse_kernel(const InT *__restrict__ A, int64_t lda, int64_t m, int64_t n, bool vec,
                          const uint32_t *__restrict__ hs, uint64_t seed, bool hashed, int32_t b,
                          BlockList blocks, int emax,
                          const float *__restrict__ col_scale, OutT *__restrict__ At, int64_t ldat,
                          float *__restrict__ scales, int64_t lds, int64_t plane_elems) {
    extern __shared__ float4 sp_smem[];
    const int kb = blocks.count * b;
    const SpSmem s = sp_layout(sp_smem, kb, b, emax);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t chunk_bytes = (int64_t)kSpChunk * sizeof(InT);

    for (int64_t r = blockIdx.x; r < m; r += gridDim.x) {
        for (int q = tid; q < kb; q += kSpThreads) s.state[q] = 0.f;
        const InT *row = A + r * lda;
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
        __syncthreads();   // the accumulators are cleared for the next row
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
    const size_t smem = sizeof(float) * (size_t)kb + (size_t)kEntryBytes * emax + sp_fixed_bytes(p->b);
    const bool vec = aligned16(A) && (lda * (int64_t)sizeof(InT)) % 16 == 0;
    auto k = col_scale ? sketch_left_sparse_kernel<InT, OutT, true> : sketch_left_sparse_kernel<InT, OutT, false>;
    OSK_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t grid = m < sp_num_sms() ? m : sp_num_sms();
    k<<<(unsigned)grid, kSpThreads, smem, st>>>(A, lda, m, n, vec, p->hs, p->seed, p->hashed != 0, p->b, blocks,
                                                emax, col_scale,
                                                (OutT *)At, ldat, scales, lds, plane_elems);
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
