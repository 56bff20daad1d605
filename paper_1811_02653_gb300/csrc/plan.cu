// Plan construction: the sketch S of Eq. 3 as device tables.
//
// Alg. 4 steps 1-2 give every index i of the sketched dimension a random sign
// and a uniform bucket, independently for each of the P = N + e blocks; step 3
// ("add the columns mapped to the same integer") needs, per block, the list of
// indices of every bucket.  Here the random draws come from splitmix64 (the
// published generator of Steele, Lea and Flood, used as a counter-based hash),
// and the bucket lists are built by a deterministic stable counting sort:
//   1. plan_hash_kernel        -- hs[j][i] = h_j(i) | sign bit
//   2. chunk_count_kernel      -- per (block, chunk of 1024 indices) bucket counts,
//                                 one warp per chunk (lanes with equal buckets
//                                 counted together; no atomics)
//   3. bucket_total_kernel     -- per (block, bucket): exclusive prefix over chunks
//   4. row_scan_kernel         -- per block: exclusive prefix over buckets -> offs
//   5. chunk_scatter_kernel    -- per (block, chunk): one warp, stable scatter in
//                                 ascending index order
// Plan creation is not on the timed path; every step is deterministic.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace osk {

namespace {

__global__ void plan_hash_kernel(int64_t n, int32_t b, uint64_t seed, uint32_t *__restrict__ hs) {
    const int j = blockIdx.y;
    const uint64_t key = block_key(seed, j);
    uint32_t *row = hs + (int64_t)j * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        row[i] = hash_code(key, i, b);
}

// A chunk of the sketched dimension per warp: the warp walks it 32 indices at a
// time; lanes whose indices share a bucket find each other (__match_any_sync),
// and the lowest of them updates that bucket's counter for all of them.  One
// warp owns a counter row, so every update is a plain read-modify-write in a
// fixed order: no atomics, the same result on every run.
constexpr int kChunk = 1024;   // indices per warp

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// cnt[(j*nchunks + ch)*b + c] = #{i in chunk ch : h_j(i) = c}
__global__ void __launch_bounds__(256) chunk_count_kernel(const uint32_t *__restrict__ hs, int64_t n, int32_t b,
                                                          int P, int nchunks, int64_t chunk,
                                                          uint32_t *__restrict__ cnt) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // warp = (block, chunk)
    const int lane = threadIdx.x & 31;
    if (t >= (int64_t)P * nchunks) return;
    const int j = (int)(t / nchunks), ch = (int)(t % nchunks);
    uint32_t *row = cnt + t * b;
    const uint32_t *hrow = hs + (int64_t)j * n;
    const int64_t i0 = ch * chunk, i1 = min(n, i0 + chunk);
    for (int64_t base = i0; base < i1; base += 32) {
        const int64_t i = base + lane;
        const bool valid = i < i1;
        const uint32_t key = valid ? (__ldg(hrow + i) & kIndexMask) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        if (valid && lane == __ffs(peers) - 1) row[key] += (uint32_t)__popc(peers);
        __syncwarp();
    }
}

// In place: cnt[j][ch][c] <- sum_{ch' < ch} cnt[j][ch'][c]; tot[j][c] = total.
__global__ void bucket_total_kernel(uint32_t *__restrict__ cnt, int32_t b, int P, int nchunks,
                                    uint32_t *__restrict__ tot) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)P * b) return;
    const int j = (int)(t / b), c = (int)(t % b);
    uint32_t run = 0;
    for (int ch = 0; ch < nchunks; ++ch) {
        uint32_t *p = cnt + ((int64_t)j * nchunks + ch) * b + c;
        const uint32_t v = *p;
        *p = run;
        run += v;
    }
    tot[t] = run;
}

// Exclusive prefix sums of one row of b values per CTA (block j), 1024 threads:
// each thread sums a contiguous run of buckets, the CTA scans the run totals,
// and each thread writes its run's prefixes; out[j][b] = the row total.
//   mode 0: values tot[j][c]                            -> offs
//   mode 1: values roundup4(offs[j][c+1] - offs[j][c])  -> poffs (padded lists)
__global__ void __launch_bounds__(1024) row_scan_kernel(const uint32_t *__restrict__ src, int32_t b, int mode,
                                                        uint32_t *__restrict__ out) {
    __shared__ uint32_t warp_tot[32];
    const int j = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (b + 1023) / 1024;
    const int c0 = min(b, tid * per), c1 = min(b, c0 + per);
    auto value = [&](int c) -> uint32_t {
        if (mode == 0) return src[(int64_t)j * b + c];
        const uint32_t *o = src + (int64_t)j * (b + 1);
        return (o[c + 1] - o[c] + 3u) & ~3u;
    };
    uint32_t mine = 0;
    for (int c = c0; c < c1; ++c) mine += value(c);
    // inclusive scan of the per-thread totals: within warps, then across warps
    uint32_t x = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    uint32_t run = x - mine + (warp > 0 ? warp_tot[warp - 1] : 0u);   // exclusive prefix of this run
    uint32_t *orow = out + (int64_t)j * (b + 1);
    for (int c = c0; c < c1; ++c) {
        orow[c] = run;
        run += value(c);
    }
    if (tid == 1023) orow[b] = warp_tot[31];
}

// Stable scatter: a warp walks its chunk in ascending order, 32 indices at a
// time; an index's position is its bucket's start, plus the bucket's cursor of
// this chunk (indices of earlier chunks and earlier steps), plus the number of
// lanes of this step with the same bucket and a lower index.
__global__ void __launch_bounds__(256) chunk_scatter_kernel(const uint32_t *__restrict__ hs, int64_t n, int32_t b,
                                                            int P, int nchunks, int64_t chunk,
                                                            uint32_t *__restrict__ cursor,
                                                            const uint32_t *__restrict__ offs,
                                                            uint32_t *__restrict__ perm) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= (int64_t)P * nchunks) return;
    const int j = (int)(t / nchunks), ch = (int)(t % nchunks);
    uint32_t *cur = cursor + t * b;
    const uint32_t *hrow = hs + (int64_t)j * n;
    const uint32_t *orow = offs + (int64_t)j * (b + 1);
    uint32_t *prow = perm + (int64_t)j * n;
    const int64_t i0 = ch * chunk, i1 = min(n, i0 + chunk);
    for (int64_t base = i0; base < i1; base += 32) {
        const int64_t i = base + lane;
        const bool valid = i < i1;
        const uint32_t v = valid ? __ldg(hrow + i) : 0xffffffffu;
        const uint32_t key = valid ? (v & kIndexMask) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(peers) - 1;
        uint32_t start = 0;
        if (valid && lane == leader) start = cur[key];
        start = __shfl_sync(0xffffffffu, start, leader);
        if (valid) prow[__ldg(orow + key) + start + (uint32_t)__popc(peers & lanemask_lt())] = (uint32_t)i | (v & kSignBit);
        __syncwarp();
        if (valid && lane == leader) cur[key] = start + (uint32_t)__popc(peers);
        __syncwarp();
    }
}

__global__ void padded_fill_kernel(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ offs,
                                   const uint32_t *__restrict__ poffs, int64_t n, int32_t b, int P,
                                   int64_t pstride, uint32_t *__restrict__ pperm) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)P * b) return;
    const int j = (int)(t / b), c = (int)(t % b);
    const uint32_t *o = offs + (int64_t)j * (b + 1);
    const uint32_t *po = poffs + (int64_t)j * (b + 1);
    const uint32_t cnt = o[c + 1] - o[c];
    const uint32_t pcnt = po[c + 1] - po[c];
    const uint32_t *src = perm + (int64_t)j * n + o[c];
    uint32_t *dst = pperm + (int64_t)j * pstride + po[c];
    for (uint32_t u = 0; u < pcnt; ++u) dst[u] = u < cnt ? src[u] : kPadEntry;
}

os_status check_params(int64_t n, int32_t b, int32_t N, int32_t e, oversketch_plan_t *out) {
    if (!out) return OS_ERR_INVALID_ARG;
    if (n < 1 || b < 1 || N < 1 || e < 0) return OS_ERR_INVALID_ARG;
    if (N + e > 64) return OS_ERR_UNSUPPORTED;
    if (n >= (int64_t(1) << 31)) return OS_ERR_UNSUPPORTED;
    if ((int64_t)(N + e) * b >= (int64_t(1) << 31)) return OS_ERR_UNSUPPORTED;
    return OS_OK;
}

void free_plan(Plan *p) {
    if (!p) return;
    if (p->hs) cudaFree(p->hs);   // one allocation holds every table
    delete p;
}

// Steps 2-5 on an existing hs table.  The counters are stream-ordered
// allocations, so freeing them does not synchronise the device.
os_status build_csr(Plan *p, cudaStream_t st) {
    const int P = p->P;
    const int64_t n = p->n;
    const int32_t b = p->b;
    // chunks of kChunk indices (one warp each), with at most 2^24 counters in total
    int64_t nchunks = (n + kChunk - 1) / kChunk;
    const int64_t cap = (int64_t(1) << 24) / ((int64_t)P * b);
    if (nchunks > cap) nchunks = cap < 1 ? 1 : cap;
    const int64_t chunk = (n + nchunks - 1) / nchunks;
    nchunks = (n + chunk - 1) / chunk;

    uint32_t *cnt = nullptr, *tot = nullptr;
    const size_t cnt_bytes = sizeof(uint32_t) * (size_t)P * nchunks * b;
    if (cudaMallocAsync(&cnt, cnt_bytes, st) != cudaSuccess) return set_cuda_error(cudaGetLastError());
    if (cudaMallocAsync(&tot, sizeof(uint32_t) * (size_t)P * b, st) != cudaSuccess) {
        cudaFreeAsync(cnt, st);
        return set_cuda_error(cudaGetLastError());
    }
    os_status s = OS_OK;
    do {
        if (cudaMemsetAsync(cnt, 0, cnt_bytes, st) != cudaSuccess) { s = OS_ERR_CUDA; break; }
        const int64_t threads = (int64_t)P * nchunks * 32;
        chunk_count_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(p->hs, n, b, P, (int)nchunks, chunk,
                                                                               cnt);
        if ((s = check_launch()) != OS_OK) break;
        bucket_total_kernel<<<(unsigned)(((int64_t)P * b + 255) / 256), 256, 0, st>>>(
            cnt, b, P, (int)nchunks, tot);
        if ((s = check_launch()) != OS_OK) break;
        row_scan_kernel<<<P, 1024, 0, st>>>(tot, b, 0, p->offs);
        if ((s = check_launch()) != OS_OK) break;
        chunk_scatter_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(p->hs, n, b, P, (int)nchunks, chunk,
                                                                                 cnt, p->offs, p->perm);
        if ((s = check_launch()) != OS_OK) break;
        row_scan_kernel<<<P, 1024, 0, st>>>(p->offs, b, 1, p->poffs);
        if ((s = check_launch()) != OS_OK) break;
        padded_fill_kernel<<<(unsigned)(((int64_t)P * b + 127) / 128), 128, 0, st>>>(
            p->perm, p->offs, p->poffs, n, b, P, p->pstride, p->pperm);
        if ((s = check_launch()) != OS_OK) break;
    } while (0);
    cudaFreeAsync(cnt, st);
    cudaFreeAsync(tot, st);
    if (s == OS_OK && cudaStreamSynchronize(st) != cudaSuccess) s = set_cuda_error(cudaGetLastError());
    return s;
}

os_status alloc_plan(int64_t n, int32_t b, int32_t N, int32_t e, uint64_t seed, Plan **out) {
    Plan *p = new Plan();
    p->n = n;
    p->b = b;
    p->N = N;
    p->e = e;
    p->P = N + e;
    p->seed = seed;
    p->hashed = 0;
    p->hs = p->perm = p->offs = p->pperm = p->poffs = nullptr;
    p->pstride = (n + 3 * (int64_t)b + 3) / 4 * 4;
    cudaGetDevice(&p->device);
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t tab = al(sizeof(uint32_t) * (size_t)p->P * n);
    const size_t otab = al(sizeof(uint32_t) * (size_t)p->P * (b + 1));
    const size_t ptab = al(sizeof(uint32_t) * (size_t)p->P * p->pstride);
    char *base = nullptr;
    if (cudaMalloc(&base, 2 * tab + 2 * otab + ptab) != cudaSuccess) {
        cudaGetLastError();
        free_plan(p);
        return OS_ERR_OOM;
    }
    p->hs = reinterpret_cast<uint32_t *>(base);
    p->perm = reinterpret_cast<uint32_t *>(base + tab);
    p->offs = reinterpret_cast<uint32_t *>(base + 2 * tab);
    p->poffs = reinterpret_cast<uint32_t *>(base + 2 * tab + otab);
    p->pperm = reinterpret_cast<uint32_t *>(base + 2 * tab + 2 * otab);
    *out = p;
    return OS_OK;
}

}  // namespace

}  // namespace osk

using namespace osk;

extern "C" os_status oversketch_plan(int64_t n, int32_t b, int32_t N, int32_t e, uint64_t seed,
                                     void *stream, oversketch_plan_t *out) {
    OSK_NVTX("oversketch_plan");
    OSK_TRY(check_params(n, b, N, e, out));
    Plan *p = nullptr;
    OSK_TRY(alloc_plan(n, b, N, e, seed, &p));
    cudaStream_t st = as_stream(stream);
    const int64_t blocks_x = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    plan_hash_kernel<<<dim3((unsigned)blocks_x, (unsigned)p->P), 256, 0, st>>>(n, b, seed, p->hs);
    os_status s = check_launch();
    if (s == OS_OK) s = build_csr(p, st);
    p->hashed = 1;
    if (s != OS_OK) {
        free_plan(p);
        return s;
    }
    *out = reinterpret_cast<oversketch_plan_t>(p);
    return OS_OK;
}

extern "C" os_status oversketch_plan_from_tables(int64_t n, int32_t b, int32_t N, int32_t e,
                                                 const uint32_t *h_host, const int8_t *sigma_host,
                                                 void *stream, oversketch_plan_t *out) {
    OSK_NVTX("oversketch_plan_from_tables");
    OSK_TRY(check_params(n, b, N, e, out));
    if (!h_host || !sigma_host) return OS_ERR_INVALID_ARG;
    const int P = N + e;
    std::vector<uint32_t> packed((size_t)P * n);
    for (size_t t = 0; t < packed.size(); ++t) {
        if ((int64_t)h_host[t] >= b || (sigma_host[t] != 1 && sigma_host[t] != -1))
            return OS_ERR_INVALID_ARG;
        packed[t] = h_host[t] | (sigma_host[t] < 0 ? kSignBit : 0u);
    }
    Plan *p = nullptr;
    OSK_TRY(alloc_plan(n, b, N, e, 0, &p));
    cudaStream_t st = as_stream(stream);
    os_status s = OS_OK;
    if (cudaMemcpyAsync(p->hs, packed.data(), packed.size() * sizeof(uint32_t),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
        s = set_cuda_error(cudaGetLastError());
    if (s == OS_OK) s = build_csr(p, st);
    if (s != OS_OK) {
        free_plan(p);
        return s;
    }
    *out = reinterpret_cast<oversketch_plan_t>(p);
    return OS_OK;
}

extern "C" os_status oversketch_plan_get_tables(oversketch_plan_t plan, uint32_t *h_host,
                                                int8_t *sigma_host, uint32_t *perm_host,
                                                uint32_t *offs_host) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !h_host || !sigma_host) return OS_ERR_INVALID_ARG;
    const size_t cnt = (size_t)p->P * p->n;
    std::vector<uint32_t> packed(cnt);
    OSK_CUDA_TRY(cudaMemcpy(packed.data(), p->hs, cnt * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    for (size_t t = 0; t < cnt; ++t) {
        h_host[t] = packed[t] & kIndexMask;
        sigma_host[t] = (packed[t] & kSignBit) ? (int8_t)-1 : (int8_t)1;
    }
    if (perm_host)
        OSK_CUDA_TRY(cudaMemcpy(perm_host, p->perm, cnt * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (offs_host)
        OSK_CUDA_TRY(cudaMemcpy(offs_host, p->offs, sizeof(uint32_t) * (size_t)p->P * (p->b + 1),
                                cudaMemcpyDeviceToHost));
    return OS_OK;
}

extern "C" os_status oversketch_plan_info(oversketch_plan_t plan, int64_t *n, int32_t *b,
                                          int32_t *N, int32_t *e) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p) return OS_ERR_INVALID_ARG;
    if (n) *n = p->n;
    if (b) *b = p->b;
    if (N) *N = p->N;
    if (e) *e = p->e;
    return OS_OK;
}

extern "C" os_status oversketch_plan_destroy(oversketch_plan_t plan) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p) return OS_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    free_plan(p);
    return OS_OK;
}
