// Many independent OverSketch products in one CUDA graph.
//
// Alg. 3 treats the blocks of a product as independent jobs; a batch of
// products multiplies that independence.  A batch object fixes the products
// (shapes, pointers, plans, masks) once, the way a CUDA graph fixes its
// nodes, and every run replays one instantiated graph:
//
//   * sketches: the products are spread over W parallel branches of the
//     graph.  A branch sketches its products one after another (left: pack +
//     gather, right: gather, kept blocks only, BF16 out) and owns one packing
//     workspace slot, so W bounds both the concurrency and the workspace.
//     Small products of different branches overlap on the GPU.
//   * GEMM: after all branches, ONE persistent tcgen05 launch runs every tile
//     of every product; tiles are ordered by descending K (longest work first)
//     and dealt round-robin to the resident CTAs.
//
// Creation can time a few configurations (branch count W, GEMM tile width)
// and keep the fastest graph.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "group.cuh"

namespace osk {

os_status sketch_left_impl(const Plan *p, const void *A, os_dtype a_t, int64_t m, int64_t lda, void *At,
                           os_dtype out_t, int64_t ldat, float *scales, const float *col_scale,
                           uint64_t block_mask, void *ws, size_t ws_bytes, cudaStream_t st,
                           const uint64_t *dmask = nullptr);
os_status sketch_right_impl(const Plan *p, const void *B, os_dtype b_t, int64_t l, int64_t ldb, void *BtT,
                            os_dtype out_t, int64_t ldbt, float *scales, uint64_t block_mask, void *ws,
                            size_t ws_bytes, cudaStream_t st, const float *row_scale = nullptr,
                            const uint64_t *dmask = nullptr);
size_t sketch_workspace_bytes(const Plan *p, int64_t F, os_dtype in_t);

namespace {

constexpr int kMaxBranches = 16;
constexpr size_t kDefaultWorkspaceLimit = size_t(16) << 30;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Batch {
    int device = 0;
    std::vector<os_problem> probs;
    os_dtype a_t = OS_F32, b_t = OS_F32;
    // sketched operands (BF16, full sketch width; only kept blocks are written)
    void *operands = nullptr;
    size_t operand_bytes = 0;
    std::vector<void *> at, bt;
    std::vector<int64_t> z;
    // packing workspace: branches x slot
    void *workspace = nullptr;
    size_t slot_bytes = 0;
    int max_branches = 1;
    // grouped GEMM descriptors, one array per tile width, LPT order
    GroupProblem *group[2] = {nullptr, nullptr};
    int32_t total_tiles[2] = {0, 0};
    // the chosen graph
    cudaGraphExec_t exec = nullptr;
    int branches = 1;
    GroupTile tile = kGroupBN256;
    int launches = 0;
    float tuned_ms = 0.f;
};

os_status free_batch(Batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto &g : b->group)
        if (g) cudaFree(g);
    if (b->workspace) cudaFree(b->workspace);
    if (b->operands) cudaFree(b->operands);
    delete b;
    return OS_OK;
}

// Products in longest-K-first order (ties: larger output first).
std::vector<int> lpt_order(const Batch &B) {
    std::vector<int> ord(B.probs.size());
    std::iota(ord.begin(), ord.end(), 0);
    auto K = [&](int i) {
        const Plan *p = reinterpret_cast<const Plan *>(B.probs[i].plan);
        return (int64_t)__builtin_popcountll(B.probs[i].mask) * p->b;
    };
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
        if (K(x) != K(y)) return K(x) > K(y);
        return B.probs[x].m * B.probs[x].l > B.probs[y].m * B.probs[y].l;
    });
    return ord;
}

os_status build_group(Batch &B, GroupTile tile) {
    const int count = (int)B.probs.size();
    std::vector<GroupProblem> h(count);
    int32_t tiles = 0;
    const std::vector<int> ord = lpt_order(B);
    for (int q = 0; q < count; ++q) {
        const int i = ord[q];
        const os_problem &pr = B.probs[i];
        const Plan *p = reinterpret_cast<const Plan *>(pr.plan);
        const int k = __builtin_popcountll(pr.mask);
        OSK_TRY(group_problem_bf16(&h[q], tile, B.at[i], B.z[i], B.bt[i], B.z[i], pr.m, pr.l, B.z[i], p->b, p->P,
                                   pr.mask, nullptr, 1.f / (float)k, 0.f, pr.C, pr.ldc));
        h[q].tile_begin = tiles;
        const int64_t t = (int64_t)h[q].tiles_m * h[q].tiles_n;
        if ((int64_t)tiles + t >= (int64_t(1) << 31)) return OS_ERR_UNSUPPORTED;
        tiles += (int32_t)t;
    }
    OSK_CUDA_TRY(cudaMalloc(&B.group[tile], sizeof(GroupProblem) * count));
    OSK_CUDA_TRY(cudaMemcpy(B.group[tile], h.data(), sizeof(GroupProblem) * count, cudaMemcpyHostToDevice));
    B.total_tiles[tile] = tiles;
    return OS_OK;
}

// Record one run into `cap` (a capturing stream): W sketch branches, then the grouped GEMM.
os_status record_run(Batch &B, int W, GroupTile tile, cudaStream_t cap, std::vector<cudaStream_t> &streams,
                     std::vector<cudaEvent_t> &events) {
    const int count = (int)B.probs.size();
    OSK_CUDA_TRY(cudaEventRecord(events[0], cap));
    // branch assignment: greedy, heaviest sketch first (work ~ (m + l) n)
    std::vector<int> ord(count);
    std::iota(ord.begin(), ord.end(), 0);
    auto work = [&](int i) { return (B.probs[i].m + B.probs[i].l) * B.probs[i].n; };
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return work(x) > work(y); });
    std::vector<int64_t> load(W, 0);
    std::vector<std::vector<int>> branch(W);
    for (int i : ord) {
        const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        branch[w].push_back(i);
        load[w] += work(i);
    }
    for (int w = 0; w < W; ++w) {
        cudaStream_t s = streams[w];
        OSK_CUDA_TRY(cudaStreamWaitEvent(s, events[0], 0));
        void *ws = (char *)B.workspace + (size_t)w * B.slot_bytes;
        for (int i : branch[w]) {
            const os_problem &pr = B.probs[i];
            const Plan *p = reinterpret_cast<const Plan *>(pr.plan);
            OSK_TRY(sketch_left_impl(p, pr.A, B.a_t, pr.m, pr.lda, B.at[i], OS_BF16, B.z[i], nullptr, nullptr,
                                     pr.mask, ws, B.slot_bytes, s));
            OSK_TRY(sketch_right_impl(p, pr.B, B.b_t, pr.l, pr.ldb, B.bt[i], OS_BF16, B.z[i], nullptr, pr.mask,
                                      ws, B.slot_bytes, s));
        }
        OSK_CUDA_TRY(cudaEventRecord(events[1 + w], s));
        OSK_CUDA_TRY(cudaStreamWaitEvent(cap, events[1 + w], 0));
    }
    return gemm_grouped_bf16(B.group[tile], count, B.total_tiles[tile], tile, cap);
}

os_status instantiate(Batch &B, int W, GroupTile tile, cudaGraphExec_t *exec, int *launches) {
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> streams(W, nullptr);
    std::vector<cudaEvent_t> events(1 + W, nullptr);
    os_status st = OS_OK;
    cudaGraph_t graph = nullptr;
    auto fail = [&](os_status s) {
        if (st == OS_OK) st = s;
    };
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return OS_ERR_CUDA;
    for (auto &s : streams)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) fail(OS_ERR_CUDA);
    for (auto &e : events)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) fail(OS_ERR_CUDA);
    if (st == OS_OK) {
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            fail(set_cuda_error(e));
        } else {
            fail(record_run(B, W, tile, cap, streams, events));
            // always end the capture, also after a failed recording
            e = cudaStreamEndCapture(cap, &graph);
            if (e != cudaSuccess) fail(set_cuda_error(e));
        }
    }
    if (st == OS_OK) {
        cudaError_t e = cudaGraphInstantiate(exec, graph, 0);
        if (e != cudaSuccess) fail(set_cuda_error(e));
    }
    if (st == OS_OK) {
        size_t n = 0;
        cudaGraphGetNodes(graph, nullptr, &n);
        std::vector<cudaGraphNode_t> nodes(n);
        cudaGraphGetNodes(graph, nodes.data(), &n);
        int k = 0;
        for (auto nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
        }
        *launches = k;
    }
    if (graph) cudaGraphDestroy(graph);
    for (auto e : events)
        if (e) cudaEventDestroy(e);
    for (auto s : streams)
        if (s) cudaStreamDestroy(s);
    cudaStreamDestroy(cap);
    return st;
}

// Median of `reps` timed replays (after one warm-up replay).
os_status time_graph(cudaGraphExec_t exec, cudaStream_t st, int reps, float *ms) {
    cudaEvent_t e0, e1;
    OSK_CUDA_TRY(cudaEventCreate(&e0));
    OSK_CUDA_TRY(cudaEventCreate(&e1));
    std::vector<float> t;
    os_status s = OS_OK;
    if (cudaGraphLaunch(exec, st) != cudaSuccess) s = OS_ERR_CUDA;
    for (int r = 0; s == OS_OK && r < reps; ++r) {
        cudaEventRecord(e0, st);
        if (cudaGraphLaunch(exec, st) != cudaSuccess) s = OS_ERR_CUDA;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) s = OS_ERR_CUDA;
        float x = 0.f;
        cudaEventElapsedTime(&x, e0, e1);
        t.push_back(x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != OS_OK) return set_cuda_error(cudaGetLastError());
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return OS_OK;
}

os_status create(const os_problem *problems, int32_t count, os_dtype a_t, os_dtype b_t, os_dtype g_t,
                 size_t ws_limit, int32_t tune, cudaStream_t st, Batch *B) {
    if (!problems || count <= 0 || count > kMaxGroup) return OS_ERR_INVALID_ARG;
    if ((a_t != OS_F32 && a_t != OS_BF16) || (b_t != OS_F32 && b_t != OS_BF16)) return OS_ERR_DTYPE;
    if (g_t != OS_BF16) return OS_ERR_DTYPE;
    OSK_CUDA_TRY(cudaGetDevice(&B->device));
    B->a_t = a_t;
    B->b_t = b_t;
    B->probs.assign(problems, problems + count);
    // validate and size
    size_t slot = 256, total = 0;
    B->z.resize(count);
    for (int i = 0; i < count; ++i) {
        const os_problem &pr = problems[i];
        const Plan *p = reinterpret_cast<const Plan *>(pr.plan);
        if (!p || !pr.A || !pr.B || !pr.C) return OS_ERR_INVALID_ARG;
        if (p->device != B->device) return OS_ERR_INVALID_ARG;
        if (pr.m <= 0 || pr.l <= 0 || pr.n != p->n) return OS_ERR_INVALID_ARG;
        if (pr.lda < pr.n || pr.ldb < pr.l || pr.ldc < pr.l) return OS_ERR_INVALID_ARG;
        OSK_TRY(check_mask(pr.mask, p->P));
        if (p->b % 64 != 0) return OS_ERR_UNSUPPORTED;   // BF16 GEMM K tile
        B->z[i] = (int64_t)p->P * p->b;
        total += align256((size_t)pr.m * B->z[i] * 2) + align256((size_t)pr.l * B->z[i] * 2);
        slot = std::max(slot, sketch_workspace_bytes(p, pr.m, a_t));
        slot = std::max(slot, sketch_workspace_bytes(p, pr.l, b_t));
    }
    slot = align256(slot);
    if (ws_limit == 0) ws_limit = kDefaultWorkspaceLimit;
    if (slot > ws_limit) return OS_ERR_WORKSPACE;
    B->slot_bytes = slot;
    B->max_branches = (int)std::min<size_t>(kMaxBranches, ws_limit / slot);
    B->max_branches = std::max(1, std::min(B->max_branches, count));
    // allocate
    OSK_CUDA_TRY(cudaMalloc(&B->operands, total));
    B->operand_bytes = total;
    B->at.resize(count);
    B->bt.resize(count);
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
        B->at[i] = (char *)B->operands + off;
        off += align256((size_t)problems[i].m * B->z[i] * 2);
        B->bt[i] = (char *)B->operands + off;
        off += align256((size_t)problems[i].l * B->z[i] * 2);
    }
    OSK_CUDA_TRY(cudaMalloc(&B->workspace, slot * B->max_branches));
    OSK_TRY(build_group(*B, kGroupBN256));
    OSK_TRY(build_group(*B, kGroupBN128));
    // one-time kernel attributes before any capture
    OSK_TRY(gemm_grouped_prepare());
    // candidates: (branches, tile); without tuning the first one
    std::vector<std::pair<int, GroupTile>> cand;
    // one branch by default: concurrent branches' strips compete for L2 (the tuner
    // picked one branch on the 256-product workload)
    const int wdef = 1;
    cand.push_back({wdef, kGroupBN256});
    if (tune) {
        cand.push_back({wdef, kGroupBN128});
        for (int w : {2, 4, 8})
            if (w <= B->max_branches && w != wdef) {
                cand.push_back({w, kGroupBN256});
                cand.push_back({w, kGroupBN128});
            }
    }
    float best = 0.f;
    for (size_t c = 0; c < cand.size(); ++c) {
        cudaGraphExec_t ex = nullptr;
        int launches = 0;
        OSK_TRY(instantiate(*B, cand[c].first, cand[c].second, &ex, &launches));
        float ms = 0.f;
        if (tune) {
            const os_status s = time_graph(ex, st, 3, &ms);
            if (s != OS_OK) {
                cudaGraphExecDestroy(ex);
                return s;
            }
        }
        if (!B->exec || ms < best) {
            if (B->exec) cudaGraphExecDestroy(B->exec);
            B->exec = ex;
            B->branches = cand[c].first;
            B->tile = cand[c].second;
            B->launches = launches;
            best = ms;
        } else {
            cudaGraphExecDestroy(ex);
        }
    }
    B->tuned_ms = tune ? best : 0.f;
    return OS_OK;
}

// ---------------------------------------------------------------------------
// The batched product with a caller-owned workspace and run-time masks
// (oversketch_matmul_batched).  Each call: the GEMM descriptors are written into
// the workspace by small kernels that carry them as launch parameters (so a
// captured graph holds them by value), the sketches of the products run one
// after another on the caller's stream (every block is sketched; CTAs of blocks
// that the device mask drops return at once), then one grouped tcgen05 launch
// reads each product's mask from device memory for its K list and its 1/k.
// Nothing is allocated.  (Sketching products concurrently on parallel branches
// measured slower: their strips compete for L2.)

constexpr int kDescPerChunk = 40;

struct DescChunk {
    int32_t first, count;
    GroupProblem items[kDescPerChunk];
};
static_assert(sizeof(DescChunk) <= 32000, "descriptor chunk exceeds the launch parameter space");

__global__ void __launch_bounds__(256) upload_groups_kernel(const __grid_constant__ DescChunk chunk,
                                                            GroupProblem *__restrict__ dst) {
    const int words = chunk.count * (int)(sizeof(GroupProblem) / 16);
    const uint4 *src = reinterpret_cast<const uint4 *>(chunk.items);
    uint4 *out = reinterpret_cast<uint4 *>(dst + chunk.first);
    for (int w = threadIdx.x; w < words; w += blockDim.x) out[w] = src[w];
}
static_assert(sizeof(GroupProblem) % 16 == 0, "descriptors are copied in 16-byte words");

struct BatchedLayout {
    size_t desc, operands, slot, total;
    std::vector<size_t> at_off, bt_off;
};

os_status batched_layout(int32_t count, const oversketch_plan_t *plans, const int64_t *m, const int64_t *n,
                         const int64_t *l, os_dtype a_t, os_dtype b_t, BatchedLayout *L) {
    if (count <= 0 || count > kMaxGroup || !plans || !m || !n || !l) return OS_ERR_INVALID_ARG;
    if ((a_t != OS_F32 && a_t != OS_BF16) || (b_t != OS_F32 && b_t != OS_BF16)) return OS_ERR_DTYPE;
    L->desc = align256(sizeof(GroupProblem) * (size_t)count);
    L->at_off.assign(count, 0);
    L->bt_off.assign(count, 0);
    size_t off = 0, slot = 256;
    for (int i = 0; i < count; ++i) {
        const Plan *p = reinterpret_cast<const Plan *>(plans[i]);
        if (!p || m[i] < 0 || l[i] < 0 || n[i] != p->n) return OS_ERR_INVALID_ARG;
        if (p->b % 64 != 0) return OS_ERR_UNSUPPORTED;   // BF16 GEMM K tile
        const int64_t z = (int64_t)p->P * p->b;
        L->at_off[i] = off;
        off += align256((size_t)m[i] * z * 2);
        L->bt_off[i] = off;
        off += align256((size_t)l[i] * z * 2);
        if (m[i] > 0 && l[i] > 0) {
            slot = std::max(slot, sketch_workspace_bytes(p, m[i], a_t));
            slot = std::max(slot, sketch_workspace_bytes(p, l[i], b_t));
        }
    }
    L->operands = off;
    L->slot = align256(slot);
    L->total = L->desc + L->operands + L->slot + 256;
    return OS_OK;
}

}  // namespace
}  // namespace osk

using namespace osk;

extern "C" os_status oversketch_matmul_batched_workspace_size(int32_t count, const oversketch_plan_t *plans,
                                                               const int64_t *m, const int64_t *n, const int64_t *l,
                                                               os_dtype a_t, os_dtype b_t, const os_opts *opts,
                                                               size_t *bytes) {
    if (!bytes) return OS_ERR_INVALID_ARG;
    if (opts && opts->gemm_dtype != OS_BF16) return OS_ERR_DTYPE;
    BatchedLayout L;
    OSK_TRY(batched_layout(count, plans, m, n, l, a_t, b_t, &L));
    *bytes = L.total;
    return OS_OK;
}

extern "C" os_status oversketch_matmul_batched(int32_t count, const oversketch_plan_t *plans,
                                               const void *const *A, const void *const *B, float *const *C,
                                               const int64_t *m, const int64_t *n, const int64_t *l, os_dtype a_t,
                                               os_dtype b_t, const uint64_t *masks, const os_opts *opts,
                                               void *workspace, size_t ws_bytes, void *stream) {
    OSK_NVTX("matmul_batched");
    if (opts && (opts->gemm_dtype != OS_BF16 || opts->col_scale || opts->symmetric || opts->flags))
        return opts->gemm_dtype != OS_BF16 ? OS_ERR_DTYPE : OS_ERR_UNSUPPORTED;
    BatchedLayout L;
    OSK_TRY(batched_layout(count, plans, m, n, l, a_t, b_t, &L));
    if (!A || !B || !C || !masks) return OS_ERR_INVALID_ARG;
    int dev = 0;
    OSK_CUDA_TRY(cudaGetDevice(&dev));
    std::vector<int> live;   // products with a non-empty C
    for (int i = 0; i < count; ++i) {
        const Plan *p = reinterpret_cast<const Plan *>(plans[i]);
        if (p->device != dev) return OS_ERR_INVALID_ARG;
        if (m[i] == 0 || l[i] == 0) continue;   // an empty C_i: nothing to read or write
        if (!A[i] || !B[i] || !C[i]) return OS_ERR_INVALID_ARG;
        live.push_back(i);
    }
    if (live.empty()) return OS_OK;
    if (!workspace || ws_bytes < L.total) return OS_ERR_WORKSPACE;
    cudaStream_t st = as_stream(stream);
    char *base = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(workspace) + 255) & ~uintptr_t(255));
    GroupProblem *desc = reinterpret_cast<GroupProblem *>(base);
    char *ops_base = base + L.desc;
    char *slots = ops_base + L.operands;
    // descriptors, longest K first (as for the batch object): the K of a product is
    // only known on the device, so the order uses its whole sketch width
    std::vector<int> ord = live;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
        const Plan *px = reinterpret_cast<const Plan *>(plans[x]), *py = reinterpret_cast<const Plan *>(plans[y]);
        const int64_t kx = (int64_t)px->P * px->b, ky = (int64_t)py->P * py->b;
        if (kx != ky) return kx > ky;
        return m[x] * l[x] > m[y] * l[y];
    });
    const int cnt = (int)ord.size();
    std::vector<GroupProblem> h(cnt);
    int32_t tiles = 0;
    for (int q = 0; q < cnt; ++q) {
        const int i = ord[q];
        const Plan *p = reinterpret_cast<const Plan *>(plans[i]);
        const int64_t z = (int64_t)p->P * p->b;
        OSK_TRY(group_problem_bf16(&h[q], kGroupBN256, ops_base + L.at_off[i], z, ops_base + L.bt_off[i], z, m[i],
                                   l[i], z, p->b, p->P, 0ull, masks + i, 1.f, 0.f, C[i], l[i]));
        h[q].tile_begin = tiles;
        const int64_t t = (int64_t)h[q].tiles_m * h[q].tiles_n;
        if ((int64_t)tiles + t >= (int64_t(1) << 31)) return OS_ERR_UNSUPPORTED;
        tiles += (int32_t)t;
    }
    OSK_TRY(gemm_grouped_prepare());
    for (int c0 = 0; c0 < cnt; c0 += kDescPerChunk) {
        DescChunk chunk;
        std::memset(&chunk, 0, sizeof(chunk));
        chunk.first = c0;
        chunk.count = std::min(kDescPerChunk, cnt - c0);
        std::memcpy(chunk.items, h.data() + c0, sizeof(GroupProblem) * chunk.count);
        upload_groups_kernel<<<1, 256, 0, st>>>(chunk, desc);
        OSK_TRY(check_launch());
    }
    // the sketches, one product after another, sharing one packing slot
    for (int i : live) {
        const Plan *p = reinterpret_cast<const Plan *>(plans[i]);
        const int64_t z = (int64_t)p->P * p->b;
        const uint64_t all = p->P >= 64 ? ~0ull : ((1ull << p->P) - 1ull);
        OSK_TRY(sketch_left_impl(p, A[i], a_t, m[i], n[i], ops_base + L.at_off[i], OS_BF16, z, nullptr, nullptr, all,
                                 slots, L.slot, st, masks + i));
        OSK_TRY(sketch_right_impl(p, B[i], b_t, l[i], l[i], ops_base + L.bt_off[i], OS_BF16, z, nullptr, all, slots,
                                  L.slot, st, nullptr, masks + i));
    }
    return gemm_grouped_bf16(desc, cnt, tiles, kGroupBN256, st);
}

extern "C" os_status oversketch_batch_create(const os_problem *problems, int32_t count, os_dtype a_t,
                                             os_dtype b_t, os_dtype gemm_dtype, size_t workspace_limit,
                                             int32_t tune, void *stream, oversketch_batch_t *batch) {
    if (!batch) return OS_ERR_INVALID_ARG;
    *batch = nullptr;
    Batch *B = new (std::nothrow) Batch();
    if (!B) return OS_ERR_OOM;
    const os_status s = create(problems, count, a_t, b_t, gemm_dtype, workspace_limit, tune, as_stream(stream), B);
    if (s != OS_OK) {
        cudaDeviceSynchronize();
        free_batch(B);
        return s;
    }
    *batch = reinterpret_cast<oversketch_batch_t>(B);
    return OS_OK;
}

extern "C" os_status oversketch_batch_run(oversketch_batch_t batch, void *stream) {
    OSK_NVTX("batch_run");
    Batch *B = reinterpret_cast<Batch *>(batch);
    if (!B || !B->exec) return OS_ERR_INVALID_ARG;
    int dev = 0;
    OSK_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != B->device) return OS_ERR_INVALID_ARG;
    OSK_CUDA_TRY(cudaGraphLaunch(B->exec, as_stream(stream)));
    return OS_OK;
}

extern "C" os_status oversketch_batch_info(oversketch_batch_t batch, os_batch_info *info) {
    Batch *B = reinterpret_cast<Batch *>(batch);
    if (!B || !info) return OS_ERR_INVALID_ARG;
    info->count = (int32_t)B->probs.size();
    info->branches = B->branches;
    info->tile_n = B->tile == kGroupBN256 ? 256 : 128;
    info->total_tiles = B->total_tiles[B->tile];
    info->kernel_launches = B->launches;
    info->operand_bytes = B->operand_bytes;
    info->workspace_bytes = B->slot_bytes * B->max_branches;
    info->tuned_ms = B->tuned_ms;
    return OS_OK;
}

extern "C" os_status oversketch_batch_destroy(oversketch_batch_t batch) {
    Batch *B = reinterpret_cast<Batch *>(batch);
    if (!B) return OS_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    return free_batch(B);
}
