/*
 * oversketch.h -- C ABI of the GB300 (sm_103a) OverSketch library.
 *
 * OverSketch (Gupta, Wang, Courtade, Ramchandran, arXiv 1811.02653) computes
 * the approximate product
 *
 *     C = (1/k) * sum_{j in mask} (A S_j) (S_j^T B)                      (*)
 *
 * where S = (S_1, ..., S_{N+e}) stacks N+e independent Count-sketch blocks of
 * width b (Eq. 3; Alg. 4 defines one block), A S and S^T B are computed by the
 * bucket sums of Alg. 4 step 3 / Alg. 5, and the sum keeps any k blocks chosen
 * by a caller mask, standing in for Alg. 3's termination rule ("stop when any
 * d/b of the z/b workers returned").  k = popcount(mask); the 1/sqrt(N) of
 * Eq. 3 on both sides is applied once as 1/k (k = N when exactly N blocks are
 * kept; keeping fewer is the "graceful degradation" of Sec. 4.1).
 *
 * Conventions (all entry points):
 *   - Matrices are row-major; ld* is the leading dimension in ELEMENTS.
 *   - Matrix pointers are DEVICE pointers owned by the caller, except where
 *     an argument is documented as host memory.  Nothing is retained after
 *     a call returns, except by plan objects.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy stream).
 *     Compute entry points are asynchronous on that stream; argument errors
 *     are detected on the host before any launch and returned synchronously.
 *   - Blocks are 0-based, j = 0 .. P-1 with P = N + e <= 64.  Bucket indices
 *     are 0-based (the paper counts 1..b).  Sketched index q = j*b + c.
 *   - The library never allocates inside compute calls; callers pass a
 *     workspace sized by oversketch_workspace_size().  Plans allocate their
 *     own device tables at creation.
 *   - Sketch outputs are UNSCALED (+-1 entries of S); only the masked
 *     product applies 1/k.
 *   - Sketched operands are stored K-major: A~ is m x z (row r contiguous
 *     over q) and B~^T is l x z (column c of B~ contiguous over q), so both
 *     feed the tensor-core GEMM without a transpose.
 *   - Empty outputs: when an output has no elements (m = 0 or l = 0, zero
 *     rows to sketch or to unsketch) a call checks its other arguments and
 *     returns OS_OK without launching anything; its data pointers may then be
 *     NULL (empty tensors often have no storage).
 */
#ifndef OVERSKETCH_H
#define OVERSKETCH_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define OS_API __attribute__((visibility("default")))
#else
#define OS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oversketch_plan_s *oversketch_plan_t;

typedef enum {
    OS_OK = 0,
    OS_ERR_INVALID_ARG = 1,   /* bad size, null pointer, misaligned ld     */
    OS_ERR_MASK = 2,          /* mask empty or selects a block >= N+e      */
    OS_ERR_DTYPE = 3,         /* dtype combination not supported           */
    OS_ERR_OOM = 4,           /* plan allocation failed                    */
    OS_ERR_CUDA = 5,          /* a CUDA runtime call failed                */
    OS_ERR_TIMEOUT = 6,       /* a bounded device wait expired             */
    OS_ERR_UNSUPPORTED = 7,   /* N+e > 64, block width not tile-aligned... */
    OS_ERR_WORKSPACE = 8      /* workspace missing or too small            */
} os_status;

typedef enum {
    OS_F32 = 0,               /* IEEE binary32                              */
    OS_BF16 = 1,              /* bfloat16, round-to-nearest-even            */
    OS_FP8E4M3 = 2,           /* OCP FP8 E4M3 + per-(row, 128-q) power-of-2 */
    OS_TF32X2 = 3             /* FP32 as two planes hi + lo: hi = x with the low 13
                                 mantissa bits cleared (exact in TF32), lo = x - hi;
                                 plane lo follows plane hi (rows * ld elements) */
} os_dtype;

/* Entries per slice of an FP8 scale array for `rows` rows (rows rounded up to
 * a multiple of 4, so every slice starts on a 16-byte boundary). */
#define OS_FP8_SCALE_LD(rows) ((((rows) + 3) / 4) * 4)

/* Human-readable name of a status code (static storage). */
OS_API const char *oversketch_status_string(os_status s);

/* Message of the last CUDA error seen by the library on this thread. */
OS_API const char *oversketch_last_cuda_error(void);

/* -------------------------------------------------------------------------
 * Plans: the sketch S of Eq. 3, built on the device.
 *
 * oversketch_plan -- Alg. 4 steps 1-2 for each of the P = N + e blocks:
 *   w = splitmix64-mix(key_j + (i+1)*gamma), key_j = mix(seed + (j+1)*gamma),
 *   h_j(i) = ((w >> 32) * b) >> 32 in [0, b), sigma_j(i) = (w & 1) ? -1 : +1,
 * then a deterministic stable counting sort of every block by bucket (the
 * "columns mapped to the same integer" of Alg. 4 step 3), kept as a
 * bucket-CSR.  n >= 1, b >= 1, N >= 1, e >= 0, N + e <= 64, n < 2^31,
 * (N+e)*b < 2^31.  The plan owns its device tables until destroyed; it may
 * be used concurrently by several calls on any streams once the creating
 * stream has reached the end of the call (the call synchronises `stream`
 * before returning).  Errors: OS_ERR_INVALID_ARG, OS_ERR_UNSUPPORTED,
 * OS_ERR_OOM, OS_ERR_CUDA.
 */
OS_API os_status oversketch_plan(int64_t n, int32_t b, int32_t N, int32_t e, uint64_t seed,
                          void *stream, oversketch_plan_t *out);

/* Same, from explicit tables in HOST memory: h[j*n + i] in [0,b) and
 * sigma[j*n + i] in {+1,-1} (for worked examples such as Eq. 2 and for
 * injective test hashes).  Errors as above, plus OS_ERR_INVALID_ARG for an
 * out-of-range entry. */
OS_API os_status oversketch_plan_from_tables(int64_t n, int32_t b, int32_t N, int32_t e,
                                      const uint32_t *h_host, const int8_t *sigma_host,
                                      void *stream, oversketch_plan_t *out);

/* Copy the plan's tables to HOST memory: h_host and sigma_host hold
 * (N+e)*n entries each (row j = block j); perm_host ((N+e)*n entries,
 * index | sign << 31, bucket-sorted per block, ascending index inside a
 * bucket) and offs_host ((N+e)*(b+1) entries) may be NULL.  Synchronous. */
OS_API os_status oversketch_plan_get_tables(oversketch_plan_t plan, uint32_t *h_host, int8_t *sigma_host,
                                     uint32_t *perm_host, uint32_t *offs_host);

/* Plan parameters (any output pointer may be NULL). */
OS_API os_status oversketch_plan_info(oversketch_plan_t plan, int64_t *n, int32_t *b, int32_t *N,
                               int32_t *e);

/* Release the plan's device tables (synchronises the device first). */
OS_API os_status oversketch_plan_destroy(oversketch_plan_t plan);

/* Number of blocks for a target accuracy (Thm. 4.1).  d = 2/(eps*theta) sketch
 * columns make the product (eps, theta)-accurate:
 *   ||AB - (AS)(S^T B)||_F^2 <= eps ||A||_F^2 ||B||_F^2 with probability >= 1 - theta.
 * With blocks of width b: *N = ceil(r*d/b) (r >= 1 multiplies the dimension, as
 * the paper's remark after the theorem does for the spectral-norm bound), and *e
 * = the smallest e with e >= p*(N + e) for a straggler fraction p in [0, 1): the
 * N + e blocks still hold N after a fraction p of them is dropped.  Host-only.
 * Errors: OS_ERR_INVALID_ARG (eps <= 0, theta outside (0,1), b < 1, r < 1, p
 * outside [0,1)); OS_ERR_UNSUPPORTED when N + e would exceed 64. */
OS_API os_status oversketch_sketch_size(double eps, double theta, int32_t b, double straggler_fraction,
                                 int32_t r, int32_t *N, int32_t *e);

/* -------------------------------------------------------------------------
 * Sketches (Alg. 5: A~ = A S block by block; B~ = S^T B).
 *
 * oversketch_sketch_left:
 *   At[r, j*b + c] = sum_{i : h_j(i) = c} sigma_j(i) * s_i * A[r, i]
 *   A: m x n, dtype a_t (OS_F32 or OS_BF16), leading dim lda >= n.
 *   col_scale: device FP32 array of n scales s_i, or NULL (s_i = 1); used
 *     for A diag(s) S, e.g. the sqrt(D) of the interior-point Hessian.
 *   At: m x z in dtype out_t with leading dim ldat >= z (z = (N+e)*b).
 *   scales: for out_t == OS_FP8E4M3, device FP32 array of (z/128) slices of
 *     OS_FP8_SCALE_LD(m) entries each (slice-major, 16-byte aligned): entry
 *     [t * OS_FP8_SCALE_LD(m) + r] = 2^e_rt with e_rt the smallest integer
 *     (clamped to [-127, 127]) such that the FP32 sums of slice t (columns
 *     128t .. 128t+127) of row r are all <= 448 * 2^e_rt in magnitude (1.0
 *     for an all-zero slice); At holds round-to-nearest-even, saturating E4M3
 *     codes of (sum / 2^e_rt).  Entries of padding rows are not written.
 *     NULL otherwise.  FP8 needs b % 128 == 0.  When the workspace also has
 *     room for m x z FP32 values after the regular workspace (ws_bytes >=
 *     roundup256(oversketch_sketch_workspace(plan, m, a_t)) + 4*m*z + 256), the
 *     FP32 sums are staged there and quantised by a second kernel instead of in
 *     the gather's epilogue (thread-block clusters of four): the same codes and
 *     scales, faster.
 *   Sums are accumulated in FP32 in ascending order of i inside a bucket;
 *   BF16 output is the round-to-nearest-even of that FP32 sum.
 *   block_mask: bit j set = compute the columns of block j; 0 = all blocks.
 *     Columns of blocks not listed are left untouched (the paper's remark
 *     that blocks missed while sketching become stragglers of the product).
 *   workspace: device memory of at least oversketch_sketch_workspace(plan, m,
 *     a_t) bytes; the operand is packed there strip-major (n rows of 512
 *     bytes per strip: 128 FP32 or 256 BF16 free indices) before the bucket
 *     gather, and with a col_scale
 *     the signed scales sigma_j(i) * s_i are laid out there in bucket-list
 *     order first (one coalesced load per 32 gathered rows).
 * oversketch_sketch_right:
 *   BtT[c, j*b + q] = sum_{i : h_j(i) = q} sigma_j(i) * s_i * B[i, c]
 *   B: n x l (ldb >= l); BtT: l x z (ldbt >= z); FP8 scales as above with
 *   OS_FP8_SCALE_LD(l) entries per slice;
 *   row_scale: n FP32 device values s_i, or NULL (s_i = 1): S^T diag(s) B,
 *     e.g. the Hessian square root diag(1/s) A of Sec. 5.2 without forming it;
 *     a term is s_i * B[i, c] rounded once, then added;
 *   block_mask as above; workspace of oversketch_sketch_workspace(plan, l, b_t)
 *   bytes (an FP32 B with 16-byte aligned rows is gathered in place in
 *   128-column strips and only a ragged remainder of fewer than 128 columns
 *   is packed there; with a row_scale the workspace also holds the signed
 *   scales in bucket-list order).
 * Errors: OS_ERR_INVALID_ARG (null pointers, ld too small, out pointers or
 *   ld not 16-byte aligned), OS_ERR_DTYPE, OS_ERR_UNSUPPORTED,
 *   OS_ERR_WORKSPACE, OS_ERR_CUDA (launch failure).
 */
OS_API os_status oversketch_sketch_workspace(oversketch_plan_t plan, int64_t free_extent, os_dtype in_t,
                                      size_t *bytes);
OS_API os_status oversketch_sketch_left(oversketch_plan_t plan, const void *A, os_dtype a_t, int64_t m,
                                 int64_t lda, void *At, os_dtype out_t, int64_t ldat, float *scales,
                                 const float *col_scale, uint64_t block_mask, void *workspace,
                                 size_t ws_bytes, void *stream);
OS_API os_status oversketch_sketch_right(oversketch_plan_t plan, const void *B, os_dtype b_t, int64_t l,
                                  int64_t ldb, void *BtT, os_dtype out_t, int64_t ldbt,
                                  float *scales, const float *row_scale, uint64_t block_mask,
                                  void *workspace, size_t ws_bytes, void *stream);

/* -------------------------------------------------------------------------
 * Left sketch of a sparse operand stored dense (Alg. 4 step 3 over the
 * nonzeros only; Sec. 4 prices sketching at O(nnz(A)(N+e))), e.g. the
 * 1%-dense constraint matrix of the interior-point Hessian A D A^T (Sec. 5.2).
 *   At[r, j*b + c] = sum_{i : A[r,i] != 0, h_j(i) = c} sigma_j(i) * s_i * A[r, i]
 * The same operation, layouts, FP8 scale rule, block_mask semantics and
 * errors as oversketch_sketch_left, without a workspace: one CTA per row
 * reads the row once and keeps all k*b sums of the listed blocks on chip.
 * Per bucket the FP32 sum runs over the nonzero members in ascending i; a
 * term is s_i * A[r,i] rounded once, then added (exact zeros are skipped,
 * which changes no sum).  Correct for any density, fast for sparse rows.
 *   Limit: with k listed blocks, k*b <= 32768 and the row's k*b FP32 sums,
 *   two tables of b bucket offsets and a buffer of 1024 entries fit in one
 *   CTA's shared memory (4*k*b + 8*b + 20*1024 bytes <= about 226 KB), else
 *   OS_ERR_UNSUPPORTED.
 */
OS_API os_status oversketch_sketch_left_sparse(oversketch_plan_t plan, const void *A, os_dtype a_t,
                                        int64_t m, int64_t lda, void *At, os_dtype out_t,
                                        int64_t ldat, float *scales, const float *col_scale,
                                        uint64_t block_mask, void *stream);

/* -------------------------------------------------------------------------
 * Left sketch without allocation.  The paper has no counterpart: this is a
 * library convenience.  Same operation, arguments and errors as
 * oversketch_sketch_left, but the packing workspace is a fixed scratch array
 * of 32 MiB in device memory that every GPU loading the library holds until
 * the process exits.  For callers that cannot allocate device memory at the
 * point where they sketch: code running while a stream is captured into a
 * CUDA graph (cudaMalloc is not permitted there), code whose memory belongs to
 * another allocator or a fixed budget, and latency-critical loops that must
 * not call cudaMalloc (it can synchronise the device).  The call allocates
 * nothing; the plan and the output are the caller's.
 *   - Limit: oversketch_sketch_workspace(plan, m, a_t) <= 32 MiB (for FP32
 *     that is about ceil(m/128) * 128 * n * 4 bytes plus 4 * (N+e) * (n + 3b)
 *     bytes of entry weights), else OS_ERR_WORKSPACE and no launch.
 *   - Arguments are checked as by oversketch_sketch_left, and an empty output
 *     (m = 0) returns OS_OK, before anything else happens.
 *   - The first call in a CUDA context looks up the scratch array's device
 *     address (cudaGetSymbolAddress) with that device current; make that first
 *     call before any stream capture.  A context created later on the same
 *     device (after cudaDeviceReset) gets its own lookup on its first call.
 *   - All calls share the array and it keeps the last call's contents; every
 *     byte a call reads is written by that call first, so nothing needs
 *     clearing.  Calls that overlap on the GPU (different streams, or several
 *     threads) race on the array: serialise them.
 */
OS_API os_status oversketch_sketch_left_noalloc(oversketch_plan_t plan, const void *A, os_dtype a_t,
                                         int64_t m, int64_t lda, void *At, os_dtype out_t,
                                         int64_t ldat, float *scales, const float *col_scale,
                                         uint64_t block_mask, void *stream);

/* -------------------------------------------------------------------------
 * Masked block-sum GEMM (Alg. 3 computation + termination + reduction; the
 * b x b block products of Alg. 2 become one GEMM whose inner dimension is
 * the concatenation of the kept blocks):
 *   C[r, c] = (alpha / k) * sum_{j in mask} sum_{q < b} At[r, j*b + q] * BtT[c, j*b + q]
 *            (+ beta * C[r, c] when beta != 0),   k = popcount(mask)
 * The 1/k of (*) is applied here, derived from the mask (the sketches are
 * unscaled); alpha = 1 gives (*), other values scale it further.
 * At: m x z (ldat), BtT: l x z (ldbt), both in dtype `dt`; FP8 operands
 * carry the per-(row, 128-q) scales produced by the sketches.  C: FP32
 * m x l (ldc).  OS_F32 operands are
 * computed at FP32 accuracy, BF16 and FP8 on the tensor cores with FP32
 * accumulation.  K tiles: 16 (FP32), 64 (BF16), 128 (FP8); b must be a
 * multiple of the K tile.  Tensor-core operands need 16-byte aligned rows.
 * Errors: OS_ERR_MASK, OS_ERR_INVALID_ARG, OS_ERR_DTYPE, OS_ERR_UNSUPPORTED
 * (b not a multiple of the K tile), OS_ERR_CUDA.
 */
OS_API os_status oversketch_gemm_masked(oversketch_plan_t plan, const void *At, int64_t ldat,
                                 const float *a_scales, const void *BtT, int64_t ldbt,
                                 const float *b_scales, os_dtype dt, int64_t m, int64_t l,
                                 uint64_t mask, float alpha, float beta, float *C, int64_t ldc,
                                 void *stream);

/* Alg. 3's termination rule per block of C: the reduction of block (i, j)
 * (rows i*bm .., columns j*bn ..) keeps its own set of sketch blocks,
 *   C(i, j) = (1/k_ij) sum_{t in masks[i*nbc + j]} At(i, t) BtT(j, t)^T  (+ beta C(i, j)),
 * nbc = ceil(l / bn), k_ij = popcount of the mask.  block_masks: DEVICE array of
 * ceil(m/bm) * nbc masks (bits >= N+e are ignored; an empty mask gives a zero
 * block).  At, BtT: BF16 sketches holding every block that any mask keeps.  bm and
 * bn: multiples of 256 (the CTA-pair tile), e.g. the paper's b x b blocks.
 * Errors: OS_ERR_INVALID_ARG, OS_ERR_UNSUPPORTED (bm or bn not a multiple of 256,
 * b not a multiple of 64), OS_ERR_CUDA. */
OS_API os_status oversketch_gemm_masked_blocks(oversketch_plan_t plan, const void *At, int64_t ldat,
                                        const void *BtT, int64_t ldbt, int64_t m, int64_t l,
                                        const uint64_t *block_masks, int64_t bm, int64_t bn,
                                        float beta, float *C, int64_t ldc, void *stream);

/* -------------------------------------------------------------------------
 * The whole product (*): left sketch, right sketch, masked GEMM.
 */
typedef struct {
    os_dtype gemm_dtype;      /* OS_F32, OS_BF16 or OS_FP8E4M3               */
    const float *col_scale;   /* device, length n, or NULL (A diag(s) S)     */
    int32_t symmetric;        /* 1: B is ignored and C = (1/k) A~_sel A~_sel^T */
    int32_t flags;            /* OS_OPT_* bits, 0 by default                  */
} os_opts;

/* os_opts.flags: A is sparse (stored dense): sketch it with
 * oversketch_sketch_left_sparse when the kept blocks fit its limit (the
 * dense path otherwise).  The result differs only in FP32 summation order. */
#define OS_OPT_SPARSE_A 1

OS_API os_status oversketch_workspace_size(oversketch_plan_t plan, int64_t m, int64_t l,
                                    os_dtype a_t, os_dtype b_t, const os_opts *opts, size_t *bytes);
OS_API os_status oversketch_matmul(oversketch_plan_t plan, const void *A, os_dtype a_t, int64_t lda,
                            const void *B, os_dtype b_t, int64_t ldb, float *C, int64_t ldc,
                            int64_t m, int64_t n, int64_t l, uint64_t mask, const os_opts *opts,
                            void *workspace, size_t ws_bytes, void *stream);

/* The same product with A, B and C in HOST memory (page-locked memory lets the
 * transfers overlap the kernels; pageable memory works, slower).  B is copied
 * first and sketched while A arrives in chunks of rows, each chunk sketched as
 * it lands; the masked GEMM runs in row panels and each panel of C is copied
 * back while the next one is computed (BF16 products; FP8 and FP32 products
 * sketch A and compute C in one piece).  The copies run on an internal stream of
 * the device, ordered after the caller's earlier work on `stream`; the call is
 * complete on `stream` once C is written (stream-ordered: synchronise `stream`
 * before reading C).  workspace: device memory of
 * oversketch_matmul_host_workspace_size bytes (the device copies of A, B and C
 * and the sketched operands).  Same arguments and errors as oversketch_matmul,
 * with the pointers A, B (ignored when symmetric) and C in host memory. */
OS_API os_status oversketch_matmul_host_workspace_size(oversketch_plan_t plan, int64_t m, int64_t l,
                                                os_dtype a_t, os_dtype b_t, const os_opts *opts,
                                                size_t *bytes);
OS_API os_status oversketch_matmul_host(oversketch_plan_t plan, const void *A, os_dtype a_t, int64_t lda,
                                 const void *B, os_dtype b_t, int64_t ldb, float *C, int64_t ldc,
                                 int64_t m, int64_t n, int64_t l, uint64_t mask, const os_opts *opts,
                                 void *workspace, size_t ws_bytes, void *stream);

/* -------------------------------------------------------------------------
 * Adjoints of the sketch restricted to the kept blocks (the backward pass of
 * (*) as a function of A and B; S_sel is S of Eq. 3 restricted to the kept
 * blocks).  The inputs hold the kept blocks only, compacted in ascending
 * block order (column / row t*b + c belongs to the t-th kept block):
 *   unsketch_cols: dX[r, i] = scale * sum_t sigma_j(i) T[r, t*b + h_j(i)],  j = kept[t]
 *                  T: m x (k*b) FP32 (ldt); dX: m x n in dtype x_t (ldx).
 *   unsketch_rows: dG[i, c] = scale * sum_t sigma_j(i) U[t*b + h_j(i), c],  j = kept[t]
 *                  U: (k*b) x l FP32 (ldu); dG: n x l in dtype g_t (ldg).
 * x_t / g_t: OS_F32 or OS_BF16.  Sums in FP32 over kept blocks in ascending
 * order.  unsketch_cols stages up to four rows of T per CTA in shared memory
 * when a row (4*k*b bytes) fits in 200 KB; longer rows are read from global
 * memory and then m <= 65535 (else OS_ERR_UNSUPPORTED).
 * Errors: OS_ERR_MASK, OS_ERR_INVALID_ARG, OS_ERR_DTYPE, OS_ERR_UNSUPPORTED,
 * OS_ERR_CUDA.
 */
OS_API os_status oversketch_unsketch_cols(oversketch_plan_t plan, const float *T, int64_t m, int64_t ldt,
                                   uint64_t mask, float scale, void *dX, os_dtype x_t,
                                   int64_t ldx, void *stream);
OS_API os_status oversketch_unsketch_rows(oversketch_plan_t plan, const float *U, int64_t l,
                                   int64_t ldu, uint64_t mask, float scale, void *dG,
                                   os_dtype g_t, int64_t ldg, void *stream);

/* -------------------------------------------------------------------------
 * Backward pass of (*) (the adjoint of Eq. 3's map S restricted to the kept
 * blocks; C is bilinear in A and B):
 *   dX = (1/k) (dC . B~_sel^T) . S_sel^T          (m x n, the gradient for A)
 *   dG = (1/k) S_sel . (A~_sel^T . dC)            (n x l, the gradient for B)
 * with k = popcount(mask), derived here from the mask.  At (m x z, ldat) and
 * BtT (l x z, ldbt) are the BF16 sketches of the forward pass (only the kept
 * blocks are read); dC: FP32 m x l (lddc).  Each side is one BF16 tensor-core
 * GEMM with FP32 accumulation (dC rounded to BF16, 1/k in the GEMM epilogue)
 * followed by an unsketch gather into dX (x_t) or dG (g_t), OS_F32 or OS_BF16.
 * With b a multiple of 128 and m, l multiples of 8 the tensor cores read At, BtT
 * and dC as they are laid out (MN-major where the product needs it, the kept
 * blocks picked by column); otherwise the kept blocks and dC are first
 * transposed into K-major copies.
 * dX or dG may be NULL: that side is skipped.  workspace: device memory of
 * oversketch_matmul_backward_workspace_size(plan, m, l, mask, dX != NULL,
 * dG != NULL) bytes (dC in BF16, any transposed copies, and the FP32 GEMM
 * results).  Asynchronous on `stream`.
 * Errors: OS_ERR_MASK, OS_ERR_INVALID_ARG, OS_ERR_DTYPE, OS_ERR_WORKSPACE,
 * OS_ERR_UNSUPPORTED (see unsketch_cols), OS_ERR_CUDA.
 */
OS_API os_status oversketch_matmul_backward_workspace_size(oversketch_plan_t plan, int64_t m, int64_t l,
                                                           uint64_t mask, int32_t need_dx, int32_t need_dg,
                                                           size_t *bytes);
OS_API os_status oversketch_matmul_backward(oversketch_plan_t plan, const void *At, int64_t ldat,
                                            const void *BtT, int64_t ldbt, const float *dC, int64_t lddc,
                                            int64_t m, int64_t l, uint64_t mask, void *dX, os_dtype x_t,
                                            int64_t ldx, void *dG, os_dtype g_t, int64_t ldg, void *workspace,
                                            size_t ws_bytes, void *stream);

/* -------------------------------------------------------------------------
 * Plain BF16 GEMM on the tensor cores (the same tcgen05 kernel with one K
 * block), used by the backward pass:
 *   C = alpha * A . B^T (+ beta * C),  A: m x K, B: n x K, both K-major BF16
 *   (16-byte aligned rows, so K % 8 == 0 when lda == K), C: m x n FP32.
 */
OS_API os_status oversketch_gemm_bf16(const void *A, int64_t lda, const void *B, int64_t ldb, int64_t m,
                               int64_t n, int64_t K, float alpha, float beta, float *C, int64_t ldc,
                               void *stream);

/* -------------------------------------------------------------------------
 * Layout conversions (data movement only):
 *   select_transpose: Y[c', r] = X[r, col(c')] for an X of rows x cols (ldx);
 *     block_mask == 0: all columns (col(c') = c'); else the columns of the
 *     blocks of width b whose bits are set, compacted in ascending order
 *     (cols % b == 0, cols / b <= 64).  Y: (selected cols) x rows (ldy).
 *   cast: Y = X elementwise, rows x cols.
 * x_t, y_t: OS_F32 or OS_BF16 (FP32 -> BF16 rounds to nearest even).
 */
OS_API os_status oversketch_select_transpose(const void *X, os_dtype x_t, int64_t rows, int64_t cols,
                                      int64_t ldx, uint64_t block_mask, int32_t b, void *Y,
                                      os_dtype y_t, int64_t ldy, void *stream);
OS_API os_status oversketch_cast(const void *X, os_dtype x_t, int64_t rows, int64_t cols, int64_t ldx,
                          void *Y, os_dtype y_t, int64_t ldy, void *stream);

/* -------------------------------------------------------------------------
 * FP64 error measurement (Def. 4.1 is stated in squared Frobenius norms):
 *   out[0] = sum (X - Y)^2, out[1] = sum Y^2, out[2] = sum X*Y, accumulated
 *   in FP64 over the rows x cols FP32 matrices X (ldx) and Y (ldy); Y may be
 *   NULL (then out[0] = sum X^2 and out[1] = out[2] = 0).  out: DEVICE array
 *   of 3 doubles, overwritten.  workspace: device memory of at least
 *   OS_FROB_WORKSPACE_BYTES (8-byte aligned) for the per-CTA partial sums.
 *   Deterministic: fixed grid, fixed summation order, no atomics.
 */
#define OS_FROB_WORKSPACE_BYTES 12288
OS_API os_status oversketch_frob(const float *X, int64_t ldx, const float *Y, int64_t ldy, int64_t rows,
                          int64_t cols, double *out, void *workspace, size_t ws_bytes,
                          void *stream);

/* -------------------------------------------------------------------------
 * Device status of the tensor-core kernels.  Every wait inside them is
 * bounded (about one second); a wait that expires makes the kernel record
 * OS_ERR_TIMEOUT here, drain its own copies, release its tensor memory and
 * return instead of hanging.  *status = OS_OK or OS_ERR_TIMEOUT; reset != 0
 * clears the word.  Synchronises `stream`.
 */
OS_API os_status oversketch_device_status(void *stream, int32_t *status, int32_t reset);

/* Test hook of the bounded waits; the paper has no counterpart.  With
 * skip_kb >= 0, the next launch of the one-CTA tensor-core GEMM (the FP8 and
 * 3xTF32 masked products, grouped BF16 launches) leaves K step skip_kb of its
 * first CTA's first tile unloaded and unarmed, and gives that CTA a wait limit
 * of limit_ns (> 0) instead of one second: the MMA warp's wait for that stage
 * runs out, the CTA records OS_ERR_TIMEOUT, waits (one second at most) for the
 * copies it did issue, frees its tensor memory and returns.  The setting is
 * consumed by that one launch; skip_kb < 0 withdraws a pending one.
 * Synchronous (device-wide symbol copies).  Errors: OS_ERR_INVALID_ARG
 * (limit_ns == 0 with skip_kb >= 0), OS_ERR_CUDA. */
OS_API os_status oversketch_test_wait_timeout(uint64_t limit_ns, int32_t skip_kb);

/* -------------------------------------------------------------------------
 * Many independent products in one call, each with its own plan, sizes and kept
 * blocks (Alg. 3: a product's block products are independent jobs, and so are
 * whole products), its mask read from DEVICE memory when the work runs:
 *   C_p = (1/k_p) (A_p S_p,sel)(S_p,sel^T B_p),  k_p = popcount(masks[p] & (2^P_p - 1)),
 * so one captured CUDA graph of the call serves a different straggler set on
 * every replay (the caller rewrites masks[] between replays).  An empty mask
 * gives C_p = 0; bits >= N_p + e_p are ignored.
 *   plans, A, B, C, m, n, l: HOST arrays of count (1 .. 1024) entries; A_p (m_p x
 *     n_p, row-major, leading dim n_p) and B_p (n_p x l_p, leading dim l_p) in
 *     a_t / b_t (OS_F32 or OS_BF16), C_p FP32 m_p x l_p (leading dim l_p), all
 *     device memory; n_p equals the plan's n, every plan on the current device
 *     with b % 64 == 0.  m_p = 0 or l_p = 0: product p is skipped (its pointers
 *     may be NULL).
 *   masks: DEVICE array of count uint64 words.
 *   opts: NULL or gemm_dtype OS_BF16 (the GEMM runs in BF16 with FP32
 *     accumulation); col_scale, symmetric and flags are not supported here.
 *   workspace: device memory of oversketch_matmul_batched_workspace_size bytes:
 *     the GEMM descriptors, every product's BF16 sketches ((m_p + l_p) z_p
 *     elements) and one packing slot.  The call allocates nothing: the
 *     descriptors are written into the workspace by kernels that carry them as
 *     launch parameters, so a captured graph holds everything it needs.
 * Work, all on `stream`: the descriptors, the sketches product after product
 * (every block is sketched; CTAs of blocks the device mask drops return at
 * once), then one persistent tcgen05 launch over the tiles of all products
 * (longest sketch first).
 * Errors: OS_ERR_INVALID_ARG, OS_ERR_DTYPE, OS_ERR_UNSUPPORTED, OS_ERR_WORKSPACE,
 * OS_ERR_CUDA.
 */
OS_API os_status oversketch_matmul_batched_workspace_size(int32_t count, const oversketch_plan_t *plans,
                                                          const int64_t *m, const int64_t *n, const int64_t *l,
                                                          os_dtype a_t, os_dtype b_t, const os_opts *opts,
                                                          size_t *bytes);
OS_API os_status oversketch_matmul_batched(int32_t count, const oversketch_plan_t *plans, const void *const *A,
                                           const void *const *B, float *const *C, const int64_t *m, const int64_t *n,
                                           const int64_t *l, os_dtype a_t, os_dtype b_t, const uint64_t *masks,
                                           const os_opts *opts, void *workspace, size_t ws_bytes, void *stream);

/* -------------------------------------------------------------------------
 * Batches of independent products (Alg. 3's blocks are independent jobs;
 * here so are whole products).  Product p is
 *   C_p = (1/k_p) (A_p S_p,sel)(S_p,sel^T B_p),  k_p = popcount(mask_p),
 * with its own sizes, plan and mask; the GEMM runs in BF16 with FP32
 * accumulation, like oversketch_matmul with gemm_dtype OS_BF16.
 *
 * oversketch_batch_create fixes the products (sizes, pointers, plans and
 * masks are captured: later runs read A_p, B_p and write C_p at the same
 * addresses) and records one CUDA graph: the sketches of the products spread
 * over W parallel branches (each with one packing workspace slot), then one
 * persistent tensor-core launch over the tiles of all products, longest K
 * first.  It allocates the sketched operands (BF16, (m_p + l_p) * z_p
 * elements per product) and W workspace slots of the largest single-product
 * packing size, W <= workspace_limit / slot (0: 16 GiB).  tune != 0 times a
 * few (W, tile width) choices on `stream` (running the products several
 * times) and keeps the fastest; tune == 0 takes W = 1 and 256-wide tiles.  Synchronous; call it outside any stream capture.
 *   problems: host array of count (1..1024) descriptors; A_p, B_p device
 *     row-major in a_t / b_t (OS_F32 or OS_BF16), C_p device FP32; every plan
 *     on the current device with b % 64 == 0; m_p, n_p, l_p >= 1.
 *   gemm_dtype: OS_BF16 (others: OS_ERR_DTYPE).
 * oversketch_batch_run launches the graph on `stream` (stream-ordered, on
 *   the device the batch was created on).  Runs of one batch must not overlap.
 * oversketch_batch_info: what the batch holds and chose.
 * Errors: OS_ERR_INVALID_ARG, OS_ERR_MASK, OS_ERR_DTYPE, OS_ERR_UNSUPPORTED,
 *   OS_ERR_WORKSPACE (one product's packing slot exceeds workspace_limit),
 *   OS_ERR_CUDA.
 */
typedef struct {
    int64_t m, n, l;
    const void *A; int64_t lda;      /* m x n */
    const void *B; int64_t ldb;      /* n x l */
    float *C; int64_t ldc;           /* m x l, FP32 */
    oversketch_plan_t plan;          /* dimension n */
    uint64_t mask;                   /* kept blocks */
} os_problem;

typedef struct oversketch_batch_s *oversketch_batch_t;

typedef struct {
    int32_t count;                   /* products */
    int32_t branches;                /* parallel sketch branches W */
    int32_t tile_n;                  /* GEMM tile width (128 x tile_n tiles) */
    int32_t total_tiles;             /* tiles of the grouped GEMM launch */
    int32_t kernel_launches;         /* kernels per run */
    size_t operand_bytes;            /* sketched operands held */
    size_t workspace_bytes;          /* packing slots held */
    float tuned_ms;                  /* median run time of the choice when tuned, else 0 */
} os_batch_info;

OS_API os_status oversketch_batch_create(const os_problem *problems, int32_t count, os_dtype a_t,
                                         os_dtype b_t, os_dtype gemm_dtype, size_t workspace_limit,
                                         int32_t tune, void *stream, oversketch_batch_t *batch);
OS_API os_status oversketch_batch_run(oversketch_batch_t batch, void *stream);
OS_API os_status oversketch_batch_info(oversketch_batch_t batch, os_batch_info *info);
OS_API os_status oversketch_batch_destroy(oversketch_batch_t batch);

#ifdef __cplusplus
}
#endif
#endif /* OVERSKETCH_H */
