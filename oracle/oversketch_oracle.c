/*
 * OverSketch CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain C99, FP64 arithmetic, optional OpenMP over independent outputs.
 * Only tests/, the package's smoke check and bench.py's CPU-baseline leg may
 * load this library.  It shares no code, header, table or constant generator
 * with the CUDA path in paper_1811_02653_gb300/csrc/.
 *
 * What it computes (OverSketch, Gupta, Wang, Courtade, Ramchandran,
 * arXiv 1811.02653):
 *   - Count-sketch blocks S_1..S_{N+e} (Alg. 4, Sec. 4.1): every index i of
 *     the sketched dimension gets, per block j, a sign sigma_j(i) in {+1,-1}
 *     (step 1: "multiply by -1 with probability 1/2") and a bucket
 *     h_j(i) in [0,b) (step 2: "map to an integer uniformly at random",
 *     0-based here; the paper counts from 1).
 *   - The stacked sketch S = (S_1,...,S_{N+e}) of Eq. 3, applied UNSCALED: the
 *     1/N of Eq. 3 appears once, as 1/k with k = number of blocks kept, in
 *     the masked product.
 *   - A~ = A S and B~ = S^T B (Alg. 5 / Alg. 4 step 3: "add the columns that
 *     map to the same integer"), optionally with a per-index column scale
 *     (A diag(s) S, used for the interior-point Hessian of Sec. 5.2).
 *   - The adjoints used by the gradient: X -> X S_sel^T style gathers.
 *
 * Hash reading (the paper names no hash): splitmix64.
 *   gamma = 0x9E3779B97F4A7C15, mix64 = the splitmix64 output finaliser
 *   (Steele, Lea, Flood 2014; Vigna's public-domain splitmix64.c).
 *   key_j  = mix64(seed + (j+1)*gamma)            (mod 2^64)
 *   w      = mix64(key_j + (i+1)*gamma)
 *   h_j(i) = ((w >> 32) * b) >> 32               (multiply-shift range map)
 *   sigma_j(i) = (w & 1) ? -1 : +1
 * key_j is the (j+1)-th output of splitmix64 seeded with `seed`, and w is the
 * (i+1)-th output of splitmix64 seeded with key_j.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#define OSK_GAMMA 0x9E3779B97F4A7C15ULL

uint64_t osk_oracle_mix64(uint64_t z)
{
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ULL;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return z;
}

/* h[j*n + i] in [0,b), sigma[j*n + i] in {+1,-1}; P = N + e blocks. */
void osk_oracle_hash(int64_t n, int32_t b, int32_t P, uint64_t seed,
                     uint32_t *h, int8_t *sigma)
{
    for (int32_t j = 0; j < P; ++j) {
        uint64_t key = osk_oracle_mix64(seed + (uint64_t)(j + 1) * OSK_GAMMA);
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            uint64_t w = osk_oracle_mix64(key + (uint64_t)(i + 1) * OSK_GAMMA);
            h[(int64_t)j * n + i] = (uint32_t)(((w >> 32) * (uint64_t)b) >> 32);
            sigma[(int64_t)j * n + i] = (w & 1ULL) ? (int8_t)-1 : (int8_t)1;
        }
    }
}

/*
 * Left sketch, Alg. 4 step 3 applied to the rows of A for every block:
 *   At[r, j*b + h_j(i)] += sigma_j(i) * s_i * A[r, i]
 * A: m x n row-major with leading dimension lda.  At: m x (P*b) row-major,
 * overwritten.  col_scale: length n, or NULL for s_i = 1.
 * Summation order: i ascending inside every bucket.
 */
void osk_oracle_sketch_left(const double *A, int64_t m, int64_t n, int64_t lda,
                            const uint32_t *h, const int8_t *sigma,
                            int32_t b, int32_t P, const double *col_scale,
                            double *At)
{
    const int64_t z = (int64_t)P * b;
    #pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m; ++r) {
        double *out = At + r * z;
        const double *row = A + r * lda;
        for (int64_t c = 0; c < z; ++c) out[c] = 0.0;
        for (int32_t j = 0; j < P; ++j) {
            const uint32_t *hj = h + (int64_t)j * n;
            const int8_t *sj = sigma + (int64_t)j * n;
            double *outj = out + (int64_t)j * b;
            for (int64_t i = 0; i < n; ++i) {
                double v = row[i];
                if (col_scale) v *= col_scale[i];
                outj[hj[i]] += (double)sj[i] * v;
            }
        }
    }
}

/*
 * Right sketch, B~ = S^T B:
 *   Bt[j*b + h_j(i), c] += sigma_j(i) * B[i, c]
 * B: n x l row-major with leading dimension ldb.  Bt: (P*b) x l row-major,
 * overwritten.  Summation order: i ascending inside every bucket.
 */
void osk_oracle_sketch_right(const double *B, int64_t n, int64_t l, int64_t ldb,
                             const uint32_t *h, const int8_t *sigma,
                             int32_t b, int32_t P, double *Bt)
{
    const int64_t z = (int64_t)P * b;
    /* Columns c are independent outputs: split them across threads. */
    #pragma omp parallel
    {
        #pragma omp for schedule(static)
        for (int64_t q = 0; q < z; ++q)
            for (int64_t c = 0; c < l; ++c) Bt[q * l + c] = 0.0;
        #pragma omp for schedule(static)
        for (int64_t c0 = 0; c0 < l; c0 += 64) {
            int64_t c1 = c0 + 64 < l ? c0 + 64 : l;
            for (int32_t j = 0; j < P; ++j) {
                const uint32_t *hj = h + (int64_t)j * n;
                const int8_t *sj = sigma + (int64_t)j * n;
                for (int64_t i = 0; i < n; ++i) {
                    double *dst = Bt + ((int64_t)j * b + hj[i]) * l;
                    const double *src = B + i * ldb;
                    double s = (double)sj[i];
                    for (int64_t c = c0; c < c1; ++c) dst[c] += s * src[c];
                }
            }
        }
    }
}

/*
 * Adjoint of the left sketch restricted to the kept blocks (the gradient of
 * C with respect to the left operand, Eq. 3 read as a linear map):
 *   dX[r, i] = scale * sum_{j in mask, ascending} sigma_j(i) * T[r, j*b + h_j(i)]
 * T: m x (P*b) row-major (ldt).  dX: m x n row-major (ldx), overwritten.
 */
void osk_oracle_unsketch_cols(const double *T, int64_t m, int64_t ldt,
                              const uint32_t *h, const int8_t *sigma,
                              int64_t n, int32_t b, int32_t P, uint64_t mask,
                              double scale, double *dX, int64_t ldx)
{
    #pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m; ++r) {
        const double *trow = T + r * ldt;
        double *xrow = dX + r * ldx;
        for (int64_t i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int32_t j = 0; j < P; ++j) {
                if (!((mask >> j) & 1ULL)) continue;
                int64_t q = (int64_t)j * b + h[(int64_t)j * n + i];
                acc += (double)sigma[(int64_t)j * n + i] * trow[q];
            }
            xrow[i] = scale * acc;
        }
    }
}

/*
 * Adjoint of the right sketch restricted to the kept blocks:
 *   dG[i, c] = scale * sum_{j in mask, ascending} sigma_j(i) * U[j*b + h_j(i), c]
 * U: (P*b) x l row-major (ldu).  dG: n x l row-major (ldg), overwritten.
 */
void osk_oracle_unsketch_rows(const double *U, int64_t l, int64_t ldu,
                              const uint32_t *h, const int8_t *sigma,
                              int64_t n, int32_t b, int32_t P, uint64_t mask,
                              double scale, double *dG, int64_t ldg)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double *grow = dG + i * ldg;
        for (int64_t c = 0; c < l; ++c) grow[c] = 0.0;
        for (int32_t j = 0; j < P; ++j) {
            if (!((mask >> j) & 1ULL)) continue;
            int64_t q = (int64_t)j * b + h[(int64_t)j * n + i];
            double s = (double)sigma[(int64_t)j * n + i];
            const double *urow = U + q * ldu;
            for (int64_t c = 0; c < l; ++c) grow[c] += s * urow[c];
        }
        for (int64_t c = 0; c < l; ++c) grow[c] *= scale;
    }
}
