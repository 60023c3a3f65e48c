/*
 * Oracle: plain, slow CPU FP64 restatement of the atom-blocked sparse-matrix operations of a
 * linear-scaling density-matrix solver (Background: sparse storage keeps every operation
 * local; Development Priorities: density-matrix minimisation and overlap inversion, both in
 * linear-scaling time).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this file; it is
 * used by tests/, by __graft_entry__.smoke() and by bench.py's CPU-baseline leg.  It shares
 * no code, header or table with the CUDA library.
 *
 * Storage convention (the oracle's own): a pattern over n atoms is a CSR by atom row,
 * row_ptr[n+1] (int64), col[nnzb] (int32, ascending within a row); block b = (i, col[b])
 * holds nb[i]*nb[col[b]] doubles, row-major, at values + off[b], off[nnzb+1] (int64),
 * blocks stored back to back with no padding.
 *
 * Every loop is written in the order of its definition; no blocking or reordering.  Sums
 * that feed scalars (traces, dots, norms) use Neumaier's compensated summation, in block
 * order, so that the oracle's own rounding is far below every tolerance it is used for.
 * Parallelism: OpenMP over independent output atom rows only; each row's arithmetic is
 * sequential, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXB 32 /* largest orbital count per atom the oracle accepts */

/* Threads the oracle's parallel loops use. */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- pattern: P_R = {(i,j) : d_min(i,j)^2 < R^2} plus every (i,i), minimum image in an
 *      orthorhombic box ---- */

/* Minimum-image squared distance, evaluated as ((dx*dx + dy*dy) + dz*dz) with
 * d_c = (x_j - x_i) - box_c * rint((x_j - x_i) / box_c).  Compiled without FMA contraction. */
static double min_image_d2(const double *pos, const double *box, int i, int j)
{
    double d2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        double d = pos[3 * j + c] - pos[3 * i + c];
        d = d - box[c] * rint(d / box[c]);
        d2 = d2 + d * d;
    }
    return d2;
}

/* Brute force over all ordered pairs: number of j with d^2 < R^2, per row i. */
void orc_pattern_count(int n, const double *pos, const double *box, double range,
                       int64_t *row_count)
{
    const double r2 = range * range;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        int64_t c = 0;
        for (int j = 0; j < n; ++j)
            if (j == i || min_image_d2(pos, box, i, j) < r2)
                ++c;
        row_count[i] = c;
    }
}

/* Second pass: columns of each row in ascending j. */
void orc_pattern_fill(int n, const double *pos, const double *box, double range,
                      const int64_t *row_ptr, int32_t *col)
{
    const double r2 = range * range;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        int64_t w = row_ptr[i];
        for (int j = 0; j < n; ++j)
            if (j == i || min_image_d2(pos, box, i, j) < r2)
                col[w++] = j;
    }
}

/* Index of block (i, j) in a pattern, or -1: binary search in row i. */
static int64_t find_block(const int64_t *rp, const int32_t *col, int i, int j)
{
    int64_t lo = rp[i], hi = rp[i + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] < j)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < rp[i + 1] && col[lo] == j) ? lo : -1;
}

int64_t orc_find_block(const int64_t *rp, const int32_t *col, int i, int j)
{
    return find_block(rp, col, i, j);
}

/* ---- masked block product ---- */

/*
 * C_ij <- beta*C_ij + alpha * sum_k A_ik B_kj for every (i, j) in P_C, k ascending over the
 * stored blocks of row i of A for which (k, j) is stored in B.  This is the definition of
 * the product kept on C's pattern (the exact masked product).  With beta == 0 the old C is
 * not read.  rows == NULL computes every row; otherwise only the n_rows listed rows.
 */
int orc_bsmm(int n, const int32_t *nb,
             const int64_t *a_rp, const int32_t *a_col, const int64_t *a_off, const double *A,
             const int64_t *b_rp, const int32_t *b_col, const int64_t *b_off, const double *B,
             const int64_t *c_rp, const int32_t *c_col, const int64_t *c_off, double *C,
             double alpha, double beta, const int32_t *rows, int n_rows)
{
    for (int i = 0; i < n; ++i)
        if (nb[i] < 1 || nb[i] > ORC_MAXB)
            return 1;
    const int count = rows ? n_rows : n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < count; ++t) {
        const int i = rows ? rows[t] : t;
        const int ni = nb[i];
        double acc[ORC_MAXB * ORC_MAXB];
        for (int64_t c = c_rp[i]; c < c_rp[i + 1]; ++c) {
            const int j = c_col[c];
            const int nj = nb[j];
            for (int e = 0; e < ni * nj; ++e)
                acc[e] = 0.0;
            for (int64_t a = a_rp[i]; a < a_rp[i + 1]; ++a) {
                const int k = a_col[a];
                const int nk = nb[k];
                const int64_t b = find_block(b_rp, b_col, k, j);
                if (b < 0)
                    continue;
                const double *Ab = A + a_off[a];
                const double *Bb = B + b_off[b];
                for (int r = 0; r < ni; ++r)
                    for (int q = 0; q < nj; ++q)
                        for (int m = 0; m < nk; ++m)
                            acc[r * nj + q] += Ab[r * nk + m] * Bb[m * nj + q];
            }
            double *Cb = C + c_off[c];
            for (int e = 0; e < ni * nj; ++e)
                Cb[e] = (beta == 0.0) ? alpha * acc[e] : beta * Cb[e] + alpha * acc[e];
        }
    }
    return 0;
}

/* Number of (i, k, j) triplets of the masked product and their useful flop count, over
 * every row (rows == NULL) or the n_rows listed rows. */
void orc_triplet_count(int n, const int32_t *nb,
                       const int64_t *a_rp, const int32_t *a_col,
                       const int64_t *b_rp, const int32_t *b_col,
                       const int64_t *c_rp, const int32_t *c_col,
                       int64_t *triplets, double *flops, const int32_t *rows, int n_rows)
{
    int64_t t_all = 0;
    double f_all = 0.0;
    const int count = rows ? n_rows : n;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : t_all, f_all)
    for (int t = 0; t < count; ++t) {
        const int i = rows ? rows[t] : t;
        for (int64_t c = c_rp[i]; c < c_rp[i + 1]; ++c) {
            const int j = c_col[c];
            for (int64_t a = a_rp[i]; a < a_rp[i + 1]; ++a) {
                const int k = a_col[a];
                if (find_block(b_rp, b_col, k, j) >= 0) {
                    t_all += 1;
                    f_all += 2.0 * nb[i] * nb[k] * nb[j];
                }
            }
        }
    }
    *triplets = t_all;
    *flops = f_all;
}

/* ---- compensated sums ---- */

typedef struct {
    double s, c;
} nsum;

static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

/*
 * Tr(A.B) = sum over (i,j) in P_A of sum_{a,b} A_ij[a,b] * B_ji[b,a], B_ji looked up in P_B
 * (absent blocks contribute zero).  Rows are summed separately, then combined in row order.
 */
double orc_trace_prod(int n, const int32_t *nb,
                      const int64_t *a_rp, const int32_t *a_col, const int64_t *a_off,
                      const double *A,
                      const int64_t *b_rp, const int32_t *b_col, const int64_t *b_off,
                      const double *B)
{
    double *row_s = (double *)calloc((size_t)n, sizeof(double));
    double *row_c = (double *)calloc((size_t)n, sizeof(double));
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < n; ++i) {
        nsum acc = {0.0, 0.0};
        const int ni = nb[i];
        for (int64_t a = a_rp[i]; a < a_rp[i + 1]; ++a) {
            const int j = a_col[a];
            const int nj = nb[j];
            const int64_t b = find_block(b_rp, b_col, j, i);
            if (b < 0)
                continue;
            for (int r = 0; r < ni; ++r)
                for (int q = 0; q < nj; ++q)
                    nsum_add(&acc, A[a_off[a] + r * nj + q] * B[b_off[b] + q * ni + r]);
        }
        row_s[i] = acc.s;
        row_c[i] = acc.c;
    }
    nsum tot = {0.0, 0.0};
    for (int i = 0; i < n; ++i) {
        nsum_add(&tot, row_s[i]);
        nsum_add(&tot, row_c[i]);
    }
    free(row_s);
    free(row_c);
    return tot.s + tot.c;
}

/* Frobenius inner product <A, B> = sum over all stored values of A*B (same pattern). */
double orc_dot(int64_t n_values, const double *A, const double *B)
{
    nsum acc = {0.0, 0.0};
    for (int64_t e = 0; e < n_values; ++e)
        nsum_add(&acc, A[e] * B[e]);
    return acc.s + acc.c;
}

/* ||M - I||_F^2 over the stored blocks: the identity lives on the diagonal blocks only. */
double orc_frob2_minus_identity(int n, const int32_t *nb, const int64_t *rp,
                                const int32_t *col, const int64_t *off, const double *M)
{
    nsum acc = {0.0, 0.0};
    for (int i = 0; i < n; ++i)
        for (int64_t b = rp[i]; b < rp[i + 1]; ++b) {
            const int j = col[b];
            const int ni = nb[i], nj = nb[j];
            for (int r = 0; r < ni; ++r)
                for (int q = 0; q < nj; ++q) {
                    double v = M[off[b] + r * nj + q] - ((i == j && r == q) ? 1.0 : 0.0);
                    nsum_add(&acc, v * v);
                }
        }
    return acc.s + acc.c;
}

/*
 * dst_ij = src_ij (transpose == 0) or dst_ij = (src_ji)^T (transpose != 0) for every
 * (i, j) in P_dst; zero where the source block is not stored.
 */
void orc_gather(int n, const int32_t *nb,
                const int64_t *s_rp, const int32_t *s_col, const int64_t *s_off,
                const double *src,
                const int64_t *d_rp, const int32_t *d_col, const int64_t *d_off, double *dst,
                int transpose)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < n; ++i)
        for (int64_t b = d_rp[i]; b < d_rp[i + 1]; ++b) {
            const int j = d_col[b];
            const int ni = nb[i], nj = nb[j];
            const int64_t s = transpose ? find_block(s_rp, s_col, j, i)
                                        : find_block(s_rp, s_col, i, j);
            for (int r = 0; r < ni; ++r)
                for (int q = 0; q < nj; ++q) {
                    double v = 0.0;
                    if (s >= 0)
                        v = transpose ? src[s_off[s] + q * ni + r] : src[s_off[s] + r * nj + q];
                    dst[d_off[b] + r * nj + q] = v;
                }
        }
}

/*
 * Per scalar row a of the matrix: centre M_aa, absolute off-diagonal sum, absolute row sum.
 * (Gershgorin discs; the largest absolute row sum bounds the spectral radius.)
 */
void orc_row_sums(int n, const int32_t *nb, const int64_t *rp, const int32_t *col,
                  const int64_t *off, const double *M, double *centre, double *radius,
                  double *abs_sum)
{
    int64_t row0 = 0;
    for (int i = 0; i < n; ++i) {
        const int ni = nb[i];
        for (int r = 0; r < ni; ++r) {
            double c = 0.0, rad = 0.0, tot = 0.0;
            for (int64_t b = rp[i]; b < rp[i + 1]; ++b) {
                const int j = col[b];
                const int nj = nb[j];
                for (int q = 0; q < nj; ++q) {
                    double v = M[off[b] + r * nj + q];
                    tot += fabs(v);
                    if (i == j && r == q)
                        c = v;
                    else
                        rad += fabs(v);
                }
            }
            centre[row0 + r] = c;
            radius[row0 + r] = rad;
            abs_sum[row0 + r] = tot;
        }
        row0 += ni;
    }
}
