/*
 * Plain CPU oracle for the rank-profile-revealing PLUQ decomposition over Z/pZ
 * (Dumas, Pernet & Sultan, "Simultaneous computation of the row and column rank
 * profiles", arXiv 1301.4438).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file: only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg load it.  It shares no code, header, table or helper with
 * the CUDA path.
 *
 * Everything is exact arithmetic in [0, p) with 64-bit intermediate products
 * ((p-1)^2 < 2^62 for p < 2^31).  No blocking, fusion or reordering beyond the
 * textbook definitions: it is meant to be checked against the paper by eye.
 *
 * Contents
 *   oracle_rank_profile      rank profile matrix R by incremental row echelon
 *                            (definition of the row/column rank profile, Sec. 1;
 *                            R of every leading submatrix, Lemma 2 and its
 *                            corollaries, Sec. 4)
 *   oracle_canonical_order   the pivot order Algorithm 1 produces, as a function
 *                            of R (the four recursive calls of Algorithm 1 and
 *                            the final block permutations S and T, Sec. 2)
 *   oracle_pluq              P, Q from the order, then L and U by elimination
 *                            without pivoting on P^T A Q^T (output contract of
 *                            Algorithm 1)
 *   oracle_pluq_alg1         a second, literal reading of Algorithm 1 (quad
 *                            recursion with MM / TRSM / PermR / PermC and the
 *                            S, T block permutations), base cases as
 *                            order-preserving rotations
 *   oracle_matmul_sub        MM(C,A,B): C <- C - A B  (Sec. 2 subroutines)
 *   oracle_trsm_*            TRSM(L,B): B <- L^{-1} B, TRSM(B,U): B <- B U^{-1}
 *   oracle_check_pluq        reconstruction A == P [L;M][U V] Q and shape checks
 *   oracle_rref              reduced row echelon form (Gauss-Jordan); nullspace
 *                            bases and particular solutions are read off it
 *                            (uses of the decomposition listed in Sec. 1)
 *   oracle_determinant       determinant by elimination with row exchanges
 *   oracle_ple / oracle_cup  PLE and CUP decompositions from their definitions
 *                            (Sec. 1): elimination with prescribed pivot
 *                            positions, pivots taken from R in column (row) order
 *
 * Readings where the paper is ambiguous (all documented in the design notes):
 *   - base cases m = 1 / n = 1 bring the pivot to the front by a cyclic
 *     rotation, not a transposition, so the order of the other rows/columns is
 *     kept (a transposition breaks the rank profile property of Sec. 4);
 *   - for n = 1 the base case permutes rows (P), not columns;
 *   - the "PermR(D,Q2^T)" and "PermR(V1,Q3^T)" steps are column permutations;
 *   - T uses the column split floor(n/2);
 *   - non-pivot rows (columns) keep their increasing order in P (Q).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- field -- */

static uint32_t add_mod(uint32_t a, uint32_t b, uint32_t p)
{
    uint64_t s = (uint64_t)a + b;
    return (uint32_t)(s >= p ? s - p : s);
}

static uint32_t sub_mod(uint32_t a, uint32_t b, uint32_t p)
{
    return a >= b ? a - b : (uint32_t)((uint64_t)a + p - b);
}

static uint32_t mul_mod(uint32_t a, uint32_t b, uint32_t p)
{
    return (uint32_t)(((uint64_t)a * b) % p);
}

/* Inverse of a (nonzero mod p) by the extended Euclidean algorithm. */
static uint32_t inv_mod(uint32_t a, uint32_t p)
{
    int64_t r0 = p, r1 = a % p, s0 = 0, s1 = 1;
    while (r1 != 0) {
        int64_t q = r0 / r1, t;
        t = r0 - q * r1; r0 = r1; r1 = t;
        t = s0 - q * s1; s0 = s1; s1 = t;
    }
    /* r0 == gcd == 1 for a field element a != 0 */
    s0 %= (int64_t)p;
    if (s0 < 0) s0 += p;
    return (uint32_t)s0;
}

int oracle_is_prime(uint32_t p)
{
    if (p < 2) return 0;
    for (uint64_t d = 2; d * d <= p; ++d)
        if (p % d == 0) return 0;
    return 1;
}

/* Status codes mirror the meaning (not the code) of the library's. */
#define O_OK 0
#define O_EINVAL (-1)
#define O_ENOTPRIME (-2)
#define O_ERANGE (-3)
#define O_ENOMEM (-4)
#define O_EINTERNAL (-7)

static int validate(const uint32_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p)
{
    if (m < 0 || n < 0) return O_EINVAL;
    if (m > 0 && n > 0 && (A == NULL || lda < n)) return O_EINVAL;
    if (p >= 0x80000000u || !oracle_is_prime(p)) return O_ENOTPRIME;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j)
            if (A[i * lda + j] >= p) return O_ERANGE;
    return O_OK;
}

/* ------------------------------------------------- rank profile matrix -- */
/*
 * R[k][t] = rho(k+1,t+1) - rho(k,t+1) - rho(k+1,t) + rho(k,t), rho(k,t) the
 * rank of the leading k x t submatrix.  Row k of A carries a one of R iff it is
 * independent of rows 0..k-1; its column is the first t such that A[k,0..t] is
 * independent of A[0..k-1, 0..t].  Incremental row echelon finds exactly that:
 * keep a basis of rows in echelon form (leading coefficient one, zeros left of
 * it) indexed by leading column, reduce row k from left to right, and the first
 * nonzero column without a basis row is its pivot column.
 *
 * col_of_row[k] = column of the one in row k of R, or -1.  Returns r, or a
 * negative status.
 */
int64_t oracle_rank_profile(const uint32_t *A, int64_t m, int64_t n, int64_t lda,
                            uint32_t p, int32_t *col_of_row)
{
    int st = validate(A, m, n, lda, p);
    if (st != O_OK) return st;
    for (int64_t k = 0; k < m; ++k) col_of_row[k] = -1;
    if (m == 0 || n == 0) return 0;

    int64_t cap = m < n ? m : n;
    uint32_t *basis = (uint32_t *)malloc((size_t)cap * (size_t)n * sizeof(uint32_t));
    int64_t *lead = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    uint32_t *row = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!basis || !lead || !row) { free(basis); free(lead); free(row); return O_ENOMEM; }
    for (int64_t c = 0; c < n; ++c) lead[c] = -1;

    int64_t r = 0;
    for (int64_t k = 0; k < m; ++k) {
        memcpy(row, A + k * lda, (size_t)n * sizeof(uint32_t));
        for (int64_t c = 0; c < n; ++c) {
            if (row[c] == 0) continue;
            if (lead[c] >= 0) {
                /* basis row has leading coefficient 1 at column c and zeros left of it */
                const uint32_t *b = basis + lead[c] * n;
                uint32_t f = row[c];
                for (int64_t j = c; j < n; ++j)
                    row[j] = sub_mod(row[j], mul_mod(f, b[j], p), p);
            } else {
                uint32_t inv = inv_mod(row[c], p);
                uint32_t *b = basis + r * n;
                for (int64_t j = 0; j < n; ++j) b[j] = mul_mod(row[j], inv, p);
                lead[c] = r;
                col_of_row[k] = (int32_t)c;
                ++r;
                break;
            }
        }
    }
    free(basis); free(lead); free(row);
    return r;
}

/* ------------------------------------------------------ canonical order -- */
/*
 * The order in which Algorithm 1 discovers the ones of R.  A call on the rows
 * `rows` and columns `cols` (increasing original indices) splits them at
 * floor(|rows|/2), floor(|cols|/2) and recurses, in this order, on
 *   A1 : top rows            x left columns
 *   F  : top rows not pivots of A1   x right columns
 *   G  : bottom rows         x left columns not pivots of A1
 *   R  : bottom rows not pivots of G x right columns not pivots of F
 * and its pivots are those of A1, F, G, R concatenated (P and Q composed with
 * the block permutations S and T).  A call with one row or one column returns
 * the (at most one) one of R inside it.  This relies on each call's rank
 * profile matrix being R restricted to its rows and columns; agreement with the
 * literal Algorithm 1 below is what the tests check.
 */
typedef struct {
    const int32_t *col_of_row; /* m */
    const int32_t *row_of_col; /* n */
    int32_t *out_r, *out_c;
    int64_t count;
} order_ctx;

static int in_sorted(const int32_t *v, int64_t len, int32_t x)
{
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (v[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo < len && v[lo] == x;
}

/* out = v minus the entries marked in `mark` (by value); returns new length */
static int64_t remove_marked(const int32_t *v, int64_t len, const unsigned char *mark, int32_t *out)
{
    int64_t t = 0;
    for (int64_t i = 0; i < len; ++i)
        if (!mark[v[i]]) out[t++] = v[i];
    return t;
}

static int order_rec(order_ctx *cx, const int32_t *rows, int64_t nr,
                     const int32_t *cols, int64_t nc,
                     unsigned char *rmark, unsigned char *cmark)
{
    if (nr == 0 || nc == 0) return O_OK;
    if (nr == 1) {
        int32_t c = cx->col_of_row[rows[0]];
        if (c >= 0 && in_sorted(cols, nc, c)) {
            cx->out_r[cx->count] = rows[0]; cx->out_c[cx->count] = c; ++cx->count;
        }
        return O_OK;
    }
    if (nc == 1) {
        int32_t rr = cx->row_of_col[cols[0]];
        if (rr >= 0 && in_sorted(rows, nr, rr)) {
            cx->out_r[cx->count] = rr; cx->out_c[cx->count] = cols[0]; ++cx->count;
        }
        return O_OK;
    }
    int64_t k = nr / 2, h = nc / 2;
    const int32_t *rt = rows, *rb = rows + k, *cl = cols, *cr = cols + h;
    int64_t nrt = k, nrb = nr - k, ncl = h, ncr = nc - h;

    int32_t *buf = (int32_t *)malloc((size_t)(nr + nc) * 2 * sizeof(int32_t));
    if (!buf) return O_ENOMEM;
    int32_t *rt2 = buf, *cl2 = buf + nr, *rb2 = buf + nr + nc, *cr2 = buf + 2 * nr + nc;
    int st;

    int64_t s1 = cx->count;
    if ((st = order_rec(cx, rt, nrt, cl, ncl, rmark, cmark))) { free(buf); return st; }
    int64_t e1 = cx->count;
    for (int64_t t = s1; t < e1; ++t) { rmark[cx->out_r[t]] = 1; cmark[cx->out_c[t]] = 1; }
    int64_t nrt2 = remove_marked(rt, nrt, rmark, rt2);
    int64_t ncl2 = remove_marked(cl, ncl, cmark, cl2);
    for (int64_t t = s1; t < e1; ++t) { rmark[cx->out_r[t]] = 0; cmark[cx->out_c[t]] = 0; }

    int64_t s2 = cx->count;
    if ((st = order_rec(cx, rt2, nrt2, cr, ncr, rmark, cmark))) { free(buf); return st; } /* F */
    int64_t e2 = cx->count;
    int64_t s3 = cx->count;
    if ((st = order_rec(cx, rb, nrb, cl2, ncl2, rmark, cmark))) { free(buf); return st; } /* G */
    int64_t e3 = cx->count;

    for (int64_t t = s3; t < e3; ++t) rmark[cx->out_r[t]] = 1;
    for (int64_t t = s2; t < e2; ++t) cmark[cx->out_c[t]] = 1;
    int64_t nrb2 = remove_marked(rb, nrb, rmark, rb2);
    int64_t ncr2 = remove_marked(cr, ncr, cmark, cr2);
    for (int64_t t = s3; t < e3; ++t) rmark[cx->out_r[t]] = 0;
    for (int64_t t = s2; t < e2; ++t) cmark[cx->out_c[t]] = 0;

    st = order_rec(cx, rb2, nrb2, cr2, ncr2, rmark, cmark); /* R */
    free(buf);
    return st;
}

/* piv_rows/piv_cols (length r) receive the ones of R in Algorithm 1's order. */
int oracle_canonical_order(int64_t m, int64_t n, const int32_t *col_of_row,
                           int32_t *piv_rows, int32_t *piv_cols, int64_t *r_out)
{
    if (m < 0 || n < 0) return O_EINVAL;
    int32_t *rows = (int32_t *)malloc((size_t)(m + 1) * sizeof(int32_t));
    int32_t *cols = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t *row_of_col = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    unsigned char *rmark = (unsigned char *)calloc((size_t)m + 1, 1);
    unsigned char *cmark = (unsigned char *)calloc((size_t)n + 1, 1);
    if (!rows || !cols || !row_of_col || !rmark || !cmark) {
        free(rows); free(cols); free(row_of_col); free(rmark); free(cmark);
        return O_ENOMEM;
    }
    for (int64_t i = 0; i < m; ++i) rows[i] = (int32_t)i;
    for (int64_t j = 0; j < n; ++j) { cols[j] = (int32_t)j; row_of_col[j] = -1; }
    for (int64_t i = 0; i < m; ++i)
        if (col_of_row[i] >= 0) {
            if (col_of_row[i] >= n || row_of_col[col_of_row[i]] >= 0) {
                free(rows); free(cols); free(row_of_col); free(rmark); free(cmark);
                return O_EINVAL; /* not a partial permutation */
            }
            row_of_col[col_of_row[i]] = (int32_t)i;
        }
    order_ctx cx = {col_of_row, row_of_col, piv_rows, piv_cols, 0};
    int st = order_rec(&cx, rows, m, cols, n, rmark, cmark);
    *r_out = cx.count;
    free(rows); free(cols); free(row_of_col); free(rmark); free(cmark);
    return st;
}

/* ----------------------------------------------------------------- PLUQ -- */
/*
 * Output contract of Algorithm 1: A = P [L;M] [U V] Q with L unit lower r x r,
 * U upper r x r, stored packed as [L\U V; M 0] (m x n, row stride ld_lu).
 * perm_p[i] = original row placed at packed row i (P[perm_p[i], i] = 1);
 * perm_q[j] = original column placed at packed column j (Q[j, perm_q[j]] = 1).
 * Pivots come in the canonical order, then non-pivot rows / columns increasing.
 * Given P and Q, elimination without pivoting on P^T A Q^T is the unique
 * packed factorisation (the leading r x r block has a unique LU with unit L).
 */
int oracle_pluq(const uint32_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                uint32_t *LU, int64_t ld_lu, int32_t *perm_p, int32_t *perm_q,
                int64_t *rank)
{
    int st = validate(A, m, n, lda, p);
    if (st != O_OK) return st;
    if (m > 0 && n > 0 && ld_lu < n) return O_EINVAL;
    for (int64_t i = 0; i < m; ++i) perm_p[i] = (int32_t)i;
    for (int64_t j = 0; j < n; ++j) perm_q[j] = (int32_t)j;
    *rank = 0;
    if (m == 0 || n == 0) return O_OK;

    int32_t *col_of_row = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    int64_t cap = m < n ? m : n;
    int32_t *pr = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    int32_t *pc = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    unsigned char *used_r = (unsigned char *)calloc((size_t)m, 1);
    unsigned char *used_c = (unsigned char *)calloc((size_t)n, 1);
    if (!col_of_row || !pr || !pc || !used_r || !used_c) { st = O_ENOMEM; goto done; }

    int64_t r = oracle_rank_profile(A, m, n, lda, p, col_of_row);
    if (r < 0) { st = (int)r; goto done; }
    int64_t r2 = 0;
    st = oracle_canonical_order(m, n, col_of_row, pr, pc, &r2);
    if (st != O_OK) goto done;
    if (r2 != r) { st = O_EINTERNAL; goto done; }

    /* P, Q vectors: pivots in canonical order, then the rest increasing */
    for (int64_t t = 0; t < r; ++t) {
        perm_p[t] = pr[t]; used_r[pr[t]] = 1;
        perm_q[t] = pc[t]; used_c[pc[t]] = 1;
    }
    int64_t t = r;
    for (int64_t i = 0; i < m; ++i) if (!used_r[i]) perm_p[t++] = (int32_t)i;
    t = r;
    for (int64_t j = 0; j < n; ++j) if (!used_c[j]) perm_q[t++] = (int32_t)j;

    /* X = P^T A Q^T */
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j)
            LU[i * ld_lu + j] = A[(int64_t)perm_p[i] * lda + perm_q[j]];

    /* elimination without pivoting over the r leading pivots */
    for (int64_t k = 0; k < r; ++k) {
        uint32_t piv = LU[k * ld_lu + k];
        if (piv == 0) { st = O_EINTERNAL; goto done; }
        uint32_t inv = inv_mod(piv, p);
        /* rows below the pivot are independent of one another within step k */
#pragma omp parallel for schedule(static) if ((m - k) * (n - k) > (1 << 16))
        for (int64_t i = k + 1; i < m; ++i) {
            uint32_t *Xi = LU + i * ld_lu;
            const uint32_t *Xk = LU + k * ld_lu;
            uint32_t l = mul_mod(Xi[k], inv, p);
            Xi[k] = l;
            if (l == 0) continue;
            for (int64_t j = k + 1; j < n; ++j)
                Xi[j] = sub_mod(Xi[j], mul_mod(l, Xk[j], p), p);
        }
    }
    /* the Schur complement left after r pivots must vanish */
    for (int64_t i = r; i < m; ++i)
        for (int64_t j = r; j < n; ++j)
            if (LU[i * ld_lu + j] != 0) { st = O_EINTERNAL; goto done; }
    *rank = r;
    st = O_OK;
done:
    free(col_of_row); free(pr); free(pc); free(used_r); free(used_c);
    return st;
}

/* ------------------------------------------------ BLAS-like subroutines -- */

/* MM(C, A, B): C <- C - A B, A M x K, B K x N, all row-major with strides. */
void oracle_matmul_sub(uint32_t *C, int64_t ldc, const uint32_t *A, int64_t lda,
                       const uint32_t *B, int64_t ldb, int64_t M, int64_t N,
                       int64_t K, uint32_t p)
{
    for (int64_t i = 0; i < M; ++i)
        for (int64_t j = 0; j < N; ++j) {
            uint32_t s = 0;
            for (int64_t l = 0; l < K; ++l)
                s = add_mod(s, mul_mod(A[i * lda + l], B[l * ldb + j], p), p);
            C[i * ldc + j] = sub_mod(C[i * ldc + j], s, p);
        }
}

/* TRSM(L, B): B <- L^{-1} B, L r x r unit lower triangular (diagonal not read). */
void oracle_trsm_left_lower_unit(const uint32_t *L, int64_t ldl, uint32_t *B,
                                 int64_t ldb, int64_t r, int64_t N, uint32_t p)
{
    for (int64_t i = 0; i < r; ++i)
        for (int64_t l = 0; l < i; ++l) {
            uint32_t f = L[i * ldl + l];
            if (f == 0) continue;
            for (int64_t j = 0; j < N; ++j)
                B[i * ldb + j] = sub_mod(B[i * ldb + j], mul_mod(f, B[l * ldb + j], p), p);
        }
}

/* TRSM(B, U): B <- B U^{-1}, U r x r upper triangular with nonzero diagonal. */
void oracle_trsm_right_upper(const uint32_t *U, int64_t ldu, uint32_t *B,
                             int64_t ldb, int64_t M, int64_t r, uint32_t p)
{
    for (int64_t j = 0; j < r; ++j) {
        uint32_t inv = inv_mod(U[j * ldu + j], p);
        for (int64_t i = 0; i < M; ++i) {
            uint32_t s = B[i * ldb + j];
            for (int64_t l = 0; l < j; ++l)
                s = sub_mod(s, mul_mod(B[i * ldb + l], U[l * ldu + j], p), p);
            B[i * ldb + j] = mul_mod(s, inv, p);
        }
    }
}

/* -------------------------------------------- literal Algorithm 1 (2nd) -- */

typedef struct { uint32_t p; int err; } a1ctx;

/* rows [r0, r0+cnt) of the block, columns [c0, c1): new row i = old row perm[i] */
static void perm_rows(uint32_t *A, int64_t lda, int64_t r0, int64_t cnt,
                      int64_t c0, int64_t c1, const int32_t *perm, a1ctx *cx)
{
    if (cnt <= 0 || c1 <= c0) return;
    uint32_t *tmp = (uint32_t *)malloc((size_t)cnt * (size_t)(c1 - c0) * sizeof(uint32_t));
    if (!tmp) { cx->err = O_ENOMEM; return; }
    for (int64_t i = 0; i < cnt; ++i)
        for (int64_t j = c0; j < c1; ++j)
            tmp[i * (c1 - c0) + (j - c0)] = A[(r0 + perm[i]) * lda + j];
    for (int64_t i = 0; i < cnt; ++i)
        for (int64_t j = c0; j < c1; ++j)
            A[(r0 + i) * lda + j] = tmp[i * (c1 - c0) + (j - c0)];
    free(tmp);
}

/* columns [c0, c0+cnt), rows [r0, r1): new column j = old column perm[j] */
static void perm_cols(uint32_t *A, int64_t lda, int64_t c0, int64_t cnt,
                      int64_t r0, int64_t r1, const int32_t *perm, a1ctx *cx)
{
    if (cnt <= 0 || r1 <= r0) return;
    uint32_t *tmp = (uint32_t *)malloc((size_t)cnt * sizeof(uint32_t));
    if (!tmp) { cx->err = O_ENOMEM; return; }
    for (int64_t i = r0; i < r1; ++i) {
        for (int64_t j = 0; j < cnt; ++j) tmp[j] = A[i * lda + c0 + perm[j]];
        for (int64_t j = 0; j < cnt; ++j) A[i * lda + c0 + j] = tmp[j];
    }
    free(tmp);
}

static int64_t alg1(uint32_t *A, int64_t m, int64_t n, int64_t lda,
                    int32_t *P, int32_t *Q, a1ctx *cx)
{
    const uint32_t p = cx->p;
    for (int64_t i = 0; i < m; ++i) P[i] = (int32_t)i;
    for (int64_t j = 0; j < n; ++j) Q[j] = (int32_t)j;
    if (m == 0 || n == 0 || cx->err) return 0;

    if (m == 1) { /* base case: first nonzero of the row, rotated to the front */
        int64_t i = 0;
        while (i < n && A[i] == 0) ++i;
        if (i == n) return 0;
        uint32_t v = A[i];
        for (int64_t j = i; j > 0; --j) { A[j] = A[j - 1]; Q[j] = Q[j - 1]; }
        A[0] = v; Q[0] = (int32_t)i;
        return 1;
    }
    if (n == 1) { /* base case: first nonzero of the column rotated to the top; scale below */
        int64_t i = 0;
        while (i < m && A[i * lda] == 0) ++i;
        if (i == m) return 0;
        uint32_t v = A[i * lda];
        for (int64_t j = i; j > 0; --j) { A[j * lda] = A[(j - 1) * lda]; P[j] = P[j - 1]; }
        A[0] = v; P[0] = (int32_t)i;
        uint32_t inv = inv_mod(v, p);
        for (int64_t j = i + 1; j < m; ++j) A[j * lda] = mul_mod(A[j * lda], inv, p);
        return 1;
    }

    const int64_t k = m / 2, h = n / 2;
    int32_t *buf = (int32_t *)malloc((size_t)(2 * m + 2 * n) * sizeof(int32_t) * 2);
    uint32_t *Icopy = NULL;
    if (!buf) { cx->err = O_ENOMEM; return 0; }
    int32_t *P1 = buf, *P2 = P1 + m, *P3 = P2 + m, *P4 = P3 + m;
    int32_t *Q1 = P4 + m, *Q2 = Q1 + n, *Q3 = Q2 + n, *Q4 = Q3 + n;

    /* A1 = PLUQ of the leading k x h block */
    int64_t r1 = alg1(A, k, h, lda, P1, Q1, cx);
    /* [B1;B2] <- P1^T A2 ; [C1 C2] <- A3 Q1^T */
    perm_rows(A, lda, 0, k, h, n, P1, cx);
    perm_cols(A, lda, 0, h, k, m, Q1, cx);
    /* D <- L1^{-1} B1 ; E <- C1 U1^{-1} */
    oracle_trsm_left_lower_unit(A, lda, A + h, lda, r1, n - h, p);
    oracle_trsm_right_upper(A, lda, A + k * lda, lda, m - k, r1, p);
    /* F <- B2 - M1 D ; G <- C2 - E V1 ; H <- A4 - E D */
    oracle_matmul_sub(A + r1 * lda + h, lda, A + r1 * lda, lda, A + h, lda, k - r1, n - h, r1, p);
    oracle_matmul_sub(A + k * lda + r1, lda, A + k * lda, lda, A + r1, lda, m - k, h - r1, r1, p);
    oracle_matmul_sub(A + k * lda + h, lda, A + k * lda, lda, A + h, lda, m - k, n - h, r1, p);
    /* F = PLUQ(F), G = PLUQ(G) */
    int64_t r2 = alg1(A + r1 * lda + h, k - r1, n - h, lda, P2, Q2, cx);
    int64_t r3 = alg1(A + k * lda + r1, m - k, h - r1, lda, P3, Q3, cx);
    /* H <- P3^T H Q2^T ; E <- P3^T E ; M1 <- P2^T M1 ; D <- D Q2^T ; V1 <- V1 Q3^T */
    perm_rows(A, lda, k, m - k, h, n, P3, cx);
    perm_cols(A, lda, h, n - h, k, m, Q2, cx);
    perm_rows(A, lda, k, m - k, 0, r1, P3, cx);
    perm_rows(A, lda, r1, k - r1, 0, r1, P2, cx);
    perm_cols(A, lda, h, n - h, 0, r1, Q2, cx);
    perm_cols(A, lda, r1, h - r1, 0, r1, Q3, cx);

    uint32_t *U2 = A + r1 * lda + h;          /* r2 x r2, upper */
    uint32_t *V2 = A + r1 * lda + h + r2;     /* r2 x (n-h-r2) */
    uint32_t *L3 = A + k * lda + r1;          /* r3 x r3, unit lower */
    uint32_t *M3 = A + (k + r3) * lda + r1;   /* (m-k-r3) x r3 */
    uint32_t *H1 = A + k * lda + h;           /* r3 x r2 */
    uint32_t *H2 = A + k * lda + h + r2;      /* r3 x (n-h-r2) */
    uint32_t *H3 = A + (k + r3) * lda + h;    /* (m-k-r3) x r2 */
    uint32_t *H4 = A + (k + r3) * lda + h + r2;
    /* I <- H1 U2^{-1} ; J <- L3^{-1} I (kept apart: I stays in place) */
    oracle_trsm_right_upper(U2, lda, H1, lda, r3, r2, p);
    if (r3 > 0 && r2 > 0) {
        Icopy = (uint32_t *)malloc((size_t)r3 * (size_t)r2 * sizeof(uint32_t));
        if (!Icopy) { cx->err = O_ENOMEM; free(buf); return 0; }
        for (int64_t i = 0; i < r3; ++i)
            for (int64_t j = 0; j < r2; ++j) Icopy[i * r2 + j] = H1[i * lda + j];
        oracle_trsm_left_lower_unit(L3, lda, Icopy, r2, r3, r2, p); /* J */
    }
    /* K <- H3 U2^{-1} ; N <- L3^{-1} H2 ; O <- N - J V2 ; R <- H4 - K V2 - M3 O */
    oracle_trsm_right_upper(U2, lda, H3, lda, m - k - r3, r2, p);
    oracle_trsm_left_lower_unit(L3, lda, H2, lda, r3, n - h - r2, p);
    if (Icopy) oracle_matmul_sub(H2, lda, Icopy, r2, V2, lda, r3, n - h - r2, r2, p);
    oracle_matmul_sub(H4, lda, H3, lda, V2, lda, m - k - r3, n - h - r2, r2, p);
    oracle_matmul_sub(H4, lda, M3, lda, H2, lda, m - k - r3, n - h - r2, r3, p);
    free(Icopy);
    /* R = PLUQ(R) */
    int64_t r4 = alg1(H4, m - k - r3, n - h - r2, lda, P4, Q4, cx);
    /* [E2 M3 0 K] <- P4^T [..] ; [D2;V2;0;O] <- [..] Q4^T */
    perm_rows(A, lda, k + r3, m - k - r3, 0, h + r2, P4, cx);
    perm_cols(A, lda, h + r2, n - h - r2, 0, k + r3, Q4, cx);

    /* S and T as index maps: new row i = old row s[i], new column j = old column t[j] */
    int32_t *s = (int32_t *)malloc((size_t)(m + n) * sizeof(int32_t));
    if (!s) { cx->err = O_ENOMEM; free(buf); return 0; }
    int32_t *t = s + m;
    int64_t a = 0;
    for (int64_t i = 0; i < r1 + r2; ++i) s[a++] = (int32_t)i;
    for (int64_t i = 0; i < r3 + r4; ++i) s[a++] = (int32_t)(k + i);
    for (int64_t i = r1 + r2; i < k; ++i) s[a++] = (int32_t)i;
    for (int64_t i = k + r3 + r4; i < m; ++i) s[a++] = (int32_t)i;
    a = 0;
    for (int64_t j = 0; j < r1; ++j) t[a++] = (int32_t)j;
    for (int64_t j = 0; j < r2; ++j) t[a++] = (int32_t)(h + j);
    for (int64_t j = 0; j < r3; ++j) t[a++] = (int32_t)(r1 + j);
    for (int64_t j = 0; j < r4; ++j) t[a++] = (int32_t)(h + r2 + j);
    for (int64_t j = r1 + r3; j < h; ++j) t[a++] = (int32_t)j;
    for (int64_t j = h + r2 + r4; j < n; ++j) t[a++] = (int32_t)j;

    /* P = Diag(P1 diag(I,P2), P3 diag(I,P4)) S ; Q = T Diag(diag(I,Q3) Q1, diag(I,Q4) Q2) */
    int32_t *dp = (int32_t *)malloc((size_t)(m + n) * sizeof(int32_t));
    if (!dp) { cx->err = O_ENOMEM; free(s); free(buf); return 0; }
    int32_t *dq = dp + m;
    for (int64_t i = 0; i < k; ++i) dp[i] = i < r1 ? P1[i] : P1[r1 + P2[i - r1]];
    for (int64_t i = 0; i < m - k; ++i) dp[k + i] = (int32_t)k + (i < r3 ? P3[i] : P3[r3 + P4[i - r3]]);
    for (int64_t j = 0; j < h; ++j) dq[j] = j < r1 ? Q1[j] : Q1[r1 + Q3[j - r1]];
    for (int64_t j = 0; j < n - h; ++j) dq[h + j] = (int32_t)h + (j < r2 ? Q2[j] : Q2[r2 + Q4[j - r2]]);
    for (int64_t i = 0; i < m; ++i) P[i] = dp[s[i]];
    for (int64_t j = 0; j < n; ++j) Q[j] = dq[t[j]];

    /* A <- S^T A T^T */
    uint32_t *tmp = (uint32_t *)malloc((size_t)m * (size_t)n * sizeof(uint32_t));
    if (!tmp) { cx->err = O_ENOMEM; free(dp); free(s); free(buf); return 0; }
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) tmp[i * n + j] = A[(int64_t)s[i] * lda + t[j]];
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) A[i * lda + j] = tmp[i * n + j];
    free(tmp); free(dp); free(s); free(buf);
    return r1 + r2 + r3 + r4;
}

int oracle_pluq_alg1(uint32_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                     int32_t *perm_p, int32_t *perm_q, int64_t *rank)
{
    int st = validate(A, m, n, lda, p);
    if (st != O_OK) return st;
    a1ctx cx = {p, O_OK};
    *rank = alg1(A, m, n, lda, perm_p, perm_q, &cx);
    return cx.err;
}

/* ------------------------------------------------------------- checks -- */
/*
 * Returns 0 iff LU (packed, ld_lu) with perm_p, perm_q, r satisfies the output
 * contract of Algorithm 1 for A: L unit lower (diagonal implicit), U upper with
 * nonzero diagonal, the trailing (m-r) x (n-r) block zero, perm_p / perm_q
 * permutations, and A[perm_p[i]][perm_q[j]] == ([L;M][U V])[i][j].
 */
int oracle_check_pluq(const uint32_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                      const uint32_t *LU, int64_t ld_lu, const int32_t *perm_p,
                      const int32_t *perm_q, int64_t r)
{
    if (r < 0 || r > m || r > n) return 1;
    unsigned char *seen = (unsigned char *)calloc((size_t)(m > n ? m : n) + 1, 1);
    if (!seen) return O_ENOMEM;
    for (int64_t i = 0; i < m; ++i) {
        if (perm_p[i] < 0 || perm_p[i] >= m || seen[perm_p[i]]) { free(seen); return 2; }
        seen[perm_p[i]] = 1;
    }
    memset(seen, 0, (size_t)(m > n ? m : n) + 1);
    for (int64_t j = 0; j < n; ++j) {
        if (perm_q[j] < 0 || perm_q[j] >= n || seen[perm_q[j]]) { free(seen); return 3; }
        seen[perm_q[j]] = 1;
    }
    free(seen);
    for (int64_t k = 0; k < r; ++k)
        if (LU[k * ld_lu + k] == 0) return 4;
    for (int64_t i = r; i < m; ++i)
        for (int64_t j = r; j < n; ++j)
            if (LU[i * ld_lu + j] != 0) return 5;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) {
            /* ([L;M] [U V])[i][j] = sum_{l < min(i+1, r)} Lfull[i][l] Ufull[l][j] */
            uint32_t s = 0;
            int64_t lim = i < r ? i : r;             /* strictly-lower part of row i */
            for (int64_t l = 0; l < lim; ++l)
                if (l <= j) s = add_mod(s, mul_mod(LU[i * ld_lu + l], LU[l * ld_lu + j], p), p);
            if (i < r && i <= j) s = add_mod(s, LU[i * ld_lu + j], p); /* unit diagonal of L */
            if (s != A[(int64_t)perm_p[i] * lda + perm_q[j]]) return 6;
        }
    return 0;
}

/* ------------------------------------------ uses of the decomposition -- */
/*
 * The introduction (Sec. 1) lists what a triangular decomposition is used
 * for: solving linear systems, the rank, the determinant, the nullspace and
 * the rank profiles.  The oracle computes the first, third and fourth from
 * their textbook definitions, independently of any PLUQ:
 *
 * oracle_rref: reduced row echelon form by Gauss-Jordan elimination, in place
 * on the m x n block A.  Pivots are searched column by column among the first
 * npiv columns only (the row operations still act on all n columns, so the
 * trailing n - npiv columns carry a right-hand side along).  In column c the
 * first row at or below the current one with a nonzero entry is swapped up,
 * scaled to a leading one, and column c is cleared in every other row.
 * piv_col[k] = column of the k-th leading one (increasing).  Returns the
 * number of pivots, or a negative status.
 *
 * The pivot columns of the RREF are the column rank profile (each is the
 * first column independent of those before it), so the kernel basis whose
 * restriction to the non-pivot coordinates is the identity, and the solution
 * whose non-pivot coordinates are zero, are unique and read off the RREF.
 */
int64_t oracle_rref(uint32_t *A, int64_t m, int64_t n, int64_t lda, int64_t npiv, uint32_t p,
                    int32_t *piv_col)
{
    int st = validate(A, m, n, lda, p);
    if (st != O_OK) return st;
    if (npiv < 0 || npiv > n) return O_EINVAL;
    int64_t k = 0;
    for (int64_t c = 0; c < npiv && k < m; ++c) {
        int64_t s = -1;
        for (int64_t i = k; i < m; ++i)
            if (A[i * lda + c] != 0) { s = i; break; }
        if (s < 0) continue;
        if (s != k)
            for (int64_t j = 0; j < n; ++j) {
                uint32_t t = A[s * lda + j];
                A[s * lda + j] = A[k * lda + j];
                A[k * lda + j] = t;
            }
        uint32_t inv = inv_mod(A[k * lda + c], p);
        for (int64_t j = 0; j < n; ++j) A[k * lda + j] = mul_mod(A[k * lda + j], inv, p);
        for (int64_t i = 0; i < m; ++i) {
            if (i == k || A[i * lda + c] == 0) continue;
            uint32_t f = A[i * lda + c];
            for (int64_t j = 0; j < n; ++j)
                A[i * lda + j] = sub_mod(A[i * lda + j], mul_mod(f, A[k * lda + j], p), p);
        }
        piv_col[k++] = (int32_t)c;
    }
    return k;
}

/*
 * Determinant of the n x n matrix A by Gaussian elimination with row
 * exchanges: the product of the pivots, negated once per exchange; zero when
 * a column has no pivot.  The 0 x 0 determinant is 1.  Returns a status.
 */
int oracle_determinant(const uint32_t *A, int64_t n, int64_t lda, uint32_t p, uint32_t *det)
{
    int st = validate(A, n, n, lda, p);
    if (st != O_OK) return st;
    uint32_t *W = (uint32_t *)malloc((size_t)(n > 0 ? n * n : 1) * sizeof(uint32_t));
    if (!W) return O_ENOMEM;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) W[i * n + j] = A[i * lda + j];
    uint32_t d = 1 % p;
    for (int64_t c = 0; c < n; ++c) {
        int64_t s = -1;
        for (int64_t i = c; i < n; ++i)
            if (W[i * n + c] != 0) { s = i; break; }
        if (s < 0) { d = 0; break; }
        if (s != c) {
            for (int64_t j = 0; j < n; ++j) {
                uint32_t t = W[s * n + j];
                W[s * n + j] = W[c * n + j];
                W[c * n + j] = t;
            }
            d = sub_mod(0, d, p);
        }
        d = mul_mod(d, W[c * n + c], p);
        uint32_t inv = inv_mod(W[c * n + c], p);
        for (int64_t i = c + 1; i < n; ++i) {
            uint32_t f = mul_mod(W[i * n + c], inv, p);
            if (f == 0) continue;
            for (int64_t j = c; j < n; ++j)
                W[i * n + j] = sub_mod(W[i * n + j], mul_mod(f, W[c * n + j], p), p);
        }
    }
    free(W);
    *det = d;
    return O_OK;
}

/* ------------------------------------------------------------- PLE / CUP -- */
/*
 * PLE and CUP decompositions (Sec. 1: PLE's E is in row echelon form and its
 * pivots give the column rank profile; CUP's C = P L is in column echelon form
 * and its pivots give the row rank profile).  The paper gives no construction,
 * so they are written out here from their definitions:
 *
 * PLE.  A = P L E with P a permutation, L (m x r) unit lower trapezoidal and E
 * (r x n) in row echelon form whose t-th row starts at column c_t, where
 * c_0 < c_1 < ... are the columns of the ones of the rank profile matrix R
 * (the column rank profile) and i_t is the row of the one in column c_t.
 * perm_p lists i_0, ..., i_{r-1}, then the other rows increasing
 * (A[perm_p[i]][.] = (L E)[i][.]).  Given P the factors are unique: they come
 * from elimination on P^T A with the prescribed pivot positions (t, c_t): for
 * t = 0 .. r-1, every row below t is reduced by row t at column c_t.
 *
 * CUP.  A = C U Q with C (m x r) in column echelon form whose t-th column
 * starts at row i_t (the row rank profile, increasing), U (r x n) unit upper
 * trapezoidal and perm_q listing the columns c_t of those pivots in that
 * order, then the other columns increasing (A[.][perm_q[j]] = (C U)[.][j]).
 * It is the transpose of the PLE of A^T.
 *
 * L (ldl = r), E (lde = n), C (ldc = r), U (ldu = n) are written densely.
 * Returns a status; *rank receives r.
 */
static int ple_dense(const uint32_t *A, int64_t m, int64_t n, int64_t lda, int trans, uint32_t p,
                     int32_t *perm, uint32_t *L, uint32_t *E, int64_t *rank)
{
    /* the matrix worked on: A (m x n) or its transpose (n x m) */
    const int64_t mm = trans ? n : m, nn = trans ? m : n;
    uint32_t *M = (uint32_t *)malloc((size_t)(mm > 0 ? mm : 1) * (size_t)(nn > 0 ? nn : 1) * 4);
    int32_t *col_of_row = (int32_t *)malloc((size_t)(mm > 0 ? mm : 1) * 4);
    int32_t *row_of_col = (int32_t *)malloc((size_t)(nn > 0 ? nn : 1) * 4);
    if (!M || !col_of_row || !row_of_col) { free(M); free(col_of_row); free(row_of_col); return O_ENOMEM; }
    for (int64_t i = 0; i < mm; ++i)
        for (int64_t j = 0; j < nn; ++j) M[i * nn + j] = trans ? A[j * lda + i] : A[i * lda + j];
    int64_t r = oracle_rank_profile(M, mm, nn, nn > 0 ? nn : 1, p, col_of_row);
    if (r < 0) { free(M); free(col_of_row); free(row_of_col); return (int)r; }
    for (int64_t j = 0; j < nn; ++j) row_of_col[j] = -1;
    for (int64_t i = 0; i < mm; ++i)
        if (col_of_row[i] >= 0) row_of_col[col_of_row[i]] = (int32_t)i;
    /* P: pivot rows in increasing order of their pivot column, then the rest */
    int64_t t = 0;
    for (int64_t j = 0; j < nn; ++j)
        if (row_of_col[j] >= 0) perm[t++] = row_of_col[j];
    for (int64_t i = 0; i < mm; ++i)
        if (col_of_row[i] < 0) perm[t++] = (int32_t)i;
    /* W = P^T M, then elimination with pivots (t, c_t) */
    uint32_t *Wm = (uint32_t *)malloc((size_t)(mm > 0 ? mm : 1) * (size_t)(nn > 0 ? nn : 1) * 4);
    if (!Wm) { free(M); free(col_of_row); free(row_of_col); return O_ENOMEM; }
    for (int64_t i = 0; i < mm; ++i)
        for (int64_t j = 0; j < nn; ++j) Wm[i * nn + j] = M[(int64_t)perm[i] * nn + j];
    for (int64_t i = 0; i < mm; ++i)
        for (int64_t k = 0; k < r; ++k) L[i * r + k] = (i == k) ? 1u : 0u;
    int st = O_OK;
    for (int64_t k = 0; k < r && st == O_OK; ++k) {
        const int64_t c = col_of_row[perm[k]];
        const uint32_t piv = Wm[k * nn + c];
        if (piv == 0) { st = O_EINTERNAL; break; }
        const uint32_t inv = inv_mod(piv, p);
        for (int64_t i = k + 1; i < mm; ++i) {
            const uint32_t f = mul_mod(Wm[i * nn + c], inv, p);
            L[i * r + k] = f;
            if (f == 0) continue;
            for (int64_t j = 0; j < nn; ++j)
                Wm[i * nn + j] = sub_mod(Wm[i * nn + j], mul_mod(f, Wm[k * nn + j], p), p);
        }
    }
    for (int64_t k = 0; k < r; ++k)
        for (int64_t j = 0; j < nn; ++j) E[k * nn + j] = Wm[k * nn + j];
    for (int64_t i = r; i < mm && st == O_OK; ++i)          /* the rank is r */
        for (int64_t j = 0; j < nn; ++j)
            if (Wm[i * nn + j] != 0) { st = O_EINTERNAL; break; }
    free(M); free(Wm); free(col_of_row); free(row_of_col);
    *rank = r;
    return st;
}

int oracle_ple(const uint32_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p,
               int32_t *perm_p, uint32_t *L, uint32_t *E, int64_t *rank)
{
    return ple_dense(A, m, n, lda, 0, p, perm_p, L, E, rank);
}

int oracle_cup(const uint32_t *A, int64_t m, int64_t n, int64_t lda, uint32_t p,
               int32_t *perm_q, uint32_t *C, uint32_t *U, int64_t *rank)
{
    /* PLE of A^T = P' L' E': C = E'^T (m x r), U = L'^T (r x n), Q = P' */
    const int64_t cap = m < n ? m : n;
    uint32_t *Lt = (uint32_t *)malloc((size_t)(n > 0 ? n : 1) * (size_t)(cap > 0 ? cap : 1) * 4);
    uint32_t *Et = (uint32_t *)malloc((size_t)(cap > 0 ? cap : 1) * (size_t)(m > 0 ? m : 1) * 4);
    if (!Lt || !Et) { free(Lt); free(Et); return O_ENOMEM; }
    int st = ple_dense(A, m, n, lda, 1, p, perm_q, Lt, Et, rank);
    const int64_t r = *rank;
    if (st == O_OK) {
        for (int64_t i = 0; i < m; ++i)
            for (int64_t k = 0; k < r; ++k) C[i * r + k] = Et[k * m + i];
        for (int64_t k = 0; k < r; ++k)
            for (int64_t j = 0; j < n; ++j) U[k * n + j] = Lt[j * r + k];
    }
    free(Lt); free(Et);
    return st;
}
