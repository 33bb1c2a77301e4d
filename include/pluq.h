/*
 * libpluq — rank-profile-revealing PLUQ decomposition over Z/pZ on one GB300.
 *
 * The method is Algorithm 1 of Dumas, Pernet & Sultan, "Simultaneous
 * computation of the row and column rank profiles" (arXiv 1301.4438): a
 * quad-recursive elimination whose permutations P and Q reveal the row and
 * column rank profiles of the matrix and of each of its leading submatrices.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Field: Z/pZ with p prime, 2 <= p < 2^31.  Elements are uint32 in [0, p).
 *    Every result is exact (bit-identical to textbook arithmetic mod p).
 *  - Matrices: row-major uint32 with a row stride (ld >= number of columns).
 *  - Pointers named d_* are DEVICE pointers (cudaMalloc'd or torch-owned),
 *    h_* are HOST pointers.  The caller owns every buffer; the library keeps no
 *    pointer after a call returns and allocates no device memory of its own:
 *    scratch comes from the caller's workspace (see pluq_workspace_size).
 *  - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Return value: a pluq_status.  Argument errors are reported before any
 *    work is queued and leave every buffer untouched.
 *
 * Permutation vectors (Algorithm 1 output, Sec. 2)
 * ------------------------------------------------
 *  perm_p[i] = original row index placed at packed row i   (P[perm_p[i], i] = 1)
 *  perm_q[j] = original column index placed at packed column j (Q[j, perm_q[j]] = 1)
 *  so that A[perm_p[i]][perm_q[j]] = ([L; M] [U V])[i][j].  The first r entries
 *  are the pivots in the order Algorithm 1 finds them; the remaining rows and
 *  columns follow in increasing order.
 */
#ifndef PLUQ_H
#define PLUQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PLUQ_OK = 0,
    PLUQ_EINVAL = -1,       /* bad size, stride, null pointer or flag */
    PLUQ_ENOTPRIME = -2,    /* p is not a prime in [2, 2^31) */
    PLUQ_ERANGE = -3,       /* an input entry is >= p (no silent reduction) */
    PLUQ_ENOMEM = -4,       /* workspace smaller than pluq_workspace_size() */
    PLUQ_ECUDA = -5,        /* a CUDA runtime call failed */
    PLUQ_ETIMEOUT = -6,     /* a bounded device-side wait gave up */
    PLUQ_EINTERNAL = -7,    /* an internal consistency check failed */
    PLUQ_EUNSUPPORTED = -8  /* the requested kernel form is not available */
} pluq_status;

/* Kernel used for the modular matrix products (MM) inside the factorisation. */
typedef enum {
    PLUQ_MM_AUTO = 0,       /* the tensor-core form */
    PLUQ_MM_SIMT = 1,       /* plain CUDA-core form: 32x32->64-bit products */
    PLUQ_MM_TENSOR = 2      /* 8-bit limbs on tcgen05 tensor cores (bf16 x bf16 -> fp32,
                               exact below 2^24), mod-p reduction in the epilogue */
} pluq_mm_kind;

/* Human-readable text of a status code (static storage). */
const char *pluq_status_string(int status);

/*
 * Bytes of device workspace pluq_mod_p needs for an m x n matrix mod p.
 * Writes the size to *h_bytes.  Depends only on (m, n, p).
 */
pluq_status pluq_workspace_size(int64_t m, int64_t n, uint32_t p, size_t *h_bytes);

/*
 * PLUQ decomposition, Algorithm 1 (Sec. 2), in place.
 *   d_A      m x n, stride lda >= n, entries in [0, p).  On return it holds the
 *            packed form [L\U V; M 0] of the Algorithm 1 output contract: L unit
 *            lower r x r (diagonal not stored), U upper r x r, V r x (n-r),
 *            M (m-r) x r, and a zero (m-r) x (n-r) block.
 *   d_perm_p m int32, d_perm_q n int32 (see the convention above).
 *   h_rank   receives r.
 *   d_work   workspace of ws_bytes >= pluq_workspace_size(m, n, p) bytes.
 *   mm_kind  a pluq_mm_kind.
 * Zero dimensions are allowed (Sec. 2): r = 0 and identity permutations.
 * The ranks of sub-blocks decide the shapes of later steps, so the call
 * returns only after the factorisation has completed on `stream`.
 * Errors: EINVAL, ENOTPRIME, ERANGE (checked on the device before any write),
 * ENOMEM, ECUDA, EUNSUPPORTED.
 */
pluq_status pluq_mod_p(uint32_t *d_A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                       int32_t *d_perm_p, int32_t *d_perm_q, int64_t *h_rank,
                       void *d_work, size_t ws_bytes, int mm_kind, void *stream);

/*
 * Many independent decompositions of uneven sizes (the families of matrices
 * Groebner-basis elimination produces), each with the contract of
 * pluq_mod_p.  Host arrays of length `count` give, per matrix, its device
 * pointer h_dA[i] (m[i] x n[i], stride lda[i]), its output vectors
 * h_dperm_p[i] / h_dperm_q[i] (device) and receive h_rank[i].  `workers` host
 * threads, each with its own non-blocking stream (created and destroyed inside
 * the call, ordered after the work already queued on `stream`) and its own
 * slice of d_work, take the matrices largest first; the kernels of different
 * matrices overlap on the GPU.  Returns after every decomposition is done;
 * the first failing status is returned (later matrices are then skipped).
 * Workspace: pluq_batched_workspace_size (workers x the largest single need).
 */
pluq_status pluq_batched_workspace_size(const int64_t *h_m, const int64_t *h_n, int64_t count,
                                        uint32_t p, int workers, size_t *h_bytes);
pluq_status pluq_mod_p_batched(uint32_t *const *h_dA, const int64_t *h_m, const int64_t *h_n,
                               const int64_t *h_lda, int64_t count, uint32_t p,
                               int32_t *const *h_dperm_p, int32_t *const *h_dperm_q,
                               int64_t *h_rank, void *d_work, size_t ws_bytes, int mm_kind,
                               int workers, void *stream);

/*
 * The same batch in ONE persistent launch (Algorithm 1, Sec. 2, for every
 * matrix; the recursion runs on the device, no host round trip).  `ctas`
 * thread blocks (0: one per SM) each take the next matrix from a device-side
 * counter, in array order (put the largest first for balance), and factor it
 * to the end on one SM.  Every argument array is DEVICE memory of length
 * `count`: d_A[i] (m[i] x n[i], stride lda[i] >= n[i]), d_m, d_n, d_lda,
 * output vectors d_perm_p[i] / d_perm_q[i] (device), and d_rank[i], which
 * receives r, or a negative status for that matrix alone (EINVAL: m or n
 * outside [0, max_m] x [0, max_n], or a null pointer or lda < n; ERANGE: an
 * entry >= p, the matrix left untouched; ETIMEOUT: a bounded wait gave up).
 * Every matrix gets the packed output contract of pluq_mod_p; results do not
 * depend on ctas.  max_m, max_n <= 2048 (sixteen base-case blocks).
 * Asynchronous on `stream`: one memset and one kernel launch, no host
 * synchronisation, so a warmed-up call can be captured in a CUDA graph and
 * replayed.  The d_rank values are valid once the stream reaches that point.
 * Workspace: pluq_batched_persistent_workspace_size(max_m, max_n, ctas),
 * 16-byte aligned; calls that share a workspace must not overlap.
 * Host-checked errors: EINVAL (count < 0, ctas < 0, max_m / max_n out of
 * range, null arrays, a workspace not 16-byte aligned), ENOTPRIME, ENOMEM
 * (workspace missing or too small), ECUDA.
 */
pluq_status pluq_batched_persistent_workspace_size(int64_t max_m, int64_t max_n, int ctas,
                                                   size_t *h_bytes);
pluq_status pluq_mod_p_batched_persistent(uint32_t *const *d_A, const int64_t *d_m,
                                          const int64_t *d_n, const int64_t *d_lda, int64_t count,
                                          int64_t max_m, int64_t max_n, uint32_t p,
                                          int32_t *const *d_perm_p, int32_t *const *d_perm_q,
                                          int64_t *d_rank, void *d_work, size_t ws_bytes, int ctas,
                                          void *stream);

/*
 * Row rank profile of A (Corollary of Lemma 2, Sec. 4): the sorted first r
 * entries of perm_p.  d_out receives r int32.  Asynchronous on `stream`.
 */
pluq_status row_rank_profile(const int32_t *d_perm_p, int64_t m, int64_t r,
                             int32_t *d_out, void *stream);

/* Column rank profile of A: the sorted first r entries of perm_q. */
pluq_status col_rank_profile(const int32_t *d_perm_q, int64_t n, int64_t r,
                             int32_t *d_out, void *stream);

/*
 * Rank profile matrix R = P diag(I_r, 0) Q (Lemma 2, Sec. 4) as its r ones:
 * R[d_rows[t], d_cols[t]] = 1, sorted by row.  The rank profiles of any leading
 * k x t submatrix of A are the rows / columns of the ones in [0,k) x [0,t).
 */
pluq_status rank_profile_matrix(const int32_t *d_perm_p, const int32_t *d_perm_q,
                                int64_t m, int64_t n, int64_t r,
                                int32_t *d_rows, int32_t *d_cols, void *stream);

/*
 * Factors of A = P [L; M] [U V] Q out of the packed result of pluq_mod_p
 * (Sec. 2, the PLUQ form at the start of the algorithm's description), in the
 * packed row / column order.  pluq_extract_L writes d_L (m x r, stride
 * ldl >= r): the unit lower trapezoid [L; M] -- the strictly lower part of
 * the first r packed columns, ones on the diagonal, zeros above it.
 * pluq_extract_U writes d_U (r x n, stride ldu >= n): the upper trapezoid
 * [U V] -- the first r packed rows on and above the diagonal, zeros below.
 * d_LU is m x n with stride lda >= n and is not modified; the output must not
 * overlap it.  Errors: EINVAL (sizes, r > min(m, n), null pointers with work
 * to do).  Asynchronous on `stream`.
 */
pluq_status pluq_extract_L(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda, int64_t r,
                           uint32_t *d_L, int64_t ldl, void *stream);
pluq_status pluq_extract_U(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda, int64_t r,
                           uint32_t *d_U, int64_t ldu, void *stream);

/*
 * LEU decomposition from the PLUQ (Corollary of the triangularity theorem,
 * Sec. 3): A = Lbar E Ubar with Lbar = P [L 0; M I_{m-r}] P^T (m x m, unit
 * lower triangular), E = P diag(I_r, 0) Q (the rank profile matrix, see
 * rank_profile_matrix) and Ubar = Q^T [U V; 0 0] Q (n x n, upper triangular),
 * in the original row and column indices.  Inputs are the packed result of
 * pluq_mod_p (d_LU, stride lda >= n, not modified) with its r, d_perm_p and
 * d_perm_q.  Either output may be null (not written); d_Lbar has stride
 * ldl >= m, d_Ubar stride ldu >= n, neither overlaps d_LU.  d_work holds
 * (m + n) int32 (inverse permutations).  Errors: EINVAL, ENOMEM (workspace).
 * Asynchronous on `stream`.
 */
pluq_status pluq_leu(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda, int64_t r,
                     const int32_t *d_perm_p, const int32_t *d_perm_q, uint32_t *d_Lbar,
                     int64_t ldl, uint32_t *d_Ubar, int64_t ldu, void *d_work, size_t ws_bytes,
                     void *stream);

/*
 * Rank profiles of the leading k x t submatrix of A (0 <= k <= m,
 * 0 <= t <= n) without forming R (Corollary of Lemma 2, Sec. 4): the ones of
 * R inside [0, k) x [0, t) are the pivots i < r with perm_p[i] < k and
 * perm_q[i] < t.  *d_count (device int32) receives their number, the rank of
 * that submatrix; d_rows / d_cols (capacity r each) receive its row and
 * column rank profiles, sorted.  Asynchronous on `stream`.
 */
pluq_status pluq_leading_rank_profiles(const int32_t *d_perm_p, const int32_t *d_perm_q,
                                       int64_t m, int64_t n, int64_t r, int64_t k, int64_t t,
                                       int32_t *d_rows, int32_t *d_cols, int32_t *d_count,
                                       void *stream);

/*
 * Uses of the decomposition (Sec. 1 names linear systems, the determinant
 * and the nullspace among them), read off the packed result of pluq_mod_p:
 * d_LU (m x n, stride lda >= n, not modified), its rank r and its d_perm_p /
 * d_perm_q, which must be the permutations pluq_mod_p returned (entries are
 * used as indices).  Because the pivot columns (rows) are the column (row)
 * rank profile, every result below is unique, not just a valid choice.
 * All are asynchronous on `stream`; products run on the kernel form mm_kind.
 * Scratch: d_work of at least pluq_uses_workspace_size(m, n, r, k, p,
 * mm_kind) bytes covers each of these calls for those sizes (k = number of
 * right-hand sides of pluq_solve, 0 otherwise).  Errors: EINVAL (sizes,
 * strides, null pointers), ENOTPRIME, ENOMEM (workspace), ECUDA.
 */
pluq_status pluq_uses_workspace_size(int64_t m, int64_t n, int64_t r, int64_t k, uint32_t p,
                                     int mm_kind, size_t *h_bytes);

/*
 * Determinant of a square A (n x n): 0 when r < n, else
 * sgn(P) sgn(Q) prod_i U[i][i] mod p, the signs from the cycle counts of
 * perm_p and perm_q.  The 0 x 0 determinant is 1.  d_det: one device uint32.
 */
pluq_status pluq_determinant(const uint32_t *d_LU, int64_t n, int64_t lda, int64_t r,
                             const int32_t *d_perm_p, const int32_t *d_perm_q, uint32_t p,
                             uint32_t *d_det, void *d_work, size_t ws_bytes, void *stream);

/*
 * Right nullspace: d_N (n x (n - r), stride ldn >= n - r) receives
 * N = Q^T [-U^{-1} V; I_{n-r}], so A N = 0 and column c of N is the unit
 * vector on the c-th column outside the column rank profile (increasing)
 * plus the combination of rank-profile columns that cancels it.  Nothing is
 * written when r = n.
 */
pluq_status pluq_right_nullspace(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda,
                                 int64_t r, const int32_t *d_perm_q, uint32_t p, uint32_t *d_N,
                                 int64_t ldn, int mm_kind, void *d_work, size_t ws_bytes,
                                 void *stream);

/*
 * Left nullspace: d_K ((m - r) x m, stride ldk >= m) receives
 * K = [-M L^{-1}, I_{m-r}] P^T, so K A = 0 and row c of K is the unit vector
 * on the c-th row outside the row rank profile (increasing) plus the
 * combination of rank-profile rows that cancels it.  Nothing is written when
 * r = m.
 */
pluq_status pluq_left_nullspace(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda,
                                int64_t r, const int32_t *d_perm_p, uint32_t p, uint32_t *d_K,
                                int64_t ldk, int mm_kind, void *d_work, size_t ws_bytes,
                                void *stream);

/*
 * A X = B for k right-hand sides: d_B (m x k, stride ldb >= k, entries in
 * [0, p), not range-checked: an entry >= p gives unspecified values but no
 * out-of-bounds access), d_X (n x k, stride ldx >= k, must not overlap d_B).
 * With Y = [L 0; M I]^{-1} P^T B, column c is solvable iff Y[r:, c] = 0;
 * *d_inconsistent (device int32) is set to 0 if every column is, else 1.
 * d_X receives Q^T [U^{-1} Y[:r, :]; 0]: for every solvable column, the
 * solution that is zero outside the column rank profile (for a nonsingular A,
 * the solution).
 */
pluq_status pluq_solve(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda, int64_t r,
                       const int32_t *d_perm_p, const int32_t *d_perm_q, uint32_t p,
                       const uint32_t *d_B, int64_t ldb, int64_t k, uint32_t *d_X, int64_t ldx,
                       int32_t *d_inconsistent, int mm_kind, void *d_work, size_t ws_bytes,
                       void *stream);

/*
 * CUP and PLE decompositions (Sec. 1: PLE's E = U Q is in row echelon form
 * and its pivots are the column rank profile; CUP's C = P L is in column
 * echelon form and its pivots are the row rank profile), from the packed
 * result of pluq_mod_p (d_LU, r, d_perm_p, d_perm_q, not modified):
 *   pluq_ple: A[d_perm_out[i]][.] = (L E)[i][.]; d_perm_out (m) lists the pivot
 *     rows in increasing order of their pivot column, then the other rows
 *     increasing; d_L (m x r, stride ldl >= r) unit lower trapezoidal; d_E
 *     (r x n, stride lde >= n) in row echelon form, row t starting at the t-th
 *     column of the column rank profile.
 *   pluq_cup: A[.][d_perm_out[j]] = (C U)[.][j]; d_perm_out (n) lists the pivot
 *     columns in increasing order of their pivot row, then the other columns
 *     increasing; d_C (m x r, stride ldc >= r) in column echelon form, column t
 *     starting at the t-th row of the row rank profile; d_U (r x n, stride
 *     ldu >= n) unit upper trapezoidal.
 * Given the permutation these factors are unique.  The paper says they follow
 * from the PLUQ by permutations only; when Algorithm 1's pivot order is not
 * increasing in column (row) order that is not so, and the construction adds
 * an r x r elimination without pivoting, a triangular solve and a product
 * (the kernels of pluq_mod_p, pluq_trsm_* and pluq_modmm, on mm_kind).
 * Scratch: d_work of at least pluq_echelon_workspace_size(m, n, r, p,
 * mm_kind) bytes.  Both return after the result is complete on `stream`.
 * Errors: EINVAL, ENOTPRIME, ENOMEM, ECUDA, EINTERNAL.
 */
pluq_status pluq_echelon_workspace_size(int64_t m, int64_t n, int64_t r, uint32_t p, int mm_kind,
                                        size_t *h_bytes);
pluq_status pluq_ple(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda, int64_t r,
                     const int32_t *d_perm_p, const int32_t *d_perm_q, uint32_t p,
                     int32_t *d_perm_out, uint32_t *d_L, int64_t ldl, uint32_t *d_E, int64_t lde,
                     int mm_kind, void *d_work, size_t ws_bytes, void *stream);
pluq_status pluq_cup(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda, int64_t r,
                     const int32_t *d_perm_p, const int32_t *d_perm_q, uint32_t p,
                     int32_t *d_perm_out, uint32_t *d_C, int64_t ldc, uint32_t *d_U, int64_t ldu,
                     int mm_kind, void *d_work, size_t ws_bytes, void *stream);

/*
 * Hot-path kernels of Algorithm 1, callable on their own.
 *
 * MM(C, A, B) of Sec. 2: C <- C - A B mod p (or C <- A B mod p when `assign`
 * is nonzero), A M x K, B K x N, C M x N.  PLUQ_MM_TENSOR runs the tensor-core
 * kernel and PLUQ_MM_SIMT the CUDA-core one whatever the size; PLUQ_MM_AUTO
 * sends products of at most the tuned number of multiply-adds (see
 * pluq_set_tuning) to the CUDA cores when C overlaps neither operand, the
 * rest to the tensor cores.  C must not overlap A or B in the SIMT form; the
 * tensor form first splits A and B into limb planes held in the workspace, so
 * C may overlap them there.  Asynchronous on `stream`.
 * Workspace: pluq_modmm_workspace_size.
 */
pluq_status pluq_modmm_workspace_size(int64_t M, int64_t N, int64_t K, uint32_t p,
                                      int mm_kind, size_t *h_bytes);
pluq_status pluq_modmm(uint32_t *d_C, int64_t ldc, const uint32_t *d_A, int64_t lda,
                       const uint32_t *d_B, int64_t ldb, int64_t M, int64_t N, int64_t K,
                       uint32_t p, int assign, int mm_kind, void *d_work, size_t ws_bytes,
                       void *stream);

/*
 * TRSM of Sec. 2.  Left: B <- L^{-1} B, L r x r unit lower (diagonal not
 * read), B r x N.  Right: B <- B U^{-1}, U r x r upper with nonzero diagonal,
 * B M x r.  Computed as the triangular inverse (recursive block formula) times
 * B on the modular MM kernels.  Asynchronous on `stream`.  Workspace:
 * pluq_trsm_workspace_size.
 */
pluq_status pluq_trsm_workspace_size(int64_t r, int64_t other, uint32_t p, int mm_kind,
                                     size_t *h_bytes);
pluq_status pluq_trsm_left_lower_unit(const uint32_t *d_L, int64_t ldl, uint32_t *d_B,
                                      int64_t ldb, int64_t r, int64_t N, uint32_t p,
                                      int mm_kind, void *d_work, size_t ws_bytes,
                                      void *stream);
pluq_status pluq_trsm_right_upper(const uint32_t *d_U, int64_t ldu, uint32_t *d_B,
                                  int64_t ldb, int64_t M, int64_t r, uint32_t p,
                                  int mm_kind, void *d_work, size_t ws_bytes, void *stream);

/*
 * PermR / PermC of Sec. 2 on a block: rows (cols) [0, count) of the block at
 * d_X are replaced by rows (cols) d_perm[0..count) of it; the block is
 * count x width (width x count).  Uses count*width*4 bytes of d_work.
 */
pluq_status pluq_perm_rows(uint32_t *d_X, int64_t ldx, int64_t count, int64_t width,
                           const int32_t *d_perm, void *d_work, size_t ws_bytes,
                           void *stream);
pluq_status pluq_perm_cols(uint32_t *d_X, int64_t ldx, int64_t height, int64_t count,
                           const int32_t *d_perm, void *d_work, size_t ws_bytes,
                           void *stream);

/*
 * Base case of the recursion (Algorithm 1 on a block of at most
 * pluq_leaf_max_rows() x pluq_leaf_max_cols()): one thread block finds the
 * block's rank profile matrix by row-echelon elimination, orders its ones as
 * Algorithm 1 would, and eliminates without pivoting in that order.  Same
 * in-place contract as pluq_mod_p; d_rank receives r (device int32).
 */
int64_t pluq_leaf_max_rows(void);
int64_t pluq_leaf_max_cols(void);
pluq_status pluq_leaf(uint32_t *d_A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                      int32_t *d_perm_p, int32_t *d_perm_q, int32_t *d_rank, void *stream);

/*
 * Instrumentation (no counterpart in the paper).  pluq_launch_count: kernels
 * launched by this library since the process started.
 * pluq_profile_enable(class_mask) starts a session that brackets every launch
 * of the kernel classes whose bit is set (bit c = class c below) with CUDA
 * events on its stream; 0 stops recording.  pluq_profile_read
 * synchronises on those events and returns, for one class, the number of
 * launches, their summed device time in ms and their summed algorithmic work:
 *   0 tensor-core MM (2 L^2 M N K digit-product flops), 1 SIMT MM (2 M N K),
 *   2 leaf (bytes of the block read+written), 3 gathers / copies (bytes),
 *   4 limb splits (bytes), 5 triangular-inverse base blocks (field ops).
 */
long long pluq_launch_count(void);

/*
 * Instrumentation (no counterpart in the paper): the measured rate of the
 * warp-level tensor-core MMA on this GPU, every SM busy for about target_ms
 * (timed with CUDA events on the legacy default stream, which it
 * synchronises).  form 0: mma.sync m16n8k32 s8 x s8 -> s32 (the integer tensor
 * path sm_103a offers; it has no integer tcgen05 MMA); form 1: mma.sync
 * m16n8k16 bf16 x bf16 -> fp32.  *h_tops receives tera-operations per second
 * (2 M N K per MMA), *h_ms the timed duration.  Errors: EINVAL, ECUDA.
 */
pluq_status pluq_measure_mma_sync_peak(int form, double target_ms, double *h_tops, double *h_ms);
pluq_status pluq_profile_enable(int class_mask);
pluq_status pluq_profile_read(int kernel_class, long long *h_launches, double *h_ms,
                              double *h_work);

/*
 * Allocation-free variant of the tensor-core pluq_modmm (the paper has no
 * counterpart: this exists for callers that cannot allocate device memory).
 * Some callers cannot hand the library a workspace: plug-ins living in a
 * process whose device memory is owned by another allocator (a framework's
 * caching allocator that has reserved the card), or latency-critical loops
 * that cannot risk an allocation failing part way.  This entry point
 * computes the same C <- C - A B (assign = 0) or C <- A B (assign != 0) mod p
 * as pluq_modmm(..., PLUQ_MM_TENSOR, ...) but keeps its limb planes in a fixed
 * device array of PLUQ_NOALLOC_SCRATCH_BYTES that the library declares
 * statically; it calls no cudaMalloc / cudaFree and no allocating routine.
 *  - Limit: the product must satisfy pluq_modmm_workspace_size(M, N, K, p,
 *    PLUQ_MM_TENSOR) <= PLUQ_NOALLOC_SCRATCH_BYTES.  For p < 2^16 (two limbs)
 *    the largest square product is M = N = K = 2000; larger products return
 *    PLUQ_ENOMEM and touch nothing.
 *  - The first call on each device looks up the array's device address with
 *    that device current (cudaGetSymbolAddress) and caches it for the life of
 *    the process; make that first call before any stream capture.  The cached
 *    address is not refreshed after cudaDeviceReset: do not call this entry
 *    point on a device after resetting it.
 *  - Every call on a device shares the one array and leaves its contents
 *    behind (every byte a call reads is written by that call first).  Calls
 *    whose kernels overlap on the GPU (different streams, or several host
 *    threads) race on it; serialise them, e.g. on one stream.
 *  - Like pluq_modmm's tensor form it is asynchronous on `stream`, and C may
 *    overlap A or B (both are copied into the scratch before C is written).
 */
#define PLUQ_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u + 8192u)
pluq_status pluq_modmm_tensor_noalloc(uint32_t *d_C, int64_t ldc, const uint32_t *d_A,
                                      int64_t lda, const uint32_t *d_B, int64_t ldb, int64_t M,
                                      int64_t N, int64_t K, uint32_t p, int assign, void *stream);

/*
 * Process-wide tuning knobs (no counterpart in the paper; chosen by the
 * package's autotuner).  leaf: blocks with both sides <= leaf (16..128) are
 * handed to the base-case kernel; small_mm_macs: products of at most this
 * many multiply-adds use the CUDA-core kernel when the output does not overlap
 * the operands.  They change speed only, never results.  Set before a call;
 * calls in flight keep the values they started with.
 */
pluq_status pluq_set_tuning(int64_t leaf, int64_t small_mm_macs);
pluq_status pluq_get_tuning(int64_t *h_leaf, int64_t *h_small_mm_macs);

/*
 * PLUQ(F) and PLUQ(G) of a recursion node are independent (the parallelism
 * Sec. 9 points out).  When both blocks have at least branch_min rows and
 * columns, G runs on another host thread with its own streams and a slice of
 * the workspace while the calling thread runs F.  Speed only, never results.
 * Default 64; EINVAL for branch_min < 1.
 */
pluq_status pluq_set_branch_min(int64_t branch_min);
int64_t pluq_get_branch_min(void);

/*
 * Before recursing into a block, the recursion tests whether the block is
 * zero (a block's rank is the number of ones of the rank profile matrix inside
 * it, so a zero block is finished at once: r = 0, P = Q = I).  Below a
 * rank-deficient node, lazy = 0 waits for that test before descending; lazy =
 * 1 descends at once and reads the answer together with the first leaf's
 * result.  Speed only, never results.  Default 0; EINVAL unless lazy is 0 or 1.
 */
pluq_status pluq_set_lazy_zero_test(int lazy);
int pluq_get_lazy_zero_test(void);

/*
 * Base-case variant (Sec. 7, the remark after Algorithm 2 on a left-looking
 * form used in the experiments): the base case's blocked elimination without
 * pivoting is right-looking (0: each 16-column panel, once factored, updates
 * every column to its right) or left-looking (1: a panel receives the updates
 * of all earlier panels just before it is factored).  Both apply the same
 * updates in the same order, so results are identical; speed only.
 * Default 0; EINVAL unless 0 or 1.
 */
pluq_status pluq_set_leaf_variant(int left_looking);
int pluq_get_leaf_variant(void);

/*
 * Node kernel (speed only, never results): below a rank-deficient node of
 * the recursion, a node of at most 2 x leaf (levels >= 1) or 4 x leaf
 * (levels = 2) on a side is computed by one thread block in one launch -- its
 * base cases and the permutations, triangular solves and products of
 * Algorithm 1's steps between them (for 4 x leaf, two levels of steps) --
 * instead of dozens of launches and host round trips.  It pays where those
 * blocks hold few pivots, deep in a rank-deficient matrix.  levels = 0 keeps
 * every node on the host-driven path.  Default 1; EINVAL outside 0..2.
 */
pluq_status pluq_set_node_kernel(int levels);
int pluq_get_node_kernel(void);

/*
 * Thread blocks of a node kernel (speed only, never results): 1 (default), or
 * a cluster of 2, 4 or 8 on as many SMs.  In a cluster the two middle base cases
 * of a step (F and G of Algorithm 1, independent of each other) run at once
 * on different blocks, and the permutations, triangular solves and products
 * between the base cases are split over the blocks.  EINVAL for other values.
 */
pluq_status pluq_set_node_cluster(int ctas);
int pluq_get_node_cluster(void);

/*
 * Failure detection (no counterpart in the paper).  Every wait inside a kernel
 * that depends on other warps (the tensor-core product's pipeline barriers,
 * the base case's step barrier) is bounded: after `tries` unsuccessful tries
 * the kernel records an error, stops its work, lets the copies and MMAs it has
 * issued finish (those waits keep their full bound), frees its tensor memory
 * and returns; the block it was computing is then unspecified.
 * pluq_set_wait_limit sets the number of tries for kernels launched
 * afterwards: a negative value restores the built-in bounds (about 2^24 and
 * 2^22 tries), 0 gives up before the first try (a way to exercise this path
 * without a fault).  pluq_device_status synchronises `stream` and returns
 * PLUQ_ETIMEOUT if any kernel of the library gave up a wait since the last
 * call (and clears that record), else PLUQ_OK or PLUQ_ECUDA.  pluq_mod_p
 * reports a wait given up inside it as PLUQ_ETIMEOUT itself.
 */
pluq_status pluq_set_wait_limit(int64_t tries);
pluq_status pluq_device_status(void *stream);

/* Number of 8-bit limbs the tensor form splits residues mod p into (1 to 4). */
int pluq_tensor_limbs(uint32_t p);

#ifdef __cplusplus
}
#endif
#endif /* PLUQ_H */
