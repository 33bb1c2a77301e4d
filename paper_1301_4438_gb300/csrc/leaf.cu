// Base case of Algorithm 1 (Sec. 2) on a block of at most 128 x 128, one
// thread block, the block resident in shared memory.
//
// The output must be the one Algorithm 1 produces, so the kernel works in
// three phases:
//  1. Row-order elimination.  Repeatedly find the first row (at or below the
//     last pivot row) with a nonzero in a column that is not yet a pivot
//     column; its first such column is the pivot.  This discovers the ones of
//     the rank profile matrix R row by row (a row is a pivot row iff it is
//     independent of the rows above it, and its pivot column is the first
//     column at which it becomes so).  The search is parallel over rows, so a
//     step costs one pivot, not one row.
//  2. Order.  The pivots of R are ordered as the quad recursion of Algorithm 1
//     meets them: split rows and columns at floor(half), recurse on A1, then on
//     the top rows not used by A1 x right columns (F), the bottom rows x left
//     columns not used by A1 (G), and the bottom rows not used by G x right
//     columns not used by F (R).  A call with one row or one column keeps the
//     single one of R it contains.
//  3. Elimination without pivoting on P^T A Q^T in that order.  When the order
//     of phase 2 equals the row order of phase 1 (always the case for generic
//     rank profiles), phase 1 already holds this factorisation and phase 3 is
//     skipped.
// Both eliminations are fraction free: at pivot k with value d_k every active
// row becomes d_k * row - row[pivot col] * pivot row, so no inverse sits on the
// sequential path.  All active rows then carry the common factor
// c_k = d_0 ... d_{k-1}; at the end U's row k is divided by c_k and L's column k
// by d_k, with the 2r inverses computed in parallel.
#include "common.cuh"

namespace pluq {
namespace {

constexpr int LM = LEAF_MAX;   // max rows and columns
constexpr int LD = LM + 1;     // padded shared-memory row
constexpr int LT = 512;        // threads
constexpr int NW = LT / 32;

struct Mask {                  // 128-bit set of row or column indices
    uint64_t w[2];
};
__device__ __forceinline__ int popc(const Mask &a) { return __popcll(a.w[0]) + __popcll(a.w[1]); }
__device__ __forceinline__ bool has(const Mask &a, int i) { return (a.w[i >> 6] >> (i & 63)) & 1; }
__device__ __forceinline__ void set(Mask &a, int i) { a.w[i >> 6] |= 1ull << (i & 63); }
__device__ __forceinline__ Mask andnot(const Mask &a, const Mask &b)
{
    return Mask{{a.w[0] & ~b.w[0], a.w[1] & ~b.w[1]}};
}
__device__ __forceinline__ int first(const Mask &a)
{
    return a.w[0] ? __ffsll(a.w[0]) - 1 : 64 + __ffsll(a.w[1]) - 1;
}
// the lowest `cnt` members of a
__device__ __forceinline__ Mask lowest(const Mask &a, int cnt)
{
    Mask out{{0, 0}};
    Mask rest = a;
    for (int t = 0; t < cnt; ++t) {
        int i = first(rest);
        set(out, i);
        rest.w[i >> 6] &= ~(1ull << (i & 63));
    }
    return out;
}

// Algorithm 1's order of the ones of R inside rows x cols, as an explicit
// stack (no device recursion): a frame splits its rows and columns at
// floor(half) and visits A1, F, G, R in turn, each child returning the rows
// and columns its pivots used.
struct Frame {
    Mask rows, cols, rt, rb, cl, cr;
    Mask r1, c1, c2, r3;
    Mask ur, uc;        // rows / columns used so far by this frame
    int stage;
};
constexpr int MAX_DEPTH = 20;

__device__ int order_pivots(Frame *stk, const int32_t *col_of_row, const int32_t *row_of_col,
                            int m, int n, int32_t *ord_row, int32_t *ord_col)
{
    int count = 0;
    int top = 0;
    Mask rows{{0, 0}}, cols{{0, 0}};
    for (int i = 0; i < m; ++i) set(rows, i);
    for (int j = 0; j < n; ++j) set(cols, j);
    stk[0].rows = rows;
    stk[0].cols = cols;
    stk[0].stage = 0;
    Mask ret_r{{0, 0}}, ret_c{{0, 0}};   // used masks returned by the last popped frame
    while (top >= 0) {
        Frame &f = stk[top];
        if (f.stage == 0) {
            f.ur = Mask{{0, 0}};
            f.uc = Mask{{0, 0}};
            const int nr = popc(f.rows), nc = popc(f.cols);
            if (nr == 0 || nc == 0 || nr == 1 || nc == 1) {
                if (nr == 1 && nc >= 1) {
                    int i = first(f.rows);
                    int c = col_of_row[i];
                    if (c >= 0 && has(f.cols, c)) {
                        ord_row[count] = i; ord_col[count] = c; ++count;
                        set(f.ur, i); set(f.uc, c);
                    }
                } else if (nc == 1 && nr >= 1) {
                    int j = first(f.cols);
                    int i = row_of_col[j];
                    if (i >= 0 && has(f.rows, i)) {
                        ord_row[count] = i; ord_col[count] = j; ++count;
                        set(f.ur, i); set(f.uc, j);
                    }
                }
                ret_r = f.ur; ret_c = f.uc;
                --top;
                continue;
            }
            f.rt = lowest(f.rows, nr / 2); f.rb = andnot(f.rows, f.rt);
            f.cl = lowest(f.cols, nc / 2); f.cr = andnot(f.cols, f.cl);
            f.stage = 1;
            if (top + 1 >= MAX_DEPTH) return -1;
            Frame &c = stk[top + 1];                       // A1
            c.rows = f.rt; c.cols = f.cl; c.stage = 0;
            ++top;
            continue;
        }
        // a child just returned (ret_r, ret_c)
        f.ur.w[0] |= ret_r.w[0]; f.ur.w[1] |= ret_r.w[1];
        f.uc.w[0] |= ret_c.w[0]; f.uc.w[1] |= ret_c.w[1];
        if (f.stage < 4 && top + 1 >= MAX_DEPTH) return -1;
        Frame &c = stk[top + 1];
        if (f.stage == 1) {
            f.r1 = ret_r; f.c1 = ret_c;
            c.rows = andnot(f.rt, f.r1); c.cols = f.cr;     // F
        } else if (f.stage == 2) {
            f.c2 = ret_c;
            c.rows = f.rb; c.cols = andnot(f.cl, f.c1);     // G
        } else if (f.stage == 3) {
            f.r3 = ret_r;
            c.rows = andnot(f.rb, f.r3); c.cols = andnot(f.cr, f.c2);   // R
        } else {
            ret_r = f.ur; ret_c = f.uc;
            --top;
            continue;
        }
        ++f.stage;
        c.stage = 0;
        ++top;
        if (top >= MAX_DEPTH) return -1;
    }
    return count;
}

struct LeafShared {
    uint32_t W[LM * LD];
    int32_t piv_row[LM], piv_col[LM];
    int32_t col_of_row[LM], row_of_col[LM];
    int32_t ord_row[LM], ord_col[LM];
    int32_t perm_p[LM], perm_q[LM];
    uint32_t dval[LM], inv_d[LM], cval[LM], inv_c[LM];
    uint32_t live[LM / 32];     // live (non-pivot) columns as a bitset
    Frame stk[MAX_DEPTH];
    int key;
    int r;
    int same;
};

// elements of the (rows x cols) update region handled by this thread:
// columns j = cbase + (tid % cw), rows i = rbase + tid / cw + g * (LT / cw)
__device__ __forceinline__ int col_width(int n)
{
    int cw = 1;
    while (cw < n) cw <<= 1;
    return cw;  // <= LM
}

__global__ void __launch_bounds__(LT) leaf_kernel(uint32_t *__restrict__ A, int m, int n,
                                                  int64_t lda, Field F, int32_t *perm_p_out,
                                                  int32_t *perm_q_out, int32_t *rank_out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LeafShared &S = *reinterpret_cast<LeafShared *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t p = F.p;
    const int cw = col_width(n);
    const int rstep = LT / cw;
    const int my_c = tid % cw, my_r0 = tid / cw;

    // load the block
    for (int e = tid; e < m * cw; e += LT) {
        int i = e / cw, j = e % cw;
        if (j < n) S.W[i * LD + j] = A[(int64_t)i * lda + j];
    }
    for (int i = tid; i < LM; i += LT) {
        S.col_of_row[i] = -1;
        S.row_of_col[i] = -1;
    }
    if (tid < LM / 32) {
        int lo = tid * 32;
        int cnt = n - lo;
        S.live[tid] = cnt >= 32 ? 0xFFFFFFFFu : (cnt <= 0 ? 0u : ((1u << cnt) - 1u));
    }
    if (tid == 0) S.r = 0;
    __syncthreads();

    // ---------------- phase 1: row-order fraction-free elimination --------
    int start = 0;
    int r = 0;
    while (start < m) {
        if (tid == 0) S.key = 0x7FFFFFFF;
        __syncthreads();
        // each warp scans its rows in increasing order, stops at the first hit
        for (int i = start + warp; i < m; i += NW) {
            int best = 0x7FFFFFFF;
#pragma unroll
            for (int s = 0; s < LM / 32; ++s) {
                int j = lane + 32 * s;
                if (j < n && ((S.live[s] >> lane) & 1) && S.W[i * LD + j] != 0) {
                    best = j < best ? j : best;
                }
            }
            best = __reduce_min_sync(0xFFFFFFFFu, best);
            if (best != 0x7FFFFFFF) {
                if (lane == 0) atomicMin(&S.key, i * LM + best);
                break;
            }
            // rows beyond the current best need not be scanned (warp-uniform test)
            const int cur = __shfl_sync(0xFFFFFFFFu, *(volatile int *)&S.key, 0);
            if (cur < (i + NW) * LM) break;
        }
        __syncthreads();
        const int key = S.key;
        if (key == 0x7FFFFFFF) break;
        const int pi = key / LM, pc = key % LM;
        const uint32_t d = S.W[pi * LD + pc];
        if (tid == 0) {
            S.piv_row[r] = pi;
            S.piv_col[r] = pc;
            S.dval[r] = d;
            S.col_of_row[pi] = pc;
            S.row_of_col[pc] = pi;
            S.live[pc >> 5] &= ~(1u << (pc & 31));
        }
        __syncthreads();   // live updated; column pc now frozen
        // rows below the pivot row: W[i][j] = d W[i][j] - W[i][pc] W[pi][j], live j
        if (my_c < n && ((S.live[my_c >> 5] >> (my_c & 31)) & 1)) {
            const uint32_t prow = S.W[pi * LD + my_c];
            for (int i = pi + 1 + my_r0; i < m; i += rstep) {
                uint32_t f = S.W[i * LD + pc];
                uint32_t *w = &S.W[i * LD + my_c];
                *w = mul_sub_mul_mod(d, *w, f, prow, F);
            }
        }
        ++r;
        start = pi + 1;
        __syncthreads();
    }

    // ---------------- phase 2: Algorithm 1's order of the pivots ----------
    if (tid == 0) {
        const int cnt = order_pivots(S.stk, S.col_of_row, S.row_of_col, m, n, S.ord_row, S.ord_col);
        int same = cnt == r ? 1 : -1;   // -1: inconsistent, reported as an error
        if (same < 0) r = 0;
        for (int t = 0; t < r; ++t)
            if (S.ord_row[t] != S.piv_row[t]) same = 0;
        // P, Q: pivots in order, then the others increasing
        int a = 0;
        for (int t = 0; t < r; ++t) S.perm_p[a++] = S.ord_row[t];
        for (int i = 0; i < m; ++i)
            if (S.col_of_row[i] < 0) S.perm_p[a++] = i;
        a = 0;
        for (int t = 0; t < r; ++t) S.perm_q[a++] = S.ord_col[t];
        for (int j = 0; j < n; ++j)
            if (S.row_of_col[j] < 0) S.perm_q[a++] = j;
        S.same = same;
        S.r = r;
    }
    __syncthreads();
    const int same = S.same;
    if (same < 0) {                 // leave the block untouched, flag the error
        if (tid == 0) *rank_out = -1;
        return;
    }

    // ---------------- phase 3: elimination without pivoting ---------------
    if (!same) {
        for (int e = tid; e < m * cw; e += LT) {
            int i = e / cw, j = e % cw;
            if (j < n) S.W[i * LD + j] = A[(int64_t)S.perm_p[i] * lda + S.perm_q[j]];
        }
        __syncthreads();
        for (int k = 0; k < r; ++k) {
            const uint32_t d = S.W[k * LD + k];
            if (tid == 0) S.dval[k] = d;
            if (my_c > k && my_c < n) {
                const uint32_t prow = S.W[k * LD + my_c];
                for (int i = k + 1 + my_r0; i < m; i += rstep) {
                    uint32_t f = S.W[i * LD + k];
                    uint32_t *w = &S.W[i * LD + my_c];
                    *w = mul_sub_mul_mod(d, *w, f, prow, F);
                }
            }
            __syncthreads();
        }
    }

    // ---------------- fix-up: divide U rows by c_k, L columns by d_k ------
    if (tid == 0) {
        uint32_t c = 1;
        for (int k = 0; k < r; ++k) {
            S.cval[k] = c;
            c = mul_mod(c, S.dval[k], F);
        }
    }
    __syncthreads();
    for (int t = tid; t < 2 * r; t += LT) {
        if (t < r) S.inv_d[t] = inv_mod(S.dval[t], p);
        else S.inv_c[t - r] = inv_mod(S.cval[t - r], p);
    }
    __syncthreads();

    // write the packed block [L\U V; M 0] in P, Q order
    for (int e = tid; e < m * cw; e += LT) {
        int i = e / cw, j = e % cw;
        if (j >= n) continue;
        uint32_t v;
        if (i < r && j >= i) {
            uint32_t w = same ? S.W[S.piv_row[i] * LD + S.perm_q[j]] : S.W[i * LD + j];
            v = mul_mod(w, S.inv_c[i], F);
        } else if (j < r && i > j) {
            uint32_t w = same ? S.W[S.perm_p[i] * LD + S.piv_col[j]] : S.W[i * LD + j];
            v = mul_mod(w, S.inv_d[j], F);
        } else {
            v = 0;
        }
        A[(int64_t)i * lda + j] = v;
    }
    for (int i = tid; i < m; i += LT) perm_p_out[i] = S.perm_p[i];
    for (int j = tid; j < n; j += LT) perm_q_out[j] = S.perm_q[j];
    if (tid == 0) *rank_out = r;
}

}  // namespace

pluq_status launch_leaf(uint32_t *A, int64_t m, int64_t n, int64_t lda, Field F, int32_t *perm_p,
                        int32_t *perm_q, int32_t *rank, cudaStream_t st)
{
    if (m < 0 || n < 0 || m > LM || n > LM) return PLUQ_EINVAL;
    if (m == 0 || n == 0) {
        // empty block: r = 0, identity permutations
        if (m) PLUQ_TRY(launch_iota(perm_p, m, st));
        if (n) PLUQ_TRY(launch_iota(perm_q, n, st));
        PLUQ_CUDA_TRY(cudaMemsetAsync(rank, 0, sizeof(int32_t), st));
        return PLUQ_OK;
    }
    static bool attr_set = false;
    const size_t smem = sizeof(LeafShared);
    if (!attr_set) {
        PLUQ_CUDA_TRY(cudaFuncSetAttribute(leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
        attr_set = true;
    }
    prof::start(prof::LEAF, st);
    leaf_kernel<<<1, LT, smem, st>>>(A, (int)m, (int)n, lda, F, perm_p, perm_q, rank);
    pluq_status s = last_launch();
    prof::stop(prof::LEAF, st, (double)m * n * 8.0);
    return s;
}

}  // namespace pluq
