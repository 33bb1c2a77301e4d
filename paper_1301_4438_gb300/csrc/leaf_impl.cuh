#pragma once
// Shared parts of the base case of Algorithm 1 (Sec. 2), used by the base
// case's own kernel (leaf.cu) and by the node kernel (node.cu), which runs
// base cases inside a node step.  Everything here has internal linkage, so
// each translation unit holds its own copy (including the step-wait error
// word, which each unit reports through its own reader).
//
// The base case works on a block of at most 128 x 128, one thread block, the
// block resident in shared memory.
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
//  3. Elimination without pivoting on P^T A Q^T in that order, by the blocked
//     path below (its leading pivots up to order r are nonzero).  When the
//     order of phase 2 equals the row order of phase 1, phase 1 already holds
//     this factorisation and phase 3 is skipped.
// Before phase 1 the kernel tries the generic case: when every leading
// principal minor of order <= min(m, n) is nonzero, R is the identity pattern
// (rho(k, t) = min(k, t)), Algorithm 1 meets the pivots on the diagonal and
// P = Q = I, so the result is the LU factorisation without pivoting.  It runs
// blocked (see generic_lu) and hands over to the three phases at the first
// zero pivot, before anything is written to global memory.
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
// word selection by value, not by index, so that masks can stay in registers
__device__ __forceinline__ bool has(const Mask &a, int i)
{
    return ((i < 64 ? a.w[0] : a.w[1]) >> (i & 63)) & 1;
}
__device__ __forceinline__ void set(Mask &a, int i)
{
    const uint64_t bit = 1ull << (i & 63);
    if (i < 64) a.w[0] |= bit;
    else a.w[1] |= bit;
}
__device__ __forceinline__ Mask andnot(const Mask &a, const Mask &b)
{
    return Mask{{a.w[0] & ~b.w[0], a.w[1] & ~b.w[1]}};
}
__device__ __forceinline__ int first(const Mask &a)
{
    return a.w[0] ? __ffsll(a.w[0]) - 1 : 64 + __ffsll(a.w[1]) - 1;
}
// the lowest k (>= 0) set bits of a 32- / 64-bit word: keep the bits up to
// the k-th set one, found with __fns (n-th set bit)
__device__ __forceinline__ uint32_t lowest32(uint32_t x, int k)
{
    if (k <= 0) return 0u;
    if (k >= __popc(x)) return x;
    const unsigned pos = __fns(x, 0, k);   // position of the k-th set bit
    return x & (uint32_t)((2ull << pos) - 1ull);
}
__device__ __forceinline__ uint64_t lowest64(uint64_t x, int k)
{
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    const int cl = __popc(lo);
    if (k <= cl) return lowest32(lo, k);
    return lo | ((uint64_t)lowest32(hi, k - cl) << 32);
}
// the lowest `cnt` members of a, in O(1)
__device__ __forceinline__ Mask lowest(const Mask &a, int cnt)
{
    const int c0 = __popcll(a.w[0]);
    if (cnt <= c0) return Mask{{lowest64(a.w[0], cnt), 0}};
    return Mask{{a.w[0], lowest64(a.w[1], cnt - c0)}};
}

// Algorithm 1's order of the ones of R inside rows x cols, as an explicit
// stack (no device recursion): a frame splits its rows and columns at
// floor(half) and visits A1, F, G, R in turn, each child returning the rows
// and columns its pivots used.
//
// Shortcut: when the ones inside a frame have increasing columns in row order
// (no two of them form a descent), Algorithm 1 meets them in row order, so the
// frame emits them at once.  Induction on the split: with no descent, F (top
// rows, right columns) and G (bottom rows, left columns) cannot both hold a
// one, and A1 < F < R and A1 < G < R in row order; each quadrant is again
// descent-free.  Generic rank profiles, and frames with at most one one, end
// here after a single pass over their rows.
struct Frame {
    Mask rows, cols, rt, rb, cl, cr;
    Mask r1, c1, c2, r3;
    Mask ur, uc;        // rows / columns used so far by this frame
    int stage;
};
constexpr int MAX_DEPTH = 20;

static_assert(LM == 128, "row and column sets are two 64-bit words");

// the first k (0 <= k <= 128) indices
__device__ __forceinline__ Mask prefix_mask(int k)
{
    return Mask{{k >= 64 ? ~0ull : (1ull << k) - 1ull,
                 k >= 128 ? ~0ull : (k > 64 ? (1ull << (k - 64)) - 1ull : 0ull)}};
}

// prow32[w] bit b: row 32 w + b holds a one of R (set by the caller's warps)
__device__ int order_pivots(Frame *stk, const int32_t *col_of_row, const int32_t *row_of_col,
                            const uint32_t *prow32, int m, int n, int32_t *ord_row,
                            int32_t *ord_col)
{
    int count = 0;
    int top = 0;
    stk[0].rows = prefix_mask(m);
    stk[0].cols = prefix_mask(n);
    stk[0].stage = 0;
    Mask ret_r{{0, 0}}, ret_c{{0, 0}};   // used masks returned by the last popped frame
    const Mask prow_mask{{(uint64_t)prow32[0] | ((uint64_t)prow32[1] << 32),
                          (uint64_t)prow32[2] | ((uint64_t)prow32[3] << 32)}};
    // The current frame lives in registers: it is copied in once per pass
    // and written back only when a child is pushed above it (a popped frame is
    // dropped).  Reading and writing its fields in shared memory one by one was
    // a chain of dependent accesses on this single thread.
    while (top >= 0) {
        Frame f = stk[top];
        if (f.stage == 0) {
            f.ur = Mask{{0, 0}};
            f.uc = Mask{{0, 0}};
            // ones of R inside the frame, in row order: descent-free?
            bool mono = true;
            int lastc = -1;
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                if (!mono) break;
                uint64_t bits = f.rows.w[w] & prow_mask.w[w];
                while (bits) {
                    const int i = 64 * w + __ffsll(bits) - 1;
                    bits &= bits - 1;
                    const int c = col_of_row[i];
                    if (c >= 0 && has(f.cols, c)) {
                        if (c < lastc) { mono = false; break; }
                        lastc = c;
                    }
                }
            }
            if (mono) {
#pragma unroll
                for (int w = 0; w < 2; ++w) {
                    uint64_t bits = f.rows.w[w] & prow_mask.w[w];
                    while (bits) {
                        const int i = 64 * w + __ffsll(bits) - 1;
                        bits &= bits - 1;
                        const int c = col_of_row[i];
                        if (c >= 0 && has(f.cols, c)) {
                            ord_row[count] = i; ord_col[count] = c; ++count;
                            set(f.ur, i); set(f.uc, c);
                        }
                    }
                }
                ret_r = f.ur; ret_c = f.uc;
                --top;
                continue;
            }
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
            stk[top] = f;
            stk[top + 1].rows = f.rt;                      // A1
            stk[top + 1].cols = f.cl;
            stk[top + 1].stage = 0;
            ++top;
            continue;
        }
        // a child just returned (ret_r, ret_c)
        f.ur.w[0] |= ret_r.w[0]; f.ur.w[1] |= ret_r.w[1];
        f.uc.w[0] |= ret_c.w[0]; f.uc.w[1] |= ret_c.w[1];
        if (f.stage < 4 && top + 1 >= MAX_DEPTH) return -1;
        Mask crows, ccols;
        if (f.stage == 1) {
            f.r1 = ret_r; f.c1 = ret_c;
            crows = andnot(f.rt, f.r1); ccols = f.cr;      // F
        } else if (f.stage == 2) {
            f.c2 = ret_c;
            crows = f.rb; ccols = andnot(f.cl, f.c1);      // G
        } else if (f.stage == 3) {
            f.r3 = ret_r;
            crows = andnot(f.rb, f.r3); ccols = andnot(f.cr, f.c2);   // R
        } else {
            ret_r = f.ur; ret_c = f.uc;
            --top;
            continue;
        }
        ++f.stage;
        stk[top] = f;
        stk[top + 1].rows = crows;
        stk[top + 1].cols = ccols;
        stk[top + 1].stage = 0;
        ++top;
        if (top >= MAX_DEPTH) return -1;
    }
    return count;
}

struct LeafShared {
    uint32_t W[LM * LD];                 // staging of the final block
    uint32_t cand[2][NW][LM];            // per-warp candidate pivot rows (double buffered)
    uint32_t pbuf[2][LM];                // pivot row of the reordered elimination
    int32_t piv_row[LM], piv_col[LM];
    int32_t col_of_row[LM], row_of_col[LM];
    int32_t ord_row[LM], ord_col[LM];
    int32_t perm_p[LM], perm_q[LM];
    uint32_t prow32[LM / 32];            // rows holding a pivot, as bits
    uint32_t dval[LM], inv_d[LM], cval[LM], inv_c[LM];
    Frame stk[MAX_DEPTH];
    unsigned long long step_bar;         // phase k completes when every warp has offered its step-k candidate
    int key[3];
    int r;
    int same;
    int abort;
    int gfail;
};

static_assert(offsetof(LeafShared, pbuf) % 16 == 0 && (LM * 4) % 16 == 0,
              "pivot-row buffer rows must be 16-byte aligned");

constexpr int NOKEY = 0x7FFFFFFF;
constexpr uint32_t STEP_WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ int g_leaf_error = 0;   // set when a step wait gives up

// Wait for phase `parity` of the step barrier (at most `limit` tries; false
// if this or another warp gave up).
__device__ __forceinline__ bool step_wait(uint32_t bar, uint32_t parity, volatile int *abort,
                                          uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 63) == 63 && *abort) return false;
    }
    *abort = 1;
    atomicExch(&g_leaf_error, 1);
    return false;
}
constexpr int MAXC = LM / 32;  // column slots per lane for the widest block

// (d w - f q) mod p
template <bool SMALLP>
__device__ __forceinline__ uint32_t ff_update(uint32_t d, uint32_t w, uint32_t f, uint32_t q,
                                              const Field &F, const Field32 &F32)
{
    if (SMALLP) {
        // p < 2^16: t = d w reduced only to [0, 2p), then t + f (p - q)
        // <= 2p - 1 + (p - 1) p < 2^32 takes a single full reduction
        const uint32_t dw = d * w;
        const uint32_t t = dw - __umulhi(dw, F32.mu) * F32.p;
        return reduce32(t + f * (F32.p - q), F32);
    }
    return mul_sub_mul_mod(d, w, f, q, F);
}

// The phase-1 update d w - f q: for p > 2^16 on residues in Montgomery form
// (the result stays in that form, one reduction of d w + f (p - q) < 2 p^2)
template <bool SMALLP>
__device__ __forceinline__ uint32_t ff_step(uint32_t d, uint32_t w, uint32_t f, uint32_t q,
                                            const Field &F, const Field32 &F32)
{
    if (SMALLP) return ff_update<true>(d, w, f, q, F, F32);
    return fold(mont_redc((uint64_t)d * w + (uint64_t)f * (F.p - q), F), F.p);
}

template <bool SMALLP>
__device__ __forceinline__ uint32_t scale(uint32_t d, uint32_t w, const Field &F, const Field32 &F32)
{
    if (SMALLP) return reduce32(d * w, F32);
    return mul_mod(d, w, F);
}

template <int CPL>
__device__ __forceinline__ uint32_t pick(const uint32_t (&v)[CPL], int s)
{
    uint32_t x = v[0];
#pragma unroll
    for (int t = 1; t < CPL; ++t)
        if (s == t) x = v[t];
    return x;
}

// Block-wide helpers for 512 threads: warp 0 turns a per-row flag into the
// positions of the flagged rows (exclusive prefix counts).
__device__ __forceinline__ int warp_prefix_count(bool flag, int lane, int &total)
{
    const unsigned b = __ballot_sync(0xFFFFFFFFu, flag);
    total = __popc(b);
    return __popc(b & ((1u << lane) - 1u));
}

// Warp 0: exclusive prefix products c_k = d_0 ... d_{k-1} of dval[0..r).
__device__ void prefix_products(LeafShared &S, int r, int lane, const Field &F)
{
    // lane owns entries 4 lane .. 4 lane + 3
    uint32_t loc[MAXC];
    uint32_t prod = 1;
#pragma unroll
    for (int t = 0; t < MAXC; ++t) {
        const int k = MAXC * lane + t;
        loc[t] = prod;                         // product of this lane's earlier entries
        if (k < r) prod = mul_mod(prod, S.dval[k], F);
    }
    // exclusive scan of the lane products
    uint32_t incl = prod;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl = mul_mod(incl, v, F);
    }
    uint32_t excl = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
    if (lane == 0) excl = 1;
#pragma unroll
    for (int t = 0; t < MAXC; ++t) {
        const int k = MAXC * lane + t;
        if (k < r) S.cval[k] = mul_mod(excl, loc[t], F);
    }
}

// Sum of up to 2^16 products of residues held exactly: one 64-bit word for
// p <= 2^16 (products < 2^32), else a = a_hi 2^16 + a_lo in two words.
template <bool SMALLP>
struct LAcc {
    uint64_t lo = 0, hi = 0;
    __device__ __forceinline__ void add(uint32_t a, uint32_t b)
    {
        if (SMALLP) {
            lo += (uint64_t)a * b;          // one widening multiply-add
        } else {
            lo += (uint64_t)(a & 0xFFFFu) * b;
            hi += (uint64_t)(a >> 16) * b;
        }
    }
    __device__ __forceinline__ uint32_t value(const Field &F, uint32_t w16) const
    {
        if (SMALLP) return reduce64(lo, F);
        return add_mod(reduce64(lo, F), mul_mod(reduce64(hi, F), w16, F), F.p);
    }
};

constexpr int PB = 16;   // panel width of the generic path

// Blocked LU without pivoting of the m x n block, staged in S.W.  Per panel of
// PB pivot columns: (1) fraction-free elimination of the panel columns by the
// warps that hold its rows (a lane per row), one named barrier per step and no
// inverse on this path; (2) the panel's pivot values d_k, their prefix
// products c_k and both inverses, in parallel, then normalisation to L21 and
// U11; (3) U12 = L11^{-1} A12, one thread per column; (4) A22 -= L21 U12, each
// element one delayed reduction.  Returns false, with A untouched, at the first
// zero pivot (the rank profile is not generic).
//
// With row / column maps (rowmap[i], colmap[j]: original row and column of
// position i, j) it factors P^T A Q^T instead, taking kcap pivots: phase 3 of
// the general path, whose pivots in Algorithm 1's order are nonzero by
// construction (the leading minors of P^T A Q^T up to order r are products of
// U's diagonal).  pid / qid are reported as given.
template <bool SMALLP>
__device__ bool generic_lu(uint32_t *__restrict__ A, int m, int n, int64_t lda, const Field &F,
                           const Field32 &F32, LeafShared &S, int32_t *perm_p_out,
                           int32_t *perm_q_out, int32_t *info_out, int info_len,
                           volatile int32_t *host_info, int32_t seq,
                           const int32_t *rowmap = nullptr, const int32_t *colmap = nullptr,
                           int kcap = -1, int pid = 1, int qid = 1, bool left = false)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t p = F.p;
    const uint32_t w16 = (uint32_t)((1ull << 16) % p);
    uint32_t *W = S.W;
    // (3) rows [q0, q0 + bq) of columns [c0, c1) <- L_qq^{-1} of themselves
    // (U of block q), one thread per column; (4) rows below the block, same
    // columns, minus L_{.,q} U_q.  The right-looking form applies both to
    // every column right of a panel as soon as it is factored; the
    // left-looking form (the variant the base-case section mentions) defers
    // them: a panel receives the updates of all earlier panels just before it
    // is factored, and the columns past the last pivot at the end.  Both apply
    // the same updates to every element in the same order.
    auto solve_block = [&](int q0, int bq, int c0, int c1) {
        for (int c = c0 + tid; c < c1; c += LT) {
            uint32_t x[PB];
#pragma unroll
            for (int i = 0; i < PB; ++i) {
                if (i < bq) {
                    LAcc<SMALLP> acc;
#pragma unroll
                    for (int k = 0; k < PB; ++k)
                        if (k < i) acc.add(W[(q0 + i) * LD + q0 + k], x[k]);
                    x[i] = sub_mod(W[(q0 + i) * LD + c], acc.value(F, w16), p);
                    W[(q0 + i) * LD + c] = x[i];
                }
            }
        }
    };
    auto update_below = [&](int q0, int bq, int c0, int c1) {
        for (int i = q0 + bq + warp; i < m; i += NW)
            for (int c = c0 + lane; c < c1; c += 32) {
                LAcc<SMALLP> acc;
#pragma unroll
                for (int k = 0; k < PB; ++k)
                    if (k < bq) acc.add(W[i * LD + q0 + k], W[(q0 + k) * LD + c]);
                W[i * LD + c] = sub_mod(W[i * LD + c], acc.value(F, w16), p);
            }
    };
    // all panels before `upto` applied to columns [c0, c1)
    auto apply_earlier = [&](int upto, int c0, int c1) {
        for (int q0 = 0; q0 < upto; q0 += PB) {
            const int bq = upto - q0 < PB ? upto - q0 : PB;
            solve_block(q0, bq, c0, c1);
            __syncthreads();
            update_below(q0, bq, c0, c1);
            __syncthreads();
        }
    };
    // asynchronous 4-byte copies: the whole block is in flight at once
    for (int i = warp; i < m; i += NW) {
        const int64_t src = rowmap ? rowmap[i] : i;
        for (int j = lane; j < n; j += 32) {
            const unsigned dst = smem_addr(&W[i * LD + j]);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst),
                         "l"(&A[src * lda + (colmap ? colmap[j] : j)])
                         : "memory");
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (tid == 0) S.gfail = 0;
    __syncthreads();
    const int kmax = kcap >= 0 ? kcap : (m < n ? m : n);
    for (int j0 = 0; j0 < kmax; j0 += PB) {
        const int b = kmax - j0 < PB ? kmax - j0 : PB;
        if (left) apply_earlier(j0, j0, j0 + b);
        const int R = m - j0;                        // panel rows
        // four lanes per panel row, four of the panel's columns each: eight rows
        // per warp, pw warps (<= 16) hold the panel
        const int pw = (R + 7) / 8;
        // (1) fraction-free elimination of the panel columns
        if (warp < pw) {
            const int sub = lane & 3;                // this lane's columns 4 sub .. 4 sub + 3
            const int rel = warp * 8 + (lane >> 2);  // this lane's panel row
            const bool act = rel < R;
            uint32_t w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = 4 * sub + u;
                w[u] = (act && c < b) ? W[(j0 + rel) * LD + j0 + c] : 0u;
            }
            // the step loop stays rolled; the four column slots are unrolled with
            // predicated bodies, so w stays in registers
            bool fail = false;
#pragma unroll 1
            for (int k = 0; k < b && !fail; ++k) {
                // the pivot row's four columns of this lane move as one 16-byte word
                if (rel == k)
                    *reinterpret_cast<uint4 *>(&S.pbuf[k & 1][4 * sub]) =
                        make_uint4(w[0], w[1], w[2], w[3]);
                if (pw > 1) asm volatile("bar.sync 1, %0;" ::"r"(pw * 32) : "memory");
                else __syncwarp();
                const uint4 qv = *reinterpret_cast<const uint4 *>(&S.pbuf[k & 1][4 * sub]);
                const uint32_t q[4] = {qv.x, qv.y, qv.z, qv.w};
                const uint32_t d = S.pbuf[k & 1][k];
                fail = d == 0;
                if (tid == 0) S.dval[k] = d;
                // this row's value in column k sits in slot k & 3 of lane k >> 2 of the quad
                uint32_t mine = w[0];
#pragma unroll
                for (int u = 1; u < 4; ++u)
                    if ((k & 3) == u) mine = w[u];
                const uint32_t fk = __shfl_sync(0xFFFFFFFFu, mine, (lane & ~3) | (k >> 2));
                if (!fail && act && rel > k) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int c = 4 * sub + u;
                        const uint32_t nv = ff_update<SMALLP>(d, w[u], fk, q[u], F, F32);
                        w[u] = (c > k && c < b) ? nv : w[u];
                    }
                }
            }
            if (fail) {
                if (tid == 0) S.gfail = 1;
            } else {
                // (2) one inversion serves the panel: with D = prod d_k,
                // c_k = prod_{j<k} d_j and s_k = prod_{j>=k} d_j,
                // 1/d_k = c_k s_{k+1} / D and 1/c_k = s_k / D
                if (pw > 1) asm volatile("bar.sync 1, %0;" ::"r"(pw * 32) : "memory");
                else __syncwarp();
                if (warp == 0) {
                    const uint32_t dv = lane < b ? S.dval[lane] : 1u;
                    uint32_t pre = dv, suf = dv;                        // inclusive scans
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, pre, o);
                        const uint32_t t = __shfl_down_sync(0xFFFFFFFFu, suf, o);
                        if (lane >= o) pre = scale<SMALLP>(pre, v, F, F32);
                        if (lane + o < 32) suf = scale<SMALLP>(suf, t, F, F32);
                    }
                    uint32_t ce = __shfl_up_sync(0xFFFFFFFFu, pre, 1);    // c_lane
                    if (lane == 0) ce = 1;
                    uint32_t se = __shfl_down_sync(0xFFFFFFFFu, suf, 1);  // s_{lane+1}
                    if (lane == 31) se = 1;
                    // D^(p-2) = 1/D (Fermat), square and multiply
                    uint32_t iD = 1, base = __shfl_sync(0xFFFFFFFFu, pre, 31);
                    for (uint32_t e = p - 2; e; e >>= 1) {
                        if (e & 1u) iD = scale<SMALLP>(iD, base, F, F32);
                        base = scale<SMALLP>(base, base, F, F32);
                    }
                    if (lane < b) {
                        S.inv_d[lane] = scale<SMALLP>(scale<SMALLP>(ce, se, F, F32), iD, F, F32);
                        S.inv_c[lane] = scale<SMALLP>(suf, iD, F, F32);
                    }
                }
                if (pw > 1) asm volatile("bar.sync 1, %0;" ::"r"(pw * 32) : "memory");
                else __syncwarp();
                // L entries (c < rel) times 1/d_c; U entries of pivot rows (c >= rel)
                // times 1/c_rel
                if (act) {
                    const uint32_t ic = rel < b ? S.inv_c[rel] : 0u;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int c = 4 * sub + u;
                        if (c < b) {
                            const uint32_t sc = c < rel ? S.inv_d[c] : ic;
                            W[(j0 + rel) * LD + j0 + c] = scale<SMALLP>(w[u], sc, F, F32);
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (S.gfail) return false;
        if (!left) {
            // (3) U12 = L11^{-1} A12 on the pivot rows; (4) A22 -= L21 U12
            solve_block(j0, b, j0 + b, n);
            __syncthreads();
            update_below(j0, b, j0 + b, n);
            __syncthreads();
        }
    }
    if (left && kmax < n) apply_earlier(kmax, kmax, n);
    // the packed block (every entry is read into W before any is written), the
    // permutations and r
    __syncthreads();
    for (int i = warp; i < m; i += NW)
        for (int j = lane; j < n; j += 32) A[(int64_t)i * lda + j] = W[i * LD + j];
    for (int i = tid; i < m; i += LT) perm_p_out[i] = rowmap ? rowmap[i] : i;
    for (int j = tid; j < n; j += LT) perm_q_out[j] = colmap ? colmap[j] : j;
    if (tid == 0) {
        info_out[0] = kmax;
        if (info_len > 2) {
            info_out[1] = pid;
            info_out[2] = qid;
        }
        if (host_info) {
            host_info[1] = kmax;
            host_info[2] = pid;
            host_info[3] = qid;
            __threadfence_system();
            host_info[0] = seq;
        }
    }
    return true;
}

// CPL column slots per lane (block width <= 32 CPL), RPW row slots per warp
// (block height <= NW RPW): only slots that can hold data are compiled in.
// The base case on the block at A with the thread block's shared memory S:
// the body of leaf_kernel, also run by the node kernel for its four blocks.
template <bool SMALLP, int CPL, int RPW>
__device__ void leaf_run(LeafShared &S, uint32_t *__restrict__ A, int m, int n, int64_t lda,
                         Field F, int32_t *perm_p_out, int32_t *perm_q_out, int32_t *info_out,
                         int info_len, volatile int32_t *host_info, int32_t seq, int try_generic,
                         uint32_t wait_limit, int left_looking)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t p = F.p;
    const Field32 F32{p, 0xFFFFFFFFu / p};
    if (try_generic && generic_lu<SMALLP>(A, m, n, lda, F, F32, S, perm_p_out, perm_q_out,
                                          info_out, info_len, host_info, seq, nullptr, nullptr,
                                          -1, 1, 1, left_looking != 0))
        return;
    __syncthreads();   // the generic attempt is over: S belongs to the three phases now

    // this warp's rows warp + NW t and this lane's columns lane + 32 s, in registers
    uint32_t w[RPW][CPL];
#pragma unroll
    for (int t = 0; t < RPW; ++t) {
        const int i = warp + NW * t;
#pragma unroll
        for (int s = 0; s < CPL; ++s) {
            const int j = lane + 32 * s;
            const uint32_t a = (i < m && j < n) ? A[(int64_t)i * lda + j] : 0u;
            w[t][s] = SMALLP ? a : to_mont(a, F);
        }
    }
    for (int i = tid; i < LM; i += LT) {
        S.col_of_row[i] = -1;
        S.row_of_col[i] = -1;
    }
    const uint32_t bar = smem_addr(&S.step_bar);
    if (tid == 0) {
        S.key[0] = NOKEY;
        S.abort = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(LT / 32) : "memory");
    }
    uint32_t live = 0;   // bit s: column lane + 32 s is not a pivot column yet
#pragma unroll
    for (int s = 0; s < CPL; ++s)
        if (lane + 32 * s < n) live |= 1u << s;
    // warp-uniform loop bounds: column slots in use, row slots below m
    const int ncl = (n + 31) / 32;
    const int tmax = warp < m ? (m - warp + NW - 1) / NW : 0;
    __syncthreads();

    // ---------------- phase 1: row-order fraction-free elimination --------
    // Step t: rows below the last pivot row are updated in registers, in row
    // order.  A warp's first row (at or below the pivot row + 1) with a live
    // nonzero is its candidate: as soon as it is known, the warp publishes the
    // row in cand[t & 1][warp], takes key[t % 3] down to (row, column) and
    // arrives on the step barrier; then it updates its remaining rows.  So a
    // step waits for every warp's first candidate row, not for all updates.
    // key[(t+1) % 3] is cleared during step t: every read of it happened before
    // the previous phase completed and every write comes after this one.
    // For p > 2^16 the registers hold Montgomery forms (zero stays zero), and
    // the pivot values and the staged rows go back to plain residues.
    int r = 0, pi = -1, pc = 0, win = 0;
    uint32_t d = 0;
    bool failed = false;
    for (int step = 0;; ++step) {
        if (tid == 0) S.key[(step + 1) % 3] = NOKEY;
        const int t0 = pi < warp ? 0 : (pi - warp) / NW + 1;   // first own row below pi
        uint32_t prow[CPL];
#pragma unroll
        for (int s = 0; s < CPL; ++s)
            prow[s] = (pi >= 0 && s < ncl) ? S.cand[(step - 1) & 1][win][lane + 32 * s] : 0u;
        const int spc = pc >> 5, lpc = pc & 31;
        bool offered = false;
#pragma unroll
        for (int t = 0; t < RPW; ++t) {
            if (t < t0) continue;
            if (t >= tmax) break;
            if (pi >= 0) {
                // d w - f q also covers f = 0 (then it scales by d); every slot is
                // computed and kept by a select, so the updates overlap
                const uint32_t f = __shfl_sync(0xFFFFFFFFu, pick<CPL>(w[t], spc), lpc);
#pragma unroll
                for (int s = 0; s < CPL; ++s) {
                    const uint32_t nv = ff_step<SMALLP>(d, w[t][s], f, prow[s], F, F32);
                    w[t][s] = (s < ncl && ((live >> s) & 1)) ? nv : w[t][s];
                }
            }
            if (!offered) {
                int best = NOKEY;
#pragma unroll
                for (int s = CPL - 1; s >= 0; --s)
                    if (s < ncl && ((live >> s) & 1) && w[t][s] != 0) best = lane + 32 * s;
                best = __reduce_min_sync(0xFFFFFFFFu, best);
                if (best != NOKEY) {
#pragma unroll
                    for (int s = 0; s < CPL; ++s)
                        if (s < ncl) S.cand[step & 1][warp][lane + 32 * s] = w[t][s];
                    if (lane == 0) atomicMin(&S.key[step % 3], (warp + NW * t) * LM + best);
                    __syncwarp();
                    if (lane == 0)
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
                    offered = true;
                }
            }
        }
        if (!offered) {
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
        }
        if (!step_wait(bar, step & 1, &S.abort, wait_limit)) {
            failed = true;
            break;
        }
        const int kv = S.key[step % 3];
        if (kv == NOKEY) break;
        pi = kv / LM;
        pc = kv % LM;
        win = pi % NW;
        d = S.cand[step & 1][win][pc];
        if ((pc & 31) == lane) live &= ~(1u << (pc >> 5));
        if (tid == 0) {
            S.piv_row[r] = pi;
            S.piv_col[r] = pc;
            S.dval[r] = SMALLP ? d : from_mont(d, F);
            S.col_of_row[pi] = pc;
            S.row_of_col[pc] = pi;
        }
        ++r;
    }
    // every warp is past its last step wait: the step barrier is retired, so
    // that a later base case in the same thread block (the node kernel) may
    // initialise it afresh
    const bool any_failed = __syncthreads_or(failed);
    if (tid == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
    if (any_failed) {
        if (tid == 0) {
            info_out[0] = -1;
            if (host_info) {
                host_info[1] = -1;
                __threadfence_system();
                host_info[0] = seq;
            }
        }
        return;
    }

    // A zero block (r = 0, which deep in the recursion of a rank-deficient
    // matrix is the common case): P = Q = I and its packed form is the block
    // itself, which phase 1 has not touched, so only the outputs are written.
    if (r == 0) {
        for (int i = tid; i < m; i += LT) perm_p_out[i] = i;
        for (int j = tid; j < n; j += LT) perm_q_out[j] = j;
        if (tid == 0) {
            info_out[0] = 0;
            if (info_len > 2) {
                info_out[1] = 1;
                info_out[2] = 1;
            }
            if (host_info) {
                host_info[1] = 0;
                host_info[2] = 1;
                host_info[3] = 1;
                __threadfence_system();
                host_info[0] = seq;
            }
        }
        return;
    }

    // ---------------- phase 2: Algorithm 1's order of the pivots ----------
    // Pivots whose columns increase in row order are already in that order
    // (see order_pivots); otherwise thread 0 runs the quad recursion.
    bool descent = false;
    for (int t = tid; t + 1 < r; t += LT) descent |= S.piv_col[t] > S.piv_col[t + 1];
    if (warp < LM / 32) {   // pivot rows as bits, for the quad recursion
        const int i = 32 * warp + lane;
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, i < m && S.col_of_row[i] >= 0);
        if (lane == 0) S.prow32[warp] = b;
    }
    descent = __syncthreads_or(descent);
    if (descent) {
        if (tid == 0) {
            const int cnt = order_pivots(S.stk, S.col_of_row, S.row_of_col, S.prow32, m, n,
                                         S.ord_row, S.ord_col);
            int same = cnt == r ? 1 : -1;
            if (same > 0)
                for (int t = 0; t < r; ++t)
                    if (S.ord_row[t] != S.piv_row[t]) same = 0;
            S.same = same;
        }
    } else {
        for (int t = tid; t < r; t += LT) {
            S.ord_row[t] = S.piv_row[t];
            S.ord_col[t] = S.piv_col[t];
        }
        if (tid == 0) S.same = 1;
    }
    __syncthreads();
    const int same = S.same;
    if (same < 0) {                 // leave the block untouched, flag the error
        if (tid == 0) {
            info_out[0] = -1;
            if (host_info) {
                host_info[1] = -1;
                __threadfence_system();
                host_info[0] = seq;
            }
        }
        return;
    }
    // P, Q: pivots in order, then the other rows / columns increasing
    for (int t = tid; t < r; t += LT) {
        S.perm_p[t] = S.ord_row[t];
        S.perm_q[t] = S.ord_col[t];
    }
    if (warp == 0) {
        int base = 0;
        for (int c0 = 0; c0 < m; c0 += 32) {
            const int i = c0 + lane;
            const bool np = i < m && S.col_of_row[i] < 0;
            int tot;
            const int pos = warp_prefix_count(np, lane, tot);
            if (np) S.perm_p[r + base + pos] = i;
            base += tot;
        }
    } else if (warp == 1) {
        int base = 0;
        for (int c0 = 0; c0 < n; c0 += 32) {
            const int j = c0 + lane;
            const bool np = j < n && S.row_of_col[j] < 0;
            int tot;
            const int pos = warp_prefix_count(np, lane, tot);
            if (np) S.perm_q[r + base + pos] = j;
            base += tot;
        }
    }
    __syncthreads();
    int pid = 1, qid = 1;
    for (int i = tid; i < m; i += LT) pid &= S.perm_p[i] == i;
    for (int j = tid; j < n; j += LT) qid &= S.perm_q[j] == j;
    pid = __syncthreads_and(pid);
    qid = __syncthreads_and(qid);

    // ---------------- phase 3: elimination without pivoting ---------------
    // P^T A Q^T in Algorithm 1's order by the blocked path (its r leading
    // pivots are nonzero), which also writes the block, P, Q and r
    if (!same) {
        __syncthreads();
        if (!generic_lu<SMALLP>(A, m, n, lda, F, F32, S, perm_p_out, perm_q_out, info_out,
                                info_len, host_info, seq, S.perm_p, S.perm_q, r, pid, qid,
                                left_looking != 0)) {
            if (tid == 0) {
                info_out[0] = -1;   // a zero pivot here contradicts the rank profile found
                if (host_info) {
                    host_info[1] = -1;
                    __threadfence_system();
                    host_info[0] = seq;
                }
            }
        }
        return;
    }

    // stage the rows in shared memory (original positions, phase 1's order is
    // Algorithm 1's)
#pragma unroll
    for (int t = 0; t < RPW; ++t) {
        const int i = warp + NW * t;
        if (i < m) {
#pragma unroll
            for (int s = 0; s < CPL; ++s)
                S.W[i * LD + lane + 32 * s] = SMALLP ? w[t][s] : from_mont(w[t][s], F);
        }
    }
    // ---------------- fix-up: divide U rows by c_k, L columns by d_k ------
    __syncthreads();
    if (warp == 0) prefix_products(S, r, lane, F);
    __syncthreads();
    for (int t = tid; t < 2 * r; t += LT) {
        if (t < r) S.inv_d[t] = inv_mod(S.dval[t], p);
        else S.inv_c[t - r] = inv_mod(S.cval[t - r], p);
    }
    __syncthreads();

    // write the packed block [L\U V; M 0] in P, Q order (phase 1's rows are in
    // original positions, its pivots in Algorithm 1's order): packed row i < r
    // is pivot row piv_row[i] over the columns perm_q, divided by c_i, from the
    // diagonal on; packed column j < r below the diagonal is pivot column
    // piv_col[j] over the rows perm_p, divided by d_j; the rest is zero (the
    // rank is r).  A warp per packed row, so the branches are uniform but for
    // the first r lanes.
    for (int i = warp; i < m; i += NW) {
        const bool urow = i < r;
        const uint32_t ic = urow ? S.inv_c[i] : 0u;
        const uint32_t *wu = S.W + (urow ? S.piv_row[i] : 0) * LD;
        const uint32_t *wl = S.W + S.perm_p[i] * LD;
        uint32_t *dst = A + (int64_t)i * lda;
        for (int j = lane; j < n; j += 32) {
            uint32_t v = 0;
            if (urow && j >= i) v = mul_mod(wu[S.perm_q[j]], ic, F);
            else if (j < r && i > j) v = mul_mod(wl[S.piv_col[j]], S.inv_d[j], F);
            dst[j] = v;
        }
    }
    for (int i = tid; i < m; i += LT) perm_p_out[i] = S.perm_p[i];
    for (int j = tid; j < n; j += LT) perm_q_out[j] = S.perm_q[j];
    if (tid == 0) {
        info_out[0] = r;
        if (info_len > 2) {
            info_out[1] = pid;
            info_out[2] = qid;
        }
        if (host_info) {
            host_info[1] = r;
            host_info[2] = pid;
            host_info[3] = qid;
            __threadfence_system();
            host_info[0] = seq;
        }
    }
}

}  // namespace
}  // namespace pluq
