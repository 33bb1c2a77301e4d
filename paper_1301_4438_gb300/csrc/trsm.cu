// TRSM of Sec. 2 on the GPU:  B <- L^{-1} B (L unit lower) and B <- B U^{-1}
// (U upper, nonzero diagonal).
//
// Triangles of at most WR = 128 rows are solved directly, in one launch, by
// blocks of BS = 32: every thread block inverts the (at most four) 32 x 32
// diagonal blocks of the triangle, then for k = 0, 1, ... computes, for its
// 32 right-hand sides,
//   left:  Y = B_k - L_{k,<k} X_{<k},   X_k = L_kk^{-1} Y
//   right: Y = B_k - X_{<k} U_{<k,k},   X_k = Y U_kk^{-1}.
// The substitution chain is thus 32 rows long (inside the diagonal inverses,
// shared by all right-hand sides) instead of r, and the rest is dot products
// on shared memory with delayed reduction.
//
// Larger triangles are inverted first and the solve becomes one modular
// product: the 128 x 128 diagonal blocks are inverted by the direct solver
// with the identity as right-hand side (all blocks in one launch), then merged
// pairwise, log2(r/128) levels, with
//     [L11 0; L21 L22]^-1 = [X11 0; -X22 L21 X11  X22],
//     [U11 U12; 0 U22]^-1 = [X11 -X11 U12 X22; 0 X22],
// every pair of a level in one batched product launch; the solve is X B (or
// B X).  The inverse costs r^3/3 field operations, small next to the r^2 N of
// the solve for the shapes Algorithm 1 produces.
#include "common.cuh"

namespace pluq {
namespace {

constexpr int WR = 128;            // largest triangle solved directly
constexpr int BS = 32;             // diagonal block of the direct solver
constexpr int NBLK = WR / BS;      // diagonal blocks of the largest triangle
constexpr int NRHS = 32;           // right-hand sides per thread block
constexpr int TT = 512;            // threads per block
constexpr int NWARP = TT / 32;     // warps per block
constexpr int RPW = BS / NWARP;    // rows (left) or right-hand sides (right) per warp
constexpr int TB = WR;             // diagonal blocks the inverses start from

// Dot product sum_l a_l b_l of residues (a, b < p), exact until read.
// p <= 2^16: one 64-bit word (each product < 2^32).  Otherwise b is split as
// b_hi 2^16 + b_lo into two words (products < 2^47, so up to 2^17 terms) and
// w16 = 2^16 mod p recombines them.  Callers pass the operand shared by
// several sums as b, so its split is computed once.
template <bool SMALLP>
struct Dot;

template <>
struct Dot<true> {
    uint64_t s = 0;
    __device__ __forceinline__ void add(uint32_t a, uint32_t b) { s += (uint64_t)a * b; }
    __device__ __forceinline__ uint32_t value(const Field &F, uint32_t) const
    {
        return reduce64(s, F);
    }
};

template <>
struct Dot<false> {
    uint64_t lo = 0, hi = 0;
    __device__ __forceinline__ void add(uint32_t a, uint32_t b)
    {
        lo += (uint64_t)a * (b & 0xFFFFu);
        hi += (uint64_t)a * (b >> 16);
    }
    __device__ __forceinline__ uint32_t value(const Field &F, uint32_t w16) const
    {
        return add_mod(reduce64(lo, F), mul_mod(reduce64(hi, F), w16, F), F.p);
    }
};

// 4-byte asynchronous global -> shared copy: every element of a staged
// triangle is in flight at once instead of one row's latency after another.
__device__ __forceinline__ void cp_async4(uint32_t *dst, const uint32_t *src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Shared memory of the direct solvers (32-bit words).  Strides are those of
// the largest triangle, so nothing depends on r; rows or columns at or past r
// are never staged and every value read from them is multiplied by zero or
// discarded.
constexpr size_t SM_TRI = (size_t)WR * WR;            // the triangle, row stride WR
constexpr size_t SM_INV = (size_t)NBLK * BS * BS;     // inverses of the diagonal blocks
constexpr size_t SM_X = (size_t)WR * NRHS;            // right-hand sides / unknowns
constexpr size_t SM_Y = (size_t)BS * NRHS;            // Y of the current block
constexpr size_t SM_LEFT = (SM_TRI + SM_INV + SM_X + SM_Y) * 4;
constexpr size_t SM_RIGHT = (SM_TRI + SM_INV + SM_X + SM_Y + WR) * 4;

// B (r x N) <- L^{-1} B, L unit lower (diagonal not read); thread block x
// takes columns [32 x, 32 x + 32) of B.  IDENT: blockIdx.y picks the diagonal
// block of L at o = blockIdx.y * blk (size min(blk, r - o)) and B receives its
// inverse there (the right-hand side is the identity).
template <bool SMALLP, bool IDENT>
__global__ void __launch_bounds__(TT) trsm_left_blocked(const uint32_t *__restrict__ L, int64_t ldl,
                                                         uint32_t *__restrict__ B, int64_t ldb,
                                                         int r, int64_t N, Field F, int blk)
{
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t *Ls = sm;                  // [WR][WR]
    uint32_t *Li = Ls + SM_TRI;         // [NBLK][BS][BS]
    uint32_t *Xs = Li + SM_INV;         // [WR][NRHS]
    uint32_t *Ys = Xs + SM_X;           // [BS][NRHS]
    if (IDENT) {
        const int64_t o = (int64_t)blockIdx.y * blk;
        L += o * (ldl + 1);
        B += o * (ldb + 1);
        r = min(blk, (int)(r - o));
        N = r;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t j = (int64_t)blockIdx.x * NRHS + lane;    // this lane's column of B
    const uint32_t w16 = (uint32_t)((1ull << 16) % F.p);
    for (int i = warp; i < r; i += NWARP) {
        for (int c = lane; c < i; c += 32) cp_async4(&Ls[i * WR + c], &L[(int64_t)i * ldl + c]);
        if (IDENT) Xs[i * NRHS + lane] = i == j ? 1u : 0u;
        else if (j < N) cp_async4(&Xs[i * NRHS + lane], &B[(int64_t)i * ldb + j]);
        else Xs[i * NRHS + lane] = 0u;
    }
    cp_async_wait_all();
    __syncthreads();

    // inverse of diagonal block `warp`: lane c computes its column c,
    // x_c = 1, x_i = -sum_{c <= l < i} L_il x_l (i > c), zero above
    const int nblk = (r + BS - 1) / BS;
    if (warp < nblk) {
        const int b0 = warp * BS;
        uint32_t x[BS];
#pragma unroll
        for (int i = 0; i < BS; ++i) {
            Dot<SMALLP> acc;
#pragma unroll
            for (int l = 0; l < i; ++l) acc.add(Ls[(b0 + i) * WR + b0 + l], x[l]);
            const uint32_t v = sub_mod(0u, acc.value(F, w16), F.p);
            x[i] = (i < lane || b0 + i >= r) ? 0u : (i == lane ? 1u : v);
        }
#pragma unroll
        for (int i = 0; i < BS; ++i) Li[(b0 + i) * BS + lane] = x[i];
    }
    __syncthreads();

    for (int k = 0; k < nblk; ++k) {
        const int b0 = k * BS;
        // Y = B_k - L_{k,<k} X_{<k}: rows b0 + warp + NWARP q, column lane
        Dot<SMALLP> acc[RPW];
        for (int l = 0; l < b0; ++l) {
            const uint32_t xv = Xs[l * NRHS + lane];
#pragma unroll
            for (int q = 0; q < RPW; ++q) acc[q].add(Ls[(b0 + warp + NWARP * q) * WR + l], xv);
        }
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int i = warp + NWARP * q;
            Ys[i * NRHS + lane] = sub_mod(Xs[(b0 + i) * NRHS + lane], acc[q].value(F, w16), F.p);
        }
        __syncthreads();
        // X_k = L_kk^{-1} Y (the inverse is zero above its diagonal and in
        // the rows and columns past r, so the full 32-term sums are exact)
        Dot<SMALLP> acc2[RPW];
#pragma unroll 8
        for (int l = 0; l < BS; ++l) {
            const uint32_t yv = Ys[l * NRHS + lane];
#pragma unroll
            for (int q = 0; q < RPW; ++q) acc2[q].add(Li[(b0 + warp + NWARP * q) * BS + l], yv);
        }
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int i = b0 + warp + NWARP * q;
            if (i < r) Xs[i * NRHS + lane] = acc2[q].value(F, w16);
        }
        __syncthreads();
    }
    if (j < N)
        for (int i = warp; i < r; i += NWARP) B[(int64_t)i * ldb + j] = Xs[i * NRHS + lane];
}

// B (M x r) <- B U^{-1}, U upper with nonzero diagonal; thread block x takes
// rows [32 x, 32 x + 32) of B.  IDENT: as for the left solve, B receives the
// inverse of the diagonal block blockIdx.y of U.
template <bool SMALLP, bool IDENT>
__global__ void __launch_bounds__(TT) trsm_right_blocked(const uint32_t *__restrict__ U, int64_t ldu,
                                                          uint32_t *__restrict__ B, int64_t ldb,
                                                          int64_t M, int r, Field F, int blk)
{
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t *Us = sm;                  // [WR][WR]
    uint32_t *Ui = Us + SM_TRI;         // [NBLK][BS][BS]
    uint32_t *Xs = Ui + SM_INV;         // [NRHS][WR]
    uint32_t *Ys = Xs + SM_X;           // [NRHS][BS]
    uint32_t *dinv = Ys + SM_Y;         // [WR]
    if (IDENT) {
        const int64_t o = (int64_t)blockIdx.y * blk;
        U += o * (ldu + 1);
        B += o * (ldb + 1);
        r = min(blk, (int)(r - o));
        M = r;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t m0 = (int64_t)blockIdx.x * NRHS;
    const uint32_t w16 = (uint32_t)((1ull << 16) % F.p);
    for (int i = warp; i < r; i += NWARP)
        for (int c = i + lane; c < r; c += 32) cp_async4(&Us[i * WR + c], &U[(int64_t)i * ldu + c]);
    for (int q = warp; q < NRHS; q += NWARP) {
        const int64_t m = m0 + q;
        for (int c = lane; c < r; c += 32) {
            if (IDENT) Xs[q * WR + c] = m == c ? 1u : 0u;
            else if (m < M) cp_async4(&Xs[q * WR + c], &B[m * ldb + c]);
            else Xs[q * WR + c] = 0u;
        }
    }
    cp_async_wait_all();
    __syncthreads();
    for (int t = threadIdx.x; t < r; t += TT) dinv[t] = pow_mod(Us[t * WR + t], F.p - 2, F);
    __syncthreads();

    // inverse of diagonal block `warp`: lane c computes its column c,
    // x_c = 1 / U_cc, x_i = -(sum_{i < l <= c} U_il x_l) / U_ii (i < c), zero below
    const int nblk = (r + BS - 1) / BS;
    if (warp < nblk) {
        const int b0 = warp * BS;
        uint32_t x[BS];
#pragma unroll
        for (int i = BS - 1; i >= 0; --i) {
            Dot<SMALLP> acc;
#pragma unroll
            for (int l = i + 1; l < BS; ++l) acc.add(Us[(b0 + i) * WR + b0 + l], x[l]);
            const uint32_t d = b0 + i < r ? dinv[b0 + i] : 0u;
            const uint32_t v = mul_mod(sub_mod(0u, acc.value(F, w16), F.p), d, F);
            x[i] = (i > lane || b0 + i >= r) ? 0u : (i == lane ? d : v);
        }
#pragma unroll
        for (int i = 0; i < BS; ++i) Ui[(b0 + i) * BS + lane] = x[i];
    }
    __syncthreads();

    for (int k = 0; k < nblk; ++k) {
        const int b0 = k * BS;
        // Y = B_k - X_{<k} U_{<k,k}: right-hand sides warp + NWARP q, column b0 + lane
        Dot<SMALLP> acc[RPW];
        for (int l = 0; l < b0; ++l) {
            const uint32_t uv = Us[l * WR + b0 + lane];
#pragma unroll
            for (int q = 0; q < RPW; ++q) acc[q].add(Xs[(warp + NWARP * q) * WR + l], uv);
        }
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int m = warp + NWARP * q;
            Ys[m * BS + lane] = sub_mod(Xs[m * WR + b0 + lane], acc[q].value(F, w16), F.p);
        }
        __syncthreads();
        // X_k = Y U_kk^{-1} (the inverse is zero below its diagonal and in the
        // rows and columns past r)
        Dot<SMALLP> acc2[RPW];
#pragma unroll 8
        for (int l = 0; l < BS; ++l) {
            const uint32_t uv = Ui[(b0 + l) * BS + lane];
#pragma unroll
            for (int q = 0; q < RPW; ++q) acc2[q].add(Ys[(warp + NWARP * q) * BS + l], uv);
        }
        if (b0 + lane < r) {
#pragma unroll
            for (int q = 0; q < RPW; ++q)
                Xs[(warp + NWARP * q) * WR + b0 + lane] = acc2[q].value(F, w16);
        }
        __syncthreads();
    }
    for (int q = warp; q < NRHS; q += NWARP) {
        const int64_t m = m0 + q;
        if (m < M)
            for (int c = lane; c < r; c += 32) B[m * ldb + c] = Xs[q * WR + c];
    }
}

// left: B (r x other) <- T^{-1} B; otherwise B (other x r) <- B T^{-1}.  With
// `blocks` > 0 the diagonal blocks of size min(WR, .) of T are inverted into B
// instead (other is ignored).
template <bool SMALLP>
pluq_status launch_trsm_blocked(bool left, const uint32_t *T, int64_t ldt, Blk B, int64_t other,
                                int r, Field F, int64_t blocks, cudaStream_t st)
{
    const int rr = blocks > 0 ? (r < WR ? r : WR) : r;
    const int64_t rhs = blocks > 0 ? rr : other;
    const int64_t nb = blocks > 0 ? blocks : 1;
    const dim3 grid((unsigned)ceil_div(rhs, NRHS), (unsigned)nb);
#define PLUQ_TRSM_ATTR(K, BYTES)                                                                   \
    {                                                                                             \
        static std::atomic<uint64_t> attr{0};                                                     \
        if (!smem_attr_once((const void *)K, (BYTES), attr)) return PLUQ_ECUDA;                    \
    }
    if (left && blocks > 0) {
        PLUQ_TRSM_ATTR((trsm_left_blocked<SMALLP, true>), SM_LEFT)
        trsm_left_blocked<SMALLP, true><<<grid, TT, SM_LEFT, st>>>(T, ldt, B.ptr, B.ld, r, 0, F, WR);
    } else if (left) {
        PLUQ_TRSM_ATTR((trsm_left_blocked<SMALLP, false>), SM_LEFT)
        trsm_left_blocked<SMALLP, false><<<grid, TT, SM_LEFT, st>>>(T, ldt, B.ptr, B.ld, r, other, F, 0);
    } else if (blocks > 0) {
        PLUQ_TRSM_ATTR((trsm_right_blocked<SMALLP, true>), SM_RIGHT)
        trsm_right_blocked<SMALLP, true><<<grid, TT, SM_RIGHT, st>>>(T, ldt, B.ptr, B.ld, 0, r, F, WR);
    } else {
        PLUQ_TRSM_ATTR((trsm_right_blocked<SMALLP, false>), SM_RIGHT)
        trsm_right_blocked<SMALLP, false><<<grid, TT, SM_RIGHT, st>>>(T, ldt, B.ptr, B.ld, other, r, F, 0);
    }
#undef PLUQ_TRSM_ATTR
    return last_launch();
}

pluq_status trsm_direct(bool left, const uint32_t *T, int64_t ldt, Blk B, int64_t other, int r,
                        Field F, int64_t blocks, cudaStream_t st)
{
    if (F.p <= 65536u) return launch_trsm_blocked<true>(left, T, ldt, B, other, r, F, blocks, st);
    return launch_trsm_blocked<false>(left, T, ldt, B, other, r, F, blocks, st);
}

// Triangles of order r <= RS: one thread per right-hand side, the triangle
// in shared memory, substitution in registers with a reduction per term.
// Thread blocks [0, nl) solve the left problem B <- L^{-1} B (thread = column
// of B), the others the right problem B <- B U^{-1} (thread = row of B), so a
// node's two solves D and E take one launch.
constexpr int RS = 16;
constexpr int ST = 128;   // threads per block of the small solver

struct SmallSolve {
    const uint32_t *T;
    int64_t ldt;
    uint32_t *B;
    int64_t ldb;
    int r;
    int64_t other;        // number of right-hand sides
};

__global__ void __launch_bounds__(ST) trsm_small_kernel(SmallSolve ls, SmallSolve rs, int nl,
                                                        Field F)
{
    __shared__ uint32_t Ts[RS][RS + 1];
    __shared__ uint32_t dinv[RS];
    const bool left = (int)blockIdx.x < nl;
    const SmallSolve &t = left ? ls : rs;
    const int r = t.r;
    const uint32_t p = F.p;
    for (int e = threadIdx.x; e < r * r; e += ST) {
        const int i = e / r, c = e - (e / r) * r;
        Ts[i][c] = t.T[(int64_t)i * t.ldt + c];
    }
    __syncthreads();
    if (!left && (int)threadIdx.x < r) dinv[threadIdx.x] = inv_mod(Ts[threadIdx.x][threadIdx.x], p);
    __syncthreads();
    const int64_t idx = (int64_t)(left ? blockIdx.x : blockIdx.x - nl) * ST + threadIdx.x;
    if (idx >= t.other) return;
    uint32_t x[RS];
    if (left) {
        // x_i = b_i - sum_{l < i} L_il x_l
#pragma unroll
        for (int i = 0; i < RS; ++i)
            if (i < r) x[i] = t.B[(int64_t)i * t.ldb + idx];
#pragma unroll
        for (int i = 1; i < RS; ++i) {
            if (i >= r) break;
            uint32_t v = x[i];
#pragma unroll
            for (int l = 0; l < RS; ++l)
                if (l < i) v = sub_mod(v, mul_mod(Ts[i][l], x[l], F), p);
            x[i] = v;
        }
#pragma unroll
        for (int i = 0; i < RS; ++i)
            if (i < r) t.B[(int64_t)i * t.ldb + idx] = x[i];
    } else {
        // x_j = (b_j - sum_{l < j} x_l U_lj) / U_jj
        uint32_t *row = t.B + idx * t.ldb;
#pragma unroll
        for (int j = 0; j < RS; ++j)
            if (j < r) x[j] = row[j];
#pragma unroll
        for (int j = 0; j < RS; ++j) {
            if (j >= r) break;
            uint32_t v = x[j];
#pragma unroll
            for (int l = 0; l < RS; ++l)
                if (l < j) v = sub_mod(v, mul_mod(x[l], Ts[l][j], F), p);
            x[j] = mul_mod(v, dinv[j], F);
        }
#pragma unroll
        for (int j = 0; j < RS; ++j)
            if (j < r) row[j] = x[j];
    }
}

pluq_status launch_trsm_small(const SmallSolve *ls, const SmallSolve *rs, Field F, cudaStream_t st)
{
    const int64_t nl = ls ? ceil_div(ls->other, ST) : 0;
    const int64_t nr = rs ? ceil_div(rs->other, ST) : 0;
    if (nl + nr == 0) return PLUQ_OK;
    if (nl + nr > INT32_MAX) return PLUQ_EINVAL;
    const SmallSolve none{};
    prof::start(prof::TRI, st);
    trsm_small_kernel<<<(unsigned)(nl + nr), ST, 0, st>>>(ls ? *ls : none, rs ? *rs : none, (int)nl,
                                                          F);
    pluq_status s = last_launch();
    prof::stop(prof::TRI, st,
               (ls ? (double)ls->r * ls->r * ls->other : 0.0) +
                   (rs ? (double)rs->r * rs->r * rs->other : 0.0));
    return s;
}

}  // namespace

bool trsm_small_for(int64_t r) { return r > 0 && r <= RS; }

pluq_status trsm_pair_small(const uint32_t *L, int64_t ldl, Blk BL, int64_t rl, int64_t N,
                            const uint32_t *U, int64_t ldu, Blk BR, int64_t M, int64_t rr,
                            Field F, cudaStream_t st)
{
    SmallSolve ls{L, ldl, BL.ptr, BL.ld, (int)rl, N};
    SmallSolve rs{U, ldu, BR.ptr, BR.ld, (int)rr, M};
    const bool use_l = rl > 0 && N > 0, use_r = rr > 0 && M > 0;
    if ((use_l && rl > RS) || (use_r && rr > RS)) return PLUQ_EINVAL;
    return launch_trsm_small(use_l ? &ls : nullptr, use_r ? &rs : nullptr, F, st);
}

pluq_status tri_inv_lower_unit(const uint32_t *L, int64_t ldl, Blk X, int64_t r, Field F,
                               int kind, Arena &ar, cudaStream_t st)
{
    if (r <= 0) return PLUQ_OK;
    PLUQ_TRY(launch_zero(X, r, r, st));
    prof::start(prof::TRI, st);
    PLUQ_TRY(trsm_direct(true, L, ldl, X, 0, (int)r, F, ceil_div(r, TB), st));
    prof::stop(prof::TRI, st, 2.0 * (double)r * TB * TB / 3.0);
    if (r <= TB) return PLUQ_OK;
    size_t mark = ar.off;
    uint32_t *T = (uint32_t *)ar.take((size_t)r * r * sizeof(uint32_t));
    if (!T) return PLUQ_ENOMEM;
    for (int64_t s = TB; s < r; s *= 2) {
        const int64_t full = r / (2 * s);
        const int64_t rem = r - full * 2 * s;
        if (full > 0) {
            // T_t = L21 X11 ; X21 = -X22 T_t
            PLUQ_TRY(launch_mm(kind, Blk{T, s}, L + s * ldl, ldl, X.ptr, X.ld, s, s, s, F,
                               MM_ASSIGN, full, 2 * s * (ldl + 1), 2 * s * (X.ld + 1), s * s, ar,
                               st));
            PLUQ_TRY(launch_mm(kind, Blk{X.ptr + s * X.ld, X.ld}, X.ptr + s * (X.ld + 1), X.ld, T,
                               s, s, s, s, F, MM_NEG_ASSIGN, full, 2 * s * (X.ld + 1), s * s,
                               2 * s * (X.ld + 1), ar, st));
        }
        if (rem > s) {
            const int64_t o = full * 2 * s, s2 = rem - s;
            PLUQ_TRY(launch_mm(kind, Blk{T, s}, L + (o + s) * ldl + o, ldl, X.ptr + o * (X.ld + 1),
                               X.ld, s2, s, s, F, MM_ASSIGN, 1, 0, 0, 0, ar, st));
            PLUQ_TRY(launch_mm(kind, Blk{X.ptr + (o + s) * X.ld + o, X.ld},
                               X.ptr + (o + s) * (X.ld + 1), X.ld, T, s, s2, s, s2, F,
                               MM_NEG_ASSIGN, 1, 0, 0, 0, ar, st));
        }
    }
    ar.off = mark;
    return PLUQ_OK;
}

pluq_status tri_inv_upper(const uint32_t *U, int64_t ldu, Blk X, int64_t r, Field F, int kind,
                          Arena &ar, cudaStream_t st)
{
    if (r <= 0) return PLUQ_OK;
    PLUQ_TRY(launch_zero(X, r, r, st));
    prof::start(prof::TRI, st);
    PLUQ_TRY(trsm_direct(false, U, ldu, X, 0, (int)r, F, ceil_div(r, TB), st));
    prof::stop(prof::TRI, st, 2.0 * (double)r * TB * TB / 3.0);
    if (r <= TB) return PLUQ_OK;
    size_t mark = ar.off;
    uint32_t *T = (uint32_t *)ar.take((size_t)r * r * sizeof(uint32_t));
    if (!T) return PLUQ_ENOMEM;
    for (int64_t s = TB; s < r; s *= 2) {
        const int64_t full = r / (2 * s);
        const int64_t rem = r - full * 2 * s;
        if (full > 0) {
            // T_t = U12 X22 ; X12 = -X11 T_t
            PLUQ_TRY(launch_mm(kind, Blk{T, s}, U + s, ldu, X.ptr + s * (X.ld + 1), X.ld, s, s, s,
                               F, MM_ASSIGN, full, 2 * s * (ldu + 1), 2 * s * (X.ld + 1), s * s,
                               ar, st));
            PLUQ_TRY(launch_mm(kind, Blk{X.ptr + s, X.ld}, X.ptr, X.ld, T, s, s, s, s, F,
                               MM_NEG_ASSIGN, full, 2 * s * (X.ld + 1), s * s, 2 * s * (X.ld + 1),
                               ar, st));
        }
        if (rem > s) {
            const int64_t o = full * 2 * s, s2 = rem - s;
            PLUQ_TRY(launch_mm(kind, Blk{T, s2}, U + o * ldu + o + s, ldu,
                               X.ptr + (o + s) * (X.ld + 1), X.ld, s, s2, s2, F, MM_ASSIGN, 1, 0,
                               0, 0, ar, st));
            PLUQ_TRY(launch_mm(kind, Blk{X.ptr + o * X.ld + o + s, X.ld}, X.ptr + o * (X.ld + 1),
                               X.ld, T, s2, s, s2, s, F, MM_NEG_ASSIGN, 1, 0, 0, 0, ar, st));
        }
    }
    ar.off = mark;
    return PLUQ_OK;
}

size_t trsm_workspace(int64_t r, int64_t other, uint32_t p, int kind)
{
    size_t w = 2 * (size_t)r * r * sizeof(uint32_t) + 4096;        // X and T
    w += (size_t)r * other * sizeof(uint32_t) + 256;               // result staging
    if (kind != PLUQ_MM_SIMT) {
        // limb planes: the solve's product, or the largest batched merge level
        size_t tc = mm_tc_workspace(other, r, r, p, 1);
        const size_t left = mm_tc_workspace(r, other, r, p, 1);
        if (left > tc) tc = left;
        for (int64_t s = TB; s < r; s *= 2) {
            const int64_t full = r / (2 * s);
            const size_t lv = mm_tc_workspace(s, s, s, p, full > 0 ? full : 1);
            if (lv > tc) tc = lv;
        }
        w += tc;
    }
    return w;
}

bool trsm_direct_for(int64_t r) { return r <= WR; }

pluq_status trsm_left_lower_unit(const uint32_t *L, int64_t ldl, Blk B, int64_t r, int64_t N,
                                 Field F, int kind, Arena &ar, cudaStream_t st)
{
    if (r <= 0 || N <= 0) return PLUQ_OK;
    if (r <= RS) {
        SmallSolve ls{L, ldl, B.ptr, B.ld, (int)r, N};
        return launch_trsm_small(&ls, nullptr, F, st);
    }
    if (r <= WR) {
        prof::start(prof::TRI, st);
        pluq_status s = trsm_direct(true, L, ldl, B, N, (int)r, F, 0, st);
        prof::stop(prof::TRI, st, (double)r * r * N);   // field operations
        return s;
    }
    size_t mark = ar.off;
    uint32_t *X = (uint32_t *)ar.take((size_t)r * r * sizeof(uint32_t));
    if (!X) return PLUQ_ENOMEM;
    PLUQ_TRY(tri_inv_lower_unit(L, ldl, Blk{X, r}, r, F, kind, ar, st));
    if (kind == PLUQ_MM_SIMT) {
        uint32_t *Y = (uint32_t *)ar.take((size_t)r * N * sizeof(uint32_t));
        if (!Y) return PLUQ_ENOMEM;
        PLUQ_TRY(launch_mm(kind, Blk{Y, N}, X, r, B.ptr, B.ld, r, N, r, F, MM_ASSIGN, 1, 0, 0, 0,
                           ar, st));
        PLUQ_TRY(launch_copy(B, Y, N, r, N, st));
    } else {
        PLUQ_TRY(launch_mm(kind, B, X, r, B.ptr, B.ld, r, N, r, F, MM_ASSIGN, 1, 0, 0, 0, ar, st));
    }
    ar.off = mark;
    return PLUQ_OK;
}

pluq_status trsm_right_upper(const uint32_t *U, int64_t ldu, Blk B, int64_t M, int64_t r,
                             Field F, int kind, Arena &ar, cudaStream_t st)
{
    if (r <= 0 || M <= 0) return PLUQ_OK;
    if (r <= RS) {
        SmallSolve rs{U, ldu, B.ptr, B.ld, (int)r, M};
        return launch_trsm_small(nullptr, &rs, F, st);
    }
    if (r <= WR) {
        prof::start(prof::TRI, st);
        pluq_status s = trsm_direct(false, U, ldu, B, M, (int)r, F, 0, st);
        prof::stop(prof::TRI, st, (double)r * r * M);   // field operations
        return s;
    }
    size_t mark = ar.off;
    uint32_t *X = (uint32_t *)ar.take((size_t)r * r * sizeof(uint32_t));
    if (!X) return PLUQ_ENOMEM;
    PLUQ_TRY(tri_inv_upper(U, ldu, Blk{X, r}, r, F, kind, ar, st));
    if (kind == PLUQ_MM_SIMT) {
        uint32_t *Y = (uint32_t *)ar.take((size_t)M * r * sizeof(uint32_t));
        if (!Y) return PLUQ_ENOMEM;
        PLUQ_TRY(launch_mm(kind, Blk{Y, r}, B.ptr, B.ld, X, r, M, r, r, F, MM_ASSIGN, 1, 0, 0, 0,
                           ar, st));
        PLUQ_TRY(launch_copy(B, Y, r, M, r, st));
    } else {
        // the tensor form stages A and B in limb planes before writing C
        PLUQ_TRY(launch_mm(kind, B, B.ptr, B.ld, X, r, M, r, r, F, MM_ASSIGN, 1, 0, 0, 0, ar, st));
    }
    ar.off = mark;
    return PLUQ_OK;
}

}  // namespace pluq
