// TRSM of Sec. 2 on the GPU:  B <- L^{-1} B (L unit lower) and B <- B U^{-1}
// (U upper, nonzero diagonal).
//
// Instead of a substitution whose critical path is one column of B per step,
// the triangle is inverted first and the solve becomes one modular product:
//   - 32 x 32 diagonal blocks are inverted by substitution, one thread block
//     per diagonal block, all blocks in one launch;
//   - blocks are then merged pairwise, log2(r/32) levels, with
//       [L11 0; L21 L22]^-1 = [X11 0; -X22 L21 X11  X22],
//       [U11 U12; 0 U22]^-1 = [X11 -X11 U12 X22; 0 X22],
//     every pair of a level in one batched product launch;
//   - the solve is X B (or B X).
// The inverse costs r^3/3 field operations, small next to the r^2 N of the
// solve for the shapes Algorithm 1 produces, and the launches per TRSM drop
// from O(r/32) to O(log(r/32)).  Triangles of at most 64 rows are solved
// directly by substitution instead (one launch).
#include "common.cuh"

namespace pluq {
namespace {


// Sum of up to 2^17 products a_l * b_l (a, b < 2^31) held exactly in 64-bit
// words.  p <= 2^16: one word (products < 2^32).  Otherwise a = a_hi 2^16 +
// a_lo and two words; w16 = 2^16 mod p recombines them.
template <bool SMALLP>
struct Acc {
    uint64_t lo = 0, hi = 0;
    __device__ __forceinline__ void add(uint32_t a, uint32_t b)
    {
        if (SMALLP) {
            lo += (uint64_t)(a * b);
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

// Direct solves for narrow triangles (r <= WR): one warp per right-hand side
// (a column of B for the left solve, a row of B for the right one), lane q
// owning triangle rows / columns q, q + 32, ...  The unknowns are produced one
// per step: the owner of the next unknown finishes it and broadcasts it with a
// shuffle, every lane adds its term into the running sums of its later rows.
// The owner's sum over the earlier terms is reduced one step ahead, so a step's
// dependency chain is one shuffle, one modular product and two subtractions.
constexpr int WR = 128, WT = 256, WPB = WT / 32;
constexpr int TB = WR;   // diagonal blocks the inverses start from

template <bool SMALLP>
__device__ __forceinline__ uint32_t prod_mod(uint32_t a, uint32_t b, const Field &F,
                                             const Field32 &F32)
{
    if (SMALLP) return reduce32(a * b, F32);
    return mul_mod(a, b, F);
}

template <int RPL, typename T>
__device__ __forceinline__ T slot_pick(const T (&v)[RPL], int s)
{
    T x = v[0];
#pragma unroll
    for (int t = 1; t < RPL; ++t)
        if (s == t) x = v[t];
    return x;
}

// odd row stride of the staged triangle: a lane per row reads without conflicts
__host__ __device__ __forceinline__ int tri_ld(int r) { return (r & 1) ? r + 2 : r + 1; }

// B (r x N) <- L^{-1} B, L unit lower (diagonal not read).  IDENT: blockIdx.y
// picks the diagonal block of L at o = blockIdx.y * blk (size min(blk, r - o))
// and B receives its inverse there (the right-hand side is the identity).
template <bool SMALLP, int RPL, bool IDENT>
__global__ void __launch_bounds__(WT) trsm_left_warp(const uint32_t *__restrict__ L, int64_t ldl,
                                                      uint32_t *__restrict__ B, int64_t ldb, int r,
                                                      int64_t N, Field F, int blk)
{
    extern __shared__ uint32_t Ls[];
    if (IDENT) {
        const int64_t o = (int64_t)blockIdx.y * blk;
        L += o * (ldl + 1);
        B += o * (ldb + 1);
        r = min(blk, (int)(r - o));
        N = r;
    }
    const int ld = tri_ld(r);
    {
        const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, l = threadIdx.x & 31;
        for (int i = w; i < r; i += nw)
#pragma unroll 4
            for (int c = l; c < i; c += 32) Ls[i * ld + c] = L[(int64_t)i * ldl + c];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *xs = Ls + r * ld + warp * WR;            // this warp's unknowns
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (j >= N) return;
    const Field32 F32{F.p, 0xFFFFFFFFu / F.p};
    const uint32_t w16 = (uint32_t)((1ull << 16) % F.p);
    uint32_t b[RPL];
    Acc<SMALLP> acc[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
        const int row = lane + 32 * t;
        if (IDENT) b[t] = row == j ? 1u : 0u;
        else b[t] = row < r ? B[(int64_t)row * ldb + j] : 0u;
    }
    uint32_t x = __shfl_sync(0xFFFFFFFFu, b[0], 0);   // x_0 = b_0
    if (lane == 0) xs[0] = x;
    uint32_t vnext = 0;                               // owner's sum for row i + 1, terms < i
    for (int i = 0; i + 1 < r; ++i) {
        const int nr = i + 1, nl = nr & 31, ns = nr >> 5;
        const uint32_t lx = Ls[nr * ld + i];
        const uint32_t xn = sub_mod(sub_mod(slot_pick<RPL>(b, ns), vnext, F.p),
                                    prod_mod<SMALLP>(lx, x, F, F32), F.p);
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int row = lane + 32 * t;
            if (row > nr && row < r) acc[t].add(Ls[row * ld + i], x);
        }
        x = __shfl_sync(0xFFFFFFFFu, xn, nl);
        if (lane == 0) xs[nr] = x;
        vnext = slot_pick<RPL>(acc, (i + 2) >> 5).value(F, w16);
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
        const int row = lane + 32 * t;
        if (row < r) B[(int64_t)row * ldb + j] = xs[row];
    }
}

// B (M x r) <- B U^{-1}, U upper with nonzero diagonal.  IDENT: as for the
// left solve, B receives the inverse of the diagonal block blockIdx.y of U.
template <bool SMALLP, int RPL, bool IDENT>
__global__ void __launch_bounds__(WT) trsm_right_warp(const uint32_t *__restrict__ U, int64_t ldu,
                                                       uint32_t *__restrict__ B, int64_t ldb,
                                                       int64_t M, int r, Field F, int blk)
{
    extern __shared__ uint32_t Us[];
    if (IDENT) {
        const int64_t o = (int64_t)blockIdx.y * blk;
        U += o * (ldu + 1);
        B += o * (ldb + 1);
        r = min(blk, (int)(r - o));
        M = r;
    }
    const int ld = tri_ld(r);
    uint32_t *dinv = Us + r * ld;
    {
        const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, l = threadIdx.x & 31;
        for (int i = w; i < r; i += nw)
#pragma unroll 4
            for (int c = i + l; c < r; c += 32) Us[i * ld + c] = U[(int64_t)i * ldu + c];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < r; t += blockDim.x) dinv[t] = inv_mod(Us[t * ld + t], F.p);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *xs = dinv + WR + warp * WR;              // this warp's unknowns
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (i >= M) return;
    const Field32 F32{F.p, 0xFFFFFFFFu / F.p};
    const uint32_t w16 = (uint32_t)((1ull << 16) % F.p);
    uint32_t b[RPL];
    Acc<SMALLP> acc[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
        const int c = lane + 32 * t;
        if (IDENT) b[t] = c == i ? 1u : 0u;
        else b[t] = c < r ? B[i * ldb + c] : 0u;
    }
    uint32_t x = prod_mod<SMALLP>(__shfl_sync(0xFFFFFFFFu, b[0], 0), dinv[0], F, F32);
    if (lane == 0) xs[0] = x;
    uint32_t vnext = 0;
    for (int l = 0; l + 1 < r; ++l) {
        const int nc = l + 1, nl = nc & 31, ns = nc >> 5;
        const uint32_t ux = Us[l * ld + nc];
        const uint32_t xn = prod_mod<SMALLP>(
            sub_mod(sub_mod(slot_pick<RPL>(b, ns), vnext, F.p), prod_mod<SMALLP>(ux, x, F, F32),
                    F.p),
            dinv[nc], F, F32);
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int c = lane + 32 * t;
            if (c > nc && c < r) acc[t].add(Us[l * ld + c], x);
        }
        x = __shfl_sync(0xFFFFFFFFu, xn, nl);
        if (lane == 0) xs[nc] = x;
        vnext = slot_pick<RPL>(acc, (l + 2) >> 5).value(F, w16);
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
        const int c = lane + 32 * t;
        if (c < r) B[i * ldb + c] = xs[c];
    }
}

// left: B (r x other) <- T^{-1} B; otherwise B (other x r) <- B T^{-1}.  With
// `blocks` > 0 the diagonal blocks of size min(WR, .) of T are inverted into B
// instead (other is ignored).
template <bool SMALLP, int RPL>
pluq_status launch_trsm_warp(bool left, const uint32_t *T, int64_t ldt, Blk B, int64_t other,
                             int r, Field F, int64_t blocks, cudaStream_t st)
{
    const int rr = blocks > 0 ? (r < WR ? r : WR) : r;
    const int64_t rhs = blocks > 0 ? rr : other;
    const int64_t nb = blocks > 0 ? blocks : 1;
    const int wpb = WPB;
    const size_t smem = ((size_t)rr * tri_ld(rr) + (left ? 0 : WR) + (size_t)wpb * WR) * sizeof(uint32_t);
    const dim3 grid((unsigned)ceil_div(rhs, wpb), (unsigned)nb);
    const int nt = 32 * wpb;
    const int full = (WR * tri_ld(WR) + WPB * WR) * 4, fullr = (WR * tri_ld(WR) + WR + WPB * WR) * 4;
#define PLUQ_TRSM_ATTR(K, BYTES)                                                                   \
    {                                                                                             \
        static const bool attr =                                                                  \
            cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, BYTES) ==        \
            cudaSuccess;                                                                          \
        if (!attr) return PLUQ_ECUDA;                                                             \
    }
    if (left && blocks > 0) {
        PLUQ_TRSM_ATTR((trsm_left_warp<SMALLP, RPL, true>), full)
        trsm_left_warp<SMALLP, RPL, true><<<grid, nt, smem, st>>>(T, ldt, B.ptr, B.ld, r, 0, F, WR);
    } else if (left) {
        PLUQ_TRSM_ATTR((trsm_left_warp<SMALLP, RPL, false>), full)
        trsm_left_warp<SMALLP, RPL, false><<<grid, nt, smem, st>>>(T, ldt, B.ptr, B.ld, r, other, F, 0);
    } else if (blocks > 0) {
        PLUQ_TRSM_ATTR((trsm_right_warp<SMALLP, RPL, true>), fullr)
        trsm_right_warp<SMALLP, RPL, true><<<grid, nt, smem, st>>>(T, ldt, B.ptr, B.ld, 0, r, F, WR);
    } else {
        PLUQ_TRSM_ATTR((trsm_right_warp<SMALLP, RPL, false>), fullr)
        trsm_right_warp<SMALLP, RPL, false><<<grid, nt, smem, st>>>(T, ldt, B.ptr, B.ld, other, r, F, 0);
    }
#undef PLUQ_TRSM_ATTR
    return last_launch();
}

pluq_status trsm_direct(bool left, const uint32_t *T, int64_t ldt, Blk B, int64_t other, int r,
                        Field F, int64_t blocks, cudaStream_t st)
{
    const bool sp = F.p <= 65536u;
    const int rb = blocks > 0 ? (r < WR ? r : WR) : r;
    const int rpl = rb <= 32 ? 1 : rb <= 64 ? 2 : 4;
    if (sp) {
        if (rpl == 1) return launch_trsm_warp<true, 1>(left, T, ldt, B, other, r, F, blocks, st);
        if (rpl == 2) return launch_trsm_warp<true, 2>(left, T, ldt, B, other, r, F, blocks, st);
        return launch_trsm_warp<true, 4>(left, T, ldt, B, other, r, F, blocks, st);
    }
    if (rpl == 1) return launch_trsm_warp<false, 1>(left, T, ldt, B, other, r, F, blocks, st);
    if (rpl == 2) return launch_trsm_warp<false, 2>(left, T, ldt, B, other, r, F, blocks, st);
    return launch_trsm_warp<false, 4>(left, T, ldt, B, other, r, F, blocks, st);
}

}  // namespace

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
