// TRSM of Sec. 2 on the GPU:  B <- L^{-1} B (L unit lower) and B <- B U^{-1}
// (U upper, nonzero diagonal).
//
// Instead of a substitution whose critical path is one column of B per step,
// the triangle is inverted first and the solve becomes one modular product:
//   - 64 x 64 diagonal blocks are inverted by substitution, one thread block
//     per diagonal block, all blocks in one launch;
//   - blocks are then merged pairwise, log2(r/64) levels, with
//       [L11 0; L21 L22]^-1 = [X11 0; -X22 L21 X11  X22],
//       [U11 U12; 0 U22]^-1 = [X11 -X11 U12 X22; 0 X22],
//     every pair of a level in one batched product launch;
//   - the solve is X B (or B X).
// The inverse costs r^3/3 field operations, small next to the r^2 N of the
// solve for the shapes Algorithm 1 produces, and the launches per TRSM drop
// from O(r/64) to O(log(r/64)).
#include "common.cuh"

namespace pluq {
namespace {

constexpr int TB = 64;

// Sum of up to 2^17 products a_l * b_l (a, b < 2^31) held exactly in two
// 64-bit words: a = a_hi 2^16 + a_lo.
struct Acc {
    uint64_t lo = 0, hi = 0;
    __device__ __forceinline__ void add(uint32_t a, uint32_t b)
    {
        lo += (uint64_t)(a & 0xFFFFu) * b;
        hi += (uint64_t)(a >> 16) * b;
    }
    __device__ __forceinline__ uint32_t value(const Field &F) const
    {
        uint32_t w16 = (uint32_t)((1ull << 16) % F.p);
        return add_mod(reduce64(lo, F), mul_mod(reduce64(hi, F), w16, F), F.p);
    }
};

// X_b = (diagonal block b of L)^-1, unit lower.  One block of TB threads per
// diagonal block; thread j owns column j of X.
__global__ void inv_lower_unit_base(const uint32_t *__restrict__ L, int64_t ldl,
                                    uint32_t *__restrict__ X, int64_t ldx, int r, Field F)
{
    __shared__ uint32_t Ls[TB][TB + 1];
    __shared__ uint32_t Xs[TB][TB + 1];
    const int b = blockIdx.x, o = b * TB;
    const int sb = min(TB, r - o);
    const int j = threadIdx.x;
    for (int i = 0; i < sb; ++i)
        if (j < sb) Ls[i][j] = L[(int64_t)(o + i) * ldl + o + j];
    __syncthreads();
    if (j < sb) {
        for (int i = 0; i < sb; ++i) {
            uint32_t v;
            if (i < j) v = 0;
            else if (i == j) v = 1;
            else {
                Acc acc;
                for (int l = j; l < i; ++l) acc.add(Ls[i][l], Xs[l][j]);
                uint32_t s = acc.value(F);
                v = s == 0 ? 0 : F.p - s;
            }
            Xs[i][j] = v;
        }
    }
    __syncthreads();
    for (int i = 0; i < sb; ++i)
        if (j < sb) X[(int64_t)(o + i) * ldx + o + j] = Xs[i][j];
}

// X_b = (diagonal block b of U)^-1, upper.
__global__ void inv_upper_base(const uint32_t *__restrict__ U, int64_t ldu,
                               uint32_t *__restrict__ X, int64_t ldx, int r, Field F)
{
    __shared__ uint32_t Us[TB][TB + 1];
    __shared__ uint32_t Xs[TB][TB + 1];
    __shared__ uint32_t dinv[TB];
    const int b = blockIdx.x, o = b * TB;
    const int sb = min(TB, r - o);
    const int j = threadIdx.x;
    for (int i = 0; i < sb; ++i)
        if (j < sb) Us[i][j] = U[(int64_t)(o + i) * ldu + o + j];
    __syncthreads();
    if (j < sb) dinv[j] = inv_mod(Us[j][j], F.p);
    __syncthreads();
    if (j < sb) {
        for (int i = sb - 1; i >= 0; --i) {
            uint32_t v;
            if (i > j) v = 0;
            else if (i == j) v = dinv[j];
            else {
                Acc acc;
                for (int l = i + 1; l <= j; ++l) acc.add(Us[i][l], Xs[l][j]);
                uint32_t s = mul_mod(acc.value(F), dinv[i], F);
                v = s == 0 ? 0 : F.p - s;
            }
            Xs[i][j] = v;
        }
    }
    __syncthreads();
    for (int i = 0; i < sb; ++i)
        if (j < sb) X[(int64_t)(o + i) * ldx + o + j] = Xs[i][j];
}

}  // namespace

pluq_status tri_inv_lower_unit(const uint32_t *L, int64_t ldl, Blk X, int64_t r, Field F,
                               int kind, Arena &ar, cudaStream_t st)
{
    if (r <= 0) return PLUQ_OK;
    PLUQ_TRY(launch_zero(X, r, r, st));
    prof::start(prof::TRI, st);
    inv_lower_unit_base<<<(unsigned)ceil_div(r, TB), TB, 0, st>>>(L, ldl, X.ptr, X.ld, (int)r, F);
    PLUQ_TRY(last_launch());
    prof::stop(prof::TRI, st, (double)r * TB * TB / 3.0);
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
    inv_upper_base<<<(unsigned)ceil_div(r, TB), TB, 0, st>>>(U, ldu, X.ptr, X.ld, (int)r, F);
    PLUQ_TRY(last_launch());
    prof::stop(prof::TRI, st, (double)r * TB * TB / 3.0);
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
    if (kind != PLUQ_MM_SIMT) w += mm_tc_workspace(other, r, r, p, 1) + mm_tc_workspace(r, r, r, p, 64);
    return w;
}

pluq_status trsm_left_lower_unit(const uint32_t *L, int64_t ldl, Blk B, int64_t r, int64_t N,
                                 Field F, int kind, Arena &ar, cudaStream_t st)
{
    if (r <= 0 || N <= 0) return PLUQ_OK;
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
