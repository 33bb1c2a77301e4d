// PLE and CUP decompositions (Sec. 1) from the packed result of pluq_mod_p.
//
// Sec. 1 relates the PLUQ to the PLE decomposition A = P L E (E in row
// echelon form, its pivots on the column rank profile) and the CUP
// decomposition A = C U Q (C in column echelon form, its pivots on the row
// rank profile), and says both follow from the PLUQ by permutations.  When
// the pivots of Algorithm 1's order are not increasing in column (row) order
// that is not so (the 2 x 2 matrix [[0, a], [b, c]] is an example), so the
// construction here adds an r x r elimination:
//
//   The LEU form (Sec. 3) gives A = sum_t Lbar e_{i_t} e_{c_t}^T Ubar over the
//   pivots (i_t, c_t).  Taken in increasing column order, the rows
//   Ur[t] = Ubar[c_t, :] form a row echelon matrix, and the columns
//   Lc[:, t] = Lbar e_{i_t} have a one at row i_t.  Put the pivot rows first
//   (P): P^T Lc = [T; B] with T[s][t] = Lbar[i_s][i_t].  Every leading
//   principal minor of T is a principal minor of the unit lower triangular
//   Lbar, so T = T_L T_U without pivoting (both unit triangular), and
//       A = P [T_L; B T_U^{-1}] (T_U Ur)
//   with T_U Ur still in row echelon form on the same columns.
//
// The same steps on the transposed view of the packed result (A^T = Q^T
// [U V]^T [L; M]^T P^T, whose left factor is lower triangular with U's
// nonzero diagonal) give the PLE of A^T, whose transpose is the CUP of A.
// T = T_L T_U comes from pluq_mod_p itself (all leading minors of T are
// nonzero, so its P and Q are identities), B T_U^{-1} from the TRSM and
// T_U Ur from the modular product.
#include <algorithm>

#include "common.cuh"

namespace pluq {
namespace {

constexpr int ET = 256;

// Element (a, b) of a triangular view of the packed result at base with row
// stride sa and column stride sb:
//   0 unit lower (a > b: stored, a == b: 1), 1 lower with its diagonal,
//   2 upper with its diagonal, 3 unit upper (a < b: stored, a == b: 1);
// zero elsewhere.  Only stored positions are read.
__device__ __forceinline__ uint32_t view_at(const uint32_t *base, int64_t sa, int64_t sb, int64_t a,
                                            int64_t b, int mode)
{
    bool stored, one = false;
    switch (mode) {
        case 0: stored = a > b; one = a == b; break;
        case 1: stored = a >= b; break;
        case 2: stored = a <= b; break;
        default: stored = a < b; one = a == b; break;
    }
    if (stored) return base[a * sa + b * sb];
    return one ? 1u : 0u;
}

// out[x][t] = view(rmap(x), cmap(t)), rmap(x) = rmap[x] for x < rlim (else
// x), cmap(t) = cmap[t]
__global__ void view_gather_kernel(uint32_t *__restrict__ out, int64_t ldo, int64_t rows,
                                   int64_t cols, const uint32_t *__restrict__ base, int64_t sa,
                                   int64_t sb, const int32_t *__restrict__ rmap, int64_t rlim,
                                   const int32_t *__restrict__ cmap, int mode)
{
    for (int64_t x = blockIdx.y; x < rows; x += gridDim.y) {
        const int64_t a = x < rlim ? (int64_t)rmap[x] : x;
        for (int64_t t = (int64_t)blockIdx.x * ET + threadIdx.x; t < cols; t += (int64_t)gridDim.x * ET)
            out[x * ldo + t] = view_at(base, sa, sb, a, (int64_t)cmap[t], mode);
    }
}

// out (or its transpose) <- W (rows x cols); rows x < unit_rows are made unit
// lower (one on the diagonal, zero above it)
__global__ void write_out_kernel(uint32_t *__restrict__ out, int64_t ldo, int trans,
                                 const uint32_t *__restrict__ W, int64_t ldw, int64_t rows,
                                 int64_t cols, int64_t unit_rows)
{
    for (int64_t x = blockIdx.y; x < rows; x += gridDim.y)
        for (int64_t t = (int64_t)blockIdx.x * ET + threadIdx.x; t < cols; t += (int64_t)gridDim.x * ET) {
            uint32_t v = W[x * ldw + t];
            if (x < unit_rows) v = x == t ? 1u : (x > t ? v : 0u);
            if (trans) out[t * ldo + x] = v;
            else out[x * ldo + t] = v;
        }
}

__global__ void iota_i32_kernel(int32_t *v, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * ET + threadIdx.x;
    if (i < n) v[i] = (int32_t)i;
}

__global__ void inverse_perm_i32_kernel(const int32_t *__restrict__ perm, int64_t n,
                                        int32_t *__restrict__ inv)
{
    const int64_t i = (int64_t)blockIdx.x * ET + threadIdx.x;
    if (i >= n) return;
    const uint32_t v = (uint32_t)perm[i];
    if ((int64_t)v < n) inv[v] = (int32_t)i;
}

// out[t] = prow[sig[t]] for t < r, prow[t] after
__global__ void perm_out_kernel(const int32_t *__restrict__ prow, const int32_t *__restrict__ sig,
                                int64_t r, int64_t m, int32_t *__restrict__ out)
{
    const int64_t t = (int64_t)blockIdx.x * ET + threadIdx.x;
    if (t < m) out[t] = t < r ? prow[sig[t]] : prow[t];
}

dim3 grid2(int64_t rows, int64_t cols)
{
    const int64_t gx = std::max<int64_t>(1, std::min<int64_t>(ceil_div(cols, ET), 64));
    const int64_t gy = std::max<int64_t>(1, std::min<int64_t>(rows, 4096));
    return dim3((unsigned)gx, (unsigned)gy);
}

// bytes of an a x b uint32 buffer, a multiple of the arena's 256-byte alignment
size_t b32(int64_t a, int64_t b) { return align_up((size_t)a * (size_t)b * 4, 256) + 256; }

// Scratch of one construction on an mm x nn view of rank r.
size_t ws_echelon(int64_t mm, int64_t nn, int64_t r, uint32_t p, int kind)
{
    size_t inner = 0;
    if (r > 0) {
        size_t w = 0;
        pluq_workspace_size(r, r, p, &w);
        inner = w;
        const size_t t = trsm_workspace(r, mm - r, p, kind);
        if (t > inner) inner = t;
        if (kind != PLUQ_MM_SIMT) {
            const size_t g = mm_tc_workspace(r, nn, r, p, 1);
            if (g > inner) inner = g;
        }
    }
    return 4 * b32(1, r) + b32(1, nn) + b32(mm, r) + 2 * b32(r, nn) + b32(r, r) + inner + 1024;
}

struct View {
    const uint32_t *base;
    int64_t sa, sb;
    int mode;
};

// PLE of the mm x nn view with pivots (prow[t], pcol[t]), t < r, in
// Algorithm 1's order, non-pivot rows prow[r..mm) increasing.  lview / uview
// read [L; M] (mm x r) and [U V] (r x nn) in packed order.  Writes the row
// permutation to perm_out (mm), L (mm x r) to Lout / its transpose and E
// (r x nn) to Eout / its transpose.
pluq_status echelon(const View &lview, const View &uview, int64_t mm, int64_t nn, int64_t r,
                    const int32_t *prow, const int32_t *pcol, uint32_t p, int kind,
                    int32_t *perm_out, uint32_t *Lout, int64_t ldl, int ltrans, uint32_t *Eout,
                    int64_t lde, int etrans, void *d_work, size_t ws_bytes, cudaStream_t st)
{
    Arena ar;
    ar.base = (char *)d_work;
    ar.size = d_work ? ws_bytes : 0;
    ar.off = 0;
    if (ar.size < ws_echelon(mm, nn, r, p, kind)) return PLUQ_ENOMEM;
    const Field F = make_field(p);
    int32_t *sig = (int32_t *)ar.take(b32(1, r));
    int32_t *keys = (int32_t *)ar.take(b32(1, r));
    int32_t *iota = (int32_t *)ar.take(b32(1, r));
    int32_t *pps = (int32_t *)ar.take(b32(1, r));
    int32_t *inv = (int32_t *)ar.take(b32(1, nn));
    uint32_t *Lw = (uint32_t *)ar.take(b32(mm, r));
    uint32_t *Uw = (uint32_t *)ar.take(b32(r, nn));
    uint32_t *Ew = (uint32_t *)ar.take(b32(r, nn));
    uint32_t *Tu = (uint32_t *)ar.take(b32(r, r));
    if (!sig || !keys || !iota || !pps || !inv || !Lw || !Uw || !Ew || !Tu) return PLUQ_ENOMEM;
    const size_t inner_off = ar.off;
    if (mm > 0 && r == 0) {
        // no pivots: the non-pivot rows, increasing, and nothing else
        return cudaMemcpyAsync(perm_out, prow, (size_t)mm * 4, cudaMemcpyDeviceToDevice, st) ==
                       cudaSuccess
                   ? PLUQ_OK
                   : PLUQ_ECUDA;
    }
    if (mm == 0 || nn == 0) return PLUQ_OK;
    // sig: the pivots in increasing column order (positions in Algorithm 1's order)
    iota_i32_kernel<<<(unsigned)ceil_div(r, ET), ET, 0, st>>>(iota, r);
    PLUQ_TRY(last_launch());
    PLUQ_TRY(launch_rank_sort(pcol, iota, r, keys, sig, st));
    perm_out_kernel<<<(unsigned)ceil_div(mm, ET), ET, 0, st>>>(prow, sig, r, mm, perm_out);
    PLUQ_TRY(last_launch());
    inverse_perm_i32_kernel<<<(unsigned)ceil_div(nn, ET), ET, 0, st>>>(pcol, nn, inv);
    PLUQ_TRY(last_launch());
    // Lw = P^T Lc: rows sig[x] (x < r) then r.., columns sig[t]; Uw = Ur in
    // original column order: Uw[t][col] = [U V][sig[t]][inv[col]]
    view_gather_kernel<<<grid2(mm, r), ET, 0, st>>>(Lw, r, mm, r, lview.base, lview.sa, lview.sb,
                                                     sig, r, sig, lview.mode);
    PLUQ_TRY(last_launch());
    view_gather_kernel<<<grid2(r, nn), ET, 0, st>>>(Uw, nn, r, nn, uview.base, uview.sa, uview.sb,
                                                     sig, r, inv, uview.mode);
    PLUQ_TRY(last_launch());
    // T = T_L T_U in place (leading minors nonzero: rank r, P = Q = I)
    ar.off = inner_off;
    int64_t rk = -1;
    {
        size_t need = 0;
        PLUQ_TRY(pluq_workspace_size(r, r, p, &need));
        void *w = ar.take(need, 256);
        if (!w) return PLUQ_ENOMEM;
        PLUQ_TRY(pluq_mod_p(Lw, r, r, r, p, pps, keys, &rk, w, need, kind, st));
        ar.off = inner_off;
    }
    if (rk != r) return PLUQ_EINTERNAL;
    // B <- B T_U^{-1}, Tu = T_U (zero below the diagonal), Ew = T_U Ur
    PLUQ_TRY(trsm_right_upper(Lw, r, Blk{Lw + r * r, r}, mm - r, r, F, kind, ar, st));
    PLUQ_TRY(launch_extract(Lw, r, r, r, Tu, r, false, st));
    PLUQ_TRY(launch_mm(kind, Blk{Ew, nn}, Tu, r, Uw, nn, r, nn, r, F, MM_ASSIGN, 1, 0, 0, 0, ar,
                       st));
    write_out_kernel<<<grid2(mm, r), ET, 0, st>>>(Lout, ldl, ltrans, Lw, r, mm, r, r);
    PLUQ_TRY(last_launch());
    write_out_kernel<<<grid2(r, nn), ET, 0, st>>>(Eout, lde, etrans, Ew, nn, r, nn, 0);
    return last_launch();
}

bool args_ok(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda, int64_t r,
             const int32_t *d_perm_p, const int32_t *d_perm_q)
{
    if (m < 0 || n < 0 || r < 0 || r > m || r > n) return false;
    if (m > 0 && n > 0 && (!d_LU || lda < n)) return false;
    if ((m > 0 && !d_perm_p) || (n > 0 && !d_perm_q)) return false;
    if (m >= (1ll << 31) || n >= (1ll << 31)) return false;
    return true;
}

int kind_or_tensor(int mm_kind) { return mm_kind == PLUQ_MM_AUTO ? PLUQ_MM_TENSOR : mm_kind; }

}  // namespace
}  // namespace pluq

using namespace pluq;

extern "C" {

pluq_status pluq_echelon_workspace_size(int64_t m, int64_t n, int64_t r, uint32_t p, int mm_kind,
                                        size_t *h_bytes)
{
    if (m < 0 || n < 0 || r < 0 || r > m || r > n || !h_bytes) return PLUQ_EINVAL;
    if (mm_kind < PLUQ_MM_AUTO || mm_kind > PLUQ_MM_TENSOR) return PLUQ_EINVAL;
    if (p >= 0x80000000u || !is_prime_u32(p)) return PLUQ_ENOTPRIME;
    const int kind = kind_or_tensor(mm_kind);
    const size_t a = ws_echelon(m, n, r, p, kind), b = ws_echelon(n, m, r, p, kind);
    *h_bytes = a > b ? a : b;
    return PLUQ_OK;
}

pluq_status pluq_ple(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda, int64_t r,
                     const int32_t *d_perm_p, const int32_t *d_perm_q, uint32_t p,
                     int32_t *d_perm_out, uint32_t *d_L, int64_t ldl, uint32_t *d_E, int64_t lde,
                     int mm_kind, void *d_work, size_t ws_bytes, void *stream)
{
    if (!args_ok(d_LU, m, n, lda, r, d_perm_p, d_perm_q)) return PLUQ_EINVAL;
    if (mm_kind < PLUQ_MM_AUTO || mm_kind > PLUQ_MM_TENSOR) return PLUQ_EINVAL;
    if (p >= 0x80000000u || !is_prime_u32(p)) return PLUQ_ENOTPRIME;
    if (m > 0 && !d_perm_out) return PLUQ_EINVAL;
    if (r > 0 && (!d_L || !d_E || ldl < r || lde < n)) return PLUQ_EINVAL;
    const View lv{d_LU, lda, 1, 0}, uv{d_LU, lda, 1, 2};
    pluq_status s = echelon(lv, uv, m, n, r, d_perm_p, d_perm_q, p, kind_or_tensor(mm_kind),
                            d_perm_out, d_L, ldl, 0, d_E, lde, 0, d_work, ws_bytes,
                            (cudaStream_t)stream);
    if (s != PLUQ_OK) return s;
    return cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess ? PLUQ_OK : PLUQ_ECUDA;
}

pluq_status pluq_cup(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda, int64_t r,
                     const int32_t *d_perm_p, const int32_t *d_perm_q, uint32_t p,
                     int32_t *d_perm_out, uint32_t *d_C, int64_t ldc, uint32_t *d_U, int64_t ldu,
                     int mm_kind, void *d_work, size_t ws_bytes, void *stream)
{
    if (!args_ok(d_LU, m, n, lda, r, d_perm_p, d_perm_q)) return PLUQ_EINVAL;
    if (mm_kind < PLUQ_MM_AUTO || mm_kind > PLUQ_MM_TENSOR) return PLUQ_EINVAL;
    if (p >= 0x80000000u || !is_prime_u32(p)) return PLUQ_ENOTPRIME;
    if (n > 0 && !d_perm_out) return PLUQ_EINVAL;
    if (r > 0 && (!d_C || !d_U || ldc < r || ldu < n)) return PLUQ_EINVAL;
    // the PLE of A^T = Q^T [U V]^T [L; M]^T P^T, read transposed: its left
    // factor is lower with U's diagonal, its right factor unit upper
    const View lv{d_LU, 1, lda, 1}, uv{d_LU, 1, lda, 3};
    pluq_status s = echelon(lv, uv, n, m, r, d_perm_q, d_perm_p, p, kind_or_tensor(mm_kind),
                            d_perm_out, d_U, ldu, 1, d_C, ldc, 1, d_work, ws_bytes,
                            (cudaStream_t)stream);
    if (s != PLUQ_OK) return s;
    return cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess ? PLUQ_OK : PLUQ_ECUDA;
}

}  // extern "C"
