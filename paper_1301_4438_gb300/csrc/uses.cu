// Uses of the decomposition that Sec. 1 lists (linear systems, determinant,
// nullspace), read off the packed result of pluq_mod_p:
//   A = P [L;M] [U V] Q,   P[perm_p[i], i] = 1,   Q[j, perm_q[j]] = 1.
//
//   det A (m = n)   sgn(P) sgn(Q) prod_i U[i][i] when r = n, else 0;
//                   sgn of a permutation = (-1)^(length - number of cycles).
//   right kernel    N = Q^T [-U^{-1} V; I_{n-r}]:  A N = P [L;M] (-V + V) = 0.
//   left kernel     K = [-M L^{-1}, I_{m-r}] P^T:  K A = (-M + M) [U V] Q = 0.
//   A X = B         Y = [L 0; M I]^{-1} P^T B; column c is solvable iff
//                   Y[r:, c] = 0, and then X = Q^T [U^{-1} Y[:r, :]; 0].
//
// Because the pivot columns of a rank-profile-revealing PLUQ are the column
// rank profile, N is the unique kernel basis that is the identity on the
// other coordinates, and X the unique solution that vanishes there (likewise
// K on the rows outside the row rank profile).
//
// The triangular inverses and the products run on the library's TRSM and
// modular MM kernels; the kernels here are the permutation parity and the
// scatters of the results into original row / column order (HBM-bound,
// coalesced along rows).
#include "common.cuh"

namespace pluq {
namespace {

constexpr int UT = 256;      // threads per block
constexpr int UC = 4 * UT;   // columns per block
constexpr int DT = 1024;     // threads of the determinant's reduction block

dim3 grid_rows(int64_t rows, int64_t cols)
{
    const int64_t gy = rows < 65535 ? rows : 65535;
    return dim3((unsigned)ceil_div(cols, UC), (unsigned)(gy > 0 ? gy : 1));
}

// inv[perm[i]] = i; entries of perm outside [0, n) are skipped.
__global__ void inverse_kernel(const int32_t *__restrict__ perm, int64_t n,
                               int32_t *__restrict__ inv)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t v = (uint32_t)perm[i];
    if ((int64_t)v < n) inv[v] = (int32_t)i;
}

// Row scatter: dst (rows x w) row i = row q = inv[i] of [W; I or 0], i.e.
// W[q][:] when q < r, else the unit vector e_{q-r} (ident) or zero.
// W is only read at q < r.
__global__ void scatter_rows_kernel(uint32_t *__restrict__ dst, int64_t ldd, int64_t rows,
                                    int64_t w, const uint32_t *__restrict__ W, int64_t ldw,
                                    const int32_t *__restrict__ inv, int64_t r, int ident)
{
    const int64_t c0 = (int64_t)blockIdx.x * UC + threadIdx.x;
    for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) {
        const int64_t q = (uint32_t)inv[i];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int64_t c = c0 + (int64_t)s * UT;
            if (c >= w) continue;
            dst[i * ldd + c] = q < r ? W[q * ldw + c] : ((ident && q - r == c) ? 1u : 0u);
        }
    }
}

// Column scatter: dst (d x cols) column i = column q = inv[i] of [W, I]:
// W[:][q] when q < r, else e_{q-r}.  W is only read at q < r.
__global__ void scatter_cols_kernel(uint32_t *__restrict__ dst, int64_t ldd, int64_t d,
                                    int64_t cols, const uint32_t *__restrict__ W, int64_t ldw,
                                    const int32_t *__restrict__ inv, int64_t r)
{
    const int64_t i0 = (int64_t)blockIdx.x * UC + threadIdx.x;
    for (int64_t c = blockIdx.y; c < d; c += gridDim.y) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int64_t i = i0 + (int64_t)s * UT;
            if (i >= cols) continue;
            const int64_t q = (uint32_t)inv[i];
            dst[c * ldd + i] = q < r ? W[c * ldw + q] : (q - r == c ? 1u : 0u);
        }
    }
}

// *flag |= (the rows x cols block has a nonzero entry)
__global__ void flag_nonzero_kernel(const uint32_t *__restrict__ Y, int64_t ldy, int64_t rows,
                                    int64_t cols, int32_t *flag)
{
    const int64_t c0 = (int64_t)blockIdx.x * UC + threadIdx.x;
    bool nz = false;
    for (int64_t i = blockIdx.y; i < rows; i += gridDim.y)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int64_t c = c0 + (int64_t)s * UT;
            if (c < cols && Y[i * ldy + c] != 0) nz = true;
        }
    if (__syncthreads_or(nz) && threadIdx.x == 0) atomicOr(flag, 1);
}

// Cycle leaders of perm_p and perm_q at once, on the functional graph
// i -> perm_p[i] (i < n) and n + j -> n + perm_q[j].  Pointer doubling:
// after round k, nxt = pi^(2^k) and lab[i] = min over pi^e(i), e < 2^k, so
// after ceil(log2 n) rounds lab[i] is the least index of i's cycle and the
// leaders are the i with lab[i] == i.  Entries outside [0, n) become fixed
// points, so every index stays in bounds whatever the input.
__global__ void jump_init_kernel(const int32_t *__restrict__ pp, const int32_t *__restrict__ pq,
                                 int64_t n, int32_t *__restrict__ nxt, int32_t *__restrict__ lab)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * n) return;
    const bool top = i < n;
    const int64_t v = (uint32_t)(top ? pp[i] : pq[i - n]);
    nxt[i] = (int32_t)(v < n ? (top ? v : n + v) : i);
    lab[i] = (int32_t)i;
}

__global__ void jump_kernel(const int32_t *__restrict__ nxt_in, const int32_t *__restrict__ lab_in,
                            int32_t *__restrict__ nxt_out, int32_t *__restrict__ lab_out,
                            int64_t len)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    const int32_t j = nxt_in[i];
    nxt_out[i] = nxt_in[j];
    lab_out[i] = min(lab_in[i], lab_in[j]);
}

// det = (-1)^(leaders) prod_i LU[i][i]: sgn(P) sgn(Q) = (-1)^((n - cP) + (n - cQ)).
__global__ void __launch_bounds__(DT) det_kernel(const uint32_t *__restrict__ LU, int64_t lda,
                                                 int64_t n, const int32_t *__restrict__ lab,
                                                 Field F, uint32_t *det)
{
    __shared__ uint32_t s_prod[DT / 32], s_par[DT / 32];
    uint32_t prod = 1, par = 0;
    for (int64_t i = threadIdx.x; i < n; i += DT) prod = mul_mod(prod, LU[i * lda + i], F);
    if (lab)
        for (int64_t i = threadIdx.x; i < 2 * n; i += DT) par ^= (uint32_t)(lab[i] == i);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        prod = mul_mod(prod, __shfl_xor_sync(0xffffffffu, prod, o), F);
        par ^= __shfl_xor_sync(0xffffffffu, par, o);
    }
    if (lane == 0) {
        s_prod[warp] = prod;
        s_par[warp] = par;
    }
    __syncthreads();
    if (warp == 0) {
        prod = s_prod[lane];
        par = s_par[lane];
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            prod = mul_mod(prod, __shfl_xor_sync(0xffffffffu, prod, o), F);
            par ^= __shfl_xor_sync(0xffffffffu, par, o);
        }
        if (lane == 0) det[0] = par ? sub_mod(0u, prod, F.p) : prod;
    }
}

int kind_of(int mm_kind) { return mm_kind == PLUQ_MM_AUTO ? PLUQ_MM_TENSOR : mm_kind; }

bool bad_modulus(uint32_t p) { return p >= 0x80000000u || !is_prime_u32(p); }

constexpr size_t SLACK = 256;

size_t bytes_u32(int64_t a, int64_t b) { return (size_t)a * (size_t)b * 4 + SLACK; }

pluq_status launch_inverse(const int32_t *perm, int64_t n, int32_t *inv, cudaStream_t st)
{
    if (n <= 0) return PLUQ_OK;
    inverse_kernel<<<(unsigned)ceil_div(n, UT), UT, 0, st>>>(perm, n, inv);
    return last_launch();
}

size_t ws_determinant(int64_t n) { return 4 * bytes_u32(2, n); }

size_t ws_right(int64_t m, int64_t n, int64_t r, uint32_t p, int kind)
{
    (void)m;
    return bytes_u32(r, r) + bytes_u32(r, n - r) + bytes_u32(1, n) +
           trsm_workspace(r, n - r, p, kind);
}

size_t ws_left(int64_t m, int64_t n, int64_t r, uint32_t p, int kind)
{
    (void)n;
    return bytes_u32(r, r) + bytes_u32(m - r, r) + bytes_u32(1, m) +
           trsm_workspace(r, m - r, p, kind);
}

size_t ws_solve(int64_t m, int64_t n, int64_t r, int64_t k, uint32_t p, int kind)
{
    size_t inner = trsm_workspace(r, k, p, kind);
    if (kind != PLUQ_MM_SIMT) {
        const size_t upd = mm_tc_workspace(m - r, k, r, p, 1);
        if (upd > inner) inner = upd;
    }
    return bytes_u32(m, k) + bytes_u32(r, k) + bytes_u32(1, n) + bytes_u32(r, r) + inner;
}

Arena arena_of(void *d_work, size_t ws_bytes)
{
    Arena ar;
    ar.base = (char *)d_work;
    ar.size = d_work ? ws_bytes : 0;
    ar.off = 0;
    return ar;
}

bool factor_args_ok(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda, int64_t r)
{
    if (m < 0 || n < 0 || r < 0 || r > m || r > n) return false;
    if (m > 0 && n > 0 && (!d_LU || lda < n)) return false;
    return true;
}

}  // namespace
}  // namespace pluq

using namespace pluq;

extern "C" {

pluq_status pluq_uses_workspace_size(int64_t m, int64_t n, int64_t r, int64_t k, uint32_t p,
                                     int mm_kind, size_t *h_bytes)
{
    if (m < 0 || n < 0 || r < 0 || r > m || r > n || k < 0 || !h_bytes) return PLUQ_EINVAL;
    if (mm_kind < PLUQ_MM_AUTO || mm_kind > PLUQ_MM_TENSOR) return PLUQ_EINVAL;
    if (bad_modulus(p)) return PLUQ_ENOTPRIME;
    const int kind = kind_of(mm_kind);
    size_t w = ws_determinant(m > n ? m : n);
    const size_t a = ws_right(m, n, r, p, kind), b = ws_left(m, n, r, p, kind),
                 c = ws_solve(m, n, r, k, p, kind);
    if (a > w) w = a;
    if (b > w) w = b;
    if (c > w) w = c;
    *h_bytes = w;
    return PLUQ_OK;
}

pluq_status pluq_determinant(const uint32_t *d_LU, int64_t n, int64_t lda, int64_t r,
                             const int32_t *d_perm_p, const int32_t *d_perm_q, uint32_t p,
                             uint32_t *d_det, void *d_work, size_t ws_bytes, void *stream)
{
    if (!factor_args_ok(d_LU, n, n, lda, r) || !d_det) return PLUQ_EINVAL;
    if (n >= (int64_t)1 << 30) return PLUQ_EINVAL;
    if (bad_modulus(p)) return PLUQ_ENOTPRIME;
    cudaStream_t st = (cudaStream_t)stream;
    const Field F = make_field(p);
    if (r < n) {
        PLUQ_CUDA_TRY(cudaMemsetAsync(d_det, 0, sizeof(uint32_t), st));
        return PLUQ_OK;
    }
    if (n == 0) {
        det_kernel<<<1, DT, 0, st>>>(d_LU, 1, 0, nullptr, F, d_det);
        return last_launch();
    }
    if (!d_perm_p || !d_perm_q) return PLUQ_EINVAL;
    Arena ar = arena_of(d_work, ws_bytes);
    if (ar.size < ws_determinant(n)) return PLUQ_ENOMEM;
    const int64_t len = 2 * n;
    int32_t *nxt[2], *lab[2];
    for (int b = 0; b < 2; ++b) {
        nxt[b] = (int32_t *)ar.take((size_t)len * 4);
        lab[b] = (int32_t *)ar.take((size_t)len * 4);
        if (!nxt[b] || !lab[b]) return PLUQ_ENOMEM;
    }
    const unsigned blocks = (unsigned)ceil_div(len, UT);
    jump_init_kernel<<<blocks, UT, 0, st>>>(d_perm_p, d_perm_q, n, nxt[0], lab[0]);
    PLUQ_TRY(last_launch());
    int cur = 0;
    for (int64_t span = 1; span < n; span *= 2) {   // cycles are at most n long
        jump_kernel<<<blocks, UT, 0, st>>>(nxt[cur], lab[cur], nxt[cur ^ 1], lab[cur ^ 1], len);
        PLUQ_TRY(last_launch());
        cur ^= 1;
    }
    det_kernel<<<1, DT, 0, st>>>(d_LU, lda, n, lab[cur], F, d_det);
    return last_launch();
}

pluq_status pluq_right_nullspace(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda,
                                 int64_t r, const int32_t *d_perm_q, uint32_t p, uint32_t *d_N,
                                 int64_t ldn, int mm_kind, void *d_work, size_t ws_bytes,
                                 void *stream)
{
    if (!factor_args_ok(d_LU, m, n, lda, r)) return PLUQ_EINVAL;
    if (mm_kind < PLUQ_MM_AUTO || mm_kind > PLUQ_MM_TENSOR) return PLUQ_EINVAL;
    if (bad_modulus(p)) return PLUQ_ENOTPRIME;
    const int64_t d = n - r;
    if (d == 0) return PLUQ_OK;
    if (!d_N || !d_perm_q || ldn < d) return PLUQ_EINVAL;
    const int kind = kind_of(mm_kind);
    Arena ar = arena_of(d_work, ws_bytes);
    if (ar.size < ws_right(m, n, r, p, kind)) return PLUQ_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    const Field F = make_field(p);
    uint32_t *X = (uint32_t *)ar.take(bytes_u32(r, r));
    uint32_t *W = (uint32_t *)ar.take(bytes_u32(r, d));
    int32_t *inv = (int32_t *)ar.take(bytes_u32(1, n));
    if (!X || !W || !inv) return PLUQ_ENOMEM;
    if (r > 0) {
        PLUQ_TRY(tri_inv_upper(d_LU, lda, Blk{X, r}, r, F, kind, ar, st));      // U^{-1}
        PLUQ_TRY(launch_mm(kind, Blk{W, d}, X, r, d_LU + r, lda, r, d, r, F,    // -U^{-1} V
                           MM_NEG_ASSIGN, 1, 0, 0, 0, ar, st));
    }
    PLUQ_TRY(launch_inverse(d_perm_q, n, inv, st));
    scatter_rows_kernel<<<grid_rows(n, d), UT, 0, st>>>(d_N, ldn, n, d, W, d, inv, r, 1);
    return last_launch();
}

pluq_status pluq_left_nullspace(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda,
                                int64_t r, const int32_t *d_perm_p, uint32_t p, uint32_t *d_K,
                                int64_t ldk, int mm_kind, void *d_work, size_t ws_bytes,
                                void *stream)
{
    if (!factor_args_ok(d_LU, m, n, lda, r)) return PLUQ_EINVAL;
    if (mm_kind < PLUQ_MM_AUTO || mm_kind > PLUQ_MM_TENSOR) return PLUQ_EINVAL;
    if (bad_modulus(p)) return PLUQ_ENOTPRIME;
    const int64_t d = m - r;
    if (d == 0) return PLUQ_OK;
    if (!d_K || !d_perm_p || ldk < m) return PLUQ_EINVAL;
    const int kind = kind_of(mm_kind);
    Arena ar = arena_of(d_work, ws_bytes);
    if (ar.size < ws_left(m, n, r, p, kind)) return PLUQ_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    const Field F = make_field(p);
    uint32_t *X = (uint32_t *)ar.take(bytes_u32(r, r));
    uint32_t *W = (uint32_t *)ar.take(bytes_u32(d, r));
    int32_t *inv = (int32_t *)ar.take(bytes_u32(1, m));
    if (!X || !W || !inv) return PLUQ_ENOMEM;
    if (r > 0) {
        PLUQ_TRY(tri_inv_lower_unit(d_LU, lda, Blk{X, r}, r, F, kind, ar, st));     // L^{-1}
        PLUQ_TRY(launch_mm(kind, Blk{W, r}, d_LU + r * lda, lda, X, r, d, r, r, F,  // -M L^{-1}
                           MM_NEG_ASSIGN, 1, 0, 0, 0, ar, st));
    }
    PLUQ_TRY(launch_inverse(d_perm_p, m, inv, st));
    scatter_cols_kernel<<<grid_rows(d, m), UT, 0, st>>>(d_K, ldk, d, m, W, r, inv, r);
    return last_launch();
}

pluq_status pluq_solve(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda, int64_t r,
                       const int32_t *d_perm_p, const int32_t *d_perm_q, uint32_t p,
                       const uint32_t *d_B, int64_t ldb, int64_t k, uint32_t *d_X, int64_t ldx,
                       int32_t *d_inconsistent, int mm_kind, void *d_work, size_t ws_bytes,
                       void *stream)
{
    if (!factor_args_ok(d_LU, m, n, lda, r) || k < 0 || !d_inconsistent) return PLUQ_EINVAL;
    if (mm_kind < PLUQ_MM_AUTO || mm_kind > PLUQ_MM_TENSOR) return PLUQ_EINVAL;
    if (bad_modulus(p)) return PLUQ_ENOTPRIME;
    if (k > 0 && m > 0 && (!d_B || ldb < k || !d_perm_p)) return PLUQ_EINVAL;
    if (k > 0 && n > 0 && (!d_X || ldx < k || !d_perm_q)) return PLUQ_EINVAL;
    const int kind = kind_of(mm_kind);
    Arena ar = arena_of(d_work, ws_bytes);
    if (ar.size < ws_solve(m, n, r, k, p, kind)) return PLUQ_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    PLUQ_CUDA_TRY(cudaMemsetAsync(d_inconsistent, 0, sizeof(int32_t), st));
    if (k == 0) return PLUQ_OK;
    const Field F = make_field(p);
    uint32_t *Y = (uint32_t *)ar.take(bytes_u32(m, k));
    uint32_t *W = (uint32_t *)ar.take(bytes_u32(r, k));
    int32_t *inv = (int32_t *)ar.take(bytes_u32(1, n));
    uint32_t *X = (uint32_t *)ar.take(bytes_u32(r, r));
    if (!Y || !W || !inv || !X) return PLUQ_ENOMEM;
    // Y = P^T B, then Y <- [L 0; M I]^{-1} Y
    PLUQ_TRY(launch_gather(Blk{Y, k}, d_B, ldb, m, k, d_perm_p, nullptr, st));
    if (r > 0) {
        PLUQ_TRY(trsm_left_lower_unit(d_LU, lda, Blk{Y, k}, r, k, F, kind, ar, st));
        if (m > r)
            PLUQ_TRY(launch_mm(kind, Blk{Y + r * k, k}, d_LU + r * lda, lda, Y, k, m - r, k, r,
                               F, MM_SUB, 1, 0, 0, 0, ar, st));
    }
    if (m > r) {
        flag_nonzero_kernel<<<grid_rows(m - r < 1024 ? m - r : 1024, k), UT, 0, st>>>(
            Y + r * k, k, m - r, k, d_inconsistent);
        PLUQ_TRY(last_launch());
    }
    if (n == 0) return PLUQ_OK;
    // W = U^{-1} Y[:r], X = Q^T [W; 0]
    if (r > 0) {
        PLUQ_TRY(tri_inv_upper(d_LU, lda, Blk{X, r}, r, F, kind, ar, st));
        PLUQ_TRY(launch_mm(kind, Blk{W, k}, X, r, Y, k, r, k, r, F, MM_ASSIGN, 1, 0, 0, 0, ar,
                           st));
    }
    PLUQ_TRY(launch_inverse(d_perm_q, n, inv, st));
    scatter_rows_kernel<<<grid_rows(n, k), UT, 0, st>>>(d_X, ldx, n, k, W, k, inv, r, 0);
    return last_launch();
}

}  // extern "C"
