// Modular matrix product on the CUDA cores: MM(C, A, B) of Sec. 2,
// C <- C - A B (mod p), plus the assign / negated-assign / add forms the
// triangular-inverse and TRSM code needs.
//
// Each product of two residues is formed exactly as a 64-bit integer and the
// sums are reduced once per output element (the delayed reduction of Sec. 6):
//   p <= 2^16 : a b < 2^32, a 64-bit accumulator holds 2^32 of them;
//   p  > 2^16 : a = a_hi 2^16 + a_lo, a_lo b < 2^47 and a_hi b < 2^46, two
//               64-bit accumulators hold 2^17 terms each (K is cut into
//               chunks of 2^16 by the launcher).
// T x T output tile per block (T = 64, 32 or 16: the largest that still gives
// every SM a block), 256 threads, (T/16)^2 outputs per thread, 16-deep K
// slices staged in shared memory.
#include <initializer_list>

#include "common.cuh"

namespace pluq {
namespace {

constexpr int BK = 16, NT = 256;
enum { MODE_SUB = 0, MODE_ASSIGN = 1, MODE_NEG_ASSIGN = 2, MODE_ADD = 3 };

template <bool BIG, int T>
__global__ void __launch_bounds__(NT) mm_simt_kernel(
    uint32_t *__restrict__ C, int64_t ldc, const uint32_t *__restrict__ A, int64_t lda,
    const uint32_t *__restrict__ B, int64_t ldb, int M, int N, int K, Field F, int mode,
    int64_t sA, int64_t sB, int64_t sC)
{
    constexpr int BM = T, BN = T, R = T / 16;   // R x R outputs per thread
    __shared__ uint32_t As[BK][BM + 4];
    __shared__ uint32_t Bs[BK][BN + 4];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
    const int64_t b = blockIdx.z;
    A += b * sA;
    B += b * sB;
    C += b * sC;

    uint64_t acc_lo[R][R], acc_hi[R][R];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc_lo[i][j] = acc_hi[i][j] = 0;

    for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
        for (int s = 0; s < R; ++s) {
            int r = tid / 16 + 16 * s, kk = tid % 16;
            int gr = row0 + r, gk = k0 + kk;
            As[kk][r] = (gr < M && gk < K) ? A[(int64_t)gr * lda + gk] : 0u;
            int idx = tid + NT * s;
            int kb = idx / BN, cb = idx % BN;
            int gk2 = k0 + kb, gc = col0 + cb;
            Bs[kb][cb] = (gk2 < K && gc < N) ? B[(int64_t)gk2 * ldb + gc] : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            uint32_t a[R], bv[R];
#pragma unroll
            for (int i = 0; i < R; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < R; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    if (BIG) {
                        acc_lo[i][j] += (uint64_t)(a[i] & 0xFFFFu) * bv[j];
                        acc_hi[i][j] += (uint64_t)(a[i] >> 16) * bv[j];
                    } else {
                        acc_lo[i][j] += (uint64_t)(a[i] * bv[j]);   // < 2^32
                    }
                }
        }
        __syncthreads();
    }

    const uint32_t p = F.p;
    const uint32_t w16 = (uint32_t)((1ull << 16) % p);
#pragma unroll
    for (int i = 0; i < R; ++i) {
        int gr = row0 + ty + 16 * i;
        if (gr >= M) continue;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            int gc = col0 + tx + 16 * j;
            if (gc >= N) continue;
            uint32_t t = reduce64(acc_lo[i][j], F);
            if (BIG) t = add_mod(t, mul_mod(reduce64(acc_hi[i][j], F), w16, F), p);
            uint32_t *c = C + (int64_t)gr * ldc + gc;
            uint32_t out;
            switch (mode) {
                case MODE_SUB: out = sub_mod(*c, t, p); break;
                case MODE_ASSIGN: out = t; break;
                case MODE_NEG_ASSIGN: out = t == 0 ? 0u : p - t; break;
                default: out = add_mod(*c, t, p); break;
            }
            *c = out;
        }
    }
}

}  // namespace

pluq_status launch_mm_simt(Blk C, const uint32_t *A, int64_t lda, const uint32_t *B,
                           int64_t ldb, int64_t M, int64_t N, int64_t K, Field F, int mode,
                           int64_t batch, int64_t sA, int64_t sB, int64_t sC, cudaStream_t st)
{
    if (M <= 0 || N <= 0 || batch <= 0) return PLUQ_OK;
    if (M > (1ll << 30) || N > (1ll << 30) || batch > 65535) return PLUQ_EINVAL;
    const bool big = F.p > 65536u;
    const int64_t kchunk = big ? (1ll << 16) : (1ll << 30);
    if (K == 0) {
        // empty product: SUB leaves C, ASSIGN / NEG_ASSIGN zero it
        if (mode == MM_SUB) return PLUQ_OK;
        for (int64_t b = 0; b < batch; ++b)
            PLUQ_TRY(launch_zero(Blk{C.ptr + b * sC, C.ld}, M, N, st));
        return PLUQ_OK;
    }
    // the largest tile that still gives every SM a block
    int tile = 16;
    for (int t : {64, 32})
        if (ceil_div(M, t) * ceil_div(N, t) * batch >= 148) {
            tile = t;
            break;
        }
    dim3 grid((unsigned)ceil_div(N, tile), (unsigned)ceil_div(M, tile), (unsigned)batch);
    for (int64_t k0 = 0; k0 < K; k0 += kchunk) {
        int64_t kc = K - k0 < kchunk ? K - k0 : kchunk;
        int md = mode;
        if (k0 > 0) md = (mode == MM_ASSIGN) ? MODE_ADD : MODE_SUB;
        prof::start(prof::SIMT_MM, st);
#define PLUQ_SIMT_CASE(BIGP, T)                                                                   \
    if (big == BIGP && tile == T)                                                                \
        mm_simt_kernel<BIGP, T><<<grid, NT, 0, st>>>(C.ptr, C.ld, A + k0, lda, B + k0 * ldb, ldb, \
                                                     (int)M, (int)N, (int)kc, F, md, sA, sB, sC);
        PLUQ_SIMT_CASE(true, 64) PLUQ_SIMT_CASE(true, 32) PLUQ_SIMT_CASE(true, 16)
        PLUQ_SIMT_CASE(false, 64) PLUQ_SIMT_CASE(false, 32) PLUQ_SIMT_CASE(false, 16)
#undef PLUQ_SIMT_CASE
        PLUQ_TRY(last_launch());
        prof::stop(prof::SIMT_MM, st, 2.0 * (double)M * N * kc * batch);
    }
    return PLUQ_OK;
}

}  // namespace pluq
