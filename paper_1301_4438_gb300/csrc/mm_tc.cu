// Modular matrix product MM(C, A, B) of Sec. 2 on the tcgen05 tensor cores.
//
// sm_103a has no integer tcgen05 MMA, so residues are carried exactly on the
// 16-bit floating-point path:
//   * every residue x is replaced by its centred representative c (|c| <= p/2)
//     and written as L balanced base-256 digits d_l (|d_l| <= 128), exact in
//     bf16 (limb split kernels below, one pass over A and B);
//   * digit planes are multiplied with tcgen05.mma kind::f16 (bf16 x bf16 ->
//     fp32 in TMEM).  Products with the same weight 256^s, s = i + j, share an
//     accumulator, so 2L-1 accumulators hold sum_k A_i B_j;
//   * each product of two digits is at most 2^14 in magnitude, and a K-chunk
//     bounds the number of terms per accumulator so that every partial sum
//     stays an integer of magnitude <= 2^24: fp32 holds it exactly whatever
//     the order of summation;
//   * after each chunk the epilogue warps drain TMEM, recombine
//     sum_s acc_s 256^s in 64-bit integers, reduce once mod p (the delayed
//     reduction of Sec. 5) and keep a running residue in spare TMEM columns;
//     after the last chunk they apply C <- C - AB (or the assign forms).
// One CTA computes a 128 x BN tile: warp 0 issues TMA loads (128B-swizzled
// K-major tiles) into a ring of shared-memory stages, one thread of warp 1
// issues the MMAs, warps 2-5 run the epilogue.  Every wait is bounded; a wait
// that gives up raises an error word and the kernel winds down.
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace pluq {

__device__ int g_tc_error = 0;

namespace {

constexpr int BM = 128, BK = 64;
constexpr int NTHREADS = 192;
constexpr uint32_t WAIT_LIMIT = 1u << 24;

template <int L> struct Cfg;
// KC_BLOCKS * 64 * (pairs per accumulator) * 2^14 <= 2^24
template <> struct Cfg<1> { static constexpr int BN = 128, STAGES = 6, KC_BLOCKS = 16; };
template <> struct Cfg<2> { static constexpr int BN = 128, STAGES = 3, KC_BLOCKS = 8; };
template <> struct Cfg<3> { static constexpr int BN = 64, STAGES = 3, KC_BLOCKS = 5; };
template <> struct Cfg<4> { static constexpr int BN = 64, STAGES = 2, KC_BLOCKS = 4; };

constexpr int pow2_at_least(int x)
{
    int v = 32;
    while (v < x) v <<= 1;
    return v;
}

template <int L> struct Geo {
    static constexpr int BN = Cfg<L>::BN, STAGES = Cfg<L>::STAGES, KCB = Cfg<L>::KC_BLOCKS;
    static constexpr int NACC = 2 * L - 1;
    static constexpr uint32_t A_TILE = BM * BK * 2, B_TILE = BN * BK * 2;
    static constexpr uint32_t STAGE = L * (A_TILE + B_TILE);
    static constexpr int TMEM_COLS = pow2_at_least(NACC * BN + BN);
    static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + 256;
};

// ------------------------------------------------------------ PTX glue --
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false if it gave up (or another role already did)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort)
{
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255) == 255 && *abort) return false;
    }
    *abort = 1;
    atomicExch(&g_tc_error, 1);
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand in 128B-swizzled rows of
// 64 bf16, 8-row core groups 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                 // version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D fp32, A = B = bf16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
        " [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0],"
        " {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
        "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// -------------------------------------------------------- limb splitting --
template <int L>
__device__ __forceinline__ void to_digits(uint32_t x, uint32_t p, __nv_bfloat16 (&d)[L])
{
    int32_t c = x > (p >> 1) ? -(int32_t)(p - x) : (int32_t)x;
#pragma unroll
    for (int l = 0; l < L - 1; ++l) {
        int32_t t = ((c + 128) & 255) - 128;
        d[l] = __float2bfloat16_rn((float)t);
        c = (c - t) >> 8;
    }
    d[L - 1] = __float2bfloat16_rn((float)c);
}

// A (M x K, row stride lda) -> planes[(b*L + l)*Mp + i][k], zero padded.
template <int L>
__global__ void split_rows_kernel(const uint32_t *__restrict__ A, int64_t lda, int64_t sA, int M,
                                  int K, int64_t Mp, int64_t Kp, uint32_t p,
                                  __nv_bfloat16 *__restrict__ planes)
{
    const int b = blockIdx.z;
    const int64_t k = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.y * 32;
    A += b * sA;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int64_t i = i0 + threadIdx.y + 8 * s;
        uint32_t x = (i < M && k < K) ? A[i * lda + k] : 0u;
        __nv_bfloat16 d[L];
        to_digits<L>(x, p, d);
#pragma unroll
        for (int l = 0; l < L; ++l) planes[((int64_t)(b * L + l) * Mp + i) * Kp + k] = d[l];
    }
}

// B (K x N, row stride ldb) -> planes[(b*L + l)*Np + j][k] (transposed), zero padded.
template <int L>
__global__ void split_cols_kernel(const uint32_t *__restrict__ B, int64_t ldb, int64_t sB, int K,
                                  int N, int64_t Np, int64_t Kp, uint32_t p,
                                  __nv_bfloat16 *__restrict__ planes)
{
    __shared__ __nv_bfloat16 tile[L][32][33];
    const int b = blockIdx.z;
    const int64_t k0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    B += b * sB;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int64_t k = k0 + threadIdx.y + 8 * s, j = j0 + threadIdx.x;
        uint32_t x = (k < K && j < N) ? B[k * ldb + j] : 0u;
        __nv_bfloat16 d[L];
        to_digits<L>(x, p, d);
#pragma unroll
        for (int l = 0; l < L; ++l) tile[l][threadIdx.y + 8 * s][threadIdx.x] = d[l];
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int64_t j = j0 + threadIdx.y + 8 * s, k = k0 + threadIdx.x;
#pragma unroll
        for (int l = 0; l < L; ++l)
            planes[((int64_t)(b * L + l) * Np + j) * Kp + k] = tile[l][threadIdx.x][threadIdx.y + 8 * s];
    }
}

// ------------------------------------------------------------- GEMM --
struct TcArgs {
    uint32_t *C;
    int64_t ldc, sC;
    int M, N, nkb;
    int Mp, Np;
    int mode;
    Field F;
    uint64_t off_lo, off_hi;   // multiples of p above the recombination bounds
    uint32_t w32;              // 2^32 mod p
};

template <int L>
__device__ __forceinline__ uint32_t recombine(const float *acc, const TcArgs &a)
{
    // sum_s acc_s 256^s, s < 4 in one 64-bit word (< 2^49 in magnitude), s >= 4 in another
    int64_t lo = 0, hi = 0;
#pragma unroll
    for (int s = 0; s < 2 * L - 1; ++s) {
        int64_t v = (int64_t)__float2int_rn(acc[s]);
        if (s < 4) lo += v * ((int64_t)1 << (8 * s));
        else hi += v * ((int64_t)1 << (8 * (s - 4)));
    }
    uint32_t t = reduce64((uint64_t)(lo + (int64_t)a.off_lo), a.F);
    if (2 * L - 1 > 4) {
        uint32_t th = reduce64((uint64_t)(hi + (int64_t)a.off_hi), a.F);
        t = add_mod(t, mul_mod(th, a.w32, a.F), a.F.p);
    }
    return t;
}

template <int L>
__global__ void __launch_bounds__(NTHREADS, 1)
    mm_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                 TcArgs a)
{
    using G = Geo<L>;
    constexpr int BN = G::BN, STAGES = G::STAGES, KCB = G::KCB, NACC = G::NACC;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t *smem = smem_raw + (sbase - raw);
    uint64_t *bars = (uint64_t *)(smem + STAGES * G::STAGE);
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * STAGES + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    auto full_bar = [&](int s) { return smem_u32(&bars[s]); };
    auto empty_bar = [&](int s) { return smem_u32(&bars[STAGES + s]); };
    const uint32_t acc_full = smem_u32(&bars[2 * STAGES]);
    const uint32_t acc_empty = smem_u32(&bars[2 * STAGES + 1]);
    auto a_tile = [&](int s, int l) { return sbase + s * G::STAGE + l * G::A_TILE; };
    auto b_tile = [&](int s, int l) { return sbase + s * G::STAGE + L * G::A_TILE + l * G::B_TILE; };

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, 128);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(G::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int bz = blockIdx.z;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int nkb = a.nkb;
    const int nchunks = (nkb + KCB - 1) / KCB;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % STAGES;
                const uint32_t ph = (kb / STAGES) & 1;
                if (!mbar_wait(empty_bar(s), ph ^ 1, abort_flag)) break;
                mbar_expect_tx(full_bar(s), G::STAGE);
#pragma unroll
                for (int l = 0; l < L; ++l)
                    tma_load_2d(a_tile(s, l), &mapA, kb * BK, (bz * L + l) * a.Mp + m0, full_bar(s));
#pragma unroll
                for (int l = 0; l < L; ++l)
                    tma_load_2d(b_tile(s, l), &mapB, kb * BK, (bz * L + l) * a.Np + n0, full_bar(s));
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(BM, BN);
            int kb = 0;
            bool ok = true;
            for (int c = 0; c < nchunks && ok; ++c) {
                if (c > 0 && !mbar_wait(acc_empty, (c - 1) & 1, abort_flag)) break;
                tc_fence_after();
                uint32_t started = 0;
                const int kend = min(nkb, (c + 1) * KCB);
                for (; kb < kend; ++kb) {
                    const int s = kb % STAGES;
                    if (!mbar_wait(full_bar(s), (kb / STAGES) & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int i = 0; i < L; ++i)
#pragma unroll
                        for (int j = 0; j < L; ++j) {
                            const int acc = i + j;
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk) {
                                const uint64_t da = sdesc(a_tile(s, i) + kk * 32);
                                const uint64_t db = sdesc(b_tile(s, j) + kk * 32);
                                mma_bf16(tmem + acc * BN, da, db, idesc, (started >> acc) & 1);
                                started |= 1u << acc;
                            }
                        }
                    mma_commit(empty_bar(s));
                }
                if (ok) mma_commit(acc_full);
            }
        }
    } else {
        // ---------------- epilogue: warps 2..5, TMEM lanes 32*(warp%4) ...
        const int q = warp % 4;
        const int row = q * 32 + lane;
        const int grow = m0 + row;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        uint32_t *Cb = a.C + (int64_t)bz * a.sC;
        const uint32_t p = a.F.p;
        for (int c = 0; c < nchunks; ++c) {
            if (!mbar_wait(acc_full, c & 1, abort_flag)) break;
            tc_fence_after();
            const bool last = c == nchunks - 1;
#pragma unroll 1
            for (int cs = 0; cs < BN; cs += 16) {
                uint32_t raw_acc[NACC][16];
#pragma unroll
                for (int s = 0; s < NACC; ++s) tmem_ld16(tl + s * BN + cs, raw_acc[s]);
                uint32_t run[16];
                if (c > 0) tmem_ld16(tl + NACC * BN + cs, run);
                tmem_wait_ld();
                uint32_t t[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float acc[NACC];
#pragma unroll
                    for (int s = 0; s < NACC; ++s) acc[s] = __uint_as_float(raw_acc[s][j]);
                    t[j] = recombine<L>(acc, a);
                    if (c > 0) t[j] = add_mod(t[j], run[j], p);
                }
                if (!last) {
                    tmem_st16(tl + NACC * BN + cs, t);
                } else if (grow < a.M) {
                    uint32_t *crow = Cb + (int64_t)grow * a.ldc + n0 + cs;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (n0 + cs + j >= a.N) break;
                        uint32_t out;
                        if (a.mode == MM_SUB) out = sub_mod(crow[j], t[j], p);
                        else if (a.mode == MM_ASSIGN) out = t[j];
                        else out = t[j] == 0 ? 0u : p - t[j];
                        crow[j] = out;
                    }
                }
            }
            if (!last) tmem_wait_st();
            tc_fence_before();
            mbar_arrive(acc_empty);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(G::TMEM_COLS)
                     : "memory");
    }
}

// ------------------------------------------------------------- host --
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    // thread-safe one-time lookup (function-local static initialisation)
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (EncodeTiledFn)p;
        return nullptr;
    }();
    return fn;
}

bool make_map(CUtensorMap *map, void *base, int64_t rows, int64_t kp, int box_rows)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int bn_for(int L) { return L <= 2 ? 128 : 64; }

template <int L>
pluq_status run_tc(Blk C, const uint32_t *A, int64_t lda, const uint32_t *B, int64_t ldb, int64_t M,
                   int64_t N, int64_t K, Field F, int mode, int64_t batch, int64_t sA, int64_t sB,
                   int64_t sC, Arena &ar, cudaStream_t st)
{
    using G = Geo<L>;
    const int64_t Mp = ceil_div(M, BM) * BM, Np = ceil_div(N, G::BN) * G::BN;
    const int64_t Kp = ceil_div(K, BK) * BK;
    const size_t mark = ar.off;
    auto *pa = (__nv_bfloat16 *)ar.take((size_t)batch * L * Mp * Kp * 2, 1024);
    auto *pb = (__nv_bfloat16 *)ar.take((size_t)batch * L * Np * Kp * 2, 1024);
    if (!pa || !pb) return PLUQ_ENOMEM;
    const uint32_t p = F.p;
    dim3 blk(32, 8);
    prof::start(prof::SPLIT, st);
    split_rows_kernel<L><<<dim3((unsigned)(Kp / 32), (unsigned)(Mp / 32), (unsigned)batch), blk, 0,
                           st>>>(A, lda, sA, (int)M, (int)K, Mp, Kp, p, pa);
    PLUQ_TRY(last_launch());
    split_cols_kernel<L><<<dim3((unsigned)(Kp / 32), (unsigned)(Np / 32), (unsigned)batch), blk, 0,
                           st>>>(B, ldb, sB, (int)K, (int)N, Np, Kp, p, pb);
    PLUQ_TRY(last_launch());
    prof::stop(prof::SPLIT, st, (double)batch * ((M + N) * K * 4.0 + (Mp + Np) * Kp * 2.0 * L));

    CUtensorMap ma, mb;
    if (!make_map(&ma, pa, batch * L * Mp, Kp, BM)) return PLUQ_ECUDA;
    if (!make_map(&mb, pb, batch * L * Np, Kp, G::BN)) return PLUQ_ECUDA;

    static const bool attr = cudaFuncSetAttribute(mm_tc_kernel<L>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)G::SMEM) == cudaSuccess;
    if (!attr) return PLUQ_ECUDA;
    TcArgs a;
    a.C = C.ptr;
    a.ldc = C.ld;
    a.sC = sC;
    a.M = (int)M;
    a.N = (int)N;
    a.nkb = (int)(Kp / BK);
    a.Mp = (int)Mp;
    a.Np = (int)Np;
    a.mode = mode;
    a.F = F;
    a.off_lo = ((1ull << 50) / p + 1) * p;
    a.off_hi = ((1ull << 42) / p + 1) * p;
    a.w32 = (uint32_t)((1ull << 32) % p);
    dim3 grid((unsigned)(Np / G::BN), (unsigned)(Mp / BM), (unsigned)batch);
    prof::start(prof::TC_MM, st);
    mm_tc_kernel<L><<<grid, NTHREADS, G::SMEM, st>>>(ma, mb, a);
    PLUQ_TRY(last_launch());
    // algorithmic tensor work: L^2 digit products of an M x K by K x N product
    prof::stop(prof::TC_MM, st, 2.0 * L * L * (double)M * N * K * batch);
    ar.off = mark;
    return PLUQ_OK;
}

}  // namespace

int tc_error_flag()
{
    int v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)) != cudaSuccess) return 0;
    if (v) cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int));
    return v;
}

size_t mm_tc_workspace(int64_t M, int64_t N, int64_t K, uint32_t p, int64_t batch)
{
    const int L = limbs_for_prime(p);
    const int64_t bn = bn_for(L);
    const int64_t Mp = ceil_div(M > 0 ? M : 1, BM) * BM, Np = ceil_div(N > 0 ? N : 1, bn) * bn;
    const int64_t Kp = ceil_div(K > 0 ? K : 1, BK) * BK;
    return (size_t)batch * L * (Mp + Np) * Kp * 2 + 4096;
}

pluq_status launch_mm_tc(Blk C, const uint32_t *A, int64_t lda, const uint32_t *B, int64_t ldb,
                         int64_t M, int64_t N, int64_t K, Field F, int mode, int64_t batch,
                         int64_t sA, int64_t sB, int64_t sC, Arena &ar, cudaStream_t st)
{
    if (M <= 0 || N <= 0 || batch <= 0) return PLUQ_OK;
    if (K == 0) {
        if (mode == MM_SUB) return PLUQ_OK;
        for (int64_t b = 0; b < batch; ++b)
            PLUQ_TRY(launch_zero(Blk{C.ptr + b * sC, C.ld}, M, N, st));
        return PLUQ_OK;
    }
    if (M > (1 << 30) || N > (1 << 30) || K > (1 << 30) || batch > 65535) return PLUQ_EINVAL;
    switch (limbs_for_prime(F.p)) {
        case 1: return run_tc<1>(C, A, lda, B, ldb, M, N, K, F, mode, batch, sA, sB, sC, ar, st);
        case 2: return run_tc<2>(C, A, lda, B, ldb, M, N, K, F, mode, batch, sA, sB, sC, ar, st);
        case 3: return run_tc<3>(C, A, lda, B, ldb, M, N, K, F, mode, batch, sA, sB, sC, ar, st);
        case 4: return run_tc<4>(C, A, lda, B, ldb, M, N, K, F, mode, batch, sA, sB, sC, ar, st);
        default: return PLUQ_EUNSUPPORTED;
    }
}

}  // namespace pluq

// ------------------------------------------------------- allocation-free --
// Scratch of pluq_modmm_tensor_noalloc: the limb planes of A and B live in this
// fixed array instead of a caller-provided workspace.  Every device that loads
// the library keeps it (PLUQ_NOALLOC_SCRATCH_BYTES) until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PLUQ_NOALLOC_SCRATCH_BYTES];

#include <mutex>

namespace pluq {
namespace {
std::mutex g_noalloc_mu;
constexpr int MAX_DEVICES = 256;
void *g_noalloc_addr[MAX_DEVICES] = {};   // device address of the array, per device ordinal
}  // namespace
}  // namespace pluq

extern "C" pluq_status pluq_modmm_tensor_noalloc(uint32_t *d_C, int64_t ldc, const uint32_t *d_A,
                                                 int64_t lda, const uint32_t *d_B, int64_t ldb,
                                                 int64_t M, int64_t N, int64_t K, uint32_t p,
                                                 int assign, void *stream)
{
    using namespace pluq;
    if (M < 0 || N < 0 || K < 0) return PLUQ_EINVAL;
    if (p < 2 || p >= 0x80000000u) return PLUQ_ENOTPRIME;
    for (uint64_t d = 2; d * d <= p; ++d)
        if (p % d == 0) return PLUQ_ENOTPRIME;
    if (M > 0 && N > 0 && (!d_C || ldc < N)) return PLUQ_EINVAL;
    if (M > 0 && K > 0 && (!d_A || lda < K)) return PLUQ_EINVAL;
    if (K > 0 && N > 0 && (!d_B || ldb < N)) return PLUQ_EINVAL;
    if (mm_tc_workspace(M, N, K, p, 1) > (size_t)PLUQ_NOALLOC_SCRATCH_BYTES) return PLUQ_ENOMEM;

    // set-up once per device, with that device current: the host-side name of
    // the array is not a device address, so look the address up and keep it
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return PLUQ_ECUDA;
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr)
                return PLUQ_ECUDA;
            g_noalloc_addr[dev] = ptr;
        }
        base = g_noalloc_addr[dev];
    }
    Arena ar;
    ar.base = (char *)base;
    ar.size = PLUQ_NOALLOC_SCRATCH_BYTES;
    ar.off = 0;
    return launch_mm_tc(Blk{d_C, ldc}, d_A, lda, d_B, ldb, M, N, K, make_field(p),
                        assign ? MM_ASSIGN : MM_SUB, 1, 0, 0, 0, ar, (cudaStream_t)stream);
}
