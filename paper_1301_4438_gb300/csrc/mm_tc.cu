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
//   * each stage's MMAs for one A digit plane i run against the L B planes
//     stacked along N (one MMA of width L*BN), so block j of the result lands
//     on accumulator i + j: L MMAs per 16-wide K step instead of L^2;
//   * the CTA is persistent: it walks output tiles (grouped along M so that
//     concurrent CTAs share A and B panels in L2) and keeps two accumulator
//     sets in TMEM, so the MMAs of one K-chunk run while the epilogue warps
//     drain the previous one;
//   * the epilogue folds each chunk into a running residue kept in registers
//     (the delayed reduction of Sec. 6: one reduction per chunk, not per
//     product): for two limbs entirely in exact fp32 arithmetic, otherwise as
//     one 64-bit dot product with the weights 256^s mod p and one Barrett
//     reduction; after a tile's last chunk it applies C <- C - AB (or the
//     assign forms) through shared memory, coalesced.
// Warp 0 issues TMA loads (128B-swizzled K-major tiles) into a ring of
// shared-memory stages, one thread of warp 1 issues the MMAs, warps 2-9 run
// the epilogue.  Every wait is bounded; a wait that gives up raises an error
// word and the kernel winds down after its own copies and MMAs have landed.
#include <cuda.h>
#include <algorithm>
#include <climits>
#include <cuda_bf16.h>

#include "common.cuh"

namespace pluq {

__device__ int g_tc_error = 0;

namespace {

constexpr int BM = 128, BK = 64;
constexpr int NTHREADS = 320;          // TMA warp, MMA warp, 8 epilogue warps
constexpr int EPI_WARPS = 8;
constexpr int GROUP_M = 8;             // tile raster: GROUP_M row tiles per column sweep
constexpr uint32_t WAIT_LIMIT = 1u << 24;

// Tile width BN: two accumulator sets of (2L-1) x BN fp32 columns fit in the
// 512 TMEM columns; the stacked MMA is L*BN wide (at most 256).
// KC_BLOCKS * 64 * (digit pairs per accumulator) * 2^14 <= 2^24.
template <int L> struct Cfg;
template <> struct Cfg<1> { static constexpr int BN = 128, STAGES = 6, KC_BLOCKS = 16; };
template <> struct Cfg<2> { static constexpr int BN = 80, STAGES = 4, KC_BLOCKS = 8; };
template <> struct Cfg<3> { static constexpr int BN = 48, STAGES = 3, KC_BLOCKS = 5; };
template <> struct Cfg<4> { static constexpr int BN = 32, STAGES = 2, KC_BLOCKS = 4; };

template <int L> struct Geo {
    static constexpr int BN = Cfg<L>::BN, STAGES = Cfg<L>::STAGES, KCB = Cfg<L>::KC_BLOCKS;
    static constexpr int NACC = 2 * L - 1;
    static constexpr int CW = BN / 2;   // columns per epilogue thread
    static constexpr uint32_t A_TILE = BM * BK * 2, B_TILE = BN * BK * 2;
    static constexpr uint32_t STAGE = L * (A_TILE + B_TILE);
    static constexpr int TMEM_COLS = 512;
    static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + 256 + EPI_WARPS * 32 * 9 * 4;
    static_assert(2 * NACC * BN <= TMEM_COLS, "two accumulator sets must fit in TMEM");
    static_assert(L * BN <= 256 && BN % 16 == 0 && CW % 8 == 0, "MMA shape");
    static_assert(B_TILE % 1024 == 0, "stacked B planes must keep the swizzle atom");
    static_assert(SMEM <= 232448, "shared memory");
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

// bounded wait of at most `limit` tries; false if it gave up (or another role
// already did)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort,
                                          uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it) {
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

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

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

// One launch splits both operands of every product of a group.  Each product
// (and each entry b of its batch) is one z-slice of the grid; block rows
// y < Mp/32 take A (M x K, row stride lda) -> planes_a[rowA + (b*L + l)*Mp + i][k],
// the others take B (K x N, row stride ldb) -> planes_b[rowB + (b*L + l)*Np + j][k],
// transposed through shared memory.  Both zero padded; Np is a multiple of the
// tile width, not necessarily of 32.
struct SplitProb {
    const uint32_t *A, *B;
    int64_t lda, sA, ldb, sB;
    int M, N, batch;
    int64_t Mp, Np, rowA, rowB;
};
constexpr int MAXG = 2;       // products per grouped launch
struct SplitArgs {
    SplitProb g[MAXG];
    int ng, K;
    int64_t Kp;
    uint32_t p;
};

template <int L>
__global__ void split_kernel(const __grid_constant__ SplitArgs sa,
                             __nv_bfloat16 *__restrict__ planes_a,
                             __nv_bfloat16 *__restrict__ planes_b)
{
    __shared__ __nv_bfloat16 tile[L][32][33];
    int b = blockIdx.z, gi = 0;
    while (gi < sa.ng - 1 && b >= sa.g[gi].batch) {
        b -= sa.g[gi].batch;
        ++gi;
    }
    const SplitProb &g = sa.g[gi];
    const int M = g.M, N = g.N, K = sa.K;
    const int64_t Mp = g.Mp, Np = g.Np, Kp = sa.Kp;
    const uint32_t p = sa.p;
    const uint32_t *A = g.A + b * g.sA;
    const uint32_t *B = g.B + b * g.sB;
    const int64_t lda = g.lda, ldb = g.ldb;
    const int64_t k0 = (int64_t)blockIdx.x * 32;
    const int64_t ya = Mp / 32, ytot = ya + (Np + 31) / 32;
    for (int64_t by = blockIdx.y; by < ytot; by += gridDim.y) {
        if (by < ya) {
            const int64_t k = k0 + threadIdx.x;
            const int64_t i0 = by * 32;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int64_t i = i0 + threadIdx.y + 8 * s;
                uint32_t x = (i < M && k < K) ? A[i * lda + k] : 0u;
                __nv_bfloat16 d[L];
                to_digits<L>(x, p, d);
#pragma unroll
                for (int l = 0; l < L; ++l)
                    planes_a[(g.rowA + (int64_t)(b * L + l) * Mp + i) * Kp + k] = d[l];
            }
            continue;
        }
        const int64_t j0 = (by - ya) * 32;
        __syncthreads();   // the previous round's reads of the tile are done
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
                if (j < Np)
                    planes_b[(g.rowB + (int64_t)(b * L + l) * Np + j) * Kp + k] =
                        tile[l][threadIdx.x][threadIdx.y + 8 * s];
        }
    }
}

// ------------------------------------------------------------- GEMM --
// One product of a grouped launch (a batch of equally shaped ones); its planes
// start at rows rowA / rowB of the stacked plane tensors.
struct TcProb {
    uint32_t *C;
    int64_t ldc, sC;
    int M, N;
    int Mp, Np;
    int ntm, ntn;              // row and column tiles of one batch entry
    int tiles;                 // tiles over the whole batch
    int rowA, rowB;
    int mode;
};
struct TcArgs {
    TcProb g[MAXG];
    int ng;
    int nkb;                   // K blocks, shared by every product of the group
    int ntiles;                // tiles over the whole group
    Field F;
    float pf, pinv;            // p and 1/p rounded to fp32 (two-limb recombination)
    uint64_t off;              // multiple of p above the recombination bound (L != 2)
    uint32_t w[7];             // 256^s mod p
    uint32_t wait_limit;       // tries of each pipeline wait before the kernel gives up
};

// Chunk recombination, two limbs (257 < p < 2^17).  Every value below is an
// integer held exactly in fp32 (magnitude < 2^24):
//   fred(x): x - q p with q = rint(x * RN(1/p)), |result| <= 0.506 p;
//   r_s = fred(acc_s); y = fred(r_1 + 256 r_2); run = fred(run + r_0 + 256 y).
// |r_1 + 256 r_2| <= 257 * 0.506 p < 2^24 and the rint magic constant needs
// |x / p| < 2^22, which holds for |x| <= 2^24 + 2^23 and p > 257.
__device__ __forceinline__ float fred(float x, float pf, float pinv)
{
    const float M = 12582912.0f;   // 1.5 * 2^23: adding it rounds to an integer
    const float q = __fsub_rn(__fmaf_rn(x, pinv, M), M);
    return __fmaf_rn(-q, pf, x);
}

template <int L>
__device__ __forceinline__ uint32_t chunk_update(const uint32_t (&raw)[2 * L - 1][8], int j,
                                                 uint32_t run, bool first, const TcArgs &a)
{
    if constexpr (L == 2) {
        const float r0 = fred(__uint_as_float(raw[0][j]), a.pf, a.pinv);
        const float r1 = fred(__uint_as_float(raw[1][j]), a.pf, a.pinv);
        const float r2 = fred(__uint_as_float(raw[2][j]), a.pf, a.pinv);
        const float y = fred(__fmaf_rn(256.0f, r2, r1), a.pf, a.pinv);
        float z = __fmaf_rn(256.0f, y, r0);
        if (!first) z = __fadd_rn(z, __uint_as_float(run));
        return __float_as_uint(fred(z, a.pf, a.pinv));
    } else {
        // sum_s acc_s (256^s mod p) + run + off: |acc_s| <= 2^24, so < 2^60
        int64_t x = (int64_t)a.off + (first ? 0 : (int64_t)run);
#pragma unroll
        for (int s = 0; s < 2 * L - 1; ++s)
            x += (int64_t)__float2int_rn(__uint_as_float(raw[s][j])) * (int64_t)(int32_t)a.w[s];
        return reduce64((uint64_t)x, a.F);
    }
}

// running value after the last chunk -> residue in [0, p)
template <int L>
__device__ __forceinline__ uint32_t chunk_final(uint32_t run, uint32_t p)
{
    if constexpr (L == 2) {
        const int v = __float2int_rn(__uint_as_float(run));   // |v| <= 0.506 p
        return (uint32_t)(v < 0 ? v + (int)p : v);
    } else {
        return run;
    }
}

// Persistent tile order: the products of the group one after the other, in
// each the batch entries one after the other, in each GROUP_M row tiles swept
// across all column tiles before the next GROUP_M.
template <int BN>
__device__ __forceinline__ void tile_of(int t, const TcArgs &a, int &gi, int &bz, int &m0, int &n0)
{
    gi = 0;
    while (gi < a.ng - 1 && t >= a.g[gi].tiles) {
        t -= a.g[gi].tiles;
        ++gi;
    }
    const TcProb &g = a.g[gi];
    const int per = g.ntm * g.ntn;
    bz = t / per;
    const int r = t - bz * per;
    const int span = GROUP_M * g.ntn;
    const int grp = r / span;
    const int first = grp * GROUP_M;
    const int gm = min(GROUP_M, g.ntm - first);
    const int w = r - grp * span;
    m0 = (first + w % gm) * BM;
    n0 = (w / gm) * BN;
}

// wait used while winding down: bounded, ignores the abort word
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity)
{
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it)
        if (mbar_try(bar, parity)) return;
    atomicExch(&g_tc_error, 1);
}

template <int L>
__global__ void __launch_bounds__(NTHREADS, 1)
    mm_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                 TcArgs a)
{
    using G = Geo<L>;
    constexpr int BN = G::BN, STAGES = G::STAGES, KCB = G::KCB, NACC = G::NACC, CW = G::CW;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t *smem = smem_raw + (sbase - raw);
    uint64_t *bars = (uint64_t *)(smem + STAGES * G::STAGE);
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * STAGES + 5);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    auto full_bar = [&](int s) { return smem_u32(&bars[s]); };
    auto empty_bar = [&](int s) { return smem_u32(&bars[STAGES + s]); };
    auto acc_full = [&](int b) { return smem_u32(&bars[2 * STAGES + b]); };
    auto acc_empty = [&](int b) { return smem_u32(&bars[2 * STAGES + 2 + b]); };
    const uint32_t mma_done = smem_u32(&bars[2 * STAGES + 4]);
    // per epilogue warp: 32 x 8 words of C, rows padded to 9 words
    uint32_t *stg_all = (uint32_t *)(smem + STAGES * G::STAGE + 256);
    auto a_tile = [&](int s, int l) { return sbase + s * G::STAGE + l * G::A_TILE; };
    auto b_tile = [&](int s, int l) { return sbase + s * G::STAGE + L * G::A_TILE + l * G::B_TILE; };

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full(b), 1);
            mbar_init(acc_empty(b), EPI_WARPS);
        }
        mbar_init(mma_done, 1);
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

    const int nkb = a.nkb;
    const int nchunks = (nkb + KCB - 1) / KCB;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0, issued = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
                int gi, bz, m0, n0;
                tile_of<BN>(t, a, gi, bz, m0, n0);
                const int ra = a.g[gi].rowA + bz * L * a.g[gi].Mp + m0;
                const int rb = a.g[gi].rowB + bz * L * a.g[gi].Np + n0;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(empty_bar(s), ph ^ 1, abort_flag, a.wait_limit)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(full_bar(s), G::STAGE);
#pragma unroll
                    for (int l = 0; l < L; ++l)
                        tma_load_2d(a_tile(s, l), &mapA, kb * BK, ra + l * a.g[gi].Mp, full_bar(s));
#pragma unroll
                    for (int l = 0; l < L; ++l)
                        tma_load_2d(b_tile(s, l), &mapB, kb * BK, rb + l * a.g[gi].Np, full_bar(s));
                    ++issued;
                    if (++s == STAGES) {
                        s = 0;
                        ph ^= 1;
                    }
                }
            }
            // wind down: the copies of the last STAGES loads must have landed
            for (uint32_t k = 0; k < (uint32_t)STAGES && k < issued; ++k) {
                if (--s < 0) {
                    s = STAGES - 1;
                    ph ^= 1;
                }
                mbar_drain(full_bar(s), ph);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t ID_ALL = idesc_bf16(BM, L * BN);
            constexpr uint32_t ID_LOW = idesc_bf16(BM, (L > 1 ? L - 1 : 1) * BN);
            constexpr uint32_t ID_ONE = idesc_bf16(BM, BN);
            int s = 0;
            uint32_t ph = 0, cc = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
                for (int c = 0; c < nchunks && ok; ++c, ++cc) {
                    const int buf = cc & 1;
                    if (!mbar_wait(acc_empty(buf), ((cc >> 1) & 1) ^ 1, abort_flag, a.wait_limit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dacc = tmem + (uint32_t)(buf * NACC * BN);
                    const int kend = min(nkb, (c + 1) * KCB);
                    for (int kb = c * KCB; kb < kend; ++kb) {
                        if (!mbar_wait(full_bar(s), ph, abort_flag, a.wait_limit)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
                            const uint64_t db = sdesc(b_tile(s, 0) + kk * 32);
                            const bool first = kb == c * KCB && kk == 0;
#pragma unroll
                            for (int i = 0; i < L; ++i) {
                                // A_i x [B_0 .. B_{L-1}] -> accumulators i .. i+L-1
                                const uint64_t da = sdesc(a_tile(s, i) + kk * 32);
                                const uint32_t d = dacc + (uint32_t)(i * BN);
                                if (!first) {
                                    mma_bf16(d, da, db, ID_ALL, 1);
                                } else if (i == 0) {
                                    mma_bf16(d, da, db, ID_ALL, 0);
                                } else {
                                    // first step of a chunk: accumulator i+L-1 is fresh
                                    mma_bf16(d, da, db, ID_LOW, 1);
                                    mma_bf16(d + (uint32_t)((L - 1) * BN), da,
                                             sdesc(b_tile(s, L - 1) + kk * 32), ID_ONE, 0);
                                }
                            }
                        }
                        mma_commit(empty_bar(s));
                        if (++s == STAGES) {
                            s = 0;
                            ph ^= 1;
                        }
                    }
                    if (ok) mma_commit(acc_full(buf));
                }
            }
            // wind down: every MMA issued above has completed
            mma_commit(mma_done);
            mbar_drain(mma_done, 0);
        }
    } else {
        // ---------------- epilogue: warps 2..9; TMEM lanes 32*(warp%4) ..,
        // column half (warp-2)/4 of the tile
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * CW);
        const uint32_t p = a.F.p;
        uint32_t *stg = stg_all + (warp - 2) * 32 * 9;
        uint32_t cc = 0;
        bool ok = true;
        uint32_t res[CW];
        for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
            int gi, bz, m0, n0;
            tile_of<BN>(t, a, gi, bz, m0, n0);
            const TcProb &g = a.g[gi];
            for (int c = 0; c < nchunks; ++c, ++cc) {
                const int buf = cc & 1;
                if (!mbar_wait(acc_full(buf), (cc >> 1) & 1, abort_flag, a.wait_limit)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tb = tl + (uint32_t)(buf * NACC * BN);
                // TMEM loads of this thread's columns in flight together, in one
                // group (or two, where the registers would not hold one)
                constexpr int NSL = CW / 8, NGRP = L == 1 ? 4 : (L == 2 ? 2 : 1);
                constexpr int GSL = (NSL + NGRP - 1) / NGRP;
#pragma unroll
                for (int g = 0; g < NGRP; ++g) {
                    uint32_t rawv[GSL][NACC][8];
#pragma unroll
                    for (int k = 0; k < GSL; ++k)
                        if (g * GSL + k < NSL)
#pragma unroll
                            for (int s = 0; s < NACC; ++s)
                                tmem_ld8(tb + s * BN + (g * GSL + k) * 8, rawv[k][s]);
                    tmem_wait_ld();
                    if (g == NGRP - 1) {
                        // accumulators read: hand the set back to the MMA issuer
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(acc_empty(buf));
                    }
#pragma unroll
                    for (int k = 0; k < GSL; ++k)
                        if (g * GSL + k < NSL)
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const int e = (g * GSL + k) * 8 + j;
                                res[e] = chunk_update<L>(rawv[k], j, res[e], c == 0, a);
                            }
                }
            }
            if (!ok) break;
            // C update, coalesced: each 32-row x 8-column block of this warp goes
            // through shared memory so that a warp access covers 4 rows x 32
            // bytes; all loads of C are in flight before the first store
            const int col0 = n0 + half * CW;
            const int rr = lane >> 3, cq = lane & 7;
            const int grow0 = m0 + q * 32 + rr;
            uint32_t *base = g.C + (int64_t)bz * g.sC + (int64_t)grow0 * g.ldc + col0 + cq;
            const int64_t step = 4 * g.ldc;
            const int rows_left = g.M - grow0;   // block row it is in range iff 4*it < rows_left
            const int cols_left = g.N - col0 - cq;
            const int mode = g.mode;
            uint32_t cv[CW];
            if (mode == MM_SUB) {
#pragma unroll
                for (int sl = 0; sl < CW / 8; ++sl)
#pragma unroll
                    for (int it = 0; it < 8; ++it)
                        cv[sl * 8 + it] = (sl * 8 < cols_left && 4 * it < rows_left)
                                              ? base[it * step + sl * 8]
                                              : 0u;
            }
#pragma unroll
            for (int sl = 0; sl < CW / 8; ++sl) {
#pragma unroll
                for (int j = 0; j < 8; ++j) stg[lane * 9 + j] = chunk_final<L>(res[sl * 8 + j], p);
                __syncwarp();
                if (sl * 8 < cols_left) {
#pragma unroll
                    for (int it = 0; it < 8; ++it)
                        if (4 * it < rows_left) {
                            const uint32_t v = stg[(it * 4 + rr) * 9 + cq];
                            uint32_t out;
                            if (mode == MM_SUB) out = sub_mod(cv[sl * 8 + it], v, p);
                            else if (mode == MM_ASSIGN) out = v;
                            else out = v == 0 ? 0u : p - v;
                            base[it * step + sl * 8] = out;
                        }
                }
                __syncwarp();
            }
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

int bn_for(int L)
{
    switch (L) {
        case 1: return Cfg<1>::BN;
        case 2: return Cfg<2>::BN;
        case 3: return Cfg<3>::BN;
        default: return Cfg<4>::BN;
    }
}

// SMs of the current device (one persistent CTA each)
int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        return 148;
    return n;
}

template <int L>
pluq_status run_tc(const MMSpec *spec, int count, int64_t K, Field F, Arena &ar, cudaStream_t st)
{
    using G = Geo<L>;
    const int64_t Kp = ceil_div(K, BK) * BK;
    SplitArgs sa{};
    TcArgs a{};
    int64_t rowsA = 0, rowsB = 0, zsplit = 0, ysplit = 1, ntiles = 0;
    double mm_work = 0, split_bytes = 0;
    for (int i = 0; i < count; ++i) {
        const MMSpec &q = spec[i];
        const int64_t Mp = ceil_div(q.M, BM) * BM, Np = ceil_div(q.N, G::BN) * G::BN;
        SplitProb &sp = sa.g[i];
        sp.A = q.A;
        sp.B = q.B;
        sp.lda = q.lda;
        sp.sA = q.sA;
        sp.ldb = q.ldb;
        sp.sB = q.sB;
        sp.M = (int)q.M;
        sp.N = (int)q.N;
        sp.batch = (int)q.batch;
        sp.Mp = Mp;
        sp.Np = Np;
        sp.rowA = rowsA;
        sp.rowB = rowsB;
        TcProb &tp = a.g[i];
        tp.C = q.C.ptr;
        tp.ldc = q.C.ld;
        tp.sC = q.sC;
        tp.M = (int)q.M;
        tp.N = (int)q.N;
        tp.Mp = (int)Mp;
        tp.Np = (int)Np;
        tp.ntm = (int)(Mp / BM);
        tp.ntn = (int)(Np / G::BN);
        const int64_t tiles = (int64_t)tp.ntm * tp.ntn * q.batch;
        if (tiles > INT32_MAX) return PLUQ_EINVAL;
        tp.tiles = (int)tiles;
        tp.rowA = (int)rowsA;
        tp.rowB = (int)rowsB;
        tp.mode = q.mode;
        rowsA += q.batch * L * Mp;
        rowsB += q.batch * L * Np;
        zsplit += q.batch;
        ysplit = std::max<int64_t>(ysplit, Mp / 32 + ceil_div(Np, 32));
        ntiles += tiles;
        mm_work += 2.0 * L * L * (double)q.M * q.N * K * q.batch;
        split_bytes += (double)q.batch * ((q.M + q.N) * K * 4.0 + (Mp + Np) * Kp * 2.0 * L);
    }
    if (rowsA > INT32_MAX || rowsB > INT32_MAX || ntiles > INT32_MAX || zsplit > 65535)
        return PLUQ_EINVAL;
    sa.ng = count;
    sa.K = (int)K;
    sa.Kp = Kp;
    sa.p = F.p;
    const size_t mark = ar.off;
    auto *pa = (__nv_bfloat16 *)ar.take((size_t)rowsA * Kp * 2, 1024);
    auto *pb = (__nv_bfloat16 *)ar.take((size_t)rowsB * Kp * 2, 1024);
    if (!pa || !pb) return PLUQ_ENOMEM;
    prof::start(prof::SPLIT, st);
    split_kernel<L><<<dim3((unsigned)(Kp / 32), (unsigned)std::min<int64_t>(ysplit, 65535),
                           (unsigned)zsplit),
                      dim3(32, 8), 0, st>>>(sa, pa, pb);
    PLUQ_TRY(last_launch());
    prof::stop(prof::SPLIT, st, split_bytes);

    CUtensorMap ma, mb;
    if (!make_map(&ma, pa, rowsA, Kp, BM)) return PLUQ_ECUDA;
    if (!make_map(&mb, pb, rowsB, Kp, G::BN)) return PLUQ_ECUDA;

    static std::atomic<uint64_t> attr{0};
    if (!smem_attr_once((const void *)mm_tc_kernel<L>, G::SMEM, attr)) return PLUQ_ECUDA;
    const uint32_t p = F.p;
    a.ng = count;
    a.wait_limit = wait_limit_or(WAIT_LIMIT);
    a.nkb = (int)(Kp / BK);
    a.ntiles = (int)ntiles;
    a.F = F;
    a.pf = (float)p;
    a.pinv = 1.0f / (float)p;
    a.off = ((uint64_t)(2 * L - 1) * (1ull << 24) + 1) * p;
    uint64_t w = 1;
    for (int s = 0; s < 7; ++s) {
        a.w[s] = (uint32_t)w;
        w = (w * 256) % p;
    }
    const int grid = (int)std::min<int64_t>(ntiles, sm_count());
    prof::start(prof::TC_MM, st);
    mm_tc_kernel<L><<<grid, NTHREADS, G::SMEM, st>>>(ma, mb, a);
    PLUQ_TRY(last_launch());
    // algorithmic tensor work: L^2 digit products of each M x K by K x N product
    prof::stop(prof::TC_MM, st, mm_work);
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

size_t mm_tc_group_workspace(const MMSpec *spec, int count, int64_t K, uint32_t p)
{
    size_t w = 0;
    for (int i = 0; i < count; ++i)
        w += mm_tc_workspace(spec[i].M, spec[i].N, K, p, spec[i].batch > 0 ? spec[i].batch : 1);
    return w;
}

pluq_status launch_mm_tc_group(const MMSpec *spec, int count, int64_t K, Field F, Arena &ar,
                               cudaStream_t st)
{
    // drop empty products; K = 0 leaves SUB alone and zeroes the assign forms
    MMSpec live[MAXG];
    int n = 0;
    if (count < 0 || count > MAXG) return PLUQ_EINVAL;
    for (int i = 0; i < count; ++i) {
        const MMSpec &q = spec[i];
        if (q.M <= 0 || q.N <= 0 || q.batch <= 0) continue;
        if (K == 0) {
            if (q.mode != MM_SUB)
                for (int64_t b = 0; b < q.batch; ++b)
                    PLUQ_TRY(launch_zero(Blk{q.C.ptr + b * q.sC, q.C.ld}, q.M, q.N, st));
            continue;
        }
        if (q.M > (1 << 30) || q.N > (1 << 30) || q.batch > 65535) return PLUQ_EINVAL;
        live[n++] = q;
    }
    if (n == 0) return PLUQ_OK;
    if (K > (1 << 30)) return PLUQ_EINVAL;
    switch (limbs_for_prime(F.p)) {
        case 1: return run_tc<1>(live, n, K, F, ar, st);
        case 2: return run_tc<2>(live, n, K, F, ar, st);
        case 3: return run_tc<3>(live, n, K, F, ar, st);
        case 4: return run_tc<4>(live, n, K, F, ar, st);
        default: return PLUQ_EUNSUPPORTED;
    }
}

pluq_status launch_mm_tc(Blk C, const uint32_t *A, int64_t lda, const uint32_t *B, int64_t ldb,
                         int64_t M, int64_t N, int64_t K, Field F, int mode, int64_t batch,
                         int64_t sA, int64_t sB, int64_t sC, Arena &ar, cudaStream_t st)
{
    MMSpec q{C, A, lda, B, ldb, M, N, mode, batch, sA, sB, sC};
    return launch_mm_tc_group(&q, 1, K, F, ar, st);
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
    if (p >= 0x80000000u || !is_prime_u32(p)) return PLUQ_ENOTPRIME;
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
