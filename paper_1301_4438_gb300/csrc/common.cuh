// Shared device/host helpers of libpluq: modular arithmetic over Z/pZ
// (p < 2^31), error plumbing, launch helpers.  Internal to the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <atomic>

#include "../../include/pluq.h"

namespace pluq {

// ----------------------------------------------------------------- field --
// Residues live in [0, p).  Products of two residues are < 2^62.
//
// Barrett reduction of x < 2^64 with mu = floor((2^64 - 1) / p): the quotient
// estimate q = hi64(x * mu) satisfies floor(x/p) - 1 <= q <= floor(x/p), so
// x - q p lies in [0, 2p) and one conditional subtraction finishes it.
//
// Montgomery form with R = 2^32 (odd p only): x is held as x R mod p, and
// mont_redc(T) = T R^{-1} mod p, in [0, 2p), for T < p R: with
// m = T pinv mod R (pinv = -1/p mod R), T + m p is divisible by R and below
// 2 p R, so one multiply-add and a shift replace Barrett's 64-bit high
// product.  r2 = R^2 mod p converts into the form.
struct Field {
    uint32_t p;
    uint64_t mu;
    uint32_t pinv, r2;
};

inline Field make_field(uint32_t p)
{
    Field f;
    f.p = p;
    f.mu = ~0ull / p;
    // Newton's iteration x <- x (2 - p x) doubles the bits of 1/p mod 2^32
    // that are right; x = p is right to 3 bits for odd p (p^2 = 1 mod 8)
    uint32_t x = p;
    for (int i = 0; i < 4; ++i) x *= 2u - p * x;
    f.pinv = (p & 1u) ? 0u - x : 0u;
    const uint64_t t = (1ull << 32) % p;
    f.r2 = (uint32_t)(t * t % p);
    return f;
}

// r mod p for r < 2p without a branch: when r < p, r - p wraps above r, so
// the unsigned minimum picks r; otherwise it picks r - p.  (Conditional
// subtractions written as ?: can turn into divergent branches, which
// serialise the independent reductions of a warp.)
__device__ __forceinline__ uint32_t fold(uint32_t r, uint32_t p) { return min(r, r - p); }

__device__ __forceinline__ uint32_t reduce64(uint64_t x, const Field &F)
{
    // q in {floor(x/p) - 1, floor(x/p)}, so x - q p < 2p < 2^32
    const uint64_t q = __umul64hi(x, F.mu);
    return fold((uint32_t)(x - q * (uint64_t)F.p), F.p);
}

__device__ __forceinline__ uint32_t mul_mod(uint32_t a, uint32_t b, const Field &F)
{
    return reduce64((uint64_t)a * b, F);
}

__device__ __forceinline__ uint32_t add_mod(uint32_t a, uint32_t b, uint32_t p)
{
    return fold(a + b, p);         // a + b < 2p < 2^32 since a, b < p < 2^31
}

__device__ __forceinline__ uint32_t sub_mod(uint32_t a, uint32_t b, uint32_t p)
{
    // a - b wraps above 2^32 - p when a < b; adding p then lands in [1, p)
    const uint32_t d = a - b;
    return min(d, d + p);
}

__device__ __forceinline__ uint32_t mont_redc(uint64_t T, const Field &F)
{
    const uint32_t m = (uint32_t)T * F.pinv;
    return (uint32_t)((T + (uint64_t)m * F.p) >> 32);
}

__device__ __forceinline__ uint32_t to_mont(uint32_t x, const Field &F)
{
    return fold(mont_redc((uint64_t)x * F.r2, F), F.p);
}

__device__ __forceinline__ uint32_t from_mont(uint32_t x, const Field &F)
{
    return fold(mont_redc(x, F), F.p);
}

// (a*b - c*d) mod p with one reduction: a*b + c*(p-d) < 2^63.
__device__ __forceinline__ uint32_t mul_sub_mul_mod(uint32_t a, uint32_t b, uint32_t c,
                                                    uint32_t d, const Field &F)
{
    uint64_t x = (uint64_t)a * b + (uint64_t)c * (d == 0 ? 0u : F.p - d);
    return reduce64(x, F);
}

// p <= 2^16: every product of two residues fits 32 bits.  Barrett with
// mu = floor((2^32 - 1) / p): q = hi32(x mu) > x/p - 2, so q >= floor(x/p) - 1
// and x - q p lies in [0, 2p).
struct Field32 {
    uint32_t p, mu;
};
inline Field32 make_field32(uint32_t p) { return Field32{p, 0xFFFFFFFFu / p}; }

__device__ __forceinline__ uint32_t reduce32(uint32_t x, const Field32 &F)
{
    return fold(x - __umulhi(x, F.mu) * F.p, F.p);
}

// Inverse of a nonzero residue by the extended Euclidean algorithm.
// a^e mod p by square and multiply (a^(p-2) is the inverse of a != 0, Fermat)
__device__ __forceinline__ uint32_t pow_mod(uint32_t a, uint32_t e, const Field &F)
{
    uint32_t x = 1;
    while (e) {
        if (e & 1u) x = mul_mod(x, a, F);
        a = mul_mod(a, a, F);
        e >>= 1;
    }
    return x;
}

__device__ __forceinline__ uint32_t inv_mod(uint32_t a, uint32_t p)
{
    uint32_t r0 = p, r1 = a;
    int64_t s0 = 0, s1 = 1;
    while (r1 != 0) {
        uint32_t q = r0 / r1;
        uint32_t t = r0 - q * r1;
        r0 = r1;
        r1 = t;
        int64_t u = s0 - (int64_t)q * s1;
        s0 = s1;
        s1 = u;
    }
    int64_t v = s0 % (int64_t)p;
    if (v < 0) v += p;
    return (uint32_t)v;
}

// --------------------------------------------------------------- limbs --
// Balanced base-256 digits of the centred representative c of x
// (c = x or x - p, |c| <= p/2): c = sum_l d_l 256^l with d_l in [-128, 127]
// for l < L-1 and |d_{L-1}| <= 128.  Every digit is an integer of magnitude
// <= 128, exact in bf16, and a digit product is at most 2^14 in magnitude.
// Primality of a 32-bit integer on the host: Miller-Rabin with the bases
// 2, 7 and 61, which decides every n < 4,759,123,141 exactly (Jaeschke 1993).
inline bool is_prime_u32(uint32_t n)
{
    if (n < 2) return false;
    for (uint32_t q : {2u, 3u, 5u, 7u, 11u, 13u, 61u}) {
        if (n == q) return true;
        if (n % q == 0) return false;
    }
    uint32_t d = n - 1;
    int s = 0;
    while ((d & 1u) == 0) {
        d >>= 1;
        ++s;
    }
    for (uint64_t a : {2ull, 7ull, 61ull}) {
        uint64_t x = 1, b = a % n;
        for (uint32_t e = d; e; e >>= 1) {       // x = a^d mod n
            if (e & 1u) x = x * b % n;
            b = b * b % n;
        }
        if (x == 1 || x == n - 1) continue;
        bool composite = true;
        for (int i = 1; i < s && composite; ++i) {
            x = x * x % n;
            if (x == n - 1) composite = false;
        }
        if (composite) return false;
    }
    return true;
}

inline int limbs_for_prime(uint32_t p)
{
    // smallest L with (p-1)/2 <= 128 (256^L - 1) / 255
    uint64_t half = (uint64_t)(p - 1) / 2;
    uint64_t cap = 128;      // 128 (256^1 - 1)/255
    int L = 1;
    while (half > cap) {
        cap = cap * 256 + 128;
        ++L;
    }
    return L;
}

// ---------------------------------------------------------------- misc --
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Arena {
    char *base = nullptr;
    size_t size = 0, off = 0;
    void *take(size_t bytes, size_t align = 256)
    {
        size_t o = align_up(off, align);
        if (o + bytes > size) return nullptr;
        off = o + bytes;
        return base + o;
    }
};

#define PLUQ_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return PLUQ_ECUDA;             \
    } while (0)

#define PLUQ_TRY(expr)                                        \
    do {                                                      \
        pluq_status _s = (expr);                              \
        if (_s != PLUQ_OK) return _s;                         \
    } while (0)

// ------------------------------------------------------------ profiling --
// Kernel classes timed by the optional profiler (see pluq_profile_read).
namespace prof {
enum Cls { TC_MM = 0, SIMT_MM = 1, LEAF = 2, MOVE = 3, SPLIT = 4, TRI = 5, NCLS = 6 };
extern std::atomic<long long> g_launches;
void start(int cls, cudaStream_t st);
void stop(int cls, cudaStream_t st, double work);
}  // namespace prof

// Dynamic shared memory above 48 KB must be opted into per kernel with
// cudaFuncSetAttribute, which acts on the current device only: do it once per
// device (bit `dev` of the caller's mask; devices past 63 every time).
inline bool smem_attr_once(const void *kernel, size_t bytes, std::atomic<uint64_t> &done)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const uint64_t bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return true;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return false;
    if (bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return true;
}

// Every kernel launch goes through here: error check and launch count.
inline pluq_status last_launch()
{
    prof::g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError() == cudaSuccess ? PLUQ_OK : PLUQ_ECUDA;
}

// --------------------------------------------------- internal launchers --
// Strided block descriptor: element (i, j) at ptr[i*ld + j].
struct Blk {
    uint32_t *ptr;
    int64_t ld;
};

enum MMMode { MM_SUB = 0, MM_ASSIGN = 1, MM_NEG_ASSIGN = 2 };

// Modular product on a batch of equally shaped problems:
//   C_b <- C_b - A_b B_b | A_b B_b | -A_b B_b (mode), b < batch, with
//   X_b = X + b * stride_X.  SIMT form.
pluq_status launch_mm_simt(Blk C, const uint32_t *A, int64_t lda, const uint32_t *B,
                           int64_t ldb, int64_t M, int64_t N, int64_t K, Field F, int mode,
                           int64_t batch, int64_t sA, int64_t sB, int64_t sC,
                           cudaStream_t st);

// Tensor-core form; scratch for limb planes comes from the arena.
pluq_status launch_mm_tc(Blk C, const uint32_t *A, int64_t lda, const uint32_t *B,
                         int64_t ldb, int64_t M, int64_t N, int64_t K, Field F, int mode,
                         int64_t batch, int64_t sA, int64_t sB, int64_t sC, Arena &ar,
                         cudaStream_t st);
size_t mm_tc_workspace(int64_t M, int64_t N, int64_t K, uint32_t p, int64_t batch);

// Independent products that share K, one split launch and one persistent
// tensor-core launch for all of them (at most two per group).
struct MMSpec {
    Blk C;
    const uint32_t *A;
    int64_t lda;
    const uint32_t *B;
    int64_t ldb;
    int64_t M, N;
    int mode;
    int64_t batch, sA, sB, sC;
};
pluq_status launch_mm_tc_group(const MMSpec *spec, int count, int64_t K, Field F, Arena &ar,
                               cudaStream_t st);
size_t mm_tc_group_workspace(const MMSpec *spec, int count, int64_t K, uint32_t p);
// Nonzero if a tensor-core kernel gave up on a bounded wait since the last
// call (reads and clears the device word); likewise for the leaf's step waits.
int tc_error_flag();
int leaf_error_flag();        // either kind of base-case kernel gave up a wait
int node_leaf_error_flag();   // the node kernel's base cases (part of leaf_error_flag)
int batch_leaf_error_flag();  // the persistent batch kernel's base cases (likewise)

// Tries of every abortable device-side wait (pluq_set_wait_limit): negative
// keeps each kernel's built-in bound.  The waits a kernel runs while winding
// down after giving up keep their full bound.
extern std::atomic<int64_t> g_wait_limit;
inline uint32_t wait_limit_or(uint32_t builtin)
{
    const int64_t v = g_wait_limit.load(std::memory_order_relaxed);
    return v < 0 ? builtin : (uint32_t)(v > 0xFFFFFFFFll ? 0xFFFFFFFFll : v);
}

// Dispatch on the kind (SIMT needs C disjoint from A and B).
pluq_status launch_mm(int kind, Blk C, const uint32_t *A, int64_t lda, const uint32_t *B,
                      int64_t ldb, int64_t M, int64_t N, int64_t K, Field F, int mode,
                      int64_t batch, int64_t sA, int64_t sB, int64_t sC, Arena &ar,
                      cudaStream_t st);

// In-place PermR / PermC of Sec. 2 on a block: rows (by_rows) or columns of
// the rows x cols block at X are replaced by rows / columns map[.] - moff of
// it.  launch_perm_ops applies up to four such ops on disjoint blocks in one
// launch (each element read and written once); an op whose staging does not
// fit a thread block's shared memory goes through `scratch` instead (gather,
// then copy back).
struct PermOp {
    uint32_t *X;
    int64_t ld;
    int64_t rows, cols;
    const int32_t *map;
    int32_t moff;
    bool by_rows;
};
pluq_status launch_perm_ops(const PermOp *ops, int count, uint32_t *scratch, size_t scratch_elems,
                            cudaStream_t st);

// Row/column gathers: dst[i][j] = src[rmap(i)][cmap(j)], maps optional.
pluq_status launch_gather(Blk dst, const uint32_t *src, int64_t lds, int64_t rows,
                          int64_t cols, const int32_t *rmap, const int32_t *cmap,
                          cudaStream_t st);
pluq_status launch_copy(Blk dst, const uint32_t *src, int64_t lds, int64_t rows,
                        int64_t cols, cudaStream_t st);
pluq_status launch_zero(Blk dst, int64_t rows, int64_t cols, cudaStream_t st);

// Triangular inverses into X (r x r, ld ldx), and the TRSMs built on them.
pluq_status tri_inv_lower_unit(const uint32_t *L, int64_t ldl, Blk X, int64_t r, Field F,
                               int kind, Arena &ar, cudaStream_t st);
pluq_status tri_inv_upper(const uint32_t *U, int64_t ldu, Blk X, int64_t r, Field F,
                          int kind, Arena &ar, cudaStream_t st);
pluq_status trsm_left_lower_unit(const uint32_t *L, int64_t ldl, Blk B, int64_t r, int64_t N,
                                 Field F, int kind, Arena &ar, cudaStream_t st);
pluq_status trsm_right_upper(const uint32_t *U, int64_t ldu, Blk B, int64_t M, int64_t r,
                             Field F, int kind, Arena &ar, cudaStream_t st);
size_t trsm_workspace(int64_t r, int64_t other, uint32_t p, int kind);
// Both solves of a node at once when both triangles are small (trsm_small_for):
// BL (rl x N) <- L^{-1} BL and BR (M x rr) <- BR U^{-1}, one launch.
bool trsm_small_for(int64_t r);
pluq_status trsm_pair_small(const uint32_t *L, int64_t ldl, Blk BL, int64_t rl, int64_t N,
                            const uint32_t *U, int64_t ldu, Blk BR, int64_t M, int64_t rr,
                            Field F, cudaStream_t st);
// true when a triangle of r rows is solved directly (no workspace used)
bool trsm_direct_for(int64_t r);

pluq_status launch_iota(int32_t *v, int64_t n, cudaStream_t st);
// out_key = key[0..r) sorted (distinct keys), out_val = val in the same order
pluq_status launch_rank_sort(const int32_t *key, const int32_t *val, int64_t r, int32_t *out_key,
                             int32_t *out_val, cudaStream_t st);
pluq_status launch_extract(const uint32_t *LU, int64_t lda, int64_t rows, int64_t cols,
                           uint32_t *X, int64_t ldx, bool lower, cudaStream_t st);
pluq_status launch_leu(const uint32_t *LU, int64_t lda, int64_t m, int64_t n, int64_t r,
                       const int32_t *perm_p, const int32_t *perm_q, uint32_t *Lbar, int64_t ldl,
                       uint32_t *Ubar, int64_t ldu, int32_t *work, cudaStream_t st);
pluq_status launch_leading_profile(const int32_t *pp, const int32_t *pq, int64_t r, int64_t k,
                                   int64_t t, int32_t *rows, int32_t *cols, int32_t *count,
                                   cudaStream_t st);

// Leaf (base case) of the recursion.
constexpr int LEAF_MAX = 128;
// info[0] = r, info[1] = (P is the identity), info[2] = (Q is the identity);
// when host_info is given (mapped pinned memory) the same three words go to
// host_info[1..3] and then seq to host_info[0].  try_generic: attempt the
// blocked path for a generic rank profile first (worth it unless the block
// lies in a rank-deficient region, where it would fail at once).
pluq_status launch_leaf(uint32_t *A, int64_t m, int64_t n, int64_t lda, Field F,
                        int32_t *perm_p, int32_t *perm_q, int32_t *info, int info_len,
                        cudaStream_t st, volatile int32_t *host_info = nullptr, int32_t seq = 0,
                        bool try_generic = true);

// Algorithm 1 on a node of at most 4 LEAF_MAX x 4 LEAF_MAX in one thread
// block: its blocks are base cases, or (above 2 LEAF_MAX) nodes whose blocks
// are; same outputs and host words as launch_leaf.  stage holds stage_words
// >= m * n words, icopy ceil(m/2) * ceil(n/2).
pluq_status launch_node(uint32_t *A, int64_t m, int64_t n, int64_t lda, Field F, int32_t *perm_p,
                        int32_t *perm_q, int32_t *info, cudaStream_t st, volatile int32_t *host_info,
                        int32_t seq, bool try_generic, uint32_t *stage, int64_t stage_words,
                        uint32_t *icopy);

// Process-wide tuning (pluq_set_tuning): leaf size of the recursion, and the
// number of multiply-adds below which a product goes to the CUDA-core kernel
// when C does not overlap A or B (launch latency dominates there).
extern std::atomic<int64_t> g_tune_leaf;
extern std::atomic<int64_t> g_tune_small_mm;
// base case: right-looking (false) or left-looking (true) blocked elimination
extern std::atomic<bool> g_tune_leaf_left;
// nodes below rank-deficient ones of at most 2 levels x 2 x leaf on a side go
// to the node kernel (0: none)
extern std::atomic<int> g_tune_node;
extern std::atomic<int> g_tune_node_ctas;   // thread blocks of a node kernel (1 or 2)

}  // namespace pluq
