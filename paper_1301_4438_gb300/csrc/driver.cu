// Algorithm 1 (Sec. 2) driven from the host, every step a kernel on the
// caller's stream, and the C-ABI entry points of include/pluq.h.
//
// The ranks r1..r4 of the four recursive calls decide the shapes of the next
// steps, so the host reads each leaf's rank back (pinned host word) before it
// continues; everything else is queued asynchronously.  Blocks are addressed
// in place inside the caller's matrix (pointer + row stride); permutations of
// a block go through a scratch copy.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <thread>
#include <vector>
#include <stdlib.h>
#include <string.h>

#include "common.cuh"

namespace pluq {

pluq_status launch_iota(int32_t *v, int64_t n, cudaStream_t st);
pluq_status launch_compose(const int32_t *p1, const int32_t *p2, const int32_t *p3,
                           const int32_t *p4, const int32_t *q1, const int32_t *q2,
                           const int32_t *q3, const int32_t *q4, int32_t *p, int32_t *q,
                           int32_t *smap, int32_t *tmap, int64_t m, int64_t n, int64_t k,
                           int64_t h, int64_t r1, int64_t r2, int64_t r3, int64_t r4,
                           cudaStream_t st);
pluq_status launch_rank_sort(const int32_t *key, const int32_t *val, int64_t r, int32_t *out_key,
                             int32_t *out_val, cudaStream_t st);
pluq_status launch_check_range(const uint32_t *A, int64_t lda, int64_t m, int64_t n, uint32_t p,
                               int32_t *flag, cudaStream_t st);
pluq_status launch_any_nonzero(const uint32_t *A, int64_t lda, int64_t m, int64_t n, int32_t *words,
                               volatile int32_t *host, int32_t seq, cudaStream_t st);

std::atomic<int64_t> g_tune_small_mm{1ll << 25};
std::atomic<int64_t> g_tune_leaf{128};

namespace {
// byte ranges [lo, hi) spanned by a batch of strided blocks
struct Span {
    uintptr_t lo, hi;
};
Span span(const uint32_t *X, int64_t ld, int64_t rows, int64_t cols, int64_t batch, int64_t stride)
{
    uintptr_t lo = (uintptr_t)X;
    uintptr_t hi = lo + (uintptr_t)(((batch - 1) * stride + (rows - 1) * ld + cols) * 4);
    return Span{lo, hi};
}
bool overlap(Span a, Span b) { return a.lo < b.hi && b.lo < a.hi; }
}  // namespace

pluq_status launch_mm(int kind, Blk C, const uint32_t *A, int64_t lda, const uint32_t *B,
                      int64_t ldb, int64_t M, int64_t N, int64_t K, Field F, int mode,
                      int64_t batch, int64_t sA, int64_t sB, int64_t sC, Arena &ar,
                      cudaStream_t st)
{
    if (M <= 0 || N <= 0 || batch <= 0) return PLUQ_OK;
    if (kind == PLUQ_MM_SIMT)
        return launch_mm_simt(C, A, lda, B, ldb, M, N, K, F, mode, batch, sA, sB, sC, st);
    // small products: one CUDA-core launch beats split + split + tensor launch,
    // as long as C is disjoint from the operands it would overwrite
    if (K > 0 && (double)M * N * K * batch <= (double)g_tune_small_mm.load(std::memory_order_relaxed)) {
        Span sc = span(C.ptr, C.ld, M, N, batch, sC);
        if (!overlap(sc, span(A, lda, M, K, batch, sA)) && !overlap(sc, span(B, ldb, K, N, batch, sB)))
            return launch_mm_simt(C, A, lda, B, ldb, M, N, K, F, mode, batch, sA, sB, sC, st);
    }
    return launch_mm_tc(C, A, lda, B, ldb, M, N, K, F, mode, batch, sA, sB, sC, ar, st);
}

namespace {


// Mapped pinned host words: a kernel writes its result words and then a
// sequence number there, and the host polls the sequence number instead of
// copying and synchronising.  Slots come from a process-wide pool so that
// concurrent callers (and the batch workers) each own one while they run.
struct HostWords {
    volatile int32_t *h = nullptr;   // host view (64 words)
    int32_t *d = nullptr;            // device view
    int32_t seq = 0;
};
std::mutex g_words_mu;
std::vector<HostWords *> g_words_free;

HostWords *acquire_words()
{
    std::lock_guard<std::mutex> lk(g_words_mu);
    if (g_words_free.empty()) {
        constexpr int SLOTS = 16, BYTES = 256;
        int32_t *h = nullptr;
        if (cudaHostAlloc((void **)&h, SLOTS * BYTES, cudaHostAllocMapped | cudaHostAllocPortable) !=
            cudaSuccess)
            return nullptr;
        int32_t *d = nullptr;
        if (cudaHostGetDevicePointer((void **)&d, h, 0) != cudaSuccess) return nullptr;
        for (int i = 0; i < SLOTS * BYTES / 4; ++i) h[i] = 0;
        for (int sl = 0; sl < SLOTS; ++sl) {
            HostWords *w = new (std::nothrow) HostWords;
            if (!w) return nullptr;
            w->h = h + sl * (BYTES / 4);
            w->d = d + sl * (BYTES / 4);
            g_words_free.push_back(w);
        }
    }
    HostWords *w = g_words_free.back();
    g_words_free.pop_back();
    return w;
}

void release_words(HostWords *w)
{
    if (!w) return;
    std::lock_guard<std::mutex> lk(g_words_mu);
    g_words_free.push_back(w);
}

// wait for a kernel to publish sequence number `seq` in host word `at`; the
// stream is queried now and then so that a failed launch cannot hang the host
pluq_status wait_words(HostWords *hw, int32_t seq, cudaStream_t st, int at = 0)
{
    for (long long it = 0;; ++it) {
        if (hw->h[at] == seq) return PLUQ_OK;
        if ((it & 0xFFFF) == 0xFFFF) {
            cudaError_t e = cudaStreamQuery(st);
            if (e == cudaSuccess) return hw->h[at] == seq ? PLUQ_OK : PLUQ_EINTERNAL;
            if (e != cudaErrorNotReady) return PLUQ_ECUDA;
        }
    }
}

// Host words 8 + 2d (sequence number) and 9 + 2d (flag) carry the zero test of
// the node at recursion depth d < ZDEPTH; word 0..3 belong to the leaf.
constexpr int ZBASE = 8, ZDEPTH = 27;

struct Ctx {
    Field F{};
    int kind = 0;
    cudaStream_t st = nullptr;
    Arena ar;                       // scratch for products / TRSM (stack discipline)
    uint32_t *gather = nullptr;     // m*n scratch for permutations
    uint32_t *icopy = nullptr;      // copy of I (r3 x r2)
    int32_t *smap = nullptr, *tmap = nullptr;   // S and T index maps of the current node
    int32_t *vstack = nullptr;      // child permutation vectors (stack discipline)
    size_t vtop = 0, vcap = 0;
    int32_t *d_rank = nullptr;      // device words: range check flag, leaf info
    HostWords *hw = nullptr;
    int64_t leaf = 128;   // blocks with both sides <= leaf go to the leaf kernel
    cudaStream_t side = nullptr;            // second stream for independent work of a node
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_done = nullptr;          // end of this context's work (branch contexts)
    struct BranchPool *pool = nullptr;      // contexts free to run PLUQ(G) on another thread
    int64_t leaves = 0;
    int64_t zero_checks = 0;
};

// Contexts that can each run one recursive call on a host thread of its own,
// with their own streams, host words and scratch (sized for a quarter of the
// matrix: the block G of any node fits).
struct BranchPool {
    std::mutex mu;
    std::vector<Ctx *> free;
    Ctx *take()
    {
        std::lock_guard<std::mutex> lk(mu);
        if (free.empty()) return nullptr;
        Ctx *c = free.back();
        free.pop_back();
        return c;
    }
    void give(Ctx *c)
    {
        std::lock_guard<std::mutex> lk(mu);
        free.push_back(c);
    }
};
constexpr int NBRANCH = 3;            // branch contexts per decomposition
constexpr int64_t BRANCH_MIN = 256;   // both F and G at least this large in each dimension
constexpr int64_t BRANCH_MATRIX_MIN = 1024;   // matrices below this get no branch contexts

// Leaf size of the recursion (pluq_set_tuning; PLUQ_LEAF in the environment
// sets the initial value).  Smaller leaves mean less one-SM elimination work
// per leaf (b^3/3 per leaf, n b^2/3 in all for an n x n full-rank matrix) but
// more recursion nodes.
int64_t leaf_size() { return g_tune_leaf.load(std::memory_order_relaxed); }

int64_t initial_leaf()
{
    const char *e = getenv("PLUQ_LEAF");
    if (e) {
        long v = strtol(e, nullptr, 10);
        if (v >= 16 && v <= LEAF_MAX) return v;
    }
    return 128;
}

// result of a (sub)decomposition: rank, and whether P / Q are identities
// (then their vectors are not needed by the parent and may be left unwritten)
struct Res {
    int64_t r = 0;
    bool pid = true, qid = true;
};

int32_t *vtake(Ctx &c, int64_t len)
{
    size_t need = (size_t)(len > 0 ? len : 1);
    need = align_up(need, 64);
    if (c.vtop + need > c.vcap) return nullptr;
    int32_t *v = c.vstack + c.vtop;
    c.vtop += need;
    return v;
}

// rows [0, rows) x cols [0, cols) of the block X <- gathered with maps (in place
// through the scratch copy)
pluq_status permute_block(Ctx &c, uint32_t *X, int64_t ldx, int64_t rows, int64_t cols,
                          const int32_t *rmap, const int32_t *cmap)
{
    if (rows <= 0 || cols <= 0 || (!rmap && !cmap)) return PLUQ_OK;
    PLUQ_TRY(launch_gather(Blk{c.gather, cols}, X, ldx, rows, cols, rmap, cmap, c.st));
    return launch_copy(Blk{X, ldx}, c.gather, cols, rows, cols, c.st);
}

// True when the (start, length) segments, taken in turn, walk 0, 1, 2, ...:
// the block permutation S or T is then the identity.
bool in_order(const int64_t (*seg)[2], int count)
{
    int64_t pos = 0;
    for (int i = 0; i < count; ++i) {
        if (seg[i][1] <= 0) continue;
        if (seg[i][0] != pos) return false;
        pos += seg[i][1];
    }
    return true;
}

// Algorithm 1 on the m x n block at A.  On return the block holds its packed
// factorisation; pp / pq hold P / Q unless out.pid / out.qid say they are the
// identity (then the vectors are not written).
pluq_status rec(Ctx &c, uint32_t *A, int64_t m, int64_t n, int64_t lda, int32_t *pp,
                int32_t *pq, Res &out, int depth, bool eager)
{
    out = Res{};
    if (m == 0 || n == 0) return PLUQ_OK;
    if (m <= c.leaf && n <= c.leaf) {
        const int32_t seq = ++c.hw->seq;
        PLUQ_TRY(launch_leaf(A, m, n, lda, c.F, pp, pq, c.d_rank + 4, 3, c.st, c.hw->d, seq,
                             !eager));
        PLUQ_TRY(wait_words(c.hw, seq, c.st));
        const int32_t r = c.hw->h[1];
        ++c.leaves;
        if (r < 0 || r > m || r > n) return PLUQ_EINTERNAL;
        out.r = r;
        out.pid = c.hw->h[2] != 0;
        out.qid = c.hw->h[3] != 0;
        return PLUQ_OK;
    }
    // A block's rank is the number of ones of R inside it, so deep in the
    // recursion of a rank-deficient matrix most blocks are exactly zero: one
    // pass over the block prunes the whole subtree (r = 0, P = Q = I).  Below a
    // node whose A1 turned out rank deficient the answer is awaited at once;
    // elsewhere (full-rank regions, where blocks are rarely zero) it is read
    // lazily: the descent into A1 goes ahead meanwhile and its first leaf (a
    // synchronisation anyway) brings the answer along.  If the block is zero,
    // so is A1, whose decomposition then changed nothing and reported r1 = 0
    // with identity permutations.
    const bool lazy = !eager && depth < ZDEPTH;
    const int32_t zseq = ++c.hw->seq;
    const int zat = ZBASE + 2 * depth;
    ++c.zero_checks;
    if (lazy) {
        PLUQ_TRY(launch_any_nonzero(A, lda, m, n, c.d_rank + 8, c.hw->d + zat, zseq, c.st));
    } else {
        PLUQ_TRY(launch_any_nonzero(A, lda, m, n, c.d_rank + 8, c.hw->d, zseq, c.st));
        PLUQ_TRY(wait_words(c.hw, zseq, c.st));
        if (c.hw->h[1] == 0) return PLUQ_OK;
    }
    const int64_t k = m / 2, h = n / 2;
    const size_t vmark = c.vtop;
    int32_t *p1 = vtake(c, k), *q1 = vtake(c, h), *p2 = vtake(c, k), *q2 = vtake(c, n - h);
    int32_t *p3 = vtake(c, m - k), *q3 = vtake(c, h), *p4 = vtake(c, m - k), *q4 = vtake(c, n - h);
    if (!q4) return PLUQ_ENOMEM;
    const Field F = c.F;
    auto at = [&](int64_t i, int64_t j) { return A + i * lda + j; };
    auto vec = [](int32_t *v, bool ident) -> int32_t * { return ident ? nullptr : v; };

    // A1 = P1 [L1;M1][U1 V1] Q1
    Res s1;
    PLUQ_TRY(rec(c, A, k, h, lda, p1, q1, s1, depth + 1, eager));
    if (lazy) {
        PLUQ_TRY(wait_words(c.hw, zseq, c.st, zat));
        if (c.hw->h[zat + 1] == 0) {
            if (s1.r != 0 || !s1.pid || !s1.qid) return PLUQ_EINTERNAL;
            c.vtop = vmark;
            return PLUQ_OK;
        }
    }
    const int64_t r1 = s1.r;
    const bool deficient = r1 < (k < h ? k : h);
    // [B1;B2] <- P1^T A2 ; [C1 C2] <- A3 Q1^T
    PLUQ_TRY(permute_block(c, at(0, h), lda, k, n - h, vec(p1, s1.pid), nullptr));
    PLUQ_TRY(permute_block(c, at(k, 0), lda, m - k, h, nullptr, vec(q1, s1.qid)));
    // D <- L1^{-1} B1 ; E <- C1 U1^{-1}, then [F;H] <- [B2;A4] - [M1;E] D and
    // G <- C2 - E V1: each pair is independent (disjoint outputs, shared
    // read-only operands).  The second of a pair runs on the side stream when
    // the arena has room for both scratch areas side by side.
    {
        const uint32_t p = F.p;
        const size_t needL = trsm_direct_for(r1) ? 0 : trsm_workspace(r1, n - h, p, c.kind);
        const size_t needR = trsm_direct_for(r1) ? 0 : trsm_workspace(r1, m - k, p, c.kind);
        Arena a2 = c.ar;
        a2.off = align_up(c.ar.off + needL, 1024);
        const bool both = r1 > 0 && n - h > 0 && m - k > 0;
        if (c.side && both && a2.off + needR <= c.ar.size) {
            PLUQ_CUDA_TRY(cudaEventRecord(c.ev_fork, c.st));
            PLUQ_CUDA_TRY(cudaStreamWaitEvent(c.side, c.ev_fork, 0));
            PLUQ_TRY(trsm_left_lower_unit(A, lda, Blk{at(0, h), lda}, r1, n - h, F, c.kind, c.ar, c.st));
            PLUQ_TRY(trsm_right_upper(A, lda, Blk{at(k, 0), lda}, m - k, r1, F, c.kind, a2, c.side));
            PLUQ_CUDA_TRY(cudaEventRecord(c.ev_join, c.side));
            PLUQ_CUDA_TRY(cudaStreamWaitEvent(c.st, c.ev_join, 0));
        } else {
            PLUQ_TRY(trsm_left_lower_unit(A, lda, Blk{at(0, h), lda}, r1, n - h, F, c.kind, c.ar, c.st));
            PLUQ_TRY(trsm_right_upper(A, lda, Blk{at(k, 0), lda}, m - k, r1, F, c.kind, c.ar, c.st));
        }
    }
    {
        const uint32_t p = F.p;
        const bool tc = c.kind != PLUQ_MM_SIMT;
        const size_t need1 = tc ? mm_tc_workspace(m - r1, n - h, r1, p, 1) : 0;
        const size_t need2 = tc ? mm_tc_workspace(m - k, h - r1, r1, p, 1) : 0;
        Arena a2 = c.ar;
        a2.off = align_up(c.ar.off + need1, 1024);
        const bool both = r1 > 0 && m - r1 > 0 && n - h > 0 && m - k > 0 && h - r1 > 0;
        cudaStream_t s2 = c.st;
        if (c.side && both && a2.off + need2 <= c.ar.size) {
            PLUQ_CUDA_TRY(cudaEventRecord(c.ev_fork, c.st));
            PLUQ_CUDA_TRY(cudaStreamWaitEvent(c.side, c.ev_fork, 0));
            s2 = c.side;
        } else {
            a2 = c.ar;
        }
        PLUQ_TRY(launch_mm(c.kind, Blk{at(r1, h), lda}, at(r1, 0), lda, at(0, h), lda, m - r1,
                           n - h, r1, F, MM_SUB, 1, 0, 0, 0, c.ar, c.st));
        PLUQ_TRY(launch_mm(c.kind, Blk{at(k, r1), lda}, at(k, 0), lda, at(0, r1), lda, m - k,
                           h - r1, r1, F, MM_SUB, 1, 0, 0, 0, a2, s2));
        if (s2 != c.st) {
            PLUQ_CUDA_TRY(cudaEventRecord(c.ev_join, c.side));
            PLUQ_CUDA_TRY(cudaStreamWaitEvent(c.st, c.ev_join, 0));
        }
    }
    // F = P2 [L2;M2][U2 V2] Q2 ; G = P3 [L3;M3][U3 V3] Q3
    // PLUQ(F) and PLUQ(G) work on disjoint blocks with their own permutation
    // vectors: with a free branch context, G runs on another host thread and
    // stream while this thread does F (the concurrency noted in Sec. 8)
    Res s2, s3;
    Ctx *bc = nullptr;
    if (c.pool && k - r1 >= BRANCH_MIN && n - h >= BRANCH_MIN && m - k >= BRANCH_MIN &&
        h - r1 >= BRANCH_MIN)
        bc = c.pool->take();
    if (bc) {
        pluq_status sg = PLUQ_OK, sf = PLUQ_OK;
        if (cudaEventRecord(c.ev_fork, c.st) != cudaSuccess ||
            cudaStreamWaitEvent(bc->st, c.ev_fork, 0) != cudaSuccess) {
            c.pool->give(bc);
            return PLUQ_ECUDA;
        }
        std::thread th;
        bool spawned = true;
        try {
            th = std::thread([&] {
                sg = rec(*bc, at(k, r1), m - k, h - r1, lda, p3, q3, s3, depth + 1, deficient);
            });
        } catch (...) {
            spawned = false;    // no thread to be had: G on this thread, on bc's stream
        }
        sf = rec(c, at(r1, h), k - r1, n - h, lda, p2, q2, s2, depth + 1, deficient);
        if (spawned) th.join();
        else sg = rec(*bc, at(k, r1), m - k, h - r1, lda, p3, q3, s3, depth + 1, deficient);
        const bool ok = cudaEventRecord(bc->ev_done, bc->st) == cudaSuccess &&
                        cudaStreamWaitEvent(c.st, bc->ev_done, 0) == cudaSuccess;
        c.pool->give(bc);
        PLUQ_TRY(sf);
        PLUQ_TRY(sg);
        if (!ok) return PLUQ_ECUDA;
    } else {
        PLUQ_TRY(rec(c, at(r1, h), k - r1, n - h, lda, p2, q2, s2, depth + 1, deficient));
        PLUQ_TRY(rec(c, at(k, r1), m - k, h - r1, lda, p3, q3, s3, depth + 1, deficient));
    }
    const int64_t r2 = s2.r, r3 = s3.r;
    int32_t *P2 = vec(p2, s2.pid), *Q2 = vec(q2, s2.qid), *P3 = vec(p3, s3.pid), *Q3 = vec(q3, s3.qid);
    // H <- P3^T H Q2^T ; E <- P3^T E ; M1 <- P2^T M1 ; D <- D Q2^T ; V1 <- V1 Q3^T
    PLUQ_TRY(permute_block(c, at(k, h), lda, m - k, n - h, P3, Q2));
    PLUQ_TRY(permute_block(c, at(k, 0), lda, m - k, r1, P3, nullptr));
    PLUQ_TRY(permute_block(c, at(r1, 0), lda, k - r1, r1, P2, nullptr));
    PLUQ_TRY(permute_block(c, at(0, h), lda, r1, n - h, nullptr, Q2));
    PLUQ_TRY(permute_block(c, at(0, r1), lda, r1, h - r1, nullptr, Q3));
    // [I;K] <- [H1;H3] U2^{-1}
    const uint32_t *U2 = at(r1, h);
    PLUQ_TRY(trsm_right_upper(U2, lda, Blk{at(k, h), lda}, m - k, r2, F, c.kind, c.ar, c.st));
    // keep I; [J N] <- L3^{-1} [I H2]
    if (r3 > 0 && r2 > 0) PLUQ_TRY(launch_copy(Blk{c.icopy, r2}, at(k, h), lda, r3, r2, c.st));
    const uint32_t *L3 = at(k, r1);
    PLUQ_TRY(trsm_left_lower_unit(L3, lda, Blk{at(k, h), lda}, r3, n - h, F, c.kind, c.ar, c.st));
    // O <- N - J V2
    PLUQ_TRY(launch_mm(c.kind, Blk{at(k, h + r2), lda}, at(k, h), lda, at(r1, h + r2), lda, r3,
                       n - h - r2, r2, F, MM_SUB, 1, 0, 0, 0, c.ar, c.st));
    if (r3 > 0 && r2 > 0) PLUQ_TRY(launch_copy(Blk{at(k, h), lda}, c.icopy, r2, r3, r2, c.st));
    // R <- H4 - K V2 - M3 O
    PLUQ_TRY(launch_mm(c.kind, Blk{at(k + r3, h + r2), lda}, at(k + r3, h), lda, at(r1, h + r2),
                       lda, m - k - r3, n - h - r2, r2, F, MM_SUB, 1, 0, 0, 0, c.ar, c.st));
    PLUQ_TRY(launch_mm(c.kind, Blk{at(k + r3, h + r2), lda}, at(k + r3, r1), lda, at(k, h + r2),
                       lda, m - k - r3, n - h - r2, r3, F, MM_SUB, 1, 0, 0, 0, c.ar, c.st));
    // R = P4 [L4;M4][U4 V4] Q4
    Res s4;
    PLUQ_TRY(rec(c, at(k + r3, h + r2), m - k - r3, n - h - r2, lda, p4, q4, s4, depth + 1,
                 deficient));
    const int64_t r4 = s4.r;
    int32_t *P4 = vec(p4, s4.pid), *Q4 = vec(q4, s4.qid);
    // [E2 M3 0 K] <- P4^T [..] ; [D2;V2;0;O] <- [..] Q4^T
    PLUQ_TRY(permute_block(c, at(k + r3, 0), lda, m - k - r3, h + r2, P4, nullptr));
    PLUQ_TRY(permute_block(c, at(0, h + r2), lda, k + r3, n - h - r2, nullptr, Q4));
    // P, Q and the block permutations S, T ; A <- S^T A T^T
    const int64_t sseg[4][2] = {{0, r1 + r2}, {k, r3 + r4}, {r1 + r2, k - r1 - r2},
                                {k + r3 + r4, m - k - r3 - r4}};
    const int64_t tseg[6][2] = {{0, r1}, {h, r2}, {r1, r3}, {h + r2, r4}, {r1 + r3, h - r1 - r3},
                                {h + r2 + r4, n - h - r2 - r4}};
    const bool s_ident = in_order(sseg, 4), t_is_id = in_order(tseg, 6);
    out.r = r1 + r2 + r3 + r4;
    out.pid = s_ident && s1.pid && s2.pid && s3.pid && s4.pid;
    out.qid = t_is_id && s1.qid && s2.qid && s3.qid && s4.qid;
    if (!out.pid || !out.qid) {
        PLUQ_TRY(launch_compose(vec(p1, s1.pid), P2, P3, P4, vec(q1, s1.qid), Q2, Q3, Q4, pp, pq,
                                c.smap, c.tmap, m, n, k, h, r1, r2, r3, r4, c.st));
    }
    if (!s_ident || !t_is_id)
        PLUQ_TRY(permute_block(c, A, lda, m, n, s_ident ? nullptr : c.smap,
                               t_is_id ? nullptr : c.tmap));
    c.vtop = vmark;
    return PLUQ_OK;
}

struct TuneInit {
    TuneInit() { g_tune_leaf.store(initial_leaf()); }
} g_tune_init;

struct Layout {
    size_t gather, icopy, maps, vstack, small, arena, total;
};

Layout layout_core(int64_t m, int64_t n, uint32_t p, int kind)
{
    Layout L{};
    const int64_t mn = m < n ? m : n;
    L.gather = align_up((size_t)m * n * 4 + 256, 256);
    L.icopy = align_up((size_t)((m + 1) / 2) * ((n + 1) / 2) * 4 + 256, 256);
    L.maps = align_up((size_t)(m + n + 2) * 4, 256);
    L.vstack = align_up((size_t)(8 * (m + n) + 64 * 64) * 4, 256);
    L.small = 256;
    L.arena = trsm_workspace(mn, m > n ? m : n, p, kind);
    if (kind != PLUQ_MM_SIMT) L.arena += mm_tc_workspace(m, n, mn, p, 1);
    L.arena = align_up(L.arena + (1 << 20), 256);
    L.total = L.gather + L.icopy + L.maps + L.vstack + L.small + L.arena;
    return L;
}

bool has_branches(int64_t m, int64_t n) { return m >= BRANCH_MATRIX_MIN && n >= BRANCH_MATRIX_MIN; }

// the main context, then NBRANCH branch contexts for ceil(m/2) x ceil(n/2)
struct Layout2 {
    Layout main, branch;
    size_t total;
};
Layout2 layout(int64_t m, int64_t n, uint32_t p, int kind, bool branches = true)
{
    Layout2 L{};
    L.main = layout_core(m, n, p, kind);
    L.total = L.main.total;
    if (branches && has_branches(m, n)) {
        L.branch = layout_core((m + 1) / 2, (n + 1) / 2, p, kind);
        L.total += NBRANCH * L.branch.total;
    }
    return L;
}

// carve one context's scratch out of w (advancing w)
void carve(Ctx &c, const Layout &L, int64_t m, char *&w)
{
    c.gather = (uint32_t *)w; w += L.gather;
    c.icopy = (uint32_t *)w; w += L.icopy;
    c.smap = (int32_t *)w;
    c.tmap = c.smap + m;
    w += L.maps;
    c.vstack = (int32_t *)w;
    c.vcap = L.vstack / 4;
    c.vtop = 0;
    w += L.vstack;
    c.d_rank = (int32_t *)w; w += L.small;
    c.ar.base = w;
    c.ar.size = L.arena;
    c.ar.off = 0;
    w += L.arena;
}

int resolve_kind(int kind)
{
    if (kind == PLUQ_MM_AUTO) return PLUQ_MM_TENSOR;
    return kind;
}

}  // namespace
}  // namespace pluq

using namespace pluq;

extern "C" {

const char *pluq_status_string(int s)
{
    switch (s) {
        case PLUQ_OK: return "ok";
        case PLUQ_EINVAL: return "invalid argument";
        case PLUQ_ENOTPRIME: return "modulus is not a prime in [2, 2^31)";
        case PLUQ_ERANGE: return "matrix entry not reduced modulo p";
        case PLUQ_ENOMEM: return "workspace too small";
        case PLUQ_ECUDA: return "CUDA runtime error";
        case PLUQ_ETIMEOUT: return "bounded device wait gave up";
        case PLUQ_EINTERNAL: return "internal consistency check failed";
        case PLUQ_EUNSUPPORTED: return "kernel form not available";
        default: return "unknown status";
    }
}

int pluq_tensor_limbs(uint32_t p) { return limbs_for_prime(p); }

pluq_status pluq_set_tuning(int64_t leaf, int64_t small_mm_macs)
{
    if (leaf < 16 || leaf > LEAF_MAX || small_mm_macs < 0) return PLUQ_EINVAL;
    g_tune_leaf.store(leaf);
    g_tune_small_mm.store(small_mm_macs);
    return PLUQ_OK;
}

pluq_status pluq_get_tuning(int64_t *h_leaf, int64_t *h_small_mm_macs)
{
    if (!h_leaf || !h_small_mm_macs) return PLUQ_EINVAL;
    *h_leaf = g_tune_leaf.load();
    *h_small_mm_macs = g_tune_small_mm.load();
    return PLUQ_OK;
}
int64_t pluq_leaf_max_rows(void) { return LEAF_MAX; }
int64_t pluq_leaf_max_cols(void) { return LEAF_MAX; }

pluq_status pluq_workspace_size(int64_t m, int64_t n, uint32_t p, size_t *h_bytes)
{
    if (m < 0 || n < 0 || !h_bytes) return PLUQ_EINVAL;
    if (p >= 0x80000000u || !is_prime_u32(p)) return PLUQ_ENOTPRIME;
    // the tensor form's scratch bounds the SIMT form's too
    *h_bytes = layout(m, n, p, PLUQ_MM_TENSOR).total;
    return PLUQ_OK;
}

}  // extern "C"

namespace pluq {
namespace {

// One decomposition on `st` with scratch at `w` (validated by the caller).
pluq_status run_one(uint32_t *d_A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                    int32_t *d_perm_p, int32_t *d_perm_q, int64_t *h_rank, char *w, int kind,
                    cudaStream_t st, HostWords *hw, bool branches)
{
    Layout2 L = layout(m, n, p, kind, branches);
    *h_rank = 0;
    if (m == 0 || n == 0) {
        PLUQ_TRY(launch_iota(d_perm_p, m, st));
        PLUQ_TRY(launch_iota(d_perm_q, n, st));
        return PLUQ_OK;
    }
    Ctx c;
    c.F = make_field(p);
    c.kind = kind;
    c.st = st;
    carve(c, L.main, m, w);
    c.hw = hw;
    c.leaf = leaf_size();
    // streams, events and host words of this decomposition's contexts live
    // until it returns
    Ctx branch[NBRANCH];
    BranchPool pool;
    struct Guard {
        Ctx &c;
        Ctx *b;
        ~Guard()
        {
            auto drop = [](Ctx &x, bool own_stream) {
                if (x.ev_fork) cudaEventDestroy(x.ev_fork);
                if (x.ev_join) cudaEventDestroy(x.ev_join);
                if (x.ev_done) cudaEventDestroy(x.ev_done);
                if (x.side) cudaStreamDestroy(x.side);
                if (own_stream && x.st) cudaStreamDestroy(x.st);
            };
            drop(c, false);
            for (int i = 0; i < NBRANCH; ++i) {
                drop(b[i], true);
                if (b[i].hw) release_words(b[i].hw);
            }
        }
    } guard{c, branch};
    auto make_streams = [](Ctx &x) {
        return cudaStreamCreateWithFlags(&x.side, cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreateWithFlags(&x.ev_fork, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&x.ev_join, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&x.ev_done, cudaEventDisableTiming) == cudaSuccess;
    };
    if (!make_streams(c)) return PLUQ_ECUDA;
    if (branches && has_branches(m, n)) {
        for (int i = 0; i < NBRANCH; ++i) {
            Ctx &b = branch[i];
            b.F = c.F;
            b.kind = kind;
            b.leaf = c.leaf;
            if (cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking) != cudaSuccess ||
                !make_streams(b))
                return PLUQ_ECUDA;
            b.hw = acquire_words();
            if (!b.hw) return PLUQ_ECUDA;
            carve(b, L.branch, (m + 1) / 2, w);
            PLUQ_CUDA_TRY(cudaMemsetAsync(b.d_rank, 0, 64, st));
            b.pool = &pool;
            pool.free.push_back(&b);
        }
        c.pool = &pool;
    }

    // every entry must already be reduced: checked before anything is written
    int32_t flag = 0;
    PLUQ_CUDA_TRY(cudaMemsetAsync(c.d_rank, 0, 64, st));
    PLUQ_TRY(launch_check_range(d_A, lda, m, n, p, c.d_rank, st));
    PLUQ_CUDA_TRY(cudaMemcpyAsync(&flag, c.d_rank, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PLUQ_CUDA_TRY(cudaStreamSynchronize(st));
    if (flag != 0) return PLUQ_ERANGE;

    Res res;
    PLUQ_TRY(rec(c, d_A, m, n, lda, d_perm_p, d_perm_q, res, 0, false));
    if (res.pid) PLUQ_TRY(launch_iota(d_perm_p, m, st));
    if (res.qid) PLUQ_TRY(launch_iota(d_perm_q, n, st));
    PLUQ_CUDA_TRY(cudaStreamSynchronize(st));
    if (tc_error_flag()) return PLUQ_ETIMEOUT;
    *h_rank = res.r;
    return PLUQ_OK;
}

pluq_status check_args(uint32_t *d_A, int64_t m, int64_t n, int64_t lda, int32_t *d_perm_p,
                       int32_t *d_perm_q)
{
    if (m < 0 || n < 0) return PLUQ_EINVAL;
    if (m > (1ll << 31) - 1 || n > (1ll << 31) - 1) return PLUQ_EINVAL;
    if ((m > 0 && !d_perm_p) || (n > 0 && !d_perm_q)) return PLUQ_EINVAL;
    if (m > 0 && n > 0 && (!d_A || lda < n)) return PLUQ_EINVAL;
    return PLUQ_OK;
}

}  // namespace
}  // namespace pluq

extern "C" {

pluq_status pluq_mod_p(uint32_t *d_A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                       int32_t *d_perm_p, int32_t *d_perm_q, int64_t *h_rank, void *d_work,
                       size_t ws_bytes, int mm_kind, void *stream)
{
    if (!h_rank) return PLUQ_EINVAL;
    PLUQ_TRY(check_args(d_A, m, n, lda, d_perm_p, d_perm_q));
    if (mm_kind < PLUQ_MM_AUTO || mm_kind > PLUQ_MM_TENSOR) return PLUQ_EINVAL;
    if (p >= 0x80000000u || !is_prime_u32(p)) return PLUQ_ENOTPRIME;
    const int kind = resolve_kind(mm_kind);
    if (!d_work || ws_bytes < layout(m, n, p, kind).total) return PLUQ_ENOMEM;
    HostWords *hw = acquire_words();
    if (!hw) return PLUQ_ECUDA;
    pluq_status s = run_one(d_A, m, n, lda, p, d_perm_p, d_perm_q, h_rank, (char *)d_work, kind,
                            (cudaStream_t)stream, hw, true);
    release_words(hw);
    return s;
}

pluq_status pluq_batched_workspace_size(const int64_t *h_m, const int64_t *h_n, int64_t count,
                                        uint32_t p, int workers, size_t *h_bytes)
{
    if (count < 0 || workers < 1 || !h_bytes || (count > 0 && (!h_m || !h_n))) return PLUQ_EINVAL;
    if (p >= 0x80000000u || !is_prime_u32(p)) return PLUQ_ENOTPRIME;
    size_t mx = 0;
    for (int64_t i = 0; i < count; ++i) {
        if (h_m[i] < 0 || h_n[i] < 0) return PLUQ_EINVAL;
        const size_t w = layout(h_m[i], h_n[i], p, PLUQ_MM_TENSOR, false).total;
        if (w > mx) mx = w;
    }
    const int64_t used = count < workers ? (count > 0 ? count : 1) : workers;
    *h_bytes = align_up(mx, 4096) * (size_t)used;
    return PLUQ_OK;
}

pluq_status pluq_mod_p_batched(uint32_t *const *h_dA, const int64_t *h_m, const int64_t *h_n,
                               const int64_t *h_lda, int64_t count, uint32_t p,
                               int32_t *const *h_dperm_p, int32_t *const *h_dperm_q,
                               int64_t *h_rank, void *d_work, size_t ws_bytes, int mm_kind,
                               int workers, void *stream)
{
    if (count < 0 || workers < 1) return PLUQ_EINVAL;
    if (count == 0) return PLUQ_OK;
    if (!h_dA || !h_m || !h_n || !h_lda || !h_dperm_p || !h_dperm_q || !h_rank) return PLUQ_EINVAL;
    if (mm_kind < PLUQ_MM_AUTO || mm_kind > PLUQ_MM_TENSOR) return PLUQ_EINVAL;
    if (p >= 0x80000000u || !is_prime_u32(p)) return PLUQ_ENOTPRIME;
    for (int64_t i = 0; i < count; ++i)
        PLUQ_TRY(check_args(h_dA[i], h_m[i], h_n[i], h_lda[i], h_dperm_p[i], h_dperm_q[i]));
    size_t need = 0;
    PLUQ_TRY(pluq_batched_workspace_size(h_m, h_n, count, p, workers, &need));
    if (!d_work || ws_bytes < need) return PLUQ_ENOMEM;
    const int kind = resolve_kind(mm_kind);
    const int T = (int)(count < workers ? count : workers);
    const size_t slice = need / (size_t)T;

    // largest matrices first, so the tail of the batch is made of small ones
    std::vector<int64_t> order(count);
    for (int64_t i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        return h_m[a] * h_n[a] > h_m[b] * h_n[b];
    });

    int dev = 0;
    PLUQ_CUDA_TRY(cudaGetDevice(&dev));
    cudaEvent_t start;
    PLUQ_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    if (cudaEventRecord(start, (cudaStream_t)stream) != cudaSuccess) {
        cudaEventDestroy(start);
        return PLUQ_ECUDA;
    }
    std::atomic<int64_t> next{0};
    std::atomic<int> first_err{PLUQ_OK};
    auto worker = [&](int t) {
        if (cudaSetDevice(dev) != cudaSuccess) { first_err.store(PLUQ_ECUDA); return; }
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            first_err.store(PLUQ_ECUDA);
            return;
        }
        HostWords *hw = acquire_words();
        if (!hw || cudaStreamWaitEvent(st, start, 0) != cudaSuccess) {
            first_err.store(PLUQ_ECUDA);
        } else {
            char *w = (char *)d_work + (size_t)t * slice;
            for (;;) {
                if (first_err.load() != PLUQ_OK) break;
                const int64_t q = next.fetch_add(1);
                if (q >= count) break;
                const int64_t i = order[q];
                pluq_status s = run_one(h_dA[i], h_m[i], h_n[i], h_lda[i], p, h_dperm_p[i],
                                        h_dperm_q[i], &h_rank[i], w, kind, st, hw, false);
                if (s != PLUQ_OK) {
                    int expect = PLUQ_OK;
                    first_err.compare_exchange_strong(expect, (int)s);
                    break;
                }
            }
        }
        release_words(hw);
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    };
    std::vector<std::thread> pool;
    pool.reserve(T);
    for (int t = 0; t < T; ++t) pool.emplace_back(worker, t);
    for (auto &th : pool) th.join();
    cudaEventDestroy(start);
    return (pluq_status)first_err.load();
}

pluq_status row_rank_profile(const int32_t *d_perm_p, int64_t m, int64_t r, int32_t *d_out,
                             void *stream)
{
    if (r < 0 || r > m || (r > 0 && (!d_perm_p || !d_out))) return PLUQ_EINVAL;
    return launch_rank_sort(d_perm_p, nullptr, r, d_out, nullptr, (cudaStream_t)stream);
}

pluq_status col_rank_profile(const int32_t *d_perm_q, int64_t n, int64_t r, int32_t *d_out,
                             void *stream)
{
    if (r < 0 || r > n || (r > 0 && (!d_perm_q || !d_out))) return PLUQ_EINVAL;
    return launch_rank_sort(d_perm_q, nullptr, r, d_out, nullptr, (cudaStream_t)stream);
}

pluq_status rank_profile_matrix(const int32_t *d_perm_p, const int32_t *d_perm_q, int64_t m,
                                int64_t n, int64_t r, int32_t *d_rows, int32_t *d_cols,
                                void *stream)
{
    if (r < 0 || r > m || r > n) return PLUQ_EINVAL;
    if (r > 0 && (!d_perm_p || !d_perm_q || !d_rows || !d_cols)) return PLUQ_EINVAL;
    return launch_rank_sort(d_perm_p, d_perm_q, r, d_rows, d_cols, (cudaStream_t)stream);
}

pluq_status pluq_extract_L(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda, int64_t r,
                           uint32_t *d_L, int64_t ldl, void *stream)
{
    if (m < 0 || n < 0 || r < 0 || r > m || r > n || lda < n) return PLUQ_EINVAL;
    if (m > 0 && r > 0 && (!d_LU || !d_L || ldl < r)) return PLUQ_EINVAL;
    return launch_extract(d_LU, lda, m, r, d_L, ldl, true, (cudaStream_t)stream);
}

pluq_status pluq_extract_U(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda, int64_t r,
                           uint32_t *d_U, int64_t ldu, void *stream)
{
    if (m < 0 || n < 0 || r < 0 || r > m || r > n || lda < n) return PLUQ_EINVAL;
    if (n > 0 && r > 0 && (!d_LU || !d_U || ldu < n)) return PLUQ_EINVAL;
    return launch_extract(d_LU, lda, r, n, d_U, ldu, false, (cudaStream_t)stream);
}

pluq_status pluq_leu(const uint32_t *d_LU, int64_t m, int64_t n, int64_t lda, int64_t r,
                     const int32_t *d_perm_p, const int32_t *d_perm_q, uint32_t *d_Lbar,
                     int64_t ldl, uint32_t *d_Ubar, int64_t ldu, void *d_work, size_t ws_bytes,
                     void *stream)
{
    if (m < 0 || n < 0 || r < 0 || r > m || r > n || lda < n) return PLUQ_EINVAL;
    if (!d_Lbar && !d_Ubar) return PLUQ_EINVAL;
    if (m > 0 && n > 0 && !d_LU) return PLUQ_EINVAL;
    if (d_Lbar && m > 0 && (!d_perm_p || ldl < m)) return PLUQ_EINVAL;
    if (d_Ubar && n > 0 && (!d_perm_q || ldu < n)) return PLUQ_EINVAL;
    if (!d_work || ws_bytes < (size_t)(m + n) * sizeof(int32_t)) return PLUQ_ENOMEM;
    return launch_leu(d_LU, lda, m, n, r, d_perm_p, d_perm_q, d_Lbar, ldl, d_Ubar, ldu,
                      (int32_t *)d_work, (cudaStream_t)stream);
}

pluq_status pluq_leading_rank_profiles(const int32_t *d_perm_p, const int32_t *d_perm_q,
                                       int64_t m, int64_t n, int64_t r, int64_t k, int64_t t,
                                       int32_t *d_rows, int32_t *d_cols, int32_t *d_count,
                                       void *stream)
{
    if (r < 0 || r > m || r > n || k < 0 || k > m || t < 0 || t > n || !d_count)
        return PLUQ_EINVAL;
    if (r > 0 && (!d_perm_p || !d_perm_q || !d_rows || !d_cols)) return PLUQ_EINVAL;
    return launch_leading_profile(d_perm_p, d_perm_q, r, k, t, d_rows, d_cols, d_count,
                                  (cudaStream_t)stream);
}

pluq_status pluq_modmm_workspace_size(int64_t M, int64_t N, int64_t K, uint32_t p, int mm_kind,
                                      size_t *h_bytes)
{
    if (M < 0 || N < 0 || K < 0 || !h_bytes) return PLUQ_EINVAL;
    if (p >= 0x80000000u || !is_prime_u32(p)) return PLUQ_ENOTPRIME;
    *h_bytes = resolve_kind(mm_kind) == PLUQ_MM_SIMT ? 0 : mm_tc_workspace(M, N, K, p, 1);
    return PLUQ_OK;
}

pluq_status pluq_modmm(uint32_t *d_C, int64_t ldc, const uint32_t *d_A, int64_t lda,
                       const uint32_t *d_B, int64_t ldb, int64_t M, int64_t N, int64_t K,
                       uint32_t p, int assign, int mm_kind, void *d_work, size_t ws_bytes,
                       void *stream)
{
    if (M < 0 || N < 0 || K < 0) return PLUQ_EINVAL;
    if (mm_kind < PLUQ_MM_AUTO || mm_kind > PLUQ_MM_TENSOR) return PLUQ_EINVAL;
    if (p >= 0x80000000u || !is_prime_u32(p)) return PLUQ_ENOTPRIME;
    if (M > 0 && N > 0 && (!d_C || ldc < N)) return PLUQ_EINVAL;
    if (M > 0 && K > 0 && (!d_A || lda < K)) return PLUQ_EINVAL;
    if (K > 0 && N > 0 && (!d_B || ldb < N)) return PLUQ_EINVAL;
    const int kind = resolve_kind(mm_kind);
    Arena ar;
    ar.base = (char *)d_work;
    ar.size = d_work ? ws_bytes : 0;
    ar.off = 0;
    if (kind != PLUQ_MM_SIMT && ar.size < mm_tc_workspace(M, N, K, p, 1)) return PLUQ_ENOMEM;
    return launch_mm(kind, Blk{d_C, ldc}, d_A, lda, d_B, ldb, M, N, K, make_field(p),
                     assign ? MM_ASSIGN : MM_SUB, 1, 0, 0, 0, ar, (cudaStream_t)stream);
}

pluq_status pluq_trsm_workspace_size(int64_t r, int64_t other, uint32_t p, int mm_kind,
                                     size_t *h_bytes)
{
    if (r < 0 || other < 0 || !h_bytes) return PLUQ_EINVAL;
    if (p >= 0x80000000u || !is_prime_u32(p)) return PLUQ_ENOTPRIME;
    *h_bytes = trsm_workspace(r, other, p, resolve_kind(mm_kind));
    return PLUQ_OK;
}

pluq_status pluq_trsm_left_lower_unit(const uint32_t *d_L, int64_t ldl, uint32_t *d_B,
                                      int64_t ldb, int64_t r, int64_t N, uint32_t p, int mm_kind,
                                      void *d_work, size_t ws_bytes, void *stream)
{
    if (r < 0 || N < 0) return PLUQ_EINVAL;
    if (mm_kind < PLUQ_MM_AUTO || mm_kind > PLUQ_MM_TENSOR) return PLUQ_EINVAL;
    if (p >= 0x80000000u || !is_prime_u32(p)) return PLUQ_ENOTPRIME;
    if (r > 0 && N > 0 && (!d_L || !d_B || ldl < r || ldb < N)) return PLUQ_EINVAL;
    const int kind = resolve_kind(mm_kind);
    if (!d_work || ws_bytes < trsm_workspace(r, N, p, kind)) return PLUQ_ENOMEM;
    Arena ar;
    ar.base = (char *)d_work;
    ar.size = ws_bytes;
    return trsm_left_lower_unit(d_L, ldl, Blk{d_B, ldb}, r, N, make_field(p), kind, ar,
                                (cudaStream_t)stream);
}

pluq_status pluq_trsm_right_upper(const uint32_t *d_U, int64_t ldu, uint32_t *d_B, int64_t ldb,
                                  int64_t M, int64_t r, uint32_t p, int mm_kind, void *d_work,
                                  size_t ws_bytes, void *stream)
{
    if (r < 0 || M < 0) return PLUQ_EINVAL;
    if (mm_kind < PLUQ_MM_AUTO || mm_kind > PLUQ_MM_TENSOR) return PLUQ_EINVAL;
    if (p >= 0x80000000u || !is_prime_u32(p)) return PLUQ_ENOTPRIME;
    if (r > 0 && M > 0 && (!d_U || !d_B || ldu < r || ldb < r)) return PLUQ_EINVAL;
    const int kind = resolve_kind(mm_kind);
    if (!d_work || ws_bytes < trsm_workspace(r, M, p, kind)) return PLUQ_ENOMEM;
    Arena ar;
    ar.base = (char *)d_work;
    ar.size = ws_bytes;
    return trsm_right_upper(d_U, ldu, Blk{d_B, ldb}, M, r, make_field(p), kind, ar,
                            (cudaStream_t)stream);
}

pluq_status pluq_perm_rows(uint32_t *d_X, int64_t ldx, int64_t count, int64_t width,
                           const int32_t *d_perm, void *d_work, size_t ws_bytes, void *stream)
{
    if (count < 0 || width < 0) return PLUQ_EINVAL;
    if (count == 0 || width == 0) return PLUQ_OK;
    if (!d_X || !d_perm || ldx < width) return PLUQ_EINVAL;
    if (!d_work || ws_bytes < (size_t)count * width * 4) return PLUQ_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    PLUQ_TRY(launch_gather(Blk{(uint32_t *)d_work, width}, d_X, ldx, count, width, d_perm, nullptr,
                           st));
    return launch_copy(Blk{d_X, ldx}, (uint32_t *)d_work, width, count, width, st);
}

pluq_status pluq_perm_cols(uint32_t *d_X, int64_t ldx, int64_t height, int64_t count,
                           const int32_t *d_perm, void *d_work, size_t ws_bytes, void *stream)
{
    if (count < 0 || height < 0) return PLUQ_EINVAL;
    if (count == 0 || height == 0) return PLUQ_OK;
    if (!d_X || !d_perm || ldx < count) return PLUQ_EINVAL;
    if (!d_work || ws_bytes < (size_t)count * height * 4) return PLUQ_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    PLUQ_TRY(launch_gather(Blk{(uint32_t *)d_work, count}, d_X, ldx, height, count, nullptr,
                           d_perm, st));
    return launch_copy(Blk{d_X, ldx}, (uint32_t *)d_work, count, height, count, st);
}

pluq_status pluq_leaf(uint32_t *d_A, int64_t m, int64_t n, int64_t lda, uint32_t p,
                      int32_t *d_perm_p, int32_t *d_perm_q, int32_t *d_rank, void *stream)
{
    if (m < 0 || n < 0 || m > LEAF_MAX || n > LEAF_MAX || !d_rank) return PLUQ_EINVAL;
    if (p >= 0x80000000u || !is_prime_u32(p)) return PLUQ_ENOTPRIME;
    if ((m > 0 && !d_perm_p) || (n > 0 && !d_perm_q)) return PLUQ_EINVAL;
    if (m > 0 && n > 0 && (!d_A || lda < n)) return PLUQ_EINVAL;
    return launch_leaf(d_A, m, n, lda, make_field(p), d_perm_p, d_perm_q, d_rank, 1,
                       (cudaStream_t)stream);
}

}  // extern "C"
