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
#include <chrono>
#include <condition_variable>
#include <functional>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>
#include <stdlib.h>
#include <stdio.h>
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
pluq_status launch_check_range(const uint32_t *A, int64_t lda, int64_t m, int64_t n, uint32_t p,
                               int32_t *flag, cudaStream_t st);
pluq_status launch_any_nonzero(const uint32_t *A, int64_t lda, int64_t m, int64_t n, int32_t *words,
                               volatile int32_t *host, int32_t seq, cudaStream_t st);

std::atomic<int64_t> g_tune_small_mm{1ll << 25};
std::atomic<int64_t> g_tune_leaf{128};
// PLUQ(G) goes to another host thread when F and G both have at least this
// many rows and columns (a free branch context permitting)
std::atomic<int64_t> g_tune_branch{64};
std::atomic<int64_t> g_wait_limit{-1};
std::atomic<bool> g_tune_leaf_left{false};
std::atomic<int> g_tune_node{1};
std::atomic<int> g_tune_node_ctas{1};
// zero test of a block below a rank-deficient node: false = wait for it before
// descending (a zero block costs one round trip), true = read it with the first
// leaf of the descent (a nonzero block costs nothing extra)
std::atomic<bool> g_tune_lazy_zero{false};

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

// Products that share K, each to the CUDA-core kernel when launch_mm would
// send it there and otherwise all together in one grouped tensor-core launch.
pluq_status launch_mm_group(int kind, const MMSpec *q, int count, int64_t K, Field F, Arena &ar,
                            cudaStream_t st)
{
    MMSpec tc[2];
    int ntc = 0;
    for (int i = 0; i < count; ++i) {
        const MMSpec &x = q[i];
        if (x.M <= 0 || x.N <= 0 || x.batch <= 0) continue;
        bool simt = kind == PLUQ_MM_SIMT;
        if (!simt && K > 0 &&
            (double)x.M * x.N * K * x.batch <= (double)g_tune_small_mm.load(std::memory_order_relaxed)) {
            Span sc = span(x.C.ptr, x.C.ld, x.M, x.N, x.batch, x.sC);
            simt = !overlap(sc, span(x.A, x.lda, x.M, K, x.batch, x.sA)) &&
                   !overlap(sc, span(x.B, x.ldb, K, x.N, x.batch, x.sB));
        }
        if (simt || ntc == 2)
            PLUQ_TRY(launch_mm(simt ? PLUQ_MM_SIMT : kind, x.C, x.A, x.lda, x.B, x.ldb, x.M, x.N, K,
                               F, x.mode, x.batch, x.sA, x.sB, x.sC, ar, st));
        else
            tc[ntc++] = x;
    }
    if (ntc == 0) return PLUQ_OK;
    return launch_mm_tc_group(tc, ntc, K, F, ar, st);
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
// Host-side instrumentation (PLUQ_HOST_STATS=1 in the environment): after
// each decomposition, stderr gets the wall time, the summed time host threads
// spent waiting for leaf / zero-test results, and the number of waits.
const bool g_host_stats = getenv("PLUQ_HOST_STATS") != nullptr;
std::atomic<long long> g_wait_ns{0}, g_waits{0};

long long now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

pluq_status wait_words(HostWords *hw, int32_t seq, cudaStream_t st, int at = 0)
{
    const long long t0 = g_host_stats ? now_ns() : 0;
    struct Acc {
        long long t0;
        ~Acc()
        {
            if (g_host_stats) {
                g_wait_ns.fetch_add(now_ns() - t0, std::memory_order_relaxed);
                g_waits.fetch_add(1, std::memory_order_relaxed);
            }
        }
    } acc{t0};
    for (long long it = 0;; ++it) {
        if (hw->h[at] == seq) return PLUQ_OK;
        if ((it & 0xFFFF) == 0xFFFF) {
            cudaError_t e = cudaStreamQuery(st);
            if (e == cudaSuccess) return hw->h[at] == seq ? PLUQ_OK : PLUQ_EINTERNAL;
            if (e != cudaErrorNotReady) return PLUQ_ECUDA;
        }
        // several branch threads may wait at once: after a short spin, give
        // the core to the others
        if (it > 4096) std::this_thread::yield();
    }
}

// Streams and events of one recursion context, cached per device and reused
// across calls: creating them costs tens of microseconds each, a fixed cost
// that small decompositions would otherwise pay on every call.
struct Streams {
    int dev = -1;
    cudaStream_t st = nullptr, side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, done = nullptr;
};
std::mutex g_streams_mu;
std::vector<Streams *> g_streams_free;

Streams *acquire_streams()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    {
        std::lock_guard<std::mutex> lk(g_streams_mu);
        for (size_t i = 0; i < g_streams_free.size(); ++i)
            if (g_streams_free[i]->dev == dev) {
                Streams *s = g_streams_free[i];
                g_streams_free[i] = g_streams_free.back();
                g_streams_free.pop_back();
                return s;
            }
    }
    Streams *s = new (std::nothrow) Streams;
    if (!s) return nullptr;
    s->dev = dev;
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming) != cudaSuccess) {
        if (s->st) cudaStreamDestroy(s->st);
        if (s->side) cudaStreamDestroy(s->side);
        if (s->fork) cudaEventDestroy(s->fork);
        if (s->join) cudaEventDestroy(s->join);
        if (s->done) cudaEventDestroy(s->done);
        delete s;
        return nullptr;
    }
    return s;
}

void release_streams(Streams *s)
{
    if (!s) return;
    std::lock_guard<std::mutex> lk(g_streams_mu);
    g_streams_free.push_back(s);
}

// Host threads that run PLUQ(G) while the thread that reached the node runs
// PLUQ(F).  A task is only handed to a worker that is idle at that moment;
// when none is, the caller runs the task itself, so no task ever waits for a
// worker (a waiting parent can never block the child it waits on).
class Workers {
  public:
    static Workers &get()
    {
        static Workers w;
        return w;
    }
    bool try_run(std::function<void()> fn)
    {
        std::lock_guard<std::mutex> lk(mu_);
        for (auto &sl : slots_)
            if (!sl->busy) {
                sl->busy = true;
                sl->fn = std::move(fn);
                sl->cv.notify_one();
                return true;
            }
        if ((int)slots_.size() >= cap_) return false;
        std::unique_ptr<Slot> sl(new (std::nothrow) Slot);
        if (!sl) return false;
        sl->busy = true;
        sl->fn = std::move(fn);
        Slot *raw = sl.get();
        try {
            raw->th = std::thread([this, raw] { loop(raw); });
        } catch (...) {
            return false;
        }
        slots_.push_back(std::move(sl));
        return true;
    }
    ~Workers()
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            for (auto &sl : slots_) {
                sl->stop = true;
                sl->cv.notify_one();
            }
        }
        for (auto &sl : slots_)
            if (sl->th.joinable()) sl->th.join();
    }

  private:
    struct Slot {
        std::thread th;
        std::condition_variable cv;
        std::function<void()> fn;
        bool busy = false, stop = false;
    };
    Workers()
    {
        const int hc = (int)std::thread::hardware_concurrency();
        cap_ = std::max(1, std::min(30, hc - 2));
    }
    void loop(Slot *sl)
    {
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            sl->cv.wait(lk, [sl] { return sl->stop || (bool)sl->fn; });
            if (!sl->fn) return;
            std::function<void()> fn = std::move(sl->fn);
            sl->fn = nullptr;
            lk.unlock();
            fn();
            lk.lock();
            sl->busy = false;
            if (sl->stop) return;
        }
    }
    std::mutex mu_;
    std::vector<std::unique_ptr<Slot>> slots_;
    int cap_ = 1;
};

// completion flag of a task handed to a worker
struct Join {
    std::mutex mu;
    std::condition_variable cv;
    bool done = false;
    void set()
    {
        std::lock_guard<std::mutex> lk(mu);
        done = true;
        cv.notify_all();
    }
    void wait()
    {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [this] { return done; });
    }
};

// Host words 8 + 2d (sequence number) and 9 + 2d (flag) carry the zero test of
// the node at recursion depth d < ZDEPTH; word 0..3 belong to the leaf.
constexpr int ZBASE = 8, ZDEPTH = 27;

struct Ctx {
    Field F{};
    int kind = 0;
    cudaStream_t st = nullptr;
    Arena ar;                       // scratch for products / TRSM (stack discipline)
    uint32_t *gather = nullptr;     // scratch for permutations too large to stage on chip
    size_t gather_elems = 0;
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
    int64_t cap_m = 0, cap_n = 0;           // largest block this context's scratch serves
    int dev = 0;                            // device of the decomposition
    int64_t leaves = 0;
    int64_t zero_checks = 0;
};

// Contexts that can each run one recursive call on a host thread of its own,
// with their own streams, host words and scratch.  They come in tiers: tier t
// serves blocks of up to ceil(m / 2^(t+1)) x ceil(n / 2^(t+1)) (the block G of a
// node at depth t fits), so PLUQ(F) and PLUQ(G) can run side by side at every
// level of the recursion, not only near the top.
constexpr int NTIER = 4;
constexpr int TIER_COUNT[NTIER] = {2, 3, 4, 6};
constexpr int NBRANCH = 2 + 3 + 4 + 6;      // branch contexts per decomposition
constexpr int64_t BRANCH_MATRIX_MIN = 256;  // matrices below this get no branch contexts

struct BranchPool {
    std::mutex mu;
    std::vector<Ctx *> free;
    // the free context with the least scratch that still holds an mb x nb block
    Ctx *take(int64_t mb, int64_t nb)
    {
        std::lock_guard<std::mutex> lk(mu);
        int best = -1;
        for (int i = 0; i < (int)free.size(); ++i)
            if (free[i]->cap_m >= mb && free[i]->cap_n >= nb &&
                (best < 0 || free[i]->cap_m * free[i]->cap_n < free[best]->cap_m * free[best]->cap_n))
                best = i;
        if (best < 0) return nullptr;
        Ctx *c = free[best];
        free[best] = free.back();
        free.pop_back();
        return c;
    }
    void give(Ctx *c)
    {
        std::lock_guard<std::mutex> lk(mu);
        free.push_back(c);
    }
};

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

// In-place row / column permutations of disjoint blocks, issued in one launch
// (ops with a null map are identities and dropped).
struct PermBatch {
    PermOp op[4];
    int n = 0;
    void rows(uint32_t *X, int64_t ld, int64_t nr, int64_t nc, const int32_t *map, int32_t moff = 0)
    {
        if (nr > 0 && nc > 0 && map) op[n++] = PermOp{X, ld, nr, nc, map, moff, true};
    }
    void cols(uint32_t *X, int64_t ld, int64_t nr, int64_t nc, const int32_t *map, int32_t moff = 0)
    {
        if (nr > 0 && nc > 0 && map) op[n++] = PermOp{X, ld, nr, nc, map, moff, false};
    }
};

pluq_status run_perms(Ctx &c, const PermBatch &b)
{
    if (b.n == 0) return PLUQ_OK;
    return launch_perm_ops(b.op, b.n, c.gather, c.gather_elems, c.st);
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
        if (r < 0 && leaf_error_flag()) return PLUQ_ETIMEOUT;
        if (r < 0 || r > m || r > n) return PLUQ_EINTERNAL;
        out.r = r;
        out.pid = c.hw->h[2] != 0;
        out.qid = c.hw->h[3] != 0;
        return PLUQ_OK;
    }
    // below a rank-deficient node, a node whose four blocks are base cases
    // runs as one step on the device (launch_node): one launch, one round trip
    const int node_levels = g_tune_node.load(std::memory_order_relaxed);
    const int64_t node_side = std::min<int64_t>((int64_t)2 * node_levels * c.leaf, 4 * LEAF_MAX);
    if (eager && node_levels > 0 && m <= node_side && n <= node_side) {
        const int32_t seq = ++c.hw->seq;
        PLUQ_TRY(launch_node(A, m, n, lda, c.F, pp, pq, c.d_rank + 4, c.st, c.hw->d, seq, false,
                             c.gather, (int64_t)c.gather_elems, c.icopy));
        PLUQ_TRY(wait_words(c.hw, seq, c.st));
        const int32_t r = c.hw->h[1];
        ++c.leaves;
        if (r < 0 && leaf_error_flag()) return PLUQ_ETIMEOUT;
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
    const bool lazy = (!eager || g_tune_lazy_zero.load(std::memory_order_relaxed)) && depth < ZDEPTH;
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
    // [B1;B2] <- P1^T A2 ; [C1 C2] <- A3 Q1^T (disjoint blocks, one launch)
    {
        PermBatch pb;
        pb.rows(at(0, h), lda, k, n - h, vec(p1, s1.pid));
        pb.cols(at(k, 0), lda, m - k, h, vec(q1, s1.qid));
        PLUQ_TRY(run_perms(c, pb));
    }
    // D <- L1^{-1} B1 ; E <- C1 U1^{-1}, then [F;H] <- [B2;A4] - [M1;E] D and
    // G <- C2 - E V1: each pair is independent (disjoint outputs, shared
    // read-only operands).  The second of a pair runs on the side stream when
    // the arena has room for both scratch areas side by side.
    if (trsm_small_for(r1)) {
        // a small triangle: both solves in one launch
        PLUQ_TRY(trsm_pair_small(A, lda, Blk{at(0, h), lda}, r1, n - h, A, lda, Blk{at(k, 0), lda},
                                 m - k, r1, F, c.st));
    } else {
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
    // [F;H] <- [B2;A4] - [M1;E] D and G <- C2 - E V1 share K = r1: one
    // grouped launch (disjoint outputs, read-only operands)
    if (r1 > 0) {
        const MMSpec q[2] = {
            {Blk{at(r1, h), lda}, at(r1, 0), lda, at(0, h), lda, m - r1, n - h, MM_SUB, 1, 0, 0, 0},
            {Blk{at(k, r1), lda}, at(k, 0), lda, at(0, r1), lda, m - k, h - r1, MM_SUB, 1, 0, 0, 0}};
        PLUQ_TRY(launch_mm_group(c.kind, q, 2, r1, F, c.ar, c.st));
    }
    // F = P2 [L2;M2][U2 V2] Q2 ; G = P3 [L3;M3][U3 V3] Q3
    // PLUQ(F) and PLUQ(G) work on disjoint blocks with their own permutation
    // vectors: with a free branch context, G runs on another host thread and
    // stream while this thread does F (the concurrency noted in Sec. 9)
    Res s2, s3;
    Ctx *bc = nullptr;
    const int64_t bmin = g_tune_branch.load(std::memory_order_relaxed);
    if (c.pool && k - r1 >= bmin && n - h >= bmin && m - k >= bmin && h - r1 >= bmin)
        bc = c.pool->take(m - k, h - r1);
    if (bc) {
        pluq_status sg = PLUQ_OK, sf = PLUQ_OK;
        if (cudaEventRecord(c.ev_fork, c.st) != cudaSuccess ||
            cudaStreamWaitEvent(bc->st, c.ev_fork, 0) != cudaSuccess) {
            c.pool->give(bc);
            return PLUQ_ECUDA;
        }
        Join jn;
        const bool handed = Workers::get().try_run([&] {
            if (cudaSetDevice(bc->dev) != cudaSuccess) sg = PLUQ_ECUDA;
            else sg = rec(*bc, at(k, r1), m - k, h - r1, lda, p3, q3, s3, depth + 1, deficient);
            jn.set();
        });
        sf = rec(c, at(r1, h), k - r1, n - h, lda, p2, q2, s2, depth + 1, deficient);
        if (handed) jn.wait();
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
    // H <- P3^T H Q2^T ; E <- P3^T E ; M1 <- P2^T M1 ; D <- D Q2^T ; V1 <- V1 Q3^T:
    // the row permutations in one launch, then the column permutations (H
    // takes both; G and F, already factored, sit between the pieces and stay)
    {
        PermBatch pr, pc;
        pr.rows(at(k, 0), lda, m - k, r1, P3);
        pr.rows(at(k, h), lda, m - k, n - h, P3);
        pr.rows(at(r1, 0), lda, k - r1, r1, P2);
        pc.cols(at(0, h), lda, r1, n - h, Q2);
        pc.cols(at(k, h), lda, m - k, n - h, Q2);
        pc.cols(at(0, r1), lda, r1, h - r1, Q3);
        PLUQ_TRY(run_perms(c, pr));
        PLUQ_TRY(run_perms(c, pc));
    }
    // [I;K] <- [H1;H3] U2^{-1}
    const uint32_t *U2 = at(r1, h);
    PLUQ_TRY(trsm_right_upper(U2, lda, Blk{at(k, h), lda}, m - k, r2, F, c.kind, c.ar, c.st));
    // keep I; [J N] <- L3^{-1} [I H2]
    if (r3 > 0 && r2 > 0) PLUQ_TRY(launch_copy(Blk{c.icopy, r2}, at(k, h), lda, r3, r2, c.st));
    const uint32_t *L3 = at(k, r1);
    PLUQ_TRY(trsm_left_lower_unit(L3, lda, Blk{at(k, h), lda}, r3, n - h, F, c.kind, c.ar, c.st));
    // O <- N - J V2 and R <- H4 - K V2 share K = r2 (disjoint outputs): one
    // grouped launch; then I goes back and R <- R - M3 O
    if (r2 > 0) {
        const MMSpec q[2] = {
            {Blk{at(k, h + r2), lda}, at(k, h), lda, at(r1, h + r2), lda, r3, n - h - r2, MM_SUB, 1,
             0, 0, 0},
            {Blk{at(k + r3, h + r2), lda}, at(k + r3, h), lda, at(r1, h + r2), lda, m - k - r3,
             n - h - r2, MM_SUB, 1, 0, 0, 0}};
        PLUQ_TRY(launch_mm_group(c.kind, q, 2, r2, F, c.ar, c.st));
    }
    if (r3 > 0 && r2 > 0) PLUQ_TRY(launch_copy(Blk{at(k, h), lda}, c.icopy, r2, r3, r2, c.st));
    PLUQ_TRY(launch_mm(c.kind, Blk{at(k + r3, h + r2), lda}, at(k + r3, r1), lda, at(k, h + r2),
                       lda, m - k - r3, n - h - r2, r3, F, MM_SUB, 1, 0, 0, 0, c.ar, c.st));
    // R = P4 [L4;M4][U4 V4] Q4
    Res s4;
    PLUQ_TRY(rec(c, at(k + r3, h + r2), m - k - r3, n - h - r2, lda, p4, q4, s4, depth + 1,
                 deficient));
    const int64_t r4 = s4.r;
    int32_t *P4 = vec(p4, s4.pid), *Q4 = vec(q4, s4.qid);
    // [E2 M3 0 K] <- P4^T [..] ; [D2;V2;0;O] <- [..] Q4^T (disjoint, one launch)
    {
        PermBatch pb;
        pb.rows(at(k + r3, 0), lda, m - k - r3, h + r2, P4);
        pb.cols(at(0, h + r2), lda, k + r3, n - h - r2, Q4);
        PLUQ_TRY(run_perms(c, pb));
    }
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
    // S only moves rows [r1+r2, k+r3+r4) and T only columns [r1, h+r2+r4) (the
    // segments before and after stay), so the passes cover those bands
    if (!s_ident) {
        PermBatch pb;
        const int64_t b0 = r1 + r2, b1 = k + r3 + r4;
        pb.rows(at(b0, 0), lda, b1 - b0, n, c.smap + b0, (int32_t)b0);
        PLUQ_TRY(run_perms(c, pb));
    }
    if (!t_is_id) {
        PermBatch pb;
        const int64_t b0 = r1, b1 = h + r2 + r4;
        pb.cols(at(0, b0), lda, m, b1 - b0, c.tmap + b0, (int32_t)b0);
        PLUQ_TRY(run_perms(c, pb));
    }
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
    L.gather = align_up((size_t)m * (n + 4) * 4 + 256, 256);
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

// block sides tier t of the branch contexts serves: ceil(x / 2^(t+1))
int64_t tier_dim(int64_t x, int t) { return (x + (2ll << t) - 1) >> (t + 1); }

// the main context, then TIER_COUNT[t] branch contexts of each tier t
struct Layout2 {
    Layout main, branch[NTIER];
    size_t total;
};
Layout2 layout(int64_t m, int64_t n, uint32_t p, int kind, bool branches = true)
{
    Layout2 L{};
    L.main = layout_core(m, n, p, kind);
    L.total = L.main.total;
    if (branches && has_branches(m, n)) {
        for (int t = 0; t < NTIER; ++t) {
            L.branch[t] = layout_core(tier_dim(m, t), tier_dim(n, t), p, kind);
            L.total += TIER_COUNT[t] * L.branch[t].total;
        }
    }
    return L;
}

// carve one context's scratch out of w (advancing w)
void carve(Ctx &c, const Layout &L, int64_t m, char *&w)
{
    c.gather = (uint32_t *)w;
    c.gather_elems = L.gather / 4;
    w += L.gather;
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

pluq_status pluq_set_branch_min(int64_t branch_min)
{
    if (branch_min < 1) return PLUQ_EINVAL;
    g_tune_branch.store(branch_min);
    return PLUQ_OK;
}

int64_t pluq_get_branch_min(void) { return g_tune_branch.load(); }

pluq_status pluq_set_leaf_variant(int left_looking)
{
    if (left_looking != 0 && left_looking != 1) return PLUQ_EINVAL;
    g_tune_leaf_left.store(left_looking != 0);
    return PLUQ_OK;
}

int pluq_get_leaf_variant(void) { return g_tune_leaf_left.load() ? 1 : 0; }

pluq_status pluq_set_node_kernel(int levels)
{
    if (levels < 0 || levels > 2) return PLUQ_EINVAL;
    g_tune_node.store(levels);
    return PLUQ_OK;
}

int pluq_get_node_kernel(void) { return g_tune_node.load(); }

pluq_status pluq_set_node_cluster(int ctas)
{
    if (ctas != 1 && ctas != 2 && ctas != 4 && ctas != 8) return PLUQ_EINVAL;
    g_tune_node_ctas.store(ctas);
    return PLUQ_OK;
}

int pluq_get_node_cluster(void) { return g_tune_node_ctas.load(); }

pluq_status pluq_set_wait_limit(int64_t tries)
{
    g_wait_limit.store(tries < 0 ? -1 : tries);
    return PLUQ_OK;
}

pluq_status pluq_device_status(void *stream)
{
    PLUQ_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    const int tc = tc_error_flag(), lf = leaf_error_flag();
    return tc || lf ? PLUQ_ETIMEOUT : PLUQ_OK;
}

pluq_status pluq_set_lazy_zero_test(int lazy)
{
    if (lazy != 0 && lazy != 1) return PLUQ_EINVAL;
    g_tune_lazy_zero.store(lazy != 0);
    return PLUQ_OK;
}

int pluq_get_lazy_zero_test(void) { return g_tune_lazy_zero.load() ? 1 : 0; }
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
    int dev = 0;
    PLUQ_CUDA_TRY(cudaGetDevice(&dev));
    Ctx c;
    c.F = make_field(p);
    c.kind = kind;
    c.st = st;
    c.dev = dev;
    carve(c, L.main, m, w);
    c.cap_m = m;
    c.cap_n = n;
    c.hw = hw;
    c.leaf = leaf_size();
    // streams, events and host words of this decomposition's contexts are
    // held until it returns (then handed back to the process-wide pools)
    Ctx branch[NBRANCH];
    Streams *sbs[NBRANCH + 1] = {};
    BranchPool pool;
    struct Guard {
        Ctx *b;
        Streams **sbs;
        ~Guard()
        {
            for (int i = 0; i < NBRANCH; ++i)
                if (b[i].hw) release_words(b[i].hw);
            for (int i = 0; i <= NBRANCH; ++i) release_streams(sbs[i]);
        }
    } guard{branch, sbs};
    auto bind = [](Ctx &x, Streams *sb, bool own_stream) {
        x.side = sb->side;
        x.ev_fork = sb->fork;
        x.ev_join = sb->join;
        x.ev_done = sb->done;
        if (own_stream) x.st = sb->st;
    };
    sbs[NBRANCH] = acquire_streams();
    if (!sbs[NBRANCH]) return PLUQ_ECUDA;
    bind(c, sbs[NBRANCH], false);
    if (branches && has_branches(m, n)) {
        int i = 0;
        for (int t = 0; t < NTIER; ++t)
            for (int u = 0; u < TIER_COUNT[t]; ++u, ++i) {
                Ctx &b = branch[i];
                b.F = c.F;
                b.kind = kind;
                b.leaf = c.leaf;
                b.dev = dev;
                sbs[i] = acquire_streams();
                if (!sbs[i]) return PLUQ_ECUDA;
                bind(b, sbs[i], true);
                b.hw = acquire_words();
                if (!b.hw) return PLUQ_ECUDA;
                b.cap_m = tier_dim(m, t);
                b.cap_n = tier_dim(n, t);
                carve(b, L.branch[t], b.cap_m, w);
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
    const long long t_start = g_host_stats ? now_ns() : 0;
    const long long w0 = g_wait_ns.load(), n0 = g_waits.load(), l0 = prof::g_launches.load();
    {
        const pluq_status rs = rec(c, d_A, m, n, lda, d_perm_p, d_perm_q, res, 0, false);
        if (rs != PLUQ_OK) {
            // a kernel that gave up a bounded wait makes later steps fail too:
            // report the wait, and leave no record behind for the next call
            cudaStreamSynchronize(st);
            const int t = tc_error_flag() | leaf_error_flag();
            return t ? PLUQ_ETIMEOUT : rs;
        }
    }
    if (g_host_stats) {
        cudaStreamSynchronize(st);
        fprintf(stderr,
                "pluq host stats: %lld x %lld: wall %.3f ms, waits %lld (%.3f ms summed over "
                "threads), launches %lld\n",
                (long long)m, (long long)n, (now_ns() - t_start) / 1e6, g_waits.load() - n0,
                (g_wait_ns.load() - w0) / 1e6, prof::g_launches.load() - l0);
    }
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
    const int mode = assign ? MM_ASSIGN : MM_SUB;
    // an explicit tensor request runs the tensor-core kernel whatever the size;
    // AUTO sends small products to the CUDA cores as the recursion does
    if (mm_kind == PLUQ_MM_TENSOR)
        return launch_mm_tc(Blk{d_C, ldc}, d_A, lda, d_B, ldb, M, N, K, make_field(p), mode, 1, 0,
                            0, 0, ar, (cudaStream_t)stream);
    return launch_mm(kind, Blk{d_C, ldc}, d_A, lda, d_B, ldb, M, N, K, make_field(p), mode, 1, 0,
                     0, 0, ar, (cudaStream_t)stream);
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
    PermOp op{d_X, ldx, count, width, d_perm, 0, true};
    return launch_perm_ops(&op, 1, (uint32_t *)d_work, ws_bytes / 4, (cudaStream_t)stream);
}

pluq_status pluq_perm_cols(uint32_t *d_X, int64_t ldx, int64_t height, int64_t count,
                           const int32_t *d_perm, void *d_work, size_t ws_bytes, void *stream)
{
    if (count < 0 || height < 0) return PLUQ_EINVAL;
    if (count == 0 || height == 0) return PLUQ_OK;
    if (!d_X || !d_perm || ldx < count) return PLUQ_EINVAL;
    if (!d_work || ws_bytes < (size_t)count * height * 4) return PLUQ_ENOMEM;
    PermOp op{d_X, ldx, height, count, d_perm, 0, false};
    return launch_perm_ops(&op, 1, (uint32_t *)d_work, ws_bytes / 4, (cudaStream_t)stream);
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
