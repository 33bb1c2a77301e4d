// Many decompositions of uneven sizes in one persistent launch (the families
// of matrices Groebner-basis elimination produces): every thread block takes
// the next matrix from a device-side counter and runs Algorithm 1 (Sec. 2) on
// it to the end, its recursion on the device (node_step, four levels above the
// base case), with no host round trip.  One launch and one memset per call, so
// the call can sit in a captured stream.
#include "node_impl.cuh"

namespace pluq {
namespace {

struct BatchArgs {
    uint32_t *const *A;
    const int64_t *m, *n, *lda;
    int32_t *const *perm_p, *const *perm_q;
    int64_t *rank;
    int64_t count, max_m, max_n;
    Field F;
    unsigned long long *next;   // matrices handed out so far
    uint32_t *stage;            // per thread block: stage_words, then icopy_words
    int64_t stage_words, icopy_words, slice_words;
    uint32_t wait_limit;
    int left_looking;
};

// dynamic shared memory: the base case's area, then the state of levels 3
// and 4 and the wide diagonal inverses
constexpr size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }
constexpr size_t OFF_L3 = al16(sizeof(LeafShared));
constexpr size_t OFF_L4 = OFF_L3 + al16(sizeof(NodeLevel<4 * LM>));
constexpr size_t OFF_DW = OFF_L4 + al16(sizeof(NodeLevel<8 * LM>));
constexpr size_t BATCH_SMEM = OFF_DW + al16(sizeof(uint32_t) * 8 * LM);

// Every thread block loops: take matrix q = next++ (in the caller's order),
// check it, factor it, write its rank or a negative status to rank[q].
template <bool SMALLP>
__global__ void __launch_bounds__(LT, 1) batch_kernel(const __grid_constant__ BatchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LeafShared &S = *reinterpret_cast<LeafShared *>(smem_raw);
    __shared__ NodeShared NS;
    __shared__ int64_t cur;
    __shared__ int32_t top_info[3];
    const int tid = threadIdx.x;
    if (tid == 0) {
        NS.l3 = reinterpret_cast<NodeLevel<4 * LM> *>(smem_raw + OFF_L3);
        NS.l4 = reinterpret_cast<NodeLevel<8 * LM> *>(smem_raw + OFF_L4);
        NS.dinv_wide = reinterpret_cast<uint32_t *>(smem_raw + OFF_DW);
    }
    const Grp<1> g{0};
    NodeArgs na{};
    na.F = a.F;
    na.stage = a.stage + (int64_t)blockIdx.x * a.slice_words;
    na.stage_words = a.stage_words;
    na.icopy = na.stage + a.stage_words;
    na.wait_limit = a.wait_limit;
    na.left_looking = a.left_looking;
    na.try_generic = 1;
    const uint32_t p = a.F.p;
    for (;;) {
        __syncthreads();   // every thread has read `cur` and the last matrix is done
        if (tid == 0) cur = (int64_t)atomicAdd(a.next, 1ull);
        __syncthreads();
        const int64_t q = cur;
        if (q >= a.count) break;
        uint32_t *A = a.A[q];
        const int64_t m = a.m[q], n = a.n[q], lda = a.lda[q];
        int32_t *pp = a.perm_p[q], *pq = a.perm_q[q];
        int64_t status;
        if (m < 0 || n < 0 || m > a.max_m || n > a.max_n || (m > 0 && !pp) || (n > 0 && !pq) ||
            (m > 0 && n > 0 && (!A || lda < n))) {
            status = PLUQ_EINVAL;
        } else if (m == 0 || n == 0) {
            for (int i = tid; i < m; i += LT) pp[i] = i;
            for (int j = tid; j < n; j += LT) pq[j] = j;
            status = 0;
        } else {
            // an entry >= p is reported before anything is written
            bool bad = false;
            for (int64_t i = tid >> 5; i < m && !bad; i += NW)
                for (int64_t j = tid & 31; j < n; j += 32) bad |= A[i * lda + j] >= p;
            if (__syncthreads_or(bad)) {
                status = PLUQ_ERANGE;
            } else {
                na.A = A;
                na.m = (int)m;
                na.n = (int)n;
                na.lda = lda;
                const int M = (int)m, N = (int)n;
                const int side = M > N ? M : N;
                if (side <= LM)
                    leaf_run_full<SMALLP>(S, A, M, N, lda, a.F, pp, pq, top_info, 1, a.wait_limit,
                                          a.left_looking);
                else if (side <= 2 * LM)
                    node_step<SMALLP, 1, 1>(S, NS, na, A, M, N, pp, pq, top_info, 1, g);
                else if (side <= 4 * LM)
                    node_step<SMALLP, 2, 1>(S, NS, na, A, M, N, pp, pq, top_info, 1, g);
                else if (side <= 8 * LM)
                    node_step<SMALLP, 3, 1>(S, NS, na, A, M, N, pp, pq, top_info, 1, g);
                else
                    node_step<SMALLP, 4, 1>(S, NS, na, A, M, N, pp, pq, top_info, 1, g);
                __syncthreads();
                status = top_info[0] < 0 ? (int64_t)PLUQ_ETIMEOUT : (int64_t)top_info[0];
            }
        }
        if (tid == 0) a.rank[q] = status;
    }
}

constexpr int64_t round_words(int64_t w) { return (w + 63) & ~(int64_t)63; }

void slice_words(int64_t max_m, int64_t max_n, int64_t &stage, int64_t &icopy, int64_t &slice)
{
    // a node's permutations stage at most three block heights of rows, each
    // padded by up to 6 words for 16-byte accesses
    stage = round_words(max_m * max_n + 24 * max_m + 64);
    icopy = round_words((max_m / 2 + 1) * (max_n / 2 + 1));
    slice = stage + icopy;
}

// default: one thread block per SM of the current device
int batch_ctas(int ctas)
{
    if (ctas > 0) return ctas;
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        return 148;
    return n;
}

}  // namespace

int batch_leaf_error_flag()
{
    int v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_leaf_error, sizeof(int)) != cudaSuccess) return 0;
    if (v) cudaMemcpyToSymbol(g_leaf_error, &z, sizeof(int));
    return v;
}

}  // namespace pluq

using namespace pluq;

extern "C" {

pluq_status pluq_batched_persistent_workspace_size(int64_t max_m, int64_t max_n, int ctas,
                                                   size_t *h_bytes)
{
    if (!h_bytes || max_m < 0 || max_n < 0 || max_m > BMAX || max_n > BMAX || ctas < 0)
        return PLUQ_EINVAL;
    int64_t st, ic, sl;
    slice_words(max_m, max_n, st, ic, sl);
    *h_bytes = 256 + (size_t)batch_ctas(ctas) * (size_t)sl * sizeof(uint32_t);
    return PLUQ_OK;
}

pluq_status pluq_mod_p_batched_persistent(uint32_t *const *d_A, const int64_t *d_m,
                                          const int64_t *d_n, const int64_t *d_lda, int64_t count,
                                          int64_t max_m, int64_t max_n, uint32_t p,
                                          int32_t *const *d_perm_p, int32_t *const *d_perm_q,
                                          int64_t *d_rank, void *d_work, size_t ws_bytes, int ctas,
                                          void *stream)
{
    if (count < 0 || ctas < 0 || max_m < 0 || max_n < 0 || max_m > BMAX || max_n > BMAX)
        return PLUQ_EINVAL;
    if (p >= 0x80000000u || !is_prime_u32(p)) return PLUQ_ENOTPRIME;
    if (count == 0) return PLUQ_OK;
    if (!d_A || !d_m || !d_n || !d_lda || !d_perm_p || !d_perm_q || !d_rank) return PLUQ_EINVAL;
    size_t need = 0;
    PLUQ_TRY(pluq_batched_persistent_workspace_size(max_m, max_n, ctas, &need));
    if (!d_work || ws_bytes < need) return PLUQ_ENOMEM;
    if ((uintptr_t)d_work & 15) return PLUQ_EINVAL;
    const int nb = (int)std::min<int64_t>(batch_ctas(ctas), count);
    cudaStream_t st = (cudaStream_t)stream;
    BatchArgs a{};
    a.A = d_A;
    a.m = d_m;
    a.n = d_n;
    a.lda = d_lda;
    a.perm_p = d_perm_p;
    a.perm_q = d_perm_q;
    a.rank = d_rank;
    a.count = count;
    a.max_m = max_m;
    a.max_n = max_n;
    a.F = make_field(p);
    a.next = (unsigned long long *)d_work;
    a.stage = (uint32_t *)((char *)d_work + 256);
    slice_words(max_m, max_n, a.stage_words, a.icopy_words, a.slice_words);
    a.wait_limit = wait_limit_or(STEP_WAIT_LIMIT);
    a.left_looking = g_tune_leaf_left.load(std::memory_order_relaxed) ? 1 : 0;
    PLUQ_CUDA_TRY(cudaMemsetAsync(d_work, 0, sizeof(unsigned long long), st));
    if (p <= 65536u) {
        static std::atomic<uint64_t> attr{0};
        if (!smem_attr_once((const void *)batch_kernel<true>, BATCH_SMEM, attr)) return PLUQ_ECUDA;
        batch_kernel<true><<<nb, LT, BATCH_SMEM, st>>>(a);
    } else {
        static std::atomic<uint64_t> attr{0};
        if (!smem_attr_once((const void *)batch_kernel<false>, BATCH_SMEM, attr)) return PLUQ_ECUDA;
        batch_kernel<false><<<nb, LT, BATCH_SMEM, st>>>(a);
    }
    return last_launch();
}

}  // extern "C"
