// Base case of Algorithm 1 (Sec. 2) on a block of at most 128 x 128, one
// thread block, the block resident in shared memory: the kernel and its
// launch.  The algorithm itself (three phases, the generic blocked path) is in
// leaf_impl.cuh.
#include "leaf_impl.cuh"

namespace pluq {
namespace {

template <bool SMALLP, int CPL, int RPW>
__global__ void __launch_bounds__(LT) leaf_kernel(uint32_t *__restrict__ A, int m, int n,
                                                  int64_t lda, Field F, int32_t *perm_p_out,
                                                  int32_t *perm_q_out, int32_t *info_out,
                                                  int info_len, volatile int32_t *host_info,
                                                  int32_t seq, int try_generic, uint32_t wait_limit,
                                                  int left_looking)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LeafShared &S = *reinterpret_cast<LeafShared *>(smem_raw);
    leaf_run<SMALLP, CPL, RPW>(S, A, m, n, lda, F, perm_p_out, perm_q_out, info_out, info_len,
                               host_info, seq, try_generic, wait_limit, left_looking);
}

}  // namespace

pluq_status launch_leaf(uint32_t *A, int64_t m, int64_t n, int64_t lda, Field F, int32_t *perm_p,
                        int32_t *perm_q, int32_t *info, int info_len, cudaStream_t st,
                        volatile int32_t *host_info, int32_t seq, bool try_generic)
{
    if (m < 0 || n < 0 || m > LM || n > LM) return PLUQ_EINVAL;
    if (m == 0 || n == 0) {
        // empty block: r = 0, identity permutations
        if (m) PLUQ_TRY(launch_iota(perm_p, m, st));
        if (n) PLUQ_TRY(launch_iota(perm_q, n, st));
        PLUQ_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t), st));
        return PLUQ_OK;
    }
    const size_t smem = sizeof(LeafShared);
    const int cpl = n <= 32 ? 1 : n <= 64 ? 2 : 4;
    const int rpw = m <= 32 ? 2 : m <= 64 ? 4 : 8;
    const bool small = F.p <= 65536u;
    const uint32_t wlim = wait_limit_or(STEP_WAIT_LIMIT);
    const int lvar = g_tune_leaf_left.load(std::memory_order_relaxed) ? 1 : 0;
    prof::start(prof::LEAF, st);
#define PLUQ_LEAF_CASE(SP, C, R)                                                                  \
    if (small == SP && cpl == C && rpw == R) {                                                   \
        static std::atomic<uint64_t> attr{0};                                                    \
        if (!smem_attr_once((const void *)leaf_kernel<SP, C, R>, smem, attr)) return PLUQ_ECUDA;  \
        leaf_kernel<SP, C, R><<<1, LT, smem, st>>>(A, (int)m, (int)n, lda, F, perm_p, perm_q,    \
                                                   info, info_len, host_info, seq,               \
                                                   try_generic ? 1 : 0, wlim, lvar);             \
    }
    PLUQ_LEAF_CASE(true, 1, 2) PLUQ_LEAF_CASE(true, 1, 4) PLUQ_LEAF_CASE(true, 1, 8)
    PLUQ_LEAF_CASE(true, 2, 2) PLUQ_LEAF_CASE(true, 2, 4) PLUQ_LEAF_CASE(true, 2, 8)
    PLUQ_LEAF_CASE(true, 4, 2) PLUQ_LEAF_CASE(true, 4, 4) PLUQ_LEAF_CASE(true, 4, 8)
    PLUQ_LEAF_CASE(false, 1, 2) PLUQ_LEAF_CASE(false, 1, 4) PLUQ_LEAF_CASE(false, 1, 8)
    PLUQ_LEAF_CASE(false, 2, 2) PLUQ_LEAF_CASE(false, 2, 4) PLUQ_LEAF_CASE(false, 2, 8)
    PLUQ_LEAF_CASE(false, 4, 2) PLUQ_LEAF_CASE(false, 4, 4) PLUQ_LEAF_CASE(false, 4, 8)
#undef PLUQ_LEAF_CASE
    pluq_status s = last_launch();
    // algorithmic work: the field operations of eliminating the block at full
    // rank, 2 m n k - (m + n) k^2 + 2/3 k^3 with k = min(m, n)
    const double k = (double)(m < n ? m : n);
    prof::stop(prof::LEAF, st, 2.0 * m * n * k - (double)(m + n) * k * k + 2.0 / 3.0 * k * k * k);
    return s;
}

int leaf_error_flag()
{
    int v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_leaf_error, sizeof(int)) != cudaSuccess) return 0;
    if (v) cudaMemcpyToSymbol(g_leaf_error, &z, sizeof(int));
    return v | node_leaf_error_flag() | batch_leaf_error_flag();
}

}  // namespace pluq
