// The node kernel: one step of Algorithm 1 (Sec. 2) on a small node, its
// base cases included, in one launch (one thread block or a cluster).
#include "node_impl.cuh"

namespace pluq {
namespace {

template <bool SMALLP, int LEVEL, int NC>
__global__ void __launch_bounds__(LT, 1) node_kernel(const __grid_constant__ NodeArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LeafShared &S = *reinterpret_cast<LeafShared *>(smem_raw);
    __shared__ NodeShared NS;
    Grp<NC> g{0};
    if constexpr (NC > 1) {
        g.rank = cluster_rank();
        g.sync();   // every CTA has started before any writes another's shared memory
    }
    node_step<SMALLP, LEVEL, NC>(S, NS, a, a.A, a.m, a.n, a.perm_p, a.perm_q, a.info,
                                 a.try_generic, g);
    if constexpr (NC > 1) {
        __threadfence();
        g.sync();   // every CTA's writes are done before the result is published
    }
    if (g.rank == 0 && threadIdx.x == 0 && a.host_info) {
        a.host_info[1] = a.info[0];
        a.host_info[2] = a.info[1];
        a.host_info[3] = a.info[2];
        __threadfence_system();
        a.host_info[0] = a.seq;
    }
}

}  // namespace

pluq_status launch_node(uint32_t *A, int64_t m, int64_t n, int64_t lda, Field F, int32_t *perm_p,
                        int32_t *perm_q, int32_t *info, cudaStream_t st, volatile int32_t *host_info,
                        int32_t seq, bool try_generic, uint32_t *stage, int64_t stage_words,
                        uint32_t *icopy)
{
    if (m <= 0 || n <= 0 || m > NMAX || n > NMAX) return PLUQ_EINVAL;
    NodeArgs a{};
    a.A = A;
    a.m = (int)m;
    a.n = (int)n;
    a.lda = lda;
    a.F = F;
    a.perm_p = perm_p;
    a.perm_q = perm_q;
    a.info = info;
    a.host_info = host_info;
    a.seq = seq;
    a.stage = stage;
    a.stage_words = stage_words;
    a.icopy = icopy;
    a.wait_limit = wait_limit_or(STEP_WAIT_LIMIT);
    a.try_generic = try_generic ? 1 : 0;
    a.left_looking = g_tune_leaf_left.load(std::memory_order_relaxed) ? 1 : 0;
    const size_t smem = sizeof(LeafShared);
    const bool two = m > 2 * LM || n > 2 * LM;   // blocks larger than base cases
    const int nc = g_tune_node_ctas.load(std::memory_order_relaxed);
    prof::start(prof::LEAF, st);
#define PLUQ_NODE_CASE(SP, LV, NCV)                                                               \
    {                                                                                             \
        static std::atomic<uint64_t> attr{0};                                                     \
        if (!smem_attr_once((const void *)node_kernel<SP, LV, NCV>, smem, attr)) return PLUQ_ECUDA; \
        if (NCV == 1) {                                                                           \
            node_kernel<SP, LV, NCV><<<1, LT, smem, st>>>(a);                                     \
        } else {                                                                                  \
            cudaLaunchConfig_t cfg = {};                                                          \
            cfg.gridDim = dim3(NCV, 1, 1);                                                        \
            cfg.blockDim = dim3(LT, 1, 1);                                                        \
            cfg.dynamicSmemBytes = smem;                                                          \
            cfg.stream = st;                                                                      \
            cudaLaunchAttribute at[1];                                                            \
            at[0].id = cudaLaunchAttributeClusterDimension;                                       \
            at[0].val.clusterDim.x = NCV;                                                         \
            at[0].val.clusterDim.y = 1;                                                           \
            at[0].val.clusterDim.z = 1;                                                           \
            cfg.attrs = at;                                                                       \
            cfg.numAttrs = 1;                                                                     \
            if (cudaLaunchKernelEx(&cfg, node_kernel<SP, LV, NCV>, a) != cudaSuccess)              \
                return PLUQ_ECUDA;                                                                \
        }                                                                                         \
    }
    if (F.p <= 65536u) {
        if (nc == 8) {
            if (two) PLUQ_NODE_CASE(true, 2, 8) else PLUQ_NODE_CASE(true, 1, 8)
        } else if (nc == 4) {
            if (two) PLUQ_NODE_CASE(true, 2, 4) else PLUQ_NODE_CASE(true, 1, 4)
        } else if (nc == 2) {
            if (two) PLUQ_NODE_CASE(true, 2, 2) else PLUQ_NODE_CASE(true, 1, 2)
        } else {
            if (two) PLUQ_NODE_CASE(true, 2, 1) else PLUQ_NODE_CASE(true, 1, 1)
        }
    } else {
        if (nc == 8) {
            if (two) PLUQ_NODE_CASE(false, 2, 8) else PLUQ_NODE_CASE(false, 1, 8)
        } else if (nc == 4) {
            if (two) PLUQ_NODE_CASE(false, 2, 4) else PLUQ_NODE_CASE(false, 1, 4)
        } else if (nc == 2) {
            if (two) PLUQ_NODE_CASE(false, 2, 2) else PLUQ_NODE_CASE(false, 1, 2)
        } else {
            if (two) PLUQ_NODE_CASE(false, 2, 1) else PLUQ_NODE_CASE(false, 1, 1)
        }
    }
#undef PLUQ_NODE_CASE
    pluq_status s = last_launch();
    const double kk = (double)(m < n ? m : n);
    prof::stop(prof::LEAF, st, 2.0 * m * n * kk - (double)(m + n) * kk * kk + 2.0 / 3.0 * kk * kk * kk);
    return s;
}

int node_leaf_error_flag()
{
    int v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_leaf_error, sizeof(int)) != cudaSuccess) return 0;
    if (v) cudaMemcpyToSymbol(g_leaf_error, &z, sizeof(int));
    return v;
}

}  // namespace pluq
