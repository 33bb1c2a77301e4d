// Tensor-core modular product (placeholder until the tcgen05 kernel lands).
#include "common.cuh"

namespace pluq {

size_t mm_tc_workspace(int64_t, int64_t, int64_t, uint32_t, int64_t) { return 0; }

pluq_status launch_mm_tc(Blk, const uint32_t *, int64_t, const uint32_t *, int64_t, int64_t,
                         int64_t, int64_t, Field, int, int64_t, int64_t, int64_t, int64_t,
                         Arena &, cudaStream_t)
{
    return PLUQ_EUNSUPPORTED;
}

}  // namespace pluq
