// Data movement of Algorithm 1 (Sec. 2): PermR / PermC on blocks, the final
// block permutations S and T, composition of P and Q from the four recursive
// calls, and the rank-profile read-outs of Sec. 4.  All HBM-bound: each
// element is read once and written once per pass, rows are walked with
// consecutive threads on consecutive 16-byte chunks (coalesced, vectorised).
#include <algorithm>

#include "common.cuh"

namespace pluq {
namespace {

constexpr int GT = 256;      // threads per block
constexpr int GC = 4 * GT;   // columns per block

// Elements by which a row-major uint32 block sits past a 16-byte boundary;
// chunks of four columns follow the global addresses, so column j of the
// block lies in chunk (j + a) / 4 of its row.
__host__ __device__ __forceinline__ int misalign(const uint32_t *X)
{
    return (int)(((uintptr_t)X >> 2) & 3);
}

// dst[i][j] = src[rmap ? rmap[i] - moff : i][cmap ? cmap[j] - moff : j].
// `a` is dst's misalignment; with `vec` (16-byte row strides, and src sharing
// dst's misalignment unless its columns are gathered) whole chunks move as
// uint4, the partial chunks at the ends of a row element by element.
__global__ void move_kernel(uint32_t *__restrict__ dst, int64_t ldd, const uint32_t *__restrict__ src,
                            int64_t lds, int64_t rows, int64_t cols, const int32_t *__restrict__ rmap,
                            const int32_t *__restrict__ cmap, int32_t moff, int a, int vec)
{
    const int64_t nq = (cols + a + 3) / 4;
    const int64_t c0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cstep = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) {
        const int64_t si = rmap ? (int64_t)(rmap[i] - moff) : i;
        const uint32_t *sr = src + si * lds;
        uint32_t *dr = dst + i * ldd;
        for (int64_t c = c0; c < nq; c += cstep) {
            const int64_t j = 4 * c - a;
            if (vec && j >= 0 && j + 4 <= cols) {
                uint4 v;
                if (cmap) {
                    v.x = sr[cmap[j] - moff];
                    v.y = sr[cmap[j + 1] - moff];
                    v.z = sr[cmap[j + 2] - moff];
                    v.w = sr[cmap[j + 3] - moff];
                } else {
                    v = *(const uint4 *)(sr + j);
                }
                *(uint4 *)(dr + j) = v;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int64_t jj = j + e;
                    if (jj >= 0 && jj < cols) dr[jj] = sr[cmap ? (int64_t)(cmap[jj] - moff) : jj];
                }
            }
        }
    }
}

// ------------------------------------------------- in-place permutations --
// PermR / PermC in place, in one pass, several disjoint blocks per launch.
//  by_rows: a thread block owns a stripe of W columns (W a multiple of 4) of
//           every row of its block, stages it in shared memory and writes row
//           i back from staged row map[i] - moff;
//  by cols: a thread block owns W whole rows, stages them and writes column j
//           from staged column map[j] - moff.
// Everything a thread block writes it has read itself first, and the stripes
// (row groups) of a block are disjoint, so no other thread block reads what
// it overwrites.
struct PTask {
    uint32_t *X;
    int64_t ld;
    int32_t rows, cols;
    const int32_t *map;
    int32_t moff;
    int32_t by_rows;
    int32_t W;
    int32_t nblk;
};
constexpr int PT_MAX = 4;
constexpr int PT_THREADS = 256;
constexpr int PB_LOADS = 4;     // 16-byte loads a thread keeps in flight
struct PTasks {
    PTask t[PT_MAX];
    int n;
};

__global__ void __launch_bounds__(PT_THREADS) perm_inplace_kernel(const __grid_constant__ PTasks ts)
{
    extern __shared__ __align__(16) uint32_t sh[];
    int b = blockIdx.x, ti = 0;
    while (ti < ts.n - 1 && b >= ts.t[ti].nblk) {
        b -= ts.t[ti].nblk;
        ++ti;
    }
    const PTask &t = ts.t[ti];
    const bool vec = (t.ld & 3) == 0;
    const int a = vec ? misalign(t.X) : 0;
    const int rows = t.rows, cols = t.cols, W = t.W;
    if (t.by_rows) {
        const int c0 = b * W - a;        // first column of the stripe (chunk aligned)
        const int nq = W / 4;
        const int tot = rows * nq;
        // batches of PB_LOADS chunks per thread: all loads of a batch in flight
        // before their shared-memory stores
        for (int q0 = threadIdx.x; q0 < tot; q0 += PT_THREADS * PB_LOADS) {
            uint4 v[PB_LOADS];
#pragma unroll
            for (int u = 0; u < PB_LOADS; ++u) {
                const int q = q0 + u * PT_THREADS;
                if (q >= tot) break;
                const int i = q / nq, c = q - i * nq, j = c0 + 4 * c;
                const uint32_t *sr = t.X + (int64_t)(t.map[i] - t.moff) * t.ld;
                if (vec && j >= 0 && j + 4 <= cols) {
                    v[u] = *(const uint4 *)(sr + j);
                } else {
                    uint32_t e4[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (j + e >= 0 && j + e < cols) e4[e] = sr[j + e];
                    v[u] = make_uint4(e4[0], e4[1], e4[2], e4[3]);
                }
            }
#pragma unroll
            for (int u = 0; u < PB_LOADS; ++u) {
                const int q = q0 + u * PT_THREADS;
                if (q >= tot) break;
                const int i = q / nq, c = q - i * nq;
                *(uint4 *)(sh + i * W + 4 * c) = v[u];
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < tot; q += PT_THREADS) {
            const int i = q / nq, c = q - i * nq, j = c0 + 4 * c;
            uint32_t *dr = t.X + (int64_t)i * t.ld;
            const uint32_t *sv = sh + i * W + 4 * c;
            if (vec && j >= 0 && j + 4 <= cols) {
                *(uint4 *)(dr + j) = *(const uint4 *)sv;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (j + e >= 0 && j + e < cols) dr[j + e] = sv[e];
            }
        }
    } else {
        const int i0 = b * W;
        const int nr = min(W, rows - i0);
        const int cs = (cols + a + 3) & ~3;   // staged row: element j at a + j
        const int nq = cs / 4;
        const int tot = nr * nq;
        for (int q0 = threadIdx.x; q0 < tot; q0 += PT_THREADS * PB_LOADS) {
            uint4 v[PB_LOADS];
#pragma unroll
            for (int u = 0; u < PB_LOADS; ++u) {
                const int q = q0 + u * PT_THREADS;
                if (q >= tot) break;
                const int i = q / nq, c = q - i * nq, j = 4 * c - a;
                const uint32_t *sr = t.X + (int64_t)(i0 + i) * t.ld;
                if (vec && j >= 0 && j + 4 <= cols) {
                    v[u] = *(const uint4 *)(sr + j);
                } else {
                    uint32_t e4[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (j + e >= 0 && j + e < cols) e4[e] = sr[j + e];
                    v[u] = make_uint4(e4[0], e4[1], e4[2], e4[3]);
                }
            }
#pragma unroll
            for (int u = 0; u < PB_LOADS; ++u) {
                const int q = q0 + u * PT_THREADS;
                if (q >= tot) break;
                const int i = q / nq, c = q - i * nq;
                *(uint4 *)(sh + i * cs + 4 * c) = v[u];
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < tot; q += PT_THREADS) {
            const int i = q / nq, c = q - i * nq, j = 4 * c - a;
            uint32_t *dr = t.X + (int64_t)(i0 + i) * t.ld;
            const uint32_t *srow = sh + i * cs + a;
            if (vec && j >= 0 && j + 4 <= cols) {
                uint4 v;
                v.x = srow[t.map[j] - t.moff];
                v.y = srow[t.map[j + 1] - t.moff];
                v.z = srow[t.map[j + 2] - t.moff];
                v.w = srow[t.map[j + 3] - t.moff];
                *(uint4 *)(dr + j) = v;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (j + e >= 0 && j + e < cols) dr[j + e] = srow[t.map[j + e] - t.moff];
            }
        }
    }
}

__global__ void fill_kernel(uint32_t *__restrict__ dst, int64_t ldd, int64_t rows, int64_t cols,
                            uint32_t v)
{
    const int64_t c0 = (int64_t)blockIdx.x * GC + threadIdx.x;
    for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int64_t j = c0 + (int64_t)s * GT;
            if (j < cols) dst[i * ldd + j] = v;
        }
    }
}

// Algorithm 1, final step: P = Diag(P1 diag(I,P2), P3 diag(I,P4)) S and
// Q = T Diag(diag(I,Q3) Q1, diag(I,Q4) Q2), with the row map of S and column
// map of T written out for the S^T A T^T pass.  A null sub-permutation is the
// identity (its recursive call had an empty block).
struct ComposeArgs {
    const int32_t *p1, *p2, *p3, *p4, *q1, *q2, *q3, *q4;
    int32_t *p, *q, *smap, *tmap;
    int64_t m, n, k, h, r1, r2, r3, r4;
};

__device__ __forceinline__ int32_t idx_or(const int32_t *v, int64_t i)
{
    return v ? v[i] : (int32_t)i;
}

__global__ void compose_kernel(ComposeArgs a)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.m) {
        const int64_t i = t;
        // S: [0, r1+r2) | [k, k+r3+r4) | [r1+r2, k) | [k+r3+r4, m)
        int64_t s;
        const int64_t top = a.r1 + a.r2, bot = a.r3 + a.r4;
        if (i < top) s = i;
        else if (i < top + bot) s = a.k + (i - top);
        else if (i < a.k + bot) s = i - bot;
        else s = i;
        a.smap[i] = (int32_t)s;
        int32_t d;
        if (s < a.k) {
            d = s < a.r1 ? idx_or(a.p1, s) : idx_or(a.p1, a.r1 + idx_or(a.p2, s - a.r1));
        } else {
            int64_t u = s - a.k;
            d = (int32_t)a.k + (u < a.r3 ? idx_or(a.p3, u) : idx_or(a.p3, a.r3 + idx_or(a.p4, u - a.r3)));
        }
        a.p[i] = d;
    }
    if (t < a.n) {
        const int64_t j = t;
        // T: [0,r1) | [h,h+r2) | [r1,r1+r3) | [h+r2,h+r2+r4) | [r1+r3,h) | [h+r2+r4,n)
        int64_t c;
        const int64_t r1 = a.r1, r2 = a.r2, r3 = a.r3, r4 = a.r4, h = a.h;
        if (j < r1) c = j;
        else if (j < r1 + r2) c = h + (j - r1);
        else if (j < r1 + r2 + r3) c = r1 + (j - r1 - r2);
        else if (j < r1 + r2 + r3 + r4) c = h + r2 + (j - r1 - r2 - r3);
        else if (j < h + r2 + r4) c = r1 + r3 + (j - r1 - r2 - r3 - r4);
        else c = j;
        a.tmap[j] = (int32_t)c;
        int32_t d;
        if (c < h) {
            d = c < r1 ? idx_or(a.q1, c) : idx_or(a.q1, r1 + idx_or(a.q3, c - r1));
        } else {
            int64_t u = c - h;
            d = (int32_t)h + (u < r2 ? idx_or(a.q2, u) : idx_or(a.q2, r2 + idx_or(a.q4, u - r2)));
        }
        a.q[j] = d;
    }
}

__global__ void iota_kernel(int32_t *v, int64_t n)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) v[t] = (int32_t)t;
}

// Sorted read-out without scratch: the position of pivot t is the number of
// pivots with a smaller key (keys are distinct row / column indices).
__global__ void rank_sort_kernel(const int32_t *__restrict__ key, const int32_t *__restrict__ val,
                                 int64_t r, int32_t *__restrict__ out_key,
                                 int32_t *__restrict__ out_val)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= r) return;
    const int32_t kt = key[t];
    int64_t pos = 0;
    for (int64_t u = 0; u < r; ++u) pos += key[u] < kt;
    out_key[pos] = kt;
    if (out_val) out_val[pos] = val[t];
}

__global__ void check_range_kernel(const uint32_t *__restrict__ A, int64_t lda, int64_t m,
                                   int64_t n, uint32_t p, int32_t *flag)
{
    const int64_t c0 = (int64_t)blockIdx.x * GC + threadIdx.x;
    for (int64_t i = blockIdx.y; i < m; i += gridDim.y)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int64_t j = c0 + (int64_t)s * GT;
            if (j < n && A[i * lda + j] >= p) atomicExch(flag, 1);
        }
}

// Factor read-out from the packed [L\U V; M 0] (Sec. 2): `lower` writes the
// rows x r unit lower trapezoid [L; M] (ones on the diagonal, zeros above),
// otherwise the r x cols upper trapezoid [U V] (zeros below the diagonal).
__global__ void extract_kernel(const uint32_t *__restrict__ LU, int64_t lda, int64_t rows,
                               int64_t cols, uint32_t *__restrict__ X, int64_t ldx, int lower)
{
    const int64_t c0 = (int64_t)blockIdx.x * GC + threadIdx.x;
    for (int64_t i = blockIdx.y; i < rows; i += gridDim.y)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int64_t j = c0 + (int64_t)s * GT;
            if (j >= cols) continue;
            uint32_t v;
            if (lower) v = j < i ? LU[i * lda + j] : (j == i ? 1u : 0u);
            else v = j >= i ? LU[i * lda + j] : 0u;
            X[i * ldx + j] = v;
        }
}

// inv[perm[i]] = i (entries of perm outside [0, n) are skipped)
__global__ void inverse_perm_kernel(const int32_t *__restrict__ perm, int64_t n,
                                    int32_t *__restrict__ inv)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t v = (uint32_t)perm[i];
    if (v < n) inv[v] = (int32_t)i;
}

// LEU read-out (Corollary of the triangularity theorem, Sec. 3), in original
// row / column indices.  lower: Lbar (m x m) = P [L 0; M I] P^T, entry (a, b)
// taken at packed position (inv[a], inv[b]); otherwise Ubar (n x n) =
// Q^T [U V; 0 0] Q, likewise.  LU is read only at positions inside the block,
// whatever inv holds.
__global__ void leu_kernel(const uint32_t *__restrict__ LU, int64_t lda, int64_t dim, int64_t r,
                           const int32_t *__restrict__ inv, uint32_t *__restrict__ X, int64_t ldx,
                           int lower)
{
    const int64_t c0 = (int64_t)blockIdx.x * GC + threadIdx.x;
    for (int64_t a = blockIdx.y; a < dim; a += gridDim.y) {
        const int64_t i = (uint32_t)inv[a];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int64_t b = c0 + (int64_t)s * GT;
            if (b >= dim) continue;
            const int64_t j = (uint32_t)inv[b];
            uint32_t v;
            if (lower) v = i == j ? 1u : ((j < r && i > j && i < dim) ? LU[i * lda + j] : 0u);
            else v = (i < r && j >= i && j < dim) ? LU[i * lda + j] : 0u;
            X[a * ldx + b] = v;
        }
    }
}

// Rank profiles of the leading k x t submatrix (Corollary of Lemma 2, Sec. 4):
// the ones of R inside [0, k) x [0, t) are the pivots i < r with
// perm_p[i] < k and perm_q[i] < t.  Each selected pivot finds its place among
// the selected ones by counting smaller rows (columns); *count gets their number.
__global__ void leading_profile_kernel(const int32_t *__restrict__ pp, const int32_t *__restrict__ pq,
                                       int64_t r, int64_t k, int64_t t, int32_t *__restrict__ rows,
                                       int32_t *__restrict__ cols, int32_t *count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r) return;
    const int32_t ri = pp[i], ci = pq[i];
    if (ri >= k || ci >= t) return;
    int64_t pr = 0, pc = 0;
    for (int64_t u = 0; u < r; ++u) {
        const int32_t ru = pp[u], cu = pq[u];
        if (ru < k && cu < t) {
            pr += ru < ri;
            pc += cu < ci;
        }
    }
    rows[pr] = ri;
    cols[pc] = ci;
    atomicAdd(count, 1);
}

// Any nonzero in the m x n block?  Blocks OR their finding into words[0] and
// count themselves in words[1]; the last block publishes the answer to the
// mapped host words (flag, then sequence number) and clears both counters.
__global__ void any_nonzero_kernel(const uint32_t *__restrict__ A, int64_t lda, int64_t m,
                                   int64_t n, int32_t *words, volatile int32_t *host, int32_t seq)
{
    const int64_t c0 = (int64_t)blockIdx.x * GC + threadIdx.x;
    bool nz = false;
    for (int64_t i = blockIdx.y; i < m && !nz; i += gridDim.y)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int64_t j = c0 + (int64_t)s * GT;
            if (j < n && A[i * lda + j] != 0) nz = true;
        }
    if (__syncthreads_or(nz) && threadIdx.x == 0) atomicOr(&words[0], 1);
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned total = gridDim.x * gridDim.y;
        if ((unsigned)atomicAdd(&words[1], 1) == total - 1) {
            const int32_t f = atomicOr(&words[0], 0);
            words[0] = 0;
            words[1] = 0;
            host[1] = f;
            __threadfence_system();
            host[0] = seq;
        }
    }
}

dim3 grid2d(int64_t rows, int64_t cols)
{
    int64_t gy = rows < 65535 ? rows : 65535;
    return dim3((unsigned)ceil_div(cols, GC), (unsigned)(gy > 0 ? gy : 1));
}

}  // namespace

namespace {
pluq_status launch_move(Blk dst, const uint32_t *src, int64_t lds, int64_t rows, int64_t cols,
                        const int32_t *rmap, const int32_t *cmap, int32_t moff, cudaStream_t st)
{
    if (rows <= 0 || cols <= 0) return PLUQ_OK;
    const int a = misalign(dst.ptr);
    const bool vec = (dst.ld & 3) == 0 && (cmap || ((lds & 3) == 0 && misalign(src) == a));
    const int64_t nq = (cols + a + 3) / 4;
    // a row of thread blocks spans a row; 1024 of them stride over the rows
    const int64_t gx = ceil_div(nq, GT);
    const int64_t gy = std::min<int64_t>(rows, 1024);
    prof::start(prof::MOVE, st);
    move_kernel<<<dim3((unsigned)gx, (unsigned)gy), GT, 0, st>>>(dst.ptr, dst.ld, src, lds, rows,
                                                                 cols, rmap, cmap, moff, a,
                                                                 vec ? 1 : 0);
    pluq_status s = last_launch();
    prof::stop(prof::MOVE, st, (double)rows * cols * 8.0);
    return s;
}

constexpr size_t PERM_SMEM_MAX = 200 * 1024;    // largest staging area of one thread block
constexpr size_t PERM_SMEM_GOAL = 96 * 1024;    // preferred: two thread blocks per SM
constexpr size_t PERM_INPLACE_ROWS_MAX = 16u << 20;   // bytes of the largest PermR staged in place

// Thread-block plan of one in-place op; false when its staging does not fit.
bool plan_inplace(const PermOp &op, PTask &t, size_t &smem)
{
    if (op.rows > (1 << 30) || op.cols > (1 << 30)) return false;
    const bool vec = (op.ld & 3) == 0;
    const int a = vec ? misalign(op.X) : 0;
    t.X = op.X;
    t.ld = op.ld;
    t.rows = (int32_t)op.rows;
    t.cols = (int32_t)op.cols;
    t.map = op.map;
    t.moff = op.moff;
    t.by_rows = op.by_rows ? 1 : 0;
    if (op.by_rows) {
        // a column stripe reads each row in 16- to 64-byte pieces 4 rows*ld
        // apart, which DRAM serves at well under the copy rate: large blocks go
        // through the scratch instead, whole rows at a time (measured on a
        // 16384^2 matrix: 1.5 TB/s staged in place, 2.9 TB/s through scratch)
        if ((size_t)op.rows * op.cols * 4 > PERM_INPLACE_ROWS_MAX) return false;
        int W = 0;
        for (int w : {16, 8, 4})
            if ((size_t)op.rows * w * 4 <= PERM_SMEM_GOAL) { W = w; break; }
        if (!W && (size_t)op.rows * 16 <= PERM_SMEM_MAX) W = 4;
        if (!W) return false;
        t.W = W;
        t.nblk = (int32_t)ceil_div(op.cols + a, W);
        smem = (size_t)op.rows * W * 4;
    } else {
        const size_t row_bytes = (size_t)((op.cols + a + 3) & ~3ll) * 4;
        if (row_bytes > PERM_SMEM_MAX) return false;
        int64_t R = (int64_t)(PERM_SMEM_GOAL / row_bytes);
        R = std::max<int64_t>(1, std::min<int64_t>(R, 16));
        R = std::min<int64_t>(R, op.rows);
        t.W = (int32_t)R;
        t.nblk = (int32_t)ceil_div(op.rows, R);
        smem = (size_t)R * row_bytes;
    }
    return true;
}
}  // namespace

pluq_status launch_gather(Blk dst, const uint32_t *src, int64_t lds, int64_t rows, int64_t cols,
                          const int32_t *rmap, const int32_t *cmap, cudaStream_t st)
{
    return launch_move(dst, src, lds, rows, cols, rmap, cmap, 0, st);
}

pluq_status launch_copy(Blk dst, const uint32_t *src, int64_t lds, int64_t rows, int64_t cols,
                        cudaStream_t st)
{
    return launch_move(dst, src, lds, rows, cols, nullptr, nullptr, 0, st);
}

pluq_status launch_perm_ops(const PermOp *ops, int count, uint32_t *scratch, size_t scratch_elems,
                            cudaStream_t st)
{
    PTasks ts{};
    size_t smem = 0;
    double bytes = 0;
    for (int i = 0; i < count; ++i) {
        const PermOp &op = ops[i];
        if (op.rows <= 0 || op.cols <= 0 || !op.map) continue;
        PTask t{};
        size_t need = 0;
        if (ts.n < PT_MAX && plan_inplace(op, t, need)) {
            ts.t[ts.n++] = t;
            smem = std::max(smem, need);
            bytes += (double)op.rows * op.cols * 8.0;
            continue;
        }
        // through the scratch: gather there (with the block's misalignment, so
        // both passes move whole chunks), then copy back
        int a = misalign(op.X);
        int64_t ldd = (op.cols + a + 3) & ~3ll;
        if ((size_t)(op.rows * ldd + a) > scratch_elems) {
            a = 0;                         // tight layout: the same moves, element by element
            ldd = op.cols;
        }
        if ((size_t)(op.rows * ldd + a) > scratch_elems) return PLUQ_ENOMEM;
        uint32_t *tmp = scratch + a;
        PLUQ_TRY(launch_move(Blk{tmp, ldd}, op.X, op.ld, op.rows, op.cols,
                             op.by_rows ? op.map : nullptr, op.by_rows ? nullptr : op.map, op.moff,
                             st));
        PLUQ_TRY(launch_move(Blk{op.X, op.ld}, tmp, ldd, op.rows, op.cols, nullptr, nullptr, 0, st));
    }
    if (ts.n == 0) return PLUQ_OK;
    int64_t blocks = 0;
    for (int i = 0; i < ts.n; ++i) blocks += ts.t[i].nblk;
    if (blocks > INT32_MAX) return PLUQ_EINVAL;
    static std::atomic<uint64_t> attr{0};
    if (!smem_attr_once((const void *)perm_inplace_kernel, PERM_SMEM_MAX, attr)) return PLUQ_ECUDA;
    prof::start(prof::MOVE, st);
    perm_inplace_kernel<<<(unsigned)blocks, PT_THREADS, smem, st>>>(ts);
    pluq_status s = last_launch();
    prof::stop(prof::MOVE, st, bytes);
    return s;
}

pluq_status launch_zero(Blk dst, int64_t rows, int64_t cols, cudaStream_t st)
{
    if (rows <= 0 || cols <= 0) return PLUQ_OK;
    fill_kernel<<<grid2d(rows, cols), GT, 0, st>>>(dst.ptr, dst.ld, rows, cols, 0u);
    return last_launch();
}

pluq_status launch_iota(int32_t *v, int64_t n, cudaStream_t st)
{
    if (n <= 0) return PLUQ_OK;
    iota_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(v, n);
    return last_launch();
}

pluq_status launch_compose(const int32_t *p1, const int32_t *p2, const int32_t *p3,
                           const int32_t *p4, const int32_t *q1, const int32_t *q2,
                           const int32_t *q3, const int32_t *q4, int32_t *p, int32_t *q,
                           int32_t *smap, int32_t *tmap, int64_t m, int64_t n, int64_t k,
                           int64_t h, int64_t r1, int64_t r2, int64_t r3, int64_t r4,
                           cudaStream_t st)
{
    ComposeArgs a{p1, p2, p3, p4, q1, q2, q3, q4, p, q, smap, tmap, m, n, k, h, r1, r2, r3, r4};
    int64_t len = m > n ? m : n;
    if (len <= 0) return PLUQ_OK;
    compose_kernel<<<(unsigned)ceil_div(len, 256), 256, 0, st>>>(a);
    return last_launch();
}

pluq_status launch_rank_sort(const int32_t *key, const int32_t *val, int64_t r, int32_t *out_key,
                             int32_t *out_val, cudaStream_t st)
{
    if (r <= 0) return PLUQ_OK;
    rank_sort_kernel<<<(unsigned)ceil_div(r, 256), 256, 0, st>>>(key, val, r, out_key, out_val);
    return last_launch();
}

pluq_status launch_extract(const uint32_t *LU, int64_t lda, int64_t rows, int64_t cols,
                           uint32_t *X, int64_t ldx, bool lower, cudaStream_t st)
{
    if (rows <= 0 || cols <= 0) return PLUQ_OK;
    extract_kernel<<<grid2d(rows, cols), GT, 0, st>>>(LU, lda, rows, cols, X, ldx, lower ? 1 : 0);
    return last_launch();
}

pluq_status launch_leu(const uint32_t *LU, int64_t lda, int64_t m, int64_t n, int64_t r,
                       const int32_t *perm_p, const int32_t *perm_q, uint32_t *Lbar, int64_t ldl,
                       uint32_t *Ubar, int64_t ldu, int32_t *work, cudaStream_t st)
{
    if (Lbar && m > 0) {
        inverse_perm_kernel<<<(unsigned)ceil_div(m, 256), 256, 0, st>>>(perm_p, m, work);
        PLUQ_TRY(last_launch());
        leu_kernel<<<grid2d(m, m), GT, 0, st>>>(LU, lda, m, r, work, Lbar, ldl, 1);
        PLUQ_TRY(last_launch());
    }
    if (Ubar && n > 0) {
        inverse_perm_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(perm_q, n, work + m);
        PLUQ_TRY(last_launch());
        leu_kernel<<<grid2d(n, n), GT, 0, st>>>(LU, lda, n, r, work + m, Ubar, ldu, 0);
        PLUQ_TRY(last_launch());
    }
    return PLUQ_OK;
}

pluq_status launch_leading_profile(const int32_t *pp, const int32_t *pq, int64_t r, int64_t k,
                                   int64_t t, int32_t *rows, int32_t *cols, int32_t *count,
                                   cudaStream_t st)
{
    PLUQ_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int32_t), st));
    if (r <= 0) return PLUQ_OK;
    leading_profile_kernel<<<(unsigned)ceil_div(r, 256), 256, 0, st>>>(pp, pq, r, k, t, rows,
                                                                      cols, count);
    return last_launch();
}

pluq_status launch_check_range(const uint32_t *A, int64_t lda, int64_t m, int64_t n, uint32_t p,
                               int32_t *flag, cudaStream_t st)
{
    if (m <= 0 || n <= 0) return PLUQ_OK;
    check_range_kernel<<<grid2d(m, n), GT, 0, st>>>(A, lda, m, n, p, flag);
    return last_launch();
}

}  // namespace pluq

namespace pluq {
pluq_status launch_any_nonzero(const uint32_t *A, int64_t lda, int64_t m, int64_t n, int32_t *words,
                               volatile int32_t *host, int32_t seq, cudaStream_t st)
{
    int64_t gy = m < 1024 ? m : 1024;
    dim3 grid((unsigned)ceil_div(n, GC), (unsigned)(gy > 0 ? gy : 1));
    any_nonzero_kernel<<<grid, GT, 0, st>>>(A, lda, m, n, words, host, seq);
    return last_launch();
}
}  // namespace pluq
