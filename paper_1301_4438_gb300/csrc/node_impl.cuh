#pragma once
// One step of Algorithm 1 (Sec. 2) on a node, its base cases included, run
// by one thread block or a cluster: the device code of the node kernel
// (node.cu) and of the persistent batch kernel (batch.cu).  Internal
// linkage, like leaf_impl.cuh: each translation unit holds its own copy.
#include "leaf_impl.cuh"

namespace pluq {
namespace {

// ------------------------------------------------------------ node kernel --
// One step of Algorithm 1 on a node whose four blocks A1, F, G, R are base
// cases (both sides at most twice the leaf size), run by one thread block or
// a cluster of two to eight: the leaves through leaf_run, the permutations, triangular
// solves and products between them by all threads on data that stays in L2.
// It replaces a dozen launches and four host round trips by one of each,
// which pays where the blocks have few pivots (deep in a rank-deficient
// matrix); the host uses it only below rank-deficient nodes.  In a cluster, F
// and G (independent, Sec. 2) run at once on the two blocks.  Each phase ends
// with a barrier over all the node's threads, so it sees the previous one
// complete.

constexpr int NMAX = 4 * LM;   // largest node side of the node kernel (two levels above the leaves)
constexpr int BMAX = 16 * LM;  // largest matrix side of the batch kernel (four levels)
constexpr int SMW = 16384;     // words of the base case's staging area a product borrows
static_assert(SMW <= LM * LD, "product scratch must fit the leaf staging area");
constexpr int MT = 64;         // output tile side of the staged products
constexpr int MKC = 64;        // K chunk of the staged products
constexpr int MNB = 16;        // staging loads per thread and K chunk
static_assert(2 * MT * MKC <= SMW && LT * MNB == 2 * MT * MKC, "one staging pass per K chunk");
constexpr int MM_TILED_K = 16; // shallower products read their operands directly

// C (M x N) <- C - A B over MT x MT output tiles, for products deep enough
// (K >= MM_TILED_K) that staging pays.  A thread holds a 4 x 2 patch of a tile
// (rows 4 w + a for warp w, columns lane + 32 b) as delayed-reduction sums;
// the tile's rows of A and columns of B pass through the shared scratch `sm`
// MKC at a time, and C is read once per tile.
template <bool SMALLP>
__device__ __noinline__ void nd_mm_sub_tiled(uint32_t *C, int64_t ldc, const uint32_t *A, int64_t lda,
                                       const uint32_t *B, int64_t ldb, int M, int N, int K,
                                       const Field F, uint32_t *sm)
{
    if (M > 0 && N > 0 && K > 0) {
        const uint32_t w16 = (uint32_t)((1ull << 16) % F.p);
        uint32_t *As = sm, *Bs = sm + MT * MKC;   // [MT][MKC], [MKC][MT]
        const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
        static_assert(NW * 4 == MT && 64 == MT, "thread patches must tile the output tile");
        for (int i0 = 0; i0 < M; i0 += MT)
            for (int j0 = 0; j0 < N; j0 += MT) {
                const int tm = min(MT, M - i0), tn = min(MT, N - j0);
                uint32_t c[4][2];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 2; ++b)
                        if (4 * w + a < tm && lane + 32 * b < tn)
                            c[a][b] = C[(int64_t)(i0 + 4 * w + a) * ldc + j0 + lane + 32 * b];
                LAcc<SMALLP> acc[4][2];
                for (int l0 = 0; l0 < K; l0 += MKC) {
                    const int kc = min(MKC, K - l0);
                    // tile rows of A (tm x kc, in a MT x MKC frame) and columns of B
                    // (kc x tn, in a MKC x MT frame): one pass of NB loads per thread
                                        uint32_t v[MNB];
#pragma unroll
                    for (int b = 0; b < MNB; ++b) {
                        const int e = tid + b * LT;
                        if (b < MNB / 2) {
                            const int i = e / MKC, l = e % MKC;
                            v[b] = i < tm && l < kc ? A[(int64_t)(i0 + i) * lda + l0 + l] : 0u;
                        } else {
                            const int l = (e - MT * MKC) / MT, j = (e - MT * MKC) % MT;
                            v[b] = l < kc && j < tn ? B[(int64_t)(l0 + l) * ldb + j0 + j] : 0u;
                        }
                    }
#pragma unroll
                    for (int b = 0; b < MNB; ++b) sm[tid + b * LT] = v[b];
                    __syncthreads();
#pragma unroll 4
                    for (int l = 0; l < kc; ++l) {
                        uint32_t x[4], y[2];
#pragma unroll
                        for (int a = 0; a < 4; ++a) x[a] = As[(4 * w + a) * MKC + l];
#pragma unroll
                        for (int b = 0; b < 2; ++b) y[b] = Bs[l * MT + lane + 32 * b];
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int b = 0; b < 2; ++b) acc[a][b].add(x[a], y[b]);
                    }
                    __syncthreads();
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 2; ++b)
                        if (4 * w + a < tm && lane + 32 * b < tn)
                            C[(int64_t)(i0 + 4 * w + a) * ldc + j0 + lane + 32 * b] =
                                sub_mod(c[a][b], acc[a][b].value(F, w16), F.p);
            }
    }
    __syncthreads();
}

// The thread blocks of a node kernel: one (NC = 1), or a cluster of NC = 2,
// 4 or 8 on as many SMs.  Each helper below does this CTA's share of a phase (rows or
// columns, or whole elements, split evenly by rank) and sets no barrier; the
// node step ends every phase with sync(), a block barrier for NC = 1 and a
// cluster barrier (release / acquire, which also orders global memory)
// otherwise.  Every CTA executes the same sequence of sync() calls: the only
// branches around them depend on data that all CTAs hold (sizes, and ranks
// and identity flags copied to every CTA after each base case).
template <int NC>
struct Grp {
    int rank;
    __device__ __forceinline__ void range(int tot, int &lo, int &hi) const
    {
        lo = (int)((int64_t)tot * rank / NC);
        hi = (int)((int64_t)tot * (rank + 1) / NC);
    }
    __device__ __forceinline__ void sync() const
    {
        if constexpr (NC == 1) {
            __syncthreads();
        } else {
            asm volatile("barrier.cluster.arrive.release;\n\t"
                         "barrier.cluster.wait.acquire;" ::: "memory");
        }
    }
};

__device__ __forceinline__ int cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}

// the word at `local` in this CTA's shared memory, in CTA `peer` of the cluster
__device__ __forceinline__ void st_peer(const void *local, int peer, int32_t v)
{
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_addr(local)), "r"(peer));
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(remote), "r"(v) : "memory");
}

// one permutation of a phase: X (rows x cols, stride ld) <- X[rmap[i]][cmap[j]]
// (a null map is the identity)
struct NdPerm {
    uint32_t *X;
    int rows, cols;
    const int32_t *rmap, *cmap;
};

// Word phase of an address within its 16-byte line.
__device__ __forceinline__ int word_phase(const void *p) { return (int)(((uintptr_t)p >> 2) & 3); }

// One warp copies `cols` words from src to dst, which share their phase:
// scalar head up to the 16-byte boundary, 16-byte body (two loads in flight
// per lane), scalar tail.
__device__ __forceinline__ void warp_row_copy16(uint32_t *dst, const uint32_t *src, int cols, int lane)
{
    const int head = min(cols, (4 - word_phase(src)) & 3);
    if (lane < head) dst[lane] = src[lane];
    const int nv = (cols - head) >> 2;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src + head);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst + head);
    int v = lane;
    for (; v + 32 < nv; v += 64) {
        const uint4 a = s4[v], b = s4[v + 32];
        d4[v] = a;
        d4[v + 32] = b;
    }
    if (v < nv) d4[v] = s4[v];
    const int t = head + 4 * nv + lane;
    if (t < cols) dst[t] = src[t];
}

// Blocks at least this wide move a row per warp (16-byte accesses where the
// row stride allows); narrower ones element by element over all threads.
constexpr int ND_ROW_COLS = 64;

// Stage layout of one op: row mode keeps every staged row at the phase of
// the block's rows (pitch a multiple of 4 words, 16-byte aligned start) so
// that both copies can use 16-byte accesses.
struct NdLayout {
    bool rowwise;
    int ph, pitch;
};

__device__ __forceinline__ NdLayout nd_layout(const NdPerm &q, bool vec)
{
    NdLayout L;
    L.rowwise = q.cols >= ND_ROW_COLS;
    L.ph = L.rowwise && vec ? word_phase(q.X) : 0;
    L.pitch = L.rowwise && vec ? ((q.cols + L.ph + 3) & ~3) : q.cols;
    return L;
}

// The permutations of a phase, on disjoint blocks, through disjoint slices of
// the global area `stage` (stage_words long): every block is gathered, then
// (after one barrier) copied back.  Wide blocks go a row per warp, CTAs taking
// row ranges: a row permutation moves whole rows with 16-byte accesses (when
// the row stride is a multiple of 4 words and the padded layout fits in the
// stage), a column permutation gathers each row's words through the map.
// Ends with its own barrier; none if no block moves.
template <int NC>
__device__ void nd_perms(const NdPerm *ops, int count, int64_t ld, uint32_t *stage,
                         int64_t stage_words, const Grp<NC> &g)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool any = false, vec = (ld & 3) == 0 && (((uintptr_t)stage) & 15) == 0;
    if (vec) {
        int64_t need = 0;
        for (int o = 0; o < count; ++o) {
            const NdPerm &q = ops[o];
            if (q.rows <= 0 || q.cols <= 0 || (!q.rmap && !q.cmap)) continue;
            const NdLayout L = nd_layout(q, true);
            need = ((need + 3) & ~(int64_t)3) + (int64_t)q.rows * L.pitch;
        }
        vec = need <= stage_words;
    }
    int64_t off = 0;
    for (int o = 0; o < count; ++o) {
        const NdPerm &q = ops[o];
        if (q.rows <= 0 || q.cols <= 0 || (!q.rmap && !q.cmap)) continue;
        any = true;
        const NdLayout L = nd_layout(q, vec);
        if (vec) off = (off + 3) & ~(int64_t)3;
        if (L.rowwise) {
            int lo, hi;
            g.range(q.rows, lo, hi);
            for (int i = lo + warp; i < hi; i += NW) {
                const uint32_t *src = q.X + (int64_t)(q.rmap ? q.rmap[i] : i) * ld;
                uint32_t *dst = stage + off + (int64_t)i * L.pitch + L.ph;
                if (q.cmap)
                    for (int j = lane; j < q.cols; j += 32) dst[j] = src[q.cmap[j]];
                else if (vec)
                    warp_row_copy16(dst, src, q.cols, lane);
                else
                    for (int j = lane; j < q.cols; j += 32) dst[j] = src[j];
            }
        } else {
            int lo, hi;
            g.range(q.rows * q.cols, lo, hi);
            for (int e = lo + (int)threadIdx.x; e < hi; e += LT) {
                const int i = e / q.cols, j = e - (e / q.cols) * q.cols;
                stage[off + e] = q.X[(int64_t)(q.rmap ? q.rmap[i] : i) * ld + (q.cmap ? q.cmap[j] : j)];
            }
        }
        off += (int64_t)q.rows * L.pitch;
    }
    if (!any) return;
    g.sync();
    off = 0;
    for (int o = 0; o < count; ++o) {
        const NdPerm &q = ops[o];
        if (q.rows <= 0 || q.cols <= 0 || (!q.rmap && !q.cmap)) continue;
        const NdLayout L = nd_layout(q, vec);
        if (vec) off = (off + 3) & ~(int64_t)3;
        if (L.rowwise) {
            int lo, hi;
            g.range(q.rows, lo, hi);
            for (int i = lo + warp; i < hi; i += NW) {
                const uint32_t *src = stage + off + (int64_t)i * L.pitch + L.ph;
                uint32_t *dst = q.X + (int64_t)i * ld;
                if (vec)
                    warp_row_copy16(dst, src, q.cols, lane);
                else
                    for (int j = lane; j < q.cols; j += 32) dst[j] = src[j];
            }
        } else {
            int lo, hi;
            g.range(q.rows * q.cols, lo, hi);
            for (int e = lo + (int)threadIdx.x; e < hi; e += LT) {
                const int i = e / q.cols, j = e - (e / q.cols) * q.cols;
                q.X[(int64_t)i * ld + j] = stage[off + e];
            }
        }
        off += (int64_t)q.rows * L.pitch;
    }
    g.sync();
}

// dst (rows x cols) <- src, this CTA's share of the rows (a row per warp) or,
// for narrow blocks, of the elements
template <int NC>
__device__ void nd_copy(uint32_t *dst, int64_t ldd, const uint32_t *src, int64_t lds, int rows,
                        int cols, const Grp<NC> &g)
{
    int lo, hi;
    if (cols >= ND_ROW_COLS) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        g.range(rows, lo, hi);
        for (int i = lo + warp; i < hi; i += NW)
            for (int j = lane; j < cols; j += 32) dst[(int64_t)i * ldd + j] = src[(int64_t)i * lds + j];
        return;
    }
    g.range(rows * cols, lo, hi);
    for (int e = lo + (int)threadIdx.x; e < hi; e += LT) {
        const int i = e / cols, j = e - (e / cols) * cols;
        dst[(int64_t)i * ldd + j] = src[(int64_t)i * lds + j];
    }
}

constexpr int TRB = 32;   // panel of the blocked triangular solves (wider triangles)

// B (r x N) <- L^{-1} B, L unit lower (diagonal not read): a thread per column
// of this CTA's share, each unknown one delayed-reduction dot product over the
// earlier ones.  Triangles of more than TRB rows go by panels of TRB rows: the
// panel's own triangle as above, then the rows below it take the panel's
// product off through nd_mm_sub_tiled (scratch `sm`), so the O(r^2 N) work
// runs as staged products.
template <bool SMALLP, int NC>
__device__ void nd_trsm_left(const uint32_t *L, int64_t ldl, uint32_t *B, int64_t ldb, int r, int N,
                             const Field &F, uint32_t *sm, const Grp<NC> &g)
{
    if (r <= 1 || N <= 0) return;
    const uint32_t w16 = (uint32_t)((1ull << 16) % F.p);
    int lo, hi;
    g.range(N, lo, hi);
    for (int i0 = 0; i0 < r; i0 += TRB) {
        const int ib = min(TRB, r - i0);
        for (int j = lo + (int)threadIdx.x; j < hi; j += LT)
            for (int i = i0 + 1; i < i0 + ib; ++i) {
                LAcc<SMALLP> acc;
                for (int l = i0; l < i; ++l)
                    acc.add(L[(int64_t)i * ldl + l], B[(int64_t)l * ldb + j]);
                B[(int64_t)i * ldb + j] = sub_mod(B[(int64_t)i * ldb + j], acc.value(F, w16), F.p);
            }
        if (i0 + ib < r) {
            __syncthreads();
            nd_mm_sub_tiled<SMALLP>(B + (int64_t)(i0 + ib) * ldb + lo, ldb, L + (int64_t)(i0 + ib) * ldl + i0,
                                    ldl, B + (int64_t)i0 * ldb + lo, ldb, r - i0 - ib, hi - lo, ib, F, sm);
        }
    }
}

// B (M x r) <- B U^{-1}, U upper with nonzero diagonal: a thread per row of
// this CTA's share; dinv (r words) receives the inverses of the diagonal.
// Triangles of more than TRB columns go by panels of TRB columns: the panel's
// columns as above, then the columns right of it take the panel's product off
// through nd_mm_sub_tiled (scratch `sm`).
template <bool SMALLP, int NC>
__device__ void nd_trsm_right(const uint32_t *U, int64_t ldu, uint32_t *B, int64_t ldb, int M, int r,
                              const Field &F, uint32_t *dinv, uint32_t *sm, const Grp<NC> &g)
{
    if (r <= 0 || M <= 0) return;
    const uint32_t w16 = (uint32_t)((1ull << 16) % F.p);
    for (int t = threadIdx.x; t < r; t += LT) dinv[t] = inv_mod(U[(int64_t)t * ldu + t], F.p);
    __syncthreads();
    int lo, hi;
    g.range(M, lo, hi);
    for (int j0 = 0; j0 < r; j0 += TRB) {
        const int jb = min(TRB, r - j0);
        for (int i = lo + (int)threadIdx.x; i < hi; i += LT) {
            uint32_t *row = B + (int64_t)i * ldb;
            for (int j = j0; j < j0 + jb; ++j) {
                LAcc<SMALLP> acc;
                for (int l = j0; l < j; ++l) acc.add(U[(int64_t)l * ldu + j], row[l]);
                row[j] = mul_mod(sub_mod(row[j], acc.value(F, w16), F.p), dinv[j], F);
            }
        }
        if (j0 + jb < r) {
            __syncthreads();
            nd_mm_sub_tiled<SMALLP>(B + (int64_t)lo * ldb + j0 + jb, ldb, B + (int64_t)lo * ldb + j0, ldb,
                                    U + (int64_t)j0 * ldu + j0 + jb, ldu, hi - lo, r - j0 - jb, jb, F, sm);
        }
    }
}

// C (M x N) <- C - A B for shallow products (K < MM_TILED_K): a row of C per
// warp.  Where the rows of C and B share their 16-byte phase (and the strides
// are multiples of 4 words) each lane takes four adjacent columns with 16-byte
// accesses, the columns before the first and after the last 16-byte boundary
// one per lane; otherwise every column is one per lane.  The K entries of A's
// row are read by the whole warp at once.  Each output one delayed reduction.
template <bool SMALLP>
__device__ void nd_mm_sub_shallow(uint32_t *C, int64_t ldc, const uint32_t *A, int64_t lda,
                                  const uint32_t *B, int64_t ldb, int M, int N, int K, const Field &F)
{
    const uint32_t w16 = (uint32_t)((1ull << 16) % F.p);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool vec = N >= 8 && ((ldc | ldb) & 3) == 0 && word_phase(C) == word_phase(B);
    const int head = vec ? min(N, (4 - word_phase(C)) & 3) : N;   // one per lane, before the body
    const int nv = vec ? (N - head) >> 2 : 0;                       // 16-byte groups
    const int tail0 = head + 4 * nv;                                // one per lane, after the body
    const int ns = head + (N - tail0);
    for (int i = warp; i < M; i += NW) {
        uint32_t *c = C + (int64_t)i * ldc;
        const uint32_t *a = A + (int64_t)i * lda;
        uint32_t av[MM_TILED_K];
#pragma unroll
        for (int l = 0; l < MM_TILED_K; ++l) av[l] = l < K ? a[l] : 0u;
        for (int v = lane; v < nv; v += 32) {
            const int j = head + 4 * v;
            LAcc<SMALLP> acc[4];
#pragma unroll
            for (int l = 0; l < MM_TILED_K; ++l)
                if (l < K) {
                    const uint4 y = *reinterpret_cast<const uint4 *>(B + (int64_t)l * ldb + j);
                    acc[0].add(av[l], y.x);
                    acc[1].add(av[l], y.y);
                    acc[2].add(av[l], y.z);
                    acc[3].add(av[l], y.w);
                }
            uint4 x = *reinterpret_cast<const uint4 *>(c + j);
            x.x = sub_mod(x.x, acc[0].value(F, w16), F.p);
            x.y = sub_mod(x.y, acc[1].value(F, w16), F.p);
            x.z = sub_mod(x.z, acc[2].value(F, w16), F.p);
            x.w = sub_mod(x.w, acc[3].value(F, w16), F.p);
            *reinterpret_cast<uint4 *>(c + j) = x;
        }
        for (int t = lane; t < ns; t += 32) {
            const int j = t < head ? t : tail0 + (t - head);
            LAcc<SMALLP> acc;
#pragma unroll
            for (int l = 0; l < MM_TILED_K; ++l)
                if (l < K) acc.add(av[l], B[(int64_t)l * ldb + j]);
            c[j] = sub_mod(c[j], acc.value(F, w16), F.p);
        }
    }
}

// C (M x N) <- C - A B, A M x K, B K x N, this CTA's share of the rows: each
// output one delayed reduction, or (K >= MM_TILED_K) through nd_mm_sub_tiled;
// ends with a block barrier where it ran
template <bool SMALLP, int NC>
__device__ void nd_mm_sub(uint32_t *C, int64_t ldc, const uint32_t *A, int64_t lda,
                          const uint32_t *B, int64_t ldb, int M, int N, int K, const Field &F,
                          uint32_t *sm, const Grp<NC> &g)
{
    int lo, hi;
    g.range(M, lo, hi);
    C += (int64_t)lo * ldc;
    A += (int64_t)lo * lda;
    M = hi - lo;
    if (M <= 0 || N <= 0 || K <= 0) return;
    if (K >= MM_TILED_K) {
        nd_mm_sub_tiled<SMALLP>(C, ldc, A, lda, B, ldb, M, N, K, F, sm);
        return;
    }
    nd_mm_sub_shallow<SMALLP>(C, ldc, A, lda, B, ldb, M, N, K, F);
    __syncthreads();
}

constexpr int NCMAX = 8;   // largest cluster of a node kernel (the portable limit)

// Per-level state of a node step: the permutations of its four blocks, the
// maps of S and T, and each block's r / P identity / Q identity.  A step of
// level l has blocks of sides up to V = 2^(l-1) LM.
template <int V>
struct NodeLevel {
    int32_t pv[8][V];          // P1, Q1, P2, Q2, P3, Q3, P4, Q4
    int32_t smap[2 * V], tmap[2 * V];
    int32_t info[4][3];
};

struct NodeShared {
    NodeLevel<LM> l1;
    NodeLevel<2 * LM> l2;
    uint32_t dinv[2 * LM];
    int32_t flags[NCMAX];      // the CTAs' zero-test results
    // levels 3 and 4 (the batch kernel only, which points them into its
    // dynamic shared memory): their state, and the diagonal inverses of
    // triangles of up to 8 LM rows
    NodeLevel<4 * LM> *l3;
    NodeLevel<8 * LM> *l4;
    uint32_t *dinv_wide;
};

// true if some entry of X (rows x cols) is nonzero; every CTA gets the answer
template <int NC>
__device__ bool nd_any_nonzero(const uint32_t *X, int64_t ld, int rows, int cols, int32_t *flags,
                               const Grp<NC> &g)
{
    int lo, hi;
    bool nz = false;
    if (cols >= ND_ROW_COLS) {
        // a row per warp, 16-byte loads where the row stride allows
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        g.range(rows, lo, hi);
        for (int i = lo + warp; i < hi && !nz; i += NW) {
            const uint32_t *row = X + (int64_t)i * ld;
            uint32_t acc = 0;
            if ((ld & 3) == 0) {
                const int head = min(cols, (4 - word_phase(row)) & 3);
                if (lane < head) acc |= row[lane];
                const int nv = (cols - head) >> 2;
                const uint4 *r4 = reinterpret_cast<const uint4 *>(row + head);
                for (int v = lane; v < nv; v += 32) {
                    const uint4 x = r4[v];
                    acc |= x.x | x.y | x.z | x.w;
                }
                const int t = head + 4 * nv + lane;
                if (t < cols) acc |= row[t];
            } else {
                for (int j = lane; j < cols; j += 32) acc |= row[j];
            }
            nz = __any_sync(0xffffffffu, acc != 0);
        }
    } else {
        g.range(rows * cols, lo, hi);
        for (int e = lo + (int)threadIdx.x; e < hi && !nz; e += LT)
            nz = X[(int64_t)(e / cols) * ld + (e - (e / cols) * cols)] != 0;
    }
    const bool mine = __syncthreads_or(nz);
    if constexpr (NC == 1) {
        return mine;
    } else {
        if ((int)threadIdx.x < NC) st_peer(&flags[g.rank], threadIdx.x, mine ? 1 : 0);
        g.sync();
        int any = 0;
        for (int c = 0; c < NC; ++c) any |= flags[c];
        g.sync();   // every CTA has read the flags before any is written again
        return any != 0;
    }
}

// the P, Q and info of block c, computed by this CTA, into the other CTAs'
// copies of the level state
template <int NC, int V>
__device__ void push_child(NodeLevel<V> &N, int c, int mb, int nb, const Grp<NC> &g)
{
    for (int peer = 0; peer < NC; ++peer) {
        if (peer == g.rank) continue;
        for (int i = threadIdx.x; i < mb; i += LT) st_peer(&N.pv[2 * c][i], peer, N.pv[2 * c][i]);
        for (int j = threadIdx.x; j < nb; j += LT) st_peer(&N.pv[2 * c + 1][j], peer, N.pv[2 * c + 1][j]);
        if (threadIdx.x < 3) st_peer(&N.info[c][threadIdx.x], peer, N.info[c][threadIdx.x]);
    }
}

struct NodeArgs {
    uint32_t *A;
    int m, n;
    int64_t lda;
    Field F;
    int32_t *perm_p, *perm_q;  // m, n
    int32_t *info;             // r, P identity, Q identity
    volatile int32_t *host_info;
    int32_t seq;
    uint32_t *stage;           // at least m * n words
    int64_t stage_words;       // its length (a padded 16-byte layout is used when it fits)
    uint32_t *icopy;           // at least (m/2 + 1) * (n/2 + 1) words
    uint32_t wait_limit;
    int try_generic, left_looking;
};

// the base case for blocks of up to LM x LM, compiled once for the node
// steps' calls
template <bool SMALLP>
__device__ __noinline__ void leaf_run_full(LeafShared &S, uint32_t *A, int m, int n, int64_t lda,
                                           Field F, int32_t *pp, int32_t *pq, int32_t *info,
                                           int try_generic, uint32_t wait_limit, int left_looking)
{
    leaf_run<SMALLP, 4, 8>(S, A, m, n, lda, F, pp, pq, info, 3, nullptr, 0, try_generic,
                           wait_limit, left_looking);
}

template <int LEVEL>
__device__ __forceinline__ auto &node_level(NodeShared &N)
{
    static_assert(LEVEL >= 1 && LEVEL <= 4, "node steps span one to four levels");
    if constexpr (LEVEL == 1) return N.l1;
    else if constexpr (LEVEL == 2) return N.l2;
    else if constexpr (LEVEL == 3) return *N.l3;
    else return *N.l4;
}

// the diagonal inverses of a step's triangles: at level l a triangle has at
// most 2^(l-1) LM rows
template <int LEVEL>
__device__ __forceinline__ uint32_t *node_dinv(NodeShared &N)
{
    if constexpr (LEVEL <= 2) return N.dinv;
    else return N.dinv_wide;
}

// One step of Algorithm 1 on the m x n block at A (both sides at most 2^LEVEL
// LM) by the NC thread blocks: blocks that are base cases go to leaf_run_full
// on one CTA (F and G on different CTAs when NC > 1, so they run at once),
// larger ones (LEVEL > 1) to a step of the level below on all CTAs.  Writes P / Q to
// pp / pq and r, P identity, Q identity to info[0..2] (-1 for r if a base
// case gave up a bounded wait); every CTA writes the same values.
template <bool SMALLP, int LEVEL, int NC>
__device__ __noinline__ void node_step(LeafShared &S, NodeShared &NS, const NodeArgs &a,
                                       uint32_t *A, int m, int n, int32_t *pp, int32_t *pq,
                                       int32_t *info, int try_generic, const Grp<NC> g)
{
    auto &N = node_level<LEVEL>(NS);
    const int tid = threadIdx.x;
    const int k = m / 2, h = n / 2;
    const int64_t lda = a.lda;
    const Field F = a.F;
    auto at = [&](int i, int j) { return A + (int64_t)i * lda + j; };
    auto done = [&](int r, int pid, int qid) {
        if (tid == 0) {
            info[0] = r;
            info[1] = pid;
            info[2] = qid;
        }
        __syncthreads();
    };
    // block c (0 A1, 1 F, 2 G, 3 R); an empty block has r = 0, P = Q = I.  A
    // base case runs on CTA `owner`, which then copies its results to the
    // others; no barrier here, the caller ends the phase
    auto child = [&](int c, uint32_t *X, int mb, int nb, int tg, int owner) {
        if (mb <= 0 || nb <= 0) {
            if (tid == 0) {
                N.info[c][0] = 0;
                N.info[c][1] = 1;
                N.info[c][2] = 1;
            }
        } else if (mb <= LM && nb <= LM) {
            if (g.rank == owner) {
                leaf_run_full<SMALLP>(S, X, mb, nb, lda, F, N.pv[2 * c], N.pv[2 * c + 1], N.info[c],
                                      tg, a.wait_limit, a.left_looking);
                if constexpr (NC > 1) {
                    __syncthreads();
                    push_child<NC>(N, c, mb, nb, g);
                }
            }
        } else {
            if constexpr (LEVEL > 1)
                node_step<SMALLP, LEVEL - 1, NC>(S, NS, a, X, mb, nb, N.pv[2 * c], N.pv[2 * c + 1],
                                                 N.info[c], tg, g);
        }
    };

    // a zero block is finished: r = 0, P = Q = I
    if (!nd_any_nonzero<NC>(A, lda, m, n, NS.flags, g)) {
        for (int i = tid; i < m; i += LT) pp[i] = i;
        for (int j = tid; j < n; j += LT) pq[j] = j;
        done(0, 1, 1);
        return;
    }
    // A1 = P1 [L1; M1] [U1 V1] Q1
    child(0, A, k, h, try_generic, 0);
    g.sync();
    const int r1 = N.info[0][0];
    if (r1 < 0) {
        done(-1, 0, 0);
        return;
    }
    const int32_t *P1 = N.info[0][1] ? nullptr : N.pv[0];
    const int32_t *Q1 = N.info[0][2] ? nullptr : N.pv[1];
    const int tg = r1 < (k < h ? k : h) ? 0 : 1;
    // [B1;B2] <- P1^T A2 ; [C1 C2] <- A3 Q1^T
    {
        const NdPerm ops[2] = {{at(0, h), k, n - h, P1, nullptr}, {at(k, 0), m - k, h, nullptr, Q1}};
        nd_perms<NC>(ops, 2, lda, a.stage, a.stage_words, g);
    }
    // D <- L1^{-1} B1 ; E <- C1 U1^{-1} ; [F;H] <- [B2;A4] - [M1;E] D ; G <- C2 - E V1
    nd_trsm_left<SMALLP, NC>(A, lda, at(0, h), lda, r1, n - h, F, S.W, g);
    nd_trsm_right<SMALLP, NC>(A, lda, at(k, 0), lda, m - k, r1, F, node_dinv<LEVEL>(NS), S.W, g);
    g.sync();
    nd_mm_sub<SMALLP, NC>(at(r1, h), lda, at(r1, 0), lda, at(0, h), lda, m - r1, n - h, r1, F, S.W, g);
    nd_mm_sub<SMALLP, NC>(at(k, r1), lda, at(k, 0), lda, at(0, r1), lda, m - k, h - r1, r1, F, S.W, g);
    g.sync();
    // F = P2 [L2;M2][U2 V2] Q2 ; G = P3 [L3;M3][U3 V3] Q3, on different CTAs
    child(1, at(r1, h), k - r1, n - h, tg, 0);
    child(2, at(k, r1), m - k, h - r1, tg, NC - 1);
    g.sync();
    const int r2 = N.info[1][0], r3 = N.info[2][0];
    if (r2 < 0 || r3 < 0) {
        done(-1, 0, 0);
        return;
    }
    const int32_t *P2 = N.info[1][1] ? nullptr : N.pv[2];
    const int32_t *Q2 = N.info[1][2] ? nullptr : N.pv[3];
    const int32_t *P3 = N.info[2][1] ? nullptr : N.pv[4];
    const int32_t *Q3 = N.info[2][2] ? nullptr : N.pv[5];
    // H <- P3^T H Q2^T ; E <- P3^T E ; M1 <- P2^T M1 ; D <- D Q2^T ; V1 <- V1 Q3^T
    {
        const NdPerm ops[5] = {{at(k, h), m - k, n - h, P3, Q2},
                               {at(k, 0), m - k, r1, P3, nullptr},
                               {at(r1, 0), k - r1, r1, P2, nullptr},
                               {at(0, h), r1, n - h, nullptr, Q2},
                               {at(0, r1), r1, h - r1, nullptr, Q3}};
        nd_perms<NC>(ops, 5, lda, a.stage, a.stage_words, g);
    }
    // [I;K] <- [H1;H3] U2^{-1} ; keep I ; [J N] <- L3^{-1} [I H2]
    nd_trsm_right<SMALLP, NC>(at(r1, h), lda, at(k, h), lda, m - k, r2, F, node_dinv<LEVEL>(NS), S.W, g);
    g.sync();
    if (r3 > 0 && r2 > 0) {
        nd_copy<NC>(a.icopy, r2, at(k, h), lda, r3, r2, g);
        g.sync();
    }
    nd_trsm_left<SMALLP, NC>(at(k, r1), lda, at(k, h), lda, r3, n - h, F, S.W, g);
    g.sync();
    // O <- N - J V2 ; R <- H4 - K V2 ; then I back and R <- R - M3 O
    nd_mm_sub<SMALLP, NC>(at(k, h + r2), lda, at(k, h), lda, at(r1, h + r2), lda, r3, n - h - r2,
                          r2, F, S.W, g);
    nd_mm_sub<SMALLP, NC>(at(k + r3, h + r2), lda, at(k + r3, h), lda, at(r1, h + r2), lda,
                          m - k - r3, n - h - r2, r2, F, S.W, g);
    g.sync();
    if (r3 > 0 && r2 > 0) nd_copy<NC>(at(k, h), lda, a.icopy, r2, r3, r2, g);
    nd_mm_sub<SMALLP, NC>(at(k + r3, h + r2), lda, at(k + r3, r1), lda, at(k, h + r2), lda,
                          m - k - r3, n - h - r2, r3, F, S.W, g);
    g.sync();
    // R = P4 [L4;M4][U4 V4] Q4
    child(3, at(k + r3, h + r2), m - k - r3, n - h - r2, tg, 0);
    g.sync();
    const int r4 = N.info[3][0];
    if (r4 < 0) {
        done(-1, 0, 0);
        return;
    }
    const int32_t *P4 = N.info[3][1] ? nullptr : N.pv[6];
    const int32_t *Q4 = N.info[3][2] ? nullptr : N.pv[7];
    // [E2 M3 0 K] <- P4^T [..] ; [D2;V2;0;O] <- [..] Q4^T
    {
        const NdPerm ops[2] = {{at(k + r3, 0), m - k - r3, h + r2, P4, nullptr},
                               {at(0, h + r2), k + r3, n - h - r2, nullptr, Q4}};
        nd_perms<NC>(ops, 2, lda, a.stage, a.stage_words, g);
    }
    // P = Diag(P1 diag(I,P2), P3 diag(I,P4)) S, Q = T Diag(diag(I,Q3) Q1, diag(I,Q4) Q2),
    // and the row map of S / column map of T (every CTA, into its own maps)
    auto ap = [](const int32_t *v, int x) { return v ? v[x] : x; };
    bool s_same = true, t_same = true;
    for (int i = tid; i < m; i += LT) {
        const int top = r1 + r2, bot = r3 + r4;
        const int sr = i < top ? i : (i < top + bot ? k + (i - top) : (i < k + bot ? i - bot : i));
        N.smap[i] = sr;
        s_same &= sr == i;
        int d;
        if (sr < k) d = sr < r1 ? ap(P1, sr) : ap(P1, r1 + ap(P2, sr - r1));
        else {
            const int u = sr - k;
            d = k + (u < r3 ? ap(P3, u) : ap(P3, r3 + ap(P4, u - r3)));
        }
        pp[i] = d;
    }
    for (int j = tid; j < n; j += LT) {
        int c;
        if (j < r1) c = j;
        else if (j < r1 + r2) c = h + (j - r1);
        else if (j < r1 + r2 + r3) c = r1 + (j - r1 - r2);
        else if (j < r1 + r2 + r3 + r4) c = h + r2 + (j - r1 - r2 - r3);
        else if (j < h + r2 + r4) c = r1 + r3 + (j - r1 - r2 - r3 - r4);
        else c = j;
        N.tmap[j] = c;
        t_same &= c == j;
        int d;
        if (c < h) d = c < r1 ? ap(Q1, c) : ap(Q1, r1 + ap(Q3, c - r1));
        else {
            const int u = c - h;
            d = h + (u < r2 ? ap(Q2, u) : ap(Q2, r2 + ap(Q4, u - r2)));
        }
        pq[j] = d;
    }
    const bool s_ident = __syncthreads_and(s_same);
    const bool t_ident = __syncthreads_and(t_same);
    // A <- S^T A T^T
    {
        const NdPerm op{A, m, n, s_ident ? nullptr : N.smap, t_ident ? nullptr : N.tmap};
        nd_perms<NC>(&op, 1, lda, a.stage, a.stage_words, g);
    }
    int pid = s_ident, qid = t_ident;
    for (int c = 0; c < 4; ++c) {
        pid &= N.info[c][1] != 0;
        qid &= N.info[c][2] != 0;
    }
    done(r1 + r2 + r3 + r4, pid, qid);
}

}  // namespace
}  // namespace pluq
