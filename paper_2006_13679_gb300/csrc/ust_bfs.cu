// BFS tree B_u of the pivot (Section 3.2, Algorithm 1).
//
// Level-synchronous bottom-up ("pull") BFS: at level L every unvisited
// vertex scans its sorted adjacency row and stops at the first neighbour at
// distance L. Because rows are sorted, that neighbour is the smallest-id
// vertex one level closer to u, which is the parent rule of B_u.
#include <algorithm>

#include "ust_common.cuh"

namespace ust {
namespace {

__global__ void bfs_init_kernel(int n, int u, int32_t *__restrict__ dist, int32_t *__restrict__ bpar)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        dist[v] = (v == u) ? 0 : -1;
        bpar[v] = -1;
    }
}

__global__ void bfs_pull_kernel(int n, int level, const int32_t *__restrict__ rp,
                                const int32_t *__restrict__ ci, int32_t *dist,
                                int32_t *__restrict__ bpar, int32_t *__restrict__ found)
{
    int any = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (dist[v] >= 0) continue;
        const int e1 = __ldg(rp + v + 1);
        for (int e = __ldg(rp + v); e < e1; ++e) {
            const int w = __ldg(ci + e);
            if (dist[w] == level) {
                dist[v] = level + 1;
                bpar[v] = w;
                any = 1;
                break;
            }
        }
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) *found = 1;
}

// stats[0] += sum of dist, stats[1] += number of unreached vertices
__global__ void bfs_sum_kernel(int n, const int32_t *__restrict__ dist, unsigned long long *stats)
{
    long long s = 0, bad = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int d = dist[v];
        if (d < 0) bad += 1; else s += d;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(stats + 0, (unsigned long long)s);
        atomicAdd(stats + 1, (unsigned long long)bad);
    }
}

// Exclusive prefix sum of dist into ptr[0..n] by one CTA (ptr[n] = total).
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) path_offsets_kernel(int n, const int32_t *__restrict__ dist,
                                                                    int32_t *__restrict__ ptr)
{
    __shared__ int s_warp[kScanThreads / 32 + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int carry = 0;
    for (int base = 0; base < n; base += kScanThreads) {
        const int i = base + threadIdx.x;
        const int x = (i < n) ? dist[i] : 0;
        int incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_warp[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const int w = s_warp[lane];
            int wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            s_warp[lane] = wi - w;
            if (lane == 31) s_warp[32] = wi;
        }
        __syncthreads();
        if (i < n) ptr[i] = carry + s_warp[wid] + incl - x;
        carry += s_warp[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) ptr[n] = carry;
}

// path[ptr[v] .. ptr[v+1]) = bfs_parent(v), its parent, ..., u
// Entry k of P(v): the edge (path[k], pchild[k]) = (a_j, a_{j-1}) with
// a_0 = v, and its owner powner[k] = v.
__global__ void path_fill_kernel(int n, int u, const int32_t *__restrict__ bpar, const int32_t *__restrict__ ptr,
                                 int32_t *__restrict__ path, int32_t *__restrict__ pchild,
                                 int32_t *__restrict__ powner)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int k = ptr[v];
        const int end = ptr[v + 1];
        int x = v;
        while (x != u && k < end) {
            const int b = x;
            x = bpar[x];
            path[k] = x;
            pchild[k] = b;
            powner[k] = v;
            ++k;
        }
    }
}

// ---------------------------------------------------------------------------
// Input checks of ust_init on the device copy of the CSR (the same checks
// the host would make, at GPU speed). Errors are OR-ed into *bad.
enum : int {
    kBadBounds = 1,    // row_ptr does not run from 0 to nnz, or is not monotone
    kBadRange = 2,     // a column index outside [0, n)
    kBadLoop = 4,      // a self-loop
    kBadOrder = 8,     // a row not strictly increasing (unsorted or duplicate)
    kBadSymmetry = 16, // an arc (v, w) without (w, v)
    kIsolated = 32,    // a vertex without arcs
};

__global__ void check_rows_kernel(int n, int nnz, const int32_t *__restrict__ rp, int *bad)
{
    int flags = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rp[0] != 0 || rp[n] != nnz)) flags |= kBadBounds;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int b = __ldg(rp + v), e = __ldg(rp + v + 1);
        if (e < b || b < 0 || e > nnz) flags |= kBadBounds;
        else if (e == b) flags |= kIsolated;
    }
    if (flags) atomicOr(bad, flags);
}

// Needs monotone row pointers from 0 to nnz (check_rows_kernel first).
__global__ void check_arcs_kernel(int n, int nnz, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                  int *bad)
{
    int flags = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x) {
        int lo = 0, hi = n;  // the row of arc k: the largest v with rp[v] <= k
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(rp + mid) <= k) lo = mid; else hi = mid;
        }
        const int v = lo, w = __ldg(ci + k);
        if (w < 0 || w >= n) {
            flags |= kBadRange;
            continue;
        }
        if (w == v) flags |= kBadLoop;
        if (k > __ldg(rp + v) && __ldg(ci + k - 1) >= w) flags |= kBadOrder;
        int a = __ldg(rp + w), z = __ldg(rp + w + 1);  // v in row w (sorted when the graph is valid)
        while (a < z) {
            const int mid = (a + z) >> 1;
            if (__ldg(ci + mid) < v) a = mid + 1; else z = mid;
        }
        if (a >= __ldg(rp + w + 1) || __ldg(ci + a) != v) flags |= kBadSymmetry;
    }
    if (flags) atomicOr(bad, flags);
}

// ---------------------------------------------------------------------------
// Pivot selection (Appendix D, choice of u): eccentricity lower bounds from
// repeated double sweeps. Packed keys make the reductions single atomics
// with the smallest id winning ties.
__global__ void max_degree_kernel(int n, const int32_t *__restrict__ rp, unsigned long long *best)
{
    unsigned long long b = 0ull;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const unsigned long long k = ((unsigned long long)(uint32_t)(__ldg(rp + v + 1) - __ldg(rp + v)) << 32) |
                                     (uint32_t)(0x7FFFFFFF - v);
        b = k > b ? k : b;
    }
    atomicMax(best, b);
}

// lb = max(lb, dist); *far = the farthest vertex; *bad |= 1 for unreached vertices
__global__ void sweep_update_kernel(int n, const int32_t *__restrict__ dist, int32_t *lb, unsigned long long *far,
                                    int *bad)
{
    unsigned long long b = 0ull;
    int unreached = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int d = dist[v];
        if (d < 0) {
            unreached = 1;
            continue;
        }
        if (d > lb[v]) lb[v] = d;
        const unsigned long long k = ((unsigned long long)(uint32_t)d << 32) | (uint32_t)(0x7FFFFFFF - v);
        b = k > b ? k : b;
    }
    atomicMax(far, b);
    if (unreached) atomicOr(bad, 1);
}

__global__ void min_bound_kernel(int n, const int32_t *__restrict__ lb, unsigned long long *best)
{
    unsigned long long b = ~0ull;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const unsigned long long k = ((unsigned long long)(uint32_t)lb[v] << 32) | (uint32_t)v;
        b = k < b ? k : b;
    }
    atomicMin(best, b);
}


// ---- biconnected-component variant (Appendix D) ---------------------------
// Rows of the block-restricted sampler: v != u keeps its neighbours inside its
// parent block, the block of the tree edge e(v) = (bfs_parent(v), v) of B_u.
// Blocks are labelled by Tarjan and Vishkin's rules over B_u (any rooted
// spanning tree serves). With preorder numbers pre, subtree sizes nd, and
// lo(v) / hi(v) the least / largest pre reached from v's subtree by a
// non-tree edge (pre(v) itself included), tree edges share a block when
//   (1) a non-tree edge (v, w) joins two unrelated subtrees: e(v) ~ e(w);
//   (2) p = bfs_parent(v) != u and v's subtree reaches outside p's subtree
//       (lo(v) < pre(p) or hi(v) >= pre(p) + nd(p)): e(v) ~ e(p).
// A non-tree edge lies in the block of e(x), x its endpoint of larger pre.
// Preorder and sizes follow the BFS levels, one launch per level.

__device__ __forceinline__ bool tree_edge(int v, int w, const int32_t *__restrict__ bpar)
{
    return bpar[w] == v || bpar[v] == w;
}

__global__ void bt_init_kernel(int n, int u, int32_t *nd, int32_t *pre, int32_t *cur, int32_t *uf)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        nd[v] = 1;
        pre[v] = 0;
        cur[v] = (v == u) ? 1 : 0;
        uf[v] = v;
    }
}

// Subtree sizes, deepest level first: nd[v] is complete when v's level runs.
__global__ void bt_size_kernel(int n, int level, const int32_t *__restrict__ dist,
                               const int32_t *__restrict__ bpar, int32_t *nd)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (dist[v] == level) atomicAdd(nd + bpar[v], nd[v]);
}

// Preorder numbers, top level first: a child takes the next free interval of
// its parent's (any child order is a preorder).
__global__ void bt_pre_kernel(int n, int level, const int32_t *__restrict__ dist,
                              const int32_t *__restrict__ bpar, const int32_t *__restrict__ nd, int32_t *pre,
                              int32_t *cur)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (dist[v] != level) continue;
        const int p = atomicAdd(cur + bpar[v], nd[v]);
        pre[v] = p;
        cur[v] = p + 1;
    }
}

// The kernels that scan adjacency rows take one warp per row, lanes striding
// the row, so that the rows of hubs do not serialise on one thread.
__device__ __forceinline__ int warp_id_global() { return (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); }
__device__ __forceinline__ int warps_global() { return (int)((gridDim.x * blockDim.x) >> 5); }

__global__ void bt_local_kernel(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                const int32_t *__restrict__ bpar, const int32_t *__restrict__ pre, int32_t *lo,
                                int32_t *hi)
{
    const int lane = threadIdx.x & 31;
    for (int v = warp_id_global(); v < n; v += warps_global()) {
        int l = pre[v], h = pre[v];
        for (int e = rp[v] + lane; e < rp[v + 1]; e += 32) {
            const int w = ci[e];
            if (tree_edge(v, w, bpar)) continue;
            l = min(l, pre[w]);
            h = max(h, pre[w]);
        }
        l = __reduce_min_sync(0xffffffffu, l);
        h = __reduce_max_sync(0xffffffffu, h);
        if (lane == 0) {
            lo[v] = l;
            hi[v] = h;
        }
    }
}

// lo / hi over subtrees, deepest level first.
__global__ void bt_lohi_kernel(int n, int level, const int32_t *__restrict__ dist,
                               const int32_t *__restrict__ bpar, int32_t *lo, int32_t *hi)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (dist[v] != level) continue;
        atomicMin(lo + bpar[v], lo[v]);
        atomicMax(hi + bpar[v], hi[v]);
    }
}

// Union-find over tree edges (named by their child vertex): roots are only
// hooked under smaller roots, finds halve paths. Reads bypass L1 so that a
// hook by another SM is seen; every loop is bounded and flags *bad.
__device__ int uf_find(int32_t *uf, int x, int n, int *bad)
{
    for (int k = 0; k <= n; ++k) {
        const int p = __ldcg(uf + x);
        if (p == x) return x;
        const int g = __ldcg(uf + p);
        if (g == p) return p;
        // path halving: x is no root, so any ancestor is a valid parent; an
        // atomic store, since other threads read uf and CAS roots meanwhile
        atomicExch(uf + x, g);
        x = g;
    }
    atomicExch(bad, 1);
    return x;
}

__device__ void uf_union(int32_t *uf, int a, int b, int n, int *bad)
{
    for (int k = 0; k <= n; ++k) {
        a = uf_find(uf, a, n, bad);
        b = uf_find(uf, b, n, bad);
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(uf + b, b, a) == b) return;
    }
    atomicExch(bad, 1);
}

__global__ void bt_rule1_kernel(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                const int32_t *__restrict__ bpar, const int32_t *__restrict__ pre,
                                const int32_t *__restrict__ nd, int32_t *uf, int *bad)
{
    const int lane = threadIdx.x & 31;
    for (int v = warp_id_global(); v < n; v += warps_global()) {
        const int pv = pre[v], end = pv + nd[v];
        for (int e = rp[v] + lane; e < rp[v + 1]; e += 32) {
            const int w = ci[e];
            if (tree_edge(v, w, bpar)) continue;
            const int pw = pre[w];
            if (pv < pw && pw >= end) uf_union(uf, v, w, n, bad);
        }
    }
}

__global__ void bt_rule2_kernel(int n, int u, const int32_t *__restrict__ bpar, const int32_t *__restrict__ pre,
                                const int32_t *__restrict__ nd, const int32_t *__restrict__ lo,
                                const int32_t *__restrict__ hi, int32_t *uf, int *bad)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (v == u) continue;
        const int p = bpar[v];
        if (p == u) continue;
        if (lo[v] < pre[p] || hi[v] >= pre[p] + nd[p]) uf_union(uf, v, p, n, bad);
    }
}

__global__ void bt_label_kernel(int n, int32_t *uf, int32_t *lab, int *bad)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        lab[v] = uf_find(uf, v, n, bad);
}

__device__ __forceinline__ int block_of(int v, int w, const int32_t *__restrict__ bpar,
                                        const int32_t *__restrict__ pre, const int32_t *__restrict__ lab)
{
    if (bpar[w] == v) return lab[w];
    if (bpar[v] == w) return lab[v];
    return pre[v] > pre[w] ? lab[v] : lab[w];
}

__global__ void wk_count_kernel(int n, int u, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                const int32_t *__restrict__ bpar, const int32_t *__restrict__ pre,
                                const int32_t *__restrict__ lab, int32_t *wdeg)
{
    const int lane = threadIdx.x & 31;
    for (int v = warp_id_global(); v < n; v += warps_global()) {
        unsigned c = 0;
        if (v != u) {
            const int pb = lab[v];
            for (int e = rp[v] + lane; e < rp[v + 1]; e += 32) c += (block_of(v, ci[e], bpar, pre, lab) == pb);
        }
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0) wdeg[v] = (int)c;
    }
}

// Order-preserving fill: the lanes keep 32 consecutive entries per step and
// place the kept ones by a ballot prefix.
__global__ void wk_fill_kernel(int n, int u, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                               const int32_t *__restrict__ bpar, const int32_t *__restrict__ pre,
                               const int32_t *__restrict__ lab, const int32_t *__restrict__ wrp, int32_t *wci,
                               int32_t *wmap)
{
    const int lane = threadIdx.x & 31;
    for (int v = warp_id_global(); v < n; v += warps_global()) {
        if (v == u) continue;
        const int pb = lab[v];
        int o = wrp[v];
        const int o1 = wrp[v + 1], e1 = rp[v + 1];
        for (int e0 = rp[v]; e0 < e1; e0 += 32) {  // uniform per warp
            const int e = e0 + lane;
            const int w = (e < e1) ? ci[e] : -1;
            const bool keep = w >= 0 && block_of(v, w, bpar, pre, lab) == pb;
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            const int at = o + __popc(m & ((1u << lane) - 1u));
            if (keep && at < o1) {
                wci[at] = w;
                wmap[at] = e;
            }
            o += __popc(m);
        }
    }
}

__global__ void wk_scatter_kernel(int64_t wnnz, const int32_t *__restrict__ wmap, const int64_t *__restrict__ src,
                                  int64_t *dst)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < wnnz; j += (int64_t)gridDim.x * blockDim.x)
        dst[wmap[j]] = src[j];
}

}  // namespace

int select_pivot(Ctx *c, int n, const int32_t *d_rp, const int32_t *d_ci, int sweeps, int start, int32_t *pivot,
                 int32_t *bound)
{
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, (int64_t)c->num_sms * 8);
    int32_t *d_dist = nullptr, *d_bpar = nullptr, *d_lb = nullptr;
    unsigned long long *d_words = nullptr;  // [0] packed key, [1] BFS flag and unreached flag
    auto release = [&]() {
        cudaFree(d_dist);
        cudaFree(d_bpar);
        cudaFree(d_lb);
        cudaFree(d_words);
    };
    if (cudaMalloc(&d_dist, (size_t)n * 4) != cudaSuccess || cudaMalloc(&d_bpar, (size_t)n * 4) != cudaSuccess ||
        cudaMalloc(&d_lb, (size_t)n * 4) != cudaSuccess || cudaMalloc(&d_words, 4 * sizeof(unsigned long long)) != cudaSuccess) {
        release();
        return fail(c, UST_ENOMEM, "pivot selection buffers");
    }
    int rc = UST_OK;
    unsigned long long key = 0ull;
    int32_t h_flag = 0;
    int32_t *d_flag = reinterpret_cast<int32_t *>(d_words + 1);
    int *d_bad = reinterpret_cast<int *>(d_words + 2);
#define SP_TRY(call)                                                                    \
    do {                                                                                \
        const cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                        \
            rc = fail(c, UST_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
            goto done;                                                                  \
        }                                                                               \
    } while (0)
    {
        SP_TRY(cudaMemsetAsync(d_lb, 0, (size_t)n * 4, c->stream));
        SP_TRY(cudaMemsetAsync(d_words, 0, 4 * sizeof(unsigned long long), c->stream));
        int s = start;
        if (s < 0) {
            max_degree_kernel<<<blocks, threads, 0, c->stream>>>(n, d_rp, d_words);
            SP_TRY(cudaGetLastError());
            SP_TRY(cudaMemcpyAsync(&key, d_words, sizeof(key), cudaMemcpyDeviceToHost, c->stream));
            SP_TRY(cudaStreamSynchronize(c->stream));
            s = 0x7FFFFFFF - (int)(uint32_t)(key & 0xFFFFFFFFull);
        }
        for (int sweep = 0; sweep < sweeps; ++sweep) {
            bfs_init_kernel<<<blocks, threads, 0, c->stream>>>(n, s, d_dist, d_bpar);
            for (int level = 0;; ++level) {
                if (level > n) {
                    rc = fail(c, UST_ETIMEOUT, "BFS did not terminate");
                    goto done;
                }
                SP_TRY(cudaMemsetAsync(d_flag, 0, sizeof(int32_t), c->stream));
                bfs_pull_kernel<<<blocks, threads, 0, c->stream>>>(n, level, d_rp, d_ci, d_dist, d_bpar, d_flag);
                SP_TRY(cudaGetLastError());
                SP_TRY(cudaMemcpyAsync(&h_flag, d_flag, sizeof(h_flag), cudaMemcpyDeviceToHost, c->stream));
                SP_TRY(cudaStreamSynchronize(c->stream));
                if (h_flag == 0) break;
            }
            SP_TRY(cudaMemsetAsync(d_words, 0, sizeof(unsigned long long), c->stream));
            sweep_update_kernel<<<blocks, threads, 0, c->stream>>>(n, d_dist, d_lb, d_words, d_bad);
            SP_TRY(cudaGetLastError());
            int bad = 0;
            SP_TRY(cudaMemcpyAsync(&key, d_words, sizeof(key), cudaMemcpyDeviceToHost, c->stream));
            SP_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, c->stream));
            SP_TRY(cudaStreamSynchronize(c->stream));
            if (bad) {
                rc = fail(c, UST_ENOTCONNECTED, "graph is not connected");
                goto done;
            }
            s = 0x7FFFFFFF - (int)(uint32_t)(key & 0xFFFFFFFFull);  // the next source: the farthest vertex
        }
        SP_TRY(cudaMemsetAsync(d_words, 0xFF, sizeof(unsigned long long), c->stream));
        min_bound_kernel<<<blocks, threads, 0, c->stream>>>(n, d_lb, d_words);
        SP_TRY(cudaGetLastError());
        SP_TRY(cudaMemcpyAsync(&key, d_words, sizeof(key), cudaMemcpyDeviceToHost, c->stream));
        SP_TRY(cudaStreamSynchronize(c->stream));
        *pivot = (int32_t)(uint32_t)(key & 0xFFFFFFFFull);
        *bound = (int32_t)(key >> 32);
    }
#undef SP_TRY
done:
    release();
    return rc;
}

int check_graph(Ctx *c, int n, int nnz, const int32_t *d_rp, const int32_t *d_ci, int *d_bad)
{
    const int threads = 256;
    const int rows = (int)std::min<int64_t>((n + threads - 1) / threads, (int64_t)c->num_sms * 8);
    const int arcs = (int)std::min<int64_t>(((int64_t)nnz + threads - 1) / threads, (int64_t)c->num_sms * 16);
    int bad = 0;
    UST_CUDA_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream));
    check_rows_kernel<<<std::max(1, rows), threads, 0, c->stream>>>(n, nnz, d_rp, d_bad);
    c->launches += 1;
    UST_CUDA_TRY(cudaGetLastError());
    UST_CUDA_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (bad & kBadBounds) return fail(c, UST_EINVAL, "row_ptr must run from 0 to nnz and be monotone");
    check_arcs_kernel<<<std::max(1, arcs), threads, 0, c->stream>>>(n, nnz, d_rp, d_ci, d_bad);
    c->launches += 1;
    UST_CUDA_TRY(cudaGetLastError());
    UST_CUDA_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (bad & kBadRange) return fail(c, UST_EINVAL, "column index out of range");
    if (bad & kBadLoop) return fail(c, UST_EINVAL, "self-loop");
    if (bad & kBadOrder) return fail(c, UST_EINVAL, "row not strictly increasing");
    if (bad & kBadSymmetry) return fail(c, UST_EINVAL, "CSR is not symmetric");
    if (bad & kIsolated) return fail(c, UST_ENOTCONNECTED, "isolated vertex");
    return UST_OK;
}

// Small graphs: one CTA does the BFS, the prefix and the paths in one
// launch; a second launch only when the path space has to grow.
int run_bfs_small(Ctx *c)
{
    int32_t *h_out = reinterpret_cast<int32_t *>(c->h_stats);
    phase_begin(c, Ctx::kEvBfs);
    for (int attempt = 0; attempt < 2; ++attempt) {
        PrepDesc d;
        d.n = c->n;
        d.u = c->pivot;
        d.rp = c->d_rp;
        d.ci = c->d_ci;
        d.dist = c->d_dist;
        d.bpar = c->d_bpar;
        d.pathptr = c->d_pathptr;
        d.path = c->d_path;
        d.pchild = c->d_path ? c->d_path + c->path_cap : nullptr;
        d.powner = c->d_path ? c->d_path + 2 * c->path_cap : nullptr;
        d.path_cap = c->d_path ? c->path_cap : 0;
        UST_CUDA_TRY(cudaMemsetAsync(c->d_flag, 0, 3 * sizeof(int32_t), c->stream));
        const int rc = run_prepare_single(c, d, c->d_flag);
        if (rc) return rc;
        UST_CUDA_TRY(cudaMemcpyAsync(h_out, c->d_flag, 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (h_out[0] & 1) return fail(c, UST_ENOTCONNECTED, "graph is not connected");
        c->ecc = h_out[1];
        c->farness = h_out[2];
        if (!(h_out[0] & 2)) break;  // the paths are in place
        if (attempt == 1) return fail(c, UST_ECUDA, "B_u: path space mismatch");
        cudaFree(c->d_path);
        c->d_path = nullptr;
        c->path_cap = 0;
        if (cudaMalloc(&c->d_path, 3 * (size_t)c->farness * sizeof(int32_t)) != cudaSuccess)
            return fail(c, UST_ENOMEM, "BFS paths");
        c->path_cap = c->farness;
    }
    phase_end(c, Ctx::kEvBfs);
    return UST_OK;
}

cudaError_t launch_exclusive_scan(int n, const int32_t *in, int32_t *out, cudaStream_t st)
{
    path_offsets_kernel<<<1, kScanThreads, 0, st>>>(n, in, out);
    return cudaGetLastError();
}

int run_bfs(Ctx *c)
{
    if (c->n <= kPrepMaxN) return run_bfs_small(c);
    const int n = c->n;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, (int64_t)c->num_sms * 8);
    phase_begin(c, Ctx::kEvBfs);
    bfs_init_kernel<<<blocks, threads, 0, c->stream>>>(n, c->pivot, c->d_dist, c->d_bpar);
    c->launches += 1;
    UST_CUDA_TRY(cudaGetLastError());
    int32_t *h_found = reinterpret_cast<int32_t *>(c->h_stats);
    int level = 0;
    for (;; ++level) {
        if (level > n) return fail(c, UST_ETIMEOUT, "BFS did not terminate");
        UST_CUDA_TRY(cudaMemsetAsync(c->d_flag, 0, sizeof(int32_t), c->stream));
        bfs_pull_kernel<<<blocks, threads, 0, c->stream>>>(n, level, c->d_rp, c->d_ci, c->d_dist,
                                                           c->d_bpar, c->d_flag);
        c->launches += 1;
        UST_CUDA_TRY(cudaGetLastError());
        UST_CUDA_TRY(cudaMemcpyAsync(h_found, c->d_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (*h_found == 0) break;
    }
    c->ecc = level;
    unsigned long long *d_sum = reinterpret_cast<unsigned long long *>(c->d_stats);
    UST_CUDA_TRY(cudaMemsetAsync(d_sum, 0, 2 * sizeof(unsigned long long), c->stream));
    bfs_sum_kernel<<<blocks, threads, 0, c->stream>>>(n, c->d_dist, d_sum);
    c->launches += 1;
    phase_end(c, Ctx::kEvBfs);
    UST_CUDA_TRY(cudaGetLastError());
    UST_CUDA_TRY(cudaMemcpyAsync(c->h_stats, d_sum, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                 c->stream));
    UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (c->h_stats[1] != 0) return fail(c, UST_ENOTCONNECTED, "graph is not connected");
    c->farness = c->h_stats[0];
    // the BFS paths P(v), flattened: sum_v dist(u, v) = f^c(u) entries
    if (c->farness > 0x7FFFFFFFll) return fail(c, UST_EINVAL, "f^c(u) exceeds 2^31 path entries");
    if (c->farness > c->path_cap) {
        cudaFree(c->d_path);
        c->d_path = nullptr;
        c->path_cap = 0;
        if (cudaMalloc(&c->d_path, 3 * (size_t)c->farness * sizeof(int32_t)) != cudaSuccess)
            return fail(c, UST_ENOMEM, "BFS paths");
        c->path_cap = c->farness;
    }
    path_offsets_kernel<<<1, kScanThreads, 0, c->stream>>>(n, c->d_dist, c->d_pathptr);
    path_fill_kernel<<<blocks, threads, 0, c->stream>>>(n, c->pivot, c->d_bpar, c->d_pathptr, c->d_path,
                                                        c->d_path + c->path_cap, c->d_path + 2 * c->path_cap);
    c->launches += 2;
    UST_CUDA_TRY(cudaGetLastError());
    return UST_OK;
}


int build_block_rows(Ctx *c)
{
    const int n = c->n, u = c->pivot;
    if (!c->d_wrp) {
        if (cudaMalloc(&c->d_wrp, ((size_t)n + 1) * 4) != cudaSuccess ||
            cudaMalloc(&c->d_wci, (size_t)c->nnz * 4) != cudaSuccess ||
            cudaMalloc(&c->d_wmap, (size_t)c->nnz * 4) != cudaSuccess)
            return fail(c, UST_ENOMEM, "block-restricted rows");
    }
    if (!c->d_bscratch && cudaMalloc(&c->d_bscratch, 6 * (size_t)n * 4) != cudaSuccess)
        return fail(c, UST_ENOMEM, "block labels");  // kept: a later ust_reset allocates nothing
    int32_t *s = c->d_bscratch;
    int32_t *nd = s, *pre = s + n, *cur = s + 2 * (size_t)n, *lo = s + 3 * (size_t)n, *hi = s + 4 * (size_t)n,
            *uf = s + 5 * (size_t)n;
    int32_t *lab = cur, *wdeg = lo;  // cur and lo are free again by then
    int *d_bad = c->d_flag;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, (int64_t)c->num_sms * 8);
    // one warp per row in the row scans
    const int wblocks = (int)std::min<int64_t>(((int64_t)n * 32 + threads - 1) / threads, (int64_t)c->num_sms * 16);
    cudaStream_t st = c->stream;
    int rc = UST_OK;
    int64_t launches = 0;
#define BT_TRY(call)                                                                     \
    do {                                                                                 \
        const cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                         \
            rc = fail(c, UST_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
            goto done;                                                                   \
        }                                                                                \
    } while (0)
    BT_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
    bt_init_kernel<<<blocks, threads, 0, st>>>(n, u, nd, pre, cur, uf);
    ++launches;
    for (int level = c->ecc; level >= 1; --level, ++launches)
        bt_size_kernel<<<blocks, threads, 0, st>>>(n, level, c->d_dist, c->d_bpar, nd);
    for (int level = 1; level <= c->ecc; ++level, ++launches)
        bt_pre_kernel<<<blocks, threads, 0, st>>>(n, level, c->d_dist, c->d_bpar, nd, pre, cur);
    bt_local_kernel<<<wblocks, threads, 0, st>>>(n, c->d_rp, c->d_ci, c->d_bpar, pre, lo, hi);
    ++launches;
    for (int level = c->ecc; level >= 1; --level, ++launches)
        bt_lohi_kernel<<<blocks, threads, 0, st>>>(n, level, c->d_dist, c->d_bpar, lo, hi);
    bt_rule1_kernel<<<wblocks, threads, 0, st>>>(n, c->d_rp, c->d_ci, c->d_bpar, pre, nd, uf, d_bad);
    bt_rule2_kernel<<<blocks, threads, 0, st>>>(n, u, c->d_bpar, pre, nd, lo, hi, uf, d_bad);
    bt_label_kernel<<<blocks, threads, 0, st>>>(n, uf, lab, d_bad);
    wk_count_kernel<<<wblocks, threads, 0, st>>>(n, u, c->d_rp, c->d_ci, c->d_bpar, pre, lab, wdeg);
    path_offsets_kernel<<<1, kScanThreads, 0, st>>>(n, wdeg, c->d_wrp);
    wk_fill_kernel<<<wblocks, threads, 0, st>>>(n, u, c->d_rp, c->d_ci, c->d_bpar, pre, lab, c->d_wrp, c->d_wci,
                                               c->d_wmap);
    launches += 6;
    BT_TRY(cudaGetLastError());
    {
        int32_t *h = reinterpret_cast<int32_t *>(c->h_stats);
        BT_TRY(cudaMemcpyAsync(h, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        BT_TRY(cudaMemcpyAsync(h + 1, c->d_wrp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        BT_TRY(cudaStreamSynchronize(st));
        if (h[0] != 0) {
            rc = fail(c, UST_ECUDA, "block labels: union-find bound reached");
            goto done;
        }
        if (h[1] < n - 1 || h[1] > c->nnz) {
            rc = fail(c, UST_ECUDA, "block-restricted rows: inconsistent arc count");
            goto done;
        }
        c->wnnz = h[1];
    }
done:
#undef BT_TRY
    c->launches += launches;
    cudaStreamSynchronize(st);
    return rc;
}

int scatter_block_counts(Ctx *c, const int64_t *d_walk_counts, int64_t *d_out)
{
    UST_CUDA_TRY(cudaMemsetAsync(d_out, 0, (size_t)c->nnz * sizeof(int64_t), c->stream));
    const int threads = 256;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((c->wnnz + threads - 1) / threads,
                                                                   (int64_t)c->num_sms * 8));
    wk_scatter_kernel<<<blocks, threads, 0, c->stream>>>(c->wnnz, c->d_wmap, d_walk_counts, d_out);
    c->launches += 1;
    UST_CUDA_TRY(cudaGetLastError());
    return UST_OK;
}

}  // namespace ust
