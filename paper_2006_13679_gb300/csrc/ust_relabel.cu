// The large-graph sampler's view of a single graph: the vertices relabelled
// in Cuthill-McKee order from the pivot.
//
// The large-graph sampler keeps a tree's per-vertex state in global memory,
// far larger than L2, so its speed is the rate of random accesses that L1
// and L2 serve. Wilson's walks, the peeling, the subtree sizes and the
// interval tests of Algorithm 2 all move along edges, so an order in which
// neighbours get nearby ids puts the entries one step touches in the same
// cache lines. Cuthill-McKee order is a breadth-first order from the pivot
// in which the vertices that vertex x discovers follow one another, by
// increasing degree (ties: smaller input id). Measured on GB300 against the
// input order with the highest-degree vertices first: 9% faster on R-MAT
// scale 22, 52% on a 2^20-vertex random hyperbolic graph (whose input ids
// carry no locality); a plain breadth-first order gained 4% and 39%, a
// depth-first order of the BFS tree -8% and 44%.
//
// Built on the device, deterministically, level by level of the BFS from the
// pivot (the B_u of ust_init): vertex w at distance d+1 is discovered by its
// neighbour at distance d of least new id, m(w); the vertices of level d+1
// take the next ids in order of (m(w), degree, input id). A stable LSD radix
// sort over 8-bit digits gives that order.
//
// Pendant vertices (degree 1, not the pivot, next to a vertex of degree 2 or
// more) then move behind the others, keeping their order: the sampler builds
// its trees on the core below them and derives their counts (see
// GraphDesc::ncore). On R-MAT graphs they are about a fifth of the vertices.
//
// Nothing the method computes changes: row v' of the relabelled CSR lists the
// same neighbours as input row orig[v'], in the same (input) order, so draw k
// of a vertex picks the same neighbour, and the sampler keys its Philox
// counters by the input id. B_u, the column solve and every output stay in
// input ids. ust_reset to another pivot keeps the order of the first.
#include <algorithm>
#include <vector>

#include "ust_common.cuh"

namespace ust {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortChunks = 8;  // items per thread and tile
constexpr int kSortTile = kSortThreads * kSortChunks;
constexpr int kBins = 256;      // 8-bit digits

int tiles_of(int count) { return (count + kSortTile - 1) / kSortTile; }

// hist[d * tiles + b]: items of tile b whose digit at `shift` is d.
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(int count, const unsigned long long *__restrict__ keys,
                                                                  int shift, int32_t *__restrict__ hist)
{
    __shared__ int h[kBins];
    for (int d = threadIdx.x; d < kBins; d += kSortThreads) h[d] = 0;
    __syncthreads();
    const int b = blockIdx.x, begin = b * kSortTile, end = min(count, begin + kSortTile);
    for (int i = begin + threadIdx.x; i < end; i += kSortThreads) atomicAdd(&h[(int)((keys[i] >> shift) & (kBins - 1))], 1);
    __syncthreads();
    for (int d = threadIdx.x; d < kBins; d += kSortThreads) hist[d * gridDim.x + b] = h[d];
}

// Stable scatter of tile b: offs[d * tiles + b] is where its first item of
// digit d goes (the exclusive scan of hist). The tile is taken in chunks of
// one item per thread, in index order; inside a chunk an item's rank among
// the equal digits before it comes from its warp's match mask and the counts
// of the warps before it (stamped with the chunk, so that no clearing is
// needed between chunks).
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(int count, const unsigned long long *__restrict__ keys,
                                                                     const int32_t *__restrict__ vals, int shift,
                                                                     const int32_t *__restrict__ offs,
                                                                     unsigned long long *__restrict__ okeys,
                                                                     int32_t *__restrict__ ovals)
{
    constexpr int kWarps = kSortThreads / 32;
    __shared__ int base[kBins];
    __shared__ int wcnt[kWarps][kBins];  // (chunk + 1) << 8 | items of the digit in the warp
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, b = blockIdx.x;
    for (int d = tid; d < kBins; d += kSortThreads) base[d] = offs[d * gridDim.x + b];
    for (int e = tid; e < kWarps * kBins; e += kSortThreads) wcnt[e / kBins][e % kBins] = 0;
    __syncthreads();
    for (int c = 0; c < kSortChunks; ++c) {
        const int i = b * kSortTile + c * kSortThreads + tid;
        const bool ok = i < count;
        const unsigned long long k = ok ? keys[i] : 0ull;
        const int32_t v = ok ? vals[i] : 0;
        const int d = ok ? (int)((k >> shift) & (kBins - 1)) : kBins;  // kBins: no item
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int stamp = (c + 1) << 8;
        if (ok && lane == __ffs(peers) - 1) wcnt[warp][d] = stamp | __popc(peers);
        __syncthreads();
        int r = 0;
        bool last = false;  // the chunk's last item of digit d moves base[d] on
        if (ok) {
            r = base[d] + __popc(peers & ((1u << lane) - 1u));
            for (int w = 0; w < warp; ++w) {
                const int e = wcnt[w][d];
                if ((e & ~0xFF) == stamp) r += e & 0xFF;
            }
            last = lane == 31 - __clz(peers);
            for (int w = warp + 1; w < kWarps; ++w)
                if ((wcnt[w][d] & ~0xFF) == stamp) last = false;
            okeys[r] = k;
            ovals[r] = v;
        }
        __syncthreads();
        if (last) base[d] = r + 1;
        __syncthreads();
    }
}

// Sorts (keys, vals)[0, count) by the low `bits` bits of the keys, stably;
// the result ends in keys/vals (the buffers swap with the spare pair).
int radix_sort(Ctx *c, int count, int bits, unsigned long long *&keys, int32_t *&vals, unsigned long long *&keys2,
               int32_t *&vals2, int32_t *hist, int32_t *offs)
{
    if (count <= 1) return UST_OK;
    const int tiles = tiles_of(count);
    for (int shift = 0; shift < bits; shift += 8) {
        radix_hist_kernel<<<tiles, kSortThreads, 0, c->stream>>>(count, keys, shift, hist);
        UST_CUDA_TRY(cudaGetLastError());
        UST_CUDA_TRY(launch_exclusive_scan(kBins * tiles, hist, offs, c->stream));
        radix_scatter_kernel<<<tiles, kSortThreads, 0, c->stream>>>(count, keys, vals, shift, offs, keys2, vals2);
        UST_CUDA_TRY(cudaGetLastError());
        c->launches += 3;
        std::swap(keys, keys2);
        std::swap(vals, vals2);
    }
    return UST_OK;
}

int bits_for(long long x)  // bits that hold 0 .. x
{
    int b = 0;
    while (b < 63 && (x >> b) != 0) ++b;
    return std::max(b, 1);
}

// keys[v] = dist(v), vals[v] = v: the vertices by level, input id inside a level
__global__ void level_keys_kernel(int n, const int32_t *__restrict__ dist, unsigned long long *__restrict__ keys,
                                  int32_t *__restrict__ vals)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        keys[v] = (unsigned long long)dist[v];
        vals[v] = v;
    }
}

// first[l] = position of the first vertex of level l < levels in the sorted list
__global__ void level_starts_kernel(int n, int levels, const unsigned long long *__restrict__ keys,
                                    int32_t *__restrict__ first)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if ((i == 0 || keys[i] != keys[i - 1]) && keys[i] < (unsigned long long)levels) first[keys[i]] = i;
}

// One warp per vertex w of the next level (list[i], in input-id order): the
// key (m(w) - L_d) << 32 | degree(w), m(w) the least new id of w's
// neighbours on level d.
__global__ void cm_keys_kernel(int cnt, const int32_t *__restrict__ list, int level, int first_id, int level_size,
                               const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                               const int32_t *__restrict__ dist, const int32_t *__restrict__ newid,
                               unsigned long long *__restrict__ keys, int32_t *__restrict__ vals, int *bad)
{
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < cnt; i += warps) {
        const int w = list[i];
        const int b = rp[w], e = rp[w + 1];
        int m = 0x7FFFFFFF;
        for (int k = b + lane; k < e; k += 32) {
            const int x = ci[k];
            if (dist[x] == level) m = min(m, newid[x]);
        }
        m = __reduce_min_sync(0xffffffffu, m);
        if (lane == 0) {
            if (m < first_id || m - first_id >= level_size) {  // the BFS levels are inconsistent
                *bad = 1;
                m = first_id;
            }
            keys[i] = ((unsigned long long)(m - first_id) << 32) | (unsigned long long)(uint32_t)(e - b);
            vals[i] = w;
        }
    }
}

__global__ void cm_assign_kernel(int cnt, int first_new, const int32_t *__restrict__ vals, int32_t *__restrict__ orig,
                                 int32_t *__restrict__ newid)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const int w = vals[i];
        orig[first_new + i] = w;
        newid[w] = first_new + i;
    }
}

// keys[i] = 1 when orig[i] is a pendant vertex: degree 1, not the pivot, and
// its neighbour of degree 2 or more (vals[i] = orig[i]); *count += pendants
__global__ void pendant_keys_kernel(int n, int u, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                    const int32_t *__restrict__ orig, unsigned long long *__restrict__ keys,
                                    int32_t *__restrict__ vals, int *count)
{
    int mine = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int v = orig[i];
        const int b = rp[v];
        bool pend = false;
        if (v != u && rp[v + 1] - b == 1) {
            const int w = ci[b];
            pend = rp[w + 1] - rp[w] >= 2;
        }
        keys[i] = pend ? 1ull : 0ull;
        vals[i] = v;
        mine += pend ? 1 : 0;
    }
    mine = __reduce_add_sync(0xffffffffu, mine);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(count, mine);
}

// deg[i] = degree of orig[i]; bad when orig is not the inverse of newid
__global__ void relabel_degrees_kernel(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ orig,
                                       const int32_t *__restrict__ newid, int32_t *__restrict__ deg, int *bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int o = orig[i];
        if (o < 0 || o >= n || newid[o] != i) {
            *bad = 1;
            deg[i] = 0;
            continue;
        }
        deg[i] = rp[o + 1] - rp[o];
    }
}

// One warp per relabelled row: sci[srp[v] + k] = newid[ci[rp[orig[v]] + k]].
__global__ void relabel_rows_kernel(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                    const int32_t *__restrict__ srp, const int32_t *__restrict__ orig,
                                    const int32_t *__restrict__ newid, int32_t *__restrict__ sci)
{
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        const int o = orig[v];
        const int src = rp[o], len = rp[o + 1] - src, dst = srp[v];
        for (int k = lane; k < len; k += 32) sci[dst + k] = newid[ci[src + k]];
    }
}

// len[v] = |P(orig[v])| = dist(orig[v])
__global__ void spath_lengths_kernel(int n, const int32_t *__restrict__ orig, const int32_t *__restrict__ dist,
                                     int32_t *__restrict__ len)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) len[v] = dist[orig[v]];
}

// The flattened BFS paths in sampler ids and sampler order: the path of
// sampler vertex v at spathptr[v], its entries in the input path's order;
// entry q is the edge (spath[q], spchild[q]) of the path of spowner[q].
__global__ void relabel_path_kernel(int n, const int32_t *__restrict__ orig, const int32_t *__restrict__ pathptr,
                                    const int32_t *__restrict__ path, const int32_t *__restrict__ pchild,
                                    const int32_t *__restrict__ spathptr, const int32_t *__restrict__ newid,
                                    int32_t *__restrict__ spath, int32_t *__restrict__ spchild,
                                    int32_t *__restrict__ spowner)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int o = orig[v];
        const int src = pathptr[o], len = pathptr[o + 1] - src, dst = spathptr[v];
        for (int k = 0; k < len; ++k) {
            spath[dst + k] = newid[path[src + k]];
            spchild[dst + k] = newid[pchild[src + k]];
            spowner[dst + k] = v;
        }
    }
}

}  // namespace

int build_relabel(Ctx *c)
{
    const int n = c->n, u = c->pivot, ecc = c->ecc;
    if (ecc < 1 || ecc >= n) return fail(c, UST_ECUDA, "relabelling: BFS levels missing");
    if (cudaMalloc(&c->d_srp, ((size_t)n + 1) * 4) != cudaSuccess ||
        cudaMalloc(&c->d_sci, (size_t)c->nnz * 4) != cudaSuccess || cudaMalloc(&c->d_orig, (size_t)n * 4) != cudaSuccess ||
        cudaMalloc(&c->d_newid, (size_t)n * 4) != cudaSuccess ||
        cudaMalloc(&c->d_spathptr, ((size_t)n + 1) * 4) != cudaSuccess)
        return fail(c, UST_ENOMEM, "relabelled graph of the sampler");
    // scratch of the construction: two (key, value) pairs of n, the level
    // list, histogram and offsets, the level starts and a flag
    const size_t hist_n = (size_t)kBins * tiles_of(n) + 1;
    char *scratch = nullptr;
    const size_t bytes = 2 * (size_t)n * 8 + 3 * (size_t)n * 4 + 2 * hist_n * 4 + ((size_t)ecc + 2) * 4 + 16;
    if (cudaMalloc(&scratch, bytes) != cudaSuccess) return fail(c, UST_ENOMEM, "relabelling scratch");
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(scratch);
    unsigned long long *keys2 = keys + n;
    int32_t *vals = reinterpret_cast<int32_t *>(keys2 + n);
    int32_t *vals2 = vals + n;
    int32_t *list = vals2 + n;
    int32_t *hist = list + n;
    int32_t *offs = hist + hist_n;
    int32_t *first = offs + hist_n;
    int *d_bad = first + ecc + 2;
    int rc = UST_OK;
    cudaStream_t st = c->stream;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, (int64_t)c->num_sms * 8);
    const int wblocks_cap = c->num_sms * 16;
    std::vector<int32_t> h_first((size_t)ecc + 2);
    int h_bad[2] = {0, 0};
#define RL_TRY(call)                                                                     \
    do {                                                                                 \
        const cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                         \
            rc = fail(c, UST_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
            goto done;                                                                   \
        }                                                                                \
    } while (0)
#define RL_RC(call)             \
    do {                        \
        rc = (call);            \
        if (rc != UST_OK) goto done; \
    } while (0)
    RL_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
    // the vertices by BFS level (input ids ascending inside a level)
    level_keys_kernel<<<blocks, threads, 0, st>>>(n, c->d_dist, keys, vals);
    RL_TRY(cudaGetLastError());
    RL_RC(radix_sort(c, n, bits_for(ecc), keys, vals, keys2, vals2, hist, offs));
    RL_TRY(cudaMemcpyAsync(list, vals, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    RL_TRY(cudaMemsetAsync(first, 0xFF, ((size_t)ecc + 2) * 4, st));
    level_starts_kernel<<<blocks, threads, 0, st>>>(n, ecc + 1, keys, first);
    RL_TRY(cudaGetLastError());
    RL_TRY(cudaMemcpyAsync(h_first.data(), first, ((size_t)ecc + 1) * 4, cudaMemcpyDeviceToHost, st));
    RL_TRY(cudaStreamSynchronize(st));
    h_first[ecc + 1] = n;
    for (int l = 0; l <= ecc; ++l)
        if (h_first[l] < 0 || h_first[l] >= h_first[l + 1] || (l == 0 && h_first[1] != 1)) {
            rc = fail(c, UST_ECUDA, "relabelling: a BFS level is empty");
            goto done;
        }
    // level 0 is the pivot; level d + 1 in order of (m(w), degree, input id)
    RL_TRY(cudaMemcpyAsync(c->d_orig, &u, 4, cudaMemcpyHostToDevice, st));
    RL_TRY(cudaMemsetAsync(c->d_newid + u, 0, 4, st));
    for (int d = 0; d < ecc; ++d) {
        const int cnt = h_first[d + 2] - h_first[d + 1];
        const int level_size = h_first[d + 1] - h_first[d];
        const int wb = (int)std::min<int64_t>(((int64_t)cnt * 32 + threads - 1) / threads, (int64_t)wblocks_cap);
        cm_keys_kernel<<<wb, threads, 0, st>>>(cnt, list + h_first[d + 1], d, h_first[d], level_size, c->d_rp, c->d_ci, c->d_dist,
                                               c->d_newid, keys, vals, d_bad);
        RL_TRY(cudaGetLastError());
        RL_RC(radix_sort(c, cnt, 32 + bits_for(level_size - 1), keys, vals, keys2, vals2, hist, offs));
        const int ab = (int)std::min<int64_t>((cnt + threads - 1) / threads, (int64_t)c->num_sms * 8);
        cm_assign_kernel<<<ab, threads, 0, st>>>(cnt, h_first[d + 1], vals, c->d_orig, c->d_newid);
        RL_TRY(cudaGetLastError());
        c->launches += 2;
    }
    // pendant vertices after the core, each part in the order above
    RL_TRY(cudaMemsetAsync(d_bad + 1, 0, sizeof(int), st));
    pendant_keys_kernel<<<blocks, threads, 0, st>>>(n, u, c->d_rp, c->d_ci, c->d_orig, keys, vals, d_bad + 1);
    RL_TRY(cudaGetLastError());
    RL_RC(radix_sort(c, n, 1, keys, vals, keys2, vals2, hist, offs));
    cm_assign_kernel<<<blocks, threads, 0, st>>>(n, 0, vals, c->d_orig, c->d_newid);
    RL_TRY(cudaGetLastError());
    c->launches += 2;
    // row pointers of the new order, checked to be a permutation on the way
    relabel_degrees_kernel<<<blocks, threads, 0, st>>>(n, c->d_rp, c->d_orig, c->d_newid, vals, d_bad);
    RL_TRY(cudaGetLastError());
    RL_TRY(launch_exclusive_scan(n, vals, c->d_srp, st));
    RL_TRY(cudaMemcpyAsync(h_bad, d_bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    RL_TRY(cudaStreamSynchronize(st));
    if (h_bad[0] || h_bad[1] < 0 || h_bad[1] >= n) {
        rc = fail(c, UST_ECUDA, "relabelling is not a permutation of the vertices");
        goto done;
    }
    relabel_rows_kernel<<<(int)std::min<int64_t>(((int64_t)n * 32 + threads - 1) / threads, (int64_t)wblocks_cap),
                          threads, 0, st>>>(n, c->d_rp, c->d_ci, c->d_srp, c->d_orig, c->d_newid, c->d_sci);
    RL_TRY(cudaGetLastError());
    c->launches += 5;
    RL_TRY(cudaStreamSynchronize(st));  // the scratch is freed below
    c->relabel_core = n - h_bad[1];
    c->relabel = true;
done:
#undef RL_TRY
#undef RL_RC
    cudaStreamSynchronize(st);
    cudaFree(scratch);
    return rc;
}

int relabel_paths(Ctx *c)
{
    if (!c->relabel) return UST_OK;
    if (c->farness > c->spath_cap) {
        cudaFree(c->d_spath);
        c->d_spath = nullptr;
        c->spath_cap = 0;
        if (cudaMalloc(&c->d_spath, 3 * (size_t)std::max<int64_t>(1, c->farness) * 4) != cudaSuccess)
            return fail(c, UST_ENOMEM, "BFS paths in sampler ids");
        c->spath_cap = c->farness;
    }
    const int n = c->n;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, (int64_t)c->num_sms * 8);
    // the path lengths go through the counts scratch (n int64, free here)
    int32_t *len = reinterpret_cast<int32_t *>(c->d_Rtmp);
    spath_lengths_kernel<<<blocks, threads, 0, c->stream>>>(n, c->d_orig, c->d_dist, len);
    UST_CUDA_TRY(cudaGetLastError());
    UST_CUDA_TRY(launch_exclusive_scan(n, len, c->d_spathptr, c->stream));
    relabel_path_kernel<<<blocks, threads, 0, c->stream>>>(n, c->d_orig, c->d_pathptr, c->d_path,
                                                           c->d_path + c->path_cap, c->d_spathptr, c->d_newid,
                                                           c->d_spath, c->d_spath + c->spath_cap,
                                                           c->d_spath + 2 * c->spath_cap);
    c->launches += 3;
    UST_CUDA_TRY(cudaGetLastError());
    int32_t sp = 0;
    UST_CUDA_TRY(cudaMemcpyAsync(&sp, c->d_newid + c->pivot, sizeof(sp), cudaMemcpyDeviceToHost, c->stream));
    UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->spivot = sp;
    // a pivot that is itself pendant (after ust_reset) keeps every vertex in the trees
    c->ncore = sp < c->relabel_core ? c->relabel_core : n;
    int32_t fc = 0;
    UST_CUDA_TRY(cudaMemcpyAsync(&fc, c->d_spathptr + c->ncore, sizeof(fc), cudaMemcpyDeviceToHost, c->stream));
    UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->core_fc = fc;
    return UST_OK;
}

}  // namespace ust
