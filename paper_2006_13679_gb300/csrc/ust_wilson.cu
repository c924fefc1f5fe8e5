// Sampling and aggregation: the loop of Algorithm 1 that samples a uniform
// spanning tree T rooted at u (Wilson's algorithm, Appendix A.2) and adds
// its Algorithm 2 counts to R.
//
// One CTA owns one tree at a time and takes work items (graph, tree) from a
// global counter (persistent kernel). Two kernels share the method:
// sample_aggregate_smem_kernel (graphs up to 65,535 vertices, per-tree words
// in shared memory) and sample_aggregate_large_kernel (larger graphs, per-tree
// records in the CTA's workspace, the highest-degree vertices' counters in
// shared memory). Per tree:
//
//  1. Cycle popping (Wilson's cycle-popping theorem, used in Appendix A.2).
//     Every vertex v != u has a stack of random neighbours, entry k being the
//     Philox draw keyed by (v, k, tree, graph); the stack tops form a
//     functional graph whose sink is u. Popping every cycle until none is
//     left gives the same tree as the loop-erased walks, whatever the order.
//     - Round 0: the cycle vertices of the first functional graph are what
//       in-degree peeling leaves behind. Peeling is asynchronous: a vertex
//       whose in-degree drops to zero is continued by the thread that removed
//       its last in-edge, so it costs O(n) atomics and no barriers.
//     - Later rounds: every new cycle passes through a vertex redrawn in the
//       previous round. Each redrawn vertex x walks the stack tops until the
//       next redrawn vertex S(x) or a vertex known to reach u; a walk that
//       meets a vertex another walk of the round passed takes that walk's
//       result. Each node of the small graph x -> S(x) is classified by
//       Brent's cycle detection (reaches u, on a cycle, or runs into one); the
//       cycle segments are popped (every vertex on them advances to its next
//       stack entry), and the parts that reach u are marked final.
//  2. DFS intervals of T (Algorithm 2's discovery/finish times), without
//     level barriers: subtree sizes by a packed "pending children | summed
//     sizes" word where the last arriving child carries the sum upwards; the
//     same atomic gives each child its offset inside its parent's interval
//     (any child order gives valid nested intervals). Preorder numbers are
//     the root-path sums of the offsets: pointer jumping in shared memory
//     (smem kernel), or top-down over the log of the arrivals read backwards,
//     chunk by chunk (large kernel).
//  3. Algorithm 2 with the inclusive subtree test over the flattened BFS paths
//     P(v): one independent test per path entry (shallow paths) or a walk per
//     vertex (deep paths, and every path in the large kernel). Counts go to
//     the CTA's partial row, summed into the int64 R exactly by a second
//     kernel in a fixed order (batches: int64 atomics).
#include <algorithm>
#include <map>
#include <mutex>

#include "ust_common.cuh"

namespace ust {
namespace {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications, key bumped by the Weyl constants between
// rounds. Only the first two output words are needed.
__device__ __forceinline__ unsigned long long philox_x64(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                         uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        c0 = hi1 ^ c1 ^ k0;
        c2 = hi0 ^ c3 ^ k1;
        c1 = lo1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return ((unsigned long long)c1 << 32) | (unsigned long long)c0;
}

// One launch of the sampler: work item i of [0, total_items) is tree
// tree_offset + tree_begin + (i - item_start[g]) of graph graphs[g], where
// item_start[g] <= i < item_start[g + 1]. A single graph is a one-entry
// array; every launch reads its graphs from device memory.
struct SampleParams {
    int max_n;  // largest graph of the launch: shared-memory and partial-count sizes
    uint32_t key0, key1;
    const GraphDesc *graphs;
    int ngraphs;
    const long long *item_start;
    long long total_items;
    long long tree_offset;
    int32_t *ws;
    long long stride;
    int32_t *Rp;  // per-CTA partial counts (single graph), stride max_n
    unsigned long long *next_tree;
    unsigned long long *stats;  // [0] draws, [1] rounds, [2] max rounds, [3] max pops in one round
    int *status;
    int max_rounds, max_steps;
    int mode;  // 0: aggregate, 1: export trees
    int32_t *next_out, *pops_out;  // mode 1: item i's tree at [i n, (i + 1) n)
    unsigned long long *edge_counts;  // when set: +1 per tree at every arc v -> parent(v) (index aoff + arc)
    unsigned long long *R_direct;   // when set, counts go to R_direct[voff + v] (batches)
};

// item_start[1] of a one-graph launch: its items end at total_items.
constexpr long long kOpenEnd = 1ll << 62;

// The graph and tree id of a work item.
__device__ __forceinline__ bool item_graph(const SampleParams &p, long long item, GraphDesc &gd, long long &t)
{
    if (item >= p.total_items) return false;
    int lo = 0, hi = p.ngraphs;  // item_start[lo] <= item < item_start[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(p.item_start + mid) <= item) lo = mid; else hi = mid;
    }
    gd = p.graphs[lo];
    t = p.tree_offset + gd.tree_begin + (item - __ldg(p.item_start + lo));
    return true;
}

// Stack entry `k` of vertex v whose input id is o (the row is v's, the
// Philox counter o's): a uniformly chosen neighbour.
__device__ __forceinline__ int stack_entry(const GraphDesc &g, uint32_t key0, uint32_t key1, int v, int o, uint32_t k,
                                           uint32_t tree)
{
    const int b = __ldg(g.rp + v);
    const int e = __ldg(g.rp + v + 1);
    const unsigned long long x = philox_x64((uint32_t)o, k, tree, g.graph, key0, key1);
    const unsigned long long idx = __umul64hi(x, (unsigned long long)(e - b));
    return __ldg(g.ci + b + (int)idx);
}

constexpr int kFinal = -1;  // mark of vertices known to reach u

// Appends val to q (length counter *cnt in shared memory) for the lanes with
// flag set; one shared atomic per warp. All 32 lanes must call it.
__device__ __forceinline__ void warp_append(bool flag, int val, int32_t *q, int *cnt)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (flag) q[base + __popc(m & ((1u << lane) - 1u))] = val;
}

// Classifies node i of the round's small graph i -> S(i) (S(i) = -1 when the
// walk from x_i reached a vertex known to reach u): returns 1 when the path
// from i ends at -1, 2 when i lies on a cycle, 0 when it runs into a cycle
// that does not contain i. Brent's cycle detection: O(tail + cycle) reads.
__device__ __forceinline__ int classify_node(const int32_t *Sx, int i, int limit)
{
    int power = 1, lam = 1;
    int tortoise = i;
    int hare = Sx[i];
    for (int guard = 0; guard <= 4 * limit + 8; ++guard) {
        if (hare < 0) return 1;
        if (hare == i) return 2;
        if (hare == tortoise) return 0;  // a cycle reached without passing i
        if (power == lam) {
            tortoise = hare;
            power <<= 1;
            lam = 0;
        }
        hare = Sx[hare];
        ++lam;
    }
    return 0;
}

// Vertices a popping-round walk passes before it starts marking them for
// other walks (short walks skip the bookkeeping).
constexpr int kQuietSteps = 0;
// The shared-memory kernel marks paths only in rounds after one whose longest
// walk exceeded this many steps (short walks gain nothing from the stops).
constexpr int kMarkMinWalk = 32;

// Independent walks a thread keeps in flight in the walk passes.
constexpr int kWalks = 4;
// Algorithm-2 path entries a thread tests at once (shallow paths), and the
// entries per vertex below which the flat form is used.
constexpr int kPairs = 4;
constexpr int kPathChunk = 4;
constexpr int kFlatDepth = 8;
// Sampler threads resident per SM that the register budget is sized for
// (64 registers per thread at most).
constexpr int kThreadsPerSm = 1024;

// ---------------------------------------------------------------------------
// Graphs above kTierMaxVertices vertices: the per-tree state lives in the
// CTA's workspace, in global memory, cached by L1 and L2.
//
// Per vertex v of the sampler's graph:
//   NXT(v) the stack top, the tree parent at the end (-1 at u), 4 bytes
//   DEP(v) the stack depth of the top, 4 bytes
//   CW(v)  64 bits, by phase: (children | in-edges removed by peeling),
//          (pending children | summed sizes), (preorder number | summed sizes)
//   MK(v)  the round mark of the popping rounds, 4 bytes
// Kept as separate compact arrays (rather than one record per vertex), the
// entries one step touches share cache lines (measured on R-MAT scale 22:
// 16-byte records of NXT, DEP and CW were 11% slower). Of a tree only the
// preorder chunk sits in shared memory: the rest of the SM's on-chip memory
// is L1 (measured: keeping the CW words of the 28,672 vertices of largest
// degree in shared memory instead was 14% slower on R-MAT scale 22 and 22%
// slower on a 2^20-vertex hyperbolic graph). A single graph is relabelled for
// the sampler in Cuthill-McKee order from the pivot (ust_relabel.cu), so that
// neighbours, whose entries walks, peeling, sizes and Algorithm 2 touch one
// after the other, sit in nearby cache lines; its pendant vertices come last
// and stay out of the trees (GraphDesc::ncore). The relabelling keeps every
// row in the input order and every draw keyed by the input id (gd.orig), so
// the trees are unchanged.
//
// Phases per tree (one CTA per tree, CTA barriers only):
//  1. first draws, in-degrees into CW (high words);
//  2. round 0: in-degree peeling; each step removes one in-edge of y with
//     one atomic on CW[y] (low word) that also says whether y is now a leaf;
//  3. the vertices left with in-edges lie on cycles: the first round list;
//  4. popping rounds as in the shared-memory sampler, marks in MK (compact
//     for the long walks of round-heavy graphs), children counts kept up to
//     date in the high words of CW;
//  5. subtree sizes and offsets by last arrivers; every arrival (vertex,
//     parent, offset) is logged, so the log lists each vertex before its
//     parent;
//  6. preorder numbers top-down over the log read backwards, chunk by chunk:
//     pre(x) = pre(parent) + offset(x), links inside a chunk resolved by
//     pointer jumping, the rare vertex whose parent comes later numbered in
//     passes afterwards;
//  7. Algorithm 2 per vertex over its flattened BFS path; the first edge
//     (bfs_parent(v), v) needs no interval (v lies in its own subtree, and
//     never below its own tree child).
struct LargeWords {
    unsigned long long *g;  // CW of vertex v at g[v]
    uint32_t *mk;           // MK of vertex v at mk[v]
    __device__ __forceinline__ unsigned long long *w(int v) const { return g + v; }
    __device__ __forceinline__ uint32_t *lo(int v) const { return reinterpret_cast<uint32_t *>(g + v); }
    __device__ __forceinline__ uint32_t *hi(int v) const { return reinterpret_cast<uint32_t *>(g + v) + 1; }
    __device__ __forceinline__ uint32_t *mark(int v) const { return mk + v; }
};

// Preorder phase: vertices per chunk and thread (a packed word each in
// shared memory, 32 KB at 1,024 threads), the tag and link values of the
// high words, and the rounds a warp waits for the parents of deferred
// vertices before leaving them to the next pass.
constexpr int kPreChunkPerThread = 4;
constexpr int kPreBatch = 4;  // of them loaded together
// Marks a leaf's entry in the arrival log (its offset field; offsets < 2^31).
constexpr int32_t kLeafBit = (int32_t)0x80000000u;
// Algorithm 2 entries per vertex loaded together in the large-graph sampler.
constexpr int kAlg2Chunk = 2;
constexpr uint32_t kPreTag = 0x80000000u;      // high word of a vertex of the current chunk
constexpr uint32_t kPreRoot = 0xFFFFFFFEu;     // link: the sum is the final number
constexpr uint32_t kPreDeferred = 0xFFFFFFFFu; // link: the parent lies in a later chunk
constexpr int kPreorderSpin = 512;

// Input id of sampler vertex v (identity when the graph is not relabelled).
__device__ __forceinline__ int orig_of(const GraphDesc &g, int v) { return g.orig ? __ldg(g.orig + v) : v; }

// Stack entry k of sampler vertex x whose input id is o (the row is x's, the
// Philox counter o's), skipping the entries that name pendant vertices (ids
// from ncore on): such an entry and the pendant vertex, whose every entry
// names x, form a 2-cycle, popped at once. Returns the entry taken and its
// depth. At most 64 deg(x) + 1024 entries are skipped; the caller's range
// check reports an id still at or above ncore. Not inlined: the kernel calls
// it only for the draws that need it, and its loop stays out of the hot path's
// registers.
__device__ __noinline__ int2 core_entry_of(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                           uint32_t graph, uint32_t key0, uint32_t key1, int x, int o, uint32_t k,
                                           uint32_t tree, int ncore)
{
    const int b = __ldg(rp + x), deg = __ldg(rp + x + 1) - b;
    const uint32_t lim = (uint32_t)min(k + 64ull * (unsigned long long)deg + 1024ull, 0xFFFFFFFFull);
    for (;;) {
        const unsigned long long r = philox_x64((uint32_t)o, k, tree, graph, key0, key1);
        const int y = __ldg(ci + b + (int)__umul64hi(r, (unsigned long long)deg));
        if (y < ncore || k >= lim) return make_int2(y, (int)k);
        ++k;
    }
}

// Appends val for the lanes with flag set, at most cap entries in all (later
// ones are dropped and counted, so an inconsistent state cannot write past
// the array). All 32 lanes must call it.
__device__ __forceinline__ void warp_append_capped(bool flag, int val, int32_t *q, int *cnt, int cap)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    const int i = base + __popc(m & ((1u << lane) - 1u));
    if (flag && i < cap) q[i] = val;
}

// A vertex id read from the per-tree state or the graph, about to be used as
// an index: outside [0, n) it means an inconsistent state. The first failing
// check records its site in stats[6] and the status; the id becomes u, which
// ends every walk and chain, so no access leaves the arrays.
__device__ __forceinline__ int checked_vertex(int v, int n, int u, int site, const SampleParams &p)
{
    if ((unsigned)v < (unsigned)n) return v;
    atomicCAS(p.stats + 6, 0ull, (unsigned long long)site);
    atomicOr(p.status, kStatusBadState);
    return u;
}

// Appends (x, parent, offset) at one position of three arrays, for the lanes
// with flag set (at most cap entries). All 32 lanes must call it.
__device__ __forceinline__ void warp_log_arrival(bool flag, int x, int par, int off, int32_t *qx, int32_t *qp,
                                                 int32_t *qo, int *cnt, int cap)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    const int i = base + __popc(m & ((1u << lane) - 1u));
    if (flag && i < cap) {
        qx[i] = x;
        qp[i] = par;
        qo[i] = off;
    }
}

// The same for 64-bit values.
__device__ __forceinline__ void warp_append_pair(bool flag, unsigned long long val, unsigned long long *q, int *cnt,
                                                 int cap)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    const int i = base + __popc(m & ((1u << lane) - 1u));
    if (flag && i < cap) q[i] = val;
}

template <int BT>
__global__ void __launch_bounds__(BT, kThreadsPerSm / BT) sample_aggregate_large_kernel(SampleParams p)
{
    extern __shared__ unsigned long long s_chunk[];  // preorder chunk: kPreChunkPerThread x BT words
    const int tid = threadIdx.x;
    const long long S_ = p.stride;
    int32_t *base = p.ws + (long long)blockIdx.x * kWsArrays * S_;
    // NXT(v): stack top, then tree parent (array 0); DEP(v): stack depth
    // (array 1); CW(v) (arrays 2, 3, 64-bit). The successor array every walk
    // step reads is kept at 4 bytes a vertex, compact for L2.
    int32_t *NXT = base, *DEP = base + S_;
    unsigned long long *CWg = reinterpret_cast<unsigned long long *>(base + 2 * S_);
    int32_t *XA = base + 4 * S_, *XB = base + 5 * S_;  // round lists, then preorder retries
    int32_t *pos = base + 6 * S_;    // index of a redrawn vertex in the round's list
    int32_t *Sx = base + 7 * S_;     // S(x) as an index into the round's list, -1 = reaches u
    int32_t *owner = base + 8 * S_;  // the walk of this round that passed a vertex
    int32_t *wlen = base + 9 * S_;   // vertices a walk passed before it stopped
    // the arrivals of the sizes pass, in order: vertex, tree parent, offset
    int32_t *ord = base + 10 * S_, *ordp = base + 11 * S_, *ordo = base + 12 * S_;
    int32_t *Rp = p.Rp + (long long)blockIdx.x * p.max_n;
    constexpr unsigned long long kChild = 1ull << 32;

    __shared__ long long s_tree;
    __shared__ int s_cnt, s_err, s_linked, s_qn, s_qh;
    __shared__ unsigned long long s_draws;
    __shared__ unsigned long long cyc[8];
    __shared__ long long tmark;
    if (tid < 8) cyc[tid] = 0ull;
#define UST_PHASE(k)                                      \
    do {                                                  \
        if (tid == 0) {                                   \
            const long long _now = clock64();             \
            cyc[k] += (unsigned long long)(_now - tmark); \
            tmark = _now;                                 \
        }                                                 \
    } while (0)

    unsigned long long my_draws = 0, my_rounds = 0;
    unsigned long long my_skips = 0;  // stack entries skipped over pendant vertices (every thread)
    int my_max_rounds = 0, my_max_pops = 0;

    for (;;) {
        if (tid == 0) s_tree = (long long)atomicAdd(p.next_tree, 1ull);
        __syncthreads();
        GraphDesc gd;
        long long t;
        if (!item_graph(p, s_tree, gd, t)) break;
        // the tree is built on the core, ids below ncore (pendant vertices
        // above are never drawn into it)
        const int n = gd.ncore, u = gd.u;
        const uint32_t tree = (uint32_t)t;
        const LargeWords W{CWg, reinterpret_cast<uint32_t *>(ordp)};
        if (tid == 0) {
            tmark = clock64();
            s_draws = (unsigned long long)(n - 1);
            s_cnt = 0;
            s_err = 0;
            s_qn = 0;
        }

        // ---- 1. first draws and in-degrees ---------------------------------
        for (int v = tid; v < n; v += BT) CWg[v] = 0ull;
        __syncthreads();
        for (int b0 = tid; b0 < n; b0 += BT * kWalks) {
            int o[kWalks], rb[kWalks], deg[kWalks];
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                const int v = b0 + k * BT;
                const bool ok = v < n && v != u;
                o[k] = ok ? orig_of(gd, v) : 0;
                rb[k] = ok ? __ldg(gd.rp + v) : 0;
                deg[k] = ok ? __ldg(gd.rp + v + 1) - rb[k] : 0;
            }
            int y[kWalks];
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                const unsigned long long x = philox_x64((uint32_t)o[k], 0u, tree, gd.graph, p.key0, p.key1);
                y[k] = (deg[k] > 0) ? __ldg(gd.ci + rb[k] + (int)__umul64hi(x, (unsigned long long)deg[k])) : -1;
            }
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                const int v = b0 + k * BT;
                if (v < n) {
                    int dep = 0;
                    if (y[k] >= n) {  // a pendant vertex: its 2-cycle pops at once
                        const int2 e = core_entry_of(gd.rp, gd.ci, gd.graph, p.key0, p.key1, v, o[k], 0u, tree, n);
                        y[k] = e.x;
                        dep = e.y;
                        my_skips += (unsigned)dep;
                    }
                    NXT[v] = y[k];
                    DEP[v] = dep;
                    if (y[k] >= 0 && y[k] != u) atomicAdd(W.w(checked_vertex(y[k], n, u, 1, p)), kChild);  // u's counters are never needed
                }
            }
        }
        __syncthreads();
        UST_PHASE(0);

        // ---- 2. round 0: in-degree peeling -----------------------------------
        // Every thread starts walks at its own leaves (no children) and keeps
        // kWalks in flight; a step adds 1 to y's removed in-edges and, when
        // that was y's last one, continues with y's successor.
        {
            // the leaves' successors first, in one coalesced sweep (the log
            // array is free until the sizes pass); walks then take them from
            // this queue, one prefetched ahead
            int32_t *Q = ord;
            if (tid == 0) s_qh = 0;
            for (int v = tid; v - (tid & 31) < n; v += BT) {  // uniform per warp
                const bool leaf = v < n && v != u && (*W.w(v) >> 32) == 0ull;
                const int y0 = leaf ? checked_vertex(NXT[v], n, u, 2, p) : u;
                warp_append_capped(leaf && y0 != u, y0, Q, &s_qn, n);
            }
            __syncthreads();
            const int qn = min(s_qn, n);
            int idx = atomicAdd(&s_qh, 1);
            int spare = (idx < qn) ? Q[idx] : u;
            int y[kWalks];
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                y[k] = spare;
                idx = (spare != u) ? atomicAdd(&s_qh, 1) : qn;
                spare = (idx < qn) ? Q[idx] : u;
            }
            bool done = false;
            for (int guard = 0; guard <= 2 * n + 2; ++guard) {
                unsigned long long old[kWalks];
                int ny[kWalks];
#pragma unroll
                for (int k = 0; k < kWalks; ++k) {
                    old[k] = 0ull;
                    ny[k] = u;
                    if (y[k] != u) {
                        old[k] = atomicAdd(W.w(y[k]), 1ull);
                    }
                }
                // y's successor only once y is peeled: a read for every step,
                // whether or not the walk goes on, cost 38% more time on R-MAT
                // scale 22 than the extra round trip of the steps that do
#pragma unroll
                for (int k = 0; k < kWalks; ++k)
                    if (y[k] != u && (uint32_t)old[k] + 1u == (uint32_t)(old[k] >> 32))
                        ny[k] = checked_vertex(NXT[y[k]], n, u, 3, p);
                bool any = false;
#pragma unroll
                for (int k = 0; k < kWalks; ++k) {
                    if (y[k] != u && (uint32_t)old[k] + 1u == (uint32_t)(old[k] >> 32)) {
                        y[k] = ny[k];  // y peeled: remove its out-edge next
                    } else {
                        y[k] = spare;
                        idx = (spare != u) ? atomicAdd(&s_qh, 1) : qn;
                        spare = (idx < qn) ? Q[idx] : u;
                    }
                    any |= (y[k] != u);
                }
                if (!any) {
                    done = true;
                    break;
                }
            }
            if (!done) s_err = 1;
        }
        __syncthreads();
        UST_PHASE(1);

        // ---- 3. the first round list: vertices with in-edges left ------------
        for (int v = tid; v - (tid & 31) < n; v += BT) {  // uniform per warp
            bool on_cycle = false;
            if (v < n) {
                const unsigned long long w = *W.w(v);
                if (v == u) {
                    *W.mark(v) = (uint32_t)kFinal;
                } else {
                    on_cycle = (uint32_t)w < (uint32_t)(w >> 32);
                    *W.mark(v) = 0u;
                }
            }
            warp_append_capped(on_cycle, v, XA, &s_cnt, n);
        }
        __syncthreads();
        UST_PHASE(2);
        int nX = min(s_cnt, n);

        // ---- 4. popping rounds -------------------------------------------------
        int rounds = 0;
        bool failed = s_err != 0;
        if (failed && tid == 0) atomicOr(p.status, kStatusBadState);
        int32_t *X = XA, *Xn = XB;
        while (!failed && nX > 0) {
            ++rounds;
            if (rounds > p.max_rounds) {
                failed = true;
                if (tid == 0) atomicOr(p.status, kStatusPopRounds);
                break;
            }
            // (a) pop: every vertex on a cycle advances to its next stack entry
            for (int i = tid; i < nX; i += BT) {
                const int x = checked_vertex(X[i], n, u, 4, p);
                if (x == u) continue;
                const uint32_t k = (uint32_t)DEP[x] + 1u;
                const int old = checked_vertex(NXT[x], n, u, 5, p);
                const int2 e = core_entry_of(gd.rp, gd.ci, gd.graph, p.key0, p.key1, x, orig_of(gd, x), k, tree, n);
                const int y = checked_vertex(e.x, n, u, 5, p);
                my_skips += (uint32_t)e.y - k;
                NXT[x] = y;
                DEP[x] = e.y;
                *W.mark(x) = (uint32_t)rounds;
                pos[x] = i;
                if (old != u) atomicAdd(W.hi(old), 0xFFFFFFFFu);  // one child less
                if (y != u) atomicAdd(W.hi(y), 1u);
            }
            if (tid == 0) {
                s_draws += (unsigned long long)nX;
                s_cnt = 0;
                s_linked = 0;
                my_max_pops = max(my_max_pops, nX);
            }
            __syncthreads();
            // (b) S(x): the first redrawn or known-final vertex after x; a walk
            //     that reaches a vertex another walk of this round passed
            //     stops and takes that walk's result (owner published before
            //     the mark, block fence), resolved after the barrier
            const int vis = -2 - rounds;
            for (int i = tid; i < nX; i += BT) {
                int y = checked_vertex(NXT[checked_vertex(X[i], n, u, 6, p)], n, u, 6, p);
                int res = -2, len = 0;
                for (int guard = 0; guard <= n; ++guard) {
                    const int m = (int)*W.mark(y);
                    const int ny = NXT[y];  // checked below, before it is used
                    if (m == kFinal) {
                        res = -1;
                        break;
                    }
                    if (m == rounds) {
                        res = pos[y];
                        break;
                    }
                    if (m == vis) {
                        __threadfence_block();
                        res = -3 - owner[y];
                        s_linked = 1;
                        break;
                    }
                    owner[y] = i;
                    __threadfence_block();  // the owner is visible before the mark
                    *W.mark(y) = (uint32_t)vis;
                    ++len;
                    y = checked_vertex(ny, n, u, 7, p);
                }
                if (res == -2) {
                    s_err = 1;
                    res = -1;
                }
                Sx[i] = res;
                wlen[i] = len;
            }
            __syncthreads();
            if (s_linked) {  // some walk stopped on another's path: resolve the links
                for (int i = tid; i < nX; i += BT) {
                    int r = Sx[i];
                    for (int guard = 0; r <= -3 && guard <= nX; ++guard) {
                        const int j = -3 - r;
                        if (j >= nX) break;  // not a walk of this round: reported below
                        r = Sx[j];
                    }
                    if (r <= -3 || r >= nX) {
                        s_err = 1;
                        r = -1;
                    }
                    Sx[i] = r;  // a reader sees the link or its result: both lead to the same end
                }
                __syncthreads();
            }
            // (c) nodes that reach -1 mark x and their walked part final; nodes
            //     on a cycle of i -> S(i) queue their whole segment for popping
            for (int i = tid; i < nX; i += BT) {
                const int kind = classify_node(Sx, i, nX);
                int y = checked_vertex(X[i], n, u, 8, p);
                if (kind == 1) {
                    const int len = wlen[i];
                    *W.mark(y) = (uint32_t)kFinal;
                    for (int k = 0; k < len; ++k) {
                        y = checked_vertex(NXT[y], n, u, 8, p);
                        *W.mark(y) = (uint32_t)kFinal;
                    }
                } else if (kind == 2) {
                    for (int guard = 0; guard <= n; ++guard) {
                        Xn[min(atomicAdd(&s_cnt, 1), n)] = y;  // more than n entries: reported below
                        y = checked_vertex(max(NXT[y], 0), n, u, 8, p);  // -1 at u: an inconsistent walk stays in the arrays
                        if ((int)*W.mark(y) == rounds) break;
                    }
                    if ((int)*W.mark(y) != rounds) s_err = 1;  // a cycle segment ends at a redrawn vertex
                }
            }
            __syncthreads();
            nX = s_cnt;
            int32_t *tmp = X;
            X = Xn;
            Xn = tmp;
            if (s_err || nX > n) {
                failed = true;
                if (tid == 0) atomicOr(p.status, kStatusBadState);
                break;
            }
            __syncthreads();
        }
        if (failed) break;
        UST_PHASE(3);
        if (tid == 0) {
            my_draws += s_draws;
            my_rounds += (unsigned long long)rounds;
            my_max_rounds = max(my_max_rounds, rounds);
        }
        if (p.edge_counts) {  // the tree's arcs v -> parent(v): the final stack entry of every v
            for (int v = tid; v < n; v += BT) {
                if (v == u) continue;
                const int o = orig_of(gd, v);
                const int b = __ldg(gd.rp + v), e = __ldg(gd.rp + v + 1);
                const uint32_t k = (uint32_t)DEP[v];
                const unsigned long long x = philox_x64((uint32_t)o, k, tree, gd.graph, p.key0, p.key1);
                const long long row = gd.rp_in ? (long long)__ldg(gd.rp_in + o) : (long long)b;  // input arc index
                atomicAdd(p.edge_counts + gd.aoff + row + (long long)__umul64hi(x, (unsigned long long)(e - b)), 1ull);
            }
        }
        if (p.mode == 1) {  // export the tree in input ids
            const long long ob = s_tree * (long long)n;
            for (int v = tid; v < n; v += BT) {
                const int o = orig_of(gd, v);
                const int tp = NXT[v];
                p.next_out[ob + o] = (tp < 0) ? -1 : orig_of(gd, tp);
                if (p.pops_out) p.pops_out[ob + o] = DEP[v];
            }
            __syncthreads();
            continue;
        }
        // the low words sum subtree sizes from now on (they still hold
        // peeling's removed in-edges)
        for (int v = tid; v < n; v += BT)
            if (*W.lo(v) != 0u) *W.lo(v) = 0u;
        if (tid == 0) {
            s_qn = 0;  // arrivals logged
            s_cnt = 0; // leaves queued
            s_qh = 0;
        }
        __syncthreads();

        // ---- 5. subtree sizes and offsets ---------------------------------------
        // A leaf's word is 0 (no children, nothing summed); an inner vertex's
        // never is (children pending, or a size summed). An arrival of x at
        // its parent adds x's size and removes one pending child in one
        // atomic, whose old value gives x's offset; the last arriver carries
        // the parent's size upwards. Arrivals are logged before their atomic.
        {
            // (leaf, parent) pairs first, in one coalesced sweep, into the
            // round lists' space (XA and XB as one 64-bit array); chains then
            // take them from this queue, one prefetched ahead
            unsigned long long *Q2 = reinterpret_cast<unsigned long long *>(XA);
            for (int v = tid; v - (tid & 31) < n; v += BT) {  // uniform per warp
                const bool leaf = v < n && v != u && *W.w(v) == 0ull;
                const int pv = leaf ? checked_vertex(NXT[v], n, u, 9, p) : u;
                warp_append_pair(leaf, ((unsigned long long)(uint32_t)v << 32) | (uint32_t)pv, Q2, &s_cnt, n);
            }
            __syncthreads();
            const int qn = min(s_cnt, n);
            constexpr unsigned long long kNone = ~0ull;
            int idx = atomicAdd(&s_qh, 1);
            unsigned long long spare = (idx < qn) ? Q2[idx] : kNone;
            int x[kWalks], par[kWalks];
            uint32_t carry[kWalks];
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                x[k] = (spare != kNone) ? (int)(spare >> 32) : -1;
                par[k] = (spare != kNone) ? (int)(uint32_t)spare : -1;
                carry[k] = 1u;
                idx = (spare != kNone) ? atomicAdd(&s_qh, 1) : qn;
                spare = (idx < qn) ? Q2[idx] : kNone;
            }
            bool done = false;
            for (int guard = 0; guard <= 2 * n + 2; ++guard) {
                unsigned long long old[kWalks];
                int gp[kWalks];
#pragma unroll
                for (int k = 0; k < kWalks; ++k) {
                    old[k] = 0ull;
                    gp[k] = -1;
                    if (par[k] >= 0) {
                        old[k] = atomicAdd(W.w(par[k]), (unsigned long long)carry[k] - kChild);
                    }
                }
                // the parent's parent only for the last arriver, which goes on
#pragma unroll
                for (int k = 0; k < kWalks; ++k)
                    if (par[k] >= 0 && par[k] != u && (old[k] >> 32) == 1ull)
                        gp[k] = checked_vertex(NXT[par[k]], n, u, 10, p);
                // log every arrival: x, its parent and its offset inside the
                // parent's interval (all lanes call)
#pragma unroll
                for (int k = 0; k < kWalks; ++k)
                    warp_log_arrival(par[k] >= 0, x[k], par[k],
                                     (1 + (int)(uint32_t)old[k]) | (carry[k] == 1u ? kLeafBit : 0), ord, ordp, ordo,
                                     &s_qn, n);
                bool any = false;
#pragma unroll
                for (int k = 0; k < kWalks; ++k) {
                    if (par[k] >= 0) {
                        if (par[k] != u && (old[k] >> 32) == 1ull) {    // the last child: carry the size upwards
                            carry[k] = (uint32_t)old[k] + carry[k] + 1u;
                            x[k] = par[k];
                            par[k] = gp[k];
                        } else {
                            x[k] = (spare != kNone) ? (int)(spare >> 32) : -1;
                            par[k] = (spare != kNone) ? (int)(uint32_t)spare : -1;
                            carry[k] = 1u;
                            idx = (spare != kNone) ? atomicAdd(&s_qh, 1) : qn;
                            spare = (idx < qn) ? Q2[idx] : kNone;
                        }
                    }
                    any |= (par[k] >= 0);
                }
                if (!__any_sync(0xffffffffu, any)) {
                    done = true;
                    break;
                }
            }
            if (!done) s_err = 1;
        }
        __syncthreads();
        if (s_err || s_qn != n - 1) {  // every vertex but u arrives exactly once
            if (tid == 0) atomicOr(p.status, kStatusBadState);
            break;
        }
        UST_PHASE(4);

        // ---- 6. preorder numbers, top-down ---------------------------------------
        // pre(u) = 0 and pre(x) = pre(parent) + offset(x) >= 1, written into
        // the high word (0 after the sizes pass: no child pending). The log
        // read backwards lists parents before their children; it is taken in
        // chunks of kPreChunkPerThread x BT vertices. A chunk's vertices are first tagged
        // (high word = kPreTag | position in the chunk); then each one finds
        // its parent numbered (an earlier chunk, or u), tagged (this chunk:
        // a link), or neither (a later chunk, which the log order makes rare:
        // deferred). Links are resolved by pointer jumping on packed
        // (link, sum) words in the CTA's workspace, and the numbers written back.
        // Deferred vertices are numbered afterwards in passes in which each
        // warp waits a bounded number of rounds for the parents; what is
        // still pending goes to the next pass.
        {
            // the chunk's packed words in shared memory; a thread's log
            // entries are loaded together before any of them is used
            volatile unsigned long long *chunk = s_chunk;
            constexpr int C = kPreChunkPerThread;
            const int total = n - 1;
            const int K = C * BT;
            if (tid == 0) s_cnt = 0;  // deferred vertices, listed in XA
            __syncthreads();
            for (int c0 = 0; c0 < total; c0 += K) {
                const int len = min(K, total - c0);
#pragma unroll 1
                for (int k0 = 0; k0 < C; k0 += kPreBatch) {  // tags; leaves are nobody's parent: no tag
                    int xs[kPreBatch];
                    int32_t os[kPreBatch];
#pragma unroll
                    for (int k = 0; k < kPreBatch; ++k) {
                        const int i = tid + (k0 + k) * BT, j = total - 1 - (c0 + i);
                        os[k] = (i < len) ? ordo[j] : kLeafBit;
                        xs[k] = (i < len) ? ord[j] : u;
                    }
#pragma unroll
                    for (int k = 0; k < kPreBatch; ++k)
                        if (!(os[k] & kLeafBit))
                            *W.hi(checked_vertex(xs[k], n, u, 11, p)) = kPreTag | (uint32_t)(tid + (k0 + k) * BT);
                }
                __syncthreads();
                // each entry's parent: numbered, tagged or neither (the
                // barrier makes the tags visible to plain loads)
#pragma unroll 1
                for (int k0 = 0; k0 < C; k0 += kPreBatch) {
                    int par[kPreBatch];
                    uint32_t off[kPreBatch], h[kPreBatch];
#pragma unroll
                    for (int k = 0; k < kPreBatch; ++k) {
                        const int i = tid + (k0 + k) * BT, j = total - 1 - (c0 + i);
                        par[k] = (i < len) ? checked_vertex(ordp[j], n, u, 13, p) : u;
                        off[k] = (i < len) ? (uint32_t)(ordo[j] & ~kLeafBit) : 0u;
                    }
#pragma unroll
                    for (int k = 0; k < kPreBatch; ++k) h[k] = (par[k] != u) ? *W.hi(par[k]) : 0u;
#pragma unroll
                    for (int k = 0; k < kPreBatch; ++k) {
                        const int i = tid + (k0 + k) * BT;
                        if (i >= len) continue;
                        uint32_t link = kPreRoot, sum = off[k];
                        if (par[k] != u) {
                            if (h[k] & kPreTag)
                                link = h[k] & ~kPreTag;  // the parent is in this chunk
                            else if (h[k] != 0u)
                                sum = h[k] + off[k];  // numbered in an earlier chunk
                            else
                                link = kPreDeferred;
                        }
                        chunk[i] = ((unsigned long long)link << 32) | sum;
                    }
                }
                __syncthreads();
                // pointer jumping: a word read while its owner rewrites it is
                // the old or the new (link, sum) pair, and both are valid
                for (int step = 0;; ++step) {
                    bool any = false;
                    if (step <= 32) {
#pragma unroll
                        for (int k = 0; k < C; ++k) {
                            const int i = tid + k * BT;
                            if (i >= len) continue;
                            const unsigned long long a = chunk[i];
                            const uint32_t l = (uint32_t)(a >> 32);
                            if (l >= kPreRoot) continue;  // resolved or deferred
                            const unsigned long long b = chunk[l];
                            const uint32_t l2 = (uint32_t)(b >> 32);
                            chunk[i] = l2 == kPreDeferred ? ((unsigned long long)kPreDeferred << 32)
                                                          : ((unsigned long long)l2 << 32) |
                                                                (uint32_t)((uint32_t)a + (uint32_t)b);
                            any = true;
                        }
                    }
                    if (!__syncthreads_or(any)) break;
                    if (step > 32) {  // a chunk of at most 2^32 entries resolves in 32 steps
                        s_err = 1;
                        break;
                    }
                }
#pragma unroll 1
                for (int k0 = 0; k0 < C; k0 += kPreBatch) {  // the numbers into the high words; deferred entries listed
                    int xs[kPreBatch];
#pragma unroll
                    for (int k = 0; k < kPreBatch; ++k) {
                        const int i = tid + (k0 + k) * BT, j = total - 1 - (c0 + i);
                        xs[k] = (i < len) ? ord[j] : u;
                    }
#pragma unroll
                    for (int k = 0; k < kPreBatch; ++k) {
                        const int i = tid + (k0 + k) * BT;
                        bool deferred = false;
                        if (i < len) {
                            const int x = checked_vertex(xs[k], n, u, 11, p);
                            const unsigned long long a = chunk[i];
                            deferred = (uint32_t)(a >> 32) != kPreRoot;
                            *W.hi(x) = deferred ? 0u : (uint32_t)a;
                        }
                        // i - lane < len is uniform per warp (BT is a multiple of 32)
                        if (i - (tid & 31) < len) warp_append_capped(deferred, total - 1 - (c0 + i), XA, &s_cnt, n);
                    }
                }
                __syncthreads();
            }
            int cnt = min(s_cnt, n);
            int32_t *list = XA, *retry = XB;
            for (int pass = 0; cnt > 0; ++pass) {
                if (pass > n) {
                    s_err = 1;
                    break;
                }
                __syncthreads();
                if (tid == 0) s_cnt = 0;
                __syncthreads();
                for (int b0 = tid; b0 - (tid & 31) < cnt; b0 += BT) {  // uniform per warp
                    const int j = (b0 < cnt) ? list[b0] : -1;
                    const bool valid = (unsigned)j < (unsigned)total;
                    const int x = valid ? checked_vertex(ord[j], n, u, 11, p) : -1;
                    const int par = valid ? checked_vertex(ordp[j], n, u, 13, p) : u;
                    const uint32_t off = valid ? (uint32_t)(ordo[j] & ~kLeafBit) : 0u;
                    uint32_t pp = 0u;
                    bool ok = !valid || par == u, written = !valid;
                    // the warp waits together, so a parent numbered by another
                    // lane is seen one round later
                    for (int spin = 0;; ++spin) {
                        if (!ok) {
                            pp = *reinterpret_cast<volatile uint32_t *>(W.hi(par));
                            ok = pp != 0u;
                        }
                        if (ok && !written) {
                            *reinterpret_cast<volatile uint32_t *>(W.hi(x)) = pp + off;
                            written = true;
                        }
                        if (__all_sync(0xffffffffu, written) || spin >= kPreorderSpin) break;
                    }
                    warp_append_capped(!written, j, retry, &s_cnt, n);
                }
                __syncthreads();
                cnt = min(s_cnt, n);
                int32_t *tmp = list;
                list = retry;
                retry = tmp;
            }
        }
        __syncthreads();
        if (s_err) {
            if (tid == 0) atomicOr(p.status, kStatusBadState);
            break;
        }
        UST_PHASE(5);

        // ---- 7. Algorithm 2 ------------------------------------------------------
        // P(v) = v, a_1 = bfs_parent(v), ..., a_d = u (at pathptr[v]; for a
        // relabelled graph in sampler ids and order). Edge (a_j+1,
        // a_j) counts +1 when T uses it downwards (parent(a_j) = a_j+1) and v
        // lies in a_j's subtree, -1 when T uses it upwards and v lies in
        // a_j+1's subtree.
        for (int b0 = tid; b0 < n; b0 += BT * kWalks) {
            int s0[kWalks], d[kWalks], prev[kWalks], nprev[kWalks], cnt[kWalks];
            uint32_t pv[kWalks];
            int dmax = 0;
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                const int v = b0 + k * BT;
                const bool ok = v < n && v != u;
                s0[k] = ok ? __ldg(gd.pathptr + v) : 0;
                d[k] = ok ? __ldg(gd.pathptr + v + 1) - s0[k] : 0;
                prev[k] = v;
                nprev[k] = ok ? NXT[v] : -2;
                pv[k] = ok ? *W.hi(v) : 0u;
                cnt[k] = 0;
                dmax = max(dmax, d[k]);
            }
            // kAlg2Chunk entries of every vertex at a time: their ancestors,
            // the ancestors' tree parents and the tested intervals are each
            // loaded together
            for (int c = 0; c < dmax; c += kAlg2Chunk) {
                int a[kWalks][kAlg2Chunk], na[kWalks][kAlg2Chunk];
#pragma unroll
                for (int k = 0; k < kWalks; ++k)
#pragma unroll
                    for (int j = 0; j < kAlg2Chunk; ++j)
                        a[k][j] = (c + j < d[k]) ? checked_vertex(__ldg(gd.path + s0[k] + c + j), n, u, 12, p) : -1;
#pragma unroll
                for (int k = 0; k < kWalks; ++k)
#pragma unroll
                    for (int j = 0; j < kAlg2Chunk; ++j)
                        na[k][j] = (a[k][j] >= 0 && a[k][j] != u) ? NXT[a[k][j]] : -1;
                int tx[kWalks][kAlg2Chunk];
#pragma unroll
                for (int k = 0; k < kWalks; ++k) {
#pragma unroll
                    for (int j = 0; j < kAlg2Chunk; ++j) {
                        // edge (a_{c+j+1}, a_{c+j}): b = a_{c+j} (v itself first)
                        const int aj = a[k][j];
                        const int bj = (j == 0) ? prev[k] : a[k][j - 1];
                        const int nbj = (j == 0) ? nprev[k] : na[k][j - 1];
                        tx[k][j] = -1;  // no interval to test; a sign is folded into the vertex id below
                        if (aj < 0) continue;
                        if (nbj == aj) {  // downwards: the interval of b
                            if (c + j == 0)
                                cnt[k] += 1;  // v lies in its own subtree
                            else
                                tx[k][j] = bj;
                        } else if (na[k][j] == bj && c + j > 0) {  // upwards: the interval of a
                            tx[k][j] = -2 - aj;
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < kWalks; ++k) {
#pragma unroll
                    for (int j = 0; j < kAlg2Chunk; ++j) {
                        const int t = tx[k][j];
                        if (t == -1) continue;
                        const int vt = t >= 0 ? t : -2 - t;
                        const unsigned long long w = *W.w(vt);
                        const uint32_t lo = (uint32_t)(w >> 32), sz = (uint32_t)w + 1u;
                        if (lo <= pv[k] && pv[k] - lo < sz) cnt[k] += (t >= 0) ? 1 : -1;
                    }
#pragma unroll
                    for (int j = 0; j < kAlg2Chunk; ++j)
                        if (a[k][j] >= 0) {
                            prev[k] = a[k][j];
                            nprev[k] = na[k][j];
                        }
                }
            }
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                const int v = b0 + k * BT;
                if (v >= n || v == u) continue;
                if (p.R_direct) {
                    if (cnt[k] != 0)
                        atomicAdd(p.R_direct + gd.voff + orig_of(gd, v), (unsigned long long)(long long)cnt[k]);
                } else {
                    Rp[v] += cnt[k];
                }
            }
        }
        __syncthreads();
        UST_PHASE(6);
        if (tid == 0) {
            unsigned long long tot = 0ull;
            for (int k = 0; k < 7; ++k) tot += cyc[k];
            cyc[7] = tot;  // running total over trees
        }
    }
#undef UST_PHASE

    if (tid == 0) {
        atomicAdd(p.stats + 0, my_draws);
        atomicAdd(p.stats + 1, my_rounds);
        atomicMax(p.stats + 2, (unsigned long long)my_max_rounds);
        atomicMax(p.stats + 3, (unsigned long long)my_max_pops);
        for (int k = 0; k < 8; ++k) atomicAdd(p.stats + 8 + k, cyc[k]);
    }
    // a skipped entry is one pop of the core vertex and one of the pendant
    // vertex it named (whose first draws the host adds)
    if (my_skips) atomicAdd(p.stats + 0, 2ull * my_skips);
}
// ---------------------------------------------------------------------------
// The same three phases for graphs of at most kTierMaxVertices vertices
// (ids below 0xFFFF), with the hot per-tree state in shared memory (4 bytes
// per vertex, one n-word array whose view changes per phase; above
// kSmemMaxVertices vertices its last words sit in a global tail):
//   peeling   16-bit remaining in-degree | 16-bit successor
//   rounds    16-bit round mark          | 16-bit successor
//   sizes     32-bit word: pending children << 16 | summed sizes
//   preorder  32-bit word: ancestor << 16 | summed offsets
// The tree's parent array, stack depths, round lists, offsets and sizes stay
// in the CTA's global workspace. 16-bit counters share a 32-bit word with a
// neighbour and are updated by adding or subtracting 1 << 16 * (v & 1); a
// count never passes below 0 or above n - 1, so halves never carry.
constexpr uint16_t kFinal16 = 0xFFFFu;
// Round marks: the round's stamp s in [1, kMaxStamp15] on redrawn vertices,
// s | kVisited16 on the vertices a walk of round s passed, kFinal16 on
// vertices known to reach u.
constexpr int kMaxStamp15 = 0x7FFE;
constexpr uint16_t kVisited16 = 0x8000u;

// Shared words of the sampler: kSmemWords 32-bit words per CTA.
constexpr int kSmemWords = ((kSmemMaxVertices + 1) / 2) * 2;
// Workspace array that holds the words beyond kSmemWords (graphs between
// kSmemMaxVertices and kTierMaxVertices vertices): at most
// kTierMaxVertices + 1 - kSmemWords words, below one array's stride.
constexpr int kTailArray = 9;
static_assert(kTailArray < kWsArrays, "the tail is one of the CTA's workspace arrays");
static_assert(kTierMaxVertices + 1 - kSmemWords <= kSmemMaxVertices,
              "the tail fits one workspace array (stride >= max_n + 2 > kSmemMaxVertices)");
static_assert(kTierMaxVertices < 0xFFFF + 1, "16-bit vertex ids stay below the 0xFFFF sentinel");

// The per-tree words of the shared-memory sampler. Word i lives in shared
// memory below kSmemWords; with kTier the words from kSmemWords on live in
// the CTA's global tail. 16-bit element i is half (i & 1) of word i >> 1.
template <bool kTier>
struct TreeWords {
    uint32_t *s;  // shared words
    uint32_t *g;  // tail: word kSmemWords + j at g[j]
    __device__ __forceinline__ uint32_t *word(int i) const
    {
        if constexpr (kTier) return i < kSmemWords ? s + i : g + (i - kSmemWords);
        return s + i;
    }
    __device__ __forceinline__ uint16_t *half(int i) const
    {
        if constexpr (kTier)
            return i < 2 * kSmemWords ? reinterpret_cast<uint16_t *>(s) + i
                                      : reinterpret_cast<uint16_t *>(g) + (i - 2 * kSmemWords);
        return reinterpret_cast<uint16_t *>(s) + i;
    }
};
// Array views into the tree words, starting at word (or half) `base`.
template <bool kTier>
struct Words32 {
    TreeWords<kTier> t;
    int base;
    __device__ __forceinline__ uint32_t &operator[](int i) const { return *t.word(base + i); }
};
template <bool kTier>
struct Halves16 {
    TreeWords<kTier> t;
    int base;
    __device__ __forceinline__ uint16_t &operator[](int i) const { return *t.half(base + i); }
};

template <class Words>
__device__ __forceinline__ uint32_t half_add(const Words &words, int v, int delta)
{
    const int sh = (v & 1) << 4;
    const uint32_t old = atomicAdd(&words[v >> 1], (uint32_t)delta << sh);
    return (old >> sh) & 0xFFFFu;
}

template <int BT, bool kTier>
__global__ void __launch_bounds__(BT, kThreadsPerSm / BT) sample_aggregate_smem_kernel(SampleParams p)
{
    extern __shared__ uint32_t s_dyn[];
    const int tid = threadIdx.x;
    const long long S_ = p.stride;
    int32_t *base = p.ws + (long long)blockIdx.x * kWsArrays * S_;
    int32_t *nxt = base;              // the tree's parent array at the end
    int32_t *pop = base + 1 * S_;     // stack depth of the current top
    int32_t *gsz = base + 2 * S_;     // subtree sizes (for Algorithm 2)
    int32_t *pos = base + 3 * S_;     // index of a redrawn vertex in the round's list
    int32_t *XA = base + 4 * S_, *XB = base + 5 * S_;
    int32_t *Sx = base + 6 * S_;
    int32_t *owner = base + 7 * S_;   // the walk of this round that passed a vertex
    int32_t *wlen = base + 8 * S_;    // vertices a walk passed before it stopped
    int32_t *off = XA;
    int32_t *Rp = p.Rp + (long long)blockIdx.x * p.max_n;
    constexpr uint32_t kC16 = 1u << 16;
    const TreeWords<kTier> tw{s_dyn, reinterpret_cast<uint32_t *>(base + kTailArray * S_)};
    const Halves16<kTier> lo16{tw, 0};  // counts, then marks
    const Words32<kTier> lo32{tw, 0};   // the same, as words
    const Words32<kTier> C{tw, 0};      // sizes / preorder words

    __shared__ long long s_tree;
    __shared__ int s_cnt, s_err, s_qn, s_qh, s_linked, s_mark_on, s_maxwalk;
    __shared__ unsigned long long s_draws;
    __shared__ unsigned long long cyc[12];
    __shared__ long long tmark;
    if (tid < 12) cyc[tid] = 0ull;
#define UST_PHASE(k)                                      \
    do {                                                  \
        if (tid == 0) {                                   \
            const long long _now = clock64();             \
            cyc[k] += (unsigned long long)(_now - tmark); \
            tmark = _now;                                 \
        }                                                 \
    } while (0)

    unsigned long long my_draws = 0, my_rounds = 0;
    unsigned long long my_skips = 0;  // stack entries skipped over pendant vertices (every thread)
    int my_max_rounds = 0, my_max_pops = 0;

    for (;;) {
        if (tid == 0) s_tree = (long long)atomicAdd(p.next_tree, 1ull);
        __syncthreads();
        GraphDesc gd;
        long long t;
        if (!item_graph(p, s_tree, gd, t)) break;
        // the tree is built on the core, ids below ncore (a relabelled graph's
        // pendant vertices above are never drawn into it)
        const int n = gd.ncore, u = gd.u;
        const uint32_t tree = (uint32_t)t;
        const int nhalf = (n + 1) >> 1;                                // words of one 16-bit array
        const Halves16<kTier> nx16{tw, 2 * nhalf};  // successors
        const int iters = (n + BT * kWalks - 1) / (BT * kWalks);
        if (tid == 0) tmark = clock64();

        // ---- 1. cycle popping --------------------------------------------
        for (int w = tid; w < nhalf; w += BT) lo32[w] = 0u;
        for (int b0 = tid; b0 < n; b0 += BT * kWalks) {
            int rb[kWalks], deg[kWalks];
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                const int v = b0 + k * BT;
                const bool ok = v < n && v != u;
                rb[k] = ok ? __ldg(gd.rp + v) : 0;
                deg[k] = ok ? __ldg(gd.rp + v + 1) - rb[k] : 0;
            }
            int y[kWalks];
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                const int v = b0 + k * BT;
                const int o = (v < n) ? orig_of(gd, v) : v;
                const unsigned long long x = philox_x64((uint32_t)o, 0u, tree, gd.graph, p.key0, p.key1);
                y[k] = (deg[k] > 0) ? __ldg(gd.ci + rb[k] + (int)__umul64hi(x, (unsigned long long)deg[k])) : -1;
            }
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                const int v = b0 + k * BT;
                if (v < n) {
                    int dep = 0;
                    if (y[k] >= n) {  // a pendant vertex: its 2-cycle pops at once
                        const int2 e =
                            core_entry_of(gd.rp, gd.ci, gd.graph, p.key0, p.key1, v, orig_of(gd, v), 0u, tree, n);
                        y[k] = e.x;
                        dep = e.y;
                        my_skips += (unsigned)dep;
                    }
                    pop[v] = dep;
                    nxt[v] = y[k];
                    nx16[v] = (uint16_t)(v == u ? u : y[k]);  // u points at itself: no walk leaves the array
                }
            }
        }
        if (tid == 0) {
            s_draws = (unsigned long long)(n - 1);
            s_cnt = 0;
            s_err = 0;
            s_qn = 0;
            s_qh = 0;
        }
        __syncthreads();
        UST_PHASE(0);
        for (int v = tid; v < n; v += BT)
            if (v != u) half_add(lo32, nx16[v], 1);  // in-degrees
        __syncthreads();
        UST_PHASE(1);
        // round 0: peel. Leaves are marked 0xFFFF first (no in-edge, so no
        // walk touches their count); a peeled vertex ends at count 0, so the
        // two never mix. Every thread scans its own vertices for leaves and
        // keeps kWalks walks in flight, all in shared memory.
        for (int v = tid; v < n; v += BT)
            if (v != u && lo16[v] == 0) half_add(lo32, v, 0xFFFF);
        __syncthreads();
        UST_PHASE(2);
        {
            int cand = tid;
            int y[kWalks];
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                y[k] = u;
                while (cand < n) {
                    const int v = cand;
                    cand += BT;
                    if (v != u && lo16[v] == kFinal16) {
                        y[k] = nx16[v];
                        if (y[k] != u) break;
                    }
                }
            }
            for (int guard = 0; guard <= 2 * n + 2; ++guard) {
                bool any = false;
#pragma unroll
                for (int k = 0; k < kWalks; ++k) {
                    if (y[k] != u && half_add(lo32, y[k], -1) == 1u) {
                        y[k] = nx16[y[k]];  // y peeled: remove its out-edge next
                    } else {
                        y[k] = u;
                        while (cand < n) {
                            const int v = cand;
                            cand += BT;
                            if (v != u && lo16[v] == kFinal16) {
                                y[k] = nx16[v];
                                if (y[k] != u) break;
                            }
                        }
                    }
                    any |= (y[k] != u);
                }
                if (!any) break;
            }
        }
        __syncthreads();
        UST_PHASE(3);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                const int v = tid + (it * kWalks + k) * BT;
                const bool cyc_v = v < n && v != u && lo16[v] != 0 && lo16[v] != kFinal16;  // on a cycle
                warp_append(cyc_v, v, XA, &s_cnt);
            }
        }
        __syncthreads();
        for (int v = tid; v < n; v += BT) lo16[v] = (v == u) ? kFinal16 : 0;  // round marks
        if (tid == 0) s_maxwalk = 0;
        __syncthreads();
        UST_PHASE(4);
        int nX = s_cnt;

        int rounds = 0;
        bool failed = false;
        int32_t *X = XA, *Xn = XB;
        while (nX > 0) {
            ++rounds;
            if (rounds > p.max_rounds) {
                failed = true;
                if (tid == 0) atomicOr(p.status, kStatusPopRounds);
                break;
            }
            const int stamp = (rounds - 1) % kMaxStamp15 + 1;
            const int vis = stamp | kVisited16;
            if (stamp == 1 && rounds > 1) {  // stamps wrap: forget old ones
                for (int v = tid; v < n; v += BT)
                    if (lo16[v] != kFinal16) lo16[v] = 0;
                __syncthreads();
            }
            // (a) pop: every vertex on a cycle advances to its next stack entry
            for (int i = tid; i < nX; i += BT) {
                const int x = X[i];
                const int ox = orig_of(gd, x);
                int k = pop[x] + 1;
                int y = stack_entry(gd, p.key0, p.key1, x, ox, (uint32_t)k, tree);
                if (y >= n) {  // a pendant vertex: skip its 2-cycle
                    const int2 e = core_entry_of(gd.rp, gd.ci, gd.graph, p.key0, p.key1, x, ox, (uint32_t)k, tree, n);
                    my_skips += (unsigned)(e.y - k);
                    y = e.x;
                    k = e.y;
                }
                pop[x] = k;
                nxt[x] = y;
                nx16[x] = (uint16_t)y;
                lo16[x] = (uint16_t)stamp;
                pos[x] = i;
            }
            if (tid == 0) {
                s_draws += (unsigned long long)nX;
                s_cnt = 0;
                s_linked = 0;
                // mark paths for other walks only while walks are long
                s_mark_on = (rounds == 1) || (s_maxwalk > kMarkMinWalk);
                s_maxwalk = 0;
                my_max_pops = max(my_max_pops, nX);
            }
            __syncthreads();
            // (b) S(x): first redrawn vertex or known-final vertex after x.
            //     A walk that reaches a vertex another walk of this round
            //     already passed stops there and takes that walk's result
            //     (the two paths coincide from there on); the links are
            //     resolved after the barrier. Links cannot form a cycle: every
            //     cycle of this round passes a redrawn vertex.
            //     A walk publishes the owner of a vertex before its mark
            //     (block fence), so a walk that sees the mark reads the
            //     owner of this round. The first kQuietSteps vertices of a
            //     walk are not marked: short walks skip the bookkeeping.
            const bool mark_on = s_mark_on;
            for (int i = tid; i < nX; i += BT) {
                int y = nx16[X[i]];
                int res = -2, len = 0;
                for (int guard = 0; guard <= n; ++guard) {
                    const int m = lo16[y];
                    if (m == kFinal16) { res = -1; break; }
                    if (m == stamp) { res = pos[y]; break; }
                    if (m == vis) {
                        __threadfence_block();
                        res = -3 - owner[y];
                        s_linked = 1;
                        break;
                    }
                    if (mark_on && len >= kQuietSteps) {
                        owner[y] = i;
                        __threadfence_block();
                        lo16[y] = (uint16_t)vis;
                    }
                    ++len;
                    y = nx16[y];
                }
                if (res == -2) { s_err = 1; res = -1; }
                Sx[i] = res;
                wlen[i] = len;
                atomicMax(&s_maxwalk, len);
            }
            __syncthreads();
            if (s_linked) {  // some walk stopped on another's path: resolve the links
                for (int i = tid; i < nX; i += BT) {
                    int r = Sx[i];
                    for (int guard = 0; r <= -3 && guard <= nX; ++guard) {
                        const int j = -3 - r;
                        if (j >= nX) break;  // not a walk of this round: reported below
                        r = Sx[j];
                    }
                    if (r <= -3 || r >= nX) { s_err = 1; r = -1; }
                    Sx[i] = r;  // a reader sees the link or its result: both lead to the same end
                }
                __syncthreads();
            }
            // (c) nodes that reach -1 mark x and their own walked part final
            //     (a linked walk's remainder is marked by its owner, which
            //     reaches -1 too); nodes on a cycle of i -> S(i) queue their
            //     whole segment (x up to S(x)) for popping; the other nodes
            //     keep their stack tops.
            for (int i = tid; i < nX; i += BT) {
                const int kind = classify_node(Sx, i, nX);
                int y = X[i];
                if (kind == 1) {
                    const int len = wlen[i];
                    lo16[y] = kFinal16;
                    for (int k = 0; k < len; ++k) {
                        y = nx16[y];
                        lo16[y] = kFinal16;
                    }
                } else if (kind == 2) {
                    for (int guard = 0; guard <= n; ++guard) {
                        Xn[min(atomicAdd(&s_cnt, 1), n)] = y;  // more than n entries: reported below
                        y = nx16[y];
                        if (lo16[y] == stamp) break;
                    }
                    if (lo16[y] != stamp) s_err = 1;  // a cycle segment ends at a redrawn vertex
                }
            }
            __syncthreads();
            nX = s_cnt;
            int32_t *tmp = X; X = Xn; Xn = tmp;
            if (s_err || nX > n) {
                failed = true;
                if (tid == 0) atomicOr(p.status, kStatusBadState);
                break;
            }
            __syncthreads();
        }
        if (failed) break;
        UST_PHASE(5);
        if (tid == 0) {
            my_draws += s_draws;
            my_rounds += (unsigned long long)rounds;
            my_max_rounds = max(my_max_rounds, rounds);
        }
        if (p.edge_counts) {  // the tree's arcs v -> parent(v): the final stack entry of every v
            for (int v = tid; v < n; v += BT) {
                if (v == u) continue;
                const int o = orig_of(gd, v);
                const int b = __ldg(gd.rp + v), e = __ldg(gd.rp + v + 1);
                const unsigned long long x = philox_x64((uint32_t)o, (uint32_t)pop[v], tree, gd.graph, p.key0, p.key1);
                const long long row = gd.rp_in ? (long long)__ldg(gd.rp_in + o) : (long long)b;  // input arc index
                atomicAdd(p.edge_counts + gd.aoff + row + (long long)__umul64hi(x, (unsigned long long)(e - b)), 1ull);
            }
        }

        if (p.mode == 1) {  // export the tree in input ids (nothing is left out of such launches)
            const long long ob = s_tree * (long long)n;
            for (int v = tid; v < n; v += BT) {
                const int o = orig_of(gd, v);
                const int tp = nxt[v];
                p.next_out[ob + o] = (tp < 0) ? -1 : orig_of(gd, tp);
                if (p.pops_out) p.pops_out[ob + o] = pop[v];
            }
            __syncthreads();
            continue;
        }
        __syncthreads();

        // ---- 2. DFS intervals ---------------------------------------------
        // Subtree sizes from the leaves: C[v] = pending children << 16 | sum
        // of finished children's sizes (0 exactly for leaves); the last child
        // continues upwards and each arrival reads its offset inside the
        // parent's interval from the same atomic.
        for (int v = tid; v < n; v += BT) C[v] = 0u;
        __syncthreads();
        for (int b0 = tid; b0 < n; b0 += BT * kWalks) {
            int y[kWalks];
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                const int v = b0 + k * BT;
                y[k] = (v < n && v != u) ? nxt[v] : -1;
            }
#pragma unroll
            for (int k = 0; k < kWalks; ++k)
                if (y[k] >= 0) atomicAdd(&C[y[k]], kC16);
        }
        __syncthreads();
        UST_PHASE(6);
        {
            // own leaves (C[v] == 0; inner vertices never return to 0), with
            // the next start and its parent fetched one step ahead
            int cand = tid;
            int sv = -1, spar = -1;
            while (cand < n) {
                const int v = cand;
                cand += BT;
                if (v != u && C[v] == 0u) {
                    sv = v;
                    spar = nxt[v];
                    break;
                }
            }
            int x[kWalks], par[kWalks];
            uint32_t carry[kWalks];
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                x[k] = sv;
                par[k] = spar;
                carry[k] = 1u;
                sv = -1;
                spar = -1;
                while (cand < n) {
                    const int v = cand;
                    cand += BT;
                    if (v != u && C[v] == 0u) {
                        sv = v;
                        spar = nxt[v];
                        break;
                    }
                }
            }
            for (int guard = 0; guard <= 2 * n + 2; ++guard) {
                uint32_t old[kWalks];
                int gp[kWalks];
#pragma unroll
                for (int k = 0; k < kWalks; ++k) {
                    old[k] = (par[k] >= 0) ? atomicAdd(&C[par[k]], carry[k] - kC16) : 0u;
                    gp[k] = (par[k] >= 0 && par[k] != u) ? nxt[par[k]] : -1;
                }
                bool any = false;
#pragma unroll
                for (int k = 0; k < kWalks; ++k) {
                    if (par[k] >= 0) {
                        off[x[k]] = 1 + (int)(old[k] & 0xFFFFu);
                        if (par[k] != u && (old[k] >> 16) == 1u) {
                            carry[k] = (old[k] & 0xFFFFu) + carry[k] + 1u;
                            x[k] = par[k];
                            par[k] = gp[k];
                        } else {
                            x[k] = sv;
                            par[k] = spar;
                            carry[k] = 1u;
                            sv = -1;
                            spar = -1;
                            while (cand < n) {
                                const int v = cand;
                                cand += BT;
                                if (v != u && C[v] == 0u) {
                                    sv = v;
                                    spar = nxt[v];
                                    break;
                                }
                            }
                        }
                    }
                    any |= (par[k] >= 0);
                }
                if (!any) break;
            }
        }
        __syncthreads();
        UST_PHASE(7);
        // preorder numbers: sizes go to global memory, then the shared words
        // become (ancestor << 16 | partial offset sum) and pointer jumping
        // sums the offsets up to u in place.
        for (int b0 = tid; b0 < n; b0 += BT * kWalks) {
            int pa[kWalks], of[kWalks];
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                const int v = b0 + k * BT;
                const bool ok = v < n && v != u;
                pa[k] = ok ? nxt[v] : u;
                of[k] = ok ? off[v] : 0;
            }
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                const int v = b0 + k * BT;
                if (v < n) {
                    gsz[v] = (int)(C[v] & 0xFFFFu) + 1;
                    C[v] = ((uint32_t)pa[k] << 16) | (uint32_t)of[k];
                }
            }
        }
        __syncthreads();
        bool jfail = true;
        for (int step = 0; step < p.max_steps + 2; ++step) {
            int pending = 0;
            for (int v = tid; v < n; v += BT) {
                const uint32_t a = C[v];
                const int j = (int)(a >> 16);
                if (j == u) continue;
                const uint32_t b = C[j];
                const int j2 = (int)(b >> 16);
                C[v] = (b & 0xFFFF0000u) | ((a + b) & 0xFFFFu);
                pending |= (j2 != u);
            }
            if (!__syncthreads_or(pending)) {
                jfail = false;
                break;
            }
        }
        if (jfail) {
            if (tid == 0) atomicOr(p.status, kStatusJumpSteps);
            break;
        }
        // the high half (now u everywhere) becomes the tree parent, so one
        // shared word per vertex serves Algorithm 2
        for (int b0 = tid; b0 < n; b0 += BT * kWalks) {
            int pa[kWalks];
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                const int v = b0 + k * BT;
                pa[k] = (v < n) ? nxt[v] : 0;
            }
#pragma unroll
            for (int k = 0; k < kWalks; ++k) {
                const int v = b0 + k * BT;
                if (v < n) C[v] = ((uint32_t)(uint16_t)pa[k] << 16) | (C[v] & 0xFFFFu);
            }
        }
        __syncthreads();
        UST_PHASE(8);

        // ---- 3. Algorithm 2 ------------------------------------------------
        // Shallow BFS paths (f^c(u) <= kFlatDepth n): one independent test per
        // path entry, updates of R by atomics. Deep paths: one thread per
        // vertex walks its own path and adds its count once.
        if (gd.fc <= kFlatDepth * n) {
            // One independent test per entry q of the flattened paths: the edge
            // (a, b) = (path[q], pchild[q]) of P(v), v = powner[q]; downwards
            // (parent(b) = a) it adds +1 when v lies in b's subtree, upwards
            // (parent(a) = b) -1 when v lies in a's subtree.
            // C[x] = parent(x) << 16 | pre(x); parent(u) reads as 0xFFFF.
            for (int q0 = tid; q0 - (tid & 31) < gd.fc; q0 += BT * kPairs) {  // uniform per warp
                int a[kPairs], b[kPairs], v[kPairs];
    #pragma unroll
                for (int k = 0; k < kPairs; ++k) {
                    const int q = q0 + k * BT;
                    const bool ok = q < gd.fc;
                    a[k] = ok ? __ldg(gd.path + q) : -1;
                    b[k] = ok ? __ldg(gd.pchild + q) : 0;
                    v[k] = ok ? __ldg(gd.powner + q) : 0;
                }
                int tx[kPairs], sg[kPairs], lo[kPairs], pv[kPairs];
    #pragma unroll
                for (int k = 0; k < kPairs; ++k) {
                    tx[k] = 0;
                    sg[k] = 0;
                    lo[k] = 0;
                    pv[k] = 0;
                    if (a[k] >= 0) {
                        const uint32_t ca = C[a[k]], cb = C[b[k]];
                        pv[k] = (int)(C[v[k]] & 0xFFFFu);
                        if ((int)(cb >> 16) == a[k]) {  // the tree uses (a, b) downwards: interval of b
                            tx[k] = b[k];
                            sg[k] = 1;
                            lo[k] = (int)(cb & 0xFFFFu);
                        } else if ((int)(ca >> 16) == b[k]) {  // upwards: interval of a
                            tx[k] = a[k];
                            sg[k] = -1;
                            lo[k] = (int)(ca & 0xFFFFu);
                        }
                    }
                }
                int sz[kPairs];
    #pragma unroll
                for (int k = 0; k < kPairs; ++k) sz[k] = (sg[k] != 0) ? gsz[tx[k]] : 0;
    #pragma unroll
                for (int k = 0; k < kPairs; ++k) {
                    // lanes testing entries of the same vertex add up first, then
                    // one of them updates R (consecutive entries share an owner)
                    if (sg[k] != 0 && lo[k] <= pv[k] && pv[k] < lo[k] + sz[k]) {
                        if (p.R_direct)
                            atomicAdd(p.R_direct + gd.voff + v[k], (unsigned long long)(long long)sg[k]);
                        else
                            atomicAdd(Rp + v[k], sg[k]);
                    }
                }
            }
        } else {
            // C[x] = parent(x) << 16 | pre(x); parent(u) reads as 0xFFFF.
            for (int v = tid; v < n; v += BT) {
                if (v == u) continue;
                const uint32_t cv = C[v];
                const int pv = (int)(cv & 0xFFFFu);
                const int s0 = __ldg(gd.pathptr + v);
                const int d = __ldg(gd.pathptr + v + 1) - s0;
                int prevb = v, prevnb = (int)(cv >> 16), prevpre = pv;
                int cnt = 0;
                for (int c = 0; c < d; c += kPathChunk) {
                    int a[kPathChunk], na[kPathChunk], pa[kPathChunk], tx[kPathChunk], sg[kPathChunk], lo[kPathChunk];
    #pragma unroll
                    for (int j = 0; j < kPathChunk; ++j) a[j] = (c + j < d) ? __ldg(gd.path + s0 + c + j) : -1;
    #pragma unroll
                    for (int j = 0; j < kPathChunk; ++j) {
                        const uint32_t w = (a[j] >= 0) ? C[a[j]] : 0xFFFE0000u;
                        na[j] = (int)(w >> 16);
                        pa[j] = (int)(w & 0xFFFFu);
                    }
    #pragma unroll
                    for (int j = 0; j < kPathChunk; ++j) {
                        const int b = (j == 0) ? prevb : a[j - 1];
                        const int nb = (j == 0) ? prevnb : na[j - 1];
                        const int pb = (j == 0) ? prevpre : pa[j - 1];
                        tx[j] = -1;
                        sg[j] = 0;
                        lo[j] = 0;
                        if (a[j] >= 0) {
                            if (nb == a[j]) {  // the tree uses (a, b) downwards: interval of b
                                tx[j] = b;
                                sg[j] = 1;
                                lo[j] = pb;
                            } else if (na[j] == b) {  // upwards: interval of a
                                tx[j] = a[j];
                                sg[j] = -1;
                                lo[j] = pa[j];
                            }
                        }
                    }
                    int sz[kPathChunk];
    #pragma unroll
                    for (int j = 0; j < kPathChunk; ++j) sz[j] = (sg[j] != 0) ? gsz[tx[j]] : 0;
    #pragma unroll
                    for (int j = 0; j < kPathChunk; ++j)
                        if (sg[j] != 0 && lo[j] <= pv && pv < lo[j] + sz[j]) cnt += sg[j];
                    prevb = a[kPathChunk - 1];
                    prevnb = na[kPathChunk - 1];
                    prevpre = pa[kPathChunk - 1];
                }
                if (p.R_direct) {
                    if (cnt != 0) atomicAdd(p.R_direct + gd.voff + v, (unsigned long long)(long long)cnt);
                } else {
                    Rp[v] += cnt;
                }
            }
        }
        __syncthreads();
        UST_PHASE(9);
        if (tid == 0) {
            unsigned long long tot = 0ull;
            for (int k = 0; k < 10; ++k) tot += cyc[k];
            cyc[10] = tot;
        }
    }
#undef UST_PHASE

    if (tid == 0) {
        atomicAdd(p.stats + 0, my_draws);
        atomicAdd(p.stats + 1, my_rounds);
        atomicMax(p.stats + 2, (unsigned long long)my_max_rounds);
        atomicMax(p.stats + 3, (unsigned long long)my_max_pops);
        for (int k = 0; k < 11; ++k) atomicAdd(p.stats + 8 + k, cyc[k]);
    }
    if (my_skips) atomicAdd(p.stats + 0, 2ull * my_skips);  // as in the large-graph kernel
}

// out[v] += sum over partial rows of Rp[c][v] (exact, fixed order).
// Row v of Rp belongs to input vertex orig[v] (v itself when orig is NULL).
// out[orig(v)] += the launch's count of v, summed over the CTAs' rows. A
// pendant vertex v (id ncore and up) lies below its one neighbour w in every
// tree, and its BFS path is w's with the edge (w, v) in front, which every
// tree uses downwards: its count per tree is 1 + w's.
__global__ void reduce_counts_kernel(int n, int rows, const int32_t *__restrict__ Rp, long long *__restrict__ out,
                                     const int32_t *__restrict__ orig, int ncore, long long trees,
                                     const int32_t *__restrict__ srp, const int32_t *__restrict__ sci)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const bool pendant = v >= ncore;
        const int src = pendant ? sci[srp[v]] : v;
        long long s = pendant ? trees : 0;
        for (int c = 0; c < rows; ++c) s += Rp[(long long)c * n + src];
        out[orig ? orig[v] : v] += s;
    }
}

// Shared counters for graphs of at most this many vertices (4 B each, below
// 2^16 so that two 16-bit halves fit one word).
constexpr int kSmemMaxN = kSmemMaxVertices;

size_t smem_bytes_for(int max_n) { return (size_t)((max_n + 1) / 2) * 2 * sizeof(uint32_t); }

int64_t stride_for(int max_n) { return ((int64_t)max_n + 2 + 31) / 32 * 32; }

// Dynamic shared memory of the large-graph sampler: the preorder chunk.
constexpr size_t large_smem_bytes(int bt) { return (size_t)kPreChunkPerThread * bt * sizeof(unsigned long long); }

// Graphs of at most kSmemMaxN vertices run the shared-memory kernel at any
// shape; up to kTierMaxVertices the same kernel with its last words in the
// workspace tail; larger graphs the large-graph kernel, built for 256
// threads and more, whose only shared array is the preorder chunk (the rest
// of the SM's on-chip memory goes to L1).
template <int BT>
cudaError_t launch_sampler(int grid, cudaStream_t st, const SampleParams &p)
{
    if (p.max_n <= kSmemMaxN) {
        const size_t bytes = smem_bytes_for(p.max_n);
        cudaError_t e = cudaFuncSetAttribute(sample_aggregate_smem_kernel<BT, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        sample_aggregate_smem_kernel<BT, false><<<grid, BT, bytes, st>>>(p);
    } else if (p.max_n <= kTierMaxVertices) {
        const size_t bytes = (size_t)kSmemWords * sizeof(uint32_t);
        cudaError_t e = cudaFuncSetAttribute(sample_aggregate_smem_kernel<BT, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        sample_aggregate_smem_kernel<BT, true><<<grid, BT, bytes, st>>>(p);
    } else {
        if constexpr (BT >= 256) {
            constexpr size_t bytes = large_smem_bytes(BT);
            cudaError_t e = cudaFuncSetAttribute(sample_aggregate_large_kernel<BT>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
            if (e != cudaSuccess) return e;
            sample_aggregate_large_kernel<BT><<<grid, BT, bytes, st>>>(p);
        } else {
            return cudaErrorInvalidConfiguration;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_shape(const LaunchCfg &cfg, int grid, cudaStream_t st, const SampleParams &p)
{
    switch (cfg.bt) {
    case 64: return launch_sampler<64>(grid, st, p);
    case 128: return launch_sampler<128>(grid, st, p);
    case 256: return launch_sampler<256>(grid, st, p);
    case 512: return launch_sampler<512>(grid, st, p);
    case 1024: return launch_sampler<1024>(grid, st, p);
    default: return cudaErrorInvalidConfiguration;
    }
}

// Resident CTAs per SM of the kernel that serves graphs of max_n vertices at
// BT threads (registers, shared memory and the SM's thread limit together).
template <int BT>
int resident_ctas(int max_n)
{
    int blocks = 0;
    if (max_n <= kSmemMaxN) {
        const size_t bytes = smem_bytes_for(max_n);
        if (cudaFuncSetAttribute(sample_aggregate_smem_kernel<BT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes) != cudaSuccess)
            return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, sample_aggregate_smem_kernel<BT, false>, BT,
                                                          bytes) != cudaSuccess)
            return 0;
    } else if (max_n <= kTierMaxVertices) {
        const size_t bytes = (size_t)kSmemWords * sizeof(uint32_t);
        if (cudaFuncSetAttribute(sample_aggregate_smem_kernel<BT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes) != cudaSuccess)
            return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, sample_aggregate_smem_kernel<BT, true>, BT,
                                                          bytes) != cudaSuccess)
            return 0;
    } else {
        if constexpr (BT >= 256) {
            constexpr size_t bytes = large_smem_bytes(BT);
            if (cudaFuncSetAttribute(sample_aggregate_large_kernel<BT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)bytes) != cudaSuccess)
                return 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, sample_aggregate_large_kernel<BT>, BT, bytes) !=
                cudaSuccess)
                return 0;
        }
    }
    return blocks;
}

int resident_ctas_for(int bt, int max_n)
{
    switch (bt) {
    case 64: return resident_ctas<64>(max_n);
    case 128: return resident_ctas<128>(max_n);
    case 256: return resident_ctas<256>(max_n);
    case 512: return resident_ctas<512>(max_n);
    case 1024: return resident_ctas<1024>(max_n);
    default: return 0;
    }
}

// Automatic threads per CTA: small trees get small CTAs (more trees in
// flight per SM, cheaper barriers), large ones a whole SM.
int default_bt(int max_n)
{
    if (max_n <= 8192) return 128;
    if (max_n <= 14336) return 256;
    if (max_n <= 28672) return 512;
    // above: one whole-SM tree per SM; the large-graph sampler's trees are
    // bound by their dependent chains, which 1,024 threads shorten most
    // (measured on R-MAT scale 22: 512 x 2 is 8% and 256 x 4 17% slower; a
    // 2^20-vertex hyperbolic graph, with its many popping rounds, gains 7%
    // at 512 x 2, which the launch-shape tuner finds)
    return 1024;
}

bool valid_bt(int bt) { return bt == 64 || bt == 128 || bt == 256 || bt == 512 || bt == 1024; }

int choose_cfg(Ctx *c, int max_n, int req_bt, int req_cps, LaunchCfg *out)
{
    int bt = valid_bt(req_bt) ? req_bt : default_bt(max_n);
    if (max_n > kTierMaxVertices && bt < 256) bt = 256;
    const int resident = resident_ctas_for(bt, max_n);
    if (resident < 1) return fail(c, UST_EINVAL, "no sampler launch shape fits this graph at the requested threads");
    const int cps = req_cps > 0 ? std::min(req_cps, resident) : resident;
    out->bt = bt;
    out->ctas = c->num_sms * cps;
    return UST_OK;
}

// Grows the workspace and partial-count arrays to at least these sizes.
int reserve_workspace(Ctx *c, int64_t ws_words, int64_t rp_words)
{
    if (ws_words > c->ws_cap) {
        cudaFree(c->d_ws);
        c->d_ws = nullptr;
        c->ws_cap = 0;
        if (cudaMalloc(&c->d_ws, (size_t)ws_words * sizeof(int32_t)) != cudaSuccess)
            return fail(c, UST_ENOMEM, "sampler workspace");
        c->ws_cap = ws_words;
    }
    if (rp_words > c->rp_cap) {
        cudaFree(c->d_Rp);
        c->d_Rp = nullptr;
        c->rp_cap = 0;
        if (cudaMalloc(&c->d_Rp, (size_t)rp_words * sizeof(int32_t)) != cudaSuccess)
            return fail(c, UST_ENOMEM, "partial counts");
        c->rp_cap = rp_words;
    }
    return UST_OK;
}

}  // namespace

int alloc_sampler(Ctx *c, int block_threads, int ctas_per_sm)
{
    c->req_bt = block_threads;
    c->req_cps = ctas_per_sm;
    int rc = choose_cfg(c, c->n, block_threads, ctas_per_sm, &c->cfg);
    if (rc) return rc;
    c->ws_stride = stride_for(c->n);
    return reserve_workspace(c, (int64_t)c->cfg.ctas * kWsArrays * c->ws_stride, (int64_t)c->cfg.ctas * c->n);
}

int alloc_batch_sampler(Ctx *c, int block_threads, int ctas_per_sm)
{
    c->req_bt = block_threads;
    c->req_cps = ctas_per_sm;
    int64_t ws = 0;
    for (int k = 0; k < kNumClasses; ++k) {
        if (c->class_maxn[k] <= 0) continue;
        // a tuned class keeps its shape unless the caller fixed one
        const bool tuned = c->class_tuned[k].bt > 0 && block_threads == 0 && ctas_per_sm == 0;
        const int bt = tuned ? c->class_tuned[k].bt : block_threads;
        const int cps = tuned ? c->class_tuned[k].ctas / std::max(1, c->num_sms) : ctas_per_sm;
        const int rc = choose_cfg(c, c->class_maxn[k], bt, cps, &c->class_cfg[k]);
        if (rc) return rc;
        ws = std::max<int64_t>(ws, (int64_t)c->class_cfg[k].ctas * kWsArrays * stride_for(c->class_maxn[k]));
    }
    return reserve_workspace(c, ws, 0);
}

// ---------------------------------------------------------------------------
// Launch-shape tuning (ust_opts.autotune). A sampler launch's shape, threads
// per CTA and resident CTAs per SM, changes its speed and never its counts.
// Each candidate shape that fits is timed on the same probe of the launch's
// own work items (their counts go to scratch and are discarded); the fastest
// is kept, and remembered per workload key for the life of the process.
namespace {

std::mutex g_tune_mutex;
std::map<TuneKey, LaunchCfg> g_tune_cache;

std::vector<LaunchCfg> tune_candidates(int num_sms, int max_n)
{
    std::vector<LaunchCfg> out;
    for (int bt : {64, 128, 256, 512, 1024}) {
        if (max_n > kTierMaxVertices && bt < 512) continue;  // slower in every measured large-graph case
        const int res = resident_ctas_for(bt, max_n);
        if (res < 1) continue;
        out.push_back(LaunchCfg{bt, num_sms * res});
        if (res >= 2) out.push_back(LaunchCfg{bt, num_sms * (res / 2)});
    }
    return out;
}

// One probe launch of `items` work items over d_graphs / d_items; counts go
// to d_scratch (indexed like a batch's R). *ms: its device time.
int probe_launch(Ctx *c, const LaunchCfg &cfg, const GraphDesc *d_graphs, const long long *d_items, int ngraphs,
                 long long items, int max_n, long long max_rounds, int64_t *d_scratch, float *ms)
{
    UST_CUDA_TRY(cudaMemsetAsync(c->d_stats, 0, 32 * sizeof(int64_t), c->stream));
    SampleParams p{};
    p.max_n = max_n;
    p.key0 = 0x5EEDu;  // any key: the probe's counts are discarded
    p.key1 = 0x7E57u;
    p.graphs = d_graphs;
    p.ngraphs = ngraphs;
    p.item_start = d_items;
    p.total_items = items;
    p.tree_offset = 0;
    p.ws = c->d_ws;
    p.stride = stride_for(max_n);
    p.Rp = c->d_Rp;
    unsigned long long *st = reinterpret_cast<unsigned long long *>(c->d_stats);
    p.next_tree = st + 4;
    p.stats = st;
    p.status = reinterpret_cast<int *>(st + 5);
    p.max_rounds = (int)std::min<long long>(max_rounds, 1ll << 30);
    int lg = 0;
    while ((1ll << lg) < (long long)max_n) ++lg;
    p.max_steps = lg + 4;
    p.mode = 0;
    p.R_direct = reinterpret_cast<unsigned long long *>(d_scratch);
    const int grid = (int)std::min<long long>(cfg.ctas, items);
    if ((int64_t)grid * kWsArrays * p.stride > c->ws_cap) return fail(c, UST_ECUDA, "tuning probe: workspace too small");
    cudaEvent_t e0 = c->ev[2 * Ctx::kEvSample], e1 = c->ev[2 * Ctx::kEvSample + 1];
    UST_CUDA_TRY(cudaEventRecord(e0, c->stream));
    const cudaError_t e = launch_shape(cfg, grid, c->stream, p);
    UST_CUDA_TRY(cudaEventRecord(e1, c->stream));
    c->launches += 1;
    if (e != cudaSuccess) return fail(c, UST_ECUDA, std::string("tuning probe launch: ") + cudaGetErrorString(e));
    UST_CUDA_TRY(cudaMemcpyAsync(c->h_stats, c->d_stats, 32 * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    UST_SYNC_TRY("tuning probe (" + std::to_string(cfg.bt) + " threads, " + std::to_string(grid) + " CTAs)");
    if (c->h_stats[5] & kStatusPopRounds) return fail(c, UST_ETIMEOUT, "a tree exceeded max_pop_rounds");
    if (c->h_stats[5])
        return fail(c, UST_ECUDA, "sampler reported an inconsistent state (check " + std::to_string(c->h_stats[6]) + ")");
    UST_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
    return UST_OK;
}

}  // namespace

int tune_launch(Ctx *c, const TuneKey &key, const GraphDesc *d_graphs, const long long *d_items, int ngraphs,
                long long items, int max_n, long long max_rounds, int64_t *d_scratch, LaunchCfg *out,
                double *best_ms_per_item)
{
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        const auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *out = it->second;
            if (best_ms_per_item) *best_ms_per_item = 0.0;
            return UST_OK;
        }
    }
    const std::vector<LaunchCfg> cands = tune_candidates(c->num_sms, max_n);
    if (cands.empty()) return fail(c, UST_EINVAL, "no sampler launch shape fits this graph");
    int64_t ws = 0;
    for (const LaunchCfg &k : cands)
        ws = std::max<int64_t>(ws, std::min<int64_t>(k.ctas, items) * kWsArrays * stride_for(max_n));
    int rc = reserve_workspace(c, ws, 0);
    if (rc) return rc;
    double best = 0.0;
    for (const LaunchCfg &k : cands) {
        float ms = 0.f;
        rc = probe_launch(c, k, d_graphs, d_items, ngraphs, items, max_n, max_rounds, d_scratch, &ms);
        if (rc) return rc;
        const double per = (double)ms / (double)items;
        if (best == 0.0 || per < best) {
            best = per;
            *out = k;
        }
    }
    c->ev_used[Ctx::kEvSample] = false;  // the probes' events are not a sampling phase
    if (best_ms_per_item) *best_ms_per_item = best;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = *out;
    return UST_OK;
}

// The single graph's descriptor: uploaded when B_u (pivot, path space) or
// the rows changed.
int upload_single_desc(Ctx *c, bool prune)
{
    GraphDesc gd{};
    gd.n = c->n;
    gd.u = c->pivot;
    gd.graph = (uint32_t)c->graph_id;
    gd.voff = 0;
    gd.tree_begin = 0;
    gd.rp = c->d_rp;
    gd.ci = c->d_ci;
    gd.bpar = c->d_bpar;
    gd.path = c->d_path;
    gd.pathptr = c->d_pathptr;
    gd.pchild = c->d_path + c->path_cap;
    gd.powner = c->d_path + 2 * c->path_cap;
    gd.fc = (int)c->farness;
    gd.aoff = 0;
    gd.orig = nullptr;
    gd.rp_in = nullptr;
    gd.ncore = c->n;
    // the large-graph sampler's relabelled view (not with the walk rows of
    // the biconnected-component variant, which the context swaps in)
    const bool relabelled = c->relabel && !c->blocks;
    if (relabelled) {
        gd.u = c->spivot;
        gd.rp = c->d_srp;
        gd.ci = c->d_sci;
        gd.path = c->d_spath;
        gd.pchild = c->d_spath + c->spath_cap;
        gd.powner = c->d_spath + 2 * c->spath_cap;
        gd.pathptr = c->d_spathptr;
        gd.orig = c->d_orig;
        gd.rp_in = c->d_rp;
        if (prune) {
            gd.ncore = c->ncore;
            gd.fc = (int)c->core_fc;  // the core's paths come first
        }
    }
    const GraphDesc &o = c->single_desc;
    const bool same = o.n == gd.n && o.u == gd.u && o.graph == gd.graph && o.rp == gd.rp && o.ci == gd.ci &&
                      o.bpar == gd.bpar && o.path == gd.path && o.pathptr == gd.pathptr && o.pchild == gd.pchild &&
                      o.powner == gd.powner && o.fc == gd.fc && o.orig == gd.orig && o.rp_in == gd.rp_in &&
                      o.ncore == gd.ncore;
    if (!c->single_desc_valid || !same) {
        c->single_desc = gd;
        const long long starts[2] = {0, kOpenEnd};
        UST_CUDA_TRY(cudaMemcpyAsync(c->d_graphs, &c->single_desc, sizeof(GraphDesc), cudaMemcpyHostToDevice,
                                     c->stream));
        UST_CUDA_TRY(cudaMemcpyAsync(c->d_items, starts, sizeof(starts), cudaMemcpyHostToDevice, c->stream));
        c->single_desc_valid = true;
    }
    return UST_OK;
}

int run_sampler(Ctx *c, int64_t t0, int64_t t1, uint64_t seed, int64_t *d_out, int32_t *d_next_out,
                int32_t *d_pops_out, int64_t *draws, int64_t *rounds, int *max_rounds, int *max_depth)
{
    if (t1 <= t0) return UST_OK;
    if (t0 < 0 || t1 > (int64_t)0xFFFFFFFFll) return fail(c, UST_EINVAL, "tree ids must lie in [0, 2^32)");
    const int mode = d_next_out ? 1 : 0;
    const int grid = (int)std::min<int64_t>(c->cfg.ctas, t1 - t0);
    if (mode == 0)
        UST_CUDA_TRY(cudaMemsetAsync(c->d_Rp, 0, (size_t)grid * c->n * sizeof(int32_t), c->stream));
    UST_CUDA_TRY(cudaMemsetAsync(c->d_stats, 0, 32 * sizeof(int64_t), c->stream));

    // pendant vertices are left out of the trees only when counts are
    // aggregated without arc counts (sampled trees and arcs need them all)
    const bool prune = mode == 0 && !c->d_ecount_tmp;
    const int drc = upload_single_desc(c, prune);
    if (drc) return drc;
    const bool relabelled = c->relabel && !c->blocks;
    const int ncore = (relabelled && prune) ? c->ncore : c->n;
    SampleParams p{};
    p.max_n = c->n;
    p.key0 = (uint32_t)(seed & 0xFFFFFFFFull);
    p.key1 = (uint32_t)(seed >> 32);
    p.graphs = c->d_graphs;
    p.ngraphs = 1;
    p.item_start = c->d_items;
    p.total_items = t1 - t0;
    p.tree_offset = t0;
    p.ws = c->d_ws;
    p.stride = c->ws_stride;
    p.Rp = c->d_Rp;
    p.edge_counts = (mode == 0) ? reinterpret_cast<unsigned long long *>(c->d_ecount_tmp) : nullptr;
    unsigned long long *st = reinterpret_cast<unsigned long long *>(c->d_stats);
    p.next_tree = st + 4;
    p.stats = st;
    p.status = reinterpret_cast<int *>(st + 5);
    // Every round pops at least one cycle and the expected number of pops per
    // tree is below sum_v deg(v) r(u, v) <= 2m ecc(u) (Lemma in Appendix A.2),
    // so the default bound is far above anything a correct run reaches.
    p.max_rounds = c->max_pop_rounds > 0
                       ? c->max_pop_rounds
                       : (int)std::min<int64_t>(16ll * ((int64_t)c->nnz * std::max(1, c->ecc) + c->n) + 1024,
                                                1ll << 30);
    int lg = 0;
    while ((1ll << lg) < (long long)c->n) ++lg;
    p.max_steps = lg + 4;
    p.mode = mode;
    p.next_out = d_next_out;
    p.pops_out = d_pops_out;

    phase_begin(c, Ctx::kEvSample);
    const cudaError_t e = launch_shape(c->cfg, grid, c->stream, p);
    phase_end(c, Ctx::kEvSample);
    c->launches += 1;
    if (e != cudaSuccess) return fail(c, UST_ECUDA, std::string("sampler launch: ") + cudaGetErrorString(e));
    if (mode == 0) {
        phase_begin(c, Ctx::kEvReduce);
        const int threads = 256;
        const int blocks = (int)std::min<int64_t>((c->n + threads - 1) / threads, (int64_t)c->num_sms * 8);
        reduce_counts_kernel<<<blocks, threads, 0, c->stream>>>(c->n, grid, c->d_Rp,
                                                                 reinterpret_cast<long long *>(d_out),
                                                                 relabelled ? c->d_orig : nullptr, ncore, t1 - t0,
                                                                 c->d_srp, c->d_sci);
        phase_end(c, Ctx::kEvReduce);
        c->launches += 1;
        UST_CUDA_TRY(cudaGetLastError());
    }
    UST_CUDA_TRY(cudaMemcpyAsync(c->h_stats, c->d_stats, 32 * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    UST_SYNC_TRY("sampler");
    const int status = (int)c->h_stats[5];
    if (status & kStatusPopRounds) return fail(c, UST_ETIMEOUT, "a tree exceeded max_pop_rounds");
    if (status & kStatusJumpSteps) return fail(c, UST_ETIMEOUT, "pointer jumping did not converge");
    if (status)
        return fail(c, UST_ECUDA, "sampler reported an inconsistent state (check " + std::to_string(c->h_stats[6]) + ")");
    // the first draws of the pendant vertices left out of the trees
    c->h_stats[0] += (t1 - t0) * (int64_t)(c->n - ncore);
    c->last_trees = t1 - t0;
    c->last_draws = c->h_stats[0];
    for (int k = 0; k < 12; ++k) c->last_phase_cycles[k] = c->h_stats[8 + k];
    if (draws) *draws = c->h_stats[0];
    if (rounds) *rounds = c->h_stats[1];
    if (max_rounds) *max_rounds = (int)c->h_stats[2];
    if (max_depth) *max_depth = (int)c->h_stats[3];
    return UST_OK;
}

}  // namespace ust

// ---------------------------------------------------------------------------
// Allocation-free variant of the tree counts (ust_tree_counts_noalloc).
//
// Some callers cannot call cudaMalloc: code whose device memory belongs to
// another allocator that must account for every byte (a framework's caching
// allocator, a fixed memory budget), or code that may not allocate once it
// has started. This variant runs B_u, the flattened BFS paths, the sampler
// and the count reduction entirely in one file-scope device array of fixed
// size; the caller passes only its inputs and its output.
//
// Limits: n <= kNoAllocMaxN vertices and f^c(u) = sum_v dist(u, v) <=
// kNoAllocMaxPath. The array is about 10.6 MB and stays resident on every GPU
// that loads this library until the process exits. Every call reuses it and
// overwrites the previous contents, so calls that overlap on the GPU (two
// streams, two host threads) race and must be serialised by the caller.
namespace ust {
namespace {

constexpr int kNoAllocMaxN = 4096;
constexpr int kNoAllocMaxPath = 262144;
constexpr int kNoAllocCtas = 32;
constexpr int kNoAllocThreads = 256;
constexpr long long kNoAllocStride = ((kNoAllocMaxN + 2 + 31) / 32) * 32;
// layout in int32 words: sampler workspace | partial counts | dist | bfs parent
//                        | path offsets | paths | stats (32 x int64)
//                        | graph descriptor and item starts
constexpr long long kNaWs = 0;
constexpr long long kNaRp = kNaWs + (long long)kNoAllocCtas * kWsArrays * kNoAllocStride;
constexpr long long kNaDist = kNaRp + (long long)kNoAllocCtas * kNoAllocMaxN;
constexpr long long kNaBpar = kNaDist + kNoAllocMaxN;
constexpr long long kNaPathPtr = kNaBpar + kNoAllocMaxN;
constexpr long long kNaPath = kNaPathPtr + ((kNoAllocMaxN + 1 + 31) / 32) * 32;
constexpr long long kNaStats = kNaPath + 3ll * kNoAllocMaxPath;  // ancestors, children, owners
constexpr long long kNaDesc = kNaStats + 2 * 32;  // one GraphDesc and two item starts
constexpr long long kNaWords = kNaDesc + 64;
static_assert(sizeof(GraphDesc) + 2 * sizeof(long long) <= 64 * sizeof(int32_t), "descriptor slot");
static_assert((kNaDesc * sizeof(int32_t)) % 16 == 0, "descriptor alignment");

static __device__ __align__(256) int32_t g_noalloc_scratch[kNaWords];

// One CTA: B_u by level-synchronous pull BFS (smallest-id parent), the
// connectivity check, f^c(u), the exclusive prefix of dist into pathptr and
// the flattened paths. Errors go to status (bit 1: disconnected, bit 2: too
// many path entries).
constexpr int kPrepThreads = 1024;
__device__ void prepare_graph(int n, int u, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              int32_t *dist, int32_t *bpar, int32_t *pathptr, int32_t *path, int32_t *pchild,
                              int32_t *powner, long long path_cap, int *status, int *ecc_out = nullptr,
                              int *fc_out = nullptr)
{
    __shared__ int s_warp[kPrepThreads / 32 + 1];
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int v = tid; v < n; v += kPrepThreads) {
        dist[v] = (v == u) ? 0 : -1;
        bpar[v] = -1;
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    int level = 0;
    for (; level < n; ++level) {
        int any = 0;
        for (int v = tid; v < n; v += kPrepThreads) {
            if (dist[v] >= 0) continue;
            for (int e = rp[v]; e < rp[v + 1]; ++e) {
                const int w = ci[e];
                if (dist[w] == level) {
                    dist[v] = level + 1;
                    bpar[v] = w;
                    any = 1;
                    break;
                }
            }
        }
        if (!__syncthreads_or(any)) break;
    }
    if (ecc_out && tid == 0) *ecc_out = level;
    // exclusive prefix of dist (unreached vertices flag the graph as disconnected)
    int carry = 0;
    for (int base = 0; base < n; base += kPrepThreads) {
        const int i = base + tid;
        const int d = (i < n) ? dist[i] : 0;
        if (d < 0) s_bad = 1;
        const int x = d > 0 ? d : 0;
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
        if (i < n) pathptr[i] = carry + s_warp[wid] + incl - x;
        carry += s_warp[32];
        __syncthreads();
    }
    if (tid == 0) {
        pathptr[n] = carry;
        if (fc_out) *fc_out = carry;
    }
    if (s_bad || carry > path_cap) {
        if (tid == 0) *status |= s_bad ? 1 : 2;
        return;
    }
    __syncthreads();
    for (int v = tid; v < n; v += kPrepThreads) {
        int k = pathptr[v];
        const int end = pathptr[v + 1];
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

__global__ void __launch_bounds__(kPrepThreads) noalloc_prepare_kernel(int n, int u, uint32_t graph,
                                                                       const int32_t *__restrict__ rp,
                                                                       const int32_t *__restrict__ ci, int32_t *dist,
                                                                       int32_t *bpar, int32_t *pathptr, int32_t *path,
                                                                       int32_t *pchild, int32_t *powner,
                                                                       int path_cap, int *status, int *ecc_out,
                                                                       GraphDesc *desc, long long *item_start)
{
    if (threadIdx.x == 0) {
        GraphDesc d;
        d.n = n;
        d.u = u;
        d.graph = graph;
        d.voff = 0;
        d.tree_begin = 0;
        d.rp = rp;
        d.ci = ci;
        d.bpar = bpar;
        d.path = path;
        d.pathptr = pathptr;
        d.pchild = pchild;
        d.powner = powner;
        d.fc = 0;  // set below, once f^c(u) is known
        d.aoff = 0;
        d.orig = nullptr;
        d.rp_in = nullptr;
        d.ncore = n;
        *desc = d;
        item_start[0] = 0;
        item_start[1] = kOpenEnd;
    }
    prepare_graph(n, u, rp, ci, dist, bpar, pathptr, path, pchild, powner, path_cap, status, ecc_out, &desc->fc);
}

// Device address of g_noalloc_scratch, looked up once per device.
constexpr int kMaxDevices = 64;
int32_t *g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mutex;

}  // namespace

}  // namespace ust

extern "C" int ust_tree_counts_noalloc(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int32_t nnz,
                                       int32_t pivot, int64_t t0, int64_t t1, uint64_t seed, int32_t graph_id,
                                       int64_t *R_out, void *stream)
{
    using namespace ust;
    if (!row_ptr || !col_idx || !R_out || n < 2 || nnz < 2 || pivot < 0 || pivot >= n || t0 < 0 || t1 < t0 ||
        t1 > (int64_t)0xFFFFFFFFll)
        return UST_EINVAL;
    if (n > kNoAllocMaxN) return UST_EINVAL;  // beyond the fixed scratch array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return UST_ECUDA;
    int32_t *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return UST_ECUDA;
            g_noalloc_ptr[dev] = static_cast<int32_t *>(ptr);
        }
        base = g_noalloc_ptr[dev];
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int32_t *ws = base + kNaWs, *Rp = base + kNaRp, *dist = base + kNaDist, *bpar = base + kNaBpar;
    int32_t *pathptr = base + kNaPathPtr, *path = base + kNaPath;
    unsigned long long *stats = reinterpret_cast<unsigned long long *>(base + kNaStats);
    // the previous call's contents stay in the array: clear what must start at zero
    if (cudaMemsetAsync(stats, 0, 32 * sizeof(unsigned long long), st) != cudaSuccess) return UST_ECUDA;
    if (cudaMemsetAsync(Rp, 0, (size_t)kNoAllocCtas * n * sizeof(int32_t), st) != cudaSuccess) return UST_ECUDA;
    int *status = reinterpret_cast<int *>(stats + 5);
    int *ecc_dev = reinterpret_cast<int *>(stats + 6);
    GraphDesc *desc = reinterpret_cast<GraphDesc *>(base + kNaDesc);
    long long *item_start = reinterpret_cast<long long *>(desc + 1);
    noalloc_prepare_kernel<<<1, kPrepThreads, 0, st>>>(n, pivot, (uint32_t)graph_id, row_ptr, col_idx, dist, bpar,
                                                        pathptr, path, path + kNoAllocMaxPath,
                                                        path + 2 * kNoAllocMaxPath, kNoAllocMaxPath, status, ecc_dev,
                                                        desc, item_start);
    if (cudaGetLastError() != cudaSuccess) return UST_ECUDA;
    unsigned long long h_stats[32];
    if (cudaMemcpyAsync(h_stats, stats, sizeof(h_stats), cudaMemcpyDeviceToHost, st) != cudaSuccess) return UST_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return UST_ECUDA;
    if (h_stats[5] & 1) return UST_ENOTCONNECTED;
    if (h_stats[5] & 2) return UST_EINVAL;  // f^c(u) beyond the fixed scratch array
    // the checks passed: only now is R_out written
    if (cudaMemsetAsync(R_out, 0, (size_t)n * sizeof(int64_t), st) != cudaSuccess) return UST_ECUDA;
    if (t1 > t0) {
        const int ecc = std::max(1, (int)(uint32_t)h_stats[6]);  // ecc(u) from B_u: the popping-round limit
        SampleParams p{};
        p.max_n = n;
        p.key0 = (uint32_t)(seed & 0xFFFFFFFFull);
        p.key1 = (uint32_t)(seed >> 32);
        p.graphs = desc;
        p.ngraphs = 1;
        p.item_start = item_start;
        p.total_items = t1 - t0;
        p.tree_offset = t0;
        p.ws = ws;
        p.stride = kNoAllocStride;
        p.Rp = Rp;
        p.next_tree = stats + 4;
        p.stats = stats;
        p.status = status;
        p.max_rounds = (int)std::min<int64_t>(16ll * ((int64_t)nnz * ecc + n) + 1024, 1ll << 30);
        int lg = 0;
        while ((1ll << lg) < (long long)n) ++lg;
        p.max_steps = lg + 4;
        p.mode = 0;
        p.next_out = nullptr;
        p.pops_out = nullptr;
        const int grid = (int)std::min<int64_t>(kNoAllocCtas, t1 - t0);
        if (launch_sampler<kNoAllocThreads>(grid, st, p) != cudaSuccess) return UST_ECUDA;
        reduce_counts_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, grid, Rp, reinterpret_cast<long long *>(R_out),
                                                                nullptr, n, 0, nullptr, nullptr);
        if (cudaGetLastError() != cudaSuccess) return UST_ECUDA;
        if (cudaMemcpyAsync(h_stats, stats, sizeof(h_stats), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return UST_ECUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return UST_ECUDA;
        if (h_stats[5] & (kStatusPopRounds | kStatusJumpSteps)) return UST_ETIMEOUT;
        if (h_stats[5]) return UST_ECUDA;
    }
    return UST_OK;
}

// ---------------------------------------------------------------------------
// Batches of graphs: B_u of every graph in one launch (one CTA per graph) and
// the sampler over (graph, tree) work items.
namespace ust {
namespace {

// out: status of graph g at [g], ecc(u) at [count + g], f^c(u) at [2 count + g]
__global__ void __launch_bounds__(kPrepThreads) batch_prepare_kernel(const PrepDesc *__restrict__ d, int count,
                                                                     int *out)
{
    const PrepDesc g = d[blockIdx.x];
    prepare_graph(g.n, g.u, g.rp, g.ci, g.dist, g.bpar, g.pathptr, g.path, g.pchild, g.powner, g.path_cap,
                  out + blockIdx.x, out + count + blockIdx.x, out + 2 * count + blockIdx.x);
}

// B_u of one graph in one CTA (small single graphs): out as above, count 1.
__global__ void __launch_bounds__(kPrepThreads) single_prepare_kernel(PrepDesc g, int *out)
{
    prepare_graph(g.n, g.u, g.rp, g.ci, g.dist, g.bpar, g.pathptr, g.path, g.pchild, g.powner, g.path_cap, out,
                  out + 1, out + 2);
}

// diag of graph blockIdx.x: L^+[u,u] = x_u, L^+[v,v] = (R[v]/tau - x_u) + 2 x_v
__global__ void batch_combine_kernel(const CombineDesc *__restrict__ d, const long long *__restrict__ R,
                                     const double *__restrict__ x, double *__restrict__ diag)
{
    const CombineDesc g = d[blockIdx.x];
    const double xu = x[g.voff + g.u];
    const double tau = (double)g.trees;
    for (int v = threadIdx.x; v < g.n; v += blockDim.x) {
        const long long i = g.voff + v;
        if (v == g.u) {
            diag[i] = xu;
        } else {
            const double r = __ddiv_rn((double)R[i], tau);
            const double t = __dsub_rn(r, xu);
            diag[i] = __dadd_rn(t, __dmul_rn(2.0, x[i]));
        }
    }
}

}  // namespace

int run_prepare_single(Ctx *c, const PrepDesc &d, int *d_out)
{
    single_prepare_kernel<<<1, kPrepThreads, 0, c->stream>>>(d, d_out);
    c->launches += 1;
    UST_CUDA_TRY(cudaGetLastError());
    return UST_OK;
}

int run_batch_prepare(Ctx *c, const PrepDesc *d_desc, int count, int *d_out)
{
    batch_prepare_kernel<<<count, kPrepThreads, 0, c->stream>>>(d_desc, count, d_out);
    c->launches += 1;
    UST_CUDA_TRY(cudaGetLastError());
    return UST_OK;
}

int run_batch_combine(Ctx *c, const CombineDesc *d_desc, int count, double *d_diag)
{
    phase_begin(c, Ctx::kEvCombine);
    batch_combine_kernel<<<count, 256, 0, c->stream>>>(d_desc, reinterpret_cast<const long long *>(c->d_R), c->d_x,
                                                       d_diag);
    phase_end(c, Ctx::kEvCombine);
    c->launches += 1;
    UST_CUDA_TRY(cudaGetLastError());
    return UST_OK;
}

int run_batch_sampler(Ctx *c, const LaunchCfg &cfg, const GraphDesc *d_graphs, const long long *d_item_start,
                      int ngraphs, long long total_items, int max_n, long long max_rounds, uint64_t seed,
                      int64_t *d_R, int64_t *draws, int64_t *rounds, int *max_round_count, int *max_pops)
{
    if (total_items <= 0) return UST_OK;
    UST_CUDA_TRY(cudaMemsetAsync(c->d_stats, 0, 32 * sizeof(int64_t), c->stream));
    SampleParams p{};
    p.max_n = max_n;
    p.key0 = (uint32_t)(seed & 0xFFFFFFFFull);
    p.key1 = (uint32_t)(seed >> 32);
    p.ws = c->d_ws;
    p.stride = stride_for(max_n);
    p.Rp = c->d_Rp;
    p.tree_offset = 0;
    if ((int64_t)std::min<long long>(cfg.ctas, total_items) * kWsArrays * p.stride > c->ws_cap)
        return fail(c, UST_ECUDA, "batch sampler: workspace smaller than the launch needs");
    unsigned long long *st = reinterpret_cast<unsigned long long *>(c->d_stats);
    p.next_tree = st + 4;
    p.stats = st;
    p.status = reinterpret_cast<int *>(st + 5);
    p.max_rounds = (int)std::min<long long>(max_rounds, 1ll << 30);
    int lg = 0;
    while ((1ll << lg) < (long long)max_n) ++lg;
    p.max_steps = lg + 4;
    p.mode = 0;
    p.graphs = d_graphs;
    p.ngraphs = ngraphs;
    p.item_start = d_item_start;
    p.total_items = total_items;
    p.R_direct = reinterpret_cast<unsigned long long *>(d_R);
    p.edge_counts = reinterpret_cast<unsigned long long *>(c->d_ecount_tmp);
    const int grid = (int)std::min<long long>(cfg.ctas, total_items);
    phase_begin(c, Ctx::kEvSample);
    const cudaError_t e = launch_shape(cfg, grid, c->stream, p);
    phase_end(c, Ctx::kEvSample);
    c->launches += 1;
    if (e != cudaSuccess) return fail(c, UST_ECUDA, std::string("batch sampler launch: ") + cudaGetErrorString(e));
    UST_CUDA_TRY(cudaMemcpyAsync(c->h_stats, c->d_stats, 32 * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    UST_SYNC_TRY("batch sampler (" + std::to_string(cfg.bt) + " threads, " + std::to_string(grid) + " CTAs)");
    const int status = (int)c->h_stats[5];
    if (status & kStatusPopRounds) return fail(c, UST_ETIMEOUT, "a tree exceeded max_pop_rounds");
    if (status & kStatusJumpSteps) return fail(c, UST_ETIMEOUT, "pointer jumping did not converge");
    if (status)
        return fail(c, UST_ECUDA, "sampler reported an inconsistent state (check " + std::to_string(c->h_stats[6]) + ")");
    c->last_trees = total_items;
    c->last_draws = c->h_stats[0];
    for (int k = 0; k < 12; ++k) c->last_phase_cycles[k] = c->h_stats[8 + k];
    if (draws) *draws = c->h_stats[0];
    if (rounds) *rounds = c->h_stats[1];
    if (max_round_count) *max_round_count = (int)c->h_stats[2];
    if (max_pops) *max_pops = (int)c->h_stats[3];
    return UST_OK;
}

}  // namespace ust
