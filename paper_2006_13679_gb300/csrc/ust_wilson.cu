// Sampling and aggregation: the loop of Algorithm 1 that samples a uniform
// spanning tree T rooted at u (Wilson's algorithm, Appendix A.2) and adds
// its Algorithm 2 counts to R.
//
// One CTA owns one tree at a time and takes tree ids from a global counter
// (persistent kernel). Per tree:
//
//  1. Cycle popping (Wilson's cycle-popping theorem, used in Appendix A.2).
//     Every vertex v != u has a stack of random neighbours, entry k being the
//     Philox draw keyed by (v, k, tree, graph). The current stack tops form a
//     functional graph. Each round classifies every unresolved vertex by
//     pointer jumping with a min-label: a vertex whose path reaches the
//     resolved set (vertices already known to reach u) is resolved and gets
//     its depth in T; every other vertex ends in a cycle, and the smallest
//     vertex of each cycle walks it once and pops it (every vertex on it
//     advances to its next stack entry). All disjoint cycles are popped in
//     the same round; by the theorem the final tree does not depend on that
//     order, so it equals the loop-erased-walk tree with the same stacks.
//  2. DFS intervals of T (Algorithm 2's discovery/finish times): vertices are
//     bucketed by depth, subtree sizes are accumulated bottom-up level by
//     level, children receive offsets from an atomic cursor of their parent
//     and preorder positions are assigned top-down. Any child order gives
//     valid nested intervals, and the subtree test does not depend on it.
//  3. Algorithm 2 with the inclusive subtree test: thread v walks P(v) up
//     B_u and adds +1 / -1 for every BFS edge that T uses downwards /
//     upwards above v. Counts go to the CTA's partial row Rp; a second kernel
//     sums the partial rows into the int64 R exactly.
#include <algorithm>

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

struct SampleParams {
    int n, u;
    uint32_t graph, key0, key1;
    const int32_t *rp, *ci, *bpar;
    int32_t *ws;
    long long stride;
    int32_t *Rp;
    long long t_begin, t_end;
    unsigned long long *next_tree;
    unsigned long long *stats;  // [0] draws, [1] rounds, [2] max rounds, [3] max depth
    int *status;
    int max_rounds, max_steps;
    int mode;  // 0: aggregate, 1: export trees
    int32_t *next_out, *pops_out;
};

// Stack entry `k` of vertex v: a uniformly chosen neighbour.
__device__ __forceinline__ int stack_entry(const SampleParams &p, int v, uint32_t k, uint32_t tree)
{
    const int b = __ldg(p.rp + v);
    const int e = __ldg(p.rp + v + 1);
    const unsigned long long x = philox_x64((uint32_t)v, k, tree, p.graph, p.key0, p.key1);
    const unsigned long long idx = __umul64hi(x, (unsigned long long)(e - b));
    return __ldg(p.ci + b + (int)idx);
}

// In-place exclusive prefix sum of a[0..len) by one CTA.
template <int BT>
__device__ void block_exclusive_scan(int32_t *a, int len, int *s_warp)
{
    constexpr int W = BT / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int carry = 0;
    for (int base = 0; base < len; base += BT) {
        const int i = base + threadIdx.x;
        const int x = (i < len) ? a[i] : 0;
        int incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_warp[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int w = (lane < W) ? s_warp[lane] : 0;
            int wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            if (lane < W) s_warp[lane] = wi - w;  // exclusive warp offsets
            if (lane == 31) s_warp[W] = wi;       // chunk total
        }
        __syncthreads();
        if (i < len) a[i] = carry + s_warp[wid] + incl - x;
        carry += s_warp[W];
        __syncthreads();
    }
}

template <int BT>
__global__ void __launch_bounds__(BT) sample_aggregate_kernel(SampleParams p)
{
    const int n = p.n, u = p.u, tid = threadIdx.x;
    int32_t *base = p.ws + (long long)blockIdx.x * kWsArrays * p.stride;
    int32_t *nxt = base;
    int32_t *pop = base + 1 * p.stride;
    int32_t *tdep = base + 2 * p.stride;
    int32_t *actA = base + 3 * p.stride;
    int32_t *actB = base + 4 * p.stride;
    int32_t *J0 = base + 5 * p.stride, *J1 = base + 6 * p.stride;
    int32_t *L0 = base + 7 * p.stride, *L1 = base + 8 * p.stride;
    int32_t *D0 = base + 9 * p.stride, *D1 = base + 10 * p.stride;
    int32_t *Rp = p.Rp + (long long)blockIdx.x * n;

    __shared__ long long s_tree;
    __shared__ int s_cnt, s_maxdepth;
    __shared__ unsigned long long s_draws;
    __shared__ int s_warp[BT / 32 + 1];

    unsigned long long my_draws = 0, my_rounds = 0;
    int my_max_rounds = 0, my_max_depth = 0;

    for (;;) {
        if (tid == 0) s_tree = p.t_begin + (long long)atomicAdd(p.next_tree, 1ull);
        __syncthreads();
        const long long t = s_tree;
        if (t >= p.t_end) break;
        const uint32_t tree = (uint32_t)t;

        // ---- 1. cycle popping --------------------------------------------
        for (int v = tid; v < n; v += BT) {
            pop[v] = 0;
            if (v == u) {
                nxt[v] = -1;
                tdep[v] = 0;
            } else {
                nxt[v] = stack_entry(p, v, 0u, tree);
                tdep[v] = -1;
            }
            if (v < n - 1) actA[v] = (v < u) ? v : v + 1;
        }
        if (tid == 0) {
            s_draws = (unsigned long long)(n - 1);
            s_maxdepth = 0;
            s_cnt = 0;
        }
        __syncthreads();

        int nact = n - 1, rounds = 0, tree_depth = 0;
        int32_t *act = actA, *act_next = actB;
        bool failed = false;
        while (nact > 0) {
            if (++rounds > p.max_rounds) {
                failed = true;
                if (tid == 0) atomicOr(p.status, kStatusPopRounds);
                break;
            }
            for (int i = tid; i < nact; i += BT) {
                const int v = act[i];
                J0[v] = nxt[v];
                L0[v] = v;
                D0[v] = 1;
            }
            __syncthreads();
            // Synchronous pointer jumping. Label L[v] = min vertex id on the
            // path from v up to (not including) J[v]; resolved vertices are
            // absorbing and carry label -1. When a step changes nothing, L[v]
            // is the minimum over everything reachable from v.
            int32_t *Jc = J0, *Lc = L0, *Dc = D0, *Jn = J1, *Ln = L1, *Dn = D1;
            bool converged = false;
            for (int step = 0; step < p.max_steps; ++step) {
                int changed = 0;
                for (int i = tid; i < nact; i += BT) {
                    const int v = act[i];
                    const int j = Jc[v];
                    const int lv = Lc[v];
                    const int dv = Dc[v];
                    int nj, nl, nd;
                    if (tdep[j] >= 0) {
                        nj = j;
                        nl = -1;
                        nd = dv;
                    } else {
                        nj = Jc[j];
                        nl = min(lv, Lc[j]);
                        nd = dv + Dc[j];
                    }
                    Jn[v] = nj;
                    Ln[v] = nl;
                    Dn[v] = nd;
                    changed |= (nl != lv) || (nl == -1 && tdep[nj] < 0);
                }
                int32_t *tmp;
                tmp = Jc; Jc = Jn; Jn = tmp;
                tmp = Lc; Lc = Ln; Ln = tmp;
                tmp = Dc; Dc = Dn; Dn = tmp;
                if (!__syncthreads_or(changed)) {
                    converged = true;
                    break;
                }
            }
            if (!converged) {
                failed = true;
                if (tid == 0) atomicOr(p.status, kStatusJumpSteps);
                break;
            }
            // Classify: resolve, or keep and pop the cycle whose minimum is v.
            for (int i = tid; i < nact; i += BT) {
                const int v = act[i];
                const int lv = Lc[v];
                if (lv == -1) {
                    const int d = Dc[v] + tdep[Jc[v]];
                    tdep[v] = d;
                    tree_depth = max(tree_depth, d);
                } else {
                    act_next[atomicAdd(&s_cnt, 1)] = v;
                    if (lv == v) {
                        int x = nxt[v], len = 1;
                        while (x != v && Lc[x] == v && len <= nact) {
                            x = nxt[x];
                            ++len;
                        }
                        if (x == v) {
                            int y = v;
                            do {
                                const int z = nxt[y];
                                const int k = pop[y] + 1;
                                pop[y] = k;
                                nxt[y] = stack_entry(p, y, (uint32_t)k, tree);
                                y = z;
                            } while (y != v);
                            atomicAdd(&s_draws, (unsigned long long)len);
                        }
                    }
                }
            }
            __syncthreads();
            nact = s_cnt;
            int32_t *tmp = act; act = act_next; act_next = tmp;
            __syncthreads();
            if (tid == 0) s_cnt = 0;
            __syncthreads();
        }
        if (failed) break;

        atomicMax(&s_maxdepth, tree_depth);
        my_max_depth = max(my_max_depth, tree_depth);
        if (tid == 0) {
            my_draws += s_draws;
            my_rounds += (unsigned long long)rounds;
            my_max_rounds = max(my_max_rounds, rounds);
        }

        if (p.mode == 1) {
            const long long off = (t - p.t_begin) * (long long)n;
            for (int v = tid; v < n; v += BT) {
                p.next_out[off + v] = nxt[v];
                if (p.pops_out) p.pops_out[off + v] = pop[v];
            }
            __syncthreads();
            continue;
        }
        __syncthreads();

        // ---- 2. DFS intervals ---------------------------------------------
        const int dmax = s_maxdepth;
        int32_t *lvl = J0, *fill = J1, *ord = actA;
        int32_t *sz = L0, *cur = L1, *off = D0, *pre = D1;
        for (int d = tid; d <= dmax + 1; d += BT) lvl[d] = 0;
        for (int v = tid; v < n; v += BT) {
            sz[v] = 1;
            cur[v] = 0;
        }
        __syncthreads();
        for (int v = tid; v < n; v += BT) atomicAdd(&lvl[tdep[v]], 1);
        __syncthreads();
        block_exclusive_scan<BT>(lvl, dmax + 2, s_warp);
        for (int d = tid; d <= dmax + 1; d += BT) fill[d] = lvl[d];
        __syncthreads();
        for (int v = tid; v < n; v += BT) ord[atomicAdd(&fill[tdep[v]], 1)] = v;
        __syncthreads();
        for (int d = dmax; d >= 1; --d) {
            const int s = lvl[d], e = lvl[d + 1];
            for (int i = s + tid; i < e; i += BT) {
                const int v = ord[i];
                atomicAdd(&sz[nxt[v]], sz[v]);
            }
            __syncthreads();
        }
        for (int v = tid; v < n; v += BT) {
            if (v != u) off[v] = 1 + atomicAdd(&cur[nxt[v]], sz[v]);
        }
        if (tid == 0) pre[u] = 0;
        __syncthreads();
        for (int d = 1; d <= dmax; ++d) {
            const int s = lvl[d], e = lvl[d + 1];
            for (int i = s + tid; i < e; i += BT) {
                const int v = ord[i];
                pre[v] = pre[nxt[v]] + off[v];
            }
            __syncthreads();
        }

        // ---- 3. Algorithm 2 ------------------------------------------------
        for (int v = tid; v < n; v += BT) {
            if (v == u) continue;
            const int pv = pre[v];
            int cnt = 0;
            int b = v;
            while (b != u) {
                const int a = __ldg(p.bpar + b);
                if (nxt[b] == a) {
                    const int lo = pre[b];
                    cnt += (lo <= pv && pv < lo + sz[b]) ? 1 : 0;
                } else if (nxt[a] == b) {
                    const int lo = pre[a];
                    cnt -= (lo <= pv && pv < lo + sz[a]) ? 1 : 0;
                }
                b = a;
            }
            Rp[v] += cnt;
        }
        __syncthreads();
    }

    if (tid == 0) {
        atomicAdd(p.stats + 0, my_draws);
        atomicAdd(p.stats + 1, my_rounds);
        atomicMax(p.stats + 2, (unsigned long long)my_max_rounds);
    }
    atomicMax(p.stats + 3, (unsigned long long)my_max_depth);
}

// out[v] += sum over partial rows of Rp[c][v] (exact, fixed order).
__global__ void reduce_counts_kernel(int n, int rows, const int32_t *__restrict__ Rp, long long *__restrict__ out)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        long long s = 0;
        for (int c = 0; c < rows; ++c) s += Rp[(long long)c * n + v];
        out[v] += s;
    }
}

template <int BT>
cudaError_t launch_sampler(int grid, cudaStream_t st, const SampleParams &p)
{
    sample_aggregate_kernel<BT><<<grid, BT, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace

int alloc_sampler(Ctx *c, int block_threads, int ctas_per_sm)
{
    if (block_threads != 256 && block_threads != 512 && block_threads != 1024) block_threads = 512;
    if (ctas_per_sm < 1) ctas_per_sm = (block_threads == 1024) ? 1 : 2048 / block_threads;
    c->block_threads = block_threads;
    c->ctas = c->num_sms * ctas_per_sm;
    c->ws_stride = ((int64_t)c->n + 2 + 31) / 32 * 32;
    const size_t ws_bytes = (size_t)c->ctas * kWsArrays * (size_t)c->ws_stride * sizeof(int32_t);
    const size_t rp_bytes = (size_t)c->ctas * (size_t)c->n * sizeof(int32_t);
    if (cudaMalloc(&c->d_ws, ws_bytes) != cudaSuccess) return fail(c, UST_ENOMEM, "sampler workspace");
    if (cudaMalloc(&c->d_Rp, rp_bytes) != cudaSuccess) return fail(c, UST_ENOMEM, "partial counts");
    return UST_OK;
}

int run_sampler(Ctx *c, int64_t t0, int64_t t1, uint64_t seed, int64_t *d_out, int32_t *d_next_out,
                int32_t *d_pops_out, int64_t *draws, int64_t *rounds, int *max_rounds, int *max_depth)
{
    if (t1 <= t0) return UST_OK;
    if (t0 < 0 || t1 > (int64_t)0xFFFFFFFFll) return fail(c, UST_EINVAL, "tree ids must lie in [0, 2^32)");
    const int mode = d_next_out ? 1 : 0;
    const int grid = (int)std::min<int64_t>(c->ctas, t1 - t0);
    if (mode == 0)
        UST_CUDA_TRY(cudaMemsetAsync(c->d_Rp, 0, (size_t)grid * c->n * sizeof(int32_t), c->stream));
    UST_CUDA_TRY(cudaMemsetAsync(c->d_stats, 0, 8 * sizeof(int64_t), c->stream));

    SampleParams p;
    p.n = c->n;
    p.u = c->pivot;
    p.graph = (uint32_t)c->graph_id;
    p.key0 = (uint32_t)(seed & 0xFFFFFFFFull);
    p.key1 = (uint32_t)(seed >> 32);
    p.rp = c->d_rp;
    p.ci = c->d_ci;
    p.bpar = c->d_bpar;
    p.ws = c->d_ws;
    p.stride = c->ws_stride;
    p.Rp = c->d_Rp;
    p.t_begin = t0;
    p.t_end = t1;
    unsigned long long *st = reinterpret_cast<unsigned long long *>(c->d_stats);
    p.next_tree = st + 4;
    p.stats = st;
    p.status = reinterpret_cast<int *>(st + 5);
    p.max_rounds = c->max_pop_rounds;
    int lg = 0;
    while ((1ll << lg) < (long long)c->n) ++lg;
    p.max_steps = lg + 4;
    p.mode = mode;
    p.next_out = d_next_out;
    p.pops_out = d_pops_out;

    cudaError_t e;
    phase_begin(c, Ctx::kEvSample);
    switch (c->block_threads) {
    case 256: e = launch_sampler<256>(grid, c->stream, p); break;
    case 1024: e = launch_sampler<1024>(grid, c->stream, p); break;
    default: e = launch_sampler<512>(grid, c->stream, p); break;
    }
    phase_end(c, Ctx::kEvSample);
    c->launches += 1;
    if (e != cudaSuccess) return fail(c, UST_ECUDA, std::string("sampler launch: ") + cudaGetErrorString(e));
    if (mode == 0) {
        phase_begin(c, Ctx::kEvReduce);
        const int threads = 256;
        const int blocks = (int)std::min<int64_t>((c->n + threads - 1) / threads, (int64_t)c->num_sms * 8);
        reduce_counts_kernel<<<blocks, threads, 0, c->stream>>>(c->n, grid, c->d_Rp,
                                                                 reinterpret_cast<long long *>(d_out));
        phase_end(c, Ctx::kEvReduce);
        c->launches += 1;
        UST_CUDA_TRY(cudaGetLastError());
    }
    UST_CUDA_TRY(cudaMemcpyAsync(c->h_stats, c->d_stats, 8 * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
    const int status = (int)c->h_stats[5];
    if (status & kStatusPopRounds) return fail(c, UST_ETIMEOUT, "a tree exceeded max_pop_rounds");
    if (status & kStatusJumpSteps) return fail(c, UST_ETIMEOUT, "pointer jumping did not converge");
    if (status) return fail(c, UST_ECUDA, "sampler reported an inconsistent state");
    c->last_trees = t1 - t0;
    c->last_draws = c->h_stats[0];
    if (draws) *draws = c->h_stats[0];
    if (rounds) *rounds = c->h_stats[1];
    if (max_rounds) *max_rounds = (int)c->h_stats[2];
    if (max_depth) *max_depth = (int)c->h_stats[3];
    return UST_OK;
}

}  // namespace ust
