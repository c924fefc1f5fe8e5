// Batches of graphs: ust_init_batch and the batch forms of sampling, the
// column solves and the diagonal combination (Algorithm 1 run for many
// graphs at once, each with its own pivot and trees).
//
// All graphs live one after another in the context's arrays. B_u of every
// graph comes from one launch (one CTA per graph); sampling is one persistent
// launch over (graph, tree) work items for the graphs small enough for the
// shared-memory sampler and one for the others; every graph's counts go
// straight into its slice of R (integer atomics, order-free); the columns are
// solved graph after graph; the diagonal is one launch (one CTA per graph).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ust_common.cuh"

namespace ust {


namespace {

int64_t tau_of(const Ctx *c, int g, double eps)
{
    const double m = (double)c->bnnz[g] / 2.0;
    const double delta = c->delta > 0 ? c->delta : 1.0 / (double)c->bn[g];
    const double a = log(2.0 * m / delta);
    const double b = 2.0 * (1.0 - c->kappa) * (1.0 - c->kappa) * eps * eps;
    return (int64_t)c->becc[g] * (int64_t)c->becc[g] * (int64_t)ceil(a / b);
}

GraphDesc desc_of(const Ctx *c, int g, long long tree_begin)
{
    GraphDesc d;
    d.n = c->bn[g];
    d.u = c->bpivot[g];
    d.graph = (uint32_t)(c->graph_id + g);
    d.voff = c->bvoff[g];
    d.tree_begin = tree_begin;
    d.rp = c->d_rp + c->bvoff[g] + g;
    d.ci = c->d_ci + c->baoff[g];
    d.bpar = c->d_bpar + c->bvoff[g];
    d.path = c->d_path + c->bpoff[g];
    d.pathptr = c->d_pathptr + c->bvoff[g] + g;
    d.pchild = c->d_path + c->path_cap + c->bpoff[g];
    d.powner = c->d_path + 2 * c->path_cap + c->bpoff[g];
    d.fc = (int)c->bfarness[g];
    d.aoff = c->baoff[g];
    d.orig = nullptr;
    d.rp_in = nullptr;
    d.ncore = d.n;
    return d;
}

// B_u of every graph in one launch (one CTA per graph): BFS parents, ecc(u)
// and f^c(u) into becc / h_prep_out; with `fill`, the flattened paths too
// (their space bpoff / bfarness must be in place).
int batch_prepare(Ctx *c, bool fill)
{
    const int B = c->batch;
    std::vector<PrepDesc> prep((size_t)B);
    for (int g = 0; g < B; ++g) {
        PrepDesc &d = prep[g];
        d.n = c->bn[g];
        d.u = c->bpivot[g];
        d.rp = c->d_rp + c->bvoff[g] + g;
        d.ci = c->d_ci + c->baoff[g];
        d.dist = c->d_dist + c->bvoff[g];
        d.bpar = c->d_bpar + c->bvoff[g];
        d.pathptr = c->d_pathptr + c->bvoff[g] + g;
        d.path = fill ? c->d_path + c->bpoff[g] : nullptr;
        d.pchild = fill ? c->d_path + c->path_cap + c->bpoff[g] : nullptr;
        d.powner = fill ? c->d_path + 2 * c->path_cap + c->bpoff[g] : nullptr;
        d.path_cap = fill ? c->bfarness[g] : 0;
    }
    phase_begin(c, Ctx::kEvBfs);
    UST_CUDA_TRY(cudaMemcpyAsync(c->d_prep, prep.data(), (size_t)B * sizeof(PrepDesc), cudaMemcpyHostToDevice,
                                 c->stream));
    UST_CUDA_TRY(cudaMemsetAsync(c->d_prep_out, 0, (size_t)B * 3 * sizeof(int32_t), c->stream));
    const int rc = run_batch_prepare(c, c->d_prep, B, c->d_prep_out);
    if (rc) return rc;
    UST_CUDA_TRY(cudaMemcpyAsync(c->h_prep_out, c->d_prep_out, (size_t)B * 3 * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, c->stream));
    phase_end(c, Ctx::kEvBfs);
    UST_SYNC_TRY(fill ? "batch B_u with paths" : "batch B_u");
    for (int g = 0; g < B; ++g) {
        const int st = c->h_prep_out[g];
        if (st & 1) return fail(c, UST_ENOTCONNECTED, "graph " + std::to_string(g) + " is not connected");
        if (fill && (st & 2)) return fail(c, UST_ECUDA, "batch B_u: path space mismatch");
        c->becc[g] = c->h_prep_out[B + g];
    }
    return UST_OK;
}

// The tuned launch shape of every size class (ust_opts.autotune): each class
// is probed with the same number of trees of each of its graphs, about
// 2,432 work items in all, counts into the scratch row of R.
int tune_batch_classes(Ctx *c, const std::vector<int32_t> &hrp)
{
    const int B = c->batch;
    for (int k = 0; k < kNumClasses; ++k) {
        std::vector<int> group;
        for (int g = 0; g < B; ++g)
            if (c->bclass[g] == k) group.push_back(g);
        if (group.empty()) continue;
        const int G = (int)group.size();
        const long long target = 2ll * c->num_sms * 8;
        const long long t = std::max<long long>(1, (target + G - 1) / G);
        std::vector<GraphDesc> descs;
        std::vector<long long> starts;
        long long nsum = 0, asum = 0, max_rounds = 1024;
        int pdeg = 1, maxn = 0;
        for (int i = 0; i < G; ++i) {
            const int g = group[i];
            descs.push_back(desc_of(c, g, 0));
            starts.push_back(t * i);
            nsum += c->bn[g];
            asum += c->bnnz[g];
            maxn = std::max(maxn, c->bn[g]);
            const int32_t *r = hrp.data() + c->bvoff[g] + g;
            pdeg = std::max(pdeg, r[c->bpivot[g] + 1] - r[c->bpivot[g]]);
            max_rounds = std::max<long long>(max_rounds,
                                             16ll * ((long long)c->bnnz[g] * std::max(1, c->becc[g]) + c->bn[g]) + 1024);
        }
        if (c->max_pop_rounds > 0) max_rounds = c->max_pop_rounds;
        starts.push_back(t * G);
        UST_CUDA_TRY(cudaMemcpyAsync(c->d_graphs, descs.data(), descs.size() * sizeof(GraphDesc),
                                     cudaMemcpyHostToDevice, c->stream));
        UST_CUDA_TRY(cudaMemcpyAsync(c->d_items, starts.data(), starts.size() * sizeof(long long),
                                     cudaMemcpyHostToDevice, c->stream));
        TuneKey key;
        key.kernel = maxn <= kSmemMaxVertices ? 0 : maxn <= kTierMaxVertices ? 1 : 2;
        key.n_bucket = k;  // the class itself
        key.avg_deg = (int)(asum / std::max<long long>(1, nsum));
        int l = 0;
        while ((1 << l) < pdeg) ++l;
        key.pivot_deg_log2 = l;
        l = 0;
        while ((1 << l) < G) ++l;
        key.graphs_log2 = l;
        key.sms = c->num_sms;
        const int rc = tune_launch(c, key, c->d_graphs, c->d_items, G, t * G, maxn, max_rounds, c->d_Rtmp,
                                   &c->class_tuned[k], nullptr);
        if (rc) return rc;
    }
    return UST_OK;
}

// Samples count[g] trees of every graph g (ids continue from btrees[g]) and
// commits them to R, or leaves R unchanged on error.
int batch_sample(Ctx *c, const std::vector<int64_t> &count, uint64_t seed)
{
    const int B = c->batch;
    std::vector<GraphDesc> descs;
    std::vector<long long> starts;
    long long total[kNumClasses] = {};
    int ngr[kNumClasses] = {}, maxn[kNumClasses] = {};
    long long max_rounds = 1024;
    std::vector<int> group[kNumClasses];
    for (int g = 0; g < B; ++g) {
        if (count[g] <= 0) continue;
        if (c->btrees[g] + count[g] > (int64_t)0xFFFFFFFFll) return fail(c, UST_EINVAL, "tree ids must stay below 2^32");
        group[c->bclass[g]].push_back(g);
        max_rounds = std::max<long long>(max_rounds,
                                         16ll * ((long long)c->bnnz[g] * std::max(1, c->becc[g]) + c->bn[g]) + 1024);
    }
    if (c->max_pop_rounds > 0) max_rounds = c->max_pop_rounds;
    // descriptors class after class; item starts likewise (|class| + 1 each)
    int desc_at[kNumClasses] = {}, start_at[kNumClasses] = {};
    for (int k = 0; k < kNumClasses; ++k) {
        desc_at[k] = (int)descs.size();
        start_at[k] = (int)starts.size();
        long long acc = 0;
        for (int g : group[k]) {
            descs.push_back(desc_of(c, g, c->btrees[g]));
            starts.push_back(acc);
            acc += count[g];
            maxn[k] = std::max(maxn[k], c->bn[g]);
        }
        starts.push_back(acc);
        total[k] = acc;
        ngr[k] = (int)group[k].size();
    }
    if (descs.empty()) return UST_OK;
    UST_CUDA_TRY(cudaMemcpyAsync(c->d_graphs, descs.data(), descs.size() * sizeof(GraphDesc), cudaMemcpyHostToDevice,
                                 c->stream));
    UST_CUDA_TRY(cudaMemcpyAsync(c->d_items, starts.data(), starts.size() * sizeof(long long), cudaMemcpyHostToDevice,
                                 c->stream));
    UST_CUDA_TRY(cudaMemcpyAsync(c->d_Rtmp, c->d_R, (size_t)c->n * 8, cudaMemcpyDeviceToDevice, c->stream));
    if (c->d_ecount)
        UST_CUDA_TRY(cudaMemcpyAsync(c->d_ecount_tmp, c->d_ecount, (size_t)c->nnz * 8, cudaMemcpyDeviceToDevice,
                                     c->stream));
    int64_t draws_total = 0, rounds_total = 0;
    phase_open(c, Ctx::kEvSample);  // both launches in one timed phase
    for (int k = 0; k < kNumClasses; ++k) {
        if (total[k] == 0) continue;
        const GraphDesc *dg = c->d_graphs + desc_at[k];
        const long long *di = c->d_items + start_at[k];
        int64_t draws = 0, rounds = 0;
        int mr = 0, mp = 0;
        const int rc = run_batch_sampler(c, c->class_cfg[k], dg, di, ngr[k], total[k], maxn[k], max_rounds, seed,
                                         c->d_Rtmp, &draws, &rounds, &mr, &mp);
        if (rc) {
            c->ev_hold[Ctx::kEvSample] = false;
            return rc;
        }
        draws_total += draws;
        rounds_total += rounds;
        c->max_rounds_seen = std::max(c->max_rounds_seen, mr);
        c->max_depth_seen = std::max(c->max_depth_seen, mp);
    }
    phase_close(c, Ctx::kEvSample);
    std::swap(c->d_R, c->d_Rtmp);
    std::swap(c->d_ecount, c->d_ecount_tmp);
    int64_t trees = 0;
    for (int g = 0; g < B; ++g) {
        if (count[g] > 0) c->btrees[g] += count[g];
        trees += count[g] > 0 ? count[g] : 0;
    }
    c->trees += trees;
    c->last_trees = trees;
    c->last_draws = draws_total;
    c->seed = seed;
    c->draws += draws_total;
    c->pop_rounds += rounds_total;
    return UST_OK;
}

int batch_solve(Ctx *c)
{
    // every graph's column in one launch, one CTA per graph
    const int B = c->batch;
    if (c->solve_fp64 && !c->d_bw64) {
        if (cudaMalloc(&c->d_bw64, 5 * (size_t)c->n * sizeof(double)) != cudaSuccess)
            return fail(c, UST_ENOMEM, "FP64 solver vectors");
    }
    std::vector<SolveTask> tasks((size_t)B);
    for (int g = 0; g < B; ++g) {
        SolveTask &t = tasks[g];
        t.n = c->bn[g];
        t.u = c->bpivot[g];
        t.rp = c->d_rp + c->bvoff[g] + g;
        t.ci = c->d_ci + c->baoff[g];
        t.heavy = c->d_heavy + c->bhoff[g];
        t.n_heavy = c->bheavy_n[g];
        t.x = c->d_x + c->bvoff[g];
        t.r64 = c->d_br64 + c->bvoff[g];
        t.w = c->solve_fp64 ? (void *)(c->d_bw64 + 5 * c->bvoff[g]) : (void *)(c->d_bw32 + 5 * c->bvoff[g]);
    }
    UST_CUDA_TRY(cudaMemcpyAsync(c->d_tasks, tasks.data(), (size_t)B * sizeof(SolveTask), cudaMemcpyHostToDevice,
                                 c->stream));
    const int rc = run_solve_cta(c, c->d_tasks, B, c->d_results, c->h_results, c->solve_fp64);
    if (rc) return rc;
    c->x_valid = true;
    return UST_OK;
}

}  // namespace

int batch_init(Ctx *c, const ust_csr *gs, const int32_t *pivots, int32_t count, const ust_opts &op)
{
    const int B = count;
    c->batch = B;
    c->bn.resize(B);
    c->bnnz.resize(B);
    c->bpivot.resize(B);
    c->becc.assign(B, 0);
    c->bvoff.assign(B + 1, 0);
    c->baoff.assign(B + 1, 0);
    c->btrees.assign(B, 0);
    for (int g = 0; g < B; ++g) {
        if (!gs[g].row_ptr || !gs[g].col_idx || gs[g].n < 2 || gs[g].nnz < 2 || pivots[g] < 0 ||
            pivots[g] >= gs[g].n)
            return fail(c, UST_EINVAL, "invalid graph or pivot in the batch (need n >= 2, nnz >= 2, 0 <= pivot < n)");
        c->bn[g] = gs[g].n;
        c->bnnz[g] = gs[g].nnz;
        c->bpivot[g] = pivots[g];
        c->bvoff[g + 1] = c->bvoff[g] + gs[g].n;
        c->baoff[g + 1] = c->baoff[g] + gs[g].nnz;
    }
    if (c->bvoff[B] > 0x7FFFFFF0ll || c->baoff[B] > 0x7FFFFFF0ll)
        return fail(c, UST_EINVAL, "batch too large for 32-bit indices");
    c->n = (int)c->bvoff[B];
    c->nnz = (int)c->baoff[B];
    c->pivot = pivots[0];
    c->bclass.assign(B, 0);
    for (int k = 0; k < kNumClasses; ++k) c->class_maxn[k] = 0;
    for (int g = 0; g < B; ++g) {
        int k = 0;
        while (c->bn[g] > kClassMaxN[k]) ++k;
        c->bclass[g] = k;
        c->class_maxn[k] = std::max(c->class_maxn[k], c->bn[g]);
    }

    // host copies of the row pointers (validation, heavy rows)
    // host copies of the row pointers (heavy rows, the path space); the
    // input checks run on the device copies below
    std::vector<int32_t> hrp((size_t)c->n + B);
    for (int g = 0; g < B; ++g) {
        int32_t *dst = hrp.data() + c->bvoff[g] + g;
        const size_t rb = ((size_t)gs[g].n + 1) * 4;
        if (gs[g].on_device)
            UST_CUDA_TRY(cudaMemcpy(dst, gs[g].row_ptr, rb, cudaMemcpyDeviceToHost));
        else
            memcpy(dst, gs[g].row_ptr, rb);
    }
    const size_t nv = (size_t)c->n, na = (size_t)c->nnz;
    if (cudaMalloc(&c->d_rp, (nv + B) * 4) != cudaSuccess) return fail(c, UST_ENOMEM, "row_ptr");
    if (cudaMalloc(&c->d_ci, na * 4) != cudaSuccess) return fail(c, UST_ENOMEM, "col_idx");
    if (cudaMalloc(&c->d_bpar, nv * 4) != cudaSuccess) return fail(c, UST_ENOMEM, "bfs parent");
    if (cudaMalloc(&c->d_dist, nv * 4) != cudaSuccess) return fail(c, UST_ENOMEM, "bfs dist");
    if (cudaMalloc(&c->d_pathptr, (nv + B) * 4) != cudaSuccess) return fail(c, UST_ENOMEM, "paths");
    if (cudaMalloc(&c->d_flag, 64) != cudaSuccess) return fail(c, UST_ENOMEM, "flag");
    if (cudaMalloc(&c->d_stats, 32 * sizeof(int64_t)) != cudaSuccess) return fail(c, UST_ENOMEM, "stats");
    if (cudaMallocHost(&c->h_stats, 32 * sizeof(int64_t)) != cudaSuccess) return fail(c, UST_ENOMEM, "pinned stats");
    if (cudaMalloc(&c->d_R, nv * 8) != cudaSuccess) return fail(c, UST_ENOMEM, "counts");
    if (cudaMalloc(&c->d_Rtmp, nv * 8) != cudaSuccess) return fail(c, UST_ENOMEM, "counts");
    if (cudaMalloc(&c->d_graphs, (size_t)B * sizeof(GraphDesc)) != cudaSuccess) return fail(c, UST_ENOMEM, "graphs");
    if (cudaMalloc(&c->d_items, ((size_t)B + kNumClasses) * sizeof(long long)) != cudaSuccess)
        return fail(c, UST_ENOMEM, "items");
    if (cudaMalloc(&c->d_comb, (size_t)B * sizeof(CombineDesc)) != cudaSuccess) return fail(c, UST_ENOMEM, "combine");
    UST_CUDA_TRY(cudaMemcpyAsync(c->d_rp, hrp.data(), hrp.size() * 4, cudaMemcpyHostToDevice, c->stream));
    for (int g = 0; g < B; ++g) {
        const cudaMemcpyKind kind = gs[g].on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        UST_CUDA_TRY(cudaMemcpyAsync(c->d_ci + c->baoff[g], gs[g].col_idx, (size_t)gs[g].nnz * 4, kind, c->stream));
    }
    UST_CUDA_TRY(cudaMemsetAsync(c->d_R, 0, nv * 8, c->stream));
    if (!op.skip_validation) {
        for (int g = 0; g < B; ++g) {
            const int rc = check_graph(c, c->bn[g], c->bnnz[g], c->d_rp + c->bvoff[g] + g, c->d_ci + c->baoff[g],
                                       c->d_flag);
            if (rc) {
                c->err = "graph " + std::to_string(g) + ": " + c->err;
                return rc;
            }
        }
    }

    // B_u of every graph: a first pass measures f^c(u) (no path space yet),
    // the second fills the paths
    if (cudaMalloc(&c->d_prep, (size_t)B * sizeof(PrepDesc)) != cudaSuccess)
        return fail(c, UST_ENOMEM, "prepare descriptors");
    if (cudaMalloc(&c->d_prep_out, (size_t)B * 3 * sizeof(int32_t)) != cudaSuccess)
        return fail(c, UST_ENOMEM, "prepare outputs");
    if (cudaMallocHost(&c->h_prep_out, (size_t)B * 3 * sizeof(int32_t)) != cudaSuccess)
        return fail(c, UST_ENOMEM, "pinned prepare outputs");
    c->bfarness.assign(B, 0);
    c->bpoff.assign(B + 1, 0);
    int rc = batch_prepare(c, false);
    if (rc) return rc;
    for (int g = 0; g < B; ++g) {
        c->bfarness[g] = c->h_prep_out[2 * B + g];
        c->bpoff[g + 1] = c->bpoff[g] + c->bfarness[g];
    }
    if (cudaMalloc(&c->d_path, 3 * (size_t)std::max<int64_t>(1, c->bpoff[B]) * 4) != cudaSuccess)
        return fail(c, UST_ENOMEM, "BFS paths");
    c->path_cap = c->bpoff[B];
    rc = batch_prepare(c, true);
    if (rc) return rc;
    c->ecc = *std::max_element(c->becc.begin(), c->becc.end());
    c->farness = c->bpoff[B];

    if (op.autotune > 0 && op.block_threads == 0 && op.ctas_per_sm == 0) {
        rc = tune_batch_classes(c, hrp);
        if (rc) return rc;
    }
    rc = alloc_batch_sampler(c, op.block_threads, op.ctas_per_sm);
    if (rc) return rc;

    // solver: heavy rows per graph, the columns, and the one-CTA solve's
    // scratch for every graph at once
    c->bheavy_n.assign(B, 0);
    c->bhoff.assign(B + 1, 0);
    std::vector<int32_t> heavy;
    for (int g = 0; g < B; ++g) {
        const int32_t *r = hrp.data() + c->bvoff[g] + g;
        for (int v = 0; v < c->bn[g]; ++v)
            if (r[v + 1] - r[v] > kHeavyRow) heavy.push_back(v);
        c->bhoff[g + 1] = (int64_t)heavy.size();
        c->bheavy_n[g] = (int)(c->bhoff[g + 1] - c->bhoff[g]);
    }
    if (cudaMalloc(&c->d_heavy, std::max<size_t>(1, heavy.size()) * 4) != cudaSuccess)
        return fail(c, UST_ENOMEM, "heavy rows");
    if (!heavy.empty())
        UST_CUDA_TRY(cudaMemcpyAsync(c->d_heavy, heavy.data(), heavy.size() * 4, cudaMemcpyHostToDevice, c->stream));
    if (cudaMalloc(&c->d_x, nv * sizeof(double)) != cudaSuccess) return fail(c, UST_ENOMEM, "columns");
    if (cudaMalloc(&c->d_br64, nv * sizeof(double)) != cudaSuccess) return fail(c, UST_ENOMEM, "solver residuals");
    if (cudaMalloc(&c->d_bw32, 5 * nv * sizeof(float)) != cudaSuccess) return fail(c, UST_ENOMEM, "solver vectors");
    if (cudaMalloc(&c->d_tasks, (size_t)B * sizeof(SolveTask)) != cudaSuccess) return fail(c, UST_ENOMEM, "tasks");
    if (cudaMalloc(&c->d_results, (size_t)B * sizeof(SolveResult)) != cudaSuccess)
        return fail(c, UST_ENOMEM, "solve results");
    if (cudaMallocHost(&c->h_results, (size_t)B * sizeof(SolveResult)) != cudaSuccess)
        return fail(c, UST_ENOMEM, "pinned solve results");
    UST_SYNC_TRY("batch set-up");
    return UST_OK;
}

int batch_reset(Ctx *c)
{
    c->trees = 0;
    c->draws = 0;
    c->pop_rounds = 0;
    c->max_rounds_seen = 0;
    c->max_depth_seen = 0;
    c->x_valid = false;
    std::fill(c->btrees.begin(), c->btrees.end(), 0);
    UST_CUDA_TRY(cudaMemsetAsync(c->d_R, 0, (size_t)c->n * 8, c->stream));
    if (c->d_ecount) UST_CUDA_TRY(cudaMemsetAsync(c->d_ecount, 0, (size_t)c->nnz * 8, c->stream));
    return batch_prepare(c, true);
}

int batch_sample_aggregate(Ctx *c, int64_t n_trees, uint64_t seed)
{
    std::vector<int64_t> count((size_t)c->batch, n_trees);
    return batch_sample(c, count, seed);
}

int64_t batch_tau(const Ctx *c, double eps)
{
    int64_t t = 0;
    for (int g = 0; g < c->batch; ++g) t = std::max(t, tau_of(c, g, eps));
    return t;
}

int batch_diag(Ctx *c, double eps, double *diag_out, int32_t out_on_device)
{
    if (eps > 0) {
        std::vector<int64_t> count((size_t)c->batch, 0);
        bool any = false;
        for (int g = 0; g < c->batch; ++g) {
            count[g] = std::max<int64_t>(0, tau_of(c, g, eps) - c->btrees[g]);
            any |= count[g] > 0;
        }
        if (any) {
            const int rc = batch_sample(c, count, c->seed);
            if (rc) return rc;
        }
    }
    for (int g = 0; g < c->batch; ++g)
        if (c->btrees[g] <= 0) return fail(c, UST_ESTATE, "a graph of the batch has no trees");
    if (!c->x_valid) {
        const int rc = batch_solve(c);
        if (rc) return rc;
    }
    std::vector<CombineDesc> cd((size_t)c->batch);
    for (int g = 0; g < c->batch; ++g) {
        cd[g].n = c->bn[g];
        cd[g].u = c->bpivot[g];
        cd[g].voff = c->bvoff[g];
        cd[g].trees = c->btrees[g];
    }
    UST_CUDA_TRY(cudaMemcpyAsync(c->d_comb, cd.data(), cd.size() * sizeof(CombineDesc), cudaMemcpyHostToDevice,
                                 c->stream));
    double *dst = diag_out;
    double *tmp = nullptr;
    if (!out_on_device) {
        if (cudaMalloc(&tmp, (size_t)c->n * sizeof(double)) != cudaSuccess) return fail(c, UST_ENOMEM, "diag");
        dst = tmp;
    }
    int rc = run_batch_combine(c, c->d_comb, c->batch, dst);
    if (!rc && !out_on_device) {
        if (cudaMemcpyAsync(diag_out, tmp, (size_t)c->n * sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            rc = fail(c, UST_ECUDA, "diag readback");
    }
    cudaFree(tmp);
    return rc;
}

int batch_column(Ctx *c)
{
    return c->x_valid ? UST_OK : batch_solve(c);
}

}  // namespace ust
