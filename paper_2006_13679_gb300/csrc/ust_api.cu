// C ABI entry points of libust.so (declared in include/ust.h).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "ust_common.cuh"

namespace ust {

int fail(Ctx *c, int code, const std::string &msg)
{
    c->err = msg;
    return code;
}

}  // namespace ust

using ust::Ctx;

namespace {

thread_local std::string g_init_error = "no error";

void release(Ctx *c)
{
    cudaFree(c->d_rp);
    cudaFree(c->d_ci);
    cudaFree(c->d_bpar);
    cudaFree(c->d_dist);
    cudaFree(c->d_flag);
    cudaFree(c->d_pathptr);
    cudaFree(c->d_path);
    cudaFree(c->d_wrp);
    cudaFree(c->d_wci);
    cudaFree(c->d_wmap);
    cudaFree(c->d_bscratch);
    cudaFree(c->d_srp);
    cudaFree(c->d_sci);
    cudaFree(c->d_orig);
    cudaFree(c->d_newid);
    cudaFree(c->d_spathptr);
    cudaFree(c->d_spath);
    cudaFree(c->d_ws);
    cudaFree(c->d_Rp);
    cudaFree(c->d_R);
    cudaFree(c->d_Rtmp);
    cudaFree(c->d_stats);
    cudaFree(c->d_f32);
    cudaFree(c->d_f64);
    cudaFree(c->d_red);
    cudaFree(c->d_x);
    cudaFree(c->d_f64inner);
    cudaFree(c->d_heavy);
    cudaFree(c->d_graphs);
    cudaFree(c->d_items);
    cudaFree(c->d_comb);
    cudaFree(c->d_prep);
    cudaFree(c->d_tasks);
    cudaFree(c->d_ecount);
    cudaFree(c->d_ecount_tmp);
    cudaFree(c->d_results);
    cudaFreeHost(c->h_results);
    cudaFree(c->d_bw32);
    cudaFree(c->d_bw64);
    cudaFree(c->d_br64);
    cudaFree(c->d_prep_out);
    cudaFreeHost(c->h_prep_out);
    for (int i = 0; i < 2 * Ctx::kEvPhases; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    if (c->h_stats) cudaFreeHost(c->h_stats);
    if (c->h_red) cudaFreeHost(c->h_red);
}

}  // namespace

namespace ust {

// Batch contexts (ust_batch.cu). The CSR contract (row_ptr monotone from 0
// to nnz, columns in range and strictly increasing per row, no self-loops,
// every arc present in both directions, no isolated vertex) is checked on the
// device by check_graph, for single graphs and for every graph of a batch.
int batch_init(Ctx *c, const ust_csr *gs, const int32_t *pivots, int32_t count, const ust_opts &op);
int batch_sample_aggregate(Ctx *c, int64_t n_trees, uint64_t seed);
int64_t batch_tau(const Ctx *c, double eps);
int batch_diag(Ctx *c, double eps, double *diag_out, int32_t out_on_device);
int batch_column(Ctx *c);
int batch_reset(Ctx *c);

}  // namespace ust

namespace {

// Context options shared by single graphs and batches.
int apply_opts(Ctx *c, const ust_opts &op, int n)
{
    c->delta = op.delta > 0 ? op.delta : 1.0 / (double)n;
    c->kappa = op.kappa > 0 ? op.kappa : 0.3;
    c->cg_tol = op.cg_tol > 0 ? op.cg_tol : 1e-9;
    c->max_pop_rounds = op.max_pop_rounds;
    c->max_cg_iters = op.max_cg_iters > 0 ? op.max_cg_iters : 20000;
    c->graph_id = op.graph_id;
    c->solve_fp64 = op.solve_fp64 != 0;
    c->stream = reinterpret_cast<cudaStream_t>(op.stream);
    UST_CUDA_TRY(cudaGetDevice(&c->device));
    for (int i = 0; i < 2 * Ctx::kEvPhases; ++i) UST_CUDA_TRY(cudaEventCreate(&c->ev[i]));
    UST_CUDA_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    return UST_OK;
}

int ilog2_ceil(long long x)
{
    int l = 0;
    while ((1ll << l) < x) ++l;
    return l;
}

// The tuned launch shape of a single graph (ust_opts.autotune = 1): probes of
// 2 x (most CTAs of any candidate) trees, at most 2,432.
int tune_single(Ctx *c, int *bt, int *cps)
{
    int32_t rp2[2] = {0, 0};
    UST_CUDA_TRY(cudaMemcpyAsync(rp2, c->d_rp + c->pivot, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
    ust::TuneKey key;
    key.kernel = c->n <= ust::kSmemMaxVertices ? 0 : c->n <= ust::kTierMaxVertices ? 1 : 2;
    key.n_bucket = (c->n + 4095) / 4096;
    key.avg_deg = (int)((int64_t)c->nnz / c->n);
    key.pivot_deg_log2 = ilog2_ceil(std::max(1, rp2[1] - rp2[0]));
    key.graphs_log2 = 0;
    key.sms = c->num_sms;
    int rc = ust::upload_single_desc(c, true);
    if (rc) return rc;
    const long long max_rounds =
        c->max_pop_rounds > 0 ? c->max_pop_rounds
                              : std::min<int64_t>(16ll * ((int64_t)c->nnz * std::max(1, c->ecc) + c->n) + 1024, 1ll << 30);
    const long long items = 2ll * c->num_sms * 8;
    ust::LaunchCfg best;
    rc = ust::tune_launch(c, key, c->d_graphs, c->d_items, 1, items, c->n, max_rounds, c->d_Rtmp, &best, nullptr);
    if (rc) return rc;
    *bt = best.bt;
    *cps = best.ctas / std::max(1, c->num_sms);
    return UST_OK;
}

int init_impl(Ctx *c, const ust_csr *g, int32_t pivot, const ust_opts *o)
{
    const int n = g->n, nnz = g->nnz;
    c->n = n;
    c->nnz = nnz;
    c->pivot = pivot;
    ust_opts def;
    ust_default_opts(&def);
    const ust_opts &op = o ? *o : def;
    const int orc = apply_opts(c, op, n);
    if (orc) return orc;

    if (cudaMalloc(&c->d_rp, ((size_t)n + 1) * 4) != cudaSuccess) return ust::fail(c, UST_ENOMEM, "row_ptr");
    if (cudaMalloc(&c->d_ci, (size_t)nnz * 4) != cudaSuccess) return ust::fail(c, UST_ENOMEM, "col_idx");
    const cudaMemcpyKind kind = g->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    UST_CUDA_TRY(cudaMemcpyAsync(c->d_rp, g->row_ptr, ((size_t)n + 1) * 4, kind, c->stream));
    UST_CUDA_TRY(cudaMemcpyAsync(c->d_ci, g->col_idx, (size_t)nnz * 4, kind, c->stream));
    if (cudaMalloc(&c->d_bpar, (size_t)n * 4) != cudaSuccess) return ust::fail(c, UST_ENOMEM, "bfs parent");
    if (cudaMalloc(&c->d_dist, (size_t)n * 4) != cudaSuccess) return ust::fail(c, UST_ENOMEM, "bfs dist");
    if (cudaMalloc(&c->d_flag, 64) != cudaSuccess) return ust::fail(c, UST_ENOMEM, "flag");
    if (cudaMalloc(&c->d_pathptr, ((size_t)n + 1) * 4) != cudaSuccess) return ust::fail(c, UST_ENOMEM, "paths");
    if (cudaMalloc(&c->d_stats, 32 * sizeof(int64_t)) != cudaSuccess) return ust::fail(c, UST_ENOMEM, "stats");
    if (cudaMallocHost(&c->h_stats, 32 * sizeof(int64_t)) != cudaSuccess)
        return ust::fail(c, UST_ENOMEM, "pinned stats");
    if (cudaMalloc(&c->d_graphs, sizeof(ust::GraphDesc)) != cudaSuccess) return ust::fail(c, UST_ENOMEM, "descriptor");
    if (cudaMalloc(&c->d_items, 2 * sizeof(long long)) != cudaSuccess) return ust::fail(c, UST_ENOMEM, "items");
    if (cudaMalloc(&c->d_R, (size_t)n * 8) != cudaSuccess) return ust::fail(c, UST_ENOMEM, "counts");
    if (cudaMalloc(&c->d_Rtmp, (size_t)n * 8) != cudaSuccess) return ust::fail(c, UST_ENOMEM, "counts");
    UST_CUDA_TRY(cudaMemsetAsync(c->d_R, 0, (size_t)n * 8, c->stream));

    // the input checks run on the device copy (the BFS then finds any vertex
    // that is not connected to the pivot)
    if (!op.skip_validation) {
        const int rc = ust::check_graph(c, n, nnz, c->d_rp, c->d_ci, c->d_flag);
        if (rc) return rc;
    }
    int rc = ust::run_bfs(c);
    if (rc) return rc;
    if (op.wilson_blocks) {
        c->blocks = true;
        rc = ust::build_block_rows(c);
        if (rc) return rc;
    } else {  // the samplers' view: Cuthill-McKee order, pendant vertices last
        rc = ust::build_relabel(c);
        if (rc) return rc;
        rc = ust::relabel_paths(c);
        if (rc) return rc;
    }
    int bt = op.block_threads, cps = op.ctas_per_sm;
    if (op.autotune > 0 && bt == 0 && cps == 0 && !c->blocks) {
        rc = tune_single(c, &bt, &cps);
        if (rc) return rc;
    }
    rc = ust::alloc_sampler(c, bt, cps);
    if (rc) return rc;
    rc = ust::alloc_solver(c);
    if (rc) return rc;
    UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->ready = true;
    return UST_OK;
}

// Sampling calls need B_u, the sampler's paths and walk rows of the current
// pivot: after a ust_reset that failed part-way they may not match.
int check_ready(Ctx *c)
{
    if (c->batch || c->ready) return UST_OK;
    return ust::fail(c, UST_ESTATE, "the last ust_reset failed: call ust_reset again before sampling");
}

// The sampler draws from the context's CSR pointers. With the
// biconnected-component variant they name the walk rows (each vertex's
// neighbours in its parent block) for the length of one sampler call; B_u,
// the checks and the solve keep using the input graph.
struct SamplingRows {
    Ctx *c;
    int32_t *rp, *ci;
    explicit SamplingRows(Ctx *ctx) : c(ctx), rp(ctx->d_rp), ci(ctx->d_ci)
    {
        if (c->blocks) {
            c->d_rp = c->d_wrp;
            c->d_ci = c->d_wci;
        }
    }
    ~SamplingRows()
    {
        c->d_rp = rp;
        c->d_ci = ci;
    }
    SamplingRows(const SamplingRows &) = delete;
    SamplingRows &operator=(const SamplingRows &) = delete;
};

int copy_out(Ctx *c, void *dst, const void *src, size_t bytes, int32_t on_device)
{
    if (!dst) return ust::fail(c, UST_EINVAL, "null output pointer");
    UST_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 c->stream));
    if (!on_device) UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return UST_OK;
}

}  // namespace

extern "C" {

void ust_default_opts(ust_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->kappa = 0.3;
    o->cg_tol = 1e-9;
}

int ust_init(const ust_csr *g, int32_t pivot, const ust_opts *o, ust_ctx **out)
{
    if (!out) return UST_EINVAL;
    *out = nullptr;
    if (!g || !g->row_ptr || !g->col_idx || g->n < 2 || g->nnz < 2 || pivot < 0 || pivot >= g->n) {
        g_init_error = "invalid graph or pivot (need n >= 2, nnz >= 2, 0 <= pivot < n)";
        return UST_EINVAL;
    }
    ust_ctx *h = new (std::nothrow) ust_ctx;
    if (!h) return UST_ENOMEM;
    const int rc = init_impl(&h->c, g, pivot, o);
    if (rc) {
        g_init_error = h->c.err;
        release(&h->c);
        delete h;
        return rc;
    }
    *out = h;
    return UST_OK;
}

int ust_init_batch(const ust_csr *gs, const int32_t *pivots, int32_t count, const ust_opts *o, ust_ctx **out)
{
    if (!out) return UST_EINVAL;
    *out = nullptr;
    if (!gs || !pivots || count < 1) {
        g_init_error = "invalid batch (need count >= 1 graphs and pivots)";
        return UST_EINVAL;
    }
    if (o && o->wilson_blocks) {
        g_init_error = "wilson_blocks applies to single-graph contexts";
        return UST_EINVAL;
    }
    ust_ctx *h = new (std::nothrow) ust_ctx;
    if (!h) return UST_ENOMEM;
    ust_opts def;
    ust_default_opts(&def);
    const ust_opts &op = o ? *o : def;
    int rc = apply_opts(&h->c, op, gs[0].n > 0 ? gs[0].n : 2);
    if (!rc) {
        rc = ust::batch_init(&h->c, gs, pivots, count, op);
        if (op.delta <= 0) h->c.delta = 0;  // per graph: 1 / n_g
    }
    if (rc) {
        g_init_error = h->c.err;
        release(&h->c);
        delete h;
        return rc;
    }
    *out = h;
    return UST_OK;
}

int ust_select_pivot(const ust_csr *g, int32_t sweeps, int32_t start, void *stream, int32_t *pivot_out,
                     int32_t *bound_out)
{
    if (!g || !g->row_ptr || !g->col_idx || g->n < 2 || g->nnz < 2 || !pivot_out || start >= g->n) {
        g_init_error = "invalid graph, start vertex or output (need n >= 2, nnz >= 2, start < n)";
        return UST_EINVAL;
    }
    Ctx c;
    c.n = g->n;
    c.nnz = g->nnz;
    c.stream = reinterpret_cast<cudaStream_t>(stream);
    int rc = UST_OK;
    int32_t *rp = const_cast<int32_t *>(g->row_ptr), *ci = const_cast<int32_t *>(g->col_idx);
    int32_t *own_rp = nullptr, *own_ci = nullptr, pivot = -1, bound = 0;
    int *d_bad = nullptr;
    if (cudaGetDevice(&c.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess ||
        cudaMalloc(&d_bad, sizeof(int)) != cudaSuccess) {
        rc = ust::fail(&c, UST_ECUDA, "device set-up");
    }
    if (!rc && !g->on_device) {
        if (cudaMalloc(&own_rp, ((size_t)g->n + 1) * 4) != cudaSuccess ||
            cudaMalloc(&own_ci, (size_t)g->nnz * 4) != cudaSuccess ||
            cudaMemcpyAsync(own_rp, g->row_ptr, ((size_t)g->n + 1) * 4, cudaMemcpyHostToDevice, c.stream) != cudaSuccess ||
            cudaMemcpyAsync(own_ci, g->col_idx, (size_t)g->nnz * 4, cudaMemcpyHostToDevice, c.stream) != cudaSuccess)
            rc = ust::fail(&c, UST_ENOMEM, "device copy of the graph");
        rp = own_rp;
        ci = own_ci;
    }
    if (!rc) rc = ust::check_graph(&c, g->n, g->nnz, rp, ci, d_bad);
    if (!rc) rc = ust::select_pivot(&c, g->n, rp, ci, sweeps > 0 ? sweeps : 10, start, &pivot, &bound);
    cudaFree(own_rp);
    cudaFree(own_ci);
    cudaFree(d_bad);
    if (rc) {
        g_init_error = c.err;
        return rc;
    }
    *pivot_out = pivot;
    if (bound_out) *bound_out = bound;
    return UST_OK;
}

int32_t ust_batch_size(const ust_ctx *h)
{
    return h ? h->c.batch : 0;
}

int ust_batch_offsets(const ust_ctx *h, int64_t *offsets_out)
{
    if (!h || !offsets_out || h->c.batch == 0) return UST_EINVAL;
    for (int g = 0; g <= h->c.batch; ++g) offsets_out[g] = h->c.bvoff[g];
    return UST_OK;
}

int ust_batch_graph_info(const ust_ctx *h, int32_t g, ust_info *out)
{
    if (!h || !out || g < 0 || g >= h->c.batch) return UST_EINVAL;
    const Ctx *c = &h->c;
    memset(out, 0, sizeof(*out));
    out->n = c->bn[g];
    out->nnz = c->bnnz[g];
    out->pivot = c->bpivot[g];
    out->ecc = c->becc[g];
    out->trees = c->btrees[g];
    out->seed = c->seed;
    out->farness = c->bfarness[g];
    out->sample_ctas = c->class_cfg[c->bclass[g]].ctas;
    out->sample_threads = c->class_cfg[c->bclass[g]].bt;
    return UST_OK;
}

int ust_reset(ust_ctx *h, int32_t pivot)
{
    if (!h) return UST_EINVAL;
    Ctx *c = &h->c;
    if (c->batch) {
        if (pivot != -1) return ust::fail(c, UST_EINVAL, "a batch keeps its pivots: pass pivot = -1");
        return ust::batch_reset(c);
    }
    if (pivot < 0 || pivot >= c->n) return ust::fail(c, UST_EINVAL, "pivot out of range");
    c->ready = false;  // set again only once B_u, the paths and the walk rows all match the new pivot
    c->pivot = pivot;
    c->trees = 0;
    c->draws = 0;
    c->pop_rounds = 0;
    c->max_rounds_seen = 0;
    c->max_depth_seen = 0;
    c->x_valid = false;
    UST_CUDA_TRY(cudaMemsetAsync(c->d_R, 0, (size_t)c->n * 8, c->stream));
    if (c->d_ecount) UST_CUDA_TRY(cudaMemsetAsync(c->d_ecount, 0, (size_t)c->nnz * 8, c->stream));
    int rc = ust::run_bfs(c);
    if (rc) return rc;
    rc = ust::relabel_paths(c);  // the large-graph sampler's paths follow the new B_u
    if (rc) return rc;
    if (c->blocks) {
        rc = ust::build_block_rows(c);  // parent blocks follow the new B_u
        if (rc) return rc;
    }
    c->ready = true;
    return UST_OK;
}

int ust_sample_aggregate(ust_ctx *h, int64_t n_trees, uint64_t seed)
{
    if (!h) return UST_EINVAL;
    Ctx *c = &h->c;
    if (n_trees < 0) return ust::fail(c, UST_EINVAL, "n_trees < 0");
    if (n_trees == 0) return UST_OK;
    if (c->batch) return ust::batch_sample_aggregate(c, n_trees, seed);
    if (const int rc = check_ready(c)) return rc;
    UST_CUDA_TRY(cudaMemcpyAsync(c->d_Rtmp, c->d_R, (size_t)c->n * 8, cudaMemcpyDeviceToDevice, c->stream));
    if (c->d_ecount)
        UST_CUDA_TRY(cudaMemcpyAsync(c->d_ecount_tmp, c->d_ecount, (size_t)c->nnz * 8, cudaMemcpyDeviceToDevice,
                                     c->stream));
    int64_t draws = 0, rounds = 0;
    int max_rounds = 0, max_depth = 0;
    int rc;
    {
        SamplingRows rows(c);
        rc = ust::run_sampler(c, c->trees, c->trees + n_trees, seed, c->d_Rtmp, nullptr, nullptr, &draws, &rounds,
                              &max_rounds, &max_depth);
    }
    if (rc) return rc;
    std::swap(c->d_R, c->d_Rtmp);
    std::swap(c->d_ecount, c->d_ecount_tmp);
    c->trees += n_trees;
    c->seed = seed;
    c->draws += draws;
    c->pop_rounds += rounds;
    c->max_rounds_seen = std::max(c->max_rounds_seen, max_rounds);
    c->max_depth_seen = std::max(c->max_depth_seen, max_depth);
    return UST_OK;
}

int64_t ust_num_trees(const ust_ctx *h)
{
    if (!h) return -1;
    const Ctx *c = &h->c;
    if (!c->batch) return c->trees;
    int64_t least = c->btrees.empty() ? 0 : c->btrees[0];
    for (const int64_t t : c->btrees) least = std::min(least, t);
    return least;
}

int64_t ust_tau(const ust_ctx *h, double eps)
{
    if (!h || !(eps > 0)) return 0;
    const Ctx *c = &h->c;
    if (c->batch) return ust::batch_tau(c, eps);
    const double m = (double)c->nnz / 2.0;
    const double a = log(2.0 * m / c->delta);
    const double b = 2.0 * (1.0 - c->kappa) * (1.0 - c->kappa) * eps * eps;
    return (int64_t)c->ecc * (int64_t)c->ecc * (int64_t)ceil(a / b);
}

int ust_diag(ust_ctx *h, double eps, double *diag_out, int32_t out_on_device)
{
    if (!h) return UST_EINVAL;
    Ctx *c = &h->c;
    if (!diag_out) return ust::fail(c, UST_EINVAL, "null output pointer");
    if (c->batch) return ust::batch_diag(c, eps, diag_out, out_on_device);
    if (eps > 0) {
        const int64_t tau = ust_tau(h, eps);
        if (c->trees < tau) {
            const int rc = ust_sample_aggregate(h, tau - c->trees, c->seed);
            if (rc) return rc;
        }
    }
    if (c->trees <= 0) return ust::fail(c, UST_ESTATE, "no trees aggregated");
    if (!c->x_valid) {
        const int rc = ust::run_solve(c);
        if (rc) return rc;
    }
    double *dst = out_on_device ? diag_out : c->d_f64 + c->n;
    int rc = ust::run_combine(c, c->trees, dst);
    if (rc) return rc;
    if (!out_on_device) return copy_out(c, diag_out, dst, (size_t)c->n * 8, 0);
    return UST_OK;
}

int ust_centralities(ust_ctx *h, double eps, double *closeness_out, double *nrwb_out, double *kirchhoff_out,
                     int32_t out_on_device)
{
    if (!h) return UST_EINVAL;
    Ctx *c = &h->c;
    const int count = c->batch ? c->batch : 1;
    // the diagonal goes to solver scratch that is free once the column is known
    double *d_diag = c->batch ? c->d_br64 : c->d_f64 + c->n;
    int rc = ust_diag(h, eps, d_diag, 1);
    if (rc) return rc;
    if (!closeness_out && !nrwb_out && !kirchhoff_out) return UST_OK;
    const size_t n = (size_t)c->n;
    double *dc = closeness_out, *dn = nrwb_out, *dk = kirchhoff_out, *tmp = nullptr;
    if (!out_on_device) {
        if (cudaMalloc(&tmp, (2 * n + (size_t)count) * sizeof(double)) != cudaSuccess)
            return ust::fail(c, UST_ENOMEM, "centrality outputs");
        dc = closeness_out ? tmp : nullptr;
        dn = nrwb_out ? tmp + n : nullptr;
        dk = kirchhoff_out ? tmp + 2 * n : nullptr;
    }
    rc = ust::run_centralities(c, c->batch ? c->d_comb : nullptr, count, d_diag, dc, dn, dk);
    if (!rc && !out_on_device) {
        if (closeness_out) rc = copy_out(c, closeness_out, dc, n * sizeof(double), 0);
        if (!rc && nrwb_out) rc = copy_out(c, nrwb_out, dn, n * sizeof(double), 0);
        if (!rc && kirchhoff_out) rc = copy_out(c, kirchhoff_out, dk, (size_t)count * sizeof(double), 0);
    }
    cudaFree(tmp);
    return rc;
}

int ust_track_edges(ust_ctx *h, int32_t on)
{
    if (!h) return UST_EINVAL;
    Ctx *c = &h->c;
    cudaFree(c->d_ecount);
    cudaFree(c->d_ecount_tmp);
    c->d_ecount = c->d_ecount_tmp = nullptr;
    if (!on) return UST_OK;
    const size_t bytes = (size_t)c->nnz * sizeof(int64_t);
    if (cudaMalloc(&c->d_ecount, bytes) != cudaSuccess || cudaMalloc(&c->d_ecount_tmp, bytes) != cudaSuccess) {
        cudaFree(c->d_ecount);
        c->d_ecount = nullptr;
        return ust::fail(c, UST_ENOMEM, "arc counts");
    }
    UST_CUDA_TRY(cudaMemsetAsync(c->d_ecount, 0, bytes, c->stream));
    UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return UST_OK;
}

int ust_get_edge_counts(ust_ctx *h, int64_t *counts_out, int32_t out_on_device)
{
    if (!h) return UST_EINVAL;
    Ctx *c = &h->c;
    if (!c->d_ecount) return ust::fail(c, UST_ESTATE, "arc counting is off (ust_track_edges)");
    if (!counts_out) return ust::fail(c, UST_EINVAL, "null output pointer");
    if (c->blocks) {  // counts of walk-row entries, moved to the input CSR's arcs
        const int rc = ust::scatter_block_counts(c, c->d_ecount, c->d_ecount_tmp);
        if (rc) return rc;
        return copy_out(c, counts_out, c->d_ecount_tmp, (size_t)c->nnz * sizeof(int64_t), out_on_device);
    }
    return copy_out(c, counts_out, c->d_ecount, (size_t)c->nnz * sizeof(int64_t), out_on_device);
}

int ust_get_counts(ust_ctx *h, int64_t *R_out, int32_t out_on_device)
{
    if (!h) return UST_EINVAL;
    return copy_out(&h->c, R_out, h->c.d_R, (size_t)h->c.n * 8, out_on_device);
}

int ust_get_column(ust_ctx *h, double *x_out, int32_t out_on_device)
{
    if (!h) return UST_EINVAL;
    Ctx *c = &h->c;
    if (!c->x_valid) {
        const int rc = c->batch ? ust::batch_column(c) : ust::run_solve(c);
        if (rc) return rc;
    }
    return copy_out(c, x_out, c->d_x, (size_t)c->n * 8, out_on_device);
}

int ust_get_bfs(ust_ctx *h, int32_t *parent_out, int32_t *dist_out)
{
    if (!h) return UST_EINVAL;
    Ctx *c = &h->c;
    if (parent_out) {
        const int rc = copy_out(c, parent_out, c->d_bpar, (size_t)c->n * 4, 0);
        if (rc) return rc;
    }
    if (dist_out) return copy_out(c, dist_out, c->d_dist, (size_t)c->n * 4, 0);
    return UST_OK;
}

int ust_tree_range_counts(ust_ctx *h, int64_t t0, int64_t t1, uint64_t seed, int64_t *R_out, int32_t out_on_device)
{
    if (!h) return UST_EINVAL;
    Ctx *c = &h->c;
    if (!R_out || t0 < 0 || t1 < t0) return ust::fail(c, UST_EINVAL, "bad tree range or output");
    if (c->batch) return ust::fail(c, UST_EINVAL, "ust_tree_range_counts applies to single-graph contexts");
    if (const int rc = check_ready(c)) return rc;
    UST_CUDA_TRY(cudaMemsetAsync(c->d_Rtmp, 0, (size_t)c->n * 8, c->stream));
    int rc;
    {
        SamplingRows rows(c);
        rc = ust::run_sampler(c, t0, t1, seed, c->d_Rtmp, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    }
    if (rc) return rc;
    return copy_out(c, R_out, c->d_Rtmp, (size_t)c->n * 8, out_on_device);
}

int ust_set_counts(ust_ctx *h, const int64_t *R_in, int64_t trees, int32_t in_on_device)
{
    if (!h) return UST_EINVAL;
    Ctx *c = &h->c;
    if (!R_in || trees < 1) return ust::fail(c, UST_EINVAL, "ust_set_counts needs counts and trees >= 1");
    UST_CUDA_TRY(cudaMemcpyAsync(c->d_R, R_in, (size_t)c->n * 8,
                                 in_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (c->batch) {  // every graph of the batch gets `trees` trees
        for (int g = 0; g < c->batch; ++g) c->btrees[g] = trees;
        c->trees = trees * c->batch;
    } else {
        c->trees = trees;
    }
    return UST_OK;
}

int ust_sample_trees(ust_ctx *h, int64_t t0, int32_t count, uint64_t seed, int32_t *next_out, int32_t *pops_out)
{
    if (!h) return UST_EINVAL;
    Ctx *c = &h->c;
    if (!next_out || count < 0 || t0 < 0) return ust::fail(c, UST_EINVAL, "bad tree range or output");
    if (c->batch) return ust::fail(c, UST_EINVAL, "ust_sample_trees applies to single-graph contexts");
    if (const int rc = check_ready(c)) return rc;
    if (count == 0) return UST_OK;
    const size_t elems = (size_t)count * (size_t)c->n;
    int32_t *d_next = nullptr, *d_pops = nullptr;
    if (cudaMalloc(&d_next, elems * 4) != cudaSuccess) return ust::fail(c, UST_ENOMEM, "tree export buffer");
    if (pops_out && cudaMalloc(&d_pops, elems * 4) != cudaSuccess) {
        cudaFree(d_next);
        return ust::fail(c, UST_ENOMEM, "tree export buffer");
    }
    int rc;
    {
        SamplingRows rows(c);
        rc = ust::run_sampler(c, t0, t0 + count, seed, nullptr, d_next, d_pops, nullptr, nullptr, nullptr, nullptr);
    }
    if (!rc) rc = copy_out(c, next_out, d_next, elems * 4, 0);
    if (!rc && pops_out) rc = copy_out(c, pops_out, d_pops, elems * 4, 0);
    cudaFree(d_next);
    cudaFree(d_pops);
    return rc;
}

int ust_get_info(const ust_ctx *h, ust_info *out)
{
    if (!h || !out) return UST_EINVAL;
    const Ctx *c = &h->c;
    memset(out, 0, sizeof(*out));
    out->n = c->n;
    out->nnz = c->nnz;
    out->pivot = c->pivot;
    out->ecc = c->ecc;
    out->trees = c->trees;
    out->seed = c->seed;
    out->draws = c->draws;
    out->pop_rounds = c->pop_rounds;
    out->max_pop_rounds = c->max_rounds_seen;
    out->max_round_pops = c->max_depth_seen;
    out->farness = c->farness;
    out->cg_iters = c->cg_iters;
    out->cg_refinements = c->cg_refinements;
    out->cg_relres = c->cg_relres;
    ust::LaunchCfg shape = c->cfg;  // a batch reports the shape of its largest graphs
    if (c->batch)
        for (int k = 0; k < ust::kNumClasses; ++k)
            if (c->class_maxn[k] > 0) shape = c->class_cfg[k];
    out->sample_ctas = shape.ctas;
    out->sample_threads = shape.bt;
    out->kernel_launches = c->launches;
    out->last_trees = c->last_trees;
    out->last_draws = c->last_draws;
    for (int k = 0; k < 12; ++k) out->last_phase_cycles[k] = c->last_phase_cycles[k];
    double *ms[Ctx::kEvPhases] = {&out->bfs_ms, &out->sample_ms, &out->reduce_ms, &out->solve_ms, &out->combine_ms};
    for (int ph = 0; ph < Ctx::kEvPhases; ++ph) {
        if (!c->ev_used[ph]) continue;
        float t = 0.0f;
        if (cudaEventSynchronize(c->ev[2 * ph + 1]) != cudaSuccess) return UST_ECUDA;
        if (cudaEventElapsedTime(&t, c->ev[2 * ph], c->ev[2 * ph + 1]) != cudaSuccess) return UST_ECUDA;
        *ms[ph] = (double)t;
    }
    return UST_OK;
}

const char *ust_last_error(const ust_ctx *h)
{
    if (!h) return g_init_error.c_str();
    return h->c.err.empty() ? "no error" : h->c.err.c_str();
}

const char *ust_strerror(int code)
{
    switch (code) {
    case UST_OK: return "UST_OK";
    case UST_EINVAL: return "UST_EINVAL";
    case UST_ENOTCONNECTED: return "UST_ENOTCONNECTED";
    case UST_ENOMEM: return "UST_ENOMEM";
    case UST_ECUDA: return "UST_ECUDA";
    case UST_ETIMEOUT: return "UST_ETIMEOUT";
    case UST_ENOTCONVERGED: return "UST_ENOTCONVERGED";
    case UST_ESTATE: return "UST_ESTATE";
    default: return "UST_E?";
    }
}

void ust_free(ust_ctx *h)
{
    if (!h) return;
    cudaStreamSynchronize(h->c.stream);
    release(&h->c);
    delete h;
}

}  // extern "C"
