// Shared declarations of libust.so (CUDA, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ust.h"

#define UST_CUDA_TRY(expr)                                                          \
    do {                                                                            \
        cudaError_t _e = (expr);                                                    \
        if (_e != cudaSuccess) {                                                    \
            return ust::fail(c, UST_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
        }                                                                           \
    } while (0)

// Waits for the context's stream; an error names the step that waited.
#define UST_SYNC_TRY(what)                                                                   \
    do {                                                                                     \
        cudaError_t _e = cudaStreamSynchronize(c->stream);                                   \
        if (_e != cudaSuccess) return ust::fail(c, UST_ECUDA, std::string(what) + ": " + cudaGetErrorString(_e)); \
    } while (0)

namespace ust {

// Device status word bits (written by kernels, read by the host).
enum : int {
    kStatusPopRounds = 1,  // a tree exceeded max_pop_rounds
    kStatusJumpSteps = 2,  // pointer jumping did not converge within its bound
    kStatusBadState = 4,   // an internal consistency check failed
};

// One graph of a launch: its CSR, pivot, B_u paths and where its trees and
// counts go. A single-graph launch fills one from SampleParams; a batch
// launch reads one per work item.
struct GraphDesc {
    int n, u;
    // The samplers build trees on sampler ids below ncore only (n: all of
    // them). The ids from ncore on are pendant vertices (degree
    // 1, not the pivot): every spanning tree hangs each from its one
    // neighbour, a draw of one by a core vertex closes a 2-cycle that is
    // popped at once (the core vertex takes its next stack entry), and its
    // counts follow from its neighbour's after the launch.
    int ncore;
    uint32_t graph;            // fourth Philox counter word
    long long voff;            // offset of the graph's vertices in batch-wide arrays
    long long tree_begin;      // first tree id of the graph in this launch
    const int32_t *rp, *ci, *bpar, *path, *pathptr;
    // entry p of the flattened BFS paths is the edge (path[p], pchild[p]) on
    // P(powner[p]); fc entries (f^c(u), or the core's when ncore < n)
    const int32_t *pchild, *powner;
    int fc;
    long long aoff;  // offset of the graph's arcs in batch-wide arc arrays
    // Relabelled graphs (single-graph contexts): rp / ci / u / path / pchild
    // / powner / pathptr are in sampler ids (the path of sampler vertex v at
    // pathptr[v], the paths listed in sampler order), orig[v] is the input id
    // of sampler vertex v (Philox counters, outputs) and rp_in the input
    // row_ptr (arc counts). NULL: ids are input ids (batches). bpar stays in
    // input ids; the samplers do not read it.
    const int32_t *orig, *rp_in;
};

// Graphs of at most this many vertices run the sampler with its per-tree
// state in shared memory (4 bytes per vertex; ids below 2^16).
constexpr int kSmemMaxVertices = 56 * 1024;
// The same sampler serves graphs up to this size (16-bit vertex ids below
// the 0xFFFF sentinel): the words beyond kSmemMaxVertices live in a small
// per-CTA tail in global memory.
constexpr int kTierMaxVertices = 0xFFFF;

// One sampler launch shape: threads per CTA (64, 128, 256, 512 or 1024) and
// the persistent CTAs of the launch (a multiple of the SM count).
struct LaunchCfg {
    int bt = 0;
    int ctas = 0;
};

// Workload key of a tuned launch shape: which sampler kernel, the size of
// the launch's largest graph, average degree and pivot degree, number of
// graphs and SMs.
struct TuneKey {
    int kernel = 0, n_bucket = 0, avg_deg = 0, pivot_deg_log2 = 0, graphs_log2 = 0, sms = 0;
    bool operator<(const TuneKey &o) const
    {
        const int a[6] = {kernel, n_bucket, avg_deg, pivot_deg_log2, graphs_log2, sms};
        const int b[6] = {o.kernel, o.n_bucket, o.avg_deg, o.pivot_deg_log2, o.graphs_log2, o.sms};
        return std::lexicographical_compare(a, a + 6, b, b + 6);
    }
};

// One linear system of the one-CTA column solve (see ust_solve_cta.cu).
struct SolveTask {
    int n = 0, u = 0;
    const int32_t *rp = nullptr, *ci = nullptr;
    const int32_t *heavy = nullptr;  // rows with more than kHeavyRow arcs
    int n_heavy = 0;
    double *x = nullptr;    // the column (output)
    double *r64 = nullptr;  // n doubles of scratch
    void *w = nullptr;      // 5 n scratch values of the inner precision
};
struct SolveResult {
    int iters = 0, refinements = 0;
    double relres = 0.0;
};
// Size classes of a batch: the graphs with at most kClassMaxN[k] vertices
// (and more than the previous bound) share one sampler launch and shape.
constexpr int kNumClasses = 7;
constexpr int kClassMaxN[kNumClasses] = {4096, 8192, 14336, 28672, kSmemMaxVertices, kTierMaxVertices, 0x7FFFFFFF};

// Per-CTA scratch of the sampling kernel: `kWsArrays` int32 arrays of
// `stride` entries each, laid out array-major inside one CTA slot (the last
// two form one 64-bit array).
// Column solve: threads per CTA, and the row length above which one whole
// CTA sums a row of the SpMV.
constexpr int kSolveThreads = 256;
constexpr int kHeavyRow = 256;
constexpr int kWsArrays = 13;

// One graph of a batched B_u launch (one CTA per graph).
struct PrepDesc {
    int n, u;
    const int32_t *rp, *ci;
    int32_t *dist, *bpar, *pathptr, *path, *pchild, *powner;
    long long path_cap;
};
// One graph of a batched diagonal combination.
struct CombineDesc {
    int n, u;
    long long voff, trees;
};
struct Ctx {
    int n = 0;
    int nnz = 0;
    int pivot = 0;
    int graph_id = 0;
    int ecc = 0;
    int64_t farness = 0;
    double delta = 0, kappa = 0.3, cg_tol = 1e-9;
    int max_pop_rounds = 0;
    int max_cg_iters = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;

    // graph and B_u
    int32_t *d_rp = nullptr, *d_ci = nullptr;
    int32_t *d_bpar = nullptr, *d_dist = nullptr;
    int32_t *d_flag = nullptr;  // BFS level flag and misc small device scalars
    int32_t *d_pathptr = nullptr, *d_path = nullptr;  // flattened BFS paths P(v): 3 x path_cap (ancestor, child, owner)
    int64_t path_cap = 0;
    // biconnected-component variant (ust_opts.wilson_blocks): the rows the
    // walks draw from, v's neighbours in its parent block, and each row
    // entry's arc in the input CSR
    bool blocks = false;
    int32_t *d_wrp = nullptr, *d_wci = nullptr, *d_wmap = nullptr;
    int32_t *d_bscratch = nullptr;  // 6 n words for the block labels, allocated with the first rows
    int64_t wnnz = 0;
    // false while B_u (and, with wilson_blocks, the walk rows and the
    // sampler's paths) may not match the pivot: from the start of a
    // ust_reset until it succeeds. Every sampling call refuses to run then.
    bool ready = false;

    // The samplers' view of a single graph (plain Wilson): vertex ids
    // relabelled in Cuthill-McKee order from the pivot of ust_init, pendant
    // vertices last; every row keeps its input order. B_u, the solve and
    // all outputs stay in input ids.
    bool relabel = false;
    int32_t *d_srp = nullptr, *d_sci = nullptr;     // relabelled CSR
    int32_t *d_orig = nullptr, *d_newid = nullptr;  // sampler id -> input id, and back
    int32_t *d_spath = nullptr;  // flattened BFS paths in sampler ids and order: 3 x spath_cap (ancestor, child, owner)
    int32_t *d_spathptr = nullptr;                  // where sampler vertex v's path starts in d_spath
    int64_t spath_cap = 0;
    int spivot = 0;                                 // the pivot's sampler id
    int relabel_core = 0;  // sampler ids below: core vertices; from here on: pendant ones
    int ncore = 0;         // the current pivot's core (n when the pivot itself is pendant)
    int64_t core_fc = 0;   // path entries of the core vertices (they come first)

    // sampling
    LaunchCfg cfg;                  // single graph: the sampler's launch shape
    int req_bt = 0, req_cps = 0;    // requested threads per CTA / CTAs per SM (0 = automatic)
    int64_t ws_stride = 0;          // single graph: words per workspace array
    int64_t ws_cap = 0, rp_cap = 0; // capacity in int32 words of d_ws and d_Rp
    int32_t *d_ws = nullptr;    // ctas * kWsArrays * stride
    int32_t *d_Rp = nullptr;    // ctas * n partial counts (single graph)
    int64_t *d_R = nullptr;     // committed counts
    int64_t *d_Rtmp = nullptr;  // scratch counts (uncommitted)
    int64_t *d_ecount = nullptr;     // trees using each arc v -> parent(v) (ust_track_edges), committed
    int64_t *d_ecount_tmp = nullptr; // the same while a call runs
    int64_t *d_stats = nullptr; // [0] draws, [1] rounds, [2] max rounds, [3] max depth, [4] next tree, [5] status
    int64_t *h_stats = nullptr; // pinned mirror

    // solve
    float *d_f32 = nullptr;     // inner PCG vectors
    double *d_f64inner = nullptr;  // inner PCG vectors of the all-FP64 solve (allocated on first use)
    int solve_n = 0;               // vertices the solver scratch is sized for
    bool solve_fp64 = false;
    double *d_f64 = nullptr;    // outer vectors
    double *d_red = nullptr;    // reduction partials
    double *h_red = nullptr;    // pinned scalars
    double *d_x = nullptr;      // column L^+[:, u]
    bool x_valid = false;
    int solve_blocks = 0;
    int32_t *d_heavy = nullptr;  // rows summed by a whole CTA in the SpMVs
    int n_heavy = 0;
    SolveTask *d_tasks = nullptr;       // one-CTA solve: one task per graph
    SolveResult *d_results = nullptr, *h_results = nullptr;
    float *d_bw32 = nullptr;            // batch: 5 n floats of inner scratch (all graphs)
    double *d_bw64 = nullptr;           // batch: 5 n doubles, FP64 inner scratch (on first use)
    double *d_br64 = nullptr;           // batch: n doubles of residual scratch

    // phase timers: event pairs for bfs, sample kernel, reduce, solve, combine
    enum { kEvBfs = 0, kEvSample = 1, kEvReduce = 2, kEvSolve = 3, kEvCombine = 4, kEvPhases = 5 };
    cudaEvent_t ev[2 * kEvPhases] = {};
    bool ev_used[kEvPhases] = {};
    bool ev_hold[kEvPhases] = {};
    int64_t launches = 0;
    int64_t last_trees = 0, last_draws = 0;
    int64_t last_phase_cycles[12] = {};

    // committed state
    int64_t trees = 0;
    uint64_t seed = 0;
    int64_t draws = 0, pop_rounds = 0;
    int max_rounds_seen = 0, max_depth_seen = 0;
    int cg_iters = 0, cg_refinements = 0;
    double cg_relres = 0;

    // batch of graphs (batch > 0): every per-vertex array holds the graphs'
    // arrays one after another, graph g starting at bvoff[g]; row_ptr and
    // pathptr hold n_g + 1 entries per graph, starting at bvoff[g] + g.
    int batch = 0;
    std::vector<int> bclass;              // size class of every graph
    int class_maxn[kNumClasses] = {};     // largest graph of every class (0 = empty)
    LaunchCfg class_cfg[kNumClasses];     // launch shape of every class
    LaunchCfg class_tuned[kNumClasses];   // the tuner's shape per class (bt 0: not tuned)
    std::vector<int> bn, bnnz, bpivot, becc, bheavy_n, bblocks;
    std::vector<int64_t> bvoff, baoff, bpoff, bhoff, btrees, bfarness;
    GraphDesc *d_graphs = nullptr;  // sampler descriptors (one for a single graph)
    GraphDesc single_desc{};        // last descriptor uploaded for a single graph
    bool single_desc_valid = false;
    long long *d_items = nullptr;
    CombineDesc *d_comb = nullptr;
    PrepDesc *d_prep = nullptr;
    int32_t *d_prep_out = nullptr, *h_prep_out = nullptr;  // 3 x batch: status, ecc, f^c(u)

    std::string err;
};

int fail(Ctx *c, int code, const std::string &msg);

// Records the start / end event of a timed phase on the context's stream.
// While a phase is held open (phase_open ... phase_close around several
// launches), the inner begin / end pairs record nothing.
inline void phase_begin(Ctx *c, int ph)
{
    if (!c->ev_hold[ph]) cudaEventRecord(c->ev[2 * ph], c->stream);
}
inline void phase_end(Ctx *c, int ph)
{
    if (c->ev_hold[ph]) return;
    cudaEventRecord(c->ev[2 * ph + 1], c->stream);
    c->ev_used[ph] = true;
}
inline void phase_open(Ctx *c, int ph)
{
    phase_begin(c, ph);
    c->ev_hold[ph] = true;
}
inline void phase_close(Ctx *c, int ph)
{
    c->ev_hold[ph] = false;
    phase_end(c, ph);
}

// Host drivers (one per translation unit).
int run_bfs(Ctx *c);
// Exclusive prefix sum of in[0, n) into out[0, n] (out[n] = total), one CTA.
cudaError_t launch_exclusive_scan(int n, const int32_t *in, int32_t *out, cudaStream_t st);
// The relabelled CSR of the large-graph sampler (ust_relabel.cu), built once
// per context, and its flattened BFS paths, rebuilt with every B_u.
int build_relabel(Ctx *c);
int relabel_paths(Ctx *c);
// The walk rows of the biconnected-component variant for the current B_u.
int build_block_rows(Ctx *c);
// Arc counts of the variant's walk rows, scattered to the input CSR's arcs.
int scatter_block_counts(Ctx *c, const int64_t *d_walk_counts, int64_t *d_out);
// The input checks of ust_init on a device CSR; d_bad: one int of scratch.
int check_graph(Ctx *c, int n, int nnz, const int32_t *d_rp, const int32_t *d_ci, int *d_bad);
// Pivot by eccentricity lower bounds from `sweeps` double-sweep BFS runs
// (start < 0: the max-degree vertex); returns the vertex of least bound.
int select_pivot(Ctx *c, int n, const int32_t *d_rp, const int32_t *d_ci, int sweeps, int start, int32_t *pivot,
                 int32_t *bound);
// Chooses the single-graph launch shape (requested or automatic) and sizes
// the workspace for it.
int alloc_sampler(Ctx *c, int block_threads, int ctas_per_sm);
// The same for every size class of a batch.
int alloc_batch_sampler(Ctx *c, int block_threads, int ctas_per_sm);
// The fastest launch shape for `items` work items of d_graphs / d_items
// (graphs of at most max_n vertices), timed on a probe whose counts go to
// d_scratch; cached per key for the process.
int tune_launch(Ctx *c, const TuneKey &key, const GraphDesc *d_graphs, const long long *d_items, int ngraphs,
                long long items, int max_n, long long max_rounds, int64_t *d_scratch, LaunchCfg *out,
                double *best_ms_per_item);
// Uploads the single graph's sampler descriptor and item starts when they
// changed; prune: trees on the core of a relabelled graph only (count
// aggregation without arc counts).
int upload_single_desc(Ctx *c, bool prune);
// mode 0: aggregate trees [t0, t1) into d_out (int64 n) - added, not assigned.
// mode 1: export next/pops of trees [t0, t1) to device buffers.
int run_sampler(Ctx *c, int64_t t0, int64_t t1, uint64_t seed, int64_t *d_out, int32_t *d_next_out,
                int32_t *d_pops_out, int64_t *draws, int64_t *rounds, int *max_rounds, int *max_depth);
int run_batch_prepare(Ctx *c, const PrepDesc *d_desc, int count, int *d_out);
// B_u, ecc, f^c(u) and (when they fit path_cap) the paths of one graph in one
// CTA; d_out: status, ecc, f^c(u).
int run_prepare_single(Ctx *c, const PrepDesc &d, int *d_out);
// Closeness, random-walk betweenness and Kirchhoff index from diagonals
// (d_graphs: one CombineDesc per graph, or NULL for the context's single graph).
int run_centralities(Ctx *c, const CombineDesc *d_graphs, int count, const double *d_diag, double *d_closeness,
                     double *d_nrwb, double *d_kirchhoff);
// Single graphs up to this many vertices get B_u from one CTA in one launch
// (f^c(u) < n^2 / 2 stays below 2^31).
constexpr int kPrepMaxN = 32768;
int run_batch_combine(Ctx *c, const CombineDesc *d_desc, int count, double *d_diag);
int run_batch_sampler(Ctx *c, const LaunchCfg &cfg, const GraphDesc *d_graphs, const long long *d_item_start,
                      int ngraphs, long long total_items, int max_n, long long max_rounds, uint64_t seed,
                      int64_t *d_R, int64_t *draws, int64_t *rounds, int *max_round_count, int *max_pops);

// Single graphs with at most this many arcs solve with one CTA; larger ones
// with the multi-kernel solver. Batches always use one CTA per graph.
constexpr int64_t kCtaSolveMaxArcs = 1 << 18;
int run_solve_cta(Ctx *c, const SolveTask *d_tasks, int count, SolveResult *d_results, SolveResult *h_results,
                  bool fp64);

// One graph's column solve: the scratch vectors of the context are sized for
// solve_n >= n vertices.
struct SolveView {
    int n = 0, u = 0;
    const int32_t *rp = nullptr, *ci = nullptr, *heavy = nullptr;
    int n_heavy = 0, blocks = 1;
    double *x = nullptr;
};
int alloc_solver(Ctx *c);
int run_solve(Ctx *c);
int run_solve_view(Ctx *c, const SolveView &g);
int run_combine(Ctx *c, int64_t tau, double *d_diag);

}  // namespace ust

struct ust_ctx {
    ust::Ctx c;
};
