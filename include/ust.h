/*
 * ust.h - C ABI of libust.so: GB300 (sm_103a) implementation of the UST
 * approximation of diag(L^+) for a connected, undirected, unweighted graph
 * (Angriman, Predari, van der Grinten, Meyerhenke, arXiv 2006.13679,
 * Algorithm 1 "ApproxDiagLpinv").
 *
 * The library computes, on one GPU:
 *   - the BFS tree B_u of the pivot u (Section 3.2, Algorithm 1),
 *   - uniform spanning trees T_t rooted at u with Wilson's algorithm
 *     (Appendix A.2), done as parallel cycle popping on per-vertex stacks,
 *   - per tree, the +-1 electrical-flow counts of Algorithm 2 along the BFS
 *     paths P(v), summed exactly into R[v] (an estimate of tau * r(u, v)),
 *   - the column x = L^+[:, u] from L x = e_u - (1/n) 1, x _|_ 1
 *     (Section 3.1 step 1, Algorithm 1), with FP32 Jacobi-PCG inside FP64
 *     iterative refinement,
 *   - diag(L^+): L^+[u,u] = x_u, L^+[v,v] = R[v]/tau - x_u + 2 x_v
 *     (Eq. diag-comp, Algorithm 1).
 *
 * Random choices. Stack entry k of vertex v in tree t is the neighbour
 *   col_idx[row_ptr[v] + floor(X * deg(v) / 2^64)],
 * X = (w1 << 32) | w0 of Philox4x32-10 (Salmon et al., SC'11) with counter
 * (v, k, t, graph_id) and key (seed mod 2^32, seed >> 32). By Wilson's
 * cycle-popping theorem the tree for (seed, t) does not depend on the order in
 * which cycles are popped, so every tree, and therefore R, is a deterministic
 * function of (graph, pivot, seed, tree ids), identical to a sequential
 * loop-erased-walk implementation with the same stacks.
 *
 * Readings of the paper fixed by this library:
 *   - Algorithm 2's subtree test is inclusive (v in the subtree of b, b
 *     included); with the printed strict test the edge into v never counts.
 *   - parent(.) in Algorithm 2 is the parent in T rooted at u.
 *   - B_u's parent of v is the smallest-id neighbour one level closer to u.
 *   - tau = ecc(u)^2 * ceil(ln(2m/delta) / (2 (1-kappa)^2 eps^2)), natural log.
 *
 * Conventions.
 *   - All functions return UST_OK (0) or a negative UST_E* code; on error the
 *     context keeps its previous committed state (R, tree count, column) and
 *     ust_last_error() describes the failure.
 *   - Host pointers are plain CPU memory; "device" pointers are CUDA device
 *     pointers on the context's device. Every pointer argument is owned by
 *     the caller; the library copies what it keeps.
 *   - Work is issued on the context's stream (ust_opts.stream, a
 *     cudaStream_t, or the legacy default stream when NULL). Functions that
 *     return data to host memory synchronise that stream before returning.
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef UST_H
#define UST_H

#include <stdint.h>

#if defined(__GNUC__)
#define UST_API __attribute__((visibility("default")))
#else
#define UST_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define UST_OK 0
#define UST_EINVAL (-1)        /* bad argument or malformed CSR (asymmetric, self-loop, unsorted/duplicate columns) */
#define UST_ENOTCONNECTED (-2) /* graph is not connected */
#define UST_ENOMEM (-3)        /* device or host allocation failed */
#define UST_ECUDA (-4)         /* CUDA runtime error */
#define UST_ETIMEOUT (-5)      /* a device loop hit its iteration bound (pop rounds, jump steps) */
#define UST_ENOTCONVERGED (-6) /* the solver did not reach cg_tol within max_cg_iters */
#define UST_ESTATE (-7)        /* call not valid in the context's state (e.g. no trees sampled) */

typedef struct ust_ctx ust_ctx;

/* Graph in CSR form, vertices 0..n-1. Row v lists the neighbours of v in
 * strictly increasing order; every edge {a, b} appears as arc a->b and b->a.
 * nnz = 2m. row_ptr has n+1 entries with row_ptr[0] = 0, row_ptr[n] = nnz.
 * on_device = 1 when both arrays are device pointers. */
typedef struct {
    int32_t n;
    int32_t nnz;
    const int32_t *row_ptr;
    const int32_t *col_idx;
    int32_t on_device;
} ust_csr;

/* Options; zero-initialised fields take the defaults in brackets. */
typedef struct {
    double delta;           /* failure probability for tau [1/n] (Algorithm 1) */
    double kappa;           /* error split between solver and sampling [0.3] (Appendix D.1) */
    double cg_tol;          /* relative residual ||b - L x|| / ||b|| of the column [1e-9] */
    int32_t max_pop_rounds; /* bound on cycle-popping rounds per tree [16 (2m ecc(u) + n) + 1024] */
    int32_t max_cg_iters;   /* bound on inner FP32 PCG iterations per refinement step [20000] */
    int32_t skip_validation; /* 1: trust the CSR; 0: check it on the device: row pointers, column
                                range, self-loops, sorted rows, symmetry, isolated vertices [0] */
    int32_t graph_id;       /* fourth Philox counter word [0] */
    int32_t block_threads;  /* threads per sampling CTA: 64, 128, 256, 512 or 1024 (the sampler of
                               graphs above 65,535 vertices: 256 or more) [0 = tuned or by graph size,
                               see autotune] */
    int32_t ctas_per_sm;    /* sampling CTAs per SM, capped by what registers and shared memory allow
                               [0 = as many as fit] */
    int32_t solve_fp64;     /* 1: run the whole column solve in FP64 (reference form) [0 = FP32 PCG
                               inside FP64 refinement] */
    int32_t wilson_blocks;  /* 1: the biconnected-component variant of Wilson's algorithm (Appendix D,
                               after Hayashi et al.): every v != u draws its stack entries only among
                               its neighbours in its parent block, the block of the edge
                               (v, bfs_parent(v)), in CSR order. Each block then samples its own
                               uniform tree rooted at its vertex nearest u; the union is a uniform
                               spanning tree directed toward u, so R keeps its meaning, but for the
                               same seed the trees differ from plain Wilson's. The rows are rebuilt
                               with B_u (ust_init, ust_reset); arc counts stay per input arc.
                               Single-graph contexts only (ust_init_batch: UST_EINVAL)
                               [0 = plain Wilson rooted at u] */
    int32_t autotune;       /* launch shapes of the sampler: 1 = tuned, -1 or 0 = fixed table
                               [0]. Tuning times every
                               candidate shape (threads per CTA x CTAs per SM that fit) on a probe of
                               the launch's own work at context creation and keeps the fastest; the
                               choice is remembered for the process per workload key (kernel, size
                               class, average and pivot degree, graph count). block_threads /
                               ctas_per_sm, when set, override it. Counts do not depend on the shape. */
    void *stream;           /* cudaStream_t to issue work on [NULL = legacy default stream] */
} ust_opts;

/* Counters of the committed state. */
typedef struct {
    int32_t n, nnz, pivot, ecc;
    int64_t trees;          /* trees aggregated into R so far, ids [0, trees) */
    uint64_t seed;          /* seed of the last sampling call */
    int64_t draws;          /* stack entries drawn over all trees (Wilson walk steps), counted as
                               for the whole graph also where the sampler leaves degree-1 vertices
                               out of its trees */
    int64_t pop_rounds;     /* cycle-popping rounds summed over trees */
    int32_t max_pop_rounds; /* largest number of rounds one tree needed */
    int32_t max_round_pops; /* most vertices popped in one cycle-popping round */
    int64_t farness;        /* f^c(u) = sum_v dist(u, v): pair tests of Algorithm 2 per tree */
    int32_t cg_iters;       /* inner PCG iterations of the last solve */
    int32_t cg_refinements; /* FP64 refinement steps of the last solve */
    double cg_relres;       /* final ||b - L x|| / ||b|| in FP64 */
    int32_t sample_ctas;    /* CTAs of the sampling launch */
    int32_t sample_threads; /* threads per sampling CTA */
    int64_t kernel_launches; /* kernels this context has launched so far */
    /* device time (CUDA events on the context's stream) of the last run of
     * each phase, in milliseconds */
    double bfs_ms;          /* B_u */
    double sample_ms;       /* the sampling/aggregation kernel alone */
    double reduce_ms;       /* summing the partial count rows */
    double solve_ms;        /* the column solve */
    double combine_ms;      /* the diagonal combination */
    int64_t last_trees;     /* trees processed by the last sampling launch */
    int64_t last_draws;     /* stack entries drawn by the last sampling launch */
    /* SM clock cycles of the last sampling launch per phase, summed over
     * trees (graphs of at most 65,535 vertices): [0] first draws,
     * [1] in-degrees, [2] leaf queue, [3] peeling, [4] cycle list, [5] later
     * popping rounds, [6] children counts and leaf queue, [7] subtree sizes
     * and offsets, [8] preorder numbers, [9] Algorithm 2, [10] whole tree,
     * [11] unused. Larger graphs fill [0] first draws and in-degrees,
     * [1] peeling, [2] cycle list, [3] later popping rounds, [4] subtree
     * sizes and offsets, [5] preorder numbers, [6] Algorithm 2, [7] whole
     * tree; [8] to [11] unused. */
    int64_t last_phase_cycles[12];
} ust_info;

/* Fills *o with the defaults. */
UST_API void ust_default_opts(ust_opts *o);

/* Creates a context for graph g and pivot u = pivot: copies the CSR to the
 * device, checks it there (unless skip_validation; see ust_csr), computes
 * B_u, ecc(u), f^c(u) and the flattened BFS paths (Section 3.2, Algorithm 1)
 * and sizes the sampler and solver scratch. Errors: UST_EINVAL (bad CSR or
 * pivot), UST_ENOTCONNECTED (an isolated vertex or a vertex B_u does not
 * reach), UST_ENOMEM, UST_ECUDA. On error *out is NULL and
 * ust_last_error(NULL) describes the failure. */
UST_API int ust_init(const ust_csr *g, int32_t pivot, const ust_opts *o, ust_ctx **out);

/* A pivot of low eccentricity (Appendix D, choice of u; Theorem 1's running
 * time grows with ecc(u)^2): `sweeps` BFS runs (<= 0: the paper's 10), the
 * first from `start` (< 0: the vertex of largest degree), each next one
 * from the vertex farthest from the previous source. Every vertex keeps the
 * largest distance seen from any source, a lower bound on its
 * eccentricity; *pivot_out is the vertex of least bound, *bound_out (may be
 * NULL) that bound. Ties go to the smallest vertex id. The graph is checked
 * as in ust_init (host or device arrays, not modified). Errors: UST_EINVAL,
 * UST_ENOTCONNECTED, UST_ENOMEM, UST_ECUDA; the message is
 * ust_last_error(NULL). */
UST_API int ust_select_pivot(const ust_csr *g, int32_t sweeps, int32_t start, void *stream, int32_t *pivot_out,
                             int32_t *bound_out);

/* Creates a context for a batch of `count` graphs gs[0..count), graph g with
 * pivot pivots[g] (Algorithm 1 for every graph at once). The graphs'
 * vertices are laid out one after another: every per-vertex output (counts,
 * columns, diagonals, B_u) holds graph 0's n_0 values, then graph 1's, and
 * so on (ust_batch_offsets gives the offsets). Graph g draws its stacks with
 * fourth Philox counter word graph_id + g. ust_sample_aggregate samples
 * n_trees trees of every graph; ust_diag(eps > 0) tops every graph up to its
 * own tau(eps); ust_tau returns the largest tau over the graphs;
 * ust_reset(c, -1) recomputes every graph's B_u with its own pivot and clears
 * all counts and columns. ust_tree_range_counts and ust_sample_trees apply to
 * single-graph contexts only (UST_EINVAL). Errors as ust_init; the message
 * names the graph. */
UST_API int ust_init_batch(const ust_csr *gs, const int32_t *pivots, int32_t count, const ust_opts *o,
                           ust_ctx **out);

/* Number of graphs of a batch context, 0 for a single-graph context. */
UST_API int32_t ust_batch_size(const ust_ctx *c);

/* count+1 vertex offsets of a batch: graph g's values are at
 * [offsets[g], offsets[g+1]) of every per-vertex output. */
UST_API int ust_batch_offsets(const ust_ctx *c, int64_t *offsets_out);

/* n, nnz, pivot, ecc, trees and f^c(u) of graph g of a batch. */
UST_API int ust_batch_graph_info(const ust_ctx *c, int32_t g, ust_info *out);

/* Re-targets the context to pivot u = pivot on the same graph: recomputes
 * B_u, ecc(u) and f^c(u) and clears R, the tree count and the cached column
 * (Algorithm 1 from its first line); with wilson_blocks the walk rows are
 * rebuilt for the new B_u (in scratch allocated by ust_init). It allocates
 * only when the new pivot's f^c(u) exceeds the flattened-path space the
 * context holds (12 bytes per entry, 16 above 65,535 vertices). A batch
 * context keeps its pivots: pivot must be -1 there. If the call fails after
 * its argument checks, the context refuses every sampling call with
 * UST_ESTATE until a ust_reset succeeds. Errors: UST_EINVAL, UST_ENOMEM,
 * UST_ECUDA. */
UST_API int ust_reset(ust_ctx *c, int32_t pivot);

/* Samples trees with ids [trees, trees + n_trees) under `seed` and adds their
 * Algorithm 2 counts to R (the sampling loop of Algorithm 1). Tree ids
 * continue across calls, so k calls of n trees equal one call of k*n trees
 * with the same seed. Tree ids must stay below 2^32. Errors: UST_EINVAL,
 * UST_ETIMEOUT (a tree exceeded max_pop_rounds; R unchanged), UST_ECUDA. */
UST_API int ust_sample_aggregate(ust_ctx *c, int64_t n_trees, uint64_t seed);

/* Writes diag(L^+) estimates (n doubles) to diag_out (device pointer when
 * out_on_device = 1). If eps > 0 and fewer than tau(eps) trees have been
 * aggregated, first samples the missing ids with the last seed (seed 0 if
 * none was given). Uses all aggregated trees: L^+[v,v] = R[v]/trees - x_u
 * + 2 x_v, with x = L^+[:, u] solved once and cached. Errors: UST_ESTATE (no
 * trees and eps <= 0), UST_ENOTCONVERGED, UST_ETIMEOUT, UST_ECUDA. */
UST_API int ust_diag(ust_ctx *c, double eps, double *diag_out, int32_t out_on_device);

/* Centralities that depend only on diag(L^+) (Section 3.1, Eq. elec-farness;
 * the normalized random-walk betweenness lemma; the Kirchhoff index
 * K = n tr(L^+)), from the estimate of ust_diag(c, eps, ...):
 *   closeness_out[v] = (n - 1) / (n L+[v,v] + tr(L+))    electrical closeness
 *   nrwb_out[v]      = 1/n + tr(L+) / ((n - 1) (n L+[v,v] + tr(L+)))
 *   kirchhoff_out[g] = n tr(L+)                           one per graph
 * n doubles each (a batch: its total n, laid out as the diagonals; one
 * Kirchhoff index per graph); any output may be NULL. The trace is a
 * fixed-order FP64 sum. Errors as ust_diag. */
UST_API int ust_centralities(ust_ctx *c, double eps, double *closeness_out, double *nrwb_out, double *kirchhoff_out,
                             int32_t out_on_device);

/* Sample size tau(eps) of Algorithm 1 for this graph and pivot. */
UST_API int64_t ust_tau(const ust_ctx *c, double eps);

/* Trees aggregated in R so far: tau of the combination in Algorithm 1 (the
 * committed count; a failed call leaves it unchanged, ust_set_counts sets
 * it, ust_reset clears it). A batch: the least count over its graphs
 * (ust_batch_graph_info gives each graph's). -1 for a NULL context. */
UST_API int64_t ust_num_trees(const ust_ctx *c);

/* R[v] as exact integers (n int64). */
UST_API int ust_get_counts(ust_ctx *c, int64_t *R_out, int32_t out_on_device);

/* Turns counting of tree arcs on (on != 0, counts start at 0) or off. While
 * on, every tree sampled by ust_sample_aggregate adds 1 at the CSR position
 * k of each of its arcs v -> parent(v) (the final stack entry of v). The
 * fraction of trees that use an undirected edge {v, w} (both arcs summed) is
 * an estimate of Pr[e in UST] = r(v, w) (Kirchhoff; Appendix on Kirchhoff
 * edge centrality, sampling USTs and counting the trees an edge appears in).
 * Costs one Philox draw and one atomic per vertex and tree. Errors:
 * UST_ENOMEM. */
UST_API int ust_track_edges(ust_ctx *c, int32_t on);

/* The arc counts (nnz int64, CSR order; a batch: all graphs' arcs one after
 * another). Committed with R: a failed call leaves them unchanged;
 * ust_reset clears them. Errors: UST_ESTATE when counting is off. */
UST_API int ust_get_edge_counts(ust_ctx *c, int64_t *counts_out, int32_t out_on_device);

/* The column x = L^+[:, u] (n doubles); solves it first if needed. */
UST_API int ust_get_column(ust_ctx *c, double *x_out, int32_t out_on_device);

/* B_u on the host: parent[v] (-1 at u) and dist[v]; either may be NULL. */
UST_API int ust_get_bfs(ust_ctx *c, int32_t *parent_out, int32_t *dist_out);

/* Counts of trees [t0, t1) under `seed` written to R_out (n int64) without
 * touching the context's R: parity checks on tree subsets. */
UST_API int ust_tree_range_counts(ust_ctx *c, int64_t t0, int64_t t1, uint64_t seed, int64_t *R_out,
                          int32_t out_on_device);

/* Replaces the context's R with R_in (n int64, exact Algorithm-2 counts of
 * `trees` trees of this graph and pivot) and its tree count with `trees`.
 * This is how counts sampled elsewhere are combined before ust_diag: the
 * paper distributes trees over processes and sums R at the end (Appendix D,
 * distributed-memory parallelism); here each GPU computes the counts of its
 * own tree-id range with ust_tree_range_counts under a common seed, the
 * integer rows are summed (an exact, order-free reduction), and the sum is
 * installed with this call. The library cannot verify R_in. The cached
 * column stays valid (it depends only on the graph and pivot). For a batch,
 * R_in holds every graph's counts (offsets as ust_batch_offsets) and every
 * graph gets `trees` trees. Errors: UST_EINVAL (NULL R_in, trees < 1),
 * UST_ECUDA. */
UST_API int ust_set_counts(ust_ctx *c, const int64_t *R_in, int64_t trees, int32_t in_on_device);

/* The sampled trees themselves: for tree ids t0 .. t0+count-1 writes
 * next_out[i*n + v] (tree parent of v, -1 at u) and, when pops_out is not
 * NULL, pops_out[i*n + v] (cycles popped at v = stack depth of the final
 * entry). Host pointers. */
UST_API int ust_sample_trees(ust_ctx *c, int64_t t0, int32_t count, uint64_t seed, int32_t *next_out,
                     int32_t *pops_out);

/* Counters of the committed state. */
UST_API int ust_get_info(const ust_ctx *c, ust_info *out);

/* Tree counts without any allocation. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, such as code
 * whose device memory belongs to another allocator that must account for
 * every byte (a framework's caching allocator, a fixed memory budget) or code
 * that may not allocate after start-up.
 *
 * Computes B_u of pivot u, then samples trees [t0, t1) under `seed` and
 * graph_id and writes their Algorithm 2 counts to R_out (n int64, device
 * pointer, overwritten): the same values as ust_tree_range_counts on a
 * context for this graph, pivot and graph_id. row_ptr and col_idx are device
 * pointers to a CSR obeying the ust_csr contract (not validated here).
 * stream is a cudaStream_t or NULL; the call synchronises it before returning.
 *
 * All scratch lives in one fixed device array inside the library (about
 * 10.6 MB, held on every GPU that loads the library until the process exits).
 * Limits: n <= 4096 and f^c(u) = sum_v dist(u, v) <= 262144. A larger n
 * returns UST_EINVAL before any work; f^c(u) is known only once B_u has been
 * computed, in the scratch array, so a larger f^c(u) returns UST_EINVAL (and
 * a graph that is not connected UST_ENOTCONNECTED) after that step. In every
 * error case R_out is left untouched. The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture. Every call reuses the same
 * array and overwrites what the previous call left there, so calls that can
 * overlap on the GPU (other streams, other host threads) race: serialise them.
 * Errors: UST_EINVAL, UST_ENOTCONNECTED, UST_ETIMEOUT, UST_ECUDA. */
UST_API int ust_tree_counts_noalloc(const int32_t *row_ptr, const int32_t *col_idx, int32_t n, int32_t nnz,
                                    int32_t pivot, int64_t t0, int64_t t1, uint64_t seed, int32_t graph_id,
                                    int64_t *R_out, void *stream);

/* Static description of the last error of this context (never NULL). */
UST_API const char *ust_last_error(const ust_ctx *c);

/* Name of an error code. */
UST_API const char *ust_strerror(int code);

/* Releases every resource of the context; NULL is a no-op. */
UST_API void ust_free(ust_ctx *c);

#ifdef __cplusplus
}
#endif

#endif /* UST_H */
