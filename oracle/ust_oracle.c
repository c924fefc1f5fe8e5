/*
 * CPU oracle for the UST approximation of diag(L^+) (Angriman, Predari,
 * van der Grinten, Meyerhenke, arXiv 2006.13679).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain, sequential
 * statement of what the method computes, used to check the CUDA library.
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load it. It shares no code, header or table with the CUDA path.
 *
 * Every function follows one passage of the paper:
 *   orc_philox4x32_10   counter-based generator of Salmon et al. (SC'11),
 *                       replacing the paper's PCG32 (Appendix D.1)
 *   orc_successor       random neighbour of v for stack entry `depth`
 *   orc_bfs             BFS tree B_u (Section 3.2, Algorithm 1)
 *   orc_wilson          Wilson's loop-erased random walks (Appendix A.2)
 *   orc_cycle_pop       explicit cycle popping on the same stacks (Wilson's
 *                       cycle-popping theorem, cited in Appendix A.2)
 *   orc_dfs_times       DFS discovery/finish timestamps alpha, Omega (Alg. 2)
 *   orc_aggregate       Algorithm 2, inclusive subtree test
 *   orc_sample_aggregate  the sampling loop of Algorithm 1 (with the
 *                       shared-memory scheme of Appendix D.2 when threads > 1)
 *   orc_cg              Jacobi-preconditioned CG for L x = e_u - 1/n
 *                       (Algorithm 1 and Appendix D.1), projected onto 1-perp
 *   orc_combine         diagonal combination, Eq. (diag-comp) / Algorithm 1
 *   orc_tau             sample size tau of Algorithm 1
 *
 * Readings where the paper is silent or ambiguous:
 *   - Algorithm 2 prints strict inequalities alpha(b) < alpha(v),
 *     Omega(v) < Omega(b); with them the edge entering v itself never counts
 *     (on the path u-b, r(u,b) would come out 0). The test is taken inclusive:
 *     v lies in the subtree of b, b included.
 *   - "parent(b) = a" refers to the parent in the UST T rooted at u.
 *   - The BFS parent of v is its smallest-id neighbour one level closer to u.
 *   - Stack entry k of vertex v in tree t of graph g under seed s is the
 *     neighbour col_idx[row_ptr[v] + floor(x * deg(v) / 2^64)], where x is
 *     the 64-bit word (w1 << 32) | w0 of Philox4x32-10 with counter
 *     (v, k, t, g) and key (s mod 2^32, s >> 32). The root never draws.
 *   - tau uses the natural logarithm; delta defaults to 1/n.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EXPORT __attribute__((visibility("default")))

/* ---------------------------------------------------------------------- */
/* Philox4x32-10: ten rounds of the Philox S-box with a Weyl key schedule. */

static void philox_round(uint32_t x[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t y0 = hi1 ^ x[1] ^ k[0];
    const uint32_t y1 = lo1;
    const uint32_t y2 = hi0 ^ x[3] ^ k[1];
    const uint32_t y3 = lo0;
    x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3;
}

ORC_EXPORT void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(x, k);
    }
    out[0] = x[0]; out[1] = x[1]; out[2] = x[2]; out[3] = x[3];
}

ORC_EXPORT int32_t orc_successor(const int32_t *row_ptr, const int32_t *col_idx, int32_t v,
                                 uint32_t depth, uint32_t tree, uint32_t graph, uint64_t seed)
{
    const uint32_t ctr[4] = {(uint32_t)v, depth, tree, graph};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    const uint64_t x = ((uint64_t)w[1] << 32) | (uint64_t)w[0];
    const uint64_t deg = (uint64_t)(row_ptr[v + 1] - row_ptr[v]);
    const uint64_t idx = (uint64_t)(((unsigned __int128)x * deg) >> 64);
    return col_idx[row_ptr[v] + (int64_t)idx];
}

/* ---------------------------------------------------------------------- */
/* BFS tree B_u. Returns ecc(u), or -1 when some vertex is unreachable.    */

ORC_EXPORT int32_t orc_bfs(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t u,
                           int32_t *dist, int32_t *parent)
{
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t v = 0; v < n; ++v) dist[v] = -1;
    int32_t head = 0, tail = 0;
    dist[u] = 0;
    queue[tail++] = u;
    while (head < tail) {
        const int32_t v = queue[head++];
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            const int32_t w = col_idx[e];
            if (dist[w] < 0) {
                dist[w] = dist[v] + 1;
                queue[tail++] = w;
            }
        }
    }
    free(queue);
    int32_t ecc = 0;
    for (int32_t v = 0; v < n; ++v) {
        if (dist[v] < 0) return -1;
        if (dist[v] > ecc) ecc = dist[v];
    }
    /* parent = smallest-id neighbour one level closer to u */
    for (int32_t v = 0; v < n; ++v) {
        parent[v] = -1;
        if (v == u) continue;
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            const int32_t w = col_idx[e];
            if (dist[w] == dist[v] - 1 && (parent[v] < 0 || w < parent[v])) parent[v] = w;
        }
    }
    return ecc;
}

/* ---------------------------------------------------------------------- */
/* Wilson's algorithm with loop-erased random walks (Appendix A.2).
 * Start vertices are taken in increasing id order. Each visit of a vertex
 * that is not yet in the tree consumes that vertex's next stack entry; the
 * last one consumed is its tree successor. next[u] = -1. pops[v] receives
 * (entries consumed - 1), the number of cycles popped at v. Returns the total
 * number of entries consumed (random walk steps). */

ORC_EXPORT int64_t orc_wilson(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t u,
                              uint32_t tree, uint32_t graph, uint64_t seed,
                              int32_t *next, int32_t *pops)
{
    uint8_t *in_tree = (uint8_t *)calloc((size_t)n, 1);
    uint32_t *used = (uint32_t *)calloc((size_t)n, sizeof(uint32_t));
    int64_t steps = 0;
    in_tree[u] = 1;
    next[u] = -1;
    for (int32_t s = 0; s < n; ++s) {
        int32_t cur = s;
        while (!in_tree[cur]) {
            next[cur] = orc_successor(row_ptr, col_idx, cur, used[cur], tree, graph, seed);
            used[cur] += 1;
            steps += 1;
            cur = next[cur];
        }
        cur = s;
        while (!in_tree[cur]) {
            in_tree[cur] = 1;
            cur = next[cur];
        }
    }
    for (int32_t v = 0; v < n; ++v) pops[v] = (v == u) ? 0 : (int32_t)used[v] - 1;
    free(in_tree);
    free(used);
    return steps;
}

/* Explicit cycle popping on the same stacks: start from every vertex's first
 * entry, then repeatedly find a cycle among the current stack tops and pop
 * it (advance every vertex on it to its next entry) until none is left. A
 * second, independent statement of the sampler for cross-checking. */

ORC_EXPORT int64_t orc_cycle_pop(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t u,
                                 uint32_t tree, uint32_t graph, uint64_t seed,
                                 int32_t *next, int32_t *pops)
{
    uint8_t *done = (uint8_t *)calloc((size_t)n, 1);
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t walk = 0; /* every walk gets a fresh stamp */
    int64_t draws = 0;
    for (int32_t v = 0; v < n; ++v) {
        mark[v] = -1;
        pops[v] = 0;
        if (v == u) {
            next[v] = -1;
            done[v] = 1;
        } else {
            next[v] = orc_successor(row_ptr, col_idx, v, 0, tree, graph, seed);
            draws += 1;
        }
    }
    int32_t remaining = n - 1;
    while (remaining > 0) {
        for (int32_t s = 0; s < n; ++s) {
            if (done[s]) continue;
            walk += 1;
            int32_t cur = s;
            mark[cur] = walk;
            for (;;) {
                const int32_t w = next[cur];
                if (done[w]) {
                    int32_t x = s;
                    while (!done[x]) {
                        done[x] = 1;
                        remaining -= 1;
                        x = next[x];
                    }
                    break;
                }
                if (mark[w] == walk) {
                    /* cycle w -> ... -> cur -> w: pop every vertex on it */
                    int32_t x = w;
                    do {
                        const int32_t y = next[x];
                        pops[x] += 1;
                        next[x] = orc_successor(row_ptr, col_idx, x, (uint32_t)pops[x], tree, graph, seed);
                        draws += 1;
                        mark[x] = -1;
                        x = y;
                    } while (x != w);
                    break;
                }
                mark[w] = walk;
                cur = w;
            }
        }
    }
    free(done);
    free(mark);
    return draws;
}

/* ---------------------------------------------------------------------- */
/* DFS of T rooted at u with the child/sibling representation of Section 3.2:
 * alpha(v) = discovery time, Omega(v) = finish time, one clock for both. */

ORC_EXPORT void orc_dfs_times(int32_t n, const int32_t *next, int32_t u, int32_t *alpha, int32_t *omega)
{
    int32_t *child = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *sibling = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *iter = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t v = 0; v < n; ++v) child[v] = -1;
    for (int32_t v = n - 1; v >= 0; --v) {
        if (v == u) continue;
        sibling[v] = child[next[v]];
        child[next[v]] = v;
    }
    int32_t clock = 0, sp = 0;
    alpha[u] = clock++;
    iter[u] = child[u];
    stack[sp++] = u;
    while (sp > 0) {
        const int32_t v = stack[sp - 1];
        const int32_t c = iter[v];
        if (c >= 0) {
            iter[v] = sibling[c];
            alpha[c] = clock++;
            iter[c] = child[c];
            stack[sp++] = c;
        } else {
            omega[v] = clock++;
            sp -= 1;
        }
    }
    free(child);
    free(sibling);
    free(iter);
    free(stack);
}

/* Algorithm 2: for every v != u and every edge (a, b) of the BFS path P(v)
 * (a = bfs_parent(b), directed away from u): +1 when a is b's parent in T and
 * v lies in T's subtree of b, -1 when b is a's parent in T and v lies in T's
 * subtree of a. Adds the counts of this tree into R. */

ORC_EXPORT void orc_aggregate(int32_t n, const int32_t *next, const int32_t *bfs_parent, int32_t u,
                              const int32_t *alpha, const int32_t *omega, int64_t *R)
{
    for (int32_t v = 0; v < n; ++v) {
        if (v == u) continue;
        int64_t c = 0;
        for (int32_t b = v; b != u; b = bfs_parent[b]) {
            const int32_t a = bfs_parent[b];
            if (next[b] == a) {
                if (alpha[b] <= alpha[v] && omega[v] <= omega[b]) c += 1;
            } else if (next[a] == b) {
                if (alpha[a] <= alpha[v] && omega[v] <= omega[a]) c -= 1;
            }
        }
        R[v] += c;
    }
}

/* The sampling loop of Algorithm 1 for tree ids [t0, t1): Wilson, DFS,
 * Algorithm 2. With threads > 1 the trees are split over OpenMP threads, each
 * with its own R, and the partial R vectors are summed at the end (the
 * shared-memory scheme of Appendix D.2). Returns the total number of random
 * walk steps. */

ORC_EXPORT int64_t orc_sample_aggregate(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                                        int32_t u, const int32_t *bfs_parent, int64_t t0, int64_t t1,
                                        uint32_t graph, uint64_t seed, int64_t *R, int32_t threads)
{
    int64_t steps = 0;
    if (threads < 1) threads = 1;
#ifdef _OPENMP
#pragma omp parallel num_threads(threads) reduction(+ : steps)
#endif
    {
        int64_t *Rl = (int64_t *)calloc((size_t)n, sizeof(int64_t));
        int32_t *next = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        int32_t *pops = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        int32_t *alpha = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        int32_t *omega = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t t = t0; t < t1; ++t) {
            steps += orc_wilson(n, row_ptr, col_idx, u, (uint32_t)t, graph, seed, next, pops);
            orc_dfs_times(n, next, u, alpha, omega);
            orc_aggregate(n, next, bfs_parent, u, alpha, omega, Rl);
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            for (int32_t v = 0; v < n; ++v) R[v] += Rl[v];
        }
        free(Rl);
        free(next);
        free(pops);
        free(alpha);
        free(omega);
    }
    return steps;
}

ORC_EXPORT int32_t orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Jacobi-preconditioned CG in FP64 for L x = e_u - (1/n) 1, then x is
 * projected onto 1-perp. Returns 0 when ||b - L x|| / ||b|| <= tol. */

static void lap_mul(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const double *p, double *q)
{
    for (int32_t v = 0; v < n; ++v) {
        double s = 0.0;
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) s += p[col_idx[e]];
        q[v] = (double)(row_ptr[v + 1] - row_ptr[v]) * p[v] - s;
    }
}

static double dot(int32_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

ORC_EXPORT int32_t orc_cg(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t u,
                          double tol, int32_t max_iter, double *x, int32_t *iters_out, double *relres_out)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    const double inv_n = 1.0 / (double)n;
    for (int32_t v = 0; v < n; ++v) {
        x[v] = 0.0;
        r[v] = (v == u ? 1.0 : 0.0) - inv_n;
    }
    const double bnorm = sqrt(dot(n, r, r));
    for (int32_t v = 0; v < n; ++v) {
        z[v] = r[v] / (double)(row_ptr[v + 1] - row_ptr[v]);
        p[v] = z[v];
    }
    double rz = dot(n, r, z);
    double relres = 1.0;
    int32_t it = 0;
    while (it < max_iter) {
        lap_mul(n, row_ptr, col_idx, p, q);
        const double alpha = rz / dot(n, p, q);
        for (int32_t v = 0; v < n; ++v) {
            x[v] += alpha * p[v];
            r[v] -= alpha * q[v];
        }
        it += 1;
        relres = sqrt(dot(n, r, r)) / bnorm;
        if (relres <= tol) break;
        for (int32_t v = 0; v < n; ++v) z[v] = r[v] / (double)(row_ptr[v + 1] - row_ptr[v]);
        const double rz_new = dot(n, r, z);
        const double beta = rz_new / rz;
        rz = rz_new;
        for (int32_t v = 0; v < n; ++v) p[v] = z[v] + beta * p[v];
    }
    double mean = 0.0;
    for (int32_t v = 0; v < n; ++v) mean += x[v];
    mean /= (double)n;
    for (int32_t v = 0; v < n; ++v) x[v] -= mean;
    /* true residual of the projected solution */
    lap_mul(n, row_ptr, col_idx, x, q);
    double rr = 0.0;
    for (int32_t v = 0; v < n; ++v) {
        const double bv = (v == u ? 1.0 : 0.0) - inv_n;
        rr += (bv - q[v]) * (bv - q[v]);
    }
    relres = sqrt(rr) / bnorm;
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = relres;
    free(r);
    free(z);
    free(p);
    free(q);
    return relres <= tol ? 0 : 1;
}

/* Eq. (diag-comp) with the estimate R[v]/tau of r(u, v):
 * L^+[u,u] = x_u, L^+[v,v] = R[v]/tau - x_u + 2 x_v, evaluated left to right. */

ORC_EXPORT void orc_combine(int32_t n, const int64_t *R, int64_t tau, const double *x, int32_t u, double *diag)
{
    const double xu = x[u];
    for (int32_t v = 0; v < n; ++v) {
        if (v == u) {
            diag[v] = xu;
        } else {
            const double r = (double)R[v] / (double)tau;
            const double t = r - xu;
            diag[v] = t + 2.0 * x[v];
        }
    }
}

/* tau = ecc(u)^2 * ceil( ln(2m/delta) / (2 (1-kappa)^2 eps^2) ) (Algorithm 1). */

ORC_EXPORT int64_t orc_tau(int32_t ecc, int64_t m, double eps, double delta, double kappa)
{
    const double a = log(2.0 * (double)m / delta);
    const double b = 2.0 * (1.0 - kappa) * (1.0 - kappa) * eps * eps;
    return (int64_t)ecc * (int64_t)ecc * (int64_t)ceil(a / b);
}
