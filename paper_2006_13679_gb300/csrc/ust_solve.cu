// The column x = L^+[:, u] (Section 3.1 step 1, Algorithm 1) and the
// diagonal combination (Eq. diag-comp).
//
// L x = b with b = e_u - (1/n) 1 is consistent (b _|_ 1) and x is taken
// _|_ 1. The paper solves it with Jacobi-preconditioned CG (Appendix D.1).
// Here the CG recurrences and the SpMV run in FP32 on the FP32 residual of an
// outer FP64 iterative refinement:
//     r = b - L x          (FP64 SpMV, FP64 sums)
//     solve L d = r        (FP32 Jacobi-PCG, to a modest inner tolerance)
//     x = x + d            (FP64)
// until ||b - L x||_2 / ||b||_2 <= cg_tol; finally x is projected onto
// 1-perp in FP64. Dot products are reduced in a fixed order (per-block
// partials, then the same warp tree in every consumer block), so the solve
// is deterministic.
#include <math.h>

#include <algorithm>
#include <vector>

#include "ust_common.cuh"

namespace ust {
namespace {

constexpr int kRowGroup = 8;  // lanes per CSR row in the SpMVs

// Sum of `count` per-block partials at stride `stride`, identical in every
// block (fixed lane assignment and shuffle tree). Called by warp 0 only.
__device__ __forceinline__ double warp_sum_partials(const double *part, int count, int stride)
{
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = lane; i < count; i += 32) s += part[(long long)i * stride];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Block-wide sum of one value per thread (fixed shuffle tree), result valid
// in thread 0.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *s_tmp)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) s_tmp[wid] = v;
    __syncthreads();
    T r = T(0);
    if (wid == 0) {
        r = (lane < kSolveThreads / 32) ? s_tmp[lane] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

// Rows with more than kHeavyRow arcs are summed by a whole CTA each (the
// first `nh` blocks of an SpMV launch); the other blocks give every light row
// a group of kRowGroup lanes. Both reductions use a fixed order.

// r64 = b - L x64; partials of sum(r) and sum(r^2).
__global__ void __launch_bounds__(kSolveThreads) residual_f64_kernel(int n, int u, const int32_t *__restrict__ rp,
                                                                     const int32_t *__restrict__ ci,
                                                                     const int32_t *__restrict__ heavy, int nh,
                                                                     const double *__restrict__ x,
                                                                     double *__restrict__ r, double *part)
{
    __shared__ double s_tmp[kSolveThreads / 32];
    const double inv_n = 1.0 / (double)n;
    if ((int)blockIdx.x < nh) {
        const int v = heavy[blockIdx.x];
        const int e0 = __ldg(rp + v), e1 = __ldg(rp + v + 1);
        double s = 0.0;
        for (int e = e0 + threadIdx.x; e < e1; e += kSolveThreads) s += x[__ldg(ci + e)];
        s = block_sum(s, s_tmp);
        if (threadIdx.x == 0) {
            const double rv = ((v == u ? 1.0 : 0.0) - inv_n) - ((double)(e1 - e0) * x[v] - s);
            r[v] = rv;
            part[blockIdx.x * 2 + 0] = rv;
            part[blockIdx.x * 2 + 1] = rv * rv;
        }
        return;
    }
    const int g = threadIdx.x % kRowGroup;
    const int rows_per_block = kSolveThreads / kRowGroup;
    const int lb = blockIdx.x - nh, lgrid = gridDim.x - nh;
    double sr = 0.0, srr = 0.0;
    for (int v0 = lb * rows_per_block; v0 < n; v0 += lgrid * rows_per_block) {
        const int v = v0 + threadIdx.x / kRowGroup;
        double s = 0.0;
        int e0 = 0, e1 = 0;
        if (v < n) {
            e0 = __ldg(rp + v);
            e1 = __ldg(rp + v + 1);
            if (e1 - e0 > kHeavyRow) e1 = e0;  // summed by a heavy-row block
            for (int e = e0 + g; e < e1; e += kRowGroup) s += x[__ldg(ci + e)];
        }
#pragma unroll
        for (int o = kRowGroup / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, kRowGroup);
        if (v < n && g == 0 && e1 > e0) {
            const double lx = (double)(e1 - e0) * x[v] - s;
            const double bv = (v == u ? 1.0 : 0.0) - inv_n;
            const double rv = bv - lx;
            r[v] = rv;
            sr += rv;
            srr += rv * rv;
        }
    }
    sr = block_sum(sr, s_tmp);
    srr = block_sum(srr, s_tmp);
    if (threadIdx.x == 0) {
        part[blockIdx.x * 2 + 0] = sr;
        part[blockIdx.x * 2 + 1] = srr;
    }
}

// Start of an inner solve: r32 = r64 - mean(r64), d = 0, z = r32 / deg,
// p = z; partials of r.z.
template <typename T>
__global__ void __launch_bounds__(kSolveThreads) inner_start_kernel(int n, int nparts, const int32_t *__restrict__ rp,
                                                                    const double *__restrict__ r64,
                                                                    const double *__restrict__ part_in,
                                                                    T *__restrict__ r, T *__restrict__ z,
                                                                    T *__restrict__ p, T *__restrict__ d,
                                                                    double *part_out)
{
    __shared__ double s_tmp[kSolveThreads / 32];
    __shared__ double s_mean;
    if (threadIdx.x < 32) {
        const double s = warp_sum_partials(part_in, nparts, 2);
        if (threadIdx.x == 0) s_mean = s / (double)n;
    }
    __syncthreads();
    const double mean = s_mean;
    double rz = 0.0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const T rv = (T)(r64[v] - mean);
        const T zv = rv / (T)(__ldg(rp + v + 1) - __ldg(rp + v));
        r[v] = rv;
        z[v] = zv;
        p[v] = zv;
        d[v] = T(0);
        rz += (double)rv * (double)zv;
    }
    rz = block_sum(rz, s_tmp);
    if (threadIdx.x == 0) part_out[blockIdx.x] = rz;
}

// q = L p in the inner precision T; partials of p.q.
template <typename T>
__global__ void __launch_bounds__(kSolveThreads) spmv_inner_kernel(int n, const int32_t *__restrict__ rp,
                                                                   const int32_t *__restrict__ ci,
                                                                   const int32_t *__restrict__ heavy, int nh,
                                                                   const T *__restrict__ p, T *__restrict__ q,
                                                                   double *part_out)
{
    __shared__ double s_tmp[kSolveThreads / 32];
    __shared__ T s_tmpf[kSolveThreads / 32];
    if ((int)blockIdx.x < nh) {
        const int v = heavy[blockIdx.x];
        const int e0 = __ldg(rp + v), e1 = __ldg(rp + v + 1);
        T s = T(0);
        for (int e = e0 + threadIdx.x; e < e1; e += kSolveThreads) s += p[__ldg(ci + e)];
        s = block_sum(s, s_tmpf);
        if (threadIdx.x == 0) {
            const T pv = p[v];
            const T qv = (T)(e1 - e0) * pv - s;
            q[v] = qv;
            part_out[blockIdx.x] = (double)pv * (double)qv;
        }
        return;
    }
    const int g = threadIdx.x % kRowGroup;
    const int rows_per_block = kSolveThreads / kRowGroup;
    const int lb = blockIdx.x - nh, lgrid = gridDim.x - nh;
    double pq = 0.0;
    for (int v0 = lb * rows_per_block; v0 < n; v0 += lgrid * rows_per_block) {
        const int v = v0 + threadIdx.x / kRowGroup;
        T s = T(0);
        int e0 = 0, e1 = 0;
        if (v < n) {
            e0 = __ldg(rp + v);
            e1 = __ldg(rp + v + 1);
            if (e1 - e0 > kHeavyRow) e1 = e0;
            for (int e = e0 + g; e < e1; e += kRowGroup) s += p[__ldg(ci + e)];
        }
#pragma unroll
        for (int o = kRowGroup / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, kRowGroup);
        if (v < n && g == 0 && e1 > e0) {
            const T pv = p[v];
            const T qv = (T)(e1 - e0) * pv - s;
            q[v] = qv;
            pq += (double)pv * (double)qv;
        }
    }
    pq = block_sum(pq, s_tmp);
    if (threadIdx.x == 0) part_out[blockIdx.x] = pq;
}

// alpha = rz / pq; d += alpha p; r -= alpha q; z = r / deg; partials of r.z
// and r.r. rz of the current iteration is in sc[par].
template <typename T>
__global__ void __launch_bounds__(kSolveThreads) pcg_update_kernel(int n, int nparts, const int32_t *__restrict__ rp,
                                                                   const double *__restrict__ part_pq,
                                                                   const double *__restrict__ sc, int par,
                                                                   T *__restrict__ d, T *__restrict__ r,
                                                                   T *__restrict__ z, const T *__restrict__ p,
                                                                   const T *__restrict__ q, double *part_out)
{
    __shared__ double s_tmp[kSolveThreads / 32];
    __shared__ T s_alpha;
    if (threadIdx.x < 32) {
        const double pq = warp_sum_partials(part_pq, nparts, 1);
        if (threadIdx.x == 0) s_alpha = (pq > 0.0) ? (T)(sc[par] / pq) : T(0);
    }
    __syncthreads();
    const T alpha = s_alpha;
    double rz = 0.0, rr = 0.0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        d[v] += alpha * p[v];
        const T rv = r[v] - alpha * q[v];
        const T zv = rv / (T)(__ldg(rp + v + 1) - __ldg(rp + v));
        r[v] = rv;
        z[v] = zv;
        rz += (double)rv * (double)zv;
        rr += (double)rv * (double)rv;
    }
    rz = block_sum(rz, s_tmp);
    rr = block_sum(rr, s_tmp);
    if (threadIdx.x == 0) {
        part_out[blockIdx.x * 2 + 0] = rz;
        part_out[blockIdx.x * 2 + 1] = rr;
    }
}

// beta = rz_new / rz; p = z + beta p; block 0 stores rz_new in sc[par ^ 1].
template <typename T>
__global__ void __launch_bounds__(kSolveThreads) pcg_direction_kernel(int n, int nparts, const double *__restrict__ part_rz,
                                                                      double *sc, int par, const T *__restrict__ z,
                                                                      T *__restrict__ p)
{
    __shared__ T s_beta;
    if (threadIdx.x < 32) {
        const double rz_new = warp_sum_partials(part_rz, nparts, 2);
        if (threadIdx.x == 0) {
            const double rz = sc[par];
            s_beta = (rz > 0.0) ? (T)(rz_new / rz) : T(0);
            if (blockIdx.x == 0) sc[par ^ 1] = rz_new;
        }
    }
    __syncthreads();
    const T beta = s_beta;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) p[v] = z[v] + beta * p[v];
}

// sc[0] = sum of the r.z partials written by inner_start_kernel.
__global__ void store_rz_kernel(int nparts, const double *__restrict__ part, double *sc)
{
    const double s = warp_sum_partials(part, nparts, 1);
    if (threadIdx.x == 0) sc[0] = s;
}

// x64 += d (FP64).
template <typename T>
__global__ void apply_correction_kernel(int n, const T *__restrict__ d, double *__restrict__ x)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) x[v] += (double)d[v];
}

// partials of sum(x)
__global__ void __launch_bounds__(kSolveThreads) sum_kernel(int n, const double *__restrict__ x, double *part)
{
    __shared__ double s_tmp[kSolveThreads / 32];
    double s = 0.0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) s += x[v];
    s = block_sum(s, s_tmp);
    if (threadIdx.x == 0) part[blockIdx.x * 2] = s;
}

// x -= mean(x)
__global__ void project_kernel(int n, int nparts, const double *__restrict__ part, double *__restrict__ x)
{
    __shared__ double s_mean;
    if (threadIdx.x < 32) {
        const double s = warp_sum_partials(part, nparts, 2);
        if (threadIdx.x == 0) s_mean = s / (double)n;
    }
    __syncthreads();
    const double mean = s_mean;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) x[v] = x[v] - mean;
}

// Eq. (diag-comp): diag[u] = x_u, diag[v] = (R[v]/tau - x_u) + 2 x_v, with
// every operation rounded separately (no contraction), in this order.
__global__ void combine_kernel(int n, int u, double tau, const long long *__restrict__ R,
                               const double *__restrict__ x, double *__restrict__ diag)
{
    const double xu = x[u];
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (v == u) {
            diag[v] = xu;
        } else {
            const double r = __ddiv_rn((double)R[v], tau);
            const double t = __dsub_rn(r, xu);
            diag[v] = __dadd_rn(t, __dmul_rn(2.0, x[v]));
        }
    }
}

}  // namespace

int alloc_solver(Ctx *c)
{
    const size_t n = (size_t)c->n;
    c->solve_n = c->n;
    c->solve_blocks = std::max(1, std::min<int>(c->num_sms * 2, (int)((n + kSolveThreads - 1) / kSolveThreads)));
    // rows summed by a whole CTA in the SpMVs
    std::vector<int32_t> rp(n + 1), heavy;
    UST_CUDA_TRY(cudaMemcpyAsync(rp.data(), c->d_rp, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (size_t v = 0; v < n; ++v)
        if (rp[v + 1] - rp[v] > kHeavyRow) heavy.push_back((int32_t)v);
    c->n_heavy = (int)heavy.size();
    if (cudaMalloc(&c->d_heavy, std::max<size_t>(1, heavy.size()) * sizeof(int32_t)) != cudaSuccess)
        return fail(c, UST_ENOMEM, "heavy rows");
    if (!heavy.empty())
        UST_CUDA_TRY(cudaMemcpyAsync(c->d_heavy, heavy.data(), heavy.size() * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, c->stream));
    if (cudaMalloc(&c->d_tasks, sizeof(SolveTask)) != cudaSuccess) return fail(c, UST_ENOMEM, "solve task");
    if (cudaMalloc(&c->d_results, sizeof(SolveResult)) != cudaSuccess) return fail(c, UST_ENOMEM, "solve result");
    if (cudaMallocHost(&c->h_results, sizeof(SolveResult)) != cudaSuccess)
        return fail(c, UST_ENOMEM, "pinned solve result");
    const size_t parts = 8 * ((size_t)c->solve_blocks + (size_t)c->n_heavy) + 8;
    if (cudaMalloc(&c->d_f32, 5 * n * sizeof(float)) != cudaSuccess) return fail(c, UST_ENOMEM, "solver FP32 vectors");
    if (cudaMalloc(&c->d_f64, 2 * n * sizeof(double)) != cudaSuccess) return fail(c, UST_ENOMEM, "solver FP64 vectors");
    if (cudaMalloc(&c->d_x, n * sizeof(double)) != cudaSuccess) return fail(c, UST_ENOMEM, "column");
    if (cudaMalloc(&c->d_red, parts * sizeof(double)) != cudaSuccess) return fail(c, UST_ENOMEM, "solver partials");
    if (cudaMallocHost(&c->h_red, parts * sizeof(double)) != cudaSuccess)
        return fail(c, UST_ENOMEM, "pinned solver partials");
    UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return UST_OK;
}

namespace {

// One solve: FP64 residual and correction outside, Jacobi-PCG in T inside.
// T = float is the mixed-precision default; T = double runs the whole CG in
// FP64 (inner tolerance below cg_tol), the reference form of the solve.
template <typename T>
int solve_impl(Ctx *c, const SolveView &g, T *r, double inner_tol)
{
    const int n = g.n, nb = g.blocks, nh = g.n_heavy, ns = nb + nh, Tn = kSolveThreads;
    cudaStream_t st = c->stream;
    T *z = r + n, *p = z + n, *q = p + n, *d = q + n;
    double *x = g.x, *r64 = c->d_f64;
    double *part_res = c->d_red;              // 2*ns
    double *part_a = part_res + 2 * ns;       // 2*ns
    double *part_b = part_a + 2 * ns;         // 2*ns
    double *sc = part_b + 2 * ns;             // 2 scalars
    phase_begin(c, Ctx::kEvSolve);
    UST_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)n * sizeof(double), st));

    const double bnorm = sqrt(1.0 - 1.0 / (double)n);  // ||e_u - 1/n||_2
    const int check_every = 8;
    int total_inner = 0, refinements = 0;
    double relres = 1.0;
    for (;;) {
        residual_f64_kernel<<<ns, Tn, 0, st>>>(n, g.u, g.rp, g.ci, g.heavy, nh, x, r64, part_res);
        c->launches += 1;
        UST_CUDA_TRY(cudaGetLastError());
        UST_CUDA_TRY(cudaMemcpyAsync(c->h_red, part_res, 2 * ns * sizeof(double), cudaMemcpyDeviceToHost, st));
        UST_CUDA_TRY(cudaStreamSynchronize(st));
        double rr = 0.0;
        for (int i = 0; i < ns; ++i) rr += c->h_red[2 * i + 1];
        relres = sqrt(rr) / bnorm;
        if (relres <= c->cg_tol) break;
        if (refinements >= 30) break;
        ++refinements;
        inner_start_kernel<T><<<nb, Tn, 0, st>>>(n, ns, g.rp, r64, part_res, r, z, p, d, part_a);
        store_rz_kernel<<<1, 32, 0, st>>>(nb, part_a, sc);
        c->launches += 2;
        UST_CUDA_TRY(cudaGetLastError());
        UST_CUDA_TRY(cudaMemcpyAsync(c->h_red, part_a, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
        UST_CUDA_TRY(cudaStreamSynchronize(st));
        double rz0 = 0.0;
        for (int i = 0; i < nb; ++i) rz0 += c->h_red[i];
        const double r0 = rr;  // ||r||^2 at the start of the inner solve
        int it = 0, par = 0;
        bool inner_done = (rz0 <= 0.0);
        while (!inner_done && it < c->max_cg_iters) {
            for (int k = 0; k < check_every && it < c->max_cg_iters; ++k, ++it) {
                spmv_inner_kernel<T><<<ns, Tn, 0, st>>>(n, g.rp, g.ci, g.heavy, nh, p, q, part_a);
                pcg_update_kernel<T><<<nb, Tn, 0, st>>>(n, ns, g.rp, part_a, sc, par, d, r, z, p, q, part_b);
                pcg_direction_kernel<T><<<nb, Tn, 0, st>>>(n, nb, part_b, sc, par, z, p);
                c->launches += 3;
                par ^= 1;
            }
            UST_CUDA_TRY(cudaGetLastError());
            UST_CUDA_TRY(cudaMemcpyAsync(c->h_red, part_b, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, st));
            UST_CUDA_TRY(cudaStreamSynchronize(st));
            double ri = 0.0;
            for (int i = 0; i < nb; ++i) ri += c->h_red[2 * i + 1];
            if (ri <= inner_tol * inner_tol * r0) inner_done = true;
        }
        total_inner += it;
        apply_correction_kernel<T><<<nb, Tn, 0, st>>>(n, d, x);
        c->launches += 1;
        UST_CUDA_TRY(cudaGetLastError());
    }
    sum_kernel<<<nb, Tn, 0, st>>>(n, x, part_res);
    project_kernel<<<nb, Tn, 0, st>>>(n, nb, part_res, x);
    c->launches += 2;
    UST_CUDA_TRY(cudaGetLastError());
    // residual of the projected solution
    residual_f64_kernel<<<ns, Tn, 0, st>>>(n, g.u, g.rp, g.ci, g.heavy, nh, x, r64, part_res);
    c->launches += 1;
    phase_end(c, Ctx::kEvSolve);
    UST_CUDA_TRY(cudaMemcpyAsync(c->h_red, part_res, 2 * ns * sizeof(double), cudaMemcpyDeviceToHost, st));
    UST_CUDA_TRY(cudaStreamSynchronize(st));
    double rr = 0.0;
    for (int i = 0; i < ns; ++i) rr += c->h_red[2 * i + 1];
    relres = sqrt(rr) / bnorm;
    c->cg_iters = total_inner;
    c->cg_refinements = refinements;
    c->cg_relres = relres;
    if (relres > c->cg_tol) return fail(c, UST_ENOTCONVERGED, "column solve did not reach cg_tol");
    return UST_OK;
}

}  // namespace

int run_solve_view(Ctx *c, const SolveView &g)
{
    if (c->solve_fp64) {
        if (!c->d_f64inner) {
            if (cudaMalloc(&c->d_f64inner, 5 * (size_t)c->solve_n * sizeof(double)) != cudaSuccess)
                return fail(c, UST_ENOMEM, "FP64 solver vectors");
        }
        return solve_impl<double>(c, g, c->d_f64inner, 0.25 * c->cg_tol);
    }
    return solve_impl<float>(c, g, c->d_f32, 1e-4);
}

int run_solve(Ctx *c)
{
    if ((int64_t)c->nnz <= kCtaSolveMaxArcs) {
        // one CTA, one launch: the FP64 residual lives in d_f64, the inner
        // vectors in d_f32 (or d_f64inner for the all-FP64 form)
        if (c->solve_fp64 && !c->d_f64inner) {
            if (cudaMalloc(&c->d_f64inner, 5 * (size_t)c->solve_n * sizeof(double)) != cudaSuccess)
                return fail(c, UST_ENOMEM, "FP64 solver vectors");
        }
        SolveTask t;
        t.n = c->n;
        t.u = c->pivot;
        t.rp = c->d_rp;
        t.ci = c->d_ci;
        t.heavy = c->d_heavy;
        t.n_heavy = c->n_heavy;
        t.x = c->d_x;
        t.r64 = c->d_f64;
        t.w = c->solve_fp64 ? (void *)c->d_f64inner : (void *)c->d_f32;
        UST_CUDA_TRY(cudaMemcpyAsync(c->d_tasks, &t, sizeof(t), cudaMemcpyHostToDevice, c->stream));
        const int rc = run_solve_cta(c, c->d_tasks, 1, c->d_results, c->h_results, c->solve_fp64);
        if (rc == UST_OK) c->x_valid = true;
        return rc;
    }
    SolveView g;
    g.n = c->n;
    g.u = c->pivot;
    g.rp = c->d_rp;
    g.ci = c->d_ci;
    g.heavy = c->d_heavy;
    g.n_heavy = c->n_heavy;
    g.blocks = c->solve_blocks;
    g.x = c->d_x;
    const int rc = run_solve_view(c, g);
    if (rc == UST_OK) c->x_valid = true;
    return rc;
}

int run_combine(Ctx *c, int64_t tau, double *d_diag)
{
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((c->n + threads - 1) / threads, (int64_t)c->num_sms * 8);
    phase_begin(c, Ctx::kEvCombine);
    combine_kernel<<<blocks, threads, 0, c->stream>>>(c->n, c->pivot, (double)tau,
                                                       reinterpret_cast<const long long *>(c->d_R), c->d_x, d_diag);
    phase_end(c, Ctx::kEvCombine);
    c->launches += 1;
    UST_CUDA_TRY(cudaGetLastError());
    return UST_OK;
}

}  // namespace ust
