// The column solve x = L^+[:, u] (Section 3.1 step 1, Algorithm 1) run by one
// CTA per linear system, start to finish in one launch: the FP64 residual
// r = b - L x (b = e_u - 1/n), the inner Jacobi-PCG (Appendix D.1) in T on
// L d = r, the FP64 correction x += d, repeated until
// ||b - L x||_2 / ||b||_2 <= tol, then the projection of x onto 1-perp.
//
// Small systems are bound by launch latency and host round trips, not by
// bandwidth: this form has neither. A batch solves every graph's column in
// one launch, one CTA per graph. The FP64 residual sums run in FP64, the
// inner dot products in the inner precision; every reduction has a fixed
// order, so the result does not depend on timing.
#include <math.h>

#include <vector>

#include "ust_common.cuh"

namespace ust {
namespace {

constexpr int kCtaThreads = 1024;

// Sum of two values over the CTA; every thread gets the same result. Lanes
// and warps are added in A (the caller's precision), the 32 warp partials in
// FP64 by warp 0 alone: FP64 arithmetic is scarce on this GPU, so no path
// spends it per thread. The order is fixed, so the sum is deterministic.
static_assert(kCtaThreads == 1024, "one warp partial per lane of warp 0");
template <typename A>
__device__ __forceinline__ void cta_sum2(A &a, A &b, double2 *s_tmp, double2 *s_res)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) s_tmp[wid] = make_double2((double)a, (double)b);
    __syncthreads();
    if (wid == 0) {
        double x = s_tmp[lane].x, y = s_tmp[lane].y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
        }
        if (lane == 0) *s_res = make_double2(x, y);
    }
    __syncthreads();
    a = (A)s_res->x;
    b = (A)s_res->y;
}

// y = L v restricted to the light rows (thread per row) and the heavy rows
// (warp per row, lanes split the arcs); returns this thread's share of v.y.
template <typename V>
__device__ __forceinline__ V spmv_rows(const SolveTask &g, const V *__restrict__ v, V *__restrict__ y)
{
    V vy = V(0);
    for (int r = threadIdx.x; r < g.n; r += kCtaThreads) {
        const int e0 = __ldg(g.rp + r), e1 = __ldg(g.rp + r + 1);
        if (e1 - e0 > kHeavyRow) continue;
        V s = V(0);
        for (int e = e0; e < e1; ++e) s += v[__ldg(g.ci + e)];
        const V yr = (V)(e1 - e0) * v[r] - s;
        y[r] = yr;
        vy += v[r] * yr;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int h = wid; h < g.n_heavy; h += kCtaThreads / 32) {
        const int r = __ldg(g.heavy + h);
        const int e0 = __ldg(g.rp + r), e1 = __ldg(g.rp + r + 1);
        V s = V(0);
        for (int e = e0 + lane; e < e1; e += 32) s += v[__ldg(g.ci + e)];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const V yr = (V)(e1 - e0) * v[r] - s;
            y[r] = yr;
            vy += v[r] * yr;
        }
    }
    return vy;
}

// r64 = b - L x; returns this thread's shares of sum(r) and sum(r^2).
__device__ __forceinline__ void residual(const SolveTask &g, double &sr, double &srr)
{
    const double inv_n = 1.0 / (double)g.n;
    double *r64 = g.r64;
    spmv_rows<double>(g, g.x, r64);  // r64 = L x
    __syncthreads();
    sr = 0.0;
    srr = 0.0;
    for (int r = threadIdx.x; r < g.n; r += kCtaThreads) {
        const double rv = ((r == g.u ? 1.0 : 0.0) - inv_n) - r64[r];
        r64[r] = rv;
        sr += rv;
        srr += rv * rv;
    }
}

template <typename T>
__global__ void __launch_bounds__(kCtaThreads) solve_cta_kernel(const SolveTask *__restrict__ tasks, double tol,
                                                                double inner_tol, int max_iters, int max_ref,
                                                                SolveResult *__restrict__ results)
{
    __shared__ double2 s_tmp[kCtaThreads / 32];
    __shared__ double2 s_res;
    const SolveTask g = tasks[blockIdx.x];
    const int n = g.n;
    T *r = reinterpret_cast<T *>(g.w), *z = r + n, *p = z + n, *q = p + n, *d = q + n;
    double *x = g.x;
    for (int v = threadIdx.x; v < n; v += kCtaThreads) x[v] = 0.0;
    __syncthreads();
    const double bnorm = sqrt(1.0 - 1.0 / (double)n);
    int total = 0, refinements = 0;
    double relres = 1.0;
    for (;;) {
        double sr, srr;
        residual(g, sr, srr);
        cta_sum2(sr, srr, s_tmp, &s_res);
        relres = sqrt(srr) / bnorm;
        if (relres <= tol || refinements >= max_ref) break;
        ++refinements;
        // inner solve of L d = r (r with its mean removed), from d = 0
        const double mean = sr / (double)n;
        T rz = T(0), rr = T(0);
        for (int v = threadIdx.x; v < n; v += kCtaThreads) {
            const T rv = (T)(g.r64[v] - mean);
            const int deg = __ldg(g.rp + v + 1) - __ldg(g.rp + v);
            const T zv = rv / (T)deg;
            r[v] = rv;
            z[v] = zv;
            p[v] = zv;
            d[v] = T(0);
            rz += rv * zv;
            rr += rv * rv;
        }
        cta_sum2(rz, rr, s_tmp, &s_res);
        const T r0 = rr;
        const T stop = (T)(inner_tol * inner_tol) * r0;
        int it = 0;
        while (rz > T(0) && it < max_iters) {
            T pq = spmv_rows<T>(g, p, q), unused = T(0);
            cta_sum2(pq, unused, s_tmp, &s_res);
            if (!(pq > T(0))) break;
            const T alpha = rz / pq;
            T rz1 = T(0), rr1 = T(0);
            for (int v = threadIdx.x; v < n; v += kCtaThreads) {
                const int deg = __ldg(g.rp + v + 1) - __ldg(g.rp + v);
                d[v] += alpha * p[v];
                const T rv = r[v] - alpha * q[v];
                const T zv = rv / (T)deg;
                r[v] = rv;
                z[v] = zv;
                rz1 += rv * zv;
                rr1 += rv * rv;
            }
            cta_sum2(rz1, rr1, s_tmp, &s_res);
            ++it;
            if (rr1 <= stop) break;
            const T beta = rz1 / rz;
            rz = rz1;
            for (int v = threadIdx.x; v < n; v += kCtaThreads) p[v] = z[v] + beta * p[v];
            __syncthreads();
        }
        total += it;
        for (int v = threadIdx.x; v < n; v += kCtaThreads) x[v] += (double)d[v];
        __syncthreads();
    }
    // projection onto 1-perp, then the residual of the projected column
    double s = 0.0, unused = 0.0;
    for (int v = threadIdx.x; v < n; v += kCtaThreads) s += x[v];
    cta_sum2(s, unused, s_tmp, &s_res);
    const double mean = s / (double)n;
    for (int v = threadIdx.x; v < n; v += kCtaThreads) x[v] -= mean;
    __syncthreads();
    double sr, srr;
    residual(g, sr, srr);
    cta_sum2(sr, srr, s_tmp, &s_res);
    if (threadIdx.x == 0) {
        SolveResult out;
        out.iters = total;
        out.refinements = refinements;
        out.relres = sqrt(srr) / bnorm;
        results[blockIdx.x] = out;
    }
}

}  // namespace

int run_solve_cta(Ctx *c, const SolveTask *d_tasks, int count, SolveResult *d_results, SolveResult *h_results,
                  bool fp64)
{
    const double inner_tol = fp64 ? 0.25 * c->cg_tol : 1e-4;
    phase_begin(c, Ctx::kEvSolve);
    if (fp64)
        solve_cta_kernel<double><<<count, kCtaThreads, 0, c->stream>>>(d_tasks, c->cg_tol, inner_tol, c->max_cg_iters,
                                                                        30, d_results);
    else
        solve_cta_kernel<float><<<count, kCtaThreads, 0, c->stream>>>(d_tasks, c->cg_tol, inner_tol, c->max_cg_iters,
                                                                       30, d_results);
    phase_end(c, Ctx::kEvSolve);
    c->launches += 1;
    UST_CUDA_TRY(cudaGetLastError());
    UST_CUDA_TRY(cudaMemcpyAsync(h_results, d_results, (size_t)count * sizeof(SolveResult), cudaMemcpyDeviceToHost,
                                 c->stream));
    UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
    int iters = 0, refinements = 0;
    double worst = 0.0;
    for (int i = 0; i < count; ++i) {
        iters += h_results[i].iters;
        refinements = std::max(refinements, h_results[i].refinements);
        worst = std::max(worst, h_results[i].relres);
    }
    c->cg_iters = iters;
    c->cg_refinements = refinements;
    c->cg_relres = worst;
    if (!(worst <= c->cg_tol)) return fail(c, UST_ENOTCONVERGED, "column solve did not reach cg_tol");
    return UST_OK;
}

}  // namespace ust
