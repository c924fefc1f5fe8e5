// Centralities that depend only on diag(L^+) (Section 3.1 and the
// normalized random-walk betweenness lemma):
//   electrical farness      f(v) = n L+[v,v] + tr(L+)           (Eq. elec-farness)
//   electrical closeness    c(v) = (n - 1) / f(v)
//   random-walk betweenness b(v) = 1/n + tr(L+) / ((n - 1) f(v))  (normalized)
//   Kirchhoff index         K    = n tr(L+)
// One CTA per graph: the trace is a fixed-order FP64 sum, then every output
// is one correctly rounded FP64 operation after another.
#include "ust_common.cuh"

namespace ust {
namespace {

constexpr int kCentThreads = 256;

__global__ void __launch_bounds__(kCentThreads) centrality_kernel(const CombineDesc *__restrict__ graphs,
                                                                  CombineDesc one, const double *__restrict__ diag,
                                                                  double *closeness, double *nrwb, double *kirchhoff)
{
    __shared__ double s_part[kCentThreads / 32];
    __shared__ double s_trace;
    const CombineDesc g = graphs ? graphs[blockIdx.x] : one;
    const double *d = diag + g.voff;
    double s = 0.0;
    for (int v = threadIdx.x; v < g.n; v += kCentThreads) s += d[v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = (threadIdx.x < kCentThreads / 32) ? s_part[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) s_trace = t;
    }
    __syncthreads();
    const double trace = s_trace, n = (double)g.n, n1 = (double)(g.n - 1);
    if (threadIdx.x == 0 && kirchhoff) kirchhoff[blockIdx.x] = __dmul_rn(n, trace);
    const double inv_n = __ddiv_rn(1.0, n);
    for (int v = threadIdx.x; v < g.n; v += kCentThreads) {
        const double f = __dadd_rn(__dmul_rn(n, d[v]), trace);
        if (closeness) closeness[g.voff + v] = __ddiv_rn(n1, f);
        if (nrwb) nrwb[g.voff + v] = __dadd_rn(inv_n, __ddiv_rn(trace, __dmul_rn(n1, f)));
    }
}

}  // namespace

int run_centralities(Ctx *c, const CombineDesc *d_graphs, int count, const double *d_diag, double *d_closeness,
                     double *d_nrwb, double *d_kirchhoff)
{
    CombineDesc one;
    one.n = c->n;
    one.u = c->pivot;
    one.voff = 0;
    one.trees = c->trees;
    centrality_kernel<<<count, kCentThreads, 0, c->stream>>>(d_graphs, one, d_diag, d_closeness, d_nrwb,
                                                             d_kirchhoff);
    c->launches += 1;
    UST_CUDA_TRY(cudaGetLastError());
    return UST_OK;
}

}  // namespace ust
