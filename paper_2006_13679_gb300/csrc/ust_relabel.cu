// The large-graph sampler's view of a single graph: the vertices relabelled
// by degree.
//
// Wilson's walks and the per-tree bookkeeping (in-degrees, peeling, subtree
// sizes, the interval tests of Algorithm 2) touch vertices in proportion to
// how often a random neighbour lands on them, that is roughly in proportion
// to degree. Sampler ids below kRelabelTop go to the vertices of largest
// degree (ties: smaller input id first), in order of decreasing degree, so
// that the most used per-vertex entries sit side by side in few cache lines
// of L1 and L2; the other vertices follow in input order (measured: 5%
// faster on R-MAT scale 22 than input order).
//
// Nothing the method computes changes: row v' of the relabelled CSR lists the
// same neighbours as input row orig[v'], in the same (input) order, so draw k
// of a vertex picks the same neighbour, and the sampler keys its Philox
// counters by the input id. B_u, the column solve and every output stay in
// input ids.
#include <algorithm>
#include <numeric>
#include <vector>

#include "ust_common.cuh"

namespace ust {
namespace {

// One warp per relabelled row: sci[srp[v] + k] = newid[ci[rp[orig[v]] + k]].
__global__ void relabel_rows_kernel(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                    const int32_t *__restrict__ srp, const int32_t *__restrict__ orig,
                                    const int32_t *__restrict__ newid, int32_t *__restrict__ sci)
{
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        const int o = orig[v];
        const int src = rp[o], len = rp[o + 1] - src, dst = srp[v];
        for (int k = lane; k < len; k += 32) sci[dst + k] = newid[ci[src + k]];
    }
}

// Flattened BFS paths in sampler ids (the entry order stays the input's).
__global__ void relabel_path_kernel(long long count, const int32_t *__restrict__ path,
                                    const int32_t *__restrict__ newid, int32_t *__restrict__ spath)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x)
        spath[q] = newid[path[q]];
}

}  // namespace

int build_relabel(Ctx *c)
{
    const int n = c->n;
    std::vector<int32_t> rp((size_t)n + 1);
    UST_CUDA_TRY(cudaMemcpyAsync(rp.data(), c->d_rp, ((size_t)n + 1) * 4, cudaMemcpyDeviceToHost, c->stream));
    UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
    const int top = std::min(n, kRelabelTop);
    std::vector<int32_t> order((size_t)n);
    std::iota(order.begin(), order.end(), 0);
    const auto by_degree = [&](int32_t a, int32_t b) {
        const int32_t da = rp[a + 1] - rp[a], db = rp[b + 1] - rp[b];
        return da != db ? da > db : a < b;
    };
    if (top < n) std::nth_element(order.begin(), order.begin() + top, order.end(), by_degree);
    std::sort(order.begin(), order.begin() + top, by_degree);
    std::vector<char> is_top((size_t)n, 0);
    for (int i = 0; i < top; ++i) is_top[order[i]] = 1;
    std::vector<int32_t> orig((size_t)n), srp((size_t)n + 1);
    std::copy(order.begin(), order.begin() + top, orig.begin());
    int k = top;
    for (int v = 0; v < n; ++v)
        if (!is_top[v]) orig[k++] = v;
    c->h_newid.assign((size_t)n, 0);
    srp[0] = 0;
    for (int i = 0; i < n; ++i) {
        c->h_newid[orig[i]] = i;
        srp[i + 1] = srp[i] + (rp[orig[i] + 1] - rp[orig[i]]);
    }
    if (cudaMalloc(&c->d_srp, ((size_t)n + 1) * 4) != cudaSuccess ||
        cudaMalloc(&c->d_sci, (size_t)c->nnz * 4) != cudaSuccess || cudaMalloc(&c->d_orig, (size_t)n * 4) != cudaSuccess ||
        cudaMalloc(&c->d_newid, (size_t)n * 4) != cudaSuccess)
        return fail(c, UST_ENOMEM, "relabelled graph of the sampler");
    UST_CUDA_TRY(cudaMemcpyAsync(c->d_srp, srp.data(), ((size_t)n + 1) * 4, cudaMemcpyHostToDevice, c->stream));
    UST_CUDA_TRY(cudaMemcpyAsync(c->d_orig, orig.data(), (size_t)n * 4, cudaMemcpyHostToDevice, c->stream));
    UST_CUDA_TRY(cudaMemcpyAsync(c->d_newid, c->h_newid.data(), (size_t)n * 4, cudaMemcpyHostToDevice, c->stream));
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>(((int64_t)n * 32 + threads - 1) / threads, (int64_t)c->num_sms * 16);
    relabel_rows_kernel<<<blocks, threads, 0, c->stream>>>(n, c->d_rp, c->d_ci, c->d_srp, c->d_orig, c->d_newid,
                                                           c->d_sci);
    c->launches += 1;
    UST_CUDA_TRY(cudaGetLastError());
    // the host vectors are freed on return: finish the copies first
    UST_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->relabel = true;
    return UST_OK;
}

int relabel_paths(Ctx *c)
{
    if (!c->relabel) return UST_OK;
    if (c->farness > c->spath_cap) {
        cudaFree(c->d_spath);
        c->d_spath = nullptr;
        c->spath_cap = 0;
        if (cudaMalloc(&c->d_spath, (size_t)std::max<int64_t>(1, c->farness) * 4) != cudaSuccess)
            return fail(c, UST_ENOMEM, "BFS paths in sampler ids");
        c->spath_cap = c->farness;
    }
    if (c->farness > 0) {
        const int threads = 256;
        const int blocks = (int)std::min<int64_t>((c->farness + threads - 1) / threads, (int64_t)c->num_sms * 8);
        relabel_path_kernel<<<blocks, threads, 0, c->stream>>>(c->farness, c->d_path, c->d_newid, c->d_spath);
        c->launches += 1;
        UST_CUDA_TRY(cudaGetLastError());
    }
    c->spivot = c->h_newid[c->pivot];
    return UST_OK;
}

}  // namespace ust
