// Learned elimination-order ranker: a small MLP cost model (features of an
// elimination sequence -> predicted log time) with hand-written forward,
// backward and Adam kernels, and the planner entry points that use it.  The
// paper chooses orders by opt_einsum's greedy or dp search (Section 3.2 and
// Appendix F, Remark on the ordering); the exhaustive / min-fill planners of
// this library remain the fallback and the reference for the ranker's regret.
//
// Network: F inputs -> H (ReLU) -> H (ReLU) -> 1, float32.  Parameters are one
// array [W1 (H x F, row-major), b1 (H), W2 (H x H), b2 (H), w3 (H), b3].
// Loss: mean squared error over the rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "ustat_internal.h"

using namespace ustat;

namespace {

constexpr int kMaxHidden = 64;
constexpr int kMaxFeat = 32;

__host__ __device__ inline int param_count(int F, int H) { return H * F + H + H * H + H + H + 1; }

// One thread per row: the forward pass; with `train`, also the per-row
// backward quantities (activations and the gradients w.r.t. each layer's
// pre-activation) and the squared error.
__global__ void mlp_rows_kernel(const float *__restrict__ params, int F, int H, const float *__restrict__ X,
                                int rows, float *__restrict__ y, const float *__restrict__ target, float *h1s,
                                float *g1s, float *h2s, float *g2s, float *dys, float *loss) {
    extern __shared__ float sp[];
    const int P = param_count(F, H);
    for (int i = threadIdx.x; i < P; i += blockDim.x) sp[i] = params[i];
    __syncthreads();
    const float *W1 = sp, *b1 = W1 + H * F, *W2 = b1 + H, *b2 = W2 + H * H, *w3 = b2 + H, *b3 = w3 + H;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    float err2 = 0.f;
    if (r < rows) {
        float x[kMaxFeat], h1[kMaxHidden], h2[kMaxHidden];
        for (int f = 0; f < F; ++f) x[f] = X[(size_t)r * F + f];
        for (int h = 0; h < H; ++h) {
            float a = b1[h];
            for (int f = 0; f < F; ++f) a = fmaf(W1[h * F + f], x[f], a);
            h1[h] = a > 0.f ? a : 0.f;
        }
        float out = b3[0];
        for (int h = 0; h < H; ++h) {
            float a = b2[h];
            for (int j = 0; j < H; ++j) a = fmaf(W2[h * H + j], h1[j], a);
            h2[h] = a > 0.f ? a : 0.f;
            out = fmaf(w3[h], h2[h], out);
        }
        if (y) y[r] = out;
        if (target) {
            const float e = out - target[r];
            err2 = e * e;
            const float dy = 2.f * e / (float)rows;
            dys[r] = dy;
            float g2[kMaxHidden];
            for (int h = 0; h < H; ++h) {
                g2[h] = h2[h] > 0.f ? dy * w3[h] : 0.f;
                g2s[(size_t)r * H + h] = g2[h];
                h2s[(size_t)r * H + h] = h2[h];
                h1s[(size_t)r * H + h] = h1[h];
            }
            for (int j = 0; j < H; ++j) {
                float a = 0.f;
                for (int h = 0; h < H; ++h) a = fmaf(W2[h * H + j], g2[h], a);
                g1s[(size_t)r * H + j] = h1[j] > 0.f ? a : 0.f;
            }
        }
    }
    if (target) {
        for (int o = 16; o > 0; o >>= 1) err2 += __shfl_xor_sync(0xffffffffu, err2, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(loss, err2 / (float)rows);
    }
}

// One thread per parameter and a chunk of rows: the sum over rows of the
// parameter's gradient terms, added into grad.
__global__ void mlp_grad_kernel(int F, int H, const float *__restrict__ X, int rows, const float *__restrict__ h1s,
                                const float *__restrict__ g1s, const float *__restrict__ h2s,
                                const float *__restrict__ g2s, const float *__restrict__ dys, int chunk,
                                float *grad) {
    const int P = param_count(F, H);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int r0 = blockIdx.y * chunk, r1 = min(rows, r0 + chunk);
    float acc = 0.f;
    int q = p;
    if (q < H * F) {
        const int h = q / F, f = q % F;
        for (int r = r0; r < r1; ++r) acc = fmaf(g1s[(size_t)r * H + h], X[(size_t)r * F + f], acc);
    } else if ((q -= H * F) < H) {
        for (int r = r0; r < r1; ++r) acc += g1s[(size_t)r * H + q];
    } else if ((q -= H) < H * H) {
        const int h = q / H, j = q % H;
        for (int r = r0; r < r1; ++r) acc = fmaf(g2s[(size_t)r * H + h], h1s[(size_t)r * H + j], acc);
    } else if ((q -= H * H) < H) {
        for (int r = r0; r < r1; ++r) acc += g2s[(size_t)r * H + q];
    } else if ((q -= H) < H) {
        for (int r = r0; r < r1; ++r) acc = fmaf(dys[r], h2s[(size_t)r * H + q], acc);
    } else {
        for (int r = r0; r < r1; ++r) acc += dys[r];
    }
    atomicAdd(grad + p, acc);
}

// Adam (Kingma and Ba): c1 = 1 - beta1^t and c2 = 1 - beta2^t come from the host.
__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int count, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    p[i] -= lr * mh / (sqrtf(vh) + eps);
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

size_t train_ws_bytes(int H, int rows) {
    return 4 * align256(sizeof(float) * (size_t)rows * H) + align256(sizeof(float) * (size_t)rows);
}

bool shape_ok(int F, int H) { return F >= 1 && F <= kMaxFeat && H >= 1 && H <= kMaxHidden; }

// candidates of every partition (part < 0) or of partition `part` only
int collect(const ustat_graph *g, const ustat_options *o, int64_t n, std::vector<std::vector<Candidate>> &cands,
            int part = -1, bool finest_only = false, const std::vector<int> *feature_order = nullptr) {
    Plan tmp;
    PlanRequest req;
    req.collect = &cands;
    req.collect_part = part;
    req.collect_only = part >= 0;
    req.finest_only = finest_only;
    req.feature_order = feature_order;
    req.n = n;
    return build_plan(g, o, &tmp, &req);
}

const int kBell[kMaxM + 1] = {1, 1, 2, 5, 15, 52, 203, 877};

}  // namespace

extern "C" {

int ustat_mlp_param_count(int features, int hidden) {
    if (!shape_ok(features, hidden)) return USTAT_ERR_INVALID_ARG;
    return param_count(features, hidden);
}

int ustat_mlp_workspace_bytes(int features, int hidden, int rows, size_t *bytes) {
    if (!shape_ok(features, hidden) || rows < 1 || !bytes) return USTAT_ERR_INVALID_ARG;
    *bytes = train_ws_bytes(hidden, rows);
    return USTAT_OK;
}

int ustat_mlp_forward(const float *params, int features, int hidden, const float *X, int rows, float *y,
                      void *stream) {
    if (!params || !X || !y || rows < 0 || !shape_ok(features, hidden)) return USTAT_ERR_INVALID_ARG;
    if (rows == 0) return USTAT_OK;
    const int smem = sizeof(float) * param_count(features, hidden);
    mlp_rows_kernel<<<(rows + 127) / 128, 128, smem, (cudaStream_t)stream>>>(
        params, features, hidden, X, rows, y, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? USTAT_OK : record_cuda_error(e);
}

int ustat_mlp_loss_grad(const float *params, int features, int hidden, const float *X, const float *target,
                        int rows, void *ws, size_t ws_bytes, float *grad, float *loss, void *stream) {
    if (!params || !X || !target || !grad || !loss || rows < 1 || !shape_ok(features, hidden))
        return USTAT_ERR_INVALID_ARG;
    const int H = hidden, F = features;
    if (!ws || ws_bytes < train_ws_bytes(H, rows) || ((uintptr_t)ws % 256) != 0) return USTAT_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;
    const size_t act = align256(sizeof(float) * (size_t)rows * H);
    float *h1s = (float *)w, *g1s = (float *)(w + act), *h2s = (float *)(w + 2 * act), *g2s = (float *)(w + 3 * act);
    float *dys = (float *)(w + 4 * act);
    const int P = param_count(F, H);
    cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * P, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e != cudaSuccess) return record_cuda_error(e);
    mlp_rows_kernel<<<(rows + 127) / 128, 128, sizeof(float) * P, st>>>(params, F, H, X, rows, nullptr, target, h1s,
                                                                          g1s, h2s, g2s, dys, loss);
    const int chunk = 256;
    dim3 grid((P + 127) / 128, (rows + chunk - 1) / chunk);
    mlp_grad_kernel<<<grid, 128, 0, st>>>(F, H, X, rows, h1s, g1s, h2s, g2s, dys, chunk, grad);
    e = cudaGetLastError();
    return e == cudaSuccess ? USTAT_OK : record_cuda_error(e);
}

int ustat_mlp_adam(float *params, const float *grad, float *m, float *v, int count, float lr, float beta1,
                   float beta2, float eps, int step, void *stream) {
    if (!params || !grad || !m || !v || count < 1 || step < 1) return USTAT_ERR_INVALID_ARG;
    double c1 = 1.0, c2 = 1.0;
    for (int i = 0; i < step; ++i) {
        c1 *= beta1;
        c2 *= beta2;
    }
    adam_kernel<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, count, lr, beta1, beta2,
                                                                        eps, (float)(1.0 - c1), (float)(1.0 - c2));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? USTAT_OK : record_cuda_error(e);
}

int ustat_order_candidates(const ustat_graph *graph, const ustat_options *opts, int64_t n, int part, int max_cand,
                           int *count, int *orders, float *features) {
    if (!graph || !opts || !count || n < 1 || max_cand < 0) return USTAT_ERR_INVALID_ARG;
    if (graph->m < 1 || graph->m > kMaxM) return graph->m > kMaxM ? USTAT_ERR_UNSUPPORTED : USTAT_ERR_INVALID_ARG;
    const bool finest = part < 0;
    if (finest) part = kBell[graph->m] - 1;   // the finest partition is last in RGS order
    if (part >= kBell[graph->m]) return USTAT_ERR_INVALID_ARG;
    std::vector<std::vector<Candidate>> cands;
    int rc = collect(graph, opts, n, cands, part, finest);
    if (rc != USTAT_OK) return rc;
    const auto &cv = cands[part];
    *count = (int)cv.size();
    for (int i = 0; i < (int)cv.size() && i < max_cand; ++i) {
        const int k = (int)cv[i].order.size();
        if (orders)
            for (int q = 0; q < graph->m; ++q) orders[(size_t)i * graph->m + q] = q < k ? cv[i].order[q] : -1;
        if (features)
            for (int f = 0; f < kRankFeatures; ++f) features[(size_t)i * kRankFeatures + f] = cv[i].feat[f];
    }
    return USTAT_OK;
}

int ustat_order_features(const ustat_graph *graph, const ustat_options *opts, int64_t n, int part,
                         const int *order, float *features) {
    if (!graph || !opts || !order || !features || n < 1) return USTAT_ERR_INVALID_ARG;
    if (graph->m < 1 || graph->m > kMaxM) return graph->m > kMaxM ? USTAT_ERR_UNSUPPORTED : USTAT_ERR_INVALID_ARG;
    const bool finest = part < 0;
    if (finest) part = kBell[graph->m] - 1;
    if (part >= kBell[graph->m]) return USTAT_ERR_INVALID_ARG;
    // the order names the partition's blocks: as many entries as blocks
    std::vector<std::vector<Candidate>> cands;
    int k = 0;
    {
        std::vector<int> probe;
        for (int q = 0; q < graph->m && order[q] >= 0; ++q) probe.push_back(order[q]);
        k = (int)probe.size();
        int rc = collect(graph, opts, n, cands, part, finest, &probe);
        if (rc != USTAT_OK) return rc;
    }
    if (cands.size() <= (size_t)part || cands[part].empty()) return USTAT_ERR_INVALID_ARG;
    for (int f = 0; f < kRankFeatures; ++f) features[f] = cands[part][0].feat[f];
    (void)k;
    return USTAT_OK;
}

int ustat_plan_orders(const ustat_plan_t *plan, int *orders) {
    if (!plan || !orders) return USTAT_ERR_INVALID_ARG;
    const Plan &P = plan->p;
    for (size_t i = 0; i < P.parts.size(); ++i)
        for (int q = 0; q < P.m; ++q) orders[i * P.m + q] = P.parts[i].order[q];
    return USTAT_OK;
}

int ustat_plan_contraction(const ustat_graph *graph, const ustat_options *opts, const int *order,
                           ustat_plan_t **out) {
    if (!graph || !opts || !out) return USTAT_ERR_INVALID_ARG;
    ustat_plan_t *p = new (std::nothrow) ustat_plan_t();
    if (!p) return USTAT_ERR_INVALID_ARG;
    std::vector<std::vector<int>> forced;
    PlanRequest req;
    req.finest_only = true;
    if (order) {
        std::vector<std::vector<int>> parts;
        // one entry per partition; only the finest (last) carries the order
        if (graph->m < 1 || graph->m > kMaxM) {
            delete p;
            return graph->m > kMaxM ? USTAT_ERR_UNSUPPORTED : USTAT_ERR_INVALID_ARG;
        }
        forced.assign((size_t)kBell[graph->m], {});
        forced.back().assign(order, order + graph->m);
        req.forced = &forced;
    }
    int rc = build_plan(graph, opts, &p->p, &req);
    if (rc != USTAT_OK) {
        delete p;
        return rc;
    }
    *out = p;
    return USTAT_OK;
}

int ustat_rank_workspace_bytes(const ustat_graph *graph, const ustat_options *opts, size_t *bytes) {
    if (!graph || !opts || !bytes) return USTAT_ERR_INVALID_ARG;
    std::vector<std::vector<Candidate>> cands;
    int rc = collect(graph, opts, 1024, cands);
    if (rc != USTAT_OK) return rc;
    size_t rows = 0;
    for (auto &c : cands) rows += c.size();
    *bytes = align256(sizeof(float) * rows * kRankFeatures) + align256(sizeof(float) * (rows ? rows : 1));
    return USTAT_OK;
}

int ustat_plan_learned(const ustat_graph *graph, const ustat_options *opts, int64_t n, const float *params,
                       int hidden, void *ws, size_t ws_bytes, void *stream, ustat_plan_t **out) {
    if (!graph || !opts || !params || !out || n < 1 || !shape_ok(kRankFeatures, hidden))
        return USTAT_ERR_INVALID_ARG;
    std::vector<std::vector<Candidate>> cands;
    int rc = collect(graph, opts, n, cands);
    if (rc != USTAT_OK) return rc;
    std::vector<float> feat;
    for (auto &cv : cands)
        for (auto &c : cv) feat.insert(feat.end(), c.feat, c.feat + kRankFeatures);
    const size_t rows = feat.size() / kRankFeatures;
    const size_t fbytes = align256(sizeof(float) * feat.size());
    if (!ws || ((uintptr_t)ws % 256) != 0 || ws_bytes < fbytes + align256(sizeof(float) * (rows ? rows : 1)))
        return USTAT_ERR_WORKSPACE;
    std::vector<float> score(rows, 0.f);
    if (rows) {
        cudaStream_t st = (cudaStream_t)stream;
        float *dX = (float *)ws, *dy = (float *)((char *)ws + fbytes);
        cudaError_t e = cudaMemcpyAsync(dX, feat.data(), sizeof(float) * feat.size(), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return record_cuda_error(e);
        rc = ustat_mlp_forward(params, kRankFeatures, hidden, dX, (int)rows, dy, stream);
        if (rc != USTAT_OK) return rc;
        e = cudaMemcpyAsync(score.data(), dy, sizeof(float) * rows, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return record_cuda_error(e);
    }
    // per partition: the candidate of least predicted time (the first on ties)
    std::vector<std::vector<int>> forced(cands.size());
    size_t r = 0;
    for (size_t pi = 0; pi < cands.size(); ++pi) {
        int best = -1;
        for (size_t c = 0; c < cands[pi].size(); ++c, ++r)
            if (best < 0 || score[r] < score[r - c + best]) best = (int)c;
        if (best >= 0) forced[pi] = cands[pi][best].order;
    }
    ustat_plan_t *p = new (std::nothrow) ustat_plan_t();
    if (!p) return USTAT_ERR_INVALID_ARG;
    PlanRequest req;
    req.forced = &forced;
    rc = build_plan(graph, opts, &p->p, &req);
    if (rc != USTAT_OK) {
        delete p;
        return rc;
    }
    *out = p;
    return USTAT_OK;
}

}  // extern "C"
