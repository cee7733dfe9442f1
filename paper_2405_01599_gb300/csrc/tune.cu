// Run-time auto-tuning (Sec. 3.1, 3.2): exhaustive before-execution timing of
// the SpMV candidates, and the restart-frequency judgement (Eq. 1, Fig. 2).
#include "common.cuh"

#include <cmath>
#include <vector>

namespace {

struct Cand {
    int variant, block, ipt;
};

std::vector<Cand> candidates(const xb_plan *p) {
    std::vector<Cand> c;
    if (p->sym) {
        for (int b : {128, 256, 512}) c.push_back({XB_VAR_SYM_ATOMIC, b, 1});
        for (int b : {128, 256, 512})
            for (int i : {4, 8, 16}) c.push_back({XB_VAR_SYM_TILE, b, i});
        // S3 partial vectors (skipped when a tile reaches too many granules)
        // and S1 with warp-aggregated atomics
        for (int b : {128, 256, 512})
            for (int i : {4, 8}) c.push_back({XB_VAR_SYM_PART, b, i});
        for (int b : {128, 256, 512}) c.push_back({XB_VAR_SYM_WAGG, b, 1});
        return c;
    }
    for (int b : {64, 128, 256, 512}) c.push_back({XB_VAR_ROW, b, 1});
    for (int b : {128, 256, 512})
        for (int i : {4, 8, 16}) c.push_back({XB_VAR_NNZ, b, i});
    for (int b : {128, 256})
        for (int i : {4, 8, 16, 32}) c.push_back({XB_VAR_SEGSCAN, b, i});
    // format conversion (Sec. 5): SELL-32-sigma, sigma = 32 (no reordering
    // across slices) or 1024 rows; skipped when its padding is too large
    for (int b : {128, 256, 512})
        for (int i : {1, 32}) c.push_back({XB_VAR_SELL, b, i});
    // format conversion: block CRS with 2x2, 3x3, 4x4 blocks (the block-size
    // AT); skipped when the zero fill is too large
    for (int b : {128, 256})
        for (int i : {2, 3, 4}) c.push_back({XB_VAR_BCSR, b, i});
    return c;
}

__global__ void k_ones(int n, double *x) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = 1.0;
}

// Time every candidate: one warm-up (which also builds the candidate's
// partition), then at most 4 timed runs with CUDA events; keep the minimum.
// Candidates whose launch shape does not fit are skipped.
int sweep(xb_plan *p, std::vector<xb_choice> &res, cudaStream_t s) {
    const int n = p->n;
    res.clear();
    if (n == 0) return XB_OK;
    double *x = nullptr, *y = nullptr;
    XB_CUDA(cudaMalloc(&x, (size_t)n * sizeof(double)));
    cudaError_t e = cudaMalloc(&y, (size_t)n * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(x);
        return xb::cuda_error(e, "tune: cudaMalloc");
    }
    k_ones<<<(n + 255) / 256, 256, 0, s>>>(n, x);
    int rc = XB_OK;
    for (const Cand &c : candidates(p)) {
        int r = xb::spmv_launch(p, c.variant, c.block, c.ipt, 1.0, x, 0.0, y, s);
        if (r == XB_EINVAL) continue;
        if (r != XB_OK) {
            rc = r;
            break;
        }
        float cmin = INFINITY;
        for (int rep = 0; rep < 4 && r == XB_OK; rep++) {
            cudaEventRecord(p->ev[0], s);
            r = xb::spmv_launch(p, c.variant, c.block, c.ipt, 1.0, x, 0.0, y, s);
            cudaEventRecord(p->ev[1], s);
            if (r != XB_OK) break;
            e = cudaEventSynchronize(p->ev[1]);
            if (e != cudaSuccess) {
                r = xb::cuda_error(e, "tune: event");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p->ev[0], p->ev[1]);
            cmin = std::min(cmin, ms);
        }
        if (r != XB_OK) {
            rc = r;
            break;
        }
        res.push_back(xb_choice{c.variant, c.block, c.ipt, cmin});
    }
    cudaStreamSynchronize(s);
    cudaFree(x);
    cudaFree(y);
    return rc;
}

}  // namespace

extern "C" {

int xb_tune_exhaustive(xb_plan *p, xb_choice *out, void *stream) {
    if (!p) return xb::set_error(XB_EINVAL, "tune: NULL plan");
    std::vector<xb_choice> res;
    XB_TRY(sweep(p, res, (cudaStream_t)stream));
    if (!res.empty()) {
        // minimum time; ties keep the earlier candidate (ROW < NNZ < SEGSCAN)
        const xb_choice *best = &res[0];
        for (const auto &c : res)
            if (c.ms < best->ms) best = &c;
        p->variant = best->variant;
        p->block = best->block;
        p->ipt = best->ipt;
        p->tuned_ms = best->ms;
    }
    // the sweep built a BSS data format copy per ipt tried: keep the chosen one
    xb::bss_trim(p, p->variant == XB_VAR_SEGSCAN ? p->ipt : 0);
    if (out) xb_plan_get_choice(p, out);
    return XB_OK;
}

int xb_tune_sweep(xb_plan *p, xb_choice *out, int32_t cap, int32_t *count, void *stream) {
    if (!p || !count || cap < 0 || (cap > 0 && !out)) return xb::set_error(XB_EINVAL, "tune_sweep: bad argument");
    std::vector<xb_choice> res;
    XB_TRY(sweep(p, res, (cudaStream_t)stream));
    xb::bss_trim(p, p->variant == XB_VAR_SEGSCAN ? p->ipt : 0);
    *count = (int32_t)res.size();
    for (int i = 0; i < (int)res.size() && i < cap; i++) out[i] = res[i];
    return XB_OK;
}

// Classes of the learned tuner's heads (variant, CTA size, items per thread,
// restart length).
static const int kBlocks[4] = {64, 128, 256, 512};
static const int kIpts[5] = {1, 4, 8, 16, 32};
static const int kRestarts[6] = {10, 20, 30, 50, 80, 120};

int xb_tune_mlp(xb_plan *p, const xb_csr *A, xb_mlp *model, xb_choice *out, int32_t *m_out,
                void *stream) {
    if (!p || !A || !model) return xb::set_error(XB_EINVAL, "tune_mlp: NULL argument");
    if (xb_mlp_param_count(model) <= 0) return xb::set_error(XB_EINVAL, "tune_mlp: bad model");
    cudaStream_t s = (cudaStream_t)stream;
    float feat[8];
    XB_TRY(xb_features(A, nullptr, feat, stream));
    float *d_x = nullptr, *d_l = nullptr;
    XB_CUDA(cudaMalloc(&d_x, 8 * sizeof(float)));
    cudaError_t e = cudaMalloc(&d_l, 64 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_x, feat, sizeof feat, cudaMemcpyHostToDevice, s);
    int r = XB_OK;
    if (e == cudaSuccess) r = xb_mlp_forward(model, d_x, 1, d_l, stream);
    float lg[64] = {0};
    if (e == cudaSuccess && r == XB_OK) e = cudaMemcpyAsync(lg, d_l, sizeof lg, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_x);
    cudaFree(d_l);
    if (r != XB_OK) return r;
    if (e != cudaSuccess) return xb::cuda_error(e, "tune_mlp");
    // masked argmax per head: the variant must fit the storage, the launch
    // shape must be one the variant supports
    auto amax = [&](int off, int K, auto ok) {
        int best = -1;
        for (int c = 0; c < K; c++)
            if (ok(c) && (best < 0 || lg[off + c] > lg[off + best])) best = c;
        return best;
    };
    const int v = amax(0, 5, [&](int c) { return xb::variant_fits(p, c); });
    const bool one_ipt = (v == XB_VAR_ROW || v == XB_VAR_SYM_ATOMIC);
    const int b = amax(5, 4, [&](int c) { return !(v == XB_VAR_SEGSCAN && kBlocks[c] > 256); });
    const int i = amax(9, 5, [&](int c) {
        if (one_ipt) return c == 0;
        if (v == XB_VAR_SEGSCAN) return c >= 1;
        return c >= 1 && c <= 3;
    });
    const int mm = amax(14, 6, [](int) { return true; });
    XB_TRY(xb_plan_set_choice(p, v, kBlocks[b], kIpts[i]));
    if (out) xb_plan_get_choice(p, out);
    if (m_out) *m_out = kRestarts[mm];
    return XB_OK;
}

double xb_mm_ratio(const double *r, int32_t s, int32_t t) {
    if (!r || t < 1 || s < t) return NAN;
    double mx = r[s - t], mn = r[s - t];
    for (int z = s - t + 1; z <= s; z++) {
        mx = std::max(mx, r[z - 1]);
        mn = std::min(mn, r[z - 1]);
    }
    return mn == 0.0 ? INFINITY : mx / mn;
}

int xb_dafrt(int32_t I, const double *samp, double theta) {
    return xb_mm_ratio(samp, I, I) < theta ? 1 : 0;
}

}  // extern "C"
