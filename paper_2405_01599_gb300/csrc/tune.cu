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
        return c;
    }
    for (int b : {64, 128, 256, 512}) c.push_back({XB_VAR_ROW, b, 1});
    for (int b : {128, 256, 512})
        for (int i : {4, 8, 16}) c.push_back({XB_VAR_NNZ, b, i});
    for (int b : {128, 256})
        for (int i : {4, 8, 16, 32}) c.push_back({XB_VAR_SEGSCAN, b, i});
    return c;
}

__global__ void k_ones(int n, double *x) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = 1.0;
}

}  // namespace

extern "C" {

int xb_tune_exhaustive(xb_plan *p, xb_choice *out, void *stream) {
    if (!p) return xb::set_error(XB_EINVAL, "tune: NULL plan");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = p->n;
    if (n == 0) {
        if (out) xb_plan_get_choice(p, out);
        return XB_OK;
    }
    double *x = nullptr, *y = nullptr;
    XB_CUDA(cudaMalloc(&x, (size_t)n * sizeof(double)));
    cudaError_t e = cudaMalloc(&y, (size_t)n * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(x);
        return xb::cuda_error(e, "tune: cudaMalloc");
    }
    k_ones<<<(n + 255) / 256, 256, 0, s>>>(n, x);
    Cand best = {p->variant, p->block, p->ipt};
    float best_ms = INFINITY;
    int rc = XB_OK;
    for (const Cand &c : candidates(p)) {
        // one warm-up (also builds the candidate's partition), then <= 4 timed runs
        int r = xb::spmv_launch(p, c.variant, c.block, c.ipt, 1.0, x, 0.0, y, s);
        if (r == XB_EINVAL) continue;  // shape does not fit (shared memory)
        if (r != XB_OK) {
            rc = r;
            break;
        }
        float cmin = INFINITY;
        for (int rep = 0; rep < 4; rep++) {
            cudaEventRecord(p->ev[0], s);
            r = xb::spmv_launch(p, c.variant, c.block, c.ipt, 1.0, x, 0.0, y, s);
            cudaEventRecord(p->ev[1], s);
            if (r != XB_OK) break;
            if (cudaEventSynchronize(p->ev[1]) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p->ev[0], p->ev[1]);
            cmin = std::min(cmin, ms);
        }
        if (r != XB_OK) {
            rc = r;
            break;
        }
        if (cmin < best_ms) {
            best_ms = cmin;
            best = c;
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(x);
    cudaFree(y);
    if (rc != XB_OK) return rc;
    p->variant = best.variant;
    p->block = best.block;
    p->ipt = best.ipt;
    p->tuned_ms = best_ms;
    if (out) xb_plan_get_choice(p, out);
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
