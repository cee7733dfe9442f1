// C-ABI entry points for SpMV and the Krylov vector operations.
#include "krylov.cuh"

#include <cmath>
#include <cstring>

namespace {

int need_plan(const xb_plan *p, const void *x, const void *y) {
    if (!p) return xb::set_error(XB_EINVAL, "NULL plan");
    if (p->n > 0 && (!x || !y)) return xb::set_error(XB_EINVAL, "NULL vector");
    if (x == y && p->n > 0) return xb::set_error(XB_EINVAL, "x and y must not alias");
    return XB_OK;
}

// Launch shape for a named variant: the plan's tuned shape when the plan's
// choice is that variant, else the default 256 threads x 8 items.
void shape_for(const xb_plan *p, int variant, int *block, int *ipt) {
    if (p->variant == variant) {
        *block = p->block;
        *ipt = p->ipt;
    } else {
        *block = 256;
        *ipt = 8;
    }
}

}  // namespace

extern "C" {

int spmv_crs(xb_plan *p, double alpha, const double *x, double beta, double *y, void *stream) {
    XB_TRY(need_plan(p, x, y));
    if (p->sym) return xb::set_error(XB_EINVAL, "spmv_crs: plan holds symmetric upper storage");
    int b, i;
    shape_for(p, XB_VAR_NNZ, &b, &i);
    return xb::spmv_launch(p, XB_VAR_NNZ, b, i, alpha, x, beta, y, (cudaStream_t)stream);
}

int spmv_sym(xb_plan *p, double alpha, const double *x, double beta, double *y, void *stream) {
    XB_TRY(need_plan(p, x, y));
    if (!p->sym) return xb::set_error(XB_EINVAL, "spmv_sym: plan is not symmetric upper storage");
    const int v = xb::variant_fits(p, p->variant) ? p->variant : XB_VAR_SYM_TILE;
    int b, i;
    shape_for(p, v, &b, &i);
    return xb::spmv_launch(p, v, b, i, alpha, x, beta, y, (cudaStream_t)stream);
}

int spmv_segscan(xb_plan *p, double alpha, const double *x, double beta, double *y, void *stream) {
    XB_TRY(need_plan(p, x, y));
    if (p->sym) return xb::set_error(XB_EINVAL, "spmv_segscan: plan holds symmetric upper storage");
    int b, i;
    shape_for(p, XB_VAR_SEGSCAN, &b, &i);
    return xb::spmv_launch(p, XB_VAR_SEGSCAN, b, i, alpha, x, beta, y, (cudaStream_t)stream);
}

int xb_spmv(xb_plan *p, int32_t variant, int32_t block, int32_t ipt, double alpha, const double *x,
            double beta, double *y, void *stream) {
    XB_TRY(need_plan(p, x, y));
    return xb::spmv_launch(p, variant, block, ipt, alpha, x, beta, y, (cudaStream_t)stream);
}

int xb_spmv_f32(xb_plan *p, int32_t variant, float alpha, const float *x, float beta, float *y,
                void *stream) {
    XB_TRY(need_plan(p, x, y));
    return xb::spmv_launch_f32(p, variant, 0, 0, alpha, x, beta, y, (cudaStream_t)stream);
}

int xb_dot(xb_plan *p, int32_t n, const double *x, const double *y, double *out, void *stream) {
    if (!p || !out || n < 0 || (n > 0 && (!x || !y)))
        return xb::set_error(XB_EINVAL, "xb_dot: bad argument");
    return xb::vdot(p, n, x, y, out, (cudaStream_t)stream);
}

int xb_axpy(int32_t n, double a, const double *x, double *y, void *stream) {
    if (n < 0 || (n > 0 && (!x || !y))) return xb::set_error(XB_EINVAL, "xb_axpy: bad argument");
    return xb::vaxpy(n, a, x, y, (cudaStream_t)stream);
}

int xb_mgs(xb_plan *p, int32_t n, int32_t k, const double *V, int64_t ld, double *w, double *h,
           void *stream) {
    if (!p || n < 0 || k < 1 || k > 512 || ld < n || !V || !w || !h)
        return xb::set_error(XB_EINVAL, "xb_mgs: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int M = k;
    XB_TRY(xb::ensure_work(p, xb::gm_doubles(M) * sizeof(double) + 256));
    double *base = static_cast<double *>(p->d_work);
    XB_CUDA(cudaMemsetAsync(base, 0, xb::gm_doubles(M) * sizeof(double), s));
    xb::GmDev st = xb::gm_layout(base, M);
    // unit scales, raw mode: a plain MGS sweep whose column is left unrotated
    std::vector<double> ones(M + 1, 1.0);
    XB_CUDA(cudaMemcpyAsync(st.sc, ones.data(), (M + 1) * sizeof(double), cudaMemcpyHostToDevice, s));
    double misc[xb::GM_NMISC] = {0};
    misc[xb::GM_BNORM] = 1.0;
    misc[xb::GM_TAU] = -1.0;
    misc[xb::GM_RAW] = 1.0;
    XB_CUDA(cudaMemcpyAsync(st.misc, misc, sizeof misc, cudaMemcpyHostToDevice, s));
    XB_TRY(xb::gm_mgs_step<double>(p, st, n, V, ld, w, k - 1, s));
    XB_CUDA(cudaMemcpyAsync(h, st.H + (size_t)(k - 1) * (M + 1), (k + 1) * sizeof(double),
                            cudaMemcpyDeviceToDevice, s));
    XB_CUDA(cudaStreamSynchronize(s));
    return XB_OK;
}

int xb_orth(xb_plan *p, int32_t n, int32_t k, const double *V, int64_t ld, double *w, double *h,
            int32_t ortho, void *stream) {
    if (!p || n < 0 || k < 1 || k > 512 || ld < n || !V || !w || !h || ortho < XB_ORTHO_MGS ||
        ortho > XB_ORTHO_BCGS)
        return xb::set_error(XB_EINVAL, "xb_orth: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int M = k;
    XB_TRY(xb::ensure_work(p, xb::gm_doubles(M) * sizeof(double) + 256));
    double *base = static_cast<double *>(p->d_work);
    XB_CUDA(cudaMemsetAsync(base, 0, xb::gm_doubles(M) * sizeof(double), s));
    xb::GmDev st = xb::gm_layout(base, M);
    // unit scales, raw mode: the column is left unrotated
    std::vector<double> ones(M + 1, 1.0);
    XB_CUDA(cudaMemcpyAsync(st.sc, ones.data(), (M + 1) * sizeof(double), cudaMemcpyHostToDevice, s));
    double misc[xb::GM_NMISC] = {0};
    misc[xb::GM_BNORM] = 1.0;
    misc[xb::GM_TAU] = -1.0;
    misc[xb::GM_RAW] = 1.0;
    XB_CUDA(cudaMemcpyAsync(st.misc, misc, sizeof misc, cudaMemcpyHostToDevice, s));
    XB_TRY(xb::gm_ortho_step<double>(p, st, n, V, ld, w, k - 1, ortho, s));
    XB_CUDA(cudaMemcpyAsync(h, st.H + (size_t)(k - 1) * (M + 1), (k + 1) * sizeof(double),
                            cudaMemcpyDeviceToDevice, s));
    XB_CUDA(cudaStreamSynchronize(s));
    return XB_OK;
}

}  // extern "C"
