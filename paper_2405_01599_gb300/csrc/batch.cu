// Batched solve of many independent systems in ONE persistent kernel launch,
// captured in a CUDA graph and replayed.  Each CTA pulls the next system from
// an atomic work queue (systems ordered largest first, so the long solves
// start early) and runs the whole restarted GMRES(m) for it with block-level
// reductions: the CTAs never wait on one another, so there is no inter-CTA
// spin.  A %globaltimer deadline bounds the launch's run time.
//
// Per system the tuner's choices apply: the restart length m and the SpMV
// mode inside the CTA (0: one thread per row; 1: one warp per row, for rows
// long or uneven enough that a thread per row would serialise).
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

struct xb_batch_dev {
    int n, nnz, m, mode, zero_x;
    int64_t ld;
    const int *rowptr, *col;
    const double *val, *b;
    double *x;
    double *ws;  // (m+1)*ld basis, then (m+1)*m Hessenberg
};

struct xb_batch {
    int count = 0;
    xb_batch_dev *d_sys = nullptr;
    xb_batch_info *d_info = nullptr;
    int *d_order = nullptr, *d_queue = nullptr;
    double *d_ws = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int grid = 0;
};

namespace {

constexpr int kBT = 512;  // threads per CTA of the batched kernel

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Sum over the CTA, result returned to every thread.
__device__ double cta_sum(double v, double *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[32] = v;
    }
    __syncthreads();
    return sh[32];
}

// y = alpha*A*x (+ beta*y when beta != 0), CTA-wide.
__device__ void cta_spmv(const xb_batch_dev &S, double alpha, const double *__restrict__ x,
                         double beta, double *__restrict__ y) {
    if (S.mode == 0) {
        for (int r = threadIdx.x; r < S.n; r += blockDim.x) {
            double s = 0.0;
            for (int k = S.rowptr[r]; k < S.rowptr[r + 1]; k++) s = fma(S.val[k], x[S.col[k]], s);
            y[r] = beta == 0.0 ? alpha * s : fma(alpha, s, beta * y[r]);
        }
    } else {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int r = w; r < S.n; r += nw) {
            double s = 0.0;
            for (int k = S.rowptr[r] + lane; k < S.rowptr[r + 1]; k += 32)
                s = fma(S.val[k], x[S.col[k]], s);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) y[r] = beta == 0.0 ? alpha * s : fma(alpha, s, beta * y[r]);
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kBT) k_batch_gmres(const xb_batch_dev *__restrict__ sys,
                                                     xb_batch_info *__restrict__ out,
                                                     const int *__restrict__ order, int count,
                                                     int *__restrict__ queue, double tol,
                                                     int maxiter, unsigned long long budget_ns) {
    __shared__ double sh[40];
    __shared__ double g[XB_BATCH_MAX_M + 1], cs[XB_BATCH_MAX_M], sn[XB_BATCH_MAX_M], yv[XB_BATCH_MAX_M];
    __shared__ int s_id, s_flag;
    __shared__ unsigned long long s_t0;
    if (threadIdx.x == 0) s_t0 = gtimer();
    __syncthreads();
    const unsigned long long t_start = s_t0;
    for (;;) {
        if (threadIdx.x == 0) s_id = atomicAdd(queue, 1);
        __syncthreads();
        const int q = s_id;
        __syncthreads();
        if (q >= count) return;
        const int id = order[q];
        const xb_batch_dev S = sys[id];
        const int n = S.n, m = S.m;
        const int64_t ld = S.ld;
        double *V = S.ws;
        double *H = S.ws + (size_t)(m + 1) * ld;  // column-major (m+1) x m
        unsigned long long ts = gtimer();
        if (S.zero_x)
            for (int i = threadIdx.x; i < n; i += blockDim.x) S.x[i] = 0.0;
        __syncthreads();
        // ||b||
        double a = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) a = fma(S.b[i], S.b[i], a);
        const double bnorm = sqrt(cta_sum(a, sh));
        int iters = 0, restarts = 0, status = XB_OK, claimed = 0;
        double tau = tol, res_true = 0.0;
        if (bnorm == 0.0) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) S.x[i] = 0.0;
            __syncthreads();
        } else {
            for (;;) {
                // r = b - A x into V_0
                for (int i = threadIdx.x; i < n; i += blockDim.x) V[i] = S.b[i];
                __syncthreads();
                cta_spmv(S, -1.0, S.x, 1.0, V);
                a = 0.0;
                for (int i = threadIdx.x; i < n; i += blockDim.x) a = fma(V[i], V[i], a);
                const double beta = sqrt(cta_sum(a, sh));
                res_true = beta / bnorm;
                if (res_true <= tol) {
                    status = XB_OK;
                    break;
                }
                if (iters >= maxiter || gtimer() - t_start > budget_ns) {
                    status = XB_ENOCONV;
                    break;
                }
                if (claimed) tau *= tol / res_true;  // fault convergence: narrow the threshold
                claimed = 0;
                const double ib = 1.0 / beta;
                for (int i = threadIdx.x; i < n; i += blockDim.x) V[i] *= ib;
                for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = 0.0;
                __syncthreads();
                if (threadIdx.x == 0) g[0] = beta;
                int k = 0;
                for (int j = 0; j < m; j++) {
                    iters++;
                    double *w = V + (size_t)(j + 1) * ld;
                    cta_spmv(S, 1.0, V + (size_t)j * ld, 0.0, w);
                    // modified Gram-Schmidt
                    double len2 = 0.0;
                    for (int i = 0; i <= j; i++) {
                        const double *vi = V + (size_t)i * ld;
                        a = 0.0;
                        for (int e = threadIdx.x; e < n; e += blockDim.x) a = fma(w[e], vi[e], a);
                        const double h = cta_sum(a, sh);
                        for (int e = threadIdx.x; e < n; e += blockDim.x) w[e] = fma(-h, vi[e], w[e]);
                        if (threadIdx.x == 0) H[(size_t)j * (m + 1) + i] = h;
                        len2 += h * h;
                        __syncthreads();
                    }
                    a = 0.0;
                    for (int e = threadIdx.x; e < n; e += blockDim.x) a = fma(w[e], w[e], a);
                    const double hn = sqrt(cta_sum(a, sh));
                    if (threadIdx.x == 0) {
                        double *col = H + (size_t)j * (m + 1);
                        col[j + 1] = hn;
                        for (int i = 0; i < j; i++) {
                            const double c0 = col[i], c1 = col[i + 1];
                            col[i] = cs[i] * c0 + sn[i] * c1;
                            col[i + 1] = -sn[i] * c0 + cs[i] * c1;
                        }
                        const double c0 = col[j];
                        const double rr = hypot(c0, hn);
                        int flag = 0;
                        if (rr == 0.0) {
                            flag = 2;
                        } else {
                            cs[j] = c0 / rr;
                            sn[j] = hn / rr;
                            col[j] = rr;
                            col[j + 1] = 0.0;
                            g[j + 1] = -sn[j] * g[j];
                            g[j] = cs[j] * g[j];
                            if (hn <= 1e-14 * sqrt(len2 + hn * hn)) flag = 1;
                            else if (fabs(g[j + 1]) / bnorm <= tau) flag = 3;
                        }
                        s_flag = flag;
                    }
                    __syncthreads();
                    const int flag = s_flag;
                    if (flag == 2) {
                        k = j;
                        status = XB_EBREAKDOWN;
                        break;
                    }
                    k = j + 1;
                    if (flag == 1) {
                        claimed = 1;
                        break;
                    }
                    const double ih = 1.0 / hn;
                    for (int e = threadIdx.x; e < n; e += blockDim.x) w[e] *= ih;
                    __syncthreads();
                    if (flag == 3) {
                        claimed = 1;
                        break;
                    }
                    if (iters >= maxiter) break;
                }
                if (status == XB_EBREAKDOWN) break;
                // R y = g, x += V y
                if (threadIdx.x == 0) {
                    for (int i = k - 1; i >= 0; i--) {
                        double s = g[i];
                        for (int c = i + 1; c < k; c++) s -= H[(size_t)c * (m + 1) + i] * yv[c];
                        yv[i] = s / H[(size_t)i * (m + 1) + i];
                    }
                }
                __syncthreads();
                for (int e = threadIdx.x; e < n; e += blockDim.x) {
                    double s = 0.0;
                    for (int i = 0; i < k; i++) s = fma(yv[i], V[(size_t)i * ld + e], s);
                    S.x[e] += s;
                }
                __syncthreads();
                restarts++;
            }
        }
        if (threadIdx.x == 0) {
            xb_batch_info inf;
            inf.status = status;
            inf.iters = iters;
            inf.restarts = restarts;
            inf.m = m;
            inf.mode = S.mode;
            inf.res_true = res_true;
            inf.ms = (double)(gtimer() - ts) * 1e-6;
            out[id] = inf;
        }
        __syncthreads();
    }
}

}  // namespace

extern "C" {

int xb_batch_destroy(xb_batch *bt) {
    if (!bt) return XB_OK;
    cudaDeviceSynchronize();
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    cudaFree(bt->d_sys);
    cudaFree(bt->d_info);
    cudaFree(bt->d_order);
    cudaFree(bt->d_queue);
    cudaFree(bt->d_ws);
    delete bt;
    return XB_OK;
}

int xb_batch_create(int32_t count, const xb_batch_sys *sys, const xb_options *opt, void *stream,
                    xb_batch **out) {
    if (count < 0 || (count > 0 && !sys) || !out) return xb::set_error(XB_EINVAL, "batch_create: bad argument");
    *out = nullptr;
    xb_options o;
    if (opt) o = *opt;
    else xb_options_default(&o);
    if (!(o.tol > 0.0)) return xb::set_error(XB_EINVAL, "batch_create: tol must be > 0");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<xb_batch_dev> h(count);
    size_t ws = 0;
    for (int i = 0; i < count; i++) {
        const xb_batch_sys &q = sys[i];
        if (q.n < 0 || q.nnz < 0 || q.m < 1 || q.m > XB_BATCH_MAX_M || (q.mode != 0 && q.mode != 1) ||
            (q.n > 0 && (!q.rowptr || !q.b || !q.x || (q.nnz > 0 && (!q.col || !q.val)))))
            return xb::set_error(XB_EINVAL, "batch_create: system %d invalid (n=%d m=%d mode=%d)", i,
                                 q.n, q.m, q.mode);
        xb_batch_dev &d = h[i];
        d.n = q.n;
        d.nnz = q.nnz;
        d.m = q.m;
        d.mode = q.mode;
        d.zero_x = q.zero_x;
        d.ld = ((int64_t)q.n + 31) / 32 * 32;
        d.rowptr = q.rowptr;
        d.col = q.col;
        d.val = q.val;
        d.b = q.b;
        d.x = q.x;
        ws += (size_t)(q.m + 1) * d.ld + (size_t)(q.m + 1) * q.m + 32;
    }
    xb_batch *bt = new xb_batch();
    bt->count = count;
    auto fail = [&](int code) {
        xb_batch_destroy(bt);
        return code;
    };
    cudaError_t e = cudaMalloc(&bt->d_ws, std::max<size_t>(ws, 1) * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(xb::set_error(XB_ENOMEM, "batch_create: %zu bytes of workspace", ws * 8));
    }
    size_t off = 0;
    for (int i = 0; i < count; i++) {
        h[i].ws = bt->d_ws + off;
        off += (size_t)(h[i].m + 1) * h[i].ld + (size_t)(h[i].m + 1) * h[i].m + 32;
    }
    // largest first: the long solves start in the first wave
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (int64_t)h[a].nnz + h[a].n > (int64_t)h[b].nnz + h[b].n;
    });
    e = cudaMalloc(&bt->d_sys, std::max(count, 1) * sizeof(xb_batch_dev));
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_info, std::max(count, 1) * sizeof(xb_batch_info));
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_order, std::max(count, 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_queue, sizeof(int));
    if (e == cudaSuccess && count > 0)
        e = cudaMemcpy(bt->d_sys, h.data(), count * sizeof(xb_batch_dev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && count > 0)
        e = cudaMemcpy(bt->d_order, order.data(), count * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(xb::cuda_error(e, "batch_create"));
    // grid: as many CTAs as fit co-resident (persistent), at most one per system
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_gmres, kBT, 0);
    if (e != cudaSuccess) return fail(xb::cuda_error(e, "batch_create: occupancy"));
    bt->grid = std::max(1, std::min(count, std::max(1, per_sm) * xb::num_sms()));
    const unsigned long long budget =
        (unsigned long long)(std::min(o.maxtime_s, 3600.0) * 1e9);
    // capture (on a private stream: the caller's may be the legacy default
    // stream, which cannot be captured): reset the queue, one persistent launch
    (void)s;
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(xb::cuda_error(e, "batch_create: capture stream"));
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return fail(xb::cuda_error(e, "batch_create: begin capture"));
    }
    cudaMemsetAsync(bt->d_queue, 0, sizeof(int), cs);
    k_batch_gmres<<<bt->grid, kBT, 0, cs>>>(bt->d_sys, bt->d_info, bt->d_order, count, bt->d_queue,
                                             o.tol, o.maxiter, budget);
    cudaError_t el = cudaGetLastError();
    e = cudaStreamEndCapture(cs, &bt->graph);
    cudaStreamDestroy(cs);
    if (el != cudaSuccess) return fail(xb::cuda_error(el, "batch_create: launch in capture"));
    if (e != cudaSuccess) return fail(xb::cuda_error(e, "batch_create: end capture"));
    e = cudaGraphInstantiate(&bt->exec, bt->graph, 0);
    if (e != cudaSuccess) return fail(xb::cuda_error(e, "batch_create: instantiate"));
    *out = bt;
    return XB_OK;
}

int xb_batch_run(xb_batch *bt, void *stream) {
    if (!bt) return xb::set_error(XB_EINVAL, "batch_run: NULL");
    if (bt->count == 0) return XB_OK;
    XB_CUDA(cudaGraphLaunch(bt->exec, (cudaStream_t)stream));
    return XB_OK;
}

int xb_batch_results(xb_batch *bt, xb_batch_info *infos, void *stream) {
    if (!bt || (bt->count > 0 && !infos)) return xb::set_error(XB_EINVAL, "batch_results: bad argument");
    if (bt->count == 0) return XB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    XB_CUDA(cudaMemcpyAsync(infos, bt->d_info, bt->count * sizeof(xb_batch_info), cudaMemcpyDeviceToHost, s));
    XB_CUDA(cudaStreamSynchronize(s));
    int worst = XB_OK;
    for (int i = 0; i < bt->count; i++)
        if (infos[i].status != XB_OK && worst == XB_OK) worst = infos[i].status;
    return worst;
}

int xb_batch_solve(int32_t count, const xb_batch_sys *sys, const xb_options *opt,
                   xb_batch_info *infos, void *stream) {
    xb_batch *bt = nullptr;
    XB_TRY(xb_batch_create(count, sys, opt, stream, &bt));
    int r = xb_batch_run(bt, stream);
    if (r == XB_OK) r = xb_batch_results(bt, infos, stream);
    xb_batch_destroy(bt);
    return r;
}

}  // extern "C"
