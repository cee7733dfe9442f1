// Batched solve of many independent systems in ONE persistent kernel launch,
// captured in a CUDA graph and replayed.
//
// The launch is a grid of 8-CTA thread-block clusters, fed by two atomic
// queues (each ordered largest first):
//   - a system with n >= kLargeN is solved by a whole cluster: every CTA
//     owns a slice of the rows, dot products are combined across the cluster
//     through distributed shared memory (every CTA sums the 8 partials in rank
//     order, so all CTAs hold identical values), and hardware cluster
//     barriers order the shared vectors; a cluster's leader pulls these;
//   - smaller systems are pulled by each CTA on its own, as soon as it is
//     free, and solved with block-level reductions only.
// Most clusters take the cluster queue first and then the other; the first
// few start on the single-CTA queue and join the cluster queue after it.
// Every cluster barrier sits on a path whose branch conditions are
// cluster-uniform (iteration counts, reduced values, and a time-budget flag
// that rank 0 decides and broadcasts through a reduction), so all CTAs of a
// cluster reach the same barriers in the same order.
//
// The solver is restarted GMRES(m) with modified Gram-Schmidt (fused: each
// pass applies the previous projection and takes the next inner product) or
// blocked classical Gram-Schmidt with block length 4 (one pass and one
// four-value reduction per block),
// Givens least squares, the true-residual check at every restart (fault
// convergence narrows the implicit threshold), and, when enabled, the
// MM-ratio restart rule of Eq. (1) / Fig. 2 / Sec. 4.3 (m grows by 5, up to
// m_max, when 5 consecutive restart residuals change by less than theta).
#include "common.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>

namespace cg = cooperative_groups;

namespace {
constexpr int kCl = 8;          // CTAs per cluster
constexpr int kBT = 512;        // threads per CTA
constexpr int kLargeN = 30000;  // systems this large are solved by a whole cluster
constexpr int kCtaRow = 1024;   // mode 1: rows longer than this are summed by the whole CTA
}  // namespace

struct xb_batch_dev {
    int n, nnz, m, m_max, mode, zero_x, coop;
    int64_t ld;
    const int *rowptr, *col;
    const double *val, *b;
    double *x;
    double *V;  // (m_max+1) * ld basis
    double *H;  // per cooperating CTA: (m_max+1) * m_max Hessenberg (column-major)
    const int *lrows;  // mode 1: the rows longer than kCtaRow, ascending
    int nl;
};

struct xb_batch {
    int count = 0;
    xb_batch_dev *d_sys = nullptr;
    xb_batch_info *d_info = nullptr;
    int *d_order = nullptr, *d_queue = nullptr;
    double *d_ws = nullptr;
    int *d_lrows = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int grid = 0;
};

namespace {

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct Smem {
    double sh[40];
    double slot[2];  // this CTA's partial of the current cluster reduction
    double sh4[4][kBT / 32], slot4[2][4], tot4[4];  // the same for 4 sums at once
    double g[XB_BATCH_MAX_M + 1], cs[XB_BATCH_MAX_M], sn[XB_BATCH_MAX_M], yv[XB_BATCH_MAX_M];
    unsigned long long t_start;
    int q;
    int flag;
};

// Sum over the CTA, result returned to every thread.
__device__ double cta_sum(double v, Smem &S) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) S.sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? S.sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) S.sh[32] = v;
    }
    __syncthreads();
    return S.sh[32];
}

// The solve's view of the work: rows [r0, r1) of this CTA, and whether the
// CTAs of the cluster cooperate on this system.
struct Part {
    int r0, r1, coop, phase;
};

// Sum over all cooperating CTAs (one cluster barrier), identical everywhere.
// The two partial slots alternate, so a slot is rewritten only after every
// CTA has passed the barrier of the reduction that follows its last read.
__device__ double coop_sum(double v, Smem &S, Part &P) {
    const double t = cta_sum(v, S);
    if (!P.coop) return t;
    cg::cluster_group cl = cg::this_cluster();
    if (threadIdx.x == 0) S.slot[P.phase] = t;
    cl.sync();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int r = 0; r < kCl; r++) tot += cl.map_shared_rank(S.slot, r)[P.phase];
        S.sh[34] = tot;
    }
    __syncthreads();
    const double tot = S.sh[34];
    __syncthreads();
    P.phase ^= 1;
    return tot;
}

// Four sums at once over all cooperating CTAs (one CTA barrier pair and one
// cluster barrier for the four), identical everywhere, in a fixed order.
__device__ void coop_sum4(double (&v)[4], Smem &S, Part &P) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; q++)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 4; q++) S.sh4[q][w] = v[q];
    __syncthreads();
    if (threadIdx.x < 4) {
        double a = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) a += S.sh4[threadIdx.x][k];
        if (P.coop) S.slot4[P.phase][threadIdx.x] = a;
        else S.tot4[threadIdx.x] = a;
    }
    if (P.coop) {
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        if (threadIdx.x < 4) {
            double tot = 0.0;
            for (int r = 0; r < kCl; r++) tot += cl.map_shared_rank(&S.slot4[0][0], r)[P.phase * 4 + threadIdx.x];
            S.tot4[threadIdx.x] = tot;
        }
        P.phase ^= 1;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; q++) v[q] = S.tot4[q];
    __syncthreads();
}

// Make every cooperating CTA's writes to the shared vectors visible to all.
__device__ __forceinline__ void coop_barrier(const Part &P) {
    if (P.coop) cg::this_cluster().sync();
    else __syncthreads();
}

// y[r0:r1] = alpha*A[r0:r1,:]*x (+ beta*y).  x is written by the other CTAs
// of the cluster during the launch, so it is read at L2 (ld.global.cg), the
// coherence point, never through the SM-local read-only path.
//   mode 0: one thread per row;
//   mode 1: rows in warp-sized blocks, one thread per row, except that rows
//           longer than 32 non-zeros are taken by the whole warp in turn
//           (lanes stride over the row, shuffle reduction), and rows longer
//           than kCtaRow (the system's list, ascending) by the whole CTA
//           after the blocks, so a power-law row of thousands of entries
//           neither serialises one thread nor one warp.
// Every row's sum has one fixed order (its stride and four interleaved
// partial sums), so results do not depend on scheduling.
__device__ __forceinline__ double row_dot(const int *__restrict__ col,
                                          const double *__restrict__ val, const double *x,
                                          int ka, int kb, int step) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int k = ka;
    for (; k + 3 * step < kb; k += 4 * step) {  // four gathers in flight
        const int c0 = __ldg(col + k), c1 = __ldg(col + k + step), c2 = __ldg(col + k + 2 * step),
                  c3 = __ldg(col + k + 3 * step);
        const double v0 = __ldg(val + k), v1 = __ldg(val + k + step), v2 = __ldg(val + k + 2 * step),
                     v3 = __ldg(val + k + 3 * step);
        s0 = fma(v0, __ldcg(x + c0), s0);
        s1 = fma(v1, __ldcg(x + c1), s1);
        s2 = fma(v2, __ldcg(x + c2), s2);
        s3 = fma(v3, __ldcg(x + c3), s3);
    }
    for (; k < kb; k += step) s0 = fma(__ldg(val + k), __ldcg(x + __ldg(col + k)), s0);
    return (s0 + s1) + (s2 + s3);
}

__device__ void part_spmv(const xb_batch_dev &D, const Part &P, Smem &S, double alpha,
                          const double *x, double beta, double *y) {
    const int *__restrict__ rp = D.rowptr;
    if (D.mode == 0) {
        for (int r = P.r0 + threadIdx.x; r < P.r1; r += blockDim.x) {
            const double s = row_dot(D.col, D.val, x, __ldg(rp + r), __ldg(rp + r + 1), 1);
            y[r] = beta == 0.0 ? alpha * s : fma(alpha, s, beta * y[r]);
        }
    } else {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int base = P.r0 + 32 * w; base < P.r1; base += 32 * nw) {  // warp-uniform
            const int r = base + lane;
            int ka = 0, kb = 0;
            if (r < P.r1) {
                ka = __ldg(rp + r);
                kb = __ldg(rp + r + 1);
            }
            const bool cta = kb - ka > kCtaRow;
            const bool lng = kb - ka > 32 && !cta;
            double s = (lng || cta) ? 0.0 : row_dot(D.col, D.val, x, ka, kb, 1);
            unsigned todo = __ballot_sync(0xffffffffu, lng);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const int la = __shfl_sync(0xffffffffu, ka, src);
                const int lb = __shfl_sync(0xffffffffu, kb, src);
                double t = row_dot(D.col, D.val, x, la + lane, lb, 32);
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                if (lane == src) s = t;
            }
            if (r < P.r1 && !cta) y[r] = beta == 0.0 ? alpha * s : fma(alpha, s, beta * y[r]);
        }
        if (D.nl > 0) {
            // the CTA's long rows: first list entry >= r0 (binary search), up to r1
            int lo = 0, hi = D.nl;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(D.lrows + mid) < P.r0) lo = mid + 1;
                else hi = mid;
            }
            for (int q = lo; q < D.nl; q++) {  // CTA-uniform
                const int r = __ldg(D.lrows + q);
                if (r >= P.r1) break;
                const int ka = __ldg(rp + r), kb = __ldg(rp + r + 1);
                const double t = cta_sum(row_dot(D.col, D.val, x, ka + (int)threadIdx.x, kb,
                                                 (int)blockDim.x), S);
                if (threadIdx.x == 0) y[r] = beta == 0.0 ? alpha * t : fma(alpha, t, beta * y[r]);
            }
        }
    }
    // rows were stored by other threads than the ones that read them next,
    // so the CTA meets before anyone reads y
    __syncthreads();
}

// One fused MGS pass over rows [r0, r1) of this CTA (four rows per thread in
// flight): OP 0 returns (w, vn); OP 1 applies w -= c vp and returns (w, vn);
// OP 2 applies w -= c vp and returns (w, w).
template <int OP>
__device__ __forceinline__ double mgs_rows(double *__restrict__ w, const double *__restrict__ vp,
                                           const double *__restrict__ vn, double c, int r0,
                                           int r1) {
    const int S = blockDim.x;
    double a0 = 0.0, a1 = 0.0;
    int e = r0 + threadIdx.x;
    for (; e + 3 * S < r1; e += 4 * S) {
        double x[4], p[4], q[4];
#pragma unroll
        for (int u = 0; u < 4; u++) x[u] = w[e + u * S];
        if (OP != 0) {
#pragma unroll
            for (int u = 0; u < 4; u++) p[u] = vp[e + u * S];
        }
        if (OP != 2) {
#pragma unroll
            for (int u = 0; u < 4; u++) q[u] = vn[e + u * S];
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (OP != 0) x[u] = fma(-c, p[u], x[u]);
            const double o = OP == 2 ? x[u] : q[u];
            if (u & 1) a1 = fma(x[u], o, a1);
            else a0 = fma(x[u], o, a0);
            if (OP != 0) w[e + u * S] = x[u];
        }
    }
    for (; e < r1; e += S) {
        double xe = w[e];
        if (OP != 0) {
            xe = fma(-c, vp[e], xe);
            w[e] = xe;
        }
        a0 = fma(xe, OP == 2 ? xe : vn[e], a0);
    }
    return a0 + a1;
}

// One block Gram-Schmidt pass over rows [r0, r1): w -= sum_{q < nu} c[q] V_{u0+q}
// (nu <= 4), then the nd <= 4 dots (w, V_{d0+q}) into a[] (or (w, w) into a[0]
// when nd == 0).  Two rows per thread, every load of both issued before their
// arithmetic (the pass is latency-bound on one SM).
template <int R>
__device__ __forceinline__ void bgs_row(double *__restrict__ w, const double *__restrict__ V,
                                        int64_t ld, int u0, int nu, const double (&c)[4], int d0,
                                        int nd, int e0, int B, double (&a)[4]) {
    double x[R], pu[R][4], pd[R][4];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int e = e0 + r * B;
        x[r] = w[e];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            pu[r][q] = q < nu ? V[(size_t)(u0 + q) * ld + e] : 0.0;
            pd[r][q] = q < nd ? V[(size_t)(d0 + q) * ld + e] : 0.0;
        }
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (q < nu) x[r] = fma(-c[q], pu[r][q], x[r]);
        if (nu > 0) w[e0 + r * B] = x[r];
        if (nd == 0) {
            a[0] = fma(x[r], x[r], a[0]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (q < nd) a[q] = fma(x[r], pd[r][q], a[q]);
        }
    }
}

__device__ __forceinline__ void bgs_rows(double *__restrict__ w, const double *__restrict__ V,
                                         int64_t ld, int u0, int nu, const double (&c)[4], int d0,
                                         int nd, int r0, int r1, double (&a)[4]) {
#pragma unroll
    for (int q = 0; q < 4; q++) a[q] = 0.0;
    const int B = blockDim.x;
    int e = r0 + threadIdx.x;
    for (; e + B < r1; e += 2 * B) bgs_row<2>(w, V, ld, u0, nu, c, d0, nd, e, B, a);
    if (e < r1) bgs_row<1>(w, V, ld, u0, nu, c, d0, nd, e, B, a);
}

__device__ void solve_one(const xb_batch_dev &D, Part &P, Smem &S, double tol, int maxiter,
                          unsigned long long deadline, int rank, double theta, int bcgs,
                          xb_batch_info *out) {
    const unsigned long long ts = gtimer();
    const int m_max = D.m_max;
    const int64_t ld = D.ld;
    double *V = D.V;
    double *H = D.H + (P.coop ? (size_t)rank * (m_max + 1) * m_max : 0);
    const int r0 = P.r0, r1 = P.r1;
    if (D.zero_x)
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) D.x[i] = 0.0;
    double a = 0.0;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) a = fma(D.b[i], D.b[i], a);
    const double bnorm = sqrt(coop_sum(a, S, P));
    int iters = 0, restarts = 0, status = XB_OK, claimed = 0, m = D.m, K = 0;
    double tau = tol, res_true = 0.0;
    double samp[5];  // restart residuals for the MM-ratio rule (same in every thread)
    if (bnorm == 0.0) {
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) D.x[i] = 0.0;
    } else {
        for (;;) {
            coop_barrier(P);  // x complete before A x
            for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) V[i] = D.b[i];
            __syncthreads();  // the SpMV reads V_0 rows through other threads
            part_spmv(D, P, S, -1.0, D.x, 1.0, V);
            a = 0.0;
            for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) a = fma(V[i], V[i], a);
            const double beta = sqrt(coop_sum(a, S, P));
            // the time budget is rank 0's decision, broadcast by a reduction
            const double late =
                coop_sum((rank == 0 && threadIdx.x == 0 && gtimer() > deadline) ? 1.0 : 0.0, S, P);
            res_true = beta / bnorm;
            if (res_true <= tol) {
                status = XB_OK;
                break;
            }
            if (iters >= maxiter || late > 0.0) {
                status = XB_ENOCONV;
                break;
            }
            if (claimed) tau *= tol / res_true;  // fault convergence: narrow the threshold
            claimed = 0;
            if (restarts > 0) {  // restart-frequency rule (Eq. 1): judge every 5 samples
                samp[K++] = res_true;
                if (K == 5) {
                    double mx = samp[0], mn = samp[0];
                    for (int z = 1; z < 5; z++) {
                        mx = fmax(mx, samp[z]);
                        mn = fmin(mn, samp[z]);
                    }
                    if (mn > 0.0 && mx / mn < theta) m = min(m + 5, m_max);
                    K = 0;
                }
            }
            const double ib = 1.0 / beta;
            for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) V[i] *= ib;
            for (int i = threadIdx.x; i <= m; i += blockDim.x) S.g[i] = 0.0;
            __syncthreads();
            if (threadIdx.x == 0) S.g[0] = beta;
            int k = 0;
            for (int j = 0; j < m; j++) {
                iters++;
                double *w = V + (size_t)(j + 1) * ld;
                coop_barrier(P);  // v_j complete
                part_spmv(D, P, S, 1.0, V + (size_t)j * ld, 0.0, w);
                double len2 = 0.0, hn;
                if (bcgs) {
                    // BCGS, block length 4: one pass per block applies the previous
                    // block's projection and takes the dots with this block
                    double c[4] = {0.0, 0.0, 0.0, 0.0}, a4[4];
                    int u0 = 0, nu = 0;
                    for (int d0 = 0; d0 <= j; d0 += 4) {
                        const int nd = min(4, j + 1 - d0);
                        bgs_rows(w, V, ld, u0, nu, c, d0, nd, r0, r1, a4);
                        coop_sum4(a4, S, P);
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            if (q < nd) {
                                if (threadIdx.x == 0) H[(size_t)j * (m_max + 1) + d0 + q] = a4[q];
                                len2 += a4[q] * a4[q];
                                c[q] = a4[q];
                            }
                        }
                        u0 = d0;
                        nu = nd;
                    }
                    bgs_rows(w, V, ld, u0, nu, c, 0, 0, r0, r1, a4);
                    hn = sqrt(coop_sum(a4[0], S, P));
                } else {
                    // fused MGS: pass i applies the projection on v_{i-1}, takes (w, v_i)
                    double hprev = 0.0;
                    for (int i = 0; i <= j; i++) {
                        const double *vi = V + (size_t)i * ld;
                        a = i == 0 ? mgs_rows<0>(w, nullptr, vi, 0.0, r0, r1)
                                   : mgs_rows<1>(w, vi - ld, vi, hprev, r0, r1);
                        const double h = coop_sum(a, S, P);
                        if (threadIdx.x == 0) H[(size_t)j * (m_max + 1) + i] = h;
                        len2 += h * h;
                        hprev = h;
                    }
                    a = mgs_rows<2>(w, V + (size_t)j * ld, nullptr, hprev, r0, r1);
                    hn = sqrt(coop_sum(a, S, P));
                }
                if (threadIdx.x == 0) {
                    double *col = H + (size_t)j * (m_max + 1);
                    col[j + 1] = hn;
                    for (int i = 0; i < j; i++) {
                        const double c0 = col[i], c1 = col[i + 1];
                        col[i] = S.cs[i] * c0 + S.sn[i] * c1;
                        col[i + 1] = -S.sn[i] * c0 + S.cs[i] * c1;
                    }
                    const double c0 = col[j];
                    const double rr = hypot(c0, hn);
                    int flag = 0;
                    if (rr == 0.0) {
                        flag = 2;
                    } else {
                        S.cs[j] = c0 / rr;
                        S.sn[j] = hn / rr;
                        col[j] = rr;
                        col[j + 1] = 0.0;
                        S.g[j + 1] = -S.sn[j] * S.g[j];
                        S.g[j] = S.cs[j] * S.g[j];
                        if (hn <= 1e-14 * sqrt(len2 + hn * hn)) flag = 1;
                        else if (fabs(S.g[j + 1]) / bnorm <= tau) flag = 3;
                    }
                    S.flag = flag;
                }
                __syncthreads();
                const int flag = S.flag;
                __syncthreads();
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
                for (int e = r0 + threadIdx.x; e < r1; e += blockDim.x) w[e] *= ih;
                if (flag == 3) {
                    claimed = 1;
                    break;
                }
                if (iters >= maxiter) break;
            }
            if (status == XB_EBREAKDOWN) break;
            // R y = g (every cooperating CTA holds the same R and g), x += V y
            if (threadIdx.x == 0) {
                for (int i = k - 1; i >= 0; i--) {
                    double s = S.g[i];
                    for (int c = i + 1; c < k; c++) s -= H[(size_t)c * (m_max + 1) + i] * S.yv[c];
                    S.yv[i] = s / H[(size_t)i * (m_max + 1) + i];
                }
            }
            __syncthreads();
            {
                const double *__restrict__ Vc = V;
                double *__restrict__ xo = D.x;
                const int B = blockDim.x;
                int e = r0 + threadIdx.x;
                for (; e + B < r1; e += 2 * B) {  // two rows per thread in flight
                    double s0 = 0.0, s1 = 0.0;
                    for (int i = 0; i < k; i++) {
                        const double yi = S.yv[i];
                        s0 = fma(yi, Vc[(size_t)i * ld + e], s0);
                        s1 = fma(yi, Vc[(size_t)i * ld + e + B], s1);
                    }
                    xo[e] += s0;
                    xo[e + B] += s1;
                }
                for (; e < r1; e += B) {
                    double s0 = 0.0;
                    for (int i = 0; i < k; i++) s0 = fma(S.yv[i], Vc[(size_t)i * ld + e], s0);
                    xo[e] += s0;
                }
            }
            restarts++;
        }
    }
    if (threadIdx.x == 0 && rank == 0) {
        xb_batch_info inf;
        inf.status = status;
        inf.iters = iters;
        inf.restarts = restarts;
        inf.m = m;
        inf.mode = D.mode;
        inf.res_true = res_true;
        inf.ms = (double)(gtimer() - ts) * 1e-6;
        *out = inf;
    }
    __syncthreads();
}

__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kBT, 1)
    k_batch_gmres(const xb_batch_dev *__restrict__ sys, xb_batch_info *__restrict__ out,
                  const int *__restrict__ order, int count, int nbig, int nsmall_cl,
                  int *__restrict__ queue, double tol, int maxiter, unsigned long long budget_ns,
                  double theta, int bcgs) {
    __shared__ Smem S;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    if (threadIdx.x == 0) S.t_start = gtimer();
    // one deadline for the whole cluster: rank 0's start plus the budget
    cl.sync();
    const unsigned long long deadline = cl.map_shared_rank(&S, 0)->t_start + budget_ns;
    cl.sync();
    // phase 1: the systems a whole cluster solves (order[0, nbig), largest
    // first), one per pull of the cluster's leader; phase 2: the single-CTA
    // systems (order[nbig, count), largest first), every CTA pulling its next
    // system as soon as it is free (no cluster barrier and no distributed
    // shared memory inside phase 2, so the CTAs of a cluster run apart).  The
    // first nsmall_cl clusters start with phase 2, so the longest single-CTA
    // solves do not wait for the end of phase 1, and join phase 1 when the
    // single-CTA queue is empty (their last systems are the smallest, so the
    // regrouping barrier waits little); the others run phase 1, then phase 2.
    const bool small_first = (int)(blockIdx.x / kCl) < nsmall_cl;  // cluster-uniform
    auto phase1 = [&]() {
        for (;;) {
            if (rank == 0 && threadIdx.x == 0) S.q = atomicAdd(queue, 1);
            cl.sync();
            const int q = cl.map_shared_rank(&S, 0)->q;
            cl.sync();  // the leader may overwrite q only after every CTA has read it
            if (q >= nbig) return;  // cluster-uniform
            const xb_batch_dev D = sys[order[q]];
            const int per = (D.n + kCl - 1) / kCl;
            Part P{min(D.n, rank * per), min(D.n, (rank + 1) * per), 1, 0};
            solve_one(D, P, S, tol, maxiter, deadline, rank, theta, bcgs, out + order[q]);
        }
    };
    auto phase2 = [&]() {
        for (;;) {
            if (threadIdx.x == 0) S.q = atomicAdd(queue + 1, 1);
            __syncthreads();
            const int q = nbig + S.q;
            __syncthreads();  // S.q is rewritten only after every thread has read it
            if (q >= count) return;  // CTA-uniform
            const xb_batch_dev D = sys[order[q]];
            Part P{0, D.n, 0, 0};
            solve_one(D, P, S, tol, maxiter, deadline, 0, theta, bcgs, out + order[q]);
        }
    };
    if (small_first) {
        phase2();
        cl.sync();  // every CTA of the cluster is free: take cluster systems
        phase1();
    } else {
        phase1();
        phase2();
    }
}

}  // namespace

namespace xb {

// One system through the persistent kernel: a single 8-CTA cluster solving
// it together (rows split over the 8 CTAs, dot products combined through
// distributed shared memory), the system's basis and Hessenberg, its
// descriptor, queue and result in the plan's workspace; no graph capture, no
// allocation after the workspace has grown.  Used by gmres_solve for small
// systems, whose multi-launch Arnoldi steps are bound by launch and
// synchronisation latency.  The whole cluster is used even below the batch's
// cluster threshold: the launch holds one cluster anyway, and 8 SMs hide more
// of the L2 latency of each Gram-Schmidt pass (n = 4096: 30.5 ms for 535
// steps, 41 ms in one CTA).
int batch_single(xb_plan *p, const double *b, double *x, const xb_options &o, int mode,
                 xb_info &inf, double *alg_bytes, cudaStream_t s) {
    xb_batch_dev d;
    std::memset(&d, 0, sizeof d);
    d.n = p->n;
    d.nnz = p->nnz;
    d.m = o.m;
    d.m_max = o.dafrt ? std::max(o.m, std::min(o.m_max, XB_BATCH_MAX_M)) : o.m;
    d.mode = mode;
    d.zero_x = 0;
    d.coop = 1;
    d.ld = ((int64_t)d.n + 31) / 32 * 32;
    d.rowptr = p->rowptr;
    d.col = p->col;
    d.val = p->val;
    d.b = b;
    d.x = x;
    const size_t nv = (size_t)(d.m_max + 1) * d.ld;
    const size_t nh = (size_t)(d.coop ? kCl : 1) * (d.m_max + 1) * d.m_max + 32;
    const size_t meta = 4096;  // descriptor, result, order, queue
    // mode 1: the rows longer than kCtaRow, from the plan's host row pointer
    std::vector<int> lr;
    if (mode == 1 && p->nnz > kCtaRow && (int)p->h_rowptr.size() == p->n + 1)
        for (int r = 0; r < p->n; r++)
            if (p->h_rowptr[r + 1] - p->h_rowptr[r] > kCtaRow) lr.push_back(r);
    XB_TRY(ensure_work(p, (nv + nh) * sizeof(double) + meta + lr.size() * sizeof(int)));
    char *w = static_cast<char *>(p->d_work);
    d.V = reinterpret_cast<double *>(w);
    d.H = d.V + nv;
    char *m0 = w + (nv + nh) * sizeof(double);
    xb_batch_dev *d_sys = reinterpret_cast<xb_batch_dev *>(m0);
    xb_batch_info *d_info = reinterpret_cast<xb_batch_info *>(m0 + 1024);
    int *d_order = reinterpret_cast<int *>(m0 + 2048);
    int *d_queue = d_order + 1;
    static_assert(sizeof(xb_batch_dev) <= 1024 && sizeof(xb_batch_info) <= 1024, "meta layout");
    d.nl = (int)lr.size();
    d.lrows = nullptr;
    if (!lr.empty()) {
        int *d_lr = reinterpret_cast<int *>(m0 + meta);
        XB_CUDA(cudaMemcpyAsync(d_lr, lr.data(), lr.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        d.lrows = d_lr;
    }
    const int zero = 0;
    XB_CUDA(cudaMemcpyAsync(d_sys, &d, sizeof d, cudaMemcpyHostToDevice, s));
    XB_CUDA(cudaMemcpyAsync(d_order, &zero, sizeof zero, cudaMemcpyHostToDevice, s));
    XB_CUDA(cudaMemsetAsync(d_queue, 0, 2 * sizeof(int), s));
    const unsigned long long budget = (unsigned long long)(std::min(o.maxtime_s, 3600.0) * 1e9);
    const double theta = o.dafrt ? o.dafrt_theta : 0.0;
    const int bcgs = o.ortho == XB_ORTHO_BCGS ? 1 : 0;
    k_batch_gmres<<<kCl, kBT, 0, s>>>(d_sys, d_info, d_order, 1, 1, 0, d_queue, o.tol, o.maxiter,
                                      budget, theta, bcgs);
    XB_LAUNCHED("k_batch_gmres (single system)");
    xb_batch_info r;
    XB_CUDA(cudaMemcpyAsync(&r, d_info, sizeof r, cudaMemcpyDeviceToHost, s));
    XB_CUDA(cudaStreamSynchronize(s));
    inf.iters = r.iters;
    inf.restarts = r.restarts;
    inf.m_final = r.m;
    inf.res_true = r.res_true;
    inf.ortho_used = bcgs ? XB_ORTHO_BCGS : XB_ORTHO_MGS;
    inf.persistent = 1;
    // algorithmic bytes: per Arnoldi step one SpMV and the Gram-Schmidt passes
    // at the cycle's mean basis size, plus a residual per restart
    const double jm = (r.m + 1) / 2.0, n = d.n;
    *alg_bytes = r.iters * (spmv_alg_bytes(p, false, 8) + (4.0 * jm + 5.0) * 8.0 * n) +
                 (r.restarts + 1) * (spmv_alg_bytes(p, true, 8) + 16.0 * n);
    if (r.status == XB_ENOCONV)
        return set_error(XB_ENOCONV, "not converged: ||b-Ax||/||b|| = %.3e > tol %.1e", r.res_true,
                         o.tol);
    return r.status;
}

}  // namespace xb

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
    cudaFree(bt->d_lrows);
    delete bt;
    return XB_OK;
}

int xb_batch_create(int32_t count, const xb_batch_sys *sys, const xb_options *opt, void *stream,
                    xb_batch **out) {
    if (count < 0 || (count > 0 && !sys) || !out) return xb::set_error(XB_EINVAL, "batch_create: bad argument");
    *out = nullptr;
    (void)stream;
    xb_options o;
    if (opt) o = *opt;
    else xb_options_default(&o);
    if (!(o.tol > 0.0)) return xb::set_error(XB_EINVAL, "batch_create: tol must be > 0");
    if (o.ortho != XB_ORTHO_MGS && o.ortho != XB_ORTHO_BCGS && o.ortho != XB_ORTHO_AUTO)
        return xb::set_error(XB_EINVAL, "batch_create: orthogonalisation must be MGS, BCGS or AUTO");
    std::vector<xb_batch_dev> h(count);
    size_t ws = 0;
    // systems with n >= coop_min are solved by a whole cluster (environment
    // variable XB_BATCH_COOP_MIN_N overrides the default)
    long coop_min = kLargeN;
    if (const char *env = std::getenv("XB_BATCH_COOP_MIN_N")) coop_min = std::max(1L, std::atol(env));
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
        d.m_max = o.dafrt ? std::max(q.m, std::min(o.m_max, XB_BATCH_MAX_M)) : q.m;
        d.mode = q.mode;
        d.zero_x = q.zero_x;
        d.coop = q.n >= coop_min ? 1 : 0;
        d.ld = ((int64_t)q.n + 31) / 32 * 32;
        d.rowptr = q.rowptr;
        d.col = q.col;
        d.val = q.val;
        d.b = q.b;
        d.x = q.x;
        ws += (size_t)(d.m_max + 1) * d.ld + (size_t)(d.coop ? kCl : 1) * (d.m_max + 1) * d.m_max + 32;
    }
    // mode 1: each system's rows longer than kCtaRow (summed by a whole CTA),
    // from a host copy of its row pointer
    std::vector<int> lr_all, rp_h;
    std::vector<size_t> lr_off(count, 0);
    for (int i = 0; i < count; i++) {
        h[i].lrows = nullptr;
        h[i].nl = 0;
        if (h[i].mode != 1 || h[i].n < 1 || h[i].nnz <= kCtaRow) continue;
        rp_h.resize((size_t)h[i].n + 1);
        cudaError_t e = cudaMemcpy(rp_h.data(), h[i].rowptr, rp_h.size() * sizeof(int),
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return xb::cuda_error(e, "batch_create: read rowptr");
        lr_off[i] = lr_all.size();
        for (int r = 0; r < h[i].n; r++)
            if (rp_h[r + 1] - rp_h[r] > kCtaRow) lr_all.push_back(r);
        h[i].nl = (int)(lr_all.size() - lr_off[i]);
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
    if (!lr_all.empty()) {
        e = cudaMalloc(&bt->d_lrows, lr_all.size() * sizeof(int));
        if (e == cudaSuccess)
            e = cudaMemcpy(bt->d_lrows, lr_all.data(), lr_all.size() * sizeof(int),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(xb::cuda_error(e, "batch_create: long-row lists"));
        for (int i = 0; i < count; i++)
            if (h[i].nl > 0) h[i].lrows = bt->d_lrows + lr_off[i];
    }
    size_t off = 0;
    for (int i = 0; i < count; i++) {
        h[i].V = bt->d_ws + off;
        off += (size_t)(h[i].m_max + 1) * h[i].ld;
        h[i].H = bt->d_ws + off;
        off += (size_t)(h[i].coop ? kCl : 1) * (h[i].m_max + 1) * h[i].m_max + 32;
    }
    // the cluster systems first, then the single-CTA ones, each part
    // largest first: the long solves start in the first wave
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (h[a].coop != h[b].coop) return h[a].coop > h[b].coop;
        return (int64_t)h[a].nnz + h[a].n > (int64_t)h[b].nnz + h[b].n;
    });
    int nbig = 0;
    for (int i = 0; i < count; i++) nbig += h[i].coop ? 1 : 0;
    e = cudaMalloc(&bt->d_sys, std::max(count, 1) * sizeof(xb_batch_dev));
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_info, std::max(count, 1) * sizeof(xb_batch_info));
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_order, std::max(count, 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_queue, 2 * sizeof(int));
    if (e == cudaSuccess && count > 0)
        e = cudaMemcpy(bt->d_sys, h.data(), count * sizeof(xb_batch_dev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && count > 0)
        e = cudaMemcpy(bt->d_order, order.data(), count * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(xb::cuda_error(e, "batch_create"));
    // persistent grid: as many whole clusters as can be co-resident
    cudaLaunchConfig_t lc;
    std::memset(&lc, 0, sizeof lc);
    lc.gridDim = dim3(kCl, 1, 1);
    lc.blockDim = dim3(kBT, 1, 1);
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, (void *)k_batch_gmres, &lc);
    if (e != cudaSuccess || clusters < 1) {
        cudaGetLastError();
        clusters = std::max(1, xb::num_sms() / kCl);
    }
    bt->grid = kCl * std::max(1, clusters);
    // clusters that take the single-CTA systems from the start: their share
    // of the work, with nnz + m n (one step's SpMV and Gram-Schmidt) as the
    // per-system weight; none without cluster systems to balance against
    double w_big = 0.0, w_small = 0.0;
    for (int i = 0; i < count; i++) {
        const double wi = (double)h[i].nnz + (double)h[i].m * h[i].n;
        (h[i].coop ? w_big : w_small) += wi;
    }
    const int ncl = std::max(1, clusters);
    int nsmall_cl = 0;
    if (nbig > 0 && w_small > 0.0)
        nsmall_cl = std::min(ncl - 1, (int)std::lround(ncl * w_small / (w_big + w_small)));
    const unsigned long long budget = (unsigned long long)(std::min(o.maxtime_s, 3600.0) * 1e9);
    const double theta = o.dafrt ? o.dafrt_theta : 0.0;  // theta 0: the rule never fires
    // orthogonalisation: MGS or BCGS (block length 4); the accuracy policy's
    // choice for AUTO (no fault switch inside the launch)
    const int ortho = o.ortho == XB_ORTHO_AUTO ? (o.tol <= 1e-10 ? XB_ORTHO_MGS : XB_ORTHO_BCGS)
                                               : o.ortho;
    const int bcgs = ortho == XB_ORTHO_BCGS ? 1 : 0;
    // capture on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured): reset the queue, one persistent launch
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(xb::cuda_error(e, "batch_create: capture stream"));
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return fail(xb::cuda_error(e, "batch_create: begin capture"));
    }
    cudaMemsetAsync(bt->d_queue, 0, 2 * sizeof(int), cs);
    k_batch_gmres<<<bt->grid, kBT, 0, cs>>>(bt->d_sys, bt->d_info, bt->d_order, count, nbig,
                                             nsmall_cl, bt->d_queue,
                                             o.tol, o.maxiter, budget, theta, bcgs);
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
