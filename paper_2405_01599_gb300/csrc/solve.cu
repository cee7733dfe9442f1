// Host drivers of the restarted Krylov solvers (stream-ordered; the host only
// reads a handful of device scalars at check points).
//
// GMRES(m): Saad-Schultz restarted GMRES with MGS Arnoldi and Givens least
// squares (Sec. 2.2 / 4.3), the restart-frequency rule of Eq. (1), Fig. 2 and
// Sec. 4.3 (DAFRT), and the fault-convergence outer check of Sec. 3.1 / 3.3.2:
// every claimed convergence is verified on the true residual b - A x in FP64;
// a false claim narrows the implicit threshold and the iteration continues.
// BiCGStab: van der Vorst's method, unpreconditioned, same outer check.
// Mixed precision: FP32 GMRES(m) (FP32 SpMV on an FP32 copy of A, FP32 basis,
// FP64 Hessenberg/Givens/least squares) as the inner solver of FP64
// iterative refinement, with FP64 fall-back when refinement stagnates.
#include "krylov.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>

namespace {

using clk = std::chrono::steady_clock;

double secs_since(clk::time_point t0) {
    return std::chrono::duration<double>(clk::now() - t0).count();
}

// Read `cnt` doubles from device to the plan's pinned mirror and wait.
int peek(xb_plan *p, const double *dev, int cnt, cudaStream_t s) {
    XB_CUDA(cudaMemcpyAsync(p->h_pin, dev, cnt * sizeof(double), cudaMemcpyDeviceToHost, s));
    XB_CUDA(cudaStreamSynchronize(s));
    return XB_OK;
}

int64_t ld_of(int64_t n) { return (n + 63) / 64 * 64; }

// Per-SpMV CUDA-event timing (opt.timing): pairs of events around each SpMV.
struct SpmvTimer {
    xb_plan *p;
    bool on;
    cudaStream_t s;
    std::vector<cudaEvent_t> ev;
    size_t used = 0;
    double ms = 0.0;
    SpmvTimer(xb_plan *p_, bool on_, cudaStream_t s_) : p(p_), on(on_), s(s_) {}
    ~SpmvTimer() {
        for (auto e : ev) cudaEventDestroy(e);
    }
    void begin() {
        if (!on) return;
        if (used + 2 > ev.size()) {
            if (ev.size() >= 8192) {
                flush();
            } else {
                for (int i = 0; i < 256; i++) {
                    cudaEvent_t e;
                    cudaEventCreate(&e);
                    ev.push_back(e);
                }
            }
        }
        cudaEventRecord(ev[used], s);
    }
    void end() {
        if (!on) return;
        cudaEventRecord(ev[used + 1], s);
        used += 2;
    }
    void flush() {
        if (!on || used == 0) return;
        cudaStreamSynchronize(s);
        for (size_t i = 0; i + 1 < used; i += 2) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
            ms += t;
        }
        used = 0;
    }
};

struct Acct {
    double bytes = 0.0;
    int spmv = 0;
    double mem = 0.0;  // largest workspace the solve requested
};

struct Spmv {
    xb_plan *p;
    int variant, block, ipt;
};

// ---- FP64 GMRES(m) ------------------------------------------------------------------

int gmres_fp64(xb_plan *p, const double *b, double *x, const xb_options &o, xb_info &inf,
               cudaStream_t s, Acct &ac, SpmvTimer &tm, clk::time_point t0, int iter_budget) {
    const int64_t n = p->n;
    // basis capacity: m, or up to m_max when the restart rule may grow m
    const int M = o.dafrt ? std::max(o.m, std::min(std::max(o.m_max, o.m), 512)) : o.m;
    int m = std::min(o.m, M);
    const int64_t ld = ld_of(n);
    const bool prec = o.precond == XB_PRECOND_ILU0;
    const size_t vbytes = (size_t)(M + 1 + (prec ? 2 : 0)) * ld * sizeof(double);
    XB_TRY(xb::ensure_work(p, vbytes + xb::gm_doubles(M) * sizeof(double) + 256));
    ac.mem = std::max(ac.mem, (double)(vbytes + xb::gm_doubles(M) * sizeof(double) + 256));
    double *V = static_cast<double *>(p->d_work);
    // right preconditioning: tz = M^{-1} v_j before the SpMV; tu = V y before x += M^{-1} tu
    double *tz = V + (size_t)(M + 1) * ld, *tu = tz + ld;
    xb::GmDev st = xb::gm_layout(V + (size_t)(M + 1 + (prec ? 2 : 0)) * ld, M);
    if (prec) XB_TRY(xb::ensure_ilu(p, s));
    const double prec_b = prec ? xb::ilu_apply_bytes(p) : 0.0;
    const double spmv_b = xb::spmv_alg_bytes(p, false, 8);

    XB_TRY(xb::vnrm2(p, n, b, st.misc + xb::GM_BNORM, s));
    XB_TRY(peek(p, st.misc + xb::GM_BNORM, 1, s));
    const double bnorm = p->h_pin[0];
    ac.bytes += 8.0 * n;
    if (bnorm == 0.0) {
        XB_TRY(xb::vfill(n, 0.0, x, s));
        inf.res_true = 0.0;
        inf.m_final = m;
        return XB_OK;
    }
    const int window = std::max(1, o.dafrt_window);
    std::vector<double> samp(window);
    int K = 0, iters = 0, restarts = 0, faults = 0, status = XB_OK;
    bool claimed = false;
    double tau = o.tol, res_true = 0.0, res_impl = 0.0;
    const int check = std::max(1, o.check_every);
    int ortho = xb::ortho_choice(o.ortho, o.tol, false);
    for (;;) {
        // true residual r = b - A x into V_0, then start the cycle
        XB_TRY(xb::residual(p, b, x, V, s));
        ac.bytes += 16.0 * n + xb::spmv_alg_bytes(p, true, 8);
        ac.spmv++;
        XB_TRY(xb::gm_cycle_init(p, st, n, V, tau, s));
        ac.bytes += 8.0 * n;
        XB_TRY(peek(p, st.misc, xb::GM_NMISC, s));
        if (prec) XB_TRY(xb::ilu_check(p));  // a preconditioner wait ran out: stop here
        res_true = p->h_pin[xb::GM_RES];
        if (res_true <= o.tol) {
            status = XB_OK;
            break;
        }
        if (iters >= iter_budget) {
            status = XB_ENOCONV;
            break;
        }
        if (secs_since(t0) > o.maxtime_s) {
            status = XB_ENOCONV;
            break;
        }
        if (claimed && !o.fault_check) {  // stop at the claim: fault convergence
            faults++;
            status = XB_EFAULT;
            break;
        }
        if (claimed) {  // fault convergence: the implicit residual lied
            faults++;
            tau *= o.tol / res_true;
            ortho = xb::ortho_choice(o.ortho, o.tol, true);
            p->h_pin[32] = tau;
            XB_CUDA(cudaMemcpyAsync(st.misc + xb::GM_TAU, p->h_pin + 32, sizeof(double),
                                    cudaMemcpyHostToDevice, s));
        }
        claimed = false;
        if (o.dafrt && restarts > 0) {
            samp[K++] = res_true;
            if (K == window) {
                if (xb_dafrt(window, samp.data(), o.dafrt_theta)) m = std::min(m + o.dafrt_dm, M);
                K = 0;
            }
        }
        int launched = 0;
        double stop = 0.0;
        for (int j = 0; j < m; j++) {
            const double *src = V + (size_t)j * ld;
            if (prec) {
                XB_TRY(xb::ilu_apply(p, src, tz, s));
                ac.bytes += prec_b;
                src = tz;
            }
            tm.begin();
            XB_TRY(xb::spmv_launch_dalpha(p, o.variant, o.block, o.ipt, st.sc + j, src,
                                          V + (size_t)(j + 1) * ld, s));
            tm.end();
            ac.bytes += spmv_b;
            ac.spmv++;
            XB_TRY(xb::gm_ortho_step<double>(p, st, n, V, ld, V + (size_t)(j + 1) * ld, j, ortho,
                                             s));
            ac.bytes += 8.0 * n * xb::ortho_passes(ortho, j);
            launched++;
            const bool last = (j == m - 1) || (iters + launched >= iter_budget);
            if ((j + 1) % check == 0 || last) {
                XB_TRY(peek(p, st.misc, xb::GM_NMISC, s));
                stop = p->h_pin[xb::GM_STOP];
                if (stop != 0.0 || last) break;
                if (secs_since(t0) > o.maxtime_s) break;
            }
        }
        XB_TRY(peek(p, st.misc, xb::GM_NMISC, s));
        stop = p->h_pin[xb::GM_STOP];
        const int k = (int)p->h_pin[xb::GM_K];
        res_impl = p->h_pin[xb::GM_RES];
        iters += (stop != 0.0) ? (stop == 2.0 ? k + 1 : k) : launched;
        if (stop == 2.0) {
            status = XB_EBREAKDOWN;
            xb::set_error(XB_EBREAKDOWN, "GMRES: zero pivot in the Hessenberg matrix (singular A)");
            break;
        }
        if (stop == 1.0) claimed = true;
        if (k > 0 && prec) {
            XB_TRY(xb::vfill(n, 0.0, tu, s));
            XB_TRY(xb::gm_update<double, double>(p, st, n, V, ld, k, tu, s));
            XB_TRY(xb::ilu_apply(p, tu, tz, s));
            XB_TRY(xb::vaxpy(n, 1.0, tz, x, s));
            ac.bytes += 8.0 * n * k + 24.0 * n + prec_b + 24.0 * n;
        } else if (k > 0) {
            XB_TRY(xb::gm_update<double, double>(p, st, n, V, ld, k, x, s));
            ac.bytes += 8.0 * n * k + 16.0 * n;
        }
        restarts++;
    }
    inf.iters += iters;
    inf.restarts += restarts;
    inf.m_final = m;
    inf.faults += faults;
    inf.ortho_used = ortho;
    inf.res_true = res_true;
    inf.res_implicit = res_impl;
    return status;
}

// ---- FP32 inner GMRES(m) from d = 0 ---------------------------------------------------

int gmres_f32_inner(xb_plan *p, const float *r32, float *d, float *V, int64_t ld, xb::GmDev st,
                    int m, double tol_in, int maxit, int ortho, const xb_options &o, Acct &ac,
                    SpmvTimer &tm, int *steps, cudaStream_t s) {
    const int64_t n = p->n;
    const double spmv_b = xb::spmv_alg_bytes(p, false, 4);
    *steps = 0;
    XB_CUDA(cudaMemsetAsync(d, 0, n * sizeof(float), s));
    bool first = true;
    const int check = std::max(1, o.check_every);
    while (*steps < maxit) {
        // r_in = r32 - A32 d (into V_0); for d = 0 this is r32 itself
        XB_CUDA(cudaMemcpyAsync(V, r32, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
        ac.bytes += 8.0 * n;
        if (!first) {
            tm.begin();
            XB_TRY(xb::spmv_launch_f32(p, o.variant, o.block, o.ipt, -1.0f, d, 1.0f, V, s));
            tm.end();
            ac.bytes += xb::spmv_alg_bytes(p, true, 4);
            ac.spmv++;
        }
        if (first) {
            // inner residuals are relative to ||r32||: store it as the cycle's BNORM
            XB_TRY(xb::gm_cycle_init_f32(p, st, n, V, tol_in, s));
            XB_CUDA(cudaMemcpyAsync(st.misc + xb::GM_BNORM, st.misc + xb::GM_BETA, sizeof(double),
                                    cudaMemcpyDeviceToDevice, s));
        }
        XB_TRY(xb::gm_cycle_init_f32(p, st, n, V, tol_in, s));
        ac.bytes += 4.0 * n;
        XB_TRY(peek(p, st.misc, xb::GM_NMISC, s));
        const double rel = p->h_pin[xb::GM_RES];
        if (p->h_pin[xb::GM_BETA] == 0.0 || rel <= tol_in) break;
        first = false;
        int launched = 0;
        double stop = 0.0;
        for (int j = 0; j < m; j++) {
            tm.begin();
            XB_TRY(xb::spmv_launch_dalpha_f32(p, o.variant, o.block, o.ipt, st.scf + j,
                                              V + (size_t)j * ld, V + (size_t)(j + 1) * ld, s));
            tm.end();
            ac.bytes += spmv_b;
            ac.spmv++;
            XB_TRY(xb::gm_ortho_step<float>(p, st, n, V, ld, V + (size_t)(j + 1) * ld, j, ortho,
                                            s));
            ac.bytes += 4.0 * n * xb::ortho_passes(ortho, j);
            launched++;
            const bool last = (j == m - 1) || (*steps + launched >= maxit);
            if ((j + 1) % check == 0 || last) {
                XB_TRY(peek(p, st.misc, xb::GM_NMISC, s));
                stop = p->h_pin[xb::GM_STOP];
                if (stop != 0.0 || last) break;
            }
        }
        XB_TRY(peek(p, st.misc, xb::GM_NMISC, s));
        stop = p->h_pin[xb::GM_STOP];
        const int k = (int)p->h_pin[xb::GM_K];
        *steps += (stop != 0.0) ? k : launched;
        if (k > 0) {
            XB_TRY(xb::gm_update<float, float>(p, st, n, V, ld, k, d, s));
            ac.bytes += 4.0 * n * k + 8.0 * n;
        }
        if (stop != 0.0) break;  // converged (or breakdown: the outer loop judges)
    }
    return XB_OK;
}

int gmres_mixed(xb_plan *p, const double *b, double *x, const xb_options &o, xb_info &inf,
                cudaStream_t s, Acct &ac, SpmvTimer &tm, clk::time_point t0) {
    (void)tm;
    const int64_t n = p->n;
    const int M = o.m;
    const int m = o.m;
    const int64_t ld = ld_of(n);
    XB_TRY(xb::ensure_val32(p, s));
    const size_t vbytes = (size_t)(M + 1) * ld * sizeof(float);
    const size_t need = vbytes + xb::gm_doubles(M) * sizeof(double) + (size_t)ld * 8 +
                        2 * (size_t)ld * 4 + 64 * sizeof(double) + 1024;
    XB_TRY(xb::ensure_work(p, need));
    ac.mem = std::max(ac.mem, (double)need);
    char *w = static_cast<char *>(p->d_work);
    float *V = reinterpret_cast<float *>(w);
    w += vbytes;
    xb::GmDev st = xb::gm_layout(reinterpret_cast<double *>(w), M);
    w += xb::gm_doubles(M) * sizeof(double);
    double *r = reinterpret_cast<double *>(w);
    w += (size_t)ld * 8;
    float *r32 = reinterpret_cast<float *>(w);
    w += (size_t)ld * 4;
    float *d = reinterpret_cast<float *>(w);
    w += (size_t)ld * 4;
    double *sc = reinterpret_cast<double *>(w);  // [0] ||b||, [1] ||r||

    XB_TRY(xb::vnrm2(p, n, b, sc, s));
    XB_TRY(peek(p, sc, 1, s));
    const double bnorm = p->h_pin[0];
    ac.bytes += 8.0 * n;
    inf.m_final = m;
    if (bnorm == 0.0) {
        XB_TRY(xb::vfill(n, 0.0, x, s));
        inf.res_true = 0.0;
        return XB_OK;
    }
    int outer = 0, slow = 0, inner_total = 0, status = XB_OK;
    double prev = INFINITY, res = 0.0;
    for (;;) {
        XB_TRY(xb::residual(p, b, x, r, s));
        ac.bytes += 16.0 * n + xb::spmv_alg_bytes(p, true, 8);
        ac.spmv++;
        XB_TRY(xb::vnrm2(p, n, r, sc + 1, s));
        ac.bytes += 8.0 * n;
        XB_TRY(peek(p, sc + 1, 1, s));
        const double rn = p->h_pin[0];
        res = rn / bnorm;
        if (res <= o.tol) {
            status = XB_OK;
            break;
        }
        if (outer >= o.max_outer || secs_since(t0) > o.maxtime_s) {
            status = XB_ENOCONV;
            break;
        }
        slow = (rn > 0.5 * prev) ? slow + 1 : 0;
        if (o.ir_fallback && slow >= 2) {  // safeguard (option): finish in FP64
            xb_info fin;
            std::memset(&fin, 0, sizeof fin);
            inf.fallback = 1;
            status = gmres_fp64(p, b, x, o, fin, s, ac, tm, t0, o.maxiter);
            inf.iters += fin.iters;
            inf.restarts += fin.restarts;
            inf.faults += fin.faults;
            res = fin.res_true;
            // FP64 workspace may have replaced ours; nothing below uses it.
            break;
        }
        prev = rn;
        XB_TRY(xb::cast_f64_to_f32_scaled(n, r, sc + 1, r32, s));
        ac.bytes += 12.0 * n;
        int steps = 0;
        // the inner solve's accuracy target is tol_inner: the policy decides on it
        const int ortho_in = xb::ortho_choice(o.ortho, o.tol_inner, inf.faults > 0);
        inf.ortho_used = ortho_in;
        XB_TRY(gmres_f32_inner(p, r32, d, V, ld, st, m, o.tol_inner, o.maxiter_inner, ortho_in, o,
                               ac, tm, &steps, s));
        inner_total += steps;
        XB_TRY(xb::add_scaled_f32(n, x, sc + 1, d, s));
        ac.bytes += 20.0 * n;
        outer++;
    }
    inf.outer = outer;
    inf.inner_iters = inner_total;
    inf.res_true = res;
    return status;
}

// ---- BiCGStab ----------------------------------------------------------------------------

int bicgstab_run(xb_plan *p, const double *b, double *x, const xb_options &o, xb_info &inf,
                 cudaStream_t s, Acct &ac, SpmvTimer &tm, clk::time_point t0) {
    const int64_t n = p->n;
    const int64_t ld = ld_of(n);
    const bool prec = o.precond == XB_PRECOND_ILU0;
    const size_t nv = prec ? 8 : 6;
    XB_TRY(xb::ensure_work(p, nv * (size_t)ld * sizeof(double) + 64 * sizeof(double)));
    ac.mem = std::max(ac.mem, (double)(nv * (size_t)ld * sizeof(double) + 64 * sizeof(double)));
    double *r = static_cast<double *>(p->d_work);
    double *rh = r + ld, *pv = rh + ld, *v = pv + ld, *sv = v + ld, *t = sv + ld;
    // right preconditioning: ph = M^{-1} p and sh = M^{-1} s feed the SpMVs and x
    double *ph = prec ? t + ld : pv, *sh = prec ? t + 2 * ld : sv;
    double *sc = t + (prec ? 3 : 1) * ld;
    if (prec) XB_TRY(xb::ensure_ilu(p, s));
    const double prec_b = prec ? xb::ilu_apply_bytes(p) : 0.0;
    const double spmv_b = xb::spmv_alg_bytes(p, false, 8);

    XB_TRY(xb::vnrm2(p, n, b, sc + xb::BI_N, s));
    XB_TRY(peek(p, sc + xb::BI_N, 1, s));
    const double bnorm = p->h_pin[0];
    ac.bytes += 8.0 * n;
    if (bnorm == 0.0) {
        XB_TRY(xb::vfill(n, 0.0, x, s));
        inf.res_true = 0.0;
        return XB_OK;
    }
    int iters = 0, restarts = 0, faults = 0, status = XB_OK;
    bool claimed = false;
    double tau = o.tol, res_true = 0.0, res_rec = 0.0;
    const int check = std::max(1, o.check_every);
    for (;;) {
        XB_TRY(xb::residual(p, b, x, r, s));
        ac.bytes += 16.0 * n + xb::spmv_alg_bytes(p, true, 8);
        ac.spmv++;
        XB_TRY(xb::vnrm2(p, n, r, sc + xb::BI_N + 1, s));
        ac.bytes += 8.0 * n;
        XB_TRY(peek(p, sc + xb::BI_N + 1, 1, s));
        if (prec) XB_TRY(xb::ilu_check(p));  // a preconditioner wait ran out: stop here
        res_true = p->h_pin[0] / bnorm;
        if (res_true <= o.tol) {
            status = XB_OK;
            break;
        }
        if (iters >= o.maxiter || secs_since(t0) > o.maxtime_s) {
            status = XB_ENOCONV;
            break;
        }
        if (claimed && !o.fault_check) {  // stop at the claim: fault convergence
            faults++;
            status = XB_EFAULT;
            break;
        }
        if (claimed) {
            faults++;
            tau *= o.tol / res_true;
            restarts++;
        } else if (iters > 0) {
            restarts++;
        }
        claimed = false;
        XB_TRY(xb::vcopy(n, r, rh, s));
        XB_TRY(xb::vfill(n, 0.0, pv, s));
        XB_TRY(xb::vfill(n, 0.0, v, s));
        ac.bytes += 32.0 * n;
        const double tb = tau * bnorm;
        XB_TRY(xb::bi_init(p, sc, n, r, tb * tb, s));
        ac.bytes += 8.0 * n;
        int flag = 0;
        while (iters < o.maxiter) {
            iters++;
            XB_TRY(xb::bi_p_update(sc, n, r, pv, v, s));
            if (prec) XB_TRY(xb::ilu_apply(p, pv, ph, s));
            tm.begin();
            XB_TRY(xb::spmv_launch(p, o.variant, o.block, o.ipt, 1.0, ph, 0.0, v, s));
            tm.end();
            XB_TRY(xb::bi_sigma(p, sc, n, rh, v, s));
            XB_TRY(xb::bi_s_update(p, sc, n, r, v, sv, s));
            if (prec) XB_TRY(xb::ilu_apply(p, sv, sh, s));
            tm.begin();
            XB_TRY(xb::spmv_launch(p, o.variant, o.block, o.ipt, 1.0, sh, 0.0, t, s));
            tm.end();
            XB_TRY(xb::bi_omega(p, sc, n, t, sv, s));
            XB_TRY(xb::bi_xr_update(p, sc, n, x, ph, sv, sh, t, r, rh, s));
            ac.bytes += 2 * spmv_b + 144.0 * n + (prec ? 2.0 * prec_b : 0.0);
            ac.spmv += 2;
            if (iters % check == 0 || iters >= o.maxiter) {
                XB_TRY(peek(p, sc, xb::BI_N, s));
                if (prec) XB_TRY(xb::ilu_check(p));
                flag = (int)p->h_pin[xb::BI_FLAG];
                res_rec = std::sqrt(p->h_pin[xb::BI_RNORM2]) / bnorm;
                if (flag != 0) break;
                if (secs_since(t0) > o.maxtime_s) break;
            }
        }
        if (flag == 1) {
            claimed = true;
            continue;
        }
        if (flag >= 2) {  // breakdown: accept only if the true residual is small
            XB_TRY(xb::residual(p, b, x, r, s));
            XB_TRY(xb::vnrm2(p, n, r, sc + xb::BI_N + 1, s));
            XB_TRY(peek(p, sc + xb::BI_N + 1, 1, s));
            res_true = p->h_pin[0] / bnorm;
            status = (res_true <= o.tol) ? XB_OK : XB_EBREAKDOWN;
            if (status != XB_OK) xb::set_error(XB_EBREAKDOWN, "BiCGStab breakdown (code %d)", flag);
            break;
        }
        // iteration or time limit inside the recurrence: loop back for the true check
    }
    inf.iters = iters;
    inf.restarts = restarts;
    inf.faults = faults;
    inf.res_true = res_true;
    inf.res_implicit = res_rec;
    return status;
}

// Whether gmres_solve may run the system as one persistent launch: small, and
// options the persistent kernels implement exactly as gmres_fp64 does.
bool small_system(const xb_plan *p, const xb_options &o) {
    if (p->n < 1 || p->n > o.small_n || p->sym) return false;
    if (o.precision != XB_PREC_FP64 || o.precond != XB_PRECOND_NONE || !o.fault_check) return false;
    if (o.ortho != XB_ORTHO_MGS && o.ortho != XB_ORTHO_BCGS) return false;
    // the persistent kernel's restart rule judges windows of 5 samples, m += 5
    if (o.dafrt && (o.dafrt_window != 5 || o.dafrt_dm != 5)) return false;
    const int mmax = o.dafrt ? std::max(o.m, o.m_max) : o.m;
    return o.m >= 1 && mmax <= XB_BATCH_MAX_M;
}

int check_args(xb_plan *p, const double *b, double *x, const xb_options &o) {
    if (!p) return xb::set_error(XB_EINVAL, "solve: NULL plan");
    if (p->n > 0 && (!b || !x)) return xb::set_error(XB_EINVAL, "solve: NULL vector");
    if (!(o.tol > 0.0)) return xb::set_error(XB_EINVAL, "solve: tol must be > 0");
    if (o.m < 1 || o.m > 512) return xb::set_error(XB_EINVAL, "solve: m=%d not in [1,512]", o.m);
    if (o.variant != XB_VAR_AUTO && !xb::variant_fits(p, o.variant))
        return xb::set_error(XB_EINVAL, "solve: SpMV variant %d does not fit the storage", o.variant);
    if (o.ortho < XB_ORTHO_MGS || o.ortho > XB_ORTHO_AUTO)
        return xb::set_error(XB_EINVAL, "solve: unknown orthogonalisation %d", o.ortho);
    if (o.precond != XB_PRECOND_NONE && o.precond != XB_PRECOND_ILU0)
        return xb::set_error(XB_EINVAL, "solve: unknown preconditioner %d", o.precond);
    if (o.precond == XB_PRECOND_ILU0 && (p->sym || o.precision != XB_PREC_FP64 || !p->subs.empty()))
        return xb::set_error(XB_EINVAL, "solve: ILU(0) needs general CRS (below 2^31 - 64 "
                                        "non-zeros) and FP64 precision");
    return XB_OK;
}

// The numerical computation policy (Sec. 2.3.2, 3.3): settings it fixes.
void apply_policy(xb_options &o, const xb_plan *p) {
    switch (o.policy) {
        case XB_POLICY_TIME:
        case XB_POLICY_ACCURACY:
            o.tuner = XB_TUNER_EXHAUSTIVE;
            o.variant = XB_VAR_AUTO;
            o.dafrt = 1;
            o.m_max = std::max(std::max(o.m_max, o.m), 128);
            if (o.policy == XB_POLICY_TIME) {
                o.ortho = xb::ortho_choice(XB_ORTHO_AUTO, o.tol, false);
                o.fault_check = 0;
            } else {
                o.ortho = XB_ORTHO_AUTO;
                o.fault_check = 1;
            }
            break;
        case XB_POLICY_MEMORY:
            o.tuner = XB_TUNER_NONE;
            o.variant = p && p->sym ? XB_VAR_SYM_ATOMIC : XB_VAR_ROW;
            o.block = 0;
            o.m = 10;
            o.dafrt = 0;
            o.ortho = XB_ORTHO_MGS;
            o.precision = XB_PREC_FP64;
            o.fault_check = 0;
            break;
        case XB_POLICY_STABLE:
            o.tuner = XB_TUNER_NONE;
            o.variant = XB_VAR_AUTO;
            o.dafrt = 0;
            o.ortho = XB_ORTHO_MGS;
            o.fault_check = 0;
            break;
        default:
            break;
    }
}

}  // namespace

namespace xb {

// Device bytes of the plan data the SpMV variant reads besides the matrix.
double spmv_meta_bytes(const xb_plan *p, int variant, int block, int ipt) {
    double b = 0.0;
    for (const auto &sb : p->subs) b += spmv_meta_bytes(sb.plan, variant, block, ipt);
    if (variant == XB_VAR_NNZ || variant == XB_VAR_SYM_TILE) {
        for (const auto &t : p->tiles)
            if (t.block == block && t.ipt == ipt) b += 4.0 * (t.ntiles + 1);
    } else if (variant == XB_VAR_SYM_PART) {
        for (const auto &t : p->tiles)
            if (t.block == block && t.ipt == ipt) b += 4.0 * (t.ntiles + 1);
        for (const auto &t : p->s3)
            if (t.block == block && t.ipt == ipt)
                b += 4.0 * (t.ntiles + 1 + 2.0 * t.nslots + 2.0 * t.ngran + 1) +
                     8.0 * t.nslots * xb::kS3Gran;
    } else if (variant == XB_VAR_BCSR) {
        for (const auto &t : p->bcsr)
            if (t.r == ipt)
                b += 4.0 * (t.nbr + 1) + 4.0 * t.nblocks + 8.0 * t.nblocks * t.r * t.r +
                     (t.d_val32 ? 4.0 * t.nblocks * t.r * t.r : 0.0);
    } else if (variant == XB_VAR_SELL) {
        for (const auto &t : p->sells)
            if (t.sigma == 32 * ipt)
                b += 8.0 * (t.nslices + 1) + 256.0 * t.nslices + 12.0 * t.total +
                     (t.d_val32 ? 4.0 * t.total : 0.0);
    } else if (variant == XB_VAR_SEGSCAN) {
        b += 4.0 * ((p->nnz + 31) / 32 + 1);
        for (const auto &c : p->bss.copies)  // the BSS data format copy
            if (c.ipt == ipt) b += 12.0 * c.total + (c.d_val32 ? 4.0 * c.total : 0.0);
        if (p->bss.d_ne_rows) b += 4.0 * p->bss.n_ne + 4.0 * (p->bss.n_ne + 1);
        for (const auto &g : p->segs)
            if (g.block == block && g.ipt == ipt) b += 4.0 * (g.nblk + 1) + 12.0 * g.nblk;
    }
    return b;
}

}  // namespace xb

namespace {

template <typename F>
int run_solver(xb_plan *p, const double *b, double *x, const xb_options *opt, xb_info *info,
               void *stream, F body) {
    xb_options o;
    if (opt) o = *opt;
    else xb_options_default(&o);
    if (o.policy < XB_POLICY_NONE || o.policy > XB_POLICY_STABLE)
        return xb::set_error(XB_EINVAL, "solve: unknown policy %d", o.policy);
    apply_policy(o, p);
    xb_info inf;
    std::memset(&inf, 0, sizeof inf);
    int st = check_args(p, b, x, o);
    if (st == XB_OK) {
        cudaStream_t s = (cudaStream_t)stream;
        Acct ac;
        SpmvTimer tm(p, o.timing != 0, s);
        const auto t0 = clk::now();
        if (p->n == 0) {
            st = XB_OK;
        } else {
            st = body(o, inf, s, ac, tm, t0);
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess && st == XB_OK) st = xb::cuda_error(e, "solve");
            if (o.precond == XB_PRECOND_ILU0 && st != XB_ECUDA) {
                const int ci = xb::ilu_check(p);
                if (ci != XB_OK) st = ci;
            }
        }
        tm.flush();
        inf.t_solve_s = secs_since(t0);
        inf.spmv_ms = tm.ms;
        inf.bytes_alg = ac.bytes;
        inf.spmv_calls = ac.spmv;
        inf.variant_used = o.variant == XB_VAR_AUTO ? p->variant : o.variant;
        inf.block_used = o.block > 0 ? o.block : p->block;
        inf.ipt_used = o.ipt > 0 ? o.ipt : p->ipt;
        inf.mem_bytes = ac.mem + xb::spmv_meta_bytes(p, inf.variant_used, inf.block_used, inf.ipt_used) +
                        (o.precision == XB_PREC_MIXED ? 4.0 * p->nnz64 : 0.0) +
                        (o.precond == XB_PRECOND_ILU0 ? 8.0 * p->nnz64 + 12.0 * p->n : 0.0);
        if (st == XB_EFAULT)
            xb::set_error(XB_EFAULT, "fault convergence: implicit residual met tol, "
                                     "||b-Ax||/||b|| = %.3e", inf.res_true);
        if (st == XB_ENOCONV)
            xb::set_error(XB_ENOCONV, "not converged: ||b-Ax||/||b|| = %.3e > tol %.1e", inf.res_true,
                          o.tol);
    }
    inf.status = st;
    if (info) *info = inf;
    return st;
}

}  // namespace

extern "C" {

int gmres_solve(xb_plan *p, const double *b, double *x, const xb_options *opt, xb_info *info,
                void *stream) {
    return run_solver(p, b, x, opt, info, stream,
                      [&](const xb_options &o, xb_info &inf, cudaStream_t s, Acct &ac,
                          SpmvTimer &tm, clk::time_point t0) {
                          if (o.tuner == XB_TUNER_EXHAUSTIVE) {
                              int r = xb_tune_exhaustive(p, nullptr, s);
                              if (r != XB_OK) return r;
                          }
                          if (o.precision == XB_PREC_MIXED)
                              return gmres_mixed(p, b, x, o, inf, s, ac, tm, t0);
                          if (small_system(p, o)) {
                              double by = 0.0;
                              // the whole system in one cluster's shared memory
                              bool ran = false;
                              int r = xb::resident_gmres(p, b, x, o, inf, &by, s, &ran);
                              if (ran || r != XB_OK) {
                                  ac.bytes += by;
                                  return r;
                              }
                              // else the batched kernel's single-system path (thread
                              // per row, or warp-sized row blocks when rows are long),
                              // whose cluster streams the basis from L2: only while a
                              // step's work (about nnz + m n) stays small does it beat
                              // the multi-launch step (measured: n = 4096 stencil 57
                              // vs 148 us per step; n = 20,000 power-law rows 592 vs
                              // 168 us on one CTA)
                              if ((double)p->nnz + (double)o.m * p->n <= 32.0 * o.small_n) {
                                  const int mode = p->max_row > 32 ? 1 : 0;
                                  r = xb::batch_single(p, b, x, o, mode, inf, &by, s);
                                  ac.bytes += by;
                                  return r;
                              }
                          }
                          return gmres_fp64(p, b, x, o, inf, s, ac, tm, t0, o.maxiter);
                      });
}

int bicgstab_solve(xb_plan *p, const double *b, double *x, const xb_options *opt, xb_info *info,
                   void *stream) {
    return run_solver(p, b, x, opt, info, stream,
                      [&](const xb_options &o, xb_info &inf, cudaStream_t s, Acct &ac,
                          SpmvTimer &tm, clk::time_point t0) {
                          if (o.tuner == XB_TUNER_EXHAUSTIVE) {
                              int r = xb_tune_exhaustive(p, nullptr, s);
                              if (r != XB_OK) return r;
                          }
                          return bicgstab_run(p, b, x, o, inf, s, ac, tm, t0);
                      });
}

}  // extern "C"
