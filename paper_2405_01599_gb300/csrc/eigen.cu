// Restarted Lanczos (symmetric) and restarted Arnoldi (general) eigensolvers
// (OpenATI_EIGENSOLVE, Sec. 2.2 / 4.3), both restarted in Krylov-Schur form
// with full re-orthogonalisation on the device.
//
// Lanczos: the nev largest eigenvalues, thick restart.
// A cycle extends the orthonormal basis v_0..v_m: w = A v_j (the plan's SpMV,
// general or symmetric storage), w orthogonalised against every basis vector
// with DGKS on the device (the coefficients are column j of the projected
// matrix T = V^T A V), v_{j+1} = w / ||w|| scaled on the device.  The m x m
// projected matrix is symmetrised and diagonalised on the host (cyclic Jacobi;
// m <= 512, so this is the small dense step, as in any Lanczos code); Ritz
// pair i has residual |beta_m s_{m-1,i}|.  A restart keeps the
// k = nev + (m - nev)/2 leading Ritz vectors (V S_k, one device pass over the
// basis), moves v_m to v_k, and T restarts as diag(theta) with row k holding
// beta_m s_{m-1,i}.
#include "deig.cuh"
#include "krylov.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

constexpr int kRotC = 8;  // outputs per thread in the basis rotation

// x *= 1 / *h (h on the device: the norm just computed by the last GS pass)
__global__ void k_scale_inv(int64_t n, double *__restrict__ x, const double *__restrict__ h) {
    const double inv = 1.0 / *h;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] *= inv;
}

// Deterministic start vector: splitmix64 of the index, mapped to [-1, 1).
__global__ void k_start_vector(int64_t n, double *__restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long z = (unsigned long long)i + 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        x[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
}

// Y[c] = sum_{i < m} V[i] S[i][c] for the RC outputs c = c_base + RC * blockIdx.y + 0..RC-1
// of this CTA; S is m x kc column-major (leading dimension m), the CTA's RC
// columns staged in shared memory.  RC is exact (a tail of kc % kRotC columns
// gets its own instantiation): the kernel is bound by the FP64 FMA pipe, so
// no padded column is computed.
template <int RC>
__global__ void __launch_bounds__(256) k_rotate(int64_t n, int m, int c_base,
                                                const double *__restrict__ V, int64_t ld,
                                                const double *__restrict__ S,
                                                double *__restrict__ Y, int64_t ldy) {
    extern __shared__ double ss[];  // m x RC
    const int c0 = c_base + blockIdx.y * RC;
    for (int t = threadIdx.x; t < m * RC; t += blockDim.x) {
        const int i = t / RC, c = t % RC;
        ss[t] = S[(size_t)(c0 + c) * m + i];
    }
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        double acc[RC];
#pragma unroll
        for (int c = 0; c < RC; c++) acc[c] = 0.0;
        for (int i = 0; i < m; i++) {
            const double v = V[(size_t)i * ld + e];
#pragma unroll
            for (int c = 0; c < RC; c++) acc[c] = fma(v, ss[i * RC + c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < RC; c++) Y[(size_t)(c0 + c) * ldy + e] = acc[c];
    }
}

// Cyclic Jacobi eigen-decomposition of the symmetric m x m matrix a
// (row-major, destroyed): a = S diag(w) S^T with S column-major (column c
// holds eigenvector c, s[c * m + r]); pairs sorted by eigenvalue, largest first.
void jacobi_eig(int m, std::vector<double> &a, std::vector<double> &w, std::vector<double> &s) {
    s.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; i++) s[(size_t)i * m + i] = 1.0;
    double fro = 0.0;
    for (double v : a) fro += v * v;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int p = 0; p < m; p++)
            for (int q = p + 1; q < m; q++)
                off += 2.0 * a[(size_t)p * m + q] * a[(size_t)p * m + q];
        if (off == 0.0 || off <= 1e-30 * fro) break;
        for (int p = 0; p < m; p++)
            for (int q = p + 1; q < m; q++) {
                const double apq = a[(size_t)p * m + q];
                if (apq == 0.0) continue;
                const double theta = (a[(size_t)q * m + q] - a[(size_t)p * m + p]) / (2.0 * apq);
                const double t = std::copysign(1.0, theta) / (std::fabs(theta) +
                                                              std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                for (int r = 0; r < m; r++) {  // columns p, q
                    const double x = a[(size_t)r * m + p], y = a[(size_t)r * m + q];
                    a[(size_t)r * m + p] = c * x - sn * y;
                    a[(size_t)r * m + q] = sn * x + c * y;
                }
                for (int r = 0; r < m; r++) {  // rows p, q
                    const double x = a[(size_t)p * m + r], y = a[(size_t)q * m + r];
                    a[(size_t)p * m + r] = c * x - sn * y;
                    a[(size_t)q * m + r] = sn * x + c * y;
                }
                for (int r = 0; r < m; r++) {  // eigenvector columns p, q
                    const double x = s[(size_t)p * m + r], y = s[(size_t)q * m + r];
                    s[(size_t)p * m + r] = c * x - sn * y;
                    s[(size_t)q * m + r] = sn * x + c * y;
                }
            }
    }
    std::vector<int> ord(m);
    for (int i = 0; i < m; i++) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
        return a[(size_t)x * m + x] > a[(size_t)y * m + y];
    });
    w.resize(m);
    std::vector<double> s2((size_t)m * m);
    for (int c = 0; c < m; c++) {
        w[c] = a[(size_t)ord[c] * m + ord[c]];
        std::memcpy(&s2[(size_t)c * m], &s[(size_t)ord[c] * m], sizeof(double) * m);
    }
    s.swap(s2);
}

template <int RC>
void rotate_cols(int64_t n, int m, int c_base, int blocks, int gx, const double *V, int64_t ld,
                 const double *dS, double *Y, int64_t ldy, cudaStream_t s) {
    k_rotate<RC><<<dim3(gx, blocks), 256, (size_t)m * RC * sizeof(double), s>>>(n, m, c_base, V,
                                                                               ld, dS, Y, ldy);
}

// Y (kc columns, stride ldy) = V (m rows, stride ld) times the m x kc matrix dS.
int rotate(int64_t n, int m, int kc, const double *V, int64_t ld, const double *dS, double *Y,
           int64_t ldy, cudaStream_t s) {
    if (kc <= 0) return XB_OK;
    const int gx = std::max(1, (int)std::min<int64_t>((n + 255) / 256, (int64_t)xb::num_sms() * 4));
    const int full = kc / kRotC, c0 = full * kRotC;
    if (full) rotate_cols<kRotC>(n, m, 0, full, gx, V, ld, dS, Y, ldy, s);
    switch (kc - c0) {
    case 1: rotate_cols<1>(n, m, c0, 1, gx, V, ld, dS, Y, ldy, s); break;
    case 2: rotate_cols<2>(n, m, c0, 1, gx, V, ld, dS, Y, ldy, s); break;
    case 3: rotate_cols<3>(n, m, c0, 1, gx, V, ld, dS, Y, ldy, s); break;
    case 4: rotate_cols<4>(n, m, c0, 1, gx, V, ld, dS, Y, ldy, s); break;
    case 5: rotate_cols<5>(n, m, c0, 1, gx, V, ld, dS, Y, ldy, s); break;
    case 6: rotate_cols<6>(n, m, c0, 1, gx, V, ld, dS, Y, ldy, s); break;
    case 7: rotate_cols<7>(n, m, c0, 1, gx, V, ld, dS, Y, ldy, s); break;
    default: break;
    }
    XB_LAUNCHED("k_rotate");
    return XB_OK;
}

// Settings of one eigensolver run under a numerical computation policy
// (Sec. 2.3.2, 3.3): TIME and ACCURACY tune the SpMV and turn the restart rule
// on (m_max >= 128); MEMORY takes the SpMV without plan metadata and a fixed
// cycle of at most 20 (at least m_min); STABLE keeps the plan's SpMV and m.
// Every policy but NONE checks the true residuals of a claimed convergence;
// ACCURACY iterates on after a miss (outer loop).  The Gram-Schmidt choice is
// the solver's.
struct EigRun {
    int variant, block, ipt, m, m_max;
    bool check, outer;
};

int eig_policy(xb_plan *p, int policy, int m_min, int m, int m_max, void *stream, EigRun &r) {
    r = EigRun{p->variant, p->block, p->ipt, m, m_max, policy != XB_POLICY_NONE,
               policy == XB_POLICY_ACCURACY};
    switch (policy) {
        case XB_POLICY_TIME:
        case XB_POLICY_ACCURACY:
            XB_TRY(xb_tune_exhaustive(p, nullptr, stream));
            r.variant = p->variant;
            r.block = p->block;
            r.ipt = p->ipt;
            r.m_max = std::max<int>(m_max, (int)std::min<int64_t>(128, std::min<int64_t>(512, p->n)));
            break;
        case XB_POLICY_MEMORY:
            r.variant = p->sym ? XB_VAR_SYM_ATOMIC : XB_VAR_ROW;
            r.block = 256;
            r.ipt = 1;
            r.m = std::max(m_min, std::min(m, 20));
            r.m_max = r.m;
            break;
        case XB_POLICY_STABLE:
            r.m_max = m;
            break;
        default:
            break;
    }
    return XB_OK;
}

}  // namespace

extern "C" {

// Numerical computation policy as for xb_arnoldi below, except that every
// policy keeps DGKS: the thick restart takes the Ritz vectors of the
// symmetrised projected matrix, which is V^T A V only while V stays
// orthonormal, and a single Gram-Schmidt pass (MGS, BCGS) lets the loss of
// orthogonality grow by orders of magnitude per restart (measured on a random
// sparse symmetric matrix, n = 3000, m = 40: 1.5e-8, 1e-5, 1.5e-2 after the
// first three cycles with MGS, against 1e-14 with DGKS).
int xb_lanczos(xb_plan *p, int32_t nev, int32_t m, int32_t m_max, double theta, double tol,
               int32_t maxrestart, int32_t policy, const double *v0, double *evals,
               double *evecs, double *resid, int32_t *counts, double *stats, void *stream) {
    if (m_max < m) m_max = m;
    if (!p || nev < 1 || m <= nev || m_max > 512 || m_max > p->n || !(tol > 0.0) ||
        maxrestart < 0 || !evals || !resid || policy < XB_POLICY_NONE ||
        policy > XB_POLICY_STABLE)
        return xb::set_error(XB_EINVAL, "lanczos: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = p->n;
    EigRun run;
    XB_TRY(eig_policy(p, policy, nev + 1, m, m_max, stream, run));
    const int variant = run.variant, block = run.block, ipt = run.ipt;
    const bool check = run.check, outer = run.outer;
    m = run.m;
    m_max = run.m_max;
    const int ortho = XB_ORTHO_DGKS;
    const int64_t ld = (n + 63) / 64 * 64;
    const int M = m_max;  // basis capacity
    const int kmax = nev + (M - nev) / 2;
    const size_t vbytes = (size_t)(M + 1 + kmax) * ld * sizeof(double);
    const size_t gbytes = xb::gm_doubles(M) * sizeof(double) + (size_t)M * M * 8 +
                          (size_t)M * 8 + 256;
    const size_t cbytes = check ? (size_t)2 * ld * sizeof(double) : 0;  // one Ritz vector + A y
    const size_t need = vbytes + gbytes + cbytes;
    XB_TRY(xb::ensure_work(p, need));
    double *V = static_cast<double *>(p->d_work);
    double *Y = V + (size_t)(M + 1) * ld;
    double *gm = Y + (size_t)kmax * ld;
    xb::GmDev st = xb::gm_layout(gm, M);
    double *dS = gm + xb::gm_doubles(M);
    double *dres = dS + (size_t)M * M;
    double *XR = reinterpret_cast<double *>(((uintptr_t)(dres + M) + 255) / 256 * 256);
    double *TMP = XR + ld;
    // raw Gram-Schmidt state: unit scales, no Givens
    XB_CUDA(cudaMemsetAsync(gm, 0, xb::gm_doubles(M) * sizeof(double), s));
    std::vector<double> ones(M + 1, 1.0);
    XB_CUDA(cudaMemcpyAsync(st.sc, ones.data(), (M + 1) * sizeof(double), cudaMemcpyHostToDevice,
                            s));
    double misc[xb::GM_NMISC] = {0};
    misc[xb::GM_BNORM] = 1.0;
    misc[xb::GM_TAU] = -1.0;
    misc[xb::GM_RAW] = 1.0;
    XB_CUDA(cudaMemcpyAsync(st.misc, misc, sizeof misc, cudaMemcpyHostToDevice, s));
    const int sg = std::max(1, (int)std::min<int64_t>((n + 255) / 256, xb::num_sms() * 8LL));
    if (v0) XB_CUDA(cudaMemcpyAsync(V, v0, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else k_start_vector<<<sg, 256, 0, s>>>(n, V);
    XB_TRY(xb::vnrm2(p, n, V, st.y, s));  // y[0] holds ||v0|| (y is unused in raw mode)
    k_scale_inv<<<sg, 256, 0, s>>>(n, V, st.y);
    XB_LAUNCHED("k_scale_inv");

    std::vector<double> T((size_t)(M + 1) * (M + 1), 0.0), H((size_t)(M + 1) * M), a, w, S;
    std::vector<double> hres(nev);
    int k = 0, steps = 0, restarts = 0, status = XB_ENOCONV, K = 0, passes = 1;
    double beta = 0.0, samp[5], tol_in = tol, true_max = -1.0;
    auto ritz_vectors = [&](double *y, int64_t ly) -> int {
        XB_CUDA(cudaMemcpyAsync(dS, S.data(), (size_t)m * nev * sizeof(double),
                                cudaMemcpyHostToDevice, s));
        return rotate(n, m, nev, V, ld, dS, y, ly, s);
    };
    for (;;) {
        for (int j = k; j < m; j++) {
            double *vj = V + (size_t)j * ld, *wv = V + (size_t)(j + 1) * ld;
            XB_TRY(xb::spmv_launch(p, variant, block, ipt, 1.0, vj, 0.0, wv, s));
            XB_TRY(xb::gm_ortho_step<double>(p, st, n, V, ld, wv, j, ortho, s));
            k_scale_inv<<<sg, 256, 0, s>>>(n, wv, st.H + (size_t)j * (M + 1) + j + 1);
            steps++;
        }
        XB_CUDA(cudaMemcpyAsync(H.data(), st.H, H.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                s));
        XB_CUDA(cudaStreamSynchronize(s));
        for (int j = k; j < m; j++)
            for (int i = 0; i <= j + 1; i++)
                T[(size_t)i * (M + 1) + j] = H[(size_t)j * (M + 1) + i];
        beta = T[(size_t)m * (M + 1) + m - 1];
        bool broke = false;
        for (int j = k; j < m; j++)
            if (!(T[(size_t)(j + 1) * (M + 1) + j] > 0.0)) broke = true;
        if (broke) {
            status = XB_EBREAKDOWN;
            xb::set_error(XB_EBREAKDOWN, "lanczos: invariant subspace before %d steps", m);
            break;
        }
        a.assign((size_t)m * m, 0.0);
        for (int i = 0; i < m; i++)
            for (int j = 0; j < m; j++)
                a[(size_t)i * m + j] =
                    0.5 * (T[(size_t)i * (M + 1) + j] + T[(size_t)j * (M + 1) + i]);
        jacobi_eig(m, a, w, S);
        bool conv = true;
        for (int i = 0; i < nev; i++) {
            evals[i] = w[i];
            resid[i] = std::fabs(beta * S[(size_t)i * m + m - 1]);
            if (resid[i] > tol_in * std::fabs(w[i])) conv = false;
        }
        if (conv && check) {
            // true residuals ||A y - theta y|| of the claimed pairs (Sec. 3.3.2),
            // one Ritz vector at a time (two vectors of workspace)
            XB_CUDA(cudaMemcpyAsync(dS, S.data(), (size_t)m * nev * sizeof(double),
                                    cudaMemcpyHostToDevice, s));
            for (int i = 0; i < nev; i++) {
                const double *y = XR;
                XB_TRY(rotate(n, m, 1, V, ld, dS + (size_t)i * m, XR, ld, s));
                XB_TRY(xb::spmv_launch(p, variant, block, ipt, 1.0, y, 0.0, TMP, s));
                XB_TRY(xb::vaxpy(n, -w[i], y, TMP, s));
                XB_TRY(xb::vnrm2(p, n, TMP, dres + i, s));
            }
            XB_CUDA(cudaMemcpyAsync(hres.data(), dres, nev * sizeof(double),
                                    cudaMemcpyDeviceToHost, s));
            XB_CUDA(cudaStreamSynchronize(s));
            true_max = 0.0;
            for (int i = 0; i < nev; i++) true_max = std::max(true_max, hres[i] / std::fabs(w[i]));
            if (true_max <= tol) {
                status = XB_OK;
            } else if (!outer) {
                status = XB_EFAULT;
                xb::set_error(XB_EFAULT, "fault convergence: Ritz residual estimates met tol, "
                              "true relative residual %.3e", true_max);
            } else {
                tol_in *= tol / true_max;
                passes++;
                conv = false;
            }
            if (conv) {
                if (evecs) XB_TRY(ritz_vectors(evecs, n));
                break;
            }
        } else if (conv) {
            status = XB_OK;
            if (evecs) XB_TRY(ritz_vectors(evecs, n));
            break;
        }
        if (restarts >= maxrestart) {
            status = XB_ENOCONV;
            if (evecs) XB_TRY(ritz_vectors(evecs, n));
            break;
        }
        // restart rule (Eq. 1): worst relative residual of the wanted pairs,
        // judged every 5 samples; m grows by 5 when the residuals stagnate
        int m_next = m;
        if (m_max > m || K > 0) {
            double worst = 0.0;
            for (int i = 0; i < nev; i++) worst = std::max(worst, resid[i] / std::fabs(w[i]));
            samp[K++] = worst;
            if (K == 5) {
                if (xb_dafrt(5, samp, theta)) m_next = std::min(m + 5, m_max);
                K = 0;
            }
        }
        // thick restart with the leading Ritz vectors of this cycle
        k = nev + (m - nev) / 2;
        XB_CUDA(cudaMemcpyAsync(dS, S.data(), (size_t)m * k * sizeof(double),
                                cudaMemcpyHostToDevice, s));
        XB_TRY(rotate(n, m, k, V, ld, dS, Y, ld, s));
        XB_CUDA(cudaMemcpyAsync(V, Y, (size_t)k * ld * sizeof(double), cudaMemcpyDeviceToDevice,
                                s));
        XB_CUDA(cudaMemcpyAsync(V + (size_t)k * ld, V + (size_t)m * ld, ld * sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
        std::fill(T.begin(), T.end(), 0.0);
        for (int i = 0; i < k; i++) {
            T[(size_t)i * (M + 1) + i] = w[i];
            T[(size_t)k * (M + 1) + i] = beta * S[(size_t)i * m + m - 1];
        }
        m = m_next;
        restarts++;
    }
    if (counts) {
        counts[0] = steps;
        counts[1] = restarts;
        counts[2] = m;
        counts[3] = ortho;
        counts[4] = passes;
    }
    if (stats) {
        stats[0] = (double)need + xb::spmv_meta_bytes(p, variant, block, ipt);
        stats[1] = true_max;
    }
    XB_CUDA(cudaStreamSynchronize(s));
    return status;
}

// Restarted Arnoldi.  A cycle extends v_0..v_m as Lanczos does, with the
// caller's Gram-Schmidt variant; the coefficients fill the m x m projected
// matrix H.  On the host H = Z T Z^H (complex Schur form), reordered so that
// the wanted eigenvalues lead; Ritz pair i has residual |h_{m,m-1}| |e_m^T y_i|
// with y_i the unit eigenvector of H.  A restart keeps the real invariant
// subspace Q (m x k, orthonormal) of the k leading eigenvalues: V_k <- V_m Q
// (one device pass), v_k <- v_m, and H restarts as Q^T H Q with row k holding
// h_{m,m-1} e_m^T Q, so A V_k = V_k (Q^T H Q) + v_k (row k) holds again.
//
// Numerical computation policy (Sec. 2.3.2, 3.3; Fig. 9-11 run Arnoldi under
// each): TIME tunes the SpMV, turns the restart rule on (m_max >= 128) and
// takes the accuracy rule's Gram-Schmidt; MEMORY takes the SpMV without plan
// metadata and a short fixed cycle (m <= 20) with MGS; STABLE keeps the
// plan's SpMV and m, MGS; ACCURACY is TIME plus the outer loop of Sec. 3.3.2:
// when the estimates claim convergence the true residuals ||A y - theta y||
// are computed, and if one misses tol the iteration continues with the
// threshold narrowed by tol / (true residual) and DGKS.  Under TIME, MEMORY
// and STABLE the same check ends the run with XB_EFAULT instead.
int xb_arnoldi(xb_plan *p, int32_t nev, int32_t m, int32_t m_max, double theta, double tol,
               int32_t maxrestart, int32_t which, int32_t ortho, int32_t policy, const double *v0,
               double *evals_re, double *evals_im, double *evecs_re, double *evecs_im,
               double *resid, int32_t *counts, double *stats, void *stream) {
    if (m_max < m) m_max = m;
    if (!p || nev < 1 || m < nev + 2 || m_max > 512 || m_max > p->n || !(tol > 0.0) ||
        maxrestart < 0 || !evals_re || !evals_im || !resid ||
        (which != XB_EIG_LR && which != XB_EIG_LM) || ortho < XB_ORTHO_MGS ||
        ortho > XB_ORTHO_AUTO || policy < XB_POLICY_NONE || policy > XB_POLICY_STABLE)
        return xb::set_error(XB_EINVAL, "arnoldi: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = p->n;
    EigRun run;
    XB_TRY(eig_policy(p, policy, nev + 2, m, m_max, stream, run));
    const int variant = run.variant, block = run.block, ipt = run.ipt;
    const bool check = run.check, outer = run.outer;
    m = run.m;
    m_max = run.m_max;
    // Gram-Schmidt: the accuracy rule under TIME / ACCURACY, MGS under MEMORY
    // and STABLE, the argument (AUTO resolved) otherwise
    if (policy == XB_POLICY_TIME || policy == XB_POLICY_ACCURACY)
        ortho = xb::ortho_choice(XB_ORTHO_AUTO, tol, false);
    else if (policy == XB_POLICY_MEMORY || policy == XB_POLICY_STABLE)
        ortho = XB_ORTHO_MGS;
    else
        ortho = xb::ortho_choice(ortho, tol, false);
    const int64_t ld = (n + 63) / 64 * 64;
    const int M = m_max;
    const int kmax = std::min(M - 1, nev + (M - nev) / 2 + 1);
    const size_t vbytes = (size_t)(M + 1 + kmax) * ld * sizeof(double);
    // dS holds Q (m x k) or the real and imaginary Ritz coefficients (2 x m x nev);
    // dres the true residual norms; XR, XI, TMP one Ritz vector (real and
    // imaginary part) and A times it
    const size_t gbytes = xb::gm_doubles(M) * sizeof(double) + (size_t)2 * M * M * 8 +
                          (size_t)2 * M * 8 + 256;
    const size_t cbytes = check ? (size_t)3 * ld * sizeof(double) : 0;  // Re y, Im y, A y
    const size_t need = vbytes + gbytes + cbytes;
    XB_TRY(xb::ensure_work(p, need));
    double *V = static_cast<double *>(p->d_work);
    double *Y = V + (size_t)(M + 1) * ld;
    double *gm = Y + (size_t)kmax * ld;
    xb::GmDev st = xb::gm_layout(gm, M);
    double *dS = gm + xb::gm_doubles(M);
    double *dres = dS + (size_t)2 * M * M;
    double *XR = reinterpret_cast<double *>(((uintptr_t)(dres + 2 * M) + 255) / 256 * 256);
    double *XI = XR + ld, *TMP = XI + ld;
    XB_CUDA(cudaMemsetAsync(gm, 0, xb::gm_doubles(M) * sizeof(double), s));
    std::vector<double> ones(M + 1, 1.0);
    XB_CUDA(cudaMemcpyAsync(st.sc, ones.data(), (M + 1) * sizeof(double), cudaMemcpyHostToDevice,
                            s));
    double misc[xb::GM_NMISC] = {0};
    misc[xb::GM_BNORM] = 1.0;
    misc[xb::GM_TAU] = -1.0;
    misc[xb::GM_RAW] = 1.0;
    XB_CUDA(cudaMemcpyAsync(st.misc, misc, sizeof misc, cudaMemcpyHostToDevice, s));
    const int sg = std::max(1, (int)std::min<int64_t>((n + 255) / 256, xb::num_sms() * 8LL));
    if (v0) XB_CUDA(cudaMemcpyAsync(V, v0, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else k_start_vector<<<sg, 256, 0, s>>>(n, V);
    XB_TRY(xb::vnrm2(p, n, V, st.y, s));
    k_scale_inv<<<sg, 256, 0, s>>>(n, V, st.y);
    XB_LAUNCHED("k_scale_inv");

    std::vector<double> T((size_t)(M + 1) * (M + 1), 0.0), H((size_t)(M + 1) * M), a, Q, AQ, S;
    std::vector<double> hres(2 * (size_t)nev);
    std::vector<xb::cplx> TS, Z, w, y;
    std::vector<int> ord;
    std::vector<signed char> kind;
    int k = 0, steps = 0, restarts = 0, status = XB_ENOCONV, K = 0, passes = 1;
    double beta = 0.0, samp[5], tol_in = tol, true_max = -1.0;
    // the wanted Ritz vectors of the current cycle (coefficients in dS) into
    // (xr, xi) with column stride lx
    auto ritz_vectors = [&](double *xr, double *xi, int64_t lx) -> int {
        XB_CUDA(cudaMemcpyAsync(dS, S.data(), S.size() * sizeof(double), cudaMemcpyHostToDevice,
                                s));
        if (xr) XB_TRY(rotate(n, m, nev, V, ld, dS, xr, lx, s));
        if (xi) XB_TRY(rotate(n, m, nev, V, ld, dS + (size_t)m * nev, xi, lx, s));
        return XB_OK;
    };
    for (;;) {
        for (int j = k; j < m; j++) {
            double *vj = V + (size_t)j * ld, *wv = V + (size_t)(j + 1) * ld;
            XB_TRY(xb::spmv_launch(p, variant, block, ipt, 1.0, vj, 0.0, wv, s));
            XB_TRY(xb::gm_ortho_step<double>(p, st, n, V, ld, wv, j, ortho, s));
            k_scale_inv<<<sg, 256, 0, s>>>(n, wv, st.H + (size_t)j * (M + 1) + j + 1);
            steps++;
        }
        XB_CUDA(cudaMemcpyAsync(H.data(), st.H, H.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                s));
        XB_CUDA(cudaStreamSynchronize(s));
        for (int j = k; j < m; j++)
            for (int i = 0; i <= j + 1; i++)
                T[(size_t)i * (M + 1) + j] = H[(size_t)j * (M + 1) + i];
        beta = T[(size_t)m * (M + 1) + m - 1];
        bool broke = false;
        for (int j = k; j < m; j++)
            if (!(T[(size_t)(j + 1) * (M + 1) + j] > 0.0)) broke = true;
        if (broke) {
            status = XB_EBREAKDOWN;
            xb::set_error(XB_EBREAKDOWN, "arnoldi: invariant subspace before %d steps", m);
            break;
        }
        a.assign((size_t)m * m, 0.0);
        for (int i = 0; i < m; i++)
            for (int j = 0; j < m; j++) a[(size_t)i * m + j] = T[(size_t)i * (M + 1) + j];
        XB_TRY(xb::schur(m, a.data(), TS, Z));
        xb::eig_order(m, TS, which, ord, kind, w);
        // kept Ritz values: k = nev + (m - nev)/2, moved by one so that no
        // conjugate pair is split
        int kk = xb::keep_count(kind, nev + (m - nev) / 2, m);
        xb::schur_reorder(m, TS, Z, ord, kk);
        bool conv = true;
        S.assign((size_t)2 * m * nev, 0.0);
        for (int i = 0; i < nev; i++) {
            xb::schur_eigvec(m, TS, Z, i, kind[i] == 0, y);
            evals_re[i] = w[i].real();
            evals_im[i] = w[i].imag();
            resid[i] = std::fabs(beta) * std::abs(y[m - 1]);
            if (!(resid[i] <= tol_in * std::abs(w[i]))) conv = false;
            for (int r = 0; r < m; r++) {
                S[(size_t)i * m + r] = y[r].real();
                S[(size_t)(nev + i) * m + r] = y[r].imag();
            }
        }
        if (conv && check) {
            // true residuals r = A x - theta x of the claimed pairs (Sec. 3.3.2),
            // one Ritz vector at a time (three vectors of workspace)
            XB_CUDA(cudaMemcpyAsync(dS, S.data(), S.size() * sizeof(double),
                                    cudaMemcpyHostToDevice, s));
            for (int i = 0; i < nev; i++) {
                const double *xr = XR, *xi = XI;
                XB_TRY(rotate(n, m, 1, V, ld, dS + (size_t)i * m, XR, ld, s));
                XB_TRY(rotate(n, m, 1, V, ld, dS + (size_t)(nev + i) * m, XI, ld, s));
                const double tr = w[i].real(), ti = w[i].imag();
                XB_TRY(xb::spmv_launch(p, variant, block, ipt, 1.0, xr, 0.0, TMP, s));
                XB_TRY(xb::vaxpy(n, -tr, xr, TMP, s));
                XB_TRY(xb::vaxpy(n, ti, xi, TMP, s));
                XB_TRY(xb::vnrm2(p, n, TMP, dres + 2 * i, s));
                XB_TRY(xb::spmv_launch(p, variant, block, ipt, 1.0, xi, 0.0, TMP, s));
                XB_TRY(xb::vaxpy(n, -tr, xi, TMP, s));
                XB_TRY(xb::vaxpy(n, -ti, xr, TMP, s));
                XB_TRY(xb::vnrm2(p, n, TMP, dres + 2 * i + 1, s));
            }
            XB_CUDA(cudaMemcpyAsync(hres.data(), dres, hres.size() * sizeof(double),
                                    cudaMemcpyDeviceToHost, s));
            XB_CUDA(cudaStreamSynchronize(s));
            true_max = 0.0;
            for (int i = 0; i < nev; i++)
                true_max = std::max(true_max,
                                    std::hypot(hres[2 * i], hres[2 * i + 1]) / std::abs(w[i]));
            if (true_max <= tol) {
                status = XB_OK;
            } else if (!outer) {
                status = XB_EFAULT;
                xb::set_error(XB_EFAULT, "fault convergence: Ritz residual estimates met tol, "
                              "true relative residual %.3e", true_max);
            } else {  // narrow the threshold, switch to DGKS, iterate on
                tol_in *= tol / true_max;
                ortho = xb::ortho_choice(XB_ORTHO_AUTO, tol, true);
                passes++;
                conv = false;
            }
            if (conv) {
                if (evecs_re || evecs_im) XB_TRY(ritz_vectors(evecs_re, evecs_im, n));
                break;
            }
        } else if (conv) {
            status = XB_OK;
            if (evecs_re || evecs_im) XB_TRY(ritz_vectors(evecs_re, evecs_im, n));
            break;
        }
        if (restarts >= maxrestart) {
            status = XB_ENOCONV;
            if (evecs_re || evecs_im) XB_TRY(ritz_vectors(evecs_re, evecs_im, n));
            break;
        }
        // restart rule (Eq. 1), as for Lanczos
        int m_next = m;
        if (m_max > m || K > 0) {
            double worst = 0.0;
            for (int i = 0; i < nev; i++) worst = std::max(worst, resid[i] / std::abs(w[i]));
            samp[K++] = worst;
            if (K == 5) {
                if (xb_dafrt(5, samp, theta)) m_next = std::min(m + 5, m_max);
                K = 0;
            }
        }
        const int got = xb::real_basis(m, Z, kk, Q);
        if (got < nev) {
            status = XB_EBREAKDOWN;
            xb::set_error(XB_EBREAKDOWN, "arnoldi: kept Schur vectors lost rank (%d < %d)", got,
                          nev);
            break;
        }
        kk = got;
        // T_k = Q^T H Q and the coupling row h_{m,m-1} e_m^T Q
        AQ.assign((size_t)m * kk, 0.0);
        for (int c = 0; c < kk; c++)
            for (int r = 0; r < m; r++) {
                double acc = 0.0;
                for (int l = 0; l < m; l++) acc += a[(size_t)r * m + l] * Q[(size_t)c * m + l];
                AQ[(size_t)c * m + r] = acc;
            }
        std::fill(T.begin(), T.end(), 0.0);
        for (int i = 0; i < kk; i++)
            for (int c = 0; c < kk; c++) {
                double acc = 0.0;
                for (int r = 0; r < m; r++) acc += Q[(size_t)i * m + r] * AQ[(size_t)c * m + r];
                T[(size_t)i * (M + 1) + c] = acc;
            }
        for (int c = 0; c < kk; c++) T[(size_t)kk * (M + 1) + c] = beta * Q[(size_t)c * m + m - 1];
        XB_CUDA(cudaMemcpyAsync(dS, Q.data(), (size_t)m * kk * sizeof(double),
                                cudaMemcpyHostToDevice, s));
        XB_TRY(rotate(n, m, kk, V, ld, dS, Y, ld, s));
        XB_CUDA(cudaMemcpyAsync(V, Y, (size_t)kk * ld * sizeof(double), cudaMemcpyDeviceToDevice,
                                s));
        XB_CUDA(cudaMemcpyAsync(V + (size_t)kk * ld, V + (size_t)m * ld, ld * sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
        k = kk;
        m = m_next;
        restarts++;
    }
    if (counts) {
        counts[0] = steps;
        counts[1] = restarts;
        counts[2] = m;
        counts[3] = ortho;
        counts[4] = passes;
    }
    if (stats) {
        stats[0] = (double)need + xb::spmv_meta_bytes(p, variant, block, ipt);
        stats[1] = true_max;
    }
    XB_CUDA(cudaStreamSynchronize(s));
    return status;
}

}  // extern "C"
