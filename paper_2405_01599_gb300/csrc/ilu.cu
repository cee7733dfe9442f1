// ILU(0) preconditioner (the preconditioner of the paper's solver runs,
// Sec. 4.3): incomplete LU factorization in the sparsity pattern of A
// (general CRS), applied as z = U^{-1} L^{-1} r.
//
// Setup: the host derives, from the pattern alone, the dependency level of
// every row for the forward substitution (level(i) = 1 + max level(k) over the
// stored k < i in row i) and for the backward one (over the stored j > i); rows
// are grouped by level.  The numeric factorization then runs level by level on
// the device, one warp per row: for each stored (i, k), k < i, in ascending k,
// l_ik = a_ik / u_kk, and every stored (i, j), j > k, subtracts l_ik u_kj when
// (k, j) is stored (binary search in row k, which an earlier level finished).
// Each substitution is one launch per level; inside a level every row is
// independent: a thread per row, with rows longer than 32 stored entries in
// the triangle taken by the whole warp (lanes stride over the row, shuffle
// reduction), and rows longer than kLongRow by a whole CTA, so a power-law row
// does not serialise one thread or one warp.  The launch sequence of both
// substitutions is captured once into a CUDA graph on fixed operand buffers
// (a 3D stencil has 3N - 2 levels per triangle, so per-launch overhead would
// otherwise dominate).
#include "common.cuh"

#include <algorithm>
#include <cstdlib>
#include <cmath>

namespace {

constexpr int kLongRow = 512;  // triangle entries above which a row gets a CTA
constexpr int kEllMax = 8;     // triangle entries up to which a row is stored as ELL

__device__ __forceinline__ int find_in_row(const int *__restrict__ ci, int lo, int hi, int j) {
    // search [lo, hi) of a sorted column list for j
    hi -= 1;
    while (lo <= hi) {
        const int mid = lo + ((hi - lo) >> 1);
        const int c = __ldg(ci + mid);
        if (c == j) return mid;
        if (c < j) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// Factor the rows listed in rows[0..cnt) (one dependency level), warp per row.
__global__ void k_ilu_factor(int cnt, const int *__restrict__ rows, const int *__restrict__ rp,
                             const int *__restrict__ ci, const int *__restrict__ dpos,
                             double *__restrict__ lu, int *__restrict__ flag) {
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= cnt) return;  // warp-uniform
    const int i = rows[w];
    const int a = rp[i], e = rp[i + 1], d = dpos[i];
    for (int p = a; p < d; p++) {
        const int k = __ldg(ci + p);
        const int dk = dpos[k];
        const double piv = lu[dk];
        if (piv == 0.0) {
            if (lane == 0) atomicExch(flag, 1);
            return;
        }
        const double lik = lu[p] / piv;
        __syncwarp();
        if (lane == 0) lu[p] = lik;
        const int ke = rp[k + 1];
        for (int q = p + 1 + lane; q < e; q += 32) {
            const int pos = find_in_row(ci, dk + 1, ke, __ldg(ci + q));
            if (pos >= 0) lu[q] = fma(-lik, lu[pos], lu[q]);
        }
        __syncwarp();  // row i's entries settled before the next l_ik is formed
    }
    if (lane == 0 && lu[d] == 0.0) atomicExch(flag, 1);
}

// One level of a substitution.  FWD: z_i = r_i - sum_{k<i} l_ik z_k over the
// stored strictly lower entries.  Backward: z_i = (z_i - sum_{j>i} u_ij z_j) / u_ii.
template <bool FWD>
__global__ void __launch_bounds__(256) k_ilu_level(int cnt, const int *__restrict__ rows,
                                                   const int *__restrict__ rp,
                                                   const int *__restrict__ ci,
                                                   const int *__restrict__ dpos,
                                                   const double *__restrict__ lu,
                                                   const double *__restrict__ r,
                                                   double *__restrict__ z) {
    const int lane = threadIdx.x & 31;
    const int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31;  // warp's first slot
    if (base >= cnt) return;  // warp-uniform
    const int slot = base + lane;
    int i = -1, ka = 0, kb = 0;
    if (slot < cnt) {
        i = rows[slot];
        const int d = dpos[i];
        ka = FWD ? rp[i] : d + 1;
        kb = FWD ? d : rp[i + 1];
    }
    const bool lng = kb - ka > 32;
    double s = 0.0;
    if (!lng)
        for (int k = ka; k < kb; k++) s = fma(__ldg(lu + k), z[__ldg(ci + k)], s);
    unsigned todo = __ballot_sync(0xffffffffu, lng);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int la = __shfl_sync(0xffffffffu, ka, src);
        const int lb = __shfl_sync(0xffffffffu, kb, src);
        double t = 0.0;
        for (int k = la + lane; k < lb; k += 32) t = fma(__ldg(lu + k), z[__ldg(ci + k)], t);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == src) s = t;
    }
    if (i >= 0) {
        if (FWD) z[i] = r[i] - s;
        else z[i] = (z[i] - s) / lu[dpos[i]];
    }
}

// One level's long rows, a CTA per row (block reduction in a fixed order).
template <bool FWD>
__global__ void __launch_bounds__(256) k_ilu_level_long(const int *__restrict__ rows,
                                                        const int *__restrict__ rp,
                                                        const int *__restrict__ ci,
                                                        const int *__restrict__ dpos,
                                                        const double *__restrict__ lu,
                                                        const double *__restrict__ r,
                                                        double *__restrict__ z) {
    __shared__ double sh[8];
    const int i = rows[blockIdx.x];
    const int d = dpos[i];
    const int ka = FWD ? rp[i] : d + 1, kb = FWD ? d : rp[i + 1];
    double t = 0.0;
    for (int k = ka + threadIdx.x; k < kb; k += blockDim.x)
        t = fma(__ldg(lu + k), z[__ldg(ci + k)], t);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[w];
        if (FWD) z[i] = r[i] - s;
        else z[i] = (z[i] - s) / lu[d];
    }
}

// One level's short rows in ELL form, a thread per row: the row index, its
// entries and (backward) its pivot are independent loads, then the gathers.
template <bool FWD>
__global__ void __launch_bounds__(256) k_ilu_ell(int cnt, int width, const int *__restrict__ rows,
                                                 const int *__restrict__ ecol,
                                                 const double *__restrict__ eval,
                                                 const double *__restrict__ diag,
                                                 const double *__restrict__ r,
                                                 double *__restrict__ z) {
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= cnt) return;
    const int i = __ldg(rows + slot);
    double s = 0.0;
    for (int t = 0; t < width; t++) {
        const long long e = (long long)t * cnt + slot;
        s = fma(__ldg(eval + e), z[__ldg(ecol + e)], s);
    }
    if (FWD) z[i] = r[i] - s;
    else z[i] = (z[i] - s) / __ldg(diag + slot);
}

// ELL values from the factors (padding entries stay 0), and the pivots in
// backward level order.
__global__ void k_ell_fill(long long cnt, const int *__restrict__ src,
                           const double *__restrict__ lu, double *__restrict__ val) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e < cnt) val[e] = src[e] >= 0 ? lu[src[e]] : 0.0;
}
__global__ void k_diag_fill(int n, const int *__restrict__ rows, const int *__restrict__ dpos,
                            const double *__restrict__ lu, double *__restrict__ diag) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) diag[s] = lu[dpos[rows[s]]];
}

// ---- persistent substitution ---------------------------------------------------
// Both substitutions in one cooperative launch (every CTA resident, one per
// SM): each level is processed by the whole grid, then a grid barrier.  The
// barrier is a counter and a generation word in global memory; a CTA that
// waits longer than `polls` polls (kernel argument; default kBarSpins) sets
// the error flag and leaves, so every wait is bounded, and every CTA then
// leaves at its next barrier too.  Values of z written by other CTAs are read
// at L2.
constexpr unsigned kBarSpins = 1u << 20;  // polls of ~0.5 us: a wait gives up after ~0.5 s

struct TriDev {
    int nlev;
    const int *meta;        // per level: off, n0, n1, w (4 ints)
    const long long *eoff;  // per level: ELL base offset
    const int *rows, *ecol;
    const double *eval, *diag;
};

__device__ __forceinline__ bool grid_bar(unsigned *bar, int *err, unsigned polls) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
            ok = 1;
        } else {
            unsigned it = 0;
            while (*gen == g && ++it < polls) {
            }
            ok = (*gen != g);
            if (!ok) atomicExch(err, 1);
        }
        __threadfence();
    }
    __syncthreads();
    return ok;
}

template <bool FWD>
__device__ void persist_level(const TriDev &t, int l, const int *__restrict__ rp,
                              const int *__restrict__ ci, const int *__restrict__ dpos,
                              const double *__restrict__ lu, const double *__restrict__ r,
                              double *z, double *sh) {
    const int off = t.meta[4 * l], c0 = t.meta[4 * l + 1], c1 = t.meta[4 * l + 2];
    const int w = t.meta[4 * l + 3];
    const int c2 = t.meta[4 * (l + 1)] - off - c0 - c1;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    // ELL tier: a thread per row
    const long long eo = t.eoff[l];
    for (int slot = gt; slot < c0; slot += gs) {
        const int i = t.rows[off + slot];
        double s = 0.0;
        for (int q = 0; q < w; q++) {
            const long long e = eo + (long long)q * c0 + slot;
            s = fma(__ldg(t.eval + e), __ldcg(z + __ldg(t.ecol + e)), s);
        }
        if (FWD) z[i] = __ldg(r + i) - s;
        else z[i] = (__ldcg(z + i) - s) / __ldg(t.diag + off + slot);
    }
    // CSR tier: thread per row, warp for rows over 32 entries
    const int lane = threadIdx.x & 31, wi = gt >> 5, nw = gs >> 5;
    for (int base = wi * 32; base < c1; base += nw * 32) {  // warp-uniform
        const int slot = base + lane;
        int i = -1, ka = 0, kb = 0;
        if (slot < c1) {
            i = t.rows[off + c0 + slot];
            const int d = dpos[i];
            ka = FWD ? rp[i] : d + 1;
            kb = FWD ? d : rp[i + 1];
        }
        const bool lng = kb - ka > 32;
        double s = 0.0;
        if (!lng)
            for (int k = ka; k < kb; k++) s = fma(__ldg(lu + k), __ldcg(z + __ldg(ci + k)), s);
        unsigned todo = __ballot_sync(0xffffffffu, lng);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int la = __shfl_sync(0xffffffffu, ka, src);
            const int lb = __shfl_sync(0xffffffffu, kb, src);
            double v = 0.0;
            for (int k = la + lane; k < lb; k += 32)
                v = fma(__ldg(lu + k), __ldcg(z + __ldg(ci + k)), v);
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == src) s = v;
        }
        if (i >= 0) {
            if (FWD) z[i] = __ldg(r + i) - s;
            else z[i] = (__ldcg(z + i) - s) / lu[dpos[i]];
        }
    }
    // long rows: a CTA per row (the loop bound is uniform over the CTA)
    for (int q = blockIdx.x; q < c2; q += gridDim.x) {
        const int i = t.rows[off + c0 + c1 + q];
        const int d = dpos[i];
        const int ka = FWD ? rp[i] : d + 1, kb = FWD ? d : rp[i + 1];
        double v = 0.0;
        for (int k = ka + threadIdx.x; k < kb; k += blockDim.x)
            v = fma(__ldg(lu + k), __ldcg(z + __ldg(ci + k)), v);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); k++) sum += sh[k];
            if (FWD) z[i] = __ldg(r + i) - sum;
            else z[i] = (__ldcg(z + i) - sum) / lu[d];
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(512, 1) k_ilu_persist(TriDev L, TriDev U, const int *rp,
                                                     const int *ci, const int *dpos,
                                                     const double *lu, const double *r,
                                                     double *z, unsigned *bar, int *err,
                                                     unsigned polls) {
    __shared__ double sh[16];
    for (int l = 0; l < L.nlev; l++) {
        persist_level<true>(L, l, rp, ci, dpos, lu, r, z, sh);
        if (!grid_bar(bar, err, polls)) return;
    }
    for (int l = 0; l < U.nlev; l++) {
        persist_level<false>(U, l, rp, ci, dpos, lu, r, z, sh);
        if (l + 1 < U.nlev && !grid_bar(bar, err, polls)) return;
    }
}

// Rows grouped by level (counting sort), ascending row order inside each tier
// of a level: ELL rows (len <= kEllMax), CSR rows (<= kLongRow), CTA rows;
// n0[l], n1[l] = the first two tiers' counts.
int tier_of(int len) { return len <= kEllMax ? 0 : (len <= kLongRow ? 1 : 2); }
void group_levels(const std::vector<int> &lev, const std::vector<int> &len, int nlev,
                  std::vector<int> &rows, std::vector<int> &off, std::vector<int> &n0,
                  std::vector<int> &n1) {
    const int n = (int)lev.size();
    off.assign(nlev + 1, 0);
    for (int i = 0; i < n; i++) off[lev[i] + 1]++;
    for (int l = 0; l < nlev; l++) off[l + 1] += off[l];
    n0.assign(nlev, 0);
    n1.assign(nlev, 0);
    for (int i = 0; i < n; i++) {
        const int t = tier_of(len[i]);
        if (t == 0) n0[lev[i]]++;
        else if (t == 1) n1[lev[i]]++;
    }
    rows.resize(n);
    std::vector<int> p0(nlev), p1(nlev), p2(nlev);
    for (int l = 0; l < nlev; l++) {
        p0[l] = off[l];
        p1[l] = off[l] + n0[l];
        p2[l] = off[l] + n0[l] + n1[l];
    }
    for (int i = 0; i < n; i++) {
        const int t = tier_of(len[i]), l = lev[i];
        rows[t == 0 ? p0[l]++ : (t == 1 ? p1[l]++ : p2[l]++)] = i;
    }
}

// ELL layout of each level's first tier: width, base offsets, columns and the
// factor position of every entry (padding: the row's first entry's column,
// whose value is final before this level, with position -1 = value 0).
// Entries of row i are positions [beg(i), end(i)) of the CRS arrays.
template <typename Beg, typename End>
void build_ell(const std::vector<int> &rows, const std::vector<int> &off,
               const std::vector<int> &n0, const std::vector<int> &ci, Beg beg, End end,
               std::vector<int> &w, std::vector<long long> &eoff, std::vector<int> &ecol,
               std::vector<int> &esrc) {
    const int nl = (int)n0.size();
    w.assign(nl, 0);
    eoff.assign(nl + 1, 0);
    for (int l = 0; l < nl; l++) {
        for (int q = 0; q < n0[l]; q++) {
            const int i = rows[off[l] + q];
            w[l] = std::max(w[l], end(i) - beg(i));
        }
        eoff[l + 1] = eoff[l] + (long long)w[l] * n0[l];
    }
    ecol.assign((size_t)eoff[nl], 0);
    esrc.assign((size_t)eoff[nl], -1);
    for (int l = 0; l < nl; l++)
        for (int q = 0; q < n0[l]; q++) {
            const int i = rows[off[l] + q];
            const int b = beg(i), len = end(i) - b;
            for (int t = 0; t < w[l]; t++) {
                const long long e = eoff[l] + (long long)t * n0[l] + q;
                ecol[e] = t < len ? ci[b + t] : ci[b];
                esrc[e] = t < len ? b + t : -1;
            }
        }
}

// Launch one substitution's levels on stream s (also used inside the capture).
template <bool FWD>
void launch_levels(const xb_plan *p, const int *d_rows, const std::vector<int> &off,
                   const std::vector<int> &n0, const std::vector<int> &n1,
                   const std::vector<int> &w, const std::vector<long long> &eoff,
                   const int *ecol, const double *eval, const double *diag, const double *r,
                   double *z, cudaStream_t s) {
    const xb::IluData &u = p->ilu;
    const int nl = (int)off.size() - 1;
    for (int l = 0; l < nl; l++) {
        const int c0 = n0[l], c1 = n1[l], c2 = off[l + 1] - off[l] - c0 - c1;
        if (c0 > 0)
            k_ilu_ell<FWD><<<(c0 + 255) / 256, 256, 0, s>>>(c0, w[l], d_rows + off[l],
                                                           ecol + eoff[l], eval + eoff[l],
                                                           diag + off[l], r, z);
        if (c1 > 0)
            k_ilu_level<FWD><<<(c1 + 255) / 256, 256, 0, s>>>(c1, d_rows + off[l] + c0, p->rowptr,
                                                             p->col, u.d_dpos, u.d_lu, r, z);
        if (c2 > 0)
            k_ilu_level_long<FWD><<<c2, 256, 0, s>>>(d_rows + off[l] + c0 + c1, p->rowptr, p->col,
                                                     u.d_dpos, u.d_lu, r, z);
    }
}

}  // namespace

namespace xb {

void ilu_free(xb_plan *p) {
    IluData &u = p->ilu;
    cudaFree(u.d_lu);
    cudaFree(u.d_dpos);
    cudaFree(u.d_lrows);
    cudaFree(u.d_urows);
    cudaFree(u.d_flag);
    cudaFree(u.d_in);
    cudaFree(u.d_out);
    cudaFree(u.d_lecol);
    cudaFree(u.d_uecol);
    cudaFree(u.d_leval);
    cudaFree(u.d_ueval);
    cudaFree(u.d_lesrc);
    cudaFree(u.d_uesrc);
    cudaFree(u.d_udiag);
    if (u.exec) cudaGraphExecDestroy(u.exec);
    if (u.graph) cudaGraphDestroy(u.graph);
    cudaFree(u.d_lmeta);
    cudaFree(u.d_umeta);
    cudaFree(u.d_leo);
    cudaFree(u.d_ueo);
    cudaFree(u.d_bar);
    cudaFree(u.d_err);
    u = IluData();
}

int ilu_levels(int n, const int *rp, const int *ci, std::vector<int> &dpos, std::vector<int> &lev,
               std::vector<int> &ulev, int *nl, int *nu) {
    dpos.assign(n, 0);
    lev.assign(n, 0);
    ulev.assign(n, 0);
    *nl = n > 0 ? 1 : 0;
    *nu = n > 0 ? 1 : 0;
    for (int i = 0; i < n; i++) {
        int d = -1, m = -1;
        for (int q = rp[i]; q < rp[i + 1]; q++) {
            const int k = ci[q];
            if (k < i) m = std::max(m, lev[k]);
            else if (k == i) d = q;
        }
        if (d < 0) return set_error(XB_EBREAKDOWN, "ILU(0): row %d has no diagonal entry", i);
        dpos[i] = d;
        lev[i] = m + 1;
        *nl = std::max(*nl, lev[i] + 1);
    }
    for (int i = n - 1; i >= 0; i--) {
        int m = -1;
        for (int q = dpos[i] + 1; q < rp[i + 1]; q++) m = std::max(m, ulev[ci[q]]);
        ulev[i] = m + 1;
        *nu = std::max(*nu, ulev[i] + 1);
    }
    return XB_OK;
}

int ensure_ilu(xb_plan *p, cudaStream_t s) {
    if (!p->subs.empty())
        return set_error(XB_EINVAL, "ILU(0): not available for a plan split into row blocks");
    IluData &u = p->ilu;
    if (u.built) return u.status == XB_OK ? XB_OK : set_error(u.status, "ILU(0): zero pivot");
    if (p->sym) return set_error(XB_EINVAL, "ILU(0) needs full (general) CRS storage");
    ilu_free(p);  // a build that failed half-way left nothing usable
    const int n = p->n, nnz = p->nnz;
    const std::vector<int> &rp = p->h_rowptr;
    std::vector<int> ci(nnz);
    if (nnz > 0) XB_CUDA(cudaMemcpy(ci.data(), p->col, (size_t)nnz * 4, cudaMemcpyDeviceToHost));
    std::vector<int> dpos, lev, ulev;
    int nl = 0, nu = 0;
    XB_TRY(ilu_levels(n, rp.data(), ci.data(), dpos, lev, ulev, &nl, &nu));
    std::vector<int> llen(n), ulen(n);
    for (int i = 0; i < n; i++) {
        llen[i] = dpos[i] - rp[i];
        ulen[i] = rp[i + 1] - dpos[i] - 1;
    }
    std::vector<int> lrows, urows;
    group_levels(lev, llen, nl, lrows, u.loff, u.ln0, u.ln1);
    group_levels(ulev, ulen, nu, urows, u.uoff, u.un0, u.un1);
    std::vector<int> lecol, lesrc, uecol, uesrc;
    build_ell(lrows, u.loff, u.ln0, ci, [&](int i) { return rp[i]; },
              [&](int i) { return dpos[i]; }, u.lw, u.leoff, lecol, lesrc);
    build_ell(urows, u.uoff, u.un0, ci, [&](int i) { return dpos[i] + 1; },
              [&](int i) { return rp[i + 1]; }, u.uw, u.ueoff, uecol, uesrc);
    auto up = [&](int **d, const std::vector<int> &h) -> int {
        XB_CUDA(cudaMalloc(d, std::max<size_t>(1, h.size()) * 4));
        if (!h.empty())
            XB_CUDA(cudaMemcpyAsync(*d, h.data(), h.size() * 4, cudaMemcpyHostToDevice, s));
        return XB_OK;
    };
    XB_TRY(up(&u.d_dpos, dpos));
    XB_TRY(up(&u.d_lrows, lrows));
    XB_TRY(up(&u.d_urows, urows));
    XB_TRY(up(&u.d_lecol, lecol));
    XB_TRY(up(&u.d_lesrc, lesrc));
    XB_TRY(up(&u.d_uecol, uecol));
    XB_TRY(up(&u.d_uesrc, uesrc));
    XB_CUDA(cudaMalloc(&u.d_leval, std::max<size_t>(1, lecol.size()) * sizeof(double)));
    XB_CUDA(cudaMalloc(&u.d_ueval, std::max<size_t>(1, uecol.size()) * sizeof(double)));
    XB_CUDA(cudaMalloc(&u.d_udiag, std::max<size_t>(1, (size_t)n) * sizeof(double)));
    XB_CUDA(cudaMalloc(&u.d_lu, std::max<size_t>(1, (size_t)nnz) * sizeof(double)));
    XB_CUDA(cudaMalloc(&u.d_flag, sizeof(int)));
    XB_CUDA(cudaMalloc(&u.d_in, std::max<size_t>(1, (size_t)n) * sizeof(double)));
    XB_CUDA(cudaMalloc(&u.d_out, std::max<size_t>(1, (size_t)n) * sizeof(double)));
    XB_CUDA(cudaMemsetAsync(u.d_flag, 0, sizeof(int), s));
    if (nnz > 0)
        XB_CUDA(cudaMemcpyAsync(u.d_lu, p->val, (size_t)nnz * sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
    for (int l = 0; l < nl; l++) {
        const int cnt = u.loff[l + 1] - u.loff[l];
        if (cnt == 0) continue;
        const int wpb = 8;  // warps per CTA
        k_ilu_factor<<<(cnt + wpb - 1) / wpb, 32 * wpb, 0, s>>>(
            cnt, u.d_lrows + u.loff[l], p->rowptr, p->col, u.d_dpos, u.d_lu, u.d_flag);
    }
    XB_LAUNCHED("k_ilu_factor");
    if (!lecol.empty())
        k_ell_fill<<<(unsigned)((lecol.size() + 255) / 256), 256, 0, s>>>(
            (long long)lecol.size(), u.d_lesrc, u.d_lu, u.d_leval);
    if (!uecol.empty())
        k_ell_fill<<<(unsigned)((uecol.size() + 255) / 256), 256, 0, s>>>(
            (long long)uecol.size(), u.d_uesrc, u.d_lu, u.d_ueval);
    if (n > 0)
        k_diag_fill<<<(n + 255) / 256, 256, 0, s>>>(n, u.d_urows, u.d_dpos, u.d_lu, u.d_udiag);
    XB_LAUNCHED("k_ell_fill");
    int flag = 0;
    XB_CUDA(cudaMemcpyAsync(&flag, u.d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    XB_CUDA(cudaStreamSynchronize(s));
    u.built = true;
    u.status = flag ? XB_EBREAKDOWN : XB_OK;
    if (flag) return set_error(XB_EBREAKDOWN, "ILU(0): zero pivot");
    // capture both substitutions (d_in -> d_out) on a private stream
    cudaStream_t cs = nullptr;
    XB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        launch_levels<true>(p, u.d_lrows, u.loff, u.ln0, u.ln1, u.lw, u.leoff, u.d_lecol,
                            u.d_leval, u.d_udiag, u.d_in, u.d_out, cs);
        launch_levels<false>(p, u.d_urows, u.uoff, u.un0, u.un1, u.uw, u.ueoff, u.d_uecol,
                             u.d_ueval, u.d_udiag, u.d_out, u.d_out, cs);
        e = cudaStreamEndCapture(cs, &u.graph);
    }
    cudaStreamDestroy(cs);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&u.exec, u.graph, 0);
    if (e != cudaSuccess) {
        u.built = false;
        return cuda_error(e, "ILU(0): capture of the substitutions");
    }
    // level tables for the persistent substitution
    auto meta = [](const std::vector<int> &off, const std::vector<int> &n0,
                   const std::vector<int> &n1, const std::vector<int> &w) {
        const int nl = (int)n0.size();
        std::vector<int> m(4 * (nl + 1), 0);
        for (int l = 0; l < nl; l++) {
            m[4 * l] = off[l];
            m[4 * l + 1] = n0[l];
            m[4 * l + 2] = n1[l];
            m[4 * l + 3] = w[l];
        }
        m[4 * nl] = off[nl];
        return m;
    };
    XB_TRY(up(&u.d_lmeta, meta(u.loff, u.ln0, u.ln1, u.lw)));
    XB_TRY(up(&u.d_umeta, meta(u.uoff, u.un0, u.un1, u.uw)));
    XB_CUDA(cudaMalloc(&u.d_leo, u.leoff.size() * sizeof(long long)));
    XB_CUDA(cudaMalloc(&u.d_ueo, u.ueoff.size() * sizeof(long long)));
    XB_CUDA(cudaMemcpyAsync(u.d_leo, u.leoff.data(), u.leoff.size() * sizeof(long long),
                            cudaMemcpyHostToDevice, s));
    XB_CUDA(cudaMemcpyAsync(u.d_ueo, u.ueoff.data(), u.ueoff.size() * sizeof(long long),
                            cudaMemcpyHostToDevice, s));
    XB_CUDA(cudaMalloc(&u.d_bar, 2 * sizeof(unsigned)));
    XB_CUDA(cudaMalloc(&u.d_err, sizeof(int)));
    XB_CUDA(cudaMemsetAsync(u.d_err, 0, sizeof(int), s));
    int dev = 0, coop = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ilu_persist, 512, 0) ==
                    cudaSuccess &&
        per >= 1)
        u.pgrid = num_sms();
    cudaGetLastError();
    XB_CUDA(cudaStreamSynchronize(s));
    return XB_OK;
}

// Which substitution to run: the persistent launch pays one grid barrier per
// level, the captured graph one kernel per non-empty row tier of a level
// (measured: ~6 us per barrier, ~4 us per graph kernel), so the persistent
// launch wins when levels hold several tiers (power-law rows) and the graph
// when every level is one ELL kernel (stencils).  XB_ILU_MODE=0/1 forces one.
int ilu_mode(const xb_plan *p, const IluData &u) {
    static const int env = [] {
        const char *e = std::getenv("XB_ILU_MODE");
        return e ? std::atoi(e) : -1;
    }();
    if (p->ilu_mode >= 0) return p->ilu_mode;
    if (env >= 0) return env;
    long long levels = (long long)u.ln0.size() + (long long)u.un0.size(), kernels = 0;
    auto tiers = [](const std::vector<int> &off, const std::vector<int> &n0,
                    const std::vector<int> &n1) {
        long long k = 0;
        for (size_t l = 0; l < n0.size(); l++)
            k += (n0[l] > 0) + (n1[l] > 0) + (off[l + 1] - off[l] > n0[l] + n1[l]);
        return k;
    };
    kernels = tiers(u.loff, u.ln0, u.ln1) + tiers(u.uoff, u.un0, u.un1);
    return 4 * kernels > 6 * levels ? 1 : 0;
}

int ilu_check(xb_plan *p) {
    IluData &u = p->ilu;
    if (!u.built || !u.d_err) return XB_OK;
    int err = 0;
    XB_CUDA(cudaMemcpy(&err, u.d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        cudaMemset(u.d_err, 0, sizeof(int));
        return set_error(XB_ETIMEOUT, "ILU(0): a level barrier wait ran out");
    }
    return XB_OK;
}

int ilu_apply(xb_plan *p, const double *r, double *z, cudaStream_t s) {
    IluData &u = p->ilu;
    XB_TRY(ensure_ilu(p, s));
    if (p->n == 0) return XB_OK;
    if (u.pgrid > 0 && ilu_mode(p, u) == 1) {
        TriDev L{(int)u.ln0.size(), u.d_lmeta, u.d_leo, u.d_lrows, u.d_lecol, u.d_leval, u.d_udiag};
        TriDev U{(int)u.un0.size(), u.d_umeta, u.d_ueo, u.d_urows, u.d_uecol, u.d_ueval, u.d_udiag};
        const int *rp = p->rowptr, *ci = p->col, *dp = u.d_dpos;
        const double *lu = u.d_lu;
        unsigned *bar = u.d_bar;
        int *err = u.d_err;
        unsigned polls = p->ilu_polls > 0 ? (unsigned)p->ilu_polls : kBarSpins;
        void *args[] = {&L, &U, (void *)&rp, (void *)&ci, (void *)&dp, (void *)&lu, (void *)&r,
                        (void *)&z, (void *)&bar, (void *)&err, (void *)&polls};
        XB_CUDA(cudaMemsetAsync(u.d_bar, 0, 2 * sizeof(unsigned), s));
        XB_CUDA(cudaLaunchCooperativeKernel((const void *)k_ilu_persist, u.pgrid, 512, args, 0, s));
        return XB_OK;
    }
    const size_t bytes = (size_t)p->n * sizeof(double);
    XB_CUDA(cudaMemcpyAsync(u.d_in, r, bytes, cudaMemcpyDeviceToDevice, s));
    XB_CUDA(cudaGraphLaunch(u.exec, s));
    XB_CUDA(cudaMemcpyAsync(z, u.d_out, bytes, cudaMemcpyDeviceToDevice, s));
    return XB_OK;
}

double ilu_apply_bytes(const xb_plan *p) {
    // both triangles once (value + column), rowptr and diagonal positions
    // twice, r read, z written by the forward pass, read and written by the
    // backward pass, and each row's level slot twice
    const double n = p->n, nnz = p->nnz;
    return 12.0 * nnz + 2.0 * 4.0 * (n + 1) + 2.0 * 4.0 * n + 8.0 * n * 4.0 + 2.0 * 4.0 * n +
           32.0 * n;  // + copies into and out of the captured solve's buffers
}

}  // namespace xb

extern "C" {

int xb_ilu0_setup(xb_plan *p, void *stream) {
    if (!p) return xb::set_error(XB_EINVAL, "ilu0_setup: NULL plan");
    return xb::ensure_ilu(p, (cudaStream_t)stream);
}

int xb_ilu0_apply(xb_plan *p, const double *r, double *z, void *stream) {
    if (!p || (p->n > 0 && (!r || !z)) || r == z)
        return xb::set_error(XB_EINVAL, "ilu0_apply: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    XB_TRY(xb::ilu_apply(p, r, z, s));
    XB_CUDA(cudaStreamSynchronize(s));
    return xb::ilu_check(p);
}

int xb_ilu0_config(xb_plan *p, int32_t mode, int32_t barrier_polls) {
    if (!p || mode < -1 || mode > 1 || barrier_polls < 0)
        return xb::set_error(XB_EINVAL, "ilu0_config: plan %p mode %d polls %d", (void *)p, mode,
                             barrier_polls);
    p->ilu_mode = mode;
    p->ilu_polls = barrier_polls;
    return XB_OK;
}

int xb_ilu0_factors(xb_plan *p, double *lu, void *stream) {
    if (!p || (p->nnz > 0 && !lu)) return xb::set_error(XB_EINVAL, "ilu0_factors: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    XB_TRY(xb::ensure_ilu(p, s));
    if (p->nnz > 0)
        XB_CUDA(cudaMemcpyAsync(lu, p->ilu.d_lu, (size_t)p->nnz * sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
    return XB_OK;
}

}  // extern "C"

extern "C" int xb_ilu_levels(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t *lev,
                             int32_t *ulev, int32_t *nlevels) {
    if (n < 0 || !rowptr || (n > 0 && !col))
        return xb::set_error(XB_EINVAL, "ilu_levels: bad argument");
    std::vector<int> d, l, u;
    int nl = 0, nu = 0;
    XB_TRY(xb::ilu_levels(n, rowptr, col, d, l, u, &nl, &nu));
    if (lev) std::copy(l.begin(), l.end(), lev);
    if (ulev) std::copy(u.begin(), u.end(), ulev);
    if (nlevels) {
        nlevels[0] = nl;
        nlevels[1] = nu;
    }
    return XB_OK;
}
