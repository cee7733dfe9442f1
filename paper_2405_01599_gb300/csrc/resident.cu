// GMRES(m) for a small system held entirely in the shared memory of one
// thread-block cluster: restarted GMRES (Sec. 2.2) with the fused MGS or the
// blocked (length 4) Gram-Schmidt pass, Givens least squares, the
// restart-frequency rule of Eq. (1) / Sec. 4.3 and the fault-convergence
// check of Sec. 3.3.2 -- the same iteration as the multi-launch FP64 solver
// and the batched kernel, with a different data layout and schedule.
//
// Cost model.  On this GPU an FP64 add or FMA issued by a warp occupies its
// SM sub-partition's FP64 pipe for about 80 cycles whatever the number of
// active lanes, so at this size a Krylov step is bound by the count of FP64
// warp instructions on its critical path (and by cluster barriers, about 400
// cycles).  Hence: one warp per sub-partition (4 warps per CTA, R rows per
// thread), the largest cluster that keeps R smallest, reductions shaped to
// use few FP64 instructions, the running Givens rotation of the previous
// entry computed while an exchange is in flight, and the rotated Hessenberg
// entries formed only at the restart, where the triangular solve needs them.
//
// Layout.  CTA r of the cluster owns rows [r rpc, (r+1) rpc); thread t holds
// the local rows t, t + 128, ... (R of them).  The thread's entries of the
// Krylov basis sit in the CTA's shared memory (basis vector i, local row l at
// V[i rpp + l], rpp = 128 R, so a warp's accesses are consecutive), its rows
// of A in an ELL copy there (column k at [k rpp + l]: the value, and the
// owning CTA and local offset of the column), and w, x, b in registers, so an
// Arnoldi step touches no global memory.
//
// Exchange.  The vector an SpMV multiplies (x at a restart, the unnormalised
// w of the previous step otherwise, the 1 / ||w|| scale applied to the
// product) is published in one of two shared buffers; every thread gathers
// the entries of its rows from the owning CTAs with ld.shared::cluster.  The
// buffers alternate, and a buffer is rewritten only after a cluster barrier
// that follows every read of it.
//
// Reductions.  One, or four at once, sums over the cluster: each warp
// reduces its lanes' partials with shuffles (four sums in a transposed tree:
// 6 adds rather than 20), and lanes store the warp's sums into the same slot
// of every CTA's slot array; every warp then sums the P = 4 ncl slots in one
// fixed order, so every thread of the cluster holds the same bits and takes
// the same branches.  The inner products of the Gram-Schmidt passes complete
// through mbarriers: the stores are st.async with complete-tx on the
// receiving CTA's mbarrier, and each CTA waits on its own mbarrier for all P
// contributions -- no fence and no cluster barrier.  Two slot arrays and two
// mbarriers alternate; a CTA can send the sums of reduction k + 2 only after
// receiving every warp's sums of k + 1, which each warp sends only after it
// has read its slots of k, and thread 0 re-arms an mbarrier right after its
// wait, so the expected byte count is set before any contribution to the next
// use can arrive.  Sums that must also publish a vector (the norm of w, the
// residual) use a cluster barrier (release / acquire) over a second pair of
// slot arrays.  Every barrier sits on a path whose conditions are such
// reduced values or step counts, so all threads of the cluster reach the same
// barriers in the same order; a final cluster barrier keeps every CTA's
// shared memory alive until no CTA can write to it.  An mbarrier wait gives
// up after 2 s (XB_ETIMEOUT), which a correct exchange never reaches.

#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

namespace {

constexpr int kMaxRow = 64;  // longest row the ELL copy takes
constexpr int kW = 4;        // warps per CTA: one per SM sub-partition
constexpr int kBT = 32 * kW;
constexpr unsigned kFull = 0xffffffffu;

struct ResArgs {
    int n, rpc, lmax, m, m_max, maxiter, bcgs;
    double tol, theta;
    unsigned long long budget_ns;
    const int *rowptr, *col;
    const double *val, *b;
    double *x;
    xb_batch_info *out;
};

// Byte offsets of the dynamic shared memory regions (doubles first).
struct ResLayout {
    size_t V, W, ev, bs, ms, H, cs, sn, g, y, ea, p2, mb, total;
};

__host__ __device__ inline ResLayout res_layout(int rpp, int lmax, int mmax, int P) {
    ResLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 15) / 16 * 16;
        return at;
    };
    L.V = take((size_t)(mmax + 1) * rpp * 8);
    L.W = take((size_t)2 * rpp * 8);
    L.ev = take((size_t)lmax * rpp * 8);
    L.bs = take((size_t)2 * 4 * P * 8);  // barrier-completed slots
    L.ms = take((size_t)2 * 4 * P * 8);  // mbarrier-completed slots
    L.H = take((size_t)(mmax + 1) * mmax * 8);
    L.cs = take((size_t)mmax * 8);
    L.sn = take((size_t)mmax * 8);
    L.g = take((size_t)(mmax + 1) * 8);
    L.y = take((size_t)mmax * 8);
    L.ea = take((size_t)lmax * rpp * 4);
    // R <= 4: each thread's part of (v_{i-1}, v_i), formed once per basis vector
    L.p2 = take(rpp <= 4 * 128 ? (size_t)(mmax + 1) * 128 * 8 : 0);
    L.mb = take(2 * 8 + 4);  // two mbarriers, the abort flag
    L.total = o;
    return L;
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// The shared::cluster address of local shared address a in CTA `rank`.
__device__ __forceinline__ unsigned map_rank(unsigned a, unsigned rank) {
    unsigned d;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(rank));
    return d;
}

__device__ __forceinline__ double ld_cluster(unsigned a) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}

__device__ __forceinline__ void st_cluster(unsigned a, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}

// Store v at shared::cluster address a and complete 8 bytes of the
// transaction count of the mbarrier at shared::cluster address mb (same CTA).
__device__ __forceinline__ void st_async(unsigned a, double v, unsigned mb) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(a),
                 "l"(__double_as_longlong(v)), "r"(mb)
                 : "memory");
}

__device__ __forceinline__ void mb_init(unsigned a) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
}

// The one arrival of a phase, expecting `bytes` of transactions.
__device__ __forceinline__ void mb_arm(unsigned a, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mb_test(unsigned a, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}

// Cluster barrier in two halves: stores before the arrive are visible to
// loads after the wait in every CTA; work between them overlaps the barrier.
__device__ __forceinline__ void cl_arrive() {
    asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
__device__ __forceinline__ void cl_wait() {
    asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ double warp_sum1(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Sum of four values over the warp, transposed: every lane returns the sum
// of value (lane >> 3) (6 adds in all).
__device__ __forceinline__ double warp_sum4(const double (&v)[4]) {
    const int lane = threadIdx.x & 31;
    const bool h16 = lane & 16, h8 = lane & 8;
    double k0 = h16 ? v[2] : v[0], k1 = h16 ? v[3] : v[1];
    const double s0 = h16 ? v[0] : v[2], s1 = h16 ? v[1] : v[3];
    k0 += __shfl_xor_sync(kFull, s0, 16);
    k1 += __shfl_xor_sync(kFull, s1, 16);
    double k = h8 ? k1 : k0;
    k += __shfl_xor_sync(kFull, h8 ? k0 : k1, 8);
    k += __shfl_xor_sync(kFull, k, 4);
    k += __shfl_xor_sync(kFull, k, 2);
    k += __shfl_xor_sync(kFull, k, 1);
    return k;
}

// Sum over the P = 4 NCL slots at `base` (one value), in a fixed order:
// lane l holds slots l (and l + 32), then log2 P levels of the tree.
template <int NCL>
__device__ __forceinline__ double slots_sum1(const double *base) {
    constexpr int P = 4 * NCL;
    const int lane = threadIdx.x & 31;
    double s = lane < P ? base[lane] : 0.0;
    if (P > 32) s += base[32 + lane];
#pragma unroll
    for (int o = (P < 32 ? P : 32) >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    // P >= 32: every lane took part, the butterfly left the total everywhere
    return P >= 32 ? s : __shfl_sync(kFull, s, 0);
}

// Four sums over the P slots of each of base[q P ...].
template <int NCL>
__device__ __forceinline__ void slots_sum4(const double *base, double (&v)[4]) {
    constexpr int P = 4 * NCL;
    const int lane = threadIdx.x & 31;
    double a[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        a[q] = lane < P ? base[q * P + lane] : 0.0;
        if (P > 32) a[q] += base[q * P + 32 + lane];
    }
    const double k = warp_sum4(a);
#pragma unroll
    for (int q = 0; q < 4; q++) v[q] = __shfl_sync(kFull, k, 8 * q);
}

template <int NCL>
struct Red {
    static constexpr int P = 4 * NCL;
    double *bs, *ms;       // barrier / mbarrier slots: 2 phases x 4 sums x P
    unsigned mb;           // shared address of the two mbarriers
    volatile int *abort;   // set when an mbarrier wait gave up
    int slot, bph, mk, K;  // this warp's slot, phases, sums per mbarrier exchange
};

// Barrier-completed sum of one value (also publishes the caller's earlier
// shared stores to the cluster): put, then the work between, then get.
template <int NCL>
__device__ __forceinline__ void bput1(double v, const Red<NCL> &R) {
    v = warp_sum1(v);
    const int lane = threadIdx.x & 31;
    if (lane < NCL)
        st_cluster(map_rank(smem_addr(R.bs + R.bph * 4 * R.P + R.slot), (unsigned)lane), v);
    cl_arrive();
}
template <int NCL>
__device__ __forceinline__ double bget1(Red<NCL> &R) {
    cl_wait();
    const double s = slots_sum1<NCL>(R.bs + R.bph * 4 * R.P);
    R.bph ^= 1;
    return s;
}
template <int NCL>
__device__ __forceinline__ void bput4(const double (&v)[4], const Red<NCL> &R) {
    const double k = warp_sum4(v);  // sum of value lane >> 3
    const int lane = threadIdx.x & 31, q = lane >> 3, r = lane & 7;
    const unsigned dst = smem_addr(R.bs + R.bph * 4 * R.P + q * R.P + R.slot);
    if (r < NCL) st_cluster(map_rank(dst, (unsigned)r), k);
    if (r + 8 < NCL) st_cluster(map_rank(dst, (unsigned)(r + 8)), k);
    cl_arrive();
}
template <int NCL>
__device__ __forceinline__ void bget4(double (&v)[4], Red<NCL> &R) {
    cl_wait();
    slots_sum4<NCL>(R.bs + R.bph * 4 * R.P, v);
    R.bph ^= 1;
}

// mbarrier-completed sums (R.K values: 1 for MGS, 4 for BCGS).
template <int NCL>
__device__ __forceinline__ void mput1(double v, const Red<NCL> &R) {
    v = warp_sum1(v);
    const int lane = threadIdx.x & 31, p = R.mk & 1;
    if (lane < NCL)
        st_async(map_rank(smem_addr(R.ms + p * 4 * R.P + R.slot), (unsigned)lane), v,
                 map_rank(R.mb + 8 * p, (unsigned)lane));
}
template <int NCL>
__device__ __forceinline__ void mput4(const double (&v)[4], const Red<NCL> &R) {
    const double k = warp_sum4(v);
    const int lane = threadIdx.x & 31, q = lane >> 3, r = lane & 7, p = R.mk & 1;
    const unsigned dst = smem_addr(R.ms + p * 4 * R.P + q * R.P + R.slot), mb = R.mb + 8 * p;
    if (r < NCL) st_async(map_rank(dst, (unsigned)r), k, map_rank(mb, (unsigned)r));
    if (r + 8 < NCL) st_async(map_rank(dst, (unsigned)(r + 8)), k, map_rank(mb, (unsigned)(r + 8)));
}
// Wait for this CTA's mbarrier of the current exchange (2 s limit), re-arm it
// for the exchange after next, return the slots.
template <int NCL>
__device__ __forceinline__ const double *mwait(Red<NCL> &R) {
    const int p = R.mk & 1;
    const unsigned a = R.mb + 8 * p, par = (unsigned)(R.mk >> 1) & 1u;
    bool done = mb_test(a, par);
    if (!done) {
        const unsigned long long t0 = gtimer();
        while (!(done = mb_test(a, par))) {
            if (*R.abort) break;
            if (gtimer() - t0 > 2000000000ull) {
                *R.abort = 1;
                break;
            }
        }
    }
    // re-arm only a completed phase (after a timeout the exchange is lost and
    // every later wait returns at once)
    if (threadIdx.x == 0 && done) mb_arm(a, (unsigned)(R.K * R.P * 8));
    R.mk++;
    return R.ms + p * 4 * R.P;
}

// The thread's R rows at once, entry k of every row in one round, so their
// gathers overlap; each row's sum keeps its storage order.
template <int R>
__device__ __forceinline__ void rows_spmv(const double *__restrict__ ev, const int *__restrict__ ea,
                                          const int (&len)[R], int rpp, unsigned buf,
                                          double (&s)[R]) {
    int lmx = 0;
#pragma unroll
    for (int r = 0; r < R; r++) {
        s[r] = 0.0;
        lmx = max(lmx, len[r]);
    }
#pragma unroll 2
    for (int k = 0; k < lmx; k++) {
#pragma unroll
        for (int r = 0; r < R; r++) {
            if (k < len[r]) {
                const int l = r * kBT + threadIdx.x;
                const int e = ea[k * rpp + l];
                const double u =
                    ld_cluster(map_rank(buf + (unsigned)(e & 0xffff) * 8u, (unsigned)e >> 16));
                s[r] = fma(ev[k * rpp + l], u, s[r]);
            }
        }
    }
}

template <int R, int NCL>
__global__ void __launch_bounds__(kBT, 1) k_gmres_resident(const ResArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int rpp = kBT * R;
    const int mmax = A.m_max, ldh = mmax + 1;
    const ResLayout L = res_layout(rpp, A.lmax, mmax, 4 * NCL);
    double *V = reinterpret_cast<double *>(smem + L.V);
    double *W = reinterpret_cast<double *>(smem + L.W);
    double *ev = reinterpret_cast<double *>(smem + L.ev);
    double *H = reinterpret_cast<double *>(smem + L.H);
    double *cs = reinterpret_cast<double *>(smem + L.cs);
    double *sn = reinterpret_cast<double *>(smem + L.sn);
    double *g = reinterpret_cast<double *>(smem + L.g);
    double *yv = reinterpret_cast<double *>(smem + L.y);
    int *ea = reinterpret_cast<int *>(smem + L.ea);
    double *P2 = reinterpret_cast<double *>(smem + L.p2);  // R <= 4 only
    const unsigned rank = cluster_rank();
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    Red<NCL> Rd;
    Rd.bs = reinterpret_cast<double *>(smem + L.bs);
    Rd.ms = reinterpret_cast<double *>(smem + L.ms);
    Rd.mb = smem_addr(smem + L.mb);
    Rd.abort = reinterpret_cast<volatile int *>(smem + L.mb + 16);
    Rd.slot = (int)rank * kW + warp;
    Rd.bph = 0;
    Rd.mk = 0;
    Rd.K = A.bcgs ? 4 : 1;
    if (t == 0) {
        *Rd.abort = 0;
        mb_init(Rd.mb);
        mb_init(Rd.mb + 8);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mb_arm(Rd.mb, (unsigned)(Rd.K * Rd.P * 8));
        mb_arm(Rd.mb + 8, (unsigned)(Rd.K * Rd.P * 8));
    }
    const bool lead = rank == 0 && t == 0;
    const unsigned long long ts = gtimer(), deadline = ts + A.budget_ns;

    // this thread's rows into the ELL copy; a column outside [0, n) is
    // counted and fails the solve (nothing is read through it)
    int len[R];
    double bi[R], x[R], w[R];
    double bad = 0.0;
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int l = r * kBT + t, row = (int)rank * A.rpc + l;
        len[r] = 0;
        bi[r] = 0.0;
        x[r] = 0.0;
        if (l < A.rpc && row < A.n) {
            const int ka = A.rowptr[row];
            len[r] = A.rowptr[row + 1] - ka;
            for (int k = 0; k < len[r]; k++) {
                int c = A.col[ka + k];
                if (c < 0 || c >= A.n) {
                    bad = 1.0;
                    c = row;
                }
                const int o = c / A.rpc;
                ea[k * rpp + l] = (o << 16) | (c - o * A.rpc);
                ev[k * rpp + l] = A.val[ka + k];
            }
            bi[r] = A.b[row];
            x[r] = A.x[row];
        }
    }
    const unsigned wbuf[2] = {smem_addr(W), smem_addr(W + rpp)};

    int iters = 0, restarts = 0, status = XB_OK, claimed = 0, m = A.m, K = 0;
    double tau = A.tol, res_true = 0.0, samp[5];
    double q4[4] = {0.0, bad, 0.0, 0.0};
#pragma unroll
    for (int r = 0; r < R; r++) q4[0] = fma(bi[r], bi[r], q4[0]);
    // the first barrier also orders the mbarrier set-up and the ELL copy
    // before any exchange or gather
    bput4(q4, Rd);
    bget4(q4, Rd);
    const double bnorm = sqrt(q4[0]);
    int wb = 0;  // buffer the next publication goes to
    if (q4[1] > 0.0) {
        status = XB_EINVAL;
    } else if (bnorm == 0.0) {
#pragma unroll
        for (int r = 0; r < R; r++) x[r] = 0.0;
    } else {
        for (;;) {
            // r = b - A x
#pragma unroll
            for (int r = 0; r < R; r++) W[wb * rpp + r * kBT + t] = x[r];
            cl_arrive();
            cl_wait();
            double rs[R];
            rows_spmv<R>(ev, ea, len, rpp, wbuf[wb], rs);
#pragma unroll
            for (int r = 0; r < R; r++) rs[r] = fma(-1.0, rs[r], bi[r]);
            wb ^= 1;
            q4[0] = 0.0;
#pragma unroll
            for (int r = 0; r < R; r++) {
                W[wb * rpp + r * kBT + t] = rs[r];  // v_0 unnormalised, for the first SpMV
                q4[0] = fma(rs[r], rs[r], q4[0]);
            }
            q4[1] = (lead && gtimer() > deadline) ? 1.0 : 0.0;
            q4[2] = *Rd.abort ? 1.0 : 0.0;
            q4[3] = 0.0;
            bput4(q4, Rd);
            bget4(q4, Rd);
            const double beta = sqrt(q4[0]);
            res_true = beta / bnorm;
            if (q4[2] > 0.0) {
                status = XB_ETIMEOUT;
                break;
            }
            if (res_true <= A.tol) {
                status = XB_OK;
                break;
            }
            if (iters >= A.maxiter || q4[1] > 0.0) {
                status = XB_ENOCONV;
                break;
            }
            if (claimed) tau *= A.tol / res_true;  // fault convergence: narrow the threshold
            claimed = 0;
            if (restarts > 0) {  // restart-frequency rule (Eq. 1): judge every 5 samples
                samp[K++] = res_true;
                if (K == 5) {
                    double mx = samp[0], mn = samp[0];
                    for (int z = 1; z < 5; z++) {
                        mx = fmax(mx, samp[z]);
                        mn = fmin(mn, samp[z]);
                    }
                    if (mn > 0.0 && mx / mn < A.theta) m = min(m + 5, mmax);
                    K = 0;
                }
            }
            double sc = 1.0 / beta;  // scale of the published vector
#pragma unroll
            for (int r = 0; r < R; r++) V[r * kBT + t] = rs[r] * sc;
            const double tol_g = tau * bnorm;  // |g_{j+1}| <= tau ||b||
            double gj = beta;                  // g_j of the least-squares right-hand side
            int k = 0;
            for (int j = 0; j < m; j++) {
                iters++;
                rows_spmv<R>(ev, ea, len, rpp, wbuf[wb], w);
#pragma unroll
                for (int r = 0; r < R; r++) w[r] *= sc;
                double len2 = 0.0, tt = 0.0;
                // Givens rotations of the previous columns, applied as the
                // column's entries arrive (while the next exchange is in
                // flight): tt is entry i rotated by G_0..G_{i-1}.  The column
                // keeps the raw entries; the rotated ones are formed again at
                // the restart, where the triangular solve needs them, so no
                // warp carries that work on the path of every exchange
                auto take = [&](int i, double h) {
                    len2 = fma(h, h, len2);
                    if (t == 0) H[j * ldh + i] = h;
                    if (i == 0) {
                        tt = h;
                    } else {
                        const double c = cs[i - 1], s = sn[i - 1];
                        tt = fma(-s, tt, c * h);
                    }
                };
                double *wn = W + (wb ^ 1) * rpp;
                double last[4];
                int nlast, i_last;
                if (A.bcgs) {
                    // blocks of 4: one exchange per block takes the block's
                    // dots after the previous block's projection
                    double c4[4] = {0.0, 0.0, 0.0, 0.0};
                    int u0 = 0, nu = 0;
                    for (int d0 = 0; d0 <= j; d0 += 4) {
                        const int nd = min(4, j + 1 - d0);
                        double a4[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
                        for (int r = 0; r < R; r++) {
                            const int l = r * kBT + t;
#pragma unroll
                            for (int q = 0; q < 4; q++)
                                if (q < nu) w[r] = fma(-c4[q], V[(u0 + q) * rpp + l], w[r]);
#pragma unroll
                            for (int q = 0; q < 4; q++)
                                if (q < nd) a4[q] = fma(w[r], V[(d0 + q) * rpp + l], a4[q]);
                        }
                        mput4(a4, Rd);
#pragma unroll
                        for (int q = 0; q < 4; q++)
                            if (q < nu) take(u0 + q, c4[q]);
                        slots_sum4<NCL>(mwait(Rd), a4);
#pragma unroll
                        for (int q = 0; q < 4; q++) c4[q] = a4[q];
                        u0 = d0;
                        nu = nd;
                    }
#pragma unroll
                    for (int r = 0; r < R; r++) {
                        const int l = r * kBT + t;
#pragma unroll
                        for (int q = 0; q < 4; q++)
                            if (q < nu) w[r] = fma(-c4[q], V[(u0 + q) * rpp + l], w[r]);
                    }
#pragma unroll
                    for (int q = 0; q < 4; q++) last[q] = c4[q];
                    nlast = nu;
                    i_last = u0;
                } else {
                    // fused MGS: pass i applies the projection on v_{i-1} and
                    // takes (w, v_i)
                    double hprev = 0.0;
                    if constexpr (R <= 4) {
                        // the thread's part of (w - h_{i-1} v_{i-1}, v_i) as
                        // (w, v_i) - h_{i-1} (v_{i-1}, v_i): the first part is
                        // formed while the previous exchange is in flight,
                        // the second once when v_i was written, so one FMA
                        // separates h_{i-1} from the next send (measured
                        // faster than the direct form at 2 and 4 rows per
                        // thread; at 8 the window's work would outgrow the
                        // exchange, and the direct form below serves it)
                        double p1 = 0.0, p2 = 0.0;
#pragma unroll
                        for (int r = 0; r < R; r++) p1 = fma(w[r], V[r * kBT + t], p1);
                        for (int i = 0; i <= j; i++) {
                            mput1(i == 0 ? p1 : fma(-hprev, p2, p1), Rd);
                            if (i > 0) {
#pragma unroll
                                for (int r = 0; r < R; r++)
                                    w[r] = fma(-hprev, V[(i - 1) * rpp + r * kBT + t], w[r]);
                            }
                            if (i < j) {
                                p1 = 0.0;
#pragma unroll
                                for (int r = 0; r < R; r++)
                                    p1 = fma(w[r], V[(i + 1) * rpp + r * kBT + t], p1);
                                p2 = P2[(i + 1) * kBT + t];
                            }
                            if (i > 0) take(i - 1, hprev);
                            hprev = slots_sum1<NCL>(mwait(Rd));
                        }
                    } else {
                        for (int i = 0; i <= j; i++) {
                            double a = 0.0;
#pragma unroll
                            for (int r = 0; r < R; r++) {
                                const int l = r * kBT + t;
                                if (i > 0) w[r] = fma(-hprev, V[(i - 1) * rpp + l], w[r]);
                                a = fma(w[r], V[i * rpp + l], a);
                            }
                            mput1(a, Rd);
                            if (i > 0) take(i - 1, hprev);
                            hprev = slots_sum1<NCL>(mwait(Rd));
                        }
                    }
#pragma unroll
                    for (int r = 0; r < R; r++) w[r] = fma(-hprev, V[j * rpp + r * kBT + t], w[r]);
                    last[0] = hprev;
                    nlast = 1;
                    i_last = j;
                }
                wb ^= 1;
                double a = 0.0;
#pragma unroll
                for (int r = 0; r < R; r++) {
                    wn[r * kBT + t] = w[r];  // published by the norm's barrier
                    a = fma(w[r], w[r], a);
                }
                bput1(a, Rd);
                for (int q = 0; q < nlast; q++) take(i_last + q, last[q]);
                const double hn2 = bget1(Rd);
                // the new rotation, from values every thread holds alike
                // (|h| <= ||A|| sqrt(m): no overflow in tt^2 + hn^2)
                int flag = 0;
                const double ihn = hn2 > 0.0 ? rsqrt(hn2) : 0.0, hn = hn2 * ihn;
                const double rr2 = fma(tt, tt, hn2);
                if (rr2 == 0.0) {
                    flag = 2;
                } else {
                    const double irr = rsqrt(rr2), c = tt * irr, s = hn * irr;
                    if (t == 0) {
                        cs[j] = c;
                        sn[j] = s;
                        H[j * ldh + j + 1] = rr2 * irr;  // the diagonal, until the restart
                        g[j] = c * gj;
                    }
                    gj = -s * gj;
                    if (hn2 <= 1e-28 * (len2 + hn2)) flag = 1;  // hn <= 1e-14 |column|
                    else if (fabs(gj) <= tol_g) flag = 3;
                }
                // thread 0's rotation, g, diagonal and raw column entries
                // visible to the CTA before their next use
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
                sc = ihn;
                double *Vn = V + (j + 1) * rpp;
#pragma unroll
                for (int r = 0; r < R; r++) Vn[r * kBT + t] = w[r] * sc;
                if constexpr (R <= 4) {
                    if (!A.bcgs) {  // MGS: (v_j, v_{j+1}), this thread's part
                        double pv = 0.0;
#pragma unroll
                        for (int r = 0; r < R; r++)
                            pv = fma(V[j * rpp + r * kBT + t], w[r] * sc, pv);
                        P2[(j + 1) * kBT + t] = pv;
                    }
                }
                if (flag == 3) {
                    claimed = 1;
                    break;
                }
                if (iters >= A.maxiter) break;
            }
            if (status == XB_EBREAKDOWN) break;
            // R y = g by columns on warp 0 (lane c holds g_c and 1 / R_cc;
            // every CTA holds the same R and g), then x += V y
            if (warp == 0) {
                __syncwarp();
                constexpr int QM = (XB_BATCH_MAX_M + 31) / 32;
                // lane c rotates column c's raw entries with G_0..G_{c-1} (the
                // arithmetic of the steps' running value) and moves its
                // diagonal into place
#pragma unroll
                for (int q = 0; q < QM; q++) {
                    const int c = lane + 32 * q;
                    if (c < k) {
                        double *col = H + c * ldh;
                        double tr = col[0];
                        for (int i = 1; i <= c; i++) {
                            const double hi = col[i], cc = cs[i - 1], ss = sn[i - 1];
                            col[i - 1] = fma(cc, tr, ss * hi);
                            tr = fma(-ss, tr, cc * hi);
                        }
                        col[c] = col[c + 1];
                    }
                }
                __syncwarp();
                double gl[QM], dl[QM];
#pragma unroll
                for (int q = 0; q < QM; q++) {
                    const int c = lane + 32 * q;
                    gl[q] = c < k ? g[c] : 0.0;
                    dl[q] = c < k ? 1.0 / H[c * ldh + c] : 0.0;
                }
                for (int i = k - 1; i >= 0; i--) {
                    const int qi = i >> 5, li = i & 31;
                    double gs = gl[0], ds = dl[0];
#pragma unroll
                    for (int q = 1; q < QM; q++)
                        if (qi == q) {
                            gs = gl[q];
                            ds = dl[q];
                        }
                    const double yi = __shfl_sync(kFull, gs, li) * __shfl_sync(kFull, ds, li);
                    if (lane == 0) yv[i] = yi;
#pragma unroll
                    for (int q = 0; q < QM; q++) {
                        const int c = lane + 32 * q;
                        if (32 * q < i && c < i) gl[q] = fma(-H[i * ldh + c], yi, gl[q]);
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < R; r++) {
                double s0 = 0.0;
                for (int i = 0; i < k; i++) s0 = fma(yv[i], V[i * rpp + r * kBT + t], s0);
                x[r] += s0;
            }
            restarts++;
        }
    }
    if (status != XB_EINVAL && status != XB_ETIMEOUT) {
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int l = r * kBT + t, row = (int)rank * A.rpc + l;
            if (l < A.rpc && row < A.n) A.x[row] = x[r];
        }
    }
    if (lead) {
        xb_batch_info inf;
        inf.status = status;
        inf.iters = iters;
        inf.restarts = restarts;
        inf.m = m;
        inf.mode = 2;
        inf.res_true = res_true;
        inf.ms = (double)(gtimer() - ts) * 1e-6;
        *A.out = inf;
    }
    // no CTA leaves while another may still write to its shared memory
    cl_arrive();
    cl_wait();
}

typedef void (*ResKernel)(const ResArgs);

template <int R>
ResKernel res_kernel_r(int ncl) {
    switch (ncl) {
        case 2: return k_gmres_resident<R, 2>;
        case 4: return k_gmres_resident<R, 4>;
        case 8: return k_gmres_resident<R, 8>;
        case 16: return k_gmres_resident<R, 16>;
        default: return nullptr;
    }
}

ResKernel res_kernel(int R, int ncl) {
    switch (R) {
        case 1: return res_kernel_r<1>(ncl);
        case 2: return res_kernel_r<2>(ncl);
        case 4: return res_kernel_r<4>(ncl);
        case 8: return res_kernel_r<8>(ncl);
        default: return nullptr;
    }
}

}  // namespace

namespace xb {

// Runs gmres_solve's FP64 GMRES(m) for plan p as one launch of the
// shared-memory-resident kernel when a cluster of 2, 4, 8 or 16 CTAs holds
// the system (at most 1024 rows per CTA, rows at most 64 long, the basis
// slice, ELL copy, Hessenberg and slots within the opt-in shared memory);
// *ran = false otherwise (nothing launched).  The cluster is the smallest
// whose CTAs hold at most 128 rows (one row per thread), else the largest
// that fits (fewest rows per thread).  The environment variable
// XB_RESIDENT_CL = 0 turns the path off, a cluster size forces it.
int resident_gmres(xb_plan *p, const double *b, double *x, const xb_options &o, xb_info &inf,
                   double *alg_bytes, cudaStream_t s, bool *ran) {
    *ran = false;
    int force = -1;
    if (const char *env = std::getenv("XB_RESIDENT_CL")) force = std::atoi(env);
    if (force == 0 || p->n < 1 || p->max_row > kMaxRow || p->n > 16 * 8 * kBT) return XB_OK;
    const int mmax = o.dafrt ? std::max(o.m, std::min(o.m_max, XB_BATCH_MAX_M)) : o.m;
    if (mmax > XB_BATCH_MAX_M) return XB_OK;
    int dev = 0, optin = 0;
    XB_CUDA(cudaGetDevice(&dev));
    XB_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int lmax = std::max(1, p->max_row);
    // candidates in order of preference
    int order[4], no = 0;
    if (force > 0) {
        order[no++] = force;
    } else {
        int first = 16;
        for (int c : {2, 4, 8, 16})
            if ((p->n + c - 1) / c <= kBT) {
                first = c;
                break;
            }
        order[no++] = first;
        for (int c : {16, 8, 4, 2})
            if (c != first) order[no++] = c;
    }
    ResArgs a;
    std::memset(&a, 0, sizeof a);
    size_t bytes = 0;
    ResKernel kern = nullptr;
    int chosen = 0;
    for (int z = 0; z < no; z++) {
        const int ncl = order[z];
        if (ncl != 2 && ncl != 4 && ncl != 8 && ncl != 16) continue;
        const int rpc = (p->n + ncl - 1) / ncl;
        int R = 1;
        while (R * kBT < rpc) R *= 2;
        ResKernel kf = res_kernel(R, ncl);
        if (!kf) continue;
        const ResLayout L = res_layout(kBT * R, lmax, mmax, ncl * kW);
        if (L.total > (size_t)optin) continue;
        XB_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
        if (ncl > 8) XB_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = ncl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(ncl);
        cfg.blockDim = dim3(kBT);
        cfg.dynamicSmemBytes = L.total;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, (void *)kf, &cfg) != cudaSuccess || clusters < 1) {
            cudaGetLastError();
            continue;
        }
        chosen = ncl;
        a.rpc = rpc;
        bytes = L.total;
        kern = kf;
        break;
    }
    if (!kern) return XB_OK;
    XB_TRY(ensure_work(p, sizeof(xb_batch_info)));
    xb_batch_info *d_info = static_cast<xb_batch_info *>(p->d_work);
    a.n = p->n;
    a.lmax = lmax;
    a.m = o.m;
    a.m_max = mmax;
    a.maxiter = o.maxiter;
    a.bcgs = o.ortho == XB_ORTHO_BCGS ? 1 : 0;
    a.tol = o.tol;
    a.theta = o.dafrt ? o.dafrt_theta : 0.0;
    a.budget_ns = (unsigned long long)(std::min(o.maxtime_s, 3600.0) * 1e9);
    a.rowptr = p->rowptr;
    a.col = p->col;
    a.val = p->val;
    a.b = b;
    a.x = x;
    a.out = d_info;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = chosen;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(chosen);
    cfg.blockDim = dim3(kBT);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    XB_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
    XB_LAUNCHED("k_gmres_resident");
    xb_batch_info r;
    XB_CUDA(cudaMemcpyAsync(&r, d_info, sizeof r, cudaMemcpyDeviceToHost, s));
    XB_CUDA(cudaStreamSynchronize(s));
    *ran = true;
    inf.iters = r.iters;
    inf.restarts = r.restarts;
    inf.m_final = r.m;
    inf.res_true = r.res_true;
    inf.ortho_used = a.bcgs ? XB_ORTHO_BCGS : XB_ORTHO_MGS;
    inf.persistent = 2;
    // algorithmic bytes, counted as for the multi-launch step: per Arnoldi
    // step one SpMV and the Gram-Schmidt passes at the cycle's mean basis
    // size, plus a residual per restart
    const double jm = (r.m + 1) / 2.0, n = a.n;
    *alg_bytes = r.iters * (spmv_alg_bytes(p, false, 8) + (4.0 * jm + 5.0) * 8.0 * n) +
                 (r.restarts + 1) * (spmv_alg_bytes(p, true, 8) + 16.0 * n);
    if (r.status == XB_EINVAL)
        return set_error(XB_EINVAL, "gmres: column index outside [0, n) in the matrix");
    if (r.status == XB_ETIMEOUT)
        return set_error(XB_ETIMEOUT, "gmres: an inner-product exchange of the cluster timed out");
    if (r.status == XB_ENOCONV)
        return set_error(XB_ENOCONV, "not converged: ||b-Ax||/||b|| = %.3e > tol %.1e", r.res_true,
                         o.tol);
    return r.status;
}

}  // namespace xb
