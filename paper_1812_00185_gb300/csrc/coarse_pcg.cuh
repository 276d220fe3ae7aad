// Whole coarse-Poisson solve (Eq. 23) in ONE kernel launch.
//
// The coarse system of a CGP step is small (tens of thousands of rows, a few MB, L2
// resident): a PCG with two kernel launches per iteration is bound by launch and
// grid-synchronisation latency.  This kernel keeps every iteration on the device and
// synchronises in one of two ways (the Sync policy):
//
//  * GridSync: a cooperative launch over the whole GPU (every CTA co-resident); the
//    reductions go through per-CTA partial sums in global memory and a software grid
//    barrier (one atomic arrive per CTA, a bounded acquire-spin; on timeout every CTA
//    leaves with CGP_ETIMEOUT instead of hanging).
//  * ClusterSync: one thread-block cluster (up to 16 CTAs); the reductions go through
//    distributed shared memory after a hardware cluster barrier.
//
// Either way every CTA adds the per-CTA sums in the same fixed order, so all CTAs hold
// bit-identical scalars and take identical branches (the barrier counts always match).
// Vectors written inside the kernel are read with ld.global.cg (L2), never through the
// incoherent L1; read-only data (pattern, values, Jacobi diagonal) goes through the
// read-only path.
//
// The PCG recurrence is Chronopoulos and Gear's: both dot products of an iteration are
// formed after its vector updates, so one grid-wide reduction (one barrier) per iteration
// suffices; w = A u is carried by a recurrence and double-buffered because the SpMV of an
// iteration gathers w at neighbouring rows while its own rows are being rewritten.
//
// Mixed precision (iterative refinement, CGP_MIXED): the outer residual r = b - A x, its
// norm and the convergence test are FP64; each inner PCG runs its SpMV and vector updates
// in FP32 on an FP32 copy of the matrix, with FP64 accumulation of the dot products.
#pragma once

#include <cooperative_groups.h>

#include "krylov.cuh"

namespace cgp {

namespace cgrp = cooperative_groups;

constexpr int kClusterThreads = 1024;
constexpr int kGridThreads = 256;
constexpr unsigned kSpinLimit = 1u << 24;   // polls of one grid barrier before giving up (~seconds)
constexpr unsigned kSpinLimitTest = 1u << 14;   // the same under the wait test hook (milliseconds)
constexpr int kStagnation = 2000;           // FP64 inner iterations without halving the best residual
constexpr int kStagnation32 = 300;          // the same for the FP32 inner solve of the mixed form

struct CoarsePcgArgs {
    SellView A;
    const double* val;      // FP64 matrix (SELL values)
    const float* valf;      // FP32 copy (mixed precision) or nullptr
    const double* dinv;
    const float* dinvf;
    double* b;              // rhs (projected in place when `project`)
    double* x;              // solution / initial guess
    const double* x_alt;    // optional second initial guess: used instead of x when its FP64 residual is smaller
    double* w64;            // FP64 work: 8 vectors of n (r, u, w0, w1, z, q, s, p)
    float* w32;             // FP32 work: 9 vectors of n (r, u, w0, w1, z, q, s, p, e)
    const double* mlump;    // non-null: fix sum m_i x_i = 0 after the solve (pure Neumann)
    KrylovState* st;        // out: iter (inner iterations), rr, bb, status, done; in: mean when project
    double tol2;
    double inner_tol;       // mixed: relative reduction asked of each inner solve
    int maxit;
    int zero_x, project, mixed;
    int max_outer;
    // GridSync only
    unsigned int* bar_count;   // zeroed before the launch
    int* bar_err;              // zeroed before the launch; set on a barrier timeout
    double* partials;          // 2 slots x gridDim x 4 doubles
    // test hook (cgp_set_wait_test; 0 otherwise): every bounded wait also waits for one
    // signal that nothing sends, under a limit of milliseconds, so the solve ends with
    // CGP_ETIMEOUT without a fault or a hang
    int wait_test;
    // the learned guess's judge (on-chip solve only; null otherwise): gate[0] = steps left in
    // which the network is not evaluated, gate[1] = consecutive steps in which its direction
    // lowered the starting residual by less than 5 %
    int* gate;
};

template <class T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

// ------------------------------------------------------------------ sync policies
struct ClusterSync {
    cgrp::cluster_group cluster;
    double (*slots)[4];
    double (*wsum)[4];
    int slot = 0;
    __device__ ClusterSync(double (*sl)[4], double (*ws)[4]) : cluster(cgrp::this_cluster()), slots(sl), wsum(ws) {}
    __device__ int part() const { return (int)cluster.block_rank(); }
    __device__ int parts() const { return (int)cluster.num_blocks(); }
    __device__ bool sync() {
        cluster.sync();
        return true;
    }
    template <int NR>
    __device__ bool sum(double (&v)[NR], double (&tot)[NR]) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            double s = warp_sum(v[k]);
            if (lane == 0) wsum[wid][k] = s;
        }
        __syncthreads();
        if (wid == 0) {
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                double s = lane < nw ? wsum[lane][k] : 0.0;
                s = warp_sum(s);
                if (lane == 0) slots[slot][k] = s;
            }
        }
        cluster.sync();
        __shared__ double bcast[4];
        if (wid == 0) {
            const int ncl = parts();
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                double s = 0.0;
                if (lane < ncl) s = cluster.map_shared_rank(&slots[slot][0], lane)[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
                if (lane == 0) bcast[k] = s;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NR; ++k) tot[k] = bcast[k];
        __syncthreads();
        slot ^= 1;
        return true;
    }
    __device__ void finish() { cluster.sync(); }   // no CTA leaves while its shared memory may be read
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

struct GridSync {
    unsigned* count;
    int* err;
    double* partials;
    double (*wsum)[4];
    unsigned gen = 0;
    int slot = 0;
    unsigned extra = 0;            // arrivals awaited beyond the grid's (1 under the wait test hook)
    unsigned limit = kSpinLimit;
    __device__ GridSync(unsigned* c, int* e, double* p, double (*ws)[4], int wait_test = 0)
        : count(c), err(e), partials(p), wsum(ws), extra(wait_test ? 1u : 0u),
          limit(wait_test ? kSpinLimitTest : kSpinLimit) {}
    __device__ int part() const { return (int)blockIdx.x; }
    __device__ int parts() const { return (int)gridDim.x; }
    __device__ bool sync() {
        __shared__ int ok;
        __syncthreads();
        ++gen;
        if (threadIdx.x == 0) {
            int good = 1;
            // arrive: a release-ordered add publishes this CTA's writes (cumulative over the
            // CTA through the barrier above); wait: acquire-spin on the counter
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
            const unsigned target = gen * gridDim.x + extra;
            unsigned spins = 0;
            for (;;) {
                const unsigned v = ld_acquire_gpu(count);
                if ((int)(v - target) >= 0) break;
                if (++spins > limit) {
                    atomicExch(err, 1);
                    good = 0;
                    break;
                }
                if ((spins & 63) == 0 && *(volatile int*)err) {
                    good = 0;
                    break;
                }
            }
            ok = good;
        }
        __syncthreads();
        return ok != 0;
    }
    template <int NR>
    __device__ bool sum(double (&v)[NR], double (&tot)[NR]) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            double s = warp_sum(v[k]);
            if (lane == 0) wsum[wid][k] = s;
        }
        __syncthreads();
        double* my = partials + ((size_t)slot * gridDim.x + blockIdx.x) * 4;
        if (wid == 0) {
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                double s = lane < nw ? wsum[lane][k] : 0.0;
                s = warp_sum(s);
                if (lane == 0) __stcg(my + k, s);
            }
        }
        if (!sync()) return false;
        // every CTA adds the gridDim partials in the same order: lane l takes l, l+32, ...
        __shared__ double bcast[4];
        if (wid == 0) {
            const double* base = partials + (size_t)slot * gridDim.x * 4;
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                double s = 0.0;
                for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(base + (size_t)b * 4 + k);
                s = warp_sum(s);
                if (lane == 0) bcast[k] = s;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NR; ++k) tot[k] = bcast[k];
        __syncthreads();
        slot ^= 1;
        return true;
    }
    __device__ void finish() {}
};

// FP32 counterpart of sell_accum (FP32 values, FP32 gathered vector, FP32 sum)
template <class Gather>
__device__ __forceinline__ float sell_accum_f(const SellView& A, const float* __restrict__ val, int sl, int lane,
                                              Gather&& g) {
    const int base = __ldg(A.ptr + sl), w = (__ldg(A.ptr + sl + 1) - base) >> 5;
    float s = 0.0f;
    for (int k0 = 0; k0 < w; k0 += 8) {
        int cj[8];
        float av[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            cj[u] = 0;
            av[u] = 0.0f;
            if (k0 + u < w) {
                const int e = base + 32 * (k0 + u) + lane;
                cj[u] = __ldg(A.col + e);
                av[u] = __ldg(val + e);
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (k0 + u < w) s += av[u] * g(cj[u]);
    }
    return s;
}

// ------------------------------------------------------------------ the solve
template <class T>
struct InnerVecs {
    T *r, *u, *w0, *w1, *z, *q, *s, *p, *e;
};

// sum_k val(row,k) * g(col(row,k)) in precision T (FP32 values for T = float)
template <class T, class Gather>
__device__ __forceinline__ T row_spmv(const SellView& A, const double* __restrict__ v64, const float* __restrict__ v32,
                                      int sl, int lane, Gather&& g) {
    if constexpr (sizeof(T) == 4) {
        return sell_accum_f(A, v32, sl, lane, g);
    } else {
        double acc[1] = {0.0};
        sell_accum<1>(A, v64, sl, lane, [&](int j, double (&o)[1]) { o[0] = g(j); }, acc);
        return acc[0];
    }
}

// Inner PCG (Chronopoulos-Gear) on A e = r0 in precision T, starting from e = 0 and from
// r = r0, u = D^{-1} r0 already in V (written before the last barrier).  gamma0 = <r0,u0>.
// Returns false on a barrier timeout.  iters counts iterations across calls.
// outcome: 0 = ended normally (target met, or stagnation), 1 = breakdown before an update
// (the iterate is intact), 2 = a non-finite value after an update (the iterate is not).
template <class T, class Sync>
__device__ bool inner_pcg(const CoarsePcgArgs& a, Sync& sy, const InnerVecs<T>& V, const T* __restrict__ dinv,
                          int s_begin, int s_end, double gamma, double stop2, int& iters, int& outcome,
                          double& rr_last, bool& done) {
    outcome = 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const SellView& A = a.A;
    // w0 = A u, delta = <w0, u>
    {
        double acc[1] = {0.0};
        for (int sl = s_begin + wid; sl < s_end; sl += nw) {
            const int i = sl * 32 + lane;
            const T wv = row_spmv<T>(A, a.val, a.valf, sl, lane, [&](int j) { return ldcg(V.u + j); });
            if (i < A.n) {
                __stcg(V.w0 + i, wv);
                acc[0] += (double)wv * (double)ldcg(V.u + i);
            }
        }
        double tot[1];
        if (!sy.template sum<1>(acc, tot)) return false;
        double delta = tot[0];
        T* wc = V.w0;
        T* wn = V.w1;
        double gamma_prev = 0.0, alpha_prev = 0.0;
        double rr_best = INFINITY;
        int best_k = 0;
        done = false;
        for (int k = 0; iters < a.maxit; ++k) {
            double alpha, beta;
            if (k == 0) {
                beta = 0.0;
                alpha = gamma / delta;
            } else {
                beta = gamma / gamma_prev;
                alpha = gamma / (delta - beta * gamma / alpha_prev);
            }
            if (!isfinite(alpha) || alpha == 0.0) {
                outcome = 1;
                return true;
            }
            const T al = (T)alpha, be = (T)beta;
            double part[3] = {0.0, 0.0, 0.0};
            for (int sl = s_begin + wid; sl < s_end; sl += nw) {
                const int i = sl * 32 + lane;
                const T n_i = row_spmv<T>(A, a.val, a.valf, sl, lane,
                                          [&](int j) { return __ldg(dinv + j) * ldcg(wc + j); });
                if (i >= A.n) continue;
                const T w_i = ldcg(wc + i);
                const T m_i = __ldg(dinv + i) * w_i;
                const T z_i = k ? n_i + be * ldcg(V.z + i) : n_i;
                const T q_i = k ? m_i + be * ldcg(V.q + i) : m_i;
                const T s_i = k ? w_i + be * ldcg(V.s + i) : w_i;
                const T p_i = k ? ldcg(V.u + i) + be * ldcg(V.p + i) : ldcg(V.u + i);
                __stcg(V.z + i, z_i);
                __stcg(V.q + i, q_i);
                __stcg(V.s + i, s_i);
                __stcg(V.p + i, p_i);
                __stcg(V.e + i, ldcg(V.e + i) + al * p_i);
                const T r_i = ldcg(V.r + i) - al * s_i;
                const T u_i = ldcg(V.u + i) - al * q_i;
                const T wn_i = w_i - al * z_i;
                __stcg(V.r + i, r_i);
                __stcg(V.u + i, u_i);
                __stcg(wn + i, wn_i);
                part[0] += (double)r_i * (double)u_i;
                part[1] += (double)wn_i * (double)u_i;
                part[2] += (double)r_i * (double)r_i;
            }
            double t3[3];
            if (!sy.template sum<3>(part, t3)) return false;
            ++iters;
            gamma_prev = gamma;
            alpha_prev = alpha;
            gamma = t3[0];
            delta = t3[1];
            rr_last = t3[2];
            if (!isfinite(t3[2]) || !isfinite(t3[0]) || !isfinite(t3[1])) {
                outcome = 2;
                return true;
            }
            if (t3[0] == 0.0 || t3[2] == 0.0) {   // exact solution reached: nothing left to do
                done = true;
                return true;
            }
            T* tmp = wc;
            wc = wn;
            wn = tmp;
            if (t3[2] <= stop2) {
                done = true;
                return true;
            }
            // the recursive residual of this recurrence can stagnate above a very tight
            // target; hand back to the caller, which restarts from the true residual.  CG
            // residual norms are not monotone, so only a long run without a new minimum counts.
            if (t3[2] < 0.5 * rr_best) {
                rr_best = t3[2];
                best_k = k;
            } else if (sizeof(T) == 4 && t3[2] > 1e4 * rr_best) {
                outcome = 2;   // the FP32 recurrence is drifting away: its iterate is not to be used
                return true;
            } else if (k - best_k > (sizeof(T) == 4 ? kStagnation32 : kStagnation)) {
                return true;   // stagnating: restart from the true residual
            }
        }
    }
    return true;
}

// Inner PCG in its classical form (two reductions per iteration) on A e = r0 in precision
// T, from e = 0 and r = r0, u = D^{-1} r0 in V; p and q use V.p/V.s (p double-buffered
// with V.q because the SpMV gathers p at neighbouring rows while rows are rewritten).
// Used for the FP32 inner solves of the mixed form, where the longer recurrence of the
// one-reduction form drifts.  Same outcome codes as inner_pcg.
template <class T, class Sync>
__device__ bool inner_pcg_classic(const CoarsePcgArgs& a, Sync& sy, const InnerVecs<T>& V,
                                  const T* __restrict__ dinv, int s_begin, int s_end, double rz, double stop2,
                                  int& iters, int& outcome, bool& done) {
    outcome = 0;
    done = false;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const SellView& A = a.A;
    T* p_old = V.u;   // the first direction is z = u itself
    T* p_new = V.p;
    T* z = V.u;       // u holds D^{-1} r
    T* q = V.q;
    double beta = 0.0, rr_best = INFINITY;
    int best_k = 0;
    for (int k = 0; iters < a.maxit; ++k) {
        // phase A: p_new = z + beta p_old (p_old = z at k = 0), q = A p_new, <p_new, q>
        const T be = (T)beta;
        double pq_acc[1] = {0.0};
        for (int sl = s_begin + wid; sl < s_end; sl += nw) {
            const int i = sl * 32 + lane;
            const T qi = row_spmv<T>(A, a.val, a.valf, sl, lane,
                                     [&](int j) { return k ? ldcg(z + j) + be * ldcg(p_old + j) : ldcg(z + j); });
            if (i < A.n) {
                const T pv = k ? ldcg(z + i) + be * ldcg(p_old + i) : ldcg(z + i);
                __stcg(p_new + i, pv);
                __stcg(q + i, qi);
                pq_acc[0] += (double)pv * (double)qi;
            }
        }
        double pq[1];
        if (!sy.template sum<1>(pq_acc, pq)) return false;
        if (!(pq[0] != 0.0) || !isfinite(pq[0])) {
            outcome = 1;
            return true;
        }
        const double alpha = rz / pq[0];
        const T al = (T)alpha;
        // phase B: e += alpha p, r -= alpha q, z = D^{-1} r; <r,z>, <r,r>
        double acc2[2] = {0.0, 0.0};
        for (int sl = s_begin + wid; sl < s_end; sl += nw) {
            const int i = sl * 32 + lane;
            if (i >= A.n) continue;
            __stcg(V.e + i, ldcg(V.e + i) + al * ldcg(p_new + i));
            const T rv = ldcg(V.r + i) - al * ldcg(q + i);
            const T zv = __ldg(dinv + i) * rv;
            __stcg(V.r + i, rv);
            __stcg(V.z + i, zv);
            acc2[0] += (double)rv * (double)zv;
            acc2[1] += (double)rv * (double)rv;
        }
        double t2[2];
        if (!sy.template sum<2>(acc2, t2)) return false;
        ++iters;
        if (!isfinite(t2[0]) || !isfinite(t2[1])) {
            outcome = 2;
            return true;
        }
        if (t2[0] == 0.0 || t2[1] == 0.0) {
            done = true;
            return true;
        }
        beta = t2[0] / rz;
        rz = t2[0];
        // from now on z lives in V.z, and the directions alternate between V.p and V.s
        z = V.z;
        p_old = p_new;
        p_new = (p_new == V.p) ? V.s : V.p;
        if (t2[1] <= stop2) {
            done = true;
            return true;
        }
        if (t2[1] < 0.5 * rr_best) {
            rr_best = t2[1];
            best_k = k;
        } else if (t2[1] > 1e4 * rr_best) {
            outcome = 2;
            return true;
        } else if (k - best_k > kStagnation32) {
            return true;
        }
    }
    return true;
}

template <class Sync>
__device__ void coarse_pcg_body(const CoarsePcgArgs& a, Sync& sy) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const SellView& A = a.A;
    const int part = sy.part(), parts = sy.parts();
    const int s_begin = (int)(((int64_t)A.nslices * part) / parts);
    const int s_end = (int)(((int64_t)A.nslices * (part + 1)) / parts);
    const double mean = a.project ? a.st->mean : 0.0;
    const double tol2 = a.tol2;
    const size_t n = (size_t)A.n;
    double* xv = a.x;
    InnerVecs<double> V64{a.w64, a.w64 + n, a.w64 + 2 * n, a.w64 + 3 * n, a.w64 + 4 * n, a.w64 + 5 * n,
                          a.w64 + 6 * n, a.w64 + 7 * n, xv};
    InnerVecs<float> V32{a.w32, a.w32 + n, a.w32 + 2 * n, a.w32 + 3 * n, a.w32 + 4 * n, a.w32 + 5 * n,
                         a.w32 + 6 * n, a.w32 + 7 * n, a.w32 + 8 * n};
    double bb = 0.0, rr_final = 0.0;
    int iters = 0, status = 0, outer = 0, used_alt = 0;
    bool mixed_now = a.mixed != 0;   // cleared if an FP32 inner solve ever produces a non-finite value
    bool converged = false;
    if (a.x_alt && !a.zero_x) {
        // the judge of the learned guess: keep whichever start has the smaller FP64 residual
        double acc[2] = {0.0, 0.0};
        for (int sl = s_begin + wid; sl < s_end; sl += nw) {
            const int i = sl * 32 + lane;
            double ax[1] = {0.0}, aa[1] = {0.0};
            sell_accum<1>(A, a.val, sl, lane, [&](int j, double (&o)[1]) { o[0] = ldcg(xv + j); }, ax);
            sell_accum<1>(A, a.val, sl, lane, [&](int j, double (&o)[1]) { o[0] = __ldg(a.x_alt + j); }, aa);
            if (i < A.n) {
                const double bi = a.b[i] - mean;
                acc[0] += (bi - ax[0]) * (bi - ax[0]);
                acc[1] += (bi - aa[0]) * (bi - aa[0]);
            }
        }
        double tot[2];
        bool ok = sy.template sum<2>(acc, tot);
        if (ok && tot[1] < tot[0]) {
            used_alt = 1;
            for (int sl = s_begin + wid; sl < s_end; sl += nw) {
                const int i = sl * 32 + lane;
                if (i < A.n) __stcg(xv + i, __ldg(a.x_alt + i));
            }
            ok = sy.sync();
        }
        if (!ok) status = CGP_ETIMEOUT;
    }
    for (; status == 0;) {
        // ---- outer residual r = b - A x (FP64), ||r||^2, ||b||^2, inner start r, u = D^{-1} r
        double acc[3] = {0.0, 0.0, 0.0};
        for (int sl = s_begin + wid; sl < s_end; sl += nw) {
            const int i = sl * 32 + lane;
            double axv[1] = {0.0};
            if (!(a.zero_x && outer == 0))
                sell_accum<1>(A, a.val, sl, lane, [&](int j, double (&o)[1]) { o[0] = ldcg(xv + j); }, axv);
            if (i < A.n) {
                double bi = a.b[i];
                if (a.project && outer == 0) {
                    bi -= mean;
                    a.b[i] = bi;
                }
                if (a.zero_x && outer == 0) __stcg(xv + i, 0.0);
                const double ri = bi - axv[0];
                if (mixed_now) {
                    const float rf = (float)ri;
                    const float uf = __ldg(a.dinvf + i) * rf;
                    __stcg(V32.r + i, rf);
                    __stcg(V32.u + i, uf);
                    __stcg(V32.e + i, 0.0f);
                    acc[2] += (double)rf * (double)uf;
                } else {
                    const double ui = __ldg(a.dinv + i) * ri;
                    __stcg(V64.r + i, ri);
                    __stcg(V64.u + i, ui);
                    acc[2] += ri * ui;
                }
                acc[0] += ri * ri;
                acc[1] += bi * bi;
            }
        }
        double tot[3];
        if (!sy.template sum<3>(acc, tot)) {
            status = CGP_ETIMEOUT;
            break;
        }
        if (outer == 0) bb = tot[1];
        const double rr0 = tot[0];
        rr_final = rr0;
        if (!isfinite(rr0)) {
            status = CGP_ENONFINITE;
            break;
        }
        if (rr0 <= tol2 * bb) {
            converged = true;
            break;
        }
        if (outer >= a.max_outer || iters >= a.maxit) {
            status = CGP_ENOTCONV;
            break;
        }
        bool inner_done = false;
        bool ok;
        int outcome = 0;
        double rr_in = 0.0;
        if (mixed_now) {
            const double stop2 = fmax(a.inner_tol * a.inner_tol * rr0, 0.25 * tol2 * bb);
            ok = inner_pcg_classic<float>(a, sy, V32, a.dinvf, s_begin, s_end, tot[2], stop2, iters, outcome,
                                          inner_done);
        } else {
            // FP64: the inner recurrence updates x itself; the next outer pass re-checks the true residual
            ok = inner_pcg<double>(a, sy, V64, a.dinv, s_begin, s_end, tot[2], 0.25 * tol2 * bb, iters, outcome,
                                   rr_in, inner_done);
        }
        if (!ok) {
            status = CGP_ETIMEOUT;
            break;
        }
        if (outcome == 2 && !mixed_now) {
            status = CGP_ENONFINITE;   // x itself is no longer finite
            break;
        }
        if (outcome == 2) {
            // the FP32 correction blew up: drop it and finish this solve with FP64 inner solves
            mixed_now = false;
        } else if (mixed_now) {
            for (int sl = s_begin + wid; sl < s_end; sl += nw) {
                const int i = sl * 32 + lane;
                if (i < A.n) __stcg(xv + i, ldcg(xv + i) + (double)ldcg(V32.e + i));
            }
        }
        // x is complete before any CTA forms the next outer residual
        if (!sy.sync()) {
            status = CGP_ETIMEOUT;
            break;
        }
        ++outer;
    }
    // ---- pure-Neumann mean fix: x -= sum(m x) / sum(m)
    if (a.mlump && status != CGP_ETIMEOUT) {
        bool ok = sy.sync();
        double acc[2] = {0.0, 0.0};
        for (int sl = s_begin + wid; sl < s_end; sl += nw) {
            const int i = sl * 32 + lane;
            if (i < A.n) {
                acc[0] += __ldg(a.mlump + i) * ldcg(xv + i);
                acc[1] += __ldg(a.mlump + i);
            }
        }
        double tot[2];
        ok = ok && sy.template sum<2>(acc, tot);
        if (ok) {
            const double mu = tot[0] / tot[1];
            for (int sl = s_begin + wid; sl < s_end; sl += nw) {
                const int i = sl * 32 + lane;
                if (i < A.n) __stcg(xv + i, ldcg(xv + i) - mu);
            }
        } else {
            status = CGP_ETIMEOUT;
        }
    }
    if (part == 0 && threadIdx.x == 0) {
        KrylovState* st = a.st;
        st->iter = iters;
        st->bb[0] = bb;
        st->rr[0] = rr_final;
        st->bb[1] = 0.0;
        st->rr[1] = 0.0;
        st->status = status ? status : (converged ? 0 : CGP_ENOTCONV);
        st->done = 1;
        st->pad[0] = outer;
        st->pad[1] = used_alt;
    }
    sy.finish();
}

static __global__ void __launch_bounds__(kClusterThreads, 1) k_pcg_cluster(CoarsePcgArgs a) {
    __shared__ double slots[2][4];
    __shared__ double wsum[kClusterThreads / 32][4];
    ClusterSync sy(slots, wsum);
    coarse_pcg_body(a, sy);
}

// Coarse solves of many independent CGP instances in ONE persistent launch: every cluster
// of the launch takes instances from a queue (the host orders them largest first) and
// solves each with the ClusterSync body; clusters never wait on one another.
static __global__ void __launch_bounds__(kClusterThreads, 1) k_pcg_batch(const CoarsePcgArgs* __restrict__ args, int ninst,
                                                                  unsigned int* queue) {
    __shared__ double slots[2][4];
    __shared__ double wsum[kClusterThreads / 32][4];
    __shared__ int job;
    ClusterSync sy(slots, wsum);
    for (;;) {
        if (sy.part() == 0 && threadIdx.x == 0) job = (int)atomicAdd(queue, 1u);
        sy.cluster.sync();
        const int j = *sy.cluster.map_shared_rank(&job, 0);
        sy.cluster.sync();   // every CTA has read rank 0's job before it can change
        if (j >= ninst) break;
        const CoarsePcgArgs a = args[j];
        coarse_pcg_body(a, sy);
    }
}

static __global__ void __launch_bounds__(kGridThreads) k_pcg_grid(CoarsePcgArgs a) {
    __shared__ double wsum[kGridThreads / 32][4];
    GridSync sy(a.bar_count, a.bar_err, a.partials, wsum, a.wait_test);
    coarse_pcg_body(a, sy);
}

}  // namespace cgp
