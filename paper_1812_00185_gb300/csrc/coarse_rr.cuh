// Register-resident variant of the one-launch FP64 coarse solve (Eq. 23).
//
// When every warp of the cooperative launch owns at most one SELL-32 slice (32 rows) and no
// row has more than kRRWidth entries, each thread keeps for its row, for the whole solve:
// the pattern, the Jacobi-scaled values A_ij / a_jj, and all PCG vectors (x, r, u, z, q,
// s, p, w).  Only two vectors ever go through memory: w (the SpMV of an iteration gathers
// w at neighbouring rows) and x / u at the few points where a full SpMV of them is needed.
// An iteration is then one gather, ~20 FP64 operations per row and one grid reduction.
// Same recurrences as coarse_pcg_body (Chronopoulos-Gear inner solve, FP64 true-residual
// outer loop with restart on stagnation, optional second initial guess, pure-Neumann mean
// fix), same results up to rounding order.
#pragma once

#include "coarse_pcg.cuh"

namespace cgp {

constexpr int kRRWidth = 16;

// true when the register-resident solve applies: width <= kRRWidth everywhere (checked by
// the caller on the host) and at most one slice per warp
__host__ __device__ __forceinline__ int rr_ctas_needed(int nslices) { return (nslices + kGridThreads / 32 - 1) / (kGridThreads / 32); }

template <class Sync>
__device__ void coarse_pcg_rr_body(const CoarsePcgArgs& a, Sync& sy) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const SellView& A = a.A;
    const int sl = (int)blockIdx.x * nw + wid;              // this warp's slice (one at most)
    const bool has = sl < A.nslices;
    const int i = sl * 32 + lane;
    const bool row = has && i < A.n;
    // ---- row data, loaded once
    int col[kRRWidth];
    double bval[kRRWidth];   // A_ij / a_jj (the unscaled A_ij are re-read for the rare full SpMVs)
    int w_ = 0, base = 0;
    double dinv_i = 0.0, b_i = 0.0;
    if (has) {
        base = __ldg(A.ptr + sl);
        w_ = (__ldg(A.ptr + sl + 1) - base) >> 5;
#pragma unroll
        for (int k = 0; k < kRRWidth; ++k) {
            col[k] = 0;
            bval[k] = 0.0;
            if (k < w_) {
                const int e = base + 32 * k + lane;
                col[k] = __ldg(A.col + e);
                bval[k] = __ldg(a.val + e) * __ldg(a.dinv + col[k]);
            }
        }
    }
    const double mean = a.project ? a.st->mean : 0.0;
    if (row) {
        dinv_i = __ldg(a.dinv + i);
        b_i = a.b[i];
        if (a.project) {
            b_i -= mean;
            a.b[i] = b_i;
        }
    }
    const size_t n = (size_t)A.n;
    double* ubuf = a.w64;              // u at the start of an inner solve
    double* wbuf[2] = {a.w64 + n, a.w64 + 2 * n};
    double* xv = a.x;
    // (B v)_i with the register-held scaled values
    auto gather_b = [&](const double* v) {
        double s = 0.0;
        double g[kRRWidth];
#pragma unroll
        for (int k = 0; k < kRRWidth; ++k) g[k] = k < w_ ? ldcg(v + col[k]) : 0.0;
#pragma unroll
        for (int k = 0; k < kRRWidth; ++k) s += bval[k] * g[k];
        return s;
    };
    // (A v)_i with the values re-read from memory; `ro` = v is read-only during the kernel
    auto gather_a = [&](const double* v, bool ro) {
        double s = 0.0;
        double g[kRRWidth], av[kRRWidth];
#pragma unroll
        for (int k = 0; k < kRRWidth; ++k) {
            g[k] = 0.0;
            av[k] = 0.0;
            if (k < w_) {
                g[k] = ro ? __ldg(v + col[k]) : ldcg(v + col[k]);
                av[k] = __ldg(a.val + base + 32 * k + lane);
            }
        }
#pragma unroll
        for (int k = 0; k < kRRWidth; ++k) s += av[k] * g[k];
        return s;
    };
    double x_i = 0.0;
    int iters = 0, status = 0, outer = 0, used_alt = 0;
    double bb = 0.0, rr_final = 0.0;
    bool converged = false;
    // ---- initial guess (the judge of a second candidate compares FP64 residuals)
    if (a.zero_x) {
        if (row) __stcg(xv + i, 0.0);
        if (!sy.sync()) status = CGP_ETIMEOUT;
    } else if (a.x_alt) {
        double acc[2] = {0.0, 0.0};
        double ax = 0.0, aa = 0.0;
        if (has) {
            ax = gather_a(xv, false);
            aa = gather_a(a.x_alt, true);
        }
        if (row) {
            acc[0] = (b_i - ax) * (b_i - ax);
            acc[1] = (b_i - aa) * (b_i - aa);
        }
        double tot[2];
        bool ok = sy.template sum<2>(acc, tot);
        if (ok && tot[1] < tot[0]) {
            used_alt = 1;
            if (row) __stcg(xv + i, __ldg(a.x_alt + i));
            ok = sy.sync();
        }
        if (!ok) status = CGP_ETIMEOUT;
    }
    if (row) x_i = ldcg(xv + i);
    while (status == 0) {
        // ---- outer: r = b - A x (x is in memory and synchronised), u = D^{-1} r
        double r_i = 0.0, u_i = 0.0;
        double acc[3] = {0.0, 0.0, 0.0};
        const double ax = has ? gather_a(xv, false) : 0.0;
        if (row) {
            r_i = b_i - ax;
            u_i = dinv_i * r_i;
            __stcg(ubuf + i, u_i);
            acc[0] = r_i * r_i;
            acc[1] = b_i * b_i;
            acc[2] = r_i * u_i;
        }
        double tot[3];
        if (!sy.template sum<3>(acc, tot)) {
            status = CGP_ETIMEOUT;
            break;
        }
        if (outer == 0) bb = tot[1];
        rr_final = tot[0];
        if (!isfinite(tot[0])) {
            status = CGP_ENONFINITE;
            break;
        }
        if (tot[0] <= a.tol2 * bb) {
            converged = true;
            break;
        }
        if (outer >= a.max_outer || iters >= a.maxit) {
            status = CGP_ENOTCONV;
            break;
        }
        // ---- inner (Chronopoulos-Gear): w0 = A u, delta = <w0, u>
        double w_i = has ? gather_a(ubuf, false) : 0.0;
        double d1[1] = {row ? w_i * u_i : 0.0};
        if (row) __stcg(wbuf[0] + i, w_i);
        double t1[1];
        if (!sy.template sum<1>(d1, t1)) {
            status = CGP_ETIMEOUT;
            break;
        }
        double gamma = tot[2], delta = t1[0], gamma_prev = 0.0, alpha_prev = 0.0;
        double z_i = 0.0, q_i = 0.0, s_i = 0.0, p_i = 0.0;
        const double stop2 = 0.25 * a.tol2 * bb;
        double rr_best = INFINITY;
        int best_k = 0, cur = 0;
        bool fatal = false;
        for (int k = 0; iters < a.maxit; ++k) {
            double alpha, beta;
            if (k == 0) {
                beta = 0.0;
                alpha = gamma / delta;
            } else {
                beta = gamma / gamma_prev;
                alpha = gamma / (delta - beta * gamma / alpha_prev);
            }
            if (!isfinite(alpha) || alpha == 0.0) break;   // restart from the true residual
            double part[3] = {0.0, 0.0, 0.0};
            const double n_i = has ? gather_b(wbuf[cur]) : 0.0;
            if (row) {
                const double m_i = dinv_i * w_i;
                z_i = n_i + beta * z_i;
                q_i = m_i + beta * q_i;
                s_i = w_i + beta * s_i;
                p_i = u_i + beta * p_i;
                x_i += alpha * p_i;
                r_i -= alpha * s_i;
                u_i -= alpha * q_i;
                w_i -= alpha * z_i;
                __stcg(wbuf[cur ^ 1] + i, w_i);
                part[0] = r_i * u_i;
                part[1] = w_i * u_i;
                part[2] = r_i * r_i;
            }
            double t3[3];
            if (!sy.template sum<3>(part, t3)) {
                status = CGP_ETIMEOUT;
                break;
            }
            ++iters;
            cur ^= 1;
            if (!isfinite(t3[0]) || !isfinite(t3[1]) || !isfinite(t3[2])) {
                fatal = true;
                break;
            }
            gamma_prev = gamma;
            alpha_prev = alpha;
            gamma = t3[0];
            delta = t3[1];
            if (t3[2] <= stop2 || t3[0] == 0.0 || t3[2] == 0.0) break;
            if (t3[2] < 0.5 * rr_best) {
                rr_best = t3[2];
                best_k = k;
            } else if (k - best_k > kStagnation) {
                break;
            }
        }
        if (status) break;
        if (fatal) {
            status = CGP_ENONFINITE;
            break;
        }
        // x to memory for the next outer residual
        if (row) __stcg(xv + i, x_i);
        if (!sy.sync()) {
            status = CGP_ETIMEOUT;
            break;
        }
        ++outer;
    }
    // ---- pure-Neumann mean fix
    if (a.mlump && status != CGP_ETIMEOUT) {
        double acc[2] = {0.0, 0.0};
        if (row) {
            acc[0] = __ldg(a.mlump + i) * x_i;
            acc[1] = __ldg(a.mlump + i);
        }
        double tot[2];
        if (sy.template sum<2>(acc, tot)) {
            x_i -= tot[0] / tot[1];
        } else {
            status = CGP_ETIMEOUT;
        }
    }
    if (row) __stcg(xv + i, x_i);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
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
}

static __global__ void __launch_bounds__(kGridThreads) k_pcg_grid_rr(CoarsePcgArgs a) {
    __shared__ double wsum[kGridThreads / 32][4];
    GridSync sy(a.bar_count, a.bar_err, a.partials, wsum, a.wait_test);
    coarse_pcg_rr_body(a, sy);
}

}  // namespace cgp
