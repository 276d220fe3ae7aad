// Initial guess of the coarse Poisson solve (Eq. 23) from the solutions of earlier steps: a
// form beyond the paper.
//
// Successive time steps solve K_c Phi = b with right-hand sides that change smoothly, so the
// new increment lies close to the span of the last few.  CGP_GUESS_PROJ starts the solve from
// the Galerkin projection onto that span (Fischer, "Projection techniques for iterative
// solution of Ax = b with successive right-hand sides", CMAME 163, 1998): with X = [x_1..x_m]
// the last m <= kProjL solutions, x0 = X c where (X^T K X) c = X^T b, which minimises the
// K-norm of the error over the span.  K x_j is not formed: each solve leaves b_j = K x_j up to
// its tolerance, so G = X^T K X is kept as G_ij = (x_i^T b_j + x_j^T b_i) / 2 from the stored
// pairs, one new row per step.  The window slides (the oldest pair is replaced).
//
// Per step: one kernel forms f = X^T b (and stores b in the slot the new pair will take) and,
// in its last block, solves the small system by a pivoted, truncated Cholesky factorisation
// in FP64 on one thread (see proj_solve_small); one kernel forms x0 = X c; after the solve, one kernel stores the new
// solution and adds its row of G.  CGP_GUESS_LEARNED uses the same x0 as the network's
// second input and as the first of the two guesses the one-launch solve combines.
#pragma once

#include "internal.cuh"
#include "krylov.cuh"

namespace cgp {

constexpr int kProjL = 8;   // solutions kept (the window)

struct ProjState {
    double G[kProjL][kProjL];   // x_i^T K x_j of the stored pairs (slot order)
    double c[kProjL];           // coefficients of the current guess
    int count;                  // valid slots (0 .. kProjL)
    int head;                   // slot the next solution takes
    int pad[2];
};

// c = a truncated solution of G c = f over the first m slots (one thread), by a Cholesky
// factorisation with diagonal pivoting: each step takes the slot whose Schur-complement
// diagonal is largest and stops once that is <= thr = max(tol, 1e-12) * max_i G_ii.  The
// stored G equals X^T K X only to the solve's tolerance (b_j = K x_j + r_j), and consecutive
// increments are nearly dependent, so the slots left out are those the kept ones already
// span to within that noise (a rank-revealing truncation); their coefficients are 0.  About
// m^3 / 3 operations on registers and local arrays of 8 x 8.
__device__ inline void proj_solve_small(ProjState* ps, const double* f, int m, double tol) {
    double g[kProjL][kProjL], L[kProjL][kProjL], y[kProjL], c[kProjL], d[kProjL];
    int piv[kProjL], used[kProjL];
    double dmax = 0.0;
    for (int i = 0; i < kProjL; ++i) {
        for (int j = 0; j < kProjL; ++j) {
            g[i][j] = (i < m && j < m) ? 0.5 * (ps->G[i][j] + ps->G[j][i]) : 0.0;
            L[i][j] = 0.0;
        }
        used[i] = i >= m;
        c[i] = 0.0;
        d[i] = g[i][i];   // Schur-complement diagonal, updated as columns are taken
        if (i < m) dmax = fmax(dmax, g[i][i]);
    }
    const double thr = fmax(tol, 1e-12) * dmax;
    int r = 0;
    for (int k = 0; k < m; ++k) {
        int best = -1;
        double bd = thr;
        for (int i = 0; i < m; ++i) {
            if (!used[i] && d[i] > bd) {
                bd = d[i];
                best = i;
            }
        }
        if (best < 0) break;
        used[best] = 1;
        piv[k] = best;
        const double lkk = sqrt(bd);
        L[best][k] = lkk;
        for (int i = 0; i < m; ++i) {
            if (used[i]) continue;
            double s = g[i][best];
            for (int p = 0; p < k; ++p) s -= L[i][p] * L[best][p];
            L[i][k] = s / lkk;
            d[i] -= L[i][k] * L[i][k];
        }
        r = k + 1;
    }
    // (L L^T) restricted to the pivots: forward then back substitution
    for (int k = 0; k < r; ++k) {
        double s = f[piv[k]];
        for (int p = 0; p < k; ++p) s -= L[piv[k]][p] * y[p];
        y[k] = s / L[piv[k]][k];
    }
    for (int k = r - 1; k >= 0; --k) {
        double s = y[k];
        for (int p = k + 1; p < r; ++p) s -= L[piv[p]][k] * c[piv[p]];
        c[piv[k]] = s / L[piv[k]][k];
    }
    for (int i = 0; i < kProjL; ++i) ps->c[i] = isfinite(c[i]) ? c[i] : 0.0;
}

// f_j = x_j^T b for the stored x_j (b as the solve will see it: range-projected by the mean
// in ks when the problem is pure Neumann); b is also stored in the slot the new pair takes.
static __global__ void __launch_bounds__(kBlock) k_proj_coef(int n, const double* __restrict__ hx, double* hb,
                                                             const double* __restrict__ b, const KrylovState* ks,
                                                             ProjState* ps, double tol, double* partials,
                                                             unsigned int* ticket) {
    const int m = ps->count, head = ps->head;
    const double mean = ks->mean;
    double v[kProjL];
#pragma unroll
    for (int j = 0; j < kProjL; ++j) v[j] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double bi = b[i] - mean;
        hb[(size_t)head * n + i] = bi;
#pragma unroll
        for (int j = 0; j < kProjL; ++j)
            if (j < m) v[j] = fma(__ldg(hx + (size_t)j * n + i), bi, v[j]);
    }
    double tot[kProjL];
    if (grid_sum<kProjL>(v, partials, ticket, tot) && threadIdx.x == 0) proj_solve_small(ps, tot, m, tol);
}

// x0 = X c (x keeps the previous increment while no solution is stored); xq, if given,
// receives a copy (the input the network saw, for recording training pairs).
// With `cond` (a graph's conditional handle, 0 otherwise) it also sets the IF condition of the
// learned network that follows: run unless the coarse solve's judge has it off (gate[0] > 0).
static __global__ void __launch_bounds__(kBlock) k_proj_combine(int n, const double* __restrict__ hx,
                                                                const ProjState* ps, double* x, double* xq,
                                                                const int* gate = nullptr,
                                                                unsigned long long cond = 0) {
    if (cond && blockIdx.x == 0 && threadIdx.x == 0)
        cudaGraphSetConditional((cudaGraphConditionalHandle)cond, __ldcg(gate) > 0 ? 0u : 1u);
    const int m = ps->count;
    double c[kProjL];
#pragma unroll
    for (int j = 0; j < kProjL; ++j) c[j] = ps->c[j];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = m ? 0.0 : x[i];
#pragma unroll
        for (int j = 0; j < kProjL; ++j)
            if (j < m) s = fma(c[j], __ldg(hx + (size_t)j * n + i), s);
        x[i] = s;
        if (xq) xq[i] = s;
    }
}

// After the solve: the new solution x goes to slot `head` (its b is there already), and row
// `head` of G is formed: G[head][j] = (x^T b_j + x_j^T b) / 2 over the other valid slots,
// G[head][head] = x^T b.
static __global__ void __launch_bounds__(kBlock) k_proj_push(int n, const double* __restrict__ x, double* hx,
                                                             const double* __restrict__ hb, ProjState* ps,
                                                             double* partials, unsigned int* ticket) {
    const int m = ps->count, head = ps->head;
    double v[kProjL];
#pragma unroll
    for (int j = 0; j < kProjL; ++j) v[j] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double xi = x[i], bi = hb[(size_t)head * n + i];
#pragma unroll
        for (int j = 0; j < kProjL; ++j) {
            if (j == head) {
                v[j] = fma(xi, bi, v[j]);
            } else if (j < m) {
                v[j] = fma(xi, hb[(size_t)j * n + i], v[j]);
                v[j] = fma(hx[(size_t)j * n + i], bi, v[j]);
            }
        }
        hx[(size_t)head * n + i] = xi;
    }
    double tot[kProjL];
    if (grid_sum<kProjL>(v, partials, ticket, tot) && threadIdx.x == 0) {
        for (int j = 0; j < kProjL; ++j) {
            if (j == head) {
                ps->G[head][head] = tot[j];
            } else if (j < m) {
                ps->G[head][j] = 0.5 * tot[j];
                ps->G[j][head] = 0.5 * tot[j];
            }
        }
        ps->count = m < kProjL ? m + 1 : kProjL;
        ps->head = (head + 1) % kProjL;
    }
}

}  // namespace cgp
