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
// in its last block, solves the small system with a truncated pseudo-inverse of G in FP64 on
// one thread (see proj_solve_small); one kernel forms x0 = X c; after the solve, one kernel stores the new
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

// c = G^+ f over the first m slots (one thread): G (symmetrised) = V diag(lambda) V^T by
// cyclic Jacobi rotations, then c = sum over lambda_i > thr of v_i (v_i^T f) / lambda_i.  The
// stored G equals X^T K X only to the solve's tolerance (b_j = K x_j + r_j), and consecutive
// increments are nearly dependent, so directions with lambda_i <= thr = max(tol, 1e-12)
// lambda_max are noise and are dropped (a truncated pseudo-inverse, not a shifted solve).
__device__ inline void proj_solve_small(ProjState* ps, const double* f, int m, double tol) {
    double a[kProjL][kProjL], v[kProjL][kProjL];
    for (int i = 0; i < kProjL; ++i)
        for (int j = 0; j < kProjL; ++j) {
            a[i][j] = (i < m && j < m) ? 0.5 * (ps->G[i][j] + ps->G[j][i]) : 0.0;
            v[i][j] = i == j ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 12; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int i = 0; i < m; ++i) {
            dia += a[i][i] * a[i][i];
            for (int j = i + 1; j < m; ++j) off += a[i][j] * a[i][j];
        }
        if (!(off > 1e-30 * dia)) break;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                if (a[p][q] == 0.0) continue;
                // rotation that zeroes a[p][q] (the smaller root of t^2 + 2 theta t - 1 = 0)
                const double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < m; ++k) {
                    const double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - s * akq;
                    a[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < m; ++k) {
                    const double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - s * aqk;
                    a[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < m; ++k) {
                    const double vkp = v[k][p], vkq = v[k][q];
                    v[k][p] = c * vkp - s * vkq;
                    v[k][q] = s * vkp + c * vkq;
                }
            }
    }
    double lmax = 0.0;
    for (int i = 0; i < m; ++i) lmax = fmax(lmax, a[i][i]);
    const double thr = fmax(tol, 1e-12) * lmax;
    double c[kProjL];
    for (int i = 0; i < kProjL; ++i) c[i] = 0.0;
    for (int e = 0; e < m; ++e) {
        if (!(a[e][e] > thr)) continue;
        double w = 0.0;
        for (int i = 0; i < m; ++i) w += v[i][e] * f[i];
        w /= a[e][e];
        for (int i = 0; i < m; ++i) c[i] += v[i][e] * w;
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
static __global__ void __launch_bounds__(kBlock) k_proj_combine(int n, const double* __restrict__ hx,
                                                                const ProjState* ps, double* x, double* xq) {
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
