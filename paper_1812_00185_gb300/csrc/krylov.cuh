// Krylov kernels for the three kinds of linear systems of a CGP step:
//  - BiCGStab (Jacobi-preconditioned) for the nonsymmetric momentum matrix of Eq. 21,
//    two right-hand sides (u and v) sharing one matrix, each with its own recurrence;
//  - PCG (Jacobi) for the SPD systems: the coarse Poisson matrix of Eq. 23 and the mass
//    matrices of Eqs. 25-26, with one or two right-hand sides.
// Scalars (alpha, beta, ...) live in device memory (KrylovState) and are produced by
// the last block of each reduction, so no host round trip is needed per iteration.
// Every kernel returns at once when the solve has finished (state->done), which lets
// a loop be replayed a fixed number of times or inside a CUDA-graph WHILE node.
#pragma once

#include "internal.cuh"

namespace cgp {

struct KrylovState {
    double rz[2], pq[2], alpha[2], beta[2], omega[2], rho[2], rr[2], bb[2];
    double mean;           // rhs projection of pure-Neumann Poisson problems
    double tol2;           // (relative tolerance)^2
    int maxit, iter, done, status;
    int compdone[2];
    int pad[2];
};

// SELL-32 pattern of a level (see Level): one warp works on one slice of 32 rows,
// lane = row within the slice, so every load of the pattern and the values is coalesced.
struct SellView {
    int n, nslices;
    const int32_t* __restrict__ ptr;
    const int32_t* __restrict__ col;
};

inline SellView sell_of(const Level& L) { return SellView{L.nv, L.nslices, L.sell_ptr, L.sell_col}; }

// warp-uniform loop over the slices of A; inside: lane, row, base (first entry), w (width)
#define CGP_SLICE_LOOP(A, sl)                                                                  \
    for (int sl = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); sl < (A).nslices;        \
         sl += (int)((gridDim.x * blockDim.x) >> 5))

template <int NC>
__device__ __forceinline__ void ldv(const double* __restrict__ p, int i, double (&o)[NC]) {
    if constexpr (NC == 2) {
        double2 v = reinterpret_cast<const double2*>(p)[i];
        o[0] = v.x;
        o[1] = v.y;
    } else {
        o[0] = p[i];
    }
}

template <int NC>
__device__ __forceinline__ void stv(double* __restrict__ p, int i, const double (&o)[NC]) {
    if constexpr (NC == 2) {
        reinterpret_cast<double2*>(p)[i] = make_double2(o[0], o[1]);
    } else {
        p[i] = o[0];
    }
}


// acc[c] += sum_k val(row, k) * g(col(row, k))[c] over the row of (slice sl, lane).
// The pattern and value loads of up to 8 entries are issued together, then the 8
// gathers, so a row costs about three dependent memory round trips (slice offset,
// pattern/values, gathered vector) instead of two per entry.
template <int NC, class T, class Gather>
__device__ __forceinline__ void sell_accum(const SellView& A, const T* __restrict__ val, int sl, int lane, Gather&& g,
                                           double (&acc)[NC]) {
    const int base = __ldg(A.ptr + sl), w = (__ldg(A.ptr + sl + 1) - base) >> 5;
    for (int k0 = 0; k0 < w; k0 += 8) {
        int cj[8];
        double av[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            cj[u] = 0;
            av[u] = 0.0;
            if (k0 + u < w) {
                const int e = base + 32 * (k0 + u) + lane;
                cj[u] = __ldg(A.col + e);
                av[u] = (double)__ldg(val + e);
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (k0 + u < w) {
                double xv[NC];
                g(cj[u], xv);
#pragma unroll
                for (int c = 0; c < NC; ++c) acc[c] += av[u] * xv[c];
            }
        }
    }
}

__device__ __forceinline__ void set_loop_condition(unsigned long long handle, int keep_going) {
#if defined(__CUDA_ARCH__)
    if (handle) cudaGraphSetConditional((cudaGraphConditionalHandle)handle, keep_going ? 1u : 0u);
#endif
}

__device__ __forceinline__ bool finite(double x) { return isfinite(x); }

// ------------------------------------------------------------------ PCG
// init: r = b - A x (x = 0 if zero_x), optional rhs projection b -= mean,
// z = D^{-1} r, p = z; rz = <r,z>, rr = <r,r>, bb = <b,b>.
template <int NC>
__global__ void __launch_bounds__(kBlock) k_pcg_init(SellView A, const double* __restrict__ val,
                                                    const double* __restrict__ dinv, double* __restrict__ b,
                                                    double* __restrict__ x, double* __restrict__ r,
                                                    double* __restrict__ z, double* __restrict__ p,
                                                    KrylovState* st, double* partials, unsigned int* ticket,
                                                    int zero_x, int project, unsigned long long cond) {
    const double mean = project ? st->mean : 0.0;
    const int lane = threadIdx.x & 31;
    double acc[3 * NC];
#pragma unroll
    for (int k = 0; k < 3 * NC; ++k) acc[k] = 0.0;
    CGP_SLICE_LOOP(A, sl) {
        const int i = sl * 32 + lane;
        double ax[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) ax[c] = 0.0;
        if (!zero_x) sell_accum<NC>(A, val, sl, lane, [&](int j, double (&o)[NC]) { ldv<NC>(x, j, o); }, ax);
        if (i < A.n) {
            double bv[NC], rv[NC], zv[NC];
            ldv<NC>(b, i, bv);
            const double d = dinv[i];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                if (project) bv[c] -= mean;
                rv[c] = bv[c] - ax[c];
                zv[c] = d * rv[c];
                acc[c] += rv[c] * zv[c];
                acc[NC + c] += rv[c] * rv[c];
                acc[2 * NC + c] += bv[c] * bv[c];
            }
            if (project) stv<NC>(b, i, bv);
            if (zero_x) {
                double zero[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) zero[c] = 0.0;
                stv<NC>(x, i, zero);
            }
            stv<NC>(r, i, rv);
            stv<NC>(z, i, zv);
            stv<NC>(p, i, zv);
        }
    }
    double tot[3 * NC];
    if (grid_sum<3 * NC>(acc, partials, ticket, tot) && threadIdx.x == 0) {
        int all = 1;
        for (int c = 0; c < 2; ++c) {
            if (c < NC) {
                st->rz[c] = tot[c];
                st->rr[c] = tot[NC + c];
                st->bb[c] = tot[2 * NC + c];
                st->beta[c] = 0.0;
                st->alpha[c] = 0.0;
                st->compdone[c] = tot[NC + c] <= st->tol2 * tot[2 * NC + c];
            } else {
                st->compdone[c] = 1;
            }
            all &= st->compdone[c];
        }
        st->iter = 0;
        st->status = 0;
        for (int c = 0; c < NC; ++c)
            if (!finite(tot[c]) || !finite(tot[NC + c])) {
                st->status = CGP_ENONFINITE;
                all = 1;
            }
        st->done = all;
        set_loop_condition(cond, !all);
    }
}

// q = A p_new with p_new = z + beta p_old computed on the fly; pq = <p_new, q>.
template <int NC>
__global__ void __launch_bounds__(kBlock) k_pcg_spmv(SellView A, const double* __restrict__ val,
                                                    const double* __restrict__ z, const double* __restrict__ pold,
                                                    double* __restrict__ pnew, double* __restrict__ q,
                                                    KrylovState* st, double* partials, unsigned int* ticket) {
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    double beta[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) beta[c] = st->beta[c];
    double acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.0;
    CGP_SLICE_LOOP(A, sl) {
        const int i = sl * 32 + lane;
        double ax[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) ax[c] = 0.0;
        sell_accum<NC>(A, val, sl, lane,
                       [&](int j, double (&o)[NC]) {
                           double zv[NC], pv[NC];
                           ldv<NC>(z, j, zv);
                           ldv<NC>(pold, j, pv);
#pragma unroll
                           for (int c = 0; c < NC; ++c) o[c] = zv[c] + beta[c] * pv[c];
                       },
                       ax);
        if (i < A.n) {
            double zv[NC], pv[NC];
            ldv<NC>(z, i, zv);
            ldv<NC>(pold, i, pv);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                pv[c] = zv[c] + beta[c] * pv[c];
                acc[c] += pv[c] * ax[c];
            }
            stv<NC>(pnew, i, pv);
            stv<NC>(q, i, ax);
        }
    }
    double tot[NC];
    if (grid_sum<NC>(acc, partials, ticket, tot) && threadIdx.x == 0) {
        for (int c = 0; c < NC; ++c) {
            st->pq[c] = tot[c];
            if (st->compdone[c]) {
                st->alpha[c] = 0.0;
            } else if (tot[c] != 0.0 && finite(tot[c])) {
                st->alpha[c] = st->rz[c] / tot[c];
            } else {
                st->alpha[c] = 0.0;
                st->compdone[c] = 1;
                st->status = finite(tot[c]) ? CGP_EBREAKDOWN : CGP_ENONFINITE;
            }
        }
    }
}

// x += alpha p, r -= alpha q, z = D^{-1} r; rz = <r,z>, rr = <r,r>; convergence test.
template <int NC>
__global__ void __launch_bounds__(kBlock) k_pcg_update(int n, const double* __restrict__ dinv,
                                                      double* __restrict__ x, double* __restrict__ r,
                                                      double* __restrict__ z, const double* __restrict__ p,
                                                      const double* __restrict__ q, KrylovState* st,
                                                      double* partials, unsigned int* ticket,
                                                      unsigned long long cond) {
    if (st->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_loop_condition(cond, 0);
        return;
    }
    double alpha[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) alpha[c] = st->alpha[c];
    double acc[2 * NC];
#pragma unroll
    for (int k = 0; k < 2 * NC; ++k) acc[k] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double xv[NC], rv[NC], pv[NC], qv[NC], zv[NC];
        ldv<NC>(x, i, xv);
        ldv<NC>(r, i, rv);
        ldv<NC>(p, i, pv);
        ldv<NC>(q, i, qv);
        const double d = dinv[i];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            xv[c] += alpha[c] * pv[c];
            rv[c] -= alpha[c] * qv[c];
            zv[c] = d * rv[c];
            acc[c] += rv[c] * zv[c];
            acc[NC + c] += rv[c] * rv[c];
        }
        stv<NC>(x, i, xv);
        stv<NC>(r, i, rv);
        stv<NC>(z, i, zv);
    }
    double tot[2 * NC];
    if (grid_sum<2 * NC>(acc, partials, ticket, tot) && threadIdx.x == 0) {
        int all = 1;
        for (int c = 0; c < NC; ++c) {
            if (!st->compdone[c]) {
                if (!finite(tot[c]) || !finite(tot[NC + c])) {
                    st->status = CGP_ENONFINITE;
                    st->compdone[c] = 1;
                } else {
                    st->beta[c] = st->rz[c] != 0.0 ? tot[c] / st->rz[c] : 0.0;
                    st->rz[c] = tot[c];
                    st->rr[c] = tot[NC + c];
                    st->compdone[c] = tot[NC + c] <= st->tol2 * st->bb[c];
                }
            } else {
                st->beta[c] = 0.0;
            }
            all &= st->compdone[c];
        }
        st->iter += 1;
        if (!all && st->iter >= st->maxit) {
            if (!st->status) st->status = CGP_ENOTCONV;
            all = 1;
        }
        st->done = all;
        set_loop_condition(cond, !all);
    }
}

// ------------------------------------------------------------------ BiCGStab (2 rhs)
// Jacobi-preconditioned BiCGStab (van der Vorst's recurrences, right preconditioning):
//   p = r + beta (p - omega v);  y = D^{-1} p;  v = A y;  alpha = rho / <rhat, v>
//   s = r - alpha v;  z = D^{-1} s;  t = A z;  omega = <t, s> / <t, t>
//   x += alpha y + omega z;  r = s - omega t;  rho' = <rhat, r>;  beta = rho'/rho * alpha/omega
struct BicgVecs {
    double *x, *r, *rhat, *p, *v, *y, *s, *z, *t;   // 2 components interleaved
};

// two-component SELL SpMV of row (sl, lane): returns A u at that row
static __device__ __forceinline__ void spmv2_row(const SellView& A, const double* __restrict__ val,
                                          const double* __restrict__ u, int sl, int lane, double (&ax)[2]) {
    ax[0] = ax[1] = 0.0;
    sell_accum<2>(A, val, sl, lane, [&](int j, double (&o)[2]) { ldv<2>(u, j, o); }, ax);
}

static __global__ void __launch_bounds__(kBlock) k_bicg_init(SellView A, const double* __restrict__ val,
                                                     const double* __restrict__ b, BicgVecs V, KrylovState* st,
                                                     double* partials, unsigned int* ticket,
                                                     unsigned long long cond) {
    const int lane = threadIdx.x & 31;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    CGP_SLICE_LOOP(A, sl) {
        const int i = sl * 32 + lane;
        double ax[2];
        spmv2_row(A, val, V.x, sl, lane, ax);
        if (i < A.n) {
            double bv[2], rv[2];
            ldv<2>(b, i, bv);
            const double zero[2] = {0.0, 0.0};
            for (int c = 0; c < 2; ++c) {
                rv[c] = bv[c] - ax[c];
                acc[c] += rv[c] * rv[c];        // rho = <rhat, r> with rhat = r
                acc[2 + c] += rv[c] * rv[c];
                acc[4 + c] += bv[c] * bv[c];
            }
            stv<2>(V.r, i, rv);
            stv<2>(V.rhat, i, rv);
            stv<2>(V.p, i, zero);
            stv<2>(V.v, i, zero);
        }
    }
    double tot[6];
    if (grid_sum<6>(acc, partials, ticket, tot) && threadIdx.x == 0) {
        int all = 1;
        st->status = 0;
        for (int c = 0; c < 2; ++c) {
            st->rho[c] = tot[c];
            st->rr[c] = tot[2 + c];
            st->bb[c] = tot[4 + c];
            st->alpha[c] = 0.0;
            st->omega[c] = 0.0;
            st->beta[c] = 0.0;
            st->compdone[c] = tot[2 + c] <= st->tol2 * tot[4 + c];
            if (!finite(tot[2 + c]) || !finite(tot[4 + c])) {
                st->status = CGP_ENONFINITE;
                st->compdone[c] = 1;
            }
            all &= st->compdone[c];
        }
        st->iter = 0;
        st->done = all;
        set_loop_condition(cond, !all);
    }
}

// p = r + beta (p - omega v); y = D^{-1} p
static __global__ void __launch_bounds__(kBlock) k_bicg_p(int n, const double* __restrict__ dinv, BicgVecs V,
                                                  const KrylovState* st) {
    if (st->done) return;
    const double beta[2] = {st->beta[0], st->beta[1]}, omega[2] = {st->omega[0], st->omega[1]};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double rv[2], pv[2], vv[2], yv[2];
        ldv<2>(V.r, i, rv);
        ldv<2>(V.p, i, pv);
        ldv<2>(V.v, i, vv);
        const double d = dinv[i];
        for (int c = 0; c < 2; ++c) {
            pv[c] = rv[c] + beta[c] * (pv[c] - omega[c] * vv[c]);
            yv[c] = d * pv[c];
        }
        stv<2>(V.p, i, pv);
        stv<2>(V.y, i, yv);
    }
}

// v = A y; alpha = rho / <rhat, v>
static __global__ void __launch_bounds__(kBlock) k_bicg_v(SellView A, const double* __restrict__ val, BicgVecs V,
                                                  KrylovState* st, double* partials, unsigned int* ticket) {
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    double acc[2] = {0.0, 0.0};
    CGP_SLICE_LOOP(A, sl) {
        const int i = sl * 32 + lane;
        double ax[2];
        spmv2_row(A, val, V.y, sl, lane, ax);
        if (i < A.n) {
            double rh[2];
            ldv<2>(V.rhat, i, rh);
            acc[0] += rh[0] * ax[0];
            acc[1] += rh[1] * ax[1];
            stv<2>(V.v, i, ax);
        }
    }
    double tot[2];
    if (grid_sum<2>(acc, partials, ticket, tot) && threadIdx.x == 0) {
        for (int c = 0; c < 2; ++c) {
            if (st->compdone[c]) {
                st->alpha[c] = 0.0;
            } else if (tot[c] != 0.0 && finite(tot[c])) {
                st->alpha[c] = st->rho[c] / tot[c];
            } else {
                st->alpha[c] = 0.0;
                st->compdone[c] = 1;
                st->status = finite(tot[c]) ? CGP_EBREAKDOWN : CGP_ENONFINITE;
            }
        }
    }
}

// s = r - alpha v; z = D^{-1} s
static __global__ void __launch_bounds__(kBlock) k_bicg_s(int n, const double* __restrict__ dinv, BicgVecs V,
                                                  const KrylovState* st) {
    if (st->done) return;
    const double alpha[2] = {st->alpha[0], st->alpha[1]};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double rv[2], vv[2], sv[2], zv[2];
        ldv<2>(V.r, i, rv);
        ldv<2>(V.v, i, vv);
        const double d = dinv[i];
        for (int c = 0; c < 2; ++c) {
            sv[c] = rv[c] - alpha[c] * vv[c];
            zv[c] = d * sv[c];
        }
        stv<2>(V.s, i, sv);
        stv<2>(V.z, i, zv);
    }
}

// t = A z; omega = <t,s>/<t,t>
static __global__ void __launch_bounds__(kBlock) k_bicg_t(SellView A, const double* __restrict__ val, BicgVecs V,
                                                  KrylovState* st, double* partials, unsigned int* ticket) {
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    CGP_SLICE_LOOP(A, sl) {
        const int i = sl * 32 + lane;
        double ax[2];
        spmv2_row(A, val, V.z, sl, lane, ax);
        if (i < A.n) {
            double sv[2];
            ldv<2>(V.s, i, sv);
            for (int c = 0; c < 2; ++c) {
                acc[c] += ax[c] * sv[c];
                acc[2 + c] += ax[c] * ax[c];
            }
            stv<2>(V.t, i, ax);
        }
    }
    double tot[4];
    if (grid_sum<4>(acc, partials, ticket, tot) && threadIdx.x == 0) {
        for (int c = 0; c < 2; ++c) {
            if (st->compdone[c]) {
                st->omega[c] = 0.0;
            } else if (tot[2 + c] > 0.0 && finite(tot[2 + c])) {
                st->omega[c] = tot[c] / tot[2 + c];
            } else {
                st->omega[c] = 0.0;   // t = 0 means s = 0: x += alpha y finishes the solve
            }
        }
    }
}

// x += alpha y + omega z; r = s - omega t; rho' = <rhat, r>; beta; convergence test
static __global__ void __launch_bounds__(kBlock) k_bicg_x(int n, BicgVecs V, KrylovState* st, double* partials,
                                                  unsigned int* ticket, unsigned long long cond) {
    if (st->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_loop_condition(cond, 0);
        return;
    }
    const double alpha[2] = {st->alpha[0], st->alpha[1]}, omega[2] = {st->omega[0], st->omega[1]};
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double xv[2], yv[2], zv[2], sv[2], tv[2], rh[2], rv[2];
        ldv<2>(V.x, i, xv);
        ldv<2>(V.y, i, yv);
        ldv<2>(V.z, i, zv);
        ldv<2>(V.s, i, sv);
        ldv<2>(V.t, i, tv);
        ldv<2>(V.rhat, i, rh);
        for (int c = 0; c < 2; ++c) {
            xv[c] += alpha[c] * yv[c] + omega[c] * zv[c];
            rv[c] = sv[c] - omega[c] * tv[c];
            acc[c] += rh[c] * rv[c];
            acc[2 + c] += rv[c] * rv[c];
        }
        stv<2>(V.x, i, xv);
        stv<2>(V.r, i, rv);
    }
    double tot[4];
    if (grid_sum<4>(acc, partials, ticket, tot) && threadIdx.x == 0) {
        int all = 1;
        for (int c = 0; c < 2; ++c) {
            if (!st->compdone[c]) {
                if (!finite(tot[c]) || !finite(tot[2 + c])) {
                    st->status = CGP_ENONFINITE;
                    st->compdone[c] = 1;
                } else {
                    st->rr[c] = tot[2 + c];
                    if (tot[2 + c] <= st->tol2 * st->bb[c]) {
                        st->compdone[c] = 1;
                    } else if (st->omega[c] == 0.0 || st->rho[c] == 0.0) {
                        st->compdone[c] = 1;
                        st->status = CGP_EBREAKDOWN;
                    } else {
                        st->beta[c] = (tot[c] / st->rho[c]) * (st->alpha[c] / st->omega[c]);
                        st->rho[c] = tot[c];
                    }
                }
            }
            if (st->compdone[c]) st->beta[c] = 0.0;
            all &= st->compdone[c];
        }
        st->iter += 1;
        if (!all && st->iter >= st->maxit) {
            if (!st->status) st->status = CGP_ENOTCONV;
            all = 1;
        }
        st->done = all;
        set_loop_condition(cond, !all);
    }
}

}  // namespace cgp
