// Krylov kernels for the three kinds of linear systems of a CGP step:
//  - BiCGStab (Jacobi-preconditioned) for the nonsymmetric momentum matrix of Eq. 21,
//    two right-hand sides (u and v) sharing one matrix, each with its own recurrence;
//  - PCG (Jacobi) for the SPD systems: the coarse Poisson matrix of Eq. 23 and the mass
//    matrices of Eqs. 25-26, with one or two right-hand sides.
// Scalars (alpha, beta, ...) live in device memory (KrylovState) and are produced by
// the last block of each reduction, so no host round trip is needed per iteration.
// Every kernel returns at once when the solve has finished (state->done), which lets
// a loop be replayed a fixed number of times or inside a CUDA-graph WHILE node.
// The kernels take the working type T of vectors, matrix values and per-row arithmetic:
// double for the FP64 solves, float for the inner solves of the mixed form (whose
// block partial sums are still added in FP64).
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
    int inner, trips;      // mixed form: FP32 inner iterations and inner loop trips of the solve
    int skip;              // inner solves: set when the outer residual already meets the tolerance
    int ir_done;           // outer solves of the mixed form: the last refinement residual met the
                           // tolerance (the FP64 loop that follows then reports done at its init)
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

template <class T> struct Vec2T;
template <> struct Vec2T<double> { using type = double2; };
template <> struct Vec2T<float> { using type = float2; };

template <int NC, class T>
__device__ __forceinline__ void ldv(const T* __restrict__ p, int i, T (&o)[NC]) {
    if constexpr (NC == 2) {
        const auto v = reinterpret_cast<const typename Vec2T<T>::type*>(p)[i];
        o[0] = v.x;
        o[1] = v.y;
    } else {
        o[0] = p[i];
    }
}

template <int NC, class T>
__device__ __forceinline__ void stv(T* __restrict__ p, int i, const T (&o)[NC]) {
    if constexpr (NC == 2) {
        typename Vec2T<T>::type v;
        v.x = o[0];
        v.y = o[1];
        reinterpret_cast<typename Vec2T<T>::type*>(p)[i] = v;
    } else {
        p[i] = o[0];
    }
}

// acc[c] += sum_k val(row, k) * g(col(row, k))[c] over the row of (slice sl, lane).
// The pattern and value loads of up to 8 entries are issued together, then the 8
// gathers, so a row costs about three dependent memory round trips (slice offset,
// pattern/values, gathered vector) instead of two per entry.
template <int NC, class V, class Acc, class Gather>
__device__ __forceinline__ void sell_accum(const SellView& A, const V* __restrict__ val, int sl, int lane, Gather&& g,
                                           Acc (&acc)[NC]) {
    const int base = __ldg(A.ptr + sl), w = (__ldg(A.ptr + sl + 1) - base) >> 5;
    for (int k0 = 0; k0 < w; k0 += 8) {
        int cj[8];
        Acc av[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            cj[u] = 0;
            av[u] = Acc(0);
            if (k0 + u < w) {
                const int e = base + 32 * (k0 + u) + lane;
                cj[u] = __ldg(A.col + e);
                av[u] = (Acc)__ldg(val + e);
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (k0 + u < w) {
                Acc xv[NC];
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
// z = D^{-1} r, p = z; rz = <r,z>, rr = <r,r>, bb = <b,b>.  An inner solve whose `skip`
// is set (the outer residual already converged) reports done at once.
template <int NC, class T = double>
__global__ void __launch_bounds__(kBlock) k_pcg_init(SellView A, const T* __restrict__ val,
                                                    const T* __restrict__ dinv, T* __restrict__ b,
                                                    T* __restrict__ x, T* __restrict__ r,
                                                    T* __restrict__ z, T* __restrict__ p,
                                                    KrylovState* st, double* partials, unsigned int* ticket,
                                                    int zero_x, int project, unsigned long long cond) {
    if (st->skip) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->iter = 0;
            st->status = 0;
            st->done = 1;
            set_loop_condition(cond, 0);
        }
        return;
    }
    const T mean = project ? (T)st->mean : T(0);
    const int lane = threadIdx.x & 31;
    T acc[3 * NC];
#pragma unroll
    for (int k = 0; k < 3 * NC; ++k) acc[k] = T(0);
    CGP_SLICE_LOOP(A, sl) {
        const int i = sl * 32 + lane;
        T ax[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) ax[c] = T(0);
        if (!zero_x) sell_accum<NC>(A, val, sl, lane, [&](int j, T (&o)[NC]) { ldv<NC>(x, j, o); }, ax);
        if (i < A.n) {
            T bv[NC], rv[NC], zv[NC];
            ldv<NC>(b, i, bv);
            const T d = dinv[i];
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
                T zero[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) zero[c] = T(0);
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
template <int NC, class T = double>
__global__ void __launch_bounds__(kBlock) k_pcg_spmv(SellView A, const T* __restrict__ val,
                                                    const T* __restrict__ z, const T* __restrict__ pold,
                                                    T* __restrict__ pnew, T* __restrict__ q,
                                                    KrylovState* st, double* partials, unsigned int* ticket) {
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    T beta[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) beta[c] = (T)st->beta[c];
    T acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = T(0);
    CGP_SLICE_LOOP(A, sl) {
        const int i = sl * 32 + lane;
        T ax[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) ax[c] = T(0);
        sell_accum<NC>(A, val, sl, lane,
                       [&](int j, T (&o)[NC]) {
                           T zv[NC], pv[NC];
                           ldv<NC>(z, j, zv);
                           ldv<NC>(pold, j, pv);
#pragma unroll
                           for (int c = 0; c < NC; ++c) o[c] = zv[c] + beta[c] * pv[c];
                       },
                       ax);
        if (i < A.n) {
            T zv[NC], pv[NC];
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

// Three-kernel form (the FP64 solves): p = z + beta p in place, then q = A p gathers p
// alone.  The stored p_j is the value the fused form recomputes for every neighbour, so the
// iterates are the same; the SpMV does one FMA per entry instead of two, which matters on a
// GPU with few FP64 units.
template <int NC, class T = double>
__global__ void __launch_bounds__(kBlock) k_pcg_pupd(int n, const T* __restrict__ z, T* __restrict__ p,
                                                    const KrylovState* st) {
    if (st->done) return;
    T beta[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) beta[c] = (T)st->beta[c];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T zv[NC], pv[NC];
        ldv<NC>(z, i, zv);
        ldv<NC>(p, i, pv);
#pragma unroll
        for (int c = 0; c < NC; ++c) pv[c] = zv[c] + beta[c] * pv[c];
        stv<NC>(p, i, pv);
    }
}

// q = A p; pq = <p, q> -> alpha (three-kernel form)
template <int NC, class T = double>
__global__ void __launch_bounds__(kBlock) k_pcg_spmv3(SellView A, const T* __restrict__ val, const T* __restrict__ p,
                                                     T* __restrict__ q, KrylovState* st, double* partials,
                                                     unsigned int* ticket) {
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    T acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = T(0);
    CGP_SLICE_LOOP(A, sl) {
        const int i = sl * 32 + lane;
        T ax[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) ax[c] = T(0);
        sell_accum<NC>(A, val, sl, lane, [&](int j, T (&o)[NC]) { ldv<NC>(p, j, o); }, ax);
        if (i < A.n) {
            T pv[NC];
            ldv<NC>(p, i, pv);
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] += pv[c] * ax[c];
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
template <int NC, class T = double>
__global__ void __launch_bounds__(kBlock) k_pcg_update(int n, const T* __restrict__ dinv,
                                                      T* __restrict__ x, T* __restrict__ r,
                                                      T* __restrict__ z, const T* __restrict__ p,
                                                      const T* __restrict__ q, KrylovState* st,
                                                      double* partials, unsigned int* ticket,
                                                      unsigned long long cond) {
    if (st->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_loop_condition(cond, 0);
        return;
    }
    T alpha[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) alpha[c] = (T)st->alpha[c];
    T acc[2 * NC];
#pragma unroll
    for (int k = 0; k < 2 * NC; ++k) acc[k] = T(0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T xv[NC], rv[NC], pv[NC], qv[NC], zv[NC];
        ldv<NC>(x, i, xv);
        ldv<NC>(r, i, rv);
        ldv<NC>(p, i, pv);
        ldv<NC>(q, i, qv);
        const T d = dinv[i];
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
template <class T>
struct BicgVecsT {
    T *x, *r, *rhat, *p, *v, *y, *s, *z, *t;   // 2 components interleaved
};
using BicgVecs = BicgVecsT<double>;

// two-component SELL SpMV of row (sl, lane): returns A u at that row
template <class T>
static __device__ __forceinline__ void spmv2_row(const SellView& A, const T* __restrict__ val,
                                                 const T* __restrict__ u, int sl, int lane, T (&ax)[2]) {
    ax[0] = ax[1] = T(0);
    sell_accum<2>(A, val, sl, lane, [&](int j, T (&o)[2]) { ldv<2>(u, j, o); }, ax);
}

// scalar steps of BiCGStab (one thread, after a grid sum), per right-hand side:
// alpha = rho / <rhat, v>
__device__ __forceinline__ void bicg_alpha(KrylovState* st, const double (&tot)[2]) {
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
// omega = <t, s> / <t, t>
__device__ __forceinline__ void bicg_omega(KrylovState* st, const double (&tot)[4]) {
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
// from <rhat, r> and <r, r> of the new residual: convergence test, beta, rho, loop control
__device__ __forceinline__ void bicg_finish(KrylovState* st, const double (&tot)[4], unsigned long long cond) {
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

// init: r = b - A x (x = 0 if zero_x), rhat = r, p = v = 0; rho, rr, bb.  An inner solve
// whose `skip` is set reports done at once.
template <class T>
static __global__ void __launch_bounds__(kBlock) k_bicg_init(SellView A, const T* __restrict__ val,
                                                     const T* __restrict__ b, BicgVecsT<T> V, KrylovState* st,
                                                     double* partials, unsigned int* ticket,
                                                     unsigned long long cond, int zero_x = 0) {
    if (st->skip) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->iter = 0;
            st->status = 0;
            st->done = 1;
            set_loop_condition(cond, 0);
        }
        return;
    }
    const int lane = threadIdx.x & 31;
    T acc[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    CGP_SLICE_LOOP(A, sl) {
        const int i = sl * 32 + lane;
        T ax[2] = {T(0), T(0)};
        if (!zero_x) spmv2_row(A, val, V.x, sl, lane, ax);
        if (i < A.n) {
            T bv[2], rv[2];
            ldv<2>(b, i, bv);
            const T zero[2] = {T(0), T(0)};
            for (int c = 0; c < 2; ++c) {
                rv[c] = bv[c] - ax[c];
                acc[c] += rv[c] * rv[c];        // rho = <rhat, r> with rhat = r
                acc[2 + c] += rv[c] * rv[c];
                acc[4 + c] += bv[c] * bv[c];
            }
            if (zero_x) stv<2>(V.x, i, zero);
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
template <class T>
static __global__ void __launch_bounds__(kBlock) k_bicg_p(int n, const T* __restrict__ dinv, BicgVecsT<T> V,
                                                  const KrylovState* st) {
    if (st->done) return;
    const T beta[2] = {(T)st->beta[0], (T)st->beta[1]}, omega[2] = {(T)st->omega[0], (T)st->omega[1]};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T rv[2], pv[2], vv[2], yv[2];
        ldv<2>(V.r, i, rv);
        ldv<2>(V.p, i, pv);
        ldv<2>(V.v, i, vv);
        const T d = dinv[i];
        for (int c = 0; c < 2; ++c) {
            pv[c] = rv[c] + beta[c] * (pv[c] - omega[c] * vv[c]);
            yv[c] = d * pv[c];
        }
        stv<2>(V.p, i, pv);
        stv<2>(V.y, i, yv);
    }
}

// v = A y; alpha = rho / <rhat, v>
template <class T>
static __global__ void __launch_bounds__(kBlock) k_bicg_v(SellView A, const T* __restrict__ val, BicgVecsT<T> V,
                                                  KrylovState* st, double* partials, unsigned int* ticket) {
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    T acc[2] = {T(0), T(0)};
    CGP_SLICE_LOOP(A, sl) {
        const int i = sl * 32 + lane;
        T ax[2];
        spmv2_row(A, val, V.y, sl, lane, ax);
        if (i < A.n) {
            T rh[2];
            ldv<2>(V.rhat, i, rh);
            acc[0] += rh[0] * ax[0];
            acc[1] += rh[1] * ax[1];
            stv<2>(V.v, i, ax);
        }
    }
    double tot[2];
    if (grid_sum<2>(acc, partials, ticket, tot) && threadIdx.x == 0) bicg_alpha(st, tot);
}

// s = r - alpha v; z = D^{-1} s
template <class T>
static __global__ void __launch_bounds__(kBlock) k_bicg_s(int n, const T* __restrict__ dinv, BicgVecsT<T> V,
                                                  const KrylovState* st) {
    if (st->done) return;
    const T alpha[2] = {(T)st->alpha[0], (T)st->alpha[1]};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T rv[2], vv[2], sv[2], zv[2];
        ldv<2>(V.r, i, rv);
        ldv<2>(V.v, i, vv);
        const T d = dinv[i];
        for (int c = 0; c < 2; ++c) {
            sv[c] = rv[c] - alpha[c] * vv[c];
            zv[c] = d * sv[c];
        }
        stv<2>(V.s, i, sv);
        stv<2>(V.z, i, zv);
    }
}

// t = A z; omega = <t,s>/<t,t>
template <class T>
static __global__ void __launch_bounds__(kBlock) k_bicg_t(SellView A, const T* __restrict__ val, BicgVecsT<T> V,
                                                  KrylovState* st, double* partials, unsigned int* ticket) {
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    CGP_SLICE_LOOP(A, sl) {
        const int i = sl * 32 + lane;
        T ax[2];
        spmv2_row(A, val, V.z, sl, lane, ax);
        if (i < A.n) {
            T sv[2];
            ldv<2>(V.s, i, sv);
            for (int c = 0; c < 2; ++c) {
                acc[c] += ax[c] * sv[c];
                acc[2 + c] += ax[c] * ax[c];
            }
            stv<2>(V.t, i, ax);
        }
    }
    double tot[4];
    if (grid_sum<4>(acc, partials, ticket, tot) && threadIdx.x == 0) bicg_omega(st, tot);
}

// x += alpha y + omega z; r = s - omega t; rho' = <rhat, r>; beta; convergence test
template <class T>
static __global__ void __launch_bounds__(kBlock) k_bicg_x(int n, BicgVecsT<T> V, KrylovState* st, double* partials,
                                                  unsigned int* ticket, unsigned long long cond) {
    if (st->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_loop_condition(cond, 0);
        return;
    }
    const T alpha[2] = {(T)st->alpha[0], (T)st->alpha[1]}, omega[2] = {(T)st->omega[0], (T)st->omega[1]};
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T xv[2], yv[2], zv[2], sv[2], tv[2], rh[2], rv[2];
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
    if (grid_sum<4>(acc, partials, ticket, tot) && threadIdx.x == 0) bicg_finish(st, tot, cond);
}

}  // namespace cgp
