// One CGP time step on the device (paper Section 2.2, Eqs. 21-26) and its host
// orchestration: eager launches with host-polled loop control, or a CUDA graph whose
// Krylov loops are conditional WHILE nodes driven by the kernels themselves.
#include <algorithm>
#include <cstring>

#include "coarse_pcg.cuh"
#include "coarse_rr.cuh"
#include "coarse_onchip.cuh"
#include "flows.cuh"
#include "guess_proj.cuh"
#include "solver.cuh"
#include "step_rows.cuh"
#include "batch_step.cuh"

namespace cgp {


// problem data of the solver's kind, with the caller's arrays for CGP_BC_USER
static BcParams bc_of(const Solver& s) {
    BcParams b = bc_from(s.prm);
    b.ud = s.user_ud;
    b.fu = s.user_f;
    return b;
}

// ---------------------------------------------------------------- per-vertex kernels
__global__ void k_init_state(int nf, const double* __restrict__ xy, const uint8_t* __restrict__ tag, BcParams bc,
                             double dt, double* __restrict__ U, double* __restrict__ Uprev, double* __restrict__ P,
                             double* __restrict__ tdev) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *tdev = 0.0;
    if (i >= nf) return;
    const double x = xy[2 * i], y = xy[2 * i + 1];
    double u, v, p;
    if (exact_field(bc, x, y, 0.0, u, v, p)) {
        U[2 * i] = u;
        U[2 * i + 1] = v;
        P[i] = p;
        exact_field(bc, x, y, -dt, u, v, p);
        Uprev[2 * i] = u;
        Uprev[2 * i + 1] = v;
        return;
    }
    u = v = 0.0;
    if (tag[i] & CGP_VEL_DIR) dirichlet_value(bc, i, x, y, 0.0, u, v);
    U[2 * i] = Uprev[2 * i] = u;
    U[2 * i + 1] = Uprev[2 * i + 1] = v;
    P[i] = 0.0;
}

// w = 2 U^n - U^{n-1} (Eq. 5's extrapolated advecting field), h = dt F^{n+1} + 2 U^n - 1/2 U^{n-1}
__global__ void k_mom_prep(int nf, const double* __restrict__ U, const double* __restrict__ Uprev,
                           const double* __restrict__ xy, BcParams bc, const double* __restrict__ tdev, double dt,
                           double* __restrict__ w, double* __restrict__ h) {
    const double tn = *tdev + dt;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
        double2 u = reinterpret_cast<const double2*>(U)[i];
        double2 up = reinterpret_cast<const double2*>(Uprev)[i];
        double fx = 0.0, fy = 0.0;
        if (bc.kind == CGP_BC_TG_PERIODIC || bc.kind == CGP_BC_USER || bc.kind == CGP_BC_JOBELIN_OPEN ||
            bc.kind == CGP_BC_JOBELIN_DISK)
            body_force(bc, i, xy[2 * i], xy[2 * i + 1], tn, fx, fy);
        reinterpret_cast<double2*>(w)[i] = make_double2(2.0 * u.x - up.x, 2.0 * u.y - up.y);
        reinterpret_cast<double2*>(h)[i] =
            make_double2(dt * fx + (2.0 * u.x - 0.5 * up.x), dt * fy + (2.0 * u.y - 0.5 * up.y));
    }
}

// Eq. 21's matrix and right-hand side, one thread per row (step_rows.cuh)
__global__ void __launch_bounds__(kBlock) k_mom_assemble(int nf, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const int32_t* __restrict__ sell_ptr, const int32_t* __restrict__ vt_ptr, const int32_t* __restrict__ vt_list,
                               const int32_t* __restrict__ tri, const double* __restrict__ geo,
                               const int32_t* __restrict__ vtslot, const double* __restrict__ S,
                               const double* __restrict__ M, const double* __restrict__ CxT,
                               const double* __restrict__ CyT, const double* __restrict__ P,
                               const double* __restrict__ w, const double* __restrict__ h,
                               const uint8_t* __restrict__ tag, const double* __restrict__ xy, BcParams bc,
                               const double* __restrict__ tdev, double dt, double* __restrict__ A,
                               double* __restrict__ dinv, double* __restrict__ b, double* __restrict__ x0) {
    __shared__ double arow[kAsmRow][kBlock];
    const double tn = *tdev + dt;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x)
        mom_assemble_row<true>(i, rowptr, col, sell_ptr, vt_ptr, vt_list, tri, geo, vtslot, S, M, CxT, CyT, P, w, h,
                               tag, xy, bc, tn, dt, A, dinv, b, x0, arow);
}

// Eqs. 22-23: r_i = -3/(2 dt) (Cx_c u~ + Cy_c v~)_i at coarse vertex i (the injected
// U~ is the first N_c entries of the fine U~); r = 0 where phi = 0; mean for the projection.
__global__ void __launch_bounds__(kBlock) k_coarse_rhs(SellView Ac, const double* __restrict__ Cxc,
                                                      const double* __restrict__ Cyc, const double* __restrict__ Ut,
                                                      const uint8_t* __restrict__ tag, double dt,
                                                      double* __restrict__ rc, KrylovState* st, int pure_neumann,
                                                      double* partials, unsigned int* ticket) {
    const int lane = threadIdx.x & 31;
    const double2* __restrict__ U2 = reinterpret_cast<const double2*>(Ut);
    double acc[1] = {0.0};
    CGP_SLICE_LOOP(Ac, sl) {
        const int i = sl * 32 + lane;
        // Cx and Cy share the coarse pattern: one pass reads each column index once and
        // gathers (u~, v~) of a column as one 16-byte load; each of the two sums keeps the
        // entry order of a row
        const int base = __ldg(Ac.ptr + sl), w = (__ldg(Ac.ptr + sl + 1) - base) >> 5;
        double sx = 0.0, sy = 0.0;
        for (int k0 = 0; k0 < w; k0 += 8) {
            int cj[8];
            double ax[8], ay[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                cj[u] = 0;
                ax[u] = ay[u] = 0.0;
                if (k0 + u < w) {
                    const int e = base + 32 * (k0 + u) + lane;
                    cj[u] = __ldg(Ac.col + e);
                    ax[u] = __ldg(Cxc + e);
                    ay[u] = __ldg(Cyc + e);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (k0 + u < w) {
                    const double2 uv = U2[cj[u]];
                    sx += ax[u] * uv.x;
                    sy += ay[u] * uv.y;
                }
            }
        }
        const double s = sx + sy;
        if (i < Ac.n) {
            double r = (tag[i] & CGP_PHI_ZERO) ? 0.0 : -1.5 / dt * s;
            rc[i] = r;
            acc[0] += r;
        }
    }
    double tot[1];
    if (grid_sum<1>(acc, partials, ticket, tot) && threadIdx.x == 0) st->mean = pure_neumann ? tot[0] / Ac.n : 0.0;
}

// Eq. 23 with a prescribed pressure on Gamma_N (has_natural_data): phi = g = p(t^{n+1}) - P^n
// at the PHI_ZERO rows and K_c[i, Gamma_N] g moved to the right-hand side of the others
// (the rows and columns of the PHI_ZERO vertices are those of the identity in the solve)
__global__ void __launch_bounds__(kBlock) k_coarse_lift(SellView Ac, const double* __restrict__ Kc,
                                                       const uint8_t* __restrict__ tag, const double* __restrict__ xy,
                                                       const double* __restrict__ P, BcParams bc,
                                                       const double* __restrict__ tdev, double dt,
                                                       double* __restrict__ rc) {
    const int lane = threadIdx.x & 31;
    const double tn = *tdev + dt;
    auto g = [&](int j) { return natural_pressure(bc, xy[2 * j], xy[2 * j + 1], tn) - P[j]; };
    CGP_SLICE_LOOP(Ac, sl) {
        const int i = sl * 32 + lane;
        double s[1] = {0.0};
        sell_accum<1>(Ac, Kc, sl, lane, [&](int j, double (&o)[1]) { o[0] = (tag[j] & CGP_PHI_ZERO) ? g(j) : 0.0; }, s);
        if (i < Ac.n) rc[i] = (tag[i] & CGP_PHI_ZERO) ? g(i) : rc[i] - s[0];
    }
}

// One level of P^T, the transposed prolongation (CGP_RESTRICT_PT).  On a red refinement the
// neighbours of an old vertex on the finer level are exactly the midpoints of its incident
// edges, each of which P sets to half of it, so y_c[i] = y_f[i] + 1/2 of the sum of y_f over
// those neighbours: a gather over the finer level's adjacency (diagonal skipped).
__global__ void k_restrict_t(int nc, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const double* __restrict__ yf, double* __restrict__ yc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
            const int j = col[q];
            if (j != i) s += yf[j];
        }
        yc[i] = yf[i] + 0.5 * s;
    }
}

// right-hand side of Eq. 23 from the restricted fine divergence y (CGP_RESTRICT_PT)
__global__ void __launch_bounds__(kBlock) k_coarse_rhs_pt(int nc, const double* __restrict__ y,
                                                         const uint8_t* __restrict__ tag, double dt,
                                                         double* __restrict__ rc, KrylovState* st, int pure_neumann,
                                                         double* partials, unsigned int* ticket) {
    double acc[1] = {0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
        const double r = (tag[i] & CGP_PHI_ZERO) ? 0.0 : -1.5 / dt * y[i];
        rc[i] = r;
        acc[0] += r;
    }
    double tot[1];
    if (grid_sum<1>(acc, partials, ticket, tot) && threadIdx.x == 0) st->mean = pure_neumann ? tot[0] / nc : 0.0;
}

// mean fix of a pure-Neumann solution: mu = sum m_i phi_i / sum m_i
__global__ void __launch_bounds__(kBlock) k_phi_mean(int n, const double* __restrict__ m, const double* __restrict__ phi,
                                                    double* __restrict__ out, double* partials, unsigned int* ticket) {
    double acc[2] = {0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        acc[0] += m[i] * phi[i];
        acc[1] += m[i];
    }
    double tot[2];
    if (grid_sum<2>(acc, partials, ticket, tot) && threadIdx.x == 0) *out = tot[0] / tot[1];
}

// plain mean of a given right-hand side (stand-alone Poisson solves)
__global__ void __launch_bounds__(kBlock) k_rhs_mean(int n, const double* __restrict__ r, KrylovState* st,
                                                    int pure_neumann, double* partials, unsigned int* ticket) {
    double acc[1] = {0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc[0] += r[i];
    double tot[1];
    if (grid_sum<1>(acc, partials, ticket, tot) && threadIdx.x == 0) st->mean = pure_neumann ? tot[0] / n : 0.0;
}

__global__ void k_sub_scalar(int n, double* __restrict__ x, const double* __restrict__ mu) {
    const double m = *mu;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] -= m;
}

// Eq. 24, one level: phi[nv_c + e] = (phi[a_e] + phi[b_e]) / 2; coincident vertices keep their value
__global__ void k_prolong(int n_new, int nv_c, const int32_t* __restrict__ parents, double* __restrict__ phi) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_new; e += gridDim.x * blockDim.x) {
        const int2 pr = reinterpret_cast<const int2*>(parents)[e];
        phi[nv_c + e] = 0.5 * (phi[pr.x] + phi[pr.y]);
    }
}

// Eq. 25 right-hand side: g = -2/3 dt (Cx phi, Cy phi), 0 on Dirichlet rows.  If lumped,
// delta = g / m directly (and no solve follows).
__global__ void __launch_bounds__(kBlock) k_corr_rhs(SellView A, const double* __restrict__ Cx,
                                                    const double* __restrict__ Cy, const double* __restrict__ phi,
                                                    const uint8_t* __restrict__ tag, double dt,
                                                    double* __restrict__ g, const double* __restrict__ mlump,
                                                    double* __restrict__ delta) {
    const int lane = threadIdx.x & 31;
    CGP_SLICE_LOOP(A, sl) {
        const int i = sl * 32 + lane;
        double ax[1] = {0.0}, ay[1] = {0.0};
        sell_accum<1>(A, Cx, sl, lane, [&](int j, double (&o)[1]) { o[0] = phi[j]; }, ax);
        sell_accum<1>(A, Cy, sl, lane, [&](int j, double (&o)[1]) { o[0] = phi[j]; }, ay);
        const double sx = ax[0], sy = ay[0];
        if (i < A.n) {
            const double c = -2.0 / 3.0 * dt;
            double2 gv = (tag[i] & CGP_VEL_DIR) ? make_double2(0.0, 0.0) : make_double2(c * sx, c * sy);
            reinterpret_cast<double2*>(g)[i] = gv;
            if (mlump) reinterpret_cast<double2*>(delta)[i] = make_double2(gv.x / mlump[i], gv.y / mlump[i]);
        }
    }
}

// D U~ = Cx u~ + Cy v~ (rotational update, Eq. 26); lumped: q = div / m directly
__global__ void __launch_bounds__(kBlock) k_div(SellView A, const double* __restrict__ Cx, const double* __restrict__ Cy,
                                               const double* __restrict__ Ut, double* __restrict__ div,
                                               const double* __restrict__ mlump, double* __restrict__ q) {
    const int lane = threadIdx.x & 31;
    CGP_SLICE_LOOP(A, sl) {
        const int i = sl * 32 + lane;
        double sx[1] = {0.0}, sy[1] = {0.0};
        sell_accum<1>(A, Cx, sl, lane, [&](int j, double (&o)[1]) { o[0] = Ut[2 * j]; }, sx);
        sell_accum<1>(A, Cy, sl, lane, [&](int j, double (&o)[1]) { o[0] = Ut[2 * j + 1]; }, sy);
        const double s = sx[0] + sy[0];
        if (i < A.n) {
            div[i] = s;
            if (mlump) q[i] = s / mlump[i];
        }
    }
}

// a new state's time (a kernel argument: no host staging) and zeroed run statistics
__global__ void k_set_time(double* tdev, double t, DeviceStats* stats) {
    static_assert(sizeof(DeviceStats) % sizeof(int64_t) == 0, "stats are zeroed as 64-bit words");
    int64_t* w = reinterpret_cast<int64_t*>(stats);
    for (int i = threadIdx.x; i < (int)(sizeof(DeviceStats) / sizeof(int64_t)); i += blockDim.x) w[i] = 0;
    if (threadIdx.x == 0) *tdev = t;
}

// end of step: U^{n-1} <- U^n, U^{n+1} = U~ + delta (Eq. 25), P^{n+1} = P^n + phi_f - chi/Re q (Eq. 26)
__global__ void k_finish(int nf, double* __restrict__ U, double* __restrict__ Uprev, const double* __restrict__ Ut,
                         const double* __restrict__ delta, double* __restrict__ P, const double* __restrict__ phi,
                         const double* __restrict__ q, int chi, double inv_re, double* __restrict__ tdev, double dt,
                         DeviceStats* stats, const KrylovState* ks, int fixed_launches, int pois_loop, int net) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
        const double2 u = reinterpret_cast<const double2*>(U)[i];
        const double2 ut = reinterpret_cast<const double2*>(Ut)[i];
        const double2 d = reinterpret_cast<const double2*>(delta)[i];
        reinterpret_cast<double2*>(Uprev)[i] = u;
        reinterpret_cast<double2*>(U)[i] = make_double2(ut.x + d.x, ut.y + d.y);
        double p = P[i] + phi[i];
        if (chi) p -= inv_re * q[i];
        P[i] = p;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *tdev = *tdev + dt;
        stats->steps += 1;
        // launches of a graph replay: the fixed kernels, 5 per BiCGStab iteration and 6 per
        // trip of an FP64 PCG loop body (two iterations per trip)
        int64_t l = fixed_launches + 5 * (int64_t)ks[KS_MOM].iter;
        for (int k = KS_POIS; k < KS_COUNT; ++k)
            if (k != KS_POIS || pois_loop) l += 6 * (int64_t)((ks[k].iter + 1) / 2);
        // FP32 inner loops of the mixed form: 5 kernels per BiCGStab trip (the Chebyshev mass
        // solves have a fixed launch count)
        l += 5 * (int64_t)ks[KS_MOM].trips;
        // the learned guess's network: `net` launches every step, or (net < 0) -net launches in
        // the steps whose coarse solve found the judge's gate open (its IF node ran)
        if (net > 0 || (net < 0 && (ks[KS_POIS].pad[1] & 2))) l += net > 0 ? net : -net;
        stats->launches += l;
        if (ks[KS_POIS].pad[1] & 1) stats->guess_used += 1;
        stats->sum_outer += ks[KS_POIS].pad[0];
        for (int k = 0; k < KS_COUNT; ++k) {
            const int it = ks[k].iter + (k != KS_POIS ? ks[k].inner : 0);   // FP64 + FP32 inner iterations
            stats->last_it[k] = it;
            stats->sum_it[k] += it;
            double r = 0.0;
            for (int c = 0; c < 2; ++c)
                if (ks[k].bb[c] > 0.0) r = fmax(r, sqrt(ks[k].rr[c] / ks[k].bb[c]));
            stats->res[k] = r;
            if (!stats->status && ks[k].status) stats->status = ks[k].status;
        }
    }
}

// scalar setup of a Krylov solve (tolerance, cap) before its init kernel
__global__ void k_ks_setup(KrylovState* st, double tol2, int maxit) {
    st->tol2 = tol2;
    st->maxit = maxit;
    st->iter = 0;
    st->done = 0;
    st->status = 0;
    st->pad[0] = 0;
    st->pad[1] = 0;
    st->skip = st->ir_done;   // refinement met the tolerance: the init keeps its residual, iter 0
    st->ir_done = 0;
}

// ---------------------------------------------------------------- loop control

static inline int prof_begin(Ctx& c, int id) {
    if (!c.prof || c.prof->n >= c.prof->cap) return -1;
    const int k = c.prof->n++;
    c.prof->id[k] = id;
    cudaEventRecord(c.prof->ev[2 * k], c.st);
    return k;
}

static inline void prof_end(Ctx& c, int k) {
    if (k >= 0) cudaEventRecord(c.prof->ev[2 * k + 1], c.st);
}

#define PL(c, pid, ...)                  \
    do {                                 \
        const int k_ = prof_begin(c, pid); \
        __VA_ARGS__;                     \
        prof_end(c, k_);                 \
    } while (0)

// bounded busy wait that keeps the stream ahead of the host while profiling
__global__ void k_spin(int iters) {
    for (int i = 0; i < iters; ++i) __nanosleep(1000);
}

static inline int grid_rows(const Solver& s, int n, int lanes) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t need = ((int64_t)n * lanes + kBlock - 1) / kBlock;
    int64_t cap = (int64_t)sms * 8;
    int g = (int)(need < cap ? need : cap);
    (void)s;
    return g < 1 ? 1 : g;
}

// Runs `init` once, then `body` until the KrylovState says done.  Eager: host polls the
// done flag after every `chunk` trips.  Capture: a WHILE conditional node whose body is
// captured on the side stream; the kernels set the condition themselves.
template <class Init, class Body>
static int krylov_loop(Ctx& c, KrylovState* ks, int max_trips, Init init, Body body) {
    Solver& s = *c.s;
    if (!c.capture) {
        if (c.prof) k_spin<<<1, 32, 0, c.st>>>(40);
        CGP_TRY(init(c.st, 0ull));
        const int chunk = c.prof ? 1 : 4;   // profiling: no trips after convergence
        for (int trip = 0; trip < max_trips; trip += chunk) {
            if (c.prof) k_spin<<<1, 32, 0, c.st>>>(40);
            for (int k = 0; k < chunk; ++k) CGP_TRY(body(c.st, 0ull));
            CGP_CUDA(cudaMemcpyAsync(s.h_flag, &ks->done, sizeof(int), cudaMemcpyDeviceToHost, c.st));
            CGP_CUDA(cudaStreamSynchronize(c.st));
            if (*s.h_flag) break;
        }
        return CGP_OK;
    }
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    CGP_CUDA(cudaStreamGetCaptureInfo(c.st, &cs, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphConditionalHandle handle;
    CGP_CUDA(cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault));
    CGP_TRY(init(c.st, (unsigned long long)handle));
    CGP_CUDA(cudaStreamGetCaptureInfo(c.st, &cs, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CGP_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp));
    cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
    CGP_CUDA(cudaStreamUpdateCaptureDependencies(c.st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    CGP_CUDA(cudaStreamBeginCaptureToGraph(s.side, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    int rc = body(s.side, (unsigned long long)handle);
    cudaGraph_t outg = nullptr;
    cudaError_t e = cudaStreamEndCapture(s.side, &outg);
    if (rc != CGP_OK) return rc;
    if (e != cudaSuccess) {
        set_error("loop body capture failed: %s", cudaGetErrorString(e));
        return CGP_ECUDA;
    }
    return CGP_OK;
}

// profile id of the p update of the PCG whose setup id is pid
static int pupd_id(int pid) {
    return pid == CGP_PROF_POIS_SETUP ? CGP_PROF_POIS_PUPD : pid == CGP_PROF_CORR_SETUP ? CGP_PROF_CORR_PUPD
                                                                                       : CGP_PROF_MASS_PUPD;
}

// PCG on (pattern A, values val, Jacobi dinv): b, x; NC components.  Three kernels per
// iteration (p update, SpMV, update); body = two iterations.
template <int NC>
static int pcg(Ctx& c, SellView A, const double* val, const double* dinv, double* b, double* x, KrylovState* ks,
               double tol, int maxit, bool zero_x, bool project, int pid) {
    Solver& s = *c.s;
    const int gs = grid_rows(s, A.nslices * 32, 1), gv = grid_rows(s, A.n, 1);
    const int pu = pupd_id(pid);
    auto init = [&, gs](cudaStream_t st, unsigned long long h) -> int {
        PL(c, pid, k_ks_setup<<<1, 1, 0, st>>>(ks, tol * tol, maxit));
        PL(c, pid + 1, k_pcg_init<NC><<<gs, kBlock, 0, st>>>(A, val, dinv, b, x, s.kr, s.kz, s.kp0, ks,
                                                                     s.partials, s.tickets, zero_x, project, h));
        CGP_LAUNCH_CHECK();
        return CGP_OK;
    };
    auto body = [&, gs, gv, pu](cudaStream_t st, unsigned long long h) -> int {
        for (int it = 0; it < 2; ++it) {
            PL(c, pu, k_pcg_pupd<NC><<<gv, kBlock, 0, st>>>(A.n, s.kz, s.kp0, ks));
            PL(c, pid + 2, k_pcg_spmv3<NC><<<gs, kBlock, 0, st>>>(A, val, s.kp0, s.kq, ks, s.partials, s.tickets));
            PL(c, pid + 3, k_pcg_update<NC><<<gv, kBlock, 0, st>>>(A.n, dinv, x, s.kr, s.kz, s.kp0, s.kq, ks,
                                                                   s.partials, s.tickets, h));
        }
        CGP_LAUNCH_CHECK();
        return CGP_OK;
    };
    return krylov_loop(c, ks, (maxit + 1) / 2 + 1, init, body);
}

static int bicgstab(Ctx& c, SellView A, const double* val, const double* dinv, const double* b, KrylovState* ks,
                    double tol, int maxit) {
    Solver& s = *c.s;
    const int gs = grid_rows(s, A.nslices * 32, 1), gv = grid_rows(s, A.n, 1);
    BicgVecs V = s.bv;
    auto init = [&, gs, V](cudaStream_t st, unsigned long long h) -> int {
        PL(c, CGP_PROF_MOM_SETUP, k_ks_setup<<<1, 1, 0, st>>>(ks, tol * tol, maxit));
        PL(c, CGP_PROF_MOM_INIT, k_bicg_init<<<gs, kBlock, 0, st>>>(A, val, b, V, ks, s.partials, s.tickets, h));
        CGP_LAUNCH_CHECK();
        return CGP_OK;
    };
    auto body = [&, gs, gv, V](cudaStream_t st, unsigned long long h) -> int {
        PL(c, CGP_PROF_BICG_P, k_bicg_p<<<gv, kBlock, 0, st>>>(A.n, dinv, V, ks));
        PL(c, CGP_PROF_BICG_V, k_bicg_v<<<gs, kBlock, 0, st>>>(A, val, V, ks, s.partials, s.tickets));
        PL(c, CGP_PROF_BICG_S, k_bicg_s<<<gv, kBlock, 0, st>>>(A.n, dinv, V, ks));
        PL(c, CGP_PROF_BICG_T, k_bicg_t<<<gs, kBlock, 0, st>>>(A, val, V, ks, s.partials, s.tickets));
        PL(c, CGP_PROF_BICG_X, k_bicg_x<<<gv, kBlock, 0, st>>>(A.n, V, ks, s.partials, s.tickets, h));
        CGP_LAUNCH_CHECK();
        return CGP_OK;
    };
    return krylov_loop(c, ks, maxit + 1, init, body);
}

// ---------------------------------------------------------------- mixed form: FP32 inner solves
// Iterative refinement for the fine-level systems of the mixed form (Eqs. 21, 25, 26): each
// sweep forms the FP64 residual r = b - A x, solves A e = r in FP32 (BiCGStab for Eq. 21 to
// a reduction kIrInnerTol of its residual norm, or less when less is left to reach the
// tolerance; fixed Chebyshev steps for the mass systems) and adds e to x in FP64.  The FP64 Krylov
// loop that follows polishes x to the tolerance and stops at once (its init sees the
// converged residual) when the sweeps already met it, so the result has the accuracy of
// the FP64 solve.  A sweep whose residual already meets the tolerance skips its inner solve.
constexpr int kIrSweeps = 3;
constexpr double kIrInnerTol = 1e-4;
constexpr int kIrInnerMaxit = 200;

template <int NC>
__global__ void __launch_bounds__(kBlock) k_ir_residual(SellView A, const double* __restrict__ val,
                                                       const double* __restrict__ b, double* __restrict__ x,
                                                       float* __restrict__ r32, KrylovState* st, KrylovState* in,
                                                       double tol2, int sweep, int zero_x, double* partials,
                                                       unsigned int* ticket) {
    const int lane = threadIdx.x & 31;
    double acc[2 * NC];
#pragma unroll
    for (int k = 0; k < 2 * NC; ++k) acc[k] = 0.0;
    CGP_SLICE_LOOP(A, sl) {
        const int i = sl * 32 + lane;
        double ax[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) ax[c] = 0.0;
        if (!zero_x) sell_accum<NC>(A, val, sl, lane, [&](int j, double (&o)[NC]) { ldv<NC>(x, j, o); }, ax);
        if (i < A.n) {
            double bv[NC], zero[NC];
            float rf[NC];
            ldv<NC>(b, i, bv);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const double r = bv[c] - ax[c];
                rf[c] = (float)r;
                zero[c] = 0.0;
                acc[c] += r * r;
                acc[NC + c] += bv[c] * bv[c];
            }
            stv<NC>(r32, i, rf);
            if (zero_x) stv<NC>(x, i, zero);
        }
    }
    double tot[2 * NC];
    if (grid_sum<2 * NC>(acc, partials, ticket, tot) && threadIdx.x == 0) {
        if (sweep == 0) {
            for (int c = 0; c < NC; ++c) st->bb[c] = tot[NC + c];
            st->inner = 0;
            st->trips = 0;
        }
        bool all = true, ok = true;
        for (int c = 0; c < NC; ++c) {
            st->rr[c] = tot[c];
            all &= tot[c] <= tol2 * st->bb[c];
            ok &= finite(tot[c]);
        }
        in->skip = (all || !ok) ? 1 : 0;
        st->ir_done = (all && ok) ? 1 : 0;
        // the inner solve aims at kIrInnerTol, or at what is left to the tolerance with a
        // factor 2 of margin in the norm when that is less (the strictest component counts)
        double t2 = kIrInnerTol * kIrInnerTol;
        if (ok) {
            double need = 1.0;
            for (int c = 0; c < NC; ++c)
                if (tot[c] > tol2 * st->bb[c]) need = fmin(need, 0.25 * tol2 * st->bb[c] / tot[c]);
            t2 = fmax(t2, need);
        }
        in->tol2 = t2;
        in->maxit = kIrInnerMaxit;
        in->iter = 0;
        in->done = 0;
        in->status = 0;
    }
}

// x += e (FP64) after an inner solve; counts its iterations and loop trips
template <int NC>
__global__ void __launch_bounds__(kBlock) k_ir_update(int n, double* __restrict__ x, const float* __restrict__ e,
                                                     KrylovState* st, const KrylovState* in, int iters_per_trip) {
    if (in->skip) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->inner += in->iter;
        if (iters_per_trip > 0) st->trips += (in->iter + iters_per_trip - 1) / iters_per_trip;
    }
    if (in->status == CGP_ENONFINITE) return;   // keep x; the FP64 loop takes over
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double xv[NC];
        float ev[NC];
        ldv<NC>(x, i, xv);
        ldv<NC>(e, i, ev);
#pragma unroll
        for (int c = 0; c < NC; ++c) xv[c] += (double)ev[c];
        stv<NC>(x, i, xv);
    }
}

// ---------------------------------------------------------------- Chebyshev mass solves
// The two fine-level mass-matrix systems of the mixed form (Eq. 25's velocity correction
// with M_0, Eq. 26's rotational term with M) run their FP32 inner solves as Chebyshev
// semi-iteration with the Jacobi preconditioner instead of PCG.  For P1 triangles the
// eigenvalues of D^{-1} M lie in [1/2, 2] (Wathen, IMA J. Numer. Anal. 7, 1987: each element
// matrix D_e^{-1} M_e has eigenvalues 1/2, 1/2, 2), and so do those of D^{-1} M_0 (its phi =
// 0 rows are identity rows, the rest a principal submatrix).  With those fixed bounds the
// iteration needs no inner products: each step is one kernel (SpMV of d, then e, r and the
// next d) with no grid-wide reduction, and k steps reduce the error by at least 2 / T_k(5/3)
// (about 3^-k; 12 steps: below 1e-5).  The recurrence (theta, delta: centre and half-width
// of the interval, sigma = theta / delta, rho_0 = 1 / sigma):
//   d_0 = D^{-1} r_0 / theta;  e += d_k,  r -= A d_k,  rho_{k+1} = 1 / (2 sigma - rho_k),
//   d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1} / delta) D^{-1} r_{k+1}.
// The FP64 residual of every refinement sweep and the FP64 PCG that follows stay the judge
// of the tolerance, as for the other refinement solves.
constexpr int kChebSweeps = 2;
constexpr int kChebSteps = 12;
constexpr double kChebLo = 0.5, kChebHi = 2.0;

// d = D^{-1} r / theta, e = 0; the step count for the statistics
template <int NC>
__global__ void __launch_bounds__(kBlock) k_cheb_init(int n, const float* __restrict__ dinv, const float* __restrict__ r,
                                                     float* __restrict__ d, float* __restrict__ e, KrylovState* in,
                                                     float inv_theta) {
    if (in->skip) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        in->iter = kChebSteps;
        in->status = 0;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float rv[NC], dv[NC], zero[NC];
        ldv<NC>(r, i, rv);
        const float di = dinv[i] * inv_theta;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            dv[c] = di * rv[c];
            zero[c] = 0.0f;
        }
        stv<NC>(d, i, dv);
        stv<NC>(e, i, zero);
    }
}

// one step: w = A d_in; e += d_in, r -= w, d_out = c1 d_in + c2 D^{-1} r
template <int NC>
__global__ void __launch_bounds__(kBlock) k_cheb_step(SellView A, const float* __restrict__ val,
                                                     const float* __restrict__ dinv, const float* __restrict__ din,
                                                     float* __restrict__ dout, float* __restrict__ r,
                                                     float* __restrict__ e, const KrylovState* in, float c1, float c2) {
    if (in->skip) return;
    const int lane = threadIdx.x & 31;
    CGP_SLICE_LOOP(A, sl) {
        const int i = sl * 32 + lane;
        // the row's own operands first: their loads overlap the SpMV's dependent chain
        float dv[NC], rv[NC], ev[NC], di = 0.0f;
        if (i < A.n) {
            ldv<NC>(din, i, dv);
            ldv<NC>(r, i, rv);
            ldv<NC>(e, i, ev);
            di = dinv[i];
        }
        float ax[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) ax[c] = 0.0f;
        sell_accum<NC>(A, val, sl, lane, [&](int j, float (&o)[NC]) { ldv<NC>(din, j, o); }, ax);
        if (i < A.n) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                ev[c] += dv[c];
                rv[c] -= ax[c];
                dv[c] = fmaf(c1, dv[c], c2 * di * rv[c]);
            }
            stv<NC>(e, i, ev);
            stv<NC>(r, i, rv);
            stv<NC>(dout, i, dv);
        }
    }
}

// FP32 copies of a matrix and its Jacobi diagonal
__global__ void k_to_f32_pair(int64_t n1, const double* __restrict__ a1, float* __restrict__ b1, int64_t n2,
                              const double* __restrict__ a2, float* __restrict__ b2) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n1; i += stride) b1[i] = (float)a1[i];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += stride) b2[i] = (float)a2[i];
}

// Mixed-form mass-matrix solve (Eqs. 25, 26): kChebSweeps refinement sweeps, each the FP64
// residual (and convergence test) of the current x, kChebSteps FP32 Chebyshev steps on
// A e = r, and x += e in FP64; then the FP64 PCG from that x to the tolerance.  Every kernel
// of a sweep returns at once when the residual had already converged.
template <int NC>
static int cheb_mixed(Ctx& c, SellView A, const double* val, const float* valf, const double* dinv, const float* dinvf,
                      double* b, double* x, KrylovState* ks, double tol, int maxit, bool zero_x, int pid, int step_id) {
    Solver& s = *c.s;
    KrylovState* in = s.ks + KS_COUNT;
    const int gs = grid_rows(s, A.nslices * 32, 1), gv = grid_rows(s, A.n, 1);
    float *fr = s.fv[0], *fe = s.fv[1], *fd[2] = {s.fv[2], s.fv[3]};
    const double theta = 0.5 * (kChebHi + kChebLo), delta = 0.5 * (kChebHi - kChebLo), sigma = theta / delta;
    for (int sw = 0; sw < kChebSweeps; ++sw) {
        PL(c, CGP_PROF_IR_RESID,
           k_ir_residual<NC><<<gs, kBlock, 0, c.st>>>(A, val, b, x, fr, ks, in, tol * tol, sw, zero_x && sw == 0,
                                                      s.partials, s.tickets));
        PL(c, CGP_PROF_F32_INIT, k_cheb_init<NC><<<gv, kBlock, 0, c.st>>>(A.n, dinvf, fr, fd[0], fe, in, (float)(1.0 / theta)));
        double rho = 1.0 / sigma;
        for (int k = 0; k < kChebSteps; ++k) {
            const double rho1 = 1.0 / (2.0 * sigma - rho);
            PL(c, step_id,
               k_cheb_step<NC><<<gs, kBlock, 0, c.st>>>(A, valf, dinvf, fd[k & 1], fd[(k + 1) & 1], fr, fe, in,
                                                        (float)(rho1 * rho), (float)(2.0 * rho1 / delta)));
            rho = rho1;
        }
        PL(c, CGP_PROF_IR_UPDATE, k_ir_update<NC><<<gv, kBlock, 0, c.st>>>(A.n, x, fe, ks, in, 0));
        CGP_LAUNCH_CHECK();
    }
    return pcg<NC>(c, A, val, dinv, b, x, ks, tol, maxit, false, false, pid);
}

// BiCGStab with FP32 inner solves (mixed form); the FP32 matrix is refreshed first
static int bicgstab_mixed(Ctx& c, SellView A, int64_t nnz, const double* val, const double* dinv, const double* b,
                          KrylovState* ks, double tol, int maxit) {
    Solver& s = *c.s;
    KrylovState* in = s.ks + KS_COUNT;
    const int gs = grid_rows(s, A.nslices * 32, 1), gv = grid_rows(s, A.n, 1);
    PL(c, CGP_PROF_TO_F32, k_to_f32_pair<<<gv, kBlock, 0, c.st>>>(nnz, val, s.Af, A.n, dinv, s.dinvAf));
    CGP_LAUNCH_CHECK();
    const BicgVecsT<float> V{s.fv[0], s.fv[1], s.fv[2], s.fv[3], s.fv[4], s.fv[5], s.fv[6], s.fv[7], s.fv[8]};
    for (int sw = 0; sw < kIrSweeps; ++sw) {
        PL(c, CGP_PROF_IR_RESID,
           k_ir_residual<2><<<gs, kBlock, 0, c.st>>>(A, val, b, s.bv.x, s.frhs, ks, in, tol * tol, sw, 0, s.partials,
                                                     s.tickets));
        CGP_LAUNCH_CHECK();
        auto init = [&, gs, V](cudaStream_t st, unsigned long long h) -> int {
            PL(c, CGP_PROF_F32_INIT,
               k_bicg_init<float><<<gs, kBlock, 0, st>>>(A, s.Af, s.frhs, V, in, s.partials, s.tickets, h, 1));
            CGP_LAUNCH_CHECK();
            return CGP_OK;
        };
        auto body = [&, gs, gv, V](cudaStream_t st, unsigned long long h) -> int {
            PL(c, CGP_PROF_F32_BICG_P, k_bicg_p<float><<<gv, kBlock, 0, st>>>(A.n, s.dinvAf, V, in));
            PL(c, CGP_PROF_F32_BICG_V, k_bicg_v<float><<<gs, kBlock, 0, st>>>(A, s.Af, V, in, s.partials, s.tickets));
            PL(c, CGP_PROF_F32_BICG_S, k_bicg_s<float><<<gv, kBlock, 0, st>>>(A.n, s.dinvAf, V, in));
            PL(c, CGP_PROF_F32_BICG_T, k_bicg_t<float><<<gs, kBlock, 0, st>>>(A, s.Af, V, in, s.partials, s.tickets));
            PL(c, CGP_PROF_F32_BICG_X, k_bicg_x<float><<<gv, kBlock, 0, st>>>(A.n, V, in, s.partials, s.tickets, h));
            CGP_LAUNCH_CHECK();
            return CGP_OK;
        };
        CGP_TRY(krylov_loop(c, in, kIrInnerMaxit + 1, init, body));
        PL(c, CGP_PROF_IR_UPDATE, k_ir_update<2><<<gv, kBlock, 0, c.st>>>(A.n, s.bv.x, V.x, ks, in, 1));
        CGP_LAUNCH_CHECK();
    }
    return bicgstab(c, A, val, dinv, b, ks, tol, maxit);
}

// ---------------------------------------------------------------- coarse solver choice
static cudaLaunchConfig_t cluster_config(int csize, cudaStream_t st, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize, 1, 1);
    cfg.blockDim = dim3(kClusterThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

int choose_coarse_solver(Solver& s, cudaStream_t st) {
    const cgp_params& p = s.prm;
    int mode = p.coarse_mode;
    if (mode == CGP_COARSE_ONCHIP && p.precision != CGP_MIXED) {
        set_error("CGP_COARSE_ONCHIP is the FP32 inner solve of CGP_MIXED");
        return CGP_EINVAL;
    }
    // the on-chip cluster solve when asked for, or by default for the mixed form if it fits
    const bool want_onchip = p.precision == CGP_MIXED && (mode == CGP_COARSE_ONCHIP || mode == CGP_COARSE_AUTO);
    if (p.precond == CGP_PRECOND_COARSE && !want_onchip) {
        set_error("CGP_PRECOND_COARSE needs the on-chip coarse solver (CGP_MIXED, coarse_mode AUTO or ONCHIP)");
        return CGP_EINVAL;
    }
    if (mode == CGP_COARSE_AUTO || mode == CGP_COARSE_ONCHIP) mode = CGP_COARSE_PERSISTENT;
    const bool allow_rr = mode == CGP_COARSE_PERSISTENT;
    if (mode == CGP_COARSE_PERSISTENT_MEM) mode = CGP_COARSE_PERSISTENT;
    s.coarse_kind = mode;
    s.coarse_fp64 = p.precision == CGP_FP64;
    s.cluster_size = 0;
    s.coarse_grid = 0;
    if (mode == CGP_COARSE_KERNELS) {
        if (p.precision == CGP_MIXED || p.guess == CGP_GUESS_LEARNED) {
            set_error("CGP_MIXED and CGP_GUESS_LEARNED need a one-launch coarse solver (persistent or cluster)");
            return CGP_EINVAL;
        }
        return CGP_OK;
    }
    int dev = 0, sms = 0;
    CGP_CUDA(cudaGetDevice(&dev));
    CGP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (mode == CGP_COARSE_PERSISTENT) {
        int coop = 0, per_sm = 0;
        CGP_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        CGP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_grid, kGridThreads, 0));
        if (!coop || per_sm < 1) {
            set_error("cooperative launch unavailable for the persistent coarse solver");
            return CGP_EINVAL;
        }
        const Level& C = s.mesh->lev[s.lc];
        // one slice per warp is enough; never more CTAs than can be co-resident
        const int need = (C.nslices + kGridThreads / 32 - 1) / (kGridThreads / 32);
        const int cap = sms * (per_sm < 2 ? per_sm : 2);
        s.coarse_grid = need < cap ? need : cap;
        if (s.coarse_grid < 1) s.coarse_grid = 1;
        // mixed precision: the whole FP32 inner solve on one cluster, if it fits on chip; the
        // largest subdomain coarse space that fits beside it (AUTO / COARSE), else Jacobi
        s.onchip_bytes = 0;
        if (want_onchip && s.oc_li) {
            std::vector<int32_t> rowptr(C.nv + 1), ptr(C.nslices + 1), col(C.nnz_sell);
            std::vector<double> xy(2 * (size_t)C.nv), val(C.nnz_sell);
            std::vector<uint8_t> tag(C.nv), in_space(C.nv);
            CGP_CUDA(cudaStreamSynchronize(st));   // the assembled K_c
            CGP_CUDA(cudaMemcpy(rowptr.data(), C.rowptr, sizeof(int32_t) * (C.nv + 1), cudaMemcpyDeviceToHost));
            CGP_CUDA(cudaMemcpy(ptr.data(), C.sell_ptr, sizeof(int32_t) * (C.nslices + 1), cudaMemcpyDeviceToHost));
            CGP_CUDA(cudaMemcpy(col.data(), C.sell_col, sizeof(int32_t) * C.nnz_sell, cudaMemcpyDeviceToHost));
            CGP_CUDA(cudaMemcpy(xy.data(), C.xy, sizeof(double) * 2 * C.nv, cudaMemcpyDeviceToHost));
            CGP_CUDA(cudaMemcpy(val.data(), s.Kc0, sizeof(double) * C.nnz_sell, cudaMemcpyDeviceToHost));
            CGP_CUDA(cudaMemcpy(tag.data(), C.tag, C.nv, cudaMemcpyDeviceToHost));
            for (int i = 0; i < C.nv; ++i) in_space[i] = (tag[i] & CGP_PHI_ZERO) ? 0 : 1;
            int optin = 0;
            CGP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
            const size_t limit = (size_t)optin - 2048;   // static shared memory of the kernel
            const bool coarse_space = p.precond != CGP_PRECOND_JACOBI;
            for (int cs : {16, 8}) {
                for (int spc : {8, 4, 2, 1, 0}) {
                    if (spc && !coarse_space) continue;
                    OnchipHostPlan P;
                    if (!onchip_plan(C.nv, rowptr, ptr, col, xy, in_space, cs, spc, limit, P)) continue;
                    if (!onchip_coarse_space(rowptr, ptr, col, val, P)) continue;
                    const OnchipKernelFn kern = onchip_kernel(P.nsub);
                    CGP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
                    CGP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit));
                    cudaLaunchAttribute attr[1];
                    cudaLaunchConfig_t cfg = cluster_config(cs, nullptr, attr);
                    cfg.blockDim = dim3(kOnchipThreads, 1, 1);
                    cfg.dynamicSmemBytes = P.bytes;
                    int n = 0;
                    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n < 1) {
                        cudaGetLastError();
                        continue;
                    }
                    auto up = [](auto* dst, const auto& v) {
                        return v.empty() ? cudaSuccess
                                         : cudaMemcpy(dst, v.data(), sizeof(v[0]) * v.size(), cudaMemcpyHostToDevice);
                    };
                    CGP_CUDA(up(s.oc_grow, P.grow));
                    CGP_CUDA(up(s.oc_soff, P.soff));
                    CGP_CUDA(up(s.oc_ebase, P.ebase));
                    CGP_CUDA(up(s.oc_width, P.width));
                    CGP_CUDA(up(s.oc_li, P.li));
                    CGP_CUDA(up(s.oc_src, P.src));
                    CGP_CUDA(up(s.oc_send_lr, P.send_lr));
                    CGP_CUDA(up(s.oc_send_dst, P.send_dst));
                    CGP_CUDA(up(s.oc_send_off, P.send_off));
                    CGP_CUDA(up(s.oc_halo_n, P.halo_n));
                    CGP_CUDA(up(s.oc_hsub, P.hsub));
                    CGP_CUDA(up(s.oc_hrow, P.hrow));
                    CGP_CUDA(up(s.oc_send_woff, P.send_woff));
                    CGP_CUDA(up(s.oc_einv, P.einv));
                    CGP_CUDA(up(s.oc_need, P.need));
                    CGP_CUDA(up(s.oc_need_n, P.need_n));
                    s.onchip = OnchipPlan{s.oc_grow, s.oc_soff, s.oc_ebase, s.oc_width, s.oc_li, s.oc_src,
                                          s.oc_send_lr, s.oc_send_dst, s.oc_send_off, s.oc_send_woff, s.oc_halo_n,
                                          s.oc_hrow, s.oc_hsub, s.oc_einv, s.oc_need, s.oc_need_n, P.rows_max,
                                          P.halo_max, P.send_max, (int)P.ent_max, P.nsub, P.wpg, P.need_max};
                    s.onchip_bytes = P.bytes;
                    s.cluster_size = cs;
                    break;
                }
                if (s.onchip_bytes) break;
            }
            if (p.precond == CGP_PRECOND_COARSE && !(s.onchip_bytes && s.onchip.nsub)) {
                set_error("the coarse system does not fit on one thread-block cluster with a coarse space");
                return CGP_EINVAL;
            }
            if (p.coarse_mode == CGP_COARSE_ONCHIP && !s.onchip_bytes) {
                set_error("the coarse system does not fit on one thread-block cluster");
                return CGP_EINVAL;
            }
        }
        // register-resident variant: every slice no wider than kRRWidth and one slice per warp
        s.coarse_rr = false;
        if (allow_rr) {
            std::vector<int32_t> ptr(C.nslices + 1);
            CGP_CUDA(cudaMemcpy(ptr.data(), C.sell_ptr, sizeof(int32_t) * (C.nslices + 1), cudaMemcpyDeviceToHost));
            int wmax = 0;
            for (int k = 0; k < C.nslices; ++k) wmax = std::max(wmax, (ptr[k + 1] - ptr[k]) / 32);
            int per_sm_rr = 0;
            CGP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_rr, k_pcg_grid_rr, kGridThreads, 0));
            s.coarse_rr = wmax <= kRRWidth && per_sm_rr > 0 && rr_ctas_needed(C.nslices) <= sms * per_sm_rr;
        }
        // mixed form, AUTO, no room on chip: the grid-wide FP64 solve (one reduction per
        // iteration) is faster on this GPU than the FP32 inner solve (two) with the same grid
        // barriers; the fine-level solves stay FP32-inner.  An explicit PERSISTENT request
        // keeps the FP32 inner solve.
        s.coarse_fp64 = p.precision == CGP_FP64 || (p.coarse_mode == CGP_COARSE_AUTO && !s.onchip_bytes);
        return CGP_OK;
    }
    CGP_CUDA(cudaFuncSetAttribute(k_pcg_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    const int cands[] = {16, 8, 4, 2};
    for (int cs : cands) {
        if (p.cluster_size && cs != p.cluster_size) continue;
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = cluster_config(cs, nullptr, attr);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_pcg_cluster, &cfg) == cudaSuccess && n > 0) {
            s.cluster_size = cs;
            break;
        }
        cudaGetLastError();
    }
    if (!s.cluster_size) {
        set_error("no thread-block cluster of the requested size fits this device");
        return CGP_EINVAL;
    }
    return CGP_OK;
}

// ---------------------------------------------------------------- pieces of a step
// Reduction asked of each FP32 inner coarse solve when tol_inner is left at 0: 1e-5 (about
// two refinement sweeps a solve) for the on-chip solve with the subdomain coarse correction
// and for the Jacobi solves of the cluster and batched forms; 1e-3 for the on-chip solve
// with Jacobi alone, whose FP32 recurrence stagnates before 1e-5 on its larger condition
// number and then wastes its stagnation window at every restart.
static double inner_tol_of(const Solver& s, bool onchip_solve) {
    if (s.prm.tol_inner > 0) return s.prm.tol_inner;
    return onchip_solve && !s.onchip.nsub ? 1e-3 : 1e-5;
}

// arguments of the one-launch coarse solver for this solver's current state
CoarsePcgArgs coarse_args(Solver& s) {
    const Level& C = s.mesh->lev[s.lc];
    CoarsePcgArgs a;
    a.A = sell_of(C);
    a.val = s.Kc0;
    a.valf = s.Kc0f;
    a.dinv = s.dinvKc;
    a.dinvf = s.dinvKcf;
    a.b = s.rc;
    a.x = s.phi;
    a.x_alt = (s.prm.guess == CGP_GUESS_LEARNED && s.guess_ready) ? s.phi_guess : nullptr;
    a.w64 = s.cw64;
    a.w32 = s.cw32;
    a.mlump = s.pure_neumann ? s.mlumpC : nullptr;
    a.st = &s.ks[KS_POIS];
    a.tol2 = s.prm.tol_poisson * s.prm.tol_poisson;
    a.inner_tol = inner_tol_of(s, s.onchip_bytes != 0);
    a.maxit = s.prm.max_it_poisson;
    a.zero_x = s.prm.guess == CGP_GUESS_ZERO;
    a.project = s.pure_neumann;
    a.mixed = !s.coarse_fp64;
    a.max_outer = 50;
    a.bar_count = s.bar_count;
    a.bar_err = s.bar_err;
    a.partials = s.coarse_partials;
    a.wait_test = s.wait_test;
    a.gate = s.onchip_bytes ? s.mlp_gate : nullptr;
    return a;
}

// the learned prediction of Phi_c (before the coarse solve, which judges it).  Captured into
// a graph, the network's launches sit in an IF node whose condition the projection kernel
// before it sets (`cond`), so while the judge has the network off a step skips its four grids.
static int learned_guess(Ctx& c, unsigned long long cond) {
    Solver& s = *c.s;
    if (!(s.prm.guess == CGP_GUESS_LEARNED && s.guess_ready)) return CGP_OK;
    const Level& Cl = s.mesh->lev[s.lc];
    const int* gate = s.onchip_bytes ? s.mlp_gate : nullptr;
    auto forward = [&](cudaStream_t st) { return mlp_forward(s.mlp, Cl, s.rc, s.phi, 1, s.phi_guess, st, gate); };
    if (!cond) {
        PL(c, CGP_PROF_MLP, CGP_TRY(forward(c.st)));
        return CGP_OK;
    }
    const cudaGraphConditionalHandle handle = (cudaGraphConditionalHandle)cond;
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    CGP_CUDA(cudaStreamGetCaptureInfo(c.st, &cs, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CGP_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp));
    cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
    CGP_CUDA(cudaStreamUpdateCaptureDependencies(c.st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    CGP_CUDA(cudaStreamBeginCaptureToGraph(s.side, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    const int rc = forward(s.side);
    cudaGraph_t outg = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s.side, &outg);
    if (rc != CGP_OK) return rc;
    if (e != cudaSuccess) {
        set_error("network capture failed: %s", cudaGetErrorString(e));
        return CGP_ECUDA;
    }
    return CGP_OK;
}

static int coarse_solve(Ctx& c) {
    Solver& s = *c.s;
    const Level& C = s.mesh->lev[s.lc];
    SellView Ac = sell_of(C);
    const bool zero_x = s.prm.guess == CGP_GUESS_ZERO;
    if (s.coarse_kind == CGP_COARSE_CLUSTER || s.coarse_kind == CGP_COARSE_PERSISTENT) {
        CoarsePcgArgs a = coarse_args(s);
        if (s.coarse_kind == CGP_COARSE_CLUSTER) {
            cudaLaunchAttribute attr[1];
            cudaLaunchConfig_t cfg = cluster_config(s.cluster_size, c.st, attr);
            PL(c, CGP_PROF_POIS_CLUSTER, CGP_CUDA(cudaLaunchKernelEx(&cfg, k_pcg_cluster, a)));
            return CGP_OK;
        }
        if (s.onchip_bytes) {
            cudaLaunchAttribute attr[1];
            cudaLaunchConfig_t cfg = cluster_config(s.cluster_size, c.st, attr);
            cfg.blockDim = dim3(kOnchipThreads, 1, 1);
            cfg.dynamicSmemBytes = s.onchip_bytes;
            PL(c, CGP_PROF_POIS_CLUSTER, CGP_CUDA(cudaLaunchKernelEx(&cfg, onchip_kernel(s.onchip.nsub), a, s.onchip)));
            return CGP_OK;
        }
        CGP_CUDA(cudaMemsetAsync(s.bar_count, 0, 2 * sizeof(unsigned int), c.st));   // counter + error word
        cudaLaunchConfig_t cfg = {};
        const bool rr = s.coarse_rr && s.coarse_fp64;
        cfg.gridDim = dim3(rr ? rr_ctas_needed(C.nslices) : s.coarse_grid, 1, 1);
        cfg.blockDim = dim3(kGridThreads, 1, 1);
        cfg.stream = c.st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (rr) PL(c, CGP_PROF_POIS_CLUSTER, CGP_CUDA(cudaLaunchKernelEx(&cfg, k_pcg_grid_rr, a)));
        else PL(c, CGP_PROF_POIS_CLUSTER, CGP_CUDA(cudaLaunchKernelEx(&cfg, k_pcg_grid, a)));
        return CGP_OK;
    }
    CGP_TRY(pcg<1>(c, Ac, s.Kc0, s.dinvKc, s.rc, s.phi, &s.ks[KS_POIS], s.prm.tol_poisson, s.prm.max_it_poisson,
                   zero_x, s.pure_neumann, CGP_PROF_POIS_SETUP));
    if (s.pure_neumann) {
        PL(c, CGP_PROF_PHI_MEAN, k_phi_mean<<<grid_rows(s, C.nv, 1), kBlock, 0, c.st>>>(C.nv, s.mlumpC, s.phi, s.scal,
                                                                                        s.partials, s.tickets));
        PL(c, CGP_PROF_PHI_SUB, k_sub_scalar<<<grid_rows(s, C.nv, 1), kBlock, 0, c.st>>>(C.nv, s.phi, s.scal));
        CGP_LAUNCH_CHECK();
    }
    return CGP_OK;
}

static int prolong_all(Ctx& c) {
    Solver& s = *c.s;
    for (int l = s.lc; l < s.lf; ++l) {
        const Level& Lc = s.mesh->lev[l];
        const Level& Lf = s.mesh->lev[l + 1];
        const int n_new = Lf.nv - Lc.nv;
        PL(c, CGP_PROF_PROLONG, k_prolong<<<grid_rows(s, n_new, 1), kBlock, 0, c.st>>>(n_new, Lc.nv, Lf.parents, s.phi));
    }
    CGP_LAUNCH_CHECK();
    return CGP_OK;
}

// Eq. 21 and the right-hand side of Eq. 23 (+ the learned prediction)
int step_pre(Ctx& c) {
    Solver& s = *c.s;
    const cgp_params& p = s.prm;
    const Level& F = s.mesh->lev[s.lf];
    const Level& C = s.mesh->lev[s.lc];
    const BcParams bc = bc_of(s);
    SellView Af = sell_of(F), Ac = sell_of(C);
    const int gv = grid_rows(s, F.nv, 1);
    PL(c, CGP_PROF_MOM_PREP, k_mom_prep<<<gv, kBlock, 0, c.st>>>(F.nv, s.U, s.Uprev, F.xy, bc, s.tdev, p.dt, s.w, s.h));
    PL(c, CGP_PROF_MOM_ASSEMBLE,
       k_mom_assemble<<<gv, kBlock, 0, c.st>>>(F.nv, F.rowptr, F.col, F.sell_ptr, F.vt_ptr, F.vt_list, F.tri, s.geo,
                                               s.vtslot, s.S, s.M, s.CxT, s.CyT, s.P, s.w, s.h, F.tag, F.xy, bc,
                                               s.tdev, p.dt, s.A, s.dinvA, s.b, s.Ut));
    CGP_LAUNCH_CHECK();
    if (p.precision == CGP_MIXED)
        CGP_TRY(bicgstab_mixed(c, Af, F.nnz_sell, s.A, s.dinvA, s.b, &s.ks[KS_MOM], p.tol_mom, p.max_it_mom));
    else
        CGP_TRY(bicgstab(c, Af, s.A, s.dinvA, s.b, &s.ks[KS_MOM], p.tol_mom, p.max_it_mom));
    // Eqs. 22-23: injection and coarse divergence
    if (p.restrict_mode == CGP_RESTRICT_PT) {
        // fine divergence, then P^T level by level (ping-pong in two Krylov work vectors that
        // are free until the coarse solve)
        PL(c, CGP_PROF_COARSE_RHS,
           k_div<<<grid_rows(s, F.nslices * 32, 1), kBlock, 0, c.st>>>(Af, s.Cx, s.Cy, s.Ut, s.div, nullptr, nullptr));
        const double* y = s.div;
        double* buf[2] = {s.kz, s.kq};
        for (int l = s.lf, b = 0; l > s.lc; --l, b ^= 1) {
            const Level& L = s.mesh->lev[l];
            const int nc = s.mesh->lev[l - 1].nv;
            PL(c, CGP_PROF_COARSE_RHS,
               k_restrict_t<<<grid_rows(s, nc, 1), kBlock, 0, c.st>>>(nc, L.rowptr, L.col, y, buf[b]));
            y = buf[b];
        }
        PL(c, CGP_PROF_COARSE_RHS,
           k_coarse_rhs_pt<<<grid_rows(s, C.nv, 1), kBlock, 0, c.st>>>(C.nv, y, C.tag, p.dt, s.rc, &s.ks[KS_POIS],
                                                                         s.pure_neumann, s.partials, s.tickets));
    } else {
        PL(c, CGP_PROF_COARSE_RHS,
           k_coarse_rhs<<<grid_rows(s, C.nslices * 32, 1), kBlock, 0, c.st>>>(
               Ac, s.Cxc, s.Cyc, s.Ut, C.tag, p.dt, s.rc, &s.ks[KS_POIS], s.pure_neumann, s.partials, s.tickets));
        if (p.bc_kind == CGP_BC_JOBELIN_OPEN)
            PL(c, CGP_PROF_COARSE_RHS, k_coarse_lift<<<grid_rows(s, C.nslices * 32, 1), kBlock, 0, c.st>>>(
                                           Ac, s.Kc, C.tag, C.xy, s.P, bc, s.tdev, p.dt, s.rc));
    }
    CGP_LAUNCH_CHECK();
    // captured with the learned guess and its judge: the IF condition of the network's launches
    unsigned long long cond = 0;
    if (c.capture && s.proj && s.prm.guess == CGP_GUESS_LEARNED && s.guess_ready && s.onchip_bytes) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        CGP_CUDA(cudaStreamGetCaptureInfo(c.st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle handle;
        CGP_CUDA(cudaGraphConditionalHandleCreate(&handle, g, 0, cudaGraphCondAssignDefault));
        cond = (unsigned long long)handle;
    }
    if (s.proj) {
        // the projection guess of the coarse solve (and the network's second input)
        const int gc = grid_rows(s, C.nv, 1);
        PL(c, CGP_PROF_PROJ, k_proj_coef<<<gc, kBlock, 0, c.st>>>(C.nv, s.hist_x, s.hist_b, s.rc, &s.ks[KS_POIS],
                                                                   s.proj, p.tol_poisson, s.partials, s.tickets));
        PL(c, CGP_PROF_PROJ, k_proj_combine<<<gc, kBlock, 0, c.st>>>(C.nv, s.hist_x, s.proj, s.phi, s.phi_q, s.mlp_gate,
                                                                      cond));
        CGP_LAUNCH_CHECK();
    }
    return learned_guess(c, cond);
}

// The rotational term of Eq. 26: M q = Cx u~ + Cy v~ (consistent M), or its lumped form.
// It needs only U~, so it may run beside the coarse solve.
static int rotational_term(Ctx& c) {
    Solver& s = *c.s;
    const cgp_params& p = s.prm;
    const Level& F = s.mesh->lev[s.lf];
    SellView Af = sell_of(F);
    const int gs = grid_rows(s, F.nslices * 32, 1);
    const bool lumped = p.mass_mode == CGP_MASS_LUMPED, mixed = p.precision == CGP_MIXED;
    PL(c, CGP_PROF_DIV,
       k_div<<<gs, kBlock, 0, c.st>>>(Af, s.Cx, s.Cy, s.Ut, s.div, lumped ? s.mlumpF : nullptr, s.qrot));
    CGP_LAUNCH_CHECK();
    if (!lumped && mixed)
        CGP_TRY(cheb_mixed<1>(c, Af, s.M, s.Mf, s.dinvM, s.dinvMf, s.div, s.qrot, &s.ks[KS_MASS], p.tol_mass,
                              p.max_it_mass, true, CGP_PROF_MASS_SETUP, CGP_PROF_CHEB_MASS));
    else if (!lumped)
        CGP_TRY(pcg<1>(c, Af, s.M, s.dinvM, s.div, s.qrot, &s.ks[KS_MASS], p.tol_mass, p.max_it_mass, true, false,
                       CGP_PROF_MASS_SETUP));
    return CGP_OK;
}

// Eqs. 24-26 and the end of the step (mass_done: the rotational term was formed already)
int step_post(Ctx& c, bool mass_done) {
    Solver& s = *c.s;
    const cgp_params& p = s.prm;
    const Level& F = s.mesh->lev[s.lf];
    SellView Af = sell_of(F);
    const int gv = grid_rows(s, F.nv, 1), gs = grid_rows(s, F.nslices * 32, 1);
    if (s.proj) {
        // the new coarse solution joins the projection window
        const int nc = s.mesh->lev[s.lc].nv;
        PL(c, CGP_PROF_PROJ, k_proj_push<<<grid_rows(s, nc, 1), kBlock, 0, c.st>>>(nc, s.phi, s.hist_x, s.hist_b,
                                                                                     s.proj, s.partials, s.tickets));
        CGP_LAUNCH_CHECK();
    }
    // Eq. 24: prolongation
    CGP_TRY(prolong_all(c));
    // Eq. 25: velocity correction
    const bool lumped = p.mass_mode == CGP_MASS_LUMPED;
    PL(c, CGP_PROF_CORR_RHS,
       k_corr_rhs<<<gs, kBlock, 0, c.st>>>(Af, s.Cx, s.Cy, s.phi, F.tag, p.dt, s.g,
                                                   lumped ? s.mlumpF : nullptr, s.delta));
    CGP_LAUNCH_CHECK();
    const bool mixed = p.precision == CGP_MIXED;
    if (!lumped && mixed)
        CGP_TRY(cheb_mixed<2>(c, Af, s.M0, s.M0f, s.dinvM0, s.dinvM0f, s.g, s.delta, &s.ks[KS_CORR], p.tol_mass,
                              p.max_it_mass, true, CGP_PROF_CORR_SETUP, CGP_PROF_CHEB_CORR));
    else if (!lumped)
        CGP_TRY(pcg<2>(c, Af, s.M0, s.dinvM0, s.g, s.delta, &s.ks[KS_CORR], p.tol_mass, p.max_it_mass, true, false,
                       CGP_PROF_CORR_SETUP));
    // Eq. 26: pressure
    if (p.chi && !mass_done) CGP_TRY(rotational_term(c));
    const bool one_launch = s.coarse_kind != CGP_COARSE_KERNELS;
    const int coarse_fixed = (one_launch ? 1 : 2 + (s.pure_neumann ? 2 : 0)) + (s.proj ? 3 : 0);
    // the network's four launches, behind the judge's IF node where the on-chip solve judges it
    const int net = (p.guess == CGP_GUESS_LEARNED && s.guess_ready) ? (s.onchip_bytes ? -4 : 4) : 0;
    // mixed: the FP32 copy of A; momentum: kIrSweeps x (residual, inner init, update); each
    // Chebyshev mass solve: kChebSweeps x (residual, init, kChebSteps steps, update)
    const int ir_fixed = mixed ? 1 + 3 * kIrSweeps +
                                     (3 + kChebSteps) * kChebSweeps * ((lumped ? 0 : 1) + (p.chi && !lumped ? 1 : 0))
                               : 0;
    const int pt_fixed = (p.restrict_mode == CGP_RESTRICT_PT ? 1 + (s.lf - s.lc) : 0) +   // k_div + the P^T levels
                         (p.bc_kind == CGP_BC_JOBELIN_OPEN ? 1 : 0);                     // k_coarse_lift
    const int fixed =
        4 + 1 + coarse_fixed + (s.lf - s.lc) + 1 + (lumped ? 0 : 2) + (p.chi ? 1 + (lumped ? 0 : 2) : 0) + 1 + ir_fixed +
        pt_fixed;
    PL(c, CGP_PROF_FINISH,
       k_finish<<<gv, kBlock, 0, c.st>>>(F.nv, s.U, s.Uprev, s.Ut, s.delta, s.P, s.phi, s.qrot, p.chi, 1.0 / p.Re,
                                         s.tdev, p.dt, s.stats, s.ks, fixed, one_launch ? 0 : 1, net));
    CGP_LAUNCH_CHECK();
    return CGP_OK;
}

static int step_body(Ctx& c) {
    Solver& s = *c.s;
    const cgp_params& p = s.prm;
    CGP_TRY(step_pre(c));
    // The on-chip coarse solve holds 16 SMs for most of the step; the rotational term of
    // Eq. 26 (its own mass solve) depends only on U~, so it runs on the other SMs meanwhile,
    // on a second stream.  Nothing on the main stream reduces into the shared scratch until
    // the branches join, before Eq. 24 (the velocity correction solve uses the same scratch).
    const bool overlap = !c.prof && s.onchip_bytes && p.chi && p.mass_mode != CGP_MASS_LUMPED && s.branch;
    if (!overlap) {
        CGP_TRY(coarse_solve(c));
        return step_post(c, false);
    }
    CGP_CUDA(cudaEventRecord(s.ev_fork, c.st));
    CGP_CUDA(cudaStreamWaitEvent(s.branch, s.ev_fork, 0));
    CGP_TRY(coarse_solve(c));
    Ctx b{c.s, s.branch, c.capture, nullptr};
    CGP_TRY(rotational_term(b));
    CGP_CUDA(cudaEventRecord(s.ev_join, s.branch));
    CGP_CUDA(cudaStreamWaitEvent(c.st, s.ev_join, 0));
    return step_post(c, true);
}

int init_state(Solver* s, cudaStream_t st) {
    const Level& F = s->mesh->lev[s->lf];
    k_init_state<<<blocks_for(F.nv), kBlock, 0, st>>>(F.nv, F.xy, F.tag, bc_of(*s), s->prm.dt, s->U, s->Uprev,
                                                      s->P, s->tdev);
    CGP_LAUNCH_CHECK();
    return CGP_OK;
}

static int build_graph(Solver& s) {
    cudaStream_t cap = nullptr;
    CGP_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    Ctx c{&s, cap, true};
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cap);
        set_error("begin capture failed: %s", cudaGetErrorString(e));
        return CGP_ECUDA;
    }
    int rc = step_body(c);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (rc != CGP_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) {
        set_error("end capture failed: %s", cudaGetErrorString(e));
        return CGP_ECUDA;
    }
    e = cudaGraphInstantiate(&s.step_exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        set_error("graph instantiation failed: %s", cudaGetErrorString(e));
        return CGP_ECUDA;
    }
    s.step_graph = g;
    return CGP_OK;
}

// ---------------------------------------------------------------- batched coarse solve
size_t coarse_args_size() { return sizeof(CoarsePcgArgs); }

void fill_coarse_args(Solver& s, void* dst) {
    CoarsePcgArgs a = coarse_args(s);
    a.inner_tol = inner_tol_of(s, false);   // the batched solve is the cluster Jacobi PCG
    memcpy(dst, &a, sizeof(a));
}

int batch_clusters(int csize, int threads, int* nclusters) {
    static bool attr_set = false;
    if (!attr_set) {
        CGP_CUDA(cudaFuncSetAttribute(k_pcg_batch, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        attr_set = true;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(csize, nullptr, attr);
    cfg.blockDim = dim3(threads, 1, 1);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_pcg_batch, &cfg) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    *nclusters = n;
    return CGP_OK;
}

int launch_batch_coarse(const void* d_args, int ninst, unsigned int* queue, int csize, int threads, int nclusters,
                        cudaStream_t st) {
    CGP_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned int), st));
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(csize, st, attr);
    cfg.gridDim = dim3(csize * nclusters, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    CGP_CUDA(cudaLaunchKernelEx(&cfg, k_pcg_batch, (const CoarsePcgArgs*)d_args, ninst, queue));
    return CGP_OK;
}

// ---------------------------------------------------------------- batched whole step
size_t batch_step_args_size() { return sizeof(BatchStepArgs); }

bool batch_step_eligible(const Solver& s) {
    return s.prm.restrict_mode == CGP_RESTRICT_INJECT &&
           (s.prm.guess == CGP_GUESS_ZERO || s.prm.guess == CGP_GUESS_PREV) && s.coarse_kind != CGP_COARSE_KERNELS;
}

void fill_batch_step_args(Solver& s, void* dst) {
    const Level& F = s.mesh->lev[s.lf];
    const Level& C = s.mesh->lev[s.lc];
    BatchStepArgs a{};
    a.nf = F.nv;
    a.Af = sell_of(F);
    a.rowptr = F.rowptr;
    a.col = F.col;
    a.sell_ptr = F.sell_ptr;
    a.vt_ptr = F.vt_ptr;
    a.vt_list = F.vt_list;
    a.tri = F.tri;
    a.vtslot = s.vtslot;
    a.geo = s.geo;
    a.xy = F.xy;
    a.S = s.S;
    a.M = s.M;
    a.M0 = s.M0;
    a.CxT = s.CxT;
    a.CyT = s.CyT;
    a.Cx = s.Cx;
    a.Cy = s.Cy;
    a.dinvM0 = s.dinvM0;
    a.dinvM = s.dinvM;
    a.mlumpF = s.mlumpF;
    a.tag = F.tag;
    a.U = s.U;
    a.Uprev = s.Uprev;
    a.P = s.P;
    a.Ut = s.Ut;
    a.w = s.w;
    a.h = s.h;
    a.A = s.A;
    a.dinvA = s.dinvA;
    a.b = s.b;
    a.g = s.g;
    a.delta = s.delta;
    a.div = s.div;
    a.qrot = s.qrot;
    a.phi = s.phi;
    a.bv = s.bv;
    a.c0 = s.kr;
    a.c1 = s.kz;
    a.c2 = s.kp0;
    a.Ac = sell_of(C);
    a.Cxc = s.Cxc;
    a.Cyc = s.Cyc;
    a.Kc = s.Kc;
    a.cxy = C.xy;
    a.ctag = C.tag;
    a.coarse = coarse_args(s);
    a.coarse.inner_tol = inner_tol_of(s, false);   // the whole-step kernel's coarse PCG is Jacobi
    a.pure_neumann = s.pure_neumann;
    a.nlev = s.lf - s.lc + 1;
    for (int l = 0; l < a.nlev; ++l) {
        a.nv[l] = s.mesh->lev[s.lc + l].nv;
        a.parents[l] = l + 1 < a.nlev ? s.mesh->lev[s.lc + l + 1].parents : nullptr;
    }
    a.bc = bc_of(s);
    a.dt = s.prm.dt;
    a.inv_re = 1.0 / s.prm.Re;
    a.tol_mom2 = s.prm.tol_mom * s.prm.tol_mom;
    a.chi = s.prm.chi;
    a.lumped = s.prm.mass_mode == CGP_MASS_LUMPED;
    a.max_it_mom = s.prm.max_it_mom;
    a.cheb_steps = cheb_steps_for(s.prm.tol_mass);
    if (s.Af) {
        a.nnz = F.nnz_sell;
        a.A32 = s.Af;
        a.dinvA32 = s.dinvAf;
        for (int k = 0; k < 9; ++k) a.fv[k] = s.fv[k];
        a.fv[9] = s.frhs;
    }
    a.tdev = s.tdev;
    a.stats = s.stats;
    a.ks = s.ks;
    memcpy(dst, &a, sizeof(a));
}

int batch_step_clusters(int csize, int threads, int* nclusters) {
    static bool attr_set = false;
    if (!attr_set) {
        CGP_CUDA(cudaFuncSetAttribute(k_batch_step, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        attr_set = true;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(csize, nullptr, attr);
    cfg.blockDim = dim3(threads, 1, 1);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_batch_step, &cfg) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    *nclusters = n;
    return CGP_OK;
}

int launch_batch_step(const void* d_args, int ninst, unsigned int* queue, int csize, int threads, int nclusters,
                      cudaStream_t st) {
    CGP_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned int), st));
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(csize, st, attr);
    cfg.gridDim = dim3(csize * nclusters, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    CGP_CUDA(cudaLaunchKernelEx(&cfg, k_batch_step, (const BatchStepArgs*)d_args, ninst, queue));
    return CGP_OK;
}

int enqueue_step(Solver* s, cudaStream_t st, bool capture) {
    Ctx c{s, st, capture};
    return step_body(c);
}

static double* vec_ptr(Solver& s, int which, size_t* n) {
    switch (which) {
        case CGP_VEC_U: *n = 2 * (size_t)s.nf; return s.U;
        case CGP_VEC_UPREV: *n = 2 * (size_t)s.nf; return s.Uprev;
        case CGP_VEC_P: *n = s.nf; return s.P;
        case CGP_VEC_UTILDE: *n = 2 * (size_t)s.nf; return s.Ut;
        case CGP_VEC_RHS_C: *n = s.nc; return s.rc;
        case CGP_VEC_PHI_C: *n = s.nc; return s.phi;
        case CGP_VEC_PHI_F: *n = s.nf; return s.phi;
        default: return nullptr;
    }
}

static int copy_out(void* dst, const void* src, size_t bytes, int where, cudaStream_t st) {
    CGP_CUDA(cudaMemcpyAsync(dst, src, bytes, where == CGP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    return CGP_OK;
}

static int copy_in(void* dst, const void* src, size_t bytes, int where, cudaStream_t st) {
    CGP_CUDA(cudaMemcpyAsync(dst, src, bytes, where == CGP_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    return CGP_OK;
}

}  // namespace cgp

using namespace cgp;

extern "C" int cgp_step(cgp_solver* h, int32_t n_steps, cgp_stream_t stream) {
    clear_error();
    if (!h || n_steps < 0) {
        set_error("cgp_step: bad arguments");
        return CGP_EINVAL;
    }
    Solver& s = h->s;
    cudaStream_t st = (cudaStream_t)stream;
    if (s.prm.use_graph) {
        if (!s.step_exec) CGP_TRY(build_graph(s));
        for (int i = 0; i < n_steps; ++i) CGP_CUDA(cudaGraphLaunch(s.step_exec, st));
        return CGP_OK;
    }
    for (int i = 0; i < n_steps; ++i) CGP_TRY(enqueue_step(&s, st, false));
    return CGP_OK;
}

static int set_user_array(cgp_solver* h, double* dst, const double* src, int32_t where, cgp_stream_t stream,
                          const char* name) {
    clear_error();
    if (!h || !src || (where != CGP_HOST && where != CGP_DEVICE)) {
        set_error("%s: bad arguments", name);
        return CGP_EINVAL;
    }
    if (h->s.prm.bc_kind != CGP_BC_USER || !dst) {
        set_error("%s: the solver's bc_kind is not CGP_BC_USER", name);
        return CGP_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CGP_TRY(copy_in(dst, src, sizeof(double) * 2 * h->s.nf, where, st));
    if (where == CGP_HOST) CGP_CUDA(cudaStreamSynchronize(st));
    return CGP_OK;
}

extern "C" int cgp_set_dirichlet(cgp_solver* h, const double* uD, int32_t where, cgp_stream_t stream) {
    return set_user_array(h, h ? h->s.user_ud : nullptr, uD, where, stream, "cgp_set_dirichlet");
}

extern "C" int cgp_set_forcing(cgp_solver* h, const double* F, int32_t where, cgp_stream_t stream) {
    return set_user_array(h, h ? h->s.user_f : nullptr, F, where, stream, "cgp_set_forcing");
}

extern "C" int cgp_record_pairs(cgp_solver* h, int32_t n_steps, double* rhs, double* prev, double* target,
                                int32_t where, cgp_stream_t stream) {
    clear_error();
    if (!h || n_steps < 0 || !rhs || !prev || !target || (where != CGP_HOST && where != CGP_DEVICE)) {
        set_error("cgp_record_pairs: bad arguments");
        return CGP_EINVAL;
    }
    Solver& s = h->s;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nc = s.nc, bytes = sizeof(double) * nc;
    for (int k = 0; k < n_steps; ++k) {
        // the network's second input: the projection guess of the step where the solver forms
        // one (copied during the step), else the increment before the step
        if (!s.proj) CGP_TRY(copy_out(prev + k * nc, s.phi, bytes, where, st));
        CGP_TRY(cgp_step(h, 1, stream));
        if (s.proj) CGP_TRY(copy_out(prev + k * nc, s.phi_q, bytes, where, st));
        CGP_TRY(copy_out(rhs + k * nc, s.rc, bytes, where, st));
        CGP_TRY(copy_out(target + k * nc, s.phi, bytes, where, st));
    }
    if (where == CGP_HOST) CGP_CUDA(cudaStreamSynchronize(st));
    return CGP_OK;
}

extern "C" int cgp_get_fields(cgp_solver* h, double* U, double* P, double* t, cgp_stats* stats, int32_t where,
                              cgp_stream_t stream) {
    clear_error();
    if (!h) {
        set_error("null solver");
        return CGP_EINVAL;
    }
    Solver& s = h->s;
    cudaStream_t st = (cudaStream_t)stream;
    if (U) CGP_TRY(copy_out(U, s.U, sizeof(double) * 2 * s.nf, where, st));
    if (P) CGP_TRY(copy_out(P, s.P, sizeof(double) * s.nf, where, st));
    // stats and time land in pinned host memory (no staged pageable copies)
    CGP_CUDA(cudaMemcpyAsync(&s.h_view->stats, s.stats, sizeof(DeviceStats), cudaMemcpyDeviceToHost, st));
    CGP_CUDA(cudaMemcpyAsync(&s.h_view->t, s.tdev, sizeof(double), cudaMemcpyDeviceToHost, st));
    CGP_CUDA(cudaStreamSynchronize(st));
    const DeviceStats ds = s.h_view->stats;
    const double th = s.h_view->t;
    if (t) *t = th;
    if (stats) {
        stats->steps = ds.steps;
        stats->launches = ds.launches;
        stats->guess_used = ds.guess_used;
        stats->sum_outer_poisson = ds.sum_outer;
        stats->t = th;
        stats->it_mom = ds.last_it[KS_MOM];
        stats->it_poisson = ds.last_it[KS_POIS];
        stats->it_corr = ds.last_it[KS_CORR];
        stats->it_mass = ds.last_it[KS_MASS];
        stats->sum_it_mom = ds.sum_it[KS_MOM];
        stats->sum_it_poisson = ds.sum_it[KS_POIS];
        stats->sum_it_corr = ds.sum_it[KS_CORR];
        stats->sum_it_mass = ds.sum_it[KS_MASS];
        stats->res_mom = ds.res[KS_MOM];
        stats->res_poisson = ds.res[KS_POIS];
        stats->status = ds.status;
    }
    return ds.status;
}

extern "C" int cgp_set_fields(cgp_solver* h, const double* U, const double* Uprev, const double* P, double t,
                              int32_t where, cgp_stream_t stream) {
    clear_error();
    if (!h || !U || !P) {
        set_error("cgp_set_fields: null argument");
        return CGP_EINVAL;
    }
    Solver& s = h->s;
    cudaStream_t st = (cudaStream_t)stream;
    CGP_TRY(copy_in(s.U, U, sizeof(double) * 2 * s.nf, where, st));
    CGP_TRY(copy_in(s.Uprev, Uprev ? Uprev : U, sizeof(double) * 2 * s.nf, where, st));
    CGP_TRY(copy_in(s.P, P, sizeof(double) * s.nf, where, st));
    k_set_time<<<1, 32, 0, st>>>(s.tdev, t, s.stats);
    CGP_LAUNCH_CHECK();
    CGP_CUDA(cudaStreamSynchronize(st));
    return CGP_OK;
}

extern "C" int cgp_get_vector(cgp_solver* h, int32_t which, double* out, int32_t where, cgp_stream_t stream) {
    clear_error();
    if (!h || !out) {
        set_error("cgp_get_vector: null argument");
        return CGP_EINVAL;
    }
    size_t n = 0;
    double* src = vec_ptr(h->s, which, &n);
    if (!src) {
        set_error("unknown vector %d", which);
        return CGP_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CGP_TRY(copy_out(out, src, n * sizeof(double), where, st));
    if (where == CGP_HOST) CGP_CUDA(cudaStreamSynchronize(st));
    return CGP_OK;
}

extern "C" int cgp_profile_step(cgp_solver* h, cgp_stream_t stream, int32_t n_ids, int32_t* counts,
                                double* total_ms) {
    clear_error();
    if (!h || !counts || !total_ms || n_ids < CGP_PROF_COUNT) {
        set_error("cgp_profile_step: bad arguments");
        return CGP_EINVAL;
    }
    Solver& s = h->s;
    cudaStream_t st = (cudaStream_t)stream;
    Prof pr;
    pr.cap = 4096;
    std::vector<cudaEvent_t> ev(2 * pr.cap);
    std::vector<int> ids(pr.cap);
    for (auto& e : ev) CGP_CUDA(cudaEventCreate(&e));
    pr.ev = ev.data();
    pr.id = ids.data();
    Ctx c{&s, st, false, &pr};
    int rc = step_body(c);
    KrylovState ks[KS_COUNT];
    if (rc == CGP_OK) {
        CGP_CUDA(cudaMemcpyAsync(ks, s.ks, sizeof(ks), cudaMemcpyDeviceToHost, st));
        CGP_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < n_ids; ++i) {
            counts[i] = 0;
            total_ms[i] = 0.0;
        }
        // launches of loop kernels after their solve finished returned at once: keep the
        // first `iter` launches of each loop kernel (they run in order)
        auto solve_of = [](int id) {
            if (id >= CGP_PROF_BICG_P && id <= CGP_PROF_BICG_X) return (int)KS_MOM;
            if (id == CGP_PROF_POIS_SPMV || id == CGP_PROF_POIS_UPDATE || id == CGP_PROF_POIS_PUPD) return (int)KS_POIS;
            if (id == CGP_PROF_CORR_SPMV || id == CGP_PROF_CORR_UPDATE || id == CGP_PROF_CORR_PUPD) return (int)KS_CORR;
            if (id == CGP_PROF_MASS_SPMV || id == CGP_PROF_MASS_UPDATE || id == CGP_PROF_MASS_PUPD) return (int)KS_MASS;
            return -1;
        };
        for (int k = 0; k < pr.n; ++k) {
            const int id = pr.id[k];
            const int sv = solve_of(id);
            if (sv >= 0 && counts[id] >= ks[sv].iter) continue;
            float ms = 0.f;
            CGP_CUDA(cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]));
            counts[id] += 1;
            total_ms[id] += ms;
        }
        if (pr.n >= pr.cap) {
            set_error("profile truncated after %d launches", pr.cap);
            rc = CGP_ENOMEM;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return rc;
}

extern "C" int cgp_set_vector(cgp_solver* h, int32_t which, const double* in, int32_t where, cgp_stream_t stream) {
    clear_error();
    if (!h || !in || (which != CGP_VEC_U && which != CGP_VEC_UPREV && which != CGP_VEC_P && which != CGP_VEC_PHI_C)) {
        set_error("cgp_set_vector: bad arguments");
        return CGP_EINVAL;
    }
    size_t n = 0;
    double* dst = vec_ptr(h->s, which, &n);
    cudaStream_t st = (cudaStream_t)stream;
    CGP_TRY(copy_in(dst, in, n * sizeof(double), where, st));
    if (where == CGP_HOST) CGP_CUDA(cudaStreamSynchronize(st));
    return CGP_OK;
}

// closed-form fields of a manufactured problem kind on every fine vertex
__global__ void k_exact_fields(int n, const double* __restrict__ xy, BcParams bc, double t, double* __restrict__ U,
                               double* __restrict__ P) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double u = 0.0, v = 0.0, p = 0.0;
        exact_field(bc, xy[2 * i], xy[2 * i + 1], t, u, v, p);
        if (U) reinterpret_cast<double2*>(U)[i] = make_double2(u, v);
        if (P) P[i] = p;
    }
}

extern "C" int cgp_exact_fields(cgp_solver* h, double t, double* U, double* P, int32_t where, cgp_stream_t stream) {
    clear_error();
    if (!h || (!U && !P) || (where != CGP_HOST && where != CGP_DEVICE)) {
        set_error("cgp_exact_fields: bad arguments");
        return CGP_EINVAL;
    }
    Solver& s = h->s;
    const BcParams bc = bc_of(s);
    if (bc.kind != CGP_BC_TG && bc.kind != CGP_BC_TG_PERIODIC && bc.kind != CGP_BC_JOBELIN_OPEN &&
        bc.kind != CGP_BC_JOBELIN_DISK) {
        set_error("cgp_exact_fields: the problem kind has no closed-form solution");
        return CGP_EINVAL;
    }
    const Level& F = s.mesh->lev[s.lf];
    cudaStream_t st = (cudaStream_t)stream;
    double* dU = U;
    double* dP = P;
    if (where == CGP_HOST) {
        // staged through the extrapolation and history vectors of Eq. 21, which every step
        // forms anew before reading them
        dU = U ? s.w : nullptr;
        dP = P ? s.h : nullptr;
    }
    k_exact_fields<<<grid_rows(s, F.nv, 1), kBlock, 0, st>>>(F.nv, F.xy, bc, t, dU, dP);
    CGP_LAUNCH_CHECK();
    if (where == CGP_HOST) {
        if (U) CGP_CUDA(cudaMemcpyAsync(U, dU, sizeof(double) * 2 * F.nv, cudaMemcpyDeviceToHost, st));
        if (P) CGP_CUDA(cudaMemcpyAsync(P, dP, sizeof(double) * F.nv, cudaMemcpyDeviceToHost, st));
        CGP_CUDA(cudaStreamSynchronize(st));
    }
    return CGP_OK;
}

extern "C" int cgp_set_wait_test(cgp_solver* h, int32_t on) {
    clear_error();
    if (!h) {
        set_error("null solver");
        return CGP_EINVAL;
    }
    h->s.wait_test = on ? 1 : 0;
    return CGP_OK;
}

extern "C" int cgp_coarse_subdomains(const cgp_solver* h, int32_t* nsub) {
    if (!h) {
        set_error("null solver");
        return CGP_EINVAL;
    }
    if (nsub) *nsub = h->s.onchip_bytes ? h->s.onchip.nsub : 0;
    return CGP_OK;
}

extern "C" int cgp_coarse_info(const cgp_solver* h, int32_t* kind, int32_t* ctas, int32_t* cluster) {
    if (!h) {
        set_error("null solver");
        return CGP_EINVAL;
    }
    const Solver& s = h->s;
    int k = s.coarse_kind, n = 0, cl = 0;
    if (k == CGP_COARSE_CLUSTER) {
        n = cl = s.cluster_size;
    } else if (k == CGP_COARSE_PERSISTENT) {
        if (s.onchip_bytes) {
            k = CGP_COARSE_ONCHIP;
            n = cl = s.cluster_size;
        } else if (s.coarse_rr && s.coarse_fp64) {
            n = rr_ctas_needed(s.mesh->lev[s.lc].nslices);
        } else {
            k = CGP_COARSE_PERSISTENT_MEM;
            n = s.coarse_grid;
        }
    }
    if (kind) *kind = k;
    if (ctas) *ctas = n;
    if (cluster) *cluster = cl;
    return CGP_OK;
}

extern "C" int cgp_poisson_solve(cgp_solver* h, const double* rhs, double* phi, int32_t* iters, int32_t where,
                                 cgp_stream_t stream) {
    clear_error();
    if (!h || !rhs || !phi) {
        set_error("cgp_poisson_solve: null argument");
        return CGP_EINVAL;
    }
    Solver& s = h->s;
    cudaStream_t st = (cudaStream_t)stream;
    CGP_TRY(copy_in(s.rc, rhs, sizeof(double) * s.nc, where, st));
    CGP_TRY(copy_in(s.phi, phi, sizeof(double) * s.nc, where, st));
    KrylovState* ks = &s.ks[KS_POIS];
    // range projection of a pure-Neumann problem uses the plain mean of the given rhs
    k_rhs_mean<<<grid_rows(s, s.nc, 1), kBlock, 0, st>>>(s.nc, s.rc, ks, s.pure_neumann, s.partials, s.tickets);
    CGP_LAUNCH_CHECK();
    Ctx c{&s, st, false};
    CGP_TRY(coarse_solve(c));
    CGP_TRY(copy_out(phi, s.phi, sizeof(double) * s.nc, where, st));
    int it = 0, status = 0;
    CGP_CUDA(cudaMemcpyAsync(&it, &ks->iter, sizeof(int), cudaMemcpyDeviceToHost, st));
    CGP_CUDA(cudaMemcpyAsync(&status, &ks->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CGP_CUDA(cudaStreamSynchronize(st));
    if (iters) *iters = it;
    return status;
}

extern "C" int cgp_prolong(cgp_solver* h, const double* phi_c, double* phi_f, int32_t where, cgp_stream_t stream) {
    clear_error();
    if (!h || !phi_c || !phi_f) {
        set_error("cgp_prolong: null argument");
        return CGP_EINVAL;
    }
    Solver& s = h->s;
    cudaStream_t st = (cudaStream_t)stream;
    CGP_TRY(copy_in(s.phi, phi_c, sizeof(double) * s.nc, where, st));
    Ctx c{&s, st, false};
    CGP_TRY(prolong_all(c));
    CGP_TRY(copy_out(phi_f, s.phi, sizeof(double) * s.nf, where, st));
    if (where == CGP_HOST) CGP_CUDA(cudaStreamSynchronize(st));
    return CGP_OK;
}
