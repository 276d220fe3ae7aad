// The whole CGP step of many independent instances in ONE persistent launch (a form beyond
// the paper).  Every thread-block cluster of the launch takes instances from a queue (the
// host orders them largest first) and advances each by one complete step of Eqs. 21-26;
// the cluster's CTAs share the rows, reduce through distributed shared memory, and
// synchronise with the hardware cluster barrier between phases; clusters never wait on one
// another.
//
//   Eq. 21     the rows of the momentum system (step_rows.cuh), then BiCGStab with Jacobi
//              for both velocity components (three cluster sums per iteration; restarted from
//              the true residual after a breakdown): FP64, or for a mixed instance FP32 inner
//              solves inside FP64 refinement, then FP64 only if the sweeps fell short
//   Eqs. 22-23 the injected coarse right-hand side (with the range projection of a
//              pure-Neumann problem and the lifted phi data of a traction boundary), then the
//              instance's one-launch coarse PCG (coarse_pcg_body: FP64, or FP32 inner / FP64
//              outer, as the instance is assembled)
//   Eq. 24     prolongation, level by level
//   Eq. 25     the correction's right-hand side and, with the consistent mass, Chebyshev
//              semi-iteration on M0 with Jacobi: the eigenvalues of D^-1 M of P1 triangles lie
//              in [1/2, 2] (every element matrix D_e^-1 M_e has eigenvalues 1/2, 1/2, 2), so the
//              steps need no inner products and their number follows from the tolerance
//              (error <= 4 * 3^-n of the initial one in the energy norm)
//   Eq. 26     the rotational term (D U~, and the same Chebyshev solve on M) and the update
// In a mixed instance the momentum BiCGStab's inner iterations run in FP32: on this GPU the
// narrow FP64 pipe is the busiest unit of the cluster's FP64 iterations.
#pragma once

#include <cooperative_groups.h>

#include "coarse_pcg.cuh"
#include "solver.cuh"
#include "step_rows.cuh"

namespace cgp {

namespace cgrp_bs = cooperative_groups;

// everything one instance's step reads and writes (device pointers into its solver)
struct BatchStepArgs {
    // fine level
    int nf;
    SellView Af;
    const int32_t *rowptr, *col, *sell_ptr, *vt_ptr, *vt_list, *tri, *vtslot;
    const double *geo, *xy, *S, *M, *M0, *CxT, *CyT, *Cx, *Cy, *dinvM0, *dinvM, *mlumpF;
    const uint8_t* tag;
    double *U, *Uprev, *P, *Ut, *w, *h, *A, *dinvA, *b, *g, *delta, *div, *qrot, *phi;
    BicgVecs bv;
    double *c0, *c1, *c2;   // Chebyshev work: residual, two directions (2 nf each)
    // mixed instances (null otherwise): FP32 copies of A (refreshed each step) and its Jacobi
    // diagonal, FP32 work vectors (2 nf each); the momentum solve then runs FP32 inner solves
    // inside FP64 refinement
    int64_t nnz;
    float *A32, *dinvA32;
    float* fv[10];
    // coarse level and its solve
    SellView Ac;
    const double *Cxc, *Cyc, *Kc, *cxy;
    const uint8_t* ctag;
    CoarsePcgArgs coarse;
    int pure_neumann;
    // prolongation: levels lc .. lf
    int nlev;
    int nv[5];
    const int32_t* parents[5];   // parents[l]: end points of the vertices added at level lc + l + 1
    // parameters
    BcParams bc;
    double dt, inv_re, tol_mom2;
    int chi, lumped, max_it_mom, cheb_steps;
    double* tdev;
    DeviceStats* stats;
    KrylovState* ks;
};

// deterministic cluster-wide sums of up to 8 values (warp -> CTA -> every CTA's slot array ->
// each CTA adds the slots in rank order); two slot sets alternate, and every sum ends with a
// cluster barrier, so a slot is rewritten only after every CTA read it
struct ClusterSum8 {
    cgrp_bs::cluster_group cl;
    double (*slots)[8];
    double (*wsum)[8];
    double* bcast;
    int slot = 0;
    __device__ ClusterSum8(double (*sl)[8], double (*ws)[8], double* bc)
        : cl(cgrp_bs::this_cluster()), slots(sl), wsum(ws), bcast(bc) {}
    template <int NR>
    __device__ void sum(const double (&v)[NR], double (&tot)[NR]) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            const double s = warp_sum(v[k]);
            if (lane == 0) wsum[wid][k] = s;
        }
        __syncthreads();
        if (wid == 0) {
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const double s = warp_sum(lane < nw ? wsum[lane][k] : 0.0);
                if (lane == 0) slots[slot][k] = s;
            }
        }
        cl.sync();
        if (wid == 0) {
            const int ncl = (int)cl.num_blocks();
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const double s = warp_sum(lane < ncl ? cl.map_shared_rank(&slots[slot][0], lane)[k] : 0.0);
                if (lane == 0) bcast[k] = s;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NR; ++k) tot[k] = bcast[k];
        slot ^= 1;
    }
};

// number of Chebyshev steps for a relative energy-norm error tol with eigenvalue bounds
// [1/2, 2] (condition 4): 4 * 3^-n <= tol
__host__ __device__ inline int cheb_steps_for(double tol) {
    int n = 1;
    double bound = 4.0 / 3.0;
    while (bound > tol && n < 200) {
        bound /= 3.0;
        ++n;
    }
    return n;
}

// Mixed instances: the momentum system runs up to kBatchIrSweeps FP64-residual sweeps around
// an FP32 BiCGStab (each asked for kBatchInnerTol of its right-hand side, or what is left to
// the tolerance), then the FP64 BiCGStab unless a sweep's residual already met the tolerance.
constexpr int kBatchIrSweeps = 3;
constexpr double kBatchInnerTol = 1e-4;
constexpr int kBatchInnerMaxit = 200;

// Chebyshev semi-iteration for B x = rhs (NC interleaved components), x = 0 at the start;
// Jacobi preconditioning, bounds [1/2, 2] of D^-1 B; one cluster barrier per step.  (It stays
// FP64 in mixed instances too: FP32 sweeps inside FP64 refinement took longer here, the
// cluster's steps being bound by latency rather than by the FP64 pipe.)
template <int NC, class T = double>
__device__ void cluster_chebyshev(const SellView& B, const T* __restrict__ val, const T* __restrict__ dinv,
                                  const T* __restrict__ rhs, T* __restrict__ x, T* __restrict__ r,
                                  T* __restrict__ d0, T* __restrict__ d1, int steps, int crank, int csize,
                                  cgrp_bs::cluster_group& cl) {
    const double theta = 1.25, delta = 0.75, sigma = theta / delta;
    const int n = B.n, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5, wid = threadIdx.x >> 5;
    for (int i = crank * blockDim.x + threadIdx.x; i < n; i += csize * blockDim.x) {
        const T di = dinv[i];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const T ri = rhs[NC * i + c];
            x[NC * i + c] = T(0);
            r[NC * i + c] = ri;
            d0[NC * i + c] = di * ri / T(theta);
        }
    }
    cl.sync();
    double rho = 1.0 / sigma;
    T* dc = d0;
    T* dn = d1;
    for (int k = 0; k < steps; ++k) {
        const double rho_n = 1.0 / (2.0 * sigma - rho);
        const T c1 = (T)(rho_n * rho), c2 = (T)(2.0 * rho_n / delta);
        for (int sl = crank * nwarp + wid; sl < B.nslices; sl += csize * nwarp) {
            const int i = sl * 32 + lane;
            T wv[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) wv[c] = T(0);
            sell_accum<NC>(B, val, sl, lane, [&](int j, T (&o)[NC]) {
#pragma unroll
                for (int c = 0; c < NC; ++c) o[c] = dc[NC * j + c];
            }, wv);
            if (i < n) {
                const T di = dinv[i];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const T dd = dc[NC * i + c];
                    x[NC * i + c] += dd;
                    const T rn = r[NC * i + c] - wv[c];
                    r[NC * i + c] = rn;
                    dn[NC * i + c] = c1 * dd + c2 * di * rn;
                }
            }
        }
        cl.sync();
        rho = rho_n;
        T* t = dc;
        dc = dn;
        dn = t;
    }
}

// BiCGStab with Jacobi for the two velocity components of one instance, on its cluster.  T:
// FP64, or FP32 for the inner solve of a refinement sweep (its per-thread partial sums are then
// FP32, the cluster sums FP64).  x starts from V.x, or from 0 with zero_x.  A breakdown (rho or
// omega vanishing before convergence) restarts from the true residual, at most `restarts`
// times.  Converged when <r, r> <= tol2 <b, b> for each component.  Returns the iterations;
// status, the last <r, r> and <b, b> go out.
template <class T>
__device__ int cluster_bicgstab(const SellView& A, const T* __restrict__ val, const T* __restrict__ dinv,
                                const T* __restrict__ b, const BicgVecsT<T>& V, double tol2, int maxit, int restarts,
                                bool zero_x, ClusterSum8& cs, cgrp_bs::cluster_group& cl, int crank, int csize,
                                int& status, double (&rr)[2], double (&bb)[2]) {
    const int n = A.n, lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int tid = crank * blockDim.x + threadIdx.x, nthr = csize * blockDim.x;
    double rho[2] = {0.0, 0.0}, alpha[2] = {0.0, 0.0}, omega[2] = {0.0, 0.0}, beta[2] = {0.0, 0.0};
    int done[2] = {0, 0}, it = 0;
    status = 0;
    for (int restart = 0; restart <= restarts; ++restart) {
        {   // r = b - A x, rhat = r, p = v = 0
            const bool zx = zero_x && restart == 0;
            T acc[4] = {T(0), T(0), T(0), T(0)};
            for (int sl = crank * nwarp + wid; sl < A.nslices; sl += csize * nwarp) {
                const int i = sl * 32 + lane;
                T ax[2] = {T(0), T(0)};
                if (!zx) spmv2_row(A, val, V.x, sl, lane, ax);
                if (i < n) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const T bv = b[2 * i + c], rv = bv - ax[c];
                        if (zx) V.x[2 * i + c] = T(0);
                        V.r[2 * i + c] = rv;
                        V.rhat[2 * i + c] = rv;
                        V.p[2 * i + c] = T(0);
                        V.v[2 * i + c] = T(0);
                        acc[c] += rv * rv;
                        acc[2 + c] += bv * bv;
                    }
                }
            }
            const double accd[4] = {(double)acc[0], (double)acc[1], (double)acc[2], (double)acc[3]};
            double tot[4];
            cs.sum(accd, tot);
            for (int c = 0; c < 2; ++c) {
                rho[c] = tot[c];
                rr[c] = tot[c];
                if (restart == 0) bb[c] = tot[2 + c];
                done[c] = !(rr[c] > tol2 * bb[c]);
                alpha[c] = omega[c] = beta[c] = 0.0;
            }
        }
        bool broke = false;
        while (!(done[0] && done[1]) && it < maxit && !broke) {
            // p = r + beta (p - omega v), y = D^-1 p
            for (int i = tid; i < n; i += nthr) {
                const T di = dinv[i];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (done[c]) continue;
                    const T pv = V.r[2 * i + c] + (T)beta[c] * (V.p[2 * i + c] - (T)omega[c] * V.v[2 * i + c]);
                    V.p[2 * i + c] = pv;
                    V.y[2 * i + c] = di * pv;
                }
            }
            cl.sync();
            {   // v = A y, alpha = rho / <rhat, v>
                T acc[2] = {T(0), T(0)};
                for (int sl = crank * nwarp + wid; sl < A.nslices; sl += csize * nwarp) {
                    const int i = sl * 32 + lane;
                    T ax[2];
                    spmv2_row(A, val, V.y, sl, lane, ax);
                    if (i < n) {
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            if (done[c]) continue;
                            V.v[2 * i + c] = ax[c];
                            acc[c] += V.rhat[2 * i + c] * ax[c];
                        }
                    }
                }
                const double accd[2] = {(double)acc[0], (double)acc[1]};
                double tot[2];
                cs.sum(accd, tot);
                for (int c = 0; c < 2; ++c) {
                    if (done[c]) continue;
                    if (!isfinite(tot[c])) {
                        done[c] = 1;
                        status = CGP_ENONFINITE;
                    } else if (tot[c] != 0.0) {
                        alpha[c] = rho[c] / tot[c];
                    } else {
                        broke = true;
                    }
                }
            }
            if (broke) break;
            // s = r - alpha v, z = D^-1 s
            for (int i = tid; i < n; i += nthr) {
                const T di = dinv[i];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (done[c]) continue;
                    const T sv = V.r[2 * i + c] - (T)alpha[c] * V.v[2 * i + c];
                    V.s[2 * i + c] = sv;
                    V.z[2 * i + c] = di * sv;
                }
            }
            cl.sync();
            {   // t = A z, omega = <t, s> / <t, t>
                T acc[4] = {T(0), T(0), T(0), T(0)};
                for (int sl = crank * nwarp + wid; sl < A.nslices; sl += csize * nwarp) {
                    const int i = sl * 32 + lane;
                    T ax[2];
                    spmv2_row(A, val, V.z, sl, lane, ax);
                    if (i < n) {
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            if (done[c]) continue;
                            V.t[2 * i + c] = ax[c];
                            acc[c] += ax[c] * V.s[2 * i + c];
                            acc[2 + c] += ax[c] * ax[c];
                        }
                    }
                }
                const double accd[4] = {(double)acc[0], (double)acc[1], (double)acc[2], (double)acc[3]};
                double tot[4];
                cs.sum(accd, tot);
                for (int c = 0; c < 2; ++c)
                    omega[c] = (!done[c] && tot[2 + c] > 0.0 && isfinite(tot[2 + c])) ? tot[c] / tot[2 + c] : 0.0;
            }
            {   // x += alpha y + omega z, r = s - omega t, <rhat, r>, <r, r>
                T acc[4] = {T(0), T(0), T(0), T(0)};
                for (int i = tid; i < n; i += nthr) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        if (done[c]) continue;
                        V.x[2 * i + c] += (T)alpha[c] * V.y[2 * i + c] + (T)omega[c] * V.z[2 * i + c];
                        const T rv = V.s[2 * i + c] - (T)omega[c] * V.t[2 * i + c];
                        V.r[2 * i + c] = rv;
                        acc[c] += V.rhat[2 * i + c] * rv;
                        acc[2 + c] += rv * rv;
                    }
                }
                const double accd[4] = {(double)acc[0], (double)acc[1], (double)acc[2], (double)acc[3]};
                double tot[4];
                cs.sum(accd, tot);
                for (int c = 0; c < 2; ++c) {
                    if (done[c]) continue;
                    if (!isfinite(tot[c]) || !isfinite(tot[2 + c])) {
                        status = CGP_ENONFINITE;
                        done[c] = 1;
                        continue;
                    }
                    rr[c] = tot[2 + c];
                    if (rr[c] <= tol2 * bb[c]) {
                        done[c] = 1;
                    } else if (omega[c] == 0.0 || tot[c] == 0.0) {
                        broke = true;
                    } else {
                        beta[c] = (tot[c] / rho[c]) * (alpha[c] / omega[c]);
                        rho[c] = tot[c];
                    }
                }
            }
            ++it;
        }
        if (!broke) break;
        if (restart == restarts) status = CGP_EBREAKDOWN;
    }
    if (!(done[0] && done[1]) && !status) status = CGP_ENOTCONV;
    return it;
}

static __global__ void __launch_bounds__(512, 1) k_batch_step(const BatchStepArgs* __restrict__ args,
                                                                         int ninst, unsigned int* queue) {
    __shared__ double slots4[2][4];
    __shared__ double wsum4[kClusterThreads / 32][4];
    __shared__ double slots8[2][8];
    __shared__ double wsum8[kClusterThreads / 32][8];
    __shared__ double bcast8[8];
    __shared__ int job;
    ClusterSync sy(slots4, wsum4);
    ClusterSum8 cs(slots8, wsum8, bcast8);
    cgrp_bs::cluster_group& cl = sy.cluster;
    const int crank = (int)cl.block_rank(), csize = (int)cl.num_blocks();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int tid = crank * blockDim.x + threadIdx.x, nthr = csize * blockDim.x;
    for (;;) {
        if (crank == 0 && threadIdx.x == 0) job = (int)atomicAdd(queue, 1u);
        cl.sync();
        const int jb = *cl.map_shared_rank(&job, 0);
        cl.sync();   // every CTA has read rank 0's job before it can change
        if (jb >= ninst) break;
        const BatchStepArgs& a = args[jb];
        const int nf = a.nf;
        const double dt = a.dt, tn = *a.tdev + dt;
        const BcParams bc = a.bc;
        // ---- Eq. 21: w = 2 U^n - U^{n-1}, h = dt F + 2 U^n - 1/2 U^{n-1}
        for (int i = tid; i < nf; i += nthr) {
            const double2 u = reinterpret_cast<const double2*>(a.U)[i];
            const double2 up = reinterpret_cast<const double2*>(a.Uprev)[i];
            double fx = 0.0, fy = 0.0;
            body_force(bc, i, a.xy[2 * i], a.xy[2 * i + 1], tn, fx, fy);
            reinterpret_cast<double2*>(a.w)[i] = make_double2(2.0 * u.x - up.x, 2.0 * u.y - up.y);
            reinterpret_cast<double2*>(a.h)[i] =
                make_double2(dt * fx + (2.0 * u.x - 0.5 * up.x), dt * fy + (2.0 * u.y - 0.5 * up.y));
        }
        cl.sync();
        for (int i = tid; i < nf; i += nthr)
            mom_assemble_row<false>(i, a.rowptr, a.col, a.sell_ptr, a.vt_ptr, a.vt_list, a.tri, a.geo, a.vtslot, a.S,
                                    a.M, a.CxT, a.CyT, a.P, a.w, a.h, a.tag, a.xy, bc, tn, dt, a.A, a.dinvA, a.b,
                                    a.Ut, nullptr);
        cl.sync();
        // ---- the momentum solve (two components), x = U~ from w.  Mixed instances: FP64
        // residual sweeps around an FP32 BiCGStab on the FP32 copy of A, then the FP64
        // BiCGStab unless a sweep's residual met the tolerance; FP64 instances: the FP64
        // BiCGStab alone (a breakdown restarts it from the true residual, at most 4 times).
        const BicgVecs V = a.bv;
        double rr[2] = {0.0, 0.0}, bb[2] = {0.0, 0.0};
        int it = 0, status = 0;
        bool polish = true;
        if (a.A32) {
            for (int64_t e = tid; e < a.nnz; e += nthr) a.A32[e] = (float)a.A[e];
            for (int i = tid; i < nf; i += nthr) a.dinvA32[i] = (float)a.dinvA[i];
            cl.sync();
            const BicgVecsT<float> W{a.fv[0], a.fv[1], a.fv[2], a.fv[3], a.fv[4], a.fv[5], a.fv[6], a.fv[7], a.fv[8]};
            float* r32 = a.fv[9];
            for (int sw = 0; sw < kBatchIrSweeps; ++sw) {
                double acc[4] = {0.0, 0.0, 0.0, 0.0};
                for (int sl = crank * nwarp + wid; sl < a.Af.nslices; sl += csize * nwarp) {
                    const int i = sl * 32 + lane;
                    double ax[2];
                    spmv2_row(a.Af, a.A, V.x, sl, lane, ax);
                    if (i < nf) {
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            const double bv = a.b[2 * i + c], rv = bv - ax[c];
                            r32[2 * i + c] = (float)rv;
                            acc[c] += rv * rv;
                            acc[2 + c] += bv * bv;
                        }
                    }
                }
                double tot[4];
                cs.sum(acc, tot);
                if (sw == 0) {
                    bb[0] = tot[2];
                    bb[1] = tot[3];
                }
                rr[0] = tot[0];
                rr[1] = tot[1];
                if (!isfinite(tot[0]) || !isfinite(tot[1])) break;   // the FP64 solve reports it
                if (rr[0] <= a.tol_mom2 * bb[0] && rr[1] <= a.tol_mom2 * bb[1]) {
                    polish = false;
                    break;
                }
                // the inner solve aims at kBatchInnerTol, or at what is left to the tolerance
                // (a factor 2 of margin in the norm) when that is less
                double t2 = kBatchInnerTol * kBatchInnerTol, need = 1.0;
                for (int c = 0; c < 2; ++c)
                    if (rr[c] > a.tol_mom2 * bb[c]) need = fmin(need, 0.25 * a.tol_mom2 * bb[c] / rr[c]);
                t2 = fmax(t2, need);
                int st_in = 0;
                double rr_in[2], bb_in[2];
                it += cluster_bicgstab<float>(a.Af, a.A32, a.dinvA32, r32, W, t2, kBatchInnerMaxit, 0, true, cs, cl,
                                              crank, csize, st_in, rr_in, bb_in);
                if (st_in == CGP_ENONFINITE) break;
                for (int i = tid; i < nf; i += nthr) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) V.x[2 * i + c] += (double)W.x[2 * i + c];
                }
                cl.sync();
            }
        }
        if (polish) {
            double bb64[2];
            it += cluster_bicgstab<double>(a.Af, a.A, a.dinvA, a.b, V, a.tol_mom2, a.max_it_mom, 4, false, cs, cl, crank,
                                           csize, status, rr, bb64);
            bb[0] = bb64[0];
            bb[1] = bb64[1];
        }
        // ---- Eqs. 22-23: r = -3/(2 dt) (Cx_c u~ + Cy_c v~) at the coarse vertices (the fine
        // prefix); phi data on PHI_ZERO vertices (zero, or lifted for a traction boundary)
        {
            const bool lift = has_natural_data(bc);
            double acc[1] = {0.0};
            for (int sl = crank * nwarp + wid; sl < a.Ac.nslices; sl += csize * nwarp) {
                const int i = sl * 32 + lane;
                double sx[1] = {0.0}, syv[1] = {0.0}, sk[1] = {0.0};
                sell_accum<1>(a.Ac, a.Cxc, sl, lane, [&](int j, double (&o)[1]) { o[0] = a.Ut[2 * j]; }, sx);
                sell_accum<1>(a.Ac, a.Cyc, sl, lane, [&](int j, double (&o)[1]) { o[0] = a.Ut[2 * j + 1]; }, syv);
                auto gN = [&](int j) { return natural_pressure(bc, a.cxy[2 * j], a.cxy[2 * j + 1], tn) - a.P[j]; };
                if (lift)
                    sell_accum<1>(a.Ac, a.Kc, sl, lane,
                                  [&](int j, double (&o)[1]) { o[0] = (a.ctag[j] & CGP_PHI_ZERO) ? gN(j) : 0.0; }, sk);
                if (i < a.Ac.n) {
                    double r;
                    if (a.ctag[i] & CGP_PHI_ZERO) r = lift ? gN(i) : 0.0;
                    else r = -1.5 / dt * (sx[0] + syv[0]) - sk[0];
                    a.coarse.b[i] = r;
                    acc[0] += r;
                }
            }
            double tot[1];
            cs.sum(acc, tot);
            if (crank == 0 && threadIdx.x == 0) a.ks[KS_POIS].mean = a.pure_neumann ? tot[0] / a.Ac.n : 0.0;
            cl.sync();
        }
        coarse_pcg_body(a.coarse, sy);   // ends with a cluster barrier
        // ---- Eq. 24: prolongation, one level after the other
        for (int l = 0; l + 1 < a.nlev; ++l) {
            const int nc_l = a.nv[l], n_new = a.nv[l + 1] - a.nv[l];
            const int2* pr = reinterpret_cast<const int2*>(a.parents[l]);
            for (int e = tid; e < n_new; e += nthr) {
                const int2 p2 = pr[e];
                a.phi[nc_l + e] = 0.5 * (a.phi[p2.x] + a.phi[p2.y]);
            }
            cl.sync();
        }
        // ---- Eq. 25: g = -2/3 dt (Cx phi, Cy phi) off the Dirichlet rows; the correction
        for (int sl = crank * nwarp + wid; sl < a.Af.nslices; sl += csize * nwarp) {
            const int i = sl * 32 + lane;
            double ax[1] = {0.0}, ay[1] = {0.0};
            sell_accum<1>(a.Af, a.Cx, sl, lane, [&](int j, double (&o)[1]) { o[0] = a.phi[j]; }, ax);
            sell_accum<1>(a.Af, a.Cy, sl, lane, [&](int j, double (&o)[1]) { o[0] = a.phi[j]; }, ay);
            if (i < nf) {
                const double c = -2.0 / 3.0 * dt;
                const double2 gv = (a.tag[i] & CGP_VEL_DIR) ? make_double2(0.0, 0.0) : make_double2(c * ax[0], c * ay[0]);
                reinterpret_cast<double2*>(a.g)[i] = gv;
                if (a.lumped) reinterpret_cast<double2*>(a.delta)[i] = make_double2(gv.x / a.mlumpF[i], gv.y / a.mlumpF[i]);
            }
        }
        cl.sync();
        if (!a.lumped)
            cluster_chebyshev<2>(a.Af, a.M0, a.dinvM0, a.g, a.delta, a.c0, a.c1, a.c2, a.cheb_steps, crank, csize, cl);
        // ---- Eq. 26: the rotational term q with M q = D U~ (or its lumped form)
        if (a.chi) {
            for (int sl = crank * nwarp + wid; sl < a.Af.nslices; sl += csize * nwarp) {
                const int i = sl * 32 + lane;
                double sx[1] = {0.0}, syv[1] = {0.0};
                sell_accum<1>(a.Af, a.Cx, sl, lane, [&](int j, double (&o)[1]) { o[0] = a.Ut[2 * j]; }, sx);
                sell_accum<1>(a.Af, a.Cy, sl, lane, [&](int j, double (&o)[1]) { o[0] = a.Ut[2 * j + 1]; }, syv);
                if (i < nf) {
                    const double s = sx[0] + syv[0];
                    a.div[i] = s;
                    if (a.lumped) a.qrot[i] = s / a.mlumpF[i];
                }
            }
            cl.sync();
            if (!a.lumped)
                cluster_chebyshev<1>(a.Af, a.M, a.dinvM, a.div, a.qrot, a.c0, a.c1, a.c2, a.cheb_steps, crank, csize,
                                     cl);
        }
        // ---- end of the step
        for (int i = tid; i < nf; i += nthr) {
            const double2 u = reinterpret_cast<const double2*>(a.U)[i];
            const double2 ut = reinterpret_cast<const double2*>(a.Ut)[i];
            const double2 d = reinterpret_cast<const double2*>(a.delta)[i];
            reinterpret_cast<double2*>(a.Uprev)[i] = u;
            reinterpret_cast<double2*>(a.U)[i] = make_double2(ut.x + d.x, ut.y + d.y);
            double p = a.P[i] + a.phi[i];
            if (a.chi) p -= a.inv_re * a.qrot[i];
            a.P[i] = p;
        }
        if (crank == 0 && threadIdx.x == 0) {
            *a.tdev = tn;
            KrylovState* ks = a.ks;
            ks[KS_MOM].iter = it;
            ks[KS_MOM].rr[0] = rr[0];
            ks[KS_MOM].rr[1] = rr[1];
            ks[KS_MOM].bb[0] = bb[0];
            ks[KS_MOM].bb[1] = bb[1];
            ks[KS_MOM].status = status;
            DeviceStats* st = a.stats;
            st->steps += 1;
            st->sum_outer += ks[KS_POIS].pad[0];
            const int its[KS_COUNT] = {it, ks[KS_POIS].iter, a.lumped ? 0 : a.cheb_steps,
                                       (a.chi && !a.lumped) ? a.cheb_steps : 0};
            for (int k = 0; k < KS_COUNT; ++k) {
                st->last_it[k] = its[k];
                st->sum_it[k] += its[k];
            }
            st->res[KS_MOM] = fmax(bb[0] > 0.0 ? sqrt(rr[0] / bb[0]) : 0.0, bb[1] > 0.0 ? sqrt(rr[1] / bb[1]) : 0.0);
            st->res[KS_POIS] = ks[KS_POIS].bb[0] > 0.0 ? sqrt(ks[KS_POIS].rr[0] / ks[KS_POIS].bb[0]) : 0.0;
            if (!st->status && status) st->status = status;
            if (!st->status && ks[KS_POIS].status) st->status = ks[KS_POIS].status;
        }
        cl.sync();   // the instance's vectors are complete before the cluster takes the next one
    }
}

}  // namespace cgp
