// Row i of the momentum system of Eq. 21 (shared by the step's kernel and the batched
// whole-step kernel):
//   A = 3/2 M + dt N(w) + dt/Re K,  N_ij = sum_T |T|/12 (W_T + w_i) . grad psi_j
//   b = dt (Cx^T P, Cy^T P) + M h     (pressure term in weak form, see the readings)
// Dirichlet rows: s_ii times the identity row, b = s_ii u_D(t^{n+1}), with s_ii the diagonal
// of S = 3/2 M + dt/Re K at that row: the same solution as the plain identity row, but rows
// of one scale, so that the relative residual test ||b - A x|| <= tol ||b|| measures the
// interior equations (with identity rows the O(1) boundary values dominate ||b|| against
// interior rows of the size of the mass matrix, O(h^2), and the test passes while the
// interior equations hold only to ~1e-4).  Also x0 = w (u_D on Dirichlet rows), dinv.
// With kShared, rows of at most kAsmRow entries are accumulated in the calling thread's
// column of arow ([entry][thread], so the lanes of a warp hit distinct banks) and written to
// A once; otherwise (and for longer rows) the entries add into A directly.
#pragma once

#include "flows.cuh"

namespace cgp {

constexpr int kAsmRow = 16;

template <bool kShared>
__device__ __forceinline__ void mom_assemble_row(
    int i, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, const int32_t* __restrict__ sell_ptr,
    const int32_t* __restrict__ vt_ptr, const int32_t* __restrict__ vt_list, const int32_t* __restrict__ tri,
    const double* __restrict__ geo, const int32_t* __restrict__ vtslot, const double* __restrict__ S,
    const double* __restrict__ M, const double* __restrict__ CxT, const double* __restrict__ CyT,
    const double* __restrict__ P, const double* __restrict__ w, const double* __restrict__ h,
    const uint8_t* __restrict__ tag, const double* __restrict__ xy, const BcParams& bc, double tn, double dt,
    double* __restrict__ A, double* __restrict__ dinv, double* __restrict__ b, double* __restrict__ x0,
    double (*arow)[kBlock]) {
    const int rb = rowptr[i], re = rowptr[i + 1];
    const int64_t e0 = sell_pos(sell_ptr, i, 0);   // entry k of the row is at e0 + 32 k
    const bool local = kShared && re - rb <= kAsmRow;
    if (tag[i] & CGP_VEL_DIR) {
        double sii = 1.0;
        for (int q = rb; q < re; ++q)
            if (col[q] == i) sii = S[e0 + 32 * (q - rb)];
        if (!(sii > 0.0)) sii = 1.0;
        for (int q = rb; q < re; ++q) A[e0 + 32 * (q - rb)] = col[q] == i ? sii : 0.0;
        dinv[i] = 1.0 / sii;
        double u, v;
        dirichlet_value(bc, i, xy[2 * i], xy[2 * i + 1], tn, u, v);
        reinterpret_cast<double2*>(b)[i] = make_double2(sii * u, sii * v);
        reinterpret_cast<double2*>(x0)[i] = make_double2(u, v);
        return;
    }
    double bx = 0.0, by = 0.0;
    for (int q = rb; q < re; ++q) {
        const int64_t e = e0 + 32 * (q - rb);
        if (local)
            arow[q - rb][threadIdx.x] = S[e];
        else
            A[e] = S[e];
        const int j = col[q];
        const double2 hj = reinterpret_cast<const double2*>(h)[j];
        const double pj = P[j];
        bx += dt * CxT[e] * pj + M[e] * hj.x;
        by += dt * CyT[e] * pj + M[e] * hj.y;
    }
    const double2 wi = reinterpret_cast<const double2*>(w)[i];
    int diag_slot = 0;
    for (int m = vt_ptr[i]; m < vt_ptr[i + 1]; ++m) {
        const int t = vt_list[m];
        const int packed = vtslot[m];
        const double* gt = geo + 7 * (int64_t)t;
        const int a0 = tri[3 * t], a1 = tri[3 * t + 1], a2 = tri[3 * t + 2];
        const double2 w0 = reinterpret_cast<const double2*>(w)[a0];
        const double2 w1 = reinterpret_cast<const double2*>(w)[a1];
        const double2 w2 = reinterpret_cast<const double2*>(w)[a2];
        const double c = gt[0] * (1.0 / 12.0);
        const double cx = c * (w0.x + w1.x + w2.x + wi.x), cy = c * (w0.y + w1.y + w2.y + wi.y);
        const int li = packed & 3;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int slot = (packed >> (8 * (k + 1))) & 255;
            const double v = dt * (cx * gt[1 + 2 * k] + cy * gt[2 + 2 * k]);
            if (local)
                arow[slot][threadIdx.x] += v;
            else
                A[e0 + 32 * slot] += v;
            if (k == li) diag_slot = slot;
        }
    }
    if (local) {
        for (int q = 0; q < re - rb; ++q) A[e0 + 32 * q] = arow[q][threadIdx.x];
        dinv[i] = 1.0 / arow[diag_slot][threadIdx.x];
    } else {
        dinv[i] = 1.0 / A[e0 + 32 * diag_slot];
    }
    if ((tag[i] & CGP_PHI_ZERO) && has_natural_data(bc)) {
        // traction boundary (Eq. 11 at t^{n+1}: -p^{n+1} n + grad u~ . n / Re = t, with the
        // prescribed p^{n+1}; the weak pressure term above carries P^n): dt int_{Gamma_N}
        // (t + (p^{n+1} - P^n) n) psi_i ds over the boundary edges (i, j), j on Gamma_N
        // too, an edge being on the boundary when one triangle has it; the integrand linear
        // on the edge: l/6 (2 t_i + t_j)
        auto tr = [&](int v, double& tx, double& ty) {
            const double xv = xy[2 * v], yv = xy[2 * v + 1];
            double nx, ny;
            natural_traction(bc, xv, yv, tn, tx, ty);
            natural_normal(bc, xv, yv, nx, ny);
            const double dp = natural_pressure(bc, xv, yv, tn) - P[v];
            tx += dp * nx;
            ty += dp * ny;
        };
        const double xi = xy[2 * i], yi = xy[2 * i + 1];
        double ti_x, ti_y;
        tr(i, ti_x, ti_y);
        for (int q = rb; q < re; ++q) {
            const int j = col[q];
            if (j == i || !(tag[j] & CGP_PHI_ZERO)) continue;
            int owners = 0;
            for (int m = vt_ptr[i]; m < vt_ptr[i + 1]; ++m) {
                const int t = vt_list[m];
                owners += (tri[3 * t] == j) + (tri[3 * t + 1] == j) + (tri[3 * t + 2] == j);
            }
            if (owners != 1) continue;
            const double xj = xy[2 * j], yj = xy[2 * j + 1];
            double tj_x, tj_y;
            tr(j, tj_x, tj_y);
            const double c = dt * hypot(xj - xi, yj - yi) / 6.0;
            bx += c * (2.0 * ti_x + tj_x);
            by += c * (2.0 * ti_y + tj_y);
        }
    }
    reinterpret_cast<double2*>(b)[i] = make_double2(bx, by);
    reinterpret_cast<double2*>(x0)[i] = wi;
}

}  // namespace cgp
