// Problem statements evaluated on the device: Dirichlet velocity data, body force and
// closed-form fields of the built-in problem kinds (paper Eqs. 3, 28-30; cgp.h CGP_BC_*).
#pragma once

#include "internal.cuh"

namespace cgp {

struct BcParams {
    int kind;
    double p0, p1, p2, p3;
    double Re;
    const double* ud = nullptr;   // CGP_BC_USER: caller's Dirichlet values (2 per vertex)
    const double* fu = nullptr;   // CGP_BC_USER: caller's body force (2 per vertex)
};

__device__ __forceinline__ void tg_shape(double x, double y, double& u, double& v, double& p) {
    const double tp = 2.0 * M_PI;
    double s2x, c2x, s2y, c2y;
    sincos(tp * x, &s2x, &c2x);
    sincos(tp * y, &s2y, &c2y);
    u = -c2x * s2y;
    v = s2x * c2y;
    p = -(cos(2.0 * tp * x) + cos(2.0 * tp * y)) / 4.0;
}

// The vortices of Sections 3.2 (open boundary, kind CGP_BC_JOBELIN_OPEN) and 3.3 (disk,
// CGP_BC_JOBELIN_DISK): the fields and the first derivatives the body force and the
// traction need.  Open: u = sin x sin(y+t), v = cos x cos(y+t), p = cos x sin(y+t).  Disk:
// u = sin(x+t) sin(y+t), v = cos(x+t) cos(y+t), p = cos(x-y+t).  Both are divergence free
// with Lap u = -2 u, Lap v = -2 v.
struct JobelinPoint {
    double u, v, p, ut, vt, ux, uy, vx, vy, px, py;
};
__device__ __forceinline__ JobelinPoint jobelin_point(int kind, double x, double y, double t) {
    JobelinPoint d;
    double sa, ca, sb, cb;
    if (kind == CGP_BC_JOBELIN_OPEN) {
        sincos(x, &sa, &ca);
        sincos(y + t, &sb, &cb);
        d.p = ca * sb;
        d.ut = sa * cb;
        d.vt = -ca * sb;
        d.px = -sa * sb;
        d.py = ca * cb;
    } else {
        sincos(x + t, &sa, &ca);
        sincos(y + t, &sb, &cb);
        const double c = x - y + t;
        d.p = cos(c);
        d.ut = ca * sb + sa * cb;
        d.vt = -sa * cb - ca * sb;
        d.px = -sin(c);
        d.py = sin(c);
    }
    d.u = sa * sb;
    d.v = ca * cb;
    d.ux = ca * sb;
    d.uy = sa * cb;
    d.vx = -sa * cb;
    d.vy = -ca * sb;
    return d;
}

// closed form (u, v, p) at (x, y, t); false if the kind has none
__device__ __forceinline__ bool exact_field(const BcParams& bc, double x, double y, double t, double& u, double& v,
                                            double& p) {
    if (bc.kind == CGP_BC_JOBELIN_OPEN || bc.kind == CGP_BC_JOBELIN_DISK) {
        const JobelinPoint d = jobelin_point(bc.kind, x, y, t);
        u = d.u;
        v = d.v;
        p = d.p;
        return true;
    }
    if (bc.kind == CGP_BC_TG) {
        tg_shape(x, y, u, v, p);
        const double e = exp(-8.0 * M_PI * M_PI * t / bc.Re);
        u *= e;
        v *= e;
        p *= e * e;
        return true;
    }
    if (bc.kind == CGP_BC_TG_PERIODIC) {
        tg_shape(x, y, u, v, p);
        const double g = cos(2.0 * M_PI * t);
        u *= g;
        v *= g;
        p *= g * g;
        return true;
    }
    return false;
}

// prescribed velocity at VEL_DIR vertex i
__device__ __forceinline__ void dirichlet_value(const BcParams& bc, int i, double x, double y, double t, double& u,
                                                double& v) {
    u = 0.0;
    v = 0.0;
    if (bc.kind == CGP_BC_USER) {
        u = bc.ud[2 * i];
        v = bc.ud[2 * i + 1];
        return;
    }
    if (bc.kind == CGP_BC_CAVITY) {
        if (y == 1.0 && x > 0.0 && x < 1.0) u = bc.p0;
        return;
    }
    if (bc.kind == CGP_BC_CHANNEL) {
        const double Umax = bc.p0, H = bc.p1;
        if (x == 0.0) u = 4.0 * Umax * y * (H - y) / (H * H);
        return;
    }
    double p;
    exact_field(bc, x, y, t, u, v, p);
}

__device__ __forceinline__ void body_force(const BcParams& bc, int i, double x, double y, double t, double& fx,
                                           double& fy) {
    fx = 0.0;
    fy = 0.0;
    if (bc.kind == CGP_BC_USER) {
        fx = bc.fu[2 * i];
        fy = bc.fu[2 * i + 1];
        return;
    }
    if (bc.kind == CGP_BC_TG_PERIODIC) {
        double u, v, p;
        tg_shape(x, y, u, v, p);
        const double g = cos(2.0 * M_PI * t);
        const double gp = -2.0 * M_PI * sin(2.0 * M_PI * t);
        const double c = gp + 8.0 * M_PI * M_PI * g / bc.Re;
        fx = c * u;
        fy = c * v;
        return;
    }
    if (bc.kind == CGP_BC_JOBELIN_OPEN || bc.kind == CGP_BC_JOBELIN_DISK) {
        // f = u_t + (u . grad) u - Lap u / Re + grad p, with Lap u = -2 u
        const JobelinPoint d = jobelin_point(bc.kind, x, y, t);
        fx = d.ut + d.u * d.ux + d.v * d.uy + 2.0 * d.u / bc.Re + d.px;
        fy = d.vt + d.u * d.vx + d.v * d.vy + 2.0 * d.v / bc.Re + d.py;
    }
}

// Data on the natural boundary Gamma_N (the PHI_ZERO vertices): the traction of Eq. 4 and
// the prescribed pressure.  Only the open-boundary vortex has any (Gamma_N = the y-axis,
// outward normal (-1, 0)); elsewhere the traction is zero and phi = 0 on Gamma_N.
__device__ __forceinline__ bool has_natural_data(const BcParams& bc) { return bc.kind == CGP_BC_JOBELIN_OPEN; }

// t = -p n + (grad u) n / Re at a Gamma_N vertex
__device__ __forceinline__ void natural_traction(const BcParams& bc, double x, double y, double t, double& tx,
                                                 double& ty) {
    const JobelinPoint d = jobelin_point(CGP_BC_JOBELIN_OPEN, x, y, t);
    tx = d.p - d.ux / bc.Re;
    ty = -d.vx / bc.Re;
}

__device__ __forceinline__ double natural_pressure(const BcParams& bc, double x, double y, double t) {
    return jobelin_point(CGP_BC_JOBELIN_OPEN, x, y, t).p;
}

// outward unit normal of Gamma_N (the y-axis)
__device__ __forceinline__ void natural_normal(const BcParams& bc, double x, double y, double& nx, double& ny) {
    nx = -1.0;
    ny = 0.0;
}

inline BcParams bc_from(const cgp_params& p) {
    BcParams b;
    b.kind = p.bc_kind;
    b.p0 = p.bc_param[0];
    b.p1 = p.bc_param[1];
    b.p2 = p.bc_param[2];
    b.p3 = p.bc_param[3];
    b.Re = p.Re;
    return b;
}

}  // namespace cgp
