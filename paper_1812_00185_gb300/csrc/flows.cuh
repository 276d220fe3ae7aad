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

// closed form (u, v, p) at (x, y, t); false if the kind has none
__device__ __forceinline__ bool exact_field(const BcParams& bc, double x, double y, double t, double& u, double& v,
                                            double& p) {
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
    }
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
