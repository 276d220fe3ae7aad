// Static P1 operators of a CGP run (paper Section 2.1, Eqs. 17-20; coarse operators by
// rediscretisation, Section 2.2) and the solver's workspace layout.
//
// Assembly is vertex-centric: the thread of row i walks the triangles around vertex i
// (ascending) and adds each element contribution to the CSR slot of the other corner,
// so every row is written by one thread and the sums are deterministic (no atomics).
#include <cstring>

#include "flows.cuh"
#include "guess_proj.cuh"
#include "solver.cuh"

namespace cgp {

// area and hat-function gradients of every triangle: geo[7t] = |T|, geo[7t+1+2k] = grad psi_k
__global__ void k_geometry(const double* __restrict__ xy, const int32_t* __restrict__ tri, int nt,
                           double* __restrict__ geo) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
    const double x0 = xy[2 * a], y0 = xy[2 * a + 1], x1 = xy[2 * b], y1 = xy[2 * b + 1];
    const double x2 = xy[2 * c], y2 = xy[2 * c + 1];
    const double det = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
    double* o = geo + 7 * (int64_t)t;
    o[0] = 0.5 * det;
    o[1] = (y1 - y2) / det;
    o[2] = (x2 - x1) / det;
    o[3] = (y2 - y0) / det;
    o[4] = (x0 - x2) / det;
    o[5] = (y0 - y1) / det;
    o[6] = (x1 - x0) / det;
}

__device__ __forceinline__ int find_slot(const int32_t* __restrict__ col, int b, int e, int j) {
    for (int q = b; q < e; ++q)
        if (col[q] == j) return q - b;
    return -1;
}

// Row i of M, K, Cx, Cy (and optionally Cx^T, Cy^T) plus the packed corner slots.
__global__ void k_static_rows(int nv, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                              const int32_t* __restrict__ sell_ptr, const int32_t* __restrict__ vt_ptr, const int32_t* __restrict__ vt_list,
                              const int32_t* __restrict__ tri, const double* __restrict__ geo,
                              double* __restrict__ M, double* __restrict__ K, double* __restrict__ Cx,
                              double* __restrict__ Cy, double* __restrict__ CxT, double* __restrict__ CyT,
                              int32_t* __restrict__ vtslot) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    const int rb = rowptr[i], re = rowptr[i + 1];
    for (int k = 0; k < re - rb; ++k) {
        const int64_t q = sell_pos(sell_ptr, i, k);
        M[q] = 0.0;
        K[q] = 0.0;
        Cx[q] = 0.0;
        Cy[q] = 0.0;
        if (CxT) CxT[q] = 0.0;
        if (CyT) CyT[q] = 0.0;
    }
    for (int m = vt_ptr[i]; m < vt_ptr[i + 1]; ++m) {
        const int t = vt_list[m];
        const double* gt = geo + 7 * (int64_t)t;
        const double area = gt[0];
        int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
        const int li = v[0] == i ? 0 : (v[1] == i ? 1 : 2);
        int slots[3];
        for (int k = 0; k < 3; ++k) slots[k] = find_slot(col, rb, re, v[k]);
        if (vtslot) vtslot[m] = li | (slots[0] << 8) | (slots[1] << 16) | (slots[2] << 24);
        const double gix = gt[1 + 2 * li], giy = gt[2 + 2 * li];
        for (int k = 0; k < 3; ++k) {
            if (slots[k] < 0) continue;   // cannot happen for a consistent adjacency
            const int64_t q = sell_pos(sell_ptr, i, slots[k]);
            const double gkx = gt[1 + 2 * k], gky = gt[2 + 2 * k];
            M[q] += area / 12.0 * (k == li ? 2.0 : 1.0);
            K[q] += area * (gix * gkx + giy * gky);
            Cx[q] += area / 3.0 * gkx;
            Cy[q] += area / 3.0 * gky;
            if (CxT) CxT[q] += area / 3.0 * gix;
            if (CyT) CyT[q] += area / 3.0 * giy;
        }
    }
}

// out = A with the rows/columns of flagged vertices replaced by the identity; dinv = 1/out_ii
__global__ void k_eliminate(int nv, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ sell_ptr, const double* __restrict__ A, const uint8_t* __restrict__ tag, int flag,
                            double* __restrict__ out, double* __restrict__ dinv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    const bool fi = (tag[i] & flag) != 0;
    double d = 1.0;
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
        const int j = col[q];
        const int64_t e = sell_pos(sell_ptr, i, q - rowptr[i]);
        double a;
        if (fi || (tag[j] & flag)) a = (i == j) ? 1.0 : 0.0;
        else a = A[e];
        out[e] = a;
        if (j == i) d = a;
    }
    dinv[i] = 1.0 / d;
}

// S = a M + c K; also dinvM = 1/M_ii and the lumped mass (row sums of M)
__global__ void k_combine(int nv, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                          const int32_t* __restrict__ sell_ptr, const double* __restrict__ M, const double* __restrict__ K, double a, double c,
                          double* __restrict__ S, double* __restrict__ dinvM, double* __restrict__ mlump) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    double sum = 0.0, d = 1.0;
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
        const int64_t e = sell_pos(sell_ptr, i, q - rowptr[i]);
        if (S) S[e] = a * M[e] + c * K[e];
        sum += M[e];
        if (col[q] == i) d = M[e];
    }
    if (dinvM) dinvM[i] = 1.0 / d;
    if (mlump) mlump[i] = sum;
}

__global__ void k_to_float(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// values of a SELL-stored operator in CSR order (for inspection)
__global__ void k_sell_to_csr(int nv, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ sell_ptr,
                              const double* __restrict__ v, double* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) out[q] = v[sell_pos(sell_ptr, i, q - rowptr[i])];
}

static int layout(Solver& s, void* base, size_t* bytes) {
    const cgp_mesh* m = s.mesh;
    const Level& F = m->lev[s.lf];
    const Level& C = m->lev[s.lc];
    Carve cv(base);
    const size_t nf = F.nv, nc = C.nv, nnzf = F.nnz_sell, nnzc = C.nnz_sell;
    s.M = cv.take<double>(nnzf);
    s.K = cv.take<double>(nnzf);
    s.Cx = cv.take<double>(nnzf);
    s.Cy = cv.take<double>(nnzf);
    s.CxT = cv.take<double>(nnzf);
    s.CyT = cv.take<double>(nnzf);
    s.S = cv.take<double>(nnzf);
    s.M0 = cv.take<double>(nnzf);
    s.A = cv.take<double>(nnzf);
    s.dinvM0 = cv.take<double>(nf);
    s.dinvM = cv.take<double>(nf);
    s.mlumpF = cv.take<double>(nf);
    s.dinvA = cv.take<double>(nf);
    s.geo = cv.take<double>((size_t)7 * F.nt);
    s.vtslot = cv.take<int32_t>((size_t)3 * F.nt);
    s.Mc = cv.take<double>(nnzc);
    s.Kc = cv.take<double>(nnzc);
    s.Kc0 = cv.take<double>(nnzc);
    s.Cxc = cv.take<double>(nnzc);
    s.Cyc = cv.take<double>(nnzc);
    s.dinvKc = cv.take<double>(nc);
    s.mlumpC = cv.take<double>(nc);
    s.geoc = cv.take<double>((size_t)7 * C.nt);
    s.Kc0f = cv.take<float>(nnzc);
    s.dinvKcf = cv.take<float>(nc);
    s.cw64 = cv.take<double>(8 * nc);
    if (s.prm.guess == CGP_GUESS_LEARNED) {
        s.phi_guess = cv.take<double>(nc);
        s.mlp.carve(cv, (int)nc, 1);
        s.mlp_gate = cv.take<int>(4);
    }
    if (s.prm.guess == CGP_GUESS_LEARNED || s.prm.guess == CGP_GUESS_PROJ) {
        s.hist_x = cv.take<double>((size_t)kProjL * nc);
        s.hist_b = cv.take<double>((size_t)kProjL * nc);
        s.phi_q = cv.take<double>(nc);
        s.proj = reinterpret_cast<ProjState*>(cv.take<double>((sizeof(ProjState) + 7) / 8));
    }
    s.cw32 = cv.take<float>(9 * nc);
    if (s.prm.precision == CGP_MIXED) {
        // on-chip plan: at most kOnchipMaxCluster x 16 warps x kOnchipRows slices; entries: the
        // matrix, plus per leaf (rows sorted by length) one slice of the longest row (<= 64),
        // plus padding to 4-entry steps
        const size_t npos = (size_t)kOnchipMaxCluster * kOnchipWarps * kOnchipRows;
        const size_t nent = nnzc + (size_t)kOnchipMaxCluster * kOnchipWarps * 32 * 64 + 96 * npos;
        s.oc_grow = cv.take<int32_t>(32 * npos);
        s.oc_ebase = cv.take<int32_t>(npos);
        s.oc_width = cv.take<int32_t>(npos);
        s.oc_soff = cv.take<int32_t>(kOnchipMaxCluster + 1);
        s.oc_send_off = cv.take<int32_t>(kOnchipMaxCluster + 1);
        s.oc_halo_n = cv.take<int32_t>(kOnchipMaxCluster);
        s.oc_li = cv.take<int32_t>(nent);
        s.oc_src = cv.take<int32_t>(nent);
        s.oc_send_lr = cv.take<int32_t>(nnzc);     // sends <= entries with a remote column
        s.oc_send_dst = cv.take<int32_t>(nnzc);
        s.oc_hsub = cv.take<uint8_t>((size_t)kOnchipMaxCluster * (nc < 65535 ? nc : 65535));
        s.oc_hrow = cv.take<int32_t>((size_t)kOnchipMaxCluster * (nc < 65535 ? nc : 65535));
        s.oc_send_woff = cv.take<int32_t>((size_t)kOnchipMaxCluster * (kOnchipWarps + 1));
        s.oc_einv = cv.take<float>((size_t)kOnchipMaxCluster * kOnchipMaxSubPerCta * kOnchipMaxCluster * kOnchipMaxSubPerCta);
        s.oc_need = cv.take<uint8_t>((size_t)kOnchipMaxCluster * kOnchipMaxCluster * kOnchipMaxSubPerCta);
        s.oc_need_n = cv.take<int32_t>(kOnchipMaxCluster);
        s.Af = cv.take<float>(nnzf);
        s.M0f = cv.take<float>(nnzf);
        s.Mf = cv.take<float>(nnzf);
        s.dinvAf = cv.take<float>(nf);
        s.dinvM0f = cv.take<float>(nf);
        s.dinvMf = cv.take<float>(nf);
        s.frhs = cv.take<float>(2 * nf);
        for (float*& v : s.fv) v = cv.take<float>(2 * nf);
    }
    s.csr_tmp = cv.take<double>(F.nnz > C.nnz ? F.nnz : C.nnz);
    s.val_begin = s.M;
    s.val_end = s.geo;
    double** vec2[] = {&s.U, &s.Uprev, &s.Ut, &s.w, &s.h, &s.b, &s.g, &s.delta,
                       &s.bv.r, &s.bv.rhat, &s.bv.p, &s.bv.v, &s.bv.y, &s.bv.s, &s.bv.z, &s.bv.t,
                       &s.kr, &s.kz, &s.kp0, &s.kp1, &s.kq};
    for (double** p : vec2) *p = cv.take<double>(2 * nf);
    s.bv.x = s.Ut;
    s.P = cv.take<double>(nf);
    s.phi = cv.take<double>(nf);
    s.rc = cv.take<double>(nc);
    s.div = cv.take<double>(nf);
    s.qrot = cv.take<double>(nf);
    if (s.prm.bc_kind == CGP_BC_USER) {
        s.user_ud = cv.take<double>(2 * nf);
        s.user_f = cv.take<double>(2 * nf);
    }
    s.partials = cv.take<double>((size_t)s.max_grid * 8);
    s.tickets = cv.take<unsigned int>(64);
    s.bar_count = cv.take<unsigned int>(2);
    s.bar_err = (int*)(s.bar_count ? s.bar_count + 1 : nullptr);
    s.coarse_partials = cv.take<double>((size_t)2 * s.max_grid * 4);
    s.ks = cv.take<KrylovState>(KS_COUNT + 1);   // + the inner state of the mixed fine solves
    s.stats = cv.take<DeviceStats>(1);
    s.tdev = cv.take<double>(1);
    s.scal = cv.take<double>(16);
    *bytes = cv.off + 256;
    return CGP_OK;
}

static int check_params(const cgp_mesh* m, const cgp_params* p) {
    if (!m || !p) {
        set_error("null mesh or params");
        return CGP_EINVAL;
    }
    if (p->k < 0 || p->k > m->n_levels || !(p->Re > 0) || !(p->dt > 0) || (p->chi != 0 && p->chi != 1) ||
        !(p->tol_mom > 0) || !(p->tol_poisson > 0) || !(p->tol_mass > 0) || p->max_it_mom < 1 ||
        p->max_it_poisson < 1 || p->max_it_mass < 1 || p->bc_kind < 0 || p->bc_kind > CGP_BC_JOBELIN_DISK ||
        (p->bc_kind == CGP_BC_JOBELIN_OPEN && p->restrict_mode != CGP_RESTRICT_INJECT) || p->restrict_mode < 0 || p->restrict_mode > CGP_RESTRICT_PT || p->precond < 0 || p->precond > CGP_PRECOND_COARSE ||
        (p->precision != CGP_FP64 && p->precision != CGP_MIXED) || p->guess < 0 || p->guess > CGP_GUESS_PROJ ||
        (p->mass_mode != CGP_MASS_CONSISTENT && p->mass_mode != CGP_MASS_LUMPED) || p->coarse_mode < 0 ||
        p->coarse_mode > CGP_COARSE_ONCHIP || p->cluster_size < 0 || p->cluster_size > 16 || p->tol_inner < 0 ||
        p->tol_inner >= 1) {
        set_error("invalid cgp_params");
        return CGP_EINVAL;
    }
    return CGP_OK;
}

static void setup_dims(Solver& s, const cgp_mesh* m, const cgp_params* p) {
    s.mesh = m;
    s.prm = *p;
    s.lf = m->n_levels;
    s.lc = m->n_levels - p->k;
    s.nf = m->lev[s.lf].nv;
    s.nc = m->lev[s.lc].nv;
    s.ntf = m->lev[s.lf].nt;
    s.nnzf = m->lev[s.lf].nnz;
    s.nnzc = m->lev[s.lc].nnz;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // grid-stride kernels: up to 8 blocks per SM, never more than the rows need
    int64_t need = (s.nf + kBlock - 1) / kBlock;
    int64_t cap = (int64_t)sms * 8;
    s.max_grid = (int)cap;
    s.grid = (int)(need < cap ? need : cap);
    if (s.grid < 1) s.grid = 1;
}

}  // namespace cgp

using namespace cgp;

extern "C" int cgp_workspace_size(const cgp_mesh* mesh, const cgp_params* params, size_t* bytes) {
    clear_error();
    CGP_TRY(check_params(mesh, params));
    if (!bytes) {
        set_error("bytes is NULL");
        return CGP_EINVAL;
    }
    Solver s;
    setup_dims(s, mesh, params);
    return layout(s, nullptr, bytes);
}

extern "C" int cgp_assemble(const cgp_mesh* mesh, const cgp_params* params, void* workspace, size_t ws_bytes,
                            cgp_stream_t stream, cgp_solver** out) {
    clear_error();
    if (!out) {
        set_error("out is NULL");
        return CGP_EINVAL;
    }
    *out = nullptr;
    CGP_TRY(check_params(mesh, params));
    cudaStream_t st = (cudaStream_t)stream;
    cgp_solver* h = new cgp_solver();
    Solver& s = h->s;
    setup_dims(s, mesh, params);
    size_t need = 0;
    layout(s, nullptr, &need);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace & 255)) {
        set_error("workspace too small or not 256-byte aligned (%zu < %zu bytes)", ws_bytes, need);
        delete h;
        return CGP_ENOMEM;
    }
    layout(s, workspace, &need);
    s.ws_bytes = ws_bytes;
    const Level& F = mesh->lev[s.lf];
    const Level& C = mesh->lev[s.lc];
    auto fail = [&](int rc) {
        cgp_solver_destroy(h);
        return rc;
    };
    // pure-Neumann coarse problem unless some coarse vertex has phi = 0
    {
        std::vector<uint8_t> tagc(C.nv);
        if (cudaMemcpy(tagc.data(), C.tag, C.nv, cudaMemcpyDeviceToHost) != cudaSuccess) {
            set_error("tag copy failed");
            return fail(CGP_ECUDA);
        }
        s.pure_neumann = true;
        for (uint8_t t : tagc)
            if (t & CGP_PHI_ZERO) s.pure_neumann = false;
    }
    k_geometry<<<blocks_for(F.nt), kBlock, 0, st>>>(F.xy, F.tri, F.nt, s.geo);
    // all SELL value arrays start at zero (padding entries stay zero)
    if (cudaMemsetAsync(s.M, 0, (char*)s.geo - (char*)s.M, st) != cudaSuccess ||
        cudaMemsetAsync(s.Mc, 0, (char*)s.geoc - (char*)s.Mc, st) != cudaSuccess) {
        set_error("workspace initialisation failed");
        return fail(CGP_ECUDA);
    }
    k_static_rows<<<blocks_for(F.nv), kBlock, 0, st>>>(F.nv, F.rowptr, F.col, F.sell_ptr, F.vt_ptr, F.vt_list, F.tri, s.geo,
                                                       s.M, s.K, s.Cx, s.Cy, s.CxT, s.CyT, s.vtslot);
    const double a = 1.5, c = params->dt / params->Re;
    k_combine<<<blocks_for(F.nv), kBlock, 0, st>>>(F.nv, F.rowptr, F.col, F.sell_ptr, s.M, s.K, a, c, s.S, s.dinvM,
                                                   s.mlumpF);
    k_eliminate<<<blocks_for(F.nv), kBlock, 0, st>>>(F.nv, F.rowptr, F.col, F.sell_ptr, s.M, F.tag, CGP_VEL_DIR,
                                                     s.M0, s.dinvM0);
    k_geometry<<<blocks_for(C.nt), kBlock, 0, st>>>(C.xy, C.tri, C.nt, s.geoc);
    k_static_rows<<<blocks_for(C.nv), kBlock, 0, st>>>(C.nv, C.rowptr, C.col, C.sell_ptr, C.vt_ptr, C.vt_list, C.tri, s.geoc,
                                                       s.Mc, s.Kc, s.Cxc, s.Cyc, nullptr, nullptr, nullptr);
    k_combine<<<blocks_for(C.nv), kBlock, 0, st>>>(C.nv, C.rowptr, C.col, C.sell_ptr, s.Mc, s.Kc, 0.0, 0.0, nullptr,
                                                   nullptr, s.mlumpC);
    k_eliminate<<<blocks_for(C.nv), kBlock, 0, st>>>(C.nv, C.rowptr, C.col, C.sell_ptr, s.Kc, C.tag, CGP_PHI_ZERO,
                                                     s.Kc0, s.dinvKc);
    k_to_float<<<blocks_for(C.nnz_sell), kBlock, 0, st>>>(C.nnz_sell, s.Kc0, s.Kc0f);
    k_to_float<<<blocks_for(C.nv), kBlock, 0, st>>>(C.nv, s.dinvKc, s.dinvKcf);
    if (s.Mf) {
        k_to_float<<<blocks_for(F.nnz_sell), kBlock, 0, st>>>(F.nnz_sell, s.M0, s.M0f);
        k_to_float<<<blocks_for(F.nnz_sell), kBlock, 0, st>>>(F.nnz_sell, s.M, s.Mf);
        k_to_float<<<blocks_for(F.nv), kBlock, 0, st>>>(F.nv, s.dinvM0, s.dinvM0f);
        k_to_float<<<blocks_for(F.nv), kBlock, 0, st>>>(F.nv, s.dinvM, s.dinvMf);
    }
    if (cudaGetLastError() != cudaSuccess) {
        set_error("assembly launch failed");
        return fail(CGP_ECUDA);
    }
    {
        int rc = choose_coarse_solver(s, st);
        if (rc != CGP_OK) return fail(rc);
    }
    if (cudaMemsetAsync(s.tickets, 0, 64 * sizeof(unsigned int), st) != cudaSuccess ||
        cudaMemsetAsync(s.ks, 0, (KS_COUNT + 1) * sizeof(KrylovState), st) != cudaSuccess ||
        cudaMemsetAsync(s.stats, 0, sizeof(DeviceStats), st) != cudaSuccess ||
        cudaMemsetAsync(s.phi, 0, sizeof(double) * s.nf, st) != cudaSuccess ||
        (s.user_ud && cudaMemsetAsync(s.user_ud, 0, sizeof(double) * 2 * s.nf, st) != cudaSuccess) ||
        (s.user_f && cudaMemsetAsync(s.user_f, 0, sizeof(double) * 2 * s.nf, st) != cudaSuccess) ||
        cudaMemsetAsync(s.scal, 0, sizeof(double) * 16, st) != cudaSuccess ||
        (s.proj && cudaMemsetAsync(s.proj, 0, sizeof(ProjState), st) != cudaSuccess) ||
        (s.mlp_gate && cudaMemsetAsync(s.mlp_gate, 0, 4 * sizeof(int), st) != cudaSuccess)) {
        set_error("workspace initialisation failed");
        return fail(CGP_ECUDA);
    }
    int rc = init_state(&s, st);
    if (rc != CGP_OK) return fail(rc);
    if (cudaStreamCreateWithFlags(&s.side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s.branch, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&s.h_flag, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&s.h_view, sizeof(Solver::HostView)) != cudaSuccess) {
        set_error("stream / pinned flag creation failed");
        return fail(CGP_ECUDA);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("assembly failed on the device: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(CGP_ECUDA);
    }
    *out = h;
    return CGP_OK;
}

extern "C" int cgp_solver_info(const cgp_solver* h, int32_t* n_fine, int32_t* n_coarse, int64_t* nnz_fine,
                               int64_t* nnz_coarse) {
    if (!h) {
        set_error("null solver");
        return CGP_EINVAL;
    }
    if (n_fine) *n_fine = h->s.nf;
    if (n_coarse) *n_coarse = h->s.nc;
    if (nnz_fine) *nnz_fine = h->s.nnzf;
    if (nnz_coarse) *nnz_coarse = h->s.nnzc;
    return CGP_OK;
}

extern "C" int cgp_get_matrix(cgp_solver* h, int32_t which, double* vals, int32_t where, cgp_stream_t stream) {
    if (!h || !vals) {
        set_error("null solver or output");
        return CGP_EINVAL;
    }
    Solver& s = h->s;
    const double* src = nullptr;
    const bool coarse = which == CGP_MAT_KC || which == CGP_MAT_CXC || which == CGP_MAT_CYC;
    switch (which) {
        case CGP_MAT_M: src = s.M; break;
        case CGP_MAT_K: src = s.K; break;
        case CGP_MAT_CX: src = s.Cx; break;
        case CGP_MAT_CY: src = s.Cy; break;
        case CGP_MAT_KC: src = s.Kc; break;
        case CGP_MAT_CXC: src = s.Cxc; break;
        case CGP_MAT_CYC: src = s.Cyc; break;
        case CGP_MAT_A: src = s.A; break;
        default: set_error("unknown matrix %d", which); return CGP_EINVAL;
    }
    const Level& L = s.mesh->lev[coarse ? s.lc : s.lf];
    const size_t n = L.nnz;
    cudaStream_t st = (cudaStream_t)stream;
    k_sell_to_csr<<<blocks_for(L.nv), kBlock, 0, st>>>(L.nv, L.rowptr, L.sell_ptr, src, s.csr_tmp);
    CGP_LAUNCH_CHECK();
    src = s.csr_tmp;
    CGP_CUDA(cudaMemcpyAsync(vals, src, n * sizeof(double),
                             where == CGP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    if (where == CGP_HOST) CGP_CUDA(cudaStreamSynchronize(st));
    return CGP_OK;
}

extern "C" void cgp_solver_destroy(cgp_solver* h) {
    if (!h) return;
    Solver& s = h->s;
    if (s.step_exec) cudaGraphExecDestroy(s.step_exec);
    if (s.step_graph) cudaGraphDestroy(s.step_graph);
    if (s.side) cudaStreamDestroy(s.side);
    if (s.branch) cudaStreamDestroy(s.branch);
    if (s.ev_fork) cudaEventDestroy(s.ev_fork);
    if (s.ev_join) cudaEventDestroy(s.ev_join);
    if (s.h_flag) cudaFreeHost(s.h_flag);
    if (s.h_view) cudaFreeHost(s.h_view);
    delete h;
}
