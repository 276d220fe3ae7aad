// Solver object of the CGP library: operators, state and work vectors of one run,
// all carved out of the caller's workspace.
#pragma once

#include "krylov.cuh"

namespace cgp {

// Bump allocator over the caller's workspace (base == nullptr: only measure).
struct Carve {
    char* base;
    size_t off = 0;
    explicit Carve(void* b) : base((char*)b) {}
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? (T*)(base + off) : nullptr;
        off += count * sizeof(T) + 16;   // 16 bytes of slack keep 2-wide vector loads in bounds
        return p;
    }
};

enum { KS_MOM = 0, KS_POIS = 1, KS_CORR = 2, KS_MASS = 3, KS_COUNT = 4 };

struct DeviceStats {
    int64_t steps;
    int64_t launches;             // kernels launched by graph-replayed steps (loop trips included)
    int64_t sum_it[KS_COUNT];
    int32_t last_it[KS_COUNT];
    int32_t status;
    int32_t pad;
    double res[KS_COUNT];
};

struct Solver {
    const cgp_mesh* mesh = nullptr;
    cgp_params prm{};
    int lf = 0, lc = 0, nf = 0, nc = 0, ntf = 0;
    int64_t nnzf = 0, nnzc = 0;
    bool pure_neumann = true;
    int grid = 0;                 // blocks of the per-vertex kernels of the fine level
    int max_grid = 0;             // most blocks any reduction kernel is launched with (8 per SM)
    size_t ws_bytes = 0;
    // fine-level static operators (values on the fine CSR pattern)
    double *M = nullptr, *K = nullptr, *Cx = nullptr, *Cy = nullptr, *CxT = nullptr, *CyT = nullptr;
    double *S = nullptr;          // 3/2 M + dt/Re K
    double *M0 = nullptr;         // M with velocity-Dirichlet rows/columns replaced by the identity
    double *dinvM0 = nullptr, *dinvM = nullptr, *mlumpF = nullptr;
    double* geo = nullptr;        // 7 per fine triangle: area, grad psi_0..2 (x, y)
    int32_t* vtslot = nullptr;    // per (vertex, incident triangle): local index | row slots of the 3 corners
    // coarse-level static operators
    double *Mc = nullptr, *Kc = nullptr, *Kc0 = nullptr, *Cxc = nullptr, *Cyc = nullptr;
    double *dinvKc = nullptr, *mlumpC = nullptr;
    double* geoc = nullptr;
    int32_t* vtslotc = nullptr;
    // per-step
    double *A = nullptr, *dinvA = nullptr;
    double *U = nullptr, *Uprev = nullptr, *Ut = nullptr, *w = nullptr, *h = nullptr, *b = nullptr;  // 2*nf
    double *P = nullptr, *phi = nullptr, *rc = nullptr, *div = nullptr, *qrot = nullptr;            // nf / nc
    double *g = nullptr, *delta = nullptr;                                                           // 2*nf
    BicgVecs bv{};
    double *kr = nullptr, *kz = nullptr, *kp0 = nullptr, *kp1 = nullptr, *kq = nullptr;             // 2*nf each
    double* partials = nullptr;
    unsigned int* tickets = nullptr;
    KrylovState* ks = nullptr;    // KS_COUNT states
    DeviceStats* stats = nullptr;
    double* tdev = nullptr;       // current time on the device
    double* scal = nullptr;       // misc device scalars (mean of phi, ...)
    // execution
    cudaStream_t side = nullptr;  // stream used to capture loop bodies
    cudaGraphExec_t step_exec = nullptr;
    cudaGraph_t step_graph = nullptr;
    int* h_flag = nullptr;        // pinned host word for eager loop control
};

// helpers implemented in step.cu / assemble.cu
int enqueue_step(Solver* s, cudaStream_t st, bool capture);
int init_state(Solver* s, cudaStream_t st);

}  // namespace cgp

struct cgp_solver {
    cgp::Solver s;
};
