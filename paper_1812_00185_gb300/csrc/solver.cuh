// Solver object of the CGP library: operators, state and work vectors of one run,
// all carved out of the caller's workspace.
#pragma once

#include "krylov.cuh"
#include "mlp.cuh"
#include "onchip_plan.cuh"

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
    int64_t guess_used;           // steps that started the coarse solve from the learned prediction
    int64_t sum_outer;            // FP64 residual sweeps of the one-launch coarse solves
    int64_t sum_it[KS_COUNT];
    int32_t last_it[KS_COUNT];
    int32_t status;
    int32_t pad;
    double res[KS_COUNT];
};

struct ProjState;   // guess_proj.cuh

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
    float *Kc0f = nullptr, *dinvKcf = nullptr;                   // FP32 copies (mixed precision)
    MlpBuffers mlp;               // learned guess (CGP_GUESS_LEARNED): weights and batch-1 activations
    bool guess_ready = false;     // weights set by cgp_guess_set
    int wait_test = 0;            // test hook of cgp_set_wait_test
    // projection guess (CGP_GUESS_PROJ, CGP_GUESS_LEARNED): the last solutions and right-hand
    // sides of the coarse solve (kProjL x n_c each), their Galerkin matrix, and the guess the
    // network sees (copied for cgp_record_pairs)
    double *hist_x = nullptr, *hist_b = nullptr, *phi_q = nullptr;
    ProjState* proj = nullptr;
    double* phi_guess = nullptr;  // n_c: the network's prediction of Phi_c
    int* mlp_gate = nullptr;      // the coarse solve's judge of the network (see CoarsePcgArgs::gate)
    double* cw64 = nullptr;       // coarse one-launch solver work: 8 FP64 vectors of n_c
    float* cw32 = nullptr;        // and 9 FP32 vectors of n_c
    int coarse_kind = 0;          // CGP_COARSE_KERNELS / _CLUSTER / _PERSISTENT (AUTO resolved)
    int cluster_size = 0;         // CTAs of the one-cluster solver
    int coarse_grid = 0;          // CTAs of the persistent (cooperative) solver
    bool coarse_rr = false;       // the persistent FP64 solve may keep its rows in registers
    double *user_ud = nullptr, *user_f = nullptr;   // CGP_BC_USER: 2*nf each
    bool coarse_fp64 = true;
    cudaStream_t branch = nullptr;                 // second stream of a step (work beside the coarse solve)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;      // the coarse solve's inner iterations run in FP64
    size_t onchip_bytes = 0;      // mixed: shared memory per CTA of the on-chip cluster solve (0 = not used)
    // mixed: workspace arrays of the on-chip plan (sized for the coarse level) and its device view
    int32_t *oc_grow = nullptr, *oc_soff = nullptr, *oc_ebase = nullptr, *oc_width = nullptr, *oc_li = nullptr;
    int32_t *oc_src = nullptr, *oc_send_lr = nullptr, *oc_send_dst = nullptr, *oc_send_off = nullptr, *oc_halo_n = nullptr;
    uint8_t* oc_hsub = nullptr;
    int32_t *oc_hrow = nullptr, *oc_send_woff = nullptr, *oc_need_n = nullptr;
    uint8_t* oc_need = nullptr;
    float* oc_einv = nullptr;
    OnchipPlan onchip{};
    unsigned int* bar_count = nullptr;   // grid barrier counter, followed by the error word
    int* bar_err = nullptr;
    double* coarse_partials = nullptr;   // 2 x max_grid x 4
    double* geoc = nullptr;
    double* csr_tmp = nullptr;    // CSR-ordered copy of one operator (cgp_get_matrix)
    double *val_begin = nullptr, *val_end = nullptr;
    int32_t* vtslotc = nullptr;
    // per-step
    double *A = nullptr, *dinvA = nullptr;
    double *U = nullptr, *Uprev = nullptr, *Ut = nullptr, *w = nullptr, *h = nullptr, *b = nullptr;  // 2*nf
    double *P = nullptr, *phi = nullptr, *rc = nullptr, *div = nullptr, *qrot = nullptr;            // nf / nc
    double *g = nullptr, *delta = nullptr;                                                           // 2*nf
    BicgVecs bv{};
    double *kr = nullptr, *kz = nullptr, *kp0 = nullptr, *kp1 = nullptr, *kq = nullptr;             // 2*nf each
    // mixed form, fine-level FP32 inner solves: FP32 copies of the matrices and Jacobi
    // diagonals (A refreshed every step), the right-hand side and the inner vectors
    float *Af = nullptr, *dinvAf = nullptr, *M0f = nullptr, *dinvM0f = nullptr, *Mf = nullptr, *dinvMf = nullptr;
    float* frhs = nullptr;        // 2*nf: FP32 residual of the current refinement sweep
    float* fv[9] = {};            // 2*nf each: inner PCG (r, z, p0, p1, q, e) / BiCGStab (x..t)
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
    struct HostView {             // pinned host copies of the stats and the time (cgp_get_fields)
        DeviceStats stats;
        double t;
    }* h_view = nullptr;
};

// Optional per-launch timing: every kernel launch of an eager step is bracketed by
// two CUDA events on the launching stream (cgp_profile_step).
struct Prof {
    int n = 0, cap = 0;
    cudaEvent_t* ev = nullptr;   // 2 per launch
    int* id = nullptr;
};

// where and how a piece of a step is enqueued
struct Ctx {
    Solver* s;
    cudaStream_t st;
    bool capture;                 // stream capture: Krylov loops become conditional WHILE nodes
    Prof* prof = nullptr;
};

// helpers implemented in step.cu / assemble.cu
int enqueue_step(Solver* s, cudaStream_t st, bool capture);
int step_pre(Ctx& c);             // Eq. 21, Eqs. 22-23 right-hand side, learned prediction
int step_post(Ctx& c, bool mass_done = false);   // Eqs. 24-26 and the end of the step
size_t coarse_args_size();
void fill_coarse_args(Solver& s, void* dst);
int batch_clusters(int csize, int threads, int* nclusters);
int launch_batch_coarse(const void* d_args, int ninst, unsigned int* queue, int csize, int threads, int nclusters,
                        cudaStream_t st);
// the batched whole step (batch_step.cuh): one persistent clustered launch for every phase
size_t batch_step_args_size();
bool batch_step_eligible(const Solver& s);
void fill_batch_step_args(Solver& s, void* dst);
int batch_step_clusters(int csize, int threads, int* nclusters);
int launch_batch_step(const void* d_args, int ninst, unsigned int* queue, int csize, int threads, int nclusters,
                      cudaStream_t st);
int choose_coarse_solver(Solver& s, cudaStream_t st);
int init_state(Solver* s, cudaStream_t st);

}  // namespace cgp

struct cgp_solver {
    cgp::Solver s;
};
