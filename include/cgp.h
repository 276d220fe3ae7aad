/*
 * cgp.h -- C ABI of the GB300 coarse-grid incremental pressure-projection (CGP) library.
 *
 * The library advances the incompressible Navier-Stokes equations (paper Eqs. 1-4)
 * with the incremental pressure-correction scheme of Section 2.1 (BDF2, Eqs. 5-16)
 * discretised by P1/P1 finite elements (Eqs. 17-20), solving the Poisson problem for
 * the pressure increment phi on a mesh k levels coarser than the velocity mesh
 * (Section 2.2, Eqs. 21-26).  All arithmetic of a time step runs in CUDA kernels on
 * one GPU; the host only enqueues work.
 *
 * Conventions shared by every entry point
 *  - Return value: CGP_OK (0) or a negative CGP_E* code; nothing throws across the ABI.
 *    cgp_last_error() gives a message for the last failure on the calling thread.
 *  - Streams: a cudaStream_t passed as cgp_stream_t (NULL = the legacy default stream).
 *    Calls enqueue work on it and return without synchronising unless stated.
 *  - Memory: inputs are copied; the caller keeps ownership of every pointer it passes.
 *    A mesh owns device memory it allocates itself; a solver lives entirely inside the
 *    caller-supplied workspace (cgp_workspace_size bytes, 256-byte aligned, device
 *    memory) and allocates nothing else on the device.
 *  - `where` arguments: CGP_HOST = pointer is host memory (the call synchronises the
 *    stream), CGP_DEVICE = pointer is device memory (the call only enqueues copies).
 *  - Vertex order: level l's vertices are the first N_l vertices of level l+1; fields
 *    are returned in the finest level's order.  Velocities are interleaved (u0,v0,u1,...).
 */
#ifndef CGP_H
#define CGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cgp_mesh cgp_mesh;      /* opaque, library-owned */
typedef struct cgp_solver cgp_solver;  /* opaque, lives in caller workspace */
typedef struct CUstream_st* cgp_stream_t;  /* identical to cudaStream_t */

enum {
    CGP_OK = 0,
    CGP_EINVAL = -1,      /* bad mesh, parameters or arguments */
    CGP_ENOTCONV = -2,    /* an iterative solve hit its iteration cap (the step completed with its last iterate) */
    CGP_EBREAKDOWN = -3,  /* a Krylov recurrence broke down (zero denominator) */
    CGP_ENONFINITE = -4,  /* a residual became NaN or Inf */
    CGP_ETIMEOUT = -5,    /* a bounded device wait expired */
    CGP_ECUDA = -6,       /* a CUDA runtime call failed */
    CGP_ENOMEM = -7       /* workspace too small / allocation failed */
};

/* per-vertex boundary flags (bitwise OR); see cgp_mesh_desc */
enum { CGP_VEL_DIR = 1, CGP_PHI_ZERO = 2 };

/* built-in problem statements (boundary data, body force, initial state) */
enum {
    CGP_BC_CAVITY = 0,       /* [0,1]^2, u=(bc_param[0],0) on y=1 with 0<x<1, u=0 on the rest of the boundary */
    CGP_BC_CHANNEL = 1,      /* u=(4 Umax y(H-y)/H^2, 0) on x=0 (Umax=bc_param[0], H=bc_param[1]), u=0 elsewhere on VEL_DIR */
    CGP_BC_TG = 2,           /* Taylor-Green vortex, paper Eqs. 28-30 */
    CGP_BC_TG_PERIODIC = 3,  /* Taylor-Green with amplitude cos(2 pi t) and the body force that makes it exact */
    CGP_BC_USER = 4,         /* caller's data: the Dirichlet velocity of every VEL_DIR vertex and the body force
                                f of Eq. 21 at t^{n+1}, given by cgp_set_dirichlet / cgp_set_forcing before
                                each step (both zero until set; they keep their values between steps) */
    CGP_BC_JOBELIN_OPEN = 5, /* Section 3.2 vortex, u = sin x sin(y+t), v = cos x cos(y+t), p = cos x sin(y+t), with
                                its body force: velocity data on the VEL_DIR vertices, and on the PHI_ZERO
                                vertices (the traction boundary, the y-axis x = 0 of [0,1]^2) the traction of
                                Eq. 4 and the pressure from the closed form, Eq. 11 read at t^{n+1}: Eq. 21
                                gains dt * int_{Gamma_N} (t + (p^{n+1} - P^n) n) psi_i ds (linear on each
                                boundary edge), Eq. 23 takes phi = p^{n+1} - P^n there (restrict_mode
                                INJECT only) */
    CGP_BC_JOBELIN_DISK = 6  /* Section 3.3 vortex, u = sin(x+t) sin(y+t), v = cos(x+t) cos(y+t), p = cos(x-y+t),
                                with its body force; velocity data on the VEL_DIR vertices (the whole
                                boundary of the disk) */
};
enum { CGP_FP64 = 0, CGP_MIXED = 1 };                   /* precision of the coarse Poisson solve */
/* initial guess of the coarse Poisson solve (Eq. 23; the paper starts from nothing in
 * particular): zero, the previous step's increment, the projection onto the last 8
 * increments (PROJ: the combination of them that minimises the K_c-norm of the error,
 * Fischer 1998), or LEARNED: the projection refined by the network's prediction (the
 * one-launch solve starts from the K_c-norm-optimal combination of the projection and the
 * prediction, so never worse than the projection; until cgp_guess_set provides weights, the
 * projection alone) */
enum { CGP_GUESS_ZERO = 0, CGP_GUESS_PREV = 1, CGP_GUESS_LEARNED = 2, CGP_GUESS_PROJ = 3 };
enum { CGP_MASS_CONSISTENT = 0, CGP_MASS_LUMPED = 1 };    /* mass matrix of Eqs. 25-26 (lumped = Eq. 27) */
enum { CGP_HOST = 0, CGP_DEVICE = 1 };

/* Base (coarsest) mesh.  All pointers are host memory, read during cgp_mesh_create.
 * Triangles must be counter-clockwise with positive area; every vertex must be used.
 * vert_tag: CGP_VEL_DIR marks the Dirichlet velocity boundary Gamma_D (Eqs. 3, 10);
 * CGP_PHI_ZERO marks vertices where phi = 0 (the traction boundary Gamma_N, Eq. 14).
 * n_levels (0..4) uniform 1->4 refinements are built (Section 2.2). */
typedef struct {
    int32_t n_vert, n_tri;
    const double* xy;          /* 2*n_vert, interleaved */
    const int32_t* tri;        /* 3*n_tri */
    const uint8_t* vert_tag;   /* n_vert */
    int32_t n_levels;
} cgp_mesh_desc;

/* Parameters of a run (paper Section 3's Re, delta t, chi and coarsening level k). */
typedef struct {
    double Re, dt;
    int32_t chi;               /* 0 = standard form, 1 = rotational form (Eq. 16 / Eq. 26) */
    int32_t k;                 /* pressure-increment mesh = finest level - k (0 <= k <= n_levels) */
    double tol_mom;            /* relative residual of the momentum solve (Eq. 21) */
    double tol_poisson;        /* relative residual of the coarse Poisson solve (Eq. 23) */
    double tol_mass;           /* relative residual of the mass-matrix solves (Eqs. 25, 26) */
    int32_t max_it_mom, max_it_poisson, max_it_mass;
    int32_t precision;         /* CGP_FP64 | CGP_MIXED */
    int32_t guess;             /* CGP_GUESS_* */
    int32_t mass_mode;         /* CGP_MASS_* */
    int32_t bc_kind;           /* CGP_BC_* */
    double bc_param[4];
    int32_t use_graph;         /* 1: replay each step as a CUDA graph with device-side loop control */
    double tol_inner;          /* CGP_MIXED: residual reduction asked of each FP32 inner coarse solve
                                  (0: 1e-5; 1e-3 for the on-chip solve with Jacobi alone) */
    int32_t coarse_mode;       /* coarse Poisson solver: CGP_COARSE_* */
    int32_t cluster_size;      /* CTAs of the cluster solver (0 = largest that fits, else 2..16) */
    int32_t restrict_mode;     /* CGP_RESTRICT_*: how the right-hand side of Eq. 23 reaches the coarse level */
    int32_t precond;           /* CGP_PRECOND_*: preconditioner of the coarse Poisson PCG */
} cgp_params;

/* INJECT (the paper, Eqs. 22-23): inject U~ at the coarse vertices, then the coarse
 * divergence.  PT (a variant, not in the paper): the fine divergence Cx u~ + Cy v~
 * restricted by the transpose of the prolongation of Eq. 24, the Galerkin-consistent
 * right-hand side; the two agree when U~ is the prolongation of a coarse field. */
enum { CGP_RESTRICT_INJECT = 0, CGP_RESTRICT_PT = 1 };

/* Preconditioner of the coarse Poisson PCG (Eq. 23).  JACOBI: M^{-1} = D^{-1}.  COARSE
 * (a variant, not in the paper): Jacobi plus an additive subdomain coarse correction,
 * M^{-1} = D^{-1} + Z E^+ Z^T with Z the indicator vectors of up to 128 compact vertex
 * subdomains (phi = 0 vertices in none) and E^+ the pseudo-inverse of E = Z^T K_c Z, built
 * once at cgp_assemble; only the ONCHIP coarse solver has it (cgp_assemble fails with
 * CGP_EINVAL otherwise).  AUTO: COARSE where the ONCHIP solver runs, JACOBI elsewhere.
 * The solution is the same to the solve's tolerance; only the iteration count changes. */
enum { CGP_PRECOND_AUTO = 0, CGP_PRECOND_JACOBI = 1, CGP_PRECOND_COARSE = 2 };

/* Coarse Poisson solver kinds.  KERNELS: two kernel launches per PCG iteration (graph
 * WHILE loop).  PERSISTENT: the whole solve in one cooperative launch over the GPU with a
 * bounded software grid barrier; in FP64, when every row has at most 16 entries and the
 * mesh fits one 32-row slice per warp, each thread keeps its row and its PCG vectors in
 * registers.  PERSISTENT_MEM: the same without register residency.  CLUSTER: the whole
 * solve in one launch of one thread-block cluster, vectors in global memory, reductions
 * through distributed shared memory.  ONCHIP (CGP_MIXED only): the FP32 inner solve on one
 * cluster of 8 or 16 CTAs with the FP32 matrix and the vectors held in distributed shared
 * memory and hardware cluster barriers (cgp_assemble fails with CGP_EINVAL if the coarse
 * system does not fit).  AUTO: ONCHIP for CGP_MIXED when it fits, else PERSISTENT.
 * CGP_MIXED needs a one-launch kind (not KERNELS). */
enum { CGP_COARSE_AUTO = 0, CGP_COARSE_KERNELS = 1, CGP_COARSE_CLUSTER = 2, CGP_COARSE_PERSISTENT = 3,
       CGP_COARSE_PERSISTENT_MEM = 4, CGP_COARSE_ONCHIP = 5 };

/* Per-run statistics. */
typedef struct {
    int64_t steps;             /* steps taken since assembly / cgp_set_fields */
    double t;                  /* current time */
    int32_t it_mom, it_poisson, it_corr, it_mass;          /* iterations of the last step */
    int64_t sum_it_mom, sum_it_poisson, sum_it_corr, sum_it_mass;
    double res_mom, res_poisson;                           /* last relative residuals (max over components) */
    int32_t status;            /* first non-zero CGP_E* code seen by any solve, else 0 */
    int64_t launches;          /* kernel launches of graph-replayed steps (Krylov loop trips included) */
    int64_t guess_used;        /* steps whose coarse solve started from the learned prediction */
    int64_t sum_outer_poisson; /* FP64 residual sweeps (refinement steps) of the one-launch coarse
                                  solves, summed over steps; 0 for CGP_COARSE_KERNELS */
} cgp_stats;

/* Library message for the last failing call of this thread ("" if none). */
const char* cgp_last_error(void);

/* ---- mesh hierarchy (Section 2.2: V_1 c ... c V_{n_levels+1} by subdividing each
 * triangle into four).  Vertex N_l + e of level l+1 is the midpoint of edge e of
 * level l, edges ranked by ascending (min vertex, max vertex); triangle t=(a,b,c)
 * has children 4t+0=(a,m_ab,m_ca), 4t+1=(m_ab,b,m_bc), 4t+2=(m_ca,m_bc,c),
 * 4t+3=(m_ab,m_bc,m_ca); a midpoint of a boundary edge gets the AND of its end
 * flags, of an interior edge 0.  Built on the device; synchronises `stream`. */
int cgp_mesh_create(const cgp_mesh_desc* desc, cgp_stream_t stream, cgp_mesh** out);
/* Sizes of level `level` (0 = base).  nnz = entries of its vertex-adjacency CSR. */
int cgp_mesh_level_info(const cgp_mesh* mesh, int32_t level, int32_t* n_vert, int32_t* n_tri, int64_t* nnz);
/* Copy level arrays to host buffers (any may be NULL; synchronises).  parents holds
 * the 2 end points of each vertex added at this level (2*(N_l - N_{l-1}) ints). */
int cgp_mesh_get_level(const cgp_mesh* mesh, int32_t level, double* xy, int32_t* tri, uint8_t* tag,
                       int32_t* rowptr, int32_t* col, int32_t* parents);
void cgp_mesh_destroy(cgp_mesh* mesh);

/* ---- solver ---- */
/* Workspace bytes cgp_assemble needs for this mesh and parameters. */
int cgp_workspace_size(const cgp_mesh* mesh, const cgp_params* params, size_t* bytes);
/* Assemble the static P1 operators (Eqs. 17-20) on the velocity level and, by
 * rediscretisation, on the pressure-increment level (Section 2.2), and set the
 * initial state of the problem kind.  workspace: device memory of at least
 * cgp_workspace_size bytes that must outlive the solver.  The mesh must outlive it too. */
int cgp_assemble(const cgp_mesh* mesh, const cgp_params* params, void* workspace, size_t ws_bytes,
                 cgp_stream_t stream, cgp_solver** out);
/* CGP_BC_USER only (CGP_EINVAL otherwise): the velocity imposed on the VEL_DIR vertices
 * and the nodal body force used by the next steps, each 2*N_f doubles (u, v interleaved,
 * fine-level vertex order; entries of non-VEL_DIR vertices of uD are ignored).  Host
 * arrays synchronise; device arrays are copied on `stream`. */
int cgp_set_dirichlet(cgp_solver* s, const double* uD, int32_t where, cgp_stream_t stream);
int cgp_set_forcing(cgp_solver* s, const double* F, int32_t where, cgp_stream_t stream);
/* Replace the state: U (2*N_f), Uprev (2*N_f, may be NULL = U), P (N_f), time t. */
int cgp_set_fields(cgp_solver* s, const double* U, const double* Uprev, const double* P, double t,
                   int32_t where, cgp_stream_t stream);
/* Advance n_steps time steps, each Eqs. 21-26: momentum solve on the fine level,
 * injection to the pressure level, coarse Poisson solve for phi, prolongation,
 * velocity correction and pressure update (chi = 0: P += phi_f; chi = 1: the
 * consistent-mass rotational update of Eq. 26).  Asynchronous; solver status is
 * latched on the device and reported by cgp_get_fields. */
int cgp_step(cgp_solver* s, int32_t n_steps, cgp_stream_t stream);
/* Copy U (2*N_f) and P (N_f) (either may be NULL) and the stats; synchronises. Returns
 * the latched solver status (CGP_OK, CGP_ENOTCONV, ...) after a successful copy. */
int cgp_get_fields(cgp_solver* s, double* U, double* P, double* t, cgp_stats* stats,
                   int32_t where, cgp_stream_t stream);

/* Intermediate vectors of the last step (for checking each equation separately). */
enum {
    CGP_VEC_U = 0,        /* 2*N_f  U^{n+1} */
    CGP_VEC_UPREV = 1,    /* 2*N_f  U^n */
    CGP_VEC_P = 2,        /* N_f    P^{n+1} */
    CGP_VEC_UTILDE = 3,   /* 2*N_f  intermediate velocity of Eq. 21 */
    CGP_VEC_RHS_C = 4,    /* N_c    right-hand side of Eq. 23 (after the range projection) */
    CGP_VEC_PHI_C = 5,    /* N_c    coarse solution of Eq. 23 (after the mean fix) */
    CGP_VEC_PHI_F = 6     /* N_f    prolonged increment of Eq. 24 */
};
int cgp_get_vector(cgp_solver* s, int32_t which, double* out, int32_t where, cgp_stream_t stream);
/* Overwrite U, UPREV, P or PHI_C (the previous coarse increment, which is the initial
 * guess of the next Poisson solve under CGP_GUESS_PREV): restores a checkpoint. */
int cgp_set_vector(cgp_solver* s, int32_t which, const double* in, int32_t where, cgp_stream_t stream);
/* Values of a static operator on its level's CSR pattern (cgp_mesh_get_level). */
enum { CGP_MAT_M = 0, CGP_MAT_K = 1, CGP_MAT_CX = 2, CGP_MAT_CY = 3,      /* velocity level */
       CGP_MAT_KC = 4, CGP_MAT_CXC = 5, CGP_MAT_CYC = 6,                   /* pressure level */
       CGP_MAT_A = 7 };                                                    /* last momentum matrix */
int cgp_get_matrix(cgp_solver* s, int32_t which, double* vals, int32_t where, cgp_stream_t stream);
/* Sizes: fine/coarse vertex counts and the CSR entry counts of both levels. */
int cgp_solver_info(const cgp_solver* s, int32_t* n_fine, int32_t* n_coarse, int64_t* nnz_fine, int64_t* nnz_coarse);
/* The coarse Poisson solver cgp_assemble picked: *kind = the CGP_COARSE_* kind that runs
 * (never AUTO; PERSISTENT_MEM when the persistent solve keeps its vectors in memory),
 * *ctas = CTAs of its launch (0 for KERNELS), *cluster = CTAs per cluster (0 if none).
 * Any output pointer may be NULL.  CGP_EINVAL before cgp_assemble. */
int cgp_coarse_info(const cgp_solver* s, int32_t* kind, int32_t* ctas, int32_t* cluster);
/* Subdomains of the coarse solve's coarse correction (0: Jacobi alone), through *nsub.
 * CGP_EINVAL before cgp_assemble. */
int cgp_coarse_subdomains(const cgp_solver* s, int32_t* nsub);
/* Closed-form fields of the built-in manufactured kinds (CGP_BC_TG: Eqs. 28-30;
 * CGP_BC_TG_PERIODIC) at time t on every fine vertex: U (2 N_f, interleaved) and P (N_f);
 * either may be NULL.  For measuring errors; CGP_EINVAL for kinds without a closed form.
 * Host (synchronises) or device (asynchronous on stream) arrays. */
int cgp_exact_fields(cgp_solver* s, double t, double* U, double* P, int32_t where, cgp_stream_t stream);
/* Test hook of the failure path (the paper has no counterpart; off unless a caller sets
 * it): with on = 1, every bounded device wait inside the one-launch coarse solves (the
 * software grid barrier of the PERSISTENT kinds, the mbarrier waits of the on-chip
 * cluster solve) also waits for one signal that nothing sends, under a limit of
 * milliseconds instead of seconds, so the solve gives up and returns CGP_ETIMEOUT while
 * the context stays usable.  Applies to launches made after the call (cgp_poisson_solve,
 * eager steps; a step graph captured before keeps the earlier setting).  on = 0 restores
 * normal waits.  CGP_EINVAL for a null solver. */
int cgp_set_wait_test(cgp_solver* s, int32_t on);

/* Eq. 23 alone: solve K_c phi = rhs (N_c values; phi=0 rows and the pure-Neumann
 * projection/mean fix as in a step) with the configured precision and tolerance.
 * phi also gives the initial guess when params.guess = CGP_GUESS_PREV.
 * Returns the solve status; iterations through *iters (may be NULL). Synchronises. */
int cgp_poisson_solve(cgp_solver* s, const double* rhs, double* phi, int32_t* iters,
                      int32_t where, cgp_stream_t stream);
/* Eq. 24 alone: phi_f (N_f) = prolongation of phi_c (N_c) over the k levels. */
int cgp_prolong(cgp_solver* s, const double* phi_c, double* phi_f, int32_t where, cgp_stream_t stream);

/* Per-kernel timing of ONE step (the state advances as in cgp_step).  The step runs
 * with eager launches, each bracketed by two CUDA events on `stream`; launches of loop
 * kernels made after their solve had converged are not counted.  counts[id] and
 * total_ms[id] (arrays of n_ids >= CGP_PROF_COUNT) receive, per kernel kind, the
 * number of launches and their summed device time.  Synchronises. */
enum {
    CGP_PROF_MOM_PREP = 0, CGP_PROF_MOM_ASSEMBLE, CGP_PROF_MOM_SETUP, CGP_PROF_MOM_INIT,
    CGP_PROF_BICG_P, CGP_PROF_BICG_V, CGP_PROF_BICG_S, CGP_PROF_BICG_T, CGP_PROF_BICG_X,
    CGP_PROF_COARSE_RHS, CGP_PROF_POIS_SETUP, CGP_PROF_POIS_INIT, CGP_PROF_POIS_SPMV, CGP_PROF_POIS_UPDATE,
    CGP_PROF_PHI_MEAN, CGP_PROF_PHI_SUB, CGP_PROF_PROLONG,
    CGP_PROF_CORR_RHS, CGP_PROF_CORR_SETUP, CGP_PROF_CORR_INIT, CGP_PROF_CORR_SPMV, CGP_PROF_CORR_UPDATE,
    CGP_PROF_DIV, CGP_PROF_MASS_SETUP, CGP_PROF_MASS_INIT, CGP_PROF_MASS_SPMV, CGP_PROF_MASS_UPDATE,
    CGP_PROF_FINISH, CGP_PROF_POIS_CLUSTER, CGP_PROF_MLP,
    /* CGP_MIXED fine-level solves: FP64 refinement residual / update, FP32 inner kernels */
    CGP_PROF_IR_RESID, CGP_PROF_IR_UPDATE, CGP_PROF_TO_F32, CGP_PROF_F32_INIT, CGP_PROF_F32_BICG_P,
    CGP_PROF_F32_BICG_V, CGP_PROF_F32_BICG_S, CGP_PROF_F32_BICG_T, CGP_PROF_F32_BICG_X,
    /* p updates of the FP64 PCG loops (three kernels per iteration) */
    CGP_PROF_POIS_PUPD, CGP_PROF_CORR_PUPD, CGP_PROF_MASS_PUPD,
    /* CGP_MIXED: FP32 Chebyshev steps of the Eq. 26 and Eq. 25 mass-matrix solves */
    CGP_PROF_CHEB_MASS, CGP_PROF_CHEB_CORR,
    /* projection guess of the coarse solve (CGP_GUESS_PROJ, CGP_GUESS_LEARNED) */
    CGP_PROF_PROJ, CGP_PROF_COUNT
};
int cgp_profile_step(cgp_solver* s, cgp_stream_t stream, int32_t n_ids, int32_t* counts, double* total_ms);

void cgp_solver_destroy(cgp_solver* s);

/* ---- batches of independent instances (not in the paper) ----
 * cgp_batch_create groups assembled solvers (any meshes and parameters; each keeps its own
 * workspace and state).  Two forms:
 *  - whole step (CGP_BATCH_WHOLE_STEP, the default when every instance qualifies: injection
 *    restriction, a zero or previous-increment coarse guess, a one-launch coarse solver):
 *    every batched step is ONE persistent launch in which thread-block clusters take
 *    instances from a queue, largest first, and run each instance's whole step of Eqs. 21-26
 *    (momentum rows and FP64 BiCGStab, coarse right-hand side and the instance's coarse PCG,
 *    prolongation, Chebyshev mass solves of Eqs. 25-26 with the eigenvalue bounds [1/2, 2] of
 *    Jacobi-scaled P1 mass matrices, pressure update), reducing through distributed shared
 *    memory; the launch is captured in a CUDA graph;
 *  - graph branches (CGP_BATCH_BRANCHES): one CUDA graph per step with every instance's
 *    momentum solve and coarse right-hand side on its own stream, ONE persistent launch for
 *    all the coarse Poisson problems, then every instance's correction and update.
 * cluster_size (0 = autotune, else 1, 2, 4, 8) and threads (0 = autotune, else 256, 512,
 * 1024) fix the persistent launch's shape; the autotuner times each candidate on the
 * instances' first step (whole step) or first coarse problems (branches), restoring their
 * state after each trial.  The batch allocates its own device memory (launch arguments, a
 * queue counter and the saved state); the solvers must outlive it.  Synchronises `stream`. */
typedef struct cgp_batch cgp_batch;
enum { CGP_BATCH_AUTO = 0, CGP_BATCH_WHOLE_STEP = 1, CGP_BATCH_BRANCHES = 2 };
int cgp_batch_create(cgp_solver* const* solvers, int32_t n, int32_t cluster_size, int32_t threads,
                     cgp_stream_t stream, cgp_batch** out);
/* The same with the form chosen (CGP_BATCH_*); CGP_EINVAL if WHOLE_STEP is asked for and an
 * instance does not qualify. */
int cgp_batch_create_mode(cgp_solver* const* solvers, int32_t n, int32_t cluster_size, int32_t threads, int32_t mode,
                          cgp_stream_t stream, cgp_batch** out);
/* The form a batch runs (CGP_BATCH_WHOLE_STEP or CGP_BATCH_BRANCHES). */
int cgp_batch_mode(const cgp_batch* b, int32_t* mode);
/* n_steps batched steps (graph launches on `stream`); per-instance results and stats via
 * cgp_get_fields on each solver. */
int cgp_batch_step(cgp_batch* b, int32_t n_steps, cgp_stream_t stream);
/* Chosen shape, clusters per launch, and the autotuner's trial times (ms; -1 = not run) for
 * the candidates (cluster, threads) = (1,256),(1,512),(1,1024),(2,256),...,(8,1024). */
int cgp_batch_info(const cgp_batch* b, int32_t* cluster_size, int32_t* threads, int32_t* nclusters, float* trial_ms,
                   int32_t n_trials);
void cgp_batch_destroy(cgp_batch* b);

/* ---- learned initial guess (not in the paper) ----
 * A per-vertex MLP on one mesh level with 1-ring mean aggregation: inputs per vertex
 * (r/rms(r), q/rms(q), x, y) with r the coarse right-hand side of Eq. 23 and q the previous
 * step's Phi_c; layers a_l = W_l [h; mean over neighbours of h] + b_l, widths 4-64-64-1,
 * ReLU between layers; prediction Phi0 = q + rms(q) a_3.  Weights are bfloat16 in the
 * forward pass (FP32 arithmetic) with FP32 master weights and Adam.  Parameter vector
 * layout: W1[64][8], b1[64], W2[64][128], b2[64], W3[1][128], b3[1] (row-major, FP32).
 * The network owns device memory allocated by cgp_mlp_create. */
typedef struct cgp_mlp cgp_mlp;
int cgp_mlp_param_count(void);
/* Network for `level` of `mesh` (the mesh must outlive it) with room for max_batch samples;
 * all parameters start at zero (then the prediction is q itself). */
int cgp_mlp_create(const cgp_mesh* mesh, int32_t level, int32_t max_batch, cgp_mlp** out);
int cgp_mlp_set_params(cgp_mlp* m, const float* params, int32_t where, cgp_stream_t stream);  /* resets Adam */
int cgp_mlp_get_params(cgp_mlp* m, float* params, int32_t where, cgp_stream_t stream);
/* pred = Phi0 for `batch` samples; r, q, pred: device arrays of batch * N doubles. Asynchronous. */
int cgp_mlp_forward(cgp_mlp* m, const double* r, const double* q, int32_t batch, double* pred, cgp_stream_t stream);
/* loss = mean (a_3 - clip((target - q)/rms(q), -10, 10))^2 and its gradient w.r.t. the parameters (host
 * array of cgp_mlp_param_count floats); r, q, target on the device.  Synchronises. */
int cgp_mlp_grad(cgp_mlp* m, const double* r, const double* q, const double* target, int32_t batch, float* grad,
                 float* loss, cgp_stream_t stream);
/* one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on a batch; loss (host, may be NULL: no sync) */
int cgp_mlp_train_step(cgp_mlp* m, const double* r, const double* q, const double* target, int32_t batch, float lr,
                       float* loss, cgp_stream_t stream);
/* Copy the network's weights into a solver assembled with guess = CGP_GUESS_LEARNED whose
 * pressure-increment level is the network's level.  Synchronises. */
int cgp_guess_set(cgp_solver* s, const cgp_mlp* m, cgp_stream_t stream);
/* Training data for the learned guess, generated by the solver itself: advances n_steps
 * steps (as cgp_step) and stores, for step k, row k (N_c values) of rhs = the right-hand
 * side of Eq. 23, prev = the network's second input (the projection guess of the step for
 * a solver assembled with CGP_GUESS_PROJ or CGP_GUESS_LEARNED, else the increment Phi_c
 * before the step) and target = the increment Phi_c the coarse solve produced.  Arrays of n_steps * N_c
 * doubles, host or device (where); host: synchronises, device: asynchronous on stream. */
int cgp_record_pairs(cgp_solver* s, int32_t n_steps, double* rhs, double* prev, double* target, int32_t where,
                     cgp_stream_t stream);
/* Copy the weights and the Adam state (moments and step count) of src into dst, on the
 * device, asynchronously on stream: one network trained on several meshes (one cgp_mlp per
 * mesh level, the state handed from one to the next between training steps). */
int cgp_mlp_copy_state(cgp_mlp* dst, const cgp_mlp* src, cgp_stream_t stream);
void cgp_mlp_destroy(cgp_mlp* m);

/* ---- allocation-free solve (the paper has no counterpart) ----
 * For callers that cannot call cudaMalloc (a host program that owns every device
 * allocation, a fixed-memory real-time loop, a plug-in handed only the buffers it may
 * touch): solves A x = b for a symmetric positive definite A with the library's Jacobi-
 * preconditioned, one-launch PCG (Chronopoulos-Gear recurrence on a cooperative grid,
 * true-residual stopping test ||b - A x|| <= tol ||b||) and allocates nothing:
 * every scratch word lives in one fixed file-scope device array of about 4.3 MB that each
 * device loading the library keeps until the process exits.
 *  - A in SELL-32 form (see cgp_mesh_get_level: slice s = rows 32s..32s+31, entries of a
 *    slice column-major, width = its longest row, padding with value 0): sell_ptr
 *    (nslices+1 offsets), sell_col, val; dinv = 1/diag(A).  n <= 65536 rows, else
 *    CGP_EINVAL.  All pointers are device memory owned by the caller.
 *  - x: initial guess on entry, solution on exit.  info: 2 device int32 written at the end
 *    of the solve: iterations, status (CGP_OK, CGP_ENOTCONV, CGP_EBREAKDOWN, ...).
 *  - Asynchronous on `stream`.  The first call on a device looks up the array's device
 *    address and the launch size (make it before any stream capture); later calls only
 *    enqueue a memset of the barrier counter, the solve and a status copy.  The address is
 *    kept per device and context: after cudaDeviceReset the next call looks it up again
 *    (that call, too, belongs before any capture).
 *  - Every call shares the one array: calls whose solves may overlap on the GPU (different
 *    streams without ordering, or other host threads) race and must not be made. */
int cgp_pcg_sell_noalloc(int32_t n, int32_t nslices, const int32_t* sell_ptr, const int32_t* sell_col,
                         const double* val, const double* dinv, const double* b, double* x, double tol,
                         int32_t maxit, int32_t* info, cgp_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* CGP_H */
