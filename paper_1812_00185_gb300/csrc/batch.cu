// Many independent CGP instances advanced together (not in the paper).
//
// Whole-step form (the default whenever every instance qualifies: injection restriction, a
// zero or previous-increment coarse guess, a one-launch coarse solver): one batched step is
// ONE persistent clustered launch (k_batch_step, batch_step.cuh) in which every cluster takes
// instances from a queue, largest first, and runs each one's entire step; the cluster size
// and threads per CTA are autotuned on the batch's own first step (the instances' state is
// saved and restored around the trials).  The launch is captured in a CUDA graph.
//
// Branch form (otherwise, or when asked for): one batched step is one CUDA graph:
//   for every instance, on its own stream (independent graph branches):
//       Eq. 21 momentum solve, Eqs. 22-23 right-hand side        (step_pre)
//   ONE persistent launch: the coarse Poisson solves of all instances; clusters take
//       instances from a queue, largest first                    (k_pcg_batch)
//   for every instance, on its own stream:
//       Eqs. 24-26, end of step                                  (step_post)
// The cluster size and the threads per CTA of the persistent launch are chosen by an
// autotuner that times every candidate on the batch's own first coarse problems (the
// instances' coarse state is saved and restored around the trials).
#include <algorithm>
#include <cstring>

#include "solver.cuh"

using namespace cgp;

struct cgp_batch {
    int whole = 0;                          // 1: whole-step persistent launch, 0: graph branches
    void* d_step_args = nullptr;            // BatchStepArgs[n], device (whole-step form)
    double* d_state = nullptr;              // saved U, U_prev, P, phi, t, stats, Krylov states (autotuning)
    std::vector<Solver*> inst;              // in launch order (largest coarse level first)
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    cudaStream_t origin = nullptr;
    void* d_args = nullptr;                 // CoarsePcgArgs[n], device
    unsigned int* d_queue = nullptr;
    double* d_save = nullptr;               // saved rhs and Phi_c of every instance (autotuning)
    int csize = 1, threads = 256, nclusters = 1;
    std::vector<float> trial_ms;            // per candidate, -1 if it does not fit
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

const int kCand[][2] = {{1, 256}, {1, 512}, {1, 1024}, {2, 256}, {2, 512}, {2, 1024},
                        {4, 256}, {4, 512}, {4, 1024}, {8, 256}, {8, 512}, {8, 1024}};
constexpr int kNumCand = sizeof(kCand) / sizeof(kCand[0]);

int save_coarse(cgp_batch* b, bool restore, cudaStream_t st) {
    size_t off = 0;
    for (Solver* s : b->inst) {
        const size_t n = (size_t)s->nc;
        if (restore) {
            CGP_CUDA(cudaMemcpyAsync(s->rc, b->d_save + off, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            CGP_CUDA(cudaMemcpyAsync(s->phi, b->d_save + off + n, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        } else {
            CGP_CUDA(cudaMemcpyAsync(b->d_save + off, s->rc, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            CGP_CUDA(cudaMemcpyAsync(b->d_save + off + n, s->phi, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
        off += 2 * n;
    }
    return CGP_OK;
}

int autotune(cgp_batch* b, int fixed_csize, int fixed_threads, cudaStream_t st) {
    // realistic coarse problems: the first step's right-hand sides
    for (Solver* s : b->inst) {
        Ctx c{s, st, false};
        CGP_TRY(step_pre(c));
    }
    CGP_TRY(save_coarse(b, false, st));
    cudaEvent_t e0, e1;
    CGP_CUDA(cudaEventCreate(&e0));
    CGP_CUDA(cudaEventCreate(&e1));
    b->trial_ms.assign(kNumCand, -1.0f);
    float best = 1e30f;
    int rc = CGP_OK;
    for (int k = 0; k < kNumCand && rc == CGP_OK; ++k) {
        const int cs = kCand[k][0], th = kCand[k][1];
        if ((fixed_csize && cs != fixed_csize) || (fixed_threads && th != fixed_threads)) continue;
        int ncl = 0;
        batch_clusters(cs, th, &ncl);
        if (ncl < 1) continue;
        if (ncl > (int)b->inst.size()) ncl = (int)b->inst.size();
        if ((rc = save_coarse(b, true, st)) != CGP_OK) break;
        cudaEventRecord(e0, st);
        if ((rc = launch_batch_coarse(b->d_args, (int)b->inst.size(), b->d_queue, cs, th, ncl, st)) != CGP_OK) break;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            set_error("batched coarse trial failed: %s", cudaGetErrorString(cudaGetLastError()));
            rc = CGP_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        b->trial_ms[k] = ms;
        if (ms < best) {
            best = ms;
            b->csize = cs;
            b->threads = th;
            b->nclusters = ncl;
        }
    }
    if (rc == CGP_OK) rc = save_coarse(b, true, st);
    if (rc == CGP_OK && cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("autotuning failed on the device");
        rc = CGP_ECUDA;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == CGP_OK && best >= 1e30f) {
        set_error("no cluster shape fits this device");
        rc = CGP_EINVAL;
    }
    return rc;
}

// every instance's step state (autotuning of the whole-step launch runs real steps)
size_t state_doubles(const Solver& s) {
    return 6 * (size_t)s.nf + 1 + (sizeof(DeviceStats) + KS_COUNT * sizeof(KrylovState) + 7) / 8;
}

int save_state(cgp_batch* b, bool restore, cudaStream_t st) {
    size_t off = 0;
    for (Solver* s : b->inst) {
        double* base = b->d_state + off;
        const size_t nf = s->nf;
        struct Piece {
            void* p;
            size_t bytes;
        } pieces[] = {{s->U, 16 * nf}, {s->Uprev, 16 * nf}, {s->P, 8 * nf}, {s->phi, 8 * nf}, {s->tdev, 8},
                      {s->stats, sizeof(DeviceStats)}, {s->ks, KS_COUNT * sizeof(KrylovState)}};
        char* q = reinterpret_cast<char*>(base);
        for (const Piece& pc : pieces) {
            if (restore) CGP_CUDA(cudaMemcpyAsync(pc.p, q, pc.bytes, cudaMemcpyDeviceToDevice, st));
            else CGP_CUDA(cudaMemcpyAsync(q, pc.p, pc.bytes, cudaMemcpyDeviceToDevice, st));
            q += pc.bytes;
        }
        off += state_doubles(*s);
    }
    return CGP_OK;
}

const int kStepCand[][2] = {{1, 256}, {1, 512}, {1, 1024}, {2, 256}, {2, 512}, {2, 1024}, {4, 256}, {4, 512},
                            {4, 1024}, {8, 256}, {8, 512}, {8, 1024}};
constexpr int kNumStepCand = sizeof(kStepCand) / sizeof(kStepCand[0]);

int autotune_whole(cgp_batch* b, int fixed_csize, int fixed_threads, cudaStream_t st) {
    CGP_TRY(save_state(b, false, st));
    cudaEvent_t e0, e1;
    CGP_CUDA(cudaEventCreate(&e0));
    CGP_CUDA(cudaEventCreate(&e1));
    b->trial_ms.assign(kNumStepCand, -1.0f);
    float best = 1e30f;
    int rc = CGP_OK;
    const int n = (int)b->inst.size();
    for (int k = 0; k < kNumStepCand && rc == CGP_OK; ++k) {
        const int cs = kStepCand[k][0], th = kStepCand[k][1];
        if ((fixed_csize && cs != fixed_csize) || (fixed_threads && th != fixed_threads)) continue;
        int ncl = 0;
        if ((rc = batch_step_clusters(cs, th, &ncl)) != CGP_OK) break;
        if (ncl < 1) continue;
        if (ncl > n) ncl = n;
        if ((rc = save_state(b, true, st)) != CGP_OK) break;
        cudaEventRecord(e0, st);
        if ((rc = launch_batch_step(b->d_step_args, n, b->d_queue, cs, th, ncl, st)) != CGP_OK) break;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            set_error("batched step trial failed: %s", cudaGetErrorString(cudaGetLastError()));
            rc = CGP_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        b->trial_ms[k] = ms;
        if (ms < best) {
            best = ms;
            b->csize = cs;
            b->threads = th;
            b->nclusters = ncl;
        }
    }
    if (rc == CGP_OK) rc = save_state(b, true, st);
    if (rc == CGP_OK && cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("autotuning failed on the device");
        rc = CGP_ECUDA;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == CGP_OK && best >= 1e30f) {
        set_error("no cluster shape fits this device");
        rc = CGP_EINVAL;
    }
    return rc;
}

int build_graph_whole(cgp_batch* b) {
    cudaStream_t o = b->origin;
    CGP_CUDA(cudaStreamBeginCapture(o, cudaStreamCaptureModeThreadLocal));
    int rc = launch_batch_step(b->d_step_args, (int)b->inst.size(), b->d_queue, b->csize, b->threads, b->nclusters, o);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(o, &g);
    if (rc != CGP_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (rc == CGP_OK) set_error("batch graph capture failed: %s", cudaGetErrorString(e));
        return rc == CGP_OK ? CGP_ECUDA : rc;
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        set_error("batch graph instantiation failed: %s", cudaGetErrorString(e));
        return CGP_ECUDA;
    }
    b->graph = g;
    return CGP_OK;
}

int build_graph(cgp_batch* b) {
    const int n = (int)b->inst.size();
    cudaStream_t o = b->origin;
    CGP_CUDA(cudaStreamBeginCapture(o, cudaStreamCaptureModeThreadLocal));
    int rc = CGP_OK;
    cudaEvent_t* ev = b->events.data();   // [0]: fork 1, [1]: fork 2, [2+2i], [3+2i]: joins of instance i
    do {
        if (cudaEventRecord(ev[0], o) != cudaSuccess) { rc = CGP_ECUDA; break; }
        for (int i = 0; i < n && rc == CGP_OK; ++i) {
            if (cudaStreamWaitEvent(b->streams[i], ev[0], 0) != cudaSuccess) { rc = CGP_ECUDA; break; }
            Ctx c{b->inst[i], b->streams[i], true};
            if ((rc = step_pre(c)) != CGP_OK) break;
            if (cudaEventRecord(ev[2 + 2 * i], b->streams[i]) != cudaSuccess ||
                cudaStreamWaitEvent(o, ev[2 + 2 * i], 0) != cudaSuccess) rc = CGP_ECUDA;
        }
        if (rc != CGP_OK) break;
        if ((rc = launch_batch_coarse(b->d_args, n, b->d_queue, b->csize, b->threads, b->nclusters, o)) != CGP_OK)
            break;
        if (cudaEventRecord(ev[1], o) != cudaSuccess) { rc = CGP_ECUDA; break; }
        for (int i = 0; i < n && rc == CGP_OK; ++i) {
            if (cudaStreamWaitEvent(b->streams[i], ev[1], 0) != cudaSuccess) { rc = CGP_ECUDA; break; }
            Ctx c{b->inst[i], b->streams[i], true};
            if ((rc = step_post(c)) != CGP_OK) break;
            if (cudaEventRecord(ev[3 + 2 * i], b->streams[i]) != cudaSuccess ||
                cudaStreamWaitEvent(o, ev[3 + 2 * i], 0) != cudaSuccess) rc = CGP_ECUDA;
        }
    } while (0);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(o, &g);
    if (rc != CGP_OK) {
        if (rc == CGP_ECUDA) set_error("batch graph capture failed: %s", cudaGetErrorString(cudaGetLastError()));
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) {
        set_error("batch graph capture failed: %s", cudaGetErrorString(e));
        return CGP_ECUDA;
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        set_error("batch graph instantiation failed: %s", cudaGetErrorString(e));
        return CGP_ECUDA;
    }
    b->graph = g;
    return CGP_OK;
}

}  // namespace

extern "C" int cgp_batch_create_mode(cgp_solver* const* solvers, int32_t n, int32_t cluster_size, int32_t threads,
                                     int32_t mode, cgp_stream_t stream, cgp_batch** out) {
    clear_error();
    if (!solvers || n < 1 || !out || cluster_size < 0 || cluster_size > 8 ||
        (threads != 0 && threads != 256 && threads != 512 && threads != 1024) || mode < CGP_BATCH_AUTO ||
        mode > CGP_BATCH_BRANCHES) {
        set_error("cgp_batch_create: bad arguments");
        return CGP_EINVAL;
    }
    *out = nullptr;
    cgp_batch* b = new cgp_batch();
    for (int i = 0; i < n; ++i) {
        if (!solvers[i]) {
            set_error("cgp_batch_create: null solver %d", i);
            delete b;
            return CGP_EINVAL;
        }
        b->inst.push_back(&solvers[i]->s);
    }
    // largest coarse problem first: the queue hands the long solves out early
    std::stable_sort(b->inst.begin(), b->inst.end(), [](const Solver* x, const Solver* y) { return x->nc > y->nc; });
    cudaStream_t st = (cudaStream_t)stream;
    auto fail = [&](int rc) {
        cgp_batch_destroy(b);
        return rc;
    };
    bool eligible = true;
    for (Solver* s : b->inst) eligible = eligible && batch_step_eligible(*s);
    if (mode == CGP_BATCH_WHOLE_STEP && !eligible) {
        set_error("cgp_batch_create: an instance does not qualify for the whole-step launch (needs injection "
                  "restriction, a zero or previous-increment guess and a one-launch coarse solver)");
        return fail(CGP_EINVAL);
    }
    if (mode != CGP_BATCH_BRANCHES && eligible) {
        b->whole = 1;
        const size_t ssz = batch_step_args_size();
        std::vector<char> h_step(ssz * n);
        size_t nstate = 0;
        for (int i = 0; i < n; ++i) {
            fill_batch_step_args(*b->inst[i], h_step.data() + ssz * i);
            nstate += state_doubles(*b->inst[i]);
        }
        if (cudaMalloc(&b->d_step_args, ssz * n) != cudaSuccess || cudaMalloc(&b->d_queue, 256) != cudaSuccess ||
            cudaMalloc(&b->d_state, nstate * sizeof(double)) != cudaSuccess) {
            set_error("cgp_batch_create: device allocation failed");
            return fail(CGP_ENOMEM);
        }
        if (cudaMemcpy(b->d_step_args, h_step.data(), ssz * n, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess) {
            set_error("cgp_batch_create: setup failed");
            return fail(CGP_ECUDA);
        }
        int rc = autotune_whole(b, cluster_size, threads, st);
        if (rc != CGP_OK) return fail(rc);
        rc = build_graph_whole(b);
        if (rc != CGP_OK) return fail(rc);
        *out = b;
        return CGP_OK;
    }
    const size_t asz = coarse_args_size();
    std::vector<char> h_args(asz * n);
    size_t save = 0;
    for (int i = 0; i < n; ++i) {
        fill_coarse_args(*b->inst[i], h_args.data() + asz * i);
        save += 2 * (size_t)b->inst[i]->nc;
    }
    if (cudaMalloc(&b->d_args, asz * n) != cudaSuccess || cudaMalloc(&b->d_queue, 256) != cudaSuccess ||
        cudaMalloc(&b->d_save, save * sizeof(double)) != cudaSuccess) {
        set_error("cgp_batch_create: device allocation failed");
        return fail(CGP_ENOMEM);
    }
    if (cudaMemcpy(b->d_args, h_args.data(), asz * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess) {
        set_error("cgp_batch_create: setup failed");
        return fail(CGP_ECUDA);
    }
    b->streams.resize(n, nullptr);
    b->events.resize(2 + 2 * (size_t)n, nullptr);
    for (auto& s : b->streams)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return fail(CGP_ECUDA);
    for (auto& e : b->events)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(CGP_ECUDA);
    int rc = autotune(b, cluster_size, threads, st);
    if (rc != CGP_OK) return fail(rc);
    rc = build_graph(b);
    if (rc != CGP_OK) return fail(rc);
    *out = b;
    return CGP_OK;
}

extern "C" int cgp_batch_create(cgp_solver* const* solvers, int32_t n, int32_t cluster_size, int32_t threads,
                                cgp_stream_t stream, cgp_batch** out) {
    return cgp_batch_create_mode(solvers, n, cluster_size, threads, CGP_BATCH_AUTO, stream, out);
}

extern "C" int cgp_batch_mode(const cgp_batch* b, int32_t* mode) {
    clear_error();
    if (!b || !mode) {
        set_error("cgp_batch_mode: null argument");
        return CGP_EINVAL;
    }
    *mode = b->whole ? CGP_BATCH_WHOLE_STEP : CGP_BATCH_BRANCHES;
    return CGP_OK;
}

extern "C" int cgp_batch_step(cgp_batch* b, int32_t n_steps, cgp_stream_t stream) {
    clear_error();
    if (!b || n_steps < 0) {
        set_error("cgp_batch_step: bad arguments");
        return CGP_EINVAL;
    }
    for (int i = 0; i < n_steps; ++i) CGP_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return CGP_OK;
}

extern "C" int cgp_batch_info(const cgp_batch* b, int32_t* cluster_size, int32_t* threads, int32_t* nclusters,
                              float* trial_ms, int32_t n_trials) {
    if (!b) {
        set_error("cgp_batch_info: null batch");
        return CGP_EINVAL;
    }
    if (cluster_size) *cluster_size = b->csize;
    if (threads) *threads = b->threads;
    if (nclusters) *nclusters = b->nclusters;
    if (trial_ms)
        for (int k = 0; k < n_trials && k < (int)b->trial_ms.size(); ++k) trial_ms[k] = b->trial_ms[k];
    return CGP_OK;
}

extern "C" void cgp_batch_destroy(cgp_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (auto e : b->events)
        if (e) cudaEventDestroy(e);
    if (b->origin) cudaStreamDestroy(b->origin);
    if (b->d_args) cudaFree(b->d_args);
    if (b->d_queue) cudaFree(b->d_queue);
    if (b->d_save) cudaFree(b->d_save);
    if (b->d_step_args) cudaFree(b->d_step_args);
    if (b->d_state) cudaFree(b->d_state);
    delete b;
}
