// Learned initial-guess network: sizes, parameter layout and device buffers (see mlp.cu).
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"

namespace cgp {

struct Carve;

constexpr int kHid = 64;
// parameter vector (FP32 master / bfloat16 copy): W1 [64][8], b1 [64], W2 [64][128], b2 [64], W3 [1][128], b3 [1]
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * 8;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * 2 * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + 2 * kHid;
constexpr int kMlpParams = kOffB3 + 1;

constexpr int kScaleBlocks = 64;   // blocks per sample of the RMS reduction

struct MlpBuffers {
    int n = 0, maxb = 0;
    float* scale = nullptr;                     // [batch][2]: RMS of r and q
    double* spart = nullptr;                    // [batch][kScaleBlocks][2]: block partial sums of r^2, q^2
    float *h0 = nullptr, *m0 = nullptr;         // [batch][4][n]
    float *a1 = nullptr, *m1 = nullptr;         // [batch][64][n] pre-activations / neighbour means
    float *a2 = nullptr, *m2 = nullptr;
    float* hv = nullptr;                        // [batch][n][64]: vertex-major copy for the 1-ring means
    float* out = nullptr;                       // [batch][n]
    __nv_bfloat16* params_bf = nullptr;         // bfloat16 copy used by the forward kernels
    float* params = nullptr;                    // FP32 master (biases are read from here)
    void carve(Carve& cv, int n, int batch);
    static size_t bytes(int n, int batch);
};

// inference forward pass (mlp_infer.cu, tensor-core 64 -> 64 layer) for `batch` samples of
// (r, q) (each n doubles, consecutive) into pred; mlp_infer_setup (once per process, before
// any capture) raises the shared-memory limit of its layer-2 kernel
int mlp_forward(const MlpBuffers& B, const Level& L, const double* r, const double* q, int batch, double* pred,
                cudaStream_t st, const int* gate = nullptr);
int mlp_infer_setup();

}  // namespace cgp
