// Inference of the learned-guess network (not in the paper): the forward pass of mlp.cu's
// network in four launches, with the one dense contraction (the 64 -> 64 layer) on the tensor
// cores.  The training kernels in mlp.cu keep every activation for the backward pass; this
// path keeps none and serves the step (batch 1) and cgp_mlp_forward.
//
//   scales    s_r, s_q = RMS of r and q: per-block partial sums (mlp.cu's k_mlp_scales), added
//             in a fixed order at the start of layer 1 (deterministic)
//   layer 1   per vertex: f_i = (r_i/s_r, q_i/s_q, x_i, y_i) and the 1-ring mean of f_j, 8 inputs
//             -> 64 (CUDA cores), h1 = relu(.) stored vertex-major [vertex][64] in FP32
//   layer 2   per 128-vertex tile: x_i = [h1_i; mean h1_j] (128) gathered into shared memory,
//             split x = hi + lo into two bfloat16 halves (hi = bf16(x), lo = bf16(x - hi)), and
//             a2 = W2 x (W2 bfloat16, 64 x 128) as two m16n8k16 BF16 MMAs per tile step with FP32
//             accumulation: W2 hi + W2 lo carries x to about 16 significant bits, so the layer
//             stays within ~1e-5 of FP32 arithmetic; h2 = relu(a2 + b2), vertex-major FP32
//   layer 3   one warp per vertex: [h2_i; mean h2_j] . W3 + b3 (warp sum), Phi0 = q + s_q out
//
// In a step, the kernels return at once while the coarse solve's judge has switched the
// network off (gate[0] > 0: its direction bought under 5 % of the starting residual in eight
// steps in a row; it is tried again after 64 steps).
// The 1-ring means add neighbours in CSR order and multiply by 1/deg, as the training path does.
#include <cuda_bf16.h>

#include "mlp.cuh"
#include "solver.cuh"

namespace cgp {

namespace {

constexpr int kL2Rows = 128;                 // vertices per layer-2 CTA (8 warps x 16 rows)
constexpr int kL2K = 2 * kHid;               // 128 inputs
constexpr int kL2Ld = kL2K + 8;              // row stride of the staged tiles (bf16), 16-byte rows, no bank conflicts
constexpr int kL2Smem = (2 * kL2Rows + kHid) * kL2Ld * 2;   // A hi, A lo, W2

// layer 1: 8 inputs -> 64 outputs per vertex, one thread per vertex
__global__ void __launch_bounds__(128) k_inf_layer1(int n, const int32_t* __restrict__ rowptr,
                                                    const int32_t* __restrict__ col, const double* __restrict__ r,
                                                    const double* __restrict__ q, const double* __restrict__ xy,
                                                    const double* __restrict__ spart, int nblk,
                                                    float* __restrict__ scale,
                                                    const __nv_bfloat16* __restrict__ W1, const float* __restrict__ b1,
                                                    float* __restrict__ h1, const int* __restrict__ gate) {
    if (gate && *gate > 0) return;   // the solve's judge has switched the network off for now
    __shared__ float w[kHid][8];
    __shared__ float bias[kHid];
    __shared__ double inv_scale[2];
    for (int e = threadIdx.x; e < kHid * 8; e += blockDim.x) w[e / 8][e % 8] = __bfloat162float(W1[e]);
    for (int e = threadIdx.x; e < kHid; e += blockDim.x) bias[e] = b1[e];
    if (threadIdx.x < 32) {
        // the feature scales: RMS of r and of q from the per-block partial sums (the same
        // sums, in the same order, as the training path's k_mlp_scales_fin); block 0 keeps
        // them for the output layer
        double s0 = 0.0, s1 = 0.0;
        for (int k = threadIdx.x; k < nblk; k += 32) {
            s0 += spart[2 * k];
            s1 += spart[2 * k + 1];
        }
        s0 = warp_sum(s0);
        s1 = warp_sum(s1);
        if (threadIdx.x == 0) {
            const double sr = sqrt(s0 / n), sq = sqrt(s1 / n);
            const float f0 = sr > 0.0 ? (float)sr : 1.0f, f1 = sq > 0.0 ? (float)sq : 1.0f;
            inv_scale[0] = 1.0 / (double)f0;   // one FP64 reciprocal per CTA: this GPU's FP64 divide is slow
            inv_scale[1] = 1.0 / (double)f1;
            if (blockIdx.x == 0) {
                scale[0] = f0;
                scale[1] = f1;
            }
        }
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double is0 = inv_scale[0], is1 = inv_scale[1];
    auto feat = [&](int j, float (&f)[4]) {
        f[0] = (float)(r[j] * is0);
        f[1] = (float)(q[j] * is1);
        f[2] = (float)xy[2 * j];
        f[3] = (float)xy[2 * j + 1];
    };
    float x[8];
    float own[4];
    feat(i, own);
    float m[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int deg = 0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int j = col[e];
        if (j == i) continue;
        ++deg;
        float f[4];
        feat(j, f);
#pragma unroll
        for (int k = 0; k < 4; ++k) m[k] += f[k];
    }
    const float inv = deg ? 1.0f / deg : 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        x[k] = own[k];
        x[4 + k] = m[k] * inv;
    }
    float4* out = reinterpret_cast<float4*>(h1 + (size_t)i * kHid);
#pragma unroll
    for (int o = 0; o < kHid; o += 4) {
        float a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float s = bias[o + u];
#pragma unroll
            for (int k = 0; k < 8; ++k) s += w[o + u][k] * x[k];
            a[u] = fmaxf(s, 0.0f);
        }
        out[o / 4] = make_float4(a[0], a[1], a[2], a[3]);
    }
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t (&r)[2]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// layer 2 on the tensor cores (see the file comment); 256 threads, kL2Smem bytes of dynamic smem
__global__ void __launch_bounds__(256) k_inf_layer2(int n, const int32_t* __restrict__ rowptr,
                                                    const int32_t* __restrict__ col, const float* __restrict__ h1,
                                                    const __nv_bfloat16* __restrict__ W2,
                                                    const float* __restrict__ b2, float* __restrict__ h2,
                                                    const int* __restrict__ gate) {
    if (gate && *gate > 0) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* ahi = reinterpret_cast<__nv_bfloat16*>(smem);
    __nv_bfloat16* alo = ahi + kL2Rows * kL2Ld;
    __nv_bfloat16* ws = alo + kL2Rows * kL2Ld;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int i0 = blockIdx.x * kL2Rows;
    // W2 (64 x 128 bf16) into shared rows of kL2Ld: 16-byte pieces
    for (int e = threadIdx.x; e < kHid * kL2K / 8; e += blockDim.x) {
        const int o = e / (kL2K / 8), k8 = e % (kL2K / 8);
        *reinterpret_cast<uint4*>(ws + o * kL2Ld + 8 * k8) = reinterpret_cast<const uint4*>(W2)[e];
    }
    // gather: thread t takes row t / 2 of the tile and features 32 (t % 2) .. 32 (t % 2) + 31
    // of the own row and of the 1-ring mean (16-byte loads), so the neighbour loads of all 128
    // rows are in flight together; then the bf16 hi and lo halves go to the shared tiles
    {
        const int row = threadIdx.x >> 1, part = threadIdx.x & 1, i = i0 + row;
        float own[32], mean[32];
#pragma unroll
        for (int f = 0; f < 32; ++f) own[f] = mean[f] = 0.0f;
        if (i < n) {
            const float4* hv4 = reinterpret_cast<const float4*>(h1);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float4 v = hv4[(size_t)i * (kHid / 4) + 8 * part + u];
                own[4 * u] = v.x;
                own[4 * u + 1] = v.y;
                own[4 * u + 2] = v.z;
                own[4 * u + 3] = v.w;
            }
            int deg = 0;
            for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                const int j = col[e];
                if (j == i) continue;
                ++deg;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float4 v = hv4[(size_t)j * (kHid / 4) + 8 * part + u];
                    mean[4 * u] += v.x;
                    mean[4 * u + 1] += v.y;
                    mean[4 * u + 2] += v.z;
                    mean[4 * u + 3] += v.w;
                }
            }
            const float inv = deg ? 1.0f / deg : 0.0f;
#pragma unroll
            for (int f = 0; f < 32; ++f) mean[f] *= inv;
        }
        // hi = bf16(x), lo = bf16(x - hi), eight values per 16-byte store
        auto put = [&](const float (&x)[32], int col0) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float a = x[8 * u + 2 * v], b = x[8 * u + 2 * v + 1];
                    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
                    const float2 hf = __bfloat1622float2(h);
                    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
                    hw[v] = *reinterpret_cast<const uint32_t*>(&h);
                    lw[v] = *reinterpret_cast<const uint32_t*>(&l);
                }
                const int off = row * kL2Ld + col0 + 8 * u;
                *reinterpret_cast<uint4*>(ahi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4*>(alo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
        };
        put(own, 32 * part);
        put(mean, kHid + 32 * part);
    }
    __syncthreads();
    // MMA: warp w computes rows 16 w .. 16 w + 15 x all 64 outputs (8 n-tiles of 8)
    float acc[8][4];
#pragma unroll
    for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[t][u] = 0.0f;
    const uint32_t ahi_s = (uint32_t)__cvta_generic_to_shared(ahi), alo_s = (uint32_t)__cvta_generic_to_shared(alo);
    const uint32_t ws_s = (uint32_t)__cvta_generic_to_shared(ws);
    // ldmatrix row addresses: A x4 (rows 0-7 / 8-15, columns k0 / k0 + 8); B x2 (n rows, k0 / k0 + 8)
    const int arow = 16 * wid + (lane & 7) + ((lane >> 3) & 1) * 8, acol = (lane >> 4) * 8;
    const int brow = lane & 7, bcol = ((lane >> 3) & 1) * 8;
#pragma unroll
    for (int k0 = 0; k0 < kL2K; k0 += 16) {
        uint32_t ah[4], al[4];
        const uint32_t aoff = (uint32_t)((arow * kL2Ld + k0 + acol) * 2);
        ldsm_x4(ahi_s + aoff, ah);
        ldsm_x4(alo_s + aoff, al);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            uint32_t b[2];
            ldsm_x2(ws_s + (uint32_t)(((8 * t + brow) * kL2Ld + k0 + bcol) * 2), b);
            mma_bf16(acc[t], ah, b);
            mma_bf16(acc[t], al, b);
        }
    }
    // epilogue: + b2, relu; C fragment rows g and g + 8, columns 8 t + 2 c, + 1
    const int g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int i = i0 + 16 * wid + g + 8 * half;
        if (i >= n) continue;
        float* out = h2 + (size_t)i * kHid;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int o = 8 * t + 2 * c;
            const float v0 = fmaxf(acc[t][2 * half] + b2[o], 0.0f);
            const float v1 = fmaxf(acc[t][2 * half + 1] + b2[o + 1], 0.0f);
            *reinterpret_cast<float2*>(out + o) = make_float2(v0, v1);
        }
    }
}

// layer 3 and the prediction: one warp per vertex
__global__ void __launch_bounds__(256) k_inf_layer3(int n, const int32_t* __restrict__ rowptr,
                                                    const int32_t* __restrict__ col, const float* __restrict__ h2,
                                                    const __nv_bfloat16* __restrict__ W3,
                                                    const float* __restrict__ b3, const float* __restrict__ scale,
                                                    const double* __restrict__ q, double* __restrict__ pred,
                                                    const int* __restrict__ gate) {
    if (gate && *gate > 0) return;
    const int lane = threadIdx.x & 31;
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (i >= n) return;
    const float2* hv = reinterpret_cast<const float2*>(h2);
    const float2 own = hv[(size_t)i * (kHid / 2) + lane];
    float2 mean = make_float2(0.0f, 0.0f);
    int deg = 0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int j = col[e];
        if (j == i) continue;
        ++deg;
        const float2 x = hv[(size_t)j * (kHid / 2) + lane];
        mean.x += x.x;
        mean.y += x.y;
    }
    const float inv = deg ? 1.0f / deg : 0.0f;
    const float s = __bfloat162float(W3[2 * lane]) * own.x + __bfloat162float(W3[2 * lane + 1]) * own.y +
                    __bfloat162float(W3[kHid + 2 * lane]) * (mean.x * inv) +
                    __bfloat162float(W3[kHid + 2 * lane + 1]) * (mean.y * inv);
    const float tot = warp_sum(s);
    if (lane == 0) pred[i] = q[i] + (double)scale[1] * (double)(tot + b3[0]);
}

}  // namespace

// mlp.cu's RMS kernels
__global__ void k_mlp_scales(int n, const double* __restrict__ r, const double* __restrict__ q,
                             double* __restrict__ spart);
__global__ void k_mlp_scales_fin(int n, int nblk, const double* __restrict__ spart, float* __restrict__ scale);

int mlp_infer_setup() {
    CGP_CUDA(cudaFuncSetAttribute(k_inf_layer2, cudaFuncAttributeMaxDynamicSharedMemorySize, kL2Smem));
    return CGP_OK;
}

int mlp_forward(const MlpBuffers& B, const Level& L, const double* r, const double* q, int batch, double* pred,
                cudaStream_t st, const int* gate) {
    const int n = B.n;
    // activations: h1 in hv, h2 in m1 (both [vertex][64] FP32 here)
    for (int b = 0; b < batch; ++b) {
        const double* rb = r + (size_t)b * n;
        const double* qb = q + (size_t)b * n;
        float* sc = B.scale + 2 * b;
        k_mlp_scales<<<dim3(kScaleBlocks, 1), kBlock, 0, st>>>(n, rb, qb, B.spart);
        k_inf_layer1<<<blocks_for(n, 128), 128, 0, st>>>(n, L.rowptr, L.col, rb, qb, L.xy, B.spart, kScaleBlocks, sc,
                                                         B.params_bf + kOffW1, B.params + kOffB1, B.hv, gate);
        k_inf_layer2<<<blocks_for(n, kL2Rows), 256, kL2Smem, st>>>(n, L.rowptr, L.col, B.hv, B.params_bf + kOffW2,
                                                                   B.params + kOffB2, B.m1, gate);
        if (pred)
            k_inf_layer3<<<blocks_for((int64_t)n * 32, 256), 256, 0, st>>>(
                n, L.rowptr, L.col, B.m1, B.params_bf + kOffW3, B.params + kOffB3, sc, qb, pred + (size_t)b * n, gate);
    }
    CGP_LAUNCH_CHECK();
    return CGP_OK;
}

}  // namespace cgp
