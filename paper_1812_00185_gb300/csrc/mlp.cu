// Learned initial guess for the coarse Poisson solve (not in the paper): a per-vertex MLP
// on the pressure-increment mesh with 1-ring mean aggregation, 3 layers, widths
// 4 -> 64 -> 64 -> 1, bfloat16 weights with FP32 arithmetic, FP32 master weights and Adam.
//
//   f_i   = (r_i / s_r, q_i / s_q, x_i, y_i)       r: coarse rhs, q: previous Phi_c, s: RMS
//   a_l,i = W_l [h_{l-1,i}; mean_{j in N(i), j != i} h_{l-1,j}] + b_l,   h_l = relu(a_l) (l < 3)
//   Phi0_i = q_i + s_q * a_3,i
//   loss  = mean over samples and vertices of (a_3,i - clip((Phi*_i - q_i) / s_q, -10, 10))^2
//           (the clip keeps transient steps, where Phi changes by many times its own size,
//           from dominating the fit; there the residual judge falls back to q anyway)
//
// Activations are stored feature-major per sample ([sample][feature][vertex]) so that a
// warp's 32 vertices read consecutive addresses.  Weight gradients are reduced in two
// deterministic passes (per-block partials, then a fixed-order sum).
#include <cuda_bf16.h>

#include "flows.cuh"
#include "mlp.cuh"
#include "solver.cuh"

namespace cgp {

// ---------------------------------------------------------------- forward kernels
// per-sample RMS of r and q: kScaleBlocks blocks per sample write partial sums of squares,
// then one warp per sample adds them in block order (deterministic)
__global__ void __launch_bounds__(kBlock) k_mlp_scales(int n, const double* __restrict__ r, const double* __restrict__ q,
                                                     double* __restrict__ spart) {
    const int b = blockIdx.y;
    double a0 = 0.0, a1 = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double rv = r[(size_t)b * n + i], qv = q[(size_t)b * n + i];
        a0 += rv * rv;
        a1 += qv * qv;
    }
    __shared__ double sm[kBlock / 32][2];
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sm[wid][0] = a0;
        sm[wid][1] = a1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s0 += sm[w][0];
            s1 += sm[w][1];
        }
        spart[((size_t)b * gridDim.x + blockIdx.x) * 2] = s0;
        spart[((size_t)b * gridDim.x + blockIdx.x) * 2 + 1] = s1;
    }
}

__global__ void k_mlp_scales_fin(int n, int nblk, const double* __restrict__ spart, float* __restrict__ scale) {
    const int b = blockIdx.x, lane = threadIdx.x;
    double s0 = 0.0, s1 = 0.0;
    for (int k = lane; k < nblk; k += 32) {
        s0 += spart[((size_t)b * nblk + k) * 2];
        s1 += spart[((size_t)b * nblk + k) * 2 + 1];
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    if (lane == 0) {
        const double sr = sqrt(s0 / n), sq = sqrt(s1 / n);
        scale[2 * b] = sr > 0.0 ? (float)sr : 1.0f;
        scale[2 * b + 1] = sq > 0.0 ? (float)sq : 1.0f;
    }
}

__global__ void k_mlp_features(int n, int batch, const double* __restrict__ r, const double* __restrict__ q,
                               const double* __restrict__ xy, const float* __restrict__ scale, float* __restrict__ h0) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * batch) return;
    const int b = (int)(t / n), i = (int)(t % n);
    float* o = h0 + (size_t)b * 4 * n;
    o[i] = (float)(r[t] / (double)scale[2 * b]);
    o[n + i] = (float)(q[t] / (double)scale[2 * b + 1]);
    o[2 * n + i] = (float)xy[2 * i];
    o[3 * n + i] = (float)xy[2 * i + 1];
}

// m[b][f][i] = mean over the 1-ring (i excluded) of act(h[b][f][j]); act = relu if RELU
template <int F, bool RELU>
__global__ void k_mlp_nmean(int n, int batch, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const float* __restrict__ h, float* __restrict__ m) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * batch) return;
    const int b = (int)(t / n), i = (int)(t % n);
    const float* hb = h + (size_t)b * F * n;
    float* mb = m + (size_t)b * F * n;
    float acc[F];
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f] = 0.0f;
    int deg = 0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int j = col[e];
        if (j == i) continue;
        ++deg;
#pragma unroll
        for (int f = 0; f < F; ++f) {
            float v = hb[(size_t)f * n + j];
            acc[f] += RELU ? fmaxf(v, 0.0f) : v;
        }
    }
    const float inv = deg ? 1.0f / deg : 0.0f;
#pragma unroll
    for (int f = 0; f < F; ++f) mb[(size_t)f * n + i] = acc[f] * inv;
}

// The 64-wide 1-ring means read vertex-major: a feature-major gather reads one 4-byte value
// per 32-byte sector for each (neighbour, feature); a vertex-major one reads each neighbour's
// 64 features as one 256-byte run.  The dense layer that produces the features also writes
// this copy, hv[b][i][f] = relu(a[b][f][i]).
// m[b][f][i] = mean over the 1-ring (i excluded) of hv[b][j][f] for 32 vertices per block: a
// warp per vertex (lanes over features, two each, neighbours in CSR order as in
// k_mlp_nmean), written back feature-major through shared memory
__global__ void __launch_bounds__(256) k_mlp_nmean64(int n, const int32_t* __restrict__ rowptr,
                                                    const int32_t* __restrict__ col, const float* __restrict__ hv,
                                                    float* __restrict__ m) {
    static_assert(kHid == 64, "two features per lane");
    __shared__ float tile[kHid][33];
    const int b = blockIdx.y, i0 = blockIdx.x * 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float2* vb = reinterpret_cast<const float2*>(hv + (size_t)b * n * kHid);
    for (int v = wid; v < 32; v += 8) {
        const int i = i0 + v;
        float ax = 0.0f, ay = 0.0f;
        int deg = 0;
        if (i < n) {
            for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                const int j = col[e];
                if (j == i) continue;
                ++deg;
                const float2 x = vb[(size_t)j * (kHid / 2) + lane];
                ax += x.x;
                ay += x.y;
            }
        }
        const float inv = deg ? 1.0f / deg : 0.0f;
        tile[2 * lane][v] = ax * inv;
        tile[2 * lane + 1][v] = ay * inv;
    }
    __syncthreads();
    float* mb = m + (size_t)b * kHid * n;
    for (int f = wid; f < kHid; f += 8) {
        const int i = i0 + lane;
        if (i < n) mb[(size_t)f * n + i] = tile[f][lane];
    }
}

// a[b][o][i] = sum_k W[o][k] x_k + bias[o], x = [act(h); m] (2*FIN inputs), summed in k
// order; with VOUT also hv[b][i][o] = relu(a[b][o][i]) (the vertex-major copy the next
// 1-ring mean gathers).  W (bf16, row-major FOUT x 2*FIN) is staged per block as FP32
// columns wt[k][o]: lane l of a warp loads 8 consecutive k of row o = l (16 bytes) and
// writes them down column l, so the transposed writes are free of bank conflicts.  With
// FOUT >= 32 two threads share a vertex (the first half of the block takes outputs
// [0, FOUT/2), the second half the rest, so a warp reads one wt row as a broadcast).  Each
// thread loads its inputs in chunks, the next chunk while it multiplies the current one,
// so the latency of the feature-major input loads overlaps the FMAs.
template <int FOUT>
__host__ __device__ constexpr int dense_vertices_per_block() { return FOUT >= 32 ? 64 : 128; }   // of 128 threads

template <int FIN, int FOUT, bool RELU_IN, bool VOUT>
__global__ void __launch_bounds__(128) k_mlp_dense(int n, int batch, const __nv_bfloat16* __restrict__ W,
                                                   const float* __restrict__ bias, const float* __restrict__ h,
                                                   const float* __restrict__ m, float* __restrict__ a,
                                                   float* __restrict__ hv) {
    constexpr int K = 2 * FIN;
    constexpr int VB = dense_vertices_per_block<FOUT>();
    constexpr int OS = 128 / VB;                        // threads per vertex
    constexpr int FO = FOUT / OS;                       // outputs per thread
    constexpr int LD = FOUT == 1 ? 1 : FOUT + 4;        // row stride of wt (16-byte rows)
    constexpr int KCMAX = FO == 1 ? 32 : 16;
    constexpr int KC = FIN < KCMAX ? FIN : KCMAX;       // inputs loaded per chunk
    constexpr int NV8 = K * FOUT / 8;                   // 16-byte pieces of W
    static_assert(FOUT % OS == 0 && (FO == 1 || FO % 4 == 0) && FIN % KC == 0 && K % 8 == 0, "dense layer shape");
    static_assert(!VOUT || FO % 4 == 0, "vertex-major copy in 16-byte stores");
    __shared__ __align__(16) float wt[K][LD];
    const uint4* W8 = reinterpret_cast<const uint4*>(W);
#pragma unroll
    for (int r = 0; r < (NV8 + 127) / 128; ++r) {
        const int f = threadIdx.x + 128 * r;
        if (f < NV8) {
            const int o = f % FOUT, k0 = 8 * (f / FOUT);
            const uint4 u = __ldg(W8 + (o * K + k0) / 8);
            const uint32_t wd[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 w2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wd[j]));
                wt[k0 + 2 * j][o] = w2.x;
                wt[k0 + 2 * j + 1][o] = w2.y;
            }
        }
    }
    __syncthreads();
    const int part = threadIdx.x / VB;
    const int64_t t = blockIdx.x * (int64_t)VB + threadIdx.x % VB;
    if (t >= (int64_t)n * batch) return;
    const int b = (int)(t / n), i = (int)(t % n);
    const int o0 = part * FO;
    float acc[FO];
#pragma unroll
    for (int o = 0; o < FO; ++o) acc[o] = bias[o0 + o];
    // chunk c holds inputs k = c KC .. c KC + KC - 1: the first FIN / KC chunks come from h
    // (with the ReLU when RELU_IN), the rest from m; two register buffers alternate, so the
    // loads of chunk c + 1 are in flight while chunk c is multiplied
    constexpr int NCH = K / KC;
    static_assert(NCH % 2 == 0, "chunks come in pairs");
    const float* hb = h + (size_t)b * FIN * n + i;
    const float* mb = m + (size_t)b * FIN * n + i;
    auto load = [&](float (&xs)[KC], int c) {
        const bool from_h = c < FIN / KC;
        const float* src = from_h ? hb + (size_t)c * KC * n : mb + (size_t)(c - FIN / KC) * KC * n;
#pragma unroll
        for (int u = 0; u < KC; ++u) {
            const float x = src[(size_t)u * n];
            xs[u] = (RELU_IN && from_h) ? fmaxf(x, 0.0f) : x;
        }
    };
    auto mul = [&](const float (&xs)[KC], int c) {
#pragma unroll
        for (int u = 0; u < KC; ++u) {
            const float* wr = &wt[c * KC + u][o0];
            if constexpr (FO % 4 == 0) {
#pragma unroll
                for (int o = 0; o < FO; o += 4) {
                    const float4 w4 = *reinterpret_cast<const float4*>(wr + o);
                    acc[o] += w4.x * xs[u];
                    acc[o + 1] += w4.y * xs[u];
                    acc[o + 2] += w4.z * xs[u];
                    acc[o + 3] += w4.w * xs[u];
                }
            } else {
#pragma unroll
                for (int o = 0; o < FO; ++o) acc[o] += wr[o] * xs[u];
            }
        }
    };
    float xa[KC], xb[KC];
    load(xa, 0);
    for (int c = 0; c < NCH; c += 2) {
        load(xb, c + 1);
        mul(xa, c);
        if (c + 2 < NCH) load(xa, c + 2);
        mul(xb, c + 1);
    }
    float* ab = a + (size_t)b * FOUT * n;
#pragma unroll
    for (int o = 0; o < FO; ++o) ab[(size_t)(o0 + o) * n + i] = acc[o];
    if constexpr (VOUT) {
        float4* vr = reinterpret_cast<float4*>(hv + ((size_t)b * n + i) * FOUT + o0);
#pragma unroll
        for (int o = 0; o < FO; o += 4)
            vr[o / 4] = make_float4(fmaxf(acc[o], 0.0f), fmaxf(acc[o + 1], 0.0f), fmaxf(acc[o + 2], 0.0f),
                                    fmaxf(acc[o + 3], 0.0f));
    }
}

// Phi0 = q + s_q * out (double)
__global__ void k_mlp_predict(int n, int batch, const double* __restrict__ q, const float* __restrict__ out,
                              const float* __restrict__ scale, double* __restrict__ pred) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * batch) return;
    const int b = (int)(t / n);
    pred[t] = q[t] + (double)scale[2 * b + 1] * (double)out[t];
}

// ---------------------------------------------------------------- backward kernels
constexpr double kTargetClip = 10.0;

// g3 = dL/da3 = 2 (a3 - clip((t - q)/s_q)) / (n * batch); loss partials per block
__global__ void __launch_bounds__(kBlock) k_mlp_loss(int n, int batch, const double* __restrict__ q,
                                                   const double* __restrict__ tgt, const float* __restrict__ out,
                                                   const float* __restrict__ scale, float* __restrict__ g3,
                                                   double* __restrict__ partials, unsigned int* ticket,
                                                   float* __restrict__ loss) {
    double acc[1] = {0.0};
    const int64_t total = (int64_t)n * batch;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / n);
        const double tn = fmin(fmax((tgt[t] - q[t]) / (double)scale[2 * b + 1], -kTargetClip), kTargetClip);
        const double d = (double)out[t] - tn;
        acc[0] += d * d;
        g3[t] = (float)(2.0 * d / (double)total);
    }
    double tot[1];
    if (grid_sum<1>(acc, partials, ticket, tot) && threadIdx.x == 0) *loss = (float)(tot[0] / (double)total);
}

// gx = W^T ga: gh (the h part, k < FIN) and gm (the mean part)
template <int FIN, int FOUT>
__global__ void __launch_bounds__(128) k_mlp_dense_bwd(int n, int batch, const __nv_bfloat16* __restrict__ W,
                                                       const float* __restrict__ ga, float* __restrict__ gh,
                                                       float* __restrict__ gm) {
    constexpr int K = 2 * FIN;
    __shared__ float w[K][FOUT];
    for (int e = threadIdx.x; e < K * FOUT; e += blockDim.x) {
        const int o = e / K, k = e % K;
        w[k][o] = __bfloat162float(W[e]);
    }
    __syncthreads();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * batch) return;
    const int b = (int)(t / n), i = (int)(t % n);
    const float* gab = ga + (size_t)b * FOUT * n;
    float g[FOUT];
#pragma unroll
    for (int o = 0; o < FOUT; ++o) g[o] = gab[(size_t)o * n + i];
    float* ghb = gh + (size_t)b * FIN * n;
    float* gmb = gm + (size_t)b * FIN * n;
    for (int k = 0; k < K; ++k) {
        float s = 0.0f;
#pragma unroll
        for (int o = 0; o < FOUT; ++o) s += w[k][o] * g[o];
        if (k < FIN) ghb[(size_t)k * n + i] = s;
        else gmb[(size_t)(k - FIN) * n + i] = s;
    }
}

// gh[j] += sum over neighbours i of j (i != j) of gm[i] / deg(i); then ga = gh * (a > 0)
template <int F>
__global__ void k_mlp_nmean_bwd(int n, int batch, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const float* __restrict__ gm, const float* __restrict__ a_prev, float* __restrict__ gh) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * batch) return;
    const int b = (int)(t / n), j = (int)(t % n);
    const float* gmb = gm + (size_t)b * F * n;
    float* ghb = gh + (size_t)b * F * n;
    const float* ab = a_prev + (size_t)b * F * n;
    float acc[F];
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f] = ghb[(size_t)f * n + j];
    for (int e = rowptr[j]; e < rowptr[j + 1]; ++e) {
        const int i = col[e];
        if (i == j) continue;
        const float inv = 1.0f / (float)(rowptr[i + 1] - rowptr[i] - 1);
#pragma unroll
        for (int f = 0; f < F; ++f) acc[f] += gmb[(size_t)f * n + i] * inv;
    }
#pragma unroll
    for (int f = 0; f < F; ++f) ghb[(size_t)f * n + j] = ab[(size_t)f * n + j] > 0.0f ? acc[f] : 0.0f;
}

// Per-block partial weight gradients: dW[o][k] = sum_rows ga[o] x[k], db[o] = sum ga[o],
// x = [act(h); m].  Rows = (sample, vertex) pairs; block c takes rows [c*kRowsPerBlock, ...).
constexpr int kRowsPerBlock = 1024;
constexpr int kTile = 32;

template <int FIN, int FOUT, bool RELU_IN>
__global__ void __launch_bounds__(256) k_mlp_wgrad(int n, int batch, const float* __restrict__ ga,
                                                   const float* __restrict__ h, const float* __restrict__ m,
                                                   float* __restrict__ partials) {
    constexpr int K = 2 * FIN;
    constexpr int NOUT = FOUT * (K + 1);
    constexpr int PER = (NOUT + 255) / 256;
    __shared__ float gt[FOUT][kTile + 1];
    __shared__ float xt[K][kTile + 1];
    float acc[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) acc[u] = 0.0f;
    const int64_t total = (int64_t)n * batch;
    const int64_t r0 = (int64_t)blockIdx.x * kRowsPerBlock;
    for (int64_t rt = r0; rt < r0 + kRowsPerBlock && rt < total; rt += kTile) {
        // stage a tile of rows
        for (int e = threadIdx.x; e < (FOUT + K) * kTile; e += blockDim.x) {
            const int f = e / kTile, rr = e % kTile;
            const int64_t row = rt + rr;
            float v = 0.0f;
            if (row < total) {
                const int b = (int)(row / n), i = (int)(row % n);
                if (f < FOUT) {
                    v = ga[((size_t)b * FOUT + f) * n + i];
                } else {
                    const int k = f - FOUT;
                    if (k < FIN) {
                        v = h[((size_t)b * FIN + k) * n + i];
                        if (RELU_IN) v = fmaxf(v, 0.0f);
                    } else {
                        v = m[((size_t)b * FIN + (k - FIN)) * n + i];
                    }
                }
            }
            if (f < FOUT) gt[f][rr] = v;
            else xt[f - FOUT][rr] = v;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int qi = threadIdx.x + 256 * u;
            if (qi < NOUT) {
                const int o = qi / (K + 1), k = qi % (K + 1);
                float s = 0.0f;
                if (k < K) {
#pragma unroll 8
                    for (int rr = 0; rr < kTile; ++rr) s += gt[o][rr] * xt[k][rr];
                } else {
#pragma unroll 8
                    for (int rr = 0; rr < kTile; ++rr) s += gt[o][rr];
                }
                acc[u] += s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int qi = threadIdx.x + 256 * u;
        if (qi < NOUT) partials[(size_t)blockIdx.x * NOUT + qi] = acc[u];
    }
}

// grad[W offset + o*K + k] / grad[b offset + o] = sum over blocks (fixed order) of the partials
__global__ void k_mlp_wgrad_reduce(int nblk, int fout, int K, const float* __restrict__ partials,
                                   float* __restrict__ gW, float* __restrict__ gb) {
    const int nout = fout * (K + 1);
    const int qi = blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= nout) return;
    double s = 0.0;
    for (int c = 0; c < nblk; ++c) s += partials[(size_t)c * nout + qi];
    const int o = qi / (K + 1), k = qi % (K + 1);
    if (k < K) gW[o * K + k] = (float)s;
    else gb[o] = (float)s;
}

__global__ void k_mlp_adam(int np, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, int t, float lr, __nv_bfloat16* __restrict__ pbf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.0f - powf(b1, (float)t));
    const float vh = vi / (1.0f - powf(b2, (float)t));
    const float pi = p[i] - lr * mh / (sqrtf(vh) + eps);
    p[i] = pi;
    pbf[i] = __float2bfloat16_rn(pi);
}

__global__ void k_mlp_to_bf16(int np, const float* __restrict__ p, __nv_bfloat16* __restrict__ pbf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < np) pbf[i] = __float2bfloat16_rn(p[i]);
}

// ---------------------------------------------------------------- host side
size_t MlpBuffers::bytes(int n, int batch) {
    Carve cv(nullptr);
    MlpBuffers B;
    B.carve(cv, n, batch);
    return cv.off;
}

void MlpBuffers::carve(Carve& cv, int n_, int batch) {
    n = n_;
    maxb = batch;
    const size_t nb = (size_t)n * batch;
    scale = cv.take<float>(2 * (size_t)batch);
    spart = cv.take<double>(2 * (size_t)kScaleBlocks * batch);
    h0 = cv.take<float>(4 * nb);
    m0 = cv.take<float>(4 * nb);
    a1 = cv.take<float>(kHid * nb);
    m1 = cv.take<float>(kHid * nb);
    a2 = cv.take<float>(kHid * nb);
    m2 = cv.take<float>(kHid * nb);
    hv = cv.take<float>(kHid * nb);
    out = cv.take<float>(nb);
    params_bf = cv.take<__nv_bfloat16>(kMlpParams);
    params = cv.take<float>(kMlpParams);
}

// the training forward pass: every activation kept (feature-major) for mlp_backward
static int mlp_forward_train(const MlpBuffers& B, const Level& L, const double* r, const double* q, int batch,
                             double* pred, cudaStream_t st) {
    const int n = B.n;
    const int64_t nb = (int64_t)n * batch;
    const int g = blocks_for(nb);
    const int gh = blocks_for(nb, dense_vertices_per_block<kHid>());
    const int g1 = blocks_for(nb, dense_vertices_per_block<1>());
    k_mlp_scales<<<dim3(kScaleBlocks, batch), kBlock, 0, st>>>(n, r, q, B.spart);
    k_mlp_scales_fin<<<batch, 32, 0, st>>>(n, kScaleBlocks, B.spart, B.scale);
    k_mlp_features<<<g, kBlock, 0, st>>>(n, batch, r, q, L.xy, B.scale, B.h0);
    k_mlp_nmean<4, false><<<g, kBlock, 0, st>>>(n, batch, L.rowptr, L.col, B.h0, B.m0);
    k_mlp_dense<4, kHid, false, true><<<gh, 128, 0, st>>>(n, batch, B.params_bf + kOffW1, B.params + kOffB1, B.h0,
                                                           B.m0, B.a1, B.hv);
    const dim3 gm((n + 31) / 32, batch);
    k_mlp_nmean64<<<gm, 256, 0, st>>>(n, L.rowptr, L.col, B.hv, B.m1);
    k_mlp_dense<kHid, kHid, true, true><<<gh, 128, 0, st>>>(n, batch, B.params_bf + kOffW2, B.params + kOffB2, B.a1,
                                                             B.m1, B.a2, B.hv);
    k_mlp_nmean64<<<gm, 256, 0, st>>>(n, L.rowptr, L.col, B.hv, B.m2);
    k_mlp_dense<kHid, 1, true, false><<<g1, 128, 0, st>>>(n, batch, B.params_bf + kOffW3, B.params + kOffB3, B.a2,
                                                           B.m2, B.out, nullptr);
    if (pred) k_mlp_predict<<<g, kBlock, 0, st>>>(n, batch, q, B.out, B.scale, pred);
    CGP_LAUNCH_CHECK();
    return CGP_OK;
}

}  // namespace cgp

using namespace cgp;

struct cgp_mlp {
    const cgp_mesh* mesh = nullptr;
    int level = 0;
    MlpBuffers B;
    void* mem = nullptr;          // one cudaMalloc: buffers + training state
    float *grad = nullptr, *adam_m = nullptr, *adam_v = nullptr, *wpart = nullptr;
    float *gA = nullptr, *gB = nullptr, *gM = nullptr, *g3 = nullptr, *loss = nullptr;
    double* partials = nullptr;
    unsigned int* ticket = nullptr;
    int adam_t = 0;
    int nblk = 0;
};

extern "C" int cgp_mlp_param_count(void) { return kMlpParams; }

extern "C" int cgp_mlp_create(const cgp_mesh* mesh, int32_t level, int32_t max_batch, cgp_mlp** out) {
    clear_error();
    if (!mesh || !out || level < 0 || level > mesh->n_levels || max_batch < 1) {
        set_error("cgp_mlp_create: bad arguments");
        return CGP_EINVAL;
    }
    *out = nullptr;
    cgp_mlp* m = new cgp_mlp();
    m->mesh = mesh;
    m->level = level;
    const int n = mesh->lev[level].nv;
    const int64_t nb = (int64_t)n * max_batch;
    m->nblk = (int)((nb + kRowsPerBlock - 1) / kRowsPerBlock);
    auto layout = [&](Carve& cv) {
        m->B.carve(cv, n, max_batch);
        m->grad = cv.take<float>(kMlpParams);
        m->adam_m = cv.take<float>(kMlpParams);
        m->adam_v = cv.take<float>(kMlpParams);
        m->wpart = cv.take<float>((size_t)m->nblk * kHid * (2 * kHid + 1));
        m->gA = cv.take<float>(kHid * nb);
        m->gB = cv.take<float>(kHid * nb);
        m->gM = cv.take<float>(kHid * nb);
        m->g3 = cv.take<float>(nb);
        m->loss = cv.take<float>(1);
        m->partials = cv.take<double>(4096);
        m->ticket = cv.take<unsigned int>(4);
    };
    Carve c0(nullptr);
    layout(c0);
    cudaError_t e = cudaMalloc(&m->mem, c0.off + 256);
    if (e != cudaSuccess) {
        set_error("cudaMalloc(%zu) failed: %s", c0.off, cudaGetErrorString(e));
        delete m;
        return CGP_ENOMEM;
    }
    Carve c1((void*)(((uintptr_t)m->mem + 255) & ~(uintptr_t)255));
    layout(c1);
    if (cudaMemset(m->adam_m, 0, sizeof(float) * kMlpParams) != cudaSuccess ||
        cudaMemset(m->adam_v, 0, sizeof(float) * kMlpParams) != cudaSuccess ||
        cudaMemset(m->ticket, 0, 4 * sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(m->B.params, 0, sizeof(float) * kMlpParams) != cudaSuccess ||
        cudaMemset(m->B.params_bf, 0, sizeof(__nv_bfloat16) * kMlpParams) != cudaSuccess) {
        set_error("cgp_mlp_create: initialisation failed");
        cudaFree(m->mem);
        delete m;
        return CGP_ECUDA;
    }
    {
        const int rc = mlp_infer_setup();
        if (rc != CGP_OK) {
            cudaFree(m->mem);
            delete m;
            return rc;
        }
    }
    *out = m;
    return CGP_OK;
}

extern "C" void cgp_mlp_destroy(cgp_mlp* m) {
    if (!m) return;
    if (m->mem) cudaFree(m->mem);
    delete m;
}

extern "C" int cgp_mlp_set_params(cgp_mlp* m, const float* params, int32_t where, cgp_stream_t stream) {
    clear_error();
    if (!m || !params) {
        set_error("cgp_mlp_set_params: null argument");
        return CGP_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CGP_CUDA(cudaMemcpyAsync(m->B.params, params, sizeof(float) * kMlpParams,
                             where == CGP_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    k_mlp_to_bf16<<<blocks_for(kMlpParams), kBlock, 0, st>>>(kMlpParams, m->B.params, m->B.params_bf);
    CGP_LAUNCH_CHECK();
    CGP_CUDA(cudaMemsetAsync(m->adam_m, 0, sizeof(float) * kMlpParams, st));
    CGP_CUDA(cudaMemsetAsync(m->adam_v, 0, sizeof(float) * kMlpParams, st));
    m->adam_t = 0;
    if (where == CGP_HOST) CGP_CUDA(cudaStreamSynchronize(st));
    return CGP_OK;
}

extern "C" int cgp_mlp_copy_state(cgp_mlp* dst, const cgp_mlp* src, cgp_stream_t stream) {
    clear_error();
    if (!dst || !src) {
        set_error("cgp_mlp_copy_state: null argument");
        return CGP_EINVAL;
    }
    if (dst == src) return CGP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t fb = sizeof(float) * kMlpParams;
    CGP_CUDA(cudaMemcpyAsync(dst->B.params, src->B.params, fb, cudaMemcpyDeviceToDevice, st));
    CGP_CUDA(cudaMemcpyAsync(dst->B.params_bf, src->B.params_bf, sizeof(__nv_bfloat16) * kMlpParams,
                             cudaMemcpyDeviceToDevice, st));
    CGP_CUDA(cudaMemcpyAsync(dst->adam_m, src->adam_m, fb, cudaMemcpyDeviceToDevice, st));
    CGP_CUDA(cudaMemcpyAsync(dst->adam_v, src->adam_v, fb, cudaMemcpyDeviceToDevice, st));
    dst->adam_t = src->adam_t;
    return CGP_OK;
}

extern "C" int cgp_mlp_get_params(cgp_mlp* m, float* params, int32_t where, cgp_stream_t stream) {
    clear_error();
    if (!m || !params) {
        set_error("cgp_mlp_get_params: null argument");
        return CGP_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CGP_CUDA(cudaMemcpyAsync(params, m->B.params, sizeof(float) * kMlpParams,
                             where == CGP_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    if (where == CGP_HOST) CGP_CUDA(cudaStreamSynchronize(st));
    return CGP_OK;
}

extern "C" int cgp_mlp_forward(cgp_mlp* m, const double* r, const double* q, int32_t batch, double* pred,
                               cgp_stream_t stream) {
    clear_error();
    if (!m || !r || !q || !pred || batch < 1 || batch > m->B.maxb) {
        set_error("cgp_mlp_forward: bad arguments");
        return CGP_EINVAL;
    }
    return mlp_forward(m->B, m->mesh->lev[m->level], r, q, batch, pred, (cudaStream_t)stream);
}

// loss and gradient (into m->grad); shared by cgp_mlp_grad and cgp_mlp_train_step
static int mlp_backward(cgp_mlp* m, const double* r, const double* q, const double* tgt, int batch,
                        cudaStream_t st) {
    const Level& L = m->mesh->lev[m->level];
    MlpBuffers& B = m->B;
    const int n = B.n;
    const int64_t nb = (int64_t)n * batch;
    CGP_TRY(mlp_forward_train(B, L, r, q, batch, nullptr, st));
    const int g = blocks_for(nb), g128 = blocks_for(nb, 128);
    const int nblk = (int)((nb + kRowsPerBlock - 1) / kRowsPerBlock);
    int gl = (int)(nb / kBlock + 1);
    if (gl > 1024) gl = 1024;
    k_mlp_loss<<<gl, kBlock, 0, st>>>(n, batch, q, tgt, B.out, B.scale, m->g3, m->partials, m->ticket, m->loss);
    // layer 3: dW3, db3; gh2 (direct) and gm2
    k_mlp_wgrad<kHid, 1, true><<<nblk, 256, 0, st>>>(n, batch, m->g3, B.a2, B.m2, m->wpart);
    k_mlp_wgrad_reduce<<<blocks_for(2 * kHid + 1), kBlock, 0, st>>>(nblk, 1, 2 * kHid, m->wpart, m->grad + kOffW3,
                                                                   m->grad + kOffB3);
    k_mlp_dense_bwd<kHid, 1><<<g128, 128, 0, st>>>(n, batch, B.params_bf + kOffW3, m->g3, m->gA, m->gM);
    k_mlp_nmean_bwd<kHid><<<g, kBlock, 0, st>>>(n, batch, L.rowptr, L.col, m->gM, B.a2, m->gA);   // gA = dL/da2
    // layer 2
    k_mlp_wgrad<kHid, kHid, true><<<nblk, 256, 0, st>>>(n, batch, m->gA, B.a1, B.m1, m->wpart);
    k_mlp_wgrad_reduce<<<blocks_for(kHid * (2 * kHid + 1)), kBlock, 0, st>>>(nblk, kHid, 2 * kHid, m->wpart,
                                                                            m->grad + kOffW2, m->grad + kOffB2);
    k_mlp_dense_bwd<kHid, kHid><<<g128, 128, 0, st>>>(n, batch, B.params_bf + kOffW2, m->gA, m->gB, m->gM);
    k_mlp_nmean_bwd<kHid><<<g, kBlock, 0, st>>>(n, batch, L.rowptr, L.col, m->gM, B.a1, m->gB);   // gB = dL/da1
    // layer 1
    k_mlp_wgrad<4, kHid, false><<<nblk, 256, 0, st>>>(n, batch, m->gB, B.h0, B.m0, m->wpart);
    k_mlp_wgrad_reduce<<<blocks_for(kHid * 9), kBlock, 0, st>>>(nblk, kHid, 8, m->wpart, m->grad + kOffW1,
                                                               m->grad + kOffB1);
    CGP_LAUNCH_CHECK();
    return CGP_OK;
}

extern "C" int cgp_mlp_grad(cgp_mlp* m, const double* r, const double* q, const double* target, int32_t batch,
                            float* grad, float* loss, cgp_stream_t stream) {
    clear_error();
    if (!m || !r || !q || !target || !grad || batch < 1 || batch > m->B.maxb) {
        set_error("cgp_mlp_grad: bad arguments");
        return CGP_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CGP_TRY(mlp_backward(m, r, q, target, batch, st));
    CGP_CUDA(cudaMemcpyAsync(grad, m->grad, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, st));
    float l = 0.f;
    CGP_CUDA(cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    CGP_CUDA(cudaStreamSynchronize(st));
    if (loss) *loss = l;
    return CGP_OK;
}

extern "C" int cgp_mlp_train_step(cgp_mlp* m, const double* r, const double* q, const double* target, int32_t batch,
                                  float lr, float* loss, cgp_stream_t stream) {
    clear_error();
    if (!m || !r || !q || !target || batch < 1 || batch > m->B.maxb || !(lr > 0)) {
        set_error("cgp_mlp_train_step: bad arguments");
        return CGP_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CGP_TRY(mlp_backward(m, r, q, target, batch, st));
    m->adam_t += 1;
    k_mlp_adam<<<blocks_for(kMlpParams), kBlock, 0, st>>>(kMlpParams, m->B.params, m->grad, m->adam_m, m->adam_v,
                                                         m->adam_t, lr, m->B.params_bf);
    CGP_LAUNCH_CHECK();
    if (loss) {
        CGP_CUDA(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        CGP_CUDA(cudaStreamSynchronize(st));
    }
    return CGP_OK;
}

extern "C" int cgp_guess_set(cgp_solver* h, const cgp_mlp* m, cgp_stream_t stream) {
    clear_error();
    if (!h || !m) {
        set_error("cgp_guess_set: null argument");
        return CGP_EINVAL;
    }
    Solver& s = h->s;
    if (!s.mlp.params || m->mesh != s.mesh || m->level != s.lc) {
        set_error("cgp_guess_set: the solver was not assembled with CGP_GUESS_LEARNED, or the network belongs to "
                  "another mesh level");
        return CGP_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CGP_CUDA(cudaMemcpyAsync(s.mlp.params, m->B.params, sizeof(float) * kMlpParams, cudaMemcpyDeviceToDevice, st));
    CGP_CUDA(cudaMemcpyAsync(s.mlp.params_bf, m->B.params_bf, sizeof(__nv_bfloat16) * kMlpParams,
                             cudaMemcpyDeviceToDevice, st));
    CGP_CUDA(cudaStreamSynchronize(st));
    s.guess_ready = true;
    return CGP_OK;
}
