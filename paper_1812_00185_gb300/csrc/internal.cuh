// Shared definitions of the CGP CUDA library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/cgp.h"

namespace cgp {

void set_error(const char* fmt, ...);
void clear_error();

#define CGP_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            cgp::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),        \
                           __FILE__, __LINE__);                                           \
            return CGP_ECUDA;                                                             \
        }                                                                                 \
    } while (0)

#define CGP_TRY(call)                    \
    do {                                 \
        int r_ = (call);                 \
        if (r_ != CGP_OK) return r_;     \
    } while (0)

#define CGP_LAUNCH_CHECK() CGP_CUDA(cudaGetLastError())

constexpr int kBlock = 256;           // threads per block of every kernel here
constexpr int kMaxAdj = 40;           // largest vertex degree + 1 the mesh kernels accept
constexpr int kMaxInc = 32;           // largest number of triangles around a vertex

inline int blocks_for(int64_t n, int per_block = kBlock) {
    int64_t b = (n + per_block - 1) / per_block;
    return (int)(b < 1 ? 1 : b);
}

// One level of the nested hierarchy, device arrays.
struct Level {
    int32_t nv = 0, nt = 0;
    int64_t nnz = 0;
    double* xy = nullptr;        // 2*nv, interleaved
    int32_t* tri = nullptr;      // 3*nt
    uint8_t* tag = nullptr;      // nv
    int32_t* rowptr = nullptr;   // nv+1 (vertex adjacency, diagonal included, columns ascending)
    int32_t* col = nullptr;      // nnz
    int32_t* parents = nullptr;  // 2*(nv - nv_prev): end points of the vertices added at this level
    int32_t* vt_ptr = nullptr;   // nv+1: triangles around each vertex
    int32_t* vt_list = nullptr;  // 3*nt, ascending per vertex
    // sliced ELL (SELL-32) view of the same pattern: slice s = rows 32s..32s+31, stored
    // column-major with the slice's longest row as width; entry (row i, k-th of its row)
    // sits at sell_ptr[i/32] + 32 k + i%32.  Padding: column = first row of the slice, value 0.
    int32_t nslices = 0;
    int64_t nnz_sell = 0;
    int32_t* sell_ptr = nullptr; // nslices+1
    int32_t* sell_col = nullptr; // nnz_sell
};

constexpr int kSlice = 32;

__host__ __device__ __forceinline__ int64_t sell_pos(const int32_t* sell_ptr, int row, int k) {
    return (int64_t)sell_ptr[row >> 5] + 32 * k + (row & 31);
}

// Exclusive scan of n int32 counts into out[0..n] (out[n] = total), on `stream`.
int exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp, cudaStream_t stream);
size_t scan_tmp_ints(int64_t n);

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sums of NR values over a warp, written to out[0..NR) by the lanes that hold them (no
// other lane writes).  A transpose reduction: with P = NR rounded up to a power of two,
// each xor-shuffle round (offsets 16, 8, ...) halves the values a lane holds, until every
// lane holds one partial row; the remaining rounds sum it.  That is P - 1 + log2(32 / P)
// adds per lane instead of 5 NR, which matters for FP64 (a warp-wide FP64 add takes 16
// clocks of this GPU's FP64 pipe).  The order of the additions is fixed.
template <int NR, class T>
__device__ __forceinline__ void warp_sums_to(const T (&v)[NR], T* out) {
    constexpr int P = NR <= 1 ? 1 : (NR <= 2 ? 2 : (NR <= 4 ? 4 : 8));
    static_assert(NR <= 8, "at most 8 values");
    const int lane = threadIdx.x & 31;
    T w[P];
#pragma unroll
    for (int i = 0; i < P; ++i) w[i] = i < NR ? v[i] : T(0);
    int row = 0;
#pragma unroll
    for (int h = P, o = 16; h > 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
        if (up) row += h / 2;
#pragma unroll
        for (int i = 0; i < h / 2; ++i) {
            const T keep = up ? w[i + h / 2] : w[i];
            const T send = up ? w[i] : w[i + h / 2];
            w[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
#pragma unroll
    for (int o = 16 / P; o > 0; o >>= 1) w[0] += __shfl_xor_sync(0xffffffffu, w[0], o);
    if ((lane & (32 / P - 1)) == 0 && row < NR) out[row] = w[0];
}

// Deterministic grid-wide sum of NR values per thread, in the precision T of the values.
// Every block writes its partial sums to partials[blockIdx.x*NR + r] (as T); the last
// block to arrive (ticket) adds the partials in a fixed order and returns true with the
// totals in tot[] (valid in every thread of that block).  Other blocks return false.  All
// blocks of the grid must call it exactly once.  The ticket is reset for the next use.
// T = float (the FP32 inner solves) keeps the whole reduction off the FP64 pipe: the
// block partials are FP32 sums already, and an FP32 tree over them adds an error far below
// the inner solves' tolerance.
template <int NR, class T>
__device__ bool grid_sum(const T (&v)[NR], double* partials, unsigned int* ticket, double (&tot)[NR]) {
    __shared__ T smt[kBlock / 32][NR];
    __shared__ T res[NR];
    __shared__ bool is_last;
    T* pt = reinterpret_cast<T*>(partials);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // warps -> CTA: the CTA's partials, written by lane 0 of warp 0
    auto cta_sum = [&](const T (&x)[NR]) {
        warp_sums_to(x, smt[wid]);
        __syncthreads();
        if (wid == 0) {
            T y[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) y[r] = lane < nw ? smt[lane][r] : T(0);
            warp_sums_to(y, res);
        }
        __syncthreads();
    };
    cta_sum(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int r = 0; r < NR; ++r) pt[(size_t)blockIdx.x * NR + r] = res[r];
        __threadfence();
        is_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    T s[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) s[r] = T(0);
    // the partial loads are issued in chunks of U per thread (64 bytes of registers), so
    // the block waits for one memory round trip per chunk instead of one per partial
    constexpr int U = (64 / (NR * (int)sizeof(T))) < 1 ? 1 : ((64 / (NR * (int)sizeof(T))) > 8 ? 8 : 64 / (NR * (int)sizeof(T)));
    for (int b0 = threadIdx.x; b0 < (int)gridDim.x; b0 += U * blockDim.x) {
        T q[U][NR];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int b = b0 + k * blockDim.x;
#pragma unroll
            for (int r = 0; r < NR; ++r) q[k][r] = b < (int)gridDim.x ? __ldcg(pt + (size_t)b * NR + r) : T(0);
        }
#pragma unroll
        for (int k = 0; k < U; ++k)
#pragma unroll
            for (int r = 0; r < NR; ++r) s[r] += q[k][r];
    }
    cta_sum(s);
    if (threadIdx.x == 0) *ticket = 0u;
#pragma unroll
    for (int r = 0; r < NR; ++r) tot[r] = (double)res[r];
    return true;
}

}  // namespace cgp

struct cgp_mesh {
    int n_levels = 0;
    int device = 0;
    cgp::Level lev[5];
    std::vector<void*> allocs;   // every cudaMalloc of this mesh, freed by cgp_mesh_destroy
};
