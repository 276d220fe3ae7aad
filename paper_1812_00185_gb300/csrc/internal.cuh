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

// Deterministic grid-wide sum of NR values per thread.  Every block writes its
// partial sums to partials[blockIdx.x*NR + r]; the last block to arrive (ticket)
// adds the partials in block order and returns true with the totals in tot[]
// (valid in every thread of that block).  Other blocks return false.  All blocks
// of the grid must call it exactly once.  The ticket is reset for the next use.
// T = float: warp and block sums in FP32, block partials and the total in FP64.
template <int NR, class T>
__device__ bool grid_sum(const T (&v)[NR], double* partials, unsigned int* ticket, double (&tot)[NR]) {
    __shared__ T smt[kBlock / 32][NR];
    __shared__ double sm[kBlock / 32][NR];
    __shared__ bool is_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        T w = warp_sum(v[r]);
        if (lane == 0) smt[wid][r] = w;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            T x = lane < nw ? smt[lane][r] : T(0);
            x = warp_sum(x);
            if (lane == 0) partials[(size_t)blockIdx.x * NR + r] = (double)x;
        }
        if (lane == 0) {
            __threadfence();
            unsigned int t = atomicAdd(ticket, 1u);
            is_last = (t == gridDim.x - 1);
        }
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double s[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) s[r] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int r = 0; r < NR; ++r) s[r] += __ldcg(partials + (size_t)b * NR + r);
    }
    __syncthreads();   // sm reuse
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        double w = warp_sum(s[r]);
        if (lane == 0) sm[wid][r] = w;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            double x = lane < nw ? sm[lane][r] : 0.0;
            x = warp_sum(x);
            if (lane == 0) sm[0][r] = x;
        }
        if (lane == 0) *ticket = 0u;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < NR; ++r) tot[r] = sm[0][r];
    return true;
}

}  // namespace cgp

struct cgp_mesh {
    int n_levels = 0;
    int device = 0;
    cgp::Level lev[5];
    std::vector<void*> allocs;   // every cudaMalloc of this mesh, freed by cgp_mesh_destroy
};
