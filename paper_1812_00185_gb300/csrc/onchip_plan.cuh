// Plan of the on-chip cluster solve of the mixed form's coarse Poisson system (types, sizes
// and the host-side planner); the kernel is in coarse_onchip.cuh.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

namespace cgp {

constexpr int kOnchipThreads = 512;       // 16 warps, up to 128 registers a thread
constexpr int kOnchipRows = 6;            // most slices (rows) a warp (thread) may own
constexpr int kOnchipMaxCluster = 16;

// slice width rounded up to whole 4-entry SpMV steps
__host__ __device__ __forceinline__ int onchip_width4(int w) { return (w + 3) & ~3; }

// Device copy of the plan (arrays in the solver workspace).  Slices are listed CTA by CTA;
// "list position" q indexes slist / ebase, and local entries are numbered over all CTAs.
struct OnchipPlan {
    const int32_t* slist;      // slices in CTA order (nslices)
    const int32_t* soff;       // ncl+1: list positions of CTA c are soff[c] .. soff[c+1]-1
    const int32_t* ebase;      // per list position: first local entry of the slice
    const int32_t* li;         // per local entry: index into the CTA's z (own rows, then halo)
    const int32_t* src;        // per local entry: the SELL entry it holds, -1 for padding
    const int32_t* send_lr;    // per send: own local row whose z goes out
    const int32_t* send_dst;   // per send: (destination rank << 16) | halo slot there
    const int32_t* send_off;   // ncl+1
    const int32_t* halo_n;     // ncl: halo values each CTA receives per push
    int rows_max, halo_max, send_max, ent_max;
};

struct OnchipHostPlan {
    int ncl = 0, rows_max = 0, halo_max = 0, send_max = 0;
    int64_t ent_max = 0;
    size_t bytes = 0;          // dynamic shared memory per CTA
    std::vector<int32_t> slist, soff, ebase, li, src, send_lr, send_dst, send_off, halo_n;
};

// Shared-memory layout of one CTA (byte offsets identical in every CTA):
//   z[rows_max + halo_max] (float, padded to 16 bytes) | red64[2][16][4] double |
//   red32[2][16][4] float | send[send_max] (local row, cluster address) | entry[ent] (local
//   index of the column's z, FP32 value bits)
__host__ __device__ __forceinline__ size_t onchip_z_bytes(int rows_max, int halo_max) {
    return (size_t)4 * (((size_t)rows_max + halo_max + 3) & ~(size_t)3);
}
__host__ __device__ __forceinline__ size_t onchip_smem_bytes(int rows_max, int halo_max, int send_max, int64_t ent) {
    return onchip_z_bytes(rows_max, halo_max) + 1536 + (size_t)8 * send_max + (size_t)8 * ent;
}

// The plan for ncl CTAs; false if the coarse system does not fit (slices per CTA, shared
// memory).  ptr / col: SELL-32 pattern of the coarse level; xy: its vertex coordinates.
bool onchip_plan(int n, const std::vector<int32_t>& ptr, const std::vector<int32_t>& col,
                 const std::vector<double>& xy, int ncl, size_t smem_limit, OnchipHostPlan& P);

}  // namespace cgp
