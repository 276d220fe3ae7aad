// Plan of the on-chip cluster solve of the mixed form's coarse Poisson system (types, sizes
// and the host-side planner); the kernel is in coarse_onchip.cuh.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

namespace cgp {

constexpr int kOnchipThreads = 512;       // 16 warps, up to 128 registers a thread
constexpr int kOnchipWarps = kOnchipThreads / 32;
constexpr int kOnchipRows = 6;            // most 32-row slices a warp may own (rows a thread owns)
constexpr int kOnchipMaxCluster = 16;
constexpr int kOnchipMaxSubPerCta = 8;    // subdomains of the coarse correction per CTA
// floats per CTA and exchange: [0, 4) sums, [4, 12) subdomain sums of A z, [12, 20) subdomain
// sums of r (every part 16-byte aligned)
constexpr int kOnchipSlot = 20;
constexpr int kOnchipSubW = 4;
constexpr int kOnchipSubR = 12;

// slice width rounded up to whole 4-entry SpMV steps
__host__ __device__ __forceinline__ int onchip_width4(int w) { return (w + 3) & ~3; }

// Device copy of the plan (arrays in the solver workspace).  The rows of the coarse system
// are split into ncl x 16 compact groups ("leaves"), one per warp of the cluster; a leaf's
// rows are laid out as up to kOnchipRows slices of 32 local rows.  List position q of CTA c
// (soff[c] <= q < soff[c+1]) is slice q / 16 of warp q % 16; its local rows are 32 (q -
// soff[c]) .. + 31.  Local entries are numbered over all CTAs.
struct OnchipPlan {
    const int32_t* grow;       // per local row: global row i, or -1 (padding row), or -2 - i
                               // (row i lies outside the coarse space: a phi = 0 row)
    const int32_t* soff;       // ncl+1
    const int32_t* ebase;      // per list position: first local entry of the slice
    const int32_t* width;      // per list position: entries per row, a multiple of 4
    const int32_t* li;         // per local entry: index into the CTA's z (own rows, then halo)
    const int32_t* src;        // per local entry: the SELL entry it holds, -1 for padding
    const int32_t* send_lr;    // per send: own local row whose value goes out
    const int32_t* send_dst;   // per send: (destination rank << 16) | halo slot there
    const int32_t* send_off;   // ncl+1
    const int32_t* send_woff;  // ncl x (16 + 1): the sends of warp w of CTA c are
                               // send_woff[17 c + w] .. send_woff[17 c + w + 1] - 1 (the warp owns their rows)
    const int32_t* halo_n;     // ncl: halo values each CTA receives per push
    const int32_t* hrow;       // ncl x halo_max: global row of each halo slot
    const uint8_t* hsub;       // ncl x halo_max: subdomain of each halo row (nsub: none)
    const float* einv;         // nsub x nsub, row-major: pseudo-inverse of E = Z^T A Z
    const uint8_t* need;       // ncl x need_max: the subdomains whose correction CTA c applies
                               // (its own, then those of its halo rows)
    const int32_t* need_n;     // ncl
    int rows_max, halo_max, send_max, ent_max;
    int nsub;                  // subdomains of the coarse correction (0: Jacobi alone)
    int wpg;                   // warps (leaves) per subdomain
    int need_max;
};

struct OnchipHostPlan {
    int ncl = 0, rows_max = 0, halo_max = 0, send_max = 0, nsub = 0, wpg = 0;
    int64_t ent_max = 0;
    size_t bytes = 0;          // dynamic shared memory per CTA
    int need_max = 0;
    std::vector<int32_t> grow, soff, ebase, width, li, src, send_lr, send_dst, send_off, send_woff, halo_n, hrow;
    std::vector<int32_t> sub;  // per global row: its subdomain, or nsub outside the coarse space
    std::vector<uint8_t> hsub, need;
    std::vector<int32_t> need_n;
    std::vector<double> E;     // nsub x nsub (FP64)
    std::vector<float> einv;   // nsub x nsub
};

// Shared-memory layout of one CTA (byte offsets identical in every CTA; hm = halo_max rounded
// up to 4, m4 = nsub rounded up to 4; every part starts on 16 bytes):
//   z[rows_max + hm] | w[rows_max] | dinv[rows_max] | recv[2][hm] | r_h[hm] | q_h[hm] |
//   dinv_h[hm] (float) | red64[2][16][4] double | red32[2][16][kOnchipSlot] float |
//   einv rows[need_max][nsub] | mu[m4 + 4] | zq[2][m4] (float) | hsub[hm16] | need[nm16] byte |
//   send[send_max] (local row, cluster address) | entry[ent] (local index of the column's z,
//   FP32 value bits)
__host__ __device__ __forceinline__ int onchip_hm(int halo_max) { return (halo_max + 3) & ~3; }
__host__ __device__ __forceinline__ size_t onchip_vec_bytes(int rows_max, int halo_max) {
    return (size_t)4 * (3 * (size_t)rows_max + 6 * (size_t)onchip_hm(halo_max));
}
__host__ __device__ __forceinline__ size_t onchip_red_bytes() { return 1024 + (size_t)4 * 2 * 16 * kOnchipSlot; }
__host__ __device__ __forceinline__ size_t onchip_cs_bytes(int nsub, int need_max, int halo_max) {
    const size_t m4 = ((size_t)nsub + 3) & ~(size_t)3;
    return (size_t)4 * need_max * nsub + 4 * (m4 + 4) + 8 * m4 + (((size_t)halo_max + 15) & ~(size_t)15) +
           (((size_t)need_max + 15) & ~(size_t)15);
}
__host__ __device__ __forceinline__ size_t onchip_smem_bytes(int rows_max, int halo_max, int send_max, int64_t ent,
                                                             int nsub, int need_max) {
    return onchip_vec_bytes(rows_max, halo_max) + onchip_red_bytes() + onchip_cs_bytes(nsub, need_max, halo_max) +
           (size_t)8 * send_max + (size_t)8 * ent;
}

// The plan for ncl CTAs with `sub_per_cta` subdomains per CTA (0, 1, 2, 4 or 8); false if the
// coarse system does not fit (rows per warp, shared memory).  rowptr: CSR row pointers of the
// coarse pattern (entry k of row i is SELL entry sell_ptr[i/32] + 32 k + i%32); xy: vertex
// coordinates; in_space[i]: row i belongs to the coarse space (not a phi = 0 row).
bool onchip_plan(int n, const std::vector<int32_t>& rowptr, const std::vector<int32_t>& sell_ptr,
                 const std::vector<int32_t>& sell_col, const std::vector<double>& xy,
                 const std::vector<uint8_t>& in_space, int ncl, int sub_per_cta, size_t smem_limit,
                 OnchipHostPlan& P);

// E = Z^T A Z from the FP64 SELL values of A and its pseudo-inverse (symmetric eigen-
// decomposition; eigenvalues below 1e-12 of the largest are dropped, which handles the
// constant null vector of a pure-Neumann problem).  False if E is not symmetric positive
// semi-definite to rounding.
bool onchip_coarse_space(const std::vector<int32_t>& rowptr, const std::vector<int32_t>& sell_ptr,
                         const std::vector<int32_t>& sell_col, const std::vector<double>& val, OnchipHostPlan& P);

}  // namespace cgp
