// On-chip mixed-precision coarse solve (Eq. 23): one thread-block cluster holds the whole
// FP32 inner problem in distributed shared memory.
//
// The coarse systems of CGP are small (tens of thousands of rows), and on this GPU the FP64
// pipe is narrow while a cluster barrier is far cheaper than a grid-wide one, so the FP32
// inner PCG of the mixed form runs on a single cluster of 8 or 16 CTAs.  A host-side plan
// (onchip_plan.cu) gives each warp a spatially compact patch of rows (each CTA the patches
// of one region).  Each CTA keeps in its shared memory:
//   * z for its own rows followed by a halo: z of the other CTAs' rows that its rows use;
//   * its rows of the FP32 matrix, 32-row slices, each entry as (index of its column's z,
//     value), widths padded to whole 4-entry steps;
//   * for the halo rows, r, q and D^{-1}, and two receive buffers;
//   * a send list: every warp stores A z of its rows that neighbours use straight into their
//     receive buffers (remote shared-memory stores);
//   * the slots of the cluster exchanges: every CTA stores its partial sums into every
//     other CTA's slot array and each CTA adds the slots in the same fixed order (identical
//     scalars everywhere);
//   * the rows of E^+ (below) for the subdomains it corrects.
// The inner iteration is PCG in the one-exchange form of Chronopoulos and Gear: w = A z,
// then a single exchange carries <r, z>, <z, w>, <r, r>, the halo copy of w and the coarse
// sums; alpha and beta follow from those, and each CTA advances q, r and z of its halo rows
// with the same recurrences (and bit for bit the same values) as their owners, so z of the
// halo never travels.  The vectors e, r, z, p, q of the own rows live in registers.  All
// inner arithmetic is FP32 on the residual scaled to unit norm.  The FP64 outer loop (true
// residual, its norm, the convergence test, x += ||r|| e) reads the FP64 matrix and x from
// global memory a few times per solve; only warp 0 of each CTA does its FP64 scalar work.
//
// Preconditioner: Jacobi, or Jacobi plus an additive subdomain coarse correction,
//     z = D^{-1} r + Z E^+ Z^T r,   E = Z^T A Z,
// where column j of Z is the indicator of subdomain j (a group of sibling warp patches; phi =
// 0 rows belong to none) and E^+ is the pseudo-inverse of the small Galerkin matrix.
// M^{-1} stays symmetric positive definite, so the iteration is still PCG; the coarse space
// removes the smooth error components Jacobi damps slowest (the iteration count drops
// several-fold on the coarse Poisson systems of CGP).  s = Z^T r follows its own recurrence
// s = Z^T r_prev - alpha Z^T q, from the subdomain sums (warp sums) of r and w that travel
// with the exchange, so it needs no exchange of its own; each CTA forms mu = E^+ s only for
// its own subdomains and those of its halo rows.
#pragma once

#include <cooperative_groups.h>

#include "coarse_pcg.cuh"
#include "onchip_plan.cuh"

namespace cgp {

// ---- shared::cluster access
__device__ __forceinline__ uint32_t oc_map(const void* p, int rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void oc_st(uint32_t addr, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void oc_st32(uint32_t addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
// all threads of all CTAs of the cluster; orders shared and global memory at cluster scope
__device__ __forceinline__ void oc_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ---- mbarrier signalling of the FP32 reductions: remote st.async stores complete bytes on
// the receiving CTA's mbarrier, so no fence or cluster barrier is needed per reduction
__device__ __forceinline__ void oc_mbar_init(uint64_t* mb, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(mb)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void oc_mbar_arrive_expect(uint64_t* mb, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(mb)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool oc_mbar_try(uint64_t* mb, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"((uint32_t)__cvta_generic_to_shared(mb)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void oc_st_async4(uint32_t addr, float a, float b, float c, float d, uint32_t mbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(addr),
                 "r"(__float_as_uint(a)), "r"(__float_as_uint(b)), "r"(__float_as_uint(c)), "r"(__float_as_uint(d)),
                 "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void oc_st_async(uint32_t addr, float v, uint32_t mbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr),
                 "r"(__float_as_uint(v)), "r"(mbar)
                 : "memory");
}
constexpr long long kOnchipWaitCycles = 4000000000LL;   // ~2 s: a wait this long means a lost signal
constexpr long long kOnchipWaitCyclesTest = 20000000LL; // ~10 ms, under the wait test hook

// what warp 0 tells its CTA after an FP64 reduction
struct OnchipScalars {
    int act;
    float stop2;               // stop threshold of the scaled inner problem on <r, r>
    double inv, norm, mu;      // 1 / ||r||, ||r|| of the outer residual; mean of the Neumann fix
};

// MR: nsub / 16 (at least 1) with the coarse correction, 0 without; it fixes how many columns
// of an E^+ row a lane holds (4, 2 or 1, interleaved across the lanes)
template <int MR>
static __global__ void __launch_bounds__(kOnchipThreads, 1) k_pcg_onchip(CoarsePcgArgs a, OnchipPlan pl) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double wsum[kOnchipWarps][4];
    __shared__ float wsum32[kOnchipWarps][6];
    __shared__ OnchipScalars sc;
    __shared__ __align__(8) uint64_t mbar[2];     // exchanges, alternating
    __shared__ uint32_t mbar_remote[kOnchipMaxCluster][2];
    __shared__ float tot32[4];
    __shared__ int abort_flag;
    const int rank = (int)cluster.block_rank(), ncl = (int)cluster.num_blocks();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = kOnchipWarps;
    const SellView& A = a.A;
    const int rows_max = pl.rows_max, hm = onchip_hm(pl.halo_max), m = pl.nsub, m4 = (m + 3) & ~3;
    float* zl = reinterpret_cast<float*>(smem);   // z: own rows, then the halo
    float* wl = zl + rows_max + hm;               // own rows: A z (the values sent out), or r at a restart
    float* dl = wl + rows_max;                    // own rows: D^{-1}
    float* recv = dl + rows_max;                  // [2][hm]: halo values received, by exchange parity
    float* rh = recv + 2 * hm;                    // halo rows: r, q and D^{-1}
    float* qh = rh + hm;
    float* dh = qh + hm;
    double* red64 = reinterpret_cast<double*>(dh + hm);
    float* red32 = reinterpret_cast<float*>(red64 + 128);
    float* einv = red32 + 2 * 16 * kOnchipSlot;   // the rows of E^+ of the subdomains in `needl`
    float* mu = einv + pl.need_max * m;           // mu[m] = 0: rows outside the coarse space
    float* zq = mu + m4 + 4;                      // [2][m4]: Z^T q, double-buffered
    uint8_t* hsub = reinterpret_cast<uint8_t*>(zq + 2 * m4);
    uint8_t* needl = hsub + ((pl.halo_max + 15) & ~15);
    uint2* send = reinterpret_cast<uint2*>(needl + ((pl.need_max + 15) & ~15));
    uint2* cent = send + pl.send_max;             // (local index of z, value bits)
    const int q0 = __ldg(pl.soff + rank), npos = __ldg(pl.soff + rank + 1) - q0;
    const int eb0 = npos > 0 ? __ldg(pl.ebase + q0) : 0;
    const int halo_self = __ldg(pl.halo_n + rank);
    const int need_n = m ? __ldg(pl.need_n + rank) : 0;
    for (int i = threadIdx.x; i < 3 * rows_max + hm; i += blockDim.x) zl[i] = 0.0f;   // z, w, D^{-1}
    for (int i = threadIdx.x; i < 4 * hm; i += blockDim.x) recv[i] = 0.0f;            // recv, r_h, q_h
    for (int h = threadIdx.x; h < hm; h += blockDim.x) {
        const bool in = h < halo_self;
        dh[h] = in ? __ldg(a.dinvf + __ldg(pl.hrow + (size_t)rank * pl.halo_max + h)) : 0.0f;
        if (h < pl.halo_max) hsub[h] = in ? __ldg(pl.hsub + (size_t)rank * pl.halo_max + h) : (uint8_t)m;
    }
    for (int i = threadIdx.x; i < need_n * m; i += blockDim.x) {
        const int idx = i / m;
        einv[i] = __ldg(pl.einv + (size_t)__ldg(pl.need + (size_t)rank * pl.need_max + idx) * m + (i - idx * m));
    }
    for (int i = threadIdx.x; i < need_n; i += blockDim.x) needl[i] = __ldg(pl.need + (size_t)rank * pl.need_max + i);
    for (int i = threadIdx.x; i < 3 * m4 + 4; i += blockDim.x) mu[i] = 0.0f;        // mu, zq
    // ---- rows of this thread: slice t of its warp is list position wid + nw * t of its CTA;
    // their matrix entries are copied to shared memory by the owning warp
    int nrow = 0;
    int base_[kOnchipRows], width_[kOnchipRows], grow_[kOnchipRows];
#pragma unroll
    for (int t = 0; t < kOnchipRows; ++t) {
        const int q = wid + nw * t;
        base_[t] = 0;
        width_[t] = 0;
        grow_[t] = -1;
        if (q < npos) {
            nrow = t + 1;
            base_[t] = __ldg(pl.ebase + q0 + q) - eb0;
            width_[t] = __ldg(pl.width + q0 + q);
            grow_[t] = __ldg(pl.grow + 32 * (size_t)(q0 + q) + lane);
            for (int k = 0; k < width_[t]; ++k) {
                const int el = base_[t] + 32 * k + lane;
                const int src = __ldg(pl.src + eb0 + el);
                cent[el] = make_uint2((uint32_t)__ldg(pl.li + eb0 + el), src >= 0 ? __float_as_uint(__ldg(a.valf + src)) : 0u);
            }
        }
    }
    auto row_of = [&](int t) {   // global row of slot t, or -1
        const int g = grow_[t];
        return g >= 0 ? g : (g == -1 ? -1 : -2 - g);
    };
    auto in_space = [&](int t) { return grow_[t] >= 0; };
    auto lrow_of = [&](int t) { return 32 * (wid + nw * t) + lane; };
    const int spc = m ? nw / pl.wpg : 0;                       // subdomains per CTA
    const int sh = m ? __ffs(spc) - 1 : 0;
    const int my_sub = m ? (rank * nw + wid) / pl.wpg : m;     // this warp's subdomain
    // sends: the receive slot's cluster address (parity 0); warp w sends entries ws0 .. ws1 - 1
    const int ns0 = __ldg(pl.send_off + rank), nsend = __ldg(pl.send_off + rank + 1) - ns0;
    for (int i = threadIdx.x; i < nsend; i += blockDim.x) {
        const int d = __ldg(pl.send_dst + ns0 + i);   // x: local row | destination rank << 16
        send[i] = make_uint2((uint32_t)__ldg(pl.send_lr + ns0 + i) | ((uint32_t)(d >> 16) << 16),
                             oc_map(recv + (d & 0xFFFF), d >> 16));
    }
    const int ws0 = __ldg(pl.send_woff + rank * (nw + 1) + wid) - ns0;
    const int ws1 = __ldg(pl.send_woff + rank * (nw + 1) + wid + 1) - ns0;
    if (threadIdx.x == 0) {
        oc_mbar_init(&mbar[0], 1);
        oc_mbar_init(&mbar[1], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < ncl) {
        mbar_remote[threadIdx.x][0] = oc_map(&mbar[0], threadIdx.x);
        mbar_remote[threadIdx.x][1] = oc_map(&mbar[1], threadIdx.x);
    }
    // remote slot addresses of the reductions: lane l < ncl stores into CTA l
    const uint32_t red64_remote = oc_map(red64, lane < ncl ? lane : 0);
    const uint32_t red32_remote = oc_map(red32, lane < ncl ? lane : 0);
    auto aborted_now = [&]() { return *reinterpret_cast<volatile int*>(&abort_flag) != 0; };
    // FP64 cluster sums (outer loop).  Partial sums go warp -> CTA (warp 0) -> every CTA's
    // slot array, one hardware cluster barrier, then the ncl slots are added; all in a fixed
    // order, so every CTA gets the same totals, in every lane of warp 0, which alone does the
    // FP64 scalar work (the FP64 pipe is narrow) and hands results to the CTA through `sc` and
    // a __syncthreads.  Consecutive reductions alternate between two slot sets.
    int slot = 0;
    auto cred64 = [&](auto& v, double (&tot)[4]) {
        constexpr int NR = sizeof(v) / sizeof(double);
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            const double s = warp_sum(v[k]);
            if (lane == 0) wsum[wid][k] = s;
        }
        __syncthreads();
        if (wid == 0) {
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const double s = __shfl_sync(0xffffffffu, warp_sum(lane < nw ? wsum[lane][k] : 0.0), 0);
                if (lane < ncl) oc_st(red64_remote + (uint32_t)(8 * ((slot * 16 + rank) * 4 + k)), s);
            }
        }
        oc_barrier();
        if (wid == 0) {
#pragma unroll
            for (int k = 0; k < NR; ++k)
                tot[k] = __shfl_sync(0xffffffffu, warp_sum(lane < ncl ? red64[(slot * 16 + lane) * 4 + k] : 0.0), 0);
        }
        slot ^= 1;
    };
    // One exchange of the FP32 inner iteration.  Each warp sends its rows of wl to the
    // neighbours' receive buffers (parity par) as soon as it has them; the CTA's sums of v
    // (three scalars) and, with the coarse space, the subdomain sums of tw (A z) and ur (r)
    // go from warp 0 to every CTA's slots.  Every remote store completes bytes on the
    // receiver's mbarrier of that parity (two, used alternately: data for exchange m + 2 can
    // only be sent once every CTA has contributed to m + 1, so after this CTA finished m);
    // warp 0 waits (bounded) for all of them, adds the scalar slots in a fixed order
    // (identical totals in every CTA) and hands them to the CTA with the verdict through a
    // __syncthreads.  A wait that runs out sets the abort flag of every CTA; the call then
    // returns false in every thread of the CTA.
    int mred = 0;
    auto exchange = [&](const float (&v)[3], float tw, float ur, float (&tot)[3]) -> bool {
        const int par = mred & 1;
        const uint32_t phase = (uint32_t)(mred >> 1) & 1u;
        ++mred;
        __syncwarp();   // the warp's wl stores before its sends read them
        if (!aborted_now()) {
            const uint32_t hoff = (uint32_t)(4 * par * hm);
            for (int i = ws0 + lane; i < ws1; i += 32) {
                const uint2 sd = send[i];
                oc_st_async(sd.y + hoff, wl[sd.x & 0xFFFF], mbar_remote[sd.x >> 16][par]);
            }
        }
        constexpr int nv = MR > 0 ? 5 : 3;
        const float x[5] = {v[0], v[1], v[2], tw, ur};
#pragma unroll
        for (int k = 0; k < nv; ++k) {
            const float s = warp_sum(x[k]);
            if (lane == 0) wsum32[wid][k] = s;
        }
        __syncthreads();
        if (wid == 0) {
            const bool live = !aborted_now();
            // 16 partials: xor rounds 8 .. 1 leave the total in lanes 0-15
            static_assert(kOnchipWarps <= 16 && kOnchipMaxCluster <= 16, "16-lane sums");
            float cs[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float x = lane < nw ? wsum32[lane][k] : 0.0f;
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                cs[k] = x;
            }
            const bool sender = live && lane < ncl;
            const uint32_t dst = red32_remote + (uint32_t)(4 * ((par * 16 + rank) * kOnchipSlot));
            const uint32_t mb = mbar_remote[lane < ncl ? lane : 0][par];
            if (sender) oc_st_async4(dst, cs[0], cs[1], cs[2], 0.0f, mb);
            if constexpr (MR > 0) {
                // subdomain g of this CTA = warps g wpg .. g wpg + wpg - 1; its sums go out as
                // eight values per vector (unused ones zero), four to a 16-byte store
                float gt = lane < nw ? wsum32[lane][3] : 0.0f, gu = lane < nw ? wsum32[lane][4] : 0.0f;
                for (int o = 1; o < pl.wpg; o <<= 1) {
                    gt += __shfl_down_sync(0xffffffffu, gt, o);
                    gu += __shfl_down_sync(0xffffffffu, gu, o);
                }
                float tv[kOnchipMaxSubPerCta], uv[kOnchipMaxSubPerCta];
#pragma unroll
                for (int g = 0; g < kOnchipMaxSubPerCta; ++g) {
                    const int from = (g < spc ? g : 0) * pl.wpg;
                    const float y1 = __shfl_sync(0xffffffffu, gt, from), y2 = __shfl_sync(0xffffffffu, gu, from);
                    tv[g] = g < spc ? y1 : 0.0f;
                    uv[g] = g < spc ? y2 : 0.0f;
                }
                if (sender) {
                    oc_st_async4(dst + 4 * kOnchipSubW, tv[0], tv[1], tv[2], tv[3], mb);
                    oc_st_async4(dst + 4 * kOnchipSubW + 16, tv[4], tv[5], tv[6], tv[7], mb);
                    oc_st_async4(dst + 4 * kOnchipSubR, uv[0], uv[1], uv[2], uv[3], mb);
                    oc_st_async4(dst + 4 * kOnchipSubR + 16, uv[4], uv[5], uv[6], uv[7], mb);
                }
            }
            // (the wait test hook expects 4 bytes more than anyone sends)
            if (lane == 0)
                oc_mbar_arrive_expect(&mbar[par], (uint32_t)(ncl * (MR > 0 ? 4 * kOnchipSlot : 16) + 4 * halo_self +
                                                             (a.wait_test ? 4 : 0)));
            bool ok = live;
            if (ok) {
                const long long t0 = clock64();
                const long long limit = a.wait_test ? kOnchipWaitCyclesTest : kOnchipWaitCycles;
                while (!oc_mbar_try(&mbar[par], phase)) {
                    if (aborted_now() || clock64() - t0 > limit) {
                        ok = false;
                        break;
                    }
                }
            }
            ok = __all_sync(0xffffffffu, ok);
#pragma unroll
            for (int k = 0; k < 3; ++k) {   // the ncl <= 16 slots, in a fixed order
                float x = lane < ncl ? red32[(par * 16 + lane) * kOnchipSlot + k] : 0.0f;
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
                if (lane == 0) tot32[k] = x;
            }
            if (!ok && lane < ncl) asm volatile("st.shared::cluster.u32 [%0], 1;" ::"r"(oc_map(&abort_flag, lane)) : "memory");
            if (lane == 0) tot32[3] = (ok && !aborted_now()) ? 1.0f : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 3; ++k) tot[k] = tot32[k];
        return tot32[3] != 0.0f;
    };
    // The coarse correction after exchange `par`: s = Z^T r of the current r, from the slot sums
    // of that exchange (u = Z^T r and t = Z^T A z of the previous iterate): s = u - al zn with
    // zn = t + be zq the new Z^T q (first call of a restart: s = u); mu = E^+ s for the
    // subdomains this CTA corrects (one warp per row of E^+), then z += mu[subdomain] in the
    // own rows and the halo, which hold D^{-1} r.  Ends with the CTA's z in shared memory.
    float z_[kOnchipRows];
    int zpar = 0;
    auto coarse = [&](int par, float al, float be, bool first) {
        if constexpr (MR > 0) {
            // lane l holds columns l, l + 32, ... (consecutive lanes, consecutive words)
            constexpr int cpl = MR == 8 ? 4 : (MR == 4 ? 2 : 1);
            float sv[cpl];
            const float* zo = zq + zpar * m4;
            float* zn_out = zq + (zpar ^ 1) * m4;
#pragma unroll
            for (int c = 0; c < cpl; ++c) {
                const int j = lane + 32 * c;
                sv[c] = 0.0f;
                if (j < m) {
                    const float* sl = red32 + (par * 16 + (j >> sh)) * kOnchipSlot + (j & (spc - 1));
                    const float zn = first ? 0.0f : fmaf(be, zo[j], sl[kOnchipSubW]);
                    sv[c] = fmaf(-al, zn, sl[kOnchipSubR]);
                    if (wid == 0) zn_out[j] = zn;
                }
            }
            zpar ^= 1;
            for (int idx = wid; idx < need_n; idx += nw) {
                const float* er = einv + idx * m;
                float acc = 0.0f;
#pragma unroll
                for (int c = 0; c < cpl; ++c) {
                    const int j = lane + 32 * c;
                    if (j < m) acc = fmaf(er[j], sv[c], acc);
                }
                acc = warp_sum(acc);
                if (lane == 0) mu[needl[idx]] = acc;
            }
            __syncthreads();
            const float mw = mu[my_sub];
#pragma unroll
            for (int t = 0; t < kOnchipRows; ++t) {
                if (t >= nrow) break;
                if (in_space(t)) z_[t] += mw;
                zl[lrow_of(t)] = z_[t];
            }
            for (int h = threadIdx.x; h < halo_self; h += blockDim.x) zl[rows_max + h] += mu[hsub[h]];
        } else {
#pragma unroll
            for (int t = 0; t < kOnchipRows; ++t) {
                if (t >= nrow) break;
                zl[lrow_of(t)] = z_[t];
            }
        }
        __syncthreads();
    };
    const double mean = a.project ? a.st->mean : 0.0;
    const double tol2 = a.tol2;
    double* xv = a.x;
    float e_[kOnchipRows], r_[kOnchipRows], p_[kOnchipRows], q_[kOnchipRows];
#pragma unroll
    for (int t = 0; t < kOnchipRows; ++t) {
        e_[t] = r_[t] = z_[t] = p_[t] = q_[t] = 0.0f;
        const int i = row_of(t);
        if (i >= 0) {
            dl[lrow_of(t)] = __ldg(a.dinvf + i);
            if (a.project) a.b[i] -= mean;
            if (a.zero_x) __stcg(xv + i, 0.0);
        }
    }
    oc_barrier();   // matrix, plan and D^{-1} loaded, b projected and x zeroed where asked
    // FP64 row of A times a global vector (`ro`: v is read-only during the launch), from the
    // SELL-32 arrays: entry k of row i sits at ptr[i / 32] + 32 k + i % 32 (padding: value 0)
    auto row_a = [&](int t, const double* v, bool ro) {
        const int i = row_of(t);
        double acc = 0.0;
        if (i >= 0) {
            const int e0 = __ldg(A.ptr + (i >> 5)), w = (__ldg(A.ptr + (i >> 5) + 1) - e0) >> 5;
            for (int k = 0; k < w; ++k) {
                const int e = e0 + 32 * k + (i & 31);
                const int j = __ldg(A.col + e);
                acc = fma(__ldg(a.val + e), ro ? __ldg(v + j) : ldcg(v + j), acc);
            }
        }
        return acc;
    };
    int iters = 0, status = 0, outer = 0, used_alt = 0;
    bool converged = false;
    double tot[4];
    // the judge of the learned guess: while gate[0] > 0 the network was not evaluated this step
    const bool alt_on = a.x_alt && !a.zero_x && !(a.gate && ldcg(a.gate) > 0);
    double rr_x = 0.0;   // ||b - A x||^2 of the first guess alone (warp 0; for the judge)
    if (alt_on) {
        // second initial guess y (the learned prediction): start from the combination
        // c1 x + c2 y that minimises the A-norm of the error over span{x, y} (a 2x2 Galerkin
        // system), which is what CG's work depends on; never worse than x or y alone
        double g[4] = {0.0, 0.0, 0.0, 0.0}, f[2] = {0.0, 0.0};   // xAx, xAy, yAy, |b - Ax|^2; x.b, y.b
#pragma unroll
        for (int t = 0; t < kOnchipRows; ++t) {
            if (t >= nrow) break;
            const double ax = row_a(t, xv, false), ay = row_a(t, a.x_alt, true);
            const int i = row_of(t);
            if (i >= 0) {
                const double xi = ldcg(xv + i), yi = __ldg(a.x_alt + i), bi = ldcg(a.b + i);
                g[0] += xi * ax;
                g[1] += xi * ay;
                g[2] += yi * ay;
                g[3] += (bi - ax) * (bi - ax);
                f[0] += xi * bi;
                f[1] += yi * bi;
            }
        }
        cred64(g, tot);
        double gt[3] = {tot[0], tot[1], tot[2]};
        rr_x = tot[3];
        cred64(f, tot);
        if (threadIdx.x == 0) {
            const double a11 = gt[0], a12 = gt[1], a22 = gt[2], f1 = tot[0], f2 = tot[1];
            const double det = a11 * a22 - a12 * a12;
            double c1 = 1.0, c2 = 0.0;
            if (isfinite(det) && det > 1e-12 * fabs(a11 * a22) && a11 > 0.0 && a22 > 0.0) {
                c1 = (f1 * a22 - f2 * a12) / det;
                c2 = (a11 * f2 - a12 * f1) / det;
            } else if (a22 > 0.0 && isfinite(f2) && (!(a11 > 0.0) || f2 * f2 / a22 > f1 * f1 / a11)) {
                c1 = 0.0;                        // x and y (nearly) parallel, or x = 0: the better one, scaled
                c2 = f2 / a22;
            } else if (a11 > 0.0 && isfinite(f1)) {
                c1 = f1 / a11;
            }
            if (!isfinite(c1) || !isfinite(c2)) {
                c1 = 1.0;
                c2 = 0.0;
            }
            sc.inv = c1;
            sc.norm = c2;
        }
        __syncthreads();
        const double c1 = sc.inv, c2 = sc.norm;
        used_alt = c2 != 0.0;
#pragma unroll
        for (int t = 0; t < kOnchipRows; ++t) {
            const int i = row_of(t);
            if (i >= 0) __stcg(xv + i, c1 * ldcg(xv + i) + c2 * __ldg(a.x_alt + i));
        }
        oc_barrier();
    }
    double bb = 0.0, rr_final = 0.0;   // meaningful in warp 0
    enum { kInner = 0, kConverged, kNonfinite, kNotconv };
    for (;;) {
        // ---- outer: r = b - A x in FP64 (global memory); the inner problem A e = r / ||r||
        double acc[2] = {0.0, 0.0};
#pragma unroll
        for (int t = 0; t < kOnchipRows; ++t) {
            if (t >= nrow) break;
            const double ax = row_a(t, xv, false);
            const int i = row_of(t);
            if (i >= 0) {
                const double bi = ldcg(a.b + i);
                const double ri = bi - ax;
                r_[t] = (float)ri;
                acc[0] += ri * ri;
                acc[1] += bi * bi;
            }
        }
        cred64(acc, tot);
        if (wid == 0) {
            if (outer == 0) {
                bb = tot[1];
                // judge: did the network's direction lower the starting residual by 5 %?
                if (a.gate && lane == 0 && rank == 0) {
                    if (alt_on) {
                        const bool useful = tot[0] < 0.9025 * rr_x;
                        const int miss = useful ? 0 : ldcg(a.gate + 1) + 1;
                        if (miss >= 8) {
                            a.gate[0] = 64;
                            a.gate[1] = 0;
                        } else {
                            a.gate[1] = miss;
                        }
                    } else if (ldcg(a.gate) > 0) {
                        a.gate[0] = ldcg(a.gate) - 1;
                    }
                }
            }
            rr_final = tot[0];
            int act = kInner;
            if (!isfinite(tot[0])) act = kNonfinite;
            else if (tot[0] <= tol2 * bb) act = kConverged;
            else if (outer >= a.max_outer || iters >= a.maxit) act = kNotconv;
            if (lane == 0) {
                sc.act = act;
                if (act == kInner) {
                    sc.norm = sqrt(tot[0]);
                    sc.inv = 1.0 / sc.norm;
                    sc.stop2 = (float)fmax(a.inner_tol * a.inner_tol, 0.25 * tol2 * bb / tot[0]);
                }
            }
        }
        __syncthreads();
        {
            const int act = sc.act;
            if (act == kNonfinite) {
                status = CGP_ENONFINITE;
                break;
            }
            if (act == kConverged) {
                converged = true;
                break;
            }
            if (act == kNotconv) {
                status = CGP_ENOTCONV;
                break;
            }
        }
        const float inv = (float)sc.inv;
        const float stop2 = sc.stop2;
        // ---- inner PCG in FP32 on the scaled residual, in the one-exchange form (Chronopoulos
        // and Gear): each iteration forms w = A z, then one exchange carries <r, z>, <z, w>,
        // <r, r>, Z^T w, Z^T r and the halo copy of w; alpha and beta follow from those
        // (alpha = <r, z> / (<z, w> - beta <r, z> / alpha_prev)), every CTA updates q, r and z
        // of its halo rows by the same recurrences as their owners (so z of the halo needs no
        // second exchange), and Z^T r of the next iterate by its own recurrence.  Every warp
        // carries the same scalars, computed from the same totals.
        float gam_prev = 1.0f, alp_prev = 1.0f, rr_best = INFINITY;
        int best_k = 0;
        bool drift = false, aborted = false;
        {
            // the scaled residual: its halo copy and Z^T r travel in the first exchange
            float ur = 0.0f;
#pragma unroll
            for (int t = 0; t < kOnchipRows; ++t) {
                if (t >= nrow) break;
                e_[t] = p_[t] = q_[t] = 0.0f;
                if (row_of(t) >= 0) {
                    r_[t] *= inv;
                    if (in_space(t)) ur += r_[t];
                } else {
                    r_[t] = 0.0f;
                }
                wl[lrow_of(t)] = r_[t];
            }
            const float v0[3] = {0.0f, 0.0f, 0.0f};
            float t0[3];
            if (!exchange(v0, 0.0f, ur, t0)) {
                aborted = true;
            } else {
                const float* rv = recv + ((mred - 1) & 1) * hm;
                for (int h = threadIdx.x; h < halo_self; h += blockDim.x) {
                    const float x = rv[h];
                    rh[h] = x;
                    qh[h] = 0.0f;
                    zl[rows_max + h] = dh[h] * x;
                }
#pragma unroll
                for (int t = 0; t < kOnchipRows; ++t) {
                    if (t >= nrow) break;
                    z_[t] = dl[lrow_of(t)] * r_[t];
                }
                coarse((mred - 1) & 1, 0.0f, 0.0f, true);
            }
        }
        for (int k = 0; !aborted; ++k) {
            if (iters >= a.maxit) break;
            // w = A z (local gathers) and the sums of this iterate
            float v[3] = {0.0f, 0.0f, 0.0f}, tw = 0.0f, ur = 0.0f;
#pragma unroll
            for (int t = 0; t < kOnchipRows; ++t) {
                if (t >= nrow) break;
                const uint2* ce = cent + base_[t] + lane;
                const int w = width_[t];
                float s = 0.0f;
                for (int k = 0; k < w; k += 4) {
                    const uint2 e0 = ce[32 * k], e1 = ce[32 * (k + 1)], e2 = ce[32 * (k + 2)], e3 = ce[32 * (k + 3)];
                    const float g0 = zl[e0.x], g1 = zl[e1.x], g2 = zl[e2.x], g3 = zl[e3.x];
                    s = fmaf(__uint_as_float(e0.y), g0, s);
                    s = fmaf(__uint_as_float(e1.y), g1, s);
                    s = fmaf(__uint_as_float(e2.y), g2, s);
                    s = fmaf(__uint_as_float(e3.y), g3, s);
                }
                wl[lrow_of(t)] = s;
                if (row_of(t) >= 0) {
                    v[0] = fmaf(r_[t], z_[t], v[0]);
                    v[1] = fmaf(z_[t], s, v[1]);
                    v[2] = fmaf(r_[t], r_[t], v[2]);
                    if (in_space(t)) {
                        tw += s;
                        ur += r_[t];
                    }
                }
            }
            float tt[3];
            if (!exchange(v, tw, ur, tt)) {
                aborted = true;
                break;
            }
            const int par = (mred - 1) & 1;
            const float gam = tt[0], del = tt[1], rho = tt[2];
            if (!isfinite(gam) || !isfinite(del) || !isfinite(rho)) {
                drift = true;
                break;
            }
            if (k >= 1) {   // rho = <r, r> of the iterate e holds
                if (rho <= stop2 || rho == 0.0f) break;
                if (rho < 0.5f * rr_best) {
                    rr_best = rho;
                    best_k = k;
                } else if (rho > 1e4f * rr_best) {
                    drift = true;
                    break;
                } else if (k - best_k > kStagnation32) {
                    break;
                }
            }
            if (!(gam > 0.0f)) break;   // restart from the true residual
            // (fast divides: a few ulp in the step coefficients, identical in every CTA)
            const float be = k >= 1 ? __fdividef(gam, gam_prev) : 0.0f;
            const float den = k >= 1 ? del - be * __fdividef(gam, alp_prev) : del;
            if (!(den > 0.0f) || !isfinite(den)) break;
            const float al = __fdividef(gam, den);
            gam_prev = gam;
            alp_prev = al;
            ++iters;
            // p = z + beta p, q = w + beta q (= A p), e += alpha p, r -= alpha q, z = D^{-1} r
#pragma unroll
            for (int t = 0; t < kOnchipRows; ++t) {
                if (t >= nrow) break;
                if (row_of(t) >= 0) {
                    const int l = lrow_of(t);
                    p_[t] = fmaf(be, p_[t], z_[t]);
                    q_[t] = fmaf(be, q_[t], wl[l]);
                    e_[t] = fmaf(al, p_[t], e_[t]);
                    r_[t] = fmaf(-al, q_[t], r_[t]);
                    z_[t] = dl[l] * r_[t];
                }
            }
            // the same for the halo rows, from the owners' w
            const float* rv = recv + par * hm;
            for (int h = threadIdx.x; h < halo_self; h += blockDim.x) {
                const float qv = fmaf(be, qh[h], rv[h]);
                const float r = fmaf(-al, qv, rh[h]);
                qh[h] = qv;
                rh[h] = r;
                zl[rows_max + h] = dh[h] * r;
            }
            coarse(par, al, be, false);
        }
        if (aborted) {
            status = CGP_ETIMEOUT;
            break;
        }
        // ---- x += ||r|| e (FP64) unless the FP32 recurrence drifted away
        if (!drift) {
            const double norm = sc.norm;
#pragma unroll
            for (int t = 0; t < kOnchipRows; ++t) {
                const int i = row_of(t);
                if (i >= 0) __stcg(xv + i, ldcg(xv + i) + norm * (double)e_[t]);
            }
        }
        oc_barrier();
        ++outer;
        if (drift && outer > 2) {
            status = CGP_ENONFINITE;   // the FP32 solve keeps failing: let the caller see it
            break;
        }
    }
    // ---- pure-Neumann mean fix
    if (a.mlump && status != CGP_ETIMEOUT) {
        double acc[2] = {0.0, 0.0};
#pragma unroll
        for (int t = 0; t < kOnchipRows; ++t) {
            const int i = row_of(t);
            if (i >= 0) {
                acc[0] += __ldg(a.mlump + i) * ldcg(xv + i);
                acc[1] += __ldg(a.mlump + i);
            }
        }
        cred64(acc, tot);
        if (threadIdx.x == 0) sc.mu = tot[0] / tot[1];
        __syncthreads();
        const double mu = sc.mu;
#pragma unroll
        for (int t = 0; t < kOnchipRows; ++t) {
            const int i = row_of(t);
            if (i >= 0) __stcg(xv + i, ldcg(xv + i) - mu);
        }
    }
    if (rank == 0 && threadIdx.x == 0) {
        KrylovState* st = a.st;
        st->iter = iters;
        st->bb[0] = bb;
        st->rr[0] = rr_final;
        st->bb[1] = 0.0;
        st->rr[1] = 0.0;
        st->status = status ? status : (converged ? 0 : CGP_ENOTCONV);
        st->done = 1;
        st->pad[0] = outer;
        st->pad[1] = used_alt | (alt_on ? 2 : 0);   // bit 1: the network ran (its gate was open)
    }
    oc_barrier();   // no CTA leaves while another may still access its shared memory
}

// the kernel instance for a plan with nsub subdomains
using OnchipKernelFn = void (*)(CoarsePcgArgs, OnchipPlan);
inline OnchipKernelFn onchip_kernel(int nsub) {
    if (nsub <= 0) return k_pcg_onchip<0>;
    const int r = nsub >= 16 ? nsub / 16 : 1;
    return r >= 8 ? k_pcg_onchip<8> : (r >= 4 ? k_pcg_onchip<4> : (r >= 2 ? k_pcg_onchip<2> : k_pcg_onchip<1>));
}

}  // namespace cgp
