// Error reporting and the exclusive scan used by mesh construction.
#include "internal.cuh"

#include <cstring>

namespace cgp {

static thread_local char g_err[1024] = {0};

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

// ---------------------------------------------------------------- scan
// Three-pass exclusive scan: per-block scan of kScanTile items, scan of the
// block totals in one block, then the block offsets are added.
constexpr int kScanItems = 16;                      // per thread
constexpr int kScanTile = kBlock * kScanItems;      // 4096 items per block
constexpr int kMaxScanBlocks = kBlock * 32;         // top-level scan: 256 threads x 32 items

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t* total) {
    __shared__ int32_t ws[kBlock / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int32_t w = lane < kBlock / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kBlock / 32) ws[lane] = w;
    }
    __syncthreads();
    int32_t pre = (wid > 0 ? ws[wid - 1] : 0) + x - v;
    *total = ws[kBlock / 32 - 1];
    __syncthreads();
    return pre;
}

__global__ void scan_tiles(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n,
                           int32_t* __restrict__ tile_sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t loc[kScanItems];
    int32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t j = base + i;
        loc[i] = j < n ? in[j] : 0;
        s += loc[i];
    }
    int32_t tot;
    int32_t pre = block_exclusive_scan(s, &tot);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t j = base + i;
        if (j < n) out[j] = pre;
        pre += loc[i];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void scan_top(int32_t* __restrict__ sums, int nb, int32_t* __restrict__ out_total) {
    constexpr int items = kMaxScanBlocks / kBlock;
    const int base = threadIdx.x * items;
    int32_t loc[items];
    int32_t s = 0;
#pragma unroll
    for (int i = 0; i < items; ++i) {
        loc[i] = base + i < nb ? sums[base + i] : 0;
        s += loc[i];
    }
    int32_t tot;
    int32_t pre = block_exclusive_scan(s, &tot);
#pragma unroll
    for (int i = 0; i < items; ++i) {
        if (base + i < nb) sums[base + i] = pre;
        pre += loc[i];
    }
    if (threadIdx.x == 0) *out_total = tot;
}

__global__ void scan_add(int32_t* __restrict__ out, int64_t n, const int32_t* __restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    const int32_t off = sums[blockIdx.x];
    for (int i = threadIdx.x; i < kScanTile; i += kBlock) {
        int64_t j = base + i;
        if (j < n) out[j] += off;
    }
}

size_t scan_tmp_ints(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 1; }

int exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp, cudaStream_t stream) {
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb < 1) nb = 1;
    if (nb > kMaxScanBlocks) {
        set_error("scan of %lld items exceeds the supported %lld", (long long)n,
                  (long long)kMaxScanBlocks * kScanTile);
        return CGP_EINVAL;
    }
    scan_tiles<<<(int)nb, kBlock, 0, stream>>>(in, out, n, tmp);
    scan_top<<<1, kBlock, 0, stream>>>(tmp, (int)nb, out + n);
    scan_add<<<(int)nb, kBlock, 0, stream>>>(out, n, tmp);
    CGP_LAUNCH_CHECK();
    return CGP_OK;
}

}  // namespace cgp

extern "C" const char* cgp_last_error(void) { return cgp::g_err; }
