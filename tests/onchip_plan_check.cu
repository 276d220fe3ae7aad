// Host-only check of the on-chip solve's plan (built by the library's onchip_plan.cu) on a
// SELL-32 pattern read from a file: every invariant the kernel relies on for in-bounds,
// correct gathers.  Usage: onchip_plan_check <pattern file> <cluster size> <shared-memory limit>
// File: int64 n, int64 nslices, int32 ptr[nslices+1], int32 col[ptr[nslices]], double xy[2n].
// Prints "OK <halo_max> <send_max> <bytes>" or "FAIL <reason>".
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../paper_1812_00185_gb300/csrc/onchip_plan.cuh"

using namespace cgp;

#define CHECK(cond, ...)                 \
    do {                                 \
        if (!(cond)) {                   \
            printf("FAIL ");             \
            printf(__VA_ARGS__);         \
            printf("\n");                \
            return 1;                    \
        }                                \
    } while (0)

int main(int argc, char** argv) {
    if (argc < 4) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    int64_t hdr[2];
    if (fread(hdr, 8, 2, f) != 2) return 2;
    const int n = (int)hdr[0], S = (int)hdr[1];
    std::vector<int32_t> ptr(S + 1);
    if (fread(ptr.data(), 4, S + 1, f) != (size_t)(S + 1)) return 2;
    std::vector<int32_t> col(ptr[S]);
    std::vector<double> xy(2 * (size_t)n);
    if (fread(col.data(), 4, ptr[S], f) != (size_t)ptr[S] || fread(xy.data(), 8, 2 * n, f) != (size_t)(2 * n)) return 2;
    fclose(f);
    const int ncl = atoi(argv[2]);
    const size_t limit = (size_t)atoll(argv[3]);
    OnchipHostPlan P;
    const bool ok = onchip_plan(n, ptr, col, xy, ncl, limit, P);
    CHECK(ok, "plan refused");
    CHECK((int)P.soff.size() == ncl + 1 && P.soff[0] == 0 && P.soff[ncl] == S, "slice offsets");
    std::vector<int> owner(S, -1), pos(S, -1);
    for (int c = 0; c < ncl; ++c) {
        CHECK(P.soff[c + 1] >= P.soff[c], "offsets not monotone");
        CHECK(P.soff[c + 1] - P.soff[c] <= (kOnchipThreads / 32) * kOnchipRows, "too many slices in CTA %d", c);
        CHECK(32 * (P.soff[c + 1] - P.soff[c]) <= P.rows_max, "rows_max");
        for (int q = P.soff[c]; q < P.soff[c + 1]; ++q) {
            const int s = P.slist[q];
            CHECK(s >= 0 && s < S && owner[s] < 0, "slice %d listed twice or out of range", s);
            owner[s] = c;
            pos[s] = q - P.soff[c];
        }
    }
    for (int s = 0; s < S; ++s) CHECK(owner[s] >= 0, "slice %d not owned", s);
    // halo contents per CTA, from the send lists of the other CTAs
    std::vector<std::vector<int>> halo(ncl, std::vector<int>(P.halo_max, -1));
    for (int o = 0; o < ncl; ++o)
        for (int i = P.send_off[o]; i < P.send_off[o + 1]; ++i) {
            const int lr = P.send_lr[i], d = P.send_dst[i], c = d >> 16, h = d & 0xFFFF;
            CHECK(c >= 0 && c < ncl && c != o, "send destination");
            CHECK(h < P.halo_n[c] && h < P.halo_max, "halo slot beyond the CTA's halo");
            CHECK(halo[c][h] == -1, "halo slot filled twice");
            CHECK(lr / 32 < P.soff[o + 1] - P.soff[o], "send of a row the CTA does not own");
            halo[c][h] = 32 * P.slist[P.soff[o] + lr / 32] + lr % 32;
        }
    for (int c = 0; c < ncl; ++c)
        for (int h = 0; h < P.halo_n[c]; ++h) CHECK(halo[c][h] >= 0, "halo slot %d of CTA %d never sent", h, c);
    // every local entry: a real entry of its own slice and lane, or padding reading its own row
    std::vector<int> seen(ptr[S], 0);
    for (int c = 0; c < ncl; ++c) {
        const int eb0 = P.soff[c] < P.soff[c + 1] ? P.ebase[P.soff[c]] : 0;
        for (int q = P.soff[c]; q < P.soff[c + 1]; ++q) {
            const int s = P.slist[q], w = (ptr[s + 1] - ptr[s]) >> 5, w4 = onchip_width4(w);
            CHECK(P.ebase[q] - eb0 + 32 * w4 <= P.ent_max, "entries beyond ent_max");
            for (int k = 0; k < w4; ++k)
                for (int l = 0; l < 32; ++l) {
                    const int64_t el = P.ebase[q] + 32 * k + l;
                    const int e = P.src[el], li = P.li[el];
                    CHECK(li >= 0 && li < P.rows_max + P.halo_max, "local index out of range");
                    if (e < 0) {
                        CHECK(k >= w && li == 32 * (q - P.soff[c]) + l, "padding entry");
                        continue;
                    }
                    CHECK(e >= ptr[s] && e < ptr[s + 1] && (e - ptr[s]) % 32 == l, "entry from another slice or lane");
                    seen[e]++;
                    const int j = col[e];
                    int g;
                    if (li < P.rows_max) {
                        CHECK(li / 32 < P.soff[c + 1] - P.soff[c], "own index beyond the CTA's rows");
                        g = 32 * P.slist[P.soff[c] + li / 32] + li % 32;
                    } else {
                        g = halo[c][li - P.rows_max];
                    }
                    CHECK(g == j, "entry resolves to column %d instead of %d", g, j);
                }
        }
    }
    for (int64_t e = 0; e < ptr[S]; ++e) CHECK(seen[e] == 1, "entry %lld placed %d times", (long long)e, seen[e]);
    CHECK(P.bytes == onchip_smem_bytes(P.rows_max, P.halo_max, P.send_max, P.ent_max) && P.bytes <= limit, "bytes");
    printf("OK %d %d %zu\n", P.halo_max, P.send_max, P.bytes);
    return 0;
}
