// Host-only check of the on-chip solve's plan (built by the library's onchip_plan.cu) on a
// coarse system read from a file: every invariant the kernel relies on for in-bounds,
// correct gathers, and the subdomain coarse space (E = Z^T A Z recomputed here from the
// matrix, and the pseudo-inverse identities of the plan's E^+).
// Usage: onchip_plan_check <file> <cluster size> <subdomains per CTA> <shared-memory limit>
// File: int64 n, int64 nslices, int32 rowptr[n+1], int32 sell_ptr[nslices+1],
//       int32 sell_col[sell_ptr[nslices]], double val[sell_ptr[nslices]], uint8 in_space[n],
//       double xy[2n].
// Prints "OK <rows_max> <halo_max> <send_max> <ent_max> <nsub> <bytes>" or "FAIL <reason>".
#include <cmath>
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

template <class T>
static bool rd(FILE* f, std::vector<T>& v, size_t n) {
    v.resize(n);
    return fread(v.data(), sizeof(T), n, f) == n;
}

int main(int argc, char** argv) {
    if (argc < 5) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    int64_t hdr[2];
    if (fread(hdr, 8, 2, f) != 2) return 2;
    const int n = (int)hdr[0], S = (int)hdr[1];
    std::vector<int32_t> rowptr, ptr, col;
    std::vector<double> val, xy;
    std::vector<uint8_t> in_space;
    if (!rd(f, rowptr, n + 1) || !rd(f, ptr, S + 1) || !rd(f, col, ptr[S]) || !rd(f, val, ptr[S]) ||
        !rd(f, in_space, n) || !rd(f, xy, 2 * (size_t)n))
        return 2;
    fclose(f);
    const int ncl = atoi(argv[2]), spc = atoi(argv[3]);
    const size_t limit = (size_t)atoll(argv[4]);
    const int W = kOnchipWarps;
    OnchipHostPlan P;
    CHECK(onchip_plan(n, rowptr, ptr, col, xy, in_space, ncl, spc, limit, P), "plan refused");
    CHECK(onchip_coarse_space(rowptr, ptr, col, val, P), "coarse space refused");
    CHECK(P.nsub == ncl * spc && (spc == 0 || P.wpg * spc == W), "subdomain counts");
    CHECK((int)P.soff.size() == ncl + 1 && P.soff[0] == 0, "slice offsets");
    const int npos = P.soff[ncl];
    CHECK((int)P.grow.size() == 32 * npos && (int)P.width.size() == npos && (int)P.ebase.size() == npos, "array sizes");
    // ---- every global row exactly once, at a warp slot the kernel visits
    std::vector<int> owner(n, -1), lrow(n, -1), warp(n, -1);
    for (int c = 0; c < ncl; ++c) {
        const int np = P.soff[c + 1] - P.soff[c];
        CHECK(np >= 0 && np % W == 0 && np / W <= kOnchipRows, "positions of CTA %d", c);
        CHECK(32 * np <= P.rows_max, "rows_max");
        for (int q = 0; q < np; ++q)
            for (int l = 0; l < 32; ++l) {
                const int g = P.grow[32 * (size_t)(P.soff[c] + q) + l];
                if (g == -1) continue;
                const int i = g >= 0 ? g : -2 - g;
                CHECK(i >= 0 && i < n && owner[i] < 0, "row %d listed twice or out of range", i);
                CHECK((g >= 0) == (in_space[i] != 0), "coarse-space flag of row %d", i);
                owner[i] = c;
                lrow[i] = 32 * q + l;
                warp[i] = c * W + q % W;
            }
    }
    for (int i = 0; i < n; ++i) CHECK(owner[i] >= 0, "row %d not owned", i);
    // ---- subdomains: a warp's rows share one; rows outside the space have none
    CHECK((int)P.sub.size() == n, "sub size");
    for (int i = 0; i < n; ++i) {
        if (!P.nsub) break;
        CHECK(in_space[i] ? P.sub[i] == warp[i] / P.wpg : P.sub[i] == P.nsub, "subdomain of row %d", i);
    }
    // ---- halo contents per CTA, from the send lists of the other CTAs
    std::vector<std::vector<int>> halo(ncl, std::vector<int>(P.halo_max, -1));
    for (int o = 0; o < ncl; ++o)
        for (int i = P.send_off[o]; i < P.send_off[o + 1]; ++i) {
            const int lr = P.send_lr[i], d = P.send_dst[i], c = d >> 16, h = d & 0xFFFF;
            CHECK(c >= 0 && c < ncl && c != o, "send destination");
            CHECK(h < P.halo_n[c] && h < P.halo_max, "halo slot beyond the CTA's halo");
            CHECK(halo[c][h] == -1, "halo slot filled twice");
            CHECK(lr >= 0 && lr < 32 * (P.soff[o + 1] - P.soff[o]), "send of a row the CTA does not own");
            const int g = P.grow[32 * (size_t)P.soff[o] + lr];
            CHECK(g != -1, "send of a padding row");
            halo[c][h] = g >= 0 ? g : -2 - g;
        }
    for (int c = 0; c < ncl; ++c)
        for (int h = 0; h < P.halo_max; ++h) {
            const uint8_t hs = P.hsub[(size_t)c * P.halo_max + h];
            if (h >= P.halo_n[c]) {
                CHECK(hs == P.nsub, "unused halo slot with a subdomain");
                continue;
            }
            CHECK(halo[c][h] >= 0, "halo slot %d of CTA %d never sent", h, c);
            CHECK(hs == (P.nsub ? P.sub[halo[c][h]] : 0), "subdomain of halo slot %d of CTA %d", h, c);
            CHECK(P.hrow[(size_t)c * P.halo_max + h] == halo[c][h], "global row of halo slot %d of CTA %d", h, c);
        }
    // ---- the sends of each warp: a contiguous segment, rows the warp owns
    CHECK((int)P.send_woff.size() == ncl * (W + 1), "send_woff size");
    for (int c = 0; c < ncl; ++c) {
        CHECK(P.send_woff[c * (W + 1)] == P.send_off[c] && P.send_woff[c * (W + 1) + W] == P.send_off[c + 1],
              "send segments of CTA %d", c);
        for (int w = 0; w < W; ++w) {
            CHECK(P.send_woff[c * (W + 1) + w] <= P.send_woff[c * (W + 1) + w + 1], "send segment order");
            for (int i = P.send_woff[c * (W + 1) + w]; i < P.send_woff[c * (W + 1) + w + 1]; ++i)
                CHECK((P.send_lr[i] / 32) % W == w, "send %d of CTA %d not owned by warp %d", i, c, w);
        }
    }
    // ---- the subdomains each CTA corrects: its own first, then every one of its halo rows,
    // each once
    CHECK((int)P.need_n.size() == ncl && (int)P.need.size() == ncl * P.need_max, "need sizes");
    for (int c = 0; c < ncl && P.nsub; ++c) {
        std::vector<int> cnt(P.nsub, 0);
        CHECK(P.need_n[c] <= P.need_max, "need_n");
        for (int k = 0; k < P.need_n[c]; ++k) {
            const int j = P.need[(size_t)c * P.need_max + k];
            CHECK(j < P.nsub && cnt[j]++ == 0, "need list of CTA %d", c);
            if (k < spc) CHECK(j == c * spc + k, "own subdomains of CTA %d first", c);
        }
        for (int h = 0; h < P.halo_n[c]; ++h) {
            const int j = P.hsub[(size_t)c * P.halo_max + h];
            CHECK(j == P.nsub || cnt[j] == 1, "halo subdomain %d of CTA %d not corrected", j, c);
        }
    }
    // ---- every local entry: a real entry of its own row, or padding reading its own row
    std::vector<int> seen(ptr[S], 0);
    for (int c = 0; c < ncl; ++c) {
        const int64_t eb0 = P.soff[c] < P.soff[c + 1] ? P.ebase[P.soff[c]] : 0;
        int64_t next = eb0;
        for (int q = P.soff[c]; q < P.soff[c + 1]; ++q) {
            const int lq = q - P.soff[c], w4 = P.width[q];
            CHECK(w4 % 4 == 0 && P.ebase[q] == next, "width / ebase of position %d", q);
            next += 32 * (int64_t)w4;
            CHECK(next - eb0 <= P.ent_max, "entries beyond ent_max");
            for (int l = 0; l < 32; ++l) {
                const int g = P.grow[32 * (size_t)q + l];
                const int i = g == -1 ? -1 : (g >= 0 ? g : -2 - g);
                const int len = i >= 0 ? rowptr[i + 1] - rowptr[i] : 0;
                CHECK(len <= w4, "row %d longer than its slice", i);
                int real = 0;
                for (int k = 0; k < w4; ++k) {
                    const int64_t el = P.ebase[q] + 32 * k + l;
                    const int e = P.src[el], li = P.li[el];
                    CHECK(li >= 0 && li < P.rows_max + P.halo_max, "local index out of range");
                    if (e < 0) {
                        CHECK(li == 32 * lq + l, "padding entry");
                        continue;
                    }
                    ++real;
                    CHECK(i >= 0 && e >= ptr[i >> 5] && (e - ptr[i >> 5]) % 32 == (i & 31) &&
                              (e - ptr[i >> 5]) / 32 < len,
                          "entry from another row");
                    seen[e]++;
                    const int j = col[e];
                    int gj;
                    if (li < P.rows_max) {
                        CHECK(li < 32 * (P.soff[c + 1] - P.soff[c]), "own index beyond the CTA's rows");
                        const int gg = P.grow[32 * (size_t)P.soff[c] + li];
                        gj = gg == -1 ? -1 : (gg >= 0 ? gg : -2 - gg);
                    } else {
                        CHECK(li - P.rows_max < P.halo_n[c], "halo index beyond the CTA's halo");
                        gj = halo[c][li - P.rows_max];
                    }
                    CHECK(gj == j, "entry resolves to column %d instead of %d", gj, j);
                }
                CHECK(real == len, "row %d has %d of %d entries", i, real, len);
            }
        }
    }
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < rowptr[i + 1] - rowptr[i]; ++k)
            CHECK(seen[ptr[i >> 5] + 32 * k + (i & 31)] == 1, "entry %d of row %d placed %d times", k, i,
                  seen[ptr[i >> 5] + 32 * k + (i & 31)]);
    // ---- coarse space: E = Z^T A Z recomputed, E^+ against the pseudo-inverse identities
    const int m = P.nsub;
    if (m) {
        std::vector<double> E((size_t)m * m, 0.0);
        for (int i = 0; i < n; ++i) {
            if (!in_space[i]) continue;
            for (int k = 0; k < rowptr[i + 1] - rowptr[i]; ++k) {
                const int64_t e = ptr[i >> 5] + 32 * k + (i & 31);
                const int j = col[e];
                if (in_space[j]) E[(size_t)(warp[i] / P.wpg) * m + warp[j] / P.wpg] += val[e];
            }
        }
        double emax = 0.0;
        for (size_t t = 0; t < E.size(); ++t) {
            emax = std::fmax(emax, std::fabs(E[t]));
            CHECK(std::fabs(E[t] - P.E[t]) <= 1e-12 * (std::fabs(E[t]) + 1.0), "E entry %zu", t);
        }
        // X = E^+ (float): E X E = E and X E X = X, relative to the sizes involved
        std::vector<double> X(P.einv.begin(), P.einv.end()), EX((size_t)m * m, 0.0), XE((size_t)m * m, 0.0);
        double xmax = 0.0;
        for (int j = 0; j < m; ++j)
            for (int k = 0; k < m; ++k) {
                xmax = std::fmax(xmax, std::fabs(X[(size_t)j * m + k]));
                CHECK(X[(size_t)j * m + k] == X[(size_t)k * m + j], "E^+ not symmetric");
            }
        for (int j = 0; j < m; ++j)
            for (int k = 0; k < m; ++k)
                for (int t = 0; t < m; ++t) {
                    EX[(size_t)j * m + k] += E[(size_t)j * m + t] * X[(size_t)t * m + k];
                    XE[(size_t)j * m + k] += X[(size_t)j * m + t] * E[(size_t)t * m + k];
                }
        double r1 = 0.0, r2 = 0.0;
        for (int j = 0; j < m; ++j)
            for (int k = 0; k < m; ++k) {
                double exe = 0.0, xex = 0.0;
                for (int t = 0; t < m; ++t) {
                    exe += EX[(size_t)j * m + t] * E[(size_t)t * m + k];
                    xex += XE[(size_t)j * m + t] * X[(size_t)t * m + k];
                }
                r1 = std::fmax(r1, std::fabs(exe - E[(size_t)j * m + k]));
                r2 = std::fmax(r2, std::fabs(xex - X[(size_t)j * m + k]));
            }
        CHECK(r1 <= 1e-4 * emax && r2 <= 1e-4 * xmax, "pseudo-inverse identities: %g %g", r1 / emax, r2 / xmax);
    }
    CHECK(P.bytes == onchip_smem_bytes(P.rows_max, P.halo_max, P.send_max, P.ent_max, P.nsub, P.need_max) &&
              P.bytes <= limit,
          "bytes");
    printf("OK %d %d %d %lld %d %zu\n", P.rows_max, P.halo_max, P.send_max, (long long)P.ent_max, P.nsub, P.bytes);
    return 0;
}
