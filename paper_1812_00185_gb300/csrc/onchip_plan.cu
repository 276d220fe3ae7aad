// Host-side plan of the on-chip cluster solve (see coarse_onchip.cuh): which CTA owns which
// SELL-32 slices of the coarse system, where every matrix entry finds its column's value in
// the owning CTA's shared memory, and which values each CTA pushes to its neighbours' halos.
//
// Vertex numbers of refined levels are not spatially local (the vertices added by a
// refinement are numbered after all older ones), so contiguous slice ranges would make most
// neighbours remote.  The slices are instead split by recursive coordinate bisection of
// their centroids into equal-count groups: each CTA owns a compact region and only values
// along region boundaries cross the cluster.  Within a slice, the order of each row's
// entries is chosen so that the 32 lanes of a gather step hit distinct shared-memory banks
// where possible (the sum a row forms is the same up to FP32 rounding order), and each
// slice's width is padded to a multiple of 4 (padding entries read the row's own z with a
// zero value), so the SpMV runs in 4-entry steps without bounds tests.
#include <algorithm>
#include <numeric>
#include <unordered_map>

#include "onchip_plan.cuh"

namespace cgp {

namespace {

// split idx[lo, hi) into `parts` groups of nearly equal size along the longer extent
void bisect(std::vector<int>& idx, int lo, int hi, int parts, const std::vector<double>& cx,
            const std::vector<double>& cy, std::vector<int>& part_of, int part0) {
    if (parts == 1) {
        for (int i = lo; i < hi; ++i) part_of[idx[i]] = part0;
        return;
    }
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int i = lo; i < hi; ++i) {
        xmin = std::min(xmin, cx[idx[i]]);
        xmax = std::max(xmax, cx[idx[i]]);
        ymin = std::min(ymin, cy[idx[i]]);
        ymax = std::max(ymax, cy[idx[i]]);
    }
    const bool byx = (xmax - xmin) >= (ymax - ymin);
    const int left = parts / 2;
    const int mid = lo + (int)(((int64_t)(hi - lo) * left) / parts);
    std::nth_element(idx.begin() + lo, idx.begin() + mid, idx.begin() + hi, [&](int a, int b) {
        const double ka = byx ? cx[a] : cy[a], kb = byx ? cx[b] : cy[b];
        return ka < kb || (ka == kb && a < b);
    });
    bisect(idx, lo, mid, left, cx, cy, part_of, part0);
    bisect(idx, mid, hi, parts - left, cx, cy, part_of, part0 + left);
}

}  // namespace

bool onchip_plan(int n, const std::vector<int32_t>& ptr, const std::vector<int32_t>& col,
                 const std::vector<double>& xy, int ncl, size_t smem_limit, OnchipHostPlan& P) {
    const int S = (int)ptr.size() - 1;
    P = OnchipHostPlan{};
    if (ncl < 1 || ncl > kOnchipMaxCluster || S < ncl) return false;
    // ---- partition of the slices
    std::vector<double> cx(S, 0.0), cy(S, 0.0);
    for (int s = 0; s < S; ++s) {
        const int i1 = std::min(n, 32 * s + 32);
        for (int i = 32 * s; i < i1; ++i) {
            cx[s] += xy[2 * (size_t)i];
            cy[s] += xy[2 * (size_t)i + 1];
        }
        cx[s] /= (i1 - 32 * s);
        cy[s] /= (i1 - 32 * s);
    }
    std::vector<int> part(S), idx(S);
    std::iota(idx.begin(), idx.end(), 0);
    bisect(idx, 0, S, ncl, cx, cy, part, 0);
    P.soff.assign(ncl + 1, 0);
    for (int s = 0; s < S; ++s) P.soff[part[s] + 1]++;
    for (int c = 0; c < ncl; ++c) P.soff[c + 1] += P.soff[c];
    int smax = 0;
    for (int c = 0; c < ncl; ++c) smax = std::max(smax, P.soff[c + 1] - P.soff[c]);
    if ((smax + kOnchipThreads / 32 - 1) / (kOnchipThreads / 32) > kOnchipRows) return false;
    P.slist.resize(S);
    std::vector<int> fill(P.soff.begin(), P.soff.end() - 1), pos(S);
    for (int s = 0; s < S; ++s) {   // ascending slice order inside each CTA
        pos[s] = fill[part[s]] - P.soff[part[s]];
        P.slist[fill[part[s]]++] = s;
    }
    P.ncl = ncl;
    P.rows_max = 32 * smax;
    // ---- local indices, halos, sends
    P.ebase.resize(S);
    std::vector<std::vector<std::pair<int, int>>> sends(ncl);   // per owner: (local row, dest rank << 16 | slot)
    std::vector<int> halo_of(ptr[S], -1);
    int64_t eb = 0;
    for (int c = 0; c < ncl; ++c) {
        std::unordered_map<int, int> halo;
        const int64_t eb0 = eb;
        for (int q = P.soff[c]; q < P.soff[c + 1]; ++q) {
            const int s = P.slist[q];
            P.ebase[q] = (int32_t)eb;
            eb += 32 * onchip_width4((ptr[s + 1] - ptr[s]) >> 5);
            for (int64_t e = ptr[s]; e < ptr[s + 1]; ++e) {
                const int j = col[e], o = part[j >> 5];
                if (o == c) continue;
                auto it = halo.find(j);
                int h;
                if (it == halo.end()) {
                    h = (int)halo.size();
                    halo.emplace(j, h);
                    sends[o].push_back({32 * pos[j >> 5] + (j & 31), (c << 16) | h});
                } else {
                    h = it->second;
                }
                halo_of[e] = h;
            }
        }
        P.ent_max = std::max<int64_t>(P.ent_max, eb - eb0);
        P.halo_max = std::max(P.halo_max, (int)halo.size());
        P.halo_n.push_back((int32_t)halo.size());
    }
    if (P.halo_max >= (1 << 16)) return false;
    P.li.assign(eb, 0);
    P.src.assign(eb, -1);
    // ---- entry order of every slice (bank-aware) and the local index of each entry
    std::vector<int> lidx(32 * 64), order(32 * 64);
    for (int q = 0; q < S; ++q) {
        const int s = P.slist[q];
        const int w = (ptr[s + 1] - ptr[s]) >> 5;
        if (w > 64) return false;
        for (int lane = 0; lane < 32; ++lane)
            for (int k = 0; k < w; ++k) {
                const int64_t e = ptr[s] + 32 * k + lane;
                const int j = col[e];
                lidx[lane * w + k] = halo_of[e] >= 0 ? P.rows_max + halo_of[e] : 32 * pos[j >> 5] + (j & 31);
            }
        // greedy: slot k takes, lane by lane, an unplaced entry whose bank no other lane of
        // the slot uses with a different address (equal addresses are a broadcast)
        std::vector<char> placed(32 * (size_t)w, 0);
        for (int k = 0; k < w; ++k) {
            int bank_addr[32];
            std::fill(bank_addr, bank_addr + 32, -1);
            for (int lane = 0; lane < 32; ++lane) {
                int best = -1, best_cost = 1 << 30;
                for (int m = 0; m < w; ++m) {
                    if (placed[lane * w + m]) continue;
                    const int a = lidx[lane * w + m], b = a & 31;
                    const int cost = (bank_addr[b] < 0 || bank_addr[b] == a) ? 0 : 1;
                    if (cost < best_cost) {
                        best_cost = cost;
                        best = m;
                        if (cost == 0) break;
                    }
                }
                placed[lane * w + best] = 1;
                order[lane * w + k] = best;
                const int a = lidx[lane * w + best];
                if (bank_addr[a & 31] < 0) bank_addr[a & 31] = a;
            }
        }
        for (int lane = 0; lane < 32; ++lane) {
            for (int k = 0; k < w; ++k) {
                const int m = order[lane * w + k];
                const int64_t dst = P.ebase[q] + 32 * k + lane;
                P.src[dst] = (int32_t)(ptr[s] + 32 * m + lane);
                P.li[dst] = lidx[lane * w + m];
            }
            for (int k = w; k < onchip_width4(w); ++k) {   // padding: own row, value 0
                const int64_t dst = P.ebase[q] + 32 * k + lane;
                P.src[dst] = -1;
                P.li[dst] = 32 * pos[s] + lane;
            }
        }
    }
    P.send_off.assign(ncl + 1, 0);
    for (int c = 0; c < ncl; ++c) {
        P.send_off[c + 1] = P.send_off[c] + (int)sends[c].size();
        P.send_max = std::max(P.send_max, (int)sends[c].size());
        for (auto& pr : sends[c]) {
            P.send_lr.push_back(pr.first);
            P.send_dst.push_back(pr.second);
        }
    }
    P.bytes = onchip_smem_bytes(P.rows_max, P.halo_max, P.send_max, P.ent_max);
    return P.bytes <= smem_limit;
}

}  // namespace cgp
