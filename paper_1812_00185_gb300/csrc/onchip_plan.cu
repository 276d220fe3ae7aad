// Host-side plan of the on-chip cluster solve (see coarse_onchip.cuh): which warp of which
// CTA owns which rows of the coarse system, where every matrix entry finds its column's value
// in the owning CTA's shared memory, which values each CTA pushes to its neighbours' halos,
// and the subdomain coarse space of the preconditioner.
//
// Vertex numbers of refined levels are not spatially local (the vertices added by a
// refinement are numbered after all older ones), so the rows are split by recursive
// coordinate bisection of the vertices into ncl x 16 leaves of equal size: each warp owns a
// compact patch, each CTA the 16 patches of one subtree, and only values along CTA region
// boundaries cross the cluster.  A subdomain of the coarse correction is the union of
// `wpg` sibling leaves, so its sums are warp sums.  Within a leaf, rows are ordered by
// length (slices of equal-length rows need little padding); within a slice, the order of
// each row's entries is chosen so that the 32 lanes of a gather step hit distinct
// shared-memory banks where possible (the sum a row forms is the same up to FP32 rounding
// order), and each slice's width is padded to a multiple of 4 (padding entries read the
// row's own z with a zero value), so the SpMV runs in 4-entry steps without bounds tests.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <unordered_map>

#include "onchip_plan.cuh"

namespace cgp {

namespace {

// split idx[lo, hi) into `parts` groups of nearly equal size along the longer extent
void bisect(std::vector<int>& idx, int lo, int hi, int parts, const std::vector<double>& xy,
            std::vector<int>& part_of, int part0) {
    if (parts == 1) {
        for (int i = lo; i < hi; ++i) part_of[idx[i]] = part0;
        return;
    }
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int i = lo; i < hi; ++i) {
        const double x = xy[2 * (size_t)idx[i]], y = xy[2 * (size_t)idx[i] + 1];
        xmin = std::min(xmin, x);
        xmax = std::max(xmax, x);
        ymin = std::min(ymin, y);
        ymax = std::max(ymax, y);
    }
    const int d = (xmax - xmin) >= (ymax - ymin) ? 0 : 1;
    const int left = parts / 2;
    const int mid = lo + (int)(((int64_t)(hi - lo) * left) / parts);
    std::nth_element(idx.begin() + lo, idx.begin() + mid, idx.begin() + hi, [&](int a, int b) {
        const double ka = xy[2 * (size_t)a + d], kb = xy[2 * (size_t)b + d];
        return ka < kb || (ka == kb && a < b);
    });
    bisect(idx, lo, mid, left, xy, part_of, part0);
    bisect(idx, mid, hi, parts - left, xy, part_of, part0 + left);
}

// cyclic Jacobi eigen-decomposition of the symmetric m x m matrix a (destroyed): eigenvalues
// in w, eigenvectors in the columns of v
void sym_eigen(int m, std::vector<double>& a, std::vector<double>& w, std::vector<double>& v) {
    v.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) v[(size_t)i * m + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                const double x = a[(size_t)i * m + j] * a[(size_t)i * m + j];
                tot += x;
                if (i != j) off += x;
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double apq = a[(size_t)p * m + q];
                if (apq == 0.0) continue;
                const double app = a[(size_t)p * m + p], aqq = a[(size_t)q * m + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < m; ++k) {   // columns p, q
                    const double akp = a[(size_t)k * m + p], akq = a[(size_t)k * m + q];
                    a[(size_t)k * m + p] = c * akp - s * akq;
                    a[(size_t)k * m + q] = s * akp + c * akq;
                }
                for (int k = 0; k < m; ++k) {   // rows p, q
                    const double apk = a[(size_t)p * m + k], aqk = a[(size_t)q * m + k];
                    a[(size_t)p * m + k] = c * apk - s * aqk;
                    a[(size_t)q * m + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < m; ++k) {
                    const double vkp = v[(size_t)k * m + p], vkq = v[(size_t)k * m + q];
                    v[(size_t)k * m + p] = c * vkp - s * vkq;
                    v[(size_t)k * m + q] = s * vkp + c * vkq;
                }
            }
    }
    w.resize(m);
    for (int i = 0; i < m; ++i) w[i] = a[(size_t)i * m + i];
}

}  // namespace

bool onchip_plan(int n, const std::vector<int32_t>& rowptr, const std::vector<int32_t>& sell_ptr,
                 const std::vector<int32_t>& sell_col, const std::vector<double>& xy,
                 const std::vector<uint8_t>& in_space, int ncl, int sub_per_cta, size_t smem_limit,
                 OnchipHostPlan& P) {
    P = OnchipHostPlan{};
    if (ncl < 1 || ncl > kOnchipMaxCluster || (ncl & (ncl - 1)) || n < 1) return false;
    if (sub_per_cta < 0 || sub_per_cta > kOnchipMaxSubPerCta || (sub_per_cta & (sub_per_cta - 1))) return false;
    const int W = kOnchipWarps, nleaf = ncl * W;
    // ---- leaves: compact groups of rows, one per warp
    std::vector<int> leaf(n), idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    bisect(idx, 0, n, nleaf, xy, leaf, 0);
    std::vector<std::vector<int>> rows(nleaf);
    for (int i = 0; i < n; ++i) rows[leaf[i]].push_back(i);
    auto len = [&](int i) { return rowptr[i + 1] - rowptr[i]; };
    int tmax = 0;
    for (auto& r : rows) {
        if ((int)r.size() > 32 * kOnchipRows) return false;
        std::stable_sort(r.begin(), r.end(), [&](int a, int b) { return len(a) > len(b); });
        tmax = std::max(tmax, ((int)r.size() + 31) / 32);
    }
    P.ncl = ncl;
    P.nsub = sub_per_cta ? ncl * sub_per_cta : 0;
    P.wpg = sub_per_cta ? W / sub_per_cta : 0;
    // ---- list positions, local rows
    P.soff.assign(ncl + 1, 0);
    std::vector<int> tc(ncl, 0);
    for (int c = 0; c < ncl; ++c) {
        for (int w = 0; w < W; ++w) tc[c] = std::max(tc[c], ((int)rows[c * W + w].size() + 31) / 32);
        P.soff[c + 1] = P.soff[c] + W * tc[c];
    }
    P.rows_max = 32 * W * tmax;
    const int npos = P.soff[ncl];
    P.grow.assign(32 * (size_t)npos, -1);
    std::vector<int> owner(n), lrow(n);
    P.sub.assign(n, P.nsub);
    for (int c = 0; c < ncl; ++c)
        for (int w = 0; w < W; ++w) {
            const auto& r = rows[c * W + w];
            for (int k = 0; k < (int)r.size(); ++k) {
                const int i = r[k], q = w + W * (k / 32), l = 32 * q + (k % 32);
                owner[i] = c;
                lrow[i] = l;
                const bool in = in_space.empty() || in_space[i];
                P.grow[32 * (size_t)P.soff[c] + l] = in ? i : -2 - i;
                if (in && P.nsub) P.sub[i] = (c * W + w) / P.wpg;
            }
        }
    // ---- slice widths, halos, sends
    P.ebase.assign(npos, 0);
    P.width.assign(npos, 0);
    std::vector<std::vector<std::pair<int, int>>> sends(ncl);   // per owner: (local row, dest rank << 16 | slot)
    std::vector<int32_t> li_of(rowptr[n]);                      // per CSR entry: local index of its column
    std::vector<std::vector<int>> halo_rows(ncl);
    int64_t eb = 0;
    for (int c = 0; c < ncl; ++c) {
        std::unordered_map<int, int> halo;
        const int64_t eb0 = eb;
        for (int q = P.soff[c]; q < P.soff[c + 1]; ++q) {
            int wmax = 0;
            for (int l = 0; l < 32; ++l) {
                const int g = P.grow[32 * (size_t)q + l];
                if (g == -1) continue;
                const int i = g >= 0 ? g : -2 - g;
                wmax = std::max(wmax, len(i));
                for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                    const int j = sell_col[sell_ptr[i >> 5] + 32 * (e - rowptr[i]) + (i & 31)];
                    if (owner[j] == c) {
                        li_of[e] = lrow[j];
                        continue;
                    }
                    auto it = halo.find(j);
                    int h;
                    if (it == halo.end()) {
                        h = (int)halo.size();
                        halo.emplace(j, h);
                        halo_rows[c].push_back(j);
                        sends[owner[j]].push_back({lrow[j], (c << 16) | h});
                    } else {
                        h = it->second;
                    }
                    li_of[e] = -1 - h;
                }
            }
            P.width[q] = onchip_width4(wmax);
            P.ebase[q] = (int32_t)eb;
            eb += 32 * (int64_t)P.width[q];
        }
        P.ent_max = std::max<int64_t>(P.ent_max, eb - eb0);
        P.halo_max = std::max(P.halo_max, (int)halo.size());
        P.halo_n.push_back((int32_t)halo.size());
    }
    if (P.halo_max >= (1 << 16) || eb >= (int64_t)1 << 31) return false;
    for (auto& e : li_of)
        if (e < 0) e = P.rows_max + (-1 - e);
    P.hsub.assign((size_t)ncl * P.halo_max, (uint8_t)P.nsub);
    P.hrow.assign((size_t)ncl * P.halo_max, 0);
    for (int c = 0; c < ncl; ++c)
        for (int h = 0; h < (int)halo_rows[c].size(); ++h) {
            P.hsub[(size_t)c * P.halo_max + h] = (uint8_t)P.sub[halo_rows[c][h]];
            P.hrow[(size_t)c * P.halo_max + h] = halo_rows[c][h];
        }
    // the subdomains each CTA corrects: its own (in order), then those of its halo rows
    std::vector<std::vector<int>> need(ncl);
    if (P.nsub) {
        for (int c = 0; c < ncl; ++c) {
            std::vector<char> seen(P.nsub, 0);
            for (int j = c * sub_per_cta; j < (c + 1) * sub_per_cta; ++j) {
                seen[j] = 1;
                need[c].push_back(j);
            }
            for (int i : halo_rows[c]) {
                const int j = P.sub[i];
                if (j < P.nsub && !seen[j]) {
                    seen[j] = 1;
                    need[c].push_back(j);
                }
            }
            P.need_max = std::max(P.need_max, (int)need[c].size());
        }
    }
    P.need.assign((size_t)ncl * P.need_max, 0);
    P.need_n.assign(ncl, 0);
    for (int c = 0; c < ncl; ++c) {
        P.need_n[c] = (int32_t)need[c].size();
        for (int k = 0; k < (int)need[c].size(); ++k) P.need[(size_t)c * P.need_max + k] = (uint8_t)need[c][k];
    }
    // ---- entry order of every slice (bank-aware) and the local index of each entry
    P.li.assign(eb, 0);
    P.src.assign(eb, -1);
    std::vector<int> lidx(32 * 64), srcs(32 * 64), order(32 * 64), cnt(32);
    for (int c = 0; c < ncl; ++c)
        for (int q = P.soff[c]; q < P.soff[c + 1]; ++q) {
            const int w4 = P.width[q];
            if (w4 > 64) return false;
            for (int l = 0; l < 32; ++l) {
                const int g = P.grow[32 * (size_t)q + l];
                cnt[l] = 0;
                if (g == -1) continue;
                const int i = g >= 0 ? g : -2 - g;
                cnt[l] = len(i);
                for (int k = 0; k < cnt[l]; ++k) {
                    lidx[l * 64 + k] = li_of[rowptr[i] + k];
                    srcs[l * 64 + k] = sell_ptr[i >> 5] + 32 * k + (i & 31);
                }
            }
            // greedy: slot k takes, lane by lane, an unplaced entry whose bank no other lane
            // of the slot uses with a different address (equal addresses are a broadcast)
            std::vector<char> placed(32 * 64, 0);
            for (int k = 0; k < w4; ++k) {
                int bank_addr[32];
                std::fill(bank_addr, bank_addr + 32, -1);
                for (int l = 0; l < 32; ++l) {
                    order[l * 64 + k] = -1;
                    if (k >= cnt[l]) continue;
                    int best = -1, best_cost = 1 << 30;
                    for (int m = 0; m < cnt[l]; ++m) {
                        if (placed[l * 64 + m]) continue;
                        const int a = lidx[l * 64 + m], b = a & 31;
                        const int cost = (bank_addr[b] < 0 || bank_addr[b] == a) ? 0 : 1;
                        if (cost < best_cost) {
                            best_cost = cost;
                            best = m;
                            if (cost == 0) break;
                        }
                    }
                    placed[l * 64 + best] = 1;
                    order[l * 64 + k] = best;
                    const int a = lidx[l * 64 + best];
                    if (bank_addr[a & 31] < 0) bank_addr[a & 31] = a;
                }
            }
            const int lq = q - P.soff[c];
            for (int l = 0; l < 32; ++l)
                for (int k = 0; k < w4; ++k) {
                    const int64_t dst = P.ebase[q] + 32 * k + l;
                    const int m = order[l * 64 + k];
                    if (m >= 0) {
                        P.src[dst] = srcs[l * 64 + m];
                        P.li[dst] = lidx[l * 64 + m];
                    } else {   // padding: own row, value 0
                        P.src[dst] = -1;
                        P.li[dst] = 32 * lq + l;
                    }
                }
        }
    // sends grouped by the warp that owns their row (local row 32 (w + 16 t) + lane)
    P.send_off.assign(ncl + 1, 0);
    P.send_woff.assign((size_t)ncl * (W + 1), 0);
    for (int c = 0; c < ncl; ++c) {
        auto& sc = sends[c];
        std::stable_sort(sc.begin(), sc.end(), [&](const std::pair<int, int>& a, const std::pair<int, int>& b) {
            return (a.first / 32) % W < (b.first / 32) % W;
        });
        P.send_off[c + 1] = P.send_off[c] + (int)sc.size();
        P.send_max = std::max(P.send_max, (int)sc.size());
        int k = 0;
        for (int w = 0; w <= W; ++w) {
            while (k < (int)sc.size() && (sc[k].first / 32) % W < w) ++k;
            P.send_woff[(size_t)c * (W + 1) + w] = P.send_off[c] + k;
        }
        for (auto& pr : sc) {
            P.send_lr.push_back(pr.first);
            P.send_dst.push_back(pr.second);
        }
    }
    P.bytes = onchip_smem_bytes(P.rows_max, P.halo_max, P.send_max, P.ent_max, P.nsub, P.need_max);
    return P.bytes <= smem_limit;
}

bool onchip_coarse_space(const std::vector<int32_t>& rowptr, const std::vector<int32_t>& sell_ptr,
                         const std::vector<int32_t>& sell_col, const std::vector<double>& val, OnchipHostPlan& P) {
    const int m = P.nsub, n = (int)rowptr.size() - 1;
    P.E.assign((size_t)m * m, 0.0);
    P.einv.assign((size_t)m * m, 0.0f);
    if (m == 0) return true;
    // E_jk = sum of a_il over rows i of subdomain j and columns l of subdomain k
    for (int i = 0; i < n; ++i) {
        const int j = P.sub[i];
        if (j >= m) continue;
        for (int k = 0; k < rowptr[i + 1] - rowptr[i]; ++k) {
            const int64_t e = sell_ptr[i >> 5] + 32 * k + (i & 31);
            const int sk = P.sub[sell_col[e]];
            if (sk < m) P.E[(size_t)j * m + sk] += val[e];
        }
    }
    double amax = 0.0;
    for (double x : P.E) amax = std::max(amax, std::fabs(x));
    for (int j = 0; j < m; ++j)
        for (int k = j + 1; k < m; ++k)
            if (std::fabs(P.E[(size_t)j * m + k] - P.E[(size_t)k * m + j]) > 1e-12 * amax) return false;
    std::vector<double> a(P.E), w, v;
    for (int j = 0; j < m; ++j)   // symmetrise exactly
        for (int k = j + 1; k < m; ++k) a[(size_t)j * m + k] = a[(size_t)k * m + j] = 0.5 * (a[(size_t)j * m + k] + a[(size_t)k * m + j]);
    sym_eigen(m, a, w, v);
    double wmax = 0.0;
    for (double x : w) wmax = std::max(wmax, std::fabs(x));
    if (!(wmax > 0.0)) return false;
    for (double x : w)
        if (x < -1e-10 * wmax) return false;   // not positive semi-definite
    std::vector<double> inv((size_t)m * m, 0.0);
    for (int e = 0; e < m; ++e) {
        if (w[e] <= 1e-12 * wmax) continue;
        const double s = 1.0 / w[e];
        for (int j = 0; j < m; ++j)
            for (int k = 0; k < m; ++k) inv[(size_t)j * m + k] += s * v[(size_t)j * m + e] * v[(size_t)k * m + e];
    }
    for (size_t t = 0; t < inv.size(); ++t) P.einv[t] = (float)inv[t];
    return true;
}

}  // namespace cgp
