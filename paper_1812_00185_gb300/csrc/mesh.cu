// Nested mesh hierarchy on the device: uniform 1->4 refinement (paper Section 2.2)
// and the vertex-adjacency CSR pattern of every level.
//
// Edge numbering without a global sort: once a level's adjacency is in CSR form
// with ascending columns, the edges (a, b), a < b, in ascending lexicographic order
// are exactly the strictly-upper entries of the CSR in storage order.  So the rank
// of edge (a, b) is (number of upper entries in rows < a) + (position of b among the
// upper entries of row a), an exclusive scan of per-row upper counts.
#include "internal.cuh"

namespace cgp {

__global__ void k_check_base(const double* __restrict__ xy, const int32_t* __restrict__ tri, int nt, int nv,
                             int* __restrict__ err) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv || a == b || b == c || a == c) {
        atomicOr(err, 1);
        return;
    }
    double det = (xy[2 * b] - xy[2 * a]) * (xy[2 * c + 1] - xy[2 * a + 1]) -
                 (xy[2 * c] - xy[2 * a]) * (xy[2 * b + 1] - xy[2 * a + 1]);
    if (!(det > 0.0)) atomicOr(err, 2);
}

__global__ void k_count_incidence(const int32_t* __restrict__ tri, int nt, int32_t* __restrict__ cnt) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    atomicAdd(&cnt[tri[3 * t]], 1);
    atomicAdd(&cnt[tri[3 * t + 1]], 1);
    atomicAdd(&cnt[tri[3 * t + 2]], 1);
}

__global__ void k_fill_incidence(const int32_t* __restrict__ tri, int nt, const int32_t* __restrict__ vt_ptr,
                                 int32_t* __restrict__ fill, int32_t* __restrict__ vt_list) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    for (int k = 0; k < 3; ++k) {
        int v = tri[3 * t + k];
        int pos = atomicAdd(&fill[v], 1);
        vt_list[vt_ptr[v] + pos] = t;
    }
}

// Sort each vertex's triangle list ascending (makes everything downstream deterministic).
__global__ void k_sort_incidence(const int32_t* __restrict__ vt_ptr, int32_t* __restrict__ vt_list, int nv,
                                 int* __restrict__ err) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int b = vt_ptr[v], e = vt_ptr[v + 1];
    if (e - b > kMaxInc || e == b) {
        atomicOr(err, e == b ? 8 : 4);
        return;
    }
    for (int i = b + 1; i < e; ++i) {
        int x = vt_list[i], j = i - 1;
        while (j >= b && vt_list[j] > x) {
            vt_list[j + 1] = vt_list[j];
            --j;
        }
        vt_list[j + 1] = x;
    }
}

// Sorted, de-duplicated neighbours of v (v included) into nb[]; returns the count.
__device__ int gather_neighbours(int v, const int32_t* __restrict__ tri, const int32_t* __restrict__ vt_ptr,
                                 const int32_t* __restrict__ vt_list, int32_t* nb) {
    int b = vt_ptr[v], e = vt_ptr[v + 1];
    if (e - b > kMaxInc) e = b + kMaxInc;
    int n = 0;
    nb[n++] = v;
    for (int i = b; i < e; ++i) {
        int t = vt_list[i];
        for (int k = 0; k < 3; ++k) {
            int u = tri[3 * t + k];
            if (u == v) continue;
            // insertion into the sorted prefix, skipping duplicates
            int j = n - 1;
            bool dup = false;
            while (j >= 0 && nb[j] >= u) {
                if (nb[j] == u) { dup = true; break; }
                --j;
            }
            if (dup) continue;
            if (n >= kMaxAdj) return -1;
            for (int m = n; m > j + 1; --m) nb[m] = nb[m - 1];
            nb[j + 1] = u;
            ++n;
        }
    }
    return n;
}

__global__ void k_adj_count(const int32_t* __restrict__ tri, const int32_t* __restrict__ vt_ptr,
                            const int32_t* __restrict__ vt_list, int nv, int32_t* __restrict__ cnt,
                            int* __restrict__ err) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int32_t nb[kMaxAdj];
    int n = gather_neighbours(v, tri, vt_ptr, vt_list, nb);
    if (n < 0) {
        atomicOr(err, 4);
        n = 0;
    }
    cnt[v] = n;
}

__global__ void k_adj_fill(const int32_t* __restrict__ tri, const int32_t* __restrict__ vt_ptr,
                           const int32_t* __restrict__ vt_list, int nv, const int32_t* __restrict__ rowptr,
                           int32_t* __restrict__ col) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int32_t nb[kMaxAdj];
    int n = gather_neighbours(v, tri, vt_ptr, vt_list, nb);
    int r = rowptr[v];
    for (int i = 0; i < n && r + i < rowptr[v + 1]; ++i) col[r + i] = nb[i];
}

__global__ void k_upper_count(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int nv,
                              int32_t* __restrict__ cnt) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int n = 0;
    for (int j = rowptr[v]; j < rowptr[v + 1]; ++j) n += col[j] > v;
    cnt[v] = n;
}

// SELL-32: entries per slice = 32 * (longest row of the slice)
__global__ void k_slice_size(const int32_t* __restrict__ rowptr, int nv, int nslices, int32_t* __restrict__ cnt) {
    int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= nslices) return;
    int w = 0;
    for (int r = 32 * sl; r < 32 * sl + 32 && r < nv; ++r) w = max(w, rowptr[r + 1] - rowptr[r]);
    cnt[sl] = 32 * w;
}

__global__ void k_sell_fill(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int nv, int nslices,
                            const int32_t* __restrict__ sell_ptr, int32_t* __restrict__ sell_col) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= 32 * nslices) return;
    const int sl = r >> 5;
    const int w = (sell_ptr[sl + 1] - sell_ptr[sl]) / 32;
    const int len = r < nv ? rowptr[r + 1] - rowptr[r] : 0;
    for (int k = 0; k < w; ++k)
        sell_col[sell_ptr[sl] + 32 * k + (r & 31)] = k < len ? col[rowptr[r] + k] : 32 * sl;
}

// Number of triangles shared by vertices a and b (both lists ascending).
__device__ int common_triangles(int a, int b, const int32_t* __restrict__ vt_ptr, const int32_t* __restrict__ vt_list) {
    int i = vt_ptr[a], ie = vt_ptr[a + 1], j = vt_ptr[b], je = vt_ptr[b + 1], n = 0;
    while (i < ie && j < je) {
        int x = vt_list[i], y = vt_list[j];
        if (x == y) { ++n; ++i; ++j; }
        else if (x < y) ++i;
        else ++j;
    }
    return n;
}

// New vertices of the next level: one per edge, at the exact FP64 midpoint.
__global__ void k_new_vertices(const double* __restrict__ xy, const uint8_t* __restrict__ tag,
                               const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const int32_t* __restrict__ ebase, const int32_t* __restrict__ vt_ptr,
                               const int32_t* __restrict__ vt_list, int nv, double* __restrict__ xy_f,
                               uint8_t* __restrict__ tag_f, int32_t* __restrict__ parents) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nv) return;
    xy_f[2 * a] = xy[2 * a];
    xy_f[2 * a + 1] = xy[2 * a + 1];
    tag_f[a] = tag[a];
    int e = ebase[a];
    const double xa = xy[2 * a], ya = xy[2 * a + 1];
    for (int j = rowptr[a]; j < rowptr[a + 1]; ++j) {
        int b = col[j];
        if (b <= a) continue;
        int id = nv + e;
        xy_f[2 * id] = 0.5 * (xa + xy[2 * b]);
        xy_f[2 * id + 1] = 0.5 * (ya + xy[2 * b + 1]);
        parents[2 * e] = a;
        parents[2 * e + 1] = b;
        bool boundary = common_triangles(a, b, vt_ptr, vt_list) == 1;
        tag_f[id] = boundary ? (uint8_t)(tag[a] & tag[b]) : (uint8_t)0;
        ++e;
    }
}

__device__ __forceinline__ int edge_id(int p, int q, const int32_t* __restrict__ rowptr,
                                       const int32_t* __restrict__ col, const int32_t* __restrict__ ebase) {
    int a = p < q ? p : q, b = p < q ? q : p;
    int k = 0;
    for (int j = rowptr[a]; j < rowptr[a + 1]; ++j) {
        int c = col[j];
        if (c > a) {
            if (c == b) return ebase[a] + k;
            ++k;
        }
    }
    return -1;   // unreachable for a valid adjacency
}

__global__ void k_children(const int32_t* __restrict__ tri, int nt, int nv, const int32_t* __restrict__ rowptr,
                           const int32_t* __restrict__ col, const int32_t* __restrict__ ebase,
                           int32_t* __restrict__ tri_f) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
    int mab = nv + edge_id(a, b, rowptr, col, ebase);
    int mbc = nv + edge_id(b, c, rowptr, col, ebase);
    int mca = nv + edge_id(c, a, rowptr, col, ebase);
    int32_t* o = tri_f + 12 * (int64_t)t;
    o[0] = a;   o[1] = mab; o[2] = mca;
    o[3] = mab; o[4] = b;   o[5] = mbc;
    o[6] = mca; o[7] = mbc; o[8] = c;
    o[9] = mab; o[10] = mbc; o[11] = mca;
}

template <class T>
static int dalloc(cgp_mesh* m, T** p, size_t count) {
    void* q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = sizeof(T);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        return CGP_ENOMEM;
    }
    m->allocs.push_back(q);
    *p = (T*)q;
    return CGP_OK;
}

static int read_err(int* d_err, cudaStream_t s, int* h) {
    CGP_CUDA(cudaMemcpyAsync(h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CGP_CUDA(cudaStreamSynchronize(s));
    return CGP_OK;
}

// Incidence lists and adjacency CSR of one level (sizes nv, nt already set, xy/tri/tag filled).
static int build_connectivity(cgp_mesh* m, Level& L, int32_t* cnt, int32_t* tmp, int* d_err, cudaStream_t s) {
    CGP_TRY(dalloc(m, &L.vt_ptr, (size_t)L.nv + 1));
    CGP_TRY(dalloc(m, &L.vt_list, (size_t)3 * L.nt));
    CGP_TRY(dalloc(m, &L.rowptr, (size_t)L.nv + 1));
    CGP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * L.nv, s));
    k_count_incidence<<<blocks_for(L.nt), kBlock, 0, s>>>(L.tri, L.nt, cnt);
    CGP_TRY(exclusive_scan(cnt, L.vt_ptr, L.nv, tmp, s));
    CGP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * L.nv, s));
    k_fill_incidence<<<blocks_for(L.nt), kBlock, 0, s>>>(L.tri, L.nt, L.vt_ptr, cnt, L.vt_list);
    k_sort_incidence<<<blocks_for(L.nv), kBlock, 0, s>>>(L.vt_ptr, L.vt_list, L.nv, d_err);
    k_adj_count<<<blocks_for(L.nv), kBlock, 0, s>>>(L.tri, L.vt_ptr, L.vt_list, L.nv, cnt, d_err);
    CGP_TRY(exclusive_scan(cnt, L.rowptr, L.nv, tmp, s));
    CGP_LAUNCH_CHECK();
    int h_err = 0;
    CGP_TRY(read_err(d_err, s, &h_err));
    if (h_err) {
        set_error("invalid mesh: %s%s", (h_err & 4) ? "a vertex has too many neighbours; " : "",
                  (h_err & 8) ? "a vertex belongs to no triangle" : "");
        return CGP_EINVAL;
    }
    int32_t nnz = 0;
    CGP_CUDA(cudaMemcpyAsync(&nnz, L.rowptr + L.nv, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CGP_CUDA(cudaStreamSynchronize(s));
    L.nnz = nnz;
    CGP_TRY(dalloc(m, &L.col, (size_t)nnz));
    k_adj_fill<<<blocks_for(L.nv), kBlock, 0, s>>>(L.tri, L.vt_ptr, L.vt_list, L.nv, L.rowptr, L.col);
    // SELL-32 view
    L.nslices = (L.nv + kSlice - 1) / kSlice;
    CGP_TRY(dalloc(m, &L.sell_ptr, (size_t)L.nslices + 1));
    k_slice_size<<<blocks_for(L.nslices), kBlock, 0, s>>>(L.rowptr, L.nv, L.nslices, cnt);
    CGP_TRY(exclusive_scan(cnt, L.sell_ptr, L.nslices, tmp, s));
    int32_t nsell = 0;
    CGP_CUDA(cudaMemcpyAsync(&nsell, L.sell_ptr + L.nslices, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CGP_CUDA(cudaStreamSynchronize(s));
    L.nnz_sell = nsell;
    CGP_TRY(dalloc(m, &L.sell_col, (size_t)nsell));
    k_sell_fill<<<blocks_for((int64_t)L.nslices * kSlice), kBlock, 0, s>>>(L.rowptr, L.col, L.nv, L.nslices,
                                                                          L.sell_ptr, L.sell_col);
    CGP_LAUNCH_CHECK();
    return CGP_OK;
}

static int create(const cgp_mesh_desc* d, cudaStream_t s, cgp_mesh* m) {
    if (!d || d->n_vert < 3 || d->n_tri < 1 || !d->xy || !d->tri || !d->vert_tag || d->n_levels < 0 ||
        d->n_levels > 4) {
        set_error("cgp_mesh_create: invalid descriptor");
        return CGP_EINVAL;
    }
    // size bound of the finest level (vertices <= nv + 3 nt per level at most; checked exactly below)
    int64_t nt_f = (int64_t)d->n_tri << (2 * d->n_levels);
    if (nt_f > (int64_t)INT32_MAX / 3) {
        set_error("cgp_mesh_create: %lld triangles on the finest level exceed the index range", (long long)nt_f);
        return CGP_EINVAL;
    }
    CGP_CUDA(cudaGetDevice(&m->device));
    m->n_levels = d->n_levels;
    Level& L0 = m->lev[0];
    L0.nv = d->n_vert;
    L0.nt = d->n_tri;
    CGP_TRY(dalloc(m, &L0.xy, (size_t)2 * L0.nv));
    CGP_TRY(dalloc(m, &L0.tri, (size_t)3 * L0.nt));
    CGP_TRY(dalloc(m, &L0.tag, (size_t)L0.nv));
    CGP_TRY(dalloc(m, &L0.parents, 2));
    CGP_CUDA(cudaMemcpyAsync(L0.xy, d->xy, sizeof(double) * 2 * L0.nv, cudaMemcpyHostToDevice, s));
    CGP_CUDA(cudaMemcpyAsync(L0.tri, d->tri, sizeof(int32_t) * 3 * L0.nt, cudaMemcpyHostToDevice, s));
    CGP_CUDA(cudaMemcpyAsync(L0.tag, d->vert_tag, L0.nv, cudaMemcpyHostToDevice, s));
    // temporaries sized for the finest level (vertex count bounded by nv + 3 nt per refinement)
    int64_t nv_bound = L0.nv;
    for (int l = 0; l < d->n_levels; ++l) nv_bound += 3 * ((int64_t)L0.nt << (2 * l));
    int32_t *cnt = nullptr, *tmp = nullptr, *ebase = nullptr;
    int* d_err = nullptr;
    std::vector<void*> scratch;
    auto tmpalloc = [&](void** p, size_t bytes) -> int {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
            return CGP_ENOMEM;
        }
        scratch.push_back(*p);
        return CGP_OK;
    };
    int rc = CGP_OK;
    do {
        if ((rc = tmpalloc((void**)&cnt, sizeof(int32_t) * (nv_bound + 1))) != CGP_OK) break;
        if ((rc = tmpalloc((void**)&ebase, sizeof(int32_t) * (nv_bound + 1))) != CGP_OK) break;
        if ((rc = tmpalloc((void**)&tmp, sizeof(int32_t) * scan_tmp_ints(nv_bound + 1))) != CGP_OK) break;
        if ((rc = tmpalloc((void**)&d_err, sizeof(int))) != CGP_OK) break;
        if (cudaMemsetAsync(d_err, 0, sizeof(int), s) != cudaSuccess) { rc = CGP_ECUDA; break; }
        k_check_base<<<blocks_for(L0.nt), kBlock, 0, s>>>(L0.xy, L0.tri, L0.nt, L0.nv, d_err);
        int h_err = 0;
        if ((rc = read_err(d_err, s, &h_err)) != CGP_OK) break;
        if (h_err) {
            set_error("invalid base mesh: %s%s", (h_err & 1) ? "bad vertex index in a triangle; " : "",
                      (h_err & 2) ? "a triangle is not counter-clockwise with positive area" : "");
            rc = CGP_EINVAL;
            break;
        }
        for (int l = 0; l <= d->n_levels && rc == CGP_OK; ++l) {
            Level& L = m->lev[l];
            if ((rc = build_connectivity(m, L, cnt, tmp, d_err, s)) != CGP_OK) break;
            if (l == d->n_levels) break;
            k_upper_count<<<blocks_for(L.nv), kBlock, 0, s>>>(L.rowptr, L.col, L.nv, cnt);
            if ((rc = exclusive_scan(cnt, ebase, L.nv, tmp, s)) != CGP_OK) break;
            int32_t ne = 0;
            if (cudaMemcpyAsync(&ne, ebase + L.nv, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) { rc = CGP_ECUDA; set_error("edge count copy failed"); break; }
            Level& F = m->lev[l + 1];
            F.nv = L.nv + ne;
            F.nt = 4 * L.nt;
            if ((rc = dalloc(m, &F.xy, (size_t)2 * F.nv)) != CGP_OK) break;
            if ((rc = dalloc(m, &F.tri, (size_t)3 * F.nt)) != CGP_OK) break;
            if ((rc = dalloc(m, &F.tag, (size_t)F.nv)) != CGP_OK) break;
            if ((rc = dalloc(m, &F.parents, (size_t)2 * ne)) != CGP_OK) break;
            k_new_vertices<<<blocks_for(L.nv), kBlock, 0, s>>>(L.xy, L.tag, L.rowptr, L.col, ebase, L.vt_ptr,
                                                               L.vt_list, L.nv, F.xy, F.tag, F.parents);
            k_children<<<blocks_for(L.nt), kBlock, 0, s>>>(L.tri, L.nt, L.nv, L.rowptr, L.col, ebase, F.tri);
            if (cudaGetLastError() != cudaSuccess) { rc = CGP_ECUDA; set_error("refinement launch failed"); break; }
        }
        if (rc == CGP_OK && cudaStreamSynchronize(s) != cudaSuccess) {
            rc = CGP_ECUDA;
            set_error("mesh construction failed on the device");
        }
    } while (0);
    for (void* p : scratch) cudaFree(p);
    return rc;
}

}  // namespace cgp

using namespace cgp;

extern "C" int cgp_mesh_create(const cgp_mesh_desc* desc, cgp_stream_t stream, cgp_mesh** out) {
    clear_error();
    if (!out) {
        set_error("cgp_mesh_create: out is NULL");
        return CGP_EINVAL;
    }
    *out = nullptr;
    cgp_mesh* m = new cgp_mesh();
    int rc = create(desc, (cudaStream_t)stream, m);
    if (rc != CGP_OK) {
        cgp_mesh_destroy(m);
        return rc;
    }
    *out = m;
    return CGP_OK;
}

extern "C" int cgp_mesh_level_info(const cgp_mesh* m, int32_t level, int32_t* n_vert, int32_t* n_tri,
                                   int64_t* nnz) {
    if (!m || level < 0 || level > m->n_levels) {
        set_error("cgp_mesh_level_info: bad mesh or level");
        return CGP_EINVAL;
    }
    const Level& L = m->lev[level];
    if (n_vert) *n_vert = L.nv;
    if (n_tri) *n_tri = L.nt;
    if (nnz) *nnz = L.nnz;
    return CGP_OK;
}

extern "C" int cgp_mesh_get_level(const cgp_mesh* m, int32_t level, double* xy, int32_t* tri, uint8_t* tag,
                                  int32_t* rowptr, int32_t* col, int32_t* parents) {
    if (!m || level < 0 || level > m->n_levels) {
        set_error("cgp_mesh_get_level: bad mesh or level");
        return CGP_EINVAL;
    }
    const Level& L = m->lev[level];
    if (xy) CGP_CUDA(cudaMemcpy(xy, L.xy, sizeof(double) * 2 * L.nv, cudaMemcpyDeviceToHost));
    if (tri) CGP_CUDA(cudaMemcpy(tri, L.tri, sizeof(int32_t) * 3 * L.nt, cudaMemcpyDeviceToHost));
    if (tag) CGP_CUDA(cudaMemcpy(tag, L.tag, L.nv, cudaMemcpyDeviceToHost));
    if (rowptr) CGP_CUDA(cudaMemcpy(rowptr, L.rowptr, sizeof(int32_t) * (L.nv + 1), cudaMemcpyDeviceToHost));
    if (col) CGP_CUDA(cudaMemcpy(col, L.col, sizeof(int32_t) * L.nnz, cudaMemcpyDeviceToHost));
    if (parents && level > 0) {
        int64_t ne = L.nv - m->lev[level - 1].nv;
        CGP_CUDA(cudaMemcpy(parents, L.parents, sizeof(int32_t) * 2 * ne, cudaMemcpyDeviceToHost));
    }
    return CGP_OK;
}

extern "C" void cgp_mesh_destroy(cgp_mesh* m) {
    if (!m) return;
    for (void* p : m->allocs) cudaFree(p);
    delete m;
}
