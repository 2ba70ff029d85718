// C ABI entry points: argument validation, mesh ingest (node numbering), buffer management.
// The arithmetic of the method lives in the kernels (ts_build.cu, ts_walk.cu, ts_ewald.cu,
// ts_column.cu); this file only prepares their inputs.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cstdlib>
#include <deque>

#include <cuda_fp16.h>

#include "ts_internal.cuh"

static thread_local std::string g_last_error;

ts_status ts_fail(ts_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

ts_status ts_cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? TS_ERR_OUT_OF_MEMORY : TS_ERR_CUDA;
}

extern "C" const char* ts_last_error(void) { return g_last_error.c_str(); }

static thread_local const char* g_fault_site = nullptr;
static thread_local int g_fault_count = 0;

FaultSite::FaultSite(const char* site) : prev_site(g_fault_site), prev_count(g_fault_count) {
    g_fault_site = site;
    g_fault_count = 0;
}

FaultSite::~FaultSite() {
    g_fault_site = prev_site;
    g_fault_count = prev_count;
}

// true if TS_FAULT names the active site and (when it gives :k) this is the site's k-th allocation
static bool fault_hit() {
    const char* f = getenv("TS_FAULT");
    if (!f || !*f || !g_fault_site) return false;
    const int k = ++g_fault_count;
    const char* colon = strchr(f, ':');
    const size_t len = colon ? (size_t)(colon - f) : strlen(f);
    if (len != strlen(g_fault_site) || strncmp(f, g_fault_site, len) != 0) return false;
    return !colon || atoi(colon + 1) == k;
}

cudaError_t ts_malloc(void** p, size_t bytes) {
    if (fault_hit()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

uint64_t ts_fnv1a(const void* data, size_t bytes, uint64_t h) {
    const unsigned char* b = (const unsigned char*)data;
    for (size_t i = 0; i < bytes; ++i) {
        h ^= b[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

cudaError_t ts_malloc_host(void** p, size_t bytes) {
    if (fault_hit()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(p, bytes);
}

extern "C" const char* ts_version(void) { return "treesolver-gb300 0.1 (sm_103a)"; }

template <typename T>
static void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

template <typename T>
static cudaError_t dalloc(T*& p, size_t count) {
    dfree(p);
    return ts_malloc((void**)&p, sizeof(T) * (count ? count : 1));
}

extern "C" ts_status ts_create(ts_ctx** out, int device, void* stream) {
    FaultSite fault_site("create");
    if (!out) return ts_fail(TS_ERR_INVALID_ARG, "ts_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    TS_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return ts_fail(TS_ERR_INVALID_ARG, "ts_create: no such device");
    DeviceGuard g(device);
    ts_ctx* c = new ts_ctx();
    c->device = device;
    cudaError_t e = cudaSuccess;
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        c->own_stream = true;
    }
    if (e == cudaSuccess) e = dalloc(c->d_status, 1);
    if (e == cudaSuccess) e = dalloc(c->d_counters, 4);
    if (e == cudaSuccess) e = dalloc(c->d_reduce, 4);
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_counters, 0, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    if (e != cudaSuccess) {
        ts_destroy(c);
        return ts_cuda_fail(e, "ts_create");
    }
    *out = c;
    return TS_OK;
}

static void free_mesh(ts_ctx* c) {
    dfree(c->d_leaf_nid); dfree(c->d_leaf_lo); dfree(c->d_leaf_size); dfree(c->d_amr_order);
    dfree(c->d_leaf_anc); dfree(c->d_bmom64); dfree(c->d_bmom32);
    free_abu(c);
    c->leaf_anc.clear();
    c->anc_max = 0;
    c->bmom_prec = 0;
    dfree(c->d_ncom32); dfree(c->d_ncen32); dfree(c->d_cell32); dfree(c->d_cellsoa); dfree(c->d_ncomsoa);
    dfree(c->d_ncom64); dfree(c->d_ncen64); dfree(c->d_cell64);
    dfree(c->d_nd_blk); dfree(c->d_nd_leaf);
    c->have_nd = false;
    dfree(c->d_range_counts); dfree(c->d_range_part);
    c->range_counts_valid = false;
    c->range_part_cap = 0;
    dfree(c->d_qcell32); dfree(c->d_qnode32); dfree(c->d_qnode64);
    c->q_n = 0;
    c->have_mesh = c->have_tree = false;
}

static void free_ewald(ts_ctx* c) {
    dfree(c->d_ew32); dfree(c->d_ew64);
    dfree(c->d_tay32); dfree(c->d_tay64);
    c->ew_host.clear();
    c->tay_host.clear();
    c->have_ewald = c->have_taylor = false;
    c->ew.tay32 = nullptr;
    c->ew.tay64 = nullptr;
}

static void free_noderay(ts_ctx* c) {
    dfree(c->d_nr_dense); dfree(c->d_nr_rec); dfree(c->d_nr_more);
    c->have_noderay = false;
}

extern "C" ts_status ts_destroy(ts_ctx* c) {
    if (!c) return TS_OK;
    DeviceGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_mesh(c);
    free_ewald(c);
    free_noderay(c);
    free_mlp(c);
    dfree(c->d_status); dfree(c->d_counters); dfree(c->d_reduce); dfree(c->d_geom);
    dfree(c->d_err); dfree(c->d_err_aux); dfree(c->d_shield_tab);
    if (c->d_sq) cudaFree(c->d_sq);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return TS_OK;
}

// ------------------------------------------------------------------------------ mesh ingest
// Validates the block octree and assigns node ids so that the 8 children of every node are
// contiguous (breadth-first over blocks, then a fixed block-tree layout per leaf-block).
static ts_status ingest_mesh(ts_ctx* c, const ts_mesh* m) {
    const int nb = m->nblocks;
    if (nb < 1 || !m->level || !m->child || !m->lo || !m->size)
        return ts_fail(TS_ERR_INVALID_ARG, "mesh: nblocks < 1 or NULL array");
    for (int a = 0; a < 3; ++a)
        if (m->bc[a] != TS_BC_ISOLATED && m->bc[a] != TS_BC_PERIODIC)
            return ts_fail(TS_ERR_INVALID_ARG, "mesh: bc must be TS_BC_ISOLATED or TS_BC_PERIODIC");
    if (m->level[0] != 1) return ts_fail(TS_ERR_INVALID_ARG, "mesh: block 0 must be the root (level 1)");
    for (int b = 0; b < nb; ++b)
        for (int a = 0; a < 3; ++a)
            if (!(m->size[3 * b + a] > 0) || !isfinite(m->lo[3 * b + a]))
                return ts_fail(TS_ERR_INVALID_ARG, "mesh: block sizes must be positive and finite");
    std::vector<int> parent(nb, -1);
    int nleaf = 0;
    for (int b = 0; b < nb; ++b) {
        const int* ch = m->child + 8 * b;
        int nneg = 0;
        for (int o = 0; o < 8; ++o) nneg += ch[o] < 0;
        if (nneg == 8) { ++nleaf; continue; }
        if (nneg != 0) return ts_fail(TS_ERR_INVALID_ARG, "mesh: a block must have 0 or 8 children");
        for (int o = 0; o < 8; ++o) {
            int cb = ch[o];
            if (cb <= 0 || cb >= nb) return ts_fail(TS_ERR_INVALID_ARG, "mesh: child index out of range");
            if (parent[cb] >= 0) return ts_fail(TS_ERR_INVALID_ARG, "mesh: block with two parents");
            parent[cb] = b;
            if (m->level[cb] != m->level[b] + 1)
                return ts_fail(TS_ERR_INVALID_ARG, "mesh: child level must be parent level + 1");
            int off[3] = {o & 1, (o >> 1) & 1, o >> 2};
            for (int a = 0; a < 3; ++a) {
                double hs = 0.5 * m->size[3 * b + a];
                double elo = m->lo[3 * b + a] + off[a] * hs;
                double tol = 1e-12 * m->size[a];
                if (fabs(m->size[3 * cb + a] - hs) > tol || fabs(m->lo[3 * cb + a] - elo) > tol)
                    return ts_fail(TS_ERR_INVALID_ARG, "mesh: child block not in its parent's octant");
            }
        }
    }
    for (int b = 1; b < nb; ++b)
        if (parent[b] < 0) return ts_fail(TS_ERR_INVALID_ARG, "mesh: block not reachable from the root");
    if ((int64_t)nleaf * TS_NCB > TS_MAX_CELLS)
        return ts_fail(TS_ERR_UNSUPPORTED, "mesh: more than 2^26 cells in one context");

    free_mesh(c);
    c->nb = nb;
    c->nleaf = nleaf;
    c->ncell = (int64_t)nleaf * TS_NCB;
    c->nint = nb + 72 * nleaf;
    for (int a = 0; a < 3; ++a) {
        c->bc[a] = m->bc[a];
        c->L[a] = m->size[a];
        c->dlo[a] = m->lo[a];
    }
    // leaf order = order in the block list
    c->leaf_blk.clear();
    std::vector<int> leaf_of(nb, -1);
    for (int b = 0; b < nb; ++b)
        if (m->child[8 * b] < 0) { leaf_of[b] = (int)c->leaf_blk.size(); c->leaf_blk.push_back(b); }
    // breadth-first node ids for blocks
    c->blk_nid.assign(nb, -1);
    std::vector<int> order;  // blocks in node-id order
    order.reserve(nb);
    c->blk_nid[0] = 0;
    order.push_back(0);
    for (size_t h = 0; h < order.size(); ++h) {
        int b = order[h];
        if (m->child[8 * b] < 0) continue;
        for (int o = 0; o < 8; ++o) {
            int cb = m->child[8 * b + o];
            c->blk_nid[cb] = (int)order.size();
            order.push_back(cb);
        }
    }
    int maxlev = 0;
    for (int b = 0; b < nb; ++b) maxlev = std::max(maxlev, m->level[b]);
    c->depth_max = maxlev - 1 + 3;  // cells of the finest leaf-blocks
    if (c->depth_max > TS_MAX_DEPTH) return ts_fail(TS_ERR_UNSUPPORTED, "mesh: tree deeper than 31 levels");
    // tables of the numerical differentiation (uploaded on first use): per block node id the first
    // child's node id (-1 for a leaf-block) and the leaf index (-1 otherwise); per leaf-block the
    // integer position of its first cell among the 2^d cells per axis of its cells' depth d
    c->nd_blk_host.assign(nb, make_int2(-1, -1));
    for (int b = 0; b < nb; ++b)
        c->nd_blk_host[c->blk_nid[b]] = make_int2(m->child[8 * b] >= 0 ? c->blk_nid[m->child[8 * b]] : -1, leaf_of[b]);
    c->nd_leaf_host.resize(nleaf);
    for (int n = 0; n < nleaf; ++n) {
        const int b = c->leaf_blk[n], d = m->level[b] + 2;
        int q[3];
        for (int a = 0; a < 3; ++a) q[a] = (int)llrint((m->lo[3 * b + a] - m->lo[a]) / m->size[a] * ldexp(1.0, d));
        c->nd_leaf_host[n] = make_int4(q[0], q[1], q[2], d);
    }

    // geometry per depth (all nodes of one depth have equal edges: Sec. 2)
    WalkGeom& G = c->geom;
    memset(&G, 0, sizeof(G));
    for (int d = 0; d <= TS_MAX_DEPTH; ++d) {
        double h2 = 0;
        for (int a = 0; a < 3; ++a) {
            double e = ldexp(m->size[a], -d);
            G.half64[d][a] = 0.5 * e;
            G.half32[d][a] = (float)(0.5 * e);
            h2 = std::max(h2, e * e);
        }
        G.hmax2_64[d] = h2;
        G.hmax2_32[d] = (float)h2;
    }
    for (int a = 0; a < 3; ++a) {
        G.pbc[a] = m->bc[a];
        G.L[a] = m->size[a];
        G.invL[a] = 1.0 / m->size[a];
    }

    // static node records: geometric centres and child words
    const int nint = c->nint;
    std::vector<float4> cen32(nint);
    std::vector<dbl4> cen64(nint);
    auto put = [&](int nid, const double cc[3], uint32_t cw) {
        cen64[nid] = dbl4{cc[0], cc[1], cc[2], (double)cw};
        float4 f;
        f.x = (float)cc[0]; f.y = (float)cc[1]; f.z = (float)cc[2];
        memcpy(&f.w, &cw, 4);
        cen32[nid] = f;
    };
    for (int b = 0; b < nb; ++b) {
        int nid = c->blk_nid[b], dep = m->level[b] - 1;
        double cc[3];
        for (int a = 0; a < 3; ++a) cc[a] = m->lo[3 * b + a] + 0.5 * m->size[3 * b + a];
        uint32_t cw;
        if (m->child[8 * b] >= 0) {
            cw = (uint32_t)c->blk_nid[m->child[8 * b]] | ((uint32_t)(dep + 1) << TS_CW_DEPTH_SHIFT);
        } else {
            int n = leaf_of[b];
            cw = (uint32_t)(nb + 72 * n) | ((uint32_t)(dep + 1) << TS_CW_DEPTH_SHIFT);
            for (int q = 0; q < 8; ++q) {
                int qq[3] = {q & 1, (q >> 1) & 1, q >> 2};
                double c1[3];
                for (int a = 0; a < 3; ++a) c1[a] = m->lo[3 * b + a] + (qq[a] + 0.5) * m->size[3 * b + a] / 2;
                put(nb + 72 * n + q, c1,
                    (uint32_t)(nb + 72 * n + 8 + 8 * q) | ((uint32_t)(dep + 2) << TS_CW_DEPTH_SHIFT));
                for (int o = 0; o < 8; ++o) {
                    int oo[3] = {o & 1, (o >> 1) & 1, o >> 2};
                    double c2[3];
                    for (int a = 0; a < 3; ++a)
                        c2[a] = m->lo[3 * b + a] + (2 * qq[a] + oo[a] + 0.5) * m->size[3 * b + a] / 4;
                    put(nb + 72 * n + 8 + 8 * q + o, c2,
                        (uint32_t)(TS_NCB * n + 64 * q + 8 * o) | TS_CW_CELLS |
                            ((uint32_t)(dep + 3) << TS_CW_DEPTH_SHIFT));
                }
            }
        }
        put(nid, cc, cw);
    }
    c->root_cw = 0;
    memcpy(&c->root_cw, &cen32[0].w, 4);

    // amr reduction order: non-leaf blocks grouped by level, deepest first
    c->amr_order.clear();
    c->amr_level_off.clear();
    for (int lev = maxlev; lev >= 1; --lev) {
        c->amr_level_off.push_back((int)c->amr_order.size());
        for (int b = 0; b < nb; ++b)
            if (m->level[b] == lev && m->child[8 * b] >= 0) c->amr_order.push_back(c->blk_nid[b]);
    }
    c->amr_level_off.push_back((int)c->amr_order.size());

    // amr ancestors of every leaf-block (node ids, nearest first), for the MPE moments
    c->anc_max = 0;
    for (int n = 0; n < nleaf; ++n) {
        int k = 0;
        for (int b = parent[c->leaf_blk[n]]; b >= 0; b = b ? parent[b] : -1) ++k;
        c->anc_max = std::max(c->anc_max, k);
    }
    c->leaf_anc.assign((size_t)nleaf * std::max(1, c->anc_max), -1);
    for (int n = 0; n < nleaf; ++n) {
        int k = 0;
        for (int b = parent[c->leaf_blk[n]]; b >= 0; b = b ? parent[b] : -1)
            c->leaf_anc[(size_t)n * c->anc_max + k++] = c->blk_nid[b];
    }

    std::vector<int> leaf_nid(nleaf);
    std::vector<double> leaf_lo(3 * (size_t)nleaf), leaf_size(3 * (size_t)nleaf);
    for (int n = 0; n < nleaf; ++n) {
        int b = c->leaf_blk[n];
        leaf_nid[n] = c->blk_nid[b];
        for (int a = 0; a < 3; ++a) {
            leaf_lo[3 * n + a] = m->lo[3 * b + a];
            leaf_size[3 * n + a] = m->size[3 * b + a];
        }
    }
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(dalloc(c->d_leaf_nid, nleaf));
    chk(dalloc(c->d_leaf_lo, 3 * (size_t)nleaf));
    chk(dalloc(c->d_leaf_size, 3 * (size_t)nleaf));
    chk(dalloc(c->d_amr_order, c->amr_order.size() + c->amr_level_off.size()));
    chk(dalloc(c->d_ncom32, nint));
    chk(dalloc(c->d_ncen32, nint));
    chk(dalloc(c->d_ncom64, nint));
    chk(dalloc(c->d_ncen64, nint));
    chk(dalloc(c->d_cell32, c->ncell));
    chk(dalloc(c->d_cellsoa, c->ncell));        // ncell / 8 groups of 8 float4
    chk(dalloc(c->d_ncomsoa, nint - 1));        // (nint - 1) / 8 groups (nint = 1 mod 8)
    chk(dalloc(c->d_cell64, c->ncell));
    if (e != cudaSuccess) { free_mesh(c); return ts_cuda_fail(e, "mesh ingest: allocation"); }
    chk(cudaMemcpyAsync(c->d_leaf_nid, leaf_nid.data(), sizeof(int) * nleaf, cudaMemcpyHostToDevice, c->stream));
    chk(cudaMemcpyAsync(c->d_leaf_lo, leaf_lo.data(), sizeof(double) * 3 * nleaf, cudaMemcpyHostToDevice, c->stream));
    chk(cudaMemcpyAsync(c->d_leaf_size, leaf_size.data(), sizeof(double) * 3 * nleaf, cudaMemcpyHostToDevice, c->stream));
    {   // node ids of the non-leaf blocks, then the per-round offsets
        std::vector<int> ord(c->amr_order);
        ord.insert(ord.end(), c->amr_level_off.begin(), c->amr_level_off.end());
        chk(cudaMemcpyAsync(c->d_amr_order, ord.data(), sizeof(int) * ord.size(), cudaMemcpyHostToDevice, c->stream));
        chk(cudaStreamSynchronize(c->stream));
    }
    chk(cudaMemcpyAsync(c->d_ncen32, cen32.data(), sizeof(float4) * nint, cudaMemcpyHostToDevice, c->stream));
    chk(cudaMemcpyAsync(c->d_ncen64, cen64.data(), sizeof(dbl4) * nint, cudaMemcpyHostToDevice, c->stream));
    // host vectors are freed at return: wait for the copies
    chk(cudaStreamSynchronize(c->stream));
    if (e != cudaSuccess) { free_mesh(c); return ts_cuda_fail(e, "mesh ingest: upload"); }
    c->have_mesh = true;
    // a new mesh invalidates BC-dependent tables
    free_ewald(c);
    return TS_OK;
}

extern "C" ts_status ts_tree_build(ts_ctx* c, const ts_mesh* mesh, const double* density) {
    FaultSite fault_site("tree_build");
    if (!c) return ts_fail(TS_ERR_INVALID_ARG, "ts_tree_build: ctx is NULL");
    if (!density) return ts_fail(TS_ERR_INVALID_ARG, "ts_tree_build: density is NULL");
    DeviceGuard g(c->device);
    if (mesh) {
        ts_status s = ingest_mesh(c, mesh);
        if (s != TS_OK) return s;
    } else if (!c->have_mesh) {
        return ts_fail(TS_ERR_NOT_BUILT, "ts_tree_build: no mesh ingested yet (mesh is NULL)");
    }
    cudaError_t e = launch_tree_build(c, density);
    if (e != cudaSuccess) return ts_cuda_fail(e, "tree build kernels");
    c->have_tree = true;
    c->rec64_valid = c->rec64;
    c->bmom_prec = 0;
    c->q_n = 0;   // the extra column quantities belong to the previous densities
    return TS_OK;
}

extern "C" ts_status ts_tree_fp64_records(ts_ctx* c, int32_t enabled) {
    if (!c) return ts_fail(TS_ERR_INVALID_ARG, "ts_tree_fp64_records: ctx is NULL");
    c->rec64 = enabled != 0;
    return TS_OK;
}

// MPE moments of the current tree, computed on first use after each build: from FP32 terms for
// the FP32 walk, from FP64 terms for the FP64 walk (which also serve a later FP32 walk).
ts_status ensure_bmoments(ts_ctx* c, bool fp64) {
    FaultSite fault_site("bmoments");
    if (c->bmom_prec >= (fp64 ? 2 : 1)) return TS_OK;
    if (!c->d_bmom64) {
        cudaError_t e = cudaSuccess;
        auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
        chk(dalloc(c->d_bmom64, c->nint));
        chk(dalloc(c->d_bmom32, c->nint));
        chk(dalloc(c->d_leaf_anc, c->leaf_anc.size()));
        chk(cudaMemcpyAsync(c->d_leaf_anc, c->leaf_anc.data(), sizeof(int) * c->leaf_anc.size(),
                            cudaMemcpyHostToDevice, c->stream));
        chk(cudaStreamSynchronize(c->stream));
        if (e != cudaSuccess) return ts_cuda_fail(e, "MPE moments: allocation");
    }
    TS_CUDA(launch_bmoments(c, fp64));
    c->bmom_prec = fp64 ? 2 : 1;
    return TS_OK;
}

extern "C" ts_status ts_mesh_info(ts_ctx* c, int64_t* ncell, int32_t* nleaf, int32_t* nblocks) {
    if (!c) return ts_fail(TS_ERR_INVALID_ARG, "ts_mesh_info: ctx is NULL");
    if (ncell) *ncell = c->have_mesh ? c->ncell : 0;
    if (nleaf) *nleaf = c->have_mesh ? c->nleaf : 0;
    if (nblocks) *nblocks = c->have_mesh ? c->nb : 0;
    return TS_OK;
}

extern "C" ts_status ts_block_moments(ts_ctx* c, double* mass, double* com) {
    if (!c || !mass || !com) return ts_fail(TS_ERR_INVALID_ARG, "ts_block_moments: NULL argument");
    if (!c->have_tree) return ts_fail(TS_ERR_NOT_BUILT, "ts_block_moments: no tree");
    DeviceGuard g(c->device);
    std::vector<dbl4> h(c->nb);
    TS_CUDA(cudaMemcpyAsync(h.data(), c->d_ncom64, sizeof(dbl4) * c->nb, cudaMemcpyDeviceToHost, c->stream));
    TS_CUDA(cudaStreamSynchronize(c->stream));
    for (int b = 0; b < c->nb; ++b) {
        const dbl4& r = h[c->blk_nid[b]];
        mass[b] = r.w;
        com[3 * b] = r.x; com[3 * b + 1] = r.y; com[3 * b + 2] = r.z;
    }
    return TS_OK;
}

// ------------------------------------------------------------------------------ Ewald field
int ew_kind(const int bc[3]) {
    if (!bc[0] && !bc[1] && !bc[2]) return TS_EW_NONE;
    if (bc[0] && bc[1] && bc[2]) return TS_EW_3P;
    if (bc[0] && bc[1] && !bc[2]) return TS_EW_2P1I;
    if (bc[0] && !bc[1] && !bc[2]) return TS_EW_1P2I;
    return -1;
}

// Cache file of the correction table: this header, then the FP64 table [n^3][4]; body_hash is the
// FNV-1a hash of the table bytes, so that a damaged body is detected and the table regenerated.
struct EwCacheHeader {
    char magic[8];          // "TSEWALD2"
    int32_t kind, n;
    double L[3];
    uint64_t body_hash;
};

extern "C" ts_status ts_ewald_field(ts_ctx* c, int32_t n, const char* cache_path) {
    FaultSite fault_site("ewald_field");
    if (!c) return ts_fail(TS_ERR_INVALID_ARG, "ts_ewald_field: ctx is NULL");
    if (!c->have_mesh) return ts_fail(TS_ERR_NOT_BUILT, "ts_ewald_field: no mesh ingested");
    if (n == 0) n = 64;
    if (n < 8 || n > 256) return ts_fail(TS_ERR_INVALID_ARG, "ts_ewald_field: n_table must be in [8, 256]");
    int kind = ew_kind(c->bc);
    if (kind < 0)
        return ts_fail(TS_ERR_UNSUPPORTED,
                       "ts_ewald_field: periodic axes must be {x,y,z}, {x,y} or {x} (Sec. 2.2.4 convention)");
    if (kind == TS_EW_NONE) return ts_fail(TS_ERR_INVALID_ARG, "ts_ewald_field: mesh has isolated BCs only");
    DeviceGuard g(c->device);
    free_ewald(c);
    EwaldDev& E = c->ew;
    const double Lx = c->L[0], b = c->L[1] / Lx, zeta = M_PI * M_PI / 4.0;  // alpha = 2/Lx
    E.kind = kind;
    E.n = n;
    E.far = kind == TS_EW_2P1I ? 2 * Lx * std::max(1.0, b) : 2 * Lx;
    for (int a = 0; a < 3; ++a) {
        double ext = c->bc[a] ? 0.5 * c->L[a] : c->L[a];
        if (!c->bc[a] && ext > E.far) ext = E.far;
        E.ext[a] = ext;
        E.inv_dx[a] = (n - 1) / ext;
        E.h[a] = ext / (n - 1);
    }
    E.taylor = 0;
    E.far_lx = Lx;
    if (kind == TS_EW_2P1I) {
        E.far_slope = 2 * M_PI / (b * Lx * Lx);
        E.far_const = 2 * sqrt(M_PI * zeta) / (M_PI * b * Lx);
    } else {
        E.far_slope = 0;
        E.far_const = -(0.57721566490153286061 - log(4 * zeta)) / Lx;
    }
    const size_t npts = (size_t)n * n * n;
    c->ew_host.assign(npts * 4, 0.0);
    bool loaded = false;
    if (cache_path) {
        FILE* f = fopen(cache_path, "rb");
        if (f) {
            EwCacheHeader h;
            if (fread(&h, sizeof(h), 1, f) == 1 && !memcmp(h.magic, "TSEWALD2", 8) && h.kind == kind &&
                h.n == n && h.L[0] == c->L[0] && h.L[1] == c->L[1] && h.L[2] == c->L[2] &&
                fread(c->ew_host.data(), sizeof(double), npts * 4, f) == npts * 4 &&
                ts_fnv1a(c->ew_host.data(), sizeof(double) * npts * 4, TS_FNV_INIT) == h.body_hash)
                loaded = true;
            fclose(f);
        }
    }
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(dalloc(c->d_ew64, npts));
    chk(dalloc(c->d_ew32, npts));
    if (e != cudaSuccess) { free_ewald(c); return ts_cuda_fail(e, "ts_ewald_field: allocation"); }
    if (loaded) {
        chk(cudaMemcpyAsync(c->d_ew64, c->ew_host.data(), sizeof(dbl4) * npts, cudaMemcpyHostToDevice, c->stream));
    } else {
        chk(launch_ewald_table(c, n, (double*)c->d_ew64));
        chk(cudaMemcpyAsync(c->ew_host.data(), c->d_ew64, sizeof(dbl4) * npts, cudaMemcpyDeviceToHost, c->stream));
    }
    chk(cudaStreamSynchronize(c->stream));
    if (e != cudaSuccess) { free_ewald(c); return ts_cuda_fail(e, "ts_ewald_field: table generation"); }
    for (size_t i = 0; i < npts * 4; ++i)
        if (!isfinite(c->ew_host[i])) { free_ewald(c); return ts_fail(TS_ERR_NUMERIC, "ts_ewald_field: non-finite table value"); }
    std::vector<float4> t32(npts);
    for (size_t i = 0; i < npts; ++i)
        t32[i] = make_float4((float)c->ew_host[4 * i], (float)c->ew_host[4 * i + 1], (float)c->ew_host[4 * i + 2],
                             (float)c->ew_host[4 * i + 3]);
    chk(cudaMemcpyAsync(c->d_ew32, t32.data(), sizeof(float4) * npts, cudaMemcpyHostToDevice, c->stream));
    chk(cudaStreamSynchronize(c->stream));
    if (e != cudaSuccess) { free_ewald(c); return ts_cuda_fail(e, "ts_ewald_field: upload"); }
    if (cache_path && !loaded) {
        FILE* f = fopen(cache_path, "wb");
        if (f) {
            EwCacheHeader h;
            memcpy(h.magic, "TSEWALD2", 8);
            h.kind = kind; h.n = n;
            for (int a = 0; a < 3; ++a) h.L[a] = c->L[a];
            h.body_hash = ts_fnv1a(c->ew_host.data(), sizeof(double) * npts * 4, TS_FNV_INIT);
            fwrite(&h, sizeof(h), 1, f);
            fwrite(c->ew_host.data(), sizeof(double), npts * 4, f);
            fclose(f);
        }
    }
    E.tab32 = c->d_ew32;
    E.tab64 = c->d_ew64;
    c->have_ewald = true;
    return TS_OK;
}

// Device copies of the numerical-differentiation tables of the current mesh.
ts_status ensure_numdiff(ts_ctx* c) {
    FaultSite fault_site("numdiff");
    if (c->have_nd) return TS_OK;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(dalloc(c->d_nd_blk, c->nd_blk_host.size()));
    chk(dalloc(c->d_nd_leaf, c->nd_leaf_host.size()));
    chk(cudaMemcpyAsync(c->d_nd_blk, c->nd_blk_host.data(), sizeof(int2) * c->nd_blk_host.size(),
                        cudaMemcpyHostToDevice, c->stream));
    chk(cudaMemcpyAsync(c->d_nd_leaf, c->nd_leaf_host.data(), sizeof(int4) * c->nd_leaf_host.size(),
                        cudaMemcpyHostToDevice, c->stream));
    chk(cudaStreamSynchronize(c->stream));
    if (e != cudaSuccess) return ts_cuda_fail(e, "numerical differentiation tables");
    c->have_nd = true;
    return TS_OK;
}

// The first-order Taylor table of the context's correction field (Sec. 2.2.5, approach 2), built
// on first use: FP64 series on the device (central-difference step 1e-5 Lx), FP32-walk records
// derived on the host.  A record of the FP32 walk is 32 bytes, one L1 sector: (C, A_c) in FP32 and
// the six Jacobian entries in FP16 divided by their largest magnitude, which the last word holds
// (the Jacobian term is a correction to the correction: 2^-11 of its largest entry is far below
// the lookup's own first-order error).
ts_status ensure_taylor(ts_ctx* c) {
    FaultSite fault_site("taylor");
    if (c->have_taylor) return TS_OK;
    if (!c->have_ewald) return ts_fail(TS_ERR_NOT_BUILT, "Taylor table: call ts_ewald_field first");
    const int n = c->ew.n;
    const size_t npts = (size_t)n * n * n;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(dalloc(c->d_tay64, 4 * npts));
    chk(dalloc(c->d_tay32, 2 * npts));
    if (e != cudaSuccess) return ts_cuda_fail(e, "Taylor table: allocation");
    std::vector<double> raw(16 * npts);
    chk(launch_ewald_taylor(c, n, 1e-5 * c->L[0], c->d_tay64));
    chk(cudaMemcpyAsync(raw.data(), c->d_tay64, sizeof(double) * raw.size(), cudaMemcpyDeviceToHost, c->stream));
    chk(cudaStreamSynchronize(c->stream));
    if (e != cudaSuccess) return ts_cuda_fail(e, "Taylor table: generation");
    c->tay_host.assign(10 * npts, 0.0);
    std::vector<float4> t32(2 * npts);
    for (size_t i = 0; i < npts; ++i) {
        const double* r = &raw[16 * i];
        for (int k = 0; k < 16; ++k)
            if (!isfinite(r[k])) return ts_fail(TS_ERR_NUMERIC, "Taylor table: non-finite value");
        // records (C, A), (Jxx, Jyy, Jzz, Jxy), (Jxz, Jyz, 0, 0) -> (C, A, Jxx, Jxy, Jxz, Jyy, Jyz, Jzz)
        double* o = &c->tay_host[10 * i];
        o[0] = r[0]; o[1] = r[1]; o[2] = r[2]; o[3] = r[3];
        o[4] = r[4]; o[5] = r[7]; o[6] = r[8]; o[7] = r[5]; o[8] = r[9]; o[9] = r[6];
        // 32-byte record: (C, A_c) in FP32, then (Jxx, Jyy), (Jzz, Jxy), (Jxz, Jyz) as FP16 pairs of
        // J / s and s = max |J| in the last word
        t32[2 * i] = make_float4((float)r[0], (float)r[1], (float)r[2], (float)r[3]);
        double s = 0;
        for (int k = 4; k < 10; ++k) s = std::max(s, fabs(r[k]));
        if (!(s > 0)) s = 1;
        const float sf = (float)s;
        auto h16 = [&](double x) {
            const __half h = __float2half_rn((float)(x / sf));
            unsigned short u;
            memcpy(&u, &h, 2);
            return (uint32_t)u;
        };
        uint4 pk;
        pk.x = h16(r[4]) | (h16(r[5]) << 16);
        pk.y = h16(r[6]) | (h16(r[7]) << 16);
        pk.z = h16(r[8]) | (h16(r[9]) << 16);
        memcpy(&pk.w, &sf, 4);
        memcpy(&t32[2 * i + 1], &pk, 16);
    }
    chk(cudaMemcpyAsync(c->d_tay32, t32.data(), sizeof(float4) * t32.size(), cudaMemcpyHostToDevice, c->stream));
    chk(cudaStreamSynchronize(c->stream));
    if (e != cudaSuccess) return ts_cuda_fail(e, "Taylor table: upload");
    c->ew.tay32 = c->d_tay32;
    c->ew.tay64 = c->d_tay64;
    c->have_taylor = true;
    return TS_OK;
}

extern "C" ts_status ts_ewald_taylor_get(ts_ctx* c, int32_t* n, double* table) {
    if (!c) return ts_fail(TS_ERR_INVALID_ARG, "ts_ewald_taylor_get: ctx is NULL");
    if (!c->have_ewald) return ts_fail(TS_ERR_NOT_BUILT, "ts_ewald_taylor_get: no Ewald table");
    DeviceGuard g(c->device);
    ts_status s = ensure_taylor(c);
    if (s != TS_OK) return s;
    if (n) *n = c->ew.n;
    if (table) memcpy(table, c->tay_host.data(), sizeof(double) * c->tay_host.size());
    return TS_OK;
}

extern "C" ts_status ts_ewald_table_get(ts_ctx* c, int32_t* n, double* extent, double* table) {
    if (!c) return ts_fail(TS_ERR_INVALID_ARG, "ts_ewald_table_get: ctx is NULL");
    if (!c->have_ewald) return ts_fail(TS_ERR_NOT_BUILT, "ts_ewald_table_get: no Ewald table");
    if (n) *n = c->ew.n;
    if (extent) for (int a = 0; a < 3; ++a) extent[a] = c->ew.ext[a];
    if (table) memcpy(table, c->ew_host.data(), sizeof(double) * c->ew_host.size());
    return TS_OK;
}

// ------------------------------------------------------------------------------ gravity
extern "C" void ts_gravity_params_default(ts_gravity_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->mac = TS_MAC_BH;
    p->theta = 0.5;
    p->safe_box = 1.2;
    p->G = 1.0;
    p->precision = TS_PREC_FP32_KAHAN;
    p->ewald = TS_EWALD_TABLE;
}

// Checks of a gravity walk request shared by ts_gravity_walk and ts_gravity_walk_abu.
ts_status validate_gravity(ts_ctx* c, const ts_gravity_params* p) {
    if (!c->have_tree) return ts_fail(TS_ERR_NOT_BUILT, "ts_gravity_walk: call ts_tree_build first");
    if (p->mac != TS_MAC_BH && p->mac != TS_MAC_APE && p->mac != TS_MAC_MPE && p->mac != TS_MAC_SUMSQ)
        return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk: unknown MAC");
    if (p->mac == TS_MAC_SUMSQ) {
        if (p->a_old_dev || !(p->a_lim > 0) || !isfinite(p->a_lim))
            return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk: the SumSquare MAC needs an absolute a_lim > 0");
        if (p->queue_max < 0 || (p->queue_max > 0 && p->queue_max < 9) || p->queue_max > (1 << 20))
            return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk: queue_max must be 0 or in [9, 2^20]");
        if (p->ewald == TS_EWALD_MLP && ew_kind(c->bc) != TS_EW_NONE)
            return ts_fail(TS_ERR_UNSUPPORTED, "ts_gravity_walk: the SumSquare walk uses the table corrections");
    }
    if (p->mac == TS_MAC_BH && !(p->theta > 0)) return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk: theta must be > 0");
    if (p->mac != TS_MAC_BH && !p->a_old_dev && !(p->a_lim > 0))
        return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk: APE/MPE need a_lim > 0 or a_old with eps_rel > 0");
    if (p->mac != TS_MAC_BH && p->a_old_dev && !(p->eps_rel > 0))
        return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk: eps_rel must be > 0 with a_old");
    if (!(p->safe_box >= 0) || !isfinite(p->G)) return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk: bad safe_box or G");
    if (p->precision != TS_PREC_FP64 && p->precision != TS_PREC_FP32_KAHAN)
        return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk: unknown precision");
    if (p->precision == TS_PREC_FP64 && !c->rec64_valid)
        return ts_fail(TS_ERR_NOT_BUILT, "ts_gravity_walk: the tree was built without FP64 records (ts_tree_fp64_records)");
    if (p->ewald != TS_EWALD_TABLE && p->ewald != TS_EWALD_MLP && p->ewald != TS_EWALD_TAYLOR)
        return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk: unknown Ewald mode");
    if (p->accel != TS_ACCEL_DIRECT && p->accel != TS_ACCEL_NUMDIFF)
        return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk: unknown acceleration mode");
    int kind = ew_kind(c->bc);
    if (kind < 0) return ts_fail(TS_ERR_UNSUPPORTED, "ts_gravity_walk: unsupported periodic axes");
    if (kind != TS_EW_NONE && p->ewald == TS_EWALD_MLP && p->mac == TS_MAC_MPE)
        return ts_fail(TS_ERR_UNSUPPORTED, "ts_gravity_walk: the learned correction runs with BH or APE only");
    if (kind != TS_EW_NONE && p->ewald == TS_EWALD_MLP) {
        if (kind != TS_EW_2P1I) return ts_fail(TS_ERR_UNSUPPORTED, "ts_gravity_walk: the learned correction covers 2P1I only");
        if (p->precision != TS_PREC_FP32_KAHAN)
            return ts_fail(TS_ERR_UNSUPPORTED, "ts_gravity_walk: the learned correction runs in FP32 only");
        if (!c->have_mlp) return ts_fail(TS_ERR_NOT_BUILT, "ts_gravity_walk: no surrogate (ts_surrogate_train/set)");
        const double b = c->L[1] / c->L[0];
        if (b < c->mlp_b[0] || b > c->mlp_b[1])
            return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk: box aspect outside the surrogate's range");
    } else if (kind != TS_EW_NONE && !c->have_ewald) {
        return ts_fail(TS_ERR_NOT_BUILT, "ts_gravity_walk: periodic/mixed BCs need ts_ewald_field first");
    }
    return TS_OK;
}

extern "C" ts_status ts_gravity_walk(ts_ctx* c, const ts_gravity_params* p, void* pot, void* acc) {
    FaultSite fault_site("walk");
    if (!c || !p) return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk: NULL ctx or params");
    if (!pot || !acc) return ts_fail(TS_ERR_INVALID_ARG, "ts_gravity_walk: NULL output");
    ts_status vs = validate_gravity(c, p);
    if (vs != TS_OK) return vs;
    const int kind = ew_kind(c->bc);
    DeviceGuard g(c->device);
    if (kind != TS_EW_NONE && p->ewald == TS_EWALD_TAYLOR) {
        ts_status s = ensure_taylor(c);
        if (s != TS_OK) return s;
    }
    if (p->mac == TS_MAC_MPE || p->mac == TS_MAC_SUMSQ) {
        ts_status s = ensure_bmoments(c, p->precision == TS_PREC_FP64);
        if (s != TS_OK) return s;
    }
    if (p->accel == TS_ACCEL_NUMDIFF) {
        ts_status s = ensure_numdiff(c);
        if (s != TS_OK) return s;
    }
    cudaError_t e = launch_gravity_walk(c, p, pot, acc);
    if (e == cudaSuccess && p->zero_mean) e = launch_zero_mean(c, p->precision, pot);
    if (e != cudaSuccess) return ts_cuda_fail(e, "gravity walk kernels");
    return TS_OK;
}

// ------------------------------------------------------------------------------ columns
extern "C" void ts_column_params_default(ts_column_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->n_side = 2;
    p->theta = 0.5;
    p->safe_box = 1.2;
    p->max_dist = 0;
}

ts_status ensure_noderay(ts_ctx* c, int nside, const int dims[3], double pmin, double pmax, int nsub) {
    FaultSite fault_site("noderay");
    if (c->have_noderay && c->nr_nside == nside && c->nr_dims[0] == dims[0] && c->nr_dims[1] == dims[1] &&
        c->nr_dims[2] == dims[2] && c->nr_psi[0] == pmin && c->nr_psi[1] == pmax && c->nr_nsub == nsub)
        return TS_OK;
    free_noderay(c);
    const int npix = 12 * nside * nside;
    const size_t nent = (size_t)dims[0] * dims[1] * dims[2];
    TS_CUDA(dalloc(c->d_nr_dense, nent * npix));
    TS_CUDA(launch_noderay_dense(c, nside, dims, pmin, pmax, nsub, c->d_nr_dense));
    std::vector<double> dense(nent * npix);
    TS_CUDA(cudaMemcpyAsync(dense.data(), c->d_nr_dense, sizeof(double) * dense.size(), cudaMemcpyDeviceToHost, c->stream));
    TS_CUDA(cudaStreamSynchronize(c->stream));
    // one 16-byte record of up to 4 (sub-cube count << 8 | pixel) pairs per entry; the weights are
    // counts over nsub^3 (the table kernel counts sub-cube centres per pixel), so counts are exact;
    // a longer row keeps 3 pairs and (offset << 8 | 255) into the continuation array
    const double n3 = (double)nsub * nsub * nsub;
    std::vector<uint32_t> rec(nent * 4, 0u), more;
    std::vector<uint32_t> row;
    for (size_t e = 0; e < nent; ++e) {
        row.clear();
        for (int i = 0; i < npix; ++i) {
            const double v = dense[e * npix + i];
            if (v > 0) {
                const long long k = llrint(v * n3);
                if (fabs(k - v * n3) > 1e-6 * n3 || k < 1 || k >= (1ll << 24))
                    return ts_fail(TS_ERR_NUMERIC, "node-ray table: weight is not a sub-cube count");
                row.push_back(((uint32_t)k << 8) | (uint32_t)i);
            }
        }
        if (row.empty()) return ts_fail(TS_ERR_NUMERIC, "node-ray table: an entry with no pixel");
        if (row.size() <= 4) {
            for (size_t k = 0; k < row.size(); ++k) rec[4 * e + k] = row[k];
        } else {
            for (int k = 0; k < 3; ++k) rec[4 * e + k] = row[k];
            if (more.size() >= (1u << 24)) return ts_fail(TS_ERR_UNSUPPORTED, "node-ray table: rows too long");
            rec[4 * e + 3] = ((uint32_t)more.size() << 8) | 255u;
            more.push_back((uint32_t)(row.size() - 3));
            more.insert(more.end(), row.begin() + 3, row.end());
        }
    }
    if (more.empty()) more.push_back(0u);
    TS_CUDA(dalloc(c->d_nr_rec, nent));
    TS_CUDA(dalloc(c->d_nr_more, more.size()));
    TS_CUDA(cudaMemcpyAsync(c->d_nr_rec, rec.data(), sizeof(uint32_t) * rec.size(), cudaMemcpyHostToDevice, c->stream));
    TS_CUDA(cudaMemcpyAsync(c->d_nr_more, more.data(), sizeof(uint32_t) * more.size(), cudaMemcpyHostToDevice,
                            c->stream));
    TS_CUDA(cudaStreamSynchronize(c->stream));
    const int kmax = (int)more.size();
    c->nr_nside = nside;
    for (int a = 0; a < 3; ++a) c->nr_dims[a] = dims[a];
    c->nr_dims[3] = npix;
    c->nr_psi[0] = pmin;
    c->nr_psi[1] = pmax;
    c->nr_nsub = nsub;
    c->nr_kmax = kmax;
    c->have_noderay = true;
    return TS_OK;
}

// Node-ray table parameters with defaults (tr_ilNTheta, tr_ilNPhi, tr_ilNNS of App. B).
ts_status column_table_params(const ts_column_params* p, int dims[3], double* pmin, double* pmax, int* nsub) {
    dims[0] = p->table_ntheta ? p->table_ntheta : 25;
    dims[1] = p->table_nphi ? p->table_nphi : 50;
    dims[2] = p->table_npsi ? p->table_npsi : 25;
    *pmin = p->table_psi_min > 0 ? p->table_psi_min : 1e-3;
    *pmax = p->table_psi_max > 0 ? p->table_psi_max : 1.0;
    *nsub = p->table_nsub ? p->table_nsub : 8;
    if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1 || dims[0] * dims[1] * dims[2] > (1 << 22) || !(*pmax > *pmin) ||
        *nsub < 1 || *nsub > 64)
        return ts_fail(TS_ERR_INVALID_ARG, "column walk: bad node-ray table parameters");
    return TS_OK;
}

extern "C" ts_status ts_column_walk(ts_ctx* c, const ts_column_params* p, float* cols) {
    FaultSite fault_site("column");
    if (!c || !p || !cols) return ts_fail(TS_ERR_INVALID_ARG, "ts_column_walk: NULL argument");
    if (!c->have_tree) return ts_fail(TS_ERR_NOT_BUILT, "ts_column_walk: call ts_tree_build first");
    if (p->n_side < 1 || p->n_side > 4)
        return ts_fail(TS_ERR_INVALID_ARG, "ts_column_walk: n_side must be in [1, 4] (N_PIX <= 192)");
    if (!(p->theta > 0) || !(p->safe_box >= 0)) return ts_fail(TS_ERR_INVALID_ARG, "ts_column_walk: bad theta/safe_box");
    int dims[3], nsub;
    double pmin, pmax;
    ts_status s0 = column_table_params(p, dims, &pmin, &pmax, &nsub);
    if (s0 != TS_OK) return s0;
    const int npix = 12 * p->n_side * p->n_side;
    if ((1 + c->q_n) * npix > 432)
        return ts_fail(TS_ERR_UNSUPPORTED, "ts_column_walk: l_q * N_PIX must be <= 432 (the maps live in shared memory)");
    DeviceGuard g(c->device);
    ts_status s = ensure_noderay(c, p->n_side, dims, pmin, pmax, nsub);
    if (s != TS_OK) return s;
    cudaError_t e = launch_column_walk(c, p, cols);
    if (e != cudaSuccess) return ts_cuda_fail(e, "column walk kernel");
    return TS_OK;
}

extern "C" ts_status ts_column_quantities(ts_ctx* c, int32_t nq, const double* q) {
    FaultSite fault_site("column");
    if (!c) return ts_fail(TS_ERR_INVALID_ARG, "ts_column_quantities: ctx is NULL");
    if (nq < 0 || nq > 2) return ts_fail(TS_ERR_INVALID_ARG, "ts_column_quantities: nq must be 0, 1 or 2");
    if (nq > 0 && !q) return ts_fail(TS_ERR_INVALID_ARG, "ts_column_quantities: NULL quantity densities");
    if (!c->have_tree) return ts_fail(TS_ERR_NOT_BUILT, "ts_column_quantities: call ts_tree_build first");
    c->q_n = 0;
    if (nq == 0) return TS_OK;
    DeviceGuard g(c->device);
    cudaError_t e = cudaSuccess;
    if (!c->d_qcell32) e = ts_malloc((void**)&c->d_qcell32, sizeof(float2) * c->ncell);
    if (e == cudaSuccess && !c->d_qnode32) e = ts_malloc((void**)&c->d_qnode32, sizeof(float2) * c->nint);
    if (e == cudaSuccess && !c->d_qnode64) e = ts_malloc((void**)&c->d_qnode64, sizeof(double2) * c->nint);
    if (e == cudaSuccess) e = launch_qsums(c, nq, q);
    if (e != cudaSuccess) return ts_cuda_fail(e, "ts_column_quantities");
    c->q_n = nq;
    return TS_OK;
}

extern "C" ts_status ts_column_shielding(ts_ctx* c, int64_t n, int32_t npix, const float* cols, const ts_shield_params* p,
                                         float* out) {
    FaultSite fault_site("column");
    if (!c || !p) return ts_fail(TS_ERR_INVALID_ARG, "ts_column_shielding: NULL ctx or params");
    if (n < 0 || npix < 1) return ts_fail(TS_ERR_INVALID_ARG, "ts_column_shielding: need n >= 0 and npix >= 1");
    if (n > 0 && (!cols || !out)) return ts_fail(TS_ERR_INVALID_ARG, "ts_column_shielding: NULL column maps or output");
    if (!(p->k_av >= 0) || !isfinite(p->k_av) || !(p->k_h2 >= 0) || !isfinite(p->k_h2) || !(p->b5 > 0) ||
        !isfinite(p->b5) || !(p->k_co >= 0) || !isfinite(p->k_co))
        return ts_fail(TS_ERR_INVALID_ARG, "ts_column_shielding: k_av, k_h2, k_co must be finite and >= 0, b5 > 0");
    const bool tab = p->co_n_co != 0 || p->co_n_h2 != 0;
    if (tab && (p->co_n_co < 2 || p->co_n_h2 < 2 || !p->co_table || !(p->co_lg_co[1] > p->co_lg_co[0]) ||
                !(p->co_lg_h2[1] > p->co_lg_h2[0])))
        return ts_fail(TS_ERR_INVALID_ARG, "ts_column_shielding: CO table needs >= 2 points per axis and increasing ranges");
    DeviceGuard g(c->device);
    const float* d_tab = nullptr;
    if (tab) {
        const size_t nt = (size_t)p->co_n_co * p->co_n_h2;
        std::vector<float> h(nt);
        for (size_t i = 0; i < nt; ++i) {
            if (!isfinite(p->co_table[i])) return ts_fail(TS_ERR_INVALID_ARG, "ts_column_shielding: non-finite CO table");
            h[i] = (float)p->co_table[i];
        }
        if (c->shield_cap < nt) {
            dfree(c->d_shield_tab);
            c->shield_cap = 0;
            TS_CUDA(dalloc(c->d_shield_tab, nt));
            c->shield_cap = nt;
        }
        TS_CUDA(cudaMemcpyAsync(c->d_shield_tab, h.data(), sizeof(float) * nt, cudaMemcpyHostToDevice, c->stream));
        TS_CUDA(cudaStreamSynchronize(c->stream));   // h is freed at return
        d_tab = c->d_shield_tab;
    }
    cudaError_t e = launch_shielding(c, n, npix, cols, p, d_tab, out);
    if (e != cudaSuccess) return ts_cuda_fail(e, "shielding kernel");
    return TS_OK;
}

extern "C" ts_status ts_column_av(ts_ctx* c, int64_t n, int32_t npix, const float* cols, double k, float* av) {
    if (!c) return ts_fail(TS_ERR_INVALID_ARG, "ts_column_av: ctx is NULL");
    if (n < 0 || npix < 1) return ts_fail(TS_ERR_INVALID_ARG, "ts_column_av: need n >= 0 and npix >= 1");
    if (!(k >= 0) || !isfinite(k)) return ts_fail(TS_ERR_INVALID_ARG, "ts_column_av: k must be finite and >= 0");
    if (n > 0 && (!cols || !av)) return ts_fail(TS_ERR_INVALID_ARG, "ts_column_av: NULL column map or output");
    DeviceGuard g(c->device);
    cudaError_t e = launch_column_av(c, n, npix, cols, k, av);
    if (e != cudaSuccess) return ts_cuda_fail(e, "column extinction kernel");
    return TS_OK;
}

extern "C" ts_status ts_noderay_table_get(ts_ctx* c, int32_t* dims4, double* table) {
    if (!c) return ts_fail(TS_ERR_INVALID_ARG, "ts_noderay_table_get: ctx is NULL");
    if (!c->have_noderay) return ts_fail(TS_ERR_NOT_BUILT, "ts_noderay_table_get: no table yet");
    if (dims4) for (int a = 0; a < 4; ++a) dims4[a] = c->nr_dims[a];
    if (table) {
        DeviceGuard g(c->device);
        size_t n = (size_t)c->nr_dims[0] * c->nr_dims[1] * c->nr_dims[2] * c->nr_dims[3];
        TS_CUDA(cudaMemcpyAsync(table, c->d_nr_dense, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
        TS_CUDA(cudaStreamSynchronize(c->stream));
    }
    return TS_OK;
}

// ------------------------------------------------------------------------------ sync / stats
extern "C" ts_status ts_sync(ts_ctx* c) {
    if (!c) return ts_fail(TS_ERR_INVALID_ARG, "ts_sync: ctx is NULL");
    DeviceGuard g(c->device);
    TS_CUDA(cudaStreamSynchronize(c->stream));
    int st = 0;
    TS_CUDA(cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) {
        TS_CUDA(cudaMemset(c->d_status, 0, sizeof(int)));
        if (st & TS_DEV_STACK_OVERFLOW) return ts_fail(TS_ERR_STACK_OVERFLOW, "walk stack overflow (tree too deep)");
        if (st & TS_DEV_NONFINITE) return ts_fail(TS_ERR_NUMERIC, "non-finite output");
        return ts_fail(TS_ERR_CUDA, "unknown device status");
    }
    return TS_OK;
}

extern "C" ts_status ts_stats(ts_ctx* c, int64_t* interactions, int64_t* mac_tests, double* last_ms) {
    if (!c) return ts_fail(TS_ERR_INVALID_ARG, "ts_stats: ctx is NULL");
    DeviceGuard g(c->device);
    unsigned long long h[2] = {0, 0};
    TS_CUDA(cudaStreamSynchronize(c->stream));
    TS_CUDA(cudaMemcpy(h, c->d_counters, sizeof(h), cudaMemcpyDeviceToHost));
    if (interactions) *interactions = (int64_t)h[0];
    if (mac_tests) *mac_tests = (int64_t)h[1];
    if (last_ms) {
        float ms = 0;
        if (c->timed) TS_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        *last_ms = ms;
    }
    return TS_OK;
}

extern "C" ts_status ts_walk_counters(ts_ctx* c, int64_t* out) {
    if (!c || !out) return ts_fail(TS_ERR_INVALID_ARG, "ts_walk_counters: NULL argument");
    DeviceGuard g(c->device);
    unsigned long long h[4] = {0, 0, 0, 0};
    TS_CUDA(cudaStreamSynchronize(c->stream));
    TS_CUDA(cudaMemcpy(h, c->d_counters, sizeof(h), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 4; ++i) out[i] = (int64_t)h[i];
    return TS_OK;
}

extern "C" ts_status ts_set_walk_grouping(ts_ctx* c, int32_t precision, int32_t tpl) {
    if (!c) return ts_fail(TS_ERR_INVALID_ARG, "ts_set_walk_grouping: ctx is NULL");
    if (precision != TS_PREC_FP64 && precision != TS_PREC_FP32_KAHAN)
        return ts_fail(TS_ERR_INVALID_ARG, "ts_set_walk_grouping: unknown precision");
    if (tpl != 1 && tpl != 2 && tpl != 4)
        return ts_fail(TS_ERR_INVALID_ARG, "ts_set_walk_grouping: targets_per_lane must be 1, 2 or 4");
    c->walk_T[precision == TS_PREC_FP64 ? 1 : 0] = tpl;
    return TS_OK;
}
