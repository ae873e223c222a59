// C ABI entry points (include/pgcp.h): argument checks, mesh upload and
// concatenation, stage orchestration and timing.  Every entry point catches
// the library's internal errors and returns a status code.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <exception>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "pgcp_internal.h"

namespace pgcp {

struct Thrown : std::exception {
    pgcp_status code;
    std::string msg;
    Thrown(pgcp_status c, std::string m) : code(c), msg(std::move(m)) {}
    const char* what() const noexcept override { return msg.c_str(); }
};

void fail(pgcp_status code, const std::string& msg) { throw Thrown(code, msg); }

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
static std::atomic<long long> g_allocs{0};
void note_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }

void check_cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    if (e == cudaErrorMemoryAllocation) fail(PGCP_E_OOM, std::string(what) + ": out of device memory");
    fail(PGCP_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {

template <typename F>
pgcp_status guard(pgcp_ctx* ctx, F&& f) {
    try {
        f();
        if (ctx) ctx->last_error.clear();
        return PGCP_OK;
    } catch (const Thrown& t) {
        if (ctx) ctx->last_error = t.msg;
        return t.code;
    } catch (const std::bad_alloc&) {
        if (ctx) ctx->last_error = "host allocation failed";
        return PGCP_E_OOM;
    } catch (const std::exception& e) {
        if (ctx) ctx->last_error = e.what();
        return PGCP_E_ARG;
    }
}

template <typename T>
void copy_in(DBuf<T>& dst, size_t off, const T* src, size_t n, int host, cudaStream_t s) {
    if (!n) return;
    if (!src) fail(PGCP_E_ARG, "null input pointer");
    PGCP_CUDA(cudaMemcpyAsync(dst.p + off, src, n * sizeof(T), host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                              s));
}

__global__ void k_offset_faces(int32_t* F, int64_t n, int32_t off, int64_t nv_mesh, uint32_t* err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t v = F[i];
    if (v < 0 || v >= nv_mesh) atomicOr(err, 1u << 31);
    F[i] = v + off;
}

struct Timer {
    cudaEvent_t a, b;
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
    double stop() {
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

void partition_impl(pgcp_ctx* ctx, int32_t n_mesh, const double* const* V, const int64_t* nv,
                    const int32_t* const* F, const int64_t* nf, const int32_t* const* labels,
                    const int32_t* cut, int64_t n_cut, int32_t host, int32_t closed, pgcp_part** out) {
    if (!ctx || !out || n_mesh <= 0) fail(PGCP_E_ARG, "null context/output or no mesh");
    cudaStream_t s = ctx->stream;
    std::unique_ptr<pgcp_part> part(new pgcp_part());
    Part& P = part->p;
    P.closed = closed ? 1 : 0;
    int64_t NV = 0, NF = 0;
    bool have_labels = labels && labels[0];
    for (int b = 0; b < n_mesh; ++b) {
        if (nv[b] <= 0 || nf[b] <= 0) fail(PGCP_E_ARG, "empty mesh");
        if (have_labels != (labels && labels[b] != nullptr)) fail(PGCP_E_ARG, "face labels for some meshes only");
        P.meshes.push_back(MeshInfo{NV, nv[b], NF, nf[b], 0, 0});
        NV += nv[b];
        NF += nf[b];
    }
    if (NV >= (1ll << 31) - 1 || NF >= (1ll << 30)) fail(PGCP_E_ARG, "mesh too large");
    P.nv = NV;
    P.nf = NF;
    P.V.alloc(3 * NV, s);
    P.F.alloc(3 * NF, s);
    DBuf<int32_t> d_labels, d_cut;
    if (have_labels) d_labels.alloc(NF, s);
    ctx->err.zero();
    for (int b = 0; b < n_mesh; ++b) {
        const MeshInfo& M = P.meshes[b];
        copy_in(P.V, 3 * M.v0, V[b], 3 * M.nv, host, s);
        copy_in(P.F, 3 * M.f0, F[b], 3 * M.nf, host, s);
        { k_offset_faces<<<(unsigned)ceil_div(3 * M.nf, 256), 256, 0, s>>>(P.F.p + 3 * M.f0, 3 * M.nf, (int32_t)M.v0,
                                                                        M.nv, ctx->err.p); ::pgcp::note_launch(); }
        if (have_labels) copy_in(d_labels, M.f0, labels[b], M.nf, host, s);
    }
    if (!have_labels && cut && n_cut > 0) {
        if (n_mesh != 1) fail(PGCP_E_ARG, "cut-edge lists are for single meshes; use face labels in a batch");
        d_cut.alloc(2 * n_cut, s);
        copy_in(d_cut, 0, cut, 2 * n_cut, host, s);
    }
    PGCP_CUDA(cudaGetLastError());
    if (read_errors(ctx) & (1u << 31)) fail(PGCP_E_ARG, "face index out of range");
    build_partition(ctx, P, have_labels ? d_labels.p : nullptr, d_cut.p, n_cut);
    // pieces of mesh b start at the label of its first face (labels rank the
    // smallest face of each piece, and mesh b's faces follow mesh b-1's)
    for (int b = 0; b < n_mesh; ++b) {
        int32_t l = 0;
        PGCP_CUDA(cudaMemcpyAsync(&l, P.face_label.p + P.meshes[b].f0, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PGCP_CUDA(cudaStreamSynchronize(s));
        P.meshes[b].piece0 = l;
    }
    for (int b = 0; b < n_mesh; ++b)
        P.meshes[b].npiece = (b + 1 < n_mesh ? P.meshes[b + 1].piece0 : P.K) - P.meshes[b].piece0;
    build_schedule(ctx, P);
    P.stats.K = P.K;
    P.stats.n_welds = (int32_t)P.welds.size();
    P.stats.n_copies = P.Nc;
    *out = part.release();
}

}  // namespace
}  // namespace pgcp

using namespace pgcp;

extern "C" {

void pgcp_default_options(pgcp_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->variant = PGCP_DISK;
    o->precision = PGCP_FP32_REFINED;
    o->tol = 1e-10;
    o->max_iters = 200000;
    o->max_refine = 8;
    o->inner_tol = 1e-4;
    o->warm_start = PGCP_WARM_WELDMAP;
    o->interior_map_fp64 = 0;
    o->block_rows_log2 = 0;
    o->local_precision = PGCP_DF64_REFINED;
}

const char* pgcp_status_string(pgcp_status s) {
    switch (s) {
        case PGCP_OK: return "ok";
        case PGCP_E_ARG: return "bad argument";
        case PGCP_E_CUDA: return "CUDA error";
        case PGCP_E_OOM: return "out of memory";
        case PGCP_E_NONMANIFOLD: return "non-manifold mesh";
        case PGCP_E_TOPOLOGY: return "piece is not a topological disk";
        case PGCP_E_SCHEDULE: return "no valid welding order";
        case PGCP_E_DEGENERATE: return "degenerate face";
        case PGCP_E_NO_CONVERGENCE: return "no convergence";
        case PGCP_E_NUMERIC: return "numeric error";
    }
    return "unknown status";
}

pgcp_status pgcp_create(pgcp_ctx** out, const pgcp_options* opt, void* stream) {
    if (!out) return PGCP_E_ARG;
    *out = nullptr;
    pgcp_ctx* c = new (std::nothrow) pgcp_ctx();
    if (!c) return PGCP_E_OOM;
    pgcp_status st = guard(c, [&] {
        if (opt) c->opt = *opt;
        else pgcp_default_options(&c->opt);
        c->stream = (cudaStream_t)stream;
        PGCP_CUDA(cudaGetDevice(&c->device));
        PGCP_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
        int coop = 0;
        PGCP_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device));
        if (!coop) fail(PGCP_E_CUDA, "device does not support cooperative launches");
        // keep freed blocks in the stream-ordered pool between calls
        cudaMemPool_t pool;
        PGCP_CUDA(cudaDeviceGetDefaultMemPool(&pool, c->device));
        uint64_t thr = UINT64_MAX;
        PGCP_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        c->err.alloc(1, c->stream);
        c->err.zero();
    });
    if (st != PGCP_OK) {
        delete c;
        return st;
    }
    *out = c;
    return PGCP_OK;
}

pgcp_status pgcp_destroy(pgcp_ctx* ctx) {
    if (!ctx) return PGCP_E_ARG;
    cudaStreamSynchronize(ctx->stream);
    delete ctx;
    return PGCP_OK;
}

pgcp_status pgcp_set_options(pgcp_ctx* ctx, const pgcp_options* opt) {
    if (!ctx || !opt) return PGCP_E_ARG;
    ctx->opt = *opt;
    return PGCP_OK;
}

int64_t pgcp_launch_count(void) { return (int64_t)g_launches.load(); }
int64_t pgcp_alloc_count(void) { return (int64_t)g_allocs.load(); }

const char* pgcp_last_error(const pgcp_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

pgcp_status pgcp_partition(pgcp_ctx* ctx, const double* V, int64_t nv, const int32_t* F, int64_t nf,
                           const int32_t* cut_edges, int64_t n_cut, const int32_t* face_labels, int32_t host_ptrs,
                           int32_t closed, pgcp_part** out) {
    return guard(ctx, [&] {
        if (!V || !F) fail(PGCP_E_ARG, "null mesh pointer");
        if (n_cut < 0) fail(PGCP_E_ARG, "negative cut-edge count");
        const double* Vs[1] = {V};
        const int32_t* Fs[1] = {F};
        const int32_t* Ls[1] = {face_labels};
        Timer t(ctx->stream);
        partition_impl(ctx, 1, Vs, &nv, Fs, &nf, Ls, cut_edges, n_cut, host_ptrs, closed, out);
        (*out)->p.stats.ms_partition = t.stop();
    });
}

pgcp_status pgcp_partition_batch(pgcp_ctx* ctx, int32_t n_mesh, const double* const* V, const int64_t* nv,
                                 const int32_t* const* F, const int64_t* nf, const int32_t* const* face_labels,
                                 int32_t host_ptrs, int32_t closed, pgcp_part** out) {
    return guard(ctx, [&] {
        if (!V || !nv || !F || !nf) fail(PGCP_E_ARG, "null batch arrays");
        Timer t(ctx->stream);
        partition_impl(ctx, n_mesh, V, nv, F, nf, face_labels, nullptr, 0, host_ptrs, closed, out);
        (*out)->p.stats.ms_partition = t.stop();
    });
}

pgcp_status pgcp_part_free(pgcp_part* part) {
    if (!part) return PGCP_E_ARG;
    delete part;
    return PGCP_OK;
}

pgcp_status pgcp_part_get_stats(const pgcp_part* part, pgcp_stats* st) {
    if (!part || !st) return PGCP_E_ARG;
    *st = part->p.stats;
    return PGCP_OK;
}

pgcp_status pgcp_part_info(const pgcp_part* part, int32_t* K, int64_t* n_copies, int64_t* nnz, int64_t* n_loop,
                           int32_t* n_welds, int32_t* n_mesh) {
    if (!part) return PGCP_E_ARG;
    const Part& P = part->p;
    if (K) *K = P.K;
    if (n_copies) *n_copies = P.Nc;
    if (nnz) *nnz = P.nnz;
    if (n_loop) *n_loop = (int64_t)P.loop_rows.size();
    if (n_welds) *n_welds = (int32_t)P.welds.size();
    if (n_mesh) *n_mesh = (int32_t)P.meshes.size();
    return PGCP_OK;
}

pgcp_status pgcp_part_get_partition(pgcp_ctx* ctx, const pgcp_part* part, int32_t* face_label, int64_t* piece_voff,
                                    int32_t* piece_verts, int64_t* loop_off, int32_t* loop_verts) {
    return guard(ctx, [&] {
        if (!part) fail(PGCP_E_ARG, "null part");
        const Part& P = part->p;
        cudaStream_t s = ctx->stream;
        if (face_label)
            PGCP_CUDA(cudaMemcpyAsync(face_label, P.face_label.p, P.nf * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        if (piece_voff)
            PGCP_CUDA(cudaMemcpyAsync(piece_voff, P.voff.data(), (P.K + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        if (piece_verts)
            PGCP_CUDA(cudaMemcpyAsync(piece_verts, P.copy_vert.p, P.Nc * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        if (loop_off)
            PGCP_CUDA(cudaMemcpyAsync(loop_off, P.loff.data(), (P.K + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        if (loop_verts)
            PGCP_CUDA(cudaMemcpyAsync(loop_verts, P.loop_glob.data(), P.loop_glob.size() * sizeof(int32_t),
                                      cudaMemcpyHostToDevice, s));
        PGCP_CUDA(cudaStreamSynchronize(s));
    });
}

pgcp_status pgcp_local_param(pgcp_ctx* ctx, pgcp_part* part) {
    return guard(ctx, [&] {
        if (!part) fail(PGCP_E_ARG, "null part");
        Part& P = part->p;
        {
            Timer t(ctx->stream);
            assemble_laplacian(ctx, P);
            P.stats.ms_assembly = t.stop();
            P.stats.nnz = P.nnz;
        }
        Timer t(ctx->stream);
        solve_dncp(ctx, P);
        P.stats.ms_local = t.stop();
    });
}

pgcp_status pgcp_part_get_csr(pgcp_ctx* ctx, const pgcp_part* part, int64_t* row_ptr, int32_t* col, double* val) {
    return guard(ctx, [&] {
        if (!part) fail(PGCP_E_ARG, "null part");
        const Part& P = part->p;
        if (!P.nnz) fail(PGCP_E_ARG, "Laplacians not assembled (call pgcp_local_param)");
        cudaStream_t s = ctx->stream;
        // piece-local columns and int64 row pointers
        std::vector<int32_t> rp(P.Nc + 1), c(P.nnz), rpiece(P.Nc);
        PGCP_CUDA(cudaMemcpyAsync(rp.data(), P.row_ptr.p, (P.Nc + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PGCP_CUDA(cudaMemcpyAsync(c.data(), P.col.p, P.nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PGCP_CUDA(cudaMemcpyAsync(rpiece.data(), P.row_piece.p, P.Nc * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PGCP_CUDA(cudaStreamSynchronize(s));
        std::vector<int64_t> rp64(P.Nc + 1);
        for (int64_t i = 0; i <= P.Nc; ++i) rp64[i] = rp[i];
        for (int64_t i = 0; i < P.Nc; ++i)
            for (int32_t j = rp[i]; j < rp[i + 1]; ++j) c[j] -= (int32_t)P.voff[rpiece[i]];
        if (row_ptr)
            PGCP_CUDA(cudaMemcpyAsync(row_ptr, rp64.data(), (P.Nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        if (col) PGCP_CUDA(cudaMemcpyAsync(col, c.data(), P.nnz * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        if (val) PGCP_CUDA(cudaMemcpyAsync(val, P.val64.p, P.nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
        PGCP_CUDA(cudaStreamSynchronize(s));
    });
}

pgcp_status pgcp_part_get_coords(pgcp_ctx* ctx, const pgcp_part* part, int32_t which, double* out) {
    return guard(ctx, [&] {
        if (!part || !out) fail(PGCP_E_ARG, "null argument");
        const Part& P = part->p;
        const DBuf<double2>* src = which == 0 ? &P.local : which == 1 ? &P.welded : which == 2 ? &P.final : nullptr;
        if (!src || !src->p) fail(PGCP_E_ARG, "requested coordinates are not computed yet");
        PGCP_CUDA(cudaMemcpyAsync(out, src->p, P.Nc * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream));
        PGCP_CUDA(cudaStreamSynchronize(ctx->stream));
    });
}

pgcp_status pgcp_weld(pgcp_ctx* ctx, pgcp_part* part) {
    return guard(ctx, [&] {
        if (!part) fail(PGCP_E_ARG, "null part");
        Part& P = part->p;
        if (!P.have_local) fail(PGCP_E_ARG, "call pgcp_local_param first");
        if (P.closed && ctx->opt.variant != PGCP_SPHERE) fail(PGCP_E_ARG, "closed surface needs the sphere variant");
        if (!P.closed && ctx->opt.variant == PGCP_SPHERE) fail(PGCP_E_ARG, "sphere variant needs a closed surface");
        Timer t(ctx->stream);
        run_welds(ctx, P);
        P.stats.ms_weld = t.stop();
    });
}

pgcp_status pgcp_global_solve(pgcp_ctx* ctx, pgcp_part* part, double* out, int32_t host_out, pgcp_stats* st) {
    return guard(ctx, [&] {
        if (!part || !out) fail(PGCP_E_ARG, "null argument");
        Part& P = part->p;
        if (!P.have_weld) fail(PGCP_E_ARG, "call pgcp_weld first");
        Timer t(ctx->stream);
        try {
            solve_final(ctx, P, out, host_out);
        } catch (...) {
            P.stats.ms_final = t.stop();
            if (st) *st = P.stats;
            throw;
        }
        P.stats.ms_final = t.stop();
        if (st) *st = P.stats;
    });
}

pgcp_status pgcp_metrics(pgcp_ctx* ctx, const pgcp_part* part, const double* U, pgcp_distortion* met) {
    return guard(ctx, [&] {
        if (!part || !U || !met) fail(PGCP_E_ARG, "null argument");
        compute_metrics(ctx, part->p, U, met);
    });
}

pgcp_status pgcp_area_distortion(pgcp_ctx* ctx, const pgcp_part* part, const double* U, double* mean_abs) {
    return guard(ctx, [&] {
        if (!part || !U || !mean_abs) fail(PGCP_E_ARG, "null argument");
        area_distortion(ctx, part->p, U, mean_abs);
    });
}

pgcp_status pgcp_area_mobius(pgcp_ctx* ctx, const pgcp_part* part, double* U, int32_t variant, pgcp_area_result* out) {
    return guard(ctx, [&] {
        if (!part || !U || !out) fail(PGCP_E_ARG, "null argument");
        area_mobius(ctx, part->p, U, variant, out);
    });
}

pgcp_status pgcp_set_piece_mask(pgcp_ctx* ctx, pgcp_part* part, const uint8_t* own) {
    return guard(ctx, [&] {
        if (!part) fail(PGCP_E_ARG, "null part");
        Part& P = part->p;
        if (!own) {
            P.own.clear();
            return;
        }
        P.own.assign(own, own + P.K);
        for (auto& v : P.own) v = v ? 1 : 0;
    });
}

pgcp_status pgcp_part_get_boundary(pgcp_ctx* ctx, const pgcp_part* part, int32_t which, double* out) {
    return guard(ctx, [&] {
        if (!part || !out) fail(PGCP_E_ARG, "null argument");
        if (which != 0 && which != 1) fail(PGCP_E_ARG, "which must be 0 (local) or 1 (welded)");
        part_get_boundary(ctx, part->p, which, out);
    });
}

pgcp_status pgcp_part_set_boundary(pgcp_ctx* ctx, pgcp_part* part, int32_t which, const double* in) {
    return guard(ctx, [&] {
        if (!part || !in) fail(PGCP_E_ARG, "null argument");
        if (which != 0 && which != 1) fail(PGCP_E_ARG, "which must be 0 (local) or 1 (welded)");
        part_set_boundary(ctx, part->p, which, in);
    });
}

pgcp_status pgcp_fix_folds(pgcp_ctx* ctx, pgcp_part* part, double* U, pgcp_fold_report* rep) {
    return guard(ctx, [&] {
        if (!ctx || !part || !U) fail(PGCP_E_ARG, "null argument");
        Part& P = part->p;
        if (P.closed) fail(PGCP_E_ARG, "the fold fix takes planar maps (free or disk parts)");
        if (!P.row_ptr.p) {
            assemble_laplacian(ctx, P);
            P.stats.nnz = P.nnz;
        }
        pgcp_fold_report r{};
        fix_folds(ctx, P, U, &r);
        if (rep) *rep = r;
    });
}

pgcp_status pgcp_metrics_noalloc(pgcp_ctx* ctx, const pgcp_part* part, const double* U, pgcp_distortion* met) {
    return guard(ctx, [&] {
        if (!ctx || !part || !U || !met) fail(PGCP_E_ARG, "null argument");
        static_assert(PGCP_METRICS_NOALLOC_MAX_FACES == (1 << 18), "header limit and library limit differ");
        if (metrics_noalloc_max_faces() != PGCP_METRICS_NOALLOC_MAX_FACES)
            fail(PGCP_E_ARG, "allocation-free metrics: header limit and library limit differ");
        compute_metrics_noalloc(ctx, part->p, U, met);
    });
}

pgcp_status pgcp_run(pgcp_ctx* ctx, const double* V, int64_t nv, const int32_t* F, int64_t nf,
                     const int32_t* cut_edges, int64_t n_cut, const int32_t* face_labels, int32_t host_ptrs,
                     double* out, pgcp_stats* st) {
    pgcp_part* part = nullptr;
    pgcp_status s = pgcp_partition(ctx, V, nv, F, nf, cut_edges, n_cut, face_labels, host_ptrs,
                                   ctx && ctx->opt.variant == PGCP_SPHERE, &part);
    if (s == PGCP_OK) s = pgcp_local_param(ctx, part);
    if (s == PGCP_OK) s = pgcp_weld(ctx, part);
    if (s == PGCP_OK) s = pgcp_global_solve(ctx, part, out, host_ptrs, st);
    if (part) pgcp_part_free(part);
    return s;
}

namespace {
pgcp_status run_variant(pgcp_ctx* ctx, int32_t variant, const double* V, int64_t nv, const int32_t* F, int64_t nf,
                        const int32_t* cut, int64_t n_cut, const int32_t* face_labels, double* out,
                        pgcp_stats* st) {
    if (!ctx) return PGCP_E_ARG;
    const int32_t saved = ctx->opt.variant;
    ctx->opt.variant = variant;
    const pgcp_status s = pgcp_run(ctx, V, nv, F, nf, cut, n_cut, face_labels, 0, out, st);
    ctx->opt.variant = saved;
    return s;
}
}  // namespace

pgcp_status pgcp_free_boundary(pgcp_ctx* ctx, const double* V, int64_t nv, const int32_t* F, int64_t nf,
                               const int32_t* cut, int64_t n_cut, const int32_t* face_labels, double* uv_out,
                               pgcp_stats* st) {
    return run_variant(ctx, PGCP_FREE, V, nv, F, nf, cut, n_cut, face_labels, uv_out, st);
}

pgcp_status pgcp_disk(pgcp_ctx* ctx, const double* V, int64_t nv, const int32_t* F, int64_t nf,
                      const int32_t* cut, int64_t n_cut, const int32_t* face_labels, double* uv_out,
                      pgcp_stats* st) {
    return run_variant(ctx, PGCP_DISK, V, nv, F, nf, cut, n_cut, face_labels, uv_out, st);
}

pgcp_status pgcp_sphere(pgcp_ctx* ctx, const double* V, int64_t nv, const int32_t* F, int64_t nf,
                        const int32_t* cut, int64_t n_cut, const int32_t* face_labels, double* xyz_out,
                        pgcp_stats* st) {
    return run_variant(ctx, PGCP_SPHERE, V, nv, F, nf, cut, n_cut, face_labels, xyz_out, st);
}

pgcp_status pgcp_batch_run(pgcp_ctx* ctx, int32_t n_mesh, const pgcp_mesh_desc* meshes, double* const* outs,
                           int32_t* mesh_status, pgcp_stats* st) {
    pgcp_part* part = nullptr;
    pgcp_status s = guard(ctx, [&] {
        if (!ctx || n_mesh <= 0 || !meshes || !outs) fail(PGCP_E_ARG, "bad batch arguments");
        for (int32_t b = 0; b < n_mesh; ++b)
            if (!outs[b] || !meshes[b].face_labels) fail(PGCP_E_ARG, "batch mesh without labels or output");
    });
    if (s != PGCP_OK) return s;
    std::vector<const double*> V(n_mesh);
    std::vector<const int32_t*> F(n_mesh), Lb(n_mesh);
    std::vector<int64_t> nv(n_mesh), nf(n_mesh);
    for (int32_t b = 0; b < n_mesh; ++b) {
        V[b] = meshes[b].V;
        F[b] = meshes[b].F;
        Lb[b] = meshes[b].face_labels;
        nv[b] = meshes[b].nv;
        nf[b] = meshes[b].nf;
    }
    s = pgcp_partition_batch(ctx, n_mesh, V.data(), nv.data(), F.data(), nf.data(), Lb.data(), 0,
                             ctx->opt.variant == PGCP_SPHERE, &part);
    if (s == PGCP_OK) s = pgcp_local_param(ctx, part);
    if (s == PGCP_OK) s = pgcp_weld(ctx, part);
    if (s == PGCP_OK) {
        const int dim = ctx->opt.variant == PGCP_SPHERE ? 3 : 2;
        int64_t total = 0;
        for (int32_t b = 0; b < n_mesh; ++b) total += nv[b];
        s = guard(ctx, [&] {
            DBuf<double> all;
            all.alloc(dim * total, ctx->stream);
            const pgcp_status g = pgcp_global_solve(ctx, part, all.p, 0, st);
            if (g != PGCP_OK) throw Thrown(g, ctx->last_error);
            int64_t off = 0;
            for (int32_t b = 0; b < n_mesh; ++b) {
                PGCP_CUDA(cudaMemcpyAsync(outs[b], all.p + dim * off, dim * nv[b] * sizeof(double),
                                          cudaMemcpyDeviceToDevice, ctx->stream));
                off += nv[b];
            }
            PGCP_CUDA(cudaStreamSynchronize(ctx->stream));
        });
    }
    if (part && mesh_status) pgcp_part_mesh_status(part, mesh_status);
    if (part) pgcp_part_free(part);
    return s;
}

pgcp_status pgcp_selftest_sort(pgcp_ctx* ctx, uint64_t* keys, int32_t* vals, int64_t n, int32_t bits) {
    return guard(ctx, [&] {
        if (!keys || !vals || n < 0 || bits < 0 || bits > 64) fail(PGCP_E_ARG, "bad sort arguments");
        radix_sort_pairs(keys, vals, n, bits, ctx->stream);
        PGCP_CUDA(cudaStreamSynchronize(ctx->stream));
    });
}

pgcp_status pgcp_selftest_scan(pgcp_ctx* ctx, const int32_t* in, int64_t* out, int64_t n, int64_t* total) {
    return guard(ctx, [&] {
        if (!in || !out || n < 0) fail(PGCP_E_ARG, "bad scan arguments");
        int64_t t = 0;
        exclusive_scan_i32_to_i64(in, out, n, ctx->stream, &t);
        PGCP_CUDA(cudaStreamSynchronize(ctx->stream));
        if (total) *total = t;
    });
}

pgcp_status pgcp_autotune(pgcp_ctx* ctx, pgcp_part* part, int32_t probe_iters, pgcp_options* chosen,
                          double* ms_per_iter) {
    return guard(ctx, [&] {
        if (!ctx || !part || !chosen) fail(PGCP_E_ARG, "null argument");
        if (probe_iters < 10) fail(PGCP_E_ARG, "probe_iters must be at least 10");
        Part& P = part->p;
        if (!P.row_ptr.p) {
            Timer t(ctx->stream);
            assemble_laplacian(ctx, P);
            P.stats.ms_assembly = t.stop();
            P.stats.nnz = P.nnz;
        }
        const pgcp_options saved = ctx->opt;
        struct Cand {
            int bps, sched, lanes, rows;
        };
        std::vector<Cand> cands;
        if (saved.local_precision == PGCP_FP64) {
            for (int lanes : {1, 2, 4})
                for (int rows : {8, 9, 10}) cands.push_back(Cand{saved.pcg_blocks_per_sm, saved.pcg_schedule, lanes, rows});
        } else if (saved.local_precision == PGCP_DF64_REFINED && saved.local_precond == 0 && !saved.deterministic) {
            // the multilevel preconditioner runs on the static schedule only, and the
            // probes compare time per iteration, which is meaningless across
            // preconditioners: the static schedule is the one candidate
            cands.push_back(Cand{saved.pcg_blocks_per_sm ? saved.pcg_blocks_per_sm : 4, 1, saved.spmv_lanes,
                                 saved.block_rows_log2});
        } else {
            // deterministic mode runs the static schedule only
            for (int sched : {1, 2, 3, 4})
                if (sched == 1 || !saved.deterministic)
                    for (int bps : {3, 4}) cands.push_back(Cand{bps, sched, saved.spmv_lanes, saved.block_rows_log2});
        }
        double best = INFINITY;
        Cand pick = cands[0];
        try {
            for (const Cand& c : cands) {
                ctx->opt.pcg_blocks_per_sm = c.bps;
                ctx->opt.pcg_schedule = c.sched;
                ctx->opt.spmv_lanes = c.lanes;
                ctx->opt.block_rows_log2 = c.rows;
                ctx->opt.max_iters = probe_iters;
                ctx->opt.max_refine = 1;
                const double ms0 = P.stats.pcg_ms;
                try {
                    solve_dncp(ctx, P);
                } catch (const Thrown& t) {
                    if (t.code != PGCP_E_NO_CONVERGENCE) throw;   // capped probe: expected
                }
                const int it = std::max(1, P.stats.dncp_iters);
                const double per = (P.stats.pcg_ms - ms0) / it;
                if (per < best) {
                    best = per;
                    pick = c;
                }
            }
        } catch (...) {
            ctx->opt = saved;
            throw;
        }
        ctx->opt = saved;
        ctx->opt.pcg_blocks_per_sm = pick.bps;
        ctx->opt.pcg_schedule = pick.sched;
        ctx->opt.spmv_lanes = pick.lanes;
        ctx->opt.block_rows_log2 = pick.rows;
        P.have_local = 0;   // the probes leave no usable local map
        *chosen = ctx->opt;
        if (ms_per_iter) *ms_per_iter = best;
    });
}

pgcp_status pgcp_part_mesh_status(const pgcp_part* part, int32_t* status) {
    if (!part || !status) return PGCP_E_ARG;
    const Part& P = part->p;
    for (size_t mi = 0; mi < P.meshes.size(); ++mi)
        status[mi] = mi < P.mesh_status.size() ? P.mesh_status[mi] : (int32_t)PGCP_OK;
    return PGCP_OK;
}

int64_t pgcp_gnn_num_params(void) { return gnn_num_params(); }

pgcp_status pgcp_gnn_create(pgcp_ctx* ctx, const float* params, pgcp_gnn** out) {
    return guard(ctx, [&] {
        if (!ctx || !params || !out) fail(PGCP_E_ARG, "null argument");
        *out = nullptr;
        auto* g = new pgcp_gnn();
        try {
            gnn_init(ctx, g, params);
        } catch (...) {
            delete g;
            throw;
        }
        *out = g;
    });
}

pgcp_status pgcp_gnn_load(pgcp_ctx* ctx, const char* path, pgcp_gnn** out) {
    return guard(ctx, [&] {
        if (!ctx || !path || !out) fail(PGCP_E_ARG, "null argument");
        FILE* f = std::fopen(path, "rb");
        if (!f) fail(PGCP_E_ARG, std::string("cannot open ") + path);
        std::vector<float> v((size_t)gnn_num_params());
        const size_t got = std::fread(v.data(), sizeof(float), v.size(), f);
        const bool extra = std::fgetc(f) != EOF;
        std::fclose(f);
        if (got != v.size() || extra) fail(PGCP_E_ARG, std::string("wrong parameter count in ") + path);
        *out = nullptr;
        auto* g = new pgcp_gnn();
        try {
            gnn_init(ctx, g, v.data());
        } catch (...) {
            delete g;
            throw;
        }
        *out = g;
    });
}

pgcp_status pgcp_gnn_free(pgcp_gnn* gnn) {
    delete gnn;
    return PGCP_OK;
}

pgcp_status pgcp_gnn_get_params(pgcp_ctx* ctx, const pgcp_gnn* gnn, float* params) {
    return guard(ctx, [&] {
        if (!ctx || !gnn || !params) fail(PGCP_E_ARG, "null argument");
        gnn_get(ctx, gnn, params);
    });
}

pgcp_status pgcp_gnn_set_params(pgcp_ctx* ctx, pgcp_gnn* gnn, const float* params) {
    return guard(ctx, [&] {
        if (!ctx || !gnn || !params) fail(PGCP_E_ARG, "null argument");
        gnn_set(ctx, gnn, params);
    });
}

pgcp_status pgcp_set_gnn(pgcp_ctx* ctx, pgcp_gnn* gnn) {
    return guard(ctx, [&] {
        if (!ctx) fail(PGCP_E_ARG, "null context");
        if (gnn && gnn->device != ctx->device) fail(PGCP_E_ARG, "network and context are on different devices");
        ctx->gnn = gnn;
    });
}

pgcp_status pgcp_gnn_inputs(pgcp_ctx* ctx, const pgcp_part* part, float* feat, float* target, float* sigma) {
    return guard(ctx, [&] {
        if (!ctx || !part || !feat || !sigma) fail(PGCP_E_ARG, "null argument");
        gnn_inputs(ctx, const_cast<Part&>(part->p), feat, target, sigma);
    });
}

pgcp_status pgcp_gnn_grad(pgcp_ctx* ctx, pgcp_gnn* gnn, const pgcp_part* part, float* grad, double* loss) {
    return guard(ctx, [&] {
        if (!ctx || !gnn || !part || !grad) fail(PGCP_E_ARG, "null argument");
        const double l = gnn_grad(ctx, gnn, const_cast<Part&>(part->p), 0, 0.f);
        PGCP_CUDA(cudaMemcpyAsync(grad, gnn->grad.p, gnn_num_params() * sizeof(float), cudaMemcpyDeviceToHost,
                                  ctx->stream));
        PGCP_CUDA(cudaStreamSynchronize(ctx->stream));
        if (loss) *loss = l;
    });
}

pgcp_status pgcp_gnn_train_step(pgcp_ctx* ctx, pgcp_gnn* gnn, const pgcp_part* part, float lr, double* loss) {
    return guard(ctx, [&] {
        if (!ctx || !gnn || !part) fail(PGCP_E_ARG, "null argument");
        if (!(lr > 0.f)) fail(PGCP_E_ARG, "learning rate must be positive");
        const double l = gnn_grad(ctx, gnn, const_cast<Part&>(part->p), 1, lr);
        if (loss) *loss = l;
    });
}

pgcp_status pgcp_gnn_predict(pgcp_ctx* ctx, const pgcp_gnn* gnn, const pgcp_part* part, double* x0) {
    return guard(ctx, [&] {
        if (!ctx || !gnn || !part || !x0) fail(PGCP_E_ARG, "null argument");
        gnn_predict(ctx, gnn, const_cast<Part&>(part->p), reinterpret_cast<double2*>(x0));
    });
}

pgcp_status pgcp_selftest_gemm_bf16(pgcp_ctx* ctx, int32_t epilogue, int32_t N, int32_t K, const void* A,
                                    const void* Bt, int64_t M, const float* bias, void* C) {
    return guard(ctx, [&] {
        if (!A || !Bt || !C || M < 0) fail(PGCP_E_ARG, "bad GEMM arguments");
        if (epilogue != 0 && !bias) fail(PGCP_E_ARG, "this epilogue needs a bias");
        ctx->err.zero();
        gemm_bf16_tc(ctx->stream, epilogue, N, K, A, K, Bt, M, bias, C, N, nullptr, 0, ctx->err.p);
        if (read_errors(ctx) & DE_TIMEOUT) fail(PGCP_E_CUDA, "tensor-core GEMM: accumulator wait timed out");
    });
}

uint64_t pgcp_selftest_umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) { return umma_desc_host(saddr, lbo, sbo); }
uint32_t pgcp_selftest_umma_idesc(int32_t m, int32_t n) { return umma_idesc_host(m, n); }

}  // extern "C"
