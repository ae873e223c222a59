// Stage drivers around the batched PCG: DNCP set-up and local frame
// (Section 4.2), final Laplace solve with the welded boundary (Section 4.5),
// gather (lowest label wins) and stereographic projection (Algorithm 3).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "pgcp_internal.h"

namespace pgcp {

namespace {

__global__ void k_dncp_init(int64_t n, uint8_t* __restrict__ fixed, double2* __restrict__ x) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        fixed[i] = 0;
        x[i] = make_double2(0.0, 0.0);
    }
}

__global__ void k_dncp_pins(const int32_t* __restrict__ pin_rows, int32_t K, uint8_t* __restrict__ fixed,
                            double2* __restrict__ x) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    int p0 = pin_rows[2 * i], p1 = pin_rows[2 * i + 1];
    fixed[p0] = 1;
    fixed[p1] = 1;
    x[p0] = make_double2(0.0, 0.0);
    x[p1] = make_double2(1.0, 0.0);
}

// rows of pieces another rank solves: fixed at 0 (their system is empty here)
__global__ void k_fix_unowned(int64_t n, const int32_t* __restrict__ row_piece, const uint8_t* __restrict__ own,
                              uint8_t* __restrict__ fixed, double2* __restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || own[row_piece[i]]) return;
    fixed[i] = 1;
    x[i] = make_double2(0.0, 0.0);
}

__global__ void k_loop_get(int64_t nl, const int32_t* __restrict__ loop_rows, const double2* __restrict__ X,
                           double* __restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nl) return;
    const double2 v = X[loop_rows[j]];
    out[2 * j] = v.x;
    out[2 * j + 1] = v.y;
}

// loop rows take the given values; with zero_inner, every other row is set to 0
__global__ void k_loop_set(int64_t n, const uint8_t* __restrict__ is_bnd, int zero_inner, double2* __restrict__ X) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && zero_inner && !is_bnd[i]) X[i] = make_double2(0.0, 0.0);
}
__global__ void k_loop_put(int64_t nl, const int32_t* __restrict__ loop_rows, const double* __restrict__ in,
                           double2* __restrict__ X) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nl) return;
    X[loop_rows[j]] = make_double2(in[2 * j], in[2 * j + 1]);
}

// translate each piece so its reference vertex is at 0
__global__ void k_translate(int64_t n, const int32_t* __restrict__ row_piece, const int32_t* __restrict__ ref_rows,
                            const double2* __restrict__ x, double2* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = ref_rows[row_piece[i]];
    double2 v = x[i];
    if (r >= 0) {
        double2 c = x[r];
        v.x = v.x - c.x;
        v.y = v.y - c.y;
    }
    out[i] = v;
}

// Start of the final solve: welded boundary values, interior from the weld map
// (or 0 for a cold start).  Pieces of meshes dropped from a batch by the
// welding get 0 everywhere: right-hand side 0, converged at once, and their
// output is NaN after the gather.
__global__ void k_final_init(int64_t n, const uint8_t* __restrict__ is_bnd, const int32_t* __restrict__ row_piece,
                             const uint8_t* __restrict__ wchart, const double2* __restrict__ welded, int cold,
                             double2* __restrict__ x) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (wchart[row_piece[i]] == 2) {
        x[i] = make_double2(0.0, 0.0);
        return;
    }
    x[i] = (is_bnd[i] || !cold) ? welded[i] : make_double2(0.0, 0.0);
}

// out[v] from the lowest-label copy; seam mismatch = max |copy - chosen copy|
__global__ void k_gather(int64_t Nc, const int32_t* __restrict__ copy_vert, const int32_t* __restrict__ first_copy,
                         const int32_t* __restrict__ row_piece, const uint8_t* __restrict__ wchart,
                         const double2* __restrict__ X,
                         int dim, double* __restrict__ out, unsigned long long* __restrict__ mism) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nc) return;
    if (wchart[row_piece[i]] == 2) return;   // piece of a mesh dropped from the batch
    const int v = copy_vert[i];
    const int f = first_copy[v];
    double a[3], b[3];
    auto coords = [&](int row, double* c) {
        double2 z = X[row];
        if (dim == 2) {
            c[0] = z.x;
            c[1] = z.y;
            c[2] = 0.0;
        } else {
            // orientation-preserving inverse stereographic projection; the
            // pieces around infinity are stored in the chart w = 1/z
            double r2 = z.x * z.x + z.y * z.y, d = 1.0 + r2;
            if (wchart[row_piece[row]] == 1) {
                c[0] = 2.0 * z.x / d;
                c[1] = 2.0 * z.y / d;
                c[2] = (1.0 - r2) / d;
            } else {
                c[0] = 2.0 * z.x / d;
                c[1] = -2.0 * z.y / d;
                c[2] = (r2 - 1.0) / d;
            }
        }
    };
    coords((int)i, a);
    if (f == (int)i) {
        for (int c = 0; c < dim; ++c) out[(int64_t)dim * v + c] = a[c];
    } else if (wchart[row_piece[f]] != 2) {   // (a first copy in a skipped piece is written elsewhere)
        coords(f, b);
        double m = 0.0;
        for (int c = 0; c < dim; ++c) m = fmax(m, fabs(a[c] - b[c]));
        atomicMax(mism, (unsigned long long)__double_as_longlong(m));
    }
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, ceil_div(n, t)); }

}  // namespace

void solve_dncp(pgcp_ctx* ctx, Part& P) {
    cudaStream_t s = ctx->stream;
    const int64_t n = P.Nc;
    DBuf<uint8_t> fixed;
    DBuf<double2> x;
    DBuf<int32_t> pins, refs;
    fixed.alloc(n, s);
    x.alloc(n, s);
    std::vector<int32_t> hp(2 * P.K), hr(P.K);
    for (int i = 0; i < P.K; ++i) {
        hp[2 * i] = (int32_t)P.pin0[i];
        hp[2 * i + 1] = (int32_t)P.pin1[i];
        hr[i] = (int32_t)P.ref[i];
    }
    pins.alloc(2 * P.K, s);
    refs.alloc(P.K, s);
    PGCP_CUDA(cudaMemcpyAsync(pins.p, hp.data(), hp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    PGCP_CUDA(cudaMemcpyAsync(refs.p, hr.data(), hr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    { k_dncp_init<<<nblk(n), 256, 0, s>>>(n, fixed.p, x.p); ::pgcp::note_launch(); }
    { k_dncp_pins<<<nblk(P.K), 256, 0, s>>>(pins.p, P.K, fixed.p, x.p); ::pgcp::note_launch(); }
    DBuf<uint8_t> own;
    if (!P.own.empty()) {
        own.alloc(P.K, s);
        PGCP_CUDA(cudaMemcpyAsync(own.p, P.own.data(), P.K, cudaMemcpyHostToDevice, s));
        { k_fix_unowned<<<nblk(n), 256, 0, s>>>(n, P.row_piece.p, own.p, fixed.p, x.p); ::pgcp::note_launch(); }
    }
    PGCP_CUDA(cudaGetLastError());
    SolveResult r = pcg_solve(ctx, P, 1, fixed.p, x.p);
    P.stats.dncp_iters = r.iters;
    P.stats.dncp_refine = r.refine;
    P.stats.dncp_relres = r.relres;
    P.local.alloc(n, s);
    { k_translate<<<nblk(n), 256, 0, s>>>(n, P.row_piece.p, refs.p, x.p, P.local.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    PGCP_CUDA(cudaStreamSynchronize(s));
    P.have_local = 1;
    if (!(r.relres <= ctx->opt.tol))
        fail(PGCP_E_NO_CONVERGENCE, "local (DNCP) solve reached relative residual " + std::to_string(r.relres));
}

void solve_final(pgcp_ctx* ctx, Part& P, double* out, int host_out) {
    cudaStream_t s = ctx->stream;
    const int64_t n = P.Nc;
    P.final.alloc(n, s);
    { k_final_init<<<nblk(n), 256, 0, s>>>(n, P.is_bnd.p, P.row_piece.p, P.d_wchart.p, P.welded.p,
                                         ctx->opt.warm_start == PGCP_WARM_COLD, P.final.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    P.stats.learned_pieces = 0;
    if (ctx->opt.warm_start == PGCP_WARM_LEARNED) P.stats.learned_pieces = learned_start(ctx, P, P.final.p);
    SolveResult r = pcg_solve(ctx, P, 0, P.is_bnd.p, P.final.p);
    P.stats.final_iters = r.iters;
    P.stats.final_refine = r.refine;
    P.stats.final_relres = r.relres;
    P.have_final = 1;
    const int dim = P.closed ? 3 : 2;
    DBuf<double> dout;
    double* o = out;
    if (host_out) {
        dout.alloc(dim * P.nv, s);
        o = dout.p;
    }
    DBuf<unsigned long long> mism;
    mism.alloc(1, s);
    mism.zero();
    // vertices in no face stay NaN (all-ones bit pattern)
    PGCP_CUDA(cudaMemsetAsync(o, 0xff, dim * P.nv * sizeof(double), s));
    { k_gather<<<nblk(n), 256, 0, s>>>(n, P.copy_vert.p, P.first_copy.p, P.row_piece.p, P.d_wchart.p, P.final.p,
                                     dim, o, mism.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    // meshes dropped from a batch by the welding: NaN output
    for (size_t mi = 0; mi < P.mesh_status.size(); ++mi)
        if (P.mesh_status[mi] != PGCP_OK)
            PGCP_CUDA(cudaMemsetAsync(o + dim * P.meshes[mi].v0, 0xff, dim * P.meshes[mi].nv * sizeof(double), s));
    unsigned long long m = 0;
    PGCP_CUDA(cudaMemcpyAsync(&m, mism.p, sizeof(m), cudaMemcpyDeviceToHost, s));
    if (host_out)
        PGCP_CUDA(cudaMemcpyAsync(out, dout.p, dim * P.nv * sizeof(double), cudaMemcpyDeviceToHost, s));
    PGCP_CUDA(cudaStreamSynchronize(s));
    double md;
    memcpy(&md, &m, sizeof(md));
    P.stats.seam_mismatch = md;
    if (!(r.relres <= ctx->opt.tol))
        fail(PGCP_E_NO_CONVERGENCE, "final Laplace solve reached relative residual " + std::to_string(r.relres));
}

void part_get_boundary(pgcp_ctx* ctx, const Part& P, int which, double* out) {
    const DBuf<double2>& X = which == 0 ? P.local : P.welded;
    if (!(which == 0 ? P.have_local : P.have_weld)) fail(PGCP_E_ARG, which == 0 ? "no local map yet" : "no welded map yet");
    const int64_t nl = (int64_t)P.loop_rows.size();
    { k_loop_get<<<nblk(nl), 256, 0, ctx->stream>>>(nl, P.d_loop_rows.p, X.p, out); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    PGCP_CUDA(cudaStreamSynchronize(ctx->stream));
}

void part_set_boundary(pgcp_ctx* ctx, Part& P, int which, const double* in) {
    cudaStream_t s = ctx->stream;
    const int64_t nl = (int64_t)P.loop_rows.size(), n = P.Nc;
    if (which == 0) {
        if (!P.have_local) fail(PGCP_E_ARG, "call pgcp_local_param before importing local boundaries");
        { k_loop_put<<<nblk(nl), 256, 0, s>>>(nl, P.d_loop_rows.p, in, P.local.p); ::pgcp::note_launch(); }
    } else {
        // the welded boundary of every piece; interior rows start at 0 (the
        // final solve's cold start); pieces this part does not own are skipped
        if (P.closed) fail(PGCP_E_ARG, "welded boundaries are imported into open parts only");
        if (!P.welded.p) P.welded.alloc(n, s);
        { k_loop_set<<<nblk(n), 256, 0, s>>>(n, P.is_bnd.p, 1, P.welded.p); ::pgcp::note_launch(); }
        { k_loop_put<<<nblk(nl), 256, 0, s>>>(nl, P.d_loop_rows.p, in, P.welded.p); ::pgcp::note_launch(); }
        P.wchart.assign(P.K, 0);
        for (int i = 0; i < P.K; ++i)
            if (!P.own.empty() && !P.own[i]) P.wchart[i] = 2;
        P.d_wchart.alloc(P.K, s);
        PGCP_CUDA(cudaMemcpyAsync(P.d_wchart.p, P.wchart.data(), P.K, cudaMemcpyHostToDevice, s));
        P.mesh_status.assign(P.meshes.size(), PGCP_OK);
        P.have_weld = 1;
    }
    PGCP_CUDA(cudaGetLastError());
    PGCP_CUDA(cudaStreamSynchronize(s));
}

}  // namespace pgcp
