// Area distortion and the Mobius area step (Section 6.2).
//
// d_area(T) = ln((A_f(T) / sum A_f) / (A(T) / sum A)) per face, A the surface
// triangle's area and A_f the planar parameter triangle's signed area.  The
// step composes a mesh's map with the member of a two-parameter Mobius family
// that minimises mean |d_area|: disk automorphisms (z - a) / (1 - conj(a) z),
// or, for a free boundary, z / (1 - q z) (a Mobius map up to a similarity,
// which leaves normalised areas unchanged).  The search is Nelder-Mead
// (Nelder and Mead, Computer Journal 7, 1965) on the host; each objective
// evaluation is two reductions over the mesh's faces on the device.  All sums
// run over a fixed grid and are added on the host in block order, so an
// evaluation is repeatable to the bit and the search takes the same path on
// every run.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <vector>

#include "pgcp_internal.h"

namespace pgcp {

namespace {

constexpr int AREA_BLOCKS = 512;
constexpr int AREA_THREADS = 256;
constexpr double NM_STEP = 0.05;
constexpr double NM_FTOL = 1e-12;
constexpr double NM_XTOL = 1e-9;
constexpr int NM_MAXIT = 500;

// family member with parameter (pr, pi) at z: disk (variant 1) or free (0)
__device__ __forceinline__ double2 mobius(int disk, double pr, double pi, double2 z) {
    double nr, ni, dr, di;
    if (disk) {   // (z - a) / (1 - conj(a) z)
        nr = z.x - pr;
        ni = z.y - pi;
        dr = 1.0 - (pr * z.x + pi * z.y);
        di = -(pr * z.y - pi * z.x);
    } else {      // z / (1 - q z)
        nr = z.x;
        ni = z.y;
        dr = 1.0 - (pr * z.x - pi * z.y);
        di = -(pr * z.y + pi * z.x);
    }
    const double m = dr * dr + di * di;
    return make_double2((nr * dr + ni * di) / m, (ni * dr - nr * di) / m);
}

__global__ void k_area_map(const double2* __restrict__ U, int64_t v0, int64_t nv, int disk, double pr, double pi,
                           double2* __restrict__ W) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x)
        W[v0 + i] = mobius(disk, pr, pi, U[v0 + i]);
}

// fixed-order block sum of two values; thread 0 writes them to part[2 * blockIdx.x]
__device__ __forceinline__ void block_sum2(double a, double b, double* part) {
    __shared__ double red[2 * (AREA_THREADS / 32)];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[2 * w] = a;
        red[2 * w + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int i = 0; i < AREA_THREADS / 32; ++i) {
            s0 += red[2 * i];
            s1 += red[2 * i + 1];
        }
        part[2 * blockIdx.x] = s0;
        part[2 * blockIdx.x + 1] = s1;
    }
}

// surface areas of the mesh's faces, and their sum per block
__global__ void __launch_bounds__(AREA_THREADS) k_area_surface(const int32_t* __restrict__ F, const double* __restrict__ V,
                                                               int64_t f0, int64_t nf, double* __restrict__ At,
                                                               double* __restrict__ part) {
    double s = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nf; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = f0 + t;
        const double* a = V + 3 * (int64_t)F[3 * f];
        const double* b = V + 3 * (int64_t)F[3 * f + 1];
        const double* c = V + 3 * (int64_t)F[3 * f + 2];
        const double e1x = b[0] - a[0], e1y = b[1] - a[1], e1z = b[2] - a[2];
        const double e2x = c[0] - a[0], e2y = c[1] - a[1], e2z = c[2] - a[2];
        const double cx = e1y * e2z - e1z * e2y, cy = e1z * e2x - e1x * e2z, cz = e1x * e2y - e1y * e2x;
        const double ar = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
        At[t] = ar;
        s += ar;
    }
    block_sum2(s, 0.0, part);
}

__device__ __forceinline__ double param_area(const int32_t* __restrict__ F, const double2* __restrict__ W, int64_t f) {
    const double2 a = W[F[3 * f]], b = W[F[3 * f + 1]], c = W[F[3 * f + 2]];
    return 0.5 * ((b.x - a.x) * (c.y - a.y) - (b.y - a.y) * (c.x - a.x));
}

// pass 1: sum of the parameter areas and the count of non-positive or non-finite ones
__global__ void __launch_bounds__(AREA_THREADS) k_area_pass1(const int32_t* __restrict__ F, const double2* __restrict__ W,
                                                             int64_t f0, int64_t nf, double* __restrict__ part) {
    double s = 0.0, bad = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nf; t += (int64_t)gridDim.x * blockDim.x) {
        const double af = param_area(F, W, f0 + t);
        if (!(af > 0.0) || !isfinite(af)) bad += 1.0;
        else s += af;
    }
    block_sum2(s, bad, part);
}

// pass 2: sum of |ln(A_f / A) - c| with c = ln(sum A_f / sum A)
__global__ void __launch_bounds__(AREA_THREADS) k_area_pass2(const int32_t* __restrict__ F, const double2* __restrict__ W,
                                                             const double* __restrict__ At, int64_t f0, int64_t nf,
                                                             double c, double* __restrict__ part) {
    double s = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nf; t += (int64_t)gridDim.x * blockDim.x)
        s += fabs(log(param_area(F, W, f0 + t) / At[t]) - c);
    block_sum2(s, 0.0, part);
}

unsigned grid_for(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(AREA_BLOCKS, ceil_div(n, AREA_THREADS)));
}

// Objective evaluations for one mesh of a part.
struct AreaMesh {
    pgcp_ctx* ctx;
    const Part& P;
    const MeshInfo& M;
    const double2* U;
    double2* W;
    double* At;
    double* part;
    std::vector<double> h;
    double sum_at = 0.0;

    AreaMesh(pgcp_ctx* c, const Part& p, const MeshInfo& m, const double2* u, double2* w, double* at, double* pt)
        : ctx(c), P(p), M(m), U(u), W(w), At(at), part(pt), h(2 * AREA_BLOCKS) {
        const unsigned g = grid_for(M.nf);
        { k_area_surface<<<g, AREA_THREADS, 0, ctx->stream>>>(P.F.p, P.V.p, M.f0, M.nf, At, part); ::pgcp::note_launch(); }
        sum_at = fetch(g)[0];
    }

    std::array<double, 2> fetch(unsigned g) {
        PGCP_CUDA(cudaGetLastError());
        PGCP_CUDA(cudaMemcpyAsync(h.data(), part, 2 * g * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        PGCP_CUDA(cudaStreamSynchronize(ctx->stream));
        std::array<double, 2> s{0.0, 0.0};
        for (unsigned b = 0; b < g; ++b) {   // block order
            s[0] += h[2 * b];
            s[1] += h[2 * b + 1];
        }
        return s;
    }

    // mean |d_area| of the coordinates X (+inf on a non-positive or non-finite area)
    double mean_abs(const double2* X) {
        const unsigned g = grid_for(M.nf);
        { k_area_pass1<<<g, AREA_THREADS, 0, ctx->stream>>>(P.F.p, X, M.f0, M.nf, part); ::pgcp::note_launch(); }
        const std::array<double, 2> s1 = fetch(g);
        if (s1[1] > 0.0 || !(s1[0] > 0.0) || !std::isfinite(s1[0])) return INFINITY;
        const double c = std::log(s1[0] / sum_at);
        { k_area_pass2<<<g, AREA_THREADS, 0, ctx->stream>>>(P.F.p, X, At, M.f0, M.nf, c, part); ::pgcp::note_launch(); }
        const double m = fetch(g)[0] / (double)M.nf;
        return std::isfinite(m) ? m : INFINITY;
    }

    void map(int disk, double pr, double pi, double2* dst) {
        k_area_map<<<grid_for(M.nv), AREA_THREADS, 0, ctx->stream>>>(U, M.v0, M.nv, disk, pr, pi, dst);
        ::pgcp::note_launch();
        PGCP_CUDA(cudaGetLastError());
    }

    double objective(int disk, double pr, double pi) {
        if (disk && !(pr * pr + pi * pi < 1.0)) return INFINITY;
        map(disk, pr, pi, W);
        return mean_abs(W);
    }
};

// Nelder-Mead on R^2 from x0 (the same steps and constants as the oracle's)
template <typename Fn>
std::array<double, 2> nelder_mead(Fn fun, std::array<double, 2> x0, double* fbest, int* evals) {
    using P2 = std::array<double, 2>;
    P2 pts[3] = {x0, {x0[0] + NM_STEP, x0[1]}, {x0[0], x0[1] + NM_STEP}};
    double val[3] = {fun(pts[0]), fun(pts[1]), fun(pts[2])};
    int n = 3;
    auto lin = [](const P2& a, const P2& b, double t) { return P2{a[0] + t * (b[0] - a[0]), a[1] + t * (b[1] - a[1])}; };
    for (int it = 0; it < NM_MAXIT; ++it) {
        int ord[3] = {0, 1, 2};
        std::stable_sort(ord, ord + 3, [&](int a, int b) { return val[a] < val[b]; });
        P2 sp[3] = {pts[ord[0]], pts[ord[1]], pts[ord[2]]};
        double sv[3] = {val[ord[0]], val[ord[1]], val[ord[2]]};
        for (int i = 0; i < 3; ++i) {
            pts[i] = sp[i];
            val[i] = sv[i];
        }
        double size = 0.0;
        for (int i = 1; i < 3; ++i)
            size = std::max(size, std::max(std::fabs(pts[i][0] - pts[0][0]), std::fabs(pts[i][1] - pts[0][1])));
        if (std::isfinite(val[2]) && val[2] - val[0] <= NM_FTOL && size <= NM_XTOL) break;
        const P2 c{0.5 * (pts[0][0] + pts[1][0]), 0.5 * (pts[0][1] + pts[1][1])};
        const P2 xr = lin(c, pts[2], -1.0);   // reflection c + (c - worst)
        const double fr = fun(xr);
        ++n;
        if (fr < val[0]) {
            const P2 xe = lin(c, pts[2], -2.0);
            const double fe = fun(xe);
            ++n;
            if (fe < fr) {
                pts[2] = xe;
                val[2] = fe;
            } else {
                pts[2] = xr;
                val[2] = fr;
            }
        } else if (fr < val[1]) {
            pts[2] = xr;
            val[2] = fr;
        } else {
            const P2 xc = fr < val[2] ? lin(c, xr, 0.5) : lin(c, pts[2], 0.5);
            const double fc = fun(xc);
            ++n;
            if (fc < std::min(fr, val[2])) {
                pts[2] = xc;
                val[2] = fc;
            } else {
                for (int i = 1; i < 3; ++i) {
                    pts[i] = lin(pts[0], pts[i], 0.5);
                    val[i] = fun(pts[i]);
                    ++n;
                }
            }
        }
    }
    int best = 0;
    for (int i = 1; i < 3; ++i)
        if (val[i] < val[best]) best = i;
    *fbest = val[best];
    *evals = n;
    return pts[best];
}

}  // namespace

void area_distortion(pgcp_ctx* ctx, const Part& P, const double* U, double* mean_abs) {
    if (P.closed) fail(PGCP_E_ARG, "area distortion: planar results only");
    cudaStream_t s = ctx->stream;
    int64_t maxf = 1;
    for (const MeshInfo& M : P.meshes) maxf = std::max<int64_t>(maxf, M.nf);
    DBuf<double> At, part;
    At.alloc(maxf, s);
    part.alloc(2 * AREA_BLOCKS, s);
    for (size_t mi = 0; mi < P.meshes.size(); ++mi) {
        AreaMesh A(ctx, P, P.meshes[mi], reinterpret_cast<const double2*>(U), nullptr, At.p, part.p);
        const double m = A.mean_abs(reinterpret_cast<const double2*>(U));
        mean_abs[mi] = std::isfinite(m) ? m : NAN;
    }
}

void area_mobius(pgcp_ctx* ctx, const Part& P, double* U, int variant, pgcp_area_result* out) {
    if (P.closed) fail(PGCP_E_ARG, "Mobius area step: planar results only");
    if (variant != PGCP_DISK && variant != PGCP_FREE) fail(PGCP_E_ARG, "Mobius area step: variant must be DISK or FREE");
    const int disk = variant == PGCP_DISK;
    cudaStream_t s = ctx->stream;
    int64_t maxf = 1;
    for (const MeshInfo& M : P.meshes) maxf = std::max<int64_t>(maxf, M.nf);
    DBuf<double> At, part;
    DBuf<double2> W;
    At.alloc(maxf, s);
    part.alloc(2 * AREA_BLOCKS, s);
    W.alloc(P.nv, s);
    double2* U2 = reinterpret_cast<double2*>(U);
    for (size_t mi = 0; mi < P.meshes.size(); ++mi) {
        AreaMesh A(ctx, P, P.meshes[mi], U2, W.p, At.p, part.p);
        pgcp_area_result& r = out[mi];
        r = pgcp_area_result{0.0, 0.0, NAN, NAN, 0, PGCP_OK};
        const double before = A.mean_abs(U2);
        if (!std::isfinite(before)) {   // dropped mesh or folded input: left as it is
            r.status = PGCP_E_NUMERIC;
            continue;
        }
        double best = INFINITY;
        int evals = 0;
        const std::array<double, 2> x = nelder_mead(
            [&](const std::array<double, 2>& p) { return A.objective(disk, p[0], p[1]); }, {0.0, 0.0}, &best, &evals);
        r.param_re = x[0];
        r.param_im = x[1];
        r.before = before;
        r.after = best;
        r.evals = evals;
        if (!(best <= before)) {   // keep the identity (the search starts there)
            r.param_re = r.param_im = 0.0;
            r.after = before;
            continue;
        }
        A.map(disk, x[0], x[1], W.p);   // then copy the mesh's rows back into U
        PGCP_CUDA(cudaMemcpyAsync(U2 + P.meshes[mi].v0, W.p + P.meshes[mi].v0, P.meshes[mi].nv * sizeof(double2),
                                  cudaMemcpyDeviceToDevice, s));
        PGCP_CUDA(cudaStreamSynchronize(s));
    }
}

}  // namespace pgcp
