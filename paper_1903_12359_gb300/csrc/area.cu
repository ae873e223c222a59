// Area distortion and the Mobius area step (Section 6.2).
//
// d_area(T) = ln((A_f(T) / sum A_f) / (A(T) / sum A)) per face, A the surface
// triangle's area and A_f the parameter triangle's area: the planar signed
// area, or on the sphere the chordal triangle's area (negative when it faces
// inwards).  The step composes a mesh's map with the member of a Mobius
// family that minimises mean |d_area|: disk automorphisms
// (z - a) / (1 - conj(a) z); for a free boundary z / (1 - q z) (a Mobius map up
// to a similarity, which leaves normalised areas unchanged); on the sphere the
// ball automorphisms T_a(x) = ((1 - |a|^2)(x - a) - |x - a|^2 a) /
// (1 - 2<a, x> + |a|^2 |x|^2) in Ahlfors' form (a conformal map of the sphere
// up to a rotation, which leaves chordal areas unchanged).  The search is Nelder-Mead
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

// T_a on points of R^3 (rows of 3 doubles)
__global__ void k_area_map3(const double* __restrict__ X, int64_t v0, int64_t nv, double ax, double ay, double az,
                            double* __restrict__ W) {
    const double aa = ax * ax + ay * ay + az * az;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        const double* x = X + 3 * (v0 + i);
        const double xa = x[0] * ax + x[1] * ay + x[2] * az;
        const double xx = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        const double dx = x[0] - ax, dy = x[1] - ay, dz = x[2] - az;
        const double dd = dx * dx + dy * dy + dz * dz;
        const double den = 1.0 - 2.0 * xa + aa * xx;
        double* w = W + 3 * (v0 + i);
        w[0] = ((1.0 - aa) * dx - dd * ax) / den;
        w[1] = ((1.0 - aa) * dy - dd * ay) / den;
        w[2] = ((1.0 - aa) * dz - dd * az) / den;
    }
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

// parameter area of face f: planar signed area (sph = 0, W as double2) or the
// chordal triangle's area with the sign of its orientation (sph = 1, rows of 3)
__device__ __forceinline__ double param_area(const int32_t* __restrict__ F, const double* __restrict__ W, int64_t f,
                                             int sph) {
    if (!sph) {
        const double2* W2 = reinterpret_cast<const double2*>(W);
        const double2 a = W2[F[3 * f]], b = W2[F[3 * f + 1]], c = W2[F[3 * f + 2]];
        return 0.5 * ((b.x - a.x) * (c.y - a.y) - (b.y - a.y) * (c.x - a.x));
    }
    const double* a = W + 3 * (int64_t)F[3 * f];
    const double* b = W + 3 * (int64_t)F[3 * f + 1];
    const double* c = W + 3 * (int64_t)F[3 * f + 2];
    const double e1x = b[0] - a[0], e1y = b[1] - a[1], e1z = b[2] - a[2];
    const double e2x = c[0] - a[0], e2y = c[1] - a[1], e2z = c[2] - a[2];
    const double cx = e1y * e2z - e1z * e2y, cy = e1z * e2x - e1x * e2z, cz = e1x * e2y - e1y * e2x;
    const double ar = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
    return cx * (a[0] + b[0] + c[0]) + cy * (a[1] + b[1] + c[1]) + cz * (a[2] + b[2] + c[2]) > 0.0 ? ar : -ar;
}

// pass 1: sum of the parameter areas and the count of non-positive or non-finite ones
__global__ void __launch_bounds__(AREA_THREADS) k_area_pass1(const int32_t* __restrict__ F, const double* __restrict__ W,
                                                             int sph, int64_t f0, int64_t nf, double* __restrict__ part) {
    double s = 0.0, bad = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nf; t += (int64_t)gridDim.x * blockDim.x) {
        const double af = param_area(F, W, f0 + t, sph);
        if (!(af > 0.0) || !isfinite(af)) bad += 1.0;
        else s += af;
    }
    block_sum2(s, bad, part);
}

// pass 2: sum of |ln(A_f / A) - c| with c = ln(sum A_f / sum A)
__global__ void __launch_bounds__(AREA_THREADS) k_area_pass2(const int32_t* __restrict__ F, const double* __restrict__ W,
                                                             int sph, const double* __restrict__ At, int64_t f0,
                                                             int64_t nf, double c, double* __restrict__ part) {
    double s = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nf; t += (int64_t)gridDim.x * blockDim.x)
        s += fabs(log(param_area(F, W, f0 + t, sph) / At[t]) - c);
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
    const double* U;   // [nv_total * dim], dim = 2 (planar) or 3 (sphere)
    double* W;
    double* At;
    double* part;
    int sph;
    std::vector<double> h;
    double sum_at = 0.0;

    AreaMesh(pgcp_ctx* c, const Part& p, const MeshInfo& m, const double* u, double* w, double* at, double* pt)
        : ctx(c), P(p), M(m), U(u), W(w), At(at), part(pt), sph(p.closed ? 1 : 0), h(2 * AREA_BLOCKS) {
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
    double mean_abs(const double* X) {
        const unsigned g = grid_for(M.nf);
        { k_area_pass1<<<g, AREA_THREADS, 0, ctx->stream>>>(P.F.p, X, sph, M.f0, M.nf, part); ::pgcp::note_launch(); }
        const std::array<double, 2> s1 = fetch(g);
        if (s1[1] > 0.0 || !(s1[0] > 0.0) || !std::isfinite(s1[0])) return INFINITY;
        const double c = std::log(s1[0] / sum_at);
        { k_area_pass2<<<g, AREA_THREADS, 0, ctx->stream>>>(P.F.p, X, sph, At, M.f0, M.nf, c, part); ::pgcp::note_launch(); }
        const double m = fetch(g)[0] / (double)M.nf;
        return std::isfinite(m) ? m : INFINITY;
    }

    // family member with parameter x applied to the mesh's rows of U, into dst
    // (planar: disk = 1 automorphisms, 0 free; sphere: T_a with a = x)
    void map(int disk, const double* x, double* dst) {
        if (sph)
            k_area_map3<<<grid_for(M.nv), AREA_THREADS, 0, ctx->stream>>>(U, M.v0, M.nv, x[0], x[1], x[2], dst);
        else
            k_area_map<<<grid_for(M.nv), AREA_THREADS, 0, ctx->stream>>>(reinterpret_cast<const double2*>(U), M.v0, M.nv,
                                                                         disk, x[0], x[1], reinterpret_cast<double2*>(dst));
        ::pgcp::note_launch();
        PGCP_CUDA(cudaGetLastError());
    }

    double objective(int disk, const double* x) {
        if (sph && !(x[0] * x[0] + x[1] * x[1] + x[2] * x[2] < 1.0)) return INFINITY;
        if (!sph && disk && !(x[0] * x[0] + x[1] * x[1] < 1.0)) return INFINITY;
        map(disk, x, W);
        return mean_abs(W);
    }
};

// Nelder-Mead on R^N from x0 (the same steps and constants as the oracle's)
template <int N, typename Fn>
std::array<double, N> nelder_mead(Fn fun, std::array<double, N> x0, double* fbest, int* evals) {
    using PN = std::array<double, N>;
    PN pts[N + 1];
    double val[N + 1];
    pts[0] = x0;
    for (int i = 0; i < N; ++i) {
        pts[i + 1] = x0;
        pts[i + 1][i] += NM_STEP;
    }
    for (int i = 0; i <= N; ++i) val[i] = fun(pts[i]);
    int n = N + 1;
    const int w = N;   // the worst after sorting
    auto lin = [](const PN& a, const PN& b, double t) {
        PN r;
        for (int d = 0; d < N; ++d) r[d] = a[d] + t * (b[d] - a[d]);
        return r;
    };
    for (int it = 0; it < NM_MAXIT; ++it) {
        int ord[N + 1];
        for (int i = 0; i <= N; ++i) ord[i] = i;
        std::stable_sort(ord, ord + N + 1, [&](int a, int b) { return val[a] < val[b]; });
        PN sp[N + 1];
        double sv[N + 1];
        for (int i = 0; i <= N; ++i) {
            sp[i] = pts[ord[i]];
            sv[i] = val[ord[i]];
        }
        for (int i = 0; i <= N; ++i) {
            pts[i] = sp[i];
            val[i] = sv[i];
        }
        double size = 0.0;
        for (int i = 1; i <= N; ++i)
            for (int d = 0; d < N; ++d) size = std::max(size, std::fabs(pts[i][d] - pts[0][d]));
        if (std::isfinite(val[w]) && val[w] - val[0] <= NM_FTOL && size <= NM_XTOL) break;
        PN c = pts[0];   // centroid of the N best
        for (int i = 1; i < N; ++i)
            for (int d = 0; d < N; ++d) c[d] = c[d] + pts[i][d];
        for (int d = 0; d < N; ++d) c[d] = c[d] / N;
        const PN xr = lin(c, pts[w], -1.0);   // reflection c + (c - worst)
        const double fr = fun(xr);
        ++n;
        if (fr < val[0]) {
            const PN xe = lin(c, pts[w], -2.0);
            const double fe = fun(xe);
            ++n;
            if (fe < fr) {
                pts[w] = xe;
                val[w] = fe;
            } else {
                pts[w] = xr;
                val[w] = fr;
            }
        } else if (fr < val[w - 1]) {
            pts[w] = xr;
            val[w] = fr;
        } else {
            const PN xc = fr < val[w] ? lin(c, xr, 0.5) : lin(c, pts[w], 0.5);
            const double fc = fun(xc);
            ++n;
            if (fc < std::min(fr, val[w])) {
                pts[w] = xc;
                val[w] = fc;
            } else {
                for (int i = 1; i <= N; ++i) {
                    pts[i] = lin(pts[0], pts[i], 0.5);
                    val[i] = fun(pts[i]);
                    ++n;
                }
            }
        }
    }
    int best = 0;
    for (int i = 1; i <= N; ++i)
        if (val[i] < val[best]) best = i;
    *fbest = val[best];
    *evals = n;
    return pts[best];
}

}  // namespace

void area_distortion(pgcp_ctx* ctx, const Part& P, const double* U, double* mean_abs) {
    cudaStream_t s = ctx->stream;
    int64_t maxf = 1;
    for (const MeshInfo& M : P.meshes) maxf = std::max<int64_t>(maxf, M.nf);
    DBuf<double> At, part;
    At.alloc(maxf, s);
    part.alloc(2 * AREA_BLOCKS, s);
    for (size_t mi = 0; mi < P.meshes.size(); ++mi) {
        AreaMesh A(ctx, P, P.meshes[mi], U, nullptr, At.p, part.p);
        const double m = A.mean_abs(U);
        mean_abs[mi] = std::isfinite(m) ? m : NAN;
    }
}

void area_mobius(pgcp_ctx* ctx, const Part& P, double* U, int variant, pgcp_area_result* out) {
    if (P.closed ? variant != PGCP_SPHERE : (variant != PGCP_DISK && variant != PGCP_FREE))
        fail(PGCP_E_ARG, P.closed ? "Mobius area step: a closed part takes variant SPHERE"
                                  : "Mobius area step: an open part takes variant DISK or FREE");
    const int disk = variant == PGCP_DISK;
    const int dim = P.closed ? 3 : 2;
    cudaStream_t s = ctx->stream;
    int64_t maxf = 1;
    for (const MeshInfo& M : P.meshes) maxf = std::max<int64_t>(maxf, M.nf);
    DBuf<double> At, part, W;
    At.alloc(maxf, s);
    part.alloc(2 * AREA_BLOCKS, s);
    W.alloc(dim * P.nv, s);
    for (size_t mi = 0; mi < P.meshes.size(); ++mi) {
        const MeshInfo& M = P.meshes[mi];
        AreaMesh A(ctx, P, M, U, W.p, At.p, part.p);
        pgcp_area_result& r = out[mi];
        r = pgcp_area_result{{0.0, 0.0, 0.0}, NAN, NAN, 0, PGCP_OK};
        const double before = A.mean_abs(U);
        if (!std::isfinite(before)) {   // dropped mesh or folded input: left as it is
            r.status = PGCP_E_NUMERIC;
            continue;
        }
        double best = INFINITY, x[3] = {0.0, 0.0, 0.0};
        int evals = 0;
        if (dim == 3) {
            const std::array<double, 3> b = nelder_mead<3>(
                [&](const std::array<double, 3>& p) { return A.objective(disk, p.data()); }, {0.0, 0.0, 0.0}, &best,
                &evals);
            for (int d = 0; d < 3; ++d) x[d] = b[d];
        } else {
            const std::array<double, 2> b = nelder_mead<2>(
                [&](const std::array<double, 2>& p) { return A.objective(disk, p.data()); }, {0.0, 0.0}, &best, &evals);
            x[0] = b[0];
            x[1] = b[1];
        }
        r.before = before;
        r.evals = evals;
        if (!(best <= before)) {   // keep the identity (the search starts there)
            r.after = before;
            continue;
        }
        r.param[0] = x[0];
        r.param[1] = x[1];
        r.param[2] = x[2];
        r.after = best;
        A.map(disk, x, W.p);   // then copy the mesh's rows back into U
        PGCP_CUDA(cudaMemcpyAsync(U + dim * M.v0, W.p + dim * M.v0, dim * M.nv * sizeof(double),
                                  cudaMemcpyDeviceToDevice, s));
        PGCP_CUDA(cudaStreamSynchronize(s));
    }
}

}  // namespace pgcp
