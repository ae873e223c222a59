// Batched Jacobi-preconditioned CG over all pieces (Sections 4.2 and 4.5).
//
// Both solve stages share one persistent cooperative kernel:
//   * Laplace (final solve, Section 4.5): L u = 0 on interior rows with the
//     welded boundary fixed; x and y are two independent right-hand sides.
//   * DNCP (Section 4.2): ((L (+) L) - M) [x; y] = 0 with two pinned vertices;
//     M couples x and y on boundary rows: for boundary row i with loop
//     neighbours prev/next,  (Q u)_x = (L x)_i - (y_next - y_prev)/2,
//                            (Q u)_y = (L y)_i + (x_next - x_prev)/2,
//     and x, y share one CG (one alpha, beta per piece).
// Fixed rows (Dirichlet boundary or pins) have inverse diagonal 0: their
// search directions stay 0 and their residual is never counted.
//
// Work is a list of row tiles, each inside one piece, so every tile has one
// piece's scalars and ends with one atomic per dot product.  Per iteration:
//   phase 1: beta = rz_k / rz_{k-1};  z = D^-1 r;  p = z + beta p;
//            q = A z + beta q  (= A p);  <p, q>
//   grid sync
//   phase 2: alpha = rz_k / <p, q>;  x += alpha p;  r -= alpha q;
//            <r, D^-1 r>,  <r, r>
//   grid sync
// A piece (and for Laplace each coordinate) stops when <r, r> <= tol^2 <b, b>;
// its tiles are then skipped.  Scalar accumulators rotate over 3 slots, so no
// extra syncs are needed to reset them.
//
// Precision: FP64, or FP32 inner solves (FP32 SpMV and vectors, per-thread
// FP32 partial sums reduced in FP64) inside FP64 iterative refinement:
// r64 = -A64 x64 is computed in FP64 from FP64 matrix values, the FP32 solve
// returns a correction, x64 += d.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "pgcp_internal.h"

namespace cg = cooperative_groups;

namespace pgcp {

namespace {

template <typename T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };

struct Tile {
    int32_t seg, lo, hi, pad;
};

template <typename T>
struct PcgArgs {
    int64_t n;
    const int32_t* __restrict__ rp;
    const int32_t* __restrict__ col;
    const T* __restrict__ val;
    const T* __restrict__ dinv;
    const int2* __restrict__ nb;   // DNCP only
    typename V2<T>::t* x;
    typename V2<T>::t* r;
    typename V2<T>::t* p;
    typename V2<T>::t* q;
    const Tile* __restrict__ tiles;
    int32_t ntiles;
    int32_t nseg;
    double* RZ;      // [3][2 nseg]
    double* RR;      // [3][2 nseg]
    double* PQ;      // [2][2 nseg]
    unsigned int* ACT;   // [3]
    const double* __restrict__ THR;   // [2 nseg] convergence thresholds on <r, r>
    int32_t* iters;  // [nseg]
    int32_t* out_iters;   // [1] iterations run
    int32_t max_iters;
    int32_t dncp;
    int32_t lanes;   // lanes per row in the SpMV (4, 8, 16 or 32)
};

template <typename T>
__device__ __forceinline__ typename V2<T>::t ld2(const typename V2<T>::t* a, int64_t i) { return a[i]; }

__device__ __forceinline__ bool col_done(const double* RR, const double* THR, int nseg, int seg, int c, bool dncp) {
    if (dncp) return RR[2 * seg] + RR[2 * seg + 1] <= THR[2 * seg] + THR[2 * seg + 1];
    return RR[2 * seg + c] <= THR[2 * seg + c];
}

template <typename T, int LANES>
__device__ void phase1_tile(const PcgArgs<T>& a, const Tile& t, int k, double* red, unsigned& act_local) {
    using T2 = typename V2<T>::t;
    const int nseg = a.nseg;
    const double* RRk = a.RR + (k % 3) * 2 * nseg;
    const double* RZk = a.RZ + (k % 3) * 2 * nseg;
    const double* RZm = a.RZ + ((k + 2) % 3) * 2 * nseg;
    const int s = t.seg;
    bool d0 = col_done(RRk, a.THR, nseg, s, 0, a.dncp);
    bool d1 = col_done(RRk, a.THR, nseg, s, 1, a.dncp);
    if (d0 && d1) return;
    if (threadIdx.x == 0) {
        act_local += 1;
        atomicMax(&a.iters[s], k + 1);
    }
    T beta0 = 0, beta1 = 0;
    if (k > 0) {
        if (a.dncp) {
            double num = RZk[2 * s] + RZk[2 * s + 1], den = RZm[2 * s] + RZm[2 * s + 1];
            beta0 = beta1 = (T)(den != 0.0 ? num / den : 0.0);
        } else {
            beta0 = (T)(RZm[2 * s] != 0.0 ? RZk[2 * s] / RZm[2 * s] : 0.0);
            beta1 = (T)(RZm[2 * s + 1] != 0.0 ? RZk[2 * s + 1] / RZm[2 * s + 1] : 0.0);
        }
    }
    const int lane_g = threadIdx.x & (LANES - 1);
    const int group = threadIdx.x / LANES;
    const int ngroups = blockDim.x / LANES;
    T acc0 = 0, acc1 = 0;   // <p, q> partials (group leaders)
    // every lane runs the same number of rounds, so the group shuffles are safe
    for (int base = t.lo; base < t.hi; base += ngroups) {
        const int row = base + group;
        const bool valid = row < t.hi;
        const T di = valid ? a.dinv[row] : (T)0;
        const bool live = di != (T)0;   // fixed rows and the tail do no work
        T w0 = 0, w1 = 0;
        if (live) {
            const int b = a.rp[row], e = a.rp[row + 1];
            for (int j = b + lane_g; j < e; j += LANES) {
                const int c = a.col[j];
                const T v = a.val[j];
                const T dc = a.dinv[c];
                const T2 rc = a.r[c];
                w0 += v * (dc * rc.x);
                w1 += v * (dc * rc.y);
            }
        }
#pragma unroll
        for (int o = LANES / 2; o > 0; o >>= 1) {
            w0 += __shfl_xor_sync(0xffffffffu, w0, o, LANES);
            w1 += __shfl_xor_sync(0xffffffffu, w1, o, LANES);
        }
        if (live && lane_g == 0) {
            if (a.dncp) {
                const int2 pn = a.nb[row];
                if (pn.x >= 0) {
                    const T2 rp_ = a.r[pn.x], rn_ = a.r[pn.y];
                    const T dp = a.dinv[pn.x], dn = a.dinv[pn.y];
                    w0 -= (T)0.5 * (dn * rn_.y - dp * rp_.y);
                    w1 += (T)0.5 * (dn * rn_.x - dp * rp_.x);
                }
            }
            const T2 ri = a.r[row];
            T2 pi = a.p[row], qi = a.q[row];
            if (!d0) {
                pi.x = di * ri.x + beta0 * pi.x;
                qi.x = w0 + beta0 * qi.x;
                acc0 += pi.x * qi.x;
            }
            if (!d1) {
                pi.y = di * ri.y + beta1 * pi.y;
                qi.y = w1 + beta1 * qi.y;
                acc1 += pi.y * qi.y;
            }
            a.p[row] = pi;
            a.q[row] = qi;
        }
    }
    // block reduction -> one atomic per value
    double v0 = (double)acc0, v1 = (double)acc1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) {
        red[2 * warp] = v0;
        red[2 * warp + 1] = v1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0, s1 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s0 += red[2 * w];
            s1 += red[2 * w + 1];
        }
        double* PQk = a.PQ + (k % 2) * 2 * nseg;
        atomicAdd(&PQk[2 * s], s0);
        atomicAdd(&PQk[2 * s + 1], s1);
    }
}

template <typename T>
__device__ void phase2_tile(const PcgArgs<T>& a, const Tile& t, int k, double* red) {
    using T2 = typename V2<T>::t;
    const int nseg = a.nseg;
    const double* RRk = a.RR + (k % 3) * 2 * nseg;
    const double* RZk = a.RZ + (k % 3) * 2 * nseg;
    const double* PQk = a.PQ + (k % 2) * 2 * nseg;
    const int s = t.seg;
    bool d0 = col_done(RRk, a.THR, nseg, s, 0, a.dncp);
    bool d1 = col_done(RRk, a.THR, nseg, s, 1, a.dncp);
    if (d0 && d1) return;
    T al0 = 0, al1 = 0;
    if (a.dncp) {
        double den = PQk[2 * s] + PQk[2 * s + 1];
        al0 = al1 = (T)(den != 0.0 ? (RZk[2 * s] + RZk[2 * s + 1]) / den : 0.0);
    } else {
        if (!d0) al0 = (T)(PQk[2 * s] != 0.0 ? RZk[2 * s] / PQk[2 * s] : 0.0);
        if (!d1) al1 = (T)(PQk[2 * s + 1] != 0.0 ? RZk[2 * s + 1] / PQk[2 * s + 1] : 0.0);
    }
    T rz0 = 0, rz1 = 0, rr0 = 0, rr1 = 0;
    for (int row = t.lo + threadIdx.x; row < t.hi; row += blockDim.x) {
        const T di = a.dinv[row];
        if (di == (T)0) continue;
        T2 xi = a.x[row], ri = a.r[row];
        const T2 pi = a.p[row], qi = a.q[row];
        xi.x += al0 * pi.x;
        xi.y += al1 * pi.y;
        ri.x -= al0 * qi.x;
        ri.y -= al1 * qi.y;
        a.x[row] = xi;
        a.r[row] = ri;
        rz0 += ri.x * (di * ri.x);
        rz1 += ri.y * (di * ri.y);
        rr0 += ri.x * ri.x;
        rr1 += ri.y * ri.y;
    }
    double v[4] = {(double)rz0, (double)rz1, (double)rr0, (double)rr1};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0)
        for (int i = 0; i < 4; ++i) red[4 * warp + i] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum[4] = {0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int i = 0; i < 4; ++i) sum[i] += red[4 * w + i];
        double* RZn = a.RZ + ((k + 1) % 3) * 2 * nseg;
        double* RRn = a.RR + ((k + 1) % 3) * 2 * nseg;
        atomicAdd(&RZn[2 * s], sum[0]);
        atomicAdd(&RZn[2 * s + 1], sum[1]);
        atomicAdd(&RRn[2 * s], sum[2]);
        atomicAdd(&RRn[2 * s + 1], sum[3]);
    }
}

template <typename T, int LANES>
__global__ void __launch_bounds__(256) k_pcg(PcgArgs<T> a) {
    cg::grid_group grid = cg::this_grid();
    __shared__ double red[4 * 8];
    __shared__ unsigned act_s;
    const int nseg = a.nseg;
    int k = 0;
    for (; k < a.max_iters; ++k) {
        // ---- phase 1
        if (threadIdx.x == 0) act_s = 0;
        if (blockIdx.x == 0) {   // reset slots for later phases (see header)
            double* RZz = a.RZ + ((k + 1) % 3) * 2 * nseg;
            double* RRz = a.RR + ((k + 1) % 3) * 2 * nseg;
            for (int i = threadIdx.x; i < 2 * nseg; i += blockDim.x) {
                RZz[i] = 0.0;
                RRz[i] = 0.0;
            }
        }
        unsigned act_local = 0;
        for (int ti = blockIdx.x; ti < a.ntiles; ti += gridDim.x) phase1_tile<T, LANES>(a, a.tiles[ti], k, red, act_local);
        if (threadIdx.x == 0 && act_local) atomicAdd(&a.ACT[k % 3], act_local);
        grid.sync();
        // ---- phase 2
        if (blockIdx.x == 0) {
            double* PQz = a.PQ + ((k + 1) % 2) * 2 * nseg;
            for (int i = threadIdx.x; i < 2 * nseg; i += blockDim.x) PQz[i] = 0.0;
            if (threadIdx.x == 0) a.ACT[(k + 1) % 3] = 0;
        }
        for (int ti = blockIdx.x; ti < a.ntiles; ti += gridDim.x) phase2_tile<T>(a, a.tiles[ti], k, red);
        grid.sync();
        const unsigned act = *(volatile unsigned*)&a.ACT[k % 3];
        if (act == 0) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.out_iters[0] = k;
}

// ---------------------------------------------------------------- helpers

// Block sum of 4 doubles; thread 0 adds them to dst[0..3] (any may be null).
__device__ void block_add4(double v0, double v1, double v2, double v3, double* d0, double* d1, double* d2,
                           double* d3) {
    __shared__ double red[4 * 32];
    double v[4] = {v0, v1, v2, v3};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0)
        for (int i = 0; i < 4; ++i) red[4 * warp + i] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum[4] = {0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int i = 0; i < 4; ++i) sum[i] += red[4 * w + i];
        if (d0) atomicAdd(d0, sum[0]);
        if (d1) atomicAdd(d1, sum[1]);
        if (d2) atomicAdd(d2, sum[2]);
        if (d3) atomicAdd(d3, sum[3]);
    }
}

// One block per tile: r = -(A x) on free rows (0 on fixed rows), and <r, r>
// (and <r, D^-1 r>) per (piece, coordinate).  only_fixed: use x only at fixed
// columns, which gives the right-hand side b of the free unknowns.
template <typename TM, typename TX>
__global__ void k_residual(const Tile* __restrict__ tiles, const int32_t* __restrict__ rp,
                           const int32_t* __restrict__ col, const TM* __restrict__ val,
                           const double* __restrict__ dinv64, const int2* __restrict__ nb, int dncp,
                           const TX* __restrict__ x, int only_fixed, double2* __restrict__ r_out,
                           double* __restrict__ RR, double* __restrict__ RZ) {
    const Tile t = tiles[blockIdx.x];
    double a0 = 0, a1 = 0, z0 = 0, z1 = 0;
    for (int i = t.lo + threadIdx.x; i < t.hi; i += blockDim.x) {
        const double di = dinv64[i];
        if (di == 0.0) {
            if (r_out) r_out[i] = make_double2(0.0, 0.0);
            continue;
        }
        double w0 = 0, w1 = 0;
        for (int j = rp[i]; j < rp[i + 1]; ++j) {
            int c = col[j];
            if (only_fixed && dinv64[c] != 0.0) continue;
            double v = (double)val[j];
            w0 += v * (double)x[c].x;
            w1 += v * (double)x[c].y;
        }
        if (dncp) {
            int2 pn = nb[i];
            if (pn.x >= 0) {
                bool up = !only_fixed || dinv64[pn.x] == 0.0, un = !only_fixed || dinv64[pn.y] == 0.0;
                double yp = up ? (double)x[pn.x].y : 0.0, yn = un ? (double)x[pn.y].y : 0.0;
                double xp = up ? (double)x[pn.x].x : 0.0, xn = un ? (double)x[pn.y].x : 0.0;
                w0 -= 0.5 * (yn - yp);
                w1 += 0.5 * (xn - xp);
            }
        }
        double r0 = -w0, r1 = -w1;
        if (r_out) r_out[i] = make_double2(r0, r1);
        a0 += r0 * r0;
        a1 += r1 * r1;
        z0 += r0 * (di * r0);
        z1 += r1 * (di * r1);
    }
    const int s = t.seg;
    block_add4(a0, a1, z0, z1, RR ? &RR[2 * s] : nullptr, RR ? &RR[2 * s + 1] : nullptr,
               RZ ? &RZ[2 * s] : nullptr, RZ ? &RZ[2 * s + 1] : nullptr);
}

// <b, b> and <b, D^-1 b> of an FP32 right-hand side, per (piece, coordinate).
__global__ void k_rhs_stats(const Tile* __restrict__ tiles, const float* __restrict__ dinv,
                            const float2* __restrict__ b, double* __restrict__ RR, double* __restrict__ RZ) {
    const Tile t = tiles[blockIdx.x];
    float a0 = 0, a1 = 0, z0 = 0, z1 = 0;
    for (int i = t.lo + threadIdx.x; i < t.hi; i += blockDim.x) {
        const float di = dinv[i];
        if (di == 0.f) continue;
        const float2 v = b[i];
        a0 += v.x * v.x;
        a1 += v.y * v.y;
        z0 += v.x * (di * v.x);
        z1 += v.y * (di * v.y);
    }
    const int s = t.seg;
    block_add4(a0, a1, z0, z1, &RR[2 * s], &RR[2 * s + 1], &RZ[2 * s], &RZ[2 * s + 1]);
}

__global__ void k_dinv(int64_t n, const double* __restrict__ diag, const uint8_t* __restrict__ fixed,
                       double* __restrict__ d64, float* __restrict__ d32) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = fixed[i] ? 0.0 : 1.0 / diag[i];
    d64[i] = d;
    d32[i] = (float)d;
}

__global__ void k_to_f32(int64_t n, const double2* __restrict__ a, float2* __restrict__ b, float2* __restrict__ zero1,
                         float2* __restrict__ zero2, float2* __restrict__ zero3) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
    zero1[i] = make_float2(0.f, 0.f);
    zero2[i] = make_float2(0.f, 0.f);
    zero3[i] = make_float2(0.f, 0.f);
}

__global__ void k_add_correction(int64_t n, const double* __restrict__ dinv64, const float2* __restrict__ d,
                                 double2* __restrict__ x) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || dinv64[i] == 0.0) return;
    x[i].x += (double)d[i].x;
    x[i].y += (double)d[i].y;
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, ceil_div(n, t)); }

template <typename T, int LANES>
void launch_pcg(pgcp_ctx* ctx, const PcgArgs<T>& a, int* grid_out) {
    int per_sm = 0;
    PGCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<T, LANES>, 256, 0));
    if (per_sm <= 0) fail(PGCP_E_CUDA, "PCG kernel cannot be resident");
    int grid = std::min<int>(per_sm * ctx->num_sms, a.ntiles);
    grid = std::max(grid, 1);
    *grid_out = grid;
    void* args[] = {(void*)&a};
    PGCP_CUDA(cudaLaunchCooperativeKernel((void*)k_pcg<T, LANES>, dim3(grid), dim3(256), args, 0, ctx->stream));
}

template <typename T>
void launch_pcg_lanes(pgcp_ctx* ctx, PcgArgs<T> a) {
    int grid = 0;
    switch (a.lanes) {
        case 4: launch_pcg<T, 4>(ctx, a, &grid); break;
        case 16: launch_pcg<T, 16>(ctx, a, &grid); break;
        case 32: launch_pcg<T, 32>(ctx, a, &grid); break;
        default: a.lanes = 8; launch_pcg<T, 8>(ctx, a, &grid); break;
    }
}

}  // namespace

// ---------------------------------------------------------------- solver driver

// Solve the batched system in place.  x holds the fixed values and the initial
// guess; fixed[i] = 1 marks fixed rows.
SolveResult pcg_solve(pgcp_ctx* ctx, Part& P, int dncp, const uint8_t* fixed, double2* x) {
    cudaStream_t s = ctx->stream;
    const pgcp_options& o = ctx->opt;
    const int64_t n = P.Nc;
    const int S = P.K;
    // tiles: rows of one piece, at most 2^log2 rows each
    int lg = o.block_rows_log2 > 0 ? o.block_rows_log2 : 11;
    const int64_t TR = 1ll << lg;
    std::vector<Tile> tiles;
    for (int i = 0; i < S; ++i)
        for (int64_t lo = P.voff[i]; lo < P.voff[i + 1]; lo += TR)
            tiles.push_back(Tile{i, (int32_t)lo, (int32_t)std::min<int64_t>(lo + TR, P.voff[i + 1]), 0});
    DBuf<Tile> d_tiles;
    d_tiles.alloc(tiles.size(), s);
    PGCP_CUDA(cudaMemcpyAsync(d_tiles.p, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, s));
    DBuf<double> dinv64;
    DBuf<float> dinv32;
    dinv64.alloc(n, s);
    dinv32.alloc(n, s);
    k_dinv<<<nblk(n), 256, 0, s>>>(n, P.diag64.p, fixed, dinv64.p, dinv32.p);
    // <b, b> per (piece, coordinate): b = -A x_fixed on free rows
    DBuf<double> BB, RRo, THR, RZ, RR, PQ;
    DBuf<unsigned int> ACT;
    DBuf<int32_t> iters, out_it;
    BB.alloc(2 * S, s);
    RRo.alloc(2 * S, s);
    THR.alloc(2 * S, s);
    RZ.alloc(3 * 2 * S, s);
    RR.alloc(3 * 2 * S, s);
    PQ.alloc(2 * 2 * S, s);
    ACT.alloc(3, s);
    iters.alloc(S, s);
    out_it.alloc(1, s);
    BB.zero();
    const unsigned nt = (unsigned)tiles.size();
    k_residual<double, double2><<<nt, 256, 0, s>>>(d_tiles.p, P.row_ptr.p, P.col.p, P.val64.p, dinv64.p, P.nb.p,
                                                  dncp, x, 1, nullptr, BB.p, nullptr);
    PGCP_CUDA(cudaGetLastError());
    std::vector<double> hBB(2 * S), hRR(2 * S), hTHR(2 * S);
    PGCP_CUDA(cudaMemcpyAsync(hBB.data(), BB.p, 2 * S * sizeof(double), cudaMemcpyDeviceToHost, s));
    PGCP_CUDA(cudaStreamSynchronize(s));
    SolveResult res;
    const double tol2 = o.tol * o.tol;
    auto relres_of = [&](const std::vector<double>& rr, bool* all_ok) {
        double worst = 0.0;
        bool ok = true;
        for (int i = 0; i < S; ++i) {
            for (int c = 0; c < 2; ++c) {
                double bb = hBB[2 * i + c], r = rr[2 * i + c];
                double rel = bb > 0 ? std::sqrt(r / bb) : (r > 0 ? INFINITY : 0.0);
                if (dncp) {
                    double b2 = hBB[2 * i] + hBB[2 * i + 1], r2 = rr[2 * i] + rr[2 * i + 1];
                    rel = b2 > 0 ? std::sqrt(r2 / b2) : (r2 > 0 ? INFINITY : 0.0);
                }
                if (!(rel <= o.tol)) ok = false;
                worst = std::max(worst, std::isfinite(rel) ? rel : 1e300);
            }
        }
        *all_ok = ok;
        return worst;
    };
    DBuf<double2> r64;
    r64.alloc(n, s);
    if (o.precision == PGCP_FP64) {
        // FP64 PCG, restarted from the true residual while recursion drift
        // leaves it above the tolerance
        DBuf<double2> p, q;
        p.alloc(n, s);
        q.alloc(n, s);
        for (int i = 0; i < 2 * S; ++i) hTHR[i] = tol2 * hBB[i];
        PGCP_CUDA(cudaMemcpyAsync(THR.p, hTHR.data(), 2 * S * sizeof(double), cudaMemcpyHostToDevice, s));
        for (int outer = 0; outer < std::max(1, o.max_refine); ++outer) {
            p.zero();
            q.zero();
            RZ.zero();
            RR.zero();
            PQ.zero();
            ACT.zero();
            iters.zero();
            k_residual<double, double2><<<nt, 256, 0, s>>>(d_tiles.p, P.row_ptr.p, P.col.p, P.val64.p, dinv64.p,
                                                          P.nb.p, dncp, x, 0, r64.p, RR.p, RZ.p);
            PGCP_CUDA(cudaMemcpyAsync(hRR.data(), RR.p, 2 * S * sizeof(double), cudaMemcpyDeviceToHost, s));
            PGCP_CUDA(cudaStreamSynchronize(s));
            bool ok = false;
            res.relres = relres_of(hRR, &ok);
            res.refine = outer;
            if (ok) return res;
            PcgArgs<double> a{n, P.row_ptr.p, P.col.p, P.val64.p, dinv64.p, P.nb.p, x, r64.p, p.p, q.p,
                              d_tiles.p, (int32_t)tiles.size(), S, RZ.p, RR.p, PQ.p, ACT.p, THR.p, iters.p,
                              out_it.p, o.max_iters, dncp, 8};
            launch_pcg_lanes<double>(ctx, a);
            int it = 0;
            PGCP_CUDA(cudaMemcpyAsync(&it, out_it.p, sizeof(int), cudaMemcpyDeviceToHost, s));
            PGCP_CUDA(cudaStreamSynchronize(s));
            res.iters += it;
        }
        RRo.zero();
        k_residual<double, double2><<<nt, 256, 0, s>>>(d_tiles.p, P.row_ptr.p, P.col.p, P.val64.p, dinv64.p,
                                                      P.nb.p, dncp, x, 0, nullptr, RRo.p, nullptr);
        PGCP_CUDA(cudaMemcpyAsync(hRR.data(), RRo.p, 2 * S * sizeof(double), cudaMemcpyDeviceToHost, s));
        PGCP_CUDA(cudaStreamSynchronize(s));
        bool ok = false;
        res.relres = relres_of(hRR, &ok);
        res.refine = std::max(1, o.max_refine);
        return res;
    }
    // ---- FP32 inner solves inside FP64 refinement
    DBuf<float2> b32, d32, p32, q32;
    b32.alloc(n, s);
    d32.alloc(n, s);
    p32.alloc(n, s);
    q32.alloc(n, s);
    const double itol2 = o.inner_tol * o.inner_tol;
    for (int outer = 0; outer < std::max(1, o.max_refine); ++outer) {
        RRo.zero();
        k_residual<double, double2><<<nt, 256, 0, s>>>(d_tiles.p, P.row_ptr.p, P.col.p, P.val64.p, dinv64.p,
                                                      P.nb.p, dncp, x, 0, r64.p, RRo.p, nullptr);
        PGCP_CUDA(cudaMemcpyAsync(hRR.data(), RRo.p, 2 * S * sizeof(double), cudaMemcpyDeviceToHost, s));
        PGCP_CUDA(cudaStreamSynchronize(s));
        bool ok = false;
        res.relres = relres_of(hRR, &ok);
        res.refine = outer;
        if (ok) return res;
        // inner solve on A32 d = r64: thresholds relative to this right-hand side;
        // pieces (coordinates) already converged are frozen
        for (int i = 0; i < S; ++i) {
            for (int c = 0; c < 2; ++c) {
                int j = 2 * i + c;
                bool conv;
                if (dncp) conv = hRR[2 * i] + hRR[2 * i + 1] <= tol2 * (hBB[2 * i] + hBB[2 * i + 1]);
                else conv = hRR[j] <= tol2 * hBB[j];
                hTHR[j] = conv ? INFINITY : std::max(itol2 * hRR[j], 0.25 * tol2 * hBB[j]);
            }
        }
        PGCP_CUDA(cudaMemcpyAsync(THR.p, hTHR.data(), 2 * S * sizeof(double), cudaMemcpyHostToDevice, s));
        k_to_f32<<<nblk(n), 256, 0, s>>>(n, r64.p, b32.p, d32.p, p32.p, q32.p);
        RZ.zero();
        RR.zero();
        PQ.zero();
        ACT.zero();
        iters.zero();
        // RZ0, RR0 of the FP32 right-hand side (x = 0 so r = b)
        k_rhs_stats<<<nt, 256, 0, s>>>(d_tiles.p, dinv32.p, b32.p, RR.p, RZ.p);
        PcgArgs<float> a{n, P.row_ptr.p, P.col.p, P.val32.p, dinv32.p, P.nb.p, d32.p, b32.p, p32.p, q32.p,
                         d_tiles.p, (int32_t)tiles.size(), S, RZ.p, RR.p, PQ.p, ACT.p, THR.p, iters.p, out_it.p,
                         o.max_iters, dncp, 8};
        launch_pcg_lanes<float>(ctx, a);
        int it = 0;
        PGCP_CUDA(cudaMemcpyAsync(&it, out_it.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        k_add_correction<<<nblk(n), 256, 0, s>>>(n, dinv64.p, d32.p, x);
        PGCP_CUDA(cudaStreamSynchronize(s));
        res.iters += it;
    }
    RRo.zero();
    k_residual<double, double2><<<nt, 256, 0, s>>>(d_tiles.p, P.row_ptr.p, P.col.p, P.val64.p, dinv64.p, P.nb.p,
                                                  dncp, x, 0, nullptr, RRo.p, nullptr);
    PGCP_CUDA(cudaMemcpyAsync(hRR.data(), RRo.p, 2 * S * sizeof(double), cudaMemcpyDeviceToHost, s));
    PGCP_CUDA(cudaStreamSynchronize(s));
    bool ok = false;
    res.relres = relres_of(hRR, &ok);
    res.refine = std::max(1, o.max_refine);
    return res;
}

}  // namespace pgcp
