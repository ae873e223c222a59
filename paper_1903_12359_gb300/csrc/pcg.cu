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
// This file holds the FP64 path (one kernel for the whole solve) and the
// solver driver.  The mixed-precision paths (FP32 or double-float inner solves
// inside FP64 iterative refinement: r64 = -A64 x64 computed in FP64 from FP64
// matrix values, the inner solve returns a correction, x64 += d) run the
// run-based kernel of pcg_df.cu.
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
    int32_t frows, fnnz;   // free rows of the tile and their stored entries
    int32_t pad2, pad3;
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
    typename V2<T>::t* z;   // D^-1 r, written in phase 2 (and by the set-up)
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
    int32_t lanes;   // threads per row in the SpMV (1, 2, 4 or 8)
    unsigned long long* work;   // [2] free rows and entries of the active tiles, summed over iterations
};

template <typename T>
__device__ __forceinline__ typename V2<T>::t ld2(const typename V2<T>::t* a, int64_t i) { return a[i]; }

__device__ __forceinline__ bool col_done(const double* RR, const double* THR, int nseg, int seg, int c, bool dncp) {
    if (dncp) return RR[2 * seg] + RR[2 * seg + 1] <= THR[2 * seg] + THR[2 * seg + 1];
    return RR[2 * seg + c] <= THR[2 * seg + c];
}

constexpr int PCG_THREADS = 512;

// Block-sum NV doubles; thread 0 receives the totals in out[].
template <int NV>
__device__ __forceinline__ void block_sum(double* v, double* red, double* out) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) red[NV * warp + i] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < NV; ++i) out[i] = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int i = 0; i < NV; ++i) out[i] += red[NV * w + i];
    }
}

// x != 0 without an FP64 compare (integer test of the bit pattern; -0 never occurs)
__device__ __forceinline__ bool nonzero(double x) { return __double_as_longlong(x) != 0; }
__device__ __forceinline__ bool nonzero(float x) { return __float_as_int(x) != 0; }

template <typename T, int LANES>
__device__ __forceinline__ void spmv_row(const PcgArgs<T>& a, int row, int lane_g, T& w0, T& w1) {
    using T2 = typename V2<T>::t;
    const int b = a.rp[row], e = a.rp[row + 1];
    for (int j = b + lane_g; j < e; j += LANES) {
        const int c = a.col[j];
        const T v = a.val[j];
        const T2 zc = a.z[c];
        w0 += v * zc.x;
        w1 += v * zc.y;
    }
}

template <typename T, int LANES>
__global__ void __launch_bounds__(PCG_THREADS) k_pcg(PcgArgs<T> a) {
    using T2 = typename V2<T>::t;
    cg::grid_group grid = cg::this_grid();
    __shared__ double red[4 * (PCG_THREADS / 32)];
    __shared__ double tot[4];
    __shared__ double sc[2];
    __shared__ int sflag[2];
    const int nseg = a.nseg;
    // this block's contiguous range of tiles
    const int tb = (int)(((int64_t)a.ntiles * blockIdx.x) / gridDim.x);
    const int te = (int)(((int64_t)a.ntiles * (blockIdx.x + 1)) / gridDim.x);
    const int lane_g = threadIdx.x & (LANES - 1);
    const int group = threadIdx.x / LANES;
    const int ngroups = blockDim.x / LANES;
    unsigned long long wrows = 0, wnnz = 0;
    int k = 0;
    for (; k < a.max_iters; ++k) {
        const double* RRk = a.RR + (k % 3) * 2 * nseg;
        const double* RZk = a.RZ + (k % 3) * 2 * nseg;
        const double* RZm = a.RZ + ((k + 2) % 3) * 2 * nseg;
        double* PQk = a.PQ + (k % 2) * 2 * nseg;
        // ---------------- phase 1: p = z + beta p, q = A z + beta q, <p, q>
        if (blockIdx.x == 0) {   // reset slots used two phases later (see header)
            double* RZz = a.RZ + ((k + 1) % 3) * 2 * nseg;
            double* RRz = a.RR + ((k + 1) % 3) * 2 * nseg;
            for (int i = threadIdx.x; i < 2 * nseg; i += blockDim.x) {
                RZz[i] = 0.0;
                RRz[i] = 0.0;
            }
        }
        int run_seg = -1;
        double run[2] = {0.0, 0.0};
        bool any = false;
        for (int ti = tb; ti < te; ++ti) {
            const Tile t = a.tiles[ti];
            const int s = t.seg;
            // the tile's scalars, computed once (FP64 divisions are expensive here)
            if (threadIdx.x == 0) {
                const bool d0 = col_done(RRk, a.THR, nseg, s, 0, a.dncp);
                const bool d1 = col_done(RRk, a.THR, nseg, s, 1, a.dncp);
                double b0 = 0.0, b1 = 0.0;
                if (k > 0) {
                    if (a.dncp) {
                        double num = RZk[2 * s] + RZk[2 * s + 1], den = RZm[2 * s] + RZm[2 * s + 1];
                        b0 = b1 = den != 0.0 ? num / den : 0.0;
                    } else {
                        b0 = RZm[2 * s] != 0.0 ? RZk[2 * s] / RZm[2 * s] : 0.0;
                        b1 = RZm[2 * s + 1] != 0.0 ? RZk[2 * s + 1] / RZm[2 * s + 1] : 0.0;
                    }
                }
                sc[0] = b0;
                sc[1] = b1;
                sflag[0] = d0;
                sflag[1] = d1;
            }
            __syncthreads();
            const bool d0 = sflag[0], d1 = sflag[1];
            const T beta0 = (T)sc[0], beta1 = (T)sc[1];
            if (d0 && d1) {
                __syncthreads();   // everyone has read the scalars before they change
                continue;
            }
            any = true;
            T acc0 = 0, acc1 = 0;
            for (int base = t.lo; base < t.hi; base += ngroups) {
                const int row = base + group;
                const bool valid = row < t.hi;
                const T di = valid ? a.dinv[row] : (T)0;
                const bool live = nonzero(di);
                T w0 = 0, w1 = 0;
                if (live) spmv_row<T, LANES>(a, row, lane_g, w0, w1);
                if (LANES > 1) {
#pragma unroll
                    for (int o = LANES / 2; o > 0; o >>= 1) {
                        w0 += __shfl_xor_sync(0xffffffffu, w0, o, LANES);
                        w1 += __shfl_xor_sync(0xffffffffu, w1, o, LANES);
                    }
                }
                if (live && lane_g == 0) {
                    if (a.dncp) {
                        const int2 pn = a.nb[row];
                        if (pn.x >= 0) {
                            const T2 zp = a.z[pn.x], zn = a.z[pn.y];
                            w0 -= (T)0.5 * (zn.y - zp.y);
                            w1 += (T)0.5 * (zn.x - zp.x);
                        }
                    }
                    const T2 zi = a.z[row];
                    T2 pi = a.p[row], qi = a.q[row];
                    if (!d0) {
                        pi.x = zi.x + beta0 * pi.x;
                        qi.x = w0 + beta0 * qi.x;
                        acc0 += pi.x * qi.x;
                    }
                    if (!d1) {
                        pi.y = zi.y + beta1 * pi.y;
                        qi.y = w1 + beta1 * qi.y;
                        acc1 += pi.y * qi.y;
                    }
                    a.p[row] = pi;
                    a.q[row] = qi;
                }
            }
            double v[2] = {(double)acc0, (double)acc1};
            block_sum<2>(v, red, tot);
            if (threadIdx.x == 0) {
                if (s != run_seg) {
                    if (run_seg >= 0) {
                        atomicAdd(&PQk[2 * run_seg], run[0]);
                        atomicAdd(&PQk[2 * run_seg + 1], run[1]);
                    }
                    run_seg = s;
                    run[0] = tot[0];
                    run[1] = tot[1];
                } else {
                    run[0] += tot[0];
                    run[1] += tot[1];
                }
                wrows += (unsigned long long)t.frows;
                wnnz += (unsigned long long)t.fnnz;
            }
        }
        if (threadIdx.x == 0) {
            if (run_seg >= 0) {
                atomicAdd(&PQk[2 * run_seg], run[0]);
                atomicAdd(&PQk[2 * run_seg + 1], run[1]);
            }
            if (any) *(volatile unsigned*)&a.ACT[k % 3] = 1u;
        }
        grid.sync();
        // ---------------- phase 2: x += alpha p, r -= alpha q, <r, z>, <r, r>
        if (blockIdx.x == 0) {
            double* PQz = a.PQ + ((k + 1) % 2) * 2 * nseg;
            for (int i = threadIdx.x; i < 2 * nseg; i += blockDim.x) PQz[i] = 0.0;
            if (threadIdx.x == 0) a.ACT[(k + 1) % 3] = 0;
        }
        double* RZn = a.RZ + ((k + 1) % 3) * 2 * nseg;
        double* RRn = a.RR + ((k + 1) % 3) * 2 * nseg;
        int run2_seg = -1;
        double run2[4] = {0, 0, 0, 0};
        for (int ti = tb; ti < te; ++ti) {
            const Tile t = a.tiles[ti];
            const int s = t.seg;
            if (threadIdx.x == 0) {
                const bool d0 = col_done(RRk, a.THR, nseg, s, 0, a.dncp);
                const bool d1 = col_done(RRk, a.THR, nseg, s, 1, a.dncp);
                double al0 = 0.0, al1 = 0.0;
                if (a.dncp) {
                    double den = PQk[2 * s] + PQk[2 * s + 1];
                    al0 = al1 = den != 0.0 ? (RZk[2 * s] + RZk[2 * s + 1]) / den : 0.0;
                } else {
                    if (!d0) al0 = PQk[2 * s] != 0.0 ? RZk[2 * s] / PQk[2 * s] : 0.0;
                    if (!d1) al1 = PQk[2 * s + 1] != 0.0 ? RZk[2 * s + 1] / PQk[2 * s + 1] : 0.0;
                }
                sc[0] = al0;
                sc[1] = al1;
                sflag[0] = d0 && d1;
            }
            __syncthreads();
            const T al0 = (T)sc[0], al1 = (T)sc[1];
            if (sflag[0]) {
                __syncthreads();
                continue;
            }
            T rz0 = 0, rz1 = 0, rr0 = 0, rr1 = 0;
            for (int row = t.lo + threadIdx.x; row < t.hi; row += blockDim.x) {
                const T di = a.dinv[row];
                if (!nonzero(di)) continue;
                T2 xi = a.x[row], ri = a.r[row];
                const T2 pi = a.p[row], qi = a.q[row];
                xi.x += al0 * pi.x;
                xi.y += al1 * pi.y;
                ri.x -= al0 * qi.x;
                ri.y -= al1 * qi.y;
                a.x[row] = xi;
                a.r[row] = ri;
                T2 zi;
                zi.x = di * ri.x;
                zi.y = di * ri.y;
                a.z[row] = zi;
                rz0 += ri.x * zi.x;
                rz1 += ri.y * zi.y;
                rr0 += ri.x * ri.x;
                rr1 += ri.y * ri.y;
            }
            double v[4] = {(double)rz0, (double)rz1, (double)rr0, (double)rr1};
            block_sum<4>(v, red, tot);
            if (threadIdx.x == 0) {
                if (s != run2_seg) {
                    if (run2_seg >= 0) {
                        atomicAdd(&RZn[2 * run2_seg], run2[0]);
                        atomicAdd(&RZn[2 * run2_seg + 1], run2[1]);
                        atomicAdd(&RRn[2 * run2_seg], run2[2]);
                        atomicAdd(&RRn[2 * run2_seg + 1], run2[3]);
                    }
                    run2_seg = s;
                    for (int i = 0; i < 4; ++i) run2[i] = tot[i];
                } else {
                    for (int i = 0; i < 4; ++i) run2[i] += tot[i];
                }
            }
        }
        if (threadIdx.x == 0 && run2_seg >= 0) {
            atomicAdd(&RZn[2 * run2_seg], run2[0]);
            atomicAdd(&RZn[2 * run2_seg + 1], run2[1]);
            atomicAdd(&RRn[2 * run2_seg], run2[2]);
            atomicAdd(&RRn[2 * run2_seg + 1], run2[3]);
        }
        grid.sync();
        const unsigned act = *(volatile unsigned*)&a.ACT[k % 3];
        if (act == 0) break;
    }
    if (threadIdx.x == 0) {
        if (wrows) atomicAdd(&a.work[0], wrows);
        if (wnnz) atomicAdd(&a.work[1], wnnz);
        if (blockIdx.x == 0) a.out_iters[0] = k;
    }
}

// ---------------------------------------------------------------- helpers

// Block sum of 4 doubles; thread 0 adds them to dst[0..3] (any may be null).
// Block sums of four values; thread 0 adds them to d0..d3 (atomics), or, with
// part, stores them at part[4 * blockIdx.x ...] for an ordered sum later.
__device__ void block_add4(double v0, double v1, double v2, double v3, double* d0, double* d1, double* d2,
                           double* d3, double* part = nullptr) {
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
        if (part) {
            for (int i = 0; i < 4; ++i) part[4 * blockIdx.x + i] = sum[i];
            return;
        }
        if (d0) atomicAdd(d0, sum[0]);
        if (d1) atomicAdd(d1, sum[1]);
        if (d2) atomicAdd(d2, sum[2]);
        if (d3) atomicAdd(d3, sum[3]);
    }
}

// One block per tile: r = -(A x) on free rows (0 on fixed rows), and <r, r>
// (and <r, D^-1 r>) per (piece, coordinate).  only_fixed: use x only at fixed
// columns, which gives the right-hand side b of the free unknowns.  part:
// per-tile sums instead of atomics (deterministic mode).
template <typename TM, typename TX>
__global__ void k_residual(const Tile* __restrict__ tiles, const int32_t* __restrict__ rp,
                           const int32_t* __restrict__ col, const TM* __restrict__ val,
                           const double* __restrict__ dinv64, const int2* __restrict__ nb, int dncp,
                           const TX* __restrict__ x, int only_fixed, double2* __restrict__ r_out,
                           double* __restrict__ RR, double* __restrict__ RZ, double2* __restrict__ z_out = nullptr,
                           double* __restrict__ part = nullptr) {
    const Tile t = tiles[blockIdx.x];
    double a0 = 0, a1 = 0, z0 = 0, z1 = 0;
    for (int i = t.lo + threadIdx.x; i < t.hi; i += blockDim.x) {
        const double di = dinv64[i];
        if (di == 0.0) {
            if (r_out) r_out[i] = make_double2(0.0, 0.0);
            if (z_out) z_out[i] = make_double2(0.0, 0.0);
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
        if (z_out) z_out[i] = make_double2(di * r0, di * r1);
        a0 += r0 * r0;
        a1 += r1 * r1;
        z0 += r0 * (di * r0);
        z1 += r1 * (di * r1);
    }
    const int s = t.seg;
    block_add4(a0, a1, z0, z1, RR ? &RR[2 * s] : nullptr, RR ? &RR[2 * s + 1] : nullptr,
               RZ ? &RZ[2 * s] : nullptr, RZ ? &RZ[2 * s + 1] : nullptr, part);
}

__global__ void k_tile_stats(Tile* tiles, const int32_t* __restrict__ rp, const uint8_t* __restrict__ fixed) {
    Tile& t = tiles[blockIdx.x];
    int fr = 0, fz = 0;
    for (int i = t.lo + threadIdx.x; i < t.hi; i += blockDim.x)
        if (!fixed[i]) {
            fr += 1;
            fz += rp[i + 1] - rp[i];
        }
    for (int o = 16; o > 0; o >>= 1) {
        fr += __shfl_xor_sync(0xffffffffu, fr, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
    }
    __shared__ int sh[2 * 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sh[2 * w] = fr;
        sh[2 * w + 1] = fz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0, b = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            a += sh[2 * i];
            b += sh[2 * i + 1];
        }
        t.frows = a;
        t.fnnz = b;
    }
}

__global__ void k_dinv(int64_t n, const double* __restrict__ diag, const uint8_t* __restrict__ fixed,
                       double* __restrict__ d64, float* __restrict__ d32) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = fixed[i] ? 0.0 : 1.0 / diag[i];
    d64[i] = d;
    d32[i] = (float)d;
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, ceil_div(n, t)); }

template <typename T, int LANES>
void launch_pcg(pgcp_ctx* ctx, const PcgArgs<T>& a, int* grid_out) {
    int per_sm = 0;
    PGCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<T, LANES>, PCG_THREADS, 0));
    if (per_sm <= 0) fail(PGCP_E_CUDA, "PCG kernel cannot be resident");
    int grid = std::min<int>(per_sm * ctx->num_sms, a.ntiles);
    grid = std::max(grid, 1);
    *grid_out = grid;
    void* args[] = {(void*)&a};
    { PGCP_CUDA(cudaLaunchCooperativeKernel((void*)k_pcg<T, LANES>, dim3(grid), dim3(PCG_THREADS), args, 0, ctx->stream)); ::pgcp::note_launch(); }
}

// Launch the persistent PCG kernel; its duration (CUDA events on the context
// stream) and algorithmic bytes go to the part's statistics.
template <typename T>
void launch_pcg_lanes(pgcp_ctx* ctx, Part& P, PcgArgs<T> a) {
    int grid = 0;
    EventPair ev;
    PGCP_CUDA(cudaMemsetAsync(a.work, 0, 2 * sizeof(unsigned long long), ctx->stream));
    PGCP_CUDA(cudaEventRecord(ev.a, ctx->stream));
    switch (a.lanes) {
        case 2: launch_pcg<T, 2>(ctx, a, &grid); break;
        case 4: launch_pcg<T, 4>(ctx, a, &grid); break;
        case 8: launch_pcg<T, 8>(ctx, a, &grid); break;
        default: a.lanes = 1; launch_pcg<T, 1>(ctx, a, &grid); break;
    }
    PGCP_CUDA(cudaEventRecord(ev.b, ctx->stream));
    unsigned long long w[2] = {0, 0};
    PGCP_CUDA(cudaMemcpyAsync(w, a.work, sizeof(w), cudaMemcpyDeviceToHost, ctx->stream));
    PGCP_CUDA(cudaEventSynchronize(ev.b));
    float ms = 0.f;
    PGCP_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
    const double Tb = (double)sizeof(T);
    P.stats.pcg_ms += ms;
    // per free row and iteration: row pointer 4 B, inverse diagonal T (phase 2),
    // vectors 2T each: z read (1) and write (1), r r/w (2), p r/w + read (3),
    // q r/w + read (3), x r/w (2) -> 24T; per stored entry: column 4 B + value T
    P.stats.pcg_bytes += (double)w[0] * (4.0 + 19.0 * Tb) + (double)w[1] * (4.0 + Tb);
    P.stats.pcg_bytes_touched += (double)w[0] * (4.0 + 25.0 * Tb) + (double)w[1] * (4.0 + Tb);
    P.stats.pcg_launches += 1;
}

}  // namespace

// ---------------------------------------------------------------- solver driver

// Solve the batched system in place.  x holds the fixed values and the initial
// guess; fixed[i] = 1 marks fixed rows.
SolveResult pcg_solve(pgcp_ctx* ctx, Part& P, int dncp, const uint8_t* fixed, double2* x) {
    cudaStream_t s = ctx->stream;
    pgcp_options o = ctx->opt;
    if (dncp) o.precision = o.local_precision;
    if (o.deterministic != 0 && o.deterministic != 1) fail(PGCP_E_ARG, "deterministic must be 0 or 1");
    if (o.deterministic && o.precision == PGCP_FP64)
        fail(PGCP_E_ARG, "deterministic mode needs a mixed-precision solver (FP32_REFINED or DF64_REFINED)");
    const int64_t n = P.Nc;
    const int S = P.K;
    // tiles: rows of one piece, at most 2^log2 rows each
    int lg = o.block_rows_log2 > 0 ? o.block_rows_log2 : 9;
    const int64_t TR = 1ll << lg;
    std::vector<Tile> tiles;
    for (int i = 0; i < S; ++i)
        for (int64_t lo = P.voff[i]; lo < P.voff[i + 1]; lo += TR)
            tiles.push_back(Tile{i, (int32_t)lo, (int32_t)std::min<int64_t>(lo + TR, P.voff[i + 1]), 0, 0, 0, 0, 0});
    DBuf<Tile> d_tiles;
    d_tiles.alloc(tiles.size(), s);
    PGCP_CUDA(cudaMemcpyAsync(d_tiles.p, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, s));
    DBuf<double> dinv64;
    DBuf<float> dinv32;
    dinv64.alloc(n, s);
    dinv32.alloc(n, s);
    { k_dinv<<<nblk(n), 256, 0, s>>>(n, P.diag64.p, fixed, dinv64.p, dinv32.p); ::pgcp::note_launch(); }
    { k_tile_stats<<<(unsigned)tiles.size(), 256, 0, s>>>(d_tiles.p, P.row_ptr.p, fixed); ::pgcp::note_launch(); }
    DBuf<unsigned long long> work;
    work.alloc(2, s);
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
    // deterministic mode: the residual kernels store per-tile sums, added here
    // on the host in tile order (tiles run through the pieces in order)
    const bool det = o.deterministic != 0;
    DBuf<double> TP;
    std::vector<double> hTP;
    if (det) {
        TP.alloc(4 * (int64_t)nt, s);
        hTP.resize(4 * (size_t)nt);
    }
    double* const tp = det ? TP.p : nullptr;
    auto fetch = [&](const DBuf<double>& acc, std::vector<double>& h) {
        if (!det) {
            PGCP_CUDA(cudaMemcpyAsync(h.data(), acc.p, 2 * S * sizeof(double), cudaMemcpyDeviceToHost, s));
            PGCP_CUDA(cudaStreamSynchronize(s));
            return;
        }
        PGCP_CUDA(cudaMemcpyAsync(hTP.data(), TP.p, hTP.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        PGCP_CUDA(cudaStreamSynchronize(s));
        std::fill(h.begin(), h.end(), 0.0);
        for (size_t t = 0; t < tiles.size(); ++t) {
            h[2 * tiles[t].seg] += hTP[4 * t];
            h[2 * tiles[t].seg + 1] += hTP[4 * t + 1];
        }
    };
    { k_residual<double, double2><<<nt, 256, 0, s>>>(d_tiles.p, P.row_ptr.p, P.col.p, P.val64.p, dinv64.p, P.nb.p,
                                                  dncp, x, 1, nullptr, BB.p, nullptr, nullptr, tp); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    std::vector<double> hBB(2 * S), hRR(2 * S), hTHR(2 * S);
    fetch(BB, hBB);
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
    if (o.precision == PGCP_DF64_REFINED || o.precision == PGCP_FP32_REFINED) {
        // run-based inner solves (double-float or FP32), FP64 residual outside
        const int f32 = o.precision == PGCP_FP32_REFINED;
        const double itol2 = o.inner_tol * o.inner_tol;
        DfSystem D;
        df_build(ctx, P, dncp, fixed, f32, D);
        // Double-float on the static schedule: every refinement step reduces
        // its own FP64 residual by DF_STEP and the next step continues the same
        // CG with the residual replaced (df_solve).  The replacement must stay a
        // small change of the recurrence residual for the search direction to
        // remain usable, so a step stops long before the recurrence drifts away
        // from the true residual (which happens near 2^-48 cond(A~)).  FP32
        // solves restart per step: continued FP32 CG took more iterations.
        constexpr double DF_STEP = 1e-3;
        const bool df_resume = !f32 && D.sched == 1 && !D.det;
        // Safeguard: near the double-float floor a continued step can break
        // down.  A step that leaves the worst FP64 residual above where it
        // started is undone (x from before the step) and the next step
        // restarts CG.
        DBuf<double2> xsave;
        if (df_resume) xsave.alloc(n, s);
        double prev_worst = INFINITY;
        bool restart = false;
        for (int outer = 0; outer < std::max(1, o.max_refine); ++outer) {
            RRo.zero();
            { k_residual<double, double2><<<nt, 256, 0, s>>>(d_tiles.p, P.row_ptr.p, P.col.p, P.val64.p, dinv64.p,
                                                          P.nb.p, dncp, x, 0, r64.p, RRo.p, nullptr, nullptr, tp); ::pgcp::note_launch(); }
            fetch(RRo, hRR);
            bool ok = false;
            res.relres = relres_of(hRR, &ok);
            res.refine = outer;
            if (ok) return res;
            if (df_resume && outer > 0 && res.relres > prev_worst) {
                PGCP_CUDA(cudaMemcpyAsync(x, xsave.p, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
                RRo.zero();
                { k_residual<double, double2><<<nt, 256, 0, s>>>(d_tiles.p, P.row_ptr.p, P.col.p, P.val64.p,
                                                              dinv64.p, P.nb.p, dncp, x, 0, r64.p, RRo.p, nullptr,
                                                              nullptr, tp); ::pgcp::note_launch(); }
                fetch(RRo, hRR);
                res.relres = relres_of(hRR, &ok);
                restart = true;
            }
            if (df_resume) PGCP_CUDA(cudaMemcpyAsync(xsave.p, x, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
            prev_worst = res.relres;
            // thresholds on the inner residual: the final tolerance (double-float),
            // or a fixed reduction of this right-hand side (FP32); converged
            // pieces (coordinates) are frozen
            for (int i = 0; i < S; ++i) {
                for (int c = 0; c < 2; ++c) {
                    const int j = 2 * i + c;
                    bool conv;
                    if (dncp) conv = hRR[2 * i] + hRR[2 * i + 1] <= tol2 * (hBB[2 * i] + hBB[2 * i + 1]);
                    else conv = hRR[j] <= tol2 * hBB[j];
                    const double step2 = f32 ? itol2 : (df_resume ? DF_STEP * DF_STEP : 0.0);
                    hTHR[j] = conv ? INFINITY : std::max(step2 * hRR[j], 0.25 * tol2 * hBB[j]);
                }
            }
            res.iters += df_solve(ctx, P, D, r64.p, x, hTHR, o.max_iters, df_resume && outer > 0 && !restart);
            restart = false;
        }
        RRo.zero();
        { k_residual<double, double2><<<nt, 256, 0, s>>>(d_tiles.p, P.row_ptr.p, P.col.p, P.val64.p, dinv64.p,
                                                      P.nb.p, dncp, x, 0, nullptr, RRo.p, nullptr, nullptr, tp); ::pgcp::note_launch(); }
        fetch(RRo, hRR);
        bool ok = false;
        res.relres = relres_of(hRR, &ok);
        res.refine = std::max(1, o.max_refine);
        return res;
    }
    if (o.precision == PGCP_FP64) {
        // FP64 PCG, restarted from the true residual while recursion drift
        // leaves it above the tolerance
        DBuf<double2> p, q, z;
        p.alloc(n, s);
        q.alloc(n, s);
        z.alloc(n, s);
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
            { k_residual<double, double2><<<nt, 256, 0, s>>>(d_tiles.p, P.row_ptr.p, P.col.p, P.val64.p, dinv64.p,
                                                          P.nb.p, dncp, x, 0, r64.p, RR.p, RZ.p, z.p); ::pgcp::note_launch(); }
            PGCP_CUDA(cudaMemcpyAsync(hRR.data(), RR.p, 2 * S * sizeof(double), cudaMemcpyDeviceToHost, s));
            PGCP_CUDA(cudaStreamSynchronize(s));
            bool ok = false;
            res.relres = relres_of(hRR, &ok);
            res.refine = outer;
            if (ok) return res;
            PcgArgs<double> a{n, P.row_ptr.p, P.col.p, P.val64.p, dinv64.p, P.nb.p, x, r64.p, p.p, q.p, z.p,
                              d_tiles.p, (int32_t)tiles.size(), S, RZ.p, RR.p, PQ.p, ACT.p, THR.p, iters.p,
                              out_it.p, o.max_iters, dncp, o.spmv_lanes, work.p};
            launch_pcg_lanes<double>(ctx, P, a);
            int it = 0;
            PGCP_CUDA(cudaMemcpyAsync(&it, out_it.p, sizeof(int), cudaMemcpyDeviceToHost, s));
            PGCP_CUDA(cudaStreamSynchronize(s));
            res.iters += it;
        }
        RRo.zero();
        { k_residual<double, double2><<<nt, 256, 0, s>>>(d_tiles.p, P.row_ptr.p, P.col.p, P.val64.p, dinv64.p,
                                                      P.nb.p, dncp, x, 0, nullptr, RRo.p, nullptr, nullptr, tp); ::pgcp::note_launch(); }
        fetch(RRo, hRR);
        bool ok = false;
        res.relres = relres_of(hRR, &ok);
        res.refine = std::max(1, o.max_refine);
        return res;
    }
    fail(PGCP_E_ARG, "unknown solver precision " + std::to_string(o.precision));
    return res;
}

}  // namespace pgcp
