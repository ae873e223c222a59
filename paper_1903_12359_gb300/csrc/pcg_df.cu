// Double-float PCG for the batched local (DNCP) and Laplace systems, inside
// FP64 iterative refinement (Sections 4.2 and 4.5 define the systems; the
// solver is this library's).
//
// Why: the GB300 FP64 pipe issues 2 DFMA per SM per cycle against 128 FFMA,
// and an FP64 Jacobi-PCG over these meshes is bound by it (14 DFMA per row in
// the SpMV alone).  FP32 alone is too coarse for the DNCP system (Jacobi-
// scaled condition number ~1e7: FP32 refinement stalls).  A double-float
// number is an unevaluated sum hi + lo of two floats, about 48 significant
// bits, computed with error-free transformations on the FP32 pipe:
//   TwoSum (Knuth), Fast2Sum (Dekker) and the FMA-based TwoProduct
//   (Ogita, Rump and Oishi, "Accurate sum and dot product", 2005).
// The __f*_rn intrinsics keep the compiler from contracting them.
//
// The system is solved in symmetrically Jacobi-scaled form,
//   A~ = S A S,  S = diag(d)^-1/2,  A~ x~ = S r64,  x += S x~,
// which is Jacobi-PCG without a preconditioner vector (z = r).  Fixed rows
// (pins, Dirichlet boundary) and fixed columns are dropped from A~, so their
// search directions stay exactly 0.  For DNCP the area term couples x and y
// on boundary rows; it is stored in the same CSR as "cross" entries (column
// stored as ~c): (A~ u)_x,i += -m y_c, (A~ u)_y,i += m x_c, with m = +1/2 for
// the next loop vertex and -1/2 for the previous one, scaled by s_i s_c.
//
// One persistent cooperative kernel runs all iterations.  Rows are split
// evenly over the blocks; a block's range is cut at piece boundaries into
// "runs", and scalars and reductions are per run (one block reduction per
// run and phase).  Per iteration:
//   phase B: beta = rr_k / rr_{k-1}; p = r + beta p; q = A~ r + beta q; <p, q>
//   grid sync
//   phase A: alpha = rr_k / <p, q>; x~ += alpha p; r -= alpha q;
//            <r, r> (scaled, drives CG) and sum d r^2 (unscaled, stopping test)
//   grid sync
// A piece (for Laplace: a coordinate) stops once its unscaled <r, r> is at or
// below its threshold; its runs are then skipped.  Accumulators rotate over 3
// (rr) and 2 (pq) slots so no extra syncs are needed to clear them.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "pgcp_internal.h"

namespace cg = cooperative_groups;

namespace pgcp {

namespace {

// ---------------------------------------------------------------- double-float

__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}

__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// acc + a * b (the lo * lo product, ~2^-48 relative, is dropped)
__device__ __forceinline__ float2 df_fma(float2 acc, float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    const float2 s = two_sum(acc.x, p);
    const float t = __fadd_rn(s.y, __fadd_rn(e, acc.y));
    return fast_two_sum(s.x, t);
}

__device__ __forceinline__ double df_to_d(float2 a) { return (double)a.x + (double)a.y; }

__device__ __forceinline__ float2 d_to_df(double d) {
    const float h = __double2float_rn(d);
    return make_float2(h, __double2float_rn(d - (double)h));
}

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 pack(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

constexpr int DF_THREADS = 256;

struct DfArgs {
    int32_t n;
    int32_t nseg;
    const int32_t* __restrict__ rp;
    const int32_t* __restrict__ col;    // ~c marks a cross (area-term) entry
    const float2* __restrict__ val;     // scaled values, double-float
    const float* __restrict__ dgn;      // diagonal of A (0 at fixed rows), for the unscaled norm
    float4* x;   // x~ (x, y components, double-float each)
    float4* r;
    float4* p;
    float4* q;
    const DfRun* __restrict__ runs;
    const int32_t* __restrict__ run_off;   // [grid + 1]
    double* RR;    // [3][2 nseg] scaled <r, r>
    double* RD;    // [3][2 nseg] unscaled sum d r^2
    double* PQ;    // [2][2 nseg]
    unsigned int* ACT;                  // [3]
    const double* __restrict__ THR;     // [2 nseg] thresholds on RD
    int32_t* out_iters;
    int32_t max_iters;
    int32_t dncp;
    unsigned long long* work;           // [2] free rows, stored entries, summed over iterations
};

__device__ __forceinline__ bool piece_done(const double* RD, const double* THR, int s, int c, bool dncp) {
    if (dncp) return RD[2 * s] + RD[2 * s + 1] <= THR[2 * s] + THR[2 * s + 1];
    return RD[2 * s + c] <= THR[2 * s + c];
}

// Sum NV doubles over the block; thread 0 gets the totals.
template <int NV>
__device__ __forceinline__ void block_sum(double* v, double* red) {
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
        for (int i = 0; i < NV; ++i) v[i] = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
#pragma unroll
            for (int i = 0; i < NV; ++i) v[i] += red[NV * w + i];
    }
}

// One stored entry of the SpMV: w += v * r_c (or the cross form).
__device__ __forceinline__ void spmv_entry(int32_t c, float2 v, const float4* __restrict__ r, float2& w0,
                                           float2& w1) {
    const bool cross = c < 0;
    const float4 rc = r[cross ? ~c : c];
    const float2 a0 = cross ? hi2(rc) : lo2(rc);
    const float2 a1 = cross ? lo2(rc) : hi2(rc);
    const float2 v0 = cross ? make_float2(-v.x, -v.y) : v;
    w0 = df_fma(w0, v0, a0);
    w1 = df_fma(w1, v, a1);
}

__global__ void __launch_bounds__(DF_THREADS) k_pcg_df(DfArgs a) {
    cg::grid_group grid = cg::this_grid();
    __shared__ double red[4 * (DF_THREADS / 32)];
    __shared__ double sc[2][2];
    __shared__ int sflag[2][2];
    const int nseg = a.nseg;
    const int rb = a.run_off[blockIdx.x], re = a.run_off[blockIdx.x + 1];
    unsigned long long wrows = 0, wnnz = 0;
    int k = 0;
    for (; k < a.max_iters; ++k) {
        const double* RRk = a.RR + (k % 3) * 2 * nseg;
        const double* RRm = a.RR + ((k + 2) % 3) * 2 * nseg;
        const double* RDk = a.RD + (k % 3) * 2 * nseg;
        double* PQk = a.PQ + (k % 2) * 2 * nseg;
        // ---------------- phase B: p = r + beta p, q = A~ r + beta q, <p, q>
        if (blockIdx.x == 0) {
            double* z1 = a.RR + ((k + 1) % 3) * 2 * nseg;
            double* z2 = a.RD + ((k + 1) % 3) * 2 * nseg;
            for (int i = threadIdx.x; i < 2 * nseg; i += blockDim.x) {
                z1[i] = 0.0;
                z2[i] = 0.0;
            }
        }
        bool any = false;
        for (int ri = rb; ri < re; ++ri) {
            const DfRun run = a.runs[ri];
            const int s = run.seg, slot = ri & 1;
            if (threadIdx.x == 0) {
                const bool d0 = piece_done(RDk, a.THR, s, 0, a.dncp);
                const bool d1 = piece_done(RDk, a.THR, s, 1, a.dncp);
                double b0 = 0.0, b1 = 0.0;
                if (k > 0) {
                    if (a.dncp) {
                        const double num = RRk[2 * s] + RRk[2 * s + 1], den = RRm[2 * s] + RRm[2 * s + 1];
                        b0 = b1 = den > 0.0 ? num / den : 0.0;
                    } else {
                        b0 = RRm[2 * s] > 0.0 ? RRk[2 * s] / RRm[2 * s] : 0.0;
                        b1 = RRm[2 * s + 1] > 0.0 ? RRk[2 * s + 1] / RRm[2 * s + 1] : 0.0;
                    }
                }
                sc[slot][0] = b0;
                sc[slot][1] = b1;
                sflag[slot][0] = d0;
                sflag[slot][1] = d1;
            }
            __syncthreads();
            const bool d0 = sflag[slot][0], d1 = sflag[slot][1];
            if (d0 && d1) continue;
            any = true;
            const float2 beta0 = d_to_df(sc[slot][0]), beta1 = d_to_df(sc[slot][1]);
            float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
            for (int row = run.lo + threadIdx.x; row < run.hi; row += blockDim.x) {
                const int b = a.rp[row], e = a.rp[row + 1];
                if (b == e) continue;   // fixed row
                float2 w0 = make_float2(0.f, 0.f), w1 = make_float2(0.f, 0.f);
                int j = b;
                for (; j + 4 <= e; j += 4) {
                    int32_t c[4];
                    float2 v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        c[u] = a.col[j + u];
                        v[u] = a.val[j + u];
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) spmv_entry(c[u], v[u], a.r, w0, w1);
                }
                for (; j < e; ++j) spmv_entry(a.col[j], a.val[j], a.r, w0, w1);
                const float4 rr = a.r[row];
                float4 pp = a.p[row], qq = a.q[row];
                float2 px = lo2(pp), py = hi2(pp), qx = lo2(qq), qy = hi2(qq);
                if (!d0) {
                    px = df_fma(lo2(rr), beta0, px);
                    qx = df_fma(w0, beta0, qx);
                    acc0 = df_fma(acc0, px, qx);
                }
                if (!d1) {
                    py = df_fma(hi2(rr), beta1, py);
                    qy = df_fma(w1, beta1, qy);
                    acc1 = df_fma(acc1, py, qy);
                }
                a.p[row] = pack(px, py);
                a.q[row] = pack(qx, qy);
            }
            double v[2] = {df_to_d(acc0), df_to_d(acc1)};
            block_sum<2>(v, red);
            if (threadIdx.x == 0) {
                atomicAdd(&PQk[2 * s], v[0]);
                atomicAdd(&PQk[2 * s + 1], v[1]);
                wrows += (unsigned long long)run.frows;
                wnnz += (unsigned long long)run.fnnz;
            }
        }
        if (threadIdx.x == 0 && any) *(volatile unsigned*)&a.ACT[k % 3] = 1u;
        grid.sync();
        // ---------------- phase A: x~ += alpha p, r -= alpha q, norms
        if (blockIdx.x == 0) {
            double* z = a.PQ + ((k + 1) % 2) * 2 * nseg;
            for (int i = threadIdx.x; i < 2 * nseg; i += blockDim.x) z[i] = 0.0;
            if (threadIdx.x == 0) a.ACT[(k + 1) % 3] = 0;
        }
        double* RRn = a.RR + ((k + 1) % 3) * 2 * nseg;
        double* RDn = a.RD + ((k + 1) % 3) * 2 * nseg;
        for (int ri = rb; ri < re; ++ri) {
            const DfRun run = a.runs[ri];
            const int s = run.seg, slot = ri & 1;
            if (threadIdx.x == 0) {
                const bool d0 = piece_done(RDk, a.THR, s, 0, a.dncp);
                const bool d1 = piece_done(RDk, a.THR, s, 1, a.dncp);
                double al0 = 0.0, al1 = 0.0;
                if (a.dncp) {
                    const double den = PQk[2 * s] + PQk[2 * s + 1];
                    al0 = al1 = den > 0.0 ? (RRk[2 * s] + RRk[2 * s + 1]) / den : 0.0;
                } else {
                    if (!d0) al0 = PQk[2 * s] > 0.0 ? RRk[2 * s] / PQk[2 * s] : 0.0;
                    if (!d1) al1 = PQk[2 * s + 1] > 0.0 ? RRk[2 * s + 1] / PQk[2 * s + 1] : 0.0;
                }
                sc[slot][0] = al0;
                sc[slot][1] = al1;
                sflag[slot][0] = d0 && d1;
            }
            __syncthreads();
            if (sflag[slot][0]) continue;
            const float2 al0 = d_to_df(sc[slot][0]), al1 = d_to_df(sc[slot][1]);
            const float2 nal0 = make_float2(-al0.x, -al0.y), nal1 = make_float2(-al1.x, -al1.y);
            float2 rr0 = make_float2(0.f, 0.f), rr1 = make_float2(0.f, 0.f);
            float rd0 = 0.f, rd1 = 0.f;
            for (int row = run.lo + threadIdx.x; row < run.hi; row += blockDim.x) {
                const float d = a.dgn[row];
                if (d == 0.f) continue;   // fixed row
                float4 xx = a.x[row], rv = a.r[row];
                const float4 pp = a.p[row], qq = a.q[row];
                const float2 x0 = df_fma(lo2(xx), al0, lo2(pp)), x1 = df_fma(hi2(xx), al1, hi2(pp));
                const float2 r0 = df_fma(lo2(rv), nal0, lo2(qq)), r1 = df_fma(hi2(rv), nal1, hi2(qq));
                a.x[row] = pack(x0, x1);
                a.r[row] = pack(r0, r1);
                rr0 = df_fma(rr0, r0, r0);
                rr1 = df_fma(rr1, r1, r1);
                rd0 = fmaf(d * r0.x, r0.x, rd0);
                rd1 = fmaf(d * r1.x, r1.x, rd1);
            }
            double v[4] = {df_to_d(rr0), df_to_d(rr1), (double)rd0, (double)rd1};
            block_sum<4>(v, red);
            if (threadIdx.x == 0) {
                atomicAdd(&RRn[2 * s], v[0]);
                atomicAdd(&RRn[2 * s + 1], v[1]);
                atomicAdd(&RDn[2 * s], v[2]);
                atomicAdd(&RDn[2 * s + 1], v[3]);
            }
        }
        grid.sync();
        if (*(volatile unsigned*)&a.ACT[k % 3] == 0u) break;
    }
    if (threadIdx.x == 0) {
        if (wrows) atomicAdd(&a.work[0], wrows);
        if (wnnz) atomicAdd(&a.work[1], wnnz);
        if (blockIdx.x == 0) a.out_iters[0] = k;
    }
}

// ---------------------------------------------------------------- set-up kernels

// Stored entries of row i of A~: free columns of a free row, plus the DNCP
// cross entries to free loop neighbours.
__global__ void k_df_count(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const uint8_t* __restrict__ fixed, const int2* __restrict__ nb, int dncp,
                           int32_t* __restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    if (!fixed[i]) {
        for (int j = rp[i]; j < rp[i + 1]; ++j) c += fixed[col[j]] ? 0 : 1;
        if (dncp) {
            const int2 pn = nb[i];
            if (pn.x >= 0) c += (fixed[pn.x] ? 0 : 1) + (fixed[pn.y] ? 0 : 1);
        }
    }
    cnt[i] = c;
}

__global__ void k_df_fill(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const double* __restrict__ val, const double* __restrict__ diag,
                          const uint8_t* __restrict__ fixed, const int2* __restrict__ nb, int dncp,
                          const int64_t* __restrict__ off, const int32_t* __restrict__ cnt,
                          int32_t* __restrict__ rp2, int32_t* __restrict__ col2,
                          float2* __restrict__ val2, double* __restrict__ sc, float* __restrict__ dgn) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = off[i];
    rp2[i] = (int32_t)o;
    if (i == n - 1) rp2[n] = (int32_t)(o + cnt[i]);
    if (fixed[i]) {
        sc[i] = 0.0;
        dgn[i] = 0.f;
        return;
    }
    const double si = 1.0 / sqrt(diag[i]);
    sc[i] = si;
    dgn[i] = (float)diag[i];
    int64_t t = o;
    for (int j = rp[i]; j < rp[i + 1]; ++j) {
        const int c = col[j];
        if (fixed[c]) continue;
        col2[t] = c;
        val2[t] = d_to_df(val[j] * si / sqrt(diag[c]));
        ++t;
    }
    if (dncp) {
        const int2 pn = nb[i];
        if (pn.x >= 0) {
            if (!fixed[pn.x]) {
                col2[t] = ~pn.x;
                val2[t] = d_to_df(-0.5 * si / sqrt(diag[pn.x]));
                ++t;
            }
            if (!fixed[pn.y]) {
                col2[t] = ~pn.y;
                val2[t] = d_to_df(0.5 * si / sqrt(diag[pn.y]));
                ++t;
            }
        }
    }
}

// frows / fnnz per run (one block per run)
__global__ void k_df_run_stats(DfRun* runs, const int32_t* __restrict__ rp2) {
    DfRun& r = runs[blockIdx.x];
    int fr = 0;
    for (int i = r.lo + threadIdx.x; i < r.hi; i += blockDim.x) fr += rp2[i + 1] > rp2[i] ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) fr += __shfl_xor_sync(0xffffffffu, fr, o);
    __shared__ int sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = fr;
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sh[w];
        r.frows = a;
        r.fnnz = rp2[r.hi] - rp2[r.lo];
    }
}

// r~ = S r64 (0 at fixed rows), x~ = p = q = 0, and slot-0 norms per run.
__global__ void k_df_prep(const DfRun* __restrict__ runs, const int32_t* __restrict__ run_off,
                          const double2* __restrict__ r64, const double* __restrict__ sc, float4* __restrict__ x,
                          float4* __restrict__ r, float4* __restrict__ p, float4* __restrict__ q,
                          double* __restrict__ RR, double* __restrict__ RD) {
    __shared__ double red[4 * (DF_THREADS / 32)];
    for (int ri = run_off[blockIdx.x]; ri < run_off[blockIdx.x + 1]; ++ri) {
        const DfRun run = runs[ri];
        double v[4] = {0, 0, 0, 0};
        for (int i = run.lo + threadIdx.x; i < run.hi; i += blockDim.x) {
            const double si = sc[i];
            const double2 ri64 = r64[i];
            const double a0 = si * ri64.x, a1 = si * ri64.y;
            const float2 f0 = d_to_df(a0), f1 = d_to_df(a1);
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            x[i] = z;
            p[i] = z;
            q[i] = z;
            r[i] = pack(f0, f1);
            if (si != 0.0) {
                v[0] += a0 * a0;
                v[1] += a1 * a1;
                v[2] += ri64.x * ri64.x;
                v[3] += ri64.y * ri64.y;
            }
        }
        block_sum<4>(v, red);
        if (threadIdx.x == 0) {
            atomicAdd(&RR[2 * run.seg], v[0]);
            atomicAdd(&RR[2 * run.seg + 1], v[1]);
            atomicAdd(&RD[2 * run.seg], v[2]);
            atomicAdd(&RD[2 * run.seg + 1], v[3]);
        }
        __syncthreads();
    }
}

// x += S x~ on free rows
__global__ void k_df_finish(int64_t n, const double* __restrict__ sc, const float4* __restrict__ xs,
                            double2* __restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double si = sc[i];
    if (si == 0.0) return;
    const float4 v = xs[i];
    x[i].x += si * df_to_d(lo2(v));
    x[i].y += si * df_to_d(hi2(v));
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, ceil_div(n, t)); }

}  // namespace

// ---------------------------------------------------------------- host side

void df_build(pgcp_ctx* ctx, Part& P, int dncp, const uint8_t* fixed, DfSystem& D) {
    cudaStream_t s = ctx->stream;
    const int64_t n = P.Nc;
    if (n >= INT32_MAX) fail(PGCP_E_ARG, "double-float PCG: too many rows");
    D.n = n;
    D.dncp = dncp;
    DBuf<int32_t> cnt;
    DBuf<int64_t> off;
    cnt.alloc(n, s);
    off.alloc(n, s);
    { k_df_count<<<nblk(n), 256, 0, s>>>(n, P.row_ptr.p, P.col.p, fixed, P.nb.p, dncp, cnt.p); ::pgcp::note_launch(); }
    int64_t nnz2 = 0;
    exclusive_scan_i32_to_i64(cnt.p, off.p, n, s, &nnz2);
    if (nnz2 >= INT32_MAX) fail(PGCP_E_ARG, "double-float PCG: too many stored entries");
    D.nnz = nnz2;
    D.rp.alloc(n + 1, s);
    D.col.alloc(std::max<int64_t>(nnz2, 1), s);
    D.val.alloc(std::max<int64_t>(nnz2, 1), s);
    D.sc.alloc(n, s);
    D.dgn.alloc(n, s);
    { k_df_fill<<<nblk(n), 256, 0, s>>>(n, P.row_ptr.p, P.col.p, P.val64.p, P.diag64.p, fixed, P.nb.p, dncp, off.p,
                                       cnt.p, D.rp.p, D.col.p, D.val.p, D.sc.p, D.dgn.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    // persistent grid and its row runs
    int per_sm = 0;
    PGCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_df, DF_THREADS, 0));
    if (per_sm <= 0) fail(PGCP_E_CUDA, "double-float PCG kernel cannot be resident");
    int grid = (int)std::min<int64_t>((int64_t)per_sm * ctx->num_sms, std::max<int64_t>(1, ceil_div(n, 32)));
    grid = std::max(grid, 1);
    D.grid = grid;
    std::vector<DfRun> runs;
    std::vector<int32_t> roff(grid + 1, 0);
    for (int b = 0; b < grid; ++b) {
        int64_t lo = n * b / grid, hi = n * (b + 1) / grid;
        roff[b] = (int32_t)runs.size();
        while (lo < hi) {
            // piece holding row lo
            const int seg = (int)(std::upper_bound(P.voff.begin(), P.voff.end(), lo) - P.voff.begin()) - 1;
            const int64_t end = std::min<int64_t>(hi, P.voff[seg + 1]);
            runs.push_back(DfRun{seg, (int32_t)lo, (int32_t)end, 0, 0, 0, 0, 0});
            lo = end;
        }
    }
    roff[grid] = (int32_t)runs.size();
    D.nruns = (int32_t)runs.size();
    D.runs.alloc(std::max<int64_t>(1, D.nruns), s);
    D.run_off.alloc(grid + 1, s);
    PGCP_CUDA(cudaMemcpyAsync(D.runs.p, runs.data(), runs.size() * sizeof(DfRun), cudaMemcpyHostToDevice, s));
    PGCP_CUDA(cudaMemcpyAsync(D.run_off.p, roff.data(), roff.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    if (D.nruns > 0) {
        { k_df_run_stats<<<(unsigned)D.nruns, 256, 0, s>>>(D.runs.p, D.rp.p); ::pgcp::note_launch(); }
    }
    D.x.alloc(n, s);
    D.r.alloc(n, s);
    D.p.alloc(n, s);
    D.q.alloc(n, s);
    const int S = P.K;
    D.RR.alloc(3 * 2 * S, s);
    D.RD.alloc(3 * 2 * S, s);
    D.PQ.alloc(2 * 2 * S, s);
    D.ACT.alloc(3, s);
    D.THR.alloc(2 * S, s);
    D.out_it.alloc(1, s);
    D.work.alloc(2, s);
    PGCP_CUDA(cudaGetLastError());
    PGCP_CUDA(cudaStreamSynchronize(s));   // host vectors above go out of scope
}

int df_solve(pgcp_ctx* ctx, Part& P, DfSystem& D, const double2* r64, double2* x, const std::vector<double>& thr,
             int max_iters) {
    cudaStream_t s = ctx->stream;
    const int S = P.K;
    D.RR.zero();
    D.RD.zero();
    D.PQ.zero();
    D.ACT.zero();
    PGCP_CUDA(cudaMemcpyAsync(D.THR.p, thr.data(), 2 * S * sizeof(double), cudaMemcpyHostToDevice, s));
    { k_df_prep<<<(unsigned)D.grid, DF_THREADS, 0, s>>>(D.runs.p, D.run_off.p, r64, D.sc.p, D.x.p, D.r.p, D.p.p,
                                                        D.q.p, D.RR.p, D.RD.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    DfArgs a{(int32_t)D.n, S, D.rp.p, D.col.p, D.val.p, D.dgn.p, D.x.p, D.r.p, D.p.p, D.q.p, D.runs.p,
             D.run_off.p, D.RR.p, D.RD.p, D.PQ.p, D.ACT.p, D.THR.p, D.out_it.p, max_iters, D.dncp, D.work.p};
    cudaEvent_t e0, e1;
    PGCP_CUDA(cudaEventCreate(&e0));
    PGCP_CUDA(cudaEventCreate(&e1));
    PGCP_CUDA(cudaMemsetAsync(D.work.p, 0, 2 * sizeof(unsigned long long), s));
    PGCP_CUDA(cudaEventRecord(e0, s));
    void* args[] = {(void*)&a};
    { PGCP_CUDA(cudaLaunchCooperativeKernel((void*)k_pcg_df, dim3(D.grid), dim3(DF_THREADS), args, 0, s)); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaEventRecord(e1, s));
    { k_df_finish<<<nblk(D.n), 256, 0, s>>>(D.n, D.sc.p, D.x.p, x); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    unsigned long long w[2] = {0, 0};
    int it = 0;
    PGCP_CUDA(cudaMemcpyAsync(w, D.work.p, sizeof(w), cudaMemcpyDeviceToHost, s));
    PGCP_CUDA(cudaMemcpyAsync(&it, D.out_it.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    PGCP_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    PGCP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    P.stats.pcg_ms += ms;
    // per free row and iteration: phase B row pointer 4, r 16, p r/w 32, q r/w 32;
    // phase A diagonal 4, x r/w 32, r r/w 32, p 16, q 16 -> 184 B;
    // per stored entry: column 4 + double-float value 8 (gathered r hits cache)
    P.stats.pcg_bytes += (double)w[0] * 184.0 + (double)w[1] * 12.0;
    P.stats.pcg_launches += 1;
    return it;
}

}  // namespace pgcp
