// Multilevel additive preconditioner for the batched double-float PCG of the
// local solves (Section 4.2 defines the DNCP systems; the preconditioner is
// this library's).
//
// The Jacobi-scaled system A~ = S A S (S = diag(A)^-1/2, fixed rows and columns
// dropped) is solved by PCG with
//   M = I + sum_l sum_b Phi_lb T_lb T_lb^T Phi_lb^T,
// an additive multilevel form over nested blocks of consecutive rows of a
// piece.  A piece's rows are its vertices in ascending global id, which the
// meshes order along a space-filling curve, so consecutive rows form compact
// patches.  Level l has blocks of 16 * 4^l rows, up to one block holding the
// whole piece.  On the rows of block b, Phi_lb spans for each coordinate (x
// and y) the monomials of xi = (X - c_b) / rho_b up to degree 1 on level 0 and
// degree 2 above (X the vertex in its piece's frame, c_b and rho_b the block's
// centroid and RMS radius), times sqrt(d_i) so that they act on scaled
// unknowns.  T_lb is upper triangular with T T^T the inverse of the block's
// Galerkin matrix Phi^T A~ Phi in an orthonormalised basis (nearly dependent
// monomials and null directions dropped), so M is symmetric positive definite
// whatever the rounding of T.
//
// The slow modes of Jacobi-PCG on the conformal energy are smooth,
// near-conformal maps, which low-degree polynomials on patches of every size
// capture.  The additive form needs no matrix products on the coarse levels:
// per iteration it takes the residual's moments per block (restriction:
// 20 products per row, then child-to-parent polynomial re-expansion), two
// small triangular products per block, and one quadratic per 16-row block
// (prolongation: the levels' polynomials are re-expanded top-down into the
// level-0 frame and added).
//
// Iteration k of the persistent kernel (static row runs, 16-aligned within
// their piece, at most ML_SEG rows):
//   phase B: beta = <r,z>_k / <r,z>_{k-1}; p = z + beta p; q = A~ z + beta q; <p, q>
//   phase A: alpha = <r,z>_k / <p,q>; x~ += alpha p; r -= alpha q; sum d r^2;
//            moments of r per block (level 0 stored, coarser levels summed)
//   phase C: z = M r; <r, z>
// with a grid sync after each phase.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "df_arith.cuh"
#include "pgcp_internal.h"

namespace cg = cooperative_groups;

namespace pgcp {

namespace {

using namespace dfa;

constexpr int MLB = 3;   // resident 256-thread blocks per SM the kernel is compiled for (80 registers)
// rows per block of level l: 16 * 4^l = 1 << ml_shift(l)
__host__ __device__ constexpr int ml_shift(int l) { return 4 + 2 * l; }
__host__ __device__ constexpr int ml_nf1(int l) { return l == 0 ? 4 : 10; }
__host__ __device__ constexpr int ml_ts(int l) { return l == 0 ? 36 : 210; }   // packed size of the full factor
// shared-memory slots per level: blocks of a level that a run of ML_SEG rows can touch
__host__ __device__ constexpr int ml_cap(int l) { return (ML_SEG >> ml_shift(l)) + 2; }
__host__ __device__ constexpr int ml_capoff(int l) {
    int o = 0;
    for (int i = 0; i < l; ++i) o += ml_cap(i);
    return o;
}
constexpr int ML_CAPTOT = ml_capoff(ML_MAXL);

// packed upper-triangular index (row-major upper triangle of an n x n matrix)
__host__ __device__ __forceinline__ int ut(int i, int j, int n) { return i * n - i * (i - 1) / 2 + (j - i); }

// the ten monomials of xi: 1, x, y, z, xx, xy, yy, xz, yz, zz
template <typename R>
__host__ __device__ __forceinline__ void mono10(R x, R y, R z, R* m) {
    m[0] = R(1);
    m[1] = x;
    m[2] = y;
    m[3] = z;
    m[4] = x * x;
    m[5] = x * y;
    m[6] = y * y;
    m[7] = x * z;
    m[8] = y * z;
    m[9] = z * z;
}
// the two factors (a, b) of quadratic monomial 4 + q: xx xy yy xz yz zz
__host__ __device__ __forceinline__ int qa(int q) { return (q == 2 || q == 4) ? 1 : (q == 5 ? 2 : 0); }
__host__ __device__ __forceinline__ int qb(int q) { return q == 0 ? 0 : (q <= 2 ? 1 : 2); }

// Moment k (0..9) of a child's rows in the parent frame, xi_p = s xi_c + t,
// from the child's ten moments mc.
__device__ __forceinline__ float mom_out(int k, const float* mc, float s, const float* t) {
    const float m0 = mc[0];
    if (k == 0) return m0;
    if (k < 4) return s * mc[k] + t[k - 1] * m0;
    const int q = k - 4, a = qa(q), b = qb(q);
    return s * s * mc[k] + s * t[b] * mc[1 + a] + s * t[a] * mc[1 + b] + t[a] * t[b] * m0;
}

// The transpose: coefficient k (0..9) in the child frame of the parent-frame
// polynomial with coefficients cp.
__device__ __forceinline__ float coef_out(int k, const float* cp, float s, const float* t) {
    if (k >= 4) return s * s * cp[k];
    float v = 0.f;
    if (k == 0) {
        v = cp[0];
#pragma unroll
        for (int a = 0; a < 3; ++a) v += t[a] * cp[1 + a];
#pragma unroll
        for (int q = 0; q < 6; ++q) v += t[qa(q)] * t[qb(q)] * cp[4 + q];
        return v;
    }
    const int a = k - 1;
    v = s * cp[k];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        if (qa(q) == a) v += s * t[qb(q)] * cp[4 + q];
        if (qb(q) == a) v += s * t[qa(q)] * cp[4 + q];
    }
    return v;
}

struct MlArgs {
    int32_t n, nseg, k0, max_iters, dncp, nl;
    int32_t resume;                     // k0 continues a solve with a replaced residual: beta of
                                        // iteration k0 divides by RRP, each piece's <r, z> of
                                        // its last active iteration
    double* RRP;                        // [2 nseg]
    const int32_t* __restrict__ rp;
    const int32_t* __restrict__ col;
    const float2* __restrict__ val;
    const float* __restrict__ dgn;
    float4* x;
    float4* r;
    float4* p;
    float4* q;
    float4* z;
    const DfRun* __restrict__ runs;
    const int32_t* __restrict__ run_off;
    double* RR;    // [3][2 nseg] <r, z>
    double* RD;    // [3][2 nseg] unscaled sum d r^2
    double* PQ;    // [2][2 nseg]
    unsigned int* ACT;
    const double* __restrict__ THR;
    int32_t* out_iters;
    unsigned long long* work;
    const int32_t* __restrict__ bofs;   // [ML_MAXL][nseg + 1]
    const int32_t* __restrict__ ltop;   // [nseg]
    const int32_t* __restrict__ pvoff;  // [nseg + 1]
    const float* __restrict__ xr;       // [3 n]
    const float4* __restrict__ geo;
    const float* __restrict__ T;
    const uint8_t* __restrict__ sep;
    float* M;                           // [2][mstride][ML_NM]
    int64_t mstride;
    int64_t lofs[ML_MAXL + 1];
    int64_t tofs[ML_MAXL + 1];
};

__device__ __forceinline__ bool done_of(const double* RD, const double* THR, int s, int c, bool dncp) {
    if (dncp) return __ldcg(RD + 2 * s) + __ldcg(RD + 2 * s + 1) <= THR[2 * s] + THR[2 * s + 1];
    return __ldcg(RD + 2 * s + c) <= THR[2 * s + c];
}

// c = T (T^T m) for a packed upper-triangular N x N factor T (compile-time
// size: every load independent and unrolled).
template <int N>
__device__ __forceinline__ void tri_coef(const float* __restrict__ T, const float* m, float* c) {
    float u[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        float a = 0.f;
#pragma unroll
        for (int i = 0; i <= j; ++i) a = fmaf(__ldg(T + ut(i, j, N)), m[i], a);
        u[j] = a;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float a = 0.f;
#pragma unroll
        for (int j = i; j < N; ++j) a = fmaf(__ldg(T + ut(i, j, N)), u[j], a);
        c[i] = a;
    }
}

// The same for one coarse block by a warp (N = 10 separable, applied to x and
// y, or N = 20): lane L holds m_L on entry and c_L on return (L < 20).  Each
// lane loads its column and row of T first, so the loads overlap.
__device__ __forceinline__ float warp_coef(const float* __restrict__ T, bool sep, float mL) {
    const int lane = threadIdx.x & 31;
    const int n = sep ? 10 : 20;
    const int h = sep ? (lane >= 10 ? 10 : 0) : 0;   // first lane of this lane's system
    const int i = lane - h;                          // output index in the system
    const bool on = lane < 20;
    float colT[20], rowT[20];
#pragma unroll
    for (int k = 0; k < 20; ++k) {
        colT[k] = (on && k <= i && k < n) ? __ldg(T + ut(k, i, n)) : 0.f;
        rowT[k] = (on && k >= i && k < n) ? __ldg(T + ut(i, k, n)) : 0.f;
    }
    float u = 0.f;
#pragma unroll
    for (int k = 0; k < 20; ++k) u = fmaf(colT[k], __shfl_sync(0xffffffffu, mL, (h + k) & 31), u);   // sum_{k<=i} T_ki m_k
    float c = 0.f;
#pragma unroll
    for (int k = 0; k < 20; ++k) c = fmaf(rowT[k], __shfl_sync(0xffffffffu, u, (h + k) & 31), c);    // sum_{k>=i} T_ik u_k
    return c;
}

// First global block of each level of piece s (lofs + bofs), loaded once per
// call into shared memory by threads 0 .. ML_MAXL-1; out also gets the
// level's first packed-factor entry.  Ends with a barrier.
__device__ __forceinline__ void ml_bases(const MlArgs& a, int s, int64_t* gb, int64_t* tf) {
    if (threadIdx.x < ML_MAXL) {
        const int l = threadIdx.x;
        gb[l] = a.lofs[l] + a.bofs[l * (a.nseg + 1) + s];
        tf[l] = a.tofs[l] - a.lofs[l] * (int64_t)ml_ts(l);   // T of global block g: T + tf[l] + g * ts(l)
    }
    __syncthreads();
}

// Restriction for one run: after the level-0 moments of the run's rows are
// stored (one half-warp per 16-row block), the coarser levels' partial moments
// from this run's rows, one (block, moment) per thread, summed into M: a block
// inside the run is stored, a block shared with other runs is added
// atomically (its slot was cleared by the run holding its first row).
// smem: two ping-pong buffers in buf; the block frames come from tab when
// it still holds this run's tables (else from global memory).
__device__ __noinline__ void ml_restrict(const MlArgs& a, const DfRun& run, float* buf, int par, const float* tab) {
    const int s = run.seg, pv = a.pvoff[s];
    const int top = min(a.ltop[s], a.nl - 1);
    float* Mp = a.M + (int64_t)par * a.mstride * ML_NM;
    const int lo = run.lo - pv, hi = run.hi - pv;
    const int nrow = a.pvoff[s + 1] - pv;
    __shared__ int64_t s_gb[ML_MAXL], s_tf[ML_MAXL];
    ml_bases(a, s, s_gb, s_tf);
    float* prev = buf;
    float* cur = buf + ml_cap(1) * ML_NM;
    for (int l = 1; l <= top; ++l) {
        const int sh = ml_shift(l), shc = ml_shift(l - 1);
        const int b0 = lo >> sh, b1 = (hi - 1) >> sh;
        const int c0 = lo >> shc, c1 = (hi - 1) >> shc;
        const int64_t gb0 = s_gb[l];
        const int64_t gc0 = s_gb[l - 1];
        for (int task = threadIdx.x; task < (b1 - b0 + 1) * 2; task += blockDim.x) {
            const int j = task >> 1, h = (task & 1) * 10;
            const int blk = b0 + j;
            const float4 gp = tab ? *reinterpret_cast<const float4*>(tab + (ml_capoff(l) + j) * 24 + 20) : a.geo[gb0 + blk];
            float acc[10];
#pragma unroll
            for (int k = 0; k < 10; ++k) acc[k] = 0.f;
            const int cl = max(blk * 4, c0), ch = min(blk * 4 + 3, c1);
            for (int c = cl; c <= ch; ++c) {
                const float4 gc = tab ? *reinterpret_cast<const float4*>(tab + (ml_capoff(l - 1) + c - c0) * 24 + 20)
                                      : a.geo[gc0 + c];
                const float sc = gp.w / gc.w;
                const float t[3] = {(gc.x - gp.x) * gp.w, (gc.y - gp.y) * gp.w, (gc.z - gp.z) * gp.w};
                const float* src = (l == 1 ? Mp + (gc0 + c) * ML_NM : prev + (c - c0) * ML_NM) + h;
                float mc[10];
#pragma unroll
                for (int k = 0; k < 10; ++k) mc[k] = src[k];
#pragma unroll
                for (int k = 0; k < 10; ++k) acc[k] += mom_out(k, mc, sc, t);
            }
            float* g = Mp + (gb0 + blk) * ML_NM + h;
            const bool inside = (blk << sh) >= lo && min((blk + 1) << sh, nrow) <= hi;
#pragma unroll
            for (int k = 0; k < 10; ++k) {
                cur[j * ML_NM + h + k] = acc[k];
                if (inside) g[k] = acc[k];
                else atomicAdd(g + k, acc[k]);
            }
        }
        __syncthreads();
        float* t = prev;
        prev = cur;
        cur = t;
    }
}

// Prolongation tables for one run: every level's coefficients c = T T^T m on
// the blocks the run touches (level 0 one thread per block, coarser levels one
// warp per block), then re-expanded top-down into the level-0 frames (one
// (block, coefficient) per thread); each level-0 slot ends with the combined
// quadratic (20 values) and the block's frame (4 values).  Also clears the
// next parity's moments of the blocks whose first row lies in this run
// (levels >= 1).
__device__ __noinline__ void ml_tables(const MlArgs& a, const DfRun& run, float* tab, int par) {
    const int s = run.seg, pv = a.pvoff[s];
    const int top = min(a.ltop[s], a.nl - 1);
    const float* Mp = a.M + (int64_t)par * a.mstride * ML_NM;
    float* Mn = a.M + (int64_t)(par ^ 1) * a.mstride * ML_NM;
    const int lo = run.lo - pv, hi = run.hi - pv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    __shared__ int64_t s_gb[ML_MAXL], s_tf[ML_MAXL];
    ml_bases(a, s, s_gb, s_tf);
    // level 0: one thread per block
    {
        const int b0 = lo >> 4, b1 = (hi - 1) >> 4;
        const int64_t gb0 = s_gb[0];
        for (int j = threadIdx.x; j <= b1 - b0; j += blockDim.x) {
            const int64_t gb = gb0 + b0 + j;
            const float* src = Mp + gb * ML_NM;
            float m[8], c[8];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                m[f] = __ldcg(src + f);
                m[4 + f] = __ldcg(src + 10 + f);
            }
            const float* T = a.T + s_tf[0] + gb * ml_ts(0);
            if (a.sep[gb]) {
                tri_coef<4>(T, m, c);
                tri_coef<4>(T, m + 4, c + 4);
            } else {
                tri_coef<8>(T, m, c);
            }
            float* dst = tab + j * 24;
#pragma unroll
            for (int f = 0; f < 10; ++f) {
                dst[f] = f < 4 ? c[f] : 0.f;
                dst[10 + f] = f < 4 ? c[4 + f] : 0.f;
            }
            const float4 g = a.geo[gb];
            dst[20] = g.x;
            dst[21] = g.y;
            dst[22] = g.z;
            dst[23] = g.w;
        }
    }
    // levels 1..top, all levels at once: separable blocks one thread each,
    // coupled blocks (boundary edges inside) one warp each
    {
        int total = 0;
        for (int l = 1; l <= top; ++l) total += ((hi - 1) >> ml_shift(l)) - (lo >> ml_shift(l)) + 1;
        auto item = [&](int w, int& l, int& j) {   // the level and block of work item w
            l = 1;
            j = w;
            while (true) {
                const int nbl = ((hi - 1) >> ml_shift(l)) - (lo >> ml_shift(l)) + 1;
                if (j < nbl) break;
                j -= nbl;
                ++l;
            }
        };
        for (int w = threadIdx.x; w < total; w += blockDim.x) {
            int l, j;
            item(w, l, j);
            const int sh = ml_shift(l);
            const int blk = (lo >> sh) + j;
            const int64_t gb = s_gb[l] + blk;
            if (!a.sep[gb]) continue;
            const float* src = Mp + gb * ML_NM;
            const float* T = a.T + s_tf[l] + gb * ml_ts(l);
            float* dst = tab + (ml_capoff(l) + j) * 24;
            float m[10], c[10];
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int f = 0; f < 10; ++f) m[f] = __ldcg(src + 10 * h + f);
                tri_coef<10>(T, m, c);
#pragma unroll
                for (int f = 0; f < 10; ++f) dst[10 * h + f] = c[f];
            }
            if ((blk << sh) >= lo)   // first row here: clear the next parity
#pragma unroll
                for (int f = 0; f < ML_NM; ++f) Mn[gb * ML_NM + f] = 0.f;
            const float4 g = a.geo[gb];
            dst[20] = g.x;
            dst[21] = g.y;
            dst[22] = g.z;
            dst[23] = g.w;
        }
        for (int w = warp; w < total; w += nwarp) {
            int l, j;
            item(w, l, j);
            const int sh = ml_shift(l);
            const int blk = (lo >> sh) + j;
            const int64_t gb = s_gb[l] + blk;
            if (a.sep[gb]) continue;   // warp-uniform
            const float mL = lane < ML_NM ? __ldcg(Mp + gb * ML_NM + lane) : 0.f;
            const float c = warp_coef(a.T + s_tf[l] + gb * ml_ts(l), false, mL);
            float* dst = tab + (ml_capoff(l) + j) * 24;
            if (lane < ML_NM) {
                dst[lane] = c;
                if ((blk << sh) >= lo) Mn[gb * ML_NM + lane] = 0.f;
            }
            if (lane == 0) {
                const float4 g = a.geo[gb];
                dst[20] = g.x;
                dst[21] = g.y;
                dst[22] = g.z;
                dst[23] = g.w;
            }
        }
    }
    __syncthreads();
    // top-down: add the parent's combined polynomial, re-expanded in the child frame
    for (int l = top - 1; l >= 0; --l) {
        const int sh = ml_shift(l);
        const int b0 = lo >> sh, b1 = (hi - 1) >> sh;
        const int pb0 = lo >> ml_shift(l + 1);
        float* tl = tab + ml_capoff(l) * 24;
        const float* tp = tab + ml_capoff(l + 1) * 24;
        for (int task = threadIdx.x; task < (b1 - b0 + 1) * 2; task += blockDim.x) {
            const int j = task >> 1, h = (task & 1) * 10;
            const int blk = b0 + j;
            float* dst = tl + j * 24;
            const float* pc = tp + ((blk >> 2) - pb0) * 24;
            const float sc = pc[23] / dst[23];
            const float t[3] = {(dst[20] - pc[20]) * pc[23], (dst[21] - pc[21]) * pc[23], (dst[22] - pc[22]) * pc[23]};
            float cp[10];
#pragma unroll
            for (int k = 0; k < 10; ++k) cp[k] = pc[h + k];
#pragma unroll
            for (int k = 0; k < 10; ++k) dst[h + k] += coef_out(k, cp, sc, t);
        }
        __syncthreads();
    }
}

// Level-0 moments of r for one 256-row pass (the warp's 32 rows are two
// 16-row blocks): every row's 20 products go through shared memory (mbuf, 20
// floats per thread), and lane l sums entry l % 20 of block l / 20 (then
// l + 32) over the block's 16 rows and stores it.
__device__ __forceinline__ void ml_moments0(const MlArgs& a, const DfRun& run, int base, int par, bool act, float d,
                                            float rx, float ry, int row, float* mbuf, const float* tab) {
    const int lane = threadIdx.x & 31;
    const int pv = a.pvoff[run.seg];
    const int64_t g0 = a.lofs[0] + a.bofs[run.seg];
    float mom[ML_NM];
#pragma unroll
    for (int f = 0; f < ML_NM; ++f) mom[f] = 0.f;
    if (act && d != 0.f) {
        const int blk = (row - pv) >> 4;
        const float4 g = tab ? *reinterpret_cast<const float4*>(tab + (blk - ((run.lo - pv) >> 4)) * 24 + 20)
                             : a.geo[g0 + blk];
        const float sd = sqrtf(d);
        float mv[10];
        mono10<float>((a.xr[3 * row] - g.x) * g.w, (a.xr[3 * row + 1] - g.y) * g.w, (a.xr[3 * row + 2] - g.z) * g.w,
                      mv);
        const float ux = sd * rx, uy = sd * ry;
#pragma unroll
        for (int f = 0; f < 10; ++f) {
            mom[f] = mv[f] * ux;
            mom[10 + f] = mv[f] * uy;
        }
    }
    float4* mine = reinterpret_cast<float4*>(mbuf + threadIdx.x * ML_NM);
#pragma unroll
    for (int f = 0; f < ML_NM / 4; ++f) mine[f] = make_float4(mom[4 * f], mom[4 * f + 1], mom[4 * f + 2], mom[4 * f + 3]);
    __syncwarp();
    const int wbase = threadIdx.x & ~31u;   // this warp's first thread (and row offset in the pass)
#pragma unroll
    for (int o = lane; o < 2 * ML_NM; o += 32) {
        const int h = o / ML_NM, f = o - h * ML_NM;
        const int r0 = base + wbase + 16 * h;   // first row of the block
        if (r0 < run.hi) {
            float v = 0.f;
#pragma unroll
            for (int r = 0; r < 16; ++r) v += mbuf[(wbase + 16 * h + r) * ML_NM + f];
            a.M[((int64_t)par * a.mstride + g0 + ((r0 - pv) >> 4)) * ML_NM + f] = v;
        }
    }
    __syncwarp();
}

template <int MINB>
__global__ void __launch_bounds__(RUN_THREADS, MINB) k_pcg_ml(const __grid_constant__ MlArgs a) {
    using A = ArithDF;
    using S = A::S;
    using V = A::V;
    cg::grid_group grid = cg::this_grid();
    __shared__ float2 red[4 * (RUN_THREADS / 32)];
    __shared__ double sc[2][2];
    __shared__ int sflag[2][2];
    __shared__ __align__(16) float tab[ML_CAPTOT * 24];
    __shared__ __align__(16) float mbuf[RUN_THREADS * ML_NM];
    __shared__ int tab_run;   // the run whose tables tab holds (-1: none)
    if (threadIdx.x == 0) tab_run = -1;
    __syncthreads();
    const int nseg = a.nseg;
    const int rb = a.run_off[blockIdx.x], re = a.run_off[blockIdx.x + 1];
    const int32_t* __restrict__ rp = a.rp;
    const int32_t* __restrict__ colp = a.col;
    const S* __restrict__ valp = a.val;
    const float* __restrict__ dgp = a.dgn;
    unsigned long long wrows = 0, wnnz = 0;

    // z = M r_j on the runs' rows and <r_j, z_j> into RR slot `slot`
    auto phase_c = [&](int j, int slot) {
        const int par = j & 1;
        double* RRn = a.RR + slot * 2 * nseg;
        const double* RDj = a.RD + (j % 3) * 2 * nseg;
        for (int ri = rb; ri < re; ++ri) {
            const DfRun run = a.runs[ri];
            const int s = run.seg;
            if (threadIdx.x == 0)
                sflag[0][0] = done_of(RDj, a.THR, s, 0, a.dncp) && done_of(RDj, a.THR, s, 1, a.dncp);
            __syncthreads();
            const bool skip = sflag[0][0];
            __syncthreads();
            if (skip) continue;
            ml_tables(a, run, tab, par);
            if (threadIdx.x == 0) tab_run = ri;
            const int pv = a.pvoff[s];
            const int c0 = (run.lo - pv) >> 4;
            S rz0 = A::zero(), rz1 = A::zero();
            for (int row = run.lo + threadIdx.x; row < run.hi; row += blockDim.x) {
                const float d = __ldg(dgp + row);
                if (d == 0.f) {
                    a.z[row] = A::vzero();
                    continue;
                }
                const V rv = a.r[row];
                const float* t0 = tab + (((row - pv) >> 4) - c0) * 24;
                float mv[10];
                mono10<float>((a.xr[3 * row] - t0[20]) * t0[23], (a.xr[3 * row + 1] - t0[21]) * t0[23],
                              (a.xr[3 * row + 2] - t0[22]) * t0[23], mv);
                float cx = 0.f, cy = 0.f;
#pragma unroll
                for (int f = 0; f < 10; ++f) {
                    cx = fmaf(t0[f], mv[f], cx);
                    cy = fmaf(t0[10 + f], mv[f], cy);
                }
                const float sd = sqrtf(d);
                const S zx = df_add(A::cx(rv), make_float2(sd * cx, 0.f));
                const S zy = df_add(A::cy(rv), make_float2(sd * cy, 0.f));
                a.z[row] = A::pack(zx, zy);
                rz0 = A::fma(rz0, A::cx(rv), zx);
                rz1 = A::fma(rz1, A::cy(rv), zy);
            }
            float2 pv2[2] = {rz0, rz1};
            double v[2];
            block_sum_df<2>(pv2, red, v);
            if (threadIdx.x == 0) {
                atomicAdd(&RRn[2 * s], v[0]);
                atomicAdd(&RRn[2 * s + 1], v[1]);
            }
            __syncthreads();
        }
    };

    int k = a.k0;
    if (k == 0 || a.resume) {
        // z_k = M r_k for a new residual (the first, or a replaced one):
        // moments of r_k (parity k & 1), then the tables and <r_k, z_k>
        if (blockIdx.x == 0)
            for (int i = threadIdx.x; i < 2 * nseg; i += blockDim.x) a.RR[(k % 3) * 2 * nseg + i] = 0.0;
        for (int ri = rb; ri < re; ++ri) {
            const DfRun run = a.runs[ri];
            for (int base = run.lo; base < run.hi; base += blockDim.x) {
                if (base + (int)(threadIdx.x & ~31u) >= run.hi) continue;   // warp beyond the run
                const int row = base + threadIdx.x;
                const bool act = row < run.hi;
                const float d = act ? __ldg(dgp + row) : 0.f;
                const V rv = act ? a.r[row] : A::vzero();
                ml_moments0(a, run, base, k & 1, act, d, rv.x, rv.z, row, mbuf, nullptr);
            }
            __syncthreads();
            ml_restrict(a, run, mbuf, k & 1, nullptr);
        }
        grid.sync();
        phase_c(k, k % 3);
        grid.sync();
    }
    for (; k < a.max_iters; ++k) {
        const double* RRk = a.RR + (k % 3) * 2 * nseg;
        const double* RRm = (a.resume && k == a.k0) ? a.RRP : a.RR + ((k + 2) % 3) * 2 * nseg;
        const double* RDk = a.RD + (k % 3) * 2 * nseg;
        double* PQk = a.PQ + (k % 2) * 2 * nseg;
        // ---------------- phase B: p = z + beta p, q = A~ z + beta q, <p, q>
        if (blockIdx.x == 0) {   // slots that phases A and C of this iteration fill
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
                const bool d0 = done_of(RDk, a.THR, s, 0, a.dncp);
                const bool d1 = done_of(RDk, a.THR, s, 1, a.dncp);
                double b0 = 0.0, b1 = 0.0;
                if (k > 0) {
                    if (a.dncp) {
                        const double num = __ldcg(RRk + 2 * s) + __ldcg(RRk + 2 * s + 1);
                        const double den = __ldcg(RRm + 2 * s) + __ldcg(RRm + 2 * s + 1);
                        b0 = b1 = den > 0.0 ? num / den : 0.0;
                    } else {
                        b0 = __ldcg(RRm + 2 * s) > 0.0 ? __ldcg(RRk + 2 * s) / __ldcg(RRm + 2 * s) : 0.0;
                        b1 = __ldcg(RRm + 2 * s + 1) > 0.0 ? __ldcg(RRk + 2 * s + 1) / __ldcg(RRm + 2 * s + 1) : 0.0;
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
            const S beta0 = A::from_d(sc[slot][0]), beta1 = A::from_d(sc[slot][1]);
            S acc0 = A::zero(), acc1 = A::zero();
            int row = run.lo + threadIdx.x;
            int bn = 0, en = 0;
            if (row < run.hi) {
                bn = __ldg(rp + row);
                en = __ldg(rp + row + 1);
            }
            for (; row < run.hi; row += blockDim.x) {
                const int b = bn, e = en;
                const int nxt = row + blockDim.x;
                if (nxt < run.hi) {
                    bn = __ldg(rp + nxt);
                    en = __ldg(rp + nxt + 1);
                    if (en > bn) {
                        prefetch_l2(colp + bn);
                        prefetch_l2(valp + bn);
                        prefetch_l2(valp + en - 1);
                        prefetch_l2(a.p + nxt);
                        prefetch_l2(a.q + nxt);
                        prefetch_l2(a.z + nxt);
                    }
                }
                if (b == e) continue;   // fixed row
                S w0 = A::zero(), w1 = A::zero();
                int j = b;
                for (; j + 4 <= e; j += 4) {
                    int32_t c[4];
                    S v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        c[u] = __ldg(colp + j + u);
                        v[u] = __ldg(valp + j + u);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) spmv_entry<A>(c[u], v[u], a.z, w0, w1);
                }
                for (; j < e; ++j) spmv_entry<A>(__ldg(colp + j), __ldg(valp + j), a.z, w0, w1);
                const V zz = a.z[row];
                const V pp = a.p[row], qq = a.q[row];
                S px = A::cx(pp), py = A::cy(pp), qx = A::cx(qq), qy = A::cy(qq);
                if (!d0) {
                    px = A::fma(A::cx(zz), beta0, px);
                    qx = A::fma(w0, beta0, qx);
                    acc0 = A::fma(acc0, px, qx);
                }
                if (!d1) {
                    py = A::fma(A::cy(zz), beta1, py);
                    qy = A::fma(w1, beta1, qy);
                    acc1 = A::fma(acc1, py, qy);
                }
                a.p[row] = A::pack(px, py);
                a.q[row] = A::pack(qx, qy);
            }
            float2 pv[2] = {A::as_df(acc0), A::as_df(acc1)};
            double v[2];
            block_sum_df<2>(pv, red, v);
            if (threadIdx.x == 0) {
                atomicAdd(&PQk[2 * s], v[0]);
                atomicAdd(&PQk[2 * s + 1], v[1]);
                wrows += (unsigned long long)run.frows;
                wnnz += (unsigned long long)run.fnnz;
            }
        }
        if (threadIdx.x == 0 && any) *(volatile unsigned*)&a.ACT[k % 3] = 1u;
        grid.sync();
        // ---------------- phase A: x~ += alpha p, r -= alpha q, sum d r^2, moments of r
        if (blockIdx.x == 0) {
            double* zq = a.PQ + ((k + 1) % 2) * 2 * nseg;
            for (int i = threadIdx.x; i < 2 * nseg; i += blockDim.x) zq[i] = 0.0;
            if (threadIdx.x == 0) a.ACT[(k + 1) % 3] = 0;
        }
        double* RDn = a.RD + ((k + 1) % 3) * 2 * nseg;
        const int par = (k + 1) & 1;
        for (int ri = rb; ri < re; ++ri) {
            const DfRun run = a.runs[ri];
            const int s = run.seg, slot = ri & 1;
            if (threadIdx.x == 0) {
                const bool d0 = done_of(RDk, a.THR, s, 0, a.dncp);
                const bool d1 = done_of(RDk, a.THR, s, 1, a.dncp);
                double al0 = 0.0, al1 = 0.0;
                if (a.dncp) {
                    const double den = __ldcg(PQk + 2 * s) + __ldcg(PQk + 2 * s + 1);
                    al0 = al1 = den > 0.0 ? (__ldcg(RRk + 2 * s) + __ldcg(RRk + 2 * s + 1)) / den : 0.0;
                } else {
                    if (!d0) al0 = __ldcg(PQk + 2 * s) > 0.0 ? __ldcg(RRk + 2 * s) / __ldcg(PQk + 2 * s) : 0.0;
                    if (!d1) al1 = __ldcg(PQk + 2 * s + 1) > 0.0 ? __ldcg(RRk + 2 * s + 1) / __ldcg(PQk + 2 * s + 1) : 0.0;
                }
                sc[slot][0] = al0;
                sc[slot][1] = al1;
                sflag[slot][0] = d0 && d1;
                // the <r, z> this step used, kept for a resumed solve: per
                // coordinate, only while the coordinate is still iterating
                if (!d0) a.RRP[2 * s] = __ldcg(RRk + 2 * s);
                if (!d1) a.RRP[2 * s + 1] = __ldcg(RRk + 2 * s + 1);
            }
            __syncthreads();
            if (sflag[slot][0]) continue;
            const S al0 = A::from_d(sc[slot][0]), al1 = A::from_d(sc[slot][1]);
            const S nal0 = A::neg(al0), nal1 = A::neg(al1);
            const float* tab_here = tab_run == ri ? tab : nullptr;   // this run's frames, from the last phase C
            float rd0 = 0.f, rd1 = 0.f;
            for (int base = run.lo; base < run.hi; base += blockDim.x) {
                if (base + (int)(threadIdx.x & ~31u) >= run.hi) continue;   // warp beyond the run
                const int row = base + threadIdx.x;
                const bool act = row < run.hi;
                float d = 0.f, l0 = 0.f, l1 = 0.f;
                if (act) {
                    const int nxt = row + blockDim.x;
                    if (nxt < run.hi) {
                        prefetch_l2(a.x + nxt);
                        prefetch_l2(a.r + nxt);
                        prefetch_l2(a.p + nxt);
                        prefetch_l2(a.q + nxt);
                    }
                    d = __ldg(dgp + row);
                    if (d != 0.f) {
                        const V xx = a.x[row], rv = a.r[row];
                        const V pp = a.p[row], qq = a.q[row];
                        const S x0 = A::fma(A::cx(xx), al0, A::cx(pp)), x1 = A::fma(A::cy(xx), al1, A::cy(pp));
                        const S r0 = A::fma(A::cx(rv), nal0, A::cx(qq)), r1 = A::fma(A::cy(rv), nal1, A::cy(qq));
                        a.x[row] = A::pack(x0, x1);
                        a.r[row] = A::pack(r0, r1);
                        l0 = A::lead(r0);
                        l1 = A::lead(r1);
                        rd0 = fmaf(d * l0, l0, rd0);
                        rd1 = fmaf(d * l1, l1, rd1);
                    }
                }
                ml_moments0(a, run, base, par, act, d, l0, l1, row, mbuf, tab_here);
            }
            float2 pv[2] = {make_float2(rd0, 0.f), make_float2(rd1, 0.f)};
            double v[2];
            block_sum_df<2>(pv, red, v);
            if (threadIdx.x == 0) {
                atomicAdd(&RDn[2 * s], v[0]);
                atomicAdd(&RDn[2 * s + 1], v[1]);
            }
            __syncthreads();
            ml_restrict(a, run, mbuf, par, tab_here);
        }
        grid.sync();
        // ---------------- phase C: z = M r, <r, z>
        phase_c(k + 1, (k + 1) % 3);
        grid.sync();
        if (*(volatile unsigned*)&a.ACT[k % 3] == 0u) break;
    }
    if (threadIdx.x == 0) {
        if (wrows) atomicAdd(&a.work[0], wrows);
        if (wnnz) atomicAdd(&a.work[1], wnnz);
        if (blockIdx.x == 0) a.out_iters[0] = k;
    }
}

// ---------------------------------------------------------------- set-up

// piece centroids (FP64), one block per piece
__global__ void k_ml_centroid(const int64_t* __restrict__ voff, const int32_t* __restrict__ copy_vert,
                              const double* __restrict__ V, double* __restrict__ cen) {
    const int s = blockIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t i = voff[s] + threadIdx.x; i < voff[s + 1]; i += blockDim.x) {
        const int64_t g = copy_vert[i];
        v[0] += V[3 * g];
        v[1] += V[3 * g + 1];
        v[2] += V[3 * g + 2];
    }
    __shared__ double sh[3][256];
    for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double n = (double)(voff[s + 1] - voff[s]);
        for (int c = 0; c < 3; ++c) cen[3 * s + c] = n > 0 ? sh[c][0] / n : 0.0;
    }
}

__global__ void k_ml_xr(int64_t n, const int32_t* __restrict__ row_piece, const int32_t* __restrict__ copy_vert,
                        const double* __restrict__ V, const double* __restrict__ cen, float* __restrict__ xr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = row_piece[i];
    const int64_t g = copy_vert[i];
    for (int c = 0; c < 3; ++c) xr[3 * i + c] = (float)(V[3 * g + c] - cen[3 * s + c]);
}

// The piece and row range of block b of level l (binary search over bofs_l).
__device__ __forceinline__ void ml_block_rows(const int32_t* __restrict__ bofs_l, int nseg, int l,
                                              const int32_t* __restrict__ pvoff, int b, int* s_out, int* r0,
                                              int* r1) {
    int lo = 0, hi = nseg;   // the largest s with bofs_l[s] <= b
    while (hi - lo > 1) {
        const int m = (lo + hi) >> 1;
        if (bofs_l[m] <= b) lo = m;
        else hi = m;
    }
    const int s = lo;
    const int j = b - bofs_l[s];
    *s_out = s;
    *r0 = pvoff[s] + (j << ml_shift(l));
    *r1 = min(pvoff[s] + ((j + 1) << ml_shift(l)), pvoff[s + 1]);
}

// Block frame: centroid and 1 / RMS radius of the block's positions.
__global__ void __launch_bounds__(128) k_ml_geo(int l, int nb, int nseg, const int32_t* __restrict__ bofs_l,
                                                const int32_t* __restrict__ pvoff, const float* __restrict__ xr,
                                                float4* __restrict__ geo) {
    const int b = blockIdx.x;
    if (b >= nb) return;
    int s, r0, r1;
    ml_block_rows(bofs_l, nseg, l, pvoff, b, &s, &r0, &r1);
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const double x = xr[3 * (int64_t)i], y = xr[3 * (int64_t)i + 1], z = xr[3 * (int64_t)i + 2];
        v[0] += x;
        v[1] += y;
        v[2] += z;
        v[3] += x * x + y * y + z * z;
    }
    __shared__ double sh[4][128];
    for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double n = (double)max(r1 - r0, 1);
        const double cx = sh[0][0] / n, cy = sh[1][0] / n, cz = sh[2][0] / n;
        const double var = sh[3][0] / n - (cx * cx + cy * cy + cz * cz);
        const double rho = var > 0.0 ? sqrt(var) : 0.0;
        geo[b] = make_float4((float)cx, (float)cy, (float)cz, rho > 0.0 ? (float)(1.0 / rho) : 1.f);
    }
}

// The block's basis at row i (the same FP32 frame the iteration uses), in FP64.
template <int NF1>
__device__ __forceinline__ void ml_basis(const float* __restrict__ xr, float4 g, int i, double* m) {
    const double x = ((double)xr[3 * (int64_t)i] - (double)g.x) * (double)g.w;
    const double y = ((double)xr[3 * (int64_t)i + 1] - (double)g.y) * (double)g.w;
    const double z = ((double)xr[3 * (int64_t)i + 2] - (double)g.z) * (double)g.w;
    double t[10];
    mono10<double>(x, y, z, t);
#pragma unroll
    for (int f = 0; f < NF1; ++f) m[f] = t[f];
}

// Per block, in FP64: the Gram matrix C = sum_i d_i m_i m_i^T (PASS 0), the
// Laplacian part G_L = sum over the block's free rows and columns of
// m_i L_ij m_j^T (PASS 1, edge form: w_ij (m_i - m_j)(m_i - m_j)^T for edges
// inside the block, plus (weight to rows outside or fixed) m_i m_i^T), and
// the area part G_K = sum_i m_i (m_next / 2 - m_prev / 2)^T over boundary rows
// (PASS 2, full NF1 x NF1).  Symmetric parts are stored packed.
// One row's contribution to a block's Gram (PASS 0), edge-form Laplacian
// (PASS 1) or area (PASS 2) matrix; the block holds rows [r0, r1).
template <int NF1, int PASS>
__device__ __forceinline__ void gram_row(int i, int r0, int r1, const float* __restrict__ xr, float4 g,
                                         const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                         const double* __restrict__ val, const double* __restrict__ diag,
                                         const uint8_t* __restrict__ fixed, const int2* __restrict__ nbr,
                                         double* acc) {
    if (fixed[i]) return;
    double mi[NF1];
    ml_basis<NF1>(xr, g, i, mi);
    if (PASS == 0) {
        const double d = diag[i];
        int t = 0;
#pragma unroll
        for (int p = 0; p < NF1; ++p)
#pragma unroll
            for (int q = p; q < NF1; ++q) acc[t++] += d * mi[p] * mi[q];
    } else if (PASS == 1) {
        double dl = 0.0;   // weight to neighbours outside the block or fixed
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const int j = col[e];
            if (j == i) continue;
            const double w = -val[e];
            if (j < r0 || j >= r1 || fixed[j]) {
                dl += w;
                continue;
            }
            if (j < i) continue;   // each inside edge once
            double mj[NF1];
            ml_basis<NF1>(xr, g, j, mj);
            double dm[NF1];
#pragma unroll
            for (int p = 0; p < NF1; ++p) dm[p] = mi[p] - mj[p];
            int t = 0;
#pragma unroll
            for (int p = 0; p < NF1; ++p)
#pragma unroll
                for (int q = p; q < NF1; ++q) acc[t++] += w * dm[p] * dm[q];
        }
        int t = 0;
#pragma unroll
        for (int p = 0; p < NF1; ++p)
#pragma unroll
            for (int q = p; q < NF1; ++q) acc[t++] += dl * mi[p] * mi[q];
    } else {
        const int2 pn = nbr[i];   // (prev, next) loop rows; -1 inside
        if (pn.x < 0) return;
        double v[NF1];
#pragma unroll
        for (int q = 0; q < NF1; ++q) v[q] = 0.0;
        if (pn.y >= r0 && pn.y < r1 && !fixed[pn.y]) {
            double mn[NF1];
            ml_basis<NF1>(xr, g, pn.y, mn);
#pragma unroll
            for (int q = 0; q < NF1; ++q) v[q] += 0.5 * mn[q];
        }
        if (pn.x >= r0 && pn.x < r1 && !fixed[pn.x]) {
            double mp[NF1];
            ml_basis<NF1>(xr, g, pn.x, mp);
#pragma unroll
            for (int q = 0; q < NF1; ++q) v[q] -= 0.5 * mp[q];
        }
#pragma unroll
        for (int p = 0; p < NF1; ++p)
#pragma unroll
            for (int q = 0; q < NF1; ++q) acc[p * NF1 + q] += mi[p] * v[q];
    }
}

template <int NF1, int PASS>
__global__ void __launch_bounds__(128) k_ml_gram(int l, int nb, int nseg, const int32_t* __restrict__ bofs_l,
                                                 const int32_t* __restrict__ pvoff, const float* __restrict__ xr,
                                                 const float4* __restrict__ geo, const int32_t* __restrict__ rp,
                                                 const int32_t* __restrict__ col, const double* __restrict__ val,
                                                 const double* __restrict__ diag, const uint8_t* __restrict__ fixed,
                                                 const int2* __restrict__ nbr, double* __restrict__ out, int chunk) {
    constexpr int NS = NF1 * (NF1 + 1) / 2;
    constexpr int NO = PASS == 2 ? NF1 * NF1 : NS;
    const int b = blockIdx.x;
    if (b >= nb) return;
    int s, r0, r1;
    ml_block_rows(bofs_l, nseg, l, pvoff, b, &s, &r0, &r1);
    const float4 g = geo[b];
    // chunk blockIdx.y of the block's rows (chunk rows each); edges to rows of
    // other chunks of the same block still count as inside (r0, r1 unchanged)
    const int c0 = r0 + (int)blockIdx.y * chunk, c1 = min(r1, c0 + chunk);
    double acc[NO];
#pragma unroll
    for (int i = 0; i < NO; ++i) acc[i] = 0.0;
    for (int i = c0 + threadIdx.x; i < c1; i += blockDim.x)
        gram_row<NF1, PASS>(i, r0, r1, xr, g, rp, col, val, diag, fixed, nbr, acc);
    // block reduction: warps by shuffles, then across the block's warps (1 to 4)
    __shared__ double sh[4][NO];
#pragma unroll
    for (int i = 0; i < NO; ++i) {
        double v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][i] = v;
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    for (int i = threadIdx.x; i < NO; i += blockDim.x) {
        double v = sh[0][i];
        for (int w = 1; w < nw; ++w) v += sh[w][i];
        out[((int64_t)b * gridDim.y + blockIdx.y) * NO + i] = v;
    }
}

// out[b][i] = sum over the block's chunks of part[b][c][i], in chunk order.
__global__ void k_ml_chunk_sum(int64_t nbo, int no, int nchunk, const double* __restrict__ part,
                               double* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nbo) return;
    const int64_t b = t / no, i = t - b * no;
    double v = 0.0;
    for (int c = 0; c < nchunk; ++c) v += part[(b * nchunk + c) * no + i];
    out[t] = v;
}


// Upper-triangular R (n x n, row-major full storage) with C ~ R^T R, dropping
// every pivot at or below eps times its diagonal entry (that row of R stays 0).
__device__ void chol_drop(const double* C, int n, double eps, double* R) {
    for (int i = 0; i < n * n; ++i) R[i] = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = C[j * n + j];
        for (int k = 0; k < j; ++k) d -= R[k * n + j] * R[k * n + j];
        if (!(C[j * n + j] > 0.0) || !(d > eps * C[j * n + j])) continue;
        const double rj = sqrt(d);
        R[j * n + j] = rj;
        for (int i = j + 1; i < n; ++i) {
            double v = C[j * n + i];
            for (int k = 0; k < j; ++k) v -= R[k * n + j] * R[k * n + i];
            R[j * n + i] = v / rj;
        }
    }
}

// Inverse of the upper-triangular U on its kept indices (U_jj != 0); rows and
// columns of dropped indices stay 0.
__device__ void triu_inv(const double* U, int n, double* X) {
    for (int i = 0; i < n * n; ++i) X[i] = 0.0;
    for (int j = n - 1; j >= 0; --j) {
        if (U[j * n + j] == 0.0) continue;
        X[j * n + j] = 1.0 / U[j * n + j];
        for (int i = j - 1; i >= 0; --i) {
            if (U[i * n + i] == 0.0) continue;
            double v = 0.0;
            for (int k = i + 1; k <= j; ++k) v += U[i * n + k] * X[k * n + j];
            X[i * n + j] = -v / U[i * n + i];
        }
    }
}

// Per block (one warp, matrices in shared memory): T = R^-1 Lg^-1 with
// C = R^T R (orthonormalisation, nearly dependent monomials dropped) and
// R^-T G R^-1 = Lg^T Lg (null directions dropped), G = [[G_L, -G_K], [G_K, G_L]]
// over (x, y).  Packed to FP32; separable blocks (G_K = 0) store the NF1 x NF1
// factor of G_L.
template <int NF1>
__global__ void __launch_bounds__(32) k_ml_factor(int nb, const double* __restrict__ Cs,
                                                  const double* __restrict__ GL, const double* __restrict__ GK,
                                                  float* __restrict__ T, uint8_t* __restrict__ sep) {
    constexpr int NS = NF1 * (NF1 + 1) / 2;
    constexpr int NF = 2 * NF1;
    __shared__ double C[NF1 * NF1], R[NF1 * NF1], Ri[NF1 * NF1];
    __shared__ double G[NF * NF], W[NF * NF], Lg[NF * NF], Li[NF * NF];
    const int b = blockIdx.x;
    if (b >= nb) return;
    const int t = threadIdx.x;
    const double* gk = GK + (int64_t)b * NF1 * NF1;
    bool nz = false;
    for (int i = t; i < NF1 * NF1; i += 32) nz = nz || gk[i] != 0.0;
    const bool separable = !__any_sync(0xffffffffu, nz);
    const int n = separable ? NF1 : NF;
    for (int i = t; i < NS; i += 32) {   // unpack the packed symmetric C and G_L
        int p = 0, o = i;
        while (o >= NF1 - p) {
            o -= NF1 - p;
            ++p;
        }
        const int q = p + o;
        const double c = Cs[(int64_t)b * NS + i], g = GL[(int64_t)b * NS + i];
        C[p * NF1 + q] = C[q * NF1 + p] = c;
        G[p * n + q] = G[q * n + p] = g;
        if (!separable) G[(NF1 + p) * n + NF1 + q] = G[(NF1 + q) * n + NF1 + p] = g;
    }
    if (!separable)
        for (int i = t; i < NF1 * NF1; i += 32) {
            const int p = i / NF1, q = i % NF1;
            // the exact G_K is antisymmetric; averaging keeps G symmetric
            const double kpq = 0.5 * (gk[p * NF1 + q] - gk[q * NF1 + p]);
            G[(NF1 + p) * n + q] = kpq;    // y rows, x columns: + K
            G[p * n + NF1 + q] = -kpq;     // x rows, y columns: - K
        }
    __syncwarp();
    if (t == 0) {
        chol_drop(C, NF1, 1e-8, R);
        triu_inv(R, NF1, Ri);
    }
    __syncwarp();
    // Rf = blockdiag(Ri, Ri); Lg (scratch) = G Rf; W = Rf^T (G Rf)
    auto rf = [&](int i, int j) { return (i / NF1 == j / NF1) ? Ri[(i % NF1) * NF1 + j % NF1] : 0.0; };
    for (int e = t; e < n * n; e += 32) {
        const int i = e / n, j = e % n;
        double v = 0.0;
        for (int k = 0; k < n; ++k) v += G[i * n + k] * rf(k, j);
        Lg[e] = v;
    }
    __syncwarp();
    for (int e = t; e < n * n; e += 32) {
        const int i = e / n, j = e % n;
        double v = 0.0;
        for (int k = 0; k < n; ++k) v += rf(k, i) * Lg[k * n + j];
        W[e] = v;
    }
    __syncwarp();
    if (t == 0) {
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) W[i * n + j] = W[j * n + i] = 0.5 * (W[i * n + j] + W[j * n + i]);
        chol_drop(W, n, 1e-10, Lg);
        triu_inv(Lg, n, Li);
    }
    __syncwarp();
    // T = Rf Li (upper triangular), packed in FP32
    float* out = T + (int64_t)b * (NF * (NF + 1) / 2);
    for (int e = t; e < n * n; e += 32) {
        const int i = e / n, j = e % n;
        if (j < i) continue;
        double v = 0.0;
        for (int k = i; k <= j; ++k) v += rf(i, k) * Li[k * n + j];
        out[ut(i, j, n)] = (float)v;
    }
    if (t == 0) sep[b] = separable ? 1 : 0;
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, ceil_div(n, t)); }

template <int NF1>
void gram_level(cudaStream_t s, int l, int nb, int K, const DfSystem& D, const Part& P, const uint8_t* fixed,
                const float4* geo, float* T, uint8_t* sep) {
    constexpr int NS = NF1 * (NF1 + 1) / 2;
    DBuf<double> Cs, GL, GK;
    Cs.alloc((size_t)nb * NS, s);
    GL.alloc((size_t)nb * NS, s);
    GK.alloc((size_t)nb * NF1 * NF1, s);
    const int32_t* bofs_l = D.ml_bofs.p + l * (K + 1);
    // threads per CTA sized to the block's rows (16 * 4^l): 32 up to 64 rows,
    // 64 for 256, else 128; blocks above 1024 rows are cut into 1024-row
    // chunks, one CTA each, whose partial sums are added in chunk order
    constexpr int CHUNK = 1024;
    const int nthr = l <= 1 ? 32 : (l == 2 ? 64 : 128);
    const int brows = 16 << (2 * l);
    const int nchunk = brows > CHUNK ? brows / CHUNK : 1;
    const int chunk = nchunk > 1 ? CHUNK : brows;
    DBuf<double> part;
    if (nchunk > 1) part.alloc((size_t)nb * nchunk * NF1 * NF1, s);
    auto pass = [&](auto kern, int no, double* out) {
        double* dst = nchunk > 1 ? part.p : out;
        { kern<<<dim3(nb, nchunk), nthr, 0, s>>>(l, nb, K, bofs_l, D.ml_pvoff.p, D.ml_xr.p, geo, P.row_ptr.p, P.col.p,
                                                 P.val64.p, P.diag64.p, fixed, P.nb.p, dst, chunk); ::pgcp::note_launch(); }
        if (nchunk > 1) {
            const int64_t nbo = (int64_t)nb * no;
            { k_ml_chunk_sum<<<(unsigned)ceil_div(nbo, (int64_t)256), 256, 0, s>>>(nbo, no, nchunk, part.p, out);
              ::pgcp::note_launch(); }
        }
    };
    pass(k_ml_gram<NF1, 0>, NS, Cs.p);
    pass(k_ml_gram<NF1, 1>, NS, GL.p);
    pass(k_ml_gram<NF1, 2>, NF1 * NF1, GK.p);
    { k_ml_factor<NF1><<<nb, 32, 0, s>>>(nb, Cs.p, GL.p, GK.p, T, sep); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
}

}  // namespace

void ml_build(pgcp_ctx* ctx, Part& P, const uint8_t* fixed, DfSystem& D) {
    cudaStream_t s = ctx->stream;
    const int K = P.K;
    const int64_t n = D.n;
    // levels per piece and block offsets
    std::vector<int32_t> ltop(K), pvoff(K + 1);
    D.ml_bofs_h.assign((size_t)ML_MAXL * (K + 1), 0);
    int nl = 1;
    for (int i = 0; i < K; ++i) {
        const int64_t ni = P.voff[i + 1] - P.voff[i];
        int t = 0;
        while (t + 1 < ML_MAXL && ((int64_t)1 << ml_shift(t)) < ni) ++t;
        ltop[i] = t;
        nl = std::max(nl, t + 1);
        pvoff[i] = (int32_t)P.voff[i];
    }
    pvoff[K] = (int32_t)P.voff[K];
    D.ml_nl = nl;
    int64_t lofs = 0, tofs = 0;
    D.ml_row_bytes = 0.0;
    for (int l = 0; l < ML_MAXL; ++l) {
        int32_t* bo = D.ml_bofs_h.data() + (size_t)l * (K + 1);
        bo[0] = 0;
        for (int i = 0; i < K; ++i) {
            const int64_t ni = P.voff[i + 1] - P.voff[i];
            const int64_t nbi = l <= ltop[i] ? ceil_div(ni, (int64_t)1 << ml_shift(l)) : 0;
            bo[i + 1] = bo[i] + (int32_t)nbi;
        }
        D.ml_lofs[l] = lofs;
        D.ml_tofs[l] = tofs;
        lofs += bo[K];
        tofs += (int64_t)bo[K] * ml_ts(l);
        if (l < nl) {
            // per row and iteration: the factor (separable size), frame, moments written and read
            const int nf1 = ml_nf1(l);
            D.ml_row_bytes += (nf1 * (nf1 + 1) / 2 * 4.0 + 16.0 + 2.0 * ML_NM * 4.0) / (double)((int64_t)1 << ml_shift(l));
        }
    }
    D.ml_lofs[ML_MAXL] = lofs;
    D.ml_tofs[ML_MAXL] = tofs;
    D.ml_bofs.alloc(D.ml_bofs_h.size(), s);
    D.ml_ltop.alloc(K, s);
    D.ml_pvoff.alloc(K + 1, s);
    PGCP_CUDA(cudaMemcpyAsync(D.ml_bofs.p, D.ml_bofs_h.data(), D.ml_bofs_h.size() * sizeof(int32_t),
                              cudaMemcpyHostToDevice, s));
    PGCP_CUDA(cudaMemcpyAsync(D.ml_ltop.p, ltop.data(), K * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    PGCP_CUDA(cudaMemcpyAsync(D.ml_pvoff.p, pvoff.data(), (K + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    // positions in each piece's frame
    DBuf<double> cen;
    cen.alloc(3 * (size_t)K, s);
    DBuf<int64_t> dvoff;
    dvoff.alloc(K + 1, s);
    PGCP_CUDA(cudaMemcpyAsync(dvoff.p, P.voff.data(), (K + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    { k_ml_centroid<<<K, 256, 0, s>>>(dvoff.p, P.copy_vert.p, P.V.p, cen.p); ::pgcp::note_launch(); }
    D.ml_xr.alloc(3 * (size_t)n, s);
    { k_ml_xr<<<nblk(n), 256, 0, s>>>(n, P.row_piece.p, P.copy_vert.p, P.V.p, cen.p, D.ml_xr.p); ::pgcp::note_launch(); }
    D.ml_geo.alloc(std::max<int64_t>(lofs, 1), s);
    D.ml_T.alloc(std::max<int64_t>(tofs, 1), s);
    D.ml_sep.alloc(std::max<int64_t>(lofs, 1), s);
    D.ml_M.alloc(2 * std::max<int64_t>(lofs, 1) * ML_NM, s);
    D.ml_T.zero();
    for (int l = 0; l < nl; ++l) {
        const int nb = D.ml_bofs_h[(size_t)l * (K + 1) + K];
        if (nb == 0) continue;
        float4* geo = D.ml_geo.p + D.ml_lofs[l];
        { k_ml_geo<<<nb, 128, 0, s>>>(l, nb, K, D.ml_bofs.p + l * (K + 1), D.ml_pvoff.p, D.ml_xr.p, geo);
          ::pgcp::note_launch(); }
        if (l == 0) gram_level<4>(s, l, nb, K, D, P, fixed, geo, D.ml_T.p + D.ml_tofs[l], D.ml_sep.p + D.ml_lofs[l]);
        else gram_level<10>(s, l, nb, K, D, P, fixed, geo, D.ml_T.p + D.ml_tofs[l], D.ml_sep.p + D.ml_lofs[l]);
    }
    D.z.alloc((size_t)n * sizeof(float4), s);
    D.z.zero();
    int per_sm = 0;
    PGCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_pcg_ml<MLB>, RUN_THREADS, 0));
    if (per_sm <= 0) fail(PGCP_E_CUDA, "preconditioned PCG kernel cannot be resident");
    D.ml_per_sm = per_sm;
    PGCP_CUDA(cudaGetLastError());
    PGCP_CUDA(cudaStreamSynchronize(s));   // host tables go out of scope
}

void ml_launch(pgcp_ctx* ctx, Part& P, DfSystem& D, int k0, int cap, bool resume) {
    MlArgs a{};
    a.n = (int32_t)D.n;
    a.nseg = P.K;
    a.k0 = k0;
    a.resume = resume ? 1 : 0;
    a.RRP = D.RRP.p;
    a.max_iters = cap;
    a.dncp = D.dncp;
    a.nl = D.ml_nl;
    a.rp = D.rp.p;
    a.col = D.col.p;
    a.val = reinterpret_cast<const float2*>(D.val.p);
    a.dgn = D.dgn.p;
    a.x = reinterpret_cast<float4*>(D.x.p);
    a.r = reinterpret_cast<float4*>(D.r.p);
    a.p = reinterpret_cast<float4*>(D.p.p);
    a.q = reinterpret_cast<float4*>(D.q.p);
    a.z = reinterpret_cast<float4*>(D.z.p);
    a.runs = D.runs.p;
    a.run_off = D.run_off.p;
    a.RR = D.RR.p;
    a.RD = D.RD.p;
    a.PQ = D.PQ.p;
    a.ACT = D.ACT.p;
    a.THR = D.THR.p;
    a.out_iters = D.out_it.p;
    a.work = D.work.p;
    a.bofs = D.ml_bofs.p;
    a.ltop = D.ml_ltop.p;
    a.pvoff = D.ml_pvoff.p;
    a.xr = D.ml_xr.p;
    a.geo = D.ml_geo.p;
    a.T = D.ml_T.p;
    a.sep = D.ml_sep.p;
    a.M = D.ml_M.p;
    a.mstride = std::max<int64_t>(D.ml_lofs[ML_MAXL], 1);
    for (int l = 0; l <= ML_MAXL; ++l) {
        a.lofs[l] = D.ml_lofs[l];
        a.tofs[l] = D.ml_tofs[l];
    }
    void* args[] = {(void*)&a};
    PGCP_CUDA(cudaLaunchCooperativeKernel((const void*)k_pcg_ml<MLB>, dim3(D.grid), dim3(RUN_THREADS), args, 0,
                                          ctx->stream));
    ::pgcp::note_launch();
}

}  // namespace pgcp
