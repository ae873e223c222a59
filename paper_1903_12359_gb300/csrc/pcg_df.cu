// Run-based persistent PCG for the batched local (DNCP) and Laplace systems,
// inside FP64 iterative refinement (Sections 4.2 and 4.5 define the systems;
// the solver is this library's).
//
// Two arithmetics share one kernel template:
// * double-float (ArithDF): a number is the unevaluated sum hi + lo of two
//   floats, about 48 significant bits, computed with error-free
//   transformations on the FP32 pipe -- TwoSum (Knuth), Fast2Sum (Dekker) and
//   the FMA-based TwoProduct (Ogita, Rump and Oishi, "Accurate sum and dot
//   product", 2005).  The __f*_rn intrinsics keep the compiler from
//   contracting them.  GB300's FP64 pipe issues 2 DFMA per SM per cycle
//   against 128 FFMA, and an FP64 PCG over these meshes is bound by it, while
//   FP32 alone is too coarse for the DNCP system (its refinement stalls).
// * FP32 (ArithF32): FP32 values and FP32 accumulation, for the Laplace solve.
// The FP64 residual outside decides convergence in both.
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
// run and phase, on the FP32 pipe in double-float).  Per iteration:
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

#include "df_arith.cuh"
#include "pgcp_internal.h"

namespace cg = cooperative_groups;

namespace pgcp {

namespace {

using namespace dfa;

// Iterations per launch of a static-schedule solve; the runs are rebuilt over
// the unconverged pieces between launches (see df_solve).
constexpr int REBALANCE_ITERS = 256;
// Resident blocks per SM the kernel is compiled for (MINB): 4 caps it at 64
// registers (32 warps per SM), 3 at 80 (24 warps, no spills in double-float).

template <typename A>
struct RunArgs {
    int32_t n;
    int32_t nseg;
    const int32_t* __restrict__ rp;
    const int32_t* __restrict__ col;        // ~c marks a cross (area-term) entry
    const typename A::S* __restrict__ val;  // scaled values
    const float* __restrict__ dgn;          // diagonal of A (0 at fixed rows), for the unscaled norm
    typename A::V* x;   // x~
    typename A::V* r;
    typename A::V* p;
    typename A::V* q;
    const DfRun* __restrict__ runs;
    const int32_t* __restrict__ run_off;    // [grid + 1]
    double* RR;    // [3][2 nseg] scaled <r, r>
    double* RD;    // [3][2 nseg] unscaled sum d r^2
    double* PQ;    // [2][2 nseg]
    unsigned int* ACT;                  // [3]
    const double* __restrict__ THR;     // [2 nseg] thresholds on RD
    int32_t* out_iters;
    int32_t max_iters;
    int32_t dncp;
    unsigned long long* work;           // [2] free rows, stored entries, summed over iterations
    // single-reduction schedule (k_pcg_cg1): second residual slot, A r in two
    // slots, s = A p in two slots (slot 0 is q), <r, A r> accumulators [3][2 nseg]
    typename A::V* r1;
    typename A::V* w0;
    typename A::V* w1;
    typename A::V* s1;
    double* DL;
    // dynamic schedule (k_pcg_dyn)
    const DfRun* __restrict__ chunks;   // RUN_THREADS-row chunks inside pieces
    int32_t nchunks;
    const int32_t* __restrict__ nch;    // [nseg] chunks per piece
    unsigned int* CTR;                  // [4] chunk counters (phase B of k: 2k % 4, phase A: 2k+1 % 4)
    unsigned int* CNTB;                 // [2][nseg] chunks of a piece reduced in phase B
    unsigned int* CNTA;                 // [2][nseg] ... in phase A
    double* ALPHA;                      // [2][2 nseg]
    double* BETA;                       // [2][2 nseg]
    unsigned int* DONEF;                // [2 nseg] coordinate converged (monotonic)
    // static schedule: first iteration of this launch (a solve may run as several
    // launches, the later ones over the rows of the unconverged pieces only)
    int32_t k0;
    // k0 continues a solve whose residual was replaced: beta of iteration k0
    // divides by RRP, each piece's <r, r> of its last active iteration
    int32_t resume;
    double* RRP;                        // [2 nseg]
    // deterministic mode (static schedule): every run stores its partial sums,
    // and a piece's total is summed over its runs in run order where needed
    int32_t det;
    int32_t nruns;
    const int32_t* __restrict__ prun;   // [2 nseg] first and one-past-last run of each piece
    double* PRR;                        // [3][nruns][2] scaled <r, r> per run
    double* PRD;                        // [3][nruns][2] unscaled sum d r^2 per run
    double* PPQ;                        // [2][nruns][2] <p, q> per run
    int32_t* RDONE;                     // [nruns][2] coordinate converged (set once, by the run's block)
    double* CRR;                        // [nruns][2] the piece's scaled <r, r> of the latest phase B
};

// NQ sums of src[q][2 i] over the runs i in [r0, r1), in a fixed order: lane l
// adds runs r0 + l, r0 + l + 32, ... in sequence, then a butterfly over the
// lanes.  IEEE addition is commutative, so every lane ends with the same bits,
// and every warp that sums the same runs gets the same totals.  The NQ loads
// of a step are issued together.  Full warp.
template <int NQ>
__device__ __forceinline__ void ordered_sums(const double* const* src, int r0, int r1, double* out) {
    double v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = 0.0;
    for (int i = r0 + (int)(threadIdx.x & 31); i < r1; i += 32) {
        double t[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) t[q] = __ldcg(src[q] + 2 * i);
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] += t[q];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
#pragma unroll
    for (int q = 0; q < NQ; ++q) out[q] = v[q];
}

// Accumulators written by other blocks (atomics, then a grid sync) are read
// through L2 (__ldcg): another SM's L1 may hold an older line.
__device__ __forceinline__ bool piece_done(const double* RD, const double* THR, int s, int c, bool dncp) {
    if (dncp) return __ldcg(RD + 2 * s) + __ldcg(RD + 2 * s + 1) <= THR[2 * s] + THR[2 * s + 1];
    return __ldcg(RD + 2 * s + c) <= THR[2 * s + c];
}

template <typename A, int MINB>
__global__ void __launch_bounds__(RUN_THREADS, MINB) k_pcg_run(RunArgs<A> a) {
    using S = typename A::S;
    using V = typename A::V;
    cg::grid_group grid = cg::this_grid();
    __shared__ float2 red[4 * (RUN_THREADS / 32)];
    __shared__ double sc[2][2];
    __shared__ int sflag[2][2];
    const int nseg = a.nseg;
    const int rb = a.run_off[blockIdx.x], re = a.run_off[blockIdx.x + 1];
    const int32_t* __restrict__ rp = a.rp;
    const int32_t* __restrict__ colp = a.col;
    const S* __restrict__ valp = a.val;
    const float* __restrict__ dgp = a.dgn;
    unsigned long long wrows = 0, wnnz = 0;
    int k = a.k0;
    for (; k < a.max_iters; ++k) {
        const double* RRk = a.RR + (k % 3) * 2 * nseg;
        const double* RRm = (a.resume && k == a.k0) ? a.RRP : a.RR + ((k + 2) % 3) * 2 * nseg;
        const double* RDk = a.RD + (k % 3) * 2 * nseg;
        double* PQk = a.PQ + (k % 2) * 2 * nseg;
        // ---------------- phase B: p = r + beta p, q = A~ r + beta q, <p, q>
        if (blockIdx.x == 0) {   // clear the slots phase A of this iteration fills
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
            if (a.det) {
                if (threadIdx.x < 32) {   // warp 0: ordered sums over the piece's runs
                    const int r0 = a.prun[2 * s], r1 = a.prun[2 * s + 1], nr2 = 2 * a.nruns;
                    bool d0 = __ldcg(a.RDONE + 2 * ri) != 0, d1 = __ldcg(a.RDONE + 2 * ri + 1) != 0;
                    double b0 = 0.0, b1 = 0.0, t[4] = {0.0, 0.0, 0.0, 0.0};
                    if (!(d0 && d1)) {
                        // this iteration's sum d r^2 and <r, r>; the previous <r, r> is cached
                        const double* PRDk = a.PRD + (k % 3) * nr2;
                        const double* PRRk = a.PRR + (k % 3) * nr2;
                        const double* src[4] = {PRDk, PRDk + 1, PRRk, PRRk + 1};
                        ordered_sums<4>(src, r0, r1, t);
                        if (a.dncp) {
                            const bool dn = t[0] + t[1] <= a.THR[2 * s] + a.THR[2 * s + 1];
                            d0 = d0 || dn;
                            d1 = d1 || dn;
                        } else {
                            d0 = d0 || t[0] <= a.THR[2 * s];
                            d1 = d1 || t[1] <= a.THR[2 * s + 1];
                        }
                        if (k > 0 && !(d0 && d1)) {
                            const double m0 = __ldcg(a.CRR + 2 * ri), m1 = __ldcg(a.CRR + 2 * ri + 1);
                            if (a.dncp) {
                                const double num = t[2] + t[3], den = m0 + m1;
                                b0 = b1 = den > 0.0 ? num / den : 0.0;
                            } else {
                                b0 = m0 > 0.0 ? t[2] / m0 : 0.0;
                                b1 = m1 > 0.0 ? t[3] / m1 : 0.0;
                            }
                        }
                    }
                    __syncwarp();   // every lane has read CRR before lane 0 replaces it
                    if (threadIdx.x == 0) {
                        if (!(d0 && d1)) {
                            a.CRR[2 * ri] = t[2];
                            a.CRR[2 * ri + 1] = t[3];
                        }
                        if (d0) a.RDONE[2 * ri] = 1;
                        if (d1) a.RDONE[2 * ri + 1] = 1;
                        sc[slot][0] = b0;
                        sc[slot][1] = b1;
                        sflag[slot][0] = d0;
                        sflag[slot][1] = d1;
                    }
                }
            } else if (threadIdx.x == 0) {
                const bool d0 = piece_done(RDk, a.THR, s, 0, a.dncp);
                const bool d1 = piece_done(RDk, a.THR, s, 1, a.dncp);
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
            __syncthreads();   // scalars of this run (double-buffered by run parity)
            const bool d0 = sflag[slot][0], d1 = sflag[slot][1];
            if (d0 && d1) continue;
            any = true;
            const S beta0 = A::from_d(sc[slot][0]), beta1 = A::from_d(sc[slot][1]);
            S acc0 = A::zero(), acc1 = A::zero();
            // software pipeline over this thread's rows: the next row's bounds are
            // loaded, and its vectors and matrix slice prefetched into L2, before
            // the current row's SpMV (prefetches hold no registers)
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
                        prefetch_l2(a.r + nxt);
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
                    for (int u = 0; u < 4; ++u) spmv_entry<A>(c[u], v[u], a.r, w0, w1);
                }
                for (; j < e; ++j) spmv_entry<A>(__ldg(colp + j), __ldg(valp + j), a.r, w0, w1);
                const V rr = a.r[row];
                const V pp = a.p[row], qq = a.q[row];
                S px = A::cx(pp), py = A::cy(pp), qx = A::cx(qq), qy = A::cy(qq);
                if (!d0) {
                    px = A::fma(A::cx(rr), beta0, px);
                    qx = A::fma(w0, beta0, qx);
                    acc0 = A::fma(acc0, px, qx);
                }
                if (!d1) {
                    py = A::fma(A::cy(rr), beta1, py);
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
                if (a.det) {
                    double* o = a.PPQ + (k % 2) * 2 * a.nruns + 2 * ri;
                    o[0] = v[0];
                    o[1] = v[1];
                } else {
                    atomicAdd(&PQk[2 * s], v[0]);
                    atomicAdd(&PQk[2 * s + 1], v[1]);
                }
                wrows += (unsigned long long)run.frows;
                wnnz += (unsigned long long)run.fnnz;
            }
        }
        if (threadIdx.x == 0 && any) *(volatile unsigned*)&a.ACT[k % 3] = 1u;
        grid.sync();
        // ---------------- phase A: x~ += alpha p, r -= alpha q, norms
        if (blockIdx.x == 0) {   // clear the slots phase B of the next iteration fills
            double* z = a.PQ + ((k + 1) % 2) * 2 * nseg;
            for (int i = threadIdx.x; i < 2 * nseg; i += blockDim.x) z[i] = 0.0;
            if (threadIdx.x == 0) a.ACT[(k + 1) % 3] = 0;
        }
        double* RRn = a.RR + ((k + 1) % 3) * 2 * nseg;
        double* RDn = a.RD + ((k + 1) % 3) * 2 * nseg;
        for (int ri = rb; ri < re; ++ri) {
            const DfRun run = a.runs[ri];
            const int s = run.seg, slot = ri & 1;
            if (a.det) {
                if (threadIdx.x < 32) {   // warp 0; the converged flags are phase B's of this iteration
                    const int r0 = a.prun[2 * s], r1 = a.prun[2 * s + 1], nr2 = 2 * a.nruns;
                    const bool d0 = __ldcg(a.RDONE + 2 * ri) != 0, d1 = __ldcg(a.RDONE + 2 * ri + 1) != 0;
                    double al0 = 0.0, al1 = 0.0;
                    if (!(d0 && d1)) {
                        // <r, r> of this iteration from phase B's cache; <p, q> summed now
                        const double n0 = __ldcg(a.CRR + 2 * ri), n1 = __ldcg(a.CRR + 2 * ri + 1);
                        const double* PPQk = a.PPQ + (k % 2) * nr2;
                        const double* src[2] = {PPQk, PPQk + 1};
                        double t[2];
                        ordered_sums<2>(src, r0, r1, t);
                        const double q0 = t[0], q1 = t[1];
                        if (a.dncp) {
                            const double den = q0 + q1;
                            al0 = al1 = den > 0.0 ? (n0 + n1) / den : 0.0;
                        } else {
                            if (!d0) al0 = q0 > 0.0 ? n0 / q0 : 0.0;
                            if (!d1) al1 = q1 > 0.0 ? n1 / q1 : 0.0;
                        }
                    }
                    if (threadIdx.x == 0) {
                        sc[slot][0] = al0;
                        sc[slot][1] = al1;
                        sflag[slot][0] = d0 && d1;
                    }
                }
            } else if (threadIdx.x == 0) {
                const bool d0 = piece_done(RDk, a.THR, s, 0, a.dncp);
                const bool d1 = piece_done(RDk, a.THR, s, 1, a.dncp);
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
                // the <r, r> this step used, kept for a resumed solve: per
                // coordinate, only while the coordinate is still iterating
                if (!d0) a.RRP[2 * s] = __ldcg(RRk + 2 * s);
                if (!d1) a.RRP[2 * s + 1] = __ldcg(RRk + 2 * s + 1);
            }
            __syncthreads();
            if (sflag[slot][0]) continue;
            const S al0 = A::from_d(sc[slot][0]), al1 = A::from_d(sc[slot][1]);
            const S nal0 = A::neg(al0), nal1 = A::neg(al1);
            S rr0 = A::zero(), rr1 = A::zero();
            float rd0 = 0.f, rd1 = 0.f;
            for (int row = run.lo + threadIdx.x; row < run.hi; row += blockDim.x) {
                const int nxt = row + blockDim.x;
                if (nxt < run.hi) {   // next row's streams into L2 (no registers held)
                    prefetch_l2(a.x + nxt);
                    prefetch_l2(a.r + nxt);
                    prefetch_l2(a.p + nxt);
                    prefetch_l2(a.q + nxt);
                }
                const float d = __ldg(dgp + row);
                if (d == 0.f) continue;   // fixed row
                const V xx = a.x[row], rv = a.r[row];
                const V pp = a.p[row], qq = a.q[row];
                const S x0 = A::fma(A::cx(xx), al0, A::cx(pp)), x1 = A::fma(A::cy(xx), al1, A::cy(pp));
                const S r0 = A::fma(A::cx(rv), nal0, A::cx(qq)), r1 = A::fma(A::cy(rv), nal1, A::cy(qq));
                a.x[row] = A::pack(x0, x1);
                a.r[row] = A::pack(r0, r1);
                rr0 = A::fma(rr0, r0, r0);
                rr1 = A::fma(rr1, r1, r1);
                const float l0 = A::lead(r0), l1 = A::lead(r1);
                rd0 = fmaf(d * l0, l0, rd0);
                rd1 = fmaf(d * l1, l1, rd1);
            }
            float2 pv[4] = {A::as_df(rr0), A::as_df(rr1), make_float2(rd0, 0.f), make_float2(rd1, 0.f)};
            double v[4];
            block_sum_df<4>(pv, red, v);
            if (threadIdx.x == 0 && a.det) {
                double* o = a.PRR + ((k + 1) % 3) * 2 * a.nruns + 2 * ri;
                double* d = a.PRD + ((k + 1) % 3) * 2 * a.nruns + 2 * ri;
                o[0] = v[0];
                o[1] = v[1];
                d[0] = v[2];
                d[1] = v[3];
            } else if (threadIdx.x == 0) {
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

// Dynamic schedule.  Blocks take RUN_THREADS-row chunks (inside one piece)
// from a global counter; the next chunk's index and descriptor are fetched
// while the current chunk runs.  Each block reduces its partial sums once per
// piece it touched; the block that completes a piece's sum (counting chunks)
// computes the piece's alpha (phase B) or beta and converged flags (phase A)
// for everyone, so no block waits on scalars at a chunk start.
template <typename A, int MINB>
__global__ void __launch_bounds__(RUN_THREADS, MINB) k_pcg_dyn(RunArgs<A> a) {
    using S = typename A::S;
    using V = typename A::V;
    cg::grid_group grid = cg::this_grid();
    __shared__ float2 red[4 * (RUN_THREADS / 32)];
    __shared__ int s_idx[3];        // chunk ring: current, next, the one after
    __shared__ DfRun s_chunk[3];
    const int nseg = a.nseg;
    const int32_t* __restrict__ rp = a.rp;
    const int32_t* __restrict__ colp = a.col;
    const S* __restrict__ valp = a.val;
    const float* __restrict__ dgp = a.dgn;
    unsigned long long wrows = 0, wnnz = 0;
    int k = 0;
    for (; k < a.max_iters; ++k) {
        const double* RRk = a.RR + (k % 3) * 2 * nseg;
        double* RRn = a.RR + ((k + 1) % 3) * 2 * nseg;
        double* RDn = a.RD + ((k + 1) % 3) * 2 * nseg;
        double* PQk = a.PQ + (k % 2) * 2 * nseg;
        const double* BETk = a.BETA + (k % 2) * 2 * nseg;
        double* BETn = a.BETA + ((k + 1) % 2) * 2 * nseg;
        double* ALPk = a.ALPHA + (k % 2) * 2 * nseg;
        unsigned* CB = a.CNTB + (k % 2) * nseg;
        unsigned* CA = a.CNTA + (k % 2) * nseg;
        // ---------------- phase B: p = r + beta p, q = A~ r + beta q, <p, q>
        if (blockIdx.x == 0) {   // slots that this iteration's phase A and the next phase B fill
            for (int i = threadIdx.x; i < 2 * nseg; i += blockDim.x) {
                RRn[i] = 0.0;
                RDn[i] = 0.0;
            }
            for (int i = threadIdx.x; i < nseg; i += blockDim.x) a.CNTB[((k + 1) % 2) * nseg + i] = 0u;
            if (threadIdx.x == 0) a.CTR[(2 * k + 2) % 4] = 0u;
        }
        bool any = false;
        {
            unsigned* ctr = a.CTR + (2 * k) % 4;
            if (threadIdx.x == 0) {
                for (int t = 0; t < 2; ++t) {
                    const int c = (int)atomicAdd(ctr, 1u);
                    s_idx[t] = c;
                    if (c < a.nchunks) s_chunk[t] = a.chunks[c];
                }
            }
            __syncthreads();
            int seg = -1, m = 0;
            S acc0 = A::zero(), acc1 = A::zero();
            auto flush = [&]() {
                float2 pv[2] = {A::as_df(acc0), A::as_df(acc1)};
                double v[2];
                block_sum_df<2>(pv, red, v);
                if (threadIdx.x == 0) {
                    atomicAdd(&PQk[2 * seg], v[0]);
                    atomicAdd(&PQk[2 * seg + 1], v[1]);
                    __threadfence();
                    const unsigned old = atomicAdd(&CB[seg], (unsigned)m);
                    if (old + (unsigned)m == (unsigned)a.nch[seg]) {   // this block completed <p, q>
                        __threadfence();
                        const double pq0 = __ldcg(PQk + 2 * seg), pq1 = __ldcg(PQk + 2 * seg + 1);
                        const double rr0 = __ldcg(RRk + 2 * seg), rr1 = __ldcg(RRk + 2 * seg + 1);
                        double al0, al1;
                        if (a.dncp) {
                            const double den = pq0 + pq1;
                            al0 = al1 = den > 0.0 ? (rr0 + rr1) / den : 0.0;
                        } else {
                            al0 = (!__ldcg(a.DONEF + 2 * seg) && pq0 > 0.0) ? rr0 / pq0 : 0.0;
                            al1 = (!__ldcg(a.DONEF + 2 * seg + 1) && pq1 > 0.0) ? rr1 / pq1 : 0.0;
                        }
                        __stcg(ALPk + 2 * seg, al0);
                        __stcg(ALPk + 2 * seg + 1, al1);
                    }
                }
            };
            // this thread's row bounds in the current chunk, loaded one chunk ahead
            int bcur = 0, ecur = 0;
            if (s_idx[0] < a.nchunks && s_chunk[0].lo + (int)threadIdx.x < s_chunk[0].hi) {
                bcur = __ldg(rp + s_chunk[0].lo + threadIdx.x);
                ecur = __ldg(rp + s_chunk[0].lo + threadIdx.x + 1);
            }
            for (int it = 0;; ++it) {
                const int c = s_idx[it % 3];
                if (c >= a.nchunks) break;
                const DfRun ch = s_chunk[it % 3];
                const int cn = s_idx[(it + 1) % 3];
                int nxt = 0;
                if (threadIdx.x == 0) nxt = (int)atomicAdd(ctr, 1u);   // two chunks ahead, in flight
                // next chunk: this thread's row bounds, and its vectors into L2
                int bn = 0, en = 0, nrow = -1;
                if (cn < a.nchunks) {
                    const DfRun chn = s_chunk[(it + 1) % 3];
                    if (chn.lo + (int)threadIdx.x < chn.hi) {
                        nrow = chn.lo + threadIdx.x;
                        bn = __ldg(rp + nrow);
                        en = __ldg(rp + nrow + 1);
                        prefetch_l2(a.p + nrow);
                        prefetch_l2(a.q + nrow);
                        prefetch_l2(a.r + nrow);
                    }
                }
                if (ch.seg != seg) {   // block-uniform
                    if (seg >= 0 && m > 0) flush();
                    seg = ch.seg;
                    m = 0;
                    acc0 = A::zero();
                    acc1 = A::zero();
                }
                const bool d0 = __ldcg(a.DONEF + 2 * seg) != 0u, d1 = __ldcg(a.DONEF + 2 * seg + 1) != 0u;
                if (!(d0 && d1)) {
                    any = true;
                    ++m;
                    const S beta0 = A::from_d(__ldcg(BETk + 2 * seg)), beta1 = A::from_d(__ldcg(BETk + 2 * seg + 1));
                    const int row = ch.lo + threadIdx.x;
                    const int b = bcur, e = ecur;
                    if (row < ch.hi && b < e) {
                        S w0 = A::zero(), w1 = A::zero();
                        int j = b;
                        for (; j + 4 <= e; j += 4) {
                            int32_t cc[4];
                            S v[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                cc[u] = __ldg(colp + j + u);
                                v[u] = __ldg(valp + j + u);
                            }
#pragma unroll
                            for (int u = 0; u < 4; ++u) spmv_entry<A>(cc[u], v[u], a.r, w0, w1);
                        }
                        for (; j < e; ++j) spmv_entry<A>(__ldg(colp + j), __ldg(valp + j), a.r, w0, w1);
                        const V rr = a.r[row];
                        const V pp = a.p[row], qq = a.q[row];
                        S px = A::cx(pp), py = A::cy(pp), qx = A::cx(qq), qy = A::cy(qq);
                        if (!d0) {
                            px = A::fma(A::cx(rr), beta0, px);
                            qx = A::fma(w0, beta0, qx);
                            acc0 = A::fma(acc0, px, qx);
                        }
                        if (!d1) {
                            py = A::fma(A::cy(rr), beta1, py);
                            qy = A::fma(w1, beta1, qy);
                            acc1 = A::fma(acc1, py, qy);
                        }
                        a.p[row] = A::pack(px, py);
                        a.q[row] = A::pack(qx, qy);
                    }
                    if (threadIdx.x == 0) {
                        wrows += (unsigned long long)ch.frows;
                        wnnz += (unsigned long long)ch.fnnz;
                    }
                }
                if (nrow >= 0 && en > bn) {   // the next row's matrix slice into L2
                    prefetch_l2(colp + bn);
                    prefetch_l2(valp + bn);
                    prefetch_l2(valp + en - 1);
                }
                bcur = bn;
                ecur = en;
                if (threadIdx.x == 0) {
                    s_idx[(it + 2) % 3] = nxt;
                    if (nxt < a.nchunks) s_chunk[(it + 2) % 3] = a.chunks[nxt];
                }
                __syncthreads();
            }
            if (seg >= 0 && m > 0) flush();
        }
        if (threadIdx.x == 0 && any) *(volatile unsigned*)&a.ACT[k % 3] = 1u;
        grid.sync();
        // ---------------- phase A: x~ += alpha p, r -= alpha q, norms
        if (blockIdx.x == 0) {
            double* z = a.PQ + ((k + 1) % 2) * 2 * nseg;
            for (int i = threadIdx.x; i < 2 * nseg; i += blockDim.x) z[i] = 0.0;
            for (int i = threadIdx.x; i < nseg; i += blockDim.x) a.CNTA[((k + 1) % 2) * nseg + i] = 0u;
            if (threadIdx.x == 0) {
                a.ACT[(k + 1) % 3] = 0;
                a.CTR[(2 * k + 3) % 4] = 0u;
            }
        }
        {
            unsigned* ctr = a.CTR + (2 * k + 1) % 4;
            if (threadIdx.x == 0) {
                for (int t = 0; t < 2; ++t) {
                    const int c = (int)atomicAdd(ctr, 1u);
                    s_idx[t] = c;
                    if (c < a.nchunks) s_chunk[t] = a.chunks[c];
                }
            }
            __syncthreads();
            int seg = -1, m = 0;
            S rr0 = A::zero(), rr1 = A::zero();
            float rd0 = 0.f, rd1 = 0.f;
            auto flush = [&]() {
                float2 pv[4] = {A::as_df(rr0), A::as_df(rr1), make_float2(rd0, 0.f), make_float2(rd1, 0.f)};
                double v[4];
                block_sum_df<4>(pv, red, v);
                if (threadIdx.x == 0) {
                    atomicAdd(&RRn[2 * seg], v[0]);
                    atomicAdd(&RRn[2 * seg + 1], v[1]);
                    atomicAdd(&RDn[2 * seg], v[2]);
                    atomicAdd(&RDn[2 * seg + 1], v[3]);
                    __threadfence();
                    const unsigned old = atomicAdd(&CA[seg], (unsigned)m);
                    if (old + (unsigned)m == (unsigned)a.nch[seg]) {   // this block completed the norms
                        __threadfence();
                        const double n0 = __ldcg(RRn + 2 * seg), n1 = __ldcg(RRn + 2 * seg + 1);
                        const double o0 = __ldcg(RRk + 2 * seg), o1 = __ldcg(RRk + 2 * seg + 1);
                        const double e0 = __ldcg(RDn + 2 * seg), e1 = __ldcg(RDn + 2 * seg + 1);
                        const double t0 = a.THR[2 * seg], t1 = a.THR[2 * seg + 1];
                        if (a.dncp) {
                            const double bt = (o0 + o1) > 0.0 ? (n0 + n1) / (o0 + o1) : 0.0;
                            __stcg(BETn + 2 * seg, bt);
                            __stcg(BETn + 2 * seg + 1, bt);
                            if (e0 + e1 <= t0 + t1) {
                                __stcg(a.DONEF + 2 * seg, 1u);
                                __stcg(a.DONEF + 2 * seg + 1, 1u);
                            }
                        } else {
                            __stcg(BETn + 2 * seg, o0 > 0.0 ? n0 / o0 : 0.0);
                            __stcg(BETn + 2 * seg + 1, o1 > 0.0 ? n1 / o1 : 0.0);
                            if (e0 <= t0) __stcg(a.DONEF + 2 * seg, 1u);
                            if (e1 <= t1) __stcg(a.DONEF + 2 * seg + 1, 1u);
                        }
                    }
                }
            };
            for (int it = 0;; ++it) {
                const int c = s_idx[it % 3];
                if (c >= a.nchunks) break;
                const DfRun ch = s_chunk[it % 3];
                const int cn = s_idx[(it + 1) % 3];
                int nxt = 0;
                if (threadIdx.x == 0) nxt = (int)atomicAdd(ctr, 1u);
                if (cn < a.nchunks) {   // next chunk's row streams into L2
                    const DfRun chn = s_chunk[(it + 1) % 3];
                    const int nrow = chn.lo + threadIdx.x;
                    if (nrow < chn.hi) {
                        prefetch_l2(a.x + nrow);
                        prefetch_l2(a.r + nrow);
                        prefetch_l2(a.p + nrow);
                        prefetch_l2(a.q + nrow);
                    }
                }
                if (ch.seg != seg) {
                    if (seg >= 0 && m > 0) flush();
                    seg = ch.seg;
                    m = 0;
                    rr0 = A::zero();
                    rr1 = A::zero();
                    rd0 = rd1 = 0.f;
                }
                const bool d0 = __ldcg(a.DONEF + 2 * seg) != 0u, d1 = __ldcg(a.DONEF + 2 * seg + 1) != 0u;
                if (!(d0 && d1)) {
                    ++m;
                    const S al0 = A::from_d(__ldcg(ALPk + 2 * seg)), al1 = A::from_d(__ldcg(ALPk + 2 * seg + 1));
                    const int row = ch.lo + threadIdx.x;
                    if (row < ch.hi) {
                        const float d = __ldg(dgp + row);
                        if (d != 0.f) {
                            const V xx = a.x[row], rv = a.r[row];
                            const V pp = a.p[row], qq = a.q[row];
                            const S x0 = A::fma(A::cx(xx), al0, A::cx(pp)), x1 = A::fma(A::cy(xx), al1, A::cy(pp));
                            const S r0 = A::fma(A::cx(rv), A::neg(al0), A::cx(qq));
                            const S r1 = A::fma(A::cy(rv), A::neg(al1), A::cy(qq));
                            a.x[row] = A::pack(x0, x1);
                            a.r[row] = A::pack(r0, r1);
                            rr0 = A::fma(rr0, r0, r0);
                            rr1 = A::fma(rr1, r1, r1);
                            const float l0 = A::lead(r0), l1 = A::lead(r1);
                            rd0 = fmaf(d * l0, l0, rd0);
                            rd1 = fmaf(d * l1, l1, rd1);
                        }
                    }
                }
                if (threadIdx.x == 0) {
                    s_idx[(it + 2) % 3] = nxt;
                    if (nxt < a.nchunks) s_chunk[(it + 2) % 3] = a.chunks[nxt];
                }
                __syncthreads();
            }
            if (seg >= 0 && m > 0) flush();
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

// Round-robin static schedule.  Block b takes the chunks b, b + G, b + 2G, ...
// (G blocks), so every block samples the whole matrix; nothing is fetched
// from a counter and no barrier separates chunks.  Partial sums go through
// warp shuffles into a per-piece table in shared memory; at the end of a phase
// the block adds each piece's total and chunk count to the global
// accumulators, and the block that completes a piece computes its scalars
// (as in the dynamic schedule).  Up to RR_MAXSEG pieces.
constexpr int RR_MAXSEG = 256;

template <typename A, int MINB>
__global__ void __launch_bounds__(RUN_THREADS, MINB) k_pcg_rr(RunArgs<A> a) {
    using S = typename A::S;
    using V = typename A::V;
    cg::grid_group grid = cg::this_grid();
    __shared__ double tab[RR_MAXSEG][4];
    __shared__ int tcnt[RR_MAXSEG];
    __shared__ double ssc[RR_MAXSEG][2];     // this phase's beta (B) or alpha (A) per piece
    __shared__ unsigned char sdn[RR_MAXSEG][2];
    const int nseg = a.nseg;
    const int lane = threadIdx.x & 31;
    const int32_t* __restrict__ rp = a.rp;
    const int32_t* __restrict__ colp = a.col;
    const S* __restrict__ valp = a.val;
    const float* __restrict__ dgp = a.dgn;
    const int G = gridDim.x;
    unsigned long long wrows = 0, wnnz = 0;
    // warp sum of a double-float value, added into the piece's table entry
    auto warp_add = [&](float2 v, double* dst) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float2 t;
            t.x = __shfl_xor_sync(0xffffffffu, v.x, o);
            t.y = __shfl_xor_sync(0xffffffffu, v.y, o);
            v = df_add(v, t);
        }
        if (lane == 0) atomicAdd(dst, df_to_d(v));
    };
    int k = 0;
    for (; k < a.max_iters; ++k) {
        const double* RRk = a.RR + (k % 3) * 2 * nseg;
        double* RRn = a.RR + ((k + 1) % 3) * 2 * nseg;
        double* RDn = a.RD + ((k + 1) % 3) * 2 * nseg;
        double* PQk = a.PQ + (k % 2) * 2 * nseg;
        const double* BETk = a.BETA + (k % 2) * 2 * nseg;
        double* BETn = a.BETA + ((k + 1) % 2) * 2 * nseg;
        double* ALPk = a.ALPHA + (k % 2) * 2 * nseg;
        unsigned* CB = a.CNTB + (k % 2) * nseg;
        unsigned* CA = a.CNTA + (k % 2) * nseg;
        // ---------------- phase B: p = r + beta p, q = A~ r + beta q, <p, q>
        if (blockIdx.x == 0) {
            for (int i = threadIdx.x; i < 2 * nseg; i += blockDim.x) {
                RRn[i] = 0.0;
                RDn[i] = 0.0;
            }
            for (int i = threadIdx.x; i < nseg; i += blockDim.x) a.CNTB[((k + 1) % 2) * nseg + i] = 0u;
        }
        for (int i = threadIdx.x; i < nseg; i += blockDim.x) {
            tab[i][0] = tab[i][1] = 0.0;
            tcnt[i] = 0;
            ssc[i][0] = __ldcg(BETk + 2 * i);
            ssc[i][1] = __ldcg(BETk + 2 * i + 1);
            sdn[i][0] = __ldcg(a.DONEF + 2 * i) != 0u;
            sdn[i][1] = __ldcg(a.DONEF + 2 * i + 1) != 0u;
        }
        __syncthreads();
        bool any = false;
        {
            int c = blockIdx.x;
            int bn = 0, en = 0;
            DfRun chn = c < a.nchunks ? a.chunks[c] : DfRun{};
            if (c < a.nchunks && chn.lo + (int)threadIdx.x < chn.hi) {
                bn = __ldg(rp + chn.lo + threadIdx.x);
                en = __ldg(rp + chn.lo + threadIdx.x + 1);
            }
            for (; c < a.nchunks; c += G) {
                const DfRun ch = chn;
                const int b = bn, e = en;
                // next chunk of this block: its descriptor and row bounds now, its streams into L2
                const int cn = c + G;
                int nrow = -1;
                bn = en = 0;
                if (cn < a.nchunks) {
                    chn = a.chunks[cn];
                    if (chn.lo + (int)threadIdx.x < chn.hi) {
                        nrow = chn.lo + threadIdx.x;
                        bn = __ldg(rp + nrow);
                        en = __ldg(rp + nrow + 1);
                        prefetch_l2(a.p + nrow);
                        prefetch_l2(a.q + nrow);
                        prefetch_l2(a.r + nrow);
                    }
                }
                const int seg = ch.seg;
                const bool d0 = sdn[seg][0], d1 = sdn[seg][1];
                if (d0 && d1) continue;
                any = true;
                const S beta0 = A::from_d(ssc[seg][0]), beta1 = A::from_d(ssc[seg][1]);
                S acc0 = A::zero(), acc1 = A::zero();
                const int row = ch.lo + threadIdx.x;
                if (row < ch.hi && b < e) {
                    S w0 = A::zero(), w1 = A::zero();
                    int j = b;
                    for (; j + 4 <= e; j += 4) {
                        int32_t cc[4];
                        S v[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            cc[u] = __ldg(colp + j + u);
                            v[u] = __ldg(valp + j + u);
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) spmv_entry<A>(cc[u], v[u], a.r, w0, w1);
                    }
                    for (; j < e; ++j) spmv_entry<A>(__ldg(colp + j), __ldg(valp + j), a.r, w0, w1);
                    const V rr = a.r[row];
                    const V pp = a.p[row], qq = a.q[row];
                    S px = A::cx(pp), py = A::cy(pp), qx = A::cx(qq), qy = A::cy(qq);
                    if (!d0) {
                        px = A::fma(A::cx(rr), beta0, px);
                        qx = A::fma(w0, beta0, qx);
                        acc0 = A::fma(acc0, px, qx);
                    }
                    if (!d1) {
                        py = A::fma(A::cy(rr), beta1, py);
                        qy = A::fma(w1, beta1, qy);
                        acc1 = A::fma(acc1, py, qy);
                    }
                    a.p[row] = A::pack(px, py);
                    a.q[row] = A::pack(qx, qy);
                }
                if (nrow >= 0 && en > bn) {
                    prefetch_l2(colp + bn);
                    prefetch_l2(valp + bn);
                    prefetch_l2(valp + en - 1);
                }
                warp_add(A::as_df(acc0), &tab[seg][0]);
                warp_add(A::as_df(acc1), &tab[seg][1]);
                if (threadIdx.x == 0) {
                    tcnt[seg] += 1;
                    wrows += (unsigned long long)ch.frows;
                    wnnz += (unsigned long long)ch.fnnz;
                }
            }
        }
        __syncthreads();
        for (int sg = threadIdx.x; sg < nseg; sg += blockDim.x) {
            const int m = tcnt[sg];
            if (m == 0) continue;
            atomicAdd(&PQk[2 * sg], tab[sg][0]);
            atomicAdd(&PQk[2 * sg + 1], tab[sg][1]);
            __threadfence();
            const unsigned old = atomicAdd(&CB[sg], (unsigned)m);
            if (old + (unsigned)m == (unsigned)a.nch[sg]) {   // this block completed <p, q>
                __threadfence();
                const double pq0 = __ldcg(PQk + 2 * sg), pq1 = __ldcg(PQk + 2 * sg + 1);
                const double rr0 = __ldcg(RRk + 2 * sg), rr1 = __ldcg(RRk + 2 * sg + 1);
                double al0, al1;
                if (a.dncp) {
                    const double den = pq0 + pq1;
                    al0 = al1 = den > 0.0 ? (rr0 + rr1) / den : 0.0;
                } else {
                    al0 = (!__ldcg(a.DONEF + 2 * sg) && pq0 > 0.0) ? rr0 / pq0 : 0.0;
                    al1 = (!__ldcg(a.DONEF + 2 * sg + 1) && pq1 > 0.0) ? rr1 / pq1 : 0.0;
                }
                __stcg(ALPk + 2 * sg, al0);
                __stcg(ALPk + 2 * sg + 1, al1);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && any) *(volatile unsigned*)&a.ACT[k % 3] = 1u;
        grid.sync();
        // ---------------- phase A: x~ += alpha p, r -= alpha q, norms
        if (blockIdx.x == 0) {
            double* z = a.PQ + ((k + 1) % 2) * 2 * nseg;
            for (int i = threadIdx.x; i < 2 * nseg; i += blockDim.x) z[i] = 0.0;
            for (int i = threadIdx.x; i < nseg; i += blockDim.x) a.CNTA[((k + 1) % 2) * nseg + i] = 0u;
            if (threadIdx.x == 0) a.ACT[(k + 1) % 3] = 0;
        }
        for (int i = threadIdx.x; i < nseg; i += blockDim.x) {
            tab[i][0] = tab[i][1] = tab[i][2] = tab[i][3] = 0.0;
            tcnt[i] = 0;
            ssc[i][0] = __ldcg(ALPk + 2 * i);
            ssc[i][1] = __ldcg(ALPk + 2 * i + 1);
            sdn[i][0] = __ldcg(a.DONEF + 2 * i) != 0u;
            sdn[i][1] = __ldcg(a.DONEF + 2 * i + 1) != 0u;
        }
        __syncthreads();
        DfRun chn = blockIdx.x < (unsigned)a.nchunks ? a.chunks[blockIdx.x] : DfRun{};
        for (int c = blockIdx.x; c < a.nchunks; c += G) {
            const DfRun ch = chn;
            const int cn = c + G;
            if (cn < a.nchunks) {
                chn = a.chunks[cn];
                const int nrow = chn.lo + threadIdx.x;
                if (nrow < chn.hi) {
                    prefetch_l2(a.x + nrow);
                    prefetch_l2(a.r + nrow);
                    prefetch_l2(a.p + nrow);
                    prefetch_l2(a.q + nrow);
                }
            }
            const int seg = ch.seg;
            const bool d0 = sdn[seg][0], d1 = sdn[seg][1];
            if (d0 && d1) continue;
            const S al0 = A::from_d(ssc[seg][0]), al1 = A::from_d(ssc[seg][1]);
            S rr0 = A::zero(), rr1 = A::zero();
            float rd0 = 0.f, rd1 = 0.f;
            const int row = ch.lo + threadIdx.x;
            if (row < ch.hi) {
                const float d = __ldg(dgp + row);
                if (d != 0.f) {
                    const V xx = a.x[row], rv = a.r[row];
                    const V pp = a.p[row], qq = a.q[row];
                    const S x0 = A::fma(A::cx(xx), al0, A::cx(pp)), x1 = A::fma(A::cy(xx), al1, A::cy(pp));
                    const S r0 = A::fma(A::cx(rv), A::neg(al0), A::cx(qq));
                    const S r1 = A::fma(A::cy(rv), A::neg(al1), A::cy(qq));
                    a.x[row] = A::pack(x0, x1);
                    a.r[row] = A::pack(r0, r1);
                    rr0 = A::fma(rr0, r0, r0);
                    rr1 = A::fma(rr1, r1, r1);
                    const float l0 = A::lead(r0), l1 = A::lead(r1);
                    rd0 = fmaf(d * l0, l0, rd0);
                    rd1 = fmaf(d * l1, l1, rd1);
                }
            }
            warp_add(A::as_df(rr0), &tab[seg][0]);
            warp_add(A::as_df(rr1), &tab[seg][1]);
            warp_add(make_float2(rd0, 0.f), &tab[seg][2]);
            warp_add(make_float2(rd1, 0.f), &tab[seg][3]);
            if (threadIdx.x == 0) tcnt[seg] += 1;
        }
        __syncthreads();
        for (int sg = threadIdx.x; sg < nseg; sg += blockDim.x) {
            const int m = tcnt[sg];
            if (m == 0) continue;
            atomicAdd(&RRn[2 * sg], tab[sg][0]);
            atomicAdd(&RRn[2 * sg + 1], tab[sg][1]);
            atomicAdd(&RDn[2 * sg], tab[sg][2]);
            atomicAdd(&RDn[2 * sg + 1], tab[sg][3]);
            __threadfence();
            const unsigned old = atomicAdd(&CA[sg], (unsigned)m);
            if (old + (unsigned)m == (unsigned)a.nch[sg]) {   // this block completed the norms
                __threadfence();
                const double n0 = __ldcg(RRn + 2 * sg), n1 = __ldcg(RRn + 2 * sg + 1);
                const double o0 = __ldcg(RRk + 2 * sg), o1 = __ldcg(RRk + 2 * sg + 1);
                const double e0 = __ldcg(RDn + 2 * sg), e1 = __ldcg(RDn + 2 * sg + 1);
                const double t0 = a.THR[2 * sg], t1 = a.THR[2 * sg + 1];
                if (a.dncp) {
                    const double bt = (o0 + o1) > 0.0 ? (n0 + n1) / (o0 + o1) : 0.0;
                    __stcg(BETn + 2 * sg, bt);
                    __stcg(BETn + 2 * sg + 1, bt);
                    if (e0 + e1 <= t0 + t1) {
                        __stcg(a.DONEF + 2 * sg, 1u);
                        __stcg(a.DONEF + 2 * sg + 1, 1u);
                    }
                } else {
                    __stcg(BETn + 2 * sg, o0 > 0.0 ? n0 / o0 : 0.0);
                    __stcg(BETn + 2 * sg + 1, o1 > 0.0 ? n1 / o1 : 0.0);
                    if (e0 <= t0) __stcg(a.DONEF + 2 * sg, 1u);
                    if (e1 <= t1) __stcg(a.DONEF + 2 * sg + 1, 1u);
                }
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

// Single-reduction schedule: CG in the form of Chronopoulos and Gear
// ("s-step iterative methods for symmetric linear systems", 1989): with
// w = A~ r and s = A~ p kept as vectors, one iteration needs one SpMV and one
// combined reduction of gamma = <r, r>, delta = <r, w>:
//   beta_k = gamma_k / gamma_{k-1},  alpha_k = gamma_k / (delta_k - beta_k gamma_k / alpha_{k-1})
//   p_k = r_k + beta_k p_{k-1};  s_k = w_k + beta_k s_{k-1}
//   x_{k+1} = x_k + alpha_k p_k;  r_{k+1} = r_k - alpha_k s_k;  w_{k+1} = A~ r_{k+1}
// so one grid sync per iteration.  A row's SpMV needs its neighbours' r_{k+1},
// which is formed on the fly from their r_k, w_k and s_{k-1}; r, w and s are
// double-buffered so no block overwrites what another still gathers.
constexpr int CG1_MAXRUNS = 16;

template <typename A>
__device__ __forceinline__ typename A::V next_r(const typename A::V& r, const typename A::V& w, const typename A::V& sp,
                                                typename A::S al0, typename A::S al1, typename A::S be0,
                                                typename A::S be1) {
    const typename A::S s0 = A::fma(A::cx(w), be0, A::cx(sp)), s1 = A::fma(A::cy(w), be1, A::cy(sp));
    return A::pack(A::fma(A::cx(r), A::neg(al0), s0), A::fma(A::cy(r), A::neg(al1), s1));
}

template <typename A, int MINB>
__global__ void __launch_bounds__(RUN_THREADS, MINB) k_pcg_cg1(RunArgs<A> a) {
    using S = typename A::S;
    using V = typename A::V;
    cg::grid_group grid = cg::this_grid();
    __shared__ float2 red[6 * (RUN_THREADS / 32)];
    __shared__ double sc[2][4];
    __shared__ int sflag[2][2];
    __shared__ double alpha_prev[CG1_MAXRUNS][2];
    const int nseg = a.nseg;
    const int rb = a.run_off[blockIdx.x], re = a.run_off[blockIdx.x + 1];
    const int32_t* __restrict__ rp = a.rp;
    const int32_t* __restrict__ colp = a.col;
    const S* __restrict__ valp = a.val;
    const float* __restrict__ dgp = a.dgn;
    V* const rbuf[2] = {a.r, a.r1};
    V* const wbuf[2] = {a.w0, a.w1};
    V* const sbuf[2] = {a.q, a.s1};
    unsigned long long wrows = 0, wnnz = 0;
    // ---------------- set-up: w_0 = A~ r_0, delta_0 = <r_0, w_0>
    for (int ri = rb; ri < re; ++ri) {
        const DfRun run = a.runs[ri];
        S d0 = A::zero(), d1 = A::zero();
        for (int row = run.lo + threadIdx.x; row < run.hi; row += blockDim.x) {
            const int b = __ldg(rp + row), e = __ldg(rp + row + 1);
            S w0 = A::zero(), w1 = A::zero();
            for (int j = b; j < e; ++j) spmv_entry<A>(__ldg(colp + j), __ldg(valp + j), a.r, w0, w1);
            const V r = a.r[row];
            a.w0[row] = A::pack(w0, w1);
            a.s1[row] = A::vzero();
            d0 = A::fma(d0, A::cx(r), w0);
            d1 = A::fma(d1, A::cy(r), w1);
        }
        float2 pv[2] = {A::as_df(d0), A::as_df(d1)};
        double v[2];
        block_sum_df<2>(pv, red, v);
        if (threadIdx.x == 0) {
            atomicAdd(&a.DL[2 * run.seg], v[0]);
            atomicAdd(&a.DL[2 * run.seg + 1], v[1]);
        }
        if (threadIdx.x < 2 && ri - rb < CG1_MAXRUNS) alpha_prev[ri - rb][threadIdx.x] = INFINITY;
    }
    grid.sync();
    int k = 0;
    for (; k < a.max_iters; ++k) {
        // four accumulator slots: k (read), k - 1 (read), k + 1 (filled now), k + 2 (cleared now)
        const double* Gk = a.RR + (k % 4) * 2 * nseg;
        const double* Gm = a.RR + ((k + 3) % 4) * 2 * nseg;
        const double* Dk = a.DL + (k % 4) * 2 * nseg;
        const double* RDk = a.RD + (k % 4) * 2 * nseg;
        double* Gn = a.RR + ((k + 1) % 4) * 2 * nseg;
        double* Dn = a.DL + ((k + 1) % 4) * 2 * nseg;
        double* RDn = a.RD + ((k + 1) % 4) * 2 * nseg;
        const V* __restrict__ rk = rbuf[k & 1];
        const V* __restrict__ wk = wbuf[k & 1];
        const V* __restrict__ sm = sbuf[(k + 1) & 1];   // s_{k-1}
        V* rn = rbuf[(k + 1) & 1];
        V* wn = wbuf[(k + 1) & 1];
        V* sk = sbuf[k & 1];
        if (blockIdx.x == 0) {
            double* g2 = a.RR + ((k + 2) % 4) * 2 * nseg;
            double* d2 = a.DL + ((k + 2) % 4) * 2 * nseg;
            double* e2 = a.RD + ((k + 2) % 4) * 2 * nseg;
            for (int i = threadIdx.x; i < 2 * nseg; i += blockDim.x) {
                g2[i] = 0.0;
                d2[i] = 0.0;
                e2[i] = 0.0;
            }
            if (threadIdx.x == 0) a.ACT[(k + 1) % 3] = 0;
        }
        bool any = false;
        for (int ri = rb; ri < re; ++ri) {
            const DfRun run = a.runs[ri];
            const int s = run.seg, slot = ri & 1, lr = ri - rb;
            if (threadIdx.x == 0) {
                const bool d0 = piece_done(RDk, a.THR, s, 0, a.dncp);
                const bool d1 = piece_done(RDk, a.THR, s, 1, a.dncp);
                double be[2] = {0.0, 0.0}, al[2] = {0.0, 0.0};
                const double g0 = __ldcg(Gk + 2 * s), g1 = __ldcg(Gk + 2 * s + 1);
                const double e0 = __ldcg(Dk + 2 * s), e1 = __ldcg(Dk + 2 * s + 1);
                if (a.dncp) {
                    const double g = g0 + g1, dl = e0 + e1;
                    const double gm = k > 0 ? __ldcg(Gm + 2 * s) + __ldcg(Gm + 2 * s + 1) : 0.0;
                    const double b = (k > 0 && gm > 0.0) ? g / gm : 0.0;
                    const double ap = alpha_prev[lr][0];
                    const double den = dl - (ap > 0.0 && isfinite(ap) ? b * g / ap : 0.0);
                    be[0] = be[1] = b;
                    al[0] = al[1] = den > 0.0 ? g / den : 0.0;
                } else {
                    const double gg[2] = {g0, g1}, ee[2] = {e0, e1};
                    for (int c = 0; c < 2; ++c) {
                        const double gm = k > 0 ? __ldcg(Gm + 2 * s + c) : 0.0;
                        const double b = (k > 0 && gm > 0.0) ? gg[c] / gm : 0.0;
                        const double ap = alpha_prev[lr][c];
                        const double den = ee[c] - (ap > 0.0 && isfinite(ap) ? b * gg[c] / ap : 0.0);
                        be[c] = b;
                        al[c] = den > 0.0 ? gg[c] / den : 0.0;
                    }
                    if (d0) al[0] = be[0] = 0.0;
                    if (d1) al[1] = be[1] = 0.0;
                }
                sc[slot][0] = al[0];
                sc[slot][1] = al[1];
                sc[slot][2] = be[0];
                sc[slot][3] = be[1];
                sflag[slot][0] = d0;
                sflag[slot][1] = d1;
                if (!(d0 && d1)) {
                    alpha_prev[lr][0] = al[0];
                    alpha_prev[lr][1] = al[1];
                }
            }
            __syncthreads();
            const bool d0 = sflag[slot][0], d1 = sflag[slot][1];
            if (d0 && d1) continue;
            any = true;
            const S al0 = A::from_d(sc[slot][0]), al1 = A::from_d(sc[slot][1]);
            const S be0 = A::from_d(sc[slot][2]), be1 = A::from_d(sc[slot][3]);
            S g0 = A::zero(), g1 = A::zero(), e0 = A::zero(), e1 = A::zero();
            float rd0 = 0.f, rd1 = 0.f;
            for (int row = run.lo + threadIdx.x; row < run.hi; row += blockDim.x) {
                const float d = __ldg(dgp + row);
                if (d == 0.f) continue;   // fixed row: r, w, s stay 0
                const V r = rk[row], w = wk[row], spv = sm[row], pv = a.p[row], xv = a.x[row];
                const S p0 = A::fma(A::cx(r), be0, A::cx(pv)), p1 = A::fma(A::cy(r), be1, A::cy(pv));
                const S s0 = A::fma(A::cx(w), be0, A::cx(spv)), s1 = A::fma(A::cy(w), be1, A::cy(spv));
                const S x0 = A::fma(A::cx(xv), al0, p0), x1 = A::fma(A::cy(xv), al1, p1);
                const S r0 = A::fma(A::cx(r), A::neg(al0), s0), r1 = A::fma(A::cy(r), A::neg(al1), s1);
                a.p[row] = A::pack(p0, p1);
                sk[row] = A::pack(s0, s1);
                a.x[row] = A::pack(x0, x1);
                rn[row] = A::pack(r0, r1);
                // w_{k+1} = A~ r_{k+1}: the neighbours' r_{k+1} formed from their r_k, w_k, s_{k-1}
                S w0 = A::zero(), w1 = A::zero();
                const int b = __ldg(rp + row), e = __ldg(rp + row + 1);
                for (int j = b; j < e; ++j) {
                    const int32_t c = __ldg(colp + j);
                    const S v = __ldg(valp + j);
                    const bool cross = c < 0;
                    const int cc = cross ? ~c : c;
                    const V rc = next_r<A>(rk[cc], wk[cc], sm[cc], al0, al1, be0, be1);
                    const S a0 = cross ? A::cy(rc) : A::cx(rc);
                    const S a1 = cross ? A::cx(rc) : A::cy(rc);
                    w0 = A::fma(w0, cross ? A::neg(v) : v, a0);
                    w1 = A::fma(w1, v, a1);
                }
                wn[row] = A::pack(w0, w1);
                g0 = A::fma(g0, r0, r0);
                g1 = A::fma(g1, r1, r1);
                e0 = A::fma(e0, r0, w0);
                e1 = A::fma(e1, r1, w1);
                const float l0 = A::lead(r0), l1 = A::lead(r1);
                rd0 = fmaf(d * l0, l0, rd0);
                rd1 = fmaf(d * l1, l1, rd1);
            }
            float2 pv[6] = {A::as_df(g0), A::as_df(g1), A::as_df(e0), A::as_df(e1), make_float2(rd0, 0.f),
                            make_float2(rd1, 0.f)};
            double v[6];
            block_sum_df<6>(pv, red, v);
            if (threadIdx.x == 0) {
                atomicAdd(&Gn[2 * s], v[0]);
                atomicAdd(&Gn[2 * s + 1], v[1]);
                atomicAdd(&Dn[2 * s], v[2]);
                atomicAdd(&Dn[2 * s + 1], v[3]);
                atomicAdd(&RDn[2 * s], v[4]);
                atomicAdd(&RDn[2 * s + 1], v[5]);
                wrows += (unsigned long long)run.frows;
                wnnz += (unsigned long long)run.fnnz;
            }
        }
        if (threadIdx.x == 0 && any) *(volatile unsigned*)&a.ACT[k % 3] = 1u;
        grid.sync();
        if (*(volatile unsigned*)&a.ACT[k % 3] == 0u) break;
    }
    if (threadIdx.x == 0) {
        if (wrows) atomicAdd(&a.work[0], wrows);
        if (wnnz) atomicAdd(&a.work[1], wnnz);
        if (blockIdx.x == 0) a.out_iters[0] = k;
    }
}

// Initial state of the dynamic schedule: converged flags from <r0, r0>, beta 0.
__global__ void k_dyn_init(int nseg, int dncp, const double* __restrict__ RD0, const double* __restrict__ THR,
                           unsigned int* __restrict__ DONEF, double* __restrict__ BETA0) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    BETA0[2 * s] = 0.0;
    BETA0[2 * s + 1] = 0.0;
    if (dncp) {
        const unsigned d = RD0[2 * s] + RD0[2 * s + 1] <= THR[2 * s] + THR[2 * s + 1] ? 1u : 0u;
        DONEF[2 * s] = d;
        DONEF[2 * s + 1] = d;
    } else {
        DONEF[2 * s] = RD0[2 * s] <= THR[2 * s] ? 1u : 0u;
        DONEF[2 * s + 1] = RD0[2 * s + 1] <= THR[2 * s + 1] ? 1u : 0u;
    }
}

// ---------------------------------------------------------------- set-up kernels

// Stored entries of row i of A~: free columns of a free row, plus the DNCP
// cross entries to free loop neighbours.
__global__ void k_run_count(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
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

template <typename A>
__global__ void k_run_fill(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const double* __restrict__ diag,
                           const uint8_t* __restrict__ fixed, const int2* __restrict__ nb, int dncp,
                           const int64_t* __restrict__ off, const int32_t* __restrict__ cnt,
                           int32_t* __restrict__ rp2, int32_t* __restrict__ col2, typename A::S* __restrict__ val2,
                           double* __restrict__ sc, float* __restrict__ dgn) {
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
        val2[t] = A::from_d(val[j] * si / sqrt(diag[c]));
        ++t;
    }
    if (dncp) {
        const int2 pn = nb[i];
        if (pn.x >= 0) {
            if (!fixed[pn.x]) {
                col2[t] = ~pn.x;
                val2[t] = A::from_d(-0.5 * si / sqrt(diag[pn.x]));
                ++t;
            }
            if (!fixed[pn.y]) {
                col2[t] = ~pn.y;
                val2[t] = A::from_d(0.5 * si / sqrt(diag[pn.y]));
                ++t;
            }
        }
    }
}

// frows / fnnz per run (one block per run)
__global__ void k_run_stats(DfRun* runs, const int32_t* __restrict__ rp2) {
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

// Sum NV doubles over the block (set-up kernels only); thread 0 gets the totals.
template <int NV>
__device__ __forceinline__ void block_sum64(double* v, double* red) {
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

// r~ = S r64 (0 at fixed rows), x~ = p = q = 0, and the slot-0 norms per run.
template <typename A>
__global__ void k_run_prep(const DfRun* __restrict__ runs, const int32_t* __restrict__ run_off,
                           const double2* __restrict__ r64, const double* __restrict__ sc, typename A::V* __restrict__ x,
                           typename A::V* __restrict__ r, typename A::V* __restrict__ p, typename A::V* __restrict__ q,
                           double* __restrict__ RR, double* __restrict__ RD, double* __restrict__ PRR0,
                           double* __restrict__ PRD0, int keep_pq) {
    __shared__ double red[4 * (RUN_THREADS / 32)];
    for (int ri = run_off[blockIdx.x]; ri < run_off[blockIdx.x + 1]; ++ri) {
        const DfRun run = runs[ri];
        double v[4] = {0, 0, 0, 0};
        for (int i = run.lo + threadIdx.x; i < run.hi; i += blockDim.x) {
            const double si = sc[i];
            const double2 ri64 = r64[i];
            const double a0 = si * ri64.x, a1 = si * ri64.y;
            const typename A::S f0 = A::from_d(a0), f1 = A::from_d(a1);
            x[i] = A::vzero();
            if (!keep_pq) {
                p[i] = A::vzero();
                q[i] = A::vzero();
            }
            r[i] = A::pack(f0, f1);
            if (si != 0.0) {
                // the stored (rounded) values, so CG starts from what it iterates on
                const double g0 = A::to_d(f0), g1 = A::to_d(f1);
                v[0] += g0 * g0;
                v[1] += g1 * g1;
                v[2] += ri64.x * ri64.x;
                v[3] += ri64.y * ri64.y;
            }
        }
        block_sum64<4>(v, red);
        if (threadIdx.x == 0 && PRR0) {   // deterministic mode: per-run sums
            PRR0[2 * ri] = v[0];
            PRR0[2 * ri + 1] = v[1];
            PRD0[2 * ri] = v[2];
            PRD0[2 * ri + 1] = v[3];
        } else if (threadIdx.x == 0) {
            atomicAdd(&RR[2 * run.seg], v[0]);
            atomicAdd(&RR[2 * run.seg + 1], v[1]);
            atomicAdd(&RD[2 * run.seg], v[2]);
            atomicAdd(&RD[2 * run.seg + 1], v[3]);
        }
        __syncthreads();
    }
}

// x += S x~ on free rows
template <typename A>
__global__ void k_run_finish(int64_t n, const double* __restrict__ sc, const typename A::V* __restrict__ xs,
                             double2* __restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double si = sc[i];
    if (si == 0.0) return;
    const typename A::V v = xs[i];
    x[i].x += si * A::to_d(A::cx(v));
    x[i].y += si * A::to_d(A::cy(v));
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, ceil_div(n, t)); }

template <typename A>
void build_typed(pgcp_ctx* ctx, Part& P, int dncp, const uint8_t* fixed, DfSystem& D, const int32_t* cnt,
                 const int64_t* off) {
    cudaStream_t s = ctx->stream;
    const int64_t n = D.n;
    D.val.alloc(std::max<int64_t>(D.nnz, 1) * sizeof(typename A::S), s);
    { k_run_fill<A><<<nblk(n), 256, 0, s>>>(n, P.row_ptr.p, P.col.p, P.val64.p, P.diag64.p, fixed, P.nb.p, dncp, off,
                                            cnt, D.rp.p, D.col.p, reinterpret_cast<typename A::S*>(D.val.p), D.sc.p,
                                            D.dgn.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    int per_sm = 0;
    const void* kern = D.minb == 3 ? (const void*)k_pcg_run<A, 3> : (const void*)k_pcg_run<A, 4>;
    PGCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RUN_THREADS, 0));
    if (per_sm <= 0) fail(PGCP_E_CUDA, "run-based PCG kernel cannot be resident");
    if (D.sched == 4) {   // the single-reduction kernel shares the static row runs
        int per_sm_cg1 = 0;
        const void* kc = D.minb == 3 ? (const void*)k_pcg_cg1<A, 3> : (const void*)k_pcg_cg1<A, 4>;
        PGCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_cg1, kc, RUN_THREADS, 0));
        if (per_sm_cg1 <= 0) fail(PGCP_E_CUDA, "single-reduction PCG kernel cannot be resident");
        per_sm = std::min(per_sm, per_sm_cg1);
        const size_t vbb = sizeof(typename A::V);
        D.r1.alloc(n * vbb, s);
        D.w0.alloc(n * vbb, s);
        D.w1.alloc(n * vbb, s);
        D.s1.alloc(n * vbb, s);
    }
    D.per_sm = per_sm;
    int per_sm_dyn = 0;
    const void* kd = D.minb == 3 ? (const void*)k_pcg_dyn<A, 3> : (const void*)k_pcg_dyn<A, 4>;
    PGCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_dyn, kd, RUN_THREADS, 0));
    if (per_sm_dyn <= 0) fail(PGCP_E_CUDA, "dynamically scheduled PCG kernel cannot be resident");
    D.dyn_grid = per_sm_dyn * ctx->num_sms;
    int per_sm_rr = 0;
    const void* kr = D.minb == 3 ? (const void*)k_pcg_rr<A, 3> : (const void*)k_pcg_rr<A, 4>;
    PGCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_rr, kr, RUN_THREADS, 0));
    if (per_sm_rr <= 0) fail(PGCP_E_CUDA, "round-robin PCG kernel cannot be resident");
    D.rr_grid = per_sm_rr * ctx->num_sms;
    const size_t vb = sizeof(typename A::V);
    D.x.alloc(n * vb, s);
    D.r.alloc(n * vb, s);
    D.p.alloc(n * vb, s);
    D.q.alloc(n * vb, s);
}

// x~ = 0 and r~ = S r64; <r~, r~> and the unscaled sum of r64^2 go to slot
// `slot` of RR and RD.  A resumed solve keeps p and q (residual replacement).
template <typename A>
void prep_typed(pgcp_ctx* ctx, Part& P, DfSystem& D, const double2* r64, int slot, bool resume) {
    cudaStream_t s = ctx->stream;
    using V = typename A::V;
    V* xv = reinterpret_cast<V*>(D.x.p);
    V* rv = reinterpret_cast<V*>(D.r.p);
    V* pv = reinterpret_cast<V*>(D.p.p);
    V* qv = reinterpret_cast<V*>(D.q.p);
    double* RRs = D.RR.p + (int64_t)slot * 2 * P.K;
    double* RDs = D.RD.p + (int64_t)slot * 2 * P.K;
    { k_run_prep<A><<<(unsigned)D.grid, RUN_THREADS, 0, s>>>(D.runs.p, D.run_off.p, r64, D.sc.p, xv, rv, pv, qv, RRs,
                                                            RDs, D.det ? D.PRR.p : nullptr,
                                                            D.det ? D.PRD.p : nullptr, resume ? 1 : 0); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    if (D.sched >= 2) {
        { k_dyn_init<<<(unsigned)std::max<int64_t>(1, ceil_div((int64_t)P.K, 256)), 256, 0, s>>>(
            P.K, D.dncp, D.RD.p, D.THR.p, D.DONEF.p, D.BETA.p); ::pgcp::note_launch(); }
        D.CTR.zero();
        D.CNTB.zero();
        D.CNTA.zero();
        PGCP_CUDA(cudaGetLastError());
    }
}

// One persistent launch: iterations k0 .. cap - 1 (it stops earlier once every
// piece has converged; out_it then holds the iteration it stopped at).
template <typename A>
void launch_typed(pgcp_ctx* ctx, Part& P, DfSystem& D, int k0, int cap, bool resume) {
    cudaStream_t s = ctx->stream;
    using V = typename A::V;
    V* xv = reinterpret_cast<V*>(D.x.p);
    V* rv = reinterpret_cast<V*>(D.r.p);
    V* pv = reinterpret_cast<V*>(D.p.p);
    V* qv = reinterpret_cast<V*>(D.q.p);
    RunArgs<A> a{(int32_t)D.n, P.K, D.rp.p, D.col.p, reinterpret_cast<const typename A::S*>(D.val.p), D.dgn.p, xv, rv,
                 pv, qv, D.runs.p, D.run_off.p, D.RR.p, D.RD.p, D.PQ.p, D.ACT.p, D.THR.p, D.out_it.p, cap,
                 D.dncp, D.work.p};
    a.k0 = k0;
    a.resume = resume ? 1 : 0;
    a.RRP = D.RRP.p;
    a.chunks = D.chunks.p;
    a.nchunks = D.nchunks;
    a.nch = D.nch.p;
    a.CTR = D.CTR.p;
    a.CNTB = D.CNTB.p;
    a.CNTA = D.CNTA.p;
    a.ALPHA = D.ALPHA.p;
    a.BETA = D.BETA.p;
    a.DONEF = D.DONEF.p;
    a.det = D.det;
    a.nruns = D.nruns;
    a.prun = D.prun.p;
    a.PRR = D.PRR.p;
    a.PRD = D.PRD.p;
    a.PPQ = D.PPQ.p;
    a.RDONE = D.RDONE.p;
    a.CRR = D.CRR.p;
    void* args[] = {(void*)&a};
    a.r1 = reinterpret_cast<V*>(D.r1.p);
    a.w0 = reinterpret_cast<V*>(D.w0.p);
    a.w1 = reinterpret_cast<V*>(D.w1.p);
    a.s1 = reinterpret_cast<V*>(D.s1.p);
    a.DL = D.DL.p;
    if (D.sched == 4) {
        const void* kern = D.minb == 3 ? (const void*)k_pcg_cg1<A, 3> : (const void*)k_pcg_cg1<A, 4>;
        { PGCP_CUDA(cudaLaunchCooperativeKernel(kern, dim3(D.grid), dim3(RUN_THREADS), args, 0, s)); ::pgcp::note_launch(); }
    } else if (D.sched == 2) {
        const void* kern = D.minb == 3 ? (const void*)k_pcg_dyn<A, 3> : (const void*)k_pcg_dyn<A, 4>;
        const int grid = std::max(1, std::min(D.dyn_grid, D.nchunks));
        { PGCP_CUDA(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(RUN_THREADS), args, 0, s)); ::pgcp::note_launch(); }
    } else if (D.sched == 3) {
        const void* kern = D.minb == 3 ? (const void*)k_pcg_rr<A, 3> : (const void*)k_pcg_rr<A, 4>;
        const int grid = std::max(1, std::min(D.rr_grid, D.nchunks));
        { PGCP_CUDA(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(RUN_THREADS), args, 0, s)); ::pgcp::note_launch(); }
    } else {
        const void* kern = D.minb == 3 ? (const void*)k_pcg_run<A, 3> : (const void*)k_pcg_run<A, 4>;
        { PGCP_CUDA(cudaLaunchCooperativeKernel(kern, dim3(D.grid), dim3(RUN_THREADS), args, 0, s)); ::pgcp::note_launch(); }
    }
}

template <typename A>
void finish_typed(pgcp_ctx* ctx, DfSystem& D, double2* x) {
    { k_run_finish<A><<<nblk(D.n), 256, 0, ctx->stream>>>(D.n, D.sc.p, reinterpret_cast<const typename A::V*>(D.x.p),
                                                          x); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
}

}  // namespace

// ---------------------------------------------------------------- host side

// Row runs of the persistent grid: the rows of the active pieces (all when
// active is null), concatenated in piece order, split into `grid` near-equal
// ranges, each range cut at piece boundaries.  With align > 1 a split inside a
// piece is moved down to a multiple of `align` rows from the piece's first row;
// with maxlen > 0 (a multiple of align) longer runs are cut into pieces of
// maxlen rows.  Returns the rows covered.
int64_t make_runs(const std::vector<int64_t>& voff, const std::vector<uint8_t>* active, int grid,
                  std::vector<DfRun>& runs, std::vector<int32_t>& roff, int align, int maxlen) {
    std::vector<int> segs;
    int64_t total = 0;
    for (int i = 0; i + 1 < (int)voff.size(); ++i)
        if (!active || (*active)[i]) {
            segs.push_back(i);
            total += voff[i + 1] - voff[i];
        }
    runs.clear();
    roff.assign(grid + 1, 0);
    size_t c = 0;
    int64_t pos = 0, cbase = 0;   // position in the concatenation; start of piece segs[c] in it
    for (int b = 0; b < grid; ++b) {
        roff[b] = (int32_t)runs.size();
        const int64_t target = b + 1 == grid ? total : total * (b + 1) / grid;
        while (pos < target && c < segs.size()) {
            const int seg = segs[c];
            const int64_t len = voff[seg + 1] - voff[seg];
            int64_t end = std::min<int64_t>(target, cbase + len);
            if (end < cbase + len && align > 1) end = cbase + (end - cbase) / align * align;
            if (end <= pos) break;   // the aligned split leaves nothing here: the next range takes it
            for (int64_t a = pos; a < end;) {
                const int64_t e = maxlen > 0 ? std::min<int64_t>(end, a + maxlen) : end;
                runs.push_back(DfRun{seg, (int32_t)(voff[seg] + (a - cbase)), (int32_t)(voff[seg] + (e - cbase)), 0, 0,
                                     0, 0, 0});
                a = e;
            }
            pos = end;
            if (pos == cbase + len) {
                cbase += len;
                ++c;
            }
        }
    }
    roff[grid] = (int32_t)runs.size();
    return total;
}

// Runs for the preconditioned kernel: when every active piece holds at least
// one block's share of the rows, each piece gets a whole number of blocks
// (its share of `grid`, largest remainders first) and its rows are split
// evenly among them at multiples of `align`, in runs of at most maxlen rows,
// so no block straddles two pieces.  Otherwise make_runs.
int64_t make_runs_by_piece(const std::vector<int64_t>& voff, const std::vector<uint8_t>* active, int grid,
                           std::vector<DfRun>& runs, std::vector<int32_t>& roff, int align, int maxlen) {
    std::vector<int> segs;
    int64_t total = 0, smallest = INT64_MAX;
    for (int i = 0; i + 1 < (int)voff.size(); ++i)
        if (!active || (*active)[i]) {
            segs.push_back(i);
            total += voff[i + 1] - voff[i];
            smallest = std::min<int64_t>(smallest, voff[i + 1] - voff[i]);
        }
    if (segs.empty() || (int)segs.size() > grid || smallest * grid < total)
        return make_runs(voff, active, grid, runs, roff, align, maxlen);
    std::vector<int> quota(segs.size());
    std::vector<std::pair<double, int>> rem;
    int used = 0;
    for (size_t c = 0; c < segs.size(); ++c) {
        const double share = (double)(voff[segs[c] + 1] - voff[segs[c]]) * grid / (double)total;
        quota[c] = std::max(1, (int)share);
        used += quota[c];
        rem.push_back({share - (double)(int)share, (int)c});
    }
    std::sort(rem.begin(), rem.end(), [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
        return x.first != y.first ? x.first > y.first : x.second < y.second;
    });
    for (size_t t = 0; used < grid && t < rem.size(); ++t, ++used) ++quota[rem[t].second];
    runs.clear();
    roff.assign(grid + 1, 0);
    int b = 0;
    for (size_t c = 0; c < segs.size() && b < grid; ++c) {
        const int seg = segs[c];
        const int64_t len = voff[seg + 1] - voff[seg];
        for (int q = 0; q < quota[c] && b < grid; ++q, ++b) {
            roff[b] = (int32_t)runs.size();
            int64_t lo = len * q / quota[c], hi = len * (q + 1) / quota[c];
            if (q > 0) lo = lo / align * align;
            if (q + 1 < quota[c]) hi = hi / align * align;
            for (int64_t a = lo; a < hi;) {
                const int64_t e = maxlen > 0 ? std::min<int64_t>(hi, a + maxlen) : hi;
                runs.push_back(DfRun{seg, (int32_t)(voff[seg] + a), (int32_t)(voff[seg] + e), 0, 0, 0, 0, 0});
                a = e;
            }
        }
    }
    for (; b <= grid; ++b) roff[b] = (int32_t)runs.size();
    return total;
}

void df_build(pgcp_ctx* ctx, Part& P, int dncp, const uint8_t* fixed, int f32, DfSystem& D) {
    cudaStream_t s = ctx->stream;
    const int64_t n = P.Nc;
    if (n >= INT32_MAX) fail(PGCP_E_ARG, "run-based PCG: too many rows");
    D.n = n;
    D.dncp = dncp;
    D.f32 = f32;
    const int bps = ctx->opt.pcg_blocks_per_sm;
    if (bps != 0 && bps != 3 && bps != 4) fail(PGCP_E_ARG, "pcg_blocks_per_sm must be 0, 3 or 4");
    D.minb = bps == 3 ? 3 : 4;
    const int sched = ctx->opt.pcg_schedule;
    if (sched < 0 || sched > 4) fail(PGCP_E_ARG, "pcg_schedule must be 0 to 4");
    D.sched = sched == 0 ? 1 : sched;
    D.det = ctx->opt.deterministic ? 1 : 0;
    if (D.det) D.sched = 1;   // ordered sums are implemented for the static schedule
    // multilevel preconditioner: double-float solves (DNCP, and Laplace when
    // the final solve runs in double-float) on the static schedule
    const int pc = ctx->opt.local_precond;
    if (pc != 0 && pc != 1) fail(PGCP_E_ARG, "local_precond must be 0 (multilevel) or 1 (Jacobi)");
    D.ml = (!f32 && !D.det && D.sched == 1 && pc == 0) ? 1 : 0;
    if (D.sched == 3 && P.K > RR_MAXSEG) D.sched = 1;   // the round-robin tables hold RR_MAXSEG pieces
    DBuf<int32_t> cnt;
    DBuf<int64_t> off;
    cnt.alloc(n, s);
    off.alloc(n, s);
    { k_run_count<<<nblk(n), 256, 0, s>>>(n, P.row_ptr.p, P.col.p, fixed, P.nb.p, dncp, cnt.p); ::pgcp::note_launch(); }
    int64_t nnz2 = 0;
    exclusive_scan_i32_to_i64(cnt.p, off.p, n, s, &nnz2);
    if (nnz2 >= INT32_MAX) fail(PGCP_E_ARG, "run-based PCG: too many stored entries");
    D.nnz = nnz2;
    D.rp.alloc(n + 1, s);
    D.col.alloc(std::max<int64_t>(nnz2, 1), s);
    D.sc.alloc(n, s);
    D.dgn.alloc(n, s);
    if (f32) build_typed<ArithF32>(ctx, P, dncp, fixed, D, cnt.p, off.p);
    else build_typed<ArithDF>(ctx, P, dncp, fixed, D, cnt.p, off.p);
    if (D.ml) ml_build(ctx, P, fixed, D);
    // persistent grid (all co-resident blocks) and its row runs
    const int per_sm = D.ml ? D.ml_per_sm : D.per_sm;
    int grid = (int)std::min<int64_t>((int64_t)per_sm * ctx->num_sms, std::max<int64_t>(1, ceil_div(n, 32)));
    grid = std::max(grid, 1);
    D.grid = grid;
    std::vector<DfRun> runs;
    std::vector<int32_t> roff;
    D.covered = D.ml ? make_runs_by_piece(P.voff, nullptr, grid, runs, roff, 16, ML_SEG)
                     : make_runs(P.voff, nullptr, grid, runs, roff);
    D.nruns = (int32_t)runs.size();
    if (D.sched == 4)
        for (int b = 0; b < grid; ++b)
            if (roff[b + 1] - roff[b] > CG1_MAXRUNS) {
                D.sched = 1;   // more pieces per block than the kernel's run table: static schedule
                break;
            }
    // room for the rebuilt runs (and, with the preconditioner, for runs cut at ML_SEG rows)
    D.runs_cap = std::max<int64_t>(D.nruns, (int64_t)grid + P.K) + (D.ml ? ceil_div(n, ML_SEG) + grid + P.K : 0);
    D.runs.alloc(std::max<int64_t>(1, D.runs_cap), s);
    D.run_off.alloc(grid + 1, s);
    // runs of a piece are consecutive (blocks and their runs follow the rows)
    std::vector<int32_t> prun(2 * (size_t)std::max(1, P.K), 0);
    for (int32_t i = (int32_t)runs.size() - 1; i >= 0; --i) prun[2 * runs[i].seg] = i;
    for (int32_t i = 0; i < (int32_t)runs.size(); ++i) prun[2 * runs[i].seg + 1] = i + 1;
    if (D.det) {
        D.prun.alloc(prun.size(), s);
        PGCP_CUDA(cudaMemcpyAsync(D.prun.p, prun.data(), prun.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        const int64_t nr = std::max<int64_t>(1, D.nruns);
        D.PRR.alloc(3 * 2 * nr, s);
        D.PRD.alloc(3 * 2 * nr, s);
        D.PPQ.alloc(2 * 2 * nr, s);
        D.RDONE.alloc(2 * nr, s);
        D.CRR.alloc(2 * nr, s);
    }
    PGCP_CUDA(cudaMemcpyAsync(D.runs.p, runs.data(), runs.size() * sizeof(DfRun), cudaMemcpyHostToDevice, s));
    PGCP_CUDA(cudaMemcpyAsync(D.run_off.p, roff.data(), roff.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    if (D.nruns > 0) {
        { k_run_stats<<<(unsigned)D.nruns, 256, 0, s>>>(D.runs.p, D.rp.p); ::pgcp::note_launch(); }
    }
    const int S = P.K;
    // chunks of RUN_THREADS rows inside each piece (dynamic schedule)
    {
        std::vector<DfRun> ch;
        std::vector<int32_t> nch(S, 0);
        for (int i = 0; i < S; ++i)
            for (int64_t lo = P.voff[i]; lo < P.voff[i + 1]; lo += RUN_THREADS) {
                ch.push_back(DfRun{i, (int32_t)lo, (int32_t)std::min<int64_t>(lo + RUN_THREADS, P.voff[i + 1]), 0, 0,
                                   0, 0, 0});
                nch[i] += 1;
            }
        D.nchunks = (int32_t)ch.size();
        D.chunks.alloc(std::max<int64_t>(1, D.nchunks), s);
        D.nch.alloc(std::max(1, S), s);
        PGCP_CUDA(cudaMemcpyAsync(D.chunks.p, ch.data(), ch.size() * sizeof(DfRun), cudaMemcpyHostToDevice, s));
        PGCP_CUDA(cudaMemcpyAsync(D.nch.p, nch.data(), S * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        if (D.nchunks > 0) {
            { k_run_stats<<<(unsigned)D.nchunks, 256, 0, s>>>(D.chunks.p, D.rp.p); ::pgcp::note_launch(); }
        }
        D.CTR.alloc(4, s);
        D.CNTB.alloc(2 * S, s);
        D.CNTA.alloc(2 * S, s);
        D.DONEF.alloc(2 * S, s);
        D.ALPHA.alloc(2 * 2 * S, s);
        D.BETA.alloc(2 * 2 * S, s);
        D.ALPHA.zero();
        D.BETA.zero();
        PGCP_CUDA(cudaStreamSynchronize(s));   // host vectors go out of scope
    }
    D.RR.alloc(4 * 2 * S, s);
    D.RRP.alloc(2 * S, s);
    D.RD.alloc(4 * 2 * S, s);
    D.DL.alloc(4 * 2 * S, s);
    D.PQ.alloc(2 * 2 * S, s);
    D.ACT.alloc(3, s);
    D.THR.alloc(2 * S, s);
    D.out_it.alloc(1, s);
    D.work.alloc(2, s);
    PGCP_CUDA(cudaGetLastError());
    PGCP_CUDA(cudaStreamSynchronize(s));   // host vectors above go out of scope
}

int df_solve(pgcp_ctx* ctx, Part& P, DfSystem& D, const double2* r64, double2* x, const std::vector<double>& thr,
             int max_iters, bool resume) {
    cudaStream_t s = ctx->stream;
    const int S = P.K;
    // Residual replacement: a resumed solve (a refinement step after the
    // first, static schedule, double-float) continues at the last solve's
    // iteration index with x~ = 0, r~ = S r64 (the FP64 residual) and the
    // same search direction p and q = A~ p, instead of restarting CG.  The
    // step's z and <r~, z> are recomputed for the new residual, and beta
    // divides by the <r~, z> of each piece's own last active iteration (RRP),
    // however long ago the piece met its step's threshold.
    resume = resume && D.resumable && D.sched == 1 && !D.det && !D.f32;
    const int k0 = resume ? D.k_last : 0;
    if (resume) {
        PGCP_CUDA(cudaMemsetAsync(D.RR.p + (k0 % 3) * 2 * S, 0, 2 * S * sizeof(double), s));
        PGCP_CUDA(cudaMemsetAsync(D.RD.p + (k0 % 3) * 2 * S, 0, 2 * S * sizeof(double), s));
    } else {
        D.RR.zero();
        D.RD.zero();
    }
    D.DL.zero();
    D.PQ.zero();
    D.ACT.zero();
    if (D.det) {
        D.PRR.zero();
        D.PRD.zero();
        D.PPQ.zero();
        D.RDONE.zero();
    }
    PGCP_CUDA(cudaMemcpyAsync(D.THR.p, thr.data(), 2 * S * sizeof(double), cudaMemcpyHostToDevice, s));
    PGCP_CUDA(cudaMemsetAsync(D.work.p, 0, 2 * sizeof(unsigned long long), s));
    // a previous solve may have left runs over some pieces only: every solve
    // starts (and its prep kernel runs) over all rows
    auto set_runs = [&](const std::vector<uint8_t>* active) {
        std::vector<DfRun> runs;
        std::vector<int32_t> roff;
        D.covered = D.ml ? make_runs_by_piece(P.voff, active, D.grid, runs, roff, 16, ML_SEG)
                         : make_runs(P.voff, active, D.grid, runs, roff);
        if ((int64_t)runs.size() > D.runs_cap) fail(PGCP_E_CUDA, "rebuilt PCG runs exceed their buffer");
        D.nruns = (int32_t)runs.size();
        PGCP_CUDA(cudaMemcpyAsync(D.runs.p, runs.data(), runs.size() * sizeof(DfRun), cudaMemcpyHostToDevice, s));
        PGCP_CUDA(cudaMemcpyAsync(D.run_off.p, roff.data(), roff.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        if (D.nruns > 0) {
            k_run_stats<<<(unsigned)D.nruns, 256, 0, s>>>(D.runs.p, D.rp.p);
            ::pgcp::note_launch();
        }
        PGCP_CUDA(cudaGetLastError());
        PGCP_CUDA(cudaStreamSynchronize(s));   // the host run lists go out of scope
    };
    if (D.covered != D.n) set_runs(nullptr);
    if (D.f32) prep_typed<ArithF32>(ctx, P, D, r64, k0 % 3, resume);
    else prep_typed<ArithDF>(ctx, P, D, r64, k0 % 3, resume);
    if (D.ml) D.ml_M.zero();   // both parities of the preconditioner's moments
    bool first = true;
    auto launch = [&](int k0, int cap) {
        EventPair ev;   // brackets the persistent kernel only
        PGCP_CUDA(cudaEventRecord(ev.a, s));
        if (D.ml) ml_launch(ctx, P, D, k0, cap, first && resume);
        else if (D.f32) launch_typed<ArithF32>(ctx, P, D, k0, cap, first && resume);
        else launch_typed<ArithDF>(ctx, P, D, k0, cap, first && resume);
        PGCP_CUDA(cudaEventRecord(ev.b, s));
        int k_end = 0;
        PGCP_CUDA(cudaMemcpyAsync(&k_end, D.out_it.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        PGCP_CUDA(cudaStreamSynchronize(s));
        float ms = 0.f;
        PGCP_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
        P.stats.pcg_ms += ms;
        P.stats.pcg_launches += 1;
        first = false;
        return k_end;
    };
    int it = k0;
    if (D.sched == 1 && !D.det) {
        // Static schedule: the solve runs in launches of REBALANCE_ITERS
        // iterations.  Between them the host reads which pieces converged;
        // when the rows of the others fall below 3/4 of the rows the runs
        // cover, the runs are rebuilt over those rows alone, so the remaining
        // pieces spread over every block again.  The per-piece accumulators
        // and vectors carry over, and the iteration index continues.
        //
        // With the multilevel preconditioner a step also ends when it stalls:
        // every unconverged piece (coordinate, for Laplace) has gone
        // STALL_ITERS iterations without halving its residual norm squared.
        // That happens only at the double-float floor, where the step cannot
        // reach its threshold; the refinement loop then takes over (normal
        // progress halves it about every hundred iterations).
        constexpr int STALL_ITERS = 2048;
        std::vector<double> rd(2 * (size_t)S), ref(2 * (size_t)S, INFINITY);
        std::vector<int> mark(2 * (size_t)S, it);
        std::vector<uint8_t> active(S, 1);
        while (true) {
            const int cap = (int)std::min<int64_t>((int64_t)k0 + max_iters, (int64_t)it + REBALANCE_ITERS);
            const int k_end = launch(it, cap);
            const bool stopped = k_end < cap;   // every piece converged
            it = k_end;
            if (stopped || it >= k0 + max_iters) break;
            PGCP_CUDA(cudaMemcpyAsync(rd.data(), D.RD.p + (it % 3) * 2 * S, 2 * S * sizeof(double),
                                      cudaMemcpyDeviceToHost, s));
            PGCP_CUDA(cudaStreamSynchronize(s));
            int64_t rows = 0;
            bool progress = false;
            auto watch = [&](int e, double v) {
                if (v <= 0.5 * ref[e]) {
                    ref[e] = v;
                    mark[e] = it;
                }
                if (it - mark[e] < STALL_ITERS) progress = true;
            };
            for (int i = 0; i < S; ++i) {
                bool done;
                if (D.dncp) {
                    done = rd[2 * i] + rd[2 * i + 1] <= thr[2 * i] + thr[2 * i + 1];
                    if (!done) watch(2 * i, rd[2 * i] + rd[2 * i + 1]);
                } else {
                    const bool d0 = rd[2 * i] <= thr[2 * i], d1 = rd[2 * i + 1] <= thr[2 * i + 1];
                    done = d0 && d1;
                    if (!d0) watch(2 * i, rd[2 * i]);
                    if (!d1) watch(2 * i + 1, rd[2 * i + 1]);
                }
                active[i] = done ? 0 : 1;
                if (!done) rows += P.voff[i + 1] - P.voff[i];
            }
            if (D.ml && rows > 0 && !progress) break;
            if (rows > 0 && 4 * rows < 3 * D.covered) set_runs(&active);
        }
    } else {
        it = launch(0, max_iters);
    }
    D.k_last = it;
    D.resumable = true;
    if (D.f32) finish_typed<ArithF32>(ctx, D, x);
    else finish_typed<ArithDF>(ctx, D, x);
    unsigned long long w[2] = {0, 0};
    PGCP_CUDA(cudaMemcpyAsync(w, D.work.p, sizeof(w), cudaMemcpyDeviceToHost, s));
    PGCP_CUDA(cudaStreamSynchronize(s));
    // Algorithmic bytes (the minimal streams of one 2-RHS Jacobi-PCG iteration,
    // T = 8 for FP64-width double-float values, 4 for FP32): per free row the
    // row pointer 4, the diagonal T and nine vector streams of 2T (gathered
    // operand, q written and read, x read and written, r read and written, p
    // read and written) -> 4 + 19T; per stored entry column 4 + value T.  At
    // seven entries a row that is 240 B (double-float) and 136 B (FP32).
    // Touched bytes (what this kernel's schedule streams): per row 8 + 22T.
    // With the multilevel preconditioner: two more vector streams (z written,
    // z read), the vertex position 12 and the preconditioner's block tables.
    const double T = D.f32 ? 4.0 : 8.0;
    if (D.ml) {
        P.stats.pcg_bytes += (double)w[0] * (4.0 + 23.0 * T + 12.0 + D.ml_row_bytes) + (double)w[1] * (4.0 + T);
        P.stats.pcg_bytes_touched += (double)w[0] * (8.0 + 26.0 * T + 24.0 + D.ml_row_bytes) + (double)w[1] * (4.0 + T);
    } else {
        P.stats.pcg_bytes += (double)w[0] * (4.0 + 19.0 * T) + (double)w[1] * (4.0 + T);
        P.stats.pcg_bytes_touched += (double)w[0] * (8.0 + 22.0 * T) + (double)w[1] * (4.0 + T);
    }
    return it - k0;
}

}  // namespace pgcp
