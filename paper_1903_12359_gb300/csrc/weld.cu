// Partial welding (Algorithms 1 and 2, Section 4.3), the disk constraint
// (geodesic algorithm, Sections 3.4 and 4.4.1) and the closed weld of a
// sphere (Section 4.4.2).
//
// Phase 1 (cooperative kernel, one grid sync per zipper step): the arc points
// a_0..a_k, b_0..b_k and the auxiliary points of every weld of a round are
// spread over the blocks.  At each step every block recomputes the step's map
// record from the current image of the point that defines it (identical FP64
// operations, so identical records), stores it, and applies it to the points
// it owns with the index rules (a block keeps its points and the metadata of
// their sequences in shared memory, and publishes every new value into one of
// two global buffers by step parity, which the next step's records read):
//   * points already zipped onto the imaginary axis take the root on their own
//     side of the axis (imaginary part of the root has the sign of Im of the
//     Mobius image);
//   * the previous zip point (at 0) takes the sequence's branch, +i or -i;
//   * the point the step zips goes to 0, the pole of a pole map to infinity.
// Phase 2 applies the recorded chain (principal root) to every other point:
// the rest of the boundary loops in FP64, the interiors in FP32 (warm start of
// the final solve).
//
// The arithmetic (Smith division, own |z|, Kahan-style principal root) is
// written to match the FP64 oracle operation for operation; this file is
// compiled without FMA contraction.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "pgcp_internal.h"

namespace cg = cooperative_groups;

namespace pgcp {

namespace {

enum Mode : int { M_PRINCIPAL = 0, M_SIGN = 1, M_BRANCH = 2, M_ZERO = 3, M_INF = 4 };

struct Pt {
    double r, i;
    int inf;
};

// ---------------------------------------------------------------- FP64 complex kernels

__device__ __forceinline__ void cdiv(double ar, double ai, double br, double bi, double& xr, double& xi) {
    // Smith (1962)
    if (fabs(br) >= fabs(bi)) {
        double r = bi / br;
        double d = br + bi * r;
        xr = (ar + ai * r) / d;
        xi = (ai - ar * r) / d;
    } else {
        double r = br / bi;
        double d = br * r + bi;
        xr = (ar * r + ai) / d;
        xi = (ai * r - ar) / d;
    }
}

__device__ __forceinline__ double chypot(double x, double y) {
    double ax = fabs(x), ay = fabs(y);
    double m = fmax(ax, ay), n = fmin(ax, ay);
    if (m == 0.0) return 0.0;
    double q = n / m;
    return m * sqrt(1.0 + q * q);
}

__device__ __forceinline__ void csqrt_p(double x, double y, double& rr, double& ri) {
    // principal root, after Kahan (1987)
    if (x == 0.0 && y == 0.0) {
        rr = 0.0;
        ri = y;
        return;
    }
    double h = chypot(x, y);
    double t = sqrt((fabs(x) + h) * 0.5);
    double t2 = t + t;
    if (x >= 0.0) {
        rr = t;
        ri = y / t2;
    } else {
        rr = fabs(y) / t2;
        ri = copysign(t, y);
    }
}

__device__ __forceinline__ void root_mode(double wr, double wi, double sr, double si, int mode, double branch,
                                          double& rr, double& ri) {
    csqrt_p(wr, wi, rr, ri);
    if (mode == M_SIGN && ri * si < 0.0) {
        rr = -rr;
        ri = -ri;
    }
    if (mode == M_BRANCH) {
        rr = 0.0;
        ri = branch;
    }
}

__device__ Pt apply_rec(const Rec& R, Pt z, int mode) {
    Pt o{0.0, 0.0, 0};
    const bool fin = !z.inf;
    switch (R.kind) {
        case R_SQRT_RATIO: {
            double wr = 1.0, wi = 0.0;
            if (fin) cdiv(z.r - R.p[2], z.i - R.p[3], z.r - R.p[0], z.i - R.p[1], wr, wi);
            csqrt_p(wr, wi, o.r, o.i);
            break;
        }
        case R_OPEN: {
            const double cr = R.p[0], ci = R.p[1];
            double Mr, Mi;
            if (fin) {
                double Dr = 1.0 - ci * z.i, Di = ci * z.r;
                cdiv(cr * z.r, cr * z.i, Dr, Di, Mr, Mi);
            } else {
                Mr = 0.0;
                Mi = -(cr / ci);
            }
            double sr = Mr * Mr - Mi * Mi, si = Mr * Mi + Mi * Mr;
            root_mode(sr - 1.0, si, Mr, Mi, mode, R.branch, o.r, o.i);
            break;
        }
        case R_CLOSE: {
            const double c1 = R.p[0], c2 = R.p[1];
            double Tr, Ti;
            if (fin) {
                double Dr = c1 + c2 * z.i, Di = -(c2 * z.r);
                cdiv(z.r, z.i, Dr, Di, Tr, Ti);
            } else {
                Tr = 0.0;
                Ti = 1.0 / c2;
            }
            double sr = Tr * Tr - Ti * Ti, si = Tr * Ti + Ti * Tr;
            root_mode(sr + 1.0, si, Tr, Ti, mode, 1.0, o.r, o.i);
            break;
        }
        case R_MOB_POLE:
        case R_POLE_SQ: {
            const double pr = R.p[0], pi = R.p[1];
            double Mr, Mi;
            if (fin) {
                double tr, ti;
                cdiv(z.r, z.i, pr, pi, tr, ti);
                cdiv(z.r, z.i, 1.0 - tr, -ti, Mr, Mi);
            } else {
                Mr = -pr;
                Mi = -pi;
            }
            if (R.kind == R_MOB_POLE) {
                o.r = Mr;
                o.i = Mi;
            } else {
                o.r = Mr * Mr - Mi * Mi;
                o.i = Mr * Mi + Mi * Mr;
            }
            break;
        }
        case R_MOBIUS: {
            const double ar = R.p[0], ai = R.p[1], br = R.p[2], bi = R.p[3];
            const double cr = R.p[4], ci = R.p[5], dr = R.p[6], di = R.p[7];
            if (fin) {
                double nr = (ar * z.r - ai * z.i) + br, ni = (ar * z.i + ai * z.r) + bi;
                double er = (cr * z.r - ci * z.i) + dr, ei = (cr * z.i + ci * z.r) + di;
                cdiv(nr, ni, er, ei, o.r, o.i);
            } else if (cr != 0.0 || ci != 0.0) {
                cdiv(ar, ai, cr, ci, o.r, o.i);
            } else {
                o.inf = 1;
            }
            break;
        }
    }
    if (mode == M_ZERO) {
        o.r = 0.0;
        o.i = 0.0;
        o.inf = 0;
    } else if (mode == M_INF) {
        o.inf = 1;
    }
    if (o.inf) {
        o.r = 0.0;
        o.i = 0.0;
    }
    return o;
}

// ---------------------------------------------------------------- record builders

__device__ Rec rec_sqrt_ratio(Pt z0, Pt z1) {
    Rec R{};
    R.kind = R_SQRT_RATIO;
    R.branch = 1.0;
    R.p[0] = z0.r;
    R.p[1] = z0.i;
    R.p[2] = z1.r;
    R.p[3] = z1.i;
    return R;
}

__device__ Rec rec_open(Pt xi, double branch, bool& ok) {
    Rec R{};
    R.kind = R_OPEN;
    R.branch = branch;
    ok = !xi.inf && xi.r > 0.0;
    double s = xi.r * xi.r + xi.i * xi.i;
    R.p[0] = xi.r / s;
    R.p[1] = xi.i / s;
    return R;
}

__device__ Rec rec_pole(int kind, Pt p, bool& ok) {
    Rec R{};
    R.kind = kind;
    R.branch = 1.0;
    ok = !p.inf;
    R.p[0] = p.r;
    R.p[1] = p.i;
    return R;
}

__device__ Rec rec_close(double a, double b, bool& ok) {
    Rec R{};
    R.kind = R_CLOSE;
    R.branch = 1.0;
    double amb = a - b;
    double c1 = ((-2.0 * a) * b) / amb;
    double c2 = (a + b) / amb;
    ok = amb != 0.0 && c1 > 0.0 && isfinite(c1) && isfinite(c2) && c2 != 0.0;
    R.p[0] = c1;
    R.p[1] = c2;
    return R;
}

__device__ __forceinline__ void cmul(double ar, double ai, double br, double bi, double& xr, double& xi) {
    xr = ar * br - ai * bi;
    xi = ar * bi + ai * br;
}

__device__ Rec rec_mobius(double ar, double ai, double br, double bi, double cr, double ci, double dr, double di) {
    Rec R{};
    R.kind = R_MOBIUS;
    R.branch = 1.0;
    R.p[0] = ar; R.p[1] = ai; R.p[2] = br; R.p[3] = bi;
    R.p[4] = cr; R.p[5] = ci; R.p[6] = dr; R.p[7] = di;
    return R;
}

// p1 -> -1, p2 -> 1, p3 -> inf
__device__ Rec rec_normalize(Pt p1, Pt p2, double p3r, double p3i) {
    double ur = p2.r - p3r, ui = p2.i - p3i;
    double vr = p2.r - p1.r, vi = p2.i - p1.i;
    double tr = ur + ur, ti = ui + ui;
    double ar = tr - vr, ai = ti - vi;
    double vp3r, vp3i, tp1r, tp1i;
    cmul(vr, vi, p3r, p3i, vp3r, vp3i);
    cmul(tr, ti, p1.r, p1.i, tp1r, tp1i);
    return rec_mobius(ar, ai, vp3r - tp1r, vp3i - tp1i, vr, vi, -vp3r, -vp3i);
}

// p1 -> 0, p2 -> inf, q -> 1 (inverted: the reciprocal)
__device__ Rec rec_sphere_frame(Pt p1, Pt p2, Pt q, bool invert) {
    double ar = q.r - p2.r, ai = q.i - p2.i;
    double cr = q.r - p1.r, ci = q.i - p1.i;
    double br, bi, dr, di;
    cmul(ar, ai, p1.r, p1.i, br, bi);
    cmul(cr, ci, p2.r, p2.i, dr, di);
    if (!invert) return rec_mobius(ar, ai, -br, -bi, cr, ci, -dr, -di);
    return rec_mobius(cr, ci, -dr, -di, ar, ai, -br, -bi);
}

// ---------------------------------------------------------------- phase 1: welds

struct SeqMeta {          // one zipper sequence (A or B side of a weld)
    int64_t off;          // first point in the point arrays
    int32_t k;            // arc length (points 0..k), extras at k+1, k+2
    int32_t job;          // weld within the round
    int32_t side;         // 0 = A (C side, +i), 1 = B (S side, -i)
    int32_t pad;
};

struct JobMeta {
    int32_t seqA, seqB;   // sequence ids
    int32_t k;
    int32_t closed;
    int64_t rec_gA, rec_gB, rec_h, rec_TA, rec_TB;   // record slots
    int64_t arc_off;      // arc outputs [k+1] per side
};

struct Phase1Args {
    double* pr;           // point arrays, two buffers of npts (step parity)
    double* pi;
    int32_t* pinf;
    int64_t npts;
    const int32_t* __restrict__ item_seq;   // sequence of each point
    const SeqMeta* __restrict__ seqs;
    int32_t nseq;
    const JobMeta* __restrict__ jobs;
    int32_t kmax;
    Rec* recs;            // record store
    double2* arcA;        // arc outputs
    double2* arcB;
    uint32_t* err;
    int32_t* fail_job;    // first failing job (for the message)
    int32_t* job_fail;    // [jobs] 1 if the job left its domain
};

// Published point values, two buffers by step parity (buffer b at offset b *
// npts): the records of step s read buffer s & 1 while the owners write the
// step's new values into the other, so no block reads a value that its owner
// has already advanced.
__device__ __forceinline__ Pt ldp(const Phase1Args& a, int b, int64_t i) {
    const int64_t j = b * a.npts + i;
    return Pt{a.pr[j], a.pi[j], a.pinf[j]};
}
__device__ __forceinline__ void stp(const Phase1Args& a, int b, int64_t i, Pt p) {
    const int64_t j = b * a.npts + i;
    a.pr[j] = p.r;
    a.pi[j] = p.i;
    a.pinf[j] = p.inf;
}

// A sequence's metadata as phase 1 keeps it in shared memory: its own
// descriptor, its weld's, and the first points of the weld's A and B sides.
struct SeqCache {
    SeqMeta m;
    JobMeta J;
    int64_t offA, offB;
};

// Record of a sequence at step `step` (0-based over the whole program) and
// whether the sequence is active.  Steps: 0..k (Alg 1: g_1..g_{k+1}),
// k+1..2k (Alg 2: h_{k-1}..h_1, h_0), 2k+1 (normalisation).  The points come
// from global memory (their owners publish them every step).
__device__ bool seq_record(const Phase1Args& a, const SeqCache& c, int step, Rec& R, bool& ok) {
    const SeqMeta& m = c.m;
    const int b = step & 1;
    const int k = m.k;
    ok = true;
    const int64_t o = m.off;
    if (step == 0) {
        R = rec_sqrt_ratio(ldp(a, b, o), ldp(a, b, o + 1));
        return true;
    }
    if (step <= k - 1) {   // OPEN for j = step + 1 in 2..k
        R = rec_open(ldp(a, b, o + step + 1), m.side == 0 ? 1.0 : -1.0, ok);
        return true;
    }
    if (step == k) {
        R = rec_pole(R_MOB_POLE, ldp(a, b, o), ok);
        return true;
    }
    if (step <= 2 * k - 1) {   // h_j, j = 2k - step... j runs k-1 .. 1
        int j = 2 * k - step;
        R = rec_close(a.pi[b * a.npts + c.offA + j], a.pi[b * a.npts + c.offB + j], ok);
        return true;
    }
    if (step == 2 * k) {
        R = rec_pole(R_POLE_SQ, ldp(a, b, c.offA), ok);
        return true;
    }
    if (step == 2 * k + 1) {
        Pt p1 = ldp(a, b, c.offA + k + 1), p2 = ldp(a, b, c.offB + k + 1);
        if (c.J.closed) {
            Pt q = ldp(a, b, c.offA + k / 2);
            R = rec_sphere_frame(p1, p2, q, m.side == 1);
        } else {
            Pt ia = ldp(a, b, c.offA + k + 2), ib = ldp(a, b, c.offB + k + 2);
            R = rec_normalize(p1, p2, (ia.r + ib.r) * 0.5, (ia.i + ib.i) * 0.5);
        }
        ok = !p1.inf && !p2.inf;
        return true;
    }
    return false;
}

__device__ int seq_mode(int k, int step, int l, int& kind_hint) {
    (void)kind_hint;
    if (l > k) return M_PRINCIPAL;   // auxiliary points
    if (step == 0) return l == 0 ? M_INF : (l == 1 ? M_ZERO : M_PRINCIPAL);
    if (step <= k - 1) {
        int j = step + 1;
        return l < j - 1 ? M_SIGN : (l == j - 1 ? M_BRANCH : (l == j ? M_ZERO : M_PRINCIPAL));
    }
    if (step == k) return l == 0 ? M_INF : (l == k ? M_ZERO : M_PRINCIPAL);
    if (step <= 2 * k - 1) {
        int j = 2 * k - step;
        return l < j ? M_SIGN : (l == j ? M_ZERO : M_PRINCIPAL);
    }
    if (step == 2 * k) return l == 0 ? M_INF : M_PRINCIPAL;
    return M_PRINCIPAL;
}

constexpr int P1_THREADS = 64;
constexpr int P1_MAXSEQ = 32;  // sequences overlapping one block's item range (checked on the host)

// Shared memory of a phase-1 block: per owned point its value (r, i, inf),
// its sequence (local index) and its index l in the sequence; the records and
// metadata of the sequences its points belong to.
constexpr int P1_PT_BYTES = 8 + 8 + 4 + 4 + 4;

__global__ void __launch_bounds__(P1_THREADS) k_weld_phase1(Phase1Args a) {
    cg::grid_group grid = cg::this_grid();
    __shared__ Rec srec[P1_MAXSEQ];
    __shared__ int sact[P1_MAXSEQ];
    __shared__ SeqCache sc[P1_MAXSEQ];
    extern __shared__ __align__(16) unsigned char p1_smem[];
    const int64_t per = (a.npts + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * per;
    const int64_t hi = min(a.npts, lo + per);
    const int np = hi > lo ? (int)(hi - lo) : 0;
    double* zr = reinterpret_cast<double*>(p1_smem);
    double* zi = zr + per;
    int32_t* zinf = reinterpret_cast<int32_t*>(zi + per);
    int32_t* zseq = zinf + per;
    int32_t* zl = zseq + per;
    const int seq_lo = lo < hi ? a.item_seq[lo] : 0;
    const int seq_hi = lo < hi ? a.item_seq[hi - 1] : -1;
    const int nsq = seq_hi - seq_lo + 1;
    if (threadIdx.x < nsq && threadIdx.x < P1_MAXSEQ) {
        SeqCache c;
        c.m = a.seqs[seq_lo + threadIdx.x];
        c.J = a.jobs[c.m.job];
        c.offA = a.seqs[c.J.seqA].off;
        c.offB = a.seqs[c.J.seqB].off;
        sc[threadIdx.x] = c;
    }
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
        const int64_t i = lo + t;
        zr[t] = a.pr[i];
        zi[t] = a.pi[i];
        zinf[t] = a.pinf[i];
        zseq[t] = a.item_seq[i] - seq_lo;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < np; t += blockDim.x)
        zl[t] = zseq[t] < P1_MAXSEQ ? (int)(lo + t - sc[zseq[t]].m.off) : 0;
    const int nsteps = 2 * a.kmax + 2;
    for (int step = 0; step < nsteps; ++step) {
        if (threadIdx.x < nsq && threadIdx.x < P1_MAXSEQ) {
            const SeqCache& c = sc[threadIdx.x];
            Rec R;
            bool ok = true;
            bool act = seq_record(a, c, step, R, ok);
            sact[threadIdx.x] = act;
            srec[threadIdx.x] = R;
            if (act && !ok) {
                atomicOr(a.err, (uint32_t)DE_WELD_DOMAIN);
                atomicMin(a.fail_job, c.m.job);
                atomicOr(&a.job_fail[c.m.job], 1);
            }
            // the block owning the first point of the sequence stores the record
            if (act && c.m.off >= lo && c.m.off < hi) {
                const int k = c.m.k;
                if (step <= k) a.recs[(c.m.side == 0 ? c.J.rec_gA : c.J.rec_gB) + step] = R;
                else if (step <= 2 * k) {
                    if (c.m.side == 0) a.recs[c.J.rec_h + (step - k - 1)] = R;
                } else {
                    a.recs[c.m.side == 0 ? c.J.rec_TA : c.J.rec_TB] = R;
                }
            }
        }
        __syncthreads();
        // apply to owned points (the normalisation step writes the arc outputs);
        // every new value is published for the other blocks' records
        for (int t = threadIdx.x; t < np; t += blockDim.x) {
            const int si = zseq[t];
            if (si >= P1_MAXSEQ || !sact[si]) continue;
            const SeqMeta& m = sc[si].m;
            const int l = zl[t];
            const Pt z{zr[t], zi[t], zinf[t]};
            if (step == 2 * m.k + 1) {
                if (l <= m.k) {
                    Pt o = apply_rec(srec[si], z, M_PRINCIPAL);
                    double2* dst = (m.side == 0 ? a.arcA : a.arcB) + sc[si].J.arc_off + l;
                    *dst = make_double2(o.r, o.i);
                    if (o.inf) {
                        atomicOr(a.err, (uint32_t)DE_WELD_DOMAIN);
                        atomicOr(&a.job_fail[m.job], 1);
                    }
                }
                continue;
            }
            int hint = 0;
            const Pt o = apply_rec(srec[si], z, seq_mode(m.k, step, l, hint));
            zr[t] = o.r;
            zi[t] = o.i;
            zinf[t] = o.inf;
            stp(a, (step + 1) & 1, lo + t, o);
        }
        grid.sync();
    }
    for (int t = threadIdx.x; t < np; t += blockDim.x) stp(a, 0, lo + t, Pt{zr[t], zi[t], zinf[t]});
}

// ---------------------------------------------------------------- phase 1: disk

struct DiskMeta {
    int64_t off;          // loop points 0..n, centre at n+1
    int32_t n;
    int32_t pad;
    int64_t rec;          // records: n+2 (g_1..g_n, pole square, disk frame)
};

struct DiskArgs {
    double* pr;           // point arrays, two buffers of npts (step parity)
    double* pi;
    int32_t* pinf;
    int64_t npts;
    const int32_t* __restrict__ item_seq;
    const DiskMeta* __restrict__ seqs;
    int32_t nseq;
    int32_t nmax;
    Rec* recs;
    uint32_t* err;
    int32_t* seq_fail;    // [nseq] 1 if the sequence left its domain
};

// Record of a disk sequence at step `step`; points from buffer step & 1 of
// the published values (two buffers of npts, as in phase 1 of the welds).
__device__ bool disk_record(const DiskArgs& a, const DiskMeta& m, int step, Rec& R, bool& ok) {
    const int n = m.n;
    const int64_t o = m.off + (step & 1) * a.npts;
    ok = true;
    if (step == 0) {
        R = rec_sqrt_ratio(Pt{a.pr[o], a.pi[o], a.pinf[o]}, Pt{a.pr[o + 1], a.pi[o + 1], a.pinf[o + 1]});
        return true;
    }
    if (step <= n - 1) {
        R = rec_open(Pt{a.pr[o + step + 1], a.pi[o + step + 1], a.pinf[o + step + 1]}, 1.0, ok);
        return true;
    }
    if (step == n) {
        R = rec_pole(R_POLE_SQ, Pt{a.pr[o], a.pi[o], a.pinf[o]}, ok);
        return true;
    }
    if (step == n + 1) {   // upper half-plane -> disk, centre image -> 0
        double cr = a.pr[o + n + 1], ci = a.pi[o + n + 1];
        ok = !a.pinf[o + n + 1] && ci > 0.0;
        R = rec_mobius(1.0, 0.0, -cr, -ci, 1.0, 0.0, -cr, ci);
        return true;
    }
    return false;
}

__device__ int disk_mode(int n, int step, int l) {
    if (l > n) return M_PRINCIPAL;
    if (step == 0) return l == 0 ? M_INF : (l == 1 ? M_ZERO : M_PRINCIPAL);
    if (step <= n - 1) {
        int j = step + 1;
        return l < j - 1 ? M_SIGN : (l == j - 1 ? M_BRANCH : (l == j ? M_ZERO : M_PRINCIPAL));
    }
    if (step == n) return l == 0 ? M_INF : (l == n ? M_ZERO : M_PRINCIPAL);
    return M_PRINCIPAL;
}

__global__ void __launch_bounds__(P1_THREADS) k_disk_phase1(DiskArgs a) {
    cg::grid_group grid = cg::this_grid();
    __shared__ Rec srec[P1_MAXSEQ];
    __shared__ int sact[P1_MAXSEQ];
    __shared__ DiskMeta sm[P1_MAXSEQ];
    extern __shared__ __align__(16) unsigned char p1_smem[];
    const int64_t per = (a.npts + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * per;
    const int64_t hi = min(a.npts, lo + per);
    const int np = hi > lo ? (int)(hi - lo) : 0;
    double* zr = reinterpret_cast<double*>(p1_smem);
    double* zi = zr + per;
    int32_t* zinf = reinterpret_cast<int32_t*>(zi + per);
    int32_t* zseq = zinf + per;
    int32_t* zl = zseq + per;
    const int seq_lo = lo < hi ? a.item_seq[lo] : 0;
    const int seq_hi = lo < hi ? a.item_seq[hi - 1] : -1;
    const int nsq = seq_hi - seq_lo + 1;
    if (threadIdx.x < nsq && threadIdx.x < P1_MAXSEQ) sm[threadIdx.x] = a.seqs[seq_lo + threadIdx.x];
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
        const int64_t i = lo + t;
        zr[t] = a.pr[i];
        zi[t] = a.pi[i];
        zinf[t] = a.pinf[i];
        zseq[t] = a.item_seq[i] - seq_lo;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < np; t += blockDim.x)
        zl[t] = zseq[t] < P1_MAXSEQ ? (int)(lo + t - sm[zseq[t]].off) : 0;
    const int nsteps = a.nmax + 2;
    for (int step = 0; step < nsteps; ++step) {
        if (threadIdx.x < nsq && threadIdx.x < P1_MAXSEQ) {
            const DiskMeta& m = sm[threadIdx.x];
            Rec R;
            bool ok = true;
            bool act = disk_record(a, m, step, R, ok);
            sact[threadIdx.x] = act;
            srec[threadIdx.x] = R;
            if (act && !ok) {
                atomicOr(a.err, (uint32_t)DE_WELD_DOMAIN);
                atomicOr(&a.seq_fail[seq_lo + threadIdx.x], 1);
            }
            if (act && m.off >= lo && m.off < hi) a.recs[m.rec + step] = R;
        }
        __syncthreads();
        const int64_t wb = ((step + 1) & 1) * a.npts;   // the buffer this step publishes into
        for (int t = threadIdx.x; t < np; t += blockDim.x) {
            const int si = zseq[t];
            if (si >= P1_MAXSEQ || !sact[si]) continue;
            const Pt o = apply_rec(srec[si], Pt{zr[t], zi[t], zinf[t]}, disk_mode(sm[si].n, step, zl[t]));
            zr[t] = o.r;
            zi[t] = o.i;
            zinf[t] = o.inf;
            a.pr[wb + lo + t] = o.r;
            a.pi[wb + lo + t] = o.i;
            a.pinf[wb + lo + t] = o.inf;
        }
        grid.sync();
    }
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
        a.pr[lo + t] = zr[t];
        a.pi[lo + t] = zi[t];
        a.pinf[lo + t] = zinf[t];
    }
}

// ---------------------------------------------------------------- phase 2

struct ChainRef {         // a chain = consecutive record ranges
    int64_t r0, n0;       // g records
    int64_t r1, n1;       // h records
    int64_t r2, n2;       // final record(s)
};

// FP64: apply one chain to listed rows (principal root); rows listed with
// arc >= 0 take arc value instead, from arc_b for odd chains (the B sides of
// welds) when arc_b is given, else from arc_vals.  Every item writes only its
// own row, so both sides of every weld of a round run in one launch.
__global__ void k_phase2_boundary(const int32_t* __restrict__ rows, const int32_t* __restrict__ arc_idx,
                                  const int32_t* __restrict__ item_chain, int64_t nitems,
                                  const ChainRef* __restrict__ chains, const Rec* __restrict__ recs,
                                  const double2* __restrict__ arc_vals, const double2* __restrict__ arc_b,
                                  double2* __restrict__ W, uint32_t* err) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nitems) return;
    const int row = rows[t];
    const int ai = arc_idx[t];
    if (ai >= 0) {
        W[row] = (arc_b && (item_chain[t] & 1)) ? arc_b[ai] : arc_vals[ai];
        return;
    }
    const ChainRef c = chains[item_chain[t]];
    Pt z{W[row].x, W[row].y, 0};
    for (int64_t j = 0; j < c.n0; ++j) z = apply_rec(recs[c.r0 + j], z, M_PRINCIPAL);
    for (int64_t j = 0; j < c.n1; ++j) z = apply_rec(recs[c.r1 + j], z, M_PRINCIPAL);
    for (int64_t j = 0; j < c.n2; ++j) z = apply_rec(recs[c.r2 + j], z, M_PRINCIPAL);
    if (z.inf || !isfinite(z.r) || !isfinite(z.i)) atomicOr(err, (uint32_t)DE_NUMERIC);
    W[row] = make_double2(z.r, z.i);
}

// ---------------------------------------------------------------- interior map (FP32)

struct RecF {
    int32_t kind;
    float p[8];
};

__global__ void k_recs_to_f32(const Rec* __restrict__ r, RecF* __restrict__ f, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    RecF o;
    o.kind = r[i].kind;
    for (int j = 0; j < 8; ++j) o.p[j] = (float)r[i].p[j];
    f[i] = o;
}

__device__ __forceinline__ float2 fdiv(float ar, float ai, float br, float bi) {
    float inv = 1.0f / (br * br + bi * bi);
    if (!(isfinite(inv))) {
        if (fabsf(br) >= fabsf(bi)) {
            float r = bi / br, d = br + bi * r;
            return make_float2((ar + ai * r) / d, (ai - ar * r) / d);
        }
        float r = br / bi, d = br * r + bi;
        return make_float2((ar * r + ai) / d, (ai * r - ar) / d);
    }
    return make_float2((ar * br + ai * bi) * inv, (ai * br - ar * bi) * inv);
}

__device__ __forceinline__ float2 fsqrt_p(float x, float y) {
    float h = hypotf(x, y);
    float t = sqrtf((fabsf(x) + h) * 0.5f);
    if (t == 0.0f) return make_float2(0.0f, y);
    if (x >= 0.0f) return make_float2(t, y / (2.0f * t));
    return make_float2(fabsf(y) / (2.0f * t), copysignf(t, y));
}

__device__ float2 apply_rec_f(const RecF& R, float2 z) {
    switch (R.kind) {
        case R_SQRT_RATIO: {
            float2 w = fdiv(z.x - R.p[2], z.y - R.p[3], z.x - R.p[0], z.y - R.p[1]);
            return fsqrt_p(w.x, w.y);
        }
        case R_OPEN: {
            float cr = R.p[0], ci = R.p[1];
            float2 M = fdiv(cr * z.x, cr * z.y, 1.0f - ci * z.y, ci * z.x);
            return fsqrt_p(M.x * M.x - M.y * M.y - 1.0f, 2.0f * M.x * M.y);
        }
        case R_CLOSE: {
            float c1 = R.p[0], c2 = R.p[1];
            float2 T = fdiv(z.x, z.y, c1 + c2 * z.y, -c2 * z.x);
            return fsqrt_p(T.x * T.x - T.y * T.y + 1.0f, 2.0f * T.x * T.y);
        }
        case R_MOB_POLE:
        case R_POLE_SQ: {
            float2 t = fdiv(z.x, z.y, R.p[0], R.p[1]);
            float2 M = fdiv(z.x, z.y, 1.0f - t.x, -t.y);
            if (R.kind == R_MOB_POLE) return M;
            return make_float2(M.x * M.x - M.y * M.y, 2.0f * M.x * M.y);
        }
        default: {
            float nr = R.p[0] * z.x - R.p[1] * z.y + R.p[2], ni = R.p[0] * z.y + R.p[1] * z.x + R.p[3];
            float er = R.p[4] * z.x - R.p[5] * z.y + R.p[6], ei = R.p[4] * z.y + R.p[5] * z.x + R.p[7];
            return fdiv(nr, ni, er, ei);
        }
    }
}

// One thread per interior row: all chains of its piece, in order.
__global__ void k_interior_map(int64_t n, const uint8_t* __restrict__ is_bnd, const int32_t* __restrict__ row_piece,
                               const int64_t* __restrict__ piece_chain_off, const int32_t* __restrict__ piece_chains,
                               const ChainRef* __restrict__ chains, const RecF* __restrict__ recs,
                               double2* __restrict__ W) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || is_bnd[i]) return;
    const int pc = row_piece[i];
    float2 z = make_float2((float)W[i].x, (float)W[i].y);
    for (int64_t c = piece_chain_off[pc]; c < piece_chain_off[pc + 1]; ++c) {
        const ChainRef ch = chains[piece_chains[c]];
        for (int64_t j = 0; j < ch.n0; ++j) z = apply_rec_f(recs[ch.r0 + j], z);
        for (int64_t j = 0; j < ch.n1; ++j) z = apply_rec_f(recs[ch.r1 + j], z);
        for (int64_t j = 0; j < ch.n2; ++j) z = apply_rec_f(recs[ch.r2 + j], z);
    }
    W[i] = make_double2((double)z.x, (double)z.y);
}

// Same in FP64 (testing option).
__global__ void k_interior_map64(int64_t n, const uint8_t* __restrict__ is_bnd, const int32_t* __restrict__ row_piece,
                                 const int64_t* __restrict__ piece_chain_off,
                                 const int32_t* __restrict__ piece_chains, const ChainRef* __restrict__ chains,
                                 const Rec* __restrict__ recs, double2* __restrict__ W) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || is_bnd[i]) return;
    const int pc = row_piece[i];
    Pt z{W[i].x, W[i].y, 0};
    for (int64_t c = piece_chain_off[pc]; c < piece_chain_off[pc + 1]; ++c) {
        const ChainRef ch = chains[piece_chains[c]];
        for (int64_t j = 0; j < ch.n0; ++j) z = apply_rec(recs[ch.r0 + j], z, M_PRINCIPAL);
        for (int64_t j = 0; j < ch.n1; ++j) z = apply_rec(recs[ch.r1 + j], z, M_PRINCIPAL);
        for (int64_t j = 0; j < ch.n2; ++j) z = apply_rec(recs[ch.r2 + j], z, M_PRINCIPAL);
    }
    W[i] = make_double2(z.r, z.i);
}

__global__ void k_gather_points(const int32_t* __restrict__ rows, const double* __restrict__ xr,
                                const double* __restrict__ xi, const int32_t* __restrict__ xinf, int64_t n,
                                const double2* __restrict__ W, double* __restrict__ pr, double* __restrict__ pi,
                                int32_t* __restrict__ pinf) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int r = rows[t];
    if (r >= 0) {
        pr[t] = W[r].x;
        pi[t] = W[r].y;
        pinf[t] = 0;
    } else {   // literal point (auxiliary)
        pr[t] = xr[t];
        pi[t] = xi[t];
        pinf[t] = xinf[t];
    }
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, ceil_div(n, t)); }

template <typename T>
void upload(DBuf<T>& d, const std::vector<T>& h, cudaStream_t s) {
    d.alloc(h.size(), s);
    if (!h.empty()) PGCP_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

// Grid of a phase-1 kernel: one point per thread, at most what stays
// resident with the per-point shared memory (P1_PT_BYTES each) that the block
// range needs; sets the kernel's dynamic shared memory limit and returns the
// bytes to launch with.
int coop_grid_pts(pgcp_ctx* ctx, const void* kernel, int64_t npts, size_t* smem) {
    int64_t grid = std::max<int64_t>(1, ceil_div(npts, (int64_t)P1_THREADS));
    for (int pass = 0; pass < 4; ++pass) {
        const int64_t per = ceil_div(npts, grid);
        *smem = (size_t)per * P1_PT_BYTES;
        if (*smem > (size_t)227 * 1024) fail(PGCP_E_ARG, "too many welding points for one phase-1 launch");
        PGCP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem));
        int per_sm = 0;
        PGCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, P1_THREADS, *smem));
        const int64_t cap = std::max<int64_t>(1, (int64_t)per_sm * ctx->num_sms);
        if (grid <= cap) return (int)grid;
        grid = cap;
    }
    const int64_t per = ceil_div(npts, grid);
    *smem = (size_t)per * P1_PT_BYTES;
    return (int)grid;
}

// Every block's contiguous item range may meet at most P1_MAXSEQ sequences.
void check_block_sequences(const std::vector<int32_t>& item_seq, int grid) {
    const int64_t n = (int64_t)item_seq.size();
    const int64_t per = ceil_div(n, grid);
    for (int64_t lo = 0; lo < n; lo += per) {
        int64_t hi = std::min(n, lo + per);
        if (item_seq[hi - 1] - item_seq[lo] + 1 > P1_MAXSEQ)
            fail(PGCP_E_ARG, "too many short welding sequences per block (batch too large for one launch)");
    }
}

}  // namespace

// ---------------------------------------------------------------- driver

void run_welds(pgcp_ctx* ctx, Part& P) {
    cudaStream_t s = ctx->stream;
    const pgcp_options& o = ctx->opt;
    const int nmesh = (int)P.meshes.size();
    // welds grouped by mesh, in order
    std::vector<std::vector<int>> by_mesh(nmesh);
    for (size_t w = 0; w < P.welds.size(); ++w) by_mesh[P.welds[w].mesh].push_back((int)w);
    // one round per level: the welds of a level (of every mesh) join disjoint components
    size_t rounds = 0;
    for (const WeldPlan& W : P.welds) rounds = std::max(rounds, (size_t)W.level + 1);
    P.welded.alloc(P.Nc, s);
    PGCP_CUDA(cudaMemcpyAsync(P.welded.p, P.local.p, P.Nc * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    // record store (sizes known from the plans)
    int64_t nrec = 0;
    std::vector<JobMeta> all_jobs(P.welds.size());
    for (size_t w = 0; w < P.welds.size(); ++w) {
        const WeldPlan& W = P.welds[w];
        JobMeta& J = all_jobs[w];
        J.k = W.k;
        J.closed = W.closed;
        J.rec_gA = nrec; nrec += W.k + 1;
        J.rec_gB = nrec; nrec += W.k + 1;
        J.rec_h = nrec; nrec += W.k;
        J.rec_TA = nrec; nrec += 1;
        J.rec_TB = nrec; nrec += 1;
    }
    std::vector<int64_t> disk_rec(nmesh, -1), disk_n(nmesh, 0);
    std::vector<std::vector<int32_t>> disk_loop(nmesh);
    if (o.variant == PGCP_DISK) {
        for (int mi = 0; mi < nmesh; ++mi) {
            const MeshInfo& M = P.meshes[mi];
            std::vector<int32_t> loop;
            if (!by_mesh[mi].empty()) loop = P.welds[by_mesh[mi].back()].new_loop;
            else loop.assign(P.loop_glob.begin() + P.loff[M.piece0], P.loop_glob.begin() + P.loff[M.piece0 + 1]);
            disk_loop[mi] = loop;
            disk_n[mi] = (int64_t)loop.size() - 1;
            disk_rec[mi] = nrec;
            nrec += (int64_t)loop.size() + 1;
        }
    }
    DBuf<Rec> recs;
    recs.alloc(std::max<int64_t>(nrec, 1), s);
    // arc outputs
    int64_t narc = 0;
    for (size_t w = 0; w < P.welds.size(); ++w) {
        all_jobs[w].arc_off = narc;
        narc += P.welds[w].k + 1;
    }
    DBuf<double2> arcA, arcB;
    arcA.alloc(std::max<int64_t>(narc, 1), s);
    arcB.alloc(std::max<int64_t>(narc, 1), s);
    DBuf<int32_t> fail_job;
    fail_job.alloc(1, s);
    std::vector<ChainRef> chains;          // per weld: A chain at 2w, B chain at 2w+1; disks after
    for (size_t w = 0; w < P.welds.size(); ++w) {
        const JobMeta& J = all_jobs[w];
        chains.push_back(ChainRef{J.rec_gA, J.k + 1, J.rec_h, J.k, J.rec_TA, 1});
        chains.push_back(ChainRef{J.rec_gB, J.k + 1, J.rec_h, J.k, J.rec_TB, 1});
    }
    std::vector<int> disk_chain(nmesh, -1);
    for (int mi = 0; mi < nmesh; ++mi)
        if (disk_rec[mi] >= 0) {
            disk_chain[mi] = (int)chains.size();
            chains.push_back(ChainRef{disk_rec[mi], disk_n[mi] + 2, 0, 0, 0, 0});
        }
    DBuf<ChainRef> d_chains;
    upload(d_chains, chains, s);
    ctx->err.zero();
    // position of a global vertex in the arc (or loop) being looked up, -1
    // elsewhere: set for one weld's arc, read for its pieces' loops, reset
    int32_t gmax = 0;
    for (int32_t g : P.loop_glob) gmax = std::max(gmax, g);
    std::vector<int64_t> gpos((size_t)gmax + 1, -1);
    // A mesh of a batch whose welding leaves its domain is dropped (status
    // NUMERIC, output NaN) and the others go on; a single mesh fails the call.
    std::vector<uint8_t> mfail(nmesh, 0);
    auto mesh_failed = [&](int mi, const std::string& why) {
        if (nmesh == 1) fail(PGCP_E_NUMERIC, why);
        mfail[mi] = 1;
    };
    // meshes with a non-finite welded boundary value (only looked at after the flag)
    auto check_finite = [&](const std::string& why) {
        if (!(read_errors(ctx) & DE_NUMERIC)) return;
        if (nmesh == 1) fail(PGCP_E_NUMERIC, why);
        std::vector<double2> hw(P.Nc);
        PGCP_CUDA(cudaMemcpyAsync(hw.data(), P.welded.p, P.Nc * sizeof(double2), cudaMemcpyDeviceToHost, s));
        PGCP_CUDA(cudaStreamSynchronize(s));
        for (int mi = 0; mi < nmesh; ++mi) {
            const MeshInfo& M = P.meshes[mi];
            for (int32_t pc = M.piece0; pc < M.piece0 + M.npiece && !mfail[mi]; ++pc)
                for (int64_t t = P.loff[pc]; t < P.loff[pc + 1]; ++t) {
                    const double2 z = hw[P.loop_rows[t]];
                    if (!std::isfinite(z.x) || !std::isfinite(z.y)) {
                        mfail[mi] = 1;
                        break;
                    }
                }
        }
        ctx->err.zero();
    };
    for (size_t r = 0; r < rounds; ++r) {
        std::vector<int> jobs_w;
        for (size_t w = 0; w < P.welds.size(); ++w)
            if ((size_t)P.welds[w].level == r && !mfail[P.welds[w].mesh]) jobs_w.push_back((int)w);
        if (jobs_w.empty()) continue;
        // ---- phase 1 inputs
        std::vector<SeqMeta> seqs;
        std::vector<JobMeta> jobs;
        std::vector<int32_t> item_seq, rows;
        std::vector<double> xr, xi;
        std::vector<int32_t> xinf;
        int kmax = 0;
        for (size_t jj = 0; jj < jobs_w.size(); ++jj) {
            const WeldPlan& W = P.welds[jobs_w[jj]];
            JobMeta J = all_jobs[jobs_w[jj]];
            kmax = std::max(kmax, W.k);
            for (int side = 0; side < 2; ++side) {
                SeqMeta m{(int64_t)item_seq.size(), W.k, (int32_t)jj, side, 0};
                const int sid = (int)seqs.size();
                if (side == 0) J.seqA = sid;
                else J.seqB = sid;
                seqs.push_back(m);
                for (int l = 0; l <= W.k; ++l) {
                    item_seq.push_back(sid);
                    rows.push_back((int32_t)(side == 0 ? W.a_rows[l] : W.b_rows[l]));
                    xr.push_back(0);
                    xi.push_back(0);
                    xinf.push_back(0);
                }
                // auxiliary points: the side's reference (0 for a single piece,
                // -1 for a welded component) and infinity
                double ref = (side == 0 ? W.a_single : W.b_single) ? 0.0 : -1.0;
                item_seq.push_back(sid); rows.push_back(-1); xr.push_back(ref); xi.push_back(0); xinf.push_back(0);
                item_seq.push_back(sid); rows.push_back(-1); xr.push_back(0); xi.push_back(0); xinf.push_back(1);
            }
            jobs.push_back(J);
        }
        const int64_t npts = (int64_t)item_seq.size();
        DBuf<int32_t> d_item_seq, d_rows, d_xinf, d_pinf;
        DBuf<double> d_xr, d_xi, d_pr, d_pi;
        DBuf<SeqMeta> d_seqs;
        DBuf<JobMeta> d_jobs;
        upload(d_item_seq, item_seq, s);
        upload(d_rows, rows, s);
        upload(d_xr, xr, s);
        upload(d_xi, xi, s);
        upload(d_xinf, xinf, s);
        upload(d_seqs, seqs, s);
        upload(d_jobs, jobs, s);
        d_pr.alloc(2 * npts, s);   // two buffers (step parity)
        d_pi.alloc(2 * npts, s);
        d_pinf.alloc(2 * npts, s);
        { k_gather_points<<<nblk(npts), 256, 0, s>>>(d_rows.p, d_xr.p, d_xi.p, d_xinf.p, npts, P.welded.p, d_pr.p,
                                                   d_pi.p, d_pinf.p); ::pgcp::note_launch(); }
        PGCP_CUDA(cudaGetLastError());
        const int32_t big = 1 << 30;
        PGCP_CUDA(cudaMemcpyAsync(fail_job.p, &big, sizeof(int32_t), cudaMemcpyHostToDevice, s));
        DBuf<int32_t> job_fail;
        job_fail.alloc(jobs.size(), s);
        job_fail.zero();
        Phase1Args a{d_pr.p, d_pi.p, d_pinf.p, npts, d_item_seq.p, d_seqs.p, (int32_t)seqs.size(), d_jobs.p, kmax,
                     recs.p, arcA.p, arcB.p, ctx->err.p, fail_job.p, job_fail.p};
        // few points per block: the FP64 work of a step is spread over many SMs;
        // at most P1_MAXSEQ sequences may meet in one block
        size_t smem = 0;
        int grid = coop_grid_pts(ctx, (const void*)k_weld_phase1, npts, &smem);
        check_block_sequences(item_seq, grid);
        void* args[] = {(void*)&a};
        { PGCP_CUDA(cudaLaunchCooperativeKernel((void*)k_weld_phase1, dim3(grid), dim3(P1_THREADS), args, smem, s)); ::pgcp::note_launch(); }
        PGCP_CUDA(cudaGetLastError());
        uint32_t e = read_errors(ctx);
        if (e & DE_WELD_DOMAIN) {
            std::vector<int32_t> jf(jobs.size());
            PGCP_CUDA(cudaMemcpy(jf.data(), job_fail.p, jf.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
            for (size_t jj = 0; jj < jf.size(); ++jj)
                if (jf[jj])
                    mesh_failed(P.welds[jobs_w[jj]].mesh,
                                "welding step out of its domain (weld " + std::to_string(jobs_w[jj]) +
                                    "): a zipper point left the right half-plane or the arc lost its order");
            ctx->err.zero();
        }
        // ---- phase 2 (boundary loops of the pieces involved)
        std::vector<int32_t> p2_rows, p2_arc, p2_chain;
        for (int wi : jobs_w) {
            const WeldPlan& W = P.welds[wi];
            if (mfail[W.mesh]) continue;
            const JobMeta& J = all_jobs[wi];
            for (int l = 0; l <= W.k; ++l) gpos[W.a_glob[l]] = l;
            auto add_piece = [&](int32_t pc, int side) {
                for (int64_t t = P.loff[pc]; t < P.loff[pc + 1]; ++t) {
                    p2_rows.push_back((int32_t)P.loop_rows[t]);
                    const int64_t l = gpos[P.loop_glob[t]];
                    p2_arc.push_back(l < 0 ? -1 : (int32_t)(J.arc_off + l));
                    p2_chain.push_back(2 * wi + side);
                }
            };
            for (int32_t pc : W.members) add_piece(pc, 0);
            for (int32_t pc : W.b_members) add_piece(pc, 1);
            for (int l = 0; l <= W.k; ++l) gpos[W.a_glob[l]] = -1;
        }
        DBuf<int32_t> d2_rows, d2_arc, d2_chain;
        upload(d2_rows, p2_rows, s);
        upload(d2_arc, p2_arc, s);
        upload(d2_chain, p2_chain, s);
        // both sides of every weld of the round in one launch (32-thread
        // blocks: few points per round, spread over every SM)
        const int64_t n2 = (int64_t)p2_rows.size();
        if (n2 > 0) {
            { k_phase2_boundary<<<nblk(n2, 32), 32, 0, s>>>(d2_rows.p, d2_arc.p, d2_chain.p, n2, d_chains.p, recs.p,
                                                          arcA.p, arcB.p, P.welded.p, ctx->err.p); ::pgcp::note_launch(); }
            PGCP_CUDA(cudaGetLastError());
        }
        PGCP_CUDA(cudaStreamSynchronize(s));
    }
    check_finite("a welded boundary point is not finite");
    // ---- disk constraint
    if (o.variant == PGCP_DISK) {
        std::vector<DiskMeta> seqs;
        std::vector<int32_t> item_seq, rows;
        std::vector<double> xr, xi;
        std::vector<int32_t> xinf;
        int nmax = 0;
        for (int mi = 0; mi < nmesh; ++mi) {
            const MeshInfo& M = P.meshes[mi];
            const auto& loop = disk_loop[mi];
            // rows: copy in the lowest-label piece of the mesh holding the vertex
            for (int32_t pc = M.piece0; pc < M.piece0 + M.npiece; ++pc)
                for (int64_t t = P.loff[pc]; t < P.loff[pc + 1]; ++t)
                    if (gpos[P.loop_glob[t]] < 0) gpos[P.loop_glob[t]] = P.loop_rows[t];
            DiskMeta m{(int64_t)item_seq.size(), (int32_t)loop.size() - 1, 0, disk_rec[mi]};
            nmax = std::max(nmax, m.n);
            const int sid = (int)seqs.size();
            seqs.push_back(m);
            for (int32_t g : loop) {
                if (gpos[g] < 0) fail(PGCP_E_ARG, "disk loop vertex on no piece loop of its mesh");
                item_seq.push_back(sid);
                rows.push_back((int32_t)gpos[g]);
                xr.push_back(0); xi.push_back(0); xinf.push_back(0);
            }
            for (int32_t pc = M.piece0; pc < M.piece0 + M.npiece; ++pc)
                for (int64_t t = P.loff[pc]; t < P.loff[pc + 1]; ++t) gpos[P.loop_glob[t]] = -1;
            double cref = by_mesh[mi].empty() ? 0.0 : -1.0;
            item_seq.push_back(sid); rows.push_back(-1); xr.push_back(cref); xi.push_back(0); xinf.push_back(0);
        }
        const int64_t npts = (int64_t)item_seq.size();
        DBuf<int32_t> d_item_seq, d_rows, d_xinf, d_pinf;
        DBuf<double> d_xr, d_xi, d_pr, d_pi;
        DBuf<DiskMeta> d_seqs;
        upload(d_item_seq, item_seq, s);
        upload(d_rows, rows, s);
        upload(d_xr, xr, s);
        upload(d_xi, xi, s);
        upload(d_xinf, xinf, s);
        upload(d_seqs, seqs, s);
        d_pr.alloc(2 * npts, s);   // two buffers (step parity)
        d_pi.alloc(2 * npts, s);
        d_pinf.alloc(2 * npts, s);
        { k_gather_points<<<nblk(npts), 256, 0, s>>>(d_rows.p, d_xr.p, d_xi.p, d_xinf.p, npts, P.welded.p, d_pr.p,
                                                   d_pi.p, d_pinf.p); ::pgcp::note_launch(); }
        DBuf<int32_t> seq_fail;
        seq_fail.alloc(seqs.size(), s);
        seq_fail.zero();
        DiskArgs a{d_pr.p, d_pi.p, d_pinf.p, npts, d_item_seq.p, d_seqs.p, (int32_t)seqs.size(), nmax, recs.p,
                   ctx->err.p, seq_fail.p};
        size_t smem = 0;
        int grid = coop_grid_pts(ctx, (const void*)k_disk_phase1, npts, &smem);
        check_block_sequences(item_seq, grid);
        void* args[] = {(void*)&a};
        { PGCP_CUDA(cudaLaunchCooperativeKernel((void*)k_disk_phase1, dim3(grid), dim3(P1_THREADS), args, smem, s)); ::pgcp::note_launch(); }
        PGCP_CUDA(cudaGetLastError());
        if (read_errors(ctx) & DE_WELD_DOMAIN) {
            std::vector<int32_t> sf(seqs.size());
            PGCP_CUDA(cudaMemcpy(sf.data(), seq_fail.p, sf.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
            for (int mi = 0; mi < nmesh; ++mi)
                if (sf[mi]) mesh_failed(mi, "disk map: a zipper point left the right half-plane");
            ctx->err.zero();
        }
        // images of the global boundary (sequence points 0..n) -> every copy
        std::vector<int32_t> p2_rows, p2_arc, p2_chain;
        std::vector<double2> dummy;
        for (int mi = 0; mi < nmesh; ++mi) {
            if (mfail[mi]) continue;
            const MeshInfo& M = P.meshes[mi];
            for (size_t l = 0; l < disk_loop[mi].size(); ++l) gpos[disk_loop[mi][l]] = (int64_t)l;
            for (int32_t pc = M.piece0; pc < M.piece0 + M.npiece; ++pc)
                for (int64_t t = P.loff[pc]; t < P.loff[pc + 1]; ++t) {
                    p2_rows.push_back((int32_t)P.loop_rows[t]);
                    const int64_t l = gpos[P.loop_glob[t]];
                    p2_arc.push_back(l < 0 ? -1 : (int32_t)(seqs[mi].off + l));
                    p2_chain.push_back(disk_chain[mi]);
                }
            for (int32_t g : disk_loop[mi]) gpos[g] = -1;
        }
        // sequence images as double2
        DBuf<double2> img;
        img.alloc(npts, s);
        {
            std::vector<double> hr(npts), hi(npts);
            PGCP_CUDA(cudaMemcpyAsync(hr.data(), d_pr.p, npts * sizeof(double), cudaMemcpyDeviceToHost, s));
            PGCP_CUDA(cudaMemcpyAsync(hi.data(), d_pi.p, npts * sizeof(double), cudaMemcpyDeviceToHost, s));
            PGCP_CUDA(cudaStreamSynchronize(s));
            std::vector<double2> h2(npts);
            for (int64_t t = 0; t < npts; ++t) h2[t] = make_double2(hr[t], hi[t]);
            PGCP_CUDA(cudaMemcpyAsync(img.p, h2.data(), npts * sizeof(double2), cudaMemcpyHostToDevice, s));
            DBuf<int32_t> d2_rows, d2_arc, d2_chain;
            upload(d2_rows, p2_rows, s);
            upload(d2_arc, p2_arc, s);
            upload(d2_chain, p2_chain, s);
            if (!p2_rows.empty())
                { k_phase2_boundary<<<nblk(p2_rows.size(), 32), 32, 0, s>>>(
                    d2_rows.p, d2_arc.p, d2_chain.p, (int64_t)p2_rows.size(), d_chains.p, recs.p, img.p, nullptr,
                    P.welded.p, ctx->err.p); ::pgcp::note_launch(); }
            PGCP_CUDA(cudaGetLastError());
            PGCP_CUDA(cudaStreamSynchronize(s));
        }
        check_finite("a disk-mapped boundary point is not finite");
    }
    // ---- interior weld map: every chain of each piece, in order (the warm
    // start of the final solve, and the learned start's input; a cold start
    // uses neither, so the interiors then keep their local coordinates)
    if (o.warm_start != PGCP_WARM_COLD) {
        std::vector<std::vector<int32_t>> pch(P.K);
        for (size_t w = 0; w < P.welds.size(); ++w) {
            const WeldPlan& W = P.welds[w];
            if (mfail[W.mesh]) continue;
            for (int32_t pc : W.members) pch[pc].push_back(2 * (int32_t)w);
            for (int32_t pc : W.b_members) pch[pc].push_back(2 * (int32_t)w + 1);
        }
        for (int mi = 0; mi < nmesh; ++mi)
            if (disk_chain[mi] >= 0 && !mfail[mi])
                for (int32_t pc = P.meshes[mi].piece0; pc < P.meshes[mi].piece0 + P.meshes[mi].npiece; ++pc)
                    pch[pc].push_back(disk_chain[mi]);
        std::vector<int64_t> off(P.K + 1, 0);
        std::vector<int32_t> flat;
        for (int32_t pc = 0; pc < P.K; ++pc) {
            flat.insert(flat.end(), pch[pc].begin(), pch[pc].end());
            off[pc + 1] = (int64_t)flat.size();
        }
        DBuf<int64_t> d_off;
        DBuf<int32_t> d_flat;
        upload(d_off, off, s);
        upload(d_flat, flat, s);
        if (!flat.empty()) {
            if (o.interior_map_fp64) {
                { k_interior_map64<<<nblk(P.Nc, 128), 128, 0, s>>>(P.Nc, P.is_bnd.p, P.row_piece.p, d_off.p, d_flat.p,
                                                                 d_chains.p, recs.p, P.welded.p); ::pgcp::note_launch(); }
            } else {
                DBuf<RecF> rf;
                rf.alloc(std::max<int64_t>(nrec, 1), s);
                { k_recs_to_f32<<<nblk(nrec), 256, 0, s>>>(recs.p, rf.p, nrec); ::pgcp::note_launch(); }
                { k_interior_map<<<nblk(P.Nc, 128), 128, 0, s>>>(P.Nc, P.is_bnd.p, P.row_piece.p, d_off.p, d_flat.p,
                                                               d_chains.p, rf.p, P.welded.p); ::pgcp::note_launch(); }
            }
            PGCP_CUDA(cudaGetLastError());
        }
        PGCP_CUDA(cudaStreamSynchronize(s));
    }
    // sphere: the pieces of each closed weld's B side are held in the chart w = 1/z
    P.wchart.assign(P.K, 0);
    for (const WeldPlan& W : P.welds)
        if (W.closed)
            for (int32_t pc : W.b_members) P.wchart[pc] = 1;
    upload(P.d_wchart, P.wchart, s);
    PGCP_CUDA(cudaStreamSynchronize(s));
    // dropped meshes: their pieces keep the local maps (finite), so the final
    // solve runs through; their output is set to NaN after the gather
    P.mesh_status.assign(nmesh, PGCP_OK);
    int nfailed = 0;
    for (int mi = 0; mi < nmesh; ++mi) {
        if (!mfail[mi]) continue;
        ++nfailed;
        P.mesh_status[mi] = PGCP_E_NUMERIC;
        const MeshInfo& M = P.meshes[mi];
        const int64_t r0 = P.voff[M.piece0], r1 = P.voff[M.piece0 + M.npiece];
        PGCP_CUDA(cudaMemcpyAsync(P.welded.p + r0, P.local.p + r0, (r1 - r0) * sizeof(double2),
                                  cudaMemcpyDeviceToDevice, s));
    }
    if (nfailed) {   // the gather skips the pieces of dropped meshes (flag 2)
        for (int mi = 0; mi < nmesh; ++mi)
            if (mfail[mi])
                for (int32_t pc = P.meshes[mi].piece0; pc < P.meshes[mi].piece0 + P.meshes[mi].npiece; ++pc)
                    P.wchart[pc] = 2;
        upload(P.d_wchart, P.wchart, s);
    }
    PGCP_CUDA(cudaStreamSynchronize(s));
    if (nfailed == nmesh) fail(PGCP_E_NUMERIC, "every mesh of the batch left the welding domain");
    P.have_weld = 1;
}

}  // namespace pgcp
