// Angle distortion and fold statistics of a result (Section 5, Section 3.5).
//
// d = angle(phi(v_i), phi(v_j), phi(v_k)) - angle(v_i, v_j, v_k) in degrees for
// every triangle corner, angles as atan2(|e1 x e2|, e1 . e2) in FP64.  Over |d|:
// mean, population sd, median and inter-quartile range (linear interpolation
// between order statistics), max.  Order statistics come from a radix sort of
// the non-negative doubles' bit patterns (order-preserving).  Flips: planar
// signed area <= 0, or a chordal triangle facing inwards on the sphere.  |mu|:
// Beltrami coefficient of the affine map from the flattened surface triangle.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pgcp_internal.h"

namespace pgcp {

namespace {

__device__ double corner_angle(const double* p, const double* q, const double* r) {
    double e1x = q[0] - p[0], e1y = q[1] - p[1], e1z = q[2] - p[2];
    double e2x = r[0] - p[0], e2y = r[1] - p[1], e2z = r[2] - p[2];
    double cx = e1y * e2z - e1z * e2y, cy = e1z * e2x - e1x * e2z, cz = e1x * e2y - e1y * e2x;
    return atan2(sqrt(cx * cx + cy * cy + cz * cz), e1x * e2x + e1y * e2y + e1z * e2z);
}

__global__ void k_face_metrics(const int32_t* __restrict__ F, int64_t nf, const double* __restrict__ V,
                               const double* __restrict__ U, int dim, uint64_t* __restrict__ keys,
                               int32_t* __restrict__ vals, double* __restrict__ acc,
                               unsigned long long* __restrict__ flips, unsigned long long* __restrict__ maxmu) {
    __shared__ double sh[3 * 32];
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double s1 = 0, s2 = 0, mx = 0;
    if (f < nf) {
        double X[3][3], Y[3][3];
        for (int c = 0; c < 3; ++c) {
            int v = F[3 * f + c];
            for (int t = 0; t < 3; ++t) X[c][t] = V[3 * (int64_t)v + t];
            for (int t = 0; t < 3; ++t) Y[c][t] = t < dim ? U[(int64_t)dim * v + t] : 0.0;
        }
        for (int c = 0; c < 3; ++c) {
            double a0 = corner_angle(X[c], X[(c + 1) % 3], X[(c + 2) % 3]);
            double a1 = corner_angle(Y[c], Y[(c + 1) % 3], Y[(c + 2) % 3]);
            double d = fabs((a1 - a0) * (180.0 / 3.14159265358979323846));
            uint64_t bits;
            memcpy(&bits, &d, sizeof(d));
            keys[3 * f + c] = bits;
            vals[3 * f + c] = 0;
            s1 += d;
            s2 += d * d;
            mx = fmax(mx, d);
        }
        bool flip;
        if (dim == 2) {
            double sa = (Y[1][0] - Y[0][0]) * (Y[2][1] - Y[0][1]) - (Y[1][1] - Y[0][1]) * (Y[2][0] - Y[0][0]);
            flip = !(sa > 0.0);
            // |mu| of the affine map from the flattened surface triangle
            double e1[3], e2[3];
            for (int t = 0; t < 3; ++t) {
                e1[t] = X[1][t] - X[0][t];
                e2[t] = X[2][t] - X[0][t];
            }
            double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
            double x2 = (e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2]) / l1;
            double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                   cz = e1[0] * e2[1] - e1[1] * e2[0];
            double y2 = sqrt(cx * cx + cy * cy + cz * cz) / l1;
            double w1r = Y[1][0] - Y[0][0], w1i = Y[1][1] - Y[0][1];
            double w2r = Y[2][0] - Y[0][0], w2i = Y[2][1] - Y[0][1];
            double fxr = w1r / l1, fxi = w1i / l1;
            double fyr = (w2r - w1r * x2 / l1) / y2, fyi = (w2i - w1i * x2 / l1) / y2;
            // f_z = (f_x - i f_y)/2, f_zbar = (f_x + i f_y)/2
            double fzr = 0.5 * (fxr + fyi), fzi = 0.5 * (fxi - fyr);
            double fbr = 0.5 * (fxr - fyi), fbi = 0.5 * (fxi + fyr);
            double mu = sqrt(fbr * fbr + fbi * fbi) / sqrt(fzr * fzr + fzi * fzi);
            if (mu == mu) atomicMax(maxmu, (unsigned long long)__double_as_longlong(mu));
        } else {
            double ax = Y[1][0] - Y[0][0], ay = Y[1][1] - Y[0][1], az = Y[1][2] - Y[0][2];
            double bx = Y[2][0] - Y[0][0], by = Y[2][1] - Y[0][1], bz = Y[2][2] - Y[0][2];
            double nx = ay * bz - az * by, ny = az * bx - ax * bz, nz = ax * by - ay * bx;
            double vol = nx * (Y[0][0] + Y[1][0] + Y[2][0]) + ny * (Y[0][1] + Y[1][1] + Y[2][1]) +
                         nz * (Y[0][2] + Y[1][2] + Y[2][2]);
            flip = !(vol > 0.0);
        }
        if (flip) atomicAdd(flips, 1ull);
    }
    // block sums
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sh[3 * w] = s1;
        sh[3 * w + 1] = s2;
        sh[3 * w + 2] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, m = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            a += sh[3 * i];
            b += sh[3 * i + 1];
            m = fmax(m, sh[3 * i + 2]);
        }
        atomicAdd(&acc[0], a);
        atomicAdd(&acc[1], b);
        atomicMax((unsigned long long*)&acc[2], (unsigned long long)__double_as_longlong(m));
    }
}

double bits_to_double(uint64_t b) {
    double d;
    memcpy(&d, &b, sizeof(d));
    return d;
}

}  // namespace

void compute_metrics(pgcp_ctx* ctx, const Part& P, const double* U, pgcp_distortion* met) {
    cudaStream_t s = ctx->stream;
    const int64_t nf = P.nf, nc = 3 * nf;
    const int dim = P.closed ? 3 : 2;
    DBuf<uint64_t> keys;
    DBuf<int32_t> vals;
    DBuf<double> acc;
    DBuf<unsigned long long> cnt;
    keys.alloc(nc, s);
    vals.alloc(nc, s);
    acc.alloc(3, s);
    cnt.alloc(2, s);
    acc.zero();
    cnt.zero();
    { k_face_metrics<<<(unsigned)std::max<int64_t>(1, ceil_div(nf, 256)), 256, 0, s>>>(
        P.F.p, nf, P.V.p, U, dim, keys.p, vals.p, acc.p, cnt.p, cnt.p + 1); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    radix_sort_pairs(keys.p, vals.p, nc, 64, s);
    double h_acc[3];
    unsigned long long h_cnt[2];
    PGCP_CUDA(cudaMemcpyAsync(h_acc, acc.p, sizeof(h_acc), cudaMemcpyDeviceToHost, s));
    PGCP_CUDA(cudaMemcpyAsync(h_cnt, cnt.p, sizeof(h_cnt), cudaMemcpyDeviceToHost, s));
    auto order_stat = [&](int64_t i) {
        uint64_t b = 0;
        PGCP_CUDA(cudaMemcpyAsync(&b, keys.p + i, sizeof(b), cudaMemcpyDeviceToHost, s));
        PGCP_CUDA(cudaStreamSynchronize(s));
        return bits_to_double(b);
    };
    auto percentile = [&](double q) {
        double pos = q / 100.0 * (double)(nc - 1);
        int64_t lo = (int64_t)std::floor(pos);
        double frac = pos - (double)lo;
        double a = order_stat(lo);
        if (lo + 1 >= nc) return a;
        double b = order_stat(lo + 1);
        return a + frac * (b - a);
    };
    PGCP_CUDA(cudaStreamSynchronize(s));
    met->n_corners = nc;
    met->mean = h_acc[0] / (double)nc;
    double var = h_acc[1] / (double)nc - met->mean * met->mean;
    met->sd = std::sqrt(std::max(var, 0.0));
    met->max = bits_to_double((uint64_t)*(unsigned long long*)&h_acc[2]);
    met->median = percentile(50.0);
    met->iqr = percentile(75.0) - percentile(25.0);
    met->flips = (int64_t)h_cnt[0];
    met->max_mu = dim == 2 ? bits_to_double(h_cnt[1]) : 0.0;
}

}  // namespace pgcp
