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
#include <mutex>
#include <string>
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

// ------------------------------------------------ allocation-free variant
//
// The same statistics as compute_metrics, with every device buffer carved out
// of one fixed file-scope array instead of the stream-ordered pool.  For
// callers that must not allocate device memory (their device memory is held
// by another allocator, or an allocation may fail or synchronise at a point
// where they cannot afford it).  Bound: METRICS_NF_MAX faces.

namespace {

constexpr int64_t METRICS_NF_MAX = int64_t(1) << 18;
constexpr int64_t NC_MAX = 3 * METRICS_NF_MAX;
constexpr int64_t RS_TILE_NA = 2048;                                   // radix sort tile (keys per block)
constexpr int64_t COUNTS_MAX = 256 * ((NC_MAX + RS_TILE_NA - 1) / RS_TILE_NA);
constexpr int64_t SCAN_WS = 256;

// byte offsets inside the scratch array; every region starts on 256 bytes
constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t OFF_KEYS = 0;
constexpr size_t OFF_K2 = OFF_KEYS + al256(NC_MAX * sizeof(uint64_t));
constexpr size_t OFF_VALS = OFF_K2 + al256(NC_MAX * sizeof(uint64_t));
constexpr size_t OFF_V2 = OFF_VALS + al256(NC_MAX * sizeof(int32_t));
constexpr size_t OFF_COUNTS = OFF_V2 + al256(NC_MAX * sizeof(int32_t));
constexpr size_t OFF_OFFS = OFF_COUNTS + al256(COUNTS_MAX * sizeof(int64_t));
constexpr size_t OFF_SCAN = OFF_OFFS + al256(COUNTS_MAX * sizeof(int64_t));
constexpr size_t OFF_ACC = OFF_SCAN + al256(SCAN_WS * sizeof(int64_t));    // acc[3] then cnt[2]: zeroed per call
constexpr size_t OFF_OUT = OFF_ACC + 256;                                  // 11 words gathered for the host
constexpr size_t SCRATCH_BYTES = OFF_OUT + 256;

static __device__ __align__(256) unsigned char g_metrics_scratch[SCRATCH_BYTES];

// out[0..2] = acc, out[3..4] = cnt, out[5..10] = keys at the six order-statistic positions
__global__ void k_metrics_collect(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ acc_cnt,
                                  const int64_t* pos, uint64_t* __restrict__ out) {
    int t = threadIdx.x;
    if (t < 5) out[t] = acc_cnt[t];
    else if (t < 11) out[t] = keys[pos[t - 5]];
}

__global__ void k_metrics_positions(int64_t* pos, int64_t p0, int64_t p1, int64_t p2, int64_t p3, int64_t p4,
                                    int64_t p5) {
    if (threadIdx.x == 0) {
        pos[0] = p0; pos[1] = p1; pos[2] = p2; pos[3] = p3; pos[4] = p4; pos[5] = p5;
    }
}

std::mutex g_scratch_mu;
unsigned char* g_scratch_ptr[64] = {};

unsigned char* scratch_for_current_device() {
    int dev = -1;
    PGCP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(PGCP_E_ARG, "device ordinal out of range for the metrics scratch table");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_metrics_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            fail(PGCP_E_CUDA, std::string("cudaGetSymbolAddress(metrics scratch): ") + cudaGetErrorString(e));
        }
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    return g_scratch_ptr[dev];
}

}  // namespace

int64_t metrics_noalloc_max_faces() { return METRICS_NF_MAX; }

void compute_metrics_noalloc(pgcp_ctx* ctx, const Part& P, const double* U, pgcp_distortion* met) {
    cudaStream_t s = ctx->stream;
    const int64_t nf = P.nf, nc = 3 * nf;
    const int dim = P.closed ? 3 : 2;
    if (nf <= 0) fail(PGCP_E_ARG, "metrics of a mesh without faces");
    if (nf > METRICS_NF_MAX)
        fail(PGCP_E_ARG, "allocation-free metrics: " + std::to_string(nf) + " faces exceeds the fixed limit of " +
                             std::to_string(METRICS_NF_MAX) + " (use pgcp_metrics)");
    int dev = -1;
    PGCP_CUDA(cudaGetDevice(&dev));
    if (dev != ctx->device) fail(PGCP_E_ARG, "allocation-free metrics: the context's device is not current");
    unsigned char* base = scratch_for_current_device();
    uint64_t* keys = reinterpret_cast<uint64_t*>(base + OFF_KEYS);
    uint64_t* k2 = reinterpret_cast<uint64_t*>(base + OFF_K2);
    int32_t* vals = reinterpret_cast<int32_t*>(base + OFF_VALS);
    int32_t* v2 = reinterpret_cast<int32_t*>(base + OFF_V2);
    int64_t* counts = reinterpret_cast<int64_t*>(base + OFF_COUNTS);
    int64_t* offs = reinterpret_cast<int64_t*>(base + OFF_OFFS);
    int64_t* scan_ws = reinterpret_cast<int64_t*>(base + OFF_SCAN);
    double* acc = reinterpret_cast<double*>(base + OFF_ACC);
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(base + OFF_ACC + 3 * sizeof(double));
    int64_t* pos = reinterpret_cast<int64_t*>(base + OFF_OUT + 11 * sizeof(uint64_t));
    uint64_t* out = reinterpret_cast<uint64_t*>(base + OFF_OUT);
    if (sort_ws_counts(nc) > COUNTS_MAX) fail(PGCP_E_ARG, "metrics scratch: radix sort tile size mismatch");

    // the only state that must start at zero: the sums, max and counters
    PGCP_CUDA(cudaMemsetAsync(acc, 0, 3 * sizeof(double) + 2 * sizeof(unsigned long long), s));
    { k_face_metrics<<<(unsigned)ceil_div(nf, 256), 256, 0, s>>>(P.F.p, nf, P.V.p, U, dim, keys, vals, acc, cnt,
                                                                 cnt + 1); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    radix_sort_pairs_noalloc(keys, vals, nc, 64, s, k2, v2, counts, offs, scan_ws, SCAN_WS);

    // percentile positions, linear interpolation between order statistics
    int64_t lo[3];
    double frac[3];
    const double q[3] = {25.0, 50.0, 75.0};
    for (int i = 0; i < 3; ++i) {
        double p = q[i] / 100.0 * (double)(nc - 1);
        lo[i] = (int64_t)std::floor(p);
        frac[i] = p - (double)lo[i];
    }
    auto hi = [&](int i) { return std::min(lo[i] + 1, nc - 1); };
    { k_metrics_positions<<<1, 32, 0, s>>>(pos, lo[0], hi(0), lo[1], hi(1), lo[2], hi(2)); ::pgcp::note_launch(); }
    { k_metrics_collect<<<1, 32, 0, s>>>(keys, reinterpret_cast<const uint64_t*>(acc), pos, out);
      ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    uint64_t h[11];
    PGCP_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
    PGCP_CUDA(cudaStreamSynchronize(s));
    auto pct = [&](int i) {
        double a = bits_to_double(h[5 + 2 * i]);
        if (lo[i] + 1 >= nc) return a;
        double b = bits_to_double(h[6 + 2 * i]);
        return a + frac[i] * (b - a);
    };
    const double s1 = bits_to_double(h[0]), s2 = bits_to_double(h[1]);
    met->n_corners = nc;
    met->mean = s1 / (double)nc;
    double var = s2 / (double)nc - met->mean * met->mean;
    met->sd = std::sqrt(std::max(var, 0.0));
    met->max = bits_to_double(h[2]);
    met->median = pct(1);
    met->iqr = pct(2) - pct(0);
    met->flips = (int64_t)h[3];
    met->max_mu = dim == 2 ? bits_to_double(h[4]) : 0.0;
}

}  // namespace pgcp
