// Learned warm start for the final Laplace solve (not in the paper; the plain
// method of Section 4.5 verifies every prediction and falls back per piece).
//
// A message-passing network over each piece's mesh graph, width 64:
//   features  F_i = [z_i / sigma, boundary flag, 1, 0 ...] (16 wide, bf16),
//             z_i = -(1/d_i) (L u_w)_i on interior rows (FP64), 0 on boundary
//             rows; sigma = RMS of |z| over the piece's interior rows
//   X_0     = relu(F W_in + b_in)                     tensor cores, K = 16
//   X_{l+1} = relu([X_l | P X_l] W_l + b_l), l < 4     aggregation P = D^-1 W
//                                                     (warp per row), then
//                                                     tensor cores, K = 128
//   out     = X_4 W_out + b_out (16 wide, columns 0, 1 used)
//   u_0     = u_w + sigma out[:, 0:2]
// Activations are bf16 [rows x 128] buffers A_l = [X_l | P X_l]; the dense
// layers run on the tcgen05 GEMM (FP32 accumulation in tensor memory).
// Training (same graph, target t = (u* - u_w) / sigma, mean squared error over
// interior rows): the backward GEMMs dA = dZ W^T also run on the tensor
// cores; weight gradients A^T dZ are FP32 reductions over rows; Adam updates
// the FP32 master weights and refreshes their bf16 copies.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <vector>

#include "pgcp_internal.h"

namespace pgcp {

namespace {

constexpr int WID = 64, FIN = 16, FOUT = 16, NL = 4;
constexpr int64_t OFF_WIN = 0, OFF_BIN = FIN * WID;
constexpr int64_t LAYER0 = OFF_BIN + WID;
constexpr int64_t LAYER_SZ = 2 * WID * WID + WID;
constexpr int64_t OFF_WOUT = LAYER0 + NL * LAYER_SZ;
constexpr int64_t OFF_BOUT = OFF_WOUT + WID * FOUT;
constexpr int64_t NPARAM = OFF_BOUT + FOUT;   // 35152
__host__ __device__ constexpr int64_t off_w(int l) { return LAYER0 + l * LAYER_SZ; }
__host__ __device__ constexpr int64_t off_b(int l) { return off_w(l) + 2 * WID * WID; }

// bf16 weight copies: forward Bt = W^T ([out x in]), backward Bt = W ([in x out])
constexpr int64_t BF_WIN_T = 0;                        // [64 x 16]
constexpr int64_t BF_L_T = BF_WIN_T + WID * FIN;       // 4 x [64 x 128]
constexpr int64_t BF_WOUT_T = BF_L_T + NL * WID * 2 * WID;   // [16 x 64]
constexpr int64_t BF_L = BF_WOUT_T + FOUT * WID;       // 4 x [128 x 64]
constexpr int64_t BF_WOUT = BF_L + NL * 2 * WID * WID; // [64 x 16]
constexpr int64_t BF_TOTAL = BF_WOUT + WID * FOUT;

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, ceil_div(n, t)); }

// ---------------------------------------------------------------- weights

__global__ void k_pack(const float* __restrict__ th, __nv_bfloat16* __restrict__ bf) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // forward copies (transposed)
    if (t < WID * FIN) {   // W_in^T [n][k] = W_in[k][n]
        const int n = (int)(t / FIN), k = (int)(t % FIN);
        bf[BF_WIN_T + t] = __float2bfloat16_rn(th[OFF_WIN + k * WID + n]);
    }
    if (t < NL * WID * 2 * WID) {
        const int l = (int)(t / (WID * 2 * WID)), r = (int)(t % (WID * 2 * WID));
        const int n = r / (2 * WID), k = r % (2 * WID);   // W_l^T [n][k] = W_l[k][n]
        bf[BF_L_T + t] = __float2bfloat16_rn(th[off_w(l) + (int64_t)k * WID + n]);
        bf[BF_L + t] = __float2bfloat16_rn(th[off_w(l) + r]);   // W_l as stored [k][n]
    }
    if (t < FOUT * WID) {   // W_out^T [n][k] = W_out[k][n]; W_out as stored [k][n]
        const int n = (int)(t / WID), k = (int)(t % WID);
        bf[BF_WOUT_T + t] = __float2bfloat16_rn(th[OFF_WOUT + (int64_t)k * FOUT + n]);
        bf[BF_WOUT + t] = __float2bfloat16_rn(th[OFF_WOUT + t]);
    }
}

__global__ void k_adam(int64_t n, float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---------------------------------------------------------------- features

// random-walk weights of the aggregation and of its transpose, per CSR entry
__global__ void k_mp_weights(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ diag, float* __restrict__ pw,
                             float* __restrict__ ptw) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double di = diag[i];
    for (int j = rp[i]; j < rp[i + 1]; ++j) {
        const int c = col[j];
        pw[j] = c == i ? 0.f : (float)(-val[j] / di);
        ptw[j] = c == i ? 0.f : (float)(-val[j] / diag[c]);
    }
}

// z = -(1/d) L u on interior rows (FP64), per-piece sums of |z|^2 and counts.
// rowv (deterministic mode): |z_i|^2 per row instead of the atomic sums zz.
__global__ void k_mp_z(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                       const double* __restrict__ val, const double* __restrict__ diag,
                       const uint8_t* __restrict__ is_bnd, const int32_t* __restrict__ row_piece,
                       const double2* __restrict__ u, float2* __restrict__ z, double* __restrict__ zz,
                       unsigned long long* __restrict__ cnt, double* __restrict__ rowv) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double s2 = 0.0;
    int inner = 0, piece = -1;
    if (i < n) {
        piece = row_piece[i];
        double2 zi = make_double2(0.0, 0.0);
        if (!is_bnd[i]) {
            double ax = 0.0, ay = 0.0;
            for (int j = rp[i]; j < rp[i + 1]; ++j) {
                const double2 uc = u[col[j]];
                ax += val[j] * uc.x;
                ay += val[j] * uc.y;
            }
            const double d = diag[i];
            zi = make_double2(-ax / d, -ay / d);
            s2 = zi.x * zi.x + zi.y * zi.y;
            inner = 1;
        }
        z[i] = make_float2((float)zi.x, (float)zi.y);
        if (rowv) rowv[i] = s2;
    }
    if (rowv) s2 = 0.0;
    // warp sums when the warp lies in one piece, else per lane
    const int lane = threadIdx.x & 31;
    const int p0 = __shfl_sync(0xffffffffu, piece, 0);
    const bool uniform = __all_sync(0xffffffffu, piece == p0 || piece < 0);
    if (uniform) {
        for (int o = 16; o > 0; o >>= 1) {
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            inner += __shfl_xor_sync(0xffffffffu, inner, o);
        }
        if (lane == 0 && p0 >= 0 && inner > 0) {
            if (!rowv) atomicAdd(&zz[p0], s2);
            atomicAdd(&cnt[p0], (unsigned long long)inner);
        }
    } else if (piece >= 0 && inner) {
        if (!rowv) atomicAdd(&zz[piece], s2);
        atomicAdd(&cnt[piece], 1ull);
    }
}

// out[s] = sum of v over the rows [off[s], off[s+1]) of piece s in a fixed
// order (deterministic mode): thread t adds rows t, t + 256, ... in sequence,
// then a fixed halving tree.  One 256-thread block per piece.
__global__ void k_seg_sum(const double* __restrict__ v, const int64_t* __restrict__ off, double* __restrict__ out) {
    __shared__ double red[256];
    const int s = blockIdx.x;
    double a = 0.0;
    for (int64_t i = off[s] + threadIdx.x; i < off[s + 1]; i += 256) a += v[i];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[s] = red[0];
}

__global__ void k_mp_sigma(int K, const double* __restrict__ zz, const unsigned long long* __restrict__ cnt,
                           float* __restrict__ sigma) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= K) return;
    const double ms = cnt[s] ? zz[s] / (double)cnt[s] : 0.0;
    sigma[s] = ms > 0.0 ? (float)sqrt(ms) : 1.f;
}

__global__ void k_mp_feat(int64_t n, const float2* __restrict__ z, const float* __restrict__ sigma,
                          const int32_t* __restrict__ row_piece, const uint8_t* __restrict__ is_bnd,
                          __nv_bfloat16* __restrict__ F, float* __restrict__ Ff) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float s = sigma[row_piece[i]];
    float f[FIN];
#pragma unroll
    for (int c = 0; c < FIN; ++c) f[c] = 0.f;
    f[0] = z[i].x / s;
    f[1] = z[i].y / s;
    f[2] = is_bnd[i] ? 1.f : 0.f;
    f[3] = 1.f;
#pragma unroll
    for (int c = 0; c < FIN; ++c) {
        const __nv_bfloat16 b = __float2bfloat16_rn(f[c]);
        F[i * FIN + c] = b;
        if (Ff) Ff[i * FIN + c] = __bfloat162float(b);
    }
}

// ---------------------------------------------------------------- aggregation

// A[:, 64:128] = P A[:, 0:64]; one warp per row, two channels per lane
__global__ void k_mp_agg(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                         const float* __restrict__ pw, __nv_bfloat16* __restrict__ A) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    float2 acc = make_float2(0.f, 0.f);
    for (int j = rp[row]; j < rp[row + 1]; ++j) {
        const float w = pw[j];
        if (w == 0.f) continue;
        const float2 x = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(A + (int64_t)col[j] * 128)[lane]);
        acc.x = fmaf(w, x.x, acc.x);
        acc.y = fmaf(w, x.y, acc.y);
    }
    reinterpret_cast<__nv_bfloat162*>(A + row * 128 + 64)[lane] = __float22bfloat162_rn(acc);
}

// dX = dA[:, 0:64] + P^T dA[:, 64:128] (FP32); one warp per row
__global__ void k_mp_agg_t(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const float* __restrict__ ptw, const float* __restrict__ dA, float* __restrict__ dX) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    float2 acc = reinterpret_cast<const float2*>(dA + row * 128)[lane];
    for (int j = rp[row]; j < rp[row + 1]; ++j) {
        const float w = ptw[j];
        if (w == 0.f) continue;
        const float2 g = reinterpret_cast<const float2*>(dA + (int64_t)col[j] * 128 + 64)[lane];
        acc.x = fmaf(w, g.x, acc.x);
        acc.y = fmaf(w, g.y, acc.y);
    }
    reinterpret_cast<float2*>(dX + row * 64)[lane] = acc;
}

// dZ = dX * (X > 0), X = A[:, 0:64] (the layer's relu output)
__global__ void k_relu_bwd(int64_t n, const float* __restrict__ dX, const __nv_bfloat16* __restrict__ A,
                           int64_t lda, __nv_bfloat16* __restrict__ dZ) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 64) return;
    const int64_t r = t >> 6;
    const int c = (int)(t & 63);
    const float x = __bfloat162float(A[r * lda + c]);
    dZ[t] = __float2bfloat16_rn(x > 0.f ? dX[t] : 0.f);
}

// dW[K x N] += A^T G, db[N] += sum of G rows (FP32 accumulation, bf16 inputs)
template <int K, int N>
__global__ void __launch_bounds__(256) k_wgrad(const __nv_bfloat16* __restrict__ A, int64_t lda,
                                               const __nv_bfloat16* __restrict__ G, int64_t ldg, int64_t rows,
                                               float* __restrict__ dW, float* __restrict__ db) {
    constexpr int CH = 32;
    constexpr int NPT = K * N / 256;
    static_assert(NPT >= 1 && N % NPT == 0, "outputs per thread");
    __shared__ float sA[CH][K];
    __shared__ float sG[CH][N];
    const int o0 = threadIdx.x * NPT;
    const int k = o0 / N, n0 = o0 % N;
    float acc[NPT];
#pragma unroll
    for (int u = 0; u < NPT; ++u) acc[u] = 0.f;
    float bacc = 0.f;
    for (int64_t r0 = (int64_t)blockIdx.x * CH; r0 < rows; r0 += (int64_t)gridDim.x * CH) {
        __syncthreads();
        for (int t = threadIdx.x; t < CH * K; t += blockDim.x) {
            const int r = t / K, c = t % K;
            sA[r][c] = r0 + r < rows ? __bfloat162float(A[(r0 + r) * lda + c]) : 0.f;
        }
        for (int t = threadIdx.x; t < CH * N; t += blockDim.x) {
            const int r = t / N, c = t % N;
            sG[r][c] = r0 + r < rows ? __bfloat162float(G[(r0 + r) * ldg + c]) : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < CH; ++r) {
            const float a = sA[r][k];
#pragma unroll
            for (int u = 0; u < NPT; ++u) acc[u] = fmaf(a, sG[r][n0 + u], acc[u]);
        }
        if (threadIdx.x < N)
            for (int r = 0; r < CH; ++r) bacc += sG[r][threadIdx.x];
    }
#pragma unroll
    for (int u = 0; u < NPT; ++u) atomicAdd(&dW[k * N + n0 + u], acc[u]);
    if (threadIdx.x < N) atomicAdd(&db[threadIdx.x], bacc);
}

// ---------------------------------------------------------------- loss, apply, residual

__global__ void k_mp_target(int64_t n, const double2* __restrict__ uw, const double2* __restrict__ us,
                            const float* __restrict__ sigma, const int32_t* __restrict__ row_piece,
                            const uint8_t* __restrict__ is_bnd, float2* __restrict__ t) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (is_bnd[i]) {
        t[i] = make_float2(0.f, 0.f);
        return;
    }
    const double s = sigma[row_piece[i]];
    t[i] = make_float2((float)((us[i].x - uw[i].x) / s), (float)((us[i].y - uw[i].y) / s));
}

// loss sum and dOut = 2 (out - t) / n_inner on interior rows (bf16 [n x 16])
__global__ void k_mp_loss(int64_t n, const float* __restrict__ out, const float2* __restrict__ t,
                          const uint8_t* __restrict__ is_bnd, double inv_n, double* __restrict__ loss,
                          __nv_bfloat16* __restrict__ dOut) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < n) {
        float g0 = 0.f, g1 = 0.f;
        if (!is_bnd[i]) {
            const float r0 = out[i * FOUT] - t[i].x, r1 = out[i * FOUT + 1] - t[i].y;
            l = (double)r0 * r0 + (double)r1 * r1;
            g0 = (float)(2.0 * r0 * inv_n);
            g1 = (float)(2.0 * r1 * inv_n);
        }
        dOut[i * FOUT] = __float2bfloat16_rn(g0);
        dOut[i * FOUT + 1] = __float2bfloat16_rn(g1);
#pragma unroll
        for (int c = 2; c < FOUT; ++c) dOut[i * FOUT + c] = __float2bfloat16_rn(0.f);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l);
}

// u0 = u_w + sigma out[:, 0:2] on interior rows
__global__ void k_mp_apply(int64_t n, const double2* __restrict__ uw, const float* __restrict__ out,
                           const float* __restrict__ sigma, const int32_t* __restrict__ row_piece,
                           const uint8_t* __restrict__ is_bnd, double2* __restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 u = uw[i];
    if (!is_bnd[i]) {
        const double s = sigma[row_piece[i]];
        u.x += s * (double)out[i * FOUT];
        u.y += s * (double)out[i * FOUT + 1];
    }
    x[i] = u;
}

// per piece: sum over interior rows of |(L x)_i|^2 (FP64 Laplace residual);
// rowv (deterministic mode): the row terms instead of the atomic sums
__global__ void k_piece_residual(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, const uint8_t* __restrict__ is_bnd,
                                 const int32_t* __restrict__ row_piece, const double2* __restrict__ x,
                                 double* __restrict__ rr, double* __restrict__ rowv) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double s2 = 0.0;
    int piece = -1;
    if (i < n) {
        piece = row_piece[i];
        if (!is_bnd[i]) {
            double ax = 0.0, ay = 0.0;
            for (int j = rp[i]; j < rp[i + 1]; ++j) {
                const double2 xc = x[col[j]];
                ax += val[j] * xc.x;
                ay += val[j] * xc.y;
            }
            s2 = ax * ax + ay * ay;
            if (!(s2 == s2)) s2 = INFINITY;   // NaN counts as no better
        }
        if (rowv) rowv[i] = s2;
    }
    if (rowv) return;
    const int p0 = __shfl_sync(0xffffffffu, piece, 0);
    if (__all_sync(0xffffffffu, piece == p0 || piece < 0)) {
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if ((threadIdx.x & 31) == 0 && p0 >= 0 && s2 != 0.0) atomicAdd(&rr[p0], s2);
    } else if (piece >= 0 && s2 != 0.0) {
        atomicAdd(&rr[piece], s2);
    }
}

// x = learned start on the pieces where it is better, else keep x
__global__ void k_choose(int64_t n, const int32_t* __restrict__ row_piece, const uint8_t* __restrict__ use,
                         const double2* __restrict__ xl, double2* __restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (use[row_piece[i]]) x[i] = xl[i];
}

}  // namespace

// ---------------------------------------------------------------- host side

namespace {

// Device buffers of one forward (and backward) pass over a part.
struct MpWork {
    int64_t n = 0;
    DBuf<float> pw, ptw;          // aggregation weights per CSR entry
    DBuf<float2> z;
    DBuf<double> zz;
    DBuf<unsigned long long> cnt;
    DBuf<float> sigma;            // [K]
    DBuf<uint16_t> F;             // [n x 16] bf16
    DBuf<uint16_t> A[NL + 1];     // [n x 128] bf16: [X_l | P X_l]
    DBuf<float> out;              // [n x 16]
    int64_t n_inner = 0;
};

void mp_inputs(pgcp_ctx* ctx, Part& P, MpWork& W, float* Ff) {
    cudaStream_t s = ctx->stream;
    const int64_t n = P.Nc;
    W.n = n;
    W.pw.alloc(std::max<int64_t>(P.nnz, 1), s);
    W.ptw.alloc(std::max<int64_t>(P.nnz, 1), s);
    { k_mp_weights<<<nblk(n), 256, 0, s>>>(n, P.row_ptr.p, P.col.p, P.val64.p, P.diag64.p, W.pw.p, W.ptw.p); ::pgcp::note_launch(); }
    W.z.alloc(n, s);
    W.zz.alloc(P.K, s);
    W.cnt.alloc(P.K, s);
    W.sigma.alloc(P.K, s);
    W.zz.zero();
    W.cnt.zero();
    DBuf<double> rowv;
    if (ctx->opt.deterministic) rowv.alloc(n, s);
    { k_mp_z<<<nblk(n), 256, 0, s>>>(n, P.row_ptr.p, P.col.p, P.val64.p, P.diag64.p, P.is_bnd.p, P.row_piece.p,
                                    P.welded.p, W.z.p, W.zz.p, W.cnt.p, rowv.p); ::pgcp::note_launch(); }
    if (ctx->opt.deterministic) {
        k_seg_sum<<<(unsigned)P.K, 256, 0, s>>>(rowv.p, P.d_voff.p, W.zz.p);
        ::pgcp::note_launch();
    }
    { k_mp_sigma<<<nblk(P.K), 256, 0, s>>>(P.K, W.zz.p, W.cnt.p, W.sigma.p); ::pgcp::note_launch(); }
    W.F.alloc(n * FIN, s);
    { k_mp_feat<<<nblk(n), 256, 0, s>>>(n, W.z.p, W.sigma.p, P.row_piece.p, P.is_bnd.p,
                                       reinterpret_cast<__nv_bfloat16*>(W.F.p), Ff); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    std::vector<unsigned long long> c(P.K);
    PGCP_CUDA(cudaMemcpyAsync(c.data(), W.cnt.p, P.K * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    PGCP_CUDA(cudaStreamSynchronize(s));
    W.n_inner = 0;
    for (auto v : c) W.n_inner += (int64_t)v;
}

void mp_forward(pgcp_ctx* ctx, const pgcp_gnn* G, Part& P, MpWork& W) {
    cudaStream_t s = ctx->stream;
    const int64_t n = W.n;
    const float* th = G->theta.p;
    const auto* bf = reinterpret_cast<const __nv_bfloat16*>(G->bf.p);
    uint32_t* err = ctx->err.p;
    for (int l = 0; l <= NL; ++l) W.A[l].alloc(n * 128, s);
    W.out.alloc(n * FOUT, s);
    gemm_bf16_tc(s, 1, WID, FIN, W.F.p, FIN, bf + BF_WIN_T, n, th + OFF_BIN, W.A[0].p, 128, nullptr, 0, err);
    for (int l = 0; l < NL; ++l) {
        auto* Al = reinterpret_cast<__nv_bfloat16*>(W.A[l].p);
        { k_mp_agg<<<nblk(n * 32), 256, 0, s>>>(n, P.row_ptr.p, P.col.p, W.pw.p, Al); ::pgcp::note_launch(); }
        gemm_bf16_tc(s, 1, WID, 2 * WID, Al, 128, bf + BF_L_T + (int64_t)l * WID * 2 * WID, n, th + off_b(l),
                     W.A[l + 1].p, 128, nullptr, 0, err);
    }
    gemm_bf16_tc(s, 2, FOUT, WID, W.A[NL].p, 128, bf + BF_WOUT_T, n, th + OFF_BOUT, W.out.p, FOUT, nullptr, 0, err);
    PGCP_CUDA(cudaGetLastError());
}

void check_tc_errors(pgcp_ctx* ctx) {
    if (read_errors(ctx) & DE_TIMEOUT) fail(PGCP_E_CUDA, "tensor-core GEMM: accumulator wait timed out");
}

}  // namespace

int64_t gnn_num_params() { return NPARAM; }

void gnn_init(pgcp_ctx* ctx, pgcp_gnn* G, const float* host_params) {
    cudaStream_t s = ctx->stream;
    G->device = ctx->device;
    G->theta.alloc(NPARAM, s);
    G->grad.alloc(NPARAM, s);
    G->m.alloc(NPARAM, s);
    G->v.alloc(NPARAM, s);
    G->bf.alloc(BF_TOTAL, s);
    G->m.zero();
    G->v.zero();
    G->step = 0;
    gnn_set(ctx, G, host_params);
}

void gnn_set(pgcp_ctx* ctx, pgcp_gnn* G, const float* host_params) {
    cudaStream_t s = ctx->stream;
    PGCP_CUDA(cudaMemcpyAsync(G->theta.p, host_params, NPARAM * sizeof(float), cudaMemcpyHostToDevice, s));
    { k_pack<<<nblk(NL * WID * 2 * WID), 256, 0, s>>>(G->theta.p, reinterpret_cast<__nv_bfloat16*>(G->bf.p)); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    PGCP_CUDA(cudaStreamSynchronize(s));
}

void gnn_get(pgcp_ctx* ctx, const pgcp_gnn* G, float* host_params) {
    PGCP_CUDA(cudaMemcpyAsync(host_params, G->theta.p, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    PGCP_CUDA(cudaStreamSynchronize(ctx->stream));
}

void gnn_inputs(pgcp_ctx* ctx, Part& P, float* Ff, float* target, float* sigma) {
    if (!P.have_weld) fail(PGCP_E_ARG, "network inputs need the welded coordinates (call pgcp_weld first)");
    MpWork W;
    ctx->err.zero();
    mp_inputs(ctx, P, W, Ff);
    cudaStream_t s = ctx->stream;
    if (target) {
        if (!P.have_final) fail(PGCP_E_ARG, "training targets need the final map (call pgcp_global_solve first)");
        { k_mp_target<<<nblk(W.n), 256, 0, s>>>(W.n, P.welded.p, P.final.p, W.sigma.p, P.row_piece.p, P.is_bnd.p,
                                               reinterpret_cast<float2*>(target)); ::pgcp::note_launch(); }
    }
    if (sigma) PGCP_CUDA(cudaMemcpyAsync(sigma, W.sigma.p, P.K * sizeof(float), cudaMemcpyDeviceToDevice, s));
    PGCP_CUDA(cudaGetLastError());
    PGCP_CUDA(cudaStreamSynchronize(s));
}

double gnn_grad(pgcp_ctx* ctx, pgcp_gnn* G, Part& P, int update, float lr) {
    if (!P.have_weld || !P.have_final)
        fail(PGCP_E_ARG, "training needs the welded and final coordinates (pgcp_weld, pgcp_global_solve)");
    cudaStream_t s = ctx->stream;
    ctx->err.zero();
    MpWork W;
    mp_inputs(ctx, P, W, nullptr);
    if (W.n_inner == 0) fail(PGCP_E_ARG, "no interior rows to train on");
    mp_forward(ctx, G, P, W);
    const int64_t n = W.n;
    const auto* bf = reinterpret_cast<const __nv_bfloat16*>(G->bf.p);
    uint32_t* err = ctx->err.p;
    DBuf<float2> tgt;
    DBuf<uint16_t> dOut, dZ;
    DBuf<float> dX, dA;
    DBuf<double> loss;
    tgt.alloc(n, s);
    dOut.alloc(n * FOUT, s);
    dZ.alloc(n * WID, s);
    dX.alloc(n * WID, s);
    dA.alloc(n * 2 * WID, s);
    loss.alloc(1, s);
    loss.zero();
    G->grad.zero();
    float* g = G->grad.p;
    const unsigned wgrid = (unsigned)std::min<int64_t>(ceil_div(n, (int64_t)32), 2 * (int64_t)ctx->num_sms);
    { k_mp_target<<<nblk(n), 256, 0, s>>>(n, P.welded.p, P.final.p, W.sigma.p, P.row_piece.p, P.is_bnd.p, tgt.p); ::pgcp::note_launch(); }
    auto* dO = reinterpret_cast<__nv_bfloat16*>(dOut.p);
    auto* dz = reinterpret_cast<__nv_bfloat16*>(dZ.p);
    { k_mp_loss<<<nblk(n), 256, 0, s>>>(n, W.out.p, tgt.p, P.is_bnd.p, 1.0 / (double)W.n_inner, loss.p, dO); ::pgcp::note_launch(); }
    // output layer
    { k_wgrad<WID, FOUT><<<wgrid, 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16*>(W.A[NL].p), 128, dO, FOUT, n,
                                               g + OFF_WOUT, g + OFF_BOUT); ::pgcp::note_launch(); }
    gemm_bf16_tc(s, 0, WID, FOUT, dO, FOUT, bf + BF_WOUT, n, nullptr, dX.p, WID, nullptr, 0, err);
    // message-passing layers, last to first
    for (int l = NL - 1; l >= 0; --l) {
        { k_relu_bwd<<<nblk(n * WID), 256, 0, s>>>(n, dX.p, reinterpret_cast<const __nv_bfloat16*>(W.A[l + 1].p), 128,
                                                  dz); ::pgcp::note_launch(); }
        { k_wgrad<2 * WID, WID><<<wgrid, 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16*>(W.A[l].p), 128, dz, WID,
                                                      n, g + off_w(l), g + off_b(l)); ::pgcp::note_launch(); }
        gemm_bf16_tc(s, 0, 2 * WID, WID, dz, WID, bf + BF_L + (int64_t)l * 2 * WID * WID, n, nullptr, dA.p, 2 * WID,
                     nullptr, 0, err);
        { k_mp_agg_t<<<nblk(n * 32), 256, 0, s>>>(n, P.row_ptr.p, P.col.p, W.ptw.p, dA.p, dX.p); ::pgcp::note_launch(); }
    }
    // input layer
    { k_relu_bwd<<<nblk(n * WID), 256, 0, s>>>(n, dX.p, reinterpret_cast<const __nv_bfloat16*>(W.A[0].p), 128, dz); ::pgcp::note_launch(); }
    { k_wgrad<FIN, WID><<<wgrid, 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16*>(W.F.p), FIN, dz, WID, n,
                                              g + OFF_WIN, g + OFF_BIN); ::pgcp::note_launch(); }
    if (update) {
        G->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, (float)G->step), c2 = 1.f - std::pow(b2, (float)G->step);
        { k_adam<<<nblk(NPARAM), 256, 0, s>>>(NPARAM, G->theta.p, g, G->m.p, G->v.p, lr, b1, b2, 1e-8f, c1, c2); ::pgcp::note_launch(); }
        { k_pack<<<nblk(NL * WID * 2 * WID), 256, 0, s>>>(G->theta.p, reinterpret_cast<__nv_bfloat16*>(G->bf.p)); ::pgcp::note_launch(); }
    }
    PGCP_CUDA(cudaGetLastError());
    double h = 0.0;
    PGCP_CUDA(cudaMemcpyAsync(&h, loss.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    PGCP_CUDA(cudaStreamSynchronize(s));
    check_tc_errors(ctx);
    return h / (double)W.n_inner;
}

void gnn_predict(pgcp_ctx* ctx, const pgcp_gnn* G, Part& P, double2* x) {
    if (!P.have_weld) fail(PGCP_E_ARG, "prediction needs the welded coordinates (call pgcp_weld first)");
    cudaStream_t s = ctx->stream;
    ctx->err.zero();
    MpWork W;
    mp_inputs(ctx, P, W, nullptr);
    mp_forward(ctx, G, P, W);
    { k_mp_apply<<<nblk(W.n), 256, 0, s>>>(W.n, P.welded.p, W.out.p, W.sigma.p, P.row_piece.p, P.is_bnd.p, x); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    PGCP_CUDA(cudaStreamSynchronize(s));
    check_tc_errors(ctx);
}

int learned_start(pgcp_ctx* ctx, Part& P, double2* x) {
    if (!ctx->gnn) fail(PGCP_E_ARG, "warm_start = PGCP_WARM_LEARNED needs a network (pgcp_set_gnn)");
    cudaStream_t s = ctx->stream;
    const int64_t n = P.Nc;
    DBuf<double2> xl;
    xl.alloc(n, s);
    gnn_predict(ctx, ctx->gnn, P, xl.p);
    DBuf<double> rr;
    DBuf<uint8_t> use;
    rr.alloc(2 * P.K, s);
    use.alloc(P.K, s);
    rr.zero();
    DBuf<double> rowv;
    const bool det = ctx->opt.deterministic != 0;
    if (det) rowv.alloc(n, s);
    for (int w = 0; w < 2; ++w) {
        { k_piece_residual<<<nblk(n), 256, 0, s>>>(n, P.row_ptr.p, P.col.p, P.val64.p, P.is_bnd.p, P.row_piece.p,
                                                  w ? xl.p : x, rr.p + w * P.K, rowv.p); ::pgcp::note_launch(); }
        if (det) {
            k_seg_sum<<<(unsigned)P.K, 256, 0, s>>>(rowv.p, P.d_voff.p, rr.p + w * P.K);
            ::pgcp::note_launch();
        }
    }
    std::vector<double> h(2 * P.K);
    PGCP_CUDA(cudaMemcpyAsync(h.data(), rr.p, 2 * P.K * sizeof(double), cudaMemcpyDeviceToHost, s));
    PGCP_CUDA(cudaStreamSynchronize(s));
    // the learned start is kept only where its FP64 residual is smaller (and finite)
    std::vector<uint8_t> u(P.K);
    int used = 0;
    for (int i = 0; i < P.K; ++i) {
        u[i] = (std::isfinite(h[P.K + i]) && h[P.K + i] < h[i]) ? 1 : 0;
        used += u[i];
    }
    PGCP_CUDA(cudaMemcpyAsync(use.p, u.data(), P.K, cudaMemcpyHostToDevice, s));
    { k_choose<<<nblk(n), 256, 0, s>>>(n, P.row_piece.p, use.p, xl.p, x); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    PGCP_CUDA(cudaStreamSynchronize(s));
    return used;
}

}  // namespace pgcp
