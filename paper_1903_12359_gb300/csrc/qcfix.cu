// Fold-over fix by quasi-conformal composition (Section 4.5 and the last step
// of Algorithm 3; Beltrami coefficient and composition formula, Section 3.5).
//
// A face folds where the Beltrami coefficient mu = f_zbar / f_z of the affine
// map from the surface triangle (laid flat in its own frame: p0 at 0, p1 on
// +x) to the parameter triangle has |mu| >= 1 - 1e-6, or where the parameter
// triangle's signed area is <= 0.  A piece that folds is composed, round after
// round, with the quasi-conformal map whose composition keeps every face's
// coefficient except within t rings of the folded faces, where its modulus is
// capped at 0.7 (round t); the composed map is the solution of the linear
// Beltrami solver with the piece's boundary values kept:
//   div(A_nu grad u) = 0 and div(A_nu grad v) = 0,
//   A_nu = [[(rho-1)^2 + tau^2, -2 tau], [-2 tau, (rho+1)^2 + tau^2]] / (1 - |nu|^2),
// nu = rho + i tau, with linear elements on the surface triangles.  Its
// element matrices have zero row sums, so the edge weights w = -K_jk assemble
// on the Laplacian's pattern like the cotangent weights (nu = 0 gives exactly
// those), and the batched Dirichlet PCG of the final solve solves it.  A piece
// that does not fold at the start of a round keeps its map bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "pgcp_internal.h"

namespace pgcp {

namespace {

constexpr double FOLD_THRESH = 1e-6;
constexpr double KAPPA = 0.7;
constexpr int ROUNDS = 16;

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, ceil_div(n, t)); }

// The face's flat frame (l1, x2, y2): p0 -> (0, 0), p1 -> (l1, 0), p2 -> (x2, y2).
__device__ __forceinline__ void face_frame(const double* __restrict__ V, const int32_t* __restrict__ copy_vert,
                                           const int32_t* f, double& l1, double& x2, double& y2) {
    double p[3][3];
    for (int c = 0; c < 3; ++c) {
        const int64_t g = copy_vert[f[c]];
        for (int k = 0; k < 3; ++k) p[c][k] = V[3 * g + k];
    }
    const double e1x = p[1][0] - p[0][0], e1y = p[1][1] - p[0][1], e1z = p[1][2] - p[0][2];
    const double e2x = p[2][0] - p[0][0], e2y = p[2][1] - p[0][1], e2z = p[2][2] - p[0][2];
    l1 = sqrt(e1x * e1x + e1y * e1y + e1z * e1z);
    x2 = (e1x * e2x + e1y * e2y + e1z * e2z) / l1;
    const double cx = e1y * e2z - e1z * e2y, cy = e1z * e2x - e1x * e2z, cz = e1x * e2y - e1y * e2x;
    y2 = sqrt(cx * cx + cy * cy + cz * cz) / l1;
}

// Per face: mu of the map X, and whether the face folds; folded faces are
// counted per piece.
__global__ void k_fold_mu(int64_t nf, const int32_t* __restrict__ cF, const int32_t* __restrict__ copy_vert,
                          const int32_t* __restrict__ row_piece, const double* __restrict__ V,
                          const double2* __restrict__ X, double2* __restrict__ mu, uint8_t* __restrict__ bad,
                          unsigned long long* __restrict__ piece_bad) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nf) return;
    const int32_t f[3] = {cF[3 * j], cF[3 * j + 1], cF[3 * j + 2]};
    double l1, x2, y2;
    face_frame(V, copy_vert, f, l1, x2, y2);
    const double2 w0 = X[f[0]], a = X[f[1]], b = X[f[2]];
    const double w1x = a.x - w0.x, w1y = a.y - w0.y, w2x = b.x - w0.x, w2y = b.y - w0.y;
    // f(x, y) = w1 (x - x2 y / y2) / l1 + w2 y / y2: f_x = w1 / l1, f_y = (w2 - w1 x2 / l1) / y2
    const double fxx = w1x / l1, fxy = w1y / l1;
    const double fyx = (w2x - w1x * x2 / l1) / y2, fyy = (w2y - w1y * x2 / l1) / y2;
    // f_z = (f_x - i f_y) / 2, f_zbar = (f_x + i f_y) / 2
    const double zr = 0.5 * (fxx + fyy), zi = 0.5 * (fxy - fyx);
    const double br = 0.5 * (fxx - fyy), bi = 0.5 * (fxy + fyx);
    const double den = zr * zr + zi * zi;
    const double mr = den > 0.0 ? (br * zr + bi * zi) / den : 0.0;
    const double mi = den > 0.0 ? (bi * zr - br * zi) / den : 0.0;
    mu[j] = make_double2(mr, mi);
    const double area = 0.5 * (w1x * w2y - w1y * w2x);
    const bool folds = !(area > 0.0) || !(sqrt(mr * mr + mi * mi) < 1.0 - FOLD_THRESH) || !(den > 0.0);
    bad[j] = folds ? 1 : 0;
    if (folds) atomicAdd(&piece_bad[row_piece[f[0]]], 1ull);
}

__global__ void k_mark_rows(int64_t nf, const int32_t* __restrict__ cF, const uint8_t* __restrict__ reg,
                            uint8_t* __restrict__ mark) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nf || !reg[j]) return;
    for (int c = 0; c < 3; ++c) mark[cF[3 * j + c]] = 1;
}

__global__ void k_mark_faces(int64_t nf, const int32_t* __restrict__ cF, const uint8_t* __restrict__ mark,
                             uint8_t* __restrict__ reg) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nf) return;
    reg[j] = (mark[cF[3 * j]] | mark[cF[3 * j + 1]] | mark[cF[3 * j + 2]]) ? 1 : 0;
}

// Edge weights of the Beltrami solver's element matrix: fw[3 j + c] = -K of the
// edge opposite corner c, K_jk = area grad(phi_j)^T A_nu grad(phi_k) in the
// face's flat frame.
__global__ void k_lbs_weights(int64_t nf, const int32_t* __restrict__ cF, const int32_t* __restrict__ copy_vert,
                              const double* __restrict__ V, const double2* __restrict__ mu,
                              const uint8_t* __restrict__ reg, double* __restrict__ fw) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nf) return;
    const int32_t f[3] = {cF[3 * j], cF[3 * j + 1], cF[3 * j + 2]};
    double l1, x2, y2;
    face_frame(V, copy_vert, f, l1, x2, y2);
    double rho = mu[j].x, tau = mu[j].y;
    const double m = sqrt(rho * rho + tau * tau);
    if (reg[j] && m > KAPPA) {
        rho *= KAPPA / m;
        tau *= KAPPA / m;
    }
    const double d = 1.0 - (rho * rho + tau * tau);
    const double a1 = ((rho - 1.0) * (rho - 1.0) + tau * tau) / d;
    const double a2 = -2.0 * tau / d;
    const double a3 = ((rho + 1.0) * (rho + 1.0) + tau * tau) / d;
    const double area = 0.5 * l1 * y2;
    const double P[3][2] = {{0.0, 0.0}, {l1, 0.0}, {x2, y2}};
    double G[3][2];
    for (int c = 0; c < 3; ++c) {   // gradient of corner c's hat function: its opposite edge rotated
        const double ex = P[(c + 2) % 3][0] - P[(c + 1) % 3][0], ey = P[(c + 2) % 3][1] - P[(c + 1) % 3][1];
        G[c][0] = -ey / (2.0 * area);
        G[c][1] = ex / (2.0 * area);
    }
    for (int c = 0; c < 3; ++c) {
        const int p = (c + 1) % 3, q = (c + 2) % 3;
        const double k = area * ((a1 * G[p][0] + a2 * G[p][1]) * G[q][0] + (a2 * G[p][0] + a3 * G[p][1]) * G[q][1]);
        fw[3 * j + c] = -k;
    }
}

__global__ void k_scatter(int64_t n, const int32_t* __restrict__ copy_vert, const double* __restrict__ U,
                          double2* __restrict__ X) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t g = copy_vert[i];
    X[i] = make_double2(U[2 * g], U[2 * g + 1]);
}

// rows of pieces that do not fold take their saved map back
__global__ void k_restore(int64_t n, const int32_t* __restrict__ row_piece, const uint8_t* __restrict__ active,
                          const double2* __restrict__ saved, double2* __restrict__ X) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || active[row_piece[i]]) return;
    X[i] = saved[i];
}

// U[v] from the copy of the lowest-label piece holding v
__global__ void k_gather2(int64_t n, const int32_t* __restrict__ copy_vert, const int32_t* __restrict__ first_copy,
                          const double2* __restrict__ X, double* __restrict__ U) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t v = copy_vert[i];
    if (first_copy[v] != (int32_t)i) return;
    U[2 * v] = X[i].x;
    U[2 * v + 1] = X[i].y;
}

}  // namespace

void fix_folds(pgcp_ctx* ctx, Part& P, double* U, pgcp_fold_report* rep) {
    cudaStream_t s = ctx->stream;
    const int64_t n = P.Nc, nf = P.nf;
    const int K = P.K;
    *rep = pgcp_fold_report{0, 0, 0, 0};
    DBuf<double2> X, saved, mu;
    DBuf<uint8_t> bad, reg, mark, active;
    DBuf<unsigned long long> pbad;
    X.alloc(n, s);
    saved.alloc(n, s);
    mu.alloc(nf, s);
    bad.alloc(nf, s);
    reg.alloc(nf, s);
    mark.alloc(n, s);
    active.alloc(K, s);
    pbad.alloc(K, s);
    { k_scatter<<<nblk(n), 256, 0, s>>>(n, P.copy_vert.p, U, X.p); ::pgcp::note_launch(); }
    std::vector<unsigned long long> hb(K);
    std::vector<uint8_t> hact(K);
    auto count = [&]() {
        pbad.zero();
        { k_fold_mu<<<nblk(nf), 256, 0, s>>>(nf, P.cF.p, P.copy_vert.p, P.row_piece.p, P.V.p, X.p, mu.p, bad.p,
                                             pbad.p); ::pgcp::note_launch(); }
        PGCP_CUDA(cudaGetLastError());
        PGCP_CUDA(cudaMemcpyAsync(hb.data(), pbad.p, K * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        PGCP_CUDA(cudaStreamSynchronize(s));
        int64_t tot = 0;
        for (int i = 0; i < K; ++i) tot += (int64_t)hb[i];
        return tot;
    };
    int64_t nbad = count();
    rep->folded_before = nbad;
    for (int i = 0; i < K; ++i) rep->pieces_fixed += hb[i] ? 1 : 0;
    if (nbad == 0) return;
    DBuf<double> fw, v64, d64;
    DBuf<float> v32;
    fw.alloc(3 * nf, s);
    v64.alloc(std::max<int64_t>(P.nnz, 1), s);
    v32.alloc(std::max<int64_t>(P.nnz, 1), s);
    d64.alloc(n, s);
    const pgcp_stats keep = P.stats;
    int t = 0;
    while (nbad > 0 && t < ROUNDS) {
        ++t;
        for (int i = 0; i < K; ++i) hact[i] = hb[i] ? 1 : 0;
        PGCP_CUDA(cudaMemcpyAsync(active.p, hact.data(), K, cudaMemcpyHostToDevice, s));
        PGCP_CUDA(cudaMemcpyAsync(reg.p, bad.p, nf, cudaMemcpyDeviceToDevice, s));
        for (int r = 0; r < t; ++r) {   // the fold region: t rings of faces sharing a vertex
            mark.zero();
            { k_mark_rows<<<nblk(nf), 256, 0, s>>>(nf, P.cF.p, reg.p, mark.p); ::pgcp::note_launch(); }
            { k_mark_faces<<<nblk(nf), 256, 0, s>>>(nf, P.cF.p, mark.p, reg.p); ::pgcp::note_launch(); }
        }
        { k_lbs_weights<<<nblk(nf), 256, 0, s>>>(nf, P.cF.p, P.copy_vert.p, P.V.p, mu.p, reg.p, fw.p);
          ::pgcp::note_launch(); }
        PGCP_CUDA(cudaGetLastError());
        assemble_values(ctx, P, fw.p, v64.p, v32.p, d64.p);
        PGCP_CUDA(cudaMemcpyAsync(saved.p, X.p, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        // the batched Dirichlet solve (boundary rows fixed) on the Beltrami
        // solver's matrix, swapped in for the Laplacian's values
        std::swap(P.val64, v64);
        std::swap(P.val32, v32);
        std::swap(P.diag64, d64);
        SolveResult res;
        try {
            res = pcg_solve(ctx, P, 0, P.is_bnd.p, X.p);
        } catch (...) {
            std::swap(P.val64, v64);
            std::swap(P.val32, v32);
            std::swap(P.diag64, d64);
            P.stats = keep;
            throw;
        }
        std::swap(P.val64, v64);
        std::swap(P.val32, v32);
        std::swap(P.diag64, d64);
        { k_restore<<<nblk(n), 256, 0, s>>>(n, P.row_piece.p, active.p, saved.p, X.p); ::pgcp::note_launch(); }
        PGCP_CUDA(cudaGetLastError());
        if (!(res.relres <= ctx->opt.tol)) {
            P.stats = keep;
            fail(PGCP_E_NO_CONVERGENCE, "fold fix: Beltrami solve reached relative residual " + std::to_string(res.relres));
        }
        nbad = count();
    }
    P.stats = keep;
    rep->rounds = t;
    rep->folded_after = nbad;
    { k_gather2<<<nblk(n), 256, 0, s>>>(n, P.copy_vert.p, P.first_copy.p, X.p, U); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    PGCP_CUDA(cudaStreamSynchronize(s));
}

}  // namespace pgcp
