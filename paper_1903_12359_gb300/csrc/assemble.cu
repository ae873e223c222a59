// Cotangent Laplacian assembly into one block-diagonal CSR (Section 4.2).
//
// For every piece, L_pq = -(cot alpha + cot beta) / 2 over the piece's faces
// (one term on a boundary edge), L_pp = -sum_q L_pq: the positive
// semidefinite sign of the paper's matrix (same Laplace solutions).
// Rows are vertex copies in piece order (ascending global id inside a piece);
// columns are rows of the same piece, ascending, with the diagonal stored.
//
//  k_face_cot    one thread per face: the three corner cotangents,
//                cot = (e1 . e2) / |e1 x e2| in FP64 (zero area -> error)
//  k_incidence   vertex -> incident faces (counting + fill)
//  k_row_count   one thread per row: distinct neighbours + 1
//  k_row_fill    one thread per row: sorted columns, accumulated weights
#include <cuda_runtime.h>

#include <algorithm>

#include "pgcp_internal.h"

namespace pgcp {

namespace {

constexpr int MAXV = 64;   // incident faces per vertex copy

__global__ void k_face_cot(const int32_t* __restrict__ cF, const int32_t* __restrict__ copy_vert,
                           const double* __restrict__ V, int64_t nf, double* __restrict__ fw, uint32_t* err) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nf) return;
    double X[3][3];
    for (int c = 0; c < 3; ++c) {
        int g = copy_vert[cF[3 * j + c]];
        X[c][0] = V[3 * (int64_t)g + 0];
        X[c][1] = V[3 * (int64_t)g + 1];
        X[c][2] = V[3 * (int64_t)g + 2];
    }
    for (int c = 0; c < 3; ++c) {
        const double* p = X[c];
        const double* q = X[(c + 1) % 3];
        const double* r = X[(c + 2) % 3];
        double e1x = q[0] - p[0], e1y = q[1] - p[1], e1z = q[2] - p[2];
        double e2x = r[0] - p[0], e2y = r[1] - p[1], e2z = r[2] - p[2];
        double dot = e1x * e2x + e1y * e2y + e1z * e2z;
        double cx = e1y * e2z - e1z * e2y, cy = e1z * e2x - e1x * e2z, cz = e1x * e2y - e1y * e2x;
        double nrm = sqrt(cx * cx + cy * cy + cz * cz);
        if (!(nrm > 0.0)) {
            atomicOr(err, (uint32_t)DE_DEGENERATE);
            fw[3 * j + c] = 0.0;
        } else {
            fw[3 * j + c] = 0.5 * (dot / nrm);   // weight of the edge opposite corner c
        }
    }
}

__global__ void k_incidence_count(const int32_t* __restrict__ cF, int64_t n3, int32_t* __restrict__ deg) {
    int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h < n3) atomicAdd(&deg[cF[h]], 1);
}

__global__ void k_incidence_fill(const int32_t* __restrict__ cF, int64_t n3, const int64_t* __restrict__ off,
                                 int32_t* __restrict__ cursor, int32_t* __restrict__ inc) {
    int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= n3) return;
    int r = cF[h];
    int pos = atomicAdd(&cursor[r], 1);
    inc[off[r] + pos] = (int32_t)h;   // half-edge id = 3 * face + corner
}

// Load and sort (by face id) the incident corners of row r.
__device__ int load_corners(int64_t r, const int64_t* __restrict__ off, const int32_t* __restrict__ inc,
                            int32_t* corners, uint32_t* err) {
    int64_t a = off[r], b = off[r + 1];
    int n = (int)(b - a);
    if (n > MAXV) {
        atomicOr(err, (uint32_t)DE_VALENCE);
        n = MAXV;
    }
    for (int i = 0; i < n; ++i) {
        int v = inc[a + i];
        int k = i;
        while (k > 0 && corners[k - 1] > v) {
            corners[k] = corners[k - 1];
            --k;
        }
        corners[k] = v;
    }
    return n;
}

__global__ void k_row_count(const int32_t* __restrict__ cF, const int64_t* __restrict__ off,
                            const int32_t* __restrict__ inc, int64_t Nc, int32_t* __restrict__ rowlen,
                            uint32_t* err) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Nc) return;
    int32_t corners[MAXV];
    int32_t nbr[2 * MAXV];
    int n = load_corners(r, off, inc, corners, err);
    int m = 0;
    for (int i = 0; i < n; ++i) {
        int h = corners[i];
        int j = h / 3, c = h - 3 * j;
        int q = cF[3 * j + (c + 1) % 3], s = cF[3 * j + (c + 2) % 3];
        for (int t = 0; t < 2; ++t) {
            int v = t ? s : q;
            bool seen = false;
            for (int u = 0; u < m; ++u) seen |= (nbr[u] == v);
            if (!seen) nbr[m++] = v;
        }
    }
    rowlen[r] = m + 1;
}

__global__ void k_row_fill(const int32_t* __restrict__ cF, const int64_t* __restrict__ off,
                           const int32_t* __restrict__ inc, const double* __restrict__ fw, int64_t Nc,
                           const int64_t* __restrict__ rowptr64, int32_t* __restrict__ rowptr,
                           int32_t* __restrict__ col, double* __restrict__ val, float* __restrict__ val32,
                           double* __restrict__ diag, uint32_t* err) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Nc) return;
    int32_t corners[MAXV];
    int32_t nbr[2 * MAXV + 1];
    double w[2 * MAXV + 1];
    int n = load_corners(r, off, inc, corners, err);
    int m = 0;
    nbr[m] = (int32_t)r;   // diagonal
    w[m++] = 0.0;
    for (int i = 0; i < n; ++i) {
        int h = corners[i];
        int j = h / 3, c = h - 3 * j;
        int q = cF[3 * j + (c + 1) % 3], s = cF[3 * j + (c + 2) % 3];
        // edge (r, q) is opposite corner c+2; edge (r, s) is opposite corner c+1
        double wq = fw[3 * j + (c + 2) % 3], ws = fw[3 * j + (c + 1) % 3];
        for (int t = 0; t < 2; ++t) {
            int v = t ? s : q;
            double wv = t ? ws : wq;
            int u = 0;
            while (u < m && nbr[u] != v) ++u;
            if (u == m) {
                nbr[m] = v;
                w[m++] = 0.0;
            }
            w[u] += wv;
        }
    }
    // sort columns ascending (insertion sort, small rows)
    for (int i = 1; i < m; ++i) {
        int v = nbr[i];
        double x = w[i];
        int k = i;
        while (k > 0 && nbr[k - 1] > v) {
            nbr[k] = nbr[k - 1];
            w[k] = w[k - 1];
            --k;
        }
        nbr[k] = v;
        w[k] = x;
    }
    double d = 0.0;
    for (int i = 0; i < m; ++i)
        if (nbr[i] != (int32_t)r) d += w[i];
    int64_t base = rowptr64[r];
    rowptr[r] = (int32_t)base;
    for (int i = 0; i < m; ++i) {
        double v = (nbr[i] == (int32_t)r) ? d : -w[i];
        col[base + i] = nbr[i];
        val[base + i] = v;
        val32[base + i] = (float)v;
    }
    diag[r] = d;
}

__global__ void k_set_last(int32_t* rowptr, int64_t Nc, int64_t nnz) { rowptr[Nc] = (int32_t)nnz; }

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, ceil_div(n, t)); }

}  // namespace

void assemble_laplacian(pgcp_ctx* ctx, Part& P) {
    cudaStream_t s = ctx->stream;
    const int64_t nf = P.nf, Nc = P.Nc;
    ctx->err.zero();
    DBuf<double> fw;
    fw.alloc(3 * nf, s);
    { k_face_cot<<<nblk(nf), 256, 0, s>>>(P.cF.p, P.copy_vert.p, P.V.p, nf, fw.p, ctx->err.p); ::pgcp::note_launch(); }
    DBuf<int32_t> deg, cursor, inc, rowlen;
    DBuf<int64_t> off, rp64;
    deg.alloc(Nc + 1, s);
    deg.zero();
    { k_incidence_count<<<nblk(3 * nf), 256, 0, s>>>(P.cF.p, 3 * nf, deg.p); ::pgcp::note_launch(); }
    off.alloc(Nc + 1, s);
    exclusive_scan_i32_to_i64(deg.p, off.p, Nc + 1, s, nullptr);
    cursor.alloc(Nc, s);
    cursor.zero();
    inc.alloc(3 * nf, s);
    { k_incidence_fill<<<nblk(3 * nf), 256, 0, s>>>(P.cF.p, 3 * nf, off.p, cursor.p, inc.p); ::pgcp::note_launch(); }
    rowlen.alloc(Nc + 1, s);
    rowlen.zero();
    { k_row_count<<<nblk(Nc, 128), 128, 0, s>>>(P.cF.p, off.p, inc.p, Nc, rowlen.p, ctx->err.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    rp64.alloc(Nc + 1, s);
    int64_t nnz = 0;
    exclusive_scan_i32_to_i64(rowlen.p, rp64.p, Nc + 1, s, &nnz);
    if (nnz >= (1ll << 31)) fail(PGCP_E_ARG, "more than 2^31 matrix entries");
    P.nnz = nnz;
    P.row_ptr.alloc(Nc + 1, s);
    P.col.alloc(nnz, s);
    P.val64.alloc(nnz, s);
    P.val32.alloc(nnz, s);
    P.diag64.alloc(Nc, s);
    { k_row_fill<<<nblk(Nc, 128), 128, 0, s>>>(P.cF.p, off.p, inc.p, fw.p, Nc, rp64.p, P.row_ptr.p, P.col.p,
                                             P.val64.p, P.val32.p, P.diag64.p, ctx->err.p); ::pgcp::note_launch(); }
    { k_set_last<<<1, 1, 0, s>>>(P.row_ptr.p, Nc, nnz); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    uint32_t e = read_errors(ctx);
    if (e & DE_DEGENERATE) fail(PGCP_E_DEGENERATE, "zero-area face");
    if (e & DE_VALENCE) fail(PGCP_E_ARG, "a vertex has more than 64 incident faces in one piece");
    // the incidence stays with the part: other element matrices on the same
    // pattern (the fold fix's Beltrami solver) are assembled from it
    P.inc_off = std::move(off);
    P.inc = std::move(inc);
    P.rp64 = std::move(rp64);
}

void assemble_values(pgcp_ctx* ctx, Part& P, const double* fw, double* val64, float* val32, double* diag64) {
    cudaStream_t s = ctx->stream;
    const int64_t Nc = P.Nc;
    if (!P.inc.p || !P.inc_off.p || !P.rp64.p) fail(PGCP_E_ARG, "the part's Laplacian is not assembled");
    DBuf<int32_t> rp, cl;   // the pattern is rewritten identically; kept apart from the part's
    rp.alloc(Nc + 1, s);
    cl.alloc(std::max<int64_t>(P.nnz, 1), s);
    ctx->err.zero();
    { k_row_fill<<<nblk(Nc, 128), 128, 0, s>>>(P.cF.p, P.inc_off.p, P.inc.p, fw, Nc, P.rp64.p, rp.p, cl.p, val64,
                                             val32, diag64, ctx->err.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    if (read_errors(ctx) & DE_VALENCE) fail(PGCP_E_ARG, "a vertex has more than 64 incident faces in one piece");
}

}  // namespace pgcp
