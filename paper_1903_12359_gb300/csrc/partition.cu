// Surface partition on the GPU (Section 4.1).
//
// 1. Edge table: every half-edge of every face is inserted into an open-
//    addressing hash table keyed by its undirected edge; a slot records the
//    two faces (with the direction each face traverses the edge).  More than
//    two faces -> non-manifold; two faces traversing the edge the same way ->
//    inconsistent orientation.
// 2. Cut edges (given as a list, or implied by face labels) are marked.
// 3. Union-find over faces across every interior, uncut edge; roots hook the
//    larger id under the smaller, so a component's root is its smallest face.
//    Labels are the ranks of the roots (exclusive scan).
// 4. Faces are ordered by (label, id) and vertex copies by (label, global id)
//    with a stable radix sort; faces are rewritten as copy rows.
// 5. Boundary half-edges of every piece (edges with one incident face in the
//    piece) are listed for the host, which walks the loops.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <vector>

#include "pgcp_internal.h"

namespace pgcp {

namespace {

constexpr uint64_t EMPTY_KEY = ~0ull;
constexpr int UF_LIMIT = 1 << 22;

__device__ __forceinline__ uint64_t edge_key(int u, int v) {
    unsigned a = (unsigned)min(u, v), b = (unsigned)max(u, v);
    return ((uint64_t)a << 32) | (uint64_t)b;
}

__device__ __forceinline__ uint64_t hash64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

__device__ __forceinline__ void set_err(uint32_t* err, uint32_t bit) { atomicOr(err, bit); }

// Slot payload: face * 2 + (u < v ? 1 : 0) for the first and second face.
__global__ void k_edge_insert(const int32_t* __restrict__ F, int64_t nf, uint64_t* __restrict__ keys,
                              int32_t* __restrict__ fa, int32_t* __restrict__ fb, int32_t* __restrict__ cnt,
                              uint64_t mask, uint32_t* err) {
    int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= 3 * nf) return;
    int64_t f = h / 3;
    int c = (int)(h - 3 * f);
    int u = F[3 * f + c], v = F[3 * f + (c + 1) % 3];
    uint64_t key = edge_key(u, v);
    int32_t payload = (int32_t)(f * 2 + (u < v ? 1 : 0));
    uint64_t s = hash64(key) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        unsigned long long old = atomicCAS((unsigned long long*)&keys[s], (unsigned long long)EMPTY_KEY,
                                           (unsigned long long)key);
        if (old == EMPTY_KEY || old == key) {
            int pos = atomicAdd(&cnt[s], 1);
            if (pos == 0) fa[s] = payload;
            else if (pos == 1) fb[s] = payload;
            else set_err(err, DE_NONMANIFOLD);
            return;
        }
        s = (s + 1) & mask;
    }
    set_err(err, DE_HASH_FULL);
}

__device__ __forceinline__ int64_t edge_lookup(const uint64_t* __restrict__ keys, uint64_t mask, uint64_t key) {
    uint64_t s = hash64(key) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        uint64_t k = keys[s];
        if (k == key) return (int64_t)s;
        if (k == EMPTY_KEY) return -1;
        s = (s + 1) & mask;
    }
    return -1;
}

__global__ void k_edge_check(const uint64_t* __restrict__ keys, const int32_t* __restrict__ fa,
                             const int32_t* __restrict__ fb, const int32_t* __restrict__ cnt,
                             const int32_t* __restrict__ labels, uint8_t* __restrict__ cut, uint64_t nslot,
                             uint32_t* err) {
    uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslot || keys[s] == EMPTY_KEY) return;
    int c = cnt[s];
    if (c > 2) set_err(err, DE_NONMANIFOLD);
    if (c == 2) {
        if ((fa[s] & 1) == (fb[s] & 1)) set_err(err, DE_ORIENT);
        if (labels) cut[s] = labels[fa[s] >> 1] != labels[fb[s] >> 1];
    }
}

__global__ void k_mark_cut(const int32_t* __restrict__ cuts, int64_t n_cut, const uint64_t* __restrict__ keys,
                           uint64_t mask, uint8_t* __restrict__ cut, int64_t nv, uint32_t* err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_cut) return;
    int u = cuts[2 * i], v = cuts[2 * i + 1];
    if (u < 0 || v < 0 || u >= nv || v >= nv || u == v) {
        set_err(err, DE_CUT_MISSING);
        return;
    }
    int64_t s = edge_lookup(keys, mask, edge_key(u, v));
    if (s < 0) set_err(err, DE_CUT_MISSING);
    else cut[s] = 1;
}

__device__ int uf_find(volatile int32_t* parent, int x) {
    // parent[x] <= x always, so the walk terminates; path halving is a benign race
    while (true) {
        int px = parent[x];
        if (px == x) return x;
        int ppx = parent[px];
        if (ppx != px) parent[x] = ppx;
        x = px;
    }
}

__global__ void k_union(const uint64_t* __restrict__ keys, const int32_t* __restrict__ fa,
                        const int32_t* __restrict__ fb, const int32_t* __restrict__ cnt,
                        const uint8_t* __restrict__ cut, uint64_t nslot, int32_t* parent, uint32_t* err) {
    uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslot || keys[s] == EMPTY_KEY || cnt[s] != 2 || cut[s]) return;
    int a = fa[s] >> 1, b = fb[s] >> 1;
    for (int it = 0; it < UF_LIMIT; ++it) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a == b) return;
        if (a > b) { int t = a; a = b; b = t; }
        int old = atomicCAS(&parent[b], b, a);   // hook the larger root under the smaller
        if (old == b) return;
        b = old;
    }
    set_err(err, DE_UNION_LIMIT);
}

// Read-only walk to the root.  The final compression must not halve paths:
// another thread's halving could overwrite parent[f] = root with a non-root
// ancestor after thread f wrote it.
__device__ int uf_root(volatile int32_t* parent, int x) {
    while (true) {
        int px = parent[x];
        if (px == x) return x;
        x = px;
    }
}

__global__ void k_uf_compress(int32_t* parent, int64_t nf, int32_t* __restrict__ is_root) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int r = uf_root(parent, (int)f);
    parent[f] = r;
    is_root[f] = (r == (int)f);
}

__global__ void k_label(const int32_t* __restrict__ parent, const int64_t* __restrict__ rank, int64_t nf,
                        int32_t* __restrict__ label, uint64_t* __restrict__ fkey, int32_t* __restrict__ fval) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int32_t l = (int32_t)rank[parent[f]];
    label[f] = l;
    fkey[f] = (uint64_t)l;
    fval[f] = (int32_t)f;
}

// segment starts of a sorted key array: off[key] = first index (keys dense 0..K-1)
__global__ void k_segment_starts(const uint64_t* __restrict__ keys, int64_t n, int64_t* __restrict__ off,
                                 int shift_div, uint64_t div) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint64_t kj = keys[j] / div;
    if (j == 0 || keys[j - 1] / div != kj) off[kj] = j;
    (void)shift_div;
}

__global__ void k_corner_keys(const int32_t* __restrict__ F, const int32_t* __restrict__ label, int64_t nf,
                              uint64_t nv, uint64_t* __restrict__ ckey, int32_t* __restrict__ cval) {
    int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= 3 * nf) return;
    int64_t f = h / 3;
    ckey[h] = (uint64_t)label[f] * nv + (uint64_t)F[h];
    cval[h] = 0;
}

__global__ void k_unique_flags(const uint64_t* __restrict__ k, int64_t n, int32_t* __restrict__ flag) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    flag[j] = (j == 0 || k[j] != k[j - 1]) ? 1 : 0;
}

__global__ void k_unique_compact(const uint64_t* __restrict__ k, const int32_t* __restrict__ flag,
                                 const int64_t* __restrict__ pos, int64_t n, uint64_t nv,
                                 uint64_t* __restrict__ ukey, int32_t* __restrict__ copy_vert,
                                 int32_t* __restrict__ row_piece) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n || !flag[j]) return;
    int64_t r = pos[j];
    ukey[r] = k[j];
    copy_vert[r] = (int32_t)(k[j] % nv);
    row_piece[r] = (int32_t)(k[j] / nv);
}

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* __restrict__ a, int64_t lo, int64_t hi,
                                                   uint64_t key) {
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Faces in piece order, as copy rows; first_copy[v] = lowest row holding v.
__global__ void k_face_rows(const int32_t* __restrict__ F, const int32_t* __restrict__ forder,
                            const int32_t* __restrict__ label, int64_t nf, const uint64_t* __restrict__ ukey,
                            const int64_t* __restrict__ voff, uint64_t nv, int32_t* __restrict__ cF,
                            int32_t* __restrict__ first_copy) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nf) return;
    int f = forder[j];
    int l = label[f];
    for (int c = 0; c < 3; ++c) {
        int v = F[3 * (int64_t)f + c];
        uint64_t key = (uint64_t)l * nv + (uint64_t)v;
        int64_t r = lower_bound_u64(ukey, voff[l], voff[l + 1], key);
        cF[3 * j + c] = (int32_t)r;
        atomicMin(&first_copy[v], (int32_t)r);
    }
}

// Boundary half-edges of the pieces: face traverses u -> v and the other face
// across the edge (if any) has another label.
__global__ void k_boundary_halfedges(const int32_t* __restrict__ F, const int32_t* __restrict__ forder,
                                     const int32_t* __restrict__ label, const int32_t* __restrict__ cF, int64_t nf,
                                     const uint64_t* __restrict__ keys, const int32_t* __restrict__ fa,
                                     const int32_t* __restrict__ fb, const int32_t* __restrict__ cnt,
                                     uint64_t mask, int64_t cap, unsigned long long* __restrict__ counter,
                                     int4* __restrict__ out, int32_t* __restrict__ out_piece) {
    int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= 3 * nf) return;
    int64_t j = h / 3;
    int c = (int)(h - 3 * j);
    int f = forder[j];
    int l = label[f];
    int u = F[3 * (int64_t)f + c], v = F[3 * (int64_t)f + (c + 1) % 3];
    int64_t s = edge_lookup(keys, mask, edge_key(u, v));
    if (s < 0) return;
    bool bnd;
    if (cnt[s] == 1) {
        bnd = true;
    } else {
        int other = ((fa[s] >> 1) == f) ? (fb[s] >> 1) : (fa[s] >> 1);
        bnd = label[other] != l;
    }
    if (!bnd) return;
    unsigned long long pos = atomicAdd(counter, 1ull);
    if ((int64_t)pos < cap) {
        out[pos] = make_int4(cF[3 * j + c], cF[3 * j + (c + 1) % 3], u, v);
        out_piece[pos] = l;
    }
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void k_iota(int32_t* p, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (int32_t)i;
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, ceil_div(n, t)); }

void raise_dev_errors(uint32_t e) {
    if (e & DE_HASH_FULL) fail(PGCP_E_CUDA, "edge table overflow");
    if (e & DE_NONMANIFOLD) fail(PGCP_E_NONMANIFOLD, "an edge is shared by more than two faces");
    if (e & DE_ORIENT) fail(PGCP_E_ARG, "faces are not consistently oriented");
    if (e & DE_CUT_MISSING) fail(PGCP_E_ARG, "a cut edge is not an edge of the mesh");
    if (e & DE_UNION_LIMIT) fail(PGCP_E_CUDA, "union-find did not settle");
}

}  // namespace

void build_partition(pgcp_ctx* ctx, Part& P, const int32_t* d_labels, const int32_t* d_cut, int64_t n_cut) {
    cudaStream_t s = ctx->stream;
    const int64_t nf = P.nf, nv = P.nv;
    if (nf <= 0 || nv <= 0) fail(PGCP_E_ARG, "empty mesh");
    if (nf >= (1ll << 30) || nv >= (1ll << 31) - 1) fail(PGCP_E_ARG, "mesh too large for int32 indices");
    ctx->err.zero();
    // ---- edge table
    uint64_t cap = 1024;
    while (cap < (uint64_t)(4 * nf)) cap <<= 1;   // ~1.5 nf edges -> load <= 0.375
    const uint64_t mask = cap - 1;
    DBuf<uint64_t> keys;
    DBuf<int32_t> fa, fb, cnt;
    DBuf<uint8_t> cut;
    keys.alloc(cap, s);
    fa.alloc(cap, s);
    fb.alloc(cap, s);
    cnt.alloc(cap, s);
    cut.alloc(cap, s);
    PGCP_CUDA(cudaMemsetAsync(keys.p, 0xff, cap * sizeof(uint64_t), s));
    cnt.zero();
    cut.zero();
    { k_edge_insert<<<nblk(3 * nf), 256, 0, s>>>(P.F.p, nf, keys.p, fa.p, fb.p, cnt.p, mask, ctx->err.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    { k_edge_check<<<nblk((int64_t)cap), 256, 0, s>>>(keys.p, fa.p, fb.p, cnt.p, d_labels, cut.p, cap, ctx->err.p); ::pgcp::note_launch(); }
    if (!d_labels && d_cut && n_cut > 0)
        { k_mark_cut<<<nblk(n_cut), 256, 0, s>>>(d_cut, n_cut, keys.p, mask, cut.p, nv, ctx->err.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    raise_dev_errors(read_errors(ctx));
    // ---- union-find
    DBuf<int32_t> parent, is_root;
    parent.alloc(nf, s);
    is_root.alloc(nf, s);
    { k_iota<<<nblk(nf), 256, 0, s>>>(parent.p, nf); ::pgcp::note_launch(); }
    { k_union<<<nblk((int64_t)cap), 256, 0, s>>>(keys.p, fa.p, fb.p, cnt.p, cut.p, cap, parent.p, ctx->err.p); ::pgcp::note_launch(); }
    { k_uf_compress<<<nblk(nf), 256, 0, s>>>(parent.p, nf, is_root.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    DBuf<int64_t> rank;
    rank.alloc(nf, s);
    int64_t K = 0;
    exclusive_scan_i32_to_i64(is_root.p, rank.p, nf, s, &K);
    raise_dev_errors(read_errors(ctx));
    P.K = (int32_t)K;
    // ---- labels, faces by (label, id)
    P.face_label.alloc(nf, s);
    DBuf<uint64_t> fkey;
    DBuf<int32_t> forder;
    fkey.alloc(nf, s);
    forder.alloc(nf, s);
    { k_label<<<nblk(nf), 256, 0, s>>>(parent.p, rank.p, nf, P.face_label.p, fkey.p, forder.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    int lbits = 1;
    while ((1ll << lbits) < K) ++lbits;
    radix_sort_pairs(fkey.p, forder.p, nf, lbits, s);
    DBuf<int64_t> d_foff;
    d_foff.alloc(K + 1, s);
    { k_segment_starts<<<nblk(nf), 256, 0, s>>>(fkey.p, nf, d_foff.p, 0, 1); ::pgcp::note_launch(); }
    P.foff.assign(K + 1, 0);
    PGCP_CUDA(cudaMemcpyAsync(P.foff.data(), d_foff.p, K * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    // ---- vertex copies by (label, global id)
    DBuf<uint64_t> ckey;
    DBuf<int32_t> cval;
    ckey.alloc(3 * nf, s);
    cval.alloc(3 * nf, s);
    { k_corner_keys<<<nblk(3 * nf), 256, 0, s>>>(P.F.p, P.face_label.p, nf, (uint64_t)nv, ckey.p, cval.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    int cbits = 1;
    while ((1ull << cbits) < (uint64_t)K * (uint64_t)nv) ++cbits;
    radix_sort_pairs(ckey.p, cval.p, 3 * nf, cbits, s);
    DBuf<int32_t> flag;
    DBuf<int64_t> pos;
    flag.alloc(3 * nf, s);
    pos.alloc(3 * nf, s);
    { k_unique_flags<<<nblk(3 * nf), 256, 0, s>>>(ckey.p, 3 * nf, flag.p); ::pgcp::note_launch(); }
    int64_t Nc = 0;
    exclusive_scan_i32_to_i64(flag.p, pos.p, 3 * nf, s, &Nc);
    P.Nc = Nc;
    DBuf<uint64_t> ukey;
    ukey.alloc(Nc, s);
    P.copy_vert.alloc(Nc, s);
    P.row_piece.alloc(Nc, s);
    { k_unique_compact<<<nblk(3 * nf), 256, 0, s>>>(ckey.p, flag.p, pos.p, 3 * nf, (uint64_t)nv, ukey.p,
                                                  P.copy_vert.p, P.row_piece.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    P.d_voff.alloc(K + 1, s);
    { k_segment_starts<<<nblk(Nc), 256, 0, s>>>(ukey.p, Nc, P.d_voff.p, 0, (uint64_t)nv); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaMemcpyAsync(P.d_voff.p + K, &P.Nc, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    P.voff.assign(K + 1, 0);
    PGCP_CUDA(cudaMemcpyAsync(P.voff.data(), P.d_voff.p, K * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PGCP_CUDA(cudaStreamSynchronize(s));
    P.voff[K] = Nc;
    P.foff[K] = nf;
    // ---- faces as copy rows; lowest-label copy of every vertex
    P.cF.alloc(3 * nf, s);
    P.first_copy.alloc(nv, s);
    { k_fill_i32<<<nblk(nv), 256, 0, s>>>(P.first_copy.p, nv, INT_MAX); ::pgcp::note_launch(); }
    { k_face_rows<<<nblk(nf), 256, 0, s>>>(P.F.p, forder.p, P.face_label.p, nf, ukey.p, P.d_voff.p,
                                         (uint64_t)nv, P.cF.p, P.first_copy.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    // ---- boundary half-edges
    const int64_t hcap = std::max<int64_t>(3 * nf, 16);
    DBuf<int4> he;
    DBuf<int32_t> hpiece;
    DBuf<unsigned long long> counter;
    he.alloc(hcap, s);
    hpiece.alloc(hcap, s);
    counter.alloc(1, s);
    counter.zero();
    { k_boundary_halfedges<<<nblk(3 * nf), 256, 0, s>>>(P.F.p, forder.p, P.face_label.p, P.cF.p, nf, keys.p, fa.p,
                                                      fb.p, cnt.p, mask, hcap, counter.p, he.p, hpiece.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    unsigned long long nh = 0;
    PGCP_CUDA(cudaMemcpyAsync(&nh, counter.p, sizeof(nh), cudaMemcpyDeviceToHost, s));
    PGCP_CUDA(cudaStreamSynchronize(s));
    std::vector<int4> h_he(nh);
    std::vector<int32_t> h_piece(nh);
    if (nh) {
        PGCP_CUDA(cudaMemcpyAsync(h_he.data(), he.p, nh * sizeof(int4), cudaMemcpyDeviceToHost, s));
        PGCP_CUDA(cudaMemcpyAsync(h_piece.data(), hpiece.p, nh * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    }
    PGCP_CUDA(cudaStreamSynchronize(s));
    // ---- loops (host): per piece, the half-edge leaving each boundary row (a
    // dense table over the piece's rows), walked from the smallest global id
    std::vector<int64_t> hoff(K + 1, 0);
    for (size_t i = 0; i < nh; ++i) ++hoff[h_piece[i] + 1];
    for (int64_t i = 0; i < K; ++i) hoff[i + 1] += hoff[i];
    std::vector<int4> hs(nh);
    {
        std::vector<int64_t> fill(hoff.begin(), hoff.end() - 1);
        for (size_t i = 0; i < nh; ++i) hs[fill[h_piece[i]]++] = h_he[i];
    }
    int64_t maxrows = 1;
    for (int64_t i = 0; i < K; ++i) maxrows = std::max<int64_t>(maxrows, P.voff[i + 1] - P.voff[i]);
    std::vector<int32_t> out_of(maxrows, -1);   // half-edge leaving a row (index into the piece's list)
    P.loff.assign(K + 1, 0);
    P.loop_rows.clear();
    P.loop_glob.clear();
    for (int64_t i = 0; i < K; ++i) {
        const int4* e = hs.data() + hoff[i];
        const int64_t ne = hoff[i + 1] - hoff[i];
        const int64_t r0 = P.voff[i];
        if (ne == 0) fail(PGCP_E_TOPOLOGY, "piece " + std::to_string(i) + " has no boundary (not a disk)");
        for (int64_t t = 0; t < ne; ++t) {
            if (e[t].x < r0 || e[t].x >= P.voff[i + 1]) {
                for (int64_t u = 0; u < t; ++u) out_of[e[u].x - r0] = -1;
                fail(PGCP_E_TOPOLOGY, "piece " + std::to_string(i) + ": boundary half-edge outside the piece");
            }
            int32_t& slot = out_of[e[t].x - r0];
            if (slot >= 0) {
                for (int64_t u = 0; u < t; ++u) out_of[e[u].x - r0] = -1;
                fail(PGCP_E_TOPOLOGY, "piece " + std::to_string(i) + " is pinched at vertex " + std::to_string(e[t].z));
            }
            slot = (int32_t)t;
        }
        auto find = [&](int row) -> int {
            if (row < r0 || row >= P.voff[i + 1]) return -1;
            return out_of[row - r0];
        };
        int start = 0;
        for (int64_t t = 1; t < ne; ++t)
            if (e[t].z < e[start].z) start = (int)t;
        int cur = start;
        size_t len = 0;
        bool broken = false;
        do {
            P.loop_rows.push_back(e[cur].x);
            P.loop_glob.push_back(e[cur].z);
            ++len;
            int nx = find(e[cur].y);
            if (nx < 0 || (int64_t)len > ne) {
                broken = true;
                break;
            }
            cur = nx;
        } while (cur != start);
        for (int64_t t = 0; t < ne; ++t) out_of[e[t].x - r0] = -1;
        if (broken) fail(PGCP_E_TOPOLOGY, "piece " + std::to_string(i) + ": broken boundary loop");
        if ((int64_t)len != ne) fail(PGCP_E_TOPOLOGY, "piece " + std::to_string(i) + " has more than one boundary loop");
        int64_t nvi = P.voff[i + 1] - P.voff[i], nfi = P.foff[i + 1] - P.foff[i];
        int64_t E = (3 * nfi + (int64_t)len) / 2;
        if ((3 * nfi + (int64_t)len) % 2 != 0 || nvi - E + nfi != 1)
            fail(PGCP_E_TOPOLOGY, "piece " + std::to_string(i) + " has Euler characteristic " +
                                      std::to_string(nvi - E + nfi) + ", not 1");
        P.loff[i + 1] = (int64_t)P.loop_rows.size();
    }
}

}  // namespace pgcp
