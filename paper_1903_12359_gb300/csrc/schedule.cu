// Host-side welding order and per-piece set-up (runs on small integer arrays).
//
// Welding order (the paper shows pieces joined one at a time, Fig. 7): per
// mesh, the component C starts as its lowest-label piece; each step joins the
// lowest-label piece S whose shared boundary with C is ONE contiguous run of
// >= 2 edges of C's loop and which touches C nowhere else, so C u S stays a
// disk.  On a closed surface the last piece shares its whole loop (closed
// weld, Section 4.4.2).
//
// Sequences: a = C's counter-clockwise loop rotated to start at the shared
// arc, b = S's loop reversed and rotated so that b_j = a_j for j <= k.
// Per piece: DNCP pins at loop positions 0 and floor(b/2); reference vertex =
// first interior vertex at or after local index floor(n/2), wrapping.
#include <cuda_runtime.h>

#include <algorithm>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "pgcp_internal.h"

namespace pgcp {

namespace {

inline uint64_t dkey(int32_t u, int32_t v) { return ((uint64_t)(uint32_t)u << 32) | (uint32_t)v; }

std::vector<int32_t> rotate_canonical(const std::vector<int32_t>& loop) {
    size_t i = std::min_element(loop.begin(), loop.end()) - loop.begin();
    std::vector<int32_t> out(loop.begin() + i, loop.end());
    out.insert(out.end(), loop.begin(), loop.begin() + i);
    return out;
}

__global__ void k_loop_setup(const int32_t* __restrict__ loop_rows, const int64_t* __restrict__ loff, int32_t K,
                             int64_t nloop, const int32_t* __restrict__ lp, int2* __restrict__ nb,
                             uint8_t* __restrict__ is_bnd) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nloop) return;
    int piece = lp[t];
    int64_t a = loff[piece], b = loff[piece + 1];
    int64_t prev = (t == a) ? b - 1 : t - 1;
    int64_t next = (t + 1 == b) ? a : t + 1;
    int r = loop_rows[t];
    nb[r] = make_int2(loop_rows[prev], loop_rows[next]);
    is_bnd[r] = 1;
}

}  // namespace

void build_schedule(pgcp_ctx* ctx, Part& P) {
    cudaStream_t s = ctx->stream;
    const int32_t K = P.K;
    auto loop_of = [&](int32_t i) {
        return std::vector<int32_t>(P.loop_glob.begin() + P.loff[i], P.loop_glob.begin() + P.loff[i + 1]);
    };
    // ---- per piece: pins and reference vertex
    P.pin0.assign(K, 0);
    P.pin1.assign(K, 0);
    P.ref.assign(K, -1);
    for (int32_t i = 0; i < K; ++i) {
        int64_t b = P.loff[i + 1] - P.loff[i];
        P.pin0[i] = P.loop_rows[P.loff[i]];
        P.pin1[i] = P.loop_rows[P.loff[i] + b / 2];
        int64_t n = P.voff[i + 1] - P.voff[i];
        std::unordered_set<int64_t> bnd(P.loop_rows.begin() + P.loff[i], P.loop_rows.begin() + P.loff[i + 1]);
        for (int64_t t = 0; t < n; ++t) {
            int64_t r = P.voff[i] + (n / 2 + t) % n;
            if (!bnd.count(r)) {
                P.ref[i] = r;
                break;
            }
        }
    }
    // ---- device loop arrays, (prev, next) of boundary rows
    const int64_t nloop = (int64_t)P.loop_rows.size();
    std::vector<int32_t> rows32(P.loop_rows.begin(), P.loop_rows.end()), lp(nloop);
    for (int32_t i = 0; i < K; ++i)
        for (int64_t t = P.loff[i]; t < P.loff[i + 1]; ++t) lp[t] = i;
    P.d_loff.alloc(K + 1, s);
    P.d_loop_rows.alloc(nloop, s);
    P.d_loop_glob.alloc(nloop, s);
    DBuf<int32_t> d_lp;
    d_lp.alloc(nloop, s);
    PGCP_CUDA(cudaMemcpyAsync(P.d_loff.p, P.loff.data(), (K + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    PGCP_CUDA(cudaMemcpyAsync(P.d_loop_rows.p, rows32.data(), nloop * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    PGCP_CUDA(cudaMemcpyAsync(P.d_loop_glob.p, P.loop_glob.data(), nloop * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    PGCP_CUDA(cudaMemcpyAsync(d_lp.p, lp.data(), nloop * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    P.nb.alloc(P.Nc, s);
    P.is_bnd.alloc(P.Nc, s);
    PGCP_CUDA(cudaMemsetAsync(P.nb.p, 0xff, P.Nc * sizeof(int2), s));
    P.is_bnd.zero();
    { k_loop_setup<<<(unsigned)std::max<int64_t>(1, ceil_div(nloop, 256)), 256, 0, s>>>(
        P.d_loop_rows.p, P.d_loff.p, K, nloop, d_lp.p, P.nb.p, P.is_bnd.p); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    PGCP_CUDA(cudaStreamSynchronize(s));   // host vectors above go out of scope

    // ---- welding order, per mesh
    P.welds.clear();
    for (size_t mi = 0; mi < P.meshes.size(); ++mi) {
        const MeshInfo& M = P.meshes[mi];
        if (M.npiece <= 1) {
            if (P.closed) fail(PGCP_E_TOPOLOGY, "a closed surface needs at least two pieces");
            continue;
        }
        std::vector<int32_t> C_loop = loop_of(M.piece0);
        std::vector<int32_t> members = {M.piece0};
        std::vector<int32_t> remaining;
        for (int32_t i = M.piece0 + 1; i < M.piece0 + M.npiece; ++i) remaining.push_back(i);
        bool first = true;
        while (!remaining.empty()) {
            bool found = false;
            WeldPlan W;
            for (int32_t sp : remaining) {
                std::vector<int32_t> S_loop = loop_of(sp);
                std::unordered_set<uint64_t> s_edges;
                for (size_t t = 0; t < S_loop.size(); ++t) s_edges.insert(dkey(S_loop[t], S_loop[(t + 1) % S_loop.size()]));
                const size_t m1 = C_loop.size();
                std::vector<char> shared(m1);
                bool any = false, all = true;
                for (size_t t = 0; t < m1; ++t) {
                    shared[t] = s_edges.count(dkey(C_loop[(t + 1) % m1], C_loop[t])) ? 1 : 0;
                    any |= shared[t];
                    all &= shared[t] != 0;
                }
                if (!any) continue;
                std::vector<int32_t> rb(S_loop.rbegin(), S_loop.rend());
                if (all) {
                    if (!(P.closed && remaining.size() == 1 && S_loop.size() == m1)) continue;
                    size_t j = std::find(rb.begin(), rb.end(), C_loop[0]) - rb.begin();
                    std::vector<int32_t> b(rb.begin() + j, rb.end());
                    b.insert(b.end(), rb.begin(), rb.begin() + j);
                    if (b != C_loop) continue;
                    W.closed = 1;
                    W.k = (int32_t)m1 - 1;
                    W.a_glob = C_loop;
                    W.b_rows.clear();
                    W.new_loop.clear();
                    std::vector<int32_t> bg = b;
                    W.piece = sp;
                    // b rows
                    std::unordered_map<int32_t, int64_t> srow;
                    for (int64_t t = P.loff[sp]; t < P.loff[sp + 1]; ++t) srow[P.loop_glob[t]] = P.loop_rows[t];
                    for (int32_t g : bg) W.b_rows.push_back(srow.at(g));
                    found = true;
                    break;
                }
                std::vector<size_t> starts;
                for (size_t t = 0; t < m1; ++t)
                    if (shared[t] && !shared[(t + m1 - 1) % m1]) starts.push_back(t);
                if (starts.size() != 1) continue;
                size_t i0 = starts[0];
                int32_t k = 0;
                while (k < (int32_t)m1 && shared[(i0 + k) % m1]) ++k;
                if (k < 2) continue;
                std::vector<int32_t> a(C_loop.begin() + i0, C_loop.end());
                a.insert(a.end(), C_loop.begin(), C_loop.begin() + i0);
                std::unordered_set<int32_t> arcv(a.begin(), a.begin() + k + 1);
                std::unordered_set<int32_t> cset(C_loop.begin(), C_loop.end());
                bool touch = false;
                for (int32_t g : S_loop)
                    if (cset.count(g) && !arcv.count(g)) touch = true;
                if (touch) continue;
                size_t j = std::find(rb.begin(), rb.end(), a[0]) - rb.begin();
                std::vector<int32_t> b(rb.begin() + j, rb.end());
                b.insert(b.end(), rb.begin(), rb.begin() + j);
                if (!std::equal(a.begin(), a.begin() + k + 1, b.begin())) continue;
                std::vector<int32_t> nl(a.begin() + k, a.end());
                nl.push_back(a[0]);
                for (size_t t = b.size(); t-- > (size_t)k + 1;) nl.push_back(b[t]);
                W.closed = 0;
                W.k = k;
                W.piece = sp;
                W.a_glob = a;
                W.new_loop = rotate_canonical(nl);
                std::unordered_map<int32_t, int64_t> srow;
                for (int64_t t = P.loff[sp]; t < P.loff[sp + 1]; ++t) srow[P.loop_glob[t]] = P.loop_rows[t];
                W.b_rows.clear();
                for (int32_t g : b) W.b_rows.push_back(srow.at(g));
                found = true;
                break;
            }
            if (!found) fail(PGCP_E_SCHEDULE, "mesh " + std::to_string(mi) +
                                                   ": no piece shares one contiguous arc with the welded component");
            W.mesh = (int32_t)mi;
            W.first = first ? 1 : 0;
            W.members = members;
            std::sort(W.members.begin(), W.members.end());
            // a rows: copy in the lowest-label member whose loop holds the vertex
            std::unordered_map<int32_t, int64_t> crow;
            for (int32_t pc : W.members)
                for (int64_t t = P.loff[pc]; t < P.loff[pc + 1]; ++t) crow.emplace(P.loop_glob[t], P.loop_rows[t]);
            W.a_rows.clear();
            for (int32_t g : W.a_glob) W.a_rows.push_back(crow.at(g));
            members.push_back(W.piece);
            remaining.erase(std::find(remaining.begin(), remaining.end(), W.piece));
            if (!W.closed) C_loop = W.new_loop;
            P.welds.push_back(std::move(W));
            first = false;
        }
        if (P.closed && !P.welds.back().closed)
            fail(PGCP_E_SCHEDULE, "closed surface did not end with a closed weld");
    }
}

}  // namespace pgcp
