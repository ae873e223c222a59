// Host-side welding order and per-piece set-up (runs on small integer arrays).
//
// Welding order: Algorithm 2 joins any two disks that share one boundary arc.
// Per mesh, components start as the pieces (ordered by lowest label) and are
// paired level by level: every unpaired component, in that order, is paired
// with the first later unpaired one whose loop shares ONE contiguous run of
// >= 2 edges with it and touches it nowhere else (so the union stays a disk);
// the earlier one is A, the later one B.  A piece's boundary thus passes
// through about log2 K welds (joining one piece at a time composes K of them,
// and the crowded boundary loses the arc order in FP64).  On a closed surface
// the last two components share their whole loops (closed weld, Section 4.4.2).
//
// Sequences: a = A's counter-clockwise loop rotated to start at the shared
// arc, b = B's loop reversed and rotated so that b_j = a_j for j <= k; each
// point is read from the copy in the lowest-label piece of its side.
// Per piece: DNCP pins at loop positions 0 and floor(b/2); reference vertex =
// first interior vertex at or after local index floor(n/2), wrapping.
#include <cuda_runtime.h>

#include <algorithm>
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
    {
        std::vector<char> bnd(P.Nc, 0);   // boundary rows
        for (int64_t r : P.loop_rows) bnd[r] = 1;
        for (int32_t i = 0; i < K; ++i) {
            int64_t b = P.loff[i + 1] - P.loff[i];
            P.pin0[i] = P.loop_rows[P.loff[i]];
            P.pin1[i] = P.loop_rows[P.loff[i] + b / 2];
            int64_t n = P.voff[i + 1] - P.voff[i];
            for (int64_t t = 0; t < n; ++t) {
                int64_t r = P.voff[i] + (n / 2 + t) % n;
                if (!bnd[r]) {
                    P.ref[i] = r;
                    break;
                }
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
    struct Comp {
        std::vector<int32_t> members;
        std::vector<int32_t> loop;
        int32_t single;
    };
    // Dense per-mesh tables over the mesh's vertex range [base, base + nv),
    // reused from mesh to mesh and cleared by epoch stamps instead of hashing:
    //   cp_off / cp: (piece, row) of every loop copy of a vertex, pieces ascending;
    //   st_b / nx_b: B's loop vertices and their successors (directed edges of B);
    //   st_a, st_arc: A's loop vertices, the shared arc's vertices.
    int64_t maxnv = 1;
    for (const MeshInfo& M : P.meshes) maxnv = std::max<int64_t>(maxnv, M.nv);
    std::vector<int64_t> cp_off(maxnv + 1);
    std::vector<std::pair<int32_t, int64_t>> cp;
    std::vector<int32_t> st_b(maxnv, 0), nx_b(maxnv, 0), st_a(maxnv, 0), st_arc(maxnv, 0), mark(K, 0);
    int32_t epoch = 0;
    int64_t base = 0;
    // copy row of each loop vertex in the lowest-label piece of `pieces` holding it
    auto rows_of = [&](const std::vector<int32_t>& pieces, const std::vector<int32_t>& ids) {
        ++epoch;
        for (int32_t pc : pieces) mark[pc] = epoch;
        std::vector<int64_t> out;
        out.reserve(ids.size());
        for (int32_t g : ids) {
            int64_t r = -1;
            for (int64_t c = cp_off[g - base]; c < cp_off[g - base + 1]; ++c)
                if (mark[cp[c].first] == epoch) {
                    r = cp[c].second;
                    break;
                }
            if (r < 0) fail(PGCP_E_SCHEDULE, "welding sequence vertex " + std::to_string(g) + " is on no member loop");
            out.push_back(r);
        }
        return out;
    };
    // the weld of B onto A, if their loops share one contiguous arc (or, for the
    // closed weld, the whole loop) and touch nowhere else
    auto pair_weld = [&](const Comp& A, const Comp& B, bool closed_final, WeldPlan& W) -> bool {
        const std::vector<int32_t>& A_loop = A.loop;
        const std::vector<int32_t>& B_loop = B.loop;
        ++epoch;
        for (size_t t = 0; t < B_loop.size(); ++t) {   // directed edges of B: g -> nx_b[g]
            st_b[B_loop[t] - base] = epoch;
            nx_b[B_loop[t] - base] = B_loop[(t + 1) % B_loop.size()];
        }
        auto b_edge = [&](int32_t u, int32_t v) { return st_b[u - base] == epoch && nx_b[u - base] == v; };
        const size_t m1 = A_loop.size();
        std::vector<char> shared(m1);
        bool any = false, all = true;
        for (size_t t = 0; t < m1; ++t) {
            shared[t] = b_edge(A_loop[(t + 1) % m1], A_loop[t]) ? 1 : 0;
            any |= shared[t];
            all &= shared[t] != 0;
        }
        if (!any) return false;
        std::vector<int32_t> rb(B_loop.rbegin(), B_loop.rend());
        W.piece = B.members.front();
        W.members = A.members;
        W.b_members = B.members;
        W.a_single = A.single;
        W.b_single = B.single;
        if (all) {
            if (!(closed_final && B_loop.size() == m1)) return false;
            size_t j = std::find(rb.begin(), rb.end(), A_loop[0]) - rb.begin();
            std::vector<int32_t> b(rb.begin() + j, rb.end());
            b.insert(b.end(), rb.begin(), rb.begin() + j);
            if (b != A_loop) return false;
            W.closed = 1;
            W.k = (int32_t)m1 - 1;
            W.a_glob = A_loop;
            W.new_loop.clear();
            W.b_rows = rows_of(B.members, b);
            return true;
        }
        std::vector<size_t> starts;
        for (size_t t = 0; t < m1; ++t)
            if (shared[t] && !shared[(t + m1 - 1) % m1]) starts.push_back(t);
        if (starts.size() != 1) return false;
        const size_t i0 = starts[0];
        int32_t k = 0;
        while (k < (int32_t)m1 && shared[(i0 + k) % m1]) ++k;
        if (k < 2) return false;
        std::vector<int32_t> a(A_loop.begin() + i0, A_loop.end());
        a.insert(a.end(), A_loop.begin(), A_loop.begin() + i0);
        for (int32_t g : A_loop) st_a[g - base] = epoch;
        for (int32_t t = 0; t <= k; ++t) st_arc[a[t] - base] = epoch;
        for (int32_t g : B_loop)   // B touches A only along the arc
            if (st_a[g - base] == epoch && st_arc[g - base] != epoch) return false;
        size_t j = std::find(rb.begin(), rb.end(), a[0]) - rb.begin();
        std::vector<int32_t> b(rb.begin() + j, rb.end());
        b.insert(b.end(), rb.begin(), rb.begin() + j);
        if (!std::equal(a.begin(), a.begin() + k + 1, b.begin())) return false;
        std::vector<int32_t> nl(a.begin() + k, a.end());
        nl.push_back(a[0]);
        for (size_t t = b.size(); t-- > (size_t)k + 1;) nl.push_back(b[t]);
        W.closed = 0;
        W.k = k;
        W.a_glob = a;
        W.new_loop = rotate_canonical(nl);
        W.b_rows = rows_of(B.members, b);
        return true;
    };
    for (size_t mi = 0; mi < P.meshes.size(); ++mi) {
        const MeshInfo& M = P.meshes[mi];
        if (M.npiece <= 1) {
            if (P.closed) fail(PGCP_E_TOPOLOGY, "a closed surface needs at least two pieces");
            continue;
        }
        base = M.v0;
        std::fill(cp_off.begin(), cp_off.begin() + M.nv + 1, 0);
        for (int32_t pc = M.piece0; pc < M.piece0 + M.npiece; ++pc)
            for (int64_t t = P.loff[pc]; t < P.loff[pc + 1]; ++t) ++cp_off[P.loop_glob[t] - base + 1];
        for (int64_t v = 0; v < M.nv; ++v) cp_off[v + 1] += cp_off[v];
        cp.resize(cp_off[M.nv]);
        {
            std::vector<int64_t> fill(cp_off.begin(), cp_off.begin() + M.nv);
            for (int32_t pc = M.piece0; pc < M.piece0 + M.npiece; ++pc)   // pieces ascending
                for (int64_t t = P.loff[pc]; t < P.loff[pc + 1]; ++t)
                    cp[fill[P.loop_glob[t] - base]++] = {pc, P.loop_rows[t]};
        }
        std::vector<Comp> comps;
        for (int32_t i = M.piece0; i < M.piece0 + M.npiece; ++i) comps.push_back(Comp{{i}, loop_of(i), 1});
        int32_t level = 0;
        while (comps.size() > 1) {
            const bool final2 = P.closed && comps.size() == 2;
            // Components that share a loop edge (pair_weld fails for all others,
            // so scanning only these keeps the pairing order): every loop edge,
            // undirected, with its component, sorted by edge.
            std::vector<std::pair<uint64_t, int32_t>> ec;
            for (size_t c = 0; c < comps.size(); ++c) {
                const std::vector<int32_t>& L = comps[c].loop;
                for (size_t t = 0; t < L.size(); ++t) {
                    const int32_t u = L[t], v = L[(t + 1) % L.size()];
                    ec.emplace_back(dkey(std::min(u, v), std::max(u, v)), (int32_t)c);
                }
            }
            std::sort(ec.begin(), ec.end());
            std::vector<std::vector<int32_t>> nbr(comps.size());
            for (size_t a = 0; a < ec.size();) {
                size_t b = a + 1;
                while (b < ec.size() && ec[b].first == ec[a].first) ++b;
                for (size_t x = a; x < b; ++x)
                    for (size_t y = a; y < b; ++y)
                        if (ec[x].second != ec[y].second) nbr[ec[x].second].push_back(ec[y].second);
                a = b;
            }
            for (auto& v : nbr) {
                std::sort(v.begin(), v.end());
                v.erase(std::unique(v.begin(), v.end()), v.end());
            }
            std::vector<char> used(comps.size(), 0);
            std::vector<Comp> next;
            for (size_t i = 0; i < comps.size(); ++i) {
                if (used[i]) continue;
                for (int32_t jj : nbr[i]) {
                    const size_t j = (size_t)jj;
                    if (j <= i || used[j]) continue;
                    WeldPlan W;
                    if (!pair_weld(comps[i], comps[j], final2, W)) continue;
                    W.mesh = (int32_t)mi;
                    W.level = level;
                    W.a_rows = rows_of(W.members, W.a_glob);
                    std::vector<int32_t> mem = comps[i].members;
                    mem.insert(mem.end(), comps[j].members.begin(), comps[j].members.end());
                    std::sort(mem.begin(), mem.end());
                    next.push_back(Comp{mem, W.new_loop, 0});
                    P.welds.push_back(std::move(W));
                    used[i] = used[j] = 1;
                    break;
                }
            }
            if (next.empty())
                fail(PGCP_E_SCHEDULE, "mesh " + std::to_string(mi) + ": no two components share one contiguous arc");
            for (size_t i = 0; i < comps.size(); ++i)
                if (!used[i]) next.push_back(comps[i]);
            std::sort(next.begin(), next.end(),
                      [](const Comp& x, const Comp& y) { return x.members.front() < y.members.front(); });
            comps.swap(next);
            ++level;
        }
        if (P.closed && !P.welds.back().closed)
            fail(PGCP_E_SCHEDULE, "closed surface did not end with a closed weld");
    }
}

}  // namespace pgcp
