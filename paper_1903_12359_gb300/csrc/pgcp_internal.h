// Internal declarations of the PGCP CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pgcp.h"

namespace pgcp {

// ------------------------------------------------------------------ errors

struct Error {
    pgcp_status code;
    std::string msg;
};

// Thrown inside the library, turned into a status at the C ABI boundary.
[[noreturn]] void fail(pgcp_status code, const std::string& msg);
// Counts every kernel launch of the library (pgcp_launch_count()).
void note_launch();
// Counts every device allocation of the library (pgcp_alloc_count()).
void note_alloc();
void check_cuda(cudaError_t e, const char* what);
#define PGCP_CUDA(call) ::pgcp::check_cuda((call), #call)

// Device-side error flags (bit set by kernels, read back by the host).
enum DevErr : uint32_t {
    DE_NONMANIFOLD = 1u << 0,
    DE_ORIENT = 1u << 1,
    DE_CUT_MISSING = 1u << 2,
    DE_DEGENERATE = 1u << 3,
    DE_VALENCE = 1u << 4,
    DE_NUMERIC = 1u << 5,
    DE_UNION_LIMIT = 1u << 6,
    DE_WELD_DOMAIN = 1u << 7,
    DE_HASH_FULL = 1u << 8,
    DE_TIMEOUT = 1u << 9,      // a bounded wait in a kernel gave up
};

// Two CUDA events, destroyed on scope exit (also when a failing call throws).
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    EventPair() {
        PGCP_CUDA(cudaEventCreate(&a));
        const cudaError_t e = cudaEventCreate(&b);
        if (e != cudaSuccess) {
            cudaEventDestroy(a);
            a = nullptr;
            check_cuda(e, "cudaEventCreate");
        }
    }
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    EventPair(const EventPair&) = delete;
    EventPair& operator=(const EventPair&) = delete;
};

// ------------------------------------------------------------------ device memory

// Stream-ordered device buffer (cudaMallocAsync / cudaFreeAsync on one stream).
template <typename T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept { *this = std::move(o); }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n; s = o.s;
            o.p = nullptr; o.n = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count, cudaStream_t stream) {
        release();
        s = stream;
        n = count;
        if (count == 0) return;
        cudaError_t e = cudaMallocAsync((void**)&p, count * sizeof(T), stream);
        note_alloc();
        if (e != cudaSuccess) {
            p = nullptr;
            n = 0;
            if (e == cudaErrorMemoryAllocation) fail(PGCP_E_OOM, "device allocation failed");
            check_cuda(e, "cudaMallocAsync");
        }
    }
    void zero() {
        if (n) PGCP_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    }
};

// ------------------------------------------------------------------ welding records

// One elementary map of a welding chain (layout shared by the phase-1 builder
// and the phase-2 appliers).
enum RecKind : int32_t { R_SQRT_RATIO = 0, R_OPEN = 1, R_MOB_POLE = 2, R_CLOSE = 3, R_POLE_SQ = 4, R_MOBIUS = 5 };

struct __align__(16) Rec {
    int32_t kind;
    int32_t pad;
    double branch;
    double p[8];
};

// ------------------------------------------------------------------ part (device state)

struct WeldPlan {             // one weld of component B onto component A, host description
    int32_t mesh;
    int32_t piece;            // lowest label of B
    int32_t k;                // shared edges
    int32_t closed;           // closed weld (sphere)
    int32_t level;            // welds of one level join disjoint components
    int32_t a_single, b_single;     // the side is one unwelded piece (reference 0, else -1)
    std::vector<int32_t> members;   // pieces of A (ascending)
    std::vector<int32_t> b_members; // pieces of B (ascending)
    std::vector<int64_t> a_rows;    // copy rows of a_0..a_m
    std::vector<int64_t> b_rows;    // copy rows of b_0..b_n
    std::vector<int32_t> a_glob;
    std::vector<int32_t> new_loop;  // global ids of the loop of A u B (empty if closed)
};

struct MeshInfo {
    int64_t v0, nv, f0, nf;   // offsets into the concatenated vertex / face arrays
    int32_t piece0, npiece;   // pieces of this mesh: [piece0, piece0 + npiece)
};

struct Part {
    // mesh (concatenated over the batch)
    int64_t nv = 0, nf = 0;
    int32_t closed = 0;
    std::vector<MeshInfo> meshes;
    DBuf<double> V;           // [nv*3]
    DBuf<int32_t> F;          // [nf*3]
    // partition
    int32_t K = 0;
    DBuf<int32_t> face_label; // [nf]
    std::vector<int64_t> voff, foff;   // host copies [K+1]
    DBuf<int64_t> d_voff;     // [K+1]
    DBuf<int32_t> copy_vert;  // [Nc] global vertex of each copy (row)
    DBuf<int32_t> row_piece;  // [Nc]
    DBuf<int32_t> cF;         // [nf*3] faces in piece order, as copy rows
    DBuf<int32_t> first_copy; // [nv] copy of the lowest-label piece holding v
    int64_t Nc = 0;
    // boundary loops
    std::vector<int64_t> loff;         // [K+1]
    std::vector<int64_t> loop_rows;    // copy rows, ccw
    std::vector<int32_t> loop_glob;    // global ids
    DBuf<int64_t> d_loff;
    DBuf<int32_t> d_loop_rows;
    DBuf<int32_t> d_loop_glob;
    DBuf<int2> nb;            // [Nc] (prev, next) loop rows for boundary rows, (-1,-1) inside
    DBuf<uint8_t> is_bnd;     // [Nc]
    std::vector<int64_t> pin0, pin1, ref;   // per piece: copy rows
    // schedule
    std::vector<WeldPlan> welds;
    // CSR (block diagonal over pieces; columns are global rows)
    DBuf<int32_t> row_ptr;    // [Nc+1] (int32: nnz < 2^31)
    DBuf<int32_t> col;
    DBuf<double> val64;
    DBuf<float> val32;
    DBuf<double> diag64;
    int64_t nnz = 0;
    DBuf<int64_t> inc_off, rp64;   // corner incidence of every row and the CSR row offsets (int64)
    DBuf<int32_t> inc;
    // coordinates
    DBuf<double2> local;      // DNCP (local frame)
    DBuf<double2> welded;     // FP64 welded coords (boundary rows exact; interior = weld map)
    DBuf<double2> final;      // final solve
    std::vector<uint8_t> wchart;   // [K] piece held in the chart w = 1/z (sphere)
    std::vector<int32_t> mesh_status;   // [meshes] PGCP_OK, or PGCP_E_NUMERIC for a dropped mesh of a batch
    DBuf<uint8_t> d_wchart;
    int32_t have_local = 0, have_weld = 0, have_final = 0;
    std::vector<uint8_t> own;   // [K] pieces this part solves (empty: all); the rest are another rank's
    pgcp_stats stats{};
};

}  // namespace pgcp

// ------------------------------------------------------------------ context

struct pgcp_gnn {
    int device = 0;
    pgcp::DBuf<float> theta, grad, m, v;   // FP32 parameters, gradient, Adam moments
    pgcp::DBuf<uint16_t> bf;               // bf16 weight copies laid out for the GEMMs
    int64_t step = 0;
};

struct pgcp_ctx {
    pgcp_options opt;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    std::string last_error;
    pgcp::DBuf<uint32_t> err;        // device error flags
    pgcp_gnn* gnn = nullptr;         // network for warm_start = PGCP_WARM_LEARNED (not owned)
};

struct pgcp_part {
    pgcp::Part p;
};

namespace pgcp {

// ------------------------------------------------------------------ primitives (primitives.cu)

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s, int64_t* total_host);
void exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s, int64_t* total_host);
// Stable LSD radix sort of (key, value) pairs by the low `bits` bits of key.
void radix_sort_pairs(uint64_t* keys, int32_t* vals, int64_t n, int bits, cudaStream_t s);
uint32_t read_errors(pgcp_ctx* ctx);
// The same sort and scan on caller-provided device workspace (no allocation).
int64_t sort_ws_counts(int64_t n);   // int64 entries needed for `counts` and for `offs`
void scan_noalloc(const int64_t* in, int64_t* out, int64_t n, int64_t* ws, int64_t ws_len, cudaStream_t s);
void radix_sort_pairs_noalloc(uint64_t* keys, int32_t* vals, int64_t n, int bits, cudaStream_t s, uint64_t* k2,
                              int32_t* v2, int64_t* counts, int64_t* offs, int64_t* scan_ws, int64_t scan_ws_len);

// ------------------------------------------------------------------ stages

struct SolveResult {
    int iters = 0;        // PCG iterations (summed over refinement steps)
    int refine = 0;       // outer refinement steps
    double relres = 0.0;  // max true FP64 relative residual over pieces and coordinates
};
// Batched PCG on all pieces; x holds fixed values and the initial guess.
SolveResult pcg_solve(pgcp_ctx* ctx, Part& P, int dncp, const uint8_t* fixed, double2* x);

// Run-based PCG (pcg_df.cu): the symmetrically Jacobi-scaled system with
// fixed rows and columns dropped, its row runs and its work vectors, in
// double-float (f32 = 0) or FP32 (f32 = 1) arithmetic.
struct DfRun {
    int32_t seg, lo, hi, frows;
    int32_t fnnz, pad0, pad1, pad2;
};
struct DfSystem {
    int64_t n = 0, nnz = 0;
    int dncp = 0, f32 = 0, grid = 0, per_sm = 0, minb = 4;
    int32_t nruns = 0;
    int64_t runs_cap = 0;      // capacity of runs (rebuilt runs of a chunked solve fit)
    int64_t covered = 0;       // rows the current runs cover
    DBuf<int32_t> rp, col;
    DBuf<unsigned char> val;   // nnz scalars (float2 or float)
    DBuf<double> sc;           // 1 / sqrt(diag), 0 at fixed rows
    DBuf<float> dgn;           // diag, 0 at fixed rows
    DBuf<DfRun> runs;
    DBuf<int32_t> run_off;
    DBuf<unsigned char> x, r, p, q;   // n row pairs (float4 or float2)
    DBuf<unsigned char> r1, w0, w1, s1;   // single-reduction schedule only
    DBuf<double> RR, RD, PQ, THR, DL;
    DBuf<double> RRP;                   // [2 nseg] each piece's <r, z> of its last active step
    DBuf<unsigned int> ACT;
    DBuf<int32_t> out_it;
    DBuf<unsigned long long> work;
    // dynamic schedule: chunks inside pieces, per-piece chunk counts, counters
    int sched = 1, dyn_grid = 0, rr_grid = 0;   // 1 static runs, 2 dynamic, 3 round-robin, 4 single-reduction
    int32_t nchunks = 0;
    DBuf<DfRun> chunks;
    DBuf<int32_t> nch;
    DBuf<unsigned int> CTR, CNTB, CNTA, DONEF;
    DBuf<double> ALPHA, BETA;
    // deterministic mode: per-run partial sums and converged flags, run range per piece
    int det = 0;
    DBuf<int32_t> prun, RDONE;
    DBuf<double> PRR, PRD, PPQ, CRR;
    // multilevel preconditioner (pcg_ml.cu): nested row blocks of every piece,
    // all levels concatenated; block b of level l is entry ml_lofs[l] + b
    int ml = 0, ml_nl = 0, ml_per_sm = 0;
    std::vector<int32_t> ml_bofs_h;     // [ML_MAXL][K+1] first block of each piece per level
    int64_t ml_lofs[16] = {0};          // [ML_MAXL+1]
    int64_t ml_tofs[16] = {0};          // [ML_MAXL+1] first packed-factor entry of each level
    double ml_row_bytes = 0.0;          // preconditioner table bytes per row and iteration
    int k_last = 0;                     // iteration index where the last solve stopped
    bool resumable = false;             // a solve ran: the next one may continue it
    DBuf<int32_t> ml_bofs, ml_ltop, ml_pvoff;
    DBuf<float> ml_xr;                  // [3n] vertex positions in their piece's frame
    DBuf<float4> ml_geo;                // per block: centroid, 1 / RMS radius
    DBuf<float> ml_T;                   // packed upper-triangular factors
    DBuf<uint8_t> ml_sep;               // per block: 1 when x and y decouple (T = diag(Tx, Tx))
    DBuf<float> ml_M;                   // [2][blocks][20] residual moments (iteration parity)
    DBuf<unsigned char> z;              // preconditioned residual (same layout as r)
};
// Multilevel preconditioner constants: a block of level l holds 16 * 4^l rows.
constexpr int ML_MAXL = 10;
constexpr int ML_NM = 20;               // moments per block: 10 monomials x (x, y)
constexpr int ML_SEG = 4096;            // longest run of the preconditioned kernel (rows)
void df_build(pgcp_ctx* ctx, Part& P, int dncp, const uint8_t* fixed, int f32, DfSystem& D);
// Row runs of the persistent grid over the active pieces (all when active is
// null): `grid` near-equal ranges, cut at piece boundaries; with align > 1 every
// cut inside a piece falls on a multiple of `align` rows from the piece's first
// row, and with maxlen > 0 no run is longer than maxlen.  Returns rows covered.
int64_t make_runs(const std::vector<int64_t>& voff, const std::vector<uint8_t>* active, int grid,
                  std::vector<DfRun>& runs, std::vector<int32_t>& roff, int align = 1, int maxlen = 0);
// Multilevel preconditioner of a double-float DNCP system (pcg_ml.cu): block
// tables and factors, after df_build has made the scaled matrix.
void ml_build(pgcp_ctx* ctx, Part& P, const uint8_t* fixed, DfSystem& D);
// One persistent launch of the preconditioned kernel over iterations k0 .. cap-1.
void ml_launch(pgcp_ctx* ctx, Part& P, DfSystem& D, int k0, int cap, bool resume);
// One inner solve of A d = r64 (thresholds on the unscaled <r, r> per piece
// and coordinate); adds d to x; returns the iterations run.
int df_solve(pgcp_ctx* ctx, Part& P, DfSystem& D, const double2* r64, double2* x, const std::vector<double>& thr,
             int max_iters, bool resume);

void build_partition(pgcp_ctx* ctx, Part& P, const int32_t* d_labels_or_null, const int32_t* d_cut, int64_t n_cut);
void build_schedule(pgcp_ctx* ctx, Part& P);
void assemble_laplacian(pgcp_ctx* ctx, Part& P);
// Values of another linear-element matrix on the Laplacian's pattern: fw[3 f + c]
// is the weight of the edge opposite corner c of face f (piece order); entries
// -sum of the weights on each edge, diagonal their row sums.
void assemble_values(pgcp_ctx* ctx, Part& P, const double* fw, double* val64, float* val32, double* diag64);
// Fold-over fix (qcfix.cu) on a planar map U [nv*2] (device, in and out).
void fix_folds(pgcp_ctx* ctx, Part& P, double* U, pgcp_fold_report* rep);
void solve_dncp(pgcp_ctx* ctx, Part& P);
void run_welds(pgcp_ctx* ctx, Part& P);
void solve_final(pgcp_ctx* ctx, Part& P, double* out, int host_out);
// Boundary exchange of a sharded run: coordinates at every loop position
// (which: 0 local map, 1 welded map), out / in device [n_loop * 2].
void part_get_boundary(pgcp_ctx* ctx, const Part& P, int which, double* out);
void part_set_boundary(pgcp_ctx* ctx, Part& P, int which, const double* in);
void compute_metrics(pgcp_ctx* ctx, const Part& P, const double* U, pgcp_distortion* met);
// Same statistics on a fixed device-side scratch array; no allocation.
void compute_metrics_noalloc(pgcp_ctx* ctx, const Part& P, const double* U, pgcp_distortion* met);
int64_t metrics_noalloc_max_faces();
// Area distortion and the Mobius area step (Section 6.2), one result per mesh.
void area_distortion(pgcp_ctx* ctx, const Part& P, const double* U, double* mean_abs);
void area_mobius(pgcp_ctx* ctx, const Part& P, double* U, int variant, pgcp_area_result* out);

// BF16 tensor-core GEMM (gemm_tc.cu): C = epi(A . Bt^T), A [M x K], Bt [N x K],
// both bf16 with K contiguous.  epi 0: store FP32; 1: + bias, ReLU, store bf16
// (and the pre-activation to Z if given); 2: + bias, store FP32.
void gemm_bf16_tc(cudaStream_t s, int epi, int N, int K, const void* A, int64_t lda, const void* Bt, int64_t M,
                  const float* bias, void* C, int64_t ldc, float* Z, int64_t ldz, uint32_t* err);
uint64_t umma_desc_host(uint32_t saddr, uint32_t lbo, uint32_t sbo);

// Learned warm start (mpnn.cu)
int64_t gnn_num_params();
void gnn_init(pgcp_ctx* ctx, pgcp_gnn* G, const float* host_params);
void gnn_set(pgcp_ctx* ctx, pgcp_gnn* G, const float* host_params);
void gnn_get(pgcp_ctx* ctx, const pgcp_gnn* G, float* host_params);
void gnn_inputs(pgcp_ctx* ctx, Part& P, float* feat, float* target, float* sigma);
double gnn_grad(pgcp_ctx* ctx, pgcp_gnn* G, Part& P, int update, float lr);
void gnn_predict(pgcp_ctx* ctx, const pgcp_gnn* G, Part& P, double2* x);
int learned_start(pgcp_ctx* ctx, Part& P, double2* x);
uint32_t umma_idesc_host(int m, int n);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace pgcp
