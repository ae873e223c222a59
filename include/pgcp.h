/*
 * pgcp.h -- C ABI of the GB300 PGCP library (parallelizable global conformal
 * parameterization of simply-connected surfaces via partial welding,
 * Choi, Leung-Liu, Gu, Lui; arXiv 1903.12359).
 *
 * The problem statement is Section 4 / Algorithm 3 of the paper: given a
 * triangle mesh (V, F) of a simply-connected surface and a set of cut edges,
 * return planar (free boundary), unit-disk or unit-sphere coordinates of every
 * vertex.
 *
 * Conventions for every entry point:
 *  - Status codes are returned; nothing traps or aborts.  After an error,
 *    pgcp_last_error(ctx) holds a one-line message.
 *  - Unless an argument says otherwise, pointers are DEVICE pointers owned by
 *    the caller, and every call is ordered on the context's CUDA stream.
 *    Calls that copy results to the host synchronise that stream.
 *  - Index arrays are 0-based int32; coordinates are float64.
 *  - V is [nv][3] row-major (x, y, z); F is [nf][3] row-major with faces
 *    oriented consistently (counter-clockwise seen from the outside).
 *  - Opaque handles are released with the matching *_free / *_destroy.
 *  - A context is bound to the device current at pgcp_create and to one
 *    stream; it is not thread-safe.
 */
#ifndef PGCP_H
#define PGCP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PGCP_OK = 0,
    PGCP_E_ARG = 1,           /* bad argument: sizes, indices, orientation, unknown cut edge */
    PGCP_E_CUDA = 2,          /* a CUDA runtime call failed */
    PGCP_E_OOM = 3,           /* device or host allocation failed */
    PGCP_E_NONMANIFOLD = 4,   /* an edge is shared by more than two faces */
    PGCP_E_TOPOLOGY = 5,      /* a piece is not a topological disk (pinch, hole, no boundary) */
    PGCP_E_SCHEDULE = 6,      /* no valid welding order (shared arc not one run of >= 2 edges) */
    PGCP_E_DEGENERATE = 7,    /* zero-area face */
    PGCP_E_NO_CONVERGENCE = 8,/* an iterative solve hit its iteration limit above tolerance */
    PGCP_E_NUMERIC = 9        /* NaN/Inf, or a welding step out of its domain */
} pgcp_status;

typedef enum { PGCP_FREE = 0, PGCP_DISK = 1, PGCP_SPHERE = 2 } pgcp_variant;
/* FP64: FP64 Jacobi-PCG.  FP32_REFINED: FP32 PCG inside FP64 iterative
 * refinement.  DF64_REFINED: double-float (hi + lo float pairs, ~48 bits) PCG
 * on the symmetrically Jacobi-scaled system inside FP64 iterative refinement;
 * runs on the FP32 pipe.  Every mode stops on the FP64 residual. */
typedef enum { PGCP_FP64 = 0, PGCP_FP32_REFINED = 1, PGCP_DF64_REFINED = 2 } pgcp_precision;
typedef enum { PGCP_WARM_COLD = 0, PGCP_WARM_WELDMAP = 1, PGCP_WARM_LEARNED = 2 } pgcp_warm_start;

typedef struct {
    int32_t variant;          /* pgcp_variant */
    int32_t precision;        /* pgcp_precision of the final Laplace solve */
    double  tol;              /* relative residual ||b - A x|| / ||b|| per piece and coordinate */
    int32_t max_iters;        /* PCG iterations per solve (inner solves for FP32_REFINED) */
    int32_t max_refine;       /* outer FP64 refinement steps (FP32_REFINED) */
    double  inner_tol;        /* relative residual reduction of one inner FP32 solve */
    int32_t warm_start;       /* pgcp_warm_start for the final Laplace solve; with PGCP_WARM_COLD the weld
                                 skips the interior map, and interior welded coordinates keep their
                                 local (DNCP) values */
    int32_t interior_map_fp64;/* 1: weld-map the interior in FP64 (else FP32) */
    int32_t block_rows_log2;  /* PCG rows per block tile (autotuner output; 0 = default) */
    int32_t local_precision;  /* pgcp_precision of the DNCP solve: default DF64_REFINED (FP32_REFINED
                                 stalls: with two pins the conditioning is beyond FP32 refinement) */
    int32_t spmv_lanes;       /* threads per matrix row in the FP64 PCG SpMV: 1, 2, 4 or 8 (autotuner
                                 output; 0 = default 1) */
    int32_t pcg_blocks_per_sm;/* resident 256-thread blocks per SM of the mixed-precision PCG kernel:
                                 3 (more registers) or 4 (more warps); autotuner output, 0 = default 4 */
    int32_t pcg_schedule;     /* mixed-precision PCG work schedule: 1 static (each block a fixed row
                                 range; the solve runs as launches of 256 iterations and the ranges
                                 are re-split over the unconverged pieces between them), 2 dynamic
                                 (blocks take 256-row chunks from a counter),
                                 3 round-robin (block b takes chunks b, b + G, ...; up to 256
                                 pieces, else 1), 4 static with one reduction per iteration
                                 (Chronopoulos-Gear form; up to 16 pieces per block, else 1);
                                 autotuner output, 0 = default static */
    int32_t deterministic;    /* 1: every floating-point reduction that steers a solve (PCG dot products,
                                 refinement residual norms, the learned start's scaling and check) is
                                 summed in a fixed order, so repeated calls with the same inputs,
                                 options and GPU model give bitwise identical results and iteration
                                 counts.  The mixed-precision PCG then runs the static schedule.  Not
                                 available with PGCP_FP64 in either solve stage (PGCP_E_ARG).
                                 0 (default): unordered atomic sums, which may differ in the last
                                 bits between runs and change the iteration count slightly. */
    int32_t local_precond;    /* preconditioner of the double-float solves (DNCP, and the final solve
                                 when precision is DF64_REFINED; static schedule, not
                                 deterministic): 0 (default) multilevel -- additive corrections by
                                 low-degree polynomials on nested blocks of 16 * 4^l rows of every
                                 piece -- or 1 Jacobi only.  Other solver settings always use Jacobi. */
    int32_t reserved[1];
} pgcp_options;

/* Per-call statistics (host struct, filled by pgcp_global_solve). */
typedef struct {
    int32_t K;                 /* pieces */
    int32_t n_welds;           /* partial (+ closed) welds performed */
    int32_t dncp_iters;        /* PCG iterations of the local solve (max over refinement steps summed) */
    int32_t final_iters;       /* PCG iterations of the final Laplace solve */
    int32_t dncp_refine;       /* outer refinement steps, local solve */
    int32_t final_refine;      /* outer refinement steps, final solve */
    double  dncp_relres;       /* max over pieces and coordinates of the true FP64 relative residual */
    double  final_relres;
    double  seam_mismatch;     /* max |coords of a vertex in two pieces| after the final solve */
    double  ms_partition, ms_assembly, ms_local, ms_weld, ms_final;  /* stage times (CUDA events) */
    int64_t nnz;               /* stored entries of all piece Laplacians */
    int64_t n_copies;          /* sum of piece vertex counts */
    double  pcg_ms;            /* summed duration of the persistent PCG kernel launches (CUDA events
                                  on the context stream), both solve stages */
    double  pcg_bytes;         /* algorithmic bytes of those launches: per active free row and
                                  iteration 4 + 19*T (row pointer, diagonal, nine vector streams of
                                  2T), per stored entry 4 + T (T = 8 for FP64 and double-float
                                  values, 4 for FP32), i.e. 240 B and 136 B a row at 7 entries */
    int32_t pcg_launches;
    int32_t learned_pieces;    /* pieces whose final solve started from the learned prediction */
    double  pcg_bytes_touched; /* bytes the kernels' schedules actually stream: per row 8 + 22*T
                                  (mixed precision) or 4 + 25*T (FP64), per entry 4 + T; the gap to
                                  pcg_bytes is traffic beyond the algorithmic minimum */
} pgcp_stats;

/* Angle-distortion statistics of a result (Section 5 definition, degrees). */
typedef struct {
    double mean, sd, median, iqr, max;   /* over |d| of all corners; sd with ddof = 0 */
    int64_t n_corners;
    int64_t flips;                        /* faces with signed area <= 0 (planar) or
                                             negative orientation on the sphere */
    double  max_mu;                       /* max |mu| of the piecewise-linear map (planar results) */
} pgcp_distortion;

typedef struct pgcp_ctx pgcp_ctx;    /* opaque; one per CUDA stream */
typedef struct pgcp_part pgcp_part;  /* opaque; partition + all per-piece device state */
typedef struct pgcp_gnn pgcp_gnn;    /* opaque; learned warm-start network (parameters, optimiser state) */

/* Default options: DISK, FP32_REFINED, tol 1e-10, 200000 iterations, 8 refinement
 * steps, inner_tol 1e-4, weld-map warm start, FP32 interior map. */
void pgcp_default_options(pgcp_options* opt);

/* Create a context on the current device.  cuda_stream: a cudaStream_t, or NULL
 * for the legacy default stream.  opt may be NULL (defaults). */
pgcp_status pgcp_create(pgcp_ctx** out, const pgcp_options* opt, void* cuda_stream);
pgcp_status pgcp_destroy(pgcp_ctx* ctx);
pgcp_status pgcp_set_options(pgcp_ctx* ctx, const pgcp_options* opt);
const char* pgcp_last_error(const pgcp_ctx* ctx);
/* Number of kernels the library has launched in this process (all contexts). */
int64_t pgcp_launch_count(void);
/* Number of device allocations the library has requested in this process (all
 * contexts; every stream-ordered cudaMallocAsync of its buffers counts). */
int64_t pgcp_alloc_count(void);
const char* pgcp_status_string(pgcp_status s);

/*
 * Surface partition (Section 4.1).  Faces are joined across every edge that is
 * neither a cut edge nor a boundary edge; each connected component is a piece.
 * Pieces are labelled by the rank of their smallest face id; a piece's
 * vertices are listed in ascending global id and its boundary loop runs
 * counter-clockwise from its smallest global id.  Every piece must be a
 * topological disk (else PGCP_E_TOPOLOGY); the welding order is fixed here
 * (else PGCP_E_SCHEDULE).
 *   V [nv*3], F [nf*3]: mesh.  cut_edges [n_cut*2]: undirected cut edges (may be
 *   NULL with n_cut = 0); or face_labels [nf] (may be NULL): every edge between
 *   faces of different labels is a cut edge (cut_edges is then ignored).
 *   host_ptrs: 1 if V, F, cut_edges, face_labels are host pointers, 0 if device.
 *   closed: 1 for a genus-0 closed surface (sphere variant: last weld closed).
 * The part copies the mesh; the caller's buffers may be freed afterwards.
 */
pgcp_status pgcp_partition(pgcp_ctx* ctx, const double* V, int64_t nv, const int32_t* F, int64_t nf,
                           const int32_t* cut_edges, int64_t n_cut, const int32_t* face_labels,
                           int32_t host_ptrs, int32_t closed, pgcp_part** out);

/* Many independent meshes in one part (batched solves, one graph of launches).
 * Each array holds per-mesh pointers; host_ptrs as above.  Pieces of mesh b
 * follow those of mesh b-1. */
pgcp_status pgcp_partition_batch(pgcp_ctx* ctx, int32_t n_mesh, const double* const* V, const int64_t* nv,
                                 const int32_t* const* F, const int64_t* nf,
                                 const int32_t* const* face_labels, int32_t host_ptrs, int32_t closed,
                                 pgcp_part** out);

pgcp_status pgcp_part_free(pgcp_part* part);

/* Statistics gathered so far by the stages run on this part (host output). */
pgcp_status pgcp_part_get_stats(const pgcp_part* part, pgcp_stats* st);

/* Sizes of a part (host outputs; any pointer may be NULL). */
pgcp_status pgcp_part_info(const pgcp_part* part, int32_t* K, int64_t* n_copies, int64_t* nnz,
                           int64_t* n_loop, int32_t* n_welds, int32_t* n_mesh);

/* Partition outputs (device outputs, caller-allocated; any may be NULL):
 * face_label [nf_total], piece_voff [K+1] (int64), piece_verts [n_copies]
 * (global vertex ids, ascending within each piece), loop_off [K+1] (int64),
 * loop_verts [n_loop] (global ids, ccw, canonical start). */
pgcp_status pgcp_part_get_partition(pgcp_ctx* ctx, const pgcp_part* part, int32_t* face_label,
                                    int64_t* piece_voff, int32_t* piece_verts, int64_t* loop_off,
                                    int32_t* loop_verts);

/*
 * Local conformal parameterization (Section 4.2): assembles every piece's
 * cotangent Laplacian (positive semidefinite sign: L_pq = -(cot a + cot b)/2,
 * L_pp = -sum_q L_pq) into one block-diagonal CSR, then solves DNCP
 *   ((L (+) L) - M) [x; y] = 0,  M_{p,n+q} = M_{n+q,p} = 1/2, M_{q,n+p} = M_{n+p,q} = -1/2
 * for every boundary edge p -> q, with loop position 0 pinned at (0, 0) and
 * position floor(b/2) at (1, 0), by batched PCG; then translates each piece so
 * its reference vertex (first interior vertex at or after local index
 * floor(n/2)) is at 0.
 */
pgcp_status pgcp_local_param(pgcp_ctx* ctx, pgcp_part* part);

/* CSR of the assembled Laplacians (device outputs, caller-allocated; any may be
 * NULL): row_ptr [n_copies+1] (int64), col [nnz] (piece-local column ids,
 * ascending, diagonal stored), val [nnz] (float64). */
pgcp_status pgcp_part_get_csr(pgcp_ctx* ctx, const pgcp_part* part, int64_t* row_ptr, int32_t* col,
                              double* val);

/* Current complex coordinates of every piece vertex copy (device output
 * [n_copies*2], (re, im) pairs, piece-major, ascending global id within a
 * piece).  which: 0 = DNCP result (local frame), 1 = welded (boundary copies
 * FP64; interior copies hold the interior weld map), 2 = final solve. */
pgcp_status pgcp_part_get_coords(pgcp_ctx* ctx, const pgcp_part* part, int32_t which, double* out);

/*
 * Partial welding (Algorithms 1 and 2) of the pieces in the fixed order, then
 * the disk constraint (geodesic algorithm on the global boundary onto the unit
 * disk) or, for a closed surface, the closed weld of the last piece.  FP64 on
 * the boundary; the interior is mapped too (FP32 by default) as the warm start
 * of the final solve.
 */
pgcp_status pgcp_weld(pgcp_ctx* ctx, pgcp_part* part);

/*
 * Final harmonic solve (Section 4.5): Laplace equation on every piece with the
 * welded boundary, batched PCG; gather (each vertex takes the copy of the
 * lowest-label piece holding it); stereographic projection for the sphere.
 *   out: [nv_total*2] (free/disk) or [nv_total*3] (sphere), device unless
 *   host_out = 1.  st: host struct, may be NULL.
 */
pgcp_status pgcp_global_solve(pgcp_ctx* ctx, pgcp_part* part, double* out, int32_t host_out, pgcp_stats* st);

/* Angle distortion, flips and max |mu| of coordinates U (device, [nv*2] or
 * [nv*3] per the part's variant) against the part's mesh.  met: host. */
pgcp_status pgcp_metrics(pgcp_ctx* ctx, const pgcp_part* part, const double* U, pgcp_distortion* met);

/*
 * Area distortion (Section 6.2): per face
 *   d_area(T) = ln( (Area(U(T)) / sum Area(U(T'))) / (Area(T) / sum Area(T')) ),
 * Area(U(T)) the parameter triangle's area (planar: signed area; sphere: the
 * chordal triangle's area, negative when it faces inwards), Area(T) the
 * surface triangle's.  mean_abs: host array, one mean |d_area| per mesh of the
 * part (NaN for a mesh dropped by the welding, or with a non-positive
 * parameter area).  U: device, [nv_total*2] (open parts) or [nv_total*3]
 * (closed parts).  Sums run in a fixed order: repeated calls give the same bits.
 */
pgcp_status pgcp_area_distortion(pgcp_ctx* ctx, const pgcp_part* part, const double* U, double* mean_abs);

/* Result of the Mobius area step for one mesh. */
typedef struct {
    double  param[3];             /* (Re, Im, 0) of alpha (disk) or q (free boundary);
                                     a (sphere); all 0 = identity */
    double  before, after;        /* mean |d_area| before and after the step */
    int32_t evals;                /* objective evaluations of the search */
    int32_t status;               /* pgcp_status of this mesh (NUMERIC: dropped or folded input) */
} pgcp_area_result;

/*
 * Mobius area step (Section 6.2): composes each mesh's map U (device,
 * [nv_total*2] or [nv_total*3], updated in place) with the Mobius
 * transformation that minimises mean |d_area| over
 *   variant PGCP_DISK: the disk automorphisms (z - alpha) / (1 - conj(alpha) z), |alpha| < 1;
 *   variant PGCP_FREE: the maps z / (1 - q z) (every Mobius map is one of these
 *                      followed by a similarity, which leaves d_area unchanged);
 *   variant PGCP_SPHERE (closed parts): the ball automorphisms
 *                      T_a(x) = ((1 - |a|^2)(x - a) - |x - a|^2 a) / (1 - 2<a,x> + |a|^2 |x|^2),
 *                      |a| < 1 (every conformal map of the sphere is one of these
 *                      followed by a rotation, which leaves chordal areas unchanged).
 * The search is Nelder-Mead on the real parameters (2 or 3) from the identity
 * (reflection 1, expansion 2, contraction and shrink 1/2, initial edge 0.05;
 * stops when the simplex spans < 1e-9 and its values < 1e-12, or after 500
 * iterations).  Parameters outside |alpha| < 1, or that give a face a
 * non-positive area, score +inf.  Each objective evaluation is a device
 * reduction over the mesh's faces (fixed order).  out: host array, one per mesh.
 * No counterpart in the paper's main algorithm: Section 6.2 proposes it as an
 * extra step.
 */
pgcp_status pgcp_area_mobius(pgcp_ctx* ctx, const pgcp_part* part, double* U, int32_t variant, pgcp_area_result* out);

/*
 * Pieces of one mesh shared among ranks (the paper's parallel scheme, Section
 * 5.6, with the exchange limited to boundaries: welding reads and writes only
 * boundary points, Sections 4.3 and 4.5).  Every rank partitions the same mesh
 * and owns some of its pieces:
 *  1. pgcp_set_piece_mask, then pgcp_local_param: DNCP maps of the owned
 *     pieces only (the rows of the other pieces are held at 0);
 *  2. pgcp_part_get_boundary(which = 0) on every rank; one rank merges the
 *     owned pieces' loop ranges of all ranks, imports them with
 *     pgcp_part_set_boundary(which = 0) and runs pgcp_weld (welds and the
 *     disk map act on boundary points); pgcp_part_get_boundary(which = 1)
 *     then holds the welded boundary of every piece;
 *  3. every rank imports that welded boundary (pgcp_part_set_boundary,
 *     which = 1; interior rows start the final solve at 0) and calls
 *     pgcp_global_solve: the owned pieces are solved, the output holds NaN
 *     at the vertices whose lowest-label copy belongs to another rank's piece.
 *  pgcp_set_piece_mask: own = host uint8 [K] (nonzero: owned), or NULL (all).
 *  pgcp_part_get_boundary / pgcp_part_set_boundary: device [n_loop * 2],
 *    (re, im) at every loop position in the order of pgcp_part_get_partition's
 *    loop_verts; which = 0 the local (DNCP) map, 1 the welded map (open
 *    parts only).  Importing which = 0 needs pgcp_local_param first.
 */
pgcp_status pgcp_set_piece_mask(pgcp_ctx* ctx, pgcp_part* part, const uint8_t* own);
pgcp_status pgcp_part_get_boundary(pgcp_ctx* ctx, const pgcp_part* part, int32_t which, double* out);
pgcp_status pgcp_part_set_boundary(pgcp_ctx* ctx, pgcp_part* part, int32_t which, const double* in);

/* Result of the fold-over fix (host struct). */
typedef struct {
    int64_t folded_before;   /* faces that folded in the input map */
    int64_t folded_after;    /* faces that still fold after the fix (0 unless rounds ran out) */
    int32_t rounds;          /* compositions made (0 when nothing folded) */
    int32_t pieces_fixed;    /* pieces that folded */
} pgcp_fold_report;

/*
 * Fold-over fix (Section 4.5 and the last step of Algorithm 3; Beltrami
 * coefficient and composition formula, Section 3.5).  A piece's map folds
 * where a face's Beltrami coefficient mu (of the affine map from the surface
 * triangle, in its own flat frame, to the parameter triangle) has |mu| >=
 * 1 - 1e-6, or its signed area is <= 0.  Every piece that folds is composed
 * with a quasi-conformal map, in rounds t = 1, 2, ... (at most 16): the
 * faces within t rings (faces sharing a vertex) of the folded faces have their
 * coefficient capped at modulus 0.7, every other face keeps it, and the map
 * with those coefficients and the piece's boundary values is solved by the
 * linear Beltrami solver (div(A_nu grad u) = 0 for both coordinates, linear
 * elements on the surface triangles; A_nu = I gives the cotangent Laplacian),
 * until no face folds.  Pieces that do not fold are left bit for bit.
 *   U: device [nv_total*2], the planar map of the part's mesh (free or disk
 *   parts; closed parts return PGCP_E_ARG), updated in place; every copy of a
 *   vertex takes U of that vertex, and the gather takes the lowest-label copy.
 *   rep: host, may be NULL.
 * The solves use the context's final-solve precision and tolerance.
 */
pgcp_status pgcp_fix_folds(pgcp_ctx* ctx, pgcp_part* part, double* U, pgcp_fold_report* rep);

/*
 * pgcp_metrics without any device allocation.  Library plumbing: the paper has
 * no counterpart.  For callers that must not allocate device memory, because
 * their device memory is held by another allocator or because an allocation
 * may fail or synchronise at a point where they cannot afford that.
 *
 * Same arguments, results and error codes as pgcp_metrics (sums are
 * accumulated with atomics, so mean and sd may differ from it in the last
 * bits; order statistics, max, flips and max |mu| are identical).  All device
 * scratch is one fixed static array inside the library (about 20 MB, sized
 * for PGCP_METRICS_NOALLOC_MAX_FACES faces); a part with more faces returns
 * PGCP_E_ARG with a message naming the limit, and pgcp_metrics serves it.
 *
 * The context's device must be current (else PGCP_E_ARG).  The first call on a
 * device looks up the scratch array's address (cudaGetSymbolAddress, which may
 * load the library's module on that device) and caches it; make that first
 * call before any stream capture on the device.  The sums, max and counters
 * in the scratch are cleared on the stream at the start of every call; the
 * rest is fully overwritten before it is read.  The scratch is shared by every
 * context on the device: calls that overlap in time (from several host threads,
 * or on several streams without ordering between them) race on it and give
 * wrong results.  The call synchronises its context's stream before returning.
 */
#define PGCP_METRICS_NOALLOC_MAX_FACES 262144
pgcp_status pgcp_metrics_noalloc(pgcp_ctx* ctx, const pgcp_part* part, const double* U, pgcp_distortion* met);

/*
 * One-shot convenience: partition + local_param + weld + global_solve.
 * variant selects the output (free: [nv*2], disk: [nv*2], sphere: [nv*3]).
 * host_ptrs = 1: V, F, cut_edges and out are host pointers (the copies are
 * part of the call).  st may be NULL.
 */
pgcp_status pgcp_run(pgcp_ctx* ctx, const double* V, int64_t nv, const int32_t* F, int64_t nf,
                     const int32_t* cut_edges, int64_t n_cut, const int32_t* face_labels,
                     int32_t host_ptrs, double* out, pgcp_stats* st);

/*
 * Per-mesh status of a batch (host int32 [n_mesh], n_mesh from pgcp_part_info;
 * library plumbing, no counterpart in the paper).  A mesh of a batch whose
 * welding leaves its domain (PGCP_E_NUMERIC: a zipper point left the right
 * half-plane, or the arc lost its order in FP64) is dropped: its output
 * vertices are NaN and the other meshes complete, so pgcp_weld and
 * pgcp_global_solve return PGCP_OK.  A single mesh, or a batch in which every
 * mesh fails, returns the error instead.
 */
pgcp_status pgcp_part_mesh_status(const pgcp_part* part, int32_t* status);

/*
 * Autotuner of the batched PCG schedule (no counterpart in the paper).  Times
 * probe_iters (>= 10) capped DNCP iterations of `part` for each candidate and
 * stores the fastest in the context options (and in *chosen):
 *   mixed-precision local solves: pcg_blocks_per_sm in {3, 4} x pcg_schedule
 *   in {static, dynamic, round-robin, one reduction};  FP64 local solves: spmv_lanes in {1, 2, 4} x
 *   block_rows_log2 in {8, 9, 10}.  With the multilevel preconditioner (double-float local solves,
 *   local_precond 0, not deterministic) the static schedule is the only candidate: the other
 *   schedules run without the preconditioner, and a time per iteration does not compare them.
 * The probes overwrite the part's local map: call pgcp_local_param afterwards.
 * ms_per_iter (may be NULL): the winner's kernel time per iteration.
 */
pgcp_status pgcp_autotune(pgcp_ctx* ctx, pgcp_part* part, int32_t probe_iters, pgcp_options* chosen,
                          double* ms_per_iter);

/*
 * Learned warm start (no counterpart in the paper).  A message-passing network
 * over each piece's mesh graph predicts the correction from the weld-map
 * start u_w to the final map; the final solve (Section 4.5) starts from
 * u_w + sigma * prediction on the pieces where that start has the smaller
 * FP64 residual, and from u_w elsewhere, so the result does not depend on the
 * network.  Architecture, features and parameter layout:
 *   F_i = [z_i / sigma, boundary flag, 1, 0 x 12] (16 wide), z_i = -(L u_w)_i / d_i
 *         on interior rows, sigma = RMS of |z| over the piece's interior rows;
 *   X_0 = relu(F W_in + b_in);  X_{l+1} = relu([X_l | P X_l] W_l + b_l), l = 0..3,
 *         P = D^-1 W the random walk of the cotan weights;  out = X_4 W_out + b_out.
 *   Parameters, one float32 vector of pgcp_gnn_num_params() = 35152 values:
 *   W_in (16 x 64), b_in (64), 4 x [W_l (128 x 64), b_l (64)], W_out (64 x 16),
 *   b_out (16); matrices row-major with rows = inputs.  Dense layers run in
 *   BF16 on the tensor cores with FP32 accumulation.
 * A part is usable for prediction after pgcp_weld, for training after
 * pgcp_global_solve (the target is its final map).
 *  pgcp_gnn_create: params = host float32 [num_params] (initial values).
 *  pgcp_gnn_load: the same from a raw little-endian float32 file.
 *  pgcp_set_gnn: network used by warm_start = PGCP_WARM_LEARNED (not owned;
 *    NULL detaches).
 *  pgcp_gnn_inputs: features feat [rows x 16] (float32, the bf16 values the
 *    network sees), targets [rows x 2] (may be NULL; needs the final map) and
 *    sigma [K], all device pointers, rows = vertex copies (pgcp_part_info).
 *  pgcp_gnn_grad: loss (mean over interior rows of |out - target|^2) and its
 *    gradient (host float32 [num_params]) at the current parameters.
 *  pgcp_gnn_train_step: one Adam step (lr) on that loss; *loss before the step.
 *  pgcp_gnn_predict: x0 [rows x 2] (device, FP64) = u_w + sigma * out.
 */
int64_t pgcp_gnn_num_params(void);
pgcp_status pgcp_gnn_create(pgcp_ctx* ctx, const float* params, pgcp_gnn** out);
pgcp_status pgcp_gnn_load(pgcp_ctx* ctx, const char* path, pgcp_gnn** out);
pgcp_status pgcp_gnn_free(pgcp_gnn* gnn);
pgcp_status pgcp_gnn_get_params(pgcp_ctx* ctx, const pgcp_gnn* gnn, float* params);
pgcp_status pgcp_gnn_set_params(pgcp_ctx* ctx, pgcp_gnn* gnn, const float* params);
pgcp_status pgcp_set_gnn(pgcp_ctx* ctx, pgcp_gnn* gnn);
pgcp_status pgcp_gnn_inputs(pgcp_ctx* ctx, const pgcp_part* part, float* feat, float* target, float* sigma);
pgcp_status pgcp_gnn_grad(pgcp_ctx* ctx, pgcp_gnn* gnn, const pgcp_part* part, float* grad, double* loss);
pgcp_status pgcp_gnn_train_step(pgcp_ctx* ctx, pgcp_gnn* gnn, const pgcp_part* part, float lr, double* loss);
pgcp_status pgcp_gnn_predict(pgcp_ctx* ctx, const pgcp_gnn* gnn, const pgcp_part* part, double* x0);

/*
 * One-call forms of Algorithm 3 per variant (Section 4.4): partition, local
 * DNCP maps, welds (+ disk or closed weld), final harmonic solve, gather.
 * V [nv*3], F [nf*3], cut [n_cut*2] (or NULL with face_labels [nf]) and the
 * output are DEVICE pointers; the output is uv [nv*2] (free, disk) or xyz
 * [nv*3] (sphere).  The variant in the context options is ignored (each call
 * sets its own); every other option applies.  st may be NULL.
 */
pgcp_status pgcp_free_boundary(pgcp_ctx* ctx, const double* V, int64_t nv, const int32_t* F, int64_t nf,
                               const int32_t* cut, int64_t n_cut, const int32_t* face_labels, double* uv_out,
                               pgcp_stats* st);
pgcp_status pgcp_disk(pgcp_ctx* ctx, const double* V, int64_t nv, const int32_t* F, int64_t nf,
                      const int32_t* cut, int64_t n_cut, const int32_t* face_labels, double* uv_out,
                      pgcp_stats* st);
pgcp_status pgcp_sphere(pgcp_ctx* ctx, const double* V, int64_t nv, const int32_t* F, int64_t nf,
                        const int32_t* cut, int64_t n_cut, const int32_t* face_labels, double* xyz_out,
                        pgcp_stats* st);

/*
 * Batched one-call form: many independent meshes (open surfaces for free and
 * disk, closed for sphere, per the context's variant) in one part, so every
 * solve stage runs once for the whole batch (one persistent PCG launch over
 * all pieces of all meshes).  Device pointers; outs[b] receives mesh b's map
 * ([nv_b*2] or [nv_b*3]).  mesh_status (host int32 [n_mesh], may be NULL)
 * gets each mesh's status (see pgcp_part_mesh_status): a mesh dropped by the
 * welding is NaN and the call still returns PGCP_OK.
 */
typedef struct {
    const double* V;
    int64_t nv;
    const int32_t* F;
    int64_t nf;
    const int32_t* face_labels;   /* [nf] piece label of every face */
} pgcp_mesh_desc;
pgcp_status pgcp_batch_run(pgcp_ctx* ctx, int32_t n_mesh, const pgcp_mesh_desc* meshes, double* const* outs,
                           int32_t* mesh_status, pgcp_stats* st);

/*
 * Self-test access to the device primitives the partition and the metrics
 * build on (no counterpart in the paper).  Device pointers, ordered on the
 * context stream.
 *  pgcp_selftest_sort: stable sort of n (key, value) pairs by the low `bits`
 *    bits of key, in place.
 *  pgcp_selftest_scan: out[i] = sum of in[0..i-1] (int32 in, int64 out);
 *    *total (host) = sum of all.
 */
pgcp_status pgcp_selftest_sort(pgcp_ctx* ctx, uint64_t* keys, int32_t* vals, int64_t n, int32_t bits);
pgcp_status pgcp_selftest_scan(pgcp_ctx* ctx, const int32_t* in, int64_t* out, int64_t n, int64_t* total);

/*
 * Self-test access to the BF16 tensor-core GEMM of the learned warm start (no
 * counterpart in the paper).  C[M x N] = epi(A[M x K] . Bt[N x K]^T): A and
 * Bt bf16, row-major with K contiguous (16-byte aligned), device pointers.
 *  epilogue 0: C fp32 [M x N];  1: C = relu(. + bias) as bf16;  2: C = . + bias
 *  (fp32).  Shapes (N, K) in {(16,16), (16,64), (64,16), (64,64), (64,128),
 *  (128,64)}, else PGCP_E_ARG.  Synchronises the context stream.
 * pgcp_selftest_umma_desc / _idesc: the shared-memory matrix descriptor and
 * the instruction descriptor the kernel issues (host computation, no GPU).
 */
pgcp_status pgcp_selftest_gemm_bf16(pgcp_ctx* ctx, int32_t epilogue, int32_t N, int32_t K, const void* A,
                                    const void* Bt, int64_t M, const float* bias, void* C);
uint64_t pgcp_selftest_umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo);
uint32_t pgcp_selftest_umma_idesc(int32_t m, int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* PGCP_H */
