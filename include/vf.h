/*
 * vf.h -- C ABI of libvf: hierarchically compressed radiosity view-factor
 * matrices on one GB300 (sm_103a).
 *
 * The library computes, for a triangle mesh, the view-factor matrix F of the
 * discrete radiosity system B = E + diag(rho) F B (Section 1, Eq.
 * radiosity-system), stores it compressed over a quadtree or octree of the
 * facets (Sections 3.1, 4), and applies it to many right-hand sides inside
 * the Jacobi solve (Sections 3, 5.1).  Every step runs in the library's own
 * CUDA kernels; host code only marshals arguments, builds the index trees
 * and schedules launches.
 *
 * Conventions
 *  - Ownership: handles are created and freed by the library.  Caller buffers
 *    (vertices, faces, X, Y, E, B, rho) are read or written during the call
 *    and never kept or freed by it.
 *  - Pointers: "host" arguments are ordinary CPU memory; "device" arguments
 *    are CUDA device pointers on the handle's device (for example the data
 *    pointer of a torch CUDA tensor).
 *  - Layout: right-hand sides are column-major N x R with an explicit leading
 *    dimension ld >= N, rows in the mesh's face order.
 *  - Streams: device work is ordered on the caller's stream (NULL = the
 *    legacy default stream).  Calls that return host data synchronise it.
 *  - Errors: every call returns a vf_status; vf_last_error() gives the
 *    calling thread's last message.  VF_E_NOCONV still writes the best
 *    iterate.  Device-side waits are bounded and report VF_E_TIMEOUT.
 *  - Threads: handles are immutable after creation and may be shared by
 *    concurrent calls on different streams.
 */
#ifndef VF_H
#define VF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vf_mesh vf_mesh;
typedef struct vf_tree vf_tree;
typedef struct vf_hmat vf_hmat;
typedef struct vf_rank_predictor vf_rank_predictor;
typedef struct CUstream_st* vf_stream; /* a cudaStream_t */

typedef enum {
    VF_OK = 0,
    VF_E_INVAL = 1,   /* bad argument (size, pointer, option) */
    VF_E_NOMEM = 2,   /* device or host allocation failed */
    VF_E_CUDA = 3,    /* a CUDA runtime call failed */
    VF_E_NOCONV = 4,  /* solve hit max_iter; outputs hold the last iterate */
    VF_E_TIMEOUT = 5, /* a bounded device-side wait gave up */
    VF_E_OOB = 6,     /* a device-side self-check fired: a tensor-core page record whose
                         shape, page extent or operand range is out of bounds (the record
                         is skipped, nothing is read or written through it) */
    VF_E_IO = 7,      /* file could not be opened, read or written */
    VF_E_CORRUPT = 8  /* file failed its magic/version/CRC checks */
} vf_status;

typedef enum { VF_PREC_FP32 = 0, VF_PREC_BF16 = 1, VF_PREC_FP8 = 2 } vf_precision;
typedef enum { VF_TREE_QUAD = 0, VF_TREE_OCT = 1 } vf_tree_kind;
typedef enum { VF_BLK_ZERO = 0, VF_BLK_DENSE = 1, VF_BLK_CSR = 2, VF_BLK_SVD = 3, VF_BLK_HIER = 4 } vf_block_kind;

/* Thread-local message of the last failing call ("" if none). */
const char* vf_last_error(void);
const char* vf_version(void);

/* Error-path testing (no counterpart in the paper).  vf_debug_fail_alloc:
 * the nth device allocation the library makes from now on (counted over
 * all threads) fails as if the device were out of memory, so the call
 * making it returns VF_E_NOMEM and releases what it holds; 0 disarms.
 * vf_set_wait_limit: the number of polls a bounded wait of the CUDA-core
 * multiply (its page copies) makes on `device` before it gives up and the
 * call reports VF_E_TIMEOUT (polls < 0 restores the default, 2^22; 0 makes
 * every such wait give up at once).  A warp that gives up still waits, with
 * the default bound, for the copies it has in flight before it stops, so
 * the kernels exit normally.  The limit is read by each kernel when it
 * starts (solve graphs included).  Errors: VF_E_INVAL, VF_E_CUDA. */
vf_status vf_debug_fail_alloc(int64_t nth);
vf_status vf_set_wait_limit(int32_t device, int64_t polls);

/* ------------------------------------------------------------------ mesh
 * Section 3: A_i, x_i, n_i of each triangle (midpoint collocation).
 * vf_mesh_create copies the host vertices (nv x 3, FP64) and faces (nf x 3,
 * int32, counter-clockwise = outward normal by the right-hand rule) to the
 * device and snaps the vertices to an integer grid: unit = 2^e with
 * extent / 2^e <= 2^18 (extent = largest bounding-box side), so every
 * visibility decision is made exactly in integers.  Geometry is computed on
 * the device in FP64 from the snapped coordinates.
 * Errors: VF_E_INVAL for nv < 3, nf < 1, a face index out of range or a
 * zero-extent vertex set; VF_E_NOMEM, VF_E_CUDA. */
typedef struct {
    int32_t device; /* CUDA device ordinal */
} vf_mesh_opts;

vf_status vf_mesh_create(const double* verts, int64_t nv, const int32_t* faces, int64_t nf,
                         const vf_mesh_opts* opts, vf_mesh** out);
void vf_mesh_destroy(vf_mesh* m);
int64_t vf_mesh_nfacets(const vf_mesh* m);
/* grid unit and the integer grid origin (base * unit = world coordinates of grid 0) */
vf_status vf_mesh_grid(const vf_mesh* m, double* unit, int64_t base[3]);
/* Host outputs in face order: area[nf], centroid[nf*3] (relative to the grid
 * origin), unit normal[nf*3]; any pointer may be NULL. */
vf_status vf_mesh_geometry(const vf_mesh* m, double* area, double* centroid, double* normal);

/* Section 3.2: V_ij = 1 iff n_i.d_ij > 0, n_j.d_ji > 0 (exact, integer) and
 * the open segment (x_i, x_j) meets no other closed triangle (edge and
 * vertex touches block; a coplanar segment is not blocked).  Rows `rows`
 * (host, nrows facet indices; NULL = all facets) are written to V (host,
 * nrows x nf bytes, row-major).  Computed by the library's BVH kernels. */
vf_status vf_mesh_visibility(const vf_mesh* m, const int64_t* rows, int64_t nrows, uint8_t* V);

/* Section 2, Eq. insolation-for-point-sun with the sun at 1 AU:
 * E[i + r*lde] = solar_flux * max(0, n_i . s_r) * V_sun(i, s_r), where
 * V_sun is 1 iff n_i . s_q > 0 and the ray from x_i along
 * s_q = round(2^20 s_r) meets no other triangle.  sun_dirs: host, R x 3
 * unit vectors.  E: device FP32, column-major, lde >= nf, face order. */
vf_status vf_mesh_insolation(const vf_mesh* m, const double* sun_dirs, int32_t R, double solar_flux,
                             float* E, int64_t lde, vf_stream stream);

/* Section 2: the Sun as a disk of finite extent, its flux a sum over point
 * sources of the form of Eq. insolation-for-point-sun.  For each sun
 * direction s_r (host, R x 3, unit), the disk of the given angular radius
 * (radians, < 0.5; the Sun at 1 AU: 4.65e-3) around s_r is cut into
 * `rings` rings of equal radial width, ring k (k = 0 the central disk) into
 * max(1, 6k) equal sectors; each cell contributes one point source at its
 * area-weighted mean radius and mid angle, weighted by its share of the
 * disk's area (1 + 3 rings (rings - 1) sources, weights summing to 1):
 * E[i + r*lde] = sum_k w_k solar_flux max(0, n_i . s_rk) V_sun(i, s_rk),
 * each V_sun as in vf_mesh_insolation, the sum in FP64.  E: device FP32,
 * column-major, face order.  Errors: VF_E_INVAL (rings outside [1, 64],
 * radius outside [0, 0.5)), VF_E_NOMEM, VF_E_CUDA. */
vf_status vf_mesh_insolation_disk(const vf_mesh* m, const double* sun_dirs, int32_t R, double solar_flux,
                                  double angular_radius, int32_t rings, float* E, int64_t lde, vf_stream stream);

/* ------------------------------------------------------------- partition
 * Algorithm 2 (quadtree on centroids, Section 4.1) and its octree analogue.
 * Each node splits at the midpoint of its own centroids' bounding box
 * (exact integer compare 2c >= lo + hi, ties go to the upper child); child
 * index 2[x>=]+[y>=] (octree 4[x>=]+2[y>=]+[z>=]); empty children dropped;
 * members keep their parent's order; nodes numbered in depth-first preorder.
 * Stops at count <= leaf_size, depth == max_depth or a zero-extent box. */
typedef struct {
    int32_t kind;      /* vf_tree_kind */
    int32_t leaf_size; /* default 64 */
    int32_t max_depth; /* default 32 */
} vf_partition_opts;

vf_status vf_partition(const vf_mesh* m, const vf_partition_opts* opts, vf_tree** out);
void vf_tree_destroy(vf_tree* t);
int64_t vf_tree_nnodes(const vf_tree* t);
/* perm[k] = face index at tree position k (host, nf entries). */
vf_status vf_tree_perm(const vf_tree* t, int32_t* perm);
/* Per node (host arrays of vf_tree_nnodes entries; any may be NULL). */
vf_status vf_tree_nodes(const vf_tree* t, int32_t* first, int32_t* count, int32_t* depth,
                        int32_t* parent);

/* -------------------------------------------------------------- assembly
 * Algorithms 1, 3 and 4 (Sections 3.3, 4.2, 4.3).  Visibility of every pair
 * is computed once on the device as a bit matrix; entries
 * F_ij = [n_i.(x_j-x_i)][n_j.(x_i-x_j)] V_ij A_j / (pi |x_i-x_j|^4) (Eq.
 * FF-def) are evaluated on the fly.  Starting at the pairs of the root's
 * children, each block pair is stored as the cheapest of: zero (no visible
 * pair), dense (4mn bytes), CSR (8 nnz + 4(m+1)), the q-truncated SVD
 * U'V'^T with q the smallest rank such that sigma_{q+1} < tol sigma_1 and
 * U' = U_q Sigma_q, V' = V_q compacted to the block's nonzero rows m' and
 * columns n' (4q(m'+n') + 4(m'+n')), or the hierarchical block over its
 * child pairs; a leaf block (two tree leaves, or m n < leaf_threshold) is
 * dense or CSR.  Ties: zero < dense < CSR < SVD < hierarchical.  A
 * hierarchical block whose nonzero children are all CSR (all dense) is
 * coalesced into one CSR (dense) block.  The SVD probe starts at rank k0
 * and doubles up to k_max; a block needing more fails the probe.  With
 * verify = 1 each accepted factorisation is checked against Algorithm 3's
 * criterion (Section 3): ||F_IJ - U'V'^T||_2 <= tol ||F_IJ||_2 (by
 * Eckart-Young the left side is sigma_{q+1}), both norms estimated by eight
 * FP64 power iterations on the GPU from one seeded start; since those
 * estimates approach the norms from below, a factorisation passes only if
 * the error's estimate is at most 0.9 tol times the norm's.  A block that
 * fails goes back to the rank doubling (counted in verify_failed).  The
 * check is on by default.
 * Errors: VF_E_INVAL, VF_E_NOMEM, VF_E_CUDA. */
typedef struct {
    double tol;             /* compression tolerance, e.g. 1e-3 */
    int64_t leaf_threshold; /* default 4096 */
    int32_t k0;             /* initial probe rank, default 8 */
    int32_t k_max;          /* largest probe rank, default 128 */
    int32_t power_iters;    /* subspace iterations of the probe, default 2 */
    int32_t verify;         /* 1: FP64 truncation check on accepted SVD blocks (the default
                               with opts = NULL and in the Python binding); 0: off */
    uint32_t precisions;    /* bit (1 << vf_precision): copies to build; FP32 always */
    const vf_rank_predictor* predictor; /* NULL: plain probe path */
    uint64_t seed;
    int32_t storage;        /* 0: compressed (Algorithm 4); 1: every leaf pair dense,
                               i.e. the uncompressed F (the comparison of the
                               terrain workload); 2: every leaf pair CSR (Algorithm 1) */
} vf_assemble_opts;

typedef struct {
    int64_t nblocks[5];     /* stored blocks per vf_block_kind (HIER counts inner nodes) */
    int64_t bytes[5];       /* FP32 payload bytes per kind */
    int64_t nnz_visible;    /* visible ordered pairs (nonzeros of F) */
    int64_t probes;         /* SVD probes run (each k counts once) */
    int64_t probes_failed;  /* probes that found no acceptable rank */
    int64_t probes_skipped; /* blocks where the byte bound ruled the SVD out */
    int64_t probes_predicted_skip; /* probes the predictor skipped */
    int64_t verify_failed;  /* SVD blocks whose check failed (rank raised) */
    int64_t predictor_audits;      /* predicted skips probed anyway (one in 8) */
    int64_t predictor_audit_wins;  /* audits whose probe stored an SVD */
    int64_t predictor_fallbacks;   /* levels whose audits failed: their skips probed after all */
    int32_t max_rank;
    double t_visibility, t_stats, t_probe, t_pack, t_total; /* seconds */
} vf_assemble_stats;

vf_status vf_assemble(const vf_mesh* m, const vf_tree* t, const vf_assemble_opts* opts,
                      vf_hmat** out, vf_assemble_stats* stats);
void vf_hmat_destroy(vf_hmat* h);
int64_t vf_hmat_nfacets(const vf_hmat* h);
/* Stored blocks (host, nblocks rows of 7 int32: row node, col node, kind, q,
 * m', n', reserved); call with desc = NULL to get the count. */
vf_status vf_hmat_blocks(const vf_hmat* h, int64_t* nblocks, int32_t* desc);
/* Total device payload bytes for one precision. */
int64_t vf_hmat_bytes(const vf_hmat* h, vf_precision p);

/* Training data from an assembly: one row per SVD probe candidate (the
 * candidates of Algorithm 3 whose byte bound allows an SVD), in the order
 * they were probed.  feats: n x VF_PRED_NFEAT (host, row-major), labels: n
 * classes (host); call with feats = labels = NULL to get n.  Features of a
 * candidate block (I, J), all from the cluster geometry and the visibility
 * counts the assembly already has:
 *   0 log2 |I|   1 log2 |J|   2 |I'|/|I| (rows with a visible pair)
 *   3 |J'|/|J|   4 nnz/(|I||J|) (visible fraction)
 *   5 distance between the clusters' mean centroids / (diameter I +
 *     diameter J) (diameters: bounding-box diagonals)
 *   6 mean normal I . mean normal J   7 |mean normal I|   8 |mean normal J|
 *   9 block height (levels above the leaf pairs)
 * Labels: the probe outcome: 0..4 = an SVD accepted with rank q in
 * (0, 8], (8, 16], (16, 32], (32, 64], (64, 128]; 5 = no SVD accepted (no
 * rank met the tolerance or the SVD could not win on bytes). */
#define VF_PRED_NFEAT 10
#define VF_PRED_NCLASS 6
vf_status vf_hmat_probe_log(const vf_hmat* h, int64_t* n, float* feats, int32_t* labels);

/* ---------------------------------------------------------- rank predictor
 * The learned part of assembly; the paper has none (it motivates it: the
 * SVD probes dominate assembly time, Section 4.3).  A 3-layer MLP:
 * standardised features -> 64 -> 64 -> VF_PRED_NCLASS, ReLU, softmax,
 * mean cross-entropy loss.  The forward pass uses FP16-rounded weights with
 * FP32 activations and accumulation; training keeps FP32 master weights
 * (Adam, lr given, betas 0.9 / 0.999) and takes the gradient at the rounded
 * weights.  Training and inference run in the library's own kernels, with
 * fixed summation orders (bit-reproducible).
 * Used by vf_assemble through opts.predictor: a candidate predicted class 5
 * with probability >= 0.9 is not probed (counted in probes_predicted_skip);
 * any other prediction c sets its first probe rank to max(k0, 8 << c).  The
 * probe and the byte test still decide every block, so the matrix meets
 * the tolerance whatever the network predicts.  Skips are audited: one in
 * eight predicted skips is probed anyway, and if at one level more than a
 * quarter of the audits (and at least two) store an SVD -- the network is
 * off the distribution it was trained on -- that level's skipped
 * candidates are probed too (predictor_fallbacks).
 * Parameters (flat FP32, VF_PRED_NPARAM): W1 (64 x 10, row-major), b1 (64),
 * W2 (64 x 64), b2 (64), W3 (6 x 64), b3 (6); then the feature means and
 * scales (10 + 10) in vf_predictor_params.
 * A predictor handle is used by one thread at a time. */
#define VF_PRED_NPARAM 5254
vf_status vf_predictor_create(int32_t device, uint64_t seed, vf_rank_predictor** out);
void vf_predictor_destroy(vf_rank_predictor* p);
/* get / set: host arrays of VF_PRED_NPARAM + 2 * VF_PRED_NFEAT floats (either may be NULL). */
vf_status vf_predictor_params(vf_rank_predictor* p, float* get, const float* set);
/* Mean loss (FP64 sum of FP32 terms) and its gradient w.r.t. the parameters
 * (host, VF_PRED_NPARAM) on n samples; feats, labels: host. */
vf_status vf_predictor_grad(vf_rank_predictor* p, const float* feats, const int32_t* labels, int64_t n, double* loss,
                            float* grad);
/* Adam over shuffled mini-batches (a seeded order; the last partial batch of
 * an epoch is dropped); the feature standardisation is set from the training
 * set first.  final_loss: the mean loss over all n samples afterwards. */
vf_status vf_predictor_train(vf_rank_predictor* p, const float* feats, const int32_t* labels, int64_t n,
                             int32_t epochs, int32_t batch, float lr, double* final_loss);
/* Classes (argmax, ties to the lower class) and, if prob != NULL,
 * probabilities (n x VF_PRED_NCLASS) of n feature rows; host arrays. */
vf_status vf_predictor_predict(const vf_rank_predictor* p, const float* feats, int64_t n, int32_t* cls, float* prob);

/* ---------------------------------------------------------------- apply
 * Algorithm 5 (Section 4.4): Y = F_hat X for R columns.  X, Y: device FP32,
 * column-major, face order (the tree permutation is applied inside).
 * p selects the factor copy (FP32 master, BF16, or FP8 E4M3); accumulation
 * is FP32.  Below 16 columns (or as tuned) the CUDA cores stream the FP32 /
 * BF16 / FP8 copy (FP8: one scale per block).  From 16 columns BF16 and FP8
 * run on the tensor cores in panels of 128 columns: BF16 as kind::f16 MMAs;
 * FP8 as kind::f8f6f4 E4M3 MMAs whose right-hand sides are FP8 too, with
 * power-of-two scales per RHS column, per matrix row and per SVD rank
 * column (exact, undone in the epilogue; values beyond E4M3's range
 * saturate).  Errors: VF_E_INVAL (R < 1, ld < N, precision not built),
 * VF_E_CUDA, VF_E_TIMEOUT, VF_E_OOB. */
vf_status vf_apply(const vf_hmat* h, vf_precision p, const float* X, int64_t ldx, int32_t R, float* Y,
                   int64_t ldy, vf_stream stream);

/* Y_t = F_hat X_t with X_t, Y_t already in tree order (row k of X_t is
 * facet perm[k]): the multiply alone, without the two permutations of
 * vf_apply.  Device FP32, column-major, leading dimension N. */
vf_status vf_apply_tree(const vf_hmat* h, vf_precision p, const float* Xt, int32_t R, float* Yt, vf_stream stream);

/* vf_apply_tree that allocates nothing, for callers that cannot allocate
 * device memory at call time: a host program whose device memory is wholly
 * committed to its own pool, or a time-critical loop that must not take an
 * allocator's latency or locks.  The paper has no counterpart: this is an
 * interface of this library, not a step of the method.
 *
 * Path: always the CUDA-core multiply over all R columns at once.  It never
 * takes the tensor-core path (BF16 or FP8 with R >= 16) or a tuned RHS block, so
 * where vf_apply_tree would take either, the two calls agree only to the
 * rounding of the precision, not bit for bit; elsewhere they run the same
 * kernels with the same RHS tile and agree exactly.
 *
 * Scratch: the multiply's T vectors, the partial sums of cut blocks and a
 * status word live in fixed-size static device arrays of libvf (17 MiB on
 * each device that loads the library's multiply module, held until the
 * process exits).  The memory is taken when that module is loaded on a
 * device; with CUDA's lazy module loading (the default) that can be this
 * call's first use, so a caller whose device memory is fully committed
 * should make one call (or any other libvf multiply) while it still has
 * 17 MiB free.
 *   T floats       npanels x RB x n_T   <= VF_STATIC_T_FLOATS    (4,194,304)
 *   partial floats npanels x RB x n_P   <= VF_STATIC_PART_FLOATS (262,144)
 * where RB = the RHS tile the autotuner recorded for (p, R) (vf_autotune,
 * vf_tune_set), else 1, 2, 4 or 8 (the smallest >= min(R, 8)); npanels =
 * ceil(R / RB), n_T = the sum of the SVD blocks' ranks and n_P = the sum of
 * rank x pieces over the (few) SVD blocks whose V' rows are cut across
 * several pieces of the multiply's work plan.  A matrix and R that need
 * more return VF_E_INVAL with the sizes in the message, and nothing is
 * launched.
 * What must start at zero: only the status word; the call clears it itself
 * (cudaMemsetAsync) before the kernels run.  T and the partial slots are
 * written before they are read.
 * The call is synchronous: it returns once the multiply has finished on
 * `stream`, after reading the status word (VF_E_TIMEOUT if a bounded
 * device-side wait gave up).
 * The first call on a device resolves the static arrays' addresses
 * (cudaGetSymbolAddress) and sets the kernels' shared-memory attributes;
 * make that first call outside any stream capture.
 * Concurrency: the arrays are shared by every caller in the process on a
 * device, so calls that overlap in time (from other threads or streams)
 * race on them and corrupt each other's results: serialise them.
 * Xt, Yt: device FP32, column-major, leading dimension N, tree order.
 * Errors: VF_E_INVAL (null, R < 1, precision not built, scratch too
 * small), VF_E_TIMEOUT, VF_E_CUDA. */
#define VF_STATIC_T_FLOATS 4194304
#define VF_STATIC_PART_FLOATS 262144
vf_status vf_apply_tree_static(const vf_hmat* h, vf_precision p, const float* Xt, int32_t R, float* Yt,
                               vf_stream stream);

/* ---------------------------------------------------------------- solve
 * B = (I - diag(rho) F)^{-1} E by Jacobi (Sections 3, 5.1): B_0 = E,
 * B_{k+1} = E + rho .* (F B_k); a column is done when
 * ||B_{k+1} - B_k||_2 <= rtol ||E||_2; a zero column returns 0.  The sweep
 * loop runs on the device inside one CUDA graph (conditional while node,
 * bounded by max_iter).  With precision BF16/FP8 and refine = 1 the inner
 * sweeps use the low-precision factors and an outer loop corrects with the
 * residual r = E - B + rho .* F B computed from the FP32 factors with FP64
 * accumulation (from 16 columns, where the BF16 / FP8 sweeps run on the
 * tensor cores: the FP32 factors and B split in BF16 hi + lo terms, FP32
 * accumulation, about 2^-16 relative).  clamp = 1 sets negative outputs to
 * 0 (Section 4.2).
 * rho: device FP32 [nf] in face order, or NULL for opts.rho.  E, B: device
 * FP32 column-major, face order.  VF_E_NOCONV: B holds the last iterate. */
typedef struct {
    double rtol;        /* default 1e-6 */
    int32_t max_iter;   /* per Jacobi loop, default 100 */
    int32_t precision;  /* vf_precision of the sweeps */
    int32_t refine;     /* 1: mixed-precision iterative refinement */
    int32_t max_refine; /* default 8 */
    double inner_rtol;  /* inner loop tolerance with refinement, default 1e-3 */
    int32_t clamp;      /* 1: B = max(B, 0) at the end */
    float rho;          /* uniform rho when the rho pointer is NULL */
} vf_solve_opts;

typedef struct {
    int32_t sweeps;           /* low-precision (or FP32) sweeps */
    int32_t refinements;      /* outer refinement steps */
    int32_t converged;        /* 1 if every column met rtol */
    int32_t kernels;          /* device kernels the call launched (graph body counted per sweep run) */
    double max_rel_residual;  /* max over columns of ||r||_2 / ||E||_2 */
} vf_solve_stats;

vf_status vf_solve(const vf_hmat* h, const float* rho, const float* E, int64_t lde, float* B, int64_t ldb,
                   int32_t R, const vf_solve_opts* opts, vf_solve_stats* stats, vf_stream stream);

/* vf_solve with HOST buffers: E (nf x R, column-major, lde), rho (nf or
 * NULL) and B are ordinary (preferably pinned) CPU memory; the host-to-device
 * copy of E and rho, the solve and the device-to-host copy of B all run in
 * the call, which returns once B is on the host. */
vf_status vf_solve_host(const vf_hmat* h, const float* rho, const float* E, int64_t lde, float* B, int64_t ldb,
                        int32_t R, const vf_solve_opts* opts, vf_solve_stats* stats, vf_stream stream);

/* Many meshes in one launch per phase and sweep (the batching workload of
 * Section 1's many right-hand sides, over many meshes): nmeshes problems,
 * each with its own F, rho (device or NULL: opts->rho), E, B (device,
 * column-major, facet order) and R.  The call solves the block-diagonal
 * system diag(F_1 ... F_k) (vf_hmat_stack, built on the first call for
 * this list of handles and kept until one of them is destroyed) with R =
 * max R_k columns, so every multiply is one work list over all meshes' row
 * tiles; convergence is judged per mesh and per column.  stats: host array
 * of nmeshes entries (sweeps and kernels are the shared ones) or NULL.
 * Errors: VF_E_INVAL (null or mismatched arguments), VF_E_NOCONV (B still
 * written), VF_E_NOMEM, VF_E_CUDA, VF_E_TIMEOUT. */
vf_status vf_solve_batched(const vf_hmat* const* F, int32_t nmeshes, const float* const* rho,
                           const float* const* E, const int64_t* lde, float* const* B, const int64_t* ldb,
                           const int32_t* R, const vf_solve_opts* opts, vf_solve_stats* stats,
                           vf_stream stream);

/* ---------------------------------------------------------- thermal
 * Section 5.1, equilibrium temperatures for R sun positions (columns of
 * E = Q_direct): with W = diag(albedo) Q_vis,
 *   W = diag(albedo) E + diag(albedo) F W      (Eq. time-indep-system-1, a
 *   Q_vis = E + F W                             radiosity system, rho = albedo)
 *   (I - F) Q_IR = F ((I - diag(albedo)) Q_vis + H)   (Eq. time-indep-system-2,
 *                                                      rho = 1)
 *   eps sigma T^4 = (1 - albedo) Q_vis + eps Q_IR      (Eq. 3d-equilbr, FP64,
 *                                                      sigma = 5.670374419e-8)
 * Q_vis = Q_direct + Q_refl.  Both solves are vf_solve calls (rtol,
 * max_iter, precision, refine as there; the multiplies between them use the
 * FP32 factors when refine = 1, else the sweeps' precision).  albedo,
 * emissivity (device FP32 [N]) and H (interior heat flux, device [N]) may
 * be NULL: the uniform opts values (H = 0) then apply.  E, Qvis, Qir, T:
 * device FP32, column-major, face order (lde, ld); Qvis and Qir may be NULL
 * (not returned).  stats: host, 2 entries (the Q_vis and Q_IR solves) or
 * NULL.  Synchronous.  The IR system converges while F's spectral radius is
 * below 1 (open surfaces).  Errors: VF_E_INVAL, VF_E_NOCONV (outputs still
 * written), VF_E_NOMEM, VF_E_CUDA, VF_E_TIMEOUT. */
typedef struct {
    double rtol;       /* both solves, default 1e-6 */
    int32_t max_iter;  /* per Jacobi loop, default 200 */
    int32_t precision; /* vf_precision of the sweeps */
    int32_t refine;    /* 1: mixed-precision refinement (BF16 / FP8 sweeps) */
    float albedo;      /* uniform albedo (when albedo is NULL), in [0, 1) */
    float emissivity;  /* uniform emissivity (when emissivity is NULL), in (0, 1] */
} vf_equilibrium_opts;

vf_status vf_equilibrium(const vf_hmat* h, const float* E, int64_t lde, int32_t R, const float* albedo,
                         const float* emissivity, const float* H, const vf_equilibrium_opts* opts, float* Qvis,
                         float* Qir, float* T, int64_t ld, vf_solve_stats* stats, vf_stream stream);

/* Algorithm 6 (Section 5.2), one time step of the fluxes of R independent
 * scenarios (columns):
 *   Q_refl' = F diag(albedo) (Q_direct' + Q_refl)
 *   Q_IR'   = F (Q_rad + (I - diag(emissivity)) Q_IR)
 *   Q_abs'  = (I - diag(albedo)) (Q_direct' + Q_refl') + diag(emissivity) Q_IR'
 * The two multiplies by F run as ONE multiply of 2R right-hand sides in
 * precision p (vf_apply).  Edirect_next = Q_direct' and Qrad = eps sigma T^4
 * of the current step are read; Qrefl and Qir are read (step n) and
 * overwritten (step n + 1); Qabs is written.  The caller advances the
 * subsurface model (or, with no heat storage, sets Q_rad' = Q_abs').
 * albedo, emissivity: device FP32 [N] or NULL (then albedo_u,
 * emissivity_u).  All blocks: device FP32, column-major, face order,
 * leading dimension ld.  Asynchronous on `stream`.  Errors: VF_E_INVAL,
 * VF_E_NOMEM, VF_E_CUDA. */
vf_status vf_flux_step(const vf_hmat* h, vf_precision p, int32_t R, const float* albedo, const float* emissivity,
                       float albedo_u, float emissivity_u, const float* Edirect_next, float* Qrefl, float* Qir,
                       const float* Qrad, float* Qabs, int64_t ld, vf_stream stream);

/* ------------------------------------------------------------ autotuning
 * What the multiply of one matrix runs with, per (precision, R): the
 * CUDA-core path's right-hand sides per pass (its RHS tile), whether BF16
 * or FP8 multiplies of >= 16 columns use the tensor cores, and the RHS block: a
 * call with more columns runs in column blocks of this width (0: all
 * columns at once).  No counterpart in the paper (its multiply is one
 * library call per block); the choice only changes speed and rounding
 * order. */
typedef struct {
    int32_t rb;          /* 1, 2, 4 or 8 */
    int32_t tensor;      /* 0 or 1 */
    int32_t rhs_block;   /* 0 or a width < R */
    float us_per_rhs;    /* measured multiply time per right-hand side (autotuner) */
} vf_tune;

/* Times the multiply of h on seeded synthetic columns (device memory the
 * call allocates) for every candidate -- rb in {1, 2, 4, 8} (8 alone from
 * 16 columns up), the tensor path (BF16 or FP8, >= 16 columns), RHS blocks of R
 * and of 64, 128, 256, ... < R
 * -- and records the fastest per right-hand side for (prec, R) in the
 * handle (and for (prec, rhs_block) when it splits); later vf_apply,
 * vf_apply_tree and vf_solve calls with that precision and R use it.  out
 * (host, may be NULL) receives the choice.  The handle's workspaces for the
 * candidates stay cached until it is destroyed.  Errors: VF_E_INVAL,
 * VF_E_NOMEM, VF_E_CUDA, VF_E_TIMEOUT. */
vf_status vf_autotune(const vf_hmat* h, vf_precision prec, int32_t R, vf_tune* out, vf_stream stream);

/* Record a choice for (prec, R) by hand (as vf_autotune would); rb must be
 * 1, 2, 4 or 8, tensor 0 or 1, rhs_block 0 or in [1, R).  Errors: VF_E_INVAL. */
vf_status vf_tune_set(const vf_hmat* h, vf_precision prec, int32_t R, const vf_tune* t);

/* The block-diagonal composition of nmeshes matrices on one device (no
 * counterpart in the paper; it batches many meshes): facets numbered mesh
 * after mesh (facet f of mesh k is row off_k + f, off_k = the sizes of the
 * meshes before it), payloads copied, one segment per mesh.  A multiply or
 * solve of the result runs all meshes in the same launches, and solves judge
 * convergence per segment and column.  The inputs stay owned by the caller;
 * the result is a new handle (vf_hmat_destroy).  A stacked matrix saved to a
 * file loads back as one segment.  Errors: VF_E_INVAL, VF_E_NOMEM, VF_E_CUDA. */
vf_status vf_hmat_stack(const vf_hmat* const* F, int32_t nmeshes, vf_hmat** out);

/* Bytes of the tensor-core multiply's pages of h (the B operands: factors
 * in BF16, terms = 1, split in hi and lo, terms = 2, or FP8 E4M3, terms =
 * 3), building them if not yet built.  A record's B operand covers runs of
 * K-chunks (16 columns; 32 for FP8, one MMA's K) that hold a nonzero of one
 * of its pieces (CSR pieces densified there) and is padded to the MMA
 * shapes (the output rows to multiples of 16).  by_kind (5 entries or
 * NULL): the bytes of dense, CSR, U', V' and empty-tile records (headers
 * and B operands); the total adds each page's 16-byte header.  No
 * counterpart in the paper.  Errors: VF_E_INVAL (no BF16 / FP8 copy),
 * VF_E_NOMEM, VF_E_CUDA. */
vf_status vf_hmat_tensor_bytes(const vf_hmat* h, int32_t terms, int64_t* total, int64_t* by_kind);

/* Release what multiplies and solves cached on h: its workspaces (per R
 * and precision), its tensor-core pages and the stacked matrices that
 * vf_solve_batched built from it; later calls rebuild them on demand.  For
 * callers that hold many matrices.  Synchronises the device; no call on h
 * may be in flight.  No counterpart in the paper.  Errors: VF_E_INVAL,
 * VF_E_CUDA. */
vf_status vf_hmat_trim(vf_hmat* h);

/* Number of segments (stacked meshes) of a matrix; 1 for an assembled one, -1 for NULL. */
int32_t vf_hmat_nsegments(const vf_hmat* h);

/* ------------------------------------------------------------ save/load
 * Versioned binary file: header, block table and payload sections, each with
 * a CRC32.  Load rejects a bad magic, version or CRC with VF_E_CORRUPT. */
vf_status vf_hmat_save(const vf_hmat* h, const char* path);
vf_status vf_hmat_load(const char* path, int32_t device, vf_hmat** out);

#ifdef __cplusplus
}
#endif
#endif /* VF_H */
