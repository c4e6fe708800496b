/*
 * smr.h - C ABI of the GB300 MLFMA-SMR library (libsmr.so).
 *
 * Multilevel fast multipole matrix-vector product and GMRES solve of the
 * PMCHWT system whose unknowns are static-mode coefficients of the electric
 * and magnetic surface currents on each particle of a metasurface
 * (Corsaro, Miano, Tamburrino, Ventre, Forestiere, arXiv 2407.21724).
 *
 * Conventions shared by every call
 *  - Every call returns int: SMR_OK (0) or a negative SMR_E_* code; the
 *    message of the last failure is smr_last_error(ctx).  No call aborts,
 *    throws or exits.
 *  - Lengths are in units of the vacuum wavelength times opts.wavelength
 *    (wavelength = 1 means lengths in wavelengths).  Impedances are
 *    normalised by the vacuum impedance.  Time dependence e^{j w t} (Sec. II).
 *  - Complex numbers are interleaved (re, im) doubles (C99 double _Complex).
 *  - Unknown vector layout x[mu][c][n][r]: particle mu (scene order), current
 *    c (0 = electric J, 1 = magnetic M), mode n (N_perp transverse modes then
 *    N_par longitudinal ones, Sec. III), right-hand side r (innermost, R of
 *    them).  N = 2 N_psi p unknowns per right-hand side (Eq. 11).
 *  - "device" pointers are CUDA global-memory pointers on ctx's device; the
 *    caller owns them and keeps them alive until the call's work on `stream`
 *    is complete.  "host" pointers are read or written before the call
 *    returns.  `stream` is a cudaStream_t (NULL = legacy default stream).
 *  - The library owns all memory it allocates (tables, level spectra,
 *    Krylov basis) until smr_destroy.
 *  - Sign conventions: T_mn = -j k <psi_m, G psi_n> and
 *    K_mn = -<psi_m, psi_n x grad' g> (Eqs. 8, 9, T_far1 and Eq. 25 read
 *    together), right-hand side [<psi, E_inc>; <psi, H_inc>] (Eqs. 18-19).
 */
#ifndef SMR_H
#define SMR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smr_ctx smr_ctx;

enum {
  SMR_OK = 0,
  SMR_E_INVALID_ARG = -1,   /* bad size, pointer, option or value            */
  SMR_E_SHAPE = -2,         /* unknown shape id or inconsistent mode counts   */
  SMR_E_OOM = -3,           /* device or host allocation failed              */
  SMR_E_CUDA = -4,          /* a CUDA runtime call or kernel launch failed    */
  SMR_E_NOT_CONVERGED = -5, /* solve hit maxit before the tolerance          */
  SMR_E_BREAKDOWN = -6,     /* Arnoldi breakdown before convergence          */
  SMR_E_NAN = -7,           /* NaN or Inf in a residual                      */
  SMR_E_TIMEOUT = -8,       /* a bounded device-side wait ran out            */
  SMR_E_STATE = -9          /* call made before smr_set_scene, or similar    */
};

enum { SMR_PREC_FP64 = 0, SMR_PREC_FP32 = 1 };
enum { SMR_LRULE_FORMULA = 0, SMR_LRULE_DOUBLE = 1 };
enum {
  SMR_PRECOND_NONE = 0,
  SMR_PRECOND_BLOCKDIAG = 1,
  SMR_PRECOND_LEARNED = 2,
  SMR_PRECOND_NEAR = 3,
  SMR_PRECOND_CLUSTER = 4
};

/* Options of a context (smr_default_opts fills the defaults in brackets). */
typedef struct {
  int device;         /* CUDA device ordinal [0]                                 */
  double wavelength;  /* vacuum wavelength in the caller's length unit [1.0]     */
  double pitch;       /* finest group size = lattice spacing [0.5]: each particle
                         is its own finest group (Sec. IV, Fig. 1a)              */
  int L0;             /* truncation order at the finest level [10] (Sec. V)      */
  int level_rule;     /* L above the finest level: SMR_LRULE_FORMULA uses
                         L = kd + 1.8 d0^{2/3} (kd)^{1/3}, d = sqrt(2) x box size
                         (Sec. IV); SMR_LRULE_DOUBLE uses L0 2^s (Sec. V)  [0]   */
  double digits;      /* d0 of the truncation formula [3.0]                       */
  int n_theta;        /* surface rule per particle: Gauss-Legendre nodes in
                         cos(theta) [16]                                          */
  int n_phi;          /* and uniform phi nodes [32]                               */
} smr_opts;

void smr_default_opts(smr_opts* opts);

/* Create a context on opts->device.  *ctx is NULL on failure (the return code
 * says why; no message object exists then). */
int smr_create(smr_ctx** ctx, const smr_opts* opts);

/* Free every device and host allocation of the context.  NULL is a no-op. */
int smr_destroy(smr_ctx* ctx);

/* Message of the last failing call on ctx ("" if none).  Owned by ctx. */
const char* smr_last_error(const smr_ctx* ctx);

/* Register a sphere of the given radius whose currents are expanded in its
 * closed-form static modes (Sec. III, Eqs. 21-25: vector spherical harmonics
 * grad_1 Y_lm / (a sqrt(l(l+1))) and r x that), n_perp transverse and n_par
 * longitudinal ones, l ascending, real harmonics in the order m = 0, 1c, 1s,
 * 2c, 2s, ...  All shapes of a context must share n_perp + n_par.
 * *shape_id receives the new id (0, 1, ...).  Must precede smr_set_scene. */
int smr_add_sphere(smr_ctx* ctx, double radius, int n_perp, int n_par, int* shape_id);

/* Register a shape given as data instead of in closed form: the form in
 * which the static modes of a meshed particle (Sec. V, stages ii and iv: RWG
 * star/loop eigenfunctions mapped to the surface) reach the solver.  Host
 * inputs, copied:
 *   pts[n_q][3]   surface quadrature points relative to the particle centre
 *   wts[n_q]      their weights (area elements; >= 0)
 *   modes[n_psi][n_q][4]  per mode and point the tangential field (x, y, z)
 *                 and its surface divergence, n_psi = n_perp + n_par, the
 *                 n_perp transverse modes first
 *   self_block[2 n_psi][2 n_psi]  complex (re, im interleaved), row-major:
 *                 Z_s of Eq. 16 with mu = nu for the media that will be
 *                 passed to smr_set_scene, [electric; magnetic] as in the
 *                 unknown vector.
 * Patterns (Eq. 26), neighbour blocks, right-hand sides and fields are then
 * computed from these samples exactly as for the closed-form spheres.
 * 1 <= n_q <= 8192; all shapes of a context share n_psi.  The points' largest
 * distance from the z axis must stay below half the pitch.  Must precede
 * smr_set_scene.  smr_add_shape_mesh produces these data from a mesh. */
int smr_add_shape_sampled(smr_ctx* ctx, int n_q, const double* pts, const double* wts, int n_perp, int n_par,
                          const double* modes, const double* self_block, int* shape_id);

/* Register a shape given by a closed triangle mesh (Sec. III and Sec. V,
 * stages i, ii and iv), host inputs, copied:
 *   verts[nv][3]   vertex positions relative to the particle centre
 *   tris[nt][3]    vertex indices, counter-clockwise seen from outside
 * The mesh must be a closed, consistently oriented, genus-0 surface with
 * outward normals (else SMR_E_SHAPE), 4 <= nt <= 1800.  RWG functions live
 * on its edges (edge = vertex pair (i, j), i < j, edges in lexicographic
 * order; the current flows out of the triangle whose vertex cycle runs
 * i -> j).  On the host in FP64 the call solves the two static eigenproblems
 * of Sec. III (Eqs. 21-25) in Galerkin form: the electrostatic one in star
 * functions, A_par v = gamma G v with A_par = <div s, g0 div' s'>, and the
 * magnetostatic one in loop functions, A_perp = <l, g0 l'>, G the Gram
 * matrix, g0 = 1/(4 pi R); inner integrals over each source triangle in
 * closed form, outer integrals by Radon's 7-point degree-5 rule, symmetric
 * parts diagonalised.  It keeps the n_perp largest gamma_perp and the n_par
 * smallest gamma_par (Sec. III), modes normalised to <psi, psi> = 1 with
 * their largest RWG coefficient positive, transverse modes first.  The
 * solver sees the modes sampled at a 3-point degree-2 rule on every
 * triangle (n_q = 3 nt points, as smr_add_shape_sampled).  smr_set_scene
 * computes the self block for the scene's media on the GPU in FP64: the
 * PMCHWT operators of both media on the modes, the 1/R and grad(1/R) parts
 * of the inner integrals in closed form (Sec. IV: Graglia 1993, Hodges 1997),
 * the remainders and the outer integrals by the 7-point rule, the K
 * operator as a principal value.  Must precede smr_set_scene.  The particle's
 * largest distance from the z axis must stay below half the pitch.  The
 * modes depend on the shape alone: the library keeps the last 32 solves of
 * the process and reuses one for an identical mesh and mode counts. */
int smr_add_shape_mesh(smr_ctx* ctx, int nv, const double* verts, int nt, const int* tris, int n_perp,
                       int n_par, int* shape_id);

/* A copy of shape `base` rotated by `angle` radians about the z axis through
 * the particle centre (the in-plane rotations of the brick and nanofin arrays
 * of Sec. V; the PB-phase lens rotates each fin by its own angle).  The
 * copy's sample points and mode fields are the base's carried by the
 * rotation R: psi'(R r) = R psi(r); weights, surface divergences, static
 * eigenvalues, RWG coefficients (smr_shape_modes) and the self block are the
 * base's (the PMCHWT operators commute with rotations).  Patterns, near
 * blocks and right-hand sides are computed for the rotated samples like any
 * other shape's.  The base must be a meshed or sampled shape (SMR_E_SHAPE for
 * a closed-form sphere, which rotation leaves unchanged); rotating a rotated
 * copy composes the angles.  Must precede smr_set_scene. */
int smr_add_shape_rotated(smr_ctx* ctx, int base, double angle, int* shape_id);

/* The static modes of a meshed shape: *n_psi and *n_edges (each if
 * non-NULL) receive the mode count and the RWG count n_e, M (if non-NULL)
 * the mode -> RWG matrix of Eq. 20
 * [n_psi][n_e] (psi_i = sum_e M[i][e] f_e), gamma (if non-NULL) the kept
 * eigenvalues [n_psi] (transverse first).  SMR_E_INVALID_ARG for a shape
 * that is not meshed. */
int smr_shape_modes(smr_ctx* ctx, int shape_id, int* n_psi, int* n_edges, double* M, double* gamma);

/* The self block Z_s (Eq. 16 with mu = nu) that the current scene uses for
 * a shape: host Z[2 n_psi][2 n_psi] complex (re, im interleaved),
 * row-major.  Needs smr_set_scene. */
int smr_self_block(smr_ctx* ctx, int shape_id, double* Z);

/* The static-mode solve of smr_add_shape_mesh alone, on the host (no
 * context, no GPU): same inputs and outputs as smr_add_shape_mesh followed
 * by smr_shape_modes.  SMR_E_SHAPE for a mesh it rejects. */
int smr_mesh_static_modes(int nv, const double* verts, int nt, const int* tris, int n_perp, int n_par,
                          int* n_edges, double* M, double* gamma);

/* Set the scene: p particles with host centres[p][3] and host shape_ids[p],
 * inner medium (eps_in, mu_in) and background (eps_out, mu_out), each a
 * complex relative value {re, im}.  Each particle belongs to the cell of a
 * square lattice of spacing opts.pitch (origin: the smallest x and y of the
 * centres) nearest its centre; the quadtree of Sec. IV is built over the
 * cells in the plane z0 = the mean height of the centres.  On a lattice
 * (every centre on a lattice point of z0, one per cell) each particle is its
 * own finest group.  A centre off its cell's lattice point (a jittered
 * lattice, a spiral, a layer of a 2.5D scene above or below z0; Sec. V)
 * keeps its 3D displacement: aggregation and receive shift its spectra to
 * and from the cell centre, and its exterior near blocks are computed for
 * the exact centre offsets, one block per distinct (shape, shape, offset).
 * Where a cell holds several particles the finest groups are the occupied
 * cells: a cell's outgoing spectrum is the sum of its particles', each
 * particle receives its cell's incoming spectrum, and the near pairs are all
 * pairs in the same or adjacent cells.  Displaced scenes must keep
 * neighbouring particles apart (bounding cylinders about z) and every
 * particle within distance opts.pitch of its cell centre (bounding radius
 * plus displacement), else SMR_E_INVALID_ARG; they run the near product,
 * aggregation and receive on the CUDA cores.  The learned parts and the
 * cluster preconditioner need at most one particle per cell.
 * Builds the quadtree, interaction lists, k-space grids, and on the GPU in
 * FP64: the patterns (Eq. 26), translation tables (Eq. 23) and near blocks
 * (Eq. 16; exterior blocks by surface quadrature, self blocks in closed form),
 * and the block-diagonal preconditioner (Sec. V, stage v).  Only real
 * (lossless) permittivities and permeabilities are accepted.  May be called
 * again to replace the scene. */
int smr_set_scene(smr_ctx* ctx, int p, const double* centres, const int* shape_ids,
                  const double eps_in[2], const double mu_in[2],
                  const double eps_out[2], const double mu_out[2]);

/* Several independent arrays in one context (a ragged batch): particle i
 * belongs to array array_ids[i] (0 .. n_arrays-1, every id used); each array's
 * host centres are in its own frame and follow the rules of smr_set_scene on
 * its own square lattice of spacing opts.pitch (cells, displacements, several
 * particles per cell).  The arrays share the shapes, media and every table, and
 * one smr_matvec covers all of them, but no interaction couples two arrays:
 * each keeps its own quadtree (levels capped at the top level of the largest
 * array), its own near pairs and its own interaction lists, so the product
 * is block diagonal over arrays.  The unknown vector stacks the arrays'
 * particles in the given order; plane-wave right-hand sides use each
 * particle's own-frame centre.  smr_solve then solves all arrays together
 * (the tolerance applies to the stacked residual). */
int smr_set_scene_arrays(smr_ctx* ctx, int p, const double* centres, const int* shape_ids,
                         const int* array_ids, const double eps_in[2], const double mu_in[2],
                         const double eps_out[2], const double mu_out[2]);

/* Sizes of the current scene. */
typedef struct {
  int p, n_psi, n_shapes, n_levels, n_arrays;
  long long n_unknowns;     /* 2 n_psi p                                       */
  int L[16], K[16], n_box[16], n_il[16];  /* per level s < n_levels          */
  long long n_near_pairs;   /* particle pairs in the near SpMV (self included) */
  int n_near_blocks;        /* distinct near blocks stored                     */
  double device_bytes;      /* tables + one set of level spectra (R = 1)       */
  int column_lanes;         /* columns in flight in FP32 products with R > 1   */
} smr_info_t;
int smr_info(smr_ctx* ctx, smr_info_t* info);

/* Right-hand sides of R unit plane waves E = pol exp(-j k khat . r),
 * H = khat x E / zeta_out (Eqs. 5, 18, 19): host khat[R][3] (unit vectors),
 * host pol[R][3] complex.  Writes device b[N][R] (layout above). */
int smr_rhs_plane_waves(smr_ctx* ctx, int R, const double* khat, const double* pol,
                        void* b, void* stream);

/* The hot path: y = Z x for R right-hand sides at once (Sec. IV): near
 * block-sparse product plus aggregation, interpolation, translation,
 * anterpolation and receive.  precision SMR_PREC_FP64 computes every step in
 * FP64; SMR_PREC_FP32 computes the steps in FP32 from FP32 copies of the
 * FP64-generated tables (x and y stay FP64 complex).  device x, y [N][R]. */
int smr_matvec(smr_ctx* ctx, int R, const void* x, void* y, int precision, void* stream);

/* Same product replayed from a CUDA graph: the first call for a given
 * (x, y, R, precision) captures every launch of smr_matvec on an internal
 * stream (ordered after the work already queued on `stream`) and later calls
 * launch the graph on `stream`, removing the per-kernel launch cost.  The
 * graph keeps the device addresses of x, y and of the library's buffers:
 * reuse it only while x and y stay allocated (smr_set_scene and a change of
 * R or precision drop all graphs).  At most 16 graphs are kept. */
int smr_matvec_graph(smr_ctx* ctx, int R, const void* x, void* y, int precision, void* stream);

/* Same, split: y_near = near-field part, y_far = MLFMA far part (either may
 * be NULL).  For per-stage parity checks. */
int smr_matvec_parts(smr_ctx* ctx, int R, const void* x, void* y_near, void* y_far,
                     int precision, void* stream);

/* Same as smr_matvec with HOST x and y (pageable or pinned): copies in,
 * multiplies, copies out on `stream`, and synchronises it before returning. */
int smr_matvec_host(smr_ctx* ctx, int R, const double* x, double* y, int precision,
                    void* stream);

/* Selects where the FP32 product runs its dense contractions for one
 * right-hand side: 1 (default) on the tensor cores (tcgen05, split TF32: each
 * FP32 operand as a sum of two TF32 values, three MMAs per step, FP32
 * accumulation), 0 on the FP32 CUDA cores.  The steps are aggregation and
 * receive (Eqs. 24-26), which need particles centred on their lattice
 * sites, and the near-field product (Eq. 16 blocks; pairs sharing a block
 * form one GEMM, one launch per lattice offset).  All need 4 n_psi <= 128;
 * otherwise the CUDA-core path runs.  The paper has no counterpart (it ran
 * on a CPU); both give the FP32 product to FP32 accuracy.  Drops captured
 * products (smr_matvec_graph) so the next call captures the new choice. */
int smr_set_tensor_cores(smr_ctx* ctx, int enable);

/* Times the launch variants of the product for one right-hand side in
 * `precision` on this scene and keeps the fastest for later products (no
 * counterpart in the paper).  Per level: translation with 8x8 target tiles
 * and the full or half direction chunk, 4x4 tiles, threads along the
 * directions (levels of at most 1024 boxes), or one CTA per direction chunk
 * over the whole level (at most 256 boxes); interpolation by the staged
 * kernel (FP32: child theta-row bands bulk-copied into shared memory) or by
 * the gather kernel with the full or half theta-row tile; anterpolation by
 * the staged kernel (FP32, where its tile fits) or by the gather kernel with
 * the full or half column chunk, 256-thread CTAs or one CTA per parent box
 * (FP32); for SMR_PREC_FP32 also
 * aggregation, receive and the near-field product on the tensor cores or the
 * CUDA cores (the near product on the tensor cores only if at least 5 %
 * faster).  Each variant is timed over three products (CUDA events around
 * every launch, the fastest kept).  Uses and overwrites the context's scratch
 * buffers; drops captured products.  1 <= R <= 256: the variants are timed on
 * single-column products, and FP32 products with R > 1 run their columns
 * through the same single-column kernels.  For SMR_PREC_FP32 and R > 1 it
 * then times R-column graph products with 1, 2, 4 and 8 column lanes (at
 * most R; smr_set_column_lanes) and keeps the fastest. */
int smr_autotune(smr_ctx* ctx, int R, int precision, void* stream);

/* Synchronises `stream` and reports errors found on the device since the
 * last check: SMR_E_TIMEOUT if a tensor-core pipeline wait ran out (that
 * product's result is invalid; the kernel stopped issuing, waited for the
 * copies and MMAs it had already issued, freed its tensor memory and
 * returned, so the context stays usable).  smr_matvec_host and smr_solve
 * make this check themselves. */
int smr_sync(smr_ctx* ctx, void* stream);

/* Polling limit of every bounded wait in the tensor-core kernels (rounds of
 * mbarrier try_wait before a wait gives up and the product reports
 * SMR_E_TIMEOUT).  rounds < 0 restores the default (2^24); 0 makes every
 * wait that has to wait give up at once, which a test uses to exercise the
 * give-up path without faulting anything.  A CTA that gives up still drains
 * its in-flight copies and MMAs with the default bound.  Drops captured
 * products.  No counterpart in the paper. */
int smr_set_wait_limit(smr_ctx* ctx, long long rounds);

/* Columns in flight in an FP32 product with R > 1 right-hand sides (1..16,
 * default 4).  Such a product runs its columns through the single-column
 * kernels; the columns are dealt round-robin to `lanes` lanes, each with its
 * own FP32 spectra, separable-pass and near-product buffers (about the
 * memory of one single-column product per lane, allocated on first use and
 * kept until smr_set_scene or smr_destroy) and its own stream, forked from
 * the caller's stream and joined before the call's last launch.  The lanes
 * overlap the launches of the upper levels, which one column leaves mostly
 * idle.  Every column's result is the same as alone (the same kernels on
 * the same data).  SMR_E_INVALID_ARG outside 1..16.  Drops captured
 * products.  No counterpart in the paper. */
int smr_set_column_lanes(smr_ctx* ctx, int lanes);

/* Overlap inside one product (1 = default, 0 = every step in order on the
 * caller's stream).  Overlapped, the near-field product runs on a side
 * stream next to the far field, and the translation of each level (Eq. 23)
 * on a second side stream as soon as that level's outgoing spectra exist;
 * the anterpolation into a level waits for its translation and the receive
 * for the near product (events; in a captured graph these are its edges).
 * The small upper-level launches then overlap the upward pass.  The result
 * is bit for bit that of the ordered product (the same kernels on the same
 * data).  Drops captured products.  No counterpart in the paper. */
int smr_set_overlap(smr_ctx* ctx, int enable);

/* z = blockdiag(Z_s^-1) r over particles: the block-diagonal preconditioner
 * of Sec. V (each block the inverse of the particle's self block).
 * device r, z [N][R]; precision as in smr_matvec. */
int smr_precond(smr_ctx* ctx, int R, const void* r, void* z, int precision, void* stream);

/* z = C^-1 r with C the cluster block-Jacobi matrix: the particles are
 * grouped into 2 x 2 clusters of lattice cells (the quadtree's level-1
 * boxes of each array) and C holds, per cluster, the cluster's part of the
 * near-field matrix (the members' self blocks, Eq. 16 with delta = 1, and
 * the near blocks between them, Eq. 16 with delta = 0).  The inverses are
 * computed on first use on the GPU in FP64 (Gauss-Jordan elimination with
 * partial pivoting, 16 (2 n_psi)^2 complex values per cluster kept in FP64
 * and FP32 until smr_set_scene or smr_destroy) and applied in `precision`.
 * Needs 8 n_psi <= 256; SMR_E_INVALID_ARG if a cluster matrix is singular.
 * Not in the paper (Sec. V uses the block-diagonal preconditioner of
 * smr_precond); smr_solve uses it with precond = SMR_PRECOND_CLUSTER.
 * device r, z [N][R]. */
int smr_precond_cluster(smr_ctx* ctx, int R, const void* r, void* z, int precision, void* stream);

typedef struct {
  double tol;      /* true relative residual ||b - Z x|| / ||b|| target [1e-4] */
  int maxit;       /* maximum inner iterations in total [2000]                 */
  int restart;     /* Krylov dimension before restart; 0 = maxit [0]           */
  int precond;     /* SMR_PRECOND_* [SMR_PRECOND_BLOCKDIAG]: BLOCKDIAG is the
                      paper's (Sec. V), M^-1 = blockdiag(Z_s)^-1 = D^-1;
                      NEAR adds the neighbour coupling by near_sweeps Jacobi
                      sweeps over the near-field matrix Z_near = D + N
                      (z <- z + D^-1 r - D^-1 Z_near z from z = D^-1 r, i.e.
                      the truncated Neumann series of Z_near^-1; it helps
                      only while the neighbour coupling is weaker than the
                      self blocks, rho(D^-1 N) < 1; not in the paper);
                      CLUSTER applies the inverse of each 2 x 2 lattice
                      cluster's near-field matrix (smr_precond_cluster; not
                      in the paper); LEARNED needs smr_nn_precond first and
                      R = 1                                                  */
  int precision;   /* SMR_PREC_FP64: plain GMRES on the FP64 product;
                      SMR_PREC_FP32: iterative refinement, outer residual with
                      the FP64 product, inner GMRES on the FP32 product and
                      preconditioner.  The inner Krylov basis is stored in
                      FP32 (Gram-Schmidt products in FP32, sums over the
                      vector, Hessenberg and Givens in FP64) [FP64]          */
  int max_outer;   /* refinement steps for SMR_PREC_FP32 [8]                   */
  int use_x0;      /* 1: x holds the initial guess on entry; 0: start at 0.
                      A column whose guess has a true residual above ||b||
                      (worse than zero) starts at 0 instead                 */
  int fallback_iters; /* SMR_PRECOND_LEARNED: if the residual has not dropped
                      10x after this many iterations, the solve switches to
                      SMR_PRECOND_BLOCKDIAG from the current iterate [40]   */
  int near_sweeps;  /* SMR_PRECOND_NEAR: Jacobi sweeps, 1..8 [1]             */
  int poly_degree;  /* 0 off, or 2..16 [0]: a polynomial in B = A M^-1 on top
                       of `precond`, the iterations run on B p(B).  p comes
                       from poly_degree Arnoldi steps of B started from b (in
                       the precision the iterations use): its roots, the
                       harmonic Ritz values (the roots of the GMRES residual
                       polynomial, 1 - x p(x) = prod (1 - x / theta_i)), are
                       applied in Leja order.  Each iteration then costs
                       poly_degree products and Gram-Schmidt against fewer
                       basis vectors.  One right-hand side only (ignored for
                       R > 1).  Not in the paper                             */
} smr_solve_opts;

typedef struct {
  int iters;            /* Arnoldi steps (one product each)                    */
  int matvecs_fp64;     /* FP64 products incl. true-residual checks            */
  int matvecs_fp32;     /* FP32 products                                       */
  int outer;            /* refinement steps (SMR_PREC_FP32)                    */
  int reorth;           /* Arnoldi steps that needed a second Gram-Schmidt pass */
  double resid_true;    /* max over r of ||b - Z_64 x|| / ||b|| at exit        */
  double seconds;       /* wall time of the call                               */
  double seconds_product;  /* device time of the Arnoldi products             */
  double seconds_precond;  /* ... of the preconditioner applications           */
  double seconds_orth;     /* ... of Gram-Schmidt (inner products, updates)     */
  int fallback_x0;      /* columns whose initial guess was replaced by zero     */
  int fallback_precond; /* 1 if the learned preconditioner was replaced by the
                           block-diagonal one (at iteration iters_learned)      */
  int iters_learned;    /* iterations run with the learned preconditioner       */
} smr_solve_stats;

void smr_default_solve_opts(smr_solve_opts* o);

/* Solve Z x = b for R right-hand sides with right-preconditioned GMRES
 * (Sec. V, stage v).  device b, x [N][R].  The R systems run in lockstep,
 * one R-column product per Arnoldi step; each stops updating once its own
 * true residual meets tol.  Returns SMR_E_NOT_CONVERGED (x still holds the
 * last iterate) if maxit is reached first.  stats may be NULL. */
int smr_solve(smr_ctx* ctx, int R, const void* b, void* x, const smr_solve_opts* opts,
              smr_solve_stats* stats, void* stream);

/* Scattered far-field amplitude F(rhat), E_s ~ F exp(-j k r)/r, at host unit
 * directions dirs[n_dir][3] from device coefficients x[N][R]:
 * F = (j k / 4 pi) [zeta (I - rr) J_hat - r x M_hat] with
 * J_hat = int J exp(j k rhat . r') dS'.  Writes device F[n_dir][3][R]
 * (Cartesian components). */
int smr_far_field(smr_ctx* ctx, int R, const void* x, int n_dir, const double* dirs,
                  void* F, void* stream);

/* Scattering and extinction cross sections of each column of device
 * coefficients x[N][R] (Sec. V outputs).  C_sca is the scattered power
 * integral of |F|^2 over the unit sphere, taken with an n_theta-point
 * Gauss-Legendre rule in cos(theta) times a 2 n_theta-point trapezoid rule
 * in phi (exact for |F|^2 band-limited to degree 2 n_theta - 1).  C_ext
 * follows the optical theorem at column r's incident direction:
 * C_ext = -(4 pi / k) Im(conj(pol_r) . F(khat_r)) / |pol_r|^2.  Host inputs
 * khat[R][3] (normalised here) and pol[R][3] complex (interleaved re, im),
 * the plane wave column r was excited with; host outputs csca[R], cext[R]
 * (units of length^2).  1 <= n_theta <= 2048; zero khat or pol gives
 * SMR_E_INVALID_ARG.  Synchronises `stream`. */
int smr_cross_sections(smr_ctx* ctx, int R, const void* x, int n_theta, const double* khat,
                       const double* pol, double* csca, double* cext, void* stream);

/* Scattered E and H at host points pts[n_pt][3] (outside every particle) by
 * direct surface quadrature with the full Green's dyadic:
 * E = -zeta L{J} + K{M}, H = -K{J} - L{M}/zeta.  Writes device
 * EH[n_pt][6][R] (Ex, Ey, Ez, Hx, Hy, Hz). */
int smr_near_field(smr_ctx* ctx, int R, const void* x, int n_pt, const double* pts,
                   void* EH, void* stream);

/* One product with a per-launch breakdown.  For each kernel launch of
 * smr_matvec, in launch order: its name, level (-1 if none), ALGORITHMIC
 * bytes (every operand read once, every result written once; tables
 * included) and flops of that launch, and its device time in ms from CUDA
 * events recorded on `stream` around the launch.  Fills at most n_max
 * entries of `out`, sets *n_out to the number of launches, and synchronises
 * `stream`.  Same arguments otherwise as smr_matvec. */
typedef struct {
  char name[24];
  int level;
  double bytes;
  double flops;
  double ms;
} smr_launch_t;
int smr_profile_matvec(smr_ctx* ctx, int R, const void* x, void* y, int precision,
                       smr_launch_t* out, int n_max, int* n_out, void* stream);

/* Right-hand sides with one plane wave per array (R = 1): particle mu of
 * array a sees E = pol_a exp(-j k khat_a . r_mu) with r_mu its own-frame
 * centre (Eqs. 5, 18, 19).  host khat[n_arrays][3], pol[n_arrays][3] complex;
 * device b[N]. */
int smr_rhs_plane_waves_arrays(smr_ctx* ctx, const double* khat, const double* pol, void* b,
                               void* stream);

/* ---- Learned initial guess (no counterpart in the paper; it feeds the
 * GMRES of Sec. V a starting point).  A 4-layer MLP (F -> W -> W -> W -> O,
 * SiLU between layers, BF16 weights with FP32 master copies, FP32
 * activations and accumulation, Adam) maps the features of one scatterer to
 * its de-phased coefficients abar = alpha exp(+j k khat . r) / scale, with
 * F = 448: for each of the 48 lattice neighbours within 2 wavelengths
 * (pitch 0.5, 0 < dx^2 + dy^2 <= 16 cells, ordered by distance then angle)
 * a one-hot shape id (8) and a presence flag (1), the scatterer's own shape
 * one-hot (8), the incidence direction (3) and real polarisation (3), two
 * zeros; and O = 4 n_psi = [Re | Im] of [electric modes, magnetic modes].
 * Shape ids must be < 8.  Incidences are one per array (host khat[n_arrays][3],
 * pol[n_arrays][3] complex).  Parameters are stored layer by layer, W_l
 * row-major [in][out] then b_l [out]. */
int smr_nn_init(smr_ctx* ctx, int width, unsigned long long seed);   /* needs a scene */
long long smr_nn_num_params(smr_ctx* ctx);
int smr_nn_get_params(smr_ctx* ctx, float* params, long long n);     /* host, FP32 master */
int smr_nn_set_params(smr_ctx* ctx, const float* params, long long n);  /* resets Adam */
/* device feat[p][448] (float) for the scene's particles */
int smr_nn_features(smr_ctx* ctx, const double* khat, const double* pol, float* feat, void* stream);
/* device tgt[p][O] (float) from device coefficients x[N] (R = 1) */
int smr_nn_targets(smr_ctx* ctx, const double* khat, const void* x, double scale, float* tgt,
                   void* stream);
/* One Adam step on the mean squared error over n rows (rows idx[0..n) of
 * feat/tgt if idx, a device int array, is not NULL); n <= 8192.  *loss
 * (host, may be NULL) receives the loss before the step. */
int smr_nn_train_step(smr_ctx* ctx, int n, const float* feat, const int* idx, const float* tgt,
                      float lr, double* loss, void* stream);
/* Loss and its gradient (host grad[num_params], may be NULL) without a step. */
int smr_nn_loss_grad(smr_ctx* ctx, int n, const float* feat, const int* idx, const float* tgt,
                     double* loss, float* grad, void* stream);
/* Learned local-coupling preconditioner for one right-hand side (no
 * counterpart in the paper): from the network's prediction x_p (as
 * smr_nn_predict) and the isolated-particle response z = blockdiag(Z_s^-1) b
 * of the device right-hand side b[N], stores D = x_p / z per unknown with
 * |D| clamped to [0.1, 10] (0.1 where the ratio is zero or undefined).
 * smr_solve with precond = SMR_PRECOND_LEARNED (R = 1) then applies
 * M^-1 r = D (blockdiag(Z_s^-1) r).  D stays until the next call or scene. */
int smr_nn_precond(smr_ctx* ctx, const double* khat, const double* pol, double scale, const void* b,
                   void* stream);
/* x0 = scale * (Y_re + j Y_im) exp(-j k khat . r) for every particle: device
 * x0[N], ready for smr_solve with use_x0 = 1. */
int smr_nn_predict(smr_ctx* ctx, const double* khat, const double* pol, double scale, void* x0,
                   void* stream);

/* Measured arithmetic peak of the current CUDA device, in TFLOP/s (no
 * context needed): kind 0 = FP32 fused multiply-add, 1 = packed two-wide
 * FP32 multiply-add, 2 = FP64 fused multiply-add; 16 independent chains per
 * thread, 8 CTAs of 256 threads per SM, one warm-up launch, the second timed
 * with CUDA events (a few ms for FP32, about 20 ms for FP64).  These are the
 * denominators of the CUDA-core roofline.  SMR_E_INVALID_ARG for another
 * kind, SMR_E_CUDA if a launch fails. */
int smr_measure_peak(int kind, double* tflops);

/* Debug and parity access (host outputs, layouts as the oracle's):
 *  smr_copy_pattern: receiving patterns of a shape, [n_psi][2][K_0] complex
 *    (theta and phi components of Eq. 26 on the level-0 grid);
 *  smr_copy_translation: T_L(khat, X) of Eq. 23 at level s for the lattice
 *    offset X = (dx, dy) x box size, [K_s] complex (FP64 table);
 *  smr_copy_near_block: the stored near block for (shape_m, shape_n, dx, dy)
 *    (dx = dy = 0: self block), [2 n_psi][2 n_psi] complex row-major; on a
 *    scene with displaced particles, the first block of that key;
 *  smr_copy_pair_block: the near block Z^{mu nu} that the product applies to
 *    x_nu for y_mu (mu = nu: self block), same layout; SMR_E_INVALID_ARG if
 *    mu and nu are not a near pair;
 *  smr_copy_level: level-s outgoing (kind 0) or incoming (kind 1) spectra of
 *    the last product, [n_box][K_s][4][R] complex, in FP64. */
int smr_copy_pattern(smr_ctx* ctx, int shape, double* out);
int smr_copy_translation(smr_ctx* ctx, int level, int dx, int dy, double* out);
int smr_copy_near_block(smr_ctx* ctx, int shape_m, int shape_n, int dx, int dy, double* out);
int smr_copy_pair_block(smr_ctx* ctx, int mu, int nu, double* out);
int smr_copy_level(smr_ctx* ctx, int level, int kind, double* out, size_t n_doubles);

/* Parity access to the launch variants (the choices smr_autotune makes),
 * for one level (0 .. n_levels - 1) or every level (-1), for products in
 * `precision` with one right-hand side:
 *  SMR_STEP_TRANSLATE: 0 built-in rule, 1 / 2 8x8 target tiles with the full
 *    / half direction chunk, 3 4x4 tiles, 4 threads along the directions, 5
 *    one CTA per direction chunk over every box of the level (levels of at
 *    most a few hundred boxes: each source spectrum read once);
 *  SMR_STEP_INTERPOLATE (into the parent of `level`): 0 built-in rule (in
 *    FP32 the staged kernel, child theta-row bands bulk-copied into shared
 *    memory, where its tile fits), 1 / 2 the gather kernel with the full /
 *    half theta-row tile, 3 the staged kernel whose threads produce two
 *    neighbouring parent columns from one window of child columns (FP32);
 *  SMR_STEP_ANTERPOLATE (into `level`): 0 built-in rule (the gather kernel),
 *    1 half its column chunk, 2 256-thread CTAs, 4 the staged kernel (FP32,
 *    parent band bulk-copied, where its tile fits), 5 the gather kernel with
 *    one CTA per parent box serving its four children (FP32: each parent tap
 *    read once for the four quadrants' shifts).
 * A variant that does not apply to a level falls back to the built-in rule.
 * Drops captured products.  No counterpart in the paper. */
enum { SMR_STEP_TRANSLATE = 0, SMR_STEP_INTERPOLATE = 1, SMR_STEP_ANTERPOLATE = 2 };
int smr_set_variant(smr_ctx* ctx, int step, int level, int precision, int variant);

/* Right-hand sides of R plane waves, like smr_rhs_plane_waves, but the call
 * allocates and frees no device memory.  For callers that cannot call
 * cudaMalloc: an application whose device memory is fully reserved by its own
 * pool allocator (an allocation from inside the library could fail, or break
 * that budget), or a latency-critical loop that cannot accept the implicit
 * device synchronisation cudaMalloc and cudaFree may cause.
 *  - khat: device [R][3] unit vectors; pol: device [R][3] complex; b: device
 *    [N][R] output (layout above).  All three are caller-owned device buffers.
 *  - The intermediate per-shape sums ([n_shapes][n_psi][2][R] complex128)
 *    live in a fixed 4 MiB array in device global memory that every GPU which
 *    loads libsmr holds until the process exits.  A call needing more
 *    (n_shapes * n_psi * 2 * R * 16 bytes > 4 MiB, i.e. R > 512 with 8 shapes
 *    of n_psi = 32 modes per current) fails with SMR_E_INVALID_ARG and a
 *    message; split R.
 *  - The first call on a device looks up that array's device address (with
 *    the context's device made current) and caches it; make that first call
 *    before any stream capture.
 *  - All calls on a device share the one array, which keeps the last call's
 *    contents; calls that overlap on the GPU (different streams or threads
 *    without ordering) race on it.  Nothing in it needs clearing: every sum
 *    a call reads was written earlier in the same call.
 *  - The call makes the context's device current and leaves it current,
 *    like the other entry points.
 *  - This entry point has no counterpart in the paper; it computes what
 *    smr_rhs_plane_waves computes. */
int smr_rhs_plane_waves_static(smr_ctx* ctx, int R, const double* khat, const double* pol,
                               void* b, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SMR_H */
