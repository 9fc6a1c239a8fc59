/*
 * macroaim.h -- C ABI of libmacroaim: GB300-native macromodel + AIM solver for
 * scattering from large arrays of PEC elements.
 *
 * Method: U. R. Patel, P. Triverio, S. V. Hum, "A Macromodeling Approach to
 * Efficiently Compute Scattering from Large Arrays of Complex Scatterers"
 * (arXiv 1712.02443).  Every entry point cites the passage that defines what it
 * computes.
 *
 * Conventions
 *  - Every call returns mm_status (0 = MM_OK).  No exception or abort crosses
 *    the ABI.  mm_last_error(ctx) returns a context-owned message for the last
 *    failure on that context (valid until the next call on it).
 *  - Handles are opaque and owned by the library; free each with its *_destroy.
 *    Destroy arrays before the types they use, types before meshes, and all of
 *    them before their context.
 *  - Input arrays are owned by the caller and copied during the call.
 *  - Units: lengths in wavelengths (the caller scales), k0 in rad/length.
 *    Time convention exp(+j w t); G(R) = exp(-j k0 R)/(4 pi R).
 *  - Complex numbers are interleaved (re, im): double[2] for MM_C128,
 *    float[2] for MM_C64.
 *  - Vectors over the array's unknowns are element-major (all unknowns of
 *    element 0, then element 1, ...; Sec. III), with the right-hand sides
 *    innermost: entry (n, j) of an (N x nrhs) block is at index n*nrhs + j.
 *  - Arguments named *_dev are device pointers on the context's device;
 *    `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    stream-ordered: they return once the work is queued unless stated
 *    otherwise.
 *  - A context is not thread-safe: use one context per host thread.
 */
#ifndef MACROAIM_H
#define MACROAIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mm_status {
  MM_OK = 0,
  MM_EINVAL = 1,      /* invalid argument, mesh or configuration            */
  MM_ENOMEM = 2,      /* host or device allocation failed                   */
  MM_ECUDA = 3,       /* CUDA runtime error (message has the CUDA string)   */
  MM_ENOCONV = 4,     /* iterative solve stopped at max_iter unconverged    */
  MM_EBREAKDOWN = 5,  /* Krylov breakdown or non-finite residual            */
  MM_ETIMEOUT = 6,    /* a bounded device wait gave up                      */
  MM_EBUSY = 7,       /* resource in use                                    */
  MM_EINTERNAL = 8    /* internal consistency check failed                  */
} mm_status;

typedef enum mm_precision {
  MM_C64 = 0,       /* complex64 operator (FP32 FFT, SpMV, macromodel product)   */
  MM_C128 = 1,      /* complex128 operator (the plain FP64 GPU form)             */
  MM_C64_BF16 = 2,  /* complex64 operator, macromodel product on tensor cores   */
                    /* with BF16 inputs and FP32 accumulation (vectors: c64)     */
  MM_C64_F16 = 3,   /* same with FP16 inputs                                     */
  MM_C128_FF = 4    /* complex128 vectors and operator data; every stage of the   */
                    /* product in float-float arithmetic (each value an           */
                    /* unevaluated sum of two floats, Dekker 1971) on the FP32    */
                    /* pipe, FP64 between the stages: within 1e-12 of the MM_C128 */
                    /* product (relative 2-norm).  mm_apply and mm_apply_batch.   */
} mm_precision;

typedef struct mm_ctx mm_ctx;
typedef struct mm_mesh mm_mesh;
typedef struct mm_type mm_type;
typedef struct mm_array mm_array;

/* ------------------------------------------------------------------ context
 * device >= 0 : CUDA device ordinal (must be an sm_103 GPU);
 * device == -1: host-only context.  Set-up calls (meshes, element types,
 *   arrays) run and can be inspected; every device call returns MM_EINVAL.  */
mm_status mm_ctx_create(int device, mm_ctx** out);
void mm_ctx_destroy(mm_ctx* ctx);
const char* mm_last_error(const mm_ctx* ctx);
/* Number of worker threads used by host set-up (default: hardware threads). */
mm_status mm_ctx_set_threads(mm_ctx* ctx, int nthreads);

/* -------------------------------------------------------------------- mesh
 * A triangulated surface: vertices xyz (nv x 3, double), triangles tri
 * (nt x 3, int32, 0-based).  Scatterer surfaces S_m may be open; equivalent
 * surfaces must be closed, manifold and outward-oriented (counter-clockwise
 * seen from outside) -- Sec. II-A.  RWG functions live on interior edges,
 * numbered in lexicographic order of (min vertex, max vertex).
 * Errors: MM_EINVAL for indices out of range, degenerate triangles or
 * non-manifold edges.                                                        */
mm_status mm_mesh_create(mm_ctx* ctx, const double* xyz, int64_t nv, const int32_t* tri, int64_t nt,
                         mm_mesh** out);
/* n_rwg: number of RWG functions; closed: 1 if closed and outward-oriented.  */
mm_status mm_mesh_info(const mm_mesh* mesh, int64_t* n_rwg, int32_t* closed);
void mm_mesh_destroy(mm_mesh* mesh);

/* ------------------------------------------------------------ element type
 * Macromodel of one distinct element (Sec. II): fills the six Stratton-Chu
 * matrices of eqs. (EFIEdiscretized1)-(EFIEdiscretized2) (eqs. (Gm_EJ_1)-(G3)),
 * LU-factors G^(E^,H^) (eq. (Hdiscretized1)), forms A, B (eq. (JM)), T
 * (eq. (Tm1)) and the composed block M = T A^-1 B applied in eq.
 * (MV_product1), plus D (Sec. IV).  FP64; computed once per distinct element
 * and shared by every identical element of an array (Sec. III).  The fills
 * run on the host (all context threads); with a device context and a
 * scatterer of at least 1024 RWG functions the dense steps (LU factorisations
 * with partial pivoting, the solves and the products) run on that GPU,
 * otherwise on the host.
 * The dual functions of eq. (Ehat_expand) are built on the barycentric
 * refinement of `equiv`.  `equiv` must be closed; k0 > 0.                    */
typedef struct mm_em_opts {
  double k0;     /* wavenumber (2*pi for lengths in wavelengths)             */
  double eta0;   /* free-space impedance; <= 0 selects 376.730313668          */
} mm_em_opts;
mm_status mm_element_type_create(mm_ctx* ctx, const mm_mesh* scatterer, const mm_mesh* equiv,
                                 const mm_em_opts* opts, mm_type** out);
typedef enum mm_type_matrix_id {
  MM_MAT_M = 0,     /* T A^-1 B           (N^ x N^)  */
  MM_MAT_D = 1,     /* <f^_m, n x f^'_n>  (N^ x N^)  */
  MM_MAT_T = 2,     /* eq. (Tm1)          (N^ x N)   */
  MM_MAT_A = 3,     /* eq. (JM)           (N x N)    */
  MM_MAT_B = 4,     /* eq. (JM)           (N x N^)   */
  MM_MAT_GHH = 5,   /* G^(E^,H^)          (N^ x N^)  */
  MM_MAT_GHE = 6,   /* G^(E^,E^)          (N^ x N^)  */
  MM_MAT_PJ = 7     /* (D - G^(E^,H^) M)^-1 (N^ x N^): inverse of the element's
                       own block of the array system (block-Jacobi)          */
} mm_type_matrix_id;
/* Copies matrix `which` (row-major, complex128 interleaved) into out_host
 * (may be NULL to query the shape).  rows/cols receive its shape.            */
mm_status mm_type_matrix(const mm_type* type, int32_t which, double* out_host, int64_t* rows, int64_t* cols);
/* Unknown counts of a type: n_scat = N (RWG on the scatterer), n_equiv = N^. */
mm_status mm_type_info(const mm_type* type, int64_t* n_scat, int64_t* n_equiv);
void mm_type_destroy(mm_type* type);

/* ------------------------------------------------------------------- array
 * Array of n_elem elements (Sec. III); element e has type types[e] and is
 * translated by offsets_xyz[3e..3e+2].  Builds the AIM operator of Sec. V:
 * grid nodes at phase + h*Z^3, stencils of (order+1)^3 nodes, projection
 * weights matching all moments up to degree `order` per axis, the Green's
 * spectrum of the zero-padded grid, and the precorrected near-field matrix
 * over basis pairs whose stencil anchors are within n_nf cells (Chebyshev).
 * Relative element offsets must be integer multiples of h (lattice-aligned
 * elements share projection weights and near-field blocks).
 * With a device context the operator is uploaded to the device.
 * Errors: MM_EINVAL (offsets off the lattice, a basis centroid on a rounding
 * tie of the grid, order < 1), MM_ENOMEM, MM_ECUDA.                          */
typedef struct mm_aim_opts {
  double h;          /* grid spacing                                          */
  int32_t order;     /* stencil order N_O (N_O + 1 nodes per axis)            */
  int32_t n_nf;      /* near-field radius N_NF in grid cells; -1: no near-field
                        correction (far-field operator only, for studies)     */
  double phase[3];   /* position of one grid node                             */
  int32_t near_csr;  /* the near field is always kept as translation-invariant
                        (type, type, lattice offset) blocks, which the device
                        products use; the expanded CSR matrix is assembled
                        for inspection (MM_EXPORT_NEAR_*) and for the
                        complex128 products, which stream it (the dense blocks
                        cost more at GB300's FP64 rate): 0 = automatic (always
                        on host-only contexts; on a device when its values in
                        both precisions and its columns fit in 8 GiB), 1 =
                        always, 2 = never                                      */
} mm_aim_opts;
mm_status mm_array_create(mm_ctx* ctx, int64_t n_elem, const mm_type* const* types, const double* offsets_xyz,
                          const mm_aim_opts* opts, mm_array** out);
typedef struct mm_array_info {
  int64_t n_unknowns;    /* N^ = sum of the elements' equivalent unknowns     */
  int64_t n_elem;
  int64_t n_types;
  int64_t grid[3];       /* AIM grid nodes per axis                           */
  int64_t fft[3];        /* padded FFT lengths per axis                       */
  int64_t nnz_near;      /* near-field nonzeros                               */
  int64_t device_bytes;  /* resident operator bytes on the device             */
  int64_t n_scat_unknowns; /* N_s = sum of the elements' scatterer RWG unknowns */
  int64_t n_near_blocks; /* distinct (type, type, lattice offset) near blocks   */
  int64_t near_block_entries; /* their dense complex entries (device: one copy per precision) */
  int32_t near_format;   /* how the device applies the near field: 0 blocks, 1 CSR rows */
} mm_array_info;
mm_status mm_array_info_get(const mm_array* array, mm_array_info* info);
/* Device bytes a solve with nrhs columns needs beyond the resident operator
 * (Krylov basis of `restart` + 1 vectors, work vectors, grids).              */
mm_status mm_array_footprint(const mm_array* array, int32_t nrhs, int32_t precision, int32_t restart,
                             size_t* bytes);
/* Host copies of set-up data (testing, inspection, checkpointing):
 *   MM_EXPORT_ANCHORS  int64 (N^ x 3)   stencil anchors (grid indices)
 *   MM_EXPORT_PI       double (N^ x S x 4) projection weights (psi = x,y,z,phi)
 *   MM_EXPORT_NEAR_PTR int64 (N^ + 1)   CSR row pointer of the near field
 *                                       (the three NEAR exports need the CSR:
 *                                       MM_EINVAL when it was not assembled)
 *   MM_EXPORT_NEAR_COL int32 (nnz)      CSR columns
 *   MM_EXPORT_NEAR_VAL double (2 nnz)   CSR values, complex128
 *   MM_EXPORT_GHAT     double (2 P)     Green's spectrum, complex128, x slowest
 * `out` may be NULL to query the element count (`count`).                   */
typedef enum mm_export_id {
  MM_EXPORT_ANCHORS = 0, MM_EXPORT_PI = 1, MM_EXPORT_NEAR_PTR = 2, MM_EXPORT_NEAR_COL = 3,
  MM_EXPORT_NEAR_VAL = 4, MM_EXPORT_GHAT = 5
} mm_export_id;
mm_status mm_array_export(const mm_array* array, int32_t which, void* out, int64_t* count);
void mm_array_destroy(mm_array* array);

/* --------------------------------------------------------------- hot path
 * y = (D - G^(E^,J^) T A^-1 B) x, eq. (MV_product1), for nrhs columns, with
 * G^(E^,J^) applied by AIM (Sec. V): per-type macromodel product u = M x and
 * v = D x, projection of u onto the grid (step i), FFT convolution with the
 * Green's spectrum (step ii), interpolation (step iii), near-field product,
 * y = v - (G_FF u + G_NF u).  x_dev, y_dev: (N^ x nrhs) complex in
 * `precision`; must not alias.  Queued on `stream`: the near-field product runs
 * on a second stream of the array beside the far-field chain (forked from and
 * joined back into `stream` with events), so the call orders like one launch on
 * `stream`.  An array serves one caller at a time.  Tuning overrides read when
 * the array is created: MACROAIM_NEAR_OVERLAP=0 keeps the near field on
 * `stream` in order; MACROAIM_NEAR_SHAPE="shape,ksplit" fixes the block
 * near-field kernel's shape instead of timing them on the first product
 * (0-4 CUDA-core tiles, k split 1-16; 5-6 tensor-core tiles, complex64 only,
 * TF32 with a three-product split, k split 1 or 2 (2 for up to 8 right-hand
 * sides); 7-9 the tensor-core direct form
 * for 16 or more right-hand sides of even count);
 * MACROAIM_NEAR=csr applies the near field as CSR rows;
 * MACROAIM_FF_SHAPE="gemm,near" fixes the tile shapes of the MM_C128_FF
 * GEMM (0-2) and near field (0-3).                                           */
mm_status mm_apply(mm_array* array, int32_t nrhs, const void* x_dev, void* y_dev, int32_t precision,
                   void* stream);
/* Products of several arrays in one call (arrays of different sizes, element
 * types and right-hand-side counts): entry i computes y_dev[i] = Z_i x_dev[i]
 * for arrays[i] with nrhs[i] columns, as mm_apply.  Each array's product runs
 * on a stream of its own, forked from `stream` and joined back into it, so the
 * products run concurrently on the device and the call orders like one launch
 * on `stream`.  Every array appears at most once; all on one device.  Once
 * every array has done a product of its width and precision (its tuners have
 * run) and none records stage events (mm_profile_enable), the call captures
 * the batch's launches into one CUDA graph and launches that graph; later
 * calls with the same arrays, widths, x_dev / y_dev pointers and precision
 * replay it as one launch (on a library stream ordered after and before
 * `stream` by events).  A graph is dropped when an array is destroyed, and not
 * used after an array's work buffers were reallocated (a product of another
 * width in between).  The batch's message on failure is on arrays[0]'s
 * context.                                                                   */
mm_status mm_apply_batch(mm_array* const* arrays, int32_t count, const int32_t* nrhs, const void* const* x_dev,
                         void* const* y_dev, int32_t precision, void* stream);
/* Number of batch graphs held for `array` (NULL: all arrays) by mm_apply_batch. */
mm_status mm_batch_graphs(const mm_array* array, int32_t* count);
/* Same operator with host buffers: copies x in, applies, copies y out, and
 * returns after the result is in y_host (synchronous).                       */
mm_status mm_apply_host(mm_array* array, int32_t nrhs, const void* x_host, void* y_host, int32_t precision);

/* Excitation V^ for nrhs plane waves (Sec. IV, eq. (V1), tested with the
 * equivalent-surface RWG functions): V^_n = <f^_n, n x n x E_inc> =
 * -<f^_n, E_inc>, E_inc = p exp(-j k0 k^.r), k^ = -(sin t cos p, sin t sin p,
 * cos t) (arriving from (theta, phi)), p = theta^ (pol 0) or phi^ (pol 1),
 * |E0| = 1.  theta/phi/pol are host arrays of length nrhs (copied before the
 * call returns); V_dev is (N^ x nrhs) in `precision`.  Queued on `stream`
 * (no host synchronisation).                                                  */
mm_status mm_rhs_planewave(mm_array* array, int32_t nrhs, const double* theta, const double* phi,
                           const int32_t* pol, void* V_dev, int32_t precision, void* stream);

/* Currents of a solution (Sec. II, eq. (JABE) and eq. (Tm1); Sec. IV after
 * eq. (finalsystem)): per element, J_e = -A_t^-1 B_t E^_e on the scatterer
 * (RWG coefficients on S_e, N_t per element) and J^_e = T_t J_e on the
 * equivalent surface (N^_t per element).  E_dev: (N^ x nrhs) complex128.
 * J_dev: (N_s x nrhs) complex128 with N_s = sum of the elements' scatterer
 * unknowns (mm_array_info.n_scat_unknowns), element-major, or NULL; Jhat_dev:
 * (N^ x nrhs) complex128 or NULL.  FP64 throughout.  Queued on `stream`.    */
mm_status mm_currents(mm_array* array, int32_t nrhs, const void* E_dev, void* J_dev, void* Jhat_dev, void* stream);

/* ------------------------------------------------------- driven elements
 * Delta-gap feed of an element type (Sec. VI: driven array elements; the
 * paper states that the macromodel carries over to them without giving the
 * equations; this library's reading): a gap of voltage V across the scatterer
 * RWG edges rwg[0..n_edges) is the impressed field V delta(xi) xi^, xi^ along
 * `direction` (3 doubles, not parallel to the gap edges); in the MoM form
 * (Z = j k0 eta0 L, right-hand side <f, E>) edge g gets f_g = s_g V l_g, s_g the
 * sign of xi^ . n_g with n_g the in-plane normal of edge g from its T+ to its
 * T- triangle (T+ the lower-numbered triangle of the edge).  The feed enters
 * the scatterer's equation, eq. (EFIEdiscretized1), so with A and B of eq. (JM)
 * the currents are J = -A^-1 B E^ + J_f V, J_f = -A^-1 f (FP64, host, per
 * volt), and the equivalent current J^ = T J carries J^_f = T J_f into the
 * exterior problem.  Set feeds before creating arrays with the type.
 * MM_EINVAL for an edge index out of range or a direction parallel to an edge. */
mm_status mm_type_set_feed(mm_type* type, int32_t n_edges, const int64_t* rwg, const double* direction);

/* Excitation of driven elements: with the feed in the scatterers, the
 * exterior system keeps the operator of eq. (finalsystem) and its right-hand
 * side becomes V^_eff = -G^(E^,J^) J^_f V (no incident field), G applied by
 * AIM like the product's coupling part (complex128).  volts: host, n_elem x
 * nrhs complex128 interleaved (element-major, right-hand sides innermost);
 * elements of types without a feed get no source.  V_dev: (N^ x nrhs)
 * complex128.  Queued on `stream`.  Add a plane-wave excitation for mixed
 * problems.  MM_EINVAL when no type of the array has a feed.               */
mm_status mm_rhs_deltagap(mm_array* array, int32_t nrhs, const double* volts, void* V_dev, void* stream);

/* Currents of a driven solution: mm_currents plus the feed's share,
 * J += J_f V and J^ += J^_f V per driven element (volts as in
 * mm_rhs_deltagap).  The port current of a gap is sum_g s_g J_g l_g.        */
mm_status mm_currents_fed(mm_array* array, int32_t nrhs, const void* E_dev, const double* volts, void* J_dev,
                          void* Jhat_dev, void* stream);

/* ----------------------------------------------------------- ground plane
 * Plane-wave excitation above a PEC plane z = z_ground by image theory (Sec.
 * VI, the reflectarrays' ground plane): the array must hold every element and
 * its image (same type at (x, y, 2 z_ground - z) for elements symmetric under
 * z -> -z in their own frame); the incident field is the plane wave plus its
 * image, E_img(r) = S E_inc(R r), R the reflection in the plane and
 * S = diag(-1, -1, 1).  The image of the wave arriving from (theta, phi) with
 * polarisation theta^ (phi^) is the wave arriving from (pi - theta, phi) with
 * theta^ (-phi^), times exp(2 j k0 z_ground cos theta): V^ is the sum of two
 * mm_rhs_planewave excitations.  Arguments as mm_rhs_planewave.             */
mm_status mm_rhs_planewave_ground(mm_array* array, int32_t nrhs, const double* theta, const double* phi,
                                  const int32_t* pol, double z_ground, void* V_dev, int32_t precision,
                                  void* stream);

/* Far-field pattern radiated by the equivalent currents (the radiation
 * integral of the array's patterns, Sec. VI): with E ~ F exp(-j k0 r)/r,
 *   F(r^) = -j k0 eta0/(4 pi) (I - r^ r^) . sum_n J^_n int f^_n exp(j k0 r^.r') dS'
 * (7-point rule per triangle; phases reduced in FP64, exponentials and sums in
 * FP32).  r^ = (sin t cos p, sin t sin p, cos t) for host arrays theta, phi of
 * length ndir.  Jhat_dev: (N^ x nrhs) complex128; F_dev: (ndir x nrhs x 3)
 * complex128, Cartesian components.  Queued on `stream`.                       */
mm_status mm_farfield(mm_array* array, int32_t nrhs, const void* Jhat_dev, int64_t ndir, const double* theta,
                      const double* phi, void* F_dev, void* stream);

/* Bistatic RCS sigma = 4 pi |F|^2 / |E0|^2 (|E0| = 1; lambda^2 units when
 * k0 = 2 pi) from mm_farfield, written to sigma_host (ndir x nrhs).
 * Synchronous.                                                                */
mm_status mm_rcs(mm_array* array, int32_t nrhs, const void* Jhat_dev, int64_t ndir, const double* theta,
                 const double* phi, double* sigma_host);

/* GMRES solve of (D - G T A^-1 B) E^ = V^ (eq. (finalsystem); Sec. V) for
 * nrhs independent columns, x0 = 0.  precision MM_C128: plain FP64 GMRES on
 * the complex128 operator.  precision MM_C64 (or a tensor-core mode) with
 * refine = 1: complex64 operator inside GMRES (Arnoldi products on a Krylov
 * basis of complex128 precision, FP64 Givens), wrapped in iterative
 * refinement against the complex128 operator until ||V^ - Z E^|| <= tol ||V^||
 * per column; opts->fp64 chooses float-float (default) or FP64 arithmetic for
 * the residual and the inner Arnoldi products (tuning override read at each
 * call: MACROAIM_FF_ARNOLDI=0 keeps the inner Arnoldi in FP64).  V_dev, E_dev: (N^ x nrhs)
 * complex128.  Synchronous: returns when done.  MM_ENOCONV if max_iter was
 * reached (E_dev holds the last iterate).                                     */
typedef struct mm_solve_opts {
  double tol;         /* relative residual target per column                  */
  int32_t restart;    /* GMRES(m) restart length                              */
  int32_t max_iter;   /* total inner iterations bound                         */
  int32_t precision;  /* operator precision inside GMRES                      */
  int32_t refine;     /* 1: FP64 outer refinement (needs a complex64 mode)    */
  double inner_tol;   /* inner GMRES tolerance when refining                  */
  int32_t orth;       /* Arnoldi orthogonalisation (classical Gram-Schmidt):
                         0 = automatic (default): one pass for the inner
                         solves of refinement, whose error the FP64 outer
                         residual corrects; selective second pass otherwise;
                         1 = one pass; 2 = second pass only for columns whose
                         norm fell below 1/sqrt(2); 3 = two passes always      */
  int32_t precond;    /* 0 = none; 1 = block-Jacobi: right preconditioning by
                         the inverse of every element's own block (MM_MAT_PJ),
                         shared by identical elements.  The solution is the
                         same; GMRES needs fewer iterations.  Not a method of
                         the paper (which names ILU), a library option.         */
  int32_t fp64;       /* the FP64-class steps of refinement solves (the
                         residual b - Z x with the complex128 operator, and the
                         inner solves' Arnoldi products on a Krylov basis of
                         complex128 precision): 0 = in float-float arithmetic
                         on the FP32 pipe (MM_C128_FF; the default), 1 = in
                         FP64                                                   */
} mm_solve_opts;
typedef struct mm_solve_stats {
  int32_t iterations;     /* inner GMRES iterations (max over columns)        */
  int32_t matvecs;        /* operator applications (all precisions)           */
  int32_t refinements;    /* outer refinement steps                           */
  int32_t converged;      /* 1 if every column met tol                        */
  double rel_residual;    /* max over columns of ||V - Z E||/||V||            */
} mm_solve_stats;
mm_status mm_solve(mm_array* array, int32_t nrhs, const void* V_dev, void* E_dev, const mm_solve_opts* opts,
                   mm_solve_stats* stats, void* stream);

/* The whole solve from host memory, for callers without device buffers:
 * the plane-wave excitation of nrhs incidences (host theta, phi, pol as in
 * mm_rhs_planewave), the solve of mm_solve with `opts`, and the solution
 * copied to E_host (N^ x nrhs complex128, interleaved).  Synchronous.  The
 * array keeps two device vectors of N^ x nrhs complex128 for these calls.
 * MM_ENOCONV still fills E_host with the last iterate.                       */
mm_status mm_solve_planewave_host(mm_array* array, int32_t nrhs, const double* theta, const double* phi,
                                  const int32_t* pol, double* E_host, const mm_solve_opts* opts,
                                  mm_solve_stats* stats);

/* The block near-field kernel shape the array chose for products of nrhs
 * columns at `precision` (MM_C64 or MM_C128): shape 0-4 CUDA-core tiles, 5-6
 * tensor-core tiles (see mm_apply); ksplit its k split.  MM_EINVAL until a
 * product of that width has run (the choice is made on the first one).       */
mm_status mm_array_near_shape(const mm_array* array, int32_t nrhs, int32_t precision, int32_t* shape,
                              int32_t* ksplit);

/* The launch choices an array made for products of nrhs columns at
 * `precision` (MM_C64 or MM_C128), -1 where none was made yet:
 * choices[0], [1]: block near-field shape and k split (mm_array_near_shape);
 * choices[2]: projection schedule, choices[3]: interpolation schedule, chosen
 * on the array's first product of that width by timing each variant with CUDA
 * events (projection with one right-hand side: 4, 2 or 1 lanes per stencil-box
 * node for variants 0-2, 3 = complex64 from the type's stencil tables, four
 * lanes per node; several: 0 = four right-hand sides per pass, 1 = one,
 * 2 = two passes through a per-element box buffer without atomics (eight or
 * more), 3 = complex64 from the type's stencil tables in shared memory, eight
 * right-hand sides per pass (eight or more, where the tables fit);
 * interpolation with one right-hand side: 4, 2 or 1 lanes per basis; eight or
 * more: 0 = eight right-hand sides per thread, 1 = one, 2 = complex64 with
 * eight right-hand sides across the lanes of a warp, 3 = the same from the
 * types' weights in shared memory).  project_ms and interp_ms (4 floats each,
 * may be NULL): the variants' times, -1 where not timed.  MACROAIM_GRID_SCHED="p,i" (read when the array is created) fixes
 * the two schedules.
 * MACROAIM_GRID_TUNE=0 (read when the array is created) keeps variant 0
 * without timing.  MM_EINVAL before any product of that width.              */
mm_status mm_array_tuning(const mm_array* array, int32_t nrhs, int32_t precision, int32_t* choices,
                          float* project_ms, float* interp_ms);

/* ------------------------------------------------- allocation-free product
 * The same product as mm_apply, for callers that cannot allocate device
 * memory: code running inside a framework that has reserved all device
 * memory for its own pool, real-time loops where a cudaMalloc would stall or
 * synchronise the device, or kernels issued from a thread that must not touch
 * the allocator.  The paper has no counterpart; this is a library service.
 *
 * Instead of the array's work buffers it uses one scratch array of at most
 * 16 MiB that lives in the library's device image (every GPU that loads the
 * library holds it until the process exits).  The caller still passes x_dev
 * and y_dev.  The call allocates nothing: no cudaMalloc, cudaFree or other
 * allocating routine.  Requirements and limits:
 *  - the scratch must hold u, v (N^ x nrhs each), the 4 nrhs grids and the
 *    partial spectra at `precision`; larger requests return MM_EINVAL with
 *    the bytes needed (the 16x16 loop array fits at either precision);
 *  - the complex64 operator is resident from mm_array_create; the complex128
 *    operator is uploaded by the first mm_apply or mm_solve at complex128, so
 *    call one of those first or this returns MM_EINVAL;
 *  - the first call on a device looks up the scratch array's device address
 *    (cudaGetSymbolAddress, once per device, with that device current); make
 *    that first call before any stream capture;
 *  - the call never times near-field kernel shapes (mm_apply does that on an
 *    array's first product at a right-hand-side count, with CUDA events and a
 *    host synchronisation): it reuses the shape that an earlier mm_apply or
 *    mm_solve chose for this count and precision, else a size rule; it
 *    creates no CUDA events and does not wait for the device;
 *  - every call shares the one scratch array and leaves its contents behind;
 *    calls that overlap on the GPU (other streams, other arrays, other
 *    threads) race on it: serialise them;
 *  - the call records nothing in the array's stage profiler and leaves the
 *    profiler's state alone (profiling may stay enabled).                     */
mm_status mm_apply_noalloc(mm_array* array, int32_t nrhs, const void* x_dev, void* y_dev, int32_t precision,
                           void* stream);

/* ---------------------------------------------------------- testing hook
 * Bounded waits of the tensor-core macromodel GEMM (MM_C64_BF16 and
 * MM_C64_F16 products): with ms > 0, the GEMMs launched afterwards (by any
 * array of the process) issue no products, so every wait of the kernel runs
 * out after ms milliseconds; the kernel then waits for its copies in flight,
 * frees its tensor memory and returns, and the call that next synchronises
 * (mm_solve, mm_apply_host) returns MM_ETIMEOUT.  ms = 0 restores normal
 * products.  For tests of the failure path only; no GPU fault is involved.
 * The paper has no counterpart.  MM_EINVAL for ms < 0.                       */
mm_status mm_test_tc_stall(int32_t ms);

/* ----------------------------------------------------------------- server
 * A solve server for streams of requests (the library's request loop; the
 * paper has none).  mm_server_create starts `workers` threads on `device`,
 * each with its own context and CUDA stream.  A submitted request (copied) is
 * admitted when its estimated device footprint fits in hbm_budget_bytes (0:
 * 80 % of the free device memory) minus the requests in flight; admitted
 * requests run concurrently (array set-up, plane-wave excitation, GMRES, copy
 * of E^ to the host), so a request that arrives while others run starts as
 * soon as a worker and memory are free.  Element types are shared read-only
 * and must outlive the server.  mm_server_poll returns MM_EBUSY while the
 * request runs (wait = 0) or blocks until it is done (wait = 1); E_host, if
 * not NULL, receives E^ (N^ x nrhs complex128; E_count doubles available).
 * mm_server_release forgets a finished request.
 * Batching: when a worker takes a request, waiting requests with the same
 * element types, offsets, AIM options and solve options join it as further
 * columns of one solve (at most 64 columns); every product and Arnoldi step
 * then covers all of them.  Green's spectra are cached across arrays of equal
 * grid size.  For short set-up, requests may set aim.near_csr = 2 (no CSR
 * assembly; the complex128 residual products then use the dense blocks).     */
typedef struct mm_server mm_server;
typedef struct mm_request {
  int64_t n_elem;
  const mm_type* const* types;   /* per element                                */
  const double* offsets_xyz;     /* n_elem x 3                                 */
  mm_aim_opts aim;
  int32_t nrhs;
  const double* theta;           /* nrhs incidences (see mm_rhs_planewave)     */
  const double* phi;
  const int32_t* pol;
  mm_solve_opts solve;
} mm_request;
typedef struct mm_result {
  int32_t done;
  int32_t status;                /* mm_status of the request                   */
  int64_t n_unknowns;
  mm_solve_stats stats;
  double queue_s, setup_s, solve_s, latency_s;   /* wall times, seconds       */
  char message[160];             /* failure message ("" when status is MM_OK)  */
  int32_t group_requests;        /* requests solved together with this one
                                    (same geometry and options; 1 = alone)    */
  int32_t group_columns;         /* columns of that solve                      */
} mm_result;
mm_status mm_server_create(int device, int32_t workers, size_t hbm_budget_bytes, mm_server** out);
mm_status mm_server_submit(mm_server* server, const mm_request* request, uint64_t* ticket);
mm_status mm_server_poll(mm_server* server, uint64_t ticket, int32_t wait, mm_result* result, double* E_host,
                         int64_t E_count);
mm_status mm_server_release(mm_server* server, uint64_t ticket);
void mm_server_destroy(mm_server* server);

/* ----------------------------------------------------------- profiling
 * With profiling enabled, every stage of every product is bracketed by CUDA
 * events on the caller's stream (a few microseconds of host overhead per
 * stage) and kernel launches are counted.  mm_profile_read synchronises the
 * recorded events and returns per-stage totals since the last enable, for the
 * products at `precision` (MM_C64, MM_C128, or -1 for both; the Krylov stage
 * is always included): ms[s] = summed device time of stage s, launches[s] =
 * kernel launches of stage s (arrays of MM_STAGE_COUNT entries).  Disabled
 * by default.                                                                 */
typedef enum mm_stage {
  MM_STAGE_GEMM = 0,     /* macromodel product [M; D] x                      */
  MM_STAGE_PROJECT = 1,  /* step (i)                                         */
  MM_STAGE_FFT_FWD = 2,  /* step (ii): z DFT + y FFT                         */
  MM_STAGE_FFT_CONV = 3, /* step (ii): x FFT, spectrum multiply, inverse x  */
  MM_STAGE_FFT_INV = 4,  /* step (ii): inverse y FFT + z DFT                 */
  MM_STAGE_INTERP = 5,   /* step (iii) and y = D x - y_ff                    */
  MM_STAGE_NEAR = 6,     /* near-field product                               */
  MM_STAGE_KRYLOV = 7,   /* GMRES orthogonalisation, updates, conversions    */
  MM_STAGE_COUNT = 8
} mm_stage;
mm_status mm_profile_enable(mm_array* array, int32_t enable);
/* Which stages record while profiling is enabled: bit s of stage_mask for stage
 * s (both precisions; default all).  Recording fewer stages perturbs the timed
 * work less (each recorded stage adds two CUDA event records per product).   */
mm_status mm_profile_stages(mm_array* array, uint32_t stage_mask);
mm_status mm_profile_read(mm_array* array, int32_t precision, double* ms, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* MACROAIM_H */
