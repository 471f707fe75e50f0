/*
 * oefe.h -- C ABI of the GB300 library for the Chebyshev-filtered subspace
 * iteration of the orthogonalized enriched finite element (OEFE) method
 * (Rufus, Kanungo, Gavini, arXiv 2010.09701).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every function returns an int status: OEFE_OK (0) or a negative
 *   OEFE_ERR_* code. No exception crosses the ABI. oefe_last_error() copies a
 *   one-line description of the last failure of a context.
 * - A context is not thread-safe. All GPU work is ordered on the CUDA stream
 *   given to oefe_create() (or oefe_set_stream()). Calls that return values
 *   in host memory synchronize that stream before returning.
 * - "device" pointers are CUDA global-memory pointers on the context's
 *   device; "host" pointers are ordinary CPU memory. The caller owns every
 *   pointer it passes; the library owns everything reachable from the
 *   context and frees it in oefe_destroy().
 * - Vector blocks X are row-major (ndof x ld) with the nv <= ld columns
 *   innermost. Rows 0 .. n_h-1 are the classical (CFE) coefficients of the
 *   global nodes, rows n_h .. n_h+n_O-1 the orthogonalized enrichment
 *   coefficients (Eq. UOEFE). Complex data are interleaved (re, im).
 * - Required call order: create -> mesh -> enrichment -> quadrature ->
 *   kpoints -> build_hamiltonian -> {apply, filter, orthonormalize,
 *   rayleigh_ritz, density, ...}. Out-of-order calls return OEFE_ERR_STATE.
 */
#ifndef OEFE_H
#define OEFE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oefe_ctx* oefe_ctx_t;

enum {
  OEFE_OK = 0,
  OEFE_ERR_ARG = -1,        /* invalid argument (size, pointer, range)        */
  OEFE_ERR_STATE = -2,      /* call made before the calls it depends on        */
  OEFE_ERR_OOM = -3,        /* device or host allocation failed                */
  OEFE_ERR_CUDA = -4,       /* a CUDA runtime call failed                      */
  OEFE_ERR_CHOLESKY = -5,   /* Gram / projected overlap not positive definite  */
  OEFE_ERR_NOTPD_MOO = -6,  /* enrichment overlap block M^oo not pos. definite */
  OEFE_ERR_TIMEOUT = -7,    /* a bounded device wait gave up                   */
  OEFE_ERR_NUMERIC = -8     /* NaN or Inf detected                             */
};

/* Element type of vector blocks. */
enum { OEFE_F64 = 0, OEFE_F32 = 1, OEFE_C128 = 2, OEFE_C64 = 3 };

/* Storage of the cell Hamiltonians (bit mask for oefe_build_hamiltonian). */
enum { OEFE_STORE_F64 = 1, OEFE_STORE_F32 = 2, OEFE_STORE_BF16X3 = 4, OEFE_STORE_BF16X6 = 8, OEFE_STORE_F64PAIR = 16,
       OEFE_STORE_COMPACT = 32 };
/* arithmetic of the FP64 cell products (oefe_set_f64_products) */
enum { OEFE_F64_NATIVE = 0, OEFE_F64_PAIRS = 1 };

/* ---------------------------------------------------------------- context */
int oefe_create(oefe_ctx_t* out, int device, void* cuda_stream);
int oefe_destroy(oefe_ctx_t ctx);
int oefe_set_stream(oefe_ctx_t ctx, void* cuda_stream);
int oefe_last_error(oefe_ctx_t ctx, char* buf, size_t len);

/* ---------------------------------------------------------------- geometry
 * oefe_mesh -- periodic cubic cell [0,a)^3 split into ncell[0]*ncell[1]*
 * ncell[2] hexahedral spectral elements of order p (Sec. III A: Lagrange
 * polynomials on GLL nodes so that the CFE overlap is diagonal).
 *   xb   host, ncell[0]+ncell[1]+ncell[2]+3 doubles: the per-axis cell
 *        boundaries, x then y then z, each increasing from 0 to a.
 *   p    1 .. 7.
 * Cell (ix,iy,iz) has index ix + ncell0 (iy + ncell1 iz); global node
 * (gx,gy,gz) has index gx + N0 (gy + N1 gz), N_d = ncell_d p.
 */
int oefe_mesh(oefe_ctx_t ctx, double a, const int ncell[3], const double* xb, int p);

/* oefe_mesh_graded -- the same with breakpoints refined toward the nuclei:
 * the distinct nuclear coordinates of an axis become breakpoints; when there
 * are at most ncell/2 of them, cells are shared out among the intervals in
 * proportion to length (at least 2 each) and graded geometrically with
 * `ratio` from both interval ends; otherwise the axis is uniform.
 *   pos  host, 3*natoms doubles.   xb_out  host, 3*(ncell+1) doubles or NULL. */
int oefe_mesh_graded(oefe_ctx_t ctx, double a, int ncell, int p, int natoms,
                     const double* pos, double ratio, double* xb_out);

/* oefe_enrichment -- atomic enrichment functions (Eqs. UOEFEAtomic,
 * KSAtomicTrunc, CutoffProperties):
 *   N^A_{I,j}(x) = exp(-i k.(x - R_I^x)) R_{I,j}(r) S_j(x - R_I^x) h(r),
 * r = |x - R_I^x|, R_I^x the nearest periodic image of nucleus I.
 *   pos   host, 3*natoms doubles (bohr).
 *   lm    host, nfun ints: angular code per function, 0 = s, 1/2/3 = p_x/p_y/p_z.
 *   R, dR host, natoms*nfun*ngrid doubles: radial function and its
 *         derivative on the uniform grid r_i = i rc/(ngrid-1) (cubic Hermite
 *         interpolation between grid points, zero for r >= rc).
 *   r0 < rc: smooth cutoff h = phi(s)/(phi(s)+phi(1-s)), s = (rc-r)/(rc-r0),
 *         phi(t) = exp(-1/t) (t > 0), which is 1 below r0 and 0 above rc;
 *         rc < a/2 is required. Function index nu = I*nfun + j. natoms may be 0. */
int oefe_enrichment(oefe_ctx_t ctx, int natoms, const double* pos, int nfun, const int* lm,
                    int ngrid, const double* R, const double* dR, double r0, double rc);

/* oefe_quadrature -- per-cell point sets (Sec. III B adaptive quadrature,
 * deterministic reading): a cell meeting no enrichment support gets
 * nq_cell^3 Gauss points; a cell meeting one gets nq_enr^3; a cell whose
 * closed box holds a nucleus is split into 8 children, recursively while a
 * child holds a nucleus, up to `depth` levels, with nq_enr^3 points per leaf.
 * Point order: cells ascending, leaves depth-first (children x fastest),
 * points x fastest. 1 <= nq_cell, nq_enr <= 12, 0 <= depth <= 12. */
int oefe_quadrature(oefe_ctx_t ctx, int nq_cell, int nq_enr, int depth);
int oefe_quadrature_count(oefe_ctx_t ctx, int64_t* nq_total);
/* host outputs: xyz 3*nq doubles, w nq doubles (either may be NULL). */
int oefe_quadrature_points(oefe_ctx_t ctx, double* xyz, double* w);

/* oefe_kpoints -- Bloch vectors (Cartesian bohr^-1, host 3*nk) and weights
 * (host nk, sum 1). For each k the library tabulates the enrichment at the
 * points, forms the orthogonalizing coefficients c_{nu,l} = int N^A N^C / m_l
 * (Eq. orthCGLL), the block M^oo = M^AA - C diag(m) C^+ (Eq. Moo) and its
 * inverse (Eq. MOEFEInv). Returns OEFE_ERR_NOTPD_MOO if M^oo is not positive
 * definite. k = 0 exactly gives real arithmetic for that k. */
int oefe_kpoints(oefe_ctx_t ctx, int nk, const double* k, const double* w);

int oefe_ndof(oefe_ctx_t ctx, int64_t* n_h, int* n_O);

/* ---------------------------------------------------------------- operators
 * oefe_build_hamiltonian -- cell matrices H^O_e(k) = T_e^+ H_e T_e for every
 * cell and k (Eq. HOEFEelelements; T maps OEFE to EFE coefficients,
 * Eq. UOEFESplit). veff_q: device, nq_total doubles, V_eff at the quadrature
 * points. store: OEFE_STORE_F64 (FP64 / complex128 matrices, needed by every
 * FP64 call), OEFE_STORE_F32 (FP32 / complex64 copies for the FP32 filter)
 * and/or one of OEFE_STORE_BF16X3 (each real plane split into bf16 hi + lo for
 * the tensor-core filter; same bytes as FP32: products H_hi X_hi + H_hi X_lo +
 * H_lo X_hi, ~2^-17 relative) and OEFE_STORE_BF16X6 (three bf16 parts hi + mid
 * + lo, 1.5x the bytes: six products, FP32-class accuracy; wins when both are
 * set). The tensor-core filter (OEFE_FILTER_BF16X3) uses whichever split is
 * stored. OEFE_STORE_F64PAIR (with OEFE_STORE_F64) also keeps each FP64 value
 * as a pair of FP32 numbers hi + lo (same bytes as FP64, about 48 significant
 * bits) for the FP32-pair products of oefe_set_f64_products.
 * OEFE_STORE_COMPACT (with OEFE_STORE_F64) keeps the FP64 and FP32-pair
 * copies in a compact layout: cells with several quadrature leaves whole,
 * single-leaf cells only as their enrichment strip (the CO block and the
 * enrichment rows), whose CFE-CFE block the FP64-class products apply by sum
 * factorization anyway (about 1/6 of the bytes at p = 6); oefe_cell_matrix then
 * returns OEFE_ERR_STATE for single-leaf cells. It needs the sum-factorized
 * products (hexahedral cells, p <= 7), else OEFE_ERR_ARG. All arithmetic of
 * the build is FP64. */
int oefe_build_hamiltonian(oefe_ctx_t ctx, const double* veff_q, int store);

/* Row/column map of one cell matrix: idx (host, n_aug ints) receives global
 * rows (nodes, then n_h + enrichment index). */
int oefe_cell_info(oefe_ctx_t ctx, int cell, int* n_aug, int* idx);
/* H^O_e of one cell (host, n_aug*n_aug doubles or complex128, row-major). */
int oefe_cell_matrix(oefe_ctx_t ctx, int ik, int cell, void* H);
/* Lumped CFE mass (host, n_h doubles) and M^oo (host, n_O^2, complex for k != 0). */
int oefe_overlap(oefe_ctx_t ctx, int ik, double* m, void* Moo);

/* Y = H^O X, and Y = (M^O)^{-1} H^O X (Eq. KSEignStandDiscrete).
 * X, Y device, (n x ld); dtype OEFE_F64 or OEFE_C128 (C128 for k != 0). */
int oefe_apply_h(oefe_ctx_t ctx, int ik, const void* X, void* Y, int nv, int ld, int dtype);
int oefe_apply_a(oefe_ctx_t ctx, int ik, const void* X, void* Y, int nv, int ld, int dtype);

/* oefe_apply_a_noalloc -- the same Y = (M^O)^{-1} H^O X as oefe_apply_a, for
 * callers that cannot allocate device memory at this point: an application
 * whose memory pool already owns the whole device, a service that must not
 * take the implicit device synchronization of cudaMalloc / cudaFree in its
 * request path, or a host framework that forbids allocation once it runs.
 * The paper has no counterpart; this is a deployment variant.
 * It allocates nothing: the per-cell products and the enrichment-row sums
 * that oefe_apply_a keeps in its growing workspace live in one fixed device
 * array of OEFE_NOALLOC_SCRATCH_BYTES bytes, compiled into the library and
 * resident on every device that loads it until the process exits. The
 * caller passes X and Y as for oefe_apply_a (the context itself was set up
 * earlier with allocations, as always).
 * - The first call on a device looks up the array's device address on that
 *   device (cudaGetSymbolAddress); make that first call outside any stream
 *   capture. The address is kept for later calls while the CUDA context it
 *   came from is still current; after a device reset (a new primary context)
 *   the next call looks it up again, so make that call outside a capture too.
 * - Problems needing more than the array (ncells * npad * nv * sizeof(scalar)
 *   rounded up to 256 bytes, plus n_O * nv * 16 bytes) are refused with
 *   OEFE_ERR_ARG; oefe_last_error gives the sizes.
 * - Every call uses the same array and overwrites what it reads (nothing
 *   needs to start at zero); calls whose GPU work overlaps (other streams,
 *   other contexts, other threads) race on it and must be serialized by the
 *   caller. The call synchronizes the context's stream before returning. */
#define OEFE_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
int oefe_apply_a_noalloc(oefe_ctx_t ctx, int ik, const void* X, void* Y, int nv, int ld, int dtype);

/* ---------------------------------------------------------------- filter
 * oefe_chebyshev_filter -- X <- p_m(A) X in place, A = (M^O)^{-1} H^O
 * (Sec. IV), with the scaled three-term recurrence: e = (b-a)/2,
 * c = (b+a)/2, sigma_1 = e/(a0-c); Y_1 = (sigma_1/e)(A - c) X;
 * Y_{j+1} = (2 sigma_{j+1}/e)(A - c)Y_j - sigma_j sigma_{j+1} Y_{j-1},
 * sigma_{j+1} = 1/(2/sigma_1 - sigma_j). The M^{-1} step (diagonal CFE mass,
 * dense FP64 (M^oo)^{-1}) and the recurrence are fused into the reduction
 * of the cell products. dtype: F64/C128 use the FP64 cell matrices, F32/C64
 * the FP32 copies (FP32 accumulation). flags: OEFE_FILTER_LAST_FP64 runs the
 * degrees before the last in FP32 and the last through the FP64 path (X
 * must then be F64/C128 storage); OEFE_FILTER_BF16X3 computes the
 * low-precision cell products on the tensor cores from the BF16x3 storage
 * (hi*hi + hi*lo + lo*hi, FP32 accumulation). */
enum { OEFE_FILTER_LAST_FP64 = 1, OEFE_FILTER_BF16X3 = 2 };
int oefe_chebyshev_filter(oefe_ctx_t ctx, int ik, void* X, int nv, int ld, int dtype, int degree,
                          double a, double b, double a0, int flags);

/* oefe_filter_batched -- the Chebyshev filter of every k-point of the context
 * at once (Sec. IV; the batched multi-k launch). Degree by degree, one
 * persistent tensor-core launch covers all (k, cell, vector block) tiles
 * (uneven nv per k allowed), the node and enrichment updates are batched
 * over k, and the low-precision degrees are captured once in a CUDA graph on
 * a private stream and replayed by later calls with the same arguments.
 * flags must contain OEFE_FILTER_BF16X3; with OEFE_FILTER_LAST_FP64 the
 * vectors are F64/C128 and the last degree runs per k in FP64, otherwise
 * they are F32/C64. X: host array of nk device pointers; nv, ld, a, b, a0:
 * host arrays of nk. The call returns after the filter has finished. */
int oefe_filter_batched(oefe_ctx_t ctx, int nk, void* const* X, const int* nv, const int* ld, int dtype,
                        int degree, const double* a, const double* b, const double* a0, int flags);

/* oefe_filter_batched_defect -- the batched filter in defect form, for a block
 * that already approximates eigenvectors: on entry X[k] holds Q (F64/C128)
 * with approximate eigenvalues theta (the Ritz pairs of the previous pass of
 * the subspace iteration, Sec. IV, Eq. ProjKS); on return X[k] = p_m(A) Q,
 * computed as p_m(A) Q = Q p_m(Theta) + D_m with Theta = diag(theta),
 *   R = A Q - Q Theta                      (one FP64-class operator application),
 *   D_0 = 0, D_1 = alpha_1 R,
 *   D_j = alpha_j [(A - c) D_{j-1} + R p_{j-1}(Theta)] + beta_j D_{j-2},
 * where c, alpha_j, beta_j and the scaled polynomials p_j are those of
 * oefe_chebyshev_filter (a three-term recurrence, so the identity is exact).
 * Every degree of D runs on the tensor cores like oefe_filter_batched (one
 * persistent launch per degree over all k, captured once in a CUDA graph; the
 * first degree needs no product), and Q p_m(Theta) + D_m is formed in FP64.
 * The low-precision rounding then scales with |D| -- about the size of the
 * residuals of Q -- instead of with |p_m(A) Q|, so directions that have
 * converged stay converged to FP64-class accuracy (the plain mixed filter
 * leaves them at about eps_FP32 times the spectral width). Any theta gives the
 * same p_m(A) Q in exact arithmetic; the Ritz values make R smallest.
 *   theta  host, sum_k nv[k] doubles (k-major), finite.
 * flags must contain OEFE_FILTER_BF16X3 (OEFE_FILTER_LAST_FP64 is ignored);
 * X, nv, ld, a, b, a0 as for oefe_filter_batched, the operator built with
 * OEFE_STORE_F64 (and OEFE_STORE_F64PAIR in pair mode) besides the split.
 * The paper filters in double precision throughout; this form is ours. */
int oefe_filter_batched_defect(oefe_ctx_t ctx, int nk, void* const* X, const int* nv, const int* ld, int dtype,
                               int degree, const double* a, const double* b, const double* a0, const double* theta,
                               int flags);

/* oefe_filter_autotune -- times the tensor-core cell-product launch shapes
 * on the given vectors and keeps the fastest for the BF16X3 filters:
 * (0) 64 vectors per tile, persistent grid of one CTA per SM, cp.async loads;
 * (1) the same with 32 vectors per tile; (2) one CTA per tile;
 * (3) the warp-specialized kernel with TMA loads (persistent); (4) the same with
 * the real part of a complex cell matrix applied to [Re X | Im X] in one
 * N = 128 MMA (complex data only); (5) the TMA kernel with 128 vectors per
 * tile (real data only: each cell matrix streams once per 128 vectors). The
 * three-part split (OEFE_STORE_BF16X6) runs on (3), (4), (5) only.
 * ms (host, 6 doubles, may be NULL) receives the time of one degree's cell
 * products for each candidate (0 when a candidate is unavailable). Vectors as
 * for oefe_filter_batched; they are read, not changed. */
int oefe_filter_autotune(oefe_ctx_t ctx, int nk, void* const* X, const int* nv, const int* ld, int dtype, double* ms);

/* oefe_set_filter_shape -- keeps launch shape `shape` (0..5, the candidates of
 * oefe_filter_autotune) for the BF16X3 filters without timing; -1 returns to
 * the untuned default ((4) on complex data, (3) on real data). A shape the stored split or
 * the data type does not have falls back at filter time: (0)-(2) run as (3)
 * for the three-part split; (4) runs as (3) on real data, (5) as (3) on
 * complex data. Every shape computes the same products up to FP32 summation
 * order. Returns OEFE_ERR_ARG for another value. */
int oefe_set_filter_shape(oefe_ctx_t ctx, int shape);

/* ---------------------------------------------------------------- subspace
 * oefe_orthonormalize -- Cholesky-QR in the M inner product, twice
 * (Sec. IV orthonormalization): S = X^+ M X = L L^+, X <- X L^{-+}.
 * The first pass equilibrates the columns by exact powers of two (X <- X D,
 * S <- D S D, D_vv = 2^-e with sqrt(S_vv) in [2^(e-1), 2^e)), which leaves
 * the result unchanged up to rounding and keeps columns of very different
 * norms (a filtered block) resolved to their own scale.
 * FP64; X must be F64/C128. cond_est (host, may be NULL) receives
 * (max L_ii / min L_ii)^2 of the first (equilibrated) pass. OEFE_ERR_CHOLESKY
 * if S is not positive definite. */
int oefe_orthonormalize(oefe_ctx_t ctx, int ik, void* X, int nv, int ld, int dtype, double* cond_est);

/* oefe_rayleigh_ritz -- H^Q = X^+ H^O X, M^Q = X^+ M X, H^Q u = eps M^Q u
 * (Eq. ProjKS), X <- X U. FP64. eig (host, nv) ascending; resid (host, nv or
 * NULL) receives ||H u - eps M u||_{M^-1} / ||u||_M per rotated vector. */
int oefe_rayleigh_ritz(oefe_ctx_t ctx, int ik, void* X, int nv, int ld, int dtype,
                       double* eig, double* resid);

/* oefe_density -- rho(x_q) = sum_k sum_a occ_{k,a} |u_{a,k}(x_q)|^2 at every
 * quadrature point (Eq. rho), u = N^C (X^c - C^T X^o) + N^A X^o.
 * X[k] device (F64/C128), occ host (sum_k nv[k] doubles, already holding
 * 2 w_k f), rho device (nq_total doubles, overwritten). */
int oefe_density(oefe_ctx_t ctx, int nk, const void* const* X, const int* nv, const int* ld,
                 int dtype, const double* occ, double* rho);

/* oefe_band_trace_grad -- gV (device, nq_total, overwritten) = d tr(X^+ H^O X)/d V_q
 * = w_q sum_v |u_v(x_q)|^2: the adjoint of the cell-level H.X application
 * with respect to the quadrature-point potential (H^O is affine in V through
 * the (|k|^2/2 + V) N_m^* N_n term of Eq. HOEFEelelements). The gradient with
 * respect to conj(X) is H^O X (oefe_apply_h). */
int oefe_band_trace_grad(oefe_ctx_t ctx, int ik, const void* X, int nv, int ld, int dtype, double* gV);

/* oefe_density_grad -- oefe_density and, from the same evaluation of the fields
 * at the quadrature points, oefe_band_trace_grad of k-point ik's block X[ik]:
 * rho as oefe_density, gV (device, nq_total doubles, overwritten) =
 * w_q sum_v |u_v(x_q)|^2 over the columns of X[ik] (Eq. rho; the adjoint of
 * Eq. HOEFEelelements with respect to V). Same arguments as oefe_density plus
 * ik (0 <= ik < nk) and gV (non-NULL); the results equal those of the two
 * separate calls (same arithmetic per point), at the cost of one pass over
 * the fields of X[ik] instead of two. */
int oefe_density_grad(oefe_ctx_t ctx, int nk, const void* const* X, const int* nv, const int* ld, int dtype,
                      const double* occ, double* rho, int ik, double* gV);

/* oefe_band_trace -- e (host, one double) = tr(X^+ H^O X) = Re sum_v x_v^+ H^O x_v,
 * the band-energy trace whose V-gradient oefe_band_trace_grad returns
 * (Eq. HOEFEelelements). HX: device (n x ld, the dtype of X) receiving H^O X,
 * or NULL (then a workspace of the context holds it). X: device F64/C128. */
int oefe_band_trace(oefe_ctx_t ctx, int ik, const void* X, int nv, int ld, int dtype, double* e, void* HX);

/* oefe_band_trace_vjp -- the backward pass of E = tr(X^+ H^O(V) X) for an upstream
 * gradient alpha (host double): gV (device, nq_total doubles, overwritten, may be
 * NULL) = alpha w_q sum_v |u_v(x_q)|^2, gX (device n x ld like X, overwritten, may
 * be NULL) = 2 alpha H^O X (the gradient with respect to X in torch's convention
 * for real and complex tensors). At least one of gV, gX. The fields and the
 * cell products are recomputed from X (nothing of the forward pass is kept). */
int oefe_band_trace_vjp(oefe_ctx_t ctx, int ik, const void* X, int nv, int ld, int dtype, double alpha, double* gV,
                        void* gX);

/* oefe_apply_h_vjp -- the backward pass of Y = H^O(V) X for a cotangent Gy of Y
 * (device, n x ld like X): H^O is affine in V through the (|k|^2/2 + V) N_m^* N_n
 * term of Eq. HOEFEelelements and Hermitian, so
 *   gV_q = w_q Re sum_v conj(u_Gy,v(x_q)) u_X,v(x_q)   (device, nq_total, overwritten, may be NULL),
 *   gX   = H^O Gy                                      (device, n x ld, overwritten, may be NULL),
 * u the fields of the columns at the quadrature points (Eq. UOEFE), both fields
 * evaluated in one pass over the points. At least one of gV, gX. */
int oefe_apply_h_vjp(oefe_ctx_t ctx, int ik, const void* X, const void* Gy, double* gV, void* gX, int nv, int ld,
                     int dtype);

/* oefe_occupations -- Fermi-Dirac occupancies f = 1/(1+exp((eps-mu)/kT))
 * (Eq. fd) with the Fermi level mu fixed by 2 sum_k w_k sum_a f = N_e
 * (Eq. ne, bisection to |dN| < 1e-12), kT = 3.166811563e-6 * T Ha. Host-only.
 *   eig  host, sum_k nv[k] eigenvalues (k-major); w host nk weights.
 *   occ  host out, sum_k nv[k]: 2 w_k f (the density weights of Eq. rho).
 *   mu, e_band  host out: Fermi level and E_band = 2 sum_k w_k sum_a f eps.
 * OEFE_ERR_ARG if N_e exceeds twice the number of states. */
int oefe_occupations(int nk, const int* nv, const double* eig, const double* w, double n_electrons,
                     double temperature, double* occ, double* mu, double* e_band);

/* oefe_upper_bound -- b >= max eig of (M^O)^{-1} H^O: largest Ritz value of
 * a `steps`-step Lanczos run in the M inner product from v0 (device, n
 * F64/C128) plus the last residual norm. The recurrence is FP64; flags = 0
 * applies A in FP64, OEFE_FILTER_BF16X3 applies it on the tensor cores
 * (BF16x3, relative error ~1e-5: enough for a filter bound). */
int oefe_upper_bound(oefe_ctx_t ctx, int ik, const void* v0, int steps, int flags, double* b);

/* ---------------------------------------------------------------- timing
 * oefe_kernel_timing -- CUDA-event timing of the cell-product kernel (the
 * dominant launch of every filter degree) on the context's stream, for the
 * vector dtypes whose bit (1 << OEFE_F64 ...) is set in dtype_mask; 0 turns
 * timing off, a non-zero mask clears the record. oefe_kernel_time returns the
 * summed device time (ms) and the launch count recorded so far; it
 * synchronizes the stream. No counterpart in the paper (instrumentation). */
int oefe_kernel_timing(oefe_ctx_t ctx, int dtype_mask);
int oefe_kernel_time(oefe_ctx_t ctx, double* ms, int64_t* launches);

/* oefe_release_workspace -- frees the context's cached scratch (the growable
 * work arrays of the operator build, the filter and the subspace calls, among
 * them the digit planes of the tensor-core Gram matrices and rotations) and
 * the captured graph of the batched filter, which points into it; later calls
 * allocate what they need again. Synchronizes the context's streams. Returns
 * OEFE_ERR_ARG for a null context. No counterpart in the paper (memory
 * management: the build's scratch is several times the filter's). */
int oefe_release_workspace(oefe_ctx_t ctx);

/* oefe_product_flops -- FP64 operations (an FMA counts two) that one FP64
 * operator application executes in its cell products for nv vectors at
 * k-point ik: cells with one quadrature leaf are applied by sum
 * factorization (the CFE block through 1D contractions, the enrichment blocks
 * dense), the others densely with three real multiplications per complex
 * product. flops: host pointer to one double. No counterpart in the paper
 * (instrumentation for the roofline). */
int oefe_product_flops(oefe_ctx_t ctx, int ik, int nv, double* flops);

/* oefe_launch_count -- process-wide number of kernel launches the library has
 * issued so far (every context; a replay of a captured graph counts each of
 * its kernels). n: host pointer to one int64. Never synchronizes. Returns
 * OEFE_ERR_ARG when n is null. No counterpart in the paper (instrumentation). */
int oefe_launch_count(int64_t* n);

/* oefe_set_f64_products -- arithmetic of the FP64-class kernels of the context.
 * mode OEFE_F64_NATIVE (default): FP64 everywhere. OEFE_F64_PAIRS: FP64-class
 * arithmetic off the FP64 pipe, which on this GPU issues at 1/64 of the FP32
 * rate:
 *   - FP32 pairs (each value an unevaluated sum of two FP32 numbers, error-free
 *     products and sums, about 2^-48 relative per operation; Dekker's
 *     double-length arithmetic) for the sum-factorized cell products of the
 *     single-leaf cells (the FP64 filter degrees, oefe_apply_h / _a, the H X of
 *     oefe_rayleigh_ritz; refined cells stay FP64), the per-V operator build,
 *     the fields of oefe_density / oefe_band_trace_grad and the Jacobi sweeps
 *     of the projected eigenproblem;
 *   - tensor-core GEMMs with exact bf16 digits (7 digits of 7 bits per value,
 *     exact FP32 accumulation, about 2^-46 of the row and column maxima per
 *     term) for the Gram matrices and rotations of oefe_orthonormalize and
 *     oefe_rayleigh_ritz (digits cut into planes for nv <= 64, inside the MMA
 *     kernels for wider blocks).
 * Inputs and outputs stay FP64; Cholesky factors, triangular inverses and the
 * setup stay FP64. The operator must be built with OEFE_STORE_F64PAIR in pair
 * mode, else the products return OEFE_ERR_STATE; the build after the switch
 * uses the new arithmetic. Returns OEFE_ERR_ARG for another mode. No
 * counterpart in the paper (the paper's machines had full-rate FP64). */
int oefe_set_f64_products(oefe_ctx_t ctx, int mode);

/* oefe_set_product_shape -- launch shape of the FP32-pair cell products of the
 * single-leaf cells. shape -1 (default): each shape is timed once at the first
 * pair product of the context and the fastest is kept; 0: 4 complex (8 real)
 * vectors per CTA of 512 threads; 1: 2 complex (4 real) vectors per CTA of
 * 384 threads; 2: 2 complex (4 real) vectors per CTA of 512 threads. Every
 * shape computes the same numbers. Returns OEFE_ERR_ARG for another value. */
int oefe_set_product_shape(oefe_ctx_t ctx, int shape);

#ifdef __cplusplus
}
#endif
#endif /* OEFE_H */
