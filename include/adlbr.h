/*
 * adlbr.h -- C ABI of the GB300 (sm_103a) AD-LBR library, libadlbr.so.
 *
 * AD-LBR is the anisotropic-diffusion scheme of J. Fehrenbach and J.-M.
 * Mirebeau, "Sparse Non-Negative Stencils for Anisotropic Diffusion"
 * (arXiv 1301.3925).  For a field of symmetric positive definite tensors D(z)
 * on a Cartesian grid, the library builds at every point the stencil V(z)
 * (6 offsets in 2D, 12 in 3D, symmetric: V = -V) and its non-negative
 * weights gamma_z(e) by lattice basis reduction (Sec. 2), and applies the
 * symmetric, matrix-free operator
 *
 *     A u = (1/2) grad E_h(u),   E_h(u) = sum_z sum_{e in V(z)} gamma_z(e) (u(z+e) - u(z))^2
 *
 * (Eq. def:E*, grid step h = 1) in explicit Euler steps u <- u - dt A u
 * (Sec. 4.4) and implicit steps (I + dt A) x = b solved by conjugate
 * gradients (Sec. 4.2, Eq. elliptic).
 *
 * Conventions for every entry point:
 *  - Arrays are device pointers owned by the caller, contiguous, row-major
 *    with x fastest: point (x, y[, z]) is element x + n0 (y + n1 z).
 *  - Work is enqueued on the given CUDA stream and is asynchronous unless the
 *    entry point says otherwise; buffers must stay alive until it completes.
 *  - Every entry point returns an adlbr_status; no exception or abort crosses
 *    the ABI.  adlbr_last_error() gives a message for the calling thread.
 *  - The library owns the storage behind an adlbr_stencils handle.
 *  - Offsets and weights are bit-exact functions of D: offsets are exactly
 *    those of an exactly D-obtuse superbase (every decision is the exact
 *    sign of a sum of integer multiples of D's entries), put in a canonical
 *    order and sign (see adlbr_stencils_export).
 */
#ifndef ADLBR_H
#define ADLBR_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ADLBR_OK = 0,
    ADLBR_E_ARG = 1,           /* null pointer, bad enum, bad scalar */
    ADLBR_E_SHAPE = 2,         /* bad grid extents or mismatched handles */
    ADLBR_E_NOT_SPD = 3,       /* some D(z) is not symmetric positive definite */
    ADLBR_E_NONFINITE = 4,     /* some D(z) has a NaN or infinite entry, or a
                                  solver's residual became non-finite */
    ADLBR_E_NOT_CONVERGED = 5, /* iteration limit reached (CG, reduction) */
    ADLBR_E_TIMEOUT = 6,       /* a bounded device-side wait gave up */
    ADLBR_E_CUDA = 7,          /* a CUDA runtime call failed */
    ADLBR_E_RANGE = 8,         /* an offset does not fit the stencil format */
    ADLBR_E_INTERNAL = 9       /* library invariant broken; in the bounds-
                                  checked build (see adlbr_version), also an
                                  index or stencil-radius check that failed */
} adlbr_status;

typedef enum { ADLBR_F64 = 0, ADLBR_F32 = 1, ADLBR_F16 = 2, ADLBR_BF16 = 3 } adlbr_dtype;

/* Boundary rule (Sec. 1): NEUMANN drops every pair (z, z+e) with z+e outside
 * the grid, V(z; h) = {e in V(z) : z + h e in Omega_h}; PERIODIC wraps. */
typedef enum { ADLBR_NEUMANN = 0, ADLBR_PERIODIC = 1 } adlbr_boundary;

typedef struct {
    int32_t dim;   /* 2 or 3 */
    int32_t bc;    /* adlbr_boundary */
    int64_t n[3];  /* extents; n[0] is x (fastest); n[2] ignored when dim == 2 */
} adlbr_grid;

typedef struct adlbr_stencils adlbr_stencils; /* opaque, library-owned */

/* Library version string.  The bounds-checked build of the library
 * (libadlbr_checked.so, compiled with -DADLBR_BOUNDS_CHECK) says
 * "bounds-checked" here.  In that build every data-dependent index of the
 * operator kernels (neighbour positions in the shared window and in the
 * grid, entries of the gather table) is checked before the access: an index
 * out of range is skipped and recorded in the handle's sticky status, and
 * the 2D AD-LBR build checks every offset of non-zero weight against the
 * bound |e| <= max(kappa(D), sqrt 2) (Sec. 4.1, Remark "Stencil
 * radius"; the sqrt 2 covers nearly isotropic tensors).  A failed check
 * is returned as ADLBR_E_INTERNAL by adlbr_stencils_check, or by
 * adlbr_stencils_destroy when no check collected it.  Results are otherwise
 * those of the normal build.  Each compute entry point and stage (tensor,
 * build, operator) also opens an NVTX range named after it, in both
 * builds. */
const char *adlbr_version(void);

/* Message describing the last non-OK status returned on the calling thread. */
const char *adlbr_last_error(void);

/*
 * adlbr_build_stencils -- the AD-LBR stencils of Sec. 2 at every grid point.
 *
 * 2D (Sec. 2, Eq. GaussAlgo and the construction after Corollary
 * ObtuseSuperBaseFromReducedBasis2; Eqs. def:Vz, def:GammaZ): a reduced basis
 * (e, f) for M ~ adj(D), f negated so that <e, M f> <= 0, superbase
 * (e0, e1, e2) = (e, f, -e-f), V = {+-e_i}, gamma(+-e_i) =
 * -<e_{i+1}^perp, D e_{i+2}^perp>/2.
 * 3D (Sec. 2, Def. ReducedBasis, Prop. MakeObtuse, Lemma Selling / Eq.
 * DSum3D): a D-obtuse superbase (e0..e3), V = {e_k x e_l}, gamma(e_k x e_l) =
 * -<e_i, D e_j>/2 for {i,j,k,l} = {0,1,2,3}.
 *
 *  g     grid (dim 2 or 3, boundary rule used by later applies).
 *  D     device, D_t elements: 2D three planes (Dxx, Dxy, Dyy), 3D six planes
 *        (Dxx, Dyy, Dzz, Dxy, Dxz, Dyz); plane k starts at element k * N,
 *        N = number of grid points.  D_t is ADLBR_F64 or ADLBR_F32.
 *  w_t   storage type of the weights: ADLBR_F64, ADLBR_F32 or ADLBR_F16 (F16
 *        keeps a per-point power-of-two scale, so small weights do not
 *        underflow).
 *  out   *out == NULL: a new handle is allocated (cudaMalloc) and returned.
 *        *out != NULL: must be a handle made for the same grid and w_t; it
 *        is rebuilt in place with no allocation (usable inside CUDA graphs).
 *
 * Points whose tensor is not SPD or not finite, or whose offsets leave the
 * storage range (|coordinate| > 2047 in 2D, > 127 for the 3D superbase),
 * get an all-zero stencil and set a sticky error flag in the handle; the
 * call itself does not synchronise.  adlbr_stencils_check() reports it.
 */
adlbr_status adlbr_build_stencils(const adlbr_grid *g, const void *D, adlbr_dtype D_t,
                                  adlbr_dtype w_t, adlbr_stencils **out, cudaStream_t stream);

/*
 * Stencil schemes.  ADLBR_SCHEME_ADLBR is the method of the paper (the
 * stencils of adlbr_build_stencils).  ADLBR_SCHEME_ANN is the paper's
 * comparison scheme A-NN, the axes-directed non-negative six-point scheme of
 * Sec. 4.1, Remark rem:WG (2D only): for D = [[a, b], [b, c]] the stencil
 * {(+-1, 0), (0, +-1), +-(p, q)} with 2 gamma(+-1, 0) = a - (p/q) b,
 * 2 gamma(0, +-1) = c - (q/p) b, 2 gamma(+-(p, q)) = b / (p q), where p, q are
 * non-zero integers with b p q >= 0, |b|/c <= |p/q| <= a/|b| (Eq. ineqPQ) and
 * max(|p|, |q|) minimal (the simplest fraction of that interval, unique;
 * every comparison is an exact sign); b = 0 gives the four-point stencil.
 * Its radius can reach the order of kappa^2 (Remark "Stencil radius").
 */
typedef enum { ADLBR_SCHEME_ADLBR = 0, ADLBR_SCHEME_ANN = 1 } adlbr_scheme;

/*
 * adlbr_build_stencils_scheme -- adlbr_build_stencils for the given scheme
 * (arguments and error rules as there; |p|, |q| > 2047 is ADLBR_E_RANGE for
 * A-NN).  An A-NN handle works with adlbr_apply, the explicit and implicit
 * steps (CG and Jacobi-PCG), adlbr_stencils_export (the canonical half-
 * stencil, as for AD-LBR) and adlbr_stencils_max_diag; the learned
 * preconditioner, the gather form and the batched step take AD-LBR handles
 * only (ADLBR_E_ARG otherwise).
 */
adlbr_status adlbr_build_stencils_scheme(const adlbr_grid *g, const void *D, adlbr_dtype D_t,
                                         adlbr_dtype w_t, int scheme, adlbr_stencils **out,
                                         cudaStream_t stream);

/* The scheme of a handle (adlbr_scheme). */
adlbr_status adlbr_stencils_scheme(const adlbr_stencils *s, int *scheme);

/* Synchronises `stream`, returns the handle's sticky build status
 * (ADLBR_OK, ADLBR_E_NONFINITE, ADLBR_E_NOT_SPD, ADLBR_E_RANGE,
 * ADLBR_E_NOT_CONVERGED, ADLBR_E_TIMEOUT when an operator kernel on this
 * handle gave up a bounded wait for a tile copy, or ADLBR_E_INTERNAL when a
 * check of the bounds-checked build failed) and clears it. */
adlbr_status adlbr_stencils_check(adlbr_stencils *s, cudaStream_t stream);

/* Grid of a handle. */
adlbr_status adlbr_stencils_grid(const adlbr_stencils *s, adlbr_grid *g);

/*
 * adlbr_stencils_export -- the canonical half-stencil of every point.
 *
 *  offs  device int16 [N][K][dim], K = 3 (2D) or 6 (3D): the offsets of
 *        V(z) / {+-1}; an offset whose weight is exactly zero is written as
 *        the zero vector; every other offset has its first non-zero
 *        coordinate (x, then y, then z) positive; the K pairs are sorted
 *        lexicographically on (x, y[, z]).
 *  w     device [N][K] weights gamma_z(+-e) in the same order: double when
 *        the handle stores F64 weights, float otherwise (F16 storage is
 *        widened exactly).
 */
adlbr_status adlbr_stencils_export(const adlbr_stencils *s, int16_t *offs, void *w,
                                   cudaStream_t stream);

/* Frees the handle (waits for the device).  Returns ADLBR_OK, or in the
 * bounds-checked build ADLBR_E_INTERNAL when a check failed that no
 * adlbr_stencils_check collected (the handle is freed all the same). */
adlbr_status adlbr_stencils_destroy(adlbr_stencils *s);

/*
 * adlbr_apply -- Au = A u with A = (1/2) grad E_h (Eq. def:E*, h = 1):
 *   (Au)(z) = sum_{e in V(z)} gamma_z(e) (u(z) - u(z+e))
 *           + sum_{(y, e): e in V(y), y + e = z} gamma_y(e) (u(z) - u(y)),
 * pairs leaving the grid dropped (NEUMANN) or wrapped (PERIODIC).
 *
 *  u    device, N elements of u_t (F64, F32, F16 or BF16).
 *  Au   device, N elements: double when u_t == ADLBR_F64, float otherwise
 *       (accumulation is in that type).  Must not alias u.
 * In the scatter form the transpose terms are added with atomic operations,
 * so the rounding of Au (and of the solvers built on it) can differ in the
 * last bits from run to run; the gather form (adlbr_operator_form) is
 * deterministic.  The dot products and norms of the solvers reduce in a
 * fixed order.  The call that builds the handle's gather table synchronises
 * the stream.
 */
adlbr_status adlbr_apply(const adlbr_stencils *s, const void *u, void *Au, adlbr_dtype u_t,
                         cudaStream_t stream);

/*
 * Form of the operator's evaluation (not in the paper, which applies an
 * assembled sparse matrix).  Both forms compute the same A u (Eq. def:E*);
 * they differ in the order of the FP32 additions only.
 *
 *  ADLBR_OP_SCATTER  one thread per point adds its own edges and pushes the
 *                    transposed terms to the far ends (shared-memory and L2
 *                    atomic additions); needs nothing but the stencils.
 *  ADLBR_OP_GATHER   each point sums its whole row and writes it once: no
 *                    atomics, so the results are the same bits from run to
 *                    run.  It needs a table built from the stencils: per
 *                    point its own weights, the weight its neighbour holds
 *                    for each shared pair (the reciprocal offset), and a list
 *                    of the remaining incoming edges, all at the point's F16
 *                    scale (exact, except a neighbour weight below 2^-14 of
 *                    the point's largest, which is rounded to the nearest F16
 *                    subnormal there).  About 28 bytes per point plus 4 per
 *                    incoming edge without a reciprocal, and 9 bytes per point
 *                    of build temporaries; cudaMalloc on the first build, one
 *                    stream synchronisation per build.  Available for 2D
 *                    handles with F16 weights, vectors in F32, F16 or BF16,
 *                    and offsets within +-127; elsewhere the scatter form
 *                    runs.  Measured slower than the scatter form on GB300
 *                    (2.0x on the 4096^2 CED stencils), so it is not the
 *                    default.
 *  ADLBR_OP_AUTO     (default) the scatter form.
 * Rebuilding the stencils in place invalidates the table; it is rebuilt when
 * next needed.
 */
typedef enum { ADLBR_OP_AUTO = 0, ADLBR_OP_SCATTER = 1, ADLBR_OP_GATHER = 2 } adlbr_operator_form;

adlbr_status adlbr_stencils_set_operator(adlbr_stencils *s, int form);

/* The handle's form setting, and 1 in *gather_ready when its gather table
 * matches the current stencils (either pointer may be NULL). */
adlbr_status adlbr_stencils_get_operator(const adlbr_stencils *s, int *form, int *gather_ready);

/* Bytes of scratch that adlbr_step_explicit needs for u_t. */
size_t adlbr_step_scratch_bytes(const adlbr_stencils *s, adlbr_dtype u_t);

/*
 * adlbr_step_explicit -- nsteps explicit Euler steps of Sec. 4.4,
 * (u^{n+1} - u^n)/dt = div(D grad u^n), i.e. u <- u - dt A u, in place.
 *
 *  u        device, N elements of u_t; the result overwrites it.  For F16 and
 *           BF16 the update is computed in FP32 and rounded once per step.
 *  scratch  device, adlbr_step_scratch_bytes(s, u_t) bytes, caller-owned:
 *           the accumulator of dt A u (scatter form), or the second buffer of
 *           the u^n -> u^{n+1} ping-pong (gather form).
 *  dt       time step; the scheme is monotone for dt <= 1 / max_z A_zz.
 */
adlbr_status adlbr_step_explicit(const adlbr_stencils *s, void *u, void *scratch, adlbr_dtype u_t,
                                 double dt, int nsteps, cudaStream_t stream);

/*
 * adlbr_build_step_explicit -- the stencils of D built into *s (Sec. 2, as
 * adlbr_build_stencils) and one explicit step u <- u - dt A u with them
 * (Sec. 4.4, as adlbr_step_explicit), the step of a loop that re-stencils
 * every step (the CED loop of Sec. 4.4).
 *
 *  g, D, D_t, w_t, s  as adlbr_build_stencils (*s == NULL allocates).
 *  u        device FP32, N elements, updated in place.
 *  scratch  device, adlbr_step_scratch_bytes(*s, ADLBR_F32) bytes (N floats).
 * For a 2D grid with FP32 D, F16 weights, a non-periodic boundary, nx % 4 ==
 * 0 and u 16-byte aligned (and the handle not set to the gather form) the
 * construction runs inside the operator's kernel: each point's stencil is
 * built, stored in the handle and applied by the same thread; once the
 * handle holds a build, each point starts from its previous stencil, which
 * is certified exactly (and repaired, or rebuilt from scratch, where it no
 * longer fits D).  Otherwise this is adlbr_build_stencils followed by
 * adlbr_step_explicit.  Either way the stencils are those of
 * adlbr_build_stencils, bit for bit as adlbr_stencils_export writes them
 * (its canonical order and signs), and u equals the two-call result to FP32
 * rounding (the order of the atomic additions).  Errors as the two calls; a failed build is reported, as
 * there, by adlbr_stencils_check.  If that check returns ADLBR_E_TIMEOUT (a
 * tile's window copy never arrived), the tiles concerned were neither built
 * nor stepped: the stencils and u are then undefined.
 */
adlbr_status adlbr_build_step_explicit(const adlbr_grid *g, const void *D, adlbr_dtype D_t, adlbr_dtype w_t,
                                       adlbr_stencils **s, float *u, void *scratch, double dt,
                                       cudaStream_t stream);

/*
 * adlbr_step_explicit_noalloc -- adlbr_step_explicit without any allocation.
 *
 * The paper has no counterpart: this entry point is for callers that cannot
 * allocate device memory while they step -- code inside a host application or
 * framework that owns the device's whole memory pool, a real-time loop that
 * must not call an allocator (cudaMalloc can block and synchronise the
 * device), or a plugin that is not allowed to allocate at all.  It computes
 * exactly what adlbr_step_explicit computes, but the scratch buffer (the
 * accumulator of dt A u) is a fixed 16 MiB array inside this library, which
 * every GPU that loads the library holds until the process exits.
 *
 *  - Limit: at most 4,194,304 grid points for F32, F16 and BF16 u and
 *    2,097,152 for F64 u; larger grids return ADLBR_E_SHAPE.
 *  - It calls no cudaMalloc, cudaFree or other allocating routine.  Its
 *    first call on a device (nsteps may be 0 for this warm-up) looks up the
 *    array's device address (cudaGetSymbolAddress) and caches it with the
 *    current context: make that first call before any stream capture.  A
 *    call under another context (for instance after cudaDeviceReset) looks
 *    the address up again.
 *  - All calls share the one array, which keeps the last call's contents
 *    (each call clears the part it uses before using it).  Calls that may
 *    overlap on the GPU -- on different streams, for different handles or
 *    from different threads -- race on it and give wrong results: serialise
 *    them.
 *  - The current device must be the handle's device (else ADLBR_E_ARG).
 */
adlbr_status adlbr_step_explicit_noalloc(const adlbr_stencils *s, void *u, adlbr_dtype u_t,
                                         double dt, int nsteps, cudaStream_t stream);

/*
 * adlbr_step_implicit -- one implicit step: solves (I + dt A) x = rhs by
 * conjugate gradients (the discretised Eq. elliptic of Sec. 4.2 with
 * lambda = dt, solved by CG as there).  FP32 vectors; every dot product and
 * norm is accumulated from exact products in float-float within a thread and
 * a warp (about 48 significant bits) and in FP64 across warps and blocks,
 * with a deterministic reduction; alpha and beta are computed on the device.  Each round starts from the true residual
 * rhs - (x + dt A x), evaluated with the operator accumulated in FP64, and
 * runs CG until the recursively updated residual satisfies
 * |r| <= rtol |rhs|; a new round (iterative refinement) follows while the
 * true residual is above rtol and still halves per round.  Because x is
 * stored in FP32, the true residual cannot go much below
 * eps_32 |I + dt A| (a few 1e-6 at dt = 200 times the explicit limit);
 * relres_out reports it.
 *
 *  rhs         device float [N].
 *  x           device float [N]: initial guess on entry, solution on exit.
 *  precond     0: plain CG.  1: flexible CG preconditioned by the U-Net of
 *              adlbr_unet_* with parameters nn (see below): z = r/d + gamma c,
 *              c the network's coarse correction, gamma its Galerkin step
 *              length <c, r - (I + dt A) r/d> / <c, (I + dt A) c> (two operator
 *              applications per iteration).  Plain CG is its
 *              fallback: when the preconditioned recursive residual grows
 *              tenfold above its best value or does not halve within 100
 *              iterations, the solve restarts from the initial guess with
 *              plain CG (iters_out then counts both; adlbr_last_fallback()
 *              returns 1).  2: CG preconditioned by the diagonal
 *              d = 1 + dt A_zz (z = r / d; alpha = <r,z> / <p,(I + dt A) p>,
 *              beta = <r,z>_new / <r,z>_old), the same stopping test and
 *              refinement rounds as plain CG; 2D and 3D.
 *  nn          preconditioner parameters (precond == 1), else ignored.
 *  iters_out   iterations performed (may be NULL).
 *  relres_out  final true relative residual |rhs - (I + dt A) x| / |rhs|.
 * Every solver (precond 0, 1, 2) stops by the same rule: refinement rounds
 * from the FP64 true residual, each run until the recursive residual meets
 * rtol, while the true residual is above rtol and still halves per round.
 * ADLBR_OK then means that the last round converged; the true residual may
 * still sit above rtol at the FP32 floor of x (adlbr_last_residual_met()
 * tells which).
 * The first call on a handle allocates its solver workspace (cudaMalloc);
 * later calls reuse it.  Synchronises the stream every few iterations.
 * Returns ADLBR_E_NOT_CONVERGED if maxit is reached first and
 * ADLBR_E_NONFINITE if the residual becomes non-finite (e.g. a NaN in rhs).
 */
adlbr_status adlbr_step_implicit(adlbr_stencils *s, const void *rhs, void *x, double dt,
                                 double rtol, int maxit, int precond, const void *nn,
                                 int *iters_out, double *relres_out, cudaStream_t stream);

/* 1 if the last preconditioned adlbr_step_implicit call of this thread fell
 * back to plain CG, else 0 (thread-local; not in the paper). */
int adlbr_last_fallback(void);

/* 1 if the last adlbr_step_implicit call of this thread ended with its true
 * relative residual (relres_out) at or below rtol, else 0 -- also when it
 * returned ADLBR_OK at the FP32 floor of x above rtol, or failed
 * (thread-local; not in the paper). */
int adlbr_last_residual_met(void);

/* ------------------------------------------------------------------------
 * Learned preconditioner network (not in the paper): a 3-level U-Net, FP32.
 *
 *   enc1: conv3x3(cin->c1) ReLU, conv3x3(c1->c1) ReLU        -> s1 (H x W)
 *   avgpool 2x2; enc2: conv3x3(c1->c2) ReLU, conv3x3(c2->c2) ReLU -> s2
 *   avgpool 2x2; mid: conv3x3(c2->c3) ReLU, conv3x3(c3->c3) ReLU
 *   nearest x2, concat [up, s2]; dec2: conv3x3(c3+c2->c2) ReLU, conv3x3 ReLU
 *   nearest x2, concat [up, s1]; dec1: conv3x3(c2+c1->c1) ReLU, conv3x3 ReLU
 *   out: conv1x1(c1->1)
 * Convolutions are cross-correlations with zero padding.  Parameters: one
 * flat float vector, per layer in the order above weights [co][ci][ky][kx]
 * then bias [co].  Tensors: device float [batch][channel][H][W].
 * ------------------------------------------------------------------------ */
typedef struct adlbr_unet adlbr_unet; /* opaque: shape and activation buffers */

/* Allocates the activation buffers for `batch` inputs of cin x H x W
 * (H, W multiples of 4; c1 <= 64). */
adlbr_status adlbr_unet_create(int cin, int c1, int c2, int c3, int batch, int H, int W,
                               adlbr_unet **out);
adlbr_status adlbr_unet_destroy(adlbr_unet *n);

/* Run this network's forward 3x3 convolutions on the tensor cores (on != 0):
 * tcgen05 implicit GEMMs with BF16 operands (activations and weights rounded
 * to BF16, accumulation in FP32; relative output differences to the FP32
 * forward of order 1e-2), weights repacked (one launch) at every forward
 * call; a preconditioned adlbr_step_implicit packs them once per solve, and
 * the parameters must not change while it runs.  For the inference path (the preconditioner): adlbr_unet_backward
 * returns ADLBR_E_ARG after a tensor-core forward.  on = 0 returns to the FP32
 * kernels.  ADLBR_E_SHAPE if a layer has other than 16, 32 or 64 output
 * channels, or if its 9 packed weight taps and 4 staged input rows
 * (2 * (9 Co + 4 * 136) * Kp bytes, Kp = Ci rounded up to 16) exceed 225 KB:
 * at most 160 input channels for Co = 16, 128 for Co = 32, 96 for Co = 64. */
adlbr_status adlbr_unet_set_tensor_cores(adlbr_unet *n, int on);
/* Number of parameters (length of the flat parameter vector). */
int64_t adlbr_unet_num_params(const adlbr_unet *n);
/* y [batch][1][H][W] = net(params, x [batch][cin][H][W]); keeps the
 * activations (and the pointer x) for adlbr_unet_backward. */
adlbr_status adlbr_unet_forward(adlbr_unet *n, const float *params, const float *x, float *y,
                                cudaStream_t stream);
/* Gradient of sum(gy * y) for the last forward: gparams (overwritten, summed
 * over the batch) and, if gx != NULL, the input gradient gx. */
adlbr_status adlbr_unet_backward(adlbr_unet *n, const float *params, const float *gy,
                                 float *gparams, float *gx, cudaStream_t stream);
/* One Adam update (Kingma & Ba) of n parameters, step count t >= 1. */
adlbr_status adlbr_adam_step(float *params, const float *grads, float *m, float *v, int64_t n,
                             double lr, double beta1, double beta2, double eps, int t,
                             cudaStream_t stream);

/*
 * Learned preconditioner for adlbr_step_implicit (precond = 1, 2D only):
 *   M(r) = r / d + s * P(N(F(r))),
 * d = 1 + dt A_zz, s = rms(r), N the U-Net with cin = 25, batch 1 and
 * H x W = (ny / 4) x (nx / 4), P the repetition of a coarse value over its
 * 4 x 4 block, and F(r) the coarse input: the 16 values of r / s in each block
 * (space to depth, channel 4 dy + dx), then the block means of
 * log(1 + dt w_k) for the three canonical half-stencil weights and of the
 * three canonical offsets / 8 (adlbr_stencils_export order).  The solver is
 * flexible CG (Polak-Ribiere beta); grid extents must be multiples of 16.
 */
typedef struct {
    adlbr_unet *net;
    const float *params; /* device, adlbr_unet_num_params(net) floats */
} adlbr_nn_precond;

/*
 * adlbr_nn_training_pairs -- (residual, error) pairs generated by the solver
 * for training the preconditioner: CG on (I + dt A) x = rhs from x0 = rhs is
 * run to convergence (x*), then the system is solved again -- by CG when
 * nn == NULL, by the preconditioned solver with nn otherwise, so that the
 * network also sees the residuals it will meet -- and at iterations 0, every,
 * 2 every, ... (at most max_pairs) the coarse input F(r_k)
 * [25][ny/4][nx/4] is recorded into feats and the target, the block means of
 * (x* - x_k - r_k / d) / s_k, [ny/4][nx/4] into targets, i.e. what N should
 * output at r_k.  xbuf: device float [N] scratch.  *n_pairs receives the
 * count.  Synchronises.
 */
adlbr_status adlbr_nn_training_pairs(adlbr_stencils *s, const float *rhs, double dt, double rtol,
                                     int maxit, int every, int max_pairs,
                                     const adlbr_nn_precond *nn, float *feats, float *targets,
                                     float *xbuf, int *n_pairs, cudaStream_t stream);

/* z = M(r) for the preconditioner above (one application; synchronises). */
adlbr_status adlbr_nn_precondition(adlbr_stencils *s, const adlbr_nn_precond *nn, double dt,
                                   const float *r, float *z, cudaStream_t stream);

/* max_z A_zz over the grid (2D or 3D; FP32 accumulation), e.g. for the
 * explicit limit dt = 1 / max A_zz.  Synchronises. */
adlbr_status adlbr_stencils_max_diag(adlbr_stencils *s, double *out, cudaStream_t stream);

/* Mean squared error loss = mean((y - t)^2) over n values (FP64 reduction)
 * and its gradient gy = 2 (y - t) / n.  loss_out may be NULL (no sync). */
adlbr_status adlbr_mse_grad(const float *y, const float *t, int64_t n, float *gy,
                            double *loss_out, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Coherence-enhancing diffusion (Sec. 4.4, Eq. parabolique; in 3D as in the
 * 3D experiments of Sec. 5), FP32.
 * ------------------------------------------------------------------------ */

/* Bytes of scratch for adlbr_ced_tensor / adlbr_ced_step on grid g. */
size_t adlbr_ced_scratch_bytes(const adlbr_grid *g);

/*
 * adlbr_ced_tensor -- the diffusion tensor D(J_rho(grad u_sigma)) of Sec. 4.4:
 * u_sigma = K_sigma * u, J_rho = K_rho * (grad u_sigma grad u_sigma^T); D has
 * the eigenvectors v1, v2 of J_rho (eigenvalues mu1 >= mu2) with eigenvalues
 * lambda1 = alpha and lambda2 = alpha + (1 - alpha) exp(-C / (mu1 - mu2)^2)
 * (exp(-C/0) = 0).  sigma, rho: standard deviations of the Gaussians, which
 * are truncated at radius int(3 s + 0.5) <= 32 and normalised; the image is
 * reflected about its border (u(-1) = u(0)) for the convolutions and for the
 * centred-difference gradient.
 *
 * In 3D, J_rho has six channels and eigenvalues mu1 >= mu2 >= mu3; D keeps
 * its eigenvectors with lambda1 = alpha, lambda2 = alpha + (1 - alpha)
 * exp(-C / (mu1 - mu2)^2), lambda3 = alpha + (1 - alpha) exp(-C / (mu1 -
 * mu3)^2) (eigen-decomposition by Jacobi rotations in FP32).
 *
 *  g        2D or 3D grid.
 *  u        device float [N].
 *  D        device float [3][N]: planes Dxx, Dxy, Dyy (2D), or [6][N]: Dxx, Dyy,
 *           Dzz, Dxy, Dxz, Dyz (3D) -- the build_stencils input.
 *  scratch  device, adlbr_ced_scratch_bytes(g) bytes.
 */
adlbr_status adlbr_ced_tensor(const adlbr_grid *g, const float *u, float *D, double sigma,
                              double rho, double alpha, double C, void *scratch,
                              cudaStream_t stream);

/*
 * adlbr_eed_tensor -- the edge-enhancing diffusion tensor of the 3D MRI
 * experiment (Sec. 5): J_rho and its eigenvectors v1, v2, v3 (eigenvalues
 * mu1 >= mu2 >= mu3) as in adlbr_ced_tensor, and D with the eigenvalues
 * lambda1 = 1 - exp(-C / mu1^2) on v1, lambda2 = 1 - exp(-C / mu2^2) on v2,
 * lambda3 = 1 on v3 (exp(-C/0) = 0).  The eigenvalues lie in (0, 1], so
 * kappa(D) = (lambda_max / lambda_min)^(1/2) grows as C falls.
 *
 *  g        3D grid (ADLBR_E_SHAPE otherwise).
 *  u, D, scratch  as adlbr_ced_tensor (D: planes Dxx, Dyy, Dzz, Dxy, Dxz, Dyz).
 *  sigma, rho  standard deviations as adlbr_ced_tensor; C > 0 and finite
 *           (ADLBR_E_ARG otherwise).
 */
adlbr_status adlbr_eed_tensor(const adlbr_grid *g, const float *u, float *D, double sigma, double rho, double C,
                              void *scratch, cudaStream_t stream);

/*
 * adlbr_ced_stencils -- adlbr_ced_tensor followed by adlbr_build_stencils
 * (F32 tensor, weights stored as w_t): the AD-LBR stencils of
 * D(J_rho(grad u_sigma)), the re-stencil of one CED step.  D goes through
 * the scratch buffer.  *s follows adlbr_build_stencils' rules (allocated when
 * NULL, rebuilt in place otherwise).
 */
adlbr_status adlbr_ced_stencils(adlbr_stencils **s, const adlbr_grid *g, const float *u,
                                void *scratch, double sigma, double rho, double alpha, double C,
                                adlbr_dtype w_t, cudaStream_t stream);

/*
 * adlbr_ced_step -- nsteps steps of the CED loop of Sec. 4.4 with a frozen
 * tensor per step (D_n = D(u(n dt)), Sec. 1): tensor (adlbr_ced_tensor),
 * then stencils and one explicit step u <- u - dt A u as
 * adlbr_build_step_explicit (the stencils of adlbr_build_stencils into *s,
 * allocated on the first call and rebuilt in place afterwards, weights
 * stored as w_t; on the grids it names, built inside the operator's kernel
 * from each point's previous stencil).  u is FP32 and updated in place.
 */
adlbr_status adlbr_ced_step(adlbr_stencils **s, const adlbr_grid *g, float *u, void *scratch,
                            double sigma, double rho, double alpha, double C, double dt,
                            int nsteps, adlbr_dtype w_t, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Batched explicit steps (not in the paper: its explicit scheme of Sec. 4.4,
 * u <- u - dt_i A_i u_i, applied to many images and volumes of uneven sizes
 * at once).
 * ------------------------------------------------------------------------ */
typedef struct adlbr_batch adlbr_batch; /* opaque: items, work list, accumulator, graph */

/*
 * adlbr_batch_create -- fixes a batch of n_items items: the stencil handles
 * s[i] (2D or 3D, any weight type, built beforehand and kept alive by the
 * caller), the FP32 u buffers u[i] (device, N_i floats each, updated in
 * place by adlbr_batch_step) and the time steps dt[i] >= 0.
 * It allocates one accumulator for all items and a work list of tiles (2D
 * tiles of the shared-window operator, 3D blocks of the scatter operator).
 * With autotune != 0 it times the accumulate kernel of every candidate tile
 * shape on this batch (u is not modified) and keeps the fastest, else the
 * first candidate (64 x 32 tiles, 32 x 8 x 4 blocks).  One step (accumulator
 * reset, one persistent accumulate kernel over the 2D tiles of all images and
 * one over the 3D blocks of all volumes, each with dynamic tile hand-out, one
 * finalize kernel) is recorded as a CUDA graph.
 * Synchronises the stream.  The handles' stencils must not be rebuilt with a
 * different shape while the batch lives (rebuilding in place is fine).
 */
adlbr_status adlbr_batch_create(int n_items, adlbr_stencils *const *s, float *const *u,
                                const double *dt, int autotune, adlbr_batch **out,
                                cudaStream_t stream);

/* nsteps explicit steps of every item: nsteps launches of the recorded
 * graph on `stream`. */
adlbr_status adlbr_batch_step(adlbr_batch *b, int nsteps, cudaStream_t stream);

/* The chosen shape (shape_out[5] = 2D tile width, height, 3D block x, y,
 * planes per thread), the tuned accumulate time in ms (0 without tuning),
 * the total number of points and of tiles.  Any pointer may be NULL. */
adlbr_status adlbr_batch_config(const adlbr_batch *b, int *shape_out, double *tuned_ms,
                                int64_t *points, int *n_tiles);

adlbr_status adlbr_batch_destroy(adlbr_batch *b);

/* ------------------------------------------------------------------------
 * Block vectors of the periodic spectral study (Sec. 4, Fig. Eigen: the
 * smallest eigenvalues of the operator on a periodic grid).  The block
 * eigensolver needs, besides A X (adlbr_apply), the Gram matrices of its
 * search blocks, linear combinations of their rows and the residual rows.
 * A block is m <= 64 rows of n FP64 values on the device, row-major with row
 * stride n.  Every sum is taken by one CTA in a fixed order: the results are
 * deterministic.  Asynchronous on `stream`; ADLBR_E_ARG for a null pointer,
 * m or k outside [1, 64] or n < 1.
 * ------------------------------------------------------------------------ */

/* G = A B^T: G[i * mb + j] = sum_p A[i][p] B[j][p] (device, ma * mb). */
adlbr_status adlbr_block_dot(const double *A, int ma, const double *B, int mb, int64_t n, double *G,
                             cudaStream_t stream);

/* out = C^T S: out[r][p] = sum_i C[i * k + r] S[i][p] for r < k, i < m (the
 * sum in order of i).  C: device, m * k, row-major.  out (k rows) must not
 * overlap S. */
adlbr_status adlbr_block_combine(const double *C, int m, int k, const double *S, int64_t n, double *out,
                                 cudaStream_t stream);

/* R[i] = AX[i] - theta[i] X[i] and rnorm[i] = ||R[i]||_2 for the m rows
 * (theta, rnorm: device, m values).  R may be AX itself. */
adlbr_status adlbr_block_residual(const double *AX, const double *X, const double *theta, int m, int64_t n,
                                  double *R, double *rnorm, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* ADLBR_H */
