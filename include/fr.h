/*
 * fr.h -- C ABI of the B300 (sm_103a) Flux Reconstruction right-hand side.
 *
 * The library evaluates the semi-discrete FR operator of Witherden, Farrington
 * & Vincent, "PyFR: An Open Source Framework for Solving Advection-Diffusion
 * Type Problems on Streaming Architectures using the Flux Reconstruction
 * Approach" (arXiv 1312.1638):
 *
 *     dU/dt = R(U) = -J^{-1} [ M3 D~ + (M1 - M3 M2) F~ ]      (Eq. negdivconf,
 *                                                           App. A)
 *
 * for the Euler and compressible Navier-Stokes equations (Sec. 4) on meshes of
 * quadrilaterals, triangles and hexahedra, with Rusanov interface fluxes
 * (App. B), LDG common solution/viscous flux (Sec. 4.3), boundary ghost states
 * (App. C) and classical RK4 time stepping (end of Sec. 2).
 *
 * Conventions shared by every call
 * --------------------------------
 * State layout (Sec. 3.3, SoA packing with variable stride |Omega_e|): one
 * buffer per element block, [nupts][nvars][ld] with column index
 * alpha*ld + n for variable alpha of element n.  ld >= nelem is chosen by the
 * library (a multiple of 128) and reported by fr_layout().  Columns n >= nelem
 * are padding: the library never reads them for anything but dense operator
 * products and leaves their output unspecified.
 *
 * Element types and node orderings (fr_eblock.nodes, host, [nelem][nnodes][ndims]):
 *   FR_QUAD 4 nodes: tensor product of {-1,1}^2, xi fastest; 9 nodes: tensor
 *           product of {-1,0,1}^2, xi fastest.
 *   FR_TRI  3 nodes: (-1,-1),(1,-1),(-1,1); 6 nodes: those, then mid-points of
 *           edges 0-1, 1-2, 2-0.
 *   FR_HEX  8 nodes: tensor product of {-1,1}^3 (xi, eta, zeta; xi fastest).
 * Faces: quad 0:eta=-1 1:xi=+1 2:eta=+1 3:xi=-1; tri 0:v0-v1 1:v1-v2 2:v2-v0;
 * hex 0:zeta=-1 1:eta=-1 2:xi=+1 3:eta=+1 4:xi=-1 5:zeta=+1.
 * Solution points: tensor Gauss-Legendre (quad, hex, xi fastest); for
 * triangles the interior nodes of the degree-(p+3) equispaced lattice (the
 * paper's Williams-Shunn points are not printed).  Flux points: Gauss-Legendre
 * on every face.  Correction functions: DG (Sec. 5).
 *
 * Precision: FR_PREC_FP64 state buffers are double; every other precision
 * uses float state buffers.
 *
 * Streams: `stream` arguments are cudaStream_t values passed as void*
 * (NULL = legacy default stream).  Calls that take a stream are
 * stream-ordered and return without synchronising the host unless stated.
 *
 * Errors: every call returns an fr_status; no exception crosses the ABI.
 * fr_last_error() returns a message for the most recent failure of that
 * context (or of fr_setup when ctx is NULL).  On error nothing is freed that
 * the caller owns.
 */
#ifndef FR_H
#define FR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fr_ctx fr_ctx;   /* opaque; owned by the library */

typedef enum {
    FR_OK = 0,
    FR_ERR_ARG = 1,          /* bad argument (NULL pointer, bad block index, ...) */
    FR_ERR_MESH = 2,         /* unmatched flux point, non-positive Jacobian ...   */
    FR_ERR_CUDA = 3,         /* a CUDA runtime call failed                         */
    FR_ERR_NONFINITE = 4,    /* a NaN/Inf was detected in a state                  */
    FR_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up                 */
    FR_ERR_UNSUPPORTED = 6,  /* combination not implemented / no GPU context       */
    FR_ERR_OOM = 7           /* device allocation failed                           */
} fr_status;

typedef enum { FR_EULER = 0, FR_NAVIER_STOKES = 1 } fr_system;
/* FR_PREC_FP64: FP64 everywhere.  FR_PREC_FP32: FP32 everywhere (CUDA-core
 * operator products).  FR_PREC_TF32X3 / FR_PREC_BF16X3: FP32 state and
 * point-wise arithmetic; dense operator products on the tensor cores with
 * both factors split in two (TF32: 11+11 bits, BF16: 8+8 bits) and three
 * products accumulated in FP32.  On quadrilaterals and hexahedra the operator
 * products take structured kernels (the "structured_*" options of
 * fr_set_option) that multiply the operators' nonzeros in FP32 in every
 * single precision, so there these contexts compute what an FP32 one does. */
typedef enum { FR_PREC_FP64 = 0, FR_PREC_FP32 = 1, FR_PREC_BF16X3 = 2, FR_PREC_TF32X3 = 3 } fr_precision;
typedef enum { FR_QUAD = 0, FR_TRI = 1, FR_HEX = 2 } fr_etype;
/* boundary types (App. C): free-stream ("supersonic inflow") ghost, subsonic
 * outflow, no-slip isothermal wall (velocity wall_v), and a second no-slip
 * isothermal wall at the same C_pT_w moving at wall2_v (the moving plate of
 * the Couette problem, Sec. 5.2) */
typedef enum { FR_BC_FREESTREAM = 0, FR_BC_OUTFLOW = 1, FR_BC_WALL = 2, FR_BC_WALL_MOVING = 3 } fr_bctype;

/* Physical and numerical parameters (Sec. 4, Sec. 4.3, App. C). */
typedef struct {
    int32_t ndims;        /* 2 or 3 */
    int32_t order;        /* polynomial order p >= 1 */
    int32_t system;       /* fr_system */
    int32_t precision;    /* fr_precision */
    double gamma;         /* ratio of specific heats */
    double mu;            /* constant dynamic viscosity (NS) */
    double prandtl;       /* Prandtl number (NS) */
    double ldg_beta;      /* LDG beta: C = (1/2-beta) u_L + (1/2+beta) u_R */
    double ldg_tau;       /* LDG penalty tau >= 0 (dissipative sign) */
    double bc_rho, bc_v[3], bc_p;   /* free-stream ghost state */
    double outflow_p;               /* subsonic-outflow pressure */
    double wall_cpTw, wall_v[3];    /* isothermal wall: C_p T_w and velocity */
    /* Perturbation form (ref_rho = 0: the plain form).  The kernels carry
     * u' = u - u_ref about the state at rest u_ref = (ref_rho, 0, E_ref) with
     * E_ref = ref_p / (gamma - 1): interpolation and gradients act on u' (exact:
     * rows of M0 sum to one, rows of M4 to zero), pressure is formed as
     * p' = (gamma-1)(E' - rho|v|^2/2), the momentum flux carries p' and the
     * energy flux is v (E' + p' - h_ref rho') with h_ref = gamma E_ref / ref_rho,
     * and h_ref times the mass flux is added back to every energy flux (point
     * and common) before the divergence, so R_E comes out whole.  The energy
     * split is exact by linearity of R in the fluxes; dropping the constant pressure
     * flux is exact wherever the mesh preserves a free stream (affine
     * elements, quadratic 2D and trilinear 3D elements at p >= 2).  Choosing
     * the mean density and pressure keeps FP32 / split-precision results
     * accurate at low Mach number, where u and the fluxes are dominated by
     * constants whose divergence vanishes. */
    double ref_rho, ref_p;
    /* Correction functions (Sec. 5.1 runs "DG, SD and HU as defined in"
     * Vincent, Castonguay and Jameson 2011): the VCJH family
     * g_R = (P_p + (eta P_{p-1} + P_{p+1}) / (1 + eta)) / 2 with eta = 0 (DG),
     * p/(p+1) (SD) or (p+1)/p (HU).  SD and HU are defined for quadrilaterals
     * and hexahedra; a mesh with triangles accepts DG only
     * (FR_ERR_UNSUPPORTED otherwise). */
    int32_t correction;   /* fr_correction */
    double wall2_v[3];    /* velocity of FR_BC_WALL_MOVING faces */
} fr_params;

typedef enum { FR_CORR_DG = 0, FR_CORR_SD = 1, FR_CORR_HU = 2 } fr_correction;

/* One block of elements of a single type, host memory, read during fr_setup only. */
typedef struct {
    int32_t etype;        /* fr_etype */
    int32_t nnodes;       /* nodes per element (4/9 quad, 3/6 tri, 8 hex) */
    int64_t nelem;
    const double* nodes;  /* [nelem][nnodes][ndims] */
} fr_eblock;

typedef struct {
    int32_t ndims;
    int32_t nblocks;
    const fr_eblock* blocks;
    int64_t nbfaces;
    const int64_t* bfaces;    /* [nbfaces][4]: block, element, face, fr_bctype */
    int32_t nperiodic;
    const double* periodic;   /* [nperiodic][ndims] translation vectors */
} fr_mesh;

/*
 * fr_setup -- build the FR discretisation of `mesh` (Sec. 2, App. A).
 * Host work: point sets, nodal bases (Vandermonde construction, Sec. 2),
 * operator matrices M0..M6 (App. A), metric terms, flux-point pairing by
 * physical coordinates (Sec. 2: a pair must coincide; periodic translations
 * tried in every combination), L side = lexicographically smaller
 * (block, element, face), each pair visited once.
 * device >= 0: allocates operators, metric terms, pair tables and scratch on
 * that CUDA device (owned by the context, freed by fr_destroy).
 * device == -1: host-only context; only the inspection calls below work and
 * fr_rhs/fr_rk4 return FR_ERR_UNSUPPORTED.
 * Errors: FR_ERR_ARG, FR_ERR_MESH (unmatched or doubly matched flux point,
 * boundary face also paired, non-positive Jacobian), FR_ERR_UNSUPPORTED,
 * FR_ERR_CUDA / FR_ERR_OOM.  *out is NULL on failure.
 */
fr_status fr_setup(const fr_mesh* mesh, const fr_params* params, int device, fr_ctx** out);

/* Layout of block `block`: points, variables, elements and the column
 * stride ld of its state buffers (Sec. 3.3).  Any output pointer may be NULL. */
fr_status fr_layout(const fr_ctx* ctx, int block, int32_t* nupts, int32_t* nfpts,
                    int32_t* nvars, int64_t* nelem, int64_t* ld);

/* Physical coordinates of the solution points of block `block` (the element
 * mapping of Sec. 2 evaluated at x~^(u)), written to host memory
 * out[ndims][nupts][nelem]. */
fr_status fr_solution_points(const fr_ctx* ctx, int block, double* out);

/* Host copy of an operator matrix of block `block` (App. A), row-major FP64.
 * which: 0..6 = M0..M6 (M5 omitted: it is diag(M0,...,M0)), 7 = M4 - M6 M0,
 * 8 = M1 - M3 M2.  If out is NULL only rows/cols are returned. */
fr_status fr_operator(const fr_ctx* ctx, int block, int which, double* out,
                      int32_t* rows, int32_t* cols);

/* Interface pairs (Sec. 2 lookup table).  With out == NULL returns the count
 * in *npairs; otherwise writes [npairs][6] = (bL, fptL, elemL, bR, fptR, elemR). */
fr_status fr_pairs(const fr_ctx* ctx, int64_t* npairs, int64_t* out);

/*
 * fr_rhs -- r = R(u) (Eq. negdivconf) on the device.
 * u[b], r[b]: device pointers, one per block, layout [nupts][nvars][ld],
 * double for FR_PREC_FP64 else float.  r may alias u (Sec. 3.6 aliasing).
 * Stream-ordered on `stream`; returns after enqueueing.
 * Errors: FR_ERR_ARG (NULL pointer), FR_ERR_UNSUPPORTED (host-only context),
 * FR_ERR_CUDA (launch failure).
 */
fr_status fr_rhs(fr_ctx* ctx, void* const* u, void* const* r, void* stream);

/*
 * fr_rhs_host -- as fr_rhs (Eq. negdivconf, App. A), but u and r are HOST buffers (any host memory;
 * pinned memory makes the copies asynchronous).  The library copies u to a
 * device staging buffer it owns, evaluates R, copies r back and synchronises
 * `stream` before returning.  u and r may alias.
 */
fr_status fr_rhs_host(fr_ctx* ctx, const void* const* u, void* const* r, void* stream);

/*
 * Forward Euler (Sec. 3 lists it among the time steppers): nsteps steps of
 * u <- u + dt R(u), in place.  Stream-ordered, no host synchronisation; the
 * first call allocates one state-sized scratch array per block.
 * FR_ERR_ARG for a NULL/misaligned pointer or nsteps < 0.
 */
fr_status fr_euler(fr_ctx* ctx, void* const* u, double dt, int nsteps, void* stream);

/*
 * DOPRI5 (Sec. 3): nsteps fixed steps of the Dormand-Prince 5(4) pair
 * (Dormand and Prince 1980), in place, propagating the 5th-order solution.
 * The slope at the new solution is reused as the first slope of the next step
 * of the same call (6 right-hand sides per step after the first, 7 for the
 * first).  err (may be NULL): on return, the RMS norm of the last step's
 * embedded error estimate E = u5 - u4 scaled per entry by
 * atol + rtol max(|u_n|, |u_n+1|) over every real entry; then the call
 * synchronises the stream.  With err NULL it is stream-ordered.  The first
 * call allocates 8 state-sized scratch arrays per block.
 * FR_ERR_ARG for bad pointers, nsteps < 0, or (err != NULL) atol <= 0 or rtol < 0.
 */
fr_status fr_dopri5(fr_ctx* ctx, void* const* u, double dt, int nsteps, double atol, double rtol, double* err,
                    void* stream);

/*
 * fr_rk4 -- advance u in place by `nsteps` classical RK4 steps of size dt
 * (end of Sec. 2; Sec. 5.1).  Uses two library-owned state registers,
 * allocated on the first call.  Unless disabled with
 * fr_set_option(ctx, "graphs", 0) or while kernel timing is enabled, one step
 * is captured once as a CUDA graph (on a private stream) and replayed nsteps
 * times on `stream`; the graph is re-captured when u's pointers or dt change.
 * Stream-ordered; returns after enqueueing.
 */
fr_status fr_rk4(fr_ctx* ctx, void* const* u, double dt, int nsteps, void* stream);

/*
 * fr_rk_step -- the stepping call of the boundary under its generic name: the
 * same classical RK4 steps (end of Sec. 2) as fr_rk4, with the same
 * arguments, behaviour and errors.
 */
fr_status fr_rk_step(fr_ctx* ctx, void* const* u, double dt, int nsteps, void* stream);

/*
 * fr_rk4_host -- as fr_rk4 (classical RK4, end of Sec. 2), but u holds HOST
 * buffers (any host memory; pinned memory makes the copies asynchronous),
 * one per block, laid out as the device state ([nupts][nvars][ld], double
 * for FR_PREC_FP64 else float).  The library copies u to a device staging
 * buffer it owns (allocated on the first host-buffer call, shared with
 * fr_rhs_host), advances it nsteps steps as fr_rk4 does (the captured step is
 * reused from call to call), copies it back into u and synchronises `stream`
 * before returning.  Errors as fr_rk4, plus FR_ERR_CUDA / FR_ERR_OOM for the
 * copies and the staging allocation.
 */
fr_status fr_rk4_host(fr_ctx* ctx, void* const* u, double dt, int nsteps, void* stream);

/*
 * Kernel-variant autotuning (not in the paper; the paper's Sec. 3.4 leaves
 * the operator products to cuBLAS, which chooses its own kernels).  On the
 * tensor-core paths every operator product (disu: M0 U; tgradu: the corrected
 * gradient with its transform; gradfpts: M0 Q; tdivf: the corrected
 * divergence, with the RK stage on the RK4 path) can run as one of several
 * kernel variants, which differ in how many 128-column subtiles a work item
 * holds (nt) and how many warps convert the state operand (cw) or drain the
 * accumulators (eg).  fr_autotune times every variant that fits each product
 * of each block (of all blocks together when they run as one launch, see the
 * option "group_blocks"): 1 + reps RK4 steps of size 0 on a private copy of u
 * (device memory allocated and freed by the call; u is not modified), in two
 * passes over the variants, kernels timed by CUDA events, and keeps the
 * fastest in the context.  It synchronises
 * `stream`.  On the FP64 / FP32 paths it does nothing.
 * fr_get_tuning writes the context's choices as text,
 * "b0:disu=1.8.3,tgradu=1.4.4,gradfpts=1.8.3,tdivf=2.8.2;b1:..." (nt.cw.eg,
 * or "default" for the built-in rule), NUL-terminated into buf (FR_ERR_ARG if
 * size is too small); fr_set_tuning applies such text (any subset of blocks
 * and products; FR_ERR_ARG, with nothing applied, for a malformed entry or a
 * variant that does not fit the product).  Changing the choices drops the
 * captured RK4 step.
 */
fr_status fr_autotune(fr_ctx* ctx, void* const* u, int reps, void* stream);
fr_status fr_get_tuning(const fr_ctx* ctx, char* buf, int64_t size);
fr_status fr_set_tuning(fr_ctx* ctx, const char* text);

/* Context options (not in the paper): "graphs" (default 1) enables the RK4-step CUDA graph of
 * fr_rk4.  "group_blocks" (default 1): on the tensor-core paths each operator
 * product of a mesh with 2 to 4 element blocks (a mixed mesh) runs as one
 * persistent launch over the work items of every block (the D
 * interpolations of the gradient, Eq. gradufpts, of every block included);
 * 0 gives every block its own launches.  Changing it drops the captured RK4 step;
 * results are the same bits either way.  "structured_interp" (default 1):
 * where every row of an element type's
 * interpolation operator M0 (App. A) has at most 8 nonzeros (quadrilaterals
 * and hexahedra: the p+1 solution points on the line through a face point;
 * entries below 1e-15 of their row's largest are dropped), the products with
 * M0 (U^(f) and the gradient at flux points) run as a structured kernel with
 * FP32 / FP64 multiply-adds of those entries, in every precision (they need
 * no split: FP32 multiply-adds are as accurate as the split products); 0
 * uses the dense operator products.  "structured_grad" (default 1, Navier-Stokes):
 * where the corrected-gradient operator [M6 | M4 - M6 M0] (Eq. tquptsm) is
 * structured (quadrilaterals and hexahedra: row (i, s) holds the p+1
 * solution points on the line through s in direction i and the two flux
 * points ending it), the gradient Q = J^-T Q~ (Eq. gradufpts) runs as one
 * structured kernel with FP32 / FP64 multiply-adds of those entries and the
 * transform in the same pass, in every precision.  1: the tensor-line form
 * (set-up checks that one p+1 x p+3 line matrix rebuilds every row; this
 * kernel also forms Q^(f) = M5 Q when "structured_interp" is on), falling
 * back to 2 where a tile does not fit shared memory; 2: the row-wise form
 * (each row's nonzeros, at most 8); 0: the dense operator product (tensor
 * cores on the split-precision paths).  "structured_div" (default 1): the
 * same choice for the divergence operator [M3 | M1 - M3 M2] (Eq. tdivflux;
 * per direction the p+1 flux values on the line through the point and the
 * two common fluxes ending it; row-wise form: at most 24 nonzeros per row),
 * with -1/J (Eq. negdivconf) and, inside fr_rk4, the RK4 stage combination
 * applied in the same pass.  Values outside 0..2 give FR_ERR_ARG.  Changing
 * either drops the captured RK4 step.  "structured_adjoint" (default 1): the
 * adjoint's transposed products (M3^T, (M1 - M3 M2)^T, M0^T, M6^T and
 * [M0^T | (M4 - M6 M0)^T], fr_adjoint_rhs and fr_rk4_adjoint) take the
 * structured kernels where their rows allow (tensor elements; at most 8,
 * resp. 24, nonzeros per row), with FP32 / FP64 multiply-adds; 0 uses the
 * dense products.  "tc_wait_limit" (default 0 = about two seconds; value >= 0) sets
 * the SM clock cycles after which a bounded wait inside the tensor-core
 * operator GEMMs gives up: the kernel then drains its own copies and MMAs,
 * returns, and fr_sync_status reports FR_ERR_TIMEOUT; the context stays
 * usable (a small value forces this path in tests; setting the option drops
 * the captured RK4 graph).  FR_ERR_ARG for an unknown name or a bad value. */
fr_status fr_set_option(fr_ctx* ctx, const char* name, int64_t value);

/*
 * fr_adjoint_rhs -- out = (dR/du)^T lambda, the discrete adjoint of fr_rhs
 * at state u (not in the paper; the transpose of the operator chain of
 * Eq. negdivconf / App. A with the Rusanov flux of App. B and the ghost
 * states of App. C; for Navier-Stokes also the LDG common solution and
 * viscous flux of Sec. 4.3 and the corrected-gradient chain of
 * Eq. tquptsm / gradufpts).  Euler and Navier-Stokes contexts on a whole
 * mesh (FR_ERR_UNSUPPORTED for a partitioned context).
 * u, lambda, out: device buffers laid out like fr_rhs's; out may not alias
 * u or lambda.  Uses context scratch allocated on the first adjoint call
 * (Navier-Stokes: two more gradient-sized arrays per block).  The
 * Navier-Stokes adjoint overwrites the context's RHS scratch, as fr_rhs does.
 * Stream-ordered.
 */
fr_status fr_adjoint_rhs(fr_ctx* ctx, void* const* u, void* const* lambda, void* const* out, void* stream);

/*
 * fr_rk4_adjoint -- reverse sweep of `nsteps` classical RK4 steps of size dt
 * from u0 (not in the paper): on entry lambda holds dK/du_N for the state
 * u_N = RK4^nsteps(u0); on return it holds dK/du0.  Stage inputs are
 * recomputed from checkpoints of the state stored every `every` steps
 * (ceil(nsteps/every) checkpoints plus `every` states of the current block
 * and 8 work states, allocated for the call and freed before returning).
 * u0 is not modified.  Euler and Navier-Stokes contexts on a whole mesh.
 * Synchronises `stream`.
 */
fr_status fr_rk4_adjoint(fr_ctx* ctx, void* const* u0, void* const* lambda, double dt, int nsteps, int every,
                         void* stream);

/*
 * fr_sum_weighted -- FP64 totals sum_e sum_rho w_rho J_rho u_{rho,alpha,n}
 * (solution-point quadrature of each variable: the conserved totals of
 * Eq. commpflux's conservation argument), written to host out[nvars].
 * Synchronises `stream`.
 */
fr_status fr_sum_weighted(fr_ctx* ctx, void* const* u, double* out, void* stream);

/*
 * fr_rk4_noalloc -- the same RK4 step as fr_rk4 (end of Sec. 2), for callers that cannot let
 * a library allocate device memory at call time.  The paper has no
 * counterpart; it exists for applications whose framework owns all device
 * memory through its own pool (a cudaMalloc behind its back fails or
 * fragments that pool) and for time-critical loops in which cudaMalloc /
 * cudaFree, which may synchronise the device, must not run.  fr_rk4 allocates
 * its two stage registers with cudaMalloc on its first call; this entry point
 * keeps them instead in a fixed device array compiled into libfr.so, of
 * FR_NOALLOC_MAX_BYTES (64 MiB), which every GPU that loads the library holds
 * until the process exits.  The call itself allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine.
 *   - Limit: the registers need 2 * nupts * nvars * ld * sizeof(real) bytes
 *     per block (each rounded up to 256); larger meshes are rejected with
 *     FR_ERR_ARG and a message naming both sizes, before anything runs.
 *   - Set-up: fr_setup looks up the array's device address on the context's
 *     device (cudaGetSymbolAddress, with that device current).  That look-up
 *     loads the part of the library that holds the array and so reserves its
 *     FR_NOALLOC_MAX_BYTES there: set up the context before the caller's pool
 *     takes the GPU's memory.  Should that look-up have failed, the first call
 *     repeats it and reports the failure (FR_ERR_CUDA); such a first call
 *     must not run inside a stream capture.
 *   - Sharing: every call, from any context or stream, uses the same array,
 *     which keeps the last call's contents (nothing needs clearing: each call
 *     writes every byte it reads).  Calls that overlap on the GPU race on it:
 *     serialise them.
 *   - Kernel timing (fr_profile_enable) is suspended during the call, since
 *     its CUDA events may allocate; the call's kernels are not timed.
 * u, dt, nsteps and stream as for fr_rk4; at most 16 element blocks.
 */
#define FR_NOALLOC_MAX_BYTES (64u * 1024u * 1024u)
fr_status fr_rk4_noalloc(fr_ctx* ctx, void* const* u, double dt, int nsteps, void* stream);

/* Reads and clears the device error flags (non-finite values seen by
 * fr_check_finite, timeouts); not in the paper.  Synchronises the device. */
fr_status fr_sync_status(fr_ctx* ctx);

/* Scans u for NaN/Inf on the device (not in the paper); the result is
 * reported by the next fr_sync_status() as FR_ERR_NONFINITE.  Stream-ordered. */
fr_status fr_check_finite(fr_ctx* ctx, void* const* u, void* stream);

/*
 * Kernel-level timing (not in the paper; its kernel names follow the kernel
 * flow of Sec. 3.6 / App. A).  fr_profile_enable(ctx, 1) makes every later kernel
 * launch of fr_rhs / fr_rk4 record a CUDA event pair on its launch stream.
 * fr_profile_read synchronises on those events and returns, per kernel, the
 * number of launches and the total event-measured milliseconds since the
 * previous read, then clears them.  names receives nkernels NUL-terminated
 * names of at most 31 characters in rows of 32 bytes.  *nkernels is always
 * set; with all three arrays NULL the call only reports the count and keeps
 * the records.
 */
fr_status fr_profile_enable(fr_ctx* ctx, int enable);
fr_status fr_profile_read(fr_ctx* ctx, int32_t* nkernels, char* names, int64_t* launches, double* ms);

/* Message for the last failure on ctx (ctx == NULL: last fr_setup failure);
 * not in the paper. */
const char* fr_last_error(const fr_ctx* ctx);

/* Frees everything the context owns (not in the paper).  Synchronises its device. */
void fr_destroy(fr_ctx* ctx);

/*
 * Measured FMA throughput (not in the paper; the paper's Sec. 6 rates its
 * kernels against the device peaks) of the CUDA cores of device cuda_device, in TFLOP/s
 * (2 flop per FMA): eight independent FP32 (resp. FP64) FMA chains per thread
 * over 8 blocks of 256 threads per SM, best of three timed launches.  Used as
 * the ALU roofline of the plain FP32 and FP64 paths.  Synchronous; sets the
 * calling thread's current device.  FR_ERR_ARG for NULL outputs, FR_ERR_CUDA
 * on any CUDA failure.
 */
fr_status fr_fma_peak(int cuda_device, double* fp32_tflops, double* fp64_tflops);

/*
 * Partitioned right-hand side (Sec. 3.6: the element set split between ranks,
 * with "int" kernels on pairs inside a partition and "mpi" kernels on pairs
 * whose other side lives on another rank, fed by an exchange of the
 * flux-point values of those pairs).
 *
 * fr_setup_part builds the context of partition `rank` of the mesh: part has
 * one entry per element, block-major (all elements of block 0, then block 1,
 * ...), with values in [0, nparts); the context holds the elements of its
 * rank (in increasing global order within each block; every block must keep
 * at least one element, else FR_ERR_ARG), the pairs and boundary faces among
 * them, and for every neighbour rank the pairs shared with it, in exchange
 * slots: first the pairs whose global L side (the same L as in fr_setup)
 * lies on the lower of the two ranks, then the others, each sorted by that
 * side's (block, element, flux point).  Both ranks derive the same slots from
 * the global pairing, so either side evaluates a shared pair with the same
 * arguments as the unpartitioned right-hand side.  Same errors as fr_setup.
 * A partitioned context serves fr_rhs_parts, fr_layout, fr_solution_points,
 * fr_operator, fr_pairs (its own pairs), fr_sum_weighted, fr_check_finite;
 * fr_rhs and the steppers return FR_ERR_UNSUPPORTED for it.
 */
fr_status fr_setup_part(const fr_mesh* mesh, const fr_params* prm, int cuda_device, const int32_t* part,
                        int32_t nparts, int32_t rank, fr_ctx** out);

/*
 * Exchange slots of a partitioned context (Sec. 3.6 "mpi" interfaces): *nnbr neighbour ranks (ascending)
 * in ranks[], their slot counts in nslots[], and for every slot, neighbour by
 * neighbour, the global L side (block, element, flux point) as 3 int64 in
 * keys[].  Arrays may be NULL (sizes only).  Host-only contexts work too.
 */
fr_status fr_part_slots(const fr_ctx* ctx, int32_t* nnbr, int32_t* ranks, int64_t* nslots, int64_t* keys);

/*
 * One right-hand side of every partition (Sec. 3.6: the kernel flow split
 * into interior ("int") and partition ("mpi") interfaces), all on the calling device:
 * parts[p] is the context of rank p, u[p] / r[p] its per-block state and
 * result pointers (layout of fr_layout on parts[p]).  Per partition and stage:
 * interpolation and packing of the shared flux-point values; exchange of the
 * packed values (device-to-device copies on a library stream, ordered after
 * the packing by events) while the interior-pair kernels run; then the
 * shared-pair kernels.  Navier-Stokes exchanges U^(f) and, after the gradient
 * stage, Q^(f).  Results equal those of fr_rhs on the whole mesh (bit for bit
 * in FP64 and FP32 arithmetic: every pair is evaluated with the same inputs).
 * Stream-ordered on `stream`.  FR_ERR_ARG for missing or mismatched contexts.
 */
fr_status fr_rhs_parts(fr_ctx* const* parts, int32_t nparts, void* const* const* u, void* const* const* r,
                       void* stream);

/* ABI version (increments on any signature change); not in the paper. */
int32_t fr_version(void);   /* 6 */

#ifdef __cplusplus
}
#endif

#endif /* FR_H */
